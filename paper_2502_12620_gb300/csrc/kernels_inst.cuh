// Explicit kernel instantiations for one (dimension, precision); included by
// the small k_<dim>_<prec>.cu translation units so they compile in parallel.
#pragma once

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "dg_device.cuh"
#include "launch.hpp"

namespace dgf {

template <int N, typename Real>
static Tab<N, Real> make_tab(const RtTables& r) {
  Tab<N, Real> t;
  for (int i = 0; i < N; ++i) {
    t.x[i] = (Real)r.x[i];
    t.w[i] = (Real)r.w[i];
    t.lp[i] = (Real)r.lp[i];
    t.lm[i] = (Real)r.lm[i];
    t.lpw[i] = (Real)(r.lp[i] / r.w[i]);
    t.lmw[i] = (Real)(r.lm[i] / r.w[i]);
    for (int j = 0; j < N; ++j) {
      t.V[i][j] = (Real)r.V[i * N + j];
      t.Vi[i][j] = (Real)r.Vi[i * N + j];
      t.Sh[i][j] = (Real)r.Sh[i * N + j];
      t.Sm[i][j] = (Real)r.Sm[i * N + j];
      t.Sp[i][j] = (Real)r.Sp[i * N + j];
      t.Snm[i][j] = (Real)r.Snm[i * N + j];
      t.Snp[i][j] = (Real)r.Snp[i * N + j];
    }
  }
  return t;
}

// The mortar variants of the stage kernel (faces whose flux the mortar passes
// give) live in their own translation units (k_<dim>_<prec>_mortar.cu).
template <int D, int P, int NS, typename Real>
cudaError_t stage_mortar_launch(const StageArgs<D, P, Real>& a, int grid, size_t smem, int comp, cudaStream_t s);
template <int D, int P, int NS, typename Real>
bool stage_mortar_prepare(size_t smem);

#define DGF_INSTANTIATE_MORTAR_NS(DIM, P, NS, REAL)                                                   \
  template <>                                                                                         \
  cudaError_t stage_mortar_launch<DIM, P, NS, REAL>(const StageArgs<DIM, P, REAL>& a, int grid,       \
                                                    size_t smem, int comp, cudaStream_t s) {          \
    if constexpr (std::is_same<REAL, float>::value) {                                                 \
      if (comp) {                                                                                     \
        k_stage<DIM, P, NS, REAL, true, true><<<grid, StageCfg<P, REAL>::NT, smem, s>>>(a);           \
        return cudaGetLastError();                                                                    \
      }                                                                                               \
    }                                                                                                 \
    if (comp) return cudaErrorInvalidValue;                                                           \
    k_stage<DIM, P, NS, REAL, false, true><<<grid, StageCfg<P, REAL>::NT, smem, s>>>(a);              \
    return cudaGetLastError();                                                                        \
  }                                                                                                   \
  template <>                                                                                         \
  bool stage_mortar_prepare<DIM, P, NS, REAL>(size_t smem) {                                          \
    if (cudaFuncSetAttribute(k_stage<DIM, P, NS, REAL, false, true>,                                  \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)  \
      return false;                                                                                   \
    if constexpr (std::is_same<REAL, float>::value) {                                                 \
      if (cudaFuncSetAttribute(k_stage<DIM, P, NS, REAL, true, true>,                                 \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) \
        return false;                                                                                 \
    }                                                                                                 \
    return true;                                                                                      \
  }
#define DGF_INSTANTIATE_MORTAR_P(DIM, P, REAL) \
  DGF_INSTANTIATE_MORTAR_NS(DIM, P, 2, REAL)   \
  DGF_INSTANTIATE_MORTAR_NS(DIM, P, 4, REAL)   \
  DGF_INSTANTIATE_MORTAR_NS(DIM, P, 8, REAL)
#define DGF_INSTANTIATE_MORTAR(DIM, REAL) \
  DGF_INSTANTIATE_MORTAR_P(DIM, 0, REAL)  \
  DGF_INSTANTIATE_MORTAR_P(DIM, 1, REAL)  \
  DGF_INSTANTIATE_MORTAR_P(DIM, 2, REAL)  \
  DGF_INSTANTIATE_MORTAR_P(DIM, 3, REAL)

// The cell-pair FP32 stage kernel (stage_pair.cuh) serves 3D forests of 8^3-cell
// blocks at p = 1, 2 in plain FP32 (RtStage::kernel 0); k_stage serves the rest.
template <int D, int P, int NS, typename Real>
constexpr bool pair_shape() {
  return D == 3 && NS == 8 && (P == 1 || P == 2) && std::is_same<Real, float>::value;
}
// launch and occupancy of the cell-pair kernel (k_3d_f32_pair<P>.cu); v
// selects its CTA shape (p = 1: 0 four CTAs per SM, 1 five)
template <int P>
cudaError_t stage_pair_launch(const StageArgs<3, P, float>& a, int grid, bool mortar, bool all_affine,
                              cudaStream_t s, int v);
template <int P>
int stage_pair_blocks_per_sm(int v);
template <int P>
cudaError_t stage_pair_launch_batch(const StageArgs<3, P, float>& a, int grid, bool all_affine, cudaStream_t s);

template <int D, int P, int NS, typename Real>
static int stage_blocks_per_sm_classic();

template <int D, int P, int NS, typename Real>
static int stage_blocks_per_sm_ns(int comp, int kernel) {
  if constexpr (pair_shape<D, P, NS, Real>()) {
    // kernel 2 (the five-CTA shape) exists at p = 1 only
    if (!comp && (kernel == 0 || (kernel == 2 && P == 1))) {
      const int nb = stage_pair_blocks_per_sm<P>(kernel == 2);
      if (nb > 0) return nb;
    }
    if (kernel == 2) return 0;
  }
  return stage_blocks_per_sm_classic<D, P, NS, Real>();
}

template <int D, int P, int NS, typename Real>
static int stage_blocks_per_sm_classic() {
  const size_t smem = stage_smem<D, P, Real>(NS, stage_rows<D, P, Real>(NS));
  int dev = 0, maxs = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem + 1024 > (size_t)maxs) return 0;
  if (cudaFuncSetAttribute(k_stage<D, P, NS, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  if constexpr (std::is_same<Real, float>::value) {
    if (cudaFuncSetAttribute(k_stage<D, P, NS, Real, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return 0;
  }
  if (!stage_mortar_prepare<D, P, NS, Real>(smem)) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage<D, P, NS, Real>, StageCfg<P, Real>::NT, smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

template <int D, int P, typename Real>
static int stage_blocks_per_sm(int n, int comp, int kernel) {
  switch (n) {
    case 2: return stage_blocks_per_sm_ns<D, P, 2, Real>(comp, kernel);
    case 4: return stage_blocks_per_sm_ns<D, P, 4, Real>(comp, kernel);
    case 8: return stage_blocks_per_sm_ns<D, P, 8, Real>(comp, kernel);
  }
  return 0;  // n_seg other than 2, 4, 8 is not instantiated
}

template <int D, int P, int NS, typename Real>
static cudaError_t stage_ns(const StageArgs<D, P, Real>& a, int slots, int comp, int all_affine, int kernel,
                            cudaStream_t s) {
  const size_t smem = stage_smem<D, P, Real>(NS, stage_rows<D, P, Real>(NS));
  const int items = a.nL * a.nchunks * (NS / stage_rows<D, P, Real>(NS));
  const int grid = items < slots ? items : slots;
  if constexpr (pair_shape<D, P, NS, Real>()) {
    if (!comp && (kernel == 0 || kernel == 2)) {
      const int g = a.nL * a.nchunks < slots ? a.nL * a.nchunks : slots;
      if constexpr (P == 1 || P == 2)
        return stage_pair_launch<P>(a, g, a.fluxmask != nullptr, all_affine != 0, s, kernel == 2 ? 1 : 0);
    }
  }
  if (a.fluxmask) return stage_mortar_launch<D, P, NS, Real>(a, grid, smem, comp, s);
  if constexpr (std::is_same<Real, float>::value) {
    if (comp) {
      k_stage<D, P, NS, Real, true><<<grid, StageCfg<P, Real>::NT, smem, s>>>(a);
      return cudaGetLastError();
    }
  }
  if (comp) return cudaErrorInvalidValue;
  k_stage<D, P, NS, Real><<<grid, StageCfg<P, Real>::NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int D, int P, typename Real>
static StageArgs<D, P, Real> make_stage_args(const RtStage& r) {
  StageArgs<D, P, Real> a;
  a.nL = r.nL;
  a.n = r.n;
  a.zchunk = r.zchunk;
  a.nchunks = D == 3 ? (r.n + r.zchunk - 1) / r.zchunk : 1;
  a.U = (const Real*)r.U;
  a.Un = (const Real*)r.Un;
  a.Uout = (Real*)r.Uout;
  a.geo = (const Real*)r.geo;
  a.gtr = (const Real*)r.gtr;
  a.hcell = (const Real*)r.hcell;
  a.affine = r.affine;
  a.ameta = (const Real*)r.ameta;
  a.kind = r.kind;
  a.nbr = r.nbr;
  a.orient = r.orient;
  a.qbits = r.qbits;
  a.dtp = r.dtp;
  a.lam_bits = r.lam_bits;
  a.status = r.status;
  a.ca = (Real)r.ca;
  a.cb = (Real)r.cb;
  a.gamma = (Real)r.gamma;
  a.mode = r.mode;
  a.last = r.last;
  a.U64 = r.U64;
  a.Uhi = r.Uhi;
  a.Ulo = r.Ulo;
  a.Din = r.Din;
  a.U64out = r.U64out;
  a.fluxmask = r.fluxmask;
  a.T = make_tab<P + 1, Real>(r.T);
  a.members = nullptr;
  a.istart = nullptr;
  a.nmem = 0;
  return a;
}

template <int D, int P, typename Real>
static cudaError_t stage_p(const RtStage& r, cudaStream_t s) {
  const StageArgs<D, P, Real> a = make_stage_args<D, P, Real>(r);
  if (r.slots <= 0) return cudaErrorInvalidConfiguration;
  switch (r.n) {
    case 2: return stage_ns<D, P, 2, Real>(a, r.slots, r.comp, r.all_affine, r.kernel, s);
    case 4: return stage_ns<D, P, 4, Real>(a, r.slots, r.comp, r.all_affine, r.kernel, s);
    case 8: return stage_ns<D, P, 8, Real>(a, r.slots, r.comp, r.all_affine, r.kernel, s);
  }
  return cudaErrorInvalidConfiguration;
}

template <int D, int P, typename Real>
static GuardArgs<D, P, Real> make_guard_args(const RtGuard& r) {
  GuardArgs<D, P, Real> a;
  a.nL = r.nL;
  a.n = r.n;
  a.mode = r.mode;
  a.U = (const Real*)r.U;
  a.U64 = r.U64;
  a.Uhi = r.Uhi;
  a.Ulo = r.Ulo;
  a.Din = r.Din;
  a.out = (Real*)r.out;
  a.kind = r.kind;
  a.nbr = r.nbr;
  a.orient = r.orient;
  a.qbits = r.qbits;
  a.copoff = r.copoff;
  a.cop = (const Real*)r.cop;
  a.ctr = (const Real*)r.ctr;
  a.fine_list = r.fine_list;
  a.nfine = r.nfine;
  a.trd = r.trd;
  a.geo = (const Real*)r.geo;
  a.gamma = (Real)r.gamma;
  a.mfine = r.mfine;
  a.nmf = r.nmf;
  a.mcoarse = r.mcoarse;
  a.nmc = r.nmc;
  a.mw = (const Real*)r.mw;
  a.msrc = r.msrc;
  a.bstate = (const Real*)r.bstate;
  a.T = make_tab<P + 1, Real>(r.T);
  return a;
}

template <int D, int P, typename Real>
static cudaError_t guard_p(const RtGuard& r, cudaStream_t s) {
  const GuardArgs<D, P, Real> a = make_guard_args<D, P, Real>(r);
  const int nt = D == 3 ? r.n * r.n : r.n;
  if (r.mode == 1) {
    // time-step path: traces of every face kind in one launch (finer faces
    // by the combine blocks unless the mortar passes replace them)
    constexpr int NTH = 32 << D;
    const size_t items = (size_t)r.nL * 2 * D * (D + 2) * nt;
    if (items >= ((size_t)1 << 32)) return cudaErrorInvalidConfiguration;  // the kernel indexes in 32 bits
    const size_t ntb = (items + NTH - 1) / NTH;
    const int nfb = r.nfine * nt;
    const bool comp = std::is_same<Real, float>::value && r.comp;
    if constexpr (std::is_same<Real, float>::value) {
      if (comp) k_guard_trace<D, P, Real, true><<<(unsigned)(ntb + nfb), NTH, 0, s>>>(a, nfb);
    }
    if (!comp) k_guard_trace<D, P, Real><<<(unsigned)(ntb + nfb), NTH, 0, s>>>(a, nfb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    constexpr int NFP = ipow(P + 1, D - 1);
    if (r.nmf > 0) {
      const size_t tot = (size_t)r.nmf * nt * NFP;
      if constexpr (std::is_same<Real, float>::value) {
        if (comp) k_mortar_fine<D, P, Real, true><<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(a);
      }
      if (!comp) k_mortar_fine<D, P, Real><<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(a);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (r.nmc > 0) {
      const size_t tot = (size_t)r.nmc * nt * (D + 2) * NFP;
      k_mortar_coarse<D, P, Real><<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(a);
      e = cudaGetLastError();
    }
    return e;
  }
  const size_t total = (size_t)r.nL * 2 * D * nt * (D + 2);
  const int th = 128;
  const size_t ctas = (size_t)r.nfine * nt * (D + 2);
  if constexpr (std::is_same<Real, float>::value) {
    if (r.comp) {
      k_guard<D, P, Real, true><<<(unsigned)((total + th - 1) / th), th, 0, s>>>(a);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess || r.nfine == 0) return e;
      k_guard_fine<D, P, Real, true><<<(unsigned)ctas, 32 << D, 0, s>>>(a);
      return cudaGetLastError();
    }
  }
  k_guard<D, P, Real><<<(unsigned)((total + th - 1) / th), th, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || r.nfine == 0) return e;
  k_guard_fine<D, P, Real><<<(unsigned)ctas, 32 << D, 0, s>>>(a);
  return cudaGetLastError();
}

template <int D, int P, typename Real>
static cudaError_t cfl_p(const RtMisc& r, cudaStream_t s) {
  const int nc = D == 3 ? r.n * r.n * r.n : r.n * r.n;
  const size_t total = (size_t)r.nL * nc * ipow(P + 1, D);
  const int th = 256;
  k_cfl<D, P, Real><<<(unsigned)((total + th - 1) / th), th, 0, s>>>(
      r.nL, r.n, (const Real*)r.U, (const Real*)r.hcell, (Real)r.gamma, r.lam_bits, r.status);
  return cudaGetLastError();
}

template <int D, int P, typename Real>
static cudaError_t project_p(const RtMisc& r, cudaStream_t s) {
  const int nc = D == 3 ? r.n * r.n * r.n : r.n * r.n;
  const size_t total = (size_t)r.nL * nc * ipow(P + 1, D) * (D + 2);
  const int th = 256;
  k_project<D, P, Real><<<(unsigned)((total + th - 1) / th), th, 0, s>>>(r.nL, r.n, r.vals, (Real*)r.Uout);
  return cudaGetLastError();
}

template <int D, int P, typename Real>
static cudaError_t totals_p(const RtMisc& r, cudaStream_t s) {
  const int nc = D == 3 ? r.n * r.n * r.n : r.n * r.n;
  const size_t total = (size_t)r.nL * nc;
  const int th = 128;
  k_totals<D, P, Real><<<(unsigned)((total + th - 1) / th), th, 0, s>>>(
      r.nL, r.n, (const Real*)r.U, r.geo64, r.part, make_tab<P + 1, double>(r.T));
  return cudaGetLastError();
}

template <int D, int P, typename Real>
static cudaError_t indicator_p(const RtMisc& r, cudaStream_t s) {
  const int nc = D == 3 ? r.n * r.n * r.n : r.n * r.n;
  const size_t total = (size_t)r.nL * nc;
  const int th = 128;
  if (total == 0) return cudaSuccess;
  k_indicator<D, P, Real><<<(unsigned)((total + th - 1) / th), th, 0, s>>>(
      r.nL, r.n, (const Real*)r.U, r.gmax, make_tab<P + 1, Real>(r.T));
  return cudaGetLastError();
}

template <int D, int P, typename Real>
static cudaError_t limit_p(const RtMisc& r, cudaStream_t s) {
  const int nc = D == 3 ? r.n * r.n * r.n : r.n * r.n;
  const size_t total = (size_t)r.nL * nc;
  const int th = 128;
  if (total == 0) return cudaSuccess;
  k_limit<D, P, Real><<<(unsigned)((total + th - 1) / th), th, 0, s>>>(
      r.nL, r.n, (Real*)r.Uout, (const Real*)r.geo, r.affine, (Real)r.gamma, (Real)r.eps, r.status,
      make_tab<P + 1, Real>(r.T));
  return cudaGetLastError();
}

template <int D, int P, typename Real>
static cudaError_t transfer_p(const RtTransfer& r, cudaStream_t s) {
  const int nc = D == 3 ? r.n * r.n * r.n : r.n * r.n;
  const size_t total = (size_t)r.nL * (D + 2) * nc;
  const int th = 128;
  if (total == 0) return cudaSuccess;
  k_transfer<D, P, Real><<<(unsigned)((total + th - 1) / th), th, 0, s>>>(
      r.nL, r.n, (const Real*)r.old, (Real*)r.out, r.mode, r.src, r.kids, r.opoff, r.cellop, (const Real*)r.ops,
      make_tab<P + 1, Real>(r.T));
  return cudaGetLastError();
}

template <int D, int P, typename Real>
static cudaError_t convert_p(size_t outer, int inner, void* X, int to_nodal, const RtTables& T, cudaStream_t s) {
  const size_t total = outer * (D + 2) * inner;
  const int th = 128;
  k_convert<D, P, Real><<<(unsigned)((total + th - 1) / th), th, 0, s>>>(outer, inner, (Real*)X, to_nodal,
                                                                       make_tab<P + 1, Real>(T));
  return cudaGetLastError();
}


// ---------------------------------------------------------------- batches
// Every forest of a batch (same dimension 3, n_seg 8, degree, FP32, plain
// form without the mortar repair) in one launch per kernel: the per-forest
// kernel arguments are packed on the host into device arrays; the kernels
// find an item's (block's) forest from prefix sums.

// work items of one forest's stage launch with the kernel r.kernel
template <int D, int P, typename Real>
static int stage_items_p(const RtStage& r) {
  const int nchunks = D == 3 ? (r.n + r.zchunk - 1) / r.zchunk : 1;
  if (r.n != 8) return -1;
  return r.nL * nchunks * (8 / stage_rows<D, P, Real>(8));  // the same count for both kernels at n = 8
}

template <int D, int P, typename Real>
static size_t stage_args_pack_p(const RtStage* r, int n, void* host) {
  if (host)
    for (int i = 0; i < n; ++i) reinterpret_cast<StageArgs<D, P, Real>*>(host)[i] = make_stage_args<D, P, Real>(r[i]);
  return sizeof(StageArgs<D, P, Real>) * (size_t)n;
}

template <int D, int P, typename Real>
static size_t guard_args_pack_p(const RtGuard* r, int n, void* host) {
  if (host)
    for (int i = 0; i < n; ++i) reinterpret_cast<GuardArgs<D, P, Real>*>(host)[i] = make_guard_args<D, P, Real>(r[i]);
  return sizeof(GuardArgs<D, P, Real>) * (size_t)n;
}

// blocks of one forest's guard-trace launch (trace blocks + finer-face blocks)
template <int D, int P, typename Real>
static long long guard_blocks_p(const RtGuard& r, int* nfb) {
  constexpr int NTH = 32 << D;
  const int nt = D == 3 ? r.n * r.n : r.n;
  const size_t items = (size_t)r.nL * 2 * D * (D + 2) * nt;
  *nfb = r.nfine * nt;
  return (long long)((items + NTH - 1) / NTH) + *nfb;
}

template <int D, int P, typename Real>
static int stage_batch_blocks_per_sm_p(int kernel, int all_affine) {
  if constexpr (D == 3 && std::is_same<Real, float>::value) {
    if constexpr (P == 1 || P == 2) {
      if (kernel == 0) return stage_pair_blocks_per_sm<P>(0);
    }
    constexpr int YS = stage_rows<D, P, Real>(8);
    const size_t smem = stage_smem<D, P, Real>(8, YS);
    if (cudaFuncSetAttribute(k_stage<D, P, 8, Real, false, false, YS, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage<D, P, 8, Real, false, false, YS, true>,
                                                      StageCfg<P, Real>::NT, smem) != cudaSuccess)
      return 0;
    (void)all_affine;
    return nb;
  }
  return 0;
}

template <int D, int P, typename Real>
static cudaError_t launch_stage_batch_p(const RtStage& common, const void* members, const int* istart, int nmem,
                                        int grid, cudaStream_t s) {
  if constexpr (D == 3 && std::is_same<Real, float>::value) {
    StageArgs<D, P, Real> a = make_stage_args<D, P, Real>(common);
    a.members = reinterpret_cast<const StageArgs<D, P, Real>*>(members);
    a.istart = istart;
    a.nmem = nmem;
    if constexpr (P == 1 || P == 2) {
      if (common.kernel == 0) return stage_pair_launch_batch<P>(a, grid, common.all_affine != 0, s);
    }
    constexpr int YS = stage_rows<D, P, Real>(8);
    const size_t smem = stage_smem<D, P, Real>(8, YS);
    k_stage<D, P, 8, Real, false, false, YS, true><<<grid, StageCfg<P, Real>::NT, smem, s>>>(a);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

template <int D, int P, typename Real>
static cudaError_t launch_guard_batch_p(const void* members, const int* bstart, const int* nfb, int nmem,
                                        long long blocks, cudaStream_t s) {
  if constexpr (D == 3 && std::is_same<Real, float>::value) {
    if (blocks <= 0 || blocks >= (1ll << 31)) return cudaErrorInvalidConfiguration;
    k_guard_trace_batch<D, P, Real><<<(unsigned)blocks, 32 << D, 0, s>>>(
        reinterpret_cast<const GuardArgs<D, P, Real>*>(members), bstart, nfb, nmem);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

#define DGF_DISPATCH_P(fn, r, s)                 \
  switch ((r).p) {                               \
    case 0: return fn<D, 0, Real>(r, s);         \
    case 1: return fn<D, 1, Real>(r, s);         \
    case 2: return fn<D, 2, Real>(r, s);         \
    case 3: return fn<D, 3, Real>(r, s);         \
    default: return cudaErrorInvalidValue;       \
  }

#define DGF_SWITCH_P(p, expr_tmpl)                                                          \
  switch (p) {                                                                              \
    case 0: { constexpr int P_ = 0; return expr_tmpl; }                                     \
    case 1: { constexpr int P_ = 1; return expr_tmpl; }                                     \
    case 2: { constexpr int P_ = 2; return expr_tmpl; }                                     \
    case 3: { constexpr int P_ = 3; return expr_tmpl; }                                     \
  }

#define DGF_INSTANTIATE(DIM, REAL)                                                          \
  template <>                                                                               \
  int stage_items<DIM, REAL>(const RtStage& r) {                                            \
    DGF_SWITCH_P(r.p, (stage_items_p<DIM, P_, REAL>(r)))                                    \
    return -1;                                                                              \
  }                                                                                         \
  template <>                                                                               \
  size_t stage_args_pack<DIM, REAL>(const RtStage* r, int n, void* host) {                  \
    DGF_SWITCH_P(r[0].p, (stage_args_pack_p<DIM, P_, REAL>(r, n, host)))                    \
    return 0;                                                                               \
  }                                                                                         \
  template <>                                                                               \
  size_t guard_args_pack<DIM, REAL>(const RtGuard* r, int n, void* host) {                  \
    DGF_SWITCH_P(r[0].p, (guard_args_pack_p<DIM, P_, REAL>(r, n, host)))                    \
    return 0;                                                                               \
  }                                                                                         \
  template <>                                                                               \
  long long guard_blocks<DIM, REAL>(const RtGuard& r, int* nfb) {                           \
    DGF_SWITCH_P(r.p, (guard_blocks_p<DIM, P_, REAL>(r, nfb)))                              \
    return -1;                                                                              \
  }                                                                                         \
  template <>                                                                               \
  int stage_batch_blocks_per_sm<DIM, REAL>(int p, int kernel, int all_affine) {             \
    DGF_SWITCH_P(p, (stage_batch_blocks_per_sm_p<DIM, P_, REAL>(kernel, all_affine)))       \
    return 0;                                                                               \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_stage_batch<DIM, REAL>(const RtStage& c, const void* m, const int* istart, int nmem,  \
                                            int grid, cudaStream_t s) {                     \
    DGF_SWITCH_P(c.p, (launch_stage_batch_p<DIM, P_, REAL>(c, m, istart, nmem, grid, s)))   \
    return cudaErrorInvalidValue;                                                           \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_guard_batch<DIM, REAL>(int p, const void* m, const int* bstart, const int* nfb,     \
                                            int nmem, long long blocks, cudaStream_t s) {   \
    DGF_SWITCH_P(p, (launch_guard_batch_p<DIM, P_, REAL>(m, bstart, nfb, nmem, blocks, s))) \
    return cudaErrorInvalidValue;                                                           \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_stage<DIM, REAL>(const RtStage& r, cudaStream_t s) {                   \
    constexpr int D = DIM;                                                                  \
    using Real = REAL;                                                                      \
    DGF_DISPATCH_P(stage_p, r, s)                                                           \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_guard<DIM, REAL>(const RtGuard& r, cudaStream_t s) {                   \
    constexpr int D = DIM;                                                                  \
    using Real = REAL;                                                                      \
    DGF_DISPATCH_P(guard_p, r, s)                                                           \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_cfl<DIM, REAL>(const RtMisc& r, cudaStream_t s) {                      \
    constexpr int D = DIM;                                                                  \
    using Real = REAL;                                                                      \
    DGF_DISPATCH_P(cfl_p, r, s)                                                             \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_project<DIM, REAL>(const RtMisc& r, cudaStream_t s) {                  \
    constexpr int D = DIM;                                                                  \
    using Real = REAL;                                                                      \
    DGF_DISPATCH_P(project_p, r, s)                                                         \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_totals<DIM, REAL>(const RtMisc& r, cudaStream_t s) {                   \
    constexpr int D = DIM;                                                                  \
    using Real = REAL;                                                                      \
    DGF_DISPATCH_P(totals_p, r, s)                                                          \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_indicator<DIM, REAL>(const RtMisc& r, cudaStream_t s) {                \
    constexpr int D = DIM;                                                                  \
    using Real = REAL;                                                                      \
    DGF_DISPATCH_P(indicator_p, r, s)                                                       \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_limit<DIM, REAL>(const RtMisc& r, cudaStream_t s) {                    \
    constexpr int D = DIM;                                                                  \
    using Real = REAL;                                                                      \
    DGF_DISPATCH_P(limit_p, r, s)                                                           \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_transfer<DIM, REAL>(const RtTransfer& r, cudaStream_t s) {             \
    constexpr int D = DIM;                                                                  \
    using Real = REAL;                                                                      \
    DGF_DISPATCH_P(transfer_p, r, s)                                                        \
  }                                                                                         \
  template <>                                                                               \
  cudaError_t launch_convert<DIM, REAL>(int p, size_t outer, int inner, void* X, int to_nodal, \
                                        const RtTables& T, cudaStream_t s) {                \
    switch (p) {                                                                            \
      case 0: return convert_p<DIM, 0, REAL>(outer, inner, X, to_nodal, T, s);              \
      case 1: return convert_p<DIM, 1, REAL>(outer, inner, X, to_nodal, T, s);              \
      case 2: return convert_p<DIM, 2, REAL>(outer, inner, X, to_nodal, T, s);              \
      case 3: return convert_p<DIM, 3, REAL>(outer, inner, X, to_nodal, T, s);              \
    }                                                                                       \
    return cudaErrorInvalidValue;                                                           \
  }                                                                                         \
  template <>                                                                               \
  int stage_occupancy<DIM, REAL>(int p, int n, int comp, int kernel) {                      \
    switch (p) {                                                                            \
      case 0: return stage_blocks_per_sm<DIM, 0, REAL>(n, comp, kernel);                    \
      case 1: return stage_blocks_per_sm<DIM, 1, REAL>(n, comp, kernel);                    \
      case 2: return stage_blocks_per_sm<DIM, 2, REAL>(n, comp, kernel);                    \
      case 3: return stage_blocks_per_sm<DIM, 3, REAL>(n, comp, kernel);                    \
    }                                                                                       \
    return 0;                                                                               \
  }                                                                                         \
  template <>                                                                               \
  size_t stage_smem_bytes<DIM, REAL>(int p, int n) {                                        \
    switch (p) {                                                                            \
      case 0: return stage_smem<DIM, 0, REAL>(n, stage_rows<DIM, 0, REAL>(n));                                           \
      case 1: return stage_smem<DIM, 1, REAL>(n, stage_rows<DIM, 1, REAL>(n));                                           \
      case 2: return stage_smem<DIM, 2, REAL>(n, stage_rows<DIM, 2, REAL>(n));                                           \
      case 3: return stage_smem<DIM, 3, REAL>(n, stage_rows<DIM, 3, REAL>(n));                                           \
    }                                                                                       \
    return 0;                                                                               \
  }

}  // namespace dgf
