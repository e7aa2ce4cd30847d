// C ABI of the block-forest DG library (declared in include/dgf.h).
//
// This layer owns the forest (host topology + device buffers), precomputes
// the FP64 geometry (trilinear coefficients per cell, cell sizes) and the
// FP64 combine operators of Sec. 3.4 for every finer-neighbour guard cell,
// and enqueues the kernels of one SSP-RK3 time increment (Sec. 4.3):
//   k_dt -> 3 x { k_guard (guard traces, Sec. 3.5) ; k_stage (residual +
//   inverse mass + stage combination, CFL minimum on the last stage) },
// captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dgf.h"
#include "forest_host.hpp"
#include "launch.hpp"

using namespace dgf;

namespace {

thread_local std::string g_err;

dgf_status fail(dgf_status code, const std::string& msg) {
  g_err = msg;
  return code;
}

struct DevScalars {
  double t, dt, t_end;
  unsigned long long lam_bits;  // min over cells of h / lambda, as double bits
  int status;
  int steps;  // time increments taken with dt > 0 since creation / dgf_set_time
};

constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

__device__ __forceinline__ void dt_one(DevScalars* s, double cfl) {
  const unsigned long long lb = s->lam_bits;
  double dt = 0.0;
  if (lb != kInfBits) {
    dt = cfl * __longlong_as_double((long long)lb);
    const double rem = s->t_end - s->t;
    if (dt > rem) dt = rem;
    if (!(dt > 0.0)) dt = 0.0;
  } else {
    s->status = -4;
  }
  s->dt = dt;
  s->t = s->t + dt;
  s->steps += dt > 0.0;
  // a zero increment evaluates no stage, so the CFL minimum is kept for the next
  if (dt > 0.0) s->lam_bits = kInfBits;
}

__global__ void k_dt(DevScalars* s, double cfl) { dt_one(s, cfl); }

// time, step count and status word of every forest of a batch
__global__ void k_batch_progress(DevScalars* const* __restrict__ s, int n, double* t, long long* steps, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    t[i] = s[i]->t;
    steps[i] = s[i]->steps;
    status[i] = s[i]->status;
  }
}

// the time increments of every forest of a batch (one thread each)
__global__ void k_dt_batch(DevScalars* const* __restrict__ s, const double* __restrict__ cfl, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dt_one(s[i], cfl[i]);
}

__global__ void k_reset_lam(DevScalars* s) { s->lam_bits = kInfBits; }

__global__ void k_set_t_end(DevScalars* s, double t_end) { s->t_end = t_end; }

__global__ void k_set_time(DevScalars* s, double t) {
  s->t = t;
  s->steps = 0;
}

// t = 0, no step taken, no end time, no CFL value yet, status 0
__global__ void k_init_scalars(DevScalars* s) {
  s->t = 0.0;
  s->dt = 0.0;
  s->t_end = __longlong_as_double((long long)kInfBits);
  s->lam_bits = kInfBits;
  s->status = 0;
  s->steps = 0;
}

// compensated form: u^n as the FP32 pair hi = fl(u^n), lo = fl(u^n - hi)
// (u^n - hi is exact in FP64), so hi + lo carries u^n to about 48 bits
__global__ void k_split(const double* __restrict__ u, float* __restrict__ hi, float* __restrict__ lo, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = u[i];
  const float h = (float)x;
  hi[i] = h;
  lo[i] = (float)(x - (double)h);
}

__global__ void k_widen(const float* __restrict__ in, double* __restrict__ out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

__global__ void k_dt_only(DevScalars* s, double cfl, double* out) {
  const unsigned long long lb = s->lam_bits;
  *out = lb == kInfBits ? 0.0 : cfl * __longlong_as_double((long long)lb);
}

// fixed-order reduction of nv arrays of length len (one CTA per variable)
__global__ void k_reduce(const double* __restrict__ part, size_t len, double* out) {
  __shared__ double red[1024];
  const int v = blockIdx.x, tid = threadIdx.x;
  double s = 0.0;
  for (size_t i = tid; i < len; i += blockDim.x) s += part[(size_t)v * len + i];
  red[tid] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) out[v] = red[0];
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (dev >= 0) {
      cudaGetDevice(&prev);
      if (prev != dev) cudaSetDevice(dev);
      else prev = -1;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Host vector whose elements are left uninitialised on resize: the large
// per-build tables are first touched by the (threaded) loops that fill them.
template <class T>
struct NoInit : std::allocator<T> {
  using value_type = T;
  template <class U>
  struct rebind {
    using other = NoInit<U>;
  };
  NoInit() = default;
  template <class U>
  NoInit(const NoInit<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new ((void*)p) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new ((void*)p) U(std::forward<A>(a)...);
  }
};
template <class T>
using hvec = std::vector<T, NoInit<T>>;

}  // namespace

struct dgf_forest {
  Forest host;
  int precision = DGF_FP64;
  int device = -1;
  double gamma = 1.4, cfl = 0.1;
  dgf_allocator alloc{};
  bool has_alloc = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t esize = 8;   // element size of the device compute buffers
  size_t sesize = 8;  // element size of the state at the C ABI
  bool comp = false;  // compensated form: u^n in FP64, stage increments in FP32
  bool all_affine = false;  // every leaf an affine block (the stage kernel needs no per-cell geometry)
  int cur = 0;        // compensated form: which U64 buffer holds u^n
  int d = 0, n = 0, p = 0, N = 0, nv = 0, M = 0, nc = 0, NG = 0, nt = 0, NFP = 0;
  int64_t nL = 0;
  RtTables tab{};
  Basis1D basis;

  struct Buf {
    void* ptr = nullptr;
    size_t bytes = 0;
  };
  Buf U64[2], hcell64, gmod64;
  Buf Uhi, Ulo;  // compensated form: u^n as the FP32 pair hi + lo, split once per step
  cudaGraphExec_t graph_alt = nullptr;  // compensated form: graph of the other u^n buffer
  Buf U[3], geo, geo64, hcell, gtr, gmod, cop, ctr, kind, nbr, orient, qbits, copoff, part, scal, tot,
      dtout, nodal, fine, affine, ameta, trd;
  int nfine = 0;
  // mortar treatment of level jumps (reading R15)
  bool mortar = false;
  Buf fluxmask, mfine, mcoarse, mw, msrc;
  int nmf = 0, nmc = 0;
  double limiter = 0.0;  // positivity limiter bound (relative); 0 = off
  Buf ind;               // refinement indicator per leaf (kept between calls)
  // host staging of the per-cell geometry, kept between builds so that a
  // rebuild after a regrid reuses its pages
  hvec<double> h_geo64, h_hcell;
  hvec<float> h_geo32, h_hcell32;
  // boundary faces: per root face 0 outflow, 1 prescribed state (bstate_h)
  std::vector<int32_t> bctag;
  std::vector<double> bstate_h;
  Buf bstate;
  int slots = 0;            // resident CTAs of the chosen stage kernel
  // resident CTAs: [0] the cell-pair kernel where it applies, [1] k_stage,
  // [2] the cell-pair kernel's five-CTA shape (p = 1; 0 elsewhere)
  int slots_k[3] = {0, 0, 0};
  int kernel = 0;           // stage kernel: 0 the cell-pair kernel where it applies, 1 k_stage
  bool grid_items = false;  // stage grid: one CTA per work item instead of the persistent CTAs
  bool have_state = false;
  bool graph_valid = false;
  cudaGraphExec_t graph = nullptr;
  double t_end_dev = NAN;
  int zchunk = 0;
  bool tuned = false;  // z-chunk length chosen by timing (first time step)
  bool timing = false;
  struct TEv {
    cudaEvent_t a, b;
    int cls;
  };
  std::vector<TEv> ev;
  double ms[3] = {0, 0, 0};
  int64_t launches[3] = {0, 0, 0};
};

namespace {

void* dev_alloc(dgf_forest* f, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (f->has_alloc) return f->alloc.alloc(f->alloc.ctx, bytes, (void*)f->stream);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}

void dev_free(dgf_forest* f, dgf_forest::Buf& b) {
  if (!b.ptr) return;
  if (f->has_alloc) {
    // the caller's allocator may hand the block out again at once: nothing
    // of this forest's may still touch it
    cudaStreamSynchronize(f->stream);
    f->alloc.free(f->alloc.ctx, b.ptr, b.bytes, (void*)f->stream);
  } else {
    cudaFree(b.ptr);
  }
  b.ptr = nullptr;
  b.bytes = 0;
}

bool ensure(dgf_forest* f, dgf_forest::Buf& b, size_t bytes) {
  if (b.ptr && b.bytes >= bytes) return true;
  dev_free(f, b);
  b.ptr = dev_alloc(f, bytes);
  b.bytes = b.ptr ? bytes : 0;
  return b.ptr != nullptr;
}

dgf_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DGF_OK;
  if (e == cudaErrorInvalidConfiguration)
    return fail(DGF_EUNSUPPORTED, std::string(what) + ": shared-memory footprint too large for "
                                                      "this (dim, p, n_seg, precision)");
  return fail(DGF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int pack_orient(const Orient& o, int d) {
  int v = 0;
  for (int a = 0; a < d; ++a) {
    v |= o.pi[a] << (2 * a);
    if (o.sg[a] < 0) v |= 1 << (6 + a);
  }
  return v;
}


template <typename V>
dgf_status upload(dgf_forest* f, dgf_forest::Buf& b, const V& v) {
  using T = typename V::value_type;
  if (!ensure(f, b, sizeof(T) * std::max<size_t>(v.size(), 1))) return fail(DGF_ENOMEM, "device allocation failed");
  if (v.empty()) return DGF_OK;
  // v is often a temporary: the copy from pageable memory may read it after
  // the call returns (the documented semantics allow it, and on a host whose
  // memory the GPU reaches directly it does), so wait before v goes away
  dgf_status st = cuda_check(
      cudaMemcpyAsync(b.ptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, f->stream), "upload");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(f->stream), "upload");
}

template <typename Fn>
void parallel_for(int64_t n, Fn&& fn);

// element-wise conversion (to the compute precision), in threaded chunks
template <typename V, typename W>
void convert_into(const V& v, W& out) {
  using T = typename W::value_type;
  out.clear();
  out.resize(v.size());
  constexpr int64_t kChunk = 1 << 16;
  parallel_for(((int64_t)v.size() + kChunk - 1) / kChunk, [&](int64_t c) {
    const size_t lo = (size_t)c * kChunk, hi = std::min(v.size(), lo + (size_t)kChunk);
    for (size_t i = lo; i < hi; ++i) out[i] = (T)v[i];
  });
}

template <typename T, typename V>
hvec<T> convert(const V& v) {
  hvec<T> out;
  convert_into(v, out);
  return out;
}

double phi(const Basis1D& B, int d, int m, const double* xi) {
  double r = 1.0;
  for (int a = 0; a < d; ++a) {
    r *= legendre(m % B.N, xi[a]);
    m /= B.N;
  }
  return r;
}

// Cholesky solve of an SPD system with several right-hand sides (FP64).
bool chol_solve(int M, std::vector<double>& A, std::vector<double>& B, int nrhs) {
  for (int j = 0; j < M; ++j) {
    double s = A[j * M + j];
    for (int k = 0; k < j; ++k) s -= A[j * M + k] * A[j * M + k];
    if (!(s > 0)) return false;
    A[j * M + j] = std::sqrt(s);
    for (int i = j + 1; i < M; ++i) {
      double t = A[i * M + j];
      for (int k = 0; k < j; ++k) t -= A[i * M + k] * A[j * M + k];
      A[i * M + j] = t / A[j * M + j];
    }
  }
  for (int r = 0; r < nrhs; ++r) {
    for (int i = 0; i < M; ++i) {
      double t = B[i * nrhs + r];
      for (int k = 0; k < i; ++k) t -= A[i * M + k] * B[k * nrhs + r];
      B[i * nrhs + r] = t / A[i * M + i];
    }
    for (int i = M - 1; i >= 0; --i) {
      double t = B[i * nrhs + r];
      for (int k = i + 1; k < M; ++k) t -= A[k * M + i] * B[k * nrhs + r];
      B[i * nrhs + r] = t / A[i * M + i];
    }
  }
  return true;
}

// DGF_STAGE_GRID=persistent|items fixes the stage grid; otherwise dflt
bool grid_env(bool dflt) {
  const char* g = getenv("DGF_STAGE_GRID");
  if (!g) return dflt;
  return strcmp(g, "items") == 0;
}

// the cell-pair FP32 stage kernel covers 3D forests of 8^3-cell blocks at
// p = 1, 2 in plain FP32
bool pair_applies(const dgf_forest* f) {
  return f->d == 3 && f->n == 8 && (f->p == 1 || f->p == 2) && f->precision == DGF_FP32 && !f->comp;
}

// Build every leaf-dependent device array: integer tables, FP64 geometry,
// cell sizes, combine operators, state and scratch buffers.
// fn(0 .. n-1) on up to 16 host threads; every index writes its own outputs,
// so the result does not depend on the schedule
template <class Fn>
void parallel_for(int64_t n, Fn&& fn) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int64_t nt = std::min<int64_t>(std::min<unsigned>(hw, 16u), n);
  if (nt <= 1) {
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int64_t> next{0};
  std::vector<std::thread> pool;
  for (int64_t t = 0; t < nt; ++t)
    pool.emplace_back([&]() {
      for (int64_t i; (i = next.fetch_add(1)) < n;) fn(i);
    });
  for (auto& th : pool) th.join();
}

dgf_status build_device(dgf_forest* f) {
  Forest& F = f->host;
  const int d = f->d, n = f->n, nf = 2 * d, M = f->M, nc = f->nc, NG = f->NG, N = f->N;
  const int64_t L = F.n_leaves();
  if (f->device >= 0 && f->stream) {
    DeviceGuard dg(f->device);
    cudaStreamSynchronize(f->stream);  // buffers may be freed or reused below
  }
  f->nL = L;
  Forest::Tables T = F.tables();

  std::vector<int> kind(L * nf), nbr(L * nf * 4), orient(L * nf), qbits(L), copoff(L * nf, -1);
  for (int64_t i = 0; i < L * nf; ++i) {
    kind[i] = T.kind[i];
    if (kind[i] == kBoundary && !f->bctag.empty() && f->bctag[(size_t)T.root[i / nf] * nf + i % nf] == 1)
      kind[i] = 4;  // prescribed state (device-side code only)
    orient[i] = pack_orient(orient_from_code(T.orient[i], d), d);
    for (int s = 0; s < 4; ++s) nbr[i * 4 + s] = (int)T.nbr[i * 4 + s];
  }
  for (int64_t i = 0; i < L; ++i) {
    int q = 0;
    for (int a = 0; a < d; ++a) q |= (T.pos[i * d + a] & 1) << a;
    qbits[i] = q;
  }

  // Face-trace descriptors of the time-step guard kernel.  For a face of kind
  // same-level, coarser or outflow, the trace seen by my guard cell (g0, g1)
  // (my tangential axes in increasing order; for a coarser neighbour the
  // coarse cell index G >> 1 of my position G on its face) at my face point
  // (q0, q1) is sum_qn l[qn] u(src, cell, point) with
  //   cell  = cbase + g0 CS0 + g1 CS1,
  //   point = (pbase + q0 PS0 + q1 PS1 + qn PSN) / nc   (strides times nc),
  // l the source face's side table (l(+1) or l(-1)): the orientation becomes
  // signed strides.  Entries: src, cbase, CS0, CS1, pbase, PS0, PS1, PSN * 2
  // + side.  The outflow trace is my own face cell's (src = me).
  std::vector<int> trd((size_t)L * nf * 8, 0);
  {
    const int Nq = f->p + 1;
    auto ipw = [](int b, int e) {
      int r = 1;
      while (e-- > 0) r *= b;
      return r;
    };
    for (int64_t i = 0; i < L; ++i)
      for (int fc = 0; fc < nf; ++fc) {
        const int k = kind[i * nf + fc];
        if (k != kSame && k != kCoarser && k != kBoundary) continue;
        const int a = fc >> 1, s = fc & 1;
        int ta[2] = {0, 0}, m = 0;
        for (int ax = 0; ax < d; ++ax)
          if (ax != a) ta[m++] = ax;
        int src = (int)i, b2 = a, s2 = s, A[2] = {ta[0], ta[1]}, sgn[2] = {1, 1};
        if (k != kBoundary) {
          const Orient o = orient_from_code(T.orient[i * nf + fc], d);
          src = nbr[(i * nf + fc) * 4];
          b2 = o.pi[a];
          s2 = o.sg[a] > 0 ? 1 - s : s;
          for (int j = 0; j < d - 1; ++j) {
            A[j] = o.pi[ta[j]];
            sgn[j] = o.sg[ta[j]];
          }
        }
        int cbase = s2 ? (n - 1) * ipw(n, b2) : 0, pbase = 0, CS[2] = {0, 0}, PS[2] = {0, 0};
        for (int j = 0; j < d - 1; ++j) {
          const int cs = ipw(n, A[j]), ps = ipw(Nq, A[j]);
          CS[j] = sgn[j] * cs;
          PS[j] = sgn[j] * ps;
          if (sgn[j] < 0) {
            cbase += (n - 1) * cs;
            pbase += (Nq - 1) * ps;
          }
        }
        int* e = &trd[((size_t)i * nf + fc) * 8];
        e[0] = src;
        e[1] = cbase;
        e[2] = CS[0];
        e[3] = CS[1];
        e[4] = pbase * nc;
        e[5] = PS[0] * nc;
        e[6] = PS[1] * nc;
        e[7] = ipw(Nq, b2) * nc * 2 + s2;
      }
  }

  // geometry: per-cell trilinear coefficients (c >= 1) and sizes h; the
  // leaves are independent, so host threads take them in any order
  std::vector<std::vector<double>> coef(L);
  hvec<double>& geo64 = f->h_geo64;
  hvec<double>& hcell = f->h_hcell;
  geo64.clear();  // no copy of the old contents when the capacity grows
  hcell.clear();
  geo64.resize((size_t)L * NG * nc);
  hcell.resize((size_t)L * nc);
  const Basis1D& B = f->basis;
  {
    // block nodes of every leaf and of its uncached ancestors, one level at a
    // time: the blocks of a level in parallel from their parents' nodes
    const std::vector<uint64_t> miss = F.uncached_nodes(F.leaves);
    auto level_of = [](uint64_t k) {
      int64_t r;
      int lev, pos[3];
      Forest::unkey(k, &r, &lev, pos);
      return lev;
    };
    size_t lo = 0;
    while (lo < miss.size()) {
      const int lev = level_of(miss[lo]);
      size_t hi = lo;
      while (hi < miss.size() && level_of(miss[hi]) == lev) ++hi;
      std::vector<std::vector<double>> X(hi - lo);
      parallel_for((int64_t)(hi - lo), [&](int64_t j) { F.compute_nodes(miss[lo + j], X[j]); });
      for (size_t j = lo; j < hi; ++j) F.put_nodes(miss[j], std::move(X[j - lo]));
      lo = hi;
    }
  }
  parallel_for(L, [&](int64_t i) {
    F.cell_coefficients(F.leaves[i], coef[i]);
    for (int g = 0; g < NG; ++g)
      for (int c = 0; c < nc; ++c) geo64[((size_t)i * NG + g) * nc + c] = coef[i][(size_t)(d + g) * nc + c];
  });

  // affine blocks: every cell a congruent parallelogram/parallelepiped ->
  // constant J dxi/dx rows and 1/J per block
  std::vector<unsigned char> affine(L, 0);
  std::vector<double> ameta((size_t)L * (d * d + 1), 0.0);
  parallel_for(L, [&](int64_t i) {
    const std::vector<double>& C = coef[i];
    double scale = 0.0;
    for (int k = d; k < (1 << d) * d; ++k)
      for (int c = 0; c < nc; ++c) scale = std::max(scale, std::fabs(C[(size_t)k * nc + c]));
    bool ok = scale > 0.0;
    for (int cm = 1; cm < (1 << d) && ok; ++cm) {
      const bool linear = (cm & (cm - 1)) == 0;
      for (int j = 0; j < d && ok; ++j) {
        const double* row = &C[((size_t)cm * d + j) * nc];
        for (int c = 0; c < nc && ok; ++c) {
          if (!linear && std::fabs(row[c]) > 1e-13 * scale) ok = false;
          if (linear && std::fabs(row[c] - row[0]) > 1e-13 * scale) ok = false;
        }
      }
    }
    if (!ok) return;
    double cc[24], A[9], Ja[9], xi[3] = {0, 0, 0};
    for (int k = 0; k < (1 << d) * d; ++k) cc[k] = C[(size_t)k * nc];
    eval_map(d, cc, xi, nullptr, A);
    const double J = det_and_cofactor(d, A, Ja);
    if (!(J > 0)) return;
    affine[i] = 1;
    for (int k = 0; k < d * d; ++k) ameta[(size_t)i * (d * d + 1) + k] = Ja[k];
    ameta[(size_t)i * (d * d + 1) + d * d] = 1.0 / J;
  });

  // cell sizes h = (cell volume)^(1/d), the volume by the Gauss rule (an
  // affine block's cells: J times the reference volume 2^d)
  parallel_for(L, [&](int64_t i) {
    if (affine[i]) {
      const double h = std::pow((double)(1 << d) / ameta[(size_t)i * (d * d + 1) + d * d], 1.0 / d);
      for (int c = 0; c < nc; ++c) hcell[(size_t)i * nc + c] = h;
      return;
    }
    for (int c = 0; c < nc; ++c) {
      double cc[8 * 3];
      for (int k = 0; k < (1 << d) * d; ++k) cc[k] = coef[i][(size_t)k * nc + c];
      double vol = 0.0;
      for (int q = 0; q < M; ++q) {
        double xi[3], wq = 1.0;
        int r = q;
        for (int a = 0; a < d; ++a) {
          xi[a] = B.x[r % N];
          wq *= B.w[r % N];
          r /= N;
        }
        double A[9], Ja[9];
        eval_map(d, cc, xi, nullptr, A);
        vol += wq * det_and_cofactor(d, A, Ja);
      }
      hcell[(size_t)i * nc + c] = std::pow(vol, 1.0 / d);
    }
  });

  // combine operators for every finer-neighbour guard cell (Eqs. (13)-(14),
  // J-weighted, integrals by each child's Gauss rule), rotated into my frame
  const int nt = f->nt;
  int64_t nops = 0;
  const int KC = (1 << d) * M;
  std::vector<int> fine_list;
  for (int64_t i = 0; i < L; ++i)
    for (int fc = 0; fc < nf; ++fc)
      if (kind[i * nf + fc] == kFiner) fine_list.push_back((int)(i * nf + fc));
  // fine neighbours that are affine blocks of one Jacobian give every guard
  // cell of a face the same operator: such a face stores one, flagged by bit
  // 0 of its entry (copoff = first operator << 1 | shared)
  std::vector<unsigned char> shared_op(fine_list.size(), 0);
  for (size_t fi = 0; fi < fine_list.size(); ++fi) {
    const int64_t i = fine_list[fi] / nf;
    const int fc = fine_list[fi] % nf;
    bool uniform = true;
    for (int sb = 0; sb < (1 << (d - 1)) && uniform; ++sb) {
      const int64_t fl = T.nbr[(i * nf + fc) * 4 + sb];
      const int64_t f0 = T.nbr[(i * nf + fc) * 4];
      uniform = affine[fl] &&
                ameta[(size_t)fl * (d * d + 1) + d * d] == ameta[(size_t)f0 * (d * d + 1) + d * d];
    }
    shared_op[fi] = uniform;
    copoff[i * nf + fc] = (int)(nops << 1) | (uniform ? 1 : 0);
    nops += uniform ? 1 : nt;
  }
  f->nfine = (int)fine_list.size();
  const int NFPh = f->NFP;
  hvec<double> cop((size_t)nops * M * KC), ctr((size_t)nops * NFPh * KC);
  std::atomic<bool> singular{false};
  parallel_for((int64_t)fine_list.size(), [&](int64_t fi) {
    {
      const int64_t i = fine_list[fi] / nf;
      const int fc = fine_list[fi] % nf;
      const Orient o = orient_from_code(T.orient[i * nf + fc], d);
      const int a = fc >> 1, s = fc & 1;
      const int b2 = o.pi[a];
      const int s2 = o.sg[a] > 0 ? 1 - s : s;
      const size_t o0 = (size_t)(copoff[i * nf + fc] >> 1);
      const int tn = shared_op[fi] ? 1 : nt;
      for (int t = 0; t < tn; ++t) {
        int g[3] = {0, 0, 0}, j = 0;
        for (int ax = 0; ax < d; ++ax) {
          if (ax == a) continue;
          g[ax] = j == 0 ? t % n : t / n;
          ++j;
        }
        int h[3] = {0, 0, 0};
        for (int ax = 0; ax < d; ++ax) {
          if (ax == a) continue;
          h[o.pi[ax]] = o.sg[ax] > 0 ? g[ax] : n - 1 - g[ax];
        }
        h[b2] = s2 == 0 ? 0 : n - 1;
        int sub = 0;
        j = 0;
        for (int ax = 0; ax < d; ++ax) {
          if (ax == a) continue;
          if (g[ax] >= n / 2) sub |= 1 << j;
          ++j;
        }
        const int64_t fine = T.nbr[(i * nf + fc) * 4 + sub];
        int cN[3] = {0, 0, 0};
        for (int ax = 0; ax < d; ++ax) cN[ax] = (2 * h[ax]) / n;
        std::vector<double> MP(M * M, 0.0), RHS((size_t)M * KC, 0.0);
        for (int e = 0; e < (1 << d); ++e) {
          int cell = 0, st = 1;
          for (int ax = 0; ax < d; ++ax) {
            cell += (2 * h[ax] + ((e >> ax) & 1) - cN[ax] * n) * st;
            st *= n;
          }
          double cc[8 * 3];
          for (int k = 0; k < (1 << d) * d; ++k) cc[k] = coef[fine][(size_t)k * nc + cell];
          for (int q = 0; q < M; ++q) {
            double xi[3], xp[3], wq = 1.0;
            int r = q;
            for (int ax = 0; ax < d; ++ax) {
              xi[ax] = B.x[r % N];
              wq *= B.w[r % N];
              xp[ax] = 0.5 * (xi[ax] + (((e >> ax) & 1) ? 1.0 : -1.0));
              r /= N;
            }
            double A[9], Ja[9];
            eval_map(d, cc, xi, nullptr, A);
            const double wj = wq * det_and_cofactor(d, A, Ja);
            double pp[64];
            for (int m = 0; m < M; ++m) pp[m] = phi(B, d, m, xp);
            for (int m = 0; m < M; ++m) {
              for (int m2 = 0; m2 < M; ++m2) MP[m * M + m2] += wj * pp[m] * pp[m2];
              // right-hand side acts on child e's values at its Gauss points
              RHS[(size_t)m * KC + e * M + q] += wj * pp[m];
            }
          }
        }
        if (!chol_solve(M, MP, RHS, KC)) {
          singular = true;
          return;
        }
        // evaluate the parent polynomial (neighbour frame) at my Gauss points:
        // my point p sits at neighbour coordinates xi_{pi[a]} = sigma_a x_{p_a}
        double* dst = &cop[(o0 + t) * M * KC];
        for (int pt = 0; pt < M; ++pt) {
          double xs[3] = {0, 0, 0};
          int rem = pt;
          for (int ax = 0; ax < d; ++ax) {
            xs[o.pi[ax]] = o.sg[ax] * B.x[rem % N];
            rem /= N;
          }
          double ph[64];
          for (int m = 0; m < M; ++m) ph[m] = phi(B, d, m, xs);
          for (int k = 0; k < KC; ++k) {
            double acc = 0.0;
            for (int m = 0; m < M; ++m) acc += ph[m] * RHS[(size_t)m * KC + k];
            dst[(size_t)k * M + pt] = acc;
          }
        }
        // trace operator: the guard cell's values on its face touching me
        // (xi_a = -1 on my + face, +1 on my - face) at my face points
        const std::vector<double>& ext = s ? B.lm : B.lp;
        double* tdst = &ctr[(o0 + t) * NFPh * KC];
        std::fill(tdst, tdst + (size_t)NFPh * KC, 0.0);
        for (int fpp = 0; fpp < NFPh; ++fpp) {
          int dig[3] = {0, 0, 0}, rem = fpp;
          for (int ax = 0; ax < d; ++ax) {
            if (ax == a) continue;
            dig[ax] = rem % N;
            rem /= N;
          }
          for (int qn = 0; qn < N; ++qn) {
            dig[a] = qn;
            int pt = 0, st = 1;
            for (int ax = 0; ax < d; ++ax) {
              pt += dig[ax] * st;
              st *= N;
            }
            for (int k = 0; k < KC; ++k) tdst[(size_t)k * NFPh + fpp] += ext[qn] * dst[(size_t)k * M + pt];
          }
        }
      }
    }
  });
  if (singular) return fail(DGF_EINVAL, "singular combine mass matrix");

  // mortar tables (reading R15): faces with a coarser neighbour take their
  // flux from the fine-side pass; faces with finer neighbours integrate those
  // fluxes against their own face test functions
  std::vector<unsigned char> fluxmask(L, 0);
  std::vector<int> mfine, mcoarse;
  std::vector<double> mw;
  std::vector<long long> msrc;
  if (f->mortar) {
    const int NSUB = 1 << (d - 1), NFPm = f->NFP;
    for (int64_t i = 0; i < L; ++i)
      for (int fc = 0; fc < nf; ++fc) {
        const int k = kind[i * nf + fc];
        if (k == kCoarser) mfine.push_back((int)(i * nf + fc));
        if (k == kFiner) mcoarse.push_back((int)(i * nf + fc));
        if (k == kCoarser || k == kFiner) fluxmask[i] |= (unsigned char)(1 << fc);
      }
    mw.assign(mcoarse.size() * NFPm * NSUB * NFPm, 0.0);
    msrc.assign(mcoarse.size() * nt * NSUB, 0);
    for (size_t mi = 0; mi < mcoarse.size(); ++mi) {
      const int64_t i = mcoarse[mi] / nf;
      const int fc = mcoarse[mi] % nf;
      const Orient o = orient_from_code(T.orient[i * nf + fc], d);
      const int a = fc >> 1, s = fc & 1;
      const int b2 = o.pi[a];
      const int s2 = o.sg[a] > 0 ? 1 - s : s;
      const int f2 = 2 * b2 + s2;
      const double sgn = -(s ? 1.0 : -1.0) * (s2 ? 1.0 : -1.0);
      int mt[2] = {0, 0}, ut[2] = {0, 0}, nmt = 0, nut = 0;  // my / the neighbour's tangential axes
      for (int ax = 0; ax < d; ++ax) {
        if (ax != a) mt[nmt++] = ax;
        if (ax != b2) ut[nut++] = ax;
      }
      // weights: my point j <- sub-face esub (bits over ut), its point k (digits over ut)
      for (int j = 0; j < NFPm; ++j)
        for (int es = 0; es < NSUB; ++es)
          for (int k = 0; k < NFPm; ++k) {
            int jd[3] = {0, 0, 0}, kd[3] = {0, 0, 0}, ed[3] = {0, 0, 0};
            for (int q = 0, rj = j, rk = k; q < d - 1; ++q, rj /= N, rk /= N) {
              jd[mt[q]] = rj % N;
              kd[ut[q]] = rk % N;
              ed[ut[q]] = (es >> q) & 1;
            }
            double wgt = sgn;
            for (int q = 0; q < d - 1; ++q) {
              const int ax = mt[q], u = o.pi[ax];
              const double xi = o.sg[ax] * 0.5 * (B.x[kd[u]] + 2.0 * ed[u] - 1.0);
              wgt *= B.w[kd[u]] * B.lagrange(jd[ax], xi) / B.w[jd[ax]];
            }
            mw[((mi * NFPm + j) * NSUB + es) * NFPm + k] = wgt;
          }
      // sources: per guard cell t, the fine leaf and its guard index per sub-face
      for (int t = 0; t < nt; ++t) {
        int g[3] = {0, 0, 0}, h[3] = {0, 0, 0}, sub = 0;
        for (int q = 0; q < d - 1; ++q) g[mt[q]] = q == 0 ? t % n : t / n;
        for (int q = 0; q < d - 1; ++q) {
          const int ax = mt[q];
          h[o.pi[ax]] = o.sg[ax] > 0 ? g[ax] : n - 1 - g[ax];
          if (g[ax] >= n / 2) sub |= 1 << q;
        }
        h[b2] = s2 == 0 ? 0 : n - 1;
        const int64_t fine = T.nbr[(i * nf + fc) * 4 + sub];
        for (int es = 0; es < NSUB; ++es) {
          int tf = 0;
          for (int q = 0, st = 1; q < d - 1; ++q, st *= n) {
            const int u = ut[q];
            const int H = 2 * h[u] + ((es >> q) & 1);
            tf += (H - (2 * h[u] / n) * n) * st;
          }
          msrc[((size_t)mi * nt + t) * NSUB + es] =
              ((long long)fine * nf + f2) * f->nv * NFPm * nt + tf;
        }
      }
    }
  }
  f->nmf = (int)mfine.size();
  f->nmc = (int)mcoarse.size();

  if (f->device < 0) return DGF_OK;
  DeviceGuard dg(f->device);
  dgf_status st;
  {
    std::vector<double> bs(f->nv, 0.0);
    if (!f->bstate_h.empty()) bs = f->bstate_h;
    st = f->precision == DGF_FP64 ? upload(f, f->bstate, bs) : upload(f, f->bstate, convert<float>(bs));
    if (st) return st;
  }
  if ((st = upload(f, f->kind, kind)) || (st = upload(f, f->nbr, nbr)) || (st = upload(f, f->orient, orient)) ||
      (st = upload(f, f->qbits, qbits)) || (st = upload(f, f->copoff, copoff)) || (st = upload(f, f->geo64, geo64)) ||
      (st = upload(f, f->fine, fine_list)) || (st = upload(f, f->trd, trd)))
    return st;
  if ((st = upload(f, f->affine, affine)) || (st = upload(f, f->hcell64, hcell))) return st;
  f->all_affine = std::all_of(affine.begin(), affine.end(), [](unsigned char a) { return a != 0; });
  if (f->mortar && ((st = upload(f, f->fluxmask, fluxmask)) || (st = upload(f, f->mfine, mfine)) ||
                    (st = upload(f, f->mcoarse, mcoarse)) || (st = upload(f, f->msrc, msrc))))
    return st;
  if (f->precision == DGF_FP64) {
    if ((st = upload(f, f->geo, geo64)) || (st = upload(f, f->hcell, hcell)) || (st = upload(f, f->cop, cop)) ||
        (st = upload(f, f->ctr, ctr)) ||
        (st = upload(f, f->ameta, ameta)))
      return st;
    if (f->mortar && (st = upload(f, f->mw, mw))) return st;
  } else {
    if (f->mortar && (st = upload(f, f->mw, convert<float>(mw)))) return st;
    convert_into(geo64, f->h_geo32);
    convert_into(hcell, f->h_hcell32);
    if ((st = upload(f, f->geo, f->h_geo32)) || (st = upload(f, f->hcell, f->h_hcell32)) ||
        (st = upload(f, f->cop, convert<float>(cop))) || (st = upload(f, f->ctr, convert<float>(ctr))) ||
        (st = upload(f, f->ameta, convert<float>(ameta))))
      return st;
  }
  const size_t sbytes = (size_t)L * f->nv * M * nc * f->esize;
  for (int k = 0; k < 3; ++k)
    if (!ensure(f, f->U[k], sbytes)) return fail(DGF_ENOMEM, "state allocation failed");
  if (f->comp) {
    for (int k = 0; k < 2; ++k)
      if (!ensure(f, f->U64[k], (size_t)L * f->nv * M * nc * sizeof(double)))
        return fail(DGF_ENOMEM, "state allocation failed");
    if (!ensure(f, f->Uhi, (size_t)L * f->nv * M * nc * sizeof(float)) ||
        !ensure(f, f->Ulo, (size_t)L * f->nv * M * nc * sizeof(float)))
      return fail(DGF_ENOMEM, "state allocation failed");
  }
  if (!ensure(f, f->gtr, (size_t)L * nf * f->nv * f->NFP * nt * f->esize) ||
      !ensure(f, f->part, (size_t)L * nc * f->nv * sizeof(double)))
    return fail(DGF_ENOMEM, "scratch allocation failed");
  // resident stage CTAs, and the z-chunk length that balances the
  // persistent CTAs best (a chunk costs its layers plus ~0.3 layer of halo)
  {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device);
    const int cp = f->comp ? 1 : 0;
    for (int kk = 0; kk < 3; ++kk) {
      int occ = 0;
      if (d == 2)
        occ = f->precision == DGF_FP64 ? stage_occupancy<2, double>(f->p, n, cp, kk)
                                       : stage_occupancy<2, float>(f->p, n, cp, kk);
      else
        occ = f->precision == DGF_FP64 ? stage_occupancy<3, double>(f->p, n, cp, kk)
                                       : stage_occupancy<3, float>(f->p, n, cp, kk);
      f->slots_k[kk] = occ * sms;
    }
    if (!(pair_applies(f) && f->p == 1)) f->slots_k[2] = 0;
    // the cell-pair kernel unless it does not apply (its slots equal k_stage's
    // then) or DGF_STAGE_KERNEL=classic|pair5; the autotuner may still pick
    // another
    f->kernel = pair_applies(f) ? 0 : 1;
    if (const char* ks = getenv("DGF_STAGE_KERNEL")) {
      if (strcmp(ks, "classic") == 0) f->kernel = 1;
      if (strcmp(ks, "pair5") == 0 && f->slots_k[2] > 0) f->kernel = 2;
    }
    f->slots = f->slots_k[f->kernel];
    f->zchunk = 1;
    if (d == 3 && f->slots > 0) {
      double best = 1e300;
      for (int z = n; z >= 1; z /= 2) {
        const int64_t items = L * ((n + z - 1) / z);
        const double rounds = (double)((items + f->slots - 1) / f->slots);
        const double cost = rounds * (z + 0.3);
        if (cost < best - 1e-9) {
          best = cost;
          f->zchunk = z;
        }
        if (z == 1) break;
      }
      if (const char* zc = getenv("DGF_ZCHUNK")) f->zchunk = std::max(1, std::min(n, atoi(zc)));
    }
  }
  f->grid_items = grid_env(false);
  f->tuned = d != 3 || (getenv("DGF_ZCHUNK") != nullptr && getenv("DGF_STAGE_KERNEL") != nullptr &&
                        getenv("DGF_STAGE_GRID") != nullptr);
  if (f->graph) {
    cudaGraphExecDestroy(f->graph);
    f->graph = nullptr;
  }
  if (f->graph_alt) {
    cudaGraphExecDestroy(f->graph_alt);
    f->graph_alt = nullptr;
  }
  f->graph_valid = false;
  return DGF_OK;
}

RtStage stage_args(dgf_forest* f, int src, int dst, double ca, double cb, int mode, int last) {
  RtStage r{};
  r.p = f->p;
  r.nL = (int)f->nL;
  r.n = f->n;
  r.zchunk = f->zchunk;
  r.slots = f->grid_items ? INT_MAX : f->slots;  // the launch takes min(items, slots) CTAs
  r.kernel = f->kernel;
  r.affine = (const unsigned char*)f->affine.ptr;
  r.all_affine = f->all_affine ? 1 : 0;
  r.ameta = f->ameta.ptr;
  r.kind = (const int*)f->kind.ptr;
  r.nbr = (const int*)f->nbr.ptr;
  r.orient = (const int*)f->orient.ptr;
  r.qbits = (const int*)f->qbits.ptr;
  r.U = f->U[src].ptr;
  r.Un = f->U[0].ptr;
  r.Uout = f->U[dst].ptr;
  r.geo = f->geo.ptr;
  r.gtr = f->gtr.ptr;
  r.hcell = f->hcell.ptr;
  r.dtp = &((DevScalars*)f->scal.ptr)->dt;
  r.lam_bits = &((DevScalars*)f->scal.ptr)->lam_bits;
  r.status = &((DevScalars*)f->scal.ptr)->status;
  r.ca = ca;
  r.cb = cb;
  r.gamma = f->gamma;
  r.mode = mode;
  r.last = last;
  if (f->comp) {
    r.comp = 1;
    r.U64 = (const double*)f->U64[f->cur].ptr;
    r.Uhi = (const float*)f->Uhi.ptr;
    r.Ulo = (const float*)f->Ulo.ptr;
    r.Din = src == 0 ? nullptr : (const float*)f->U[src].ptr;
    r.U64out = (double*)f->U64[1 - f->cur].ptr;
  }
  if (f->mortar) r.fluxmask = (const unsigned char*)f->fluxmask.ptr;
  r.T = f->tab;
  return r;
}

RtGuard guard_args(dgf_forest* f, int src, void* out, int mode) {
  RtGuard r{};
  r.p = f->p;
  r.nL = (int)f->nL;
  r.n = f->n;
  r.mode = mode;
  r.U = f->U[src].ptr;
  r.out = out;
  r.kind = (const int*)f->kind.ptr;
  r.nbr = (const int*)f->nbr.ptr;
  r.orient = (const int*)f->orient.ptr;
  r.qbits = (const int*)f->qbits.ptr;
  r.copoff = (const int*)f->copoff.ptr;
  r.cop = f->cop.ptr;
  r.ctr = f->ctr.ptr;
  r.fine_list = (const int*)f->fine.ptr;
  r.nfine = f->nfine;
  r.trd = (const int*)f->trd.ptr;
  r.geo = f->geo.ptr;
  r.gamma = f->gamma;
  r.bstate = f->bstate.ptr;
  if (f->mortar && mode == 1) {
    r.nfine = 0;  // the coarse side's flux comes from the mortar passes
    r.mfine = (const int*)f->mfine.ptr;
    r.nmf = f->nmf;
    r.mcoarse = (const int*)f->mcoarse.ptr;
    r.nmc = f->nmc;
    r.mw = f->mw.ptr;
    r.msrc = (const long long*)f->msrc.ptr;
  }
  if (f->comp) {
    r.comp = 1;
    r.U64 = (const double*)f->U64[f->cur].ptr;
    r.Uhi = (const float*)f->Uhi.ptr;
    r.Ulo = (const float*)f->Ulo.ptr;
    r.Din = src == 0 ? nullptr : (const float*)f->U[src].ptr;
  }
  r.T = f->tab;
  return r;
}

// device state buffer u^n (nodal) and whether it is FP64
void* state_ptr(dgf_forest* f) { return f->comp ? f->U64[f->cur].ptr : f->U[0].ptr; }
bool state_f64(dgf_forest* f) { return f->precision != DGF_FP32; }

RtMisc misc_args(dgf_forest* f, int src) {
  RtMisc r{};
  r.p = f->p;
  r.nL = (int)f->nL;
  r.n = f->n;
  void* u = src == 0 ? state_ptr(f) : f->U[src].ptr;
  r.U = u;
  r.Uout = u;
  r.hcell = state_f64(f) ? f->hcell64.ptr : f->hcell.ptr;
  r.geo64 = (const double*)f->geo64.ptr;
  r.part = (double*)f->part.ptr;
  r.gamma = f->gamma;
  r.lam_bits = &((DevScalars*)f->scal.ptr)->lam_bits;
  r.status = &((DevScalars*)f->scal.ptr)->status;
  r.T = f->tab;
  return r;
}

cudaError_t do_stage(dgf_forest* f, const RtStage& r) {
  if (f->d == 2) return f->precision == DGF_FP64 ? launch_stage<2, double>(r, f->stream) : launch_stage<2, float>(r, f->stream);
  return f->precision == DGF_FP64 ? launch_stage<3, double>(r, f->stream) : launch_stage<3, float>(r, f->stream);
}
// compensated form: split u^n into the FP32 pair the stage inputs read
// (nothing to do in the other precisions)
cudaError_t split_state(dgf_forest* f) {
  if (!f->comp) return cudaSuccess;
  const size_t n = (size_t)f->nL * f->nv * f->M * f->nc;
  k_split<<<(unsigned)((n + 255) / 256), 256, 0, f->stream>>>((const double*)f->U64[f->cur].ptr, (float*)f->Uhi.ptr,
                                                                (float*)f->Ulo.ptr, n);
  return cudaGetLastError();
}

cudaError_t do_guard(dgf_forest* f, const RtGuard& r) {
  if (f->d == 2) return f->precision == DGF_FP64 ? launch_guard<2, double>(r, f->stream) : launch_guard<2, float>(r, f->stream);
  return f->precision == DGF_FP64 ? launch_guard<3, double>(r, f->stream) : launch_guard<3, float>(r, f->stream);
}
cudaError_t do_cfl(dgf_forest* f, const RtMisc& r) {
  if (f->d == 2) return state_f64(f) ? launch_cfl<2, double>(r, f->stream) : launch_cfl<2, float>(r, f->stream);
  return state_f64(f) ? launch_cfl<3, double>(r, f->stream) : launch_cfl<3, float>(r, f->stream);
}
cudaError_t do_project(dgf_forest* f, const RtMisc& r) {
  if (f->d == 2) return state_f64(f) ? launch_project<2, double>(r, f->stream) : launch_project<2, float>(r, f->stream);
  return state_f64(f) ? launch_project<3, double>(r, f->stream) : launch_project<3, float>(r, f->stream);
}
cudaError_t do_totals(dgf_forest* f, const RtMisc& r) {
  if (f->d == 2) return state_f64(f) ? launch_totals<2, double>(r, f->stream) : launch_totals<2, float>(r, f->stream);
  return state_f64(f) ? launch_totals<3, double>(r, f->stream) : launch_totals<3, float>(r, f->stream);
}
cudaError_t do_indicator(dgf_forest* f, const RtMisc& r) {
  if (f->d == 2) return state_f64(f) ? launch_indicator<2, double>(r, f->stream) : launch_indicator<2, float>(r, f->stream);
  return state_f64(f) ? launch_indicator<3, double>(r, f->stream) : launch_indicator<3, float>(r, f->stream);
}
// the limiter runs on a compute-precision stage buffer
cudaError_t do_limit(dgf_forest* f, void* buf) {
  RtMisc r = misc_args(f, 0);
  r.Uout = buf;
  r.geo = f->geo.ptr;
  r.affine = (const unsigned char*)f->affine.ptr;
  r.eps = f->limiter;
  if (f->d == 2) return f->precision == DGF_FP64 ? launch_limit<2, double>(r, f->stream) : launch_limit<2, float>(r, f->stream);
  return f->precision == DGF_FP64 ? launch_limit<3, double>(r, f->stream) : launch_limit<3, float>(r, f->stream);
}
cudaError_t do_transfer(dgf_forest* f, const RtTransfer& r) {
  if (f->d == 2) return state_f64(f) ? launch_transfer<2, double>(r, f->stream) : launch_transfer<2, float>(r, f->stream);
  return state_f64(f) ? launch_transfer<3, double>(r, f->stream) : launch_transfer<3, float>(r, f->stream);
}

// modal <-> nodal in place; dbl selects the element type of X
cudaError_t do_convert(dgf_forest* f, void* X, size_t outer, int inner, int to_nodal, bool dbl) {
  if (f->d == 2)
    return dbl ? launch_convert<2, double>(f->p, outer, inner, X, to_nodal, f->tab, f->stream)
               : launch_convert<2, float>(f->p, outer, inner, X, to_nodal, f->tab, f->stream);
  return dbl ? launch_convert<3, double>(f->p, outer, inner, X, to_nodal, f->tab, f->stream)
             : launch_convert<3, float>(f->p, outer, inner, X, to_nodal, f->tab, f->stream);
}

// compute-precision buffer -> state-precision buffer (compensated form: FP32 -> FP64)
dgf_status widen(dgf_forest* f, const void* in, void* out, size_t count) {
  k_widen<<<(unsigned)((count + 255) / 256), 256, 0, f->stream>>>((const float*)in, (double*)out, count);
  return cuda_check(cudaGetLastError(), "widen");
}

dgf_status require_device(dgf_forest* f) {
  if (!f) return fail(DGF_EINVAL, "null forest");
  if (f->device < 0) return fail(DGF_ESTATE, "host-only forest has no device state");
  return DGF_OK;
}

dgf_status init_lambda(dgf_forest* f) {
  DevScalars* s = (DevScalars*)f->scal.ptr;
  k_reset_lam<<<1, 1, 0, f->stream>>>(s);
  dgf_status st = cuda_check(cudaGetLastError(), "reset");
  if (st) return st;
  return cuda_check(do_cfl(f, misc_args(f, 0)), "cfl");
}

// Autotuner for the stage kernel: time one residual evaluation (mode 1,
// written to a scratch stage buffer, the state is untouched) for every
// stage kernel that applies to the forest (the cell-pair kernel and
// k_stage, each with its own persistent grid) and every z-chunk length n,
// n/2, ..., 1, and keep the fastest pair (median of 3 launches).  Choices
// so far, by (device, dim, p, n, precision, leaves, all affine): a forest of
// a shape already timed in this process takes the earlier choice.
// DGF_ZCHUNK fixes the chunk length, DGF_STAGE_KERNEL=classic|pair the kernel.
std::mutex g_tune_mutex;
struct TuneChoice {
  int zchunk, kernel;
  bool grid_items;
};
std::map<std::vector<long long>, TuneChoice> g_tune_cache;

dgf_status autotune(dgf_forest* f) {
  f->tuned = true;
  if (f->d != 3 || f->slots <= 0) return DGF_OK;
  const std::vector<long long> key = {f->device, f->d, f->p, f->n, f->precision, (long long)f->nL, f->all_affine};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      if (!getenv("DGF_ZCHUNK")) f->zchunk = it->second.zchunk;
      if (!getenv("DGF_STAGE_KERNEL")) f->kernel = it->second.kernel;
      f->grid_items = grid_env(it->second.grid_items);
      f->slots = f->slots_k[f->kernel];
      return DGF_OK;
    }
  }
  dgf_status st = cuda_check(split_state(f), "split");
  if (!st) st = cuda_check(do_guard(f, guard_args(f, 0, f->gtr.ptr, 1)), "guard");
  if (st) return st;
  std::vector<int> kernels;
  const char* ks = getenv("DGF_STAGE_KERNEL");
  // the cell-pair kernel is a candidate only where it applies (distinct
  // slots), its five-CTA shape at p = 1; DGF_STAGE_KERNEL=pair|pair5|classic
  // keeps one
  const bool any = ks == nullptr;
  if ((any || strcmp(ks, "pair") == 0) && pair_applies(f) && f->slots_k[0] > 0) kernels.push_back(0);
  if ((any || strcmp(ks, "pair5") == 0) && f->slots_k[2] > 0) kernels.push_back(2);
  if (any || strcmp(ks, "classic") == 0 || kernels.empty()) kernels.push_back(1);
  std::vector<int> zs;
  if (getenv("DGF_ZCHUNK")) zs.push_back(f->zchunk);
  else
    for (int z = f->n; z >= 1; z /= 2) zs.push_back(z);
  std::vector<int> grids;  // 0 persistent CTAs, 1 one CTA per work item
  if (getenv("DGF_STAGE_GRID")) grids.push_back(grid_env(false) ? 1 : 0);
  else grids = {0, 1};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int best_z = f->zchunk, best_k = f->kernel;
  bool best_g = f->grid_items;
  float best = 1e30f;
  for (int kk : kernels) {
    f->kernel = kk;
    f->slots = f->slots_k[kk];
    for (int gm : grids)
    for (int z : zs) {
      f->zchunk = z;
      f->grid_items = gm != 0;
      float t[3];
      for (int r = 0; r < 4; ++r) {
        cudaEventRecord(a, f->stream);
        cudaError_t e = do_stage(f, stage_args(f, 0, 1, 0.0, 1.0, 1, 0));
        cudaEventRecord(b, f->stream);
        if (e != cudaSuccess) {
          cudaEventDestroy(a);
          cudaEventDestroy(b);
          return cuda_check(e, "autotune");
        }
        cudaEventSynchronize(b);
        if (r > 0) cudaEventElapsedTime(&t[r - 1], a, b);  // first launch warms up
      }
      std::sort(t, t + 3);
      // k_stage must beat the cell-pair kernel by 2 % to be chosen, so that
      // timing noise does not flip the choice (the kernels round differently)
      const float tt = kk == 1 && !kernels.empty() && kernels[0] == 0 ? t[1] * 1.02f : t[1];
      if (tt < best) {
        best = tt;
        best_z = z;
        best_k = kk;
        best_g = gm != 0;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  f->zchunk = best_z;
  f->kernel = best_k;
  f->grid_items = best_g;
  f->slots = f->slots_k[best_k];
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = {best_z, best_k, best_g};
  return DGF_OK;
}

// enqueue one time increment; timing mode records events around kernels
dgf_status enqueue_step(dgf_forest* f) {
  DevScalars* s = (DevScalars*)f->scal.ptr;
  // kernels one call launches: the guard call adds the mortar passes
  const int guard_kernels = 1 + (f->mortar && f->nmf > 0) + (f->mortar && f->nmc > 0);
  auto rec = [&](int cls, auto&& launch, int kernels = 1) -> dgf_status {
    cudaEvent_t a = nullptr, b = nullptr;
    if (f->timing) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, f->stream);
    }
    cudaError_t e = launch();
    if (f->timing) {
      cudaEventRecord(b, f->stream);
      f->ev.push_back({a, b, cls});
      f->launches[cls] += kernels;
    }
    return cuda_check(e, cls == 0 ? "dt" : (cls == 1 ? "guard" : "stage"));
  };
  dgf_status st = rec(0, [&]() {
    k_dt<<<1, 1, 0, f->stream>>>(s, f->cfl);
    return cudaGetLastError();
  });
  if (st) return st;
  if (f->comp && (st = rec(0, [&]() { return split_state(f); }))) return st;
  // Shu-Osher SSP-RK3: (src, dst, a, b): dst = a U^n + b (src + dt L(src)).
  // Compensated form: U[1], U[2] hold the FP32 increments delta^(1), delta^(2)
  // (delta^(k+1) = b (delta^(k) + dt L)), the last stage writes u^(n+1) in FP64.
  const int src[3] = {0, 1, 2}, dst[3] = {1, 2, 0};
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int k = 0; k < 3; ++k) {
    if ((st = rec(1, [&]() { return do_guard(f, guard_args(f, src[k], f->gtr.ptr, 1)); }, guard_kernels)))
      return st;
    if ((st = rec(2, [&]() { return do_stage(f, stage_args(f, src[k], dst[k], ca[k], cb[k], 0, k == 2)); })))
      return st;
    if (f->limiter > 0.0 && (st = rec(1, [&]() { return do_limit(f, f->U[dst[k]].ptr); }))) return st;
  }
  return DGF_OK;
}

dgf_status set_t_end(dgf_forest* f, double t_end) {
  if (f->t_end_dev == t_end) return DGF_OK;
  DevScalars* s = (DevScalars*)f->scal.ptr;
  f->t_end_dev = t_end;
  // a kernel argument, not a copy from host memory: stream-ordered, and no
  // host value has to outlive the call
  k_set_t_end<<<1, 1, 0, f->stream>>>(s, t_end);
  return cuda_check(cudaGetLastError(), "t_end");
}

dgf_status copy_state(dgf_forest* f, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  dgf_status st = cuda_check(cudaMemcpyAsync(dst, src, bytes, kind, f->stream), "state copy");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(f->stream), "sync");
}

}  // namespace

// =================================================================== ABI
extern "C" {

const char* dgf_last_error(void) { return g_err.c_str(); }

dgf_status dgf_forest_create(const dgf_forest_desc* desc, const dgf_allocator* allocator, dgf_forest** out) {
  if (!desc || !out) return fail(DGF_EINVAL, "null argument");
  *out = nullptr;
  if (desc->precision != DGF_FP64 && desc->precision != DGF_FP32 && desc->precision != DGF_FP32_COMP)
    return fail(DGF_EINVAL, "bad precision");
  if (!(desc->gamma > 1.0) || !(desc->cfl > 0.0)) return fail(DGF_EINVAL, "gamma must be > 1 and cfl > 0");
  if ((desc->nonconforming != DGF_NC_PAPER && desc->nonconforming != DGF_NC_MORTAR) || desc->reserved != 0)
    return fail(DGF_EINVAL, "nonconforming must be DGF_NC_PAPER or DGF_NC_MORTAR (reserved 0)");
  dgf_forest* f = new (std::nothrow) dgf_forest();
  if (!f) return fail(DGF_ENOMEM, "host allocation failed");
  if (!f->host.init(desc->dim, desc->n_seg, desc->p, desc->n_nodes, desc->nodes, desc->n_roots,
                    desc->root_corners, desc->root_cell_nodes, desc->n_periodic, desc->periodic)) {
    std::string e = f->host.error;
    delete f;
    return fail(DGF_EINVAL, e);
  }
  f->precision = desc->precision;
  f->device = desc->device;
  f->gamma = desc->gamma;
  f->cfl = desc->cfl;
  f->esize = desc->precision == DGF_FP64 ? 8 : 4;
  f->sesize = desc->precision == DGF_FP32 ? 4 : 8;
  f->comp = desc->precision == DGF_FP32_COMP;
  f->mortar = desc->nonconforming == DGF_NC_MORTAR;
  f->d = desc->dim;
  f->n = desc->n_seg;
  f->p = desc->p;
  f->N = f->p + 1;
  f->nv = f->d + 2;
  f->M = (int)std::pow(f->N, f->d);
  f->nc = (int)std::pow(f->n, f->d);
  f->NG = ((1 << f->d) - 1) * f->d;
  f->nt = (int)std::pow(f->n, f->d - 1);
  f->NFP = (int)std::pow(f->N, f->d - 1);
  f->basis.build(f->N);
  RtTables& T = f->tab;
  T.N = f->N;
  for (int i = 0; i < f->N; ++i) {
    T.x[i] = f->basis.x[i];
    T.w[i] = f->basis.w[i];
    T.lp[i] = f->basis.lp[i];
    T.lm[i] = f->basis.lm[i];
  }
  for (int i = 0; i < f->N * f->N; ++i) {
    T.V[i] = f->basis.V[i];
    T.Vi[i] = f->basis.Vi[i];
    T.Sh[i] = f->basis.Sh[i];
    T.Sm[i] = f->basis.Sm[i];
    T.Sp[i] = f->basis.Sp[i];
    T.Snm[i] = f->basis.Snm[i];
    T.Snp[i] = f->basis.Snp[i];
  }
  if (allocator) {
    f->alloc = *allocator;
    f->has_alloc = allocator->alloc && allocator->free;
  }
  if (f->device >= 0 && f->n != 2 && f->n != 4 && f->n != 8) {
    delete f;
    return fail(DGF_EUNSUPPORTED, "the device kernels are instantiated for n_seg in {2, 4, 8}");
  }
  if (f->device >= 0) {
    DeviceGuard dg(f->device);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || f->device >= ndev) {
      delete f;
      return fail(DGF_ECUDA, "no such CUDA device");
    }
    if (cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete f;
      return fail(DGF_ECUDA, "stream creation failed");
    }
    f->own_stream = true;
    if (!ensure(f, f->scal, sizeof(DevScalars)) || !ensure(f, f->tot, 8 * sizeof(double)) ||
        !ensure(f, f->dtout, sizeof(double))) {
      dgf_forest_destroy(f);
      return fail(DGF_ENOMEM, "device allocation failed");
    }
    f->t_end_dev = INFINITY;
    // initialised by a kernel on the forest's stream (a cudaMemcpy from host
    // memory would run on the legacy stream, which the forest's non-blocking
    // stream is not ordered against, and may land after its first kernels)
    k_init_scalars<<<1, 1, 0, f->stream>>>((DevScalars*)f->scal.ptr);
    if (cudaGetLastError() != cudaSuccess) {
      dgf_forest_destroy(f);
      return fail(DGF_ECUDA, "device scalars");
    }
  }
  dgf_status st = build_device(f);
  if (st) {
    std::string e = g_err;
    dgf_forest_destroy(f);
    return fail(st, e);
  }
  if (f->device >= 0) {
    DeviceGuard dg(f->device);
    if ((st = cuda_check(cudaStreamSynchronize(f->stream), "create"))) {
      dgf_forest_destroy(f);
      return st;
    }
  }
  *out = f;
  return DGF_OK;
}

dgf_status dgf_forest_destroy(dgf_forest* f) {
  if (!f) return DGF_OK;
  if (f->device >= 0) {
    DeviceGuard dg(f->device);
    cudaStreamSynchronize(f->stream);
    if (f->graph) cudaGraphExecDestroy(f->graph);
    if (f->graph_alt) cudaGraphExecDestroy(f->graph_alt);
    for (auto& e : f->ev) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    dgf_forest::Buf* bufs[] = {&f->U[0], &f->U[1], &f->U[2], &f->geo, &f->geo64, &f->hcell, &f->gtr,
                               &f->gmod, &f->cop, &f->ctr, &f->kind, &f->nbr, &f->orient, &f->qbits, &f->copoff,
                               &f->part, &f->scal, &f->tot, &f->dtout, &f->nodal, &f->fine, &f->affine, &f->ameta,
                               &f->U64[0], &f->U64[1], &f->hcell64, &f->gmod64, &f->Uhi, &f->Ulo, &f->fluxmask,
                               &f->mfine, &f->mcoarse, &f->mw, &f->msrc, &f->ind, &f->bstate, &f->trd};
    for (auto* b : bufs) dev_free(f, *b);
    if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
  }
  delete f;
  return DGF_OK;
}

dgf_status dgf_set_stream(dgf_forest* f, void* stream) {
  if (dgf_status st = require_device(f)) return st;
  DeviceGuard dg(f->device);
  cudaStreamSynchronize(f->stream);
  if (f->own_stream) cudaStreamDestroy(f->stream);
  f->own_stream = false;
  f->stream = (cudaStream_t)stream;
  if (f->graph) cudaGraphExecDestroy(f->graph);
  if (f->graph_alt) cudaGraphExecDestroy(f->graph_alt);
  f->graph = nullptr;
  f->graph_alt = nullptr;
  f->graph_valid = false;
  return DGF_OK;
}

static dgf_status regrid(dgf_forest* f, const std::vector<uint64_t>& old_leaves);

dgf_status dgf_block_refine(dgf_forest* f, const int64_t* ids, int64_t n) {
  if (!f || (n > 0 && !ids)) return fail(DGF_EINVAL, "null argument");
  std::vector<uint64_t> keys;
  for (int64_t i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= f->host.n_leaves()) return fail(DGF_EINVAL, "leaf id out of range");
    keys.push_back(f->host.leaves[ids[i]]);
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  std::vector<uint64_t> old = f->host.leaves;
  auto saved = f->host.tree;
  if (!f->host.refine(keys)) {
    f->host.tree = saved;
    f->host.order_leaves();
    return fail(DGF_EINVAL, f->host.error);
  }
  return regrid(f, old);
}

dgf_status dgf_block_coarsen(dgf_forest* f, const int64_t* ids, int64_t n) {
  if (!f || (n > 0 && !ids)) return fail(DGF_EINVAL, "null argument");
  std::vector<uint64_t> parents;
  for (int64_t i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= f->host.n_leaves()) return fail(DGF_EINVAL, "leaf id out of range");
    int64_t r;
    int lev, pos[3];
    Forest::unkey(f->host.leaves[ids[i]], &r, &lev, pos);
    if (lev <= 1) return fail(DGF_EINVAL, "a root block has no parent");
    int pp[3] = {pos[0] >> 1, pos[1] >> 1, pos[2] >> 1};
    parents.push_back(Forest::key(r, lev - 1, pp));
  }
  std::sort(parents.begin(), parents.end());
  parents.erase(std::unique(parents.begin(), parents.end()), parents.end());
  std::vector<uint64_t> old = f->host.leaves;
  bool viol = false;
  if (!f->host.coarsen(parents, &viol)) return fail(DGF_EBALANCE, f->host.error);
  return regrid(f, old);
}

// per-leaf refinement indicator into host memory (synchronises)
static dgf_status indicator_host(dgf_forest* f, std::vector<double>& g) {
  if (dgf_status st = require_device(f)) return st;
  if (!f->have_state) return fail(DGF_ESTATE, "no state set");
  DeviceGuard dg(f->device);
  const int64_t L = f->nL;
  dgf_forest::Buf& gb = f->ind;
  if (!ensure(f, gb, sizeof(unsigned long long) * std::max<int64_t>(L, 1)))
    return fail(DGF_ENOMEM, "device allocation failed");
  dgf_status st = cuda_check(cudaMemsetAsync(gb.ptr, 0, sizeof(unsigned long long) * L, f->stream), "memset");
  RtMisc r = misc_args(f, 0);
  r.gmax = (unsigned long long*)gb.ptr;
  if (!st) st = cuda_check(do_indicator(f, r), "indicator");
  g.assign(L, 0.0);
  if (!st) st = copy_state(f, g.data(), gb.ptr, sizeof(double) * L, cudaMemcpyDeviceToHost);
  return st;
}

dgf_status dgf_indicator(dgf_forest* f, double* out) {
  if (!f || !out) return fail(DGF_EINVAL, "null argument");
  std::vector<double> g;
  dgf_status st = indicator_host(f, g);
  if (st) return st;
  std::memcpy(out, g.data(), sizeof(double) * g.size());
  return DGF_OK;
}

dgf_status dgf_adapt_with(dgf_forest* f, const double* g, double refine_above, double coarsen_below,
                          int32_t max_level, int64_t* n_refined, int64_t* n_coarsened) {
  if (!f || !g) return fail(DGF_EINVAL, "null argument");
  if (max_level < 1 || max_level > 12) return fail(DGF_EINVAL, "max_level must be in [1, 12]");
  const int64_t L = f->host.n_leaves();
  for (int64_t i = 0; i < L; ++i)
    if (std::isnan(g[i])) return fail(DGF_ENONFINITE, "indicator: non-positive mean density or NaN");
  std::vector<uint64_t> refine_keys, low;
  for (int64_t i = 0; i < L; ++i) {
    const uint64_t k = f->host.leaves[i];
    int64_t r;
    int lev, pos[3];
    Forest::unkey(k, &r, &lev, pos);
    if (g[i] > refine_above && lev < max_level) refine_keys.push_back(k);
    if (g[i] < coarsen_below) low.push_back(k);
  }
  std::sort(low.begin(), low.end());
  std::vector<uint64_t> old = f->host.leaves;
  const int64_t nc = f->host.adapt(refine_keys, low);
  if (n_refined) *n_refined = (int64_t)refine_keys.size();
  if (n_coarsened) *n_coarsened = nc;
  if (refine_keys.empty() && nc == 0) return DGF_OK;
  return regrid(f, old);
}

dgf_status dgf_adapt(dgf_forest* f, double refine_above, double coarsen_below, int32_t max_level,
                     int64_t* n_refined, int64_t* n_coarsened) {
  if (!f) return fail(DGF_EINVAL, "null argument");
  if (max_level < 1 || max_level > 12) return fail(DGF_EINVAL, "max_level must be in [1, 12]");
  std::vector<double> g;
  dgf_status st = indicator_host(f, g);
  if (st) return st;
  return dgf_adapt_with(f, g.data(), refine_above, coarsen_below, max_level, n_refined, n_coarsened);
}

dgf_status dgf_set_boundary(dgf_forest* f, const int32_t* root_face_kind, const double* state) {
  if (!f || !root_face_kind || !state) return fail(DGF_EINVAL, "null argument");
  const int nf = 2 * f->d;
  std::vector<int32_t> tags(root_face_kind, root_face_kind + f->host.R * nf);
  for (int32_t t : tags)
    if (t != 0 && t != 1) return fail(DGF_EINVAL, "boundary kinds must be 0 (outflow) or 1 (prescribed state)");
  for (int v = 0; v < f->nv; ++v)
    if (!std::isfinite(state[v])) return fail(DGF_EINVAL, "non-finite boundary state");
  f->bctag = tags;
  f->bstate_h.assign(state, state + f->nv);
  return build_device(f);
}

dgf_status dgf_leaf_count(const dgf_forest* f, int64_t* n) {
  if (!f || !n) return fail(DGF_EINVAL, "null argument");
  *n = f->host.n_leaves();
  return DGF_OK;
}

dgf_status dgf_leaf_table(const dgf_forest* f, int32_t* root, int32_t* level, int32_t* pos, int32_t* kind,
                          int64_t* nbr, int32_t* orient) {
  if (!f) return fail(DGF_EINVAL, "null forest");
  Forest::Tables T = f->host.tables();
  if (root) std::memcpy(root, T.root.data(), T.root.size() * sizeof(int32_t));
  if (level) std::memcpy(level, T.level.data(), T.level.size() * sizeof(int32_t));
  if (pos) std::memcpy(pos, T.pos.data(), T.pos.size() * sizeof(int32_t));
  if (kind) std::memcpy(kind, T.kind.data(), T.kind.size() * sizeof(int32_t));
  if (nbr) std::memcpy(nbr, T.nbr.data(), T.nbr.size() * sizeof(int64_t));
  if (orient) std::memcpy(orient, T.orient.data(), T.orient.size() * sizeof(int32_t));
  return DGF_OK;
}

dgf_status dgf_quad_points(const dgf_forest* fc, double* xyz) {
  if (!fc || !xyz) return fail(DGF_EINVAL, "null argument");
  dgf_forest* f = const_cast<dgf_forest*>(fc);
  const int d = f->d, M = f->M, nc = f->nc, N = f->N;
  std::vector<double> coef;
  for (int64_t i = 0; i < f->host.n_leaves(); ++i) {
    f->host.cell_coefficients(f->host.leaves[i], coef);
    for (int c = 0; c < nc; ++c) {
      double cc[8 * 3];
      for (int k = 0; k < (1 << d) * d; ++k) cc[k] = coef[(size_t)k * nc + c];
      for (int q = 0; q < M; ++q) {
        double xi[3], A[9];
        int r = q;
        for (int a = 0; a < d; ++a) {
          xi[a] = f->basis.x[r % N];
          r /= N;
        }
        eval_map(d, cc, xi, &xyz[(((size_t)i * nc + c) * M + q) * d], A);
      }
    }
  }
  return DGF_OK;
}

dgf_status dgf_state_size(const dgf_forest* f, int64_t* n) {
  if (!f || !n) return fail(DGF_EINVAL, "null argument");
  *n = f->host.n_leaves() * f->nv * f->M * f->nc;
  return DGF_OK;
}

dgf_status dgf_set_state(dgf_forest* f, const void* src, int is_device) {
  if (dgf_status st = require_device(f)) return st;
  if (!src) return fail(DGF_EINVAL, "null source");
  DeviceGuard dg(f->device);
  const size_t bytes = (size_t)f->nL * f->nv * f->M * f->nc * f->sesize;
  void* U = state_ptr(f);
  dgf_status st = cuda_check(
      cudaMemcpyAsync(U, src, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, f->stream),
      "set_state");
  if (st) return st;
  // a host source is read by the copy engine possibly after the copy call
  // returns: wait before the caller may release it
  if (!is_device && (st = cuda_check(cudaStreamSynchronize(f->stream), "set_state"))) return st;
  // the device holds values at the Gauss points: u = V K per (leaf, var, cell)
  if ((st = cuda_check(do_convert(f, U, (size_t)f->nL, f->nc, 1, state_f64(f)), "to nodal"))) return st;
  f->have_state = true;
  return init_lambda(f);
}

dgf_status dgf_get_state(dgf_forest* f, void* dst, int is_device) {
  if (dgf_status st = require_device(f)) return st;
  if (!dst) return fail(DGF_EINVAL, "null destination");
  if (!f->have_state) return fail(DGF_ESTATE, "no state set");
  DeviceGuard dg(f->device);
  const size_t bytes = (size_t)f->nL * f->nv * f->M * f->nc * f->sesize;
  void* tmp = f->comp ? f->U64[1 - f->cur].ptr : f->U[1].ptr;  // free between time steps
  dgf_status st = cuda_check(cudaMemcpyAsync(tmp, state_ptr(f), bytes, cudaMemcpyDeviceToDevice, f->stream),
                             "get_state");
  if (st) return st;
  if ((st = cuda_check(do_convert(f, tmp, (size_t)f->nL, f->nc, 0, state_f64(f)), "to modal"))) return st;
  return copy_state(f, dst, tmp, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
}

dgf_status dgf_set_state_nodal(dgf_forest* f, const double* vals, int is_device) {
  if (dgf_status st = require_device(f)) return st;
  if (!vals) return fail(DGF_EINVAL, "null source");
  DeviceGuard dg(f->device);
  const size_t bytes = (size_t)f->nL * f->nc * f->M * f->nv * sizeof(double);
  const double* src = vals;
  dgf_status st;
  if (!is_device) {
    if (!ensure(f, f->nodal, bytes)) return fail(DGF_ENOMEM, "scratch allocation failed");
    if ((st = cuda_check(cudaMemcpyAsync(f->nodal.ptr, vals, bytes, cudaMemcpyHostToDevice, f->stream), "copy")))
      return st;
    src = (const double*)f->nodal.ptr;
  }
  RtMisc r = misc_args(f, 0);
  r.vals = src;
  if ((st = cuda_check(do_project(f, r), "project"))) return st;
  f->have_state = true;
  if ((st = init_lambda(f))) return st;
  return cuda_check(cudaStreamSynchronize(f->stream), "sync");
}

dgf_status dgf_fill_guardcells(dgf_forest* f, void* guard, int is_device) {
  if (dgf_status st = require_device(f)) return st;
  if (!guard) return fail(DGF_EINVAL, "null destination");
  if (!f->have_state) return fail(DGF_ESTATE, "no state set");
  DeviceGuard dg(f->device);
  const size_t count = (size_t)f->nL * 2 * f->d * f->nv * f->M * f->nt;
  if (!ensure(f, f->gmod, count * f->esize)) return fail(DGF_ENOMEM, "guard allocation failed");
  dgf_status st = cuda_check(split_state(f), "split");
  if (!st) st = cuda_check(do_guard(f, guard_args(f, 0, f->gmod.ptr, 0)), "guard");
  if (st) return st;
  const bool dbl = f->precision == DGF_FP64;
  if ((st = cuda_check(do_convert(f, f->gmod.ptr, (size_t)f->nL * 2 * f->d, f->nt, 0, dbl), "to modal"))) return st;
  const void* out = f->gmod.ptr;
  if (f->comp) {
    if (!ensure(f, f->gmod64, count * sizeof(double))) return fail(DGF_ENOMEM, "guard allocation failed");
    if ((st = widen(f, f->gmod.ptr, f->gmod64.ptr, count))) return st;
    out = f->gmod64.ptr;
  }
  return copy_state(f, guard, out, count * f->sesize, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
}

dgf_status dgf_dg_residual(dgf_forest* f, void* dst, int is_device) {
  if (dgf_status st = require_device(f)) return st;
  if (!dst) return fail(DGF_EINVAL, "null destination");
  if (!f->have_state) return fail(DGF_ESTATE, "no state set");
  DeviceGuard dg(f->device);
  dgf_status st = cuda_check(split_state(f), "split");
  if (!st) st = cuda_check(do_guard(f, guard_args(f, 0, f->gtr.ptr, 1)), "guard");
  if (st) return st;
  if ((st = cuda_check(do_stage(f, stage_args(f, 0, 1, 0.0, 1.0, 1, 0)), "stage"))) return st;
  const bool dbl = f->precision == DGF_FP64;
  if ((st = cuda_check(do_convert(f, f->U[1].ptr, (size_t)f->nL, f->nc, 0, dbl), "to modal"))) return st;
  const size_t count = (size_t)f->nL * f->nv * f->M * f->nc;
  const void* out = f->U[1].ptr;
  if (f->comp) {
    if ((st = widen(f, f->U[1].ptr, f->U64[1 - f->cur].ptr, count))) return st;
    out = f->U64[1 - f->cur].ptr;
  }
  return copy_state(f, dst, out, count * f->sesize, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
}

dgf_status dgf_rk_step(dgf_forest* f, double t_end, double* dt_out) {
  if (dgf_status st = require_device(f)) return st;
  if (!f->have_state) return fail(DGF_ESTATE, "no state set");
  DeviceGuard dg(f->device);
  dgf_status st = set_t_end(f, t_end);
  if (st) return st;
  if (!f->tuned && (st = autotune(f))) return st;
  if (f->timing) {
    if ((st = enqueue_step(f))) return st;
  } else {
    // one graph per time increment (two for the compensated form, one per u^n buffer)
    cudaGraphExec_t& G = (f->comp && f->cur == 1) ? f->graph_alt : f->graph;
    if (!G) {
      cudaGraph_t g = nullptr;
      if ((st = cuda_check(cudaStreamBeginCapture(f->stream, cudaStreamCaptureModeThreadLocal), "capture")))
        return st;
      dgf_status est = enqueue_step(f);
      cudaError_t e = cudaStreamEndCapture(f->stream, &g);
      if (est) {
        if (g) cudaGraphDestroy(g);
        return est;
      }
      if ((st = cuda_check(e, "end capture"))) return st;
      e = cudaGraphInstantiate(&G, g, 0);
      cudaGraphDestroy(g);
      if ((st = cuda_check(e, "instantiate"))) return st;
      f->graph_valid = true;
    }
    if ((st = cuda_check(cudaGraphLaunch(G, f->stream), "graph launch"))) return st;
  }
  if (f->comp) f->cur ^= 1;  // u^(n+1) was written to the other FP64 buffer
  if (dt_out) {
    DevScalars* s = (DevScalars*)f->scal.ptr;
    if ((st = cuda_check(cudaMemcpyAsync(dt_out, &s->dt, sizeof(double), cudaMemcpyDeviceToHost, f->stream), "dt")))
      return st;
    return cuda_check(cudaStreamSynchronize(f->stream), "sync");
  }
  return DGF_OK;
}

dgf_status dgf_get_time(dgf_forest* f, double* t) {
  if (dgf_status st = require_device(f)) return st;
  if (!t) return fail(DGF_EINVAL, "null argument");
  DeviceGuard dg(f->device);
  DevScalars* s = (DevScalars*)f->scal.ptr;
  return copy_state(f, t, &s->t, sizeof(double), cudaMemcpyDeviceToHost);
}

dgf_status dgf_set_time(dgf_forest* f, double t) {
  if (dgf_status st = require_device(f)) return st;
  DeviceGuard dg(f->device);
  k_set_time<<<1, 1, 0, f->stream>>>((DevScalars*)f->scal.ptr, t);
  dgf_status st = cuda_check(cudaGetLastError(), "set_time");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(f->stream), "set_time");
}

dgf_status dgf_step_count(dgf_forest* f, int64_t* steps) {
  if (dgf_status st = require_device(f)) return st;
  if (!steps) return fail(DGF_EINVAL, "null argument");
  DeviceGuard dg(f->device);
  DevScalars* s = (DevScalars*)f->scal.ptr;
  int v = 0;
  dgf_status st = copy_state(f, &v, &s->steps, sizeof(int), cudaMemcpyDeviceToHost);
  *steps = v;
  return st;
}

dgf_status dgf_compute_dt(dgf_forest* f, double* dt) {
  if (dgf_status st = require_device(f)) return st;
  if (!dt) return fail(DGF_EINVAL, "null argument");
  if (!f->have_state) return fail(DGF_ESTATE, "no state set");
  DeviceGuard dg(f->device);
  dgf_status st = init_lambda(f);
  if (st) return st;
  DevScalars* s = (DevScalars*)f->scal.ptr;
  k_dt_only<<<1, 1, 0, f->stream>>>(s, f->cfl, (double*)f->dtout.ptr);
  if ((st = cuda_check(cudaGetLastError(), "dt"))) return st;
  return copy_state(f, dt, f->dtout.ptr, sizeof(double), cudaMemcpyDeviceToHost);
}

dgf_status dgf_conserved_totals(dgf_forest* f, double* totals) {
  if (dgf_status st = require_device(f)) return st;
  if (!totals) return fail(DGF_EINVAL, "null argument");
  if (!f->have_state) return fail(DGF_ESTATE, "no state set");
  DeviceGuard dg(f->device);
  dgf_status st = cuda_check(do_totals(f, misc_args(f, 0)), "totals");
  if (st) return st;
  k_reduce<<<f->nv, 1024, 0, f->stream>>>((const double*)f->part.ptr, (size_t)f->nL * f->nc, (double*)f->tot.ptr);
  if ((st = cuda_check(cudaGetLastError(), "reduce"))) return st;
  return copy_state(f, totals, f->tot.ptr, f->nv * sizeof(double), cudaMemcpyDeviceToHost);
}

dgf_status dgf_status_word(dgf_forest* f, int32_t* status, int reset) {
  if (dgf_status st = require_device(f)) return st;
  if (!status) return fail(DGF_EINVAL, "null argument");
  DeviceGuard dg(f->device);
  DevScalars* s = (DevScalars*)f->scal.ptr;
  int v = 0;
  dgf_status st = copy_state(f, &v, &s->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (st) return st;
  *status = v;
  if (reset) {
    int z = 0;
    return copy_state(f, &s->status, &z, sizeof(int), cudaMemcpyHostToDevice);
  }
  return DGF_OK;
}

dgf_status dgf_tuning(const dgf_forest* f, int32_t* zchunk, int32_t* resident_ctas) {
  if (!f) return fail(DGF_EINVAL, "null forest");
  if (zchunk) *zchunk = f->zchunk;
  if (resident_ctas) *resident_ctas = f->slots;
  return DGF_OK;
}

dgf_status dgf_stage_kernel(const dgf_forest* f, int32_t* kernel) {
  if (!f || !kernel) return fail(DGF_EINVAL, "null argument");
  *kernel = f->kernel;
  return DGF_OK;
}

dgf_status dgf_stage_grid(const dgf_forest* f, int32_t* per_item) {
  if (!f || !per_item) return fail(DGF_EINVAL, "null argument");
  *per_item = f->grid_items ? 1 : 0;
  return DGF_OK;
}

dgf_status dgf_set_limiter(dgf_forest* f, double eps) {
  if (dgf_status st = require_device(f)) return st;
  if (f->comp && eps > 0.0) return fail(DGF_EUNSUPPORTED, "the limiter is not available for DGF_FP32_COMP");
  if (!(eps >= 0.0 && eps < 1.0)) return fail(DGF_EINVAL, "eps must be in [0, 1)");
  DeviceGuard dg(f->device);
  cudaStreamSynchronize(f->stream);
  f->limiter = eps;
  if (f->graph) cudaGraphExecDestroy(f->graph);
  if (f->graph_alt) cudaGraphExecDestroy(f->graph_alt);
  f->graph = f->graph_alt = nullptr;
  f->graph_valid = false;
  return DGF_OK;
}

dgf_status dgf_limit(dgf_forest* f) {
  if (dgf_status st = require_device(f)) return st;
  if (!f->have_state) return fail(DGF_ESTATE, "no state set");
  if (!(f->limiter > 0.0)) return fail(DGF_ESTATE, "no limiter set (dgf_set_limiter)");
  DeviceGuard dg(f->device);
  dgf_status st = cuda_check(do_limit(f, f->U[0].ptr), "limit");
  if (st) return st;
  return init_lambda(f);
}

dgf_status dgf_set_timing(dgf_forest* f, int on) {
  if (dgf_status st = require_device(f)) return st;
  f->timing = on != 0;
  return DGF_OK;
}

dgf_status dgf_kernel_times(dgf_forest* f, double* ms, int64_t* launches, int n_classes) {
  if (dgf_status st = require_device(f)) return st;
  DeviceGuard dg(f->device);
  dgf_status st = cuda_check(cudaStreamSynchronize(f->stream), "sync");
  if (st) return st;
  for (auto& e : f->ev) {
    float m = 0.f;
    cudaEventElapsedTime(&m, e.a, e.b);
    f->ms[e.cls] += m;
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  f->ev.clear();
  for (int c = 0; c < n_classes && c < 3; ++c) {
    if (ms) ms[c] = f->ms[c];
    if (launches) launches[c] = f->launches[c];
    f->ms[c] = 0;
    f->launches[c] = 0;
  }
  return DGF_OK;
}

}  // extern "C"

// ------------------------------------------------------------- regrid
// Nodal combine operator of one parent cell (Eqs. (13)-(14), reading R6):
// u_P(x_q) = sum_e sum_k op[q][e Q + k] u_e(x_k), the J-weighted L2
// projection onto the parent cell's polynomials of its 2^d children, every
// integral by the child's own Gauss rule, evaluated at the parent's points.
static bool combine_op_cell(dgf_forest* f, const double* const* child_coef, double* op) {
  const int d = f->d, N = f->N, M = f->M, NW = 1 << d, KC = NW * M;
  const Basis1D& B = f->basis;
  std::vector<double> MP((size_t)M * M, 0.0), R((size_t)M * KC, 0.0);
  for (int e = 0; e < NW; ++e) {
    for (int q = 0; q < M; ++q) {
      double xi[3], xp[3], wq = 1.0;
      int rq = q;
      for (int a = 0; a < d; ++a) {
        xi[a] = B.x[rq % N];
        wq *= B.w[rq % N];
        xp[a] = 0.5 * (xi[a] + (((e >> a) & 1) ? 1.0 : -1.0));
        rq /= N;
      }
      double A[9], Ja[9];
      eval_map(d, child_coef[e], xi, nullptr, A);
      const double wj = wq * det_and_cofactor(d, A, Ja);
      double ph[64];
      for (int m = 0; m < M; ++m) ph[m] = phi(B, d, m, xp);
      for (int m = 0; m < M; ++m) {
        for (int m2 = 0; m2 < M; ++m2) MP[(size_t)m * M + m2] += wj * ph[m] * ph[m2];
        R[(size_t)m * KC + e * M + q] += wj * ph[m];
      }
    }
  }
  if (!chol_solve(M, MP, R, KC)) return false;
  for (int q = 0; q < M; ++q) {
    double xq[3];
    for (int a = 0, rq = q; a < d; ++a, rq /= N) xq[a] = B.x[rq % N];
    double ph[64];
    for (int m = 0; m < M; ++m) ph[m] = phi(B, d, m, xq);
    for (int k = 0; k < KC; ++k) {
      double acc = 0.0;
      for (int m = 0; m < M; ++m) acc += ph[m] * R[(size_t)m * KC + k];
      op[(size_t)q * KC + k] = acc;
    }
  }
  return true;
}

// New leaves get their state from the old ones on the device: copies,
// splits (Eqs. (11)-(12)) or combines (Eqs. (13)-(14)), Sec. 3.4; the old
// state buffer is kept until the transfer kernel has run.
static dgf_status regrid(dgf_forest* f, const std::vector<uint64_t>& old_leaves) {
  const bool carry = f->device >= 0 && f->have_state;
  if (!carry) return build_device(f);
  const int d = f->d, n = f->n, N = f->N, M = f->M, nc = f->nc, NW = 1 << d;
  DeviceGuard dg(f->device);
  cudaStreamSynchronize(f->stream);
  dgf_forest::Buf old;
  dgf_forest::Buf& live = f->comp ? f->U64[f->cur] : f->U[0];
  old = live;
  live = dgf_forest::Buf();
  const bool was_tuned = f->tuned;
  const int tuned_z = f->zchunk, tuned_k = f->kernel;
  const bool tuned_g = f->grid_items;
  dgf_status st = build_device(f);
  if (was_tuned && f->d == 3) {
    // a regrid keeps the tuned stage kernel and chunk length (re-timing every
    // regrid costs more than it gains)
    f->tuned = true;
    if (!getenv("DGF_ZCHUNK")) f->zchunk = tuned_z;
    f->grid_items = grid_env(tuned_g);
    if (!getenv("DGF_STAGE_KERNEL")) {
      f->kernel = tuned_k;
      f->slots = f->slots_k[tuned_k];
    }
  }
  if (st) {
    dev_free(f, old);
    f->have_state = false;
    return st;
  }
  std::unordered_map<uint64_t, int64_t> old_index;
  for (size_t i = 0; i < old_leaves.size(); ++i) old_index[old_leaves[i]] = (int64_t)i;
  const int64_t L = f->host.n_leaves();
  std::vector<int> mode(L, 0), src(L, 0), kids((size_t)L * NW, 0);
  std::vector<long long> opoff(L, 0);  // combine leaves: first entry in cellop
  std::vector<int64_t> combine_leaves;
  for (int64_t i = 0; i < L; ++i) {
    const uint64_t k = f->host.leaves[i];
    auto it = old_index.find(k);
    if (it != old_index.end()) {
      src[i] = (int)it->second;
      continue;
    }
    int64_t r;
    int lev, pos[3];
    Forest::unkey(k, &r, &lev, pos);
    int pp[3] = {pos[0] >> 1, pos[1] >> 1, pos[2] >> 1};
    auto pit = old_index.find(Forest::key(r, lev - 1, pp));
    if (pit != old_index.end()) {
      mode[i] = 1;
      src[i] = (int)pit->second;
      int bits = 0;
      for (int a = 0; a < d; ++a) bits |= (pos[a] & 1) << a;
      kids[(size_t)i * NW] = bits;
      continue;
    }
    mode[i] = 2;
    for (int c = 0; c < NW; ++c) {
      int kp[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) kp[a] = 2 * pos[a] + ((c >> a) & 1);
      auto kt = old_index.find(Forest::key(r, lev + 1, kp));
      if (kt == old_index.end()) {
        dev_free(f, old);
        f->have_state = false;
        return fail(DGF_EINVAL, "regrid: a new block is neither kept, split nor combined");
      }
      kids[(size_t)i * NW + c] = (int)kt->second;
    }
    opoff[i] = (long long)combine_leaves.size() * nc;
    combine_leaves.push_back(i);
  }
  // combine operators (host, FP64): a parent cell whose children all have
  // the same constant Jacobian uses the shared reference operator (stored
  // first); any other cell gets its own
  const size_t opsz = (size_t)M * NW * M;
  std::vector<std::vector<double>> ccoef((size_t)combine_leaves.size() * NW);
  for (size_t j = 0; j < combine_leaves.size(); ++j) {
    int64_t r;
    int lev, pos[3];
    Forest::unkey(f->host.leaves[combine_leaves[j]], &r, &lev, pos);
    for (int c = 0; c < NW; ++c) {
      int kp[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) kp[a] = 2 * pos[a] + ((c >> a) & 1);
      f->host.cell_coefficients(Forest::key(r, lev + 1, kp), ccoef[j * NW + c]);
    }
  }
  const int64_t ncomb = (int64_t)combine_leaves.size() * nc;
  auto child_cells = [&](int64_t jc, double (*cc)[24]) {
    const size_t j = (size_t)(jc / nc);
    const int c = (int)(jc % nc);
    int I[3] = {0, 0, 0};
    for (int a = 0, rr = c; a < d; ++a, rr /= n) I[a] = rr % n;
    for (int e = 0; e < NW; ++e) {
      int cb = 0, cell = 0;
      for (int a = 0, st2 = 1; a < d; ++a, st2 *= n) {
        const int H = 2 * I[a] + ((e >> a) & 1);
        cb |= (H / n) << a;
        cell += (H % n) * st2;
      }
      const std::vector<double>& C = ccoef[j * NW + cb];
      for (int kk = 0; kk < NW * d; ++kk) cc[e][kk] = C[(size_t)kk * nc + cell];
    }
  };
  // which cells need their own operator
  std::vector<unsigned char> own(ncomb, 0);
  parallel_for(ncomb, [&](int64_t jc) {
    double cc[8][24];
    child_cells(jc, cc);
    double J0 = 0.0;
    for (int e = 0; e < NW && !own[jc]; ++e)
      for (int q = 0; q < M; ++q) {
        double xi[3];
        for (int a = 0, rq = q; a < d; ++a, rq /= N) xi[a] = f->basis.x[rq % N];
        double A[9], Ja[9];
        eval_map(d, cc[e], xi, nullptr, A);
        const double J = det_and_cofactor(d, A, Ja);
        if (e == 0 && q == 0) J0 = J;
        if (std::fabs(J - J0) > 1e-12 * std::fabs(J0)) {
          own[jc] = 1;
          break;
        }
      }
  });
  std::vector<long long> cellop(std::max<int64_t>(ncomb, 1), 0);
  size_t nops = ncomb > 0 ? 1 : 0;
  for (int64_t jc = 0; jc < ncomb; ++jc)
    if (own[jc]) cellop[jc] = (long long)(opsz * nops++);
  std::vector<double> ops(opsz * nops, 0.0);
  std::atomic<bool> singular{false};
  if (ncomb > 0) {
    // the reference operator: children of a unit cube cell
    double cc[8][24];
    const double* cp[8];
    for (int e = 0; e < NW; ++e) {
      for (int kk = 0; kk < NW * d; ++kk) cc[e][kk] = 0.0;
      for (int a = 0; a < d; ++a) cc[e][((1 << a)) * d + a] = 0.25;  // x_a = xi_a / 4 (any constant J)
      cp[e] = cc[e];
    }
    if (!combine_op_cell(f, cp, &ops[0])) singular = true;
  }
  parallel_for(ncomb, [&](int64_t jc) {
    if (!own[jc]) return;
    double cc[8][24];
    const double* cp[8];
    child_cells(jc, cc);
    for (int e = 0; e < NW; ++e) cp[e] = cc[e];
    if (!combine_op_cell(f, cp, &ops[(size_t)cellop[jc]])) singular = true;
  });
  if (singular) {
    dev_free(f, old);
    f->have_state = false;
    return fail(DGF_EINVAL, "singular combine mass matrix");
  }
  dgf_forest::Buf bm, bs, bk, bo, bc, bops;
  auto cleanup = [&]() {
    cudaStreamSynchronize(f->stream);
    dgf_forest::Buf* all[] = {&old, &bm, &bs, &bk, &bo, &bc, &bops};
    for (auto* b : all) dev_free(f, *b);
  };
  if ((st = upload(f, bm, mode)) || (st = upload(f, bs, src)) || (st = upload(f, bk, kids)) ||
      (st = upload(f, bo, opoff)) || (st = upload(f, bc, cellop)) ||
      (st = state_f64(f) ? upload(f, bops, ops) : upload(f, bops, convert<float>(ops)))) {
    cleanup();
    f->have_state = false;
    return st;
  }
  RtTransfer tr{};
  tr.p = f->p;
  tr.nL = (int)L;
  tr.n = n;
  tr.old = old.ptr;
  tr.out = state_ptr(f);
  tr.mode = (const int*)bm.ptr;
  tr.src = (const int*)bs.ptr;
  tr.kids = (const int*)bk.ptr;
  tr.opoff = (const long long*)bo.ptr;
  tr.cellop = (const long long*)bc.ptr;
  tr.ops = bops.ptr;
  tr.T = f->tab;
  st = cuda_check(do_transfer(f, tr), "transfer");
  cleanup();
  if (st) {
    f->have_state = false;
    return st;
  }
  return init_lambda(f);
}

// ------------------------------------------------------ residual without allocation
// For callers that cannot allocate device memory once a forest exists (for
// example code running inside a CUDA graph capture, or a host process whose
// memory is handed out by a pool it does not own): the guard traces that
// dgf_dg_residual keeps in forest-owned scratch live here in a file-scope
// device array instead.  The array is part of the library image, so every
// GPU that loads the library holds it until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// address of the scratch array on the current device (set up once per device)
dgf_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return fail(DGF_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[device]) {
    // a device reset since the last call invalidates the cached address:
    // look it up again when the driver no longer knows it as device memory
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, g_noalloc_ptr[device]) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      g_noalloc_ptr[device] = nullptr;
    }
  }
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_check(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "scratch address");
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return DGF_OK;
}

// device memory of the forest's device (plain or managed)?  Host pointers
// would reach the kernels and fault there, so they are refused up front.
bool on_device(const void* p, int device) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

}  // namespace

extern "C" dgf_status dgf_dg_residual_noalloc(dgf_forest* f, const void* U_nodal, void* L_nodal) {
  if (dgf_status st = require_device(f)) return st;
  if (!U_nodal || !L_nodal) return fail(DGF_EINVAL, "null state pointer");
  if (U_nodal == L_nodal) return fail(DGF_EINVAL, "input and output must not alias");
  if (((uintptr_t)U_nodal | (uintptr_t)L_nodal) & 15)
    return fail(DGF_EINVAL, "state pointers must be 16-byte aligned");
  if (f->comp) return fail(DGF_EUNSUPPORTED, "dgf_dg_residual_noalloc: compensated forests are not supported");
  DeviceGuard dg(f->device);
  if (!on_device(U_nodal, f->device) || !on_device(L_nodal, f->device))
    return fail(DGF_EINVAL, "dgf_dg_residual_noalloc: state pointers must be device memory of the forest's device");
  const size_t need = (size_t)f->nL * 2 * f->d * f->nv * f->NFP * f->nt * f->esize;
  if (need > kNoAllocScratchBytes)
    return fail(DGF_EUNSUPPORTED, "dgf_dg_residual_noalloc: the guard traces of this forest need " +
                                      std::to_string(need) + " bytes, above the 16 MiB static scratch");
  void* scratch = nullptr;
  dgf_status st = noalloc_scratch(f->device, &scratch);
  if (st) return st;
  RtGuard g = guard_args(f, 0, scratch, 1);
  g.U = U_nodal;
  if ((st = cuda_check(do_guard(f, g), "guard"))) return st;
  RtStage s = stage_args(f, 0, 1, 0.0, 1.0, 1, 0);
  s.U = U_nodal;
  s.Un = U_nodal;
  s.Uout = L_nodal;
  s.gtr = scratch;
  return cuda_check(do_stage(f, s), "stage");
}

// ================================================================ batches
// Several forests advanced together: one launch of each kernel per stage for
// all of them (the per-forest kernel arguments live in device arrays; the
// kernels find each work item's forest from prefix sums), captured in one
// CUDA graph per membership.  Every forest keeps its own time, end time,
// time increment and CFL minimum, and each work item does the arithmetic of
// the forest's own single-forest stage in the same kernel, so a forest's
// result does not depend on the other members.
struct dgf_batch {
  int device = -1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<dgf_forest*> mem;
  int p = -1, kernel = 1, all_affine = 0, slots = 0, items = 0, zchunk = 8;
  long long gblocks = 0;
  // device arrays, kept and grown (never shrunk) across membership changes,
  // so that admitting or retiring a member frees nothing (cudaFree would
  // synchronise the whole device); written by one copy on the batch stream
  // from a pinned host staging buffer
  void* dev = nullptr;
  size_t dev_cap = 0;
  void* host = nullptr;
  size_t host_cap = 0;
  void* prog_dev = nullptr;   // progress gather: [n] t, [n] steps, [n] status
  void* prog_host = nullptr;  // pinned
  int prog_cap = 0;
  void* sargs[3] = {nullptr, nullptr, nullptr};
  void* gargs[3] = {nullptr, nullptr, nullptr};
  int* istart = nullptr;
  int* bstart = nullptr;
  int* nfb = nullptr;
  DevScalars** scal = nullptr;
  double* cfl = nullptr;
  cudaGraphExec_t graph = nullptr;
};

namespace {

// forget the members' arrays and graph (the allocations stay for reuse)
void batch_reset(dgf_batch* b) {
  for (int k = 0; k < 3; ++k) b->sargs[k] = b->gargs[k] = nullptr;
  b->istart = b->bstart = b->nfb = nullptr;
  b->scal = nullptr;
  b->cfl = nullptr;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->items = 0;
  b->gblocks = 0;
}

void batch_release(dgf_batch* b) {
  batch_reset(b);
  if (b->dev) cudaFree(b->dev);
  if (b->host) cudaFreeHost(b->host);
  if (b->prog_dev) cudaFree(b->prog_dev);
  if (b->prog_host) cudaFreeHost(b->prog_host);
  b->dev = b->host = b->prog_dev = b->prog_host = nullptr;
  b->dev_cap = b->host_cap = 0;
  b->prog_cap = 0;
}

// one time increment of every member: dt of each, then 3 x (guard traces, stage)
dgf_status batch_enqueue(dgf_batch* b) {
  const int n = (int)b->mem.size();
  k_dt_batch<<<(n + 127) / 128, 128, 0, b->stream>>>(b->scal, b->cfl, n);
  dgf_status st = cuda_check(cudaGetLastError(), "dt");
  if (st) return st;
  dgf_forest* f0 = b->mem[0];
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int k = 0; k < 3; ++k) {
    if ((st = cuda_check(launch_guard_batch<3, float>(b->p, b->gargs[k], b->bstart, b->nfb, n, b->gblocks,
                                                       b->stream),
                         "batch guard")))
      return st;
    RtStage c = stage_args(f0, 0, 1, ca[k], cb[k], 0, k == 2);
    c.kernel = b->kernel;
    c.all_affine = b->all_affine;
    // one CTA per work item, not a persistent grid: a batch stage of several
    // large members runs for tens of ms, and CTAs that retire after each
    // item let work of other streams (a solve being built, on a stream of
    // higher priority) onto the SMs meanwhile
    const int grid = b->items;
    if ((st = cuda_check(launch_stage_batch<3, float>(c, b->sargs[k], b->istart, n, grid, b->stream),
                         "batch stage")))
      return st;
  }
  return DGF_OK;
}

}  // namespace

extern "C" {

dgf_status dgf_batch_create(int32_t device, void* stream, dgf_batch** out) {
  if (!out) return fail(DGF_EINVAL, "null argument");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(DGF_EINVAL, "no such device");
  dgf_batch* b = new dgf_batch();
  b->device = device;
  DeviceGuard dg(device);
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(DGF_ECUDA, "stream creation failed");
    }
    b->own_stream = true;
  }
  *out = b;
  return DGF_OK;
}

dgf_status dgf_batch_destroy(dgf_batch* b) {
  if (!b) return DGF_OK;
  DeviceGuard dg(b->device);
  cudaStreamSynchronize(b->stream);
  batch_release(b);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return DGF_OK;
}

dgf_status dgf_batch_set(dgf_batch* b, dgf_forest* const* forests, const double* t_end, int32_t n) {
  if (!b || (n > 0 && (!forests || !t_end)) || n < 0) return fail(DGF_EINVAL, "null argument");
  DeviceGuard dg(b->device);
  cudaStreamSynchronize(b->stream);
  batch_reset(b);
  b->mem.assign(forests, forests + n);
  if (n == 0) return DGF_OK;
  dgf_forest* f0 = forests[0];
  for (int i = 0; i < n; ++i) {
    dgf_forest* f = forests[i];
    if (!f || f->device != b->device) return fail(DGF_EINVAL, "batch members must be forests on the batch's device");
    if (f->d != 3 || f->n != 8 || f->precision != DGF_FP32 || f->comp || f->mortar || f->limiter > 0.0)
      return fail(DGF_EUNSUPPORTED,
                  "batches take 3D FP32 forests of 8^3-cell blocks in the plain form, without the mortar repair "
                  "or the limiter");
    if (f->p != f0->p) return fail(DGF_EINVAL, "batch members must have one degree");
    if (!f->have_state) return fail(DGF_ESTATE, "batch member without a state");
    // the member's own stream must have finished its work
    if (cudaStreamSynchronize(f->stream) != cudaSuccess) return fail(DGF_ECUDA, "member stream");
  }
  b->p = f0->p;
  b->kernel = pair_applies(f0) ? 0 : 1;
  if (const char* ks = getenv("DGF_STAGE_KERNEL"))
    if (strcmp(ks, "classic") == 0) b->kernel = 1;
  b->all_affine = 1;
  for (auto* f : b->mem) b->all_affine &= f->all_affine ? 1 : 0;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  b->slots = stage_batch_blocks_per_sm<3, float>(b->p, b->kernel, b->all_affine) * sms;
  if (b->slots <= 0) return fail(DGF_EUNSUPPORTED, "batch stage kernel does not fit the device");
  // prefix sums of work items and guard blocks; per-stage argument arrays
  std::vector<int> istart(n + 1, 0), bstart(n + 1, 0), nfb(n, 0);
  std::vector<DevScalars*> scal(n);
  std::vector<double> cfl(n);
  const int src[3] = {0, 1, 2}, dst[3] = {1, 2, 0};
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
  std::vector<RtStage> rs[3];
  std::vector<RtGuard> rg[3];
  long long gb = 0;
  // one z-chunk length for the batch, from its total block count and the
  // persistent grid: a chunk costs its layers plus ~0.6 layer of start-up
  // (the lower layer's load and trace), the value that reproduces the
  // single-forest autotuner's choices from 64 to 4096 blocks at p = 1..3;
  // the result does not depend on it
  b->zchunk = f0->n;
  {
    int64_t blocks = 0;
    for (auto* f : b->mem) blocks += f->nL;
    double best = 1e300;
    for (int z = f0->n; z >= 1; z /= 2) {
      const int64_t items = blocks * ((f0->n + z - 1) / z);
      const double cost = (double)((items + b->slots - 1) / b->slots) * (z + 0.6);
      if (cost < best - 1e-9) {
        best = cost;
        b->zchunk = z;
      }
      if (z == 1) break;
    }
    if (const char* zc = getenv("DGF_ZCHUNK")) b->zchunk = std::max(1, std::min(f0->n, atoi(zc)));
  }
  for (int i = 0; i < n; ++i) {
    dgf_forest* f = forests[i];
    for (int k = 0; k < 3; ++k) {
      rs[k].push_back(stage_args(f, src[k], dst[k], ca[k], cb[k], 0, k == 2));
      rs[k].back().zchunk = b->zchunk;
      rg[k].push_back(guard_args(f, src[k], f->gtr.ptr, 1));
    }
    const int it = stage_items<3, float>(rs[0].back());
    if (it < 0) return fail(DGF_EUNSUPPORTED, "batch member tiling");
    istart[i + 1] = istart[i] + it;
    const long long g = guard_blocks<3, float>(rg[0].back(), &nfb[i]);
    gb += g;
    if (gb >= (1ll << 31)) return fail(DGF_EUNSUPPORTED, "batch too large for one guard launch");
    bstart[i + 1] = (int)gb;
    scal[i] = (DevScalars*)f->scal.ptr;
    cfl[i] = f->cfl;
    f->t_end_dev = t_end[i];
    k_set_t_end<<<1, 1, 0, b->stream>>>((DevScalars*)f->scal.ptr, t_end[i]);
    dgf_status st = cuda_check(cudaGetLastError(), "t_end");
    if (st) return st;
  }
  b->items = istart[n];
  b->gblocks = gb;
  // one device allocation holds every array (256-byte aligned pieces)
  const size_t ss = stage_args_pack<3, float>(rs[0].data(), n, nullptr);
  const size_t gs = guard_args_pack<3, float>(rg[0].data(), n, nullptr);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t sz[5] = {istart.size() * sizeof(int), bstart.size() * sizeof(int), nfb.size() * sizeof(int),
                        scal.size() * sizeof(DevScalars*), cfl.size() * sizeof(double)};
  size_t total = 3 * al(ss) + 3 * al(gs);
  for (size_t x : sz) total += al(x);
  if (total > b->dev_cap) {
    const size_t cap = std::max(total, 2 * b->dev_cap) + (64 << 10);
    if (b->dev) cudaFree(b->dev);
    b->dev = nullptr;
    b->dev_cap = 0;
    if (cudaMalloc(&b->dev, cap) != cudaSuccess) return fail(DGF_ENOMEM, "batch allocation failed");
    b->dev_cap = cap;
  }
  if (total > b->host_cap) {
    const size_t cap = std::max(total, 2 * b->host_cap) + (64 << 10);
    if (b->host) cudaFreeHost(b->host);
    b->host = nullptr;
    b->host_cap = 0;
    if (cudaMallocHost(&b->host, cap) != cudaSuccess) return fail(DGF_ENOMEM, "batch staging allocation failed");
    b->host_cap = cap;
  }
  unsigned char* h = (unsigned char*)b->host;
  unsigned char* d = (unsigned char*)b->dev;
  size_t off = 0;
  for (int k = 0; k < 3; ++k) {
    stage_args_pack<3, float>(rs[k].data(), n, h + off);
    b->sargs[k] = d + off;
    off += al(ss);
    guard_args_pack<3, float>(rg[k].data(), n, h + off);
    b->gargs[k] = d + off;
    off += al(gs);
  }
  const void* srcs[5] = {istart.data(), bstart.data(), nfb.data(), scal.data(), cfl.data()};
  void* dsts[5];
  for (int i = 0; i < 5; ++i) {
    memcpy(h + off, srcs[i], sz[i]);
    dsts[i] = d + off;
    off += al(sz[i]);
  }
  b->istart = (int*)dsts[0];
  b->bstart = (int*)dsts[1];
  b->nfb = (int*)dsts[2];
  b->scal = (DevScalars**)dsts[3];
  b->cfl = (double*)dsts[4];
  dgf_status st = cuda_check(cudaMemcpyAsync(b->dev, b->host, off, cudaMemcpyHostToDevice, b->stream), "batch upload");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(b->stream), "batch set");
}

dgf_status dgf_batch_step(dgf_batch* b, int32_t steps) {
  if (!b || steps < 0) return fail(DGF_EINVAL, "bad argument");
  if (b->mem.empty() || steps == 0) return DGF_OK;
  DeviceGuard dg(b->device);
  dgf_status st;
  if (!b->graph) {
    cudaGraph_t g = nullptr;
    if ((st = cuda_check(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "capture")))
      return st;
    dgf_status est = batch_enqueue(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (est) {
      if (g) cudaGraphDestroy(g);
      return est;
    }
    if ((st = cuda_check(e, "end capture"))) return st;
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if ((st = cuda_check(e, "instantiate"))) return st;
  }
  for (int i = 0; i < steps; ++i)
    if ((st = cuda_check(cudaGraphLaunch(b->graph, b->stream), "graph launch"))) return st;
  return DGF_OK;
}

dgf_status dgf_batch_progress(dgf_batch* b, double* t, int64_t* steps, int32_t* status) {
  if (!b || (!b->mem.empty() && (!t || !steps || !status))) return fail(DGF_EINVAL, "null argument");
  const int n = (int)b->mem.size();
  if (n == 0) return DGF_OK;
  DeviceGuard dg(b->device);
  const size_t bytes = (size_t)n * (sizeof(double) + sizeof(long long) + sizeof(int));
  if (n > b->prog_cap) {
    const int cap = std::max(n, 2 * b->prog_cap);
    const size_t cb = (size_t)cap * (sizeof(double) + sizeof(long long) + sizeof(int));
    if (b->prog_dev) cudaFree(b->prog_dev);
    if (b->prog_host) cudaFreeHost(b->prog_host);
    b->prog_dev = b->prog_host = nullptr;
    b->prog_cap = 0;
    if (cudaMalloc(&b->prog_dev, cb) != cudaSuccess || cudaMallocHost(&b->prog_host, cb) != cudaSuccess)
      return fail(DGF_ENOMEM, "batch progress buffers");
    b->prog_cap = cap;
  }
  double* dt_ = (double*)b->prog_dev;
  long long* ds = (long long*)(dt_ + n);
  int* dst = (int*)(ds + n);
  k_batch_progress<<<(n + 127) / 128, 128, 0, b->stream>>>(b->scal, n, dt_, ds, dst);
  dgf_status st = cuda_check(cudaGetLastError(), "batch progress");
  if (!st) st = cuda_check(cudaMemcpyAsync(b->prog_host, b->prog_dev, bytes, cudaMemcpyDeviceToHost, b->stream),
                           "batch progress copy");
  if (!st) st = cuda_check(cudaStreamSynchronize(b->stream), "batch progress sync");
  if (st) return st;
  const double* ht = (const double*)b->prog_host;
  const long long* hs = (const long long*)(ht + n);
  const int* hst = (const int*)(hs + n);
  for (int i = 0; i < n; ++i) {
    t[i] = ht[i];
    steps[i] = hs[i];
    status[i] = hst[i];
  }
  return DGF_OK;
}

dgf_status dgf_batch_query(dgf_batch* b, int32_t* idle) {
  if (!b || !idle) return fail(DGF_EINVAL, "null argument");
  DeviceGuard dg(b->device);
  const cudaError_t e = cudaStreamQuery(b->stream);
  if (e == cudaSuccess) {
    *idle = 1;
    return DGF_OK;
  }
  if (e == cudaErrorNotReady) {
    cudaGetLastError();
    *idle = 0;
    return DGF_OK;
  }
  return cuda_check(e, "batch query");
}

dgf_status dgf_batch_sync(dgf_batch* b) {
  if (!b) return fail(DGF_EINVAL, "null batch");
  DeviceGuard dg(b->device);
  return cuda_check(cudaStreamSynchronize(b->stream), "batch sync");
}

}  // extern "C"
