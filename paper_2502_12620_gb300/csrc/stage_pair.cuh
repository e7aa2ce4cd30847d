// FP32 stage kernel for 3D blocks of 8^3 cells at p = 1 and 2, written for
// the issue rate of sm_103a.
//
// It computes the same thing as k_stage (Sec. 2, Eqs. (3)-(5): volume
// integral with the contravariant fluxes, Lax-Friedrichs face fluxes, the
// diagonal inverse mass at the Gauss points, the SSP-RK stage combination
// and, on the last stage, the CFL minimum of Sec. 4.3), organised so that
// every instruction does twice the work and data stays in registers:
//
//  * Cell pairs.  A thread owns two x-neighbouring cells (i, i+1), i even,
//    and does all of its floating-point work on float2 pairs with the
//    packed FP32 instructions (fma/add/mul .f32x2); shared-memory accesses
//    are 8-byte pairs.
//  * Warp = face point.  Warp w of the CTA handles one face-point index fp
//    (p+1)^2 warps: (q_y, q_z) in the x sweep, (q_x, q_z) in y, (q_x, q_y)
//    in z); its 32 lanes are the 32 cell pairs of a layer (lane = 4 j + m,
//    cells 2m, 2m+1 of row j).  x- and y-neighbour traces and face fluxes
//    move between lanes with warp shuffles; z-face fluxes are carried in
//    registers from layer to layer, since a lane keeps its cells' column.
//  * The layer sweep is double buffered: while a layer is computed, the
//    next one (state and, for curved blocks, the 21 trilinear
//    coefficients per cell) arrives by TMA bulk copies (cp.async.bulk,
//    256-byte rows) completed on an mbarrier.
//
// Per layer: x lines (volume flux, derivative, x faces, lift) -> residual
// in shared memory; y lines (+= the same along y); z lines (+= along z, the
// z face above against the next layer's trace, 1/J) -> stage combination
// straight to global memory, CFL minimum on the last stage.
#pragma once

#include "dg_device.cuh"

namespace dgf {
namespace pairk {

constexpr int kStatusTimeout = -5;

// ------------------------------------------------------------ float2 math
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(1.0f / a.x, 1.0f / a.y); }
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void sts2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
__device__ __forceinline__ float2 shfl_up2(float2 v, int d) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int d) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// ------------------------------------------------- TMA bulk copy, mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// one 256-byte row global -> shared, completing on bar (plain, not multicast)
__device__ __forceinline__ void bulk_row(float* dst, const float* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// earlier generic-proxy reads of a buffer are ordered before the async
// proxy's writes into it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// bulk prefetch of a global row into L2 (no completion to wait for)
__device__ __forceinline__ void prefetch_row_l2(const float* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// bounded wait for the phase with the given parity; false if it gave up.
// The retry loop is a single asm statement, so that the compiler keeps its
// register allocation across the wait (a C++ loop around try_wait made it
// spill the live state of the z sweep).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t.reg .u32 c;\n\t"
      "mov.u32 c, 0;\n\t"
      "mov.u32 %0, 0;\n"
      "LAB_WAIT:\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "@p bra LAB_DONE;\n\t"
      "add.u32 c, c, 1;\n\t"
      "setp.lt.u32 p, c, %3;\n\t"
      "@p bra LAB_WAIT;\n\t"
      "bra LAB_END;\n"
      "LAB_DONE:\n\t"
      "mov.u32 %0, 1;\n"
      "LAB_END:\n\t"
      "}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(1u << 22)
      : "memory");
  return ok != 0;
}

// keeps the compiler from merging two evaluations of the same metric (one
// for the face normals before the face fluxes, one for the volume points
// after them), so the metric is not held in registers across the fluxes
__device__ __forceinline__ void reload_fence() { asm volatile("" ::: "memory"); }

// ------------------------------------------------------------- Euler, x2
// F . a for a pair of states (Eq. (2)); also returns v.a, p and 1/rho
__device__ __forceinline__ void flux2(const float2 (&u)[5], const float2 (&a)[3], float2 gm1, float2 (&F)[5],
                                      float2& vn, float2& pr) {
  const float2 ri = rcp2(u[0]);
  const float2 mn = fma2(u[3], a[2], fma2(u[2], a[1], mul(u[1], a[0])));
  const float2 ke = fma2(u[3], u[3], fma2(u[2], u[2], mul(u[1], u[1])));
  vn = mul(mn, ri);
  pr = mul(gm1, fma2(mul(ke, ri), f2(-0.5f), u[4]));
  F[0] = mn;
  F[1] = fma2(u[1], vn, mul(pr, a[0]));
  F[2] = fma2(u[2], vn, mul(pr, a[1]));
  F[3] = fma2(u[3], vn, mul(pr, a[2]));
  F[4] = mul(add(u[4], pr), vn);
}

// Lax-Friedrichs flux (Eq. (5), dissipative sign) for two face points at
// once; a = area vector from L to R.  Both physical fluxes are summed into
// the result term by term (fewer live registers than forming F(U_L) and
// F(U_R) first).  A NaN wave speed (negative density or pressure)
// propagates into the flux, as in lf_flux.
__device__ __forceinline__ void lf2(const float2 (&uL)[5], const float2 (&uR)[5], const float2 (&a)[3], float2 gam,
                                    float2 gm1, float2 (&Fh)[5]) {
  const float2 riL = rcp2(uL[0]), riR = rcp2(uR[0]);
  const float2 mnL = fma2(uL[3], a[2], fma2(uL[2], a[1], mul(uL[1], a[0])));
  const float2 mnR = fma2(uR[3], a[2], fma2(uR[2], a[1], mul(uR[1], a[0])));
  const float2 keL = fma2(uL[3], uL[3], fma2(uL[2], uL[2], mul(uL[1], uL[1])));
  const float2 keR = fma2(uR[3], uR[3], fma2(uR[2], uR[2], mul(uR[1], uR[1])));
  const float2 vL = mul(mnL, riL), vR = mul(mnR, riR);
  const float2 pL = mul(gm1, fma2(mul(keL, riL), f2(-0.5f), uL[4]));
  const float2 pR = mul(gm1, fma2(mul(keR, riR), f2(-0.5f), uR[4]));
  const float2 an = sqrt2(fma2(a[2], a[2], fma2(a[1], a[1], mul(a[0], a[0]))));
  const float2 sL = fma2(sqrt2(mul(mul(gam, pL), riL)), an, abs2(vL));
  const float2 sR = fma2(sqrt2(mul(mul(gam, pR), riR)), an, abs2(vR));
  float2 al;
  al.x = (sL.x > sR.x || sL.x != sL.x) ? sL.x : sR.x;
  al.y = (sL.y > sR.y || sL.y != sL.y) ? sL.y : sR.y;
  const float2 h = f2(0.5f);
  const float2 pp = add(pL, pR);
  Fh[0] = mul(h, fma2(al, sub(uL[0], uR[0]), add(mnL, mnR)));
#pragma unroll
  for (int jx = 0; jx < 3; ++jx)
    Fh[1 + jx] = mul(h, fma2(al, sub(uL[1 + jx], uR[1 + jx]),
                             fma2(uL[1 + jx], vL, fma2(uR[1 + jx], vR, mul(pp, a[jx])))));
  Fh[4] = mul(h, fma2(al, sub(uL[4], uR[4]), fma2(add(uL[4], pL), vL, mul(add(uR[4], pR), vR))));
}

// Metric along a line in direction DIR for a pair of cells (see LineGeo):
// J dxi_DIR/dx (s) = c0 + c1 s + c2 s^2, J(s) = e . (J dxi_DIR/dx)(s), from
// the trilinear coefficients of both cells in shared memory ([21][64]).
template <int DIR>
struct LineGeo2 {
  float2 c0[3], c1[3], c2[3], e[3];
  __device__ __forceinline__ void init(const float* __restrict__ G, int cl, const float (&xi)[3]) {
    float2 al[3][3], be[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < 3; ++j) al[a][j] = be[a][j] = f2(0.f);
#pragma unroll
    for (int c = 1; c < 8; ++c) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float2 x = lds2(G + ((c - 1) * 3 + j) * 64 + cl);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (!((c >> a) & 1)) continue;
          float fac = 1.f;
          bool has_s = false;
#pragma unroll
          for (int bb = 0; bb < 3; ++bb) {
            if (bb == a || !((c >> bb) & 1)) continue;
            if (bb == DIR) has_s = true;
            else fac *= xi[bb];
          }
          if (has_s) be[a][j] = fma2(x, f2(fac), be[a][j]);
          else al[a][j] = fma2(x, f2(fac), al[a][j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) e[j] = al[DIR][j];
    constexpr int i1 = (DIR + 1) % 3, i2 = (DIR + 2) % 3;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      c0[j] = sub(mul(al[i1][j1], al[i2][j2]), mul(al[i1][j2], al[i2][j1]));
      c1[j] = add(sub(mul(al[i1][j1], be[i2][j2]), mul(al[i1][j2], be[i2][j1])),
                  sub(mul(be[i1][j1], al[i2][j2]), mul(be[i1][j2], al[i2][j1])));
      c2[j] = sub(mul(be[i1][j1], be[i2][j2]), mul(be[i1][j2], be[i2][j1]));
    }
  }
  __device__ __forceinline__ void at(float s, float2 (&Ja)[3]) const {
#pragma unroll
    for (int j = 0; j < 3; ++j) Ja[j] = fma2(f2(s), fma2(f2(s), c2[j], c1[j]), c0[j]);
  }
  __device__ __forceinline__ float2 jac(const float2 (&Ja)[3]) const {
    return fma2(e[2], Ja[2], fma2(e[1], Ja[1], mul(e[0], Ja[0])));
  }
};

// V selects the CTA shape at p = 1 (0: four CTAs per SM, 1: five); one
// shape at p = 2
template <int P, int V = 0>
struct PairCfg {
  static constexpr int N = P + 1, Q = N * N * N, NFP = N * N, NV = 5;
  static constexpr int NT = 32 * NFP;  // one warp per face point
  static constexpr int ROWS = NV * Q;  // 256-byte state rows of a layer
  static constexpr int NG = 21;        // trilinear coefficient rows of a layer
  // shared memory: 2 state layers, 2 geometry layers, the residual layer
  static constexpr size_t SMEM = (size_t)(2 * ROWS * 64 + 2 * NG * 64 + ROWS * 64) * sizeof(float);
  // resident CTAs per SM: shared memory allows 2 at p = 2 (about 114 KB each)
  // and 5 at p = 1; at p = 1 four CTAs leave 128 registers per thread (16
  // warps, 4 per scheduler), five only 96 (more warps, more spills: the
  // autotuner times both)
  static constexpr int MINB = P <= 1 ? (V ? 5 : 4) : 2;
};

}  // namespace pairk

// AFF: every block of the forest is affine (no per-cell geometry is read;
// the curved code paths are not compiled into this instantiation)
// BATCH: one launch for every forest of a batch (A.members; the tables and
// stage coefficients of A are common to all of them).
template <int P, bool MORTAR, bool AFF, bool BATCH = false, int V = 0>
__global__ void __launch_bounds__(pairk::PairCfg<P, V>::NT, pairk::PairCfg<P, V>::MINB)
    k_stage_pair(const __grid_constant__ StageArgs<3, P, float> A) {
  static_assert(!(BATCH && MORTAR), "batches run without the mortar repair");
  using namespace pairk;
  using C = PairCfg<P, V>;
  constexpr int N = C::N, Q = C::Q, NFP = C::NFP, NV = 5, ROWS = C::ROWS, NG = C::NG;
  constexpr int n = 8, LAY = 64, nc = 512, nt = 64;
  const auto& T = A.T;
  const int tid = threadIdx.x;
  const int w = tid >> 5, lane = tid & 31;
  const int m = lane & 3, j = lane >> 2;  // cell pair (2m, 2m+1) of row j
  const int i0 = 2 * m;
  const int cl = i0 + n * j;              // first cell of the pair in the layer
  const int fa = w % N, fb = w / N;       // digits of this warp's face point
  if (!BATCH && A.mode == 0 && *A.dtp == 0.0) return;  // t_end reached: identity, nothing evaluated

  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* Us = reinterpret_cast<float*>(smem_raw);  // [2][ROWS][64]
  float* Gs = Us + 2 * ROWS * LAY;                 // [2][NG][64]
  float* Rs = Gs + 2 * NG * LAY;                   // [ROWS][64]
  __shared__ __align__(8) uint64_t bar[2];
  // per warp: U^n rows of the warp's z lines, copied into the residual rows
  // the warp has just read (those rows belong to that warp in the z sweep)
  __shared__ __align__(8) uint64_t wbar[C::NFP];
  __shared__ float sam[10];

  const float2 gam = f2(A.gamma), gm1 = f2(A.gamma - 1.f);
  float2 dt2 = f2(BATCH ? 0.f : (float)*A.dtp);  // per forest of a batch: per item
  const float2 ca2 = f2(A.ca), cb2 = f2(A.cb);
  float xq[N];
#pragma unroll
  for (int q = 0; q < N; ++q) xq[q] = T.x[q];
  // Gauss points of this warp's face-point digits (selected, not indexed, so
  // that nothing lives in local memory)
  float xa = xq[0], xb = xq[0];
#pragma unroll
  for (int q = 1; q < N; ++q) {
    xa = fa == q ? xq[q] : xa;
    xb = fb == q ? xq[q] : xb;
  }

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    for (int i = 0; i < C::NFP; ++i) mbar_init(&wbar[i], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t ph0 = 0, ph1 = 0;  // phase parity of each buffer's barrier
  bool pend0 = false, pend1 = false;  // a copy into the buffer not yet waited for
  uint32_t phw = 0;                   // phase parity of this warp's barrier
  bool wfail = false;                 // this warp's bounded wait gave up
  const bool use_un = A.mode == 0 && A.ca != 0.f;
  float lam_min = 3.0e38f;
  bool bad = false;
  int* cur_status = A.status;

  const int items = BATCH ? __ldg(&A.istart[A.nmem]) : A.nL * A.nchunks;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    // the forest of this item (a batch member, or the one forest)
    const StageArgs<3, P, float>* Mp = &A;
    int li = item;
    if constexpr (BATCH) {
      const int mi = batch_member(A.istart, A.nmem, item);
      Mp = A.members + mi;
      li = item - __ldg(&A.istart[mi]);
      if (A.mode == 0 && *Mp->dtp == 0.0) continue;  // that forest has reached its end time
      dt2 = f2((float)*Mp->dtp);
    }
    const StageArgs<3, P, float>& M = *Mp;
    cur_status = M.status;
    const int b = li / M.nchunks;
    const int chunk = li - b * M.nchunks;
    const int k0 = chunk * M.zchunk;
    const int k1 = min(n, k0 + M.zchunk);
    const size_t boff = (size_t)b * NV * Q * nc;
    const float* __restrict__ Ub = M.U + boff;
    const float* __restrict__ Unb = M.Un + boff;
    const float* __restrict__ Geo = M.geo + (size_t)b * NG * nc;
    const float* __restrict__ Tb = M.gtr + (size_t)b * 6 * NV * NFP * nt;
    const float* __restrict__ Hb = M.hcell + (size_t)b * nc;
    float* __restrict__ Ob = M.Uout;
    const bool aff = AFF || M.affine[b] != 0;
    const int fmask = MORTAR ? M.fluxmask[b] : 0;
    const uint32_t bytes = (uint32_t)((ROWS + (aff ? 0 : NG)) * LAY * sizeof(float));
    // one layer (state rows, and the coefficient rows of a curved block) into buffer k & 1
    auto issue = [&](int k) {
      const int bf = k & 1;
      if (bf) pend1 = true;
      else pend0 = true;
      if (tid == 0) mbar_arrive_expect(&bar[bf], bytes);
      if (tid < ROWS + NG) fence_proxy_async();
      if (tid < ROWS) {
        bulk_row(Us + (bf * ROWS + tid) * LAY, Ub + (size_t)tid * nc + k * LAY, LAY * sizeof(float), &bar[bf]);
        // U^n of the same layer, read by the stage combination a layer later
        if (A.ca != 0.f) prefetch_row_l2(Unb + (size_t)tid * nc + k * LAY, LAY * sizeof(float));
      } else if (!aff && tid < ROWS + NG) {
        const int g = tid - ROWS;
        bulk_row(Gs + (bf * NG + g) * LAY, Geo + (size_t)g * nc + k * LAY, LAY * sizeof(float), &bar[bf]);
      }
    };
    auto wait = [&](int k) -> bool {
      const int bf = k & 1;
      const bool ok = mbar_wait(&bar[bf], bf ? ph1 : ph0);
      if (bf) {
        ph1 ^= 1u;
        pend1 = false;
      } else {
        ph0 ^= 1u;
        pend0 = false;
      }
      return ok;
    };
#define GTR(f, v, fp, t) Tb[(((size_t)(f) * NV + (v)) * NFP + (fp)) * nt + (t)]

    __syncthreads();  // the previous item is done with every buffer
    if (aff && tid < 10) sam[tid] = M.ameta[(size_t)b * 10 + tid];
    if (k0 > 0) issue(k0 - 1);
    issue(k0);
    bool ok = true;
    if (k0 > 0) ok = wait(k0 - 1) && ok;
    ok = wait(k0) && ok;
    if (__syncthreads_or(!ok)) goto timeout;

    // ------------------------------------ z face below the first layer
    // (the carried flux of an unchunked sweep: the layer below's top trace
    // and metric against this layer's bottom trace, or the guard trace)
    const int fpZ = w;  // (q_x, q_y) = (fa, fb)
    float2 Fbot[NV];
    {
      const float* Uc = Us + (k0 & 1) * ROWS * LAY;
      float2 tm[NV], tl[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float2 s = f2(0.f);
#pragma unroll
        for (int qz = 0; qz < N; ++qz) s = fma2(f2(T.lm[qz]), lds2(Uc + (v * Q + fpZ + NFP * qz) * LAY + cl), s);
        tm[v] = s;
      }
      float2 Ja[3];
      if (k0 == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) tl[v] = lds2(&GTR(4, v, fpZ, cl));
        if (aff) {
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) Ja[jj] = f2(sam[6 + jj]);
        } else {
          LineGeo2<2> lg;
          const float xi[3] = {xa, xb, 0.f};
          lg.init(Gs + (k0 & 1) * NG * LAY, cl, xi);
          lg.at(-1.f, Ja);
        }
      } else {
        const float* Ul = Us + ((k0 - 1) & 1) * ROWS * LAY;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float2 s = f2(0.f);
#pragma unroll
          for (int qz = 0; qz < N; ++qz) s = fma2(f2(T.lp[qz]), lds2(Ul + (v * Q + fpZ + NFP * qz) * LAY + cl), s);
          tl[v] = s;
        }
        if (aff) {
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) Ja[jj] = f2(sam[6 + jj]);
        } else {
          LineGeo2<2> lg;
          const float xi[3] = {xa, xb, 0.f};
          lg.init(Gs + ((k0 - 1) & 1) * NG * LAY, cl, xi);
          lg.at(1.f, Ja);
        }
      }
      lf2(tl, tm, Ja, gam, gm1, Fbot);
      if (MORTAR && k0 == 0 && (fmask & 16)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) Fbot[v] = tl[v];  // the z- face flux itself
      }
    }

    for (int k = k0; k < k1; ++k) {
      // layer k-1 is done: its buffer and the residual layer are free
      if (__syncthreads_or(wfail)) goto timeout;
      if (k + 1 < n) issue(k + 1);
      const float* Uc = Us + (k & 1) * ROWS * LAY;
      const float* Gc = Gs + (k & 1) * NG * LAY;
      const int tg_row = j + n * k;  // guard cell of my row on the x faces

      // ----------------------------------------------------- x lines
      // traces -> faces -> lifts -> volume flux and weak derivative, with
      // the state read twice from shared memory rather than held (registers)
      {
        const int fpX = w;  // (q_y, q_z)
        float2 tm[NV], tp[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          tm[v] = tp[v] = f2(0.f);
#pragma unroll
          for (int qx = 0; qx < N; ++qx) {
            const float2 x = lds2(Uc + (v * Q + qx + N * fpX) * LAY + cl);
            tm[v] = fma2(f2(T.lm[qx]), x, tm[v]);
            tp[v] = fma2(f2(T.lp[qx]), x, tp[v]);
          }
        }
        // face normals at xi_x = -1 (both cells) and +1; the metric along the
        // line is evaluated again for the volume points below
        float2 Jm[3], Jp[3];
        if (aff) {
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) Jm[jj] = Jp[jj] = f2(sam[jj]);
        } else {
          LineGeo2<0> lg;
          const float xi[3] = {0.f, xa, xb};
          lg.init(Gc, cl, xi);
          lg.at(-1.f, Jm);
          lg.at(1.f, Jp);
        }
        reload_fence();
        // left face of each cell of the pair: (face i0, face i0+1)
        float2 Fl[NV];
        float Fr[NV];
        {
          float2 uL[NV], Ja[3];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const float nb = __shfl_up_sync(0xffffffffu, tp[v].y, 1);
            uL[v] = make_float2(m == 0 ? GTR(0, v, fpX, tg_row) : nb, tp[v].x);
          }
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) Ja[jj] = Jm[jj];
          lf2(uL, tm, Ja, gam, gm1, Fl);
        }
        if (MORTAR && m == 0 && (fmask & 1)) {
#pragma unroll
          for (int v = 0; v < NV; ++v) Fl[v].x = GTR(0, v, fpX, tg_row);
        }
        // right faces: the next pair's left face; the block's x+ face on m == 3
#pragma unroll
        for (int v = 0; v < NV; ++v) Fr[v] = __shfl_down_sync(0xffffffffu, Fl[v].x, 1);
        if (m == 3) {
          if (MORTAR && (fmask & 2)) {
#pragma unroll
            for (int v = 0; v < NV; ++v) Fr[v] = GTR(1, v, fpX, tg_row);
          } else {
            float ul[NV], ur[NV], Jr[3], Fh[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              ul[v] = tp[v].y;
              ur[v] = GTR(1, v, fpX, tg_row);
            }
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) Jr[jj] = Jp[jj].y;
            lf_flux<3, float>(ul, ur, Jr, A.gamma, Fh);
#pragma unroll
            for (int v = 0; v < NV; ++v) Fr[v] = Fh[v];
          }
        }
        LineGeo2<0> lg;
        if (!aff) {
          const float xi[3] = {0.f, xa, xb};
          lg.init(Gc, cl, xi);
        }
        float2 r[N][NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float2 fr = make_float2(Fl[v].y, Fr[v]);
#pragma unroll
          for (int qx = 0; qx < N; ++qx) r[qx][v] = fma2(f2(T.lmw[qx]), Fl[v], mul(f2(-T.lpw[qx]), fr));
        }
#pragma unroll
        for (int jj = 0; jj < N; ++jj) {
          float2 uq[NV], Jq[3], G[NV], vn, pr;
#pragma unroll
          for (int v = 0; v < NV; ++v) uq[v] = lds2(Uc + (v * Q + jj + N * fpX) * LAY + cl);
          if (aff) {
#pragma unroll
            for (int jx = 0; jx < 3; ++jx) Jq[jx] = f2(sam[jx]);
          } else {
            lg.at(xq[jj], Jq);
          }
          flux2(uq, Jq, gm1, G, vn, pr);
#pragma unroll
          for (int qx = 0; qx < N; ++qx)
#pragma unroll
            for (int v = 0; v < NV; ++v) r[qx][v] = fma2(f2(T.Sh[qx][jj]), G[v], r[qx][v]);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int qx = 0; qx < N; ++qx) sts2(Rs + (v * Q + qx + N * fpX) * LAY + cl, r[qx][v]);
      }
      __syncthreads();

      // ----------------------------------------------------- y lines
      {
        const int fpY = w;  // (q_x, q_z)
        const int tg_col = i0 + n * k;
        float2 tm[NV], tp[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          tm[v] = tp[v] = f2(0.f);
#pragma unroll
          for (int qy = 0; qy < N; ++qy) {
            const float2 x = lds2(Uc + (v * Q + fa + N * qy + NFP * fb) * LAY + cl);
            tm[v] = fma2(f2(T.lm[qy]), x, tm[v]);
            tp[v] = fma2(f2(T.lp[qy]), x, tp[v]);
          }
        }
        float2 Jm[3], Jp[3];
        if (aff) {
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) Jm[jj] = Jp[jj] = f2(sam[3 + jj]);
        } else {
          LineGeo2<1> lg;
          const float xi[3] = {xa, 0.f, xb};
          lg.init(Gc, cl, xi);
          lg.at(-1.f, Jm);
          lg.at(1.f, Jp);
        }
        reload_fence();
        // bottom face of my row: the row below's top trace, or the guard trace
        float2 Fb[NV], Ft[NV];
        {
          float2 uL[NV], Ja[3];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const float2 nb = shfl_up2(tp[v], 4);
            uL[v] = j == 0 ? lds2(&GTR(2, v, fpY, tg_col)) : nb;
          }
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) Ja[jj] = Jm[jj];
          lf2(uL, tm, Ja, gam, gm1, Fb);
        }
        if (MORTAR && j == 0 && (fmask & 4)) {
#pragma unroll
          for (int v = 0; v < NV; ++v) Fb[v] = lds2(&GTR(2, v, fpY, tg_col));
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) Ft[v] = shfl_down2(Fb[v], 4);
        if (j == n - 1) {
          float2 ur[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) ur[v] = lds2(&GTR(3, v, fpY, tg_col));
          if (MORTAR && (fmask & 8)) {
#pragma unroll
            for (int v = 0; v < NV; ++v) Ft[v] = ur[v];
          } else {
            lf2(tp, ur, Jp, gam, gm1, Ft);
          }
        }
        LineGeo2<1> lg;
        if (!aff) {
          const float xi[3] = {xa, 0.f, xb};
          lg.init(Gc, cl, xi);
        }
        float2 r[N][NV];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int qy = 0; qy < N; ++qy)
            r[qy][v] = fma2(f2(T.lmw[qy]), Fb[v],
                            fma2(f2(-T.lpw[qy]), Ft[v], lds2(Rs + (v * Q + fa + N * qy + NFP * fb) * LAY + cl)));
#pragma unroll
        for (int jj = 0; jj < N; ++jj) {
          float2 uq[NV], Jq[3], G[NV], vn, pr;
#pragma unroll
          for (int v = 0; v < NV; ++v) uq[v] = lds2(Uc + (v * Q + fa + N * jj + NFP * fb) * LAY + cl);
          if (aff) {
#pragma unroll
            for (int jx = 0; jx < 3; ++jx) Jq[jx] = f2(sam[3 + jx]);
          } else {
            lg.at(xq[jj], Jq);
          }
          flux2(uq, Jq, gm1, G, vn, pr);
#pragma unroll
          for (int qy = 0; qy < N; ++qy)
#pragma unroll
            for (int v = 0; v < NV; ++v) r[qy][v] = fma2(f2(T.Sh[qy][jj]), G[v], r[qy][v]);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int qy = 0; qy < N; ++qy) sts2(Rs + (v * Q + fa + N * qy + NFP * fb) * LAY + cl, r[qy][v]);
      }
      __syncthreads();
      if (k + 1 < n) {
        const bool okn = wait(k + 1);
        if (__syncthreads_or(!okn)) goto timeout;
      }

      // ----------------------------------------------------- z lines + stage
      {
        float2 tp[NV], Ft[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          tp[v] = f2(0.f);
#pragma unroll
          for (int qz = 0; qz < N; ++qz) tp[v] = fma2(f2(T.lp[qz]), lds2(Uc + (v * Q + fpZ + NFP * qz) * LAY + cl), tp[v]);
        }
        {
          // the next layer's bottom trace (same arithmetic as at a chunk start)
          float2 th[NV], Ja[3];
          if (k + 1 < n) {
            const float* Un1 = Us + ((k + 1) & 1) * ROWS * LAY;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              float2 s = f2(0.f);
#pragma unroll
              for (int qz = 0; qz < N; ++qz)
                s = fma2(f2(T.lm[qz]), lds2(Un1 + (v * Q + fpZ + NFP * qz) * LAY + cl), s);
              th[v] = s;
            }
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) th[v] = lds2(&GTR(5, v, fpZ, cl));
          }
          if (aff) {
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) Ja[jj] = f2(sam[6 + jj]);
          } else {
            LineGeo2<2> lg;
            const float xi[3] = {xa, xb, 0.f};
            lg.init(Gc, cl, xi);
            lg.at(1.f, Ja);
          }
          reload_fence();
          lf2(tp, th, Ja, gam, gm1, Ft);
          if (MORTAR && k == n - 1 && (fmask & 32)) {
#pragma unroll
            for (int v = 0; v < NV; ++v) Ft[v] = th[v];  // the z+ face flux itself
          }
        }
        LineGeo2<2> lg;
        if (!aff) {
          const float xi[3] = {xa, xb, 0.f};
          lg.init(Gc, cl, xi);
        }
        float2 r[N][NV], iJ[N];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int qz = 0; qz < N; ++qz)
            r[qz][v] = fma2(f2(T.lmw[qz]), Fbot[v],
                            fma2(f2(-T.lpw[qz]), Ft[v], lds2(Rs + (v * Q + fpZ + NFP * qz) * LAY + cl)));
#pragma unroll
        for (int jj = 0; jj < N; ++jj) {
          float2 uq[NV], Jq[3], G[NV], vn, pr;
#pragma unroll
          for (int v = 0; v < NV; ++v) uq[v] = lds2(Uc + (v * Q + fpZ + NFP * jj) * LAY + cl);
          if (aff) {
#pragma unroll
            for (int jx = 0; jx < 3; ++jx) Jq[jx] = f2(sam[6 + jx]);
            iJ[jj] = f2(sam[9]);
          } else {
            lg.at(xq[jj], Jq);
            iJ[jj] = rcp2(lg.jac(Jq));
          }
          flux2(uq, Jq, gm1, G, vn, pr);
#pragma unroll
          for (int qz = 0; qz < N; ++qz)
#pragma unroll
            for (int v = 0; v < NV; ++v) r[qz][v] = fma2(f2(T.Sh[qz][jj]), G[v], r[qz][v]);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) Fbot[v] = Ft[v];
        // U^n of the z line's points (prefetched into L2 a layer ahead), all
        // loads issued before the first use
        float2 un[N][NV];
        if (use_un) {
#pragma unroll
          for (int qz = 0; qz < N; ++qz)
#pragma unroll
            for (int v = 0; v < NV; ++v)
              un[qz][v] = __ldcg(reinterpret_cast<const float2*>(Unb + (size_t)(v * Q + fpZ + NFP * qz) * nc + k * LAY + cl));
        }
        // stage combination straight to global memory, CFL on the last stage
        const size_t gcell = boff + (size_t)k * LAY + cl;  // (v, q) row offsets added below
        float2 hc = f2(0.f);
        if (A.last) hc = __ldg(reinterpret_cast<const float2*>(Hb + k * LAY + cl));
#pragma unroll
        for (int qz = 0; qz < N; ++qz) {
          const int q = fpZ + NFP * qz;
          float2 o[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const float2 s = mul(r[qz][v], iJ[qz]);
            const size_t gi = gcell + (size_t)(v * Q + q) * nc;
            float2 val;
            if (A.mode == 1) {
              val = s;
            } else {
              val = mul(cb2, fma2(dt2, s, lds2(Uc + (v * Q + q) * LAY + cl)));
              if (use_un) val = fma2(ca2, un[qz][v], val);
            }
            *reinterpret_cast<float2*>(Ob + gi) = val;
            o[v] = val;
          }
          if (A.last) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float r0 = e ? o[0].y : o[0].x;
              const float m1 = e ? o[1].y : o[1].x;
              const float m2 = e ? o[2].y : o[2].x;
              const float m3 = e ? o[3].y : o[3].x;
              const float en = e ? o[4].y : o[4].x;
              const float ri = 1.f / r0;
              const float ke = m1 * m1 + m2 * m2 + m3 * m3;
              const float sv = (fabsf(m1) + fabsf(m2) + fabsf(m3)) * ri;
              const float pr = (A.gamma - 1.f) * (en - 0.5f * ke * ri);
              if (!(r0 > 0.f) || !(pr > 0.f) || !(pr < 3.0e38f)) {
                bad = true;
              } else {
                const float lam = sv + 3.f * sqrtf(A.gamma * pr * ri);
                const float hv = (e ? hc.y : hc.x) / lam;
                lam_min = hv < lam_min ? hv : lam_min;
              }
            }
          }
        }
      }
    }
    if constexpr (BATCH) {
      // the CFL minimum and the status belong to this item's forest
      if (A.last) {
        cta_min_atomic<C::NT>((double)lam_min, M.lam_bits);
        lam_min = 3.0e38f;
        if (__syncthreads_or(bad) && tid == 0) atomicExch(M.status, kStatusNonFinite);
        bad = false;
      }
    }
#undef GTR
  }
  if (false) {
  timeout:
    // a bounded wait gave up: report it, wait (bounded) for the copies still
    // in flight into this CTA's buffers, then leave
    if (tid == 0) atomicExch(cur_status, kStatusTimeout);
    if (pend0) mbar_wait(&bar[0], ph0);
    if (pend1) mbar_wait(&bar[1], ph1);
    // a warp whose own wait gave up retries it once (bounded) before leaving
    if (wfail) mbar_wait(&wbar[w], phw ^ 1u);
    return;
  }
  if (!BATCH && A.last) {
    // block min of h/lambda -> one atomic per CTA
    double v = (double)lam_min;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_xor_sync(0xffffffffu, v, o);
      v = u < v ? u : v;
    }
    __shared__ double red[32];
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
      v = lane < C::NT / 32 ? red[lane] : 3.0e38;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
      }
      if (lane == 0 && v < 3.0e38) atomicMin(A.lam_bits, (unsigned long long)__double_as_longlong(v));
    }
    if (bad) atomicExch(A.status, kStatusNonFinite);
  }
}

// launch (grid = persistent CTAs, or one per work item) and resident CTAs
// per SM, for the launch layer in kernels_inst.cuh; v = the CTA shape
template <int P, int V>
cudaError_t stage_pair_launch_v(const StageArgs<3, P, float>& a, int grid, bool mortar, bool all_affine,
                                cudaStream_t s) {
  using C = pairk::PairCfg<P, V>;
  if (mortar) {
    if (all_affine) k_stage_pair<P, true, true, false, V><<<grid, C::NT, C::SMEM, s>>>(a);
    else k_stage_pair<P, true, false, false, V><<<grid, C::NT, C::SMEM, s>>>(a);
  } else {
    if (all_affine) k_stage_pair<P, false, true, false, V><<<grid, C::NT, C::SMEM, s>>>(a);
    else k_stage_pair<P, false, false, false, V><<<grid, C::NT, C::SMEM, s>>>(a);
  }
  return cudaGetLastError();
}

template <int P>
cudaError_t stage_pair_launch(const StageArgs<3, P, float>& a, int grid, bool mortar, bool all_affine,
                              cudaStream_t s, int v) {
  if constexpr (P == 1) {
    if (v) return stage_pair_launch_v<P, 1>(a, grid, mortar, all_affine, s);
  }
  return stage_pair_launch_v<P, 0>(a, grid, mortar, all_affine, s);
}

// one launch over the forests of a batch (a.members); plain form, no mortar
template <int P>
cudaError_t stage_pair_launch_batch(const StageArgs<3, P, float>& a, int grid, bool all_affine, cudaStream_t s) {
  using C = pairk::PairCfg<P>;
  if (all_affine) k_stage_pair<P, false, true, true><<<grid, C::NT, C::SMEM, s>>>(a);
  else k_stage_pair<P, false, false, true><<<grid, C::NT, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int P, bool MORTAR, bool AFF, bool BATCH = false, int V = 0>
int pair_blocks_per_sm_one() {
  using C = pairk::PairCfg<P, V>;
  if (cudaFuncSetAttribute(k_stage_pair<P, MORTAR, AFF, BATCH, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)C::SMEM) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage_pair<P, MORTAR, AFF, BATCH, V>, C::NT, C::SMEM) !=
      cudaSuccess)
    return 0;
  return nb;
}

// the fewest resident CTAs over the instantiations one forest may launch
// (shape v; the batch instantiations have shape 0)
template <int P>
int stage_pair_blocks_per_sm(int v) {
  int o[6];
  if (P == 1 && v) {
    o[0] = pair_blocks_per_sm_one<P, false, false, false, 1>();
    o[1] = pair_blocks_per_sm_one<P, true, false, false, 1>();
    o[2] = pair_blocks_per_sm_one<P, false, true, false, 1>();
    o[3] = pair_blocks_per_sm_one<P, true, true, false, 1>();
    o[4] = o[5] = o[0];
  } else {
    o[0] = pair_blocks_per_sm_one<P, false, false>();
    o[1] = pair_blocks_per_sm_one<P, true, false>();
    o[2] = pair_blocks_per_sm_one<P, false, true>();
    o[3] = pair_blocks_per_sm_one<P, true, true>();
    o[4] = pair_blocks_per_sm_one<P, false, false, true>();
    o[5] = pair_blocks_per_sm_one<P, false, true, true>();
  }
  int lo = o[0];
  for (int i = 1; i < 6; ++i) lo = o[i] < lo ? o[i] : lo;
  return lo;
}

}  // namespace dgf
