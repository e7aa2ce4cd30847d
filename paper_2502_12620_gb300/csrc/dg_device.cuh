// Device code of the block-forest DG path (compressible Euler, SSP-RK3).
//
// What the kernels compute (arXiv 2502.12620):
//   Sec. 2, Eqs. (3)-(5): per cell, M dK/dt = R with the volume term
//   int F . grad(phi) dV and the face term -oint F^ phi dS, F^ the
//   Lax-Friedrichs flux; SSP-RK3 stage combination.
//   Sec. 3.5, Eqs. (15)-(17): guard cells from same-level (copy), coarser
//   (split S) and finer (combine C) neighbours, all rotated into the
//   receiving block's frame.
//
// How (GB300 design, not the paper's): on the device the state is held as
// values at the (p+1)^d Gauss points (SoA [leaf][var][point][cell]); the
// modal coefficients of the C ABI are converted at the boundary (u = V K).
// With the (p+1)-point rule the mass matrix is M = V^T diag(wJ) V, so
// V M^{-1} = diag(1/(wJ)) V^{-T}: the inverse mass is diagonal and the
// volume and face integrals become 1D line operations (weak derivative Sh,
// boundary lifts l(+-1)/w).  Rotations map Gauss points onto Gauss points,
// split and combine become small nodal operators.
// The residual is accumulated in shared memory by directional sweeps; every
// interior face flux is computed once; the stage combination and, on the
// last stage, the CFL minimum are fused into the epilogue.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

namespace dgf {

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// status codes shared with dgf.h
constexpr int kStatusNonFinite = -4;

// 1D reference tables for N = p+1 Gauss points (filled on the host in FP64).
template <int N, typename Real>
struct Tab {
  Real x[N], w[N];
  Real V[N][N];    // V[q][k]  = P_k(x_q)           modal -> nodal
  Real Vi[N][N];   // Vi[k][q] = (2k+1)/2 w_q P_k    nodal -> modal
  Real Sh[N][N];   // Sh[q][j] = (w_j / w_q) l_j'... weak derivative, see host
  Real lpw[N];     // l_q(+1) / w_q
  Real lmw[N];     // l_q(-1) / w_q
  Real lp[N];      // l_q(+1)
  Real lm[N];      // l_q(-1)
  Real Sm[N][N];   // split to the lower child [l][k] (modal)
  Real Sp[N][N];   // split to the upper child [l][k] (modal)
  Real Snm[N][N];  // nodal split: Snm[i][j] = l_j((x_i - 1)/2), lower child
  Real Snp[N][N];  // nodal split: Snp[i][j] = l_j((x_i + 1)/2), upper child
};

// Decoded orientation of a (leaf, face): pi[a] in bits 2a..2a+1, sign bit
// of axis a in bit 6+a.
__device__ __forceinline__ int opi(int packed, int a) { return (packed >> (2 * a)) & 3; }
__device__ __forceinline__ int osg(int packed, int a) { return ((packed >> (6 + a)) & 1) ? -1 : 1; }

// ------------------------------------------------------------- tensor ops
// out[o] = sum_k A[qa(o)][k] in[o with qa -> k] along axis AX (compile time)
template <int D, int N, int AX, typename Real>
__device__ __forceinline__ void apply_axis(const Real (&A)[N][N], const Real* in, Real* out) {
  constexpr int S = ipow(N, AX);
  constexpr int M = ipow(N, D);
#pragma unroll
  for (int o = 0; o < M; ++o) {
    const int qa = (o / S) % N;
    const int base = o - qa * S;
    Real acc = Real(0);
#pragma unroll
    for (int k = 0; k < N; ++k) acc += A[qa][k] * in[base + k * S];
    out[o] = acc;
  }
}

// apply A along every axis: in -> out (in is clobbered)
template <int D, int N, typename Real>
__device__ __forceinline__ void apply_all(const Real (&A)[N][N], Real* a, Real* b) {
  apply_axis<D, N, 0, Real>(A, a, b);
  if constexpr (D == 1) {
#pragma unroll
    for (int i = 0; i < ipow(N, D); ++i) a[i] = b[i];
  } else if constexpr (D == 2) {
    apply_axis<D, N, 1, Real>(A, b, a);
  } else {
    apply_axis<D, N, 1, Real>(A, b, a);
    apply_axis<D, N, 2, Real>(A, a, b);
#pragma unroll
    for (int i = 0; i < ipow(N, D); ++i) a[i] = b[i];
  }
}

// --------------------------------------------------------------- geometry
// Trilinear (bilinear) map x(xi) = sum_c X_c prod_{a in c} xi_a; the kernels
// keep X_c for c = 1..2^D-1 (the constant term is not needed): coefficient
// (c, j) lives at g = (c-1)*D + j.
template <int D, typename Real>
__device__ __forceinline__ void tangents(const Real* X, int stride, const Real* xi,
                                         Real (&t)[D][D]) {
  // t[a][j] = d x_j / d xi_a
#define XC(c, j) X[(((c)-1) * D + (j)) * stride]
  if constexpr (D == 2) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      t[0][j] = XC(1, j) + XC(3, j) * xi[1];
      t[1][j] = XC(2, j) + XC(3, j) * xi[0];
    }
  } else {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      t[0][j] = XC(1, j) + XC(3, j) * xi[1] + XC(5, j) * xi[2] + XC(7, j) * xi[1] * xi[2];
      t[1][j] = XC(2, j) + XC(3, j) * xi[0] + XC(6, j) * xi[2] + XC(7, j) * xi[0] * xi[2];
      t[2][j] = XC(4, j) + XC(5, j) * xi[0] + XC(6, j) * xi[1] + XC(7, j) * xi[0] * xi[1];
    }
  }
#undef XC
}

// Row `dir` of J d xi/dx (contravariant basis vector scaled by J).
template <int D, typename Real>
__device__ __forceinline__ void contra_row(const Real (&t)[D][D], int dir, Real (&Ja)[D]) {
  if constexpr (D == 2) {
    if (dir == 0) {
      Ja[0] = t[1][1];
      Ja[1] = -t[1][0];
    } else {
      Ja[0] = -t[0][1];
      Ja[1] = t[0][0];
    }
  } else {
    const int i1 = (dir + 1) % 3, i2 = (dir + 2) % 3;
    Ja[0] = t[i1][1] * t[i2][2] - t[i1][2] * t[i2][1];
    Ja[1] = t[i1][2] * t[i2][0] - t[i1][0] * t[i2][2];
    Ja[2] = t[i1][0] * t[i2][1] - t[i1][1] * t[i2][0];
  }
}

template <int D, typename Real>
__device__ __forceinline__ Real jacobian_det(const Real (&t)[D][D]) {
  if constexpr (D == 2) {
    return t[0][0] * t[1][1] - t[1][0] * t[0][1];
  } else {
    Real c[3];
    contra_row<3, Real>(t, 0, c);
    return t[0][0] * c[0] + t[0][1] * c[1] + t[0][2] * c[2];
  }
}

// ------------------------------------------------------------------ Euler
// Flux along an (unnormalised) vector a: F . a  (Eq. (2), Eq. (23)).
template <int D, typename Real>
__device__ __forceinline__ void flux_along(const Real (&u)[D + 2], const Real (&a)[D], Real gm1,
                                           Real (&F)[D + 2]) {
  const Real ri = Real(1) / u[0];
  Real vn = Real(0), ke = Real(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    vn += u[1 + j] * a[j];
    ke += u[1 + j] * u[1 + j];
  }
  vn *= ri;
  const Real p = gm1 * (u[D + 1] - Real(0.5) * ke * ri);
  F[0] = u[0] * vn;
#pragma unroll
  for (int j = 0; j < D; ++j) F[1 + j] = u[1 + j] * vn + p * a[j];
  F[D + 1] = (u[D + 1] + p) * vn;
}

// Lax-Friedrichs flux (Eq. (5), dissipative sign) times the face area
// element: a = area vector pointing from L to R (|a| = dS / d(face ref)).
template <int D, typename Real>
__device__ __forceinline__ void lf_flux(const Real (&uL)[D + 2], const Real (&uR)[D + 2],
                                        const Real (&a)[D], Real gamma, Real (&Fh)[D + 2]) {
  const Real gm1 = gamma - Real(1);
  Real FL[D + 2], FR[D + 2];
  flux_along<D, Real>(uL, a, gm1, FL);
  flux_along<D, Real>(uR, a, gm1, FR);
  Real an2 = Real(0), vnL = Real(0), vnR = Real(0), keL = Real(0), keR = Real(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    an2 += a[j] * a[j];
    vnL += uL[1 + j] * a[j];
    vnR += uR[1 + j] * a[j];
    keL += uL[1 + j] * uL[1 + j];
    keR += uR[1 + j] * uR[1 + j];
  }
  const Real riL = Real(1) / uL[0], riR = Real(1) / uR[0];
  const Real pL = gm1 * (uL[D + 1] - Real(0.5) * keL * riL);
  const Real pR = gm1 * (uR[D + 1] - Real(0.5) * keR * riR);
  const Real an = sqrt(an2);
  const Real sL = fabs(vnL * riL) + sqrt(gamma * pL * riL) * an;
  const Real sR = fabs(vnR * riR) + sqrt(gamma * pR * riR) * an;
  // a NaN speed (negative pressure or density at a face point) propagates
  // into the flux, so the state and then the status word report it
  const Real alpha = (sL > sR || sL != sL) ? sL : sR;
#pragma unroll
  for (int v = 0; v < D + 2; ++v) Fh[v] = Real(0.5) * (FL[v] + FR[v] + alpha * (uL[v] - uR[v]));
}

// 16-byte vector <-> array of VEC elements (float4: 4 floats, double2: 2 doubles)
template <int VEC, typename V, typename Real>
__device__ __forceinline__ void vload(const V* p, Real (&a)[VEC]) {
  const V x = *p;
  a[0] = x.x;
  a[1] = x.y;
  if constexpr (VEC == 4) {
    a[2] = x.z;
    a[3] = x.w;
  }
}
template <int VEC, typename V, typename Real>
__device__ __forceinline__ void vstore(V* p, const Real (&a)[VEC]) {
  V x;
  x.x = a[0];
  x.y = a[1];
  if constexpr (VEC == 4) {
    x.z = a[2];
    x.w = a[3];
  }
  *p = x;
}

// ------------------------------------------------------------ kernel args
template <int D, int P, typename Real>
struct StageArgs {
  int nL, n, zchunk, nchunks;
  const Real* __restrict__ U;    // stage input U^(k)
  const Real* __restrict__ Un;   // U^n
  Real* __restrict__ Uout;       // stage output (or L(U) when mode == 1)
  const Real* __restrict__ geo;  // [b][g][cell] trilinear coefficients
  const Real* __restrict__ gtr;  // [b][f][v][fp][t] guard traces
  const Real* __restrict__ hcell;  // [b][cell]
  const unsigned char* __restrict__ affine;  // [b] 1 if every cell has the same constant metric
  const Real* __restrict__ ameta;  // [b][D*D+1]: rows of J dxi/dx, then 1/J
  const int* __restrict__ kind;    // [b][f] neighbour kind
  const int* __restrict__ nbr;     // [b][f][4]
  const int* __restrict__ orient;  // [b][f] packed decoded orientation
  const int* __restrict__ qbits;   // [b] pos & 1 bits
  const double* __restrict__ dtp;
  unsigned long long* lam_bits;
  int* status;
  Real ca, cb, gamma;
  int mode, last;
  const double* __restrict__ U64;  // compensated form: u^n in FP64 (the last stage's update)
  const float* __restrict__ Uhi;   // compensated form: u^n = hi + lo in FP32 (every stage input)
  const float* __restrict__ Ulo;
  const float* __restrict__ Din;   // compensated form: delta^(k), null at stage 1
  double* __restrict__ U64out;     // compensated form, last stage: u^(n+1) in FP64
  const unsigned char* __restrict__ fluxmask;  // [b] bit f: gtr holds face f's flux (mortar), or null
  // batch launch (every forest of a batch in one launch): per-forest
  // arguments in device memory, work items of forest m in
  // [istart[m], istart[m+1]); null for a single-forest launch
  const StageArgs* members;
  const int* istart;
  int nmem;
  Tab<P + 1, Real> T;
};

// index of the batch member whose range [start[m], start[m+1]) holds i
__device__ __forceinline__ int batch_member(const int* __restrict__ start, int nmem, int i) {
  int lo = 0, hi = nmem - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&start[mid]) <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// CTA minimum of v (one value per thread) folded into *dst with one atomic;
// every thread of the CTA calls it
template <int NTHR>
__device__ __forceinline__ void cta_min_atomic(double v, unsigned long long* dst) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u < v ? u : v;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (NTHR + 31) / 32 ? red[lane] : 3.0e38;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_xor_sync(0xffffffffu, v, o);
      v = u < v ? u : v;
    }
    // a CTA whose cells were all inadmissible contributes nothing, so a
    // broken state leaves no CFL value and the next dt is 0
    if (lane == 0 && v < 3.0e38) atomicMin(dst, (unsigned long long)__double_as_longlong(v));
  }
  __syncthreads();
}

// Stage input u^(k) at a flat index: one array (plain), or u^n plus the FP32
// increment delta^(k) (compensated SSP-RK3: the state accumulates in FP64,
// each stage changes it by an O(dt) increment kept in FP32).  The stages read
// u^n as the FP32 pair hi + lo (hi = fl(u^n), lo = fl(u^n - hi), split once per
// time step), so the input hi + (lo + delta) costs FP32 adds only; it is
// within one FP32 rounding of fl(u^n + delta).
template <typename Real, bool COMP>
struct StateIn {
  const Real* u;
  const double* u64;  // u^n in FP64 (the last stage's update reads it)
  const float* hi;
  const float* lo;
  const float* d;
  __device__ __forceinline__ Real operator()(size_t i) const {
    if constexpr (COMP) {
      float x = __ldcg(&lo[i]);
      if (d) x += __ldcg(&d[i]);
      return (Real)(__ldcg(&hi[i]) + x);
    } else {
      return u[i];
    }
  }
  // VEC = 16 / sizeof(Real) consecutive values from index i (a multiple of
  // VEC) with 16-byte L2 loads; element for element the same arithmetic as
  // operator()
  template <int VEC>
  __device__ __forceinline__ void vec(size_t i, Real (&a)[VEC]) const {
    static_assert(VEC * sizeof(Real) == 16, "16-byte groups");
    static_assert(!COMP || sizeof(Real) == 4, "the compensated form computes in FP32");
    if constexpr (COMP) {
      const float4 h = __ldcg(reinterpret_cast<const float4*>(hi + i));
      float4 x = __ldcg(reinterpret_cast<const float4*>(lo + i));
      if (d) {
        const float4 q = __ldcg(reinterpret_cast<const float4*>(d + i));
        x.x += q.x;
        x.y += q.y;
        x.z += q.z;
        x.w += q.w;
      }
      a[0] = h.x + x.x;
      a[1] = h.y + x.y;
      a[2] = h.z + x.z;
      a[3] = h.w + x.w;
    } else {
      using V = typename std::conditional<sizeof(Real) == 4, float4, double2>::type;
      const V q = __ldcg(reinterpret_cast<const V*>(u + i));
      a[0] = q.x;
      a[1] = q.y;
      if constexpr (VEC == 4) {
        a[2] = q.z;
        a[3] = q.w;
      }
    }
  }
};

template <int D, int P, typename Real>
struct GuardArgs {
  int nL, n, mode;  // mode 0: modal guard cells; 1: traces
  const Real* __restrict__ U;
  const double* __restrict__ U64;  // compensated form: u^n in FP64
  const float* __restrict__ Uhi;   // compensated form: u^n = hi + lo in FP32
  const float* __restrict__ Ulo;
  const float* __restrict__ Din;   // compensated form: delta^(k), null at stage 1
  Real* __restrict__ out;
  const int* __restrict__ kind;    // [b][f]
  const int* __restrict__ nbr;     // [b][f][4]
  const int* __restrict__ orient;  // [b][f] packed decoded orientation
  const int* __restrict__ qbits;   // [b] pos & 1 bits
  const int* __restrict__ copoff;  // [b][f] first combine operator << 1 | shared by all guard cells; -1: none
  const Real* __restrict__ cop;    // [op][2^D M][M]: column k' of the operator is contiguous
  const Real* __restrict__ ctr;    // [op][2^D M][NFP]: the same operator followed by my face trace
  const int* __restrict__ fine_list;  // [nfine] leaf * 2D + face of every finer-neighbour face
  int nfine;
  const int* __restrict__ trd;        // [b][f][8] face-trace descriptors (kinds 0, 1, 3), see k_guard_trace
  // mortar mode (reading R15)
  const Real* __restrict__ geo;       // [b][g][cell] trilinear coefficients
  Real gamma;
  const int* __restrict__ mfine;      // [nmf] leaf * 2D + face of every face with a coarser neighbour
  int nmf;
  const int* __restrict__ mcoarse;    // [nmc] leaf * 2D + face of every face with finer neighbours
  int nmc;
  const Real* __restrict__ mw;        // [nmc][NFP][2^(D-1) NFP] coarse point <- fine sub-face points
  const long long* __restrict__ msrc; // [nmc][nt][2^(D-1)] gtr offset of (fine leaf, face, v 0, point 0, t)
  const Real* __restrict__ bstate;    // [NV] state of prescribed-state boundary faces (kind 4)
  Tab<P + 1, Real> T;
};

// threads per CTA and CTAs per SM of the stage kernel (registers and shared
// memory decide: FP32 at p = 2 runs 2 x 448 threads per SM, 72 registers)
#ifndef DGF_STAGE_NT_F32
#define DGF_STAGE_NT_F32 448
#endif
// FP32 at p <= 1: smaller CTAs, four per SM (a layer's line work is a third
// of p = 2's; measured faster on forests of a thousand leaves and more,
// slower on the 71-leaf cube)
#ifndef DGF_STAGE_NT_F32_P1
#define DGF_STAGE_NT_F32_P1 256
#endif
#ifndef DGF_STAGE_MINB_F32_P1
#define DGF_STAGE_MINB_F32_P1 4
#endif
template <int P, typename Real>
struct StageCfg {
  static constexpr int NT = sizeof(Real) == 4 ? (P <= 1 ? DGF_STAGE_NT_F32_P1 : P <= 2 ? DGF_STAGE_NT_F32 : 512)
                                              : (P <= 1 ? 512 : 256);
  static constexpr int MINB = sizeof(Real) == 4 ? (P <= 1 ? DGF_STAGE_MINB_F32_P1 : P <= 2 ? 2 : 1) : 1;
};

// shared-memory footprint of the stage kernel (bytes): nodal layer, residual
// layer, x- and y-face fluxes, carried z-face flux
template <int D, int P, typename Real>
__host__ __device__ constexpr size_t stage_smem(int n, int rows) {
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D), NFP = ipow(N, D - 1);
  const size_t ncl = (size_t)n * rows;
  size_t us = NV * Q * ncl;
  size_t rs = us;
  size_t fx = (size_t)NV * NFP * (n + 1) * rows, fy = (size_t)NV * NFP * (rows + 1) * n;
  size_t fz = D == 3 ? (size_t)NV * NFP * ncl : 0;
  return (us + rs + fx + fy + fz) * sizeof(Real);
}

// rows of a layer one work item sweeps: the whole layer when its buffers fit
// the 227 KB of shared memory a CTA may use, else a slab of n/2, n/4, ...
// rows (FP64 at p = 3 with n = 8)
template <int D, int P, typename Real>
__host__ __device__ constexpr int stage_rows(int n) {
  int r = n;
  while (r > 1 && stage_smem<D, P, Real>(n, r) + 2048 > 232448) r /= 2;
  return r;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Metric along a line in direction DIR (coordinate s = xi_DIR) at fixed
// transverse reference coordinates: for a (bi/tri)linear map the tangents
// x_a (a != DIR) are affine in s and x_DIR is constant, so
//   J dxi_DIR/dx (s) = c0 + c1 s + c2 s^2,   J(s) = x_DIR . (J dxi_DIR/dx)(s).
template <int D, int DIR, typename Real>
struct LineGeo {
  Real c0[D], c1[D], c2[D], e[D];
  __device__ __forceinline__ void init(const Real* __restrict__ X, int stride, const Real* xi) {
    Real al[D][D], be[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int j = 0; j < D; ++j) al[a][j] = be[a][j] = Real(0);
#pragma unroll
    for (int c = 1; c < (1 << D); ++c) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (!((c >> a) & 1)) continue;
        Real fac = Real(1);
        bool has_s = false;
#pragma unroll
        for (int bb = 0; bb < D; ++bb) {
          if (bb == a || !((c >> bb) & 1)) continue;
          if (bb == DIR) has_s = true;
          else fac *= xi[bb];
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const Real x = __ldg(&X[((c - 1) * D + j) * stride]);
          if (has_s) be[a][j] += x * fac;
          else al[a][j] += x * fac;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < D; ++j) e[j] = al[DIR][j];
    if constexpr (D == 2) {
      const int o = 1 - DIR;
      const Real sg = DIR == 0 ? Real(1) : Real(-1);
      // DIR 0: (y_eta, -x_eta); DIR 1: (-y_xi, x_xi)
      c0[0] = sg * al[o][1];
      c0[1] = -sg * al[o][0];
      c1[0] = sg * be[o][1];
      c1[1] = -sg * be[o][0];
      c2[0] = c2[1] = Real(0);
    } else {
      constexpr int i1 = (DIR + 1) % 3, i2 = (DIR + 2) % 3;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        c0[j] = al[i1][j1] * al[i2][j2] - al[i1][j2] * al[i2][j1];
        c1[j] = al[i1][j1] * be[i2][j2] - al[i1][j2] * be[i2][j1] + be[i1][j1] * al[i2][j2] -
                be[i1][j2] * al[i2][j1];
        c2[j] = be[i1][j1] * be[i2][j2] - be[i1][j2] * be[i2][j1];
      }
    }
  }
  __device__ __forceinline__ void at(Real s, Real (&Ja)[D]) const {
#pragma unroll
    for (int j = 0; j < D; ++j) Ja[j] = c0[j] + s * (c1[j] + s * c2[j]);
  }
  __device__ __forceinline__ Real jac(const Real (&Ja)[D]) const {
    Real J = Real(0);
#pragma unroll
    for (int j = 0; j < D; ++j) J += e[j] * Ja[j];
    return J;
  }
};

// J dxi_DIR/dx at one reference point (faces), from the trilinear coefficients
template <int D, typename Real>
__device__ __forceinline__ void point_row(const Real* __restrict__ X, int stride, const Real* xi, int dir,
                                          Real (&Ja)[D]) {
  Real tg[D][D];
#define XC(c, j) __ldg(&X[(((c)-1) * D + (j)) * stride])
  if constexpr (D == 2) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      tg[0][j] = XC(1, j) + XC(3, j) * xi[1];
      tg[1][j] = XC(2, j) + XC(3, j) * xi[0];
    }
  } else {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (dir != 0) tg[0][j] = XC(1, j) + XC(3, j) * xi[1] + (XC(5, j) + XC(7, j) * xi[1]) * xi[2];
      if (dir != 1) tg[1][j] = XC(2, j) + XC(3, j) * xi[0] + (XC(6, j) + XC(7, j) * xi[0]) * xi[2];
      if (dir != 2) tg[2][j] = XC(4, j) + XC(5, j) * xi[0] + (XC(6, j) + XC(7, j) * xi[0]) * xi[1];
    }
  }
#undef XC
  contra_row<D, Real>(tg, dir, Ja);
}

// point index of face point fp (tangential digits, axes != ax in increasing
// order) with digit qn on the normal axis ax
template <int D, int N>
__device__ __forceinline__ int face_point_index(int ax, int fp, int qn) {
  constexpr int S1 = N, S2 = N * N;
  if constexpr (D == 2) {
    return ax == 0 ? qn + fp * S1 : fp + qn * S1;
  } else {
    const int a0 = fp % N, a1 = fp / N;
    if (ax == 0) return qn + a0 * S1 + a1 * S2;
    if (ax == 1) return a0 + qn * S1 + a1 * S2;
    return a0 + a1 * S1 + qn * S2;
  }
}

// ============================================================ stage kernel
// Persistent CTAs; work item = (leaf, z-chunk); a CTA sweeps the layers of
// its chunk.  Per layer: nodal values to shared memory; x and y face fluxes
// (each face once); x volume + lift; y volume + lift (and the halo trace of
// the next layer); z volume + z faces (carried between layers) and 1/J;
// SSP-RK combination point by point, with the CFL minimum on the last stage.
// BATCH: one launch for every forest of a batch (A.members; the tables and
// stage coefficients of A are common to all of them).
template <int D, int P, int NS, typename Real, bool COMP = false, bool MORTAR = false,
          int YS = stage_rows<D, P, Real>(NS), bool BATCH = false>
__global__ void __launch_bounds__(StageCfg<P, Real>::NT, StageCfg<P, Real>::MINB)
    k_stage(const __grid_constant__ StageArgs<D, P, Real> A) {
  static_assert(!(BATCH && (COMP || MORTAR)), "batches run the plain form without the mortar repair");
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D), NFP = ipow(N, D - 1);
  constexpr int NG = ((1 << D) - 1) * D;
  constexpr int n = NS;
  constexpr int YR = YS;                 // rows of the layer one item sweeps (a slab)
  constexpr int NYS = n / YR;            // slabs per layer
  constexpr int LAY = n * n;             // cells of a layer (of the block in 2D)
  constexpr int NCL = n * YR;            // cells of a slab
  constexpr int nc = D == 3 ? LAY * n : LAY;
  constexpr int nt = D == 3 ? n * n : n;  // guard cells per face
  constexpr int NFX = (n + 1) * YR * NFP;  // x faces of a slab
  constexpr int NFY = (YR + 1) * n * NFP;  // y faces of a slab
  const auto& T = A.T;
  const Real gamma = A.gamma;
  const Real gm1 = gamma - Real(1);
  Real dt = BATCH ? Real(0) : Real(*A.dtp);  // per forest of a batch: per item
  const int tid = threadIdx.x;
  constexpr int nthr = StageCfg<P, Real>::NT;
  if (!BATCH && A.mode == 0 && *A.dtp == 0.0) {
    // t_end reached: the increment is the identity and no stage is evaluated
    // (the CFL minimum of the last evaluated stage stays in place)
    if constexpr (COMP) {
      if (A.last) {
        const size_t tot = (size_t)A.nL * NV * Q * nc;
        for (size_t i = (size_t)blockIdx.x * nthr + tid; i < tot; i += (size_t)gridDim.x * nthr)
          A.U64out[i] = A.U64[i];
      }
    }
    return;
  }

  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Real sx[N];
  __shared__ Real sam[D * D + 1];
  constexpr int RSZ = NV * Q * NCL;
  Real* us = reinterpret_cast<Real*>(smem_raw);
  Real* rs = us + NV * Q * NCL;
  Real* fx = rs + RSZ;
  Real* fy = fx + NV * NFP * (n + 1) * YR;
  Real* fz = fy + NV * NFP * (YR + 1) * n;
  Real* tb = fx;   // halo traces reuse the x-face buffer when it is free
  if (tid < N) sx[tid] = T.x[tid];

  Real lam_min = Real(3.0e38);
  bool bad = false;
  const int items = BATCH ? __ldg(&A.istart[A.nmem]) : A.nL * A.nchunks * NYS;

#define US(v, q, c) us[((v) * Q + (q)) * NCL + (c)]
#define RS(v, q, c) rs[((v) * Q + (q)) * NCL + (c)]
// x faces: [v][fp][row j][face fi]; y faces: [v][fp][face fi][column i]
#define FX(v, fp, j, fi) fx[(((v) * NFP + (fp)) * YR + (j)) * (n + 1) + (fi)]
#define FY(v, fp, fi, i) fy[(((v) * NFP + (fp)) * (YR + 1) + (fi)) * n + (i)]
#define TB(v, fp, c) tb[((v) * NFP + (fp)) * NCL + (c)]
#define FZ(v, fp, c) fz[((v) * NFP + (fp)) * NCL + (c)]
#define GTR(f, v, fp, t) Tb[(((size_t)(f) * NV + (v)) * NFP + (fp)) * nt + (t)]

  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    // the forest of this item (a batch member, or the one forest)
    const StageArgs<D, P, Real>* Mp = &A;
    int li = item;
    if constexpr (BATCH) {
      const int m = batch_member(A.istart, A.nmem, item);
      Mp = A.members + m;
      li = item - __ldg(&A.istart[m]);
      if (A.mode == 0 && *Mp->dtp == 0.0) continue;  // that forest has reached its end time
      dt = Real(*Mp->dtp);
    }
    const StageArgs<D, P, Real>& M = *Mp;
    const int b = li / (M.nchunks * NYS);
    const int chunk = (li / NYS) % M.nchunks;
    const int j0 = NYS == 1 ? 0 : (li % NYS) * YR;  // first row of the slab
    const int k0 = D == 3 ? chunk * M.zchunk : 0;
    const int k1 = D == 3 ? min(n, k0 + M.zchunk) : 1;
    const Real* __restrict__ Ub = M.U + (size_t)b * NV * Q * nc;
    const Real* __restrict__ Unb = M.Un + (size_t)b * NV * Q * nc;
    const size_t boff = (size_t)b * NV * Q * nc;
    const StateIn<Real, COMP> Sb{M.U + boff, COMP ? M.U64 + boff : nullptr, COMP ? M.Uhi + boff : nullptr,
                                 COMP ? M.Ulo + boff : nullptr, (COMP && M.Din) ? M.Din + boff : nullptr};
    Real* __restrict__ Ob = M.Uout + (size_t)b * NV * Q * nc;
    const Real* __restrict__ Gb = M.geo + (size_t)b * NG * nc;
    const Real* __restrict__ Tb = M.gtr + (size_t)b * 2 * D * NV * NFP * nt;
    const Real* __restrict__ Hb = M.hcell + (size_t)b * nc;
    double* __restrict__ O64 = COMP ? M.U64out + boff : nullptr;
    const bool aff = M.affine[b] != 0;
    const int fmask = MORTAR ? M.fluxmask[b] : 0;  // faces whose flux is given (mortar mode)
    __syncthreads();  // previous item is done with the shared buffers
    if (aff && tid < D * D + 1) sam[tid] = M.ameta[(size_t)b * (D * D + 1) + tid];

    for (int k = k0; k < k1; ++k) {
      const int cbase = (D == 3 ? k * LAY : 0) + j0 * n;  // first cell of the slab
      const Real* __restrict__ Gk = Gb + cbase;  // geometry of this slab, stride nc
      // ------------------------------------------- L2 prefetch of what comes next
      {
        constexpr int lpr = (NCL * (int)sizeof(Real) + 127) / 128;
        for (int w = tid; w < NV * Q * lpr; w += nthr) {
          const int r = w / lpr, l = w - r * lpr;
          if constexpr (COMP) {
            if (D == 3 && k + 1 < n) {
              const size_t o = (size_t)r * nc + cbase + LAY + l * (128 / sizeof(Real));
              prefetch_l2(Sb.hi + o);
              prefetch_l2(Sb.lo + o);
              if (Sb.d) prefetch_l2(Sb.d + o);
            }
          } else {
            if (D == 3 && k + 1 < n) prefetch_l2(Ub + (size_t)r * nc + cbase + LAY + l * (128 / sizeof(Real)));
            if (A.mode == 0 && A.ca != Real(0)) prefetch_l2(Unb + (size_t)r * nc + cbase + l * (128 / sizeof(Real)));
          }
        }
      }
      // ------------------------------------------- P1: layer k to shared memory
      {
        constexpr int VEC = 16 / sizeof(Real);
        using V4 = typename std::conditional<sizeof(Real) == 4, float4, double2>::type;
        constexpr int PER_ROW = NCL / VEC;
        for (int w = tid; w < NV * Q * PER_ROW; w += nthr) {
          const int r = w / PER_ROW, cv = (w - r * PER_ROW) * VEC;
          Real x[VEC];
          Sb.template vec<VEC>((size_t)r * nc + cbase + cv, x);
          vstore<VEC>(reinterpret_cast<V4*>(us + r * NCL + cv), x);
        }
      }
      if constexpr (D == 3) {
        if (k == k0) {
          // halo trace below the first layer: guard (z-) or the layer below,
          // HV consecutive cells per thread with 16-byte loads and stores
          {
            constexpr int HV = 16 / (int)sizeof(Real);
            constexpr int NCV = NCL / HV;
            using V = typename std::conditional<sizeof(Real) == 4, float4, double2>::type;
            static_assert(NCL % HV == 0, "a slab holds whole 16-byte groups of cells");
            for (int w = tid; w < NCV * NV * NFP; w += nthr) {
              const int c0 = (w % NCV) * HV, fp = (w / NCV) % NFP, v = w / (NCV * NFP);
              Real tr[HV];
              if (k0 == 0) {
                vload<HV>(reinterpret_cast<const V*>(&GTR(4, v, fp, j0 * n + c0)), tr);
              } else {
#pragma unroll
                for (int e = 0; e < HV; ++e) tr[e] = Real(0);
#pragma unroll
                for (int qz = 0; qz < N; ++qz) {
                  Real x[HV];
                  Sb.template vec<HV>(((size_t)v * Q + fp + NFP * qz) * nc + cbase - LAY + c0, x);
#pragma unroll
                  for (int e = 0; e < HV; ++e) tr[e] += T.lp[qz] * x[e];
                }
              }
              vstore<HV>(reinterpret_cast<V*>(&TB(v, fp, c0)), tr);
            }
          }
          __syncthreads();
          for (int w = tid; w < NCL * NFP; w += nthr) {
            const int c = w % NCL, fp = w / NCL;
            if (k0 == 0 && (fmask & 16)) {
#pragma unroll
              for (int v = 0; v < NV; ++v) FZ(v, fp, c) = TB(v, fp, c);  // the z- face flux itself
              continue;
            }
            Real uL[NV], uR[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              uL[v] = TB(v, fp, c);
              Real s = Real(0);
#pragma unroll
              for (int qz = 0; qz < N; ++qz) s += T.lm[qz] * US(v, fp + NFP * qz, c);
              uR[v] = s;
            }
            Real Ja[3], Fh[NV];
            if (aff) {
#pragma unroll
              for (int j = 0; j < 3; ++j) Ja[j] = sam[6 + j];
            } else if (k0 == 0) {
              const Real xi[3] = {sx[fp % N], sx[fp / N], Real(-1)};
              point_row<3, Real>(Gk + c, nc, xi, 2, Ja);
            } else {
              // the metric of the layer below at its top face, exactly as the
              // carried flux of an unchunked sweep, so the result does not
              // depend on the chunk length
              const Real xi[3] = {sx[fp % N], sx[fp / N], Real(0)};
              LineGeo<3, 2, Real> lg;
              lg.init(Gk - LAY + c, nc, xi);
              lg.at(Real(1), Ja);
            }
            lf_flux<3, Real>(uL, uR, Ja, gamma, Fh);
#pragma unroll
            for (int v = 0; v < NV; ++v) FZ(v, fp, c) = Fh[v];
          }
        }
      }
      __syncthreads();

      // ------------------------------------------- P2: x and y face fluxes
      for (int w = tid; w < NFX + NFY; w += nthr) {
        const bool ydir = w >= NFX;
        const int ww = ydir ? w - NFX : w;
        Real uL[NV], uR[NV], Ja[D], Fh[NV];
        if (!ydir) {
          const int fi = ww % (n + 1);
          const int j = (ww / (n + 1)) % YR;
          const int fp = ww / ((n + 1) * YR);
          const int cl = (fi - 1) + n * j, cr = fi + n * j;
          const int tg = D == 3 ? j0 + j + n * k : j0 + j;  // guard cell of this row
          if ((fi == 0 && (fmask & 1)) || (fi == n && (fmask & 2))) {
#pragma unroll
            for (int v = 0; v < NV; ++v) FX(v, fp, j, fi) = GTR(fi == 0 ? 0 : 1, v, fp, tg);
            continue;
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            if (fi == 0) {
              uL[v] = GTR(0, v, fp, tg);
            } else {
              Real s = Real(0);
#pragma unroll
              for (int qx = 0; qx < N; ++qx) s += T.lp[qx] * US(v, qx + N * fp, cl);
              uL[v] = s;
            }
            if (fi == n) {
              uR[v] = GTR(1, v, fp, tg);
            } else {
              Real s = Real(0);
#pragma unroll
              for (int qx = 0; qx < N; ++qx) s += T.lm[qx] * US(v, qx + N * fp, cr);
              uR[v] = s;
            }
          }
          if (aff) {
#pragma unroll
            for (int jj = 0; jj < D; ++jj) Ja[jj] = sam[jj];
          } else {
            Real xi[D];
            xi[0] = fi == n ? Real(1) : Real(-1);
            xi[1] = sx[fp % N];
            if constexpr (D == 3) xi[2] = sx[fp / N];
            point_row<D, Real>(Gk + (fi == n ? cl : cr), nc, xi, 0, Ja);
          }
          lf_flux<D, Real>(uL, uR, Ja, gamma, Fh);
#pragma unroll
          for (int v = 0; v < NV; ++v) FX(v, fp, j, fi) = Fh[v];
        } else {
          const int i = ww % n;
          const int fi = (ww / n) % (YR + 1);
          const int fp = ww / ((YR + 1) * n);  // qx + N qz
          const int qx = fp % N, qz = fp / N;
          const int cl = i + n * (fi - 1), cr = i + n * fi;
          const int tg = D == 3 ? i + n * k : i;
          // block faces at the first and last row; a slab's other edge rows
          // take the neighbouring row's trace from the stage input in memory
          const bool bot = fi == 0 && j0 == 0, top = fi == YR && j0 + YR == n;
          if ((bot && (fmask & 4)) || (top && (fmask & 8))) {
#pragma unroll
            for (int v = 0; v < NV; ++v) FY(v, fp, fi, i) = GTR(bot ? 2 : 3, v, fp, tg);
            continue;
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            if (bot) {
              uL[v] = GTR(2, v, fp, tg);
            } else if (fi == 0) {
              Real s = Real(0);
#pragma unroll
              for (int qy = 0; qy < N; ++qy)
                s += T.lp[qy] * Sb(((size_t)v * Q + qx + N * qy + N * N * qz) * nc + cbase + cl);
              uL[v] = s;
            } else {
              Real s = Real(0);
#pragma unroll
              for (int qy = 0; qy < N; ++qy) s += T.lp[qy] * US(v, qx + N * qy + N * N * qz, cl);
              uL[v] = s;
            }
            if (top) {
              uR[v] = GTR(3, v, fp, tg);
            } else if (fi == YR) {
              Real s = Real(0);
#pragma unroll
              for (int qy = 0; qy < N; ++qy)
                s += T.lm[qy] * Sb(((size_t)v * Q + qx + N * qy + N * N * qz) * nc + cbase + cr);
              uR[v] = s;
            } else {
              Real s = Real(0);
#pragma unroll
              for (int qy = 0; qy < N; ++qy) s += T.lm[qy] * US(v, qx + N * qy + N * N * qz, cr);
              uR[v] = s;
            }
          }
          if (aff) {
#pragma unroll
            for (int jj = 0; jj < D; ++jj) Ja[jj] = sam[D + jj];
          } else {
            Real xi[D];
            xi[0] = sx[qx];
            xi[1] = top ? Real(1) : Real(-1);
            if constexpr (D == 3) xi[2] = sx[qz];
            point_row<D, Real>(Gk + (top ? cl : cr), nc, xi, 1, Ja);
          }
          lf_flux<D, Real>(uL, uR, Ja, gamma, Fh);
#pragma unroll
          for (int v = 0; v < NV; ++v) FY(v, fp, fi, i) = Fh[v];
        }
      }
      __syncthreads();
      // ------------------------------------------- P3: x volume + lift (rs =)
      for (int w = tid; w < NCL * NFP; w += nthr) {
        const int c = w % NCL, fp = w / NCL;
        const int i = c % n, j = c / n;
        Real xi[D];
        xi[0] = Real(0);
        xi[1] = sx[fp % N];
        if constexpr (D == 3) xi[2] = sx[fp / N];
        LineGeo<D, 0, Real> lg;
        if (!aff) lg.init(Gk + c, nc, xi);
        Real F[N][NV];
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          Real u[NV], Ja[D], Fq[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) u[v] = US(v, qx + N * fp, c);
          if (aff) {
#pragma unroll
            for (int jj = 0; jj < D; ++jj) Ja[jj] = sam[jj];
          } else {
            lg.at(T.x[qx], Ja);
          }
          flux_along<D, Real>(u, Ja, gm1, Fq);
#pragma unroll
          for (int v = 0; v < NV; ++v) F[qx][v] = Fq[v];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const Real fm = FX(v, fp, j, i);
          const Real fpl = FX(v, fp, j, i + 1);
#pragma unroll
          for (int qx = 0; qx < N; ++qx) {
            Real s = Real(0);
#pragma unroll
            for (int jj = 0; jj < N; ++jj) s += T.Sh[qx][jj] * F[jj][v];
            RS(v, qx + N * fp, c) = s - T.lpw[qx] * fpl + T.lmw[qx] * fm;
          }
        }
      }
      __syncthreads();
      // ------------------------------------------- P4: y volume + lift (rs +=)
      //                                            and the halo trace above
      constexpr int NY = NCL * NFP;
      // halo items: HV consecutive cells with 16-byte loads and stores
      constexpr int HV = 16 / (int)sizeof(Real);
      constexpr int ny_total = NY + ((D == 3) ? NCL * NV * NFP / HV : 0);
      static_assert(NCL % HV == 0, "a slab holds whole 16-byte groups of cells");
      for (int w = tid; w < ny_total; w += nthr) {
        if (w < NY) {
          const int c = w % NCL, fp = w / NCL;
          const int i = c % n, j = c / n;
          const int qx = fp % N, qz = fp / N;
          Real xi[D];
          xi[0] = sx[qx];
          xi[1] = Real(0);
          if constexpr (D == 3) xi[2] = sx[qz];
          LineGeo<D, 1, Real> lg;
          if (!aff) lg.init(Gk + c, nc, xi);
          Real F[N][NV];
          Real iJ[N];
#pragma unroll
          for (int qy = 0; qy < N; ++qy) {
            Real u[NV], Ja[D], Fq[NV];
            const int q = qx + N * qy + N * N * qz;
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v] = US(v, q, c);
            if (aff) {
#pragma unroll
              for (int jj = 0; jj < D; ++jj) Ja[jj] = sam[D + jj];
              iJ[qy] = sam[D * D];
            } else {
              lg.at(T.x[qy], Ja);
              if constexpr (D == 2) iJ[qy] = Real(1) / lg.jac(Ja);
            }
            flux_along<D, Real>(u, Ja, gm1, Fq);
#pragma unroll
            for (int v = 0; v < NV; ++v) F[qy][v] = Fq[v];
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const Real fm = FY(v, fp, j, i);
            const Real fpl = FY(v, fp, j + 1, i);
#pragma unroll
            for (int qy = 0; qy < N; ++qy) {
              Real s = Real(0);
#pragma unroll
              for (int jj = 0; jj < N; ++jj) s += T.Sh[qy][jj] * F[jj][v];
              const int q = qx + N * qy + N * N * qz;
              Real r = RS(v, q, c) + s - T.lpw[qy] * fpl + T.lmw[qy] * fm;
              if constexpr (D == 2) r *= iJ[qy];
              RS(v, q, c) = r;
            }
          }
        } else if constexpr (D == 3) {
          const int ww = w - NY;
          using V = typename std::conditional<sizeof(Real) == 4, float4, double2>::type;
          constexpr int NCV = NCL / HV;
          const int c0 = (ww % NCV) * HV, fp = (ww / NCV) % NFP, v = ww / (NCV * NFP);
          Real tr[HV];
          if (k == n - 1) {
            vload<HV>(reinterpret_cast<const V*>(&GTR(5, v, fp, j0 * n + c0)), tr);
          } else {
#pragma unroll
            for (int e = 0; e < HV; ++e) tr[e] = Real(0);
#pragma unroll
            for (int qz = 0; qz < N; ++qz) {
              Real x[HV];
              Sb.template vec<HV>(((size_t)v * Q + fp + NFP * qz) * nc + cbase + LAY + c0, x);
#pragma unroll
              for (int e = 0; e < HV; ++e) tr[e] += T.lm[qz] * x[e];
            }
          }
          vstore<HV>(reinterpret_cast<V*>(&TB(v, fp, c0)), tr);
        }
      }
      __syncthreads();

      if constexpr (D == 3) {
        // ------------------------------------------- P5: z volume + z faces, 1/J
        for (int w = tid; w < NCL * NFP; w += nthr) {
          const int c = w % NCL, fp = w / NCL;
          const int qx = fp % N, qy = fp / N;
          const Real xi[3] = {sx[qx], sx[qy], Real(0)};
          LineGeo<3, 2, Real> lg;
          if (!aff) lg.init(Gk + c, nc, xi);
          Real F[N][NV];
          Real iJ[N];
#pragma unroll
          for (int qz = 0; qz < N; ++qz) {
            Real u[NV], Ja[3], Fq[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v] = US(v, fp + NFP * qz, c);
            if (aff) {
#pragma unroll
              for (int jj = 0; jj < 3; ++jj) Ja[jj] = sam[6 + jj];
              iJ[qz] = sam[9];
            } else {
              lg.at(T.x[qz], Ja);
              iJ[qz] = Real(1) / lg.jac(Ja);
            }
            flux_along<3, Real>(u, Ja, gm1, Fq);
#pragma unroll
            for (int v = 0; v < NV; ++v) F[qz][v] = Fq[v];
          }
          // top face flux: own top trace vs the halo trace above
          Real uL[NV], uR[NV], Fh[NV], Ja[3];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            Real s = Real(0);
#pragma unroll
            for (int qz = 0; qz < N; ++qz) s += T.lp[qz] * US(v, fp + NFP * qz, c);
            uL[v] = s;
            uR[v] = TB(v, fp, c);
          }
          if (k == n - 1 && (fmask & 32)) {
#pragma unroll
            for (int v = 0; v < NV; ++v) Fh[v] = uR[v];  // the z+ face flux itself
          } else {
            if (aff) {
#pragma unroll
              for (int jj = 0; jj < 3; ++jj) Ja[jj] = sam[6 + jj];
            } else {
              lg.at(Real(1), Ja);
            }
            lf_flux<3, Real>(uL, uR, Ja, gamma, Fh);
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const Real fbot = FZ(v, fp, c);
#pragma unroll
            for (int qz = 0; qz < N; ++qz) {
              Real s = Real(0);
#pragma unroll
              for (int jj = 0; jj < N; ++jj) s += T.Sh[qz][jj] * F[jj][v];
              const int q = fp + NFP * qz;
              RS(v, q, c) = (RS(v, q, c) + s - T.lpw[qz] * Fh[v] + T.lmw[qz] * fbot) * iJ[qz];
            }
            FZ(v, fp, c) = Fh[v];
          }
        }
        __syncthreads();
      }

      // ------------------------------------------- P6: SSP-RK combination (+ CFL)
      {
        // VEC consecutive cells per thread: 16-byte shared and global accesses
        constexpr int VEC = 16 / sizeof(Real);
        using V = typename std::conditional<sizeof(Real) == 4, float4, double2>::type;
        constexpr int NCV = NCL / VEC;
        for (int w = tid; w < NCV * Q; w += nthr) {
          const int c0 = (w % NCV) * VEC, q = w / NCV;
          Real o[NV][VEC];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const size_t gi = ((size_t)v * Q + q) * nc + cbase + c0;
            Real r[VEC], val[VEC];
            vload<VEC>(reinterpret_cast<const V*>(&RS(v, q, c0)), r);
            if (A.mode == 1) {
#pragma unroll
              for (int e = 0; e < VEC; ++e) val[e] = r[e];
            } else if constexpr (COMP) {
              // delta^(k+1) = b_k (delta^(k) + dt L); last stage: u^(n+1) = u^n + delta^(3) in FP64
              Real din[VEC];
#pragma unroll
              for (int e = 0; e < VEC; ++e) din[e] = Real(0);
              if (Sb.d) {
                const float4 x = __ldcg(reinterpret_cast<const float4*>(Sb.d + gi));
                vload<VEC>(&x, din);
              }
#pragma unroll
              for (int e = 0; e < VEC; ++e) val[e] = A.cb * (din[e] + dt * r[e]);
              if (A.last) {
#pragma unroll
                for (int e = 0; e < VEC; e += 2) {
                  const double2 un = __ldcg(reinterpret_cast<const double2*>(Sb.u64 + gi + e));
                  const double2 nw = make_double2(un.x + (double)val[e], un.y + (double)val[e + 1]);
                  *reinterpret_cast<double2*>(O64 + gi + e) = nw;
                  val[e] = (Real)nw.x;
                  val[e + 1] = (Real)nw.y;
                }
              }
            } else {
              Real u[VEC];
              vload<VEC>(reinterpret_cast<const V*>(&US(v, q, c0)), u);
#pragma unroll
              for (int e = 0; e < VEC; ++e) val[e] = A.cb * (u[e] + dt * r[e]);
              if (A.ca != Real(0)) {
                Real un[VEC];
                const V x = __ldcg(reinterpret_cast<const V*>(&Unb[gi]));
                vload<VEC>(&x, un);
#pragma unroll
                for (int e = 0; e < VEC; ++e) val[e] += A.ca * un[e];
              }
            }
            // the compensated last stage keeps its result in FP64 only
            if (!(COMP && A.mode != 1 && A.last)) vstore<VEC>(reinterpret_cast<V*>(&Ob[gi]), val);
#pragma unroll
            for (int e = 0; e < VEC; ++e) o[v][e] = val[e];
          }
          if (A.last) {
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
              const Real ri = Real(1) / o[0][e];
              Real ke = Real(0), sv = Real(0);
#pragma unroll
              for (int jj = 0; jj < D; ++jj) {
                ke += o[1 + jj][e] * o[1 + jj][e];
                sv += fabs(o[1 + jj][e]) * ri;
              }
              const Real pr = gm1 * (o[D + 1][e] - Real(0.5) * ke * ri);
              if (!(o[0][e] > Real(0)) || !(pr > Real(0)) || !(pr < Real(3.0e38))) {
                bad = true;
              } else {
                const Real lam = sv + Real(D) * sqrt(gamma * pr * ri);
                const Real hv = Hb[cbase + c0 + e] / lam;
                lam_min = hv < lam_min ? hv : lam_min;
              }
            }
          }
        }
      }
      __syncthreads();
    }
    if constexpr (BATCH) {
      // the CFL minimum and the status belong to this item's forest
      if (A.last) {
        cta_min_atomic<nthr>((double)lam_min, M.lam_bits);
        lam_min = Real(3.0e38);
        if (__syncthreads_or(bad) && tid == 0) atomicExch(M.status, kStatusNonFinite);
        bad = false;
      }
    }
  }
#undef US
#undef RS
#undef FX
#undef FY
#undef TB
#undef FZ
#undef GTR

  if (!BATCH && A.last) {
    // block min of h/lambda -> one atomic per CTA
    double v = (double)lam_min;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double u = __shfl_xor_sync(0xffffffffu, v, o);
      v = u < v ? u : v;
    }
    __shared__ double red[32];
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
      v = lane < (nthr + 31) / 32 ? red[lane] : 3.0e38;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
      }
      // a CTA whose cells were all inadmissible contributes nothing, so a
      // broken state leaves no CFL value and the next dt is 0
      if (lane == 0 && v < 3.0e38) atomicMin(A.lam_bits, (unsigned long long)__double_as_longlong(v));
    }
    if (bad) atomicExch(A.status, kStatusNonFinite);
  }
}

// ============================================================ guard kernels
// Sec. 3.5, Eqs. (15)-(17), on nodal values.  The stage kernel needs, for
// every block face, the guard cell's trace at my face Gauss points in my
// frame (mode 1); the C ABI's standalone fill needs the guard cells' values
// at my Gauss points (mode 0, converted to modes afterwards).  Same-level
// and coarser neighbours: the trace is taken in the neighbour's frame and
// scattered into my point order (rotations map Gauss points onto Gauss
// points).  Finer neighbours use k_guard_fine.

// source-frame face point j -> my face point index, for my face axis a and
// the neighbour's face axis b2 (orientation packed as in opi/osg)
template <int D, int N>
__device__ __forceinline__ int map_face_point(int j, int a, int b2, int pk) {
  if constexpr (D == 2) {
    const int t0 = 1 - a;  // my only tangential axis
    return osg(pk, t0) > 0 ? j : N - 1 - j;
  } else {
    const int u0 = b2 == 0 ? 1 : 0;  // first source tangential axis
    const int qu0 = j % N, qu1 = j / N;
    const int t0 = a == 0 ? 1 : 0, t1 = a == 2 ? 1 : 2;  // my tangential axes
    const int s0 = opi(pk, t0) == u0 ? qu0 : qu1;
    const int s1 = opi(pk, t1) == u0 ? qu0 : qu1;
    const int q0 = osg(pk, t0) > 0 ? s0 : N - 1 - s0;
    const int q1 = osg(pk, t1) > 0 ? s1 : N - 1 - s1;
    return q0 + N * q1;
  }
}

// source-frame volume point (digits js[]) -> my point index
template <int D, int N>
__device__ __forceinline__ int map_point(const int* js, int pk) {
  int m = 0, st = 1;
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    const int d = js[opi(pk, ax)];
    m += (osg(pk, ax) > 0 ? d : N - 1 - d) * st;
    st *= N;
  }
  return m;
}

// one thread per (leaf, face, guard cell t, var); finer faces are skipped
template <int D, int P, typename Real, bool COMP = false>
__global__ void __launch_bounds__(128) k_guard(const GuardArgs<D, P, Real> A) {
  const StateIn<Real, COMP> S{A.U, A.U64, A.Uhi, A.Ulo, A.Din};
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D), NFP = ipow(N, D - 1);
  const int n = A.n;
  const int nt = D == 3 ? n * n : n;
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t total = (size_t)A.nL * 2 * D * nt * NV;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= total) return;
  const int t = (int)(w % nt);
  const int v = (int)((w / nt) % NV);
  const int f = (int)((w / ((size_t)nt * NV)) % (2 * D));
  const int b = (int)(w / ((size_t)nt * NV * 2 * D));
  const int a = f >> 1, s = f & 1;
  const int kind = A.kind[b * 2 * D + f];
  if (kind == 2) return;
  const auto& T = A.T;
  int g[3] = {0, 0, 0};
  {
    int j = 0;
    for (int ax = 0; ax < D; ++ax) {
      if (ax == a) continue;
      g[ax] = j == 0 ? (t % n) : (t / n);
      ++j;
    }
  }
  const int pk = A.orient[b * 2 * D + f];
  auto cell_of = [&](const int* h) {
    int c = 0, st = 1;
    for (int ax = 0; ax < D; ++ax) {
      c += h[ax] * st;
      st *= n;
    }
    return c;
  };
  Real* out_vol = A.out + (((size_t)b * 2 * D + f) * NV + v) * Q * nt + t;
  Real* out_trace = A.out + (((size_t)b * 2 * D + f) * NV + v) * NFP * nt + t;

  if (kind == 4) {  // prescribed state: a constant guard cell
    const Real u = A.bstate[v];
    if (A.mode == 0) {
#pragma unroll
      for (int q = 0; q < Q; ++q) out_vol[(size_t)q * nt] = u;
    } else {
#pragma unroll
      for (int fp = 0; fp < NFP; ++fp) out_trace[(size_t)fp * nt] = u;
    }
    return;
  }
  if (kind == 3) {  // outflow: the guard is the mirror image of my face cell
    int h[3] = {g[0], g[1], g[2]};
    h[a] = s ? n - 1 : 0;
    const size_t src0 = ((size_t)b * NV + v) * Q * nc + cell_of(h);
    if (A.mode == 0) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        int d[3] = {q % N, (q / N) % N, q / (N * N)};
        d[a] = N - 1 - d[a];
        out_vol[(size_t)q * nt] = S(src0 + (size_t)(d[0] + N * d[1] + N * N * d[2]) * nc);
      }
    } else {
#pragma unroll
      for (int fp = 0; fp < NFP; ++fp) {
        Real acc = Real(0);
#pragma unroll
        for (int qn = 0; qn < N; ++qn)
          acc += (s ? T.lp[qn] : T.lm[qn]) * S(src0 + (size_t)face_point_index<D, N>(a, fp, qn) * nc);
        out_trace[(size_t)fp * nt] = acc;
      }
    }
    return;
  }
  const int b2 = opi(pk, a);
  const int s2 = osg(pk, a) > 0 ? 1 - s : s;
  int h[3] = {0, 0, 0}, e[3] = {0, 0, 0};
  if (kind == 0) {
    for (int ax = 0; ax < D; ++ax) {
      if (ax == a) continue;
      h[opi(pk, ax)] = osg(pk, ax) > 0 ? g[ax] : n - 1 - g[ax];
    }
  } else {  // coarser: my guard is child e of the coarse cell h (neighbour frame)
    const int qb = A.qbits[b];
    for (int ax = 0; ax < D; ++ax) {
      if (ax == a) continue;
      const int G = ((qb >> ax) & 1) * n + g[ax];
      const int hh = G >> 1, ee = G & 1;
      h[opi(pk, ax)] = osg(pk, ax) > 0 ? hh : n - 1 - hh;
      e[opi(pk, ax)] = osg(pk, ax) > 0 ? ee : 1 - ee;
    }
    e[b2] = s2 == 0 ? 0 : 1;
  }
  h[b2] = s2 == 0 ? 0 : n - 1;
  const size_t src0 = ((size_t)A.nbr[(b * 2 * D + f) * 4] * NV + v) * Q * nc + cell_of(h);

  if (A.mode == 1) {
    // trace on the neighbour's face (b2, s2) at its face points
    Real tr[NFP];
#pragma unroll
    for (int j = 0; j < NFP; ++j) {
      Real acc = Real(0);
#pragma unroll
      for (int qn = 0; qn < N; ++qn)
        acc += (s2 ? T.lp[qn] : T.lm[qn]) * S(src0 + (size_t)face_point_index<D, N>(b2, j, qn) * nc);
      tr[j] = acc;
    }
    if (kind == 1) {
      // split (Eqs. (11)-(12)): interpolate the coarse face trace to the
      // Gauss points of the child face, along each tangential axis
      Real t2[NFP];
      if constexpr (D == 2) {
        const int u0 = 1 - b2;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          Real acc = Real(0);
#pragma unroll
          for (int jj = 0; jj < N; ++jj) acc += (e[u0] ? T.Snp[i][jj] : T.Snm[i][jj]) * tr[jj];
          t2[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) tr[i] = t2[i];
      } else {
        const int u0 = b2 == 0 ? 1 : 0, u1 = b2 == 2 ? 1 : 2;
#pragma unroll
        for (int i1 = 0; i1 < N; ++i1)
#pragma unroll
          for (int i0 = 0; i0 < N; ++i0) {
            Real acc = Real(0);
#pragma unroll
            for (int jj = 0; jj < N; ++jj) acc += (e[u0] ? T.Snp[i0][jj] : T.Snm[i0][jj]) * tr[jj + N * i1];
            t2[i0 + N * i1] = acc;
          }
#pragma unroll
        for (int i1 = 0; i1 < N; ++i1)
#pragma unroll
          for (int i0 = 0; i0 < N; ++i0) {
            Real acc = Real(0);
#pragma unroll
            for (int jj = 0; jj < N; ++jj) acc += (e[u1] ? T.Snp[i1][jj] : T.Snm[i1][jj]) * t2[i0 + N * jj];
            tr[i0 + N * i1] = acc;
          }
      }
    }
#pragma unroll
    for (int j = 0; j < NFP; ++j) out_trace[(size_t)map_face_point<D, N>(j, a, b2, pk) * nt] = tr[j];
    return;
  }
  // mode 0: full guard cell at my Gauss points
  Real u[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) u[q] = S(src0 + (size_t)q * nc);
  if (kind == 1) {
    Real u2[Q];
    if (e[0]) apply_axis<D, N, 0, Real>(T.Snp, u, u2);
    else apply_axis<D, N, 0, Real>(T.Snm, u, u2);
    if (e[1]) apply_axis<D, N, 1, Real>(T.Snp, u2, u);
    else apply_axis<D, N, 1, Real>(T.Snm, u2, u);
    if constexpr (D == 3) {
      if (e[2]) apply_axis<D, N, 2, Real>(T.Snp, u, u2);
      else apply_axis<D, N, 2, Real>(T.Snm, u, u2);
#pragma unroll
      for (int q = 0; q < Q; ++q) u[q] = u2[q];
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int js[3] = {q % N, (q / N) % N, q / (N * N)};
    out_vol[(size_t)map_point<D, N>(js, pk) * nt] = u[q];
  }
}

// Finer neighbours (Eqs. (13)-(14)): one CTA per (finer face, guard cell t,
// var) with one warp per fine child e; warp e applies child e's columns of
// the precomputed, already rotated nodal operator, the partial sums are
// added in fixed child order, and (mode 1) the trace at my face is formed.
template <int D, int P, typename Real, bool COMP = false>
__global__ void __launch_bounds__(32 << D) k_guard_fine(const GuardArgs<D, P, Real> A) {
  const StateIn<Real, COMP> S{A.U, A.U64, A.Uhi, A.Ulo, A.Din};
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D), NFP = ipow(N, D - 1);
  constexpr int NW = 1 << D;
  constexpr int KC = NW * Q;
  __shared__ Real srcs[NW][Q];
  __shared__ Real part[NW][Q];
  const int n = A.n;
  const int nt = D == 3 ? n * n : n;
  const int nc = D == 3 ? n * n * n : n * n;
  const int lane = threadIdx.x & 31, e = threadIdx.x >> 5;
  const size_t item = blockIdx.x;
  const int t = (int)(item % nt);
  const int v = (int)((item / nt) % NV);
  const int bf = A.fine_list[item / ((size_t)nt * NV)];
  const int b = bf / (2 * D), f = bf % (2 * D);
  const int a = f >> 1, s = f & 1;
  const int pk = A.orient[bf];
  const auto& T = A.T;
  int g[3] = {0, 0, 0};
  {
    int j = 0;
    for (int ax = 0; ax < D; ++ax) {
      if (ax == a) continue;
      g[ax] = j == 0 ? (t % n) : (t / n);
      ++j;
    }
  }
  const int b2 = opi(pk, a);
  const int s2 = osg(pk, a) > 0 ? 1 - s : s;
  int h[3] = {0, 0, 0}, sub = 0, j = 0;
  for (int ax = 0; ax < D; ++ax) {
    if (ax == a) continue;
    h[opi(pk, ax)] = osg(pk, ax) > 0 ? g[ax] : n - 1 - g[ax];
    if (g[ax] >= n / 2) sub |= 1 << j;
    ++j;
  }
  h[b2] = s2 == 0 ? 0 : n - 1;
  const int fine = A.nbr[bf * 4 + sub];
  int c = 0, st = 1;
  for (int ax = 0; ax < D; ++ax) {
    const int cN = (2 * h[ax]) / n;
    c += (2 * h[ax] + ((e >> ax) & 1) - cN * n) * st;
    st *= n;
  }
  for (int q = lane; q < Q; q += 32) srcs[e][q] = S((((size_t)fine * NV + v) * Q + q) * nc + c);
  __syncwarp();
  const int co = A.copoff[bf];  // first operator << 1 | one operator shared by every guard cell
  const Real* op = A.cop + ((size_t)(co >> 1) + ((co & 1) ? 0 : t)) * KC * Q + (size_t)e * Q * Q;
  for (int p = lane; p < Q; p += 32) {
    Real acc0 = Real(0), acc1 = Real(0);
#pragma unroll 4
    for (int q = 0; q + 1 < Q; q += 2) {
      acc0 += __ldg(&op[(size_t)q * Q + p]) * srcs[e][q];
      acc1 += __ldg(&op[(size_t)(q + 1) * Q + p]) * srcs[e][q + 1];
    }
    if (Q & 1) acc0 += __ldg(&op[(size_t)(Q - 1) * Q + p]) * srcs[e][Q - 1];
    part[e][p] = acc0 + acc1;
  }
  __syncthreads();
  if (e != 0) return;
  Real* K = srcs[0];  // reuse: every warp is past its reads of srcs
  for (int p = lane; p < Q; p += 32) {
    Real acc = Real(0);
#pragma unroll
    for (int ee = 0; ee < NW; ++ee) acc += part[ee][p];
    if (A.mode == 0) A.out[((((size_t)b * 2 * D + f) * NV + v) * Q + p) * nt + t] = acc;
    K[p] = acc;
  }
  if (A.mode == 0) return;
  __syncwarp();
  // trace of the guard cell (my frame) on its face touching me: xi_a = -+1
  for (int fp = lane; fp < NFP; fp += 32) {
    Real acc = Real(0);
    for (int qn = 0; qn < N; ++qn) acc += (s ? T.lm[qn] : T.lp[qn]) * K[face_point_index<D, N>(a, fp, qn)];
    A.out[((((size_t)b * 2 * D + f) * NV + v) * NFP + fp) * nt + t] = acc;
  }
}

// Guard traces for the time step (mode 1), one launch: the first
// n_fine_blocks blocks run the finer-face combine (one block per finer face
// and guard cell, all vars, one warp per fine child), the remaining blocks
// compute the traces of same-level, coarser, outflow and prescribed-state
// faces, one thread per (leaf, face, guard cell, var), from the host-built
// face-trace descriptors (source cell and face points as affine functions
// of my guard-cell and face-point digits).
// The body handles block `bid` of one forest's launch; k_guard_trace runs it
// for one forest, k_guard_trace_batch for the forests of a batch (each
// forest's blocks after the previous forests').
template <int D, int P, typename Real, bool COMP = false>
__device__ __forceinline__ void guard_trace_block(const GuardArgs<D, P, Real>& A, int n_fine_blocks, unsigned bid) {
  const StateIn<Real, COMP> S{A.U, A.U64, A.Uhi, A.Ulo, A.Din};
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D), NFP = ipow(N, D - 1);
  constexpr int NW = 1 << D;
  constexpr int KC = NW * Q;
  constexpr int NTH = 32 << D;
  const int n = A.n;
  const int nt = D == 3 ? n * n : n;
  const int nc = D == 3 ? n * n * n : n * n;
  const auto& T = A.T;
  // n and nt are powers of two: guard-cell digits by shifts and masks (the
  // launch keeps the thread count below 2^32)
  const int ln = 31 - __clz(n), lnt = (D - 1) * ln;
  if ((int)bid >= n_fine_blocks) {
    const size_t total = (size_t)A.nL * 2 * D * nt * NV;
    const size_t wl = (size_t)(bid - n_fine_blocks) * NTH + threadIdx.x;
    if (wl >= total) return;
    const unsigned w = (unsigned)wl;
    const int t = (int)(w & (unsigned)(nt - 1));
    const unsigned r = w >> lnt;
    const int v = (int)(r % NV);
    const int f = (int)((r / NV) % (2 * D));
    const int b = (int)(r / (NV * 2 * D));
    const int kind = A.kind[b * 2 * D + f];
    if (kind == 2) return;
    Real* out_trace = A.out + (((size_t)b * 2 * D + f) * NV + v) * NFP * nt + t;
    if (kind == 4) {  // prescribed state
#pragma unroll
      for (int fp = 0; fp < NFP; ++fp) out_trace[(size_t)fp * nt] = A.bstate[v];
      return;
    }
    // same-level, coarser or outflow (my own face cell): the source cell and
    // its face points are affine in my guard-cell and face-point digits, the
    // orientation folded into signed strides (host-built descriptor)
    const int4 d0 = __ldg(reinterpret_cast<const int4*>(A.trd + (size_t)(b * 2 * D + f) * 8));
    const int4 d1 = __ldg(reinterpret_cast<const int4*>(A.trd + (size_t)(b * 2 * D + f) * 8 + 4));
    int g0 = t & (n - 1), g1 = t >> ln;
    int e0 = 0, e1 = 0;
    if (kind == 1) {
      // my position on the coarse face: coarse cell G >> 1, child half G & 1
      const int a = f >> 1, qb = A.qbits[b];
      const int t0 = a == 0 ? 1 : 0, t1 = a == 2 ? 1 : 2;  // my tangential axes
      const int G0 = ((qb >> t0) & 1) * n + g0;
      e0 = G0 & 1;
      g0 = G0 >> 1;
      if constexpr (D == 3) {
        const int G1 = ((qb >> t1) & 1) * n + g1;
        e1 = G1 & 1;
        g1 = G1 >> 1;
      }
    }
    const size_t src0 = ((size_t)d0.x * NV + v) * Q * nc + (d0.y + g0 * d0.z + g1 * d0.w) + d1.x;
    const int PN = d1.w >> 1;
    Real lq[N];
#pragma unroll
    for (int qn = 0; qn < N; ++qn) lq[qn] = (d1.w & 1) ? T.lp[qn] : T.lm[qn];
    Real tr[NFP];
#pragma unroll
    for (int q1 = 0; q1 < (D == 3 ? N : 1); ++q1)
#pragma unroll
      for (int q0 = 0; q0 < N; ++q0) {
        Real acc = Real(0);
#pragma unroll
        for (int qn = 0; qn < N; ++qn) acc += lq[qn] * S(src0 + (ptrdiff_t)(q0 * d1.y + q1 * d1.z + qn * PN));
        tr[q0 + N * q1] = acc;
      }
    if (kind == 1) {  // split (Eqs. (11)-(12)) of the coarse face trace, in my frame
      Real t2[NFP];
      if constexpr (D == 2) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          Real acc = Real(0);
#pragma unroll
          for (int jj = 0; jj < N; ++jj) acc += (e0 ? T.Snp[i][jj] : T.Snm[i][jj]) * tr[jj];
          t2[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) tr[i] = t2[i];
      } else {
#pragma unroll
        for (int i1 = 0; i1 < N; ++i1)
#pragma unroll
          for (int i0 = 0; i0 < N; ++i0) {
            Real acc = Real(0);
#pragma unroll
            for (int jj = 0; jj < N; ++jj) acc += (e0 ? T.Snp[i0][jj] : T.Snm[i0][jj]) * tr[jj + N * i1];
            t2[i0 + N * i1] = acc;
          }
#pragma unroll
        for (int i1 = 0; i1 < N; ++i1)
#pragma unroll
          for (int i0 = 0; i0 < N; ++i0) {
            Real acc = Real(0);
#pragma unroll
            for (int jj = 0; jj < N; ++jj) acc += (e1 ? T.Snp[i1][jj] : T.Snm[i1][jj]) * t2[i0 + N * jj];
            tr[i0 + N * i1] = acc;
          }
      }
    }
#pragma unroll
    for (int j = 0; j < NFP; ++j) out_trace[(size_t)j * nt] = tr[j];
    return;
  }
  // ---- finer faces: one block per (finer face, guard cell t), all vars;
  // warp e applies fine child e's columns of the trace operator
  constexpr int NPAIR = NV * NFP;
  __shared__ Real sv[NW][NV][Q];
  __shared__ Real pv[NW][NPAIR];
  const unsigned item = bid;
  const int lane = threadIdx.x & 31, e = threadIdx.x >> 5;
  const int t = (int)(item & (unsigned)(nt - 1));
  const int bf = A.fine_list[item >> lnt];
  const int b = bf / (2 * D), f = bf % (2 * D);
  const int a = f >> 1, s = f & 1;
  const int pk = A.orient[bf];
  int g[3] = {0, 0, 0};
  {
    int j = 0;
    for (int ax = 0; ax < D; ++ax) {
      if (ax == a) continue;
      g[ax] = j == 0 ? (t % n) : (t / n);
      ++j;
    }
  }
  const int b2 = opi(pk, a);
  const int s2 = osg(pk, a) > 0 ? 1 - s : s;
  int h[3] = {0, 0, 0}, sub = 0, j = 0;
  for (int ax = 0; ax < D; ++ax) {
    if (ax == a) continue;
    h[opi(pk, ax)] = osg(pk, ax) > 0 ? g[ax] : n - 1 - g[ax];
    if (g[ax] >= n / 2) sub |= 1 << j;
    ++j;
  }
  h[b2] = s2 == 0 ? 0 : n - 1;
  const int fine = A.nbr[bf * 4 + sub];
  int c = 0, st = 1;
  for (int ax = 0; ax < D; ++ax) {
    const int cN = (2 * h[ax]) / n;
    c += (2 * h[ax] + ((e >> ax) & 1) - cN * n) * st;
    st *= n;
  }
  for (int i = lane; i < NV * Q; i += 32) {
    const int v = i / Q, q = i % Q;
    sv[e][v][q] = S((((size_t)fine * NV + v) * Q + q) * nc + c);
  }
  __syncwarp();
  const int co = A.copoff[bf];  // first operator << 1 | one operator shared by every guard cell
  const Real* op = A.ctr + ((size_t)(co >> 1) + ((co & 1) ? 0 : t)) * KC * NFP + (size_t)e * Q * NFP;
  for (int pr = lane; pr < NPAIR; pr += 32) {
    const int v = pr / NFP, fp = pr % NFP;
    Real acc0 = Real(0), acc1 = Real(0);
#pragma unroll 4
    for (int q = 0; q + 1 < Q; q += 2) {
      acc0 += __ldg(&op[(size_t)q * NFP + fp]) * sv[e][v][q];
      acc1 += __ldg(&op[(size_t)(q + 1) * NFP + fp]) * sv[e][v][q + 1];
    }
    if (Q & 1) acc0 += __ldg(&op[(size_t)(Q - 1) * NFP + fp]) * sv[e][v][Q - 1];
    pv[e][pr] = acc0 + acc1;
  }
  __syncthreads();
  for (int pr = threadIdx.x; pr < NPAIR; pr += NTH) {
    Real acc = Real(0);
#pragma unroll
    for (int ee = 0; ee < NW; ++ee) acc += pv[ee][pr];
    const int v = pr / NFP, fp = pr % NFP;
    A.out[((((size_t)b * 2 * D + f) * NV + v) * NFP + fp) * nt + t] = acc;
  }
}

template <int D, int P, typename Real, bool COMP = false>
__global__ void __launch_bounds__(32 << D) k_guard_trace(const __grid_constant__ GuardArgs<D, P, Real> A,
                                                         int n_fine_blocks) {
  guard_trace_block<D, P, Real, COMP>(A, n_fine_blocks, blockIdx.x);
}

// guard traces of every forest of a batch in one launch: block ranges per
// forest in bstart (prefix sums of n_fine_blocks + trace blocks)
template <int D, int P, typename Real>
__global__ void __launch_bounds__(32 << D) k_guard_trace_batch(const GuardArgs<D, P, Real>* __restrict__ As,
                                                               const int* __restrict__ bstart,
                                                               const int* __restrict__ nfb, int nmem) {
  const int m = batch_member(bstart, nmem, (int)blockIdx.x);
  guard_trace_block<D, P, Real, false>(As[m], __ldg(&nfb[m]), blockIdx.x - (unsigned)__ldg(&bstart[m]));
}

// ============================================================ mortar mode
// Reading R15.  Fine side: at every face point of a face with a coarser
// neighbour, the Lax-Friedrichs flux along +xi_a (Eq. (5), reading R3) from
// my own trace and the prolonged coarse trace already in the guard-trace
// buffer, with my face metric; it overwrites that trace, and the stage kernel
// takes it as the face flux.  One thread per (face, guard cell, face point).
template <int D, int P, typename Real, bool COMP = false>
__global__ void __launch_bounds__(128) k_mortar_fine(const GuardArgs<D, P, Real> A) {
  const StateIn<Real, COMP> S{A.U, A.U64, A.Uhi, A.Ulo, A.Din};
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D), NFP = ipow(N, D - 1);
  constexpr int NG = ((1 << D) - 1) * D;
  const int n = A.n;
  const int nt = D == 3 ? n * n : n;
  const int nc = D == 3 ? n * n * n : n * n;
  const auto& T = A.T;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (size_t)A.nmf * nt * NFP) return;
  const int fp = (int)(w % NFP);
  const int t = (int)((w / NFP) % nt);
  const int bf = A.mfine[w / ((size_t)NFP * nt)];
  const int b = bf / (2 * D), f = bf % (2 * D);
  const int a = f >> 1, s = f & 1;
  int h[3] = {0, 0, 0};
  Real xi[D];
  {
    int j = 0;
    for (int ax = 0; ax < D; ++ax) {
      if (ax == a) continue;
      h[ax] = j == 0 ? (t % n) : (t / n);
      xi[ax] = T.x[j == 0 ? fp % N : fp / N];
      ++j;
    }
  }
  h[a] = s ? n - 1 : 0;
  xi[a] = s ? Real(1) : Real(-1);
  int cell = 0;
  for (int ax = 0, st = 1; ax < D; ++ax, st *= n) cell += h[ax] * st;
  Real own[NV], gst[NV], Ja[D], Fh[NV];
  Real* slot = A.out + ((size_t)bf * NV * NFP + fp) * nt + t;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const size_t src0 = ((size_t)b * NV + v) * Q * nc + cell;
    Real acc = Real(0);
#pragma unroll
    for (int qn = 0; qn < N; ++qn)
      acc += (s ? T.lp[qn] : T.lm[qn]) * S(src0 + (size_t)face_point_index<D, N>(a, fp, qn) * nc);
    own[v] = acc;
    gst[v] = slot[(size_t)v * NFP * nt];
  }
  point_row<D, Real>(A.geo + (size_t)b * NG * nc + cell, nc, xi, a, Ja);
  if (s) lf_flux<D, Real>(own, gst, Ja, A.gamma, Fh);
  else lf_flux<D, Real>(gst, own, Ja, A.gamma, Fh);
#pragma unroll
  for (int v = 0; v < NV; ++v) slot[(size_t)v * NFP * nt] = Fh[v];
}

// Coarse side: the flux at my face point j is the fine sub-face fluxes
// integrated against my face test function l_j and divided by its weight,
// (1/w_j) sum_sub sum_k w_k l_j(xi(x_k)) F_k, rotated into my frame with the
// orientation's sign folded into the precomputed weights.  One thread per
// (face, guard cell, variable, face point).
template <int D, int P, typename Real>
__global__ void __launch_bounds__(128) k_mortar_coarse(const GuardArgs<D, P, Real> A) {
  constexpr int N = P + 1, NV = D + 2, NFP = ipow(N, D - 1);
  constexpr int NSUB = 1 << (D - 1);
  const int n = A.n;
  const int nt = D == 3 ? n * n : n;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (size_t)A.nmc * nt * NV * NFP) return;
  const int j = (int)(w % NFP);
  const int v = (int)((w / NFP) % NV);
  const int t = (int)((w / ((size_t)NFP * NV)) % nt);
  const int i = (int)(w / ((size_t)NFP * NV * nt));
  const Real* __restrict__ wt = A.mw + ((size_t)i * NFP + j) * NSUB * NFP;
  const long long* __restrict__ src = A.msrc + ((size_t)i * nt + t) * NSUB;
  Real acc = Real(0);
#pragma unroll
  for (int e = 0; e < NSUB; ++e) {
    const Real* __restrict__ F = A.out + src[e] + (size_t)v * NFP * nt;
#pragma unroll
    for (int k = 0; k < NFP; ++k) acc += wt[e * NFP + k] * F[(size_t)k * nt];
  }
  A.out[(((size_t)A.mcoarse[i] * NV + v) * NFP + j) * nt + t] = acc;
}

// ============================================================ adaptation
// Refinement indicator (reading R16): per cell g = 2 |(K_e1, .., K_eD)| / K_0
// of the density's Legendre modes (K = V^{-1} u from the Gauss-point values);
// the block keeps the maximum as the bits of a non-negative double.  One
// thread per (leaf, cell).
template <int D, int P, typename Real>
__global__ void k_indicator(int nL, int n, const Real* __restrict__ U, unsigned long long* __restrict__ gmax,
                            Tab<P + 1, Real> T) {
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D);
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (size_t)nL * nc) return;
  const int b = (int)(w / nc), c = (int)(w % nc);
  const Real* u = U + (size_t)b * NV * Q * nc + c;
  Real k0 = Real(0), ke[D];
#pragma unroll
  for (int a = 0; a < D; ++a) ke[a] = Real(0);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const Real x = u[(size_t)q * nc];
    Real w0 = Real(1);
    int r = q;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      w0 *= T.Vi[0][r % N];
      r /= N;
    }
    k0 += w0 * x;
    if constexpr (N > 1) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        Real wa = Real(1);
        int rr = q;
#pragma unroll
        for (int bb = 0; bb < D; ++bb) {
          wa *= T.Vi[bb == a ? 1 : 0][rr % N];
          rr /= N;
        }
        ke[a] += wa * x;
      }
    }
  }
  Real g2 = Real(0);
#pragma unroll
  for (int a = 0; a < D; ++a) g2 += ke[a] * ke[a];
  const double g = N > 1 ? 2.0 * sqrt((double)g2) / (double)k0 : 0.0;
  if (g >= 0.0) atomicMax(&gmax[b], (unsigned long long)__double_as_longlong(g));
  else atomicMax(&gmax[b], 0x7FF8000000000000ull);  // NaN or a non-positive mean: flag as huge
}

// ============================================================ positivity
// Smallest t in [0, 1] with p(ubar + t du) = eps_p: rho p / (gamma - 1) =
// E rho - |m|^2 / 2 makes f(t) = (E(t) - eps_p/(gamma-1)) rho(t) - |m(t)|^2/2
// a quadratic a t^2 + b t + c with f(0) = c > 0 > f(1).
template <int D, typename Real>
__device__ __forceinline__ Real pressure_root(const Real (&ub)[D + 2], const Real (&du)[D + 2], Real eps_p,
                                              Real gm1) {
  const Real Eb = ub[D + 1] - eps_p / gm1;
  Real a = du[D + 1] * du[0], b = Eb * du[0] + du[D + 1] * ub[0], c = Eb * ub[0];
#pragma unroll
  for (int j = 1; j <= D; ++j) {
    a -= Real(0.5) * du[j] * du[j];
    b -= ub[j] * du[j];
    c -= Real(0.5) * ub[j] * ub[j];
  }
  if (fabs(a) < Real(1e-30)) {
    const Real t = -c / b;
    return t < Real(0) ? Real(0) : (t > Real(1) ? Real(1) : t);
  }
  Real disc = b * b - Real(4) * a * c;
  disc = disc > Real(0) ? sqrt(disc) : Real(0);
  const Real r0 = (-b - disc) / (Real(2) * a), r1 = (-b + disc) / (Real(2) * a);
  Real t = Real(2);
  if (r0 >= Real(0) && r0 <= Real(1)) t = r0;
  if (r1 >= Real(0) && r1 <= Real(1) && r1 < t) t = r1;
  return t > Real(1) ? Real(0) : t;
}

// Positivity-preserving scaling (reading R17: Zhang & Shu): per cell, the
// J-weighted mean ubar; theta_1 brings the density to >= eps rho_bar and
// theta_2 the pressure to >= eps p(ubar) at every volume and face Gauss
// point; the cell becomes ubar + theta_1 theta_2 (u - ubar) (only written
// when limited).  A cell whose mean is not admissible sets the status word.
// One thread per (leaf, cell).
template <int D, int P, typename Real>
__global__ void k_limit(int nL, int n, Real* __restrict__ U, const Real* __restrict__ geo,
                        const unsigned char* __restrict__ affine, Real gamma, Real eps, int* status,
                        Tab<P + 1, Real> T) {
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D), NFP = ipow(N, D - 1);
  constexpr int NG = ((1 << D) - 1) * D;
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (size_t)nL * nc) return;
  const int b = (int)(w / nc), c = (int)(w % nc);
  Real* u = U + (size_t)b * NV * Q * nc + c;
  const Real gm1 = gamma - Real(1);
  // J-weighted mean
  Real ub[NV], wsum = Real(0);
#pragma unroll
  for (int v = 0; v < NV; ++v) ub[v] = Real(0);
  const bool aff = affine[b] != 0;
  for (int q = 0; q < Q; ++q) {
    Real xi[D], wq = Real(1);
    for (int a = 0, r = q; a < D; ++a, r /= N) {
      xi[a] = T.x[r % N];
      wq *= T.w[r % N];
    }
    if (!aff) {
      Real t[D][D];
      tangents<D, Real>(geo + (size_t)b * NG * nc + c, nc, xi, t);
      wq *= jacobian_det<D, Real>(t);
    }
    wsum += wq;
#pragma unroll
    for (int v = 0; v < NV; ++v) ub[v] += wq * u[((size_t)v * Q + q) * nc];
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) ub[v] /= wsum;
  Real ke = Real(0);
#pragma unroll
  for (int j = 1; j <= D; ++j) ke += ub[j] * ub[j];
  const Real pb = gm1 * (ub[D + 1] - Real(0.5) * ke / ub[0]);
  if (!(ub[0] > Real(0) && pb > Real(0))) {
    atomicExch(status, -4);
    return;
  }
  const Real eps_r = eps * ub[0], eps_p = eps * pb;
  // check point k: volume point k < Q, else face point (k - Q) of face f
  auto point = [&](int k, Real (&x)[NV]) {
    if (k < Q) {
#pragma unroll
      for (int v = 0; v < NV; ++v) x[v] = u[((size_t)v * Q + k) * nc];
      return;
    }
    const int f = (k - Q) / NFP, fp = (k - Q) % NFP, a = f >> 1, s = f & 1;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Real acc = Real(0);
#pragma unroll
      for (int qn = 0; qn < N; ++qn)
        acc += (s ? T.lp[qn] : T.lm[qn]) * u[((size_t)v * Q + face_point_index<D, N>(a, fp, qn)) * nc];
      x[v] = acc;
    }
  };
  constexpr int NCHK = Q + 2 * D * NFP;
  Real rmin = ub[0];
  for (int k = 0; k < NCHK; ++k) {
    Real x[NV];
    point(k, x);
    rmin = x[0] < rmin ? x[0] : rmin;
  }
  const Real th1 = rmin >= eps_r ? Real(1) : fmin(Real(1), (ub[0] - eps_r) / (ub[0] - rmin));
  Real th2 = Real(1);
  for (int k = 0; k < NCHK; ++k) {
    Real x[NV], du[NV];
    point(k, x);
    Real kx = Real(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      du[v] = th1 * (x[v] - ub[v]);
      x[v] = ub[v] + du[v];
    }
#pragma unroll
    for (int j = 1; j <= D; ++j) kx += x[j] * x[j];
    const Real p = gm1 * (x[D + 1] - Real(0.5) * kx / x[0]);
    if (p < eps_p) {
      const Real t = pressure_root<D, Real>(ub, du, eps_p, gm1);
      th2 = t < th2 ? t : th2;
    }
  }
  const Real theta = th1 * th2;
  if (!(theta < Real(1))) return;
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Real& x = u[((size_t)v * Q + q) * nc];
      x = ub[v] + theta * (x - ub[v]);
    }
}

// State transfer after a regrid (Sec. 3.4): new leaf i copies an old leaf,
// splits its old parent (Eqs. (11)-(12): the parent polynomial at the
// child's Gauss points) or combines its old children (Eqs. (13)-(14): the
// J-weighted projection by a host-built nodal operator: a shared one where
// the children's Jacobian is one constant, else one per cell).  One thread
// per (new leaf, variable, cell).
template <int D, int P, typename Real>
__global__ void k_transfer(int nL, int n, const Real* __restrict__ old, Real* __restrict__ out,
                           const int* __restrict__ mode, const int* __restrict__ src,
                           const int* __restrict__ kids, const long long* __restrict__ opoff,
                           const long long* __restrict__ cellop, const Real* __restrict__ ops,
                           Tab<P + 1, Real> T) {
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D), NW = 1 << D;
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (size_t)nL * NV * nc) return;
  const int c = (int)(w % nc);
  const int v = (int)((w / nc) % NV);
  const int i = (int)(w / ((size_t)nc * NV));
  Real* o = out + ((size_t)i * NV + v) * Q * nc + c;
  const int m = mode[i];
  int I[3] = {0, 0, 0};
  for (int a = 0, r = c; a < D; ++a, r /= n) I[a] = r % n;
  if (m == 0) {
    const Real* s = old + ((size_t)src[i] * NV + v) * Q * nc + c;
#pragma unroll
    for (int q = 0; q < Q; ++q) o[(size_t)q * nc] = s[(size_t)q * nc];
    return;
  }
  if (m == 1) {
    const int bits = kids[(size_t)i * NW];  // child position bits
    int pc = 0, e[3] = {0, 0, 0};
    for (int a = 0, st = 1; a < D; ++a, st *= n) {
      const int H = ((bits >> a) & 1) * n + I[a];
      pc += (H >> 1) * st;
      e[a] = H & 1;
    }
    const Real* s = old + ((size_t)src[i] * NV + v) * Q * nc + pc;
    Real a0[Q], a1[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) a0[q] = s[(size_t)q * nc];
    if (e[0]) apply_axis<D, N, 0, Real>(T.Snp, a0, a1);
    else apply_axis<D, N, 0, Real>(T.Snm, a0, a1);
    if constexpr (D == 2) {
      if (e[1]) apply_axis<D, N, 1, Real>(T.Snp, a1, a0);
      else apply_axis<D, N, 1, Real>(T.Snm, a1, a0);
    } else {
      if (e[1]) apply_axis<D, N, 1, Real>(T.Snp, a1, a0);
      else apply_axis<D, N, 1, Real>(T.Snm, a1, a0);
      if (e[2]) apply_axis<D, N, 2, Real>(T.Snp, a0, a1);
      else apply_axis<D, N, 2, Real>(T.Snm, a0, a1);
#pragma unroll
      for (int q = 0; q < Q; ++q) a0[q] = a1[q];
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) o[(size_t)q * nc] = a0[q];
    return;
  }
  // combine: the 2^D old child cells under this cell, in child order e
  const Real* op = ops + (size_t)cellop[(size_t)opoff[i] + c];
  Real acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) acc[q] = Real(0);
  for (int e = 0; e < NW; ++e) {
    int cb = 0, cc = 0;
    for (int a = 0, st = 1; a < D; ++a, st *= n) {
      const int H = 2 * I[a] + ((e >> a) & 1);
      cb |= (H / n) << a;
      cc += (H % n) * st;
    }
    const Real* s = old + ((size_t)kids[(size_t)i * NW + cb] * NV + v) * Q * nc + cc;
    for (int k = 0; k < Q; ++k) {
      const Real x = s[(size_t)k * nc];
#pragma unroll
      for (int q = 0; q < Q; ++q) acc[q] += op[(size_t)q * NW * Q + e * Q + k] * x;
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) o[(size_t)q * nc] = acc[q];
}

// ============================================================ conversions
// modal <-> nodal on arrays shaped [outer][var][mode or point][inner],
// in place (each thread reads all its values before writing)
template <int D, int P, typename Real>
__global__ void k_convert(size_t outer, int inner, Real* __restrict__ X, int to_nodal, Tab<P + 1, Real> T) {
  constexpr int N = P + 1, NV = D + 2, M = ipow(N, D);
  const size_t total = outer * NV * inner;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= total) return;
  const int c = (int)(w % inner);
  const size_t ov = w / inner;  // outer * NV + v
  Real* base = X + ov * M * inner + c;
  Real a[M], t2[M];
#pragma unroll
  for (int m = 0; m < M; ++m) a[m] = base[(size_t)m * inner];
  if (to_nodal) apply_all<D, N, Real>(T.V, a, t2);
  else apply_all<D, N, Real>(T.Vi, a, t2);
#pragma unroll
  for (int m = 0; m < M; ++m) base[(size_t)m * inner] = a[m];
}

// ============================================================ CFL kernel
// dt candidates of the current (nodal) state, used before the first step.
template <int D, int P, typename Real>
__global__ void k_cfl(int nL, int n, const Real* __restrict__ U, const Real* __restrict__ hcell,
                      Real gamma, unsigned long long* lam_bits, int* status) {
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D);
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t total = (size_t)nL * nc * Q;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double best = 3.0e38;
  bool bad = false;
  if (w < total) {
    const int c = (int)(w % nc);
    const int q = (int)((w / nc) % Q);
    const int b = (int)(w / ((size_t)Q * nc));
    Real u[NV];
    for (int v = 0; v < NV; ++v) u[v] = U[(((size_t)b * NV + v) * Q + q) * nc + c];
    const Real ri = Real(1) / u[0];
    Real ke = Real(0), sv = Real(0);
    for (int j = 0; j < D; ++j) {
      ke += u[1 + j] * u[1 + j];
      sv += fabs(u[1 + j]) * ri;
    }
    const Real p = (gamma - Real(1)) * (u[D + 1] - Real(0.5) * ke * ri);
    if (!(u[0] > Real(0)) || !(p > Real(0)) || !(p < Real(3.0e38))) bad = true;
    else best = (double)(hcell[(size_t)b * nc + c] / (sv + Real(D) * sqrt(gamma * p * ri)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    double u = __shfl_xor_sync(0xffffffffu, best, o);
    best = u < best ? u : best;
  }
  if ((threadIdx.x & 31) == 0 && best < 3.0e38)
    atomicMin(lam_bits, (unsigned long long)__double_as_longlong(best));
  if (bad) atomicExch(status, kStatusNonFinite);
}

// ============================================================ projection
// FP64 point values [leaf][cell][q][var] -> nodal state [leaf][var][q][cell]:
// with the (p+1)-point rule the L2 projection is interpolation at the Gauss
// points, i.e. the nodal values themselves.
template <int D, int P, typename Real>
__global__ void k_project(int nL, int n, const double* __restrict__ vals, Real* __restrict__ U) {
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D);
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t total = (size_t)nL * nc * Q * NV;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= total) return;
  const int c = (int)(w % nc);
  const int q = (int)((w / nc) % Q);
  const int v = (int)((w / ((size_t)nc * Q)) % NV);
  const int b = (int)(w / ((size_t)nc * Q * NV));
  U[w] = (Real)vals[(((size_t)b * nc + c) * Q + q) * NV + v];
}

// ============================================================ totals
// per cell, FP64: T_v = sum_q w_q J_q u_v(q) (geometry in FP64)
template <int D, int P, typename Real>
__global__ void k_totals(int nL, int n, const Real* __restrict__ U, const double* __restrict__ geo64,
                         double* __restrict__ part, Tab<P + 1, double> T) {
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D);
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t total = (size_t)nL * nc;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= total) return;
  const int c = (int)(w % nc);
  const int b = (int)(w / nc);
  double wj[Q];
  const double* X = geo64 + (size_t)b * ((1 << D) - 1) * D * nc + c;
  for (int q = 0; q < Q; ++q) {
    double xi[D];
    double wq = 1.0;
    int rq = q;
    for (int ax = 0; ax < D; ++ax) {
      xi[ax] = T.x[rq % N];
      wq *= T.w[rq % N];
      rq /= N;
    }
    double tg[D][D];
    tangents<D, double>(X, nc, xi, tg);
    wj[q] = wq * jacobian_det<D, double>(tg);
  }
  for (int v = 0; v < NV; ++v) {
    double s = 0.0;
    for (int q = 0; q < Q; ++q) s += wj[q] * (double)U[(((size_t)b * NV + v) * Q + q) * nc + c];
    part[(size_t)v * total + w] = s;
  }
}

}  // namespace dgf
