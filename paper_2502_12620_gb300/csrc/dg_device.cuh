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
// How (GB300 design, not the paper's): the state is stored modally
// (tensor Legendre, SoA [leaf][var][mode][cell]); inside a CTA one layer of
// a block is converted to nodal values at the (p+1)^d Gauss points, which
// makes the (p+1)-point mass matrix diagonal (M = V^T diag(wJ) V, so
// V M^{-1} = diag(1/(wJ)) V^{-T}) and turns the volume and face integrals
// into 1D line operations (weak derivative Sh, boundary lifts l(+-1)/w).
// The residual is accumulated in shared memory by directional sweeps; every
// interior face flux is computed once; the stage combination and, on the
// last stage, the CFL minimum are fused into the epilogue.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

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
  Real Sm[N][N];   // split to the lower child [l][k]
  Real Sp[N][N];   // split to the upper child [l][k]
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

// Trace of a modal cell polynomial on face (AX, side): collapse along AX with
// P_k(+1) = 1 or P_k(-1) = (-1)^k, then nodal values at the face Gauss points
// (tangential axes in increasing order).  out has N^(D-1) entries.
template <int D, int N, int AX, typename Real>
__device__ __forceinline__ void modal_trace(const Tab<N, Real>& T, const Real* K, int side,
                                            Real* out) {
  constexpr int M = ipow(N, D);
  constexpr int MF = ipow(N, D - 1);
  constexpr int S = ipow(N, AX);
  Real c[MF];
#pragma unroll
  for (int f = 0; f < MF; ++f) {
    // f enumerates the tangential multi-index (axes != AX in increasing order)
    const int lo = f % S;          // axes below AX
    const int hi = f / S;          // axes above AX
    const int base = lo + hi * S * N;
    Real acc = Real(0);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const Real sgn = (side > 0 || (k & 1) == 0) ? Real(1) : Real(-1);
      acc += sgn * K[base + k * S];
    }
    c[f] = acc;
  }
  (void)M;
  if constexpr (D == 2) {
    apply_axis<1, N, 0, Real>(T.V, c, out);
  } else {
    Real tmp[MF];
    apply_axis<2, N, 0, Real>(T.V, c, tmp);
    apply_axis<2, N, 1, Real>(T.V, tmp, out);
  }
}

template <int D, int N, typename Real>
__device__ __forceinline__ void modal_trace_rt(const Tab<N, Real>& T, const Real* K, int axis,
                                               int side, Real* out) {
  if (axis == 0) modal_trace<D, N, 0, Real>(T, K, side, out);
  else if (axis == 1) modal_trace<D, N, 1, Real>(T, K, side, out);
  else if constexpr (D == 3) modal_trace<D, N, 2, Real>(T, K, side, out);
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
  const Real alpha = sL > sR ? sL : sR;
#pragma unroll
  for (int v = 0; v < D + 2; ++v) Fh[v] = Real(0.5) * (FL[v] + FR[v] + alpha * (uL[v] - uR[v]));
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
  const double* __restrict__ dtp;
  unsigned long long* lam_bits;
  int* status;
  Real ca, cb, gamma;
  int mode, last;
  Tab<P + 1, Real> T;
};

template <int D, int P, typename Real>
struct GuardArgs {
  int nL, n, mode;  // mode 0: modal guard cells; 1: traces
  const Real* __restrict__ U;
  Real* __restrict__ out;
  const int* __restrict__ kind;    // [b][f]
  const int* __restrict__ nbr;     // [b][f][4]
  const int* __restrict__ orient;  // [b][f] packed decoded orientation
  const int* __restrict__ qbits;   // [b] pos & 1 bits
  const int* __restrict__ copoff;  // [b][f] first combine operator or -1
  const Real* __restrict__ cop;    // [op][2^D M][M]: column k' of the operator is contiguous
  const int* __restrict__ fine_list;  // [nfine] leaf * 2D + face of every finer-neighbour face
  int nfine;
  Tab<P + 1, Real> T;
};

// threads per CTA and CTAs per SM of the stage kernel (registers and shared
// memory decide: FP32 up to p=2 runs 2 x 512 threads per SM)
template <int P, typename Real>
struct StageCfg {
  static constexpr int NT = sizeof(Real) == 4 ? 512 : (P <= 1 ? 512 : 256);
  static constexpr int MINB = (sizeof(Real) == 4 && P <= 2) ? 2 : 1;
};

// shared-memory footprint of the stage kernel (bytes)
template <int D, int P, typename Real>
__host__ __device__ constexpr size_t stage_smem(int n) {
  constexpr int N = P + 1, NV = D + 2, Q = ipow(N, D), NFP = ipow(N, D - 1);
  constexpr int NG = ((1 << D) - 1) * D;
  const size_t ncl = (size_t)n * n;
  size_t us = NV * Q * ncl, rs = us;
  size_t fs = (size_t)NV * NFP * (n + 1) * n;
  size_t fz = D == 3 ? (size_t)NV * NFP * ncl : 0;
  size_t gs = (size_t)NG * ncl;
  return (us + rs + fs + fz + gs) * sizeof(Real);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// metric of one cell: affine blocks use block constants, curvilinear cells
// their trilinear coefficients (held in registers by the caller)
template <int D, typename Real>
struct CellMetric {
  bool aff;
  const Real* am;  // shared: rows of J dxi/dx, then 1/J
  const Real* X;   // shared: trilinear coefficients of the cell, stride ncl
  int stride;
  __device__ __forceinline__ void load(bool affine, const Real* amsh, const Real* gs, int ncl, int c) {
    aff = affine;
    am = amsh;
    X = gs + c;
    stride = ncl;
  }
  __device__ __forceinline__ void row(const Real* xi, int dir, Real (&Ja)[D]) const {
    if (aff) {
#pragma unroll
      for (int j = 0; j < D; ++j) Ja[j] = am[dir * D + j];
    } else {
      Real tg[D][D];
      tangents<D, Real>(X, stride, xi, tg);
      contra_row<D, Real>(tg, dir, Ja);
    }
  }
  // row `dir` and 1/J at one point
  __device__ __forceinline__ Real row_inv_jac(const Real* xi, int dir, Real (&Ja)[D]) const {
    if (aff) {
#pragma unroll
      for (int j = 0; j < D; ++j) Ja[j] = am[dir * D + j];
      return am[D * D];
    }
    Real tg[D][D];
    tangents<D, Real>(X, stride, xi, tg);
    contra_row<D, Real>(tg, dir, Ja);
    Real J = Real(0);
#pragma unroll
    for (int j = 0; j < D; ++j) J += tg[dir][j] * Ja[j];
    return Real(1) / J;
  }
};

// ============================================================ stage kernel
// Persistent CTAs; work item = (leaf, z-chunk); a CTA sweeps the layers of
// its chunk.  Per layer: modal -> nodal in shared memory, x and y face
// fluxes (each face once) and volume terms, z faces carried between layers,
// 1/J, nodal -> modal, SSP-RK combination, CFL minimum on the last stage.
template <int D, int P, typename Real>
__global__ void __launch_bounds__(StageCfg<P, Real>::NT, StageCfg<P, Real>::MINB)
    k_stage(const StageArgs<D, P, Real> A) {
  constexpr int N = P + 1, NV = D + 2, M = ipow(N, D), Q = M, NFP = ipow(N, D - 1);
  constexpr int NG = ((1 << D) - 1) * D;
  const int n = A.n;
  const int NCL = n * n;
  const int nc = D == 3 ? NCL * n : NCL;
  const int nt = D == 3 ? n * n : n;  // guard cells per face
  const auto& T = A.T;
  const Real gamma = A.gamma;
  const Real gm1 = gamma - Real(1);
  const Real dt = Real(*A.dtp);
  const int tid = threadIdx.x, nthr = blockDim.x;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Real sx[N];
  __shared__ Real sam[D * D + 1];
  Real* us = reinterpret_cast<Real*>(smem_raw);
  Real* rs = us + NV * Q * NCL;
  Real* fs = rs + NV * Q * NCL;
  Real* fz = fs + NV * NFP * (n + 1) * n;
  Real* gs = fz + (D == 3 ? NV * NFP * NCL : 0);
  Real* tb = fs;  // top/bottom halo traces reuse the in-layer face buffer
  if (tid < N) sx[tid] = T.x[tid];

  const size_t ustride = (size_t)nc;
  Real lam_min = Real(3.0e38);
  bool bad = false;
  const int items = A.nL * A.nchunks;

#define US(v, q, c) us[((v) * Q + (q)) * NCL + (c)]
#define RS(v, q, c) rs[((v) * Q + (q)) * NCL + (c)]
#define GS(g, c) gs[(g) * NCL + (c)]
#define GTR(f, v, fp, t) Tb[(((size_t)(f) * NV + (v)) * NFP + (fp)) * nt + (t)]
// x faces: [v][fp][row j][face fi]; y faces: [v][fp][face fi][column i]
#define FX(v, fp, j, fi) fs[(((v) * NFP + (fp)) * n + (j)) * (n + 1) + (fi)]
#define FY(v, fp, fi, i) fs[(((v) * NFP + (fp)) * (n + 1) + (fi)) * n + (i)]

  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int b = item / A.nchunks;
    const int chunk = item % A.nchunks;
    const int k0 = D == 3 ? chunk * A.zchunk : 0;
    const int k1 = D == 3 ? min(n, k0 + A.zchunk) : 1;
    const Real* Ub = A.U + (size_t)b * NV * M * nc;
    const Real* Unb = A.Un + (size_t)b * NV * M * nc;
    Real* Ob = A.Uout + (size_t)b * NV * M * nc;
    const Real* Gb = A.geo + (size_t)b * NG * nc;
    const Real* Tb = A.gtr + (size_t)b * 2 * D * NV * NFP * nt;
    const bool aff = A.affine[b] != 0;
    __syncthreads();  // previous item is done with the shared buffers
    if (aff && tid < D * D + 1) sam[tid] = A.ameta[(size_t)b * (D * D + 1) + tid];

    for (int k = k0; k < k1; ++k) {
      const int cbase = D == 3 ? k * NCL : 0;
      // ------------------------------------------- L2 prefetch of what comes next
      {
        const int lines_per_row = (NCL * (int)sizeof(Real) + 127) / 128;
        const int rows = NV * M;
        for (int w = tid; w < rows * lines_per_row; w += nthr) {
          const int r = w / lines_per_row, l = w % lines_per_row;
          if (D == 3 && k + 1 < n)
            prefetch_l2(Ub + (size_t)r * ustride + (k + 1) * NCL + l * (128 / sizeof(Real)));
          if (A.mode == 0 && A.ca != Real(0)) prefetch_l2(Unb + (size_t)r * ustride + cbase + l * (128 / sizeof(Real)));
        }
      }
      // ------------------------------------------- load layer k (modal -> nodal)
      for (int w = tid; w < NCL * NV; w += nthr) {
        const int c = w % NCL, v = w / NCL;
        Real a[M], t2[M];
#pragma unroll
        for (int m = 0; m < M; ++m) a[m] = Ub[((size_t)v * M + m) * ustride + cbase + c];
        apply_all<D, N, Real>(T.V, a, t2);
#pragma unroll
        for (int q = 0; q < Q; ++q) US(v, q, c) = a[q];
      }
      if (!aff) {
        for (int w = tid; w < NCL * NG; w += nthr) {
          const int c = w % NCL, g = w / NCL;
          GS(g, c) = Gb[(size_t)g * nc + cbase + c];
        }
      }
      __syncthreads();

      if constexpr (D == 3) {
        if (k == k0) {
          // bottom halo trace of the first layer: guard (z-) or the layer below
          for (int w = tid; w < NCL * NV; w += nthr) {
            const int c = w % NCL, v = w / NCL;
            Real tr[NFP];
            if (k0 == 0) {
#pragma unroll
              for (int fp = 0; fp < NFP; ++fp) tr[fp] = GTR(4, v, fp, c);
            } else {
              Real K[M];
#pragma unroll
              for (int m = 0; m < M; ++m) K[m] = Ub[((size_t)v * M + m) * ustride + (k0 - 1) * NCL + c];
              modal_trace<3, N, 2, Real>(T, K, +1, tr);
            }
#pragma unroll
            for (int fp = 0; fp < NFP; ++fp) tb[(v * NFP + fp) * NCL + c] = tr[fp];
          }
          __syncthreads();
          for (int w = tid; w < NCL * NFP; w += nthr) {
            const int c = w % NCL, fp = w / NCL;
            Real uL[NV], uR[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              uL[v] = tb[(v * NFP + fp) * NCL + c];
              Real s = Real(0);
#pragma unroll
              for (int qz = 0; qz < N; ++qz) s += T.lm[qz] * US(v, fp + NFP * qz, c);
              uR[v] = s;
            }
            CellMetric<3, Real> cm;
            cm.load(aff, sam, gs, NCL, c);
            const Real xi[3] = {sx[fp % N], sx[fp / N], Real(-1)};
            Real Ja[3], Fh[NV];
            cm.row(xi, 2, Ja);
            lf_flux<3, Real>(uL, uR, Ja, gamma, Fh);
#pragma unroll
            for (int v = 0; v < NV; ++v) fz[(v * NFP + fp) * NCL + c] = Fh[v];
          }
          __syncthreads();
        }
      }

      // ------------------------------------------------- x faces
      for (int w = tid; w < (n + 1) * n * NFP; w += nthr) {
        const int fi = w % (n + 1);
        const int j = (w / (n + 1)) % n;
        const int fp = w / ((n + 1) * n);
        const int t = D == 3 ? j + n * k : j;
        Real uL[NV], uR[NV];
        const int cl = (fi - 1) + n * j, cr = fi + n * j;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (fi == 0) {
            uL[v] = GTR(0, v, fp, t);
          } else {
            Real s = Real(0);
#pragma unroll
            for (int qx = 0; qx < N; ++qx) s += T.lp[qx] * US(v, qx + N * fp, cl);
            uL[v] = s;
          }
          if (fi == n) {
            uR[v] = GTR(1, v, fp, t);
          } else {
            Real s = Real(0);
#pragma unroll
            for (int qx = 0; qx < N; ++qx) s += T.lm[qx] * US(v, qx + N * fp, cr);
            uR[v] = s;
          }
        }
        CellMetric<D, Real> cm;
        cm.load(aff, sam, gs, NCL, fi == n ? cl : cr);
        Real xi[D];
        xi[0] = fi == n ? Real(1) : Real(-1);
        xi[1] = sx[fp % N];
        if constexpr (D == 3) xi[2] = sx[fp / N];
        Real Ja[D], Fh[NV];
        cm.row(xi, 0, Ja);
        lf_flux<D, Real>(uL, uR, Ja, gamma, Fh);
#pragma unroll
        for (int v = 0; v < NV; ++v) FX(v, fp, j, fi) = Fh[v];
      }
      __syncthreads();
      // ------------------------------------------------- x volume + lift
      for (int w = tid; w < NCL * NFP; w += nthr) {
        const int c = w % NCL, fp = w / NCL;
        const int i = c % n, j = c / n;
        CellMetric<D, Real> cm;
        cm.load(aff, sam, gs, NCL, c);
        Real xi[D];
        xi[1] = sx[fp % N];
        if constexpr (D == 3) xi[2] = sx[fp / N];
        Real F[N][NV];
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          Real u[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) u[v] = US(v, qx + N * fp, c);
          xi[0] = T.x[qx];
          Real Ja[D], Fq[NV];
          cm.row(xi, 0, Ja);
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
      // ------------------------------------------------- y faces
      for (int w = tid; w < (n + 1) * n * NFP; w += nthr) {
        const int i = w % n;
        const int fi = (w / n) % (n + 1);
        const int fp = w / ((n + 1) * n);  // qx + N qz
        const int qx = fp % N, qz = fp / N;
        const int t = D == 3 ? i + n * k : i;
        Real uL[NV], uR[NV];
        const int cl = i + n * (fi - 1), cr = i + n * fi;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (fi == 0) {
            uL[v] = GTR(2, v, fp, t);
          } else {
            Real s = Real(0);
#pragma unroll
            for (int qy = 0; qy < N; ++qy) s += T.lp[qy] * US(v, qx + N * qy + N * N * qz, cl);
            uL[v] = s;
          }
          if (fi == n) {
            uR[v] = GTR(3, v, fp, t);
          } else {
            Real s = Real(0);
#pragma unroll
            for (int qy = 0; qy < N; ++qy) s += T.lm[qy] * US(v, qx + N * qy + N * N * qz, cr);
            uR[v] = s;
          }
        }
        CellMetric<D, Real> cm;
        cm.load(aff, sam, gs, NCL, fi == n ? cl : cr);
        Real xi[D];
        xi[0] = sx[qx];
        xi[1] = fi == n ? Real(1) : Real(-1);
        if constexpr (D == 3) xi[2] = sx[qz];
        Real Ja[D], Fh[NV];
        cm.row(xi, 1, Ja);
        lf_flux<D, Real>(uL, uR, Ja, gamma, Fh);
#pragma unroll
        for (int v = 0; v < NV; ++v) FY(v, fp, fi, i) = Fh[v];
      }
      __syncthreads();
      // ------------------------------------------------- y volume + lift
      for (int w = tid; w < NCL * NFP; w += nthr) {
        const int c = w % NCL, fp = w / NCL;
        const int i = c % n, j = c / n;
        const int qx = fp % N, qz = fp / N;
        CellMetric<D, Real> cm;
        cm.load(aff, sam, gs, NCL, c);
        Real xi[D];
        xi[0] = sx[qx];
        if constexpr (D == 3) xi[2] = sx[qz];
        Real F[N][NV];
        Real iJ[N];
#pragma unroll
        for (int qy = 0; qy < N; ++qy) {
          Real u[NV];
          const int q = qx + N * qy + N * N * qz;
#pragma unroll
          for (int v = 0; v < NV; ++v) u[v] = US(v, q, c);
          xi[1] = T.x[qy];
          Real Ja[D], Fq[NV];
          if constexpr (D == 2) iJ[qy] = cm.row_inv_jac(xi, 1, Ja);
          else cm.row(xi, 1, Ja);
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
      }
      __syncthreads();

      if constexpr (D == 3) {
        // ------------------------------------------- top halo trace of layer k
        for (int w = tid; w < NCL * NV; w += nthr) {
          const int c = w % NCL, v = w / NCL;
          Real tr[NFP];
          if (k == n - 1) {
#pragma unroll
            for (int fp = 0; fp < NFP; ++fp) tr[fp] = GTR(5, v, fp, c);
          } else {
            Real K[M];
#pragma unroll
            for (int m = 0; m < M; ++m) K[m] = Ub[((size_t)v * M + m) * ustride + (k + 1) * NCL + c];
            modal_trace<3, N, 2, Real>(T, K, -1, tr);
          }
#pragma unroll
          for (int fp = 0; fp < NFP; ++fp) tb[(v * NFP + fp) * NCL + c] = tr[fp];
        }
        __syncthreads();
        // ------------------------------------------- z volume + z faces, 1/J
        for (int w = tid; w < NCL * NFP; w += nthr) {
          const int c = w % NCL, fp = w / NCL;
          const int qx = fp % N, qy = fp / N;
          CellMetric<3, Real> cm;
          cm.load(aff, sam, gs, NCL, c);
          Real xi[3] = {sx[qx], sx[qy], Real(0)};
          Real F[N][NV];
          Real iJ[N];
#pragma unroll
          for (int qz = 0; qz < N; ++qz) {
            Real u[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v] = US(v, fp + NFP * qz, c);
            xi[2] = T.x[qz];
            Real Ja[3], Fq[NV];
            iJ[qz] = cm.row_inv_jac(xi, 2, Ja);
            flux_along<3, Real>(u, Ja, gm1, Fq);
#pragma unroll
            for (int v = 0; v < NV; ++v) F[qz][v] = Fq[v];
          }
          // top face flux: own top trace vs the halo trace above
          Real uL[NV], uR[NV], Fh[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            Real s = Real(0);
#pragma unroll
            for (int qz = 0; qz < N; ++qz) s += T.lp[qz] * US(v, fp + NFP * qz, c);
            uL[v] = s;
            uR[v] = tb[(v * NFP + fp) * NCL + c];
          }
          {
            xi[2] = Real(1);
            Real Ja[3];
            cm.row(xi, 2, Ja);
            lf_flux<3, Real>(uL, uR, Ja, gamma, Fh);
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const Real fbot = fz[(v * NFP + fp) * NCL + c];
#pragma unroll
            for (int qz = 0; qz < N; ++qz) {
              Real s = Real(0);
#pragma unroll
              for (int jj = 0; jj < N; ++jj) s += T.Sh[qz][jj] * F[jj][v];
              const int q = fp + NFP * qz;
              RS(v, q, c) = (RS(v, q, c) + s - T.lpw[qz] * Fh[v] + T.lmw[qz] * fbot) * iJ[qz];
            }
            fz[(v * NFP + fp) * NCL + c] = Fh[v];
          }
        }
        __syncthreads();
      }

      // ------------------------------------------------- epilogue
      for (int w = tid; w < NCL * NV; w += nthr) {
        const int c = w % NCL, v = w / NCL;
        Real a[M], t2[M];
#pragma unroll
        for (int q = 0; q < Q; ++q) a[q] = RS(v, q, c);
        apply_all<D, N, Real>(T.Vi, a, t2);  // a = modal L(U)
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const size_t gi = ((size_t)v * M + m) * ustride + cbase + c;
          Real o;
          if (A.mode == 1) {
            o = a[m];
          } else {
            o = A.cb * (Ub[gi] + dt * a[m]);
            if (A.ca != Real(0)) o += A.ca * Unb[gi];
          }
          Ob[gi] = o;
          a[m] = o;
        }
        if (A.last) {
          apply_all<D, N, Real>(T.V, a, t2);
#pragma unroll
          for (int q = 0; q < Q; ++q) US(v, q, c) = a[q];
        }
      }
      if (A.last) {
        __syncthreads();
        for (int w = tid; w < NCL * Q; w += nthr) {
          const int c = w % NCL, q = w / NCL;
          Real u[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) u[v] = US(v, q, c);
          const Real ri = Real(1) / u[0];
          Real ke = Real(0), sv = Real(0);
#pragma unroll
          for (int j = 0; j < D; ++j) {
            ke += u[1 + j] * u[1 + j];
            sv += fabs(u[1 + j]) * ri;
          }
          const Real p = gm1 * (u[D + 1] - Real(0.5) * ke * ri);
          if (!(u[0] > Real(0)) || !(p > Real(0)) || !(p < Real(3.0e38))) {
            bad = true;
          } else {
            const Real lam = sv + Real(D) * sqrt(gamma * p * ri);
            const Real hv = A.hcell[(size_t)b * nc + cbase + c] / lam;
            lam_min = hv < lam_min ? hv : lam_min;
          }
        }
      }
      __syncthreads();
    }
  }
#undef US
#undef RS
#undef GS
#undef GTR
#undef FX
#undef FY

  if (A.last) {
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
      if (lane == 0) atomicMin(A.lam_bits, (unsigned long long)__double_as_longlong(v));
    }
    if (bad) atomicExch(A.status, kStatusNonFinite);
  }
}

// ============================================================ guard kernels
// Sec. 3.5, Eqs. (15)-(17).  The stage kernel needs, for every block face,
// the guard cell's trace at my face Gauss points in my frame; the ABI's
// standalone fill needs the guard cells' modal coefficients in my frame.
// Same-level and coarser neighbours: the trace (or the modes) is computed in
// the neighbour's frame and scattered into my point (mode) order, so no
// register array is indexed at run time.  Finer neighbours use k_guard_fine.

// source-frame face point j -> my face point index, for my face axis a and
// the neighbour's face axis b2 (orientation packed as in opi/osg)
template <int D, int N>
__device__ __forceinline__ int map_face_point(int j, int a, int b2, int pk) {
  if constexpr (D == 2) {
    const int t0 = 1 - a;  // my only tangential axis
    const int q = j;       // source tangential index
    return osg(pk, t0) > 0 ? q : N - 1 - q;
  } else {
    const int u0 = b2 == 0 ? 1 : 0;  // first source tangential axis
    const int qu0 = j % N, qu1 = j / N;
    const int t0 = a == 0 ? 1 : 0, t1 = a == 2 ? 1 : 2;   // my tangential axes
    const int s0 = opi(pk, t0) == u0 ? qu0 : qu1;
    const int s1 = opi(pk, t1) == u0 ? qu0 : qu1;
    const int q0 = osg(pk, t0) > 0 ? s0 : N - 1 - s0;
    const int q1 = osg(pk, t1) > 0 ? s1 : N - 1 - s1;
    return q0 + N * q1;
  }
}

// source mode ms (digits in the neighbour's frame) -> my mode and sign
template <int D, int N>
__device__ __forceinline__ int map_mode(int ms, int pk, float* sign) {
  int k[3] = {0, 0, 0};
  int r = ms;
#pragma unroll
  for (int u = 0; u < D; ++u) {
    k[u] = r % N;
    r /= N;
  }
  int m = 0, st = 1;
  float sg = 1.f;
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    const int ka = k[opi(pk, ax)];
    m += ka * st;
    st *= N;
    if (osg(pk, ax) < 0 && (ka & 1)) sg = -sg;
  }
  *sign = sg;
  return m;
}

// one thread per (leaf, face, guard cell t, var); finer faces are skipped
template <int D, int P, typename Real>
__global__ void __launch_bounds__(128) k_guard(const GuardArgs<D, P, Real> A) {
  constexpr int N = P + 1, NV = D + 2, M = ipow(N, D), NFP = ipow(N, D - 1);
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
  auto load = [&](int leaf, const int* h, Real* dst) {
    int c = 0, st = 1;
    for (int ax = 0; ax < D; ++ax) {
      c += h[ax] * st;
      st *= n;
    }
    const Real* src = A.U + ((size_t)leaf * NV + v) * M * nc + c;
#pragma unroll
    for (int m = 0; m < M; ++m) dst[m] = src[(size_t)m * nc];
  };
  Real* out_modal = A.out + (((size_t)b * 2 * D + f) * NV + v) * M * nt + t;
  Real* out_trace = A.out + (((size_t)b * 2 * D + f) * NV + v) * NFP * nt + t;

  if (kind == 3) {  // outflow: the guard is the mirror image of my face cell
    int h[3] = {g[0], g[1], g[2]};
    h[a] = s ? n - 1 : 0;
    Real K[M];
    load(b, h, K);
    if (A.mode == 0) {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        int ka = m;
        for (int u = 0; u < a; ++u) ka /= N;
        out_modal[(size_t)m * nt] = (ka % N) & 1 ? -K[m] : K[m];
      }
    } else {
      Real tr[NFP];
      modal_trace_rt<D, N, Real>(T, K, a, s ? +1 : -1, tr);
#pragma unroll
      for (int fp = 0; fp < NFP; ++fp) out_trace[(size_t)fp * nt] = tr[fp];
    }
    return;
  }
  const int b2 = opi(pk, a);
  const int s2 = osg(pk, a) > 0 ? 1 - s : s;
  int h[3] = {0, 0, 0};
  Real S[M];
  if (kind == 0) {
    for (int ax = 0; ax < D; ++ax) {
      if (ax == a) continue;
      h[opi(pk, ax)] = osg(pk, ax) > 0 ? g[ax] : n - 1 - g[ax];
    }
    h[b2] = s2 == 0 ? 0 : n - 1;
    load(A.nbr[(b * 2 * D + f) * 4], h, S);
  } else {  // coarser: split of Eqs. (11)-(12) in tensor form, neighbour frame
    const int qb = A.qbits[b];
    int e[3] = {0, 0, 0};
    for (int ax = 0; ax < D; ++ax) {
      if (ax == a) continue;
      const int G = ((qb >> ax) & 1) * n + g[ax];
      const int hh = G >> 1, ee = G & 1;
      h[opi(pk, ax)] = osg(pk, ax) > 0 ? hh : n - 1 - hh;
      e[opi(pk, ax)] = osg(pk, ax) > 0 ? ee : 1 - ee;
    }
    h[b2] = s2 == 0 ? 0 : n - 1;
    e[b2] = s2 == 0 ? 0 : 1;
    Real S2[M];
    load(A.nbr[(b * 2 * D + f) * 4], h, S);
    if (e[0]) apply_axis<D, N, 0, Real>(T.Sp, S, S2);
    else apply_axis<D, N, 0, Real>(T.Sm, S, S2);
    if (e[1]) apply_axis<D, N, 1, Real>(T.Sp, S2, S);
    else apply_axis<D, N, 1, Real>(T.Sm, S2, S);
    if constexpr (D == 3) {
      if (e[2]) apply_axis<D, N, 2, Real>(T.Sp, S, S2);
      else apply_axis<D, N, 2, Real>(T.Sm, S, S2);
#pragma unroll
      for (int m = 0; m < M; ++m) S[m] = S2[m];
    }
  }
  if (A.mode == 0) {
#pragma unroll
    for (int ms = 0; ms < M; ++ms) {
      float sg;
      const int m = map_mode<D, N>(ms, pk, &sg);
      out_modal[(size_t)m * nt] = sg < 0 ? -S[ms] : S[ms];
    }
  } else {
    // trace on the neighbour's face (b2, s2), then into my point order
    Real tr[NFP];
    modal_trace_rt<D, N, Real>(T, S, b2, s2 ? +1 : -1, tr);
#pragma unroll
    for (int j = 0; j < NFP; ++j) out_trace[(size_t)map_face_point<D, N>(j, a, b2, pk) * nt] = tr[j];
  }
}

// Finer neighbours (Eqs. (13)-(14)): one warp per (finer face, guard cell t,
// var); the 2^D x M fine-cell modes are staged in shared memory and lane m
// forms output mode m with the precomputed, already rotated operator.
template <int D, int P, typename Real>
__global__ void __launch_bounds__(128) k_guard_fine(const GuardArgs<D, P, Real> A) {
  constexpr int N = P + 1, NV = D + 2, M = ipow(N, D), NFP = ipow(N, D - 1);
  constexpr int KC = (1 << D) * M;
  __shared__ Real stage[4][KC + M];
  const int n = A.n;
  const int nt = D == 3 ? n * n : n;
  const int nc = D == 3 ? n * n * n : n * n;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const size_t item = (size_t)blockIdx.x * 4 + wib;
  if (item >= (size_t)A.nfine * nt * NV) return;
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
  Real* src = stage[wib];
  Real* K = stage[wib] + KC;
  for (int i = lane; i < KC; i += 32) {
    const int e = i / M, k = i % M;
    int c = 0, st = 1;
    for (int ax = 0; ax < D; ++ax) {
      const int cN = (2 * h[ax]) / n;
      c += (2 * h[ax] + ((e >> ax) & 1) - cN * n) * st;
      st *= n;
    }
    src[i] = A.U[(((size_t)fine * NV + v) * M + k) * nc + c];
  }
  __syncwarp();
  const Real* op = A.cop + (size_t)(A.copoff[bf] + t) * KC * M;
  for (int m = lane; m < M; m += 32) {
    Real acc = Real(0);
    for (int i = 0; i < KC; ++i) acc += op[(size_t)i * M + m] * src[i];
    if (A.mode == 0) A.out[((((size_t)b * 2 * D + f) * NV + v) * M + m) * nt + t] = acc;
    K[m] = acc;
  }
  if (A.mode == 0) return;
  __syncwarp();
  // trace of the guard cell (my frame) on its face touching me: xi_a = -+1
  const int side = s ? -1 : +1;
  for (int fp = lane; fp < NFP; fp += 32) {
    int qt[3] = {0, 0, 0}, jj = 0, r = fp;
    for (int ax = 0; ax < D; ++ax) {
      if (ax == a) continue;
      qt[ax] = r % N;
      r /= N;
      ++jj;
    }
    Real acc = Real(0);
    for (int m = 0; m < M; ++m) {
      Real ph = Real(1);
      int rm = m;
      for (int ax = 0; ax < D; ++ax) {
        const int k = rm % N;
        rm /= N;
        if (ax == a) ph *= (side > 0 || (k & 1) == 0) ? Real(1) : Real(-1);
        else ph *= T.V[qt[ax]][k];
      }
      acc += ph * K[m];
    }
    A.out[((((size_t)b * 2 * D + f) * NV + v) * NFP + fp) * nt + t] = acc;
  }
}

// ============================================================ CFL kernel
// dt candidates of the current state (used once before the first step).
template <int D, int P, typename Real>
__global__ void k_cfl(int nL, int n, const Real* __restrict__ U, const Real* __restrict__ hcell,
                      Real gamma, unsigned long long* lam_bits, int* status, Tab<P + 1, Real> T) {
  constexpr int N = P + 1, NV = D + 2, M = ipow(N, D), Q = M;
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t total = (size_t)nL * nc * Q;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double best = 3.0e38;
  bool bad = false;
  if (w < total) {
    const int q = (int)(w % Q);
    const int c = (int)((w / Q) % nc);
    const int b = (int)(w / ((size_t)Q * nc));
    Real u[NV];
    for (int v = 0; v < NV; ++v) {
      const Real* src = U + ((size_t)b * NV + v) * M * nc + c;
      Real s = Real(0);
      for (int m = 0; m < M; ++m) {
        Real ph = Real(1);
        int rq = q, rm = m;
        for (int ax = 0; ax < D; ++ax) {
          ph *= T.V[rq % N][rm % N];
          rq /= N;
          rm /= N;
        }
        s += ph * src[(size_t)m * nc];
      }
      u[v] = s;
    }
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
// nodal FP64 values [leaf][cell][q][var] -> modal (interpolation at Gauss
// points = the (p+1)-point L2 projection).
template <int D, int P, typename Real>
__global__ void k_project(int nL, int n, const double* __restrict__ vals, Real* __restrict__ U,
                          Tab<P + 1, double> T) {
  constexpr int N = P + 1, NV = D + 2, M = ipow(N, D), Q = M;
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t total = (size_t)nL * nc * NV;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= total) return;
  const int v = (int)(w % NV);
  const int c = (int)((w / NV) % nc);
  const int b = (int)(w / ((size_t)NV * nc));
  double a[M], t2[M];
  for (int q = 0; q < Q; ++q) a[q] = vals[(((size_t)b * nc + c) * Q + q) * NV + v];
  apply_all<D, N, double>(T.Vi, a, t2);
  for (int m = 0; m < M; ++m) U[(((size_t)b * NV + v) * M + m) * nc + c] = (Real)a[m];
}

// ============================================================ totals
// per cell, FP64: T_v = sum_q w_q J_q u_v(q) (geometry in FP64)
template <int D, int P, typename Real>
__global__ void k_totals(int nL, int n, const Real* __restrict__ U, const double* __restrict__ geo64,
                         double* __restrict__ part, Tab<P + 1, double> T) {
  constexpr int N = P + 1, NV = D + 2, M = ipow(N, D), Q = M;
  constexpr int NG = ((1 << D) - 1) * D;
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t total = (size_t)nL * nc;
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= total) return;
  const int c = (int)(w % nc);
  const int b = (int)(w / nc);
  double wj[Q];
  const double* X = geo64 + (size_t)b * NG * nc + c;
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
    double a[M], t2[M];
    for (int m = 0; m < M; ++m) a[m] = (double)U[(((size_t)b * NV + v) * M + m) * nc + c];
    apply_all<D, N, double>(T.V, a, t2);
    double s = 0.0;
    for (int q = 0; q < Q; ++q) s += wj[q] * a[q];
    part[(size_t)v * total + w] = s;
  }
}

}  // namespace dgf
