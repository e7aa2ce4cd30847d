// Type-erased launch descriptors passed from the C ABI layer to the
// per-(dimension, precision) translation units that instantiate the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dgf {

// 1D reference tables in FP64, N <= 4 (converted to the kernel precision).
struct RtTables {
  int N;
  double x[4], w[4], V[16], Vi[16], Sh[16], lp[4], lm[4], Sm[16], Sp[16], Snm[16], Snp[16];
};

struct RtStage {
  int p, nL, n, zchunk, slots;
  int kernel;  // 0: the cell-pair kernel where it applies, 1: k_stage
  const void* U;
  const void* Un;
  void* Uout;
  const void* geo;
  const void* gtr;
  const void* hcell;
  const unsigned char* affine;
  int all_affine;  // every leaf affine
  const void* ameta;
  const int* kind;
  const int* nbr;
  const int* orient;
  const int* qbits;
  const double* dtp;
  unsigned long long* lam_bits;
  int* status;
  double ca, cb, gamma;
  int mode, last;
  int comp;             // compensated form (FP32 kernels only)
  const double* U64;    // compensated: u^n
  const float* Uhi;     // compensated: u^n = hi + lo in FP32, read by every stage
  const float* Ulo;
  const float* Din;     // compensated: delta^(k) or null
  double* U64out;       // compensated, last stage: u^(n+1)
  const unsigned char* fluxmask;  // mortar mode: per block, faces whose flux is in gtr
  RtTables T;
};

struct RtGuard {
  int p, nL, n, mode;
  int comp;
  const double* U64;
  const float* Uhi;
  const float* Ulo;
  const float* Din;
  const void* U;
  void* out;
  const int* kind;
  const int* nbr;
  const int* orient;
  const int* qbits;
  const int* copoff;
  const void* cop;
  const void* ctr;
  const int* fine_list;
  int nfine;
  const int* trd;  // [leaf][face][8] face-trace descriptors (kinds 0, 1, 3)
  // mortar mode: fine-side and coarse-side faces, coarse-side weights/sources
  const void* geo;
  double gamma;
  const int* mfine;
  int nmf;
  const int* mcoarse;
  int nmc;
  const void* mw;
  const long long* msrc;
  const void* bstate;  // prescribed boundary state (nv values, compute precision)
  RtTables T;
};

// state transfer after a regrid (new leaves from old ones)
struct RtTransfer {
  int p, nL, n;
  const void* old;
  void* out;
  const int* mode;        // [new leaf] 0 copy, 1 split, 2 combine
  const int* src;         // [new leaf] old leaf (copy, split)
  const int* kids;        // [new leaf][2^d] old children (combine); [0] = position bits (split)
  const long long* opoff; // [new leaf] combine leaves: first entry of its cells in cellop
  const long long* cellop; // [combine cell] element offset of its operator in ops
  const void* ops;        // [op][Q][2^d Q]; op 0 = the reference (constant-Jacobian) operator
  RtTables T;
};

struct RtMisc {
  int p, nL, n;
  const void* U;
  void* Uout;
  const void* hcell;
  const double* vals;
  const double* geo64;
  double* part;
  double gamma;
  unsigned long long* lam_bits;
  int* status;
  unsigned long long* gmax;  // refinement indicator per leaf (double bits)
  const void* geo;           // limiter: trilinear coefficients (compute precision)
  const unsigned char* affine;
  double eps;                // limiter bound, relative to the cell mean
  RtTables T;
};

// returns cudaErrorInvalidConfiguration when the shared-memory footprint
// exceeds what the device allows
template <int D, typename Real>
cudaError_t launch_stage(const RtStage& r, cudaStream_t s);
template <int D, typename Real>
cudaError_t launch_guard(const RtGuard& r, cudaStream_t s);
template <int D, typename Real>
cudaError_t launch_cfl(const RtMisc& r, cudaStream_t s);
template <int D, typename Real>
cudaError_t launch_project(const RtMisc& r, cudaStream_t s);
template <int D, typename Real>
cudaError_t launch_totals(const RtMisc& r, cudaStream_t s);
template <int D, typename Real>
cudaError_t launch_indicator(const RtMisc& r, cudaStream_t s);
template <int D, typename Real>
cudaError_t launch_limit(const RtMisc& r, cudaStream_t s);
template <int D, typename Real>
cudaError_t launch_transfer(const RtTransfer& r, cudaStream_t s);
// modal <-> nodal in place on [outer][var][mode/point][inner]
template <int D, typename Real>
cudaError_t launch_convert(int p, size_t outer, int inner, void* X, int to_nodal, const RtTables& T,
                           cudaStream_t s);
template <int D, typename Real>
size_t stage_smem_bytes(int p, int n);
// batches (3D, n_seg 8, FP32, plain form): per-forest argument packing on the
// host (host == nullptr: size only), work items / blocks per forest,
// resident CTAs of the batch stage kernel, and the batch launches
template <int D, typename Real>
int stage_items(const RtStage& r);
template <int D, typename Real>
size_t stage_args_pack(const RtStage* r, int n, void* host);
template <int D, typename Real>
size_t guard_args_pack(const RtGuard* r, int n, void* host);
template <int D, typename Real>
long long guard_blocks(const RtGuard& r, int* nfb);
template <int D, typename Real>
int stage_batch_blocks_per_sm(int p, int kernel, int all_affine);
template <int D, typename Real>
cudaError_t launch_stage_batch(const RtStage& common, const void* members, const int* istart, int nmem, int grid,
                               cudaStream_t s);
template <int D, typename Real>
cudaError_t launch_guard_batch(int p, const void* members, const int* bstart, const int* nfb, int nmem,
                               long long blocks, cudaStream_t s);
// resident stage CTAs per SM (0: does not fit)
template <int D, typename Real>
int stage_occupancy(int p, int n, int comp, int kernel);

}  // namespace dgf
