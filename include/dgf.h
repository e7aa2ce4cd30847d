/*
 * dgf.h -- C ABI of the GB300 block-forest discontinuous Galerkin library.
 *
 * The library implements the per-block explicit DG residual and SSP
 * Runge-Kutta stage update for the compressible Euler equations on a forest
 * of unstructured root blocks (arXiv 2502.12620):
 *   - Sec. 2, Eqs. (1)-(5): DG weak form, mass matrix, Lax-Friedrichs flux;
 *   - Sec. 3.1-3.3, Eq. (6): forest of quad/oct trees, N_seg^d cells per
 *     block with (bi/tri)linearly interpolated nodes;
 *   - Sec. 3.4, Eqs. (11)-(14): L2 data inheritance (split S, combine C);
 *   - Sec. 3.5, Eqs. (15)-(17): guard-cell fill with relative rotation;
 *   - Sec. 4.3: CFL time increment, snapshot, guard fill, face fluxes,
 *     volume integral and update.
 *
 * Conventions (all calls):
 *   - Every call returns a dgf_status: DGF_OK (0) or a negative code.  No
 *     exception crosses the ABI.  dgf_last_error() returns a thread-local
 *     message describing the last failure on the calling thread.
 *   - A forest is an opaque handle created by dgf_forest_create and owned by
 *     the caller until dgf_forest_destroy.  Device buffers belong to the
 *     forest; they come from the caller's dgf_allocator (if given) or from
 *     cudaMalloc.  Host arrays passed in are copied before the call returns
 *     (a call that copies one to the device waits for that copy).
 *   - GPU work is enqueued on the stream set by dgf_set_stream (default: a
 *     non-blocking stream the forest creates and owns).  Only calls that
 *     return host values or read host arrays synchronise with that stream.
 *   - Pointers flagged "device" must be device pointers valid on the forest's
 *     device; "host" pointers are plain host memory.  An is_device argument
 *     selects between the two.
 *
 * Data formats (the same in every call):
 *   - d = dim in {2,3}; n = n_seg; N = p+1; nv = d+2 conserved variables
 *     (rho, rho*u_1..rho*u_d, E); M = N^d modes per variable.
 *   - Modal state: tensor Legendre coefficients (unnormalised P_k), SoA
 *     layout [leaf][var][mode][cell], mode m = sum_a k_a N^a, cell
 *     c = sum_a i_a n^a (x fastest), leaves in canonical forest order.
 *     Element type: float for DGF_FP32 forests, double otherwise.
 *   - Canonical forest order: root by root, depth first, children
 *     c = sum_a bit_a 2^a.  Face f = 2*axis + side (side 1 = +xi).
 *   - Neighbour kinds: 0 same level, 1 coarser, 2 finer, 3 domain boundary
 *     (outflow: the guard cell mirrors the face cell).
 *   - Orientation code of a neighbour: my axis a maps to its axis pi[a] with
 *     sign sigma[a]; code = perm_index(pi) * 2^d + sum_a [sigma[a] < 0] 2^a,
 *     perm_index = rank of pi in lexicographic order of permutations.
 */
#ifndef DGF_H
#define DGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dgf_status;

#define DGF_OK 0
#define DGF_EINVAL (-1)       /* bad argument or malformed forest            */
#define DGF_ENOMEM (-2)       /* host or device allocation failed            */
#define DGF_ECUDA (-3)        /* a CUDA runtime call failed                  */
#define DGF_ENONFINITE (-4)   /* rho <= 0, p <= 0 or NaN met on the device   */
#define DGF_ETIMEOUT (-5)     /* a bounded device wait gave up               */
#define DGF_EBALANCE (-6)     /* refine/coarsen would break 2:1 balance      */
#define DGF_ESTATE (-7)       /* call out of order (e.g. no state set)       */
#define DGF_EUNSUPPORTED (-8) /* valid but unsupported size (e.g. smem)      */

#define DGF_FP64 0
#define DGF_FP32 1
/* Compensated FP32 (SSP-RK3 of Sec. 2 with the state accumulated in FP64):
 * u^n is kept in FP64, each stage keeps its increment delta^(k) = u^(k) - u^n
 * in FP32 (delta^(k+1) = b_k (delta^(k) + dt L(u^n + delta^(k))), b = 1, 1/4,
 * 2/3) and u^(n+1) = u^n + delta^(3) is formed in FP64; the residual runs in
 * FP32, reading u^n as the FP32 pair hi + lo (hi = fl(u^n), lo = fl(u^n - hi),
 * split once per step) so that a stage input costs FP32 adds only.  The
 * state, residual and guard cells at this ABI are double. */
#define DGF_FP32_COMP 2

/* Fluxes across a level jump.  DGF_NC_PAPER: each side evaluates the
 * Lax-Friedrichs flux at its own face points from its guard cells (Sec. 3.5,
 * Eqs. (16)-(17)); the totals then drift at level jumps, although Sec. 6
 * claims conservation.  DGF_NC_MORTAR: the fine side's fluxes (computed with
 * the prolonged coarse trace of Eq. (16)) are also the coarse side's: the
 * coarse face flux at its point j is (1/w_j) sum_k w_k l_j(xi(x_k)) F_k over
 * the fine sub-face points, which conserves the totals to round-off.  Not a
 * paper option: it is the repair of the conservation claim. */
#define DGF_NC_PAPER 0
#define DGF_NC_MORTAR 1

typedef struct dgf_forest dgf_forest;

/* Forest description (Sec. 3.1-3.3).  Root blocks are hexahedra (3D) or
 * quadrilaterals (2D) given by 2^d corner node ids in local lexicographic
 * order (corner bit a = local coordinate a at +1).  Root faces are glued by
 * shared corner ids or, failing that, by corner positions shifted by a sum
 * c_1 t_1 + ... + c_k t_k of the periodic translations (c_i in {-1,0,1}). */
typedef struct {
  int32_t dim;        /* 2 or 3                                             */
  int32_t n_seg;      /* cells per block edge: even, 2..16                  */
  int32_t p;          /* polynomial degree 0..3                             */
  int32_t precision;  /* DGF_FP64, DGF_FP32 or DGF_FP32_COMP                */
  int32_t device;     /* CUDA device ordinal; -1 = host-only forest that
                         answers topology/geometry queries only             */
  int32_t n_periodic; /* number of periodic translations, 0..3             */
  int32_t nonconforming; /* level jumps: DGF_NC_PAPER or DGF_NC_MORTAR       */
  int32_t reserved;   /* must be 0                                          */
  double gamma;       /* ideal-gas ratio of Eq. (23), e.g. 1.4              */
  double cfl;         /* CFL number of the time increment (Sec. 4.3)        */
  double periodic[9]; /* n_periodic vectors of dim components, packed       */
  int64_t n_nodes;
  const double* nodes;           /* host, n_nodes*dim, copied               */
  int64_t n_roots;
  const int64_t* root_corners;   /* host, n_roots*2^dim, copied             */
  const double* root_cell_nodes; /* host, nullable: n_roots*(n_seg+1)^dim*dim
                                    cell nodes per root in local order; if
                                    NULL they follow from Eq. (6)            */
} dgf_forest_desc;

/* Optional device allocator.  alloc returns NULL on failure; free is given
 * the size and stream of the matching alloc.  The library uses the memory
 * on its forest's stream and on batch streams, in no order the allocator
 * knows of: alloc must return memory that no work pending on any stream
 * still touches (a caching allocator must not hand out a block freed on a
 * stream that has work queued after the free, and should serve the
 * library from a stream of its own).  Before it calls free the library
 * synchronises the forest's stream; a batch holding the forest must be
 * synchronised by the caller before the forest is regridded or destroyed. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* ptr, size_t bytes, void* stream);
} dgf_allocator;

/* Thread-local message of the last failed call on this thread. */
const char* dgf_last_error(void);

/* Build the root forest (Sec. 3.1): validates the description, glues root
 * faces, computes rotations, and (device >= 0) allocates device buffers.
 * allocator may be NULL.  On success *out owns everything. */
dgf_status dgf_forest_create(const dgf_forest_desc* desc, const dgf_allocator* allocator,
                             dgf_forest** out);
dgf_status dgf_forest_destroy(dgf_forest* f);

/* Stream for all GPU work of this forest (a cudaStream_t, NULL = legacy);
 * waits for the work enqueued on the previous one. */
dgf_status dgf_set_stream(dgf_forest* f, void* stream);

/* Refinement (Sec. 3.1, 3.3, 3.4): refine the given leaves (ids in the
 * current canonical order), then refine coarser leaves until every face
 * joins leaves at most one level apart.  A state set before the call is
 * carried over on the device: new children by the split of Eqs. (11)-(12).
 * Leaf ids are renumbered afterwards. */
dgf_status dgf_block_refine(dgf_forest* f, const int64_t* leaf_ids, int64_t n);
/* Coarsen the parents of the given leaves (all 2^d children of each parent
 * must be leaves).  DGF_EBALANCE (forest unchanged) if 2:1 balance would
 * break.  A state is carried over on the device by the combine of Eqs.
 * (13)-(14). */
dgf_status dgf_block_coarsen(dgf_forest* f, const int64_t* leaf_ids, int64_t n);

/* Refinement indicator per leaf (the paper refines by thresholds on cell
 * quantities, Sec. 5-6, without a formula): per cell
 * g = 2 |(K_e1, .., K_ed)| / K_0 of the density's Legendre modes (mean K_0,
 * degree-one modes K_ea; h |grad rho| / rho_mean on a cube cell of edge h),
 * the leaf's value the largest over its cells; 0 for p = 0; NaN when a cell
 * has a non-positive mean density.  Computed on the device in the forest's
 * precision.  out: host, n_leaves doubles.  Synchronises. */
dgf_status dgf_indicator(dgf_forest* f, double* out);
/* One adaptation (Sec. 3.4 for the data): leaves with indicator above
 * refine_above and level below max_level are refined (2:1 closure may refine
 * more); then, visiting the leaves in canonical order, each sibling group of
 * leaves all below coarsen_below is coarsened when its first child (all
 * position bits even) is met, unless 2:1 face balance forbids it.  The state
 * follows on the device: copy, split (Eqs. (11)-(12)), combine (Eqs.
 * (13)-(14), J-weighted).  n_refined: leaves refined by the threshold (not
 * counting the closure); n_coarsened: parents restored (both nullable).
 * Leaf ids change.  DGF_ENONFINITE if an indicator is NaN. */
dgf_status dgf_adapt(dgf_forest* f, double refine_above, double coarsen_below, int32_t max_level,
                     int64_t* n_refined, int64_t* n_coarsened);
/* The same adaptation with a caller-supplied indicator (host, n_leaves
 * doubles, e.g. from dgf_indicator or a criterion of the caller's own).
 * Works on host-only forests (topology only). */
dgf_status dgf_adapt_with(dgf_forest* f, const double* indicator, double refine_above, double coarsen_below,
                          int32_t max_level, int64_t* n_refined, int64_t* n_coarsened);

/* Boundary conditions of the root faces that have no neighbour (Sec. 5-6
 * use outflow and inflow boundaries): root_face_kind[root * 2d + face] is 0
 * for outflow (the guard cell mirrors my face cell, the default) or 1 for a
 * prescribed constant state (inflow / far field: the guard cell is `state`,
 * nv conserved values, host).  Entries of faces that have a neighbour are
 * ignored.  Leaf faces inherit their root face's kind.  The device tables are
 * rebuilt; a state set before the call is kept. */
dgf_status dgf_set_boundary(dgf_forest* f, const int32_t* root_face_kind, const double* state);

/* Number of leaf blocks. */
dgf_status dgf_leaf_count(const dgf_forest* f, int64_t* n_leaves);
/* Integer leaf tables (host arrays sized by dgf_leaf_count = L):
 *   root[L], level[L] (roots are level 1), pos[L*dim] (block coordinates at
 *   its level in the root's frame), kind[L*2d], nbr[L*2d*4] (neighbour leaf
 *   ids; for kind 2 entry s is the fine leaf on sub-face s = sum_j bit_j 2^j
 *   over my tangential axes in increasing order; unused entries -1),
 *   orient[L*2d].  Any pointer may be NULL. */
dgf_status dgf_leaf_table(const dgf_forest* f, int32_t* root, int32_t* level, int32_t* pos,
                          int32_t* kind, int64_t* nbr, int32_t* orient);
/* Physical volume quadrature points, host [leaf][cell][q][dim] (FP64),
 * q = sum_a q_a N^a over (p+1)-point Gauss-Legendre nodes. */
dgf_status dgf_quad_points(const dgf_forest* f, double* xyz);

/* Number of state values (leaves * nv * M * n^d). */
dgf_status dgf_state_size(const dgf_forest* f, int64_t* n_values);
/* Copy in / out the modal state (layout above; forest element type). */
dgf_status dgf_set_state(dgf_forest* f, const void* src, int is_device);
dgf_status dgf_get_state(dgf_forest* f, void* dst, int is_device);
/* Set the state from FP64 point values [leaf][cell][q][var] at the volume
 * quadrature points: the (p+1)-point L2 projection of Eq. (4)'s mass matrix,
 * i.e. interpolation at the Gauss points. */
dgf_status dgf_set_state_nodal(dgf_forest* f, const double* vals, int is_device);

/* Standalone guard-cell fill (Sec. 3.5, Eqs. (15)-(17)) of the current state:
 * writes modal guard cells [leaf][face][var][mode][t] (forest element type),
 * t = sum_j g_j n^j over my tangential cell coordinates, in my frame. */
dgf_status dgf_fill_guardcells(dgf_forest* f, void* guard, int is_device);
/* L(U) = M^{-1} R of Eqs. (3)-(4) for the current state, modal layout. */
dgf_status dgf_dg_residual(dgf_forest* f, void* dst, int is_device);

/* One SSP-RK3 time increment (Sec. 2 last paragraph; Sec. 4.3): dt = CFL *
 * min over cells and quadrature points of h / sum_i(|u_i| + c), clipped so
 * that time does not pass t_end; three stages of guard fill + residual +
 * Shu-Osher combination.  dt stays on the device; if dt_out is non-NULL the
 * call synchronises and returns it.  Once t = t_end the increment is zero and
 * leaves the state unchanged bit for bit (no stage is evaluated), so a
 * scheduler may enqueue steps past t_end. */
dgf_status dgf_rk_step(dgf_forest* f, double t_end, double* dt_out);
/* Current time (synchronises) / reset it; dgf_set_time also zeroes the
 * step count below. */
dgf_status dgf_get_time(dgf_forest* f, double* t);
dgf_status dgf_set_time(dgf_forest* f, double t);
/* Number of time increments taken with dt > 0 since creation or the last
 * dgf_set_time (increments clipped to dt = 0 at t_end are not counted);
 * synchronises the forest's stream.  Bookkeeping for schedulers: the paper
 * has no counterpart. */
dgf_status dgf_step_count(dgf_forest* f, int64_t* steps);
/* CFL time increment of the current state (synchronises). */
dgf_status dgf_compute_dt(dgf_forest* f, double* dt);

/* Conserved totals T_v = sum_cells sum_q w_q J_q u_v(q), FP64, fixed-order
 * reduction; totals[nv] host (synchronises). */
dgf_status dgf_conserved_totals(dgf_forest* f, double* totals);

/* Positivity-preserving limiter (the paper uses limiters for its cylinder
 * case, Sec. 6, without details; this is the scaling limiter of Zhang & Shu,
 * J. Comput. Phys. 229 (2010)): after every RK stage each cell is scaled
 * toward its J-weighted mean u_bar so that rho >= eps rho_bar and
 * p >= eps p(u_bar) at every volume and face Gauss point (density first,
 * then pressure through a quadratic in the scaling factor); the mean is
 * kept.  eps in (0, 1) turns it on, 0 off.  A cell whose mean is not
 * admissible sets DGF_ENONFINITE in the status word.  dt of the next step is
 * taken from the unlimited last stage.  DGF_EUNSUPPORTED for
 * DGF_FP32_COMP forests.  dgf_limit applies it once to the current state
 * (for initial data). */
dgf_status dgf_set_limiter(dgf_forest* f, double eps);
dgf_status dgf_limit(dgf_forest* f);

/* Device status word: 0 or DGF_ENONFINITE (synchronises); reset clears it. */
dgf_status dgf_status_word(dgf_forest* f, int32_t* status, int reset);

/* Tile of the stage kernel: a work item is a z-chunk of zchunk cell layers
 * of one block (3D), resident_ctas the persistent grid size.  The first
 * dgf_rk_step of a 3D forest times one residual evaluation for every chunk
 * length n_seg, n_seg/2, ..., 1 (with each stage kernel and grid, see
 * dgf_stage_kernel and dgf_stage_grid) and keeps the fastest; later forests of the
 * same device, dimension, degree, n_seg, precision and leaf count in the
 * process reuse that choice, and a regrid keeps it (the environment variable
 * DGF_ZCHUNK fixes it instead).  The chunk length changes no bit of any result.  Not a paper
 * quantity: the paper's per-block loop (Sec. 4.3) has no tiling. */
dgf_status dgf_tuning(const dgf_forest* f, int32_t* zchunk, int32_t* resident_ctas);

/* Which stage kernel the forest's time step launches (host value, no sync):
 * 0 = the cell-pair FP32 kernel (3D forests of 8^3-cell blocks at p = 1, 2
 * in plain FP32: f32x2 arithmetic on cell pairs, TMA-staged layers; four
 * CTAs per SM at p = 1), 1 = the general layer-sweep kernel, 2 = the
 * cell-pair kernel in its five-CTA shape (p = 1 only: more warps, fewer
 * registers).  The first dgf_rk_step of a 3D forest times every kernel that
 * applies and keeps the fastest (the z-chunk length and the grid are tuned
 * with it); DGF_STAGE_KERNEL=pair|pair5|classic in the environment pins the
 * choice.  The two kernels round differently, so results agree within the
 * FP32 tolerance, not bit for bit; a given kernel is bitwise reproducible
 * and independent of the z-chunk length.  The paper has no counterpart (a
 * tuning report). */
dgf_status dgf_stage_kernel(const dgf_forest* f, int32_t* kernel);

/* The stage kernel's grid (host value, no sync): *per_item = 0 for the
 * persistent grid (resident_ctas CTAs of dgf_tuning walking the work items),
 * 1 for one CTA per work item (the hardware scheduler hands out the items).
 * Timed by the autotuner with the kernel and the chunk length;
 * DGF_STAGE_GRID=persistent|items pins it.  Changes no bit of any result. */
dgf_status dgf_stage_grid(const dgf_forest* f, int32_t* per_item);

/* Kernel timing: when on, rk_step launches stage by stage (no graph) with
 * CUDA events around every kernel; dgf_kernel_times synchronises and returns
 * summed milliseconds and kernel launch counts for the classes 0 = dt,
 * 1 = guard (with the mortar passes and the limiter), 2 = stage, then resets
 * the sums. */
dgf_status dgf_set_timing(dgf_forest* f, int on);
dgf_status dgf_kernel_times(dgf_forest* f, double* ms, int64_t* launches, int n_classes);

/* Residual without any allocation.  The paper has no counterpart: this call
 * exists for callers that cannot allocate device memory after the forest is
 * built (code that runs while a CUDA graph is being captured, or a process
 * whose device memory all comes from a pool it does not own).  It computes
 * the same L(U) as dgf_dg_residual, but on caller-owned device buffers in
 * the nodal layout the kernels use, [leaf][var][point][cell] with point
 * q = sum_a q_a N^a over the (p+1)-point Gauss-Legendre nodes and
 * u(q) = sum_m K_m phi_m(x_q) (forest element type).
 *   U_nodal  device, input state, read only;
 *   L_nodal  device, output, must not alias U_nodal.
 * Both must be 16-byte aligned (the kernels move 16-byte vectors) and be
 * device (or managed) memory of the forest's device; DGF_EINVAL otherwise,
 * before anything is launched.
 * The guard traces go to a 16 MiB array compiled into the library (a
 * file-scope __device__ array; every GPU that loads the library holds it
 * until the process exits).  Forests whose guard traces need more than
 * 16 MiB get DGF_EUNSUPPORTED.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress), so make the first call on
 * each device outside any stream capture.  The address is kept per device
 * for the life of the process; after a cudaDeviceReset the next call finds
 * it stale and looks it up again (so that call, too, belongs outside a
 * capture).  No cudaMalloc, cudaFree or
 * allocator callback is made.  All calls share the one array and every call
 * overwrites what it reads, so nothing needs clearing, but calls whose GPU
 * work overlaps (several streams, several host threads, several forests on
 * the same device) race on it: order them on one stream.  Asynchronous on
 * the forest's stream. */
dgf_status dgf_dg_residual_noalloc(dgf_forest* f, const void* U_nodal, void* L_nodal);

/* Batches: several independent forests advanced together, one launch of
 * each kernel per stage for all of them (the paper's per-block loop of
 * Sec. 4.3 run over the blocks of every member; the members' kernel
 * arguments live in device arrays and each work item finds its forest from
 * prefix sums), one CUDA graph per membership.  Members keep their own
 * time, end time, time increment (Sec. 4.3 CFL step, reading R5) and CFL
 * minimum; a member at its end time is left unchanged by further steps, so
 * a member's result is the one it gets as the only member of a batch.
 * Members: forests on the batch's device, 3D, n_seg 8, one degree p, FP32
 * plain form (DGF_FP32), no mortar repair, no limiter, state set
 * (DGF_EUNSUPPORTED / DGF_EINVAL / DGF_ESTATE otherwise).  The batch owns
 * small device arrays (cudaMalloc); the forests keep owning their state.
 * Work items are z-chunks of blocks, one chunk length for the batch chosen
 * from its total block count to fill the persistent grid (DGF_ZCHUNK fixes
 * it); like the single-forest tiling it changes no bit of any result.
 *   dgf_batch_create   device ordinal; stream (cudaStream_t) or NULL for an
 *                      own stream.
 *   dgf_batch_set      replace the members (n may be 0) and set each
 *                      member's end time t_end[i]; waits for the members'
 *                      own streams and the batch stream.  Call again after
 *                      a member is regridded, refined or destroyed.
 *   dgf_batch_step     enqueue `steps` time increments of every member on
 *                      the batch stream (asynchronous).
 *   dgf_batch_sync     wait for the batch stream (dgf_batch_query: has it
 *                      finished?); member queries
 *                      (dgf_get_time, dgf_get_state, ...) run on the
 *                      member's own stream, so sync the batch first.
 * No counterpart in the paper beyond the per-block loop (a serving layer). */
typedef struct dgf_batch dgf_batch;
dgf_status dgf_batch_create(int32_t device, void* stream, dgf_batch** out);
dgf_status dgf_batch_destroy(dgf_batch* b);
dgf_status dgf_batch_set(dgf_batch* b, dgf_forest* const* forests, const double* t_end, int32_t n);
dgf_status dgf_batch_step(dgf_batch* b, int32_t steps);
dgf_status dgf_batch_sync(dgf_batch* b);
/* idle = 1 when all work enqueued on the batch stream has finished (no wait). */
dgf_status dgf_batch_query(dgf_batch* b, int32_t* idle);
/* Time, step count (increments with dt > 0) and status word of every member,
 * in member order, after the work enqueued so far (waits for the batch
 * stream): one gather on the device, one copy. */
dgf_status dgf_batch_progress(dgf_batch* b, double* t, int64_t* steps, int32_t* status);

#ifdef __cplusplus
}
#endif

#endif /* DGF_H */
