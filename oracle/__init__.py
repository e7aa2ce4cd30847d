"""FP64 CPU oracle for the block-forest DG residual and SSP-RK stage update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, links or executes anything here, and this package imports nothing
from the product: the two share only the seeded input generators in
``workloads``.

What it computes, written plainly from the paper (arXiv 2502.12620):
  * Sec. 2, Eqs. (1)-(5): DG weak form of the compressible Euler equations
    per cell, mass-matrix solve, Lax-Friedrichs numerical flux.
  * Sec. 3.1/3.3: block forest of root trees, N_seg^d cells per block whose
    nodes are the (bi/tri)linear interpolation of Eq. (6).
  * Sec. 3.4, Eqs. (11)-(14): L2 data inheritance (split S, combine C).
  * Sec. 3.5, Eqs. (15)-(17): guard-cell fill (copy / split / combine, each
    followed by the relative rotation of the neighbour frame).
  * Sec. 4.3: the time-increment procedure (CFL step, snapshot, guard fill,
    face fluxes, volume integral, update) with the SSP Runge-Kutta scheme.

Every routine favours a reader checking it against the paper over speed:
brute-force quadrature with the full tensor basis evaluated at every point,
dense mass matrices assembled by quadrature and solved with a dense solver,
L2 projections evaluated by quadrature, no sum factorisation.

Readings where the paper is silent or ambiguous (each one is listed in the
design notes of the repository):
  R1 basis: tensor Legendre P_k (unnormalised), (p+1)^d modes per variable,
     mode index m = sum_a k_a (p+1)^a.
  R2 quadrature: (p+1)-point Gauss-Legendre per axis for every volume and
     face integral, including the mass matrix.
  R3 LF flux: dissipative sign, F = 1/2[(F(U_L)+F(U_R)).n + alpha (U_L-U_R)]
     with n the unit normal out of the L side and alpha the larger of
     |u.n|+c on the two sides at each face point.
  R4 time stepping: 3-stage SSP-RK3 (Shu-Osher form), guard fill every stage.
  R5 CFL: dt = CFL * min over cells and quadrature points of
     h / sum_i(|u_i| + c), h = (cell volume)^(1/d).
  R6 combine operator C: J-weighted L2 projection whose integrals use each
     child cell's own Gauss rule (so restriction(prolongation(u)) = u).
  R7 rotation: signed axis permutation derived from matching corner nodes.
  R15 level jumps: the paper's guard scheme (Sec. 3.5) is the default; the
     paper claims conservation for it (Sec. 6), which does not hold when
     the two sides evaluate the flux from different data.  The "mortar"
     option restores it: the fine side's fluxes at its face points are also
     the coarse side's, integrated against the coarse test functions.
  R16 adaptation (the paper gives no indicator formula): per cell
     g = 2 |(K_e1, .., K_ed)| / K_0 of the density modes, block indicator the
     maximum over its cells; refine above a threshold (with 2:1 closure),
     then one pass in canonical leaf order coarsening sibling groups below a
     threshold where 2:1 balance allows (``adapt.py``).
  R11 boundaries: unmatched root faces are outflow (the guard cell mirrors
     my face cell) unless tagged as a prescribed constant state (inflow /
     far field).
  R17 positivity: optional scaling limiter of Zhang & Shu (2010) after every
     RK stage, toward the J-weighted cell mean, checked at the volume and
     face Gauss points (``limiter.py``).

Parity pins: every function here is pinned by the not-gpu tests in
``tests/test_oracle_*.py`` against closed forms, invariants and independent
brute-force solvers; none is "parity unpinned".
"""
