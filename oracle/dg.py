"""DG residual, guard-cell fill, data inheritance and SSP-RK3 (oracle; test infrastructure).

State layout (an interface format shared with the product): U[leaf][var][mode][cell],
leaves in the canonical forest order, var in (rho, rho u_1..u_d, E), mode
m = sum_a k_a N^a, cell = sum_a i_a n^a.

Plain FP64, brute force: every volume/face integral evaluates the full tensor
basis at every Gauss point; every mass matrix is assembled by quadrature and
solved densely; every projection (split, combine, rotation) is an L2
projection evaluated by quadrature.
"""
from __future__ import annotations

import numpy as np

from . import basis as B
from .euler import GAMMA, lax_friedrichs, physical_flux, primitives, sound_speed
from .forest import BOUNDARY, COARSER, FINER, SAME, orient_decode


# ----------------------------------------------------------------- geometry
def shape_functions(xi):
    """Eq. (6) shape functions N_k(xi) = prod_a (1 + s_{k,a} xi_a)/2 and their
    reference gradients, for corners k in bit order.  xi: (P, d)."""
    xi = np.atleast_2d(xi)
    P, d = xi.shape
    bits = B.all_corner_bits(d)
    N = np.ones((P, 2 ** d))
    dN = np.ones((P, 2 ** d, d))
    for k, b in enumerate(bits):
        for a in range(d):
            s = 1.0 if b[a] else -1.0
            fa = 0.5 * (1.0 + s * xi[:, a])
            N[:, k] *= fa
            for g in range(d):
                dN[:, k, g] *= (0.5 * s) if g == a else fa
    return N, dN


def map_points(corners, xi):
    """Physical points x(xi) for every cell: corners (C, 2^d, d) -> (C, P, d)."""
    N, _ = shape_functions(xi)
    return np.einsum("pk,ckj->cpj", N, corners)


def jacobian(corners, xi):
    """A[c, p, j, a] = d x_j / d xi_a;  J = det A;  Ja[c,p,i,j] = J d xi_i/d x_j."""
    _, dN = shape_functions(xi)
    A = np.einsum("pka,ckj->cpja", dN, corners)
    J = np.linalg.det(A)
    Ja = J[..., None, None] * np.linalg.inv(A)
    return A, J, Ja


# --------------------------------------------------------------- utilities
class Ops:
    """Reference-element tables for degree p in d dimensions."""

    def __init__(self, d, p):
        self.d, self.p, self.N = d, p, p + 1
        N = self.N
        self.M = N ** d
        self.xq, self.wq = B.tensor_points(d, N)
        self.Phi = B.eval_basis(self.xq, N)          # (Q, M)
        self.dPhi = B.eval_basis_grad(self.xq, N)     # (Q, M, d)
        self.faces = []
        for f in range(2 * d):
            a, s = divmod(f, 2)
            xf, wf = B.face_points(d, N, a, s)
            self.faces.append((xf, wf, B.eval_basis(xf, N)))
        # unweighted reference mass matrix by quadrature
        self.Mref = self.Phi.T @ (self.wq[:, None] * self.Phi)

    def ref_project(self, vals):
        """Reference-measure L2 projection of values given at the volume
        Gauss points: vals (..., Q) -> (..., M)."""
        rhs = np.einsum("qm,...q->...m", self.Phi * self.wq[:, None], vals)
        return np.einsum("mn,...n->...m", np.linalg.inv(self.Mref), rhs)


def _cells(d, n):
    return B.lattice(d, n)


def _cidx(I, n):
    return sum(int(I[a]) * n ** a for a in range(len(I)))


def _rotate(ops, K, pi, sigma):
    """R^n of Eq. (15): the polynomial given by K (..., M) in the source frame,
    re-expressed in my frame, where my reference coordinate xi_a corresponds
    to the source coordinate xi^s_{pi[a]} = sigma[a] xi_a.  Evaluated as the
    L2 projection of the rotated polynomial onto my basis (Sec. 3.5)."""
    d = ops.d
    xs = np.zeros_like(ops.xq)
    for a in range(d):
        xs[:, pi[a]] = sigma[a] * ops.xq[:, a]
    vals = np.einsum("qm,...m->...q", B.eval_basis(xs, ops.N), K)
    return ops.ref_project(vals)


def _split(ops, K_parent, corners_parent, e):
    """Eqs. (11)-(12): child e of a parent cell.  M_C K_C = R with
    R_l = int_{child} phi^C_l phi^P_j k^P_j dV, both integrals by the child's
    Gauss rule with the child's Jacobian (J_child = J_parent / 2^d)."""
    d = ops.d
    xP = (ops.xq + (2.0 * np.asarray(e) - 1.0)) * 0.5
    _, JP, _ = jacobian(corners_parent[None], xP)
    Jc = JP[0] / 2 ** d
    uP = np.einsum("qm,...m->...q", B.eval_basis(xP, ops.N), K_parent)
    W = ops.wq * Jc
    Mc = ops.Phi.T @ (W[:, None] * ops.Phi)
    R = np.einsum("qm,...q->...m", ops.Phi * W[:, None], uP)
    return np.einsum("mn,...n->...m", np.linalg.inv(Mc), R)


def _combine(ops, K_children, corners_children):
    """Eqs. (13)-(14) with reading R6: M_P K_P = sum_i R^(i),
    R^(i)_l = int_{child i} phi^P_l phi^C_j k^C_j dV and
    M_P = sum_i int_{child i} phi^P phi^P dV, every integral by child i's own
    Gauss rule with child i's Jacobian.  K_children: (2^d, ..., M) in child
    order e = sum_a bit_a 2^a; corners_children: (2^d, 2^d, d)."""
    d = ops.d
    MP = np.zeros((ops.M, ops.M))
    R = 0.0
    for i, e in enumerate(B.all_corner_bits(d)):
        xP = (ops.xq + (2.0 * np.asarray(e) - 1.0)) * 0.5
        PhiP = B.eval_basis(xP, ops.N)
        _, Jc, _ = jacobian(corners_children[i][None], ops.xq)
        W = ops.wq * Jc[0]
        MP += PhiP.T @ (W[:, None] * PhiP)
        uc = np.einsum("qm,...m->...q", ops.Phi, K_children[i])
        R = R + np.einsum("qm,...q->...m", PhiP * W[:, None], uc)
    return np.einsum("mn,...n->...m", np.linalg.inv(MP), R)


# ---------------------------------------------------------------- the solver
class Solver:
    """One forest + degree p: guard fill, residual, SSP-RK3, CFL, totals."""

    def __init__(self, forest, p, gamma=GAMMA, cfl=0.1, nonconforming="paper", limiter=None,
                 boundary=None):
        """nonconforming: "paper" (the guard scheme of Sec. 3.5 on both sides
        of a level jump) or "mortar" (reading R15: the coarse side takes the
        fine side's fluxes, integrated against its own test functions).
        limiter: None, or eps of the positivity limiter (reading R17) applied
        after every Runge-Kutta stage.
        boundary: None (every domain boundary face is outflow), or
        (tags, state): tags[root][face] = 1 makes that root face's guard
        cells the constant conserved state `state` (inflow / far field,
        reading R11), 0 keeps outflow."""
        assert nonconforming in ("paper", "mortar")
        self.F = forest
        self.d, self.n, self.p = forest.d, forest.n, p
        self.ops = Ops(self.d, p)
        self.gamma, self.cfl = gamma, cfl
        self.nonconforming = nonconforming
        self.limiter = limiter
        self.boundary = boundary
        self.nv = self.d + 2
        self._rot_cache = {}
        self.refresh()

    def refresh(self):
        """Re-derive leaf lists and per-leaf geometry after a regrid."""
        self._nbr_maps = self._build_nbr_maps()
        self.leaves = self.F.leaves()
        self.index = {k: i for i, k in enumerate(self.leaves)}
        self.corners = [self.F.cell_corners(k) for k in self.leaves]
        ops = self.ops
        self.geo_vol = []
        for C in self.corners:
            _, J, Ja = jacobian(C, ops.xq)
            self.geo_vol.append((J, Ja))
        self.geo_face = []
        for C in self.corners:
            per = []
            for f in range(2 * self.d):
                xf, wf, Pf = ops.faces[f]
                _, Jf, Jaf = jacobian(C, xf)
                per.append(Jaf)
            self.geo_face.append(per)
        self.kinds = [[self._face_kind(li, f) for f in range(2 * self.d)]
                      for li in range(len(self.leaves))]

    def _face_kind(self, li, f):
        """SAME, COARSER, FINER or BOUNDARY for face f of leaf li."""
        r, lev, pos = self.leaves[li]
        nb = self.F.neighbour_coords(r, lev, pos, f)
        if nb is None:
            return BOUNDARY
        r2, q, _, _ = nb
        if (r2, lev, q) in self.F.tree:
            return SAME if self.F.is_leaf((r2, lev, q)) else FINER
        return COARSER

    def _coarse_points(self, li, f):
        """Face f of leaf li has a coarser neighbour (the geometry of Eq. (16)):
        the coarse leaf index and, per guard index t, the coarse cell across my
        face cell t and the coarse cell's reference coordinates of my face
        Gauss points (the fine face is half of the coarse face per tangential
        axis; my axis a maps to the coarse axis pi[a] with sign sigma[a])."""
        F, ops, d, n = self.F, self.ops, self.d, self.n
        r, lev, pos = self.leaves[li]
        a, s = divmod(f, 2)
        tang = [t for t in range(d) if t != a]
        qbits = [x & 1 for x in pos]
        r2, Q, (pi, sigma), f2 = F.neighbour_coords(r, lev - 1, tuple(x >> 1 for x in pos), f)
        b2, s2 = divmod(f2, 2)
        xf = ops.faces[f][0]
        out = []
        for t in range(n ** (d - 1)):
            g = [0] * d
            for j, tt in enumerate(tang):
                g[tt] = (t // n ** j) % n
            h = [0] * d
            xc = np.zeros((len(xf), d))
            for tt in tang:
                G = qbits[tt] * n + g[tt]
                h[pi[tt]] = (G >> 1) if sigma[tt] > 0 else n - 1 - (G >> 1)
                xc[:, pi[tt]] = sigma[tt] * 0.5 * (xf[:, tt] + 2 * (G & 1) - 1)
            h[b2] = 0 if s2 == 0 else n - 1
            xc[:, b2] = -1.0 if s2 == 0 else 1.0
            out.append((_cidx(h, n), xc))
        return self.index[(r2, lev - 1, Q)], out

    def _build_nbr_maps(self):
        """Per face: the cell across it inside the block, or the guard index."""
        d, n = self.d, self.n
        maps = []
        for f in range(2 * d):
            a, s = divmod(f, 2)
            tang = [t for t in range(d) if t != a]
            src = np.zeros(n ** d, np.int64)
            inside = np.zeros(n ** d, bool)
            for c, I in enumerate(_cells(d, n)):
                J2 = list(I)
                J2[a] += 1 if s else -1
                if 0 <= J2[a] < n:
                    src[c], inside[c] = _cidx(J2, n), True
                else:
                    src[c] = sum(I[tt] * n ** j for j, tt in enumerate(tang))
            maps.append((src, inside))
        return maps

    def shape(self):
        return (len(self.leaves), self.nv, self.ops.M, self.n ** self.d)

    # ------------------------------------------------------------ guard fill
    def _rotation_matrix(self, pi, sigma):
        """Matrix of R^n (Eq. (15)): my coefficients = T @ source coefficients,
        built column by column from the quadrature projection in _rotate."""
        key = (tuple(pi), tuple(sigma))
        if key not in self._rot_cache:
            self._rot_cache[key] = _rotate(self.ops, np.eye(self.ops.M), pi, sigma).T
        return self._rot_cache[key]

    def guard_face(self, U, li, f):
        """Coefficients (nv, M, n^(d-1)), in leaf li's frame, of the guard
        cells next to face f; guard t sits at my tangential cell coordinates
        g_{t_j} = (t // n^j) % n (tangential axes t_j increasing).
        Sec. 3.5, Eqs. (15)-(17)."""
        F, ops, d, n = self.F, self.ops, self.d, self.n
        r, lev, pos = self.leaves[li]
        a, s = divmod(f, 2)
        tang = [t for t in range(d) if t != a]
        nt = n ** (d - 1)
        out = np.zeros((self.nv, ops.M, nt))
        gs = []
        for t in range(nt):
            g = [0] * d
            for j, tt in enumerate(tang):
                g[tt] = (t // n ** j) % n
            gs.append(g)
        nb = F.neighbour_coords(r, lev, pos, f)
        if nb is None and self.boundary is not None and self.boundary[0][r][f] == 1:
            # prescribed state: a constant guard cell (mode 0 only, P_0 = 1)
            out[:, 0, :] = np.asarray(self.boundary[1], float)[:, None]
            return out
        if nb is None:
            # outflow: mirror image of my own face cell across the face
            sign = np.array([(-1.0) ** k[a] for k in B.mode_indices(d, ops.N)])
            for t, g in enumerate(gs):
                own = list(g)
                own[a] = n - 1 if s else 0
                out[:, :, t] = U[li][:, :, _cidx(own, n)] * sign
            return out
        r2, q, (pi, sigma), f2 = nb
        b2, s2 = divmod(f2, 2)
        if (r2, lev, q) in F.tree:
            hs = []
            for g in gs:
                h = [0] * d
                for tt in tang:
                    h[pi[tt]] = g[tt] if sigma[tt] > 0 else n - 1 - g[tt]
                h[b2] = 0 if s2 == 0 else n - 1
                hs.append(h)
            if F.is_leaf((r2, lev, q)):                               # Eq. (15)
                T = self._rotation_matrix(pi, sigma)
                src = U[self.index[(r2, lev, q)]][:, :, [_cidx(h, n) for h in hs]]
                return np.einsum("mk,vkt->vmt", T, src)
            for t, h in enumerate(hs):                                 # Eq. (17)
                cN = [(2 * h[u]) // n for u in range(d)]
                fine = (r2, lev + 1, tuple(2 * q[u] + cN[u] for u in range(d)))
                fi = self.index[fine]
                Ks, Cs = [], []
                for e in B.all_corner_bits(d):
                    cell = [2 * h[u] + e[u] - cN[u] * n for u in range(d)]
                    Ks.append(U[fi][:, :, _cidx(cell, n)])
                    Cs.append(self.corners[fi][_cidx(cell, n)])
                KP = _combine(ops, np.array(Ks), np.array(Cs))
                out[:, :, t] = _rotate(ops, KP, pi, sigma)
            return out
        # coarser neighbour                                            Eq. (16)
        qbits = [x & 1 for x in pos]
        assert qbits[a] == s, "a coarser neighbour lies outside my parent"
        r2, Q, (pi, sigma), f2 = F.neighbour_coords(r, lev - 1, tuple(x >> 1 for x in pos), f)
        b2, s2 = divmod(f2, 2)
        ci = self.index[(r2, lev - 1, Q)]
        for t, g in enumerate(gs):
            h = [0] * d
            e = [0] * d
            for tt in tang:
                G = qbits[tt] * n + g[tt]
                h[pi[tt]] = (G >> 1) if sigma[tt] > 0 else n - 1 - (G >> 1)
                e[pi[tt]] = (G & 1) if sigma[tt] > 0 else 1 - (G & 1)
            h[b2] = 0 if s2 == 0 else n - 1
            e[b2] = 0 if s2 == 0 else 1
            Ks = U[ci][:, :, _cidx(h, n)]
            Kchild = _split(ops, Ks, self.corners[ci][_cidx(h, n)], e)
            out[:, :, t] = _rotate(ops, Kchild, pi, sigma)
        return out

    def fill_guardcells(self, U, leaves=None):
        """G[leaf][face][var][mode][t], t = sum_j g_{t_j} n^j (all leaves,
        or only the listed ones; the others stay zero)."""
        d, n = self.d, self.n
        nl = len(self.leaves)
        G = np.zeros((nl, 2 * d, self.nv, self.ops.M, n ** (d - 1)))
        for li in (range(nl) if leaves is None else leaves):
            for f in range(2 * d):
                G[li, f] = self.guard_face(U, li, f)
        return G

    # -------------------------------------------------------------- residual
    def residual(self, U, G=None, leaves=None):
        """L(U) = M^{-1} R per cell (Eqs. (3)-(4)); guard cells from Sec. 3.5.
        ``leaves`` restricts the evaluation to a subset (others stay zero).

        Mortar mode (reading R15): a face with finer neighbours gets no flux
        of its own; instead every fine face point's flux F_h (the fine side's
        Lax-Friedrichs flux, out of the fine cell, per fine reference area)
        enters the coarse cell's residual as + sum_k w_k phi_m(xi_c(x_k)) F_h,k
        -- the same surface integral, parametrised by the fine face."""
        ops, d, n, nv = self.ops, self.d, self.n, self.nv
        mortar = self.nonconforming == "mortar"
        todo = range(len(self.leaves)) if (leaves is None or mortar) else leaves
        if G is None:
            G = self.fill_guardcells(U, None if mortar else leaves)
        out = np.zeros_like(U)
        nc = n ** d
        R_all, extra = {}, {}
        for li in todo:
            K = np.transpose(U[li], (2, 0, 1))                      # (nc, nv, M)
            J, Ja = self.geo_vol[li]
            uq = np.einsum("qm,cvm->cqv", ops.Phi, K)
            Fq = physical_flux(uq, self.gamma)                      # (nc,Q,nv,d_j)
            Ft = np.einsum("cqij,cqvj->cqvi", Ja, Fq)               # contravariant
            R = np.einsum("q,cqvi,qmi->cvm", ops.wq, Ft, ops.dPhi, optimize=True)
            for f in range(2 * d):
                a, s = divmod(f, 2)
                xf, wf, Pf = ops.faces[f]
                Pf_opp = ops.faces[2 * a + (1 - s)][2]
                uL = np.einsum("fm,cvm->cfv", Pf, K)
                src, inside = self._nbr_maps[f]
                KR = np.where(inside[:, None, None], K[np.where(inside, src, 0)],
                              np.transpose(G[li, f], (2, 0, 1))[np.where(inside, 0, src)])
                uR = np.einsum("fm,cvm->cfv", Pf_opp, KR)
                area = (1.0 if s else -1.0) * self.geo_face[li][f][:, :, a, :]  # (nc,nf,d)
                dS = np.linalg.norm(area, axis=-1)
                nhat = area / dS[..., None]
                Fh = lax_friedrichs(uL, uR, nhat, self.gamma) * dS[..., None]
                if mortar and self.kinds[li][f] == FINER:
                    Fh[~inside] = 0.0  # the fine side's fluxes arrive below
                R -= np.einsum("f,fm,cfv->cvm", wf, Pf, Fh, optimize=True)
                if mortar and self.kinds[li][f] == COARSER:
                    ci, pts = self._coarse_points(li, f)
                    Rc = extra.setdefault(ci, np.zeros((nc, nv, ops.M)))
                    for c in np.nonzero(~inside)[0]:
                        hc, xc = pts[src[c]]
                        Pc = B.eval_basis(xc, ops.N)
                        Rc[hc] += np.einsum("f,fm,fv->vm", wf, Pc, Fh[c])
            R_all[li] = R
        for li in (range(len(self.leaves)) if leaves is None else leaves):
            R = R_all[li] + extra[li] if li in extra else R_all[li]
            J, _ = self.geo_vol[li]
            Mc = np.einsum("q,cq,qm,qn->cmn", ops.wq, J, ops.Phi, ops.Phi, optimize=True)
            Kdot = np.linalg.solve(Mc[:, None], R[..., None])[..., 0]
            out[li] = np.transpose(Kdot, (1, 2, 0))
        return out

    # ------------------------------------------------------------ time march
    def dt(self, U):
        """Reading R5: CFL * min over cells, quad points of h/sum_i(|u_i|+c)."""
        ops, d = self.ops, self.d
        best = np.inf
        for li in range(len(self.leaves)):
            K = np.transpose(U[li], (2, 0, 1))
            J, _ = self.geo_vol[li]
            uq = np.einsum("qm,cvm->cqv", ops.Phi, K)
            _, vel, _ = primitives(uq, self.gamma)
            c = sound_speed(uq, self.gamma)
            lam = np.sum(np.abs(vel), axis=-1) + d * c
            h = np.einsum("q,cq->c", ops.wq, J) ** (1.0 / d)
            best = min(best, float(np.min(h[:, None] / lam)))
        return self.cfl * best

    def _limit(self, U):
        if getattr(self, "limiter", None) is None:
            return U
        from .limiter import positivity_limit
        return positivity_limit(self, U, self.limiter)[0]

    def ssp_rk3_step(self, U, dt):
        """Shu-Osher SSP-RK3 (Sec. 2, last paragraph; reading R4), with the
        positivity limiter after every stage when enabled (reading R17)."""
        u1 = self._limit(U + dt * self.residual(U))
        u2 = self._limit(0.75 * U + 0.25 * (u1 + dt * self.residual(u1)))
        return self._limit(U / 3.0 + 2.0 / 3.0 * (u2 + dt * self.residual(u2)))

    def run(self, U, steps, t_end=np.inf):
        t = 0.0
        for _ in range(steps):
            dt = min(self.dt(U), t_end - t)
            if dt <= 0:
                break
            U = self.ssp_rk3_step(U, dt)
            t += dt
        return U, t

    def totals(self, U):
        """T_v = sum_cells sum_q w_q J_q u_v(q)."""
        ops = self.ops
        T = np.zeros(self.nv)
        for li in range(len(self.leaves)):
            K = np.transpose(U[li], (2, 0, 1))
            J, _ = self.geo_vol[li]
            uq = np.einsum("qm,cvm->cqv", ops.Phi, K)
            T += np.einsum("q,cq,cqv->v", ops.wq, J, uq, optimize=True)
        return T

    # ------------------------------------------------------------ projection
    def quad_points(self):
        """Physical volume Gauss points [leaf][cell][q][d]."""
        return np.array([map_points(C, self.ops.xq) for C in self.corners])

    def project(self, fun):
        """L2 projection (reading R2 quadrature) of fun(x[..., d]) -> (..., nv)."""
        ops = self.ops
        U = np.zeros(self.shape())
        for li, C in enumerate(self.corners):
            x = map_points(C, ops.xq)
            vals = fun(x)                                           # (nc, Q, nv)
            J, _ = self.geo_vol[li]
            Mc = np.einsum("q,cq,qm,qn->cmn", ops.wq, J, ops.Phi, ops.Phi, optimize=True)
            rhs = np.einsum("q,cq,qm,cqv->cvm", ops.wq, J, ops.Phi, vals, optimize=True)
            K = np.linalg.solve(Mc[:, None], rhs[..., None])[..., 0]
            U[li] = np.transpose(K, (1, 2, 0))
        return U

    def l2_error(self, U, fun):
        """sqrt(sum_v int (u_v - f_v)^2 dV) / sqrt(sum_v int f_v^2 dV)."""
        ops = self.ops
        num = den = 0.0
        for li, C in enumerate(self.corners):
            x = map_points(C, ops.xq)
            ex = fun(x)
            K = np.transpose(U[li], (2, 0, 1))
            uq = np.einsum("qm,cvm->cqv", ops.Phi, K)
            J, _ = self.geo_vol[li]
            num += float(np.einsum("q,cq,cqv->", ops.wq, J, (uq - ex) ** 2, optimize=True))
            den += float(np.einsum("q,cq,cqv->", ops.wq, J, ex ** 2, optimize=True))
        return np.sqrt(num / den)

    # ---------------------------------------------------- data inheritance
    def regrid_state(self, old_solver, U_old):
        """State on the current leaves from the state on old_solver's leaves:
        unchanged leaves copy, new children use the split of Eqs. (11)-(12),
        new parents use the combine of Eqs. (13)-(14) (Sec. 3.4)."""
        d, n, ops = self.d, self.n, self.ops
        U = np.zeros(self.shape())
        for li, key in enumerate(self.leaves):
            if key in old_solver.index:
                U[li] = U_old[old_solver.index[key]]
                continue
            r, lev, pos = key
            parent = (r, lev - 1, tuple(x >> 1 for x in pos))
            if parent in old_solver.index:
                pi = old_solver.index[parent]
                cb = [x & 1 for x in pos]
                for c, I in enumerate(_cells(d, n)):
                    H = [cb[a] * n + I[a] for a in range(d)]
                    Pc = [h >> 1 for h in H]
                    e = [h & 1 for h in H]
                    pc = _cidx(Pc, n)
                    U[li][:, :, c] = _split(ops, U_old[pi][:, :, pc],
                                            old_solver.corners[pi][pc], e)
                continue
            for c, I in enumerate(_cells(d, n)):
                Ks, Cs = [], []
                for e in B.all_corner_bits(d):
                    H = [2 * I[a] + e[a] for a in range(d)]
                    cb = [h // n for h in H]
                    kid = (r, lev + 1, tuple(2 * pos[a] + cb[a] for a in range(d)))
                    ki = old_solver.index[kid]
                    cc = _cidx([H[a] - cb[a] * n for a in range(d)], n)
                    Ks.append(U_old[ki][:, :, cc])
                    Cs.append(old_solver.corners[ki][cc])
                U[li][:, :, c] = _combine(ops, np.array(Ks), np.array(Cs))
        return U


__all__ = ["Solver", "Ops", "jacobian", "map_points", "shape_functions",
           "SAME", "COARSER", "FINER", "BOUNDARY", "orient_decode"]
