"""Seeded synthetic workloads shared by the CUDA path's tests/bench and the oracle.

This module holds *inputs only*: root-block node lattices, per-root cell nodes
(optionally jittered), root-frame rotations, refinement lists, initial-condition
formulas evaluated at given physical points, and random valid modal states.  It
holds none of the DG method's arithmetic (no basis, quadrature, projection,
flux or time stepping), so that both independent implementations can consume
exactly the same inputs.

Conventions shared by every consumer (they describe the input format):
  * ``dim`` d in {2, 3}; ``n_seg`` cells per block edge (Sec. 3.3).
  * A root block is given by its 2^d corner node ids in *local lexicographic*
    order: corner bit a (value 0 -> local coordinate -1, 1 -> +1) is bit a of
    the corner index (x fastest).
  * ``root_cell_nodes[r]`` is the (n_seg+1)^d x d array of the root's cell
    nodes in local lexicographic order (x fastest).
  * Conserved variables are (rho, rho*u_1..rho*u_d, E) with gamma = 1.4
    (Eq. 2 and the ideal-gas law Eq. 23).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

GAMMA = 1.4


# --------------------------------------------------------------------------
# root-frame rotations (proper signed axis permutations)
# --------------------------------------------------------------------------
def proper_rotations(d):
    """All proper signed permutations (perm, signs) of d axes.

    Local axis a of a rotated root maps to global axis perm[a] with sign
    signs[a].  'Proper' means determinant +1 (8 in 2D... 4 proper, 24 in 3D).
    """
    out = []
    for perm in itertools.permutations(range(d)):
        # parity of the permutation
        inv = sum(1 for i in range(d) for j in range(i + 1, d) if perm[i] > perm[j])
        psign = -1 if inv % 2 else 1
        for signs in itertools.product((1, -1), repeat=d):
            if psign * int(np.prod(signs)) == 1:
                out.append((tuple(perm), tuple(signs)))
    return out


def _local_to_global_index(I, n, perm, signs):
    """Map a local lattice index I (0..n per axis) to a global offset."""
    d = len(perm)
    g = [0] * d
    for a in range(d):
        g[perm[a]] = I[a] if signs[a] > 0 else n - I[a]
    return g


# --------------------------------------------------------------------------
# lattice forests
# --------------------------------------------------------------------------
def lattice_forest(d, roots_per_axis, extent, n_seg, *, jitter=0.0,
                   rotate_roots=False, seed=0, origin=None, periodic=True):
    """Roots on a regular lattice of ``roots_per_axis^d`` blocks.

    roots_per_axis: an int, or one count per axis (anisotropic roots, e.g.
        (1, 3): a strip of three roots, each glued to itself across x).
    extent: physical edge length of the whole domain (cube/square).
    jitter: cell nodes strictly interior to the domain are moved by a seeded
        uniform offset in [-jitter*h, +jitter*h] per coordinate (h = cell size);
        nodes on the domain boundary stay fixed so periodic faces stay planar.
    rotate_roots: each root gets a seeded proper rotation of its local frame,
        so neighbouring roots see each other through non-trivial orientations.
    Returns a dict with keys dim, n_seg, nodes, root_corners, root_cell_nodes,
    periodic (list of translation vectors), root_block (lattice coords),
    root_frame ((perm, signs) per root).
    """
    rng = np.random.default_rng(seed)
    if np.ndim(roots_per_axis) == 0:
        Bs = (int(roots_per_axis),) * d
    else:
        Bs = tuple(int(b) for b in roots_per_axis)
        assert len(Bs) == d
    n = int(n_seg)
    G = tuple(B * n + 1 for B in Bs)  # global lattice nodes per axis
    hs = [extent / (B * n) for B in Bs]
    org = np.zeros(d) if origin is None else np.asarray(origin, float)

    # global cell-node lattice, index order x fastest: lat[k][j][i] in 3D
    axes = [org[a] + hs[a] * np.arange(G[a]) for a in range(d)]
    grids = np.meshgrid(*axes, indexing="ij")  # grids[a][i0,i1,...]
    lat = np.stack(grids, axis=-1)  # shape G + (d,), index [i0,i1,..]
    if jitter > 0.0:
        interior = np.ones(G, bool)
        for a in range(d):
            sl = [slice(None)] * d
            sl[a] = 0
            interior[tuple(sl)] = False
            sl[a] = G[a] - 1
            interior[tuple(sl)] = False
        if len(set(Bs)) == 1:
            noise = rng.uniform(-jitter * hs[0], jitter * hs[0], size=lat.shape)
        else:
            noise = rng.uniform(-jitter, jitter, size=lat.shape) * np.asarray(hs)
        lat = lat + noise * interior[..., None]

    # block-corner nodes: lattice points at multiples of n
    Cs = [B + 1 for B in Bs]
    ncorner = int(np.prod(Cs))
    nodes = np.zeros((ncorner, d))
    ids = {}
    for flat in range(ncorner):
        c, r = [], flat
        for a in range(d):
            c.append(r % Cs[a])
            r //= Cs[a]
        ids[tuple(c)] = flat
        nodes[flat] = lat[tuple(ci * n for ci in c)]

    rots = proper_rotations(d)
    root_corners, root_cell_nodes, root_block, root_frame = [], [], [], []
    for flat in range(int(np.prod(Bs))):
        b, r = [], flat
        for a in range(d):
            b.append(r % Bs[a])
            r //= Bs[a]
        if rotate_roots:
            perm, signs = rots[int(rng.integers(len(rots)))]
        else:
            perm, signs = tuple(range(d)), (1,) * d
        corners = []
        for k in range(2 ** d):
            kap = [(k >> a) & 1 for a in range(d)]
            off = _local_to_global_index(kap, 1, perm, signs)
            corners.append(ids[tuple(b[a] + off[a] for a in range(d))])
        # local node li (x fastest) -> global lattice index, all at once
        li = np.arange((n + 1) ** d)
        gidx = [None] * d
        for a in range(d):
            Ia = (li // (n + 1) ** a) % (n + 1)
            gidx[perm[a]] = b[perm[a]] * n + (Ia if signs[a] > 0 else n - Ia)
        cn = lat[tuple(gidx)]
        root_corners.append(corners)
        root_cell_nodes.append(cn)
        root_block.append(tuple(b))
        root_frame.append((perm, signs))

    per = []
    if periodic:
        for a in range(d):
            v = np.zeros(d)
            v[a] = extent
            per.append(v)
    return dict(dim=d, n_seg=n, nodes=nodes,
                root_corners=np.asarray(root_corners, np.int64),
                root_cell_nodes=np.asarray(root_cell_nodes),
                periodic=per, root_block=root_block, root_frame=root_frame,
                extent=float(extent), origin=org)


def single_root_2d(n_seg=4, refine=True):
    """One square root covering the periodic unit square, glued to itself
    across both axes (the first root set of the 2D convection test, Sec. 5);
    with ``refine`` its corner child is refined again, so the 2:1 closure and
    the level jumps wrap around the periodic faces."""
    w = lattice_forest(2, 1, 1.0, n_seg)
    if refine:
        w["refine"] = [[(0, 1, (0, 0))], [(0, 2, (0, 0))]]
    return w


def three_root_strip_2d(n_seg=4, seed=1, refine=True):
    """Three rectangular roots stacked along y over the periodic unit square,
    each in a seeded rotated local frame (the third root set of the 2D
    convection test, Sec. 5: roots in relative rotation); every root is glued
    to itself across x and to its neighbours across y."""
    w = lattice_forest(2, (1, 3), 1.0, n_seg, rotate_roots=True, seed=seed)
    if refine:
        w["refine"] = [[(1, 1, (0, 0))]]
    return w


def local_child_toward(frame, global_dir_bits):
    """Child position (local frame bits) whose global offset bits are given."""
    perm, signs = frame
    d = len(perm)
    c = [0] * d
    for a in range(d):
        want = global_dir_bits[perm[a]]
        c[a] = want if signs[a] > 0 else 1 - want
    return tuple(c)


# --------------------------------------------------------------------------
# the five workload shapes
# --------------------------------------------------------------------------
def vortex2d_forest():
    """2D periodic [0,10]^2, 4x4 root quads of 8x8 cells, central 2x2 roots
    refined once (28 leaves, 1792 cells).  Refinement list is in
    (root, level, pos) form, applied in order."""
    f = lattice_forest(2, 4, 10.0, 8)
    refine = []
    for r, b in enumerate(f["root_block"]):
        if b[0] in (1, 2) and b[1] in (1, 2):
            refine.append((r, 1, (0, 0)))
    f["refine"] = [refine]
    f["p"] = 2
    f["cfl"] = 0.1
    return f


def jitter3d_forest(seed=0, n_seg=8, rotate_roots=True, jitter=0.1):
    """3D unit cube, 2x2x2 hex roots with seeded rotated local frames and
    +-10% interior node jitter; all roots refined once, then the level-2
    block of root 0 touching the domain centre refined again (71 leaves,
    36,352 cells at n_seg=8)."""
    f = lattice_forest(3, 2, 1.0, n_seg, jitter=jitter,
                       rotate_roots=rotate_roots, seed=seed)
    first = [(r, 1, (0, 0, 0)) for r in range(8)]
    c = local_child_toward(f["root_frame"][0], (1, 1, 1))
    f["refine"] = [first, [(0, 2, c)]]
    f["p"] = 2
    f["cfl"] = 0.1
    return f


def periodic_cube_forest(B, n_seg=8, rotate_roots=False, seed=0):
    """3D periodic unit cube of B^3 single-level root blocks."""
    f = lattice_forest(3, B, 1.0, n_seg, rotate_roots=rotate_roots, seed=seed)
    f["refine"] = []
    return f


# --------------------------------------------------------------------------
# initial conditions (point formulas -> conserved variables)
# --------------------------------------------------------------------------
def prim_to_cons(rho, vel, p, gamma=GAMMA):
    """(rho, velocity[..., d], p) -> conserved (..., d+2)  (Eq. 2, Eq. 23)."""
    vel = np.asarray(vel)
    d = vel.shape[-1]
    out = np.empty(np.shape(rho) + (d + 2,))
    out[..., 0] = rho
    for a in range(d):
        out[..., 1 + a] = rho * vel[..., a]
    out[..., d + 1] = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=-1)
    return out


def isentropic_vortex(x, *, beta=5.0, centre=(5.0, 5.0), scale=1.0,
                      free=(1.0, 1.0, 1.0, 1.0, 1.0), gamma=GAMMA):
    """Shu/Yee isentropic vortex (strength beta, unit core) in the x-y plane,
    extruded along z in 3D.  ``scale`` maps the domain to the vortex box
    (x_vortex = scale * x).  free = (rho, u, v[, w], p) of the free stream.
    Periodic images are ignored."""
    x = np.asarray(x, float)
    d = x.shape[-1]
    X = scale * x[..., 0] - centre[0]
    Y = scale * x[..., 1] - centre[1]
    r2 = X * X + Y * Y
    e = np.exp(0.5 * (1.0 - r2))
    du = -beta / (2 * math.pi) * e * Y
    dv = beta / (2 * math.pi) * e * X
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    vel = np.zeros(x.shape[:-1] + (d,))
    vel[..., 0] = free[1] + du
    vel[..., 1] = free[2] + dv
    if d == 3:
        vel[..., 2] = free[3]
    return prim_to_cons(rho, vel, p, gamma)


def vortex_exact(x, t, *, scale=1.0, centre=(5.0, 5.0), period=10.0, **kw):
    """The vortex translated by the free stream (u=v=1) over time t, with the
    centre wrapped into the periodic box of edge ``period`` (vortex units)."""
    c = ((centre[0] + t * scale) % period, (centre[1] + t * scale) % period)
    x = np.asarray(x, float)
    # shift every point to the nearest periodic image of the moved centre
    X = scale * x[..., 0]
    Y = scale * x[..., 1]
    dx = (X - c[0] + period / 2) % period - period / 2
    dy = (Y - c[1] + period / 2) % period - period / 2
    xs = np.array(x, copy=True)
    xs[..., 0] = (dx + centre[0]) / scale
    xs[..., 1] = (dy + centre[1]) / scale
    return isentropic_vortex(xs, scale=scale, centre=centre, **kw)


def free_stream(x, state=(1.0, 0.3, -0.2, 0.1, 1.0), gamma=GAMMA):
    x = np.asarray(x, float)
    d = x.shape[-1]
    rho = np.full(x.shape[:-1], state[0])
    vel = np.zeros(x.shape[:-1] + (d,))
    for a in range(d):
        vel[..., a] = state[1 + a]
    p = np.full(x.shape[:-1], state[-1])
    return prim_to_cons(rho, vel, p, gamma)


def blast(x, centre, r0=0.1, width=1.0 / 128, gamma=GAMMA):
    """Spherical blast: inside (rho, p) = (8, 10), outside (1, 1), at rest,
    interface smoothed by a tanh of the given width."""
    x = np.asarray(x, float)
    d = x.shape[-1]
    r = np.sqrt(np.sum((x - np.asarray(centre)) ** 2, axis=-1))
    s = 0.5 * (1.0 - np.tanh((r - r0) / width))
    rho = 1.0 + 7.0 * s
    p = 1.0 + 9.0 * s
    vel = np.zeros(x.shape[:-1] + (d,))
    return prim_to_cons(rho, vel, p, gamma)


def blast_centre(seed):
    return np.random.default_rng(seed).uniform(0.4, 0.6, size=3)


# --------------------------------------------------------------------------
# a stream of independent solves (continuous batching)
# --------------------------------------------------------------------------
def serving_mix(n_requests, *, rate=20.0, seed=0, blocks=(64, 8192), degrees=(1, 2, 3),
                t_end=(0.05, 0.5), t_scale=1.0, n_seg=8):
    """Requests arriving by a Poisson process of `rate` per second.  Each is a
    3D periodic unit cube of B^3 single-level roots, with the block count
    drawn log-uniformly in `blocks` and rounded to the nearest cube; the
    initial condition is a blast or the extruded vortex with probability 1/2
    each; p is uniform over `degrees`; t_end is uniform in `t_end` times
    `t_scale`.  Returns plain dicts (no forest is built here)."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    out = []
    for i in range(n_requests):
        nb = math.exp(rng.uniform(math.log(blocks[0]), math.log(blocks[1])))
        B = max(1, int(round(nb ** (1.0 / 3.0))))
        kind = "blast" if rng.uniform() < 0.5 else "vortex"
        p = int(degrees[rng.integers(len(degrees))])
        te = float(rng.uniform(*t_end)) * t_scale
        centre = rng.uniform(0.4, 0.6, size=3)
        out.append(dict(rid=i, arrival=float(arrivals[i]), B=B, n_seg=n_seg, p=p, t_end=te,
                        kind=kind, centre=centre))
    return out


def serving_initial(req):
    """Initial-condition formula of a serving_mix request: the blast with its
    interface one cell wide, or the vortex scaled to the unit cube."""
    if req["kind"] == "blast":
        width = 1.0 / (req["B"] * req["n_seg"])
        return lambda x: blast(x, req["centre"], width=width)
    return lambda x: isentropic_vortex(x, scale=10.0, centre=(5.0, 5.0))


# --------------------------------------------------------------------------
# random valid modal states (for element-wise parity tests)
# --------------------------------------------------------------------------
def random_modal_state(n_leaves, d, n_seg, p, seed=0, amp=0.05):
    """Modal coefficients in the SoA layout [leaf][var][mode][cell].

    Mode 0 (the cell mean of unnormalised tensor Legendre P_k, mode index
    m = sum_a k_a (p+1)^a) carries a positive state near
    (rho, u, p) = (1, 0.3, 1); higher modes carry small seeded noise, so that
    density and pressure stay positive at every quadrature point.
    """
    rng = np.random.default_rng(seed)
    N = p + 1
    M = N ** d
    nc = n_seg ** d
    nv = d + 2
    U = np.zeros((n_leaves, nv, M, nc))
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, size=(n_leaves, nc))
    vel = 0.3 + 0.2 * rng.uniform(-1, 1, size=(n_leaves, nc, d))
    pr = 1.0 + 0.1 * rng.uniform(-1, 1, size=(n_leaves, nc))
    cons = prim_to_cons(rho, vel, pr)  # (L, nc, nv)
    U[:, :, 0, :] = np.transpose(cons, (0, 2, 1))
    if M > 1:
        a = amp * 3.0 / math.sqrt(M)
        U[:, :, 1:, :] = a * rng.uniform(-1, 1, size=(n_leaves, nv, M - 1, nc))
        U[:, 0, 1:, :] *= 0.5
    return U


# --------------------------------------------------------------------------
# small hand-checkable forests
# --------------------------------------------------------------------------
def rotated_pair_2d(n_seg=2, refine_root0=True):
    """Two unit root quads on [0,2]x[0,1], periodic in x and y.  Root 1's
    local x axis is global +y and its local y axis is global -x.  No cell
    nodes are given: they follow from the corners."""
    nodes = np.array([(0, 0), (1, 0), (2, 0), (0, 1), (1, 1), (2, 1)], float)
    f = dict(dim=2, n_seg=n_seg, nodes=nodes,
             root_corners=np.array([[0, 1, 3, 4], [2, 5, 1, 4]], np.int64),
             root_cell_nodes=None,
             periodic=[np.array([2.0, 0.0]), np.array([0.0, 1.0])])
    f["refine"] = [[(0, 1, (0, 0))]] if refine_root0 else []
    return f


def smooth_x_state(x, Lx=2.0):
    """A smooth periodic state that depends on the first coordinate only."""
    x = np.asarray(x, float)
    d = x.shape[-1]
    s = 2 * math.pi * x[..., 0] / Lx
    rho = 1.0 + 0.2 * np.sin(s)
    vel = np.zeros(x.shape[:-1] + (d,))
    vel[..., 0] = 0.5 + 0.1 * np.cos(s)
    pr = 1.0 + 0.1 * np.sin(s + 0.3)
    return prim_to_cons(rho, vel, pr)


ADVECT_VEL = (0.3, -0.2, 0.1)


def advected_polynomial(x, p):
    """rho a polynomial of total degree p in x, constant velocity ADVECT_VEL
    and constant pressure 1 (a state whose Euler flux is a polynomial of
    degree p)."""
    x = np.asarray(x, float)
    d = x.shape[-1]
    X = [x[..., a] for a in range(d)]
    rho = 1.0 + 0.1 * X[0] + 0.2 * X[1] - (0.15 * X[2] if d == 3 else 0.0)
    if p >= 2:
        rho = rho + 0.05 * X[0] * X[1] - 0.04 * X[1] ** 2
    if p >= 3:
        rho = rho + 0.02 * X[0] ** 3 - 0.03 * X[0] * X[1] * X[-1]
    if p == 0:
        rho = np.full(x.shape[:-1], 1.2)
    vel = np.broadcast_to(np.array(ADVECT_VEL[:d]), x.shape[:-1] + (d,))
    return prim_to_cons(rho, vel, np.ones(x.shape[:-1]))


def smooth_state(x, extent=1.0):
    """A smooth periodic state varying along every axis."""
    x = np.asarray(x, float)
    d = x.shape[-1]
    s = 2 * math.pi * x / extent
    rho = 1.0 + 0.2 * np.prod(np.sin(s), axis=-1) + 0.1 * np.cos(s[..., 0])
    vel = 0.3 + 0.1 * np.cos(s + 0.5)
    pr = 1.0 + 0.1 * np.sin(np.sum(s, axis=-1))
    return prim_to_cons(rho, vel, pr)
