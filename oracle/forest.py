"""Block forest topology and block geometry (oracle; test infrastructure).

Sec. 3.1: blocks form quad/oct trees grown from unstructured root blocks; the
root blocks are at refinement level 1 and the neighbour relation of a new
block follows from its parent's neighbours and its position among its
siblings; the array R records the relative rotation of each neighbour.
Sec. 3.3: a block holds N_seg^d cells whose nodes follow from the block's
configuration nodes by the (bi/tri)linear interpolation of Eq. (6); a child's
nodes follow from its parent by the same interpolation.

Canonical rules (the C++ forest in the product follows the same rules from
its own code; integer tables must agree bit for bit):
  * face f = 2*axis + side (side 0: xi_axis = -1, side 1: +1).
  * root faces are matched by corner nodes: first by shared node ids, then
    by positions shifted by a periodic translation sum_i c_i t_i with
    c in {-1,0,1}^k (itertools.product order, zero vector skipped); the first
    match in (root, face, shift) order wins.
  * orientation of a neighbour = signed axis permutation (pi, sigma): my axis
    a maps to the neighbour's axis pi[a] with sign sigma[a]; code =
    perm_index * 2^d + sum_a [sigma[a] < 0] 2^a, perm_index the position of
    pi in itertools.permutations(range(d)).
  * leaves are ordered root by root, depth first, children in order
    c = sum_a bit_a 2^a.
  * neighbour kinds: 0 same level, 1 coarser, 2 finer, 3 domain boundary;
    for kind 2 the 2^(d-1) fine leaves are listed by sub-face index
    sum_j bit_{t_j} 2^j over my tangential axes t_j in increasing order.
  * 2:1 balance across faces is enforced by refining the coarser side.
"""
from __future__ import annotations

import itertools

import numpy as np

from .basis import all_corner_bits

SAME, COARSER, FINER, BOUNDARY = 0, 1, 2, 3


def perm_list(d):
    return list(itertools.permutations(range(d)))


def orient_code(pi, sigma):
    d = len(pi)
    k = perm_list(d).index(tuple(pi))
    bits = sum((1 << a) for a in range(d) if sigma[a] < 0)
    return k * (1 << d) + bits


def orient_decode(code, d):
    k, bits = divmod(code, 1 << d)
    pi = perm_list(d)[k]
    sigma = tuple(-1 if (bits >> a) & 1 else 1 for a in range(d))
    return pi, sigma


class BalanceError(RuntimeError):
    pass


class Forest:
    def __init__(self, dim, n_seg, nodes, root_corners, root_cell_nodes=None,
                 periodic=(), tol=1e-9):
        self.d = int(dim)
        self.n = int(n_seg)
        self.nodes = np.asarray(nodes, float)
        self.root_corners = np.asarray(root_corners, np.int64)
        self.R = len(self.root_corners)
        self.periodic = [np.asarray(t, float) for t in periodic]
        scale = 1.0 + float(np.max(np.abs(self.nodes))) if len(self.nodes) else 1.0
        self.tol = tol * scale
        d, n = self.d, self.n
        if root_cell_nodes is None:
            self.root_nodes = [self._interp_from_corners(r) for r in range(self.R)]
        else:
            self.root_nodes = [np.asarray(x, float).reshape((n + 1) ** d, d)
                               for x in root_cell_nodes]
        self.root_face = {}
        self._match_root_faces()
        self.tree = {}
        for r in range(self.R):
            self.tree[(r, 1, (0,) * d)] = True
        self._node_cache = {}
        self._order = None

    # ---------------------------------------------------------------- roots
    def _interp_from_corners(self, r):
        """Eq. (6): node at reference point xi = sum_k N_k(xi) r_k,
        N_k = prod_a (1 + s_{k,a} xi_a)/2."""
        d, n = self.d, self.n
        X = self.nodes[self.root_corners[r]]
        out = np.zeros(((n + 1) ** d, d))
        for li in range((n + 1) ** d):
            I = [(li // (n + 1) ** a) % (n + 1) for a in range(d)]
            xi = [-1.0 + 2.0 * I[a] / n for a in range(d)]
            for k, bits in enumerate(all_corner_bits(d)):
                wgt = 1.0
                for a in range(d):
                    s = 1.0 if bits[a] else -1.0
                    wgt *= 0.5 * (1.0 + s * xi[a])
                out[li] += wgt * X[k]
        return out

    def _face_corners(self, f):
        a, s = divmod(f, 2)
        return [k for k, b in enumerate(all_corner_bits(self.d)) if b[a] == s]

    def _shifts(self):
        k = len(self.periodic)
        out = []
        for c in itertools.product((-1, 0, 1), repeat=k):
            if all(ci == 0 for ci in c):
                continue
            v = np.zeros(self.d)
            for ci, t in zip(c, self.periodic):
                v = v + ci * t
            out.append(v)
        return out

    def _match_root_faces(self):
        d = self.d
        shifts = self._shifts()
        for r in range(self.R):
            for f in range(2 * d):
                mine = self._face_corners(f)
                ids = [int(self.root_corners[r][k]) for k in mine]
                pos = [self.nodes[i] for i in ids]
                found = None
                for r2 in range(self.R):
                    for f2 in range(2 * d):
                        if (r2, f2) == (r, f):
                            continue
                        theirs = self._face_corners(f2)
                        ids2 = [int(self.root_corners[r2][k]) for k in theirs]
                        # shared node ids
                        if sorted(ids) == sorted(ids2):
                            corr = {k: theirs[ids2.index(i)] for k, i in zip(mine, ids)}
                            found = (r2, f2, corr)
                            break
                        pos2 = [self.nodes[i] for i in ids2]
                        for t in shifts:
                            corr = {}
                            for k, x in zip(mine, pos):
                                hit = [k2 for k2, y in zip(theirs, pos2)
                                       if np.max(np.abs(x + t - y)) <= self.tol]
                                if len(hit) != 1:
                                    break
                                corr[k] = hit[0]
                            if len(corr) == len(mine) and len(set(corr.values())) == len(mine):
                                found = (r2, f2, corr)
                                break
                        if found:
                            break
                    if found:
                        break
                if found is None:
                    continue
                r2, f2, corr = found
                self.root_face[(r, f)] = (r2, f2, self._orientation(f, f2, corr))

    def _orientation(self, f, f2, corr):
        d = self.d
        a, s = divmod(f, 2)
        b2, s2 = divmod(f2, 2)
        bits = all_corner_bits(d)
        pi = [None] * d
        sigma = [None] * d
        pi[a] = b2
        sigma[a] = 1 if s != s2 else -1
        base = [k for k in corr if all(bits[k][t] == 0 for t in range(d) if t != a)][0]
        for t in range(d):
            if t == a:
                continue
            other = [k for k in corr
                     if bits[k][t] == 1 and all(bits[k][u] == 0 for u in range(d) if u not in (a, t))][0]
            kb, ko = bits[corr[base]], bits[corr[other]]
            diff = [u for u in range(d) if kb[u] != ko[u]]
            assert len(diff) == 1 and diff[0] != b2
            pi[t] = diff[0]
            sigma[t] = 1 if ko[diff[0]] == 1 else -1
        # check the whole corner map
        for k, k2 in corr.items():
            for t in range(d):
                if t == a:
                    continue
                want = bits[k][t] if sigma[t] > 0 else 1 - bits[k][t]
                assert bits[k2][pi[t]] == want
        return tuple(pi), tuple(sigma)

    # ---------------------------------------------------------------- trees
    def neighbour_coords(self, r, lev, pos, f):
        """Same-level block coordinates across face f, or None at a boundary.

        Returns (root, pos, (pi, sigma), f2) with f2 the neighbour's face."""
        d = self.d
        a, s = divmod(f, 2)
        L = 1 << (lev - 1)
        p2 = list(pos)
        p2[a] += 1 if s else -1
        if 0 <= p2[a] < L:
            return r, tuple(p2), (tuple(range(d)), (1,) * d), 2 * a + (1 - s)
        if (r, f) not in self.root_face:
            return None
        r2, f2, (pi, sigma) = self.root_face[(r, f)]
        q = [0] * d
        for t in range(d):
            if t != a:
                q[pi[t]] = pos[t] if sigma[t] > 0 else L - 1 - pos[t]
        b2, s2 = divmod(f2, 2)
        q[b2] = 0 if s2 == 0 else L - 1
        return r2, tuple(q), (pi, sigma), f2

    def is_leaf(self, key):
        return self.tree.get(key) is True

    def leaves(self):
        if self._order is None:
            out = []
            for r in range(self.R):
                self._dfs((r, 1, (0,) * self.d), out)
            self._order = out
        return self._order

    def _dfs(self, key, out):
        if self.tree[key]:
            out.append(key)
            return
        r, lev, pos = key
        for bits in all_corner_bits(self.d):
            self._dfs((r, lev + 1, tuple(2 * pos[a] + bits[a] for a in range(self.d))), out)

    def _containing_leaf(self, r, lev, pos):
        """Leaf at level <= lev containing same-level block (r, lev, pos)."""
        l = lev
        while l >= 1:
            key = (r, l, tuple(p >> (lev - l) for p in pos))
            v = self.tree.get(key)
            if v is True:
                return key
            if v is False:
                return None  # region is refined at this level
            l -= 1
        return None

    def _refine_key(self, key):
        assert self.tree[key] is True
        r, lev, pos = key
        self.tree[key] = False
        for bits in all_corner_bits(self.d):
            self.tree[(r, lev + 1, tuple(2 * pos[a] + bits[a] for a in range(self.d)))] = True
        self._order = None

    def _violations(self):
        out = []
        for key in self.leaves():
            r, lev, pos = key
            for f in range(2 * self.d):
                nb = self.neighbour_coords(r, lev, pos, f)
                if nb is None:
                    continue
                r2, q, _, _ = nb
                if (r2, lev, q) in self.tree:
                    continue
                c = self._containing_leaf(r2, lev, q)
                if c is not None and c[1] < lev - 1:
                    out.append(c)
        return out

    def refine(self, keys):
        """Refine the given leaves, then close under 2:1 face balance."""
        for key in keys:
            if self.tree.get(key) is not True:
                raise ValueError(f"not a leaf: {key}")
        for key in keys:
            self._refine_key(key)
        while True:
            v = self._violations()
            if not v:
                break
            for key in sorted(set(v)):
                if self.tree.get(key) is True:
                    self._refine_key(key)

    def coarsen(self, parents):
        """Coarsen the given internal blocks whose 2^d children are leaves.
        Raises BalanceError (forest unchanged) if 2:1 balance would break."""
        d = self.d
        saved = dict(self.tree)
        try:
            for key in parents:
                r, lev, pos = key
                kids = [(r, lev + 1, tuple(2 * pos[a] + b[a] for a in range(d)))
                        for b in all_corner_bits(d)]
                if self.tree.get(key) is not False or any(self.tree.get(k) is not True for k in kids):
                    raise BalanceError(f"cannot coarsen {key}")
                for k in kids:
                    del self.tree[k]
                self.tree[key] = True
                self._order = None
            if self._violations():
                raise BalanceError("coarsening would break 2:1 balance")
        except BalanceError:
            self.tree = saved
            self._order = None
            raise

    # ---------------------------------------------------------------- tables
    def leaf_table(self):
        """Integer tables (root, level, pos, kind, nbr, orient) in leaf order."""
        d = self.d
        leaves = self.leaves()
        index = {k: i for i, k in enumerate(leaves)}
        nL = len(leaves)
        nf = 2 * d
        root = np.zeros(nL, np.int32)
        level = np.zeros(nL, np.int32)
        pos = np.zeros((nL, d), np.int32)
        kind = np.zeros((nL, nf), np.int32)
        nbr = -np.ones((nL, nf, 4), np.int64)
        orient = np.zeros((nL, nf), np.int32)
        for i, (r, lev, p) in enumerate(leaves):
            root[i], level[i], pos[i] = r, lev, p
            for f in range(nf):
                nb = self.neighbour_coords(r, lev, p, f)
                if nb is None:
                    kind[i, f] = BOUNDARY
                    continue
                r2, q, (pi, sigma), f2 = nb
                orient[i, f] = orient_code(pi, sigma)
                key = (r2, lev, q)
                v = self.tree.get(key)
                if v is True:
                    kind[i, f] = SAME
                    nbr[i, f, 0] = index[key]
                elif v is False:
                    kind[i, f] = FINER
                    a = f // 2
                    tang = [t for t in range(d) if t != a]
                    b2, s2 = divmod(f2, 2)
                    for sub in range(1 << (d - 1)):
                        cc = [0] * d
                        for j, t in enumerate(tang):
                            bit = (sub >> j) & 1
                            cc[pi[t]] = bit if sigma[t] > 0 else 1 - bit
                        cc[b2] = 0 if s2 == 0 else 1
                        ck = (r2, lev + 1, tuple(2 * q[u] + cc[u] for u in range(d)))
                        nbr[i, f, sub] = index[ck]
                else:
                    kind[i, f] = COARSER
                    ck = (r2, lev - 1, tuple(x >> 1 for x in q))
                    nbr[i, f, 0] = index[ck]
        return dict(root=root, level=level, pos=pos, kind=kind, nbr=nbr, orient=orient)

    # -------------------------------------------------------------- geometry
    def block_nodes(self, key):
        """(n+1)^d x d cell nodes of a tree node (root: given; child: Eq. (6)
        applied to the parent's cells at the half-cell points)."""
        if key in self._node_cache:
            return self._node_cache[key]
        d, n = self.d, self.n
        r, lev, pos = key
        if lev == 1:
            out = self.root_nodes[r]
        else:
            parent = (r, lev - 1, tuple(p >> 1 for p in pos))
            c = [p & 1 for p in pos]
            PX = self.block_nodes(parent)
            out = np.zeros(((n + 1) ** d, d))
            for li in range((n + 1) ** d):
                I = [(li // (n + 1) ** a) % (n + 1) for a in range(d)]
                H = [c[a] * n + I[a] for a in range(d)]
                Pc = [min(H[a] // 2, n - 1) for a in range(d)]
                xi = [float(H[a] - 2 * Pc[a] - 1) for a in range(d)]
                for bits in all_corner_bits(d):
                    wgt = 1.0
                    for a in range(d):
                        wgt *= 0.5 * (1.0 + (1.0 if bits[a] else -1.0) * xi[a])
                    if wgt == 0.0:
                        continue
                    J = [Pc[a] + bits[a] for a in range(d)]
                    out[li] += wgt * PX[sum(J[a] * (n + 1) ** a for a in range(d))]
        self._node_cache[key] = out
        return out

    def cell_corners(self, key):
        """(n^d, 2^d, d): corner positions of every cell, corner order bits."""
        d, n = self.d, self.n
        X = self.block_nodes(key)
        out = np.zeros((n ** d, 2 ** d, d))
        for c in range(n ** d):
            I = [(c // n ** a) % n for a in range(d)]
            for k, bits in enumerate(all_corner_bits(d)):
                out[c, k] = X[sum((I[a] + bits[a]) * (n + 1) ** a for a in range(d))]
        return out


def build(workload):
    """Forest from a ``workloads`` dict, with its refinement list applied."""
    f = Forest(workload["dim"], workload["n_seg"], workload["nodes"],
               workload["root_corners"], workload.get("root_cell_nodes"),
               workload.get("periodic", ()))
    for batch in workload.get("refine", []):
        f.refine([(r, lev, tuple(p)) for (r, lev, p) in batch])
    return f
