"""Python binding of libdgf.so, the GB300 block-forest DG library (C ABI in include/dgf.h).

Argument marshalling only: every step of the DG path (guard fill, residual,
inverse mass, SSP-RK3 stage combination, CFL minimum, totals) runs in the
library's CUDA kernels.  Device memory comes from PyTorch's caching
allocator through the library's allocator hook; there is no CPU fallback:
if the shared library is missing, importing the binding's entry points
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgf.so")

FP64, FP32, FP32_COMP = 0, 1, 2
NC_PAPER, NC_MORTAR = 0, 1  # fluxes across level jumps (include/dgf.h)
SAME, COARSER, FINER, BOUNDARY = 0, 1, 2, 3
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE",
          -5: "ETIMEOUT", -6: "EBALANCE", -7: "ESTATE", -8: "EUNSUPPORTED"}


class DgfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_seg", ctypes.c_int32), ("p", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("n_periodic", ctypes.c_int32), ("nonconforming", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("cfl", ctypes.c_double), ("periodic", ctypes.c_double * 9),
                ("n_nodes", ctypes.c_int64), ("nodes", ctypes.POINTER(ctypes.c_double)),
                ("n_roots", ctypes.c_int64), ("root_corners", ctypes.POINTER(ctypes.c_int64)),
                ("root_cell_nodes", ctypes.POINTER(ctypes.c_double))]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN)]


_lib = None

# (name, argtypes) of every entry point declared in include/dgf.h
_P = ctypes.c_void_p
_SIGS = {
    "dgf_forest_create": [ctypes.POINTER(_Desc), ctypes.POINTER(_Allocator), ctypes.POINTER(_P)],
    "dgf_forest_destroy": [_P],
    "dgf_set_stream": [_P, _P],
    "dgf_block_refine": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64],
    "dgf_block_coarsen": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64],
    "dgf_leaf_count": [_P, ctypes.POINTER(ctypes.c_int64)],
    "dgf_leaf_table": [_P, _P, _P, _P, _P, _P, _P],
    "dgf_quad_points": [_P, _P],
    "dgf_state_size": [_P, ctypes.POINTER(ctypes.c_int64)],
    "dgf_set_state": [_P, _P, ctypes.c_int],
    "dgf_get_state": [_P, _P, ctypes.c_int],
    "dgf_set_state_nodal": [_P, _P, ctypes.c_int],
    "dgf_fill_guardcells": [_P, _P, ctypes.c_int],
    "dgf_dg_residual": [_P, _P, ctypes.c_int],
    "dgf_rk_step": [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
    "dgf_get_time": [_P, ctypes.POINTER(ctypes.c_double)],
    "dgf_indicator": [_P, ctypes.POINTER(ctypes.c_double)],
    "dgf_set_boundary": [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)],
    "dgf_set_limiter": [_P, ctypes.c_double],
    "dgf_limit": [_P],
    "dgf_adapt": [_P, ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                  ctypes.POINTER(ctypes.c_int64)],
    "dgf_adapt_with": [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "dgf_step_count": [_P, ctypes.POINTER(ctypes.c_int64)],
    "dgf_set_time": [_P, ctypes.c_double],
    "dgf_compute_dt": [_P, ctypes.POINTER(ctypes.c_double)],
    "dgf_conserved_totals": [_P, _P],
    "dgf_status_word": [_P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int],
    "dgf_set_timing": [_P, ctypes.c_int],
    "dgf_tuning": [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "dgf_stage_kernel": [_P, ctypes.POINTER(ctypes.c_int32)],
    "dgf_stage_grid": [_P, ctypes.POINTER(ctypes.c_int32)],
    "dgf_kernel_times": [_P, _P, _P, ctypes.c_int],
    "dgf_dg_residual_noalloc": [_P, _P, _P],
    "dgf_batch_create": [ctypes.c_int32, _P, ctypes.POINTER(_P)],
    "dgf_batch_destroy": [_P],
    "dgf_batch_set": [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_double), ctypes.c_int32],
    "dgf_batch_step": [_P, ctypes.c_int32],
    "dgf_batch_sync": [_P],
    "dgf_batch_query": [_P, ctypes.POINTER(ctypes.c_int32)],
    "dgf_batch_progress": [_P, _P, _P, _P],
}


def lib():
    """Load libdgf.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdgf.so not built at {LIB_PATH}; run "
                              "python -m paper_2502_12620_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int32
        L.dgf_last_error.argtypes = []
        L.dgf_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(code):
    if code != 0:
        raise DgfError(code, lib().dgf_last_error().decode())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


_LIB_STREAMS = {}
_LIB_STREAMS_LOCK = __import__("threading").Lock()


def library_stream(device=0):
    """The stream the library's device memory is drawn on from torch's
    caching allocator.  Nothing runs on it: torch hands a freed block to a
    new allocation of the same stream at once, even while kernels queued
    there may still touch it, and the library uses its memory on its own
    streams, which torch does not order against.  Drawing on a stream of
    its own keeps the library's blocks apart from every tensor's; the
    library synchronises its stream before it frees a block."""
    import torch
    with _LIB_STREAMS_LOCK:
        s = _LIB_STREAMS.get(device)
        if s is None:
            s = _LIB_STREAMS[device] = torch.cuda.Stream(device=device)
    return s


def reserve_memory(nbytes, device=0):
    """Grow torch's cached pool of the library's stream by nbytes (allocated
    and released at once), so that later forest allocations are served from
    it without new device allocations."""
    import torch
    with torch.cuda.stream(library_stream(device)):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device=torch.device("cuda", device))
        del t


class _TorchAllocator:
    """Device memory for the library from torch's caching allocator, on the
    library's own stream (library_stream)."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        lib_stream = library_stream(device)

        def _alloc(ctx, nbytes, stream):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), device, lib_stream)
            except Exception:
                return None
            self.live[p] = nbytes
            return p

        def _free(ctx, ptr, nbytes, stream):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self._a = _ALLOC_FN(_alloc)
        self._f = _FREE_FN(_free)
        self.struct = _Allocator(None, self._a, self._f)


class Forest:
    """A block forest with its DG state on one GPU (or host-only, device=-1)."""

    def __init__(self, dim, n_seg, p, nodes, root_corners, root_cell_nodes=None, periodic=(),
                 precision=FP64, device=0, gamma=1.4, cfl=0.1, torch_memory=True, nonconforming="paper"):
        L = lib()
        self.dim, self.n_seg, self.p = int(dim), int(n_seg), int(p)
        self.precision = (FP32 if precision in (FP32, "fp32", "f32") else
                          FP32_COMP if precision in (FP32_COMP, "fp32_comp") else FP64)
        self.device = int(device)
        self.nv = self.dim + 2
        self.N = self.p + 1
        self.M = self.N ** self.dim
        self.nc = self.n_seg ** self.dim
        self.nt = self.n_seg ** (self.dim - 1)
        self.dtype = np.float32 if self.precision == FP32 else np.float64  # ABI element type
        nodes = np.ascontiguousarray(nodes, np.float64)
        corners = np.ascontiguousarray(root_corners, np.int64)
        cell = None if root_cell_nodes is None else np.ascontiguousarray(root_cell_nodes, np.float64)
        d = _Desc()
        d.dim, d.n_seg, d.p, d.precision, d.device = self.dim, self.n_seg, self.p, self.precision, self.device
        per = list(periodic)
        d.n_periodic = len(per)
        for i, t in enumerate(per):
            for j in range(self.dim):
                d.periodic[i * self.dim + j] = float(t[j])
        if nonconforming not in ("paper", "mortar"):
            raise ValueError("nonconforming must be 'paper' or 'mortar'")
        self.nonconforming = nonconforming
        d.nonconforming = NC_MORTAR if nonconforming == "mortar" else NC_PAPER
        d.gamma, d.cfl = float(gamma), float(cfl)
        d.n_nodes = nodes.shape[0]
        d.nodes = nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_roots = corners.shape[0]
        d.root_corners = corners.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.root_cell_nodes = (cell.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                             if cell is not None else ctypes.POINTER(ctypes.c_double)())
        self._alloc = None
        aptr = None
        if self.device >= 0 and torch_memory:
            self._alloc = _TorchAllocator(self.device)
            aptr = ctypes.byref(self._alloc.struct)
        h = ctypes.c_void_p()
        _check(L.dgf_forest_create(ctypes.byref(d), aptr, ctypes.byref(h)))
        self.h = h

    @classmethod
    def from_workload(cls, w, p=None, precision=FP64, device=0, cfl=None, **kw):
        f = cls(w["dim"], w["n_seg"], w.get("p", 2) if p is None else p, w["nodes"],
                w["root_corners"], w.get("root_cell_nodes"), w.get("periodic", ()),
                precision=precision, device=device,
                cfl=w.get("cfl", 0.1) if cfl is None else cfl, **kw)
        for batch in w.get("refine", []):
            T = f.leaf_table()
            index = {(int(T["root"][i]), int(T["level"][i]), tuple(int(x) for x in T["pos"][i])): i
                     for i in range(len(T["root"]))}
            f.refine([index[(r, lev, tuple(pos))] for (r, lev, pos) in batch])
        return f

    def set_stream(self, stream):
        """Run this forest's GPU work on a torch.cuda.Stream (or raw handle)."""
        h = getattr(stream, "cuda_stream", stream)
        _check(lib().dgf_set_stream(self.h, ctypes.c_void_p(int(h))))
        self._stream = stream

    # ------------------------------------------------------------ topology
    def close(self):
        if getattr(self, "h", None):
            lib().dgf_forest_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    @property
    def device_bytes(self):
        """Device bytes the library holds for this forest (0 when it allocates
        through CUDA directly)."""
        return sum(self._alloc.live.values()) if self._alloc is not None else 0

    @property
    def n_leaves(self):
        n = ctypes.c_int64()
        _check(lib().dgf_leaf_count(self.h, ctypes.byref(n)))
        return n.value

    def leaf_table(self):
        L, d = self.n_leaves, self.dim
        nf = 2 * d
        out = dict(root=np.zeros(L, np.int32), level=np.zeros(L, np.int32),
                   pos=np.zeros((L, d), np.int32), kind=np.zeros((L, nf), np.int32),
                   nbr=np.zeros((L, nf, 4), np.int64), orient=np.zeros((L, nf), np.int32))
        _check(lib().dgf_leaf_table(self.h, *[_ptr(out[k]) for k in
                                               ("root", "level", "pos", "kind", "nbr", "orient")]))
        return out

    def refine(self, leaf_ids):
        ids = np.ascontiguousarray(leaf_ids, np.int64)
        _check(lib().dgf_block_refine(self.h, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(ids)))

    def coarsen(self, leaf_ids):
        ids = np.ascontiguousarray(leaf_ids, np.int64)
        _check(lib().dgf_block_coarsen(self.h, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(ids)))

    def set_boundary(self, root_face_kind, state):
        """Root faces without a neighbour: 0 outflow, 1 prescribed state
        (root_face_kind: [roots][2 dim]); state: nv conserved values."""
        tags = np.ascontiguousarray(root_face_kind, np.int32)
        st = np.ascontiguousarray(state, np.float64)
        assert st.shape == (self.nv,)
        _check(lib().dgf_set_boundary(self.h, tags.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      st.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def indicator(self):
        """Refinement indicator per leaf (see dgf_indicator)."""
        out = np.zeros(self.n_leaves)
        _check(lib().dgf_indicator(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def adapt(self, refine_above, coarsen_below, max_level, indicator=None):
        """One adaptation step (indicator: per-leaf values, default the
        device's own); returns (leaves refined by the threshold, parents
        coarsened)."""
        nr, nc = ctypes.c_int64(), ctypes.c_int64()
        if indicator is None:
            _check(lib().dgf_adapt(self.h, float(refine_above), float(coarsen_below), int(max_level),
                                   ctypes.byref(nr), ctypes.byref(nc)))
        else:
            g = np.ascontiguousarray(indicator, np.float64)
            assert g.shape == (self.n_leaves,)
            _check(lib().dgf_adapt_with(self.h, g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        float(refine_above), float(coarsen_below), int(max_level),
                                        ctypes.byref(nr), ctypes.byref(nc)))
        return nr.value, nc.value

    def quad_points(self):
        out = np.zeros((self.n_leaves, self.nc, self.M, self.dim))
        _check(lib().dgf_quad_points(self.h, _ptr(out)))
        return out

    # --------------------------------------------------------------- state
    @property
    def state_shape(self):
        return (self.n_leaves, self.nv, self.M, self.nc)

    def _is_torch(self, x):
        return type(x).__module__.startswith("torch")

    def set_state(self, U):
        if self._is_torch(U):
            assert U.is_cuda and U.is_contiguous() and U.numel() == int(np.prod(self.state_shape))
            import torch
            torch.cuda.current_stream().synchronize()
            _check(lib().dgf_set_state(self.h, ctypes.c_void_p(U.data_ptr()), 1))
        else:
            a = np.ascontiguousarray(U, self.dtype).reshape(self.state_shape)
            _check(lib().dgf_set_state(self.h, _ptr(a), 0))

    def get_state(self, out=None):
        if out is not None and self._is_torch(out):
            _check(lib().dgf_get_state(self.h, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        a = np.empty(self.state_shape, self.dtype) if out is None else out
        _check(lib().dgf_get_state(self.h, _ptr(a), 0))
        return a

    def set_state_nodal(self, vals):
        """Point values [leaf][cell][point][var] in FP64 (numpy, or a CUDA tensor)."""
        if self._is_torch(vals):
            import torch
            assert vals.is_cuda and vals.is_contiguous() and vals.dtype == torch.float64
            assert vals.numel() == self.n_leaves * self.nc * self.M * self.nv
            torch.cuda.current_stream().synchronize()
            _check(lib().dgf_set_state_nodal(self.h, ctypes.c_void_p(vals.data_ptr()), 1))
            return
        v = np.ascontiguousarray(vals, np.float64).reshape(self.n_leaves, self.nc, self.M, self.nv)
        _check(lib().dgf_set_state_nodal(self.h, _ptr(v), 0))

    def project(self, fun):
        """Set the state to the (p+1)-point projection of fun(x[..., d])."""
        self.set_state_nodal(fun(self.quad_points()))

    def fill_guardcells(self):
        G = np.empty((self.n_leaves, 2 * self.dim, self.nv, self.M, self.nt), self.dtype)
        _check(lib().dgf_fill_guardcells(self.h, _ptr(G), 0))
        return G

    def dg_residual(self):
        R = np.empty(self.state_shape, self.dtype)
        _check(lib().dgf_dg_residual(self.h, _ptr(R), 0))
        return R

    # ---------------------------------------------------------- time march
    def rk_step(self, t_end=float("inf"), return_dt=False):
        if return_dt:
            dt = ctypes.c_double()
            _check(lib().dgf_rk_step(self.h, float(t_end), ctypes.byref(dt)))
            return dt.value
        _check(lib().dgf_rk_step(self.h, float(t_end), None))
        return None

    def run(self, steps, t_end=float("inf")):
        for _ in range(steps):
            self.rk_step(t_end)
        return self.time

    @property
    def time(self):
        t = ctypes.c_double()
        _check(lib().dgf_get_time(self.h, ctypes.byref(t)))
        return t.value

    @property
    def step_count(self):
        """Time increments taken with dt > 0 since creation / set_time."""
        n = ctypes.c_int64()
        _check(lib().dgf_step_count(self.h, ctypes.byref(n)))
        return n.value

    def set_time(self, t):
        _check(lib().dgf_set_time(self.h, float(t)))

    def compute_dt(self):
        dt = ctypes.c_double()
        _check(lib().dgf_compute_dt(self.h, ctypes.byref(dt)))
        return dt.value

    def conserved_totals(self):
        T = np.zeros(self.nv)
        _check(lib().dgf_conserved_totals(self.h, _ptr(T)))
        return T

    def set_limiter(self, eps):
        """Positivity limiter after every RK stage (eps > 0), or off (0)."""
        _check(lib().dgf_set_limiter(self.h, float(eps)))

    def limit(self):
        """Apply the positivity limiter to the current state once."""
        _check(lib().dgf_limit(self.h))

    def status_word(self, reset=False):
        s = ctypes.c_int32()
        _check(lib().dgf_status_word(self.h, ctypes.byref(s), int(reset)))
        return s.value

    def tuning(self):
        z = ctypes.c_int32()
        c = ctypes.c_int32()
        _check(lib().dgf_tuning(self.h, ctypes.byref(z), ctypes.byref(c)))
        k = ctypes.c_int32()
        _check(lib().dgf_stage_kernel(self.h, ctypes.byref(k)))
        g = ctypes.c_int32()
        _check(lib().dgf_stage_grid(self.h, ctypes.byref(g)))
        return {"zchunk": z.value, "resident_ctas": c.value, "stage_kernel": ("pair", "classic", "pair5")[k.value],
                "stage_grid": ("persistent", "items")[g.value]}

    def set_timing(self, on):
        _check(lib().dgf_set_timing(self.h, int(on)))

    def kernel_times(self):
        ms = np.zeros(3)
        cnt = np.zeros(3, np.int64)
        _check(lib().dgf_kernel_times(self.h, _ptr(ms), _ptr(cnt), 3))
        return {"dt": (ms[0], int(cnt[0])), "guard": (ms[1], int(cnt[1])), "stage": (ms[2], int(cnt[2]))}


class Batch:
    """Forests advanced together: one launch of each kernel per stage for
    all members (3D FP32 forests of 8^3-cell blocks, one degree, plain form).
    Each member keeps its own time, end time and time increment."""

    def __init__(self, device=0, stream=None):
        self.device = int(device)
        h = _P()
        raw = None if stream is None else ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
        _check(lib().dgf_batch_create(self.device, raw, ctypes.byref(h)))
        self.h = h
        self.members = []

    def set(self, forests, t_ends):
        """Replace the members; t_ends[i] is member i's end time."""
        n = len(forests)
        hs = (_P * max(1, n))(*[f.h for f in forests])
        te = (ctypes.c_double * max(1, n))(*[float(t) for t in t_ends])
        _check(lib().dgf_batch_set(self.h, hs, te, n))
        self.members = list(forests)

    def step(self, steps=1):
        _check(lib().dgf_batch_step(self.h, int(steps)))

    def sync(self):
        _check(lib().dgf_batch_sync(self.h))

    def idle(self):
        v = ctypes.c_int32()
        _check(lib().dgf_batch_query(self.h, ctypes.byref(v)))
        return bool(v.value)

    def progress(self):
        """(time, steps, status) arrays of the members, in member order."""
        n = len(self.members)
        t = np.zeros(n)
        st = np.zeros(n, np.int64)
        ss = np.zeros(n, np.int32)
        if n:
            _check(lib().dgf_batch_progress(self.h, _ptr(t), _ptr(st), _ptr(ss)))
        return t, st, ss

    def close(self):
        if getattr(self, "h", None):
            lib().dgf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Forest", "Batch", "DgfError", "lib", "FP64", "FP32", "FP32_COMP", "NC_PAPER", "NC_MORTAR", "LIB_PATH"]
