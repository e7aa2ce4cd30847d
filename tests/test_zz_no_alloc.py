"""The residual entry point that allocates nothing (dgf_dg_residual_noalloc).

Some callers cannot allocate device memory once a forest exists: code that
runs while a CUDA graph is being captured, or a process whose device memory
all comes from a pool it does not own.  For them the library keeps the
guard-trace scratch of the residual in a fixed 16 MiB device array compiled
into the library.  These tests call that entry point through the C ABI twice
in a row (on two different states, so stale scratch contents would show)
and check each result against dgf_dg_residual, the allocating entry point,
within the parity tolerance of the other GPU tests, in FP64 and FP32, with
the paper's level-jump scheme and the mortar repair (whose passes also write
into the scratch), in 3D and 2D.  They also check that the calls leave the
device's free memory unchanged, that a forest whose guard traces exceed the
array is refused, and that host pointers are refused before any launch.  The
file name makes pytest collect it after every other test file.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
DGF_EINVAL, DGF_EUNSUPPORTED = -1, -8


def _to_nodal(U, d, p):
    """Modal [leaf][var][mode][cell] -> values at the Gauss points."""
    N = p + 1
    x, _ = np.polynomial.legendre.leggauss(N)
    V = np.array([[np.polynomial.legendre.legval(xq, [0] * k + [1]) for k in range(N)] for xq in x])
    L, nv, M, nc = U.shape
    A = U.reshape((L, nv) + (N,) * d + (nc,))
    # mode index m = sum_a k_a N^a -> array axes are (k_{d-1}, ..., k_0)
    for ax in range(d):
        A = np.moveaxis(np.tensordot(V, A, axes=([1], [2 + (d - 1 - ax)])), 0, 2 + (d - 1 - ax))
    return A.reshape(L, nv, M, nc)


CASES = {
    "fp64-paper-3d": ("fp64", "paper", lambda: W.jitter3d_forest(seed=2, n_seg=4)),
    "fp32-paper-3d": ("fp32", "paper", lambda: W.jitter3d_forest(seed=2, n_seg=4)),
    "fp32-mortar-3d": ("fp32", "mortar", lambda: W.jitter3d_forest(seed=3, n_seg=4)),
    "fp64-mortar-2d": ("fp64", "mortar", lambda: W.rotated_pair_2d(n_seg=4)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_residual_matches_allocating_residual(case):
    import torch

    import paper_2502_12620_gb300 as pkg

    lib = pkg.lib()
    prec, mode, mk = CASES[case]
    w = mk()  # has finer, coarser and rotated faces
    p = 2
    f = pkg.Forest.from_workload(w, p=p, precision=pkg.FP64 if prec == "fp64" else pkg.FP32, nonconforming=mode)
    d = f.dim
    tdt = torch.float64 if prec == "fp64" else torch.float32
    out = torch.empty(f.state_shape, dtype=tdt, device="cuda")
    Un = torch.empty(f.state_shape, dtype=tdt, device="cuda")
    free = []
    for seed in (5, 6):
        U = W.random_modal_state(f.n_leaves, d, f.n_seg, p, seed=seed).astype(f.dtype)
        f.set_state(U)
        ref = _to_nodal(f.dg_residual().astype(np.float64), d, p)
        Un.copy_(torch.from_numpy(_to_nodal(U.astype(np.float64), d, p)).to(tdt))
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        code = lib.dgf_dg_residual_noalloc(f.h, ctypes.c_void_p(Un.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert code == 0, lib.dgf_last_error().decode()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got = out.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < TOL[prec], err
    # the calls made no device allocation (the second pair follows a warm call)
    assert free[2] == free[3], free
    f.close()


def test_noalloc_refuses_forests_beyond_the_scratch_size():
    """125 leaves of 8^3 cells at p = 3 in FP64 need 30 MiB of guard traces."""
    import torch

    import paper_2502_12620_gb300 as pkg

    lib = pkg.lib()
    f = pkg.Forest.from_workload(W.periodic_cube_forest(5), p=3, precision=pkg.FP64)
    a = torch.zeros(f.state_shape, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    code = lib.dgf_dg_residual_noalloc(f.h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()))
    assert code == DGF_EUNSUPPORTED
    assert "16 MiB" in lib.dgf_last_error().decode()
    f.close()


def test_noalloc_refuses_host_pointers():
    """Host buffers would reach the kernels and fault there: refused first."""
    import torch

    import paper_2502_12620_gb300 as pkg

    lib = pkg.lib()
    f = pkg.Forest.from_workload(W.jitter3d_forest(seed=2, n_seg=2), p=1, precision=pkg.FP64)
    h = np.zeros(int(np.prod(f.state_shape)) + 2, np.float64)
    off = (-h.ctypes.data % 16) // 8
    hp = ctypes.c_void_p(h.ctypes.data + 8 * off)
    d = torch.zeros(f.state_shape, dtype=torch.float64, device="cuda")
    dp = ctypes.c_void_p(d.data_ptr())
    assert lib.dgf_dg_residual_noalloc(f.h, hp, dp) == DGF_EINVAL
    assert lib.dgf_dg_residual_noalloc(f.h, dp, hp) == DGF_EINVAL
    assert "device memory" in lib.dgf_last_error().decode()
    f.close()
