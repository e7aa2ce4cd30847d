"""The residual entry point that allocates nothing (dgf_dg_residual_noalloc).

Some callers cannot allocate device memory once a forest exists: code that
runs while a CUDA graph is being captured, or a process whose device memory
all comes from a pool it does not own.  For them the library keeps the
guard-trace scratch of the residual in a fixed 16 MiB device array compiled
into the library.  This test calls that entry point through the C ABI twice
in a row (on two different states, so stale scratch contents would show)
and checks each result against dgf_dg_residual, the allocating entry point,
within the FP64 parity tolerance of the other GPU tests.  The file name makes
pytest collect it after every other test file.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def test_noalloc_residual_matches_allocating_residual():
    import torch

    import paper_2502_12620_gb300 as pkg

    lib = pkg.lib()
    w = W.jitter3d_forest(seed=2, n_seg=4)  # has finer, coarser and rotated faces
    f = pkg.Forest.from_workload(w, p=2, precision=pkg.FP64)
    out = torch.empty(f.state_shape, dtype=torch.float64, device="cuda")
    for seed in (5, 6):
        U = W.random_modal_state(f.n_leaves, 3, 4, 2, seed=seed)
        f.set_state(U)
        ref = _to_nodal(f.dg_residual().astype(np.float64), 3, 2)
        Un = torch.from_numpy(_to_nodal(U, 3, 2)).cuda()
        out.fill_(np.nan)
        torch.cuda.synchronize()
        code = lib.dgf_dg_residual_noalloc(f.h, ctypes.c_void_p(Un.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert code == 0, lib.dgf_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < TOL, err
    f.close()
