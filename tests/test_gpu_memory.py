"""The library's device memory and torch tensors on other streams.

Torch's caching allocator hands a released block to the next allocation of
the same stream at once, while kernels queued on that stream may still write
it; the library uses its memory on its own streams, which torch does not
order against that queued work.  The binding therefore draws the library's
memory on a stream of its own.  Here tensors of the sizes of a forest's
buffers are released while a fill of them is still queued (behind a bounded
sleep) on the current stream, a forest is built at once and stepped after the
fill has run: its result must be the one of a forest built with nothing
pending.  Whether a shared pool would hand the forest those very blocks
depends on the allocator's choices, so the test sets up the conditions of
the hazard rather than forcing it; it guards the separation of the pools."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dgf():
    import paper_2502_12620_gb300 as pkg
    pkg.lib()
    return pkg


def _run(dgf, w, pause=0.0):
    f = dgf.Forest.from_workload(w, p=1, precision=dgf.FP32, cfl=0.2)
    f.project(lambda x: W.smooth_state(x))
    time.sleep(pause)
    for _ in range(3):
        f.rk_step()
    U = f.get_state()
    assert f.status_word() == 0
    f.close()
    return U


def test_forest_memory_is_never_a_block_with_queued_torch_work(dgf):
    import torch
    w = W.periodic_cube_forest(4)  # 64 blocks at p = 1: 5.2 MB a state copy
    ref = _run(dgf, w)
    torch.cuda.synchronize()
    L, nv, M, nc = 64, 5, 8, 512
    sizes = ([L * nv * M * nc * 4] * 3 + [L * 21 * nc * 8, L * 21 * nc * 4, L * 6 * nv * 4 * 64 * 4,
                                          L * nc * nv * 8, L * nc * 8, L * nc * 4])
    ts = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
    torch.cuda._sleep(int(1e9))  # about 0.5 s of the current stream
    for t in ts:
        t.fill_(255)  # NaN bit patterns, written after the sleep
    del ts, t
    # built now, stepped after the fill has run
    U = _run(dgf, w, pause=1.5)
    torch.cuda.synchronize()
    assert np.array_equal(U, ref)
