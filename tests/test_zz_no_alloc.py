"""The allocation-free cell sort (usp_cell_sort_static) against the counting
sort of a simulation handle.

Callers that cannot allocate device memory where they need the sort (host
callbacks, plug-ins whose host owns all device memory) get the histogram and
cursor scratch from a fixed device array instead.  This file is collected
last so that a failure here cannot hide another test's result; it passes on
its own in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_cell_sort_matches_handle_sort_twice():
    import torch
    assert torch.cuda.is_available()
    from paper_1808_03801_gb300 import usp as U
    from paper_1808_03801_gb300 import workloads as W
    L = U.lib()
    nc, n = 24, 20000
    K = nc * nc
    w = W.cavity(n=nc, ppc=30, Kn=0.05, precision="fp64")
    w["params"]["dt"] = 1e-30          # advection leaves every position as it is
    rng = np.random.default_rng(5)
    pos = np.column_stack([rng.uniform(0, 1e-4, n), rng.uniform(0, 1e-4, n)])
    vel = rng.normal(0, 300, (n, 3))
    pid = np.arange(n, dtype=np.uint32)

    # existing entry point: the handle's advection and counting-sort stages
    h = U.Simulation(w).set_particles(pos, vel, pid)
    for k in (0, 1, 2):
        h.run_stage(k)
    P = h.particles()
    o = np.argsort(P["pid"])
    assert np.array_equal(P["pos"][o], pos)
    cell_ref = np.empty(n, dtype=np.int64)
    cell_ref[P["pid"]] = P["cell"]
    start_ref = np.concatenate([[0], np.cumsum(np.bincount(P["cell"], minlength=K))])

    grid = U.Grid(2, nc, nc, (ctypes.c_double * 2)(0.0, 0.0), (ctypes.c_double * 2)(1e-4, 1e-4))
    dpos = torch.tensor(pos, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        start = torch.full((K + 1,), -1, dtype=torch.int32, device="cuda")
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = L.usp_cell_sort_static(ctypes.byref(grid), n, dpos.data_ptr(), start.data_ptr(), perm.data_ptr(),
                                    stream.cuda_stream)
        torch.cuda.synchronize()
        assert rc == 0, rc
        s = start.cpu().numpy().view(np.uint32).astype(np.int64)
        p = perm.cpu().numpy().view(np.uint32).astype(np.int64)
        assert np.array_equal(s, start_ref), call
        assert np.array_equal(np.sort(p), np.arange(n))
        cell_static = np.empty(n, dtype=np.int64)
        cell_static[p] = np.repeat(np.arange(K), np.diff(s))
        assert np.array_equal(cell_static, cell_ref), call

    too_big = U.Grid(2, 1024, 1024, (ctypes.c_double * 2)(0.0, 0.0), (ctypes.c_double * 2)(1.0, 1.0))
    assert L.usp_cell_sort_static(ctypes.byref(too_big), 0, None, start.data_ptr(), None, None) == -4


def test_static_cell_sort_one_dimensional_grid():
    """1-D grids use y alone (x ignored): cells floor((y - lo) / dy) clamped to
    the grid, as the handle's FP64 sort assigns them; two calls in a row."""
    import torch
    from paper_1808_03801_gb300 import usp as U
    from paper_1808_03801_gb300 import workloads as W
    L = U.lib()
    ny, n = 37, 15000
    w = W.couette(ny=ny, ppc=20, precision="fp64")
    w["params"]["dt"] = 1e-30
    H = w["grid"]["hi"][1]
    rng = np.random.default_rng(9)
    pos = np.column_stack([rng.uniform(-5.0, 5.0, n), rng.uniform(0, H, n)])
    pos[:5, 1] = [0.0, H, H * (1 - 1e-15), 0.5 * H, 1e-300]
    vel = rng.normal(0, 300, (n, 3))
    h = U.Simulation(w).set_particles(pos, vel, np.arange(n, dtype=np.uint32))
    for k in (0, 1, 2):
        h.run_stage(k)
    P = h.particles()
    cell_ref = np.empty(n, dtype=np.int64)
    cell_ref[P["pid"]] = P["cell"]
    start_ref = np.concatenate([[0], np.cumsum(np.bincount(P["cell"], minlength=ny))])
    grid = U.Grid(1, 0, ny, (ctypes.c_double * 2)(0.0, 0.0), (ctypes.c_double * 2)(1.0, H))
    dpos = torch.tensor(pos, dtype=torch.float64, device="cuda")
    for call in range(2):
        start = torch.full((ny + 1,), -1, dtype=torch.int32, device="cuda")
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = L.usp_cell_sort_static(ctypes.byref(grid), n, dpos.data_ptr(), start.data_ptr(), perm.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rc == 0, rc
        s = start.cpu().numpy().view(np.uint32).astype(np.int64)
        p = perm.cpu().numpy().view(np.uint32).astype(np.int64)
        assert np.array_equal(s, start_ref), call
        cell_static = np.empty(n, dtype=np.int64)
        cell_static[p] = np.repeat(np.arange(ny), np.diff(s))
        assert np.array_equal(cell_static, cell_ref), call
