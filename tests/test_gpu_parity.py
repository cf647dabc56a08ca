"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.

FP64 mode: integer work (particle sets, cell ids, counts) bit-exact, every
particle's position and velocity within 1e-12 relative (scale sqrt(R T_ref)
for velocities, the cell size for positions), fields within 1e-10.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1808_03801_gb300 import workloads as W
from tests._util import KB_M_AR, assert_particles_close, by_pid

pytestmark = pytest.mark.gpu

VSCALE = math.sqrt(KB_M_AR * W.T0)


@pytest.fixture(scope="module")
def usp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1808_03801_gb300 import usp as U
    U.lib()
    return U


def _pair(w, usp, init=True):
    g = usp.Simulation(w)
    o = oracle.OracleSim(w)
    if init:
        g.init_particles()
        o.init_particles()
    return g, o


def _cell_size(w):
    gr = w["grid"]
    return (gr["hi"][1] - gr["lo"][1]) / gr["ny"]


def test_philox_bit_exact(usp):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, size=(20000, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x1234ABCD, 0x0BADF00D)
    got = usp.debug_philox(ctr, key)
    want = np.array([oracle.philox(c, key) for c in ctr[:2000]])
    assert np.array_equal(got[:2000], want)


def test_init_matches_oracle(usp):
    w = W.cavity(n=12, ppc=40, Kn=0.05, precision="fp64", steps=1)
    w["regions"].append({"lo": (0.0, 0.0), "hi": (0.5e-4, 0.5e-4), "n": W.N0 * 0.5, "T": 350.0,
                         "u": (20.0, 0.0, -5.0)})
    g, o = _pair(w, usp)
    assert_particles_close(g.particles(), o.particles(), VSCALE, 1e-4 / 12, rtol=1e-14)


def test_dt_and_viscosity_derivation(usp):
    w = W.couette(ny=10, ppc=10)
    g, o = _pair(w, usp, init=False)
    inf = g.info()
    assert math.isclose(inf["dt"], o.dt, rel_tol=1e-14)
    assert math.isclose(inf["mu_ref"], o.mu_ref, rel_tol=1e-14)


@pytest.mark.parametrize("name,steps", [("couette", 20), ("cavity", 12), ("sod", 15), ("slit", 10),
                                        ("poiseuille", 15)])
def test_fp64_step_parity(usp, name, steps):
    if name == "couette":
        w = W.couette(ny=100, ppc=100, precision="fp64")
    elif name == "cavity":
        w = W.cavity(n=24, ppc=30, Kn=0.01, precision="fp64")
    elif name == "sod":
        w = W.sod(ny=200, ppc_left=80, precision="fp64")
    elif name == "slit":
        w = W.slit(nx=40, ny=20, ppc=30, precision="fp64")
    else:
        w = W.poiseuille(ny=50, ppc=60, precision="fp64")
    g, o = _pair(w, usp)
    g.step(steps)
    o.step(steps)
    assert_particles_close(g.particles(), o.particles(), VSCALE, _cell_size(w))
    fg, fo = g.sample(), o.fields()
    assert np.array_equal(fg[15], fo[15])        # particles per cell
    scale = np.maximum(np.abs(fo), np.abs(fo).max(axis=1, keepdims=True) * 1e-3)
    assert np.all(np.abs(fg - fo) <= 1e-10 * scale + 1e-300)
    fa, oa = g.sample(averaged=True), o.fields(averaged=True)
    assert np.all(np.abs(fa - oa) <= 1e-10 * np.maximum(np.abs(oa), np.abs(oa).max(1, keepdims=True) * 1e-3))
    pg, po = g.params(), o.params()
    assert np.array_equal(pg[:, 14], po[:, 14])   # valid cells
    assert np.array_equal(pg[:, 15], po[:, 15])   # relaxed counts (integer decisions)
    sel = po[:, 14] > 0
    assert np.allclose(pg[sel, 4:14], po[sel, 4:14], rtol=1e-10, atol=1e-12 * VSCALE)
    if name == "slit":
        ig = g.info()
        assert ig["n_particles"] == o.n
        assert ig["counters"][2] == o.counters()[2] and ig["counters"][3] == o.counters()[3]
        assert ig["counters"][7] == o.counters()[4]


def test_stagewise_sort_parity(usp):
    """After advection and the counting sort, cell ids and counts are bit-exact
    and the storage is grouped by cell."""
    w = W.cavity(n=16, ppc=25, Kn=0.02, precision="fp64")
    g, o = _pair(w, usp)
    g.step(3)
    o.step(3)
    for k in (0, 1, 2):
        g.run_stage(k)
    for ph in (oracle.PH_STREAM, oracle.PH_RESERVOIR, oracle.PH_SORT):
        o.phase(ph)
    P = g.particles()
    assert np.all(np.diff(P["cell"]) >= 0)
    assert np.array_equal(np.bincount(P["cell"], minlength=256), o.counts())
    assert_particles_close(P, o.particles(), VSCALE, 1e-4 / 16)
    for k in (3, 4, 5, 6):
        g.run_stage(k)
    for ph in (oracle.PH_MOMENTS, oracle.PH_PARAMS, oracle.PH_RELAX, oracle.PH_SAMPLE):
        o.phase(ph)
    assert_particles_close(g.particles(), o.particles(), VSCALE, 1e-4 / 16)


@pytest.mark.parametrize("mode", ["usp", "sp", "fixed"])
def test_homogeneous_modes(usp, mode):
    n = 20000
    w = W.homogeneous_box(ppc=n, dt_over_tauc=3.0, mode=mode, fixed_pne=0.4)
    pos, vel, pid = W.bimaxwellian(n, seed=3, heat_skew=0.5)
    g = usp.Simulation(w).set_particles(pos, vel, pid)
    o = oracle.OracleSim(w).set_particles(pos, vel, pid)
    g.step(4)
    o.step(4)
    assert_particles_close(g.particles(), o.particles(), VSCALE, 1e-6)


def test_edge_cases_empty_and_sparse_cells(usp):
    """Empty cells, cells with one to a few particles and an empty domain.

    With two or three particles in a cell the sample stress can put almost all
    thermal energy on one axis, which makes RT I + (1 - 1/Pr) sigma*/rho nearly
    singular; its Cholesky factor then amplifies rounding-order differences
    (one-pass shifted sums on the GPU, two-pass sums in the oracle) by the
    condition number, so this sparse case is held to 1e-9 instead of 1e-12.
    Integer work stays bit-exact."""
    w = W.cavity(n=10, ppc=3, Kn=0.05, precision="fp64")
    w["regions"] = [{"lo": (0.0, 0.0), "hi": (0.5e-4, 1e-4), "n": W.N0, "T": W.T0, "u": (0, 0, 0)}]
    g, o = _pair(w, usp)
    g.step(6)
    o.step(6)
    assert_particles_close(g.particles(), o.particles(), VSCALE, 1e-5, rtol=1e-9)
    assert np.array_equal(g.params()[:, 15], o.params()[:, 15])
    assert np.array_equal(g.sample()[15], o.fields()[15])
    w2 = W.couette(ny=8, ppc=10)
    w2["regions"] = []
    g2 = usp.Simulation(w2).init_particles()
    g2.step(3)
    assert g2.info()["n_particles"] == 0


def test_capacity_and_argument_errors(usp):
    w = W.couette(ny=10, ppc=10)
    bad = dict(w, params=dict(w["params"], ppc_ref=0))
    with pytest.raises(usp.UspError) as e:
        usp.Simulation(bad)
    assert e.value.status == -1
    g = usp.Simulation(w)
    with pytest.raises(usp.UspError) as e:
        g.step(1)
    assert e.value.status == -6   # not initialised


def test_batch_fp64_matches_alone_per_particle(usp):
    """A simulation stepped inside a batch with uneven neighbours gives the same
    particles as the oracle (and so as the same simulation alone) to 1e-12."""
    w = W.couette(ny=40, ppc=50, precision="fp64")
    mixed = usp.Simulation(w).init_particles()
    others = [usp.Simulation(W.cavity(n=10, ppc=20, Kn=0.05, precision="fp64", seed=4)).init_particles(),
              usp.Simulation(W.slit(nx=20, ny=10, ppc=15, precision="fp64", seed=6)).init_particles()]
    B = usp.Batch(hbm_budget=8 << 30)
    for s in [mixed] + others:
        assert B.admit(s) == 0
    B.step(12)
    B.retire(mixed)
    o = oracle.OracleSim(w).init_particles()
    o.step(12)
    assert_particles_close(mixed.particles(), o.particles(), VSCALE, _cell_size(w))
    for s in others:
        B.retire(s)
    ws = W.slit(nx=20, ny=10, ppc=15, precision="fp64", seed=6)
    os_ = oracle.OracleSim(ws).init_particles()
    os_.step(12)
    assert_particles_close(others[1].particles(), os_.particles(), VSCALE, _cell_size(ws))


@pytest.mark.parametrize("pipeline", ["plain", "fused"])
def test_reload_reuses_storage(usp, pipeline):
    """Loading particles again into a handle (same size: the storage is kept;
    much smaller: it is reallocated) gives the state of a fresh handle: FP64
    per particle after steps (plain), identical particles right after the
    load (fused, FP32)."""
    prec = "fp64" if pipeline == "plain" else "fp32"
    w = W.couette(ny=40, ppc=50, precision=prec)
    w["params"]["pipeline"] = pipeline
    first = usp.Simulation(w).init_particles()
    P0 = first.particles()
    first.step(3)
    sub = {k: v[: len(v) // 8] for k, v in P0.items()}
    for P in (P0, sub, P0):
        first.set_particles(P["pos"], P["vel"], P["pid"])
        fresh = usp.Simulation(w).set_particles(P["pos"], P["vel"], P["pid"])
        if pipeline == "plain":
            first.step(4)
            fresh.step(4)
            assert_particles_close(first.particles(), fresh.particles(), VSCALE, _cell_size(w))
        else:
            a, b = by_pid(first.particles()), by_pid(fresh.particles())
            for k in ("pid", "pos", "vel", "cell"):
                assert np.array_equal(a[k], b[k]), k
            first.step(4)
            fresh.step(4)
            assert first.info()["n_particles"] == fresh.info()["n_particles"] == len(P["pid"])
        fresh.close()


def test_flux_plane_fp64_parity(usp):
    """The net count through the slit plane (the flow of Eq. 41) equals the
    oracle's after every step (paper slit: delta = 20, vacuum downstream)."""
    w = W.slit(nx=40, ny=20, ppc=30, precision="fp64", pressure_ratio=math.inf, delta=20.0)
    g, o = _pair(w, usp)
    for _ in range(25):
        g.step(1)
        o.step(1)
        assert g.info()["counters"][7] == o.counters()[4]
    assert o.counters()[4] > 0
    assert_particles_close(g.particles(), o.particles(), VSCALE, _cell_size(w))


def test_flux_plane_across_y_fp64_parity(usp):
    w = W.cavity(n=24, ppc=30, Kn=0.01, precision="fp64")
    w["params"].update(flux_axis=2, flux_pos=0.37 * w["grid"]["hi"][1])
    g, o = _pair(w, usp)
    g.step(12)
    o.step(12)
    assert g.info()["counters"][7] == o.counters()[4]
    assert o.counters()[4] != 0 or o.counters()[2] == 0


@pytest.mark.parametrize("pipeline", ["plain", "fused"])
def test_flux_plane_fp32_counts_change_of_side(usp, pipeline):
    """FP32 paths (no oracle stream to match): in a closed box each step adds
    to the count exactly the change in particles at or above the plane."""
    w = W.cavity(n=32, ppc=40, Kn=0.01, precision="fp32", seed=5)
    L = w["grid"]["hi"][0]
    w["segments"] = [{"pos": 0.5 * L, "lo": 0.6 * L, "hi": L, "kind": "diffuse", "T": W.T0,
                      "u": (0.0, 0.0, 0.0)}]
    w["params"].update(flux_axis=1, flux_pos=0.5 * L, pipeline=pipeline)
    p32 = float(np.float32(0.5 * L))
    g = usp.Simulation(w).init_particles()
    moved = 0
    for _ in range(8):
        before = int((g.particles()["pos"][:, 0] >= p32).sum())
        c0 = g.info()["counters"][7]
        g.step(1)
        d = g.info()["counters"][7] - c0
        assert d == int((g.particles()["pos"][:, 0] >= p32).sum()) - before
        moved += abs(d)
    assert moved > 0


@pytest.mark.parametrize("axis,pos", [(1, 2.0), (2, 0.0), (3, 0.5), (2, 0.5)])
def test_flux_plane_argument_errors(usp, axis, pos):
    if axis == 2 and pos == 0.5:
        w = W.homogeneous_box(ppc=10)            # periodic y
        pos *= w["grid"]["hi"][1]
    else:
        w = W.cavity(n=8, ppc=5, precision="fp64")
        pos *= w["grid"]["hi"][0]
    w["params"].update(flux_axis=axis, flux_pos=pos)
    with pytest.raises(usp.UspError) as e:
        usp.Simulation(w)
    assert e.value.status == -1


@pytest.mark.parametrize("name", ["sod", "slit"])
def test_fp64_gll_average_parity(usp, name):
    """Kn_GLL from the Eq. 34 averages (steady-flow option): particles,
    parameters and fields match the oracle as in the instantaneous reading."""
    if name == "sod":
        w = W.sod(ny=200, ppc_left=80, precision="fp64")
    else:
        w = W.slit(nx=40, ny=20, ppc=30, precision="fp64", pressure_ratio=math.inf, delta=20.0)
    w["params"].update(gll_average=1, n_avg=10)
    g, o = _pair(w, usp)
    g.step(15)
    o.step(15)
    assert_particles_close(g.particles(), o.particles(), VSCALE, _cell_size(w))
    pg, po = g.params(), o.params()
    assert np.array_equal(pg[:, 14], po[:, 14])
    sel = po[:, 14] > 0
    assert np.allclose(pg[sel, 13], po[sel, 13], rtol=1e-10, atol=1e-13)   # P_ne
    fa, oa = g.sample(averaged=True), o.fields(averaged=True)
    assert np.all(np.abs(fa - oa) <= 1e-10 * np.maximum(np.abs(oa), np.abs(oa).max(1, keepdims=True) * 1e-3))


@pytest.mark.parametrize("name,opts", [
    ("cavity", dict(selection="fixed_count")),
    ("sod", dict(mode="spesbgk", es_sampler="gallis_torczynski")),
    ("slit", dict(mode="spesbgk", selection="fixed_count", es_sampler="gallis_torczynski")),
])
def test_fp64_ablation_parity(usp, name, opts):
    """SP-ESBGK ablations on the plain FP64 path (fixed-count selection of
    Eq. 9, the Gallis-Torczynski sampler of Eqs. 10-11, the SP-ESBGK step of
    Eq. 8b): per particle against the oracle, relaxed counts bit-exact."""
    if name == "cavity":
        w = W.cavity(n=24, ppc=30, Kn=0.01, precision="fp64")
    elif name == "sod":
        w = W.sod(ny=200, ppc_left=80, precision="fp64")
    else:
        w = W.slit(nx=40, ny=20, ppc=30, precision="fp64")
    w["params"].update(opts)
    g, o = _pair(w, usp)
    g.step(10)
    o.step(10)
    assert_particles_close(g.particles(), o.particles(), VSCALE, _cell_size(w))
    pg, po = g.params(), o.params()
    assert np.array_equal(pg[:, 14], po[:, 14])
    assert np.array_equal(pg[:, 15], po[:, 15])
    assert po[:, 15].sum() > 0
    sel = po[:, 14] > 0
    assert np.allclose(pg[sel, 10:14], po[sel, 10:14], rtol=1e-10, atol=1e-300)
    fg, fo = g.sample(), o.fields()
    scale = np.maximum(np.abs(fo), np.abs(fo).max(axis=1, keepdims=True) * 1e-3)
    assert np.all(np.abs(fg - fo) <= 1e-10 * scale + 1e-300)
    assert g.info()["counters"][0] == o.counters()[0]


def test_torch_allocator_handle_matches_cudamalloc(usp):
    """A handle whose device memory comes from PyTorch's caching allocator
    (usp_allocator) holds it in torch's accounting while it lives, hands it
    all back on close, and steps like a handle on cudaMalloc (FP64, to the
    rounding of the sums)."""
    import torch
    w = W.couette(ny=20, ppc=50, precision="fp64", seed=3)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    a = usp.Simulation(w, allocator="torch").init_particles()
    held = torch.cuda.memory_allocated() - before
    assert held >= a.info()["device_bytes"] > 0
    b = usp.Simulation(w).init_particles()
    a.step(5)
    b.step(5)
    dy = (w["grid"]["hi"][1] - w["grid"]["lo"][1]) / w["grid"]["ny"]
    assert_particles_close(a.particles(), b.particles(), math.sqrt(KB_M_AR * W.T0), dy)
    a.close()
    b.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
