"""Pins of the oracle's counting plane (the net particle flow behind the slit's
reduced mass flow rate, Eq. 41).

* Side-change identity: in a closed box, the count added by one advection
  equals the change in the number of particles at or above the plane, read
  from the particle positions (planes across x and across y, with a plate
  that ends on the plane).
* Effusion: from a uniform Maxwellian half-space (nothing on the other
  side), the particles through a plane in one free flight of length dt
  number n sqrt(kT / (2 pi m)) dt per unit area -- the one-sided flux that
  also gives the free-molecular slit flow Mdot_fm = a p_1 / (sqrt(pi) v_1)
  of Eq. 41.  The test checks both forms.
* Configurations that cannot define the plane are rejected.
"""
import copy
import math

import numpy as np
import pytest

import oracle
from paper_1808_03801_gb300 import workloads as W

KB = 1.380649e-23


def _above(o, axis, pos):
    P = o.particles()
    return int((P["pos"][:, axis - 1] >= pos).sum())


@pytest.mark.parametrize("axis,frac", [(1, 0.5), (2, 0.37)])
def test_count_equals_change_of_side(axis, frac):
    w = W.cavity(n=16, ppc=20, Kn=0.01, precision="fp64", seed=3)
    L = w["grid"]["hi"][0]
    pos = frac * L
    w["segments"] = [{"pos": 0.5 * L, "lo": 0.6 * L, "hi": L, "kind": "diffuse", "T": W.T0,
                      "u": (0.0, 0.0, 0.0)}]
    w["params"]["flux_axis"] = axis
    w["params"]["flux_pos"] = pos
    o = oracle.OracleSim(w).init_particles()
    total = 0
    for _ in range(6):
        before = _above(o, axis, pos)
        c0 = o.counters()[4]
        o.phase(0)   # advection
        d = o.counters()[4] - c0
        assert d == _above(o, axis, pos) - before
        total += abs(d)
        for ph in range(1, 7):
            o.phase(ph)
    assert total > 0   # the flights did cross the plane


def _effusion_box(n_left_cols=10, ppc=400, ny=4, hop=0.2):
    """x in [-L, L] (diffuse ends), y periodic; gas only at x < 0; dt such
    that a thermal speed sqrt(kT/m) covers hop * L in one step."""
    L, H = 1.0e-5, 2.0e-6
    faces = [W._face("diffuse"), W._face("diffuse"), W._face("periodic"), W._face("periodic")]
    regions = [{"lo": (-L, 0.0), "hi": (0.0, H), "n": W.N0, "T": W.T0, "u": (0.0, 0.0, 0.0)},
               {"lo": (0.0, 0.0), "hi": (L, H), "n": 0.0, "T": W.T0, "u": (0.0, 0.0, 0.0)}]
    w = W._base(2, 2 * n_left_cols, ny, (-L, 0.0), (L, H), faces, Kn=0.1, L_ref=L, dt_over_tauc=1.0,
                ppc=ppc, precision="fp64", regions=regions, seed=11)
    w["params"]["dt"] = hop * L / math.sqrt(KB * W.T0 / W.M_AR)
    w["params"]["flux_axis"] = 1
    w["params"]["flux_pos"] = 0.0
    return w, L, H


def test_effusion_matches_one_sided_flux():
    w, L, H = _effusion_box()
    o = oracle.OracleSim(w).init_particles()
    n_left = o.n
    assert _above(o, 1, 0.0) == 0
    o.phase(0)
    count = int(o.counters()[4])
    theta = KB * W.T0 / W.M_AR
    n_area = n_left / (L * H)                           # simulated particles per unit area
    expected = n_area * H * o.dt * math.sqrt(theta / (2.0 * math.pi))
    assert abs(count - expected) < 4.5 * math.sqrt(expected), (count, expected)
    # the same count as a mass flow against Mdot_fm = a p_1 / (sqrt(pi) v_1),
    # a = H: (count m / dt) / (H n m v_1 / (2 sqrt(pi))) -> 1
    v1 = math.sqrt(2.0 * theta)
    ratio = (count / o.dt) / (H * n_area * v1 / (2.0 * math.sqrt(math.pi)))
    assert abs(ratio - 1.0) < 4.5 / math.sqrt(expected)
    # nothing comes back through the plane: every crossing went forward
    P = o.particles()
    assert int((P["pos"][:, 0] >= 0.0).sum()) == count


def test_reverse_flight_counts_negative():
    """The mirror image (gas only at x >= 0) counts the same flow negative."""
    w, L, H = _effusion_box()
    w["regions"] = [{"lo": (-L, 0.0), "hi": (0.0, H), "n": 0.0, "T": W.T0, "u": (0.0, 0.0, 0.0)},
                    {"lo": (0.0, 0.0), "hi": (L, H), "n": W.N0, "T": W.T0, "u": (0.0, 0.0, 0.0)}]
    o = oracle.OracleSim(w).init_particles()
    o.phase(0)
    P = o.particles()
    assert int(o.counters()[4]) == -int((P["pos"][:, 0] < 0.0).sum()) < 0


@pytest.mark.parametrize("change", ["outside", "on_face", "x_in_1d", "periodic", "bad_axis"])
def test_plane_rejected(change):
    if change == "x_in_1d":
        w = W.couette(ny=10, ppc=10)
        w["params"].update(flux_axis=1, flux_pos=0.5)
    elif change == "periodic":
        w = W.homogeneous_box(ppc=10)
        w["params"].update(flux_axis=2, flux_pos=0.5 * w["grid"]["hi"][1])
    else:
        w = W.cavity(n=8, ppc=5, precision="fp64")
        L = w["grid"]["hi"][0]
        axis, pos = {"outside": (1, 1.5 * L), "on_face": (2, 0.0), "bad_axis": (3, 0.5 * L)}[change]
        w["params"].update(flux_axis=axis, flux_pos=pos)
    with pytest.raises(ValueError):
        oracle.OracleSim(w)


def test_slit_without_plane_counts_nothing():
    w = W.slit(nx=20, ny=10, ppc=10, precision="fp64")
    w2 = copy.deepcopy(w)
    w2["params"]["flux_axis"] = 0
    a = oracle.OracleSim(w).init_particles().step(5)
    b = oracle.OracleSim(w2).init_particles().step(5)
    assert b.counters()[4] == 0
    assert np.array_equal(a.counters()[:4], b.counters()[:4])   # counting changes nothing else
    Pa, Pb = a.particles(), b.particles()
    assert np.array_equal(Pa["pos"], Pb["pos"]) and np.array_equal(Pa["vel"], Pb["vel"])


def test_count_with_reservoir_faces_counts_exits_at_the_face():
    """Slit with reservoirs at both ends (vacuum downstream) and the plate:
    after the advection phase the particles that left through a reservoir
    face are still listed, at the face they crossed, so the count of the
    phase equals the change of side over all listed particles -- including
    the ones about to be removed."""
    w = W.slit(nx=40, ny=20, ppc=20, precision="fp64", pressure_ratio=math.inf, delta=20.0,
               dt_over_tauc=3.0, reservoir_cols=3)
    o = oracle.OracleSim(w).init_particles()
    removed = 0
    for _ in range(8):
        before = _above(o, 1, 0.0)
        c0, r0 = o.counters()[4], o.counters()[2]
        o.phase(0)
        exits = o.counters()[2] - r0          # left through a reservoir face in this flight
        assert o.counters()[4] - c0 == _above(o, 1, 0.0) - before
        removed += exits
        for ph in range(1, 7):
            o.phase(ph)
    assert removed > 0                          # some flights did end on a reservoir face
    assert o.counters()[4] > 0                  # net flow toward the vacuum


def test_reduced_mass_flow_is_one_for_free_molecular_effusion():
    """The product's Eq. 41 normalisation (usp.reduced_mass_flow, host
    arithmetic only) applied to the oracle's effusion count through an open
    plane of height H gives W = 1: Mdot_fm = a p_1 / (sqrt(pi) v_1) is the
    free-molecular flow, and the helper's symmetric doubling is matched by
    taking a = 2H."""
    from paper_1808_03801_gb300 import usp as U
    w, L, H = _effusion_box()
    o = oracle.OracleSim(w).init_particles()
    o.phase(0)
    count = int(o.counters()[4])
    w["faces"][0] = dict(w["faces"][0], n=W.N0)   # the gas state the flow comes from
    w["slit_width"] = 2.0 * H
    Wr = U.reduced_mass_flow(w, count, 1, o.dt)
    # the particles per unit area of the filled half set the expected count
    n_left = sum(1 for x in o.particles()["pos"][:, 0] if x < 0.0) + count
    expected = n_left / (L * H) * H * o.dt * math.sqrt(KB * W.T0 / W.M_AR / (2.0 * math.pi))
    assert abs(Wr - 1.0) < 4.5 / math.sqrt(expected), Wr
