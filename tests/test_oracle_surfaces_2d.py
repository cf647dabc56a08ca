"""Pins of the oracle's 2-D surface logic (Table 1 steps 1-2: free flight with
wall interactions "similar to DSMC"; zero-thickness plates of Sec. 4.5).

Each case is a closed form of the flight, not a restatement of the code:

* a box with four specular faces: each axis unfolds independently into mirror
  images, whatever the order of the hits, so the final position and the signs
  of the velocity follow from the straight path alone;
* a specular plate: a crossing inside its span mirrors x about the plate,
  a crossing outside it passes straight;
* a diffuse plate and a diffuse x-face: the particle is re-emitted from the
  exact hit point back to its own side, with a Rayleigh normal speed and
  Gaussian tangential components about the wall velocity (full
  accommodation), and flies straight for the rest of the step;
* an exact corner hit: the x-face takes the hit first (its re-emission uses
  the wall draw with bounce index 0), and the y-face is met next at zero
  distance.
"""
import math

import numpy as np
from scipy import stats

import oracle
from oracle import PH_STREAM
from paper_1808_03801_gb300 import workloads as W

KB = 1.380649e-23
R = KB / W.M_AR
L = 1.0e-4


def _face(kind, T=W.T0, u=(0.0, 0.0, 0.0)):
    return {"kind": kind, "T": float(T), "u": tuple(u), "n": 0.0}


def _box(faces, lo=(0.0, 0.0), hi=(L, L), n=8, dt=1.0e-8, segments=()):
    w = W.cavity(n=n, ppc=10, Kn=0.01, precision="fp64")
    w["grid"]["lo"], w["grid"]["hi"] = tuple(lo), tuple(hi)
    w["faces"] = list(faces)
    w["segments"] = list(segments)
    w["params"]["dt"] = dt
    return w


def _fly(w, pos, vel):
    s = oracle.OracleSim(w)
    s.set_particles(pos, vel, np.arange(len(pos), dtype=np.uint32))
    s.phase(PH_STREAM)
    P = s.particles()
    o = np.argsort(P["pid"])
    return {k: v[o] for k, v in P.items()}


def _unfold(p, c, lo, hi, t):
    s = (p + c * t - lo) / (hi - lo)
    m = np.floor(s)
    r = s - m
    even = (m.astype(np.int64) % 2) == 0
    return np.where(even, lo + r * (hi - lo), hi - r * (hi - lo)), np.where(even, c, -c)


def test_specular_box_unfolds_both_axes():
    dt = 1.0e-7
    w = _box([_face("specular")] * 4, dt=dt)
    rng = np.random.default_rng(31)
    n = 4000
    pos = rng.uniform(0, L, (n, 2))
    vel = np.clip(rng.normal(0, 1000.0, (n, 3)), -2900.0, 2900.0)   # <= 3 hits per axis
    P = _fly(w, pos, vel)
    for ax in range(2):
        p_exp, c_exp = _unfold(pos[:, ax], vel[:, ax], 0.0, L, dt)
        assert np.allclose(P["pos"][:, ax], p_exp, rtol=0, atol=1e-12 * L)
        assert np.array_equal(P["vel"][:, ax], c_exp)
    assert np.array_equal(P["vel"][:, 2], vel[:, 2])
    assert (np.abs(vel[:, :2]) * dt > L).any(axis=1).sum() > 100   # many multi-hit flights


def _plate_setup(kind, T=W.T0, u=(0.0, 0.0, 0.0)):
    dt = 1.0e-8
    seg = {"pos": 0.0, "lo": 0.3 * L, "hi": 0.8 * L, "kind": kind, "T": float(T), "u": tuple(u)}
    w = _box([_face("specular")] * 4, lo=(-L, 0.0), hi=(L, L), dt=dt, segments=[seg])
    return w, dt, seg


def test_specular_plate_mirrors_inside_its_span():
    w, dt, seg = _plate_setup("specular")
    rng = np.random.default_rng(32)
    n = 6000
    pos = np.column_stack([rng.uniform(-0.1 * L, 0.1 * L, n), rng.uniform(0.15 * L, 0.85 * L, n)])
    vel = np.clip(rng.normal(0, 400.0, (n, 3)), -1000.0, 1000.0)
    P = _fly(w, pos, vel)
    t_h = (0.0 - pos[:, 0]) / vel[:, 0]
    y_h = pos[:, 1] + vel[:, 1] * t_h
    hit = (t_h > 0) & (t_h <= dt) & (y_h >= seg["lo"]) & (y_h <= seg["hi"])
    x_free = pos[:, 0] + vel[:, 0] * dt
    x_exp = np.where(hit, -x_free, x_free)
    cx_exp = np.where(hit, -vel[:, 0], vel[:, 0])
    assert np.allclose(P["pos"][:, 0], x_exp, rtol=0, atol=1e-12 * L)
    assert np.allclose(P["pos"][:, 1], pos[:, 1] + vel[:, 1] * dt, rtol=0, atol=1e-12 * L)
    assert np.array_equal(P["vel"][:, 0], cx_exp)
    assert np.array_equal(P["vel"][:, 1:], vel[:, 1:])
    crossed_outside = (t_h > 0) & (t_h <= dt) & ~hit
    assert hit.sum() > 500 and crossed_outside.sum() > 100


def _check_accommodation(cn, ct1, ct2, u1, u2, T):
    th = R * T
    assert stats.kstest(cn / math.sqrt(th), "rayleigh").pvalue > 1e-3
    assert stats.kstest((ct1 - u1) / math.sqrt(th), "norm").pvalue > 1e-3
    assert stats.kstest((ct2 - u2) / math.sqrt(th), "norm").pvalue > 1e-3
    # a wrong wall temperature or a missing wall velocity is far outside these
    assert abs(np.mean(ct1) - u1) < 5 * math.sqrt(th / len(ct1))


def test_diffuse_plate_reemits_from_the_hit_point():
    Tp, up = 350.0, (0.0, 60.0, -40.0)
    w, dt, seg = _plate_setup("diffuse", Tp, up)
    rng = np.random.default_rng(33)
    n = 20000
    side = np.where(rng.random(n) < 0.5, -1.0, 1.0)            # start left (-1) or right (+1) of the plate
    cx = -side * 800.0
    x0 = side * rng.uniform(0, 0.5 * 800.0 * dt, n)
    pos = np.column_stack([x0, rng.uniform(0.45 * L, 0.65 * L, n)])
    vel = np.column_stack([cx, rng.normal(0, 100.0, n), rng.normal(0, 100.0, n)])
    P = _fly(w, pos, vel)
    t_h = -x0 / cx
    rest = dt - t_h
    v = P["vel"]
    assert np.all(np.sign(v[:, 0]) == side)                    # back to the side it came from
    assert np.allclose(P["pos"][:, 0], v[:, 0] * rest, rtol=0, atol=1e-12 * L)
    assert np.allclose(P["pos"][:, 1], pos[:, 1] + vel[:, 1] * t_h + v[:, 1] * rest, rtol=0, atol=1e-12 * L)
    _check_accommodation(np.abs(v[:, 0]), v[:, 1], v[:, 2], up[1], up[2], Tp)


def test_diffuse_x_face_reemits_from_the_hit_point():
    Tw, uw = 320.0, (0.0, 45.0, 0.0)
    dt = 1.0e-8
    faces = [_face("specular"), _face("diffuse", Tw, uw), _face("specular"), _face("specular")]
    w = _box(faces, dt=dt)
    rng = np.random.default_rng(34)
    n = 20000
    x0 = L - rng.uniform(0, 0.5 * 800.0 * dt, n)
    pos = np.column_stack([x0, rng.uniform(0.3 * L, 0.7 * L, n)])
    vel = np.column_stack([np.full(n, 800.0), rng.normal(0, 100.0, n), rng.normal(0, 100.0, n)])
    P = _fly(w, pos, vel)
    t_h = (L - x0) / 800.0
    rest = dt - t_h
    v = P["vel"]
    assert np.all(v[:, 0] < 0)
    assert np.allclose(P["pos"][:, 0], L + v[:, 0] * rest, rtol=0, atol=1e-12 * L)
    assert np.allclose(P["pos"][:, 1], pos[:, 1] + vel[:, 1] * t_h + v[:, 1] * rest, rtol=0, atol=1e-12 * L)
    _check_accommodation(-v[:, 0], v[:, 1], v[:, 2], uw[1], uw[2], Tw)


def _u01(word):
    return (float(word) + 0.5) * 2.0 ** -32


def test_exact_corner_hit_goes_to_the_x_face_first():
    """Heading exactly at the corner of a diffuse x-lo face and a specular y-lo
    face: the x-face is met first (bounce index 0 of the wall draw: Rayleigh
    normal speed from word 0, tangential normals from words 1-2 by Box-Muller),
    then the y-face at zero distance flips a downward y component."""
    Tw = 300.0
    dt = 1.0e-8
    faces = [_face("diffuse", Tw), _face("specular"), _face("specular"), _face("specular")]
    w = _box(faces, dt=dt)
    seed = w["seed"]
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    n = 64
    a = 1000.0 * (1.0 + np.arange(n) / n)
    x0 = 0.25 * 2.0 ** -16 * np.ones(n)        # t_x = x0 / a and t_y = 2 x0 / (2 a): equal in FP64
    pos = np.column_stack([x0, 2.0 * x0])
    vel = np.column_stack([-a, -2.0 * a, np.zeros(n)])
    t_h = x0 / a
    assert np.array_equal((0.0 - pos[:, 0]) / vel[:, 0], (0.0 - pos[:, 1]) / vel[:, 1])
    P = _fly(w, pos, vel)
    th = R * Tw
    for i in range(n):
        wd = oracle.philox(np.array([i, 0, 2, 0], dtype=np.uint32), key)
        cx = math.sqrt(-2.0 * th * math.log(_u01(wd[0])))
        r = math.sqrt(-2.0 * math.log(_u01(wd[1])))
        cy = math.sqrt(th) * r * math.cos(2.0 * math.pi * _u01(wd[2]))
        cz = math.sqrt(th) * r * math.sin(2.0 * math.pi * _u01(wd[2]))
        rest = dt - t_h[i]
        want_v = np.array([cx, abs(cy), cz])
        assert np.allclose(P["vel"][i], want_v, rtol=1e-12, atol=1e-9), (i, P["vel"][i], want_v)
        assert np.allclose(P["pos"][i], [cx * rest, abs(cy) * rest], rtol=1e-12, atol=1e-12 * L), i
