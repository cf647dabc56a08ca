"""ctypes access to the plain FP64 CPU oracle (oracle/usp_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The product library never imports this
package, and this package imports nothing from the product.

Workload dicts (see paper_1808_03801_gb300/workloads.py for the format) are
translated into the oracle's own configuration struct here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "usp_oracle.c")
SO = os.path.join(HERE, "liborc.so")

NFIELDS = 16
FIELD_NAMES = ["n", "u0", "u1", "u2", "T", "pxx", "pyy", "pzz", "pxy", "pxz", "pyz",
               "q0", "q1", "q2", "Pne", "Nc"]
PH_STREAM, PH_RESERVOIR, PH_SORT, PH_MOMENTS, PH_PARAMS, PH_RELAX, PH_SAMPLE = range(7)
_BC = {"diffuse": 0, "specular": 1, "periodic": 2, "reservoir": 3}
_MODE = {"usp": 0, "sp": 1, "fixed": 2, "spesbgk": 3}
MAXSEG = 4


class _Config(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("T_ref", ctypes.c_double), ("mu_ref", ctypes.c_double),
        ("omega", ctypes.c_double), ("Pr", ctypes.c_double),
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
        ("face_kind", ctypes.c_int * 4), ("face_T", ctypes.c_double * 4),
        ("face_u", (ctypes.c_double * 3) * 4), ("face_n", ctypes.c_double * 4),
        ("nseg", ctypes.c_int),
        ("seg_pos", ctypes.c_double * MAXSEG), ("seg_lo", ctypes.c_double * MAXSEG),
        ("seg_hi", ctypes.c_double * MAXSEG), ("seg_kind", ctypes.c_int * MAXSEG),
        ("seg_T", ctypes.c_double * MAXSEG), ("seg_u", (ctypes.c_double * 3) * MAXSEG),
        ("Kn", ctypes.c_double), ("L_ref", ctypes.c_double), ("n_ref", ctypes.c_double),
        ("dt", ctypes.c_double), ("dt_over_tauc", ctypes.c_double),
        ("body_accel", ctypes.c_double * 3),
        ("ppc_ref", ctypes.c_int), ("n_avg", ctypes.c_int), ("mode", ctypes.c_int),
        ("fixed_pne", ctypes.c_double), ("reservoir_cols", ctypes.c_int),
        ("flux_axis", ctypes.c_int), ("flux_pos", ctypes.c_double), ("gll_average", ctypes.c_int),
        ("selection", ctypes.c_int), ("es_sampler", ctypes.c_int),
        ("weighted", ctypes.c_int), ("r_p", ctypes.c_double), ("weight_average", ctypes.c_int),
    ]


class _Region(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2), ("n", ctypes.c_double),
                ("T", ctypes.c_double), ("u", ctypes.c_double * 3)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, plain -O2)."""
    if force or not os.path.exists(SO) or os.path.getmtime(SO) < os.path.getmtime(SRC):
        tmp = SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, SO)
    return SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i32, i64, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_double)
        P = ctypes.POINTER
        L.orc_create.restype = vp
        L.orc_create.argtypes = [P(_Config)]
        L.orc_destroy.argtypes = [vp]
        L.orc_init_particles.argtypes = [vp, P(_Region), i32, u64]
        L.orc_set_particles.argtypes = [vp, i64, vp, vp, vp, u32, u64]
        L.orc_phase.argtypes = [vp, i32]
        L.orc_step.argtypes = [vp, i32]
        L.orc_num_particles.restype = i64
        L.orc_num_particles.argtypes = [vp]
        L.orc_num_cells.argtypes = [vp]
        L.orc_dt.restype = dbl
        L.orc_dt.argtypes = [vp]
        L.orc_mu_ref.restype = dbl
        L.orc_mu_ref.argtypes = [vp]
        L.orc_step_index.restype = u32
        L.orc_step_index.argtypes = [vp]
        for f in ("orc_get_particles",):
            getattr(L, f).argtypes = [vp, vp, vp, vp, vp]
        L.orc_get_counts.argtypes = [vp, vp]
        L.orc_get_weights.argtypes = [vp, vp]
        L.orc_get_fields.argtypes = [vp, i32, vp]
        L.orc_get_params.argtypes = [vp, vp]
        L.orc_get_counters.argtypes = [vp, vp]
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_u01.restype = dbl
        L.orc_u01.argtypes = [u32]
        _lib = L
    return _lib


def philox(ctr, key):
    """Philox4x32-10 words for one counter (4 x u32) and key (2 x u32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def u01(x: int) -> float:
    return lib().orc_u01(int(x))


def make_config(w: dict) -> _Config:
    c = _Config()
    g, gr, pr = w["gas"], w["grid"], w["params"]
    c.mass, c.T_ref, c.mu_ref, c.omega, c.Pr = g["mass"], g["T_ref"], g["mu_ref"], g["omega"], g["Pr"]
    c.dim, c.nx, c.ny = gr["dim"], gr["nx"], gr["ny"]
    for i in range(2):
        c.lo[i], c.hi[i] = gr["lo"][i], gr["hi"][i]
    for f, face in enumerate(w["faces"]):
        c.face_kind[f] = _BC[face["kind"]]
        c.face_T[f] = face["T"]
        for d in range(3):
            c.face_u[f][d] = face["u"][d]
        c.face_n[f] = face.get("n", 0.0)
    segs = w.get("segments", [])
    c.nseg = len(segs)
    for i, s in enumerate(segs):
        c.seg_pos[i], c.seg_lo[i], c.seg_hi[i] = s["pos"], s["lo"], s["hi"]
        c.seg_kind[i] = _BC[s["kind"]]
        c.seg_T[i] = s["T"]
        for d in range(3):
            c.seg_u[i][d] = s["u"][d]
    c.Kn, c.L_ref, c.n_ref = pr["Kn"], pr["L_ref"], pr["n_ref"]
    c.dt, c.dt_over_tauc = pr["dt"], pr["dt_over_tauc"]
    for d in range(3):
        c.body_accel[d] = pr["body_accel"][d]
    c.ppc_ref, c.n_avg, c.mode = pr["ppc_ref"], pr["n_avg"], _MODE[pr["mode"]]
    c.fixed_pne, c.reservoir_cols = pr["fixed_pne"], pr["reservoir_cols"]
    c.flux_axis, c.flux_pos = int(pr.get("flux_axis", 0)), float(pr.get("flux_pos", 0.0))
    c.gll_average = int(pr.get("gll_average", 0))
    c.selection = {"bernoulli": 0, "fixed_count": 1}[pr.get("selection", "bernoulli")]
    c.es_sampler = {"cholesky": 0, "gallis_torczynski": 1}[pr.get("es_sampler", "cholesky")]
    c.weighted = int(pr.get("weighted", 0))
    c.r_p = float(pr.get("r_p", 10.0))
    c.weight_average = int(pr.get("weight_average", 0))
    return c


class OracleSim:
    """One simulation held by the oracle."""

    def __init__(self, w: dict):
        self.w = w
        self._cfg = make_config(w)
        self._h = lib().orc_create(ctypes.byref(self._cfg))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.dim = w["grid"]["dim"]
        self.K = lib().orc_num_cells(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    # state set-up
    def init_particles(self, regions=None, seed=None):
        regions = self.w["regions"] if regions is None else regions
        seed = self.w["seed"] if seed is None else seed
        arr = (_Region * max(1, len(regions)))()
        for i, r in enumerate(regions):
            for d in range(2):
                arr[i].lo[d], arr[i].hi[d] = r["lo"][d], r["hi"][d]
            arr[i].n, arr[i].T = r["n"], r["T"]
            for d in range(3):
                arr[i].u[d] = r["u"][d]
        rc = lib().orc_init_particles(self._h, arr, len(regions), int(seed))
        if rc:
            raise RuntimeError("orc_init_particles failed")
        return self

    def set_particles(self, pos, vel, pid, next_pid=None, seed=None):
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 2)
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        pid = np.ascontiguousarray(pid, dtype=np.uint32)
        n = len(pid)
        nxt = int(pid.max()) + 1 if next_pid is None and n else (next_pid or 0)
        seed = self.w["seed"] if seed is None else seed
        rc = lib().orc_set_particles(self._h, n, pos.ctypes.data, vel.ctypes.data, pid.ctypes.data, nxt,
                                     int(seed))
        if rc:
            raise RuntimeError("orc_set_particles failed")
        return self

    # time stepping
    def step(self, n=1):
        lib().orc_step(self._h, int(n))
        return self

    def phase(self, ph):
        lib().orc_phase(self._h, int(ph))
        return self

    # queries
    @property
    def n(self):
        return int(lib().orc_num_particles(self._h))

    @property
    def dt(self):
        return float(lib().orc_dt(self._h))

    @property
    def mu_ref(self):
        return float(lib().orc_mu_ref(self._h))

    @property
    def step_index(self):
        return int(lib().orc_step_index(self._h))

    def particles(self):
        n = self.n
        pos = np.zeros((n, 2))
        vel = np.zeros((n, 3))
        pid = np.zeros(n, dtype=np.uint32)
        cell = np.zeros(n, dtype=np.int32)
        lib().orc_get_particles(self._h, pos.ctypes.data, vel.ctypes.data, pid.ctypes.data, cell.ctypes.data)
        w = np.zeros(n)
        lib().orc_get_weights(self._h, w.ctypes.data)
        return {"pos": pos, "vel": vel, "pid": pid, "cell": cell, "w": w}

    def counts(self):
        out = np.zeros(self.K, dtype=np.int32)
        lib().orc_get_counts(self._h, out.ctypes.data)
        return out

    def fields(self, averaged=False):
        out = np.zeros((NFIELDS, self.K))
        lib().orc_get_fields(self._h, int(bool(averaged)), out.ctypes.data)
        return out

    def params(self):
        out = np.zeros((self.K, 16))
        lib().orc_get_params(self._h, out.ctypes.data)
        return out

    def counters(self):
        out = np.zeros(5, dtype=np.int64)
        lib().orc_get_counters(self._h, out.ctypes.data)
        return out
