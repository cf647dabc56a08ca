"""Thin ctypes binding of the C ABI in include/usp.h (libusp.so).

Argument marshalling only: every stage of the particle update runs in the
CUDA kernels of libusp.so.  Loading fails loudly when the library is missing;
there is no CPU fallback.  PyTorch, when present, supplies the CUDA stream
and (optionally) the device allocator.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

NEXT_PID_AUTO = 0xFFFFFFFF   # usp_set_particles: one past the largest loaded id
OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "CAPACITY", -5: "TIMEOUT", -6: "STATE"}
NFIELDS = 16
NPRM = 16
FIELD_NAMES = ["n", "u0", "u1", "u2", "T", "pxx", "pyy", "pzz", "pxy", "pxz", "pyz", "q0", "q1", "q2",
               "Pne", "Nc"]
BC = {"diffuse": 0, "specular": 1, "periodic": 2, "reservoir": 3}
MODE = {"usp": 0, "sp": 1, "fixed": 2, "spesbgk": 3}
SELECTION = {"bernoulli": 0, "fixed_count": 1}
SAMPLER = {"cholesky": 0, "gallis_torczynski": 1}
PRECISION = {"fp64": 0, "fp32": 1}
PIPELINE = {"plain": 0, "fused": 1}
MAXSEG = 4

c_double, c_int, c_int32, c_int64, c_uint32, c_uint64, c_size_t, c_void_p = (
    ctypes.c_double, ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64,
    ctypes.c_size_t, ctypes.c_void_p)


class Gas(ctypes.Structure):
    _fields_ = [("mass", c_double), ("T_ref", c_double), ("mu_ref", c_double), ("omega", c_double),
                ("Pr", c_double)]


class Grid(ctypes.Structure):
    _fields_ = [("dim", c_int), ("nx", c_int), ("ny", c_int), ("lo", c_double * 2), ("hi", c_double * 2)]


class Bc(ctypes.Structure):
    _fields_ = [("kind", c_int), ("T", c_double), ("u", c_double * 3), ("n", c_double)]


class WallSegment(ctypes.Structure):
    _fields_ = [("pos", c_double), ("lo", c_double), ("hi", c_double), ("kind", c_int), ("T", c_double),
                ("u", c_double * 3)]


class Params(ctypes.Structure):
    _fields_ = [("Kn", c_double), ("L_ref", c_double), ("n_ref", c_double), ("dt", c_double),
                ("dt_over_tauc", c_double), ("body_accel", c_double * 3), ("ppc_ref", c_int),
                ("n_avg", c_int), ("mode", c_int), ("fixed_pne", c_double), ("reservoir_cols", c_int),
                ("precision", c_int), ("pipeline", c_int), ("capacity_factor", c_double),
                ("slab_count", c_int), ("slab_index", c_int), ("slab_group", c_int),
                ("flux_axis", c_int), ("flux_pos", c_double), ("gll_average", c_int),
                ("selection", c_int), ("es_sampler", c_int), ("weighted", c_int), ("r_p", c_double),
                ("weight_average", c_int)]


class Region(ctypes.Structure):
    _fields_ = [("lo", c_double * 2), ("hi", c_double * 2), ("n", c_double), ("T", c_double),
                ("u", c_double * 3)]


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)),
                ("free", ctypes.CFUNCTYPE(None, c_void_p, c_void_p)), ("ctx", c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("n_particles", c_int64), ("capacity", c_int64), ("n_cells", c_int32), ("precision", c_int32),
                ("pipeline", c_int32), ("step", c_uint32), ("dt", c_double), ("mu_ref", c_double),
                ("counters", c_int64 * 8), ("device_bytes", c_size_t), ("next_pid", c_uint32)]


class UspError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"usp status {status} ({ERRORS.get(status, '?')}): {msg}")
        self.status = status


_lib = None


def lib(build_if_missing: bool = True):
    """Load libusp.so (building it with nvcc first when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"libusp.so not built ({LIB_PATH}); run paper_1808_03801_gb300.build.build()")
        _build.build()
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "usp_create": (c_int, [P(Gas), P(Grid), P(Bc), P(WallSegment), c_int, P(Params), P(Allocator), c_void_p,
                               P(c_void_p)]),
        "usp_init_particles": (c_int, [c_void_p, P(Region), c_int, c_uint64]),
        "usp_set_particles": (c_int, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_uint32, c_uint64]),
        "usp_step": (c_int, [c_void_p, c_int]),
        "usp_sample_macro": (c_int, [c_void_p, c_int, c_void_p, c_size_t, c_int]),
        "usp_get_particles": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, P(c_int64)]),
        "usp_get_weights": (c_int, [c_void_p, c_void_p, c_int64, P(c_int64)]),
        "usp_run_stage": (c_int, [c_void_p, c_int]),
        "usp_get_params": (c_int, [c_void_p, c_void_p, c_size_t]),
        "usp_debug_philox": (c_int, [c_int64, c_void_p, c_uint32, c_uint32, c_void_p]),
        "usp_get_info": (c_int, [c_void_p, P(Info)]),
        "usp_synchronize": (c_int, [c_void_p]),
        "usp_destroy": (c_int, [c_void_p]),
        "usp_last_error": (ctypes.c_char_p, [c_void_p]),
        "usp_status_string": (ctypes.c_char_p, [c_int]),
        "usp_batch_create": (c_int, [c_size_t, c_int, c_void_p, P(c_void_p)]),
        "usp_batch_admit": (c_int, [c_void_p, c_void_p]),
        "usp_batch_step": (c_int, [c_void_p, c_int]),
        "usp_batch_retire": (c_int, [c_void_p, c_void_p]),
        "usp_batch_info": (c_int, [c_void_p, P(c_int), P(c_size_t)]),
        "usp_batch_destroy": (c_int, [c_void_p]),
        "usp_batch_run_stage": (c_int, [c_void_p, c_int]),
        "usp_fused_supported": (c_int, []),
        "usp_set_tuning": (c_int, [c_void_p, c_int, c_int]),
        "usp_get_tuning": (c_int, [c_void_p, P(c_int), P(c_int)]),
        "usp_cell_sort_static": (c_int, [P(Grid), c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


_STAGES = {
    "plain": [(0, "k_stream"), (2, "k_scan+k_scatter"), (3, "k_moments"), (4, "k_params"), (5, "k_relax"),
              (6, "k_finish")],
    "fused": [(10, "k_g2"), (12, "k_g1"), (13, "k_params_f"), (14, "k_lay_sum+scan+put+k_step_end")],
}
_LAUNCHES = {"plain": 7, "fused": 7}


def fused_available() -> bool:
    return hasattr(lib(), "usp_fused_supported") and bool(lib().usp_fused_supported())


def stage_list(pipeline: str):
    """(stage id, kernel names) of one step, for per-kernel timing."""
    return list(_STAGES[pipeline])


def launches_per_step(pipeline: str, reservoir: bool = False) -> int:
    return _LAUNCHES[pipeline] + (1 if reservoir else 0)


def exported_symbols():
    return [n for n in dir(lib()) if n.startswith("usp_")]


def _resolve_stream(stream):
    """(torch stream object or None, raw cudaStream_t).  The legacy default
    stream cannot be captured into a CUDA graph, so when the caller gives no
    stream and torch's current stream is the default one, a new torch stream
    is created for the handle."""
    if isinstance(stream, int):
        return None, stream
    if stream is not None:
        return stream, int(stream.cuda_stream)
    try:
        import torch
        if torch.cuda.is_available():
            cur = torch.cuda.current_stream()
            if cur.cuda_stream == 0:
                cur = torch.cuda.Stream()
            return cur, int(cur.cuda_stream)
    except Exception:
        pass
    return None, None


def _torch_allocator():
    import torch
    dev = torch.cuda.current_device()

    @ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)
    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        except Exception:
            return None

    @ctypes.CFUNCTYPE(None, c_void_p, c_void_p)
    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a = Allocator()
    a.alloc = _alloc
    a.free = _free
    a.ctx = None
    return a, (_alloc, _free)


def make_structs(w: dict, pipeline: str | None = None):
    g, gr, pr = w["gas"], w["grid"], w["params"]
    gas = Gas(g["mass"], g["T_ref"], g["mu_ref"], g["omega"], g["Pr"])
    grid = Grid(gr["dim"], gr["nx"], gr["ny"], (c_double * 2)(*gr["lo"]), (c_double * 2)(*gr["hi"]))
    faces = (Bc * 4)()
    for i, f in enumerate(w["faces"]):
        faces[i] = Bc(BC[f["kind"]], f["T"], (c_double * 3)(*f["u"]), f.get("n", 0.0))
    segs = (WallSegment * MAXSEG)()
    for i, s in enumerate(w.get("segments", [])):
        segs[i] = WallSegment(s["pos"], s["lo"], s["hi"], BC[s["kind"]], s["T"], (c_double * 3)(*s["u"]))
    pipe = pipeline or pr.get("pipeline", "plain")
    params = Params(pr["Kn"], pr["L_ref"], pr["n_ref"], pr["dt"], pr["dt_over_tauc"],
                    (c_double * 3)(*pr["body_accel"]), pr["ppc_ref"], pr["n_avg"], MODE[pr["mode"]],
                    pr["fixed_pne"], pr["reservoir_cols"], PRECISION[pr["precision"]], PIPELINE[pipe],
                    float(pr.get("capacity_factor", 0.0)), int(pr.get("slab_count", 0)),
                    int(pr.get("slab_index", 0)), int(pr.get("slab_group", 0)),
                    int(pr.get("flux_axis", 0)), float(pr.get("flux_pos", 0.0)),
                    int(pr.get("gll_average", 0)), SELECTION[pr.get("selection", "bernoulli")],
                    SAMPLER[pr.get("es_sampler", "cholesky")], int(pr.get("weighted", 0)),
                    float(pr.get("r_p", 10.0)), int(pr.get("weight_average", 0)))
    return gas, grid, faces, segs, len(w.get("segments", [])), params


def _regions(regions):
    arr = (Region * max(1, len(regions)))()
    for i, r in enumerate(regions):
        arr[i] = Region((c_double * 2)(*r["lo"]), (c_double * 2)(*r["hi"]), r["n"], r["T"], (c_double * 3)(*r["u"]))
    return arr


class Simulation:
    """One USP-ESBGK simulation on the GPU (a usp_handle)."""

    def __init__(self, w: dict, stream=None, allocator=None, pipeline=None):
        self.w = w
        self._keep = None
        L = lib()
        gas, grid, faces, segs, nseg, params = make_structs(w, pipeline)
        alloc_p = None
        if allocator == "torch":
            a, self._keep = _torch_allocator()
            self._alloc_struct = a
            alloc_p = ctypes.byref(a)
        h = c_void_p()
        self.stream, ptr = _resolve_stream(stream)
        rc = L.usp_create(ctypes.byref(gas), ctypes.byref(grid), faces, segs, nseg, ctypes.byref(params), alloc_p,
                          ptr, ctypes.byref(h))
        if rc != OK:
            raise UspError(rc, "usp_create rejected the workload")
        self._h = h
        self.dim = w["grid"]["dim"]
        # cells owned by this handle (a slab of a decomposed domain owns
        # ny / slab_count rows)
        slabs = max(1, int(w["params"].get("slab_count", 0)))
        self.K = (w["grid"]["nx"] if self.dim == 2 else 1) * (w["grid"]["ny"] // slabs)

    def _check(self, rc, what):
        if rc != OK:
            msg = lib().usp_last_error(self._h)
            raise UspError(rc, f"{what}: {msg.decode() if msg else ''}")

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().usp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_particles(self, regions=None, seed=None):
        regions = self.w["regions"] if regions is None else regions
        seed = self.w["seed"] if seed is None else seed
        self._check(lib().usp_init_particles(self._h, _regions(regions), len(regions), int(seed)),
                    "usp_init_particles")
        return self

    def set_particles(self, pos, vel, pid, next_pid=None, seed=None):
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 2)
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        pid = np.ascontiguousarray(pid, dtype=np.uint32)
        n = len(pid)
        nxt = NEXT_PID_AUTO if next_pid is None else int(next_pid)   # AUTO: found on the device
        seed = self.w["seed"] if seed is None else seed
        self._check(lib().usp_set_particles(self._h, n, pos.ctypes.data, vel.ctypes.data, pid.ctypes.data, nxt,
                                            int(seed)), "usp_set_particles")
        return self

    def step(self, n=1):
        self._check(lib().usp_step(self._h, int(n)), "usp_step")
        return self

    def run_stage(self, k):
        self._check(lib().usp_run_stage(self._h, int(k)), "usp_run_stage")
        return self

    def synchronize(self):
        self._check(lib().usp_synchronize(self._h), "usp_synchronize")

    def info(self):
        inf = Info()
        self._check(lib().usp_get_info(self._h, ctypes.byref(inf)), "usp_get_info")
        return {"n_particles": inf.n_particles, "capacity": inf.capacity, "n_cells": inf.n_cells,
                "precision": inf.precision, "pipeline": inf.pipeline, "step": inf.step, "dt": inf.dt,
                "mu_ref": inf.mu_ref, "counters": list(inf.counters), "device_bytes": inf.device_bytes,
                "next_pid": inf.next_pid}

    def sample(self, averaged=False, out=None):
        """Fields [16, K] as numpy (host) or into a device tensor `out`."""
        which = 1 if averaged else 0
        if out is not None:
            self._check(lib().usp_sample_macro(self._h, which, c_void_p(out.data_ptr()), out.numel(), 1),
                        "usp_sample_macro")
            return out
        a = np.zeros((NFIELDS, self.K))
        self._check(lib().usp_sample_macro(self._h, which, a.ctypes.data, a.size, 0), "usp_sample_macro")
        return a

    def particles(self):
        n = c_int64()
        inf = self.info()
        cap = inf["capacity"]
        pos = np.zeros((cap, 2))
        vel = np.zeros((cap, 3))
        pid = np.zeros(cap, dtype=np.uint32)
        cell = np.zeros(cap, dtype=np.int32)
        rc = lib().usp_get_particles(self._h, pos.ctypes.data, vel.ctypes.data, pid.ctypes.data, cell.ctypes.data,
                                     cap, ctypes.byref(n))
        self._check(rc, "usp_get_particles")
        m = n.value
        out = {"pos": pos[:m], "vel": vel[:m], "pid": pid[:m], "cell": cell[:m]}
        if self.w["params"].get("weighted"):
            wt = np.zeros(cap)
            nw = c_int64()
            self._check(lib().usp_get_weights(self._h, wt.ctypes.data, cap, ctypes.byref(nw)), "usp_get_weights")
            assert nw.value == m
            out["w"] = wt[:m]
        return out

    def set_tuning(self, fused_R=0, grid_per_sm=0):
        self._check(lib().usp_set_tuning(self._h, int(fused_R), int(grid_per_sm)), "usp_set_tuning")
        return self

    def tuning(self):
        r, g = c_int(), c_int()
        self._check(lib().usp_get_tuning(self._h, ctypes.byref(r), ctypes.byref(g)), "usp_get_tuning")
        return {"fused_R": r.value, "grid_per_sm": g.value}

    def params(self):
        out = np.zeros((self.K, NPRM))
        self._check(lib().usp_get_params(self._h, out.ctypes.data, out.size), "usp_get_params")
        return out


def reduced_mass_flow(w: dict, net: int, steps: int, dt: float) -> float:
    """Reduced mass flow rate W = Mdot / Mdot_fm through the slit (Eq. 41).

    net: particles counted through the plane (counters[7] difference) over
    `steps` steps of length dt.  Mdot counts both halves of the symmetric
    slit (the simulated domain is the upper half); each particle stands for
    n_ref / ppc_ref * dx * dy molecules per unit depth.  Mdot_fm = a p_1 /
    (sqrt(pi) v_1) is the free-molecular flow of the planar slit of width a,
    with p_1 and v_1 = sqrt(2 k T_1 / m) of the upstream reservoir (face
    x-lo)."""
    kB = 1.380649e-23
    gr, pr, up = w["grid"], w["params"], w["faces"][0]
    m = w["gas"]["mass"]
    dx = (gr["hi"][0] - gr["lo"][0]) / gr["nx"]
    dy = (gr["hi"][1] - gr["lo"][1]) / gr["ny"]
    molecules = pr["n_ref"] / pr["ppc_ref"] * dx * dy
    mdot = 2.0 * m * molecules * net / (steps * dt)
    p1 = up["n"] * kB * up["T"]
    v1 = math.sqrt(2.0 * kB * up["T"] / m)
    return mdot / (w["slit_width"] * p1 / (math.sqrt(math.pi) * v1))


def debug_philox(ctr, key):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    rc = lib().usp_debug_philox(len(ctr), ctr.ctypes.data, int(key[0]), int(key[1]), out.ctypes.data)
    if rc != OK:
        raise UspError(rc, "usp_debug_philox")
    return out


class Batch:
    """Many simulations advanced together by the same graph-captured launches."""

    def __init__(self, hbm_budget: int, max_sims: int = 1024, stream=None):
        b = c_void_p()
        self.stream, ptr = _resolve_stream(stream)
        rc = lib().usp_batch_create(int(hbm_budget), int(max_sims), ptr, ctypes.byref(b))
        if rc != OK:
            raise UspError(rc, "usp_batch_create")
        self._b = b

    def admit(self, sim: Simulation) -> int:
        """Returns 0 when admitted, a negative status otherwise (CAPACITY: no room yet)."""
        return lib().usp_batch_admit(self._b, sim.handle)

    def retire(self, sim: Simulation):
        rc = lib().usp_batch_retire(self._b, sim.handle)
        if rc != OK:
            raise UspError(rc, "usp_batch_retire")

    def step(self, n=1):
        rc = lib().usp_batch_step(self._b, int(n))
        if rc != OK:
            raise UspError(rc, "usp_batch_step")

    def run_stage(self, k):
        rc = lib().usp_batch_run_stage(self._b, int(k))
        if rc != OK:
            raise UspError(rc, "usp_batch_run_stage")

    def info(self):
        n, b = c_int(), c_size_t()
        lib().usp_batch_info(self._b, ctypes.byref(n), ctypes.byref(b))
        return n.value, b.value

    def close(self):
        if getattr(self, "_b", None):
            lib().usp_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
