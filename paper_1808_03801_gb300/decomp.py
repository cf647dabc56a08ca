"""Spatial decomposition of one domain into slabs of rows, stepped together.

The paper's method has no decomposition; this is how one domain would be
spread over several devices.  Here the slabs are handles of one batch on one
GPU: a particle that crosses into another slab is written into that slab's
buckets during the step, and the Kn_GLL stencil (Eq. 18) of a boundary row
reads the adjacent slab's row.  The host side splits a global particle state
by row (`owner_rows`), which is also the routing rule a multi-device run
would use to exchange particles.
"""
from __future__ import annotations

import copy

import numpy as np

from . import usp as U


def slab_workloads(w: dict, nslabs: int, group: int = 1) -> list[dict]:
    """The workload of every slab: the same grid, faces and parameters, each
    slab owning ny / nslabs consecutive rows.  Particles move between slabs,
    so each slab's storage is sized for 3x its initial count."""
    ny = w["grid"]["ny"]
    if nslabs < 2 or ny % nslabs:
        raise ValueError("ny must be a multiple of the slab count (>= 2)")
    out = []
    for k in range(nslabs):
        ws = copy.deepcopy(w)
        ws["params"]["pipeline"] = "fused"
        ws["params"]["slab_count"] = nslabs
        ws["params"]["slab_index"] = k
        ws["params"]["slab_group"] = group
        ws["params"]["capacity_factor"] = max(float(ws["params"].get("capacity_factor", 0.0)), 3.0)
        out.append(ws)
    return out


def owner_rows(pos: np.ndarray, w: dict, nslabs: int) -> np.ndarray:
    """Slab of every particle: its grid row computed in FP32 exactly as the
    device does for FP32 storage, divided by the rows per slab."""
    gr = w["grid"]
    lo = np.float32(gr["lo"][1])
    dy = np.float32((gr["hi"][1] - gr["lo"][1]) / gr["ny"])
    y = np.asarray(pos)[:, 1].astype(np.float32)
    row = np.floor((y - lo) / dy).astype(np.int64)
    row = np.clip(row, 0, gr["ny"] - 1)
    return row // (gr["ny"] // nslabs)


def split(P: dict, w: dict, nslabs: int) -> list[dict]:
    """Per-slab particle arrays (pos, vel, pid) of a global state."""
    own = owner_rows(P["pos"], w, nslabs)
    return [{k: np.ascontiguousarray(P[k][own == s]) for k in ("pos", "vel", "pid")} for s in range(nslabs)]


class DecomposedSim:
    """One domain as `nslabs` slab handles in one batch."""

    def __init__(self, w: dict, nslabs: int, group: int = 1, hbm_budget: int = 64 << 30):
        self.w = w
        self.nslabs = nslabs
        self.slabs = [U.Simulation(ws) for ws in slab_workloads(w, nslabs, group)]
        self.batch = U.Batch(hbm_budget=hbm_budget, max_sims=nslabs)
        self._admitted = False

    def load(self, P: dict, next_pid: int | None = None):
        """Distribute a global particle state (pos, vel, pid) over the slabs."""
        self._retire()
        nxt = int(P["pid"].max()) + 1 if next_pid is None and len(P["pid"]) else next_pid
        for sim, part in zip(self.slabs, split(P, self.w, self.nslabs)):
            sim.set_particles(part["pos"], part["vel"], part["pid"], next_pid=nxt)
        return self

    def _admit(self):
        if not self._admitted:
            for sim in self.slabs:
                rc = self.batch.admit(sim)
                if rc != U.OK:
                    raise U.UspError(rc, "usp_batch_admit")
            self._admitted = True

    def _retire(self):
        if self._admitted:
            for sim in self.slabs:
                self.batch.retire(sim)
            self._admitted = False

    def step(self, n: int = 1):
        self._admit()
        self.batch.step(n)
        return self

    def sample(self, averaged: bool = False) -> np.ndarray:
        """Fields of the whole domain, [field][global cell]."""
        return np.concatenate([s.sample(averaged=averaged) for s in self.slabs], axis=1)

    def particles(self) -> dict:
        """The whole domain's particles (pending relaxation applied), cells as
        global ids."""
        self._retire()
        parts = [s.particles() for s in self.slabs]
        return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}

    def n_particles(self) -> int:
        return sum(s.info()["n_particles"] for s in self.slabs)

    def counters(self) -> np.ndarray:
        return np.sum([s.info()["counters"] for s in self.slabs], axis=0)

    def close(self):
        self._retire()
        self.batch.close()
        for s in self.slabs:
            s.close()


# --------------------------------------------------------------------------
# Host-side exchange between ranks that each own one slab (the protocol a
# multi-device run uses between steps; here exercised on CPU ranks).
# --------------------------------------------------------------------------
def exchange_particles(P: dict, w: dict, nslabs: int, rank: int, dist) -> dict:
    """Send every particle of this rank that now lies in another slab to its
    owner and receive the ones that entered this slab.  P: local particles
    (pos, vel, pid); returns the particles this rank owns afterwards, in
    (kept in order, then received by source rank) order."""
    own = owner_rows(P["pos"], w, nslabs)
    out = [{k: P[k][own == r] for k in ("pos", "vel", "pid")} for r in range(nslabs)]
    gathered = [None] * nslabs
    dist.all_gather_object(gathered, out)
    keep = out[rank]
    recv = [gathered[src][rank] for src in range(nslabs) if src != rank]
    return {k: np.concatenate([keep[k]] + [r[k] for r in recv]) for k in ("pos", "vel", "pid")}


def exchange_halo(rows: np.ndarray, rank: int, nslabs: int, dist, periodic: bool = False):
    """Per-cell values of this slab's rows ([rows][...]): returns the row just
    below the slab and the row just above it from the neighbouring ranks (None
    at a non-periodic domain edge) -- the stencil input of Eq. 18 across a
    slab boundary."""
    gathered = [None] * nslabs
    dist.all_gather_object(gathered, (rows[0], rows[-1]))
    below = rank - 1
    above = rank + 1
    if periodic:
        below %= nslabs
        above %= nslabs
    lo = gathered[below][1] if 0 <= below < nslabs else None
    hi = gathered[above][0] if 0 <= above < nslabs else None
    return lo, hi
