"""Continuous-batching server of coupling steps.

Many simulations send coupling-step requests (new actuator-point positions
for their next step) as they arrive.  The server keeps each admitted
simulation's grid, fields, bins and relaxation state resident on the device,
admits simulations by their HBM footprint under a budget, and advances every
simulation whose next request has arrived in one batched launch sequence
(al_batch_run_subset) -- a *wave*.  Waves alternate between CUDA streams, so a
wave forms and launches while earlier ones are still running; a simulation
with a step in flight waits for it (steps of one simulation are ordered).
Evicted simulations free their slot and memory for waiting ones.

`PlainServer` is the reference path: one al_sample_drag_spread per request
in arrival order on one stream, with the same copies and admission.

The schedulers only decide what runs when; every device operation goes
through a backend (`CudaBackend`: PyTorch memory and streams plus the CUDA
library), so the scheduling can be checked on the host with a stand-in.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np


@dataclass
class Sim:
    """One client simulation: its initial workload and step count.  Request
    k carries positions P0 + k dt Pdot (the synthetic beam motion)."""
    wl: object
    n_steps: int
    dt: float = 1e-3

    def footprint(self) -> int:
        g, b = self.wl.grid, self.wl.beams
        es = 8 if g.precision == "fp64" else 4
        fields = (3 + 3 + (1 if g.has_alpha else 0)) * es * g.n_cells          # U, S, alpha
        points = b.n_points * (es * 3 * 5 + 120)                                 # P, Pdot, F, staging + scratch
        bricks = ((g.nx + 15) // 16) * ((g.ny + 15) // 16) * ((g.nz + 3) // 4)   # lowest brick height
        mask = bricks * ((b.n_lines + 31) // 32) * 4 + bricks * 24
        return int(fields + points + mask + 4096)

    def positions(self, k: int) -> np.ndarray:
        return self.wl.step.P.astype(np.float64) + (k * self.dt) * self.wl.step.Pdot.astype(np.float64)


@dataclass
class Stats:
    latencies: List[float] = field(default_factory=list)
    completed: int = 0
    waves: int = 0
    wave_sizes: List[int] = field(default_factory=list)
    admitted: int = 0
    peak_mem: int = 0
    wall: float = 0.0

    def summary(self):
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"completed": self.completed, "steps_per_s": self.completed / max(self.wall, 1e-12),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_wave": float(np.mean(self.wave_sizes)) if self.wave_sizes else 0.0,
                "waves": self.waves, "admitted": self.admitted, "peak_resident_bytes": self.peak_mem,
                "wall_s": self.wall}


def poisson_arrivals(sims: List[Sim], rate: float, seed: int):
    """Request stream: every simulation issues its n_steps requests; the
    inter-arrival times of the merged stream are exponential with mean 1/rate
    and each arrival belongs to a simulation drawn at random among those with
    requests left (so per-simulation order is kept)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    left = np.array([s.n_steps for s in sims])
    nxt = np.zeros(len(sims), dtype=np.int64)
    total = int(left.sum())
    t = np.cumsum(rng.exponential(1.0 / rate, size=total))
    out = []
    for a in range(total):
        live = np.flatnonzero(left)
        s = int(live[rng.integers(len(live))])
        out.append((float(t[a]), s, int(nxt[s])))
        nxt[s] += 1
        left[s] -= 1
    return out


class CudaBackend:
    """Device side of the servers: resident instances with pinned staging
    buffers, the slot batch, streams and events."""

    def __init__(self, device="cuda"):
        self.device = device

    def stream(self):
        import torch
        return torch.cuda.Stream(device=self.device)

    def resident(self, sim: Sim):
        return _Resident(sim, self.device)

    def batch(self, n_slots: int, precision: str):
        from .al import Batch
        return Batch([], use_graph=False, reserve=(n_slots, precision))

    def stream_ctx(self, stream):
        import torch
        return torch.cuda.stream(stream)

    def mark(self, stream):
        import torch
        ev = torch.cuda.Event()
        ev.record(stream)
        return ev

    @staticmethod
    def done(ev) -> bool:
        return ev.query()

    @staticmethod
    def sync(stream) -> None:
        stream.synchronize()

    def sync_all(self) -> None:
        import torch
        torch.cuda.synchronize()


class _Resident:
    def __init__(self, sim: Sim, device):
        import torch
        from .al import Instance
        self.sim = sim
        self.inst = Instance(sim.wl, device=device)
        dt = self.inst.dtype
        self.hP = torch.empty(self.inst.P.shape, dtype=dt).pin_memory()
        self.hF = torch.empty(self.inst.F.shape, dtype=dt).pin_memory()

    def upload(self, k: int) -> None:
        # positions of step k into pinned host memory (the client's payload), then to the device
        np.copyto(self.hP.numpy(), self.sim.positions(k), casting="same_kind")
        self.inst.P.copy_(self.hP, non_blocking=True)

    def download(self) -> None:
        self.hF.copy_(self.inst.F, non_blocking=True)

    def step(self, stream) -> None:
        self.inst.step(stream=stream)

    def result_F(self) -> np.ndarray:
        return self.hF.numpy()[:, :self.sim.wl.beams.n_points].copy()

    def result_S(self) -> np.ndarray:
        return self.inst.S.cpu().numpy().copy()

    def close(self) -> None:
        self.inst.close()


class _Base:
    def __init__(self, sims: List[Sim], hbm_budget: int, backend=None, record: bool = False):
        self.sims = sims
        self.budget = int(hbm_budget)
        self.be = backend if backend is not None else CudaBackend()
        self.stats = Stats()
        self.mem = 0
        self.res: Dict[int, object] = {}
        self.done_steps = [0] * len(sims)
        self.busy = [False] * len(sims)
        self.record = record
        self.results: Dict[Tuple[int, int], np.ndarray] = {}     # (sim, step) -> F
        self.final_S: Dict[int, np.ndarray] = {}

    def _fits(self, s: int) -> bool:
        return self.mem + self.sims[s].footprint() <= self.budget or not self.res

    def _admit(self, s: int) -> bool:
        if not self._fits(s):
            return False
        self.res[s] = self.be.resident(self.sims[s])
        self.mem += self.sims[s].footprint()
        self.stats.admitted += 1
        self.stats.peak_mem = max(self.stats.peak_mem, self.mem)
        return True

    def _evict(self, s: int):
        r = self.res.pop(s)
        r.close()
        self.mem -= self.sims[s].footprint()

    def _finish(self, s: int, k: int, t_arrival: float, now: float):
        st = self.stats
        st.latencies.append(now - t_arrival)
        st.completed += 1
        r = self.res[s]
        if self.record:
            self.results[(s, k)] = r.result_F()
        self.busy[s] = False
        self.done_steps[s] += 1
        if self.done_steps[s] == self.sims[s].n_steps:
            if self.record:
                self.final_S[s] = r.result_S()
            return True
        return False


class BatchServer(_Base):
    """Continuous batching over al_batch_run_subset."""

    def __init__(self, sims, hbm_budget, *, n_slots=64, n_streams=2, max_wave=64, backend=None, record=False):
        super().__init__(sims, hbm_budget, backend, record)
        prec = sims[0].wl.grid.precision
        self.batch = self.be.batch(n_slots, prec)
        self.free_slots = deque(range(n_slots))
        self.slot_of: Dict[int, int] = {}
        self.streams = [self.be.stream() for _ in range(n_streams)]
        self.max_wave = max_wave
        self.inflight = deque()           # (event, stream index, [(sim, step, t_arrival)])

    def _admit(self, s):
        if not self.free_slots or not super()._admit(s):
            return False
        slot = self.free_slots.popleft()
        self.slot_of[s] = slot
        # bind the slot and wait, so every stream sees the new descriptor
        self.batch.assign(slot, self.res[s].inst, stream=self.streams[0])
        self.be.sync(self.streams[0])
        return True

    def _evict(self, s):
        slot = self.slot_of.pop(s)
        self.batch.assign(slot, None, stream=self.streams[0])
        self.be.sync(self.streams[0])
        super()._evict(s)
        self.free_slots.append(slot)

    def run(self, arrivals):
        st = self.stats
        n_req = len(arrivals)
        pending = [deque() for _ in self.sims]
        wait_adm, queued = deque(), set()
        ai = 0
        t0 = time.perf_counter()
        busy_streams = set()
        while st.completed < n_req:
            now = time.perf_counter() - t0
            while ai < n_req and arrivals[ai][0] <= now:
                t, s, k = arrivals[ai]
                pending[s].append((k, t))
                if s not in self.res and s not in queued:
                    wait_adm.append(s)
                    queued.add(s)
                ai += 1
            # retire finished waves
            while self.inflight and self.be.done(self.inflight[0][0]):
                ev, si, items = self.inflight.popleft()
                busy_streams.discard(si)
                done = time.perf_counter() - t0
                for s, k, ta in items:
                    if self._finish(s, k, ta, done):
                        self._evict(s)
            # admissions in arrival order
            while wait_adm:
                s = wait_adm[0]
                if not self._admit(s):
                    break
                wait_adm.popleft()
                queued.discard(s)
            # form and launch a wave: every resident simulation whose next step has arrived
            free = [i for i in range(len(self.streams)) if i not in busy_streams]
            if free:
                wave = []
                for s in self.res:
                    if not self.busy[s] and pending[s] and pending[s][0][0] == self.done_steps[s]:
                        wave.append(s)
                        if len(wave) >= self.max_wave:
                            break
                if wave:
                    si = free[0]
                    stream = self.streams[si]
                    items = []
                    with self.be.stream_ctx(stream):
                        for s in wave:
                            k, ta = pending[s].popleft()
                            self.res[s].upload(k)
                            self.busy[s] = True
                            items.append((s, k, ta))
                        self.batch.run_subset([self.slot_of[s] for s in wave], stream=stream)
                        for s in wave:
                            self.res[s].download()
                        ev = self.be.mark(stream)
                    self.inflight.append((ev, si, items))
                    busy_streams.add(si)
                    st.waves += 1
                    st.wave_sizes.append(len(wave))
                    continue
            if ai < n_req and not self.inflight:
                time.sleep(max(0.0, min(1e-4, arrivals[ai][0] - now)))
        self.be.sync_all()
        st.wall = time.perf_counter() - t0
        for s in list(self.res):
            self._evict(s)
        self.batch.close()
        return st


class PlainServer(_Base):
    """Reference path: one al_sample_drag_spread per request on one stream,
    the oldest processable request first, with the same admission rule."""

    def run(self, arrivals):
        st = self.stats
        n_req = len(arrivals)
        ai = 0
        queue = []                        # arrived, not yet processed (arrival order)
        stream = self.be.stream()
        t0 = time.perf_counter()
        while st.completed < n_req:
            now = time.perf_counter() - t0
            while ai < n_req and arrivals[ai][0] <= now:
                queue.append(arrivals[ai])
                ai += 1
            pick = None
            for qi, (t, s, k) in enumerate(queue):
                if s in self.res:
                    if self.done_steps[s] == k:
                        pick = qi
                        break
                elif self._admit(s):
                    pick = qi
                    break
            if pick is None:
                if ai < n_req:
                    time.sleep(max(0.0, min(1e-4, arrivals[ai][0] - now)))
                continue
            t, s, k = queue.pop(pick)
            r = self.res[s]
            with self.be.stream_ctx(stream):
                r.upload(k)
                r.step(stream)
                r.download()
            self.be.sync(stream)
            st.waves += 1
            st.wave_sizes.append(1)
            if self._finish(s, k, t, time.perf_counter() - t0):
                self._evict(s)
        st.wall = time.perf_counter() - t0
        for s in list(self.res):
            self._evict(s)
        return st
