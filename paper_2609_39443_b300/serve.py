"""Continuous-batching server of coupling steps: the scheduling side.

Many simulations send coupling-step requests (new actuator-point positions
for their next step) as they arrive.  The library's server (al_server_*)
keeps each admitted simulation resident on the device, advances every
resident simulation whose next request has arrived in one batched launch
sequence (a wave, over al_batch_run_subset), alternates waves between two
streams so that one forms while the previous one runs, and moves each
wave's positions and forces in one host-to-device and one device-to-host
copy.  What stays here is scheduling: arrivals, admission in arrival order
by device bytes (the library's al_footprint of the instance plus the
simulation's own buffers, one allocation each), release of finished
simulations, and latency / throughput statistics.

`PlainServer` is the reference path: one al_sample_drag_spread per request
in arrival order on one stream, with the same admission rule.

Every device operation goes through a backend (`CudaBackend`), so the
scheduling can be checked on the host with a stand-in.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

PAGE = 2 << 20          # the driver commits device memory in 2 MiB pages


def _pages(nbytes: int) -> int:
    return -(-int(nbytes) // PAGE) * PAGE


@dataclass
class Sim:
    """One client simulation: its initial workload and step count.  Request
    k carries positions P0 + k dt V, a smooth synthetic beam motion: each
    line bends about its first node, V at a node being the line's mean Pdot
    times the node's arc length from the first node over the line's length
    (a beam solver hands back smooth centrelines; moving every node by its
    own random velocity would crumple the lines instead)."""
    wl: object
    n_steps: int
    dt: float = 1e-3
    _V: Optional[np.ndarray] = field(default=None, init=False, repr=False)
    _P0: Optional[np.ndarray] = field(default=None, init=False, repr=False)

    @property
    def n_points(self) -> int:
        return int(self.wl.beams.n_points)

    def dtype(self):
        return np.float64 if self.wl.grid.precision == "fp64" else np.float32

    def buffer_bytes(self) -> int:
        """Device bytes of the simulation's own buffers (fields, points,
        outputs) in their one allocation."""
        g, b = self.wl.grid, self.wl.beams
        es = 8 if g.precision == "fp64" else 4
        n = (6 + (1 if g.has_alpha else 0)) * g.n_cells + 9 * max(b.n_points, 1)     # U, S, alpha; P, Pdot, F
        return _pages(es * n + 6 * 8 + 16 * 4 + 4096)

    def velocity(self) -> np.ndarray:
        """V (3, N_p): the smooth motion of the requests' positions."""
        if self._V is None:
            P = np.asarray(self.wl.step.P, dtype=np.float64)
            Pd = np.asarray(self.wl.step.Pdot, dtype=np.float64)
            off = np.asarray(self.wl.beams.line_off, dtype=np.int64)
            cnt = np.diff(off)
            nl, n = len(cnt), P.shape[1]
            line = np.repeat(np.arange(nl), cnt)                      # the line of every node
            mean = np.stack([np.bincount(line, weights=Pd[c], minlength=nl) for c in range(3)])
            mean /= np.maximum(cnt, 1)[None, :]
            # arc length from the line's first node: a running sum over all
            # nodes of the segment lengths inside lines, less its value there
            ds = np.linalg.norm(np.diff(P, axis=1), axis=0) if n > 1 else np.zeros(0)
            ds = ds * (line[1:] == line[:-1])
            run = np.concatenate([[0.0], np.cumsum(ds)])
            first = off[:-1][line]
            s = run - run[first]
            last = np.maximum(off[1:] - 1, off[:-1])
            length = (run[np.minimum(last, max(n - 1, 0))] - run[np.minimum(off[:-1], max(n - 1, 0))])[line] \
                if n else np.zeros(0)
            frac = np.where(cnt[line] < 2, 1.0, s / np.maximum(length, 1e-300))
            self._V = mean[:, line] * frac[None, :]
        return self._V

    def positions(self, k: int) -> np.ndarray:
        """P0 + k dt V, evaluated in the simulation's precision."""
        if self._P0 is None:
            self._P0 = np.ascontiguousarray(self.wl.step.P, dtype=self.dtype())
            self._V = np.ascontiguousarray(self.velocity(), dtype=self.dtype())
        return self._P0 + self.dtype()(k * self.dt) * self._V


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


def instance_footprint(sim: Sim) -> int:
    """al_footprint of the simulation's instance (one is created and destroyed)."""
    from .al import Grid
    g = Grid(sim.wl.grid)
    try:
        g.load_beams(sim.wl.beams)
        return g.footprint()
    finally:
        g.close()


class _Buffers:
    """One simulation's device buffers in one cudaMalloc of whole pages (so
    the bytes declared at admission are the bytes the device gives up): U,
    S, alpha (fields), P, Pdot, F (points), totals and status."""

    def __init__(self, sim: Sim, device):
        from cuda.bindings import runtime as cudart
        from .al import AL_STATUS_N, StepIn, StepOut
        self._rt = cudart
        wl = sim.wl
        es = 8 if wl.grid.precision == "fp64" else 4
        dt = np.float64 if es == 8 else np.float32
        nc, npts = int(wl.grid.n_cells), max(int(wl.beams.n_points), 1)
        self.nbytes = sim.buffer_bytes()
        self.nc, self.es, self.dt = nc, es, dt
        err, base = cudart.cudaMalloc(self.nbytes)
        if err != cudart.cudaError_t.cudaSuccess:
            raise MemoryError(f"cudaMalloc({self.nbytes}): {err}")
        self.base = int(base)
        off = [0]

        def take(nbytes):
            o = (off[0] + 255) // 256 * 256
            off[0] = o + nbytes
            return self.base + o

        U = [take(nc * es) for _ in range(3)]
        self.S = [take(nc * es) for _ in range(3)]
        alpha = take(nc * es) if wl.grid.has_alpha else None
        P = [take(npts * es) for _ in range(3)]
        Pdot = [take(npts * es) for _ in range(3)]
        F = [take(npts * es) for _ in range(3)]
        totals, status = take(6 * 8), take(AL_STATUS_N * 4)
        assert off[0] <= self.nbytes
        st = wl.step
        for a in range(3):
            self._put(U[a], st.U[a], dt)
            if wl.beams.n_points:
                self._put(P[a], st.P[a], dt)
                self._put(Pdot[a], st.Pdot[a], dt)
        if alpha is not None:
            self._put(alpha, st.alpha, dt)
        cudart.cudaMemset(totals, 0, 6 * 8)
        cudart.cudaMemset(status, 0, AL_STATUS_N * 4)
        self.sin, self.sout = StepIn(), StepOut()
        for a in range(3):
            self.sin.U[a], self.sin.P[a], self.sin.Pdot[a] = U[a], P[a], Pdot[a]
            self.sout.S[a], self.sout.F[a] = self.S[a], F[a]
        self.sin.alpha = alpha
        import ctypes as C
        self.sout.totals = C.cast(C.c_void_p(totals), C.POINTER(C.c_double))
        self.sout.status = C.cast(C.c_void_p(status), C.POINTER(C.c_int))

    def _put(self, dst, host, dt):
        h = np.ascontiguousarray(host, dtype=dt)
        err, = self._rt.cudaMemcpy(dst, h.ctypes.data, h.nbytes, self._rt.cudaMemcpyKind.cudaMemcpyHostToDevice)
        if err != self._rt.cudaError_t.cudaSuccess:
            raise RuntimeError(f"cudaMemcpy: {err}")

    def S_host(self) -> np.ndarray:
        out = np.empty((3, self.nc), dtype=self.dt)
        for a in range(3):
            self._rt.cudaMemcpy(out[a].ctypes.data, self.S[a], self.nc * self.es,
                                self._rt.cudaMemcpyKind.cudaMemcpyDeviceToHost)
        return out

    def __del__(self):
        if getattr(self, "base", 0):
            self._rt.cudaFree(self.base)
            self.base = 0


class CudaBackend:
    """Device side of the servers: the library's server with each
    simulation's buffers, and the resident instances of the plain path."""

    def __init__(self, device="cuda"):
        self.device = device

    def server(self, budget, max_sims, max_wave, max_points, precision):
        from .al import Server
        return Server(budget, max_sims, max_wave, max_points, precision)

    def buffers(self, sim: Sim):
        return _Buffers(sim, self.device)

    def final_S(self, buffers) -> np.ndarray:
        return buffers.S_host()

    def resident(self, sim: Sim):
        return _Resident(sim, self.device)

    def stream(self):
        import torch
        return torch.cuda.Stream(device=self.device)

    def stream_ctx(self, stream):
        import torch
        return torch.cuda.stream(stream)

    @staticmethod
    def sync(stream) -> None:
        stream.synchronize()


class _Resident:
    """The plain path's simulation: an instance stepped alone."""

    def __init__(self, sim: Sim, device):
        import torch
        from .al import Instance
        self.sim = sim
        self.inst = Instance(sim.wl, device=device)
        dt = self.inst.dtype
        self.hP = torch.empty(self.inst.P.shape, dtype=dt).pin_memory()
        self.hF = torch.empty(self.inst.F.shape, dtype=dt).pin_memory()

    def footprint(self) -> int:
        i = self.inst
        own = sum(t.numel() * t.element_size() for t in (i.U, i.P, i.Pdot, i.S, i.F, i.totals, i.status)
                  + ((i.alpha,) if i.alpha is not None else ()))
        return self.inst.grid.footprint() + _pages(own)

    def upload(self, k: int) -> None:
        np.copyto(self.hP.numpy(), self.sim.positions(k), casting="same_kind")
        self.inst.P.copy_(self.hP, non_blocking=True)

    def download(self) -> None:
        self.hF.copy_(self.inst.F, non_blocking=True)

    def step(self, stream) -> None:
        self.inst.step(stream=stream)

    def result_F(self) -> np.ndarray:
        return self.hF.numpy()[:, :self.sim.n_points].copy()

    def result_S(self) -> np.ndarray:
        return self.inst.S.cpu().numpy().copy()

    def close(self) -> None:
        self.inst.close()


class BatchServer:
    """Continuous batching through the library's server: this side admits
    simulations in arrival order, submits each arrived request, polls for
    completions and releases finished simulations."""

    def __init__(self, sims: List[Sim], hbm_budget: int, *, n_slots: int = 64, max_wave: int = 64, backend=None,
                 record: bool = False, preadmit: bool = False):
        self.sims = sims
        self.preadmit = preadmit          # admit (in order of first arrival) before the clock starts
        self.budget = int(hbm_budget)
        self.n_slots = int(n_slots)
        self.max_wave = min(int(max_wave), self.n_slots)
        self.be = backend if backend is not None else CudaBackend()
        self.record = record
        self.stats = Stats()
        self.results: Dict[Tuple[int, int], np.ndarray] = {}     # (sim, step) -> F
        self.final_S: Dict[int, np.ndarray] = {}

    def run(self, arrivals):
        st = self.stats
        sims = self.sims
        pts = sorted(max(s.n_points, 1) for s in sims)
        wave_points = max(pts[-1], min(sum(pts[-self.max_wave:]), 1 << 22))     # staging of one wave
        srv = self.be.server(self.budget, self.n_slots, self.max_wave, wave_points, sims[0].wl.grid.precision)
        n_req = len(arrivals)
        slot: Dict[int, int] = {}                 # simulation -> server slot
        bufs: Dict[int, object] = {}
        waiting: Dict[int, deque] = {}            # arrived before admission: (step, arrival)
        adm_queue: deque = deque()
        inflight: Dict[int, tuple] = {}           # tag -> (sim, step, arrival, P, F)
        done_steps = [0] * len(sims)
        releases, refused_at = 0, -1              # admission is retried after each release
        ai = 0
        if self.preadmit:                         # a warm server: simulations resident before requests
            for _, s, _ in arrivals:
                if s in slot or s in waiting:
                    continue
                used, resident = srv.footprint()
                if resident >= self.n_slots or (resident and used + sims[s].buffer_bytes() > self.budget):
                    break
                b = self.be.buffers(sims[s])
                q = srv.admit(sims[s].wl.grid, sims[s].wl.beams, b.sin, b.sout, b.nbytes)
                if q is None:
                    break
                slot[s], bufs[s] = q, b
                st.admitted += 1
                sims[s].positions(0)              # the client's motion, ready before the clock too
            st.peak_mem = srv.footprint()[0]
        t0 = time.perf_counter()

        def submit(s, k, ta):
            tag = s * 1_000_000 + k
            P = sims[s].positions(k)
            F = np.empty_like(P)
            inflight[tag] = (s, k, ta, P, F)
            srv.submit(slot[s], P, F, tag)

        while st.completed < n_req:
            now = time.perf_counter() - t0
            while ai < n_req and arrivals[ai][0] <= now:
                t, s, k = arrivals[ai]
                ai += 1
                if s in slot:
                    submit(s, k, t)
                else:
                    if s not in waiting:
                        waiting[s] = deque()
                        adm_queue.append(s)
                    waiting[s].append((k, t))
            # admissions in arrival order; after a refusal the head waits for a release
            while adm_queue and refused_at != releases:
                s = adm_queue[0]
                used, resident = srv.footprint()
                if resident >= self.n_slots or (resident and used + sims[s].buffer_bytes() > self.budget):
                    refused_at = releases
                    break
                b = self.be.buffers(sims[s])
                q = srv.admit(sims[s].wl.grid, sims[s].wl.beams, b.sin, b.sout, b.nbytes)
                if q is None:
                    del b
                    refused_at = releases
                    break
                adm_queue.popleft()
                slot[s], bufs[s] = q, b
                st.admitted += 1
                st.peak_mem = max(st.peak_mem, srv.footprint()[0])
                for k, t in waiting.pop(s):
                    submit(s, k, t)
            # completions (waiting for the oldest wave when nothing else can happen)
            idle = (not adm_queue or refused_at == releases) and \
                (ai >= n_req or arrivals[ai][0] > time.perf_counter() - t0 + 2e-4)
            tags = srv.poll(wait=bool(inflight) and idle)
            now = time.perf_counter() - t0
            for tag in tags:
                s, k, ta, P, F = inflight.pop(tag)
                st.latencies.append(now - ta)
                st.completed += 1
                done_steps[s] += 1
                if self.record:
                    self.results[(s, k)] = F[:, :sims[s].n_points]
                if done_steps[s] == sims[s].n_steps:
                    if self.record:
                        self.final_S[s] = self.be.final_S(bufs[s])
                    srv.release(slot.pop(s))
                    del bufs[s]
                    releases += 1
            if not tags and not inflight and ai < n_req and not adm_queue:
                time.sleep(max(0.0, min(1e-4, arrivals[ai][0] - (time.perf_counter() - t0))))
        st.wall = time.perf_counter() - t0
        st.waves, steps = srv.waves()
        st.wave_sizes = [steps / max(st.waves, 1)]
        srv.close()
        return st


class PlainServer:
    """Reference path: one al_sample_drag_spread per request on one stream,
    the oldest processable request first, with the same admission rule."""

    def __init__(self, sims: List[Sim], hbm_budget: int, backend=None, record: bool = False,
                 preadmit: bool = False):
        self.sims = sims
        self.preadmit = preadmit
        self.budget = int(hbm_budget)
        self.be = backend if backend is not None else CudaBackend()
        self.record = record
        self.stats = Stats()
        self.mem = 0
        self.res: Dict[int, object] = {}
        self.fp: Dict[int, int] = {}
        self.done_steps = [0] * len(sims)
        self.results: Dict[Tuple[int, int], np.ndarray] = {}
        self.final_S: Dict[int, np.ndarray] = {}

    def _admit(self, s: int) -> bool:
        r = self.be.resident(self.sims[s])
        fp = r.footprint()
        if self.res and self.mem + fp > self.budget:
            r.close()
            return False
        self.res[s], self.fp[s] = r, fp
        self.mem += fp
        self.stats.admitted += 1
        self.stats.peak_mem = max(self.stats.peak_mem, self.mem)
        return True

    def run(self, arrivals):
        st = self.stats
        n_req = len(arrivals)
        ai = 0
        queue = []                        # arrived, not yet processed (arrival order)
        stream = self.be.stream()
        if self.preadmit:
            for _, s, _ in arrivals:
                if s not in self.res:
                    if not self._admit(s):
                        break
                    self.sims[s].positions(0)     # the client's motion, ready before the clock too
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
            st.latencies.append(time.perf_counter() - t0 - t)
            st.completed += 1
            if self.record:
                self.results[(s, k)] = r.result_F()
            self.done_steps[s] += 1
            if self.done_steps[s] == self.sims[s].n_steps:
                if self.record:
                    self.final_S[s] = r.result_S()
                self.res.pop(s).close()
                self.mem -= self.fp.pop(s)
        st.wall = time.perf_counter() - t0
        for s in list(self.res):
            self.res.pop(s).close()
        return st
