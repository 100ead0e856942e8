"""Host logic of the continuous-batching server, with a stand-in for the
library's server (no GPU): every request completes once, each simulation's
steps run in order and never two at a time, no wave holds a simulation
twice, resident device bytes never exceed the budget, admission follows
arrival order, and slots are reused after release."""
import numpy as np
import pytest

from paper_2609_39443_b300 import workloads as W
from paper_2609_39443_b300.serve import BatchServer, PlainServer, Sim, poisson_arrivals

LIB = 3 << 20                       # the stand-in's library bytes per simulation


class _Bufs:
    def __init__(self, sim):
        self.nbytes = sim.buffer_bytes()
        self.sin = self.sout = self
        self.steps = 0


class FakeServer:
    """The semantics of al_server_*: slots, a budget on declared bytes, one
    step per simulation in flight, waves on two streams that complete after
    a few polls (or at once when waited for)."""

    def __init__(self, budget, max_sims, max_wave, max_points, precision, polls=2):
        self.budget, self.max_sims, self.max_wave, self.polls = budget, max_sims, max_wave, polls
        self.slots = [None] * max_sims
        self.used = 0
        self.inflight = []                    # waves: [countdown, [(slot, tag, F)]]
        self.done = []
        self.n_waves = self.n_steps = 0
        self.peak = 0
        self.wave_log = []

    def admit(self, grid, beams, sin, sout, nbytes):
        free = [i for i, x in enumerate(self.slots) if x is None]
        if not free or self.used + nbytes + LIB > self.budget:
            return None
        q = free[0]
        self.slots[q] = {"buf": sin, "bytes": nbytes + LIB, "queue": [], "busy": False}
        self.used += nbytes + LIB
        self.peak = max(self.peak, self.used)
        return q

    def submit(self, q, P, F, tag):
        assert self.slots[q] is not None, "submit to a free slot"
        self.slots[q]["queue"].append((tag, F))

    def _retire(self, w):
        for q, tag, F in w[1]:
            m = self.slots[q]
            F[...] = m["buf"].steps                  # the step this request ran as
            m["buf"].steps += 1
            m["busy"] = False
            self.done.append(tag)

    def poll(self, wait=False):
        for w in list(self.inflight):
            w[0] -= 1
            if w[0] < 0:
                self.inflight.remove(w)
                self._retire(w)
        while len(self.inflight) < 2:
            items = []
            for q, m in enumerate(self.slots):
                if m is not None and not m["busy"] and m["queue"] and len(items) < self.max_wave:
                    tag, F = m["queue"].pop(0)
                    m["busy"] = True
                    items.append((q, tag, F))
            if not items:
                break
            assert len({q for q, _, _ in items}) == len(items), "a simulation twice in one wave"
            self.inflight.append([self.polls, items])
            self.wave_log.append([q for q, _, _ in items])
            self.n_waves += 1
            self.n_steps += len(items)
        if wait and not self.done and self.inflight:
            self._retire(self.inflight.pop(0))
        out, self.done = self.done, []
        return out

    def release(self, q):
        m = self.slots[q]
        assert not m["queue"] and not m["busy"], "release with work left"
        self.used -= m["bytes"]
        self.slots[q] = None

    def footprint(self):
        return self.used, sum(m is not None for m in self.slots)

    def waves(self):
        return self.n_waves, self.n_steps

    def close(self):
        assert all(m is None for m in self.slots), "simulations left resident"


class _Res:
    def __init__(self, sim):
        self.sim = sim
        self.next_k, self.staged, self.in_flight = 0, None, False

    def footprint(self):
        return self.sim.buffer_bytes() + LIB

    def upload(self, k):
        assert not self.in_flight and k == self.next_k, (k, self.next_k)
        self.staged, self.in_flight = k, True

    def step(self, stream):
        self.next_k += 1
        self.in_flight = False

    def download(self):
        pass

    def result_F(self):
        return np.array([self.staged])

    def result_S(self):
        return np.array([self.next_k])

    def close(self):
        pass


class _Ctx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


class FakeBackend:
    def __init__(self):
        self.servers = []

    def server(self, budget, max_sims, max_wave, max_points, precision):
        s = FakeServer(budget, max_sims, max_wave, max_points, precision)
        self.servers.append(s)
        return s

    def buffers(self, sim):
        return _Bufs(sim)

    def final_S(self, b):
        return np.array([b.steps])

    def resident(self, sim):
        return _Res(sim)

    def stream(self):
        return object()

    def stream_ctx(self, stream):
        return _Ctx()

    @staticmethod
    def sync(stream):
        pass


def _sims(n=12, steps=5):
    wls = [W.make_random(100 + i, 20 + 4 * (i % 3), 16, 12, n_lines=1 + i % 3, kinds=("stem",)) for i in range(n)]
    return [Sim(w, steps) for w in wls]


@pytest.mark.parametrize("rate", [300.0, 50000.0])
@pytest.mark.parametrize("server", ["batched", "plain"])
def test_scheduler_invariants(server, rate):
    sims = _sims()
    budget = 3 * max(s.buffer_bytes() + LIB for s in sims)          # about three resident at a time
    arr = poisson_arrivals(sims, rate, seed=7)
    be = FakeBackend()
    if server == "batched":
        srv = BatchServer(sims, budget, n_slots=4, backend=be, record=True)
    else:
        srv = PlainServer(sims, budget, backend=be, record=True)
    st = srv.run(arr)
    assert st.completed == len(arr) == sum(s.n_steps for s in sims)
    assert sorted(srv.results) == sorted((s, k) for s in range(len(sims)) for k in range(sims[s].n_steps))
    for (s, k), v in srv.results.items():
        assert int(np.ravel(v)[0]) == k                     # each request ran as its own step, in order
    assert all(int(srv.final_S[s][0]) == sims[s].n_steps for s in range(len(sims)))
    assert st.peak_mem <= budget
    assert st.admitted == len(sims)
    assert len(st.latencies) == len(arr) and min(st.latencies) >= 0.0
    if server == "batched":
        fs = be.servers[0]
        assert fs.peak <= budget
        assert sum(len(w) for w in fs.wave_log) == len(arr)
        assert st.waves == len(fs.wave_log)
    else:
        assert not srv.res                                   # everything released at the end


def test_admission_follows_arrival_order():
    """With room for one simulation at a time, simulations are admitted in
    the order of their first arrivals."""
    sims = _sims(6, 3)
    budget = max(s.buffer_bytes() + LIB for s in sims)
    arr = poisson_arrivals(sims, 2000.0, seed=5)
    first = []
    for _, s, _ in arr:
        if s not in first:
            first.append(s)
    be = FakeBackend()
    srv = BatchServer(sims, budget, n_slots=2, backend=be, record=True)
    order = []
    orig = FakeServer.admit

    def spy(self, grid, beams, sin, sout, nbytes):
        q = orig(self, grid, beams, sin, sout, nbytes)
        if q is not None:
            order.append(next(i for i, x in enumerate(sims) if x.wl.grid is grid))
        return q

    FakeServer.admit = spy
    try:
        srv.run(arr)
    finally:
        FakeServer.admit = orig
    assert order == first


def test_poisson_arrivals_keep_per_simulation_order():
    sims = _sims(5, 7)
    arr = poisson_arrivals(sims, 1000.0, seed=3)
    assert len(arr) == 35
    assert all(a[0] <= b[0] for a, b in zip(arr, arr[1:]))
    for s in range(5):
        ks = [k for _, ss, k in arr if ss == s]
        assert ks == list(range(7))


def _motion_by_line(wl):
    """The served motion written out line by line: V = the line's mean Pdot
    times the node's arc length from the first node over the line's length
    (a line of one node moves with its own Pdot)."""
    P = np.asarray(wl.step.P, dtype=np.float64)
    Pd = np.asarray(wl.step.Pdot, dtype=np.float64)
    off = wl.beams.line_off
    V = np.zeros_like(P)
    for l in range(len(off) - 1):
        a, b = int(off[l]), int(off[l + 1])
        mean = Pd[:, a:b].mean(axis=1, keepdims=True) if b > a else None
        if b - a == 1:
            V[:, a:b] = mean
        elif b - a > 1:
            s = [0.0]
            for i in range(a + 1, b):
                s.append(s[-1] + float(np.linalg.norm(P[:, i] - P[:, i - 1])))
            V[:, a:b] = mean * (np.array(s) / max(s[-1], 1e-300))[None, :]
    return V


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_served_motion_matches_its_definition(seed):
    # stems, arcs, random walks, single points and repeated nodes
    wl = W.make_random(seed, 20, 16, 12, n_lines=7, kinds=("stem", "arc", "random", "point", "dup"))
    sim = Sim(wl, 3)
    V = sim.velocity()
    ref = _motion_by_line(wl)
    assert np.abs(V - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300)
    # every line's first node stays put unless the line is a single point
    off = wl.beams.line_off
    for l in range(len(off) - 1):
        if off[l + 1] - off[l] > 1:
            assert np.all(V[:, off[l]] == 0.0)
    # request k: P0 + k dt V in the simulation's precision
    P2 = sim.positions(2)
    assert P2.dtype == np.float32
    np.testing.assert_allclose(P2, (wl.step.P + np.float32(2 * sim.dt) * V).astype(np.float32), rtol=1e-6, atol=1e-7)
