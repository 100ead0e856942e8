"""Host logic of the continuous-batching server, with a stand-in backend
(no GPU): every request completes once, each simulation's steps run in
order and never two at a time, no wave holds a simulation twice, resident
memory never exceeds the HBM budget, and slots are reused after eviction."""
import numpy as np
import pytest

from paper_2609_39443_b300 import workloads as W
from paper_2609_39443_b300.serve import BatchServer, PlainServer, Sim, poisson_arrivals


class _Event:
    def __init__(self, polls):
        self.polls = polls

    def done(self):
        self.polls -= 1
        return self.polls < 0


class _Res:
    def __init__(self, sim, log):
        self.sim, self.log = sim, log
        self.inst = self                 # what the batch binds to a slot
        self.next_k, self.staged, self.in_flight, self.closed = 0, None, False, False

    def upload(self, k):
        assert not self.in_flight, "a step of this simulation is already in flight"
        assert k == self.next_k, (k, self.next_k)
        self.staged, self.in_flight = k, True

    def step(self, stream):
        self.advance()

    def advance(self):
        assert self.in_flight
        self.next_k += 1
        self.in_flight = False

    def download(self):
        pass

    def result_F(self):
        return np.array([self.staged])

    def result_S(self):
        return np.array([self.next_k])

    def close(self):
        self.closed = True


class _Batch:
    def __init__(self, n_slots):
        self.slots = [None] * n_slots
        self.waves = []

    def assign(self, slot, inst, stream=None):
        self.slots[slot] = inst

    def run_subset(self, idx, stream=None):
        assert len(set(idx)) == len(idx), "a slot twice in one wave"
        for i in idx:
            assert self.slots[i] is not None, "run of an unbound slot"
            self.slots[i].advance()
        self.waves.append(list(idx))

    def close(self):
        pass


class _Ctx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


class FakeBackend:
    def __init__(self, polls=2):
        self.polls = polls
        self.batches = []
        self.log = []

    def stream(self):
        return object()

    def resident(self, sim):
        return _Res(sim, self.log)

    def batch(self, n_slots, precision):
        b = _Batch(n_slots)
        self.batches.append(b)
        return b

    def stream_ctx(self, stream):
        return _Ctx()

    def mark(self, stream):
        return _Event(self.polls)

    @staticmethod
    def done(ev):
        return ev.done()

    @staticmethod
    def sync(stream):
        pass

    def sync_all(self):
        pass


def _sims(n=12, steps=5):
    wls = [W.make_random(100 + i, 20 + 4 * (i % 3), 16, 12, n_lines=1 + i % 3, kinds=("stem",)) for i in range(n)]
    return [Sim(w, steps) for w in wls]


@pytest.mark.parametrize("rate", [300.0, 50000.0])
@pytest.mark.parametrize("server", ["batched", "plain"])
def test_scheduler_invariants(server, rate):
    sims = _sims()
    budget = 3 * max(s.footprint() for s in sims)          # about three resident at a time
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
        assert int(v[0]) == k                                # the staged step is the one reported
    assert all(int(srv.final_S[s][0]) == sims[s].n_steps for s in range(len(sims)))
    assert st.peak_mem <= budget
    assert st.admitted == len(sims)
    assert not srv.res                                       # everything evicted at the end
    assert len(st.latencies) == len(arr) and min(st.latencies) >= 0.0
    if server == "batched":
        waves = be.batches[0].waves
        assert sum(len(w) for w in waves) == len(arr)
        assert st.waves == len(waves)


def test_poisson_arrivals_keep_per_simulation_order():
    sims = _sims(5, 7)
    arr = poisson_arrivals(sims, 1000.0, seed=3)
    assert len(arr) == 35
    assert all(a[0] <= b[0] for a, b in zip(arr, arr[1:]))
    for s in range(5):
        ks = [k for _, ss, k in arr if ss == s]
        assert ks == list(range(7))
