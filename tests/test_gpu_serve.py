"""Continuous batching on the device: simulations served in a mix of waves
(with admission by HBM footprint forcing some to wait for others to leave)
produce, step for step, the same line forces and final momentum source as
each simulation run alone, bit for bit."""
import numpy as np
import pytest

from paper_2609_39443_b300 import workloads as W
from paper_2609_39443_b300.serve import BatchServer, Sim, poisson_arrivals

from helpers import BRICK_PASSES

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("reflect", [False, True], ids=["truncated", "reflected-bed"])
def test_served_mix_equals_each_simulation_alone(reflect):
    import torch
    from paper_2609_39443_b300.al import Instance
    wls = W.make_batched(31, 6, max_cells=64 * 48 * 40)
    if reflect:                     # every other simulation reflects its kernel at the bed
        wls = [W.with_reflect(w, W.REFLECT_Z_LO) if i % 2 == 0 else w for i, w in enumerate(wls)]
    sims = [Sim(w, 3) for w in wls]
    budget = int(2.5 * max(s.footprint() for s in sims))     # two or three resident at a time
    arr = poisson_arrivals(sims, 5000.0, seed=11)
    srv = BatchServer(sims, budget, n_slots=4, record=True)
    st = srv.run(arr)
    assert st.completed == len(arr)
    assert st.peak_mem <= budget
    for s, sim in enumerate(sims):
        inst = Instance(sim.wl, options=BRICK_PASSES)
        for k in range(sim.n_steps):
            inst.set_points(P=sim.positions(k))
            inst.step()
            torch.cuda.synchronize()
            F = inst.F[:, :sim.wl.beams.n_points].cpu().numpy()
            np.testing.assert_array_equal(F, srv.results[(s, k)])
        np.testing.assert_array_equal(inst.S.cpu().numpy(), srv.final_S[s])
        inst.close()
