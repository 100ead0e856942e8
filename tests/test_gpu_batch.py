"""Batched form (al_batch_*): every instance's result in the batch equals its
result alone, bit for bit, with and without CUDA-graph replay, over several
steps (so the relaxation state advances in both)."""
import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W

from helpers import BRICK_PASSES, compare

pytestmark = pytest.mark.gpu


def _instances(seed=0, n=6):
    wls = W.make_batched(seed, n, max_cells=96 * 64 * 64)
    wls.append(W.make_random(seed + 99, 37, 29, 21, n_lines=6,
                             kinds=("stem", "arc", "random", "flat", "point", "dup")))
    return wls


def _outputs(inst):
    return (inst.S.cpu().numpy().copy(), inst.F.cpu().numpy().copy(), inst.totals.cpu().numpy().copy(),
            inst.status.cpu().numpy().copy())


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_alone_bitwise(use_graph):
    import torch
    from paper_2609_39443_b300.al import Batch, Instance
    wls = _instances(1)
    alone = [Instance(w, options=BRICK_PASSES) for w in wls]
    inb = [Instance(w) for w in wls]
    batch = Batch(inb, use_graph=use_graph)
    for step in range(3):
        for a in alone:
            a.status.zero_()
            a.step()
        for b in inb:
            b.status.zero_()
        batch.run()
        torch.cuda.synchronize()
        for a, b in zip(alone, inb):
            oa, ob = _outputs(a), _outputs(b)
            for x, y in zip(oa, ob):
                np.testing.assert_array_equal(x, y)
    # and the first instance matches the oracle after the third step
    batch.close()
    for x in alone + inb:
        x.close()


def test_batch_against_oracle():
    import torch
    from paper_2609_39443_b300.al import Batch, Instance
    wls = _instances(2, n=4)
    inst = [Instance(w) for w in wls]
    batch = Batch(inst, use_graph=True)
    batch.run()
    torch.cuda.synchronize()
    for w, i in zip(wls, inst):
        g = {"S": i.S.double().cpu().numpy(), "F": i.F[:, :w.beams.n_points].double().cpu().numpy(),
             "totals": i.totals.cpu().numpy(), "status": i.status.cpu().numpy()}
        o = oracle.sample_drag_spread(w)
        compare(w, g, o, label=w.name, sumF_ref="abs")
    batch.close()
    for i in inst:
        i.close()


def test_batch_with_a_full_size_instance_against_oracle():
    """An instance at the batched workload's largest grid (256 x 128 x 128
    cells, 600 stems of 60 CVs) run inside a batch beside smaller ones, its
    S compared element by element with the FP64 oracle: the full size
    reaches the oracle directly, not only through batch = alone."""
    import torch
    from paper_2609_39443_b300.al import Batch, Instance
    big = W.random_canopy(123, 256, 128, 128, 0.005, 600, 60, 2.5, name="batch_full")
    wls = [big] + W.make_batched(5, 3, max_cells=64 * 48 * 40)
    inst = [Instance(w) for w in wls]
    batch = Batch(inst, use_graph=True)
    batch.run()
    torch.cuda.synchronize()
    for w, i in zip(wls, inst):
        g = {"S": i.S.double().cpu().numpy(), "F": i.F[:, :w.beams.n_points].double().cpu().numpy(),
             "totals": i.totals.cpu().numpy(), "status": i.status.cpu().numpy()}
        compare(w, g, oracle.sample_drag_spread(w), label=w.name)    # downstream drag: the net criterion
    batch.close()
    for i in inst:
        i.close()
