"""al_footprint and the record arena's lifetime: the library's device
memory per instance is what al_footprint reports (cudaMemGetInfo before and
after), and the record arena is held only while the options use records."""
import numpy as np
import pytest

from paper_2609_39443_b300 import workloads as W

from helpers import compare, run_gpu

pytestmark = pytest.mark.gpu


def _free():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_footprint_counts_what_the_library_allocates():
    import torch
    from paper_2609_39443_b300.al import Grid, OPT_RECORD, OPT_WEIGHTS, WEIGHTS_BRICK, WEIGHTS_SEGMENT
    wl = W.make_canopy(0, 2.0, nx=128, ny=64, nz=64, n_sx=10, n_sy=10)
    torch.cuda.empty_cache()
    f0 = _free()
    g = Grid(wl.grid)
    g.load_beams(wl.beams)                         # default options: brick weights, no arena
    f1 = _free()
    fp = g.footprint()
    # three allocations at most, counted in whole 2 MiB pages: the free-memory
    # drop equals the footprint up to the driver's own bookkeeping
    assert fp > 0
    assert abs((f0 - f1) - fp) <= 4 * 2 ** 20, (f0 - f1, fp)
    g.set_option(OPT_WEIGHTS, WEIGHTS_SEGMENT)     # records on by default: the arena appears
    fp_rec = g.footprint()
    f2 = _free()
    assert fp_rec > fp
    assert abs((f1 - f2) - (fp_rec - fp)) <= 8 * 2 ** 20
    g.set_option(OPT_RECORD, 0)                    # records off: the arena goes
    assert g.footprint() == fp
    f3 = _free()
    assert abs(f3 - f1) <= 8 * 2 ** 20
    g.set_option(OPT_RECORD, 1)
    g.set_option(OPT_WEIGHTS, WEIGHTS_BRICK)       # brick weights never record
    assert g.footprint() == fp
    g.close()


def test_autotuner_keeps_the_arena_only_for_a_recording_choice():
    from paper_2609_39443_b300.al import Instance
    from paper_2609_39443_b300.al import Grid  # noqa: F401
    import oracle
    wl = W.make_canopy(1, 2.0, nx=128, ny=64, nz=64, n_sx=10, n_sy=10)
    inst = Instance(wl)
    base = inst.grid.footprint()
    wmode, bz, rec, _ = inst.autotune(trials=1)
    fp = inst.grid.footprint()
    assert (fp > base) == bool(rec and wmode == 1), (fp, base, wmode, rec)
    g = run_gpu(wl, inst=inst)
    compare(wl, g, oracle.sample_drag_spread(wl), label="after autotune")
    inst.close()
