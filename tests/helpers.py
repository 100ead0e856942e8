"""Shared helpers of the test-suite: run one workload through the CUDA
library and compare the outputs with the FP64 oracle."""
import numpy as np

# tolerances of the comparison (FP32 instances): S element-wise against
# max|S|, total transferred force, conservation of the resultant.
TOL_S_FP32 = 1e-5
TOL_SUMF_FP32 = 1e-6
TOL_CONS_FP32 = 1e-6
# FP64 instances run the same arithmetic in double precision.
TOL_S_FP64 = 1e-11
TOL_SUMF_FP64 = 1e-12
TOL_CONS_FP64 = 1e-12

# A batch (al_batch_*, and the server built on it) runs the brick passes for
# every brick; an instance alone takes the column march where its bricks
# allow.  Both are checked against the oracle; bit for bit, a batch equals
# its instances run alone with the column march off.
from paper_2609_39443_b300.al import OPT_COLUMN  # noqa: E402

BRICK_PASSES = {OPT_COLUMN: 0}


def run_gpu(wl, steps=1, inst=None):
    """Run `steps` coupling steps of a workload; returns numpy outputs of the last."""
    import torch
    from paper_2609_39443_b300.al import Instance
    own = inst is None
    if own:
        inst = Instance(wl)
    for _ in range(steps):
        inst.status.zero_()
        inst.step()
    torch.cuda.synchronize()
    out = {"S": inst.S.double().cpu().numpy(), "F": inst.F[:, :wl.beams.n_points].double().cpu().numpy(),
           "totals": inst.totals.cpu().numpy(), "status": inst.status.cpu().numpy()}
    if own:
        inst.close()
    return out


def tolerances(wl):
    if wl.grid.precision == "fp64":
        return TOL_S_FP64, TOL_SUMF_FP64, TOL_CONS_FP64
    return TOL_S_FP32, TOL_SUMF_FP32, TOL_CONS_FP32


def compare(wl, g, o, *, line_mask=None, cell_mask=None, label="", sumF_ref="net"):
    """Assert GPU outputs g match oracle outputs o; returns the error metrics.

    S: max over cells of |S_gpu - S_oracle| relative to max|S_oracle|.
    F: max over points of |F_gpu - F_oracle| relative to max|F_oracle|.
    sumF: |sum F_gpu - sum F_oracle| relative to |sum F_oracle| ("net"), or to
    sum |F_oracle| ("abs").  The random cases use "abs": their lines point
    every way (arcs, random walks, horizontal lines) in fields with random
    components, so the loads largely cancel and |sum F| can be orders of
    magnitude below sum |F|; the FP32 rounding of each F_i is relative to
    |F_i|, so |sum F| is not a scale it can be measured against there.  The
    configured workloads (canopy, flume, plain), whose loads point
    downstream and do not cancel, use "net", the criterion as stated.
    cons: |sum S V + sum F| on the GPU relative to sum |F|."""
    tS, tF, tC = tolerances(wl)
    out = {}
    Fo, Fg = o["F"], g["F"]
    fscale = max(np.abs(Fo).max(), 1e-300) if Fo.size else 1.0
    out["F_max_err"] = float(np.abs(Fg - Fo).max() / fscale) if Fo.size else 0.0
    sumF_o, sumF_g = Fo.sum(axis=1), g["totals"][:3]
    den = np.linalg.norm(sumF_o) if sumF_ref == "net" else np.abs(Fo).sum()
    out["sumF_rel"] = float(np.linalg.norm(sumF_g - sumF_o) / max(den, 1e-300))
    So, Sg = o["S"], g["S"]
    if cell_mask is not None:
        So, Sg = So[:, cell_mask], Sg[:, cell_mask]
    sscale = max(np.abs(So).max(), 1e-300) if So.size else 1.0
    err = np.abs(Sg - So).max(axis=0) if So.size else np.zeros(0)
    out["S_max_err"] = float(err.max() / sscale) if err.size else 0.0
    if line_mask is None:
        scale = max(np.abs(Fo).sum(), 1e-300)
        out["cons"] = float(np.abs(g["totals"][:3] + g["totals"][3:]).max() / scale)
        # the device total sum S V against the sum of the S array itself
        out["sumSV"] = float(np.abs(g["totals"][3:] - g["S"].sum(axis=1) * wl.grid.h ** 3).max() / scale)
    msg = f"{label}: {out}"
    if out["S_max_err"] > tS:
        j = int(np.argmax(err))
        msg += f" worst cell {j}: gpu {Sg[:, j]} oracle {So[:, j]}"
    assert out["S_max_err"] <= tS, msg
    assert out["F_max_err"] <= 10 * tF, msg
    assert out["sumF_rel"] <= tF, msg
    if "cons" in out:
        assert out["cons"] <= tC, msg
        assert out["sumSV"] <= tC, msg
    return out
