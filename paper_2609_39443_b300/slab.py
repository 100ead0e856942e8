"""One grid split along x into slabs, one per rank (Sec. 3.2.5: the
reduce / broadcast pairs of the parallel update, here a single exchange).

The decomposition is the library's (al_slab_plan, host code): rank r owns
whole brick columns [x0, x1) of the grid; its local grid adds a halo of
cells each side, wide enough that every point whose segments come within
3 eps of an owned cell samples inside it; it takes, whole, every line whose
reach meets its owned cells.  Each rank runs the step on its local grid with
AL_OPT_OWN_X0/X1 set: al_step_begin computes the points' forces and the
partial nodal weights over the owned cells (fixed-point integers); the
ranks add their partials over the global point index (one integer
all-reduce, exact and free of rank order); al_step_end normalises with the
summed weights and writes the owned cells of S.  A point's force is read
from the rank that owns its cell.

This module holds the host side (plan, local workload, the exchange); every
step of the method runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, replace

import numpy as np


class SlabDesc(C.Structure):
    _fields_ = [("x0", C.c_int), ("x1", C.c_int), ("lx0", C.c_int), ("lx1", C.c_int), ("halo", C.c_int),
                ("n_lines", C.c_int)]


@dataclass
class SlabPlan:
    rank: int
    n_ranks: int
    x0: int
    x1: int
    lx0: int
    lx1: int
    halo: int
    lines: np.ndarray          # global indices of the lines the rank takes (increasing)
    owner: np.ndarray          # owner rank of every global point
    points: np.ndarray         # global indices of the rank's local points (its lines' points, in order)


def plan(wl, n_ranks: int, rank: int) -> SlabPlan:
    """al_slab_plan for the workload's projection positions."""
    from .al import BeamArrays, Grid, check, lib
    L = lib()
    b = wl.beams
    P = wl.step.P if wl.step.P_spread is None else wl.step.P_spread
    Ph = np.ascontiguousarray(P, dtype=np.float64)
    gd, ba = Grid.descriptor(wl.grid), BeamArrays(b)
    out = SlabDesc()
    lines = np.zeros(max(b.n_lines, 1), dtype=np.int32)
    owner = np.zeros(max(b.n_points, 1), dtype=np.int32)
    check(L.al_slab_plan(C.addressof(gd), C.addressof(ba.desc), Ph.ctypes.data, int(n_ranks), int(rank),
                         C.addressof(out), lines.ctypes.data, owner.ctypes.data), "al_slab_plan")
    ln = lines[:out.n_lines].astype(np.int64)
    off = np.asarray(b.line_off, dtype=np.int64)
    pts = np.concatenate([np.arange(off[l], off[l + 1]) for l in ln]) if len(ln) else np.zeros(0, np.int64)
    return SlabPlan(rank, n_ranks, out.x0, out.x1, out.lx0, out.lx1, out.halo, ln,
                    owner[:b.n_points].astype(np.int64), pts)


def local_workload(wl, p: SlabPlan):
    """The rank's workload: the local grid (cells [lx0, lx1) along x), its
    fields, and the lines it takes with their points (same order)."""
    from .workloads import BeamSpec, StepInput, Workload
    g, b, s = wl.grid, wl.beams, wl.step
    nxl = p.lx1 - p.lx0
    o = list(g.origin)
    o[0] = o[0] + p.lx0 * g.h
    gl = replace(g, nx=nxl, origin=tuple(o))

    def cells(a, ncomp):
        if a is None:
            return None
        v = np.asarray(a).reshape((ncomp, g.nz, g.ny, g.nx))[..., p.lx0:p.lx1]
        return np.ascontiguousarray(v).reshape((ncomp, -1)) if ncomp > 1 else np.ascontiguousarray(v).ravel()

    def pts(a):
        return None if a is None else np.ascontiguousarray(np.asarray(a)[:, p.points])

    off = np.asarray(b.line_off, dtype=np.int64)
    cnt = off[p.lines + 1] - off[p.lines]
    loff = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)

    def per_line(a):
        return None if a is None else np.ascontiguousarray(np.asarray(a)[p.lines])

    bl = BeamSpec(line_off=loff, d=per_line(b.d), cdn=per_line(b.cdn), cdt=per_line(b.cdt), eps=per_line(b.eps),
                  ell_s=per_line(b.ell_s), alpha_f=per_line(b.alpha_f),
                  cv_len=np.ascontiguousarray(np.asarray(b.cv_len)[p.points]),
                  n_p=b.n_p, g_up=b.g_up, tau=b.tau, sample_mode=b.sample_mode, proj_mode=b.proj_mode,
                  drag_mode=b.drag_mode, tangents_given=b.tangents_given, cm_n=per_line(b.cm_n),
                  cm_t=per_line(b.cm_t), wall_reflect=b.wall_reflect)
    sl = StepInput(U=cells(s.U, 3), P=pts(s.P), Pdot=pts(s.Pdot), alpha=cells(s.alpha, 1),
                   P_spread=pts(s.P_spread), tangent=pts(s.tangent), U_prev=cells(s.U_prev, 3),
                   Pddot=pts(s.Pddot), dt=s.dt)
    return Workload(f"{wl.name}_slab{p.rank}of{p.n_ranks}", gl, bl, sl)


class SlabRank:
    """One rank's instance on its local grid (device), stepped in two
    phases around the exchange of the partial weights."""

    def __init__(self, wl, n_ranks: int, rank: int, device="cuda", plan_=None):
        import torch
        from .al import OPT_OWN_X0, OPT_OWN_X1, Instance
        self.plan = plan_ if plan_ is not None else plan(wl, n_ranks, rank)
        self.global_np = wl.beams.n_points
        self.wl_local = local_workload(wl, self.plan)
        p = self.plan
        self.inst = Instance(self.wl_local, device=device,
                             options={OPT_OWN_X0: p.x0 - p.lx0, OPT_OWN_X1: p.x1 - p.lx0})
        self.gidx = torch.as_tensor(p.points, dtype=torch.int64, device=device)
        self.w = torch.zeros(max(len(p.points), 1), dtype=torch.int64, device=device)

    def begin(self, stream=None):
        from .al import _stream_ptr, check, lib
        sin, sout = self.inst.descriptors()
        check(lib().al_step_begin(self.inst.grid.h, C.byref(sin), C.byref(sout), _stream_ptr(stream)),
              "al_step_begin")
        check(lib().al_weights_get(self.inst.grid.h, self.w.data_ptr(), _stream_ptr(stream)), "al_weights_get")

    def partial(self, glob):
        """Add this rank's partial weights into glob (int64, global N_p)."""
        if len(self.plan.points):
            glob.index_add_(0, self.gidx, self.w[:len(self.plan.points)])

    def end(self, glob, stream=None):
        """Finish the step with the summed weights glob."""
        from .al import _stream_ptr, check, lib
        if len(self.plan.points):
            self.w[:len(self.plan.points)] = glob[self.gidx]
        check(lib().al_weights_set(self.inst.grid.h, self.w.data_ptr(), _stream_ptr(stream)), "al_weights_set")
        sin, sout = self.inst.descriptors()
        check(lib().al_step_end(self.inst.grid.h, C.byref(sin), C.byref(sout), _stream_ptr(stream)),
              "al_step_end")

    def step(self, allreduce):
        """One step; allreduce(t) sums the int64 tensor t over the ranks in
        place (torch.distributed.all_reduce)."""
        import torch
        self.begin()
        glob = torch.zeros(max(self.global_np, 1), dtype=torch.int64, device=self.w.device)
        self.partial(glob)
        allreduce(glob)
        self.end(glob)

    def owned_S(self) -> np.ndarray:
        """S of the owned cells, (3, nz, ny, x1 - x0)."""
        g, p = self.wl_local.grid, self.plan
        S = self.inst.S.cpu().numpy().reshape(3, g.nz, g.ny, g.nx)
        return S[..., p.x0 - p.lx0:p.x1 - p.lx0].copy()

    def owned_F(self):
        """(global indices, F (3, n)) of the points this rank owns."""
        p = self.plan
        keep = p.owner[p.points] == p.rank
        F = self.inst.F[:, :len(p.points)].cpu().numpy()
        return p.points[keep], F[:, keep]

    def close(self):
        self.inst.close()
