"""Thin ctypes binding of the C ABI in include/al.h.

Argument marshalling only: every step of the method runs in the CUDA
library ``libal.so``.  PyTorch provides device memory and streams.  The
library must be built (``python -m paper_2609_39443_b300.build``); if it is
missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libal.so")

AL_OK, AL_ERR_ARG, AL_ERR_CUDA, AL_ERR_OOM, AL_ERR_STATE, AL_ERR_TIMEOUT, AL_ERR_CAPACITY = 0, -1, -2, -3, -4, -5, -6
AL_FP32, AL_FP64 = 0, 1
AL_STATUS_N = 16
(ST_PA_OUTSIDE, ST_PS_OUTSIDE, ST_FALLBACK, ST_FALLBACK_ZERO, ST_ZERO_WEIGHT, ST_DEPOSIT_LOST,
 ST_REFINED, ST_IRREGULAR, ST_SUPPORT, ST_REPLAYED, ST_COLUMN) = range(11)
ST_GUARD = 15

OPT_WEIGHTS, OPT_BRICK_Z, OPT_SPREAD_CTAS, OPT_SPREAD, OPT_RECORD, OPT_COLUMN = 1, 2, 3, 4, 5, 6
OPT_OWN_X0, OPT_OWN_X1 = 7, 8
WEIGHTS_BRICK, WEIGHTS_SEGMENT = 0, 1
SPREAD_GATHER, SPREAD_SCATTER = 0, 1

TRACE_N = 6
PHASES = ("points", "mask", "weights", "normalise", "spread", "totals")

_vp = C.c_void_p
_dp = C.POINTER(C.c_double)


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("origin", C.c_double * 3), ("precision", C.c_int), ("has_alpha", C.c_int),
                ("rho1", C.c_double), ("rho2", C.c_double), ("rho_const", C.c_double)]


class BeamDesc(C.Structure):
    _fields_ = [("n_lines", C.c_int), ("line_off", C.POINTER(C.c_int)), ("d", _dp), ("cdn", _dp),
                ("cdt", _dp), ("eps", _dp), ("ell_s", _dp), ("alpha_f", _dp), ("cv_len", _dp),
                ("n_p", C.c_double * 3), ("g_up", C.c_double * 3), ("tau", C.c_double),
                ("sample_mode", C.c_int), ("drag_mode", C.c_int), ("tangents_given", C.c_int),
                ("cm_n", _dp), ("cm_t", _dp), ("proj_mode", C.c_int),
                ("wall_reflect", C.c_int)]


class StepIn(C.Structure):
    _fields_ = [("U", _vp * 3), ("alpha", _vp), ("P", _vp * 3), ("Pdot", _vp * 3),
                ("P_spread", _vp * 3), ("tangent", _vp * 3), ("U_prev", _vp * 3), ("Pddot", _vp * 3),
                ("dt", C.c_double)]


class StepOut(C.Structure):
    _fields_ = [("S", _vp * 3), ("F", _vp * 3), ("totals", _dp), ("status", C.POINTER(C.c_int))]


class ServerDesc(C.Structure):
    _fields_ = [("hbm_budget", C.c_ulonglong), ("max_sims", C.c_int), ("max_wave", C.c_int),
                ("max_points", C.c_int), ("precision", C.c_int)]


class ALError(RuntimeError):
    pass


_lib = None


def lib():
    """Load libal.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ALError(f"CUDA library not built: {LIB_PATH} (python -m paper_2609_39443_b300.build)")
        L = C.CDLL(LIB_PATH)
        L.al_create_grid.argtypes = [C.POINTER(GridDesc), C.POINTER(_vp)]
        L.al_load_beams.argtypes = [_vp, C.POINTER(BeamDesc)]
        L.al_sample_drag_spread.argtypes = [_vp, C.POINTER(StepIn), C.POINTER(StepOut), _vp]
        L.al_destroy.argtypes = [_vp]
        L.al_get_state.argtypes = [_vp, _vp, C.POINTER(C.c_int), _vp]
        L.al_set_state.argtypes = [_vp, _vp, C.c_int, _vp]
        L.al_sizes.argtypes = [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
        L.al_footprint.argtypes = [_vp, C.POINTER(C.c_ulonglong)]
        L.al_launches.argtypes = [_vp, C.POINTER(C.c_longlong)]
        L.al_beam_quasistatic.argtypes = [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double), _vp * 3, _vp * 3,
                                          _vp * 3, _vp]
        L.al_batch_create.argtypes = [C.POINTER(_vp)]
        L.al_batch_add.argtypes = [_vp, _vp, C.POINTER(StepIn), C.POINTER(StepOut)]
        L.al_batch_commit.argtypes = [_vp, C.c_int, C.c_int]
        L.al_batch_reserve.argtypes = [_vp, C.c_int, C.c_int]
        L.al_batch_run_subset.argtypes = [_vp, C.POINTER(C.c_int), C.c_int, _vp]
        L.al_batch_assign.argtypes = [_vp, C.c_int, _vp, C.POINTER(StepIn), C.POINTER(StepOut), _vp]
        L.al_batch_run.argtypes = [_vp, _vp]
        L.al_batch_destroy.argtypes = [_vp]
        L.al_line_forces_noalloc.argtypes = [C.POINTER(GridDesc), C.POINTER(BeamDesc), C.POINTER(StepIn),
                                             C.POINTER(_vp), C.POINTER(_vp), C.POINTER(C.c_int), _vp]
        L.al_trace_enable.argtypes = [_vp, C.c_int]
        L.al_set_option.argtypes = [_vp, C.c_int, C.c_int]
        L.al_autotune.argtypes = [_vp, C.POINTER(StepIn), C.POINTER(StepOut), C.c_int, _vp, C.POINTER(C.c_int)]
        L.al_batch_set_option.argtypes = [_vp, C.c_int, C.c_int]
        L.al_batch_autotune.argtypes = [_vp, C.c_int, _vp, C.POINTER(C.c_int)]
        L.al_batch_launches.argtypes = [_vp, C.POINTER(C.c_longlong)]
        L.al_trace_last.argtypes = [_vp, C.POINTER(C.c_float)]
        L.al_step_begin.argtypes = [_vp, C.POINTER(StepIn), C.POINTER(StepOut), _vp]
        L.al_step_host.argtypes = [_vp, C.POINTER(StepIn), C.POINTER(StepOut), C.POINTER(StepIn),
                                   C.POINTER(StepOut), _vp]
        L.al_step_end.argtypes = [_vp, C.POINTER(StepIn), C.POINTER(StepOut), _vp]
        L.al_weights_get.argtypes = [_vp, _vp, _vp]
        L.al_weights_set.argtypes = [_vp, _vp, _vp]
        L.al_slab_plan.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, _vp, _vp, _vp]
        L.al_server_create.argtypes = [C.POINTER(ServerDesc), C.POINTER(_vp)]
        L.al_server_set_timeout.argtypes = [_vp, C.c_double]
        L.al_server_admit.argtypes = [_vp, C.POINTER(GridDesc), C.POINTER(BeamDesc), C.POINTER(StepIn),
                                      C.POINTER(StepOut), C.c_ulonglong, C.POINTER(C.c_int)]
        L.al_server_submit.argtypes = [_vp, C.c_int, _vp, _vp, C.c_longlong]
        L.al_server_poll.argtypes = [_vp, C.POINTER(C.c_longlong), C.c_int, C.POINTER(C.c_int), C.c_int]
        L.al_server_release.argtypes = [_vp, C.c_int]
        L.al_server_footprint.argtypes = [_vp, C.POINTER(C.c_ulonglong), C.POINTER(C.c_int)]
        L.al_server_stats.argtypes = [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.al_server_destroy.argtypes = [_vp]
        L.al_error_string.restype = C.c_char_p
        L.al_error_string.argtypes = [C.c_int]
        L.al_last_cuda_error.restype = C.c_char_p
        _lib = L
    return _lib


def check(rc: int, what: str = "") -> None:
    if rc != AL_OK:
        L = lib()
        msg = L.al_error_string(rc).decode()
        if rc == AL_ERR_CUDA or rc == AL_ERR_OOM:
            msg += " (" + L.al_last_cuda_error().decode() + ")"
        raise ALError(f"{what}: {msg} [{rc}]")


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def _three(x) -> Sequence:
    """(3, N) tensor or sequence of 3 tensors -> 3 tensors (no copy)."""
    if x is None:
        return (None, None, None)
    return (x[0], x[1], x[2])


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class BeamArrays:
    """Host copies of a beam descriptor's arrays, kept alive for the call."""

    def __init__(self, beams):
        self.off = np.ascontiguousarray(beams.line_off, dtype=np.int32)
        self.arr = [np.ascontiguousarray(x, dtype=np.float64)
                    for x in (beams.d, beams.cdn, beams.cdt, beams.eps, beams.ell_s, beams.alpha_f, beams.cv_len)]

        def p(a, ct=C.c_double):
            return a.ctypes.data_as(C.POINTER(ct))

        cm_n, cm_t = getattr(beams, "cm_n", None), getattr(beams, "cm_t", None)
        self.cm = [np.ascontiguousarray(x, dtype=np.float64) for x in (cm_n, cm_t)] if cm_n is not None else []
        self.desc = BeamDesc(int(beams.n_lines), p(self.off, C.c_int), *[p(a) for a in self.arr],
                             (C.c_double * 3)(*map(float, beams.n_p)), (C.c_double * 3)(*map(float, beams.g_up)),
                             float(beams.tau), int(beams.sample_mode), int(beams.drag_mode),
                             int(bool(beams.tangents_given)), *([p(a) for a in self.cm] or [None, None]),
                             int(getattr(beams, "proj_mode", 0)),
                             int(getattr(beams, "wall_reflect", 0)))


def step_descriptors(U, P, Pdot, S, F, *, alpha=None, P_spread=None, tangent=None, totals=None, status=None,
                     U_prev=None, Pddot=None, dt=0.0):
    """al_step_in / al_step_out for the given device tensors."""
    sin = StepIn()
    for a, t in enumerate(_three(U_prev)):
        sin.U_prev[a] = _ptr(t)
    for a, t in enumerate(_three(Pddot)):
        sin.Pddot[a] = _ptr(t)
    sin.dt = float(dt)
    for a, t in enumerate(_three(U)):
        sin.U[a] = _ptr(t)
    for a, t in enumerate(_three(P)):
        sin.P[a] = _ptr(t)
    for a, t in enumerate(_three(Pdot)):
        sin.Pdot[a] = _ptr(t)
    for a, t in enumerate(_three(P_spread)):
        sin.P_spread[a] = _ptr(t)
    for a, t in enumerate(_three(tangent)):
        sin.tangent[a] = _ptr(t)
    sin.alpha = _ptr(alpha)
    sout = StepOut()
    for a, t in enumerate(_three(S)):
        sout.S[a] = _ptr(t)
    for a, t in enumerate(_three(F)):
        sout.F[a] = _ptr(t)
    sout.totals = C.cast(_ptr(totals), _dp) if totals is not None else None
    sout.status = C.cast(_ptr(status), C.POINTER(C.c_int)) if status is not None else None
    return sin, sout


class Grid:
    """One actuator-line instance: al_create_grid / al_load_beams /
    al_sample_drag_spread / al_destroy."""

    @staticmethod
    def descriptor(grid) -> GridDesc:
        return GridDesc(int(grid.nx), int(grid.ny), int(grid.nz), float(grid.h),
                        (C.c_double * 3)(*map(float, grid.origin)),
                        AL_FP64 if grid.precision == "fp64" else AL_FP32, int(bool(grid.has_alpha)),
                        float(grid.rho1), float(grid.rho2), float(grid.rho_const))

    def __init__(self, grid):
        self.spec = grid
        self.desc = Grid.descriptor(grid)
        h = _vp()
        check(lib().al_create_grid(C.byref(self.desc), C.byref(h)), "al_create_grid")
        self.h = h
        self.n_points = 0
        self.n_lines = 0

    def load_beams(self, beams) -> None:
        ba = BeamArrays(beams)
        check(lib().al_load_beams(self.h, C.byref(ba.desc)), "al_load_beams")
        self.n_points = int(beams.n_points)
        self.n_lines = int(beams.n_lines)

    def step(self, U, P, Pdot, S, F, *, alpha=None, P_spread=None, tangent=None, totals=None,
             status=None, stream=None, U_prev=None, Pddot=None, dt=0.0) -> None:
        """Enqueue one coupling step.  U, S: (3, N_c); P, Pdot, F, P_spread,
        tangent: (3, N_p) CUDA tensors of the grid precision (or sequences
        of three 1-D tensors); totals: float64[6]; status: int32[16]."""
        sin, sout = step_descriptors(U, P, Pdot, S, F, alpha=alpha, P_spread=P_spread, tangent=tangent,
                                     totals=totals, status=status, U_prev=U_prev, Pddot=Pddot, dt=dt)
        check(lib().al_sample_drag_spread(self.h, C.byref(sin), C.byref(sout), _stream_ptr(stream)),
              "al_sample_drag_spread")

    def get_state(self, f_prev, stream=None) -> bool:
        hp = C.c_int(0)
        check(lib().al_get_state(self.h, _ptr(f_prev), C.byref(hp), _stream_ptr(stream)), "al_get_state")
        return bool(hp.value)

    def set_state(self, f_prev, has_prev: bool, stream=None) -> None:
        check(lib().al_set_state(self.h, _ptr(f_prev), int(bool(has_prev)), _stream_ptr(stream)), "al_set_state")

    def set_option(self, option: int, value: int) -> None:
        """al_set_option: execution choices that leave results within the
        parity tolerances (e.g. OPT_WEIGHTS = WEIGHTS_BRICK | WEIGHTS_SEGMENT)."""
        check(lib().al_set_option(self.h, int(option), int(value)), "al_set_option")

    def beam_quasistatic(self, EI, axis, P0, F, P_out, stream=None) -> None:
        """al_beam_quasistatic: each node's load F as a static point load on a
        linear Euler-Bernoulli cantilever per line (rest positions P0, unit
        `axis`, bending stiffness EI per line); writes P_out (device tensors)."""
        ei = np.ascontiguousarray(np.broadcast_to(np.asarray(EI, float), (self.n_lines,)), dtype=np.float64)
        ax = (C.c_double * 3)(*map(float, axis))
        rows = [(_vp * 3)(*[_ptr(t) for t in _three(x)]) for x in (P0, F, P_out)]
        check(lib().al_beam_quasistatic(self.h, ei.ctypes.data_as(C.POINTER(C.c_double)), ax, rows[0], rows[1],
                                        rows[2], _stream_ptr(stream)), "al_beam_quasistatic")

    def footprint(self) -> int:
        """al_footprint: device bytes the library holds for this instance."""
        b = C.c_ulonglong(0)
        check(lib().al_footprint(self.h, C.byref(b)), "al_footprint")
        return int(b.value)

    def launches(self) -> int:
        """al_launches: kernels this instance's steps have launched so far."""
        n = C.c_longlong(0)
        check(lib().al_launches(self.h, C.byref(n)), "al_launches")
        return int(n.value)

    def trace(self, on: bool = True) -> None:
        check(lib().al_trace_enable(self.h, int(bool(on))), "al_trace_enable")

    def trace_last(self):
        """Per-phase milliseconds of the last step (points, mask, weights,
        normalise, spread, totals); waits for that step."""
        ms = (C.c_float * TRACE_N)()
        check(lib().al_trace_last(self.h, ms), "al_trace_last")
        return list(ms)

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().al_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Instance:
    """A Grid plus device-resident copies of one workload's inputs and its
    output buffers (data movement only)."""

    def __init__(self, wl, device="cuda", options=None):
        import torch
        self.wl = wl
        self.device = device
        dt = torch.float64 if wl.grid.precision == "fp64" else torch.float32
        self.dtype = dt
        s = wl.step

        def dev(a):
            return None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(device)

        self.U, self.P, self.Pdot = dev(s.U), dev(s.P), dev(s.Pdot)
        self.alpha, self.P_spread, self.tangent = dev(s.alpha), dev(s.P_spread), dev(s.tangent)
        self.U_prev, self.Pddot = dev(getattr(s, "U_prev", None)), dev(getattr(s, "Pddot", None))
        self.dt_prev = float(getattr(s, "dt", 0.0) or 0.0)
        self.S = torch.empty((3, wl.grid.n_cells), dtype=dt, device=device)
        self.F = torch.empty((3, max(wl.beams.n_points, 1)), dtype=dt, device=device)
        self.totals = torch.zeros(6, dtype=torch.float64, device=device)
        self.status = torch.zeros(AL_STATUS_N, dtype=torch.int32, device=device)
        self.grid = Grid(wl.grid)
        self.grid.load_beams(wl.beams)
        for opt, value in (options or {}).items():   # al_set_option for each (option, value)
            self.grid.set_option(opt, value)

    def step(self, stream=None):
        self.grid.step(self.U, self.P, self.Pdot, self.S, self.F, alpha=self.alpha, P_spread=self.P_spread,
                       tangent=self.tangent if self.wl.beams.tangents_given else None,
                       totals=self.totals, status=self.status, stream=stream,
                       U_prev=self.U_prev, Pddot=self.Pddot, dt=self.dt_prev)

    _FIELDS = ("U", "P", "Pdot", "alpha", "P_spread", "tangent", "U_prev", "Pddot", "S", "F")

    def own_buffers(self) -> dict:
        """This instance's device inputs and outputs, by field name."""
        return {k: getattr(self, k) for k in self._FIELDS}

    def buffers(self) -> dict:
        """A second set of device buffers shaped like own_buffers() (for
        al_step_host calls that alternate two sets)."""
        import torch
        return {k: (None if getattr(self, k) is None else torch.empty_like(getattr(self, k))) for k in self._FIELDS}

    def step_host(self, host: dict, dev: Optional[dict] = None, stream=None):
        """al_step_host: host holds pinned host tensors by field name (the
        inputs, and S and F to receive the results); dev is a device buffer
        set (own_buffers() by default).  totals and status are the
        instance's."""
        d = dev if dev is not None else self.own_buffers()
        tg = self.wl.beams.tangents_given
        hin, hout = step_descriptors(host["U"], host["P"], host["Pdot"], host.get("S"), host.get("F"),
                                     alpha=host.get("alpha"), P_spread=host.get("P_spread"),
                                     tangent=host.get("tangent") if tg else None, U_prev=host.get("U_prev"),
                                     Pddot=host.get("Pddot"), dt=self.dt_prev)
        din, dout = step_descriptors(d["U"], d["P"], d["Pdot"], d["S"], d["F"], alpha=d["alpha"],
                                     P_spread=d["P_spread"], tangent=d["tangent"] if tg else None,
                                     totals=self.totals, status=self.status, U_prev=d["U_prev"],
                                     Pddot=d["Pddot"], dt=self.dt_prev)
        check(lib().al_step_host(self.grid.h, C.byref(hin), C.byref(hout), C.byref(din), C.byref(dout),
                                 _stream_ptr(stream)), "al_step_host")

    def set_points(self, P=None, Pdot=None, P_spread=None):
        import torch
        if P is not None:
            self.P.copy_(torch.as_tensor(np.ascontiguousarray(P), dtype=self.dtype))
        if Pdot is not None:
            self.Pdot.copy_(torch.as_tensor(np.ascontiguousarray(Pdot), dtype=self.dtype))
        if P_spread is not None:
            self.P_spread.copy_(torch.as_tensor(np.ascontiguousarray(P_spread), dtype=self.dtype))

    def autotune(self, trials: int = 3, stream=None):
        """al_autotune on this instance's step; returns (weights mode, brick height, records,
        column march)."""
        sin, sout = self.descriptors()
        ch = C.c_int(0)
        check(lib().al_autotune(self.grid.h, C.byref(sin), C.byref(sout), int(trials), _stream_ptr(stream),
                                C.byref(ch)), "al_autotune")
        v = ch.value
        return (v // 100) % 10, v % 100, (v // 1000) % 10, v // 10000

    def descriptors(self):
        return step_descriptors(self.U, self.P, self.Pdot, self.S, self.F, alpha=self.alpha,
                                P_spread=self.P_spread,
                                tangent=self.tangent if self.wl.beams.tangents_given else None,
                                totals=self.totals, status=self.status,
                                U_prev=self.U_prev, Pddot=self.Pddot, dt=self.dt_prev)

    def close(self):
        self.grid.close()


class Batch:
    """al_batch_*: many instances advanced by one launch per phase.
    reserve=(n_slots, precision) adds empty slots for al_batch_assign."""

    def __init__(self, instances, use_graph=True, spread_ctas_per_sm=0, reserve=None):
        h = _vp()
        check(lib().al_batch_create(C.byref(h)), "al_batch_create")
        self.h = h
        self.instances = list(instances)
        self._desc = {}
        for q, inst in enumerate(self.instances):
            sin, sout = inst.descriptors()
            self._desc[q] = (sin, sout)
            check(lib().al_batch_add(self.h, inst.grid.h, C.byref(sin), C.byref(sout)), "al_batch_add")
        if reserve is not None:
            n, prec = reserve
            check(lib().al_batch_reserve(self.h, int(n), AL_FP64 if prec == "fp64" else AL_FP32),
                  "al_batch_reserve")
        check(lib().al_batch_commit(self.h, int(bool(use_graph)), int(spread_ctas_per_sm)), "al_batch_commit")

    def run(self, stream=None):
        check(lib().al_batch_run(self.h, _stream_ptr(stream)), "al_batch_run")

    def set_option(self, option: int, value: int) -> None:
        check(lib().al_batch_set_option(self.h, int(option), int(value)), "al_batch_set_option")

    def autotune(self, trials: int = 2, stream=None):
        """al_batch_autotune; returns (brick height, CTAs per SM (0 = as many as fit))."""
        ch = C.c_int(0)
        check(lib().al_batch_autotune(self.h, int(trials), _stream_ptr(stream), C.byref(ch)), "al_batch_autotune")
        return ch.value // 10, ch.value % 10

    def launches(self) -> int:
        """al_batch_launches: kernels the batch's runs have launched so far."""
        n = C.c_longlong(0)
        check(lib().al_batch_launches(self.h, C.byref(n)), "al_batch_launches")
        return n.value

    def run_subset(self, idx, stream=None):
        arr = (C.c_int * len(idx))(*[int(i) for i in idx])
        check(lib().al_batch_run_subset(self.h, arr, len(idx), _stream_ptr(stream)), "al_batch_run_subset")

    def assign(self, slot, inst, stream=None):
        if inst is None:
            check(lib().al_batch_assign(self.h, int(slot), None, None, None, _stream_ptr(stream)), "al_batch_assign")
            self._desc.pop(slot, None)
            return
        sin, sout = inst.descriptors()
        self._desc[slot] = (sin, sout)
        check(lib().al_batch_assign(self.h, int(slot), inst.grid.h, C.byref(sin), C.byref(sout),
                                    _stream_ptr(stream)), "al_batch_assign")

    def close(self):
        if getattr(self, "h", None):
            lib().al_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def line_forces_noalloc(grid, beams, U, P, Pdot, F, *, alpha=None, tangent=None, f_prev=None, status=None,
                        U_prev=None, Pddot=None, dt=0.0, stream=None) -> None:
    """al_line_forces_noalloc: per-CV line loads F (3, N_p) without an
    al_grid and without device allocation (tensors are the caller's).  The
    inertia inputs are used when the beams carry cm_n / cm_t."""
    gd = GridDesc(int(grid.nx), int(grid.ny), int(grid.nz), float(grid.h),
                  (C.c_double * 3)(*map(float, grid.origin)), AL_FP64 if grid.precision == "fp64" else AL_FP32,
                  int(bool(grid.has_alpha)), float(grid.rho1), float(grid.rho2), float(grid.rho_const))
    ba = BeamArrays(beams)
    sin, _ = step_descriptors(U, P, Pdot, U, F, alpha=alpha, tangent=tangent, U_prev=U_prev, Pddot=Pddot, dt=dt)
    fp = (_vp * 3)(*[_ptr(t) for t in _three(f_prev)]) if f_prev is not None else None
    fo = (_vp * 3)(*[_ptr(t) for t in _three(F)])
    st = C.cast(_ptr(status), C.POINTER(C.c_int)) if status is not None else None
    check(lib().al_line_forces_noalloc(C.byref(gd), C.byref(ba.desc), C.byref(sin), fp, fo, st,
                                       _stream_ptr(stream)), "al_line_forces_noalloc")


class Server:
    """al_server_*: continuous batching of coupling-step requests in the
    library.  Simulations are admitted with their own device buffers
    (descriptors as for al_sample_drag_spread); requests carry host positions
    and receive host line forces; poll() retires finished waves and launches
    the next one."""

    def __init__(self, hbm_budget: int, max_sims: int, max_wave: int, max_points: int, precision: str = "fp32"):
        self.desc = ServerDesc(int(hbm_budget), int(max_sims), int(max_wave), int(max_points),
                               AL_FP64 if precision == "fp64" else AL_FP32)
        h = _vp()
        check(lib().al_server_create(C.byref(self.desc), C.byref(h)), "al_server_create")
        self.h = h
        self._done = (C.c_longlong * 4096)()

    def admit(self, grid_spec, beams, sin, sout, caller_bytes: int) -> Optional[int]:
        """The slot of the admitted simulation, or None when it does not fit
        (no free slot, too many points, or over the budget)."""
        gd = Grid.descriptor(grid_spec)
        ba = BeamArrays(beams)
        sim = C.c_int(-1)
        rc = lib().al_server_admit(self.h, C.byref(gd), C.byref(ba.desc), C.byref(sin), C.byref(sout),
                                   int(caller_bytes), C.byref(sim))
        if rc == AL_ERR_CAPACITY:
            return None
        check(rc, "al_server_admit")
        return int(sim.value)

    def submit(self, sim: int, P_host: np.ndarray, F_host: np.ndarray, tag: int) -> None:
        """P_host / F_host: C-contiguous (3, N_p) host arrays of the precision,
        kept alive by the caller until the tag is reported."""
        check(lib().al_server_submit(self.h, int(sim), P_host.ctypes.data, F_host.ctypes.data, int(tag)),
              "al_server_submit")

    def poll(self, wait: bool = False):
        n = C.c_int(0)
        check(lib().al_server_poll(self.h, self._done, len(self._done), C.byref(n), int(bool(wait))),
              "al_server_poll")
        return [int(self._done[i]) for i in range(n.value)]

    def release(self, sim: int) -> None:
        check(lib().al_server_release(self.h, int(sim)), "al_server_release")

    def set_timeout(self, seconds: float) -> None:
        """Limit of the waits of poll(wait=True) and release(); past it they
        raise with AL_ERR_TIMEOUT and the step stays in flight."""
        check(lib().al_server_set_timeout(self.h, float(seconds)), "al_server_set_timeout")

    def footprint(self):
        """(device bytes held by the resident simulations, how many are resident)"""
        b, r = C.c_ulonglong(0), C.c_int(0)
        check(lib().al_server_footprint(self.h, C.byref(b), C.byref(r)), "al_server_footprint")
        return int(b.value), int(r.value)

    def waves(self):
        """(waves launched, steps they carried)"""
        w, n = C.c_longlong(0), C.c_longlong(0)
        check(lib().al_server_stats(self.h, C.byref(w), C.byref(n)), "al_server_stats")
        return int(w.value), int(n.value)

    def close(self) -> None:
        if getattr(self, "h", None):
            check(lib().al_server_destroy(self.h), "al_server_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
