"""FP64 CPU oracle of the actuator-line transfer operators.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its binding) never touches it, and it shares no
code with that path: the arithmetic lives in ``al_oracle.c``, a plain C
restatement of the paper's equations (Secs. 3.2.2-3.2.4), and this module
only marshals numpy arrays into it.

All inputs are promoted to FP64 before the call, so a comparison against
the CUDA path measures the kernel's error and not input rounding.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build, LIB_PATH

_HERE = os.path.dirname(os.path.abspath(__file__))

ST_PA_OUTSIDE, ST_PS_OUTSIDE, ST_FALLBACK, ST_FALLBACK_ZERO, ST_ZERO_WEIGHT, ST_DEPOSIT_LOST = range(6)
ST_N = 8


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double),
                ("o", C.c_double * 3), ("has_alpha", C.c_int), ("rho1", C.c_double),
                ("rho2", C.c_double), ("rho_const", C.c_double)]


class _Beams(C.Structure):
    _fields_ = [("n_lines", C.c_int), ("line_off", C.POINTER(C.c_int)),
                ("d", C.POINTER(C.c_double)), ("cdn", C.POINTER(C.c_double)),
                ("cdt", C.POINTER(C.c_double)), ("eps", C.POINTER(C.c_double)),
                ("ell_s", C.POINTER(C.c_double)), ("alpha_f", C.POINTER(C.c_double)),
                ("cv_len", C.POINTER(C.c_double)), ("n_p", C.c_double * 3),
                ("g_up", C.c_double * 3), ("tau", C.c_double), ("sample_mode", C.c_int),
                ("drag_mode", C.c_int), ("proj_mode", C.c_int),
                ("cm_n", C.POINTER(C.c_double)), ("cm_t", C.POINTER(C.c_double)),
                ("wall_reflect", C.c_int)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        src = os.path.join(_HERE, "al_oracle.c")
        if (not os.path.exists(LIB_PATH)) or os.path.getmtime(LIB_PATH) < os.path.getmtime(src):
            _build()
        lib = C.CDLL(LIB_PATH)
        dp = C.POINTER(C.c_double)
        lib.or_point_step.argtypes = [C.POINTER(_Grid), C.POINTER(_Beams), dp, dp, dp, dp, dp, dp,
                                      dp, dp, C.c_double, dp, dp, dp, dp, C.POINTER(C.c_longlong)]
        lib.or_project.argtypes = [C.POINTER(_Grid), C.POINTER(_Beams), dp, dp, C.c_int,
                                   C.POINTER(C.c_ubyte), dp, dp, C.POINTER(C.c_longlong), C.c_int]
        lib.or_sample_field.argtypes = [C.POINTER(_Grid), dp, C.c_int, C.c_int, C.c_double, dp, dp]
        lib.or_count_support.argtypes = [C.POINTER(_Grid), C.POINTER(_Beams), dp, C.c_int]
        lib.or_count_support.restype = C.c_longlong
        lib.or_closest_segment.argtypes = [dp, C.c_int, dp, C.POINTER(C.c_int), dp]
        lib.or_seg_kernel.argtypes = [dp, dp, dp, C.c_double, dp]
        lib.or_beam_quasistatic.argtypes = [C.POINTER(_Beams), dp, dp, dp, dp, dp]
        lib.or_closest_segment.restype = C.c_double
        lib.or_project_slab.argtypes = [C.POINTER(_Grid), C.POINTER(_Beams), dp, dp, C.c_int, C.c_int, dp, dp, dp]
        _lib = lib
    return _lib


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, ct=C.c_double):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def _grid(g):
    return _Grid(g.nx, g.ny, g.nz, float(g.h), (C.c_double * 3)(*map(float, g.origin)),
                 int(bool(g.has_alpha)), float(g.rho1), float(g.rho2), float(g.rho_const))


class _BeamsHold:
    """Keeps the arrays behind a _Beams struct alive."""

    def __init__(self, b):
        self.off = np.ascontiguousarray(b.line_off, dtype=np.int32)
        self.arr = [_f64(x) for x in (b.d, b.cdn, b.cdt, b.eps, b.ell_s, b.alpha_f, b.cv_len)]
        cm_n, cm_t = getattr(b, "cm_n", None), getattr(b, "cm_t", None)
        self.cm = [_f64(cm_n), _f64(cm_t)] if cm_n is not None else [None, None]
        self.s = _Beams(int(b.n_lines), _ptr(self.off, C.c_int), *[_ptr(a) for a in self.arr],
                        (C.c_double * 3)(*map(float, b.n_p)), (C.c_double * 3)(*map(float, b.g_up)),
                        float(b.tau), int(b.sample_mode), int(b.drag_mode), int(getattr(b, "proj_mode", 0)),
                        _ptr(self.cm[0]), _ptr(self.cm[1]), int(getattr(b, "wall_reflect", 0)))


def sample(grid, field, mode, p, eps=0.0):
    """Sample an SoA field (ncomp, N_c) at point p; returns (inside, value).
    eps: kernel width of the Gaussian volume average (mode 2)."""
    f = _f64(field)
    ncomp = 1 if f.ndim == 1 else f.shape[0]
    out = np.zeros(ncomp)
    g = _grid(grid)
    pp = _f64(np.asarray(p))
    ok = _load().or_sample_field(C.byref(g), _ptr(f), ncomp, int(mode), float(eps), _ptr(pp), _ptr(out))
    return bool(ok), out


def seg_kernel(c, A, B, eps):
    """(K0, K1): integral of the 3-D Gaussian along segment A -> B seen from c,
    and its first moment in t / L (the segment-integrated projection)."""
    K = np.zeros(2)
    c, A, B = (_f64(np.asarray(v)) for v in (c, A, B))
    _load().or_seg_kernel(_ptr(c), _ptr(A), _ptr(B), float(eps), _ptr(K))
    return K


def beam_quasistatic(beams, EI, axis, P0, F):
    """Quasi-static reconstruction: every node's load as a static point load
    on a linear Euler-Bernoulli cantilever along `axis` (rest positions P0,
    root at each line's first node); returns the displaced positions."""
    EI = _f64(np.broadcast_to(np.asarray(EI, float), (beams.n_lines,)).copy())
    ax = _f64(np.asarray(axis, float))
    P0, Ff = _f64(P0), _f64(F)
    out = np.zeros_like(P0)
    bh = _BeamsHold(beams)
    _load().or_beam_quasistatic(C.byref(bh.s), _ptr(EI), _ptr(ax), _ptr(P0), _ptr(Ff), _ptr(out))
    return out


def point_step(grid, beams, step, f_prev=None):
    """Sampling, drag and relaxation for every actuator point (Secs. 3.2.2-3.2.3).
    Returns F = f L (3, N_p), f (3, N_p), e_t, P_s and status counters."""
    lib = _load()
    np_ = beams.n_points
    U, al = _f64(step.U), _f64(step.alpha)
    P, Pd, T = _f64(step.P), _f64(step.Pdot), _f64(step.tangent) if beams.tangents_given else None
    fp = _f64(f_prev)
    Up, Pdd = _f64(getattr(step, "U_prev", None)), _f64(getattr(step, "Pddot", None))
    dt = float(getattr(step, "dt", 0.0) or 0.0)
    F, f, et, Ps = (np.zeros((3, np_)) for _ in range(4))
    st = np.zeros(ST_N, dtype=np.int64)
    g, bh = _grid(grid), _BeamsHold(beams)
    lib.or_point_step(C.byref(g), C.byref(bh.s), _ptr(U), _ptr(al), _ptr(P), _ptr(Pd), _ptr(T),
                      _ptr(fp), _ptr(Up), _ptr(Pdd), dt, _ptr(F), _ptr(f), _ptr(et), _ptr(Ps),
                      _ptr(st, C.c_longlong))
    return {"F": F, "f": f, "e_t": et, "P_s": Ps, "status": st}


def project(grid, beams, P_spread, F, *, cull=True, line_mask=None, n_threads=0):
    """Normalised Gaussian projection of the per-CV loads F (Sec. 3.2.4).
    Returns S (3, N_c), the nodal weights w (N_p) and status counters."""
    lib = _load()
    Ps, Ff = _f64(P_spread), _f64(F)
    S = np.zeros((3, grid.n_cells))
    w = np.zeros(beams.n_points)
    st = np.zeros(ST_N, dtype=np.int64)
    m = None if line_mask is None else np.ascontiguousarray(line_mask, dtype=np.uint8)
    g, bh = _grid(grid), _BeamsHold(beams)
    lib.or_project(C.byref(g), C.byref(bh.s), _ptr(Ps), _ptr(Ff), int(bool(cull)),
                   _ptr(m, C.c_ubyte), _ptr(S), _ptr(w), _ptr(st, C.c_longlong), int(n_threads))
    return {"S": S, "w": w, "status": st}


def project_slab(grid, beams, P_spread, F, x0, x1, w_in=None):
    """The projection over the cells with x index in [x0, x1) only (a slab,
    Sec. 3.2.5).  w_in None: returns {"w": the slab's partial nodal weights};
    else (w_in the full weights): {"S": the slab's sources}."""
    lib = _load()
    Ps, Ff = _f64(P_spread), _f64(F)
    g, bh = _grid(grid), _BeamsHold(beams)
    if w_in is None:
        w = np.zeros(beams.n_points)
        lib.or_project_slab(C.byref(g), C.byref(bh.s), _ptr(Ps), _ptr(Ff), int(x0), int(x1), None, None, _ptr(w))
        return {"w": w}
    wi = _f64(w_in)
    S = np.zeros((3, grid.n_cells))
    lib.or_project_slab(C.byref(g), C.byref(bh.s), _ptr(Ps), _ptr(Ff), int(x0), int(x1), _ptr(wi), _ptr(S), None)
    return {"S": S}


def sample_drag_spread(workload, f_prev=None, *, line_mask=None, n_threads=0, cull=True):
    """One coupling step: point_step then project at P_spread (or P).
    totals = [sum F (3), sum S V (3)] in FP64."""
    g, b, s = workload.grid, workload.beams, workload.step
    ps = point_step(g, b, s, f_prev)
    Psp = s.P if s.P_spread is None else s.P_spread
    pr = project(g, b, Psp, ps["F"], cull=cull, line_mask=line_mask, n_threads=n_threads)
    V = g.h ** 3
    totals = np.concatenate([ps["F"].sum(axis=1), pr["S"].sum(axis=1) * V])
    status = ps["status"] + pr["status"]
    return {"S": pr["S"], "F": ps["F"], "f": ps["f"], "w": pr["w"], "e_t": ps["e_t"],
            "P_s": ps["P_s"], "totals": totals, "status": status}


def count_support(grid, beams, P_spread, n_threads=0):
    """Number of (cell, line) pairs with r <= 3 eps."""
    g, bh = _grid(grid), _BeamsHold(beams)
    Ps = _f64(P_spread)
    return int(_load().or_count_support(C.byref(g), C.byref(bh.s), _ptr(Ps), int(n_threads)))


def closest_segment(X, c):
    """Closest segment of the polyline X (3, n) to point c: (seg, s, r)."""
    Xf = _f64(X)
    cc = _f64(np.asarray(c))
    k = C.c_int(0)
    sv = C.c_double(0.0)
    r2 = _load().or_closest_segment(_ptr(Xf), int(Xf.shape[1]), _ptr(cc), C.byref(k), C.byref(sv))
    return int(k.value), float(sv.value), float(np.sqrt(r2))
