"""Seeded synthetic inputs for the actuator-line transfer operators.

This module only *generates* inputs: grids, velocity / volume-fraction fields
and beam centrelines with their per-line coefficients.  It contains none of
the method's arithmetic (no sampling, no drag, no projection), so that the
FP64 oracle and the CUDA path can both be fed from it without sharing any
of the computation they are compared on.

Geometry follows the paper's workloads: a cantilever in a channel
(Sec. 5), a canopy of flexible stems and the wave flume of Sec. 7
(depth, amplitude and period of the primary condition; stem diameter and
CV length of the flume stem).  Everything is drawn from
``numpy.random.Generator(PCG64(seed))``.

Layout conventions shared by every consumer:
  * cell (i, j, k) has centre ``origin + ((i+1/2) h, (j+1/2) h, (k+1/2) h)``
    and linear index ``i + nx * (j + ny * k)`` (x fastest);
  * fields are SoA arrays of shape ``(3, N_c)`` (velocity) and ``(N_c,)``
    (volume fraction alpha);
  * points are SoA arrays of shape ``(3, N_p)``; line ``l`` owns points
    ``line_off[l] .. line_off[l+1]-1`` ordered from root to tip.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

G_ACC = 9.81

SAMPLE_TRILINEAR = 0
SAMPLE_CELL = 1
SAMPLE_GAUSS = 2        # Gaussian-weighted volume average over the projection kernel's support
DRAG_DISCRETE = 0
DRAG_SPLIT = 1


@dataclass
class GridSpec:
    nx: int
    ny: int
    nz: int
    h: float
    origin: tuple = (0.0, 0.0, 0.0)
    precision: str = "fp32"          # storage/compute type of fields, S and F
    has_alpha: bool = False
    rho1: float = 1000.0             # phase-1 density (alpha = 1)
    rho2: float = 1.2                # phase-2 density (alpha = 0)
    rho_const: float = 1000.0        # density when there is no alpha field

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dtype(self):
        return np.float64 if self.precision == "fp64" else np.float32


@dataclass
class BeamSpec:
    line_off: np.ndarray             # int32 [n_lines + 1]
    d: np.ndarray                    # float64 [n_lines] drag reference length
    cdn: np.ndarray                  # float64 [n_lines]
    cdt: np.ndarray                  # float64 [n_lines]
    eps: np.ndarray                  # float64 [n_lines] Gaussian width (m)
    ell_s: np.ndarray                # float64 [n_lines] sampling distance (m)
    alpha_f: np.ndarray              # float64 [n_lines] relaxation factor
    cv_len: np.ndarray               # float64 [N_p] CV length L_i
    n_p: tuple = (0.0, 0.0, 0.0)     # sampling-plane normal (0 = none)
    g_up: tuple = (-1.0, 0.0, 0.0)   # global upstream fallback direction
    tau: float = 1e-6                # fallback threshold on |u0_n| (m/s)
    sample_mode: int = SAMPLE_TRILINEAR
    proj_mode: int = 0          # 0 nearest segment (the paper's), 1 segment-integrated 3-D Gaussian
    drag_mode: int = DRAG_DISCRETE
    tangents_given: bool = False
    cm_n: Optional[np.ndarray] = None   # float64 [n_lines] added-mass coefficients (None: no inertia term)
    cm_t: Optional[np.ndarray] = None
    wall_reflect: int = 0       # bit 2a (2a + 1): the low (high) face of axis a reflects the kernel

    @property
    def n_lines(self) -> int:
        return int(len(self.line_off) - 1)

    @property
    def n_points(self) -> int:
        return int(self.line_off[-1])


@dataclass
class StepInput:
    U: np.ndarray                    # (3, N_c)
    P: np.ndarray                    # (3, N_p) actuator points
    Pdot: np.ndarray                 # (3, N_p) actuator-point velocities
    alpha: Optional[np.ndarray] = None       # (N_c,)
    P_spread: Optional[np.ndarray] = None    # (3, N_p) positions used by the projection
    tangent: Optional[np.ndarray] = None     # (3, N_p) caller tangents
    U_prev: Optional[np.ndarray] = None      # (3, N_c) fluid velocity one time step earlier
    Pddot: Optional[np.ndarray] = None       # (3, N_p) actuator-point accelerations
    dt: float = 0.0                          # time step between U_prev and U (s)


@dataclass
class Workload:
    name: str
    grid: GridSpec
    beams: BeamSpec
    step: StepInput
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _centres_1d(n: int, h: float, o: float) -> np.ndarray:
    return o + (np.arange(n, dtype=np.float64) + 0.5) * h


def _beams_from_lines(lines: List[np.ndarray], cv_len: List[np.ndarray], *,
                      d, cdn, cdt, eps, ell_s, alpha_f=1.0, **kw) -> BeamSpec:
    n = len(lines)
    counts = np.array([ln.shape[1] for ln in lines], dtype=np.int64)
    off = np.zeros(n + 1, dtype=np.int32)
    off[1:] = np.cumsum(counts)

    def per_line(v):
        a = np.asarray(v, dtype=np.float64)
        return np.full(n, float(a)) if a.ndim == 0 else a.astype(np.float64).copy()

    return BeamSpec(line_off=off, d=per_line(d), cdn=per_line(cdn), cdt=per_line(cdt),
                    eps=per_line(eps), ell_s=per_line(ell_s), alpha_f=per_line(alpha_f),
                    cv_len=np.concatenate(cv_len).astype(np.float64) if n else np.zeros(0),
                    **kw)


def _stem(root, height, n_cv, bend, psi):
    """CV centres of a stem rooted at ``root`` growing along +z with a
    quadratic deflection ``bend * (s/H)^2`` in the horizontal direction psi."""
    s = (np.arange(n_cv, dtype=np.float64) + 0.5) * (height / n_cv)
    q = (s / height) ** 2
    x = root[0] + bend * np.cos(psi) * q
    y = root[1] + bend * np.sin(psi) * q
    z = root[2] + s
    return np.stack([x, y, z])


def _solenoidal_modes(rng, grid: GridSpec, n_modes: int, nmax: int):
    """Sum of ``n_modes`` divergence-free Fourier modes a sin(k.x + phi),
    a perpendicular to k, with integer wave-vector indices 1 <= |n| <= nmax."""
    Lx, Ly, Lz = grid.nx * grid.h, grid.ny * grid.h, grid.nz * grid.h
    xs = _centres_1d(grid.nx, grid.h, grid.origin[0]).astype(np.float32)
    ys = _centres_1d(grid.ny, grid.h, grid.origin[1]).astype(np.float32)
    zs = _centres_1d(grid.nz, grid.h, grid.origin[2]).astype(np.float32)
    out = np.zeros((3, grid.nz, grid.ny, grid.nx), dtype=np.float32)
    m = 0
    while m < n_modes:
        nvec = rng.integers(-nmax, nmax + 1, size=3)
        nn = float(np.sqrt((nvec ** 2).sum()))
        if nn < 1.0 or nn > nmax:
            continue
        k = 2.0 * np.pi * np.array([nvec[0] / Lx, nvec[1] / Ly, nvec[2] / Lz])
        a = rng.normal(size=3)
        a -= a.dot(k) / k.dot(k) * k
        a /= np.linalg.norm(a)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        px = (k[0] * xs).astype(np.float32)[None, None, :]
        py = (k[1] * ys).astype(np.float32)[None, :, None]
        pz = (k[2] * zs + phi).astype(np.float32)[:, None, None]
        s = np.sin(px + py + pz)
        for c in range(3):
            out[c] += np.float32(a[c]) * s
        m += 1
    return out.reshape(3, -1)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def make_plain(seed: int = 0) -> Workload:
    """Plain method, FP64: 64x32x32 cells, h = 0.01 m, one wall-mounted
    cantilever of 20 CVs (L = 0.2 m, d = 0.01 m) in U = (0.5,0,0) + noise."""
    rng = _rng(seed)
    grid = GridSpec(64, 32, 32, 0.01, precision="fp64", rho_const=1000.0)
    nc = grid.n_cells
    U = rng.normal(0.0, 0.05, size=(3, nc))
    U[0] += 0.5
    delta = rng.uniform(0.0, 0.03)
    psi = rng.uniform(0.0, 2.0 * np.pi)
    P = _stem((0.20, 0.16, 0.0), 0.2, 20, delta, psi)
    Pdot = rng.normal(0.0, 0.01, size=P.shape)
    h = grid.h
    beams = _beams_from_lines([P], [np.full(20, 0.2 / 20)], d=0.01, cdn=1.2, cdt=0.01,
                              eps=2 * h, ell_s=3 * 2 * h + h)
    return Workload("plain_fp64_64x32x32", grid, beams,
                    StepInput(U=U.astype(np.float64), P=P, Pdot=Pdot))


def make_canopy(seed: int = 0, eps_cells: float = 2.0, *, nx=256, ny=128, nz=128,
                h=0.005, n_sx=20, n_sy=20, n_cv=60, height=0.3) -> Workload:
    """Vegetation canopy, FP32 fields: log-law profile plus 32 solenoidal
    Fourier modes at 10 % intensity; a 20x20 staggered array of stems
    (spacing 0.04 m x 0.025 m, odd rows shifted 0.02 m), 60 CVs each,
    d = 0.006 m, quadratic bending <= 0.03 m along +x +- 15 deg."""
    rng = _rng(seed)
    grid = GridSpec(nx, ny, nz, h, precision="fp32", rho_const=1000.0)
    Lx, Ly = nx * h, ny * h
    zc = _centres_1d(nz, h, 0.0)
    ustar, kappa, z0 = 0.01, 0.41, 1e-3
    ux = (ustar / kappa) * np.log1p(zc / z0)
    modes = _solenoidal_modes(rng, grid, 32, 8)
    ux_mean = float(ux.mean())
    rms = float(np.sqrt((modes.astype(np.float64) ** 2).mean()))
    modes *= np.float32(0.1 * ux_mean / max(rms, 1e-30))
    U = modes
    U[0] += np.repeat(ux.astype(np.float32), ny * nx)
    sx, sy, shift = 0.04, 0.025, 0.02
    x0 = (Lx - ((n_sx - 1) * sx + shift)) / 2.0
    y0 = (Ly - (n_sy - 1) * sy) / 2.0
    lines, lens = [], []
    for j in range(n_sy):
        for i in range(n_sx):
            root = (x0 + i * sx + (shift if j % 2 else 0.0), y0 + j * sy, 0.0)
            bend = rng.uniform(0.0, 0.03)
            psi = np.deg2rad(rng.uniform(-15.0, 15.0))
            lines.append(_stem(root, height, n_cv, bend, psi))
            lens.append(np.full(n_cv, height / n_cv))
    P = np.concatenate(lines, axis=1)
    Pdot = rng.normal(0.0, 0.02, size=P.shape)
    eps = eps_cells * h
    beams = _beams_from_lines(lines, lens, d=0.006, cdn=1.2, cdt=0.01, eps=eps,
                              ell_s=3 * eps + h)
    return Workload(f"canopy_{nx}x{ny}x{nz}_eps{eps_cells:g}h", grid, beams,
                    StepInput(U=U.astype(np.float32), P=P.astype(np.float32),
                              Pdot=Pdot.astype(np.float32)),
                    meta={"eps_cells": eps_cells})


def make_walls(seed: int = 0, *, nx=40, ny=36, nz=30, h=0.01, precision="fp32") -> Workload:
    """Lines against the grid faces, for the kernel reflected at walls:
    - a stem rooted on the bed in the x- / y- corner;
    - a stem rooted on the bed next to the y- face;
    - a horizontal line along the x+ face;
    - an arc under the top face near y+;
    - a single point in the x+ / y+ / z+ corner.
    Every node lies inside the grid box.  The flow is uniform plus noise,
    eps is drawn in [1.5, 2.5] h, and l_s = h / 2."""
    rng = _rng(seed)
    grid = GridSpec(nx, ny, nz, h, precision=precision, rho_const=1000.0)
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    t = np.linspace(0.0, 1.0, 16)
    th = np.linspace(0.0, np.pi, 12)
    lines = [
        np.stack([h * (0.7 + 2.0 * rng.uniform(0.5, 1.0) * t ** 2), h * (1.1 + rng.uniform(0.0, 1.0) * t),
                  0.6 * Lz * t]),
        np.stack([0.5 * Lx + h * rng.uniform(-2.0, 2.0) * t, np.full_like(t, h * rng.uniform(2.0, 3.0)),
                  0.5 * Lz * t]),
        np.stack([Lx - h * (1.5 + 0.5 * np.sin(3.0 * t)), 0.2 * Ly + 0.6 * Ly * t, np.full_like(t, 0.5 * Lz)]),
        np.stack([0.3 * Lx + 4.0 * h * np.cos(th), Ly - h * (2.5 + 1.5 * np.sin(th)), Lz - h * (1.2 + 2.0 * np.sin(th))]),
        np.array([[Lx - 0.8 * h], [Ly - 1.2 * h], [Lz - 0.9 * h]]),
    ]
    for P in lines:
        assert (P >= 0.0).all() and (P[0] <= Lx).all() and (P[1] <= Ly).all() and (P[2] <= Lz).all()
    lens = [np.full(P.shape[1], max(float(np.linalg.norm(np.diff(P, axis=1), axis=0).mean()) if P.shape[1] > 1
                                    else h, 1e-9)) for P in lines]
    U = rng.normal(0.0, 0.03, size=(3, grid.n_cells))
    U[0] += 0.3
    U[1] += 0.05
    P = np.concatenate(lines, axis=1)
    Pdot = rng.normal(0.0, 0.01, size=P.shape)
    eps = rng.uniform(1.5, 2.5) * h
    beams = _beams_from_lines(lines, lens, d=0.005, cdn=1.2, cdt=0.01, eps=eps, ell_s=0.5 * h)
    ft = np.float64 if precision == "fp64" else np.float32
    return Workload(f"walls_{nx}x{ny}x{nz}", grid, beams,
                    StepInput(U=U.astype(ft), P=P.astype(ft), Pdot=Pdot.astype(ft)))


def wave_number(omega: float, depth: float) -> float:
    """Root of the linear dispersion relation omega^2 = g k tanh(k depth)."""
    k = omega * omega / G_ACC
    for _ in range(100):
        f = G_ACC * k * np.tanh(k * depth) - omega * omega
        df = G_ACC * np.tanh(k * depth) + G_ACC * k * depth / np.cosh(k * depth) ** 2
        k_new = k - f / df
        if abs(k_new - k) < 1e-15 * k:
            k = k_new
            break
        k = k_new
    return float(k)


def make_flume(seed: int = 0, *, nx=1024, ny=256, nz=128, h=0.004, n_sx=100, n_sy=40,
               n_cv=80, height=0.4) -> Workload:
    """Free-surface wave flume, FP32: linear-wave orbital velocity (depth
    0.3 m, amplitude 0.05 m, period 1.5 s), a 3-cell smeared interface at
    eta = A sin(kx), 4000 surface-piercing stems of 80 CVs (d = 0.004 m),
    eps = 2h, sampling plane normal y, l_s = 7h."""
    rng = _rng(seed)
    grid = GridSpec(nx, ny, nz, h, precision="fp32", has_alpha=True, rho1=1000.0, rho2=1.2)
    depth, A, T = 0.3, 0.05, 1.5
    omega = 2.0 * np.pi / T
    k = wave_number(omega, depth)
    t0 = rng.uniform(0.0, T)
    xc = _centres_1d(nx, h, 0.0)
    zc = _centres_1d(nz, h, 0.0)
    eta = A * np.sin(k * xc)                                   # (nx,)
    ze = np.minimum(zc[:, None], depth + eta[None, :])         # (nz, nx)
    ph = k * xc[None, :] - omega * t0
    amp = A * omega / np.sinh(k * depth)
    u = amp * np.cosh(k * ze) * np.cos(ph)
    w = amp * np.sinh(k * ze) * np.sin(ph)
    alpha = np.clip(0.5 - (zc[:, None] - depth - eta[None, :]) / (3.0 * h), 0.0, 1.0)
    u *= alpha
    w *= alpha
    nc = grid.n_cells
    U = np.zeros((3, nz, ny, nx), dtype=np.float32)
    U[0] = u.astype(np.float32)[:, None, :]
    U[2] = w.astype(np.float32)[:, None, :]
    al = np.broadcast_to(alpha.astype(np.float32)[:, None, :], (nz, ny, nx)).reshape(nc).copy()
    sx, sy = 0.04, 0.025
    y0 = (ny * h - (n_sy - 1) * sy) / 2.0
    lines, lens = [], []
    for j in range(n_sy):
        for i in range(n_sx):
            root = (0.06 + i * sx, y0 + j * sy, 0.0)
            bend = rng.uniform(-0.03, 0.03)
            lines.append(_stem(root, height, n_cv, bend, 0.0))
            lens.append(np.full(n_cv, height / n_cv))
    P = np.concatenate(lines, axis=1)
    Pdot = rng.normal(0.0, 0.02, size=P.shape)
    beams = _beams_from_lines(lines, lens, d=0.004, cdn=1.2, cdt=0.01, eps=2 * h,
                              ell_s=7 * h, n_p=(0.0, 1.0, 0.0), g_up=(-1.0, 0.0, 0.0))
    return Workload(f"flume_{nx}x{ny}x{nz}", grid, beams,
                    StepInput(U=U.reshape(3, nc), P=P.astype(np.float32),
                              Pdot=Pdot.astype(np.float32), alpha=al),
                    meta={"k": k, "t0": t0})


def make_random(seed: int, nx: int, ny: int, nz: int, *, h: float = 0.01,
                n_lines: int = 3, precision: str = "fp32", has_alpha: bool = False,
                eps_cells=(1.5, 3.0), n_cv=(2, 24), kinds=("stem", "arc", "random"),
                sample_mode: int = SAMPLE_TRILINEAR, drag_mode: int = DRAG_DISCRETE,
                n_p=(0.0, 0.0, 0.0)) -> Workload:
    """Small random instance for edge-case tests.  Line kinds:
    ``stem``   gently bent vertical stem;
    ``arc``    tightly curved arc (radius of a few kernel widths);
    ``random`` random walk of short steps (sharp turns, fold-backs);
    ``flat``   horizontal line along a random direction;
    ``point``  a single actuator point;
    ``dup``    a line with repeated (zero-length) segments.
    Lines may leave the domain."""
    rng = _rng(seed)
    grid = GridSpec(nx, ny, nz, h, precision=precision, has_alpha=has_alpha,
                    rho1=1000.0, rho2=1.2, rho_const=1000.0)
    L = np.array([nx, ny, nz], dtype=np.float64) * h
    nc = grid.n_cells
    U = rng.normal(0.0, 0.1, size=(3, nc))
    U[0] += 0.4
    alpha = rng.uniform(0.0, 1.0, size=nc) if has_alpha else None
    lines, lens, eps, ell = [], [], [], []
    for _ in range(n_lines):
        kind = kinds[int(rng.integers(len(kinds)))]
        m = int(rng.integers(n_cv[0], n_cv[1] + 1))
        e = rng.uniform(*eps_cells) * h
        start = rng.uniform(0.15, 0.85, size=3) * L
        if kind == "stem":
            step = rng.uniform(0.6, 1.6) * h
            pts = _stem((start[0], start[1], 0.05 * L[2]), step * m, m,
                        rng.uniform(0, 0.3) * step * m, rng.uniform(0, 2 * np.pi))
        elif kind == "arc":
            rad = rng.uniform(1.0, 4.0) * e
            th = np.linspace(0, rng.uniform(1.0, 5.0), m)
            ax = rng.normal(size=3); ax /= np.linalg.norm(ax)
            b1 = np.cross(ax, rng.normal(size=3)); b1 /= np.linalg.norm(b1)
            b2 = np.cross(ax, b1)
            pts = start[:, None] + rad * (np.cos(th) * b1[:, None] + np.sin(th) * b2[:, None]) \
                + 0.3 * e * th * ax[:, None]
        elif kind == "flat":
            d = rng.normal(size=3); d[2] = 0.0; d /= np.linalg.norm(d)
            step = rng.uniform(0.5, 2.0) * h
            pts = start[:, None] + step * np.arange(m)[None, :] * d[:, None]
        elif kind == "point":
            m = 1
            pts = start[:, None].copy()
        elif kind == "dup":
            step = rng.uniform(0.6, 1.6) * h
            pts = start[:, None] + step * np.arange(m)[None, :] * np.array([0.2, 0.1, 1.0])[:, None]
            if m >= 3:
                pts[:, m // 2] = pts[:, m // 2 - 1]
        else:  # random walk
            steps = rng.normal(size=(3, m)) * rng.uniform(0.5, 1.5) * h
            pts = start[:, None] + np.cumsum(steps, axis=1)
        lines.append(pts)
        seg = np.linalg.norm(np.diff(pts, axis=1), axis=0) if pts.shape[1] > 1 else np.array([h])
        cvl = np.empty(pts.shape[1])
        cvl[:] = max(float(np.mean(seg)) if seg.size else h, 0.5 * h)
        lens.append(cvl)
        eps.append(e)
        ell.append(3 * e + h)
    P = np.concatenate(lines, axis=1)
    Pdot = rng.normal(0.0, 0.03, size=P.shape)
    dt = grid.dtype
    beams = _beams_from_lines(lines, lens, d=rng.uniform(0.004, 0.012, size=n_lines),
                              cdn=rng.uniform(0.8, 1.5, size=n_lines),
                              cdt=rng.uniform(0.0, 0.05, size=n_lines),
                              eps=np.array(eps), ell_s=np.array(ell),
                              alpha_f=rng.uniform(0.3, 1.0, size=n_lines),
                              sample_mode=sample_mode, drag_mode=drag_mode, n_p=n_p)
    return Workload(f"random_{seed}_{nx}x{ny}x{nz}", grid, beams,
                    StepInput(U=U.astype(dt), P=P.astype(dt), Pdot=Pdot.astype(dt),
                              alpha=None if alpha is None else alpha.astype(dt)))


def make_batched(seed: int = 0, n_instances: int = 64, *, max_cells: Optional[int] = None):
    """Batched form: independent instances whose grid sizes (32..256 x
    32..128 x 32..128, multiples of 8), stem counts (1..2000), CVs per stem
    (10..100) and kernel widths (1.5..3 h) are drawn log-uniformly."""
    rng = _rng(seed)
    out = []

    def logu(a, b):
        return float(np.exp(rng.uniform(np.log(a), np.log(b))))

    for n in range(n_instances):
        nx = int(round(logu(32, 256) / 8)) * 8
        ny = int(round(logu(32, 128) / 8)) * 8
        nz = int(round(logu(32, 128) / 8)) * 8
        if max_cells is not None:
            while nx * ny * nz > max_cells and nx > 8:
                nx -= 8
        h = 0.005
        eps_c = logu(1.5, 3.0)
        n_st = int(round(logu(1, 2000)))
        n_cv = int(round(logu(10, 100)))
        sub = int(rng.integers(0, 2 ** 31 - 1))
        out.append(random_canopy(sub, nx, ny, nz, h, n_st, n_cv, eps_c, name=f"batch{n}"))
    return out


def random_canopy(seed, nx, ny, nz, h, n_stems, n_cv, eps_cells, name="canopy"):
    rng = _rng(seed)
    grid = GridSpec(nx, ny, nz, h, precision="fp32", rho_const=1000.0)
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    zc = _centres_1d(nz, h, 0.0)
    ux = (0.01 / 0.41) * np.log1p(zc / 1e-3)
    modes = _solenoidal_modes(rng, grid, 8, 4)
    rms = float(np.sqrt((modes.astype(np.float64) ** 2).mean()))
    modes *= np.float32(0.1 * float(ux.mean()) / max(rms, 1e-30))
    U = modes
    U[0] += np.repeat(ux.astype(np.float32), ny * nx)
    eps = eps_cells * h
    height = 0.5 * Lz
    margin = 3 * eps + 3 * eps + h + 0.03
    lines, lens = [], []
    for _ in range(n_stems):
        root = (rng.uniform(margin, max(Lx - margin, margin + 1e-9)),
                rng.uniform(margin, max(Ly - margin, margin + 1e-9)), 0.0)
        lines.append(_stem(root, height, n_cv, rng.uniform(0.0, 0.03),
                           np.deg2rad(rng.uniform(-15.0, 15.0))))
        lens.append(np.full(n_cv, height / n_cv))
    P = np.concatenate(lines, axis=1)
    Pdot = rng.normal(0.0, 0.02, size=P.shape)
    beams = _beams_from_lines(lines, lens, d=0.006, cdn=1.2, cdt=0.01, eps=eps,
                              ell_s=3 * eps + h)
    return Workload(f"{name}_{nx}x{ny}x{nz}_{n_stems}x{n_cv}", grid, beams,
                    StepInput(U=U.astype(np.float32), P=P.astype(np.float32),
                              Pdot=Pdot.astype(np.float32)),
                    meta={"eps_cells": eps_cells})


def with_inertia(wl: Workload, seed: int, *, cm_n: float = 1.0, cm_t: float = 0.1, dt: float = 1e-3,
                 accel: float = 2.0) -> Workload:
    """The same workload with the Morison inertia inputs: added-mass
    coefficients on every line, the velocity one step dt earlier
    (U_prev = U - dt a with a a smooth random acceleration field of RMS
    `accel` m/s^2) and random actuator-point accelerations of RMS accel/2."""
    rng = _rng(seed)
    g = wl.grid
    a = _solenoidal_modes(rng, g, 4, 4).astype(np.float64)
    a *= accel / max(float(np.sqrt((a ** 2).mean())), 1e-30)
    dtype = wl.step.U.dtype
    U_prev = (wl.step.U.astype(np.float64) - dt * a).astype(dtype)
    Pddot = rng.normal(0.0, 0.5 * accel, size=wl.step.P.shape).astype(wl.step.P.dtype)
    nl = wl.beams.n_lines
    beams = replace(wl.beams, cm_n=np.full(nl, float(cm_n)), cm_t=np.full(nl, float(cm_t)))
    return replace(wl, name=wl.name + "_inertia", beams=beams,
                   step=replace(wl.step, U_prev=U_prev, Pddot=Pddot, dt=float(dt)))


def with_sample_mode(wl: Workload, mode: str) -> Workload:
    """The same workload with another sampling operator on every line
    ("trilinear", "cell" or "gauss")."""
    m = {"trilinear": SAMPLE_TRILINEAR, "cell": SAMPLE_CELL, "gauss": SAMPLE_GAUSS}[mode]
    return replace(wl, name=f"{wl.name}_{mode}" if m != wl.beams.sample_mode else wl.name,
                   beams=replace(wl.beams, sample_mode=m))


REFLECT_X_LO, REFLECT_X_HI, REFLECT_Y_LO, REFLECT_Y_HI, REFLECT_Z_LO, REFLECT_Z_HI = (1 << a for a in range(6))


def with_reflect(wl: Workload, mask: int) -> Workload:
    """The same workload with the kernel reflected at the grid faces in
    `mask` (REFLECT_* bits; 0: the paper's truncated kernel)."""
    return replace(wl, name=f"{wl.name}_reflect{mask}" if mask else wl.name,
                   beams=replace(wl.beams, wall_reflect=int(mask)))


def with_projection(wl: Workload, mode: str) -> Workload:
    """The same workload with another projection ("nearest" or "integrated")."""
    m = {"nearest": 0, "integrated": 1}[mode]
    return replace(wl, name=f"{wl.name}_{mode}" if m != wl.beams.proj_mode else wl.name,
                   beams=replace(wl.beams, proj_mode=m))


def advance(wl: Workload, seed: int, dt: float = 1e-3) -> Workload:
    """Next coupling step of a served simulation: positions move by
    Pdot * dt plus N(0, (1e-4 h)^2) jitter (a synthetic beam update)."""
    rng = _rng(seed)
    P = wl.step.P.astype(np.float64)
    P = P + wl.step.Pdot.astype(np.float64) * dt + rng.normal(0.0, 1e-4 * wl.grid.h, size=P.shape)
    return replace(wl, step=replace(wl.step, P=P.astype(wl.step.P.dtype)))


CONFIGS = {
    "plain": make_plain,
    "canopy": make_canopy,
    "flume": make_flume,
}
