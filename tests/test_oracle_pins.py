"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong sign, a transposed index or operand, a wrong normalisation)
fails at least one of them.  None of them compares the oracle with itself
under a re-typed formula: they use closed forms, exact reproductions,
invariants, brute force and the golden values under tests/golden/.
"""
import os
from dataclasses import replace

import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W
from paper_2609_39443_b300.workloads import BeamSpec, GridSpec, StepInput, Workload

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def _beams(line_off, cv_len, **kw):
    n = len(line_off) - 1
    base = dict(d=0.01, cdn=1.2, cdt=0.01, eps=0.02, ell_s=0.07, alpha_f=1.0)
    base.update(kw.pop("per_line", {}))
    arrs = {k: np.full(n, float(v)) if np.ndim(v) == 0 else np.asarray(v, float) for k, v in base.items()}
    return BeamSpec(line_off=np.asarray(line_off, np.int32), cv_len=np.asarray(cv_len, float), **arrs, **kw)


def _uniform(grid, u):
    U = np.zeros((3, grid.n_cells))
    for a in range(3):
        U[a] = u[a]
    return U


# ----------------------------------------------------------------------------
# sampling (Eqs. almPreliminaryVelocity, almRelativeVelocity; trilinear reading)
# ----------------------------------------------------------------------------

def test_trilinear_reproduces_affine_fields():
    rng = np.random.default_rng(1)
    g = GridSpec(7, 5, 6, 0.1, origin=(0.3, -0.2, 1.0))
    idx = np.arange(g.n_cells)
    i, j, k = idx % g.nx, (idx // g.nx) % g.ny, idx // (g.nx * g.ny)
    xc = np.stack([g.origin[0] + (i + .5) * g.h, g.origin[1] + (j + .5) * g.h, g.origin[2] + (k + .5) * g.h])
    A = rng.normal(size=(3, 3))
    b = rng.normal(size=3)
    U = A @ xc + b[:, None]
    for _ in range(200):
        # interior points (at least half a cell from the walls): exact
        p = np.array(g.origin) + (0.5 + rng.uniform(0, 1, 3) * (np.array([g.nx, g.ny, g.nz]) - 1)) * g.h
        ok, v = oracle.sample(g, U, 0, p)
        assert ok
        np.testing.assert_allclose(v, A @ p + b, rtol=0, atol=1e-12)


def test_trilinear_cell_centres_and_wall_extension():
    rng = np.random.default_rng(2)
    g = GridSpec(4, 3, 5, 0.5)
    f = rng.normal(size=(1, g.n_cells))
    for c in [(0, 0, 0), (3, 2, 4), (1, 2, 3)]:
        p = (np.array(c) + 0.5) * g.h
        ok, v = oracle.sample(g, f, 0, p)
        assert ok and v[0] == pytest.approx(f[0, c[0] + g.nx * (c[1] + g.ny * c[2])], abs=1e-14)
    # in the half cell next to the x = 0 wall the wall cell's value is extended
    fx = np.tile(np.arange(g.nx, dtype=float) * 3.0 + 1.0, g.ny * g.nz)[None]
    ok, v = oracle.sample(g, fx, 0, np.array([0.1, 0.7, 1.3]) * g.h + np.array([0, 0, 0]))
    assert ok and v[0] == pytest.approx(1.0, abs=1e-14)


def test_cell_mode_returns_the_containing_cell():
    rng = np.random.default_rng(3)
    g = GridSpec(6, 4, 5, 0.25, origin=(1.0, 2.0, -1.0))
    f = rng.normal(size=(3, g.n_cells))
    for _ in range(100):
        c = rng.integers([0, 0, 0], [g.nx, g.ny, g.nz])
        frac = rng.uniform(0.05, 0.95, 3)
        p = np.array(g.origin) + (c + frac) * g.h
        ok, v = oracle.sample(g, f, 1, p)
        assert ok
        np.testing.assert_array_equal(v, f[:, c[0] + g.nx * (c[1] + g.ny * c[2])])
    # a point on a face goes to the upper cell (floor rule)
    ok, v = oracle.sample(g, f, 1, np.array(g.origin) + np.array([2.0, 1.5, 3.25]) * g.h)
    np.testing.assert_array_equal(v, f[:, 2 + g.nx * (1 + g.ny * 3)])


def test_outside_points_are_reported():
    g = GridSpec(4, 4, 4, 1.0)
    f = np.ones((1, g.n_cells))
    assert not oracle.sample(g, f, 0, [-1e-9, 1, 1])[0]
    assert not oracle.sample(g, f, 0, [4.0, 1, 1])[0]
    assert oracle.sample(g, f, 0, [0.0, 1, 3.999999])[0]


# ----------------------------------------------------------------------------
# kernel-weighted volume average (sampling mode 2, the smooth sampler of Sec. 6)
# ----------------------------------------------------------------------------

def _centres(g):
    idx = np.arange(g.n_cells)
    i, j, k = idx % g.nx, (idx // g.nx) % g.ny, idx // (g.nx * g.ny)
    return np.stack([g.origin[0] + (i + .5) * g.h, g.origin[1] + (j + .5) * g.h, g.origin[2] + (k + .5) * g.h])


def test_gauss_average_weights_are_the_truncated_gaussian():
    """Sampling the identity field (one component per cell) returns every
    cell's normalised weight at once.  The weights are positive exactly on
    the cells whose centre lies within 3 eps of p (walls included), sum to
    one, and the ratio of any two is exp(-(r_a^2 - r_b^2) / eps^2), which
    does not involve the normaliser."""
    rng = np.random.default_rng(11)
    g = GridSpec(9, 8, 10, 0.1, origin=(0.3, -0.2, 0.1))
    ident = np.eye(g.n_cells)
    C = _centres(g)
    for eps in (0.07, 0.13, 0.21):
        for _ in range(4):
            p = np.array(g.origin) + rng.uniform(0.1, 0.9, 3) * np.array([g.nx, g.ny, g.nz]) * g.h
            ok, w = oracle.sample(g, ident, W.SAMPLE_GAUSS, p, eps)
            assert ok
            r2 = ((C - p[:, None]) ** 2).sum(0)
            inside = r2 <= (3 * eps) ** 2
            assert np.array_equal(w > 0, inside)
            assert w.sum() == pytest.approx(1.0, abs=1e-14)
            a = np.flatnonzero(inside)
            k0 = a[np.argmin(r2[a])]
            np.testing.assert_allclose(w[a] / w[k0], np.exp(-(r2[a] - r2[k0]) / eps ** 2), rtol=1e-12)


def test_gauss_average_reproduces_affine_fields_at_symmetric_points():
    """About a cell centre, a cell corner or the middle of an edge or a face
    the lattice of centres and the Gaussian weights are mirror-symmetric on
    every axis, so with the support inside the grid the weighted centroid
    is p itself and an affine field is reproduced; elsewhere the centroid
    is not p and in general it is not."""
    rng = np.random.default_rng(12)
    g = GridSpec(16, 15, 17, 0.05, origin=(-0.4, 0.2, 0.0))
    A = rng.normal(size=(3, 3))
    b = rng.normal(size=3)
    U = A @ _centres(g) + b[:, None]
    eps = 0.08                                     # 3 eps = 4.8 cells
    for frac in [(0.5, 0.5, 0.5), (0, 0, 0), (0.5, 0, 0), (0, 0.5, 0.5), (0.5, 0.5, 0)]:
        p = np.array(g.origin) + (np.array([8, 7, 8]) + np.array(frac)) * g.h
        ok, v = oracle.sample(g, U, W.SAMPLE_GAUSS, p, eps)
        assert ok
        np.testing.assert_allclose(v, A @ p + b, rtol=0, atol=1e-12)
    p = np.array(g.origin) + np.array([8.3, 7.1, 8.2]) * g.h
    assert np.abs(oracle.sample(g, U, W.SAMPLE_GAUSS, p, eps)[1] - (A @ p + b)).max() > 1e-6


def test_gauss_average_of_a_constant_field_at_walls():
    """Near a wall the support is cut and the weights renormalise over the
    cells present: a constant field is still returned exactly."""
    g = GridSpec(8, 6, 7, 0.1)
    f = np.stack([np.full(g.n_cells, 1.7), np.full(g.n_cells, -0.3)])
    for p in ([0.001, 0.001, 0.001], [0.79, 0.3, 0.35], [0.4, 0.599, 0.699]):
        ok, v = oracle.sample(g, f, W.SAMPLE_GAUSS, np.array(p), 0.12)
        assert ok
        np.testing.assert_allclose(v, [1.7, -0.3], rtol=1e-14)
    assert not oracle.sample(g, f, W.SAMPLE_GAUSS, np.array([0.8, 0.3, 0.3]), 0.12)[0]


def test_gauss_average_narrow_kernel_is_the_containing_cell():
    """As eps -> 0 the normalised average tends to the value at the nearest
    cell centre, the containing cell's.  With 3 eps below half a cell no
    other centre can enter; when not even that one does, the containing
    cell's value is returned too."""
    rng = np.random.default_rng(13)
    g = GridSpec(6, 5, 7, 0.2, origin=(1.0, 2.0, -1.0))
    f = rng.normal(size=(3, g.n_cells))
    for _ in range(100):
        c = rng.integers([0, 0, 0], [g.nx, g.ny, g.nz])
        p = np.array(g.origin) + (c + rng.uniform(0.05, 0.95, 3)) * g.h
        ref = f[:, c[0] + g.nx * (c[1] + g.ny * c[2])]
        for eps in (0.01, 0.03):                   # 3 eps = 0.15 h and 0.45 h
            ok, v = oracle.sample(g, f, W.SAMPLE_GAUSS, p, eps)
            assert ok
            np.testing.assert_allclose(v, ref, rtol=1e-15, atol=0)


def test_gauss_average_is_continuous_across_faces():
    """The containing cell's value jumps where the point crosses a face; the
    volume average moves only by O(|step| / eps) plus at most the weight
    e^-9 of a cell leaving the truncated support."""
    rng = np.random.default_rng(14)
    g = GridSpec(12, 12, 12, 0.1)
    f = rng.normal(size=(1, g.n_cells))
    for x0 in (0.6, 0.3):
        xs = x0 + np.array([-1e-7, 1e-7])
        cell = [oracle.sample(g, f, W.SAMPLE_CELL, np.array([x, 0.63, 0.57]))[1][0] for x in xs]
        avg = [oracle.sample(g, f, W.SAMPLE_GAUSS, np.array([x, 0.63, 0.57]), 0.15)[1][0] for x in xs]
        assert abs(cell[1] - cell[0]) > 1e-3
        assert abs(avg[1] - avg[0]) < 1e-4


# ----------------------------------------------------------------------------
# tangent, sampling point and fallback (Sec. 3.2.2, Eq. almSamplingPoint)
# ----------------------------------------------------------------------------

def _line_workload(P, U, Pdot=None, grid=None, **beamkw):
    grid = grid or GridSpec(40, 40, 40, 0.01)
    n = P.shape[1]
    b = _beams([0, n], np.full(n, beamkw.pop("cv", 0.01)), **beamkw)
    return Workload("pin", grid, b, StepInput(U=U, P=P, Pdot=np.zeros_like(P) if Pdot is None else Pdot))


def test_tangent_straight_line_and_circle():
    g = GridSpec(40, 40, 40, 0.01)
    d = np.array([0.3, -0.4, 0.866])
    d /= np.linalg.norm(d)
    P = np.array([0.2, 0.2, 0.05])[:, None] + 0.01 * np.arange(9)[None] * d[:, None]
    r = oracle.point_step(g, _line_workload(P, _uniform(g, (0.5, 0, 0))).beams,
                          _line_workload(P, _uniform(g, (0.5, 0, 0))).step)
    np.testing.assert_allclose(r["e_t"], np.repeat(d[:, None], 9, axis=1), atol=1e-14)
    # equally spaced points on a circle: interior tangents are perpendicular to the radius
    th = np.linspace(0.2, 2.0, 12)
    c0 = np.array([0.2, 0.2, 0.2])
    P = c0[:, None] + 0.05 * np.stack([np.cos(th), np.sin(th), 0 * th])
    wl = _line_workload(P, _uniform(g, (0.5, 0, 0)))
    et = oracle.point_step(g, wl.beams, wl.step)["e_t"]
    radial = P - c0[:, None]
    np.testing.assert_allclose((et[:, 1:-1] * radial[:, 1:-1]).sum(0), 0, atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(et, axis=0), 1, atol=1e-14)
    np.testing.assert_allclose(et[:, 0], (P[:, 1] - P[:, 0]) / np.linalg.norm(P[:, 1] - P[:, 0]), atol=1e-15)


def test_sampling_point_in_uniform_flow_is_straight_upstream():
    g = GridSpec(40, 40, 40, 0.01)
    P = np.stack([np.full(10, 0.2), np.full(10, 0.2), 0.05 + 0.01 * np.arange(10)])
    wl = _line_workload(P, _uniform(g, (0.5, 0.0, 0.0)), per_line=dict(ell_s=0.07))
    r = oracle.point_step(g, wl.beams, wl.step)
    np.testing.assert_allclose(r["P_s"], P - np.array([0.07, 0, 0])[:, None], atol=1e-15)
    assert r["status"][oracle.ST_FALLBACK] == 0


def test_sampling_plane_projection_bounds_the_offset():
    rng = np.random.default_rng(4)
    g = GridSpec(40, 40, 40, 0.01)
    U = _uniform(g, (0.4, 0.3, 0.0)) + rng.normal(0, 0.01, size=(3, g.n_cells))
    P = np.stack([np.full(10, 0.2), np.full(10, 0.2), 0.05 + 0.01 * np.arange(10)])
    wl = _line_workload(P, U, per_line=dict(ell_s=0.07), n_p=(0.0, 1.0, 0.0))
    r = oracle.point_step(g, wl.beams, wl.step)
    off = r["P_s"] - P
    np.testing.assert_allclose(off[1], 0.0, atol=1e-16)
    assert (np.linalg.norm(off, axis=0) <= 0.07 + 1e-15).all()
    assert (np.linalg.norm(off, axis=0) < 0.07 - 1e-3).all()     # y part removed, not renormalised


def test_fallback_direction():
    g = GridSpec(40, 40, 40, 0.01)
    P = np.stack([np.full(6, 0.2), np.full(6, 0.2), 0.1 + 0.01 * np.arange(6)])
    U = _uniform(g, (0.3, 0.1, 0.2))
    Pdot = np.repeat(np.array([0.3, 0.1, 0.2])[:, None], 6, axis=1)   # no relative flow
    wl = _line_workload(P, U, Pdot, per_line=dict(ell_s=0.05), g_up=(-1.0, 0.0, 1.0))
    r = oracle.point_step(g, wl.beams, wl.step)
    assert r["status"][oracle.ST_FALLBACK] == 6
    # g_up projected on the cross-section plane (perpendicular to z) and renormalised
    np.testing.assert_allclose(r["P_s"] - P, np.repeat(np.array([-0.05, 0, 0])[:, None], 6, 1), atol=1e-15)
    np.testing.assert_allclose(r["F"], 0.0, atol=1e-30)
    wl = _line_workload(P, U, Pdot, per_line=dict(ell_s=0.05), g_up=(0.0, 0.0, 1.0))
    r = oracle.point_step(g, wl.beams, wl.step)
    assert r["status"][oracle.ST_FALLBACK_ZERO] == 6
    np.testing.assert_allclose(r["P_s"], P, atol=0)


# ----------------------------------------------------------------------------
# line force (Eqs. almLineForce, fext_drag, almForceRelaxation)
# ----------------------------------------------------------------------------

def test_cylinder_drag_golden():
    gd = _golden("cylinder_drag.txt")
    n = int(gd["n_cv"])
    g = GridSpec(64, 32, 32, 0.01, rho_const=gd["rho"])
    P = np.stack([np.full(n, 0.2), np.full(n, 0.16), (np.arange(n) + 0.5) * gd["length"] / n])
    wl = _line_workload(P, _uniform(g, (gd["U0"], 0, 0)), grid=g, cv=gd["length"] / n,
                        per_line=dict(d=gd["d"], cdn=gd["cdn"], cdt=0.37))
    r = oracle.point_step(g, wl.beams, wl.step)
    np.testing.assert_allclose(r["F"][0], gd["F_per_cv"], rtol=1e-14)
    np.testing.assert_allclose(r["F"][1:], 0.0, atol=1e-18)
    np.testing.assert_allclose(r["f"][0], gd["f_per_length"], rtol=1e-14)
    assert r["F"][0].sum() == pytest.approx(gd["F_total"], rel=1e-14)


@pytest.mark.parametrize("sample_mode", [W.SAMPLE_TRILINEAR, W.SAMPLE_CELL, W.SAMPLE_GAUSS])
@pytest.mark.parametrize("drag_mode", [W.DRAG_DISCRETE, W.DRAG_SPLIT])
def test_inclined_cylinder_closed_form(drag_mode, sample_mode):
    theta = 0.6                                     # angle between line and flow
    U0, rho, d, cdn, cdt = 0.7, 1000.0, 0.01, 1.3, 0.05
    g = GridSpec(60, 20, 60, 0.01, rho_const=rho)
    t = np.array([np.cos(theta), 0.0, np.sin(theta)])
    P = np.array([0.2, 0.1, 0.2])[:, None] + 0.01 * np.arange(8)[None] * t[:, None]
    wl = _line_workload(P, _uniform(g, (U0, 0, 0)), grid=g, cv=0.01,
                        per_line=dict(d=d, cdn=cdn, cdt=cdt), drag_mode=drag_mode, sample_mode=sample_mode)
    F = oracle.point_step(g, wl.beams, wl.step)["F"] / 0.01
    Ut = U0 * np.cos(theta) * t
    Un = np.array([U0, 0, 0]) - Ut
    if drag_mode == W.DRAG_DISCRETE:      # |U_r| (C_dn U_n + C_dt U_t)
        f = 0.5 * rho * d * U0 * (cdn * Un + cdt * Ut)
    else:                                 # C_dn |U_n| U_n + C_dt |U_t| U_t
        f = 0.5 * rho * d * (cdn * np.linalg.norm(Un) * Un + cdt * np.linalg.norm(Ut) * Ut)
    np.testing.assert_allclose(F, np.repeat(f[:, None], 8, 1), rtol=1e-13, atol=1e-15)
    # normal magnitude: 1/2 rho d C_dn U0^2 sin(theta) vs ... sin^2(theta)
    p = 1 if drag_mode == W.DRAG_DISCRETE else 2
    assert np.linalg.norm(F[:, 3] - (F[:, 3] @ t) * t) == pytest.approx(0.5 * rho * d * cdn * U0 ** 2 * np.sin(theta) ** p, rel=1e-13)


# ----------------------------------------------------------------------------
# inertia (Eq. fext_addedmass; the paper's model has C_Mn = C_Mt = 0)
# ----------------------------------------------------------------------------

def _inertia_workload(P, U, U_prev, dt, *, Pddot=None, cm_n=1.0, cm_t=0.0, cdn=0.0, cdt=0.0, rho=1000.0, d=0.02):
    g = GridSpec(60, 24, 60, 0.01, rho_const=rho)
    wl = _line_workload(P, U, grid=g, cv=0.01, per_line=dict(d=d, cdn=cdn, cdt=cdt))
    wl.beams.cm_n = np.full(1, float(cm_n))
    wl.beams.cm_t = np.full(1, float(cm_t))
    wl.step.U_prev, wl.step.dt = U_prev, dt
    wl.step.Pddot = Pddot
    return wl


def _vertical(n=8):
    return np.stack([np.full(n, 0.3), np.full(n, 0.12), 0.1 + 0.01 * np.arange(n)])


@pytest.mark.parametrize("cm_n", [0.0, 1.0, 0.7])
def test_inertia_in_uniformly_accelerating_flow(cm_n):
    """A fixed cylinder in a uniform flow accelerating at a: f = rho A (1 + C_Mn) a
    (the classical Morison inertia coefficient; 1 is the Froude-Krylov part)."""
    rho, d, a, dt, U0 = 1000.0, 0.02, 0.8, 0.01, 0.3
    P = _vertical()
    g = GridSpec(60, 24, 60, 0.01, rho_const=rho)
    wl = _inertia_workload(P, _uniform(g, (U0, 0, 0)), _uniform(g, (U0 - a * dt, 0, 0)), dt, cm_n=cm_n)
    f = oracle.point_step(wl.grid, wl.beams, wl.step)["f"]
    A = np.pi * d * d / 4
    np.testing.assert_allclose(f[0], rho * A * (1.0 + cm_n) * a, rtol=1e-12)
    np.testing.assert_allclose(f[1:], 0.0, atol=1e-12)


def test_inertia_of_an_accelerating_cylinder_in_still_fluid():
    """The added mass opposes the body's acceleration: f = -rho A C_Mn a_b."""
    rho, d, cm = 1000.0, 0.02, 1.3
    P = _vertical()
    g = GridSpec(60, 24, 60, 0.01, rho_const=rho)
    ab = np.array([0.5, -0.2, 0.0])
    wl = _inertia_workload(P, _uniform(g, (0, 0, 0)), _uniform(g, (0, 0, 0)), 0.01,
                           Pddot=np.repeat(ab[:, None], P.shape[1], 1), cm_n=cm, cm_t=0.4)
    f = oracle.point_step(wl.grid, wl.beams, wl.step)["f"]
    A = np.pi * d * d / 4
    np.testing.assert_allclose(f, np.repeat((-rho * A * cm * ab)[:, None], P.shape[1], 1), rtol=1e-12, atol=1e-15)


def test_inertia_splits_along_the_tangent():
    """An inclined cylinder in flow accelerating along x: the tangential and
    normal parts of the acceleration take C_Mt and C_Mn, the Froude-Krylov
    part is along x."""
    theta, rho, d, a, dt, cmn, cmt = 0.5, 1000.0, 0.02, 0.9, 0.02, 1.1, 0.25
    t = np.array([np.cos(theta), 0.0, np.sin(theta)])
    P = np.array([0.2, 0.12, 0.2])[:, None] + 0.01 * np.arange(8)[None] * t[:, None]
    g = GridSpec(60, 24, 60, 0.01, rho_const=rho)
    wl = _inertia_workload(P, _uniform(g, (0.4, 0, 0)), _uniform(g, (0.4 - a * dt, 0, 0)), dt,
                           cm_n=cmn, cm_t=cmt)
    f = oracle.point_step(wl.grid, wl.beams, wl.step)["f"]
    af = np.array([a, 0.0, 0.0])
    at = (af @ t) * t
    want = rho * np.pi * d * d / 4 * (cmt * at + cmn * (af - at) + af)
    np.testing.assert_allclose(f, np.repeat(want[:, None], 8, 1), rtol=1e-12, atol=1e-14)


def test_inertia_adds_to_the_drag():
    """Drag from the current velocity plus the inertia term, nothing else."""
    rho, d, a, dt, U0, cdn = 1000.0, 0.02, 0.6, 0.01, 0.5, 1.2
    P = _vertical()
    g = GridSpec(60, 24, 60, 0.01, rho_const=rho)
    wl = _inertia_workload(P, _uniform(g, (U0, 0, 0)), _uniform(g, (U0 - a * dt, 0, 0)), dt, cm_n=1.0, cdn=cdn)
    f = oracle.point_step(wl.grid, wl.beams, wl.step)["f"]
    want = 0.5 * rho * d * cdn * U0 * U0 + rho * np.pi * d * d / 4 * 2.0 * a
    np.testing.assert_allclose(f[0], want, rtol=1e-12)


def test_relative_velocity_is_galilean():
    rng = np.random.default_rng(5)
    wl = W.make_random(11, 24, 20, 22, n_lines=3, kinds=("stem",))
    c = np.array([0.13, -0.07, 0.05])
    wl2 = Workload("s", wl.grid, wl.beams, StepInput(U=wl.step.U + c[:, None], P=wl.step.P,
                                                      Pdot=wl.step.Pdot + c[:, None]))
    # upstream direction and forces depend on U - Pdot only (field noise is the same)
    r1 = oracle.point_step(wl.grid, wl.beams, wl.step)
    r2 = oracle.point_step(wl2.grid, wl2.beams, wl2.step)
    np.testing.assert_allclose(r2["F"], r1["F"], rtol=1e-9, atol=1e-12)
    # moving the beam with the flow reduces the load; a sign error would increase it
    wl3 = Workload("s", wl.grid, wl.beams, StepInput(U=wl.step.U, P=wl.step.P,
                                                      Pdot=wl.step.Pdot + np.array([0.2, 0, 0])[:, None]))
    r3 = oracle.point_step(wl3.grid, wl3.beams, wl3.step)
    assert r3["F"][0].sum() < r1["F"][0].sum()
    del rng


def test_relaxation_blend():
    wl = W.make_random(12, 24, 20, 22, n_lines=2, kinds=("stem",))
    r0 = oracle.point_step(wl.grid, wl.beams, wl.step)
    f_prev = np.random.default_rng(6).normal(size=r0["f"].shape)
    r1 = oracle.point_step(wl.grid, wl.beams, wl.step, f_prev=f_prev)
    af = np.repeat(wl.beams.alpha_f, np.diff(wl.beams.line_off))
    np.testing.assert_allclose(r1["f"], af * r0["f"] + (1 - af) * f_prev, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(r1["F"], r1["f"] * wl.beams.cv_len, rtol=1e-14)


def test_mixture_density():
    g = GridSpec(40, 40, 40, 0.01, has_alpha=True, rho1=1000.0, rho2=1.2)
    P = np.stack([np.full(5, 0.2), np.full(5, 0.2), 0.1 + 0.01 * np.arange(5)])
    out = {}
    for a in (1.0, 0.0, 0.3):
        wl = _line_workload(P, _uniform(g, (0.5, 0, 0)), grid=g)
        wl.step.alpha = np.full(g.n_cells, a)
        out[a] = oracle.point_step(g, wl.beams, wl.step)["F"][0]
    np.testing.assert_allclose(out[0.0] / out[1.0], 1.2 / 1000.0, rtol=1e-13)
    np.testing.assert_allclose(out[0.3] / out[1.0], (0.3 * 1000 + 0.7 * 1.2) / 1000.0, rtol=1e-13)


# ----------------------------------------------------------------------------
# projection (Eqs. almProjectionPoint, almGaussian, almMomentumSource)
# ----------------------------------------------------------------------------

def test_closest_segment_against_dense_polyline_sampling():
    rng = np.random.default_rng(7)
    for trial in range(30):
        n = int(rng.integers(2, 12))
        X = np.cumsum(rng.normal(size=(3, n)), axis=1)
        c = rng.normal(size=3) * 2 + X.mean(axis=1)
        k, s, r = oracle.closest_segment(X, c)
        # brute force: 20001 points on every segment
        tt = np.linspace(0, 1, 20001)
        best = np.inf
        for j in range(n - 1):
            pts = X[:, j, None] + tt[None] * (X[:, j + 1] - X[:, j])[:, None]
            dd = np.linalg.norm(pts - c[:, None], axis=0)
            best = min(best, dd.min())
        assert r <= best + 1e-12
        assert r == pytest.approx(best, abs=1e-3 * np.linalg.norm(np.diff(X, axis=1), axis=0).max())
        foot = X[:, k] + s * (X[:, k + 1] - X[:, k])
        assert np.linalg.norm(foot - c) == pytest.approx(r, rel=1e-12)
        assert 0.0 <= s <= 1.0


def _straight_z_line(g, x, y, z0, dz, n, F):
    P = np.stack([np.full(n, x), np.full(n, y), z0 + dz * np.arange(n)])
    b = _beams([0, n], np.full(n, dz), per_line=dict(eps=2 * g.h))
    return b, P, np.asarray(F, float)


def test_gaussian_shape_between_cells_of_one_segment():
    g = GridSpec(24, 24, 24, 1.0)
    # line along z through cell centres (x, y) = (12.5, 12.5); nodes every 2 cells
    n = 6
    F = np.zeros((3, n)); F[0] = 1.0
    b, P, F = _straight_z_line(g, 12.5, 12.5, 4.5, 2.0, n, F)
    S = oracle.project(g, b, P, F)["S"][0].reshape(g.nz, g.ny, g.nx)
    eps = 2.0
    # cells at the same height (same segment and s) at r = 1 and r = sqrt(5), 2
    s0 = S[9, 12, 12]
    np.testing.assert_allclose(S[9, 12, 13] / s0, np.exp(-(1.0 ** 2) / eps ** 2), rtol=1e-13)
    np.testing.assert_allclose(S[9, 13, 14] / s0, np.exp(-5.0 / eps ** 2), rtol=1e-13)
    np.testing.assert_allclose(S[9, 12, 10] / s0, np.exp(-4.0 / eps ** 2), rtol=1e-13)
    # cut-off at r = 3 eps = 6 is inclusive: (6, 0) kept, (6, 1) dropped
    assert S[9, 12, 18] != 0.0 and S[9, 13, 18] == 0.0
    np.testing.assert_allclose(S[9, 12, 18] / s0, np.exp(-9.0), rtol=1e-12)
    # the source opposes the load (minus sign of Eq. almMomentumSource)
    assert s0 < 0


def test_nodal_interpolation_weights():
    g = GridSpec(24, 24, 24, 1.0)
    n = 4
    F = np.zeros((3, n)); F[0] = [1.0, 3.0, -2.0, 5.0]; F[2] = [0.5, 0.0, 1.5, -1.0]
    b, P, F = _straight_z_line(g, 12.5, 12.5, 6.5, 4.0, n, F)
    r = oracle.project(g, b, P, F)
    S, w = r["S"], r["w"]
    fhat = F / w
    eps = 2.0
    for z, seg, s in [(7, 0, 0.25), (9, 0, 0.75), (12, 1, 0.5), (17, 2, 0.75)]:
        for (x, y) in [(12, 12), (13, 12), (12, 10)]:
            rr2 = (x - 12) ** 2 + (y - 12) ** 2
            eta = np.exp(-rr2 / eps ** 2) / (np.pi * eps ** 2)
            want = -eta * ((1 - s) * fhat[:, seg] + s * fhat[:, seg + 1])
            np.testing.assert_allclose(S[:, x + 24 * (y + 24 * z)], want, rtol=1e-12, atol=1e-15)


def test_gaussian_normalisation_converges_to_truncated_integral():
    gd = _golden("gaussian_truncation.txt")
    g = GridSpec(40, 40, 30, 1.0)
    n = 11
    eps = 4.0
    P = np.stack([np.full(n, 20.0), np.full(n, 20.0), 4.5 + 2.0 * np.arange(n)])
    b = _beams([0, n], np.full(n, 2.0), per_line=dict(eps=eps))
    F = np.ones((3, n))
    w = oracle.project(g, b, P, F)["w"]
    # interior nodes: w_k -> L_k (1 - e^-9) for a well-resolved kernel
    np.testing.assert_allclose(w[3:-3] / 2.0, gd["retained_fraction"], rtol=2e-4)
    assert np.exp(-9.0) == pytest.approx(gd["discarded_fraction"], rel=1e-15)


def test_conservation_on_random_lines():
    for seed in range(6):
        wl = W.make_random(100 + seed, 26, 22, 20, n_lines=5, precision="fp64",
                           kinds=("stem", "arc", "random", "flat", "point", "dup"))
        r = oracle.sample_drag_spread(wl)
        F, SV = r["totals"][:3], r["totals"][3:]
        scale = np.abs(r["F"]).sum()
        lost = r["status"][oracle.ST_DEPOSIT_LOST]
        if lost == 0:
            assert np.abs(F + SV).max() <= 1e-12 * scale


def test_cull_has_no_effect_bitwise():
    for seed in range(4):
        wl = W.make_random(200 + seed, 16, 14, 12, n_lines=3, precision="fp64",
                           kinds=("stem", "arc", "random", "point"))
        ps = oracle.point_step(wl.grid, wl.beams, wl.step)
        a = oracle.project(wl.grid, wl.beams, wl.step.P, ps["F"], cull=True)
        b = oracle.project(wl.grid, wl.beams, wl.step.P, ps["F"], cull=False)
        np.testing.assert_array_equal(a["S"], b["S"])
        np.testing.assert_array_equal(a["w"], b["w"])


def test_superposition_over_lines_and_linearity():
    wl = W.make_random(300, 26, 22, 20, n_lines=4, precision="fp64", kinds=("stem", "arc"))
    ps = oracle.point_step(wl.grid, wl.beams, wl.step)
    full = oracle.project(wl.grid, wl.beams, wl.step.P, ps["F"])["S"]
    acc = np.zeros_like(full)
    for l in range(wl.beams.n_lines):
        m = np.zeros(wl.beams.n_lines, np.uint8); m[l] = 1
        acc += oracle.project(wl.grid, wl.beams, wl.step.P, ps["F"], line_mask=m)["S"]
    np.testing.assert_allclose(acc, full, rtol=1e-13, atol=1e-13 * np.abs(full).max())
    s2 = oracle.project(wl.grid, wl.beams, wl.step.P, -2.5 * ps["F"])["S"]
    np.testing.assert_allclose(s2, -2.5 * full, rtol=1e-14, atol=1e-14 * np.abs(full).max())


def test_integer_translation_and_mirror():
    g = GridSpec(20, 20, 20, 0.25)
    rng = np.random.default_rng(8)
    n = 7
    # dyadic coordinates so the translated set-up is represented exactly
    P = np.stack([2.5 + np.round(rng.uniform(-0.5, 0.5, n) * 64) / 64,
                  2.0 + np.round(rng.uniform(-0.5, 0.5, n) * 64) / 64,
                  1.75 + 0.25 * np.arange(n)])
    F = rng.normal(size=(3, n))
    b = _beams([0, n], np.full(n, 0.25), per_line=dict(eps=0.5))
    S = oracle.project(g, b, P, F)["S"].reshape(3, 20, 20, 20)
    # shift by (+2, +1, -1) cells; the support stays inside the grid in both positions
    S2 = oracle.project(g, b, P + np.array([0.5, 0.25, -0.25])[:, None], F)["S"].reshape(3, 20, 20, 20)
    np.testing.assert_allclose(S2[:, :-1, 1:, 2:], S[:, 1:, :-1, :-2], rtol=1e-12, atol=1e-12 * np.abs(S).max())
    # mirror y -> 5 - y (the grid spans [0, 5]): S_y flips, x and z are mirrored copies
    Pm = P.copy(); Pm[1] = 5.0 - P[1]
    Fm = F.copy(); Fm[1] = -F[1]
    Sm = oracle.project(g, b, Pm, Fm)["S"].reshape(3, 20, 20, 20)
    np.testing.assert_allclose(Sm[0], S[0][:, ::-1, :], rtol=1e-12, atol=1e-12 * np.abs(S).max())
    np.testing.assert_allclose(Sm[1], -S[1][:, ::-1, :], rtol=1e-12, atol=1e-12 * np.abs(S).max())
    np.testing.assert_allclose(Sm[2], S[2][:, ::-1, :], rtol=1e-12, atol=1e-12 * np.abs(S).max())


def test_zero_weight_nodes_are_deposited():
    g = GridSpec(12, 12, 12, 1.0)
    # kernel much narrower than a cell, nodes away from cell centres: no cell within 3 eps
    P = np.array([[3.2, 5.7, 8.9], [4.1, 4.3, 6.6], [2.2, 6.9, 9.3]])
    F = np.array([[1.0, -2.0, 0.5], [0.3, 0.2, 0.1], [-1.0, 0.0, 2.0]])
    b = _beams([0, 3], np.ones(3), per_line=dict(eps=0.05))
    r = oracle.project(g, b, P, F)
    assert r["status"][oracle.ST_ZERO_WEIGHT] == 3
    np.testing.assert_array_equal(r["w"], 0.0)
    for k in range(3):
        c = np.floor(P[:, k]).astype(int)
        np.testing.assert_allclose(r["S"][:, c[0] + 12 * (c[1] + 12 * c[2])], -F[:, k], rtol=1e-15)
    np.testing.assert_allclose(r["S"].sum(axis=1), -F.sum(axis=1), rtol=1e-14)


def test_plain_config_totals():
    # the plain case without its noise: a straight rigid vertical cylinder at
    # rest in U = (0.5, 0, 0) takes exactly the golden total of Eq.
    # almLineForce, 1/2 rho d C_dn U0^2 L = 0.3 N (tests/golden/cylinder_drag.txt)
    gold = _golden("cylinder_drag.txt")
    wl = W.make_plain(0)
    n = wl.beams.n_points
    P = np.zeros((3, n))
    P[0], P[1] = 0.20, 0.16
    P[2] = np.cumsum(wl.beams.cv_len) - 0.5 * wl.beams.cv_len
    U = np.zeros_like(wl.step.U)
    U[0] = gold["U0"]
    clean = replace(wl, step=replace(wl.step, U=U, P=P, Pdot=np.zeros_like(P)))
    r = oracle.sample_drag_spread(clean)
    assert r["totals"][0] == pytest.approx(gold["F_total"], rel=1e-12)
    assert np.abs(r["totals"][1:3]).max() < 1e-15
    assert np.abs(r["totals"][:3] + r["totals"][3:]).max() < 1e-14
    # the seeded case: U has N(0, 0.05^2) noise per component, so each CV's
    # drag (proportional to |U_r| U_n) varies by about 2 x 0.05 / 0.5 = 20 %
    # and the sum of 20 CVs by 20 % / sqrt(20) = 4.5 %; three standard
    # deviations bound it at 13.5 %
    r = oracle.sample_drag_spread(wl)
    assert np.abs(r["totals"][:3] + r["totals"][3:]).max() < 1e-14
    assert r["totals"][0] == pytest.approx(gold["F_total"], rel=0.135)
    assert (r["status"][:2] == 0).all()


# ----------------------------------------------------------------------------
# segment-integrated projection (the variant Sec. 6 proposes)
# ----------------------------------------------------------------------------

def _g3_moments(c, A, B, eps):
    """Quadrature of the 3-D Gaussian along A -> B: (int G3, int (t/L) G3)."""
    from scipy.integrate import quad
    D = B - A
    L = np.linalg.norm(D)

    def g3(t):
        x = c - (A + t * D / L)
        return np.exp(-(x @ x) / eps ** 2) / (np.pi ** 1.5 * eps ** 3)
    k0 = quad(g3, 0.0, L, epsabs=0, epsrel=1e-13, limit=200)[0]
    k1 = quad(lambda t: t / L * g3(t), 0.0, L, epsabs=0, epsrel=1e-13, limit=200)[0]
    return np.array([k0, k1])


def test_segment_kernel_matches_quadrature():
    rng = np.random.default_rng(21)
    for _ in range(40):
        eps = rng.uniform(0.5, 2.0)
        A, B = rng.normal(size=3), rng.normal(size=3) * 2.0
        c = (A + B) / 2 + rng.normal(size=3) * eps
        np.testing.assert_allclose(oracle.seg_kernel(c, A, B, eps), _g3_moments(c, A, B, eps), rtol=1e-9, atol=1e-300)


def test_segment_kernel_splits_exactly_at_a_node():
    """A segment cut in two at its midpoint carries the same kernel: the
    integrals add, and the midpoint node's share splits linearly."""
    rng = np.random.default_rng(22)
    for _ in range(40):
        eps = rng.uniform(0.3, 1.5)
        A, B = rng.normal(size=3), rng.normal(size=3) * 3.0
        M = (A + B) / 2
        c = M + rng.normal(size=3) * eps
        K = oracle.seg_kernel(c, A, B, eps)
        K1, K2 = oracle.seg_kernel(c, A, M, eps), oracle.seg_kernel(c, M, B, eps)
        wa, wb = K[0] - K[1], K[1]
        wa1, wb1, wa2, wb2 = K1[0] - K1[1], K1[1], K2[0] - K2[1], K2[1]
        np.testing.assert_allclose(K[0], K1[0] + K2[0], rtol=1e-12)
        np.testing.assert_allclose(wa, wa1 + 0.5 * (wb1 + wa2), rtol=1e-11, atol=1e-14 * K[0])
        np.testing.assert_allclose(wb, wb2 + 0.5 * (wb1 + wa2), rtol=1e-11, atol=1e-14 * K[0])


def test_segment_kernel_long_segment_is_the_2d_gaussian():
    """Far from the ends the integral across a long segment is the 2-D
    kernel of Eq. almGaussian, and the first moment places it at t0 / L."""
    eps = 0.7
    A, B = np.array([0.0, 0.0, -50.0]), np.array([0.0, 0.0, 50.0])
    for r, z in ((0.0, 3.0), (0.9, -7.0), (1.8, 20.0)):
        c = np.array([r * 0.6, r * 0.8, z])
        K = oracle.seg_kernel(c, A, B, eps)
        eta = np.exp(-(r / eps) ** 2) / (np.pi * eps ** 2)
        np.testing.assert_allclose(K[0], eta, rtol=1e-12)
        np.testing.assert_allclose(K[1], eta * (z + 50.0) / 100.0, rtol=1e-12)
    # a zero-length segment carries nothing
    assert np.all(oracle.seg_kernel(np.ones(3), A, A, eps) == 0.0)


def _integrated(wl):
    return W.with_projection(wl, "integrated")


def test_integrated_projection_conserves_and_matches_on_one_node_lines():
    for seed in (5, 6):
        wl = W.make_random(seed, 26, 22, 20, n_lines=6, precision="fp64",
                           kinds=("stem", "arc", "random", "point"))
        r0 = oracle.sample_drag_spread(wl)
        r1 = oracle.sample_drag_spread(_integrated(wl))
        F = r1["F"]
        SV = r1["S"].sum(axis=1) * wl.grid.h ** 3
        np.testing.assert_allclose(SV, -F.sum(axis=1), rtol=0, atol=1e-12 * np.abs(F).sum())
        # one-node lines project the same way in both modes
        single = [l for l in range(wl.beams.n_lines) if wl.beams.line_off[l + 1] - wl.beams.line_off[l] == 1]
        for l in single:
            mask = np.zeros(wl.beams.n_lines, np.uint8)
            mask[l] = 1
            a = oracle.project(wl.grid, wl.beams, wl.step.P, r0["F"], line_mask=mask)["S"]
            b = oracle.project(wl.grid, _integrated(wl).beams, wl.step.P, r0["F"], line_mask=mask)["S"]
            np.testing.assert_array_equal(a, b)


def test_integrated_projection_inside_a_straight_line():
    """A long straight line with equal loads.  The integrated kernel gives
    every interior node the weight of its CV length (the nearest-segment
    weights jitter with the number of cell layers each segment's slab holds:
    the seams Sec. 6 names), and inside the line the source is the 2-D
    Gaussian of Eq. almGaussian times the load per length."""
    g = GridSpec(40, 40, 60, 0.01)
    n, L, eps = 41, 0.0125, 0.016
    x0, y0 = 0.2003, 0.1997
    P = np.stack([np.full(n, x0), np.full(n, y0), 0.05 + L * np.arange(n)])
    wl = _line_workload(P, _uniform(g, (0.5, 0, 0)), grid=g, cv=L, per_line=dict(eps=eps))
    F = oracle.point_step(wl.grid, wl.beams, wl.step)["F"]
    p0 = oracle.project(wl.grid, wl.beams, wl.step.P, F)
    p1 = oracle.project(wl.grid, _integrated(wl).beams, wl.step.P, F)
    inner = slice(12, 29)
    np.testing.assert_allclose(p1["w"][inner] / L, 1.0, atol=1e-3)
    assert np.abs(p0["w"][inner] / L - 1.0).max() > 1e-2
    idx = np.arange(g.n_cells)
    i, j, k = idx % g.nx, (idx // g.nx) % g.ny, idx // (g.nx * g.ny)
    r2 = ((i + 0.5) * g.h - x0) ** 2 + ((j + 0.5) * g.h - y0) ** 2
    interior = (k >= 20) & (k <= 35)
    expect = -np.outer(F[:, 20] / L, np.exp(-r2[interior] / eps ** 2) / (np.pi * eps ** 2))
    expect[:, r2[interior] > (3 * eps) ** 2] = 0.0
    scale = np.abs(expect).max()
    assert np.abs(p1["S"][:, interior] - expect).max() / scale < 2e-3


def test_integrated_projection_sends_each_node_share_to_its_end():
    """One segment, the load on its first node only: the load per length
    falls linearly from that node to the other, so the source's centroid
    along the axis lies a third of the way along the segment (the shares
    swapped would put it at two thirds)."""
    g = GridSpec(30, 30, 60, 0.01)
    P = np.array([[0.15, 0.15], [0.15, 0.15], [0.12, 0.42]])
    wl = _line_workload(P, _uniform(g, (0.5, 0, 0)), grid=g, cv=0.15, per_line=dict(eps=0.02))
    F = np.zeros((3, 2))
    F[0, 0] = 1.0
    S = oracle.project(wl.grid, _integrated(wl).beams, wl.step.P, F)["S"][0]
    z = (np.arange(g.n_cells) // (g.nx * g.ny) + 0.5) * g.h
    zc = (np.abs(S) * z).sum() / np.abs(S).sum()
    assert abs(zc - (0.12 + 0.30 / 3)) < 0.005, zc


# ----------------------------------------------------------------------------
# quasi-static reconstruction: point loads on a linear Euler-Bernoulli
# cantilever (the structural check of Sec. 7)
# ----------------------------------------------------------------------------

def _stem(n, L=1.0, axis=(0.0, 0.0, 1.0), root=(0.2, -0.1, 0.3), n_lines=1):
    ax = np.asarray(axis, float) / np.linalg.norm(axis)
    s = np.linspace(0.0, L, n)
    P0 = np.concatenate([np.asarray(root)[:, None] + s[None] * ax[:, None]] * n_lines, axis=1)
    b = BeamSpec(line_off=np.arange(n_lines + 1, dtype=np.int32) * n, d=np.ones(n_lines), cdn=np.ones(n_lines),
                 cdt=np.ones(n_lines), eps=np.ones(n_lines), ell_s=np.ones(n_lines), alpha_f=np.ones(n_lines),
                 cv_len=np.full(n * n_lines, L / (n - 1)))
    return b, P0, ax, s


def test_cantilever_tip_load_curve():
    """w(x) = P x^2 (3L - x) / (6 EI) under a tip load P."""
    b, P0, ax, s = _stem(41, L=0.8)
    F = np.zeros_like(P0)
    F[0, -1], F[1, -1] = 0.3, -0.2
    EI = 0.0259
    dP = oracle.beam_quasistatic(b, EI, ax, P0, F) - P0
    w = s ** 2 * (3 * 0.8 - s) / (6 * EI)
    np.testing.assert_allclose(dP[0], 0.3 * w, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(dP[1], -0.2 * w, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(dP[2], 0.0, atol=1e-15)


def test_cantilever_uniform_load_converges_to_closed_form():
    """Nodal point loads q L / (n - 1) (halved at the ends) tend to the
    distributed load q: tip deflection q L^4 / (8 EI)."""
    for n, tol in ((101, 2e-4), (401, 2e-5)):
        b, P0, ax, s = _stem(n, L=0.4)
        q, EI = 0.758, 0.02591
        F = np.zeros_like(P0)
        F[1] = q * 0.4 / (n - 1)
        F[1, 0] *= 0.5
        F[1, -1] *= 0.5
        tip = (oracle.beam_quasistatic(b, EI, ax, P0, F) - P0)[1, -1]
        assert abs(tip / (q * 0.4 ** 4 / (8 * EI)) - 1) < tol


def test_cantilever_axial_loads_reciprocity_and_rotation():
    rng = np.random.default_rng(31)
    b, P0, ax, s = _stem(17, L=0.5)
    EI = 0.7
    # loads along the axis bend nothing
    F = np.outer(ax, rng.normal(size=17))
    np.testing.assert_allclose(oracle.beam_quasistatic(b, EI, ax, P0, F), P0, atol=1e-15)
    # Maxwell-Betti: the deflection at i under a unit load at k equals that at k under a unit load at i
    for i, k in ((3, 11), (16, 5), (8, 8)):
        Fi, Fk = np.zeros_like(P0), np.zeros_like(P0)
        Fi[0, i], Fk[0, k] = 1.0, 1.0
        d_k = (oracle.beam_quasistatic(b, EI, ax, P0, Fi) - P0)[0, k]
        d_i = (oracle.beam_quasistatic(b, EI, ax, P0, Fk) - P0)[0, i]
        assert d_k == pytest.approx(d_i, rel=1e-13)
    # rotating stem and loads together rotates the deflection
    th = 0.7
    Rm = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    F = rng.normal(size=(3, 17))
    d0 = oracle.beam_quasistatic(b, EI, ax, P0, F) - P0
    b2, P2, ax2, _ = _stem(17, L=0.5, axis=Rm @ ax, root=Rm @ np.array([0.2, -0.1, 0.3]))
    d2 = oracle.beam_quasistatic(b2, EI, ax2, P2, Rm @ F) - P2
    np.testing.assert_allclose(d2, Rm @ d0, rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------------------
# reflected kernel at the grid faces (the one-sided kernel of Sec. 6, read as
# a mirror): pinned against the plain truncated kernel of the mirror lines
# ----------------------------------------------------------------------------

def _mirror(P, g, axis, high):
    """P mirrored across the low (high) face of `axis` of grid g."""
    Q = np.array(P, float, copy=True)
    face = g.origin[axis] + ((g.nx, g.ny, g.nz)[axis] * g.h if high else 0.0)
    Q[axis] = 2.0 * face - Q[axis]
    return Q


def _corner_line(g):
    # a bent line rooted on the z- face near the x- / y- edge, inside the grid
    n = 7
    t = np.linspace(0.0, 1.0, n)
    P = np.stack([g.origin[0] + g.h * (1.3 + 2.0 * t ** 2), g.origin[1] + g.h * (0.8 + 0.7 * t),
                  g.origin[2] + g.h * 7.0 * t])
    b = _beams([0, n], np.full(n, g.h), per_line=dict(eps=1.5 * g.h))
    F = np.stack([np.linspace(1.0, 2.0, n), np.linspace(-0.5, 0.5, n), np.full(n, 0.25)])
    return P, b, F


@pytest.mark.parametrize("faces", [(0, 1, 2), (2,), (0,)])
def test_reflected_weights_are_the_mirror_lines_weights(faces):
    """w_k with reflection = sum over the line's mirror images of their plain
    (truncated) w_k: each ghost cell sees the line as the grid cell it mirrors
    sees the mirrored line."""
    g = GridSpec(14, 12, 13, 0.01, origin=(0.1, -0.2, 0.05), precision="fp64")
    P, b, F = _corner_line(g)
    mask = sum(1 << (2 * a) for a in faces)
    wr = oracle.project(g, replace(b, wall_reflect=mask), P, F)["w"]
    total = np.zeros_like(wr)
    for bits in range(1 << len(faces)):
        Q = P
        for i, a in enumerate(faces):
            if bits >> i & 1:
                Q = _mirror(Q, g, a, False)
        total += oracle.project(g, b, Q, F)["w"]
    np.testing.assert_allclose(wr, total, rtol=1e-12)
    plain = oracle.project(g, b, P, F)["w"]
    assert (wr >= plain).all() and (wr > plain).any()
    if 2 in faces:
        assert wr[0] > 1.5 * plain[0]                             # the root sits on the z- face


def test_reflected_source_is_the_mirror_lines_sources():
    """S with reflection at the x+ and z- faces equals the plain sources of the
    line and its mirror images, each carrying F_k w_k(image) / w_k(reflected):
    the fold puts every ghost's share in the cell it mirrors."""
    g = GridSpec(12, 11, 13, 0.01, precision="fp64")
    P, b, F = _corner_line(g)
    P[0] = g.nx * g.h - (P[0] - g.origin[0])          # near the x+ face instead
    mask = (1 << 1) | (1 << 4)
    r = oracle.project(g, replace(b, wall_reflect=mask), P, F)
    images = [P, _mirror(P, g, 0, True), _mirror(P, g, 2, False), _mirror(_mirror(P, g, 0, True), g, 2, False)]
    S = np.zeros_like(r["S"])
    for Q in images:
        wq = oracle.project(g, b, Q, F)["w"]
        S += oracle.project(g, b, Q, F * (wq / r["w"]))["S"]
    np.testing.assert_allclose(r["S"], S, rtol=1e-11, atol=1e-12 * np.abs(S).max())


def test_reflection_conserves_and_leaves_far_lines_alone():
    for seed in range(4):
        wl = W.make_random(400 + seed, 18, 16, 14, n_lines=4, precision="fp64",
                           kinds=("stem", "arc", "random", "point"))
        plain = oracle.sample_drag_spread(wl)
        r = oracle.sample_drag_spread(W.with_reflect(wl, 63))
        assert r["status"][oracle.ST_DEPOSIT_LOST] == 0
        np.testing.assert_allclose(r["totals"][3:], -r["totals"][:3], atol=1e-12 * np.abs(r["F"]).sum())
        np.testing.assert_array_equal(r["F"], plain["F"])
        # brute force over every cell and ghost cell gives the same bits
        b = oracle.project(wl.grid, W.with_reflect(wl, 63).beams, wl.step.P, r["F"], cull=False)
        np.testing.assert_array_equal(b["S"], r["S"])
    # a line farther than 3 eps from every face: reflection changes nothing
    g = GridSpec(30, 30, 30, 0.01, precision="fp64")
    bl, P, F = _straight_z_line(g, 0.155, 0.145, 0.09, 0.02, 6, np.ones((3, 6)))
    a = oracle.project(g, bl, P, F)
    c = oracle.project(g, replace(bl, wall_reflect=63), P, F)
    np.testing.assert_array_equal(a["S"], c["S"])
    np.testing.assert_array_equal(a["w"], c["w"])
