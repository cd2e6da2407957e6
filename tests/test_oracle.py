"""Pins for the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each compares the oracle with
an independent statement (a dense library solve, a closed form, a textbook
table, an invariant, brute force or an analytic function), chosen so that a
dropped term, a wrong sign or index, or a transposed axis fails at least one.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2005_13193_gb300 import synth

TWO_PI = 2 * math.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_periodic(n):
    """The periodic (1/6, 4/6, 1/6) matrix of Sec. 2.2 written out densely."""
    A = np.zeros((n, n))
    for j in range(n):
        A[j, j] += 4 / 6
        A[j, (j - 1) % n] += 1 / 6
        A[j, (j + 1) % n] += 1 / 6
    return A


# ---------------------------------------------------------------- solve ----

@pytest.mark.parametrize("n", list(range(3, 17)) + [32, 33])
def test_cyclic_solve_matches_dense_lu(n):
    rng = np.random.default_rng(n)
    g = rng.standard_normal(n)
    c = oracle.cyclic_solve(g)
    ref = np.linalg.solve(dense_periodic(n), g)
    np.testing.assert_allclose(c, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [3, 4, 5, 8, 12, 31, 64])
def test_impulse_response_closed_form(n):
    # Periodic Green's function of (z^-1 + 4 + z)/6: the infinite-line inverse
    # is sqrt(3) r^|d| with r = sqrt(3)-2 (roots of z^2+4z+1); summing its
    # periodic images gives sqrt(3)(r^d + r^(n-d))/(1 - r^n), 0 <= d < n.
    r = math.sqrt(3) - 2
    e0 = np.zeros(n)
    e0[0] = 1.0
    c = oracle.cyclic_solve(e0)
    closed = np.array([math.sqrt(3) * (r ** d + r ** (n - d)) / (1 - r ** n)
                       for d in range(n)])
    np.testing.assert_allclose(c, closed, rtol=0, atol=1e-14)
    # row sums of A are 1, so the inverse preserves constants
    assert abs(c.sum() - 1.0) < 1e-14
    # the windowed oracle's kernel is the same closed form
    for d in range(-n, 2 * n):
        assert abs(oracle.green(n, d) - closed[d % n]) < 1e-14


@pytest.mark.parametrize("n,m", [(8, 1), (16, 3), (17, 5), (32, 16), (12, 6)])
def test_single_fourier_mode_1d(n, m):
    # A acts on e^{i k x_j} as multiplication by (4 + 2 cos(kh))/6.
    j = np.arange(n)
    for phase in (0.0, 0.7):
        g = np.cos(2 * np.pi * m * j / n + phase)
        lam = (4 + 2 * np.cos(2 * np.pi * m / n)) / 6
        np.testing.assert_allclose(oracle.cyclic_solve(g), g / lam, rtol=0, atol=1e-13)


def test_spline_coeffs_3d_fourier_mode_and_padding():
    nx, ny, nz = 10, 12, 14
    mx, my, mz = 2, 3, 5
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    g = np.cos(2 * np.pi * (mx * x / nx + my * y / ny + mz * z / nz) + 0.3)
    field = np.stack([g, 2 * g, -g])
    coef = oracle.spline_coeffs(field)
    lam = [(4 + 2 * np.cos(2 * np.pi * m / n)) / 6 for m, n in ((mx, nx), (my, ny), (mz, nz))]
    interior = field / (lam[0] * lam[1] * lam[2])
    assert coef.shape == (3, nz + 3, ny + 3, nx + 3)
    # padded P holds node (P-1) mod N on every axis (one ghost below, two above)
    iz = (np.arange(nz + 3) - 1) % nz
    iy = (np.arange(ny + 3) - 1) % ny
    ix = (np.arange(nx + 3) - 1) % nx
    expect = interior[:, iz][:, :, iy][:, :, :, ix]
    np.testing.assert_allclose(coef, expect, rtol=0, atol=1e-13)


def test_spline_coeffs_dense_kronecker():
    # Whole 3D system (A_z kron A_y kron A_x) solved densely on an anisotropic grid,
    # so a swapped axis or a missed direction fails.
    nx, ny, nz = 3, 4, 5
    field = synth.random_field((nx, ny, nz), ncomp=2, seed=7)
    K = np.kron(dense_periodic(nz), np.kron(dense_periodic(ny), dense_periodic(nx)))
    coef = oracle.spline_coeffs(field)
    for c in range(2):
        ref = np.linalg.solve(K, field[c].reshape(-1)).reshape(nz, ny, nx)
        np.testing.assert_allclose(coef[c, 1:nz + 1, 1:ny + 1, 1:nx + 1], ref,
                                   rtol=0, atol=1e-13)


# ---------------------------------------------------------------- basis ----

def _golden_basis():
    rows = []
    with open(os.path.join(GOLDEN, "bspline_basis.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(Fraction(v)) for v in line.split()])
    return rows


def test_basis_textbook_values():
    rows = _golden_basis()
    assert len(rows) == 3
    for row in rows:
        b, db = oracle.basis(row[0])
        np.testing.assert_allclose(b, row[1:5], rtol=0, atol=1e-15)
        np.testing.assert_allclose(db, row[5:9], rtol=0, atol=1e-15)


@pytest.mark.parametrize("t", [0.0, 0.1, 0.25, 0.5, 0.77, 0.999])
def test_basis_moments(t):
    # nodes a-1, a, a+1, a+2 sit at offsets -1, 0, 1, 2 from cell a: the cubic
    # B-spline reproduces 1 and linear functions, and its second moment about
    # the point is the variance 1/3 of the cardinal cubic B-spline.
    b, db = oracle.basis(t)
    off = np.array([-1.0, 0.0, 1.0, 2.0])
    assert abs(b.sum() - 1) < 1e-15
    assert abs((b * off).sum() - t) < 1e-15
    assert abs((b * (off - t) ** 2).sum() - 1 / 3) < 1e-15
    assert abs(db.sum()) < 1e-15
    assert abs((db * off).sum() - 1) < 1e-15
    assert (b >= 0).all()


def test_locate_periodic_shadow():
    # L = 8, n = 16: inv_h = 2 and all values below are exact binary numbers, so
    # the shadow image x + m L must give bit-identical (cell, t).
    for x in (0.0, 0.25, 3.3125, 7.9375, 5.5):
        c0, t0 = oracle.locate(x, 8.0, 16)
        for m in (-3, -1, 1, 2, 1000):
            c, t = oracle.locate(x + 8.0 * m, 8.0, 16)
            assert (c, t) == (c0, t0)
    assert oracle.locate(-0.25, 8.0, 16) == (15, 0.5)
    assert oracle.locate(3.75, 8.0, 16) == (7, 0.5)


# --------------------------------------------------------------- interp ----

def test_node_reproduction():
    n = (12, 10, 9)
    field = synth.random_field(n, ncomp=3, seed=3)
    coef = oracle.spline_coeffs(field)
    L = (TWO_PI, 5.0, 3.0)
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    pos = np.stack([x.ravel() * L[0] / n[0], y.ravel() * L[1] / n[1], z.ravel() * L[2] / n[2]])
    vel = oracle.interp(coef, pos, L=L)
    np.testing.assert_allclose(vel, field.reshape(3, -1), rtol=0, atol=1e-12)


def test_constants_are_exact():
    n = 8
    field = np.stack([np.full((n, n, n), v) for v in (1.5, -2.0, 0.25)])
    coef = oracle.spline_coeffs(field)
    np.testing.assert_allclose(coef[0], 1.5, rtol=0, atol=1e-14)
    pos = synth.uniform_particles(500, seed=1) * 3 - 5  # includes shadow images
    vel, grad = oracle.interp(coef, pos, grad=True)
    np.testing.assert_allclose(vel, [[1.5], [-2.0], [0.25]] * np.ones((1, 500)), atol=1e-13)
    np.testing.assert_allclose(grad, 0.0, atol=1e-12)


def _analytic(pos):
    x, y, z = pos
    u = np.sin(x) * np.cos(2 * y) * np.sin(z + 0.4)
    du = np.stack([np.cos(x) * np.cos(2 * y) * np.sin(z + 0.4),
                   -2 * np.sin(x) * np.sin(2 * y) * np.sin(z + 0.4),
                   np.sin(x) * np.cos(2 * y) * np.cos(z + 0.4)])
    return u, du


def _analytic_field(n):
    h = TWO_PI / n
    z, y, x = np.meshgrid(np.arange(n) * h, np.arange(n) * h, np.arange(n) * h, indexing="ij")
    u, _ = _analytic(np.stack([x, y, z]))
    return u[None]


def test_fourth_order_convergence():
    # Sec. 2.2: cubic splines are fourth-order accurate (values) and the
    # derivative converges at third order.
    pos = synth.uniform_particles(400, seed=11)
    exact, dexact = _analytic(pos)
    errs, gerrs = [], []
    for n in (16, 32, 64):
        coef = oracle.spline_coeffs(_analytic_field(n))
        vel, grad = oracle.interp(coef, pos, grad=True)
        errs.append(np.abs(vel[0] - exact).max())
        gerrs.append(np.abs(grad[0] - dexact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12 < r1 < 20 and 13 < r2 < 19, errs
    g1, g2 = gerrs[0] / gerrs[1], gerrs[1] / gerrs[2]
    assert 6 < g1 < 11 and 6.5 < g2 < 10, gerrs


def test_c2_continuity_across_faces():
    n = 8
    coef = oracle.spline_coeffs(synth.random_field(n, ncomp=1, seed=5))
    h = TWO_PI / n
    rng = np.random.default_rng(0)
    for axis in range(3):
        base = rng.uniform(0, TWO_PI, size=(3, 50))
        face = (np.floor(base[axis] / h) + 1) * h
        d = 1e-7 * h
        lo, hi = base.copy(), base.copy()
        lo[axis] = face - d
        hi[axis] = face + d
        vlo, glo = oracle.interp(coef, lo, grad=True)
        vhi, ghi = oracle.interp(coef, hi, grad=True)
        scale = np.abs(coef).max()
        assert np.abs(vlo - vhi).max() < 1e-5 * scale
        assert np.abs(glo - ghi).max() < 1e-4 * scale / h
        # second derivative along the axis: one-sided differences of the gradient
        e = 1e-4 * h
        lo2, hi2 = lo.copy(), hi.copy()
        lo2[axis] -= e
        hi2[axis] += e
        _, glo2 = oracle.interp(coef, lo2, grad=True)
        _, ghi2 = oracle.interp(coef, hi2, grad=True)
        s_lo = (glo[0, axis] - glo2[0, axis]) / e
        s_hi = (ghi2[0, axis] - ghi[0, axis]) / e
        assert np.abs(s_lo - s_hi).max() < 1e-2 * scale / h ** 2


def test_gradient_matches_central_differences():
    n = (10, 12, 9)
    coef = oracle.spline_coeffs(synth.random_field(n, ncomp=3, seed=8))
    pos = synth.uniform_particles(1024, seed=9)
    _, grad = oracle.interp(coef, pos, grad=True)
    hfd = 1e-6
    for d in range(3):
        p1, p0 = pos.copy(), pos.copy()
        p1[d] += hfd
        p0[d] -= hfd
        fd = (oracle.interp(coef, p1) - oracle.interp(coef, p0)) / (2 * hfd)
        np.testing.assert_allclose(grad[:, d], fd, rtol=0, atol=2e-7 * np.abs(grad).max())


# ------------------------------------------------------------- backward ----

def test_backward_field_is_the_transpose():
    # u = J v is linear in the field v: <w, J v> = <J^T w, v> exactly up to rounding.
    n = (9, 8, 11)
    v = synth.random_field(n, ncomp=3, seed=21)
    pos = synth.uniform_particles(300, seed=22) * 1.5 - 2.0
    w = np.random.default_rng(23).standard_normal((3, 300))
    coef = oracle.spline_coeffs(v)
    Jv = oracle.interp(coef, pos)
    _, JTw = oracle.interp_backward(coef, pos, w, want_pos=False)
    lhs = float((w * Jv).sum())
    rhs = float((JTw * v).sum())
    assert abs(lhs - rhs) < 1e-11 * (abs(lhs) + 1)
    # also against an explicit column of J^T: perturb one node
    e = np.zeros_like(v)
    e[1, 3, 4, 5] = 1.0
    col = oracle.interp(oracle.spline_coeffs(e), pos)
    assert abs(float((w * col).sum()) - JTw[1, 3, 4, 5]) < 1e-13


def test_backward_positions_match_fd():
    n = 10
    coef = oracle.spline_coeffs(synth.random_field(n, ncomp=3, seed=31))
    pos = synth.uniform_particles(256, seed=32)
    w = np.random.default_rng(33).standard_normal((3, 256))
    g_pos, _ = oracle.interp_backward(coef, pos, w, want_field=False)
    hfd = 1e-6
    for d in range(3):
        p1, p0 = pos.copy(), pos.copy()
        p1[d] += hfd
        p0[d] -= hfd
        fd = ((w * oracle.interp(coef, p1)).sum(0) - (w * oracle.interp(coef, p0)).sum(0)) / (2 * hfd)
        np.testing.assert_allclose(g_pos[d], fd, rtol=0, atol=1e-6)


# ---------------------------------------------------------------- binning ----

def test_binning_brute_force():
    n, brick = (20, 16, 12), (8, 4, 5)
    L = (TWO_PI, 3.0, 7.5)
    pos = synth.uniform_particles(2000, seed=41)
    pos = pos / TWO_PI * np.array(L)[:, None] * 3 - np.array(L)[:, None]  # shadows too
    bin_of, offs, perm = oracle.bin_particles(n, brick, pos, L=L)
    nb = [-(-n[d] // brick[d]) for d in range(3)]
    keys = []
    for p in range(pos.shape[1]):
        b = []
        for d in range(3):
            s = pos[d, p] * (n[d] / L[d])
            cell = int(math.floor(s)) % n[d]
            b.append(cell // brick[d])
        keys.append((b[2] * nb[1] + b[1]) * nb[0] + b[0])
    keys = np.array(keys)
    np.testing.assert_array_equal(bin_of, keys)
    counts = np.bincount(keys, minlength=nb[0] * nb[1] * nb[2])
    np.testing.assert_array_equal(offs, np.concatenate([[0], np.cumsum(counts)]))
    np.testing.assert_array_equal(perm, np.argsort(keys, kind="stable"))


# -------------------------------------------------------------------- RK2 ----

def test_rk2_constant_field_is_exact():
    n = 8
    field = np.stack([np.full((n, n, n), v) for v in (0.5, -1.25, 2.0)])
    coef = oracle.spline_coeffs(field)
    pos = synth.uniform_particles(100, seed=51)
    new, u1 = oracle.rk2_step(coef, pos, 1e-3)
    vel = np.array([[0.5], [-1.25], [2.0]])
    # coefficients of a constant are the constant to ~1 ulp; the step is x + dt*u
    np.testing.assert_allclose(new, pos + 1e-3 * vel, rtol=0, atol=1e-15)
    np.testing.assert_allclose(u1, vel * np.ones((1, 100)), rtol=0, atol=1e-14)


def test_rk2_heun_against_analytic_field():
    # u = (sin z, sin x, sin y): Heun with the exact field vs the oracle's
    # spline field; the difference is dt * (spline error O(h^4)).
    n, dt = 48, 1e-2
    h = TWO_PI / n
    z, y, x = np.meshgrid(np.arange(n) * h, np.arange(n) * h, np.arange(n) * h, indexing="ij")
    field = np.stack([np.sin(z), np.sin(x), np.sin(y)])
    coef = oracle.spline_coeffs(field)
    pos = synth.uniform_particles(200, seed=52)

    def f(p):
        return np.stack([np.sin(p[2]), np.sin(p[0]), np.sin(p[1])])

    u1 = f(pos)
    xs = pos + dt * u1
    exact = pos + dt / 2 * (u1 + f(xs))
    new, _ = oracle.rk2_step(coef, pos, dt)
    err = np.abs(new - exact).max()
    assert err < dt * 5e-6, err
    # a forward-Euler step would be off by O(dt^2) ~ 1e-4 * 1/2
    assert np.abs(pos + dt * u1 - exact).max() > 100 * err


def test_rk2_time_dependent_field_uses_both():
    n = 8
    c0 = oracle.spline_coeffs(np.stack([np.full((n, n, n), 1.0)] * 3))
    c1 = oracle.spline_coeffs(np.stack([np.full((n, n, n), 3.0)] * 3))
    pos = synth.uniform_particles(10, seed=53)
    new, _ = oracle.rk2_step(c0, pos, 0.1, coef_np1=c1)
    np.testing.assert_allclose(new, pos + 0.1 * 2.0, atol=1e-14)


# -------------------------------------------------------------- windowed ----

@pytest.mark.parametrize("n", [64, 128])
def test_windowed_matches_full_oracle(n):
    # the windowed evaluation (the periodic inverse cut to |d| <= 24 per axis,
    # a 52^3 window per particle) against the full solve, at two grid sizes,
    # with particles on and next to the periodic boundary besides random ones
    field = synth.random_field(n, ncomp=3, seed=61 + n).astype(np.float32)
    edge = np.array([[0.0, 2 * np.pi - 1e-12, np.pi, 1e-12],
                     [2 * np.pi - 1e-9, 0.0, 1e-9, np.pi],
                     [np.pi, 1e-12, 2 * np.pi - 1e-12, 0.0]])
    pos = np.concatenate([synth.uniform_particles(40, seed=62 + n), edge], axis=1)
    full = oracle.interp(oracle.spline_coeffs(field.astype(np.float64)), pos)
    win = oracle.interp_windowed(field, pos)
    np.testing.assert_allclose(win, full, rtol=0, atol=1e-12 * np.abs(full).max())


def test_nonfinite_position_is_reported():
    coef = oracle.spline_coeffs(synth.random_field(6, ncomp=3, seed=1))
    pos = synth.uniform_particles(4, seed=2)
    pos[1, 2] = np.nan
    vel = oracle.interp(coef, pos, allow_nonfinite=True)
    assert np.isnan(vel[:, 2]).all() and np.isfinite(vel[:, [0, 1, 3]]).all()
    with pytest.raises(oracle.OracleError):
        oracle.interp(coef, pos)


# ----------------------------------------------------- second derivatives ----

def test_hessian_matches_central_differences_of_the_gradient():
    # d2u/dxa dxb from central differences (h = 1e-5) of the oracle's gradient,
    # which is computed by a different sum (b' instead of b'')
    n = (10, 12, 9)
    coef = oracle.spline_coeffs(synth.random_field(n, ncomp=3, seed=18))
    pos = synth.uniform_particles(512, seed=19)
    hess = oracle.interp_hessian(coef, pos)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    hfd = 1e-5
    for e, (a, b) in enumerate(pairs):
        p1, p0 = pos.copy(), pos.copy()
        p1[b] += hfd
        p0[b] -= hfd
        _, g1 = oracle.interp(coef, p1, grad=True)
        _, g0 = oracle.interp(coef, p0, grad=True)
        fd = (g1[:, a] - g0[:, a]) / (2 * hfd)
        np.testing.assert_allclose(hess[:, e], fd, rtol=0, atol=1e-7 * np.abs(hess).max())


def test_hessian_mixed_partials_commute():
    # d/dy (du/dx) and d/dx (du/dy) from differences agree with the one stored
    n = 12
    coef = oracle.spline_coeffs(synth.random_field(n, ncomp=1, seed=20))
    pos = synth.uniform_particles(256, seed=21)
    hess = oracle.interp_hessian(coef, pos)
    hfd = 1e-5
    for e, (a, b) in ((3, (0, 1)), (4, (0, 2)), (5, (1, 2))):
        outs = []
        for da, db in ((a, b), (b, a)):
            p1, p0 = pos.copy(), pos.copy()
            p1[db] += hfd
            p0[db] -= hfd
            _, g1 = oracle.interp(coef, p1, grad=True)
            _, g0 = oracle.interp(coef, p0, grad=True)
            outs.append((g1[0, da] - g0[0, da]) / (2 * hfd))
        np.testing.assert_allclose(outs[0], outs[1], rtol=0, atol=1e-7 * np.abs(hess).max())
        np.testing.assert_allclose(hess[0, e], outs[0], rtol=0, atol=1e-7 * np.abs(hess).max())


def test_hessian_is_linear_inside_a_cell():
    # the cubic B-spline's second derivative is piecewise linear: along x
    # inside one cell d2u/dx2 at the midpoint is the mean of the two ends
    n = 8
    coef = oracle.spline_coeffs(synth.random_field(n, ncomp=1, seed=22))
    h = TWO_PI / n
    rng = np.random.default_rng(3)
    base = rng.uniform(0, TWO_PI, size=(3, 100))
    cell = np.floor(base[0] / h)
    lo, mid, hi = base.copy(), base.copy(), base.copy()
    lo[0] = (cell + 0.1) * h
    mid[0] = (cell + 0.5) * h
    hi[0] = (cell + 0.9) * h
    hl, hm, hh = (oracle.interp_hessian(coef, p)[0, 0] for p in (lo, mid, hi))
    np.testing.assert_allclose(hm, 0.5 * (hl + hh), rtol=0, atol=1e-10 * np.abs(hm).max())


def test_hessian_convergence():
    # second derivatives of the interpolant of a smooth field converge at
    # least at second order in h (d2/dx2 shows third order, the mixed one
    # second, at random points); a wrong basis or scale does not converge
    pos = synth.uniform_particles(400, seed=23)
    x, y, z = pos
    exact = -np.sin(x) * np.cos(2 * y) * np.sin(z + 0.4)          # d2u/dx2
    exact_xy = -2 * np.cos(x) * np.sin(2 * y) * np.sin(z + 0.4)   # d2u/dxdy
    errs, errs_xy = [], []
    for n in (16, 32, 64):
        hess = oracle.interp_hessian(oracle.spline_coeffs(_analytic_field(n)), pos)
        errs.append(np.abs(hess[0, 0] - exact).max())
        errs_xy.append(np.abs(hess[0, 3] - exact_xy).max())
    for e in (errs, errs_xy):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert r1 > 3.0 and r2 > 3.0, e  # first order would give 2
        assert e[2] < 1e-3, e


def test_lagrangian_accel_closed_forms():
    n = 16
    pos = synth.uniform_particles(300, seed=24)
    # a spatially constant field changing in time: a = (u1 - u0) / dt exactly
    f0 = np.ones((3, n, n, n)) * np.array([1.0, -2.0, 0.5])[:, None, None, None]
    f1 = f0 * 1.5
    acc = oracle.lagrangian_accel(oracle.spline_coeffs(f0), pos, oracle.spline_coeffs(f1), 0.25)
    np.testing.assert_allclose(acc, (0.5 / 0.25) * f0[:, 0, 0, 0][:, None] * np.ones_like(acc),
                               rtol=0, atol=1e-12)
    # a steady shear flow u = (sin y, 0, 0) has no convective acceleration
    h = TWO_PI / n
    z, y, x = np.meshgrid(np.arange(n) * h, np.arange(n) * h, np.arange(n) * h, indexing="ij")
    f = np.stack([np.sin(y), np.zeros_like(y), np.zeros_like(y)])
    acc = oracle.lagrangian_accel(oracle.spline_coeffs(f), pos)
    assert np.abs(acc).max() < 1e-12
    # u = (sin y, sin z, 0): (u . grad) u = (sin z cos y, 0, 0), third order in h
    errs = []
    for n in (16, 32, 64):
        h = TWO_PI / n
        z, y, x = np.meshgrid(np.arange(n) * h, np.arange(n) * h, np.arange(n) * h,
                              indexing="ij")
        f = np.stack([np.sin(y), np.sin(z), np.zeros_like(y)])
        acc = oracle.lagrangian_accel(oracle.spline_coeffs(f), pos)
        ex = np.sin(pos[2]) * np.cos(pos[1])
        errs.append(max(np.abs(acc[0] - ex).max(), np.abs(acc[1:]).max()))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6 < r1 < 11 and 6.5 < r2 < 10, errs


def test_truncated_inverse_full_circulant_is_the_solve():
    # with 2K + 1 = N on every axis the cut convolution keeps every entry of
    # the periodic inverse: it must equal the Thomas + Sherman-Morrison solve
    rng = np.random.default_rng(41)
    f = rng.standard_normal((2, 9, 9, 9))
    np.testing.assert_allclose(oracle.spline_coeffs_truncated(f, 4), oracle.spline_coeffs(f),
                               rtol=0, atol=1e-13)
    f = rng.standard_normal((1, 7, 7, 7))
    np.testing.assert_allclose(oracle.spline_coeffs_truncated(f, 3), oracle.spline_coeffs(f),
                               rtol=0, atol=1e-13)


def test_truncated_inverse_error_bound_and_rate():
    # the entries beyond |d| = K sum to at most 2 sqrt3 |r|^(K+1) / (1 - |r|)
    # per axis; through three axes with sum |G| = 3 each the error is below
    # 27 times that of max|g|, and it shrinks by r^2 per two more taps
    rng = np.random.default_rng(42)
    f = rng.standard_normal((1, 48, 40, 36))
    exact = oracle.spline_coeffs(f)
    r = abs(math.sqrt(3.0) - 2.0)
    errs = []
    for K in (4, 6, 8, 10, 12, 15):
        e = np.abs(oracle.spline_coeffs_truncated(f, K) - exact).max()
        tail = 2 * math.sqrt(3.0) * r ** (K + 1) / (1 - r)
        assert e <= 27 * tail * np.abs(f).max(), (K, e)
        errs.append(e)
    for a, b in zip(errs[:4], errs[1:5]):
        assert 0.03 < b / a < 0.15, errs  # r^2 = 0.072


def test_truncated_inverse_constant_field_closed_form():
    # a constant maps to the constant times the cube of the kept entries' sum,
    # a geometric series: sqrt3 (1 + 2 r (1 - r^K) / (1 - r)) (N large, r^N ~ 0)
    r = math.sqrt(3.0) - 2.0
    c = np.full((1, 64, 64, 64), 1.7)
    for K in (1, 3, 7, 15):
        S = math.sqrt(3.0) * (1 + 2 * r * (1 - r ** K) / (1 - r))
        np.testing.assert_allclose(oracle.spline_coeffs_truncated(c, K), 1.7 * S ** 3,
                                   rtol=0, atol=1e-13)
