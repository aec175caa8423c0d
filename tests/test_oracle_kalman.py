"""Pins of the oracle's Kalman building blocks against mathematics that does
not go through the oracle's own formulas:

* transport: closed-form circle/helix geometry (tests/helpers.Helix),
* transport Jacobian: finite differences of the transported parameters,
* update: the information-form posterior and the chi2 identity,
* rotation: rigid rotation of a helix point and direction,
* chained fit at Bz = 0: batch maximum-a-posteriori least squares (scipy).
"""
import math

import numpy as np
import pytest

import oracle
from helpers import Helix, row_x

CINIT = np.array([0.01, 0, 0.0225, 0, 0, 0.04, 0, 0, 0, 0.25, 0, 0, 0, 0, 400.0])


def ix(i, j):
    return i * (i + 1) // 2 + j if i >= j else j * (j + 1) // 2 + i


def full(c15):
    return np.array([[c15[ix(i, j)] for j in range(5)] for i in range(5)])


def pack(M):
    return np.array([M[i, j] for i in range(5) for j in range(i + 1)])


def local_state(hx, alpha, x, side=1, zref=0.0):
    y, s, arc, z = hx.at_local_x(alpha, x)
    zeta = -side * (z - zref)  # drift coordinate up to a constant: dzeta/ds = -side tan(lambda)
    return np.array([y, zeta, s, -side * hx.tanl, hx.q / hx.pt]), arc


def random_helices(rng, n, bz):
    out = []
    while len(out) < n:
        pt = rng.uniform(0.12, 5.0)
        hx = Helix(pt, rng.uniform(-0.9, 0.9), math.radians(10 + rng.uniform(-8, 8)), int(rng.choice([-1, 1])),
                   bz=bz)
        a = math.radians(10)
        r1, r2 = sorted(rng.choice(152, 2, replace=False))
        if rng.uniform() < 0.5:
            r1, r2 = r2, r1
        x1, x2 = row_x(r1), row_x(r2)
        if hx.at_local_x(a, x1) is None or hx.at_local_x(a, x2) is None:
            continue
        out.append((hx, a, x1, x2))
    return out


@pytest.mark.parametrize("bz", [0.5, -0.5])
def test_propagation_matches_closed_form_helix(bz):
    """Transport of (y, zeta, sin phi) between pad rows equals the circle
    geometry to 1e-9 cm, both outward and inward, both field signs."""
    rng = np.random.default_rng(1)
    worst = 0.0
    for hx, a, x1, x2 in random_helices(rng, 400, bz):
        p1, s1 = local_state(hx, a, x1)
        p2, s2 = local_state(hx, a, x2)
        rc, xo, po, _ = oracle.propagate(x1, p1, CINIT, x2, bz)
        if abs(p2[2]) >= 0.999 or abs(p1[2]) >= 0.999:
            continue
        assert rc == 0
        assert xo == x2
        d = np.abs(po - p2)
        worst = max(worst, d[0], d[1])
        assert d[0] < 1e-9 and d[1] < 1e-9 and d[2] < 1e-12, (d, hx.pt)
        assert po[3] == p1[3] and po[4] == p1[4]
    assert worst < 1e-9


def test_straight_line_transport_at_zero_field():
    p = np.array([1.0, 2.0, 0.3, -0.7, 1.5])
    rc, x, po, _ = oracle.propagate(100.0, p, CINIT, 150.0, 0.0)
    assert rc == 0
    tphi = 0.3 / math.sqrt(1 - 0.09)
    assert abs(po[0] - (1.0 + 50 * tphi)) < 1e-12
    assert abs(po[1] - (2.0 - 0.7 * 50 * math.sqrt(1 + tphi**2))) < 1e-12
    assert po[2] == 0.3


def fd_jacobian(f, p, h=1e-6):
    J = np.zeros((5, 5))
    for j in range(5):
        e = np.zeros(5)
        e[j] = h * max(1.0, abs(p[j]))
        J[:, j] = (f(p + e) - f(p - e)) / (2 * e[j])
    return J


def test_transport_jacobian_matches_finite_differences():
    """C -> J C J^T with J checked column by column: with C = e_j e_j^T the
    transported covariance's column j is J[:, j] (J_jj = 1).  Every entry is
    exact except d zeta / d(q/pT), a three-point quadrature."""
    rng = np.random.default_rng(2)
    for hx, a, x1, x2 in random_helices(rng, 150, 0.5):
        p1, _ = local_state(hx, a, x1)
        if abs(p1[2]) > 0.9:
            continue

        def f(p):
            rc, _, po, _ = oracle.propagate(x1, p, CINIT, x2, 0.5)
            assert rc == 0
            return po

        try:
            Jfd = fd_jacobian(f, p1)
        except AssertionError:
            continue
        for j in range(5):
            E = np.zeros((5, 5))
            E[j, j] = 1.0
            rc, _, _, c = oracle.propagate(x1, p1, pack(E), x2, 0.5)
            col = full(c)[:, j]
            for i in range(5):
                tol = 1e-6 * (1 + abs(Jfd[i, j]))
                if (i, j) == (1, 4):
                    tol = 2e-4 * abs(Jfd[i, j]) + 1e-6
                assert abs(col[i] - Jfd[i, j]) <= tol, (i, j, col[i], Jfd[i, j])


def test_update_equals_information_form():
    rng = np.random.default_rng(3)
    V = np.diag([0.01, 0.0225])
    H = np.zeros((2, 5))
    H[0, 0] = H[1, 1] = 1
    for _ in range(200):
        A = rng.normal(size=(5, 5))
        C = A @ A.T * rng.uniform(0.001, 1.0) + np.eye(5) * 1e-3
        p = rng.normal(size=5)
        m = p[:2] + rng.normal(size=2) * 0.3
        rc, po, co, chi2 = oracle.update(p, pack(C), m[0], m[1])
        assert rc == 0
        Ci = np.linalg.inv(C)
        P = np.linalg.inv(Ci + H.T @ np.linalg.inv(V) @ H)
        pp = P @ (Ci @ p + H.T @ np.linalg.inv(V) @ m)
        np.testing.assert_allclose(po, pp, rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose(full(co), P, rtol=1e-7, atol=1e-10)
        # chi2 identity of the Kalman update
        r_post = m - pp[:2]
        chi_id = (pp - p) @ Ci @ (pp - p) + r_post @ np.linalg.inv(V) @ r_post
        assert abs(chi2 - chi_id) < 1e-7 * (1 + chi_id)


def test_rotation_matches_rigid_frame_change():
    """Rotating the frame by +-20 deg then transporting to a pad row equals
    the helix seen directly in the new frame; the covariance follows the
    finite-difference Jacobian of rotate-then-transport."""
    rng = np.random.default_rng(4)
    n = 0
    for _ in range(400):
        hx = Helix(rng.uniform(0.15, 3.0), rng.uniform(-0.8, 0.8), math.radians(20 + rng.uniform(-3, 3)),
                   int(rng.choice([-1, 1])))
        a1, a2 = math.radians(10), math.radians(30)
        r = int(rng.integers(20, 140))
        x1, x2 = row_x(r), row_x(r + 2)
        if hx.at_local_x(a1, x1) is None or hx.at_local_x(a2, x2) is None:
            continue
        zr = hx.at_local_x(a1, x1)[3]
        p1, _ = local_state(hx, a1, x1, zref=zr)
        p2, _ = local_state(hx, a2, x2, zref=zr)
        if max(abs(p1[2]), abs(p2[2])) > 0.9:
            continue
        rc, xr, pr, cr = oracle.rotate(x1, p1, CINIT, a2 - a1)
        assert rc == 0
        assert abs(xr - (x1 * math.cos(a2 - a1) + p1[0] * math.sin(a2 - a1))) < 1e-12
        rc, xo, po, co = oracle.propagate(xr, pr, cr, x2, 0.5)
        assert rc == 0
        assert abs(po[0] - p2[0]) < 1e-9 and abs(po[1] - p2[1]) < 1e-9 and abs(po[2] - p2[2]) < 1e-11

        def f(p):
            rc, xx, pp, _ = oracle.rotate(x1, p, CINIT, a2 - a1)
            rc2, _, pq, _ = oracle.propagate(xx, pp, CINIT, x2, 0.5)
            return pq

        J = fd_jacobian(f, p1, 1e-5)
        C0 = full(CINIT)
        np.testing.assert_allclose(full(co), J @ C0 @ J.T, rtol=2e-3, atol=1e-7)
        n += 1
    assert n > 50


def _line(rng, x):
    s_true, t_true = rng.uniform(-0.4, 0.4), rng.uniform(-1, 1)
    c_true = math.sqrt(1 - s_true**2)
    y = 2.0 + (x - x[0]) * s_true / c_true + rng.normal(0, 0.1, len(x))
    z = 5.0 + t_true * (x - x[0]) / c_true + rng.normal(0, 0.15, len(x))
    return s_true, t_true, y, z


def test_zero_field_fit_with_known_direction_equals_linear_least_squares():
    """At Bz = 0 with sin(phi) known (prior variance ~0) the measurement model
    is linear in (y0, zeta0, t): the chained filter must then equal the
    closed-form weighted linear least squares with the same Gaussian prior
    (normal equations solved by numpy)."""
    rng = np.random.default_rng(5)
    x = np.array([row_x(r) for r in range(0, 152, 3)])
    for _ in range(20):
        s_true, t_true, y, z = _line(rng, x)
        c = math.sqrt(1 - s_true**2)
        t_seed = t_true + rng.normal(0, 0.05)
        C0 = np.diag([0.01, 0.0225, 1e-300, 0.25, 400.0])
        rc, p, cov = oracle.fit_points(x, y, z, 0.0, [0, 0, s_true, t_seed, 0.0], pack(C0))
        assert rc == 0
        # unknowns theta = (y0, zeta0, t) at x[0]; rows: measurements + priors
        n = len(x)
        A = np.zeros((2 * n + 1, 3))
        b = np.zeros(2 * n + 1)
        w = np.zeros(2 * n + 1)
        A[:n, 0] = 1.0
        b[:n] = y - (x - x[0]) * s_true / c
        w[:n] = 1 / 0.01
        A[n:2 * n, 1] = 1.0
        A[n:2 * n, 2] = (x - x[0]) / c
        b[n:2 * n] = z
        w[n:2 * n] = 1 / 0.0225
        A[2 * n, 2] = 1.0
        b[2 * n] = t_seed
        w[2 * n] = 1 / 0.25
        N = A.T @ (w[:, None] * A)
        th = np.linalg.solve(N, A.T @ (w * b))
        cov_th = np.linalg.inv(N)
        yl = th[0] + (x[-1] - x[0]) * s_true / c
        zl = th[1] + th[2] * (x[-1] - x[0]) / c
        assert abs(p[0] - yl) < 1e-10 and abs(p[1] - zl) < 1e-10 and abs(p[3] - th[2]) < 1e-12
        # covariance of t and of the transported y, zeta
        Tz = np.array([0, 1, (x[-1] - x[0]) / c])
        assert abs(cov[9] - cov_th[2, 2]) < 1e-12
        assert abs(cov[2] - Tz @ cov_th @ Tz) < 1e-12
        assert abs(cov[0] - cov_th[0, 0]) < 1e-12


def test_zero_field_fit_close_to_batch_map():
    """With sin(phi) free the model is mildly nonlinear; the chained filter
    stays within 10 % of a standard deviation of the batch MAP estimate
    (the exact equality is pinned by the linear case above)."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(6)
    x = np.array([row_x(r) for r in range(0, 152, 3)])
    for _ in range(20):
        s_true, t_true, y, z = _line(rng, x)
        seed = np.array([0, 0, s_true + rng.normal(0, 0.01), t_true + rng.normal(0, 0.01), 0.0])
        rc, p, c = oracle.fit_points(x, y, z, 0.0, seed)
        assert rc == 0

        def res(th):
            y0, z0, s, t = th
            cc = math.sqrt(1 - s * s)
            ry = (y0 + (x - x[0]) * s / cc - y) / 0.1
            rz = (z0 + t * (x - x[0]) / cc - z) / 0.15
            return np.concatenate([ry, rz, [(s - seed[2]) / 0.2, (t - seed[3]) / 0.5]])

        sol = scipy_opt.least_squares(res, [y[0], z[0], seed[2], seed[3]], xtol=1e-15, ftol=1e-15, gtol=1e-15)
        y0, z0, s, t = sol.x
        cc = math.sqrt(1 - s * s)
        yl = y0 + (x[-1] - x[0]) * s / cc
        zl = z0 + t * (x[-1] - x[0]) / cc
        d = [abs(p[0] - yl) / math.sqrt(c[0]), abs(p[1] - zl) / math.sqrt(c[2]),
             abs(p[2] - s) / math.sqrt(c[5]), abs(p[3] - t) / math.sqrt(c[9])]
        assert max(d) < 0.1
        assert p[4] == 0.0 and abs(c[14] - 400.0) < 1e-9
