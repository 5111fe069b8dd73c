"""Pins of the oracle's higher-order shapes (B-spline degree r = 2, 3; §4.7, Table 2).

* The centred cardinal B-splines and their derivatives equal scipy's B-spline basis elements
  on the same knots (a library routine, not the oracle's recursion).
* Partition of unity of the point shape, and of the split-Gauss orbit weights S̄.
* Split-Gauss orbit weights S̄ and orbit gradient D_i A equal adaptive quadrature of the
  point shape along the path (the definitions Eq. (split-Sbar), Eq. (split-DA)).
* With 2 n_q - 1 >= 3r (§4.7), the exact orbit chain rule R_A = 0 (Eq. (RA-test)) holds to
  roundoff for random fields; the unsplit path leaves a defect once it crosses a knot, and
  that defect shrinks with the degree (Table 2's qualitative order; its exact values depend
  on fields the paper does not state).
* Planted mistake: splitting at the linear spline's knots (integers) instead of the quadratic
  spline's (half-integers) breaks the chain rule.
* A whole step with r = 2 and r = 3 conserves energy and keeps the gauge / Gauss residuals.
"""

import numpy as np
import pytest
from scipy import integrate
from scipy.interpolate import BSpline

from oracle import mesh, orbit
from oracle import pic as opic


def _grid(n=(7, 6, 5), L=(1.4, 1.2, 1.0)):
    return mesh.Grid(n, L)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_bspline_matches_scipy_basis_element(r):
    knots = np.arange(r + 2) - 0.5 * (r + 1)            # centred knots of degree r
    ref = BSpline.basis_element(knots, extrapolate=False)
    x = np.linspace(-0.5 * (r + 1) + 1e-9, 0.5 * (r + 1) - 1e-9, 2001)
    x = x[np.abs(x - np.round(x * 2) / 2) > 1e-7]      # off the knots (both lattices)
    np.testing.assert_allclose(orbit.bspline(x, r), np.nan_to_num(ref(x)), rtol=0, atol=1e-14)
    np.testing.assert_allclose(orbit.bspline_deriv(x, r), np.nan_to_num(ref.derivative()(x)), rtol=0, atol=1e-13)
    assert np.all(orbit.bspline(np.array([-0.5 * (r + 1) - 0.1, 0.5 * (r + 1) + 0.1]), r) == 0.0)


@pytest.mark.parametrize("r", [2, 3])
def test_point_shape_partition_of_unity(r):
    grid = _grid()
    rng = np.random.default_rng(20 + r)
    xi = rng.uniform(0, 1, (500, 3)) * np.asarray(grid.n)
    nodes, S, dS = orbit.point_shape(xi, grid, r)
    assert nodes.shape == (500, (r + 1) ** 3, 3)
    np.testing.assert_allclose(S.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(dS.sum(axis=1), 0.0, rtol=0, atol=1e-12)
    assert np.all(S >= -1e-16)


def _point_S(xi, g, n, r):
    val = 1.0
    for a in range(3):
        dd = xi[a] - g[a]
        dd = dd - n[a] * np.round(dd / n[a])
        val *= float(orbit.bspline(np.array([dd]), r)[0])
    return val


def _point_dS(xi, g, n, H, j, r):
    val = 1.0
    for a in range(3):
        dd = xi[a] - g[a]
        dd = dd - n[a] * np.round(dd / n[a])
        f = orbit.bspline_deriv(np.array([dd]), r)[0] / H[a] if a == j else orbit.bspline(np.array([dd]), r)[0]
        val *= float(f)
    return val


def _dense(ow, i, grid, what="w", j=None):
    out = np.zeros(grid.n)
    for k in range(ow.w.shape[1]):
        out[tuple(ow.nodes[i, k])] += ow.w[i, k] if what == "w" else ow.T0[i, k, j]
    return out


@pytest.mark.parametrize("r", [2, 3])
def test_split_gauss_weights_match_adaptive_quadrature(r):
    grid = _grid()
    n, H = grid.n, np.asarray(grid.H)
    xi0 = np.array([[2.3, 1.45, 3.1], [4.9, 0.6, 0.55], [1.2, 2.2, 2.7]])
    beta = np.array([[0.9, -0.4, 0.25], [-1.3, 0.7, -0.2], [0.05, 0.0, 1.6]])
    nq = (3 * r + 2) // 2
    ow = orbit.gauss_weights(xi0, beta, grid, nq=nq, split=True, order=r)
    kn = orbit.breakpoints(xi0 - orbit.knot_offset(r), beta)
    for i in range(xi0.shape[0]):
        pts = [p for p in kn[i] if 0 < p < 1]
        Wd = _dense(ow, i, grid)
        for g in np.ndindex(*n):
            if abs(Wd[g]) < 1e-300 and _point_S(xi0[i] + 0.5 * beta[i], g, n, r) == 0.0:
                continue
            ref = integrate.quad(lambda s: _point_S(xi0[i] + s * beta[i], g, n, r), 0, 1, points=pts or None,
                                 epsabs=1e-15, epsrel=1e-13, limit=200)[0]
            assert abs(Wd[g] - ref) < 1e-12, (i, g, Wd[g], ref)
        for j in range(3):
            Td = _dense(ow, i, grid, "T0", j)
            for g in np.ndindex(*n):
                ref = integrate.quad(lambda s: _point_dS(xi0[i] + s * beta[i], g, n, H, j, r), 0, 1,
                                     points=pts or None, epsabs=1e-14, epsrel=1e-12, limit=200)[0]
                assert abs(Td[g] - ref) < 1e-10 * max(1.0, 1.0 / H[j]), (i, j, g, Td[g], ref)
        np.testing.assert_allclose(ow.w[i].sum(), 1.0, rtol=0, atol=1e-14)


def _RA(xi0, beta, An, An1, dt, grid, ow, r):
    H = np.asarray(grid.H)
    vbar = beta * H / dt
    Ubar = orbit.gather((An1 - An) / dt, ow).T
    DA = orbit.orbit_gradient(An, An1, ow)
    end = orbit.point_gather(An1, xi0 + beta, grid, r).T
    start = orbit.point_gather(An, xi0, grid, r).T
    return end - start - dt * (Ubar + np.einsum("ilj,ij->il", DA, vbar))


@pytest.mark.parametrize("r", [2, 3])
def test_exact_chain_rule_split_and_defect_unsplit(r):
    grid = _grid()
    rng = np.random.default_rng(30 + r)
    xi0 = rng.uniform(0, 1, (400, 3)) * np.asarray(grid.n)
    beta = rng.uniform(-1.5, 1.5, (400, 3))
    An, An1 = rng.normal(size=(3,) + grid.n), rng.normal(size=(3,) + grid.n)
    nq = (3 * r + 2) // 2                                   # smallest n_q with 2 n_q - 1 >= 3 r
    split = orbit.gauss_weights(xi0, beta, grid, nq=nq, split=True, order=r)
    assert np.abs(_RA(xi0, beta, An, An1, 0.1, grid, split, r)).max() < 1e-12
    unsplit = orbit.gauss_weights(xi0, beta, grid, nq=nq, split=False, order=r)
    assert np.abs(_RA(xi0, beta, An, An1, 0.1, grid, unsplit, r)).max() > 1e-6
    # planted mistake: split at the knots of the other lattice (integers for r = 2, half-integers for r = 3)
    saved = orbit.knot_offset
    try:
        orbit.knot_offset = lambda order: 0.5 - saved(order)
        bad = orbit.gauss_weights(xi0, beta, grid, nq=nq, split=True, order=r)
    finally:
        orbit.knot_offset = saved
    assert np.abs(_RA(xi0, beta, An, An1, 0.1, grid, bad, r)).max() > 1e-8


def test_unsplit_defect_decreases_with_degree():
    """Table 2: crossing a knot by 0.10 cell, the unsplit full-path rule's defect falls with the
    degree while the split rule stays at roundoff (smooth 1D fields varying in x)."""
    grid = mesh.Grid((16, 4, 4), (1.0, 0.25, 0.25))
    x = np.arange(16) * grid.H[0]
    k = 2 * np.pi
    An = np.zeros((3,) + grid.n)
    An1 = np.zeros((3,) + grid.n)
    An[0] = (np.sin(k * x) + 0.3 * np.cos(2 * k * x))[:, None, None]
    An1[0] = (np.sin(k * x + 0.2) + 0.3 * np.cos(2 * k * x - 0.1))[:, None, None]
    defects, splits = [], []
    for r in (1, 2, 3):
        koff = orbit.knot_offset(r)
        knot = 7.0 + koff
        xi0 = np.array([[knot + 0.1 - 0.5, 1.5, 2.5]])
        beta = np.array([[0.5, 0.0, 0.0]])
        nq = 8
        un = orbit.gauss_weights(xi0, beta, grid, nq=nq, split=False, order=r)
        sp = orbit.gauss_weights(xi0, beta, grid, nq=nq, split=True, order=r)
        defects.append(np.abs(_RA(xi0, beta, An, An1, 0.1, grid, un, r)).max())
        splits.append(np.abs(_RA(xi0, beta, An, An1, 0.1, grid, sp, r)).max())
    assert defects[0] > defects[1] > defects[2] > 1e-12
    assert max(splits) < 1e-14


@pytest.mark.parametrize("r", [2, 3])
def test_whole_step_conserves_energy(r):
    import pic_inputs as pi
    n, L = (5, 5, 4), (1.0, 1.0, 0.8)
    x, v, q, m = pi.random_twostream(n, L, 1, 0.3, 1e-2, 2e-2, 4000 + r)
    cfg = opic.Config(n=n, L=L, dt=0.1, picard_tol=1e-14, quadrature="gauss", nq=(3 * r + 2) // 2, order=r)
    st = opic.init(x, v, q, m, cfg)
    e0 = sum(opic.energy(st, cfg))
    for _ in range(2):
        st, info = opic.step(st, cfg)
        assert info["converged"]
        assert abs(info["R_total"]) <= 1e-13 * (info["K1"] + info["W1"])
        assert np.abs(info["RA"]).max() <= 1e-13
        assert np.abs(info["partition_of_unity"]).max() <= 1e-13
        md = opic.mesh_diagnostics(st, cfg)
        assert np.abs(md["gauge"]).max() <= 1e-11 and np.abs(md["gauss"]).max() <= 1e-11
    assert abs(sum(opic.energy(st, cfg)) - e0) <= 1e-13 * e0
