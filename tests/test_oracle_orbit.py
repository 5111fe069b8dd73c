"""Pins of the oracle's orbit integrals against facts fixed by the paper and the mathematics.

* Breakpoints vs brute-force knot scanning (§4.7, Eq. (breakpoint-set)).
* Closed-form orbit weights (Appendix A) and orbit gradient (Appendix B) vs adaptive
  quadrature of the point shape along the path (the definitions Eq. (orbit-average-shape)
  and Eq. (DA-def) integrated numerically, with no use of the closed forms).
* Partition of unity (Appendix A): sum_g S̄_ig = 1.
* Split Gauss rule equals the closed form for 2 n_q - 1 >= 3 (§4.7, §5.4).
* Exact orbit chain rule (Lemma "exact orbit chain rule", Eq. (exact-chain-rule)).
* Unsplit full-path quadrature leaves a chain-rule defect once the path crosses a knot
  (Table 1, Table 2 r = 1); the paper's exact Table values depend on fields it does not
  state, so only their roundoff bar and the qualitative contrast are pinned here.
"""

import numpy as np
import pytest
from scipy import integrate

from oracle import mesh, orbit


def _grid(n=(6, 5, 4), L=(1.2, 1.0, 0.8)):
    return mesh.Grid(n, L)


def _random_orbits(rng, npart, n, maxcells):
    xi0 = rng.uniform(0, 1, (npart, 3)) * np.asarray(n)
    beta = rng.uniform(-maxcells, maxcells, (npart, 3))
    return xi0, beta


def _special_orbits(n):
    """Edge cases: start on a knot, zero displacement on an axis, end on a knot, multi-knot."""
    xi0 = np.array([
        [2.0, 1.5, 0.25],       # start exactly on an x knot
        [1.25, 2.5, 1.75],      # zero displacement in y and z
        [0.5, 0.5, 0.5],        # ends exactly on knots in x
        [3.9, 0.1, 2.2],        # multi-knot crossings, wrap-around in y
        [n[0] - 0.3, 3.3, 3.7], # wrap-around in x (beyond the upper face)
        [1.3, 1.7, 2.1],        # no motion at all
    ])
    beta = np.array([
        [0.7, -0.4, 0.3],
        [1.6, 0.0, 0.0],
        [0.5, 0.2, -0.1],
        [-2.7, -1.4, 2.3],
        [0.9, -0.2, 0.6],
        [0.0, 0.0, 0.0],
    ])
    return xi0, beta


def _point_S(xi, g, n):
    """S_g at a single point xi (cell units): product of hat functions, periodic in g."""
    val = 1.0
    for a in range(3):
        dd = xi[a] - g[a]
        dd = dd - n[a] * np.round(dd / n[a])
        val *= max(0.0, 1.0 - abs(dd))
    return val


def _point_dS(xi, g, n, H, j):
    """d S_g / d x_j at a point that is not on a knot."""
    val = 1.0
    for a in range(3):
        dd = xi[a] - g[a]
        dd = dd - n[a] * np.round(dd / n[a])
        if a == j:
            if abs(dd) >= 1.0:
                return 0.0
            val *= -np.sign(dd) / H[a]
        else:
            val *= max(0.0, 1.0 - abs(dd))
    return val


def _bruteforce_knot_params(x, b):
    """Orbit parameters in (0, 1) at which x + s b crosses an integer, by scanning integers."""
    if b == 0:
        return []
    lo, hi = min(x, x + b), max(x, x + b)
    out = []
    for k in range(int(np.floor(lo)) - 1, int(np.ceil(hi)) + 2):
        s = (k - x) / b
        if 0 < s < 1:
            out.append(s)
    return out


def test_breakpoints_match_bruteforce_scan():
    rng = np.random.default_rng(1)
    n = (6, 5, 4)
    xi0, beta = _random_orbits(rng, 200, n, 3.0)
    xs, bs = _special_orbits(n)
    xi0 = np.concatenate([xi0, xs])
    beta = np.concatenate([beta, bs])
    s = orbit.breakpoints(xi0, beta)
    for i in range(xi0.shape[0]):
        expect = sorted(set([0.0, 1.0] + sum((_bruteforce_knot_params(xi0[i, a], beta[i, a]) for a in range(3)), [])))
        got = sorted(set(s[i].tolist()))
        assert np.allclose(got, expect, rtol=0, atol=1e-15), (i, got, expect)
        # each segment of positive length stays inside one cell on every axis
        for m in range(s.shape[1] - 1):
            a0, a1 = s[i, m], s[i, m + 1]
            if a1 - a0 <= 1e-12:
                continue
            probe = a0 + (a1 - a0) * np.array([1e-9, 0.25, 0.5, 0.75, 1 - 1e-9])
            cells = np.floor(xi0[i][None, :] + probe[:, None] * beta[i][None, :])
            assert np.all(cells == cells[0]), (i, m)


def _dense_weights(ow, npart, grid):
    """Accumulate entry weights into dense per-particle node arrays."""
    out = np.zeros((npart,) + grid.n)
    for i in range(npart):
        for k in range(ow.w.shape[1]):
            out[(i,) + tuple(ow.nodes[i, k])] += ow.w[i, k]
    return out


def test_closed_form_weights_match_adaptive_quadrature():
    grid = _grid()
    n = grid.n
    rng = np.random.default_rng(2)
    xi0, beta = _random_orbits(rng, 6, n, 2.5)
    xs, bs = _special_orbits(n)
    xi0 = np.concatenate([xi0, xs])
    beta = np.concatenate([beta, bs])
    ow = orbit.closed_form_weights(xi0, beta, grid)
    dense = _dense_weights(ow, xi0.shape[0], grid)
    for i in range(xi0.shape[0]):
        brk = sorted(set(sum((_bruteforce_knot_params(xi0[i, a], beta[i, a]) for a in range(3)), [])))
        for g in np.ndindex(*n):
            f = lambda s: _point_S(xi0[i] + s * beta[i], g, n)
            val, _ = integrate.quad(f, 0.0, 1.0, points=brk or None, epsabs=1e-14, epsrel=1e-13, limit=200)
            assert abs(dense[(i,) + g] - val) < 2e-13, (i, g, dense[(i,) + g], val)


def test_closed_form_gradient_matches_adaptive_quadrature():
    grid = _grid()
    n, H = grid.n, grid.H
    rng = np.random.default_rng(3)
    xi0, beta = _random_orbits(rng, 4, n, 2.2)
    xs, bs = _special_orbits(n)
    xi0 = np.concatenate([xi0, xs[:5]])
    beta = np.concatenate([beta, bs[:5]])
    An = rng.normal(size=(3,) + n)
    An1 = rng.normal(size=(3,) + n)
    ow = orbit.closed_form_weights(xi0, beta, grid)
    DA = orbit.orbit_gradient(An, An1, ow)
    for i in range(xi0.shape[0]):
        brk = sorted(set(sum((_bruteforce_knot_params(xi0[i, a], beta[i, a]) for a in range(3)), [])))
        for l in range(3):
            for j in range(3):
                def f(s):
                    x = xi0[i] + s * beta[i]
                    tot = 0.0
                    for g in np.ndindex(*n):
                        dS = _point_dS(x, g, n, H, j)
                        if dS != 0.0:
                            tot += ((1 - s) * An[(l,) + g] + s * An1[(l,) + g]) * dS
                    return tot
                val, _ = integrate.quad(f, 0.0, 1.0, points=brk or None, epsabs=1e-13, epsrel=1e-12, limit=200)
                assert abs(DA[i, l, j] - val) < 1e-11 * max(1.0, abs(val)), (i, l, j, DA[i, l, j], val)


def test_partition_of_unity():
    grid = _grid((8, 8, 8), (1.0, 1.0, 1.0))
    rng = np.random.default_rng(4)
    xi0, beta = _random_orbits(rng, 20000, grid.n, 3.5)
    ow = orbit.closed_form_weights(xi0, beta, grid, with_gradient=False)
    err = np.abs(np.sum(ow.w, axis=1) - 1.0)
    assert err.max() <= 8 * np.finfo(float).eps


@pytest.mark.parametrize("nq", [2, 3, 5, 8, 16])
def test_split_gauss_equals_closed_form(nq):
    """§5.4: with r = 1 and a split rule that is exact (2 n_q - 1 >= 3), the answer is identical."""
    grid = _grid()
    rng = np.random.default_rng(5)
    xi0, beta = _random_orbits(rng, 300, grid.n, 2.0)
    An = rng.normal(size=(3,) + grid.n)
    An1 = rng.normal(size=(3,) + grid.n)
    G = rng.normal(size=(3,) + grid.n)
    cf = orbit.closed_form_weights(xi0, beta, grid)
    gq = orbit.gauss_weights(xi0, beta, grid, nq=nq)
    np.testing.assert_allclose(orbit.gather(G, gq), orbit.gather(G, cf), rtol=0, atol=1e-13)
    np.testing.assert_allclose(orbit.orbit_gradient(An, An1, gq), orbit.orbit_gradient(An, An1, cf),
                               rtol=0, atol=1e-11)
    q_vbar = rng.normal(size=(xi0.shape[0], 3))
    np.testing.assert_allclose(orbit.deposit(q_vbar, gq, grid), orbit.deposit(q_vbar, cf, grid),
                               rtol=0, atol=1e-11)


def _chain_rule_residual(xi0, beta, An, An1, dt, grid, ow):
    """R_A of Eq. (RA-test) with U^{n+1/2} := (A^{n+1} - A^n)/dt (Eq. (A-U-CN))."""
    H = np.asarray(grid.H)
    vbar = beta * H / dt
    U_half = (An1 - An) / dt
    Ubar = orbit.gather(U_half, ow).T
    DA = orbit.orbit_gradient(An, An1, ow)
    end = orbit.point_gather(An1, xi0 + beta, grid).T
    start = orbit.point_gather(An, xi0, grid).T
    return end - start - dt * (Ubar + np.einsum("ilj,ij->il", DA, vbar))


def test_exact_orbit_chain_rule_random_fields():
    grid = _grid()
    rng = np.random.default_rng(6)
    xi0, beta = _random_orbits(rng, 5000, grid.n, 2.5)
    xs, bs = _special_orbits(grid.n)
    xi0 = np.concatenate([xi0, xs])
    beta = np.concatenate([beta, bs])
    An = rng.normal(size=(3,) + grid.n)
    An1 = rng.normal(size=(3,) + grid.n)
    ow = orbit.closed_form_weights(xi0, beta, grid)
    RA = _chain_rule_residual(xi0, beta, An, An1, 0.1, grid, ow)
    assert np.abs(RA).max() < 1e-13


def test_deposit_gather_identity():
    """Eq. (deposit-gather-identity): sum_i q vbar . Gbar_i = sum_g J_g . G_g dV."""
    grid = _grid()
    rng = np.random.default_rng(7)
    xi0, beta = _random_orbits(rng, 3000, grid.n, 2.0)
    q_vbar = rng.normal(size=(xi0.shape[0], 3))
    G = rng.normal(size=(3,) + grid.n)
    ow = orbit.closed_form_weights(xi0, beta, grid, with_gradient=False)
    J = orbit.deposit(q_vbar, ow, grid)
    lhs = np.sum(q_vbar * orbit.gather(G, ow).T)
    rhs = np.sum(J * G) * grid.dV
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(q_vbar)) * np.abs(G).max()


def _table_orbit(cross, beta=0.5):
    """A particle moving in x that crosses the knot at xi = 3 by ``cross`` cells (1D test of §4.7)."""
    start = 3.0 + cross - beta
    xi0 = np.array([[start, 1.5, 2.5]])
    b = np.array([[beta, 0.0, 0.0]])
    return xi0, b


def _table_fields(grid):
    """Smooth prescribed 1D fields A^n, A^{n+1} varying in x only (the paper's fields are not stated)."""
    x = np.arange(grid.n[0]) * grid.H[0]
    k = 2 * np.pi / grid.L[0]
    An = np.zeros((3,) + grid.n)
    An1 = np.zeros((3,) + grid.n)
    An[0] = (np.sin(k * x) + 0.3 * np.cos(2 * k * x))[:, None, None]
    An1[0] = (np.sin(k * x + 0.2) + 0.3 * np.cos(2 * k * x - 0.1))[:, None, None]
    return An, An1


def _load_tables():
    rows = {}
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "chain_rule_tables.txt")
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, deg, cross, unsplit, split = line.split()
        rows[(key, int(deg), float(cross))] = (float(unsplit), float(split))
    return rows


@pytest.mark.parametrize("cross", [0.01, 0.10])
def test_table1_split_restores_chain_rule_unsplit_does_not(cross):
    """Table 1 (r = 1): split-path residual at roundoff; full-path Gauss rule leaves a defect."""
    tables = _load_tables()
    paper_unsplit, paper_split = tables[("table1", 1, cross)]
    grid = mesh.Grid((8, 4, 4), (1.0, 1.0, 1.0))
    An, An1 = _table_fields(grid)
    xi0, beta = _table_orbit(cross)
    split = orbit.gauss_weights(xi0, beta, grid, nq=16, split=True)
    unsplit = orbit.gauss_weights(xi0, beta, grid, nq=16, split=False)
    r_split = np.abs(_chain_rule_residual(xi0, beta, An, An1, 0.1, grid, split)).max()
    r_unsplit = np.abs(_chain_rule_residual(xi0, beta, An, An1, 0.1, grid, unsplit)).max()
    assert r_split <= 10 * paper_split           # roundoff, as in the paper's split column
    assert r_unsplit > 1e6 * r_split             # a real defect once the knot is crossed
    assert r_unsplit > 1e-3 * paper_unsplit      # same order of magnitude band as the paper's defect


def test_unsplit_equals_split_without_crossing():
    grid = mesh.Grid((8, 4, 4), (1.0, 1.0, 1.0))
    An, An1 = _table_fields(grid)
    xi0 = np.array([[3.1, 1.5, 2.5]])
    beta = np.array([[0.5, 0.0, 0.0]])
    split = orbit.gauss_weights(xi0, beta, grid, nq=16, split=True)
    unsplit = orbit.gauss_weights(xi0, beta, grid, nq=16, split=False)
    r1 = _chain_rule_residual(xi0, beta, An, An1, 0.1, grid, split)
    r2 = _chain_rule_residual(xi0, beta, An, An1, 0.1, grid, unsplit)
    assert np.abs(r1).max() < 1e-15 and np.abs(r2).max() < 1e-15


def test_planted_mistake_dropping_C_term_breaks_chain_rule(monkeypatch):
    """A plausible Appendix B mistake (omit the C^{(m)} term) must fail the chain-rule pin."""
    grid = _grid()
    rng = np.random.default_rng(8)
    xi0, beta = _random_orbits(rng, 500, grid.n, 1.5)
    An = rng.normal(size=(3,) + grid.n)
    An1 = rng.normal(size=(3,) + grid.n)
    ow = orbit.closed_form_weights(xi0, beta, grid)
    ow.T1[:] = 0.0
    RA = _chain_rule_residual(xi0, beta, An, An1, 0.1, grid, ow)
    assert np.abs(RA).max() > 1e-3


def test_planted_mistake_global_s_ignored_breaks_chain_rule():
    """Appendix B stresses that A^{(m)} depends on the global s_m; anchoring at 0 must fail."""
    grid = _grid()
    rng = np.random.default_rng(9)
    xi0, beta = _random_orbits(rng, 500, grid.n, 2.5)
    An = rng.normal(size=(3,) + grid.n)
    An1 = rng.normal(size=(3,) + grid.n)
    ow = orbit.closed_form_weights(xi0, beta, grid)
    ow.s[:] = 0.0
    RA = _chain_rule_residual(xi0, beta, An, An1, 0.1, grid, ow)
    assert np.abs(RA).max() > 1e-3
