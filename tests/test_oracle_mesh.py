"""Pins of the oracle's mesh side against closed forms and the paper's theorems.

* Central difference of a Fourier mode equals i sin(theta)/H times the mode (closed form,
  evaluated from cos/sin directly).
* Operator identities the theorems need: Delta_h = nabla_h . nabla_h, summation by parts,
  div curl = 0, curl grad = 0, curl curl = grad div - Delta_h (§3.3 proof, §4.6).
* CN vacuum mode: the exact per-mode CN solve of Eq. (cn-field-update) equals the
  closed-form Cayley rotation u^n = u^0 cos(n theta), tan(theta/2) = omega dt / 2.
* The per-mode solution satisfies the CN equations written with the real-space stencil.
* Poisson and null-mode projection (§5.4 initial data).
* Theorem "gauge and Gauss preservation": with continuity-advanced rho and arbitrary
  J, G_h and R_h stay at roundoff (and a planted compact Laplacian breaks it).
* Field energy balance Eq. (field-energy-final).
"""

import numpy as np

from oracle import mesh


def _grid(n=(8, 6, 10), L=(1.0, 1.3, 0.7)):
    return mesh.Grid(n, L)


def _coords(grid):
    return np.meshgrid(*[np.arange(grid.n[a]) * grid.H[a] for a in range(3)], indexing="ij")


def test_central_difference_of_fourier_mode():
    grid = _grid()
    X = _coords(grid)
    m = (2, 1, 3)
    k = [2 * np.pi * m[a] / grid.L[a] for a in range(3)]
    phase = k[0] * X[0] + k[1] * X[1] + k[2] * X[2]
    f = np.sin(phase)
    for a in range(3):
        expect = np.sin(k[a] * grid.H[a]) / grid.H[a] * np.cos(phase)
        np.testing.assert_allclose(mesh.d(f, a, grid), expect, atol=1e-12)


def test_operator_identities():
    grid = _grid()
    rng = np.random.default_rng(11)
    f = rng.normal(size=grid.n)
    g = rng.normal(size=grid.n)
    F = rng.normal(size=(3,) + grid.n)
    np.testing.assert_allclose(mesh.lap(f, grid), mesh.div(mesh.grad(f, grid), grid), atol=1e-10)
    for a in range(3):
        assert abs(np.sum(f * mesh.d(g, a, grid)) + np.sum(mesh.d(f, a, grid) * g)) < 1e-10
    assert np.abs(mesh.div(mesh.curl(F, grid), grid)).max() < 1e-10
    assert np.abs(mesh.curl(mesh.grad(f, grid), grid)).max() < 1e-10
    lhs = mesh.curl(mesh.curl(F, grid), grid)
    rhs = mesh.grad(mesh.div(F, grid), grid) - np.stack([mesh.lap(F[c], grid) for c in range(3)])
    np.testing.assert_allclose(lhs, rhs, atol=1e-8)


def test_lap_symbol_matches_stencil():
    grid = _grid()
    rng = np.random.default_rng(12)
    f = rng.normal(size=grid.n)
    via_symbol = np.real(np.fft.ifftn(grid.lap_symbol() * np.fft.fftn(f)))
    np.testing.assert_allclose(via_symbol, mesh.lap(f, grid), atol=1e-9)


def test_cn_vacuum_mode_is_cayley_rotation():
    grid = _grid()
    X = _coords(grid)
    m = (1, 2, 1)
    k = [2 * np.pi * m[a] / grid.L[a] for a in range(3)]
    u0 = np.cos(k[0] * X[0] + k[1] * X[1] + k[2] * X[2])
    kappa, dt = 1.3, 0.07
    omega = kappa * np.sqrt(sum((np.sin(k[a] * grid.H[a]) / grid.H[a]) ** 2 for a in range(3)))
    theta = 2.0 * np.arctan(0.5 * omega * dt)
    u, w = u0.copy(), np.zeros(grid.n)
    zero = np.zeros(grid.n)
    for nstep in range(1, 41):
        u, w = mesh.cn_update(u, w, zero, 1.0, dt, kappa, grid)
        np.testing.assert_allclose(u, np.cos(nstep * theta) * u0, atol=1e-12)
        np.testing.assert_allclose(w, -omega * np.sin(nstep * theta) * u0, atol=1e-11)


def test_cn_solution_satisfies_stencil_equations():
    grid = _grid()
    rng = np.random.default_rng(13)
    u0, w0, src = rng.normal(size=(3,) + grid.n)
    kappa, coef, dt = 1.0, 0.8, 0.1
    u1, w1 = mesh.cn_update(u0, w0, src, coef, dt, kappa, grid)
    r1 = (u1 - u0) / dt - 0.5 * (w1 + w0)
    r2 = (w1 - w0) / dt - kappa ** 2 * mesh.lap(0.5 * (u1 + u0), grid) - kappa ** 2 * coef * src
    assert np.abs(r1).max() < 1e-11 and np.abs(r2).max() < 1e-9


def test_poisson_and_null_projection():
    grid = _grid((8, 6, 4), (1.0, 1.0, 1.0))
    rng = np.random.default_rng(14)
    rho = mesh.project_out_null(rng.normal(size=grid.n), grid)
    I = np.meshgrid(*[np.arange(grid.n[a]) for a in range(3)], indexing="ij")
    for a in np.ndindex(2, 2, 2):
        pattern = (-1.0) ** (a[0] * I[0] + a[1] * I[1] + a[2] * I[2])
        assert abs(np.sum(rho * pattern)) < 1e-12
    phi = mesh.poisson(rho, 1.7, grid)
    np.testing.assert_allclose(-mesh.lap(phi, grid), 1.7 * rho, atol=1e-11)


def _constrained_start(grid, rng, sigma1):
    rho = mesh.project_out_null(rng.normal(size=grid.n), grid)
    phi = mesh.poisson(rho, sigma1, grid)
    return phi, np.zeros(grid.n), np.zeros((3,) + grid.n), np.zeros((3,) + grid.n), rho


def _run_fields(grid, lap_fn=None, steps=12):
    rng = np.random.default_rng(15)
    kappa, sigma2, dt = 1.2, 0.9, 0.05
    sigma1 = kappa ** 2 * sigma2          # Eq. (Maxwell_scaling)
    phi, psi, A, U, rho = _constrained_start(grid, rng, sigma1)
    out = []
    for _ in range(steps):
        J = rng.normal(size=(3,) + grid.n)
        rho1 = mesh.continuity(rho, J, dt, grid)
        phi1, psi1, A1, U1 = mesh.cn_fields(phi, psi, A, U, 0.5 * (rho1 + rho), J, dt, kappa, sigma1, sigma2, grid)
        W0 = mesh.field_energy(phi, U, A, sigma1, sigma2, grid)
        W1 = mesh.field_energy(phi1, U1, A1, sigma1, sigma2, grid)
        Eh = mesh.efield(0.5 * (phi1 + phi), 0.5 * (U1 + U), grid)
        work = np.sum(J * Eh) * grid.dV
        phi, psi, A, U, rho = phi1, psi1, A1, U1, rho1
        G = mesh.gauge_residual(psi, A, kappa, grid)
        R = mesh.gauss_residual(phi, U, rho, sigma1, grid)
        out.append((np.abs(G).max(), np.abs(R).max(), W1 - W0 + dt * work, W1))
    return out


def test_gauge_gauss_preserved_and_field_energy_balance():
    grid = _grid((8, 8, 6), (1.0, 1.1, 0.9))
    for G, R, Rfield, W in _run_fields(grid):
        assert G < 1e-11 and R < 1e-10
        assert abs(Rfield) < 1e-12 * max(1.0, W)


def test_planted_compact_laplacian_breaks_gauge(monkeypatch):
    """Using the compact 7-point Laplacian in the CN solve (Delta_h != nabla_h . nabla_h) must fail."""
    grid = _grid((8, 8, 6), (1.0, 1.1, 0.9))
    orig = mesh.Grid.lap_symbol

    def compact(self):
        th = self.wavenumbers()
        return sum(-(2 - 2 * np.cos(th[a])) / self.H[a] ** 2 for a in range(3))

    monkeypatch.setattr(mesh.Grid, "lap_symbol", compact)
    res = _run_fields(grid)
    monkeypatch.setattr(mesh.Grid, "lap_symbol", orig)
    assert max(G for G, _, _, _ in res) > 1e-6 or max(R for _, R, _, _ in res) > 1e-6
