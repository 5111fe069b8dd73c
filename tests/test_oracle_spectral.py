"""Pins of the oracle's spectral operators (ops = "spectral", the paper's choice in §3.3).

* D_a of a Fourier mode below the Nyquist index is k_a times the differentiated mode
  (closed form), and D_a of the Nyquist checkerboard is zero (the reading that keeps D_a
  real and skew-adjoint).
* The identities the theorems need: Delta_h = nabla_h . nabla_h, summation by parts,
  div curl = 0, curl grad = 0, curl curl = grad div - Delta_h.
* CN vacuum mode: the Cayley rotation with the exact dispersion omega = kappa |k|.
* Poisson of a single mode: phi = sigma1 rho / |k|^2.
* Gauge / Gauss preservation and field-energy balance over a run with random currents, and
  energy conservation of whole particle steps.
"""

import numpy as np

from oracle import mesh
from oracle import pic as opic


def _grid(n=(8, 6, 10), L=(1.0, 1.3, 0.7)):
    return mesh.Grid(n, L, "spectral")


def _coords(grid):
    return np.meshgrid(*[np.arange(grid.n[a]) * grid.H[a] for a in range(3)], indexing="ij")


def test_spectral_derivative_of_fourier_modes():
    grid = _grid()
    X = _coords(grid)
    m = (2, 1, 3)
    k = [2 * np.pi * m[a] / grid.L[a] for a in range(3)]
    phase = k[0] * X[0] + k[1] * X[1] + k[2] * X[2]
    f = np.sin(phase)
    for a in range(3):
        np.testing.assert_allclose(mesh.d(f, a, grid), k[a] * np.cos(phase), atol=1e-11)
    I = np.meshgrid(*[np.arange(grid.n[a]) for a in range(3)], indexing="ij")
    nyq = (-1.0) ** I[0]                                   # Nyquist mode along x (n_x even)
    assert np.abs(mesh.d(nyq, 0, grid)).max() < 1e-12


def test_spectral_operator_identities():
    grid = _grid()
    rng = np.random.default_rng(41)
    f, g = rng.normal(size=(2,) + grid.n)
    F = rng.normal(size=(3,) + grid.n)
    np.testing.assert_allclose(mesh.lap(f, grid), mesh.div(mesh.grad(f, grid), grid), atol=1e-8)
    for a in range(3):
        assert abs(np.sum(f * mesh.d(g, a, grid)) + np.sum(mesh.d(f, a, grid) * g)) < 1e-9
    assert np.abs(mesh.div(mesh.curl(F, grid), grid)).max() < 1e-9
    assert np.abs(mesh.curl(mesh.grad(f, grid), grid)).max() < 1e-9
    lhs = mesh.curl(mesh.curl(F, grid), grid)
    rhs = mesh.grad(mesh.div(F, grid), grid) - np.stack([mesh.lap(F[c], grid) for c in range(3)])
    np.testing.assert_allclose(lhs, rhs, atol=1e-7)


def test_spectral_cn_vacuum_mode_is_cayley_rotation():
    grid = _grid()
    X = _coords(grid)
    m = (1, 2, 1)
    k = [2 * np.pi * m[a] / grid.L[a] for a in range(3)]
    u0 = np.cos(k[0] * X[0] + k[1] * X[1] + k[2] * X[2])
    kappa, dt = 1.3, 0.07
    omega = kappa * np.sqrt(sum(kk * kk for kk in k))       # exact dispersion of the continuum
    theta = 2.0 * np.arctan(0.5 * omega * dt)
    u, w = u0.copy(), np.zeros(grid.n)
    zero = np.zeros(grid.n)
    for nstep in range(1, 31):
        u, w = mesh.cn_update(u, w, zero, 1.0, dt, kappa, grid)
        np.testing.assert_allclose(u, np.cos(nstep * theta) * u0, atol=1e-11)


def test_spectral_poisson_single_mode():
    grid = _grid((8, 8, 8), (1.0, 1.0, 1.0))
    X = _coords(grid)
    k = 2 * np.pi * np.array([1.0, 2.0, 0.0])
    rho = np.cos(k[0] * X[0] + k[1] * X[1])
    phi = mesh.poisson(rho, 1.7, grid)
    np.testing.assert_allclose(phi, 1.7 * rho / np.dot(k, k), atol=1e-13)


def test_spectral_gauge_gauss_and_field_energy_over_a_run():
    grid = _grid((8, 8, 6), (1.0, 1.1, 0.9))
    rng = np.random.default_rng(42)
    kappa, sigma2, dt = 1.2, 0.9, 0.05
    sigma1 = kappa ** 2 * sigma2
    rho = mesh.project_out_null(rng.normal(size=grid.n), grid)
    phi, psi = mesh.poisson(rho, sigma1, grid), np.zeros(grid.n)
    A, U = np.zeros((3,) + grid.n), np.zeros((3,) + grid.n)
    for _ in range(10):
        J = rng.normal(size=(3,) + grid.n)
        rho1 = mesh.continuity(rho, J, dt, grid)
        phi1, psi1, A1, U1 = mesh.cn_fields(phi, psi, A, U, 0.5 * (rho1 + rho), J, dt, kappa, sigma1, sigma2, grid)
        W0 = mesh.field_energy(phi, U, A, sigma1, sigma2, grid)
        W1 = mesh.field_energy(phi1, U1, A1, sigma1, sigma2, grid)
        work = np.sum(J * mesh.efield(0.5 * (phi1 + phi), 0.5 * (U1 + U), grid)) * grid.dV
        phi, psi, A, U, rho = phi1, psi1, A1, U1, rho1
        assert np.abs(mesh.gauge_residual(psi, A, kappa, grid)).max() < 1e-10
        assert np.abs(mesh.gauss_residual(phi, U, rho, sigma1, grid)).max() < 1e-9
        assert abs(W1 - W0 + dt * work) < 1e-12 * max(1.0, W1)


def test_spectral_whole_steps_conserve_energy():
    import pic_inputs as pi
    n, L = (8, 6, 6), (1.2, 1.0, 1.0)
    x, v, q, m = pi.random_twostream(n, L, 2, 0.3, 1e-2, 2e-2, 4100)
    cfg = opic.Config(n=n, L=L, dt=0.1, picard_tol=1e-14, ops="spectral")
    st = opic.init(x, v, q, m, cfg)
    for _ in range(3):
        st, info = opic.step(st, cfg)
        assert info["converged"]
        assert abs(info["R_total"]) <= 1e-13 * (info["K1"] + info["W1"])
        assert np.abs(info["RA"]).max() <= 1e-14
        md = opic.mesh_diagnostics(st, cfg)
        assert np.abs(md["gauge"]).max() <= 1e-10 and np.abs(md["gauss"]).max() <= 1e-10
