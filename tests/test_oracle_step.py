"""Pins of the oracle's whole time step (Algorithm 1) against what the paper proves and measures.

* Theorem "discrete total energy conservation": R_total at roundoff for the converged
  split-orbit step; R_field and R_particle (Eq. (R-field), Eq. (R-particle)) at solver
  tolerance; R_A (Eq. (RA-test)) at roundoff; partition of unity; exact continuity;
  gauge and Gauss residuals (§5.1) at roundoff.
* The unsplit comparison run (§5.4): G_h, R_h still at roundoff, R_A and the energy
  defect not (figures of §5.4).
* Split Gauss quadrature reproduces the closed-form step (§5.4, "the answer is identical").
* Cold two-stream linear growth (§5.4 physics) against the cold symmetric two-beam
  dispersion relation 1 = (w_p^2/2)[(w - k v0)^-2 + (w + k v0)^-2], started on its
  growing eigenmode.
* Planted mistakes: pushing with (D A) instead of (D A)^T must break energy
  conservation.
* The energy error of a step closed from a non-converged iterate v* (the final sweep of §5.4
  from v*): the field-energy balance and the orbit's power balance hold for the orbit of v*
  whatever v* is, so R_total = (m/2) sum_i (v_i^{n+1} - v_i^n) . (G(v*)_i - v*_i), second order
  in the step's velocity change and the fixed-point residual.  The mixed path's tolerance and
  its final sweep's check of the accepted iterate's own residual rest on this identity.
"""

import numpy as np
import pytest

import pic_inputs as pi
from oracle import mesh, orbit, pic


def _c1_small(per_beam=8, n=(8, 8, 8), tol=1e-14):
    w = pi.WORKLOADS["twostream-8c-8k"]
    x, v, q, m = pi.random_twostream(n, w.L, per_beam, w.v0, w.eps, 0.0, w.seed)
    cfg = pic.Config(n=n, L=w.L, dt=w.dt, picard_tol=tol)
    return pic.init(x, v, q, m, cfg), cfg


def _check_step_identities(info, new, cfg, E0):
    grid = cfg.grid()
    assert info["converged"]
    assert abs(info["R_total"]) <= 1e-14 * E0
    assert abs(info["R_field"]) <= 1e-14 * E0
    assert abs(info["R_particle"]) <= 1e-13 * E0
    assert np.abs(info["RA"]).max() <= 1e-15
    assert np.abs(info["partition_of_unity"]).max() <= 8 * np.finfo(float).eps
    assert np.abs(info["continuity"]).max() <= 1e-14 * max(1.0, np.abs(new.rho).max())
    md = pic.mesh_diagnostics(new, cfg)
    assert np.abs(md["gauge"]).max() <= 1e-12
    assert np.abs(md["gauss"]).max() <= 1e-12 * max(1.0, np.abs(new.rho).max())
    # the power identity of Eq. (power-test)
    assert abs(info["particle_work"] - info["mesh_work"]) <= 1e-13 * max(1e-3, abs(info["mesh_work"]))


def test_split_step_conserves_energy_and_constraints():
    st, cfg = _c1_small()
    K, W = pic.energy(st, cfg)
    E0 = K + W
    for _ in range(4):
        new, info = pic.step(st, cfg)
        _check_step_identities(info, new, cfg, E0)
        st = new
    K1, W1 = pic.energy(st, cfg)
    assert abs((K1 + W1) - E0) <= 1e-14 * E0


def test_initial_state_satisfies_constraints():
    st, cfg = _c1_small()
    md = pic.mesh_diagnostics(st, cfg)
    assert np.abs(md["gauge"]).max() == 0.0
    assert np.abs(md["gauss"]).max() <= 1e-12
    assert abs(np.mean(st.rho)) <= 1e-15
    np.testing.assert_array_equal(st.vprev, st.v)


def test_split_gauss_step_equals_closed_form_step():
    st, cfg = _c1_small(per_beam=2)
    cfg_g = pic.Config(n=cfg.n, L=cfg.L, dt=cfg.dt, picard_tol=cfg.picard_tol, quadrature="gauss", nq=2)
    a, ia = pic.step(st, cfg)
    b, ib = pic.step(st, cfg_g)
    assert ia["converged"] and ib["converged"]
    np.testing.assert_allclose(b.v, a.v, rtol=0, atol=1e-14)
    np.testing.assert_allclose(b.P, a.P, rtol=0, atol=1e-16)
    np.testing.assert_allclose(b.phi, a.phi, rtol=0, atol=1e-13)
    np.testing.assert_allclose(b.A, a.A, rtol=0, atol=1e-15)


def test_unsplit_run_keeps_constraints_but_breaks_chain_rule():
    st, cfg = _c1_small(per_beam=2)
    cfg_u = pic.Config(n=cfg.n, L=cfg.L, dt=cfg.dt, picard_tol=1e-13, quadrature="gauss", nq=16, split=False)
    K, W = pic.energy(st, cfg)
    E0 = K + W
    ra_split, ra_unsplit, rp_unsplit = 0.0, 0.0, 0.0
    s1, s2 = st, st
    for _ in range(3):
        s1, i1 = pic.step(s1, cfg)
        s2, i2 = pic.step(s2, cfg_u)
        assert i1["converged"] and i2["converged"]
        ra_split = max(ra_split, np.abs(i1["RA"]).max())
        ra_unsplit = max(ra_unsplit, np.abs(i2["RA"]).max())
        rp_unsplit = max(rp_unsplit, abs(i2["R_particle"]))
        md = pic.mesh_diagnostics(s2, cfg_u)
        assert np.abs(md["gauge"]).max() <= 1e-12
        assert np.abs(md["gauss"]).max() <= 1e-11
        assert abs(i2["R_field"]) <= 1e-14 * E0
    assert ra_unsplit > 1e6 * max(ra_split, 1e-22)
    assert rp_unsplit > 1e-12 * E0


def test_nonconvergence_keeps_state():
    st, cfg = _c1_small(per_beam=2)
    cfg1 = pic.Config(n=cfg.n, L=cfg.L, dt=cfg.dt, picard_tol=1e-14, picard_max=1)
    new, info = pic.step(st, cfg1)
    assert not info["converged"]
    assert new is st


def _eigenmode_start(nx=16, pairs=16, E0=1e-4, v0=0.2):
    """Lattice start (§5.4) displaced and kicked along the growing eigenmode of the cold beams."""
    L = (2 * np.pi / 3, 0.5, 0.5)
    x, v, q, m = pi.lattice_twostream((nx, 2, 2), L, pairs, v0, 0.0, mode=1)
    k = 2 * np.pi / L[0]
    a = k * v0
    gam = np.sqrt(-(2 * a * a + 1 - np.sqrt(1 + 8 * a * a)) / 2)
    npair = x.shape[0] // 2
    for s, sl in [(1, slice(0, npair)), (-1, slice(npair, None))]:
        om = 1j * gam
        dv = -1j * E0 / (om - s * a)                 # cold-fluid velocity response (q/m = -1)
        dn = (k * 0.5) * dv / (om - s * a)           # beam density response (n0/2 per beam)
        disp = 1j * dn / (k * 0.5)                   # displacement giving that density
        x0 = x[sl, 0].copy()
        x[sl, 0] = np.mod(x0 + np.real(disp * np.exp(1j * k * x0)), L[0])
        v[sl, 0] += np.real(dv * np.exp(1j * k * x0))
    cfg = pic.Config(n=(nx, 2, 2), L=L, dt=0.1, picard_tol=1e-12)
    return pic.init(x, v, q, m, cfg), cfg, gam


def test_two_stream_linear_growth_matches_dispersion_relation():
    st, cfg, gam = _eigenmode_start()
    amps = []
    for _ in range(40):
        st, info = pic.step(st, cfg)
        assert info["converged"]
        amps.append(abs(np.fft.fft(st.rho.mean(axis=(1, 2)))[1]))
    t = 0.1 * np.arange(1, 41)
    sel = t >= 0.5
    g = np.polyfit(t[sel], np.log(np.asarray(amps)[sel]), 1)[0]
    assert abs(g - gam) <= 0.02 * gam, (g, gam)


def _transverse_A_start(amp=0.05, nx=8, pairs=4):
    """Lattice start (§5.4) whose fields depend on x only, with a transverse A_y(x) seeded.

    Every y-z cell holds the same particles, so deposits, and hence all fields, stay
    independent of y and z.  A_y(x) = amp sin(k x) is divergence free, so the Lorenz
    gauge still holds with psi = 0; P = m v + q A_h(x) keeps the canonical relation.
    """
    L = (2 * np.pi / 3, 0.6, 0.6)
    n = (nx, 4, 4)
    x, v, q, m = pi.lattice_twostream(n, L, pairs, 0.2, 1e-3, mode=1)
    cfg = pic.Config(n=n, L=L, dt=0.1, picard_tol=1e-13)
    st = pic.init(x, v, q, m, cfg)
    grid = cfg.grid()
    xs = np.arange(n[0]) * grid.H[0]
    A = np.zeros((3,) + n)
    A[1] = (amp * np.sin(2 * np.pi * xs / L[0]))[:, None, None]
    A[2] = (0.5 * amp * np.cos(4 * np.pi * xs / L[0]))[:, None, None]
    st = pic.replace(st, A=A)
    st = pic.replace(st, P=st.m * st.v + st.q * orbit.point_gather(A, st.xi, grid).T)
    return st, cfg


def test_split_step_conserves_energy_with_strong_vector_potential():
    st, cfg = _transverse_A_start()
    assert np.abs(pic.mesh_diagnostics(st, cfg)["gauge"]).max() < 1e-12
    K, W = pic.energy(st, cfg)
    E0 = K + W
    for _ in range(3):
        new, info = pic.step(st, cfg)
        assert info["converged"]
        assert abs(info["R_total"]) <= 1e-13 * E0
        assert abs(info["R_particle"]) <= 1e-12 * E0
        assert np.abs(info["RA"]).max() <= 1e-14
        md = pic.mesh_diagnostics(new, cfg)
        assert np.abs(md["gauge"]).max() <= 1e-11
        st = new


def test_canonical_momentum_conserved_along_symmetry_directions():
    """With fields independent of y and z, Eq. (orbit-P-update) leaves P_y and P_z unchanged.

    (D_i A)^T vbar has j-th entry sum_l int A_l(s) d_j S dot vbar_l, and sum_g A_g d_y S_g
    vanishes when A_g does not depend on y (partition of unity along y); the mesh gradient
    of phi has no y or z part either.  This mirrors Eq. (model-Pdot): P_j is conserved
    when the potentials do not depend on x_j.
    """
    st, cfg = _transverse_A_start()
    P0 = st.P.copy()
    for _ in range(3):
        st, info = pic.step(st, cfg)
        assert info["converged"]
    assert np.abs(st.P[:, 1:] - P0[:, 1:]).max() <= 1e-18
    assert np.abs(st.P[:, 0] - P0[:, 0]).max() > 1e-9       # the x momentum does change


def test_planted_transposed_push_breaks_momentum_symmetry(monkeypatch):
    """Pushing with (D A) vbar instead of (D A)^T vbar conserves energy (v.Mv = v.M^T v,
    Eq. (DA-cancellation)) but not the symmetry-direction canonical momentum: the pin above
    must catch it."""
    st, cfg = _transverse_A_start()
    orig = orbit.orbit_gradient
    monkeypatch.setattr(orbit, "orbit_gradient", lambda An, An1, ow: orig(An, An1, ow).transpose(0, 2, 1))
    new, info = pic.step(st, cfg)
    monkeypatch.setattr(orbit, "orbit_gradient", orig)
    assert info["converged"]
    assert np.abs(new.P[:, 1:] - st.P[:, 1:]).max() > 1e-10


def _random_strong_A_start(amp):
    """Random particles with a smooth divergence-free A^n: particles that creep across knots
    make the plain Picard map non-contractive (the orbit average of d_j S in D_i A is very
    sensitive to their own transverse velocity)."""
    st, cfg = _c1_small(per_beam=4, tol=1e-13)
    grid = cfg.grid()
    rng = np.random.default_rng(21)
    F = np.stack([mesh.project_out_null(rng.normal(size=grid.n), grid) for _ in range(3)])
    for _ in range(2):
        F = F + 0.25 * np.stack([mesh.lap(F[c], grid) * min(grid.H) ** 2 for c in range(3)])
    A = mesh.curl(F, grid)
    A *= amp / np.abs(A).max()
    st = pic.replace(st, A=A)
    st = pic.replace(st, P=st.m * st.v + st.q * orbit.point_gather(A, st.xi, grid).T)
    return st, cfg


def test_secant_relaxation_restores_convergence_and_keeps_conservation():
    """§4.8: conservation is a property of the converged discrete equations, not of the solver.
    Plain Picard (Algorithm 1's update) cycles on this state; the oscillation-gated secant
    relaxation converges to tau and the step conserves energy to roundoff."""
    st, cfg = _random_strong_A_start(0.05)
    plain = pic.Config(n=cfg.n, L=cfg.L, dt=cfg.dt, picard_tol=1e-13, picard_max=30, picard_accel=False)
    accel = pic.Config(n=cfg.n, L=cfg.L, dt=cfg.dt, picard_tol=1e-13, picard_max=30, picard_accel=True)
    _, ip = pic.step(st, plain)
    new, ia = pic.step(st, accel)
    assert not ip["converged"]
    assert ia["converged"]
    E0 = sum(pic.energy(st, accel))
    assert abs(ia["R_total"]) <= 1e-14 * E0 and np.abs(ia["RA"]).max() <= 1e-14


def test_relaxation_is_plain_picard_when_contracting():
    st, cfg = _c1_small(per_beam=4)
    plain = pic.Config(n=cfg.n, L=cfg.L, dt=cfg.dt, picard_tol=1e-14, picard_accel=False)
    a, ia = pic.step(st, cfg)
    b, ib = pic.step(st, plain)
    assert ia["iterations"] == ib["iterations"]
    # the gate may still fire on roundoff-level components, so agreement is to roundoff
    assert np.abs(a.v - b.v).max() <= 1e-15 * np.abs(b.v).max()


def test_stopping_on_one_updates_errors_is_accurate_to_tolerance():
    """Algorithm 1 stops once the current and velocity fixed-point errors of one update (v^p to
    v^{p+1}) are below tau; the accepted step then agrees with a step solved far below tau
    to tau's order, and its energy identity holds to roundoff."""
    st, cfg = _c1_small(per_beam=4, tol=1e-13)
    tight = pic.Config(n=cfg.n, L=cfg.L, dt=cfg.dt, picard_tol=1e-16, picard_max=40)
    a, ia = pic.step(st, cfg)
    b, ib = pic.step(st, tight)
    assert ia["converged"] and ib["converged"] and ib["iterations"] > ia["iterations"]
    for name in ("v", "P", "phi", "A"):
        x, y = getattr(a, name), getattr(b, name)
        assert np.linalg.norm(x - y) <= 1e-12 * np.linalg.norm(y), name
    E0 = sum(pic.energy(st, cfg))
    assert abs(ia["R_total"]) <= 1e-14 * E0


@pytest.mark.parametrize("scale", [1e-6, 1e-8, 1e-10])
def test_energy_error_of_an_unconverged_iterate_is_the_residual_product(scale):
    w = pi.WORKLOADS["twostream-8c-8k"]
    x, v, q, m = pi.random_twostream((8, 8, 8), w.L, 4, w.v0, w.eps, 1e-2, 77)
    cfg = pic.Config(n=(8, 8, 8), L=w.L, dt=w.dt, picard_tol=1e-14)
    grid = cfg.grid()
    st = pic.init(x, v, q, m, cfg)
    for _ in range(3):
        st, _ = pic.step(st, cfg)
    conv, _ = pic.step(st, cfg)
    K0, W0 = pic.energy(st, cfg)
    E0 = K0 + W0
    rng = np.random.default_rng(3)
    vstar = conv.v + scale * np.abs(conv.v).max() * rng.normal(size=conv.v.shape)
    it = pic.picard_iteration(st, vstar, cfg, grid)
    K1 = 0.5 * m * np.sum(it["v_new"] ** 2)
    W1 = mesh.field_energy(it["phi"], it["U"], it["A"], cfg.sigma1, cfg.sigma2, grid)
    R = (K1 + W1) - E0
    pred = 0.5 * m * np.sum((it["v_new"] - st.v) * (it["v_new"] - vstar))
    assert abs(pred) > 1e3 * 1e-16 * E0 or scale == 1e-10     # a defect well above roundoff
    assert abs(R - pred) <= 1e-15 * E0, (R / E0, pred / E0)
    # and the identity's content: the defect is second order, |R| <= |dv| |G(v*) - v*| m / 2
    bound = 0.5 * m * np.linalg.norm(it["v_new"] - st.v) * np.linalg.norm(it["v_new"] - vstar)
    assert abs(R) <= bound * (1 + 1e-6) + 1e-15 * E0

