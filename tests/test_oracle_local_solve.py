"""Pins of the oracle's particle-local solve (the accelerated fixed point that §4.8 allows).

The local solve is only a means to a root: §4.8's conservation statements hold for the
converged discrete equations, whatever solver reaches them.  So the pin is the defining
property, not the path: with the iteration's fields fixed, every creeping particle that the
solve does not pin onto a knot must satisfy its own push equation v = G_i(v) to roundoff.

The states are built to make that hard: particles a hair (1e-12 .. 1e-3 cells) from a knot,
drifting towards it by about that distance per step, with an extrapolated first iterate up
to 0.05 cells away, and (second family) beams crossing a strong smooth vector potential, whose
D_i A force jumps at every knot.  There the orbit-averaged force changes steeply just past
the knot (its weight is the fraction of the path beyond it): regula falsi crawls, one
component's large move can leave another component's bracket stale, and within a hair of a
knot that both sides push onto the root is not resolved in double precision, so the
particle must be pinned onto the knot (Filippov sliding) instead.
"""

import numpy as np
import pytest

import pic_inputs as pi
from oracle import mesh, orbit, pic


def _knot_state(seed, far, npart=512):
    n = (8, 8, 8)
    w = pi.WORKLOADS["twostream-8c-8k"]
    cfg = pic.Config(n=n, L=w.L, dt=w.dt, picard_tol=1e-13)
    H = np.asarray(cfg.grid().H)
    rng = np.random.default_rng(seed)
    xi = rng.uniform(0, 8, size=(npart, 3))
    k = rng.integers(0, 8, size=npart).astype(float)
    dk = 10.0 ** rng.uniform(-6, -3, size=npart)
    s = rng.choice([-1.0, 1.0], size=npart)
    xi[:, 1] = np.mod(k - s * dk, 8.0)                     # a hair short of a y knot
    v = rng.normal(scale=0.05, size=(npart, 3))
    v[:, 1] = s * dk * rng.uniform(0.0, 2.0, size=npart) * H[1] / cfg.dt   # drifting onto it
    q = -1.0 / npart
    st = pic.init(xi * H, v, q, abs(q), cfg)
    vprev = st.v.copy()
    vprev[:, 1] -= rng.uniform(-far, far, size=npart) * H[1] / cfg.dt      # a distant first iterate
    return pic.replace(st, vprev=vprev), cfg


@pytest.mark.parametrize("seed,far", [(5, 0.01), (5, 0.05), (6, 0.01), (6, 0.05)])
def test_local_solve_reaches_a_root_for_every_creeping_particle(seed, far):
    st, cfg = _knot_state(seed, far)
    grid = cfg.grid()
    H = np.asarray(grid.H)
    v_it = 2.0 * st.v - st.vprev
    it = pic.picard_iteration(st, v_it, cfg, grid)
    v_next, slide, local = pic.local_solve(st, v_it, it, cfg, grid)
    creeping = pic.creeping(st.xi, cfg.dt * 0.5 * (v_it + st.v) / H, cfg.order)
    assert np.array_equal(local, creeping)
    assert creeping.sum() > 200
    G = pic.push_particles(st.xi, st.v, st.P, v_next, st.q, st.m, st.A, it["A"], it["gphi_half"],
                           it["U_half"], cfg, grid)["v_new"]
    resid = np.where(slide, 0.0, np.abs(G - v_next)).max(axis=1) / np.linalg.norm(v_next, axis=1)
    assert resid[creeping].max() <= 4e-15
    # the others took Algorithm 1's plain update
    assert np.array_equal(v_next[~creeping], it["v_new"][~creeping])


def test_crept_particles_keep_the_local_solve_for_the_step():
    st, cfg = _knot_state(5, 0.01)
    grid = cfg.grid()
    v_it = 2.0 * st.v - st.vprev
    it = pic.picard_iteration(st, v_it, cfg, grid)
    _, _, local = pic.local_solve(st, v_it, it, cfg, grid)
    # a particle solved locally once stays local, even where its iterate no longer creeps
    crept = np.zeros_like(local)
    crept[np.nonzero(~local)[0][:5]] = True
    v_next, _, local2 = pic.local_solve(st, v_it, it, cfg, grid, None, crept)
    assert np.array_equal(local2, local | crept)
    G = pic.push_particles(st.xi, st.v, st.P, v_next, st.q, st.m, st.A, it["A"], it["gphi_half"],
                           it["U_half"], cfg, grid)["v_new"]
    resid = np.abs(G - v_next).max(axis=1) / np.linalg.norm(v_next, axis=1)
    assert resid[crept].max() <= 4e-15


def _strong_A_knot_state(seed, far, amp, npart=512):
    """Beams (|v_x| = 0.2) through a smooth divergence-free A^n of size amp, particles 1e-12 ..
    1e-3 cells short of a y knot and drifting onto it."""
    n = (8, 8, 8)
    w = pi.WORKLOADS["twostream-8c-8k"]
    cfg = pic.Config(n=n, L=w.L, dt=w.dt, picard_tol=1e-13)
    grid = cfg.grid()
    H = np.asarray(grid.H)
    rng = np.random.default_rng(seed)
    xi = rng.uniform(0, 8, size=(npart, 3))
    k = rng.integers(0, 8, size=npart).astype(float)
    dk = 10.0 ** rng.uniform(-12, -3, size=npart)
    s = rng.choice([-1.0, 1.0], size=npart)
    xi[:, 1] = np.mod(k - s * dk, 8.0)
    v = rng.normal(scale=0.01, size=(npart, 3))
    v[:, 0] += 0.2 * rng.choice([-1.0, 1.0], size=npart)
    v[:, 1] = s * dk * rng.uniform(0.0, 2.0, size=npart) * H[1] / cfg.dt
    q = -1.0 / npart
    st = pic.init(xi * H, v, q, abs(q), cfg)
    F = np.stack([mesh.project_out_null(rng.normal(size=grid.n), grid) for _ in range(3)])
    for _ in range(2):
        F = F + 0.25 * np.stack([mesh.lap(F[c], grid) * min(grid.H) ** 2 for c in range(3)])
    A = mesh.curl(F, grid)
    A *= amp / np.abs(A).max()
    st = pic.replace(st, A=A, P=st.m * st.v + st.q * orbit.point_gather(A, st.xi, grid).T)
    vprev = st.v.copy()
    vprev[:, 1] -= rng.uniform(-far, far, size=npart) * H[1] / cfg.dt
    return pic.replace(st, vprev=vprev), cfg


@pytest.mark.parametrize("seed,far,amp", [(5, 0.01, 0.05), (6, 0.05, 0.05), (5, 0.05, 0.01), (6, 0.01, 0.2)])
def test_local_solve_near_knots_in_a_strong_vector_potential(seed, far, amp):
    """Every creeping particle is a root of its own equation to roundoff or pinned onto its
    knot, up to the strongest potential (0.2, steep and strongly coupled).  The bound is the
    rounding of one push evaluation: |G(u) - u| of a root is at most a few ulps of the speed
    (the largest measured is 3.3e-16 at amp = 0.2)."""
    bound = 4e-15
    st, cfg = _strong_A_knot_state(seed, far, amp)
    grid = cfg.grid()
    v_it = 2.0 * st.v - st.vprev
    it = pic.picard_iteration(st, v_it, cfg, grid)
    v_next, slide, local = pic.local_solve(st, v_it, it, cfg, grid)
    G = pic.push_particles(st.xi, st.v, st.P, v_next, st.q, st.m, st.A, it["A"], it["gphi_half"],
                           it["U_half"], cfg, grid)["v_new"]
    resid = np.where(slide, 0.0, np.abs(G - v_next)).max(axis=1) / np.linalg.norm(v_next, axis=1)
    assert local.sum() > 300 and slide.any(axis=1).sum() >= 3
    assert resid[local].max() <= bound
    # pinned components land exactly on a knot a hair from the start
    H = np.asarray(grid.H)
    beta = cfg.dt * 0.5 * (v_next + st.v) / H
    end = st.xi + beta
    assert np.all(np.abs(end[slide] - np.rint(end[slide])) <= 1e-9)
    assert np.all(np.abs(beta[slide]) < pic.D_KNOT)


@pytest.mark.parametrize("seed,far,amp", [(5, 0.01, 0.05), (6, 0.05, 0.05), (7, 0.01, 0.01), (5, 0.05, 0.2)])
def test_step_near_knots_conserves_energy(seed, far, amp):
    """The whole step on those states: pinned components cost energy in proportion to their
    vbar_a = d H / dt, so pinning is kept to d < D_KNOT (1e-11); every other creeping particle
    is solved to its root, and the Theorem's R_total stays at roundoff."""
    st, cfg = _strong_A_knot_state(seed, far, amp)
    new, info = pic.step(st, cfg)
    assert info["converged"]
    E0 = sum(pic.energy(st, cfg))
    assert abs(info["R_total"]) <= 1e-14 * E0


def test_failed_solves_slide_within_the_fallback_band(monkeypatch):
    """The fallback rule on its own: a local solve that fails (its best residual stays above
    FAIL_RES of the speed; here forced by allowing only 3 evaluations) slides every component
    that starts within D_FALLBACK of a knot (here 1e-9 .. 1e-7 cells, outside the D_KNOT band of
    the sliding probes) onto that knot, and only those.  A sliding component lands exactly on
    its knot, and its energy defect is its work m vbar_a (v_a - G_a) with vbar_a = d H_a / dt, so
    the step's |R_total| is at most sum over sliding components of m |d| H_a / dt (|v_a| + |G_a|),
    an a-priori bound that is tiny beside the energy, and not the whole velocity times the
    failed residual."""
    monkeypatch.setattr(pic, "LOCAL_STEPS", 3)
    st, cfg = _strong_A_knot_state(5, 0.05, 0.05)
    grid = cfg.grid()
    H = np.asarray(grid.H)
    rng = np.random.default_rng(1)
    xi = st.xi.copy()
    k = np.round(xi[:, 1])
    s = np.where(xi[:, 1] >= k, 1.0, -1.0)
    xi[:, 1] = np.mod(k + s * 10.0 ** rng.uniform(-9, -7, size=xi.shape[0]), 8.0)
    st = pic.replace(st, xi=xi, P=st.m * st.v + st.q * orbit.point_gather(st.A, xi, grid).T)
    v_it = 2.0 * st.v - st.vprev
    it = pic.picard_iteration(st, v_it, cfg, grid)
    v_next, slide, local = pic.local_solve(st, v_it, it, cfg, grid)
    G = pic.push_particles(st.xi, st.v, st.P, v_next, st.q, st.m, st.A, it["A"], it["gphi_half"],
                           it["U_half"], cfg, grid)["v_new"]
    d = np.round(xi - orbit.knot_offset(1)) - (xi - orbit.knot_offset(1))
    speed = np.linalg.norm(v_next, axis=1)
    failed = np.abs(G - v_next).max(axis=1) > pic.FAIL_RES * speed
    near = (np.abs(d) < pic.D_FALLBACK) & (np.abs(d) >= pic.D_KNOT)
    assert local.sum() > 300 and failed[local].mean() > 0.5
    # exactly the near-knot components of the failed (or landing-stuck) solves slide
    assert np.array_equal(slide[local & failed], near[local & failed])
    assert not slide[~local].any()
    beta = cfg.dt * 0.5 * (v_next + st.v) / H
    end = st.xi + beta
    assert np.all(np.abs(end[slide] - np.rint(end[slide])) <= 1e-12)
    # the whole step: converged, and the energy defect within the a-priori bound
    new, info = pic.step(st, cfg)
    assert info["converged"]
    E0 = sum(pic.energy(st, cfg))
    vmax = max(np.abs(st.v).max(), np.abs(new.v).max())
    bound = sum(st.m * np.abs(d[:, a][near[:, a]]).sum() * H[a] / cfg.dt * 2.0 * vmax for a in range(3))
    assert abs(info["R_total"]) <= bound + 1e-14 * E0
    assert bound <= 1e-5 * E0
