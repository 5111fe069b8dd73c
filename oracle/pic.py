"""One time step of the orbit-discrete-gradient CN potential PIC method (test infrastructure only).

Follows Algorithm 1 ("Picard iteration for the orbit-discrete-gradient CN potential PIC
step") in the paper's order, with the orbit push of §4.4 (Eq. (orbit-push)), the
initial data of §5.4 and the diagnostics of §5.1-§5.3.

Readings of points the paper leaves open (each is listed in the design notes):

* History velocity at the first step: v^{-1} := v^0, so the first guess is v^0.
* Picard norms: e_v = ||v^{n+1,p+1} - v^{n+1,p}||_2 / ||v^{n+1,p+1}||_2 over all
  particles and components, v^{n+1,p+1} being the next iterate (G(v^{n+1,p}) itself for
  plain Picard); e_J = ||J(v^{n+1,p+1}) - J(v^{n+1,p})||_2 / (||J(v^{n+1,p+1})||_2 +
  J_scale), the change of the orbit current made by the same update, with
  J_scale = sqrt(N_cells) * sum_i |q_i| |v_i^n| / |Omega| (a floor, because the
  paired beams start with J ~ 0, §5.4).  Converged when both are <= tau; the current
  of v^{n+1,p+1} is the one the final sweep then uses.
* Final consistency sweep (§5.4): after convergence at iterate p, one more iteration
  is run from v^{n+1,p+1}; its current, fields, orbit integrals and particle state
  are the accepted step and feed the diagnostics.
* Not converged after p = 0..p_max: the step is reported as not converged (the
  caller keeps the old state).
* Accelerated fixed point (§4.8 states that conservation holds for any converged
  solver, accelerated fixed-point methods included).  A particle whose orbit crosses a
  knot on an axis where it moves very little (|beta_a| < 0.1 cells, "creeping") has a
  step force that is very sensitive to its own velocity: the orbit average of d_j S in
  D_i A changes with the fraction of the path beyond the knot.  The particle-local
  feedback can exceed 1, and plain Picard then stalls or cycles on it (also when an
  iterate flips between crossing and just missing the knot).  With
  ``picard_accel`` each iteration therefore solves, for the creeping particles only, the
  particle's own equation v = G_i(v) with the iteration's fields held fixed (per component:
  secant steps while they converge, else growing steps along g until the root is bracketed,
  then bracketed steps that respect the knots; at most LOCAL_STEPS evaluations; the best
  evaluation is kept; see local_solve).  A particle that barely crosses a knot can have no
  root near its iterate (the two sides of the crossing threshold push the same way);
  g = G - u is continuous and G bounded, so a root lies in the direction of g.  A particle
  that starts on or a hair from a knot that both sides push it onto has no root that
  double precision resolves (G changes by the full jump of d_a S within the hair); it then
  lands exactly on the knot and slides along it (Filippov solution), which keeps the energy
  identities to the size of its tiny vbar_a.  So does a particle whose iterate change has
  stopped shrinking faster than SLOW_RATIO per iteration (see slow_particles).  A particle
  solved locally once keeps the local solve for the rest of the step.  Every other
  particle takes Algorithm 1's update v^{p+1} = G(v^p).  The outer loop then contracts at
  the rate of the weak particle-field coupling.  With ``picard_accel=False`` every particle
  takes the plain update.
* Initial charge: rho_g = sum_i q_i S_g(x_i) / dV plus the ion background, with the
  null modes of Delta_h (the mean and the checkerboards) removed; Poisson's 1/eps0 is
  read as sigma1.
"""

from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from . import mesh, orbit

CHUNK = 32768
BETA_CREEP = 0.1      # cells: "creeping" knot crossings get a particle-local solve
D_KNOT = 1e-11        # cells: starting this close to a knot counts as creeping and is probed
                      # for sliding (about the rounding of a position landed on a knot, with
                      # margin: farther out the knot-piece step resolves the root)
SLIDE_PROBE = 1e-12   # cells: the sliding test probes SLIDE_PROBE short of landing on the knot
SLIDE_FAR = 64.0      # ... and max(SLIDE_PROBE, SLIDE_FAR |d|) past it (98% of that path beyond)
D_FALLBACK = 1e-6     # cells: a failed solve slides the components that start this near a knot
FAIL_RES = 1e-10      # failed: the best residual is above FAIL_RES x the particle's speed
BETA_TRIAL = 1.0      # cells: trial orbits stay within this beyond the iterate's own, per axis
LOCAL_STEPS = 32      # at most this many extra push evaluations per creeping particle
LOCAL_TOL = 1e-15     # local residual target, relative to the particle's speed
OMEGA_MAX = 8.0       # bound on the secant step factor
SLOW_RATIO = 0.25     # a plain particle whose change did not shrink below SLOW_RATIO of the
SLOW_FLOOR = 1e-12   # previous one (and exceeds SLOW_FLOOR x its speed) is solved locally


@dataclass
class Config:
    n: tuple
    L: tuple
    dt: float
    kappa: float = 1.0
    sigma1: float = 1.0
    sigma2: float = 1.0
    picard_tol: float = 1e-14
    picard_max: int = 16
    split: bool = True
    picard_accel: bool = True    # particle-local solves for creeping and slow particles (see step())
    quadrature: str = "closed"   # "closed" (Appendices A/B) or "gauss" (§4.7 split Gauss rule)
    nq: int = 16
    n0: float = 1.0              # ion background density (§5.4)
    order: int = 1               # B-spline degree r (1, 2, 3); r > 1 needs quadrature "gauss"
    ops: str = "central2"        # spatial operators: "central2" or "spectral" (§3.3)

    def grid(self):
        return mesh.Grid(self.n, self.L, self.ops)


@dataclass
class State:
    xi: np.ndarray      # (np, 3) position in cell units, wrapped to [0, n)
    v: np.ndarray       # (np, 3) v^n
    P: np.ndarray       # (np, 3) canonical momentum P^n
    vprev: np.ndarray   # (np, 3) history velocity v^{n-1}
    q: float
    m: float
    phi: np.ndarray
    psi: np.ndarray
    A: np.ndarray       # (3, nx, ny, nz)
    U: np.ndarray
    rho: np.ndarray
    extra: dict = field(default_factory=dict)


def wrap_cells(xi, n):
    """Wrap cell-unit positions onto [0, n_a) per axis."""
    nn = np.asarray(n, dtype=np.float64)
    w = xi - nn * np.floor(xi / nn)
    return np.where(w >= nn, w - nn, w)


def orbit_weights(xi0, beta, cfg, grid, with_gradient=True):
    if cfg.quadrature == "closed":
        if cfg.order != 1:
            raise ValueError("the closed forms of Appendices A/B are for linear splines (order 1)")
        return orbit.closed_form_weights(xi0, beta, grid, cfg.split, with_gradient)
    if cfg.quadrature == "gauss":
        return orbit.gauss_weights(xi0, beta, grid, cfg.nq, cfg.split, cfg.order)
    raise ValueError(cfg.quadrature)


def _chunks(npart):
    for a in range(0, npart, CHUNK):
        yield slice(a, min(a + CHUNK, npart))


# --- Initial data (§5.4) ---------------------------------------------------------------

def point_deposit(xi, q, grid, order=1):
    """rho_e,g = sum_i q S_g(x_i) / dV (Eq. (source-moments), with the 1/dV of Eq. (orbit-current))."""
    rho = np.zeros(grid.n)
    for sl in _chunks(xi.shape[0]):
        nodes, S, _ = orbit.point_shape(xi[sl], grid, order)
        rho += np.bincount(orbit.flat_index(nodes, grid.n).ravel(), weights=(q * S).ravel() / grid.dV,
                           minlength=grid.ncell).reshape(grid.n)
    return rho


def init(x, v, q, m, cfg):
    """Initial state from particle positions x (physical units) and velocities v (§5.4)."""
    grid = cfg.grid()
    H = np.asarray(grid.H)
    xi = wrap_cells(np.asarray(x, dtype=np.float64) / H, grid.n)
    v = np.array(v, dtype=np.float64)
    rho_e = point_deposit(xi, q, grid, cfg.order)
    rho = rho_e + cfg.n0
    rho = rho - np.mean(rho)
    rho = mesh.project_out_null(rho, grid)
    phi = mesh.poisson(rho, cfg.sigma1, grid)
    A = np.zeros((3,) + grid.n)
    P = m * v + q * orbit.point_gather(A, xi, grid, cfg.order).T
    return State(xi=xi, v=v, P=P, vprev=v.copy(), q=float(q), m=float(m), phi=phi,
                 psi=np.zeros(grid.n), A=A, U=np.zeros((3,) + grid.n), rho=rho)


# --- Algorithm 1 ---------------------------------------------------------------------

def orbit_current(st, v_it, cfg, grid):
    """The orbit current of the iterate v_it (Eq. (orbit-current)), split-path weights."""
    H = np.asarray(grid.H)
    vbar = 0.5 * (v_it + st.v)                       # orbit implied by the iterate
    beta = cfg.dt * vbar / H                         # unwrapped displacement in cell units
    J = np.zeros((3,) + grid.n)
    for sl in _chunks(st.xi.shape[0]):
        ow = orbit_weights(st.xi[sl], beta[sl], cfg, grid, with_gradient=False)
        J += orbit.deposit(st.q * vbar[sl], ow, grid)
    return J


def picard_iteration(st, v_it, cfg, grid, diagnostics=False, slide=None, J=None):
    """One pass of the Algorithm 1 loop body for the end-of-step velocity iterate ``v_it``
    (``J``: its orbit current, when already computed)."""
    dt = cfg.dt
    vbar = 0.5 * (v_it + st.v)                       # orbit implied by the iterate
    if J is None:
        J = orbit_current(st, v_it, cfg, grid)
    # continuity (Eq. (cn-continuity)) and CN potential solve (Eq. (cn-field-update))
    rho1 = mesh.continuity(st.rho, J, dt, grid)
    rho_half = 0.5 * (rho1 + st.rho)
    phi1, psi1, A1, U1 = mesh.cn_fields(st.phi, st.psi, st.A, st.U, rho_half, J, dt,
                                        cfg.kappa, cfg.sigma1, cfg.sigma2, grid)
    # midpoint mesh fields
    gphi_half = mesh.grad(0.5 * (phi1 + st.phi), grid)
    U_half = 0.5 * (U1 + st.U)
    pushed = push_particles(st.xi, st.v, st.P, v_it, st.q, st.m, st.A, A1, gphi_half, U_half, cfg, grid,
                            diagnostics, slide)
    P1, xi1, v_new = pushed["P"], pushed["xi"], pushed["v_new"]
    diag = pushed.get("diag")
    out = dict(J=J, rho=rho1, phi=phi1, psi=psi1, A=A1, U=U1, P=P1, xi=xi1, v_new=v_new, vbar=vbar,
               gphi_half=gphi_half, U_half=U_half)
    if diagnostics:
        E_half = -gphi_half - U_half
        diag["mwork"] = float(np.sum(J * E_half) * grid.dV)               # sum_g J . E dV
        out["diag"] = diag
    return out


def push_particles(xi, v, P, v_it, q, m, A0, A1, gphi_half, U_half, cfg, grid, diagnostics=False, slide=None):
    """Orbit gather and canonical-momentum push of Algorithm 1 for the given particles.

    Uses the midpoint mesh fields of the current iterate: grad_h phi^{n+1/2} (3, n...),
    A^n and A^{n+1} for the orbit-discrete gradient, and U^{n+1/2} (diagnostics only).
    ``slide`` (np, 3) marks components sliding onto a knot (see local_solve): there the
    orbit lands on the knot, v^{n+1}_a is the iterate itself and P_a = m v_a + q A_h,a(x^{n+1}).
    """
    H = np.asarray(grid.H)
    dt = cfg.dt
    vbar = 0.5 * (v_it + v)
    beta = dt * vbar / H
    npart = xi.shape[0]
    P1 = np.empty((npart, 3))
    xi1 = np.empty((npart, 3))
    v_new = np.empty((npart, 3))
    diag = {"RA": np.empty((npart, 3)), "pu": np.empty(npart), "pwork": 0.0} if diagnostics else None
    for sl in _chunks(npart):
        ow = orbit_weights(xi[sl], beta[sl], cfg, grid)
        gphibar = orbit.gather(gphi_half, ow).T                     # (np, 3)  Eq. (gphibar-definition)
        DA = orbit.orbit_gradient(A0, A1, ow)                       # (np, l, j)  Eq. (DA-def)
        DAT_vbar = np.einsum("ilj,il->ij", DA, vbar[sl])            # ((D A)^T vbar)_j
        P1[sl] = P[sl] + dt * (-q * gphibar + q * DAT_vbar)          # Eq. (orbit-P-update)
        xend = xi[sl] + beta[sl]                                     # Eq. (orbit-x-update), unwrapped
        xi1[sl] = wrap_cells(xend, grid.n)
        A_end = orbit.point_gather(A1, xi1[sl], grid, cfg.order).T   # A_h^{n+1}(x^{n+1})
        v_new[sl] = (P1[sl] - q * A_end) / m                         # Eq. (orbit-v-update)
        if slide is not None:
            sv = slide[sl]
            v_new[sl] = np.where(sv, v_it[sl], v_new[sl])
            P1[sl] = np.where(sv, m * v_new[sl] + q * A_end, P1[sl])
        if diagnostics:
            Ubar = orbit.gather(U_half, ow).T                        # Eq. (Ubar-def)
            A_start = orbit.point_gather(A0, xi[sl], grid, cfg.order).T
            DA_vbar = np.einsum("ilj,ij->il", DA, vbar[sl])          # (D A) vbar
            diag["RA"][sl] = A_end - A_start - dt * (Ubar + DA_vbar)     # Eq. (RA-test)
            diag["pu"][sl] = np.sum(ow.w, axis=1) - 1.0                  # Appendix A partition of unity
            Ebar = -gphibar - Ubar                                       # Eq. (orbit-E-gather)
            diag["pwork"] += float(np.sum(q * vbar[sl] * Ebar))
    out = {"P": P1, "xi": xi1, "v_new": v_new}
    if diagnostics:
        out["diag"] = diag
    return out


def creeping(xi, beta, order=1):
    """Particles that, on an axis with |beta_a| < BETA_CREEP (cells), get within 2 |beta_a| of
    the next knot ahead (d in (0, 1]) or start within D_KNOT of any knot: the orbits that
    cross a knot while barely moving, those that nearly do, and those hovering on a knot (an
    iterate can flip between crossing and not crossing).  Knots of the degree-r spline."""
    xi = xi - orbit.knot_offset(order)
    f = np.zeros(xi.shape[0], dtype=bool)
    for a in range(3):
        x, b = xi[:, a], beta[:, a]
        d = np.where(b > 0, np.floor(x) + 1.0 - x, x - (np.ceil(x) - 1.0))
        near = np.minimum(x - np.floor(x), np.ceil(x) - x)
        f |= (np.abs(b) < BETA_CREEP) & (((b != 0) & (d < 2.0 * np.abs(b))) | (near < D_KNOT))
    return f


def local_solve(st, v_it, it, cfg, grid, pinned=None, crept=None):
    """Next iterate: G(v^p) for most particles; for the creeping ones a root of
    g(u) = G_i(u) - u with this iteration's fields fixed, per component.

    * Sliding.  For a component starting within D_KNOT of a knot (signed distance d), g is
      probed SLIDE_PROBE short of landing on that knot and max(SLIDE_PROBE, SLIDE_FAR |d|)
      past it, where the path beyond the knot carries most of the orbit average.  If both
      sides push onto the knot, the root lies within that hair of the knot, where G changes
      by the full jump of the orbit-averaged d_a S: double precision does not resolve it.
      The component then lands exactly on the knot (beta_a = d, the Filippov sliding
      solution) and the push completes it with v^{n+1}_a = u_a and P_a from the canonical
      relation.  The energy identities are kept to the size of the a-component work and
      a-column of D_i A, both multiplied by vbar_a = d H_a / dt < D_KNOT H_a / dt.
    * Otherwise: secant steps (factor clamped to [-OMEGA_MAX, OMEGA_MAX]) while each one at
      least halves |g|, so a nearby root is found first; else steps u + f g along g with
      f = 2, 4, 8, ... (g is continuous there and G bounded, so g changes sign that way);
      inside a bracket, the new point replaces the end of the same sign:
      - a bracket whose interior holds the velocity that lands the orbit exactly on a knot
        is first split there: the force weight of the path beyond a knot makes G steep just
        past it, so g is smooth only between such landings;
      - inside one knot-free piece past a crossing (landing beta_L), G in cells is close to
        A + B beta_L / beta: steep near the knot, flat far past it.  The step solves
        beta = A + B beta_L / beta exactly for the line through the two ends (a quadratic
        in beta, its root inside the bracket); elsewhere it is the regula falsi point;
      - the components share each evaluation, so one component's sign change can come from
        another component's move, and regula falsi can stagnate: a bracket whose same end
        is replaced twice running is released and followed by a secant step.
      At most LOCAL_STEPS evaluations, ending once one of them has every component's |g|
      within LOCAL_TOL of the particle's speed; the evaluation with the smallest
      largest-component |g| is kept (the components are coupled, so a mix of components
      from different evaluations is no root).

    ``pinned`` (np, 3): components found sliding earlier in this step; they stay pinned, so
    that the outer iteration cannot cycle between pinned and free.  ``crept`` (np,): the
    particles solved locally earlier in this step; they keep the local solve for the rest of
    the step, so that no particle alternates between the local and the plain update.
    Returns (v_next, slide mask, crept mask)."""
    H = np.asarray(grid.H)
    G = it["v_new"]
    v_next = G.copy()
    slide = np.zeros(G.shape, dtype=bool)
    beta = cfg.dt * 0.5 * (v_it + st.v) / H
    local = creeping(st.xi, beta, cfg.order)
    if crept is not None:
        local = local | crept
    idx = np.nonzero(local)[0]
    if idx.size == 0:
        return v_next, slide, local

    def Gf(u):
        return push_particles(st.xi[idx], st.v[idx], st.P[idx], u, st.q, st.m, st.A, it["A"], it["gphi_half"],
                              it["U_half"], cfg, grid)["v_new"]

    x0 = st.xi[idx]
    vn = st.v[idx]
    u0, r0 = v_it[idx], G[idx] - v_it[idx]
    u1 = G[idx]
    # sliding probes, one axis at a time on the base vector u1
    koff = orbit.knot_offset(cfg.order)
    d_knot = np.round(x0 - koff) - (x0 - koff)
    near = np.abs(d_knot) < D_KNOT
    u_land = 2.0 * d_knot * H / cfg.dt - vn
    sl = np.zeros(u1.shape, dtype=bool) if pinned is None else pinned[idx].copy()
    for a in range(3):
        cand = near[:, a] & ~sl[:, a]
        if not np.any(cand):
            continue
        d = d_knot[:, a]
        far = np.maximum(SLIDE_PROBE, SLIDE_FAR * np.abs(d))
        um, up = u1.copy(), u1.copy()
        um[:, a] = 2.0 * (d - np.where(d > 0, SLIDE_PROBE, far)) * H[a] / cfg.dt - vn[:, a]
        up[:, a] = 2.0 * (d + np.where(d > 0, far, SLIDE_PROBE)) * H[a] / cfg.dt - vn[:, a]
        gm = Gf(um)[:, a] - um[:, a]
        gp = Gf(up)[:, a] - up[:, a]
        sl[:, a] |= cand & (gm > 0) & (gp < 0)
    u1 = np.where(sl, u_land, u1)
    r1 = Gf(u1) - u1
    r0 = np.where(sl, 0.0, r0)
    r1 = np.where(sl, 0.0, r1)
    speed = np.maximum(np.linalg.norm(u0, axis=1), 1e-300)
    tol = LOCAL_TOL * speed
    # the best evaluation so far: the smallest largest-component |g| (all components of one
    # evaluation, since they are coupled; pinned components land on their knot)
    m0, m1 = np.abs(r0).max(axis=1), np.abs(r1).max(axis=1)
    best_u = np.where(sl, u_land, np.where((m1 < m0)[:, None], u1, u0))
    best_r = np.minimum(m0, m1)
    br = ~sl & (r0 * r1 < 0)                          # bracketed components
    ua, ga, ub, gb = u0.copy(), r0.copy(), u1.copy(), r1.copy()
    side = np.zeros_like(u0)
    secant_ok = np.abs(r1) <= 0.5 * np.abs(r0)        # the plain step at least halved |g|
    fac = np.full_like(u0, 2.0)
    rep = np.zeros(u0.shape, dtype=np.int64)          # consecutive replacements of one end
    c = cfg.dt * 0.5 / H                              # beta = c (u + v^n): orbit length in cells
    xk = x0 - koff                                    # start on the knot lattice
    blim = np.abs(c * (u0 + vn)) + BETA_TRIAL         # bound on the trial orbits, per axis
    for _ in range(LOCAL_STEPS - 1):
        if np.all(best_r <= tol):
            break
        with np.errstate(divide="ignore", invalid="ignore"):
            sec = -(u1 - u0) / (r1 - r0)
            fp = ub - gb * (ub - ua) / (gb - ga)
            # Both ends past the same last knot (landing beta_L): on that knot-free piece the
            # image G, in cells, is close to A + B w with w = beta_L / beta (the path beyond
            # the knot weights the force there), steep near the knot and flat far past it.
            # The step solves beta = A + B w exactly for the line through the two ends:
            # D beta^2 - c1 beta - e = 0, its root inside the bracket.
            ba, bb = c * (ua + vn), c * (ub + vn)
            la = np.where(ba > 0, np.floor(xk + ba) - xk, np.ceil(xk + ba) - xk)
            lb = np.where(bb > 0, np.floor(xk + bb) - xk, np.ceil(xk + bb) - xk)
            Ga, Gb = c * ga + ba, c * gb + bb
            wa, wb = la / ba, la / bb
            D = wb - wa
            c1 = Ga * D - (Gb - Ga) * wa
            e = (Gb - Ga) * la
            qq = 0.5 * (c1 + np.copysign(np.sqrt(np.maximum(c1 * c1 + 4.0 * D * e, 0.0)), c1))
            x1, x2 = qq / D, -e / qq
            blo, bhi = np.minimum(ba, bb), np.maximum(ba, bb)
            in1, in2 = (x1 > blo) & (x1 < bhi), (x2 > blo) & (x2 < bhi)
            bstar = np.where(in1, x1, x2)
            fpm = 2.0 * bstar * H / cfg.dt - vn
            piece = ((la == lb) & (la != 0.0) & (la * ba > 0) & (la * bb > 0) & (c1 * c1 + 4.0 * D * e >= 0.0)
                     & (in1 | in2) & np.isfinite(fpm))
        fp = np.where(piece, fpm, fp)
        sec = np.where(np.isfinite(sec), np.clip(sec, -OMEGA_MAX, OMEGA_MAX), 1.0)
        expand = ~br & ~secant_ok
        # the knot landing strictly inside the bracket (the highest one, if several)
        lo, hi = np.minimum(ua, ub), np.maximum(ua, ub)
        b_lo, b_hi = c * (lo + vn), c * (hi + vn)
        b_land = (np.ceil(xk + b_hi) - 1.0) - xk
        u_split = 2.0 * b_land * H / cfg.dt - vn
        split = br & (b_land > b_lo) & (u_split > lo) & (u_split < hi)
        u2 = np.where(br & np.isfinite(fp), fp, np.where(expand, u1 + fac * r1, u1 + sec * r1))
        u2 = np.where(split, u_split, u2)
        u2 = np.where(sl, u_land, u2)
        # trial orbits stay within BETA_TRIAL cells beyond the iterate's own orbit, per axis
        # (the growing steps along g would otherwise run past any neighbourhood of the root)
        u2 = np.clip(u2, -blim / c - vn, blim / c - vn)
        fac = np.where(expand, 2.0 * fac, fac)
        r2 = np.where(sl, 0.0, Gf(u2) - u2)
        m2 = np.abs(r2).max(axis=1)
        better = m2 < best_r
        best_u = np.where(better[:, None], u2, best_u)
        best_r = np.where(better, m2, best_r)
        secant_ok = secant_ok & (np.abs(r2) <= 0.5 * np.abs(r1))
        # bracket bookkeeping: the new point replaces the end whose g has its sign
        same_b = br & (r2 * gb > 0)
        same_a = br & ~same_b
        side_before = side
        ub, gb = np.where(same_b, u2, ub), np.where(same_b, r2, gb)
        ua, ga = np.where(same_a, u2, ua), np.where(same_a, r2, ga)
        side = np.where(same_b, 1.0, np.where(same_a, -1.0, side))
        new_br = ~sl & ~br & (r2 * r1 < 0)
        ua, ga = np.where(new_br, u1, ua), np.where(new_br, r1, ga)
        ub, gb = np.where(new_br, u2, ub), np.where(new_br, r2, gb)
        br = br | new_br
        # the same end replaced twice running: the kept end is stale (its g was taken before
        # the other components moved: they share each evaluation) or regula falsi stagnates;
        # the bracket is released and the next step is a secant one from two fresh points
        rep = np.where((same_b & (side_before > 0)) | (same_a & (side_before < 0)), rep + 1,
                       np.where(same_a | same_b, 1, rep))
        release = br & (rep >= 2)
        br = br & ~release
        secant_ok = secant_ok | release
        rep = np.where(release, 0, rep)
        side = np.where(release, 0.0, side)
        u0, r0, u1, r1 = u1, r1, u2, r2
    # A solve that ends above the tolerance on the landing of its nearest knot, or that fails
    # (best residual above FAIL_RES of the speed) with a component starting within D_FALLBACK
    # of a knot: that root lies in the hair past the knot that double precision (or the steps)
    # did not resolve, and the component slides onto the knot.  Its energy defect is then
    # bounded by vbar_a = d H / dt times its residual, where it would otherwise be the whole
    # velocity times that residual; below FAIL_RES the residual itself costs less.
    failed = best_r > FAIL_RES * speed
    sl = sl | ((best_r > tol)[:, None] & (best_u == u_land)) | (failed[:, None] & (np.abs(d_knot) < D_FALLBACK))
    best_u = np.where(sl, u_land, best_u)
    v_next[idx] = best_u
    if pinned is not None:
        slide |= pinned
    slide[idx] = sl
    return v_next, slide, local


def slow_particles(v_it, v_prev, G):
    """The plain-update particles whose iterate change did not shrink below SLOW_RATIO of the
    previous one (max-norm over components, above SLOW_FLOOR of the particle's speed): their
    own feedback is too strong for the outer iteration, as for orbits that cross a knot just
    past their creeping range once the force jumps at knots grow.  They take the local solve
    from then on.  A contracting outer loop (field-driven changes) shrinks every change far
    faster than SLOW_RATIO, so it flags almost none."""
    dnew = np.abs(G - v_it).max(axis=1)
    dold = np.abs(v_it - v_prev).max(axis=1)
    return (dnew > SLOW_RATIO * dold) & (dnew > SLOW_FLOOR * np.linalg.norm(v_it, axis=1))


def j_scale(st, grid):
    return np.sqrt(grid.ncell) * abs(st.q) * np.sum(np.linalg.norm(st.v, axis=1)) / grid.volume


def step(st, cfg):
    """Advance one time step (Algorithm 1 plus the final consistency sweep of §5.4).

    Returns (new_state, info).  ``info['converged']`` is False when p_max was reached;
    the caller then keeps ``st``.
    """
    grid = cfg.grid()
    v_it = 2.0 * st.v - st.vprev                     # extrapolated initial iterate
    J_it = None                                      # orbit current of v_it, once known
    jsc = j_scale(st, grid)
    hist = []
    converged = False
    slide = None
    crept = None
    v_prev = None
    for p in range(cfg.picard_max + 1):
        it = picard_iteration(st, v_it, cfg, grid, J=J_it)
        if cfg.picard_accel:
            if v_prev is not None:
                slow = slow_particles(v_it, v_prev, it["v_new"])
                crept = slow if crept is None else crept | slow
            v_next, slide, crept = local_solve(st, v_it, it, cfg, grid, slide, crept)
        else:
            v_next, slide = it["v_new"], None
        vnorm = np.linalg.norm(v_next)
        e_v = np.linalg.norm(v_next - v_it) / vnorm if vnorm > 0 else 0.0   # no particles: no error
        # the current fixed-point error of the same update v^p -> v^{p+1}: the orbit current of
        # the new iterate (the one the next iteration, or the final sweep, uses) against J^p
        J_next = orbit_current(st, v_next, cfg, grid)
        num, den = np.linalg.norm(J_next - it["J"]), np.linalg.norm(J_next) + jsc
        e_J = num / den if den > 0 else (np.inf if num > 0 else 0.0)       # no current at all: no error
        hist.append((float(e_v), float(e_J)))
        if e_v <= cfg.picard_tol and e_J <= cfg.picard_tol:
            converged = True
            break
        v_prev = v_it
        v_it = v_next
        J_it = J_next
    info = {"converged": converged, "iterations": len(hist), "errors": hist}
    if not converged:
        return st, info
    fin = picard_iteration(st, v_next, cfg, grid, diagnostics=True, slide=slide)
    new = State(xi=fin["xi"], v=fin["v_new"], P=fin["P"], vprev=st.v.copy(), q=st.q, m=st.m,
                phi=fin["phi"], psi=fin["psi"], A=fin["A"], U=fin["U"], rho=fin["rho"])
    K0, W0 = energy(st, cfg)
    K1, W1 = energy(new, cfg)
    d = fin["diag"]
    info.update(
        K0=K0, W0=W0, K1=K1, W1=W1,
        mesh_work=d["mwork"], particle_work=d["pwork"],
        R_field=W1 - W0 + cfg.dt * d["mwork"],                  # Eq. (R-field)
        R_particle=K1 - K0 - cfg.dt * d["pwork"],               # Eq. (R-particle)
        R_total=(K1 + W1) - (K0 + W0),                          # Eq. (R-total)
        RA=d["RA"], partition_of_unity=d["pu"],
        continuity=new.rho - st.rho + cfg.dt * mesh.div(fin["J"], grid),
        J=fin["J"], vbar=fin["vbar"],
    )
    return new, info


# --- Energies and mesh diagnostics (§4.1, §5.1) ----------------------------------------

def kinetic_energy(st):
    """K = sum_i m_i |v_i|^2 / 2 (Eq. (particle-energy))."""
    return float(0.5 * st.m * np.sum(st.v * st.v))


def energy(st, cfg):
    grid = cfg.grid()
    return kinetic_energy(st), mesh.field_energy(st.phi, st.U, st.A, cfg.sigma1, cfg.sigma2, grid)


def mesh_diagnostics(st, cfg):
    grid = cfg.grid()
    return {
        "gauge": mesh.gauge_residual(st.psi, st.A, cfg.kappa, grid),
        "gauss": mesh.gauss_residual(st.phi, st.U, st.rho, cfg.sigma1, grid),
    }


def positions(st, cfg):
    """Physical positions x = xi * H."""
    return st.xi * np.asarray(cfg.grid().H)


def run(st, cfg, nsteps):
    """Advance nsteps; stops early (returning the last good state) if a step fails to converge."""
    infos = []
    for _ in range(nsteps):
        new, info = step(st, cfg)
        infos.append(info)
        if not info["converged"]:
            break
        st = new
    return st, infos


__all__ = ["Config", "State", "init", "step", "run", "energy", "kinetic_energy",
           "mesh_diagnostics", "picard_iteration", "wrap_cells", "positions", "replace"]
