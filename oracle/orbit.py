"""Particle-orbit side of the oracle (test infrastructure only; see ``oracle/__init__``).

Positions are carried in cell units: ``xi = x / H`` per axis, so that the linear
B-spline knots (the mesh nodes, §2.3 Eq. (Ah-mesh) with r = 1) are the integers and
``S_g(x) = prod_a max(0, 1 - |xi_a - g_a|)``.  A straight orbit over one step is
``xi(s) = xi0 + s * beta`` with ``beta = dx / H`` the unwrapped displacement in cell
units (§4.2, Eq. (particle-orbit)); it is wrapped onto the periodic mesh only when a
node index is formed ("periodic wrapping is applied to the mesh index only after the
local stencil has been identified", Appendix A).

Every orbit integral is returned as a list of K entries per particle, each entry a
mesh node with coefficients:

* ``w``      -- contribution to the orbit-averaged shape S̄_ig (Eq. (orbit-average-shape));
* ``s``      -- the global orbit parameter at which A_g(s) = (1-s) A^n + s A^{n+1}
               is anchored (s_m of Appendix B, or the quadrature point);
* ``T0[j]``, ``T1[j]`` -- so that the entry adds
               ``((1-s) A^n_g + s A^{n+1}_g) * T0[j] + (A^{n+1}_g - A^n_g) * T1[j]``
               to [D_i A]_{l j} (Appendix B: T0 multiplies A^{(m)}_{l nu}, T1 multiplies
               C^{(m)}_{l nu}; both already include the factor sigma_{nu_j} / H_j).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class OrbitWeights:
    nodes: np.ndarray   # (np, K, 3) int64, wrapped node indices
    w: np.ndarray       # (np, K)
    s: np.ndarray       # (np, K)
    T0: np.ndarray      # (np, K, 3)
    T1: np.ndarray      # (np, K, 3)


def knot_offset(order):
    """Knot positions of the degree-r B-spline centred on the nodes, in cell units: the
    integers for odd r and the half-integers for even r (the nodes sit at the integers)."""
    return 0.5 if order % 2 == 0 else 0.0


def bspline(x, r):
    """Centred cardinal B-spline of degree r at x (support |x| < (r + 1)/2): the Cox--de Boor
    recursion N_k(y) = [y N_{k-1}(y) + (k + 1 - y) N_{k-1}(y - 1)] / k, N_0 = 1 on [0, 1),
    evaluated at y = x + (r + 1)/2."""
    def N(k, y):
        if k == 0:
            return ((y >= 0.0) & (y < 1.0)).astype(np.float64)
        return (y * N(k - 1, y) + (k + 1 - y) * N(k - 1, y - 1.0)) / k
    return N(r, np.asarray(x, dtype=np.float64) + 0.5 * (r + 1))


def bspline_deriv(x, r):
    """d/dx of the centred B-spline of degree r >= 1: N_r'(y) = N_{r-1}(y) - N_{r-1}(y - 1) on
    y = x + (r + 1)/2, i.e. S_{r-1}(x + 1/2) - S_{r-1}(x - 1/2) (right-continuous at knots)."""
    x = np.asarray(x, dtype=np.float64)
    return bspline(x + 0.5, r - 1) - bspline(x - 0.5, r - 1)


def breakpoints(xi0, beta, split=True):
    """Sorted breakpoints 0 = s_0 <= s_1 <= ... <= s_M = 1 of each orbit (§4.7, Eq. (breakpoint-set)).

    The set is {0, 1} together with every s = (xi - x^n_a)/dx_a in the open interval (0, 1)
    at which axis a crosses a knot xi (an integer in cell units); an axis with dx_a = 0
    contributes nothing.  Instead of removing duplicates, repeated values are kept: they
    create segments of length zero, whose contributions are exactly zero.  Padding slots
    are filled with 1.0 for the same reason.  With ``split=False`` only {0, 1} is
    returned (the unsplit comparison run of §5.4).
    """
    npart = xi0.shape[0]
    cols = [np.zeros(npart), np.ones(npart)]
    if split:
        for a in range(3):
            x = xi0[:, a]
            b = beta[:, a]
            if npart == 0:
                continue
            # an open interval of length |b| holds at most ceil(|b|) integers
            kmax = int(np.ceil(np.max(np.abs(b))))
            for j in range(1, kmax + 1):
                knot = np.where(b > 0, np.floor(x) + j, np.ceil(x) - j)
                with np.errstate(divide="ignore", invalid="ignore"):
                    s = (knot - x) / b
                ok = (b != 0) & (s > 0) & (s < 1)
                cols.append(np.where(ok, s, 1.0))
    s = np.sort(np.stack(cols, axis=1), axis=1)
    # every valid crossing sorts before the 1.0 padding: keep the columns any orbit uses
    used = int(np.max(np.sum(s < 1.0, axis=1))) if npart else 1
    return np.concatenate([s[:, :used], np.ones((npart, 1))], axis=1)


def _wrap(idx, n):
    return np.mod(idx, np.asarray(n, dtype=np.int64))


def closed_form_weights(xi0, beta, grid, split=True, with_gradient=True):
    """Exact first-order orbit weights (Appendix A) and orbit gradient terms (Appendix B).

    For each segment [s_m, s_{m+1}] of length h_m: the stencil cell is the cell that
    contains the segment midpoint; r_{a,m} is the normalised start coordinate in that
    cell; lambda/mu give w_{a,nu}(eta) = lambda + mu*eta; c0..c3 give I_nu; the
    transverse products d0..d2 give the two bracketed terms of I^D_{lj,nu}.
    With ``with_gradient=False`` T0 and T1 are left at zero (deposit-only use).
    """
    s = breakpoints(xi0, beta, split)
    sm = s[:, :-1]
    h = s[:, 1:] - s[:, :-1]
    mid = 0.5 * (s[:, 1:] + s[:, :-1])
    npart, M = sm.shape
    cell = np.floor(xi0[:, None, :] + mid[:, :, None] * beta[:, None, :]).astype(np.int64)
    r = xi0[:, None, :] + sm[:, :, None] * beta[:, None, :] - cell        # r_{a,m}
    bet = np.broadcast_to(beta[:, None, :], r.shape)                       # beta_a

    nodes, W, S, T0s, T1s = [], [], [], [], []
    for nu in np.ndindex(2, 2, 2):
        L = np.empty_like(r)
        Mu = np.empty_like(r)
        for a in range(3):
            if nu[a] == 0:
                L[..., a] = 1.0 - r[..., a]
                Mu[..., a] = -bet[..., a]
            else:
                L[..., a] = r[..., a]
                Mu[..., a] = bet[..., a]
        Lx, Ly, Lz = L[..., 0], L[..., 1], L[..., 2]
        Mx, My, Mz = Mu[..., 0], Mu[..., 1], Mu[..., 2]
        c0 = Lx * Ly * Lz
        c1 = Mx * Ly * Lz + Lx * My * Lz + Lx * Ly * Mz
        c2 = Mx * My * Lz + Mx * Ly * Mz + Lx * My * Mz
        c3 = Mx * My * Mz
        I = c0 * h + c1 / 2 * h ** 2 + c2 / 3 * h ** 3 + c3 / 4 * h ** 4
        T0 = np.zeros(r.shape)
        T1 = np.zeros(r.shape)
        for j in (range(3) if with_gradient else ()):
            p, q = [a for a in range(3) if a != j]
            d0 = L[..., p] * L[..., q]
            d1 = Mu[..., p] * L[..., q] + L[..., p] * Mu[..., q]
            d2 = Mu[..., p] * Mu[..., q]
            sgn = -1.0 if nu[j] == 0 else 1.0
            T0[..., j] = sgn / grid.H[j] * (d0 * h + d1 / 2 * h ** 2 + d2 / 3 * h ** 3)
            T1[..., j] = sgn / grid.H[j] * (d0 / 2 * h ** 2 + d1 / 3 * h ** 3 + d2 / 4 * h ** 4)
        nodes.append(_wrap(cell + np.asarray(nu, dtype=np.int64), grid.n))
        W.append(I)
        S.append(sm)
        T0s.append(T0)
        T1s.append(T1)
    # entries ordered (segment, nu)
    return OrbitWeights(
        nodes=np.stack(nodes, axis=2).reshape(npart, M * 8, 3),
        w=np.stack(W, axis=2).reshape(npart, M * 8),
        s=np.stack(S, axis=2).reshape(npart, M * 8),
        T0=np.stack(T0s, axis=2).reshape(npart, M * 8, 3),
        T1=np.stack(T1s, axis=2).reshape(npart, M * 8, 3),
    )


def point_shape(xi, grid, order=1):
    """Point values of the (r + 1)^3 tensor-product B-splines of degree r = ``order`` that are
    non-zero around ``xi`` (§2.3, Eq. (Ah-mesh)).

    Returns (nodes (np, K, 3), S (np, K), dS (np, K, 3)) with K = (r + 1)^3 and
    dS[..., j] = d S_g / d x_j.  The nodes are those of the knot interval holding xi; on a knot
    the derivative is taken from the interval above.
    """
    first = np.floor(xi - knot_offset(order)).astype(np.int64) - (order - 1) // 2
    nodes, S, dS = [], [], []
    for nu in np.ndindex(order + 1, order + 1, order + 1):
        g = first + np.asarray(nu, dtype=np.int64)
        w = [bspline(xi[:, a] - g[:, a], order) for a in range(3)]
        dw = [bspline_deriv(xi[:, a] - g[:, a], order) / grid.H[a] for a in range(3)]
        nodes.append(_wrap(g, grid.n))
        S.append(w[0] * w[1] * w[2])
        dS.append(np.stack([dw[0] * w[1] * w[2], w[0] * dw[1] * w[2], w[0] * w[1] * dw[2]], axis=1))
    return np.stack(nodes, axis=1), np.stack(S, axis=1), np.stack(dS, axis=1)


def gauss_weights(xi0, beta, grid, nq=16, split=True, order=1):
    """Orbit integrals by an n_q-point Gauss-Legendre rule on every segment (§4.7, §5.4).

    With ``split=True`` the rule is applied on each knot-free segment (knots of the degree-r
    spline, r = ``order``), where it is exact for 2 n_q - 1 >= 3r; with ``split=False`` one
    rule covers the whole path [0, 1], which is the unsplit comparison run.  The integrands
    are the point shape S_g(x(s)) and A_{l,g}(s) d_j S_g(x(s)) themselves.
    """
    t, wq = np.polynomial.legendre.leggauss(nq)
    t = 0.5 * (t + 1.0)
    wq = 0.5 * wq
    s = breakpoints(xi0 - knot_offset(order), beta, split)
    sm = s[:, :-1]
    h = s[:, 1:] - s[:, :-1]
    npart, M = sm.shape
    nodes, W, S, T0s, T1s = [], [], [], [], []
    for m in range(M):
        for q in range(nq):
            sq = sm[:, m] + h[:, m] * t[q]
            xq = xi0 + sq[:, None] * beta
            nd, Sv, dS = point_shape(xq, grid, order)
            fac = (h[:, m] * wq[q])[:, None]
            nodes.append(nd)
            W.append(fac * Sv)
            S.append(np.broadcast_to(sq[:, None], Sv.shape))
            T0s.append(fac[:, :, None] * dS)
            T1s.append(np.zeros_like(dS))
    return OrbitWeights(
        nodes=np.concatenate(nodes, axis=1),
        w=np.concatenate(W, axis=1),
        s=np.concatenate(S, axis=1),
        T0=np.concatenate(T0s, axis=1),
        T1=np.concatenate(T1s, axis=1),
    )


# --- Operations built on the orbit weights (§4.2, §4.3, §4.4) --------------------------

def _take(G, nodes):
    """G[..., nodes] for a mesh array G of shape (..., nx, ny, nz)."""
    return G[..., nodes[..., 0], nodes[..., 1], nodes[..., 2]]


def gather(G, ow):
    """Orbit gather bar G_i = sum_g G_g S̄_ig (Eq. (orbit-gather-general)).  G is (3, n...) or (n...)."""
    vals = _take(G, ow.nodes)                                  # (..., np, K)
    return np.sum(vals * ow.w, axis=-1)


def flat_index(nodes, n):
    """Row-major flat index of node (ix, iy, iz) in a mesh of shape n."""
    return (nodes[..., 0] * n[1] + nodes[..., 1]) * n[2] + nodes[..., 2]


def deposit(q_vbar, ow, grid):
    """Orbit current J_g = (1/dV) sum_i q_i vbar_i S̄_ig (Eq. (orbit-current)), sequential scatter-add."""
    J = np.zeros((3,) + grid.n)
    idx = flat_index(ow.nodes, grid.n).ravel()
    for c in range(3):
        J[c] = np.bincount(idx, weights=(q_vbar[:, c:c + 1] * ow.w).ravel() / grid.dV,
                           minlength=grid.ncell).reshape(grid.n)
    return J


def orbit_gradient(An, An1, ow):
    """[D_i A]_{l j} (Eq. (DA-def), split form Eq. (split-DA), closed form Appendix B).

    Each entry contributes A^{(m)}_{l,nu} * T0[j] + C^{(m)}_{l,nu} * T1[j] with
    A^{(m)} = (1 - s_m) A^n_g + s_m A^{n+1}_g and C^{(m)} = A^{n+1}_g - A^n_g.
    Returns an array (np, 3, 3) indexed [i, l, j].
    """
    a_n = _take(An, ow.nodes)          # (3, np, K)
    a_1 = _take(An1, ow.nodes)
    Am = (1.0 - ow.s) * a_n + ow.s * a_1
    C = a_1 - a_n
    DA = np.einsum("lik,ikj->ilj", Am, ow.T0) + np.einsum("lik,ikj->ilj", C, ow.T1)
    return DA


def point_gather(G, xi, grid, order=1):
    """Mesh interpolant G_h(x) = sum_g G_g S_g(x) at points (Eq. (Ah-mesh))."""
    nodes, S, _ = point_shape(xi, grid, order)
    return np.sum(_take(G, nodes) * S, axis=-1)
