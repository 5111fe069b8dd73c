"""Periodic mesh side of the oracle (test infrastructure only; see ``oracle/__init__``).

Layout: a scalar mesh field is a float64 array ``f[ix, iy, iz]`` of shape
``(nx, ny, nz)``; a vector field is ``F[c, ix, iy, iz]`` of shape ``(3, nx, ny, nz)``.
Node ``g = (ix, iy, iz)`` sits at ``x_g = (ix*Hx, iy*Hy, iz*Hz)`` (node-collocated,
"unstaggered", §3).

Spatial operators (the reading used throughout, stated in the design notes):
the paper's theorems (§3.3 Theorem "gauge and Gauss preservation", §4.6 field energy
balance) need periodic first-derivative operators ``D_a`` that are skew-adjoint and
commute, and a Laplacian equal to ``sum_a D_a D_a``.  Two choices are provided:
``ops="central2"`` (default), the second-order central difference
``D_a f = (f[i+1] - f[i-1]) / (2 H_a)`` with the matching wide Laplacian
``Delta_h = sum_a D_a D_a`` (radius-2 stencil per axis); and ``ops="spectral"``, the
paper's Fourier operators (§3.3): symbol ``i k_a`` with ``k_a = 2 pi m_a / L_a``, the
Nyquist symbol (2 |m_a| = n_a) set to zero so that ``D_a`` stays real and skew-adjoint,
and ``Delta_h = sum_a D_a D_a`` with symbol ``-sum_a k_a^2`` (zero on the same 8 modes).
"""

from __future__ import annotations

import numpy as np


class Grid:
    """Periodic box ``[0,Lx) x [0,Ly) x [0,Lz)`` with ``n = (nx, ny, nz)`` nodes (§5.4)."""

    def __init__(self, n, L, ops="central2"):
        if ops not in ("central2", "spectral"):
            raise ValueError(ops)
        self.ops = ops
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.H = tuple(self.L[a] / self.n[a] for a in range(3))
        self.dV = self.H[0] * self.H[1] * self.H[2]
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.volume = self.L[0] * self.L[1] * self.L[2]

    # --- Fourier symbols ---------------------------------------------------------
    def wavenumbers(self):
        """Integer-mode angles theta_a = 2 pi m_a / n_a broadcast to the mesh shape."""
        th = []
        for a in range(3):
            m = np.fft.fftfreq(self.n[a]) * self.n[a]
            shape = [1, 1, 1]
            shape[a] = self.n[a]
            th.append((2.0 * np.pi * m / self.n[a]).reshape(shape))
        return th

    def d_symbol(self, a):
        """Symbol of D_a acting on exp(i theta x/H): i sin(theta)/H (central difference), or
        i k = i theta / H with the Nyquist mode set to 0 (spectral)."""
        th = self.wavenumbers()[a]
        if self.ops == "central2":
            return 1j * np.sin(th) / self.H[a]
        m = np.rint(th * self.n[a] / (2.0 * np.pi))
        return np.where(2 * np.abs(m) == self.n[a], 0.0, 1j * th / self.H[a])

    def lap_symbol(self):
        """Symbol of Delta_h = sum_a D_a D_a (<= 0): the sum of the squared D_a symbols."""
        s = np.zeros(self.n)
        for a in range(3):
            s = s + np.real(self.d_symbol(a) ** 2)
        return s

    def null_mask(self):
        """Modes on which Delta_h's symbol is exactly zero (theta_a in {0, pi} on every axis)."""
        th = self.wavenumbers()
        mask = np.ones(self.n, dtype=bool)
        for a in range(3):
            m = np.fft.fftfreq(self.n[a]) * self.n[a]
            ok = (m == 0) | (2 * np.abs(m) == self.n[a])
            shape = [1, 1, 1]
            shape[a] = self.n[a]
            mask = mask & ok.reshape(shape)
        return mask


# --- Real-space stencil operators (§3.2, §4.1) ----------------------------------------

def d(f, a, grid):
    """D_a along axis ``a``: the central difference (f[i+1] - f[i-1]) / (2 H_a), periodic, or
    (spectral) multiplication of the Fourier coefficients by the D_a symbol."""
    if grid.ops == "central2":
        return (np.roll(f, -1, axis=a) - np.roll(f, 1, axis=a)) / (2.0 * grid.H[a])
    return np.real(np.fft.ifftn(grid.d_symbol(a) * np.fft.fftn(f)))


def grad(f, grid):
    """Mesh gradient nabla_h f (three components)."""
    return np.stack([d(f, a, grid) for a in range(3)])


def div(F, grid):
    """Mesh divergence nabla_h . F = sum_a D_a F_a."""
    return d(F[0], 0, grid) + d(F[1], 1, grid) + d(F[2], 2, grid)


def lap(f, grid):
    """Delta_h f = sum_a D_a D_a f (the wide Laplacian that makes Delta_h = nabla_h . nabla_h)."""
    return sum(d(d(f, a, grid), a, grid) for a in range(3))


def curl(F, grid):
    """Mesh curl nabla_h x F (§4.1, Eq. (fields-from-potentials-discrete))."""
    return np.stack([
        d(F[2], 1, grid) - d(F[1], 2, grid),
        d(F[0], 2, grid) - d(F[2], 0, grid),
        d(F[1], 0, grid) - d(F[0], 1, grid),
    ])


# --- Crank--Nicolson potential update (§3.2, Eq. (cn-field-update)) -------------------

def cn_update(u, w, src, coef, dt, kappa, grid):
    """One CN step of the pair ``du/dt = w, dw/dt = kappa^2 Delta_h u + kappa^2 coef src``.

    Solves, exactly for every Fourier mode (2x2 linear system per mode, Cramer's rule),
        (u1 - u0)/dt = (w1 + w0)/2
        (w1 - w0)/dt = kappa^2 lam (u1 + u0)/2 + kappa^2 coef src
    where lam is the Delta_h symbol and ``src`` is the time-centred source
    (rho^{n+1/2} with coef = sigma1, or one component of J^{n+1/2} with coef = sigma2).
    Returns (u1, w1).
    """
    lam = grid.lap_symbol()
    U0 = np.fft.fftn(u)
    W0 = np.fft.fftn(w)
    S = np.fft.fftn(src)
    b = 0.5 * dt * kappa ** 2 * lam          # coefficient of (u1 + u0) in the w equation
    # [ 1      -dt/2 ] [u1]   [ u0 + dt/2 w0                      ]
    # [ -b       1   ] [w1] = [ w0 + b u0 + dt kappa^2 coef S       ]
    r1 = U0 + 0.5 * dt * W0
    r2 = W0 + b * U0 + dt * kappa ** 2 * coef * S
    det = 1.0 - 0.5 * dt * b
    U1 = (r1 + 0.5 * dt * r2) / det
    W1 = (r2 + b * r1) / det
    return np.real(np.fft.ifftn(U1)), np.real(np.fft.ifftn(W1))


def cn_fields(phi, psi, A, U, rho_half, J_half, dt, kappa, sigma1, sigma2, grid):
    """CN update of (phi, psi, A, U) from (rho^{n+1/2}, J^{n+1/2}) (Eq. (cn-field-update))."""
    phi1, psi1 = cn_update(phi, psi, rho_half, sigma1, dt, kappa, grid)
    A1 = np.empty_like(A)
    U1 = np.empty_like(U)
    for c in range(3):
        A1[c], U1[c] = cn_update(A[c], U[c], J_half[c], sigma2, dt, kappa, grid)
    return phi1, psi1, A1, U1


def continuity(rho, J_half, dt, grid):
    """rho^{n+1} = rho^n - dt nabla_h . J^{n+1/2} (Eq. (cn-continuity))."""
    return rho - dt * div(J_half, grid)


def project_out_null(f, grid):
    """Remove the components of ``f`` on the null modes of Delta_h (mean and checkerboards)."""
    F = np.fft.fftn(f)
    F[grid.null_mask()] = 0.0
    return np.real(np.fft.ifftn(F))


def poisson(rho, sigma1, grid):
    """phi with -Delta_h phi = sigma1 rho, zero on the null modes of Delta_h (§5.4 initial data)."""
    lam = grid.lap_symbol()
    R = np.fft.fftn(rho)
    null = grid.null_mask()
    P = np.zeros_like(R)
    P[~null] = sigma1 * R[~null] / (-lam[~null])
    return np.real(np.fft.ifftn(P))


# --- Fields and energies (§4.1) ------------------------------------------------------

def efield(phi, U, grid):
    """E = -nabla_h phi - U (Eq. (fields-from-potentials-discrete))."""
    return -grad(phi, grid) - U


def bfield(A, grid):
    """B = nabla_h x A (Eq. (fields-from-potentials-discrete))."""
    return curl(A, grid)


def field_energy(phi, U, A, sigma1, sigma2, grid):
    """W = sum_g (|E_g|^2/(2 sigma1) + |B_g|^2/(2 sigma2)) dV (Eq. (field-energy))."""
    E = efield(phi, U, grid)
    B = bfield(A, grid)
    return float((np.sum(E * E) / (2.0 * sigma1) + np.sum(B * B) / (2.0 * sigma2)) * grid.dV)


def gauge_residual(psi, A, kappa, grid):
    """G_h = psi/kappa^2 + nabla_h . A (§5.1, Eq. (gauge-diagnostic))."""
    return psi / kappa ** 2 + div(A, grid)


def gauss_residual(phi, U, rho, sigma1, grid):
    """R_h = nabla_h . E - sigma1 rho (§5.1, Eq. (gauss-diagnostic))."""
    return div(efield(phi, U, grid), grid) - sigma1 * rho
