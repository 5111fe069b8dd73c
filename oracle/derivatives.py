"""Reference derivatives of the step map (test infrastructure only).

The adjoint of the implicit step differentiates the field energy after N steps, W^N, with
respect to the initial data: the perturbation amplitude, the beam speed and the initial
canonical momenta.  That derivative has a plain definition, the limit of the difference
quotient, and this module writes it out on the oracle's own steps: a central difference,
Richardson-extrapolated,

    D(h) = (f(+h) - f(-h)) / (2 h),    R(h) = (4 D(h/2) - D(h)) / 3,

whose truncation error is O(h^4) for a smooth f.  The step map is only C^0 where an orbit
endpoint crosses a knot (D_i A is continuous but not differentiable there, §4.3), and a
particle-local solve that slides onto a knot switches branch; a quotient that straddles such
an event is not a derivative, so h must stay well inside the gap to the nearest one.
"""

from __future__ import annotations

import numpy as np

from . import pic


def richardson(f, h):
    """Derivative at 0 of the scalar function f(s) from central differences at h and h/2,
    Richardson-extrapolated (error O(h^4) for smooth f)."""
    d1 = (f(h) - f(-h)) / (2.0 * h)
    d2 = (f(0.5 * h) - f(-0.5 * h)) / h
    return (4.0 * d2 - d1) / 3.0


def field_energy_after(x, v, q, m, cfg, nsteps):
    """W^N: the field energy (Eq. (field-energy)) after nsteps converged oracle steps from the
    initial data (x, v); raises if a step does not converge."""
    st = pic.init(x, v, q, m, cfg)
    for _ in range(nsteps):
        st, info = pic.step(st, cfg)
        if not info["converged"]:
            raise RuntimeError("a step did not converge")
    return pic.energy(st, cfg)[1]


def directional_derivative(make_data, cfg, nsteps, h):
    """d W^N / ds at s = 0 along a family of initial data make_data(s) -> (x, v, q, m)."""
    return richardson(lambda s: field_energy_after(*make_data(s), cfg, nsteps), h)
