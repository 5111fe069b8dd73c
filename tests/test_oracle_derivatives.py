"""Pins of the reference derivatives (oracle/derivatives.py) the adjoint is checked against.

* The Richardson-extrapolated central difference against closed-form derivatives, to its
  O(h^4) bound (a one-sided or unextrapolated quotient fails it).
* The whole multi-step map on the paper's quiet lattice start (§5.4, velocity perturbation
  eps sin(k x)): in the linear regime every field is proportional to eps, so the field energy
  after N steps is W^N = c eps^2 up to nonlinear terms of relative size O(eps^2), and
  dW^N/d eps = 2 W^N / eps.  The measured gap shrinks a hundredfold when eps shrinks tenfold.
"""

import numpy as np
import pytest

import pic_inputs as pi
from oracle import derivatives as dv
from oracle import pic


def test_richardson_matches_closed_form_derivatives():
    f = lambda s: np.sin(1.3 + s) * np.exp(0.7 * s)
    exact = np.cos(1.3) + 0.7 * np.sin(1.3)
    assert abs(dv.richardson(f, 1e-2) - exact) <= 1e-9
    g = lambda s: (2.0 + s) ** 5
    assert abs(dv.richardson(g, 1e-2) - 5 * 2.0 ** 4) <= 1e-8 * 80.0
    # the plain central difference at the same h misses by O(h^2)
    d1 = (f(1e-2) - f(-1e-2)) / 2e-2
    assert abs(d1 - exact) > 1e-6


@pytest.mark.parametrize("eps,nsteps,bound", [(1e-3, 2, 1e-6), (1e-3, 5, 2e-6), (1e-4, 5, 2e-8)])
def test_field_energy_derivative_scales_as_eps_squared(eps, nsteps, bound):
    n, L = (8, 2, 2), (2 * np.pi / 3, 0.5, 0.5)
    cfg = pic.Config(n=n, L=L, dt=0.1, picard_tol=1e-14)
    make = lambda s: pi.lattice_twostream(n, L, 8, 0.2, eps + s)
    W = dv.field_energy_after(*make(0.0), cfg, nsteps)
    d = dv.directional_derivative(make, cfg, nsteps, 1e-2 * eps)
    assert W > 0
    assert abs(d - 2.0 * W / eps) <= bound * 2.0 * W / eps
