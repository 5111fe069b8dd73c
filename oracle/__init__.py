"""FP64 CPU oracle for the energy-conserving unstaggered Lorenz-gauge potential PIC step.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product path (the CUDA library and its Python binding) never imports, calls or
links anything here, and this package imports nothing from the product.

What it is
----------
A plain, slow, obviously-correct numpy implementation of what one time step of the
method computes, written from the paper (arXiv 2606.15035, "An Energy-Conserving
Unstaggered Electromagnetic-Potential Particle-in-Cell Method, Part I"):

* ``oracle.mesh``  -- periodic mesh operators, the Crank--Nicolson (CN) potential
  update solved exactly per Fourier mode (§3.2, Eq. (cn-field-update)), continuity
  (Eq. (cn-continuity)), energies (§4.1) and mesh diagnostics (§5.1).
* ``oracle.orbit`` -- straight orbits, knot breakpoints (§4.7, Eq. (breakpoint-set)),
  the exact first-order orbit weights (Appendix A), the exact first-order orbit
  gradient (Appendix B), and a generic Gauss-Legendre path quadrature (§4.7) used
  both for the unsplit comparison run and as an independent check of the closed forms.
* ``oracle.pic``   -- initialisation (§5.4), the Picard iteration of one step
  (Algorithm 1) with the orbit push (§4.4, Eq. (orbit-push)), energies and the
  particle-side diagnostics (§5.2, §5.3).

All arithmetic is float64.  Library primitives used as single steps: ``numpy.fft``
(the exact per-mode CN solve and the Poisson solve), ``numpy.sort`` (breakpoint
ordering) and ``numpy.add.at`` (sequential scatter-add).

Pins: every function here is checked in ``tests/test_oracle_*.py`` against facts the
paper or the mathematics fix (closed forms, identities the paper proves, brute-force
quadrature on tiny inputs, the cold two-stream dispersion relation), not against
itself.  No function is "parity unpinned" except the exact Table 1/2 values, which
depend on fields the paper does not state (see the test module headers).
"""

from . import mesh, orbit, pic  # noqa: F401
