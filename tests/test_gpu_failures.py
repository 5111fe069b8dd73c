"""Failure detection without a GPU fault: each device-side error status is provoked from the
host with inputs the library checks (a non-finite velocity, an orbit longer than the
supported number of knot crossings, a wait bound shorter than a bulk copy's latency), and the
step must return that status, keep the committed state bit for bit, and leave the context
usable: once the cause is removed the next step converges.

None of these faults, traps or hangs the GPU: the non-finite velocity and the long orbit
are found by the kernels' own checks (every mesh index is wrapped, every segment loop is
bounded), and the short wait bound makes each FP32 push block give up its first wait, wait
with the full bound for the copies it has in flight, and stop."""

import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

NAMES = ("x", "v", "P", "vprev", "phi", "psi", "rho", "A", "U")


@pytest.fixture(scope="module")
def sim(cuda_ok):
    from paper_2606_15035_gb300 import build
    build.build()
    from paper_2606_15035_gb300 import sim as s
    return s


def same_state(a, b):
    for name in NAMES:
        assert np.array_equal(getattr(a, name), getattr(b, name), equal_nan=True), name


def c1(sim, precision=0):
    w = pi.WORKLOADS["twostream-8c-8k"]
    x, v, q, m = pi.random_twostream(w.n, w.L, 2, w.v0, w.eps, 1e-3, 4100)
    cfg = sim.pic_config_default(n=w.n, L=w.L, dt=w.dt, picard_tol=1e-13, precision=precision)
    return sim.PicSim(cfg, x, v, q, m)


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_velocity_is_reported_and_the_state_kept(sim, precision):
    s = c1(sim, precision)
    s.step(1)
    good = s.get_state()
    bad = s.get_state()
    bad.v[17, 1] = np.nan
    s.set_state(bad)
    before = s.get_state()                          # positions as stored (cell units) after the set
    with pytest.raises(sim.PicError) as e:
        s.step(1)
    assert e.value.status == 5                      # PIC_ERR_NONFINITE
    assert np.isnan(before.v[17, 1])
    same_state(s.get_state(), before)
    s.set_state(good)                               # the cause removed: the context works again
    assert s.step(1).converged
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_orbit_beyond_the_segment_capacity_is_reported(sim, precision):
    """One particle crossing 70 knots in one step (the kernels support 64 orbit pieces)."""
    n, L = (128, 4, 4), (4.0, 1.0, 1.0)
    H = L[0] / n[0]
    x, v, q, m = pi.random_twostream(n, L, 1, 0.2 * H / 0.1, 1e-3, 0.0, 4200)
    cfg = sim.pic_config_default(n=n, L=L, dt=0.1, picard_tol=1e-13, precision=precision)
    s = sim.PicSim(cfg, x, v, q, m)
    assert s.step(1).converged
    good = s.get_state()
    bad = s.get_state()
    bad.v[3] = (70.0 * H / 0.1, 0.0, 0.0)
    bad.vprev[3] = bad.v[3]
    s.set_state(bad)
    before = s.get_state()
    with pytest.raises(sim.PicError) as e:
        s.step(1)
    assert e.value.status == 6                      # PIC_ERR_SEGMENTS
    same_state(s.get_state(), before)
    s.set_state(good)
    assert s.step(1).converged
    s.close()


def test_bounded_copy_wait_gives_up_and_the_context_stays_usable(sim):
    """PIC_MIXED with a one-cycle bound on the FP32 push's waits for its staged particle chunks:
    every block gives up its first wait (a bulk copy from HBM takes far longer), the step
    returns PIC_ERR_TIMEOUT with the state kept, and with the default bound restored the same
    step converges to what an untouched context computes."""
    s, ref = c1(sim, 1), c1(sim, 1)
    s.step(1)
    ref.step(1)
    before = s.get_state()
    s.set_wait_limit(1)
    with pytest.raises(sim.PicError) as e:
        s.step(1)
    assert e.value.status == 8                      # PIC_ERR_TIMEOUT
    same_state(s.get_state(), before)
    s.set_wait_limit(2_000_000_000)
    assert s.step(1).converged
    ref.step(1)
    a, b = s.get_state(), ref.get_state()
    for name in ("v", "P", "phi", "A"):
        d = np.linalg.norm(getattr(a, name) - getattr(b, name)) / np.linalg.norm(getattr(b, name))
        assert d <= 1e-11, (name, d)
    with pytest.raises(sim.PicError):
        s.set_wait_limit(0)
    s.close()
    ref.close()
