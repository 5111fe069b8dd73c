"""Deterministic mode (pic_config.deterministic = 1): a stable radix sort, exact fixed-point
deposits and index-ordered local solves make every step a function of its inputs alone.
Checked bit for bit: two contexts on the same inputs, and a run inside an ensemble against
the same run alone; the mode still matches the FP64 oracle like the default mode."""

import numpy as np
import pytest

import pic_inputs as pi
from oracle import pic as opic

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "P", "vprev", "phi", "psi", "rho", "A", "U")


@pytest.fixture(scope="module")
def sim(cuda_ok):
    from paper_2606_15035_gb300 import build
    build.build()
    from paper_2606_15035_gb300 import sim as s
    return s


def _inputs(n=(12, 10, 8), per_beam=6, vth=2e-3, seed=3001):
    side = 2 * np.pi / 3
    x, v, q, m = pi.random_twostream(n, (side,) * 3, per_beam, 0.25, 1e-2, vth, seed)
    return n, (side,) * 3, x, v, q, m


def _bitwise_equal(a, b):
    for name in FIELDS:
        assert np.array_equal(getattr(a, name), getattr(b, name)), name


@pytest.mark.parametrize("precision", [0, 1])
def test_two_runs_are_bitwise_equal(sim, precision):
    n, L, x, v, q, m = _inputs()
    cfg = sim.pic_config_default(n=n, L=L, dt=0.15, picard_tol=1e-13, precision=precision, deterministic=1)
    a, b = sim.PicSim(cfg, x, v, q, m), sim.PicSim(cfg, x, v, q, m)
    for _ in range(4):
        ia, ib = a.step(1), b.step(1)
        assert ia.iterations == ib.iterations and ia.e_v == ib.e_v and ia.e_J == ib.e_J
        _bitwise_equal(a.get_state(), b.get_state())
    assert a.energy().total == b.energy().total
    a.close()
    b.close()


def test_ensemble_run_is_bitwise_equal_to_the_run_alone(sim):
    n, L, x, v, q, m = _inputs()
    n2, L2, x2, v2, q2, m2 = _inputs(n=(8, 8, 8), per_beam=4, seed=3002)
    cfg = sim.pic_config_default(n=n, L=L, dt=0.15, picard_tol=1e-13, deterministic=1)
    cfg2 = sim.pic_config_default(n=n2, L=L2, dt=0.1, picard_tol=1e-13, precision=1, deterministic=1)
    ens = sim.PicEnsemble([(cfg, x, v, q, m), (cfg2, x2, v2, q2, m2)], autotune=True)
    ens.step(3)
    solo = sim.PicSim(cfg, x, v, q, m)
    solo.step(3)
    _bitwise_equal(ens.runs[0].get_state(), solo.get_state())
    solo.close()
    solo2 = sim.PicSim(cfg2, x2, v2, q2, m2)
    solo2.step(3)
    _bitwise_equal(ens.runs[1].get_state(), solo2.get_state())
    solo2.close()
    ens.close()


def test_deterministic_mode_matches_the_oracle(sim):
    w = pi.WORKLOADS["twostream-8c-8k"]
    x, v, q, m = pi.workload_particles(w)
    cfg = sim.pic_config_default(n=w.n, L=w.L, dt=w.dt, picard_tol=1e-13, deterministic=1)
    s = sim.PicSim(cfg, x, v, q, m)
    ocfg = opic.Config(n=w.n, L=w.L, dt=w.dt, picard_tol=1e-13)
    o = opic.init(x, v, q, m, ocfg)
    for _ in range(3):
        assert s.step(1).converged
        o, _ = opic.step(o, ocfg)
    st = s.get_state()
    for name, ref in (("v", o.v), ("P", o.P), ("phi", o.phi), ("A", o.A), ("rho", o.rho)):
        got = getattr(st, name)
        scale = max(np.linalg.norm(ref), 1e-14 * np.sqrt(ref.size))
        assert np.linalg.norm(got - ref) / scale <= 1e-12, name
    s.close()
