"""The seeded input generator: known-answer SplitMix64 finaliser, shapes, neutrality, determinism."""

import numpy as np

import pic_inputs as pi
from pic_inputs import twostream


def test_splitmix64_finaliser_known_answer():
    # SplitMix64 with state 0: the first output is mix(0x9E3779B97F4A7C15) = 0xE220A8397B1DCDAF.
    z = twostream._mix(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_workload_shapes_and_neutrality():
    w = pi.WORKLOADS["twostream-8c-8k"]
    x, v, q, m = pi.workload_particles(w)
    assert x.shape == (8192, 3) and v.shape == (8192, 3)
    assert q < 0 and m == -q
    vol = np.prod(w.L)
    assert abs(q * x.shape[0] + vol) < 1e-12 * vol          # electrons balance n0 = 1
    assert np.all(x >= 0) and np.all(x < np.asarray(w.L))
    half = x.shape[0] // 2
    np.testing.assert_array_equal(x[:half], x[half:])        # beams share positions
    np.testing.assert_array_equal(v[:half, 0], 0.2)
    np.testing.assert_array_equal(v[half:, 0], -0.2)


def test_deterministic_and_thermal_spread():
    n = (4, 4, 4)
    L = (1.0, 1.0, 1.0)
    a = pi.random_twostream(n, L, 64, 0.2, 1e-3, 1e-4, 77)
    b = pi.random_twostream(n, L, 64, 0.2, 1e-3, 1e-4, 77)
    c = pi.random_twostream(n, L, 64, 0.2, 1e-3, 1e-4, 78)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert np.abs(a[0] - c[0]).max() > 0.1
    dv = a[1][:, 1:]
    assert abs(np.std(dv) - 1e-4) < 5e-6 and abs(np.mean(dv)) < 5e-6


def test_ensemble_runs_are_seeded_and_in_range():
    import pic_inputs as pi
    a, b = pi.ensemble_runs(), pi.ensemble_runs()
    assert a == b and len(a) == 64
    assert {r.n[0] for r in a} == {16, 24, 32, 48}
    assert all(4 <= r.per_beam_per_cell <= 32 for r in a)
    assert all(0.1 <= r.v0 <= 0.3 and 1e-4 <= r.eps <= 1e-2 for r in a)
    assert len({r.seed for r in a}) == 64
    x, v, q, m = pi.ensemble_particles(a[0])
    assert x.shape == (a[0].n_particles, 3) and np.isclose(abs(v[:, 0]).max(), a[0].v0, rtol=0.2)
