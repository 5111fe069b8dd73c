"""Ensembles of independent runs (pic_ensemble_*): each run of an ensemble must compute what
the same run computes alone, whatever the other runs are (different meshes, particle counts,
beam parameters and precisions), and a failing run must not stop the others."""

import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim(cuda_ok):
    from paper_2606_15035_gb300 import build
    build.build()
    from paper_2606_15035_gb300 import sim as s
    return s


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


RUNS = [  # (mesh, particles per beam per cell, v0, eps, seed, precision)
    ((8, 8, 8), 8, 0.2, 1e-3, 2001, 0),
    ((6, 5, 4), 6, 0.3, 1e-2, 2002, 0),
    ((12, 12, 12), 4, 0.15, 1e-3, 2003, 1),
    ((8, 8, 8), 4, 0.25, 5e-3, 2004, 1),
]


def _runs(sim, overrides=None):
    out = []
    side = 2 * np.pi / 3
    for k, (n, ppb, v0, eps, seed, prec) in enumerate(RUNS):
        x, v, q, m = pi.random_twostream(n, (side,) * 3, ppb, v0, eps, 0.0, seed)
        kw = dict(n=n, L=(side,) * 3, dt=0.1, picard_tol=1e-13, precision=prec)
        kw.update((overrides or {}).get(k, {}))
        out.append((sim.pic_config_default(**kw), x, v, q, m))
    return out


def test_ensemble_runs_match_the_same_runs_alone(sim):
    runs = _runs(sim)
    ens = sim.PicEnsemble(runs)
    infos, sts = ens.step(3)
    assert sts == [0] * len(runs)
    for k, (cfg, x, v, q, m) in enumerate(runs):
        assert infos[k].steps_done == 3 and infos[k].converged
        solo = sim.PicSim(cfg, x, v, q, m)
        solo.step(3)
        a, b = ens.runs[k].get_state(), solo.get_state()
        tol = 1e-12 if cfg.precision == 0 else 1e-11
        for name in ("x", "v", "P", "vprev", "phi", "A", "rho"):
            assert rel(getattr(a, name), getattr(b, name)) <= tol, (k, name, rel(getattr(a, name), getattr(b, name)))
        ea, eb = ens.runs[k].energy().total, solo.energy().total
        assert abs(ea - eb) <= 1e-13 * abs(eb)
        solo.close()
    ens.close()


def test_ensemble_members_match_the_oracle(sim):
    """An FP64 member and a mixed member of the ensemble against the FP64 oracle after three
    steps (the mixed path refines to the same tolerance in FP64, so it solves the same
    equations): state within 1e-12 (FP64) and 1e-11 (mixed)."""
    from oracle import pic as opic
    runs = _runs(sim)
    ens = sim.PicEnsemble(runs)
    _, sts = ens.step(3)
    assert sts == [0] * len(runs)
    for k in (1, 2):                       # (6, 5, 4) FP64 and (12, 12, 12) mixed
        cfg, x, v, q, m = runs[k]
        n, L = tuple(cfg.n), tuple(cfg.L)
        ocfg = opic.Config(n=n, L=L, dt=cfg.dt, picard_tol=cfg.picard_tol, picard_max=cfg.picard_max)
        o = opic.init(x, v, q, m, ocfg)
        for _ in range(3):
            o, oinfo = opic.step(o, ocfg)
            assert oinfo["converged"]
        a = ens.runs[k].get_state()
        tol = 1e-12 if cfg.precision == 0 else 1e-11
        Lv = np.asarray(L)
        d = a.x - opic.positions(o, ocfg)
        assert np.abs((d + 0.5 * Lv) % Lv - 0.5 * Lv).max() <= tol * Lv.max()
        for name in ("v", "P", "vprev", "phi", "psi", "A", "U", "rho"):
            b = getattr(o, name)
            scale = max(np.linalg.norm(b), 1e-14 * np.sqrt(b.size))
            err = np.linalg.norm(getattr(a, name) - b) / scale
            assert err <= tol, (k, name, err)
    ens.close()


def test_a_failing_run_does_not_stop_the_others(sim):
    # run 1 cannot converge (tolerance below roundoff, two iterations allowed)
    runs = _runs(sim, {1: dict(picard_tol=1e-30, picard_max=1)})
    ens = sim.PicEnsemble(runs)
    before = ens.runs[1].get_state()
    infos, sts = ens.step(2, raise_on_error=False)
    assert sts[1] == 4                         # PIC_ERR_NO_CONVERGENCE
    assert [sts[k] for k in (0, 2, 3)] == [0, 0, 0]
    assert [infos[k].steps_done for k in (0, 2, 3)] == [2, 2, 2] and infos[1].steps_done == 0
    after = ens.runs[1].get_state()            # nothing of the failed run was committed
    for name in ("x", "v", "P", "phi", "A"):
        assert np.array_equal(getattr(after, name), getattr(before, name)), name
    with pytest.raises(sim.PicError):
        ens.step(1)
    ens.close()


def test_autotune_picks_a_grid_and_leaves_the_state_alone(sim):
    """pic_autotune times candidate grids on scratch buffers only: the committed state and
    the following steps are those of an untuned context (up to the FP64 atomics' order)."""
    for k in (0, 2):   # an FP64 and a mixed run
        cfg, x, v, q, m = _runs(sim)[k]
        a, b = sim.PicSim(cfg, x, v, q, m), sim.PicSim(cfg, x, v, q, m)
        before = a.get_state()
        bps, bps32 = a.autotune()
        assert bps in (2, 4, 8, 16) and bps32 in (4, 8, 16)
        assert a.autotune() == (bps, bps32)          # cached
        after = a.get_state()
        for name in ("x", "v", "P", "vprev", "phi", "psi", "A", "U", "rho"):
            assert np.array_equal(getattr(after, name), getattr(before, name)), name
        a.step(2)
        b.step(2)
        sa, sb = a.get_state(), b.get_state()
        tol = 1e-12 if cfg.precision == 0 else 1e-11
        for name in ("x", "v", "P", "phi", "A"):
            assert rel(getattr(sa, name), getattr(sb, name)) <= tol, (k, name)
        a.close()
        b.close()
