"""The bench's roofline bookkeeping on CPU, from hand-made profiles (the fields of
pic_profile_t that bench.py reads): which kernel carries the line's `roofline` object, and the
arithmetic of the FP64 iteration, final-sweep and FP32-pair summaries.  The profile sums the
orbit pieces of FP64 and FP32-pair iterations together, so the FP64 roofline must count only
the FP64 launches' share of them."""

import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NP = 1000


def _prof(push=0, pair=0, commit=1, push_ms=0.0, pair_ms=0.0, commit_ms=2.0, pieces=1.5, spieces=1.25):
    launches = push + pair
    return SimpleNamespace(
        push_launches=push, push_ms=push_ms, pushpair_launches=pair, pushpair_ms=pair_ms,
        commit_launches=commit, commit_ms=commit_ms, particle_pushes=push * NP,
        push_pieces=int(pieces * launches * NP), scatter_pieces=int(spieces * launches * NP),
        push32_launches=0, push32_ms=0.0, push32_chunks=0, push32_chunks_global=0,
        local_ms=0.0, mesh_ms=0.0, scatter_ms=0.0, sort_ms=0.0, launches=10)


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def test_mean_pieces_divides_by_both_kinds_of_iteration(bench):
    p = _prof(push=1, pair=3)
    mp, msc = bench.mean_pieces(p, NP)
    assert mp == pytest.approx(1.5) and msc == pytest.approx(1.25)
    assert bench.mean_pieces(_prof(), NP) == (0.0, 0.0)


def test_fp64_roofline_counts_only_fp64_launches(bench):
    alone = bench.fp64_push_roofline(_prof(push=2, push_ms=4.0), "x")
    mixed = bench.fp64_push_roofline(_prof(push=2, pair=6, push_ms=4.0), "x")
    # the same two FP64 launches: the pair launches' pieces must not inflate their flops
    assert mixed["flops_per_launch"] == pytest.approx(alone["flops_per_launch"])
    per = NP * (bench.FLOPS_PER_PARTICLE + 1.5 * bench.FLOPS_PER_PUSH_PIECE + 1.25 * bench.FLOPS_PER_SCATTER_PIECE)
    assert alone["flops_per_launch"] == pytest.approx(per)
    assert alone["achieved"] == pytest.approx(2 * per / 4e-3 / 1e12)
    assert bench.fp64_push_roofline(_prof(push=0, pair=3), "x") is None


def test_final_sweep_roofline_uses_the_scattered_orbits_pieces(bench):
    r = bench.final_sweep_roofline(_prof(pair=1, pair_ms=3.0, commit=1, commit_ms=2.0), "x", NP)
    per = NP * (bench.FLOPS_PER_PARTICLE + 1.25 * bench.FLOPS_PER_PUSH_PIECE)
    assert r["flops_per_launch"] == pytest.approx(per)
    assert r["achieved"] == pytest.approx(per / 2e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert bench.final_sweep_roofline(_prof(commit=0, commit_ms=0.0), "x", NP) is None


def test_pair_summary_is_reported_only_when_pairs_ran(bench):
    assert bench.pair_push_summary(_prof(push=1, push_ms=1.0), NP, 10.0) is None
    s = bench.pair_push_summary(_prof(pair=2, pair_ms=6.0), NP, 12.0)
    assert s["ms_per_launch"] == pytest.approx(3.0) and s["share_of_step"] == pytest.approx(0.5)
    per = NP * (bench.FLOPS_PER_PARTICLE + 1.5 * bench.FLOPS_PER_PUSH_PIECE + 1.25 * bench.FLOPS_PER_SCATTER_PIECE)
    assert s["fp64_equivalent_tflops"] == pytest.approx(per / 3e-3 / 1e12)


def test_kernel_shares_include_the_pair_push(bench):
    sh = bench.kernel_shares(_prof(pair=1, pair_ms=5.0, commit_ms=3.0), 10.0)
    assert sh["k_push_df (FP32-pair iterations)"] == pytest.approx(0.5)
    assert sh["k_push (FP64 final sweep)"] == pytest.approx(0.3)
