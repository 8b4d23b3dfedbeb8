"""The bench's shared-memory and roofline models on CPU: the bank-conflict
constants against a Monte Carlo of random lattice reads, the scaling of the
captured DRAM traffic by the pair count with its source-hash guard, and the
mirror / near-kernel rooflines."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def expected_max_load(balls, bins, trials, rng):
    """Mean of the largest bin count when `balls` land uniformly in `bins`."""
    hits = rng.integers(bins, size=(trials, balls))
    counts = np.zeros((trials, bins), dtype=np.int32)
    np.add.at(counts, (np.repeat(np.arange(trials), balls), hits.ravel()), 1)
    return counts.max(axis=1).mean()


def test_random_wavefront_constants():
    # a warp's random 16-byte reads: 4 phases of 8 lanes over 8 groups of 4 banks;
    # 8-byte: 2 phases of 16 lanes over 16 bank pairs; 4-byte: 32 lanes over 32 banks
    # (lattices have thousands of cells, so two lanes rarely share an address)
    rng = np.random.default_rng(7)
    assert abs(bench.RANDOM_WAVEFRONTS[16] / 4 - expected_max_load(8, 8, 200000, rng)) < 0.01
    assert abs(bench.RANDOM_WAVEFRONTS[8] / 2 - expected_max_load(16, 16, 200000, rng)) < 0.01
    assert abs(bench.RANDOM_WAVEFRONTS[4] - expected_max_load(32, 32, 200000, rng)) < 0.01


def test_traffic_scaled_by_pairs_and_guarded_by_hash(monkeypatch):
    src = bench.TRAFFIC_SCALED_FROM["cube_3lambda_49152tri_73728rwg_4pt_fp32"]
    b, n = bench.TRAFFIC[src]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: bench.TRAFFIC_HASH)
    assert bench.kernel_traffic(src, n) == b
    assert abs(bench.kernel_traffic("cube_3lambda_49152tri_73728rwg_4pt_fp32", 16 * n) - 16 * b) < 1e-6 * b
    assert bench.kernel_traffic("unknown", n) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.kernel_traffic(src, n) is None  # the kernel changed since the capture


def test_other_kernel_rooflines(monkeypatch):
    pk = {"hbm_gbs": 6000.0}
    monkeypatch.setattr(bench, "near_source_hash", lambda: bench.NEAR_FP64_OPS_HASH)
    r = bench.other_kernel_rooflines("w", 1e9, 1.0, 2.0, 1000, pk, 2000.0)
    assert abs(r["mirror"]["achieved"] - 2e9 / 1e-3 / 1e9) < 1e-9 and abs(r["mirror"]["frac"] - 2000 / 6000) < 1e-12
    peak = bench.SM_COUNT * bench.FP64_OPS_PER_SM_CLOCK * 2000.0 * 1e6
    assert abs(r["near"]["achieved"] - bench.NEAR_FP64_OPS_PER_TASK * 1000 / 2e-3) < 1e-6
    assert abs(r["near"]["frac"] - r["near"]["achieved"] / peak) < 1e-12
    monkeypatch.setattr(bench, "near_source_hash", lambda: "0" * 16)
    assert bench.other_kernel_rooflines("w", 1e9, 1.0, 2.0, 1000, pk, 2000.0)["near"]["frac"] is None
