"""The benchmark's host-side bookkeeping (CPU): the stored-oracle reader and comparison behind every
``max_abs_vs_oracle``, the per-launch traffic lookup keyed by the kernel sources' hash, and the entry
and byte counts behind ``value``, ``roofline.achieved`` and the batched form's fraction of HBM.
"""

import json
import os

import numpy as np
import pytest

import bench
import oracle
from oracle.eta import Spectral
from paper_1205_6872_gb300 import layout as ly
from paper_1205_6872_gb300 import workloads as wl


def test_golden_reader_against_the_oracle():
    """golden_rho returns the oracle's rho at each stored step (row-major M x M, real and imaginary parts
    in that order): rerun the oracle on the small spin-boson workload and compare entry by entry."""
    p = wl.spin_boson_L6()
    gold = bench.golden_rho("spin_boson_L6")
    steps = sorted(gold)
    assert steps[0] == 0 and steps[-1] == p.N
    want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, steps)
    for k in steps:
        assert gold[k].shape == (2, 2)
        assert np.abs(gold[k] - want[k]).max() <= 1e-13
    # rho is Hermitian, so a transposed reading conjugates the off-diagonal entries: a step where they have
    # an imaginary part makes the comparison above catch it
    assert any(abs(gold[k][0, 1].imag) > 1e-3 for k in steps)


def test_golden_reader_shapes_and_invariants():
    for name in ("spin_boson_L14", "biased_L12", "three_level_L8", "quantum_dot_L11"):
        gold = bench.golden_rho(name)
        assert gold, name
        M = 3 if name.startswith("three") else 2
        for k, r in gold.items():
            assert r.shape == (M, M)
            assert abs(np.trace(r) - 1.0) <= 1e-6, (name, k)
            assert np.abs(r - r.conj().T).max() <= 1e-12, (name, k)
    assert bench.golden_rho("no_such_workload") is None


def test_vs_oracle():
    gold = {3: np.array([[0.5, 0.1 + 0.2j], [0.1 - 0.2j, 0.5]])}
    rho = gold[3] + np.array([[0.0, 1e-3j], [0.0, -2e-3]])
    assert bench.vs_oracle(rho, gold, 3) == pytest.approx(2e-3)
    assert bench.vs_oracle(rho.reshape(-1), gold, 3) == pytest.approx(2e-3)  # flat rho is reshaped
    assert bench.vs_oracle(rho, gold, 4) is None
    assert bench.vs_oracle(rho, None, 3) is None


def test_recorded_traffic_follows_the_source_hash(monkeypatch):
    path = os.path.join(bench.ROOT, "profiles", "traffic_per_launch.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert rows
    sha = bench.kernel_source_sha()
    for key, value, row_sha in rows:
        got = bench.recorded_traffic(key)
        assert got == (float(value) if row_sha == sha else None)
    assert bench.recorded_traffic("no_such_kernel") is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    assert all(bench.recorded_traffic(r[0]) is None for r in rows)


def test_measured_peak():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    peak, kind = bench.measured_peaks()
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_entry_counts():
    p = wl.spin_boson_L14()
    assert bench.tensor_entries(p, False) == 4 ** 14
    # the half layout stores the M^2-entry fiber of every canonical (L-1)-digit prefix: M^2 C(L-1) entries,
    # C(n) = ((M^2)^n + M^n) / 2
    assert bench.tensor_entries(p, True) == 4 * (4 ** 13 + 2 ** 13) // 2 == 2 * 4 ** 13 + 2 ** 14 == ly.count(14, 2)
    q = wl.three_level_L8()
    assert bench.tensor_entries(q, False) == 9 ** 8
    assert bench.tensor_entries(q, True) == 9 * (9 ** 7 + 3 ** 7) // 2 == 21_533_202
    assert bench.element_updates(p) == 4 ** 14 * (1000 - 14 + 1)


def test_batch_bytes():
    """One read and one write per stored entry per step: growth n = 1..L-1 (A_n to A_{n+1}), steady steps
    (A_L to A_L), the final readout (a read only); instances within the resident limit move nothing."""
    p = wl.spin_boson_L6()
    p.L, p.N = 3, 5
    e = 8
    full = (4 + 16) * e + (16 + 64) * e + 2 * 64 * e + 2 * 64 * e + 64 * e
    assert bench.batch_hbm_bytes([p], False, e, resident_bytes=0) == full
    half = [ly.count(n, 2) for n in range(1, 4)]
    want_half = (half[0] + half[1]) * e + (half[1] + half[2]) * e + 2 * half[2] * e + 2 * half[2] * e + half[2] * e
    assert bench.batch_hbm_bytes([p], True, e, resident_bytes=0) == want_half
    assert bench.batch_hbm_bytes([p], False, e) == 0  # 2 x 64 x 8 B fits the 32 KB resident limit
    assert bench.batch_updates([p]) == 64 * 3
