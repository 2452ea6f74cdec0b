"""The Hermitian half layout helpers (CPU): sizes, bijection, round trips, and the symmetry itself.

The symmetry A(conj path) = conj(A(path)) is checked on oracle tensors: a
Hermitian rho0 propagated by the oracle's recurrence yields tensors with it,
for the two-level (M = 2) and the three-level (M = 3) system.
"""

import numpy as np
import pytest

import oracle
import oracle.recurrence as rec
from oracle.eta import Spectral
from paper_1205_6872_gb300 import layout as ly


@pytest.mark.parametrize("n", range(0, 8))
def test_canonical_order_is_a_transversal_of_conjugation(n):
    idx = ly.canonical_order(n)
    assert idx.size == ly.canonical_count(n) == (4 ** n + 2 ** n) // 2
    assert np.unique(idx).size == idx.size
    conj = ly.conj_index(np.arange(4 ** n), n)
    assert np.array_equal(conj[conj], np.arange(4 ** n))        # an involution
    canon = np.zeros(4 ** n, bool)
    canon[idx] = True
    # every index is canonical or has a canonical conjugate; both only when self-conjugate
    assert np.all(canon | canon[conj])
    both = canon & canon[conj]
    assert np.array_equal(np.nonzero(both)[0], np.nonzero(conj == np.arange(4 ** n))[0])


@pytest.mark.parametrize("n", range(1, 8))
def test_device_layout_covers_every_index_up_to_conjugation(n):
    idx = ly.canonical_indices(n)
    assert idx.size == ly.count(n) == 2 * 4 ** (n - 1) + 2 ** n
    assert np.unique(idx).size == idx.size
    conj = ly.conj_index(np.arange(4 ** n), n)
    stored = np.zeros(4 ** n, bool)
    stored[idx] = True
    assert np.all(stored | stored[conj])
    # fibers: prefix c occupies entries 4c .. 4c+3, last digits 0..3 in order
    assert np.array_equal(idx.reshape(-1, 4) % 4, np.tile(np.arange(4), (ly.canonical_count(n - 1), 1)))


def test_round_trip():
    rng = np.random.default_rng(0)
    for n in range(0, 6):
        A = ly.symmetrize(rng.normal(size=4 ** n) + 1j * rng.normal(size=4 ** n), n)
        assert np.allclose(ly.from_half(ly.to_half(A, n), n), A)


def test_oracle_tensors_have_the_symmetry():
    s = np.array([1.0, -1.0])
    H = np.array([[0.3, 1.0], [1.0, -0.3]])
    rho0 = np.array([[0.7, 0.2 - 0.3j], [0.2 + 0.3j, 0.3]])
    run = oracle.OracleRun(s, H, Spectral("ohmic_exp", 0.4, 3.0), 1.0, 0.15, 5)
    A = rec.initial_tensor(run.eta, s, rho0)
    for n in range(1, 12):
        G, g, n_in, summed = rec.step_tables(run.eta, s, run.K, 5, n)
        A = rec.apply_step(A, G, g, n_in, summed)
        digits = n_in if summed else n_in + 1
        conj = ly.conj_index(np.arange(4 ** digits), digits)
        assert np.abs(A[conj] - np.conj(A)).max() < 1e-14 * max(1.0, np.abs(A).max()), n


# ---- M = 3: points (a, b) = 3a + b, conjugation (a, b) -> (b, a) swaps 1 <-> 3, 2 <-> 6, 5 <-> 7

@pytest.mark.parametrize("n", range(0, 6))
def test_m3_canonical_order_is_a_transversal_of_conjugation(n):
    idx = ly.canonical_order(n, 3)
    assert idx.size == ly.canonical_count(n, 3) == (9 ** n + 3 ** n) // 2
    assert np.unique(idx).size == idx.size
    conj = ly.conj_index(np.arange(9 ** n), n, 3)
    assert np.array_equal(conj[conj], np.arange(9 ** n))
    canon = np.zeros(9 ** n, bool)
    canon[idx] = True
    assert np.all(canon | canon[conj])
    both = canon & canon[conj]
    assert np.array_equal(np.nonzero(both)[0], np.nonzero(conj == np.arange(9 ** n))[0])


def test_m3_conjugation_digit_map():
    # one digit: the transpose of the 3 x 3 point grid
    assert list(ly.conj_index(np.arange(9), 1, 3)) == [0, 3, 6, 1, 4, 7, 2, 5, 8]
    assert list(ly.canonical_order(1, 3)) == [1, 2, 5, 0, 4, 8]


@pytest.mark.parametrize("n", range(1, 6))
def test_m3_device_layout_covers_every_index_up_to_conjugation(n):
    idx = ly.canonical_indices(n, 3)
    assert idx.size == ly.count(n, 3) == 9 * ((9 ** (n - 1) + 3 ** (n - 1)) // 2)
    assert np.unique(idx).size == idx.size
    conj = ly.conj_index(np.arange(9 ** n), n, 3)
    stored = np.zeros(9 ** n, bool)
    stored[idx] = True
    assert np.all(stored | stored[conj])
    assert np.array_equal(idx.reshape(-1, 9) % 9, np.tile(np.arange(9), (ly.canonical_count(n - 1, 3), 1)))


def test_m3_round_trip():
    rng = np.random.default_rng(1)
    for n in range(0, 5):
        A = ly.symmetrize(rng.normal(size=9 ** n) + 1j * rng.normal(size=9 ** n), n, 3)
        assert np.allclose(ly.from_half(ly.to_half(A, n, 3), n, 3), A)


def test_m3_oracle_tensors_have_the_symmetry():
    from paper_1205_6872_gb300 import workloads as wl
    p = wl.three_level_L8()
    run = oracle.OracleRun(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, 3)
    A = rec.initial_tensor(run.eta, p.s, p.rho0)
    for n in range(1, 7):
        G, g, n_in, summed = rec.step_tables(run.eta, p.s, run.K, 3, n)
        A = rec.apply_step(A, G, g, n_in, summed)
        digits = n_in if summed else n_in + 1
        conj = ly.conj_index(np.arange(9 ** digits), digits, 3)
        assert np.abs(A[conj] - np.conj(A)).max() < 1e-14 * max(1.0, np.abs(A).max()), n
