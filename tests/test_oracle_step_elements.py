"""Pin of the oracle's per-entry step checker ``oracle.recurrence.step_elements`` (CPU only).

``step_elements`` evaluates chosen output entries of one tensor-propagator step
on their own (plain Python loops over the digits of the output index).  The GPU
tests at full size (memory length 14, where the oracle cannot run whole steps
inside a test) check sampled outputs against it, so it is pinned here against
``apply_step`` -- the oracle's whole-tensor step, itself pinned by the explicit
sum over every forward/backward path and by the closed forms -- on EVERY output
index: growth steps (n < L, no summed digit), the first summing step (n = L,
the point-0 eta joins the oldest digit) and steady steps (n > L), for M = 2 and
M = 3.  A digit-order slip, a dropped self factor or a wrong summed-digit table
in either function changes some outputs and fails here.
"""

import numpy as np
import pytest

from oracle import recurrence as rec
from oracle.eta import unpack_eta
from oracle.system import pair_propagator_K, propagator_U
from paper_1205_6872_gb300 import workloads as wl


def _system(M, seed):
    if M == 2:
        return np.array([1.0, -1.0]), np.array([[0.3, 1.0], [1.0, -0.3]], dtype=complex)
    return np.array([-1.0, 0.0, 1.0]), wl.random_hermitian(3, seed)


CASES = [(2, L, n) for L in range(1, 7) for n in sorted({1, max(1, L - 1), L, L + 1, L + 3})]
CASES += [(3, L, n) for L in (1, 2, 3, 4) for n in sorted({1, max(1, L - 1), L, L + 2})]


@pytest.mark.parametrize("M,L,n", CASES)
def test_step_elements_equals_apply_step_everywhere(M, L, n):
    s, H = _system(M, 40 + L)
    eta = unpack_eta(wl.random_eta(L, seed=100 * M + 10 * L + n, scale=0.2), L)
    K = pair_propagator_K(propagator_U(H, 0.2))
    G, g, n_in, summed = rec.step_tables(eta, s, K, L, n)
    A = wl.random_tensor((M * M) ** n_in, seed=7 * n + L)
    whole = rec.apply_step(A, G, g, n_in, summed)
    assert summed == (n >= L)
    assert whole.size == (M * M) ** (n_in + (0 if summed else 1))
    got = rec.step_elements(A, G, g, n_in, summed, range(whole.size))
    scale = max(1.0, float(np.abs(whole).max()))
    assert np.abs(got - whole).max() <= 1e-13 * scale


def test_step_elements_sees_a_planted_digit_swap():
    # the check above has teeth: swapping two kept digits of the index changes the outputs
    M, L, n = 2, 4, 6
    s, H = _system(M, 3)
    eta = unpack_eta(wl.random_eta(L, seed=5, scale=0.2), L)
    K = pair_propagator_K(propagator_U(H, 0.2))
    G, g, n_in, summed = rec.step_tables(eta, s, K, L, n)
    A = wl.random_tensor((M * M) ** n_in, seed=9)
    whole = rec.apply_step(A, G, g, n_in, summed)
    Gs = G.copy()
    Gs[[1, 2]] = G[[2, 1]]  # digits 1 and 2 exchanged: a plausible indexing mistake
    wrong = rec.step_elements(A, Gs, g, n_in, summed, range(whole.size))
    assert np.abs(wrong - whole).max() > 1e-3
