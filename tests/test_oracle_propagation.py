"""Pins for the oracle's tensor-propagator recurrence (CPU only).

* J = 0: exact unitary evolution e^{-iHt} rho0 e^{iHt} (two-level closed form;
  scipy's Pade expm for M = 3), for any dt and memory length.
* Brute force: the explicit sum over every forward/backward path, with eta
  taken per box pair of that path, equals the recurrence for L < N and L >= N,
  M = 2 and 3, both endpoint treatments.
* Pure dephasing (diagonal H): the independent-boson closed form with the
  closed-form Ohmic eta (no quadrature), for L >= N and L < N.
* Invariants: Tr rho = Tr rho0 and rho = rho^dagger at every step.
* Primary memory cost: Table 1's PMC column against 64 M^{2(L+1)} bytes.
"""

import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle.eta import Spectral
from closed_forms import U_two_level, pure_dephasing_rho
from paper_1205_6872_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
ZERO = Spectral("ohmic_exp", 0.0, 5.0)


@pytest.mark.parametrize("eps,W", [(0.0, 1.0), (0.5, 1.0), (-0.3, 0.7)])
@pytest.mark.parametrize("L", [1, 3, 6])
def test_zero_coupling_is_unitary(eps, W, L):
    dt = 0.25
    H = np.array([[eps, W], [W, -eps]])
    rho0 = np.array([[0.7, 0.2 - 0.1j], [0.2 + 0.1j, 0.3]])
    steps = [0, 1, 2, L, L + 1, 3 * L + 2, 40]
    got = oracle.propagate([1, -1], H, ZERO, 1.0, dt, L, rho0, steps)
    for k in steps:
        U = U_two_level(eps, W, k * dt)
        want = U @ rho0 @ U.conj().T
        assert np.abs(got[k] - want).max() < 1e-13, k


def test_zero_coupling_spin_boson_closed_form():
    # rho0 = |0><0|, H = [[0,1],[1,0]]: rho00 = cos^2 t, rho01 = (i/2) sin 2t
    got = oracle.propagate([1, -1], [[0, 1], [1, 0]], ZERO, 5.0, 0.25, 6, [[1, 0], [0, 0]],
                           list(range(0, 101, 7)))
    for k, r in got.items():
        t = 0.25 * k
        assert abs(r[0, 0] - math.cos(t) ** 2) < 1e-13
        assert abs(r[0, 1] - 0.5j * math.sin(2 * t)) < 1e-13


def test_zero_coupling_three_level():
    H = wl.random_hermitian(3, 1205)
    rho0 = wl.random_pure_state(3, 6872)
    dt = 0.2
    got = oracle.propagate([-1, 0, 1], H, Spectral("superohmic_gauss", 0.0, 2.0), 2.0, dt, 3,
                           rho0, [0, 1, 3, 4, 17])
    for k, r in got.items():
        U = scipy.linalg.expm(-1j * H * k * dt)
        assert np.abs(r - U @ rho0 @ U.conj().T).max() < 1e-12, k


BF_CASES = [
    # (M, L, N, endpoint)
    (2, 1, 4, "strang"), (2, 2, 5, "strang"), (2, 3, 3, "strang"), (2, 5, 4, "strang"),
    (2, 4, 7, "strang"), (2, 2, 6, "interior"), (2, 6, 5, "interior"),
    (3, 2, 4, "strang"), (3, 4, 3, "strang"), (3, 1, 3, "interior"),
]


@pytest.mark.parametrize("M,L,N,endpoint", BF_CASES)
def test_recurrence_equals_brute_force(M, L, N, endpoint):
    if M == 2:
        H = np.array([[0.5, 1.0], [1.0, -0.5]])
        s = [1.0, -1.0]
        spec, beta, dt = Spectral("ohmic_exp", 0.3, 5.0), 1.0, 0.1
        rho0 = np.array([[1, 0], [0, 0]], dtype=complex)
    else:
        H = wl.random_hermitian(3, 7)
        s = [-1.0, 0.0, 1.0]
        spec, beta, dt = Spectral("superohmic_gauss", 0.05, 2.0), 2.0, 0.2
        rho0 = wl.random_pure_state(3, 8)
    rec = oracle.propagate(s, H, spec, beta, dt, L, rho0, list(range(N + 1)), endpoint=endpoint)
    for n in range(N + 1):
        bf = oracle.rho_bruteforce(s, H, spec, beta, dt, L, rho0, n, endpoint=endpoint)
        assert np.abs(rec[n] - bf).max() < 1e-13, (n, rec[n], bf)


def test_brute_force_distinguishes_endpoint_treatments():
    # the Strang and interior readouts differ once the bath is on
    H = np.array([[0.0, 1.0], [1.0, 0.0]])
    spec = Spectral("ohmic_exp", 0.5, 2.5)
    a = oracle.rho_bruteforce([1, -1], H, spec, 0.5, 0.15, 3, np.diag([1.0, 0.0]), 4, "strang")
    b = oracle.rho_bruteforce([1, -1], H, spec, 0.5, 0.15, 3, np.diag([1.0, 0.0]), 4, "interior")
    assert np.abs(a - b).max() > 1e-4


@pytest.mark.parametrize("L,N", [(6, 4), (6, 6), (2, 7), (3, 12), (1, 5)])
@pytest.mark.parametrize("beta", [math.inf, 1.0])
def test_pure_dephasing_closed_form(L, N, beta):
    a, wc, dt = 0.3, 5.0, 0.1
    E = np.array([0.4, -0.25])
    s = [1.0, -1.0]
    rho0 = np.array([[0.6, 0.3 + 0.2j], [0.3 - 0.2j, 0.4]])
    spec = Spectral("ohmic_exp", a, wc)
    got = oracle.propagate(s, np.diag(E), spec, beta, dt, L, rho0, list(range(N + 1)))
    for n in range(N + 1):
        want = pure_dephasing_rho(s, E, rho0, a, wc, beta, dt, L, n)
        assert np.abs(got[n] - want).max() < 1e-13, (n, got[n], want)


def test_pure_dephasing_three_level():
    a, wc, dt, beta = 0.2, 3.0, 0.2, 2.0
    E = np.array([0.3, -0.1, 0.5])
    s = [-1.0, 0.0, 1.0]
    rho0 = wl.random_pure_state(3, 11)
    got = oracle.propagate(s, np.diag(E), Spectral("ohmic_exp", a, wc), beta, dt, 3, rho0, [1, 2, 3, 6])
    for n, r in got.items():
        assert np.abs(r - pure_dephasing_rho(s, E, rho0, a, wc, beta, dt, 3, n)).max() < 1e-13


@pytest.mark.parametrize("name", ["spin_boson_L6"])
def test_invariants_full_run(name):
    p = wl.CONFIGS[name]()
    got = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0,
                           range(p.N + 1))
    for k, r in got.items():
        assert abs(np.trace(r) - 1.0) < 1e-13, k
        assert np.abs(r - r.conj().T).max() < 1e-13, k


def test_invariants_three_level_short():
    p = wl.three_level_L8()
    got = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, 4, p.rho0,
                           range(0, 13))
    for k, r in got.items():
        assert abs(np.trace(r) - 1.0) < 1e-13, k
        assert np.abs(r - r.conj().T).max() < 1e-13, k


def test_primary_memory_cost_table1():
    # Table 1 (Sec. IV): PMC column, M = 2; Eq. primaryMemoryCost: 64 M^{2(L+1)} bytes
    rows = []
    with open(os.path.join(HERE, "golden", "table1_pmc.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                L, val, unit = line.split()
                rows.append((int(L), float(val), unit))
    scale = {"KB": 1e3, "MB": 1e6, "GB": 1e9}
    for L, val, unit in rows:
        pmc = 64 * 2 ** (2 * (L + 1))
        printed = val * scale[unit]
        assert abs(pmc - printed) / pmc < 1e-3, (L, pmc, printed)
