"""The seeded synthetic inputs follow their stated recipes and are reproducible (CPU only)."""

import numpy as np

from paper_1205_6872_gb300 import workloads as wl


def _same(p, q):
    return (p.M == q.M and p.L == q.L and p.N == q.N and p.jkind == q.jkind and p.ja == q.ja and p.wc == q.wc
            and p.beta == q.beta and p.dt == q.dt and np.array_equal(p.s, q.s) and np.array_equal(p.H, q.H)
            and np.array_equal(p.rho0, q.rho0))


def test_configs_are_reproducible():
    for name, make in wl.CONFIGS.items():
        a, b = make(), make()
        if isinstance(a, list):
            assert all(_same(x, y) for x, y in zip(a, b)), name
        else:
            assert _same(a, b), name


def test_config_parameters():
    p = wl.spin_boson_L14()
    assert (p.M, p.L, p.N, p.ja, p.wc, p.beta, p.dt) == (2, 14, 1000, 0.5, 2.5, 0.5, 0.15)
    assert np.array_equal(p.H, np.array([[0, 1], [1, 0]], complex))
    p = wl.biased_L12()
    assert (p.L, p.N, p.ja, p.wc, p.beta, p.dt) == (12, 400, 0.3, 5.0, 1.0, 0.1)
    assert np.array_equal(p.H, np.array([[0.5, 1], [1, -0.5]], complex))
    p = wl.spin_boson_L6()
    assert (p.L, p.N, p.ja, p.wc, p.beta, p.dt) == (6, 100, 0.1, 7.5, 5.0, 0.25)
    p = wl.three_level_L8()
    assert (p.M, p.L, p.N, p.jkind, p.ja, p.wc, p.beta, p.dt) == (3, 8, 300, wl.SUPEROHMIC_GAUSS, 0.05, 2.0, 2.0, 0.2)
    assert np.allclose(p.H, p.H.conj().T)
    assert abs(np.trace(p.rho0) - 1.0) < 1e-14 and np.allclose(p.rho0, p.rho0.conj().T)
    assert np.linalg.matrix_rank(p.rho0) == 1  # a pure state


def test_batched_256_recipe():
    probs = wl.batched_256()
    assert len(probs) == 256
    Ls = np.array([p.L for p in probs])
    assert Ls.min() >= 4 and Ls.max() <= 11 and len(set(Ls)) == 8
    for p in probs:
        assert p.N == 200 and p.dt == 0.25 and p.M == 2
        assert 0.01 <= p.ja <= 0.5 and 1.0 <= p.wc <= 10.0 and 0.2 <= p.beta <= 10.0
        eps = p.H[0, 0].real
        assert -1.0 <= eps <= 1.0 and np.array_equal(p.H, np.array([[eps, 1], [1, -eps]], complex))
    # mean (M^2)^L near the stated 6.99e5
    assert 5e5 < np.mean(4.0 ** Ls) < 9e5


def test_quantum_dot_units():
    p = wl.quantum_dot()
    assert abs(p.beta - 0.3055) < 1e-3            # hbar / (k_B 25 K) in ps
    assert p.jkind == wl.SUPEROHMIC_GAUSS and abs(p.ja - np.pi * 0.027) < 1e-15 and p.wc == 2.2
    assert np.array_equal(p.s, np.array([0.0, 1.0])) and (p.L, p.N) == (11, 1000)
    sweep = wl.pulse_area_sweep(n=8)
    areas = [2 * p.H[0, 1].real * p.N * p.dt for p in sweep]   # Omega t_final
    assert np.allclose(areas, [5 * np.pi * (j + 1) / 8 for j in range(8)])
