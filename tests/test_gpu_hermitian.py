"""The Hermitian half layout on the GPU against the oracle (full tensors converted on the host)."""

import json
import os

import numpy as np
import pytest

import oracle
import oracle.recurrence as rec
from oracle.eta import Spectral
from paper_1205_6872_gb300 import layout as ly
from paper_1205_6872_gb300 import workloads as wl
from test_gpu_parity import _empty_dev, _from_dev, _to_dev, representable

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {64: 1e-12, 32: 1e-5, 48: 1e-12}


@pytest.fixture(scope="module")
def q():
    assert torch.cuda.is_available()
    from paper_1205_6872_gb300 import quapi
    quapi.load()
    return quapi


S2 = np.array([1.0, -1.0])
H2 = np.array([[0.5, 1.0], [1.0, -0.5]], complex)


@pytest.mark.parametrize("prec", [64, 32, 48])
@pytest.mark.parametrize("L,n", [(6, 1), (6, 3), (6, 5), (6, 6), (6, 7), (1, 1), (1, 4), (2, 2), (9, 9), (9, 25),
                                 (10, 12), (11, 11), (11, 14)])
def test_half_layout_single_step(q, L, n, prec):
    eta = wl.random_eta(L, seed=300 + L + n)
    etad = oracle.unpack_eta(eta, L)
    K = oracle.pair_propagator_K(oracle.propagator_U(H2, 0.1))
    n_in = min(n, L)
    A = ly.symmetrize(wl.random_tensor(4 ** n_in, seed=n + 7 * L), n_in)
    A = ly.from_half(representable(ly.to_half(A, n_in), prec), n_in)  # what the device stores
    G, g, _, summed = rec.step_tables(etad, S2, K, L, n)
    want = rec.apply_step(A, G, g, n_in, summed)
    out_digits = n_in if summed else n_in + 1
    Gr, gr, _ = rec.readout_tables(etad, S2, K, L, n)
    want_rho = rec.apply_readout(A, Gr, gr, n_in)
    ctx = q.quapi_setup_eta(S2, H2, eta, 0.1, L, q.quapi_opts_init(precision=prec, hermitian=1))
    try:
        dA = _to_dev(ly.to_half(A, n_in), prec)
        dout = _empty_dev(ly.count(out_digits), prec)
        drho = torch.zeros(4, dtype=torch.complex128, device="cuda")
        q.quapi_step_device(ctx, n, dA, dout, drho)
        drho2 = torch.zeros(4, dtype=torch.complex128, device="cuda")
        q.quapi_readout_static(ctx, n, dA, drho2)
        torch.cuda.synchronize()
        got = _from_dev(dout, prec)
        got_rho, got_rho2 = drho.cpu().numpy(), drho2.cpu().numpy()
    finally:
        q.quapi_destroy(ctx)
    scale = np.abs(want).max() + 1.0
    tol = 2e-6 if prec == 32 else 1e-13
    assert np.abs(got - ly.to_half(want, out_digits)).max() <= tol * scale
    rtol = (1e-6 if prec == 32 else 1e-13) * max(1.0, np.abs(want_rho).max())
    assert np.abs(got_rho - want_rho).max() <= rtol
    assert np.abs(got_rho2 - got_rho).max() <= rtol


@pytest.mark.parametrize("prec", [64, 32, 48])
def test_half_layout_propagation_small(q, prec):
    p = wl.spin_boson_L6()
    rho0 = np.array([[0.7, 0.2 - 0.3j], [0.2 + 0.3j, 0.3]])
    steps = [0, 1, 2, 5, 6, 7, 30, 100]
    want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, rho0, steps)
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                        q.quapi_opts_init(precision=prec, hermitian=1))
    try:
        got = q.quapi_propagate(ctx, rho0, steps, 2)
        with pytest.raises(q.QuapiError) as e:
            q.quapi_propagate(ctx, np.array([[1, 1j], [1j, 0]]), steps, 2)   # not Hermitian
        assert e.value.status == q.QUAPI_ERR_ARG
    finally:
        q.quapi_destroy(ctx)
    for i, k in enumerate(steps):
        assert np.abs(got[i] - want[k]).max() <= TOL[prec], k


@pytest.mark.parametrize("prec", [64, 32, 48])
@pytest.mark.parametrize("endpoint", [0, 1])
def test_half_layout_every_step_both_endpoints(q, endpoint, prec):
    """Readout at every step (the paper's allPoints), growth included, in both end-point modes."""
    p = wl.spin_boson_L6()
    steps = list(range(p.N + 1))
    want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, steps,
                            endpoint="strang" if endpoint == 0 else "interior")
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                        q.quapi_opts_init(precision=prec, hermitian=1, endpoint_mode=endpoint))
    try:
        got = q.quapi_propagate(ctx, p.rho0, steps, 2)
    finally:
        q.quapi_destroy(ctx)
    err = max(float(np.abs(got[i] - want[k]).max()) for i, k in enumerate(steps))
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", [64, 32, 48])
def test_half_layout_biased_workload_against_stored_oracle(q, prec):
    """Biased spin-boson (memory length 12, 400 steps, bias 0.5) in the half layout."""
    p = wl.biased_L12()
    with open(os.path.join(HERE, "golden", "biased_L12.json")) as fh:
        g = json.load(fh)
    steps = [int(k) for k in g["steps"]]
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                        q.quapi_opts_init(precision=prec, hermitian=1))
    try:
        got = q.quapi_propagate(ctx, p.rho0, steps, 2)
    finally:
        q.quapi_destroy(ctx)
    worst = max(float(np.abs(got[i] - np.array([complex(a, b) for a, b in g["rho"][str(k)]]).reshape(2, 2)).max())
                for i, k in enumerate(steps))
    print(f"biased_L12 half layout precision {prec}: max abs error vs oracle = {worst:.3e}")
    assert worst <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32, 48])
def test_half_layout_bench_workload_against_stored_oracle(q, prec):
    p = wl.spin_boson_L14()
    with open(os.path.join(HERE, "golden", "spin_boson_L14.json")) as fh:
        g = json.load(fh)
    steps = [int(k) for k in g["steps"]]
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                        q.quapi_opts_init(precision=prec, hermitian=1))
    try:
        got = q.quapi_propagate(ctx, p.rho0, steps, 2)
    finally:
        q.quapi_destroy(ctx)
    worst = max(float(np.abs(got[i] - np.array([complex(a, b) for a, b in g["rho"][str(k)]]).reshape(2, 2)).max())
                for i, k in enumerate(steps))
    print(f"spin_boson_L14 half layout precision {prec}: max abs error vs oracle = {worst:.3e}")
    assert worst <= TOL[prec]


def test_half_layout_checkpoint_and_rejections(q):
    p = wl.spin_boson_L6()
    c1 = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(hermitian=1))
    c2 = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(hermitian=1))
    try:
        q.quapi_propagate(c1, p.rho0, [12], 2)
        n, state = q.quapi_get_state(c1)
        assert n == 11 and state.nbytes == 16 * ly.count(6)
        q.quapi_set_state(c2, n, state)
        a = q.quapi_propagate_resume(c1, [40], 2)
        b = q.quapi_propagate_resume(c2, [40], 2)
        assert np.array_equal(a, b)
        bad = np.array(p.rho0, dtype=np.complex128).reshape(2, 2).copy()
        bad[0, 1] += 0.1j  # no longer Hermitian: the half layout cannot hold its tensor
        with pytest.raises(q.QuapiError) as e:
            q.quapi_propagate_batch([c1], [bad], [10])
        assert e.value.status == q.QUAPI_ERR_ARG
    finally:
        q.quapi_destroy(c1)
        q.quapi_destroy(c2)
    # the three-level half layout needs a Hermitian rho0 too (batched form)
    c3 = q.quapi_setup([-1, 0, 1], np.eye(3), "ohmic_exp", 0.1, 5.0, 1.0, 0.1, 3, q.quapi_opts_init(hermitian=1))
    try:
        with pytest.raises(q.QuapiError) as e:
            q.quapi_propagate_batch([c3], [np.array([[1, 1j, 0], [1j, 0, 0], [0, 0, 0]])], [4], M=3)
        assert e.value.status == q.QUAPI_ERR_ARG
    finally:
        q.quapi_destroy(c3)


def _random_half_tensor(L, seed, prec):
    """A random tensor with the Hermitian symmetry, in the device half layout (self-conjugate prefixes
    get real entries at digits 0 and 3 and conjugate entries at 1 and 2), representable in prec."""
    Ah = wl.random_tensor(ly.count(L), seed=seed)
    pref = ly.canonical_order(L - 1)
    lo_bits = pref & int("01" * (L - 1), 2)
    hi_bits = (pref & int("10" * (L - 1), 2)) >> 1
    sc = np.nonzero(lo_bits == hi_bits)[0]  # every digit 0 or 3
    Ah[4 * sc] = Ah[4 * sc].real
    Ah[4 * sc + 3] = Ah[4 * sc + 3].real
    Ah[4 * sc + 2] = np.conj(Ah[4 * sc + 1])
    return representable(Ah, prec)


@pytest.mark.parametrize("prec", [32, 64, 48])
def test_half_layout_full_size_step_sampled(q, prec):
    """The headline configuration (memory length 14, steady step, half layout) launched as bench.py
    times it: sampled outputs of one step, and the full end-point readout, against the oracle."""
    p = wl.spin_boson_L14()
    L, n = p.L, p.L + 1
    eta = oracle.pack_eta(oracle.eta_table(Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, L))
    etad = oracle.unpack_eta(eta, L)
    K = oracle.pair_propagator_K(oracle.propagator_U(p.H, p.dt))
    Ah = _random_half_tensor(L, seed=77, prec=prec)
    A = ly.from_half(Ah, L)
    np.testing.assert_array_equal(ly.to_half(A, L), Ah)
    G, gg, n_in, summed = rec.step_tables(etad, p.s, K, L, n)
    ctx = q.quapi_setup_eta(p.s, p.H, eta, p.dt, L, q.quapi_opts_init(precision=prec, hermitian=1))
    try:
        dA = _to_dev(Ah, prec)
        dout = _empty_dev(ly.count(L), prec)
        q.quapi_step_device(ctx, n, dA, dout, None)
        rho = torch.zeros(4, dtype=torch.complex128, device="cuda")
        q.quapi_step_device(ctx, L + 3, dA, None, rho)
        torch.cuda.synchronize()
        rng = np.random.Generator(np.random.PCG64(9))
        cnt = ly.count(L)
        pos = np.concatenate([np.arange(64), cnt - 1 - np.arange(64), rng.integers(0, cnt, 2048)])
        got = _from_dev(dout[torch.from_numpy(pos).cuda()], prec)
        got_rho = rho.cpu().numpy()
    finally:
        q.quapi_destroy(ctx)
        del dA
    full_idx = ly.canonical_indices(L)[pos]
    want = rec.step_elements(A, G, gg, n_in, summed, full_idx)
    tol = 2e-6 if prec == 32 else 1e-13
    assert np.abs(got - want).max() <= tol * (np.abs(want).max() + 1.0)
    Gr, gr, n_in_r = rec.readout_tables(etad, p.s, K, L, L + 3)
    want_rho = rec.apply_readout(A, Gr, gr, n_in_r)
    term = np.sqrt(np.mean(np.abs(A) ** 2))
    rtol = (1e-6 if prec == 32 else 1e-14) * term * np.sqrt(4 ** (L + 1)) + 1e-12 * np.abs(want_rho).max()
    assert np.abs(got_rho - want_rho).max() <= rtol, (got_rho, want_rho)
    # the Hermitian layout's readout is Hermitian by construction
    assert abs(got_rho[1] - np.conj(got_rho[2])) <= 1e-12 * max(1.0, abs(got_rho[1]))
