"""The Hermitian half layout of the three-level system (M = 3) on the GPU against the oracle.

Points x = 3a + b; conjugation (a, b) -> (b, a) swaps 1 <-> 3, 2 <-> 6, 5 <-> 7.  Full tensors are
converted on the host (paper_1205_6872_gb300.layout with M = 3, whose order and the symmetry itself
are pinned in test_layout.py); single steps are compared element by element with the oracle's step,
and whole propagations with the oracle's rho (the three-level workload against its stored 300-step
run).
"""

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
S3 = np.array([-1.0, 0.0, 1.0])


@pytest.fixture(scope="module")
def q():
    assert torch.cuda.is_available()
    from paper_1205_6872_gb300 import quapi
    quapi.load()
    return quapi


S3_UNEVEN = np.array([-1.0, 0.3, 1.0])  # unequally spaced: rows 1 and 5 (and 3 and 7) differ


@pytest.mark.parametrize("prec", [64, 32, 48])
@pytest.mark.parametrize("L,n,uneven", [(4, 1, 0), (4, 2, 0), (4, 3, 0), (4, 4, 0), (4, 5, 0), (4, 11, 0), (1, 1, 0),
                                        (1, 3, 0), (2, 2, 0), (6, 6, 0), (6, 9, 0), (7, 8, 0),
                                        (4, 3, 1), (4, 5, 1), (6, 9, 1), (7, 8, 1)])
def test_m3_half_layout_single_step(q, L, n, uneven, prec):
    s3 = S3_UNEVEN if uneven else S3
    H = wl.random_hermitian(3, 50 + L)
    eta = wl.random_eta(L, seed=400 + L + n)
    etad = oracle.unpack_eta(eta, L)
    K = oracle.pair_propagator_K(oracle.propagator_U(H, 0.2))
    n_in = min(n, L)
    A = ly.symmetrize(wl.random_tensor(9 ** n_in, seed=n + 11 * L), n_in, 3)
    A = ly.from_half(representable(ly.to_half(A, n_in, 3), prec), n_in, 3)  # what the device stores
    G, g, _, summed = rec.step_tables(etad, s3, K, L, n)
    want = rec.apply_step(A, G, g, n_in, summed)
    out_digits = n_in if summed else n_in + 1
    Gr, gr, _ = rec.readout_tables(etad, s3, K, L, n)
    want_rho = rec.apply_readout(A, Gr, gr, n_in)
    ctx = q.quapi_setup_eta(s3, H, eta, 0.2, L, q.quapi_opts_init(precision=prec, hermitian=1))
    try:
        dA = _to_dev(ly.to_half(A, n_in, 3), prec)
        dout = _empty_dev(ly.count(out_digits, 3), prec)
        drho = torch.zeros(9, dtype=torch.complex128, device="cuda")
        q.quapi_step_device(ctx, n, dA, dout, drho)
        drho2 = torch.zeros(9, dtype=torch.complex128, device="cuda")
        q.quapi_step_device(ctx, n, dA, None, drho2)   # the readout alone
        torch.cuda.synchronize()
        got = _from_dev(dout, prec)
        got_rho, got_rho2 = drho.cpu().numpy(), drho2.cpu().numpy()
    finally:
        q.quapi_destroy(ctx)
    scale = np.abs(want).max() + 1.0
    tol = 2e-6 if prec == 32 else 1e-13
    assert np.abs(got - ly.to_half(want, out_digits, 3)).max() <= tol * scale
    rtol = (1e-6 if prec == 32 else 1e-13) * max(1.0, np.abs(want_rho).max())
    assert np.abs(got_rho - want_rho).max() <= rtol
    assert np.abs(got_rho2 - want_rho).max() <= rtol


@pytest.mark.parametrize("prec", [64, 32, 48])
@pytest.mark.parametrize("endpoint", [0, 1])
def test_m3_half_layout_every_step(q, endpoint, prec):
    """rho at every step (growth included) of a three-level run, both end-point treatments."""
    p = wl.three_level_L8()
    L, N = 4, 24
    steps = list(range(N + 1))
    want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, L, p.rho0, steps,
                            endpoint="strang" if endpoint == 0 else "interior")
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, L,
                        q.quapi_opts_init(precision=prec, hermitian=1, endpoint_mode=endpoint))
    try:
        got = q.quapi_propagate(ctx, p.rho0, steps, 3)
    finally:
        q.quapi_destroy(ctx)
    err = max(float(np.abs(got[i] - want[k]).max()) for i, k in enumerate(steps))
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", [64, 32, 48])
def test_m3_half_layout_workload_against_stored_oracle(q, prec):
    """The three-level workload (memory length 8, 43 M entries in the full layout, 300 steps)."""
    p = wl.three_level_L8()
    with open(os.path.join(HERE, "golden", "three_level_L8.json")) as fh:
        g = json.load(fh)
    steps = [int(k) for k in g["steps"]]
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                        q.quapi_opts_init(precision=prec, hermitian=1))
    try:
        got = q.quapi_propagate(ctx, p.rho0, steps, 3)
    finally:
        q.quapi_destroy(ctx)
    worst = max(float(np.abs(got[i] - np.array([complex(a, b) for a, b in g["rho"][str(k)]]).reshape(3, 3)).max())
                for i, k in enumerate(steps))
    print(f"three_level_L8 half layout precision {prec}: max abs error vs oracle = {worst:.3e}")
    assert worst <= TOL[prec]


def test_m3_half_layout_checkpoint_round_trip(q):
    p = wl.three_level_L8()
    L = 5
    opts = q.quapi_opts_init(precision=64, hermitian=1)
    a = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, L, opts)
    b = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, L, opts)
    try:
        whole = q.quapi_propagate(a, p.rho0, [17], 3)[0]
        q.quapi_propagate(b, p.rho0, [9], 3)
        n, state = q.quapi_get_state(b)
        assert n == 8 and state.nbytes == ly.count(L, 3) * 16
        q.quapi_set_state(b, n, state)
        resumed = q.quapi_propagate_resume(b, [17], 3)[0]
    finally:
        q.quapi_destroy(a)
        q.quapi_destroy(b)
    assert np.abs(resumed - whole).max() <= 1e-13


@pytest.mark.parametrize("prec", [64, 32, 48])
def test_m3_half_layout_batched_against_oracle(q, prec):
    """Three-level instances in the half layout through the batched launch: memory lengths 2..6 (the
    smallest stay in shared memory), final steps in the growth phase, at the first summing step and
    beyond; each rho(t_N) against the oracle."""
    probs, Ns = [], [5, 2, 9, 4, 14, 6, 11]
    for i, L in enumerate([2, 3, 4, 4, 5, 6, 6]):
        p = wl.three_level_L8()
        p.L = L
        p.H = wl.random_hermitian(3, 70 + i)
        probs.append(p)
    ctxs = [q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                          q.quapi_opts_init(precision=prec, hermitian=1)) for p in probs]
    try:
        for rep in range(2):  # the second call replays the captured graph
            got = q.quapi_propagate_batch(ctxs, [p.rho0 for p in probs], Ns, M=3)
            for p, N, r in zip(probs, Ns, got):
                want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, [N])[N]
                assert np.abs(r - want).max() <= TOL[prec], (p.L, N, rep)
    finally:
        for c in ctxs:
            q.quapi_destroy(c)
