"""GPU parity at the workloads' full sizes (FP64 form 1e-12, FP32 form 1e-5 max abs on rho).

Expected rho values come from tests/golden/*.json, written by make_golden.py
from the FP64 oracle alone.  At the bench size (4^14 entries) single steps are
also checked element by element on sampled outputs, and the full readout of a
random tensor against the oracle's readout.
"""

import json
import os

import numpy as np
import pytest

import oracle
import oracle.recurrence as rec
from oracle.eta import Spectral
from paper_1205_6872_gb300 import workloads as wl
from test_gpu_parity import _empty_dev, _from_dev, _to_dev, representable

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))

TOL = {64: 1e-12, 32: 1e-5, 48: 1e-12}


def _golden(name):
    path = os.path.join(HERE, "golden", f"{name}.json")
    if not os.path.exists(path):
        pytest.fail(f"missing stored oracle values {path}; run tests/golden/make_golden.py {name}")
    with open(path) as fh:
        return json.load(fh)


def _c(v):
    return np.array([complex(a, b) for a, b in v])


@pytest.fixture(scope="module")
def q():
    assert torch.cuda.is_available()
    from paper_1205_6872_gb300 import quapi
    quapi.load()
    return quapi


@pytest.mark.parametrize("prec", [64, 32, 48])
@pytest.mark.parametrize("name", ["spin_boson_L6", "biased_L12", "three_level_L8", "spin_boson_L14"])
def test_workload_against_stored_oracle(q, name, prec):
    p = wl.CONFIGS[name]()
    g = _golden(name)
    steps = [int(k) for k in g["steps"]]
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(precision=prec))
    try:
        # the device eta must agree with the oracle's before rho can
        eta = q.quapi_get_eta(ctx, p.L)
        assert np.abs(eta - _c(g["eta"])).max() < 1e-14 + 1e-13 * np.abs(eta).max()
        got = q.quapi_propagate(ctx, p.rho0, steps, p.M)
    finally:
        q.quapi_destroy(ctx)
    worst = 0.0
    for i, k in enumerate(steps):
        want = _c(g["rho"][str(k)]).reshape(p.M, p.M)
        worst = max(worst, float(np.abs(got[i] - want).max()))
    print(f"{name} precision {prec}: max |rho_gpu - rho_oracle| over {len(steps)} steps = {worst:.3e}")
    assert worst <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
def test_batched_instances_sequential(q, prec):
    probs = wl.batched_256()
    g = _golden("batched_256")
    worst = 0.0
    for p, rec_ in zip(probs, g["instances"]):
        ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(precision=prec))
        try:
            got = q.quapi_propagate(ctx, p.rho0, [p.N], p.M)[0]
        finally:
            q.quapi_destroy(ctx)
        worst = max(worst, float(np.abs(got - _c(rec_["rho"]).reshape(2, 2)).max()))
    print(f"batched_256 sequential precision {prec}: max abs error = {worst:.3e}")
    assert worst <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32, 48])
@pytest.mark.parametrize("n", [13, 14, 15])
def test_full_size_step_sampled(q, prec, n):
    """Growth into the full tensor (n = 13), the first summing step (n = 14), a steady step (n = 15)."""
    p = wl.spin_boson_L14()
    L, M2 = p.L, 4
    eta = oracle.pack_eta(oracle.eta_table(Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, L))
    etad = oracle.unpack_eta(eta, L)
    K = oracle.pair_propagator_K(oracle.propagator_U(p.H, p.dt))
    n_in = min(n, L)
    A = representable(wl.random_tensor(M2 ** n_in, seed=n), prec)
    G, gg, n_in_o, summed = rec.step_tables(etad, p.s, K, L, n)
    out_size = M2 ** n_in if summed else M2 ** (n_in + 1)
    ctx = q.quapi_setup_eta(p.s, p.H, eta, p.dt, L, q.quapi_opts_init(precision=prec))
    try:
        dA = _to_dev(A, prec)
        dout = _empty_dev(out_size, prec)
        q.quapi_step_device(ctx, n, dA, dout, None)
        torch.cuda.synchronize()
        rng = np.random.Generator(np.random.PCG64(5))
        idx = np.concatenate([np.arange(64), out_size - 1 - np.arange(64), rng.integers(0, out_size, 2048)])
        got = _from_dev(dout[torch.from_numpy(idx).cuda()], prec)
    finally:
        q.quapi_destroy(ctx)
    want = rec.step_elements(A, G, gg, n_in_o, summed, idx)
    scale = np.abs(want).max() + 1.0
    tol = 2e-6 if prec == 32 else 1e-13
    assert np.abs(got - want).max() <= tol * scale


@pytest.mark.parametrize("prec", [64, 32, 48])
def test_full_size_readout(q, prec):
    """rho read out of a random 4^14-entry tensor (steady state, end-point tables) vs the oracle."""
    p = wl.spin_boson_L14()
    L, M2 = p.L, 4
    eta = oracle.pack_eta(oracle.eta_table(Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, L))
    etad = oracle.unpack_eta(eta, L)
    K = oracle.pair_propagator_K(oracle.propagator_U(p.H, p.dt))
    A = representable(wl.random_tensor(M2 ** L, seed=21), prec)
    n = L + 3
    ctx = q.quapi_setup_eta(p.s, p.H, eta, p.dt, L, q.quapi_opts_init(precision=prec))
    try:
        dA = _to_dev(A, prec)
        rho = torch.zeros(M2, dtype=torch.complex128, device="cuda")
        q.quapi_step_device(ctx, n, dA, None, rho)
        torch.cuda.synchronize()
        got = rho.cpu().numpy()
    finally:
        q.quapi_destroy(ctx)
        del dA
    Gr, gr, n_in = rec.readout_tables(etad, p.s, K, L, n)
    want = rec.apply_readout(A, Gr, gr, n_in)
    # random-sign sum of 4^15 terms: relative rounding error ~ eps * sqrt(#terms) of the term scale
    term = np.sqrt(np.mean(np.abs(A) ** 2))
    tol = (1e-6 if prec == 32 else 1e-14) * term * np.sqrt(M2 ** (L + 1)) + 1e-12 * np.abs(want).max()
    assert np.abs(got - want).max() <= tol, (got, want)


def test_full_size_invariants_fp32(q):
    p = wl.spin_boson_L14()
    steps = [0, 1, 7, 14, 15, 100, 500, 1000]
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(precision=32))
    try:
        got = q.quapi_propagate(ctx, p.rho0, steps, p.M)
    finally:
        q.quapi_destroy(ctx)
    for r in got:
        assert abs(np.trace(r) - 1.0) < 1e-5
        assert np.abs(r - r.conj().T).max() < 1e-5


def test_maximum_size_memory_length_16(q):
    """dkmax = 16 (4^16 = 4.3 G entries, > 2^31): full layout FP32 (69 GB of tensors), half layout FP32
    and half layout DF64 agree with each other and keep the trace and Hermiticity invariants."""
    p = wl.spin_boson_L14()
    L, steps = 16, [0, 5, 16, 17, 20]
    res = {}
    for name, prec, half in (("fp32_full", 32, 0), ("fp32_half", 32, 1), ("df64_half", 48, 1)):
        ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, L,
                            q.quapi_opts_init(precision=prec, hermitian=half))
        try:
            res[name] = q.quapi_propagate(ctx, p.rho0, steps, 2)
        finally:
            q.quapi_destroy(ctx)
        torch.cuda.empty_cache()
    for r in res["df64_half"]:
        assert abs(np.trace(r) - 1.0) < 1e-12
        assert np.abs(r - r.conj().T).max() < 1e-12
    for name in ("fp32_full", "fp32_half"):
        assert np.abs(res[name] - res["df64_half"]).max() < 1e-5, name
    # the first steps stay within reach of the oracle's growth phase: check them exactly
    want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, L, p.rho0, [5])[5]
    assert np.abs(res["df64_half"][1] - want).max() < 1e-12
