"""The paper's own model system (Sec. III, driven quantum dot) on the GPU against the oracle."""

import numpy as np
import pytest

import oracle
from oracle.eta import Spectral
from paper_1205_6872_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    assert torch.cuda.is_available()
    from paper_1205_6872_gb300 import quapi
    quapi.load()
    return quapi


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5)])
def test_quantum_dot_short(q, prec, tol):
    p = wl.quantum_dot(L=7, N=60)
    steps = [0, 1, 5, 7, 8, 30, 60]
    want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, steps)
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(precision=prec))
    try:
        got = q.quapi_propagate(ctx, p.rho0, steps, 2)
    finally:
        q.quapi_destroy(ctx)
    for i, k in enumerate(steps):
        assert np.abs(got[i] - want[k]).max() <= tol, k


def test_pulse_area_sweep_batched(q):
    """rho_11(t_final) against pulse area, one batched launch (the paper's justFinalPoint use case)."""
    probs = wl.pulse_area_sweep(n=8, L=6, N=40)
    ctxs = [q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(precision=64))
            for p in probs]
    try:
        got = q.quapi_propagate_batch(ctxs, [p.rho0 for p in probs], [p.N for p in probs])
    finally:
        for c in ctxs:
            q.quapi_destroy(c)
    for p, r in zip(probs, got):
        want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, [p.N])[p.N]
        assert np.abs(r - want).max() <= 1e-12


# ---- the paper's settings at full size (Sec. IV profiled run: Delta k_max = 11, 1000 steps) against the
# stored oracle values (tests/golden/quantum_dot_L11.json and pulse_area_sweep_64.json, make_golden.py)

import json  # noqa: E402
import os  # noqa: E402

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


@pytest.mark.parametrize("half", [0, 1])
@pytest.mark.parametrize("prec", [64, 32, 48])
def test_quantum_dot_full_size_against_stored_oracle(q, prec, half):
    p = wl.quantum_dot()
    g = _golden("quantum_dot_L11")
    assert (g["L"], g["N"]) == (p.L, p.N) == (11, 1000)
    steps = [int(k) for k in g["steps"]]
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                        q.quapi_opts_init(precision=prec, hermitian=half))
    try:
        eta = q.quapi_get_eta(ctx, p.L)
        assert np.abs(eta - _c(g["eta"])).max() < 1e-14 + 1e-13 * np.abs(eta).max()
        got = q.quapi_propagate(ctx, p.rho0, steps, p.M)
    finally:
        q.quapi_destroy(ctx)
    worst = max(float(np.abs(got[i] - _c(g["rho"][str(k)]).reshape(2, 2)).max()) for i, k in enumerate(steps))
    print(f"quantum_dot_L11 precision {prec} half {half}: max |rho_gpu - rho_oracle| over {len(steps)} steps = "
          f"{worst:.3e}")
    assert worst <= TOL[prec]


@pytest.mark.parametrize("half", [0, 1])
@pytest.mark.parametrize("prec", [64, 32, 48])
def test_pulse_area_sweep_64_batched_against_stored_oracle(q, prec, half):
    """64 pulse areas at Delta k_max = 11, rho at t_final only (justFinalPoint), one batched launch."""
    g = _golden("pulse_area_sweep_64")
    probs = wl.pulse_area_sweep(n=64, L=g["L"], N=g["N"])
    ctxs = [q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                          q.quapi_opts_init(precision=prec, hermitian=half)) for p in probs]
    try:
        got = q.quapi_propagate_batch(ctxs, [p.rho0 for p in probs], [p.N for p in probs])
    finally:
        for c in ctxs:
            q.quapi_destroy(c)
    worst = max(float(np.abs(r - _c(inst["rho"]).reshape(2, 2)).max()) for r, inst in zip(got, g["instances"]))
    print(f"pulse_area_sweep_64 precision {prec} half {half}: max |rho_gpu - rho_oracle| = {worst:.3e}")
    assert worst <= TOL[prec]
