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
