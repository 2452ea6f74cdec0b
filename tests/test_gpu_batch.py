"""Batched propagation (one persistent, graph-captured launch) against the oracle (GPU)."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from oracle.eta import Spectral
from paper_1205_6872_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def q():
    assert torch.cuda.is_available()
    from paper_1205_6872_gb300 import quapi
    quapi.load()
    return quapi


def _c(v):
    return np.array([complex(a, b) for a, b in v])


def _ctxs(q, probs, prec, tune=0, hermitian=0):
    return [q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                          q.quapi_opts_init(precision=prec, tune=tune, hermitian=hermitian)) for p in probs]


@pytest.mark.parametrize("half", [0, 1])
@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5), (48, 1e-12)])
def test_batched_256_against_stored_oracle(q, prec, tol, half):
    """half = 1: the tiled instances keep their tensors in the Hermitian half layout."""
    probs = wl.batched_256()
    with open(os.path.join(HERE, "golden", "batched_256.json")) as fh:
        g = json.load(fh)
    ctxs = _ctxs(q, probs, prec, hermitian=half)
    try:
        for rep in range(2):  # second call replays the captured graph
            got = q.quapi_propagate_batch(ctxs, [p.rho0 for p in probs], [p.N for p in probs])
            worst = max(float(np.abs(r - _c(x["rho"]).reshape(2, 2)).max()) for r, x in zip(got, g["instances"]))
            print(f"batched_256 precision {prec} half layout {half} call {rep}: max abs error vs oracle = {worst:.3e}")
            assert worst <= tol
    finally:
        for c in ctxs:
            q.quapi_destroy(c)


@pytest.mark.parametrize("half", [0, 1])
@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5), (48, 1e-12)])
def test_batched_mixed_final_steps(q, prec, tol, half):
    """Final steps 0, 1, below and above L, several memory lengths, M = 2 (readouts in the growth phase too)."""
    base = wl.batched_256(n=12, seed=3)
    Ns = [0, 1, 2, 3, 5, 9, 11, 12, 20, 33, 47, 60]
    probs = base
    ctxs = _ctxs(q, probs, prec, hermitian=half)
    try:
        got = q.quapi_propagate_batch(ctxs, [p.rho0 for p in probs], Ns)
    finally:
        for c in ctxs:
            q.quapi_destroy(c)
    for p, N, r in zip(probs, Ns, got):
        want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, [N])[N]
        assert np.abs(r - want).max() <= tol, (p.L, N)


def test_batched_half_and_full_layouts_together(q):
    """Half-layout and full-layout contexts in one batch, tiled memory lengths 6..12, and L = 1 (a
    one-digit tensor whose prefixes have no digits): each instance matches the oracle."""
    probs = wl.batched_256(n=10, seed=17, N=30)
    Ls = [1, 6, 7, 8, 9, 10, 11, 12, 7, 9]
    for p, L in zip(probs, Ls):
        p.L = L
    ctxs = [q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                          q.quapi_opts_init(precision=64, hermitian=i % 2)) for i, p in enumerate(probs)]
    Ns = [30, 30, 25, 30, 12, 30, 11, 30, 7, 30]
    try:
        got = q.quapi_propagate_batch(ctxs, [p.rho0 for p in probs], Ns)
    finally:
        for c in ctxs:
            q.quapi_destroy(c)
    for p, N, r in zip(probs, Ns, got):
        want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, [N])[N]
        assert np.abs(r - want).max() <= 1e-12, (p.L, N)


def test_batched_three_level_df64(q):
    """M = 3 in the DF64 form (FP64-equivalent on the FP32 pipes) against the oracle."""
    probs = []
    for i, L in enumerate([2, 3, 4, 5]):
        p = wl.three_level_L8()
        p.L = L
        p.H = wl.random_hermitian(3, 60 + i)
        probs.append(p)
    Ns = [7, 3, 12, 9]
    ctxs = _ctxs(q, probs, 48)
    try:
        got = q.quapi_propagate_batch(ctxs, [p.rho0 for p in probs], Ns, M=3)
    finally:
        for c in ctxs:
            q.quapi_destroy(c)
    for p, N, r in zip(probs, Ns, got):
        want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, [N])[N]
        assert np.abs(r - want).max() <= 1e-12


def test_batched_three_level(q):
    probs = []
    for i, L in enumerate([2, 3, 4, 5]):
        p = wl.three_level_L8()
        p.L = L
        p.H = wl.random_hermitian(3, 40 + i)
        probs.append(p)
    Ns = [7, 3, 12, 9]
    ctxs = _ctxs(q, probs, 64)
    try:
        got = q.quapi_propagate_batch(ctxs, [p.rho0 for p in probs], Ns, M=3)
    finally:
        for c in ctxs:
            q.quapi_destroy(c)
    for p, N, r in zip(probs, Ns, got):
        want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, [N])[N]
        assert np.abs(r - want).max() <= 1e-12


@pytest.mark.parametrize("half", [0, 1])
def test_batched_autotuned_matches(q, half):
    probs = wl.batched_256(n=24, seed=9, N=40)
    ctxs = _ctxs(q, probs, 32, tune=1, hermitian=half)
    try:
        got = q.quapi_propagate_batch(ctxs, [p.rho0 for p in probs], [p.N for p in probs])
    finally:
        for c in ctxs:
            q.quapi_destroy(c)
    for p, r in zip(probs, got):
        want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, [p.N])[p.N]
        assert np.abs(r - want).max() <= 1e-5


def test_batched_argument_errors(q):
    probs = wl.batched_256(n=2, seed=1, N=10)
    c64 = _ctxs(q, probs[:1], 64)[0]
    c32 = _ctxs(q, probs[1:], 32)[0]
    try:
        with pytest.raises(q.QuapiError) as e:
            q.quapi_propagate_batch([c64, c32], [p.rho0 for p in probs], [10, 10])
        assert e.value.status == q.QUAPI_ERR_UNSUPPORTED
        with pytest.raises(q.QuapiError) as e:
            q.quapi_propagate_batch([c64, c64], [p.rho0 for p in probs], [10, 10])
        assert e.value.status == q.QUAPI_ERR_ARG
        with pytest.raises(q.QuapiError) as e:
            q.quapi_propagate_batch([c64], [probs[0].rho0], [-1])
        assert e.value.status == q.QUAPI_ERR_ARG
    finally:
        q.quapi_destroy(c64)
        q.quapi_destroy(c32)


_TIMEOUT_SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1205_6872_gb300 import quapi as q, workloads as wl
probs = wl.batched_256(n=6, seed=2, N=30)
for p in probs:
    p.L = 8   # every instance tiled (too big to stay in shared memory)
ctxs = [q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(precision=32))
        for p in probs]
try:
    q.quapi_propagate_batch(ctxs, [p.rho0 for p in probs], [p.N for p in probs])
    print("NO_ERROR")
except q.QuapiError as e:
    print("STATUS", e.status)
# the contexts stay usable after the device wait gave up
r = q.quapi_propagate(ctxs[0], probs[0].rho0, [5], 2)
print("TRACE", float(np.trace(r[0]).real))
for c in ctxs:
    q.quapi_destroy(c)
"""


def test_batched_bounded_wait_reports_timeout(tmp_path):
    """A dependency nothing satisfies (host-side fault injection): the kernel's
    bounded wait expires, the call returns QUAPI_ERR_TIMEOUT, the GPU stays usable."""
    script = tmp_path / "timeout_case.py"
    script.write_text(_TIMEOUT_SCRIPT)
    env = dict(os.environ, QUAPI_FAULT="batch_wait", QUAPI_WAIT_MS="50")
    out = subprocess.run([sys.executable, str(script), ROOT], env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr
    assert "STATUS 4" in out.stdout, out.stdout
    trace = float(out.stdout.split("TRACE")[1].split()[0])
    assert abs(trace - 1.0) < 1e-5
