"""Propagation graph replay (GPU).

A repeated quapi_propagate_device / quapi_propagate call with the same rho0 buffer, rho slots and step
list is captured as a CUDA graph on its second occurrence and replayed from then on.  The replay runs
the same kernels in the same order, so every rho must be bitwise equal to the direct run's (and to a
context with the replay turned off, QUAPI_GRAPH=0); the kernel-launch counter and the kept state
(quapi_get_state) must read as after a direct run, and new arguments must run directly again.
"""

import numpy as np
import pytest

from paper_1205_6872_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    assert torch.cuda.is_available()
    from paper_1205_6872_gb300 import quapi
    quapi.load()
    return quapi


def _problem(kind):
    if kind == "three_level":
        p = wl.three_level_L8()
        p.L, p.N = 4, 40
        return p
    p = wl.biased_L12()
    p.L, p.N = 8, 60
    return p


CASES = [("spin_boson", 32, 1), ("spin_boson", 32, 0), ("spin_boson", 48, 1), ("spin_boson", 64, 0),
         ("three_level", 32, 1), ("three_level", 64, 0)]


def _device_runs(q, p, prec, half, steps, reps):
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                        q.quapi_opts_init(precision=prec, hermitian=half))
    try:
        rho0 = torch.tensor(np.asarray(p.rho0).reshape(-1), dtype=torch.complex128, device="cuda")
        out = torch.empty(len(steps) * p.M * p.M, dtype=torch.complex128, device="cuda")
        rhos, launches, states = [], [], []
        for _ in range(reps):
            out.fill_(float("nan"))
            l0 = q.quapi_kernel_launches()
            q.quapi_propagate_device(ctx, rho0, steps, out)
            torch.cuda.synchronize()
            launches.append(q.quapi_kernel_launches() - l0)
            rhos.append(out.cpu().numpy().copy())
            states.append(q.quapi_get_state(ctx))
        return rhos, launches, states
    finally:
        q.quapi_destroy(ctx)


@pytest.mark.parametrize("kind,prec,half", CASES)
def test_replay_matches_direct_run(q, kind, prec, half, monkeypatch):
    p = _problem(kind)
    steps = [0, 3, p.L, p.L + 1, p.N // 2, p.N]
    rhos, launches, states = _device_runs(q, p, prec, half, steps, 4)  # direct, capture, replay, replay
    monkeypatch.setenv("QUAPI_GRAPH", "0")
    ref, ref_launches, ref_states = _device_runs(q, p, prec, half, steps, 1)
    assert np.all(np.isfinite(ref[0]))
    for r in rhos:
        assert np.array_equal(r.view(np.uint8), ref[0].view(np.uint8))
    assert launches == [ref_launches[0]] * 4
    for n, buf in states:
        assert n == ref_states[0][0] and np.array_equal(buf, ref_states[0][1])


def test_new_arguments_run_directly(q):
    """Changing the step list after a replay runs the new propagation (then replays it)."""
    p = _problem("spin_boson")
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                        q.quapi_opts_init(precision=32, hermitian=1))
    try:
        rho0 = torch.tensor(np.asarray(p.rho0).reshape(-1), dtype=torch.complex128, device="cuda")
        got = {}
        for steps in ([p.N], [p.N], [p.N], [5, p.N - 7], [5, p.N - 7], [5, p.N - 7], [p.N]):
            out = torch.empty(len(steps) * 4, dtype=torch.complex128, device="cuda")
            q.quapi_propagate_device(ctx, rho0, steps, out)
            torch.cuda.synchronize()
            r = out.cpu().numpy().reshape(len(steps), 2, 2)
            for k, v in zip(steps, r):
                got.setdefault(k, []).append(v)
    finally:
        q.quapi_destroy(ctx)
    for k, vs in got.items():
        for v in vs[1:]:
            assert np.array_equal(v, vs[0]), k


def test_host_api_replay_and_all_points(q):
    """quapi_propagate (host rho0 and rho) with rho at every step: repeated calls replay bitwise."""
    p = _problem("spin_boson")
    steps = list(range(p.N + 1))
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                        q.quapi_opts_init(precision=32, hermitian=1))
    try:
        runs = [q.quapi_propagate(ctx, p.rho0, steps, 2) for _ in range(3)]
        rho0b = np.array(p.rho0, dtype=np.complex128) * 0.5 + 0.25 * np.eye(2)  # new contents, same buffers
        other = q.quapi_propagate(ctx, rho0b, steps, 2)
    finally:
        q.quapi_destroy(ctx)
    for r in runs[1:]:
        assert np.array_equal(r, runs[0])
    assert np.abs(other - runs[0]).max() > 1e-3  # the replay reads the rho0 copied in by this call
    assert np.allclose([np.trace(r) for r in other], 1.0, atol=1e-5)
