"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances: FP64 form 1e-12 max abs on rho elements; FP32 form 1e-5 max abs on
rho.  Single-step checks on random tensors compare every output element,
relative to the largest input magnitude times the number of factors.
"""

import numpy as np
import pytest

import oracle
import oracle.recurrence as rec
from oracle.eta import Spectral
from paper_1205_6872_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1205_6872_gb300 import quapi
    quapi.load()
    return quapi


def _problem(M, seed=3):
    if M == 2:
        return dict(s=np.array([1.0, -1.0]), H=np.array([[0.5, 1.0], [1.0, -0.5]], complex),
                    spec=Spectral("ohmic_exp", 0.3, 5.0), beta=1.0, dt=0.1,
                    rho0=np.array([[1, 0], [0, 0]], complex))
    return dict(s=np.array([-1.0, 0.0, 1.0]), H=wl.random_hermitian(3, seed),
                spec=Spectral("superohmic_gauss", 0.05, 2.0), beta=2.0, dt=0.2,
                rho0=wl.random_pure_state(3, seed + 1))


def _ctx(q, pr, L, prec, eta=None, endpoint=0):
    opts = q.quapi_opts_init(precision=prec, endpoint_mode=endpoint)
    if eta is not None:
        return q.quapi_setup_eta(pr["s"], pr["H"], eta, pr["dt"], L, opts)
    return q.quapi_setup(pr["s"], pr["H"], pr["spec"].kind, pr["spec"].a, pr["spec"].wc, pr["beta"],
                         pr["dt"], L, opts)


# ---------------------------------------------------------------- setup kernels

@pytest.mark.parametrize("M,L", [(2, 1), (2, 6), (2, 14), (3, 4)])
def test_eta_quadrature_matches_oracle(q, M, L):
    pr = _problem(M)
    ctx = _ctx(q, pr, L, q.QUAPI_FP64)
    try:
        got = q.quapi_get_eta(ctx, L)
    finally:
        q.quapi_destroy(ctx)
    want = oracle.pack_eta(oracle.eta_table(pr["spec"], pr["beta"], pr["dt"], L))
    err = np.abs(got - want)
    assert err.max() <= 1e-14 + 1e-13 * np.abs(want).max(), err.max()


@pytest.mark.parametrize("name", ["spin_boson_L6", "biased_L12", "three_level_L8", "spin_boson_L14"])
def test_eta_workloads(q, name):
    p = wl.CONFIGS[name]()
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init())
    try:
        got = q.quapi_get_eta(ctx, p.L)
    finally:
        q.quapi_destroy(ctx)
    want = oracle.pack_eta(oracle.eta_table(Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L))
    assert np.abs(got - want).max() <= 1e-14 + 1e-13 * np.abs(want).max()


def _tab_ctx(q, spec, beta, L, prec=64, dt=0.1):
    pr = _problem(2)
    return q.quapi_setup(pr["s"], pr["H"], "tabulated", 0.0, 1.0, beta, dt, L,
                         q.quapi_opts_init(precision=prec), omega=spec.omega, values=spec.values)


@pytest.mark.parametrize("table", ["ramp", "ohmic"])
@pytest.mark.parametrize("beta", [0.7, 5.0])
def test_eta_tabulated_matches_oracle(q, table, beta):
    """Tabulated J: the device quadrature (panels aligned to the table) against the oracle's."""
    L = 6
    if table == "ramp":
        om = np.linspace(3.0, 21.0, 7)
        spec = Spectral.tabulated(om, 0.4 * om)
    else:
        om = np.linspace(0.5, 100.0, 200)
        spec = Spectral.tabulated(om, Spectral("ohmic_exp", 0.3, 5.0).J(om))
    ctx = _tab_ctx(q, spec, beta, L)
    try:
        got = q.quapi_get_eta(ctx, L)
    finally:
        q.quapi_destroy(ctx)
    want = oracle.pack_eta(oracle.eta_table(spec, beta, 0.1, L))
    assert np.abs(got - want).max() <= 1e-14 + 1e-13 * np.abs(want).max()


def test_eta_tabulated_ramp_zero_temperature_closed_form(q):
    """J = c w on [0, Om] at beta = 1e7 (thermal part ~ 1/beta^2): the device eta against the sine and
    cosine integral forms of the self box and of the interior neighbour pair."""
    from test_oracle_eta import _ramp_pair, _ramp_self
    c, Om, dt, L = 0.4, 21.0, 0.1, 3
    om = np.linspace(Om / 5, Om, 5)
    ctx = _tab_ctx(q, Spectral.tabulated(om, c * om), 1e7, L, dt=dt)
    try:
        got = q.quapi_get_eta(ctx, L)
    finally:
        q.quapi_destroy(ctx)
    # packed layout: interior[0..L], point0[0..L-1], end_self, end[0..L-1], end_point0[0..L-1], self0
    assert abs(got[0] - _ramp_self(c, Om, dt)) <= 1e-13
    assert abs(got[1] - _ramp_pair(c, Om, dt, dt, dt)) <= 1e-13
    assert abs(got[2 * L + 1] - _ramp_self(c, Om, 0.5 * dt)) <= 1e-13
    assert abs(got[-1] - _ramp_self(c, Om, 0.5 * dt)) <= 1e-13


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5)])
def test_tabulated_propagation_matches_oracle(q, prec, tol):
    pr = _problem(2)
    om = np.linspace(0.25, 60.0, 240)
    spec = Spectral.tabulated(om, Spectral("ohmic_exp", 0.3, 5.0).J(om))
    L, steps = 5, [0, 1, 4, 5, 6, 20, 40]
    want = oracle.propagate(pr["s"], pr["H"], spec, pr["beta"], pr["dt"], L, pr["rho0"], steps)
    ctx = _tab_ctx(q, spec, pr["beta"], L, prec=prec, dt=pr["dt"])
    try:
        got = q.quapi_propagate(ctx, pr["rho0"], steps, 2)
    finally:
        q.quapi_destroy(ctx)
    for i, k in enumerate(steps):
        assert np.abs(got[i] - want[k]).max() <= tol, k


def test_tabulated_argument_errors(q):
    pr = _problem(2)
    bad = [([1.0, 0.5], [1.0, 1.0]),    # not ascending
           ([0.0, 1.0], [0.0, 1.0]),    # omega[0] not > 0
           ([1.0, 2.0], [1.0, -1.0]),   # negative J
           ([1.0, np.inf], [1.0, 1.0]),
           ([], [])]
    for om, va in bad:
        with pytest.raises(q.QuapiError) as e:
            q.quapi_setup(pr["s"], pr["H"], "tabulated", 0.0, 1.0, 1.0, 0.1, 3, q.quapi_opts_init(),
                          omega=om, values=va)
        assert e.value.status == q.QUAPI_ERR_ARG, (om, va)
    with pytest.raises(q.QuapiError) as e:  # tabulated kind without a table
        q.quapi_setup(pr["s"], pr["H"], "tabulated", 0.0, 1.0, 1.0, 0.1, 3, q.quapi_opts_init())
    assert e.value.status == q.QUAPI_ERR_ARG


@pytest.mark.parametrize("M", [2, 3])
def test_propagator_matches_oracle(q, M):
    pr = _problem(M)
    ctx = _ctx(q, pr, 2, q.QUAPI_FP64)
    try:
        U, K = q.quapi_get_propagator(ctx, M)
    finally:
        q.quapi_destroy(ctx)
    Uo = oracle.propagator_U(pr["H"], pr["dt"])
    assert np.abs(U - Uo).max() < 1e-14
    assert np.abs(K - oracle.pair_propagator_K(Uo)).max() < 1e-14


# ---------------------------------------------------------------- single steps on random tensors

def to_df(a):
    """complex128 -> double-float layout {re_hi, im_hi, re_lo, im_lo} (float32 x 4 per entry)."""
    a = np.asarray(a, dtype=np.complex128)
    h = a.astype(np.complex64)
    l = (a - h.astype(np.complex128)).astype(np.complex64)
    out = np.empty((a.size, 4), dtype=np.float32)
    out[:, 0], out[:, 1], out[:, 2], out[:, 3] = h.real, h.imag, l.real, l.imag
    return out


def from_df(x):
    x = np.asarray(x, dtype=np.float32).reshape(-1, 4).astype(np.float64)
    return (x[:, 0] + x[:, 2]) + 1j * (x[:, 1] + x[:, 3])


def representable(A, prec):
    """The values the device form stores for A (what both sides must start from)."""
    if prec == 32:
        return A.astype(np.complex64).astype(np.complex128)
    if prec == 48:
        return from_df(to_df(A))
    return A


def _to_dev(a, prec):
    if prec == 48:
        return torch.from_numpy(to_df(a)).cuda()
    t = torch.from_numpy(np.ascontiguousarray(a))
    t = t.to(torch.complex128 if prec == 64 else torch.complex64)
    return t.cuda()


def _from_dev(t, prec):
    if prec == 48:
        return from_df(t.cpu().numpy())
    return t.cpu().numpy().astype(np.complex128)


def _empty_dev(n, prec):
    if prec == 48:
        return torch.empty((n, 4), dtype=torch.float32, device="cuda")
    return torch.empty(n, dtype=torch.complex128 if prec == 64 else torch.complex64, device="cuda")


STEP_CASES = [
    # (M, L, n): growth steps (n < L), the first summing step (n == L), steady steps
    (2, 6, 1), (2, 6, 3), (2, 6, 5), (2, 6, 6), (2, 6, 7), (2, 6, 40),
    (2, 1, 1), (2, 1, 9), (2, 2, 2), (2, 5, 12), (2, 9, 9), (2, 9, 30),
    (3, 4, 2), (3, 4, 4), (3, 4, 11), (3, 1, 3), (3, 6, 6), (3, 6, 8),
]


@pytest.mark.parametrize("prec", [64, 32, 48])
@pytest.mark.parametrize("M,L,n", STEP_CASES)
def test_single_step_random_tensor(q, M, L, n, prec):
    pr = _problem(M)
    eta = wl.random_eta(L, seed=100 + L + n)
    etad = oracle.unpack_eta(eta, L)
    K = oracle.pair_propagator_K(oracle.propagator_U(pr["H"], pr["dt"]))
    M2 = M * M
    n_in = min(n, L)
    A = representable(wl.random_tensor(M2 ** n_in, seed=7 * n + L), prec)  # both sides start equal
    G, g, n_in_o, summed = rec.step_tables(etad, pr["s"], K, L, n)
    want = rec.apply_step(A, G, g, n_in_o, summed)
    Gr, gr, _ = rec.readout_tables(etad, pr["s"], K, L, n)
    want_rho = rec.apply_readout(A, Gr, gr, n_in_o)
    ctx = _ctx(q, pr, L, prec, eta=eta)
    try:
        dA = _to_dev(A, prec)
        dout = _empty_dev(want.size, prec)
        drho = torch.zeros(M2, dtype=torch.complex128, device="cuda")
        q.quapi_step_device(ctx, n, dA, dout, drho)
        torch.cuda.synchronize()
        got = _from_dev(dout, prec)
        got_rho = drho.cpu().numpy()
    finally:
        q.quapi_destroy(ctx)
    # element scale: |T| * sum |A| over the summed index
    scale = np.abs(want).max() + 1.0
    tol = 2e-6 if prec == 32 else 1e-13
    assert np.abs(got - want).max() <= tol * scale, np.abs(got - want).max()
    rscale = np.abs(A).sum() * np.abs(G).max() ** n_in
    rtol = 1e-6 if prec == 32 else 1e-13
    assert np.abs(got_rho - want_rho).max() <= rtol * max(1.0, np.abs(want_rho).max()) + 1e-15 * rscale


# ---------------------------------------------------------------- full propagations

@pytest.mark.parametrize("endpoint", [0, 1])
def test_spin_boson_L6_fp64_all_steps(q, endpoint):
    p = wl.spin_boson_L6()
    spec = Spectral(p.jkind, p.ja, p.wc)
    steps = list(range(p.N + 1))
    want = oracle.propagate(p.s, p.H, spec, p.beta, p.dt, p.L, p.rho0, steps,
                            endpoint="strang" if endpoint == 0 else "interior")
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                        q.quapi_opts_init(precision=64, endpoint_mode=endpoint))
    try:
        got = q.quapi_propagate(ctx, p.rho0, steps, p.M)
    finally:
        q.quapi_destroy(ctx)
    err = max(np.abs(got[i] - want[k]).max() for i, k in enumerate(steps))
    assert err <= 1e-12, err


@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (48, 1e-12)])
def test_spin_boson_L6_reduced_forms_all_steps(q, prec, tol):
    p = wl.spin_boson_L6()
    spec = Spectral(p.jkind, p.ja, p.wc)
    steps = list(range(p.N + 1))
    want = oracle.propagate(p.s, p.H, spec, p.beta, p.dt, p.L, p.rho0, steps)
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(precision=prec))
    try:
        got = q.quapi_propagate(ctx, p.rho0, steps, p.M)
    finally:
        q.quapi_destroy(ctx)
    err = max(np.abs(got[i] - want[k]).max() for i, k in enumerate(steps))
    assert err <= tol, err


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5), (48, 1e-12)])
@pytest.mark.parametrize("M,L,N", [(2, 1, 30), (2, 3, 2), (2, 8, 60), (3, 3, 25), (3, 5, 12)])
def test_small_propagations(q, M, L, N, prec, tol):
    pr = _problem(M, seed=5)
    steps = sorted(set([0, 1, 2, min(L, N), N // 2, N]))
    want = oracle.propagate(pr["s"], pr["H"], pr["spec"], pr["beta"], pr["dt"], L, pr["rho0"], steps)
    ctx = _ctx(q, pr, L, prec)
    try:
        got = q.quapi_propagate(ctx, pr["rho0"], steps, M)
    finally:
        q.quapi_destroy(ctx)
    for i, k in enumerate(steps):
        assert np.abs(got[i] - want[k]).max() <= tol, (k, got[i], want[k])


def test_only_step_zero(q):
    pr = _problem(2)
    ctx = _ctx(q, pr, 4, 64)
    try:
        got = q.quapi_propagate(ctx, pr["rho0"], [0], 2)
    finally:
        q.quapi_destroy(ctx)
    assert np.array_equal(got[0], pr["rho0"])


# ---------------------------------------------------------------- argument errors

def test_argument_errors(q):
    pr = _problem(2)
    with pytest.raises(q.QuapiError) as e:
        q.quapi_setup(pr["s"], [[0, 1], [2, 0]], "ohmic_exp", 0.1, 5.0, 1.0, 0.1, 4)
    assert e.value.status == q.QUAPI_ERR_ARG
    with pytest.raises(q.QuapiError) as e:
        q.quapi_setup(pr["s"], pr["H"], "ohmic_exp", 0.1, 5.0, 1.0, -0.1, 4)
    assert e.value.status == q.QUAPI_ERR_ARG
    with pytest.raises(q.QuapiError) as e:
        q.quapi_setup(np.zeros(4), np.eye(4), "ohmic_exp", 0.1, 5.0, 1.0, 0.1, 4)
    assert e.value.status == q.QUAPI_ERR_ARG
    with pytest.raises(q.QuapiError) as e:
        q.quapi_setup(pr["s"], pr["H"], "ohmic_exp", 0.1, 5.0, 1.0, 0.1, 0)
    assert e.value.status == q.QUAPI_ERR_ARG
    ctx = _ctx(q, pr, 3, 64)
    try:
        with pytest.raises(q.QuapiError) as e:
            q.quapi_propagate(ctx, pr["rho0"], [3, 2], 2)
        assert e.value.status == q.QUAPI_ERR_ARG
        with pytest.raises(q.QuapiError) as e:
            q.quapi_propagate(ctx, pr["rho0"], [-1, 2], 2)
        assert e.value.status == q.QUAPI_ERR_ARG
        with pytest.raises(q.QuapiError) as e:
            q.quapi_propagate(ctx, pr["rho0"], [], 2)          # empty time grid
        assert e.value.status == q.QUAPI_ERR_ARG
        with pytest.raises(q.QuapiError) as e:
            q.quapi_step_device(ctx, 0, 1, 1, None)             # no path point 0 step
        assert e.value.status == q.QUAPI_ERR_ARG
    finally:
        q.quapi_destroy(ctx)
    # device buffers must be 16-byte aligned: rejected before any kernel runs
    ctx = _ctx(q, pr, 3, 32)
    try:
        A = torch.zeros(4 ** 3 + 2, dtype=torch.complex64, device="cuda")
        B = torch.zeros(4 ** 3 + 2, dtype=torch.complex64, device="cuda")
        rho = torch.zeros(4, dtype=torch.complex128, device="cuda")
        for a_in, a_out in ((A[1:], B[:-2]), (A[:-2], B[1:])):   # one complex64 = 8 bytes off
            with pytest.raises(q.QuapiError) as e:
                q.quapi_step_device(ctx, 4, a_in, a_out, None)
            assert e.value.status == q.QUAPI_ERR_ARG
        with pytest.raises(q.QuapiError) as e:
            q.quapi_readout_static(ctx, 4, A[1:], rho)
        assert e.value.status == q.QUAPI_ERR_ARG
        q.quapi_step_device(ctx, 4, A[:-2], B[:-2], rho)        # aligned views work
        torch.cuda.synchronize()
    finally:
        q.quapi_destroy(ctx)


# ---------------------------------------------------------------- checkpoint / resume

@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5), (48, 1e-12)])
def test_checkpoint_resume_matches_uninterrupted(q, prec, tol):
    p = wl.spin_boson_L6()
    full_steps = [10, 25, 40, 60]
    want = oracle.propagate(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L, p.rho0, full_steps)
    c1 = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(precision=prec))
    c2 = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, q.quapi_opts_init(precision=prec))
    try:
        first = q.quapi_propagate(c1, p.rho0, [10, 25], p.M)
        n, state = q.quapi_get_state(c1)
        assert n == 24
        # a fresh context with the same inputs continues from the saved tensor
        q.quapi_set_state(c2, n, state)
        rest = q.quapi_propagate_resume(c2, [40, 60], p.M)
        # and the original context can continue too
        rest1 = q.quapi_propagate_resume(c1, [40, 60], p.M)
        with pytest.raises(q.QuapiError) as e:
            q.quapi_propagate_resume(c1, [30], p.M)   # not after the kept tensor (now A_59)
        assert e.value.status == q.QUAPI_ERR_ARG
        with pytest.raises(q.QuapiError):
            q.quapi_set_state(c2, 3, state)            # size does not match A_3
    finally:
        q.quapi_destroy(c1)
        q.quapi_destroy(c2)
    for got, k in zip(list(first) + list(rest), full_steps):
        assert np.abs(got - want[k]).max() <= tol, k
    for got, k in zip(rest1, [40, 60]):
        assert np.abs(got - want[k]).max() <= tol, k


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5), (48, 1e-12)])
def test_autotuned_step_matches_oracle(q, prec, tol):
    """opts.tune picks the steady-step launch shape by timing; results must not change."""
    pr = _problem(2, seed=5)
    L, steps = 8, [0, 3, 8, 9, 40]
    want = oracle.propagate(pr["s"], pr["H"], pr["spec"], pr["beta"], pr["dt"], L, pr["rho0"], steps)
    ctx = q.quapi_setup(pr["s"], pr["H"], pr["spec"].kind, pr["spec"].a, pr["spec"].wc, pr["beta"], pr["dt"], L,
                        q.quapi_opts_init(precision=prec, tune=1))
    try:
        got = q.quapi_propagate(ctx, pr["rho0"], steps, 2)
    finally:
        q.quapi_destroy(ctx)
    for i, k in enumerate(steps):
        assert np.abs(got[i] - want[k]).max() <= tol, k
