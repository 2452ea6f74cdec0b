"""quapi_readout_static against quapi_step_device's readout (GPU).

quapi_readout_static serves callers that must not allocate device memory
when they read rho out (their memory pool already owns the free memory, or a
cudaMalloc would stall a time-critical loop).  It keeps the readout's partial
sums in a fixed array inside the library instead.  This file is collected last
on purpose, and each check runs the new entry point twice in a row, because
every call reuses that one array.  It covers the three precisions (FP64, FP32,
the double-float DF64 form) and both tensor layouts (full, and the Hermitian
half layout, where the rows of rho below the diagonal are written as the
conjugates of the rows above it), for M = 2 and M = 3.
"""

import numpy as np
import pytest

from paper_1205_6872_gb300 import layout
from paper_1205_6872_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _to_dev(a, prec):
    """complex128 host tensor -> device tensor in the storage of the form (DF64: {re_hi, im_hi, re_lo, im_lo})."""
    if prec == 48:
        h = a.astype(np.complex64)
        lo = (a - h.astype(np.complex128)).astype(np.complex64)
        x = np.stack([h.real, h.imag, lo.real, lo.imag], axis=1).astype(np.float32)
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return torch.from_numpy(a).to(torch.complex128 if prec == 64 else torch.complex64).cuda()


CASES = [(2, 6, 3, 0), (2, 6, 6, 0), (2, 6, 9, 0), (2, 12, 20, 0), (3, 4, 7, 0),
         (2, 6, 3, 1), (2, 6, 9, 1), (2, 12, 20, 1), (2, 1, 4, 1), (3, 4, 7, 1), (3, 6, 6, 1)]


@pytest.mark.parametrize("prec", [64, 32, 48])
@pytest.mark.parametrize("M,L,n,half", CASES)
def test_readout_static_matches_step_readout(M, L, n, half, prec):
    assert torch.cuda.is_available()
    from paper_1205_6872_gb300 import quapi as q
    if M == 2:
        s, H = [1.0, -1.0], np.array([[0.5, 1.0], [1.0, -0.5]])
    else:
        s, H = [-1.0, 0.0, 1.0], wl.random_hermitian(3, 4)
    ctx = q.quapi_setup_eta(s, H, wl.random_eta(L, seed=n), 0.1, L,
                            q.quapi_opts_init(precision=prec, hermitian=half))
    try:
        d = min(n, L)
        entries = layout.count(d, M) if half else (M * M) ** d
        A = _to_dev(wl.random_tensor(entries, seed=n + L), prec)
        want = torch.zeros(M * M, dtype=torch.complex128, device="cuda")
        q.quapi_step_device(ctx, n, A, None, want)
        got = []
        for _ in range(2):
            r = torch.full((M * M,), float("nan"), dtype=torch.complex128, device="cuda")
            q.quapi_readout_static(ctx, n, A, r)
            got.append(r)
        torch.cuda.synchronize()
        w = want.cpu().numpy()
        assert np.all(np.isfinite(w))
        tol = (1e-6 if prec == 32 else 1e-13) * max(1.0, np.abs(w).max())
        for r in got:
            assert np.abs(r.cpu().numpy() - w).max() <= tol
    finally:
        q.quapi_destroy(ctx)


def test_readout_static_rejects_bad_arguments():
    from paper_1205_6872_gb300 import quapi as q
    ctx = q.quapi_setup_eta([1.0, -1.0], np.eye(2), wl.random_eta(3, seed=1), 0.1, 3)
    try:
        A = torch.zeros(16, dtype=torch.complex128, device="cuda")
        r = torch.zeros(4, dtype=torch.complex128, device="cuda")
        with pytest.raises(q.QuapiError) as e:
            q.quapi_readout_static(ctx, 0, A, r)
        assert e.value.status == q.QUAPI_ERR_ARG
        with pytest.raises(q.QuapiError) as e:
            q.quapi_readout_static(ctx, 2, A, None)
        assert e.value.status == q.QUAPI_ERR_ARG
    finally:
        q.quapi_destroy(ctx)
