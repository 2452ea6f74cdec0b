"""One step at the largest memory lengths the library accepts, against the oracle (GPU).

M = 2 with memory length 16 (half layout: 2.15 G stored entries, 17 GB per FP32 tensor; full layout:
4.29 G entries, 34 GB) and M = 3 with memory length 10 (half layout: 1.74 G entries): the sizes where the
kernels' index arithmetic comes closest to its limits (32-bit canonical positions and output indices).
The full tensors do not fit the host, so the input is a closed-form function of the stored position,
filled on the device with integer tensor operations, and the oracle's per-entry checker
(`oracle.recurrence.step_elements`, pinned against the whole-tensor step) reads any entry of the full
tensor through a lazy view that evaluates the same function.  The canonical positions of the half layout
are computed here from the layout's definition (most significant digit first: each canonical point's
block of plain continuations, then each self-conjugate point's canonical sub-layout).
"""

import numpy as np
import pytest

import oracle
import oracle.recurrence as rec
from oracle.eta import Spectral
from paper_1205_6872_gb300 import layout as ly
from paper_1205_6872_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    assert torch.cuda.is_available()
    from paper_1205_6872_gb300 import quapi
    quapi.load()
    return quapi


def _points(M):
    tops = [a * M + b for a in range(M) for b in range(M) if a < b]
    selfs = [a * M + a for a in range(M)]
    conj = [(x % M) * M + x // M for x in range(M * M)]
    return tops, selfs, conj


def _digits(v, n, Q):
    out = []
    for _ in range(n):
        out.append(v % Q)
        v //= Q
    return out[::-1]  # most significant first


def _canonical(prefix, n, M):
    tops, selfs, _ = _points(M)
    for d in _digits(prefix, n, M * M):
        if d in tops:
            return True
        if d not in selfs:
            return False
    return True


def _position(prefix, n, M):
    """Canonical position of a canonical n-digit prefix (plain digits), in the layout's order."""
    tops, selfs, _ = _points(M)
    Q = M * M
    idx = 0
    for level in range(n, 0, -1):
        P = Q ** (level - 1)
        d = (prefix // P) % Q
        if d in tops:
            return idx + tops.index(d) * P + prefix % P
        idx += len(tops) * P + selfs.index(d) * ly.canonical_count(level - 1, M)
    return idx


def _conj(v, n, M):
    _, _, conj = _points(M)
    Q = M * M
    out, scale = 0, 1
    for _ in range(n):
        out += conj[v % Q] * scale
        v //= Q
        scale *= Q
    return out


def _F(j):
    """The stored value at device position j (the same formula as _fill)."""
    return complex((j % 97) / 97.0 - 0.5, (j % 89) / 89.0 - 0.5)


def _fill(count, dtype):
    """Device tensor of count entries with value _F(position), built in chunks of integer arithmetic."""
    t = torch.empty(count, dtype=dtype, device="cuda")
    step = 1 << 28
    for s in range(0, count, step):
        j = torch.arange(s, min(count, s + step), dtype=torch.int64, device="cuda")
        re = (j % 97).to(torch.float64) / 97.0 - 0.5
        im = (j % 89).to(torch.float64) / 89.0 - 0.5
        t[s:s + j.numel()] = torch.complex(re, im).to(dtype)
        del j, re, im
    return t


class HalfView:
    """The full n-digit tensor that a half-layout device tensor holds, entry by entry."""

    def __init__(self, n, M, dtype):
        self.n, self.M, self.Q = n, M, M * M
        self.tops, self.selfs, self.conjpt = _points(M)
        self.round = (lambda z: complex(np.complex64(z))) if dtype == torch.complex64 else (lambda z: z)

    def stored(self, c, d):
        """Entry d of the stored fiber of canonical prefix position c, after the self-conjugate fix-up."""
        return self.round(_F(self.Q * c + d))

    def __getitem__(self, idx):
        idx = int(idx)
        prefix, d = divmod(idx, self.Q)
        npre = self.n - 1
        if _canonical(prefix, npre, self.M):
            c = _position(prefix, npre, self.M)
            if _conj(prefix, npre, self.M) == prefix:  # self-conjugate prefix: its fiber has the symmetry itself
                if d in self.selfs:
                    return complex(self.stored(c, d).real, 0.0)
                if d not in self.tops:
                    return self.stored(c, self.conjpt[d]).conjugate()
            return self.stored(c, d)
        return self[_conj(idx, self.n, self.M)].conjugate()


def _fix_self_conjugate(t, n, M):
    """Give the fibers of self-conjugate prefixes the symmetry (real self-conjugate entries, conjugate pairs)."""
    tops, selfs, conjpt = _points(M)
    Q = M * M
    npre = n - 1
    prefixes = [0]
    for _ in range(npre):
        prefixes = [p * Q + s for p in prefixes for s in selfs]
    pos = torch.tensor([_position(p, npre, M) for p in prefixes], dtype=torch.int64, device="cuda")
    for d in selfs:
        e = Q * pos + d
        t[e] = t[e].real.to(t.dtype)
    for d in range(Q):
        if d not in tops and d not in selfs:
            t[Q * pos + d] = torch.conj(t[Q * pos + conjpt[d]])


def _system(M):
    if M == 2:
        return np.array([1.0, -1.0]), np.array([[0.3, 1.0], [1.0, -0.3]], dtype=complex)
    return np.array([-1.0, 0.0, 1.0]), wl.random_hermitian(3, 1205)


@pytest.mark.parametrize("M,L", [(2, 16), (3, 10)])
def test_half_layout_step_at_the_largest_memory_length(q, M, L):
    s, H = _system(M)
    Q = M * M
    spec = Spectral("ohmic_exp", 0.1, 5.0)
    eta = oracle.pack_eta(oracle.eta_table(spec, 2.0, 0.1, L))
    etad = oracle.unpack_eta(eta, L)
    K = oracle.pair_propagator_K(oracle.propagator_U(H, 0.1))
    n = L + 1  # a steady step: the input holds L points, the oldest is summed
    G, gg, n_in, summed = rec.step_tables(etad, s, K, L, n)
    count = ly.count(L, M)
    ctx = q.quapi_setup_eta(s, H, eta, 0.1, L, q.quapi_opts_init(precision=32, hermitian=1))
    try:
        dA = _fill(count, torch.complex64)
        _fix_self_conjugate(dA, L, M)
        dout = torch.empty(count, dtype=torch.complex64, device="cuda")
        q.quapi_step_device(ctx, n, dA, dout, None)
        torch.cuda.synchronize()
        del dA
        rng = np.random.Generator(np.random.PCG64(16))
        pos = np.concatenate([np.arange(48), count - 1 - np.arange(48), rng.integers(0, count, 600)])
        got = dout[torch.from_numpy(pos).cuda()].cpu().numpy().astype(np.complex128)
    finally:
        q.quapi_destroy(ctx)
        torch.cuda.empty_cache()
    A = HalfView(L, M, torch.complex64)
    npre = L - 1
    full_idx = []
    for p in pos:  # the plain index of each sampled output position (same layout, L digits)
        c, d = divmod(int(p), Q)
        prefix = 0
        # decode canonical position c of an npre-digit prefix by walking the layout's blocks
        tops, selfs, _ = _points(M)
        rest, digits = c, []
        for level in range(npre, 0, -1):
            P = Q ** (level - 1)
            if rest < len(tops) * P:
                t, r = divmod(rest, P)
                prefix = ((prefix * Q + tops[t]) * P) + r
                break
            rest -= len(tops) * P
            cn = ly.canonical_count(level - 1, M)
            t, rest = divmod(rest, cn)
            prefix = prefix * Q + selfs[t]
        full_idx.append(prefix * Q + d)
    want = rec.step_elements(A, G, gg, n_in, summed, full_idx)
    scale = np.abs(want).max() + 1.0
    assert np.abs(got - want).max() <= 2e-6 * scale


def test_full_layout_step_at_the_largest_memory_length(q):
    """M = 2, memory length 16 in the full layout (4.29 G entries; 64-bit fiber indices, TMA rows)."""
    M, L = 2, 16
    s, H = _system(M)
    spec = Spectral("ohmic_exp", 0.1, 5.0)
    eta = oracle.pack_eta(oracle.eta_table(spec, 2.0, 0.1, L))
    etad = oracle.unpack_eta(eta, L)
    K = oracle.pair_propagator_K(oracle.propagator_U(H, 0.1))
    n = L + 1
    G, gg, n_in, summed = rec.step_tables(etad, s, K, L, n)
    count = 4 ** L
    ctx = q.quapi_setup_eta(s, H, eta, 0.1, L, q.quapi_opts_init(precision=32))
    try:
        dA = _fill(count, torch.complex64)
        dout = torch.empty(count, dtype=torch.complex64, device="cuda")
        q.quapi_step_device(ctx, n, dA, dout, None)
        torch.cuda.synchronize()
        del dA
        rng = np.random.Generator(np.random.PCG64(17))
        idx = np.concatenate([np.arange(48), count - 1 - np.arange(48), rng.integers(0, count, 600)])
        got = dout[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
    finally:
        q.quapi_destroy(ctx)
        torch.cuda.empty_cache()

    class FullView:
        def __getitem__(self, i):
            return complex(np.complex64(_F(int(i))))

    want = rec.step_elements(FullView(), G, gg, n_in, summed, idx)
    assert np.abs(got - want).max() <= 2e-6 * (np.abs(want).max() + 1.0)
