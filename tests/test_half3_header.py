"""The M = 3 half-layout index helpers of the CUDA header (``csrc/half_layout.cuh``) on the host (CPU).

The helpers are ``__host__ __device__``, so a small host program built with nvcc (no kernel launched)
prints, for every canonical position c of every prefix length n <= 6, what each helper returns:
``half3_decode``, ``half3_decode_pair``, ``half3_decode_run``, ``half3_position``, ``self_conjugate3``,
``conj_digits3``, ``half3_count`` and ``half3_entries``.  They are compared with the half layout written
out in Python (``paper_1205_6872_gb300.layout``, itself pinned against oracle tensors in test_layout.py):
the canonical prefix at each position, its own conjugacy, the canonical position of the prefix without its
last digit, and the run property the step kernels' fast path relies on (position c + i holds prefix f + i,
whose last-digit-free prefix sits at h + (f % 9 + i) / 9, for every i < run).
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1205_6872_gb300 import build as B
from paper_1205_6872_gb300 import layout as ly

NMAX = 6

PROGRAM = r"""
#include <cstdio>
#include "half_layout.cuh"
using namespace quapi;
int main() {
    for (int n = 0; n <= %(nmax)d; ++n) {
        const uint32_t cnt = half3_count(n);
        std::printf("# %%d %%u %%lld\n", n, cnt, (long long)half3_entries(n));
        for (uint32_t c = 0; c < cnt; ++c) {
            uint32_t f1, f2, f3, h2, h3, run;
            bool s1, s2, s3, sh2, sh3;
            half3_decode(c, n, f1, s1);
            half3_decode_pair(c, n, f2, s2, h2, sh2);
            half3_decode_run(c, n, f3, s3, h3, sh3, run);
            std::printf("%%d %%u %%u %%d %%u %%d %%u %%d %%u %%d %%u %%d %%u %%u %%d %%u\n", n, c, f1, (int)s1, f2, (int)s2,
                        h2, (int)sh2, f3, (int)s3, h3, (int)sh3, run, half3_position(f1, n),
                        (int)self_conjugate3(f1, n), conj_digits3(f1, n));
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    if shutil.which(B.NVCC) is None:
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("half3")
    src = d / "half3_host.cu"
    src.write_text(PROGRAM % {"nmax": NMAX})
    exe = d / "half3_host"
    subprocess.run([B.NVCC] + B.ARCH + ["-O1", "-std=c++17", "-I", os.path.join(B.ROOT, "include"),
                                        "-I", B.CSRC, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    heads, rows = {}, []
    for line in out.splitlines():
        if line.startswith("#"):
            _, n, cnt, ent = line.split()
            heads[int(n)] = (int(cnt), int(ent))
        else:
            rows.append(line)
    data = np.loadtxt(rows, dtype=np.int64).reshape(-1, 16)
    return heads, data


def test_counts(table):
    heads, _ = table
    for n in range(NMAX + 1):
        assert heads[n] == (ly.canonical_count(n, 3), ly.count(n, 3))


@pytest.mark.parametrize("n", range(NMAX + 1))
def test_decode_position_and_conjugation(table, n):
    _, data = table
    t = data[data[:, 0] == n]
    order = ly.canonical_order(n, 3)
    c, f1, s1, f2, s2, h2, sh2, f3, s3, h3, sh3, run, pos, selfc, conjf = t[:, 1:].T
    assert np.array_equal(c, np.arange(len(order)))
    assert np.array_equal(f1, order) and np.array_equal(f2, order) and np.array_equal(f3, order)
    conj = ly.conj_index(order, n, 3)
    sc = (conj == order).astype(np.int64)
    for s in (s1, s2, s3, selfc):
        assert np.array_equal(s, sc)
    assert np.array_equal(pos, c)
    assert np.array_equal(conjf, conj)
    if n == 0:
        return
    # canonical position of f / 9 among the canonical (n-1)-digit prefixes, and whether it is self-conjugate
    sub = ly.canonical_order(n - 1, 3)
    where = {int(v): i for i, v in enumerate(sub)}
    fh = order // 9
    want_h = np.array([where[int(v)] for v in fh], dtype=np.int64)
    assert np.array_equal(h2, want_h) and np.array_equal(h3, want_h)
    shc = (ly.conj_index(fh, n - 1, 3) == fh).astype(np.int64)
    assert np.array_equal(sh2, shc) and np.array_equal(sh3, shc)


@pytest.mark.parametrize("n", range(2, NMAX + 1))
def test_run_property(table, n):
    """run(c) is 0 at self-conjugate prefixes; inside a run the next position holds the next plain prefix,
    its run is one shorter, and the canonical position of its last-digit-free prefix advances when the last
    digit wraps (f % 9 = 8 -> 0)."""
    _, data = table
    t = data[data[:, 0] == n]
    f, h, run, sc = t[:, 8], t[:, 10], t[:, 12], t[:, 9]
    assert np.all(run[sc == 1] == 0)
    assert np.any(run > 0)
    i = np.nonzero(run >= 2)[0]
    assert np.array_equal(f[i + 1], f[i] + 1)
    assert np.array_equal(run[i + 1], run[i] - 1)
    assert np.array_equal(h[i + 1], h[i] + (f[i] % 9 + 1) // 9)
    # with h checked against the layout at every position (test above), these recurrences make the fast
    # path's h + (f % 9 + i) / 9 the true position for every i < run
