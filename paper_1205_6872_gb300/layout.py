"""Hermitian half layout of the augmented tensor (M = 2 or 3), host-side conversion helpers.

A path point of an M-level system is x = (s+, s-) = a M + b (digit value in base
M^2).  Swapping the forward and backward path of every point (x = (a, b) ->
x-bar = (b, a)) conjugates a path's weight (K and every influence factor go to
their complex conjugates), so for a Hermitian rho(0) the tensor obeys
A(x-bar_1 .. x-bar_n) = conj(A(x_1 .. x_n)).  The points with a = b are their own
conjugates ("self-conjugate": 0 and 3 for M = 2; 0, 4 and 8 for M = 3); the other
points come in pairs, and the member with a < b is the pair's *canonical* one
(1 for M = 2; 1, 2 and 5 for M = 3, conjugates 3, 6 and 7).  An index is canonical
when its most significant digit that is not self-conjugate is a canonical point;
indices made only of self-conjugate digits are their own conjugates.  Only
canonical entries are stored, in this recursive order for n digits (most
significant first):

    [top digit = each canonical point in increasing order: all (M^2)^(n-1)
     continuations, plain base-M^2 order]
    [top digit = each self-conjugate point in increasing order: the canonical
     layout of the remaining n-1 digits]

giving C(n) = ((M^2)^n + M^n) / 2 canonical indices.  For M = 2 the order is
[top 1: 4^(n-1) plain][top 0: C(n-1)][top 3: C(n-1)].  The device layout keeps
whole fibers of the last digit: for n >= 1 it stores, for every canonical prefix
of n - 1 digits in the order above, the M^2 entries of its fiber (a prefix made
only of self-conjugate digits also keeps the redundant entries of its last
digit, the conjugates of other entries of the same fiber).  That is M^2 C(n-1)
entries (1 for n = 0), and canonical prefix c starts at entry M^2 c.

These helpers convert between the full and the half layout (used by tests,
checkpoints and callers that inspect tensors); the device kernels compute the
same positions themselves.
"""

from __future__ import annotations

import numpy as np


def _points(M: int):
    """(canonical points, self-conjugate points, conjugate of every point) for an M-level system."""
    tops = [a * M + b for a in range(M) for b in range(M) if a < b]
    selfs = [a * M + a for a in range(M)]
    conj = [(x % M) * M + x // M for x in range(M * M)]
    return tops, selfs, conj


def canonical_count(n: int, M: int = 2) -> int:
    """C(n): canonical n-digit indices."""
    return ((M * M) ** n + M ** n) // 2


def count(n: int, M: int = 2) -> int:
    """Entries of the device half layout of an n-digit tensor."""
    return 1 if n == 0 else M * M * canonical_count(n - 1, M)


def canonical_order(n: int, M: int = 2) -> np.ndarray:
    """Plain indices of the canonical n-digit indices, in half-layout order."""
    if n == 0:
        return np.zeros(1, dtype=np.int64)
    tops, selfs, _ = _points(M)
    Q = M * M
    sub = canonical_order(n - 1, M)
    top = Q ** (n - 1)
    parts = [x * top + np.arange(top, dtype=np.int64) for x in tops]
    parts += [d * top + sub for d in selfs]
    return np.concatenate(parts)


def canonical_indices(n: int, M: int = 2) -> np.ndarray:
    """Plain (full-layout) index of every entry of the device half layout, in order."""
    if n == 0:
        return np.zeros(1, dtype=np.int64)
    Q = M * M
    prefixes = canonical_order(n - 1, M)
    return (Q * prefixes[:, None] + np.arange(Q, dtype=np.int64)[None, :]).reshape(-1)


def to_half(A_full: np.ndarray, n: int, M: int = 2) -> np.ndarray:
    """Full tensor ((M^2)^n entries) -> device half layout (count(n) entries)."""
    A_full = np.asarray(A_full)
    if A_full.shape[0] != (M * M) ** n:
        raise ValueError("full tensor must have (M^2)^n entries")
    return A_full[canonical_indices(n, M)]


def conj_index(idx: np.ndarray, n: int, M: int = 2) -> np.ndarray:
    """Plain index of the conjugate path ((a, b) -> (b, a) in every digit)."""
    idx = np.asarray(idx, dtype=np.int64)
    _, _, conj = _points(M)
    cmap = np.asarray(conj, dtype=np.int64)
    Q = M * M
    out = np.zeros_like(idx)
    rest = idx.copy()
    scale = 1
    for _ in range(n):
        out += cmap[rest % Q] * scale
        rest //= Q
        scale *= Q
    return out


def from_half(A_half: np.ndarray, n: int, M: int = 2) -> np.ndarray:
    """Half layout -> full tensor, filling the missing entries as conjugates of stored ones."""
    A_half = np.asarray(A_half)
    idx = canonical_indices(n, M)
    out = np.empty((M * M) ** n, dtype=np.result_type(A_half.dtype, np.complex64))
    out[conj_index(idx, n, M)] = np.conj(A_half)
    out[idx] = A_half
    return out


def symmetrize(A_full: np.ndarray, n: int, M: int = 2) -> np.ndarray:
    """The Hermitian-symmetric part (A + conj(A o conj)) / 2 of an arbitrary full tensor."""
    A_full = np.asarray(A_full)
    c = conj_index(np.arange((M * M) ** n, dtype=np.int64), n, M)
    return 0.5 * (A_full + np.conj(A_full[c]))
