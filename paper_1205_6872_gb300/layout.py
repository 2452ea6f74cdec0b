"""Hermitian half layout of the augmented tensor (M = 2), host-side conversion helpers.

Swapping the forward and backward path of every point (x = (s+, s-) -> x-bar =
(s-, s+)) conjugates a path's weight (K and every influence factor go to their
complex conjugates), so for a Hermitian rho(0) the tensor obeys
A(x-bar_1 .. x-bar_n) = conj(A(x_1 .. x_n)).  For M = 2 the point values are
0 = (+,+), 1 = (+,-), 2 = (-,+), 3 = (-,-); conjugation swaps 1 and 2 and keeps
0 and 3.  An index is *canonical* when its most significant digit that is not
0 or 3 is a 1; indices made only of 0s and 3s are their own conjugates (their
entries are real).  Only canonical entries are stored, in this recursive order
for n digits (most significant first):

    [top digit 1: all 4^(n-1) continuations, plain base-4 order]
    [top digit 0: the canonical layout of the remaining n-1 digits]
    [top digit 3: the canonical layout of the remaining n-1 digits]

giving C(n) = (4^n + 2^n) / 2 entries instead of 4^n.  Consequently the
fibers of the last digit stay contiguous (4 entries, or 3 for a
self-conjugate prefix, stored as last digit 1, 0, 3).

These helpers convert between the full and the half layout (used by tests,
checkpoints and callers that inspect tensors); the device kernels compute the
same positions themselves.
"""

from __future__ import annotations

import numpy as np


def count(n: int) -> int:
    """C(n): canonical entries of an n-digit tensor."""
    return (4 ** n + 2 ** n) // 2


def canonical_indices(n: int) -> np.ndarray:
    """Plain (full-layout) indices of the canonical entries, in half-layout order."""
    if n == 0:
        return np.zeros(1, dtype=np.int64)
    sub = canonical_indices(n - 1)
    top = 4 ** (n - 1)
    return np.concatenate([1 * top + np.arange(top, dtype=np.int64), 0 * top + sub, 3 * top + sub])


def to_half(A_full: np.ndarray, n: int) -> np.ndarray:
    """Full tensor (4^n entries) -> half layout (C(n) entries)."""
    A_full = np.asarray(A_full)
    if A_full.shape[0] != 4 ** n:
        raise ValueError("full tensor must have 4^n entries")
    return A_full[canonical_indices(n)]


def conj_index(idx: np.ndarray, n: int) -> np.ndarray:
    """Plain index of the conjugate path (digits 1 <-> 2 in every position)."""
    idx = np.asarray(idx, dtype=np.int64)
    lo_bits = idx & int("01" * n or "0", 2)
    hi_bits = idx & int("10" * n or "0", 2)
    return (lo_bits << 1) | (hi_bits >> 1)


def from_half(A_half: np.ndarray, n: int) -> np.ndarray:
    """Half layout -> full tensor, filling conjugate entries as conj(A)."""
    A_half = np.asarray(A_half)
    idx = canonical_indices(n)
    out = np.empty(4 ** n, dtype=np.result_type(A_half.dtype, np.complex64))
    out[idx] = A_half
    out[conj_index(idx, n)] = np.conj(A_half)
    out[idx] = A_half
    return out


def symmetrize(A_full: np.ndarray, n: int) -> np.ndarray:
    """The Hermitian-symmetric part (A + conj(A o conj)) / 2 of an arbitrary full tensor."""
    A_full = np.asarray(A_full)
    c = conj_index(np.arange(4 ** n, dtype=np.int64), n)
    return 0.5 * (A_full + np.conj(A_full[c]))
