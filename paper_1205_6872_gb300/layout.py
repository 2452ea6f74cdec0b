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

giving C(n) = (4^n + 2^n) / 2 canonical indices.  The device layout keeps
whole fibers of the last digit: for n >= 1 it stores, for every canonical
prefix of n - 1 digits in the order above, the 4 entries of its fiber (a
prefix of only 0s and 3s also keeps its redundant last digit 2, the
conjugate of its last digit 1).  That is 4 C(n-1) entries (1 for n = 0),
every fiber is 4 consecutive, aligned entries, and canonical prefix c
starts at entry 4 c.

These helpers convert between the full and the half layout (used by tests,
checkpoints and callers that inspect tensors); the device kernels compute the
same positions themselves.
"""

from __future__ import annotations

import numpy as np


def canonical_count(n: int) -> int:
    """C(n): canonical n-digit indices."""
    return (4 ** n + 2 ** n) // 2


def count(n: int) -> int:
    """Entries of the device half layout of an n-digit tensor."""
    return 1 if n == 0 else 4 * canonical_count(n - 1)


def canonical_order(n: int) -> np.ndarray:
    """Plain indices of the canonical n-digit indices, in half-layout order."""
    if n == 0:
        return np.zeros(1, dtype=np.int64)
    sub = canonical_order(n - 1)
    top = 4 ** (n - 1)
    return np.concatenate([1 * top + np.arange(top, dtype=np.int64), 0 * top + sub, 3 * top + sub])


def canonical_indices(n: int) -> np.ndarray:
    """Plain (full-layout) index of every entry of the device half layout, in order."""
    if n == 0:
        return np.zeros(1, dtype=np.int64)
    prefixes = canonical_order(n - 1)
    return (4 * prefixes[:, None] + np.arange(4, dtype=np.int64)[None, :]).reshape(-1)


def to_half(A_full: np.ndarray, n: int) -> np.ndarray:
    """Full tensor (4^n entries) -> device half layout (count(n) entries)."""
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
    """Half layout -> full tensor, filling the missing entries as conjugates of stored ones."""
    A_half = np.asarray(A_half)
    idx = canonical_indices(n)
    out = np.empty(4 ** n, dtype=np.result_type(A_half.dtype, np.complex64))
    out[conj_index(idx, n)] = np.conj(A_half)
    out[idx] = A_half
    return out


def symmetrize(A_full: np.ndarray, n: int) -> np.ndarray:
    """The Hermitian-symmetric part (A + conj(A o conj)) / 2 of an arbitrary full tensor."""
    A_full = np.asarray(A_full)
    c = conj_index(np.arange(4 ** n, dtype=np.int64), n)
    return 0.5 * (A_full + np.conj(A_full[c]))
