"""Bare system propagators (oracle, FP64).  Test infrastructure only.

The path-integral expression for <s_N^+|rho(t)|s_N^->  (Sec. II) carries, per
time step, the forward factor <s_{k+1}^+| e^{-i H dt} |s_k^+> and the backward
factor <s_k^-| e^{+i H dt} |s_{k+1}^-> = conj(<s_{k+1}^-| e^{-i H dt} |s_k^->).
The basis is the one H is given in, whose coordinate eigenvalues are s.

A path point x = (s^+, s^-) is stored as the flat index x = i_plus * M + i_minus,
the row-major position of rho[i_plus, i_minus].
"""

from __future__ import annotations

import numpy as np


def propagator_U(H, dt: float) -> np.ndarray:
    """U = exp(-i H dt) for Hermitian H, by eigendecomposition (numpy eigh)."""
    H = np.asarray(H, dtype=np.complex128)
    if not np.allclose(H, H.conj().T, atol=1e-12, rtol=0):
        raise ValueError("H must be Hermitian")
    lam, V = np.linalg.eigh(H)
    return (V * np.exp(-1j * lam * dt)) @ V.conj().T


def pair_propagator_K(U) -> np.ndarray:
    """K[x', x] = U[a', a] * conj(U[b', b]) with x' = a' M + b', x = a M + b."""
    U = np.asarray(U, dtype=np.complex128)
    M = U.shape[0]
    K = np.empty((M * M, M * M), dtype=np.complex128)
    for ap in range(M):
        for bp in range(M):
            for a in range(M):
                for b in range(M):
                    K[ap * M + bp, a * M + b] = U[ap, a] * np.conj(U[bp, b])
    return K


def coupling_d(s):
    """Per path point x: (s^+, s^-, d = s^+ - s^-) as arrays over the M^2 flat indices."""
    s = np.asarray(s, dtype=np.float64)
    M = s.shape[0]
    sp = np.repeat(s, M)
    sm = np.tile(s, M)
    return sp, sm, sp - sm


def influence_factor(eta: complex, s, ) -> np.ndarray:
    """I[x_later, x_earlier] = exp(-d(x_later) (eta s^+(x_earlier) - conj(eta) s^-(x_earlier))).

    One pair term of the discretised influence functional (Sec. II, Eq. for I).
    """
    sp, sm, d = coupling_d(s)
    return np.exp(-d[:, None] * (eta * sp[None, :] - np.conj(eta) * sm[None, :]))


def influence_self(eta: complex, s) -> np.ndarray:
    """The k = k' term: exp(-d(x) (eta s^+(x) - conj(eta) s^-(x))) per point x."""
    sp, sm, d = coupling_d(s)
    return np.exp(-d * (eta * sp - np.conj(eta) * sm))
