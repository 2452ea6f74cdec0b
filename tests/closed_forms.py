"""Closed forms that pin the oracle independently of its quadrature and recurrence.

Derivations (hbar = k_B = 1):

Ohmic bath with exponential cutoff, J(w) = (pi/2) a w e^{-w/wc}.  Expanding
coth(beta w/2) = 1 + 2 sum_{n>=1} e^{-n beta w} in the bath response function
(Sec. II, Eq. bathResponseFunction) and using int_0^inf w e^{-z w} dw = 1/z^2:

    Re alpha(tau) = (a/2) sum_{n>=0} c_n Re[1/(p_n + i tau)^2],   Im alpha(tau) = (a/2) Im[1/(p_0 + i tau)^2],
    p_n = 1/wc + n beta,  c_0 = 1,  c_n = 2.

Since 1/(p + i tau)^2 = F''(tau) with F(tau) = ln(p + i tau), the double
integral over later box [a, b] and earlier box [c, d] is
F(b-c) - F(a-c) - F(b-d) + F(a-d); over one box of width w with t'' < t' it
is F(w) - F(0) - w F'(0).  The n >= 1 tail sums in closed form through
ln|Gamma| because prod_{n>=1} (n + z_j) telescopes when sum_j e_j = 0.
At zero temperature (beta = inf) only the n = 0 term remains.

Two-level Hamiltonian H = [[eps, W], [W, -eps]]: H^2 = (eps^2 + W^2) I, so
exp(-i H t) = cos(w t) I - i sin(w t) H / w with w = sqrt(eps^2 + W^2).
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import loggamma


def _F(p, tau):
    return np.log(p + 1j * tau)


def eta_box_ohmic(a, wc, beta, later, earlier):
    """Closed-form eta for the Ohmic bath over two boxes (or one box with itself)."""
    A, B = later
    C, D = earlier
    p0 = 1.0 / wc
    if abs(A - C) < 1e-15 and abs(B - D) < 1e-15:
        w = B - A
        zero_T = _F(p0, w) - _F(p0, 0.0) - w * 1j / p0
        val = 0.5 * a * zero_T
        if not math.isinf(beta):
            z0 = p0 / beta
            zw = (p0 + 1j * w) / beta
            tail = loggamma(1.0 + z0).real - loggamma(1.0 + zw).real
            val += 0.5 * a * 2.0 * tail
        return complex(val)
    taus = [B - C, A - C, B - D, A - D]
    e = [1.0, -1.0, -1.0, 1.0]
    zero_T = sum(ej * _F(p0, t) for ej, t in zip(e, taus))
    val = 0.5 * a * zero_T
    if not math.isinf(beta):
        tail = -sum(ej * loggamma(1.0 + (p0 + 1j * t) / beta).real for ej, t in zip(e, taus))
        val += 0.5 * a * 2.0 * tail
    return complex(val)


def U_two_level(eps, W, t):
    w = math.sqrt(eps * eps + W * W)
    H = np.array([[eps, W], [W, -eps]], dtype=np.complex128)
    return math.cos(w * t) * np.eye(2) - 1j * math.sin(w * t) / w * H


def strang_boxes(N, dt):
    """Time boxes of points 0..N of a path ending at N (0: [0, dt/2]; N: [(N-1/2)dt, N dt])."""
    out = [(0.0, 0.5 * dt)]
    for k in range(1, N):
        out.append(((k - 0.5) * dt, (k + 0.5) * dt))
    out.append(((N - 0.5) * dt, N * dt))
    return out


def pure_dephasing_rho(s, E, rho0, a, wc, beta, dt, L, N):
    """rho(N dt) for diagonal H = diag(E): only constant paths survive.

    rho_ab(t) = rho_ab(0) e^{-i (E_a - E_b) t} exp(-(s_a - s_b)(s_a Phi - s_b conj(Phi))),
    Phi = sum of eta over every pair of boxes at distance <= L (for L >= N this
    is the self term of the single box [0, t], because the boxes tile [0, t]).
    """
    s = np.asarray(s, float)
    M = len(s)
    if N == 0:
        return np.asarray(rho0, complex).copy()
    boxes = strang_boxes(N, dt)
    if L >= N:
        Phi = eta_box_ohmic(a, wc, beta, (0.0, N * dt), (0.0, N * dt))
    else:
        Phi = 0.0
        for k in range(N + 1):
            for kp in range(max(0, k - L), k + 1):
                Phi += eta_box_ohmic(a, wc, beta, boxes[k], boxes[kp])
    out = np.empty((M, M), dtype=np.complex128)
    for i in range(M):
        for j in range(M):
            out[i, j] = rho0[i, j] * np.exp(-1j * (E[i] - E[j]) * N * dt) * np.exp(
                -(s[i] - s[j]) * (s[i] * Phi - s[j] * np.conj(Phi)))
    return out
