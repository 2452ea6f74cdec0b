"""Tensor-propagator recurrence for rho(t) (oracle, FP64).  Test infrastructure only.

The reduced density matrix at t_N = N dt is the truncated path sum of Sec. II:

  rho_N(x_N) = sum_{x_0..x_{N-1}} rho0(x_0) prod_k K(x_{k+1}, x_k)
               * exp(- sum_{k=0}^{N} sum_{k'=max(0,k-L)}^{k} d(x_k)(eta_kk' s_k'^+ - conj(eta_kk') s_k'^-))

(memory truncation at distance L = Delta k_max; the printed outer limit of the
influence-functional sum is read as running over every point k = 0..N).  The
tensor propagator scheme (Sec. I, Makri-Makarov) evaluates it exactly with an
augmented tensor A_n holding the newest min(n+1, L) path points:

  A_0(x_0)  = rho0(x_0) exp(-d(x_0)(eta_00 s_0^+ - conj(eta_00) s_0^-))
  A_n       = T_n A_{n-1}: multiply by the factors that join the new point n
              to the stored points (K with the previous point, one I per pair
              at distance <= L, the self term), and, once A_{n-1} already holds
              L points (n >= L), sum over the oldest one.
  rho_N     = the same product for the final point N, with its end-point
              (Strang) eta values, summed over every stored point.

The end-point readout happens before the oldest index is summed, so rho at
any step N uses the half box [(N - 1/2) dt, N dt] of Eqs. etaNNgeneralStrang
and etaNkgeneralStrang, while A keeps propagating with interior eta values.
``endpoint='interior'`` instead reads rho with the final point treated as an
interior one.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import clib
from .eta import Spectral, eta_table, unpack_eta
from .system import (coupling_d, influence_factor, influence_self, pair_propagator_K,
                     propagator_U)


def _digit_points(n_in: int, n: int):
    """Path point held in each digit of the tensor A_{n-1} that feeds step n."""
    first = n - n_in
    return [first + p for p in range(n_in)]


def step_tables(eta: dict, s, K, L: int, n: int):
    """Per-digit factor tables for the step that adds path point n (n >= 1).

    Returns (G, g, n_in, summed): G[p] couples point n to the point in digit p
    of A_{n-1}; K is folded into the newest digit's table; g is point n's self
    factor with the interior eta; summed says whether digit 0 is summed.
    """
    n_in = min(n, L)
    M2 = len(s) ** 2
    G = np.empty((n_in, M2, M2), dtype=np.complex128)
    for p, point in enumerate(_digit_points(n_in, n)):
        dk = n - point
        e = eta["point0"][n - 1] if point == 0 else eta["interior"][dk]
        G[p] = influence_factor(e, s)
    G[n_in - 1] = G[n_in - 1] * K
    g = influence_self(eta["interior"][0], s)
    return G, g, n_in, n >= L


def readout_tables(eta: dict, s, K, L: int, N: int, endpoint: str = "strang"):
    """Per-digit factor tables that read rho_N out of A_{N-1} (N >= 1)."""
    n_in = min(N, L)
    M2 = len(s) ** 2
    G = np.empty((n_in, M2, M2), dtype=np.complex128)
    for p, point in enumerate(_digit_points(n_in, N)):
        dk = N - point
        if endpoint == "strang":
            e = eta["end_point0"][N - 1] if point == 0 else eta["end"][dk - 1]
        else:
            e = eta["point0"][N - 1] if point == 0 else eta["interior"][dk]
        G[p] = influence_factor(e, s)
    G[n_in - 1] = G[n_in - 1] * K
    g = influence_self(eta["end_self"] if endpoint == "strang" else eta["interior"][0], s)
    return G, g, n_in


def initial_tensor(eta: dict, s, rho0) -> np.ndarray:
    rho0 = np.asarray(rho0, dtype=np.complex128).reshape(-1)
    return rho0 * influence_self(eta["self0"], s)


def apply_step(A, G, g, n_in: int, summed: bool) -> np.ndarray:
    M2 = G.shape[1]
    if summed:
        out = np.empty(M2 ** n_in, dtype=np.complex128)
        return clib.call("oracle_step", M2, n_in, A, G, g, out)
    out = np.empty(M2 ** (n_in + 1), dtype=np.complex128)
    return clib.call("oracle_grow", M2, n_in, A, G, g, out)


def apply_readout(A, G, g, n_in: int) -> np.ndarray:
    M2 = G.shape[1]
    out = np.empty(M2, dtype=np.complex128)
    return clib.call("oracle_readout", M2, n_in, A, G, g, out)


@dataclass
class OracleRun:
    """One oracle problem: system, bath, discretisation (Sec. II's program inputs)."""

    s: np.ndarray
    H: np.ndarray
    spec: Spectral
    beta: float
    dt: float
    L: int
    eta: dict = None
    endpoint: str = "strang"
    K: np.ndarray = field(init=False)

    def __post_init__(self):
        self.s = np.asarray(self.s, dtype=np.float64)
        self.H = np.asarray(self.H, dtype=np.complex128)
        if self.eta is None:
            self.eta = eta_table(self.spec, self.beta, self.dt, self.L)
        elif not isinstance(self.eta, dict):
            self.eta = unpack_eta(self.eta, self.L)
        self.K = pair_propagator_K(propagator_U(self.H, self.dt))

    def run(self, rho0, steps, on_step=None):
        """rho at each requested step (dict step -> M x M matrix)."""
        M = len(self.s)
        steps = sorted(set(int(k) for k in steps))
        out = {}
        if not steps:
            return out
        N = steps[-1]
        want = set(steps)
        if 0 in want:
            out[0] = np.asarray(rho0, dtype=np.complex128).reshape(M, M).copy()
        A = initial_tensor(self.eta, self.s, rho0)
        for n in range(1, N + 1):
            if n in want:
                G, g, n_in = readout_tables(self.eta, self.s, self.K, self.L, n, self.endpoint)
                out[n] = apply_readout(A, G, g, n_in).reshape(M, M)
            if n < N:
                G, g, n_in, summed = step_tables(self.eta, self.s, self.K, self.L, n)
                A = apply_step(A, G, g, n_in, summed)
            if on_step is not None:
                on_step(n, A)
        return out


def propagate(s, H, spec, beta, dt, L, rho0, steps, eta=None, endpoint="strang"):
    """Convenience wrapper: rho at the requested steps for one problem."""
    return OracleRun(s, H, spec, beta, dt, L, eta=eta, endpoint=endpoint).run(rho0, steps)


def step_elements(A, G, g, n_in: int, summed: bool, indices):
    """Selected output entries of one step, each evaluated on its own (plain Python loops).

    For output index o = x_new * S + i (S = M2^(n_in - summed)), the entry is
    g[x_new] * prod over the kept digits of G[p][x_new][digit] times either
    A[i] (growth) or sum_{d0} G[0][x_new][d0] * A[i * M2 + d0] (summed step).
    """
    M2 = G.shape[1]
    kept = n_in - (1 if summed else 0)
    S = M2 ** kept
    out = []
    for o in indices:
        o = int(o)
        xn, i = divmod(o, S)
        prod = complex(g[xn])
        rest = i
        for q in range(kept):
            digit = rest % M2
            rest //= M2
            p = q + (1 if summed else 0)
            prod *= complex(G[p, xn, digit])
        if summed:
            acc = 0j
            for d0 in range(M2):
                acc += complex(G[0, xn, d0]) * complex(A[i * M2 + d0])
            out.append(prod * acc)
        else:
            out.append(prod * complex(A[i]))
    return np.array(out, dtype=np.complex128)
