"""The truncated path sum by explicit enumeration of every path (oracle).  Test infrastructure only.

Evaluates, for tiny N, the path-integral expression of Sec. II directly:

  rho_N(x_N) = sum over all (x_0 .. x_{N-1}) of
      rho0(x_0) * prod_{k=0}^{N-1} K(x_{k+1}, x_k)
      * exp(- sum_{k=0}^{N} sum_{k'=max(0,k-L)}^{k} d(x_k) (eta_kk' s_k'^+ - conj(eta_kk') s_k'^-))

with each eta_kk' computed from the two time boxes of points k and k' of this
particular path length N (``strang_box``), with no interior / point-0 / end
classification.  It is independent of the tensor recurrence's bookkeeping.
"""

from __future__ import annotations

import numpy as np

from .eta import eta_boxes, strang_box
from .system import coupling_d, pair_propagator_K, propagator_U


def rho_bruteforce(s, H, spec, beta, dt, L, rho0, N, endpoint="strang", eta_fn=None):
    """rho at step N (M x M) by summing all (M^2)^N paths; ``eta_fn(later, earlier)`` may override eta."""
    s = np.asarray(s, dtype=np.float64)
    M = len(s)
    M2 = M * M
    rho0 = np.asarray(rho0, dtype=np.complex128).reshape(-1)
    if N == 0:
        return rho0.reshape(M, M).copy()
    if eta_fn is None:
        def eta_fn(later, earlier):
            return eta_boxes(spec, beta, later, earlier)
    K = pair_propagator_K(propagator_U(H, dt))
    sp, sm, d = coupling_d(s)
    boxes = [strang_box(k, N, dt, endpoint) for k in range(N + 1)]
    # every path as digits x_0..x_N
    npaths = M2 ** (N + 1)
    idx = np.arange(npaths, dtype=np.int64)
    x = np.empty((N + 1, npaths), dtype=np.int64)
    for k in range(N + 1):
        x[k] = (idx // (M2 ** k)) % M2
    w = rho0[x[0]].copy()
    for k in range(N):
        w *= K[x[k + 1], x[k]]
    expo = np.zeros(npaths, dtype=np.complex128)
    cache = {}
    for k in range(N + 1):
        for kp in range(max(0, k - L), k + 1):
            key = (boxes[k], boxes[kp])
            if key not in cache:
                cache[key] = eta_fn(boxes[k], boxes[kp])
            e = cache[key]
            expo += d[x[k]] * (e * sp[x[kp]] - np.conj(e) * sm[x[kp]])
    w *= np.exp(-expo)
    rho = np.zeros(M2, dtype=np.complex128)
    np.add.at(rho, x[N], w)
    return rho.reshape(M, M)
