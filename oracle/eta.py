"""eta coefficients of the discretised influence functional (oracle, FP64).

Test infrastructure only.

Sec. II defines the bath response function (Eq. bathResponseFunction)

    alpha(t) = (1/pi) int_0^inf J(w) [coth(beta w / 2) cos(w t) - i sin(w t)] dw

and each eta_{kk'} as the double integral of alpha(t' - t'') over the time box
of the later point (t') and the box of the earlier point (t''); for k = k' the
inner integral stops at t' (Eqs. etaKK'generalTrotter .. etaNkgeneralStrang).

Swapping the order of integration gives one frequency integral per box pair.
For disjoint boxes of widths w1 (later) and w2 (earlier) whose centres are a
distance D apart, int int e^{i w (t'-t'')} = e^{i w D} 4 sin(w w1/2) sin(w w2/2) / w^2, so

    eta = (1/pi) int J(w)/w^2 * 4 sin(w w1/2) sin(w w2/2)
                          * [coth(beta w/2) cos(w D) - i sin(w D)] dw ,

and for a box of width w with itself
int_0^w dt' int_0^t' cos(w u) du = (1 - cos w w)/w^2 and the sine analogue
(w w - sin w w)/w^2, so

    eta_self = (1/pi) int J(w)/w^2 [coth(beta w/2)(1 - cos w w) + i (sin w w - w w)] dw .

Box placement (reading of Eqs. etaN0generalStrang .. etaNkgeneralStrang, which
label the end boxes "Strang"): point 0 owns [0, dt/2], an interior point k owns
[(k - 1/2) dt, (k + 1/2) dt] and the final point N owns [(N - 1/2) dt, N dt].
This is the placement under which the boxes tile [0, N dt] exactly.  The
interior formula as printed ([k dt, (k+1) dt]) gives the same interior-interior
values because alpha depends only on t' - t''.  eta_00's upper limit, printed
as "t", is read as dt/2 (Eq. eta00generalStrang, consistent with its
neighbours).
"""

from __future__ import annotations

import math
import warnings
from dataclasses import dataclass

import numpy as np
from scipy import integrate

OHMIC_EXP = "ohmic_exp"            # J = (pi/2) a w exp(-w/wc)
SUPEROHMIC_GAUSS = "superohmic_gauss"  # J = a w^3 exp(-(w/wc)^2)  (Eq. superOhmicJwithGaussianCutoff)
TABULATED = "tabulated"            # J piecewise linear through (0, 0) and the table, 0 above its last node


@dataclass(frozen=True)
class Spectral:
    """Spectral distribution function J(w) (Eq. spectralDistribution): a parametric form, or a
    table (omega ascending, omega[0] > 0) read as the piecewise-linear function through (0, 0)
    and (omega[i], values[i]), zero above omega[-1]."""

    kind: str
    a: float = 0.0
    wc: float = 1.0
    omega: tuple = ()
    values: tuple = ()

    @staticmethod
    def tabulated(omega, values) -> "Spectral":
        return Spectral(TABULATED, omega=tuple(float(x) for x in omega), values=tuple(float(x) for x in values))

    def J_over_w2(self, w):
        """J(w)/w^2, written so that it stays finite and accurate as w -> 0."""
        w = np.asarray(w, dtype=np.float64)
        if self.kind == OHMIC_EXP:
            return (math.pi / 2.0) * self.a * np.exp(-w / self.wc) / w
        if self.kind == SUPEROHMIC_GAUSS:
            return self.a * w * np.exp(-(w / self.wc) ** 2)
        if self.kind == TABULATED:
            return self.J(w) / (w * w)
        raise ValueError(f"unknown spectral density kind {self.kind!r}")

    def J(self, w):
        w = np.asarray(w, dtype=np.float64)
        if self.kind == TABULATED:
            xp = np.concatenate([[0.0], np.asarray(self.omega)])
            fp = np.concatenate([[0.0], np.asarray(self.values)])
            return np.interp(w, xp, fp, right=0.0)
        return self.J_over_w2(w) * w * w

    def omega_max(self) -> float:
        """Upper frequency limit: the table's last node, or where J's cutoff factor is below ~1e-18."""
        if self.kind == TABULATED:
            return float(self.omega[-1])
        if self.kind == OHMIC_EXP:
            return 42.0 * self.wc
        return 7.0 * self.wc


def _coth_half(beta: float, w):
    """coth(beta w / 2); beta = inf means zero temperature (coth -> 1)."""
    if math.isinf(beta):
        return np.ones_like(w)
    return 1.0 / np.tanh(0.5 * beta * w)


def _sin_minus_x(x):
    """sin(x) - x without cancellation for small |x| (Taylor series below |x| = 1)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.sin(x) - x
    small = np.abs(x) < 1.0
    if np.any(small):
        xs = x[small]
        x2 = xs * xs
        term = -xs * x2 / 6.0
        acc = term.copy()
        for k in range(2, 12):
            term = -term * x2 / ((2 * k) * (2 * k + 1))
            acc = acc + term
        out[small] = acc
    return out


def _quad(f, a, b, breaks):
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        val, _err = integrate.quad(f, a, b, epsabs=1e-17, epsrel=1e-14, limit=4000,
                                   points=breaks if breaks else None)
    return val


def _breaks(spec: Spectral, wmax: float):
    if spec.kind == TABULATED:  # J has a kink at every node
        return [x for x in spec.omega if 0.0 < x < wmax]
    # a few fixed interior break points around the cutoff scale help QUADPACK
    pts = [x * spec.wc for x in (0.25, 1.0, 3.0, 8.0, 20.0) if x * spec.wc < wmax]
    return pts


def eta_pair(spec: Spectral, beta: float, w1: float, w2: float, D: float) -> complex:
    """eta for two disjoint boxes (widths w1 later, w2 earlier, centre distance D)."""
    wmax = spec.omega_max()

    def common(w):
        return spec.J_over_w2(w) * 4.0 * np.sin(0.5 * w * w1) * np.sin(0.5 * w * w2) / math.pi

    def f_re(w):
        return float(common(w) * _coth_half(beta, w) * np.cos(w * D))

    def f_im(w):
        return float(-common(w) * np.sin(w * D))

    br = _breaks(spec, wmax)
    return complex(_quad(f_re, 0.0, wmax, br), _quad(f_im, 0.0, wmax, br))


def eta_self(spec: Spectral, beta: float, w: float) -> complex:
    """eta of a box of width w with itself (inner integral up to t')."""
    wmax = spec.omega_max()

    def f_re(x):
        one_minus_cos = 2.0 * np.sin(0.5 * x * w) ** 2
        return float(spec.J_over_w2(x) * _coth_half(beta, x) * one_minus_cos / math.pi)

    def f_im(x):
        return float(spec.J_over_w2(x) * _sin_minus_x(np.array([x * w]))[0] / math.pi)

    br = _breaks(spec, wmax)
    return complex(_quad(f_re, 0.0, wmax, br), _quad(f_im, 0.0, wmax, br))


def eta_boxes(spec: Spectral, beta: float, later, earlier) -> complex:
    """eta over the box ``later`` = (a, b) for t' and ``earlier`` = (c, d) for t''.

    Identical boxes give the self term (t'' < t'); otherwise the boxes must be
    disjoint with the earlier one first.
    """
    a, b = later
    c, d = earlier
    if abs(a - c) < 1e-15 and abs(b - d) < 1e-15:
        return eta_self(spec, beta, b - a)
    if d > a + 1e-12 * max(1.0, abs(a)):
        raise ValueError("boxes overlap or are out of order")
    return eta_pair(spec, beta, b - a, d - c, 0.5 * (a + b) - 0.5 * (c + d))


def strang_box(k: int, N: int, dt: float, endpoint: str = "strang"):
    """Time box owned by path point k of a path ending at N.

    endpoint='strang': point 0 -> [0, dt/2], 0<k<N -> [(k-1/2)dt, (k+1/2)dt],
    point N -> [(N-1/2)dt, N dt].  endpoint='interior': the final point is
    treated like an interior one, [(N-1/2)dt, (N+1/2)dt].
    """
    if k == 0:
        return (0.0, 0.5 * dt)
    if k == N and endpoint == "strang":
        return ((N - 0.5) * dt, N * dt)
    return ((k - 0.5) * dt, (k + 0.5) * dt)


def eta_table(spec: Spectral, beta: float, dt: float, L: int) -> dict:
    """Every eta the tensor propagator with memory length L needs (4L+3 values).

    Keys (each computed from explicit boxes, Strang placement):
      interior[dk], dk = 0..L   -- eta_{k,k-dk} for two interior points (dk = 0: self box)
      point0[k-1],  k = 1..L    -- eta_{k0}: interior point k with point 0 (Eq. etaK0generalStrang)
      end_self                  -- eta_NN (Eq. etaNNgeneralStrang)
      end[dk-1],    dk = 1..L   -- eta_{N,N-dk}: final point with an interior point (Eq. etaNkgeneralStrang)
      end_point0[N-1], N = 1..L -- eta_{N0}: final point with point 0 (Eq. etaN0generalStrang)
      self0                     -- eta_00 (Eq. eta00generalStrang, upper limit read as dt/2)
    """
    far = 10 * (L + 2)  # any interior index well inside the path: alpha is stationary
    interior = [eta_boxes(spec, beta, strang_box(far, 10 * far, dt), strang_box(far, 10 * far, dt))]
    for dk in range(1, L + 1):
        interior.append(eta_boxes(spec, beta, strang_box(far + dk, 10 * far, dt),
                                  strang_box(far, 10 * far, dt)))
    point0 = [eta_boxes(spec, beta, strang_box(k, 10 * far, dt), strang_box(0, 10 * far, dt))
              for k in range(1, L + 1)]
    Nf = far  # a final point far from 0
    end_self = eta_boxes(spec, beta, strang_box(Nf, Nf, dt), strang_box(Nf, Nf, dt))
    end = [eta_boxes(spec, beta, strang_box(Nf, Nf, dt), strang_box(Nf - dk, Nf, dt))
           for dk in range(1, L + 1)]
    end_point0 = [eta_boxes(spec, beta, strang_box(N, N, dt), strang_box(0, N, dt))
                  for N in range(1, L + 1)]
    self0 = eta_boxes(spec, beta, strang_box(0, Nf, dt), strang_box(0, Nf, dt))
    return dict(L=L, interior=np.array(interior), point0=np.array(point0),
                end_self=complex(end_self), end=np.array(end),
                end_point0=np.array(end_point0), self0=complex(self0))


def pack_eta(tab: dict) -> np.ndarray:
    """Flatten an eta table into the 4L+3 order of the C ABI's eta input.

    Order: interior[0..L], point0[0..L-1], end_self, end[0..L-1],
    end_point0[0..L-1], self0.
    """
    return np.concatenate([tab["interior"], tab["point0"], [tab["end_self"]], tab["end"],
                           tab["end_point0"], [tab["self0"]]]).astype(np.complex128)


def unpack_eta(v, L: int) -> dict:
    v = np.asarray(v, dtype=np.complex128)
    if v.shape != (4 * L + 3,):
        raise ValueError("eta vector must have 4L+3 entries")
    o = 0
    interior = v[o:o + L + 1]; o += L + 1
    point0 = v[o:o + L]; o += L
    end_self = complex(v[o]); o += 1
    end = v[o:o + L]; o += L
    end_point0 = v[o:o + L]; o += L
    self0 = complex(v[o])
    return dict(L=L, interior=interior, point0=point0, end_self=end_self, end=end,
                end_point0=end_point0, self0=self0)
