"""Pins for the oracle's eta coefficients (CPU only).

* Ohmic bath: closed forms at zero and finite temperature (closed_forms.py),
  which use logarithms and ln|Gamma| instead of any frequency quadrature.
* Any bath: a direct 2-D Gauss-Legendre integration over the two time boxes of
  alpha(t' - t''), with alpha evaluated from its definition (Sec. II, Eq.
  bathResponseFunction).  This checks the oracle's reduction of the double
  integral to one frequency integral (the 4 sin sin / w^2 and self-box kernels).
* Strang tiling: the eta of every pair of boxes of a path sums to the single
  self-box eta of [0, t] (the boxes tile the triangle t'' < t' exactly).
"""

import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle.eta import Spectral, eta_boxes, strang_box
from closed_forms import eta_box_ohmic, strang_boxes

OHMIC_CASES = [(0.3, 5.0), (0.1, 7.5), (0.5, 2.5)]


@pytest.mark.parametrize("a,wc", OHMIC_CASES)
@pytest.mark.parametrize("beta", [math.inf, 5.0, 1.0, 0.5])
def test_self_box_closed_form(a, wc, beta):
    sp = Spectral("ohmic_exp", a, wc)
    for w in (0.05, 0.125, 0.25, 1.0, 3.0):
        got = eta_boxes(sp, beta, (1.0, 1.0 + w), (1.0, 1.0 + w))
        want = eta_box_ohmic(a, wc, beta, (1.0, 1.0 + w), (1.0, 1.0 + w))
        assert abs(got - want) <= 1e-14 * max(1.0, abs(want)), (w, got, want)


@pytest.mark.parametrize("a,wc", OHMIC_CASES)
@pytest.mark.parametrize("beta", [math.inf, 5.0, 1.0, 0.5])
def test_disjoint_boxes_closed_form(a, wc, beta):
    sp = Spectral("ohmic_exp", a, wc)
    dt = 0.15
    cases = [
        (strang_box(3, 99, dt), strang_box(2, 99, dt)),      # interior neighbours
        (strang_box(9, 99, dt), strang_box(1, 99, dt)),      # interior, distance 8
        (strang_box(5, 99, dt), strang_box(0, 99, dt)),      # interior with point 0
        (strang_box(7, 7, dt), strang_box(6, 7, dt)),        # end point with neighbour
        (strang_box(7, 7, dt), strang_box(0, 7, dt)),        # end point with point 0
        (strang_box(1, 1, dt), strang_box(0, 1, dt)),        # N = 1: two half boxes
        (strang_box(40, 99, dt), strang_box(1, 99, dt)),     # far apart
    ]
    for later, earlier in cases:
        got = eta_boxes(sp, beta, later, earlier)
        want = eta_box_ohmic(a, wc, beta, later, earlier)
        assert abs(got - want) <= 2e-15 + 1e-12 * abs(want), (later, earlier, got, want)


def _alpha(spec, beta, t):
    """alpha(t) straight from its definition (coth cos - i sin form)."""
    wmax = spec.omega_max()

    def re(w):
        return spec.J(w) * (1.0 / math.tanh(0.5 * beta * w)) * math.cos(w * t) / math.pi

    def im(w):
        return -spec.J(w) * math.sin(w * t) / math.pi

    kw = dict(epsabs=1e-15, epsrel=1e-13, limit=2000)
    return complex(integrate.quad(re, 0.0, wmax, **kw)[0], integrate.quad(im, 0.0, wmax, **kw)[0])


def _box_2d(spec, beta, later, earlier, n=12):
    x, wgt = np.polynomial.legendre.leggauss(n)
    a, b = later
    c, d = earlier
    tp = 0.5 * (b - a) * x + 0.5 * (a + b)
    wp = 0.5 * (b - a) * wgt
    total = 0.0
    same = abs(a - c) < 1e-15 and abs(b - d) < 1e-15
    for t1, w1 in zip(tp, wp):
        hi = t1 if same else d
        lo = c
        tq = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        wq = 0.5 * (hi - lo) * wgt
        for t2, w2 in zip(tq, wq):
            total += w1 * w2 * _alpha(spec, beta, t1 - t2)
    return total


@pytest.mark.parametrize("spec,beta", [
    (Spectral("superohmic_gauss", 0.05, 2.0), 2.0),
    (Spectral("ohmic_exp", 0.3, 1.0), 1.0),
])
def test_box_integral_of_alpha(spec, beta):
    dt = 0.2
    for later, earlier in [(strang_box(3, 9, dt), strang_box(1, 9, dt)),
                           (strang_box(2, 9, dt), strang_box(0, 9, dt)),
                           (strang_box(4, 4, dt), strang_box(3, 4, dt)),
                           (strang_box(2, 9, dt), strang_box(2, 9, dt)),
                           (strang_box(0, 9, dt), strang_box(0, 9, dt))]:
        got = eta_boxes(spec, beta, later, earlier)
        want = _box_2d(spec, beta, later, earlier)
        assert abs(got - want) <= 1e-11 * max(1.0, abs(want)), (later, earlier, got, want)


@pytest.mark.parametrize("spec,beta", [
    (Spectral("superohmic_gauss", 0.05, 2.0), 2.0),
    (Spectral("ohmic_exp", 0.5, 2.5), 0.5),
])
@pytest.mark.parametrize("N", [1, 2, 5])
def test_strang_boxes_tile_the_triangle(spec, beta, N):
    dt = 0.2
    boxes = strang_boxes(N, dt)
    total = 0.0
    for k in range(N + 1):
        for kp in range(k + 1):
            total += eta_boxes(spec, beta, boxes[k], boxes[kp])
    whole = eta_boxes(spec, beta, (0.0, N * dt), (0.0, N * dt))
    assert abs(total - whole) <= 1e-13 * max(1.0, abs(whole))


def test_eta_table_layout_roundtrip():
    sp = Spectral("ohmic_exp", 0.3, 5.0)
    tab = oracle.eta_table(sp, 1.0, 0.1, 5)
    v = oracle.pack_eta(tab)
    assert v.shape == (4 * 5 + 3,)
    back = oracle.unpack_eta(v, 5)
    for k in ("interior", "point0", "end", "end_point0"):
        assert np.array_equal(back[k], tab[k])
    # eta_00 and eta_NN are both half-box self terms: equal by stationarity
    assert abs(tab["self0"] - tab["end_self"]) < 1e-16
    # the first interior entry is the full-box self term
    assert abs(tab["interior"][0] - eta_box_ohmic(0.3, 5.0, 1.0, (0, 0.1), (0, 0.1))) < 1e-15


# ---------------------------------------------------------------- tabulated J(w)

def _cin(x):
    """Cin(x) = int_0^x (1 - cos t)/t dt = gamma + ln x - Ci(x) (series near 0)."""
    from scipy.special import sici
    x = abs(float(x))
    if x == 0.0:
        return 0.0
    if x < 1e-2:
        return x * x / 4.0 - x ** 4 / 96.0 + x ** 6 / 4320.0
    return np.euler_gamma + math.log(x) - sici(x)[1]


def _si(x):
    from scipy.special import sici
    return float(sici(float(x))[0])


def _ramp_self(c, Om, w):
    """Zero temperature, J = c w on [0, Om] and 0 above: self-box eta via Si and Cin."""
    return (c / math.pi) * complex(_cin(Om * w), _si(Om * w) - Om * w)


def _ramp_pair(c, Om, w1, w2, D):
    """Zero temperature, the same J: disjoint boxes (4 sin sin = 2 (cos wu - cos wv), u, v the half
    difference and half sum of the widths), reduced to Cin and Si of (D +- u) Om, (D +- v) Om."""
    u, v = 0.5 * (w1 - w2), 0.5 * (w1 + w2)
    re = _cin((D + v) * Om) - _cin((D + u) * Om) + _cin((D - v) * Om) - _cin((D - u) * Om)
    im = -(_si((D + u) * Om) + _si((D - u) * Om) - _si((D + v) * Om) - _si((D - v) * Om))
    return (c / math.pi) * complex(re, im)


def test_tabulated_table_reading():
    sp = Spectral.tabulated([0.5, 1.0, 3.0], [2.0, 1.0, 4.0])
    assert sp.J(np.array([0.0, 0.25, 0.5, 0.75, 1.0, 2.0, 3.0, 3.5]))[0] == 0.0
    np.testing.assert_allclose(sp.J(np.array([0.25, 0.5, 0.75, 1.0, 2.0, 3.0, 3.5])),
                               [1.0, 2.0, 1.5, 1.0, 2.5, 4.0, 0.0], rtol=0, atol=1e-15)
    assert sp.omega_max() == 3.0


@pytest.mark.parametrize("Om,nodes", [(6.0, 2), (25.0, 9)])
def test_tabulated_linear_ramp_closed_form(Om, nodes):
    """A table on the line J = c w (any node count: the same function) at zero temperature against
    the sine and cosine integrals, for every box pair kind the propagator uses."""
    c = 0.4
    om = np.linspace(Om / nodes, Om, nodes)
    sp = Spectral.tabulated(om, c * om)
    dt = 0.2
    for w in (0.5 * dt, dt):
        got = eta_boxes(sp, math.inf, (1.0, 1.0 + w), (1.0, 1.0 + w))
        want = _ramp_self(c, Om, w)
        assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (w, got, want)
    cases = [
        (strang_box(3, 99, dt), strang_box(2, 99, dt)),      # touching interior boxes (D - v = 0)
        (strang_box(9, 99, dt), strang_box(1, 99, dt)),
        (strang_box(5, 99, dt), strang_box(0, 99, dt)),      # with point 0 (half box)
        (strang_box(7, 7, dt), strang_box(6, 7, dt)),        # end point (half box)
        (strang_box(1, 1, dt), strang_box(0, 1, dt)),        # two half boxes
    ]
    for later, earlier in cases:
        w1, w2 = later[1] - later[0], earlier[1] - earlier[0]
        D = 0.5 * (later[0] + later[1]) - 0.5 * (earlier[0] + earlier[1])
        got = eta_boxes(sp, math.inf, later, earlier)
        want = _ramp_pair(c, Om, w1, w2, D)
        assert abs(got - want) <= 1e-14 + 1e-12 * abs(want), (later, earlier, got, want)


def test_tabulated_ohmic_converges_to_parametric():
    """A table of the Ohmic J on [0, 20 wc] approaches the parametric eta as the nodes get denser
    (linear interpolation: error ~ h^2, a quarter per halving of h)."""
    a, wc, beta, dt = 0.3, 5.0, 1.0, 0.1
    par = Spectral("ohmic_exp", a, wc)
    boxes = [((1.0, 1.1), (1.0, 1.1)), (strang_box(4, 99, dt), strang_box(1, 99, dt)),
             (strang_box(6, 6, dt), strang_box(0, 6, dt))]
    want = np.array([eta_boxes(par, beta, *b) for b in boxes])
    errs = []
    for n in (100, 200):
        om = np.linspace(20.0 * wc / n, 20.0 * wc, n)
        tab = Spectral.tabulated(om, par.J(om))
        got = np.array([eta_boxes(tab, beta, *b) for b in boxes])
        errs.append(np.abs(got - want).max() / np.abs(want).max())
    assert errs[0] < 3e-2 and errs[1] < 0.35 * errs[0], errs
