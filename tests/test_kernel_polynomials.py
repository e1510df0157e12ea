"""The FP32 sweep evaluates the segment weights below x = 1/4 from degree-4
polynomials written as literals in `csrc/sweep.cuh` (Chebyshev
interpolants). This test reads those literals from the source and checks
them against the functions they stand for, in float64 and in float32 Horner
evaluation, so a mistyped coefficient fails here without a GPU:

    q(x)      = (1 - e^-x) / x                (seg_eq)
    w_up(x)/x = ((1 - e^-x)/x - e^-x) / x     (seg_weights, seg_dwp: d w_p/dx = w_up/x)
    w_p(x)/x  = (1 - (1 - e^-x)/x) / x        (seg_weights)
"""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2107_08145_b300", "csrc",
                   "sweep.cuh")

NUM = r"(-?\d+\.\d+)f"
HORNER = re.compile(NUM + r" \+ x \* \(" + NUM + r" \+ x \* \(" + NUM + r" \+ x \* \(" + NUM + r" \+ x \* " + NUM)


def _polys():
    """Every degree-4 Horner literal in the sweep source, low order first."""
    src = open(SRC).read()
    return [tuple(float(v) for v in m.groups()) for m in HORNER.finditer(src)]


def _q(x):
    return -np.expm1(-x) / x


def _wu_over_x(x):
    return (_q(x) - np.exp(-x)) / x


def _exact_wp_over_x(x):
    # w_p / x = (1 - q) / x = (x - (1 - e^-x)) / x^2 = (x + expm1(-x)) / x^2, by series for small x
    out = np.empty_like(x)
    small = x < 1e-3
    xs = x[small]
    out[small] = 0.5 - xs / 6 + xs ** 2 / 24 - xs ** 3 / 120
    xl = x[~small]
    out[~small] = (xl + np.expm1(-xl)) / xl ** 2
    return out


def _exact_wu_over_x(x):
    # w_up / x = ((1 - e)/x - e)/x, by series for small x: 1/2 - x/3 + x^2/8 - x^3/30
    out = np.empty_like(x)
    small = x < 1e-3
    xs = x[small]
    out[small] = 0.5 - xs / 3 + xs ** 2 / 8 - xs ** 3 / 30
    xl = x[~small]
    out[~small] = _wu_over_x(xl)
    return out


def _exact_q(x):
    out = np.empty_like(x)
    small = x < 1e-6
    out[small] = 1.0 - x[small] / 2
    out[~small] = _q(x[~small])
    return out


def _horner(c, x, dtype):
    x = x.astype(dtype)
    acc = np.full_like(x, dtype(c[4]))
    for k in (3, 2, 1, 0):
        acc = (acc * x + dtype(c[k])).astype(dtype)
    return acc.astype(np.float64)


def _match(c):
    x = np.linspace(1e-7, 0.25, 20001)
    errs = {}
    for name, f in (("q", _exact_q), ("wu/x", _exact_wu_over_x), ("wp/x", _exact_wp_over_x)):
        ref = f(x)
        errs[name] = np.max(np.abs(_horner(c, x, np.float64) - ref) / np.abs(ref))
    return min(errs, key=errs.get), errs


def test_every_polynomial_interpolates_its_function():
    polys = _polys()
    # q in seg_eq; w_up/x and w_p/x in seg_weights; w_up/x again in seg_dwp
    assert len(polys) == 4, polys
    names = []
    for c in polys:
        name, errs = _match(c)
        names.append(name)
        assert errs[name] < 5e-9, (c, errs)
    assert sorted(names) == ["q", "wp/x", "wu/x", "wu/x"], names


def test_float32_evaluation_is_within_an_ulp_or_two():
    x = np.linspace(1e-7, 0.25, 20001)
    for c in _polys():
        name, _ = _match(c)
        f = {"q": _exact_q, "wu/x": _exact_wu_over_x, "wp/x": _exact_wp_over_x}[name]
        ref = f(x.astype(np.float32).astype(np.float64))
        err = np.max(np.abs(_horner(c, x, np.float32) - ref) / np.abs(ref))
        assert err < 2.5e-7, (name, err)


def test_switch_point_continuity():
    """At the switch point x = 1/4 the polynomial and the exp/divide form agree
    to FP32 rounding, so selecting between them leaves no visible step."""
    x = 0.25
    for c in _polys():
        name, _ = _match(c)
        f = {"q": _exact_q, "wu/x": _exact_wu_over_x, "wp/x": _exact_wp_over_x}[name]
        ref = f(np.array([x]))[0]
        assert abs(_horner(c, np.array([x]), np.float64)[0] - ref) / abs(ref) < 5e-9


REG_SRC = os.path.join(os.path.dirname(SRC), "sweep_reg.cuh")


def _reg_array(name):
    """A `constexpr double name[5] = {...};` literal array of the register sweep."""
    src = open(REG_SRC).read()
    m = re.search(r"constexpr double " + name + r"\[5\] = \{([^}]*)\}", src)
    assert m, name
    return tuple(float(v) for v in m.group(1).split(","))


def test_register_sweep_literals():
    """The register sweep's q polynomial (kQPolyX) and its checkpoint's
    dw_p/dx = w_up/x polynomial (kDwpX) interpolate their functions, and the
    latter evaluated in y = -x log2(e) with the float32 coefficients the kernel
    forms stays within a few float32 ulps."""
    x = np.linspace(1e-7, 0.25, 20001)
    cq, cd = _reg_array("kQPolyX"), _reg_array("kDwpX")
    assert np.max(np.abs(_horner(cq, x, np.float64) - _exact_q(x)) / _exact_q(x)) < 5e-9
    ref = _exact_wu_over_x(x)
    assert np.max(np.abs(_horner(cd, x, np.float64) - ref) / ref) < 5e-9
    ln2 = np.log(2.0)
    ky = [-cd[i] * (-ln2) ** i for i in range(5)]  # negated, in y
    y = (-x / ln2).astype(np.float32)
    assert np.max(np.abs(-_horner(ky, y, np.float32) - ref) / ref) < 2.5e-7
