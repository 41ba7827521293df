"""Pins of the oracle's changeover functions (Sec. 2.1.1, Eq. cutfuncW).

The paper prints W(y; gamma) but not K; K follows from W(r) = r int_r^inf
K/s^2 ds as K = W - y dW/dy.  These tests rebuild W symbolically from the
printed coefficients (tests/golden/changeover_W.json) and check the oracle's
K against W - y W', so a wrong coefficient in the oracle's K fails here.
"""
import json
import os

import numpy as np
import pytest

sympy = pytest.importorskip("sympy")

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "changeover_W.json")))
GAMMAS = [sympy.Rational(1, 10), sympy.Rational(3, 10), sympy.Rational(1, 2)]


def _printed_W(g, y7=None):
    y = sympy.Symbol("y", positive=True)
    loc = {"g": g, "log": sympy.log, "y": y}
    terms = GOLD["f_terms"]
    c7 = sympy.sympify(y7 if y7 is not None else terms["y7"], locals=loc)
    f = (c7 * y**7
         + sympy.sympify(terms["y6"], locals=loc) * y**6
         + sympy.sympify(terms["y5"], locals=loc) * y**5
         + sympy.sympify(terms["y4"], locals=loc) * y**4
         + sympy.sympify(terms["y3"], locals=loc) * y**3
         + sympy.sympify(terms["y2"], locals=loc) * y**2
         + sympy.sympify(terms["ylogy"], locals=loc) * y * sympy.log(y)
         + sympy.sympify(terms["const"], locals=loc)) / sympy.sympify(GOLD["denominator"], locals=loc)
    W_mid = f + (1 - f.subs(y, 1)) * y
    c_in = sympy.sympify(GOLD["inner_slope"], locals=loc)
    return y, W_mid, c_in


@pytest.mark.parametrize("g", GAMMAS)
def test_printed_W_is_continuous_under_reading_C1(g):
    y, W_mid, c_in = _printed_W(g)
    assert abs(float(W_mid.subs(y, g) - c_in * g)) < 1e-14
    assert abs(float(W_mid.subs(y, 1)) - 1.0) < 1e-14
    # the slope of W is continuous too (so K is continuous: K(gamma) = 0)
    assert abs(float(sympy.diff(W_mid, y).subs(y, g) - c_in)) < 1e-12


def test_other_reading_of_garbled_term_breaks_continuity():
    g = GAMMAS[0]
    y = sympy.Symbol("y", positive=True)
    _, W_ok, c_in = _printed_W(g)
    # reading "-10/3y^7" as -10/(3 y^7) instead of -(10/3) y^7
    _, W_bad, _ = _printed_W(g, y7="-10/3/y**14")
    assert abs(float(W_bad.subs(y, g) - c_in * g)) > 1e-3


@pytest.mark.parametrize("g", GAMMAS)
def test_K_equals_W_minus_y_dW(orc, g):
    y, W_mid, _ = _printed_W(g)
    import mpmath
    mpmath.mp.dps = 40
    K_expr = sympy.lambdify(y, W_mid - y * sympy.diff(W_mid, y), "mpmath")
    gf = float(g)
    for yv in np.linspace(gf, 1.0, 41)[1:-1]:
        ref = float(K_expr(mpmath.mpf(float(yv))))
        # the degree-7 polynomial cancels terms of size ~100 down to ~1 near
        # y = 1, so FP64 evaluation is good to ~100 ulp
        assert abs(orc.changeover_K(yv, gf) - ref) < 1e-13, (yv, ref)


@pytest.mark.parametrize("g", [0.1, 0.3])
def test_K_limits_and_derivative(orc, g):
    assert orc.changeover_K(0.0, g) == 0.0
    assert orc.changeover_K(g, g) == 0.0
    assert orc.changeover_K(0.5 * g, g) == 0.0
    assert orc.changeover_K(1.0, g) == 1.0
    assert orc.changeover_K(7.0, g) == 1.0
    for yv in np.linspace(g, 1.0, 23)[1:-1]:
        h = 1e-6
        fd = (orc.changeover_K(yv + h, g) - orc.changeover_K(yv - h, g)) / (2 * h)
        assert abs(orc.changeover_dKdy(yv, g) - fd) < 1e-7
    # S'(x) vanishes at both ends of the transition
    assert orc.changeover_dKdy(g + 1e-9, g) < 1e-20
    assert orc.changeover_dKdy(1.0 - 1e-9, g) < 1e-20
    # K is monotone on [gamma, 1]
    ks = [orc.changeover_K(v, g) for v in np.linspace(g, 1.0, 200)]
    assert np.all(np.diff(ks) >= 0.0)


def test_soft_plus_hard_pair_is_newtonian(orc):
    """K + (1 - K) = 1: the soft force (Eq. softforce) plus the pair part of the
    hard force (Eq. hardforce) is the Newtonian pair force."""
    rng = np.random.default_rng(5)
    n = 12
    s = {k: rng.normal(size=n) * 1e-3 for k in ("x", "y", "z", "vx", "vy", "vz")}
    s["x"] = s["x"] + 1.0
    s["m"] = rng.uniform(0.5, 2.0, n) * 1e-9
    r_out = rng.uniform(0.5e-3, 3e-3, n)     # many pairs fall inside the transition
    p = orc.Params(m_star=0.0, gamma=0.1)
    soft = orc.direct_soft(s, r_out, p)
    hard = np.array([orc.hard_acc_jerk(s, r_out, p, k)[0] for k in range(n)])
    pos = np.stack([s["x"], s["y"], s["z"]], 1)
    newton = np.zeros((n, 3))
    for i in range(n):
        d = pos[i] - pos
        r = np.linalg.norm(d, axis=1)
        r[i] = np.inf
        newton[i] = -(s["m"][:, None] * d / r[:, None] ** 3).sum(0)
    err = np.abs(soft + hard - newton).max() / np.abs(newton).max()
    assert err < 1e-14
    # and the split is non-trivial: both parts carry force
    assert np.abs(soft).max() > 1e-3 * np.abs(newton).max()
    assert np.abs(hard).max() > 1e-3 * np.abs(newton).max()
