"""Pins of the oracle's quadrature weights (App. C, Sec. 2.4) against values
the paper prints and against identities fixed by the mathematics."""
import math
import os
import pathlib

import numpy as np
import pytest
from scipy import integrate

from oracle import quadrature as Q
from tests.conftest import GOLDEN


def _poly(c, x):
    return sum(ci * x ** i for i, ci in enumerate(c))


def _closed_forms():
    out = {}
    for line in pathlib.Path(os.path.join(GOLDEN, "app_c_closed_forms.txt")).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        left, right = line.split("|")
        f = left.split()
        name, sign, k = f[0], float(f[1]), float(f[2])
        a = [float(x) for x in f[3:]]
        b = [float(x) for x in right.split()]
        out[name] = (sign, k, a, b)
    return out


def _eval_closed(entry, nu):
    sign, k, a, b = entry
    return sign * (_poly(a, nu) - _poly(b, nu) * math.exp(-nu)) / (k * nu ** 3)


NAMES = {0: ("c0_m3", "c0_m2", "c0_m1", "c0_0"),
         1: ("c1_m2", "c1_m1", "c1_0", "c1_1"),
         2: ("c2_m1", "c2_0", "c2_1", "c2_2")}


@pytest.mark.parametrize("nu", [0.6, 1.0, 2.0, 4.0])
def test_substencil_weights_match_printed_closed_forms(nu):
    cf = _closed_forms()
    for r in range(3):
        got = Q.local_weights(nu, Q.SUBSTENCILS[6][r])
        want = np.array([_eval_closed(cf[n], nu) for n in NAMES[r]])
        # closed forms cancel like nu^-3; at nu >= 0.6 they keep ~1e-13
        np.testing.assert_allclose(got, want, rtol=2e-12, atol=1e-14)


def test_printed_c_m1_0_is_garbled():
    cf = _closed_forms()
    nu = 2.0   # (at nu = 1 the printed nu^2 and the corrected nu^3 coincide)
    got = Q.local_weights(nu, Q.SUBSTENCILS[6][0])[2]
    assert abs(_eval_closed(cf["c0_m1_as_printed"], nu) - got) > 1e-2
    assert abs(_eval_closed(cf["c0_m1"], nu) - got) < 1e-13


def _linear_weight_forms():
    out = {}
    for line in pathlib.Path(os.path.join(GOLDEN, "app_c_linear_weights.txt")).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = [p.split() for p in line.split("|")]
        name = parts[0][0]
        an, bn, ad, bd = ([float(x) for x in p] for p in parts[1:5])
        kpow, fac = (float(x) for x in parts[5])
        out[name] = (an, bn, ad, bd, kpow, fac)
    return out


def _eval_lw(entry, nu):
    an, bn, ad, bd, kpow, fac = entry
    e = math.exp(-nu)
    return (_poly(an, nu) - _poly(bn, nu) * e) / (fac * nu ** kpow * (_poly(ad, nu) - _poly(bd, nu) * e))


@pytest.mark.parametrize("nu", [0.5, 1.0, 2.0, 3.0])
def test_linear_weight_d2_matches_print(nu):
    d = Q.linear_weights(nu, 6)
    lw = _linear_weight_forms()
    assert abs(d[2] - _eval_lw(lw["d2"], nu)) < 1e-11
    assert abs(d.sum() - 1.0) < 1e-14


def test_linear_weight_d0_reading():
    # printed d_0 is garbled (its value at nu=1/2 is 0.4917); the definition
    # of Sec. 2.4 fixes d_0 = c_{-3}(big) / c_{-3}^{(0)}.
    nu = 0.5
    d = Q.linear_weights(nu, 6)
    big = Q.local_weights(nu, Q.STENCIL[6])
    c0 = Q.local_weights(nu, Q.SUBSTENCILS[6][0])
    assert abs(d[0] - big[0] / c0[0]) < 1e-14
    assert abs(_eval_lw(_linear_weight_forms()["d0_printed"], nu) - d[0]) > 0.2
    assert abs(d[0] - 0.178550) < 1e-5


def test_linear_weight_small_nu_limits():
    # nu -> 0: the rules become cell averages; classic limits 11/60, 19/30, 11/60
    d6 = Q.linear_weights(1e-6, 6)
    np.testing.assert_allclose(d6, [11 / 60, 19 / 30, 11 / 60], atol=1e-6)
    d5 = Q.linear_weights(1e-6, 5)
    np.testing.assert_allclose(d5, [11 / 300, 97 / 150, 19 / 60], atol=1e-6)
    assert np.all(Q.linear_weights(0.7, 5) > 0)


def test_small_nu_limit_cell_average():
    # c_l / nu -> integral of ell_l over the cell = (11,-93,802,802,-93,11)/1440
    nu = 1e-7
    c = Q.local_weights(nu, Q.STENCIL[6]) / nu
    np.testing.assert_allclose(c * 1440, [11, -93, 802, 802, -93, 11], atol=1e-4)


@pytest.mark.parametrize("npts", [3, 5, 6])
@pytest.mark.parametrize("nu", [0.01, 0.4, 2.0])
def test_moment_identities(npts, nu):
    # sum_l c_l l^m = nu * int_{-1}^0 e^{nu t} t^m dt for m < npts (exactness
    # of the interpolant on polynomials), integrated independently by scipy.
    c = Q.local_weights(nu, Q.STENCIL[npts])
    offs = np.array(Q.STENCIL[npts], dtype=float)
    for m in range(npts):
        ref, _ = integrate.quad(lambda t: nu * math.exp(nu * t) * t ** m, -1.0, 0.0,
                                epsabs=1e-16, epsrel=1e-14)
        assert abs(np.sum(c * offs ** m) - ref) < 1e-14 * max(1.0, abs(ref) / nu) * 10
    # m = 0 in closed form: sum c = 1 - e^{-nu}
    assert abs(c.sum() - (1 - math.exp(-nu))) < 4e-15


def _printed_betas():
    rows = []
    for line in pathlib.Path(os.path.join(GOLDEN, "app_c_smoothness.txt")).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        _, a, b = line.split("|")
        rows.append((np.array([float(x) for x in a.split()]), np.array([float(x) for x in b.split()])))
    return rows


def test_smoothness_indicators_match_printed():
    rows = _printed_betas()
    g = np.random.default_rng(7)
    for _ in range(20):
        v = g.standard_normal(6)
        for r in range(3):
            M = Q.smoothness_matrix(Q.SUBSTENCILS[6][r], Q.smoothness_orders(6))
            got = v[r:r + 4] @ M @ v[r:r + 4]
            a, b = rows[r]
            want = 13.0 / 12.0 * (a @ v) ** 2 + 0.25 * (b @ v) ** 2
            assert abs(got - want) < 1e-12 * max(1.0, want)


def test_quadratic_smoothness_indicator_jiang_shu():
    # orders (1,2) on {-1,0,1} for the cell [-1,0]: a quadratic through
    # (-1,a),(0,b),(1,c) has p_tt = a-2b+c and p_t(t) = (c-a)/2 + t (a-2b+c).
    # int_{-1}^0 p_t^2 dt + p_tt^2, worked by hand:
    a, b, c = 0.3, -1.1, 2.0
    s2 = a - 2 * b + c
    s1 = (c - a) / 2
    want = s1 ** 2 - s1 * s2 + s2 ** 2 / 3 + s2 ** 2
    M = Q.smoothness_matrix((-1, 0, 1), (1, 2))
    v = np.array([a, b, c])
    assert abs(v @ M @ v - want) < 1e-13
