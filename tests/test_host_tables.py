"""The library's host-side quadrature tables (exponential moments by series
and recurrence, Lagrange monomials, linear weights) against the oracle's
Gauss-Legendre construction -- host code only, no GPU needed."""
import os

import numpy as np
import pytest

from oracle.quadrature import STENCIL, QuadratureRule


@pytest.fixture(scope="module")
def M():
    from paper_2007_03041_gb300 import molt
    if not os.path.exists(molt.LIB_PATH):
        from paper_2007_03041_gb300 import build
        build.build()
    molt.load_library()
    return molt


@pytest.mark.parametrize("npts", [3, 5, 6])
@pytest.mark.parametrize("nu", [1e-3, 0.0125, 0.088, 0.4, 2.0 / 3.0, 1.0, 1.7, 4.0])
def test_library_quadrature_tables_match_oracle(M, npts, nu):
    c, sub, d = M.molt_quadrature_weights(npts, nu)
    rule = QuadratureRule(nu, npts)
    want = np.zeros(6)
    for o, w in zip(STENCIL[npts], rule.c):
        want[o + 3] = w
    np.testing.assert_allclose(c, want, rtol=1e-11, atol=1e-15 * nu)
    if npts == 3:
        assert not any(sub[0] + sub[1] + sub[2]) and not any(d)
        return
    m = len(rule.sub_offsets[0])
    for r in range(3):
        np.testing.assert_allclose(sub[r][:m], rule.sub_c[r], rtol=1e-11, atol=1e-15 * nu)
        assert all(v == 0.0 for v in sub[r][m:])
    np.testing.assert_allclose(d, rule.d, rtol=1e-11)
    if npts == 5:
        np.testing.assert_allclose(M.molt_weno_linear_weights(nu), d, rtol=0, atol=0)


def test_library_rejects_bad_rules(M):
    with pytest.raises(M.MoltError):
        M.molt_quadrature_weights(4, 0.5)
    with pytest.raises(M.MoltError):
        M.molt_quadrature_weights(6, 0.0)
    with pytest.raises(M.MoltError):
        M.molt_quadrature_weights(6, float("nan"))
