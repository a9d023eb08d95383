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


@pytest.mark.parametrize("npts", [3, 5, 6])
@pytest.mark.parametrize("alpha", [0.5, 6.0, 80.0])
def test_library_nonuniform_tables_match_oracle(M, npts, alpha):
    """The library's point tables of a non-uniform periodic line (16-point
    Gauss-Legendre in C++) against the oracle's (48-point, numpy)."""
    from oracle import nonuniform
    from oracle.quadrature import STENCIL
    n, L = 37, 2 * np.pi
    xi = L * np.arange(n) / n
    x = 0.25 + xi + 0.35 * np.sin(xi)
    cR, cL, q = M.molt_nonuniform_weights(x, L, alpha, npts)
    wR, wL, wq = nonuniform.weights(x, L, alpha, npts)
    for m, o in enumerate(STENCIL[npts]):
        np.testing.assert_allclose(cR[o + 3], wR[:, m], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(cL[o + 3], wL[:, m], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(q, wq, rtol=1e-14)
    unused = [k for k in range(6) if k - 3 not in STENCIL[npts]]
    assert np.all(cR[unused] == 0) and np.all(cL[unused] == 0)


@pytest.mark.parametrize("alpha", [0.5, 6.0, 80.0])
def test_library_nonuniform_weno_tables_match_oracle(M, alpha):
    """The library's WENO-Z point tables (substencil rules, local d_r, and the
    (a, b) form of the smoothness indicators) against the oracle's (rules,
    least-squares d_r, indicator matrices in physical coordinates)."""
    from oracle import nonuniform
    n, L = 37, 2 * np.pi
    w = 1.0 + 0.6 * np.random.default_rng(4).uniform(-1, 1, n)
    x = 0.1 + np.concatenate([[0.0], np.cumsum(w)[:-1]]) * (L / w.sum())
    wR, wL = M.molt_nonuniform_weno_weights(x, L, alpha)
    t = nonuniform.weno_tables(x, L, alpha, 5)
    V = np.random.default_rng(5).standard_normal((n, 5))
    for side, tab in (("R", wR), ("L", wL)):
        ref = t[side]
        for r in range(3):
            for j in range(3):
                np.testing.assert_allclose(tab[3 * r + j], ref["sub"][:, r, j], rtol=1e-12, atol=1e-15)
            np.testing.assert_allclose(tab[9 + r], ref["d"][:, r], rtol=1e-10, atol=1e-13)
            vals = V[:, r:r + 3]
            a = sum(tab[12 + 3 * r + j] * vals[:, j] for j in range(3))
            b = sum(tab[21 + 3 * r + j] * vals[:, j] for j in range(3))
            beta_lib = a * a - a * b + 4.0 / 3.0 * b * b
            beta_ref = np.einsum("ia,iab,ib->i", vals, ref["M"][:, r], vals)
            np.testing.assert_allclose(beta_lib, beta_ref, rtol=1e-10, atol=1e-14)
    with pytest.raises(M.MoltError):
        M.molt_nonuniform_weno_weights(x[::-1], L, alpha)


@pytest.mark.parametrize("npts", [3, 5, 6])
def test_library_dirichlet_nonuniform_tables_match_oracle(M, npts):
    """period == 0: a Dirichlet line with both boundary nodes; the stencils
    reach mirrored ghost nodes.  The rows the recurrences use match the
    oracle; J_R(x_0), J_L(x_N) and q_0 are zero (the recurrences start there)."""
    from oracle import nonuniform
    from oracle.quadrature import STENCIL
    N, a, b, alpha = 30, 0.2, 2.9, 11.0
    t = np.linspace(0.0, 1.0, N + 1)
    x = a + (b - a) * (t + 0.3 * np.sin(2 * np.pi * t) / (2 * np.pi))
    cR, cL, q = M.molt_nonuniform_weights(x, 0.0, alpha, npts)
    wR, wL, wq = nonuniform.weights(x, None, alpha, npts)
    for m, o in enumerate(STENCIL[npts]):
        np.testing.assert_allclose(cR[o + 3][1:], wR[1:, m], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(cL[o + 3][:-1], wL[:-1, m], rtol=1e-12, atol=1e-15)
    assert np.all(cR[:, 0] == 0) and np.all(cL[:, -1] == 0) and q[0] == 0
    np.testing.assert_allclose(q[1:], wq[1:], rtol=1e-14)


def test_library_dirichlet_nonuniform_weno_tables_match_oracle(M):
    from oracle import nonuniform
    N, alpha = 25, 6.0
    t = np.linspace(0.0, 1.0, N + 1)
    x = np.pi * (t + 0.25 * np.sin(2 * np.pi * t) / (2 * np.pi))
    wR, wL = M.molt_nonuniform_weno_weights(x, 0.0, alpha)
    ref = nonuniform.weno_tables(x, None, alpha, 5)
    for side, tab, rows in (("R", wR, slice(1, None)), ("L", wL, slice(None, -1))):
        for r in range(3):
            for j in range(3):
                np.testing.assert_allclose(tab[3 * r + j][rows], ref[side]["sub"][rows, r, j], rtol=1e-12,
                                           atol=1e-15)
            np.testing.assert_allclose(tab[9 + r][rows], ref[side]["d"][rows, r], rtol=1e-10, atol=1e-13)
    assert np.all(wR[:9, 0] == 0) and np.all(wL[:9, -1] == 0)
    np.testing.assert_allclose(wR[9:12, 0], 1.0 / 3.0)
    with pytest.raises(M.MoltError):
        M.molt_nonuniform_weights(x[:3], 0.0, alpha, 6)                       # fewer than 4 nodes
    with pytest.raises(M.MoltError):
        M.molt_nonuniform_weights(x, -1.0, alpha, 6)                          # negative period
