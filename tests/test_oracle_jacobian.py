"""Pins of the oracle's Jacobian J = df/dy (Eq. e:jac).

The oracle forms J by forward-mode dual numbers through its source function.  It is pinned
against complex-step differentiation (a different derivative technique, exact to roundoff for
analytic functions) and a central finite difference.  Comparisons use the gross-magnitude scale
of the row: near equilibrium a net rate is the small difference of large forward and reverse
rates, and a purely relative test would be meaningless.
"""
import numpy as np
import pytest

from tests.conftest import states

CASES = [("h2_13", "h2_fresh"), ("ch4_53", "ch4_partial"), ("ch4_111", "ch4_front")]


def complex_step_jacobian(m, y, P, h=1e-30):
    N = m.N
    J = np.zeros((N, N))
    for j in range(N):
        dj = h * max(abs(y[j]), 1e-12)
        yc = y.astype(np.complex128)
        yc[j] += 1j * dj
        J[:, j] = m.source_cplx(yc, P).imag / dj
    return J


def row_scale(J, y):
    """Gross magnitude per row: sum_j |J_ij| |y_j| + tiny."""
    return np.abs(J) @ np.maximum(np.abs(y), 1e-12)


@pytest.mark.parametrize("name,recipe", CASES)
def test_dual_jacobian_matches_complex_step(omech, name, recipe):
    m = omech(name)
    st = states(name, 3, recipe, 21)
    y = m.state_from_TY(st.T, st.Y)
    J = m.jacobian(y, st.P)
    for c in range(3):
        Jc = complex_step_jacobian(m, y[c], st.P[c])
        scale = row_scale(Jc, y[c])[:, None] / np.maximum(np.abs(y[c]), 1e-12)[None, :]
        err = np.abs(J[c] - Jc) / (np.abs(Jc) + scale)
        assert err.max() <= 1e-13, (c, err.max())


def test_jacobian_central_difference(omech):
    m = omech("h2_13")
    st = states("h2_13", 2, "h2_fresh", 22)
    y = m.state_from_TY(st.T, st.Y)
    J = m.jacobian(y, st.P)
    for c in range(2):
        Jfd = np.zeros((m.N, m.N))
        for j in range(m.N):
            d = 1e-6 * max(abs(y[c, j]), 1e-9)
            yp, ym = y[c].copy(), y[c].copy()
            yp[j] += d
            ym[j] -= d
            Jfd[:, j] = (m.source(yp, st.P[c])[0] - m.source(ym, st.P[c])[0]) / (2 * d)
        scale = row_scale(J[c], y[c])[:, None] / np.maximum(np.abs(y[c]), 1e-12)[None, :]
        assert (np.abs(J[c] - Jfd) / (np.abs(J[c]) + scale)).max() <= 1e-6


def test_jacobian_on_both_nasa_ranges(omech):
    """The T column crosses the NASA range switch: check just below and above Tmid."""
    m = omech("ch4_53")
    st = states("ch4_53", 1, "ch4_partial", 23)
    for T in (999.5, 1000.5):
        y = m.state_from_TY([T], st.Y)[0]
        J = m.jacobian(y, st.P[0])[0]
        Jc = complex_step_jacobian(m, y, st.P[0])
        scale = row_scale(Jc, y)[:, None] / np.maximum(np.abs(y), 1e-12)[None, :]
        assert (np.abs(J - Jc) / (np.abs(Jc) + scale)).max() <= 1e-13


def test_jacobian_wrt_lnA_directional(omech):
    """Complex step in ln A (the differentiable parameters) against a central difference."""
    m = omech("h2_13")
    st = states("h2_13", 1, "h2_fresh", 24)
    y = m.state_from_TY(st.T, st.Y)[0]
    lnA = m.lnA.copy()
    rng = np.random.default_rng(0)
    v = rng.normal(size=m.nr)
    d_cs = m.source_cplx(y, st.P[0], lnA + 1e-30j * v).imag / 1e-30
    e = 1e-6
    d_fd = (m.source(y, st.P[0], lnA + e * v)[0] - m.source(y, st.P[0], lnA - e * v)[0]) / (2 * e)
    assert np.allclose(d_cs, d_fd, rtol=1e-6, atol=1e-9 * np.abs(d_cs).max())
