"""Pins of the oracle's ROS4 integrator (Sec. 2.3, Eq. e:ros and its transformed form).

The paper prints no coefficients; the oracle carries the Hairer-Wanner L-stable ROS4 set in the
transformed variables.  The tests map it back to the untransformed (alpha, gamma, b) of Eq. e:ros
(Gamma = (diag(1/gamma) - C)^-1, alpha = A Gamma, b^T = m^T Gamma) and check:
  * the 8 order conditions of order 4 and the 4 of the embedded order-3 solution;
  * the stability function R(z) = 1 + z b^T (I - z B)^-1 1, |R(iw)| <= 1, R(inf) ~ 0;
  * one step on y' = A y reproduces R(hA) y0 (closed form, scalar and 2x2);
  * adaptive integration of y' = lambda y reaches exp(lambda t) within tolerance;
  * convergence order 4 of fixed-step runs and h^4 scaling of the error estimate on a
    nonlinear, moderately stiff mechanism (tests/golden/tiny_hon7.mech);
  * agreement with classical RK4 at tiny steps (an integrator sharing nothing with ROS4).
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O

ATM = 101325.0


def untransformed(tab=O.ROS4):
    t = O.tableau(tab)
    g, s = t["gamma"], t["s"]
    Gamma = np.linalg.inv(np.diag([1 / g] * s) - t["c"])
    alpha = t["a"] @ Gamma
    b = t["m"] @ Gamma
    bh = (t["m"] - t["e"]) @ Gamma
    return g, Gamma, alpha, b, bh


def order_residuals(g, Gamma, alpha, b):
    beta = alpha + np.tril(Gamma, -1)
    bp = beta.sum(1)
    al = alpha.sum(1)
    return np.array([
        b.sum() - 1,
        b @ bp - (0.5 - g),
        b @ al ** 2 - 1 / 3,
        b @ beta @ bp - (1 / 6 - g + g * g),
        b @ al ** 3 - 0.25,
        (b * al) @ alpha @ bp - (1 / 8 - g / 3),
        b @ beta @ al ** 2 - (1 / 12 - g / 3),
        b @ beta @ beta @ bp - (1 / 24 - g / 2 + 1.5 * g * g - g ** 3),
    ])


def R(z, tab=O.ROS4):
    g, Gamma, alpha, b, _ = untransformed(tab)
    B = alpha + Gamma
    s = len(b)
    return 1 + z * b @ np.linalg.solve(np.eye(s) - z * B, np.ones(s))


def test_gamma_constant_and_lower_triangular():
    g, Gamma, alpha, b, bh = untransformed()
    assert np.allclose(np.diag(Gamma), g, rtol=0, atol=1e-15)
    assert np.allclose(np.triu(Gamma, 1), 0, atol=1e-15)
    assert np.allclose(np.triu(alpha), 0, atol=1e-15)


def test_order_conditions():
    g, Gamma, alpha, b, bh = untransformed()
    assert np.abs(order_residuals(g, Gamma, alpha, b)).max() < 1e-14
    # the embedded solution is of order 3 but not 4
    r = order_residuals(g, Gamma, alpha, bh)
    assert np.abs(r[:4]).max() < 1e-14
    assert np.abs(r[4:]).max() > 1e-4


def test_stability_function():
    # A-stable on the imaginary axis, L-stable up to the 5-digit rounding of gamma = 0.57282
    for w in np.logspace(-3, 6, 200):
        assert abs(R(1j * w)) <= 1 + 1e-12
    assert abs(R(-1e14)) < 2e-5
    for x in np.logspace(-2, 8, 100):
        assert abs(R(-x)) <= 1 + 1e-12


@pytest.mark.parametrize("z", [-1e-3, -0.3, -2.0, -50.0, -1e6, 0.7])
def test_one_step_scalar_closed_form(z):
    h = 0.01
    A = np.array([[z / h]])
    y1, err = O.step_linear(A, [1.5], h)
    assert y1[0] == pytest.approx(R(z).real * 1.5, rel=1e-13, abs=1e-15)


def test_one_step_matrix_closed_form():
    """2x2 rotation-decay system: the step equals R(hA) y0 evaluated by eigen-decomposition."""
    A = np.array([[-1.0, 40.0], [-40.0, -1.0]])
    h = 0.05
    y0 = np.array([1.0, -0.5])
    y1, _ = O.step_linear(A, y0, h)
    lam, V = np.linalg.eig(A)
    Rm = (V @ np.diag([R(h * l) for l in lam]) @ np.linalg.inv(V)).real
    assert np.allclose(y1, Rm @ y0, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("lam", [-1.0, -30.0, 2.0])
def test_adaptive_exponential(lam):
    for rtol in (1e-6, 1e-9):
        y, status, attempts = O.integrate_linear(np.array([[lam]]), [1.0], 1.0, rtol, 1e-14)
        assert status == O.OK
        assert abs(y[0] - np.exp(lam)) <= 5 * (rtol * np.exp(lam) + 1e-14)


def test_adaptive_stiff_linear_system():
    A = np.array([[-1e6, 1.0], [0.0, -1.0]])
    y, status, attempts = O.integrate_linear(A, [1.0, 1.0], 1.0, 1e-8, 1e-14)
    exact = scipy.linalg.expm(A) @ np.array([1.0, 1.0])
    assert status == O.OK
    assert np.allclose(y, exact, rtol=1e-6, atol=1e-12)
    assert attempts < 2000


def _tiny_state(m, T=1100.0):
    Y = np.array([0.02, 0.2, 0.01, 1e-4, 1e-4, 1e-3, 0.0])
    Y[-1] = 1 - Y.sum()
    return m.state_from_TY([T], [Y])[0]


def test_convergence_order_four(omech):
    m = omech("tiny_hon7.mech")
    y0 = _tiny_state(m)
    dt = 2e-5
    ref, _ = m.integrate(y0, ATM, dt, fixed_steps=8192)
    sc = 1e-10 + 1e-6 * np.abs(ref[0])
    errs = []
    for K in (32, 64, 128):
        yk, _ = m.integrate(y0, ATM, dt, fixed_steps=K)
        errs.append(np.sqrt(np.mean(((yk[0] - ref[0]) / sc) ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 4.0) < 0.15), orders


def test_error_estimate_scales_as_h4(omech):
    m = omech("tiny_hon7.mech")
    y0 = _tiny_state(m)
    sc = 1e-10 + 1e-6 * np.abs(y0)
    es = []
    for h in (2e-5 / 64, 2e-5 / 128, 2e-5 / 256):
        _, e = m.step(y0, ATM, h)
        es.append(np.sqrt(np.mean((e / sc) ** 2)))
    orders = np.log2(np.array(es[:-1]) / np.array(es[1:]))
    assert np.all(np.abs(orders - 4.0) < 0.15), orders


def test_matches_classical_rk4(omech):
    """Explicit RK4 with 20000 steps (Richardson-checked) against adaptive ROS4 at rtol 1e-10."""
    m = omech("tiny_hon7.mech")
    y0 = _tiny_state(m, 1050.0)
    dt = 2e-5

    def rk4(K):
        y = y0.copy()
        h = dt / K
        f = lambda v: m.source(v, ATM)[0]
        for _ in range(K):
            k1 = f(y)
            k2 = f(y + 0.5 * h * k1)
            k3 = f(y + 0.5 * h * k2)
            k4 = f(y + h * k3)
            y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        return y

    a, b = rk4(10000), rk4(20000)
    sc = 1e-14 + 1e-10 * np.abs(b)
    assert np.max(np.abs(a - b) / sc) < 1.0  # the RK4 reference is converged
    yr, info = m.integrate(y0, ATM, dt, rtol=1e-10, atol=1e-16)
    assert info["status"][0] == O.OK
    assert np.max(np.abs(yr[0] - b) / (1e-14 + np.abs(b))) <= 1e-8


def test_controller_records(omech):
    """Attempts = accepted + rejected; the accepted step sizes sum to dt; replaying them in
    double reproduces the adaptive result bit for bit."""
    m = omech("h2_13")
    from tests.conftest import states
    st = states("h2_13", 4, "h2_fresh", 31)
    y = m.state_from_TY(st.T, st.Y)
    yo, info = m.integrate(y, st.P, 1e-6)
    assert np.all(info["attempts"] == info["accepted"] + info["rejected"])
    for c in range(4):
        yl, hs, status, hout = m.integrate_log(y[c], st.P[c], 1e-6)
        assert status == O.OK and len(hs) == info["accepted"][c]
        assert abs(hs.sum() - 1e-6) <= 1e-6 * 1e-12
        assert np.array_equal(yl, yo[c])
        assert np.array_equal(m.replay(y[c], st.P[c], hs), yo[c])
        assert hout == info["h"][c]


def test_failure_statuses(omech):
    m = omech("ch4_53")
    from tests.conftest import states
    st = states("ch4_53", 2, "ch4_partial", 32)
    y = m.state_from_TY(st.T, st.Y)
    _, info = m.integrate(y, st.P, 1e-6, max_steps=2)
    assert np.all(info["status"] == O.MAX_STEPS) and np.all(info["attempts"] == 2)
    _, info = m.integrate(y, st.P, 1e-6, h_min=1e-3)
    assert np.all(info["status"] == O.H_UNDERFLOW)
    bad = y.copy()
    bad[0, 3] = np.nan
    yb, info = m.integrate(bad, st.P, 1e-6)
    assert info["status"][0] == O.NONFINITE and info["status"][1] == O.OK
    _, info = m.integrate(y, st.P, 1e-6, T_min=5000.0)
    assert np.all(info["status"] == O.SKIPPED)


# ---------------------------------------------------------------- the other methods of Table T:solvers
# ROS3 and RODAS3 (Sandu et al. 1997), RODAS4 (Hairer & Wanner): order 3(2), 3(2), 4(3).
OTHERS = [(O.ROS3, 3), (O.RODAS3, 3), (O.RODAS4, 4)]
NCOND = {2: 2, 3: 4, 4: 8}


@pytest.mark.parametrize("tab,order", OTHERS + [(O.ROS4, 4)])
def test_tableau_order_conditions_all_methods(tab, order):
    g, Gamma, alpha, b, bh = untransformed(tab)
    assert O.tableau(tab)["order"] == order
    assert np.allclose(np.diag(Gamma), g, rtol=0, atol=1e-13)  # (inverse of a 6 x 6 matrix)
    r = order_residuals(g, Gamma, alpha, b)
    assert np.abs(r[:NCOND[order]]).max() < 1e-14
    if order < 4:
        assert np.abs(r[NCOND[order]:]).max() > 1e-4  # and not of the next order
    rh = order_residuals(g, Gamma, alpha, bh)
    assert np.abs(rh[:NCOND[order - 1]]).max() < 1e-14


@pytest.mark.parametrize("tab,order", OTHERS)
def test_l_stability_all_methods(tab, order):
    for w in np.logspace(-3, 6, 100):
        assert abs(R(1j * w, tab)) <= 1 + 1e-12
    assert abs(R(-1e12, tab)) < 1e-10


@pytest.mark.parametrize("tab,order", OTHERS)
def test_one_step_closed_form_all_methods(tab, order):
    A = np.array([[-1.0, 40.0], [-40.0, -1.0]])
    h = 0.05
    y0 = np.array([1.0, -0.5])
    y1, _ = O.step_linear(A, y0, h, tab)
    lam, V = np.linalg.eig(A)
    Rm = (V @ np.diag([R(h * l, tab) for l in lam]) @ np.linalg.inv(V)).real
    assert np.allclose(y1, Rm @ y0, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("tab,order", OTHERS)
def test_convergence_order_all_methods(omech, tab, order):
    m = omech("tiny_hon7.mech")
    y0 = _tiny_state(m)
    dt = 2e-5
    ref, _ = m.integrate(y0, ATM, dt, fixed_steps=8192, tableau=tab)
    sc = 1e-10 + 1e-6 * np.abs(ref[0])
    errs = []
    for K in (32, 64, 128):
        yk, _ = m.integrate(y0, ATM, dt, fixed_steps=K, tableau=tab)
        errs.append(np.sqrt(np.mean(((yk[0] - ref[0]) / sc) ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - order) < 0.2), orders


@pytest.mark.parametrize("tab,order", OTHERS)
def test_adaptive_all_methods_agree(omech, tab, order):
    """Every method reaches the same state within its tolerance (tight run as reference)."""
    m = omech("tiny_hon7.mech")
    y0 = _tiny_state(m, 1050.0)
    ref, _ = m.integrate(y0, ATM, 2e-5, rtol=1e-12, atol=1e-20, tableau=O.ROS4)
    yk, info = m.integrate(y0, ATM, 2e-5, rtol=1e-8, atol=1e-16, tableau=tab)
    assert info["status"][0] == O.OK
    assert np.max(np.abs(yk[0] - ref[0]) / (1e-14 + np.abs(ref[0]))) <= 1e-6
