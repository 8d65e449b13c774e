"""Pins of the oracle's explicit Runge-Kutta-Fehlberg 4(5) (the explicit solver of Table
T:solvers), carried as a tableau with u_i = h f(Y_i):
  * Butcher order conditions: all 17 rooted-tree conditions up to order 5 for the propagated
    weights, the 8 up to order 4 for the embedded ones (which fail order 5), row sums c = A 1;
  * one step on y' = A y reproduces the stability polynomial R(hA) y0;
  * fixed-step convergence order 5 and h^5 scaling of the error estimate on a non-stiff run;
  * adaptive integration agrees with a tight ROS4 run (an integrator sharing no stage code).
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests.test_oracle_ros4 import ATM, _tiny_state


def _rk():
    t = O.tableau(O.RKF45)
    A = t["a"]
    b = t["m"]
    bh = t["m"] - t["e"]
    return t, A, b, bh, A.sum(1)


def conditions(A, b, c):
    """Residuals of the rooted-tree order conditions, orders 1..5 (1 + 1 + 2 + 4 + 9)."""
    Ac = A @ c
    return np.array([
        b.sum() - 1,
        b @ c - 1 / 2,
        b @ c ** 2 - 1 / 3, b @ Ac - 1 / 6,
        b @ c ** 3 - 1 / 4, b @ (c * Ac) - 1 / 8, b @ (A @ c ** 2) - 1 / 12, b @ (A @ Ac) - 1 / 24,
        b @ c ** 4 - 1 / 5, b @ (c ** 2 * Ac) - 1 / 10, b @ (c * (A @ c ** 2)) - 1 / 15,
        b @ (c * (A @ Ac)) - 1 / 30, b @ Ac ** 2 - 1 / 20, b @ (A @ c ** 3) - 1 / 20,
        b @ (A @ (c * Ac)) - 1 / 40, b @ (A @ (A @ c ** 2)) - 1 / 60, b @ (A @ (A @ Ac)) - 1 / 120,
    ])


def test_order_conditions():
    t, A, b, bh, c = _rk()
    assert t["explicit"] and t["s"] == 6 and t["order"] == 5
    assert np.allclose(np.triu(A), 0.0)  # explicit
    assert np.allclose(c, [0, 1 / 4, 3 / 8, 12 / 13, 1, 1 / 2], rtol=0, atol=1e-15)
    assert np.abs(conditions(A, b, c)).max() < 1e-14
    rh = conditions(A, bh, c)
    assert np.abs(rh[:8]).max() < 1e-14 and np.abs(rh[8:]).max() > 1e-4


def R(z):
    t, A, b, _, _ = _rk()
    return 1 + z * b @ np.linalg.solve(np.eye(6) - z * A, np.ones(6))


@pytest.mark.parametrize("z", [-0.1, -1.5, 0.3])
def test_stability_polynomial(z):
    import math
    # order 5: R agrees with exp through z^5; the z^6 coefficient is b^T A^5 1
    t, A, b, _, _ = _rk()
    poly = sum(z ** k / math.factorial(k) for k in range(6)) + z ** 6 * (b @ np.linalg.matrix_power(A, 5) @ np.ones(6))
    assert abs(R(z) - poly) < 1e-14 * max(1.0, abs(poly))
    y1, _ = O.step_linear(np.array([[z]]), np.array([1.0]), 1.0, O.RKF45)
    assert abs(y1[0] - R(z)) < 1e-14


def test_one_step_matrix_closed_form():
    A = np.array([[-1.0, 3.0], [-3.0, -1.0]])
    h = 0.2
    y0 = np.array([1.0, -0.5])
    y1, _ = O.step_linear(A, y0, h, O.RKF45)
    lam, V = np.linalg.eig(A)
    Rm = (V @ np.diag([R(h * l) for l in lam]) @ np.linalg.inv(V)).real
    assert np.allclose(y1, Rm @ y0, rtol=1e-13, atol=1e-14)


def test_convergence_order_five_and_error_estimate(omech):
    m = omech("tiny_hon7.mech")
    y0 = _tiny_state(m, 900.0)  # cool enough for an explicit method at these step sizes
    dt = 1e-4
    ref, _ = m.integrate(y0, ATM, dt, fixed_steps=8192, tableau=O.RKF45)
    sc = 1e-10 + 1e-6 * np.abs(ref[0])
    errs = []
    for K in (32, 64, 128):
        yk, _ = m.integrate(y0, ATM, dt, fixed_steps=K, tableau=O.RKF45)
        errs.append(np.sqrt(np.mean(((yk[0] - ref[0]) / sc) ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 5) < 0.3), orders
    est = [np.abs(m.step(y0[None], ATM, h, tableau=O.RKF45)[1][0]).max() for h in (dt / 32, dt / 64)]
    assert abs(np.log2(est[0] / est[1]) - 5) < 0.3


def test_adaptive_agrees_with_tight_ros4(omech):
    m = omech("tiny_hon7.mech")
    y0 = _tiny_state(m, 900.0)
    ref, _ = m.integrate(y0, ATM, 2e-6, rtol=1e-12, atol=1e-20, tableau=O.ROS4)
    yk, info = m.integrate(y0, ATM, 2e-6, rtol=1e-8, atol=1e-16, tableau=O.RKF45)
    assert info["status"][0] == O.OK
    assert np.max(np.abs(yk[0] - ref[0]) / (1e-14 + np.abs(ref[0]))) <= 1e-6
