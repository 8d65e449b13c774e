"""Pins of the oracle's W-method (ROS2 of Verwer et al. 1999, the method class the paper names
for reusing Jacobians and their factorisations) and of its Jacobian-reuse policy:
  * the stability function of the transformed coefficients equals the one of the method as
    published (k-form), R(z) = 1 + 2zu - z u^2 + z^2 u^2 / 2 with u = 1/(1 - g z), and it vanishes
    at infinity (L-stability) for g = 1 + 1/sqrt(2);
  * second order for ANY matrix in place of the Jacobian (a stale, perturbed or zero W), while
    ROS4 with the same stale W drops to first order (it is not a W-method);
  * the reuse policy: replaying it step by step with one-step calls gives the integrator's
    result (to rounding) with the same attempts and Jacobian evaluations; a cache carried into the next call is reused; reused results stay within
    the tolerance of a tight solution."""
import numpy as np

from oracle import oracle as O

ATM = 101325.0
G = 1.0 + 1.0 / np.sqrt(2.0)


def _tiny_state(m, T=1100.0):
    Y = np.array([0.02, 0.2, 0.01, 1e-4, 1e-4, 1e-3, 0.0])
    Y[-1] = 1 - Y.sum()
    return m.state_from_TY([T], [Y])[0]


def test_stability_function_and_l_stability():
    for z in (-0.3, -2.0, -17.0, 0.4 + 0.0):
        ynew, _ = O.step_linear(np.array([[z]]), np.array([1.0]), 1.0, tab=O.ROS2W)
        u = 1.0 / (1.0 - G * z)
        assert abs(ynew[0] - (1 + 2 * z * u - z * u * u + 0.5 * z * z * u * u)) < 1e-14
    ynew, _ = O.step_linear(np.array([[-1e12]]), np.array([1.0]), 1.0, tab=O.ROS2W)
    assert abs(ynew[0]) < 1e-10
    t = O.tableau(O.ROS2W)
    assert t["s"] == 2 and t["order"] == 2 and abs(t["gamma"] - G) < 1e-15


def _fixed_step_orders(m, tab, W, y0, dt=2e-5, Ks=(64, 128, 256)):
    ref, _ = m.integrate(y0, ATM, dt, fixed_steps=8192)
    sc = 1e-10 + 1e-6 * np.abs(ref[0])
    errs = []
    for K in Ks:
        y, h = y0.copy(), dt / K
        for _ in range(K):
            Wk = W if W is not None else m.jacobian(y[None], np.array([ATM]))[0]
            y, _ = m.step_w(y, ATM, h, Wk, tableau=tab)
        errs.append(np.sqrt(np.mean(((y - ref[0]) / sc) ** 2)))
    return np.log2(np.array(errs[:-1]) / np.array(errs[1:]))


def test_second_order_for_any_matrix(omech):
    m = omech("tiny_hon7.mech")
    y0 = _tiny_state(m)
    J0 = m.jacobian(y0[None], np.array([ATM]))[0]
    E = np.random.default_rng(0).normal(size=J0.shape) * np.abs(J0) * 0.3
    for W in (None, J0 + E, np.zeros_like(J0)):
        orders = _fixed_step_orders(m, O.ROS2W, W, y0)
        assert np.all(np.abs(orders - 2.0) < 0.1), orders
    # the same stale matrix costs ROS4 three orders: it is no W-method
    orders = _fixed_step_orders(m, O.ROS4, J0 + E, y0)
    assert np.all(np.abs(orders - 1.0) < 0.1), orders


def test_reuse_policy_replayed_step_by_step(omech):
    """integrate_w equals a step-by-step replay of the policy: reuse W while h is unchanged and the
    cache is younger than 32 accepted steps, else a fresh Jacobian; controller as the others."""
    m = omech("h2_13")
    from tests.conftest import states
    st = states("h2_13", 4, "h2_fresh", 501)
    y0 = m.state_from_TY(st.T, st.Y)
    dt, rtol, atol = 1e-5, 1e-6, 1e-10
    cache = m.w_cache(4)
    y, info = m.integrate_w(y0, st.P, dt, cache)
    for c in range(4):
        yc, t, h, W, hW, age, nj, att, rej = y0[c].copy(), 0.0, dt, None, 0.0, 0, 0, 0, False
        while True:
            last = t + 1.0001 * h >= dt
            hh = dt - t if last else h
            if not (hW == hh and age < 32):
                W, hW, age, nj = m.jacobian(yc[None], st.P[c:c + 1])[0], hh, 0, nj + 1
            yn, e = m.step_w(yc, st.P[c], hh, W)
            att += 1
            sc = atol + rtol * np.maximum(np.abs(yc), np.abs(yn))
            err = np.sqrt(np.mean((e / sc) ** 2))
            fac = min(6.0, max(0.2, 0.9 * max(err, 1e-10) ** -0.5))
            if err <= 1.0:
                yc, age = yn, age + 1
                if rej:
                    fac = min(fac, 1.0)
                rej = False
                if last:
                    break
                t, h = t + hh, hh * fac
            else:
                rej, h = True, hh * fac
        # (the error norm sums in another order here: equal up to rounding)
        assert np.allclose(yc, y[c], rtol=1e-12, atol=0)
        assert info["attempts"][c] == att and info["n_jac"][c] == nj and cache[2][c] == age
        assert abs(cache[1][c] - hW) <= 1e-12 * hW


def test_cache_carried_into_the_next_call(omech):
    """Near equilibrium a split step is one step of size dt: the second call reuses the first
    call's Jacobian (no evaluation) and still meets the tolerance of a tight solution."""
    m = omech("h2_13")
    from tests.conftest import states
    st = states("h2_13", 6, "h2_fresh", 502)
    y0 = m.state_from_TY(st.T, st.Y)
    yq, _ = m.integrate(y0, st.P, 1e-2)  # relax towards equilibrium
    cache = m.w_cache(6)
    h = np.zeros(6)
    y1, i1 = m.integrate_w(yq, st.P, 1e-6, cache, h=h)
    y2, i2 = m.integrate_w(y1, st.P, 1e-6, cache, h=i1["h"])
    assert np.all(i1["n_jac"] >= 1) and np.all(i2["status"] == 0)
    quiet = (i1["attempts"] == 1) & (i2["attempts"] == 1)
    assert quiet.sum() >= 3 and np.all(i2["n_jac"][quiet] == 0)
    yt, _ = m.integrate(y1, st.P, 1e-6, rtol=1e-12, atol=1e-16)
    w = 1e-10 + 1e-6 * np.abs(yt)
    assert np.sqrt(np.mean(((y2 - yt) / w) ** 2, axis=1)).max() <= 10.0
