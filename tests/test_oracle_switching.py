"""Pins of the oracle's per-cell switching between the explicit RKF45 and a Rosenbrock method
(the stiffness-aware policy the GPU path mirrors): dispatch to the right integrator, fall-back from
the initial state when the explicit budget runs out, and the stiffness rule computed
independently from the oracle's Jacobian."""
import numpy as np

from oracle import oracle as O
from tests.conftest import states


def _rho(om, y, P, rtol=1e-6, atol=1e-10):
    """max_i sum_j |J_ij| w_j / w_i with w = atol + rtol |y|, from the oracle's Jacobian."""
    J = om.jacobian(y[None], np.array([P]))[0]
    w = atol + rtol * np.abs(y)
    return np.max((np.abs(J) * w[None, :]).sum(axis=1) / w)


def test_explicit_cells_take_rkf45_under_their_budget(omech):
    om = omech("h2_13")
    st = states("h2_13", 24, "h2_fresh", 401)
    y0 = om.state_from_TY(st.T, st.Y)
    meth = np.full(24, 500, dtype=np.int32)
    y, info = om.integrate_auto(y0, st.P, 1e-6, meth)
    ye, ie = om.integrate(y0, st.P, 1e-6, tableau=4, max_steps=500, threads=1)
    assert np.all(info["status"] == 0) and np.all(ie["status"] == 0)
    assert np.array_equal(y, ye) and np.array_equal(info["attempts"], ie["attempts"])
    assert np.array_equal(meth, 4 * ie["attempts"] + 8)


def test_budget_exhausted_falls_back_to_rosenbrock_from_the_initial_state(omech):
    om = omech("ch4_53")
    st = states("ch4_53", 12, "ch4_partial", 402)
    y0 = om.state_from_TY(st.T, st.Y)
    h0 = np.full(12, 1e-8)
    meth = np.full(12, 3, dtype=np.int32)  # far too few explicit attempts for stiff cells
    y, info = om.integrate_auto(y0, st.P, 1e-6, meth, h=h0)
    yr, ir = om.integrate(y0, st.P, 1e-6, h=h0, threads=1)
    assert np.all(info["status"] == 0)
    assert np.array_equal(y, yr) and np.array_equal(info["attempts"], ir["attempts"])
    assert np.array_equal(info["h"], ir["h"])
    for c in range(12):  # stiff cells: the rule keeps them on the Rosenbrock method
        a = ir["attempts"][c]
        assert meth[c] == (4 * a + 8 if 1e-6 * _rho(om, y0[c], st.P[c]) <= 3 * a else 0)
    assert np.all(meth == 0)


def test_stiffness_rule_matches_the_jacobian_bound(omech):
    """After a Rosenbrock integration the next method follows dt * rho <= 3 attempts, rho from
    the Jacobian at the initial state (computed here with numpy from the oracle's Jacobian)."""
    om = omech("h2_13")
    st = states("h2_13", 40, "h2_fresh", 403)
    y0 = om.state_from_TY(st.T, st.Y)
    meth = np.zeros(40, dtype=np.int32)
    y, info = om.integrate_auto(y0, st.P, 1e-6, meth)
    yr, ir = om.integrate(y0, st.P, 1e-6, threads=1)
    assert np.array_equal(y, yr)
    want = np.array([4 * a + 8 if 1e-6 * _rho(om, y0[c], st.P[c]) <= 3 * a else 0
                     for c, a in enumerate(ir["attempts"])], dtype=np.int32)
    assert np.array_equal(meth, want)
    assert (meth > 0).mean() > 0.5  # these H2 cells are not stiff over 1 us


def test_skipped_and_nonfinite_cells_keep_their_method(omech):
    om = omech("h2_13")
    st = states("h2_13", 3, "h2_fresh", 404)
    y0 = om.state_from_TY(st.T, st.Y)
    y0[1, 0] = np.nan
    y0[2, 0] = 200.0
    meth = np.array([0, 7, 9], dtype=np.int32)
    y, info = om.integrate_auto(y0, st.P, 1e-6, meth, T_min=300.0)
    assert info["status"].tolist() == [0, 3, 4]
    assert meth[1] == 7 and meth[2] == 9


def test_w_method_alternative_for_quiescent_cells(omech):
    """With the W-method as the alternative: a cell whose Rosenbrock split step was one attempt
    moves to the W-method (budget 12) and empties its cache; on the W-method it reuses the
    factorisation across calls (cache age grows, step size kept)."""
    om = omech("h2_13")
    st = states("h2_13", 8, "h2_fresh", 405)
    y0 = om.state_from_TY(st.T, st.Y)
    yq, _ = om.integrate(y0[:4], st.P[:4], 1e-2)  # four relaxed cells, four fresh ones
    y = np.concatenate([yq, y0[4:]])
    meth = np.zeros(8, dtype=np.int32)
    cache = om.w_cache(8)
    h = np.zeros(8)
    y1, i1 = om.integrate_auto(y, st.P, 1e-6, meth, h=h, alt=O.ROS2W, cache=cache)
    assert np.all(cache[1] == 0.0)  # emptied by the Rosenbrock integration
    yr, ir = om.integrate(y, st.P, 1e-6, threads=1)
    assert np.array_equal(y1, yr)
    quiescent = (ir["attempts"] == 1) & (ir["h"] >= 2e-6)
    assert np.array_equal(meth, np.where(quiescent, 12, 0).astype(np.int32))
    assert np.all(meth[:4] == 12)
    y2, i2 = om.integrate_auto(y1, st.P, 1e-6, meth, h=i1["h"], alt=O.ROS2W, cache=cache)
    assert np.all(i2["status"] == 0)
    assert np.all(cache[1][:4] > 0) and np.all(cache[2][:4] == i2["attempts"][:4])
    age = cache[2][:4].copy()
    y3, i3 = om.integrate_auto(y2, st.P, 1e-6, meth, h=i2["h"], alt=O.ROS2W, cache=cache)
    quiet = i3["attempts"][:4] == 1
    assert quiet.any() and np.all(cache[2][:4][quiet] == age[quiet] + 1)  # reused, aged by one


def test_w_method_entry_needs_a_step_margin(omech):
    """A single-attempt Rosenbrock split step sends a cell to the W-method only when the step-size
    controller proposes at least 2 dt next: four cells relaxed for 1e-4 s, one step of 2e-4 s each,
    two with a proposal below the margin (the one step only just fitted) and two above."""
    om = omech("h2_13")
    st = states("h2_13", 8, "h2_fresh", 405)
    P = st.P[:4]
    yq, _ = om.integrate(om.state_from_TY(st.T[:4], st.Y[:4]), P, 1e-4)
    dt = 2e-4
    yr, ir = om.integrate(yq, P, dt, threads=1)
    assert np.all(ir["attempts"] == 1)
    below = ir["h"] < 2 * dt
    assert below.any() and not below.all()  # both branches of the rule
    meth = np.zeros(4, dtype=np.int32)
    y, info = om.integrate_auto(yq, P, dt, meth, alt=O.ROS2W, cache=om.w_cache(4))
    assert np.array_equal(y, yr)
    assert np.array_equal(meth, np.where(below, 0, 12).astype(np.int32))
