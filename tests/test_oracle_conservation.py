"""Invariants of the oracle's integrated solution and its sensitivities.

* Elements: a Rosenbrock step with the exact Jacobian preserves every linear invariant of the
  ODE, and element counts sum_k a_ek n_k are linear invariants (every reaction is element
  balanced), so they hold to roundoff.
* Mass: the bath gas closure of Eq. (e:n_nsp) (read on a unit-mass basis) keeps sum_k W_k n_k = 1.
* Enthalpy: the adiabatic constant-pressure energy balance keeps the mixture enthalpy
  sum_k n_k h_k(T); Rosenbrock does not preserve this nonlinear invariant exactly, so it holds
  to the integration tolerance.
* Equilibrium: integrated long enough, every reversible reaction reaches q_f = q_r and the
  composition equals the minimum of the Gibbs energy at the final (T, P) found independently by
  the element-potential method.
* Sensitivities: complex-step derivatives through a frozen step sequence (replay) agree with
  central differences of the same map.
"""
import numpy as np
import pytest
import scipy.optimize

from oracle import oracle as O
from tests.conftest import states

ATM = 101325.0


def enthalpy(m, y):
    n = m.moles_all(y)
    return np.array([sum(n[c, k] * m.thermo(k, y[c, 0])[1] * y[c, 0] for k in range(m.ns))
                     for c in range(y.shape[0])])


@pytest.mark.parametrize("name,recipe,dt", [("h2_13", "h2_fresh", 1e-3),
                                             ("ch4_53", "ch4_partial", 1e-6)])
def test_elements_mass_enthalpy(omech, name, recipe, dt):
    m = omech(name)
    st = states(name, 4, recipe, 51)
    y = m.state_from_TY(st.T, st.Y)
    yo, info = m.integrate(y, st.P, dt)
    assert np.all(info["status"] == O.OK)
    n0, n1 = m.moles_all(y), m.moles_all(yo)
    e0, e1 = m.elem @ n0.T, m.elem @ n1.T
    assert np.abs(e1 - e0).max() <= 1e-12 * np.abs(e0).max()
    assert np.abs(n1 @ m.W - 1.0).max() <= 1e-14
    H0, H1 = enthalpy(m, y), enthalpy(m, yo)
    # |dH| within the tolerance-scaled error of the temperature: cp * (rtol T + atol)
    cp = np.array([sum(n1[c, k] * m.thermo(k, yo[c, 0])[0] for k in range(m.ns))
                   for c in range(4)])
    assert np.all(np.abs(H1 - H0) <= 10 * cp * (1e-6 * yo[:, 0]))


def gibbs_equilibrium(m, T, P, b, n_guess):
    """Moles per kg minimising G at (T, P) under element totals b (element-potential method)."""
    g = np.array([m.thermo(k, T)[1] - m.thermo(k, T)[2] for k in range(m.ns)])  # g/RT
    A = m.elem.astype(float)
    active = b > 0

    def n_of(x):
        lam, lnN = x[:-1], x[-1]
        return np.exp(lnN + np.log(ATM / P) - g + lam @ A[active])

    def res(x):
        n = n_of(x)
        return np.concatenate([(A[active] @ n - b[active]) / b[active],
                               [(n.sum() - np.exp(x[-1])) / np.exp(x[-1])]])

    # start from element potentials fitted to a nearby composition (the problem is convex, so
    # the root is unique; the start only has to be in its basin for the Newton-type solver)
    lnN = np.log(n_guess.sum())
    lam0, *_ = np.linalg.lstsq(A[active].T, np.log(n_guess) + g - lnN - np.log(ATM / P),
                               rcond=None)
    x0 = np.concatenate([lam0 + 0.05, [lnN + 0.05]])
    sol = scipy.optimize.root(res, x0, method="hybr", tol=1e-14)
    assert sol.success
    return n_of(sol.x)


def test_long_time_equilibrium(omech):
    m = omech("tiny_hon7.mech")
    Y = np.array([[0.02, 0.2, 0.01, 1e-4, 1e-4, 1e-3, 0.0]])
    Y[:, -1] = 1 - Y.sum(1)
    y = m.state_from_TY([1100.0], Y)
    yo, info = m.integrate(y, ATM, 100.0, rtol=1e-8, atol=1e-16)
    assert info["status"][0] == O.OK
    r = m.rates(yo[0], ATM)
    assert np.all(np.abs(r["qf"] - r["qr"]) <= 1e-9 * np.maximum(r["qf"], r["qr"]))
    n = m.moles_all(yo)[0]
    neq = gibbs_equilibrium(m, yo[0, 0], ATM, m.elem @ n, n)
    assert np.allclose(n, neq, rtol=1e-7, atol=1e-14)


def test_replay_sensitivities_complex_step_vs_fd(omech):
    m = omech("h2_13")
    st = states("h2_13", 1, "h2_fresh", 52)
    y0 = m.state_from_TY(st.T, st.Y)[0]
    P = st.P[0]
    yT, hs, status, _ = m.integrate_log(y0, P, 1e-6)
    assert status == O.OK and len(hs) > 2
    rng = np.random.default_rng(3)
    dy = rng.normal(size=m.N) * np.maximum(np.abs(y0), 1e-9)
    dl = rng.normal(size=m.nr)
    hc = 1e-30
    cs = m.replay_cplx(y0 + 1j * hc * dy, P, hs, lnA=m.lnA + 1j * hc * dl).imag / hc
    e = 1e-7
    fd = (m.replay(y0 + e * dy, P, hs, lnA=m.lnA + e * dl)
          - m.replay(y0 - e * dy, P, hs, lnA=m.lnA - e * dl)) / (2 * e)
    assert np.allclose(cs, fd, rtol=1e-5, atol=1e-7 * np.abs(cs).max())
