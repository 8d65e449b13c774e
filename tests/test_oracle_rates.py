"""Pins of the oracle's rate constants, rates of progress and source terms.

Hand cases on one-reaction mechanisms (the species block of tests/golden/tiny_hon7.mech plus one
reaction written here) fix the Chemkin-to-SI unit conversion and the Arrhenius form; limits fix
the falloff forms (Troe with Fcent = 1 is Lindemann, Pr -> inf gives k_inf, Pr -> 0 gives
k0 [M]); thermodynamic consistency fixes the reverse rate (q = 0 exactly where the mass-action
ratio equals K_c); reaction orders fix the mass-action products and the third-body factor.
"""
import math
import os

import numpy as np
import pytest

from tests.conftest import GOLDEN

R_U = 8314.462618
R_CAL = 1.987204258640832
ATM = 101325.0


def _species_block():
    lines = open(os.path.join(GOLDEN, "tiny_hon7.mech")).read().splitlines()
    out = []
    for ln in lines:
        if ln.startswith("REACTIONS"):
            break
        if ln.startswith("#") or not ln.strip():
            continue
        out.append(ln)
    return out


def one_reaction(tmp_path, rxn_lines, tag):
    path = tmp_path / ("r_%s.mech" % tag)
    body = _species_block() + ["REACTIONS 1"] + rxn_lines + ["END"]
    path.write_text("\n".join(body) + "\n")
    from oracle import oracle as O
    return O.Mechanism(str(path))


SP = ["H2", "O2", "H2O", "H", "O", "OH", "N2"]


def state(m, T, P, X):
    """y from mole fractions X (dict) at T, P."""
    Xv = np.array([X.get(s, 0.0) for s in SP])
    Xv[-1] = 1.0 - Xv[:-1].sum()
    Y = Xv * m.W / (Xv * m.W).sum()
    return m.state_from_TY([T], [Y])[0], Xv


def conc(T, P, X):
    return X * P / (R_U * T)  # kmol/m^3


def test_bimolecular_unit_conversion(tmp_path):
    # H2 + O <=> H + OH with A = 2e13 cm^3/mol/s, b = 0, Ea = 0: k = 2e10 m^3/kmol/s
    m = one_reaction(tmp_path, ["R ELEM 2 H2 1 O 1 2 H 1 OH 1 2.0e13 0.0 0.0"], "bi")
    T, P = 1200.0, 2 * ATM
    y, X = state(m, T, P, {"H2": 0.1, "O": 0.01, "O2": 0.1})
    r = m.rates(y, P)
    assert r["kf"][0] == pytest.approx(2.0e10, rel=1e-14)
    Cc = conc(T, P, X)
    assert np.allclose(r["C"], Cc, rtol=1e-13)
    assert r["qf"][0] == pytest.approx(2.0e10 * Cc[0] * Cc[4], rel=1e-13)


def test_arrhenius_temperature_dependence(tmp_path):
    # k = A T^b exp(-Ea / (R T)) in cgs, converted: 1 cm^3/mol = 1e-3 m^3/kmol
    A, b, Ea = 3.0e12, 1.7, 12000.0
    m = one_reaction(tmp_path, ["R ELEM 2 H2 1 O 1 2 H 1 OH 1 %r %r %r" % (A, b, Ea)], "arr")
    for T in (800.0, 1500.0, 2300.0):
        y, _ = state(m, T, ATM, {"H2": 0.1, "O": 0.01})
        k_cgs = A * T ** b * math.exp(-Ea / (R_CAL * T))
        assert m.rates(y, ATM)["kf"][0] == pytest.approx(k_cgs * 1e-3, rel=1e-13)


def test_third_body_units_and_efficiencies(tmp_path):
    # 2 H + M <=> H2 + M, A = 1e18 cm^6/mol^2/s -> 1e12 (m^3/kmol)^2/s; [M] = sum eff_k C_k
    m = one_reaction(tmp_path, ["R THIRD 1 H 2 1 H2 1 1.0e18 0.0 0.0", "EFF 2 H2O 6.0 O2 0.5"],
                     "tb")
    T, P = 1500.0, 5 * ATM
    y, X = state(m, T, P, {"H": 0.02, "H2O": 0.2, "O2": 0.1, "H2": 0.05})
    r = m.rates(y, P)
    Cc = conc(T, P, X)
    eff = np.ones(7)
    eff[SP.index("H2O")] = 6.0
    eff[SP.index("O2")] = 0.5
    M = (eff * Cc).sum()
    assert r["kf"][0] == pytest.approx(1.0e12, rel=1e-14)
    assert r["qf"][0] == pytest.approx(1.0e12 * Cc[3] ** 2 * M, rel=1e-12)


def _falloff(tmp_path, kind, troe=None, tag="fo"):
    lines = ["R %s 2 H 1 OH 1 1 H2O 1 1.0e13 0.3 1000.0" % kind, "EFF 0",
             "LOW 1.0e18 -1.2 500.0"]
    if troe:
        lines.append("TROE %r %r %r %r" % troe)
    return one_reaction(tmp_path, lines, tag)


def _kinf_k0(T):
    kinf = 1.0e13 * T ** 0.3 * math.exp(-1000.0 / (R_CAL * T)) * 1e-3
    k0 = 1.0e18 * T ** -1.2 * math.exp(-500.0 / (R_CAL * T)) * 1e-6
    return kinf, k0


def test_lindemann_blend(tmp_path):
    m = _falloff(tmp_path, "LIND", tag="lind")
    T, P = 1300.0, 3 * ATM
    y, X = state(m, T, P, {"H": 0.01, "OH": 0.01, "H2O": 0.1})
    kinf, k0 = _kinf_k0(T)
    M = conc(T, P, X).sum()
    Pr = k0 * M / kinf
    assert m.rates(y, P)["kf"][0] == pytest.approx(kinf * Pr / (1 + Pr), rel=1e-13)


def test_troe_with_unit_fcent_is_lindemann(tmp_path):
    # a = 0, T*** -> inf: Fcent = exp(-T/T***) = 1, so log10 F = 0
    mt = _falloff(tmp_path, "TROE", troe=(0.0, 1e300, 1000.0, 0.0), tag="troe1")
    ml = _falloff(tmp_path, "LIND", tag="lind1")
    for T, P in [(900.0, 0.1 * ATM), (1600.0, 10 * ATM), (2400.0, 50 * ATM)]:
        y, _ = state(mt, T, P, {"H": 0.01, "OH": 0.01, "H2O": 0.1})
        assert mt.rates(y, P)["kf"][0] == pytest.approx(ml.rates(y, P)["kf"][0], rel=1e-14)


def test_lindemann_pressure_limits(tmp_path):
    """k -> k_inf as Pr -> inf and k -> k0 [M] as Pr -> 0."""
    m = _falloff(tmp_path, "LIND", tag="limL")
    T = 1400.0
    kinf, k0 = _kinf_k0(T)
    P = 1e14 * ATM
    y, X = state(m, T, P, {"H": 0.01, "OH": 0.01, "H2O": 0.1})
    assert m.rates(y, P)["kf"][0] == pytest.approx(kinf, rel=1e-8)
    P = 1e-14 * ATM
    y, X = state(m, T, P, {"H": 0.01, "OH": 0.01, "H2O": 0.1})
    M = conc(T, P, X).sum()
    assert m.rates(y, P)["kf"][0] == pytest.approx(k0 * M, rel=1e-8)


def test_troe_broadening_hand_case(tmp_path):
    """k_Troe / k_Lindemann = F(Pr, Fcent) of Gilbert, Luther & Troe (1983):
    Fcent = (1-a) e^(-T/T***) + a e^(-T/T*) + e^(-T**/T), c = -0.4 - 0.67 log Fcent,
    n = 0.75 - 1.27 log Fcent, f1 = (log Pr + c) / (n - 0.14 (log Pr + c)),
    log F = log Fcent / (1 + f1^2), logs base 10; F < 1 away from the pole of f1."""
    troe = (0.6, 200.0, 2000.0, 5000.0)
    mt = _falloff(tmp_path, "TROE", troe=troe, tag="hcT")
    ml = _falloff(tmp_path, "LIND", tag="hcL")
    a, T3, T1, T2 = troe
    for T, P in [(1000.0, 0.5 * ATM), (1400.0, 5 * ATM), (2000.0, 40 * ATM)]:
        y, X = state(mt, T, P, {"H": 0.01, "OH": 0.01, "H2O": 0.1})
        kinf, k0 = _kinf_k0(T)
        Pr = k0 * conc(T, P, X).sum() / kinf
        Fc = (1 - a) * math.exp(-T / T3) + a * math.exp(-T / T1) + math.exp(-T2 / T)
        c = -0.4 - 0.67 * math.log10(Fc)
        n = 0.75 - 1.27 * math.log10(Fc)
        f1 = (math.log10(Pr) + c) / (n - 0.14 * (math.log10(Pr) + c))
        F = 10 ** (math.log10(Fc) / (1 + f1 * f1))
        assert F < 1.0
        ratio = mt.rates(y, P)["kf"][0] / ml.rates(y, P)["kf"][0]
        assert ratio == pytest.approx(F, rel=1e-13)


def test_detailed_balance(tmp_path):
    """q = 0 exactly when the mass-action ratio equals K_c = exp(-dG/RT) (P_atm / R T)^dnu."""
    m = one_reaction(tmp_path, ["R ELEM 1 OH 2 2 O 1 H2O 1 2.0e12 0.0 1000.0"], "db")
    T, P = 1700.0, 4 * ATM
    cp, h, s = zip(*[m.thermo(k, T) for k in range(m.ns)])
    g = np.array(s) - np.array(h)  # s/R - h/RT per species
    iO, iH2O, iOH = SP.index("O"), SP.index("H2O"), SP.index("OH")
    Kc = math.exp(g[iO] + g[iH2O] - 2 * g[iOH])  # dnu = 0
    # choose C_O C_H2O / C_OH^2 = Kc by setting X_O from the others
    X = {"OH": 0.01, "H2O": 0.05, "H2": 0.1}
    X["O"] = Kc * X["OH"] ** 2 / X["H2O"]
    y, _ = state(m, T, P, X)
    r = m.rates(y, P)
    assert abs(r["qf"][0] - r["qr"][0]) <= 1e-13 * r["qf"][0]
    assert np.all(np.abs(r["omega"]) <= 1e-13 * 2 * r["qf"][0])


def test_reverse_rate_pressure_dependence(tmp_path):
    """For dnu != 0 the reverse constant carries (P_atm/RT)^(-dnu): kr ratio across T fixed."""
    m = one_reaction(tmp_path, ["R THIRD 1 H 2 1 H2 1 1.0e18 0.0 0.0"], "kc")
    iH, iH2 = SP.index("H"), SP.index("H2")
    for T in (1000.0, 2000.0):
        y, _ = state(m, T, ATM, {"H": 0.01, "H2": 0.1})
        r = m.rates(y, ATM)
        _, hH, sH = m.thermo(iH, T)
        _, hH2, sH2 = m.thermo(iH2, T)
        Kc = math.exp((sH2 - hH2) - 2 * (sH - hH)) * (ATM / (R_U * T)) ** (-1)
        assert r["kr"][0] == pytest.approx(r["kf"][0] / Kc, rel=1e-12)


def test_mass_action_orders(omech):
    """Scaling P at fixed T and composition scales every concentration by the same factor:
    a plain bimolecular rate scales with its square, a third-body rate with the cube."""
    m = omech("tiny_hon7.mech")
    Y = np.array([0.02, 0.2, 0.01, 1e-3, 1e-3, 1e-3, 0.0])
    Y[-1] = 1 - Y.sum()
    y = m.state_from_TY([1300.0], [Y])[0]
    r1 = m.rates(y, ATM)
    r2 = m.rates(y, 3 * ATM)
    order = {0: 2, 1: 2, 2: 2, 3: 2, 4: 3}
    for r, o in order.items():
        assert r2["qf"][r] / r1["qf"][r] == pytest.approx(3.0 ** o, rel=1e-12)
        # reverse sides: 0..3 bimolecular, 4 (H2 + M) bimolecular with M
        assert r2["qr"][r] / r1["qr"][r] == pytest.approx(3.0 ** (2 if r < 4 else 2), rel=1e-12)


def test_source_is_mass_and_element_conservative(omech):
    """Every reaction is element balanced, so sum_k W_k dn_k/dt = 0 (bath gas included) and
    element production vanishes."""
    from tests.conftest import states
    for name, recipe in [("h2_13", "h2_fresh"), ("ch4_53", "ch4_partial")]:
        m = omech(name)
        st = states(name, 16, recipe, 5)
        y = m.state_from_TY(st.T, st.Y)
        f = m.source(y, st.P)
        for c in range(16):
            r = m.rates(y[c], st.P[c])
            om = r["omega"]
            gross = np.abs(m.nu_f - m.nu_r).T @ (r["qf"] + r["qr"])
            assert abs((m.W * om).sum()) <= 1e-12 * (m.W * gross).sum()
            assert np.all(np.abs(m.elem @ om) <= 1e-12 * (m.elem @ gross + 1e-300))
