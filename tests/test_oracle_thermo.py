"""Pins of the oracle's NASA-7 thermodynamics (cp/R, h/RT, s/R).

The paper delegates thermodynamics to pyJac (Sec. 2.1); the oracle uses the NASA-7 polynomial
forms.  These tests fix them by properties that any mistake in a coefficient, a power or the
range switch breaks: dh/dT = cp and ds/dT = cp/T (complex-step derivative of the oracle's own
h and s), continuity at Tmid, the reference values at 298.15 K written into the spec by the
generator (which never evaluates these functions), and the monatomic ideal-gas limit cp = 5/2 R.
"""
import numpy as np
import pytest

MECHS = ["h2_13", "ch4_53", "ch4_111"]
TS = [300.0, 650.0, 999.0, 1001.0, 1500.0, 2400.0, 3500.0]


@pytest.mark.parametrize("name", MECHS)
def test_enthalpy_derivative_is_cp(omech, name):
    m = omech(name)
    hstep = 1e-20
    for k in range(m.ns):
        for T in TS:
            cp, hRT, sR = m.thermo(k, T)
            _, hc, sc = m.thermo_cplx(k, T + 1j * hstep)
            dH = (hc * (T + 1j * hstep)).imag / hstep  # d(h/R)/dT
            dS = sc.imag / hstep
            assert abs(dH - cp) <= 1e-12 * abs(cp), (k, T)
            assert abs(dS - cp / T) <= 1e-12 * abs(cp / T), (k, T)


@pytest.mark.parametrize("name", MECHS)
def test_continuity_at_tmid(omech, name):
    m = omech(name)
    for k in range(m.ns):
        Tm = m.Tmid[k]
        lo = np.array(m.thermo(k, Tm * (1 - 1e-15)))
        hi = np.array(m.thermo(k, Tm))
        # h/RT and s/R continuous; cp continuous by construction of the generator
        assert np.allclose(lo, hi, rtol=1e-9, atol=1e-9), (k, lo, hi)


@pytest.mark.parametrize("name", MECHS)
def test_reference_state_values(omech, name):
    m = omech(name)
    T0 = 298.15
    for k in range(m.ns):
        cp, hRT, sR = m.thermo(k, T0)
        assert abs(hRT * T0 - m.hf_R[k]) <= 1e-9 * max(1.0, abs(m.hf_R[k])), k
        assert abs(sR - m.s_R[k]) <= 1e-10 * abs(m.s_R[k]), k


def test_monatomic_heat_capacity(omech):
    m = omech("h2_13")
    atoms = [k for k in range(m.ns) if m.elem[:, k].sum() == 1]
    assert atoms, "the H/O/N mechanism has atoms H, O, N"
    for k in atoms:
        for T in TS:
            assert m.thermo(k, T)[0] == 2.5


def _nasa_lines(path):
    """{species: (LO, HI)} read from the spec text."""
    out, cur = {}, None
    for line in open(path):
        t = line.split()
        if not t:
            continue
        if t[0] == "SP":
            cur = t[1]
        elif t[0] in ("LO", "HI"):
            out.setdefault(cur, {})[t[0]] = np.array([float(v) for v in t[1:8]])
    return out


def test_range_switch_follows_spec_lines(omech, mech_path):
    """cp/R below Tmid follows the LO line of the spec and at/above Tmid the HI line."""
    m = omech("ch4_53")
    nasa = _nasa_lines(mech_path("ch4_53"))
    names = list(nasa.keys())
    for k, name in enumerate(names):
        for T, key in [(500.0, "LO"), (999.0, "LO"), (1000.0, "HI"), (2200.0, "HI")]:
            a = nasa[name][key]
            cp = a[0] + a[1] * T + a[2] * T ** 2 + a[3] * T ** 3 + a[4] * T ** 4
            assert abs(m.thermo(k, T)[0] - cp) <= 1e-13 * abs(cp), (name, T)
