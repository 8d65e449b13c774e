"""Seeded synthetic inputs: kinetic mechanisms (plain-text spec files) and CFD-cell states.

This module is the one piece shared by the CUDA path, the tests and the CPU oracle. It
produces *inputs only*: a reaction mechanism (species with NASA-7 thermodynamics, element
balanced reversible reactions with Arrhenius / third-body / Lindemann / Troe rate data) and
cell states (T, P, mass fractions).  It evaluates no source term, rate, Jacobian or
integrator step.  The only arithmetic here builds the inputs themselves: it fits heat-capacity
curves to NASA-7 polynomials, chooses kinetic parameters and mixes compositions.

Mechanism shape follows the statement of the problem in Sec. 2.1 (state of T and species
moles, last species = bath gas N2, Eq. (e:state_vec)/(e:n_nsp)); the paper takes its kinetics from
GRI-Mech 3.0 (53 species / 325 reactions), which is not reproduced: species formulas and
reactions are drawn at random under element balance, and only the sizes match.

Spec file format (whitespace separated, '#' comments, one record per line)::

    MECHANISM <name> <seed>
    ELEMENTS <e1> <e2> ...
    SPECIES <Ns>
    SP <name> <W [kg/kmol]> <count e1> <count e2> ... <Tlow> <Tmid> <Thigh> <hf298/R [K]> <s298/R>
    LO <a1> ... <a7>           # NASA-7 coefficients, T < Tmid
    HI <a1> ... <a7>           # NASA-7 coefficients, T >= Tmid
    REACTIONS <Nr>
    R <type> <nreac> (<sp> <nu>)... <nprod> (<sp> <nu>)... <A> <b> <Ea>
    EFF <k> (<sp> <eff>)...    # types THIRD, LIND, TROE; species not listed have efficiency 1
    LOW <A0> <b0> <Ea0>        # types LIND, TROE: low-pressure limit
    TROE <a> <T3> <T1> <T2>    # type TROE; T2 <= 0 means "no T** term"
    END

``type`` is ELEM (plain mass action), THIRD (q multiplied by [M]), LIND (Lindemann falloff) or
TROE (Troe falloff).  Rate units follow the Chemkin convention: A in (cm^3/mol)^(order-1)/s,
where the order counts reactant stoichiometric coefficients plus one for the explicit +M of
THIRD reactions (LOW lines count the +M as well); Ea in cal/mol.  Every reaction is
reversible, its reverse rate coming from the equilibrium constant.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

ATOMIC_W = {"C": 12.011, "H": 1.008, "N": 14.007, "O": 15.999}
VALENCE = {"C": 4, "H": 1, "N": 3, "O": 2}
NAME_ORDER = ("C", "H", "N", "O")
R_KJ = 8.314462618e-3  # kJ/(mol K): converts kJ/mol to K for the h/R entries of the spec
ATM = 101325.0

# ----------------------------------------------------------------------------- data types


@dataclasses.dataclass
class Species:
    name: str
    counts: Dict[str, int]
    W: float
    hf_R: float  # standard enthalpy of formation at 298.15 K divided by R, in K
    s_R: float  # standard entropy at 298.15 K divided by R
    lo: List[float]
    hi: List[float]
    Tlow: float = 300.0
    Tmid: float = 1000.0
    Thigh: float = 5000.0


@dataclasses.dataclass
class Reaction:
    kind: str  # ELEM | THIRD | LIND | TROE
    reac: List[Tuple[int, int]]  # (species index, nu)
    prod: List[Tuple[int, int]]
    A: float  # Chemkin units (cm, mol, s)
    b: float
    Ea: float  # cal/mol
    eff: List[Tuple[int, float]] = dataclasses.field(default_factory=list)
    low: Optional[Tuple[float, float, float]] = None
    troe: Optional[Tuple[float, float, float, float]] = None


@dataclasses.dataclass
class Mechanism:
    name: str
    seed: int
    elements: List[str]
    species: List[Species]
    reactions: List[Reaction]

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return len(self.reactions)

    def index(self, name: str) -> int:
        for i, s in enumerate(self.species):
            if s.name == name:
                return i
        raise KeyError(name)

    def weights(self) -> np.ndarray:
        return np.array([s.W for s in self.species])

    def element_matrix(self) -> np.ndarray:
        """[n_elements, n_species] atom counts."""
        return np.array([[s.counts.get(e, 0) for s in self.species] for e in self.elements],
                        dtype=float)


# ----------------------------------------------------------------------------- species


def formula_name(counts: Dict[str, int]) -> str:
    out = []
    for e in NAME_ORDER:
        c = counts.get(e, 0)
        if c:
            out.append(e + (str(c) if c > 1 else ""))
    return "".join(out)


def parse_formula(name: str) -> Dict[str, int]:
    counts: Dict[str, int] = {}
    i = 0
    while i < len(name):
        e = name[i]
        i += 1
        j = i
        while j < len(name) and name[j].isdigit():
            j += 1
        counts[e] = counts.get(e, 0) + (int(name[i:j]) if j > i else 1)
        i = j
    return counts


def _n_atoms(c: Dict[str, int]) -> int:
    return sum(c.values())


def _unpaired(c: Dict[str, int]) -> int:
    n = _n_atoms(c)
    v = sum(VALENCE[e] * k for e, k in c.items())
    if n == 1:
        return v
    return (v - 2 * (n - 1)) % 2


def _feasible(c: Dict[str, int]) -> bool:
    n = _n_atoms(c)
    if n == 0 or n > 9:
        return False
    heavy = n - c.get("H", 0)
    if heavy == 0:
        return c.get("H", 0) in (1, 2)
    v_heavy = sum(VALENCE[e] * k for e, k in c.items() if e != "H")
    # the heavy atoms form a tree and hydrogens hang off the remaining valence
    return c.get("H", 0) <= v_heavy - 2 * (heavy - 1)


CORE_HON = ["H2", "O2", "H2O", "H", "O", "OH", "HO2", "H2O2", "N", "NO", "NO2", "N2O", "N2"]
CORE_C = ["CO", "CO2", "CH4", "CH3", "CH2O", "HCO"]


def _species_formulas(elements: Sequence[str], n_species: int, rng) -> List[Dict[str, int]]:
    if set(elements) == {"H", "O", "N"}:
        if n_species != len(CORE_HON):
            raise ValueError("an H/O/N mechanism has exactly %d species" % len(CORE_HON))
        return [parse_formula(s) for s in CORE_HON]
    core = [s for s in CORE_HON if s != "N2"] + CORE_C
    chosen = [parse_formula(s) for s in core]
    seen = {formula_name(c) for c in chosen} | {"N2"}
    cands = []
    for c_, h_, n_, o_ in itertools.product(range(4), range(9), range(3), range(4)):
        cnt = {k: v for k, v in zip(NAME_ORDER, (c_, h_, n_, o_)) if v}
        if not cnt or not _feasible(cnt):
            continue
        if formula_name(cnt) in seen:
            continue
        cands.append(cnt)
    # prefer small species (as in real mechanisms) but keep the draw random
    w = np.array([1.0 / (1.0 + _n_atoms(c)) ** 2 for c in cands])
    k = n_species - 1 - len(chosen)
    if k < 0:
        raise ValueError("too few species for the C/H/O/N core")
    pick = rng.choice(len(cands), size=k, replace=False, p=w / w.sum())
    chosen += [cands[i] for i in sorted(pick)]
    chosen.append({"N": 2})  # bath gas last
    return chosen


def _cp_model(T: np.ndarray, n_atoms: int, thetas: np.ndarray) -> np.ndarray:
    """Heat capacity cp/R of an ideal gas: translation + rotation + Einstein vibrations."""
    cp = np.full_like(T, 2.5)
    if n_atoms == 1:
        return cp
    cp += 1.0 if n_atoms == 2 else 1.5
    for th in thetas:
        x = th / T
        ex = np.exp(-x)
        cp += x * x * ex / (1.0 - ex) ** 2
    return cp


def _fit_cp(Ta: float, Tb: float, n_atoms: int, thetas) -> np.ndarray:
    T = np.linspace(Ta, Tb, 64)
    cp = _cp_model(T, n_atoms, thetas)
    x = T / 1000.0
    V = np.vander(x, 5, increasing=True)
    c, *_ = np.linalg.lstsq(V, cp, rcond=None)
    return c / np.array([1.0, 1e3, 1e6, 1e9, 1e12])  # polynomial coefficients in T


def _h_poly(a: Sequence[float], T: float) -> float:
    """Integral of the cp/R polynomial from 0 to T, i.e. h/R without the a6 constant."""
    return a[0] * T + a[1] * T ** 2 / 2 + a[2] * T ** 3 / 3 + a[3] * T ** 4 / 4 + a[4] * T ** 5 / 5


def _s_poly(a: Sequence[float], T: float) -> float:
    return a[0] * math.log(T) + a[1] * T + a[2] * T ** 2 / 2 + a[3] * T ** 3 / 3 + a[4] * T ** 4 / 4


def _make_species(counts: Dict[str, int], rng) -> Species:
    n = _n_atoms(counts)
    W = sum(ATOMIC_W[e] * k for e, k in counts.items())
    # enthalpy of formation (kJ/mol) from a crude bond model: radicals cost ~200 kJ/mol,
    # H bound to C and O bound to H/C stabilise the molecule; plus seeded noise
    u = _unpaired(counts)
    c, h, o = counts.get("C", 0), counts.get("H", 0), counts.get("O", 0)
    hf = 200.0 * min(u, 1) + 60.0 * max(u - 1, 0) + 87.0 * c - 40.0 * min(h, 4 * c)
    hf -= 240.0 * min(o, (h + 4 * c) / 2.0)
    if formula_name(counts) not in ("H2", "O2", "N2"):
        hf += rng.normal(0.0, 15.0)
    s = 14.0 + 2.5 * math.log(W) + 1.5 * (n - 1) + rng.normal(0.0, 0.5)
    if n == 1:
        thetas = np.zeros(0)
    else:
        nv = 1 if n == 2 else 3 * n - 6
        thetas = np.exp(rng.uniform(math.log(400.0), math.log(4500.0), size=nv))
    Tlow, Tmid, Thigh = 300.0, 1000.0, 5000.0
    lo = list(_fit_cp(Tlow, Tmid, n, thetas))
    hi = list(_fit_cp(Tmid, Thigh, n, thetas))
    if n == 1:
        lo = [2.5, 0.0, 0.0, 0.0, 0.0]
        hi = [2.5, 0.0, 0.0, 0.0, 0.0]
    # make cp continuous at Tmid by moving the constant of the high range
    cp_lo_mid = sum(lo[i] * Tmid ** i for i in range(5))
    cp_hi_mid = sum(hi[i] * Tmid ** i for i in range(5))
    hi[0] += cp_lo_mid - cp_hi_mid
    hf_R = hf / R_KJ
    T0 = 298.15
    a6_lo = hf_R - _h_poly(lo, T0)
    a7_lo = s - _s_poly(lo, T0)
    # h and s continuous at Tmid
    a6_hi = _h_poly(lo, Tmid) + a6_lo - _h_poly(hi, Tmid)
    a7_hi = _s_poly(lo, Tmid) + a7_lo - _s_poly(hi, Tmid)
    return Species(formula_name(counts), dict(counts), W, hf_R, s, lo + [a6_lo, a7_lo],
                   hi + [a6_hi, a7_hi], Tlow, Tmid, Thigh)


# ----------------------------------------------------------------------------- reactions


def _evec(sp: Species, elements) -> Tuple[int, ...]:
    return tuple(sp.counts.get(e, 0) for e in elements)


def _draw_arrhenius(rng, order: int, ea_max: float) -> Tuple[float, float, float]:
    """A log-uniform in [1e6, 1e16] within the collision limit at 1500 K, b in [-2, 2],
    Ea uniform in [0, ea_max] kcal/mol (returned in cal/mol)."""
    cap = {1: 14.0, 2: 14.5, 3: 17.0}[order]
    while True:
        b = rng.uniform(-2.0, 2.0)
        hi = min(16.0, cap - b * math.log10(1500.0))
        if hi > 6.5:
            break
    lA = rng.uniform(6.0, hi)
    return 10.0 ** lA, b, rng.uniform(0.0, ea_max) * 1000.0


def make_mechanism(n_species: int, n_reactions: int, n_third: int, n_falloff: int,
                   n_troe: int, elements: Sequence[str], seed: int,
                   name: Optional[str] = None) -> Mechanism:
    """Draw an element-balanced reversible mechanism (see module docstring)."""
    rng = np.random.default_rng(seed)
    elements = list(elements)
    formulas = _species_formulas(elements, n_species, rng)
    species = [_make_species(c, rng) for c in formulas]
    ns = len(species)
    ev = [_evec(s, elements) for s in species]
    hf = np.array([s.hf_R for s in species])

    pairs: Dict[Tuple[int, ...], List[Tuple[int, int]]] = {}
    for i in range(ns):
        for j in range(i, ns):
            key = tuple(a + b for a, b in zip(ev[i], ev[j]))
            pairs.setdefault(key, []).append((i, j))
    single: Dict[Tuple[int, ...], List[int]] = {}
    for k in range(ns):
        single.setdefault(ev[k], []).append(k)

    recomb = []  # (i, j, k): i + j -> k
    for key, plist in pairs.items():
        for k in single.get(key, []):
            for (i, j) in plist:
                if k not in (i, j):
                    recomb.append((i, j, k))
    exch = []  # ((i, j), (k, l))
    for key, plist in pairs.items():
        for p, q in itertools.combinations(plist, 2):
            exch.append((p, q))
    rng.shuffle(recomb)
    order = rng.permutation(len(exch))
    exch = [exch[i] for i in order]

    used = set()
    reactions: List[Reaction] = []
    covered = np.zeros(ns, bool)
    n_tb_total = n_third + n_falloff
    if len(recomb) < n_tb_total:
        raise ValueError("not enough association reactions for the third-body/falloff count")

    def sig(r, p):
        return (tuple(sorted(r)), tuple(sorted(p)))

    def add(kind, r, p):
        a, b_ = sig(r, p), sig(p, r)
        if a in used or b_ in used:
            return False
        used.add(a)
        used.add(b_)
        reac = [(s, r.count(s)) for s in sorted(set(r))]
        prod = [(s, p.count(s)) for s in sorted(set(p))]
        if kind == "ELEM":
            A, b, Ea = _draw_arrhenius(rng, len(r), 50.0)
            rx = Reaction("ELEM", reac, prod, A, b, Ea)
        else:
            if kind == "THIRD":
                A, b, Ea = _draw_arrhenius(rng, len(r) + 1, 5.0)
                rx = Reaction("THIRD", reac, prod, A, b, Ea)
            else:
                A, b, Ea = _draw_arrhenius(rng, len(r), 10.0)
                A0 = 10.0 ** rng.uniform(12.0, 19.0)
                low = (A0, rng.uniform(-3.0, 0.0), rng.uniform(0.0, 3.0) * 1000.0)
                rx = Reaction(kind, reac, prod, A, b, Ea, low=low)
                if kind == "TROE":
                    T2 = rng.uniform(3000.0, 10000.0) if rng.random() < 0.5 else 0.0
                    rx.troe = (rng.uniform(0.3, 0.8), rng.uniform(50.0, 500.0),
                               rng.uniform(500.0, 5000.0), T2)
            neff = int(rng.integers(0, 5))
            effs = rng.choice(ns, size=min(neff, ns), replace=False)
            rx.eff = [(int(k), float(math.exp(rng.uniform(math.log(0.4), math.log(12.0)))))
                      for k in sorted(effs)]
        reactions.append(rx)
        for s in r + p:
            covered[s] = True
        return True

    kinds = ["TROE"] * n_troe + ["LIND"] * (n_falloff - n_troe) + ["THIRD"] * n_third
    it = iter(recomb)
    for kind in kinds:
        while True:
            i, j, k = next(it)
            if add(kind, [i, j], [k]):
                break

    def oriented(p, q):
        dh_fwd = hf[q[0]] + hf[q[1]] - hf[p[0]] - hf[p[1]]
        return (list(p), list(q)) if dh_fwd <= 0 else (list(q), list(p))

    n_elem = n_reactions - len(reactions)
    # cover every species at least once, then fill at random
    by_species: Dict[int, List[int]] = {}
    for idx, (p, q) in enumerate(exch):
        for s in set(p + q):
            by_species.setdefault(s, []).append(idx)
    for s in range(ns):
        if covered[s] or n_elem == 0:
            continue
        for idx in by_species.get(s, []):
            r, p = oriented(*exch[idx])
            if add("ELEM", r, p):
                n_elem -= 1
                break
    for (pp, qq) in exch:
        if n_elem == 0:
            break
        r, p = oriented(pp, qq)
        if add("ELEM", r, p):
            n_elem -= 1
    if n_elem:
        raise ValueError("not enough distinct exchange reactions")
    # order: plain reactions first, then third-body, then falloff (stable within a kind)
    rank = {"ELEM": 0, "THIRD": 1, "LIND": 2, "TROE": 3}
    reactions.sort(key=lambda rx: rank[rx.kind])
    return Mechanism(name or "synth%d_%d" % (ns, n_reactions), seed, elements, species,
                     reactions)


# ----------------------------------------------------------------------------- spec file


def write_spec(mech: Mechanism, path: str) -> None:
    f = repr
    lines = ["# synthetic mechanism; see paper_2205_05681_gb300/synth.py for the format",
             "MECHANISM %s %d" % (mech.name, mech.seed),
             "ELEMENTS " + " ".join(mech.elements),
             "SPECIES %d" % mech.n_species]
    for s in mech.species:
        cnt = " ".join(str(s.counts.get(e, 0)) for e in mech.elements)
        lines.append("SP %s %s %s %s %s %s %s %s" % (s.name, f(s.W), cnt, f(s.Tlow), f(s.Tmid),
                                                    f(s.Thigh), f(s.hf_R), f(s.s_R)))
        lines.append("LO " + " ".join(f(float(a)) for a in s.lo))
        lines.append("HI " + " ".join(f(float(a)) for a in s.hi))
    lines.append("REACTIONS %d" % mech.n_reactions)
    names = [s.name for s in mech.species]
    for rx in mech.reactions:
        side = lambda lst: "%d %s" % (len(lst), " ".join("%s %d" % (names[k], nu) for k, nu in lst))
        lines.append("R %s %s %s %s %s %s" % (rx.kind, side(rx.reac), side(rx.prod), f(rx.A),
                                            f(rx.b), f(rx.Ea)))
        if rx.kind != "ELEM":
            effs = " ".join("%s %s" % (names[k], f(e)) for k, e in rx.eff)
            lines.append(("EFF %d %s" % (len(rx.eff), effs)).rstrip())
        if rx.low is not None:
            lines.append("LOW %s %s %s" % tuple(f(float(v)) for v in rx.low))
        if rx.troe is not None:
            lines.append("TROE %s %s %s %s" % tuple(f(float(v)) for v in rx.troe))
    lines.append("END")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


# ----------------------------------------------------------------------------- the workloads

MECHS = {
    # name: (Ns, Nr, n_third, n_falloff, n_troe, elements, seed)
    "h2_13": (13, 27, 4, 1, 1, ("H", "O", "N"), 1301),
    "ch4_53": (53, 325, 30, 25, 20, ("C", "H", "O", "N"), 5301),
    "ch4_111": (111, 784, 70, 60, 45, ("C", "H", "O", "N"), 11101),
}


def mechanism(name: str) -> Mechanism:
    ns, nr, ntb, nfo, ntr, el, seed = MECHS[name]
    return make_mechanism(ns, nr, ntb, nfo, ntr, el, seed, name=name)


def mechanism_file(name: str, directory: str) -> str:
    """Write (once) and return the spec path of a named workload mechanism."""
    import os
    os.makedirs(directory, exist_ok=True)
    path = os.path.join(directory, name + ".mech")
    if not os.path.exists(path):
        tmp = path + ".tmp%d" % os.getpid()
        write_spec(mechanism(name), tmp)
        os.replace(tmp, path)
    return path


def _mole_to_mass(mech: Mechanism, X: np.ndarray) -> np.ndarray:
    Y = X * mech.weights()
    return Y / Y.sum(axis=-1, keepdims=True)


def _fuel_air(mech: Mechanism, fuel: str, phi: float) -> np.ndarray:
    """Mole fractions of fuel + air (O2 + 3.76 N2) at equivalence ratio phi."""
    c = parse_formula(fuel)
    o2_st = c.get("C", 0) + c.get("H", 0) / 4.0 - c.get("O", 0) / 2.0
    X = np.zeros(mech.n_species)
    X[mech.index(fuel)] = 1.0
    X[mech.index("O2")] = o2_st / phi
    X[mech.index("N2")] = 3.76 * o2_st / phi
    return X / X.sum()


def _products(mech: Mechanism, fuel: str, phi: float) -> np.ndarray:
    """Mole fractions of complete-combustion products (CO/H2 split when rich)."""
    c = parse_formula(fuel)
    C_, H_ = c.get("C", 0), c.get("H", 0)
    o2_st = C_ + H_ / 4.0 - c.get("O", 0) / 2.0
    O_av = 2.0 * o2_st / phi + c.get("O", 0)
    X = np.zeros(mech.n_species)
    X[mech.index("N2")] = 3.76 * o2_st / phi
    if O_av >= 2 * C_ + H_ / 2.0:  # lean or stoichiometric
        if C_:
            X[mech.index("CO2")] = C_
        X[mech.index("H2O")] = H_ / 2.0
        X[mech.index("O2")] = (O_av - 2 * C_ - H_ / 2.0) / 2.0
    else:
        co = C_
        o_left = O_av - co
        h2o = min(H_ / 2.0, max(o_left, 0.0))
        o_left -= h2o
        co2 = min(co, max(o_left, 0.0))
        if C_:
            X[mech.index("CO")] = co - co2
            X[mech.index("CO2")] = co2
        X[mech.index("H2O")] = h2o
        X[mech.index("H2")] = H_ / 2.0 - h2o
    return X / X.sum()


def _radical_pool(mech: Mechanism, rng, n: int, lo: float, hi: float, exclude) -> np.ndarray:
    ex = {mech.index(s) for s in exclude if s in [sp.name for sp in mech.species]}
    Y = np.exp(rng.uniform(math.log(lo), math.log(hi), size=(n, mech.n_species)))
    Y[:, sorted(ex)] = 0.0
    return Y


@dataclasses.dataclass
class States:
    T: np.ndarray  # [C] K
    P: np.ndarray  # [C] Pa
    Y: np.ndarray  # [C, Ns] mass fractions (sum to 1)


def make_states(mech: Mechanism, n_cells: int, recipe: str, seed: int) -> States:
    """Seeded cell states for the named recipe.

    recipes:
      ``h2_fresh``     T~U(1000,1600) K, P~U(1,25) atm, Y = random fuel/O2/N2 with Y_N2 >= 0.5,
                       plus a log-uniform 1e-8..1e-5 radical pool, renormalised
      ``ch4_partial``  T~U(800,2200), P~U(1,50) atm, phi~U(0.5,2), Y = (1-xi)*unburnt + xi*products,
                       xi~U(0,1), plus a log-uniform 1e-8..1e-3 radical pool, renormalised
      ``ch4_front``    90% near-equilibrium products at U(1800,2400) K with a 1e-6..1e-4 radical pool,
                       10% ignition-front cells at U(1000,1300) K: (1-xi)*unburnt + xi*products,
                       xi~U(0,0.5), phi~U(0.5,1.5), with a 1e-6..1e-2 radical pool (the radical-rich
                       reaction zone; over 20 split steps of 1 us these need 10-20x the step
                       attempts of the relaxed product cells), randomly interleaved; P~U(1,50) atm
      ``ch4_ign``      fresh mixture, phi~U(0.5,2), T~U(900,1400), P~U(1,40) atm, seeded with a
                       1e-4..3e-2 radical pool (by mass, renormalised) so that the cells ignite
                       within 1e-4 s (median temperature rise ~540 K, a tenth above 1000 K)
      ``ch4_ign_wide`` fresh mixture, phi~U(0.5,2), T~U(900,1500), P~U(1,50) atm, pool 1e-8..1e-6
    """
    rng = np.random.default_rng(seed)
    C = n_cells
    ns = mech.n_species
    names = [s.name for s in mech.species]
    fuel = "H2" if "CH4" not in names else "CH4"
    main = {fuel, "O2", "N2", "H2O", "CO2", "CO", "H2"}
    if recipe == "h2_fresh":
        T = rng.uniform(1000.0, 1600.0, C)
        P = rng.uniform(1.0, 25.0, C) * ATM
        d = rng.dirichlet(np.ones(3), size=C)
        Y = np.zeros((C, ns))
        Y[:, mech.index("H2")] = 0.5 * d[:, 0]
        Y[:, mech.index("O2")] = 0.5 * d[:, 1]
        Y[:, mech.index("N2")] = 0.5 + 0.5 * d[:, 2]
        # trace radicals: a pure fuel/O2/N2 mixture has no chain carriers and would not react
        Y += _radical_pool(mech, rng, C, 1e-8, 1e-5, main)
    elif recipe in ("ch4_partial", "ch4_ign", "ch4_ign_wide"):
        if recipe == "ch4_partial":
            T = rng.uniform(800.0, 2200.0, C)
            P = rng.uniform(1.0, 50.0, C) * ATM
            xi = rng.uniform(0.0, 1.0, C)
            lo, hi = 1e-8, 1e-3
        else:
            Tmax, Pmax = (1400.0, 40.0) if recipe == "ch4_ign" else (1500.0, 50.0)
            T = rng.uniform(900.0, Tmax, C)
            P = rng.uniform(1.0, Pmax, C) * ATM
            xi = np.zeros(C)
            # ch4_ign: radical-seeded cells that ignite within 1e-4 s (a trace pool leaves these
            # mixtures in their induction period over that interval)
            lo, hi = (1e-4, 3e-2) if recipe == "ch4_ign" else (1e-8, 1e-6)
        phi = rng.uniform(0.5, 2.0, C)
        Y = np.zeros((C, ns))
        for i in range(C):
            Yu = _mole_to_mass(mech, _fuel_air(mech, fuel, phi[i]))
            Yb = _mole_to_mass(mech, _products(mech, fuel, phi[i]))
            Y[i] = (1 - xi[i]) * Yu + xi[i] * Yb
        Y += _radical_pool(mech, rng, C, lo, hi, main)
    elif recipe == "ch4_front":
        front = rng.random(C) < 0.10
        T = np.where(front, rng.uniform(1000.0, 1300.0, C), rng.uniform(1800.0, 2400.0, C))
        P = rng.uniform(1.0, 50.0, C) * ATM
        phi = np.where(front, rng.uniform(0.5, 1.5, C), rng.uniform(0.7, 1.3, C))
        xi = rng.uniform(0.0, 0.5, C)  # progress of a front cell between unburnt and burnt
        pool_b = _radical_pool(mech, rng, C, 1e-6, 1e-4, main)
        pool_f = _radical_pool(mech, rng, C, 1e-6, 1e-2, main)
        Y = np.zeros((C, ns))
        for i in range(C):
            if front[i]:
                Yu = _mole_to_mass(mech, _fuel_air(mech, fuel, phi[i]))
                Yb = _mole_to_mass(mech, _products(mech, fuel, phi[i]))
                Y[i] = (1 - xi[i]) * Yu + xi[i] * Yb + pool_f[i]
            else:
                Y[i] = _mole_to_mass(mech, _products(mech, fuel, phi[i])) + pool_b[i]
    else:
        raise ValueError(recipe)
    Y = Y / Y.sum(axis=1, keepdims=True)
    return States(T.astype(np.float64), P.astype(np.float64), Y.astype(np.float64))


# the workloads: (mechanism, cells, recipe, state seed, dt [s], split steps)
WORKLOADS = {
    "h2_13_fwd": ("h2_13", 1024, "h2_fresh", 7, 1e-6, 1),
    "ch4_53_fwd": ("ch4_53", 65536, "ch4_partial", 8, 1e-6, 1),
    "ch4_111_batched": ("ch4_111", 262144, "ch4_front", 9, 1e-6, 20),
    "ch4_53_adjoint": ("ch4_53", 16384, "ch4_ign", 10, 1e-4, 1),
    "ch4_111_adjoint": ("ch4_111", 65536, "ch4_ign_wide", 11, 5e-4, 1),
    # the 13-species cells at a batch that fills the GPU (method comparison at throughput)
    "h2_13_wide": ("h2_13", 65536, "h2_fresh", 12, 1e-6, 1),
}
