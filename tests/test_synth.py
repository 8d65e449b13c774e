"""The seeded input generator: mechanisms have the stated sizes and kinds, every reaction is
element- and mass-balanced, the bath gas is last, states are valid mass fractions in the recipe
ranges, and the same seed gives the same inputs (the GPU and the oracle read the same cells)."""
import numpy as np
import pytest

from paper_2205_05681_gb300 import synth


@pytest.mark.parametrize("name", sorted(synth.MECHS))
def test_mechanism_sizes_kinds_and_balance(name):
    ns, nr, n_third, n_fall, n_troe, elements, _ = synth.MECHS[name]
    m = synth.mechanism(name)
    assert m.n_species == ns and m.n_reactions == nr
    kinds = [r.kind for r in m.reactions]
    assert kinds.count("TROE") == n_troe
    assert kinds.count("LIND") + kinds.count("TROE") == n_fall
    assert kinds.count("THIRD") == n_third
    assert m.species[-1].name == "N2"
    E = m.element_matrix()  # [element][species]
    W = m.weights()
    for r in m.reactions:
        net = np.zeros(m.n_species)
        for k, v in r.reac:
            net[k] -= v
        for k, v in r.prod:
            net[k] += v
        assert np.all(E @ net == 0), r
        assert abs(W @ net) < 1e-9 * W.max()
    covered = {k for r in m.reactions for k, _ in r.reac + r.prod}
    assert len(covered) >= m.n_species - 1  # every species but possibly the bath gas reacts


@pytest.mark.parametrize("name,recipe,Trange,Prange", [
    ("h2_13", "h2_fresh", (1000.0, 1600.0), (1.0, 25.0)),
    ("ch4_53", "ch4_partial", (800.0, 2200.0), (1.0, 50.0)),
    ("ch4_53", "ch4_ign", (900.0, 1400.0), (1.0, 40.0)),
])
def test_states_are_valid_and_seeded(name, recipe, Trange, Prange):
    m = synth.mechanism(name)
    st = synth.make_states(m, 500, recipe, 21)
    assert st.Y.shape == (500, m.n_species)
    assert np.all(st.Y >= 0.0) and np.allclose(st.Y.sum(1), 1.0, rtol=0, atol=1e-13)
    assert np.all((st.T >= Trange[0]) & (st.T <= Trange[1]))
    P = st.P / synth.ATM
    assert np.all((P >= Prange[0]) & (P <= Prange[1]))
    again = synth.make_states(m, 500, recipe, 21)
    assert np.array_equal(again.T, st.T) and np.array_equal(again.Y, st.Y)
    other = synth.make_states(m, 500, recipe, 22)
    assert not np.array_equal(other.T, st.T)


def test_spec_file_round_trip_is_deterministic(tmp_path):
    a = synth.mechanism_file("ch4_53", str(tmp_path / "a"))
    b = synth.mechanism_file("ch4_53", str(tmp_path / "b"))
    assert open(a).read() == open(b).read()
