"""A mechanism file's reaction order is the user's: the library regroups reactions into its own
kernel order (by branch structure) and must map run-time ln A inputs and per-reaction outputs
back.  Here: the shuffling helper itself, on the oracle (no GPU)."""
import os

import numpy as np

from tests.conftest import shuffled_spec, states


def test_shuffled_spec_is_the_same_mechanism(mech_path, tmp_path):
    from oracle import oracle as O
    src = mech_path("ch4_53")
    dst = os.path.join(str(tmp_path), "ch4_53_shuffled.mech")
    perm = shuffled_spec(src, dst, 5)
    a, b = O.Mechanism(src), O.Mechanism(dst)
    assert a.nr == b.nr and not np.array_equal(perm, np.arange(a.nr))
    assert np.array_equal(b.lnA, a.lnA[perm])
    st = states("ch4_53", 16, "ch4_partial", 9)
    y = a.state_from_TY(st.T, st.Y)
    fa, fb = a.source(y, st.P), b.source(y, st.P)
    assert np.allclose(fa, fb, rtol=1e-12, atol=1e-12 * np.abs(fa).max())
