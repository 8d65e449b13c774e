"""chem_adjoint_noalloc: the discrete adjoint for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: code that runs inside a CUDA stream capture, applications
whose device memory belongs to a fixed pool or to another framework, or embedded solvers that may
only use the buffers handed to them.  chem_adjoint_noalloc takes its scratch (queue counter,
recomputed segment states, per-team partial gradients) from a fixed static array in the adjoint
module instead of a caller-provided workspace.

Through the C ABI, two calls in a row must return the gradients of chem_adjoint (the workspace
entry point) on the same tape, within the tolerance the adjoint tests use for results that differ
only in summation order; a checkpoint interval whose scratch cannot fit in the static array must
be refused with a clear error before anything is launched.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,recipe,dt,n,interval", [("h2_13", "h2_fresh", 1e-5, 64, 8),
                                                        ("ch4_53", "ch4_ign", 1e-6, 16, 8),
                                                        ("ch4_53", "ch4_ign", 1e-5, 64, 512)])
def test_noalloc_adjoint_matches_workspace_adjoint(mech_path, name, recipe, dt, n, interval):
    """The last case keeps 512 accepted states per team: only 38 teams' scratch fits in the
    static array, fewer than the 64 cells, so the launch is shrunk and teams refill."""
    import torch
    from tests.conftest import states
    from tests.gpu_helpers import gpu_mech, to_dev
    g = gpu_mech(mech_path(name), team=64, block=64)
    st = states(name, n, recipe, 301)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    tape = g.make_tape(n, 4096, interval)
    status = torch.full((n,), -1, dtype=torch.int32, device=T.device)
    g.integrate_ckpt(T, P, Y, dt, tape, status=status)
    assert (status.cpu().numpy() == 0).all()
    gT = 2.0 * (T - 1500.0)
    gY = torch.zeros_like(Y)
    gY[1] = 1.0
    ref = [x.cpu().numpy() for x in g.adjoint(P, gT, gY, tape)]
    for _ in range(2):  # the second call reuses the static scratch left by the first
        out = (torch.full((g.nr,), float("nan"), dtype=torch.float64, device=T.device),
               torch.full((n,), float("nan"), dtype=torch.float64, device=T.device),
               torch.full((g.ns, n), float("nan"), dtype=torch.float64, device=T.device))
        g.adjoint_noalloc(P, gT, gY, tape, *out)
        torch.cuda.synchronize()
        for a, b in zip(ref, out):
            b = b.cpu().numpy()
            assert np.all(np.isfinite(b))
            assert np.allclose(b, a, rtol=1e-9, atol=1e-12 * np.abs(a).max())


def test_noalloc_adjoint_refuses_oversized_scratch(mech_path):
    import torch
    from paper_2205_05681_gb300 import chem
    from tests.conftest import states
    from tests.gpu_helpers import gpu_mech, to_dev
    g = gpu_mech(mech_path("ch4_53"), team=64, block=64)
    n = 4
    st = states("ch4_53", n, "ch4_ign", 302)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    # one cell's segment alone (30000 states x 53 species) exceeds the 8 MiB static array
    tape = g.make_tape(n, 1, 30000)
    out = (torch.zeros(g.nr, dtype=torch.float64, device=T.device),
           torch.zeros(n, dtype=torch.float64, device=T.device),
           torch.zeros((g.ns, n), dtype=torch.float64, device=T.device))
    with pytest.raises(chem.ChemError, match="static scratch"):
        g.adjoint_noalloc(P, torch.ones_like(T), torch.zeros_like(Y), tape, *out)
