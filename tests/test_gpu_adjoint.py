"""Parity of the discrete adjoint (CUDA, through the C ABI) with the CPU oracle.

The adjoint differentiates the discrete ROS4 map with the accepted step sizes frozen.  The
oracle computes the same derivative independently by complex-step differentiation of its own
integrator replaying the GPU's accepted step sizes (exact to roundoff, no subtractive
cancellation).  Tolerance (stated): |g - g_oracle| <= 1e-6 (|g_oracle| + 1e-3 max|g_oracle|)
per component, and for directional derivatives <= 1e-6 relative to the scale of the gradient.
"""
import numpy as np
import pytest

from tests.conftest import states
from tests.gpu_helpers import gpu_mech, gpu_state, to_dev

pytestmark = pytest.mark.gpu

WORK = {"h2_13": "h2_fresh", "ch4_53": "ch4_ign"}


@pytest.fixture(scope="module")
def gm(mech_path):
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = gpu_mech(mech_path(name), team=64, block=64)
        return cache[name]

    return get


@pytest.mark.parametrize("name", ["h2_13", "ch4_53"])
def test_vjp_parity(omech, gm, name):
    om, g = omech(name), gm(name)
    st = states(name, 24, "h2_fresh" if name == "h2_13" else "ch4_partial", 201)
    y = om.state_from_TY(st.T, st.Y)
    rng = np.random.default_rng(1)
    v = rng.normal(size=y.shape) / np.maximum(np.abs(om.source(y, st.P)), 1e-30)
    gy, gp = g.eval_vjp(to_dev(y[:, 0]), to_dev(st.P), to_dev(y[:, 1:].T), to_dev(v.T))
    gy, gp = gy.cpu().numpy().T, gp.cpu().numpy().T
    J = om.jacobian(y, st.P, threads=16)
    for c in range(len(y)):
        ref = J[c].T @ v[c]
        scale = np.abs(J[c]).T @ np.abs(v[c])
        assert np.all(np.abs(gy[c] - ref) <= 1e-11 * (np.abs(ref) + scale)), c
    # parameter part against complex step of v^T f in each ln A direction (first 6 cells)
    for c in range(6):
        ref = np.zeros(om.nr)
        for r in range(om.nr):
            d = np.zeros(om.nr, dtype=complex)
            d[r] = 1e-30j
            ref[r] = (v[c] @ om.source_cplx(y[c], st.P[c], lnA=om.lnA + d).imag) / 1e-30
        scale = np.abs(ref).max()
        assert np.all(np.abs(gp[c] - ref) <= 1e-11 * (np.abs(ref) + 1e-3 * scale)), c


def _forward_with_tape(g, st, dt, interval, cap=4096):
    import torch
    n = len(st.T)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    tape = g.make_tape(n, cap, interval)
    status = torch.full((n,), -1, dtype=torch.int32, device=T.device)
    g.integrate_ckpt(T, P, Y, dt, tape, status=status)
    assert (status.cpu().numpy() == 0).all()
    return T, P, Y, tape


@pytest.mark.parametrize("name,dt,n", [("h2_13", 1e-5, 6), ("ch4_53", 1e-6, 3)])
def test_adjoint_gradient_vs_complex_step(omech, gm, name, dt, n):
    import torch
    om, g = omech(name), gm(name)
    st = states(name, n, WORK[name], 202)
    T, P, Y, tape = _forward_with_tape(g, st, dt, interval=4)
    nacc = tape.n_accepted().cpu().numpy()
    hs_all = tape.step_sizes().cpu().numpy()
    rng = np.random.default_rng(2)
    Ttarget = T.cpu().numpy() + rng.normal(0.0, 5.0, n)
    # loss L = sum_c (T_c - T_target,c)^2
    gT = 2.0 * (T - torch.tensor(Ttarget, device=T.device))
    gY = torch.zeros_like(Y)
    g_lnA, gT0, gY0 = g.adjoint(P, gT, gY, tape)
    g_lnA = g_lnA.cpu().numpy()
    gy0 = np.zeros((n, om.N))
    gy0[:, 0] = gT0.cpu().numpy()
    gy0[:, 1:] = gY0.cpu().numpy().T[:, :-1] * om.W[:-1]
    y0 = om.state_from_TY(st.T, st.Y)

    def loss_dir(dy, dl):
        tot = 0.0
        for c in range(n):
            hs = hs_all[: nacc[c], c]
            yT = om.replay_cplx(y0[c] + 1e-30j * dy[c], st.P[c], hs, lnA=om.lnA + 1e-30j * dl)
            Tv = yT[0]
            tot += ((Tv - Ttarget[c]) ** 2).imag / 1e-30
        return tot

    # directional derivatives along random directions in (y0, lnA)
    for k in range(3):
        dy = rng.normal(size=(n, om.N)) * np.maximum(np.abs(y0), 1e-12)
        dl = rng.normal(size=om.nr)
        ref = loss_dir(dy, dl)
        got = (gy0 * dy).sum() + g_lnA @ dl
        scale = (np.abs(gy0 * dy).sum() + np.abs(g_lnA * dl).sum())
        assert abs(got - ref) <= 1e-6 * scale, (k, got, ref, scale)
    # per-component ln A gradient (all reactions for the small mechanism, a sample otherwise)
    rs = range(om.nr) if om.nr <= 30 else rng.choice(om.nr, 12, replace=False)
    ref = {}
    for r in rs:
        dl = np.zeros(om.nr)
        dl[r] = 1.0
        ref[r] = loss_dir(np.zeros((n, om.N)), dl)
    mx = max(abs(v) for v in ref.values())
    for r in rs:
        assert abs(g_lnA[r] - ref[r]) <= 1e-6 * (abs(ref[r]) + 1e-3 * mx), (r, g_lnA[r], ref[r])


def test_checkpoint_interval_does_not_change_gradient(omech, gm):
    import torch
    name = "h2_13"
    om, g = omech(name), gm(name)
    st = states(name, 32, WORK[name], 203)
    outs = []
    for interval in (1, 3, 16):
        T, P, Y, tape = _forward_with_tape(g, st, 1e-5, interval)
        gT = torch.ones_like(T)
        gY = torch.zeros_like(Y)
        gY[3] = 1.0
        outs.append([x.cpu().numpy() for x in g.adjoint(P, gT, gY, tape)])
    for a, b in zip(outs[0], outs[1]):
        assert np.allclose(a, b, rtol=1e-9, atol=1e-12 * np.abs(a).max())
    for a, b in zip(outs[0], outs[2]):
        assert np.allclose(a, b, rtol=1e-9, atol=1e-12 * np.abs(a).max())


def test_autograd_function(omech, gm):
    import torch
    from paper_2205_05681_gb300 import chem
    name = "h2_13"
    om, g = omech(name), gm(name)
    st = states(name, 16, WORK[name], 204)
    T0 = to_dev(st.T).requires_grad_(True)
    Y0 = to_dev(st.Y.T).requires_grad_(True)
    lnA = to_dev(g.lnA()).requires_grad_(True)
    P = to_dev(st.P)
    F = chem.chem_integrate_fn()
    T, Y = F.apply(T0, Y0, lnA, g, P, 1e-5, 1e-6, 1e-10, 4096, 8)
    loss = ((T - 1500.0) ** 2).sum() + Y[2].sum()
    loss.backward()
    # same numbers as the explicit C-ABI adjoint
    T2, P2, Y2, tape = _forward_with_tape(g, st, 1e-5, 8)
    gT = 2.0 * (T2 - 1500.0)
    gY = torch.zeros_like(Y2)
    gY[2] = 1.0
    g_lnA, gT0, gY0 = g.adjoint(P2, gT, gY, tape)
    assert torch.allclose(lnA.grad, g_lnA, rtol=1e-9, atol=1e-12 * g_lnA.abs().max().item())
    assert torch.allclose(T0.grad, gT0, rtol=1e-9)
    assert torch.allclose(Y0.grad, gY0, rtol=1e-9, atol=1e-12 * gY0.abs().max().item())


def test_tape_full_stops_at_the_recorded_map(omech, gm):
    """A full tape stops the cell before any unrecorded step: the returned state is the oracle's
    replay of exactly the recorded step sizes, and autograd refuses to differentiate it."""
    import torch
    from paper_2205_05681_gb300 import chem
    name = "h2_13"
    om, g = omech(name), gm(name)
    n = 8
    st = states(name, n, "h2_fresh", 205)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    tape = g.make_tape(n, 2, 1)
    status = torch.full((n,), -1, dtype=torch.int32, device=T.device)
    g.integrate_ckpt(T, P, Y, 1e-4, tape, status=status)
    s = status.cpu().numpy()
    nacc = tape.n_accepted().cpu().numpy()
    hs = tape.step_sizes().cpu().numpy()
    assert (s == chem.STATUS_TAPE_FULL).all() and (nacc == 2).all()
    y0 = om.state_from_TY(st.T, st.Y)
    yg = gpu_state(om, T, Y)
    for c in range(n):
        yr = om.replay(y0[c], st.P[c], hs[:2, c])
        w = 1e-10 + 1e-6 * np.abs(yr)
        assert np.sqrt(np.mean(((yg[c] - yr) / w) ** 2)) <= 1e-5, c
    F = chem.chem_integrate_fn()
    T0 = to_dev(st.T).requires_grad_(True)
    Tf, Yf = F.apply(T0, to_dev(st.Y.T), to_dev(g.lnA()), g, P, 1e-4, 1e-6, 1e-10, 2, 1)
    with pytest.raises(chem.ChemError, match="did not reach"):
        Tf.sum().backward()


def _pool(fn, jobs, workers=16):
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, jobs))


def test_adjoint_through_ignition_queue_refill(omech, gm):
    """The adjoint workload's regime: 53 species through ignition over 1e-4 s, checkpoints every 16
    accepted steps (several segments per cell), more cells than adjoint teams so that the reverse
    queue refills.  Per cell, every component of dL/dy0 of a seeded sample of cells against the
    oracle's complex-step replay of the same accepted step sizes; dL/dlnA (a second sweep with the
    loss on the sampled cells only) per reaction for a sample of reactions, and along random
    directions against central differences of the oracle's replay (relative step 1e-6)."""
    import torch
    name = "ch4_53"
    om, g = omech(name), gm(name)
    n, dt = 2432, 1e-4
    st = states(name, n, "ch4_ign", 10)
    T, P, Y, tape = _forward_with_tape(g, st, dt, interval=16)
    nacc = tape.n_accepted().cpu().numpy()
    hs_all = tape.step_sizes().cpu().numpy()
    assert nacc.max() > 2 * 16  # several checkpoint segments per cell
    rng = np.random.default_rng(7)
    Tf = T.cpu().numpy()
    Ttarget = Tf + rng.normal(0.0, 5.0, n)
    gT = 2.0 * (T - torch.tensor(Ttarget, device=T.device))
    gY = torch.zeros_like(Y)
    _, gT0, gY0 = g.adjoint(P, gT, gY, tape)
    gT0, gY0 = gT0.cpu().numpy(), gY0.cpu().numpy()
    y0 = om.state_from_TY(st.T, st.Y)
    idx = np.sort(rng.choice(n, 10, replace=False))

    def cell_grad_component(job):
        c, i = job
        hs = hs_all[: nacc[c], c]
        d = np.zeros(om.N, dtype=complex)
        d[i] = 1e-30j * max(abs(y0[c, i]), 1e-12)
        yT = om.replay_cplx(y0[c] + d, st.P[c], hs)
        return ((yT[0] - Ttarget[c]) ** 2).imag / 1e-30 / max(abs(y0[c, i]), 1e-12)

    jobs = [(c, i) for c in idx for i in range(om.N)]
    ref = np.array(_pool(cell_grad_component, jobs)).reshape(len(idx), om.N)
    got = np.zeros((len(idx), om.N))
    got[:, 0] = gT0[idx]
    got[:, 1:] = gY0[:-1, idx].T * om.W[:-1]
    for j, c in enumerate(idx):
        mx = np.abs(ref[j]).max()
        assert np.all(np.abs(got[j] - ref[j]) <= 1e-6 * (np.abs(ref[j]) + 1e-3 * mx)), (c, j)
    # dL/dlnA of the loss restricted to the sampled cells (every other cell seeds zero)
    mask = torch.zeros(n, dtype=torch.float64, device=T.device)
    mask[torch.tensor(idx, device=T.device)] = 1.0
    g_lnA, _, _ = g.adjoint(P, gT * mask, gY, tape)
    g_lnA = g_lnA.cpu().numpy()

    def lnA_component(job):
        c, r = job
        dl = np.zeros(om.nr, dtype=complex)
        dl[r] = 1e-30j
        yT = om.replay_cplx(y0[c], st.P[c], hs_all[: nacc[c], c], lnA=om.lnA + dl)
        return ((yT[0] - Ttarget[c]) ** 2).imag / 1e-30

    rs = np.sort(rng.choice(om.nr, 16, replace=False))
    vals = np.array(_pool(lnA_component, [(c, r) for r in rs for c in idx])).reshape(len(rs), -1)
    ref_l = vals.sum(axis=1)
    mx = np.abs(ref_l).max()
    assert np.all(np.abs(g_lnA[rs] - ref_l) <= 1e-6 * (np.abs(ref_l) + 1e-3 * mx)), \
        (g_lnA[rs], ref_l)

    # central differences of the oracle's replay along random directions in (y0, lnA)
    def loss(eps, dy, dl):
        tot = 0.0
        for j, c in enumerate(idx):
            yT = om.replay(y0[c] + eps * dy[j], st.P[c], hs_all[: nacc[c], c], lnA=om.lnA + eps * dl)
            tot += (yT[0] - Ttarget[c]) ** 2
        return tot

    for k in range(2):
        dy = rng.normal(size=(len(idx), om.N)) * np.maximum(np.abs(y0[idx]), 1e-12)
        dl = rng.normal(size=om.nr) * np.abs(om.lnA)
        eps = 1e-6
        fd = (loss(eps, dy, dl) - loss(-eps, dy, dl)) / (2 * eps)
        gy = np.zeros((len(idx), om.N))
        gy[:, 0] = gT0[idx]
        gy[:, 1:] = gY0[:-1, idx].T * om.W[:-1]
        an = (gy * dy).sum() + g_lnA @ dl
        assert abs(an - fd) <= 1e-6 * (abs(fd) + np.abs(gy * dy).sum() * 1e-3), (k, an, fd)


def test_adjoint_111_species(omech, mech_path):
    """The 111-species mechanism in its default (256-lane) configuration: directional derivatives
    and a sample of components of dL/dy0 and dL/dlnA against the oracle's complex-step replay."""
    import torch
    name = "ch4_111"
    om = omech(name)
    g = gpu_mech(mech_path(name))
    n, dt = 3, 2e-5
    st = states(name, n, "ch4_ign_wide", 206)
    T, P, Y, tape = _forward_with_tape(g, st, dt, interval=4)
    nacc = tape.n_accepted().cpu().numpy()
    hs_all = tape.step_sizes().cpu().numpy()
    rng = np.random.default_rng(8)
    Ttarget = T.cpu().numpy() + rng.normal(0.0, 5.0, n)
    gT = 2.0 * (T - torch.tensor(Ttarget, device=T.device))
    g_lnA, gT0, gY0 = g.adjoint(P, gT, torch.zeros_like(Y), tape)
    g_lnA, gT0, gY0 = g_lnA.cpu().numpy(), gT0.cpu().numpy(), gY0.cpu().numpy()
    y0 = om.state_from_TY(st.T, st.Y)
    gy = np.zeros((n, om.N))
    gy[:, 0] = gT0
    gy[:, 1:] = gY0[:-1].T * om.W[:-1]

    def loss_dir(job):
        c, dy, dl = job
        yT = om.replay_cplx(y0[c] + 1e-30j * dy, st.P[c], hs_all[: nacc[c], c],
                            lnA=om.lnA + 1e-30j * dl)
        return ((yT[0] - Ttarget[c]) ** 2).imag / 1e-30

    # sampled components: 8 state entries per cell, 10 reactions (summed over the cells)
    comps = rng.choice(om.N, 8, replace=False)
    jobs = []
    for c in range(n):
        for i in comps:
            dy = np.zeros(om.N)
            dy[i] = 1.0
            jobs.append((c, dy, np.zeros(om.nr)))
    rs = rng.choice(om.nr, 10, replace=False)
    for r in rs:
        for c in range(n):
            dl = np.zeros(om.nr)
            dl[r] = 1.0
            jobs.append((c, np.zeros(om.N), dl))
    dirs = []
    for k in range(2):
        dy = rng.normal(size=(n, om.N)) * np.maximum(np.abs(y0), 1e-12)
        dl = rng.normal(size=om.nr)
        dirs.append((dy, dl))
        for c in range(n):
            jobs.append((c, dy[c], dl))
    vals = np.array(_pool(loss_dir, jobs))
    k = 0
    for c in range(n):
        ref = vals[k:k + len(comps)]
        k += len(comps)
        mx = np.abs(ref).max()
        assert np.all(np.abs(gy[c, comps] - ref) <= 1e-6 * (np.abs(ref) + 1e-3 * mx)), c
    ref_l = vals[k:k + len(rs) * n].reshape(len(rs), n).sum(axis=1)
    k += len(rs) * n
    mx = max(np.abs(ref_l).max(), 1e-300)
    assert np.all(np.abs(g_lnA[rs] - ref_l) <= 1e-6 * (np.abs(ref_l) + 1e-3 * mx)), (g_lnA[rs], ref_l)
    for dy, dl in dirs:
        ref = vals[k:k + n].sum()
        k += n
        got = (gy * dy).sum() + g_lnA @ dl
        scale = np.abs(gy * dy).sum() + np.abs(g_lnA * dl).sum()
        assert abs(got - ref) <= 1e-6 * scale, (got, ref, scale)
