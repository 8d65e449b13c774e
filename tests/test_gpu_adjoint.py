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


def test_tape_full_status(gm):
    import torch
    from paper_2205_05681_gb300 import chem
    g = gm("h2_13")
    st = states("h2_13", 8, "h2_fresh", 205)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    tape = g.make_tape(8, 2, 1)
    status = torch.full((8,), -1, dtype=torch.int32, device=T.device)
    g.integrate_ckpt(T, P, Y, 1e-4, tape, status=status)
    s = status.cpu().numpy()
    assert (s == chem.STATUS_TAPE_FULL).all() or ((s == 0) | (s == chem.STATUS_TAPE_FULL)).all()
    assert (tape.n_accepted().cpu().numpy() <= 2).all()
