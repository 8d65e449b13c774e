"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same seeded inputs.

Tolerances (stated, from the problem statement's bounds):
  * source terms and Jacobian: |x - x_oracle| <= 1e-12 (|x_oracle| + g), where g is the gross
    magnitude of the row (sum of |forward| + |reverse| contributions for f; the largest entry of
    the row for J), because near equilibrium net rates cancel;
  * integrated states: the weighted RMS norm of Eq. (e:ivp_norm), with the solver's rtol=1e-6
    and atol=1e-10 as weights, <= 1e-5 per cell, for cells whose accepted/rejected step
    sequence matches the oracle's (identical attempt counts); cells where round-off flipped an
    accept/reject decision (allowed in at most 2% of cells) must lie within 10 tolerance units
    of a tight (rtol 1e-10) oracle solution, i.e. be as valid a rtol=1e-6 solution as the
    oracle's own.
"""
import numpy as np
import pytest

from tests.conftest import shuffled_spec, states
from tests.gpu_helpers import gpu_mech, gpu_state, gross_f, to_dev, weighted_norm

pytestmark = pytest.mark.gpu

WORK = {"h2_13": "h2_fresh", "ch4_53": "ch4_partial", "ch4_111": "ch4_front"}
CONFIGS = {
    "h2_13": [(1, 32), (4, 64), (8, 128), (16, 128), (32, 64), (32, 128), (64, 64), (128, 128)],
    "ch4_53": [(16, 64), (32, 32), (32, 64), (64, 64), (128, 128), (256, 256)],
    "ch4_111": [(32, 32), (128, 128), (256, 256)],
}
PARAMS = [(n, t, b) for n in CONFIGS for (t, b) in CONFIGS[n]]


@pytest.fixture(scope="module")
def gmech(mech_path):
    cache = {}

    def get(name, team, block):
        key = (name, team, block)
        if key not in cache:
            cache[key] = gpu_mech(mech_path(name), team=team, block=block)
        return cache[key]

    return get


def _inputs(om, name, n, seed):
    st = states(name, n, WORK[name], seed)
    y = om.state_from_TY(st.T, st.Y)
    return st, y


@pytest.mark.parametrize("name,team,block", PARAMS)
def test_eval_source_parity(omech, gmech, name, team, block):
    om = omech(name)
    g = gmech(name, team, block)
    n = {"h2_13": 1000, "ch4_53": 300, "ch4_111": 100}[name]
    st, y = _inputs(om, name, n, 101)
    f = g.eval_source(to_dev(y[:, 0]), to_dev(st.P), to_dev(y[:, 1:].T)).cpu().numpy().T
    fo = om.source(y, st.P)
    for c in range(n):
        gr = gross_f(om, y[c], st.P[c])
        err = np.abs(f[c] - fo[c]) / (np.abs(fo[c]) + gr + 1e-300)
        assert err.max() <= 1e-12, (c, err.max(), np.argmax(err))


@pytest.mark.parametrize("name,team,block", PARAMS)
def test_eval_jacobian_parity(omech, gmech, name, team, block):
    om = omech(name)
    g = gmech(name, team, block)
    n = {"h2_13": 200, "ch4_53": 40, "ch4_111": 12}[name]
    st, y = _inputs(om, name, n, 102)
    J = g.eval_jacobian(to_dev(y[:, 0]), to_dev(st.P), to_dev(y[:, 1:].T)).cpu().numpy().T
    J = J.reshape(n, om.N, om.N)
    Jo = om.jacobian(y, st.P, threads=16)
    for c in range(n):
        rowmax = np.abs(Jo[c]).max(axis=1, keepdims=True)
        err = np.abs(J[c] - Jo[c]) / (np.abs(Jo[c]) + rowmax + 1e-300)
        assert err.max() <= 1e-12, (c, err.max(), np.unravel_index(np.argmax(err), err.shape))


def _check_integration(om, st, y0, yg, info_att, dt, label):
    yo, info = om.integrate(y0, st.P, dt, threads=16)
    assert np.all(info["status"] == 0)
    same = info["attempts"] == info_att
    e = weighted_norm(yo, yg)
    assert np.all(e[same] <= 1e-5), (label, e[same].max(), np.argmax(np.where(same, e, 0)))
    flips = np.where(~same)[0]
    assert len(flips) <= max(1, int(0.02 * len(same))), (label, len(flips))
    if len(flips):
        yt, it = om.integrate(y0[flips], st.P[flips], dt, rtol=1e-10, atol=1e-14, threads=16)
        assert np.all(weighted_norm(yt, yg[flips]) <= 10.0), label
    return e, len(flips)


@pytest.mark.parametrize("name,team,block", PARAMS)
def test_integrate_parity(omech, gmech, name, team, block):
    import torch
    om = omech(name)
    g = gmech(name, team, block)
    n = {"h2_13": 777, "ch4_53": 150, "ch4_111": 40}[name]
    st, y0 = _inputs(om, name, n, 103)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    status = torch.full((n,), -1, dtype=torch.int32, device=T.device)
    att = torch.zeros(n, dtype=torch.int32, device=T.device)
    h = torch.zeros(n, dtype=torch.float64, device=T.device)
    g.integrate(T, P, Y, 1e-6, h=h, status=status, opts=g.opts(attempts=att))
    assert (status.cpu().numpy() == 0).all()
    yg = gpu_state(om, T, Y)
    _check_integration(om, st, y0, yg, att.cpu().numpy(), 1e-6, (name, team, block))
    # mass closure written back: sum Y = 1
    assert np.abs(Y.sum(0).cpu().numpy() - 1.0).max() < 1e-13
    assert (h.cpu().numpy() > 0).all()


@pytest.mark.parametrize("name", ["h2_13", "ch4_53"])
def test_plain_driver_matches_persistent(omech, gmech, name):
    """The one-launch-per-attempt driver runs the same per-cell arithmetic: equal results up to
    the summation order of the shared-memory reductions of multi-lane teams."""
    import torch
    from paper_2205_05681_gb300 import chem
    om = omech(name)
    team, block = {"h2_13": (8, 128), "ch4_53": (32, 64)}[name]
    g = gmech(name, team, block)
    n = 300
    st, y0 = _inputs(om, name, n, 104)
    outs = []
    for mode in (chem.MODE_PERSISTENT, chem.MODE_PLAIN):
        T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
        h = torch.zeros(n, dtype=torch.float64, device=T.device)
        st_ = torch.full((n,), -1, dtype=torch.int32, device=T.device)
        att = torch.zeros(n, dtype=torch.int32, device=T.device)
        o = g.opts(mode=mode, attempts=att)
        g.integrate(T, P, Y, 1e-6, h=h, status=st_, opts=o)
        outs.append([x.cpu().numpy() for x in (T, Y, h, st_, att)])
    (T1, Y1, h1, s1, a1), (T2, Y2, h2, s2, a2) = outs
    assert np.array_equal(s1, s2)
    same = a1 == a2
    assert same.mean() >= 0.99
    assert np.allclose(T1[same], T2[same], rtol=1e-10, atol=0)
    assert np.allclose(Y1[:, same], Y2[:, same], rtol=1e-8, atol=1e-16)
    assert np.allclose(h1[same], h2[same], rtol=1e-6)


def _bench_config_mech(mech_path, name):
    """The mechanism as bench.py loads it: no kernel override, so the launch configuration is the
    library's default for this mechanism size (chem_kernel_config reports it)."""
    return gpu_mech(mech_path(name))


def _sampled_parity(om, st, g, n, n_sample, seed, label):
    """Integrate all n cells in one call (default launch configuration) and compare a seeded
    sample of cells, plus the last cell (ragged tail of the work queue), with the oracle."""
    import torch
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    att = torch.zeros(n, dtype=torch.int32, device=T.device)
    status = torch.full((n,), -1, dtype=torch.int32, device=T.device)
    g.integrate(T, P, Y, 1e-6, status=status, opts=g.opts(attempts=att))
    assert (status.cpu().numpy() == 0).all()
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(n - 1, n_sample - 1, replace=False))
    idx = np.append(idx, n - 1)
    yg = gpu_state(om, T, Y)[idx]
    y0 = om.state_from_TY(st.T[idx], st.Y[idx])

    class Sub:
        P = st.P[idx]

    _check_integration(om, Sub, y0, yg, att.cpu().numpy()[idx], 1e-6, label)
    return att.cpu().numpy()


def _resident_teams(g):
    """Teams of the persistent launch: SMs x resident blocks x teams per block."""
    import torch
    cfg = g.kernel_config()
    per_block = cfg["block"] if cfg["team"] == 1 else max(1, cfg["block"] // cfg["team"])
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return cfg, sms, per_block


def test_full_size_sampled_53(omech, mech_path):
    """65,536 cells of the 53-species workload in the launch configuration the bench times (the
    library default, two warps per cell), so every team pulls many cells from the queue; a
    sample of cells against the oracle one by one."""
    name = "ch4_53"
    om = omech(name)
    g = _bench_config_mech(mech_path, name)
    cfg = g.kernel_config()
    assert (cfg["team"], cfg["block"]) == (64, 64)
    n = 65536
    st = states(name, n, WORK[name], 8)
    _sampled_parity(om, st, g, n, 48, 0, "full53")


def test_full_size_sampled_111_refill(omech, mech_path):
    """The 111-species default (256 lanes per cell, register-resident stage solves) on at least
    three cells per resident team, so that every team refills from the queue at least twice."""
    name = "ch4_111"
    om = omech(name)
    g = _bench_config_mech(mech_path, name)
    cfg, sms, per_block = _resident_teams(g)
    assert (cfg["team"], cfg["block"]) == (256, 256)
    n = 3 * sms * 2 * per_block + 17  # two resident blocks per SM, plus a ragged tail
    st = states(name, n, "ch4_partial", 21)
    _sampled_parity(om, st, g, n, 40, 1, "refill111")


def test_full_size_sampled_13_wide(omech, mech_path):
    """The 13-species cells at the 65,536-cell batch (h2_13_wide) in the default configuration."""
    name = "h2_13"
    om = omech(name)
    g = _bench_config_mech(mech_path, name)
    n = 65536
    st = states(name, n, "h2_fresh", 12)
    _sampled_parity(om, st, g, n, 64, 2, "wide13")


def test_edge_cases(omech, gmech):
    import torch
    from paper_2205_05681_gb300 import chem
    name = "h2_13"
    om = omech(name)
    g = gmech(name, 32, 64)
    dev = torch.device("cuda:0")
    # empty batch: a no-op
    e = torch.zeros(0, dtype=torch.float64, device=dev)
    g.integrate(e, e, torch.zeros((om.ns, 0), dtype=torch.float64, device=dev), 1e-6)
    st, y0 = _inputs(om, name, 5, 105)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    T[1] = float("nan")
    T[2] = 200.0  # below T_min
    T0, Y0 = T.clone(), Y.clone()
    status = torch.full((5,), -1, dtype=torch.int32, device=dev)
    att = torch.full((5,), -1, dtype=torch.int32, device=dev)
    g.integrate(T, P, Y, 1e-6, status=status, opts=g.opts(T_min=300.0, attempts=att))
    s = status.cpu().numpy()
    assert s[1] == chem.STATUS_NONFINITE and s[2] == chem.STATUS_SKIPPED
    assert s[0] == 0 and s[3] == 0 and s[4] == 0
    assert att.cpu().numpy()[1] == 0 and att.cpu().numpy()[2] == 0
    assert torch.equal(Y[:, 2], Y0[:, 2]) and T[2].item() == 200.0
    # max_steps and h_min failures are reported per cell
    T, Y = to_dev(st.T), to_dev(st.Y.T)
    status.fill_(-1)
    g.integrate(T, P, Y, 1e-3, status=status, opts=g.opts(max_steps=2, attempts=att))
    assert (status.cpu().numpy() == chem.STATUS_MAX_STEPS).all()
    assert (att.cpu().numpy() == 2).all()
    T, Y = to_dev(st.T), to_dev(st.Y.T)
    g.integrate(T, P, Y, 1e-6, status=status, opts=g.opts(h_min=1.0))
    assert (status.cpu().numpy() == chem.STATUS_H_UNDERFLOW).all()
    # a single cell, and bad arguments raise instead of launching
    st1, y1 = _inputs(om, name, 1, 106)
    T, P, Y = to_dev(st1.T), to_dev(st1.P), to_dev(st1.Y.T)
    g.integrate(T, P, Y, 1e-6)
    yo, _ = om.integrate(y1, st1.P, 1e-6)
    assert weighted_norm(yo, gpu_state(om, T, Y)).max() <= 1e-5
    with pytest.raises(chem.ChemError):
        g.integrate(T, P, Y, -1.0)
    with pytest.raises(chem.ChemError):
        g.integrate(T, P, Y, 1e-6, workspace=torch.zeros(8, dtype=torch.uint8, device=dev))


def test_lnA_override(omech, gmech):
    """The ln A parameters passed at run time replace the built-in ones in f and in the step."""
    name = "h2_13"
    om = omech(name)
    g = gmech(name, 32, 64)
    rng = np.random.default_rng(7)
    lnA = om.lnA + rng.normal(0.0, 0.3, om.nr)
    st, y = _inputs(om, name, 64, 107)
    f = g.eval_source(to_dev(y[:, 0]), to_dev(st.P), to_dev(y[:, 1:].T), lnA=to_dev(lnA))
    fo = om.source(y, st.P, lnA=lnA)
    assert np.allclose(f.cpu().numpy().T, fo, rtol=1e-11, atol=1e-11 * np.abs(fo).max())
    assert np.array_equal(g.lnA(), om.lnA) or np.allclose(g.lnA(), om.lnA, rtol=1e-15, atol=0)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    g.integrate(T, P, Y, 1e-6, opts=g.opts(lnA=to_dev(lnA)))
    yo, _ = om.integrate(y, st.P, 1e-6, lnA=lnA)
    assert weighted_norm(yo, gpu_state(om, T, Y)).max() <= 1e-5


def test_host_entry_point(omech, gmech):
    """chem_integrate_host: host arrays in, host arrays out."""
    name = "ch4_53"
    om = omech(name)
    g = gmech(name, 32, 64)
    st, y0 = _inputs(om, name, 64, 108)
    T = st.T.copy()
    Y = np.ascontiguousarray(st.Y.T)
    h = np.zeros(64)
    status = np.full(64, -1, dtype=np.int32)
    g.integrate_host(T, np.ascontiguousarray(st.P), Y, 1e-6, h=h, status=status)
    assert (status == 0).all() and (h > 0).all()
    yo, _ = om.integrate(y0, st.P, 1e-6, threads=16)
    assert weighted_norm(yo, om.state_from_TY(T, Y.T)).max() <= 1e-5


def test_h_carries_across_split_steps(omech, gmech):
    """h_out of one call is the first step of the next (BatchedChemistryModel reuse)."""
    import torch
    name = "h2_13"
    om = omech(name)
    g = gmech(name, 32, 64)
    st, y0 = _inputs(om, name, 128, 109)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    h = torch.zeros(128, dtype=torch.float64, device=T.device)
    y = y0.copy()
    hh = np.zeros(128)
    for _ in range(3):
        g.integrate(T, P, Y, 1e-6, h=h)
        y, info = om.integrate(y, st.P, 1e-6, h=hh)
        hh = info["h"]
    assert weighted_norm(y, gpu_state(om, T, Y)).max() <= 1e-5
    assert np.allclose(h.cpu().numpy(), hh, rtol=1e-6)


def test_autotune_picks_a_valid_config(omech, mech_path):
    """chem_autotune times the candidate configurations on a sample and sets the fastest; the
    integration that follows still matches the oracle."""
    from tests.gpu_helpers import gpu_mech
    name = "h2_13"
    om = omech(name)
    g = gpu_mech(mech_path(name))
    st, y0 = _inputs(om, name, 512, 110)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    pick = g.autotune(T, P, Y, 1e-6)
    assert (pick["team"], pick["block"]) in [(1, 32), (4, 64), (8, 64), (8, 128), (16, 64),
                                             (16, 128), (32, 32), (32, 64), (64, 64), (128, 128),
                                             (256, 256)]
    assert pick["sample_ms"] > 0
    cfg = g.kernel_config()
    assert (cfg["team"], cfg["block"]) == (pick["team"], pick["block"])
    assert np.array_equal(T.cpu().numpy(), st.T)  # the sample was copied, inputs untouched
    g.integrate(T, P, Y, 1e-6)
    yo, _ = om.integrate(y0, st.P, 1e-6)
    assert weighted_norm(yo, gpu_state(om, T, Y)).max() <= 1e-5


def _oracle_splits(om, y0, P, dt, nsplit, rtol=1e-6, atol=1e-10):
    """The oracle over consecutive split steps with h carried: final state and per-split attempts."""
    y, hh = y0.copy(), np.zeros(len(y0))
    att = np.zeros((nsplit, len(y0)), dtype=np.int64)
    for s in range(nsplit):
        y, info = om.integrate(y, P, dt, rtol=rtol, atol=atol, h=hh, threads=16)
        assert np.all(info["status"] == 0)
        att[s] = info["attempts"]
        hh = info["h"]
    return y, att


def _check_split_sequence(om, P, y0, yg, att_gpu, dt, label):
    """Multi-split form of the flip rule: cells whose per-split attempt counts all equal the
    oracle's must be within 1e-5 in the weighted norm; cells where round-off flipped an
    accept/reject decision in any split step (at most 2% of cells) must lie within 10 tolerance
    units of the oracle at rtol 1e-10 over the same split steps."""
    nsplit = att_gpu.shape[0]
    yo, att_o = _oracle_splits(om, y0, P, dt, nsplit)
    same = np.all(att_o == att_gpu, axis=0)
    e = weighted_norm(yo, yg)
    assert np.all(e[same] <= 1e-5), (label, e[same].max(), np.argmax(np.where(same, e, 0)))
    flips = np.where(~same)[0]
    assert len(flips) <= max(1, int(0.02 * len(same))), (label, len(flips))
    if len(flips):
        yt, _ = _oracle_splits(om, y0[flips], P[flips], dt, nsplit, rtol=1e-10, atol=1e-14)
        assert np.all(weighted_norm(yt, yg[flips]) <= 10.0), label
    return e, att_o


def _capture_splits(g, T, P, Y, h, ws, dt, nsplit, att, att_hist):
    """nsplit consecutive split steps (h carried) captured in one CUDA graph; per-split attempt
    counts copied into att_hist[s] inside the graph."""
    import torch

    def body():
        for s in range(nsplit):
            g.integrate(T, P, Y, dt, h=h, opts=g.opts(attempts=att), workspace=ws)
            att_hist[s].copy_(att)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        body()
    return graph, body


def test_cuda_graph_of_split_steps(omech, gmech):
    """Three consecutive split steps (h carried) captured in one CUDA graph and replayed give the
    eager result (to rounding) and the oracle's within the parity bound."""
    import torch
    name = "ch4_53"
    om = omech(name)
    g = gmech(name, 64, 64)
    n, nsplit = 96, 3
    st, y0 = _inputs(om, name, n, 111)
    T0, P, Y0 = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    T, Y = T0.clone(), Y0.clone()
    h = torch.zeros(n, dtype=torch.float64, device=T.device)
    att = torch.zeros(n, dtype=torch.int32, device=T.device)
    hist = torch.zeros((nsplit, n), dtype=torch.int32, device=T.device)
    ws = g.workspace(n)
    graph, body = _capture_splits(g, T, P, Y, h, ws, 1e-6, nsplit, att, hist)
    T.copy_(T0); Y.copy_(Y0); h.zero_(); hist.zero_()
    body()  # eager
    torch.cuda.synchronize()
    eager = [x.cpu().numpy() for x in (T, Y, h, hist)]
    T.copy_(T0); Y.copy_(Y0); h.zero_(); hist.zero_()
    graph.replay()
    torch.cuda.synchronize()
    # the team's shared-memory atomics sum in a run-dependent order: equal to rounding
    for a, b in zip(eager[:3], (T, Y, h)):
        assert np.allclose(b.cpu().numpy(), a, rtol=1e-9, atol=1e-18)
    assert (hist.cpu().numpy() == eager[3]).all(axis=0).mean() >= 0.98
    _check_split_sequence(om, st.P, y0, gpu_state(om, T, Y), hist.cpu().numpy(), 1e-6, "graph53")


def _front_inputs(om, n, seed, n_templates=8, t_relax=1e-3):
    """Flame-front workload on n cells: ignition-front cells as generated; the near-equilibrium
    product cells are n_templates product states relaxed by the oracle for t_relax and tiled
    with a 1e-9 relative perturbation of the mass fractions (the oracle prepares the inputs of
    both sides)."""
    st = states("ch4_111", n, "ch4_front", seed)
    y0 = om.state_from_TY(st.T, st.Y)
    prod = np.where(st.T >= 1500.0)[0]
    k = min(n_templates, len(prod))
    yt, info = om.integrate(y0[prod[:k]], st.P[prod[:k]], t_relax, threads=16)
    assert np.all(info["status"] == 0)
    Tt, Yt = om.TY_from_state(yt)
    rng = np.random.default_rng(seed + 1)
    src = np.arange(len(prod)) % k
    T, P, Y = st.T.copy(), st.P.copy(), st.Y.copy()
    T[prod] = Tt[src]
    P[prod] = st.P[prod[:k]][src]
    Yp = Yt[src] * (1.0 + 1e-9 * rng.standard_normal((len(prod), Yt.shape[1])))
    Y[prod] = Yp / Yp.sum(axis=1, keepdims=True)

    class St:
        pass

    out = St()
    out.T, out.P, out.Y = T, P, Y
    return out, prod


def test_config3_graph_20_splits_111(omech, mech_path):
    """The batched flame-front configuration: 111 species, relaxed product cells interleaved with
    ignition-front cells, 20 split steps (h carried) replayed from one captured CUDA graph in the
    default launch configuration, more cells than resident teams; sampled front and product cells
    against the oracle over the same 20 split steps."""
    import torch
    name = "ch4_111"
    om = omech(name)
    g = _bench_config_mech(mech_path, name)
    n, nsplit, dt = 4096, 20, 1e-6
    st, prod = _front_inputs(om, n, 9)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    h = torch.zeros(n, dtype=torch.float64, device=T.device)
    att = torch.zeros(n, dtype=torch.int32, device=T.device)
    hist = torch.zeros((nsplit, n), dtype=torch.int32, device=T.device)
    ws = g.workspace(n)
    T0, Y0 = T.clone(), Y.clone()
    graph, body = _capture_splits(g, T, P, Y, h, ws, dt, nsplit, att, hist)
    T.copy_(T0); Y.copy_(Y0); h.zero_()
    graph.replay()
    torch.cuda.synchronize()
    hist_np = hist.cpu().numpy()
    tot = hist_np.sum(axis=0)
    front = np.setdiff1d(np.arange(n), prod)
    # the stated stiffness contrast: front cells need >= 10x the attempts of the median cell
    assert tot[front].max() >= 10 * np.median(tot), (tot[front].max(), np.median(tot))
    rng = np.random.default_rng(5)
    idx = np.sort(np.concatenate([rng.choice(front, 24, replace=False),
                                  rng.choice(prod, 24, replace=False)]))
    yg = gpu_state(om, T, Y)[idx]
    y0 = om.state_from_TY(st.T[idx], st.Y[idx])
    _check_split_sequence(om, st.P[idx], y0, yg, hist_np[:, idx], dt, "config3")
    assert (h.cpu().numpy() > 0).all()


@pytest.mark.parametrize("tab", [1, 2, 3])
@pytest.mark.parametrize("name", ["h2_13", "ch4_53"])
def test_other_rosenbrock_methods(omech, gmech, name, tab):
    """ROS3, RODAS3 and RODAS4 (the other methods of the paper's solver table) against the
    oracle running the same method, same tolerances as ROS4."""
    import torch
    om = omech(name)
    g = gmech(name, 64, 64)
    n = {"h2_13": 400, "ch4_53": 80}[name]
    st, y0 = _inputs(om, name, n, 112 + tab)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    status = torch.full((n,), -1, dtype=torch.int32, device=T.device)
    att = torch.zeros(n, dtype=torch.int32, device=T.device)
    g.integrate(T, P, Y, 1e-6, status=status, opts=g.opts(attempts=att, tableau=tab))
    assert (status.cpu().numpy() == 0).all()
    yo, info = om.integrate(y0, st.P, 1e-6, threads=16, tableau=tab)
    yg = gpu_state(om, T, Y)
    same = info["attempts"] == att.cpu().numpy()
    assert same.mean() >= 0.98
    assert weighted_norm(yo, yg)[same].max() <= 1e-5


@pytest.mark.parametrize("team,block", [(64, 64), (32, 64), (1, 32)])
def test_rkf45_parity(omech, gmech, team, block):
    """The explicit RKF45 of the paper's solver table on the non-stiff H2 cells (1 us split
    steps) against the oracle running RKF45: same per-cell result for matching step sequences,
    and it finishes the split step in fewer attempts than ROS4 on these cells."""
    import torch
    name = "h2_13"
    om = omech(name)
    g = gmech(name, team, block)
    n = 400
    st, y0 = _inputs(om, name, n, 141)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    status = torch.full((n,), -1, dtype=torch.int32, device=T.device)
    att = torch.zeros(n, dtype=torch.int32, device=T.device)
    g.integrate(T, P, Y, 1e-6, status=status, opts=g.opts(attempts=att, tableau=4))
    assert (status.cpu().numpy() == 0).all()
    yo, info = om.integrate(y0, st.P, 1e-6, threads=16, tableau=4)
    yg = gpu_state(om, T, Y)
    same = info["attempts"] == att.cpu().numpy()
    assert same.mean() >= 0.98
    assert weighted_norm(yo, yg)[same].max() <= 1e-5
    _, info4 = om.integrate(y0, st.P, 1e-6, threads=16)
    assert att.cpu().numpy().mean() < info4["attempts"].mean()


def test_rkf45_on_stiff_cells_reports_max_steps(gmech):
    """On stiff chemistry the explicit method's stable steps are tiny: the cells stop at the
    attempt limit (a per-cell status, not a fault), their last accepted state finite."""
    import torch
    from paper_2205_05681_gb300 import chem
    g = gmech("ch4_53", 64, 64)
    st = states("ch4_53", 32, "ch4_partial", 142)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    status = torch.full((32,), -1, dtype=torch.int32, device=T.device)
    g.integrate(T, P, Y, 1e-6, status=status, opts=g.opts(tableau=chem.RKF45, max_steps=2000))
    s = status.cpu().numpy()
    assert set(s.tolist()) <= {0, 1, 2} and (s != 0).sum() >= 8
    assert torch.isfinite(T).all() and torch.isfinite(Y).all()


def test_interleaved_reaction_order(mech_dir, mech_path):
    """A file with reactions of every kind interleaved: the library runs them in its own
    branch-grouped kernel order and maps run-time ln A, the per-reaction VJP rows and the
    integration back to the file's order (oracle on the same file)."""
    import os
    import torch
    from oracle import oracle as O
    dst = os.path.join(mech_dir, "ch4_53_interleaved.mech")
    shuffled_spec(mech_path("ch4_53"), dst, 11)
    om = O.Mechanism(dst)
    g = gpu_mech(dst, team=64, block=64)
    st = states("ch4_53", 96, "ch4_partial", 131)
    y = om.state_from_TY(st.T, st.Y)
    lnA = om.lnA + np.random.default_rng(3).normal(0.0, 0.2, om.nr)
    f = g.eval_source(to_dev(y[:, 0]), to_dev(st.P), to_dev(y[:, 1:].T), lnA=to_dev(lnA))
    f = f.cpu().numpy().T
    fo = om.source(y, st.P, lnA=lnA)
    for c in range(len(y)):
        err = np.abs(f[c] - fo[c]) / (np.abs(fo[c]) + gross_f(om, y[c], st.P[c]) + 1e-300)
        assert err.max() <= 1e-12, (c, err.max())
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    att = torch.zeros(len(y), dtype=torch.int32, device=T.device)
    g.integrate(T, P, Y, 1e-6, opts=g.opts(attempts=att))
    _check_integration(om, st, y, gpu_state(om, T, Y), att.cpu().numpy(), 1e-6, "interleaved")
    # (d f / d lnA)^T v rows in file order, against complex step of v^T f
    v = np.random.default_rng(4).normal(size=y.shape) / np.maximum(np.abs(om.source(y, st.P)), 1e-30)
    _, gp = g.eval_vjp(to_dev(y[:2, 0]), to_dev(st.P[:2]), to_dev(y[:2, 1:].T), to_dev(v[:2].T))
    gp = gp.cpu().numpy().T
    ref = np.zeros(om.nr)
    for r in range(om.nr):
        d = np.zeros(om.nr, dtype=complex)
        d[r] = 1e-30j
        ref[r] = (v[0] @ om.source_cplx(y[0], st.P[0], lnA=om.lnA + d).imag) / 1e-30
    assert np.all(np.abs(gp[0] - ref) <= 1e-11 * (np.abs(ref) + 1e-3 * np.abs(ref).max()))


def test_cost_ordered_queue(omech, mech_path):
    """chem_cost_order returns a permutation of the cells by decreasing cost bucket, and a work
    queue in that order gives every cell the result of the index-order queue (the order only
    decides which team takes a cell when); the oracle on a sample."""
    import torch
    name = "ch4_53"
    om = omech(name)
    g = _bench_config_mech(mech_path, name)
    n = 3000
    st = states(name, n, WORK[name], 31)
    T0, P, Y0 = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    att = torch.zeros(n, dtype=torch.int32, device=T0.device)
    T, Y = T0.clone(), Y0.clone()
    g.integrate(T, P, Y, 1e-6, opts=g.opts(attempts=att))
    ref = (T.cpu().numpy(), Y.cpu().numpy(), att.cpu().numpy())
    order = g.cost_order(att)
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(n))
    c = np.minimum(ref[2][o], 1023)
    assert np.all(np.diff(c) <= 0)
    T, Y = T0.clone(), Y0.clone()
    att2 = torch.zeros(n, dtype=torch.int32, device=T0.device)
    g.integrate(T, P, Y, 1e-6, opts=g.opts(attempts=att2, order=order))
    assert (att2.cpu().numpy() == ref[2]).mean() >= 0.99
    assert np.allclose(T.cpu().numpy(), ref[0], rtol=1e-9, atol=0)
    assert np.allclose(Y.cpu().numpy(), ref[1], rtol=1e-8, atol=1e-16)
    idx = np.append(o[:20], o[-4:])  # the most and the least expensive cells

    class Sub:
        P = st.P[idx]

    y0 = om.state_from_TY(st.T[idx], st.Y[idx])
    _check_integration(om, Sub, y0, gpu_state(om, T, Y)[idx], att2.cpu().numpy()[idx], 1e-6,
                       "cost-order")
    # cost buckets above 1023 share the top bucket; negative costs the bottom one
    cost = torch.tensor(np.array([5, 2000, -3, 1023, 7], dtype=np.int32), device=T0.device)
    assert g.cost_order(cost).cpu().numpy().tolist()[2:] == [4, 0, 2]


@pytest.mark.parametrize("name,team,block,alt", [("h2_13", 4, 64, 4), ("h2_13", 64, 64, 4),
                                                 ("ch4_53", 64, 64, 4), ("h2_13", 4, 64, 5),
                                                 ("ch4_111", 256, 256, 5)])
def test_per_cell_method_switching(omech, gmech, name, team, block, alt):
    """Per-cell switching between an alternative method (RKF45 by the stiffness rule, or the
    W-method with its factorisation cache for quiescent cells) and ROS4 over consecutive split
    steps (the method array carried like h) against the oracle running the same policy: the same
    method choices, and per cell the oracle's state within 1e-5 when its attempt counts match
    (flip rule as elsewhere)."""
    import torch
    om = omech(name)
    g = gmech(name, team, block)
    n = {"h2_13": 600, "ch4_53": 120, "ch4_111": 40}[name]
    nsplit, dt = (3 if alt == 4 else 5), 1e-6
    if name == "ch4_111":  # relaxed product cells and ignition-front cells
        st, _ = _front_inputs(om, n, 17)
        y0 = om.state_from_TY(st.T, st.Y)
    else:
        st, y0 = _inputs(om, name, n, 151)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    h = torch.zeros(n, dtype=torch.float64, device=T.device)
    att = torch.zeros(n, dtype=torch.int32, device=T.device)
    status = torch.full((n,), -1, dtype=torch.int32, device=T.device)
    meth = torch.zeros(n, dtype=torch.int32, device=T.device)
    jc = g.jac_cache(n) if alt == 5 else None
    o = g.opts(attempts=att, cell_method=meth, jac_cache=jc, alt_tableau=alt)
    ws = g.workspace(n, o)
    cache = om.w_cache(n) if alt == 5 else None
    y, hh = y0.copy(), np.zeros(n)
    mo = np.zeros(n, dtype=np.int32)
    same = np.ones(n, dtype=bool)
    for s in range(nsplit):
        g.integrate(T, P, Y, dt, h=h, status=status, opts=o, workspace=ws)
        y, info = om.integrate_auto(y, st.P, dt, mo, h=hh, threads=16, alt=alt, cache=cache)
        hh = info["h"]
        assert (status.cpu().numpy() == 0).all() and np.all(info["status"] == 0)
        mg = meth.cpu().numpy()
        same &= (mg == mo) & (att.cpu().numpy() == info["attempts"])
        # the method chosen for the next split step (its budget follows the attempt count)
        assert ((mg > 0) != (mo > 0)).mean() <= 0.02, (s, ((mg > 0) != (mo > 0)).sum())
    if alt == 5:  # quiescent cells move to the W-method (the partly reacted H2 cells: some)
        assert (mo > 0).mean() > (0.15 if name == "h2_13" else 0.5)
    elif name == "h2_13":
        assert (mo > 0).mean() > 0.5  # most of these cells run explicitly after the first step
    else:
        assert (mo == 0).all()  # stiff cells stay on the Rosenbrock method
    yg = gpu_state(om, T, Y)
    e = weighted_norm(y, yg)
    assert np.all(e[same] <= 1e-5), (e[same].max(), np.argmax(np.where(same, e, 0)))
    flips = np.where(~same)[0]
    # a flip can happen at every split step's decisions: at most 2% of the cells per split step
    assert len(flips) <= max(1, int(np.ceil(0.02 * n * nsplit))), len(flips)
    if len(flips):
        yt, _ = _oracle_splits(om, y0[flips], st.P[flips], dt, nsplit, rtol=1e-10, atol=1e-14)
        assert np.all(weighted_norm(yt, yg[flips]) <= 10.0)


@pytest.mark.parametrize("name,team,block", [("h2_13", 4, 64), ("ch4_53", 64, 64),
                                             ("ch4_111", 256, 256)])
def test_w_method_with_factorisation_reuse(omech, gmech, name, team, block):
    """The W-method ROS2 with its factorisation cache carried over consecutive split steps against
    the oracle's W-method with its Jacobian cache: the same reuse decisions (each cell's cache
    step size and age after every split step) and states within 1e-5 for matching attempt
    sequences (flip rule as elsewhere)."""
    import torch
    from paper_2205_05681_gb300 import chem
    om = omech(name)
    g = gmech(name, team, block)
    n = {"h2_13": 400, "ch4_53": 96, "ch4_111": 48}[name]
    nsplit, dt = 4, 1e-6
    st, y0 = _inputs(om, name, n, 161)
    if name != "h2_13":  # partly relaxed cells: the regime where the factorisation is reused
        yq, _ = om.integrate(y0, st.P, 1e-4, threads=16)
        st.T, st.Y = om.TY_from_state(yq)
        y0 = om.state_from_TY(st.T, st.Y)
    T, P, Y = to_dev(st.T), to_dev(st.P), to_dev(st.Y.T)
    h = torch.zeros(n, dtype=torch.float64, device=T.device)
    att = torch.zeros(n, dtype=torch.int32, device=T.device)
    status = torch.full((n,), -1, dtype=torch.int32, device=T.device)
    jc = g.jac_cache(n)
    stride = jc.numel() // n
    o = g.opts(attempts=att, tableau=chem.ROS2W, jac_cache=jc)
    cache = om.w_cache(n)
    y, hh = y0.copy(), np.zeros(n)
    same = np.ones(n, dtype=bool)
    reused = 0
    for s in range(nsplit):
        g.integrate(T, P, Y, dt, h=h, status=status, opts=o)
        y, info = om.integrate_w(y, st.P, dt, cache, h=hh, threads=16)
        hh = info["h"]
        assert (status.cpu().numpy() == 0).all() and np.all(info["status"] == 0)
        c = jc.view(n, stride).cpu().numpy()
        same &= att.cpu().numpy() == info["attempts"]
        # the same reuse decisions: equal ages, and cache step sizes equal up to the drift of the
        # step-size sequences (rounding; a different decision would store another step's size)
        same &= (c[:, -1] == cache[2]) & (np.abs(c[:, -2] - cache[1]) <= 1e-6 * cache[1])
        if s > 0:
            reused += int((info["n_jac"] == 0).sum())
    assert reused > 0  # the cache was used across calls
    yg = gpu_state(om, T, Y)
    e = weighted_norm(y, yg)
    assert np.all(e[same] <= 1e-5), (e[same].max(), np.argmax(np.where(same, e, 0)))
    flips = np.where(~same)[0]
    # a flip can happen at every split step's decisions: at most 2% of the cells per split step
    assert len(flips) <= max(1, int(np.ceil(0.02 * n * nsplit))), len(flips)
    if len(flips):
        yt, _ = _oracle_splits(om, y0[flips], st.P[flips], dt, nsplit, rtol=1e-10, atol=1e-14)
        assert np.all(weighted_norm(yt, yg[flips]) <= 10.0)
