"""GPU checkpoints, event tape and calibration adjoint.

- Restoring a checkpoint and running on gives bit-identical results.
- The event tape recorded by the CUDA step kernel equals the oracle's own
  tape of the same run field by field (the runs are bit-identical).
- The CUDA adjoint equals the CPU reference adjoint (oracle/adjoint.py, itself
  pinned against forward-mode derivatives and finite differences).
- The CUDA adjoint equals central finite differences (h = 1e-3) of the CUDA
  frozen-event replay to 1e-3 relative.
- The checkpointed backward pass (segments of 120 steps, re-run and taped
  from their checkpoints) equals the single-tape adjoint.
- The torch.autograd.Function gives a descent direction for a link-speed loss.
"""
import numpy as np
import pytest

import nets
from oracle import adjoint as A
from oracle import oracle as O
from paper_2007_03614_b300 import calibrate, manta, synth
from paper_2007_03614_b300.build import build

pytestmark = pytest.mark.gpu

NONE = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build()
    manta.load_library()


def _theta(cfg, n):
    return np.array([[cfg.v0f[c], cfg.T[c], cfg.a[c], cfg.b[c], cfg.s0[c]] for c in range(n)], np.float64)


def test_checkpoint_restore_is_bit_exact():
    import torch
    net = synth.tiny_network()
    tr = synth.tiny_trips(net)
    g = manta.Sim(net, stream=torch.cuda.Stream())
    nets.load(g, tr)
    g.step(400)
    ck = g.checkpoint()
    assert ck.step == 400 and ck.nbytes > 0
    g.step(300)
    a = (g.snapshot(), g.stats(), g.lane_map(), g.edge_counters(1))
    g.restore(ck)
    assert g.stats()["step"] == 400
    g.step(300)
    b = (g.snapshot(), g.stats(), g.lane_map(), g.edge_counters(1))
    for key in ("id", "edge", "lane", "dwell", "route_pos"):
        assert np.array_equal(a[0][key], b[0][key]), key
    for key in ("x", "v"):
        assert np.array_equal(a[0][key].view(np.uint32), b[0][key].view(np.uint32)), key
    assert a[1] == b[1]
    assert np.array_equal(a[2], b[2])
    for key in a[3]:
        assert np.array_equal(a[3][key], b[3][key]), key
    ck.close()
    g.close()


@pytest.fixture(scope="module", params=[0.0, 0.1], ids=["edge-limits", "per-driver-limits"])
def taped(request):
    """The same 600-step run (calibration grid, 1500 trips, 1-minute windows)
    with its event tape, on the oracle and on the GPU; once with every driver
    at the edge's speed limit, once with per-driver limits (Section IV-B)."""
    import torch
    net = synth.calib_network()
    tr = synth.calib_trips(net, n_trips=1500)
    cfg = dict(stats_window_steps=120, n_stats_windows=5, speed_sigma_frac=request.param)
    o = O.OracleSim(net, **cfg)
    nets.load(o, tr)
    ot = o.record_tape(600)
    o.step(600)
    g = manta.Sim(net, stream=torch.cuda.Stream(), **cfg)
    nets.load(g, tr)
    g.tape_start(600)
    g.step(600)
    gt = g.tape_copy(600)
    return net, tr, o, ot, g, gt


def test_tape_matches_the_oracle(taped):
    net, tr, o, ot, g, gt = taped
    of = ot["flags"]
    present = (of & 1) != 0
    gp = (gt["flags"] & 1) != 0
    assert np.array_equal(present, gp)
    assert present.sum() > 20_000
    for key in ("x", "v", "s", "vL", "bnd", "lim"):
        assert np.array_equal(ot[key][present].view(np.uint32), gt[key][present].view(np.uint32)), key
    assert np.array_equal(ot["C"][present].astype(np.uint32), gt["cells"][present])
    gf = gt["flags"][present]
    of = of[present]
    assert np.array_equal((of >> 1) & 3, (gf >> 1) & 3)            # kind
    assert np.array_equal((of >> 3) & 1, (gf >> 3) & 1)            # ballistic branch
    assert np.array_equal((of >> 4) & 3, (gf >> 4) & 3)            # clamp
    assert np.array_equal((of >> 6) & 7, (gf >> 6) & 7)            # outcome
    assert np.array_equal((of >> 9) & 7, (gf >> 12) & 15)          # road class
    os_ = ot["sample"][present]
    gs = gt["sample"][present].astype(np.int64)
    assert np.array_equal(np.where(os_ < 0, NONE, os_), gs)
    # every outcome and event kind occurs in this run
    for sh, width, n in ((1, 3, 3), (6, 7, 5)):
        assert len(np.unique((of >> sh) & width)) == n


def _seed(tape_sample, tape_flags, n_cells, target_seed=7):
    present = (tape_flags & 1) != 0
    out = (tape_flags >> 6) & 7
    use = present & (out != 4) & (tape_sample >= 0) & (tape_sample != NONE)
    cnt = np.bincount(tape_sample[use].astype(np.int64), minlength=n_cells).astype(np.float64)
    obs = cnt > 0
    target = np.where(obs, np.random.default_rng(target_seed).uniform(2.0, 12.0, n_cells), 0.0)
    return cnt, obs, target


def test_gpu_adjoint_matches_the_reference(taped):
    import torch
    net, tr, o, ot, g, gt = taped
    E = len(net.edge_src)
    n_cells = 5 * E
    dt = float(o.cfg.dt)
    theta = _theta(o.cfg, 3)
    cnt, obs, target = _seed(ot["sample"], ot["flags"], n_cells)
    sums, _, _, _ = A.replay(ot, theta, dt, n_cells)
    m = np.where(obs, sums / np.maximum(cnt, 1.0), 0.0)
    seed = np.where(obs, 2.0 * (m - target) / (obs.sum() * np.maximum(cnt, 1.0)), 0.0)
    ref, rlx, rlv = A.adjoint(ot, theta, dt, seed, 3)
    dev = torch.device("cuda")
    N = tr.n_trips
    lx = torch.zeros(N, dtype=torch.float64, device=dev)
    lv = torch.zeros(N, dtype=torch.float64, device=dev)
    grad = torch.zeros(40, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    g.adjoint(torch.as_tensor(seed, device=dev), lx, lv, grad)
    torch.cuda.synchronize()
    got = grad[:15].cpu().numpy().reshape(3, 5)
    scale = np.max(np.abs(ref))
    assert scale > 0
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-12 * scale)
    np.testing.assert_allclose(lx.cpu().numpy(), rlx, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(lv.cpu().numpy(), rlv, rtol=1e-9, atol=1e-12)


def test_gpu_adjoint_matches_replay_differences(taped):
    import torch
    net, tr, o, ot, g, gt = taped
    E = len(net.edge_src)
    n_cells = 5 * E
    theta = _theta(o.cfg, 3)
    cnt, obs, target = _seed(gt["sample"], gt["flags"], n_cells)
    dev = torch.device("cuda")
    N = tr.n_trips
    cnt_t = torch.as_tensor(cnt, device=dev)
    obs_t = torch.as_tensor(obs, device=dev)
    target_t = torch.as_tensor(target, device=dev)

    def replay_mean(th):
        x = torch.zeros(N, dtype=torch.float64, device=dev)
        v = torch.zeros(N, dtype=torch.float64, device=dev)
        pr = torch.zeros(N, dtype=torch.uint8, device=dev)
        sums = torch.zeros(n_cells, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        g.replay(th, x, v, pr, sums)
        torch.cuda.synchronize()
        return torch.where(obs_t, sums / cnt_t.clamp(min=1.0), torch.zeros_like(sums))

    def loss(th):
        m = replay_mean(th)
        return float(((m - target_t)[obs_t] ** 2).sum() / obs_t.sum())

    m = replay_mean(theta)
    seed = torch.where(obs_t, 2.0 * (m - target_t) / (obs_t.sum() * cnt_t.clamp(min=1.0)), torch.zeros_like(m))
    lx = torch.zeros(N, dtype=torch.float64, device=dev)
    lv = torch.zeros(N, dtype=torch.float64, device=dev)
    grad = torch.zeros(40, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    g.adjoint(seed.contiguous(), lx, lv, grad)
    torch.cuda.synchronize()
    adj = grad[:15].cpu().numpy().reshape(3, 5)
    scale = np.max(np.abs(adj))
    h = 1e-3
    for c in range(3):
        for j in range(5):
            tp, tm = theta.copy(), theta.copy()
            tp[c, j] += h
            tm[c, j] -= h
            fd = (loss(tp) - loss(tm)) / (2 * h)
            assert abs(fd - adj[c, j]) <= 1e-3 * max(abs(fd), 1e-3 * scale), (c, A.PARAMS[j], fd, adj[c, j])


def test_gpu_adjoint_and_replay_are_bit_reproducible(taped):
    """Two sweeps over the same tape give the same bits: gradient, lam_x and
    lam_v of the adjoint, and the state and speed sums of a replay with
    perturbed parameters (no sum depends on the order GPU threads run in)."""
    import torch
    net, tr, o, ot, g, gt = taped
    E = len(net.edge_src)
    n_cells = 5 * E
    dev = torch.device("cuda")
    N = tr.n_trips
    theta = _theta(o.cfg, 3)
    rng = np.random.default_rng(5)
    seed = torch.as_tensor(rng.normal(size=n_cells) * 1e-3, device=dev)
    th_p = theta * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, theta.shape))
    runs = []
    for _ in range(2):
        lx = torch.full((N,), 0.25, dtype=torch.float64, device=dev)
        lv = torch.full((N,), -0.5, dtype=torch.float64, device=dev)
        grad = torch.zeros(15, dtype=torch.float64, device=dev)
        x = torch.zeros(N, dtype=torch.float64, device=dev)
        v = torch.zeros(N, dtype=torch.float64, device=dev)
        pr = torch.zeros(N, dtype=torch.uint8, device=dev)
        sums = torch.full((n_cells,), 1.0, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        g.adjoint(seed, lx, lv, grad)
        g.replay(th_p, x, v, pr, sums)
        torch.cuda.synchronize()
        runs.append([t.cpu().numpy() for t in (grad, lx, lv, x, v, pr, sums)])
    assert np.abs(runs[0][0]).max() > 0 and (runs[0][6] != 1.0).sum() > 100
    for a, b in zip(*runs):
        assert a.tobytes() == b.tobytes()


def test_checkpointed_backward_equals_single_tape():
    import torch
    net = synth.calib_network()
    tr = synth.calib_trips(net, n_trips=1500)
    run = calibrate.LinkSpeedRun(net, tr, n_steps=600, window_steps=120, checkpoint_every=120)
    theta = _theta(manta.default_config(), 3)
    mean, cnt = run.forward(theta)
    G = torch.as_tensor(np.random.default_rng(3).normal(size=tuple(mean.shape)), device=mean.device)
    G = torch.where(cnt > 0, G, torch.zeros_like(G))
    got = run.backward(G)
    # one tape over the whole run
    g = manta.Sim(net, stream=torch.cuda.Stream(), stats_window_steps=120, n_stats_windows=5)
    nets.load(g, tr)
    g.tape_start(600)
    g.step(600)
    dev = torch.device("cuda")
    seed = torch.where(cnt > 0, G / cnt.clamp(min=1.0), torch.zeros_like(G)).reshape(-1).contiguous()
    lx = torch.zeros(tr.n_trips, dtype=torch.float64, device=dev)
    lv = torch.zeros(tr.n_trips, dtype=torch.float64, device=dev)
    grad = torch.zeros(40, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    g.adjoint(seed, lx, lv, grad)
    torch.cuda.synchronize()
    ref = grad[:15].cpu().numpy().reshape(3, 5)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-14 * np.max(np.abs(ref)))
    run.close()
    g.close()


def test_autograd_gives_a_descent_direction():
    import torch
    net = synth.calib_network()
    tr = synth.calib_trips(net, n_trips=3000)
    run = calibrate.LinkSpeedRun(net, tr, n_steps=1200, window_steps=600, checkpoint_every=120)
    rng = np.random.default_rng(11)
    # hidden parameters within the calibration bounds of Section III-A
    hidden = np.stack([rng.uniform(0.9, 1.1, 3), rng.uniform(1.0, 2.0, 3), rng.uniform(1.0, 2.5, 3),
                       rng.uniform(1.5, 3.5, 3), rng.uniform(1.5, 3.0, 3)], axis=1)
    with torch.no_grad():
        target = calibrate.link_speeds(torch.as_tensor(hidden), run).clone()
    obs = run.cnt > 0
    theta = torch.as_tensor(_theta(manta.default_config(), 3), dtype=torch.float64).requires_grad_(True)

    def loss_of(th):
        m = calibrate.link_speeds(th, run)
        return ((m - target)[obs] ** 2).mean()

    L0 = loss_of(theta)
    L0.backward()
    gr = theta.grad.detach().clone()
    assert torch.isfinite(gr).all() and gr.abs().max() > 0
    d = -gr / gr.abs().max()
    better = []
    for eps in (0.1, 0.05, 0.02, 0.01):
        with torch.no_grad():
            better.append(float(loss_of(theta.detach() + eps * d)) < float(L0))
    assert any(better), (float(L0), better)
    run.close()


def test_perturbation_search_reduces_the_objective():
    """The paper's calibration loop (Section III-A): 5 parameter sets per
    iteration, run batched as copies of the network; the objective (Eq. 5,
    mean absolute link-speed difference) ends below where it started."""
    import torch
    net = synth.calib_network()
    tr = synth.calib_trips(net, n_trips=3000)
    hidden = {"a": 2.2, "b": 3.0, "T": 1.1, "s0": 2.6}
    one = calibrate.copies(net, tr, 1)
    g = manta.Sim(one.net, stream=torch.cuda.Stream(), stats_window_steps=600, n_stats_windows=2, n_classes=1,
                  v0f=[1.0], a=[hidden["a"]], b=[hidden["b"]], T=[hidden["T"]], s0=[hidden["s0"]])
    g.load_trips(one.trips.route_off, one.trips.route_edges, one.trips.depart_time_s)
    g.step(1200)
    target, tcnt = calibrate.link_speed_cells(g, 2, 0, int(net.n_edges))
    g.close()
    cfg = manta.default_config()
    theta0 = {"a": cfg.a[0], "b": cfg.b[0], "T": cfg.T[0], "s0": cfg.s0[0]}
    out = calibrate.perturbation_search(net, tr, target, tcnt, theta0, iters=4, sets=5, n_steps=1200,
                                        window_steps=600, seed=5)
    h = out["history"]
    start = h[0]["objectives"][0]           # the starting set, run in copy 0
    assert h[-1]["objective"] < start, [x["objective"] for x in h]
    assert all(x["range"] == pytest.approx(0.1 ** i) for i, x in enumerate(h))
