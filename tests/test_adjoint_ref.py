"""CPU pins of the reference adjoint (oracle/adjoint.py) used to check the
calibration gradient of the CUDA library.

- On a lone vehicle accelerating on a free road, the adjoint equals the
  tangent (forward-mode) derivative of the ballistic IDM recurrence along the
  recorded trajectory, written out here on its own.
- On a congested grid run, the adjoint equals central finite differences
  (h = 1e-3) of the frozen-event replay, to 1e-3 relative.
- The replay with the run's own parameters reproduces the run's link speeds.
"""
import numpy as np
import pytest

import nets
from oracle import adjoint as A
from oracle import oracle as O
from paper_2007_03614_b300 import synth


def _theta(cfg, n_classes):
    return np.array([[cfg.v0f[c], cfg.T[c], cfg.a[c], cfg.b[c], cfg.s0[c]] for c in range(n_classes)],
                    dtype=np.float64)


def test_lone_vehicle_matches_forward_mode():
    """v_{k+1} = v_k + a (1 - (v_k / v0)^4) dt from rest on a free road; the
    loss is the mean of the speed samples.  Tangents dv/da and dv/dv0f follow
    d(v_{k+1}) = d(v_k) (1 + dt dacc/dv) + dt dacc/dtheta."""
    net = nets.line(12, length=400.0, speed=20.0)
    o = O.OracleSim(net, stats_window_steps=100000, n_stats_windows=1)
    nets.load(o, nets.trips([list(range(12))], [0.0]))
    K = 120
    tape = o.record_tape(K)
    o.step(K)
    cfg = o.cfg
    theta = _theta(cfg, 1)
    dt = float(cfg.dt)
    n_cells = net.n_edges if hasattr(net, "n_edges") else len(net.edge_src)
    present = (tape["flags"][:, 0] & 1) != 0
    samples = (tape["sample"][:, 0] >= 0) & present
    n_s = int(samples.sum())
    assert n_s > 50
    # dLoss/d(sample) for loss = mean of all samples; cells differ by edge, so
    # use per-sample seeds: every sample of every cell weighs 1 / n_s
    seed = np.full(n_cells, 1.0 / n_s)
    grad, _, _ = A.adjoint(tape, theta, dt, seed, 1)
    # forward mode, written out for this free-road case
    v0f, T, a, b, s0 = theta[0]
    lim = 20.0
    v0 = lim * float(v0f)
    dv_da = dv_dv0f = 0.0
    tot_da = tot_dv0f = 0.0
    first = int(np.argmax(present))
    for t in range(first, K):
        if not present[t]:
            break
        v = float(tape["v"][t, 0])          # derivatives along the recorded (binary32) trajectory
        r = v / v0
        acc = a * (1.0 - r ** 4)
        assert acc * dt + v >= 0.0
        dacc_dv = -4.0 * a * r ** 3 / v0
        dacc_da = 1.0 - r ** 4
        dacc_dv0f = 4.0 * a * r ** 4 / v0 * lim
        dv_da, dv_dv0f = (dv_da * (1.0 + dt * dacc_dv) + dt * dacc_da,
                          dv_dv0f * (1.0 + dt * dacc_dv) + dt * dacc_dv0f)
        if samples[t]:
            tot_da += dv_da / n_s
            tot_dv0f += dv_dv0f / n_s
    assert grad[0, 2] == pytest.approx(tot_da, rel=1e-9)
    assert grad[0, 0] == pytest.approx(tot_dv0f, rel=1e-9)
    assert grad[0, 1] == 0.0 and grad[0, 3] == 0.0 and grad[0, 4] == 0.0   # no leader: T, b, s0 unused


@pytest.fixture(scope="module")
def grid_run():
    net = synth.calib_network()
    tr = synth.calib_trips(net, n_trips=1500)
    o = O.OracleSim(net, stats_window_steps=120, n_stats_windows=5)
    nets.load(o, tr)
    tape = o.record_tape(600)
    o.step(600)
    return net, o, tape


def _cells(tape, n_cells):
    present = (tape["flags"] & 1) != 0
    out = (tape["flags"] >> 6) & 7
    use = present & (out != 4) & (tape["sample"] >= 0)
    return np.bincount(tape["sample"][use], minlength=n_cells).astype(np.float64)


def test_replay_reproduces_the_run(grid_run):
    net, o, tape = grid_run
    E = len(net.edge_src)
    theta = _theta(o.cfg, 3)
    sums, _, _, _ = A.replay(tape, theta, float(o.cfg.dt), 5 * E)
    cnt = _cells(tape, 5 * E)
    obs = cnt > 0
    assert obs.sum() > 500
    ref = np.concatenate([o.edge_counters(w)["speed_sum"].astype(np.float64) / 1048576.0 for w in range(5)])
    ref_cnt = np.concatenate([o.edge_counters(w)["speed_cnt"].astype(np.float64) for w in range(5)])
    assert np.array_equal(ref_cnt, cnt)
    # the run sums truncated binary32 speeds; the replay sums binary64 ones
    assert np.max(np.abs(sums[obs] / cnt[obs] - ref[obs] / cnt[obs])) < 2e-3


def test_adjoint_matches_central_differences(grid_run):
    net, o, tape = grid_run
    E = len(net.edge_src)
    n_cells = 5 * E
    dt = float(o.cfg.dt)
    theta = _theta(o.cfg, 3)
    cnt = _cells(tape, n_cells)
    obs = cnt > 0
    rng = np.random.default_rng(7)
    target = np.where(obs, rng.uniform(2.0, 12.0, n_cells), 0.0)

    def loss(th):
        sums, _, _, _ = A.replay(tape, th, dt, n_cells)
        m = np.where(obs, sums / np.maximum(cnt, 1.0), 0.0)
        return float(np.sum((m - target)[obs] ** 2) / obs.sum())

    sums, _, _, _ = A.replay(tape, theta, dt, n_cells)
    m = np.where(obs, sums / np.maximum(cnt, 1.0), 0.0)
    seed = np.where(obs, 2.0 * (m - target) / (obs.sum() * np.maximum(cnt, 1.0)), 0.0)
    grad, _, _ = A.adjoint(tape, theta, dt, seed, 3)
    h = 1e-3
    scale = np.max(np.abs(grad))
    assert scale > 0
    checked = 0
    for c in range(3):
        for j in range(5):
            tp, tm = theta.copy(), theta.copy()
            tp[c, j] += h
            tm[c, j] -= h
            fd = (loss(tp) - loss(tm)) / (2 * h)
            assert abs(fd - grad[c, j]) <= 1e-3 * max(abs(fd), 1e-3 * scale), (c, A.PARAMS[j], fd, grad[c, j])
            checked += abs(grad[c, j]) > 1e-3 * scale
    assert checked >= 10        # most parameters of all three classes matter in this run
