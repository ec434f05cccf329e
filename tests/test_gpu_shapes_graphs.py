"""Launch shapes, the autotuner and CUDA-graph replay of the step kernel.

Every launch shape of the step kernel, every autotuned run and every replay
of a captured graph must give the trajectory of plain manta_step calls bit
for bit, and that trajectory must equal the oracle's.
"""
import numpy as np
import pytest

import nets
from oracle import oracle as O
from paper_2007_03614_b300 import manta, synth
from paper_2007_03614_b300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build()
    manta.load_library()


def _same(a, b, where):
    """Snapshots, counters and lane maps of two simulations agree bit for bit."""
    sa, sb = a.snapshot(), b.snapshot()
    for key in ("id", "edge", "lane", "dwell", "route_pos"):
        assert np.array_equal(sa[key], sb[key]), (where, key)
    for key in ("x", "v"):
        assert np.array_equal(sa[key].view(np.uint32), sb[key].view(np.uint32)), (where, key)
    ta, tb = a.stats(), b.stats()
    for key in ta:
        assert ta[key] == tb[key], (where, key, ta[key], tb[key])
    assert np.array_equal(a.lane_map(), b.lane_map()), where
    for w in range(3):
        ea, eb = a.edge_counters(w), b.edge_counters(w)
        for key in ea:
            assert np.array_equal(ea[key], eb[key]), (where, w, key)


@pytest.fixture(scope="module")
def tiny():
    net = synth.tiny_network()
    return net, synth.tiny_trips(net)


@pytest.fixture(scope="module")
def oracle_at(tiny):
    """The oracle's state at a few step counts (one run)."""
    net, tr = tiny
    o = O.OracleSim(net)
    nets.load(o, tr)
    out = {}
    done = 0
    for k in (600, 840, 1200, 3600):
        o.step(k - done)
        done = k
        out[k] = (o.snapshot(), o.stats(), o.lane_map())
    return out


def _same_as_oracle(g, ref, where):
    so, to, mo = ref
    sg = g.snapshot()
    for key in ("id", "edge", "lane", "dwell", "route_pos"):
        assert np.array_equal(so[key], sg[key]), (where, key)
    for key in ("x", "v"):
        assert np.array_equal(so[key].view(np.uint32), sg[key].view(np.uint32)), (where, key)
    tg = g.stats()
    for key in to:
        assert to[key] == tg[key], (where, key)
    assert np.array_equal(mo, g.lane_map()), where


def test_shape_table():
    shapes = manta.variants()
    assert len(shapes) >= 2
    for t, b in shapes:
        assert t % 32 == 0 and 32 <= t <= 1024 and b >= 1


@pytest.mark.parametrize("v", range(4))
def test_every_launch_shape_matches_the_oracle(tiny, oracle_at, v):
    if v >= len(manta.variants()):
        pytest.skip("no such shape")
    net, tr = tiny
    g = manta.Sim(net)
    g.variant = v
    assert g.variant == v
    nets.load(g, tr)
    for _ in range(4):
        g.step(300)
    _same_as_oracle(g, oracle_at[1200], f"shape {v}")
    g.close()


def test_graph_replay_equals_direct_steps(tiny, oracle_at):
    import torch
    net, tr = tiny
    a = manta.Sim(net, stream=torch.cuda.Stream())
    b = manta.Sim(net, stream=torch.cuda.Stream())
    nets.load(a, tr)
    nets.load(b, tr)
    gr = b.graph(120)
    gr.launch(5)             # 600 steps
    _same_as_oracle(b, oracle_at[600], "after 5 replays")
    b.step(30)               # direct steps between replays
    gr.launch(1)             # 750
    a.step(750)
    _same(a, b, "750 steps")
    gr.launch(0)
    b.step(90)               # 840
    _same_as_oracle(b, oracle_at[840], "840 steps")
    gr.close()
    # a graph spanning more than one launch (2048 steps per launch)
    g2 = b.graph(2760)
    g2.launch(1)             # 3600
    _same_as_oracle(b, oracle_at[3600], "3600 steps")
    g2.close()
    a.close()
    b.close()


def test_autotune_keeps_the_trajectory(tiny, oracle_at):
    import torch
    net, tr = tiny
    g = manta.Sim(net, stream=torch.cuda.Stream())
    nets.load(g, tr)
    n = len(manta.variants())
    chosen, ms = g.autotune(trial_steps=30, rounds=2)   # advances 2 x n x 30 steps
    assert 0 <= chosen < n and g.variant == chosen
    assert ms.shape == (n,) and np.all(ms > 0)
    assert g.stats()["step"] == 2 * n * 30
    g.step(1200 - 2 * n * 30)
    _same_as_oracle(g, oracle_at[1200], "after autotune")
    g.close()


def test_shape_and_graph_argument_errors(tiny):
    net, tr = tiny
    g = manta.Sim(net)
    with pytest.raises(manta.MantaError):
        g.variant = len(manta.variants())
    with pytest.raises(manta.MantaError):
        g.graph(10)          # no trips loaded yet
    nets.load(g, tr)
    with pytest.raises(manta.MantaError):
        g.graph(10)          # created on the default stream
    with pytest.raises(manta.MantaError):
        g.autotune(trial_steps=0)
    g.close()


def test_red_light_is_slower_than_green_light():
    """Section IV-C trend on a small grid: every node a flashing red (2 s stop,
    one vehicle at a time) against every node green, same trips and routes:
    red is slower, in the first and in the busiest statistics window."""
    import dataclasses
    net = synth.calib_network()
    tr = synth.calib_trips(net, n_trips=4000)
    speeds = {}
    for name, t in (("green", 0), ("red", 1)):
        n2 = dataclasses.replace(net, node_type=np.full_like(net.node_type, t))
        g = manta.Sim(n2, stats_window_steps=600, n_stats_windows=4)
        nets.load(g, tr)
        g.step(2400)
        w = []
        for k in range(4):
            ec = g.edge_counters(k)
            c = ec["speed_cnt"].astype(np.float64)
            w.append((ec["speed_sum"].astype(np.float64).sum() / 1048576.0 / max(c.sum(), 1.0), c.sum()))
        speeds[name] = w
        g.close()
    busiest = int(np.argmax([c for _, c in speeds["green"]]))
    assert speeds["red"][0][0] < speeds["green"][0][0]
    assert speeds["red"][busiest][0] < speeds["green"][busiest][0]
