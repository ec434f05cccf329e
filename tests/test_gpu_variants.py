"""Test builds of the same CUDA sources against the CPU oracle, bit for bit.

- lccap: a block keeps at most 4 lane-change candidates in shared memory, so
  nearly every candidate goes through the block's overflow region of the
  global candidate list (the product build overflows only when a block lists
  more than ~2,100 candidates in one step).
- walk8 / walk16: leader-walk batches of 64 / 128 bytes and of 128 / 256 bytes
  (first batch / later batches) instead of 32 / 64.

Each is compared every step on mixed small networks (lane changes, merges,
stop signs, signals, closures) and at checkpoints on the tiny workload and on
the full metro network with the 07:30-07:35 trips.
"""
import numpy as np
import pytest

import nets
from oracle import oracle as O
from paper_2007_03614_b300 import manta, synth
from paper_2007_03614_b300.build import build, build_variant
from test_gpu_parity import _compare, _compare_all, _subset

pytestmark = pytest.mark.gpu

VARIANTS = ("lccap", "walk8", "walk16")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build()


def _pair(lib, net, tr, closures=(), **cfg):
    o = O.OracleSim(net, **cfg)
    g = manta.Sim(net, library=lib, **cfg)
    for (e, l, k0, k1) in closures:
        o.set_lane_closure(e, l, k0, k1)
        g.set_lane_closure(e, l, k0, k1)
    nets.load(o, tr)
    nets.load(g, tr)
    return o, g


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_small_mixed_every_step(variant):
    from test_oracle_bruteforce import CFGS, _scenario, closures_for
    lib = build_variant(variant)
    for seed, ci in ((1, 0), (2, 1), (3, 2), (4, 3)):
        net, tr = _scenario(seed, n_trips=40)
        cfg = dict(CFGS[ci])
        cfg["seed"] = 100 + seed
        o, g = _pair(lib, net, tr, closures=closures_for(net, seed) if ci == 1 else (), **cfg)
        for k in range(400):
            o.step(1)
            g.step(1)
            _compare(o, g, f"{variant} seed {seed} cfg {ci} step {k}")
        _compare_all(o, g)
        g.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_tiny_workload(variant):
    lib = build_variant(variant)
    net = synth.tiny_network()
    tr = synth.tiny_trips(net)
    o, g = _pair(lib, net, tr)
    for k in range(0, 1800, 100):
        o.step(100)
        g.step(100)
        _compare(o, g, f"{variant} step {k + 100}")
    _compare_all(o, g, windows=range(3))
    if variant == "lccap":
        # every gap-acceptance evaluation read its candidate from the overflow region
        assert g.stats()["lc_evals"] > 300
    g.close()


@pytest.fixture(scope="module")
def metro_window(metro):
    net, tr = metro
    return net, _subset(tr, 7.5 * 3600, 7.5 * 3600 + 300)


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_metro_window(variant, metro_window):
    lib = build_variant(variant)
    net, sub = metro_window
    t0 = int(7.5 * 3600 / 0.5)
    o, g = _pair(lib, net, sub, t0_step=t0, n_stats_windows=4)
    for k in range(0, 400, 200):
        o.step(200)
        g.step(200)
        _compare(o, g, f"{variant} metro step {k + 200}")
    _compare_all(o, g, windows=(0,))
    g.close()
