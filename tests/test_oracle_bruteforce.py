"""T8: the oracle's lane-map implementation agrees bit for bit with a naive
list-based statement of the same step on tiny networks (pins the lane-map
indexing: row offsets, route-relative scan, boundaries, lane masks)."""
import numpy as np
import pytest

import nets
from naive_model import Naive
from oracle import oracle as O
from paper_2007_03614_b300 import synth


def _scenario(seed, n_trips=20, nx=3, ny=3):
    """A 3x3 lattice with mixed road classes and node controls; trips follow
    seeded random walks of 8-16 edges (contiguous but not shortest) so that
    vehicles meet at merges, queue at stop signs and signals and change lanes."""
    rng = np.random.default_rng(seed)
    net = synth.lattice(nx, ny, arterial_every=2, len_median_m=35.0, len_sigma=0.4, len_min_m=20.0,
                        len_max_m=70.0, speed_mps=(11.0, 14.0, 20.0), lanes=(1, 2, 3), seed=seed)
    n = net.n_nodes
    kinds = rng.integers(0, 3, n)
    net.node_type = kinds.astype(np.uint8)
    net.node_cycle_steps = np.where(kinds == 2, 20, 0).astype(np.int32)
    net.node_offset_steps = rng.integers(0, 20, n).astype(np.int32)
    net.edge_green_start = rng.integers(0, 10, net.n_edges).astype(np.int16)
    net.edge_green_len = np.full(net.n_edges, 10, np.int16)
    outs = {v: [e for e in range(net.n_edges) if net.edge_src[e] == v] for v in range(n)}
    routes = []
    for _ in range(n_trips):
        e = int(rng.integers(0, net.n_edges))
        r = [e]
        for _ in range(int(rng.integers(7, 16))):
            e = int(rng.choice(outs[int(net.edge_dst[e])]))
            r.append(e)
        routes.append(r)
    tr = nets.trips(routes, rng.uniform(0.0, 40.0, n_trips))
    return net, tr


CFGS = [dict(), dict(lc_len_scale_m=100.0), dict(idm_textbook=1, lc_len_scale_m=30.0, s0=[1.0, 3.5, 2.0]),
        dict(speed_sigma_frac=0.15)]


def closures_for(net, seed):
    """Seeded incident closures on a few multi-lane edges: (edge, lane, k0, k1)."""
    rng = np.random.default_rng(1000 + seed)
    multi = np.nonzero(net.edge_lanes >= 2)[0]
    out = []
    for e in rng.choice(multi, size=min(3, len(multi)), replace=False):
        lane = int(rng.integers(0, net.edge_lanes[e]))
        k0 = int(rng.integers(0, 150))
        out.append((int(e), lane, k0, k0 + int(rng.integers(50, 300))))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("ci", range(len(CFGS)))
def test_oracle_equals_naive(seed, ci):
    net, tr = _scenario(seed)
    cfg = dict(O.DEFAULTS)
    cfg.update(CFGS[ci])
    cfg["seed"] = 100 + seed
    s = O.OracleSim(net, **cfg)
    nets.load(s, tr)
    nv = Naive(net, tr, cfg)
    if ci == 1:
        for (e, l, k0, k1) in closures_for(net, seed):
            s.set_lane_closure(e, l, k0, k1)
            nv.closures[(e, l)] = (k0, k1)
    for k in range(500):
        s.step(1)
        nv.step()
        a, b = s.snapshot(), nv.snapshot()
        for key in ("id", "edge", "lane", "dwell", "route_pos"):
            assert np.array_equal(a[key], b[key]), (k, key, a[key], b[key])
        for key in ("x", "v"):
            assert np.array_equal(a[key].view(np.uint32), b[key].view(np.uint32)), (k, key, a[key], b[key])
    st = s.stats()
    for key, val in nv.st.items():
        assert st[key] == val, (key, st[key], val)
    assert st["lc_evals"] == 0 or st["lc_cells_scanned"] > 0
    ec = s.edge_counters(0)
    assert list(ec["entries"]) == nv.entry and list(ec["exits"]) == nv.exit
    for e in range(net.n_edges):
        sm, cn = nv.ssum.get((0, e), (0, 0))
        assert int(ec["speed_sum"][e]) == sm and int(ec["speed_cnt"][e]) == cn
    assert st["arrived"] > 0
