"""manta_run_noalloc: a whole small simulation whose device state lives in the
library's static arena instead of cudaMalloc'd memory, for callers that cannot
allocate device memory (a host application whose device memory is wholly held
by its own pool allocator, or a loop that must not stall on the driver's
allocator).  Its results must equal those of the allocating entry points bit
for bit, on two calls in a row (the second call reuses the arena the first one
left behind), and after a different workload has dirtied the arena.

Collected last on purpose: a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_2007_03614_b300 import manta, synth
from paper_2007_03614_b300.build import build

pytestmark = pytest.mark.gpu


def _allocating(net, tr, n_steps, **cfg):
    g = manta.Sim(net, **cfg)
    g.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
    g.step(n_steps)
    st, sn = g.stats(), g.snapshot()
    g.close()
    return st, sn


def _same(a, b):
    sa, na = a
    sb, nb = b
    assert sa == sb
    for key in ("id", "edge", "lane", "dwell", "route_pos"):
        assert np.array_equal(na[key], nb[key]), key
    for key in ("x", "v"):
        assert np.array_equal(na[key].view(np.uint32), nb[key].view(np.uint32)), key


def test_no_alloc_matches_allocating_path_twice():
    import torch
    assert torch.cuda.is_available()
    build()
    net = synth.tiny_network()
    tr = synth.tiny_trips(net, n_trips=1000)
    ref = _allocating(net, tr, 700)
    assert ref[0]["on_network"] > 0
    first = manta.run_noalloc(net, tr, 700)
    _same(first, ref)
    second = manta.run_noalloc(net, tr, 700)     # same arena, left dirty by the first call
    _same(second, ref)
    # a different workload in between must not leak into the next call
    tr2 = synth.tiny_trips(net, n_trips=400, seed=9)
    _same(manta.run_noalloc(net, tr2, 300, seed=5), _allocating(net, tr2, 300, seed=5))


def test_no_alloc_dirty_arena_with_per_driver_limits():
    """Per-driver speed limits (Section IV-B) and a non-default seed, on an
    arena left dirty by a different, larger workload: still bit for bit the
    allocating path.  (The entry point takes no lane closures; the closure
    windows it uploads are empty on every call.)"""
    import torch
    assert torch.cuda.is_available()
    build()
    net = synth.tiny_network()
    manta.run_noalloc(net, synth.tiny_trips(net, n_trips=1000, seed=3), 900, seed=11)
    tr = synth.tiny_trips(net, n_trips=600, seed=21)
    cfg = dict(speed_sigma_frac=0.05, seed=77)
    a = manta.run_noalloc(net, tr, 500, **cfg)
    b = _allocating(net, tr, 500, **cfg)
    assert b[0]["on_network"] > 0
    _same(a, b)


def test_no_alloc_rejects_workloads_beyond_the_arena():
    build()
    net = synth.lattice(60, 60, arterial_every=1, len_median_m=100.0, len_sigma=0.0, len_min_m=100.0,
                        len_max_m=100.0, lanes=(2, 2, 2))
    tr = synth.tiny_trips(net, n_trips=100)
    with pytest.raises(manta.MantaError) as ei:
        manta.run_noalloc(net, tr, 10)
    assert ei.value.status == manta.E_INVALID and "MiB static arena" in str(ei.value)
