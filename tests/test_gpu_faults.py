"""Failure detection without a GPU fault.

- The bounds-checked build (index checks on every device write of the step
  kernel) gives the oracle's results bit for bit; with the lane-map capacity
  it checks against lowered below the buffer's real size, an in-bounds write
  fails its check: the launch ends at the next grid barrier, the host gets
  MANTA_E_DEVICE naming the site, later steps are refused, and the CUDA
  context keeps working.
- Host-side fault injection: making the nth device allocation or the nth
  host-to-device copy fail, for every n that manta_create and
  manta_load_trips reach, gives MANTA_E_OOM / MANTA_E_CUDA and a clean
  manta_destroy (device memory returns to where it was).
"""
import numpy as np
import pytest

import nets
from oracle import oracle as O
from paper_2007_03614_b300 import manta, synth
from paper_2007_03614_b300.build import build, build_variant
from test_gpu_parity import _compare, _compare_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build()
    manta.load_library()


def test_checked_build_matches_the_oracle():
    lib = build_variant("check")
    assert manta.debug_checks(lib) and not manta.debug_checks()
    net = synth.tiny_network()
    tr = synth.tiny_trips(net)
    o = O.OracleSim(net)
    g = manta.Sim(net, library=lib)
    nets.load(o, tr)
    nets.load(g, tr)
    for k in range(0, 900, 150):
        o.step(150)
        g.step(150)
        _compare(o, g, f"checked build step {k + 150}")
    _compare_all(o, g, windows=(0, 1))
    g.close()


def test_index_check_fails_in_bounds_and_the_context_survives():
    lib = build_variant("check")
    net = synth.tiny_network()
    tr = synth.tiny_trips(net)
    g = manta.Sim(net, library=lib)
    nets.load(g, tr)
    g.debug_limit_map(g.lane_map().size // 2)       # the upper half of each buffer is now "out of bounds"
    g.step(300)
    with pytest.raises(manta.MantaError) as ei:
        g.stats()
    assert ei.value.status == manta.E_DEVICE and "site" in str(ei.value)
    with pytest.raises(manta.MantaError) as ei:
        g.step(1)
    assert ei.value.status == manta.E_STATE
    g.close()
    # the context is fine: a new simulation on the same library runs bit for bit
    o = O.OracleSim(net)
    g2 = manta.Sim(net, library=lib)
    nets.load(o, tr)
    nets.load(g2, tr)
    o.step(300)
    g2.step(300)
    _compare_all(o, g2)
    g2.close()


def _create_and_load(net, tr):
    g = None
    try:
        g = manta.Sim(net)
        nets.load(g, tr)
        g.step(5)
        g.stats()
        return None
    except manta.MantaError as e:
        return e.status
    finally:
        if g is not None:
            g.close()


@pytest.mark.parametrize("kind,expect", [(0, manta.E_OOM), (1, manta.E_CUDA)])
def test_host_fault_injection_every_allocation_and_copy(kind, expect):
    import torch
    net = synth.tiny_network()
    tr = synth.tiny_trips(net, n_trips=200)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    seen = 0
    for nth in range(1, 400):
        manta.debug_fail_nth(kind, nth)
        st = _create_and_load(net, tr)
        manta.debug_fail_nth(kind, 0)
        if st is None:
            break                     # nth is past the last allocation / copy: the run succeeded
        assert st == expect, (nth, st)
        seen += 1
    else:
        raise AssertionError("fault injection never ran out of sites")
    assert seen > 10
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)
    # and nothing is left armed: a plain run works
    assert _create_and_load(net, tr) is None
