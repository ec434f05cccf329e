"""The C ABI library: it loads, exports every entry point include/manta.h
declares, its config struct matches the header's layout, and argument
validation fails cleanly -- all without a GPU (no call here reaches CUDA)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import nets
from paper_2007_03614_b300 import build as B
from paper_2007_03614_b300 import manta

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "manta.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return manta.load_library()


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"MANTA_API\s+[\w\s\*]+?\b(manta_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    assert set(names) == set(manta.EXPORTS)
    out = subprocess.check_output(["nm", "-D", "--defined-only", manta.LIB_PATH]).decode()
    exported = set(re.findall(r"\bT (manta_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)
    # nothing else leaks out under the manta_ prefix
    assert exported == set(names)


def test_config_layout_matches_header(lib):
    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "manta.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(manta_config), offsetof(manta_config, lc_x0_m),
         offsetof(manta_config, t0_step), offsetof(manta_config, seed), offsetof(manta_config, speed_sigma_frac),
         sizeof(manta_stats_t), offsetof(manta_stats_t, route_reads), offsetof(manta_stats_t, lc_cells_scanned));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(probe)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c])
        vals = list(map(int, subprocess.check_output([exe]).split()))
    M, S = manta.MantaConfig, manta.MantaStats
    assert vals == [C.sizeof(M), M.lc_x0_m.offset, M.t0_step.offset, M.seed.offset, M.speed_sigma_frac.offset,
                    C.sizeof(S), S.route_reads.offset, S.lc_cells_scanned.offset]


def test_default_config(lib):
    c = manta.default_config()
    assert c.dt == 0.5 and c.cell_m == 1.0 and c.veh_len_cells == 5 and c.horizon_cells == 256
    assert abs(c.alpha_lo - 0.05) < 1e-7 and abs(c.alpha_hi - 0.40) < 1e-7 and c.lc_x0_m == 1.0
    assert c.stop_dwell_steps == 4 and c.stats_window_steps == 600 and c.idm_textbook == 0
    assert c.speed_sigma_frac == 0.0


def _create(net, **cfg):
    lib = manta.load_library()
    conf = manta.default_config(**cfg)
    h = C.c_void_p()
    a = [np.ascontiguousarray(x) if x is not None else None for x in (
        net.edge_src, net.edge_dst, net.edge_lanes, net.edge_length_m, net.edge_speed_limit_mps, net.edge_class,
        net.node_type, net.node_cycle_steps, net.node_offset_steps, net.edge_green_start, net.edge_green_len,
        net.conn_lane_mask)]
    rc = lib.manta_create(len(net.node_type), len(net.edge_src), *[None if x is None else x.ctypes.data for x in a],
                          C.byref(conf), None, C.byref(h))
    return rc, lib.manta_last_error().decode()


@pytest.mark.parametrize("over,frag", [
    (dict(cell_m=2.0), "cell_m"), (dict(dt=0.0), "dt"), (dict(horizon_cells=4), "horizon"),
    (dict(n_classes=0), "n_classes"), (dict(a=[0.0] * 8), "class"), (dict(stop_dwell_steps=0), "stop_dwell"),
    (dict(t0_step=-1), "t0_step"), (dict(speed_sigma_frac=-0.1), "speed_sigma_frac"),
    (dict(speed_sigma_frac=1.5), "speed_sigma_frac"), (dict(speed_sigma_frac=float("nan")), "speed_sigma_frac")])
def test_create_rejects_bad_config(lib, over, frag):
    rc, msg = _create(nets.line(2), **over)
    assert rc == manta.E_INVALID and frag in msg


def test_create_rejects_bad_network(lib):
    net = nets.line(2)
    net.edge_dst = np.array([1, 7], np.int32)            # node out of range
    rc, msg = _create(net)
    assert rc == manta.E_INVALID and "edge 1" in msg
    net = nets.line(2)
    net.edge_lanes = np.array([1, 9], np.uint8)          # more than 8 lanes
    assert _create(net)[0] == manta.E_INVALID
    net = nets.line(2, node_type=[0, 2, 0])              # signal node without a cycle
    assert _create(net)[0] == manta.E_INVALID
    net = nets.line(2)
    net.edge_class = np.array([0, 5], np.uint8)          # class >= n_classes
    assert _create(net)[0] == manta.E_INVALID


def test_calls_on_null_handles_fail_cleanly(lib):
    """Every entry point that takes a simulation, graph or checkpoint rejects
    NULL with MANTA_E_INVALID (or a documented sentinel) without touching CUDA."""
    P = C.c_void_p
    out = P()
    lib.manta_step.argtypes = [P, C.c_int64]
    assert lib.manta_step(None, 1) == manta.E_INVALID
    assert lib.manta_load_trips(None, 0, None, None, None) == manta.E_INVALID
    assert lib.manta_set_lane_closure(None, 0, 0, 0, 1) == manta.E_INVALID
    assert lib.manta_set_variant(None, 0) == manta.E_INVALID
    assert lib.manta_get_variant(None) == -1
    assert lib.manta_autotune(None, 10, 1, None, None) == manta.E_INVALID
    assert lib.manta_graph_capture(None, 10, C.byref(out)) == manta.E_INVALID and not out.value
    assert lib.manta_graph_launch(None) == manta.E_INVALID
    assert lib.manta_checkpoint_save(None, C.byref(out)) == manta.E_INVALID and not out.value
    assert lib.manta_checkpoint_restore(None, None) == manta.E_INVALID
    assert lib.manta_checkpoint_step(None) == -1 and lib.manta_checkpoint_bytes(None) == 0
    assert lib.manta_tape_start(None, 10) == manta.E_INVALID
    assert lib.manta_tape_stop(None) == manta.E_INVALID
    n = C.c_int64()
    assert lib.manta_tape_copy(None, None, 0, C.byref(n)) == manta.E_INVALID
    assert lib.manta_adjoint(None, None, None, None, None) == manta.E_INVALID
    assert lib.manta_replay(None, None, None, None, None, None) == manta.E_INVALID
    # releasing NULL is a no-op
    lib.manta_graph_destroy(None)
    lib.manta_checkpoint_destroy(None)
    lib.manta_destroy(None)


def test_launch_shape_table(lib):
    n = lib.manta_variant_count()
    assert n >= 2
    t, b = C.c_int32(), C.c_int32()
    for v in range(n):
        assert lib.manta_variant_info(v, C.byref(t), C.byref(b)) == manta.OK
        assert t.value % 32 == 0 and b.value >= 1
    assert lib.manta_variant_info(n, C.byref(t), C.byref(b)) == manta.E_INVALID
    assert lib.manta_variant_info(-1, None, None) == manta.E_INVALID
