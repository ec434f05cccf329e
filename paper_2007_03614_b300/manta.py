"""Python binding of libmanta.so (argument marshalling only).

Every step of the simulation runs in the library's CUDA kernels; this module
only converts numpy arrays to pointers and statuses to exceptions.  It raises
if the native library is missing -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MANTA_LIBRARY may point at another build of the same library (e.g. a tuning variant).
LIB_PATH = os.environ.get("MANTA_LIBRARY") or os.path.join(_HERE, "libmanta.so")

OK, E_INVALID, E_ROUTE, E_STATE, E_OOM, E_CUDA, E_TIMEOUT, E_DEVICE = 0, -1, -2, -3, -4, -5, -6, -7
NODE_GREEN, NODE_STOP, NODE_SIGNAL = 0, 1, 2


class MantaConfig(C.Structure):
    _fields_ = [("dt", C.c_float), ("cell_m", C.c_float),
                ("veh_len_cells", C.c_int32), ("horizon_cells", C.c_int32), ("n_classes", C.c_int32),
                ("v0f", C.c_float * 8), ("T", C.c_float * 8), ("a", C.c_float * 8),
                ("b", C.c_float * 8), ("s0", C.c_float * 8),
                ("lc_x0_m", C.c_float), ("lc_len_scale_m", C.c_float),
                ("alpha_lo", C.c_float), ("alpha_hi", C.c_float),
                ("g_low", C.c_float), ("g_high", C.c_float), ("g_speed_split", C.c_float),
                ("stop_dwell_steps", C.c_int32), ("stop_v_eps", C.c_float),
                ("stats_window_steps", C.c_int32), ("n_stats_windows", C.c_int32),
                ("idm_textbook", C.c_int32),
                ("t0_step", C.c_int64), ("seed", C.c_uint64), ("speed_sigma_frac", C.c_float)]


class MantaStats(C.Structure):
    _fields_ = [("step", C.c_int64), ("loaded", C.c_int64), ("departed", C.c_int64),
                ("arrived", C.c_int64), ("on_network", C.c_int64), ("waiting", C.c_int64),
                ("vehicle_updates", C.c_uint64), ("cells_scanned", C.c_uint64),
                ("clamps", C.c_uint64), ("lane_changes", C.c_uint64),
                ("lc_evals", C.c_uint64), ("route_reads", C.c_uint64),
                ("lc_cells_scanned", C.c_uint64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


# Every entry point declared in include/manta.h.
EXPORTS = ("manta_default_config", "manta_create", "manta_load_trips", "manta_step", "manta_stats",
           "manta_edge_counters", "manta_snapshot", "manta_lane_map", "manta_lane_map_bytes",
           "manta_destroy", "manta_last_error", "manta_selftest_barrier_timeout", "manta_run_noalloc",
           "manta_phase_times", "manta_set_lane_closure", "manta_variant_count", "manta_variant_info",
           "manta_set_variant", "manta_get_variant", "manta_autotune", "manta_graph_capture",
           "manta_graph_launch", "manta_graph_destroy", "manta_checkpoint_save", "manta_checkpoint_restore",
           "manta_checkpoint_step", "manta_checkpoint_bytes", "manta_checkpoint_destroy", "manta_tape_start",
           "manta_tape_stop", "manta_tape_copy", "manta_adjoint", "manta_replay", "manta_place",
           "manta_debug_checks", "manta_debug_limit_map", "manta_debug_fail_nth")

_lib = None


class MantaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"manta status {status}: {msg}")
        self.status = status


_libs = {}


def load_library(path=None):
    """Load libmanta.so (build it first with paper_2007_03614_b300.build), or,
    with `path`, another build of the same library (a test variant); each
    path is loaded once."""
    global _lib
    path = path or LIB_PATH
    if path not in _libs:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run paper_2007_03614_b300.build.build()")
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.manta_default_config.argtypes = [C.POINTER(MantaConfig)]
        lib.manta_create.restype = C.c_int
        lib.manta_create.argtypes = [C.c_int32, C.c_int32] + [P] * 12 + [C.POINTER(MantaConfig), P, C.POINTER(P)]
        lib.manta_load_trips.restype = C.c_int
        lib.manta_load_trips.argtypes = [P, C.c_int64, P, P, P]
        lib.manta_step.restype = C.c_int
        lib.manta_step.argtypes = [P, C.c_int64]
        lib.manta_stats.restype = C.c_int
        lib.manta_stats.argtypes = [P, C.POINTER(MantaStats)]
        lib.manta_edge_counters.restype = C.c_int
        lib.manta_edge_counters.argtypes = [P, P, P, P, P, C.c_int32]
        lib.manta_snapshot.restype = C.c_int
        lib.manta_snapshot.argtypes = [P, C.c_int64, C.POINTER(C.c_int64), P, P, P, P, P, P, P]
        lib.manta_lane_map.restype = C.c_int
        lib.manta_lane_map.argtypes = [P, P, C.c_int64, C.POINTER(C.c_int64)]
        lib.manta_lane_map_bytes.restype = C.c_int64
        lib.manta_lane_map_bytes.argtypes = [P]
        lib.manta_destroy.argtypes = [P]
        lib.manta_last_error.restype = C.c_char_p
        lib.manta_run_noalloc.restype = C.c_int
        lib.manta_run_noalloc.argtypes = ([C.c_int32, C.c_int32] + [P] * 12 + [C.POINTER(MantaConfig), C.c_int64]
                                          + [P] * 3 + [C.c_int64, P, C.POINTER(MantaStats), C.c_int64,
                                                       C.POINTER(C.c_int64)] + [P] * 7)
        lib.manta_set_lane_closure.restype = C.c_int
        lib.manta_set_lane_closure.argtypes = [P, C.c_int32, C.c_int32, C.c_int64, C.c_int64]
        lib.manta_phase_times.restype = C.c_int
        lib.manta_phase_times.argtypes = [P, P]
        lib.manta_selftest_barrier_timeout.restype = C.c_int
        lib.manta_selftest_barrier_timeout.argtypes = [C.c_int32, P]
        lib.manta_variant_count.restype = C.c_int32
        lib.manta_variant_count.argtypes = []
        lib.manta_variant_info.restype = C.c_int
        lib.manta_variant_info.argtypes = [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        lib.manta_set_variant.restype = C.c_int
        lib.manta_set_variant.argtypes = [P, C.c_int32]
        lib.manta_get_variant.restype = C.c_int32
        lib.manta_get_variant.argtypes = [P]
        lib.manta_autotune.restype = C.c_int
        lib.manta_autotune.argtypes = [P, C.c_int64, C.c_int32, C.POINTER(C.c_int32), P]
        lib.manta_graph_capture.restype = C.c_int
        lib.manta_graph_capture.argtypes = [P, C.c_int64, C.POINTER(P)]
        lib.manta_graph_launch.restype = C.c_int
        lib.manta_graph_launch.argtypes = [P]
        lib.manta_graph_destroy.argtypes = [P]
        lib.manta_checkpoint_save.restype = C.c_int
        lib.manta_checkpoint_save.argtypes = [P, C.POINTER(P)]
        lib.manta_checkpoint_restore.restype = C.c_int
        lib.manta_checkpoint_restore.argtypes = [P, P]
        lib.manta_checkpoint_step.restype = C.c_int64
        lib.manta_checkpoint_step.argtypes = [P]
        lib.manta_checkpoint_bytes.restype = C.c_int64
        lib.manta_checkpoint_bytes.argtypes = [P]
        lib.manta_checkpoint_destroy.argtypes = [P]
        lib.manta_tape_start.restype = C.c_int
        lib.manta_tape_start.argtypes = [P, C.c_int64]
        lib.manta_tape_stop.restype = C.c_int
        lib.manta_tape_stop.argtypes = [P]
        lib.manta_tape_copy.restype = C.c_int
        lib.manta_tape_copy.argtypes = [P, P, C.c_int64, C.POINTER(C.c_int64)]
        lib.manta_adjoint.restype = C.c_int
        lib.manta_adjoint.argtypes = [P, P, P, P, P]
        lib.manta_replay.restype = C.c_int
        lib.manta_replay.argtypes = [P, P, P, P, P, P]
        lib.manta_place.restype = C.c_int
        lib.manta_place.argtypes = [P, C.c_int64, P, P, P, P, P]
        lib.manta_debug_checks.restype = C.c_int32
        lib.manta_debug_checks.argtypes = []
        lib.manta_debug_limit_map.restype = C.c_int
        lib.manta_debug_limit_map.argtypes = [P, C.c_int64]
        lib.manta_debug_fail_nth.restype = C.c_int
        lib.manta_debug_fail_nth.argtypes = [C.c_int32, C.c_int64]
        _libs[path] = lib
    if path == LIB_PATH:
        _lib = _libs[path]
    return _libs[path]


def _check(rc, lib=None):
    if rc != OK:
        raise MantaError(rc, (lib or _lib).manta_last_error().decode())


def default_config(**over) -> MantaConfig:
    lib = load_library()
    c = MantaConfig()
    lib.manta_default_config(C.byref(c))
    for k, v in over.items():
        if isinstance(v, (list, tuple, np.ndarray)):
            arr = getattr(c, k)
            for i in range(8):
                arr[i] = float(v[i]) if i < len(v) else float(v[-1])
        else:
            setattr(c, k, v)
    return c


def _torch():
    import torch
    return torch


def _p(a):
    return None if a is None else a.ctypes.data


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)     # torch.cuda.Stream


# one record of the event tape (manta_tape_record in include/manta.h)
TAPE_DTYPE = np.dtype([("x", np.float32), ("v", np.float32), ("s", np.float32), ("vL", np.float32),
                       ("bnd", np.float32), ("lim", np.float32), ("cells", np.uint32), ("flags", np.uint32),
                       ("sample", np.uint32), ("pad", np.uint32)])


class Sim:
    """One simulation on the current CUDA device (see include/manta.h)."""

    def __init__(self, net, stream=None, library=None, **cfg):
        lib = load_library(library)
        self._lib = lib
        self.cfg = default_config(**cfg)
        keep = []

        def arr(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(np.asarray(a, dtype=dt))
            keep.append(a)
            return a

        self.n_edges = int(len(net.edge_src))
        self.n_nodes = int(len(net.node_type))
        h = C.c_void_p()
        rc = lib.manta_create(self.n_nodes, self.n_edges,
                              _p(arr(net.edge_src, np.int32)), _p(arr(net.edge_dst, np.int32)),
                              _p(arr(net.edge_lanes, np.uint8)), _p(arr(net.edge_length_m, np.float32)),
                              _p(arr(net.edge_speed_limit_mps, np.float32)), _p(arr(net.edge_class, np.uint8)),
                              _p(arr(net.node_type, np.uint8)), _p(arr(net.node_cycle_steps, np.int32)),
                              _p(arr(net.node_offset_steps, np.int32)), _p(arr(net.edge_green_start, np.int16)),
                              _p(arr(net.edge_green_len, np.int16)), _p(arr(net.conn_lane_mask, np.uint32)),
                              C.byref(self.cfg), _stream_handle(stream), C.byref(h))
        _check(rc, lib)
        self._h = h
        self.n_trips = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.manta_destroy(self._h)
            self._h = None

    __del__ = close

    def load_trips(self, route_off, route_edges, depart_time_s):
        ro = np.ascontiguousarray(route_off, dtype=np.int64)
        re = np.ascontiguousarray(route_edges, dtype=np.int32)
        dt = np.ascontiguousarray(depart_time_s, dtype=np.float32)
        _check(self._lib.manta_load_trips(self._h, len(dt), _p(ro), _p(re), _p(dt)), self._lib)
        self.n_trips = len(dt)

    def place(self, trip, route_pos, lane, x, v):
        """Put waiting trips on the network at (route position, lane, x, v)
        before the first step (manta_place)."""
        a = [np.ascontiguousarray(trip, np.int64), np.ascontiguousarray(route_pos, np.int32),
             np.ascontiguousarray(lane, np.uint8), np.ascontiguousarray(x, np.float32),
             np.ascontiguousarray(v, np.float32)]
        _check(self._lib.manta_place(self._h, len(a[0]), *[_p(q) for q in a]), self._lib)

    def debug_limit_map(self, n_bytes):
        """Test hook of the bounds-checked build (manta_debug_limit_map)."""
        _check(self._lib.manta_debug_limit_map(self._h, int(n_bytes)), self._lib)

    def set_lane_closure(self, edge, lane, k0, k1):
        _check(self._lib.manta_set_lane_closure(self._h, int(edge), int(lane), int(k0), int(k1)), self._lib)

    def step(self, n=1):
        _check(self._lib.manta_step(self._h, int(n)), self._lib)

    def stats(self) -> dict:
        s = MantaStats()
        _check(self._lib.manta_stats(self._h, C.byref(s)), self._lib)
        return s.as_dict()

    def edge_counters(self, window=0) -> dict:
        E = self.n_edges
        out = dict(entries=np.zeros(E, np.uint32), exits=np.zeros(E, np.uint32),
                   speed_sum=np.zeros(E, np.uint64), speed_cnt=np.zeros(E, np.uint32))
        _check(self._lib.manta_edge_counters(self._h, _p(out["entries"]), _p(out["exits"]),
                                             _p(out["speed_sum"]), _p(out["speed_cnt"]), int(window)), self._lib)
        return out

    def snapshot(self) -> dict:
        n = max(self.n_trips, 1)
        out = dict(x=np.zeros(n, np.float32), v=np.zeros(n, np.float32), edge=np.zeros(n, np.int32),
                   lane=np.zeros(n, np.uint8), id=np.zeros(n, np.uint32), dwell=np.zeros(n, np.uint8),
                   route_pos=np.zeros(n, np.int32))
        cnt = C.c_int64()
        _check(self._lib.manta_snapshot(self._h, n, C.byref(cnt), *[_p(out[k]) for k in
                                                                   ("x", "v", "edge", "lane", "id", "dwell",
                                                                    "route_pos")]), self._lib)
        return {k: a[:cnt.value] for k, a in out.items()}

    def phase_times_ms(self) -> np.ndarray:
        out = np.zeros(4, np.float64)
        _check(self._lib.manta_phase_times(self._h, _p(out)), self._lib)
        return out

    @property
    def variant(self) -> int:
        return int(self._lib.manta_get_variant(self._h))

    @variant.setter
    def variant(self, v):
        _check(self._lib.manta_set_variant(self._h, int(v)), self._lib)

    def autotune(self, trial_steps=60, rounds=1):
        """Times every launch shape on the live run (which advances by
        rounds x shapes x trial_steps steps) and keeps the one with the least
        time per vehicle update; returns (chosen shape, score of every shape
        in ms per million vehicle updates)."""
        n = int(self._lib.manta_variant_count())
        ms = np.zeros(n, np.float32)
        ch = C.c_int32()
        _check(self._lib.manta_autotune(self._h, int(trial_steps), int(rounds), C.byref(ch), _p(ms)), self._lib)
        return ch.value, ms

    def checkpoint(self) -> "Checkpoint":
        return Checkpoint(self)

    def restore(self, ckpt: "Checkpoint"):
        _check(self._lib.manta_checkpoint_restore(self._h, ckpt._h), self._lib)

    def tape_start(self, n_steps):
        _check(self._lib.manta_tape_start(self._h, int(n_steps)), self._lib)

    def tape_stop(self):
        _check(self._lib.manta_tape_stop(self._h), self._lib)

    def tape_copy(self, n_steps) -> dict:
        """The recorded tape as arrays of shape (n_steps, n_trips)."""
        N = max(self.n_trips, 1)
        rec = np.zeros(int(n_steps) * N, dtype=TAPE_DTYPE)
        n = C.c_int64()
        _check(self._lib.manta_tape_copy(self._h, rec.ctypes.data, rec.size, C.byref(n)), self._lib)
        return {k: rec[k].reshape(int(n_steps), N) for k in TAPE_DTYPE.names}

    def adjoint(self, seed, lam_x, lam_v, grad):
        """Reverse sweep over the recorded tape segment; arguments are CUDA
        float64 tensors (see manta_adjoint in include/manta.h)."""
        for t in (seed, lam_x, lam_v, grad):
            assert t.is_cuda and t.dtype == _torch().float64 and t.is_contiguous()
        _check(self._lib.manta_adjoint(self._h, seed.data_ptr(), lam_x.data_ptr(), lam_v.data_ptr(),
                                       grad.data_ptr()), self._lib)

    def replay(self, theta, x, v, present, sums):
        """Frozen-event replay of the recorded segment with parameters theta
        (5 x n_classes, host); x, v, sums CUDA float64, present CUDA uint8."""
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
        for t in (x, v, sums):
            assert t.is_cuda and t.dtype == _torch().float64 and t.is_contiguous()
        assert present.is_cuda and present.dtype == _torch().uint8
        _check(self._lib.manta_replay(self._h, th.ctypes.data, x.data_ptr(), v.data_ptr(), present.data_ptr(),
                                      sums.data_ptr()), self._lib)

    def graph(self, n_steps) -> "Graph":
        return Graph(self, n_steps)

    def lane_map(self) -> np.ndarray:
        nb = int(self._lib.manta_lane_map_bytes(self._h))
        buf = np.zeros(max(nb, 1), np.uint8)
        cnt = C.c_int64()
        _check(self._lib.manta_lane_map(self._h, _p(buf), buf.size, C.byref(cnt)), self._lib)
        return buf[:cnt.value]


def variants() -> list:
    """Launch shapes of the step kernel as (threads per block, min blocks per SM)."""
    lib = load_library()
    out = []
    for v in range(lib.manta_variant_count()):
        t, b = C.c_int32(), C.c_int32()
        _check(lib.manta_variant_info(v, C.byref(t), C.byref(b)))
        out.append((t.value, b.value))
    return out


class Graph:
    """Captured launches advancing a Sim by n_steps per replay (include/manta.h)."""

    def __init__(self, sim, n_steps):
        self._lib = sim._lib
        self.sim = sim
        self.n_steps = int(n_steps)
        h = C.c_void_p()
        _check(self._lib.manta_graph_capture(sim._h, self.n_steps, C.byref(h)), self._lib)
        self._h = h

    def launch(self, times=1):
        for _ in range(times):
            _check(self._lib.manta_graph_launch(self._h), self._lib)

    def close(self):
        if self._h:
            self._lib.manta_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Checkpoint:
    """Saved device state of a Sim (include/manta.h); destroy before the Sim."""

    def __init__(self, sim):
        self._lib = sim._lib
        h = C.c_void_p()
        _check(self._lib.manta_checkpoint_save(sim._h, C.byref(h)), self._lib)
        self._h = h

    @property
    def step(self) -> int:
        return int(self._lib.manta_checkpoint_step(self._h))

    @property
    def nbytes(self) -> int:
        return int(self._lib.manta_checkpoint_bytes(self._h))

    def close(self):
        if self._h:
            self._lib.manta_checkpoint_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_barrier_timeout(limit_ms=100, stream=None) -> int:
    """Runs the bounded-wait self test; returns the status (E_TIMEOUT expected)."""
    lib = load_library()
    return int(lib.manta_selftest_barrier_timeout(int(limit_ms), _stream_handle(stream)))


def run_noalloc(net, trips, n_steps, stream=None, **cfg):
    """A whole small simulation with no device allocation (manta_run_noalloc):
    returns (stats, snapshot) exactly as Sim would."""
    lib = load_library()
    conf = default_config(**cfg)
    keep = []

    def arr(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(np.asarray(a, dtype=dt))
        keep.append(a)
        return a

    n = max(trips.n_trips, 1)
    out = dict(x=np.zeros(n, np.float32), v=np.zeros(n, np.float32), edge=np.zeros(n, np.int32),
               lane=np.zeros(n, np.uint8), id=np.zeros(n, np.uint32), dwell=np.zeros(n, np.uint8),
               route_pos=np.zeros(n, np.int32))
    st = MantaStats()
    cnt = C.c_int64()
    rc = lib.manta_run_noalloc(
        int(len(net.node_type)), int(len(net.edge_src)),
        _p(arr(net.edge_src, np.int32)), _p(arr(net.edge_dst, np.int32)), _p(arr(net.edge_lanes, np.uint8)),
        _p(arr(net.edge_length_m, np.float32)), _p(arr(net.edge_speed_limit_mps, np.float32)),
        _p(arr(net.edge_class, np.uint8)), _p(arr(net.node_type, np.uint8)), _p(arr(net.node_cycle_steps, np.int32)),
        _p(arr(net.node_offset_steps, np.int32)), _p(arr(net.edge_green_start, np.int16)),
        _p(arr(net.edge_green_len, np.int16)), _p(arr(net.conn_lane_mask, np.uint32)), C.byref(conf),
        int(trips.n_trips), _p(arr(trips.route_off, np.int64)), _p(arr(trips.route_edges, np.int32)),
        _p(arr(trips.depart_time_s, np.float32)), int(n_steps), _stream_handle(stream), C.byref(st), n,
        C.byref(cnt), *[_p(out[k]) for k in ("x", "v", "edge", "lane", "id", "dwell", "route_pos")])
    _check(rc)
    return st.as_dict(), {k: a[:cnt.value] for k, a in out.items()}


def debug_checks(library=None) -> bool:
    """Whether the library build checks device write indices (manta_debug_checks)."""
    return bool(load_library(library).manta_debug_checks())


def debug_fail_nth(kind, nth, library=None):
    """Host-side fault injection (manta_debug_fail_nth): kind 0 device
    allocations, 1 host-to-device copies; nth = 0 turns it off."""
    lib = load_library(library)
    _check(lib.manta_debug_fail_nth(int(kind), int(nth)), lib)
