"""Python binding of the CPU oracle (manta_oracle.c).

TEST INFRASTRUCTURE: only tests/, ``__graft_entry__.smoke()`` and bench.py's
cpu_baseline / reference legs may import this module.  It shares no code with
the CUDA library or its binding; configuration is passed as a plain dict.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "manta_oracle.c")
_LIB = os.path.join(_HERE, "libmanta_oracle.so")

# Strict binary32: no contraction into FMA, no fast-math, SSE2 scalar math.
CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
          "-msse2", "-mfpmath=sse", "-fno-strict-aliasing"]


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", *CFLAGS, "-o", _LIB, _SRC, "-lm"])
    return _LIB


class OracleConfig(C.Structure):
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


class OracleStats(C.Structure):
    _fields_ = [("step", C.c_int64), ("loaded", C.c_int64), ("departed", C.c_int64),
                ("arrived", C.c_int64), ("on_network", C.c_int64), ("waiting", C.c_int64),
                ("vehicle_updates", C.c_uint64), ("cells_scanned", C.c_uint64),
                ("clamps", C.c_uint64), ("lane_changes", C.c_uint64),
                ("lc_evals", C.c_uint64), ("route_reads", C.c_uint64),
                ("lc_cells_scanned", C.c_uint64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


DEFAULTS = dict(dt=0.5, cell_m=1.0, veh_len_cells=5, horizon_cells=256, n_classes=3,
                v0f=[1.0] * 8, T=[1.5] * 8, a=[1.0] * 8, b=[2.0] * 8, s0=[2.0] * 8,
                lc_x0_m=1.0, lc_len_scale_m=1.0, alpha_lo=0.05, alpha_hi=0.40,
                g_low=3.0, g_high=7.5, g_speed_split=11.176, stop_dwell_steps=4, stop_v_eps=0.1,
                stats_window_steps=600, n_stats_windows=96, idm_textbook=0, t0_step=0, seed=1,
                speed_sigma_frac=0.0)


def make_config(**over) -> OracleConfig:
    d = dict(DEFAULTS)
    d.update(over)
    c = OracleConfig()
    for k, v in d.items():
        if isinstance(v, (list, tuple, np.ndarray)):
            arr = getattr(c, k)
            for i in range(8):
                arr[i] = float(v[i]) if i < len(v) else float(v[-1])
        else:
            setattr(c, k, v)
    return c


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        lib.oracle_create.restype = P
        lib.oracle_create.argtypes = [C.c_int32, C.c_int32] + [P] * 12 + [C.POINTER(OracleConfig), C.c_char_p, C.c_int]
        lib.oracle_load_trips.restype = C.c_int
        lib.oracle_load_trips.argtypes = [P, C.c_int64, P, P, P, C.c_char_p, C.c_int]
        lib.oracle_step.restype = C.c_int
        lib.oracle_step.argtypes = [P, C.c_int64, C.c_char_p, C.c_int]
        lib.oracle_stats.argtypes = [P, C.POINTER(OracleStats)]
        lib.oracle_edge_counters.argtypes = [P, P, P, P, P, C.c_int32]
        lib.oracle_snapshot.restype = C.c_int64
        lib.oracle_snapshot.argtypes = [P, C.c_int64, P, P, P, P, P, P, P]
        lib.oracle_lane_map.restype = C.c_int64
        lib.oracle_lane_map.argtypes = [P, P, C.c_int64]
        lib.oracle_map_bytes.restype = C.c_int64
        lib.oracle_map_bytes.argtypes = [P]
        lib.oracle_edge_cells.restype = C.c_int32
        lib.oracle_edge_cells.argtypes = [P, C.c_int32]
        lib.oracle_permit.restype = C.c_uint32
        lib.oracle_permit.argtypes = [P, C.c_int32]
        lib.oracle_place.restype = C.c_int
        lib.oracle_place.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, C.c_float, C.c_float]
        lib.oracle_place_many.restype = C.c_int64
        lib.oracle_place_many.argtypes = [P, C.c_int64, P, P, P, P, P]
        lib.oracle_check.restype = C.c_int
        lib.oracle_check.argtypes = [P, C.c_char_p, C.c_int]
        lib.oracle_destroy.argtypes = [P]
        lib.oracle_set_tape.argtypes = [P, C.c_int64, C.c_int64] + [P] * 9
        lib.oracle_set_lane_closure.restype = C.c_int
        lib.oracle_set_lane_closure.argtypes = [P, C.c_int32, C.c_int32, C.c_int64, C.c_int64]
        lib.oracle_splitmix64.restype = C.c_uint64
        lib.oracle_splitmix64.argtypes = [C.c_uint64]
        lib.oracle_rng_u.restype = C.c_float
        lib.oracle_rng_u.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_uint64]
        lib.oracle_rng_n.restype = C.c_float
        lib.oracle_rng_n.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_uint64]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class OracleError(RuntimeError):
    pass


class OracleSim:
    """The oracle simulation: same calls, same semantics as the CUDA library."""

    def __init__(self, net, **cfg):
        lib = _load()
        self._lib = lib
        self.cfg = make_config(**cfg)
        self._keep = []

        def arr(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(np.asarray(a, dtype=dt))
            self._keep.append(a)
            return a

        self.n_edges = int(len(net.edge_src))
        self.n_nodes = int(len(net.node_type))
        err = C.create_string_buffer(256)
        h = lib.oracle_create(self.n_nodes, self.n_edges,
                              _p(arr(net.edge_src, np.int32)), _p(arr(net.edge_dst, np.int32)),
                              _p(arr(net.edge_lanes, np.uint8)), _p(arr(net.edge_length_m, np.float32)),
                              _p(arr(net.edge_speed_limit_mps, np.float32)), _p(arr(net.edge_class, np.uint8)),
                              _p(arr(net.node_type, np.uint8)), _p(arr(net.node_cycle_steps, np.int32)),
                              _p(arr(net.node_offset_steps, np.int32)), _p(arr(net.edge_green_start, np.int16)),
                              _p(arr(net.edge_green_len, np.int16)),
                              _p(arr(net.conn_lane_mask, np.uint32)), C.byref(self.cfg), err, 256)
        self._keep = []
        if not h:
            raise OracleError(err.value.decode())
        self._h = h
        self.n_trips = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_destroy(self._h)
            self._h = None

    __del__ = close

    def load_trips(self, route_off, route_edges, depart_time_s):
        ro = np.ascontiguousarray(route_off, dtype=np.int64)
        re = np.ascontiguousarray(route_edges, dtype=np.int32)
        dt = np.ascontiguousarray(depart_time_s, dtype=np.float32)
        err = C.create_string_buffer(256)
        rc = self._lib.oracle_load_trips(self._h, len(dt), _p(ro), _p(re), _p(dt), err, 256)
        if rc != 0:
            raise OracleError(f"load_trips {rc}: {err.value.decode()}")
        self.n_trips = len(dt)

    def step(self, n=1):
        err = C.create_string_buffer(256)
        rc = self._lib.oracle_step(self._h, int(n), err, 256)
        if rc != 0:
            raise OracleError(f"step {rc}: {err.value.decode()}")

    def stats(self) -> dict:
        s = OracleStats()
        self._lib.oracle_stats(self._h, C.byref(s))
        return s.as_dict()

    def snapshot(self) -> dict:
        n = max(self.n_trips, 1)
        out = dict(x=np.zeros(n, np.float32), v=np.zeros(n, np.float32), edge=np.zeros(n, np.int32),
                   lane=np.zeros(n, np.uint8), id=np.zeros(n, np.uint32), dwell=np.zeros(n, np.uint8),
                   route_pos=np.zeros(n, np.int32))
        c = self._lib.oracle_snapshot(self._h, n, *[_p(out[k]) for k in
                                                    ("x", "v", "edge", "lane", "id", "dwell", "route_pos")])
        return {k: a[:c] for k, a in out.items()}

    def lane_map(self) -> np.ndarray:
        """Current lane map: edges in id order, lanes in order, C_e bytes each."""
        buf = np.zeros(int(self._lib.oracle_map_bytes(self._h)), np.uint8)
        n = self._lib.oracle_lane_map(self._h, _p(buf), buf.size)
        return buf[:n]

    def edge_cells(self) -> np.ndarray:
        return np.array([self._lib.oracle_edge_cells(self._h, e) for e in range(self.n_edges)], np.int32)

    def edge_counters(self, window=0) -> dict:
        E = self.n_edges
        out = dict(entries=np.zeros(E, np.uint32), exits=np.zeros(E, np.uint32),
                   speed_sum=np.zeros(E, np.uint64), speed_cnt=np.zeros(E, np.uint32))
        self._lib.oracle_edge_counters(self._h, _p(out["entries"]), _p(out["exits"]), _p(out["speed_sum"]),
                                       _p(out["speed_cnt"]), int(window))
        return out

    def permit(self, node) -> int:
        return int(self._lib.oracle_permit(self._h, int(node)))

    def place(self, trip, route_pos, lane, x, v):
        rc = self._lib.oracle_place(self._h, int(trip), int(route_pos), int(lane), float(x), float(v))
        if rc != 0:
            raise OracleError(f"place {rc}")

    def place_many(self, trip, route_pos, lane, x, v):
        """place() for every placement, in order."""
        a = [np.ascontiguousarray(trip, np.int64), np.ascontiguousarray(route_pos, np.int32),
             np.ascontiguousarray(lane, np.uint8), np.ascontiguousarray(x, np.float32),
             np.ascontiguousarray(v, np.float32)]
        rc = self._lib.oracle_place_many(self._h, len(a[0]), *[_p(q) for q in a])
        if rc != 0:
            raise OracleError(f"place_many: placement {-1 - rc} failed")

    def set_lane_closure(self, edge, lane, k0, k1):
        rc = self._lib.oracle_set_lane_closure(self._h, int(edge), int(lane), int(k0), int(k1))
        if rc != 0:
            raise OracleError(f"set_lane_closure {rc}")

    def record_tape(self, n_steps):
        """Record the event tape of the next n_steps steps (oracle_set_tape);
        returns the dict of arrays, shape (n_steps, n_trips), filled as the
        steps run."""
        T, N = int(n_steps), max(self.n_trips, 1)
        st = self.stats()["step"]
        tape = {k: np.zeros((T, N), np.float32) for k in ("x", "v", "s", "vL", "bnd", "lim")}
        tape["C"] = np.zeros((T, N), np.int32)
        tape["flags"] = np.zeros((T, N), np.int32)
        tape["sample"] = np.full((T, N), -1, np.int64)
        tape["k0"] = st
        self._tape = tape
        self._lib.oracle_set_tape(self._h, st, T, *[_p(tape[k]) for k in
                                                   ("x", "v", "s", "vL", "bnd", "lim", "C", "flags", "sample")])
        return tape

    def stop_tape(self):
        self._lib.oracle_set_tape(self._h, 0, 0, *([None] * 9))

    def check(self):
        msg = C.create_string_buffer(256)
        rc = self._lib.oracle_check(self._h, msg, 256)
        if rc != 0:
            raise OracleError(f"invariant {rc}: {msg.value.decode()}")


def splitmix64(x: int) -> int:
    return int(_load().oracle_splitmix64(x))


def rng_u(seed, vid, k, stream) -> float:
    return float(_load().oracle_rng_u(seed, vid, k, stream))


def rng_n(seed, vid, k, s) -> float:
    return float(_load().oracle_rng_n(seed, vid, k, s))
