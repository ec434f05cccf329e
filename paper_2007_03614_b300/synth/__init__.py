"""Seeded synthetic road networks and trip tables (input generation only).

Stands in for the paper's data pipeline -- the OSM street network (Section II-A),
the TAZ-level demand with nodes sampled uniformly inside each zone (Section II-B)
and the shortest-path routing computed only for the OD pairs needed (Section II-C).
None of the simulation's arithmetic lives here; both the CPU oracle and the CUDA
library consume the arrays this module returns.

``Network`` and ``Trips`` are plain containers of numpy arrays whose names match
the arguments of ``manta_create`` / ``manta_load_trips``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libmanta_synth.so")


def build(force: bool = False) -> str:
    """Compile synth.c into an in-tree shared library (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-o", _LIB, _SRC, "-lm"])
    return _LIB


class _Net(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_edges", C.c_int32),
                ("edge_src", C.POINTER(C.c_int32)), ("edge_dst", C.POINTER(C.c_int32)),
                ("edge_lanes", C.POINTER(C.c_uint8)), ("edge_class", C.POINTER(C.c_uint8)),
                ("edge_length_m", C.POINTER(C.c_float)), ("edge_speed_mps", C.POINTER(C.c_float)),
                ("node_type", C.POINTER(C.c_uint8)),
                ("node_cycle", C.POINTER(C.c_int32)), ("node_offset", C.POINTER(C.c_int32)),
                ("edge_green_start", C.POINTER(C.c_int16)), ("edge_green_len", C.POINTER(C.c_int16)),
                ("n_conn", C.c_int64), ("conn_lane_mask", C.POINTER(C.c_uint32)),
                ("node_i", C.POINTER(C.c_int32)), ("node_j", C.POINTER(C.c_int32)),
                ("edge_dir", C.POINTER(C.c_uint8)), ("node_trip_ok", C.POINTER(C.c_uint8))]


class _LatticeParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32),
                ("arterial_every", C.c_int32), ("freeway_every", C.c_int32),
                ("local_keep", C.c_double),
                ("len_median_m", C.c_double), ("len_sigma", C.c_double),
                ("len_min_m", C.c_double), ("len_max_m", C.c_double),
                ("speed_mps", C.c_float * 3), ("lanes", C.c_uint8 * 3),
                ("signal_cycle_steps", C.c_int32), ("signal_green_steps", C.c_int32),
                ("signals_at", C.c_int32), ("all_stop", C.c_int32), ("limited_access", C.c_int32),
                ("seed", C.c_uint64)]


class _Trips(C.Structure):
    _fields_ = [("n_trips", C.c_int64),
                ("origin", C.POINTER(C.c_int32)), ("dest", C.POINTER(C.c_int32)),
                ("depart_time_s", C.POINTER(C.c_float)),
                ("route_off", C.POINTER(C.c_int64)), ("route_edges", C.POINTER(C.c_int32)),
                ("n_route_edges", C.c_int64), ("n_unroutable", C.c_int64)]


class _TripParams(C.Structure):
    _fields_ = [("n_trips", C.c_int64), ("od_model", C.c_int32),
                ("zones_x", C.c_int32), ("zones_y", C.c_int32), ("pool_per_zone", C.c_int32),
                ("spacing_km", C.c_double), ("beta_km", C.c_double), ("zone_mass_sigma", C.c_double),
                ("depart_model", C.c_int32),
                ("t_lo_s", C.c_double), ("t_hi_s", C.c_double), ("mean_s", C.c_double),
                ("sd_s", C.c_double), ("mean2_s", C.c_double), ("sd2_s", C.c_double), ("w2", C.c_double),
                ("seed", C.c_uint64), ("n_threads", C.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        lib.synth_lattice.restype = C.POINTER(_Net)
        lib.synth_lattice.argtypes = [C.POINTER(_LatticeParams)]
        lib.synth_net_free.argtypes = [C.POINTER(_Net)]
        lib.synth_make_trips.restype = C.POINTER(_Trips)
        lib.synth_make_trips.argtypes = [C.POINTER(_Net), C.POINTER(_TripParams)]
        lib.synth_trips_free.argtypes = [C.POINTER(_Trips)]
        _lib = lib
    return _lib


def _copy(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


@dataclass
class Network:
    """A directed road network in the layout ``manta_create`` takes."""
    edge_src: np.ndarray
    edge_dst: np.ndarray
    edge_lanes: np.ndarray
    edge_length_m: np.ndarray
    edge_speed_limit_mps: np.ndarray
    edge_class: np.ndarray
    node_type: np.ndarray
    node_cycle_steps: np.ndarray
    node_offset_steps: np.ndarray
    edge_green_start: np.ndarray
    edge_green_len: np.ndarray
    conn_lane_mask: np.ndarray | None
    node_i: np.ndarray | None = None
    node_j: np.ndarray | None = None
    edge_dir: np.ndarray | None = None
    node_trip_ok: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.node_type.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.edge_src.shape[0])


@dataclass
class Trips:
    """Trips in the layout ``manta_load_trips`` takes (route CSR + departure times)."""
    route_off: np.ndarray      # int64 [n+1]
    route_edges: np.ndarray    # int32
    depart_time_s: np.ndarray  # float32 [n], seconds since midnight
    origin: np.ndarray | None = None
    dest: np.ndarray | None = None

    @property
    def n_trips(self) -> int:
        return int(self.depart_time_s.shape[0])


# Road classes used by the lattice generator: local, arterial, freeway.
CLASS_LOCAL, CLASS_ARTERIAL, CLASS_FREEWAY = 0, 1, 2


def lattice(nx, ny, *, arterial_every=0, freeway_every=0, local_keep=1.0,
            len_median_m=100.0, len_sigma=0.0, len_min_m=20.0, len_max_m=2000.0,
            speed_mps=(11.111, 19.444, 29.167), lanes=(1, 2, 4),
            signal_cycle_steps=120, signal_green_steps=60, signals_at=0, all_stop=False,
            limited_access=False, seed=1) -> Network:
    lib = _load()
    p = _LatticeParams()
    p.nx, p.ny = nx, ny
    p.arterial_every, p.freeway_every = arterial_every, freeway_every
    p.local_keep = local_keep
    p.len_median_m, p.len_sigma, p.len_min_m, p.len_max_m = len_median_m, len_sigma, len_min_m, len_max_m
    for i in range(3):
        p.speed_mps[i] = speed_mps[i]
        p.lanes[i] = lanes[i]
    p.signal_cycle_steps, p.signal_green_steps = signal_cycle_steps, signal_green_steps
    p.signals_at, p.all_stop, p.seed = signals_at, int(all_stop), seed
    p.limited_access = int(limited_access)
    h = lib.synth_lattice(C.byref(p))
    n = h.contents
    try:
        N, E = n.n_nodes, n.n_edges
        net = Network(
            edge_src=_copy(n.edge_src, E, np.int32), edge_dst=_copy(n.edge_dst, E, np.int32),
            edge_lanes=_copy(n.edge_lanes, E, np.uint8),
            edge_length_m=_copy(n.edge_length_m, E, np.float32),
            edge_speed_limit_mps=_copy(n.edge_speed_mps, E, np.float32),
            edge_class=_copy(n.edge_class, E, np.uint8),
            node_type=_copy(n.node_type, N, np.uint8),
            node_cycle_steps=_copy(n.node_cycle, N, np.int32),
            node_offset_steps=_copy(n.node_offset, N, np.int32),
            edge_green_start=_copy(n.edge_green_start, E, np.int16),
            edge_green_len=_copy(n.edge_green_len, E, np.int16),
            conn_lane_mask=_copy(n.conn_lane_mask, n.n_conn, np.uint32),
            node_i=_copy(n.node_i, N, np.int32), node_j=_copy(n.node_j, N, np.int32),
            edge_dir=_copy(n.edge_dir, E, np.uint8), node_trip_ok=_copy(n.node_trip_ok, N, np.uint8))
    finally:
        lib.synth_net_free(h)
    net.meta = dict(kind="lattice", nx=nx, ny=ny, seed=seed)
    return net


def make_trips(net: Network, n_trips, *, od_model="uniform", zones=(20, 25), pool_per_zone=None,
               spacing_km=0.15, beta_km=10.0, zone_mass_sigma=1.0,
               depart="uniform", t_lo_s=0.0, t_hi_s=600.0, mean_s=0.0, sd_s=1.0,
               mean2_s=0.0, sd2_s=1.0, w2=0.0, seed=1, n_threads=None) -> Trips:
    lib = _load()
    cn = _Net()
    keep = []

    def ptr(a, ct):
        a = np.ascontiguousarray(a)
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(ct))

    cn.n_nodes, cn.n_edges = net.n_nodes, net.n_edges
    cn.edge_src, cn.edge_dst = ptr(net.edge_src, C.c_int32), ptr(net.edge_dst, C.c_int32)
    cn.edge_length_m = ptr(net.edge_length_m.astype(np.float32), C.c_float)
    cn.edge_speed_mps = ptr(net.edge_speed_limit_mps.astype(np.float32), C.c_float)
    tok = net.node_trip_ok if net.node_trip_ok is not None else np.ones(net.n_nodes, np.uint8)
    cn.node_trip_ok = ptr(tok.astype(np.uint8), C.c_uint8)
    ni = net.node_i if net.node_i is not None else np.zeros(net.n_nodes, np.int32)
    nj = net.node_j if net.node_j is not None else np.zeros(net.n_nodes, np.int32)
    cn.node_i, cn.node_j = ptr(ni.astype(np.int32), C.c_int32), ptr(nj.astype(np.int32), C.c_int32)
    tp = _TripParams()
    tp.n_trips = n_trips
    tp.od_model = {"uniform": 0, "gravity": 1}[od_model]
    tp.zones_x, tp.zones_y = zones
    # origin pool: per zone for the gravity model (default 16); for uniform OD a
    # pool over the whole network (default 0 = every node may be an origin)
    tp.pool_per_zone = (16 if od_model == "gravity" else 0) if pool_per_zone is None else pool_per_zone
    tp.spacing_km, tp.beta_km, tp.zone_mass_sigma = spacing_km, beta_km, zone_mass_sigma
    tp.depart_model = {"uniform": 0, "normal": 1, "bimodal": 2}[depart]
    tp.t_lo_s, tp.t_hi_s, tp.mean_s, tp.sd_s = t_lo_s, t_hi_s, mean_s, sd_s
    tp.mean2_s, tp.sd2_s, tp.w2 = mean2_s, sd2_s, w2
    tp.seed = seed
    tp.n_threads = n_threads or os.cpu_count() or 1
    h = lib.synth_make_trips(C.byref(cn), C.byref(tp))
    t = h.contents
    try:
        if t.n_unroutable:
            raise RuntimeError(f"{t.n_unroutable} trips had no route")
        trips = Trips(route_off=_copy(t.route_off, n_trips + 1, np.int64),
                      route_edges=_copy(t.route_edges, t.n_route_edges, np.int32),
                      depart_time_s=_copy(t.depart_time_s, n_trips, np.float32),
                      origin=_copy(t.origin, n_trips, np.int32), dest=_copy(t.dest, n_trips, np.int32))
    finally:
        lib.synth_trips_free(h)
    return trips


# ---------------------------------------------------------------- workloads --
def tiny_network(seed=1) -> Network:
    """10x10 grid, 100 m edges, 2 lanes per direction, 50 km/h, fixed-time
    signals (two 30 s phases, 120-step cycle) at the 64 interior nodes,
    boundary nodes uncontrolled."""
    return lattice(10, 10, arterial_every=1, len_median_m=100.0, len_sigma=0.0,
                   len_min_m=100.0, len_max_m=100.0, speed_mps=(13.889, 13.889, 13.889),
                   lanes=(2, 2, 2), signals_at=2, seed=seed)


def tiny_trips(net: Network, n_trips=1000, seed=1) -> Trips:
    """Uniform-random OD node pairs, departures uniform over the first 10 min."""
    return make_trips(net, n_trips, od_model="uniform", depart="uniform", t_lo_s=0.0,
                      t_hi_s=600.0, seed=seed, pool_per_zone=0)


def calib_network(seed=3) -> Network:
    """Calibration case: 20x20 grid, 100 m edges, three road classes (local
    1 lane 40 km/h; arterial every 5th line, 2 lanes 70 km/h; freeway every
    10th line, 4 lanes 105 km/h), fixed-time signals at arterial crossings."""
    return lattice(20, 20, arterial_every=5, freeway_every=10, len_median_m=100.0, len_sigma=0.0,
                   len_min_m=100.0, len_max_m=100.0, speed_mps=(11.111, 19.444, 29.167), lanes=(1, 2, 4),
                   signals_at=1, seed=seed)


def calib_trips(net: Network, n_trips=20_000, seed=3) -> Trips:
    """Uniform-random OD node pairs, departures uniform over the first 20 min."""
    return make_trips(net, n_trips, od_model="uniform", depart="uniform", t_lo_s=0.0,
                      t_hi_s=1200.0, seed=seed, pool_per_zone=0)


METRO_SIDE = 482


def metro_network(seed=2, side=METRO_SIDE) -> Network:
    """Metro-shaped synthetic network: lattice with local (1 lane, 40 km/h),
    arterial every 8th line (2 lanes, 70 km/h) and limited-access freeway
    every 32nd line (4 lanes, 105 km/h; local streets pass over it, arterials
    and freeways meet it at interchanges); lognormal lengths (median 120 m,
    sigma 0.8); local segments thinned to about 550k directed edges;
    fixed-time signals at arterial crossings; no trip starts or ends on a
    freeway."""
    return lattice(side, side, arterial_every=8, freeway_every=32, local_keep=0.57,
                   len_median_m=120.0, len_sigma=0.8, len_min_m=20.0, len_max_m=2000.0,
                   speed_mps=(11.111, 19.444, 29.167), lanes=(1, 2, 4),
                   signals_at=1, limited_access=True, seed=seed)


# Decay length of the gravity model: 5.4 km makes the mean route length on the
# metro-shaped network about 11.5 km, the mean trip distance the paper reports
# for its routes (Section IV-B, 11.3 km).
METRO_BETA_KM = 5.4


def metro_trips(net: Network, n_trips=3_200_000, seed=2, t_lo_s=5 * 3600.0, t_hi_s=12 * 3600.0,
                n_threads=None) -> Trips:
    """Gravity OD over 20x25 zones (lognormal masses, exp(-d / 5.4 km)), origins
    from a pool of 16 nodes per zone, destinations uniform in the zone;
    departures normal(08:00, 75 min) truncated to [05:00, 12:00)."""
    return make_trips(net, n_trips, od_model="gravity", zones=(20, 25), pool_per_zone=16,
                      spacing_km=0.15, beta_km=METRO_BETA_KM, depart="normal", t_lo_s=t_lo_s, t_hi_s=t_hi_s,
                      mean_s=8 * 3600.0, sd_s=75 * 60.0, seed=seed, n_threads=n_threads)


STRESS_SIDE = 822


def stress_network(seed=4, side=STRESS_SIDE) -> Network:
    """Megaregion-shaped synthetic network: the metro generator on a lattice
    about 3x the area (822 x 822 nodes, about 1.6M directed edges)."""
    return lattice(side, side, arterial_every=8, freeway_every=32, local_keep=0.57,
                   len_median_m=120.0, len_sigma=0.8, len_min_m=20.0, len_max_m=2000.0,
                   speed_mps=(11.111, 19.444, 29.167), lanes=(1, 2, 4),
                   signals_at=1, limited_access=True, seed=seed)


def stress_trips(net: Network, n_trips=10_000_000, seed=4, n_threads=None) -> Trips:
    """Gravity OD as for the metro workload; departures bimodal, 0.6 N(07:45,
    60 min) + 0.4 N(11:00, 60 min), truncated to [04:00, 13:00)."""
    return make_trips(net, n_trips, od_model="gravity", zones=(20, 25), pool_per_zone=16,
                      spacing_km=0.15, beta_km=METRO_BETA_KM, depart="bimodal", t_lo_s=4 * 3600.0,
                      t_hi_s=13 * 3600.0, mean_s=7.75 * 3600.0, sd_s=3600.0, mean2_s=11 * 3600.0, sd2_s=3600.0,
                      w2=0.4, seed=seed, n_threads=n_threads)


def incident_closures(net: Network, n=200, k0=int(7.5 * 7200), k1=9 * 7200, seed=4):
    """Lane 0 closed on n random freeway edges over steps [k0, k1) (07:30-09:00
    at dt = 0.5 s): (edge, lane, k0, k1) tuples."""
    fw = np.nonzero(net.edge_class == 2)[0]
    pick = np.random.default_rng(seed).choice(fw, size=min(n, fw.size), replace=False)
    return [(int(e), 0, int(k0), int(k1)) for e in np.sort(pick)]


# --------------------------------------------------------------- dense state --
@dataclass
class Placement:
    """Trips put directly on the network (the arguments of ``manta_place``)."""
    trip: np.ndarray        # int64
    route_pos: np.ndarray   # int32: entry of the trip's route
    lane: np.ndarray        # uint8
    x: np.ndarray           # float32: front position, cells from the start of the edge
    v: np.ndarray           # float32: speed, m/s

    @property
    def n(self) -> int:
        return int(self.trip.shape[0])


def dense_state(net: Network, tr: Trips, depart_lo_s, depart_hi_s, *, seed=5, head_frac=0.15,
                last_edge_frac=0.0, slot_cells=8, min_cells=8) -> Placement:
    """A busy traffic state to start a run from, instead of an empty network.

    Every trip departing in [depart_lo_s, depart_hi_s) is put somewhere along
    its own route: a route entry drawn uniformly (or, with probability
    `last_edge_frac`, its last entry, so it arrives soon), a lane drawn
    uniformly among that edge's lanes, and a front cell in one of the edge's
    slots of `slot_cells` cells (cell = slot * slot_cells + 0..3, so fronts in
    one lane are at least slot_cells - 3 = 5 cells apart).  With probability
    `head_frac` the slot is the edge's last one, at 50-100% of the speed
    limit, so many vehicles reach a node in the first steps; otherwise the
    slot is uniform and the speed uniform in [0, limit).  One vehicle per
    (edge, lane, slot): of several drawn, the first in a seeded random order
    stays and the others stay waiting in their departure queues.  An edge has
    max(min_cells, round(length / 1 m)) cells, the lane map's cell rule of
    Section II-D with the default vehicle length and jam gap.  Placements are
    returned in trip order."""
    rng = np.random.default_rng(seed)
    cand = np.nonzero((tr.depart_time_s >= depart_lo_s) & (tr.depart_time_s < depart_hi_s))[0].astype(np.int64)
    n = cand.size
    ro = tr.route_off
    rlen = ro[cand + 1] - ro[cand]
    pos = np.minimum((rng.random(n) * rlen).astype(np.int64), rlen - 1)
    last = rng.random(n) < last_edge_frac
    pos[last] = rlen[last] - 1
    e = tr.route_edges[ro[cand] + pos].astype(np.int64)
    lanes = net.edge_lanes.astype(np.int64)[e]
    lane = np.minimum((rng.random(n) * lanes).astype(np.int64), lanes - 1)
    cells = np.maximum(min_cells, np.floor(net.edge_length_m.astype(np.float64) + 0.5).astype(np.int64))[e]
    n_slot = (cells - 4) // slot_cells + 1
    head = rng.random(n) < head_frac
    slot = np.where(head, n_slot - 1, np.minimum((rng.random(n) * n_slot).astype(np.int64), n_slot - 1))
    cell = slot * slot_cells + rng.integers(0, 4, n)
    lim = net.edge_speed_limit_mps.astype(np.float64)[e]
    v = np.where(head, lim * rng.uniform(0.5, 1.0, n), lim * rng.random(n))
    x = cell + rng.random(n) * 0.999
    # one vehicle per (edge, lane, slot)
    lane0 = np.concatenate([[0], np.cumsum(net.edge_lanes.astype(np.int64))[:-1]])
    key = (lane0[e] + lane) * (1 << 20) + slot
    order = rng.permutation(n)
    _, first = np.unique(key[order], return_index=True)
    keep = np.sort(order[first])
    return Placement(trip=cand[keep], route_pos=pos[keep].astype(np.int32), lane=lane[keep].astype(np.uint8),
                     x=x[keep].astype(np.float32), v=v[keep].astype(np.float32))


# ------------------------------------------------------------------ ensemble --
@dataclass
class Ensemble:
    """Independent scenarios merged into one network and one trip table.

    Scenario s owns nodes [node_off[s], node_off[s+1]), edges [edge_off[s],
    edge_off[s+1]) and trips [trip_off[s], trip_off[s+1]); no edge connects two
    scenarios, so one simulation of the union advances all of them at once."""
    net: Network
    trips: Trips
    node_off: np.ndarray
    edge_off: np.ndarray
    trip_off: np.ndarray
    scenarios: list


def union(parts) -> Ensemble:
    """Disjoint union of (Network, Trips) pairs (node, edge and trip ids offset)."""
    nets_, trs = [p[0] for p in parts], [p[1] for p in parts]
    node_off = np.concatenate([[0], np.cumsum([n.n_nodes for n in nets_])]).astype(np.int64)
    edge_off = np.concatenate([[0], np.cumsum([n.n_edges for n in nets_])]).astype(np.int64)
    trip_off = np.concatenate([[0], np.cumsum([t.n_trips for t in trs])]).astype(np.int64)
    cat = lambda name, dt: np.concatenate([getattr(n, name) for n in nets_]).astype(dt)
    net = Network(
        edge_src=np.concatenate([n.edge_src + node_off[i] for i, n in enumerate(nets_)]).astype(np.int32),
        edge_dst=np.concatenate([n.edge_dst + node_off[i] for i, n in enumerate(nets_)]).astype(np.int32),
        edge_lanes=cat("edge_lanes", np.uint8), edge_length_m=cat("edge_length_m", np.float32),
        edge_speed_limit_mps=cat("edge_speed_limit_mps", np.float32), edge_class=cat("edge_class", np.uint8),
        node_type=cat("node_type", np.uint8), node_cycle_steps=cat("node_cycle_steps", np.int32),
        node_offset_steps=cat("node_offset_steps", np.int32), edge_green_start=cat("edge_green_start", np.int16),
        edge_green_len=cat("edge_green_len", np.int16),
        conn_lane_mask=np.concatenate([n.conn_lane_mask for n in nets_]).astype(np.uint32))
    route_edges = np.concatenate([t.route_edges + edge_off[i] for i, t in enumerate(trs)]).astype(np.int32)
    route_off = np.zeros(int(trip_off[-1]) + 1, np.int64)
    base = 0
    for i, t in enumerate(trs):
        route_off[trip_off[i] + 1: trip_off[i + 1] + 1] = t.route_off[1:] + base
        base += int(t.route_off[-1])
    trips = Trips(route_off=route_off, route_edges=route_edges,
                  depart_time_s=np.concatenate([t.depart_time_s for t in trs]).astype(np.float32))
    return Ensemble(net=net, trips=trips, node_off=node_off, edge_off=edge_off, trip_off=trip_off, scenarios=[])


def ensemble_scenarios(n=64, seed=100, edges_range=(5_000, 100_000), trips_range=(10_000, 500_000),
                       closed_frac=(0.0, 0.05), window_s=3600.0, t0_s=7 * 3600.0):
    """What-if scenarios of uneven size: lattice networks (plain grids for even
    scenario indices, the arterial/freeway hierarchy for odd ones) with edge
    counts log-uniform in `edges_range`, trip counts log-uniform in
    `trips_range`, a random fraction of local segments closed before routing,
    departures over one hour from t0 (per-scenario seeds seed + i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        target_e = float(np.exp(rng.uniform(np.log(edges_range[0]), np.log(edges_range[1]))))
        n_trips = int(np.exp(rng.uniform(np.log(trips_range[0]), np.log(trips_range[1]))))
        closed = float(rng.uniform(*closed_frac))
        hier = i % 2 == 1
        keep = 0.57 * (1.0 - closed) if hier else 0.75 * (1.0 - closed)
        # directed edges ~ 2 * 2 * side^2 * keep-ish: solve for the side
        side = max(12, int(np.sqrt(target_e / (4.0 * (keep if not hier else 0.62)))))
        if hier:
            net = lattice(side, side, arterial_every=8, freeway_every=32, local_keep=keep, len_median_m=120.0,
                          len_sigma=0.8, len_min_m=20.0, len_max_m=2000.0, signals_at=1, limited_access=True,
                          seed=seed + i)
        else:
            net = lattice(side, side, arterial_every=4, local_keep=keep, len_median_m=120.0, len_sigma=0.5,
                          len_min_m=20.0, len_max_m=1000.0, signals_at=1, seed=seed + i)
        tr = make_trips(net, n_trips, od_model="uniform", depart="uniform", t_lo_s=t0_s, t_hi_s=t0_s + window_s,
                        seed=seed + i, pool_per_zone=256)
        out.append((net, tr))
    return out
