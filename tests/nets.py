"""Small hand-built road networks and trip tables for the tests.

Each builder returns a ``synth.Network`` (the array layout ``manta_create``
takes) so the same objects feed the oracle, the naive reference and the CUDA
library.
"""
from __future__ import annotations

import numpy as np

from paper_2007_03614_b300.synth import Network, Trips

GREEN, STOP, SIGNAL = 0, 1, 2


def network(n_nodes, edges, node_type=None, cycle=None, offset=None, green=None, conn=None):
    """edges: list of (src, dst, lanes, length_m, speed_mps, class)."""
    E = len(edges)
    a = np.array(edges, dtype=np.float64)
    nt = np.zeros(n_nodes, np.uint8) if node_type is None else np.asarray(node_type, np.uint8)
    cyc = np.zeros(n_nodes, np.int32) if cycle is None else np.asarray(cycle, np.int32)
    off = np.zeros(n_nodes, np.int32) if offset is None else np.asarray(offset, np.int32)
    gs = np.zeros(E, np.int16)
    gl = np.zeros(E, np.int16)
    if green is not None:
        for e, (s, l) in green.items():
            gs[e], gl[e] = s, l
    return Network(edge_src=a[:, 0].astype(np.int32), edge_dst=a[:, 1].astype(np.int32),
                   edge_lanes=a[:, 2].astype(np.uint8), edge_length_m=a[:, 3].astype(np.float32),
                   edge_speed_limit_mps=a[:, 4].astype(np.float32), edge_class=a[:, 5].astype(np.uint8),
                   node_type=nt, node_cycle_steps=cyc, node_offset_steps=off,
                   edge_green_start=gs, edge_green_len=gl,
                   conn_lane_mask=None if conn is None else np.asarray(conn, np.uint32))


def trips(routes, depart_time_s):
    off = np.zeros(len(routes) + 1, np.int64)
    for i, r in enumerate(routes):
        off[i + 1] = off[i] + len(r)
    edges = np.concatenate([np.asarray(r, np.int32) for r in routes]) if routes else np.zeros(0, np.int32)
    return Trips(route_off=off, route_edges=edges, depart_time_s=np.asarray(depart_time_s, np.float32))


def line(n_edges, length=200.0, lanes=1, speed=20.0, cls=0, node_type=None, **kw):
    edges = [(i, i + 1, lanes, length, speed, cls) for i in range(n_edges)]
    return network(n_edges + 1, edges, node_type=node_type, **kw)


def ring(n_edges, length=100.0, lanes=1, speed=20.0, cls=0):
    edges = [(i, (i + 1) % n_edges, lanes, length, speed, cls) for i in range(n_edges)]
    return network(n_edges, edges)


def merge(length=100.0, speed=13.889, lanes=1, node_type=GREEN):
    """Edges 0: 0->2 and 1: 1->2 merge into edge 2: 2->3."""
    edges = [(0, 2, lanes, length, speed, 0), (1, 2, lanes, length, speed, 0), (2, 3, lanes, length, speed, 0)]
    nt = [GREEN, GREEN, node_type, GREEN]
    return network(4, edges, node_type=nt)


def load(sim, tr: Trips):
    sim.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
