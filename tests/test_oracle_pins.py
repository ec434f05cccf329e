"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of the expected values below comes from the CUDA path or from the
oracle itself: they are closed forms (IDM ODE, IDM steady state), published
generator outputs, invariants, or hand traces.
"""
import math
import os

import numpy as np
import pytest

import nets
from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
G64 = 0x9E3779B97F4A7C15


# ---------------------------------------------------------------- RNG pins --
def test_splitmix64_reference_outputs():
    """SplitMix64 (Steele, Lea, Flood 2014): outputs from state 0."""
    vals = [int(l.strip(), 16) for l in open(os.path.join(HERE, "golden", "splitmix64_reference.txt"))
            if l.strip() and not l.startswith("#")]
    got = [O.splitmix64((i * G64) & (2**64 - 1)) for i in range(3)]
    assert got == vals


def test_uniform_and_irwin_hall_moments():
    """U in [0,1) with mean 1/2, var 1/12; the Irwin-Hall normal has mean 0, var 1,
    support [-6, 6] (epsilon of Eqs. 3-4: mean 0, sd 1 m)."""
    u = np.array([O.rng_u(7, i, 3, 0) for i in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.003
    n = np.array([O.rng_n(7, i, 3, 1) for i in range(20000)])
    assert n.min() >= -6.0 and n.max() <= 6.0
    assert abs(n.mean()) < 0.03 and abs(n.var() - 1.0) < 0.04
    # different streams and steps are different draws
    assert O.rng_n(7, 5, 3, 1) != O.rng_n(7, 5, 3, 2)
    assert O.rng_u(7, 5, 3, 0) != O.rng_u(7, 5, 4, 0)


def test_per_driver_speed_limits():
    """Section IV-B: every driver draws its own maximum speed on each edge it
    enters, around the edge's limit s with standard deviation 2 sigma_s (here
    sigma_s = f s).  Over many (driver, edge) pairs the drawn limits have mean
    s and standard deviation 2 f s; a driver keeps its limit for the whole
    edge and draws again on the next; with f = 0 every driver has s."""
    n_edges, s_lim, f = 6, 20.0, 0.1
    lengths = [300.0 + 37.0 * i for i in range(n_edges)]      # distinct lengths: the cell count names the edge
    net = nets.network(n_edges + 1, [(i, i + 1, 1, lengths[i], s_lim, 0) for i in range(n_edges)])
    n_trips = 500
    tr = nets.trips([list(range(n_edges))] * n_trips, [2.0 * i for i in range(n_trips)])
    for frac in (0.0, f):
        o = O.OracleSim(net, speed_sigma_frac=frac)
        nets.load(o, tr)
        tape = o.record_tape(2400)
        o.step(2400)
        present = (tape["flags"] & 1) != 0
        t_idx, ids = np.nonzero(present)
        lim = tape["lim"][t_idx, ids].astype(np.float64)
        cells = tape["C"][t_idx, ids]
        if frac == 0.0:
            assert np.all(lim == s_lim)
            continue
        groups = {}
        for i, c, l in zip(ids.tolist(), cells.tolist(), lim.tolist()):
            groups.setdefault((i, c), set()).add(l)
        assert all(len(v) == 1 for v in groups.values())          # constant along the edge
        per = np.array([next(iter(v)) for v in groups.values()])
        assert len(per) > 1500
        z = (per / s_lim - 1.0) / (2.0 * f)
        assert abs(z.mean()) < 0.1 and abs(z.std() - 1.0) < 0.07
        assert len(np.unique(per)) > 0.95 * len(per)                # drivers and edges draw apart
        by_driver = {}
        for (i, c), v in groups.items():
            by_driver.setdefault(i, set()).update(v)
        assert sum(len(v) > 1 for v in by_driver.values()) > 0.9 * len(by_driver)


def test_lone_driver_settles_at_its_own_limit():
    """With no leader the fixed point of Eq. 1 is v = v0: a lone driver on a long
    free road ends at its own drawn limit (times v0f = 1), not the edge's."""
    net = nets.line(1, length=8000.0, speed=20.0)
    tr = nets.trips([[0]], [0.0])
    o = O.OracleSim(net, speed_sigma_frac=0.1, seed=5)
    nets.load(o, tr)
    tape = o.record_tape(700)
    o.step(700)
    lim = float(tape["lim"][-1, 0])
    v = float(o.snapshot()["v"][0])
    assert lim != 20.0
    assert abs(v - lim) <= 1e-4 * lim


def test_defaults_match_paper_constants():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "paper_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows[parts[0]] = parts[1:]
    d = O.DEFAULTS
    assert d["dt"] == float(rows["dt"][0])
    assert d["cell_m"] == float(rows["cell_m"][0])
    assert d["lc_x0_m"] == float(rows["lc_x0_m"][0])
    assert d["alpha_lo"] == float(rows["alpha_lo"][0]) and d["alpha_hi"] == float(rows["alpha_hi"][0])
    assert d["stop_dwell_steps"] * d["dt"] == float(rows["stop_s"][0])
    lo, hi = map(float, rows["gap_low_range"][:2])
    assert lo <= d["g_low"] <= hi
    lo, hi = map(float, rows["gap_high_range"][:2])
    assert lo <= d["g_high"] <= hi
    for key, name in (("a", "a_range"), ("b", "b_range"), ("T", "T_range"), ("s0", "s0_range")):
        lo, hi = map(float, rows[name][:2])
        assert all(lo <= x <= hi for x in d[key])
    assert abs(d["g_speed_split"] - 25 * 0.44704) < 1e-3   # 25 mph


# ------------------------------------------------------- T1: free-flow ODE --
def _lone_vehicle(dt, n_updates, v0=20.0, a=1.0):
    net = nets.line(20, length=2000.0, speed=v0)
    tr = nets.trips([list(range(20))], [0.0])
    s = O.OracleSim(net, dt=dt, a=[a] * 8)
    nets.load(s, tr)
    s.step(1)                      # departure at step 0 (enters at x = 0, v = 0)
    out = []
    for _ in range(n_updates):
        s.step(1)
        sn = s.snapshot()
        out.append((float(sn["v"][0]), int(sn["route_pos"][0]), float(sn["x"][0])))
    return out


def _t_of_v(v, v0, a):
    """Closed form of the free-road IDM ODE dv/dt = a (1 - (v/v0)^4), v(0) = 0."""
    u = v / v0
    return v0 / (2 * a) * (math.atanh(u) + math.atan(u))


def _v_of_t(t, v0, a):
    lo, hi = 0.0, v0 * (1 - 1e-15)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _t_of_v(mid, v0, a) < t:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_free_flow_matches_float64_replay():
    """Same discrete map (explicit velocity step, ballistic position) in float64."""
    v0, a, dt = 20.0, 1.0, 0.5
    traj = _lone_vehicle(dt, 200, v0, a)
    v, x = 0.0, 0.0
    for vg, rp, xg in traj:
        acc = a * (1 - (v / v0) ** 4)
        x = x + v * dt + 0.5 * acc * dt * dt
        v = v + acc * dt
        assert abs(vg - v) <= 2e-5 * max(1.0, v)
        assert abs(rp * 2000.0 + xg - x) <= 2e-3
    assert traj[-1][0] > 19.0


def test_free_flow_first_order_convergence_to_ode():
    """|v_k - v(t_k)| is first order in dt: halving dt halves the error."""
    v0, a, t = 20.0, 1.0, 20.0
    exact = _v_of_t(t, v0, a)
    e1 = abs(_lone_vehicle(0.5, int(t / 0.5), v0, a)[-1][0] - exact)
    e2 = abs(_lone_vehicle(0.25, int(t / 0.25), v0, a)[-1][0] - exact)
    assert e1 < 0.05 * v0
    assert 1.7 < e1 / e2 < 2.3


# ------------------------------------------- link-speed statistic (A10) --
def _link_speed_trace(lengths, x, v, n_steps, t0, W, v0=25.0, a=1.0, dt=0.5):
    """Float64 trace of a lone vehicle on a line of green edges, written from
    the definitions alone: Eq. 1 free-road term (delta = 4), the ballistic
    step, the one-node-per-step clamp (at most C_e + C_next - 1, speed 0 when
    clamped), the crossing into the next edge, and the link-speed sample of
    Sections IV-A/B taken once per vehicle-step AFTER the step: the speed the
    vehicle ends the step with, on the edge it ends the step on, in window
    (k - t0) // W.  Returns {(window, edge): [speeds]} and the smallest
    distance of any tentative position from a decision threshold (an edge end
    or a clamp bound), so the caller can check that the binary32 run takes the
    same discrete decisions."""
    C = [max(8, int(round(L_))) for L_ in lengths]
    e = 0
    samples = {}
    margin = float("inf")
    for k in range(t0, t0 + n_steps):
        acc = a * (1.0 - (v / v0) ** 4)
        vt = v + acc * dt
        assert vt >= 0.0
        xt = x + v * dt + 0.5 * acc * dt * dt
        xn, vn = xt, vt
        if e + 1 < len(C):
            cap = C[e] + C[e + 1] - 1
            margin = min(margin, abs(xt - cap), abs(xt - C[e]))
            if xt > cap:
                xn, vn = max(x, float(cap)), 0.0
            if xn >= C[e]:
                xn -= C[e]
                e += 1
        x, v = xn, vn
        samples.setdefault(((k - t0) // W, e), []).append(v)
    return samples, margin


def test_link_speed_statistic_window_edge_and_sample():
    """Pins which (window, edge) cell each vehicle-step's speed sample lands
    in and which speed is sampled: against an independent float64 trace, the
    per-(window, edge) counts are exact and the fixed-point sums agree within
    the float32/float64 gap of T1.  A sample taken before the clamp (the first
    step is clamped from 25 m/s to 0 at the one-node bound), on the edge left
    in a crossing step, before the step (the old speed), or in a window shifted
    by one step fails here."""
    lengths = [300.0, 8.0, 60.0, 45.0, 120.0, 37.0, 250.0, 3000.0]
    t0, W, n_steps = 13, 40, 260
    x0, v0_init = 296.5, 25.0
    net = nets.network(len(lengths) + 1, [(i, i + 1, 1, L_, 25.0, 0) for i, L_ in enumerate(lengths)])
    tr = nets.trips([list(range(len(lengths)))], [1e7])
    o = O.OracleSim(net, t0_step=t0, stats_window_steps=W, n_stats_windows=10)
    nets.load(o, tr)
    o.place(0, 0, 0, x0, v0_init)
    o.step(n_steps)
    expect, margin = _link_speed_trace(lengths, x0, v0_init, n_steps, t0, W)
    assert margin > 0.05
    # the trace covers what the pin is about: a clamped first step, several
    # crossings, crossings inside windows and windows inside edges
    assert expect[(0, 1)][0] == 0.0
    edges_seen = {e for (_, e) in expect}
    assert len(edges_seen) >= 6 and len({w for (w, _) in expect}) >= 6
    assert any(len({e for (w, e) in expect if w == w0}) > 1 for w0 in range(7))
    got_cnt, got_sum = {}, {}
    for w in range(10):
        ec = o.edge_counters(w)
        for e in np.nonzero(ec["speed_cnt"])[0]:
            got_cnt[(w, int(e))] = int(ec["speed_cnt"][e])
            got_sum[(w, int(e))] = int(ec["speed_sum"][e])
    assert got_cnt == {key: len(vs) for key, vs in expect.items()}
    for key, vs in expect.items():
        fx = sum(int(v * 1048576.0) for v in vs)
        # T1's bound per sample (2e-5 relative on v) in units of 2^-20 m/s, plus truncation
        tol = sum(2e-5 * max(1.0, v) * 1048576.0 + 1.0 for v in vs)
        assert abs(got_sum[key] - fx) <= tol, (key, got_sum[key], fx, tol)


# ------------------------------------------------------ T2: ring equilibrium --
def _ring_sim(n_veh, ring_edges=4, edge_len=100.0, v_init=0.0, laps=400, **cfg):
    total = int(ring_edges * edge_len)
    d = total // n_veh
    net = nets.ring(ring_edges, length=edge_len, speed=20.0)
    routes = []
    for i in range(n_veh):
        e0 = (i * d) // int(edge_len)
        routes.append([(e0 + j) % ring_edges for j in range(ring_edges * laps)])
    tr = nets.trips(routes, [1e7] * n_veh)
    s = O.OracleSim(net, **cfg)
    nets.load(s, tr)
    for i in range(n_veh):
        s.place(i, 0, 0, float((i * d) % int(edge_len)) + 0.5, v_init)
    return s, d


def _ieq(v, s, v0=20.0, a=1.0, b=2.0, T=1.5, s0=2.0):
    code = min(254, int(v * 8 + 0.5))
    dv = v - code * 0.125
    return 1 - (v / v0) ** 4 - ((s0 + v * T + v * dv / (2 * math.sqrt(a * b))) / s) ** 2


def _equilibrium_speeds(s):
    """All roots of the steady-state relation. The one-byte leader speed makes
    it piecewise continuous (one piece per speed code), so each piece is
    bisected on its own."""
    roots = []
    for code in range(0, 161):
        lo, hi = max(0.0, (code - 0.5) / 8), min(20.0, (code + 0.5) / 8)
        lo, hi = lo + 1e-12, hi - 1e-12
        if lo >= hi or (_ieq(lo, s) > 0) == (_ieq(hi, s) > 0):
            continue
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if (_ieq(mid, s) > 0) == (_ieq(lo, s) > 0):
                lo = mid
            else:
                hi = mid
        roots.append(0.5 * (lo + hi))
    return roots


@pytest.mark.parametrize("n_veh", [4, 8])
def test_ring_converges_to_idm_steady_state(n_veh):
    """Homogeneous ring: every vehicle settles at the speed solving the IDM
    equilibrium 1 - (v/v0)^4 - (s*(v, dv)/s)^2 = 0 with s = d - L and the
    leader speed seen through the one-byte code (Treiber & Kesting 2013)."""
    s, d = _ring_sim(n_veh, a=[1.0] * 8)
    s.step(3000)
    vs = []
    for _ in range(100):
        s.step(1)
        vs.append(s.snapshot()["v"].copy())
    vs = np.array(vs)
    roots = _equilibrium_speeds(d - 5)
    assert roots
    assert min(abs(vs.mean() - r) for r in roots) < 2e-3, (vs.mean(), roots)
    assert vs.std() < 5e-3
    s.check()


def test_ring_jam_below_minimum_gap():
    """Spacing d with d - L <= s0: the IDM interaction term is >= the free
    term at v = 0, so a queue at rest never moves."""
    s, d = _ring_sim(60, edge_len=105.0, v_init=0.0)        # 420 cells / 60: d = 7 -> s = 2 = s0
    assert d == 7
    s.step(200)
    sn = s.snapshot()
    assert np.all(sn["v"] == 0.0)
    assert s.stats()["arrived"] == 0


# --------------------------------------------- T3/T4: conservation, no overlap --
def _lane_orders(sn):
    orders = {}
    for i in np.argsort(-(sn["edge"].astype(np.int64) * 10**7 + sn["lane"].astype(np.int64) * 10**6
                          - sn["x"].astype(np.float64))):
        orders.setdefault((int(sn["edge"][i]), int(sn["lane"][i])), []).append(int(sn["id"][i]))
    return orders


def test_tiny_conservation_overlap_fifo():
    from paper_2007_03614_b300 import synth
    net = synth.tiny_network()
    tr = synth.tiny_trips(net)
    s = O.OracleSim(net)
    nets.load(s, tr)
    prev = None
    for k in range(2000):
        s.step(1)
        s.check()                       # map == vehicles, fronts >= L apart, conservation
        st = s.stats()
        assert st["departed"] == st["arrived"] + st["on_network"]
        assert st["loaded"] == st["departed"] + st["waiting"]
        sn = s.snapshot()
        cur = _lane_orders(sn)
        if prev is not None:
            # vehicles that stayed in the same lane keep their order (no overtaking in a lane)
            for key, ids in cur.items():
                old = prev.get(key, [])
                common = [i for i in ids if i in set(old)]
                old_common = [i for i in old if i in set(common)]
                assert common == old_common, (k, key)
        prev = cur
    st = s.stats()
    assert st["arrived"] == 1000 and st["on_network"] == 0
    ec = s.edge_counters(0)
    assert int(ec["entries"].sum()) == int(ec["exits"].sum())


# ------------------------------------------------------------- T5: merge --
def test_merge_lowest_id_wins_hand_trace():
    """Two vehicles reach the merge node in the same step: the lower id enters
    the out-edge, the other is held at its position with v = 0; next step the
    held one finds the winner in front and stays."""
    net = nets.merge(length=100.0, speed=13.889)
    routes = [[0, 2]] * 8
    routes[3] = [0, 2]
    routes[7] = [1, 2]
    tr = nets.trips(routes, [1e7] * 8)
    s = O.OracleSim(net)
    nets.load(s, tr)
    s.place(3, 0, 0, 99.75, 2.0)
    s.place(7, 0, 0, 99.75, 2.0)
    s.step(1)
    sn = s.snapshot()
    byid = {int(i): j for j, i in enumerate(sn["id"])}
    # hand trace of Eq. 1 on a free road and the ballistic update:
    acc = 1.0 * (1 - (2.0 / 13.889) ** 4)
    x_new = 99.75 + 2.0 * 0.5 + 0.5 * acc * 0.25
    w, l = byid[3], byid[7]
    assert sn["edge"][w] == 2 and abs(sn["x"][w] - (x_new - 100.0)) < 1e-5
    assert abs(sn["v"][w] - (2.0 + acc * 0.5)) < 1e-5
    assert sn["edge"][l] == 1 and sn["x"][l] == np.float32(99.75) and sn["v"][l] == 0.0
    ec = s.edge_counters(0)
    assert ec["entries"][2] == 1 and ec["exits"][0] == 1 and ec["exits"][1] == 0
    # step 2: 7 sees 3 at cell 0 of edge 2: gap 0 - 99 - 5 < 0 -> stays put
    s.step(1)
    sn = s.snapshot()
    byid = {int(i): j for j, i in enumerate(sn["id"])}
    assert sn["edge"][byid[7]] == 1 and sn["v"][byid[7]] == 0.0
    # a few steps later 3 has moved on and 7 follows onto edge 2
    s.step(20)
    sn = s.snapshot()
    byid = {int(i): j for j, i in enumerate(sn["id"])}
    assert sn["edge"][byid[7]] == 2
    assert sn["x"][byid[3]] - sn["x"][byid[7]] >= 5
    s.check()


def test_departure_competes_with_crossing():
    """A departure onto edge 2 and a crossing into lane 0 of edge 2 in the same
    step: the lower id wins, the other waits (departure) or is held (crossing)."""
    for dep_id, cross_id in ((1, 5), (5, 1)):
        net = nets.merge()
        routes = [[0, 2]] * 6
        routes[dep_id] = [2]
        routes[cross_id] = [0, 2]
        tr = nets.trips(routes, [1e7 if i not in (dep_id,) else 0.0 for i in range(6)])
        s = O.OracleSim(net)
        nets.load(s, tr)
        s.place(cross_id, 0, 0, 99.75, 2.0)
        s.step(1)
        sn = s.snapshot()
        byid = {int(i): j for j, i in enumerate(sn["id"])}
        if dep_id < cross_id:
            assert dep_id in byid and sn["edge"][byid[dep_id]] == 2 and sn["x"][byid[dep_id]] == 0.0
            assert sn["edge"][byid[cross_id]] == 0 and sn["v"][byid[cross_id]] == 0.0
        else:
            assert dep_id not in byid
            assert sn["edge"][byid[cross_id]] == 2
        s.check()


# --------------------------------------------------- T6: signal and stop sign --
def test_red_signal_stop_and_go():
    """Fixed-time signal: the approach is red for steps [0, 60) of each 120-step
    cycle. A vehicle stops short of the stop line and leaves once it turns green."""
    edges = [(0, 1, 1, 150.0, 13.889, 0), (1, 2, 1, 1000.0, 13.889, 0)]
    net = nets.network(3, edges, node_type=[0, 2, 0], cycle=[0, 120, 0], green={0: (60, 60)})
    tr = nets.trips([[0, 1]], [0.0])
    s = O.OracleSim(net)
    nets.load(s, tr)
    xs = []
    for k in range(60):
        s.step(1)
        sn = s.snapshot()
        xs.append((int(sn["edge"][0]), float(sn["x"][0]), float(sn["v"][0])))
    e, x, v = xs[-1]
    assert e == 0 and v < 0.05
    assert 150 - 1 - 2 - 1.5 <= x <= 150 - 1        # within about s0 of the stop line, never past it
    s.step(40)
    sn = s.snapshot()
    assert sn["edge"][0] == 1                        # crossed after the light turned green at k = 60


def test_stop_sign_dwell_permit_round_robin():
    """Flashing red: each vehicle stops for 4 steps (2 s) and holds the node's
    only permit while crossing; in-lanes are served in round-robin order."""
    edges = [(0, 2, 1, 60.0, 13.889, 0), (1, 2, 1, 60.0, 13.889, 0), (2, 3, 1, 400.0, 13.889, 0)]
    net = nets.network(4, edges, node_type=[0, 0, 1, 0])
    routes = [[0, 2], [1, 2], [0, 2], [1, 2]]
    tr = nets.trips(routes, [1e7] * 4)
    s = O.OracleSim(net)
    nets.load(s, tr)
    s.place(0, 0, 0, 40.0, 0.0)
    s.place(1, 0, 0, 40.0, 0.0)
    s.place(2, 0, 0, 20.0, 0.0)
    s.place(3, 0, 0, 20.0, 0.0)
    order, permits = [], []
    seen = set()
    for k in range(600):
        s.step(1)
        permits.append(s.permit(2))
        sn = s.snapshot()
        for i, e in zip(sn["id"], sn["edge"]):
            if e == 2 and int(i) not in seen:
                seen.add(int(i))
                order.append(int(i))
        s.check()
    assert order == [0, 1, 2, 3]                     # round robin over in-lanes (edge 0, edge 1, ...)
    # never two vehicles hold/cross at once: a permit changes only to NONE in between holders
    holders = [p for p in permits if p != 0xFFFFFFFF]
    assert sorted(set(holders)) == [0, 1, 2, 3]


# -------------------------------------------------------- T7: lane change --
def _gap_eval(v, va, vb, lead_gap, lag_gap, alpha, eps_a, eps_b, g):
    glead = max(g, g + alpha * v + alpha * (v - va)) + eps_a      # Eq. 3
    glag = max(g, g + alpha * v + alpha * (v - vb)) + eps_b       # Eq. 4
    return lead_gap >= glead and lag_gap >= glag, glead, glag


@pytest.mark.parametrize("lead_at,lag_at", [(80, 30), (62, 30), (80, 45), (80, 20), (80, 40), (80, 38)])
def test_discretionary_change_gap_acceptance_hand_trace(lead_at, lag_at):
    """Vehicle 0 at cell 50 (v = 10) behind a slow leader in lane 0 (cell 60);
    lane 1 has a lead at `lead_at` and a lag at `lag_at`. On an even step the
    target is lane 1; the change happens iff Eqs. 3-4 accept both gaps."""
    net = nets.line(1, length=300.0, lanes=2, speed=20.0)
    tr = nets.trips([[0]] * 4, [1e7] * 4)
    seed = 11
    s = O.OracleSim(net, seed=seed)
    nets.load(s, tr)
    s.place(0, 0, 0, 50.2, 10.0)
    s.place(1, 0, 0, 60.2, 2.0)
    s.place(2, 0, 1, lead_at + 0.2, 6.0)
    s.place(3, 0, 1, lag_at + 0.2, 12.0)
    k = 0
    alpha = 0.05 + 0.35 * O.rng_u(seed, 0, 0, 3)
    eps_a, eps_b = O.rng_n(seed, 0, k, 1), O.rng_n(seed, 0, k, 2)
    L = 5
    overlap = abs(lead_at - 50) < L or abs(lag_at - 50) < L
    ok, gl, gg = _gap_eval(10.0, 6.0, 12.0, lead_at - L - 50, 50 - L - lag_at, alpha, eps_a, eps_b, 3.0)
    # the own gap is 60 - 5 - 50 = 5; the target lead gap must be larger
    own_ok = (lead_at - L - 50) > 5
    expected = ok and own_ok and not overlap
    assert abs((lead_at - L - 50) - gl) > 0.05 and abs((50 - L - lag_at) - gg) > 0.05  # not a rounding tie
    s.step(1)
    sn = s.snapshot()
    byid = {int(i): j for j, i in enumerate(sn["id"])}
    assert int(sn["lane"][byid[0]]) == (1 if expected else 0)
    assert s.stats()["lane_changes"] == (1 if expected else 0)


@pytest.mark.parametrize("lead_at,lag_at,cells", [
    # vehicle 0 (cell 50, lane 0, behind the slow vehicle 1 at cell 60) is evaluated in full:
    # own lane 51..60 (10), target lead 55..80 (26), overlap window 46..54 (9), lead again (26),
    # lag 45..20 downward (26); vehicle 1 finds nothing ahead in 61..299 (239)
    (80, 20, 10 + 26 + 9 + 26 + 26 + 239),
    # target lead at 62: 55..62 (8) twice; lag 45..30 (16)
    (62, 30, 10 + 8 + 9 + 8 + 16 + 239),
    # a lane-1 vehicle at 48 overlaps: the overlap scan stops at its third cell
    (80, 48, 10 + 26 + 3 + 239),
    # target lead at 58 leaves no more room than the own lane: rejected after 55..58 (4)
    (58, 20, 10 + 4 + 239),
])
def test_lane_change_scan_cells_hand_count(lead_at, lag_at, cells):
    """lc_cells_scanned counts every lane-map cell the lane-change rule's scans
    read (Section II-D: own-lane leader and target lead of a discretionary
    change, then the lateral-overlap window, the lead and the lag of Eqs. 3-4),
    each scan from its first cell to its hit or the end of its range.  Counted
    here by hand on the hand-trace layout above for the first step (even: the
    target is lane 1; the lane-1 vehicles have no lane 2 to move to)."""
    net = nets.line(1, length=300.0, lanes=2, speed=20.0)
    tr = nets.trips([[0]] * 4, [1e7] * 4)
    s = O.OracleSim(net, seed=11)
    nets.load(s, tr)
    s.place(0, 0, 0, 50.2, 10.0)
    s.place(1, 0, 0, 60.2, 2.0)
    s.place(2, 0, 1, lead_at + 0.2, 6.0)
    s.place(3, 0, 1, lag_at + 0.2, 12.0)
    assert int(s.edge_cells()[0]) == 300
    s.step(1)
    assert s.stats()["lc_cells_scanned"] == cells


def test_mandatory_change_probability_eq2():
    """Eq. 2 with x0 = 1 m: at 1 m from the end the change is certain (if the
    gaps accept); far from the end (m ~ 0) it never happens."""
    # edge 0 (2 lanes) -> edge 1 turns right: only lane 0 may continue
    edges = [(0, 1, 2, 200.0, 13.889, 0), (1, 2, 1, 200.0, 13.889, 0)]
    net = nets.network(3, edges, conn=[1])
    for x, expect in ((150.3, 0), (198.3, 1)):
        tr = nets.trips([[0, 1]], [1e7])
        s = O.OracleSim(net)
        nets.load(s, tr)
        s.place(0, 0, 1, x, 0.0)
        s.step(1)          # k = 0: dir = +1, away from lane 0: nothing
        s.step(1)          # k = 1: dir = -1, toward lane 0
        sn = s.snapshot()
        assert int(sn["lane"][0]) == (0 if expect else 1)


def test_wrong_lane_is_a_late_merge_not_a_stop():
    """A vehicle that reaches the node still in a lane not allowed for its next
    edge is not held there (that would deadlock two vehicles needing each
    other's lanes): it enters lane min(l, lanes - 1) of the next edge."""
    edges = [(0, 1, 2, 100.0, 13.889, 0), (1, 2, 2, 200.0, 13.889, 0)]
    net = nets.network(3, edges, conn=[1])          # only lane 0 may continue
    tr = nets.trips([[0, 1], [0, 1]], [1e7, 1e7])
    s = O.OracleSim(net)
    nets.load(s, tr)
    s.place(0, 0, 1, 60.0, 10.0)                    # lane 1 (wrong), moving
    s.place(1, 0, 0, 60.0, 10.0)                    # lane 0 alongside all the way: no room to change
    crossed_from = None
    for _ in range(20):
        prev = s.snapshot()
        s.step(1)
        s.check()
        sn = s.snapshot()
        byid = {int(i): j for j, i in enumerate(sn["id"])}
        pj = {int(i): j for j, i in enumerate(prev["id"])}
        j = byid[0]
        assert sn["v"][j] > 0.0                      # never held at the stop line
        if sn["edge"][j] == 1 and crossed_from is None:
            crossed_from = int(prev["lane"][pj[0]])
    assert crossed_from == 1                         # still in the disallowed lane at the node
    assert sn["edge"][byid[0]] == 1 and sn["lane"][byid[0]] == 1


# ------------------------------------------------------------ lane closures --
def test_closed_lane_obstacle_and_mandatory_change():
    """An incident closure holds a stationary obstacle from mid-edge on: a
    vehicle behind it in a one-lane road stops short of it; in a two-lane road
    it changes lanes (mandatory) and passes."""
    # one lane: stops behind the obstacle at cell C/2 = 100
    net = nets.line(1, length=200.0, lanes=1, speed=13.889)
    tr = nets.trips([[0]], [1e7])
    s = O.OracleSim(net)
    nets.load(s, tr)
    s.set_lane_closure(0, 0, 0, 1000)
    s.place(0, 0, 0, 20.0, 10.0)
    s.step(200)
    sn = s.snapshot()
    assert sn["v"][0] < 0.05 and 100 - 1 - 2 - 1.5 <= sn["x"][0] <= 100 - 1
    # two lanes: the vehicle leaves the closed lane before the obstacle and arrives
    net = nets.line(1, length=200.0, lanes=2, speed=13.889)
    s = O.OracleSim(net, lc_len_scale_m=30.0)
    nets.load(s, tr)
    s.set_lane_closure(0, 0, 0, 1000)
    s.place(0, 0, 0, 20.0, 10.0)
    for _ in range(60):
        s.step(1)
        sn = s.snapshot()
        if len(sn["id"]) and sn["x"][0] >= 100:
            assert sn["lane"][0] == 1
    assert s.stats()["arrived"] == 1 and s.stats()["lane_changes"] == 1


def test_closed_lane_blocks_entry_and_departures_until_reopened():
    net = nets.line(2, length=100.0, lanes=1, speed=13.889)
    tr = nets.trips([[0, 1], [1]], [0.0, 0.0])
    s = O.OracleSim(net)
    nets.load(s, tr)
    s.set_lane_closure(1, 0, 0, 100)            # lane 0 of edge 1 closed for steps [0, 100)
    s.step(80)
    sn = s.snapshot()
    byid = {int(i): j for j, i in enumerate(sn["id"])}
    assert 1 not in byid                          # the departure onto edge 1 waits
    assert sn["edge"][byid[0]] == 0 and sn["v"][byid[0]] < 0.05   # held at the node
    s.step(60)
    st = s.stats()
    assert st["departed"] == 2                    # both moved on after step 100
    with pytest.raises(O.OracleError):
        s.set_lane_closure(0, 0, 0, 10)          # only before the first step


def test_ensemble_union_is_disjoint():
    """The union of scenarios keeps every route inside its own scenario and the
    oracle accepts it (contiguous routes, edge and node ids offset)."""
    from paper_2007_03614_b300 import synth
    sc = synth.ensemble_scenarios(n=3, seed=3, edges_range=(500, 2000), trips_range=(100, 400))
    ens = synth.union(sc)
    for s in range(3):
        a, b = ens.trip_off[s], ens.trip_off[s + 1]
        r = ens.trips.route_edges[ens.trips.route_off[a]:ens.trips.route_off[b]]
        assert r.min() >= ens.edge_off[s] and r.max() < ens.edge_off[s + 1]
    o = O.OracleSim(ens.net, t0_step=50400)
    nets.load(o, ens.trips)
    o.step(100)
    o.check()
