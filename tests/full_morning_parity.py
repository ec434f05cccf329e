"""Whole-morning parity of the CUDA path against the CPU oracle on the headline
workload: the metro-shaped network and 3.2M trips, 05:00-12:00 at dt = 0.5 s
(50,400 steps).  Too long for the test suite (the oracle needs hours on one
core), so it runs as a script in three parts:

    python tests/full_morning_parity.py --side oracle --out DIR_A    # CPU, hours
    python tests/full_morning_parity.py --side gpu --out DIR_B       # one B300, seconds
    python tests/full_morning_parity.py --compare DIR_A DIR_B

With --case peak-hour both sides start instead from the dense peak-hour state
(the trips departing 07:00-07:30 placed along their routes at 07:30, the
07:00-08:00 trips loaded) and run one hour, to 08:30 (about 40 min on one
core).  With --case stress-incident they run the stress megaregion (~1.6M
edges) from 08:00 to 09:00 with its incident lane closures active: the trips
departing 07:45-08:00 placed along their routes (none in a closed lane), the
07:45-08:05 trips loaded.  With --case late-morning they run the metro network
from 11:00 to 12:00 from the dense late-morning state (the trips departing
09:30-11:00 placed along their routes, the 09:30-11:05 trips loaded).

Each side writes, at each checkpoint (08:00 and 12:00; 08:30 for the peak
hour), a digest of its whole state: SHA-256
of every snapshot array (vehicles sorted by trip id; x and v as bit patterns),
of the entry and exit counters, and of every statistics window's speed sums
and counts, plus the statistics themselves.  The comparison requires every
digest and statistic to be equal.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

T0_STEP = 36000                      # 05:00
CHECKPOINTS = {"08:00": 21600, "12:00": 50400}
PEAK_CHECKPOINTS = {"08:30": 7200}   # steps after 07:30
STRESS_CHECKPOINTS = {"08:30": 3600, "09:00": 7200}   # steps after 08:00
LATE_CHECKPOINTS = {"11:30": 3600, "12:00": 7200}     # steps after 11:00


def _subset(tr, lo_s, hi_s):
    from paper_2007_03614_b300 import synth
    sel = np.nonzero((tr.depart_time_s >= lo_s) & (tr.depart_time_s < hi_s))[0]
    routes = [tr.route_edges[tr.route_off[i]:tr.route_off[i + 1]] for i in sel]
    off = np.zeros(len(sel) + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in routes])
    return synth.Trips(route_off=off, route_edges=np.concatenate(routes).astype(np.int32),
                       depart_time_s=tr.depart_time_s[sel])


def _stress_case():
    from paper_2007_03614_b300 import synth
    net = synth.stress_network()
    tr = synth.stress_trips(net)
    clo = synth.incident_closures(net)
    lo = 8 * 3600
    sub = _subset(tr, lo - 900, lo + 300)
    pl = synth.dense_state(net, sub, lo - 900, lo, head_frac=0.15, seed=13)
    closed = {(e, l) for (e, l, _, _) in clo}
    e = sub.route_edges[sub.route_off[pl.trip] + pl.route_pos]
    keep = np.array([(int(a), int(b)) not in closed for a, b in zip(e, pl.lane)])
    args = [a[keep] for a in (pl.trip, pl.route_pos, pl.lane, pl.x, pl.v)]
    return net, sub, int(lo / 0.5), args, clo
WINDOW_STEPS = 600


def _h(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def digest(sim, steps_done: int) -> dict:
    st = sim.stats()
    sn = sim.snapshot()
    order = np.argsort(sn["id"], kind="stable")
    out = {"stats": {k: int(v) for k, v in st.items()}, "snapshot": {}}
    for key, dt in (("id", np.uint32), ("edge", np.int32), ("lane", np.uint8), ("dwell", np.uint8),
                    ("route_pos", np.int32)):
        out["snapshot"][key] = _h(np.asarray(sn[key]).astype(dt)[order])
    for key in ("x", "v"):
        out["snapshot"][key] = _h(np.asarray(sn[key], dtype=np.float32)[order].view(np.uint32))
    ec = sim.edge_counters(0)
    out["entries"] = _h(np.asarray(ec["entries"], dtype=np.uint32))
    out["exits"] = _h(np.asarray(ec["exits"], dtype=np.uint32))
    out["windows"] = []
    for w in range((steps_done + WINDOW_STEPS - 1) // WINDOW_STEPS):
        e = sim.edge_counters(w)
        out["windows"].append([_h(np.asarray(e["speed_sum"], dtype=np.uint64)),
                               _h(np.asarray(e["speed_cnt"], dtype=np.uint32))])
    return out


def run(side: str, out_dir: str, case: str = "morning") -> None:
    import bench
    os.makedirs(out_dir, exist_ok=True)
    t0, checkpoints, place, closures = T0_STEP, CHECKPOINTS, None, ()
    if case == "stress-incident":
        net, tr, t0, place, closures = _stress_case()
        checkpoints = STRESS_CHECKPOINTS
    else:
        net, tr = bench.workload()
    if case == "peak-hour":
        t0, tr, pl = bench.peak_sample(net, tr)
        checkpoints = PEAK_CHECKPOINTS
        place = [pl.trip, pl.route_pos, pl.lane, pl.x, pl.v]
    elif case == "late-morning":
        from paper_2007_03614_b300 import synth
        lo = 11 * 3600
        tr = _subset(tr, lo - 5400, lo + 300)
        pl = synth.dense_state(net, tr, lo - 5400, lo, head_frac=0.1, seed=11)
        t0, checkpoints = int(lo / 0.5), LATE_CHECKPOINTS
        place = [pl.trip, pl.route_pos, pl.lane, pl.x, pl.v]
    if side == "oracle":
        from oracle import oracle as O
        sim = O.OracleSim(net, t0_step=t0)
    else:
        import torch
        from paper_2007_03614_b300 import manta
        sim = manta.Sim(net, stream=torch.cuda.Stream(), t0_step=t0)
    for (e, l, k0, k1) in closures:
        sim.set_lane_closure(e, l, k0, k1)
    sim.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
    if place is not None:
        if side == "oracle":
            sim.place_many(*place)
        else:
            sim.place(*place)
    done, t_start = 0, time.time()
    for name, target in checkpoints.items():
        while done < target:
            n = min(1800, target - done)
            sim.step(n)
            done += n
            print(f"{side} step {done} ({time.time() - t_start:.0f} s)", flush=True)
        d = digest(sim, done)
        d["side"], d["at"], d["steps"] = side, name, done
        with open(os.path.join(out_dir, f"{side}_{name.replace(':', '')}.json"), "w") as f:
            json.dump(d, f)
        print(f"{side} {name}: {d['stats']}", flush=True)


def compare(a_dir: str, b_dir: str) -> int:
    bad = 0
    names = sorted({f.rsplit("_", 1)[1][:-5] for d in (a_dir, b_dir) for f in os.listdir(d) if f.endswith(".json")})
    for name in [n[:2] + ":" + n[2:] for n in names]:
        tag = name.replace(":", "")
        fa = [f for f in os.listdir(a_dir) if f.endswith(f"_{tag}.json")]
        fb = [f for f in os.listdir(b_dir) if f.endswith(f"_{tag}.json")]
        if not fa or not fb:
            print(f"{name}: missing ({fa}, {fb})")
            bad += 1
            continue
        a = json.load(open(os.path.join(a_dir, fa[0])))
        b = json.load(open(os.path.join(b_dir, fb[0])))
        same = {k: a[k] == b[k] for k in ("stats", "snapshot", "entries", "exits", "windows")}
        print(f"{name}: steps {a['steps']}, on network {a['stats']['on_network']}, "
              f"vehicle updates {a['stats']['vehicle_updates']}: "
              + ", ".join(f"{k} {'equal' if v else 'DIFFERENT'}" for k, v in same.items()))
        bad += sum(not v for v in same.values())
    return bad


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", choices=["oracle", "gpu"])
    ap.add_argument("--out")
    ap.add_argument("--compare", nargs=2)
    ap.add_argument("--case", choices=["morning", "peak-hour", "stress-incident", "late-morning"],
                    default="morning")
    args = ap.parse_args()
    if args.compare:
        sys.exit(1 if compare(*args.compare) else 0)
    run(args.side, args.out, args.case)
