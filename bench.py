"""Benchmark: vehicle-updates/s of the metro-shaped morning (05:00-12:00,
dt = 0.5 s, 3.2M trips, ~550k edges) on one B300, through the C ABI.

A bench "step" is one chunk of `--chunk` simulated time steps (default 1800 =
15 simulated minutes) of the whole hot path: departures, lane changes, leader
scans, IDM, merges, arrivals, lane-map writes, statistics.  `--warmup W`
chunks run untimed, then `--steps K` chunks are timed with CUDA events on the
simulation's stream; the default W + K = 28 chunks is the whole morning.

Between timed chunks the L2 is flushed (a 256 MB write, outside the events);
the working set (two 140 MB lane maps, 1.8 GB of routes) is larger than L2.

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload.  With torchrun (N > 1) every rank runs an independent
replica of the same workload (the update does not shard without an exchange
step); value = updates of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vehicle-updates/s & wall-time of 3.2M-trip morning at dt=0.5 s; % HBM peak"
UNIT = "vehicle-updates/s"
T0_STEP = 36000                     # 05:00 at dt = 0.5 s
MORNING_STEPS = 50400               # 05:00-12:00

# Algorithmic bytes of one step of the method (the scope table's measurement
# row): per vehicle update, the state a structure-of-arrays layout must read
# (x 4, v 4, route cursor 4, edge 4, lane/flags/dwell 2, previous cell 4 = 22 B)
# and write (18 B), the edge record it needs (12 B), the map byte written and
# the one cleared (1 + 1); per lane-map cell read by a scan, 1 B: the leader
# scans (cells_scanned) and the lane-change rule's scans (lc_cells_scanned:
# own-lane leader, target-lane lead, lateral-overlap window, lead and lag);
# per node a scan crosses, the next route entry (4 B); per gap-acceptance
# evaluation, the lead and lag cells (8 B); per departure, 16 B.
BYTES_PER_UPDATE = 54
BYTES_PER_CELL = 1
BYTES_PER_BOUNDARY = 4
BYTES_PER_LC_EVAL = 8
BYTES_PER_DEPARTURE = 16
# Reported beside it, not in it: the per-edge speed statistic's read-modify-
# write (sum 8 + count 4, read and written) per vehicle update.
BYTES_STATS_PER_UPDATE = 24
# What this implementation's layout moves per unit (48-byte vehicle records
# read twice and written once, active-list entries, statistics; an edge record,
# signal window and node type per node crossed; a 64-byte window per
# gap-acceptance evaluation): context for the DRAM traffic, not the roofline.
LAYOUT_BYTES = {"per_update": 162, "per_cell": 1, "per_route_read": 29, "per_lc_eval": 64}
KERNEL_SOURCES = ("paper_2007_03614_b300/csrc/step_kernel.cuh", "paper_2007_03614_b300/csrc/sim.cuh")
TRAFFIC_PROFILE = "profiles/metro_step_kernel_ncu.md"
WORKLOAD = ("metro-shaped morning: ~550k directed edges / ~218k nodes, 3.2M trips, "
            "05:00-12:00 departures N(08:00, 75 min), dt = 0.5 s")
PEAK_HOUR = (7.5 * 3600, 8.5 * 3600)


def algorithmic_bytes(d: dict, lc_scans: bool = True) -> int:
    """The algorithmic bytes of the counters in d; lc_scans=False leaves out
    the lane-change scans' cells (the figure reported before they were
    counted)."""
    return (d["vehicle_updates"] * BYTES_PER_UPDATE + d["cells_scanned"] * BYTES_PER_CELL
            + (d["lc_cells_scanned"] * BYTES_PER_CELL if lc_scans else 0)
            + d["route_reads"] * BYTES_PER_BOUNDARY + d["lc_evals"] * BYTES_PER_LC_EVAL
            + d["departed"] * BYTES_PER_DEPARTURE)


def layout_bytes(d: dict) -> int:
    return (d["vehicle_updates"] * LAYOUT_BYTES["per_update"] + d["cells_scanned"] * LAYOUT_BYTES["per_cell"]
            + d["route_reads"] * LAYOUT_BYTES["per_route_read"] + d["lc_evals"] * LAYOUT_BYTES["per_lc_eval"])


def host_cpu() -> dict:
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    try:
        usable = len(os.sched_getaffinity(0))
    except Exception:
        usable = os.cpu_count()
    return {"nproc": usable, "cpu_count": os.cpu_count(), "model": model}


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    # over the sources with comments and blank lines removed, so that a
    # comment edit does not invalidate counters taken on the same code
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_traffic_per_update():
    """DRAM bytes per vehicle update from the committed ncu summary, if it was
    taken on the kernel as it is now (same source hash); else None."""
    try:
        import re
        vals = {}
        for line in open(os.path.join(ROOT, TRAFFIC_PROFILE)):
            m = re.match(r"\s*-\s*(kernel_sha256|dram_bytes_per_vehicle_update):\s*`([^`]*)`", line)
            if m:
                vals[m.group(1)] = m.group(2)
        if vals.get("kernel_sha256") == kernel_hash():
            return float(vals["dram_bytes_per_vehicle_update"])
    except Exception:
        pass
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, world


def aggregate_ranks(elapsed_s: float, updates: int, device="cpu"):
    """Whole-job figures over the ranks of a replica run: the slowest rank's
    time and the sum of every rank's vehicle updates (each rank simulates its
    own replica; nothing else is exchanged).  Single process: unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_s), float(updates)
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def workload(seed=2):
    from paper_2007_03614_b300 import synth
    net = synth.metro_network(seed=seed)
    tr = synth.metro_trips(net, seed=seed)
    return net, tr


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].isdigit():
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [int(r[1]) for r in rows]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for nm, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": int(statistics.median(sm)), "sm_max_mhz": int(rows[0][2]), "samples": len(rows),
                "reasons": sorted(reasons)}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2007_03614_b300 import manta
    from paper_2007_03614_b300.build import build

    rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world > 1:
        build() if rank == 0 else None
    if world > 1:
        dist.barrier()
    manta.load_library()
    net, tr = workload()
    stream = torch.cuda.Stream()
    chunk = args.chunk
    if args.profile_case:
        # a small case for counter captures: the trips departing 07:30-08:00 on
        # the full network, 1200 warm-up steps from an empty network at 07:30
        lo = 7.5 * 3600
        off, edges, dep = _sample(tr, lo, lo + 1800)
        sim = manta.Sim(net, stream=stream, t0_step=int(lo / 0.5), n_stats_windows=8)
        sim.load_trips(off, edges, dep)
        sim.step(1200)
        u0 = sim.stats()["vehicle_updates"]
        for _ in range(args.steps):
            sim.step(chunk)
        st = sim.stats()
        print(json.dumps({"profile_case": True, "kernel_sha256": kernel_hash(),
                          "updates_in_profiled_launches": st["vehicle_updates"] - u0, "stats": st,
                          "phase_ms": [float(x) for x in sim.phase_times_ms()]}))
        return
    if args.profile_peak:
        # the headline workload from 05:00 to --profile-at (default 07:45) in
        # untimed launches of 1800 steps, then `--steps` launches of `--chunk`
        # steps: the case for counter captures of that traffic state
        sim = manta.Sim(net, stream=stream, t0_step=T0_STEP)
        sim.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
        n = int(args.profile_at * 3600 / 0.5) - T0_STEP
        while n > 0:
            sim.step(min(1800, n))
            n -= 1800
        u0 = sim.stats()["vehicle_updates"]
        ph0 = sim.phase_times_ms()
        for _ in range(args.steps):
            sim.step(chunk)
        st = sim.stats()
        print(json.dumps({"profile_peak": True, "kernel_sha256": kernel_hash(),
                          "updates_in_profiled_launches": st["vehicle_updates"] - u0, "stats": st,
                          "phase_ms": [float(x) - float(y) for x, y in zip(sim.phase_times_ms(), ph0)]}))
        return
    # ---- device-resident run (the headline value) ----
    sim = manta.Sim(net, stream=stream, t0_step=T0_STEP)
    sim.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    keys = ("vehicle_updates", "cells_scanned", "lc_cells_scanned", "route_reads", "lc_evals", "clamps",
            "lane_changes", "departed", "arrived")

    def timed_chunk():
        with torch.cuda.stream(stream):
            flush.fill_(1)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            sim.step(chunk)
            ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / 1000.0

    warm_times = [timed_chunk() for _ in range(args.warmup)]
    s0 = sim.stats()
    ph0 = sim.phase_times_ms()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    times, per_chunk = [], []
    prev = s0
    with Clocks(local) as clk:
        for _ in range(args.steps):
            times.append(timed_chunk())
            cur = sim.stats()             # outside the events: counters of this chunk
            per_chunk.append({k: cur[k] - prev[k] for k in keys})
            prev = cur
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    s1 = sim.stats()
    phase_ms = [round(float(a - b), 2) for a, b in zip(sim.phase_times_ms(), ph0)]
    elapsed = sum(times)
    d = {k: s1[k] - s0[k] for k in keys}
    elapsed, total_updates = aggregate_ranks(elapsed, d["vehicle_updates"], device="cuda")
    sim.close()
    del flush
    # ---- end to end through the C ABI from host buffers: always the whole
    # morning (05:00-12:00), create and load included ----
    e2e, morning = None, None
    n_morning = (MORNING_STEPS + chunk - 1) // chunk
    if not args.no_e2e:
        torch.cuda.synchronize()
        h2d = sum(a.nbytes for a in (net.edge_src, net.edge_dst, net.edge_lanes, net.edge_length_m,
                                      net.edge_speed_limit_mps, net.edge_class, net.node_type, net.node_cycle_steps,
                                      net.node_offset_steps, net.edge_green_start, net.edge_green_len,
                                      net.conn_lane_mask, tr.route_off, tr.route_edges, tr.depart_time_s))
        t0 = time.perf_counter()
        sim2 = manta.Sim(net, stream=stream, t0_step=T0_STEP)
        sim2.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
        t_load = time.perf_counter() - t0
        left = MORNING_STEPS
        while left > 0:
            sim2.step(min(chunk, left))
            left -= chunk
            st = sim2.stats()                 # device -> host read of the step's result
        upd = st["vehicle_updates"]
        t_e2e = time.perf_counter() - t0
        morning = round(t_e2e - t_load, 3)
        e2e = {"value": upd / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d // n_morning),
               "d2h_bytes_per_step": 96, "seconds": round(t_e2e, 3), "create_load_s": round(t_load, 3),
               "sim_steps": MORNING_STEPS, "bench_steps": n_morning,
               "window": "05:00-12:00 (the whole morning, whatever --steps/--warmup are)"}
        sim2.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    per_launch_s = elapsed / max(1, args.steps)
    bytes_alg = algorithmic_bytes(d)
    achieved = bytes_alg / max(1, args.steps) / per_launch_s / 1e9
    tpu = measured_traffic_per_update()
    traffic = None if tpu is None else int(tpu * d["vehicle_updates"] / max(1, args.steps))
    # per simulated hour and over the peak hour (07:30-08:30)
    first = T0_STEP + args.warmup * chunk
    hours, peak_chunks = {}, []
    for i, (t, c) in enumerate(zip(times, per_chunk)):
        k_lo = first + i * chunk
        t_s = k_lo * 0.5
        hours.setdefault(int(t_s // 3600), []).append((t, c))
        if PEAK_HOUR[0] <= t_s and t_s + chunk * 0.5 <= PEAK_HOUR[1]:
            peak_chunks.append((t, c))

    def summary(rows):
        tt = sum(r[0] for r in rows)
        cc = {k: sum(r[1][k] for r in rows) for k in keys}
        ab = algorithmic_bytes(cc)
        u = max(1, cc["vehicle_updates"])
        return {"seconds": round(tt, 4), "vehicle_updates": cc["vehicle_updates"],
                "updates_per_s": cc["vehicle_updates"] / tt, "algorithmic_bytes_per_update": round(ab / u, 2),
                "cells_per_update": round(cc["cells_scanned"] / u, 2),
                "lc_cells_per_update": round(cc["lc_cells_scanned"] / u, 2),
                "achieved_gbs": round(ab / tt / 1e9, 1), "frac": round(ab / tt / 1e9 / peak, 4)}

    hourly = {f"{h:02d}:00-{h + 1:02d}:00": summary(r) for h, r in sorted(hours.items())}
    peak_hour = summary(peak_chunks) if len(peak_chunks) == 4 else None
    out = {
        "metric": METRIC, "value": total_updates / elapsed, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded metro-shaped lattice network and gravity-model trips)",
        "config": {"workload": WORKLOAD,
                   "sim_steps_per_bench_step": chunk, "t0_step": T0_STEP,
                   "timed_sim_window": [first, first + args.steps * chunk],
                   "l2": "flushed between timed steps (256 MB write) and working set > L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "gpu_launches": args.steps * ((chunk + 2047) // 2048),
        "morning_wall_s": morning,
        "morning_wall_note": "05:00-12:00 stepped through the C ABI with a stats read per bench step, create "
                             "and load excluded (the e2e run)",
        "morning_device_s": round(sum(warm_times) + elapsed, 3) if args.warmup + args.steps >= n_morning else None,
        "counters": d,
        "phase_ms_timed": phase_ms,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": int(bytes_alg / max(1, args.steps)),
                     "algorithmic_bytes_per_update": round(bytes_alg / max(1, d["vehicle_updates"]), 2),
                     "formula": f"{BYTES_PER_UPDATE} B/update + {BYTES_PER_CELL} B/cell read by a leader "
                                f"scan or a lane-change scan + {BYTES_PER_BOUNDARY} B/route read + "
                                f"{BYTES_PER_LC_EVAL} B/gap-acceptance evaluation + {BYTES_PER_DEPARTURE} B/departure",
                     "frac_without_lane_change_scans": round(
                         algorithmic_bytes(d, lc_scans=False) / max(1, args.steps) / per_launch_s / 1e9 / peak, 4),
                     "frac_with_link_statistics": round(
                         (bytes_alg + BYTES_STATS_PER_UPDATE * d["vehicle_updates"]) / max(1, args.steps)
                         / per_launch_s / 1e9 / peak, 4),
                     "peak_hour": peak_hour,
                     "traffic_model": {"bytes_per_launch": int(layout_bytes(d) / max(1, args.steps)),
                                       "per_unit": LAYOUT_BYTES}},
        "hourly": hourly,
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(net, tr, args.cpu_steps, stream)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def _sample(tr, lo_s, hi_s):
    sel = np.nonzero((tr.depart_time_s >= lo_s) & (tr.depart_time_s < hi_s))[0]
    ro = tr.route_off
    lens = ro[sel + 1] - ro[sel]
    off = np.zeros(len(sel) + 1, np.int64)
    off[1:] = np.cumsum(lens)
    idx = np.concatenate([np.arange(ro[i], ro[i + 1]) for i in sel]) if len(sel) else np.zeros(0, np.int64)
    return off, tr.route_edges[idx], tr.depart_time_s[sel]


def peak_sample(net, tr):
    """The bounded sample the CPU oracle is timed on: a dense peak-hour state
    on the full metro network -- every trip departing 07:00-07:30 put along
    its route at 07:30 by the seeded dense-state generator (about the number
    of vehicles on the network at the peak) -- with the trips departing
    07:00-08:00 loaded (the unplaced ones depart from their queues)."""
    from paper_2007_03614_b300 import synth
    lo = 7.5 * 3600
    off, edges, dep = _sample(tr, lo - 1800, lo + 1800)
    sub = synth.Trips(route_off=off, route_edges=edges, depart_time_s=dep)
    pl = synth.dense_state(net, sub, lo - 1800, lo, seed=7)
    return int(lo / 0.5), sub, pl


def cpu_baseline(net, tr, n_steps, stream=None):
    """The CPU oracle, single-threaded, on a bounded sample: `n_steps` steps
    from the dense peak-hour state of peak_sample; the GPU's rate on the
    identical sample is reported beside it."""
    from oracle import oracle as O
    t0, sub, pl = peak_sample(net, tr)
    s = O.OracleSim(net, t0_step=t0, n_stats_windows=4)
    s.load_trips(sub.route_off, sub.route_edges, sub.depart_time_s)
    s.place_many(pl.trip, pl.route_pos, pl.lane, pl.x, pl.v)
    t = time.perf_counter()
    s.step(n_steps)
    dt = time.perf_counter() - t
    upd = s.stats()["vehicle_updates"]
    s.close()
    out = {"value": upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "host": host_cpu(),
           "sample": f"dense peak-hour state on the metro network: {pl.n} vehicles placed at 07:30 "
                     f"(trips departing 07:00-07:30), {sub.n_trips} trips loaded; {n_steps} steps, "
                     f"{upd} vehicle updates in {dt:.1f} s"}
    if stream is not None:
        import torch
        from paper_2007_03614_b300 import manta
        g = manta.Sim(net, stream=stream, t0_step=t0, n_stats_windows=4)
        g.load_trips(sub.route_off, sub.route_edges, sub.depart_time_s)
        g.place(pl.trip, pl.route_pos, pl.lane, pl.x, pl.v)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        g.step(n_steps)
        ev1.record(stream)
        ev1.synchronize()
        gu = g.stats()["vehicle_updates"]
        g.close()
        gt = ev0.elapsed_time(ev1) / 1000.0
        out["gpu_same_sample"] = {"value": gu / gt, "seconds": gt, "vehicle_updates": gu,
                                  "same_updates_as_oracle": gu == upd}
    return out


def _oracle_scenario(job):
    """One ensemble scenario on the CPU oracle for n_steps steps from 07:00
    (a worker of the ensemble's CPU baseline)."""
    net, tr, t0, n_steps = job
    from oracle import oracle as O
    s = O.OracleSim(net, t0_step=t0, n_stats_windows=16)
    s.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
    t = time.perf_counter()
    s.step(n_steps)
    dt = time.perf_counter() - t
    upd = s.stats()["vehicle_updates"]
    s.close()
    return upd, dt


def _warm_worker(_):
    from oracle import oracle as O
    O.build()
    return 0


def ensemble_cpu_baseline(sc, t0, n_steps):
    """The oracle on every scenario of the ensemble for n_steps steps, (a) one
    process running them one after another, (b) one process per usable host
    core (independent scenarios, spawn-started pool): scenario-steps/s and
    vehicle-updates/s of each."""
    import multiprocessing as mp
    jobs = [(net, tr, t0, n_steps) for net, tr in sc]
    out = {"sample": f"{len(sc)} scenarios x {n_steps} steps from 07:00", "host": host_cpu()}
    t = time.perf_counter()
    res = [_oracle_scenario(j) for j in jobs]
    one = time.perf_counter() - t
    upd = sum(r[0] for r in res)
    out["one_process"] = {"seconds": one, "scenario_steps_per_s": len(sc) * n_steps / one,
                          "vehicle_updates_per_s": upd / one, "cores": 1}
    nproc = out["host"]["nproc"] or 1
    with mp.get_context("spawn").Pool(nproc) as pool:
        pool.map(_warm_worker, range(nproc))        # process start and imports, untimed
        t = time.perf_counter()
        res = pool.map(_oracle_scenario, jobs, chunksize=1)
        many = time.perf_counter() - t
    out["per_core_processes"] = {"seconds": many, "scenario_steps_per_s": len(sc) * n_steps / many,
                                 "vehicle_updates_per_s": sum(r[0] for r in res) / many, "cores": nproc}
    out["vehicle_updates"] = upd
    return out


def run_ensemble(args):
    """64 uneven what-if scenarios, one simulated hour each (07:00-08:00), run
    (a) batched: one simulation of the disjoint union.  On a first instance
        the autotuner times every launch shape of the step kernel (on the
        live run) and picks one; every timed instance is then advanced by
        replaying a CUDA graph captured for the whole hour (setup untimed);
    (b) sequential: one simulation per scenario, one after another, with
        plain step calls in the default shape.
    A bench step is one complete ensemble; value = scenarios/s of (a)."""
    import torch

    from paper_2007_03614_b300 import manta, synth
    from paper_2007_03614_b300.build import build
    rank, world = _dist()
    if rank != 0:
        return
    build()
    manta.load_library()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    sc = synth.ensemble_scenarios(n=args.scenarios)
    ens = synth.union(sc)
    t0 = int(7 * 3600 / 0.5)
    steps = 7200

    def make(net, tr):
        sim = manta.Sim(net, stream=stream, t0_step=t0, n_stats_windows=16)
        sim.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
        return sim

    def timed(fn):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        fn()
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / 1000.0

    # autotune on a first instance of the union (2 rounds of 300 steps per shape)
    sim = make(ens.net, ens.trips)
    chosen, tune_ms = sim.autotune(trial_steps=300, rounds=2)
    sim.close()
    shapes = manta.variants()
    batched, plain, upd = [], [], 0
    for it in range(args.warmup + args.steps):
        sim = make(ens.net, ens.trips)
        sim.variant = chosen
        gr = sim.graph(steps)
        dt = timed(lambda: gr.launch(1))
        if it >= args.warmup:
            batched.append(dt)
            upd = sim.stats()["vehicle_updates"]
        gr.close()
        sim.close()
        if it == args.warmup:
            # the same ensemble advanced by plain step calls, for comparison
            sim = make(ens.net, ens.trips)
            sim.variant = chosen
            plain.append(timed(lambda: sim.step(steps)))
            sim.close()
    seq = 0.0
    seq_upd = 0
    for net, tr in sc:
        sim = make(net, tr)
        seq += timed(lambda: sim.step(steps))
        seq_upd += sim.stats()["vehicle_updates"]
        sim.close()
    tb = sum(batched) / len(batched)
    n = len(sc)
    print(json.dumps({
        "metric": f"scenarios/s ({n} uneven what-if scenarios, 1 simulated hour each at dt = 0.5 s)",
        "value": n / tb, "unit": "scenarios/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * tb, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ensemble", "scenarios": n, "edges_total": int(ens.net.n_edges),
                   "trips_total": int(ens.trips.n_trips),
                   "edges_per_scenario": [int(x) for x in np.diff(ens.edge_off)],
                   "trips_per_scenario": [int(x) for x in np.diff(ens.trip_off)],
                   "sim_steps": steps, "t0_step": t0},
        "autotune": {"shapes": [list(x) for x in shapes],
                     "ms_per_million_updates": [float(x) for x in tune_ms], "trial_steps": 300, "rounds": 2,
                     "chosen": list(shapes[chosen])},
        "batched": {"seconds": tb, "scenarios_per_s": n / tb, "vehicle_updates": upd,
                    "vehicle_updates_per_s": upd / tb, "launch": "CUDA graph replay",
                    "plain_step_calls_seconds": plain[0] if plain else None},
        "sequential": {"seconds": seq, "scenarios_per_s": n / seq, "vehicle_updates": seq_upd,
                       "vehicle_updates_per_s": seq_upd / seq, "shape": list(shapes[0])},
        "batched_over_sequential": seq / tb,
        "batched_scenario_steps_per_s": n * steps / tb,
        "cpu_baseline": None if args.no_cpu_baseline else ensemble_cpu_baseline(sc, t0, args.ens_cpu_steps),
        "gpu_launches": args.steps * ((steps + 2047) // 2048)}))


def run_calibrate(args):
    """Calibration case: 20x20 grid (3 road classes), 20k trips over 20 min,
    3,600 steps; loss = mean squared error of the 5-minute link speeds against
    those of a hidden, seed-drawn parameter set.  Reports the time of one
    gradient (forward run with a checkpoint every 120 steps, then the
    checkpointed adjoint), the agreement of the adjoint with central finite
    differences (h = 1e-3) of the frozen-event replay of the whole run, and a
    few gradient steps from the default parameters."""
    import torch

    from paper_2007_03614_b300 import calibrate, manta, synth
    from paper_2007_03614_b300.build import build
    rank, world = _dist()
    if rank != 0:
        return
    build()
    manta.load_library()
    torch.cuda.set_device(0)
    net = synth.calib_network()
    tr = synth.calib_trips(net)
    steps, K = 3600, 120
    run = calibrate.LinkSpeedRun(net, tr, n_steps=steps, window_steps=600, checkpoint_every=K)
    rng = np.random.default_rng(2024)
    hidden = np.stack([rng.uniform(0.9, 1.1, 3), rng.uniform(1.0, 2.0, 3), rng.uniform(1.0, 2.5, 3),
                       rng.uniform(1.5, 3.5, 3), rng.uniform(1.5, 3.0, 3)], axis=1)
    with torch.no_grad():
        target = calibrate.link_speeds(torch.as_tensor(hidden), run).clone()
    obs = run.cnt > 0
    cfg = manta.default_config()
    theta0 = np.array([[cfg.v0f[c], cfg.T[c], cfg.a[c], cfg.b[c], cfg.s0[c]] for c in range(3)], np.float64)

    def loss_of(th):
        m = calibrate.link_speeds(th, run)
        return ((m - target)[obs] ** 2).mean()

    # timing of one gradient
    fw, bw = [], []
    for it in range(max(1, args.warmup) + max(1, args.steps)):
        th = torch.as_tensor(theta0).clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L = loss_of(th)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        upd = run.sim.stats()["vehicle_updates"]     # before the backward pass rewinds the run
        torch.cuda.synchronize()
        t1b = time.perf_counter()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if it >= max(1, args.warmup):
            fw.append(t1 - t0)
            bw.append(t2 - t1b)
    grad_ckpt = th.grad.detach().numpy().copy()
    with torch.no_grad():
        m_run = calibrate.link_speeds(torch.as_tensor(theta0), run).reshape(-1).clone()
    # finite differences of the frozen-event replay over the whole run
    dev = torch.device("cuda")
    g = manta.Sim(net, stream=run.stream, stats_window_steps=600, n_stats_windows=6)
    g.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
    g.tape_start(steps)
    g.step(steps)
    E, N = net.n_edges, tr.n_trips
    cnt = run.cnt.reshape(-1)
    obs_f = obs.reshape(-1)
    tgt = target.reshape(-1)

    def replay_loss(th):
        x = torch.zeros(N, dtype=torch.float64, device=dev)
        v = torch.zeros(N, dtype=torch.float64, device=dev)
        pr = torch.zeros(N, dtype=torch.uint8, device=dev)
        sums = torch.zeros(6 * E, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        g.replay(th, x, v, pr, sums)
        torch.cuda.synchronize()
        m = torch.where(obs_f, sums / cnt.clamp(min=1.0), torch.zeros_like(sums))
        return m, float(((m - tgt)[obs_f] ** 2).mean())

    m0, _ = replay_loss(theta0)
    seed = torch.where(obs_f, 2.0 * (m0 - tgt) / (obs_f.sum() * cnt.clamp(min=1.0)), torch.zeros_like(m0))
    lx = torch.zeros(N, dtype=torch.float64, device=dev)
    lv = torch.zeros(N, dtype=torch.float64, device=dev)
    gr = torch.zeros(40, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    ta = time.perf_counter()
    g.adjoint(seed.contiguous(), lx, lv, gr)
    torch.cuda.synchronize()
    adjoint_ms = 1000.0 * (time.perf_counter() - ta)
    adj = gr[:15].cpu().numpy().reshape(3, 5)
    # the same reverse sweep seeded from the run's own (fixed-point) means, as the
    # checkpointed backward pass is: the two must agree to rounding
    seed_run = torch.where(obs_f, 2.0 * (m_run - tgt) / (obs_f.sum() * cnt.clamp(min=1.0)), torch.zeros_like(m_run))
    lx.zero_(); lv.zero_()
    gr2 = torch.zeros(40, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    g.adjoint(seed_run.contiguous(), lx, lv, gr2)
    torch.cuda.synchronize()
    adj_run = gr2[:15].cpu().numpy().reshape(3, 5)
    fd = np.zeros((3, 5))
    h = 1e-3
    for c in range(3):
        for j in range(5):
            tp, tm = theta0.copy(), theta0.copy()
            tp[c, j] += h
            tm[c, j] -= h
            fd[c, j] = (replay_loss(tp)[1] - replay_loss(tm)[1]) / (2 * h)
    scale = float(np.max(np.abs(adj)))
    rel = np.abs(fd - adj) / np.maximum(np.abs(fd), 1e-3 * scale)
    g.close()
    # gradient steps from the default parameters with a backtracking line
    # search on the simulated (not frozen) loss: a step is taken only if it
    # lowers the loss, else the step length halves (the frozen-event gradient
    # is exact locally, but a step can move events)
    lo = np.array([0.5, 0.1, 1.0, 1.0, 1.0])
    hi = np.array([1.5, 2.0, 10.0, 10.0, 5.0])     # v0f, then the bounds of Section III-A
    th_np = theta0.copy()
    losses, accepted = [], []
    step = 0.2
    for _ in range(args.calib_iters):
        th = torch.as_tensor(th_np).clone().requires_grad_(True)
        L = loss_of(th)
        L.backward()
        Lv = float(L.detach())
        losses.append(Lv)
        d = -th.grad.numpy()
        d = d / max(np.max(np.abs(d)), 1e-30)
        took = None
        for _ in range(5):
            cand = np.clip(th_np + step * d, lo, hi)
            with torch.no_grad():
                Lc = float(loss_of(torch.as_tensor(cand)))
            if Lc < Lv:
                took = step
                th_np = cand
                break
            step *= 0.5
        accepted.append(took)
        if took is None:
            break
    with torch.no_grad():
        losses.append(float(loss_of(torch.as_tensor(th_np))))
    run.close()
    t_grad = float(np.mean(fw) + np.mean(bw))
    print(json.dumps({
        "metric": "calibration gradients/s (20x20 grid, 3 road classes, 20k trips, 3,600 steps, "
                  "checkpoint every 120 steps)",
        "value": 1.0 / t_grad, "unit": "gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_grad, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 simulation, f64 adjoint", "data": "synthetic",
        "config": {"workload": "calibrate", "edges": int(E), "trips": int(N), "sim_steps": steps,
                   "checkpoint_every": K, "windows": 6, "params": list(calibrate.PARAMS)},
        "forward_s": float(np.mean(fw)), "backward_s": float(np.mean(bw)), "vehicle_updates": int(upd),
        "adjoint_kernel_ms_full_tape": adjoint_ms,
        "fd_check": {"h": h, "max_rel_err": float(np.max(rel)), "adjoint": adj.tolist(), "fd": fd.tolist()},
        "checkpointed_vs_full_tape_max_rel": float(np.max(np.abs(grad_ckpt - adj_run) /
                                                          np.maximum(np.abs(adj_run), 1e-3 * scale))),
        "descent": {"method": "normalised gradient steps, backtracking on the simulated loss",
                    "loss": losses, "accepted_step": accepted, "hidden": hidden.tolist(),
                    "theta_final": th_np.tolist()},
        "gpu_launches": None}))


def hourly_speeds(sim, n_windows, mps_to_mph=2.2369362920544):
    """Per statistics window: mean over edges of each edge's mean speed, and
    the sample-weighted mean speed, in mph."""
    out = []
    for w in range(n_windows):
        ec = sim.edge_counters(w)
        s = ec["speed_sum"].astype(np.float64) / 1048576.0
        c = ec["speed_cnt"].astype(np.float64)
        m = c > 0
        out.append({"edge_mean_mph": float(np.mean(s[m] / c[m]) * mps_to_mph) if m.any() else None,
                    "sample_mean_mph": float(s.sum() / max(c.sum(), 1.0) * mps_to_mph),
                    "edges_observed": int(m.sum()), "samples": int(c.sum())})
    return out


def run_redgreen(args):
    """Section IV-C experiment on the metro-shaped workload: every node a
    flashing red (stop: 2 s stop, then one vehicle at a time in round robin)
    against every node green, same trips and routes, 05:00-12:00.  Reports
    hourly link speeds of both and the trend (red slower than green in the
    05:00-06:00 and 08:00-09:00 slices; both slower at the peak)."""
    import dataclasses

    import torch

    from paper_2007_03614_b300 import manta
    from paper_2007_03614_b300.build import build
    rank, world = _dist()
    if rank != 0:
        return
    build()
    manta.load_library()
    torch.cuda.set_device(0)
    net, tr = workload()
    stream = torch.cuda.Stream()
    res = {}
    for name, ntype in (("green", 0), ("red", 1)):
        n2 = dataclasses.replace(net, node_type=np.full_like(net.node_type, ntype))
        sim = manta.Sim(n2, stream=stream, t0_step=T0_STEP, stats_window_steps=7200, n_stats_windows=7)
        sim.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sim.step(50400)
        ev1.record(stream)
        ev1.synchronize()
        st = sim.stats()
        res[name] = {"wall_s": ev0.elapsed_time(ev1) / 1000.0, "stats": st, "hourly": hourly_speeds(sim, 7)}
        sim.close()
    g, r = res["green"]["hourly"], res["red"]["hourly"]
    trend = {
        "red_slower_05_06": r[0]["edge_mean_mph"] < g[0]["edge_mean_mph"],
        "red_slower_08_09": r[3]["edge_mean_mph"] < g[3]["edge_mean_mph"],
        "green_drop_05_06_to_08_09_mph": g[0]["edge_mean_mph"] - g[3]["edge_mean_mph"],
        "red_drop_05_06_to_08_09_mph": r[0]["edge_mean_mph"] - r[3]["edge_mean_mph"],
    }
    print(json.dumps({
        "metric": "Section IV-C red-light / green-light link speeds (metro-shaped morning)",
        "value": r[3]["edge_mean_mph"], "unit": "mph (red, 08:00-09:00, mean of edge means)", "n_gpus": 1,
        "steps": 1, "warmup": 0, "higher_is_better": True, "data": "synthetic",
        "config": {"workload": "redgreen", "hours": ["05-06", "06-07", "07-08", "08-09", "09-10", "10-11", "11-12"]},
        "green": res["green"], "red": res["red"], "trend": trend,
        "paper_mph": {"green": {"05-06": 24.5, "08-09": 17.8}, "red": {"05-06": 17.5, "08-09": 12.9}}}))


def run_search(args):
    """The paper's calibration loop (Section III-A) on the calibration case
    (20x20 grid, 20k trips, 3,600 steps): 5 parameter sets {a, b, T, s0} per
    iteration run batched as 5 copies of the network in one simulation,
    against link speeds of a hidden parameter set; also times the same 5 sets
    run one after another.  Drivers draw their own speed limit on every edge
    (Section IV-B) with sigma_s = --sigma-frac x the edge's limit."""
    import torch

    from paper_2007_03614_b300 import calibrate, manta, synth
    from paper_2007_03614_b300.build import build
    rank, world = _dist()
    if rank != 0:
        return
    build()
    manta.load_library()
    torch.cuda.set_device(0)
    net = synth.calib_network()
    tr = synth.calib_trips(net)
    steps, W = 3600, 6
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(2025)
    hidden = {"a": float(rng.uniform(1.0, 2.5)), "b": float(rng.uniform(1.5, 3.5)),
              "T": float(rng.uniform(1.0, 2.0)), "s0": float(rng.uniform(1.5, 3.0))}
    one = calibrate.copies(net, tr, 1)

    def single(th):
        g = manta.Sim(one.net, stream=stream, stats_window_steps=600, n_stats_windows=W, n_classes=1, v0f=[1.0],
                      a=[th["a"]], b=[th["b"]], T=[th["T"]], s0=[th["s0"]], speed_sigma_frac=args.sigma_frac)
        g.load_trips(one.trips.route_off, one.trips.route_edges, one.trips.depart_time_s)
        g.step(steps)
        out = calibrate.link_speed_cells(g, W, 0, int(net.n_edges))
        g.close()
        return out

    target, tcnt = single(hidden)
    cfg = manta.default_config()
    theta0 = {"a": cfg.a[0], "b": cfg.b[0], "T": cfg.T[0], "s0": cfg.s0[0]}
    t0 = time.perf_counter()
    res = calibrate.perturbation_search(net, tr, target, tcnt, theta0, iters=args.calib_iters, sets=5,
                                        n_steps=steps, window_steps=600, seed=1, stream=stream,
                                        speed_sigma_frac=args.sigma_frac)
    t_batched = (time.perf_counter() - t0) / len(res["history"])
    # the same five sets of the first iteration, one simulation each
    t1 = time.perf_counter()
    for c in range(5):
        single({k: v for k, v in theta0.items()})
    t_seq = time.perf_counter() - t1
    mph = 2.2369362920544
    print(json.dumps({
        "metric": "calibration iterations/s (Section III-A loop: 5 parameter sets per iteration, batched)",
        "value": 1.0 / t_batched, "unit": "iterations/s", "n_gpus": 1, "steps": len(res["history"]),
        "warmup": 0, "ms_per_step": 1000.0 * t_batched, "higher_is_better": True, "data": "synthetic",
        "config": {"workload": "search", "edges": int(net.n_edges), "trips": int(tr.n_trips), "sim_steps": steps,
                   "sets": 5, "windows": W, "speed_sigma_frac": args.sigma_frac},
        "seconds_per_iteration": {"batched_5_copies": t_batched, "sequential_5_runs": t_seq},
        "hidden": hidden, "start": theta0,
        "objective_mph": [h["objective"] * mph for h in res["history"]],
        "history": res["history"], "gpu_launches": None}))


def run_stress(args):
    """Stress configuration: the metro generator on ~3x the area (~1.6M
    edges), 10M trips departing 04:00-13:00 (bimodal), lane 0 closed on 200
    random freeway edges 07:30-09:00; the whole 9 h (64,800 steps) timed in
    launches of 1800 steps."""
    import torch

    from paper_2007_03614_b300 import manta, synth
    from paper_2007_03614_b300.build import build
    rank, world = _dist()
    if rank != 0:
        return
    build()
    manta.load_library()
    torch.cuda.set_device(0)
    tg = time.perf_counter()
    net = synth.stress_network()
    tr = synth.stress_trips(net)
    gen_s = time.perf_counter() - tg
    clo = synth.incident_closures(net)
    stream = torch.cuda.Stream()
    t0 = int(4 * 3600 / 0.5)
    steps = 64800
    sim = manta.Sim(net, stream=stream, t0_step=t0, stats_window_steps=7200, n_stats_windows=9)
    for (e, l, k0, k1) in clo:
        sim.set_lane_closure(e, l, k0, k1)
    sim.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    times = []
    with Clocks(0) as clk:
        for i in range(steps // args.chunk):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            sim.step(args.chunk)
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1) / 1000.0)
    d = sim.stats()
    el = float(sum(times))
    peak, peak_kind = _peaks()
    ab = algorithmic_bytes(d)
    hourly = hourly_speeds(sim, 9)
    sim.close()
    print(json.dumps({
        "metric": "vehicle-updates/s & wall-time of the 10M-trip megaregion day at dt=0.5 s; % HBM peak",
        "value": d["vehicle_updates"] / el, "unit": "vehicle-updates/s", "n_gpus": 1, "steps": len(times),
        "warmup": 0, "ms_per_step": 1000.0 * el / len(times), "higher_is_better": True, "data": "synthetic",
        "dtype": "f32",
        "config": {"workload": "stress: ~3x metro extent, 10M trips 04:00-13:00 bimodal, 200 freeway lane "
                               "closures 07:30-09:00", "edges": int(net.n_edges), "nodes": int(net.n_nodes),
                   "trips": int(tr.n_trips), "route_entries": int(tr.route_edges.size), "sim_steps": steps,
                   "t0_step": t0, "l2": "flushed between launches (256 MB write)"},
        "wall_s": el, "generation_s": gen_s, "counters": d,
        "roofline": {"bound": "hbm", "achieved": ab / el / 1e9, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": ab / el / 1e9 / peak, "algorithmic_bytes": int(ab)},
        "hourly": hourly, "clocks": clk.summary(), "gpu_launches": len(times)}))


def run_eq2(args):
    """Sensitivity of the morning to Eq. 2's length scale: the paper prints
    Eq. 2 without a unit for x (x0 = 1); the default reading takes metres,
    so lambda = 1 m and mandatory changes happen only a few metres before
    the node.  The metro-shaped morning (05:00-12:00) runs once per lambda
    in `--lambdas` on the same trips; reported per run: lane changes,
    gap-acceptance evaluations, clamps, arrivals, vehicles left at 12:00,
    hourly link speeds and device time."""
    import torch

    from paper_2007_03614_b300 import manta
    from paper_2007_03614_b300.build import build
    rank, world = _dist()
    if rank != 0:
        return
    build()
    manta.load_library()
    torch.cuda.set_device(0)
    net, tr = workload()
    stream = torch.cuda.Stream()
    runs = {}
    for lam in args.lambdas:
        sim = manta.Sim(net, stream=stream, t0_step=T0_STEP, stats_window_steps=7200, n_stats_windows=7,
                        lc_len_scale_m=float(lam))
        sim.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        left = MORNING_STEPS
        while left > 0:
            sim.step(min(1800, left))
            left -= 1800
        ev1.record(stream)
        ev1.synchronize()
        st = sim.stats()
        runs[str(lam)] = {"lc_len_scale_m": float(lam), "wall_s": ev0.elapsed_time(ev1) / 1000.0,
                          "updates_per_s": st["vehicle_updates"] / (ev0.elapsed_time(ev1) / 1000.0),
                          "stats": st, "hourly": hourly_speeds(sim, 7)}
        sim.close()
    print(json.dumps({
        "metric": "Eq. 2 length-scale sensitivity (metro-shaped morning 05:00-12:00)",
        "value": None, "unit": None, "n_gpus": 1, "steps": 1, "warmup": 0, "data": "synthetic",
        "config": {"workload": "eq2", "lambdas_m": [float(x) for x in args.lambdas], "sim_steps": MORNING_STEPS},
        "runs": runs}))


def run_reference(args):
    """The oracle (this paper has no reference code) on the dense peak-hour
    sample of peak_sample: each bench step is --ref-chunk oracle time steps."""
    rank, world = _dist()
    if rank != 0:
        return
    net, tr = workload()
    from oracle import oracle as O
    t0, sub, pl = peak_sample(net, tr)
    s = O.OracleSim(net, t0_step=t0, n_stats_windows=4)
    s.load_trips(sub.route_off, sub.route_edges, sub.depart_time_s)
    s.place_many(pl.trip, pl.route_pos, pl.lane, pl.x, pl.v)
    per = args.ref_chunk
    for _ in range(args.warmup):
        s.step(per)
    u0 = s.stats()["vehicle_updates"]
    t = time.perf_counter()
    for _ in range(args.steps):
        s.step(per)
    dt = time.perf_counter() - t
    upd = s.stats()["vehicle_updates"] - u0
    v = upd / dt
    sample = (f"dense peak-hour state on the metro network ({pl.n} vehicles placed at 07:30, {sub.n_trips} "
              f"trips loaded); each bench step = {per} oracle time steps")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * dt / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sim_steps_per_bench_step": per,
                   "sample": "the oracle on a bounded sample of the workload (see cpu_baseline.sample)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=25)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--chunk", type=int, default=1800)
    ap.add_argument("--impl", default="manta", choices=["manta", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=40)
    ap.add_argument("--ref-chunk", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="metro",
                    choices=["metro", "ensemble", "calibrate", "redgreen", "search", "stress", "eq2"])
    ap.add_argument("--lambdas", type=float, nargs="+", default=[1.0, 10.0, 100.0],
                    help="Eq. 2 length scales (m) of --workload eq2")
    ap.add_argument("--scenarios", type=int, default=64)
    ap.add_argument("--ens-cpu-steps", type=int, default=300,
                    help="steps per scenario of the ensemble's CPU oracle baseline")
    ap.add_argument("--calib-iters", type=int, default=6, help="gradient steps of --workload calibrate")
    ap.add_argument("--sigma-frac", type=float, default=0.05,
                    help="per-driver speed limits of --workload search: sigma_s / speed limit (Section IV-B)")
    ap.add_argument("--profile-case", action="store_true",
                    help="small case for ncu: 07:30-08:00 trips, 1200-step warm-up launch, then --steps launches")
    ap.add_argument("--profile-peak", action="store_true",
                    help="counter-capture case: the headline workload run to --profile-at, then --steps launches "
                         "of --chunk steps")
    ap.add_argument("--profile-at", type=float, default=7.75,
                    help="time of day (hours) at which --profile-peak starts its captured launches")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        raise SystemExit("need --steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "calibrate":
        run_calibrate(args)
    elif args.workload == "redgreen":
        run_redgreen(args)
    elif args.workload == "search":
        run_search(args)
    elif args.workload == "stress":
        run_stress(args)
    elif args.workload == "eq2":
        run_eq2(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
