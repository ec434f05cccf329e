"""Gradient of simulated link speeds with respect to the per-class IDM
parameters, for calibration (Section III-A; Eq. 1).

The paper calibrates a, b, T and s0 against link speeds by a random search.
Here the same objective gets an exact gradient along the simulated run:

- Every discrete event of the run is held fixed (leader gap and speed code,
  lane, signal and stop state, merge outcome, ballistic branch, clamp).
  The link speeds are then a smooth function of theta[c] = (v0f, T, a, b,
  s0) for each road class c.
- The forward pass runs the simulation and saves a device checkpoint every
  `checkpoint_every` steps.
- The backward pass works through the segments from last to first. It
  restores a segment's checkpoint, runs the segment again while recording
  its event tape, and sweeps the per-vehicle adjoint backward through it
  (manta_adjoint), carrying the adjoint of every vehicle's (x, v) from one
  segment to the previous one.
- Nothing but the checkpoints and one segment's tape is kept.

`link_speeds(theta, run)` is a torch.autograd.Function: it returns the mean
speed of every (statistics window, edge) cell, from the run's own
fixed-point speed sums.  A loss written in torch on those speeds
back-propagates to theta.  The derivative of a cell mean with respect to one
speed sample is 1 / count.
"""
from __future__ import annotations

import numpy as np

from . import manta

PARAMS = ("v0f", "T", "a", "b", "s0")


class LinkSpeedRun:
    """One simulated run whose link speeds are differentiated.

    net, trips: as for manta.Sim / Sim.load_trips.  The run covers n_steps
    steps from t0_step; statistics windows of window_steps steps (n_windows
    of them).  theta arrays are (n_classes, 5) in PARAMS order; other
    configuration fields pass through **cfg."""

    def __init__(self, net, trips, *, n_steps, t0_step=0, window_steps=600, n_windows=None,
                 checkpoint_every=120, stream=None, **cfg):
        import torch
        self.net, self.trips = net, trips
        self.n_steps = int(n_steps)
        self.t0 = int(t0_step)
        self.window_steps = int(window_steps)
        self.n_windows = int(n_windows if n_windows is not None else -(-self.n_steps // self.window_steps))
        self.K = int(checkpoint_every)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.cfg = dict(cfg)
        self.n_classes = int(self.cfg.pop("n_classes", int(np.max(net.edge_class)) + 1))
        self.sim = None
        self.ckpts = []
        self.cnt = None

    def _make_sim(self, theta):
        th = np.asarray(theta, dtype=np.float64).reshape(self.n_classes, 5)
        per = {name: [float(th[c, j]) for c in range(self.n_classes)] for j, name in enumerate(PARAMS)}
        sim = manta.Sim(self.net, stream=self.stream, t0_step=self.t0, stats_window_steps=self.window_steps,
                        n_stats_windows=self.n_windows, n_classes=self.n_classes, **per, **self.cfg)
        sim.load_trips(self.trips.route_off, self.trips.route_edges, self.trips.depart_time_s)
        return sim

    def close(self):
        for c, _ in self.ckpts:
            c.close()
        self.ckpts = []
        if self.sim is not None:
            self.sim.close()
            self.sim = None

    def forward(self, theta):
        """Runs the simulation with parameters theta; returns the mean speed
        and the sample count of every (window, edge) cell as CUDA float64
        tensors of shape (n_windows, n_edges)."""
        import torch
        self.close()
        self.sim = self._make_sim(theta)
        done = 0
        while done < self.n_steps:
            n = min(self.K, self.n_steps - done)
            self.ckpts.append((self.sim.checkpoint(), n))
            self.sim.step(n)
            done += n
        E = self.sim.n_edges
        ssum = np.zeros((self.n_windows, E), np.float64)
        cnt = np.zeros((self.n_windows, E), np.float64)
        for w in range(self.n_windows):
            ec = self.sim.edge_counters(w)
            ssum[w] = ec["speed_sum"].astype(np.float64) / 1048576.0
            cnt[w] = ec["speed_cnt"]
        mean = np.where(cnt > 0, ssum / np.maximum(cnt, 1.0), 0.0)
        dev = torch.device("cuda")
        self.cnt = torch.as_tensor(cnt, device=dev)
        return torch.as_tensor(mean, device=dev), self.cnt

    def backward(self, grad_mean):
        """dLoss/dtheta as a (n_classes, 5) float64 array, given dLoss/d(mean
        speed) of every cell (a (n_windows, n_edges) tensor)."""
        import torch
        assert self.sim is not None, "forward first"
        dev = torch.device("cuda")
        g = grad_mean.to(device=dev, dtype=torch.float64).contiguous()
        seed = torch.where(self.cnt > 0, g / self.cnt.clamp(min=1.0), torch.zeros_like(g)).reshape(-1).contiguous()
        N = max(self.sim.n_trips, 1)
        lam_x = torch.zeros(N, dtype=torch.float64, device=dev)
        lam_v = torch.zeros(N, dtype=torch.float64, device=dev)
        grad = torch.zeros(40, dtype=torch.float64, device=dev)
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            for ck, n in reversed(self.ckpts):
                self.sim.restore(ck)
                self.sim.tape_start(n)
                self.sim.step(n)
                self.sim.adjoint(seed, lam_x, lam_v, grad)
            self.sim.tape_stop()
        self.stream.synchronize()
        return grad[:5 * self.n_classes].reshape(self.n_classes, 5).cpu().numpy()


def _function():
    import torch

    class LinkSpeeds(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, run):
            mean, _ = run.forward(theta.detach().cpu().numpy())
            ctx.run = run
            ctx.meta = (theta.dtype, theta.device)
            return mean

        @staticmethod
        def backward(ctx, grad_mean):
            g = ctx.run.backward(grad_mean)
            dtype, device = ctx.meta
            return torch.as_tensor(g, dtype=dtype, device=device), None

    return LinkSpeeds


_LinkSpeeds = None


def link_speeds(theta, run: LinkSpeedRun):
    """Mean speed of every (window, edge) cell of `run` simulated with
    parameters theta (a (n_classes, 5) tensor, PARAMS order), differentiable
    with respect to theta."""
    global _LinkSpeeds
    if _LinkSpeeds is None:
        _LinkSpeeds = _function()
    return _LinkSpeeds.apply(theta, run)


# ------------------------------------------------------------------ random search
SEARCH_PARAMS = ("a", "b", "T", "s0")
# Section III-A: a, b in [1, 10] m/s^2, T in [0.1, 2] s, s0 in [1, 5] m
SEARCH_BOUNDS = {"a": (1.0, 10.0), "b": (1.0, 10.0), "T": (0.1, 2.0), "s0": (1.0, 5.0)}


def copies(net, trips, n):
    """Disjoint union of n copies of (net, trips) in which every edge of copy
    i carries road class i, so that copy i runs with the IDM parameters of
    class i.  Returns (Ensemble, edge offsets)."""
    from . import synth
    ens = synth.union([(net, trips)] * n)
    cls = np.zeros(ens.net.n_edges, np.uint8)
    for i in range(n):
        cls[ens.edge_off[i]:ens.edge_off[i + 1]] = i
    ens.net.edge_class = cls
    return ens


def link_speed_cells(sim, n_windows, edge_lo, edge_hi):
    """Mean speed and sample count of every (window, edge) cell of edges
    [edge_lo, edge_hi), as (n_windows, edges) arrays."""
    m = np.zeros((n_windows, edge_hi - edge_lo))
    c = np.zeros_like(m)
    for w in range(n_windows):
        ec = sim.edge_counters(w)
        s = ec["speed_sum"][edge_lo:edge_hi].astype(np.float64) / 1048576.0
        c[w] = ec["speed_cnt"][edge_lo:edge_hi]
        m[w] = np.where(c[w] > 0, s / np.maximum(c[w], 1.0), 0.0)
    return m, c


def perturbation_search(net, trips, target, target_cnt, theta0, *, iters=5, sets=5, r0=1.0, decay=0.1,
                        n_steps, t0_step=0, window_steps=600, n_windows=None, tol_mps=0.05 / 2.2369362920544,
                        seed=0, stream=None, **cfg):
    """The paper's calibration loop (Section III-A, Eq. 5).

    Every iteration runs `sets` parameter sets {a, b, T, s0} (one set for all
    vehicles): the current nominal and sets - 1 perturbations of it, each
    parameter moved by U[-r, r] and clipped to the bounds of Section III-A,
    with r = r0 at the first iteration and 10x smaller at each next one.  The
    sets run together as one simulation of the disjoint union of `sets` copies
    of the network and trips (copy i with the parameters of set i; the
    nominal runs in copy 0, whose trip ids, and so random draws, are those of
    a single run).  The objective of a set is the mean absolute difference
    between its link speeds and `target` over the (window, edge) cells observed
    in both (Eq. 5, the L1 norm over matched edges).  The best set becomes the
    next nominal; the loop stops early once the objective is below tol_mps
    (0.05 mph).

    theta0: dict of the four starting values.  target, target_cnt: (windows,
    edges) arrays of mean speeds (m/s) and sample counts.  Returns a dict with
    the nominal and objective after each iteration."""
    import torch
    rng = np.random.default_rng(seed)
    n_windows = int(n_windows if n_windows is not None else -(-int(n_steps) // int(window_steps)))
    stream = stream if stream is not None else torch.cuda.Stream()
    ens = copies(net, trips, sets)
    E = int(net.n_edges)
    nominal = {k: float(theta0[k]) for k in SEARCH_PARAMS}
    history = []
    r = float(r0)
    for it in range(iters):
        cand = [dict(nominal)]
        for _ in range(sets - 1):
            th = {}
            for k in SEARCH_PARAMS:
                lo, hi = SEARCH_BOUNDS[k]
                th[k] = float(np.clip(nominal[k] + rng.uniform(-r, r), lo, hi))
            cand.append(th)
        per = {k: [c[k] for c in cand] for k in SEARCH_PARAMS}
        sim = manta.Sim(ens.net, stream=stream, t0_step=t0_step, stats_window_steps=window_steps,
                        n_stats_windows=n_windows, n_classes=sets, v0f=[1.0] * sets, **per, **cfg)
        sim.load_trips(ens.trips.route_off, ens.trips.route_edges, ens.trips.depart_time_s)
        sim.step(int(n_steps))
        obj = []
        for i in range(sets):
            m, c = link_speed_cells(sim, n_windows, int(ens.edge_off[i]), int(ens.edge_off[i]) + E)
            both = (c > 0) & (target_cnt > 0)
            obj.append(float(np.mean(np.abs(m[both] - target[both]))) if both.any() else float("inf"))
        sim.close()
        best = int(np.argmin(obj))
        nominal = cand[best]
        history.append({"iteration": it, "range": r, "objective": obj[best], "objectives": obj,
                        "nominal": dict(nominal)})
        if obj[best] < tol_mps:
            break
        r *= decay
    return {"nominal": nominal, "history": history}
