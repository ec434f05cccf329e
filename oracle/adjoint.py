"""Reference adjoint of simulated link speeds with respect to the per-class
IDM parameters, on the CPU, in binary64 (calibration, Section III; Eq. 1).

TEST INFRASTRUCTURE.  Only tests/ may use it.  It reads the oracle's own event
tape (OracleSim.record_tape) and shares nothing with the CUDA library.

Along a recorded run every discrete event is held fixed: the leader gap and
speed (the lane map holds integer cells and speed codes), lane choice, signal
and stop state, merge outcome, ballistic branch and clamp.  Each vehicle's
state then follows, step by step,

    acc = a (1 - (v/v0)^4)                                   free road
    acc = a (1 - (v/v0)^4 - (s*/s)^2),
          s* = s0 + v T + v (v - vL) / (2 sqrt(a b))         behind a leader (Eq. 1, delta = 4)
    (x, v) <- (x + v dt + acc dt^2 / 2, v + acc dt)          if v + acc dt >= 0
    (x, v) <- (x - v^2 / (2 acc), 0)                         otherwise (ballistic step)

then the recorded clamp (old position kept, or set to the bound, with speed
0) and node outcome (crossed: x - C; held: old x or C - 1 with speed 0;
arrived: leaves), with v0 = speed limit * v0f of the edge's class.  The
parameters are theta[c] = (v0f, T, a, b, s0) for road class c.

`replay` runs the recorded events forward with any theta (used for finite
differences); `adjoint` carries dLoss/d(x, v) backward through the same steps.
The loss sees the run only through its speed samples (one per vehicle-step
in a statistics cell after the step); `seed` holds dLoss/d(sample).
"""
import numpy as np

PARAMS = ("v0f", "T", "a", "b", "s0")


def _unpack(flags):
    present = (flags & 1) != 0
    kind = (flags >> 1) & 3          # 0 free, 1 interacting, 2 stopped in place
    ballistic = (flags >> 3) & 1
    clamp = (flags >> 4) & 3         # 0 none, 1 old position kept, 2 bound
    outcome = (flags >> 6) & 7       # 0 stayed, 1 crossed, 2 held (old x), 3 held (stop line), 4 arrived
    cls = (flags >> 9) & 7
    return present, kind, ballistic, clamp, outcome, cls


def acceleration(theta, cls, lim, v, interact, s, vL):
    """Eq. 1 acceleration and its derivatives: returns acc, dacc/dv and
    dacc/dtheta (array (5, n) in PARAMS order) for vectors of vehicles."""
    th = np.asarray(theta, dtype=np.float64)
    v0f, T, a, b, s0 = (th[cls, j] for j in range(5))
    v0 = lim * v0f
    r = v / v0
    acc = a * (1.0 - r ** 4)
    dv = -4.0 * a * r ** 3 / v0
    dth = np.zeros((5,) + v.shape)
    dth[0] = 4.0 * a * r ** 4 / v0 * lim
    dth[2] = 1.0 - r ** 4
    if np.any(interact):
        D = 2.0 * np.sqrt(a * b)
        dyn = v * (v - vL) / D
        ss = s0 + v * T + dyn
        safe_s = np.where(interact, s, 1.0)
        q = ss / safe_s
        m = interact.astype(np.float64)
        acc = acc - m * a * q * q
        dq = -2.0 * a * q / safe_s * m          # d(-a q^2) per unit change of s*
        dv = dv + dq * (T + (2.0 * v - vL) / D)
        dth[1] += dq * v
        dth[2] += -m * q * q + dq * (-dyn / (2.0 * a))
        dth[3] += dq * (-dyn / (2.0 * b))
        dth[4] += dq
    return acc, dv, dth


def replay(tape, theta, dt, n_cells, x0=None, v0=None, present0=None):
    """Frozen-event replay: returns (sums of replayed sample speeds per
    statistics cell, final x, v, present)."""
    T, N = tape["flags"].shape
    x = np.zeros(N) if x0 is None else x0.copy()
    v = np.zeros(N) if v0 is None else v0.copy()
    prev = np.zeros(N, bool) if present0 is None else present0.copy()
    sums = np.zeros(n_cells)
    for t in range(T):
        present, kind, ball, clamp, out, cls = _unpack(tape["flags"][t])
        enter = present & ~prev
        x = np.where(enter, tape["x"][t].astype(np.float64), x)
        v = np.where(enter, tape["v"][t].astype(np.float64), v)
        lim = np.where(present, tape["lim"][t].astype(np.float64), 1.0)
        acc, _, _ = acceleration(theta, cls, lim, v, kind == 1,
                                 tape["s"][t].astype(np.float64), tape["vL"][t].astype(np.float64))
        moving = (kind != 2) & (clamp == 0)
        with np.errstate(divide="ignore", invalid="ignore"):
            xb = np.where(ball == 1, x + v * dt + 0.5 * acc * dt * dt, x - v * v / (2.0 * acc))
        vb = np.where(ball == 1, v + acc * dt, 0.0)
        xp = np.where(moving, xb, np.where(clamp == 2, tape["bnd"][t].astype(np.float64), x))
        vp = np.where(moving, vb, 0.0)
        C = tape["C"][t].astype(np.float64)
        xn = np.select([out == 1, out == 2, out == 3], [xp - C, x, C - 1.0], xp)
        vn = np.where((out == 0) | (out == 1), vp, 0.0)
        keep = present & (out != 4)
        smp = tape["sample"][t]
        use = keep & (smp >= 0) & ((out == 0) | (out == 1))
        np.add.at(sums, smp[use], vn[use])
        x = np.where(keep, xn, x)
        v = np.where(keep, vn, v)
        prev = keep
    return sums, x, v, prev


def adjoint(tape, theta, dt, seed, n_classes, lam_x=None, lam_v=None):
    """Reverse sweep: returns (dLoss/dtheta as (n_classes, 5), adjoint of the
    state entering the tape)."""
    T, N = tape["flags"].shape
    lx = np.zeros(N) if lam_x is None else lam_x.copy()
    lv = np.zeros(N) if lam_v is None else lam_v.copy()
    grad = np.zeros((n_classes, 5))
    for t in range(T - 1, -1, -1):
        present, kind, ball, clamp, out, cls = _unpack(tape["flags"][t])
        live = present & (out != 4)
        smp = tape["sample"][t]
        sampled = live & (smp >= 0) & ((out == 0) | (out == 1))
        lv = lv + np.where(sampled, seed[np.maximum(smp, 0)], 0.0)
        passes = (out == 0) | (out == 1)                      # the step's result carries on
        lxp = np.where(live & passes, lx, 0.0)
        lvp = np.where(live & passes, lv, 0.0)
        lx0 = np.where(live & (out == 2), lx, 0.0)            # held: keeps its old position
        lv0 = np.zeros(N)
        x_kept = live & ((kind == 2) | (clamp == 1))          # x' = x, v' = 0
        lx0 = lx0 + np.where(x_kept, lxp, 0.0)
        moving = live & (kind != 2) & (clamp == 0)
        v = tape["v"][t].astype(np.float64)
        lim = np.where(present, tape["lim"][t].astype(np.float64), 1.0)
        acc, dv, dth = acceleration(theta, cls, lim, v, kind == 1,
                                    tape["s"][t].astype(np.float64), tape["vL"][t].astype(np.float64))
        with np.errstate(divide="ignore", invalid="ignore"):
            ga = np.where(ball == 1, lxp * 0.5 * dt * dt + lvp * dt, lxp * v * v / (2.0 * acc * acc))
            dlv = np.where(ball == 1, lxp * dt + lvp, lxp * (-v / acc))
        ga = np.where(moving, ga, 0.0)
        lx0 = lx0 + np.where(moving, lxp, 0.0)
        lv0 = lv0 + np.where(moving, dlv + ga * dv, 0.0)
        for j in range(5):
            np.add.at(grad[:, j], cls[moving], (ga * dth[j])[moving])
        lx = np.where(present, lx0, 0.0)
        lv = np.where(present, lv0, 0.0)
    return grad, lx, lv
