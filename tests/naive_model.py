"""A deliberately naive, list-based statement of the simulation step.

No lane map: every neighbour query is an explicit search over the list of
vehicles (leader = nearest vehicle ahead along the route, lanes as lists).
It exists only to pin the oracle's lane-map indexing: on tiny networks the two
must agree bit for bit.  binary32 arithmetic via numpy float32 scalars.
"""
from __future__ import annotations

import math

import numpy as np

F = np.float32
M64 = (1 << 64) - 1


def _sm64(x):
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _key(seed, vid, k, stream):
    return _sm64(seed ^ ((vid * 0x9E3779B97F4A7C15) & M64) ^ ((k * 0xC2B2AE3D27D4EB4F) & M64) ^ stream)


def _u(seed, vid, k, stream):
    return F(_key(seed, vid, k, stream) >> 40) * F(2.0 ** -24)


def _n(seed, vid, k, s):
    acc = sum(_key(seed, vid, k, 16 * s + j) >> 40 for j in range(12))
    return F(acc - 6 * (1 << 24)) * F(2.0 ** -24)


def _code(v):
    return min(254, int(v * F(8.0) + F(0.5)))


class Veh:
    __slots__ = ("id", "e", "l", "x", "v", "r", "dwell", "status")


class Naive:
    def driver_limit(self, v):
        """Section IV-B: the driver's own limit on its current edge, s (1 + 2 f z)
        floored at s / 4, z the normal draw of stream 4 keyed by the global
        route entry; the edge's limit s when f = 0."""
        s = self.lim[v.e]
        f = F(self.cfg.get("speed_sigma_frac", 0.0))
        if not f > F(0.0):
            return s
        z = _n(self.cfg["seed"], v.id, self.roff[v.id] + v.r, 4)
        q = F(1.0) + (F(2.0) * f) * z
        if q < F(0.25):
            q = F(0.25)
        return s * q

    def __init__(self, net, tr, cfg):
        self.cfg = cfg
        L = cfg["veh_len_cells"]
        s0max = max(cfg["s0"][: cfg["n_classes"]])
        cmin = L + math.ceil(s0max) + 1
        self.E = len(net.edge_src)
        self.src, self.dst = list(map(int, net.edge_src)), list(map(int, net.edge_dst))
        self.nl = list(map(int, net.edge_lanes))
        self.cls = list(map(int, net.edge_class))
        self.lim = [F(x) for x in net.edge_speed_limit_mps]
        self.C = [max(cmin, int(np.floor(float(x) + 0.5))) for x in net.edge_length_m]
        self.ntype = list(map(int, net.node_type))
        self.ncyc = list(map(int, net.node_cycle_steps))
        self.noff = list(map(int, net.node_offset_steps))
        self.gs, self.gl = list(map(int, net.edge_green_start)), list(map(int, net.edge_green_len))
        # lane masks by (in-edge, out-edge)
        self.mask = {}
        outs = {n: sorted(e for e in range(self.E) if self.src[e] == n) for n in range(len(self.ntype))}
        j = 0
        for e in range(self.E):
            for e2 in outs[self.dst[e]]:
                m = (1 << self.nl[e]) - 1
                if net.conn_lane_mask is not None:
                    m &= int(net.conn_lane_mask[j])
                self.mask[(e, e2)] = m
                j += 1
        self.inlanes = {n: [(e, l) for e in range(self.E) if self.dst[e] == n for l in range(self.nl[e])]
                        for n in range(len(self.ntype))}
        self.closures = {}                      # (edge, lane) -> (k0, k1)
        self.permit = {n: None for n in range(len(self.ntype))}
        self.rr = {n: 0 for n in range(len(self.ntype))}
        self.roff = list(map(int, tr.route_off))
        self.routes = [list(map(int, tr.route_edges[tr.route_off[i]:tr.route_off[i + 1]]))
                       for i in range(len(tr.depart_time_s))]
        self.dstep = [math.ceil(float(t) / float(cfg["dt"])) for t in tr.depart_time_s]
        self.V = []
        for i in range(len(self.routes)):
            v = Veh()
            v.id, v.status, v.dwell = i, 0, 0
            self.V.append(v)
        self.departed_flag = [False] * len(self.routes)
        self.k = cfg["t0_step"]
        self.st = dict(departed=0, arrived=0, vehicle_updates=0, cells_scanned=0, clamps=0,
                       lane_changes=0, lc_evals=0, route_reads=0, lc_cells_scanned=0)
        self.entry = [0] * self.E
        self.exit = [0] * self.E

    # ------------------------------------------------------------ helpers --
    def on(self):
        return [v for v in self.V if v.status == 1]

    def cell(self, v):
        return int(np.floor(v.x))

    def in_lane(self, e, l):
        return [w for w in self.on() if w.e == e and w.l == l]

    def green(self, e, k):
        n = self.dst[e]
        if self.ntype[n] != 2:
            return True
        m = (k - self.noff[n]) % self.ncyc[n]
        return self.gs[e] <= m < self.gs[e] + self.gl[e]

    def closed(self, e, l, k):
        w = self.closures.get((e, l))
        return w is not None and w[0] <= k < w[1]

    def next_edge(self, v):
        r = self.routes[v.id]
        return r[v.r + 1] if v.r + 1 < len(r) else None

    # ----------------------------------------------------------- lane change --
    def _scan_up(self, occ, lo, hi):
        """First occupied cell in [lo, hi] of a lane whose occupied front cells
        are `occ` (None if none); the cells an upward scan reads to find it
        are added to lc_cells_scanned."""
        hits = [c for c in occ if lo <= c <= hi]
        hit = min(hits) if hits else None
        self.st["lc_cells_scanned"] += (hit - lo + 1) if hit is not None else max(0, hi - lo + 1)
        return hit

    def _scan_down(self, occ, hi, lo):
        """Last occupied cell in [lo, hi] (None if none), counted as a
        downward scan from hi."""
        hits = [c for c in occ if lo <= c <= hi]
        hit = max(hits) if hits else None
        self.st["lc_cells_scanned"] += (hi - hit + 1) if hit is not None else max(0, hi - lo + 1)
        return hit

    def lc_decide(self, v, k):
        c = self.cfg
        L, H = c["veh_len_cells"], c["horizon_cells"]
        e, l = v.e, v.l
        if self.nl[e] < 2:
            return None
        d = 1 if k % 2 == 0 else -1
        lt = l + d
        if lt < 0 or lt >= self.nl[e]:
            return None
        if self.closed(e, lt, k):
            return None
        cell = self.cell(v)
        e2 = self.next_edge(v)
        mask = self.mask[(e, e2)] if e2 is not None else 0xFF
        if e2 is not None:
            open_ = 0
            for q in range(self.nl[e]):
                if not self.closed(e2, min(q, self.nl[e2] - 1), k):
                    open_ |= 1 << q
            if mask & open_:
                mask &= open_
        ok_l, ok_lt = (mask >> l) & 1, (mask >> lt) & 1
        obst = self.C[e] // 2
        closed_here = self.closed(e, l, k) and cell < obst
        mandatory = False
        if closed_here:
            mandatory = True
        elif e2 is not None and not ok_l:
            up = [q - l for q in range(l + 1, self.nl[e]) if (mask >> q) & 1]
            dn = [l - q for q in range(0, l) if (mask >> q) & 1]
            dp = min(up) if up else 99
            dm = min(dn) if dn else 99
            toward = (dp < 99 and dp <= dm) if d > 0 else (dm < 99 and dm <= dp)
            if not toward:
                return None
            mandatory = True
        elif not ok_lt:
            return None
        hi = min(cell + H, self.C[e] - 1)
        target = self.in_lane(e, lt)
        if mandatory:
            dist = (obst - 1 - cell) if closed_here else (self.C[e] - 1 - cell)
            xm = float(dist) * float(c["cell_m"])
            x0, lam = float(F(c["lc_x0_m"])), float(F(c["lc_len_scale_m"]))
            m = 1.0 if xm <= x0 else math.exp(-((xm - x0) / lam) ** 2)
            if not (_u(c["seed"], v.id, k, 0) < F(m)):
                return None
        else:
            if not (v.v > 0):
                return None            # a stopped vehicle has no slower leader
            co = self._scan_up([self.cell(w) for w in self.in_lane(e, l)], cell + 1, hi)
            if co is None:
                return None
            lv = [w for w in self.in_lane(e, l) if self.cell(w) == co][0]
            if not (F(_code(lv.v)) * F(0.125) < v.v):
                return None
            own_gap = co - L - cell
            ta = self._scan_up([self.cell(w) for w in target], cell + L, hi)
            if ta is not None and not (ta - L - cell > own_gap):
                return None
        self.st["lc_evals"] += 1
        tcells = [self.cell(w) for w in target]
        if self._scan_up(tcells, max(0, cell - L + 1), min(cell + L - 1, self.C[e] - 1)) is not None:
            return None                # lateral overlap
        ca = self._scan_up(tcells, cell + L, hi)
        cb = self._scan_down(tcells, cell - L, max(0, cell - H))
        lead = [w for w in target if self.cell(w) == ca] if ca is not None else []
        lag = [w for w in target if self.cell(w) == cb] if cb is not None else []
        g = F(c["g_low"]) if v.v < F(c["g_speed_split"]) else F(c["g_high"])
        alpha = F(c["alpha_lo"]) + (F(c["alpha_hi"]) - F(c["alpha_lo"])) * _u(c["seed"], v.id, 0, 3)
        if lead:
            a = min(lead, key=self.cell)
            va = F(_code(a.v)) * F(0.125)
            t = g + alpha * v.v
            t = t + alpha * (v.v - va)
            glead = max(g, t) + _n(c["seed"], v.id, k, 1)
            if not (F(self.cell(a) - L - cell) >= glead):
                return None
        if lag:
            b = max(lag, key=self.cell)
            vb = F(_code(b.v)) * F(0.125)
            t = g + alpha * v.v
            t = t + alpha * (v.v - vb)
            glag = max(g, t) + _n(c["seed"], v.id, k, 2)
            if not (F(cell - L - self.cell(b)) >= glag):
                return None
        return lt

    # ------------------------------------------------------------- leader --
    def leader(self, v, k):
        """Nearest event ahead along the route: a vehicle, a holding node or the
        route end; found by searching every vehicle on the route's lanes."""
        c = self.cfg
        L, H = c["veh_len_cells"], c["horizon_cells"]
        cell = self.cell(v)
        limit = cell + H
        route = self.routes[v.id]
        segs = []           # (edge, lane, base, route index)
        base, lane, r = 0, v.l, v.r
        while True:
            e = route[r]
            segs.append((e, lane, base, r))
            base += self.C[e]
            if base > limit or r + 1 >= len(route):
                break
            r += 1
            lane = min(lane, self.nl[route[r]] - 1)
        best_p, best_w = None, None
        for w in self.on():
            # the vehicle itself counts when its route comes back to its own lane
            # within the horizon: the lane map holds no identities
            for (e, l, b, _) in segs:
                if w.e == e and w.l == l:
                    p = b + self.cell(w)
                    if cell < p <= limit and (best_p is None or p < best_p):
                        best_p, best_w = p, w
        reads = 0
        out = dict(kind="free", reached_own=False, stop_only=False)
        e0, l0 = segs[0][0], segs[0][1]
        obst = self.C[e0] // 2
        if self.closed(e0, l0, k) and cell < obst and obst <= limit and (best_p is None or best_p >= obst):
            out.update(kind="virtual", cL=obst + L - 1, vL=F(0.0))
            self.st["cells_scanned"] += obst - 1 - cell
            return out
        for si, (e, l, b, r) in enumerate(segs):
            B = b + self.C[e]
            if best_p is not None and best_p < B:
                break
            if B > limit:
                break
            if r + 1 >= len(route):
                out["end"] = B
                break
            reads += 1
            n = self.dst[e]
            nxt = route[r + 1]
            blocked = self.ntype[n] == 2 and not self.green(e, k)
            if self.closed(nxt, min(l, self.nl[nxt] - 1), k):
                blocked = True
            if si == 0:
                stop_np = self.ntype[n] == 1 and self.permit[n] != v.id
                out["reached_own"] = True
                out["stop_only"] = stop_np
                blocked = blocked or stop_np
            elif self.ntype[n] == 1:
                blocked = True
            if blocked:
                out.update(kind="virtual", cL=B + L - 1, vL=F(0.0))
                self.st["cells_scanned"] += B - 1 - cell
                self.st["route_reads"] += reads
                return out
        self.st["route_reads"] += reads
        if best_p is not None and (out.get("end") is None or best_p < out["end"]):
            out.update(kind="leader", cL=best_p, vL=F(_code(best_w.v)) * F(0.125))
            self.st["cells_scanned"] += best_p - cell
            return out
        if out.get("end") is not None:
            self.st["cells_scanned"] += out["end"] - 1 - cell
        else:
            self.st["cells_scanned"] += H
        out["kind"] = "free"
        return out

    # --------------------------------------------------------------- step --
    def step(self):
        c = self.cfg
        k = self.k
        L = c["veh_len_cells"]
        dt = F(c["dt"])
        on = self.on()
        dec = {v.id: self.lc_decide(v, k) for v in on}
        for v in on:
            if dec[v.id] is not None:
                v.l = dec[v.id]
                self.st["lane_changes"] += 1
        deps = {}
        for e in range(self.E):
            cand = [i for i in range(len(self.routes)) if self.routes[i][0] == e and self.V[i].status == 0]
            if not cand:
                continue
            j = min(cand, key=lambda i: (self.dstep[i], i))
            if self.dstep[j] > k:
                continue
            if self.closed(e, 0, k):
                continue
            need = min(self.C[e], L + math.ceil(float(F(c["s0"][self.cls[e]]))))
            if any(self.cell(w) < need for w in self.in_lane(e, 0)):
                continue
            deps[e] = j
        upd = {}
        for v in on:
            e = v.e
            p = self.cls[e]
            a, b, T, s0 = F(c["a"][p]), F(c["b"][p]), F(c["T"][p]), F(c["s0"][p])
            v0 = self.driver_limit(v) * F(c["v0f"][p])
            cell = self.cell(v)
            ld = self.leader(v, k)
            r1 = v.v / v0
            r2 = r1 * r1
            r4 = r2 * r2
            stop = False
            acc = F(0.0)
            if ld["kind"] == "free":
                acc = a * (F(1.0) - r4)
            else:
                s = F(ld["cL"] - cell - L)
                if s <= F(0.0):
                    stop = True
                else:
                    dv = v.v - ld["vL"]
                    dyn = (v.v * dv) / (F(2.0) * np.sqrt(a * b))
                    if c["idm_textbook"]:
                        ss = s0 + max(F(0.0), v.v * T + dyn)
                    else:
                        ss = (s0 + v.v * T) + dyn
                    q = ss / s
                    acc = a * ((F(1.0) - r4) - q * q)
            if stop:
                xn, vn = v.x, F(0.0)
            else:
                vt = v.v + acc * dt
                if vt >= F(0.0):
                    xt = v.x + (v.v * dt + (F(0.5) * acc) * (dt * dt))
                    vv = vt
                else:
                    xt = v.x - (v.v * v.v) / (F(2.0) * acc)
                    vv = F(0.0)
                bnd = None
                if ld["kind"] != "free":
                    bnd = ld["cL"] - L
                e2 = self.next_edge(v)
                if e2 is not None:
                    cap = self.C[e] + self.C[e2] - 1
                    if bnd is None or cap < bnd:
                        bnd = cap
                if bnd is not None and xt > F(bnd):
                    xn, vn = max(v.x, F(bnd)), F(0.0)
                    self.st["clamps"] += 1
                else:
                    xn, vn = xt, vv
            dwn = 0
            last = self.next_edge(v) is None
            zone = self.C[e] - 1 - (math.ceil(float(s0)) + 2)
            if (not last) and ld["reached_own"] and ld["stop_only"] and int(np.floor(xn)) >= zone \
                    and vn < F(c["stop_v_eps"]):
                dwn = min(255, v.dwell + 1)
            kind, tgt = "stay", None
            if xn >= F(self.C[e]):
                e2 = self.next_edge(v)
                if e2 is None:
                    kind = "arrive"
                else:
                    kind, tgt = "cross", (e2, min(v.l, self.nl[e2] - 1))
            upd[v.id] = (xn, vn, dwn, kind, tgt)
        reqs = {}
        for i, u in upd.items():
            if u[3] == "cross":
                reqs.setdefault(u[4], []).append(i)
        for e, j in deps.items():
            reqs.setdefault((e, 0), []).append(j)
        winners = {t: min(ids) for t, ids in reqs.items()}
        w = (k - c["t0_step"]) // c["stats_window_steps"]
        sums = getattr(self, "ssum", {})
        self.ssum = sums
        for v in on:
            xn, vn, dwn, kind, tgt = upd[v.id]
            if kind == "arrive":
                v.status = 2
                self.exit[v.e] += 1
                self.st["arrived"] += 1
                continue
            if kind == "cross":
                if winners[tgt] == v.id:
                    n = self.dst[v.e]
                    if self.ntype[n] == 1 and self.permit[n] == v.id:
                        self.permit[n] = None
                    self.exit[v.e] += 1
                    self.entry[tgt[0]] += 1
                    v.x = xn - F(self.C[v.e])
                    v.e, v.l = tgt
                    v.r += 1
                    v.v, v.dwell = vn, 0
                else:
                    v.x = max(v.x, F(self.C[v.e] - 1))
                    v.v, v.dwell = F(0.0), dwn
            else:
                v.x, v.v, v.dwell = xn, vn, dwn
            if k >= c["t0_step"] and w < c["n_stats_windows"]:
                key = (w, v.e)
                s_, n_ = sums.get(key, (0, 0))
                sums[key] = (s_ + int(v.v * F(1048576.0)), n_ + 1)
        for e, j in deps.items():
            if winners[(e, 0)] != j:
                continue
            v = self.V[j]
            v.e, v.l, v.x, v.v, v.r, v.dwell, v.status = e, 0, F(0.0), F(0.0), 0, 0, 1
            self.entry[e] += 1
            self.st["departed"] += 1
        self.st["vehicle_updates"] += len(on)
        # stop permits for k + 1
        for n in range(len(self.ntype)):
            if self.ntype[n] != 1 or self.permit[n] is not None:
                continue
            lanes = self.inlanes[n]
            m = len(lanes)
            for t in range(m):
                idx = (self.rr[n] + t) % m
                e, l = lanes[idx]
                here = self.in_lane(e, l)
                if not here:
                    continue
                h = max(here, key=lambda q: q.x)
                if h.dwell >= c["stop_dwell_steps"]:
                    self.permit[n] = h.id
                    self.rr[n] = (idx + 1) % m
                    break
        self.k = k + 1

    def snapshot(self):
        on = sorted(self.on(), key=lambda q: q.id)
        return dict(id=np.array([q.id for q in on], np.uint32), x=np.array([q.x for q in on], np.float32),
                    v=np.array([q.v for q in on], np.float32), edge=np.array([q.e for q in on], np.int32),
                    lane=np.array([q.l for q in on], np.uint8), dwell=np.array([q.dwell for q in on], np.uint8),
                    route_pos=np.array([q.r for q in on], np.int32))
