"""FP64 three-weight ADMM iteration over the planning factor graph
(test infrastructure only).

Factor graph (Section 3.3): one equality node per break-point variable
x_i(s), i in [p], s = 0..eta.  Nodes s = 0 and s = eta hold the fixed start
and goal; each carries a position factor that always sends weight infinity
(the endpoints are constants, Section 3).  Minimizer nodes:

* kinetic factor (i, s), s < eta: f = c_{i,s} |x_i(s) - x_i(s+1)|^2 with
  c_{i,s} = C_{i,s} / (p eta) (Eq. velo_cost_pair_wise); weight rho0 always;
* collision factor (s, i < j): f^coll_{r_i, r_j} on the four nodes
  (i,s), (i,s+1), (j,s), (j,s+1) (Eq. f_coll_def); weight 0 or rho0;
* wall factor (w, i, s): f^wall for wall w (Eq. wall_minimizer); 0 or rho0;
* optional maximum / minimum velocity factors (i, s): |x_i(s) - x_i(s+1)|
  <= vmax_{i,s} or >= vmin_{i,s} (Eq. max_vel_min and the reversed
  inequality, Appendices F and G); 0 or rho0.

``energy=False`` drops the kinetic factors: the feasibility problem of
Eq. basic_opt_prob (Section 4 compares it with the energy problem), where
break-points can receive only zero weights.

``vo=True`` is the local planner of Section 5 (Eq. unconst_opt_RVO through
the minimizers of Appendix H) on eta = 2 break-point segments: s = 0 holds the
current positions x_i(0) (fixed), s = 1 the positions x_i after one epoch
(free), s = 2 the reference positions x_ref_i (fixed, in ``goal``).  The
collision, wall and velocity factors exist on segment 0 only (Eqs.
minimizer_rvo_coll and minimizer_rvo_wall: g^coll and g^wall with the x(0)
end fixed), the kinetic factor on segment 1 only, where it is
C'_i |x_i - x_ref_i|^2 (Eq. minimizer_rvo_cost: g^cost with the x_ref end
fixed); C'_i comes from ``cost[:, 1]`` (with ``cost_unnorm``).

One iteration is the seven steps of Appendix B, in order.  Readings where the
text is silent or its figure is missing (the special u and back-weight rules of
Fig. special_update_rules):

* back weights (step 6): infinity at a node if any incoming weight is
  infinity; 0 if all incoming weights are 0; rho0 otherwise;
* u step (step 7): u += alpha (x - z) on an edge whose forward and back
  weights are both rho0 (the scaled-dual form; identical to the printed
  alpha/rho0 form when rho0 = 1), or u += (alpha / rho0) (x - z) as printed
  under ``u_literal``, rho0 being the value in force in that iteration (the
  warm-up value during the warm-up); every other edge resets u to 0, or keeps
  u unchanged under ``u_keep``;
* ties inside a minimizer go to the lowest energy, then the smallest angle
  (see ``oracle.prox``);
* initial state: z = start for every break-point except the goal node,
  u = 0, back weights rho0 inside and infinity at the fixed ends;
* standard-ADMM mode (``admm``): Appendix B notes that with every weight at
  rho0 the method is classical ADMM.  Collision and wall factors then always
  send rho0 (their minimizer still returns x = n when the n-trajectories are
  feasible); the fixed ends stay constants with weight infinity.

Weights are kept as classes 0 (zero), 1 (rho0), 2 (infinity).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

from . import prox

W0, WR, WI = 0, 1, 2
INF = math.inf


@dataclass
class Problem:
    p: int
    eta: int
    start: np.ndarray          # (p, 2)
    goal: np.ndarray           # (p, 2)
    radius: np.ndarray         # (p,)
    cost: np.ndarray           # (p, eta) C_{i,s}
    walls: np.ndarray          # (n_walls, 4)
    rho0: float = 1.0
    alpha: float = 0.1
    u_keep: bool = False
    u_literal: bool = False     # u step (alpha / rho0)(x - z) as printed in App. B step 7
    cost_unnorm: bool = False
    admm: bool = False          # standard ADMM: every factor always sends rho0
    energy: bool = True         # kinetic-energy factors present
    vmax: np.ndarray | None = None   # (p, eta) limits of |x(s+1) - x(s)|, or None
    vmin: np.ndarray | None = None
    vo: bool = False            # one-epoch velocity-obstacle problem (Section 5), eta = 2
    warm_iters: int = 0
    warm_rho: float = 0.0

    @property
    def n_walls(self):
        return int(self.walls.shape[0])

    def c(self):
        """Per-factor kinetic coefficients c_{i,s}, shape (p, eta)."""
        if self.cost_unnorm:
            return self.cost.astype(np.float64)
        return self.cost.astype(np.float64) / (self.p * self.eta)

    def rho_at(self, k):
        """rho0 in force at iteration k (optional warm-up schedule of Section 4)."""
        return self.warm_rho if k < self.warm_iters else self.rho0

    @classmethod
    def from_instance(cls, inst, **kw):
        cost = np.asarray(inst.cost_w, dtype=np.float64)
        if cost.ndim == 1:
            cost = np.repeat(cost[:, None], inst.eta, axis=1)
        return cls(p=inst.p, eta=inst.eta, start=np.asarray(inst.start, dtype=np.float64),
                   goal=np.asarray(inst.goal, dtype=np.float64),
                   radius=np.asarray(inst.radius, dtype=np.float64), cost=cost,
                   walls=np.asarray(inst.walls, dtype=np.float64).reshape(-1, 4),
                   rho0=float(inst.rho0), alpha=float(inst.alpha), **kw)


@dataclass
class State:
    z: np.ndarray              # (p, eta+1, 2)
    u_coll: np.ndarray         # (eta, P, 4, 2) edges (i,s), (i,s+1), (j,s), (j,s+1)
    u_kin: np.ndarray          # (eta, p, 2, 2) edges (i,s), (i,s+1)
    u_wall: np.ndarray         # (n_walls, eta, p, 2, 2)
    wback: np.ndarray          # (p, eta+1) back-weight class
    k: int = 0
    u_vel: dict = field(default_factory=dict)   # "max" / "min" -> (eta, p, 2, 2)

    def copy(self):
        return State(self.z.copy(), self.u_coll.copy(), self.u_kin.copy(), self.u_wall.copy(),
                     self.wback.copy(), self.k, {k: v.copy() for k, v in self.u_vel.items()})


@dataclass
class Info:
    active_coll: np.ndarray    # (eta, P) bool: forward weight rho0
    active_wall: np.ndarray    # (n_walls, eta, p) bool
    residual: float            # max(primal, dz) of this iteration
    primal: float              # max over weighted edges |x - z^{k+1}|_inf
    dz: float                  # max |z^{k+1} - z^k|_inf
    extra: dict = field(default_factory=dict)


def pairs(p):
    """Collision-factor pair list, lexicographic (i < j)."""
    return np.triu_indices(p, 1)


def initial_state(prob: Problem) -> State:
    """z^0 = start at every break-point but the goal node; u^0 = 0; back
    weights rho0 inside, infinity at the fixed ends (Section 4)."""
    p, eta = prob.p, prob.eta
    z = np.repeat(prob.start[:, None, :], eta + 1, axis=1).copy()
    z[:, eta] = prob.goal
    P = p * (p - 1) // 2
    wback = np.full((p, eta + 1), WR, dtype=np.int8)
    wback[:, 0] = WI
    wback[:, eta] = WI
    u_vel = {kind: np.zeros((eta, p, 2, 2)) for kind, lim in (("max", prob.vmax), ("min", prob.vmin))
             if lim is not None}
    return State(z=z, u_coll=np.zeros((eta, P, 4, 2)), u_kin=np.zeros((eta, p, 2, 2)),
                 u_wall=np.zeros((prob.n_walls, eta, p, 2, 2)), wback=wback, k=0, u_vel=u_vel)


def _wnum(cls, rho0):
    return 0.0 if cls == W0 else (rho0 if cls == WR else INF)


def iterate(prob: Problem, st: State, record_edges: bool = False, record_branches: bool = False):
    """One TWA iteration (Appendix B steps 1-7).  Returns (new_state, Info).

    record_branches stores, per collision and wall factor, the relative
    distance margin (d - R) / R of the activity test and, for active factors,
    the minimizer's relative energy gap to its runner-up direction (inf when
    inactive): the two places where a lower-precision solver may take the
    other branch."""
    p, eta = prob.p, prob.eta
    assert not (prob.admm and (not prob.energy or prob.vmax is not None or prob.vmin is not None)), \
        "standard-ADMM mode is defined here with the kinetic factors only"
    assert not prob.vo or eta == 2, "the velocity-obstacle problem has eta = 2"
    kin_segs = [s for s in range(eta) if prob.energy and not (prob.vo and s == 0)]
    con_segs = {0} if prob.vo else set(range(eta))   # collision, wall, velocity factors
    rho0 = prob.rho_at(st.k)
    z = st.z
    wb = st.wback
    cc = prob.c()
    iu, ju = pairs(p)
    Rpair = prob.radius[iu] + prob.radius[ju]
    pinned = np.zeros((p, eta + 1), dtype=bool)
    pinned[:, 0] = True
    pinned[:, eta] = True

    num = np.zeros((p, eta + 1, 2))    # sum of rho * m over finite positive weights
    den = np.zeros((p, eta + 1))       # sum of those weights
    edges = []                         # (node_i, node_s, m, weight) for record_edges

    # --- kinetic factors: steps 1-4 -------------------------------------
    x_kin = np.empty_like(st.u_kin)
    n_kin = np.empty_like(st.u_kin)
    for s in kin_segs:
        n_kin[s, :, 0] = z[:, s] - st.u_kin[s, :, 0]
        n_kin[s, :, 1] = z[:, s + 1] - st.u_kin[s, :, 1]
        for i in range(p):
            x_kin[s, i, 0], x_kin[s, i, 1] = prox.energy_prox(
                n_kin[s, i, 0], n_kin[s, i, 1], _wnum(wb[i, s], rho0),
                _wnum(wb[i, s + 1], rho0), cc[i, s])
    m_kin = x_kin + st.u_kin
    for s in kin_segs:
        for e, ss in ((0, s), (1, s + 1)):
            num[:, ss] += rho0 * m_kin[s, :, e]
            den[:, ss] += rho0
            if record_edges:
                for i in range(p):
                    edges.append((i, ss, m_kin[s, i, e].copy(), rho0))

    # --- collision factors ----------------------------------------------
    active_coll = np.zeros((eta, iu.shape[0]), dtype=bool)
    coll_x = []  # per s: (indices, x (nact, 4, 2))
    if record_branches:
        coll_margin = np.empty((eta, iu.shape[0]))
        coll_gap = np.full((eta, iu.shape[0]), INF)
    for s in range(eta):
        if s not in con_segs:
            coll_x.append((np.zeros(0, dtype=np.int64), np.zeros((0, 4, 2))))
            if record_branches:
                coll_margin[s] = INF
            continue
        u = st.u_coll[s]
        n = np.stack([z[iu, s], z[iu, s + 1], z[ju, s], z[ju, s + 1]], axis=1) - u
        c_lo = n[:, 2] - n[:, 0]
        c_hi = n[:, 3] - n[:, 1]
        dseg = prox.dist_point_segment(np.zeros_like(c_lo), c_lo, c_hi)
        act = dseg < Rpair
        if record_branches:
            coll_margin[s] = (dseg - Rpair) / Rpair
        idx = np.nonzero(act)[0]
        xa = np.empty((idx.shape[0], 4, 2))
        for k, q in enumerate(idx):
            i, j = iu[q], ju[q]
            out = prox.coll_prox(n[q, 0], n[q, 1], n[q, 2], n[q, 3],
                                 _wnum(wb[i, s], rho0), _wnum(wb[i, s + 1], rho0),
                                 _wnum(wb[j, s], rho0), _wnum(wb[j, s + 1], rho0), Rpair[q],
                                 want_gap=record_branches)
            assert out[4], "activity test disagrees with the minimizer's own test"
            xa[k] = np.stack(out[:4])
            if record_branches:
                coll_gap[s, q] = out[5]
        active_coll[s] = act
        if prob.admm:
            # every pair is weighted: x = n for the feasible ones
            idx_w = np.arange(iu.shape[0])
            xw = n.copy()
            xw[idx] = xa
            coll_x.append((idx_w, xw))
            idx, xa = idx_w, xw
        else:
            coll_x.append((idx, xa))
        if idx.shape[0]:
            ma = xa + u[idx]
            nodes_i = (iu[idx], iu[idx], ju[idx], ju[idx])
            nodes_s = (s, s + 1, s, s + 1)
            for e in range(4):
                np.add.at(num, (nodes_i[e], nodes_s[e]), rho0 * ma[:, e])
                np.add.at(den, (nodes_i[e], nodes_s[e]), rho0)
                if record_edges:
                    for k in range(idx.shape[0]):
                        edges.append((int(nodes_i[e][k]), nodes_s[e], ma[k, e].copy(), rho0))

    # --- wall factors ------------------------------------------------------
    nw = prob.n_walls
    active_wall = np.zeros((nw, eta, p), dtype=bool)
    wall_x = {}
    if record_branches:
        wall_margin = np.empty((nw, eta, p))
        wall_gap = np.full((nw, eta, p), INF)
    for w in range(nw):
        xL = prob.walls[w, :2]
        xR = prob.walls[w, 2:]
        for s in range(eta):
            if s not in con_segs:
                if record_branches:
                    wall_margin[w, s] = INF
                continue
            u = st.u_wall[w, s]
            n_lo = z[:, s] - u[:, 0]
            n_hi = z[:, s + 1] - u[:, 1]
            dw = prox.dist_segment_segment(n_lo, n_hi, xL[None, :], xR[None, :])
            act = dw < prob.radius
            if record_branches:
                wall_margin[w, s] = (dw - prob.radius) / prob.radius
            weighted = np.ones(p, dtype=bool) if prob.admm else act
            for i in np.nonzero(weighted)[0]:
                out = prox.wall_prox(n_lo[i], n_hi[i], _wnum(wb[i, s], rho0),
                                     _wnum(wb[i, s + 1], rho0), xL, xR, prob.radius[i],
                                     want_gap=record_branches)
                x_lo, x_hi, a = out[:3]
                assert a == act[i]
                if record_branches and a:
                    wall_gap[w, s, i] = out[3]
                wall_x[(w, s, i)] = (x_lo, x_hi)
                for e, ss, xv in ((0, s, x_lo), (1, s + 1, x_hi)):
                    mv = xv + u[i, e]
                    num[i, ss] += rho0 * mv
                    den[i, ss] += rho0
                    if record_edges:
                        edges.append((i, ss, mv.copy(), rho0))
            active_wall[w, s] = act

    # --- velocity factors (Appendices F, G) --------------------------------
    vel_x = {}
    active_vel = {}
    vel_margin = {}
    for kind, lim in (("max", prob.vmax), ("min", prob.vmin)):
        if lim is None:
            continue
        u = st.u_vel[kind]
        act = np.zeros((eta, p), dtype=bool)
        vel_margin[kind] = np.full((eta, p), INF)
        for s in sorted(con_segs):
            for i in range(p):
                n_lo = z[i, s] - u[s, i, 0]
                n_hi = z[i, s + 1] - u[s, i, 1]
                if lim[i, s] > 0.0 and math.isfinite(lim[i, s]):
                    vel_margin[kind][s, i] = (float(np.linalg.norm(n_lo - n_hi)) - lim[i, s]) / lim[i, s]
                x_lo, x_hi, a = prox.velocity_prox(n_lo, n_hi, _wnum(wb[i, s], rho0),
                                                   _wnum(wb[i, s + 1], rho0), lim[i, s], kind)
                act[s, i] = a
                if not a:
                    continue
                vel_x[(kind, s, i)] = (x_lo, x_hi)
                for e, ss, xv in ((0, s, x_lo), (1, s + 1, x_hi)):
                    mv = xv + u[s, i, e]
                    num[i, ss] += rho0 * mv
                    den[i, ss] += rho0
                    if record_edges:
                        edges.append((i, ss, mv.copy(), rho0))
        active_vel[kind] = act

    # --- step 5: consensus z ----------------------------------------------
    z_new = np.empty_like(z)
    pos = den > 0
    z_new[pos] = num[pos] / den[pos][:, None]
    # all incoming weights zero: treat them as 1, i.e. the plain mean of every
    # incoming m.  Every factor at such a node is inactive and returns x = n,
    # so each of its messages is m = n + u = z^k: the mean is z^k.
    zero_nodes = (~pos) & (~pinned)
    z_new[zero_nodes] = z[zero_nodes]
    z_new[:, 0] = prob.start
    z_new[:, eta] = prob.goal

    # --- step 6: back weights ---------------------------------------------
    wb_new = np.where(pos, WR, W0).astype(np.int8)
    wb_new[:, 0] = WI
    wb_new[:, eta] = WI

    # --- step 7: u update -------------------------------------------------
    a = prob.alpha / rho0 if prob.u_literal else prob.alpha
    primal = 0.0
    new = st.copy()
    new.z = z_new
    new.wback = wb_new
    new.k = st.k + 1

    def upd(u_old, x, i_node, s_node, fwd_active):
        """u for one edge family; arrays broadcast over leading dims."""
        ok = fwd_active & (wb_new[i_node, s_node] == WR)
        step = u_old + a * (x - z_new[i_node, s_node])
        reset = u_old if prob.u_keep else np.zeros_like(u_old)
        return np.where(ok[..., None], step, reset)

    # kinetic: forward weight always rho0
    for s in kin_segs:
        allp = np.arange(p)
        for e, ss in ((0, s), (1, s + 1)):
            new.u_kin[s, :, e] = upd(st.u_kin[s, :, e], x_kin[s, :, e], allp, np.full(p, ss),
                                     np.ones(p, dtype=bool))
            primal = max(primal, float(np.max(np.abs(x_kin[s, :, e] - z_new[:, ss]), initial=0.0)))
    # collision: inactive factors have x = n and forward weight 0
    for s in range(eta):
        idx, xa = coll_x[s]
        u = st.u_coll[s]
        new.u_coll[s] = u if prob.u_keep else 0.0
        if idx.shape[0]:
            nodes_i = (iu[idx], iu[idx], ju[idx], ju[idx])
            nodes_s = (s, s + 1, s, s + 1)
            for e in range(4):
                si = np.full(idx.shape[0], nodes_s[e])
                new.u_coll[s][idx, e] = upd(u[idx, e], xa[:, e], nodes_i[e], si,
                                            np.ones(idx.shape[0], dtype=bool))
                primal = max(primal, float(np.max(np.abs(xa[:, e] - z_new[nodes_i[e], nodes_s[e]]))))
    # velocity factors: inactive ones reset u (or keep it)
    for kind, act in active_vel.items():
        u_old = st.u_vel[kind]
        new.u_vel[kind] = u_old.copy() if prob.u_keep else np.zeros_like(u_old)
        for (kd, s, i), (x_lo, x_hi) in vel_x.items():
            if kd != kind:
                continue
            for e, ss, xv in ((0, s, x_lo), (1, s + 1, x_hi)):
                new.u_vel[kind][s, i, e] = upd(u_old[s, i, e][None], xv[None], np.array([i]),
                                               np.array([ss]), np.array([True]))[0]
                primal = max(primal, float(np.max(np.abs(xv - z_new[i, ss]))))
    # walls
    for w in range(nw):
        for s in range(eta):
            if not prob.u_keep:
                new.u_wall[w, s] = 0.0
        for (w_, s, i), (x_lo, x_hi) in wall_x.items():
            if w_ != w:
                continue
            for e, ss, xv in ((0, s, x_lo), (1, s + 1, x_hi)):
                new.u_wall[w, s, i, e] = upd(st.u_wall[w, s, i, e][None], xv[None],
                                             np.array([i]), np.array([ss]),
                                             np.array([True]))[0]
                primal = max(primal, float(np.max(np.abs(xv - z_new[i, ss]))))
    dz = float(np.max(np.abs(z_new - z)))
    info = Info(active_coll=active_coll, active_wall=active_wall, residual=max(primal, dz),
                primal=primal, dz=dz)
    info.extra["active_vel"] = active_vel
    info.extra["vel_margin"] = vel_margin
    if record_branches:
        info.extra.update(coll_margin=coll_margin, coll_gap=coll_gap, wall_margin=wall_margin,
                          wall_gap=wall_gap)
    if record_edges:
        info.extra["edges"] = edges
        info.extra["x_kin"] = x_kin
        info.extra["coll_x"] = coll_x
    return new, info


def solve(prob: Problem, tol: float, max_iter: int, st: State | None = None):
    """Iterate until the residual of an iteration drops below tol (or
    max_iter iterations).  Returns (state, iterations, last residual)."""
    st = initial_state(prob) if st is None else st
    res = INF
    for it in range(max_iter):
        st, info = iterate(prob, st)
        res = info.residual
        if res < tol:
            return st, it + 1, res
    return st, max_iter, res


def total_cost(prob: Problem, z: np.ndarray) -> float:
    """f^cost of Eq. velo_cost_pair_wise at the break-points z (p, eta+1, 2)."""
    d = z[:, 1:] - z[:, :-1]
    return float(np.sum(prob.c() * np.sum(d * d, axis=-1)))


def min_clearance(prob: Problem, z: np.ndarray):
    """Smallest ratio dist / (r_i + r_j) over every pair and segment, and the
    smallest dist / r_i over every agent, segment and wall (1 = touching)."""
    p, eta = prob.p, prob.eta
    iu, ju = pairs(p)
    R = prob.radius[iu] + prob.radius[ju]
    worst = INF
    for s in range(eta):
        c_lo = z[ju, s] - z[iu, s]
        c_hi = z[ju, s + 1] - z[iu, s + 1]
        if iu.shape[0]:
            d = prox.dist_point_segment(np.zeros_like(c_lo), c_lo, c_hi)
            worst = min(worst, float(np.min(d / R)))
    wworst = INF
    for w in range(prob.n_walls):
        for s in range(eta):
            d = prox.dist_segment_segment(z[:, s], z[:, s + 1], prob.walls[w, None, :2],
                                          prob.walls[w, None, 2:])
            wworst = min(wworst, float(np.min(d / prob.radius)))
    return worst, wworst


def straight_lines(prob: Problem) -> np.ndarray:
    """Constant-velocity lines from start to goal, (p, eta+1, 2)."""
    t = np.arange(prob.eta + 1) / prob.eta
    return prob.start[:, None, :] + t[None, :, None] * (prob.goal - prob.start)[:, None, :]
