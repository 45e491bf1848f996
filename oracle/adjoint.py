"""FP64 reference adjoint of K unrolled TWA iterations (test infrastructure
only).

z^K(theta) is the break-point iterate after K iterations (Appendix B) from
the initial state of Section 4, theta = (start, goal, radii, cost weights).
Given dL/dz^K this returns dL/dtheta with every branch choice frozen: which
factors are active at each iteration and which candidate direction each
minimizer picked.  Under the reset rule (u = 0 on edges whose forward weight
was 0) an inactive factor carries no gradient, so the recursion only visits
each iteration's active collision factors and the kinetic factors.

Per-factor Jacobians are taken by central differences of the oracle's own
minimizers (``oracle.prox``) in FP64, so this reference is independent of
any analytic derivation; the differences use a step of 1e-6 of the problem
scale, small enough not to change the minimizer's branch in the cases the
tests use.  Wall factors and velocity-limit factors are gated like the
collision factors (their u lives only while they stay active).  The local
planner's epoch (``vo``) is the same recursion on its graph.  The
feasibility mode, standard-ADMM mode, kept u and the rho warm-up are not
covered.
"""
from __future__ import annotations

import math

import numpy as np

from . import prox, twa

INF = math.inf


def _coll_fn(nv, R, wl, wh):
    """x (8,) = g^coll(n (8,)) for one active pair; wl/wh: weight at the lower
    and upper ends (rho0 or inf)."""
    n = nv.reshape(4, 2)
    out = prox.coll_prox(n[0], n[1], n[2], n[3], wl, wh, wl, wh, R)
    return np.concatenate(out[:4])


def _jac_fd(f, v, h):
    """Central-difference Jacobian of f at v (columns per input entry)."""
    f0 = f(v)
    J = np.zeros((f0.shape[0], v.shape[0]))
    for q in range(v.shape[0]):
        e = np.zeros_like(v)
        e[q] = h
        J[:, q] = (f(v + e) - f(v - e)) / (2 * h)
    return J


def record(prob: twa.Problem, K: int):
    """Forward K iterations, keeping what the adjoint needs per iteration:
    the state at the start of the iteration and which collision factors and
    gated segment factors (walls, velocity limits) were active."""
    assert prob.energy and not prob.admm and not prob.u_keep and prob.warm_iters == 0
    st = twa.initial_state(prob)
    tape = []
    for _ in range(K):
        new, info = twa.iterate(prob, st)
        seg = set()
        for w, s, i in zip(*np.nonzero(info.active_wall)):
            seg.add(("w", int(w), int(s), int(i)))
        for kind, act in info.extra["active_vel"].items():
            for s, i in zip(*np.nonzero(act)):
                seg.add(("v", kind, int(s), int(i)))
        tape.append((st, info.active_coll, seg))
        st = new
    return st, tape


def _seg_factor(prob, st, key):
    """(u (2, 2), minimizer of n (4,) -> x (4,) with radius argument, radius
    index or None) of a gated segment factor at state st."""
    rho = prob.rho0
    typ, w, s, i = key
    wl = INF if s == 0 else rho
    wh = INF if s + 1 == prob.eta else rho
    if typ == "w":
        xL, xR = prob.walls[w, :2], prob.walls[w, 2:]
        f = lambda v, r: np.concatenate(prox.wall_prox(v[:2], v[2:], wl, wh, xL, xR, r)[:2])
        return st.u_wall[w, s, i], f, i
    lim = (prob.vmax if w == "max" else prob.vmin)[i, s]
    f = lambda v, r: np.concatenate(prox.velocity_prox(v[:2], v[2:], wl, wh, lim, w)[:2])
    return st.u_vel[w][s, i], f, None


def branches(prob: twa.Problem, K: int) -> np.ndarray:
    """Branch of every collision factor in each of K iterations: 0 inactive,
    else 1 + (lower end moved) + 2 (upper end moved), where an end moved when
    the minimizer changed the relative position x_j - x_i there, i.e. its
    hinge [R - <v, n>]_+ was positive.  Two runs with equal codes took the
    same smooth piece of the minimizers everywhere."""
    iu, ju = twa.pairs(prob.p)
    st = twa.initial_state(prob)
    out = np.zeros((K, prob.eta, iu.shape[0]), dtype=np.int8)
    for k in range(K):
        new, info = twa.iterate(prob, st, record_edges=True)
        for s, (idx, xa) in enumerate(info.extra["coll_x"]):
            for q, x in zip(idx, xa):
                nl = st.z[ju[q], s] - st.u_coll[s, q, 2] - (st.z[iu[q], s] - st.u_coll[s, q, 0])
                nh = st.z[ju[q], s + 1] - st.u_coll[s, q, 3] - (st.z[iu[q], s + 1] - st.u_coll[s, q, 1])
                sc = 1e-12 * max(1.0, float(np.abs(nl).max()), float(np.abs(nh).max()))
                lo = float(np.abs((x[2] - x[0]) - nl).max()) > sc
                hi = float(np.abs((x[3] - x[1]) - nh).max()) > sc
                out[k, s, q] = 1 + int(lo) + 2 * int(hi)
        st = new
    return out


def seg_branches(prob: twa.Problem, K: int):
    """Per iteration, the active gated segment factors (walls, velocity
    limits) with a code 1 + (lower end moved) + 2 (upper end moved): two runs
    with equal lists took the same branches of those minimizers."""
    _, tape = record(prob, K)
    out = []
    for st, _, seg in tape:
        codes = {}
        for key in seg:
            u, fn, _ = _seg_factor(prob, st, key)
            _, _, s, i = key
            nv = np.concatenate([st.z[i, s] - u[0], st.z[i, s + 1] - u[1]])
            x = fn(nv, prob.radius[i])
            sc = 1e-12 * max(1.0, float(np.abs(nv).max()))
            codes[key] = 1 + int(np.abs(x[:2] - nv[:2]).max() > sc) + 2 * int(np.abs(x[2:] - nv[2:]).max() > sc)
        out.append(codes)
    return out


def backward(prob: twa.Problem, K: int, dz_K: np.ndarray, h: float | None = None):
    """dL/d(start, goal, radius, cost) for dL/dz^K = dz_K (p, eta+1, 2)."""
    p, eta = prob.p, prob.eta
    rho, alpha = prob.rho0, prob.alpha
    iu, ju = twa.pairs(p)
    cc = prob.c()
    norm = 1.0 if prob.cost_unnorm else 1.0 / (p * eta)
    scale = max(1.0, float(np.max(np.abs(prob.start))), float(np.max(np.abs(prob.goal))))
    h = 1e-6 * scale if h is None else h
    _, tape = record(prob, K)
    g_start = np.zeros((p, 2))
    g_goal = np.zeros((p, 2))
    g_rad = np.zeros(p)
    g_cost = np.zeros((p, eta))
    zbar = dz_K.astype(np.float64).copy()          # adjoint of z^{k+1}
    ubar_coll = {}                                   # (s, q) -> (4, 2) adjoint of u^{k+1}
    ubar_seg = {}                                    # gated segment factor -> (2, 2)
    ubar_kin = np.zeros((eta, p, 2, 2))
    free = np.ones((p, eta + 1), dtype=bool)
    free[:, 0] = False
    free[:, eta] = False
    # the local planner has its kinetic factor on the second segment only
    kin_segs = [1] if prob.vo else list(range(eta))

    for k in range(K - 1, -1, -1):
        st, act, seg = tape[k]
        z, u_coll, u_kin = st.z, st.u_coll, st.u_kin
        # fixed ends of z^{k+1}
        g_start += zbar[:, 0]
        g_goal += zbar[:, eta]
        # step 7: u^{k+1} = u + alpha (x - z^{k+1}) on active edges at free nodes
        zhat = zbar.copy()
        cnt = np.zeros((p, eta + 1))
        for s in kin_segs:
            cnt[:, s] += 1.0
            cnt[:, s + 1] += 1.0
            zhat[:, s] -= alpha * ubar_kin[s, :, 0] * free[:, s, None]
            zhat[:, s + 1] -= alpha * ubar_kin[s, :, 1] * free[:, s + 1, None]
        for s in range(eta):
            for q in np.nonzero(act[s])[0]:
                ub = ubar_coll.get((s, q), np.zeros((4, 2)))
                for e, (ag, ss) in enumerate(((iu[q], s), (iu[q], s + 1), (ju[q], s), (ju[q], s + 1))):
                    cnt[ag, ss] += 1.0
                    if free[ag, ss]:
                        zhat[ag, ss] -= alpha * ub[e]
        for key in seg:
            ub = ubar_seg.get(key, np.zeros((2, 2)))
            _, _, s, i = key
            for e, ss in ((0, s), (1, s + 1)):
                cnt[i, ss] += 1.0
                if free[i, ss]:
                    zhat[i, ss] -= alpha * ub[e]
        # step 5: z^{k+1} = mean of m over active edges (free nodes)
        mbar_node = np.where(free[..., None], zhat / np.maximum(cnt, 1.0)[..., None], 0.0)
        new_zbar = np.zeros_like(zbar)
        new_ubar_kin = np.zeros_like(ubar_kin)
        new_ubar_coll = {}
        # kinetic factors
        for s in kin_segs:
            for i in range(p):
                wl = INF if s == 0 else rho
                wh = INF if s + 1 == eta else rho
                nv = np.concatenate([z[i, s] - u_kin[s, i, 0], z[i, s + 1] - u_kin[s, i, 1]])
                c = cc[i, s]
                f = lambda v: np.concatenate(prox.energy_prox(v[:2], v[2:], wl, wh, c))
                J = _jac_fd(f, nv, h)
                fc = lambda cv: np.concatenate(prox.energy_prox(nv[:2], nv[2:], wl, wh, cv))
                dxdc = (fc(c + 1e-7) - fc(c - 1e-7)) / 2e-7
                ub = ubar_kin[s, i]
                xbar = np.zeros(4)
                ubar_acc = ub.copy()
                for e, ss in ((0, s), (1, s + 1)):
                    if free[i, ss]:
                        xbar[2 * e:2 * e + 2] = alpha * ub[e] + mbar_node[i, ss]
                        ubar_acc[e] = ub[e] + mbar_node[i, ss]
                    else:
                        ubar_acc[e] = 0.0
                nbar = J.T @ xbar
                g_cost[i, s] += float(dxdc @ xbar) * norm
                new_zbar[i, s] += nbar[:2]
                new_zbar[i, s + 1] += nbar[2:]
                # u^k of a kinetic edge at a free node is live (always active)
                for e, ss in ((0, s), (1, s + 1)):
                    if free[i, ss]:
                        new_ubar_kin[s, i, e] = ubar_acc[e] - nbar[2 * e:2 * e + 2]
        # collision factors
        for s in range(eta):
            wl = INF if s == 0 else rho
            wh = INF if s + 1 == eta else rho
            for q in np.nonzero(act[s])[0]:
                i, j = iu[q], ju[q]
                R = prob.radius[i] + prob.radius[j]
                nodes = ((i, s), (i, s + 1), (j, s), (j, s + 1))
                nv = np.concatenate([z[a, b] - u_coll[s, q, e] for e, (a, b) in enumerate(nodes)])
                J = _jac_fd(lambda v: _coll_fn(v, R, wl, wh), nv, h)
                dxdR = (_coll_fn(nv, R + h, wl, wh) - _coll_fn(nv, R - h, wl, wh)) / (2 * h)
                ub = ubar_coll.get((s, q), np.zeros((4, 2)))
                xbar = np.zeros(8)
                ubar_acc = np.zeros((4, 2))
                for e, (a, b) in enumerate(nodes):
                    if free[a, b]:
                        xbar[2 * e:2 * e + 2] = alpha * ub[e] + mbar_node[a, b]
                        ubar_acc[e] = ub[e] + mbar_node[a, b]
                nbar = J.T @ xbar
                gR = float(dxdR @ xbar)
                g_rad[i] += gR
                g_rad[j] += gR
                out = np.zeros((4, 2))
                for e, (a, b) in enumerate(nodes):
                    new_zbar[a, b] += nbar[2 * e:2 * e + 2]
                    if free[a, b]:
                        out[e] = ubar_acc[e] - nbar[2 * e:2 * e + 2]
                new_ubar_coll[(s, q)] = out
        # gated segment factors (walls, velocity limits)
        new_ubar_seg = {}
        for key in seg:
            u, fn, ri = _seg_factor(prob, st, key)
            _, _, s, i = key
            nv = np.concatenate([z[i, s] - u[0], z[i, s + 1] - u[1]])
            r = prob.radius[i]
            J = _jac_fd(lambda v: fn(v, r), nv, h)
            ub = ubar_seg.get(key, np.zeros((2, 2)))
            xbar = np.zeros(4)
            out = np.zeros((2, 2))
            for e, ss in ((0, s), (1, s + 1)):
                if free[i, ss]:
                    xbar[2 * e:2 * e + 2] = alpha * ub[e] + mbar_node[i, ss]
            nbar = J.T @ xbar
            if ri is not None:
                g_rad[ri] += float(((fn(nv, r + h) - fn(nv, r - h)) / (2 * h)) @ xbar)
            for e, ss in ((0, s), (1, s + 1)):
                new_zbar[i, ss] += nbar[2 * e:2 * e + 2]
                if free[i, ss]:
                    out[e] = ub[e] + mbar_node[i, ss] - nbar[2 * e:2 * e + 2]
            new_ubar_seg[key] = out
        # u^k of a collision factor is live only if it was active at k-1
        prev_act = tape[k - 1][1] if k > 0 else None
        prev_seg = tape[k - 1][2] if k > 0 else set()
        ubar_coll = {}
        ubar_seg = {key: v for key, v in new_ubar_seg.items() if key in prev_seg}
        if prev_act is not None:
            for (s, q), v in new_ubar_coll.items():
                if prev_act[s, q]:
                    ubar_coll[(s, q)] = v
            # factors active at k-1 but not at k: u^k fed only the (frozen)
            # activity test at k, so their adjoint is 0
        ubar_kin = new_ubar_kin
        zbar = new_zbar
    # z^0: start at every break-point but the goal node (Section 4)
    g_start += zbar[:, :eta].sum(axis=1)
    g_goal += zbar[:, eta]
    return g_start, g_goal, g_rad, g_cost


def zK(prob: twa.Problem, K: int) -> np.ndarray:
    st = twa.initial_state(prob)
    for _ in range(K):
        st, _ = twa.iterate(prob, st)
    return st.z
