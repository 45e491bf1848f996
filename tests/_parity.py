"""Helpers shared by the GPU parity tests: run the oracle to an iterate, import
that state into the CUDA planner, run one GPU iteration and compare.

Tolerance: an FP32 entry matches when |gpu - oracle| <= TOL * L, with L the
workload's coordinate scale max(1, |start|_inf, |goal|_inf, |walls|_inf).
The bound is relative to the layout's scale, not to each entry: every u and
x - z is a difference of coordinates of size up to L, each rounded to FP32
(half an ulp of L, 6e-8 L), and the minimizers' and consensus' arithmetic on
those coordinates adds a few ulps of L, so an entry of size 1e-3 L cannot be
computed to 2e-5 of itself.  ``compare`` also reports, per array, the median
and largest entrywise error relative to max(|oracle|, TOL * L).

Branches.  A factor whose activity test sits within MARGIN of the collision
distance, or whose minimizer has a runner-up direction within GAP in energy,
may legitimately go the other way in FP32.  Such factors (per the oracle's
own FP64 diagnostics) may disagree on the activity bit; any other
disagreement fails.  Entries depending on a factor whose branch differs or may
differ are left out of the value comparison and counted.
"""
import numpy as np

from oracle import twa

TOL = 2e-5
MARGIN = 1e-4
GAP = 1e-3
TAINT_MARGIN = 1.0


def scale_of(prob):
    vals = [1.0, np.max(np.abs(prob.start)), np.max(np.abs(prob.goal))]
    if prob.n_walls:
        vals.append(np.max(np.abs(prob.walls)))
    return float(max(vals))


def oracle_state(prob, k):
    st = twa.initial_state(prob)
    for _ in range(k):
        st, _ = twa.iterate(prob, st)
    return st


def make_planner(prob, flags=0, **kw):
    import paper_1311_4527_gb300 as pk
    cost = prob.cost
    flags = flags | (pk.PLAN_COST_UNNORM if prob.cost_unnorm else 0)
    if prob.u_keep:
        flags |= pk.PLAN_U_KEEP
    if prob.u_literal:
        flags |= pk.PLAN_U_LITERAL
    if prob.warm_iters:
        kw.setdefault("warm_iters", prob.warm_iters)
        kw.setdefault("warm_rho", prob.warm_rho)
    if prob.admm:
        flags |= pk.PLAN_ADMM
    return pk.Planner(prob.start, prob.goal, prob.radius, prob.eta, cost_w=cost,
                      walls=prob.walls if prob.n_walls else None, rho0=prob.rho0,
                      alpha=prob.alpha, flags=flags, energy=prob.energy, vmax=prob.vmax,
                      vmin=prob.vmin, **kw)


def gpu_step(prob, st, flags=0, planner=None):
    """Import oracle state st, run one GPU iteration, export as numpy."""
    pl = planner or make_planner(prob, flags)
    pl.import_state(st.z, st.u_coll, st.u_kin, st.u_wall if prob.n_walls else None, st.k)
    if st.u_vel:
        pl.import_velocity_state(st.u_vel.get("max"), st.u_vel.get("min"))
    if not prob.energy:
        # a factor alone at a node leaves u = 0 there, so the classes cannot
        # be read back from u: import the oracle's
        pl.import_back_weights(st.wback)
    pl.iterate(1)
    out = gpu_export(prob, pl)
    if planner is None:
        pl.close()
    return out


def differing_nodes(prob, new, gpu, tol=TOL):
    """Break-points where the GPU's state and the oracle's state `new` differ
    by more than tol * L: in z, in the back-weight class, in the u of a factor
    that reads them, or in a factor's activity.  Used as prior_bad when both
    sides take a further step from their own iterates."""
    L = scale_of(prob)
    p, eta = prob.p, prob.eta
    iu, ju = twa.pairs(p)
    lim = tol * L
    bad = np.any(np.abs(gpu["z"] - new.z) > lim, axis=-1) | (gpu["wback"] != new.wback)
    if iu.size:
        du = np.any(np.abs(gpu["u_coll"] - new.u_coll) > lim, axis=(-1, -2))   # (eta, P)
        for s in range(eta):
            q = np.nonzero(du[s])[0]
            for arr in (iu[q], ju[q]):
                bad[arr, s] = True
                bad[arr, s + 1] = True
    dk = np.any(np.abs(gpu["u_kin"] - new.u_kin) > lim, axis=(-1, -2))           # (eta, p)
    bad[:, :-1] |= dk.T
    bad[:, 1:] |= dk.T
    if prob.n_walls:
        dw = np.any(np.abs(gpu["u_wall"] - new.u_wall) > lim, axis=(-1, -2)).any(axis=0)
        bad[:, :-1] |= dw.T
        bad[:, 1:] |= dw.T
    return bad


def gpu_export(prob, pl):
    """The planner's current state in the oracle's layout, as numpy."""
    ex = pl.export_state()
    out = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in ex.items()}
    if prob.vmax is not None or prob.vmin is not None:
        out["vel"] = {k: (u.cpu().numpy(), a.cpu().numpy().astype(bool))
                      for k, (u, a) in pl.export_velocity_state().items()}
    out["wback"] = pl.export_back_weights().cpu().numpy()
    return out


def compare(prob, new, info, gpu, tol=TOL, prior_bad=None, return_bad=False):
    """Compare the oracle's iterate `new` (with its Info, recorded with
    record_branches=True) to the GPU export.  Returns a stats dict; raises
    AssertionError on any mismatch outside the rules above.

    prior_bad: (p, eta+1) break-points left out of the previous step's
    comparison, when both sides continued from their own iterates.  Their z
    and u may differ, so every factor that reads one of them may differ in
    activity and output: those factors are treated like near-ties, and the
    kinetic factors touching them taint both their break-points.
    return_bad: also return the break-points left out here."""
    L = scale_of(prob)
    p, eta = prob.p, prob.eta
    iu, ju = twa.pairs(p)
    stats = {}
    prior = np.zeros((p, eta + 1), dtype=bool) if prior_bad is None else prior_bad
    seg_prior = prior[:, :-1] | prior[:, 1:]                # (p, eta)
    # --- branch classification --------------------------------------------
    act_o = info.active_coll
    act_g = gpu["act_coll"].astype(bool)
    cm, cg = info.extra["coll_margin"], info.extra["coll_gap"]
    tainted = np.stack([seg_prior[iu, s] | seg_prior[ju, s] for s in range(eta)]) if iu.size \
        else np.zeros_like(act_o)
    # a tainted pair farther apart than twice its collision distance stays
    # inactive on both sides (its inputs differ by far less than that)
    near = (np.abs(cm) < MARGIN) | (tainted & (np.abs(cm) < TAINT_MARGIN))
    ambiguous = near | (act_o & (cg < GAP)) | (tainted & act_o)
    differ = act_o != act_g
    bad = differ & ~near
    assert not bad.any(), f"{int(bad.sum())} collision factors disagree on activity away from the boundary"
    excl = differ | ambiguous
    stats["coll_active"] = int(act_o.sum())
    stats["coll_active_gpu"] = int(act_g.sum())
    stats["coll_excluded"] = int(excl.sum())
    bad_node = prior.copy()
    bad_node[:, :-1] |= seg_prior    # a kinetic factor reading a tainted node changes both ends
    bad_node[:, 1:] |= seg_prior
    for s in range(eta):
        q = np.nonzero(excl[s])[0]
        for arr in (iu[q], ju[q]):
            bad_node[arr, s] = True
            bad_node[arr, s + 1] = True
    if prob.n_walls:
        aw_o = info.active_wall
        aw_g = gpu["act_wall"].astype(bool)
        wm, wg = info.extra["wall_margin"], info.extra["wall_gap"]
        wtaint = np.broadcast_to(seg_prior.T[None, :, :], wm.shape)
        wnear = (np.abs(wm) < MARGIN) | (wtaint & (np.abs(wm) < TAINT_MARGIN))
        wamb = wnear | (aw_o & (wg < GAP)) | (wtaint & aw_o)
        wdiff = aw_o != aw_g
        wbad = wdiff & ~wnear
        assert not wbad.any(), f"{int(wbad.sum())} wall factors disagree on activity away from the boundary"
        wex = wdiff | wamb
        stats["wall_active"] = int(aw_o.sum())
        stats["wall_excluded"] = int(wex.sum())
        for w in range(prob.n_walls):
            for s in range(eta):
                idx = np.nonzero(wex[w, s])[0]
                bad_node[idx, s] = True
                bad_node[idx, s + 1] = True
    vex = {}
    for kind, act_v in info.extra.get("active_vel", {}).items():
        vm = info.extra["vel_margin"][kind]
        vg = gpu["vel"][kind][1]
        vdiff = act_v != vg
        vnear = (np.abs(vm) < MARGIN) | (seg_prior.T & (np.abs(vm) < TAINT_MARGIN))
        vbad = vdiff & ~vnear
        assert not vbad.any(), f"{int(vbad.sum())} {kind}-velocity factors disagree away from the limit"
        vex[kind] = vdiff | vnear | (seg_prior.T & act_v)
        stats[f"v{kind}_active"] = int(act_v.sum())
        for s_, i_ in zip(*np.nonzero(vex[kind])):
            bad_node[i_, s_] = True
            bad_node[i_, s_ + 1] = True
    stats["nodes_excluded"] = int(bad_node.sum())
    # back weights of the new iterate (step 6), away from excluded factors
    wdiff = (gpu["wback"] != new.wback) & ~bad_node
    assert not wdiff.any(), f"{int(wdiff.sum())} break-points differ in back weight"
    # --- values --------------------------------------------------------------
    def rel(name, d, ref, mask):
        """Median and largest |d| / max(|ref|, TOL L) over the compared entries."""
        if not mask.any():
            return
        r = (d / np.maximum(np.abs(ref), tol * L))[mask]
        stats[name + "_relmed"] = float(np.median(r))
        stats[name + "_relmax"] = float(np.max(r))

    dz = np.abs(gpu["z"] - new.z)
    worst = float(np.max(dz[~bad_node])) if (~bad_node).any() else 0.0
    stats["z_maxerr"] = worst / L
    rel("z", dz, new.z, np.broadcast_to(~bad_node[..., None], dz.shape))
    assert worst <= tol * L, f"z error {worst} > {tol * L}"
    seg_bad = bad_node[:, :-1] | bad_node[:, 1:]            # (p, eta)
    ok = ~excl
    for s in range(eta):
        ok[s] &= ~(seg_bad[iu, s] | seg_bad[ju, s])
    du = np.abs(gpu["u_coll"] - new.u_coll)
    worst = float(np.max(du[ok])) if ok.any() else 0.0
    stats["u_coll_maxerr"] = worst / L
    # entrywise: the u of factors active in the oracle (every other u is 0 on both sides)
    rel("u_coll", du, new.u_coll, np.broadcast_to((ok & act_o)[..., None, None], du.shape))
    stats["coll_compared_active"] = int((ok & act_o).sum())
    assert worst <= tol * L, f"u_coll error {worst} > {tol * L}"
    kin_ok = ~seg_bad.T                                     # (eta, p)
    for kind, ex_v in vex.items():
        okv = ~ex_v & kin_ok
        dv = np.abs(gpu["vel"][kind][0] - new.u_vel[kind])
        worst = float(np.max(dv[okv])) if okv.any() else 0.0
        stats[f"u_v{kind}_maxerr"] = worst / L
        assert worst <= tol * L, f"u_v{kind} error {worst} > {tol * L}"
    dk = np.abs(gpu["u_kin"] - new.u_kin)
    worst = float(np.max(dk[kin_ok])) if kin_ok.any() else 0.0
    stats["u_kin_maxerr"] = worst / L
    rel("u_kin", dk, new.u_kin, np.broadcast_to(kin_ok[..., None, None], dk.shape))
    assert worst <= tol * L, f"u_kin error {worst} > {tol * L}"
    if prob.n_walls:
        okw = ~wex & ~seg_bad.T[None, :, :]
        dw = np.abs(gpu["u_wall"] - new.u_wall)
        worst = float(np.max(dw[okw])) if okw.any() else 0.0
        stats["u_wall_maxerr"] = worst / L
        assert worst <= tol * L, f"u_wall error {worst} > {tol * L}"
    if return_bad:
        return stats, bad_node
    return stats
