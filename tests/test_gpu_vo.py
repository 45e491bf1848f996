"""The velocity-obstacle local planner on the GPU (PLAN_VO, plan_vo_epoch)
against the oracle's (oracle.vo): one-iteration parity inside an epoch,
positions epoch by epoch, and the whole circle swap reaching its
destinations without collision."""
import numpy as np
import pytest

import workloads
from oracle import prox, twa, vo

import _parity as par

pytestmark = pytest.mark.gpu
RHO = 10.0


def _clearance(x0, x, radius):
    iu, ju = twa.pairs(x0.shape[0])
    d = prox.dist_point_segment(np.zeros((iu.shape[0], 2)), x0[ju] - x0[iu], x[ju] - x[iu])
    return float(np.min(d / (radius[iu] + radius[ju])))


def _vo_planner(prob, **kw):
    import paper_1311_4527_gb300 as pk
    return pk.Planner(prob.start, prob.goal, prob.radius, 2, cost_w=prob.cost[:, 1],
                      rho0=prob.rho0, alpha=prob.alpha, vo=True, **kw)


@pytest.mark.parametrize("case", ["head_on", "circle4"])
def test_vo_iteration_parity(case):
    if case == "head_on":
        x0 = np.array([[-0.5, 0.01], [0.5, -0.01]])
        prob = vo.problem(x0, vo.targets(x0, np.array([[2.0, 0.0], [-2.0, 0.0]]), 0.8),
                          np.array([0.2, 0.2]), np.array([1.0, 1.001]), rho0=RHO)
    else:
        inst = workloads.circle4()
        prob = vo.problem(inst.start, vo.targets(inst.start, inst.goal, 0.9), inst.radius,
                          1 + 0.001 * np.arange(4), rho0=RHO)
    st = twa.initial_state(prob)
    done = 0
    active = 0
    for k in (0, 3, 30, 100):
        while done < k:
            st, _ = twa.iterate(prob, st)
            done += 1
        new, info = twa.iterate(prob, st, record_branches=True)
        pl = _vo_planner(prob)
        gpu = par.gpu_step(prob, st, planner=pl)
        pl.close()
        stats = par.compare(prob, new, info, gpu)
        active += stats["coll_active"]
        assert not info.active_coll[1].any() and not gpu["act_coll"][1].any()
    assert active > 0


def test_vo_epochs_follow_the_oracle():
    import paper_1311_4527_gb300 as pk
    inst = workloads.circle4()
    c = 1 + 0.001 * np.arange(4)
    xs, its = vo.simulate(inst.start, inst.goal, inst.radius, c, 0.25, 0.5, 6, 1e-8, 6000, rho0=RHO)
    pl = pk.Planner.velocity_obstacle(inst.start, inst.goal, inst.radius, c, 0.25, rho0=RHO,
                                      tol=1e-7, max_iter=6000, check_every=1)
    for e in range(6):
        conv, it, r, md = pl.vo_epoch(0.5)
        assert conv, (e, it, r)
        x, _ = pl.endpoints()
        assert np.abs(x - xs[e + 1]).max() <= 1e-4, (e, x, xs[e + 1])
        assert abs(it - its[e]) <= 0.2 * its[e] + 5, (e, it, its[e])
    pl.close()


def test_vo_circle_swap_reaches_the_destinations():
    import paper_1311_4527_gb300 as pk
    inst = workloads.circle4()
    c = 1 + 0.001 * np.arange(4)
    pl = pk.Planner.velocity_obstacle(inst.start, inst.goal, inst.radius, c, 0.25, rho0=RHO,
                                      tol=1e-6, max_iter=8000, check_every=5)
    x_prev = inst.start.astype(np.float64)
    for e in range(40):
        conv, it, r, md = pl.vo_epoch(0.5)
        x = pl.endpoints()[0].astype(np.float64)
        assert _clearance(x_prev, x, inst.radius) >= 1 - 1e-4, e
        x_prev = x
        if md < 1e-3:
            break
    pl.close()
    assert md < 1e-3, md


def test_endpoint_update_of_the_local_planner_checks_starts_only():
    """plan_set_endpoints on a PLAN_VO plan (checked on the device): the goals
    are reference points and may overlap, so only starts are tested; an
    overlap among the starts is refused and leaves the plan unchanged; a goal
    far outside the old layout is applied and the iteration stays finite
    (the new extent sets the fixed-point scale)."""
    import paper_1311_4527_gb300 as pk
    x0 = np.array([[-0.5, 0.01], [0.5, -0.01], [0.0, 0.6]])
    r = np.array([0.2, 0.2, 0.15])
    prob = vo.problem(x0, vo.targets(x0, np.array([[2.0, 0.0], [-2.0, 0.0], [0.0, -2.0]]), 0.8), r,
                      np.array([1.0, 1.001, 1.002]), rho0=RHO)
    with _vo_planner(prob) as pl:
        pl.iterate(5)
        z0 = pl.trajectory_host()
        goal = prob.goal.copy()
        goal[1] = goal[0]                       # overlapping reference points: allowed
        pl.set_endpoints(prob.start, goal)
        z = pl.trajectory_host()
        assert np.array_equal(z[:, -1], goal.astype(np.float32))
        bad = prob.start.copy()
        bad[2] = bad[0] + np.array([0.1, 0.0])  # starts 0 and 2 overlap
        with pytest.raises(pk.PlanError) as e:
            pl.set_endpoints(bad, goal)
        assert e.value.status == "PLAN_EINFEASIBLE_INPUT" and "start positions of agents 0 and 2" in str(e.value)
        assert np.array_equal(pl.trajectory_host(), z)
        far = goal.copy()
        far[2] = [0.0, -500.0]
        pl.set_endpoints(prob.start, far)
        pl.iterate(20)
        zf = pl.trajectory_host()
        assert np.all(np.isfinite(zf)) and np.array_equal(zf[:, -1], far.astype(np.float32))
        assert not np.array_equal(z0, zf)
