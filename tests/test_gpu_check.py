"""plan_check: the FP64 final feasibility and cost check on the device (total
cost of Eq. velo_cost_pair_wise, clearances of Eq. basic_opt_prob, endpoint
error) against the oracle's own functions evaluated in FP64 on the same FP32
break-points."""
import numpy as np
import pytest

import workloads
from oracle import twa

import _parity as par

pytestmark = pytest.mark.gpu


def _both(prob, pl):
    """The device check and the oracle's functions on the same break-points and
    on the plan's own (FP32) radii and walls."""
    import copy
    prob = copy.copy(prob)
    prob.radius = prob.radius.astype(np.float32).astype(np.float64)
    prob.walls = prob.walls.astype(np.float32).astype(np.float64)
    z = pl.trajectory().cpu().numpy().astype(np.float64)
    got = pl.check()
    coll, wall = twa.min_clearance(prob, z)
    ref = dict(total_cost=twa.total_cost(prob, z), min_pair_clearance=coll, min_wall_clearance=wall,
               max_endpoint_error=max(np.abs(z[:, 0] - prob.start.astype(np.float32)).max(),
                                      np.abs(z[:, -1] - prob.goal.astype(np.float32)).max()))
    return got, ref


def _agree(got, ref):
    assert abs(got["total_cost"] - ref["total_cost"]) <= 1e-12 * ref["total_cost"] + 1e-300
    for key in ("min_pair_clearance", "min_wall_clearance"):
        if np.isinf(ref[key]):
            assert np.isinf(got[key]), key
        else:
            assert abs(got[key] - ref[key]) <= 1e-9 * max(ref[key], 1e-3), (key, got[key], ref[key])
    assert got["max_endpoint_error"] == ref["max_endpoint_error"]


def test_check_on_the_converged_circle4():
    import paper_1311_4527_gb300 as pk
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    with pk.Planner.from_instance(inst, check_every=1) as pl:
        conv, _, _ = pl.solve()
        assert conv
        got, ref = _both(prob, pl)
    _agree(got, ref)
    assert got["min_pair_clearance"] >= 1.0 - 1e-4 and np.isinf(got["min_wall_clearance"])
    assert got["max_endpoint_error"] == 0.0


def test_check_on_square1024_mid_solve():
    """p = 1024, eta = 16 with its four walls after 100 iterations (8.4M
    pair-segments, 65,536 agent-wall-segments)."""
    import paper_1311_4527_gb300 as pk
    inst = workloads.square1024()
    prob = twa.Problem.from_instance(inst)
    with pk.Planner.from_instance(inst) as pl:
        pl.iterate(100)
        got, ref = _both(prob, pl)
    _agree(got, ref)


def test_check_sees_overlaps_and_wall_crossings():
    """Break-points imported so that two agents overlap and one segment
    crosses a wall: the check reports the oracle's ratios (0 for the
    crossing); ragged p = 72 with walls."""
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(72, 6, seed=11)
    prob = twa.Problem.from_instance(inst)
    st = twa.initial_state(prob)
    st.z[:, 1:-1] = st.z[:, :1] + 0.5 * (st.z[:, -1:] - st.z[:, :1])
    st.z[5, 3] = st.z[9, 3] + 0.3 * (inst.radius[5] + inst.radius[9])   # overlap at s = 3
    st.z[7, 2] = np.array([-1.0, 3.0])                                   # crosses the x = 0 wall
    with par.make_planner(prob) as pl:
        pl.import_state(st.z, st.u_coll, st.u_kin, st.u_wall, 0)
        got, ref = _both(prob, pl)
    _agree(got, ref)
    assert got["min_wall_clearance"] == 0.0 and got["min_pair_clearance"] < 0.5


def test_check_of_a_local_planner_epoch():
    """A velocity-obstacle plan: clearances on segment 0, cost C'_i |x - x_ref|^2
    on segment 1."""
    import paper_1311_4527_gb300 as pk
    inst = workloads.circle_swap(4, 2, 0.15, 0.01, 2)
    with pk.Planner.velocity_obstacle(inst.start, inst.goal, inst.radius, np.ones(4), 0.2) as pl:
        pl.vo_epoch(0.5)
        z = pl.trajectory().cpu().numpy().astype(np.float64)
        st, gl = pl.endpoints()
        got = pl.check()
    r32 = inst.radius.astype(np.float32).astype(np.float64)
    R = r32[:, None] + r32[None, :]
    worst = np.inf
    for i in range(4):
        for j in range(i + 1, 4):
            a, b = z[j, 0] - z[i, 0], z[j, 1] - z[i, 1]
            d = b - a
            t = np.clip(-(a @ d) / (d @ d), 0.0, 1.0) if d @ d > 0 else 0.0
            worst = min(worst, np.linalg.norm(a + t * d) / R[i, j])
    assert abs(got["min_pair_clearance"] - worst) <= 1e-9 * worst
    cost = float(np.sum((z[:, 2] - z[:, 1]) ** 2))
    assert abs(got["total_cost"] - cost) <= 1e-12 * cost
