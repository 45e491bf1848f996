"""GPU solver behaviour over many iterations: convergence on the p=4 circle
swap to the oracle's cost, feasibility of converged plans, determinism, the
dense-state and bit-gated modes agreeing bit for bit, warm-start re-planning
and the non-finite detector."""
import json
import math
import os

import numpy as np
import pytest

import workloads
from oracle import twa

import _parity as par

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _solve(inst, **kw):
    import paper_1311_4527_gb300 as pk
    pl = pk.Planner.from_instance(inst, check_every=kw.pop("check_every", 1), **kw)
    conv, it, res = pl.solve()
    z = pl.trajectory().cpu().numpy().astype(np.float64)
    pl.close()
    return conv, it, res, z


def test_circle4_converged_cost_matches_the_oracle():
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    g = json.load(open(os.path.join(HERE, "golden", "circle4_eta4.json")))
    conv, it, res, z = _solve(inst)
    assert conv, (it, res)
    cost = twa.total_cost(prob, z)
    assert abs(cost - g["total_cost"]) <= 1e-3 * g["total_cost"], (cost, g["total_cost"])
    coll, _ = twa.min_clearance(prob, z)
    assert coll >= 1.0 - 1e-4
    assert np.abs(z[:, 0] - inst.start).max() <= 1e-6 * par.scale_of(prob) + 1e-7
    assert np.abs(z[:, -1] - inst.goal).max() <= 1e-6 * par.scale_of(prob) + 1e-7
    # the converged plan is close to the oracle's, not just equally cheap
    assert np.abs(z - np.array(g["z"])).max() <= 1e-3


def test_circle100_converges_to_a_feasible_plan():
    """The p = 100 circle swap (rho0 = 2, alpha = 0.1) reaches the 1e-6
    residual in about 154,000 iterations (the 20,000-iteration cap of the
    p = 4 case is far too short for it); the plan is then collision-free to
    (r_i + r_j)(1 - 1e-4) and keeps its endpoints, checked both by the FP64
    device check and by the oracle's functions on the same break-points."""
    import paper_1311_4527_gb300 as pk
    inst = workloads.circle100()
    prob = twa.Problem.from_instance(inst)
    with pk.Planner.from_instance(inst, max_iter=300000, check_every=1000) as pl:
        conv, it, res = pl.solve()
        z = pl.trajectory().cpu().numpy().astype(np.float64)
        chk = pl.check()
    assert conv, (it, res)
    assert 100000 <= it <= 250000, it
    coll, _ = twa.min_clearance(prob, z)
    assert coll >= 1.0 - 1e-4 and chk["min_pair_clearance"] >= 1.0 - 1e-4
    assert chk["max_endpoint_error"] <= 1e-6
    assert np.array_equal(z[:, 0], inst.start.astype(np.float32))
    assert abs(chk["total_cost"] - twa.total_cost(prob, z)) <= 1e-12 * chk["total_cost"]


@pytest.mark.parametrize("name", ["circle100", "square256", "square1024"])
def test_dense_and_gated_state_are_bitwise_identical(name):
    """The gated state's bounding-circle filter drops no pair the exact test
    would find active, and its tile order (crowded tiles of the previous
    iteration first, the rest segment-minor) changes nothing: both modes take
    the same branches everywhere (unit circle; a 40 x 40-scale square where
    the filter's margin is set by large coordinates; the p = 1024 square,
    whose crowded tiles are dispatched first)."""
    import paper_1311_4527_gb300 as pk
    if name == "circle100":
        inst = workloads.circle100()
    elif name == "square256":
        inst = workloads.small_square(256, 8, seed=5, side=40.0)
    else:
        inst = workloads.square1024()
    zs, acts = [], []
    for flags in (0, pk.PLAN_DENSE_STATE):
        pl = pk.Planner.from_instance(inst, flags=flags)
        pl.iterate(150)
        zs.append(pl.trajectory().cpu().numpy())
        acts.append(pl.info()["active_coll"])
        pl.close()
    assert np.array_equal(zs[0], zs[1])
    assert acts[0] == acts[1]


def test_runs_are_deterministic():
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(100, 8, seed=3)
    outs = []
    for _ in range(2):
        pl = pk.Planner.from_instance(inst)
        r = pl.iterate(60, residual=True)
        outs.append((pl.trajectory().cpu().numpy(), r, pl.info()["active_coll"]))
        pl.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2]


def test_residual_matches_the_oracle_definition():
    import paper_1311_4527_gb300 as pk
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    st = twa.initial_state(prob)
    pl = pk.Planner.from_instance(inst)
    for k in range(12):
        st, info = twa.iterate(prob, st)
        r = pl.iterate(1, residual=True)
        assert abs(r - info.residual) <= 2e-5 * max(1.0, info.residual), (k, r, info.residual)
    pl.close()


def test_warm_start_replanning_moves_the_goals():
    import paper_1311_4527_gb300 as pk
    inst = workloads.circle4()
    pl = pk.Planner.from_instance(inst, check_every=1)
    conv, it, _ = pl.solve()
    assert conv
    goal = inst.goal * 1.2
    pl.set_endpoints(inst.start, goal)
    z = pl.trajectory().cpu().numpy()
    assert np.allclose(z[:, -1], goal.astype(np.float32))
    r = pl.iterate(2000, residual=True)
    z = pl.trajectory().cpu().numpy()
    prob = twa.Problem.from_instance(inst)
    prob.goal = goal
    coll, _ = twa.min_clearance(prob, z.astype(np.float64))
    assert r < 1e-3 and coll >= 1.0 - 1e-3
    pl.close()


def test_non_finite_state_is_reported():
    import paper_1311_4527_gb300 as pk
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    st = twa.initial_state(prob)
    st.z[1, 2] = np.nan  # injected on the host into the imported state
    pl = pk.Planner.from_instance(inst, check_every=1, max_iter=5)
    pl.import_state(st.z, st.u_coll, st.u_kin, None, 0)
    with pytest.raises(pk.PlanError) as e:
        pl.solve()
    assert e.value.status == "PLAN_ENUMERIC"
    pl.close()


def test_info_counts():
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(72, 6, seed=11)
    pl = pk.Planner.from_instance(inst)
    pl.iterate(3)
    inf = pl.info()
    assert inf["n_coll"] == 6 * 72 * 71 // 2 and inf["n_kin"] == 6 * 72
    assert inf["n_wall"] == 4 * 6 * 72 and inf["k"] == 3
    ex = pl.export_state()
    assert inf["active_coll"] == int(ex["act_coll"].sum().item())
    pl.close()


def test_admm_and_twa_converge_on_circle4_like_the_oracle():
    """Standard ADMM and TWA on the p = 4 circle: each GPU solve converges to
    the oracle's cost for that mode, and TWA needs fewer iterations."""
    import paper_1311_4527_gb300 as pk
    inst = workloads.circle4()
    its = {}
    for admm in (False, True):
        prob = twa.Problem.from_instance(inst, admm=admm)
        st, o_it, _ = twa.solve(prob, inst.tol, inst.max_iter)
        conv, it, res, z = _solve(inst, flags=pk.PLAN_ADMM if admm else 0)
        assert conv
        assert abs(twa.total_cost(prob, z) - twa.total_cost(prob, st.z)) <= 1e-3 * twa.total_cost(prob, st.z)
        assert abs(it - o_it) <= 0.05 * o_it + 5
        its[admm] = it
    assert its[False] < its[True]


def _first_violation(start, goal, radius, walls):
    """Brute force, in the device check's order: start pairs, goal pairs,
    start-wall, goal-wall; then the lower agent, then the partner."""
    p = start.shape[0]
    X32 = [np.asarray(start, np.float32).astype(np.float64), np.asarray(goal, np.float32).astype(np.float64)]
    r = np.asarray(radius, np.float32).astype(np.float64)
    for which in (0, 1):
        X = X32[which]
        for i in range(p):
            d2 = np.sum((X[i + 1:] - X[i]) ** 2, axis=1)
            hit = np.nonzero(d2 < (r[i] + r[i + 1:]) ** 2)[0]
            if hit.size:
                return f"{'goal' if which else 'start'} positions of agents {i} and {i + 1 + hit[0]} overlap"
    W = np.asarray(walls, np.float32).astype(np.float64)
    for which in (0, 1):
        X = X32[which]
        for i in range(p):
            for w in range(W.shape[0]):
                a, b = W[w, :2], W[w, 2:]
                d = b - a
                t = np.clip(np.dot(X[i] - a, d) / np.dot(d, d), 0.0, 1.0)
                if np.sum((a + t * d - X[i]) ** 2) < r[i] ** 2:
                    return f"{'goal' if which else 'start'} of agent {i} is within its radius of wall {w}"
    return None


def test_set_endpoints_checks_new_positions_on_the_device():
    """plan_set_endpoints refuses overlapping starts or goals and positions
    within a wall's reach (checked on the device), names the first violation
    like a brute-force enumeration, and leaves the plan unchanged; feasible
    new endpoints are applied."""
    import torch
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(72, 6, seed=11)
    rng = np.random.default_rng(4)
    with pk.Planner.from_instance(inst) as pl:
        pl.iterate(5)
        z0 = pl.trajectory().clone()
        cases = []
        for _ in range(4):
            st, gl = inst.start.copy(), inst.goal.copy()
            i, j = rng.choice(inst.p, size=2, replace=False)
            ang = rng.uniform(0, 2 * np.pi)
            X = st if rng.uniform() < 0.5 else gl
            X[j] = X[i] + 0.9 * (inst.radius[i] + inst.radius[j]) * np.array([np.cos(ang), np.sin(ang)])
            cases.append((st, gl))
        st = inst.start.copy()
        st[7] = [0.5 * inst.radius[7], 3.0]          # inside the x = 0 wall's reach
        cases.append((st, inst.goal.copy()))
        for st, gl in cases:
            expect = _first_violation(st, gl, inst.radius, inst.walls)
            assert expect is not None
            with pytest.raises(pk.PlanError) as e:
                pl.set_endpoints(st, gl)
            assert e.value.status == "PLAN_EINFEASIBLE_INPUT"
            assert expect in str(e.value), (expect, str(e.value))
            assert torch.equal(pl.trajectory(), z0)
        new_goal = inst.goal.copy()
        new_goal[0] += 0.05
        assert _first_violation(inst.start, new_goal, inst.radius, inst.walls) is None
        pl.set_endpoints(inst.start, new_goal)
        z = pl.trajectory().cpu().numpy()
        assert np.array_equal(z[:, -1], new_goal.astype(np.float32))
        assert np.array_equal(z[:, 0], inst.start.astype(np.float32))


def test_asynchronous_endpoint_updates_report_at_the_next_synchronising_call():
    """plan_set_endpoints_async: a feasible update is applied before the next
    iteration; an infeasible one is not applied and is reported by the next
    call that synchronises (here the trajectory to the host), after which
    the plan takes further updates."""
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(72, 6, seed=11)
    with pk.Planner.from_instance(inst) as pl:
        pl.iterate(5)
        g1 = inst.goal.copy()
        g1[0] += 0.05
        assert _first_violation(inst.start, g1, inst.radius, inst.walls) is None
        pl.set_endpoints(inst.start, g1, wait=False)
        pl.iterate(3)
        z = pl.trajectory_host()
        assert np.array_equal(z[:, -1], g1.astype(np.float32))
        bad = inst.start.copy()
        bad[9] = bad[5] + 0.5 * (inst.radius[5] + inst.radius[9]) * np.array([1.0, 0.0])
        expect = _first_violation(bad, g1, inst.radius, inst.walls)
        assert expect is not None
        pl.set_endpoints(bad, g1, wait=False)          # returns before the check
        pl.iterate(2)
        with pytest.raises(pk.PlanError) as e:
            pl.trajectory_host()
        assert e.value.status == "PLAN_EINFEASIBLE_INPUT" and expect in str(e.value)
        z = pl.trajectory_host()                        # settled: no error any more
        assert np.array_equal(z[:, 0], inst.start.astype(np.float32))
        assert np.array_equal(z[:, -1], g1.astype(np.float32))
        st, gl = pl.endpoints()
        assert np.array_equal(st, inst.start.astype(np.float32)) and np.array_equal(gl, g1.astype(np.float32))
        g2 = g1.copy()
        g2[1] += 0.05
        pl.set_endpoints(inst.start, g2, wait=False)
        assert pl.iterate(1, residual=True) >= 0.0
        assert np.array_equal(pl.trajectory_host()[:, -1], g2.astype(np.float32))


def test_device_endpoint_check_at_large_p():
    """p = 4100 (129 agent tiles, the last holding four agents): every warp of
    the check takes several tile-pair tasks, and the update is applied by
    whichever block finishes last.  Violations planted in the last tile pair,
    in the goals only, among both starts and goals, and against a wall, are
    each reported as the brute-force enumeration's first; a feasible update
    is applied."""
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(4100, 2, seed=23)
    p = inst.p
    assert _first_violation(inst.start, inst.goal, inst.radius, inst.walls) is None
    with pk.Planner.from_instance(inst) as pl:
        pl.iterate(2)
        z0 = pl.trajectory_host()
        cases = []
        gl = inst.goal.copy()
        gl[p - 1] = gl[p - 2] + 0.5 * (inst.radius[p - 2] + inst.radius[p - 1]) * np.array([0.0, 1.0])
        cases.append((inst.start.copy(), gl))
        st = inst.start.copy()
        st[p - 1] = st[3] + 0.5 * (inst.radius[3] + inst.radius[p - 1]) * np.array([1.0, 0.0])
        cases.append((st, gl))
        gl2 = inst.goal.copy()
        gl2[p - 1] = [inst.walls[:, [0, 2]].max() - 0.5 * inst.radius[p - 1], gl2[p - 1][1]]
        cases.append((inst.start.copy(), gl2))
        for st, g in cases:
            expect = _first_violation(st, g, inst.radius, inst.walls)
            assert expect is not None
            with pytest.raises(pk.PlanError) as e:
                pl.set_endpoints(st, g)
            assert e.value.status == "PLAN_EINFEASIBLE_INPUT" and expect in str(e.value), (expect, str(e.value))
            assert np.array_equal(pl.trajectory_host(), z0)
        g3 = inst.goal.copy()
        g3[:, 1] += 1e-3
        if _first_violation(inst.start, g3, inst.radius, inst.walls) is None:
            pl.set_endpoints(inst.start, g3)
            z = pl.trajectory_host()
            assert np.array_equal(z[:, -1], g3.astype(np.float32))
            assert np.array_equal(z[:, 0], inst.start.astype(np.float32))


def test_trajectory_to_pinned_and_pageable_host_memory():
    """plan_get_trajectory into page-locked host memory (16-byte aligned and
    misaligned destinations, nothing written outside them) and into pageable
    memory gives the device trajectory bit for bit."""
    import torch
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(72, 6, seed=11)
    with pk.Planner.from_instance(inst) as pl:
        pl.iterate(7)
        ref = pl.trajectory().cpu().numpy()
        n = ref.size
        pinned = torch.zeros(n + 8, dtype=torch.float32).pin_memory()
        for off in (0, 1, 3):
            pinned.fill_(-1.0)
            view = pinned.numpy()[off:off + n].reshape(ref.shape)
            pl.trajectory_host(view)
            assert np.array_equal(view, ref), off
            assert np.all(pinned.numpy()[:off] == -1.0) and np.all(pinned.numpy()[off + n:] == -1.0)
        pageable = np.full(ref.shape, -1.0, dtype=np.float32)
        pl.trajectory_host(pageable)
        assert np.array_equal(pageable, ref)


def test_non_finite_endpoints_are_refused():
    """A NaN or infinite coordinate in the new starts or goals is refused with
    PLAN_EINVAL (by the device check: waiting, or at the next synchronising
    call), naming the first such agent, and the plan keeps its endpoints."""
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(72, 6, seed=11)
    with pk.Planner.from_instance(inst) as pl:
        pl.iterate(3)
        z0 = pl.trajectory_host()
        for bad_val, which, agent in ((np.nan, 0, 40), (np.inf, 1, 5), (-np.inf, 0, 71)):
            st, gl = inst.start.copy(), inst.goal.copy()
            (st if which == 0 else gl)[agent, 1] = bad_val
            # an overlap further on must not hide it
            gl[70] = gl[69]
            with pytest.raises(pk.PlanError) as e:
                pl.set_endpoints(st, gl)
            assert e.value.status == "PLAN_EINVAL" and f"agent {agent}" in str(e.value), str(e.value)
            assert np.array_equal(pl.trajectory_host(), z0)
            pl.set_endpoints(st, gl, wait=False)
            with pytest.raises(pk.PlanError) as e:
                pl.trajectory_host()
            assert e.value.status == "PLAN_EINVAL" and f"agent {agent}" in str(e.value), str(e.value)
            assert np.array_equal(pl.trajectory_host(), z0)


def test_endpoint_update_above_the_device_check_size():
    """p = 8200 (more than the 8192 agents the device check takes): the host
    grid check refuses an overlap and a position within a wall's reach, and
    leaves the plan unchanged; feasible endpoints are copied and applied by
    the single-block update kernel (fixed break-points of both z buffers,
    the fixed-point scale), after which iterations stay finite; the
    asynchronous form is refused."""
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(8200, 1, seed=29)
    p = inst.p
    with pk.Planner.from_instance(inst) as pl:
        z0 = pl.trajectory_host()
        st = inst.start.copy()
        st[p - 1] = st[p - 2] + 0.5 * (inst.radius[p - 2] + inst.radius[p - 1]) * np.array([1.0, 0.0])
        with pytest.raises(pk.PlanError) as e:
            pl.set_endpoints(st, inst.goal)
        assert e.value.status == "PLAN_EINFEASIBLE_INPUT" and "overlap" in str(e.value)
        gl = inst.goal.copy()
        gl[5] = [0.5 * inst.radius[5], gl[5][1]]  # within the x = 0 wall's reach
        with pytest.raises(pk.PlanError) as e:
            pl.set_endpoints(inst.start, gl)
        assert e.value.status == "PLAN_EINFEASIBLE_INPUT" and "wall" in str(e.value)
        assert np.array_equal(pl.trajectory_host(), z0)
        with pytest.raises(pk.PlanError) as e:
            pl.set_endpoints(inst.start, inst.goal, wait=False)
        assert e.value.status == "PLAN_EUNSUPPORTED"
        # starts and goals exchanged: both configurations were feasible
        pl.set_endpoints(inst.goal, inst.start)
        pl.iterate(3)
        z = pl.trajectory_host()
        assert np.all(np.isfinite(z))
        assert np.array_equal(z[:, 0], inst.goal.astype(np.float32))
        assert np.array_equal(z[:, -1], inst.start.astype(np.float32))
