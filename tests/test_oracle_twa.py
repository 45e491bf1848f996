"""Pins of the oracle's TWA iteration (Appendix B over the graph of Section
3.3) against invariants and closed-form optima.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import workloads
from oracle import twa

HERE = os.path.dirname(os.path.abspath(__file__))


def _problem(start, goal, radius, eta, cost=None, walls=None, rho0=1.0, **kw):
    start = np.asarray(start, dtype=np.float64)
    p = start.shape[0]
    if cost is None:
        cost = np.ones((p, eta))
    return twa.Problem(p=p, eta=eta, start=start, goal=np.asarray(goal, dtype=np.float64),
                       radius=np.asarray(radius, dtype=np.float64), cost=np.asarray(cost, dtype=np.float64),
                       walls=np.zeros((0, 4)) if walls is None else np.asarray(walls, dtype=np.float64),
                       rho0=rho0, **kw)


def test_single_agent_free_space_straight_line():
    """Appendix A: one agent in free space ends on the straight line."""
    prob = _problem([[0.0, 0.0]], [[3.0, 1.0]], [0.2], eta=8, cost_unnorm=True)
    st, it, res = twa.solve(prob, 1e-10, 20000)
    assert res < 1e-10
    assert np.allclose(st.z, twa.straight_lines(prob), atol=1e-8)


def test_well_separated_agents_converge_to_straight_lines():
    """No collision factor ever activates, so the optimum of the kinetic cost
    with fixed ends is the constant-velocity line of every agent."""
    start = [[0.0, 0.0], [0.0, 5.0], [0.0, 10.0]]
    goal = [[4.0, 1.0], [4.0, 6.0], [4.0, 11.0]]
    prob = _problem(start, goal, [0.3, 0.3, 0.3], eta=5, cost_unnorm=True)
    st = twa.initial_state(prob)
    for _ in range(3000):
        st, info = twa.iterate(prob, st)
        assert not info.active_coll.any()
    assert np.allclose(st.z, twa.straight_lines(prob), atol=1e-8)
    assert np.all(st.u_coll == 0.0)


def test_per_segment_costs_reach_the_tridiagonal_optimum():
    """With costs C_s that vary along the path, the optimum of
    sum_s c_s |x_{s+1} - x_s|^2 with fixed ends solves a tridiagonal linear
    system (solved here directly with a banded solver)."""
    from scipy.linalg import solve_banded
    rng = np.random.default_rng(3)
    eta = 6
    c = rng.uniform(0.5, 3.0, size=eta)
    x0, xe = np.array([0.0, 0.0]), np.array([2.0, -1.0])
    prob = _problem([x0], [xe], [0.1], eta=eta, cost=c[None, :], cost_unnorm=True)
    st, it, res = twa.solve(prob, 1e-11, 50000)
    # normal equations for the free points x_1..x_{eta-1}
    nfree = eta - 1
    ab = np.zeros((3, nfree))
    ab[1] = c[:-1] + c[1:]
    ab[0, 1:] = -c[1:-1]
    ab[2, :-1] = -c[1:-1]
    rhs = np.zeros((nfree, 2))
    rhs[0] += c[0] * x0
    rhs[-1] += c[-1] * xe
    x = solve_banded((1, 1), ab, rhs)
    assert np.allclose(st.z[0, 1:eta], x, atol=1e-8)


def test_circle4_converges_to_a_feasible_plan():
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    st, it, res = twa.solve(prob, inst.tol, inst.max_iter)
    assert res < inst.tol
    coll, wall = twa.min_clearance(prob, st.z)
    assert coll >= 1.0 - 1e-4
    assert np.array_equal(st.z[:, 0], prob.start) and np.array_equal(st.z[:, -1], prob.goal)
    # avoiding the centre costs energy over the colliding straight lines
    assert twa.total_cost(prob, st.z) > twa.total_cost(prob, twa.straight_lines(prob))
    with open(os.path.join(HERE, "golden", "circle4_eta4.json")) as f:
        g = json.load(f)
    assert it == g["iterations"]
    assert abs(twa.total_cost(prob, st.z) - g["total_cost"]) <= 1e-12 * g["total_cost"]


def test_consensus_is_a_convex_combination_of_incoming_messages():
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    st = twa.initial_state(prob)
    seen_active = False
    for _ in range(40):
        new, info = twa.iterate(prob, st, record_edges=True)
        seen_active |= bool(info.active_coll.any())
        by_node = {}
        for i, s, m, w in info.extra["edges"]:
            by_node.setdefault((i, s), []).append(m)
        for (i, s), ms in by_node.items():
            if s in (0, prob.eta):
                continue
            ms = np.array(ms)
            assert np.all(new.z[i, s] >= ms.min(axis=0) - 1e-12)
            assert np.all(new.z[i, s] <= ms.max(axis=0) + 1e-12)
        st = new
    assert seen_active


def _permuted(prob, perm):
    return twa.Problem(p=prob.p, eta=prob.eta, start=prob.start[perm], goal=prob.goal[perm],
                       radius=prob.radius[perm], cost=prob.cost[perm], walls=prob.walls,
                       rho0=prob.rho0, alpha=prob.alpha)


def test_agent_relabelling_permutes_the_iterates():
    inst = workloads.circle_swap(6, 4, None, 0.02, 77, radius_range=(0.1, 0.2))
    prob = twa.Problem.from_instance(inst)
    perm = np.array([3, 0, 5, 1, 4, 2])
    q = _permuted(prob, perm)
    a, b = twa.initial_state(prob), twa.initial_state(q)
    for _ in range(60):
        a, ia = twa.iterate(prob, a)
        b, ib = twa.iterate(q, b)
    assert np.allclose(b.z, a.z[perm], atol=1e-12)


def test_translation_moves_the_plan_and_leaves_u():
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    shift = np.array([3.0, -2.0])
    q = twa.Problem(p=prob.p, eta=prob.eta, start=prob.start + shift, goal=prob.goal + shift,
                    radius=prob.radius, cost=prob.cost, walls=prob.walls, rho0=prob.rho0,
                    alpha=prob.alpha)
    a, b = twa.initial_state(prob), twa.initial_state(q)
    for _ in range(50):
        a, _ = twa.iterate(prob, a)
        b, _ = twa.iterate(q, b)
    assert np.allclose(b.z, a.z + shift, atol=1e-11)
    assert np.allclose(b.u_coll, a.u_coll, atol=1e-11)


def test_one_segment_has_no_free_variable():
    prob = _problem([[0.0, 0.0], [1.0, 0.0]], [[1.0, 1.0], [0.0, 1.0]], [0.2, 0.2], eta=1)
    st = twa.initial_state(prob)
    st2, info = twa.iterate(prob, st)
    assert np.array_equal(st2.z, st.z)
    assert info.dz == 0.0


def test_inactive_factors_reset_u_or_keep_it():
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    st = twa.initial_state(prob)
    for _ in range(30):
        st, info = twa.iterate(prob, st)
    inactive = ~info.active_coll
    assert np.all(st.u_coll[inactive] == 0.0)
    assert np.any(st.u_coll[info.active_coll] != 0.0)
    keep = twa.Problem.from_instance(inst, u_keep=True)
    st = twa.initial_state(keep)
    for _ in range(30):
        prev = st.u_coll.copy()
        st, info = twa.iterate(keep, st)
        assert np.array_equal(st.u_coll[~info.active_coll], prev[~info.active_coll])


def test_literal_dual_step_is_the_scaled_step_with_alpha_over_rho():
    """App. B step 7 as printed, u += (alpha / rho0)(x - z): with rho0 = 1 it
    is the scaled-dual step exactly; with rho0 = 2 it is that step with
    alpha / 2 (the minimizers and the consensus do not see alpha); during a
    warm-up it divides by the warm-up rho of each iteration."""
    inst = workloads.circle4()
    a = twa.Problem.from_instance(inst, u_literal=True)
    b = twa.Problem.from_instance(inst)
    sa, sb = twa.initial_state(a), twa.initial_state(b)
    for _ in range(40):
        sa, _ = twa.iterate(a, sa)
        sb, _ = twa.iterate(b, sb)
    assert np.array_equal(sa.z, sb.z) and np.array_equal(sa.u_coll, sb.u_coll)
    a = twa.Problem.from_instance(inst, u_literal=True)
    a.rho0 = 2.0
    b = twa.Problem.from_instance(inst)
    b.rho0, b.alpha = 2.0, inst.alpha / 2.0
    sa, sb = twa.initial_state(a), twa.initial_state(b)
    for _ in range(40):
        sa, _ = twa.iterate(a, sa)
        sb, _ = twa.iterate(b, sb)
    assert np.allclose(sa.z, sb.z, atol=1e-13) and np.allclose(sa.u_kin, sb.u_kin, atol=1e-13)
    # warm-up: the first 3 iterations divide alpha by warm_rho = 0.25 (4 alpha)
    a = twa.Problem.from_instance(inst, u_literal=True, warm_iters=3, warm_rho=0.25)
    b = twa.Problem.from_instance(inst, warm_iters=3, warm_rho=0.25)
    b.alpha = 4.0 * inst.alpha
    sa, sb = twa.initial_state(a), twa.initial_state(b)
    for _ in range(3):
        sa, _ = twa.iterate(a, sa)
        sb, _ = twa.iterate(b, sb)
    assert np.allclose(sa.u_kin, sb.u_kin, atol=1e-13) and np.any(sa.u_kin != 0.0)
    b.alpha = inst.alpha
    for _ in range(5):
        sa, _ = twa.iterate(a, sa)
        sb, _ = twa.iterate(b, sb)
    assert np.allclose(sa.z, sb.z, atol=1e-13)


def test_fixed_ends_stay_exact_and_edges_to_them_carry_no_u():
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    st = twa.initial_state(prob)
    for _ in range(25):
        st, _ = twa.iterate(prob, st)
        assert np.array_equal(st.z[:, 0], prob.start)
        assert np.array_equal(st.z[:, prob.eta], prob.goal)
        assert np.all(st.u_kin[0, :, 0] == 0.0) and np.all(st.u_kin[-1, :, 1] == 0.0)
        assert np.all(st.u_coll[0, :, 0] == 0.0) and np.all(st.u_coll[0, :, 2] == 0.0)


def test_corridor_swap_touches_the_walls_and_stays_feasible():
    """Two agents swap ends of a corridor whose height leaves 0.62 for two
    disks that need 0.6 to pass: both collision and wall factors activate,
    and the converged plan touches the walls without crossing them."""
    walls = [[-1.0, 0.0, 5.0, 0.0], [-1.0, 1.22, 5.0, 1.22]]
    prob = _problem([[0.0, 0.62], [4.0, 0.6]], [[4.0, 0.66], [0.0, 0.62]], [0.3, 0.3], eta=8,
                    walls=walls, cost_unnorm=True)
    st = twa.initial_state(prob)
    walls_active = 0
    for _ in range(20000):
        st, info = twa.iterate(prob, st)
        walls_active = max(walls_active, int(info.active_wall.sum()))
        if info.residual < 1e-7:
            break
    assert info.residual < 1e-7
    assert walls_active > 0
    coll, wall = twa.min_clearance(prob, st.z)
    assert coll >= 1.0 - 1e-4 and wall >= 1.0 - 1e-4
    assert wall <= 1.0 + 1e-4      # the plan does lean on a wall


def test_wall_factor_pushes_a_passing_agent_clear():
    """One agent whose straight line passes too close to a wall converges to
    a feasible path that bends under it and leans on the wall's end caps."""
    # the straight line y = 0.4 passes 0.1 from this wall; radius 0.3
    walls = [[-1.0, 0.5, 1.0, 0.5]]
    prob = _problem([[-3.0, 0.4]], [[3.0, 0.4]], [0.3], eta=8, walls=walls, cost_unnorm=True)
    st, it, res = twa.solve(prob, 1e-9, 30000)
    assert res < 1e-9
    coll, wall = twa.min_clearance(prob, st.z)
    assert 1.0 - 1e-4 <= wall <= 1.0 + 1e-4
    _, wall_sl = twa.min_clearance(prob, twa.straight_lines(prob))
    assert wall_sl < 1.0          # the unconstrained optimum was infeasible
    # mirror symmetry of the problem about x = 0 survives in the plan
    assert np.allclose(st.z[0, :, 0], -st.z[0, ::-1, 0], atol=1e-8)


# ---------------------------------------------------------------------------
# standard-ADMM mode (Appendix B: every weight rho0)
# ---------------------------------------------------------------------------

def _separated(admm):
    start = [[0.0, 0.0], [0.0, 5.0], [0.0, 10.0]]
    goal = [[4.0, 1.0], [4.0, 6.0], [4.0, 11.0]]
    return _problem(start, goal, [0.3, 0.3, 0.3], eta=4, cost_unnorm=True, admm=admm)


def test_admm_first_step_is_damped_by_the_node_degree():
    """From the same start, every feasible collision factor sends m = z, so
    an interior node's move is the TWA move over p (2 kinetic edges among
    2(p-1) + 2)."""
    a, _ = twa.iterate(_separated(False), twa.initial_state(_separated(False)))
    b, _ = twa.iterate(_separated(True), twa.initial_state(_separated(True)))
    z0 = twa.initial_state(_separated(False)).z
    assert np.allclose((b.z - z0)[:, 1:-1], (a.z - z0)[:, 1:-1] / 3, atol=1e-14)


def test_admm_mode_still_reaches_the_straight_lines():
    """The feasible collision factors' pull towards the previous iterate
    vanishes at the fixed point, which stays the constant-velocity lines."""
    prob = _separated(True)
    st, it, res = twa.solve(prob, 1e-9, 50000)
    assert res < 1e-9
    assert np.allclose(st.z, twa.straight_lines(prob), atol=1e-7)
    assert np.abs(st.u_coll).max() < 1e-6


def test_admm_mode_updates_u_on_feasible_factors():
    prob = _separated(True)
    st = twa.initial_state(prob)
    for _ in range(3):
        st, info = twa.iterate(prob, st)
    assert not info.active_coll.any()
    assert np.any(st.u_coll != 0.0)  # weighted although never colliding
