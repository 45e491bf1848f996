"""Pins of the oracle's velocity-obstacle local planner (Section 5, the
minimizers of Appendix H), CPU only: unconstrained agents go to x_ref; a
head-on pair reaches a collision-free local minimum of Eq. rec_col_avoi_pos;
the epoch loop brings the p = 4 circle swap to its destinations with no
collision along the way."""
import numpy as np

import workloads
from oracle import prox, twa, vo

RHO = 10.0  # rho0 well above C' (the epoch solve stalls for rho0 <= C', reading R20)


def _objective(x, x_ref, c):
    return float(np.sum(c * np.sum((x - x_ref) ** 2, axis=1)))


def _clearance(x0, x, radius):
    iu, ju = twa.pairs(x0.shape[0])
    d = prox.dist_point_segment(np.zeros((iu.shape[0], 2)), x0[ju] - x0[iu], x[ju] - x[iu])
    return float(np.min(d / (radius[iu] + radius[ju])))


def test_free_agents_reach_their_reference_positions():
    x0 = np.array([[0.0, 0.0], [5.0, 5.0], [-5.0, 3.0]])
    dest = np.array([[3.0, 0.0], [5.0, 9.0], [-5.0, 2.5]])
    x, it, res, prob = vo.epoch(x0, dest, np.full(3, 0.3), np.ones(3), 1.0, 1e-12, 5000, rho0=RHO)
    assert res < 1e-12
    assert np.allclose(x, vo.targets(x0, dest, 1.0), atol=1e-10)
    assert np.allclose(prob.goal, [[1.0, 0.0], [5.0, 6.0], [-5.0, 2.5]])


def test_head_on_pair_reaches_a_feasible_local_minimum():
    x0 = np.array([[-0.5, 0.01], [0.5, -0.01]])
    dest = np.array([[2.0, 0.0], [-2.0, 0.0]])
    r = np.array([0.2, 0.2])
    c = np.array([1.0, 1.001])
    x, it, res, prob = vo.epoch(x0, dest, r, c, 0.8, 1e-10, 20000, rho0=RHO)
    assert res < 1e-10
    cl = _clearance(x0, x, r)
    assert 1 - 1e-9 <= cl <= 1 + 1e-6  # the constraint is active
    # no feasible point nearby is better (local minimum of Eq. rec_col_avoi_pos)
    rng = np.random.default_rng(7)
    f0 = _objective(x, prob.goal, c)
    worse = 0
    for _ in range(2000):
        y = x + rng.normal(size=x.shape) * 1e-3
        if _clearance(x0, y, r) >= 1.0:
            assert _objective(y, prob.goal, c) >= f0 - 1e-12
            worse += 1
    assert worse > 100


def test_circle_swap_epochs_reach_the_destinations_without_collision():
    inst = workloads.circle4()
    c = 1 + 0.001 * np.arange(4)  # the paper's symmetry breaking for CONF1
    xs, its = vo.simulate(inst.start, inst.goal, inst.radius, c, 0.25, 0.5, 30, 1e-8, 6000,
                          rho0=RHO)
    assert np.linalg.norm(xs[-1] - inst.goal, axis=1).max() < 1e-3
    for e in range(len(its)):
        assert _clearance(xs[e], xs[e + 1], inst.radius) >= 1 - 1e-6, e
