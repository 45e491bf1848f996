"""GPU parity: one FP32 CUDA iteration from an oracle iterate against the FP64
oracle's next iterate, entry by entry (see tests/_parity.py for the rules).
Cases span one tile and several tiles with ragged tails, walls, fixed ends,
the U_KEEP reading, the printed (alpha / rho0) dual step with and without the
rho warm-up, and the dense-state streaming mode."""
import numpy as np
import pytest

import workloads
from oracle import twa

import _parity as par

pytestmark = pytest.mark.gpu


def _run(prob, ks, flags=0):
    """Parity at each iterate k in ks; returns the stats of every step."""
    out = []
    st = twa.initial_state(prob)
    done = 0
    for k in sorted(ks):
        while done < k:
            st, _ = twa.iterate(prob, st)
            done += 1
        new, info = twa.iterate(prob, st, record_branches=True)
        gpu = par.gpu_step(prob, st, flags=flags)
        stats = par.compare(prob, new, info, gpu)
        stats["k"] = k
        out.append(stats)
    return out


def _prob(inst, **kw):
    return twa.Problem.from_instance(inst, **kw)


@pytest.mark.parametrize("dense", [False, True])
def test_circle4_parity_along_the_solve(dense):
    import paper_1311_4527_gb300 as pk
    prob = _prob(workloads.circle4())
    stats = _run(prob, [0, 1, 5, 40, 200], flags=pk.PLAN_DENSE_STATE if dense else 0)
    assert sum(s["coll_active"] for s in stats) > 0
    assert all(s["coll_excluded"] <= 2 for s in stats), stats


def test_circle100_parity():
    prob = _prob(workloads.circle100())
    stats = _run(prob, [0, 12])
    for s in stats:
        # near-ties are few; each one hides every node it touches, and at the
        # first iteration all 4950 pairs of the last segment share nodes
        assert s["coll_excluded"] <= 0.02 * s["coll_active"], s
        assert s["coll_compared_active"] > 0, s


def test_square_with_walls_ragged_tiles_parity():
    # p = 72: three 32-agent tiles, the last one ragged; walls on all sides
    inst = workloads.small_square(72, 6, seed=11)
    prob = _prob(inst, cost_unnorm=True)
    stats = _run(prob, [0, 3, 25])
    assert sum(s["coll_active"] for s in stats) > 0


def test_ragged_single_extra_agent_parity():
    # p = 33: a second tile holding one agent
    inst = workloads.circle_swap(33, 3, None, 0.004, 321, radius_range=(0.02, 0.05))
    prob = _prob(inst)
    _run(prob, [0, 7])


def test_single_agent_and_single_segment():
    prob = _prob(workloads.circle_swap(1, 5, 0.1, 0.0, 5))
    _run(prob, [0, 3])
    inst = workloads.circle_swap(6, 1, 0.1, 0.01, 6)
    prob = _prob(inst)
    st = twa.initial_state(prob)
    new, info = twa.iterate(prob, st, record_branches=True)
    gpu = par.gpu_step(prob, st)
    par.compare(prob, new, info, gpu)
    assert np.array_equal(gpu["z"], st.z.astype(np.float32))


def test_u_keep_reading_parity():
    prob = _prob(workloads.circle4(), u_keep=True)
    _run(prob, [0, 6, 30])


def test_literal_dual_step_parity():
    """App. B step 7 as printed, u += (alpha / rho0)(x - z), on the p = 100
    circle, whose rho0 = 2 makes it differ from the scaled-dual step."""
    prob = _prob(workloads.circle100(), u_literal=True)
    stats = _run(prob, [0, 12])
    for s in stats:
        assert s["coll_excluded"] <= 0.02 * s["coll_active"], s
    assert stats[-1]["coll_compared_active"] > 0


def test_literal_dual_step_across_the_rho_warm_up():
    """The warm-up of Section 4 (rho = warm_rho for the first iterations):
    the first iteration after it finishes the last warm-up iteration's dual
    step, which divides alpha by warm_rho."""
    prob = _prob(workloads.circle4(), u_literal=True, warm_iters=3, warm_rho=0.25)
    _run(prob, [0, 2, 3, 4, 9])


def test_per_segment_costs_and_unnormalised_cost_parity():
    inst = workloads.circle_swap(5, 6, 0.2, 0.01, 55)
    rng = np.random.default_rng(0)
    prob = _prob(inst, cost_unnorm=True)
    prob.cost = rng.uniform(0.5, 2.0, size=(5, 6))
    _run(prob, [0, 10])


def test_full_size_square1024_one_iteration():
    """p=1024, eta=16, 4 walls (8.4M collision factors) in the launch
    configuration the benchmark times: the first iteration and one from the
    oracle's second iterate, compared entry by entry."""
    prob = _prob(workloads.square1024())
    stats = _run(prob, [0, 2])
    for s in stats:
        assert s["coll_active"] > 10000
        assert s["coll_excluded"] < 0.01 * s["coll_active"], s


def test_full_size_square1024_from_a_crowded_iterate():
    """The state the benchmark times: p = 1024, eta = 16 with walls from the
    oracle's iterate 20 (about 19,000 active pairs, previously active pairs
    dealt over each warp).  One GPU step from that iterate, then a second
    from the GPU's own state, in which the tiles that needed many exact
    tests in the first step are dispatched first, each against the oracle's
    next iterate (the second step leaves out the break-points where the two
    states it starts from differ, and everything that reads them)."""
    prob = _prob(workloads.square1024())
    st = par.oracle_state(prob, 20)
    new1, info1 = twa.iterate(prob, st, record_branches=True)
    new2, info2 = twa.iterate(prob, new1, record_branches=True)
    with par.make_planner(prob) as pl:
        g1 = par.gpu_step(prob, st, planner=pl)
        s1 = par.compare(prob, new1, info1, g1)
        pl.iterate(1)
        g2 = par.gpu_export(prob, pl)
        s2 = par.compare(prob, new2, info2, g2, prior_bad=par.differing_nodes(prob, new1, g1))
    for s in (s1, s2):
        assert s["coll_active"] > 10000, s
    assert s1["coll_excluded"] < 0.01 * s1["coll_active"], s1
    assert s1["coll_compared_active"] > 0.5 * s1["coll_active"], s1
    # at this density the first step's near-ties reach many neighbours in the
    # second (every factor reading a break-point that differs is left out, and
    # every u reading a break-point so reached), so fewer pairs remain
    assert s2["coll_compared_active"] > 500, s2


def test_standard_admm_mode_parity():
    prob = _prob(workloads.circle4(), admm=True)
    _run(prob, [0, 4, 40])
    prob = _prob(workloads.small_square(40, 5, seed=9), cost_unnorm=True, admm=True)
    _run(prob, [0, 6])


def test_interior_wall_segments_parity():
    """Static obstacles beyond the bounding box (Section 3.2): five interior
    axis-aligned wall segments plus the four sides; p = 48 (two tiles, the
    second ragged)."""
    inst = workloads.obstacle_square(48, 6, 10.0, 5, 7)
    prob = _prob(inst, cost_unnorm=True)
    stats = _run(prob, [0, 3, 30, 150])
    assert sum(s.get("wall_active", 0) for s in stats) > 0, stats


def test_more_active_walls_than_minimizer_ctas_parity():
    """An obstacle course (p = 300, eta = 8, the four sides and 60 interior
    walls) with about 1,600 active wall factors: more than the minimizer pass
    has CTAs, so it deals the walls over all its warps before the collision
    groups.  Parity at the oracle's iterates 0 and 3."""
    inst = workloads.obstacle_square(300, 8, 25.0, 60, 3)
    prob = _prob(inst)
    stats = _run(prob, [0, 3])
    for s in stats:
        assert s.get("wall_active", 0) > 1000, s
        assert s["coll_excluded"] <= 0.02 * s["coll_active"], s
