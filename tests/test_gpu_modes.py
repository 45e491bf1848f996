"""GPU parity and solves of the variant factors and modes: the feasibility
problem without kinetic factors (zero back weights and the minimizers' zero-
weight limits), maximum / minimum velocity factors (Appendices F, G), and the
recovery of collision-free paths from a stopped energy solve (switching the
kinetic factors off)."""
import numpy as np
import pytest

import workloads
from oracle import twa

import _parity as par

pytestmark = pytest.mark.gpu


def _run(prob, ks):
    out = []
    st = twa.initial_state(prob)
    done = 0
    for k in sorted(ks):
        while done < k:
            st, _ = twa.iterate(prob, st)
            done += 1
        new, info = twa.iterate(prob, st, record_branches=True)
        gpu = par.gpu_step(prob, st)
        stats = par.compare(prob, new, info, gpu)
        stats["k"] = k
        out.append(stats)
    return out


def _seg_lengths(z):
    return np.linalg.norm(z[:, 1:] - z[:, :-1], axis=-1)


def test_feasibility_parity_circle4():
    prob = twa.Problem.from_instance(workloads.circle4(), energy=False)
    stats = _run(prob, [0, 1, 2, 4, 8, 12])
    assert sum(s["coll_active"] for s in stats) > 0


def test_feasibility_parity_with_walls_and_zero_weight_nodes():
    inst = workloads.obstacle_square(40, 5, 9.0, 4, 3)
    prob = twa.Problem.from_instance(inst, cost_unnorm=True, energy=False)
    # the oracle run reaches break-points with only zero incoming weights
    st = twa.initial_state(prob)
    for _ in range(3):
        st, _ = twa.iterate(prob, st)
    assert (st.wback[:, 1:-1] == twa.W0).any()
    stats = _run(prob, [0, 3, 10])
    assert sum(s["coll_active"] for s in stats) > 0


@pytest.mark.parametrize("kind", ["max", "min", "both_no_energy"])
def test_velocity_factor_parity(kind):
    inst = workloads.circle4()
    if kind == "max":
        prob = twa.Problem.from_instance(inst, vmax=np.full((4, 4), 0.5))
    elif kind == "min":
        prob = twa.Problem.from_instance(inst, vmin=np.full((4, 4), 0.42))
    else:
        prob = twa.Problem.from_instance(inst, vmax=np.full((4, 4), 0.62),
                                         vmin=np.full((4, 4), 0.05), energy=False)
    stats = _run(prob, [0, 2, 10, 60])
    keys = [k for k in stats[0] if k.startswith("v") and k.endswith("_active")]
    assert keys and sum(s[k] for s in stats for k in keys) > 0, stats


def test_feasibility_solve_matches_the_oracle_iteration_count():
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst, energy=False)
    st, it_o, res = twa.solve(prob, 1e-7, 2000)
    pl = par.make_planner(prob, check_every=1, tol=1e-7)
    conv, it, r = pl.solve()
    z = pl.trajectory().cpu().numpy().astype(np.float64)
    pl.close()
    assert conv and abs(it - it_o) <= 2, (it, it_o)
    assert twa.min_clearance(prob, z)[0] >= 1 - 1e-4


def test_velocity_limit_holds_at_gpu_convergence():
    inst = workloads.circle4()
    vmax = np.full((4, 4), 0.56)
    prob = twa.Problem.from_instance(inst, vmax=vmax)
    pl = par.make_planner(prob, check_every=10)
    conv, it, r = pl.solve()
    z = pl.trajectory().cpu().numpy().astype(np.float64)
    pl.close()
    assert conv
    assert np.all(_seg_lengths(z) <= vmax * (1 + 1e-4))
    assert twa.min_clearance(prob, z)[0] >= 1 - 1e-4


def test_feasibility_at_scale():
    """p = 100 circle swap without kinetic factors: a collision-free plan in
    a few hundred iterations at most."""
    inst = workloads.circle100()
    prob = twa.Problem.from_instance(inst, energy=False)
    pl = par.make_planner(prob, check_every=10, tol=1e-6, max_iter=5000)
    conv, it, r = pl.solve()
    z = pl.trajectory().cpu().numpy().astype(np.float64)
    pl.close()
    assert conv, (it, r)
    assert twa.min_clearance(prob, z)[0] >= 1 - 1e-4


def test_feasibility_parity_p256():
    """p = 256 random square with walls, no kinetic factors: one GPU
    iteration from the oracle's iterates 0 and 40 (thousands of active
    collision factors, zero-weight break-points)."""
    inst = workloads.small_square(256, 8, 5)
    prob = twa.Problem.from_instance(inst, energy=False)
    stats = _run(prob, [0, 40])
    for s in stats:
        assert s["coll_active"] > 1000 and s["coll_excluded"] <= 0.02 * s["coll_active"], s


def test_recovery_of_a_stopped_energy_solve():
    """A p = 48 random-square energy solve stopped after 300 iterations
    still collides; switching the kinetic factors off (the feasibility
    problem from that state) reaches a collision-free plan in about the
    oracle's number of iterations (the paper's recovery of a non-colliding
    plan at low cost)."""
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(48, 8, 2)
    prob = twa.Problem.from_instance(inst)
    st = twa.initial_state(prob)
    for _ in range(300):
        st, _ = twa.iterate(prob, st)
    assert twa.min_clearance(prob, st.z)[0] < 1 - 1e-3
    pf = twa.Problem.from_instance(inst, energy=False)
    for k_o in range(1, 3001):
        st, info = twa.iterate(pf, st)
        if info.residual < 1e-9:
            break
    pl = pk.Planner.from_instance(inst)
    pl.iterate(300)
    pl.set_energy(False)
    k = 0
    r = 1.0
    while r > 1e-9 and k < 3000:
        r = pl.iterate(1, residual=True)
        k += 1
    z = pl.trajectory().cpu().numpy().astype(np.float64)
    pl.close()
    after = twa.min_clearance(prob, z)
    assert r <= 1e-9 and after[0] >= 1 - 1e-4 and after[1] >= 1 - 1e-4, (k, r, after)
    assert abs(k - k_o) <= 0.25 * k_o + 10, (k, k_o)
