"""Pins of the oracle's variant factors and modes, CPU only: the maximum and
minimum velocity minimizers (Appendices F and G), the zero-weight limits the
feasibility problem needs, the feasibility-only mode (no kinetic factors,
Eq. basic_opt_prob), and velocity limits inside the energy problem."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

import workloads
from oracle import prox, twa

INF = math.inf
Z = np.zeros(2)


def _objective(x, n, w):
    return 0.5 * w[0] * np.sum((x[:2] - n[:2]) ** 2) + 0.5 * w[1] * np.sum((x[2:] - n[2:]) ** 2)


def _slsqp(n, w, C, kind, starts):
    """Global minimum over several starts of the constrained problem, by a
    general-purpose solver (no use of the appendix's closed form)."""
    sign = 1.0 if kind == "max" else -1.0
    cons = {"type": "ineq", "fun": lambda x: sign * (C * C - np.sum((x[:2] - x[2:]) ** 2))}
    best = None
    for x0 in starts:
        r = minimize(_objective, x0, args=(n, w), constraints=[cons], method="SLSQP",
                     options={"ftol": 1e-14, "maxiter": 500})
        if r.success and cons["fun"](r.x) >= -1e-9 and (best is None or r.fun < best.fun):
            best = r
    return best


@pytest.mark.parametrize("kind", ["max", "min"])
def test_velocity_minimizers_match_a_general_solver(kind):
    rng = np.random.default_rng(41 if kind == "max" else 42)
    checked = 0
    for _ in range(120):
        n = rng.normal(size=4)
        w = rng.uniform(0.2, 3.0, size=2)
        L = float(np.linalg.norm(n[:2] - n[2:]))
        C = L * rng.uniform(0.3, 0.9) if kind == "max" else L * rng.uniform(1.1, 2.5)
        x_lo, x_hi, act = prox.velocity_prox(n[:2], n[2:], w[0], w[1], C, kind)
        assert act
        x = np.concatenate([x_lo, x_hi])
        assert abs(np.linalg.norm(x_lo - x_hi) - C) <= 1e-9 * max(1.0, C)
        starts = [n.copy(), n + rng.normal(size=4) * 0.5, n + rng.normal(size=4) * 2.0,
                  np.concatenate([n[:2] + C * rng.normal(size=2), n[2:]])]
        best = _slsqp(n, w, C, kind, starts)
        if best is None:  # the general solver failed from every start
            continue
        assert _objective(x, n, w) <= best.fun + 1e-8 * max(1.0, best.fun), (n, w, C)
        checked += 1
    assert checked > 90


@pytest.mark.parametrize("kind", ["max", "min"])
def test_velocity_minimizer_inactive_and_limit_weights(kind):
    rng = np.random.default_rng(43)
    for _ in range(50):
        n_lo, n_hi = rng.normal(size=(2, 2))
        L = float(np.linalg.norm(n_lo - n_hi))
        # inside the limit: x = n, inactive
        C_in = 2 * L if kind == "max" else 0.5 * L
        x_lo, x_hi, act = prox.velocity_prox(n_lo, n_hi, 1.0, 1.0, C_in, kind)
        assert not act and np.array_equal(x_lo, n_lo) and np.array_equal(x_hi, n_hi)
        C = 0.5 * L if kind == "max" else 2 * L
        # an infinite weight keeps its end: the limit of a large finite weight
        for wl, wh in ((INF, 1.0), (1.0, INF), (0.0, 1.0), (1.0, 0.0), (0.0, 0.0)):
            big = {INF: 1e9, 0.0: 1e-9}
            fl, fh = big.get(wl, wl), big.get(wh, wh)
            if wl == 0.0 and wh == 0.0:
                fl = fh = 1.0
            ref = prox.velocity_prox(n_lo, n_hi, fl, fh, C, kind)
            got = prox.velocity_prox(n_lo, n_hi, wl, wh, C, kind)
            assert got[2] and np.allclose(got[0], ref[0], atol=1e-7) and np.allclose(got[1], ref[1], atol=1e-7)


def test_min_velocity_with_coincident_ends_uses_the_stated_direction():
    x_lo, x_hi, act = prox.velocity_prox([1.0, 2.0], [1.0, 2.0], 1.0, 3.0, 0.4, "min")
    assert act and np.allclose(x_hi - x_lo, [0.4, 0.0])
    assert np.allclose(0.25 * x_lo + 0.75 * x_hi, [1.0, 2.0])  # weighted mean kept


@pytest.mark.parametrize("capsule", [False, True])
def test_one_sided_zero_weight_is_the_small_weight_limit(capsule):
    """region_prox with one weight 0 (the other finite) against the same
    problem with that weight 1e-8: the argmin converges at rate O(eps)."""
    rng = np.random.default_rng(44 + capsule)
    c0, c1 = (np.array([-0.4, 0.1]), np.array([0.5, -0.2])) if capsule else (Z, Z)
    n = 0
    for _ in range(300):
        r = rng.uniform(0.3, 0.8)
        a, b = rng.normal(size=(2, 2)) * 0.7
        if prox.dist_segment_segment(a, b, c0, c1) >= r:
            continue
        for zero_lo in (True, False):
            w = (0.0, 1.0) if zero_lo else (1.0, 0.0)
            we = (1e-8, 1.0) if zero_lo else (1.0, 1e-8)
            got = prox.region_prox(a, b, w[0], w[1], c0, c1, r)
            ref = prox.region_prox(a, b, we[0], we[1], c0, c1, r)
            err = max(np.abs(got[0] - ref[0]).max(), np.abs(got[1] - ref[1]).max())
            assert err <= 1e-5, (a, b, r, zero_lo, err)
            assert prox.dist_segment_segment(got[0], got[1], c0, c1) >= r * (1 - 1e-9)
        n += 1
    assert n > 100


def test_project_out():
    assert np.allclose(prox.project_out([0.1, 0.0], Z, Z, 0.5), [0.5, 0.0])
    assert np.allclose(prox.project_out([0.0, 0.0], Z, Z, 0.5), [0.5, 0.0])
    assert np.allclose(prox.project_out([2.0, 3.0], Z, Z, 0.5), [2.0, 3.0])
    q = prox.project_out([0.3, 0.1], [0.0, 0.0], [1.0, 0.0], 0.25)
    assert np.allclose(q, [0.3, 0.25])
    q = prox.project_out([0.3, 0.0], [0.0, 0.0], [1.0, 0.0], 0.25)  # on the axis
    assert np.allclose(q, [0.3, 0.25])


def _circle4(**kw):
    return twa.Problem.from_instance(workloads.circle4(), **kw)


@pytest.fixture(scope="module")
def energy_solution():
    prob = _circle4()
    st, it, res = twa.solve(prob, 1e-6, 20000)
    assert res < 1e-6
    return prob, st, it


def _seg_lengths(z):
    return np.linalg.norm(z[:, 1:] - z[:, :-1], axis=-1)


def test_feasibility_mode_finds_a_collision_free_plan_fast(energy_solution):
    """Without the kinetic factors (Eq. basic_opt_prob alone) the circle
    swap converges in a small fraction of the energy problem's iterations
    (Section 4 compares the two) to a collision-free plan, and break-points
    with only zero incoming weights occur on the way."""
    _, _, it_energy = energy_solution
    prob = _circle4(energy=False)
    st = twa.initial_state(prob)
    saw_zero = False
    for it in range(1, 2001):
        st, info = twa.iterate(prob, st)
        saw_zero |= bool((st.wback[:, 1:-1] == twa.W0).any())
        if info.residual < 1e-9:
            break
    assert info.residual < 1e-9 and saw_zero
    assert it < it_energy / 10
    coll, _ = twa.min_clearance(prob, st.z)
    assert coll >= 1.0 - 1e-9
    assert np.array_equal(st.z[:, 0], prob.start) and np.array_equal(st.z[:, -1], prob.goal)


def test_loose_velocity_limits_change_nothing(energy_solution):
    prob0, st0, it0 = energy_solution
    L = _seg_lengths(st0.z)
    # every segment of every iterate stays below 10x the longest converged one
    # (the first iterate's jump to the goal included); a zero minimum never binds
    prob = _circle4(vmax=np.full((4, 4), 10 * L.max()), vmin=np.zeros((4, 4)))
    st, it, res = twa.solve(prob, 1e-6, 20000)
    assert it == it0 and np.array_equal(st.z, st0.z)


def test_max_velocity_limit_holds_at_convergence(energy_solution):
    prob0, st0, _ = energy_solution
    L = _seg_lengths(st0.z)
    vmax = np.full((4, 4), 0.9 * L.max())
    prob = _circle4(vmax=vmax)
    st, it, res = twa.solve(prob, 1e-6, 20000)
    assert res < 1e-6
    assert np.all(_seg_lengths(st.z) <= vmax * (1 + 1e-4))
    assert twa.min_clearance(prob, st.z)[0] >= 1 - 1e-4
    # (the cost may land below the unconstrained run's: both are local optima
    # of a nonconvex problem)


def test_min_velocity_limit_holds_at_convergence(energy_solution):
    prob0, st0, _ = energy_solution
    L = _seg_lengths(st0.z)
    vmin = np.full((4, 4), 1.1 * L.min())
    prob = _circle4(vmin=vmin)
    st, it, res = twa.solve(prob, 1e-6, 20000)
    assert res < 1e-6
    assert np.all(_seg_lengths(st.z) >= vmin * (1 - 1e-4))
    assert twa.min_clearance(prob, st.z)[0] >= 1 - 1e-4


def test_max_velocity_feasibility_without_energy():
    vmax = np.full((4, 4), 0.6)
    prob = _circle4(vmax=vmax, energy=False)
    st, it, res = twa.solve(prob, 1e-9, 5000)
    assert res < 1e-9
    assert np.all(_seg_lengths(st.z) <= vmax * (1 + 1e-9))
    assert twa.min_clearance(prob, st.z)[0] >= 1 - 1e-9
