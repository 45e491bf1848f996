"""Pins of the oracle's reference adjoint of K unrolled TWA iterations
(Appendix B from the initial state of Section 4), CPU only.

The adjoint is checked against things it does not compute itself: central
differences of the whole K-iteration map (with every factor's activity and
minimizer branch checked to be identical on both sides of the step), the exact
affine map of a single agent, and the identities that follow from the
method's symmetries (translation equivariance and positive homogeneity of
degree one in positions and radii)."""
import numpy as np
import pytest

import workloads
from oracle import adjoint, twa

K = 200
EPS = 1e-6
SEEDS = {"start": 11, "goal": 12, "radius": 33, "cost": 14}


def _acts(prob, k):
    return adjoint.branches(prob, k)


def _shift(prob, sign, d):
    pr = twa.Problem(p=prob.p, eta=prob.eta, start=prob.start + sign * EPS * d["start"],
                     goal=prob.goal + sign * EPS * d["goal"],
                     radius=prob.radius + sign * EPS * d["radius"],
                     cost=prob.cost + sign * EPS * d["cost"], walls=prob.walls,
                     rho0=prob.rho0, alpha=prob.alpha, cost_unnorm=prob.cost_unnorm)
    return pr


@pytest.fixture(scope="module")
def circle():
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    rng = np.random.default_rng(2024)
    W = rng.standard_normal((prob.p, prob.eta + 1, 2))
    grads = adjoint.backward(prob, K, W)
    return prob, W, grads, _acts(prob, K)


@pytest.mark.parametrize("group", ["start", "goal", "radius", "cost"])
def test_adjoint_matches_central_differences_of_the_unrolled_map(circle, group):
    """<dL/dtheta, d> against (L(theta + eps d) - L(theta - eps d)) / 2 eps
    for L = <W, z^K>, one parameter group at a time, K = 200 on the p = 4
    circle swap: collision factors switch off and on again along the way,
    and a free segment takes both the both-ends-moved and the one-end-moved
    minimizer branches.
    Both perturbed runs take every branch the same way as the base run."""
    prob, W, (gs, gg, gr, gc), A0 = circle
    act = A0 > 0
    assert (A0[:, 2] == 4).any() and (A0[:, 2] == 2).any() and (act[1:] & ~act[:-1]).any()
    rng = np.random.default_rng(SEEDS[group])
    d = {k: np.zeros_like(getattr(prob, k)) for k in ("start", "goal", "radius", "cost")}
    d[group] = rng.standard_normal(d[group].shape)
    pp, pm = _shift(prob, 1, d), _shift(prob, -1, d)
    assert np.array_equal(_acts(pp, K), A0) and np.array_equal(_acts(pm, K), A0)
    fd = ((W * adjoint.zK(pp, K)).sum() - (W * adjoint.zK(pm, K)).sum()) / (2 * EPS)
    g = {"start": gs, "goal": gg, "radius": gr, "cost": gc}[group]
    an = float((g * d[group]).sum())
    assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-3), (group, an, fd)


def test_translation_equivariance_identity(circle):
    """Moving every start and goal by t moves z^K by t, so the position
    gradients of L = <W, z^K> sum to the sum of W."""
    prob, W, (gs, gg, gr, gc), _ = circle
    lhs = gs.sum(axis=0) + gg.sum(axis=0)
    assert np.allclose(lhs, W.reshape(-1, 2).sum(axis=0), rtol=1e-7, atol=1e-7)


def test_homogeneity_identity(circle):
    """z^K is positively homogeneous of degree one in (start, goal, radii):
    scaling all three by s scales z^K by s (the minimizers are homogeneous
    and the updates linear).  Euler's identity then gives
    sum g_start . start + g_goal . goal + g_r . r = <W, z^K>."""
    prob, W, (gs, gg, gr, gc), _ = circle
    lhs = (gs * prob.start).sum() + (gg * prob.goal).sum() + (gr * prob.radius).sum()
    rhs = (W * adjoint.zK(prob, K)).sum()
    assert abs(lhs - rhs) <= 1e-7 * max(1.0, abs(rhs))


def test_single_agent_map_is_affine_and_the_adjoint_is_its_transpose():
    """One agent: only kinetic factors, so z^K is affine in (start, goal);
    its exact Jacobian is read column by column from unit steps of size 1."""
    rng = np.random.default_rng(5)
    prob = twa.Problem(p=1, eta=5, start=np.array([[0.3, -0.2]]), goal=np.array([[2.0, 1.5]]),
                       radius=np.array([0.2]), cost=rng.uniform(0.5, 2.0, (1, 5)),
                       walls=np.zeros((0, 4)), rho0=1.0, alpha=0.1)
    k = 30
    W = rng.standard_normal((1, 6, 2))
    gs, gg, gr, gc = adjoint.backward(prob, k, W)
    base = (W * adjoint.zK(prob, k)).sum()
    for which, g in (("start", gs), ("goal", gg)):
        for c in range(2):
            pr = twa.Problem(**{**prob.__dict__})
            arr = getattr(prob, which).copy()
            arr[0, c] += 1.0
            setattr(pr, which, arr)
            col = (W * adjoint.zK(pr, k)).sum() - base
            assert abs(col - g[0, c]) <= 1e-9 * max(1.0, abs(col)), (which, c, col, g[0, c])
    assert np.all(gr == 0.0)


def test_zero_weight_loss_gives_zero_gradient(circle):
    prob = circle[0]
    gs, gg, gr, gc = adjoint.backward(prob, 20, np.zeros((prob.p, prob.eta + 1, 2)))
    for g in (gs, gg, gr, gc):
        assert np.all(g == 0.0)


def _pinned_case():
    """Three agents crossing near their starts: collision factors on the first
    segment (lower end fixed) and the last (upper end fixed) are active."""
    return twa.Problem(p=3, eta=3, start=np.array([[0.0, 0.0], [0.45, 0.05], [0.2, 0.5]]),
                       goal=np.array([[1.0, 0.1], [-0.6, 0.0], [0.2, -0.6]]),
                       radius=np.array([0.2, 0.2, 0.15]), cost=np.ones((3, 3)),
                       walls=np.zeros((0, 4)), rho0=1.0, alpha=0.1)


@pytest.mark.parametrize("seed", [1, 3])
def test_adjoint_with_fixed_end_collision_branches(seed):
    """The fixed-end minimizers (one weight infinite) in the gradient: every
    parameter group perturbed at once, K = 120, no branch flips."""
    prob = _pinned_case()
    k = 120
    A0 = _acts(prob, k)
    assert (A0[:, 0] == 3).any() and (A0[:, -1] == 2).any()
    W = np.random.default_rng(7).standard_normal((3, 4, 2))
    g = adjoint.backward(prob, k, W)
    r = np.random.default_rng(seed)
    d = {n: r.standard_normal(getattr(prob, n).shape) for n in ("start", "goal", "radius", "cost")}
    pp, pm = _shift(prob, 1, d), _shift(prob, -1, d)
    assert np.array_equal(_acts(pp, k), A0) and np.array_equal(_acts(pm, k), A0)
    fd = ((W * adjoint.zK(pp, k)).sum() - (W * adjoint.zK(pm, k)).sum()) / (2 * EPS)
    an = sum(float((gi * d[n]).sum()) for gi, n in zip(g, ("start", "goal", "radius", "cost")))
    assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-3), (an, fd)


def _corridor():
    """Two agents swapping along a corridor too narrow to pass without the
    walls' factors becoming active."""
    return twa.Problem(p=2, eta=4, start=np.array([[-1.2, 0.05], [1.2, -0.05]]),
                       goal=np.array([[1.2, -0.02], [-1.2, 0.02]]), radius=np.array([0.2, 0.2]),
                       cost=np.ones((2, 4)),
                       walls=np.array([[-3.0, 0.36, 3.0, 0.36], [3.0, -0.36, -3.0, -0.36]]),
                       rho0=1.0, alpha=0.1)


def _velocity_limited():
    return twa.Problem.from_instance(workloads.circle4(), vmax=np.full((4, 4), 0.56),
                                     vmin=np.full((4, 4), 0.3))


@pytest.mark.parametrize("case", ["walls", "velocity"])
def test_adjoint_through_gated_segment_factors(case):
    """Wall factors (a corridor swap) and maximum / minimum velocity factors
    in the gradient: every parameter group perturbed at once, K = 150, no
    branch flips (collision and segment-factor branch tapes equal)."""
    prob = _corridor() if case == "walls" else _velocity_limited()
    k = 150
    sb = adjoint.seg_branches(prob, k)
    assert sum(len(x) for x in sb) > 100
    A0 = _acts(prob, k)
    W = np.random.default_rng(7).standard_normal((prob.p, prob.eta + 1, 2))
    g = adjoint.backward(prob, k, W)
    for seed in (1, 2):
        r = np.random.default_rng(seed)
        d = {n: r.standard_normal(getattr(prob, n).shape) for n in ("start", "goal", "radius", "cost")}
        runs = []
        for sign in (1, -1):
            pr = _shift(prob, sign, d)
            pr.walls, pr.vmax, pr.vmin = prob.walls, prob.vmax, prob.vmin
            assert np.array_equal(_acts(pr, k), A0) and adjoint.seg_branches(pr, k) == sb
            runs.append((W * adjoint.zK(pr, k)).sum())
        fd = (runs[0] - runs[1]) / (2 * EPS)
        an = sum(float((gi * d[n]).sum()) for gi, n in zip(g, ("start", "goal", "radius", "cost")))
        assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-3), (seed, an, fd)


def test_adjoint_of_a_local_planner_epoch():
    """The velocity-obstacle epoch (Section 5): gradient of its solution
    after K = 150 iterations with respect to the current positions x(0)
    (start), the reference positions (goal), radii and the C'_i, against
    central differences, no branch flips."""
    from oracle import vo
    x0 = np.array([[-0.5, 0.01], [0.5, -0.01], [0.05, 0.6]])
    dest = np.array([[2.0, 0.0], [-2.0, 0.0], [0.0, -2.0]])
    prob = vo.problem(x0, vo.targets(x0, dest, 0.8), np.array([0.2, 0.2, 0.15]),
                      np.array([1.0, 1.001, 1.002]), rho0=10.0)
    k = 150
    A0 = _acts(prob, k)
    assert A0.any() and not A0[:, 1].any()
    W = np.random.default_rng(3).standard_normal((3, 3, 2))
    g = adjoint.backward(prob, k, W)
    assert np.all(g[3][:, 0] == 0.0)  # no kinetic factor on the epoch's own motion
    r = np.random.default_rng(1)
    d = {n: r.standard_normal(getattr(prob, n).shape) for n in ("start", "goal", "radius", "cost")}
    d["cost"][:, 0] = 0.0
    runs = []
    for sign in (1, -1):
        pr = _shift(prob, sign, d)
        pr.vo, pr.cost_unnorm = True, True
        assert np.array_equal(_acts(pr, k), A0)
        runs.append((W * adjoint.zK(pr, k)).sum())
    fd = (runs[0] - runs[1]) / (2 * EPS)
    an = sum(float((gi * d[n]).sum()) for gi, n in zip(g, ("start", "goal", "radius", "cost")))
    assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-3), (an, fd)
