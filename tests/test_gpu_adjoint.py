"""GPU adjoint (plan_unroll / plan_backward / unrolled_trajectory) against the
FP64 oracle adjoint on small instances, and against the identities that hold
at any size on the p = 256 circle swap with K = 2000 unrolled iterations.

Error bound of the FP32 adjoint: every entry of each gradient group within
2e-4 of that group's largest magnitude (measured: 3e-5 on the p = 4 circle,
3e-7 on the fixed-end case; the FP32 forward drifts from the FP64
one by ~1e-6 relative per iteration, and the minimizer Jacobians are
evaluated in FP32 at that drifted point)."""
import numpy as np
import pytest

import workloads
from oracle import adjoint, twa

pytestmark = pytest.mark.gpu
GROUPS = ("start", "goal", "radius", "cost")
TOL = 2e-4


def _planner(prob, **kw):
    import paper_1311_4527_gb300 as pk
    return pk.Planner(prob.start, prob.goal, prob.radius, prob.eta, cost_w=prob.cost,
                      walls=prob.walls if prob.n_walls else None, rho0=prob.rho0,
                      alpha=prob.alpha, vmax=prob.vmax, vmin=prob.vmin, vo=prob.vo, **kw)


def _gpu_grads(pl, K, W, every=0):
    import torch
    pl.unroll(K, every)
    g = pl.backward(torch.tensor(W, dtype=torch.float32))
    return [x.cpu().numpy().astype(np.float64) for x in g]


def _activity_matches(prob, K):
    """The GPU forward takes the oracle's activity pattern in all K iterations."""
    _, tape = adjoint.record(prob, K)
    pl = _planner(prob)
    for k in range(K):
        pl.iterate(1)
        act = pl.export_state()["act_coll"].cpu().numpy().astype(bool)
        if not np.array_equal(act, tape[k][1]):
            pl.close()
            return False
    pl.close()
    return True


def _rel_err(g, ref):
    return max(float(np.abs(a - b).max()) / max(float(np.abs(b).max()), 1e-12)
               for a, b in zip(g, ref) if np.abs(b).max() > 0)


def _pinned_case():
    return twa.Problem(p=3, eta=3, start=np.array([[0.0, 0.0], [0.45, 0.05], [0.2, 0.5]]),
                       goal=np.array([[1.0, 0.1], [-0.6, 0.0], [0.2, -0.6]]),
                       radius=np.array([0.2, 0.2, 0.15]), cost=np.ones((3, 3)),
                       walls=np.zeros((0, 4)), rho0=1.0, alpha=0.1)


def _corridor():
    return twa.Problem(p=2, eta=4, start=np.array([[-1.2, 0.05], [1.2, -0.05]]),
                       goal=np.array([[1.2, -0.02], [-1.2, 0.02]]), radius=np.array([0.2, 0.2]),
                       cost=np.ones((2, 4)),
                       walls=np.array([[-3.0, 0.36, 3.0, 0.36], [3.0, -0.36, -3.0, -0.36]]),
                       rho0=1.0, alpha=0.1)


def _vo_epoch():
    from oracle import vo
    x0 = np.array([[-0.5, 0.01], [0.5, -0.01], [0.05, 0.6]])
    dest = np.array([[2.0, 0.0], [-2.0, 0.0], [0.0, -2.0]])
    return vo.problem(x0, vo.targets(x0, dest, 0.8), np.array([0.2, 0.2, 0.15]),
                      np.array([1.0, 1.001, 1.002]), rho0=10.0)


@pytest.mark.parametrize("case", ["circle4", "pinned3", "walls", "velocity", "local_planner"])
def test_adjoint_matches_the_oracle_adjoint(case):
    prob = {"circle4": lambda: twa.Problem.from_instance(workloads.circle4()),
            "pinned3": _pinned_case, "walls": _corridor,
            "velocity": lambda: twa.Problem.from_instance(
                workloads.circle4(), vmax=np.full((4, 4), 0.56), vmin=np.full((4, 4), 0.3)),
            "local_planner": _vo_epoch}[case]()
    K = {"circle4": 200, "pinned3": 120, "walls": 150, "velocity": 150, "local_planner": 150}[case]
    assert _activity_matches(prob, K)
    W = np.random.default_rng(2024).standard_normal((prob.p, prob.eta + 1, 2))
    ref = adjoint.backward(prob, K, W)
    pl = _planner(prob)
    g = _gpu_grads(pl, K, W)
    pl.close()
    for name, a, b in zip(GROUPS, g, ref):
        scale = max(float(np.abs(b).max()), 1e-6)
        assert np.abs(a - b).max() <= TOL * scale, (name, np.abs(a - b).max() / scale)


def test_checkpoint_interval_and_repeat_calls_do_not_change_the_gradient():
    prob = twa.Problem.from_instance(workloads.circle4())
    W = np.random.default_rng(3).standard_normal((prob.p, prob.eta + 1, 2))
    pl = _planner(prob)
    a = _gpu_grads(pl, 150, W, every=0)      # ceil(sqrt(150)) = 13, ragged last segment
    b = _gpu_grads(pl, 150, W, every=150)    # one segment, no recompute past iteration 0
    c = _gpu_grads(pl, 150, W, every=1)      # a checkpoint before every iteration
    import torch
    d = [x.cpu().numpy().astype(np.float64) for x in pl.backward(torch.tensor(W, dtype=torch.float32))]
    pl.close()
    for x in (b, c, d):
        assert _rel_err(x, a) <= 1e-5


def test_unroll_equals_plain_iterations_and_backward_leaves_iteration_K():
    import torch
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    pl = _planner(prob)
    pl.iterate(90)
    z90 = pl.trajectory().cpu().numpy()
    pl.unroll(90)
    assert np.array_equal(pl.trajectory().cpu().numpy(), z90)
    pl.backward(torch.zeros((prob.p, prob.eta + 1, 2)))
    assert np.array_equal(pl.trajectory().cpu().numpy(), z90)
    assert pl.info()["k"] == 90
    pl.close()


def test_zero_iterations_and_single_agent():
    W = np.random.default_rng(9).standard_normal((1, 6, 2))
    prob = twa.Problem(p=1, eta=5, start=np.array([[0.3, -0.2]]), goal=np.array([[2.0, 1.5]]),
                       radius=np.array([0.2]), cost=np.array([[1.0, 2.0, 0.5, 1.5, 1.0]]),
                       walls=np.zeros((0, 4)), rho0=1.0, alpha=0.1)
    pl = _planner(prob)
    for K in (0, 1, 30):
        g = _gpu_grads(pl, K, W)
        ref = adjoint.backward(prob, K, W)
        for name, a, b in zip(GROUPS, g, ref):
            assert np.allclose(a, b, rtol=1e-5, atol=1e-5), (K, name, a, b)
    pl.close()


def test_errors():
    import paper_1311_4527_gb300 as pk
    import torch
    prob = twa.Problem.from_instance(workloads.circle4())
    pl = _planner(prob)
    with pytest.raises(pk.PlanError) as e:
        pl.backward(torch.zeros((prob.p, prob.eta + 1, 2)))
    assert e.value.status == "PLAN_EINVAL"
    pl.unroll(5)
    pl.iterate(1)  # the state moved on: the tape no longer describes it
    with pytest.raises(pk.PlanError):
        pl.backward(torch.zeros((prob.p, prob.eta + 1, 2)))
    pl.close()
    feas = pk.Planner.from_instance(workloads.circle4(), energy=False)
    with pytest.raises(pk.PlanError) as e:
        feas.unroll(3)
    assert e.value.status == "PLAN_EUNSUPPORTED"
    feas.close()


@pytest.fixture(scope="module")
def circle256():
    """The differentiation workload: p = 256 circle swap, r = 0.02, eta = 8,
    K = 2000, loss = final kinetic energy + 10 x squared collision slack."""
    import torch
    import paper_1311_4527_gb300 as pk
    from paper_1311_4527_gb300 import losses
    inst = workloads.circle256()
    dev = torch.device("cuda")
    start = torch.tensor(inst.start, dtype=torch.float32, device=dev, requires_grad=True)
    goal = torch.tensor(inst.goal, dtype=torch.float32, device=dev, requires_grad=True)
    radius = torch.tensor(inst.radius, dtype=torch.float32, device=dev, requires_grad=True)
    cost = torch.tensor(inst.cost_w, dtype=torch.float32, device=dev, requires_grad=True)
    pl = pk.Planner.from_instance(inst)
    z = pk.unrolled_trajectory(pl, start, goal, radius, cost, 2000)
    loss = losses.plan_loss(z, radius.detach(), cost.detach())
    dz, = torch.autograd.grad(loss, z, retain_graph=True)
    loss.backward()
    out = dict(pl=pl, inst=inst, z=z.detach(), dz=dz, start=start, goal=goal, radius=radius, cost=cost)
    yield out
    pl.close()


def test_autograd_function_runs_the_adjoint(circle256):
    import torch
    d = circle256
    g = d["pl"].backward(d["dz"])
    for t, x in zip((d["start"], d["goal"], d["radius"], d["cost"]), g):
        assert t.grad is not None and torch.isfinite(t.grad).all()
        assert torch.allclose(t.grad, x, rtol=1e-5, atol=1e-6)


def test_translation_identity_at_full_size(circle256):
    """z^K(start + t, goal + t) = z^K + t, so the position gradients sum to
    the sum of dL/dz^K."""
    d = circle256
    lhs = (d["start"].grad.double().sum(0) + d["goal"].grad.double().sum(0)).cpu().numpy()
    rhs = d["dz"].double().reshape(-1, 2).sum(0).cpu().numpy()
    scale = float(d["dz"].double().abs().sum())
    assert np.abs(lhs - rhs).max() <= 1e-4 * scale, (lhs, rhs, scale)


def test_homogeneity_identity_at_full_size(circle256):
    """z^K is positively homogeneous of degree one in (start, goal, radii), so
    sum g_start . start + g_goal . goal + g_r . r = <dL/dz^K, z^K>."""
    d = circle256
    f = lambda t: t.detach().double()
    lhs = float((f(d["start"].grad) * f(d["start"])).sum() + (f(d["goal"].grad) * f(d["goal"])).sum()
                + (f(d["radius"].grad) * f(d["radius"])).sum())
    rhs = float((f(d["dz"]) * f(d["z"])).sum())
    scale = float((f(d["dz"]).abs() * f(d["z"]).abs()).sum())
    assert abs(lhs - rhs) <= 1e-3 * scale, (lhs, rhs, scale)
    assert float(d["radius"].grad.abs().sum()) > 0.0
