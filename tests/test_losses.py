"""The torch trajectory losses of the differentiable planner against the
oracle's cost and clearance measures, CPU only."""
import numpy as np
import torch

import workloads
from oracle import prox, twa
from paper_1311_4527_gb300 import losses


def test_kinetic_energy_is_the_oracle_total_cost():
    inst = workloads.small_square(20, 5, seed=4)
    prob = twa.Problem.from_instance(inst)
    z = np.random.default_rng(1).normal(size=(20, 6, 2))
    got = losses.kinetic_energy(torch.tensor(z), torch.tensor(prob.cost))
    assert abs(float(got) - twa.total_cost(prob, z)) <= 1e-12 * max(1.0, abs(float(got)))
    got1 = losses.kinetic_energy(torch.tensor(z), torch.tensor(prob.cost[:, 0]))
    assert abs(float(got1) - float(got)) <= 1e-12 * abs(float(got))


def test_collision_slack_by_brute_force():
    rng = np.random.default_rng(2)
    p, eta = 7, 3
    z = rng.uniform(0, 1.5, size=(p, eta + 1, 2))
    r = rng.uniform(0.1, 0.3, size=p)
    want = 0.0
    for i in range(p):
        for j in range(i + 1, p):
            for s in range(eta):
                d = prox.dist_point_segment(np.zeros(2), z[j, s] - z[i, s], z[j, s + 1] - z[i, s + 1])
                want += max(r[i] + r[j] - float(d), 0.0) ** 2
    got = float(losses.collision_slack(torch.tensor(z), torch.tensor(r), chunk=5))
    assert want > 0 and abs(got - want) <= 1e-9 * want


def test_min_clearance_matches_the_oracle():
    inst = workloads.small_square(30, 4, seed=8)
    prob = twa.Problem.from_instance(inst)
    rng = np.random.default_rng(3)
    z = rng.uniform(0, inst.walls.max(), size=(30, 5, 2))
    z[:, 0] = inst.start
    want = twa.min_clearance(prob, z)
    got = losses.min_clearance(torch.tensor(z), torch.tensor(inst.radius), inst.walls)
    assert abs(got[0] - want[0]) <= 1e-9 * max(1.0, want[0]) and abs(got[1] - want[1]) <= 1e-9 * max(1.0, want[1])
