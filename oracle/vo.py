"""The local planner of Section 5 on the FP64 oracle (test infrastructure
only): velocity-obstacle collision avoidance solved one epoch at a time by
the TWA.

One epoch (Eq. rec_col_avoi_pos): from the current positions x_i(0), choose
the positions x_i reached after the epoch's horizon tau, minimising
sum_i C'_i |x_i - x_ref_i|^2 with x_ref_i = x_i(0) + v_ref_i tau, such that
agents moving linearly from x_i(0) to x_i do not collide.  The factor graph
is the oracle's ``vo`` problem (eta = 2; see ``oracle.twa``).

Between epochs (Section 5): the agents follow the planned velocity
(x_i - x_i(0)) / tau for a fraction ``advance`` of the horizon and re-plan.
The preferred velocity points at the agent's destination with length at
most ``step`` / tau (so x_ref_i = x_i(0) + the destination offset clipped to
length ``step``).  The paper breaks CONF1's symmetry with C_i = 1 + 0.001 i.
"""
from __future__ import annotations

import numpy as np

from . import twa


def targets(x0, dest, step):
    """x_ref_i = x_i(0) + (dest_i - x_i(0)) clipped to length step."""
    d = dest - x0
    L = np.linalg.norm(d, axis=1, keepdims=True)
    scale = np.where(L > step, step / np.maximum(L, 1e-300), 1.0)
    return x0 + scale * d


def problem(x0, x_ref, radius, c_prime, walls=None, rho0=1.0, alpha=0.1) -> twa.Problem:
    p = x0.shape[0]
    cost = np.zeros((p, 2))
    cost[:, 1] = c_prime
    return twa.Problem(p=p, eta=2, start=np.asarray(x0, dtype=np.float64),
                       goal=np.asarray(x_ref, dtype=np.float64),
                       radius=np.asarray(radius, dtype=np.float64), cost=cost,
                       walls=np.zeros((0, 4)) if walls is None else np.asarray(walls, dtype=np.float64),
                       rho0=rho0, alpha=alpha, cost_unnorm=True, vo=True)


def epoch(x0, dest, radius, c_prime, step, tol, max_iter, walls=None, rho0=1.0, alpha=0.1):
    """Solve one epoch.  Returns (x, iterations, residual, problem)."""
    prob = problem(x0, targets(x0, dest, step), radius, c_prime, walls, rho0, alpha)
    st, it, res = twa.solve(prob, tol, max_iter)
    return st.z[:, 1].copy(), it, res, prob


def simulate(x0, dest, radius, c_prime, step, advance, epochs, tol, max_iter, walls=None,
             rho0=1.0, alpha=0.1):
    """Epoch loop.  Returns the positions after each epoch (epochs + 1, p, 2)
    and the iterations of each epoch's solve."""
    xs = [np.asarray(x0, dtype=np.float64).copy()]
    its = []
    x = xs[0]
    for _ in range(epochs):
        x1, it, res, _ = epoch(x, dest, radius, c_prime, step, tol, max_iter, walls, rho0, alpha)
        x = x + advance * (x1 - x)
        xs.append(x.copy())
        its.append(it)
    return np.stack(xs), its
