"""Trajectory losses for the differentiable planner (plain PyTorch ops on
the break-points z, shape (p, eta+1, 2); autograd gives dL/dz, which
``Planner.backward`` / ``unrolled_trajectory`` carry back to the inputs).

The paper has no loss of its own: these are the quantities it reports on a
plan, the kinetic energy of Section 1 and the collision clearance, written
as functions of z.
"""
from __future__ import annotations


def kinetic_energy(z, cost_w):
    """sum over agents and segments of C_{i,s} |z_{i,s+1} - z_{i,s}|^2
    (the objective of Section 1 with the planner's default normalisation
    1 / (p eta)); cost_w is (p,) or (p, eta)."""
    import torch
    p, E1, _ = z.shape
    eta = E1 - 1
    d = z[:, 1:] - z[:, :-1]
    c = cost_w if cost_w.dim() == 2 else cost_w[:, None].expand(p, eta)
    return (c * (d * d).sum(-1)).sum() / (p * eta)


def collision_slack(z, radius, chunk: int = 1 << 16):
    """sum over pairs i < j and segments s of [R_ij - d_ij,s]_+^2, d the
    closest distance of the two agents while both move linearly along
    segment s (the relative position sweeps the segment from
    z_j,s - z_i,s to z_j,s+1 - z_i,s+1), R_ij = r_i + r_j."""
    import torch
    p = z.shape[0]
    iu, ju = torch.triu_indices(p, p, 1, device=z.device)
    total = z.new_zeros(())
    for a in range(0, iu.numel(), chunk):
        i, j = iu[a:a + chunk], ju[a:a + chunk]
        c0 = z[j, :-1] - z[i, :-1]
        c1 = z[j, 1:] - z[i, 1:]
        d = c1 - c0
        dd = (d * d).sum(-1)
        t = (-(c0 * d).sum(-1) / dd.clamp_min(1e-30)).clamp(0.0, 1.0)
        q = c0 + t[..., None] * d
        dist = torch.sqrt((q * q).sum(-1) + 1e-30)
        R = (radius[i] + radius[j])[:, None]
        total = total + (torch.relu(R - dist) ** 2).sum()
    return total


def plan_loss(z, radius, cost_w, weight: float = 10.0):
    """Final kinetic energy + weight x the squared collision slack."""
    return kinetic_energy(z, cost_w) + weight * collision_slack(z, radius)


def _point_segment(q, a, b):
    """Distance from points q to segments [a, b] (broadcasting, last dim 2)."""
    import torch
    d = b - a
    dd = (d * d).sum(-1)
    t = (((q - a) * d).sum(-1) / dd.clamp_min(1e-30)).clamp(0.0, 1.0)
    c = a + t[..., None] * d
    return torch.sqrt(((q - c) ** 2).sum(-1))


def _cross(u, v):
    return u[..., 0] * v[..., 1] - u[..., 1] * v[..., 0]


def min_clearance(z, radius, walls=None, chunk: int = 1 << 16):
    """Smallest distance / (r_i + r_j) over agent pairs and segments (agents
    moving linearly between break-points), and smallest distance / r_i over
    agents, segments and wall segments (walls: (n, 4) rows xL, xR); 1 means
    touching.  Returns two floats (inf when there is nothing to measure)."""
    import torch
    p = z.shape[0]
    zero = z.new_zeros(2)
    worst = float("inf")
    iu, ju = torch.triu_indices(p, p, 1, device=z.device)
    for a in range(0, iu.numel(), chunk):
        i, j = iu[a:a + chunk], ju[a:a + chunk]
        d = _point_segment(zero, z[j, :-1] - z[i, :-1], z[j, 1:] - z[i, 1:])
        worst = min(worst, float((d / (radius[i] + radius[j])[:, None]).min()))
    wworst = float("inf")
    if walls is not None and len(walls):
        w = torch.as_tensor(walls, dtype=z.dtype, device=z.device).reshape(-1, 4)
        a0, a1 = z[:, None, :-1], z[:, None, 1:]                    # (p, 1, eta, 2)
        b0, b1 = w[None, :, None, :2], w[None, :, None, 2:]         # (1, nw, 1, 2)
        d = torch.minimum(torch.minimum(_point_segment(a0, b0, b1), _point_segment(a1, b0, b1)),
                          torch.minimum(_point_segment(b0, a0, a1), _point_segment(b1, a0, a1)))
        d1, d2 = _cross(a1 - a0, b0 - a0), _cross(a1 - a0, b1 - a0)
        d3, d4 = _cross(b1 - b0, a0 - b0), _cross(b1 - b0, a1 - b0)
        crossing = (d1 * d2 < 0) & (d3 * d4 < 0)
        d = torch.where(crossing, torch.zeros_like(d), d)
        wworst = float((d / radius[:, None, None]).min())
    return worst, wworst
