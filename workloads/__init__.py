"""Seeded synthetic planning instances.

This module only draws inputs: agent radii, start and goal positions, cost
weights, walls and the solver parameters that go with each workload.  It holds
none of the planner's arithmetic, so both the FP64 oracle and the CUDA path may
take their inputs from here.

The workloads follow the paper's two scenario families (Section 4):

* CONF1, "circle swap": agents evenly spaced on a circle, each one travelling
  to the antipodal point.
* CONF2, "random square": starts and goals drawn uniformly in a square, with
  rejection so that neither configuration overlaps.

Every instance uses ``numpy.random.default_rng(seed)`` and a fixed draw order,
so the same name always gives the same arrays.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SEED_BASE = 13114527


@dataclass
class Instance:
    """One planning problem (the inputs of ``plan_create``).

    Arrays are float64 here; each consumer casts to its own precision.
    """

    name: str
    p: int                       # agents
    eta: int                     # segments; break-points s = 0..eta
    T: float                     # horizon (timestamps only; not in the cost)
    start: np.ndarray            # (p, 2)
    goal: np.ndarray             # (p, 2)
    radius: np.ndarray           # (p,)
    cost_w: np.ndarray           # (p,) C_i of the kinetic-energy cost
    walls: np.ndarray            # (n_walls, 4) rows [xL.x, xL.y, xR.x, xR.y]
    rho0: float
    alpha: float
    tol: float
    max_iter: int
    recipe: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_walls(self) -> int:
        return int(self.walls.shape[0])


def _circle_positions(p: int, radius: float) -> np.ndarray:
    ang = 2.0 * math.pi * np.arange(p) / p
    return radius * np.stack([np.cos(ang), np.sin(ang)], axis=1)


def _circle_radius_for(radius: np.ndarray) -> float:
    """Circle radius that keeps neighbouring agents apart.

    The paper's CONF1 radius formula is ambiguous (singular at p=4), so the
    circle is sized from the radii instead: 1.25 x the tightest neighbour
    requirement, and never below 1.
    """
    p = radius.shape[0]
    if p < 2:
        return 1.0
    need = float(np.max(radius + np.roll(radius, -1)))
    return max(1.0, 1.25 * need / (2.0 * math.sin(math.pi / p)))


def circle_swap(p: int, eta: int, radius, jitter: float, seed: int, *,
                rho0: float = 1.0, alpha: float = 0.1, tol: float = 1e-6,
                max_iter: int = 20000, radius_range=None, name=None) -> Instance:
    """CONF1: agents on a circle swap with their antipodes (Section 4).

    Draw order: radii (only when ``radius_range`` is given), then the start
    jitter.  Each goal is the antipode of the agent's nominal (unjittered)
    circle point.  Negating the jittered start instead would make every pair's
    relative motion pass exactly through the origin at the first iteration, an
    exact tie of the collision minimizer.
    """
    rng = np.random.default_rng(seed)
    if radius_range is not None:
        r = rng.uniform(radius_range[0], radius_range[1], size=p)
    else:
        r = np.full(p, float(radius))
    rc = _circle_radius_for(r)
    nominal = _circle_positions(p, rc)
    start = nominal + rng.uniform(-jitter, jitter, size=(p, 2))
    goal = -nominal
    return Instance(
        name=name or f"circle{p}_eta{eta}", p=p, eta=eta, T=1.0, start=start, goal=goal,
        radius=r, cost_w=np.ones(p), walls=np.zeros((0, 4)), rho0=rho0, alpha=alpha,
        tol=tol, max_iter=max_iter,
        recipe=(f"circle swap: p={p} on a circle of radius {rc:.6g}, jitter U(+-{jitter}) per "
                f"coordinate, goals = antipodes of the nominal circle points, eta={eta}, seed={seed}"),
        extra={"circle_radius": rc})


def _rejection_positions(rng, r: np.ndarray, side: float, max_tries: int = 100000) -> np.ndarray:
    """Sequentially place disks of radius r_i uniformly in [r_i, side-r_i]^2 so
    that no two overlap (touching allowed)."""
    p = r.shape[0]
    pos = np.zeros((p, 2))
    for i in range(p):
        for _ in range(max_tries):
            cand = rng.uniform(r[i], side - r[i], size=2)
            if i == 0:
                break
            d = np.hypot(pos[:i, 0] - cand[0], pos[:i, 1] - cand[1])
            if np.all(d >= r[:i] + r[i]):
                break
        else:
            raise RuntimeError("rejection sampling did not place every agent")
        pos[i] = cand
    return pos


def random_square(p: int, eta: int, side: float, r_lo: float, r_hi: float, seed: int, *,
                  walls: bool = True, rho0: float = 1.0, alpha: float = 0.1,
                  tol: float | None = None, max_iter: int = 20000, name=None) -> Instance:
    """CONF2: random starts and goals in a square (Section 4), with the four
    sides of the square as wall factors.

    Draw order: radii, then starts (sequential rejection), then goals.
    """
    rng = np.random.default_rng(seed)
    r = rng.uniform(r_lo, r_hi, size=p)
    start = _rejection_positions(rng, r, side)
    goal = _rejection_positions(rng, r, side)
    w = np.zeros((0, 4))
    if walls:
        L = float(side)
        w = np.array([[0, 0, L, 0], [L, 0, L, L], [L, L, 0, L], [0, L, 0, 0]], dtype=np.float64)
    if tol is None:
        tol = 1e-6 * max(1.0, side)
    return Instance(
        name=name or f"square{p}_eta{eta}", p=p, eta=eta, T=1.0, start=start, goal=goal,
        radius=r, cost_w=np.ones(p), walls=w, rho0=rho0, alpha=alpha, tol=tol,
        max_iter=max_iter,
        recipe=(f"random square: p={p}, side {side}, radii U[{r_lo},{r_hi}], starts and goals "
                f"rejection-sampled in [r_i, side-r_i]^2 without overlap, "
                f"{w.shape[0]} walls, eta={eta}, seed={seed}"))


def _clear_of_walls(pos: np.ndarray, r: float, walls: np.ndarray) -> bool:
    """pos at distance >= r from every axis-aligned wall segment."""
    for x0, y0, x1, y1 in walls:
        cx = min(max(pos[0], min(x0, x1)), max(x0, x1))
        cy = min(max(pos[1], min(y0, y1)), max(y0, y1))
        if math.hypot(pos[0] - cx, pos[1] - cy) < r:
            return False
    return True


def obstacle_square(p: int, eta: int, side: float, n_obstacles: int, seed: int, *,
                    r_lo: float = 0.2, r_hi: float = 0.4, rho0: float = 1.0,
                    alpha: float = 0.1, max_iter: int = 20000, name=None) -> Instance:
    """CONF2 with static obstacles: the random square's four sides plus
    n_obstacles interior wall segments (Section 3.2), each axis-aligned,
    horizontal or vertical with equal odds, of length U[side/8, side/4],
    centred uniformly in the middle 80% of the square.  Starts and goals are
    rejection-sampled without overlap and at least r_i from every wall.

    Draw order: radii, walls, then starts, then goals (each position drawn
    until it clears the walls and the disks placed before it).
    """
    rng = np.random.default_rng(seed)
    r = rng.uniform(r_lo, r_hi, size=p)
    L = float(side)
    walls = [[0, 0, L, 0], [L, 0, L, L], [L, L, 0, L], [0, L, 0, 0]]
    for _ in range(n_obstacles):
        half = 0.5 * rng.uniform(L / 8, L / 4)
        cx, cy = rng.uniform(0.1 * L, 0.9 * L, size=2)
        if rng.uniform() < 0.5:
            walls.append([cx - half, cy, cx + half, cy])
        else:
            walls.append([cx, cy - half, cx, cy + half])
    w = np.asarray(walls, dtype=np.float64)

    def place():
        pos = np.zeros((p, 2))
        for i in range(p):
            for _ in range(100000):
                cand = rng.uniform(r[i], L - r[i], size=2)
                if not _clear_of_walls(cand, r[i], w[4:]):
                    continue
                d = np.hypot(pos[:i, 0] - cand[0], pos[:i, 1] - cand[1])
                if np.all(d >= r[:i] + r[i]):
                    break
            else:
                raise RuntimeError("rejection sampling did not place every agent")
            pos[i] = cand
        return pos

    start = place()
    goal = place()
    return Instance(
        name=name or f"obstacles{p}_eta{eta}_s{seed}", p=p, eta=eta, T=1.0, start=start,
        goal=goal, radius=r, cost_w=np.ones(p), walls=w, rho0=rho0, alpha=alpha,
        tol=1e-6 * max(1.0, L), max_iter=max_iter,
        recipe=(f"random square with obstacles: p={p}, side {side}, radii U[{r_lo},{r_hi}], "
                f"4 sides + {n_obstacles} axis-aligned interior walls of length U[side/8, side/4], "
                f"starts and goals clear of walls and of each other, eta={eta}, seed={seed}"))


# --- the named workloads -----------------------------------------------------

def circle4() -> Instance:
    """p=4 circle swap, r=0.15, jitter +-0.01, eta=4, rho=1 (CPU-sized)."""
    return circle_swap(4, 4, 0.15, 0.01, SEED_BASE + 0, rho0=1.0, name="circle4_eta4")


def circle100() -> Instance:
    """p=100 circle swap, radii U[0.02,0.05], jitter +-0.005, eta=8, rho=2."""
    return circle_swap(100, 8, None, 0.005, SEED_BASE + 1, rho0=2.0,
                       radius_range=(0.02, 0.05), name="circle100_eta8")


def square1024() -> Instance:
    """p=1024 random square [0,40]^2, radii U[0.2,0.4], eta=16, 4 walls."""
    return random_square(1024, 16, 40.0, 0.2, 0.4, SEED_BASE + 2, rho0=1.0,
                         name="square1024_eta16")


def circle256() -> Instance:
    """p=256 circle swap, r=0.02, eta=8 (the unrolled-gradient workload)."""
    return circle_swap(256, 8, 0.02, 0.005, SEED_BASE + 4, rho0=1.0, name="circle256_eta8")


NAMED = {
    "circle4_eta4": circle4,
    "circle100_eta8": circle100,
    "square1024_eta16": square1024,
    "circle256_eta8": circle256,
}


def by_name(name: str) -> Instance:
    return NAMED[name]()


def small_square(p: int, eta: int, seed: int, side: float | None = None, walls: bool = True,
                 rho0: float = 1.0) -> Instance:
    """A reduced random square with the same area coverage as the p=1024 one
    (about 18% of the square covered by agent disks); used for parity cases
    that must finish quickly on the CPU."""
    if side is None:
        side = 40.0 * math.sqrt(p / 1024.0)
    return random_square(p, eta, side, 0.2, 0.4, seed, walls=walls, rho0=rho0,
                         name=f"square{p}_eta{eta}_s{seed}")


def batch_instances(n: int = 512, seed: int = SEED_BASE + 3):
    """Uneven instances for the batched form: p ~ U{8..256}, eta in {4,8,16},
    circle swap or random square 50/50, radii U[0.02,0.05] (square side chosen
    for ~18% coverage)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n):
        p = int(rng.integers(8, 257))
        eta = int(rng.choice([4, 8, 16]))
        sub = int(rng.integers(0, 2**31 - 1))
        if rng.uniform() < 0.5:
            inst = circle_swap(p, eta, None, 0.005, sub, radius_range=(0.02, 0.05),
                               name=f"batch{b}_circle{p}_eta{eta}")
        else:
            er2 = (0.02**2 + 0.02 * 0.05 + 0.05**2) / 3.0
            side = math.sqrt(p * math.pi * er2 / 0.18)
            inst = random_square(p, eta, side, 0.02, 0.05, sub, walls=False,
                                 name=f"batch{b}_square{p}_eta{eta}")
        out.append(inst)
    return out
