"""FP64 minimizers of the planning factors (test infrastructure only).

Each minimizer g_b returns the argmin of its factor function plus the weighted
squared distance to the incoming n-messages (Eq. general_minimizer_definition,
Section 2).  Weights are numbers in [0, inf]; ``math.inf`` is a pinned end.

Notation follows the paper: ``n_lo``/``n_hi`` are the messages for the two
consecutive break-points of a segment (underline / overline in the paper),
``rho_lo``/``rho_hi`` their incoming weights, ``x_*`` the outputs.

How the non-convex minimizers are solved (Appendices D and I).  The paper maps
the agent-obstacle minimizer to a springs-and-slab system and minimises a 1-D
energy over the slab direction theta.  Restated exactly: a segment
[v_lo, v_hi] stays out of the open convex region R (a disk, or the capsule of
radius r around a wall segment) iff some unit normal n(theta) separates them,
i.e. <v_lo, n> >= h(theta) and <v_hi, n> >= h(theta) where h is R's support
function.  For a fixed theta the best v's are the projections
v = a + [h - <a, n>]_+ n, so the minimizer reduces to min over theta of

    E(theta) = w_lo/2 [h - <a,n>]_+^2 + w_hi/2 [h - <b,n>]_+^2 .

Both springs stretched is the paper's tangent-slab scenario (a); one hinge at
zero is its compressed-spring scenario (b).  E is C^1 away from the capsule's
two kink directions, so its global minimum is one of: a stationary point of
the both-stretched piece (roots of a degree-4 polynomial in e^{i theta}, found
with numpy's companion-matrix root finder), a stationary point of a
single-stretched piece (theta along a - c or b - c for a circle centre c), or
a kink.  The oracle evaluates E at every candidate and keeps the lowest, with
ties (within 1e-12 relative) going to the smallest theta in [0, 2 pi).
"""
from __future__ import annotations

import math

import numpy as np

INF = math.inf
TWO_PI = 2.0 * math.pi
TIE_REL = 1e-12


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------

def dist_point_segment(q, p0, p1):
    """Euclidean distance from point q to segment [p0, p1] (arrays (..., 2))."""
    q = np.asarray(q, dtype=np.float64)
    p0 = np.asarray(p0, dtype=np.float64)
    p1 = np.asarray(p1, dtype=np.float64)
    d = p1 - p0
    dd = np.sum(d * d, axis=-1)
    t = np.where(dd > 0, np.sum((q - p0) * d, axis=-1) / np.where(dd > 0, dd, 1.0), 0.0)
    t = np.clip(t, 0.0, 1.0)
    c = p0 + t[..., None] * d
    return np.sqrt(np.sum((q - c) ** 2, axis=-1))


def _cross(u, v):
    return u[..., 0] * v[..., 1] - u[..., 1] * v[..., 0]


def dist_segment_segment(a0, a1, b0, b1):
    """Euclidean distance between segments [a0, a1] and [b0, b1] in the plane."""
    a0, a1, b0, b1 = (np.asarray(v, dtype=np.float64) for v in (a0, a1, b0, b1))
    d1 = _cross(a1 - a0, b0 - a0)
    d2 = _cross(a1 - a0, b1 - a0)
    d3 = _cross(b1 - b0, a0 - b0)
    d4 = _cross(b1 - b0, a1 - b0)
    crossing = (d1 * d2 < 0) & (d3 * d4 < 0)
    m = np.minimum(np.minimum(dist_point_segment(a0, b0, b1), dist_point_segment(a1, b0, b1)),
                   np.minimum(dist_point_segment(b0, a0, a1), dist_point_segment(b1, a0, a1)))
    return np.where(crossing, 0.0, m)


def segments_collide(n_lo_i, n_hi_i, n_lo_j, n_hi_j, R):
    """True iff two agents moving at constant velocity along [n_lo_i, n_hi_i]
    and [n_lo_j, n_hi_j] come closer than R = r_i + r_j (Eq. f_coll_def).
    Touching (distance exactly R) is not a collision (footnote to
    Eq. basic_opt_prob): the test is strict."""
    c_lo = np.asarray(n_lo_j, dtype=np.float64) - np.asarray(n_lo_i, dtype=np.float64)
    c_hi = np.asarray(n_hi_j, dtype=np.float64) - np.asarray(n_hi_i, dtype=np.float64)
    return dist_point_segment(np.zeros_like(c_lo), c_lo, c_hi) < R


def segment_hits_wall(n_lo, n_hi, xL, xR, r):
    """True iff an agent of radius r moving along [n_lo, n_hi] comes closer than
    r to the wall segment [xL, xR] (Eq. wall_minimizer); strict like above."""
    return dist_segment_segment(n_lo, n_hi, xL, xR) < r


# --------------------------------------------------------------------------
# energy minimizer (Appendix E)
# --------------------------------------------------------------------------

def energy_prox(n_lo, n_hi, rho_lo, rho_hi, c):
    """Minimizer of c |x_lo - x_hi|^2 + rho_lo/2 |x_lo - n_lo|^2 + rho_hi/2 |x_hi - n_hi|^2
    (Appendix E, Eq. energy_minimizer_output).

    Infinite weights pin that end (x = n there, the limit of the closed form);
    both weights zero is resolved in the limit rho_lo = rho_hi -> 0+ as the
    appendix prescribes.
    """
    n_lo = np.asarray(n_lo, dtype=np.float64)
    n_hi = np.asarray(n_hi, dtype=np.float64)
    C = float(c)
    if rho_lo == INF and rho_hi == INF:
        return n_lo.copy(), n_hi.copy()
    if rho_lo == INF:
        if rho_hi == 0.0 and C > 0.0:
            return n_lo.copy(), n_lo.copy()
        return n_lo.copy(), (rho_hi * n_hi + 2.0 * C * n_lo) / (2.0 * C + rho_hi)
    if rho_hi == INF:
        if rho_lo == 0.0 and C > 0.0:
            return n_hi.copy(), n_hi.copy()
        return (rho_lo * n_lo + 2.0 * C * n_hi) / (2.0 * C + rho_lo), n_hi.copy()
    if rho_lo == 0.0 and rho_hi == 0.0:
        if C > 0.0:
            mid = 0.5 * (n_lo + n_hi)
            return mid, mid.copy()
        return n_lo.copy(), n_hi.copy()
    den = 2.0 * C * (rho_lo + rho_hi) + rho_lo * rho_hi
    common = 2.0 * C * (rho_lo * n_lo + rho_hi * n_hi)
    x_lo = (rho_lo * rho_hi * n_lo + common) / den
    x_hi = (rho_lo * rho_hi * n_hi + common) / den
    return x_lo, x_hi


# --------------------------------------------------------------------------
# maximum and minimum velocity minimizers (Appendices F and G)
# --------------------------------------------------------------------------

def velocity_prox(n_lo, n_hi, rho_lo, rho_hi, C, kind):
    """Minimizer of rho_lo/2 |x_lo - n_lo|^2 + rho_hi/2 |x_hi - n_hi|^2 subject
    to |x_lo - x_hi| <= C (kind "max", Appendix F) or >= C (kind "min",
    Appendix G).  Returns (x_lo, x_hi, active): inactive (the n's already
    satisfy the limit) gives x = n and outgoing weights 0 (Section 3.3).

    Active finite weights follow the appendix: with
    lambda = (|n_lo - n_hi| / C - 1) / (1/rho_lo + 1/rho_hi),
    x_lo = (rho_lo (rho_hi + lambda) n_lo + lambda rho_hi n_hi) /
           (rho_lo rho_hi + lambda (rho_lo + rho_hi)) and symmetrically x_hi,
    which scales x_lo - x_hi to length C along n_lo - n_hi.  An infinite
    weight keeps that end; a zero weight against a positive one moves only
    the zero-weight end (the limit rho -> 0+); both zero are equal weights
    (as the appendices prescribe).  For "min" with n_lo = n_hi the direction
    is undefined; x_hi - x_lo is then taken along (1, 0) (reading R19).
    """
    n_lo = np.asarray(n_lo, dtype=np.float64)
    n_hi = np.asarray(n_hi, dtype=np.float64)
    C = float(C)
    d = n_lo - n_hi
    L = math.hypot(d[0], d[1])
    active = (L > C) if kind == "max" else (L < C)
    if not active:
        return n_lo.copy(), n_hi.copy(), False
    if rho_lo == INF and rho_hi == INF:
        return n_lo.copy(), n_hi.copy(), True
    if rho_lo == 0.0 and rho_hi == 0.0:
        rho_lo = rho_hi = 1.0
    u = d / L if L > 0.0 else np.array([-1.0, 0.0])   # unit x_lo - x_hi
    if rho_lo == INF or rho_hi == 0.0:
        return n_lo.copy(), n_lo - C * u, True
    if rho_hi == INF or rho_lo == 0.0:
        return n_hi + C * u, n_hi.copy(), True
    if L == 0.0:
        mean = (rho_lo * n_lo + rho_hi * n_hi) / (rho_lo + rho_hi)
        return (mean + (rho_hi / (rho_lo + rho_hi)) * C * u,
                mean - (rho_lo / (rho_lo + rho_hi)) * C * u, True)
    lam = (L / C - 1.0) / (1.0 / rho_lo + 1.0 / rho_hi)
    den = rho_lo * rho_hi + lam * (rho_lo + rho_hi)
    x_lo = (rho_lo * (rho_hi + lam) * n_lo + lam * rho_hi * n_hi) / den
    x_hi = (rho_hi * (rho_lo + lam) * n_hi + lam * rho_lo * n_lo) / den
    return x_lo, x_hi, True


# --------------------------------------------------------------------------
# agent-obstacle minimizer on a disk or capsule (Appendices D and I)
# --------------------------------------------------------------------------

def _unit(theta):
    return np.array([math.cos(theta), math.sin(theta)])


def _angle(v):
    return math.atan2(v[1], v[0]) % TWO_PI


def support(theta, c0, c1, r):
    """Support function h(theta) of the capsule {points within r of [c0, c1]}
    (a disk when c0 == c1).  This is the paper's contact map P(theta) of
    Appendix I in support-function form: the contact circle is the one at c1
    when <c1 - c0, n> >= 0, else the one at c0."""
    n = _unit(theta)
    return max(float(np.dot(c0, n)), float(np.dot(c1, n))) + r


def hinge_energy(theta, a, b, w_lo, w_hi, c0, c1, r):
    """E(theta) of the module docstring (both weights finite)."""
    n = _unit(theta)
    h = support(theta, c0, c1, r)
    ga = max(h - float(np.dot(a, n)), 0.0)
    gb = max(h - float(np.dot(b, n)), 0.0)
    return 0.5 * w_lo * ga * ga + 0.5 * w_hi * gb * gb


def _stationary_both_stretched(a, b, w_lo, w_hi, R):
    """Angles of all stationary points of f(theta) = w_lo (R - <a,n>)^2 +
    w_hi (R - <b,n>)^2 (a disk of radius R at the origin).

    f'(theta)/2 = R (Sx sin - Sy cos) - D/2 sin 2theta + Pxy cos 2theta with
    S = w_lo a + w_hi b, P = w_lo a a^T + w_hi b b^T, D = Pxx - Pyy.  Writing
    w = e^{i theta} and multiplying by 2 i w^2 gives the quartic
    (-D/2 + i Pxy) w^4 + R (Sx - i Sy) w^3 - R (Sx + i Sy) w + (D/2 + i Pxy).
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    S = w_lo * a + w_hi * b
    Pxx = w_lo * a[0] * a[0] + w_hi * b[0] * b[0]
    Pyy = w_lo * a[1] * a[1] + w_hi * b[1] * b[1]
    Pxy = w_lo * a[0] * a[1] + w_hi * b[0] * b[1]
    D = Pxx - Pyy
    coeffs = np.array([complex(-0.5 * D, Pxy), complex(R * S[0], -R * S[1]), 0.0,
                       complex(-R * S[0], -R * S[1]), complex(0.5 * D, Pxy)])
    scale = float(np.max(np.abs(coeffs)))
    if scale == 0.0:
        return []
    coeffs = coeffs / scale
    coeffs[np.abs(coeffs) < 1e-15] = 0.0
    if np.all(coeffs == 0):
        return []
    roots = np.roots(coeffs)

    def g(t):
        return (R * (S[0] * math.sin(t) - S[1] * math.cos(t))
                - 0.5 * D * math.sin(2 * t) + Pxy * math.cos(2 * t))

    def dg(t):
        return (R * (S[0] * math.cos(t) + S[1] * math.sin(t))
                - D * math.cos(2 * t) - 2.0 * Pxy * math.sin(2 * t))

    out = []
    for w in roots:
        t = math.atan2(w.imag, w.real)
        for _ in range(4):  # Newton polish in FP64
            d = dg(t)
            if d == 0.0:
                break
            t_new = t - g(t) / d
            if abs(g(t_new)) < abs(g(t)):
                t = t_new
            else:
                break
        out.append(t % TWO_PI)
    return out


def _tangent_normals(q, c, r):
    """Unit normals n with <q - c, n> = r (the two tangent directions from the
    external point q to the circle of radius r at c)."""
    d = np.asarray(q, dtype=np.float64) - np.asarray(c, dtype=np.float64)
    L2 = float(np.dot(d, d))
    if L2 < r * r * (1.0 - 1e-12):  # a point on the circle up to rounding has one tangent
        return []
    s = math.sqrt(max(L2 - r * r, 0.0))
    perp = np.array([-d[1], d[0]])
    return [(r * d + s * perp) / L2, (r * d - s * perp) / L2]


def _gap(cands, energies, best):
    """Relative energy gap from the chosen direction to the best candidate at
    a clearly different angle (> 1e-3 rad): small values mark near-ties that
    a lower-precision solver may break the other way."""
    e = np.asarray(energies)
    eb = float(np.min(e))
    g = INF
    for t, ei in zip(cands, e):
        d = abs((t - best + math.pi) % TWO_PI - math.pi)
        if d > 1e-3:
            g = min(g, (float(ei) - eb) / max(abs(eb), 1e-300))
    return g


def _pick(cands, energies):
    """Lowest energy; ties within TIE_REL go to the smallest angle in [0, 2pi)."""
    e = np.asarray(energies)
    emin = float(np.min(e))
    tol = TIE_REL * max(abs(emin), 1e-300)
    best = None
    for t, ei in zip(cands, e):
        if ei <= emin + tol and (best is None or t < best):
            best = t
    return best


def project_out(q, c0, c1, r):
    """Closest point to q outside the open capsule of radius r around
    [c0, c1] (q itself when it is outside).  A point on the axis goes out
    along the normal of smallest angle in [0, 2pi) (along (1, 0) for a
    disk)."""
    q = np.asarray(q, dtype=np.float64)
    c0 = np.asarray(c0, dtype=np.float64)
    c1 = np.asarray(c1, dtype=np.float64)
    e = c1 - c0
    ee = float(np.dot(e, e))
    t = 0.0 if ee == 0.0 else min(1.0, max(0.0, float(np.dot(q - c0, e)) / ee))
    c = c0 + t * e
    d = q - c
    L = math.hypot(d[0], d[1])
    if L >= r:
        return q.copy()
    if L > 0.0:
        return c + (r / L) * d
    if ee == 0.0:
        return c + np.array([r, 0.0])
    n1 = np.array([-e[1], e[0]]) / math.sqrt(ee)
    n = n1 if _angle(n1) < _angle(-n1) else -n1
    return c + r * n


def region_prox(a, b, w_lo, w_hi, c0, c1, r, want_gap=False):
    """Minimizer of w_lo/2 |v_lo - a|^2 + w_hi/2 |v_hi - b|^2 subject to the
    segment [v_lo, v_hi] staying out of the open capsule of radius r around
    [c0, c1] (Eqs. wall_min_explicit_opt_problem and
    wall_minimizer_line_constraint; a disk when c0 == c1).

    Returns (v_lo, v_hi, theta) with theta the separating direction (None when
    [a, b] is already feasible or both ends are pinned).  w = inf pins that
    end; both weights zero is the equal-weight limit of Appendix D; one weight
    zero and the other finite is the limit of that weight -> 0+ (reading R18:
    the other end moves out of the region, then this end solves the
    fixed-end problem).  With
    want_gap a fourth value is returned: the relative energy gap to the
    runner-up direction (see ``_gap``).
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c0 = np.asarray(c0, dtype=np.float64)
    c1 = np.asarray(c1, dtype=np.float64)
    if dist_segment_segment(a, b, c0, c1) >= r:
        return (a.copy(), b.copy(), None) + ((INF,) if want_gap else ())
    if w_lo == INF and w_hi == INF:
        return (a.copy(), b.copy(), None) + ((INF,) if want_gap else ())
    if w_lo == 0.0 and w_hi == 0.0:
        w_lo = w_hi = 1.0  # equal weights: the argmin does not depend on their value
    if w_lo == 0.0 and w_hi != INF or w_hi == 0.0 and w_lo != INF:
        # One weight -> 0+ with the other finite: the limit of the argmin is
        # lexicographic.  The weighted end moves the least any feasible
        # segment allows, which is out of the region (a segment shrunk to that
        # point is feasible); the free end then solves the fixed-end problem.
        if w_lo == 0.0:
            v_hi = project_out(b, c0, c1, r)
            out = region_prox(a, v_hi, 1.0, INF, c0, c1, r, want_gap=want_gap)
            return (out[0], v_hi) + tuple(out[2:])
        v_lo = project_out(a, c0, c1, r)
        out = region_prox(v_lo, b, INF, 1.0, c0, c1, r, want_gap=want_gap)
        return (v_lo, out[1]) + tuple(out[2:])

    centres = [c0] if np.array_equal(c0, c1) else [c0, c1]
    kinks = []
    if len(centres) == 2:
        e = c1 - c0
        kinks = [_angle(np.array([-e[1], e[0]])), _angle(np.array([e[1], -e[0]]))]

    if w_lo == INF or w_hi == INF:
        # One end pinned: v at that end is fixed; theta ranges over the arc of
        # directions that separate the pinned point from the region.
        pin, free, w_free = (a, b, w_hi) if w_lo == INF else (b, a, w_lo)
        if w_free == 0.0:
            w_free = 1.0  # the free end's argmin does not depend on its weight
        cands = list(kinks)
        for c in centres:
            cands += [_angle(n) for n in _tangent_normals(pin, c, r)]
            cands.append(_angle(free - c))
        scale = max(1.0, float(np.max(np.abs(np.concatenate([pin, free, c0, c1])))))
        feas, energies = [], []
        for t in cands:
            n = _unit(t)
            h = support(t, c0, c1, r)
            if float(np.dot(pin, n)) - h >= -1e-12 * scale:
                g = max(h - float(np.dot(free, n)), 0.0)
                feas.append(t)
                energies.append(0.5 * w_free * g * g)
        if not feas:
            raise ValueError("pinned end lies inside the obstacle region")
        t = _pick(feas, energies)
        n = _unit(t)
        h = support(t, c0, c1, r)
        v_free = free + max(h - float(np.dot(free, n)), 0.0) * n
        extra = (_gap(feas, energies, t),) if want_gap else ()
        if w_lo == INF:
            return (a.copy(), v_free, t) + extra
        return (v_free, b.copy(), t) + extra

    cands = [0.0] + list(kinks)
    for c in centres:
        cands += _stationary_both_stretched(a - c, b - c, w_lo, w_hi, r)
        for v in (a - c, b - c):
            if np.any(v != 0.0):
                cands.append(_angle(v))
    energies = [hinge_energy(t, a, b, w_lo, w_hi, c0, c1, r) for t in cands]
    t = _pick(cands, energies)
    n = _unit(t)
    h = support(t, c0, c1, r)
    v_lo = a + max(h - float(np.dot(a, n)), 0.0) * n
    v_hi = b + max(h - float(np.dot(b, n)), 0.0) * n
    return (v_lo, v_hi, t) + ((_gap(cands, energies, t),) if want_gap else ())


def wall_prox(n_lo, n_hi, rho_lo, rho_hi, xL, xR, r, want_gap=False):
    """g^wall (Eq. wall_minimizer_problem): agent of radius r avoiding the
    wall segment [xL, xR].  Returns (x_lo, x_hi, active) where active is the
    outgoing-weight decision (Section 3.3.2: rho0 iff the n-segment hits the
    wall, else 0)."""
    n_lo = np.asarray(n_lo, dtype=np.float64)
    n_hi = np.asarray(n_hi, dtype=np.float64)
    if not segment_hits_wall(n_lo, n_hi, xL, xR, r):
        return (n_lo.copy(), n_hi.copy(), False) + ((INF,) if want_gap else ())
    out = region_prox(n_lo, n_hi, rho_lo, rho_hi, xL, xR, r, want_gap=want_gap)
    return (out[0], out[1], True) + ((out[3],) if want_gap else ())


# --------------------------------------------------------------------------
# agent-agent minimizer through the agent-obstacle one (Appendix C)
# --------------------------------------------------------------------------

def _pair_reduction(n, n2, rho, rho2):
    """Reduce rho/2|x - n|^2 + rho2/2|x2 - n2|^2 to the relative coordinate
    v = x2 - x and the sum u = x + x2 (Appendix C).

    Returns (target, weight, recover) so that for fixed v the best u is
    recover(v) and the remaining cost is weight/2 |v - target|^2 + const.
    The sum-coordinate recovery is Eq. linear_tranformation_wall_coll_2.  The
    v-problem is completed exactly: target n2 - n and weight rho rho2/(rho +
    rho2).  For rho == rho2 this is the appendix's Eq.
    linear_tranformation_wall_coll_1 (target 2(rho2 n2 - rho n)/(rho + rho2),
    weight (rho + rho2)/4); for unequal weights the appendix's form does not
    minimise the stated objective, so the exact completion is used.
    """
    n = np.asarray(n, dtype=np.float64)
    n2 = np.asarray(n2, dtype=np.float64)
    target = n2 - n
    if rho == INF and rho2 == INF:
        return target, INF, (lambda v: n + n2)
    if rho == INF:
        return target, rho2, (lambda v: v + 2.0 * n)
    if rho2 == INF:
        return target, rho, (lambda v: -v + 2.0 * n2)
    if rho == 0.0 and rho2 == 0.0:
        return target, 0.0, (lambda v: n + n2)
    s = rho + rho2
    return target, rho * rho2 / s, (lambda v: (rho - rho2) / s * v + 2.0 * (rho * n + rho2 * n2) / s)


def coll_prox(n_lo_i, n_hi_i, n_lo_j, n_hi_j, rho_lo_i, rho_hi_i, rho_lo_j, rho_hi_j, R,
              want_gap=False):
    """g^coll (Eq. coll_minimizer_problem) for agents i and j with R = r_i + r_j.

    Returns (x_lo_i, x_hi_i, x_lo_j, x_hi_j, active).  Inactive (the two
    n-trajectories do not collide) returns x = n and active False (outgoing
    weights 0, Section 3.3.1); otherwise the argmin through Eq.
    wall_min_goes_to_coll_min with a zero-length wall at the origin.
    """
    n_lo_i, n_hi_i, n_lo_j, n_hi_j = (np.asarray(v, dtype=np.float64)
                                      for v in (n_lo_i, n_hi_i, n_lo_j, n_hi_j))
    if not segments_collide(n_lo_i, n_hi_i, n_lo_j, n_hi_j, R):
        return ((n_lo_i.copy(), n_hi_i.copy(), n_lo_j.copy(), n_hi_j.copy(), False)
                + ((INF,) if want_gap else ()))
    t_lo, w_lo, rec_lo = _pair_reduction(n_lo_i, n_lo_j, rho_lo_i, rho_lo_j)
    t_hi, w_hi, rec_hi = _pair_reduction(n_hi_i, n_hi_j, rho_hi_i, rho_hi_j)
    zero = np.zeros(2)
    out = region_prox(t_lo, t_hi, w_lo, w_hi, zero, zero, R, want_gap=want_gap)
    v_lo, v_hi = out[0], out[1]
    u_lo = rec_lo(v_lo)
    u_hi = rec_hi(v_hi)
    return ((0.5 * (u_lo - v_lo), 0.5 * (u_hi - v_hi), 0.5 * (u_lo + v_lo), 0.5 * (u_hi + v_hi),
             True) + ((out[3],) if want_gap else ()))


def coll_objective(x, n, rho):
    """The quadratic part of Eq. coll_minimizer_problem (x, n: four 2-vectors
    in the order lo_i, hi_i, lo_j, hi_j; rho: four weights, finite)."""
    return sum(0.5 * rho[k] * float(np.sum((np.asarray(x[k]) - np.asarray(n[k])) ** 2))
               for k in range(4))
