"""The CUDA path's FP32 minimizers (csrc/twa_math.cuh), compiled for the host
by tests/minimizer_harness.cu, against the FP64 oracle on random inputs:
feasible outputs and energies at the oracle's minimum up to FP32 rounding.
CPU only (needs nvcc, which builds the harness)."""
import ctypes
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import prox

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1311_4527_gb300", "csrc")
FP = ctypes.POINTER(ctypes.c_float)


@pytest.fixture(scope="module")
def H():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp(prefix="twa_harness_")
    so = os.path.join(d, "libharness.so")
    subprocess.run([nvcc, "-x", "cu", "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                    "-I", CSRC, "-o", so, os.path.join(HERE, "minimizer_harness.cu")],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(so)
    lib.h_iters.restype = ctypes.c_longlong
    return lib


def _a(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    return a, a.ctypes.data_as(FP)


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _E(vl, vh, a, b, wl, wh):
    return 0.5 * wl * np.sum((vl - a) ** 2) + 0.5 * wh * np.sum((vh - b) ** 2)


def _disk(H, a, b, wl, wh, R):
    A, pa = _a(a)
    B, pb = _a(b)
    out = np.zeros(4, np.float32)
    H.h_disk_prox_free(pa, pb, ctypes.c_float(wl), ctypes.c_float(wh), ctypes.c_float(R),
                       out.ctypes.data_as(FP))
    return out[:2].astype(np.float64), out[2:].astype(np.float64)


def _capsule(H, a, b, wl, wh, c0, c1, r):
    A, pa = _a(a)
    B, pb = _a(b)
    C0, p0 = _a(c0)
    C1, p1 = _a(c1)
    out = np.zeros(4, np.float32)
    H.h_capsule_prox_free(pa, pb, ctypes.c_float(wl), ctypes.c_float(wh), p0, p1, ctypes.c_float(r),
                          out.ctypes.data_as(FP))
    return out[:2].astype(np.float64), out[2:].astype(np.float64)


def _tol(e, scale):
    # FP32 rounding of positions of size `scale` costs ~1e-6 scale in each
    # displacement, i.e. ~1e-6 scale sqrt(E) in energy
    return 1e-5 * e + 4e-6 * scale * math.sqrt(e) + 1e-10


def test_disk_minimizer_matches_the_oracle(H):
    rng = np.random.default_rng(21)
    zero = np.zeros(2)
    n = 0
    for _ in range(3000):
        R = float(np.float32(rng.uniform(0.2, 1.0)))
        a, b = _f32(rng.normal(size=(2, 2)) * 0.8)
        if prox.dist_point_segment(zero, a, b) >= R:
            continue
        wl, wh = (0.5, 0.5) if n % 2 else tuple(_f32(rng.uniform(0.2, 3.0, size=2)))
        vl, vh = _disk(H, a, b, wl, wh, R)
        ol, oh, _ = prox.region_prox(a, b, wl, wh, zero, zero, R)
        assert prox.dist_point_segment(zero, vl, vh) >= R * (1 - 1e-6)
        e_g, e_o = _E(vl, vh, a, b, wl, wh), _E(ol, oh, a, b, wl, wh)
        assert e_g <= e_o + _tol(e_o, 2.0), (a, b, wl, wh, R, e_g, e_o)
        n += 1
    assert n > 1000


def test_capsule_minimizer_matches_the_oracle(H):
    rng = np.random.default_rng(22)
    n = 0
    for k in range(2000):
        if k % 2:
            c0, c1 = _f32([0.0, 0.0]), _f32([40.0, 0.0])      # a long wall, agent near it
            a = _f32([rng.uniform(1, 39), rng.uniform(0.0, 0.5)])
            b = _f32(a + rng.normal(size=2) * 0.8)
            scale = 40.0
        else:
            c0, c1 = _f32(rng.normal(size=(2, 2)))
            a, b = _f32(rng.normal(size=(2, 2)) * 1.2)
            scale = 3.0
        r = float(np.float32(rng.uniform(0.1, 0.5)))
        if prox.dist_segment_segment(a, b, c0, c1) >= r:
            continue
        wl, wh = tuple(_f32(rng.uniform(0.2, 3.0, size=2)))
        vl, vh = _capsule(H, a, b, wl, wh, c0, c1, r)
        ol, oh, _ = prox.region_prox(a, b, wl, wh, c0, c1, r)
        assert prox.dist_segment_segment(vl, vh, c0, c1) >= r * (1 - 1e-5) - 1e-6 * scale
        e_g, e_o = _E(vl, vh, a, b, wl, wh), _E(ol, oh, a, b, wl, wh)
        assert e_g <= e_o + _tol(e_o, scale), (a, b, wl, wh, c0, c1, r, e_g, e_o)
        n += 1
    assert n > 500


def test_capsule_minimizer_on_the_wall_line_and_at_an_end_centre(H):
    """Targets where the end-circle skip decides signs near zero: on the
    wall's line beyond an end, on the perpendicular through an end, and at an
    end centre (an exact energy tie between directions), against the
    oracle's minimizer; the skip rule keeps the circle's candidates for the
    targets beyond the end or at its centre."""
    rng = np.random.default_rng(31)
    n = 0
    for k in range(600):
        L = float(np.float32(rng.uniform(0.5, 40.0)))
        ang = rng.uniform(0, 2 * np.pi)
        e = np.array([np.cos(ang), np.sin(ang)])
        c0 = _f32(rng.normal(size=2) * 3)
        c1 = _f32(c0 + L * e)
        r = float(np.float32(rng.uniform(0.1, 0.5)))
        ci = k % 2
        cc, out = (c1, e) if ci else (c0, -e)
        kind = (k // 2) % 3
        if kind == 0:        # on the line through the wall, a little beyond the end
            a = _f32(cc + rng.uniform(0.0, r) * out)
        elif kind == 1:      # on the perpendicular through the end
            a = _f32(cc + rng.uniform(-r, r) * np.array([-e[1], e[0]]))
        else:                # at the end centre
            a = _f32(cc)
        b = _f32(a + rng.normal(size=2) * 0.5)
        wl, wh = (0.5, 0.5) if k % 3 else tuple(_f32(rng.uniform(0.2, 3.0, size=2)))
        A, pa = _a(a)
        B, pb = _a(b)
        C0, p0 = _a(c0)
        C1, p1 = _a(c1)
        if kind != 1:  # beyond the end, or at its centre: that circle is never skipped
            assert not H.h_capsule_end_dominated(pa, pb, p0, p1, ci), (a, b, ci, kind)
        if prox.dist_segment_segment(a, b, c0, c1) >= r:
            continue
        vl, vh = _capsule(H, a, b, wl, wh, c0, c1, r)
        ol, oh, _ = prox.region_prox(a, b, wl, wh, c0, c1, r)
        scale = float(np.abs(np.concatenate([c0, c1, a, b])).max()) + 1.0
        assert prox.dist_segment_segment(vl, vh, c0, c1) >= r * (1 - 1e-5) - 1e-6 * scale
        e_g, e_o = _E(vl, vh, a, b, wl, wh), _E(ol, oh, a, b, wl, wh)
        assert e_g <= e_o + _tol(e_o, scale), (a, b, wl, wh, c0, c1, r, e_g, e_o)
        n += 1
    assert n > 200


def test_capsule_end_circle_skip_is_sound(H):
    """Where the FP32 wall minimizer skips an end circle's candidates, no
    direction of that circle's half-plane (where it gives the capsule's
    support) has a lower capsule energy than the better kink: checked in
    FP64 on 4,096 directions of the half-plane, for walls long and short
    and targets near the wall, past its ends and across its line."""
    rng = np.random.default_rng(29)
    th = np.linspace(0.0, 2 * np.pi, 4096, endpoint=False)
    dirs = np.stack([np.cos(th), np.sin(th)], axis=1)
    checked = 0
    for k in range(3000):
        if k % 2:
            c0, c1 = _f32([0.0, 0.0]), _f32([rng.uniform(0.5, 40.0), 0.0])
            a = _f32([rng.uniform(-3, c1[0] + 3), rng.uniform(-1.0, 1.0)])
        else:
            c0, c1 = _f32(rng.normal(size=(2, 2)) * 2)
            a = _f32(rng.normal(size=2) * 2)
        b = _f32(a + rng.normal(size=2) * 1.0)
        r = float(np.float32(rng.uniform(0.1, 0.5)))
        wl, wh = (0.5, 0.5) if k % 3 else (0.5, 1.5)
        e = c1 - c0
        nu = np.array([-e[1], e[0]]) / np.linalg.norm(e)

        def energy(n):
            h = np.maximum(n @ c0, n @ c1) + r
            ga = np.maximum(h - n @ a, 0.0)
            gb = np.maximum(h - n @ b, 0.0)
            return 0.5 * wl * ga * ga + 0.5 * wh * gb * gb

        kink = min(energy(nu[None])[0], energy(-nu[None])[0])
        for ci in (0, 1):
            A, pa = _a(a)
            B, pb = _a(b)
            C0, p0 = _a(c0)
            C1, p1 = _a(c1)
            if not H.h_capsule_end_dominated(pa, pb, p0, p1, ci):
                continue
            cc, other = (c1, c0) if ci else (c0, c1)
            half = dirs[dirs @ (cc - other) >= 0.0]
            emin = energy(half).min()
            assert emin >= kink * (1 - 1e-9) - 1e-12, (a, b, c0, c1, r, ci, emin, kink)
            checked += 1
    assert checked > 1000


def test_pinned_minimizers_match_the_oracle(H):
    rng = np.random.default_rng(23)
    zero = np.zeros(2)
    n = 0
    for _ in range(2000):
        R = float(np.float32(rng.uniform(0.2, 0.8)))
        q = _f32(rng.normal(size=2) * 1.5)
        w = _f32(rng.normal(size=2))
        if np.linalg.norm(q) <= R * 1.001 or prox.dist_point_segment(zero, q, w) >= R:
            continue
        Q, pq = _a(q)
        W, pw = _a(w)
        out = np.zeros(2, np.float32)
        H.h_disk_prox_pinned(pq, pw, ctypes.c_float(R), out.ctypes.data_as(FP))
        v = out.astype(np.float64)
        ol, oh, _ = prox.region_prox(q, w, math.inf, 1.0, zero, zero, R)
        assert prox.dist_point_segment(zero, q, v) >= R * (1 - 1e-6)
        e_g, e_o = 0.5 * np.sum((v - w) ** 2), 0.5 * np.sum((oh - w) ** 2)
        assert e_g <= e_o + _tol(e_o, 2.0)
        n += 1
    assert n > 500


def test_energy_minimizer_matches_the_oracle(H):
    rng = np.random.default_rng(24)
    for _ in range(500):
        nl, nh = _f32(rng.normal(size=(2, 2)) * 10)
        rho, c = float(np.float32(rng.uniform(0.1, 3))), float(np.float32(rng.uniform(0, 2)))
        for pl, ph in ((0, 0), (1, 0), (0, 1)):
            N1, p1 = _a(nl)
            N2, p2 = _a(nh)
            out = np.zeros(4, np.float32)
            H.h_energy_prox(p1, p2, ctypes.c_float(rho), pl, ph, ctypes.c_float(c), out.ctypes.data_as(FP))
            ol, oh = prox.energy_prox(nl, nh, math.inf if pl else rho, math.inf if ph else rho, c)
            assert np.allclose(out[:2], ol, atol=2e-5 * 10) and np.allclose(out[2:], oh, atol=2e-5 * 10)


def test_secular_iterations_stay_few(H):
    """Newton on the concave secular function from the left converges in a
    handful of steps (the latency of the minimizer pass)."""
    rng = np.random.default_rng(25)
    zero = np.zeros(2)
    calls = iters = worst = 0
    for _ in range(2000):
        R = float(rng.uniform(0.2, 1.0))
        a, b = rng.normal(size=(2, 2)) * 0.8
        if prox.dist_point_segment(zero, a, b) >= R:
            continue
        H.h_reset_iters()
        _disk(H, a, b, 0.5, 0.5, R)
        k = H.h_iters(0)
        iters += k
        worst = max(worst, k)
        calls += 1
    assert iters / calls < 5 and worst <= 12


def _jt(f, v, xb, h):
    """J(v)^T xb by central differences of f in FP64."""
    out = np.zeros_like(v)
    for q in range(v.shape[0]):
        e = np.zeros_like(v)
        e[q] = h
        out[q] = float(xb @ ((f(v + e) - f(v - e)) / (2 * h)))
    return out


def _coll_fd(n, R, wl, wh):
    nn = n.reshape(4, 2)
    return np.concatenate(prox.coll_prox(nn[0], nn[1], nn[2], nn[3], wl, wh, wl, wh, R)[:4])


def test_collision_adjoint_matches_oracle_differences(H):
    """The FP32 adjoint of the pair collision minimizer (twa_adjoint.cuh)
    against J^T xbar of the FP64 oracle minimizer by central differences, on
    random active pairs, free and with either end fixed.  Pairs whose oracle
    minimum is a near-tie, or whose differences at two step sizes disagree
    (a branch boundary within the step), are skipped."""
    rng = np.random.default_rng(31)
    errs = {0: [], 1: [], 2: []}
    tags = set()
    for trial in range(3000):
        pin = trial % 3  # 0 free, 1 lower end fixed, 2 upper end fixed
        R = float(np.float32(rng.uniform(0.2, 0.8)))
        n = _f32(rng.normal(size=8) * 0.6)
        if not prox.segments_collide(n[0:2], n[2:4], n[4:6], n[6:8], R):
            continue
        if pin == 1 and np.linalg.norm(n[4:6] - n[0:2]) < R * 1.01:
            continue
        if pin == 2 and np.linalg.norm(n[6:8] - n[2:4]) < R * 1.01:
            continue
        wl = math.inf if pin == 1 else 1.0
        wh = math.inf if pin == 2 else 1.0
        if prox.coll_prox(n[0:2], n[2:4], n[4:6], n[6:8], wl, wh, wl, wh, R, want_gap=True)[5] < 1e-3:
            continue
        xb = rng.normal(size=8)
        if pin == 1:
            xb[0:2] = xb[4:6] = 0.0
        if pin == 2:
            xb[2:4] = xb[6:8] = 0.0
        f = lambda v: _coll_fd(v, R, wl, wh)
        r1, r2 = _jt(f, n, xb, 1e-6), _jt(f, n, xb, 1e-5)
        if np.abs(r1 - r2).max() > 1e-5 * (1 + np.abs(r1).max()):
            continue
        dR = float(xb @ (_coll_fd(n, R + 1e-6, wl, wh) - _coll_fd(n, R - 1e-6, wl, wh))) / 2e-6
        ref = np.concatenate([r1, [dR]])
        N, pn = _a(n)
        X, px = _a(xb)
        out = np.zeros(9, np.float32)
        H.h_coll_vjp(pn, int(pin == 1), int(pin == 2), ctypes.c_float(R), ctypes.c_float(1.0), px,
                     out.ctypes.data_as(FP))
        errs[pin].append(np.abs(out - ref).max() / (1 + np.abs(ref).max()))
        if pin == 0:
            c = n[4:6] - n[0:2], n[6:8] - n[2:4]
            A, pa = _a(c[0])
            B, pb = _a(c[1])
            tags.add(H.h_disk_tag(pa, pb, ctypes.c_float(0.5), ctypes.c_float(0.5), ctypes.c_float(R)))
    for pin, e in errs.items():
        e = np.asarray(e)
        assert e.size > 200, (pin, e.size)
        assert np.median(e) < 1e-6 and e.max() < 5e-4, (pin, np.median(e), e.max())
    assert {1, 2, 4} <= tags  # global, and both single-hinge directions


def test_energy_adjoint_matches_oracle_differences(H):
    rng = np.random.default_rng(32)
    for _ in range(200):
        nl, nh = _f32(rng.normal(size=(2, 2)) * 3)
        rho, c = float(np.float32(rng.uniform(0.1, 3))), float(np.float32(rng.uniform(0, 2)))
        xb = rng.normal(size=4)
        for pl, ph in ((0, 0), (1, 0), (0, 1)):
            wl, wh = (math.inf if pl else rho), (math.inf if ph else rho)
            v = np.concatenate([nl, nh])
            f = lambda u: np.concatenate(prox.energy_prox(u[:2], u[2:], wl, wh, c))
            ref_n = _jt(f, v, xb, 1e-4)
            fc = lambda cc: np.concatenate(prox.energy_prox(nl, nh, wl, wh, cc))
            ref_c = float(xb @ (fc(c + 1e-6) - fc(c - 1e-6))) / 2e-6
            N1, p1 = _a(nl)
            N2, p2 = _a(nh)
            X, px = _a(xb)
            out = np.zeros(5, np.float32)
            H.h_energy_vjp(p1, p2, ctypes.c_float(rho), pl, ph, ctypes.c_float(c), px, out.ctypes.data_as(FP))
            ref = np.concatenate([ref_n, [ref_c]])
            assert np.abs(out - ref).max() <= 1e-5 * (1 + np.abs(ref).max()), (pl, ph, out, ref)


def test_wall_adjoint_matches_oracle_differences(H):
    """The FP32 adjoint of the wall minimizer (capsule, free and with either
    end fixed) against J^T xbar of the FP64 oracle wall minimizer by central
    differences; near-ties and branch boundaries within the step skipped."""
    rng = np.random.default_rng(33)
    wall = np.array([-0.6, 0.1, 0.7, -0.2])
    errs = {0: [], 1: [], 2: []}
    for trial in range(1500):
        pin = trial % 3
        r = float(np.float32(rng.uniform(0.2, 0.5)))
        n = _f32(rng.normal(size=4) * 0.8)
        if prox.dist_segment_segment(n[:2], n[2:], wall[:2], wall[2:]) >= r:
            continue
        if pin == 1 and prox.dist_point_segment(n[:2], wall[:2], wall[2:]) < r * 1.01:
            continue
        if pin == 2 and prox.dist_point_segment(n[2:], wall[:2], wall[2:]) < r * 1.01:
            continue
        wl = math.inf if pin == 1 else 1.0
        wh = math.inf if pin == 2 else 1.0
        if prox.wall_prox(n[:2], n[2:], wl, wh, wall[:2], wall[2:], r, want_gap=True)[3] < 1e-3:
            continue
        xb = rng.normal(size=4)
        if pin == 1:
            xb[:2] = 0.0
        if pin == 2:
            xb[2:] = 0.0
        f = lambda v, rr=r: np.concatenate(prox.wall_prox(v[:2], v[2:], wl, wh, wall[:2], wall[2:], rr)[:2])
        r1, r2 = _jt(f, n, xb, 1e-6), _jt(f, n, xb, 1e-5)
        if np.abs(r1 - r2).max() > 1e-5 * (1 + np.abs(r1).max()):
            continue
        dr = float(xb @ (f(n, r + 1e-6) - f(n, r - 1e-6))) / 2e-6
        ref = np.concatenate([r1, [dr]])
        N, pn = _a(n)
        Wl, pw = _a(wall)
        X, px = _a(xb)
        out = np.zeros(5, np.float32)
        H.h_wall_vjp(pn, int(pin == 1), int(pin == 2), pw, ctypes.c_float(r), ctypes.c_float(1.0), px,
                     out.ctypes.data_as(FP))
        errs[pin].append(np.abs(out - ref).max() / (1 + np.abs(ref).max()))
    for pin, e in errs.items():
        e = np.asarray(e)
        assert e.size > 100, (pin, e.size)
        assert np.median(e) < 1e-6 and e.max() < 5e-4, (pin, np.median(e), e.max())


def test_velocity_adjoint_matches_oracle_differences(H):
    rng = np.random.default_rng(34)
    for kind in ("max", "min"):
        for _ in range(200):
            n = _f32(rng.normal(size=4))
            L = float(np.linalg.norm(n[:2] - n[2:]))
            C = float(np.float32(L * (0.6 if kind == "max" else 1.6)))
            xb = rng.normal(size=4)
            for pin in (0, 1, 2):
                wl = math.inf if pin == 1 else 1.0
                wh = math.inf if pin == 2 else 1.0
                x = xb.copy()
                if pin == 1:
                    x[:2] = 0.0
                if pin == 2:
                    x[2:] = 0.0
                f = lambda v: np.concatenate(prox.velocity_prox(v[:2], v[2:], wl, wh, C, kind)[:2])
                ref = _jt(f, n, x, 1e-6)
                N, pn = _a(n)
                X, px = _a(x)
                out = np.zeros(4, np.float32)
                H.h_velocity_vjp(pn, int(pin == 1), int(pin == 2), ctypes.c_float(C), px,
                                 out.ctypes.data_as(FP))
                assert np.abs(out - ref).max() <= 2e-5 * (1 + np.abs(ref).max()), (kind, pin, out, ref)
