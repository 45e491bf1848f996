"""The warp-cooperative capsule (wall) minimizer against the sequential one,
both on the GPU, on random and degenerate capsule problems.  They evaluate
the same candidates with the same tie-break, but inlined into different code
the compiler may fuse a different set of multiply-adds, so the results agree
to FP32 rounding rather than bit for bit: equal energies, feasible, and the
same positions except where two candidates tie within rounding."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import prox

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1311_4527_gb300", "csrc")
FP = ctypes.POINTER(ctypes.c_float)


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tempfile.mkdtemp(prefix="capsule_warp_")
    so = os.path.join(d, "libcapsule_warp.so")
    subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-I", CSRC, "-o", so,
                    os.path.join(HERE, "capsule_warp_harness.cu")], check=True, capture_output=True)
    return ctypes.CDLL(so)


def _inputs(n, seed):
    """Agent segments near walls of the 40 x 40 square and of random short
    walls, plus degenerate cases: coincident ends, points on the wall axis,
    zero-length walls."""
    rng = np.random.default_rng(seed)
    q = np.zeros((n, 11))
    for k in range(n):
        kind = k % 4
        r = rng.uniform(0.2, 0.4)
        if kind == 0:      # a square edge, agent near it
            c0, c1 = np.array([0.0, 0.0]), np.array([40.0, 0.0])
            a = np.array([rng.uniform(-2, 42), rng.uniform(-0.3, r + 0.2)])
        elif kind == 1:    # random short wall, agent around it
            c0 = rng.uniform(0, 10, 2)
            c1 = c0 + rng.normal(0, 2, 2)
            a = c0 + rng.normal(0, 1.5, 2)
        elif kind == 2:    # zero-length wall (a post)
            c0 = rng.uniform(0, 10, 2)
            c1 = c0.copy()
            a = c0 + rng.normal(0, 0.5, 2)
        else:              # on the wall's axis
            c0, c1 = np.array([0.0, 0.0]), np.array([5.0, 0.0])
            a = np.array([rng.uniform(-1, 6), 0.0])
        L = rng.choice([0.0, rng.uniform(0, 3)])
        ang = rng.uniform(0, 2 * np.pi)
        b = a + L * np.array([np.cos(ang), np.sin(ang)])
        w = rng.choice([0.5, 1.0]) if k % 3 else 0.5
        q[k] = [*a, *b, *c0, *c1, w, w if k % 5 else 2 * w, r]
    return np.ascontiguousarray(q, dtype=np.float32)


def test_warp_capsule_matches_sequential(lib):
    q = _inputs(20000, 1311_4527)
    n = q.shape[0]
    seq = np.zeros((n, 4), dtype=np.float32)
    war = np.zeros((n, 4), dtype=np.float32)
    rc = lib.capsule_compare(q.ctypes.data_as(FP), ctypes.c_int(n), seq.ctypes.data_as(FP),
                             war.ctypes.data_as(FP))
    assert rc == 0
    assert np.isfinite(seq).all() and np.isfinite(war).all()
    q64 = q.astype(np.float64)
    a, b, c0, c1 = q64[:, 0:2], q64[:, 2:4], q64[:, 4:6], q64[:, 6:8]
    wl, wh, r = q64[:, 8], q64[:, 9], q64[:, 10]
    scale = np.max(np.abs(q64[:, :8]), axis=1) + r

    def energy(v):
        v = v.astype(np.float64)
        return 0.5 * wl * ((v[:, 0:2] - a) ** 2).sum(1) + 0.5 * wh * ((v[:, 2:4] - b) ** 2).sum(1)

    es, ew = energy(seq), energy(war)
    tol = 1e-5 * es + 4e-6 * scale * np.sqrt(es) + 1e-10
    bad = np.nonzero(np.abs(ew - es) > tol)[0]
    assert bad.size == 0, f"{bad.size} energy mismatches, first inputs {q[bad[:3]]}"
    for k in range(n):  # feasible: the moved segment keeps distance r from the wall
        d = prox.dist_segment_segment(war[k, :2].astype(np.float64), war[k, 2:].astype(np.float64),
                                      c0[k], c1[k])
        assert d >= r[k] * (1 - 1e-5) - 1e-6 * scale[k], (k, q[k], war[k], d)
    close = np.abs(war.astype(np.float64) - seq).max(axis=1) <= 1e-4 * scale
    assert close.mean() >= 0.999, f"{(~close).sum()} results differ beyond rounding"
