"""The C-ABI library builds for sm_103a, loads, exports every symbol that
include/plan.h declares, and rejects bad input on the host before touching a
GPU.  CPU only: no kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1311_4527_gb300 as pk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pk.build()
    return pk.load_library()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "plan.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(plan_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    assert _declared_symbols() == sorted(pk.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_built_for_sm_103a(lib):
    # the one nvcc target of the build
    import importlib
    b = importlib.import_module("paper_1311_4527_gb300.build")
    assert b.ARCH == "-gencode=arch=compute_103a,code=sm_103a"
    assert os.path.exists(pk.LIB)


def _cfg(p, eta, **kw):
    return pk.make_config(p, eta, **kw)


def test_workspace_size_scales_with_the_problem(lib):
    n1, n2 = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.plan_workspace_size(ctypes.byref(_cfg(64, 8)), ctypes.byref(n1)) == 0
    assert lib.plan_workspace_size(ctypes.byref(_cfg(128, 8)), ctypes.byref(n2)) == 0
    # collision state grows with the number of tile pairs: 3 -> 10 for 2 -> 4 tiles
    assert n2.value > 3 * n1.value
    assert n1.value % 256 == 0


def test_workspace_size_rejects_bad_sizes(lib):
    n = ctypes.c_size_t()
    assert lib.plan_workspace_size(ctypes.byref(_cfg(0, 8)), ctypes.byref(n)) == 1
    assert lib.plan_workspace_size(ctypes.byref(_cfg(4, 0)), ctypes.byref(n)) == 1
    assert lib.plan_workspace_size(None, ctypes.byref(n)) == 1


def _create(lib, cfg, start, goal, radius, cost=None, walls=None):
    p = cfg.p
    f = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    st, gl, rd = f(start), f(goal), f(radius)
    cw = f(np.ones(p) if cost is None else cost)
    wl = f(np.zeros((1, 4)) if walls is None else walls)
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    h = ctypes.c_void_p()
    code = lib.plan_create(ctypes.byref(cfg), ptr(st), ptr(gl), ptr(rd), ptr(cw), ptr(wl),
                           None, 0, None, ctypes.byref(h))
    return code, lib.plan_last_error().decode()


def test_overlapping_starts_are_rejected_on_the_host(lib):
    code, msg = _create(lib, _cfg(2, 4), [[0, 0], [0.1, 0]], [[5, 0], [0, 5]], [0.2, 0.2])
    assert code == 6 and "start" in msg


def test_overlapping_goals_are_rejected_on_the_host(lib):
    code, msg = _create(lib, _cfg(2, 4), [[0, 0], [3, 0]], [[5, 5], [5.3, 5]], [0.2, 0.2])
    assert code == 6 and "goal" in msg


def test_endpoint_inside_a_wall_is_rejected(lib):
    cfg = _cfg(1, 4, n_walls=1)
    code, msg = _create(lib, cfg, [[0, 0.1]], [[3, 3]], [0.2], walls=[[-1, 0, 1, 0]])
    assert code == 6 and "wall" in msg


def test_touching_endpoints_are_allowed_by_the_check(lib):
    """Distance exactly r_i + r_j passes the host check (touching is feasible);
    the call then fails only because there is no GPU here, or succeeds."""
    code, msg = _create(lib, _cfg(2, 4), [[0, 0], [0.5, 0]], [[5, 0], [0, 5]], [0.25, 0.25])
    assert code != 6


def test_bad_parameters_are_rejected(lib):
    for kw in (dict(rho0=0.0), dict(alpha=-1.0), dict(flags=1 << 20), dict(max_iter=-1)):
        code, _ = _create(lib, _cfg(2, 4, **kw), [[0, 0], [3, 0]], [[5, 5], [0, 5]], [0.2, 0.2])
        assert code == 1, kw
    code, _ = _create(lib, _cfg(2, 4), [[0, 0], [3, 0]], [[5, 5], [0, 5]], [0.2, -0.2])
    assert code == 1
    code, _ = _create(lib, _cfg(2, 4), [[0, np.nan], [3, 0]], [[5, 5], [0, 5]], [0.2, 0.2])
    assert code == 1


def test_differentiation_entry_points_reject_null_plans(lib):
    f = ctypes.POINTER(ctypes.c_float)
    assert lib.plan_check(None, None, None, None, None) == 1
    assert lib.plan_set_endpoints_async(None, None, None) == 1
    assert lib.plan_batch_import_state(None, 0, None, None, None, None) == 1
    assert lib.plan_batch_export_state(None, 0, None, None, None, None, None, None) == 1
    assert lib.plan_backward(None, 1, None, None, None, None, None) == 1
    assert lib.plan_unroll(None, 10, 0) == 1
    assert lib.plan_set_params(None, None, None) == 1


def test_static_entry_point_rejects_a_problem_that_does_not_fit(lib):
    """plan_iterate_static refuses sizes beyond its static scratch array
    before it touches any pointer."""
    cfg = pk.make_config(1024, 16, n_walls=4)
    dummy = np.zeros(8, dtype=np.float32)
    ptr = ctypes.c_void_p(dummy.ctypes.data)
    code = lib.plan_iterate_static(ctypes.byref(cfg), *([ptr] * 15), 0, None)
    assert code == 2
    assert b"static array" in lib.plan_last_error()


def test_static_entry_point_checks_its_parameters_first(lib):
    """plan_iterate_static validates rho0, alpha and the warm-up like
    plan_create, before any pointer is used."""
    dummy = np.zeros(8, dtype=np.float32)
    ptr = ctypes.c_void_p(dummy.ctypes.data)
    for kw in (dict(rho0=float("nan")), dict(alpha=0.0), dict(warm_iters=5, warm_rho=0.0),
               dict(warm_iters=5, warm_rho=float("nan")), dict(warm_iters=-1)):
        cfg = pk.make_config(8, 4, **kw)
        assert lib.plan_iterate_static(ctypes.byref(cfg), *([ptr] * 15), 0, None) == 1, kw
    code, _ = _create(lib, _cfg(2, 4, warm_iters=5, warm_rho=0.0), [[0, 0], [3, 0]],
                      [[5, 5], [0, 5]], [0.2, 0.2])
    assert code == 1


@pytest.mark.parametrize("seed", range(4))
def test_grid_overlap_check_matches_brute_force(lib, seed):
    """The host check finds an overlapping pair anywhere in a large layout
    (its neighbour grid must not miss pairs across cell borders)."""
    import workloads
    inst = workloads.small_square(300, 4, seed=100 + seed)
    start = inst.start.copy()
    rng = np.random.default_rng(seed)
    i, j = rng.choice(300, size=2, replace=False)
    # move agent j to overlap agent i by a small amount, in a random direction
    ang = rng.uniform(0, 2 * np.pi)
    d = (inst.radius[i] + inst.radius[j]) * 0.999
    start[j] = start[i] + d * np.array([np.cos(ang), np.sin(ang)])
    code, msg = _create(lib, _cfg(300, 4, n_walls=0), start, inst.goal, inst.radius)
    assert code == 6 and "start" in msg
    # and the unmodified layout passes the check (fails later only for lack of a GPU)
    code, msg = _create(lib, _cfg(300, 4, n_walls=0), inst.start, inst.goal, inst.radius)
    assert code != 6


def test_variant_entry_points_reject_null_plans(lib):
    f = ctypes.c_float
    assert lib.plan_set_velocity_limits(None, None, None) == 1
    assert lib.plan_export_velocity_state(None, None, None, None, None) == 1
    assert lib.plan_import_velocity_state(None, None, None) == 1
    assert lib.plan_set_energy(None, 0) == 1
    assert lib.plan_export_back_weights(None, None) == 1
    assert lib.plan_import_back_weights(None, None) == 1
    assert lib.plan_vo_epoch(None, None, f(0.1), f(0.5), None, None, None) == 1
    assert lib.plan_get_endpoints(None, None, None) == 1


def test_mode_flag_combinations_are_checked_on_the_host(lib):
    args = ([[0, 0], [3, 0]], [[5, 5], [0, 5]], [0.2, 0.2])
    # the local planner has eta = 2 and the kinetic factors
    code, msg = _create(lib, _cfg(2, 4, flags=pk.PLAN_VO), *args)
    assert code == 1 and "eta = 2" in msg
    code, _ = _create(lib, _cfg(2, 2, flags=pk.PLAN_VO | pk.PLAN_NO_ENERGY), *args)
    assert code == 1
    # standard ADMM keeps the kinetic factors and has no velocity factors
    for extra in (pk.PLAN_NO_ENERGY, pk.PLAN_VMAX, pk.PLAN_VMIN):
        code, _ = _create(lib, _cfg(2, 4, flags=pk.PLAN_ADMM | extra), *args)
        assert code == 7, extra


def test_local_planner_goals_may_overlap_but_starts_may_not(lib):
    """A velocity-obstacle epoch's goal node holds reference points, which
    are not tested against each other; the current positions are."""
    code, _ = _create(lib, _cfg(2, 2, flags=pk.PLAN_VO), [[0, 0], [3, 0]], [[1, 1], [1.1, 1]],
                      [0.2, 0.2])
    assert code != 6
    code, msg = _create(lib, _cfg(2, 2, flags=pk.PLAN_VO), [[0, 0], [0.1, 0]], [[1, 1], [4, 1]],
                        [0.2, 0.2])
    assert code == 6 and "start" in msg


def test_static_and_batch_paths_refuse_the_variant_modes(lib):
    cfg = pk.make_config(8, 4, flags=pk.PLAN_NO_ENERGY)
    dummy = np.zeros(8, dtype=np.float32)
    ptr = ctypes.c_void_p(dummy.ctypes.data)
    assert lib.plan_iterate_static(ctypes.byref(cfg), *([ptr] * 15), 0, None) == 7
    cfgs = (pk.plan_config * 1)(pk.make_config(2, 4, flags=pk.PLAN_VMAX))
    arr = (ctypes.c_void_p * 1)(dummy.ctypes.data)
    h = ctypes.c_void_p()
    code = lib.plan_batch_create(1, cfgs, arr, arr, arr, arr, None, None, 0, None, ctypes.byref(h))
    assert code == 7


def test_problems_beyond_32_bit_pair_slots_are_rejected(lib):
    n = ctypes.c_size_t()
    # 65,536 agents x 16 segments: 2,098,176 tile pairs x 16 x 1,024 > 2^32 slots
    assert lib.plan_workspace_size(ctypes.byref(_cfg(65536, 16)), ctypes.byref(n)) == 1
    assert lib.plan_workspace_size(ctypes.byref(_cfg(65536, 1)), ctypes.byref(n)) == 0
