"""The allocation-free entry point plan_iterate_static, called through the C
ABI, against the ordinary planner path (plan_create + plan_iterate).

It serves callers that may not allocate GPU memory themselves (a framework
that owns all device memory, a real-time loop where cudaMalloc is not
allowed); its temporaries live in a static device array shared by every
call.  Two calls in a row check that what the array keeps from the previous
call does not leak into the next one.  This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 2e-5


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def _static_step(lib, pk, inst, state, k):
    import torch
    p, eta, nw = inst.p, inst.eta, inst.n_walls
    cfg = pk.make_config(p, eta, rho0=inst.rho0, alpha=inst.alpha, n_walls=nw)
    ins = dict(start=_dev(inst.start), goal=_dev(inst.goal), radius=_dev(inst.radius),
               cost=_dev(inst.cost_w), walls=_dev(inst.walls) if nw else None)
    out = {name: torch.empty_like(state[name]) for name in ("z", "u_coll", "u_kin", "u_wall")}
    out["act_coll"] = torch.empty_like(state["act_coll"])
    out["act_wall"] = torch.empty_like(state["act_wall"])
    stream = torch.cuda.current_stream()
    code = lib.plan_iterate_static(
        ctypes.byref(cfg), _ptr(ins["start"]), _ptr(ins["goal"]), _ptr(ins["radius"]),
        _ptr(ins["cost"]), _ptr(ins["walls"]), _ptr(state["z"]), _ptr(state["u_coll"]),
        _ptr(state["u_kin"]), _ptr(state["u_wall"]), _ptr(out["z"]), _ptr(out["u_coll"]),
        _ptr(out["u_kin"]), _ptr(out["u_wall"]), _ptr(out["act_coll"]), _ptr(out["act_wall"]),
        int(k), ctypes.c_void_p(stream.cuda_stream))
    assert code == 0, lib.plan_last_error().decode()
    stream.synchronize()
    return out


def _close(a, b, L):
    a = a.float().cpu().numpy()
    b = b.float().cpu().numpy()
    return float(np.max(np.abs(a - b))) if a.size else 0.0


@pytest.mark.parametrize("name", ["square72_walls", "circle100"])
def test_static_scratch_iteration_matches_the_planner_twice(name):
    import paper_1311_4527_gb300 as pk
    pk.build()
    lib = pk.load_library()
    inst = workloads.small_square(72, 6, seed=11) if name == "square72_walls" else workloads.circle100()
    L = max(1.0, float(np.max(np.abs(inst.start))), float(np.max(np.abs(inst.goal))))
    with pk.Planner.from_instance(inst) as pl:
        pl.iterate(5)
        s5 = pl.export_state()
        pl.iterate(1)
        s6 = pl.export_state()
        pl.iterate(1)
        s7 = pl.export_state()
    o6 = _static_step(lib, pk, inst, s5, s5["k"])
    o7 = _static_step(lib, pk, inst, o6, s5["k"] + 1)
    for ref, got in ((s6, o6), (s7, o7)):
        for key in ("z", "u_coll", "u_kin", "u_wall"):
            assert _close(ref[key], got[key], L) <= TOL * L, key
        assert _close(ref["act_coll"], got["act_coll"], L) == 0.0
        assert _close(ref["act_wall"], got["act_wall"], L) == 0.0
