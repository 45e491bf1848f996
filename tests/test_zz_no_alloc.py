"""The allocation-free entry point plan_iterate_static, called through the C
ABI, against the ordinary planner path (plan_create + plan_iterate).

It serves callers that may not allocate GPU memory themselves (a framework
that owns all device memory, a real-time loop where cudaMalloc is not
allowed); its temporaries live in a static device array shared by every
call.  Calls in a row, on problems of different sizes, check that what the
array keeps from the previous call does not leak into the next one; a
warmed-up call must leave the device's free memory and torch's allocator
untouched; a message out of the consensus range must show up as NaN in
z_out.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import twa

pytestmark = pytest.mark.gpu

TOL = 2e-5


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def _inputs(inst):
    return dict(start=_dev(inst.start), goal=_dev(inst.goal), radius=_dev(inst.radius),
                cost=_dev(inst.cost_w), walls=_dev(inst.walls) if inst.n_walls else None)


def _outputs(state):
    import torch
    out = {name: torch.empty_like(state[name]) for name in ("z", "u_coll", "u_kin", "u_wall")}
    out["act_coll"] = torch.empty_like(state["act_coll"])
    out["act_wall"] = torch.empty_like(state["act_wall"])
    return out


def _call(lib, pk, inst, ins, state, out, k):
    import torch
    cfg = pk.make_config(inst.p, inst.eta, rho0=inst.rho0, alpha=inst.alpha, n_walls=inst.n_walls)
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


def _static_step(lib, pk, inst, state, k):
    return _call(lib, pk, inst, _inputs(inst), state, _outputs(state), k)


def _maxdiff(a, b):
    a = a.float().cpu().numpy()
    b = b.float().cpu().numpy()
    return float(np.max(np.abs(a - b))) if a.size else 0.0


def _scale(inst):
    return max(1.0, float(np.max(np.abs(inst.start))), float(np.max(np.abs(inst.goal))))


def _planner_states(pk, inst, k0, n):
    """The planner's exported states at iterations k0 .. k0 + n."""
    out = []
    with pk.Planner.from_instance(inst) as pl:
        pl.iterate(k0)
        out.append(pl.export_state())
        for _ in range(n):
            pl.iterate(1)
            out.append(pl.export_state())
    return out


def _assert_same(ref, got, L):
    for key in ("z", "u_coll", "u_kin", "u_wall"):
        assert _maxdiff(ref[key], got[key]) <= TOL * L, key
    assert _maxdiff(ref["act_coll"], got["act_coll"]) == 0.0
    assert _maxdiff(ref["act_wall"], got["act_wall"]) == 0.0


def _lib():
    import paper_1311_4527_gb300 as pk
    pk.build()
    return pk, pk.load_library()


@pytest.mark.parametrize("name", ["square72_walls", "circle100"])
def test_static_scratch_iteration_matches_the_planner_twice(name):
    pk, lib = _lib()
    inst = workloads.small_square(72, 6, seed=11) if name == "square72_walls" else workloads.circle100()
    L = _scale(inst)
    s5, s6, s7 = _planner_states(pk, inst, 5, 2)
    o6 = _static_step(lib, pk, inst, s5, s5["k"])
    o7 = _static_step(lib, pk, inst, o6, s5["k"] + 1)
    _assert_same(s6, o6, L)
    _assert_same(s7, o7, L)


def test_a_smaller_problem_after_a_larger_one_sees_no_leftovers():
    """The array keeps the previous call's contents at other offsets: a p = 72
    problem with walls, then the p = 4 circle (no walls, other layout), then
    the p = 72 problem again, each against its own planner."""
    pk, lib = _lib()
    big = workloads.small_square(72, 6, seed=11)
    small = workloads.circle4()
    b5, b6 = _planner_states(pk, big, 30, 1)
    c5, c6 = _planner_states(pk, small, 30, 1)
    _assert_same(b6, _static_step(lib, pk, big, b5, b5["k"]), _scale(big))
    _assert_same(c6, _static_step(lib, pk, small, c5, c5["k"]), _scale(small))
    _assert_same(b6, _static_step(lib, pk, big, b5, b5["k"]), _scale(big))


def test_a_warmed_up_call_allocates_nothing():
    """Once the outputs exist and the first call has looked the array up, a
    call changes neither the device's free memory nor torch's allocator."""
    import torch
    pk, lib = _lib()
    inst = workloads.small_square(72, 6, seed=11)
    s0, s1 = _planner_states(pk, inst, 8, 1)
    ins, out = _inputs(inst), _outputs(s0)
    _call(lib, pk, inst, ins, s0, out, s0["k"])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for _ in range(3):
        _call(lib, pk, inst, ins, s0, out, s0["k"])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
    _assert_same(s1, out, _scale(inst))


def test_a_message_out_of_range_turns_z_out_into_nan():
    """A non-finite z_in entry, or a u large enough that a message leaves the
    consensus sums' fixed-point range (checked on the host with the oracle's
    own messages), sets every entry of z_out to NaN; the next clean call is
    unaffected."""
    import torch
    pk, lib = _lib()
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    L = _scale(inst)
    s5, s6 = _planner_states(pk, inst, 5, 1)
    bad = {k: (v.clone() if hasattr(v, "clone") else v) for k, v in s5.items()}
    bad["z"][1, 2, 0] = float("nan")
    out = _static_step(lib, pk, inst, bad, s5["k"])
    assert torch.isnan(out["z"]).all()
    _assert_same(s6, _static_step(lib, pk, inst, s5, s5["k"]), L)

    bad = {k: (v.clone() if hasattr(v, "clone") else v) for k, v in s5.items()}
    bad["u_kin"][1, 2, 0, 0] = 1.0e6   # the lower edge of agent 2's kinetic factor on segment 1
    st = twa.State(z=bad["z"].cpu().numpy().astype(np.float64),
                   u_coll=bad["u_coll"].cpu().numpy().astype(np.float64),
                   u_kin=bad["u_kin"].cpu().numpy().astype(np.float64),
                   u_wall=np.zeros((0, inst.eta, inst.p, 2, 2)),
                   wback=twa.initial_state(prob).wback, k=s5["k"])
    _, info = twa.iterate(prob, st, record_edges=True)
    bound = 8.0 * (L + 1.0)
    assert max(float(np.max(np.abs(m))) for (_, _, m, _) in info.extra["edges"]) > bound
    out = _static_step(lib, pk, inst, bad, s5["k"])
    assert torch.isnan(out["z"]).all()
    _assert_same(s6, _static_step(lib, pk, inst, s5, s5["k"]), L)
