"""GB300 three-weight ADMM multi-agent trajectory planner.

Python binding of the C ABI in ``include/plan.h`` (Bento, Derbinsky,
Alonso-Mora and Yedidia, "A message-passing algorithm for multi-agent
trajectory planning", NIPS 2013).  The binding only marshals arguments: every
step of an iteration runs in the CUDA kernels of ``csrc/plan.cu``.  PyTorch
provides device memory (the workspace and state buffers) and streams.

The library is required: importing works without it, but creating a
``Planner`` raises if ``libplan.so`` is missing or no CUDA device is present.
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_float, c_int, c_longlong, c_size_t, c_uint, c_void_p

import numpy as np

from .build import LIB, build  # noqa: F401

__all__ = ["Planner", "PlannerBatch", "PlanError", "load_library", "unrolled_trajectory",
           "PLAN_U_KEEP", "PLAN_COST_UNNORM", "PLAN_COST_PER_SEGMENT", "PLAN_DENSE_STATE",
           "PLAN_ADMM", "PLAN_NO_ENERGY", "PLAN_VMAX", "PLAN_VMIN", "PLAN_VO", "PLAN_U_LITERAL",
           "EXPORTED_SYMBOLS"]

PLAN_U_KEEP = 1 << 0
PLAN_COST_UNNORM = 1 << 1
PLAN_COST_PER_SEGMENT = 1 << 2
PLAN_DENSE_STATE = 1 << 3
PLAN_ADMM = 1 << 4
PLAN_NO_ENERGY = 1 << 5
PLAN_VMAX = 1 << 6
PLAN_VMIN = 1 << 7
PLAN_VO = 1 << 8
PLAN_U_LITERAL = 1 << 9

STATUS = {0: "PLAN_OK", 1: "PLAN_EINVAL", 2: "PLAN_ENOMEM", 3: "PLAN_ECUDA", 4: "PLAN_ENOTCONV",
          5: "PLAN_ENUMERIC", 6: "PLAN_EINFEASIBLE_INPUT", 7: "PLAN_EUNSUPPORTED"}

EXPORTED_SYMBOLS = ["plan_workspace_size", "plan_create", "plan_reset", "plan_set_endpoints",
                    "plan_iterate", "plan_solve", "plan_get_trajectory", "plan_export_state",
                    "plan_import_state", "plan_get_info", "plan_backward", "plan_destroy",
                    "plan_last_error", "plan_iterate_static", "plan_profile",
                    "plan_batch_workspace_size", "plan_batch_create", "plan_batch_iterate",
                    "plan_batch_solve", "plan_batch_get_trajectory", "plan_batch_autotune",
                    "plan_batch_set_shape", "plan_batch_destroy", "plan_set_params",
                    "plan_unroll", "plan_set_velocity_limits", "plan_export_velocity_state",
                    "plan_import_velocity_state", "plan_set_energy", "plan_export_back_weights",
                    "plan_import_back_weights", "plan_vo_epoch", "plan_get_endpoints",
                    "plan_check", "plan_batch_import_state", "plan_batch_export_state",
                    "plan_set_endpoints_async"]


class PlanError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class plan_config(ctypes.Structure):
    _fields_ = [("p", c_int), ("eta", c_int), ("T", c_float), ("rho0", c_float),
                ("alpha", c_float), ("warm_iters", c_int), ("warm_rho", c_float),
                ("tol", c_float), ("max_iter", c_int), ("check_every", c_int),
                ("n_walls", c_int), ("flags", c_uint)]


class plan_info(ctypes.Structure):
    _fields_ = [("n_coll", c_longlong), ("n_kin", c_longlong), ("n_wall", c_longlong),
                ("n_pos", c_longlong), ("active_coll", c_longlong), ("active_wall", c_longlong),
                ("k", c_int), ("tile", c_int), ("workspace_bytes", c_size_t)]


_lib = None


def load_library(path: str | None = None):
    """Load libplan.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"the planner's CUDA library is not built ({path}); "
                           "run paper_1311_4527_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    fp = POINTER(c_float)
    lib.plan_workspace_size.argtypes = [POINTER(plan_config), POINTER(c_size_t)]
    lib.plan_create.argtypes = [POINTER(plan_config), fp, fp, fp, fp, fp, c_void_p, c_size_t,
                                c_void_p, POINTER(c_void_p)]
    lib.plan_reset.argtypes = [c_void_p]
    lib.plan_set_endpoints.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.plan_set_endpoints_async.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.plan_iterate.argtypes = [c_void_p, c_int, fp]
    lib.plan_solve.argtypes = [c_void_p, POINTER(c_int), fp]
    lib.plan_get_trajectory.argtypes = [c_void_p, c_void_p, c_int]
    lib.plan_export_state.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p, POINTER(c_int)]
    lib.plan_import_state.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int]
    lib.plan_get_info.argtypes = [c_void_p, POINTER(plan_info)]
    lib.plan_backward.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.plan_set_params.argtypes = [c_void_p, fp, fp]
    lib.plan_unroll.argtypes = [c_void_p, c_int, c_int]
    lib.plan_set_velocity_limits.argtypes = [c_void_p, fp, fp]
    lib.plan_export_velocity_state.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.plan_import_velocity_state.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.plan_set_energy.argtypes = [c_void_p, c_int]
    lib.plan_export_back_weights.argtypes = [c_void_p, c_void_p]
    lib.plan_import_back_weights.argtypes = [c_void_p, c_void_p]
    lib.plan_vo_epoch.argtypes = [c_void_p, c_void_p, c_float, c_float, POINTER(c_int), fp, fp]
    lib.plan_get_endpoints.argtypes = [c_void_p, fp, fp]
    lib.plan_iterate_static.argtypes = [POINTER(plan_config)] + [c_void_p] * 15 + [c_int, c_void_p]
    lib.plan_profile.argtypes = [c_void_p, c_int, fp, POINTER(c_int)]
    dp = POINTER(ctypes.c_double)
    lib.plan_check.argtypes = [c_void_p, dp, dp, dp, dp]
    pp = POINTER(c_void_p)
    lib.plan_batch_workspace_size.argtypes = [c_int, POINTER(plan_config), POINTER(c_size_t)]
    lib.plan_batch_create.argtypes = [c_int, POINTER(plan_config), pp, pp, pp, pp, pp, c_void_p,
                                      c_size_t, c_void_p, POINTER(c_void_p)]
    lib.plan_batch_iterate.argtypes = [c_void_p, c_int]
    lib.plan_batch_solve.argtypes = [c_void_p, POINTER(c_int), fp, POINTER(c_int)]
    lib.plan_batch_get_trajectory.argtypes = [c_void_p, c_int, c_void_p, c_int]
    lib.plan_batch_import_state.argtypes = [c_void_p, c_int] + [c_void_p] * 4
    lib.plan_batch_export_state.argtypes = [c_void_p, c_int] + [c_void_p] * 6
    lib.plan_batch_autotune.argtypes = [c_void_p, c_int, POINTER(c_int)]
    lib.plan_batch_set_shape.argtypes = [c_void_p, c_int, c_int, c_int]
    lib.plan_batch_destroy.argtypes = [c_void_p]
    lib.plan_batch_destroy.restype = None
    lib.plan_destroy.argtypes = [c_void_p]
    lib.plan_destroy.restype = None
    lib.plan_last_error.restype = ctypes.c_char_p
    for name in EXPORTED_SYMBOLS:
        f = getattr(lib, name)
        if name not in ("plan_destroy", "plan_last_error", "plan_batch_destroy"):
            f.restype = c_int
    _lib = lib
    return lib


def _check(code):
    if code != 0:
        msg = _lib.plan_last_error().decode(errors="replace")
        raise PlanError(code, msg)


def _f32_host(a, shape, n):
    """a as a C-contiguous float32 array of the given shape (n entries; no
    copy when it already is one)."""
    if type(a) is np.ndarray and a.dtype == np.float32 and a.size == n and a.flags.c_contiguous:
        return a
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(shape))


def _f32(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(shape))
    return a, a.ctypes.data_as(POINTER(c_float))


def make_config(p, eta, rho0=1.0, alpha=0.1, tol=1e-6, max_iter=20000, n_walls=0, flags=0,
                check_every=50, warm_iters=0, warm_rho=0.0, T=1.0):
    return plan_config(p=p, eta=eta, T=T, rho0=rho0, alpha=alpha, warm_iters=warm_iters,
                       warm_rho=warm_rho, tol=tol, max_iter=max_iter, check_every=check_every,
                       n_walls=n_walls, flags=flags)


class Planner:
    """One planning problem on one GPU.

    ``Planner(start, goal, radius, eta, cost_w=..., walls=..., rho0=..., ...)``
    or ``Planner.from_instance(inst)`` for a ``workloads.Instance``.
    The workspace is a torch uint8 tensor on the current CUDA device; work is
    enqueued on the current torch stream.
    """

    def __init__(self, start, goal, radius, eta, cost_w=None, walls=None, rho0=1.0, alpha=0.1,
                 tol=1e-6, max_iter=20000, flags=0, check_every=50, warm_iters=0, warm_rho=0.0,
                 T=1.0, device=None, stream=None, energy=True, vmax=None, vmin=None, vo=False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Planner needs a CUDA device (there is no CPU fallback)")
        lib = load_library()
        start = np.asarray(start, dtype=np.float64).reshape(-1, 2)
        p = start.shape[0]
        if cost_w is None:
            cost_w = np.ones(p)
        cost_w = np.asarray(cost_w, dtype=np.float64)
        if cost_w.ndim == 2:
            flags |= PLAN_COST_PER_SEGMENT
        if not energy:
            flags |= PLAN_NO_ENERGY
        if vo:
            flags |= PLAN_VO
        if vmax is not None:
            flags |= PLAN_VMAX
        if vmin is not None:
            flags |= PLAN_VMIN
        walls = np.zeros((0, 4)) if walls is None else np.asarray(walls, dtype=np.float64).reshape(-1, 4)
        self.p, self.eta, self.n_walls = p, int(eta), int(walls.shape[0])
        self.flags = flags
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        self.cfg = make_config(p, self.eta, rho0, alpha, tol, max_iter, self.n_walls, flags,
                               check_every, warm_iters, warm_rho, T)
        nbytes = c_size_t(0)
        _check(lib.plan_workspace_size(byref(self.cfg), byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self._keep = []
        self._ep_ptrs = None  # (start, goal, address, address) of the last in-place endpoints
        self._z_ptr = None    # (out, address) of the last trajectory_host destination
        st, st_p = _f32(start, (p, 2))
        gl, gl_p = _f32(goal, (p, 2))
        rd, rd_p = _f32(radius, (p,))
        cw, cw_p = _f32(cost_w, cost_w.shape)
        wl, wl_p = _f32(walls if self.n_walls else np.zeros((1, 4)), (-1, 4))
        h = c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.plan_create(byref(self.cfg), st_p, gl_p, rd_p, cw_p, wl_p,
                                   c_void_p(self.workspace.data_ptr()), nbytes.value,
                                   c_void_p(self.stream.cuda_stream), byref(h)))
        self._h = h
        if vmax is not None or vmin is not None:
            self.set_velocity_limits(vmax, vmin)

    @classmethod
    def from_instance(cls, inst, **kw):
        args = dict(rho0=inst.rho0, alpha=inst.alpha, tol=inst.tol, max_iter=inst.max_iter,
                    T=inst.T)
        args.update(kw)
        return cls(inst.start, inst.goal, inst.radius, inst.eta, cost_w=inst.cost_w,
                   walls=inst.walls, **args)

    # -- lifecycle -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- iteration ----------------------------------------------------------
    def reset(self):
        _check(_lib.plan_reset(self._h))

    def iterate(self, k: int = 1, residual: bool = False):
        """Run k iterations; with residual=True return the last one's residual."""
        if residual:
            r = c_float(0.0)
            _check(_lib.plan_iterate(self._h, int(k), byref(r)))
            return float(r.value)
        _check(_lib.plan_iterate(self._h, int(k), None))
        return None

    def solve(self):
        """Iterate to the tolerance.  Returns (converged, iterations, residual)."""
        it = c_int(0)
        r = c_float(0.0)
        code = _lib.plan_solve(self._h, byref(it), byref(r))
        if code not in (0, 4):
            _check(code)
        return code == 0, int(it.value), float(r.value)

    def set_endpoints(self, start, goal, wait=True):
        """New fixed endpoints, keeping the current iterate.  wait=False
        returns before the device check: an infeasible update is then
        reported (and not applied) by the next call that synchronises."""
        # raw addresses: this call sits in per-step control loops, where
        # building ctypes pointer objects costs more than the call itself;
        # the addresses of arrays passed again (refilled in place) are kept
        f = _lib.plan_set_endpoints if wait else _lib.plan_set_endpoints_async
        c = self._ep_ptrs
        if c is not None and c[0] is start and c[1] is goal:
            _check(f(self._h, c[2], c[3]))
            return
        st = _f32_host(start, (self.p, 2), 2 * self.p)
        gl = _f32_host(goal, (self.p, 2), 2 * self.p)
        sp, gp = st.ctypes.data, gl.ctypes.data
        self._ep_ptrs = (start, goal, sp, gp) if (st is start and gl is goal) else None
        _check(f(self._h, sp, gp))

    def set_params(self, radius=None, cost_w=None):
        """Replace the radii and/or cost weights (same layout as at creation)."""
        rd = _f32(radius, (self.p,)) if radius is not None else (None, None)
        cw = None, None
        if cost_w is not None:
            shape = (self.p, self.eta) if self.flags & PLAN_COST_PER_SEGMENT else (self.p,)
            cw = _f32(cost_w, shape)
        _check(_lib.plan_set_params(self._h, rd[1], cw[1]))

    # -- velocity limits and the feasibility problem -------------------------
    def set_velocity_limits(self, vmax=None, vmin=None):
        """Per-segment limits (p, eta) on |x(s+1) - x(s)|; scalars broadcast."""
        full = lambda v: np.broadcast_to(np.asarray(v, dtype=np.float64), (self.p, self.eta))
        mx = _f32(full(vmax), (self.p, self.eta)) if vmax is not None else (None, None)
        mn = _f32(full(vmin), (self.p, self.eta)) if vmin is not None else (None, None)
        _check(_lib.plan_set_velocity_limits(self._h, mx[1], mn[1]))

    def set_energy(self, on: bool):
        """Switch the kinetic factors on or off (off: the feasibility problem
        from the current state)."""
        _check(_lib.plan_set_energy(self._h, 1 if on else 0))

    def export_velocity_state(self):
        import torch
        dev = self.device
        out = {}
        ptr = lambda t: c_void_p(t.data_ptr()) if t is not None else None
        u = {k: torch.empty((self.eta, self.p, 2, 2), dtype=torch.float32, device=dev)
             if self.flags & f else None for k, f in (("max", PLAN_VMAX), ("min", PLAN_VMIN))}
        a = {k: torch.empty((self.eta, self.p), dtype=torch.uint8, device=dev)
             if self.flags & f else None for k, f in (("max", PLAN_VMAX), ("min", PLAN_VMIN))}
        _check(_lib.plan_export_velocity_state(self._h, ptr(u["max"]), ptr(u["min"]),
                                               ptr(a["max"]), ptr(a["min"])))
        torch.cuda.current_stream(dev).synchronize()
        for k in ("max", "min"):
            if u[k] is not None:
                out[k] = (u[k], a[k])
        return out

    def import_velocity_state(self, u_vmax=None, u_vmin=None):
        import torch
        dev = self.device
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(dev) if a is not None else None
        um, un = t(u_vmax), t(u_vmin)
        self._keep_vel = [um, un]
        ptr = lambda x: c_void_p(x.data_ptr()) if x is not None else None
        _check(_lib.plan_import_velocity_state(self._h, ptr(um), ptr(un)))
        torch.cuda.current_stream(dev).synchronize()

    @classmethod
    def velocity_obstacle(cls, x0, dest, radius, c_prime, step, walls=None, rho0=10.0, **kw):
        """A one-epoch velocity-obstacle planner (Section 5): current
        positions x0, destinations dest, per-agent cost C'_i; step bounds
        |x_ref - x0|.  Advance it with ``vo_epoch``, which sets the reference
        points x_ref on the device at the start of every epoch (until the
        first epoch the goal node holds x0)."""
        x0 = np.asarray(x0, dtype=np.float64).reshape(-1, 2)
        pl = cls(x0, x0, radius, 2, cost_w=c_prime, walls=walls, rho0=rho0, vo=True, **kw)
        import torch
        pl._dest = torch.as_tensor(np.ascontiguousarray(dest, dtype=np.float32)).to(pl.device)
        pl._step = float(step)
        return pl

    def vo_epoch(self, advance: float = 0.5, dest=None, step=None):
        """One epoch: re-target, solve, advance.  Returns (converged,
        iterations, residual, largest remaining distance to dest)."""
        import torch
        if dest is not None:
            self._dest = torch.as_tensor(np.ascontiguousarray(dest, dtype=np.float32)).to(self.device)
        if step is not None:
            self._step = float(step)
        it, r, md = c_int(0), c_float(0.0), c_float(0.0)
        code = _lib.plan_vo_epoch(self._h, c_void_p(self._dest.data_ptr()), c_float(self._step),
                                  c_float(advance), byref(it), byref(r), byref(md))
        if code not in (0, 4):
            _check(code)
        return code == 0, int(it.value), float(r.value), float(md.value)

    def endpoints(self):
        """Current (start, goal) as (p, 2) float32 host arrays (for a
        velocity-obstacle planner: x(0) and x_ref)."""
        st = np.empty((self.p, 2), dtype=np.float32)
        gl = np.empty((self.p, 2), dtype=np.float32)
        _check(_lib.plan_get_endpoints(self._h, st.ctypes.data_as(POINTER(c_float)),
                                       gl.ctypes.data_as(POINTER(c_float))))
        return st, gl

    def export_back_weights(self):
        """(p, eta+1) uint8 classes: 0 zero, 1 rho0, 2 infinite."""
        import torch
        out = torch.empty((self.p, self.eta + 1), dtype=torch.uint8, device=self.device)
        _check(_lib.plan_export_back_weights(self._h, c_void_p(out.data_ptr())))
        torch.cuda.current_stream(self.device).synchronize()
        return out

    def import_back_weights(self, classes):
        import torch
        t = torch.as_tensor(np.ascontiguousarray(classes, dtype=np.uint8)).to(self.device)
        _check(_lib.plan_import_back_weights(self._h, c_void_p(t.data_ptr())))
        torch.cuda.current_stream(self.device).synchronize()

    # -- differentiation ---------------------------------------------------
    def unroll(self, K: int, checkpoint_every: int = 0):
        """Reset to the initial state and run K iterations, keeping
        checkpoints for ``backward`` (0 = every ceil(sqrt(K)) iterations)."""
        _check(_lib.plan_unroll(self._h, int(K), int(checkpoint_every)))
        self._unrolled = int(K)

    def backward(self, dL_dz):
        """Gradient of L(z^K) after ``unroll(K)``: dL_dz is a (p, eta+1, 2)
        tensor.  Returns (d_start, d_goal, d_radius, d_cost_w) float32 device
        tensors, d_cost_w laid out like the cost weights."""
        import torch
        dev = self.device
        g = torch.as_tensor(dL_dz, dtype=torch.float32).to(dev).contiguous()
        if tuple(g.shape) != (self.p, self.eta + 1, 2):
            raise ValueError(f"dL_dz must have shape {(self.p, self.eta + 1, 2)}")
        d_start = torch.empty((self.p, 2), dtype=torch.float32, device=dev)
        d_goal = torch.empty((self.p, 2), dtype=torch.float32, device=dev)
        d_radius = torch.empty((self.p,), dtype=torch.float32, device=dev)
        shape = (self.p, self.eta) if self.flags & PLAN_COST_PER_SEGMENT else (self.p,)
        d_cost = torch.empty(shape, dtype=torch.float32, device=dev)
        ptr = lambda t: c_void_p(t.data_ptr())
        _check(_lib.plan_backward(self._h, getattr(self, "_unrolled", -1), ptr(g), ptr(d_start),
                                  ptr(d_goal), ptr(d_radius), ptr(d_cost)))
        return d_start, d_goal, d_radius, d_cost

    # -- state ------------------------------------------------------------
    def trajectory(self):
        """Break-points z as a (p, eta+1, 2) float32 device tensor."""
        import torch
        z = torch.empty((self.p, self.eta + 1, 2), dtype=torch.float32, device=self.device)
        _check(_lib.plan_get_trajectory(self._h, c_void_p(z.data_ptr()), 1))
        return z

    def trajectory_host(self, out: np.ndarray | None = None):
        c = self._z_ptr
        if c is not None and out is c[0]:
            _check(_lib.plan_get_trajectory(self._h, c[1], 0))
            return out
        if out is None:
            out = np.empty((self.p, self.eta + 1, 2), dtype=np.float32)
        elif (type(out) is not np.ndarray or out.dtype != np.float32 or not out.flags.c_contiguous
              or not out.flags.writeable or out.size != self.p * (self.eta + 1) * 2):
            raise ValueError("out must be a writeable C-contiguous float32 array of "
                             f"{self.p * (self.eta + 1) * 2} entries")
        else:
            self._z_ptr = (out, out.ctypes.data)
        _check(_lib.plan_get_trajectory(self._h, out.ctypes.data, 0))
        return out

    def n_pairs(self):
        return self.p * (self.p - 1) // 2

    def export_state(self):
        """State at the start of the next iteration, in the paper's variables."""
        import torch
        P = self.n_pairs()
        dev = self.device
        z = torch.empty((self.p, self.eta + 1, 2), dtype=torch.float32, device=dev)
        u_coll = torch.empty((self.eta, P, 4, 2), dtype=torch.float32, device=dev)
        u_kin = torch.empty((self.eta, self.p, 2, 2), dtype=torch.float32, device=dev)
        u_wall = torch.empty((self.n_walls, self.eta, self.p, 2, 2), dtype=torch.float32, device=dev)
        act_coll = torch.empty((self.eta, P), dtype=torch.uint8, device=dev)
        act_wall = torch.empty((self.n_walls, self.eta, self.p), dtype=torch.uint8, device=dev)
        k = c_int(0)
        ptr = lambda t: c_void_p(t.data_ptr()) if t.numel() else None
        _check(_lib.plan_export_state(self._h, ptr(z), ptr(u_coll), ptr(u_kin), ptr(u_wall),
                                      ptr(act_coll), ptr(act_wall), byref(k)))
        torch.cuda.current_stream(dev).synchronize()
        return dict(z=z, u_coll=u_coll, u_kin=u_kin, u_wall=u_wall, act_coll=act_coll,
                    act_wall=act_wall, k=int(k.value))

    def import_state(self, z, u_coll, u_kin, u_wall, k: int):
        import torch
        dev = self.device
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        zt, uk = t(z), t(u_kin)
        uc = t(u_coll) if self.p > 1 else None
        uw = t(u_wall) if self.n_walls else None
        self._keep = [zt, uc, uk, uw]
        ptr = lambda x: c_void_p(x.data_ptr()) if x is not None else None
        _check(_lib.plan_import_state(self._h, ptr(zt), ptr(uc), ptr(uk), ptr(uw), int(k)))
        torch.cuda.current_stream(dev).synchronize()

    def profile_start(self):
        """Time each kernel of the following iterations with CUDA events."""
        _check(_lib.plan_profile(self._h, 1, None, None))

    def profile_stop(self):
        """Average ms per iteration of the three passes: test (collision
        tests with the kinetic factors and wall tests in the same launch),
        minimizer (walls and pairs) and consensus."""
        ms = (c_float * 4)()
        n = c_int(0)
        _check(_lib.plan_profile(self._h, 0, ms, byref(n)))
        return dict(test=ms[0], minimizer=ms[1], consensus=ms[3], iterations=n.value)

    def check(self):
        """FP64 final check of the current break-points on the device:
        total kinetic cost, smallest pair clearance / (r_i + r_j), smallest
        wall clearance / r_i and largest endpoint error (plan_check)."""
        v = [ctypes.c_double() for _ in range(4)]
        _check(_lib.plan_check(self._h, *(byref(x) for x in v)))
        return dict(total_cost=v[0].value, min_pair_clearance=v[1].value,
                    min_wall_clearance=v[2].value, max_endpoint_error=v[3].value)

    def info(self):
        inf = plan_info()
        _check(_lib.plan_get_info(self._h, byref(inf)))
        return {f: getattr(inf, f) for f, _ in plan_info._fields_}


class PlannerBatch:
    """Many independent problems advanced together (one launch per pass).

    ``PlannerBatch([inst, ...], flags=0, check_every=50)`` with
    ``workloads.Instance`` members; members must share the state-mode flags.
    """

    def __init__(self, instances, flags=0, check_every=50, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("PlannerBatch needs a CUDA device (there is no CPU fallback)")
        lib = load_library()
        self.instances = list(instances)
        n = len(self.instances)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        cfgs = (plan_config * n)()
        self._arrays = []
        ptrs = {k: (c_void_p * n)() for k in ("start", "goal", "radius", "cost", "walls")}
        for b, inst in enumerate(self.instances):
            cw = np.asarray(inst.cost_w, dtype=np.float64)
            fl = flags | (PLAN_COST_PER_SEGMENT if cw.ndim == 2 else 0)
            cfgs[b] = make_config(inst.p, inst.eta, inst.rho0, inst.alpha, inst.tol, inst.max_iter,
                                  inst.n_walls, fl, check_every, 0, 0.0, inst.T)
            arrs = dict(start=_f32(inst.start, (inst.p, 2))[0], goal=_f32(inst.goal, (inst.p, 2))[0],
                        radius=_f32(inst.radius, (inst.p,))[0], cost=_f32(cw, cw.shape)[0],
                        walls=_f32(inst.walls, (-1, 4))[0] if inst.n_walls else None)
            self._arrays.append(arrs)
            for k, a in arrs.items():
                ptrs[k][b] = a.ctypes.data if a is not None else None
        self.cfgs = cfgs
        nbytes = c_size_t(0)
        _check(lib.plan_batch_workspace_size(n, cfgs, byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        h = c_void_p()
        _check(lib.plan_batch_create(n, cfgs, ptrs["start"], ptrs["goal"], ptrs["radius"],
                                     ptrs["cost"], ptrs["walls"], c_void_p(self.workspace.data_ptr()),
                                     nbytes.value, c_void_p(self.stream.cuda_stream), byref(h)))
        self._h = h
        self.n = n

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.plan_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def iterate(self, k=1):
        _check(_lib.plan_batch_iterate(self._h, int(k)))

    def solve(self):
        """Returns (iterations per member, residual per member, number converged)."""
        its = (c_int * self.n)()
        res = (c_float * self.n)()
        nc = c_int(0)
        _check(_lib.plan_batch_solve(self._h, its, res, byref(nc)))
        return list(its), list(res), nc.value

    def autotune(self, iters_per_candidate=8):
        ch = (c_int * 3)()
        _check(_lib.plan_batch_autotune(self._h, int(iters_per_candidate), ch))
        return dict(rows_per_warp=ch[0], prox_ctas_per_sm=ch[1], iterations_per_graph=ch[2])

    def set_shape(self, rows_per_warp, prox_ctas_per_sm, iterations_per_graph):
        _check(_lib.plan_batch_set_shape(self._h, int(rows_per_warp), int(prox_ctas_per_sm),
                                         int(iterations_per_graph)))

    def import_state(self, member, z, u_coll, u_kin, u_wall):
        """Replace one member's state (oracle layouts, host arrays) at the
        batch's current iteration."""
        import torch
        inst = self.instances[member]
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(self.device)
        keep = [t(z), t(u_coll) if inst.p > 1 else None, t(u_kin), t(u_wall) if inst.n_walls else None]
        ptr = lambda x: c_void_p(x.data_ptr()) if x is not None else None
        _check(_lib.plan_batch_import_state(self._h, int(member), *(ptr(x) for x in keep)))

    def export_state(self, member):
        """One member's state in the oracle's layouts (as Planner.export_state)."""
        import torch
        inst = self.instances[member]
        p, eta, nw = inst.p, inst.eta, inst.n_walls
        P = p * (p - 1) // 2
        dev = self.device
        out = dict(z=torch.empty((p, eta + 1, 2), dtype=torch.float32, device=dev),
                   u_coll=torch.empty((eta, P, 4, 2), dtype=torch.float32, device=dev),
                   u_kin=torch.empty((eta, p, 2, 2), dtype=torch.float32, device=dev),
                   u_wall=torch.empty((nw, eta, p, 2, 2), dtype=torch.float32, device=dev),
                   act_coll=torch.empty((eta, P), dtype=torch.uint8, device=dev),
                   act_wall=torch.empty((nw, eta, p), dtype=torch.uint8, device=dev))
        ptr = lambda t: c_void_p(t.data_ptr()) if t.numel() else None
        _check(_lib.plan_batch_export_state(self._h, int(member), ptr(out["z"]), ptr(out["u_coll"]),
                                            ptr(out["u_kin"]), ptr(out["u_wall"]),
                                            ptr(out["act_coll"]), ptr(out["act_wall"])))
        return out

    def trajectory(self, member):
        import torch
        inst = self.instances[member]
        z = torch.empty((inst.p, inst.eta + 1, 2), dtype=torch.float32, device=self.device)
        _check(_lib.plan_batch_get_trajectory(self._h, int(member), c_void_p(z.data_ptr()), 1))
        return z


def _unrolled_function():
    import torch

    class UnrolledTrajectory(torch.autograd.Function):
        """z^K of K unrolled TWA iterations as a differentiable function of
        (start, goal, radius, cost_w); backward runs the planner's adjoint
        kernels (plan_backward) with the forward run's branches frozen."""

        @staticmethod
        def forward(ctx, start, goal, radius, cost_w, planner, K, checkpoint_every):
            host = lambda t: t.detach().to("cpu", torch.float32).numpy()
            planner.set_endpoints(host(start), host(goal))
            planner.set_params(host(radius), host(cost_w))
            planner.unroll(K, checkpoint_every)
            ctx.planner = planner
            ctx.shapes = (start.shape, goal.shape, radius.shape, cost_w.shape)
            ctx.devices = (start.device, goal.device, radius.device, cost_w.device)
            return planner.trajectory().to(start.device)

        @staticmethod
        def backward(ctx, gz):
            grads = ctx.planner.backward(gz.detach().to(ctx.planner.device, torch.float32))
            out = tuple(g.reshape(sh).to(dv) for g, sh, dv in zip(grads, ctx.shapes, ctx.devices))
            return out + (None, None, None)

    return UnrolledTrajectory


_UNROLLED = None


def unrolled_trajectory(planner: "Planner", start, goal, radius, cost_w, K: int,
                        checkpoint_every: int = 0):
    """Differentiable z^K (p, eta+1, 2) after K iterations from the initial
    state, for torch tensors start, goal (p, 2), radius (p,) and cost_w
    (laid out as the planner's cost weights).  The planner's inputs are
    replaced by these values."""
    global _UNROLLED
    if _UNROLLED is None:
        _UNROLLED = _unrolled_function()
    return _UNROLLED.apply(start, goal, radius, cost_w, planner, int(K), int(checkpoint_every))
