"""Thin Python binding of the C ABI in include/chem.h (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module only passes device pointers
of torch tensors (FP64, cell-fastest [component, cell] layout), sizes and the current CUDA
stream.  It raises if the compiled library is missing: there is no CPU fallback.

Names follow the C ABI without the ``chem_`` prefix: mech_load, eval_source, eval_jacobian,
integrate, integrate_workspace, integrate_host, kernel_config.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

from . import build as _build

MODE_PERSISTENT = 0
MODE_PLAIN = 1
STATUS_OK, STATUS_MAX_STEPS, STATUS_H_UNDERFLOW, STATUS_NONFINITE, STATUS_SKIPPED = 0, 1, 2, 3, 4

EXPORTS = ["chem_mech_load", "chem_mech_compile_only", "chem_mech_free", "chem_mech_info",
           "chem_mech_lnA", "chem_eval_source", "chem_eval_jacobian", "chem_integrate_workspace",
           "chem_integrate", "chem_integrate_host", "chem_kernel_config", "chem_autotune",
           "chem_tape_bytes", "chem_integrate_ckpt", "chem_adjoint_workspace", "chem_adjoint",
           "chem_eval_vjp", "chem_adjoint_noalloc", "chem_fp64_probe", "chem_cost_order",
           "chem_cost_order_workspace", "chem_jac_cache_bytes", "chem_last_error"]
STATUS_TAPE_FULL = 5

CACHE_DIR = os.environ.get("CHEM_CACHE_DIR", os.path.join(os.path.dirname(__file__), "_cache"))


class BuildOpts(C.Structure):
    _fields_ = [("team", C.c_int32), ("block", C.c_int32), ("verbose", C.c_int32),
                ("cache_dir", C.c_char_p), ("adjoint", C.c_int32), ("tableau", C.c_int32)]


class TapeStruct(C.Structure):
    _fields_ = [("mem", C.c_void_p), ("bytes", C.c_size_t), ("n_cells", C.c_int64),
                ("capacity", C.c_int32), ("interval", C.c_int32)]


class IntOpts(C.Structure):
    _fields_ = [("max_steps", C.c_int32), ("h_min", C.c_double), ("T_min", C.c_double),
                ("mode", C.c_int32), ("team", C.c_int32), ("block", C.c_int32),
                ("lnA", C.c_void_p), ("attempts", C.c_void_p), ("tableau", C.c_int32),
                ("order", C.c_void_p), ("cell_method", C.c_void_p),
                ("jac_cache", C.c_void_p), ("alt_tableau", C.c_int32)]


_lib = None
_lock = threading.Lock()


class ChemError(RuntimeError):
    pass


def library(build_if_missing: bool = True):
    """Load libchem.so (building it in-tree first if asked)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise ChemError("libchem.so is not built (run paper_2205_05681_gb300/build.py)")
            lib = C.CDLL(path)
            vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
            lib.chem_last_error.restype = C.c_char_p
            lib.chem_mech_load.argtypes = [C.c_char_p, C.POINTER(BuildOpts), C.POINTER(vp)]
            lib.chem_mech_compile_only.argtypes = [C.c_char_p, C.POINTER(BuildOpts), C.c_char_p,
                                                   C.c_size_t]
            lib.chem_mech_free.argtypes = [vp]
            lib.chem_mech_info.argtypes = [vp] + [C.POINTER(C.c_int32)] * 3
            lib.chem_mech_lnA.argtypes = [vp, vp]
            lib.chem_eval_source.argtypes = [vp, i64, vp, vp, vp, vp, i64, vp, vp]
            lib.chem_eval_jacobian.argtypes = [vp, i64, vp, vp, vp, vp, i64, vp, vp]
            lib.chem_integrate_workspace.restype = C.c_size_t
            lib.chem_integrate_workspace.argtypes = [vp, i64, C.POINTER(IntOpts)]
            lib.chem_integrate.argtypes = [vp, i64, vp, vp, vp, i64, dbl, dbl, dbl, vp, vp,
                                           C.POINTER(IntOpts), vp, C.c_size_t, vp]
            lib.chem_integrate_host.argtypes = [vp, i64, vp, vp, vp, dbl, dbl, dbl, vp, vp,
                                                C.POINTER(IntOpts), vp]
            lib.chem_kernel_config.argtypes = [vp, C.POINTER(IntOpts)] + [C.POINTER(C.c_int32)] * 4
            lib.chem_tape_bytes.restype = C.c_size_t
            lib.chem_tape_bytes.argtypes = [vp, i64, C.c_int32, C.c_int32]
            lib.chem_integrate_ckpt.argtypes = [vp, i64, vp, vp, vp, i64, dbl, dbl, dbl, vp, vp,
                                                C.POINTER(IntOpts), C.POINTER(TapeStruct), vp,
                                                C.c_size_t, vp]
            lib.chem_adjoint_workspace.restype = C.c_size_t
            lib.chem_adjoint_workspace.argtypes = [vp, i64, C.POINTER(IntOpts), C.c_int32]
            lib.chem_adjoint.argtypes = [vp, i64, vp, vp, vp, i64, C.POINTER(TapeStruct),
                                         C.POINTER(IntOpts), vp, vp, vp, vp, C.c_size_t, vp]
            lib.chem_eval_vjp.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, i64, vp, vp]
            lib.chem_adjoint_noalloc.argtypes = [vp, i64, vp, vp, vp, i64, C.POINTER(TapeStruct),
                                                 C.POINTER(IntOpts), vp, vp, vp, vp]
            lib.chem_fp64_probe.argtypes = [vp] + [C.POINTER(C.c_double)] * 3
            lib.chem_cost_order_workspace.restype = C.c_size_t
            lib.chem_cost_order_workspace.argtypes = []
            lib.chem_cost_order.argtypes = [vp, i64, vp, vp, vp, C.c_size_t, vp]
            lib.chem_jac_cache_bytes.restype = C.c_size_t
            lib.chem_jac_cache_bytes.argtypes = [vp, i64]
            lib.chem_autotune.argtypes = [vp, i64, vp, vp, vp, i64, dbl, dbl, dbl, vp,
                                          C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_float)]
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != 0:
        raise ChemError("chem error %d: %s" % (rc, library().chem_last_error().decode()))


ROS4, ROS3, RODAS3, RODAS4 = 0, 1, 2, 3  # Rosenbrock methods (CHEM_ROS4 ...)
RKF45 = 4  # explicit Runge-Kutta-Fehlberg 4(5) (CHEM_RKF45), for non-stiff cells
ROS2W = 5  # the W-method ROS2 (CHEM_ROS2W), with a factorisation cache (jac_cache)


def compile_only(spec_path: str, team: int = 0, block: int = 0, cache_dir: Optional[str] = None,
                 verbose: bool = False, adjoint: bool = False, tableau: int = ROS4) -> str:
    """Generate and NVRTC-compile a mechanism's kernels for sm_103a (no GPU needed)."""
    buf = C.create_string_buffer(1 << 16)
    o = BuildOpts(team, block, int(verbose), cache_dir.encode() if cache_dir else None,
                  int(adjoint), int(tableau))
    _check(library().chem_mech_compile_only(spec_path.encode(), C.byref(o), buf, len(buf)))
    return buf.value.decode(errors="replace")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _req(t, name, dtype=None, shape=None):
    import torch
    dtype = dtype or torch.float64
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ChemError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ChemError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ChemError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ChemError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return t


class Mechanism:
    """A loaded mechanism: tables on the host, compiled sm_103a kernels on the current device."""

    def __init__(self, spec_path: str, team: int = 0, block: int = 0, verbose: bool = False,
                 cache_dir: Optional[str] = CACHE_DIR):
        lib = library()
        if cache_dir:
            os.makedirs(cache_dir, exist_ok=True)
        self._lib = lib
        self.spec_path = spec_path
        h = C.c_void_p()
        o = BuildOpts(team, block, int(verbose), cache_dir.encode() if cache_dir else None, 0, 0)
        _check(lib.chem_mech_load(spec_path.encode(), C.byref(o), C.byref(h)))
        self._h = h
        ns, nr, ne = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib.chem_mech_info(h, C.byref(ns), C.byref(nr), C.byref(ne)))
        self.ns, self.nr, self.ne = ns.value, nr.value, ne.value
        self.N = self.ns

    def __del__(self):
        try:
            self._lib.chem_mech_free(self._h)
        except Exception:
            pass

    def lnA(self):
        import numpy as np
        out = np.zeros(self.nr)
        _check(self._lib.chem_mech_lnA(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    # ------------------------------------------------------------------ evaluation
    def eval_source(self, T, P, n, lnA=None, stream=None):
        """T, P [C]; n [Ns-1, C] -> f [Ns, C] (f[0] = dT/dt)."""
        import torch
        Cn = T.shape[0]
        _req(T, "T", shape=(Cn,)); _req(P, "P", shape=(Cn,)); _req(n, "n", shape=(self.ns - 1, Cn))
        if lnA is not None:
            _req(lnA, "lnA", shape=(self.nr,))
        f = torch.empty((self.ns, Cn), dtype=torch.float64, device=T.device)
        _check(self._lib.chem_eval_source(self._h, Cn, _ptr(T), _ptr(P), _ptr(n), _ptr(f), Cn,
                                          _ptr(lnA), _stream(stream)))
        return f

    def eval_jacobian(self, T, P, n, lnA=None, stream=None):
        """-> J [Ns*Ns, C], row-major within a cell."""
        import torch
        Cn = T.shape[0]
        _req(T, "T", shape=(Cn,)); _req(P, "P", shape=(Cn,)); _req(n, "n", shape=(self.ns - 1, Cn))
        if lnA is not None:
            _req(lnA, "lnA", shape=(self.nr,))
        J = torch.empty((self.ns * self.ns, Cn), dtype=torch.float64, device=T.device)
        _check(self._lib.chem_eval_jacobian(self._h, Cn, _ptr(T), _ptr(P), _ptr(n), _ptr(J), Cn,
                                            _ptr(lnA), _stream(stream)))
        return J

    # ------------------------------------------------------------------ integration
    def opts(self, mode=MODE_PERSISTENT, max_steps=0, h_min=0.0, T_min=0.0, team=0, block=0,
             lnA=None, attempts=None, tableau=ROS4, order=None, cell_method=None,
             jac_cache=None, alt_tableau=0) -> IntOpts:
        return IntOpts(max_steps, h_min, T_min, mode, team, block,
                       None if lnA is None else lnA.data_ptr(),
                       None if attempts is None else attempts.data_ptr(), int(tableau),
                       None if order is None else order.data_ptr(),
                       None if cell_method is None else cell_method.data_ptr(),
                       None if jac_cache is None else jac_cache.data_ptr(), int(alt_tableau))

    def jac_cache(self, n_cells: int, device="cuda"):
        """An empty (zeroed) W-method factorisation cache for n_cells cells (float64 tensor)."""
        import torch
        nbytes = int(self._lib.chem_jac_cache_bytes(self._h, n_cells))
        return torch.zeros(nbytes // 8, dtype=torch.float64, device=device)

    def cost_order(self, cost, order=None, workspace=None, stream=None):
        """Cells by decreasing cost (int32 [C] device) -> order int32 [C] (chem_cost_order)."""
        import torch
        Cn = cost.shape[0]
        _req(cost, "cost", dtype=torch.int32, shape=(Cn,))
        if order is None:
            order = torch.empty(Cn, dtype=torch.int32, device=cost.device)
        _req(order, "order", dtype=torch.int32, shape=(Cn,))
        if workspace is None:
            nb = int(self._lib.chem_cost_order_workspace())
            workspace = torch.empty((nb + 255) // 256 * 256, dtype=torch.uint8, device=cost.device)
        _check(self._lib.chem_cost_order(self._h, Cn, _ptr(cost), _ptr(order), _ptr(workspace),
                                         workspace.numel(), _stream(stream)))
        return order

    def integrate_workspace(self, n_cells: int, opts: Optional[IntOpts] = None) -> int:
        o = opts or self.opts()
        return int(self._lib.chem_integrate_workspace(self._h, n_cells, C.byref(o)))

    def workspace(self, n_cells: int, opts: Optional[IntOpts] = None, device="cuda"):
        import torch
        nbytes = self.integrate_workspace(n_cells, opts)
        return torch.empty((nbytes + 255) // 256 * 256, dtype=torch.uint8, device=device)

    def integrate(self, T, P, Y, dt, rtol=1e-6, atol=1e-10, h=None, status=None, opts=None,
                  workspace=None, stream=None):
        """In place: T [C], Y [Ns, C] (mass fractions); h [C] in/out (optional)."""
        import torch
        Cn = T.shape[0]
        _req(T, "T", shape=(Cn,)); _req(P, "P", shape=(Cn,)); _req(Y, "Y", shape=(self.ns, Cn))
        if h is not None:
            _req(h, "h", shape=(Cn,))
        if status is not None:
            _req(status, "status", dtype=torch.int32, shape=(Cn,))
        o = opts or self.opts()
        if workspace is None:
            workspace = self.workspace(Cn, o, device=T.device)
        _check(self._lib.chem_integrate(self._h, Cn, _ptr(T), _ptr(P), _ptr(Y), Cn, dt, rtol,
                                        atol, _ptr(h), _ptr(status), C.byref(o),
                                        _ptr(workspace), workspace.numel(), _stream(stream)))
        return T, Y

    def integrate_host(self, T, P, Y, dt, rtol=1e-6, atol=1e-10, h=None, status=None,
                       opts=None, stream=None):
        """Numpy (host) arrays in place: T [C], P [C], Y [Ns, C] C-contiguous float64."""
        import numpy as np
        Cn = T.shape[0]
        for a, nm in ((T, "T"), (P, "P"), (Y, "Y")):
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise ChemError("%s must be C-contiguous float64" % nm)
        if Y.shape != (self.ns, Cn):
            raise ChemError("Y must be [Ns, C]")
        hp = None if h is None else h.ctypes.data_as(C.c_void_p)
        sp = None if status is None else status.ctypes.data_as(C.c_void_p)
        o = opts or self.opts()
        _check(self._lib.chem_integrate_host(self._h, Cn, T.ctypes.data_as(C.c_void_p),
                                             P.ctypes.data_as(C.c_void_p),
                                             Y.ctypes.data_as(C.c_void_p), dt, rtol, atol, hp, sp,
                                             C.byref(o), _stream(stream)))

    # ------------------------------------------------------------------ adjoint
    def make_tape(self, n_cells: int, capacity: int = 2048, interval: int = 16, device="cuda"):
        """Device memory for one checkpointed forward (see chem_tape_bytes)."""
        import torch
        nbytes = int(self._lib.chem_tape_bytes(self._h, n_cells, capacity, interval))
        if nbytes == 0:
            raise ChemError("bad tape sizes")
        buf = torch.empty((nbytes + 255) // 256 * 256, dtype=torch.uint8, device=device)
        return Tape(buf, n_cells, capacity, interval)

    def integrate_ckpt(self, T, P, Y, dt, tape, rtol=1e-6, atol=1e-10, h=None, status=None,
                       opts=None, workspace=None, stream=None):
        """chem_integrate that records `tape` for chem_adjoint (in place on T, Y)."""
        import torch
        Cn = T.shape[0]
        _req(T, "T", shape=(Cn,)); _req(P, "P", shape=(Cn,)); _req(Y, "Y", shape=(self.ns, Cn))
        o = opts or self.opts()
        if workspace is None:
            workspace = torch.empty(256, dtype=torch.uint8, device=T.device)
        _check(self._lib.chem_integrate_ckpt(self._h, Cn, _ptr(T), _ptr(P), _ptr(Y), Cn, dt, rtol,
                                             atol, _ptr(h), _ptr(status), C.byref(o),
                                             C.byref(tape.struct), _ptr(workspace),
                                             workspace.numel(), _stream(stream)))
        return T, Y

    def adjoint(self, P, gT, gY, tape, opts=None, stream=None):
        """Reverse sweep: returns (g_lnA [Nr], gT0 [C], gY0 [Ns, C])."""
        import torch
        Cn = P.shape[0]
        _req(P, "P", shape=(Cn,)); _req(gT, "gT", shape=(Cn,)); _req(gY, "gY", shape=(self.ns, Cn))
        o = opts or self.opts()
        nb = int(self._lib.chem_adjoint_workspace(self._h, Cn, C.byref(o), tape.interval))
        if nb == 0:
            _check(-1)
        ws = torch.empty((nb + 255) // 256 * 256, dtype=torch.uint8, device=P.device)
        g_lnA = torch.empty(self.nr, dtype=torch.float64, device=P.device)
        gT0 = torch.empty(Cn, dtype=torch.float64, device=P.device)
        gY0 = torch.empty((self.ns, Cn), dtype=torch.float64, device=P.device)
        _check(self._lib.chem_adjoint(self._h, Cn, _ptr(P), _ptr(gT), _ptr(gY), Cn,
                                      C.byref(tape.struct), C.byref(o), _ptr(g_lnA), _ptr(gT0),
                                      _ptr(gY0), _ptr(ws), ws.numel(), _stream(stream)))
        return g_lnA, gT0, gY0

    def adjoint_noalloc(self, P, gT, gY, tape, g_lnA, gT0, gY0, opts=None, stream=None):
        """chem_adjoint without a workspace (static scratch in the adjoint module); the caller
        provides the output tensors g_lnA [Nr], gT0 [C], gY0 [Ns, C]."""
        Cn = P.shape[0]
        _req(P, "P", shape=(Cn,)); _req(gT, "gT", shape=(Cn,)); _req(gY, "gY", shape=(self.ns, Cn))
        _req(g_lnA, "g_lnA", shape=(self.nr,)); _req(gT0, "gT0", shape=(Cn,))
        _req(gY0, "gY0", shape=(self.ns, Cn))
        o = opts or self.opts()
        _check(self._lib.chem_adjoint_noalloc(self._h, Cn, _ptr(P), _ptr(gT), _ptr(gY), Cn,
                                              C.byref(tape.struct), C.byref(o), _ptr(g_lnA),
                                              _ptr(gT0), _ptr(gY0), _stream(stream)))
        return g_lnA, gT0, gY0

    def eval_vjp(self, T, P, n, v, lnA=None, stream=None):
        """gy = J^T v [Ns, C] and gp = (df/dlnA)^T v [Nr, C] per cell."""
        import torch
        Cn = T.shape[0]
        _req(T, "T", shape=(Cn,)); _req(P, "P", shape=(Cn,)); _req(n, "n", shape=(self.ns - 1, Cn))
        _req(v, "v", shape=(self.ns, Cn))
        gy = torch.empty((self.ns, Cn), dtype=torch.float64, device=T.device)
        gp = torch.empty((self.nr, Cn), dtype=torch.float64, device=T.device)
        _check(self._lib.chem_eval_vjp(self._h, Cn, _ptr(T), _ptr(P), _ptr(n), _ptr(v), _ptr(gy),
                                       _ptr(gp), Cn, _ptr(lnA), _stream(stream)))
        return gy, gp

    def autotune(self, T, P, Y, dt, rtol=1e-6, atol=1e-10, stream=None):
        """Choose and set the fastest (team, block) on a sample of these cells; returns it."""
        Cn = T.shape[0]
        _req(T, "T", shape=(Cn,)); _req(P, "P", shape=(Cn,)); _req(Y, "Y", shape=(self.ns, Cn))
        t, b, ms = C.c_int32(), C.c_int32(), C.c_float()
        _check(self._lib.chem_autotune(self._h, Cn, _ptr(T), _ptr(P), _ptr(Y), Cn, dt, rtol, atol,
                                       _stream(stream), C.byref(t), C.byref(b), C.byref(ms)))
        return {"team": t.value, "block": b.value, "sample_ms": ms.value}

    def kernel_config(self, opts: Optional[IntOpts] = None):
        o = opts or self.opts()
        t, b, s, r = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(self._lib.chem_kernel_config(self._h, C.byref(o), C.byref(t), C.byref(b),
                                            C.byref(s), C.byref(r)))
        return {"team": t.value, "block": b.value, "smem": s.value, "regs": r.value}


def fp64_probe(stream=None):
    """FP64 pipe throughput of the current GPU: {"dfma_tflops", "exp_cost", "log_cost"} (the
    last two in FMA-equivalents of pipe time), from chem_fp64_probe."""
    lib = library()
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(lib.chem_fp64_probe(_stream(stream), C.byref(a), C.byref(b), C.byref(c)))
    return {"dfma_tflops": a.value, "exp_cost": b.value, "log_cost": c.value}


class Tape:
    """Device memory of one checkpointed forward (chem_tape)."""

    def __init__(self, buf, n_cells, capacity, interval):
        self.buf = buf
        self.n_cells, self.capacity, self.interval = n_cells, capacity, interval
        self.struct = TapeStruct(buf.data_ptr(), buf.numel(), n_cells, capacity, interval)

    def n_accepted(self):
        """Accepted steps per cell (int32 [n_cells] view of the tape's first block)."""
        import torch
        return self.buf[: 4 * self.n_cells].view(torch.int32)

    def step_sizes(self):
        """Accepted step sizes, float64 [capacity, n_cells] view (layout of chem_tape_bytes)."""
        import torch
        off = (4 * self.n_cells + 255) // 256 * 256
        n = 8 * self.n_cells * self.capacity
        return self.buf[off: off + n].view(torch.float64).view(self.capacity, self.n_cells)


def chem_integrate_fn():
    """torch.autograd.Function: (T0 [C], Y0 [Ns, C], lnA [Nr]) -> (T [C], Y [Ns, C]) with
    gradients from the checkpointed discrete adjoint."""
    import torch

    class ChemIntegrate(torch.autograd.Function):
        @staticmethod
        def forward(ctx, T0, Y0, lnA, mech, P, dt, rtol, atol, capacity, interval):
            T, Y = T0.detach().clone(), Y0.detach().clone()
            lnA = lnA.detach().contiguous()
            tape = mech.make_tape(T.shape[0], capacity, interval, device=T.device)
            status = torch.empty(T.shape[0], dtype=torch.int32, device=T.device)
            mech.integrate_ckpt(T, P, Y, dt, tape, rtol=rtol, atol=atol, status=status,
                                opts=mech.opts(lnA=lnA))
            ctx.mech, ctx.tape, ctx.lnA = mech, tape, lnA
            ctx.save_for_backward(P)
            ctx.status = status
            return T, Y

        @staticmethod
        def backward(ctx, gT, gY):
            (P,) = ctx.saved_tensors
            bad = int((ctx.status != STATUS_OK).sum().item())
            if bad:
                # a cell that stopped early (attempt limit, step underflow, full tape, bad input)
                # did not integrate to dt: its gradient would belong to a different map
                codes = sorted(set(ctx.status[ctx.status != STATUS_OK].tolist()))
                raise ChemError("backward through chem_integrate_ckpt: %d cell(s) did not reach "
                                "dt (status codes %s); enlarge the tape capacity or max_steps"
                                % (bad, codes))
            T_like = P
            gT = torch.zeros_like(T_like) if gT is None else gT.contiguous()
            gY = (torch.zeros((ctx.mech.ns, P.shape[0]), dtype=torch.float64, device=P.device)
                  if gY is None else gY.contiguous())
            g_lnA, gT0, gY0 = ctx.mech.adjoint(P, gT, gY, ctx.tape,
                                               opts=ctx.mech.opts(lnA=ctx.lnA))
            return gT0, gY0, g_lnA, None, None, None, None, None, None, None

    return ChemIntegrate
