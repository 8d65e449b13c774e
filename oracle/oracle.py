"""Python handle on the CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg, never by the product package.

Arrays are numpy float64 in the oracle's natural per-cell layout: y[cell, i] with
y = [T, n_1, ..., n_{Ns-1}] (n in kmol per kg of mixture), Jacobians J[cell, i, j] = df_i/dy_j.
Conversion between mass fractions and the state vector is done here in numpy (n_k = Y_k / W_k,
and Y_Ns = 1 - sum of the others), independently of the CUDA path's own conversion kernel.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
LIB = os.path.join(HERE, "_build", "liboracle.so")

OK, MAX_STEPS, H_UNDERFLOW, NONFINITE, SKIPPED = 0, 1, 2, 3, 4

_lib = None
_lock = threading.Lock()

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (plain -O2, no fast-math, no FP contraction)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC",
                               "-pthread", SRC, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            vp = C.c_void_p
            lib.orc_last_error.restype = C.c_char_p
            lib.orc_load.restype = vp
            lib.orc_load.argtypes = [C.c_char_p]
            lib.orc_free.argtypes = [vp]
            lib.orc_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
            lib.orc_species.argtypes = [vp, _dp, _ip, _dp, _dp, _dp]
            lib.orc_reactions.argtypes = [vp, _ip, _dp, _ip, _ip]
            lib.orc_thermo.argtypes = [vp, C.c_int, C.c_double] + [C.POINTER(C.c_double)] * 3
            lib.orc_thermo_cplx.argtypes = [vp, C.c_int, C.c_double, C.c_double, _dp]
            lib.orc_source.argtypes = [vp, C.c_int, _dp, _dp, vp, _dp]
            lib.orc_source_cplx.argtypes = [vp, _dp, vp, C.c_double, vp, vp, _dp, _dp]
            lib.orc_jacobian.argtypes = [vp, C.c_int, _dp, _dp, vp, _dp, C.c_int]
            lib.orc_rates.argtypes = [vp, _dp, C.c_double, vp] + [_dp] * 6
            lib.orc_tableau.argtypes = [C.c_int, _dp]
            lib.orc_step_linear.argtypes = [C.c_int, _dp, _dp, C.c_double, _dp, _dp, C.c_int]
            lib.orc_integrate_linear.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double,
                                                 C.c_double, C.POINTER(C.c_int), C.c_int]
            lib.orc_step.argtypes = [vp, _dp, C.c_double, vp, C.c_double, _dp, _dp, C.c_int]
            lib.orc_integrate.argtypes = [vp, C.c_int, _dp, _dp, vp, C.c_double, C.c_double,
                                          C.c_double, vp, vp, vp, vp, vp, C.c_int, C.c_double,
                                          C.c_double, C.c_int, C.c_int, C.c_int]
            lib.orc_integrate_auto.argtypes = [vp, C.c_int, _dp, _dp, vp, C.c_double, C.c_double,
                                               C.c_double, vp, vp, vp, _ip, C.c_int, C.c_double,
                                               C.c_int, C.c_int, C.c_int, vp, vp, vp]
            lib.orc_integrate_w.argtypes = [vp, C.c_int, _dp, _dp, vp, C.c_double, C.c_double,
                                            C.c_double, vp, vp, vp, vp, _dp, _dp, _ip, C.c_int,
                                            C.c_int, C.c_int]
            lib.orc_step_w.argtypes = [vp, _dp, C.c_double, vp, C.c_double, _dp, _dp, _dp, C.c_int]
            lib.orc_integrate_log.argtypes = [vp, _dp, C.c_double, vp, C.c_double, C.c_double,
                                              C.c_double, C.c_double, C.c_int, _dp, C.c_int,
                                              C.POINTER(C.c_int), C.POINTER(C.c_double)]
            lib.orc_replay_cplx.argtypes = [vp, _dp, _dp, C.c_double, vp, vp, _dp, C.c_int]
            lib.orc_replay.argtypes = [vp, _dp, C.c_double, vp, _dp, C.c_int]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


ROS4, ROS3, RODAS3, RODAS4 = 0, 1, 2, 3  # the Rosenbrock methods of Table T:solvers
RKF45 = 4  # the explicit Runge-Kutta-Fehlberg 4(5) of the same table
ROS2W = 5  # the second-order W-method ROS2 (Verwer et al. 1999), used with Jacobian reuse
TABLEAUX = {"ROS4": ROS4, "ROS3": ROS3, "RODAS3": RODAS3, "RODAS4": RODAS4, "RKF45": RKF45}


def tableau(tab: int = ROS4) -> dict:
    """Transformed coefficients of a Rosenbrock method: s stages, a, c (s x s), m, e, gamma; for
    the explicit RKF45 (`explicit` true) a is the Butcher matrix, m and e the weights of the
    propagated solution and of the error estimate (c, gamma zero)."""
    out = np.zeros(88)
    _load().orc_tableau(int(tab), out)
    s = int(out[0])
    return {"s": s, "order": int(out[1]), "gamma": out[2],
            "a": out[3:39].reshape(6, 6)[:s, :s], "c": out[39:75].reshape(6, 6)[:s, :s],
            "m": out[75:81][:s], "e": out[81:87][:s], "explicit": bool(out[87])}


def step_linear(A, y, h, tab: int = ROS4):
    A = _f64(A)
    y = _f64(y)
    ynew = np.zeros_like(y)
    err = np.zeros_like(y)
    _load().orc_step_linear(len(y), A, y, h, ynew, err, int(tab))
    return ynew, err


def integrate_linear(A, y, dt, rtol, atol, tab: int = ROS4):
    A = _f64(A)
    y = _f64(y).copy()
    att = C.c_int(0)
    st = _load().orc_integrate_linear(len(y), A, y, dt, rtol, atol, C.byref(att), int(tab))
    return y, st, att.value


class Mechanism:
    """An oracle-side parsed mechanism (oracle.cpp's own spec reader)."""

    def __init__(self, path: str):
        lib = _load()
        self._lib = lib
        h = lib.orc_load(path.encode())
        if not h:
            raise RuntimeError(lib.orc_last_error().decode())
        self._h = h
        ns, nr, ne = C.c_int(), C.c_int(), C.c_int()
        lib.orc_info(h, C.byref(ns), C.byref(nr), C.byref(ne))
        self.ns, self.nr, self.ne = ns.value, nr.value, ne.value
        self.N = self.ns
        self.W = np.zeros(self.ns)
        self.elem = np.zeros(self.ne * self.ns, dtype=np.int32)
        self.Tmid = np.zeros(self.ns)
        self.hf_R = np.zeros(self.ns)
        self.s_R = np.zeros(self.ns)
        lib.orc_species(h, self.W, self.elem, self.Tmid, self.hf_R, self.s_R)
        self.elem = self.elem.reshape(self.ne, self.ns)
        self.kind = np.zeros(self.nr, dtype=np.int32)
        self.lnA = np.zeros(self.nr)
        nuf = np.zeros(self.nr * self.ns, dtype=np.int32)
        nur = np.zeros(self.nr * self.ns, dtype=np.int32)
        lib.orc_reactions(h, self.kind, self.lnA, nuf, nur)
        self.nu_f = nuf.reshape(self.nr, self.ns)
        self.nu_r = nur.reshape(self.nr, self.ns)

    def __del__(self):
        try:
            self._lib.orc_free(self._h)
        except Exception:
            pass

    # --------------------------------------------------------------------- conversions
    def state_from_TY(self, T, Y):
        """y = [T, Y_1/W_1, ..., Y_{Ns-1}/W_{Ns-1}] per cell (unit-mass basis)."""
        T = np.atleast_1d(np.asarray(T, dtype=np.float64))
        Y = np.atleast_2d(np.asarray(Y, dtype=np.float64))
        y = np.empty((len(T), self.ns))
        y[:, 0] = T
        y[:, 1:] = Y[:, :-1] / self.W[:-1]
        return y

    def TY_from_state(self, y):
        y = np.atleast_2d(y)
        Y = np.empty((y.shape[0], self.ns))
        Y[:, :-1] = y[:, 1:] * self.W[:-1]
        Y[:, -1] = 1.0 - Y[:, :-1].sum(axis=1)
        return y[:, 0].copy(), Y

    def moles_all(self, y):
        """All Ns species moles per kg, the bath gas closed by mass conservation."""
        y = np.atleast_2d(y)
        n = np.empty((y.shape[0], self.ns))
        n[:, :-1] = y[:, 1:]
        n[:, -1] = (1.0 - (y[:, 1:] * self.W[:-1]).sum(axis=1)) / self.W[-1]
        return n

    # --------------------------------------------------------------------- evaluation
    def thermo(self, k, T):
        cp, h, s = C.c_double(), C.c_double(), C.c_double()
        self._lib.orc_thermo(self._h, int(k), float(T), C.byref(cp), C.byref(h), C.byref(s))
        return cp.value, h.value, s.value

    def thermo_cplx(self, k, T):
        out = np.zeros(6)
        self._lib.orc_thermo_cplx(self._h, int(k), T.real, T.imag, out)
        return out[0] + 1j * out[1], out[2] + 1j * out[3], out[4] + 1j * out[5]

    def source(self, y, P, lnA=None):
        y = _f64(np.atleast_2d(y))
        P = _f64(np.broadcast_to(np.asarray(P, dtype=np.float64), (y.shape[0],)))
        lnA = None if lnA is None else _f64(lnA)
        f = np.zeros_like(y)
        self._lib.orc_source(self._h, y.shape[0], y, P, _ptr(lnA), f)
        return f

    def source_cplx(self, y, P, lnA=None):
        y = np.asarray(y, dtype=np.complex128)
        yr, yi = _f64(y.real), _f64(y.imag)
        fr = np.zeros(self.ns)
        fi = np.zeros(self.ns)
        if lnA is None:
            lr = li = None
        else:
            lnA = np.asarray(lnA, dtype=np.complex128)
            lr, li = _f64(lnA.real), _f64(lnA.imag)
        self._lib.orc_source_cplx(self._h, yr, _ptr(yi), float(P), _ptr(lr), _ptr(li), fr, fi)
        return fr + 1j * fi

    def jacobian(self, y, P, lnA=None, threads: int = 1):
        y = _f64(np.atleast_2d(y))
        P = _f64(np.broadcast_to(np.asarray(P, dtype=np.float64), (y.shape[0],)))
        lnA = None if lnA is None else _f64(lnA)
        J = np.zeros((y.shape[0], self.ns, self.ns))
        self._lib.orc_jacobian(self._h, y.shape[0], y, P, _ptr(lnA), J, threads)
        return J

    def rates(self, y, P, lnA=None):
        y = _f64(y)
        lnA = None if lnA is None else _f64(lnA)
        kf, kr, qf, qr = (np.zeros(self.nr) for _ in range(4))
        om, Cc = np.zeros(self.ns), np.zeros(self.ns)
        self._lib.orc_rates(self._h, y, float(P), _ptr(lnA), kf, kr, qf, qr, om, Cc)
        return {"kf": kf, "kr": kr, "qf": qf, "qr": qr, "omega": om, "C": Cc}

    def step(self, y, P, h, lnA=None, tableau=ROS4):
        y = _f64(y)
        lnA = None if lnA is None else _f64(lnA)
        ynew, err = np.zeros_like(y), np.zeros_like(y)
        self._lib.orc_step(self._h, y, float(P), _ptr(lnA), float(h), ynew, err, int(tableau))
        return ynew, err

    def integrate(self, y, P, dt, rtol=1e-6, atol=1e-10, h=None, lnA=None, max_steps=100000,
                  h_min=1e-20, T_min=0.0, fixed_steps=0, threads=None, tableau=ROS4):
        """Integrate every cell over [0, dt]; returns (y, info dict)."""
        y = _f64(np.atleast_2d(y)).copy()
        n = y.shape[0]
        P = _f64(np.broadcast_to(np.asarray(P, dtype=np.float64), (n,)))
        hh = np.zeros(n) if h is None else _f64(np.broadcast_to(h, (n,))).copy()
        st, att, acc, rej = (np.zeros(n, dtype=np.int32) for _ in range(4))
        lnA = None if lnA is None else _f64(lnA)
        threads = threads or os.cpu_count() or 1
        self._lib.orc_integrate(self._h, n, y, P, _ptr(lnA), dt, rtol, atol, _ptr(hh), _ptr(st),
                                _ptr(att), _ptr(acc), _ptr(rej), max_steps, h_min, T_min,
                                fixed_steps, threads, int(tableau))
        return y, {"h": hh, "status": st, "attempts": att, "accepted": acc, "rejected": rej}

    def integrate_auto(self, y, P, dt, method, rtol=1e-6, atol=1e-10, h=None, lnA=None,
                       max_steps=100000, T_min=0.0, threads: int = 1, tableau: int = ROS4,
                       alt: int = RKF45, cache=None):
        """Per-cell switching between the alternative method `alt` (RKF45, or ROS2W with `cache`
        from w_cache()) and the Rosenbrock method `tableau` (see orc_integrate_auto).
        method: int32 [C], updated in place.  Returns (y, info)."""
        y = _f64(np.atleast_2d(y)).copy()
        n = y.shape[0]
        P = _f64(np.broadcast_to(np.asarray(P, dtype=np.float64), (n,)))
        hh = np.zeros(n) if h is None else _f64(h).copy()
        st = np.zeros(n, dtype=np.int32)
        att = np.zeros(n, dtype=np.int32)
        assert method.dtype == np.int32 and method.flags["C_CONTIGUOUS"] and len(method) == n
        lnA = None if lnA is None else _f64(lnA)
        W, hW, age = cache if cache is not None else (None, None, None)
        if alt == ROS2W:
            assert cache is not None and W.shape == (n, self.N, self.N)
        self._lib.orc_integrate_auto(self._h, n, y, P, _ptr(lnA), dt, rtol, atol, _ptr(hh),
                                     _ptr(st), _ptr(att), method, max_steps, T_min, threads,
                                     tableau, alt, _ptr(W), _ptr(hW), _ptr(age))
        return y, {"status": st, "attempts": att, "h": hh}

    def w_cache(self, n):
        """An empty Jacobian cache of the W-method for n cells: (W [n, N, N], h_W [n], age [n])."""
        return (np.zeros((n, self.N, self.N)), np.zeros(n), np.zeros(n, dtype=np.int32))

    def integrate_w(self, y, P, dt, cache, rtol=1e-6, atol=1e-10, h=None, lnA=None,
                    max_steps=100000, threads: int = 1, tableau: int = ROS2W):
        """The W-method with Jacobian reuse (orc_integrate_w); cache from w_cache(), updated in
        place.  Returns (y, info) with info["n_jac"] the Jacobian evaluations per cell."""
        y = _f64(np.atleast_2d(y)).copy()
        n = y.shape[0]
        P = _f64(np.broadcast_to(np.asarray(P, dtype=np.float64), (n,)))
        hh = np.zeros(n) if h is None else _f64(h).copy()
        st, att, nj = (np.zeros(n, dtype=np.int32) for _ in range(3))
        W, hW, age = cache
        assert W.flags["C_CONTIGUOUS"] and W.shape == (n, self.N, self.N)
        lnA = None if lnA is None else _f64(lnA)
        self._lib.orc_integrate_w(self._h, n, y, P, _ptr(lnA), dt, rtol, atol, _ptr(hh), _ptr(st),
                                  _ptr(att), _ptr(nj), W.reshape(-1), hW, age, max_steps,
                                  threads, tableau)
        return y, {"status": st, "attempts": att, "h": hh, "n_jac": nj}

    def step_w(self, y, P, h, W, lnA=None, tableau: int = ROS2W):
        """One step of size h with the matrix W in place of the Jacobian: (y_new, error vector)."""
        yn, e = np.zeros(self.N), np.zeros(self.N)
        lnA = None if lnA is None else _f64(lnA)
        self._lib.orc_step_w(self._h, _f64(y), float(P), _ptr(lnA), h, _f64(W).reshape(-1), yn, e,
                             tableau)
        return yn, e

    def integrate_log(self, y, P, dt, rtol=1e-6, atol=1e-10, h0=0.0, lnA=None, max_steps=100000):
        y = _f64(y).copy()
        cap = max_steps + 1
        hs = np.zeros(cap)
        st, hout = C.c_int(), C.c_double()
        lnA = None if lnA is None else _f64(lnA)
        n = self._lib.orc_integrate_log(self._h, y, float(P), _ptr(lnA), dt, rtol, atol, h0,
                                        max_steps, hs, cap, C.byref(st), C.byref(hout))
        return y, hs[:n].copy(), st.value, hout.value

    def replay(self, y, P, hs, lnA=None):
        y = _f64(y).copy()
        lnA = None if lnA is None else _f64(lnA)
        self._lib.orc_replay(self._h, y, float(P), _ptr(lnA), _f64(hs), len(hs))
        return y

    def replay_cplx(self, y, P, hs, lnA=None):
        y = np.asarray(y, dtype=np.complex128)
        yr, yi = _f64(y.real).copy(), _f64(y.imag).copy()
        if lnA is None:
            lr = li = None
        else:
            lnA = np.asarray(lnA, dtype=np.complex128)
            lr, li = _f64(lnA.real), _f64(lnA.imag)
        self._lib.orc_replay_cplx(self._h, yr, yi, float(P), _ptr(lr), _ptr(li), _f64(hs),
                                  len(hs))
        return yr + 1j * yi
