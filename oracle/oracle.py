"""ctypes front end of the C oracle (heataco_oracle.c) -- test infrastructure only.

The oracle is a plain sequential restatement of the decoder of arXiv
2601.19041 (Sec. III, Algorithms 1 and 2).  This module only builds it with
gcc, marshals numpy arrays into its structs and reads its state back; all the
arithmetic lives in the C file.  Every oracle function is pinned to something
other than itself; the pins are listed in the C file's header and live in
tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "heataco_oracle.c")
LIB = os.path.join(HERE, "liborc.so")

# -O2 without fast-math and without FMA contraction: every FP operation in the
# source is one IEEE operation on both x86-64 and aarch64.
CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fno-math-errno",
          "-fPIC", "-shared", "-Wall", "-Wextra", "-Wno-unused-parameter", "-Wno-stringop-overflow"]


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


class _Inst(C.Structure):
    _fields_ = [("n", C.c_int32), ("kind", C.c_int32), ("coords", C.c_void_p),
                ("cost", C.c_void_p), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("val_is_half", C.c_int32), ("symmetrize", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("m", C.c_int32), ("k", C.c_int32), ("iterations", C.c_int32),
                ("alpha", C.c_double), ("beta", C.c_double), ("rho", C.c_double),
                ("theta_h", C.c_double), ("eps", C.c_double), ("c_cap", C.c_double),
                ("q_level", C.c_double), ("p_best", C.c_double), ("logw_clip", C.c_double),
                ("degree_target", C.c_int32), ("local_search", C.c_int32),
                ("baseline_scope", C.c_int32), ("ls_k", C.c_int32), ("schedule", C.c_int32),
                ("kappa_mode", C.c_int32), ("seed", C.c_uint64)]


F = dict(cand=1, cdist=2, conf=3, base=4, evid=5, logev=6, W=7, tau=8, choice=9,
         nn_tour=10, gb_tour=11, tours=12, lens=13, ib_tour=14, trace_ib=15,
         trace_Lib=16, trace_Lgb=17, nbr=18, scalars=19, ints=20, rb_tour=21, trace_Lrb=22,
         trace_code=23)

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
        L.orc_draw.restype = C.c_uint32
        L.orc_exp.argtypes = [C.c_double]; L.orc_exp.restype = C.c_double
        L.orc_ln.argtypes = [C.c_double]; L.orc_ln.restype = C.c_double
        L.orc_roulette.argtypes = [C.c_void_p, C.c_int, C.c_float]; L.orc_roulette.restype = C.c_int
        L.orc_quantile7.argtypes = [C.c_void_p, C.c_int64, C.c_double]
        L.orc_quantile7.restype = C.c_double
        L.orc_create.argtypes = [C.POINTER(_Inst), C.POINTER(_Params), C.POINTER(C.c_int32)]
        L.orc_create.restype = C.c_void_p
        L.orc_iterate.argtypes = [C.c_void_p, C.c_int32]
        L.orc_get.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_two_opt.argtypes = [C.POINTER(_Inst), C.c_void_p, C.c_int, C.c_void_p]
        L.orc_three_opt.argtypes = [C.POINTER(_Inst), C.c_void_p, C.c_int, C.c_void_p]
        L.orc_two_opt_directed.argtypes = [C.POINTER(_Inst), C.c_void_p, C.c_int, C.c_void_p]
        L.orc_tour_length.argtypes = [C.POINTER(_Inst), C.c_void_p]
        L.orc_tour_length.restype = C.c_double
        L.orc_dist.argtypes = [C.POINTER(_Inst), C.c_int, C.c_int]; L.orc_dist.restype = C.c_double
        L.orc_key.argtypes = [C.POINTER(_Inst), C.c_int, C.c_int]; L.orc_key.restype = C.c_float
        L.orc_heat.argtypes = [C.POINTER(_Inst), C.c_int, C.c_int]; L.orc_heat.restype = C.c_double
        L.orc_ugb.argtypes = [C.c_int32]; L.orc_ugb.restype = C.c_int
        L.orc_branching.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int]
        L.orc_branching.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class _InstHolder:
    """Keeps the numpy buffers alive for as long as the C struct points at them."""

    def __init__(self, inst):
        self.coords = None if inst.coords is None else np.ascontiguousarray(inst.coords, np.float32)
        self.cost = None if inst.cost is None else np.ascontiguousarray(inst.cost, np.float32)
        self.rowptr = np.ascontiguousarray(inst.rowptr, np.int32)
        self.col = np.ascontiguousarray(inst.col, np.int32)
        half = inst.val.dtype == np.float16
        self.val = np.ascontiguousarray(inst.val, np.float16 if half else np.float32)
        if not self.val.size:          # an empty heatmap still needs valid pointers
            self.col = np.zeros(1, np.int32)
            self.val = np.zeros(1, np.float16 if half else np.float32)
        self.s = _Inst(inst.n, inst.kind, _ptr(self.coords), _ptr(self.cost), _ptr(self.rowptr),
                       _ptr(self.col), _ptr(self.val), int(half), int(inst.symmetrize))


def _params(p) -> _Params:
    return _Params(p.m, p.k, p.iterations, p.alpha, p.beta, p.rho, p.theta_h, p.eps, p.c_cap,
                   p.q_level, p.p_best, p.logw_clip, p.degree_target, p.local_search,
                   p.baseline_scope, p.ls_k, getattr(p, "schedule", 0), getattr(p, "kappa_mode", 0), p.seed)


class Oracle:
    """One decode run on the CPU: preparation on construction, then ``iterate``."""

    def __init__(self, inst, params):
        self._inst = _InstHolder(inst)
        self._p = _params(params)
        st = C.c_int32(0)
        self.h = lib().orc_create(C.byref(self._inst.s), C.byref(self._p), C.byref(st))
        if not self.h:
            raise ValueError(f"oracle rejected the instance (status {st.value})")
        ints = self._get_raw("ints", np.int64, 10)
        self.n, self.k_eff, self.k_pad = int(ints[0]), int(ints[1]), int(ints[2])
        self.m = params.m
        self.ls_k = int(ints[5])
        self.iterations = params.iterations

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def _get_raw(self, field, dtype, count):
        out = np.empty(count, dtype)
        r = lib().orc_get(self.h, F[field], out.ctypes.data, out.nbytes)
        if r < 0:
            raise RuntimeError(f"orc_get({field}) failed")
        return out

    def iterate(self, iters: int):
        if lib().orc_iterate(self.h, iters) != 0:
            raise RuntimeError("orc_iterate failed")
        return self

    def get(self, field):
        n, kp, m = self.n, self.k_pad, self.m
        shapes = dict(cand=(np.int32, (n, kp)), cdist=(np.float64, (n, kp)),
                      conf=(np.float64, (n, kp)), base=(np.float64, (n,)),
                      evid=(np.float64, (n, kp)), logev=(np.float64, (n, kp)),
                      W=(np.float32, (n, kp)), tau=(np.float32, (n, kp)),
                      choice=(np.float32, (n, kp)), nn_tour=(np.int32, (n,)),
                      gb_tour=(np.int32, (n,)), tours=(np.int32, (m, n)),
                      lens=(np.float64, (m,)), ib_tour=(np.int32, (n,)),
                      trace_ib=(np.int32, (max(self.iterations, 1),)),
                      trace_Lib=(np.float64, (max(self.iterations, 1),)),
                      trace_Lgb=(np.float64, (max(self.iterations, 1),)),
                      trace_Lrb=(np.float64, (max(self.iterations, 1),)),
                      trace_code=(np.int32, (max(self.iterations, 1),)),
                      rb_tour=(np.int32, (n,)),
                      nbr=(np.int32, (n, max(self.ls_k, 1))))
        dt, shp = shapes[field]
        return self._get_raw(field, dt, int(np.prod(shp))).reshape(shp)

    def scalars(self) -> dict:
        s = self._get_raw("scalars", np.float64, 14)
        keys = ("q90", "Rhat", "kappa", "p_x", "L_nn", "tau_max64", "tau_min64", "tau_max",
                "tau_min", "L_gb", "L_ib", "n_lambda", "L_rb", "edges_per_n")
        return dict(zip(keys, s.tolist()))

    def ints(self) -> dict:
        v = self._get_raw("ints", np.int64, 10)
        return dict(zip(("n", "k_eff", "k_pad", "t", "n_fallback", "ls_k", "n_restarts", "t_restart",
                         "t_rbimp", "u_gb"), v.tolist()))


def solve(inst, params):
    """Full decode: (best tour, best length, oracle handle)."""
    o = Oracle(inst, params).iterate(params.iterations)
    return o.get("gb_tour"), o.scalars()["L_gb"], o


# ------------------------------------------------------------------ small helpers

def philox(ctr, key):
    c = np.asarray(ctr, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def draw(seed, t, a, s):
    return int(lib().orc_draw(seed, t, a, s))


def exp(x):
    return lib().orc_exp(float(x))


def ln(x):
    return lib().orc_ln(float(x))


def roulette(w, u):
    w = np.ascontiguousarray(w, np.float32)
    return lib().orc_roulette(w.ctypes.data, len(w), C.c_float(u))


def quantile7(x_sorted, q):
    x = np.ascontiguousarray(x_sorted, np.float64)
    return lib().orc_quantile7(x.ctypes.data, len(x), q)


def two_opt(inst, nbr, tour):
    h = _InstHolder(inst)
    nb = np.ascontiguousarray(nbr, np.int32)
    t = np.ascontiguousarray(tour, np.int32).copy()
    moves = lib().orc_two_opt(C.byref(h.s), nb.ctypes.data, nb.shape[1], t.ctypes.data)
    return t, moves


def two_opt_directed(inst, nbr, tour):
    h = _InstHolder(inst)
    nb = np.ascontiguousarray(nbr, np.int32)
    t = np.ascontiguousarray(tour, np.int32).copy()
    moves = lib().orc_two_opt_directed(C.byref(h.s), nb.ctypes.data, nb.shape[1], t.ctypes.data)
    return t, moves


def three_opt(inst, nbr, tour):
    h = _InstHolder(inst)
    nb = np.ascontiguousarray(nbr, np.int32)
    t = np.ascontiguousarray(tour, np.int32).copy()
    moves = lib().orc_three_opt(C.byref(h.s), nb.ctypes.data, nb.shape[1], t.ctypes.data)
    return t, moves


def tour_length(inst, tour):
    h = _InstHolder(inst)
    t = np.ascontiguousarray(tour, np.int32)
    return lib().orc_tour_length(C.byref(h.s), t.ctypes.data)


def dist(inst, i, j):
    h = _InstHolder(inst)
    return lib().orc_dist(C.byref(h.s), i, j)


def heat(inst, i, j):
    h = _InstHolder(inst)
    return lib().orc_heat(C.byref(h.s), i, j)


def ugb(s):
    return int(lib().orc_ugb(int(s)))


def branching(tau, cand, dstar):
    tau = np.ascontiguousarray(tau, np.float32)
    cand = np.ascontiguousarray(cand, np.int32)
    n, kp = tau.shape
    return lib().orc_branching(tau.ctypes.data, cand.ctypes.data, n, kp, int(dstar))
