"""Python binding of libheataco.so (the C ABI in include/heataco.h).

Argument marshalling only: every step of the decoder runs in the library's
CUDA kernels.  PyTorch supplies the device workspace and the stream.  There
is no CPU fallback: if the library is missing or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libheataco.so")

HAC_OK, HAC_EINVAL, HAC_ENOMEM, HAC_ECUDA, HAC_ETIMEOUT, HAC_EUNSUPPORTED, HAC_EBUSY = 0, -1, -2, -3, -4, -5, -6

FIELDS = dict(CAND=1, CDIST=2, CONF=3, BASE=4, EVID=5, W=6, TAU=7, CHOICE=8, NN_TOUR=9,
              GB_TOUR=10, IB_TOUR=11, TOURS=12, LENS=13, SCALARS=14, NBR=15, TRACE=16, FBL=17, FBL2=18)
SCALAR_KEYS = ("q90", "Rhat", "kappa", "p_x", "L_nn", "tau_max64", "tau_min64", "tau_max",
               "tau_min", "L_gb", "L_ib", "n_lambda", "t", "ib", "n_fallback", "k_pad", "L_rb", "n_restarts",
               "t_restart", "u_gb", "edges_per_n")


class HeatACOError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = _lib().hac_strerror(status).decode() if _LIB is not None else str(status)
        if status == HAC_ECUDA and _LIB is not None:
            msg += f" (cudaError {_LIB.hac_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [{status}]")


class hac_instance(C.Structure):
    _fields_ = [("n", C.c_int32), ("kind", C.c_int32), ("coords", C.c_void_p),
                ("cost", C.c_void_p), ("h_rowptr", C.c_void_p), ("h_col", C.c_void_p),
                ("h_val", C.c_void_p), ("h_nnz", C.c_int64), ("h_dtype", C.c_int32),
                ("symmetrize", C.c_int32)]


class hac_params(C.Structure):
    _fields_ = [("m", C.c_int32), ("k", C.c_int32), ("iterations", C.c_int32),
                ("alpha", C.c_double), ("beta", C.c_double), ("rho", C.c_double),
                ("theta_h", C.c_double), ("eps", C.c_double), ("c_cap", C.c_double),
                ("q_level", C.c_double), ("p_best", C.c_double), ("logw_clip", C.c_double),
                ("degree_target", C.c_int32), ("local_search", C.c_int32),
                ("baseline_scope", C.c_int32), ("ls_k", C.c_int32), ("schedule", C.c_int32),
                ("kappa_mode", C.c_int32), ("seed", C.c_uint64)]


class hac_exec(C.Structure):
    _fields_ = [("ants_per_warp", C.c_int32), ("warps_per_block", C.c_int32),
                ("use_graph", C.c_int32), ("fused", C.c_int32), ("fallback_list", C.c_int32),
                ("profile", C.c_int32), ("cluster_log2", C.c_int32), ("parts", C.c_int32)]


class hac_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("ant_steps", C.c_int64),
                ("fallback_steps", C.c_int64), ("kappa", C.c_double), ("edges_per_n", C.c_double),
                ("L_nn", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hac_server_cfg(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("iters_per_tick", C.c_int32), ("max_n", C.c_int32),
                ("steps_per_tick", C.c_int32), ("step_min_n", C.c_int32), ("step_ants_per_warp", C.c_int32),
                ("step_warps_per_block", C.c_int32), ("exec", hac_exec)]


_LIB = None

# every symbol include/heataco.h declares, with (restype, argtypes)
SIGNATURES = {
    "hac_version": (C.c_int, []),
    "hac_last_cuda_error": (C.c_int, []),
    "hac_strerror": (C.c_char_p, [C.c_int]),
    "hac_params_default": (C.c_int, [C.POINTER(hac_params), C.c_int32]),
    "hac_exec_default": (C.c_int, [C.POINTER(hac_exec)]),
    "hac_batch_workspace_size": (C.c_int, [C.POINTER(hac_instance), C.POINTER(hac_params), C.c_int32,
                                           C.c_int32, C.POINTER(C.c_size_t)]),
    "hac_batch_create": (C.c_int, [C.POINTER(hac_instance), C.POINTER(hac_params), C.c_int32, C.c_int32,
                                   C.c_void_p, C.c_size_t, C.POINTER(hac_exec), C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "hac_batch_iterate": (C.c_int, [C.c_void_p, C.c_int32]),
    "hac_batch_run": (C.c_int, [C.c_void_p]),
    "hac_batch_sync": (C.c_int, [C.c_void_p]),
    "hac_batch_read": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t]),
    "hac_batch_results": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.c_void_p]),
    "hac_batch_counters": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "hac_batch_destroy": (C.c_int, [C.c_void_p]),
    "hac_batch_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "hac_batch_kernel_time": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double),
                                        C.POINTER(C.c_int64)]),
    "hac_solve": (C.c_int, [C.POINTER(hac_instance), C.POINTER(hac_params), C.c_int32, C.c_void_p,
                            C.c_size_t, C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_void_p]),
    "hac_solve_batch": (C.c_int, [C.POINTER(hac_instance), C.POINTER(hac_params), C.c_int32, C.c_int32,
                                  C.c_void_p, C.c_size_t, C.POINTER(hac_exec), C.POINTER(C.c_void_p),
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hac_solve_noalloc": (C.c_int, [C.POINTER(hac_instance), C.POINTER(hac_params), C.c_int32,
                                    C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "hac_batch_autotune": (C.c_int, [C.POINTER(hac_instance), C.POINTER(hac_params), C.c_int32, C.c_int32,
                                     C.c_void_p, C.c_size_t, C.c_int32, C.c_void_p, C.POINTER(hac_exec),
                                     C.POINTER(C.c_double)]),
    "hac_server_request_bytes": (C.c_int, [C.POINTER(hac_instance), C.POINTER(hac_params),
                                           C.POINTER(C.c_size_t)]),
    "hac_server_create": (C.c_int, [C.POINTER(hac_server_cfg), C.c_void_p, C.c_size_t, C.c_void_p,
                                    C.POINTER(C.c_void_p)]),
    "hac_server_submit": (C.c_int, [C.c_void_p, C.POINTER(hac_instance), C.POINTER(hac_params),
                                    C.POINTER(C.c_uint64)]),
    "hac_server_tick": (C.c_int, [C.c_void_p]),
    "hac_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(C.c_double)]),
    "hac_server_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_size_t), C.POINTER(C.c_int32)]),
    "hac_server_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "hac_server_destroy": (C.c_int, [C.c_void_p]),
}


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise HeatACOError(HAC_EUNSUPPORTED, f"{LIB_PATH} is not built (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status, what):
    if status != HAC_OK:
        raise HeatACOError(status, what)


# ------------------------------------------------------------------ marshalling

def _np_ptr(a):
    return None if a is None else a.ctypes.data


class _Marshal:
    """Holds host (numpy) or device (torch) buffers for as long as the library may read them."""

    def __init__(self, instances, params, on_device: bool, pin: bool = False):
        self.keep = []
        n = len(instances)
        self.ins = (hac_instance * n)()
        self.ps = (hac_params * n)()
        for b, (inst, p) in enumerate(zip(instances, params)):
            self.ins[b] = self._instance(inst, on_device, pin)
            self.ps[b] = to_c_params(p)

    def _buf(self, a, dtype, on_device, pin):
        if a is None:
            return None
        if on_device:
            import torch
            t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a, dtype))
            t = t.to(device="cuda").contiguous()
            self.keep.append(t)
            return t.data_ptr()
        arr = np.ascontiguousarray(a, dtype)
        if pin:
            import torch
            t = torch.empty(arr.shape, dtype=torch.from_numpy(arr[:0]).dtype, pin_memory=True)
            t.numpy()[...] = arr
            self.keep.append(t)
            return t.data_ptr()
        self.keep.append(arr)
        return _np_ptr(arr)

    def _instance(self, inst, on_device, pin):
        half = str(inst.val.dtype).endswith("float16")
        nnz = int(len(inst.col))
        val = inst.val if nnz else np.zeros(1, np.float16 if half else np.float32)
        col = inst.col if nnz else np.zeros(1, np.int32)
        return hac_instance(
            inst.n, inst.kind,
            self._buf(inst.coords, np.float32, on_device, pin),
            self._buf(inst.cost, np.float32, on_device, pin),
            self._buf(inst.rowptr, np.int32, on_device, pin),
            self._buf(col, np.int32, on_device, pin),
            self._buf(val, np.float16 if half else np.float32, on_device, pin),
            nnz, 1 if half else 0, int(inst.symmetrize))


def to_c_params(p) -> hac_params:
    return hac_params(p.m, p.k, p.iterations, p.alpha, p.beta, p.rho, p.theta_h, p.eps, p.c_cap,
                      p.q_level, p.p_best, p.logw_clip, p.degree_target, p.local_search,
                      p.baseline_scope, p.ls_k, getattr(p, "schedule", 0), getattr(p, "kappa_mode", 0), p.seed)


def make_exec(ants_per_warp=0, warps_per_block=0, use_graph=1, fused=0, fallback_list=0, profile=0,
              cluster_log2=0, parts=0):
    return hac_exec(ants_per_warp, warps_per_block, use_graph, fused, fallback_list, profile, cluster_log2, parts)


# ------------------------------------------------------------------ C-named calls

def hac_version():
    return _lib().hac_version()


def hac_params_default(kind: int) -> hac_params:
    p = hac_params()
    _check(_lib().hac_params_default(C.byref(p), kind), "hac_params_default")
    return p


def hac_batch_workspace_size(instances, params, inputs_on_device=False) -> int:
    m = _Marshal(instances, params, inputs_on_device)
    out = C.c_size_t(0)
    _check(_lib().hac_batch_workspace_size(m.ins, m.ps, len(instances), int(inputs_on_device),
                                           C.byref(out)), "hac_batch_workspace_size")
    return out.value


class Batch:
    """A resident batch of instances (hac_batch_* calls)."""

    def __init__(self, instances, params, exec_=None, inputs_on_device=False, stream=None,
                 pin=False, workspace=None):
        import torch
        if not torch.cuda.is_available():
            raise HeatACOError(HAC_ECUDA, "no CUDA device")
        self.instances = list(instances)
        self.params = list(params)
        self.count = len(self.instances)
        self._m = _Marshal(self.instances, self.params, inputs_on_device, pin)
        size = C.c_size_t(0)
        _check(_lib().hac_batch_workspace_size(self._m.ins, self._m.ps, self.count, int(inputs_on_device),
                                               C.byref(size)), "hac_batch_workspace_size")
        self.ws_bytes = size.value
        if workspace is None or workspace.numel() < self.ws_bytes:
            workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.exec = exec_ if exec_ is not None else make_exec()
        h = C.c_void_p()
        _check(_lib().hac_batch_create(self._m.ins, self._m.ps, self.count, int(inputs_on_device),
                                       C.c_void_p(workspace.data_ptr()), C.c_size_t(workspace.numel()),
                                       C.byref(self.exec), C.c_void_p(self.stream.cuda_stream),
                                       C.byref(h)), "hac_batch_create")
        self.h = h

    # lifecycle ------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.stream.synchronize()
            _lib().hac_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # calls ----------------------------------------------------------------
    def iterate(self, iters: int):
        _check(_lib().hac_batch_iterate(self.h, iters), "hac_batch_iterate")
        return self

    def run(self):
        _check(_lib().hac_batch_run(self.h), "hac_batch_run")
        return self

    def sync(self):
        _check(_lib().hac_batch_sync(self.h), "hac_batch_sync")
        return self

    def _shape(self, b, field):
        inst, p = self.instances[b], self.params[b]
        n, kp, m = inst.n, 4 * ((p.k + 3) // 4), p.m
        return {
            "CAND": (np.int32, (n, kp)), "CDIST": (np.float64, (n, kp)), "CONF": (np.float64, (n, kp)),
            "BASE": (np.float64, (n,)), "EVID": (np.float64, (n, kp)), "W": (np.float32, (n, kp)),
            "TAU": (np.float32, (n, kp)), "CHOICE": (np.float32, (n, kp)),
            "NN_TOUR": (np.int32, (n,)), "GB_TOUR": (np.int32, (n,)), "IB_TOUR": (np.int32, (n,)),
            "TOURS": (np.int32, (m, n)), "LENS": (np.float64, (m,)),
            "SCALARS": (np.float64, (21,)), "NBR": (np.int32, (n, p.ls_k)),
            "TRACE": (np.float64, (max(p.iterations, 1), 5)),
            "FBL": (np.int32, (n, 32)), "FBL2": (np.uint16, (n, 256)),
        }[field]

    def read(self, b: int, field: str):
        dt, shp = self._shape(b, field)
        out = np.empty(shp, dt)
        _check(_lib().hac_batch_read(self.h, b, FIELDS[field], out.ctypes.data, out.nbytes),
               f"hac_batch_read({field})")
        return out

    def scalars(self, b: int) -> dict:
        v = self.read(b, "SCALARS")
        return dict(zip(SCALAR_KEYS, v.tolist()))

    def results(self, pinned_out=None):
        tours = pinned_out if pinned_out is not None else [np.empty(i.n, np.int32) for i in self.instances]
        ptrs = (C.c_void_p * self.count)(*[t.ctypes.data if isinstance(t, np.ndarray) else t.data_ptr()
                                           for t in tours])
        lens = np.empty(self.count, np.float64)
        _check(_lib().hac_batch_results(self.h, ptrs, lens.ctypes.data), "hac_batch_results")
        return tours, lens

    def counters(self):
        a, f = C.c_int64(0), C.c_int64(0)
        _check(_lib().hac_batch_counters(self.h, C.byref(a), C.byref(f)), "hac_batch_counters")
        return a.value, f.value

    def launches(self) -> int:
        v = C.c_int64(0)
        _check(_lib().hac_batch_launches(self.h, C.byref(v)), "hac_batch_launches")
        return v.value

    def kernel_time(self, group: int):
        """(ms, launches) of kernel group 0 construction, 1 iteration tail, 2 preparation,
        3 fused iterations."""
        ms, k = C.c_double(0), C.c_int64(0)
        _check(_lib().hac_batch_kernel_time(self.h, group, C.byref(ms), C.byref(k)), "hac_batch_kernel_time")
        return ms.value, k.value


def autotune(instances, params, trial_iters=10, inputs_on_device=False, stream=None, workspace=None):
    """(best hac_exec, ms per iteration) from hac_batch_autotune."""
    import torch
    m = _Marshal(instances, params, inputs_on_device)
    size = C.c_size_t(0)
    _check(_lib().hac_batch_workspace_size(m.ins, m.ps, len(instances), int(inputs_on_device), C.byref(size)),
           "hac_batch_workspace_size")
    if workspace is None or workspace.numel() < size.value:
        workspace = torch.empty(size.value, dtype=torch.uint8, device="cuda")
    stream = stream if stream is not None else torch.cuda.Stream()
    best, ms = hac_exec(), C.c_double(0)
    _check(_lib().hac_batch_autotune(m.ins, m.ps, len(instances), int(inputs_on_device),
                                     C.c_void_p(workspace.data_ptr()), C.c_size_t(workspace.numel()),
                                     trial_iters, C.c_void_p(stream.cuda_stream), C.byref(best), C.byref(ms)),
           "hac_batch_autotune")
    return best, ms.value


def solve_batch(instances, params, exec_=None, inputs_on_device=False):
    with Batch(instances, params, exec_, inputs_on_device) as bt:
        bt.run()
        return bt.results()


def solve(instance, params, exec_=None):
    tours, lens = solve_batch([instance], [params], exec_)
    return tours[0], float(lens[0])


def hac_solve(instance, params, stream=None):
    """hac_solve with host inputs and no workspace (the library takes one from
    the stream-ordered pool for the call): (T_gb, L_gb, stats dict)."""
    m = _Marshal([instance], [params], False)
    tour = np.empty(instance.n, np.int32)
    length = C.c_double(0.0)
    st = hac_stats()
    _check(_lib().hac_solve(m.ins, m.ps, 0, None, 0, tour.ctypes.data, C.byref(length), C.byref(st),
                            None if stream is None else C.c_void_p(stream)), "hac_solve")
    return tour, length.value, st.as_dict()


# ------------------------------------------------------------------ serving

def hac_server_request_bytes(instance, params) -> int:
    m = _Marshal([instance], [params], False)
    out = C.c_size_t(0)
    _check(_lib().hac_server_request_bytes(m.ins, m.ps, C.byref(out)), "hac_server_request_bytes")
    return out.value


class Server:
    """Continuous-batching decode server (hac_server_* calls) on a device workspace
    of `ws_bytes` bytes (a uint8 torch tensor)."""

    def __init__(self, ws_bytes: int, max_slots: int = 64, iters_per_tick: int = 10, max_n: int = 10000,
                 exec_=None, stream=None, workspace=None, steps_per_tick: int = 0, step_min_n: int = 0,
                 step_ants_per_warp: int = 1, step_warps_per_block: int = 8):
        import torch
        if not torch.cuda.is_available():
            raise HeatACOError(HAC_ECUDA, "no CUDA device")
        if workspace is None or workspace.numel() < ws_bytes:
            workspace = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.cfg = hac_server_cfg(max_slots, iters_per_tick, max_n, steps_per_tick, step_min_n,
                                  step_ants_per_warp, step_warps_per_block,
                                  exec_ if exec_ is not None else make_exec(fused=1))
        self.sizes = {}
        h = C.c_void_p()
        _check(_lib().hac_server_create(C.byref(self.cfg), C.c_void_p(workspace.data_ptr()),
                                        C.c_size_t(workspace.numel()), C.c_void_p(self.stream.cuda_stream),
                                        C.byref(h)), "hac_server_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib().hac_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, instance, params):
        """Ticket (int > 0), or None when no slot or memory is free (HAC_EBUSY)."""
        m = _Marshal([instance], [params], False)
        t = C.c_uint64(0)
        st = _lib().hac_server_submit(self.h, m.ins, m.ps, C.byref(t))
        if st == HAC_EBUSY:
            return None
        _check(st, "hac_server_submit")
        self.sizes[t.value] = instance.n
        return t.value

    def tick(self):
        _check(_lib().hac_server_tick(self.h), "hac_server_tick")

    def poll(self, ticket: int):
        """(tour, length) once finished, else None."""
        n = self.sizes.get(ticket)
        tour = np.empty(n if n is not None else 0, np.int32)
        ln = C.c_double(0)
        st = _lib().hac_server_poll(self.h, ticket, tour.ctypes.data if n is not None else None, C.byref(ln))
        if st == HAC_EBUSY:
            return None
        _check(st, "hac_server_poll")
        del self.sizes[ticket]
        return tour, ln.value

    def stats(self, device_error: bool = False) -> dict:
        r, f, fb, de = C.c_int32(0), C.c_int32(0), C.c_size_t(0), C.c_int32(0)
        _check(_lib().hac_server_stats(self.h, C.byref(r), C.byref(f), C.byref(fb),
                                       C.byref(de) if device_error else None), "hac_server_stats")
        out = dict(resident=r.value, finished=f.value, free_bytes=fb.value)
        if device_error:
            out["device_error"] = de.value
        return out

    def launches(self) -> int:
        v = C.c_int64(0)
        _check(_lib().hac_server_launches(self.h, C.byref(v)), "hac_server_launches")
        return v.value
