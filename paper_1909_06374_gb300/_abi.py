"""ctypes binding of the C ABI in include/agnlc.h (argument marshalling only).

Every function keeps the C name and argument order; pointers may be given as
ints, torch tensors (their data_ptr) or numpy arrays; streams as ints,
torch.cuda.Stream objects or None (legacy default stream).  A non-OK status
raises LcError carrying the status and lc_last_error(), except where a
function documents LC_PENDING as a normal result.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_d, c_u32, c_u64, c_i32, c_sz, c_p = (ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_int32, ctypes.c_size_t, ctypes.c_void_p)

LC_OK, LC_PENDING = 0, 1
LC_ERR_INVALID, LC_ERR_NOMEM, LC_ERR_CUDA, LC_ERR_TIMEOUT, LC_ERR_BUSY, LC_ERR_UNKNOWN_TICKET = \
    -1, -2, -3, -4, -5, -6
LC_FP32, LC_FP64 = 0, 1


LC_TK_GAUSSIAN, LC_TK_FIXED_AMPLITUDE = 0, 1
LC_TARGETS_REALISED, LC_TARGETS_PSD = 0, 1


class LcPsd(ctypes.Structure):
    _fields_ = [("f_br", c_d), ("alpha_low", c_d), ("alpha_high", c_d), ("coeffs", c_i32), ("targets", c_i32)]


LC_ERDF_SHARP, LC_ERDF_SMOOTH, LC_ERDF_LOGNORMAL = 0, 1, 2


class LcErdf(ctypes.Structure):
    _fields_ = [("log_lmin", c_d), ("log_lmax", c_d), ("log_lbreak", c_d), ("slope_low", c_d),
                ("slope_high", c_d), ("linear_space", c_i32), ("kind", c_i32), ("sigma", c_d)]


class LcJob(ctypes.Structure):
    _fields_ = [("log2n", c_u32), ("iters", c_u32), ("dt", c_d), ("psd", LcPsd), ("erdf", LcErdf),
                ("seed", c_u64), ("curve_id", c_u64)]


class LcError(RuntimeError):
    def __init__(self, status, fn, msg):
        super().__init__(f"{fn}: {status_name(status)} ({status}): {msg}")
        self.status = status


_SIGS = {
    "lc_status_string": (ctypes.c_char_p, [c_i32]),
    "lc_last_error": (ctypes.c_char_p, []),
    "lc_plan_create": (c_i32, [ctypes.POINTER(LcJob), c_sz, c_i32, c_i32, ctypes.POINTER(c_p)]),
    "lc_plan_workspace_bytes": (c_i32, [c_p, ctypes.POINTER(c_sz)]),
    "lc_plan_total_samples": (c_i32, [c_p, ctypes.POINTER(c_sz)]),
    "lc_generate": (c_i32, [c_p, c_p, c_p, c_p]),
    "lc_generate_host": (c_i32, [c_p, c_p, c_p, c_p]),
    "lc_setup": (c_i32, [c_p, c_p, c_p]),
    "lc_iterate": (c_i32, [c_p, c_u32, c_p]),
    "lc_get_state": (c_i32, [c_p, c_p, c_p]),
    "lc_set_state": (c_i32, [c_p, c_p, c_p]),
    "lc_rank_replace": (c_i32, [c_p, c_p, c_p, c_p]),
    "lc_plan_buffer": (c_i32, [c_p, c_i32, ctypes.POINTER(c_p), ctypes.POINTER(c_sz)]),
    "lc_plan_last_launches": (c_i32, [c_p, ctypes.POINTER(c_u64)]),
    "lc_plan_timing": (c_i32, [c_p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "lc_plan_set_convergence": (c_i32, [c_p, c_p, c_u32]),
    "lc_plan_convergence": (c_i32, [c_p, c_p, c_p]),
    "lc_periodogram": (c_i32, [c_p, c_p, c_i32, c_p, c_p]),
    "lc_structure_function": (c_i32, [c_p, c_p, c_p, c_sz, c_p, c_p]),
    "lc_plan_profile": (c_i32, [c_p, c_p, c_sz, c_p]),
    "lc_plan_destroy": (c_i32, [c_p]),
    "lc_generate_noalloc": (c_i32, [ctypes.POINTER(LcJob), c_p, c_p]),
    "lc_server_create": (c_i32, [c_i32, c_sz, c_i32, ctypes.POINTER(c_p)]),
    "lc_submit": (c_i32, [c_p, ctypes.POINTER(LcJob), ctypes.POINTER(c_u64)]),
    "lc_poll": (c_i32, [c_p, c_u64, c_p, ctypes.POINTER(c_u64)]),
    "lc_server_stats": (c_i32, [c_p, ctypes.POINTER(c_u64), ctypes.POINTER(c_u64), ctypes.POINTER(c_u64)]),
    "lc_server_destroy": (c_i32, [c_p]),
    "lc_server_trace": (c_i32, [c_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(c_u64), ctypes.POINTER(c_u64)]),
    "lc_plan_footprint": (c_i32, [ctypes.POINTER(LcJob), c_sz, c_i32, ctypes.POINTER(c_sz)]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load the CUDA library, compiling it first if it is missing or stale.
    There is no fallback: without the library every call fails."""
    global _lib
    with _lock:
        if _lib is None:
            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("CUDA library missing: " + _build.LIB)
            L = ctypes.CDLL(_build.LIB, mode=ctypes.RTLD_LOCAL)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_name(status: int) -> str:
    return load().lc_status_string(status).decode()


def last_error() -> str:
    return load().lc_last_error().decode()


def _check(status, fn, allow=(LC_OK,)):
    if status not in allow:
        raise LcError(status, fn, last_error())
    return status


def ptr(x):
    """Raw address of a tensor / array / int (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return c_p(x)
    if hasattr(x, "data_ptr"):
        return c_p(x.data_ptr())
    if hasattr(x, "ctypes"):
        return c_p(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_ptr(s):
    if s is None:
        return None
    if isinstance(s, int):
        return c_p(s)
    return c_p(s.cuda_stream)


def make_job(j) -> LcJob:
    """LcJob from a job dict (keys as in workloads.job)."""
    return LcJob(int(j["log2n"]), int(j["iters"]), float(j["dt"]),
                 LcPsd(float(j["f_br"]), float(j["alpha_low"]), float(j["alpha_high"]), int(j.get("tk_coeffs", 0)),
                       int(j.get("tk_targets", 0))),
                 LcErdf(float(j["log_lmin"]), float(j["log_lmax"]), float(j["log_lbreak"]),
                        float(j["slope_low"]), float(j["slope_high"]), int(j.get("linear_space", 0)),
                        int(j.get("erdf_kind", 0)), float(j.get("sigma", 0.0))),
                 int(j["seed"]), int(j["curve_id"]))


def job_array(jobs):
    arr = (LcJob * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = j if isinstance(j, LcJob) else make_job(j)
    return arr


# ------------------------------------------------------------- entry points
def lc_plan_create(jobs, prec=LC_FP32, device=0):
    arr = job_array(jobs)
    out = c_p()
    _check(load().lc_plan_create(arr, len(jobs), int(prec), int(device), ctypes.byref(out)), "lc_plan_create")
    return out


def lc_plan_workspace_bytes(plan):
    v = c_sz()
    _check(load().lc_plan_workspace_bytes(plan, ctypes.byref(v)), "lc_plan_workspace_bytes")
    return v.value


def lc_plan_total_samples(plan):
    v = c_sz()
    _check(load().lc_plan_total_samples(plan, ctypes.byref(v)), "lc_plan_total_samples")
    return v.value


def lc_generate(plan, out_x, out_tk=None, stream=None):
    _check(load().lc_generate(plan, ptr(out_x), ptr(out_tk), stream_ptr(stream)), "lc_generate")


def lc_generate_host(plan, out_x_host, out_tk_host=None, stream=None):
    _check(load().lc_generate_host(plan, ptr(out_x_host), ptr(out_tk_host), stream_ptr(stream)),
           "lc_generate_host")


def lc_setup(plan, out_tk=None, stream=None):
    _check(load().lc_setup(plan, ptr(out_tk), stream_ptr(stream)), "lc_setup")


def lc_iterate(plan, iters=0, stream=None):
    _check(load().lc_iterate(plan, int(iters), stream_ptr(stream)), "lc_iterate")


def lc_get_state(plan, out_x, stream=None):
    _check(load().lc_get_state(plan, ptr(out_x), stream_ptr(stream)), "lc_get_state")


def lc_set_state(plan, in_x, stream=None):
    _check(load().lc_set_state(plan, ptr(in_x), stream_ptr(stream)), "lc_set_state")


def lc_rank_replace(plan, x_adj, out_x, stream=None):
    _check(load().lc_rank_replace(plan, ptr(x_adj), ptr(out_x), stream_ptr(stream)), "lc_rank_replace")


def lc_plan_buffer(plan, which):
    p, n = c_p(), c_sz()
    _check(load().lc_plan_buffer(plan, int(which), ctypes.byref(p), ctypes.byref(n)), "lc_plan_buffer")
    return p.value, n.value


def lc_plan_last_launches(plan):
    v = c_u64()
    _check(load().lc_plan_last_launches(plan, ctypes.byref(v)), "lc_plan_last_launches")
    return v.value


def lc_plan_timing(plan):
    """(setup_ms, iterate_ms) of the last run, from CUDA events on the plan's stream."""
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(load().lc_plan_timing(plan, ctypes.byref(a), ctypes.byref(b)), "lc_plan_timing")
    return a.value, b.value


def lc_plan_set_convergence(plan, thresholds, history):
    """thresholds: None or a sequence of ncurves floats (host)."""
    import numpy as np
    if thresholds is None:
        _check(load().lc_plan_set_convergence(plan, None, int(history)), "lc_plan_set_convergence")
        return
    t = np.ascontiguousarray(thresholds, dtype=np.float64)
    _check(load().lc_plan_set_convergence(plan, t.ctypes.data_as(c_p), int(history)), "lc_plan_set_convergence")


def lc_plan_convergence(plan, ncurves, history):
    """(deltas [ncurves, history] float64, iters_run [ncurves] uint32) of the last run."""
    import numpy as np
    d = np.empty((ncurves, history), dtype=np.float64)
    r = np.empty(ncurves, dtype=np.uint32)
    _check(load().lc_plan_convergence(plan, d.ctypes.data_as(c_p), r.ctypes.data_as(c_p)), "lc_plan_convergence")
    return d, r


def lc_periodogram(plan, x, rms, out_p, stream=None):
    _check(load().lc_periodogram(plan, ptr(x), int(bool(rms)), ptr(out_p), stream_ptr(stream)), "lc_periodogram")


def lc_structure_function(plan, x, lags, out_sf2, stream=None):
    import numpy as np
    L = np.ascontiguousarray(lags, dtype=np.uint32)
    _check(load().lc_structure_function(plan, ptr(x), L.ctypes.data_as(c_p), L.size, ptr(out_sf2),
                                        stream_ptr(stream)), "lc_structure_function")


def lc_plan_profile(plan):
    """Per-group device ms of one extra iteration (see agnlc.h) as a dict."""
    ms = (ctypes.c_float * 5)()
    cnt = (c_u64 * 4)()
    _check(load().lc_plan_profile(plan, ms, 5, cnt), "lc_plan_profile")
    names = ("fft", "sort_hist_scan", "sort_scatter", "resident", "convergence")
    out = {n: float(v) for n, v in zip(names, ms)}
    out["scatter_launches"], out["sorted_elements"], out["fused_elements"] = int(cnt[0]), int(cnt[1]), int(cnt[2])
    out["bucket_elements"] = int(cnt[3])
    return out


def lc_plan_destroy(plan):
    _check(load().lc_plan_destroy(plan), "lc_plan_destroy")


def lc_generate_noalloc(job, out_x, stream=None):
    j = job if isinstance(job, LcJob) else make_job(job)
    _check(load().lc_generate_noalloc(ctypes.byref(j), ptr(out_x), stream_ptr(stream)), "lc_generate_noalloc")


def lc_server_create(device=0, hbm_budget_bytes=0, prec=LC_FP32):
    out = c_p()
    _check(load().lc_server_create(int(device), int(hbm_budget_bytes), int(prec), ctypes.byref(out)),
           "lc_server_create")
    return out


def lc_submit(server, job):
    t = c_u64()
    j = job if isinstance(job, LcJob) else make_job(job)
    _check(load().lc_submit(server, ctypes.byref(j), ctypes.byref(t)), "lc_submit")
    return t.value


def lc_poll(server, ticket, out_host=None):
    """Returns (status, latency_ns); status LC_PENDING or LC_OK."""
    lat = c_u64()
    s = load().lc_poll(server, c_u64(ticket), ptr(out_host), ctypes.byref(lat))
    _check(s, "lc_poll", allow=(LC_OK, LC_PENDING))
    return s, lat.value


def lc_server_stats(server):
    a, b, c = c_u64(), c_u64(), c_u64()
    _check(load().lc_server_stats(server, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "lc_server_stats")
    return a.value, b.value, c.value


def lc_server_destroy(server):
    _check(load().lc_server_destroy(server), "lc_server_destroy")


def lc_server_trace(server):
    """dict(busy_ms, overlap_ms, free_samples, capacity) of a server (see agnlc.h)."""
    b, o, f, c = ctypes.c_double(), ctypes.c_double(), c_u64(), c_u64()
    _check(load().lc_server_trace(server, ctypes.byref(b), ctypes.byref(o), ctypes.byref(f), ctypes.byref(c)),
           "lc_server_trace")
    return {"busy_ms": b.value, "overlap_ms": o.value, "free_samples": f.value, "capacity": c.value}


def lc_plan_footprint(jobs, prec=LC_FP32):
    """Device bytes lc_plan_create would allocate for these jobs (host only)."""
    arr = job_array(jobs)
    n = c_sz()
    _check(load().lc_plan_footprint(arr, len(jobs), int(prec), ctypes.byref(n)), "lc_plan_footprint")
    return n.value
