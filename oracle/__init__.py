"""FP64 CPU oracle for the AGN light-curve generator (Sartori et al. 2019, Sec. 2.1).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path (the CUDA
library and its Python binding) never imports this package.

The arithmetic lives in ``oracle.c`` (plain C, FP64, ``-ffp-contract=off``); this
module builds it with gcc on first use and exposes numpy wrappers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-fvisibility=hidden", "-pthread"]


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc) if it is missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The loaded oracle library.  ORACLE_LIB names another build of oracle.c
    to load instead (the mutation test loads copies with a planted mistake)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("ORACLE_LIB")
            if not path:
                path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            d, u32, u64, i32, sz = (ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64,
                                    ctypes.c_int, ctypes.c_size_t)
            sig = {
                "or_philox4x32_10": (None, [P, P, P]),
                "or_u01": (d, [u32, u32]),
                "or_spec_exp": (d, [d]),
                "or_spec_log": (d, [d]),
                "or_spec_log1p": (d, [d]),
                "or_erdf_icdf": (d, [P, i32, d]),
                "or_erdf_draws": (None, [P, i32, i32, u64, u64, i32, sz, P]),
                "or_erdf_density": (d, [P, i32, i32, d]),
                "or_erdf_table": (None, [P, i32, i32, P]),
                "or_erdf_icdf_tab": (d, [P, P, d]),
                "or_psd": (d, [d, d, d, d]),
                "or_tk_spectrum": (None, [u32, d, P, i32, u64, u64, P]),
                "or_dft": (None, [sz, P, P, i32]),
                "or_fft": (None, [sz, P, P, i32]),
                "or_r2c": (None, [sz, P, P]),
                "or_c2r": (None, [sz, P, P]),
                "or_tk_series": (None, [u32, d, P, i32, i32, u64, u64, P, P, P]),
                "or_argsort": (None, [sz, P, P]),
                "or_sort": (None, [sz, P]),
                "or_iterate": (None, [u32, P, P, P, u32, P, P]),
                "or_delta": (d, [sz, P, P]),
                "or_periodogram": (None, [sz, P, d, i32, P]),
                "or_structure_function": (None, [sz, P, sz, P, P]),
                "or_iterate_conv": (u32, [u32, P, P, P, u32, d, P]),
                "or_generate": (None, [u32, P, P, u32, u64, u64, i32, P, P, P, P]),
                "or_generate_batch": (i32, [sz, P, P, P, P, P, P, i32, i32, P]),
                "or_spec_exp_v": (None, [sz, P, P]),
                "or_spec_log_v": (None, [sz, P, P]),
                "or_spec_log1p_v": (None, [sz, P, P]),
                "or_erdf_icdf_v": (None, [P, i32, sz, P, P]),
                "or_philox_v": (None, [sz, P, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- primitives
def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ctr (..., 4) under keys key (..., 2) -> (..., 4) uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    lib().or_philox_v(ctr.shape[0], _p(ctr), _p(key), _p(out))
    return out


def u01(w0: int, w1: int) -> float:
    return lib().or_u01(w0, w1)


def spec_exp(x):
    x = _f64(np.atleast_1d(x)); out = np.empty_like(x)
    lib().or_spec_exp_v(x.size, _p(x), _p(out)); return out


def spec_log(x):
    x = _f64(np.atleast_1d(x)); out = np.empty_like(x)
    lib().or_spec_log_v(x.size, _p(x), _p(out)); return out


def spec_log1p(x):
    x = _f64(np.atleast_1d(x)); out = np.empty_like(x)
    lib().or_spec_log1p_v(x.size, _p(x), _p(out)); return out


def erdf_icdf(erdf, U, linear_space=0):
    e = _f64(erdf); U = _f64(np.atleast_1d(U)); out = np.empty_like(U)
    lib().or_erdf_icdf_v(_p(e), int(linear_space), U.size, _p(U), _p(out)); return out


ERDF_TABLE = 4096  # intervals of the tabulated CDF (kinds 1, 2)


def _erdf6(erdf, sigma=None):
    """{log_lmin, log_lmax, log_lbreak, slope_low, slope_high, sigma}."""
    e = list(np.asarray(erdf, dtype=np.float64).ravel())
    if len(e) == 5:
        e.append(0.0 if sigma is None else float(sigma))
    elif sigma is not None:
        e[5] = float(sigma)
    return _f64(e)


def erdf_draws(erdf, n, seed, curve_id, prec=0, linear_space=0, kind=0, sigma=None):
    e = _erdf6(erdf, sigma); out = np.empty(n, dtype=np.float64)
    lib().or_erdf_draws(_p(e), int(linear_space), int(kind), seed, curve_id, prec, n, _p(out)); return out


def erdf_density(erdf, u, kind, linear_space=0, sigma=None):
    """Unnormalised ERDF density in u = log10 lambda (kinds 0, 1, 2)."""
    e = _erdf6(erdf, sigma)
    return np.array([lib().or_erdf_density(_p(e), int(kind), int(linear_space), float(v))
                     for v in np.atleast_1d(u)])


def erdf_table(erdf, kind, linear_space=0, sigma=None):
    """Unnormalised CDF at the ERDF_TABLE + 1 grid nodes."""
    e = _erdf6(erdf, sigma); F = np.empty(ERDF_TABLE + 1)
    lib().or_erdf_table(_p(e), int(kind), int(linear_space), _p(F)); return F


def erdf_icdf_tab(erdf, F, U, sigma=None):
    e = _erdf6(erdf, sigma); F = _f64(F)
    return np.array([lib().or_erdf_icdf_tab(_p(e), _p(F), float(v)) for v in np.atleast_1d(U)])


def psd(f, f_br, a_low, a_high):
    return lib().or_psd(float(f), float(f_br), float(a_low), float(a_high))


def tk_spectrum(log2n, dt, psd_params, seed, curve_id, coeffs=0) -> np.ndarray:
    """coeffs 0: TK95 Gaussian coefficients; 1: fixed amplitude sqrt(P), random phase."""
    n = 1 << log2n
    ps = _f64(psd_params); X = np.empty(2 * (n // 2 + 1), dtype=np.float64)
    lib().or_tk_spectrum(log2n, dt, _p(ps), int(coeffs), seed, curve_id, _p(X))
    return X[0::2] + 1j * X[1::2]


def dft(z, sign=-1):
    z = np.ascontiguousarray(z, dtype=np.complex128); out = np.empty_like(z)
    lib().or_dft(z.size, _p(z), _p(out), sign); return out


def fft(z, sign=-1):
    z = np.ascontiguousarray(z, dtype=np.complex128); out = np.empty_like(z)
    lib().or_fft(z.size, _p(z), _p(out), sign); return out


def r2c(x):
    x = _f64(x); out = np.empty(x.size // 2 + 1, dtype=np.complex128)
    lib().or_r2c(x.size, _p(x), _p(out)); return out


def c2r(Y, n):
    Y = np.ascontiguousarray(Y, dtype=np.complex128); out = np.empty(n, dtype=np.float64)
    lib().or_c2r(n, _p(Y), _p(out)); return out


def tk_series(log2n, dt, psd_params, seed, curve_id, coeffs=0, targets=0):
    """Normalised TK95 series, target amplitudes A (n/2+1) and sigma
    (targets 1: the amplitudes of the PSD itself)."""
    n = 1 << log2n
    ps = _f64(psd_params)
    x = np.empty(n); A = np.empty(n // 2 + 1); sig = np.empty(1)
    lib().or_tk_series(log2n, dt, _p(ps), int(coeffs), int(targets), seed, curve_id, _p(x), _p(A), _p(sig))
    return x, A, float(sig[0])


def argsort(v):
    v = _f64(v); perm = np.empty(v.size, dtype=np.int64)
    lib().or_argsort(v.size, _p(v), _p(perm)); return perm


def sort(v):
    """Ascending sort of a copy (the sort of the ERDF draws)."""
    v = _f64(v).copy()
    lib().or_sort(v.size, _p(v)); return v


def iterate(A, s, x, iters, want_adj=False):
    """Run `iters` E13 iterations from state x; returns (x, x_adj_last, perm_last)."""
    x = _f64(x).copy(); A = _f64(A); s = _f64(s)
    n = x.size; log2n = n.bit_length() - 1
    assert 1 << log2n == n and A.size == n // 2 + 1 and s.size == n
    xa = np.empty(n) if want_adj else None
    perm = np.empty(n, dtype=np.int64) if want_adj else None
    lib().or_iterate(log2n, _p(A), _p(s), _p(x), iters,
                     _p(xa) if want_adj else None, _p(perm) if want_adj else None)
    return x, xa, perm


def delta(x_old, x_new) -> float:
    """Eq. 4: rms over the samples of log10(x_new / x_old)."""
    a = _f64(x_old); b = _f64(x_new)
    assert a.size == b.size
    return float(lib().or_delta(a.size, _p(a), _p(b)))


def iterate_conv(A, s, x, iters, thr=0.0):
    """Iterations with the Sec. 3.2.2 stop: returns (x, deltas[:run], run)."""
    x = _f64(x).copy(); A = _f64(A); s = _f64(s)
    n = x.size; log2n = n.bit_length() - 1
    assert 1 << log2n == n and A.size == n // 2 + 1 and s.size == n
    d = np.full(max(int(iters), 1), np.nan)
    run = int(lib().or_iterate_conv(log2n, _p(A), _p(s), _p(x), int(iters), float(thr), _p(d)))
    return x, d[:run], run


def periodogram(x, dt=1.0, rms=False):
    """Eq. A2 (or the rms-normalised Eq. A4) at j = 0..N/2."""
    x = _f64(x); P = np.empty(x.size // 2 + 1)
    lib().or_periodogram(x.size, _p(x), float(dt), int(bool(rms)), _p(P)); return P


def structure_function(x, lags):
    """Eq. A6: SF(tau)^2 at integer lags (samples)."""
    x = _f64(x); L = np.ascontiguousarray(lags, dtype=np.uint32); out = np.empty(L.size)
    lib().or_structure_function(x.size, _p(x), L.size, _p(L), _p(out)); return out


def job_modes(job) -> np.ndarray:
    """{linear_space, ERDF kind, TK coefficients, target amplitudes} of a job dict."""
    return np.array([job.get("linear_space", 0), job.get("erdf_kind", 0), job.get("tk_coeffs", 0),
                     job.get("tk_targets", 0)], dtype=np.int32)


def job_params(job) -> np.ndarray:
    """Flatten a job dict into the oracle's 10-double parameter block."""
    return np.array([job["dt"], job["f_br"], job["alpha_low"], job["alpha_high"],
                     job["log_lmin"], job["log_lmax"], job["log_lbreak"],
                     job["slope_low"], job["slope_high"], job.get("sigma", 0.0)], dtype=np.float64)


def generate(job, prec=0, want=("x",)):
    """Whole generator for one job dict; returns a dict with the requested arrays
    among x (final series), tk (normalised TK95 series), A, s (sorted draws)."""
    log2n = int(job["log2n"]); n = 1 << log2n
    par = job_params(job)
    out = {k: (np.empty(n // 2 + 1) if k == "A" else np.empty(n)) for k in ("x", "tk", "A", "s")}
    modes = job_modes(job)
    lib().or_generate(log2n, _p(par), _p(modes), int(job["iters"]),
                      int(job["seed"]), int(job["curve_id"]), prec, _p(out["x"]),
                      _p(out["tk"]) if "tk" in want else None,
                      _p(out["A"]) if "A" in want else None,
                      _p(out["s"]) if "s" in want else None)
    return {k: out[k] for k in want}


def generate_batch(jobs, prec=0, nthreads=1):
    """Final series of many jobs, concatenated in job order; returns (x, threads_used)."""
    nc = len(jobs)
    log2n = np.array([j["log2n"] for j in jobs], dtype=np.uint32)
    par = np.ascontiguousarray(np.stack([job_params(j) for j in jobs]))
    modes = np.ascontiguousarray(np.stack([job_modes(j) for j in jobs]))
    iters = np.array([j["iters"] for j in jobs], dtype=np.uint32)
    seed = np.array([j["seed"] for j in jobs], dtype=np.uint64)
    cid = np.array([j["curve_id"] for j in jobs], dtype=np.uint64)
    total = int(sum(1 << int(l) for l in log2n))
    out = np.empty(total)
    used = lib().or_generate_batch(nc, _p(log2n), _p(par), _p(modes), _p(iters), _p(seed),
                                   _p(cid), prec, int(nthreads), _p(out))
    return out, int(used)
