"""GB300-native generator of AGN Eddington-ratio light curves (Sartori et al. 2019,
Sec. 2.1): TK95 realisation of a bending power-law PSD, ERDF draws, and the
iterative amplitude-adjusted Fourier transform, in hand-written sm_103a CUDA
kernels behind the C ABI of include/agnlc.h.

``_abi`` is the thin ctypes binding (same names as the C ABI); ``Plan`` is a
small convenience wrapper that allocates outputs with torch.
"""
from __future__ import annotations

from . import _abi
from ._abi import (LC_FP32, LC_FP64, LcError, lc_generate, lc_generate_host, lc_get_state, lc_iterate,
                   lc_periodogram, lc_plan_buffer, lc_plan_convergence, lc_plan_create, lc_plan_destroy,
                   lc_plan_last_launches, lc_plan_profile, lc_structure_function,
                   lc_plan_set_convergence, lc_plan_timing, lc_plan_total_samples, lc_plan_workspace_bytes,
                   lc_plan_footprint, lc_poll, lc_rank_replace, lc_server_create, lc_server_destroy,
                   lc_server_stats, lc_server_trace, lc_set_state, lc_setup, lc_submit)

__all__ = ["Plan", "LC_FP32", "LC_FP64", "LcError", "lc_plan_create", "lc_generate", "lc_generate_host",
           "lc_setup", "lc_iterate", "lc_get_state", "lc_set_state", "lc_rank_replace", "lc_plan_buffer",
           "lc_plan_last_launches", "lc_plan_timing", "lc_plan_total_samples", "lc_plan_workspace_bytes", "lc_plan_destroy",
           "lc_plan_set_convergence", "lc_plan_convergence", "lc_periodogram", "lc_structure_function",
           "lc_plan_profile",
           "lc_plan_footprint",
           "lc_server_create", "lc_submit", "lc_poll", "lc_server_stats", "lc_server_trace", "lc_server_destroy"]


class Plan:
    """Owns an lc_plan; outputs are torch tensors on the plan's device."""

    def __init__(self, jobs, prec=LC_FP32, device=0):
        import torch
        self.jobs = list(jobs)
        self.prec = prec
        self.device = device
        self.handle = lc_plan_create(self.jobs, prec, device)
        self.total = lc_plan_total_samples(self.handle)
        self.dtype = torch.float32 if prec == LC_FP32 else torch.float64
        self.offsets = [0]
        for j in self.jobs:
            self.offsets.append(self.offsets[-1] + (1 << int(j["log2n"])))

    def _stream(self, stream):
        import torch
        return stream if stream is not None else torch.cuda.current_stream(self.device)

    def empty(self):
        import torch
        return torch.empty(self.total, dtype=self.dtype, device=f"cuda:{self.device}")

    def generate(self, out=None, out_tk=None, stream=None):
        out = self.empty() if out is None else out
        lc_generate(self.handle, out, out_tk, self._stream(stream))
        return out

    def setup(self, out_tk=None, stream=None):
        lc_setup(self.handle, out_tk, self._stream(stream))

    def iterate(self, iters=0, stream=None):
        lc_iterate(self.handle, iters, self._stream(stream))

    def get_state(self, stream=None):
        out = self.empty()
        lc_get_state(self.handle, out, self._stream(stream))
        return out

    def set_state(self, x, stream=None):
        lc_set_state(self.handle, x, self._stream(stream))

    def rank_replace(self, x_adj, out=None, stream=None):
        """out[perm[r]] = s[r] per curve, perm the stable argsort of x_adj."""
        out = self.empty() if out is None else out
        lc_rank_replace(self.handle, x_adj, out, self._stream(stream))
        return out

    def buffer(self, which):
        """Copy of plan buffer `which` (0 state, 1 amplitudes, 2 sorted draws)."""
        import torch
        ptr, nbytes = lc_plan_buffer(self.handle, which)
        esize = 4 if self.prec == LC_FP32 else 8

        class _View:  # zero-copy view of the library-owned device buffer
            __cuda_array_interface__ = {"shape": (nbytes // esize,), "typestr": "<f%d" % esize,
                                        "data": (ptr, False), "version": 3, "strides": None}

        torch.cuda.current_stream(self.device).synchronize()
        return torch.as_tensor(_View(), device=f"cuda:{self.device}").clone()

    def set_convergence(self, thresholds=None, history=None):
        """Turn on the Sec. 3.2.2 convergence test (Eq. 4) with per-curve
        thresholds (None: never stop); history defaults to the largest job count."""
        h = int(history) if history is not None else max(1, max(int(j["iters"]) for j in self.jobs))
        lc_plan_set_convergence(self.handle, thresholds, h)
        self.history = h

    def convergence(self):
        """(deltas [ncurves, history], iters_run [ncurves]) of the last run."""
        return lc_plan_convergence(self.handle, len(self.jobs), self.history)

    def periodogram(self, x, rms=False, stream=None):
        """Eq. A2 (or Eq. A4) of every curve of x; float64 tensor laid out like A."""
        import torch
        nh = sum((1 << int(j["log2n"])) // 2 + 1 for j in self.jobs)
        out = torch.empty(nh, dtype=torch.float64, device=f"cuda:{self.device}")
        lc_periodogram(self.handle, x, rms, out, self._stream(stream))
        return out

    def structure_function(self, x, lags, stream=None):
        """Eq. A6: SF(tau)^2 of every curve at integer lags; float64 [ncurves, nlags]."""
        import torch
        out = torch.empty((len(self.jobs), len(lags)), dtype=torch.float64, device=f"cuda:{self.device}")
        lc_structure_function(self.handle, x, lags, out, self._stream(stream))
        return out

    def curve(self, x, c):
        return x[self.offsets[c]:self.offsets[c + 1]]

    def close(self):
        if self.handle is not None:
            lc_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
