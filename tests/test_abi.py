"""The C-ABI library builds, loads and exports every entry point that
include/agnlc.h declares; the ctypes structures match the C layout; argument
validation happens on the host (no GPU needed)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1909_06374_gb300 import _abi, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "agnlc.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^LC_API\s+[\w\s\*]+?\b(lc_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["lc_plan_create", "lc_generate", "lc_submit", "lc_poll", "lc_plan_destroy",
                 "lc_server_create", "lc_server_destroy", "lc_status_string"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = _abi.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.library_path()], capture_output=True, text=True)
    exported = set(re.findall(r"\bT (lc_\w+)", out.stdout))
    assert set(declared_functions()) <= exported
    # nothing else with the lc_ prefix leaks out of the library
    assert exported <= set(declared_functions())


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) == set(_abi._SIGS)


def test_struct_layout_matches_c():
    prog = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "agnlc.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(lc_job), offsetof(lc_job, dt),
             offsetof(lc_job, psd), offsetof(lc_job, erdf), offsetof(lc_job, seed),
             offsetof(lc_job, curve_id), sizeof(lc_erdf), offsetof(lc_erdf, linear_space),
             offsetof(lc_erdf, kind), offsetof(lc_erdf, sigma), sizeof(lc_psd));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "p")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    J, E, P = _abi.LcJob, _abi.LcErdf, _abi.LcPsd
    assert vals == [ctypes.sizeof(J), J.dt.offset, J.psd.offset, J.erdf.offset, J.seed.offset,
                    J.curve_id.offset, ctypes.sizeof(E), E.linear_space.offset, E.kind.offset, E.sigma.offset,
                    ctypes.sizeof(P)]


def test_status_strings():
    assert _abi.status_name(0) == "LC_OK"
    assert _abi.status_name(-4) == "LC_ERR_TIMEOUT"
    assert _abi.status_name(99) == "LC_UNKNOWN_STATUS"


@pytest.mark.parametrize("bad", [dict(log2n=3), dict(log2n=28), dict(dt=0.0), dict(f_br=-1.0),
                                 dict(log_lbreak=0.5), dict(log_lmin=0.0), dict(alpha_high=float("nan")),
                                 dict(slope_low=float("inf")), dict(erdf_kind=3), dict(erdf_kind=-1),
                                 dict(erdf_kind=2, sigma=0.0), dict(erdf_kind=2, sigma=0.001),
                                 dict(erdf_kind=2, sigma=0.5, log_lbreak=-40.0),
                                 dict(erdf_kind=1, log_lbreak=0.5), dict(tk_coeffs=2), dict(tk_targets=-1)])
def test_invalid_jobs_are_rejected_before_any_device_work(bad):
    j = workloads.job(10, 3, 0, 0)
    j.update(bad)
    with pytest.raises(_abi.LcError) as e:
        _abi.lc_plan_create([j])
    assert e.value.status == _abi.LC_ERR_INVALID
    assert "job 0" in str(e.value)


def test_null_arguments_are_rejected():
    lib = _abi.load()
    assert lib.lc_plan_create(None, 0, 0, 0, None) == _abi.LC_ERR_INVALID
    assert lib.lc_generate(None, None, None, None) == _abi.LC_ERR_INVALID
    assert lib.lc_plan_destroy(None) == _abi.LC_ERR_INVALID
    assert lib.lc_iterate(None, 1, None) == _abi.LC_ERR_INVALID
    assert lib.lc_poll(None, 0, None, None) != _abi.LC_OK

