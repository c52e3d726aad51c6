"""The C-ABI library loads and exports every function include/*.h declares (no GPU needed)."""

import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2408_08129_gb300 import _binding

    return _binding.LIB_PATH


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dg_mesh_create", "dg_apply_explicit", "dg_apply_implicit", "imex_rk2_step",
                     "dg_apply_grad", "dg_apply_div", "dg_conservation"):
        assert required in names


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = sorted(_declared() - exported)
    assert not missing, missing


def test_library_loads_and_reports_errors_without_gpu(libpath):
    import ctypes

    from paper_2408_08129_gb300 import _binding as B

    assert B.lib.dg_version().startswith(b"dg_atmo")
    # null arguments are rejected with DG_EINVAL and a message, never a crash
    assert B.lib.dg_mesh_create(None, None, None) == -1
    assert b"null" in B.lib.dg_last_error()
    assert B.lib.dg_apply_explicit(None, None, None, None, 0, 0, None) == -1
    o = B.SolverOpts()
    B.lib.dg_solver_opts_default(ctypes.byref(o))
    assert o.picard == 3 and o.restart == 30 and o.tol == 1e-12
