"""The C-ABI library builds for sm_103a and exports every entry point include/tpe.h declares.
No kernel is launched (CPU only)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tpe.h")).read()
    return sorted(set(re.findall(r"TPE_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)))


def test_header_declares_the_paper_entry_points():
    names = _declared()
    for n in ["tp_energy", "tp_differential", "sobolev_apply", "sobolev_gradient", "descent_step", "tp_create"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2006_07859_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2006_07859_gb300 import tpe
    assert sorted(tpe.EXPORTED) == _declared()


def test_library_loads_without_gpu():
    import ctypes
    from paper_2006_07859_gb300 import build, tpe
    build.build()
    L = tpe.library()
    p = tpe.TpParams()
    L.tp_default_params(ctypes.byref(p))        # pure host function
    assert p.alpha == 2.0 and p.beta == 4.5 and p.cg_rtol == 1e-6


def test_struct_layouts_match_header():
    """Compile a tiny C program against tpe.h and compare sizeof/offsetof with the ctypes mirrors."""
    import ctypes
    import tempfile
    from paper_2006_07859_gb300 import tpe
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "tpe.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(tp_params), offsetof(tp_params, independent),
         sizeof(tp_step_info), offsetof(tp_step_info, rel_res), sizeof(tp_solve_info),
         offsetof(tp_params, warm_start));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(tpe.TpParams), tpe.TpParams.independent.offset, ctypes.sizeof(tpe.TpStepInfo),
                    tpe.TpStepInfo.rel_res.offset, ctypes.sizeof(tpe.TpSolveInfo), tpe.TpParams.warm_start.offset]
