"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads
without a GPU, exports every entry point include/nlh.h declares, and the
ctypes structures of the binding have the C compiler's layout."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2407_06834_gb300 import build_native, nlh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_symbols():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(nlh_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build_native.build()
    lib = C.CDLL(path)
    names = declared_symbols()
    assert "nlh_solve" in names and "nlh_matvec" in names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(nlh.SIGNATURES) >= names - {"nlh_plan"}


def test_version_and_error_without_gpu():
    lib = nlh.load()
    assert lib.nlh_version().decode().startswith("nlh")
    # argument validation happens before any CUDA call
    st = lib.nlh_plan_destroy(None)
    assert st == 0
    assert lib.nlh_plan_get_info(None, None) == -1
    assert "NULL" in lib.nlh_last_error().decode()


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "nlh_net.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(nlh_plan_desc),'
                   ' sizeof(nlh_plan_info), sizeof(nlh_solve_opts), sizeof(nlh_solve_info),'
                   ' offsetof(nlh_plan_desc, torus_fill), offsetof(nlh_solve_opts, x0), offsetof(nlh_solve_opts, x0_check), offsetof(nlh_solve_opts, precond),'
                   ' sizeof(nlh_net_batch), offsetof(nlh_net_batch, beta), offsetof(nlh_solve_info, x0_rejected),'
                   ' offsetof(nlh_plan_desc, window_first), offsetof(nlh_plan_desc, reduce), offsetof(nlh_plan_desc, reduce_ctx),'
                   ' offsetof(nlh_plan_info, window_count), offsetof(nlh_plan_desc, image),'
                   ' offsetof(nlh_plan_desc, patch_pad), offsetof(nlh_plan_info, coords_from_image));'
                   ' return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    assert out == [C.sizeof(nlh.PlanDesc), C.sizeof(nlh.PlanInfo), C.sizeof(nlh.SolveOpts),
                   C.sizeof(nlh.SolveInfo), nlh.PlanDesc.torus_fill.offset,
                   nlh.SolveOpts.x0.offset, nlh.SolveOpts.x0_check.offset, nlh.SolveOpts.precond.offset, C.sizeof(nlh.NetBatch),
                   nlh.NetBatch.beta.offset, nlh.SolveInfo.x0_rejected.offset,
                   nlh.PlanDesc.window_first.offset, nlh.PlanDesc.reduce.offset,
                   nlh.PlanDesc.reduce_ctx.offset, nlh.PlanInfo.window_count.offset,
                   nlh.PlanDesc.image.offset, nlh.PlanDesc.patch_pad.offset,
                   nlh.PlanInfo.coords_from_image.offset]
