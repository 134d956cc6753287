"""The C-ABI library builds, loads, and exports every entry point include/swi.h declares.

No compute call is made here (no GPU on the CPU runner)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    with open(os.path.join(ROOT, "include", "swi.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(swi_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_01139_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_call_list():
    d = _declared()
    for name in ("swi_create", "swi_set_potential", "swi_set_absorber", "swi_set_windows", "swi_solve",
                 "swi_transmission", "swi_grad", "swi_last_error", "swi_destroy"):
        assert name in d


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_export_list_matches_header():
    import paper_1606_01139_gb300 as swi
    assert sorted(swi.EXPORTS) == _declared()


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_1606_01139_gb300 as swi
    saved = swi._lib
    try:
        swi._lib = None
        with pytest.raises(RuntimeError):
            swi.load(str(tmp_path / "missing.so"))
    finally:
        swi._lib = saved


def test_create_without_device_reports_an_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import paper_1606_01139_gb300 as swi
    swi.load()
    with pytest.raises(swi.SwiError):
        swi.Context(10, 10, 20, 0.5, stream=0)


def test_null_context_is_rejected_by_every_entry_taking_one(lib):
    # no device needed: each call validates its context before touching CUDA
    import paper_1606_01139_gb300 as swi
    swi.load()
    L = swi._lib
    assert L.swi_solve(None, None, None) == swi.SWI_EINVAL
    assert L.swi_refine(None, None, None) == swi.SWI_EINVAL
    assert L.swi_residuals(None, None) == swi.SWI_EINVAL
    assert L.swi_transmission(None, 1, None, None) == swi.SWI_EINVAL
    assert L.swi_set_contraction(None, 0) == swi.SWI_EINVAL
    assert L.swi_set_windows_complex(None, 1, None, None, None) == swi.SWI_EINVAL


def test_batch_solve_validates_its_arguments_before_any_device_call(lib):
    import paper_1606_01139_gb300 as swi
    swi.load()
    L = swi._lib
    assert L.swi_solve_batch(0, None, None, 0, None, None) == swi.SWI_EINVAL
    nulls = (ctypes.c_void_p * 2)(None, None)
    assert L.swi_solve_batch(2, ctypes.cast(nulls, ctypes.c_void_p), None, 0, None, None) == swi.SWI_EINVAL
    assert b"null context" in L.swi_last_error(None)


def test_binding_structs_match_the_header(tmp_path):
    # the ctypes structures of the binding have the C layout of include/swi.h:
    # size and the offset of every field, compiled with the host C compiler
    import shutil
    import subprocess
    import paper_1606_01139_gb300 as swi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("swi_solve_opts", swi.SolveOpts), ("swi_solve_info", swi.SolveInfo),
             ("swi_window_info", swi.WindowInfo), ("swi_refine_opts", swi.RefineOpts),
             ("swi_refine_info", swi.RefineInfo), ("swi_plan_opts", swi.PlanOpts), ("swi_plan_info", swi.PlanInfo),
             ("swi_kernel_stats", swi.KernelStats)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "swi.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
