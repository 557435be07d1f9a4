"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/fsqr.h declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2601_02826_gb300 import build, fsqr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fsqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int64_t|int|void|const char \*)\s*\*?\s*(fsqr_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fsqr_fit", "fsqr_fit_batch", "fsqr_predict", "fsqr_lambda_max", "fsqr_eta",
                 "fsqr_kkt", "fsqr_create", "fsqr_destroy"):
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(fsqr.EXPORTS)


def test_version_and_default_options_without_gpu():
    L = fsqr.load()
    assert L.fsqr_version() >= 10000
    o = fsqr.default_opts()
    assert o.tol == 1e-6 and o.check_every == 10 and o.max_iter == 100000
    assert o.digits == 4 and o.max_group == 4 and o.precision == fsqr.FP64


def test_struct_layouts_match_header(tmp_path):
    """Compiles a C probe against include/fsqr.h and compares every field offset."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"fsqr_design": fsqr.Design, "fsqr_opts": fsqr.Opts, "fsqr_info": fsqr.Info,
               "fsqr_profile": fsqr.Profile}
    cname = {"lambda_": "lambda"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fsqr.h"', "int main(void){"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{sname} {f} %zu\\n", offsetof({sname}, {cname.get(f, f)}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for sname, cls in structs.items():
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for f, _ in cls._fields_:
            assert got[(sname, f)] == getattr(cls, f).offset, (sname, f)


def test_create_fails_cleanly_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = fsqr.load()
    h = ctypes.c_void_p()
    assert L.fsqr_create(ctypes.byref(h), 0, None) != 0


def test_header_declares_the_new_entry_points():
    h = open(os.path.join(ROOT, "include", "fsqr.h")).read()
    for name in ("fsqr_fit_lla", "fsqr_path_stats", "fsqr_interval_coverage", "fsqr_wait_selftest"):
        assert name + "(" in h, name
