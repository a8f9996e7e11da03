"""The C-ABI library loads and exports every symbol include/evc.h declares (no GPU)."""
import os
import re

import pytest

from paper_1602_02306_gb300 import evc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "evc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(evc_[a-z_]+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    from paper_1602_02306_gb300 import build
    build.build()
    return evc.load()


def test_header_declares_the_binding_names():
    assert sorted(evc.EXPORTED) == _declared()


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_version_without_gpu(lib):
    assert evc.evc_version() == 10000


def test_null_context_is_rejected_without_gpu(lib):
    assert lib.evc_set_precond(None, 0, 0.0, 0.0) == evc.EVC_EINVAL
    assert lib.evc_count(None, 0.0, 1.0, 4, 4, 0.0, 0, None, None, None) == evc.EVC_EINVAL
    assert lib.evc_workspace_bytes(None, 1, 1, 1) == 0
    assert lib.evc_last_error(None) == b"null context"


def _header_constants():
    src = open(os.path.join(ROOT, "include", "evc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"(EVC_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            consts[name] = int(val)
    for name, val in re.findall(r"#define\s+(EVC_[A-Z0-9_]+)\s+(-?\d+)", src):
        consts[name] = int(val)
    return consts


def _header_structs():
    src = open(os.path.join(ROOT, "include", "evc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.findall(r"typedef struct\s*\{(.*?)\}\s*(evc_[a-z_]+)\s*;", src, flags=re.S)


def test_binding_constants_match_the_header():
    consts = _header_constants()
    assert len(consts) > 30
    for name, val in consts.items():
        assert getattr(evc, name, None) == val, name


def test_binding_structs_match_the_c_layout(tmp_path):
    # sizes and field offsets as a C compiler lays the header's structs out,
    # against the ctypes mirrors of the binding
    import ctypes
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = _header_structs()
    assert {n for _, n in structs} >= {"evc_csr", "evc_prof_rec", "evc_tuning", "evc_result",
                                        "evc_server_counters"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "evc.h"', "int main(void) {"]
    for body, name in structs:
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in re.findall(r"([A-Za-z_][A-Za-z0-9_]*)\s*;", body):
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    seen = 0
    for line in out.splitlines():
        name, field, val = line.split()
        cls = getattr(evc, name)
        if field == "size":
            assert ctypes.sizeof(cls) == int(val), name
        else:
            assert getattr(cls, field).offset == int(val), (name, field)
        seen += 1
    assert seen > 30


def test_missing_library_fails_loudly():
    # no CPU fallback: without libevc.so every entry point raises
    import subprocess
    import sys
    code = ("from paper_1602_02306_gb300 import evc\n"
            "try:\n"
            "    evc.load('/nonexistent/libevc.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "    raise SystemExit(3)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 3 and "not built" in r.stdout
