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
