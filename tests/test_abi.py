"""The C-ABI library builds for sm_103a and exports every entry point include/ffe.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ffe.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ffe_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2404_01531_gb300 import build, ffe
    if not os.path.exists(ffe.LIB_PATH):
        build.build()
    return ffe.LIB_PATH


def test_header_declares_the_boundary():
    names = declared()
    for n in ("ffe_create", "ffe_set_initial", "ffe_rhs", "ffe_step", "ffe_destroy", "ffe_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ffe_[a-z_0-9]+)\b", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    from paper_2404_01531_gb300 import ffe
    assert sorted(ffe.EXPORTS) == declared()
    lib = ffe.load()
    for n in declared():
        assert hasattr(lib, n)


def test_library_is_device_code_for_sm_103a(lib_path):
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", lib_path], capture_output=True, text=True)
    assert "sm_103a" in out.stdout


def test_last_error_starts_empty(lib_path):
    from paper_2404_01531_gb300 import ffe
    assert ffe.load().ffe_last_error() == b""
