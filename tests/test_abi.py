"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/ecc.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1806_02637_gb300 as ecc
from paper_1806_02637_gb300 import build as ecc_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ecc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ecc_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("ecc_create", "ecc_destroy", "ecc_last_error", "ecc_precompute_radon_derivative", "ecc_evaluate",
              "ecc_scan_consistency_host", "ecc_status", "ecc_version"):
        assert n in names


def test_library_exports_every_declared_symbol():
    so = ecc_build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ecc_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(so)
    for n in _declared():
        assert hasattr(lib, n)


def test_null_context_is_rejected_without_touching_the_gpu():
    lib = ecc.load()
    assert lib.ecc_version() >= 100
    rc = lib.ecc_evaluate(None, 2, None, None, None, None, 8, 8, 8, 8, 0, 8, 0.0, None, 1, None, None, None, None)
    assert rc == -1
    assert b"ctx" in lib.ecc_last_error(None)
    rc = lib.ecc_precompute_radon_derivative(None, 1, None, None, 8, 8, 8, 8, 0, None, None, None)
    assert rc == -1


def test_sources_are_sm103a_only():
    assert ecc_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    for src in ecc_build.sources():
        text = open(src).read()
        assert "wgmma" not in text
