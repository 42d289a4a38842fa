"""CPU checks of the C ABI: the library builds, loads, and exports every declared symbol."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jfnk.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(jfnk_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2406_17234_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (jfnk_\w+)", out))
    declared = _declared()
    assert len(declared) >= 18
    missing = [s for s in declared if s not in exported]
    assert not missing, missing


def test_binding_declares_every_symbol(lib_path):
    from paper_2406_17234_gb300 import binding
    binding._lib = None
    lib = binding.load(lib_path)
    for name in _declared():
        assert name in binding._SIGNATURES, name
        getattr(lib, name)


def test_default_options_without_gpu(lib_path):
    from paper_2406_17234_gb300 import binding
    o = binding.default_options()
    assert o.rtol == 1e-2 and o.ftol == 1e-4 and o.fdrop == 1e-2 and o.krylov_max == 50
