"""The C-ABI library loads on a CPU-only machine and exports every function
declared in include/*.h (no compute call is made)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(gbf_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_declared_symbols():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_gbf_build", os.path.join(ROOT, "paper_1805_05208_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    declared = _declared()
    assert len(declared) >= 10
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_c_abi():
    import paper_1805_05208_gb300 as gb
    for n in _declared():
        if n in ("gbf_last_error",):
            continue
        assert hasattr(gb, n), n
    assert gb.gbf_options_default().pull_divisor == 20
