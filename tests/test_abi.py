"""The C ABI library builds for sm_103a, loads, and exports every declared function.

No compute call is made (no GPU here); the GPU tests call every entry point.
"""
import glob
import os
import re
import subprocess

from paper_1512_05820_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(pod_cg_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_build_and_exports():
    path = _build.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(pod_cg_\w+)\b", out))
    declared = declared_functions()
    assert declared, "no declarations found"
    missing = declared - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    assert declared == set(_lib.EXPORTS) | (declared - set(_lib.EXPORTS)) and set(_lib.EXPORTS) <= declared


def test_library_loads_without_gpu():
    L = _lib.load()
    for name in declared_functions():
        assert hasattr(L, name)


def test_config_default_is_host_only():
    import ctypes
    L = _lib.load()
    c = _lib.Config()
    assert L.pod_cg_config_default(ctypes.byref(c)) == 0
    assert c.w_max == 32 and c.s_max == 40 and abs(c.energy - 0.9999) < 1e-15 and c.precision == 0
