"""The C ABI library builds for sm_103a, loads, and exports every declared function.

No compute call is made (no GPU here); the GPU tests call every entry point.
"""
import ctypes
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


STRUCTS = {"pod_cg_config": "Config", "pod_cg_csr": "CSRStruct", "pod_cg_stats": "Stats",
           "pod_cg_batch_seq": "BatchSeq", "pod_cg_batch_sysstat": "BatchSysStat",
           "pod_cg_krylov_config": "KrylovConfig"}


def test_struct_layouts_match_header(tmp_path):
    """Every struct the binding passes through the ABI has the header's size and field
    offsets (a C program compiled against include/pod_cg.h prints them)."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pod_cg.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        S = getattr(_lib, pyname)
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in S._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            c, field, v = ln.split()
            got[(c, field)] = int(v)
    for cname, pyname in STRUCTS.items():
        S = getattr(_lib, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(S), cname
        for f, _ in S._fields_:
            assert got[(cname, f)] == getattr(S, f).offset, (cname, f)


BAD_CONFIGS = [
    dict(w_max=0), dict(w_max=65), dict(s_max=0), dict(s_max=65), dict(energy=1.5), dict(energy=float("nan")),
    dict(k_max=-1), dict(max_refine=-1), dict(precision=2), dict(keep_factors=-1), dict(loop_mode=3),
    dict(proj_form=2), dict(spmv_lanes=3), dict(spmv_lanes=64), dict(inner_tol=0.0), dict(inner_tol=1.0),
    dict(three_stage=3), dict(three_stage=1, y_max=41), dict(three_stage=1, y_max=0),
    dict(three_stage=1, energy_y=1.5), dict(three_stage=1, tol_stage2=-1.0),
    dict(three_stage=1, tol_stage2=float("inf")), dict(three_stage=2, tol_inner=1.0),
    dict(three_stage=2, precision=1), dict(bsr=2), dict(pod_metric=2), dict(use_tc_gram=1, precision=0),
    dict(use_tc_gram=2, precision=1), dict(use_tc_gram=-2), dict(w_select=2), dict(w_select=-1),
]


def test_create_rejects_bad_configuration():
    """pod_cg_create checks the configuration on the host before any device call: each bad
    field gives ERR_ARG (1), no handle, and a message from pod_cg_last_error(NULL)."""
    L = _lib.load()
    for bad in BAD_CONFIGS:
        c = _lib.Config()
        assert L.pod_cg_config_default(ctypes.byref(c)) == 0
        for k, v in bad.items():
            setattr(c, k, v)
        h = ctypes.c_void_p(123)
        st = L.pod_cg_create(1000, ctypes.byref(c), None, ctypes.byref(h))
        assert st == 1, (bad, st)
        assert not h.value, bad
        assert L.pod_cg_last_error(None), bad
    h = ctypes.c_void_p()
    assert L.pod_cg_create(0, None, None, ctypes.byref(h)) == 1
    assert L.pod_cg_create(10, None, None, None) == 1


def test_every_declaration_cites_its_passage():
    """Each entry point's comment in include/pod_cg.h names the passage of the paper that
    defines its operation (a Section, Algorithm, Equation or Theorem), or says that it has
    no counterpart in the paper."""
    text = open(os.path.join(ROOT, "include", "pod_cg.h")).read()
    decl = r"/\*((?:(?!\*/).)*)\*/\s*(?:pod_cg_status|const char\*|size_t)\s+(pod_cg_\w+)\s*\("
    missing = [name for com, name in re.findall(decl, text, flags=re.S)
               if not re.search(r"Section|Algorithm|Eq\.|Theorem|no counterpart in the paper", com)]
    assert not missing, missing


def test_gram_noalloc_scratch_covers_every_shape():
    """The allocation-free Gram keeps its scratch in a fixed array of 65,536 doubles. On a
    152-SM GB300 every product it accepts (p, q <= 65) must fit: the split-K shape gives
    about four partial 8x8 tiles per SM, whatever n."""
    L = _lib.load()
    cap = 65536 * 8
    worst = 0
    for n in (1, 31, 256, 4097, 100_000, 2_097_152, 2**31 - 1):
        for p in range(1, 66):
            for q in range(1, 66):
                need = L.pod_cg_gram_workspace_for(n, p, q, 152)
                assert 0 < need <= cap, (n, p, q, need)
                worst = max(worst, need)
    assert worst <= 352_256   # (4 * 152 + 81 - 1) tiles of 64 doubles
    assert L.pod_cg_gram_workspace_for(0, 1, 1, 152) == 0
