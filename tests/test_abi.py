"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/hd.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+(hd_[a-z0-9_]+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1807_08692_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1807_08692_gb300 import hd
    declared = set(_declared())
    assert set(hd._SIGS) <= declared
    assert set(hd.exported_symbols()) == set(hd._SIGS)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1807_08692_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
                assert "oracle/" not in txt, f


def test_binding_marshals_element_types():
    # numpy inputs become the ABI's element types; a tensor of the wrong type
    # is refused (it would be passed by pointer and misread)
    import numpy as np
    import torch
    from paper_1807_08692_gb300 import hd
    a = hd._typed(np.arange(5, dtype=np.int64), np.int32, "int32")
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"] and list(a) == [0, 1, 2, 3, 4]
    assert hd._typed([0.5, 1.5], np.float32, "float32").dtype == np.float32
    assert hd._typed(None, np.int32, "int32") is None
    t = torch.zeros(3, dtype=torch.int32)
    assert hd._typed(t, np.int32, "int32") is t
    import pytest
    with pytest.raises(TypeError):
        hd._typed(torch.zeros(3, dtype=torch.int64), np.int32, "int32")
    with pytest.raises(TypeError):
        hd._typed(torch.zeros(3, dtype=torch.float64), np.float32, "float32")


def test_every_entry_point_is_documented():
    # each declaration in include/hd.h follows a comment block (argument meaning,
    # layout, ownership, errors) or shares the block of the declaration before it
    txt = open(os.path.join(ROOT, "include", "hd.h")).read()
    lines = txt.splitlines()
    undocumented = []
    for i, line in enumerate(lines):
        m = re.match(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+(hd_[a-z0-9_]+)\s*\(", line)
        if not m:
            continue
        k = i - 1
        while k >= 0 and lines[k].strip() == "":
            k -= 1
        prev = lines[k].strip() if k >= 0 else ""
        # a comment ends right above, or the line above continues a documented
        # declaration group (an earlier declaration's trailing argument line)
        if not (prev.endswith("*/") or prev.endswith(");") or prev.endswith(",")):
            undocumented.append(m.group(1))
    assert not undocumented, undocumented
    assert "/*" in txt and txt.count("Sec.") + txt.count("Eq.") >= 10
