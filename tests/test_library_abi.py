"""The C-ABI library builds, loads and exports every entry point of
include/pdfgpu.h (CPU only: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\**\s*([A-Za-z_]\w*)\s*\(([^;{]*?)\)\s*;",
                             text, flags=re.M):
            names.append(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for must in ["pdf_load_grid", "pdf_bind_values", "pdf_free_grid", "xfxQ2", "xfxQ", "xfxQ2_pw",
                 "alphasQ2", "xfxQ2_backward", "pdf_batch_prepare", "pdf_batch_run",
                 "pdf_get_status", "pdf_last_error", "pdf_lumi", "pdf_lumi_backward"]:
        assert must in names, must


def test_every_declaration_cites_its_passage():
    """Each entry point of include/*.h is documented by the comment right
    before it, and that comment cites the passage of the paper that defines
    the operation (a "Sec." reference) or says that the call goes beyond the
    paper (or that the paper has no counterpart)."""
    decl = re.compile(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\**\s*([A-Za-z_]\w*)\s*\(([^;{]*?)\)\s*;", re.M)
    missing = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        for m in decl.finditer(text):
            before = text[:m.start()]
            comment = before[before.rfind("/*"):before.rfind("*/")]
            low = comment.lower()
            if not ("Sec." in comment or "beyond the paper" in low or "no counterpart" in low):
                missing.append(m.group(1))
    assert not missing, missing


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2012_08221_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.pdf_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.pdf_last_error(), bytes)


def test_python_binding_declares_the_same_entry_points():
    from paper_2012_08221_gb300 import _lib
    declared = set(declared_functions())
    bound = set(_lib.SIGNATURES) | {"pdf_last_error"}
    assert declared == bound, (declared ^ bound)


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA path are independent: neither includes or
    imports the other."""
    csrc = os.path.join(ROOT, "paper_2012_08221_gb300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                s = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|include)\s+[\"<]?(\w+)", s), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            s = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2012_08221_gb300" not in s, f
            assert "pdfgpu" not in s, f
