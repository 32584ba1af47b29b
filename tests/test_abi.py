"""The C-ABI library builds, loads and exports every symbol the header
declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "scr_gb300.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("scr_create", "scr_setup", "scr_solve", "scr_iters", "scr_residual", "scr_destroy",
                 "mm_setup", "mm_solve"):
        assert must in names


def test_library_builds_and_exports_every_symbol():
    from paper_2206_06996_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_tracks_header():
    from paper_2206_06996_gb300 import abi
    assert sorted(abi.EXPORTED) == declared_functions()


def test_default_options_without_gpu():
    # scr_default_opts touches no device
    from paper_2206_06996_gb300 import abi
    lib = abi.load_library(build_if_missing=True)
    o = abi.Opts()
    assert lib.scr_default_opts(ctypes.byref(o)) == 0
    assert o.rtol == 1e-8 and o.restart == 30 and o.rtol_A == 1e-3 and o.max_it == 200
    # the defaults the header documents for the GPU-side choices
    assert (o.vec, o.pdl, o.l2_prefetch, o.cuda_graphs, o.graph_krylov) == (1, 1, 192, 1, 2)
    assert (o.mapped_scalars, o.tangent_resetup, o.newton, o.nrhs) == (1, 1, 0, 1)
    assert (o.inner_vcycles, o.inter_vcycles, o.amg_coarse_bf16) == (0, 0, 1)
    assert lib.scr_default_opts(None) == abi.SCR_INVALID_ARG


def test_options_struct_layout_matches_header():
    from paper_2206_06996_gb300 import abi
    src = open(HEADER).read()
    body = src[src.index("typedef struct {\n  double rtol;"):]
    body = body[: body.index("} scr_opts;")]
    fields = re.findall(r"\b(\w+)\s*;", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    decl = []
    for line in re.sub(r"/\*.*?\*/", "", body, flags=re.S).splitlines():
        line = line.strip().rstrip(";")
        if not line or line.startswith("typedef"):
            continue
        parts = line.split(None, 1)
        if len(parts) == 2:
            decl.extend(v.strip() for v in parts[1].split(","))
    assert [f for f, _ in abi.Opts._fields_] == decl, (decl, fields)


def test_tune_file_round_trip_without_gpu(tmp_path):
    """scr_tune_load / scr_tune_save: decisions read from a file come back
    out unchanged; malformed files and invalid kernel codes are rejected."""
    import paper_2206_06996_gb300 as pkg
    good = tmp_path / "tune.txt"
    good.write_text("# comment\n9044975 616337 616337 3 3 8 1 102\n620434 616337 76959 3 3 4 1 101\n")
    pkg.tune_load(str(good))
    out = tmp_path / "out.txt"
    pkg.tune_save(str(out))
    lines = [l.split() for l in out.read_text().splitlines() if not l.startswith("#")]
    assert ["9044975", "616337", "616337", "3", "3", "8", "1", "102"] in lines
    assert ["620434", "616337", "76959", "3", "3", "4", "1", "101"] in lines
    for bad in ("1 2 3\n", "10 10 10 3 3 8 1 150\n", "10 -1 10 3 3 8 1 101\n"):
        f = tmp_path / "bad.txt"
        f.write_text(bad)
        with pytest.raises(pkg.ScrError):
            pkg.tune_load(str(f))
    with pytest.raises(pkg.ScrError):
        pkg.tune_load(str(tmp_path / "missing.txt"))


def _struct_fields(src: str, start: str, end: str) -> list:
    body = src[src.index(start):]
    body = body[: body.index(end)]
    decl = []
    for line in re.sub(r"/\*.*?\*/", "", body, flags=re.S).splitlines():
        line = line.strip().rstrip(";")
        if not line or line.startswith("typedef"):
            continue
        m = re.match(r"(long long|double|int|float)\s+(.*)", line)
        if m:
            decl.extend(v.strip() for v in m.group(2).split(","))
    return decl


def test_stats_struct_layout_matches_header():
    from paper_2206_06996_gb300 import abi
    src = open(HEADER).read()
    decl = _struct_fields(src, "typedef struct {\n  int outer_iters;", "} scr_stats;")
    assert [f for f, _ in abi.Stats._fields_] == decl
    assert "pc_graph_runs" in decl
