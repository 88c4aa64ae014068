"""The C-ABI library loads and exports every entry point include/bidomain.h
declares; host-only calls (defaults, status strings) work without a GPU."""
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bidomain.h")
GOLD = os.path.join(ROOT, "tests", "golden", "gamg_appendix_a.json")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?[\s\*]+([A-Za-z_]\w*)\s*\([^;{]*\)\s*;",
                       src, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("BD_")))


@pytest.fixture(scope="module")
def L():
    from paper_2311_13914_gb300 import _build, binding

    _build.build()
    return binding


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("bd_assemble", "amg_setup", "amg_solve", "bd_step", "amg_setup_from_csr",
                 "amg_vcycle", "bd_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) == set(L.EXPORTS)


def test_defaults_follow_appendix_a(L):
    gold = json.load(open(GOLD))
    o = L.amg_options_default()
    assert o.theta == gold["threshold"]
    assert o.coarse_eq_limit == gold["coarse_eq_limit"]
    assert o.cheb_degree == gold["mg_levels_ksp_max_it"]
    assert o.esteig_steps == gold["esteig_ksp_max_it"]
    assert (o.eig_lo, o.eig_hi) == (gold["chebyshev_esteig"][1], gold["chebyshev_esteig"][3])
    # App. A squares the first level's graph; the default squares every level
    assert o.square_levels >= gold["square_graph"]
    s = L.solve_options_default()
    assert s.rtol == 1e-8 and s.max_it > 0 and s.warm_start == 0


def test_defaults_match_oracle(L, oracle_lib):
    o = L.amg_options_default()
    d = oracle_lib.DEFAULT_OPTS
    for k in ("theta", "coarse_eq_limit", "max_levels", "cheb_degree", "esteig_steps", "eig_lo",
              "eig_hi", "seed", "square_levels"):
        assert getattr(o, k) == d[k], k
    assert o.precision == 0  # the plain FP64 form is the default
    assert o.autotune == 0   # lanes from the row-length rule unless asked
    rm = L.bd_rm_params_default()
    for k, v in oracle_lib.RM_PARAMS.items():
        assert getattr(rm, k) == v


def test_strerror_names_every_status(L):
    for st in range(0, -10, -1):
        assert L.strerror(st) != "unknown status"
    assert L.strerror(-99) == "unknown status"


def test_struct_layouts_match_header(L):
    import ctypes as C

    # field order and sizes of the public structs (all naturally aligned)
    assert C.sizeof(L.Mesh) == 3 * 4 + 4 + 3 * 8
    assert C.sizeof(L.Params) == 7 * 8
    assert C.sizeof(L.AmgOptions) == 8 + 5 * 4 + 4 + 2 * 8 + 8 + 4 + 4
    assert C.sizeof(L.SolveOptions) == 8 + 3 * 4 + 4
    assert C.sizeof(L.SolveInfo) == 2 * 4 + 3 * 8 + 8
    assert C.sizeof(L.KernelProfile) == 8 + 3 * 8 + 4 + 4 + 8
    assert [f for f, _ in L.KernelProfile._fields_] == ["launches", "total_ms", "bytes", "flops",
                                                        "precision", "fp64_ops"]
