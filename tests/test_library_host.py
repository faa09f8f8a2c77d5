"""Host-side checks of the C ABI library (no GPU needed).

The library must build for sm_103a, load, and export every entry point that
include/dpgmg.h declares; no compute call is made here.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dpgmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dpgmg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2304_01728_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_abi(libpath):
    from paper_2304_01728_gb300 import dpgmg
    assert set(declared_functions()) <= set(dpgmg.EXPORTS)
    L = dpgmg.lib()
    assert L.dpgmg_strerror(-2).decode() == "device memory budget exceeded"
    op = dpgmg.make_opts()
    assert op.tol == 1e-8 and op.nu_pre == 1 and op.nu_post == 1


def test_query_sizes_without_device(libpath):
    from paper_2304_01728_gb300 import dpgmg, workloads
    w = workloads.config2()
    pb, keep = dpgmg.make_problem(**w["problem"])
    nt, nf, nb = dpgmg.dpgmg_query_sizes(pb, dpgmg.make_opts(**w["opts"]))
    assert nt == 188561 and nf == 4096 * 4 * 27
    assert nb > 1e9
    pb.dp = 2
    with pytest.raises(dpgmg.DpgmgError):
        dpgmg.dpgmg_query_sizes(pb, dpgmg.make_opts(**w["opts"]))


def test_struct_layouts_match_header(libpath):
    from paper_2304_01728_gb300 import dpgmg
    # sizes of the ABI structs on LP64 (x86_64 and aarch64 agree)
    assert ctypes.sizeof(dpgmg.dpgmg_problem) == 176
    assert ctypes.sizeof(dpgmg.dpgmg_opts) == 48
    assert ctypes.sizeof(dpgmg.dpgmg_stats) == 64
    assert ctypes.sizeof(dpgmg.dpgmg_level_desc) == 88


@pytest.mark.parametrize("n,p", [((3, 2, 4), 3), ((2, 2, 2), 1), ((1, 3, 2), 5)])
def test_dof_map_matches_the_oracle_numbering(libpath, n, p):
    """dpgmg_dof_map (host only) against the oracle's own DOF table: entity
    kind, doubled centre and modes of every global trace DOF, in order."""
    import numpy as np
    from oracle.mesh import Mesh
    from paper_2304_01728_gb300 import dpgmg
    pb, keep = dpgmg.make_problem(n=n, p=p, omega=3.0)
    nt, _, _ = dpgmg.dpgmg_query_sizes(pb, dpgmg.make_opts())
    got = dpgmg.dpgmg_dof_map(pb, nt)
    tab = Mesh(n, p).dof_table()
    assert len(tab) == nt
    kinds = {"v": 0, "e": 1, "f": 2, "u": 3}
    for g, (k, ctr, modes) in enumerate(tab):
        row = got[g]
        assert row[0] == kinds[k] and tuple(row[1:4]) == tuple(ctr), (g, row, k, ctr)
        if k == "v":
            assert tuple(row[4:]) == (-1, -1, -1)
        elif k == "e":
            assert tuple(row[4:6]) == modes and row[6] == -1, (g, row, modes)
        else:
            assert tuple(row[4:]) == modes, (g, row, modes)
    with pytest.raises(dpgmg.DpgmgError):
        dpgmg.dpgmg_dof_map(pb, nt + 1)
