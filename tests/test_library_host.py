"""Host-side checks of the C ABI library (no GPU needed).

The library must build for sm_103a, load, and export every entry point that
include/dpgmg.h declares; no compute call is made here.
"""
import ctypes
import os
import re

import numpy as np
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
    # rule R2 blocks are smaller at the boundary: less patch storage
    nt2, _, nb2 = dpgmg.dpgmg_query_sizes(pb, dpgmg.make_opts(**dict(w["opts"], flags=dpgmg.FLAG_PATCH_R2)))
    assert nt2 == nt and nb2 < nb
    with pytest.raises(dpgmg.DpgmgError):
        dpgmg.dpgmg_query_sizes(pb, dpgmg.make_opts(**dict(w["opts"], flags=1 << 20)))
    # recomputed patches: no stored inverses in the estimate; mixed FP32 factors only
    _, _, nb3 = dpgmg.dpgmg_query_sizes(pb, dpgmg.make_opts(**dict(w["opts"], flags=dpgmg.FLAG_RECOMPUTE_PATCHES)))
    assert nb3 < nb
    for bad in [dict(precision="fp64"), dict(flags=dpgmg.FLAG_RECOMPUTE_PATCHES | dpgmg.FLAG_PATCH_FP64),
                dict(flags=dpgmg.FLAG_RECOMPUTE_PATCHES | dpgmg.FLAG_CG_C128)]:
        o = dict(w["opts"], flags=dpgmg.FLAG_RECOMPUTE_PATCHES)
        o.update(bad)
        with pytest.raises(dpgmg.DpgmgError):
            dpgmg.dpgmg_query_sizes(pb, dpgmg.make_opts(**o))
    pb.dp = 2
    with pytest.raises(dpgmg.DpgmgError):
        dpgmg.dpgmg_query_sizes(pb, dpgmg.make_opts(**w["opts"]))


def test_struct_layouts_match_header(libpath, tmp_path):
    # every field offset and struct size of the binding's ctypes mirrors against
    # the C compiler's view of include/dpgmg.h
    import shutil
    import subprocess
    from paper_2304_01728_gb300 import dpgmg
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = [dpgmg.dpgmg_problem, dpgmg.dpgmg_opts, dpgmg.dpgmg_stats, dpgmg.dpgmg_level_desc]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dpgmg.h"', 'int main(void) {']
    expect = []
    for st in structs:
        name = st.__name__
        lines.append('printf("%%zu\\n", sizeof(%s));' % name)
        expect.append(ctypes.sizeof(st))
        for fname, _ in st._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (name, fname))
            expect.append(getattr(st, fname).offset)
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect


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


@pytest.mark.parametrize("n,p", [((3, 2, 4), 2), ((1, 2, 1), 4)])
def test_boundary_points_are_the_oracle_face_rule(libpath, n, p):
    # the documented order (sides (d, s), faces j1 fastest, points a fastest)
    # at the oracle's boundary load rule: Gauss-Legendre with p + 5 points
    from oracle.basis import gauss01
    from paper_2304_01728_gb300 import dpgmg
    x0, x1 = np.array([0.5, -1.0, 0.0]), np.array([2.0, 1.0, 3.0])
    pb, keep = dpgmg.make_problem(n=n, p=p, omega=3.0, x0=tuple(x0), x1=tuple(x1))
    pts = dpgmg.dpgmg_boundary_points(pb)
    xg, _ = gauss01(p + 5)
    h = (x1 - x0) / np.asarray(n)
    ref = []
    for d in range(3):
        t1, t2 = [e for e in range(3) if e != d]
        for s in range(2):
            for j2 in range(n[t2]):
                for j1 in range(n[t1]):
                    for b in xg:
                        for a in xg:
                            X = np.zeros(3)
                            X[d] = x1[d] if s else x0[d]
                            X[t1] = x0[t1] + (j1 + a) * h[t1]
                            X[t2] = x0[t2] + (j2 + b) * h[t2]
                            ref.append(X)
    ref = np.array(ref)
    assert pts.shape == ref.shape
    assert np.abs(pts - ref).max() < 1e-13


def test_binding_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the public structs have the C compiler's size and
    field offsets (a field added to one side only would shift every later one)."""
    import shutil
    import subprocess
    from paper_2304_01728_gb300 import dpgmg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [dpgmg.dpgmg_problem, dpgmg.dpgmg_opts, dpgmg.dpgmg_stats, dpgmg.dpgmg_level_desc]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dpgmg.h"', "int main(void) {"]
    for S in structs:
        t = S.__name__
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (t, t))
        for f in S._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (t, f[0], t, f[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for S in structs:
        t = S.__name__
        assert got[(t, "sizeof")] == ctypes.sizeof(S), t
        for f in S._fields_:
            assert got[(t, f[0])] == getattr(S, f[0]).offset, (t, f[0])
