"""Host index structures of the library (csrc/host_mesh.cpp) against the
oracle, on the CPU.

A small C++ driver, compiled here against host_mesh.cpp, prints the vertex
patches (rules R1 and R2), on an h level the smoothed skeleton DOFs and the
macro patches, and the entity-shared CSR operator's column lists (column
entities expanded to DOFs by the same range rule the device uses).
The oracle gives the same objects from its own definitions: the patch rules of
Sec. 3 ("V-cycle and smoother") from entity centres and adjacency, and the
sparsity of the assembled condensed operator from the element DOF maps.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.assembly import build_fine
from oracle.hierarchy import PATCH_RULES, _p_injection, _p_selection, build_hierarchy
from oracle.mesh import Mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_01728_gb300", "csrc")

DRIVER = r"""
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include "host_mesh.h"
using namespace dpgmg;
int main(int argc, char** argv) {
  int n[3] = {atoi(argv[1]), atoi(argv[2]), atoi(argv[3])};
  const int p = atoi(argv[4]);
  double a[3] = {0, 0, 0}, b[3] = {1, 1, 1};
  MeshL m;
  m.init(n, p, a, b);
  std::vector<std::vector<int64_t>> groups(m.nelem);
  std::vector<int64_t> ent(m.loc.size());
  for (int64_t e = 0; e < m.nelem; ++e) {
    m.elem_entities(e, ent.data());
    for (int64_t E : ent)
      if (E >= 0) groups[e].push_back(E);
    std::sort(groups[e].begin(), groups[e].end());
    groups[e].erase(std::unique(groups[e].begin(), groups[e].end()), groups[e].end());
  }
  if (p > 1) {   // p transition to p - 1 on the same mesh
    MeshL mc;
    mc.init(n, p - 1, a, b);
    std::vector<int32_t> sel, inj;
    p_selection(p, sel);
    p_injection(m, mc, inj);
    printf("selection %d\n%zu", 1, sel.size());
    for (int32_t v : sel) printf(" %d", v);
    printf("\ninjection %d\n%zu", 1, inj.size());
    for (int32_t v : inj) printf(" %d", v);
    printf("\n");
  }
  std::vector<char> sm(m.ndof, 1);
  for (int r2 = 0; r2 < 2; ++r2) {
    Patches P = build_patches(m, sm, 2, n, r2 != 0);
    std::vector<int64_t> ps = patch_sizes(m, false, 2, n, r2 != 0);   // the memory estimate's sizes
    printf("psizes %d 1\n%zu", r2, ps.size());
    for (int64_t v : ps) printf(" %lld", (long long)v);
    printf("\n");
    printf("patches %d %zu\n", r2, P.ptr.size() - 1);
    for (size_t j = 0; j + 1 < P.ptr.size(); ++j) {
      printf("%lld", (long long)(P.ptr[j + 1] - P.ptr[j]));
      for (int64_t q = P.ptr[j]; q < P.ptr[j + 1]; ++q) printf(" %d", P.dofs[q]);
      printf("\n");
    }
  }
  if (argc > 5 && n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0) {   // h transition to n / 2
    int nc[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    MeshL mc;
    mc.init(nc, p, a, b);
    MacroHost M = build_macro(m, mc);
    printf("smask 1\n%lld", (long long)m.ndof);
    for (int64_t g = 0; g < m.ndof; ++g) printf(" %d", (int)M.smask[g]);
    printf("\n");
    printf("inclusion %lld\n", (long long)m.ndof);   // rows of P: count, then (column, value) pairs
    for (int64_t g = 0; g < m.ndof; ++g) {
      printf("%lld", (long long)(2 * (M.P_ptr[g + 1] - M.P_ptr[g])));
      for (int64_t q = M.P_ptr[g]; q < M.P_ptr[g + 1]; ++q)
        printf(" %d %lld", M.P_col[q], (long long)llround(M.P_val[q] * 1099511627776.0));   // value x 2^40
      printf("\n");
    }
    std::vector<char> s2(M.smask.begin(), M.smask.end());
    for (int r2 = 0; r2 < 2; ++r2) {
      Patches P = build_patches(m, s2, 4, nc, r2 != 0);
      std::vector<int64_t> ps = patch_sizes(m, true, 4, nc, r2 != 0);
      printf("msizes %d 1\n%zu", r2, ps.size());
      for (int64_t v : ps) printf(" %lld", (long long)v);
      printf("\n");
      printf("macro %d %zu\n", r2, P.ptr.size() - 1);
      for (size_t j = 0; j + 1 < P.ptr.size(); ++j) {
        printf("%lld", (long long)(P.ptr[j + 1] - P.ptr[j]));
        for (int64_t q = P.ptr[j]; q < P.ptr[j + 1]; ++q) printf(" %d", P.dofs[q]);
        printf("\n");
      }
    }
  }
  ECSRHost H = build_ecsr(m, groups);
  printf("ecsr %lld\n", (long long)m.ndof);
  for (int64_t r = 0; r < m.ndof; ++r) {
    const int32_t E = H.row_ent[r];
    if (E < 0) { printf("0\n"); continue; }
    std::vector<int64_t> cols;
    for (int64_t q = H.cent_ptr[E]; q < H.cent_ptr[E + 1]; ++q) {
      int64_t s;
      int nd;
      H.er.range(H.col_ent[q], &s, &nd);
      for (int k = 0; k < nd; ++k) cols.push_back(s + k);
    }
    if ((int64_t)cols.size() != H.col_ptr[E + 1] - H.col_ptr[E]) return 3;
    printf("%zu", cols.size());
    for (int64_t c : cols) printf(" %lld", (long long)c);
    printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("hostidx")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-O1", "-std=c++17", "-pthread", "-I", CSRC, str(src),
                    os.path.join(CSRC, "host_mesh.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def run_driver(exe, n, p, macro=False):
    args = [exe, str(n[0]), str(n[1]), str(n[2]), str(p)] + (["macro"] if macro else [])
    out = subprocess.run(args, check=True, capture_output=True, text=True).stdout.split("\n")
    res, i = {}, 0
    while i < len(out):
        head = out[i].split()
        if not head:
            i += 1
            continue
        cnt = int(head[-1])
        rows = []
        for line in out[i + 1:i + 1 + cnt]:
            v = [int(x) for x in line.split()]
            assert v[0] == len(v) - 1
            rows.append(np.array(v[1:], dtype=np.int64))
        res[tuple(head[:-1])] = rows
        i += 1 + cnt
    return res


@pytest.mark.parametrize("n,p", [((4, 4, 4), 2), ((3, 2, 4), 3), ((2, 3, 2), 1)])
def test_patches_and_operator_pattern_match_oracle(driver, n, p):
    got = run_driver(driver, n, p)
    mesh = Mesh(n, p)
    table = mesh.dof_table()
    smask = np.ones(mesh.n_dof, dtype=bool)
    for r2, rule in ((0, "R1"), (1, "R2")):
        ref = PATCH_RULES[rule](mesh, mesh, table, "p", smask)
        mine = got[("patches", str(r2))]
        assert len(mine) == len(ref)
        # the sizes the memory estimate uses (dpgmg_query_sizes) are those of the built patches
        assert np.array_equal(got[("psizes", str(r2))][0], [len(x) for x in ref])
        for a, b in zip(mine, ref):
            assert np.array_equal(a, b)
    if p > 1:   # p transition: local selection and the coarse -> fine injection
        assert np.array_equal(got[("selection",)][0], _p_selection(p))
        assert np.array_equal(got[("injection",)][0], _p_injection(mesh, Mesh(n, p - 1)))
    fs = build_fine(n, p, 3.0)
    A, _ = fs.assemble()
    A = A.tocsr()
    rows = got[("ecsr",)]
    assert len(rows) == mesh.n_dof
    for r in range(mesh.n_dof):
        ref = np.sort(A.indices[A.indptr[r]:A.indptr[r + 1]])
        assert np.array_equal(rows[r], ref), r


@pytest.mark.parametrize("n,p", [((4, 4, 4), 2), ((4, 2, 4), 1)])
def test_macro_smoothing_space_and_patches_match_oracle(driver, n, p):
    """h level: the smoothed DOFs (the coarse elements' skeleton) and the macro
    vertex patches (coarse element width 4 in doubled fine units) under both
    rules, against the oracle's hierarchy on the same mesh."""
    got = run_driver(driver, n, p, macro=True)
    fs = build_fine(n, p, 3.0)
    mask = got[("smask",)][0].astype(bool)
    for r2, rule in ((0, "R1"), (1, "R2")):
        levels = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, n_levels=2, p_min=p, patch_rule=rule)
        lev = levels[1]
        assert lev.kind == "h"
        assert np.array_equal(mask, lev.smask)
        if r2 == 0:   # natural inclusion P (fine x coarse): two-scale tables against the oracle's fit
            Pref = lev.P.tocsr()
            Pref.sort_indices()
            rows = got[("inclusion",)]
            assert len(rows) == Pref.shape[0]
            for g, row in enumerate(rows):
                cols, vals = row[0::2], row[1::2] / 2.0 ** 40
                keep = np.abs(Pref.data[Pref.indptr[g]:Pref.indptr[g + 1]]) > 1e-12
                rc = Pref.indices[Pref.indptr[g]:Pref.indptr[g + 1]][keep]
                rv = Pref.data[Pref.indptr[g]:Pref.indptr[g + 1]][keep]
                assert np.array_equal(cols, rc), g
                assert np.allclose(vals, rv, rtol=0, atol=1e-11), g
        mine = got[("macro", str(r2))]
        assert len(mine) == len(lev.patches)
        assert np.array_equal(got[("msizes", str(r2))][0], [len(x) for x in lev.patches])
        for a, b in zip(mine, lev.patches):
            assert np.array_equal(a, b)
