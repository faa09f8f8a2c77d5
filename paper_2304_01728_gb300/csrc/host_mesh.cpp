// Host-side mesh, numbering and multigrid index structures (see host_mesh.h).
#include "host_mesh.h"

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <stdexcept>
#include <thread>
#include <tuple>

namespace dpgmg {

// ---------------------------------------------------------------- 1D bases
static void legendre_all(int nmax, double x, double* P, double* dP) {
  // L_a(x) = P_a(2x - 1) and d/dx, by Bonnet's recurrence in xi = 2x - 1
  double xi = 2.0 * x - 1.0;
  P[0] = 1.0;
  dP[0] = 0.0;
  if (nmax >= 1) { P[1] = xi; dP[1] = 1.0; }
  for (int k = 1; k < nmax; ++k) {
    P[k + 1] = ((2 * k + 1) * xi * P[k] - k * P[k - 1]) / (k + 1);
    dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k];
  }
  for (int k = 0; k <= nmax; ++k) dP[k] *= 2.0;
}

static void h1_all(int p, double x, double* V, double* D) {
  std::vector<double> P(p + 2), dP(p + 2);
  legendre_all(std::max(p, 1), x, P.data(), dP.data());
  V[0] = 1.0 - x; D[0] = -1.0;
  if (p >= 1) { V[1] = x; D[1] = 1.0; }
  for (int k = 2; k <= p; ++k) {
    double s = std::sqrt(2.0 * (2 * k - 1));
    V[k] = (P[k] - P[k - 2]) / s;
    D[k] = (dP[k] - dP[k - 2]) / s;
  }
}

void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  // Newton iteration on P_n from Chebyshev-like initial guesses
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged root
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
      double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1);
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) { p1 = z; p0 = 1.0; }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);   // 2/((1-z^2)P'^2) scaled by 1/2
  }
}

Tables1D make_tables(int p) {
  Tables1D t;
  t.p = p;
  t.pt = p + 1;
  int pt = t.pt;
  int n1 = pt + 1;
  t.nql = pt + 4;
  std::vector<double> xg, wg;
  gauss_legendre01(pt + 3, xg, wg);
  t.Mleg.resize(n1);
  for (int a = 0; a < n1; ++a) t.Mleg[a] = 1.0 / (2 * a + 1);
  t.D.assign(n1 * n1, 0.0);
  t.S.assign(n1 * n1, 0.0);
  t.Phi.assign((p + 1) * n1, 0.0);
  std::vector<double> P(n1 + 1), dP(n1 + 1), V(p + 2), DV(p + 2);
  for (size_t q = 0; q < xg.size(); ++q) {
    legendre_all(pt, xg[q], P.data(), dP.data());
    h1_all(p, xg[q], V.data(), DV.data());
    for (int a = 0; a < n1; ++a)
      for (int b = 0; b < n1; ++b) {
        t.D[a * n1 + b] += wg[q] * dP[a] * P[b];
        t.S[a * n1 + b] += wg[q] * dP[a] * dP[b];
      }
    for (int k = 0; k <= p; ++k)
      for (int b = 0; b < n1; ++b) t.Phi[k * n1 + b] += wg[q] * V[k] * P[b];
  }
  t.phi_end.assign((p + 1) * 2, 0.0);
  t.phi_end[0 * 2 + 0] = 1.0;
  if (p >= 1) t.phi_end[1 * 2 + 1] = 1.0;
  gauss_legendre01(t.nql, t.xq, t.wq);
  t.Lq.assign(n1 * t.nql, 0.0);
  for (int q = 0; q < t.nql; ++q) {
    legendre_all(pt, t.xq[q], P.data(), dP.data());
    for (int a = 0; a < n1; ++a) t.Lq[a * t.nql + q] = P[a];
  }
  return t;
}

// -------------------------------------------------------- local functions
std::vector<LocFn> local_trace_functions(int p) {
  std::vector<LocFn> out;
  for (int c = 0; c <= p; ++c)
    for (int b = 0; b <= p; ++b)
      for (int a = 0; a <= p; ++a)
        if (std::min(a, std::min(b, c)) < 2) {
          LocFn f{};
          f.type = 0;
          f.idx[0] = a; f.idx[1] = b; f.idx[2] = c;
          out.push_back(f);
        }
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s)
      for (int b = 0; b < p; ++b)
        for (int a = 0; a < p; ++a) {
          LocFn f{};
          f.type = 1; f.d = d; f.s = s; f.a = a; f.b = b;
          out.push_back(f);
        }
  return out;
}

int n_trace_local(int p) { return (p + 1) * (p + 1) * (p + 1) - (p - 1) * (p - 1) * (p - 1) + 6 * p * p; }

static void tang(int d, int& t1, int& t2) {
  t1 = d == 0 ? 1 : 0;
  t2 = d == 2 ? 1 : 2;
}

// ------------------------------------------------------------------- mesh
void MeshL::init(const int nn[3], int pp, const double a[3], const double b[3]) {
  p = pp;
  nelem = 1;
  for (int d = 0; d < 3; ++d) {
    n[d] = nn[d];
    x0[d] = a[d];
    x1[d] = b[d];
    h[d] = (b[d] - a[d]) / nn[d];
    nelem *= nn[d];
  }
  nV = (int64_t)(n[0] + 1) * (n[1] + 1) * (n[2] + 1);
  nE = nF = nFi = 0;
  for (int d = 0; d < 3; ++d) {
    int64_t e = 1, f = 1, fi = 1;
    for (int k = 0; k < 3; ++k) {
      e *= n[k] + (k != d);
      f *= n[k] + (k == d);
      fi *= n[k] - (k == d);
    }
    nEd[d] = e;
    nFd[d] = f;
    nFid[d] = fi;
    nE += e;
    nF += f;
    nFi += fi;
  }
  offE = nV;
  offF = offE + nE * (p - 1);
  offU = offF + nF * (int64_t)(p - 1) * (p - 1);
  ndof = offU + nFi * (int64_t)p * p;
  entE = nV;
  entF = entE + nE;
  entU = entF + nF;
  nent = entU + nFi;
  loc = local_trace_functions(p);
}

int64_t MeshL::vertex(const int c[3]) const {
  int64_t ext[3] = {n[0] + 1, n[1] + 1, n[2] + 1};
  return lin(c, ext);
}
int64_t MeshL::edge(int d, const int c[3]) const {
  int64_t ext[3];
  for (int k = 0; k < 3; ++k) ext[k] = n[k] + (k != d);
  int64_t off = 0;
  for (int k = 0; k < d; ++k) off += nEd[k];
  return off + lin(c, ext);
}
int64_t MeshL::face(int d, const int c[3]) const {
  int64_t ext[3];
  for (int k = 0; k < 3; ++k) ext[k] = n[k] + (k == d);
  int64_t off = 0;
  for (int k = 0; k < d; ++k) off += nFd[k];
  return off + lin(c, ext);
}
int64_t MeshL::iface(int d, const int c[3]) const {
  int64_t ext[3];
  for (int k = 0; k < 3; ++k) ext[k] = n[k] - (k == d);
  int cc[3] = {c[0], c[1], c[2]};
  cc[d] -= 1;
  int64_t off = 0;
  for (int k = 0; k < d; ++k) off += nFid[k];
  return off + lin(cc, ext);
}

void MeshL::elem_dofs(int64_t e, int64_t* out) const {
  int ec[3];
  elem_coord(e, ec);
  for (size_t li = 0; li < loc.size(); ++li) {
    const LocFn& f = loc[li];
    if (f.type == 0) {
      int pos[3], nv = 0, bd = -1, vd = -1;
      for (int d = 0; d < 3; ++d) {
        if (f.idx[d] < 2) { pos[d] = ec[d] + f.idx[d]; ++nv; vd = d; }
        else { pos[d] = ec[d]; bd = d; }
      }
      if (nv == 3) out[li] = vertex(pos);
      else if (nv == 2) out[li] = offE + edge(bd, pos) * (p - 1) + (f.idx[bd] - 2);
      else {
        int t1, t2;
        tang(vd, t1, t2);
        out[li] = offF + face(vd, pos) * (int64_t)(p - 1) * (p - 1) + (f.idx[t1] - 2) +
                  (int64_t)(p - 1) * (f.idx[t2] - 2);
      }
    } else {
      int pos[3] = {ec[0], ec[1], ec[2]};
      pos[f.d] += f.s;
      if (boundary_face(f.d, pos)) out[li] = -1;
      else out[li] = offU + iface(f.d, pos) * (int64_t)p * p + f.a + (int64_t)p * f.b;
    }
  }
}

void MeshL::elem_entities(int64_t e, int64_t* out) const {
  int ec[3];
  elem_coord(e, ec);
  for (size_t li = 0; li < loc.size(); ++li) {
    const LocFn& f = loc[li];
    int ctr[3];
    if (f.type == 0) {
      for (int d = 0; d < 3; ++d) ctr[d] = 2 * ec[d] + (f.idx[d] < 2 ? 2 * f.idx[d] : 1);
      out[li] = entity_at(ctr, false);
    } else {
      int t1, t2;
      tang(f.d, t1, t2);
      ctr[f.d] = 2 * (ec[f.d] + f.s);
      ctr[t1] = 2 * ec[t1] + 1;
      ctr[t2] = 2 * ec[t2] + 1;
      out[li] = entity_at(ctr, true);
    }
  }
}

int64_t MeshL::entity_at(const int ctr[3], bool uhat) const {
  int odd[3], nodd = 0;
  int c[3];
  for (int d = 0; d < 3; ++d) {
    odd[d] = ctr[d] & 1;
    nodd += odd[d];
    c[d] = ctr[d] >> 1;
  }
  if (uhat) {
    if (nodd != 2) return -1;
    int d = !odd[0] ? 0 : (!odd[1] ? 1 : 2);
    if (boundary_face(d, c)) return -1;
    return entU + iface(d, c);
  }
  if (nodd == 0) return vertex(c);
  if (nodd == 1) {
    int d = odd[0] ? 0 : (odd[1] ? 1 : 2);
    return entE + edge(d, c);
  }
  if (nodd == 2) {
    int d = !odd[0] ? 0 : (!odd[1] ? 1 : 2);
    return entF + face(d, c);
  }
  return -1;
}

void MeshL::ent_range(int64_t E, int64_t* start, int* nd) const {
  if (E < entE) { *start = E; *nd = 1; }
  else if (E < entF) { *start = offE + (E - entE) * (p - 1); *nd = p - 1; }
  else if (E < entU) { *start = offF + (E - entF) * (int64_t)(p - 1) * (p - 1); *nd = (p - 1) * (p - 1); }
  else { *start = offU + (E - entU) * (int64_t)p * p; *nd = p * p; }
}

int64_t MeshL::dof_entity(int64_t g) const {
  if (g < offE) return g;
  if (g < offF) return entE + (g - offE) / (p - 1);
  if (g < offU) return entF + (g - offF) / ((int64_t)(p - 1) * (p - 1));
  return entU + (g - offU) / ((int64_t)p * p);
}

static void unlin(int64_t k, const int64_t ext[3], int c[3]) {
  c[0] = (int)(k % ext[0]);
  c[1] = (int)((k / ext[0]) % ext[1]);
  c[2] = (int)(k / (ext[0] * ext[1]));
}

void MeshL::ent_center(int64_t E, int ctr[3]) const {
  int c[3];
  if (E < entE) {
    int64_t ext[3] = {n[0] + 1, n[1] + 1, n[2] + 1};
    unlin(E, ext, c);
    for (int d = 0; d < 3; ++d) ctr[d] = 2 * c[d];
    return;
  }
  if (E < entF) {
    int64_t k = E - entE;
    int d = 0;
    while (k >= nEd[d]) { k -= nEd[d]; ++d; }
    int64_t ext[3];
    for (int q = 0; q < 3; ++q) ext[q] = n[q] + (q != d);
    unlin(k, ext, c);
    for (int q = 0; q < 3; ++q) ctr[q] = 2 * c[q] + (q == d);
    return;
  }
  if (E < entU) {
    int64_t k = E - entF;
    int d = 0;
    while (k >= nFd[d]) { k -= nFd[d]; ++d; }
    int64_t ext[3];
    for (int q = 0; q < 3; ++q) ext[q] = n[q] + (q == d);
    unlin(k, ext, c);
    for (int q = 0; q < 3; ++q) ctr[q] = 2 * c[q] + (q != d);
    return;
  }
  int64_t k = E - entU;
  int d = 0;
  while (k >= nFid[d]) { k -= nFid[d]; ++d; }
  int64_t ext[3];
  for (int q = 0; q < 3; ++q) ext[q] = n[q] - (q == d);
  unlin(k, ext, c);
  c[d] += 1;
  for (int q = 0; q < 3; ++q) ctr[q] = 2 * c[q] + (q != d);
}

// ----------------------------------------------------------------- levels
std::vector<LevelSpec> plan_levels(const int n[3], int p, int n_levels, int p_min) {
  std::vector<LevelSpec> out;
  LevelSpec s{};
  for (int d = 0; d < 3; ++d) s.n[d] = n[d];
  s.p = p;
  s.kind_below = 0;
  out.push_back(s);
  while ((int)out.size() < n_levels) {
    LevelSpec c = out.back();
    if (c.p > p_min) {
      out.back().kind_below = 1;
      c.p -= 1;
    } else if (c.n[0] % 2 == 0 && c.n[1] % 2 == 0 && c.n[2] % 2 == 0 && c.n[0] >= 2 &&
               c.n[1] >= 2 && c.n[2] >= 2) {
      out.back().kind_below = 2;
      for (int d = 0; d < 3; ++d) c.n[d] /= 2;
    } else {
      break;
    }
    c.kind_below = 0;
    out.push_back(c);
  }
  return out;
}

// ------------------------------------------------------------------- ECSR
// Number of host threads for a loop of n items: up to 16, at least 256 items each.
static int64_t host_threads(int64_t n) {
  const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
  return std::min<int64_t>({hw, (int64_t)16, std::max<int64_t>(1, n / 256)});
}

// Runs body(t, lo, hi) for t < nt over contiguous ranges of [0, n), one host
// thread each (nt = host_threads(n), or the given count).
template <class F>
static void parallel_chunks(int64_t n, int64_t nt, F&& body) {
  if (nt <= 1) {
    body((int64_t)0, (int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; ++t) th.emplace_back([&, t]() { body(t, n * t / nt, n * (t + 1) / nt); });
  for (auto& x : th) x.join();
}

// Runs body(lo, hi) over [0, n) in contiguous ranges on host_threads(n) threads.
template <class F>
static void parallel_ranges(int64_t n, F&& body) {
  parallel_chunks(n, host_threads(n), [&](int64_t, int64_t lo, int64_t hi) { body(lo, hi); });
}

void host_parallel(int64_t n, const std::function<void(int64_t, int64_t)>& body) { parallel_ranges(n, body); }

ECSRHost build_ecsr(const MeshL& m, const std::vector<std::vector<int64_t>>& groups) {
  ECSRHost A;
  A.nrows = m.ndof;
  // entity -> groups containing it (CSR)
  std::vector<int64_t> eg_ptr(m.nent + 1, 0);
  for (const auto& g : groups)
    for (int64_t E : g) ++eg_ptr[E + 1];
  for (int64_t E = 0; E < m.nent; ++E) eg_ptr[E + 1] += eg_ptr[E];
  std::vector<int32_t> eg(eg_ptr.back());
  {
    std::vector<int64_t> fill(eg_ptr.begin(), eg_ptr.end() - 1);
    for (size_t g = 0; g < groups.size(); ++g)
      for (int64_t E : groups[g]) eg[fill[E]++] = (int32_t)g;
  }
  // row entities in entity order
  std::vector<int64_t> rows;
  for (int64_t E = 0; E < m.nent; ++E) {
    if (eg_ptr[E + 1] == eg_ptr[E]) continue;
    int64_t st;
    int nd;
    m.ent_range(E, &st, &nd);
    if (nd > 0) rows.push_back(E);
  }
  const int64_t R = (int64_t)rows.size();
  // per row entity: sorted distinct column entities (a stamp per entity drops
  // repeats before the sort), kept per thread in one flat buffer, and the
  // row's column DOF count
  const int64_t nt = host_threads(R);
  std::vector<std::vector<int32_t>> buf((size_t)std::max<int64_t>(nt, 1));
  std::vector<int32_t> nb_cnt(R);
  std::vector<int64_t> ncol(R);
  parallel_chunks(R, nt, [&](int64_t t, int64_t lo, int64_t hi) {
    std::vector<int32_t> stamp(m.nent, -1);
    std::vector<int32_t> cols;
    std::vector<int32_t>& out = buf[t];
    for (int64_t r = lo; r < hi; ++r) {
      const int64_t E = rows[r];
      cols.clear();
      for (int64_t q = eg_ptr[E]; q < eg_ptr[E + 1]; ++q)
        for (int64_t F : groups[eg[q]])
          if (stamp[F] != (int32_t)r) {
            stamp[F] = (int32_t)r;
            cols.push_back((int32_t)F);
          }
      std::sort(cols.begin(), cols.end());
      int64_t c = 0;
      for (int32_t F : cols) {
        int64_t fs;
        int fn;
        m.ent_range(F, &fs, &fn);
        c += fn;
      }
      out.insert(out.end(), cols.begin(), cols.end());
      nb_cnt[r] = (int32_t)cols.size();
      ncol[r] = c;
    }
  });
  A.row_ent.assign(m.ndof, -1);
  A.ent_start.resize(R);
  A.ent_nd.resize(R);
  A.col_ptr.assign(R + 1, 0);
  A.val_ptr.assign(R + 1, 0);
  A.nnz_alg = 0;
  for (int64_t r = 0; r < R; ++r) {
    int64_t st;
    int nd;
    m.ent_range(rows[r], &st, &nd);
    A.ent_start[r] = st;
    A.ent_nd[r] = nd;
    A.col_ptr[r + 1] = A.col_ptr[r] + ncol[r];
    A.val_ptr[r + 1] = A.val_ptr[r] + ncol[r] * nd;
    A.nnz_alg += ncol[r] * nd;
    for (int k = 0; k < nd; ++k) A.row_ent[st + k] = (int32_t)r;
  }
  // column entity lists: the per-thread buffers in row order
  A.cent_ptr.assign(R + 1, 0);
  for (int64_t r = 0; r < R; ++r) A.cent_ptr[r + 1] = A.cent_ptr[r] + nb_cnt[r];
  A.col_ent.resize(A.cent_ptr[R]);   // left uninitialised (NoInitAlloc): every entry is written below
  parallel_chunks(R, nt, [&](int64_t t, int64_t lo, int64_t hi) {
    if (lo < hi) std::copy(buf[t].begin(), buf[t].end(), A.col_ent.begin() + A.cent_ptr[lo]);
  });
  A.er = EntRanges{m.entE, m.entF, m.entU, m.offE, m.offF, m.offU, m.p};
  return A;
}

// ------------------------------------------------------- boundary points
int64_t boundary_face_offsets(const int n[3], int64_t off[6]) {
  int64_t k = 0;
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    for (int s = 0; s < 2; ++s) {
      off[2 * d + s] = k;
      k += (int64_t)n[t1] * n[t2];
    }
  }
  return k;
}

void boundary_points(const int n[3], const double x0[3], const double x1[3], int p, std::vector<double>& xyz) {
  Tables1D T = make_tables(p);
  const int nq = T.nql;
  int64_t off[6];
  const int64_t nf = boundary_face_offsets(n, off);
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = (x1[d] - x0[d]) / n[d];
  xyz.assign((size_t)nf * nq * nq * 3, 0.0);
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    for (int s = 0; s < 2; ++s)
      for (int j2 = 0; j2 < n[t2]; ++j2)
        for (int j1 = 0; j1 < n[t1]; ++j1) {
          const int64_t f = off[2 * d + s] + j1 + (int64_t)n[t1] * j2;
          // the element stage's own expressions: element corner + s h, corner + x_q h
          const double cd = x0[d] + (s ? n[d] - 1 : 0) * h[d];
          const double c1 = x0[t1] + j1 * h[t1], c2 = x0[t2] + j2 * h[t2];
          for (int qb = 0; qb < nq; ++qb)
            for (int qa = 0; qa < nq; ++qa) {
              double* o = &xyz[(size_t)((f * nq + qb) * nq + qa) * 3];
              o[d] = cd + s * h[d];
              o[t1] = c1 + T.xq[qa] * h[t1];
              o[t2] = c2 + T.xq[qb] * h[t2];
            }
        }
  }
}

// ---------------------------------------------------------------- patches
// Coarse vertex indices along one axis whose patches take an entity with
// centre coordinate ctr (half-element units of the level's mesh, coarse
// element width H).  Off a coarse plane: the two planes around it.  On an
// interior coarse plane: that plane.  On a boundary plane, rule R1 (every
// adjacent (macro-)element has the vertex as a corner) also takes the plane
// one element inside; rule R2 (the vertex lies in the closure of the entity's
// coarse entity) takes the boundary plane only.
int patch_axis_span(int ctr, int H, int nco, bool r2, int W[2]) {
  const int top = H * nco;
  if (ctr % H != 0) {
    W[0] = ctr / H;
    W[1] = ctr / H + 1;
    return 2;
  }
  if (!r2 && ctr == 0) { W[0] = 0; W[1] = 1; return 2; }
  if (!r2 && ctr == top) { W[0] = nco - 1; W[1] = nco; return 2; }
  W[0] = ctr / H;
  return 1;
}

Patches build_patches(const MeshL& m, const std::vector<char>& smask, int H, const int nco[3], bool r2) {
  Patches P;
  const int64_t npatch = (int64_t)(nco[0] + 1) * (nco[1] + 1) * (nco[2] + 1);
  // Entities in order (their DOFs are consecutive and increasing with the
  // entity), split into contiguous ranges over host threads: pass 0 counts per
  // (thread, patch), pass 1 writes each thread's DOFs after those of the
  // threads before it, so every patch lists its DOFs in increasing order.
  const int64_t nt = host_threads(m.nent);
  std::vector<int64_t> cnt((size_t)(nt * npatch), 0);
  auto visit = [&](int64_t lo, int64_t hi, auto&& emit) {
    for (int64_t E = lo; E < hi; ++E) {
      int64_t st;
      int nd;
      m.ent_range(E, &st, &nd);
      if (nd == 0) continue;
      int ctr[3], W[3][2], c[3];
      m.ent_center(E, ctr);
      for (int d = 0; d < 3; ++d) c[d] = patch_axis_span(ctr[d], H, nco[d], r2, W[d]);
      for (int a = 0; a < c[0]; ++a)
        for (int b = 0; b < c[1]; ++b)
          for (int q = 0; q < c[2]; ++q) {
            const int64_t w = W[0][a] + (int64_t)(nco[0] + 1) * (W[1][b] + (int64_t)(nco[1] + 1) * W[2][q]);
            for (int k = 0; k < nd; ++k)
              if (smask[st + k]) emit(w, st + k);
          }
    }
  };
  parallel_chunks(m.nent, nt, [&](int64_t t, int64_t lo, int64_t hi) {
    int64_t* ct = cnt.data() + t * npatch;
    visit(lo, hi, [&](int64_t w, int64_t) { ++ct[w]; });
  });
  P.ptr.assign(npatch + 1, 0);
  for (int64_t w = 0; w < npatch; ++w) {   // cnt becomes each thread's first position in patch w
    int64_t acc = P.ptr[w];
    for (int64_t t = 0; t < nt; ++t) {
      const int64_t c = cnt[t * npatch + w];
      cnt[t * npatch + w] = acc;
      acc += c;
    }
    P.ptr[w + 1] = acc;
  }
  P.dofs.resize(P.ptr[npatch]);
  parallel_chunks(m.nent, nt, [&](int64_t t, int64_t lo, int64_t hi) {
    int64_t* fill = cnt.data() + t * npatch;
    visit(lo, hi, [&](int64_t w, int64_t g) { P.dofs[fill[w]++] = (int32_t)g; });
  });
  P.val_ptr.assign(npatch + 1, 0);
  for (int64_t j = 0; j < npatch; ++j) {
    int64_t nj = P.ptr[j + 1] - P.ptr[j];
    P.val_ptr[j + 1] = P.val_ptr[j] + nj * patch_ld(nj);
  }
  // slots of each DOF
  std::vector<int64_t> sc(m.ndof + 1, 0);
  for (int32_t g : P.dofs) ++sc[g + 1];
  for (int64_t g = 0; g < m.ndof; ++g) sc[g + 1] += sc[g];
  P.slot_ptr = sc;
  P.slots.assign(P.dofs.size(), 0);
  std::vector<int64_t> f(sc.begin(), sc.end() - 1);
  for (size_t k = 0; k < P.dofs.size(); ++k) P.slots[f[P.dofs[k]]++] = (int32_t)k;
  return P;
}

std::vector<int64_t> patch_sizes(const MeshL& m, bool macro, int H, const int nco[3], bool r2) {
  std::vector<int64_t> cnt((size_t)(nco[0] + 1) * (nco[1] + 1) * (nco[2] + 1), 0);
  for (int64_t E = 0; E < m.nent; ++E) {
    int64_t st;
    int nd;
    m.ent_range(E, &st, &nd);
    if (nd == 0) continue;
    int ctr[3];
    m.ent_center(E, ctr);
    if (macro) {   // entity on the skeleton of the coarse mesh (a flat coordinate on a coarse plane)
      bool on = false;
      for (int d = 0; d < 3; ++d)
        if (!(ctr[d] & 1) && ctr[d] % 4 == 0) on = true;
      if (!on) continue;
    }
    int W[3][2], c[3];
    for (int d = 0; d < 3; ++d) c[d] = patch_axis_span(ctr[d], H, nco[d], r2, W[d]);
    for (int a = 0; a < c[0]; ++a)
      for (int b = 0; b < c[1]; ++b)
        for (int q = 0; q < c[2]; ++q)
          cnt[W[0][a] + (int64_t)(nco[0] + 1) * (W[1][b] + (int64_t)(nco[1] + 1) * W[2][q])] += nd;
  }
  return cnt;
}

// ----------------------------------------------------------- transitions
void p_selection(int p, std::vector<int32_t>& sel) {
  auto fine = local_trace_functions(p);
  auto crs = local_trace_functions(p - 1);
  sel.clear();
  for (const LocFn& c : crs) {
    for (size_t i = 0; i < fine.size(); ++i) {
      const LocFn& f = fine[i];
      bool eq = f.type == c.type &&
                (f.type == 0 ? (f.idx[0] == c.idx[0] && f.idx[1] == c.idx[1] && f.idx[2] == c.idx[2])
                             : (f.d == c.d && f.s == c.s && f.a == c.a && f.b == c.b));
      if (eq) { sel.push_back((int32_t)i); break; }
    }
  }
}

void p_injection(const MeshL& mf, const MeshL& mc, std::vector<int32_t>& inj) {
  inj.assign(mc.ndof, -1);
  int pc = mc.p, pf = mf.p;
  for (int64_t g = 0; g < mc.ndof; ++g) {
    int64_t E = mc.dof_entity(g), st;
    int nd;
    mc.ent_range(E, &st, &nd);
    int64_t k = g - st;
    int ctr[3];
    mc.ent_center(E, ctr);
    bool uh = E >= mc.entU;
    int64_t Ef = mf.entity_at(ctr, uh), sf;
    int ndf;
    mf.ent_range(Ef, &sf, &ndf);
    int64_t off;
    if (E < mc.entE) off = 0;
    else if (E < mc.entF) off = k;                                    // mode 2 + k
    else if (E < mc.entU) {
      int64_t m1 = k % (pc - 1), m2 = k / (pc - 1);
      off = m1 + (int64_t)(pf - 1) * m2;
    } else {
      int64_t a = k % pc, b = k / pc;
      off = a + (int64_t)pf * b;
    }
    inj[g] = (int32_t)(sf + off);
  }
}

// Natural inclusion in 1D: coarse function phi^c_A on [0,1] expressed on the
// fine halves [0,1/2], [1/2,1].  Node values at 0, 1/2, 1 give the hat
// coefficients; bubble coefficients come from the Legendre expansion of the
// derivative (phi_m' = sqrt(2(2m-1)) P_{m-1}(2x-1)).
static double h1_val(int p, int A, double x) {
  std::vector<double> V(p + 2), D(p + 2);
  h1_all(p, x, V.data(), D.data());
  return V[A];
}
static double h1_bubble_coef(int p, int A, int hh, int m) {
  std::vector<double> xg, wg, V(p + 2), D(p + 2), P(p + 3), dP(p + 3);
  gauss_legendre01(p + 2, xg, wg);
  double acc = 0.0;
  for (size_t q = 0; q < xg.size(); ++q) {
    h1_all(p, 0.5 * (hh + xg[q]), V.data(), D.data());
    legendre_all(p, xg[q], P.data(), dP.data());
    acc += wg[q] * 0.5 * D[A] * P[m - 1];
  }
  return (2 * m - 1) * acc / std::sqrt(2.0 * (2 * m - 1));
}
static double leg_twoscale(int p, int a, int hh, int m) {
  std::vector<double> xg, wg, Pc(p + 2), dPc(p + 2), P(p + 2), dP(p + 2);
  gauss_legendre01(p + 2, xg, wg);
  double acc = 0.0;
  for (size_t q = 0; q < xg.size(); ++q) {
    legendre_all(std::max(p, 1), 0.5 * (hh + xg[q]), Pc.data(), dPc.data());
    legendre_all(std::max(p, 1), xg[q], P.data(), dP.data());
    acc += wg[q] * Pc[a] * P[m];
  }
  return (2 * m + 1) * acc;
}

namespace {
struct KDof { int ctr[3]; int kind; int m1, m2; bool bnd; };  // kind 0 v, 1 e, 2 f, 3 u
}

MacroHost build_macro(const MeshL& mf, const MeshL& mc) {
  MacroHost M;
  const int p = mf.p;
  // ---- K-local enumeration of the fine DOFs in a closed coarse element
  std::vector<KDof> kd;
  for (int pass = 0; pass < 2; ++pass)       // p-hat entities, then u-hat
    for (int cz = 0; cz <= 4; ++cz)
      for (int cy = 0; cy <= 4; ++cy)
        for (int cx = 0; cx <= 4; ++cx) {
          int c[3] = {cx, cy, cz};
          int nodd = (cx & 1) + (cy & 1) + (cz & 1);
          bool bnd = false;
          for (int d = 0; d < 3; ++d)
            if (!(c[d] & 1) && (c[d] == 0 || c[d] == 4)) bnd = true;
          KDof k{};
          for (int d = 0; d < 3; ++d) k.ctr[d] = c[d];
          k.bnd = bnd;
          if (pass == 0) {
            if (nodd == 0) { k.kind = 0; kd.push_back(k); }
            else if (nodd == 1) {
              for (int m = 2; m <= p; ++m) { k.kind = 1; k.m1 = m; kd.push_back(k); }
            } else if (nodd == 2) {
              for (int m2 = 2; m2 <= p; ++m2)
                for (int m1 = 2; m1 <= p; ++m1) { k.kind = 2; k.m1 = m1; k.m2 = m2; kd.push_back(k); }
            }
          } else if (nodd == 2) {
            for (int b = 0; b < p; ++b)
              for (int a = 0; a < p; ++a) { k.kind = 3; k.m1 = a; k.m2 = b; kd.push_back(k); }
          }
        }
  std::vector<int> order;
  for (size_t i = 0; i < kd.size(); ++i) if (kd[i].bnd) order.push_back((int)i);
  M.nS = (int)order.size();
  for (size_t i = 0; i < kd.size(); ++i) if (!kd[i].bnd) order.push_back((int)i);
  M.nI = (int)order.size() - M.nS;
  std::vector<KDof> kl;
  for (int i : order) kl.push_back(kd[i]);
  std::map<std::tuple<int, int, int, int, int, int>, int> key;
  for (size_t i = 0; i < kl.size(); ++i)
    key[std::make_tuple(kl[i].ctr[0], kl[i].ctr[1], kl[i].ctr[2], kl[i].kind, kl[i].m1, kl[i].m2)] = (int)i;

  // ---- child local -> K-local
  const auto& loc = mf.loc;
  M.nloc_f = (int)loc.size();
  M.child_map.assign(8 * loc.size(), -1);
  for (int o = 0; o < 8; ++o) {
    int oc[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
    for (size_t li = 0; li < loc.size(); ++li) {
      const LocFn& f = loc[li];
      int c[3], kind, m1 = 0, m2 = 0;
      if (f.type == 0) {
        int nv = 0, bd = -1, vd = -1;
        for (int d = 0; d < 3; ++d) {
          if (f.idx[d] < 2) { c[d] = 2 * oc[d] + 2 * f.idx[d]; ++nv; vd = d; }
          else { c[d] = 2 * oc[d] + 1; bd = d; }
        }
        if (nv == 3) kind = 0;
        else if (nv == 2) { kind = 1; m1 = f.idx[bd]; }
        else { kind = 2; int t1, t2; tang(vd, t1, t2); m1 = f.idx[t1]; m2 = f.idx[t2]; }
      } else {
        int t1, t2;
        tang(f.d, t1, t2);
        c[f.d] = 2 * oc[f.d] + 2 * f.s;
        c[t1] = 2 * oc[t1] + 1;
        c[t2] = 2 * oc[t2] + 1;
        kind = 3; m1 = f.a; m2 = f.b;
      }
      M.child_map[o * loc.size() + li] = key.at(std::make_tuple(c[0], c[1], c[2], kind, m1, m2));
    }
  }

  // ---- global fine DOF of each K-local DOF
  auto dof_of = [&](const int Kc[3], const KDof& k) -> int64_t {
    int g[3];
    for (int d = 0; d < 3; ++d) g[d] = 4 * Kc[d] + k.ctr[d];
    int64_t E = mf.entity_at(g, k.kind == 3);
    if (E < 0) return -1;
    int64_t st;
    int nd;
    mf.ent_range(E, &st, &nd);
    if (k.kind == 0) return st;
    if (k.kind == 1) return st + (k.m1 - 2);
    if (k.kind == 2) return st + (k.m1 - 2) + (int64_t)(p - 1) * (k.m2 - 2);
    return st + k.m1 + (int64_t)p * k.m2;
  };
  int64_t nK = mc.nelem;
  M.S_glob.assign(nK * M.nS, -1);
  M.I_glob.assign(nK * M.nI, -1);
  M.groups.resize(nK);
  M.smask.assign(mf.ndof, 0);
  parallel_ranges(nK, [&](int64_t lo, int64_t hi) {
    for (int64_t K = lo; K < hi; ++K) {
      int Kc[3];
      mc.elem_coord(K, Kc);
      for (int a = 0; a < M.nS; ++a) {
        int64_t g = dof_of(Kc, kl[a]);
        M.S_glob[K * M.nS + a] = g;
        if (g >= 0) M.groups[K].push_back(mf.dof_entity(g));
      }
      for (int a = 0; a < M.nI; ++a) M.I_glob[K * M.nI + a] = dof_of(Kc, kl[M.nS + a]);
      auto& gr = M.groups[K];
      std::sort(gr.begin(), gr.end());
      gr.erase(std::unique(gr.begin(), gr.end()), gr.end());
    }
  });
  for (int64_t q = 0; q < nK * M.nS; ++q)
    if (M.S_glob[q] >= 0) M.smask[M.S_glob[q]] = 1;

  // ---- natural inclusion on one coarse element (identical for all K)
  const auto& locc = mc.loc;
  M.nloc_c = (int)locc.size();
  M.IK.assign((size_t)M.nS * locc.size(), 0.0);
  for (int a = 0; a < M.nS; ++a) {
    const KDof& k = kl[a];
    for (size_t j = 0; j < locc.size(); ++j) {
      const LocFn& f = locc[j];
      double coef = 0.0;
      if (f.type == 0 && k.kind != 3) {
        // fine 1D function per axis: node (even coordinate) or bubble
        int bub[3] = {0, 0, 0};
        if (k.kind == 1) { for (int d = 0; d < 3; ++d) if (k.ctr[d] & 1) bub[d] = k.m1; }
        if (k.kind == 2) {
          int nd = -1;
          for (int d = 0; d < 3; ++d) if (!(k.ctr[d] & 1)) nd = d;
          int t1, t2;
          tang(nd, t1, t2);
          bub[t1] = k.m1;
          bub[t2] = k.m2;
        }
        coef = 1.0;
        for (int d = 0; d < 3; ++d) {
          if (!(k.ctr[d] & 1)) coef *= h1_val(p, f.idx[d], k.ctr[d] / 4.0);
          else coef *= h1_bubble_coef(p, f.idx[d], (k.ctr[d] - 1) / 2, bub[d]);
          if (coef == 0.0) break;
        }
      } else if (f.type == 1 && k.kind == 3) {
        int nd = -1;
        for (int d = 0; d < 3; ++d) if (!(k.ctr[d] & 1)) nd = d;
        if (nd == f.d && k.ctr[nd] == 4 * f.s) {
          int t1, t2;
          tang(nd, t1, t2);
          coef = leg_twoscale(p, f.a, (k.ctr[t1] - 1) / 2, k.m1) *
                 leg_twoscale(p, f.b, (k.ctr[t2] - 1) / 2, k.m2);
        }
      }
      if (std::fabs(coef) < 1e-15) coef = 0.0;
      M.IK[(size_t)a * locc.size() + j] = coef;
    }
  }

  // ---- S-slot CSR per fine DOF (slots in increasing K)
  M.sslot_ptr.assign(mf.ndof + 1, 0);
  for (int64_t s = 0; s < nK * M.nS; ++s)
    if (M.S_glob[s] >= 0) ++M.sslot_ptr[M.S_glob[s] + 1];
  for (int64_t g = 0; g < mf.ndof; ++g) M.sslot_ptr[g + 1] += M.sslot_ptr[g];
  M.sslots.assign(M.sslot_ptr[mf.ndof], 0);
  {
    std::vector<int64_t> f(M.sslot_ptr.begin(), M.sslot_ptr.end() - 1);
    for (int64_t s = 0; s < nK * M.nS; ++s)
      if (M.S_glob[s] >= 0) M.sslots[f[M.S_glob[s]]++] = (int32_t)s;
  }
  // ---- global P (fine rows) and P^T (coarse rows).  Row g of P is row a of
  // I_K in the coarse numbering of any coarse element K whose skeleton holds g
  // at local index a (the same values for every such K); the first such K
  // (its first S-slot) gives it, columns in increasing coarse DOF.
  const size_t nlc = locc.size();
  M.P_ptr.assign(mf.ndof + 1, 0);
  auto row_of = [&](int64_t g, std::vector<int64_t>& cg, std::vector<std::pair<int64_t, double>>& out) {
    out.clear();
    if (M.sslot_ptr[g + 1] == M.sslot_ptr[g]) return;
    const int64_t s = M.sslots[M.sslot_ptr[g]];
    const int64_t K = s / M.nS;
    const int a = (int)(s % M.nS);
    mc.elem_dofs(K, cg.data());
    for (size_t j = 0; j < nlc; ++j) {
      const double v = M.IK[(size_t)a * nlc + j];
      if (v != 0.0 && cg[j] >= 0) out.emplace_back(cg[j], v);
    }
    std::sort(out.begin(), out.end());
  };
  parallel_ranges(mf.ndof, [&](int64_t lo, int64_t hi) {
    std::vector<int64_t> cg(nlc);
    std::vector<std::pair<int64_t, double>> r;
    for (int64_t g = lo; g < hi; ++g) {
      row_of(g, cg, r);
      M.P_ptr[g + 1] = (int64_t)r.size();
    }
  });
  for (int64_t g = 0; g < mf.ndof; ++g) M.P_ptr[g + 1] += M.P_ptr[g];
  M.P_col.assign(M.P_ptr[mf.ndof], 0);
  M.P_val.assign(M.P_ptr[mf.ndof], 0.0);
  parallel_ranges(mf.ndof, [&](int64_t lo, int64_t hi) {
    std::vector<int64_t> cg(nlc);
    std::vector<std::pair<int64_t, double>> r;
    for (int64_t g = lo; g < hi; ++g) {
      row_of(g, cg, r);
      for (size_t q = 0; q < r.size(); ++q) {
        M.P_col[M.P_ptr[g] + q] = (int32_t)r[q].first;
        M.P_val[M.P_ptr[g] + q] = r[q].second;
      }
    }
  });
  M.PT_ptr.assign(mc.ndof + 1, 0);
  for (int64_t q = 0; q < M.P_ptr[mf.ndof]; ++q) ++M.PT_ptr[M.P_col[q] + 1];
  for (int64_t g = 0; g < mc.ndof; ++g) M.PT_ptr[g + 1] += M.PT_ptr[g];
  M.PT_col.assign(M.P_ptr[mf.ndof], 0);
  M.PT_val.assign(M.P_ptr[mf.ndof], 0.0);
  {
    std::vector<int64_t> f(M.PT_ptr.begin(), M.PT_ptr.end() - 1);
    for (int64_t g = 0; g < mf.ndof; ++g)   // rows in increasing g: each P^T row in increasing fine DOF
      for (int64_t q = M.P_ptr[g]; q < M.P_ptr[g + 1]; ++q) {
        const int64_t r = M.P_col[q];
        M.PT_col[f[r]] = (int32_t)g;
        M.PT_val[f[r]++] = M.P_val[q];
      }
  }
  return M;
}

}  // namespace dpgmg
