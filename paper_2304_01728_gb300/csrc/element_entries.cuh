// Closed-form entries of the element Gram matrix and enriched stiffness
// matrix of the broken ultraweak acoustics formulation on an axis-aligned
// hexahedron (Sec. 2, Eq. variational-formulation and Eq. Gnorm).
//
// All trial, trace and test functions are tensor products of 1D Legendre
// (L_a) and hierarchical H^1 (phi_k) functions on the unit interval, so
// every volume or face integral is a product of three 1D integrals taken
// from small tables:
//   Mleg[a]   = int L_a L_a = 1/(2a+1)           (Legendre mass, diagonal)
//   D[a][b]   = int L_a' L_b                      (derivative on the first)
//   S[a][b]   = int L_a' L_b'
//   Phi[k][b] = int phi_k L_b                     (H^1 trace vs Legendre test)
// and the endpoint values L_a(0) = (-1)^a, L_a(1) = 1, phi_k(0), phi_k(1).
//
// Test space (enrichment dp = 1, pt = p + 1): q = L_a L_b L_c, a,b,c <= pt;
// v = e_d L_a L_b L_c with degree pt along d and pt-1 across.  The test
// inner product of Eq. Gnorm (alpha = 1) is complex Hermitian; writing
// v = i v' makes it real symmetric:
//   G'(q,q')  = (beta^2 + 1)(q, q') + (grad q, grad q')
//   G'(v,v')  = (div v, div v') + (w^2 + 1)(v, v')
//   G'(q,v')  = beta (div v', q) - w (v', grad q)          beta = w / c^2
// and the enriched stiffness B' = D^H B has its v-rows multiplied by -i.
// Then B^* G^{-1} B = B'^* G'^{-1} B' (D = diag(1, i) is unitary), so the
// Gram Cholesky runs in real arithmetic.
#pragma once
#include <cuda_runtime.h>

namespace dpgmg {

// Function descriptors (packed in int4):
//   test  : x = kind (0,1,2 = v_x, v_y, v_z; 3 = q), (y, z, w) = Legendre indices
//   field : x = comp (0 = p, 1..3 = u_x, u_y, u_z),  (y, z, w) = Legendre indices
//   trace : x = 0 p-hat with (y, z, w) = H^1 indices;
//           x = 1 u-hat with y = normal axis d, z = side s, w = a + 256 b
struct Tab1D {
  int p, pt, n1;          // n1 = pt + 1
  const double* Mleg;     // [n1]
  const double* D;        // [n1][n1]
  const double* S;        // [n1][n1]
  const double* Phi;      // [p+1][n1]
};

__host__ __device__ inline double tM(const Tab1D& t, int a, int b) { return a == b ? t.Mleg[a] : 0.0; }
__host__ __device__ inline double tD(const Tab1D& t, int a, int b) { return t.D[a * t.n1 + b]; }
__host__ __device__ inline double tS(const Tab1D& t, int a, int b) { return t.S[a * t.n1 + b]; }
__host__ __device__ inline double tPhi(const Tab1D& t, int k, int b) { return t.Phi[k * t.n1 + b]; }
__host__ __device__ inline double Lend(int a, int s) { return s ? 1.0 : ((a & 1) ? -1.0 : 1.0); }
__host__ __device__ inline double phiend(int k, int s) { return (k == s) ? 1.0 : 0.0; }

__host__ __device__ inline int idx_of(const int4& f, int e) { return e == 0 ? f.y : (e == 1 ? f.z : f.w); }

// Real Gram entry G'[i][j] (test functions ti, tj).
__host__ __device__ inline double gram_entry(const Tab1D& t, int4 ti, int4 tj, const double h[3],
                                             double beta, double omega) {
  const double J = h[0] * h[1] * h[2];
  if (ti.x == 3 && tj.x == 3) {
    double mm = 1.0;
    for (int e = 0; e < 3; ++e) mm *= tM(t, idx_of(ti, e), idx_of(tj, e));
    double g = (beta * beta + 1.0) * J * mm;
    for (int d = 0; d < 3; ++d) {
      double f = tS(t, idx_of(ti, d), idx_of(tj, d)) / (h[d] * h[d]);
      if (f == 0.0) continue;
      for (int e = 0; e < 3; ++e)
        if (e != d) f *= tM(t, idx_of(ti, e), idx_of(tj, e));
      g += J * f;
    }
    return g;
  }
  if (ti.x != 3 && tj.x != 3) {
    const int di = ti.x, dj = tj.x;
    double f = 1.0;
    for (int e = 0; e < 3; ++e) {
      int a = idx_of(ti, e), b = idx_of(tj, e);
      double v;
      if (e == di && e == dj) v = tS(t, b, a);
      else if (e == dj) v = tD(t, b, a);        // derivative on v_j
      else if (e == di) v = tD(t, a, b);        // derivative on v_i
      else v = tM(t, a, b);
      f *= v;
      if (f == 0.0) break;
    }
    double g = J * f / (h[di] * h[dj]);
    if (di == dj) {
      double mm = 1.0;
      for (int e = 0; e < 3; ++e) mm *= tM(t, idx_of(ti, e), idx_of(tj, e));
      g += (omega * omega + 1.0) * J * mm;
    }
    return g;
  }
  // mixed: q-row with v-column (or the symmetric case)
  int4 q = ti.x == 3 ? ti : tj;
  int4 v = ti.x == 3 ? tj : ti;
  const int d = v.x;
  double f1 = 1.0, f2 = 1.0;   // (div v, q) and (v, d_d q)
  for (int e = 0; e < 3; ++e) {
    int a = idx_of(q, e), b = idx_of(v, e);
    if (e == d) { f1 *= tD(t, b, a); f2 *= tD(t, a, b); }
    else { double m = tM(t, a, b); f1 *= m; f2 *= m; }
  }
  return J / h[d] * (beta * f1 - omega * f2);
}

// Entry of the enriched stiffness B'[i][j] = conj(alpha_i) b(phi_j, psi_i)
// (alpha = 1 on q rows, i on v rows) for a field column.
__host__ __device__ inline double2 bfield_entry(const Tab1D& t, int4 ti, int4 fj, const double h[3],
                                                double beta, double omega) {
  const double J = h[0] * h[1] * h[2];
  double re = 0.0, im = 0.0;
  if (ti.x == 3) {
    if (fj.x == 0) {          // (i beta p, q)
      double mm = 1.0;
      for (int e = 0; e < 3; ++e) mm *= tM(t, idx_of(fj, e), idx_of(ti, e));
      im = beta * J * mm;
    } else {                  // -(u_d, d_d q)
      const int d = fj.x - 1;
      double f = 1.0;
      for (int e = 0; e < 3; ++e)
        f *= (e == d) ? tD(t, idx_of(ti, e), idx_of(fj, e)) : tM(t, idx_of(fj, e), idx_of(ti, e));
      re = -J / h[d] * f;
    }
  } else {
    const int di = ti.x;
    if (fj.x == 0) {          // -(p, div v)
      double f = 1.0;
      for (int e = 0; e < 3; ++e)
        f *= (e == di) ? tD(t, idx_of(ti, e), idx_of(fj, e)) : tM(t, idx_of(fj, e), idx_of(ti, e));
      re = -J / h[di] * f;
    } else if (fj.x - 1 == di) {  // (i w u, v)
      double mm = 1.0;
      for (int e = 0; e < 3; ++e) mm *= tM(t, idx_of(fj, e), idx_of(ti, e));
      im = omega * J * mm;
    }
    // v-row: multiply by -i: (re + i im)(-i) = im - i re
    double r2 = im, i2 = -re;
    re = r2;
    im = i2;
  }
  return make_double2(re, im);
}

// Trace column: p-hat (<phat, v.n_K>, plus <phat, Z^-1 q> on boundary faces)
// or u-hat (s <uhat, q> on an interior face; zero on Gamma).  bmask bit
// 2d+s marks boundary face (d, s).
__host__ __device__ inline double2 btrace_entry(const Tab1D& t, int4 ti, int4 tj, const double h[3],
                                                double invZ, int bmask) {
  double re = 0.0;
  if (tj.x == 0) {
    if (ti.x != 3) {
      const int d = ti.x;
      double tf = 1.0;
      for (int e = 0; e < 3; ++e)
        if (e != d) tf *= h[e] * tPhi(t, idx_of(tj, e), idx_of(ti, e));
      if (tf != 0.0) {
        int k = idx_of(tj, d), a = idx_of(ti, d);
        double s0 = -phiend(k, 0) * Lend(a, 0), s1 = phiend(k, 1) * Lend(a, 1);
        re = tf * (s0 + s1);
      }
      return make_double2(0.0, -re);   // v-row scaled by -i
    }
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        if (!((bmask >> (2 * d + s)) & 1)) continue;
        int k = idx_of(tj, d), a = idx_of(ti, d);
        double nv = phiend(k, s) * Lend(a, s);
        if (nv == 0.0) continue;
        double tf = 1.0;
        for (int e = 0; e < 3; ++e)
          if (e != d) tf *= h[e] * tPhi(t, idx_of(tj, e), idx_of(ti, e));
        re += invZ * nv * tf;
      }
    return make_double2(re, 0.0);
  }
  // u-hat
  const int d = tj.y, s = tj.z, a = tj.w & 255, b = tj.w >> 8;
  if (ti.x != 3 || ((bmask >> (2 * d + s)) & 1)) return make_double2(0.0, 0.0);
  int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  double sg = s ? 1.0 : -1.0;
  re = sg * Lend(idx_of(ti, d), s) * h[t1] * h[t2] * tM(t, a, idx_of(ti, t1)) * tM(t, b, idx_of(ti, t2));
  return make_double2(re, 0.0);
}

}  // namespace dpgmg
