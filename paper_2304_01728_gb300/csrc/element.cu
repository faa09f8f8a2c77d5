// Batched element-local DPG work (Sec. 2 of the paper; the per-element steps
// of the fine-grid assembly):
//   k_elem_build     Gram G' (real form), enriched stiffness B' and load l'
//   k_elem_potrf     G' = L L^T                      (real FP64 Cholesky)
//   k_elem_trsm      W = L^-1 [B' | l']              (optimal test functions)
//   k_elem_herk      K = W^H W = [B l]^* G^-1 [B l]  (DPG element matrix + load)
//   k_elem_condense  static condensation of the 4p^3 field DOFs (Sec. 1.2):
//                    K_c = K_tt - K_tf K_ff^-1 K_ft, F_c = F_t - K_tf K_ff^-1 F_f
// One CTA per element; elements are processed in chunks that bound the
// scratch memory.  All arithmetic is FP64.
//
// Real path.  Scaling the trial functions p and p-hat by i (u, u-hat by 1)
// on top of the test scaling v -> i v makes B' and the load real on every
// element without impedance boundary faces when the source is real (the
// impedance term <p-hat, Z^-1 q> is the only complex entry).  Such elements
// run TRSM, K = W^T W and the condensation in real arithmetic (a quarter of
// the complex flops); the unit phases are put back on the outputs:
// K_c[i][j] = beta_i conj(beta_j) K'_c[i][j], F_c[i] = beta_i F'_c[i].
#include <algorithm>
#include <cstdlib>
#include <map>
#include <cmath>

#include "common.cuh"
#include "element_entries.cuh"
#include "internal.h"

namespace dpgmg {

struct ElemArgs {
  int n[3];
  double x0[3], h[3];
  double omega;
  int p, nt, nf, ntr, m, nql;
  const double* c;        // per element wavespeed
  int src;
  double sc[3], sw, sa, wd[3];
  int mfm;
  const double2* mfc;     // [4][m][m][m]
  double bx0[3], bL[3];
  const int4 *tf, *ff, *tr;
  Tab1D tab;
  const double *xq, *wq, *Lq;  // load rule and L_a at its points ([n1][nql])
  const double2* u0s;      // caller's impedance load samples at the boundary points, or null
  int64_t u0off[6];        // first boundary face of side (d, s) in the sample list
  const int64_t* elist;    // element ids of the batch list
  int64_t e0;
  double* G;
  int nph;                 // number of p-hat trace columns (split path)
  const int* phq;          // per trace column: its index among the p-hat columns, or -1
  void* W;                 // [chunk][nt][m+1] of the path's scalar type
  void* K;                 // [chunk][m+1][m+1]
  double2* Eout;
  double2* Fc;
  double2* Yrec;
  int* info;
};

__device__ __forceinline__ double2 cexp_i(double phase) {
  double s, c;
  sincos(phase, &s, &c);
  return make_double2(c, s);
}

// Manufactured polynomial (p_ex, u_ex) and gradients at a physical point.
__device__ void mf_eval(const ElemArgs& a, const double x[3], double2 val[4], double2 grad[4][3]) {
  const int m = a.mfm;
  double L[3][8], dL[3][8];
  for (int d = 0; d < 3; ++d) {
    double X = (x[d] - a.bx0[d]) / a.bL[d];
    double xi = 2.0 * X - 1.0;
    L[d][0] = 1.0;
    dL[d][0] = 0.0;
    if (m > 1) { L[d][1] = xi; dL[d][1] = 1.0; }
    for (int k = 1; k + 1 < m; ++k) {
      L[d][k + 1] = ((2 * k + 1) * xi * L[d][k] - k * L[d][k - 1]) / (k + 1);
      dL[d][k + 1] = dL[d][k - 1] + (2 * k + 1) * L[d][k];
    }
    for (int k = 0; k < m; ++k) dL[d][k] *= 2.0 / a.bL[d];
  }
  for (int comp = 0; comp < 4; ++comp) {
    double2 v = make_double2(0, 0), g0 = v, g1 = v, g2 = v;
    const double2* C = a.mfc + (size_t)comp * m * m * m;
    for (int cc = 0; cc < m; ++cc)
      for (int b = 0; b < m; ++b)
        for (int aa = 0; aa < m; ++aa) {
          double2 co = C[(cc * m + b) * m + aa];
          double t0 = L[0][aa] * L[1][b] * L[2][cc];
          double t1 = dL[0][aa] * L[1][b] * L[2][cc];
          double t2 = L[0][aa] * dL[1][b] * L[2][cc];
          double t3 = L[0][aa] * L[1][b] * dL[2][cc];
          v.x += co.x * t0; v.y += co.y * t0;
          g0.x += co.x * t1; g0.y += co.y * t1;
          g1.x += co.x * t2; g1.y += co.y * t2;
          g2.x += co.x * t3; g2.y += co.y * t3;
        }
    val[comp] = v;
    grad[comp][0] = g0;
    grad[comp][1] = g1;
    grad[comp][2] = g2;
  }
}

// Volume data f, g at a point (Sec. 2 strong form with sources).
__device__ void src_volume(const ElemArgs& a, double c, const double x[3], double2& f, double2 g[3]) {
  f = make_double2(0, 0);
  g[0] = g[1] = g[2] = make_double2(0, 0);
  if (a.src == DPGMG_SRC_GAUSSIAN) {
    double r2 = 0;
    for (int d = 0; d < 3; ++d) r2 += (x[d] - a.sc[d]) * (x[d] - a.sc[d]);
    f.x = a.sa * exp(-r2 / (2.0 * a.sw * a.sw));
  } else if (a.src == DPGMG_SRC_MANUFACTURED) {
    double2 val[4], gr[4][3];
    mf_eval(a, x, val, gr);
    double bt = a.omega / (c * c);
    // f = i w c^-2 p + div u ; g = i w u + grad p
    f.x = -bt * val[0].y + gr[1][0].x + gr[2][1].x + gr[3][2].x;
    f.y = bt * val[0].x + gr[1][0].y + gr[2][1].y + gr[3][2].y;
    for (int d = 0; d < 3; ++d) {
      g[d].x = -a.omega * val[1 + d].y + gr[0][d].x;
      g[d].y = a.omega * val[1 + d].x + gr[0][d].y;
    }
  }
}

// Impedance load u0 at a boundary point with outward normal n.
__device__ double2 src_u0(const ElemArgs& a, double c, const double x[3], const double nrm[3]) {
  if (a.src == DPGMG_SRC_PLANE_WAVE) {
    double dx = a.wd[0] * x[0] + a.wd[1] * x[1] + a.wd[2] * x[2];
    double dn = a.wd[0] * nrm[0] + a.wd[1] * nrm[1] + a.wd[2] * nrm[2];
    double2 pv = cexp_i(-a.omega * dx / c);
    double s = (1.0 - dn) / c;
    return make_double2(s * pv.x, s * pv.y);
  }
  if (a.src == DPGMG_SRC_MANUFACTURED) {
    double2 val[4], gr[4][3];
    mf_eval(a, x, val, gr);
    double2 r = make_double2(val[0].x / c, val[0].y / c);
    for (int d = 0; d < 3; ++d) {
      r.x -= val[1 + d].x * nrm[d];
      r.y -= val[1 + d].y * nrm[d];
    }
    return r;
  }
  return make_double2(0, 0);
}

__device__ __forceinline__ void elem_geom(const ElemArgs& a, int64_t e, int ec[3], double corner[3], int& bmask) {
  ec[0] = (int)(e % a.n[0]);
  ec[1] = (int)((e / a.n[0]) % a.n[1]);
  ec[2] = (int)(e / ((int64_t)a.n[0] * a.n[1]));
  bmask = 0;
  for (int d = 0; d < 3; ++d) {
    corner[d] = a.x0[d] + ec[d] * a.h[d];
    if (ec[d] == 0) bmask |= 1 << (2 * d);
    if (ec[d] == a.n[d] - 1) bmask |= 1 << (2 * d + 1);
  }
}

// scalar of the path from a complex (test-scaled) entry; rot = the trial
// function carries the phase i
template <class T> __device__ __forceinline__ T to_path(double2 v, bool rot);
template <> __device__ __forceinline__ double2 to_path<double2>(double2 v, bool) { return v; }
template <> __device__ __forceinline__ double to_path<double>(double2 v, bool rot) { return rot ? -v.y : v.x; }

// Shared memory of the load builder: the four source arrays at the nq^3
// points and the first partial contraction (4 n1 nq^2 values).
__host__ __device__ inline size_t build_load_smem(int nq, int n1) {
  return ((size_t)4 * nq * nq * nq + (size_t)4 * n1 * nq * nq) * sizeof(double2) + 64;
}

// Volume load l' of one element (Sec. 2: (f, v) + (g, q); v rows scaled by
// -i in the real form) into out[i * stride], i < nt.  The test functions are
// tensor products L_a(x) L_b(y) L_c(z) of the 1D functions tabulated at the
// load rule's points, so the quadrature sums factor axis by axis (sum
// factorisation): for each of the four source arrays S (f and the three
// components of g) T[a][b][c] = sum_qc L_c sum_qb L_b sum_qa L_a S[qc][qb][qa],
// 4 (n1 nq^3 + n1^2 nq^2 + n1^3 nq) products instead of nt nq^3; every test
// function then reads its entry of T.  sh2: build_load_smem(nq, n1) bytes.
template <class T>
__device__ void build_load(const ElemArgs& a, const double corner[3], double c, double2* sh2, T* out, size_t stride) {
  const int nq = a.nql, nq2 = nq * nq, nq3 = nq2 * nq, nt = a.nt, n1 = a.tab.n1;
  double2* fv = sh2;                 // [nq3]
  double2* gv = sh2 + nq3;           // [3][nq3]
  const double J = a.h[0] * a.h[1] * a.h[2];
  for (int q = threadIdx.x; q < nq3; q += blockDim.x) {
    int qa = q % nq, qb = (q / nq) % nq, qc = q / (nq * nq);
    double x[3] = {corner[0] + a.xq[qa] * a.h[0], corner[1] + a.xq[qb] * a.h[1], corner[2] + a.xq[qc] * a.h[2]};
    double2 f, g[3];
    src_volume(a, c, x, f, g);
    double w = a.wq[qa] * a.wq[qb] * a.wq[qc] * J;
    fv[q] = make_double2(f.x * w, f.y * w);
    for (int d = 0; d < 3; ++d) gv[d * nq3 + q] = make_double2(g[d].x * w, g[d].y * w);
  }
  __syncthreads();
  // T1[s][a][qc][qb] = sum_qa L_a(qa) S_s[qc][qb][qa]
  double2* T1 = sh2 + 4 * nq3;
  const int n1q2 = n1 * nq2;
  for (int q = threadIdx.x; q < 4 * n1q2; q += blockDim.x) {
    const int arr = q / n1q2, rem = q % n1q2, ia = rem / nq2, cb = rem % nq2;
    const double2* S = sh2 + (size_t)arr * nq3 + (size_t)cb * nq;
    const double* L = a.Lq + ia * nq;
    double2 acc = make_double2(0, 0);
    for (int qa = 0; qa < nq; ++qa) {
      acc.x += S[qa].x * L[qa];
      acc.y += S[qa].y * L[qa];
    }
    T1[q] = acc;
  }
  __syncthreads();
  // T2[s][a][b][qc] = sum_qb L_b(qb) T1[s][a][qc][qb]   (over the source arrays' space)
  double2* T2 = sh2;
  const int n12q = n1 * n1 * nq;
  for (int q = threadIdx.x; q < 4 * n12q; q += blockDim.x) {
    const int arr = q / n12q, rem = q % n12q, ia = rem / (n1 * nq), rem2 = rem % (n1 * nq), ib = rem2 / nq,
              qc = rem2 % nq;
    const double2* S = T1 + (size_t)arr * n1q2 + (size_t)ia * nq2 + (size_t)qc * nq;
    const double* L = a.Lq + ib * nq;
    double2 acc = make_double2(0, 0);
    for (int qb = 0; qb < nq; ++qb) {
      acc.x += S[qb].x * L[qb];
      acc.y += S[qb].y * L[qb];
    }
    T2[q] = acc;
  }
  __syncthreads();
  // T3[s][a][b][c] = sum_qc L_c(qc) T2[s][a][b][qc]   (over T1's space)
  double2* T3 = T1;
  const int n13 = n1 * n1 * n1;
  for (int q = threadIdx.x; q < 4 * n13; q += blockDim.x) {
    const int arr = q / n13, rem = q % n13, ab = rem / n1, ic = rem % n1;
    const double2* S = T2 + (size_t)arr * n12q + (size_t)ab * nq;
    const double* L = a.Lq + ic * nq;
    double2 acc = make_double2(0, 0);
    for (int qc = 0; qc < nq; ++qc) {
      acc.x += S[qc].x * L[qc];
      acc.y += S[qc].y * L[qc];
    }
    T3[q] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    int4 t = a.tf[i];
    const int arr = t.x == 3 ? 0 : 1 + t.x;
    double2 acc = T3[(size_t)arr * n13 + (t.y * n1 + t.z) * n1 + t.w];
    if (t.x != 3) acc = make_double2(acc.y, -acc.x);
    out[(size_t)i * stride] = to_path<T>(acc, false);
  }
  __syncthreads();
}

// Split path (boundary elements, real source): with the trial phases of the
// real path, B' = B_r + i B_i where B_i is non-zero only in the p-hat columns
// (the impedance term <p-hat, Z^-1 q> on boundary faces).  The builder writes
// one real matrix [B_r | l' | B_i(p-hat columns)] of row length m + 1 + nph.
template <class T, bool SPLIT = false>
__global__ void __launch_bounds__(CTA_THREADS) k_elem_build(ElemArgs a) {
  extern __shared__ double2 sh2[];
  const int64_t le = blockIdx.x;
  const int64_t e = a.elist[a.e0 + le];
  int ec[3], bmask;
  double corner[3];
  elem_geom(a, e, ec, corner, bmask);
  const double c = a.c[e];
  const double beta = a.omega / (c * c);
  const int nt = a.nt, m = a.m, ldw = SPLIT ? m + 1 + a.nph : m + 1;
  double* G = a.G + le * (size_t)nt * nt;
  // per-element slot of nt (m+1) complex values (the split path's real rows fit in it)
  T* W = SPLIT ? reinterpret_cast<T*>(reinterpret_cast<double2*>(a.W) + le * (size_t)nt * (m + 1))
               : reinterpret_cast<T*>(a.W) + le * (size_t)nt * ldw;
  for (int64_t q = threadIdx.x; q < (int64_t)nt * nt; q += blockDim.x) {
    int i = (int)(q / nt), j = (int)(q % nt);
    G[q] = (j <= i) ? gram_entry(a.tab, a.tf[i], a.tf[j], a.h, beta, a.omega) : 0.0;
  }
  for (int64_t q = threadIdx.x; q < (int64_t)nt * m; q += blockDim.x) {
    int i = (int)(q / m), j = (int)(q % m);
    double2 v = (j < a.nf) ? bfield_entry(a.tab, a.tf[i], a.ff[j], a.h, beta, a.omega)
                           : btrace_entry(a.tab, a.tf[i], a.tr[j - a.nf], a.h, 1.0 / c, bmask);
    const bool rot = (j < a.nf) ? a.ff[j].x == 0 : a.tr[j - a.nf].x == 0;
    W[(size_t)i * ldw + j] = to_path<T>(v, rot);
    if (SPLIT && j >= a.nf) {
      const int q = a.phq[j - a.nf];
      // imaginary part of the phased value i v (p-hat columns carry the phase i)
      if (q >= 0) reinterpret_cast<double*>(W)[(size_t)i * ldw + m + 1 + q] = v.x;
    }
  }
  // ---- load l' (v rows scaled by -i)
  const int nq = a.nql;
  const int n1 = a.tab.n1;
  double2* fv = sh2;                 // [nq3]
  build_load<T>(a, corner, c, sh2, W + m, ldw);
  // boundary faces: <u0, q>, u0 from the source and/or the caller's samples
  if (a.src != DPGMG_SRC_GAUSSIAN || a.u0s) {
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        if (!((bmask >> (2 * d + s)) & 1)) continue;
        int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        for (int q = threadIdx.x; q < nq * nq; q += blockDim.x) {
          int qa = q % nq, qb = q / nq;
          double x[3];
          x[d] = corner[d] + s * a.h[d];
          x[t1] = corner[t1] + a.xq[qa] * a.h[t1];
          x[t2] = corner[t2] + a.xq[qb] * a.h[t2];
          double nrm[3] = {0, 0, 0};
          nrm[d] = s ? 1.0 : -1.0;
          double2 u = src_u0(a, c, x, nrm);
          if (a.u0s) {
            // samples of face (ec[t1], ec[t2]) of side (d, s), points qa along t1 fastest
            const int64_t f = a.u0off[2 * d + s] + ec[t1] + (int64_t)a.n[t1] * ec[t2];
            const double2 v = a.u0s[(f * nq + qb) * nq + qa];
            u.x += v.x;
            u.y += v.y;
          }
          double w = a.wq[qa] * a.wq[qb] * a.h[t1] * a.h[t2];
          fv[q] = make_double2(u.x * w, u.y * w);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
          int4 t = a.tf[i];
          if (t.x != 3) continue;
          int id[3] = {t.y, t.z, t.w};
          double endv = (s ? 1.0 : ((id[d] & 1) ? -1.0 : 1.0));
          double2 acc = make_double2(0, 0);
          for (int q = 0; q < nq * nq; ++q) {
            int qa = q % nq, qb = q / nq;
            double bv = endv * a.Lq[id[t1] * nq + qa] * a.Lq[id[t2] * nq + qb];
            acc.x += fv[q].x * bv;
            acc.y += fv[q].y * bv;
          }
          // boundary loads only occur on the complex path
          double2* o = reinterpret_cast<double2*>(&W[(size_t)i * ldw + m]);
          o->x += acc.x;
          o->y += acc.y;
        }
        __syncthreads();
      }
  }
  (void)n1;
}

__global__ void __launch_bounds__(CTA_THREADS) k_elem_potrf(ElemArgs a) {
  extern __shared__ double sh[];
  const int64_t le = blockIdx.x;
  double* G = a.G + le * (size_t)a.nt * a.nt;
  int info = cta_potrf<double>(G, a.nt, a.nt, sh);
  if (threadIdx.x == 0 && info) atomicOr(a.info, 1);
}

template <class T>
__global__ void __launch_bounds__(CTA_THREADS) k_elem_trsm(ElemArgs a) {
  extern __shared__ char shc[];
  const int64_t le = blockIdx.x;
  const double* G = a.G + le * (size_t)a.nt * a.nt;
  T* W = reinterpret_cast<T*>(a.W) + le * (size_t)a.nt * (a.m + 1);
  cta_trsm_lower<double, T>(G, a.nt, a.nt, W, a.m + 1, a.m + 1, shc);
}

template <class T>
__global__ void __launch_bounds__(CTA_THREADS) k_elem_herk(ElemArgs a) {
  extern __shared__ unsigned char shraw[];
  const int64_t le = blockIdx.x;
  const int ld = a.m + 1;
  const T* W = reinterpret_cast<const T*>(a.W) + le * (size_t)a.nt * ld;
  T* K = reinterpret_cast<T*>(a.K) + le * (size_t)ld * ld;
  // K = W^H W is Hermitian: lower tiles plus their mirror
  cta_herk_lower<T>(W, a.nt, ld, ld, K, ld, reinterpret_cast<T*>(shraw), false);
}

// ---- split path: real TRSM and HERK on [B_r | l' | B_i(p-hat)], then the
// complex K' = W^H W from the real Gram matrix R of the extended columns:
//   Re K'[a][b] = R[a][b] + R[a~][b~],   Im K'[a][b] = R[a][b~] - R[a~][b]
// (a~ = the imaginary column of a, terms absent where a has none).
__global__ void __launch_bounds__(CTA_THREADS) k_elem_trsm_split(ElemArgs a) {
  extern __shared__ char shc[];
  const int64_t le = blockIdx.x;
  const int ld2 = a.m + 1 + a.nph;
  const double* G = a.G + le * (size_t)a.nt * a.nt;
  double* W = reinterpret_cast<double*>(reinterpret_cast<double2*>(a.W) + le * (size_t)a.nt * (a.m + 1));
  cta_trsm_lower<double, double>(G, a.nt, a.nt, W, ld2, ld2, shc);
}

__global__ void __launch_bounds__(CTA_THREADS) k_elem_herk_split(ElemArgs a) {
  extern __shared__ unsigned char shraw[];
  const int64_t le = blockIdx.x;
  const int ld = a.m + 1, ld2 = ld + a.nph;
  const double* W = reinterpret_cast<const double*>(reinterpret_cast<const double2*>(a.W) + le * (size_t)a.nt * ld);
  double* R = reinterpret_cast<double*>(reinterpret_cast<double2*>(a.K) + le * (size_t)ld * ld);
  cta_herk_lower<double>(W, a.nt, ld2, ld2, R, ld2, reinterpret_cast<double*>(shraw), false);
}

// R (real, ld2 x ld2, in the K slot) -> complex K' (ld x ld) in the same slot,
// staged through the element's W slot (no longer needed after the HERK)
__global__ void __launch_bounds__(CTA_THREADS) k_elem_split_assemble(ElemArgs a) {
  const int64_t le = blockIdx.x;
  const int ld = a.m + 1, ld2 = ld + a.nph, nf = a.nf, m = a.m;
  double2* Kc = reinterpret_cast<double2*>(a.K) + le * (size_t)ld * ld;
  const double* R = reinterpret_cast<const double*>(Kc);
  double2* T = reinterpret_cast<double2*>(a.W) + le * (size_t)a.nt * ld;
  for (int q = threadIdx.x; q < ld * ld; q += blockDim.x) {
    const int i = q / ld, j = q % ld;
    const int qi = (i >= nf && i < m) ? a.phq[i - nf] : -1;
    const int qj = (j >= nf && j < m) ? a.phq[j - nf] : -1;
    double re = R[(size_t)i * ld2 + j], im = 0.0;
    if (qi >= 0 && qj >= 0) re += R[(size_t)(ld + qi) * ld2 + ld + qj];
    if (qj >= 0) im += R[(size_t)i * ld2 + ld + qj];
    if (qi >= 0) im -= R[(size_t)(ld + qi) * ld2 + j];
    T[q] = make_double2(re, im);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < ld * ld; q += blockDim.x) Kc[q] = T[q];
}

// complex output of the path's value; ph = 0: x1, 1: x i, 2: x (-i)
template <class T> __device__ __forceinline__ double2 phased(T v, int ph);
template <> __device__ __forceinline__ double2 phased<double2>(double2 v, int) { return v; }
template <> __device__ __forceinline__ double2 phased<double>(double v, int ph) {
  return ph == 0 ? make_double2(v, 0.0) : (ph == 1 ? make_double2(0.0, v) : make_double2(0.0, -v));
}
// the split path's complex values carry the unit phases too
__device__ __forceinline__ double2 phased_c(double2 v, int ph) {
  return ph == 0 ? v : (ph == 1 ? make_double2(-v.y, v.x) : make_double2(v.y, -v.x));
}
template <class T, bool PH> __device__ __forceinline__ double2 out_value(T v, int ph) { return phased<T>(v, ph); }
template <class T> __device__ __forceinline__ T from_c128(double2 v);
template <> __device__ __forceinline__ double from_c128<double>(double2 v) { return v.x; }
template <> __device__ __forceinline__ double2 from_c128<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ double2 out_value<double2, true>(double2 v, int ph) { return phased_c(v, ph); }
__device__ __forceinline__ int phase_of(bool a_i, bool b_i) { return (a_i && !b_i) ? 1 : ((!a_i && b_i) ? 2 : 0); }

template <class T, bool PH = false>
__global__ void __launch_bounds__(CTA_THREADS) k_elem_condense(ElemArgs a) {
  extern __shared__ unsigned char shraw[];
  T* sh = reinterpret_cast<T*>(shraw);
  const int64_t le = blockIdx.x;
  const int64_t e = a.elist[a.e0 + le];
  const int ld = a.m + 1, nf = a.nf, ntr = a.ntr;
  T* K = reinterpret_cast<T*>(a.K) + le * (size_t)ld * ld;
  int info = cta_potrf<T>(K, nf, ld, sh);
  if (threadIdx.x == 0 && info) atomicOr(a.info, 2);
  cta_trsm_lower<T, T>(K, nf, ld, K + nf, ntr + 1, ld, reinterpret_cast<char*>(sh));
  cta_trsm_lower_h<T>(K, nf, ld, K + nf, ntr + 1, ld, reinterpret_cast<char*>(sh));
  cta_gemm<T>(false, ntr, ntr + 1, nf, -1.0, K + (size_t)nf * ld, ld, K + nf, ld, 1.0, K + (size_t)nf * ld + nf, ld,
              sh);
  double2* E = a.Eout + e * (size_t)ntr * ntr;
  for (int q = threadIdx.x; q < ntr * ntr; q += blockDim.x) {
    int i = q / ntr, j = q % ntr;
    E[q] = out_value<T, PH>(K[(size_t)(nf + i) * ld + nf + j], phase_of(a.tr[i].x == 0, a.tr[j].x == 0));
  }
  for (int i = threadIdx.x; i < ntr; i += blockDim.x)
    a.Fc[e * ntr + i] = out_value<T, PH>(K[(size_t)(nf + i) * ld + a.m], a.tr[i].x == 0 ? 1 : 0);
  double2* Y = a.Yrec + e * (size_t)nf * (ntr + 1);
  for (int q = threadIdx.x; q < nf * (ntr + 1); q += blockDim.x) {
    int i = q / (ntr + 1), j = q % (ntr + 1);
    const bool fi = a.ff[i].x == 0;
    const int ph = (j < ntr) ? phase_of(fi, a.tr[j].x == 0) : (fi ? 1 : 0);
    Y[q] = out_value<T, PH>(K[(size_t)i * ld + nf + j], ph);
  }
}

// ---- element classes (constant coefficients): G, B and the condensed matrix
// of an element depend on (h, omega, c) and its impedance faces only, so one
// representative per class runs the full pipeline and every other member of
// the class computes only what its load changes.  Member b (element mem_e[b],
// representative in slot mem_slot[b] of the current batch) uses the
// representative's scratch: G = L (Gram Cholesky), W = L^-1 [B | l | B_i],
// and after condensation K = [L_ff | Y ; K_tf | K_c].  Per member scratch
// (stride doubles): w [nt] (even-padded), F [m] complex, u [nf] complex.
//
// Stage 1 (after the representatives' HERK, before the split path overwrites
// W): w = L^-1 l', F = W_B'^H w, the load column of K; on the split path
// Re F_a = sum_k W[k][a] w_k, Im F_a = -sum_k W[k][a~] w_k as in
// k_elem_split_assemble.  Members are listed class by class, and chunk q =
// (slot, first member b0, count <= MCB) holds members of one class.
// k_elem_member_rhs builds the load l' of every member as column j of the
// chunk's block X_q (nt x MCB, row-major); k_elem_member_solve then applies
// the class's factors to the whole block, X = L^-1 X (one triangular solve
// with MCB right-hand sides) and F = W_B'^T X (a product), so the
// representative's factors are read once per chunk instead of once per
// member, and writes each member's F into its scratch.
constexpr int MCB = 32;
__global__ void __launch_bounds__(CTA_THREADS) k_elem_member_rhs(ElemArgs a, const int64_t* __restrict__ mem_e,
                                                                 const int4* __restrict__ chunks, double* X) {
  extern __shared__ double2 sh2[];
  const int4 ch = chunks[blockIdx.x];
  const int j = blockIdx.y;
  if (j >= ch.z) return;   // uniform over the CTA
  const int64_t e = mem_e[ch.y + j];
  int ec[3], bmask;
  double corner[3];
  elem_geom(a, e, ec, corner, bmask);
  build_load<double>(a, corner, a.c[e], sh2, X + (size_t)blockIdx.x * a.nt * MCB + j, MCB);
}

template <bool SPLIT>
__global__ void __launch_bounds__(CTA_THREADS) k_elem_member_solve(ElemArgs a, const int4* __restrict__ chunks,
                                                                   double* X, double* Ft, double* scr,
                                                                   int64_t stride) {
  extern __shared__ double2 sh2[];
  const int4 ch = chunks[blockIdx.x];
  const int slot = ch.x, cnt = ch.z;
  const int nt = a.nt, m = a.m, nf = a.nf;
  double* Xq = X + (size_t)blockIdx.x * nt * MCB;
  double* Fq = Ft + (size_t)blockIdx.x * (m + (SPLIT ? a.nph : 0)) * MCB;
  const double* L = a.G + (size_t)slot * nt * nt;
  cta_trsm_lower<double, double>(L, nt, nt, Xq, cnt, MCB, reinterpret_cast<char*>(sh2));
  const int ldw = SPLIT ? m + 1 + a.nph : m + 1;
  const double* W = SPLIT ? reinterpret_cast<const double*>(reinterpret_cast<const double2*>(a.W) + (size_t)slot * nt * (m + 1))
                          : reinterpret_cast<const double*>(a.W) + (size_t)slot * nt * ldw;
  double* shd = reinterpret_cast<double*>(sh2);
  // Fq[jj][b] = sum_k W[k][jj] X[k][b]; split path: rows m .. m + nph - 1 from W's B_i columns
  cta_gemm<double>(true, m, cnt, nt, 1.0, W, ldw, Xq, MCB, 0.0, Fq, MCB, shd);
  if (SPLIT && a.nph) cta_gemm<double>(true, a.nph, cnt, nt, 1.0, W + m + 1, ldw, Xq, MCB, 0.0, Fq + (size_t)m * MCB,
                                       MCB, shd);
  for (int q = threadIdx.x; q < cnt * m; q += blockDim.x) {
    const int b = q / m, jj = q % m;
    const int qj = (SPLIT && jj >= nf) ? a.phq[jj - nf] : -1;
    double2* F = reinterpret_cast<double2*>(scr + (size_t)(ch.y + b) * stride + nt + (nt & 1));
    F[jj] = make_double2(Fq[(size_t)jj * MCB + b], qj >= 0 ? -Fq[(size_t)(m + qj) * MCB + b] : 0.0);
  }
}

// Stage 2 (after the representatives' condensation), per chunk of one class:
// U = K_ff^-1 [F_f of the members] (two triangular solves with MCB
// right-hand sides), F_c = F_t - K_tf U (a product); outputs as
// k_elem_condense writes them, with the load-independent parts (K_c, the
// recovery columns of the traces) copied from the representative.
template <class T, bool PH>
__global__ void __launch_bounds__(CTA_THREADS) k_elem_member_condense(ElemArgs a, const int64_t* __restrict__ mem_e,
                                                                      const int4* __restrict__ chunks, double* Ub,
                                                                      double* Cb, double* scr, int64_t stride) {
  extern __shared__ unsigned char shraw[];
  const int4 ch = chunks[blockIdx.x];
  const int slot = ch.x, cnt = ch.z;
  const int64_t rep = a.elist[a.e0 + slot];
  const int nt = a.nt, m = a.m, nf = a.nf, ntr = a.ntr, ld = m + 1;
  const T* K = reinterpret_cast<const T*>(a.K) + (size_t)slot * ld * ld;
  T* U = reinterpret_cast<T*>(Ub) + (size_t)blockIdx.x * nf * MCB;
  T* Cq = reinterpret_cast<T*>(Cb) + (size_t)blockIdx.x * ntr * MCB;
  auto Fm = [&](int b) { return reinterpret_cast<const double2*>(scr + (size_t)(ch.y + b) * stride + nt + (nt & 1)); };
  for (int q = threadIdx.x; q < cnt * m; q += blockDim.x) {
    const int b = q / m, i = q % m;
    const T v = from_c128<T>(Fm(b)[i]);
    if (i < nf) U[(size_t)i * MCB + b] = v;
    else Cq[(size_t)(i - nf) * MCB + b] = v;
  }
  __syncthreads();
  cta_trsm_lower<T, T>(K, nf, ld, U, cnt, MCB, reinterpret_cast<char*>(shraw));
  cta_trsm_lower_h<T>(K, nf, ld, U, cnt, MCB, reinterpret_cast<char*>(shraw));
  cta_gemm<T>(false, ntr, cnt, nf, -1.0, K + (size_t)nf * ld, ld, U, MCB, 1.0, Cq, MCB, reinterpret_cast<T*>(shraw));
  for (int q = threadIdx.x; q < cnt * ntr; q += blockDim.x) {
    const int b = q / ntr, i = q % ntr;
    a.Fc[mem_e[ch.y + b] * ntr + i] = out_value<T, PH>(Cq[(size_t)i * MCB + b], a.tr[i].x == 0 ? 1 : 0);
  }
  const double2* Er = a.Eout + rep * (size_t)ntr * ntr;
  const double2* Yr = a.Yrec + rep * (size_t)nf * (ntr + 1);
  for (int b = 0; b < cnt; ++b) {
    const int64_t e = mem_e[ch.y + b];
    double2* E = a.Eout + e * (size_t)ntr * ntr;
    for (int q = threadIdx.x; q < ntr * ntr; q += blockDim.x) E[q] = Er[q];
    double2* Y = a.Yrec + e * (size_t)nf * (ntr + 1);
    for (int q = threadIdx.x; q < nf * (ntr + 1); q += blockDim.x) {
      const int i = q / (ntr + 1), j = q % (ntr + 1);
      Y[q] = j < ntr ? Yr[q] : out_value<T, PH>(U[(size_t)i * MCB + b], a.ff[i].x == 0 ? 1 : 0);
    }
  }
}

// fields[e][i] = Y_F[i] - sum_j Y_K[i][j] x[dofs[e][j]]
__global__ void k_recover(const double2* Yrec, const int64_t* dofs, const double2* x, double2* out,
                          int64_t nelem, int nf, int ntr) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= nelem * nf) return;
  int64_t e = gid / nf;
  int i = (int)(gid % nf);
  const double2* Y = Yrec + (e * nf + i) * (size_t)(ntr + 1);
  double2 acc = Y[ntr];
  for (int j = 0; j < ntr; ++j) {
    int64_t g = dofs[e * ntr + j];
    if (g < 0) continue;
    double2 y = Y[j], v = x[g];
    acc.x -= y.x * v.x - y.y * v.y;
    acc.y -= y.x * v.y + y.y * v.x;
  }
  out[gid] = acc;
}

// ------------------------------------------------------------------- host
static void make_descriptors(int p, std::vector<int4>& tf, std::vector<int4>& ff, std::vector<int4>& tr) {
  const int pt = p + 1;
  tf.clear();
  ff.clear();
  tr.clear();
  for (int c = 0; c <= pt; ++c)
    for (int b = 0; b <= pt; ++b)
      for (int a = 0; a <= pt; ++a) tf.push_back(make_int4(3, a, b, c));
  for (int d = 0; d < 3; ++d) {
    int ext[3];
    for (int e = 0; e < 3; ++e) ext[e] = (e == d) ? pt : pt - 1;
    for (int c = 0; c <= ext[2]; ++c)
      for (int b = 0; b <= ext[1]; ++b)
        for (int a = 0; a <= ext[0]; ++a) tf.push_back(make_int4(d, a, b, c));
  }
  for (int comp = 0; comp < 4; ++comp)
    for (int c = 0; c < p; ++c)
      for (int b = 0; b < p; ++b)
        for (int a = 0; a < p; ++a) ff.push_back(make_int4(comp, a, b, c));
  for (const LocFn& f : local_trace_functions(p))
    tr.push_back(f.type == 0 ? make_int4(0, f.idx[0], f.idx[1], f.idx[2])
                             : make_int4(1, f.d, f.s, f.a + 256 * f.b));
}

// Elements per batch of the element stage: at most 4096 and at most 8 GiB of scratch.
int64_t element_chunk(int64_t nel, size_t per_elem) {
  int64_t c = (int64_t)(((size_t)8 << 30) / per_elem);
  return std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(nel, 4096), c));
}

static size_t smem_bytes_dense(size_t elt) { return (size_t)(NB * NB + 2 * TL * NB) * elt + 64; }

// Condensed element matrices L.E of level L (c: wavespeed per element of L's
// mesh).  On the finest level the condensed loads, the recovery blocks and
// the flop count are kept for the solve; on a coarser level ("stored" coarse
// operators) they are scratch.
static void element_core(SystemImpl& S, Level& L, const std::vector<double>& cvals, bool finest, cudaStream_t st);

void element_stage(SystemImpl& S, cudaStream_t st) { element_core(S, S.levels.back(), S.wavespeed, true, st); }

void element_stage_level(SystemImpl& S, Level& L, cudaStream_t st) {
  // stored coarse operators need a wavespeed per coarse element: only constant c is allowed
  std::vector<double> c((size_t)L.mesh.nelem, S.wavespeed.empty() ? 1.0 : S.wavespeed[0]);
  element_core(S, L, c, false, st);
}

static void element_core(SystemImpl& S, Level& L, const std::vector<double>& cvals, bool finest, cudaStream_t st) {
  const MeshL& m = L.mesh;
  const int p = m.p;
  std::vector<int4> tf, ff, tr;
  make_descriptors(p, tf, ff, tr);
  Tables1D T = make_tables(p);
  Alloc& A = S.mem;

  ElemArgs a{};
  for (int d = 0; d < 3; ++d) {
    a.n[d] = m.n[d];
    a.x0[d] = m.x0[d];
    a.h[d] = m.h[d];
    a.sc[d] = S.pb.src_center[d];
    a.bx0[d] = S.pb.x0[d];
    a.bL[d] = S.pb.x1[d] - S.pb.x0[d];
  }
  double dn = std::sqrt(S.pb.wave_dir[0] * S.pb.wave_dir[0] + S.pb.wave_dir[1] * S.pb.wave_dir[1] +
                        S.pb.wave_dir[2] * S.pb.wave_dir[2]);
  for (int d = 0; d < 3; ++d) a.wd[d] = dn > 0 ? S.pb.wave_dir[d] / dn : 0.0;
  a.omega = S.pb.omega;
  a.p = p;
  a.nt = (int)tf.size();
  a.nf = (int)ff.size();
  a.ntr = (int)tr.size();
  a.m = a.nf + a.ntr;
  a.nql = T.nql;
  a.src = S.pb.source;
  a.sw = S.pb.src_width;
  a.sa = S.pb.src_amp;
  a.mfm = S.pb.mf_order;
  a.c = upload(A, cvals, st);
  std::vector<double2> mfc(S.mf_coeffs.size() / 2);
  for (size_t i = 0; i < mfc.size(); ++i) mfc[i] = make_double2(S.mf_coeffs[2 * i], S.mf_coeffs[2 * i + 1]);
  a.mfc = upload(A, mfc, st);
  a.tf = upload(A, tf, st);
  a.ff = upload(A, ff, st);
  a.tr = upload(A, tr, st);
  {
    // index of every p-hat trace column among the p-hat columns (split path)
    std::vector<int> phq(tr.size(), -1);
    int q = 0;
    for (size_t j = 0; j < tr.size(); ++j)
      if (tr[j].x == 0) phq[j] = q++;
    a.nph = q;
    a.phq = upload(A, phq, st);
  }
  a.tab.p = p;
  a.tab.pt = p + 1;
  a.tab.n1 = p + 2;
  a.tab.Mleg = upload(A, T.Mleg, st);
  a.tab.D = upload(A, T.D, st);
  a.tab.S = upload(A, T.S, st);
  a.tab.Phi = upload(A, T.Phi, st);
  a.xq = upload(A, T.xq, st);
  a.wq = upload(A, T.wq, st);
  a.Lq = upload(A, T.Lq, st);
  if (finest && !S.u0.empty()) {
    // caller's impedance load samples (finest mesh only: the stored coarse
    // operators of coarser meshes keep only their matrices)
    std::vector<double2> u0(S.u0.size() / 2);
    for (size_t i = 0; i < u0.size(); ++i) u0[i] = make_double2(S.u0[2 * i], S.u0[2 * i + 1]);
    a.u0s = upload(A, u0, st);
    boundary_face_offsets(m.n, a.u0off);
  }
  a.info = A.arr<int>(1);
  DPG_CUDA(cudaMemsetAsync(a.info, 0, sizeof(int), st));

  const int64_t nel = m.nelem;
  if (finest) {
    S.nelem = nel;
    S.nf = a.nf;
    S.ntr = a.ntr;
  }
  L.nloc = a.ntr;
  L.E = A.arr<double2>((size_t)nel * a.ntr * a.ntr);
  double2* Fc = A.arr<double2>((size_t)nel * a.ntr);
  double2* Yrec = A.arr<double2>((size_t)nel * a.nf * (a.ntr + 1));
  if (finest) {
    S.Fc = Fc;
    S.Yrec = Yrec;
  }
  a.Eout = L.E;
  a.Fc = Fc;
  a.Yrec = Yrec;

  // scratch per element: G (nt^2 doubles), W (nt (m+1)), K ((m+1)^2)
  const size_t per = (size_t)a.nt * a.nt * 8 + (size_t)a.nt * (a.m + 1) * 16 + (size_t)(a.m + 1) * (a.m + 1) * 16;
  int64_t chunk = element_chunk(nel, per);
  a.G = A.arr<double>((size_t)chunk * a.nt * a.nt);
  a.W = A.arr<double2>((size_t)chunk * a.nt * (a.m + 1));
  a.K = A.arr<double2>((size_t)chunk * (a.m + 1) * (a.m + 1));

  const size_t sm_build = build_load_smem(T.nql, p + 2);
  // Function attributes are process-wide and systems may be set up concurrently
  // (serving slots), so the limit is the largest any order p <= 5 needs.
  const size_t sm_build_max = build_load_smem(10, 7);   // p = 5
  const size_t sm_real = smem_bytes_dense(8);
  const size_t sm_cplx = smem_bytes_dense(16);
  DPG_CUDA(cudaFuncSetAttribute(k_elem_build<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_build_max));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_build<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_build_max));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_real));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_trsm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cplx));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_trsm<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cplx));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_herk<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cplx));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_herk<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cplx));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_condense<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cplx));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_condense<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cplx));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_build<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sm_build_max));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_trsm_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cplx));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_herk_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cplx));
  DPG_CUDA(cudaFuncSetAttribute(k_elem_condense<double2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sm_cplx));
  // element lists: real path (no impedance face, real source) and complex path
  // element lists: real path (no impedance face, real source), split path
  // (impedance faces, Gaussian source: the only complex entries are the
  // impedance terms of the p-hat columns) and complex path (other sources)
  std::vector<int64_t> lreal, lsplit, lcplx;
  const bool real_src = S.pb.source != DPGMG_SRC_MANUFACTURED;
  const int64_t ld1 = a.m + 1, ld2 = ld1 + a.nph;
  const bool split_ok = S.pb.source == DPGMG_SRC_GAUSSIAN && a.u0s == nullptr && ld2 * ld2 <= 2 * ld1 * ld1;
  for (int64_t e = 0; e < nel; ++e) {
    int ec[3];
    m.elem_coord(e, ec);
    bool interior = true;
    for (int d = 0; d < 3; ++d)
      if (ec[d] == 0 || ec[d] == m.n[d] - 1) interior = false;
    if (interior && real_src) lreal.push_back(e);
    else if (split_ok) lsplit.push_back(e);
    else lcplx.push_back(e);
  }
  int64_t* dreal = upload(A, lreal, st);
  int64_t* dsplit = upload(A, lsplit, st);
  int64_t* dcplx = upload(A, lcplx, st);
  auto run_split = [&](const int64_t* dl, int64_t cnt) {
    a.elist = dl;
    for (int64_t e0 = 0; e0 < cnt; e0 += chunk) {
      a.e0 = e0;
      const int nb = (int)std::min<int64_t>(chunk, cnt - e0);
      k_elem_build<double, true><<<nb, CTA_THREADS, sm_build, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_potrf<<<nb, CTA_THREADS, sm_real, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_trsm_split<<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_herk_split<<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_split_assemble<<<nb, CTA_THREADS, 0, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_condense<double2, true><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
    }
  };
  auto run_list = [&](const int64_t* dl, int64_t cnt, bool real) {
    a.elist = dl;
    for (int64_t e0 = 0; e0 < cnt; e0 += chunk) {
      a.e0 = e0;
      const int nb = (int)std::min<int64_t>(chunk, cnt - e0);
      if (real) k_elem_build<double><<<nb, CTA_THREADS, sm_build, st>>>(a);
      else k_elem_build<double2><<<nb, CTA_THREADS, sm_build, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_potrf<<<nb, CTA_THREADS, sm_real, st>>>(a);
      DPG_CHECK_LAUNCH();
      if (real) k_elem_trsm<double><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      else k_elem_trsm<double2><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
      if (real) k_elem_herk<double><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      else k_elem_herk<double2><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
      if (real) k_elem_condense<double><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      else k_elem_condense<double2><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
    }
  };
  // Element classes (Gaussian source: real loads, no boundary loads): the key
  // (impedance-face mask, wavespeed) fixes G, B and the condensed matrix, so
  // one representative per class runs the full pipeline and the other
  // members run the two member stages.  Used when the classes are few (at
  // most nel / 4) and their representatives fit one batch; DPGMG_ELEMENT_REUSE=0
  // runs every element through the full pipeline.
  bool reuse = S.pb.source == DPGMG_SRC_GAUSSIAN && lcplx.empty();
  if (const char* ev = std::getenv("DPGMG_ELEMENT_REUSE")) reuse = reuse && std::atoi(ev) != 0;
  std::vector<int64_t> rreps, sreps, rmem, smem;   // representatives and members (real / split path)
  std::vector<int> rslot, sslot;                   // member -> slot of its representative
  if (reuse) {
    std::map<std::pair<int, double>, int> cls;
    for (int64_t e = 0; e < nel; ++e) {
      int ec[3];
      m.elem_coord(e, ec);
      int bm = 0;
      for (int d = 0; d < 3; ++d) {
        if (ec[d] == 0) bm |= 1 << (2 * d);
        if (ec[d] == m.n[d] - 1) bm |= 1 << (2 * d + 1);
      }
      const bool interior = bm == 0;
      std::vector<int64_t>& reps = interior ? rreps : sreps;
      auto it = cls.find(std::make_pair(bm, cvals[e]));
      if (it == cls.end()) {
        cls.emplace(std::make_pair(bm, cvals[e]), (int)reps.size());
        reps.push_back(e);
      } else {
        (interior ? rmem : smem).push_back(e);
        (interior ? rslot : sslot).push_back(it->second);
      }
    }
    reuse = (int64_t)(rreps.size() + sreps.size()) * 4 <= nel && (int64_t)rreps.size() <= chunk &&
            (int64_t)sreps.size() <= chunk;
  }
  const int64_t mstride = (a.nt + (a.nt & 1)) + 2 * (int64_t)a.m + 2 * (int64_t)a.nf;   // member scratch (doubles)
  // members listed class by class, cut into chunks of at most MCB members of one class
  auto chunk_members = [](std::vector<int64_t>& mem, std::vector<int>& slot) {
    std::vector<size_t> ord(mem.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t u, size_t v) { return slot[u] < slot[v]; });
    std::vector<int64_t> m2(mem.size());
    std::vector<int> s2(mem.size());
    for (size_t i = 0; i < ord.size(); ++i) {
      m2[i] = mem[ord[i]];
      s2[i] = slot[ord[i]];
    }
    mem.swap(m2);
    slot.swap(s2);
    std::vector<int4> ch;
    for (size_t i = 0; i < mem.size();) {
      size_t j = i;
      while (j < mem.size() && slot[j] == slot[i] && (int)(j - i) < MCB) ++j;
      ch.push_back(make_int4(slot[i], (int)i, (int)(j - i), 0));
      i = j;
    }
    return ch;
  };
  if (reuse) {
    const size_t sm_mem = std::max(sm_build_max, sm_cplx);
    DPG_CUDA(cudaFuncSetAttribute(k_elem_member_condense<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm_cplx));
    DPG_CUDA(cudaFuncSetAttribute(k_elem_member_condense<double2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm_cplx));
    double* scr = A.arr<double>((size_t)std::max<int64_t>((int64_t)std::max(rmem.size(), smem.size()), 1) * mstride);
    const std::vector<int4> rch = chunk_members(rmem, rslot), sch = chunk_members(smem, sslot);
    const size_t nch = std::max<size_t>(std::max(rch.size(), sch.size()), 1);
    double* Xb = A.arr<double>(nch * (size_t)a.nt * MCB);
    double* Fb = A.arr<double>(nch * (size_t)(a.m + a.nph) * MCB);
    double* Ub = A.arr<double>(nch * (size_t)a.nf * MCB * 2);    // K_ff^-1 F_f blocks (complex at most)
    double* Cb = A.arr<double>(nch * (size_t)a.ntr * MCB * 2);   // condensed load blocks
    DPG_CUDA(cudaFuncSetAttribute(k_elem_member_rhs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_mem));
    DPG_CUDA(cudaFuncSetAttribute(k_elem_member_solve<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cplx));
    DPG_CUDA(cudaFuncSetAttribute(k_elem_member_solve<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cplx));
    auto member_loads = [&](const std::vector<int4>& ch, const int64_t* de, bool split) {
      int4* dch = upload(A, ch, st);
      k_elem_member_rhs<<<dim3((unsigned)ch.size(), MCB), CTA_THREADS, sm_mem, st>>>(a, de, dch, Xb);
      DPG_CHECK_LAUNCH();
      if (split) k_elem_member_solve<true><<<(unsigned)ch.size(), CTA_THREADS, sm_cplx, st>>>(a, dch, Xb, Fb, scr, mstride);
      else k_elem_member_solve<false><<<(unsigned)ch.size(), CTA_THREADS, sm_cplx, st>>>(a, dch, Xb, Fb, scr, mstride);
      DPG_CHECK_LAUNCH();
      A.release(dch);
    };
    if (!rreps.empty()) {
      int64_t* dl = upload(A, rreps, st);
      a.elist = dl;
      a.e0 = 0;
      const int nb = (int)rreps.size(), nm = (int)rmem.size();
      int64_t* de = nm ? upload(A, rmem, st) : nullptr;
      k_elem_build<double><<<nb, CTA_THREADS, sm_build, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_potrf<<<nb, CTA_THREADS, sm_real, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_trsm<double><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_herk<double><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
      if (nm) member_loads(rch, de, false);
      k_elem_condense<double><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
      if (nm) {
        int4* dch = upload(A, rch, st);
        k_elem_member_condense<double, false><<<(unsigned)rch.size(), CTA_THREADS, sm_cplx, st>>>(a, de, dch, Ub, Cb,
                                                                                                   scr, mstride);
        DPG_CHECK_LAUNCH();
        A.release(dch);
        A.release(de);
      }
      A.release(dl);
    }
    if (!sreps.empty()) {
      int64_t* dl = upload(A, sreps, st);
      a.elist = dl;
      a.e0 = 0;
      const int nb = (int)sreps.size(), nm = (int)smem.size();
      int64_t* de = nm ? upload(A, smem, st) : nullptr;
      k_elem_build<double, true><<<nb, CTA_THREADS, sm_build, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_potrf<<<nb, CTA_THREADS, sm_real, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_trsm_split<<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_herk_split<<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
      if (nm) member_loads(sch, de, true);   // before the assembly below reuses the W slots
      k_elem_split_assemble<<<nb, CTA_THREADS, 0, st>>>(a);
      DPG_CHECK_LAUNCH();
      k_elem_condense<double2, true><<<nb, CTA_THREADS, sm_cplx, st>>>(a);
      DPG_CHECK_LAUNCH();
      if (nm) {
        int4* dch = upload(A, sch, st);
        k_elem_member_condense<double2, true><<<(unsigned)sch.size(), CTA_THREADS, sm_cplx, st>>>(a, de, dch, Ub, Cb,
                                                                                                   scr, mstride);
        DPG_CHECK_LAUNCH();
        A.release(dch);
        A.release(de);
      }
      A.release(dl);
    }
    A.release(Cb);
    A.release(Ub);
    A.release(Fb);
    A.release(Xb);
    A.release(scr);
  } else {
    run_list(dreal, (int64_t)lreal.size(), true);
    run_split(dsplit, (int64_t)lsplit.size());
    run_list(dcplx, (int64_t)lcplx.size(), false);
  }
  if (finest) {
    // algorithmic multiply-adds (an FMA is 2 flops, a complex FMA 8): Gram
    // Cholesky nt^3/6, W = L^-1 [B l] nt^2 (m+1)/2, K = W^H W (lower)
    // (m+1)^2 nt/2, field condensation nf^3/6 + nf^2 (ntr+1) + ntr (ntr+1) nf
    const double n = a.nt, m1 = a.m + 1, nf = a.nf, t1 = a.ntr + 1.0;
    const double fma_g = n * n * n / 6.0;
    const double fma_w = n * n * m1 / 2.0 + m1 * m1 * n / 2.0 + nf * nf * nf / 6.0 + nf * nf * t1 + a.ntr * t1 * nf;
    // split path: real TRSM and HERK over m + 1 + nph columns, complex condensation
    const double m2 = (double)ld2, fma_c = nf * nf * nf / 6.0 + nf * nf * t1 + a.ntr * t1 * nf;
    const double fma_s = n * n * m2 / 2.0 + m2 * m2 * n / 2.0;
    if (reuse) {
      // representatives: the full count; members: w = L^-1 l (nt^2/2), F = W^H w, u = K_ff^-1 F_f
      // (nf^2), F_c = F_t - K_tf u (ntr nf); the split path's F over m + nph real columns
      const double mem_r = n * n / 2.0 + a.m * n + nf * nf + a.ntr * nf;
      const double mem_s_real = n * n / 2.0 + (a.m + a.nph) * n, mem_s_cplx = nf * nf + a.ntr * nf;
      S.elem_flops = (double)rreps.size() * (2.0 * fma_g + 2.0 * fma_w) +
                     (double)sreps.size() * (2.0 * fma_g + 2.0 * fma_s + 8.0 * fma_c) +
                     (double)rmem.size() * 2.0 * mem_r + (double)smem.size() * (2.0 * mem_s_real + 8.0 * mem_s_cplx);
    } else {
      S.elem_flops = (double)lreal.size() * (2.0 * fma_g + 2.0 * fma_w) +
                     (double)lsplit.size() * (2.0 * fma_g + 2.0 * fma_s + 8.0 * fma_c) +
                     (double)lcplx.size() * (2.0 * fma_g + 8.0 * fma_w);
    }
  }
  int info = 0;
  DPG_CUDA(cudaMemcpyAsync(&info, a.info, sizeof(int), cudaMemcpyDeviceToHost, st));
  DPG_CUDA(cudaStreamSynchronize(st));
  A.release(a.G);
  A.release(a.W);
  A.release(a.K);
  A.release(dreal);
  A.release(dsplit);
  A.release(dcplx);
  a.G = nullptr;
  a.W = nullptr;
  a.K = nullptr;
  a.elist = nullptr;
  if (finest) {
    S.eargs = std::make_shared<ElemArgs>(a);
  } else {
    A.release(Fc);
    A.release(Yrec);
  }
  if (info) throw Err{DPGMG_ERR_NOT_HPD, "element Gram or field block not positive definite"};
}

// DPG error indicator (Sec. 1.2: the minimised residual is the method's
// built-in error indicator; it drives the refinements of Sec. 3):
//   eta_K^2 = (l - B u_K)^* G^-1 (l - B u_K)
// for the element trial vector u_K = [fields, local traces].  With the test
// scaling of the real form (G = D G' D^H, B = D B', l = D l', D unitary and
// diagonal) this is || L^-1 (l' - B' u_K) ||^2 with G' = L L^T.  Per element
// (after k_elem_build<double2> and k_elem_potrf on the same chunk): r = l' -
// B' u_K into the load column, forward substitution, squared norm.
__global__ void __launch_bounds__(CTA_THREADS) k_elem_eta(ElemArgs a, const double2* __restrict__ fields,
                                                          const int64_t* __restrict__ dofs,
                                                          const double2* __restrict__ x, double* __restrict__ eta2) {
  extern __shared__ unsigned char she[];
  const int64_t le = blockIdx.x;
  const int64_t e = a.elist[a.e0 + le];
  const int nt = a.nt, m = a.m, ldw = m + 1;
  const double* L = a.G + le * (size_t)nt * nt;
  double2* W = reinterpret_cast<double2*>(a.W) + le * (size_t)nt * ldw;
  double2* u = reinterpret_cast<double2*>(she);               // [m]
  char* tsm = reinterpret_cast<char*>(u + m);                   // triangular-solve scratch
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    if (j < a.nf) {
      u[j] = fields[e * a.nf + j];
    } else {
      const int64_t g = dofs[e * a.ntr + (j - a.nf)];
      u[j] = g >= 0 ? x[g] : make_double2(0.0, 0.0);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    const double2* row = W + (size_t)i * ldw;
    double2 acc = row[m];
    for (int j = 0; j < m; ++j) acc = Ops<double2>::fnma(row[j], u[j], acc);
    W[(size_t)i * ldw + m] = acc;
  }
  __syncthreads();
  cta_trsm_lower<double, double2>(L, nt, nt, W + m, 1, ldw, tsm);
  __shared__ double red[CTA_THREADS / 32];
  double s2 = 0.0;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    const double2 y = W[(size_t)i * ldw + m];
    s2 += y.x * y.x + y.y * y.y;
  }
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < CTA_THREADS / 32; ++w) t += red[w];
    eta2[e] = t;
  }
}

void error_indicator(SystemImpl& S, const double2* x, double* eta2, cudaStream_t st) {
  if (!S.eargs) throw Err{DPGMG_ERR_ARG, "the system has no element stage"};
  ElemArgs a = *S.eargs;
  Alloc& A = S.mem;
  const Level& L = S.levels.back();
  const int64_t nel = S.nelem;
  double2* fields = A.arr<double2>((size_t)std::max<int64_t>(nel * a.nf, 1));
  recover_fields(S, x, fields, st);
  std::vector<int64_t> all(nel);
  for (int64_t e = 0; e < nel; ++e) all[e] = e;
  int64_t* dall = upload(A, all, st);
  const size_t per = (size_t)a.nt * a.nt * 8 + (size_t)a.nt * (a.m + 1) * 16;
  const int64_t chunk = element_chunk(nel, per);
  a.G = A.arr<double>((size_t)chunk * a.nt * a.nt);
  a.W = A.arr<double2>((size_t)chunk * a.nt * (a.m + 1));
  a.elist = dall;
  a.info = A.arr<int>(1);
  DPG_CUDA(cudaMemsetAsync(a.info, 0, sizeof(int), st));
  const size_t sm_build = build_load_smem(a.nql, a.tab.n1);
  const size_t sm_real = smem_bytes_dense(8);
  const size_t sm_eta = (size_t)a.m * sizeof(double2) + smem_bytes_dense(16);
  DPG_CUDA(cudaFuncSetAttribute(k_elem_eta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_eta));
  for (int64_t e0 = 0; e0 < nel; e0 += chunk) {
    a.e0 = e0;
    const int nb = (int)std::min<int64_t>(chunk, nel - e0);
    k_elem_build<double2><<<nb, CTA_THREADS, sm_build, st>>>(a);
    DPG_CHECK_LAUNCH();
    k_elem_potrf<<<nb, CTA_THREADS, sm_real, st>>>(a);
    DPG_CHECK_LAUNCH();
    k_elem_eta<<<nb, CTA_THREADS, sm_eta, st>>>(a, fields, L.dofs, x, eta2);
    DPG_CHECK_LAUNCH();
  }
  int info = 0;
  DPG_CUDA(cudaMemcpyAsync(&info, a.info, sizeof(int), cudaMemcpyDeviceToHost, st));
  DPG_CUDA(cudaStreamSynchronize(st));
  A.release(a.G);
  A.release(a.W);
  A.release(a.info);
  A.release(dall);
  A.release(fields);
  if (info) throw Err{DPGMG_ERR_NOT_HPD, "element Gram not positive definite"};
}

void recover_fields(SystemImpl& S, const double2* x, double2* fields, cudaStream_t st) {
  const Level& L = S.levels.back();
  int64_t n = S.nelem * S.nf;
  k_recover<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S.Yrec, L.dofs, x, fields, S.nelem, (int)S.nf,
                                                        (int)S.ntr);
  DPG_CHECK_LAUNCH();
}

}  // namespace dpgmg
