// Shared device helpers: complex arithmetic and CTA-cooperative dense
// linear algebra on row-major matrices in global memory.
//
// The batched element, macro-element and patch kernels run one CTA per
// small dense problem (n up to ~1100).  The routines below are blocked
// (block size NB) with shared-memory staging of the diagonal block and of
// the operand tiles of the trailing updates.  They assume blockDim.x == 256.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace dpgmg {

// ------------------------------------------------------------- scalar ops
template <class T> struct Ops;

template <> struct Ops<double> {
  using R = double;
  __device__ __forceinline__ static double zero() { return 0.0; }
  __device__ __forceinline__ static double add(double a, double b) { return a + b; }
  __device__ __forceinline__ static double sub(double a, double b) { return a - b; }
  __device__ __forceinline__ static double mul(double a, double b) { return a * b; }
  __device__ __forceinline__ static double mulc(double a, double b) { return a * b; }   // a conj(b)
  __device__ __forceinline__ static double fma(double a, double b, double c) { return ::fma(a, b, c); }
  __device__ __forceinline__ static double fmac(double a, double b, double c) { return ::fma(a, b, c); }  // a conj(b) + c
  __device__ __forceinline__ static double fnmac(double a, double b, double c) { return ::fma(-a, b, c); } // c - a conj(b)
  __device__ __forceinline__ static double fnma(double a, double b, double c) { return ::fma(-a, b, c); }  // c - a b
  __device__ __forceinline__ static double conj(double a) { return a; }
  __device__ __forceinline__ static double re(double a) { return a; }
  __device__ __forceinline__ static double scale(double a, double s) { return a * s; }
  __device__ __forceinline__ static double from_re(double r) { return r; }
};

template <> struct Ops<float> {
  using R = float;
  __device__ __forceinline__ static float zero() { return 0.f; }
  __device__ __forceinline__ static float add(float a, float b) { return a + b; }
  __device__ __forceinline__ static float sub(float a, float b) { return a - b; }
  __device__ __forceinline__ static float mul(float a, float b) { return a * b; }
  __device__ __forceinline__ static float mulc(float a, float b) { return a * b; }
  __device__ __forceinline__ static float fma(float a, float b, float c) { return fmaf(a, b, c); }
  __device__ __forceinline__ static float fmac(float a, float b, float c) { return fmaf(a, b, c); }
  __device__ __forceinline__ static float fnmac(float a, float b, float c) { return fmaf(-a, b, c); }
  __device__ __forceinline__ static float fnma(float a, float b, float c) { return fmaf(-a, b, c); }
  __device__ __forceinline__ static float conj(float a) { return a; }
  __device__ __forceinline__ static float re(float a) { return a; }
  __device__ __forceinline__ static float scale(float a, float s) { return a * s; }
  __device__ __forceinline__ static float from_re(float r) { return r; }
};

template <class V, class S> struct CplxOps {
  using R = S;
  __device__ __forceinline__ static V mk(S r, S i) { V v; v.x = r; v.y = i; return v; }
  __device__ __forceinline__ static V zero() { return mk(S(0), S(0)); }
  __device__ __forceinline__ static V add(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
  __device__ __forceinline__ static V sub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
  __device__ __forceinline__ static V mul(V a, V b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
  __device__ __forceinline__ static V mulc(V a, V b) { return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
  __device__ __forceinline__ static V fma(V a, V b, V c) {
    return mk(c.x + a.x * b.x - a.y * b.y, c.y + a.x * b.y + a.y * b.x);
  }
  __device__ __forceinline__ static V fmac(V a, V b, V c) {   // a conj(b) + c
    return mk(c.x + a.x * b.x + a.y * b.y, c.y + a.y * b.x - a.x * b.y);
  }
  __device__ __forceinline__ static V fnmac(V a, V b, V c) {  // c - a conj(b)
    return mk(c.x - a.x * b.x - a.y * b.y, c.y - a.y * b.x + a.x * b.y);
  }
  __device__ __forceinline__ static V fnma(V a, V b, V c) {   // c - a b
    return mk(c.x - a.x * b.x + a.y * b.y, c.y - a.x * b.y - a.y * b.x);
  }
  __device__ __forceinline__ static V conj(V a) { return mk(a.x, -a.y); }
  __device__ __forceinline__ static S re(V a) { return a.x; }
  __device__ __forceinline__ static V scale(V a, S s) { return mk(a.x * s, a.y * s); }
  __device__ __forceinline__ static V from_re(S r) { return mk(r, S(0)); }
};
template <> struct Ops<double2> : CplxOps<double2, double> {};
template <> struct Ops<float2> : CplxOps<float2, float> {};

// Element colours of a structured grid: (ex mod 2, ey mod 2, ez mod 2).  Two
// elements of one colour share no vertex, edge or face, so an assembly pass
// over one colour has no write conflicts; the 8 passes run in colour order,
// which fixes the order of every sum (assembly is bitwise reproducible, unlike
// FP64 atomics).
__device__ __forceinline__ int elem_color(int64_t e, int n0, int n1) {
  const int64_t ex = e % n0, ey = (e / n0) % n1, ez = e / ((int64_t)n0 * n1);
  return (int)((ex & 1) | ((ey & 1) << 1) | ((ez & 1) << 2));
}

// ------------------------------------------------------- CTA dense kernels
constexpr int CTA_THREADS = 256;
constexpr int NB = 32;          // panel width
constexpr int TL = 32;          // output tile edge of the tiled updates

// The CTAs that share one dense problem.  Team<false> is one CTA (the
// default of every routine below).  Team<true> is a thread-block cluster of
// `n` CTAs on different SMs: each routine gives every output tile to one CTA
// (`rank`), the CTAs meet at cluster barriers between dependent phases, and
// global reads of the shared matrix bypass L1 (another SM may have written
// them since this SM cached the line).  Tile ownership is by absolute tile
// coordinates, so every entry is computed by the same instructions in the
// same order as with one CTA: results are bitwise those of Team<false>.
template <bool CL>
struct Team {
  int rank = 0, n = 1;
  __device__ __forceinline__ void sync() const {
    if constexpr (CL) {
      asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    } else {
      __syncthreads();
    }
  }
  template <class T>
  __device__ __forceinline__ T ld(const T* p) const {
    if constexpr (CL) return __ldcg(p);
    else return *p;
  }
  // owner of lower-triangle tile (I, J), J <= I: round robin over the packed index
  __device__ __forceinline__ bool own2(int I, int J) const {
    if constexpr (CL) return (((int64_t)I * (I + 1) / 2 + J) % n) == rank;
    else return true;
  }
  // owner of column tile t: zigzag (0..n-1, n-1..0, ...), which balances the
  // triangular work of the column tiles of a triangular inverse
  __device__ __forceinline__ bool own_col(int t) const {
    if constexpr (CL) {
      const int c = t / n, q = t % n;
      return ((c & 1) ? n - 1 - q : q) == rank;
    } else {
      return true;
    }
  }
  // owner of row tile t (plain copies)
  __device__ __forceinline__ bool own_row(int t) const {
    if constexpr (CL) return t % n == rank;
    else return true;
  }
};

// In-place lower Cholesky A = L L^H of an n x n Hermitian matrix (row-major,
// leading dimension lda).  The strict upper triangle is not referenced and
// is left unchanged.  Returns 0 or k+1 if the k-th pivot is not positive.
// smem: >= NB*NB + 2*TL*NB elements of T.
template <class T, bool CL = false>
__device__ int cta_potrf(T* A, int n, int lda, T* smem, Team<CL> tm = Team<CL>()) {
  using O = Ops<T>;
  using R = typename O::R;
  T* D = smem;
  T* Pi = smem + NB * NB;
  T* Pj = Pi + TL * NB;
  __shared__ int info;
  __shared__ R rdiag[NB];   // 1 / L[j][j] of the current diagonal block
  const int tid = threadIdx.x;
  if (tid == 0) info = 0;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    // diagonal block -> shared, unblocked factorisation.  With a cluster every
    // CTA factors its own copy; the cluster barrier keeps the owner's write-back
    // of the factored block (below) from reaching A before every CTA has read it.
    for (int e = tid; e < kb * kb; e += blockDim.x) {
      int i = e / kb, j = e % kb;
      D[i * NB + j] = tm.ld(&A[(size_t)(k0 + i) * lda + k0 + j]);
    }
    if constexpr (CL) tm.sync();
    else __syncthreads();
    for (int j = 0; j < kb; ++j) {
      if (tid == 0) {
        R d = O::re(D[j * NB + j]);
        if (!(d > R(0))) { if (info == 0) info = k0 + j + 1; d = R(1); }
        D[j * NB + j] = O::from_re(sqrt(d));
        rdiag[j] = R(1) / O::re(D[j * NB + j]);
      }
      __syncthreads();
      const R inv = rdiag[j];
      for (int i = j + 1 + tid; i < kb; i += blockDim.x) D[i * NB + j] = O::scale(D[i * NB + j], inv);
      __syncthreads();
      // rank-1 update of the remaining lower part
      int rem = kb - j - 1;
      for (int e = tid; e < rem * rem; e += blockDim.x) {
        int i = j + 1 + e / rem, c = j + 1 + e % rem;
        if (c <= i) D[i * NB + c] = O::fnmac(D[i * NB + j], D[c * NB + j], D[i * NB + c]);
      }
      __syncthreads();
    }
    if (tm.own2(k0 / TL, k0 / TL)) {
      for (int e = tid; e < kb * kb; e += blockDim.x) {
        int i = e / kb, j = e % kb;
        if (j <= i) A[(size_t)(k0 + i) * lda + k0 + j] = D[i * NB + j];
      }
    }
    // panel: rows below solve x L_kk^H = a
    const int k1 = k0 + kb;
    for (int i = k1 + tid; i < n; i += blockDim.x) {
      if (!tm.own2(i / TL, k0 / TL)) continue;
      T* row = A + (size_t)i * lda + k0;
      T x[NB];
      for (int j = 0; j < kb; ++j) {
        T v = tm.ld(&row[j]);
        for (int t = 0; t < j; ++t) v = O::fnmac(x[t], D[j * NB + t], v);
        x[j] = O::scale(v, rdiag[j]);
      }
      for (int j = 0; j < kb; ++j) row[j] = x[j];
    }
    tm.sync();
    // trailing update A[i][j] -= sum_t L[i][t] conj(L[j][t]), lower part
    const int m = n - k1;
    const int nt = (m + TL - 1) / TL;
    for (int bi = 0; bi < nt; ++bi) {
      for (int bj = 0; bj <= bi; ++bj) {
        const int i0 = k1 + bi * TL, j0 = k1 + bj * TL;
        if (!tm.own2(i0 / TL, j0 / TL)) continue;
        for (int e = tid; e < TL * NB; e += blockDim.x) {
          int r = e / NB, t = e % NB;
          Pi[e] = (i0 + r < n && t < kb) ? tm.ld(&A[(size_t)(i0 + r) * lda + k0 + t]) : O::zero();
          Pj[e] = (j0 + r < n && t < kb) ? tm.ld(&A[(size_t)(j0 + r) * lda + k0 + t]) : O::zero();
        }
        __syncthreads();
        for (int e = tid; e < TL * TL; e += blockDim.x) {
          int r = e / TL, c = e % TL;
          int i = i0 + r, j = j0 + c;
          if (i < n && j <= i) {
            T acc = O::zero();
            for (int t = 0; t < kb; ++t) acc = O::fmac(Pi[r * NB + t], Pj[c * NB + t], acc);
            size_t o = (size_t)i * lda + j;
            A[o] = O::sub(tm.ld(&A[o]), acc);
          }
        }
        __syncthreads();
      }
    }
    if constexpr (CL) tm.sync();
  }
  __syncthreads();
  return info;
}

// Mixed products of a triangular-factor entry (real or complex) with a
// right-hand-side entry (complex or real of the same precision).
__device__ __forceinline__ double2 lmul(double l, double2 b) { return make_double2(l * b.x, l * b.y); }
__device__ __forceinline__ double2 lmul(double2 l, double2 b) { return Ops<double2>::mul(l, b); }
__device__ __forceinline__ float2 lmul(float l, float2 b) { return make_float2(l * b.x, l * b.y); }
__device__ __forceinline__ float2 lmul(float2 l, float2 b) { return Ops<float2>::mul(l, b); }
__device__ __forceinline__ double lmul(double l, double b) { return l * b; }
__device__ __forceinline__ float lmul(float l, float b) { return l * b; }

// Solve L X = B in place (L lower triangular n x n of type TLt, B n x nrhs
// of type TB; TLt may be the real type of TB).  smem (bytes): room for
// NB*NB + TL*NB elements of TLt followed by NB*TL elements of TB.
template <class TLt, class TB>
__device__ void cta_trsm_lower(const TLt* L, int n, int ldl, TB* B, int nrhs, int ldb, char* smem) {
  using OL = Ops<TLt>;
  using OB = Ops<TB>;
  using RB = typename OB::R;
  TLt* D = reinterpret_cast<TLt*>(smem);
  TLt* Lt = D + NB * NB;
  TB* Xt = reinterpret_cast<TB*>(Lt + TL * NB);
  __shared__ RB rdiag[NB];
  const int tid = threadIdx.x;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    for (int e = tid; e < kb * kb; e += blockDim.x) {
      int i = e / kb, j = e % kb;
      D[i * NB + j] = (j <= i) ? L[(size_t)(k0 + i) * ldl + k0 + j] : OL::zero();
    }
    if (tid < kb) rdiag[tid] = RB(1) / OL::re(L[(size_t)(k0 + tid) * ldl + k0 + tid]);
    __syncthreads();
    // diagonal solve: one thread per right-hand-side column
    for (int c = tid; c < nrhs; c += blockDim.x) {
      TB x[NB];
      for (int r = 0; r < kb; ++r) {
        TB v = B[(size_t)(k0 + r) * ldb + c];
        for (int t = 0; t < r; ++t) v = OB::sub(v, lmul(D[r * NB + t], x[t]));
        x[r] = OB::scale(v, rdiag[r]);
        B[(size_t)(k0 + r) * ldb + c] = x[r];
      }
    }
    __syncthreads();
    // update rows below: B[i][c] -= sum_t L[i][k0+t] X[k0+t][c]
    const int k1 = k0 + kb;
    for (int i0 = k1; i0 < n; i0 += TL) {
      for (int e = tid; e < TL * NB; e += blockDim.x) {
        int r = e / NB, t = e % NB;
        Lt[e] = (i0 + r < n && t < kb) ? L[(size_t)(i0 + r) * ldl + k0 + t] : OL::zero();
      }
      for (int c0 = 0; c0 < nrhs; c0 += TL) {
        for (int e = tid; e < NB * TL; e += blockDim.x) {
          int t = e / TL, c = e % TL;
          Xt[e] = (t < kb && c0 + c < nrhs) ? B[(size_t)(k0 + t) * ldb + c0 + c] : OB::zero();
        }
        __syncthreads();
        for (int e = tid; e < TL * TL; e += blockDim.x) {
          int r = e / TL, c = e % TL;
          int i = i0 + r, cc = c0 + c;
          if (i < n && cc < nrhs) {
            TB acc = OB::zero();
            for (int t = 0; t < kb; ++t) acc = OB::add(acc, lmul(Lt[r * NB + t], Xt[t * TL + c]));
            size_t o = (size_t)i * ldb + cc;
            B[o] = OB::sub(B[o], acc);
          }
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();
}

// Solve L^H X = B in place (backward substitution), complex L and B of the
// same type T.  smem as cta_trsm_lower.
template <class T>
__device__ void cta_trsm_lower_h(const T* L, int n, int ldl, T* B, int nrhs, int ldb, char* smem) {
  using O = Ops<T>;
  using R = typename O::R;
  T* D = reinterpret_cast<T*>(smem);
  T* Lt = D + NB * NB;
  T* Xt = Lt + TL * NB;
  __shared__ R rdiag[NB];
  const int tid = threadIdx.x;
  const int nblk = (n + NB - 1) / NB;
  for (int kbI = nblk - 1; kbI >= 0; --kbI) {
    const int k0 = kbI * NB;
    const int kb = min(NB, n - k0);
    for (int e = tid; e < kb * kb; e += blockDim.x) {
      int i = e / kb, j = e % kb;
      D[i * NB + j] = (j <= i) ? L[(size_t)(k0 + i) * ldl + k0 + j] : O::zero();
    }
    if (tid < kb) rdiag[tid] = R(1) / O::re(L[(size_t)(k0 + tid) * ldl + k0 + tid]);
    __syncthreads();
    // diagonal: (L_kk^H) x = b  ->  x_r = (b_r - sum_{t>r} conj(D[t][r]) x_t) / D[r][r]
    for (int c = tid; c < nrhs; c += blockDim.x) {
      T x[NB];
      for (int r = kb - 1; r >= 0; --r) {
        T v = B[(size_t)(k0 + r) * ldb + c];
        for (int t = r + 1; t < kb; ++t) v = O::sub(v, O::mul(O::conj(D[t * NB + r]), x[t]));
        x[r] = O::scale(v, rdiag[r]);
        B[(size_t)(k0 + r) * ldb + c] = x[r];
      }
    }
    __syncthreads();
    // update rows above: B[i][c] -= sum_t conj(L[k0+t][i]) X[k0+t][c], i < k0
    for (int i0 = 0; i0 < k0; i0 += TL) {
      for (int e = tid; e < TL * NB; e += blockDim.x) {
        int r = e / NB, t = e % NB;     // Lt[r][t] = conj(L[k0+t][i0+r])
        Lt[e] = (i0 + r < k0 && t < kb) ? O::conj(L[(size_t)(k0 + t) * ldl + i0 + r]) : O::zero();
      }
      for (int c0 = 0; c0 < nrhs; c0 += TL) {
        for (int e = tid; e < NB * TL; e += blockDim.x) {
          int t = e / TL, c = e % TL;
          Xt[e] = (t < kb && c0 + c < nrhs) ? B[(size_t)(k0 + t) * ldb + c0 + c] : O::zero();
        }
        __syncthreads();
        for (int e = tid; e < TL * TL; e += blockDim.x) {
          int r = e / TL, c = e % TL;
          int i = i0 + r, cc = c0 + c;
          if (i < k0 && cc < nrhs) {
            T acc = O::zero();
            for (int t = 0; t < kb; ++t) acc = O::fma(Lt[r * NB + t], Xt[t * TL + c], acc);
            size_t o = (size_t)i * ldb + cc;
            B[o] = O::sub(B[o], acc);
          }
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();
}

// C (m x n) = beta*C + alpha * op(A) * B where op(A) = A^H (A is k x m,
// transA = true) or A (m x k).  B is k x n.  All of type T (alpha real).
// smem: 2*TL*NB elements of T.
template <class T>
__device__ void cta_gemm(bool transA, int m, int n, int k, typename Ops<T>::R alpha,
                         const T* A, int lda, const T* B, int ldb,
                         typename Ops<T>::R beta, T* C, int ldc, T* smem) {
  using O = Ops<T>;
  T* At = smem;               // At[r][t]: op(A)[i0+r][k0+t]
  T* Bt = smem + TL * NB;     // Bt[t][c]: B[k0+t][j0+c]
  const int tid = threadIdx.x;
  constexpr int PER = TL * TL / CTA_THREADS;   // outputs per thread
  for (int i0 = 0; i0 < m; i0 += TL) {
    for (int j0 = 0; j0 < n; j0 += TL) {
      T acc[PER];
      for (int q = 0; q < PER; ++q) acc[q] = O::zero();
      for (int k0 = 0; k0 < k; k0 += NB) {
        for (int e = tid; e < TL * NB; e += blockDim.x) {
          int r = e / NB, t = e % NB;
          T v = O::zero();
          if (i0 + r < m && k0 + t < k)
            v = transA ? O::conj(A[(size_t)(k0 + t) * lda + i0 + r]) : A[(size_t)(i0 + r) * lda + k0 + t];
          At[e] = v;
        }
        for (int e = tid; e < NB * TL; e += blockDim.x) {
          int t = e / TL, c = e % TL;
          Bt[e] = (k0 + t < k && j0 + c < n) ? B[(size_t)(k0 + t) * ldb + j0 + c] : O::zero();
        }
        __syncthreads();
        for (int q = 0; q < PER; ++q) {
          int e = tid + q * CTA_THREADS;
          int r = e / TL, c = e % TL;
          T a = acc[q];
#pragma unroll 8
          for (int t = 0; t < NB; ++t) a = O::fma(At[r * NB + t], Bt[t * TL + c], a);
          acc[q] = a;
        }
        __syncthreads();
      }
      for (int q = 0; q < PER; ++q) {
        int e = tid + q * CTA_THREADS;
        int r = e / TL, c = e % TL;
        int i = i0 + r, j = j0 + c;
        if (i < m && j < n) {
          size_t o = (size_t)i * ldc + j;
          T v = O::scale(acc[q], alpha);
          C[o] = (beta == 0) ? v : O::add(O::scale(C[o], beta), v);
        }
      }
    }
  }
  __syncthreads();
}

// X = L^-1 in place of X = I (L lower triangular, n x n).  Blocks of X above
// the diagonal stay zero and are skipped: n^3/6 multiply-adds.
// smem: as cta_trsm_lower<T, T>.
template <class T, bool CL = false>
__device__ void cta_trinv_lower(const T* L, int n, int ldl, T* X, int ldx, char* smem, Team<CL> tm = Team<CL>()) {
  using O = Ops<T>;
  using R = typename O::R;
  T* D = reinterpret_cast<T*>(smem);
  T* Lt = D + NB * NB;
  T* Xt = Lt + TL * NB;
  __shared__ R rdiag[NB];
  const int tid = threadIdx.x;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    const int k1 = k0 + kb;
    for (int e = tid; e < kb * kb; e += blockDim.x) {
      int i = e / kb, j = e % kb;
      D[i * NB + j] = (j <= i) ? tm.ld(&L[(size_t)(k0 + i) * ldl + k0 + j]) : O::zero();
    }
    if (tid < kb) rdiag[tid] = R(1) / O::re(tm.ld(&L[(size_t)(k0 + tid) * ldl + k0 + tid]));
    __syncthreads();
    for (int c = tid; c < k1; c += blockDim.x) {
      if (!tm.own_col(c / TL)) continue;
      T x[NB];
      for (int r = 0; r < kb; ++r) {
        T v = tm.ld(&X[(size_t)(k0 + r) * ldx + c]);
        for (int t = 0; t < r; ++t) v = O::fnma(D[r * NB + t], x[t], v);
        x[r] = O::scale(v, rdiag[r]);
        X[(size_t)(k0 + r) * ldx + c] = x[r];
      }
    }
    __syncthreads();
    for (int i0 = k1; i0 < n; i0 += TL) {
      for (int e = tid; e < TL * NB; e += blockDim.x) {
        int r = e / NB, t = e % NB;
        Lt[e] = (i0 + r < n && t < kb) ? tm.ld(&L[(size_t)(i0 + r) * ldl + k0 + t]) : O::zero();
      }
      for (int c0 = 0; c0 < k1; c0 += TL) {
        if (!tm.own_col(c0 / TL)) continue;
        for (int e = tid; e < NB * TL; e += blockDim.x) {
          int t = e / TL, c = e % TL;
          Xt[e] = (t < kb && c0 + c < k1) ? tm.ld(&X[(size_t)(k0 + t) * ldx + c0 + c]) : O::zero();
        }
        __syncthreads();
        for (int e = tid; e < TL * TL; e += blockDim.x) {
          int r = e / TL, c = e % TL;
          int i = i0 + r, cc = c0 + c;
          if (i < n && cc < k1) {
            T acc = O::zero();
            for (int t = 0; t < kb; ++t) acc = O::fma(Lt[r * NB + t], Xt[t * TL + c], acc);
            size_t o = (size_t)i * ldx + cc;
            X[o] = O::sub(tm.ld(&X[o]), acc);
          }
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();
}

// M = X^H X (M n x n, X kdim x n): only the lower tiles are computed, the
// strictly upper tiles are written as their conjugate mirror (half the flops
// of a full product).  With `tri` X is lower triangular (kdim = n) and each
// tile sums only over rows k >= its first row (X[k][i] = 0 for k < i):
// n^3/6 multiply-adds.  smem: 2*TL*NB elements of T.
template <class T, bool CL = false>
__device__ void cta_herk_lower(const T* X, int kdim, int n, int ldx, T* M, int ldm, T* smem, bool tri,
                               Team<CL> tm = Team<CL>()) {
  using O = Ops<T>;
  T* At = smem;
  T* Bt = smem + TL * NB;
  const int tid = threadIdx.x;
  constexpr int PER = TL * TL / CTA_THREADS;
  for (int i0 = 0; i0 < n; i0 += TL) {
    for (int j0 = 0; j0 <= i0; j0 += TL) {
      if (!tm.own2(i0 / TL, j0 / TL)) continue;
      T acc[PER];
      for (int q = 0; q < PER; ++q) acc[q] = O::zero();
      for (int k0 = tri ? i0 : 0; k0 < kdim; k0 += NB) {
        for (int e = tid; e < TL * NB; e += blockDim.x) {
          int r = e / NB, t = e % NB;
          At[e] = (i0 + r < n && k0 + t < kdim) ? O::conj(tm.ld(&X[(size_t)(k0 + t) * ldx + i0 + r])) : O::zero();
        }
        for (int e = tid; e < NB * TL; e += blockDim.x) {
          int t = e / TL, c = e % TL;
          Bt[e] = (k0 + t < kdim && j0 + c < n) ? tm.ld(&X[(size_t)(k0 + t) * ldx + j0 + c]) : O::zero();
        }
        __syncthreads();
        for (int q = 0; q < PER; ++q) {
          int e = tid + q * CTA_THREADS;
          int r = e / TL, c = e % TL;
          T a = acc[q];
#pragma unroll 8
          for (int t = 0; t < NB; ++t) a = O::fma(At[r * NB + t], Bt[t * TL + c], a);
          acc[q] = a;
        }
        __syncthreads();
      }
      for (int q = 0; q < PER; ++q) {
        int e = tid + q * CTA_THREADS;
        int r = e / TL, c = e % TL;
        int i = i0 + r, j = j0 + c;
        if (i < n && j < n) {
          M[(size_t)i * ldm + j] = acc[q];
          if (j0 < i0) M[(size_t)j * ldm + i] = O::conj(acc[q]);
        }
      }
    }
  }
  __syncthreads();
}

template <class T, bool CL = false>
__device__ void cta_herk_lower_tri(const T* X, int n, int ldx, T* M, int ldm, T* smem, Team<CL> tm = Team<CL>()) {
  cta_herk_lower<T, CL>(X, n, n, ldx, M, ldm, smem, true, tm);
}

}  // namespace dpgmg
