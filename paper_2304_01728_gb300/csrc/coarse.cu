// Coarsest level of the V-cycle: direct solve with the dense operator A_0
// (the paper solves its initial mesh directly, Sec. 4 list).
//
// Setup (in the V-cycle precision: complex128 on the FP64 path, complex64 on
// the mixed path):
//   A_0 = sum of the level-0 element matrices      (dense, N0 x N0)
//   A_0 = L L^H                                    (blocked right-looking Cholesky)
//   X   = L^-1                                     (blocked forward substitution, B = I)
// X is stored packed twice: its lower triangle by rows and its conjugate
// transpose (upper triangle of L^-H) by rows, so each V-cycle application
//   e = L^-H (L^-1 r)
// is two dense triangular matrix-vector products with no sequential
// dependency between rows (one warp per row, coalesced row reads).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace dpgmg {

constexpr int CNB = 64;   // block width of the dense kernels

template <class C> __device__ __forceinline__ C warp_sum_c(C v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// one colour pass (elem_color) of the dense assembly: no two elements of the pass share a DOF
__global__ void k_dense_scatter(double2* A, int64_t N, const double2* E, const int64_t* dofs, int nloc, int n0,
                                int n1, int color) {
  const int64_t e = blockIdx.x;
  if (elem_color(e, n0, n1) != color) return;
  for (int q = blockIdx.y * blockDim.x + threadIdx.x; q < nloc * nloc; q += gridDim.y * blockDim.x) {
    int i = q / nloc, j = q % nloc;
    int64_t gi = dofs[e * nloc + i], gj = dofs[e * nloc + j];
    if (gi < 0 || gj < 0) continue;
    const double2 v = E[e * (size_t)nloc * nloc + q];
    double2& o = A[gi * N + gj];
    o = make_double2(o.x + v.x, o.y + v.y);
  }
}

__global__ void k_narrow_mat(const double2* a, float2* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// ---------------------------------------------------------------- Cholesky
// One CTA per step: Cholesky of the diagonal block A[k0:k0+kb, k0:k0+kb]
// (written back, lower triangle) and its triangular inverse L_kk^-1, stored
// as a CNB x CNB block (zero outside the kb x kb lower triangle) at
// Dinv + (k0 / CNB) CNB^2: the panel below is then a plain product with it,
// and the inverse phase reuses it.
template <class C>
__global__ void __launch_bounds__(CTA_THREADS) k_dense_diag(C* A, int64_t N, int64_t ld, int k0, C* Dinv,
                                                            int* info) {
  extern __shared__ unsigned char shraw[];
  using O = Ops<C>;
  using R = typename O::R;
  constexpr int LD = CNB + 1;
  C* D = reinterpret_cast<C*>(shraw);   // [CNB][LD] the block, then L_kk
  C* X = D + CNB * LD;                  // [CNB][LD] L_kk^-1
  __shared__ R rdiag[CNB];
  const int kb = (int)(N - k0 < CNB ? N - k0 : CNB);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (int q = tid; q < kb * kb; q += blockDim.x) {
    const int i = q / kb, c = q % kb;
    D[i * LD + c] = c <= i ? A[(size_t)(k0 + i) * ld + k0 + c] : O::zero();
  }
  __syncthreads();
  // right-looking, one barrier per column: step j updates the trailing lower
  // entries with L[i][j] conj(L[c][j]) (column j scaled on the fly) and writes
  // the scaled column j - 1, which step j does not read
  int bad = 0;
  R sprev = R(1), rsprev = R(1);
  for (int j = 0; j < kb; ++j) {
    R d = O::re(D[j * LD + j]);
    if (!(d > R(0))) {
      if (!bad) bad = k0 + j + 1;
      d = R(1);
    }
    const R s = sqrt(d), rs = R(1) / s;
    if (j > 0)
      for (int i = j - 1 + tid; i < kb; i += blockDim.x)
        D[i * LD + j - 1] = i == j - 1 ? O::from_re(sprev) : O::scale(D[i * LD + j - 1], rsprev);
    for (int i = j + 1 + ty; i < kb; i += 16) {
      const C lij = O::scale(D[i * LD + j], rs);
      for (int c = j + 1 + tx; c <= i; c += 16) D[i * LD + c] = O::fnmac(lij, O::scale(D[c * LD + j], rs), D[i * LD + c]);
    }
    sprev = s;
    rsprev = rs;
    __syncthreads();
  }
  for (int i = kb - 1 + tid; i < kb; i += blockDim.x) D[i * LD + kb - 1] = O::from_re(sprev);
  __syncthreads();
  for (int q = tid; q < kb * kb; q += blockDim.x) {
    const int i = q / kb, c = q % kb;
    if (c <= i) A[(size_t)(k0 + i) * ld + k0 + c] = D[i * LD + c];
  }
  if (tid < kb) rdiag[tid] = R(1) / O::re(D[tid * LD + tid]);
  __syncthreads();
  // X = L_kk^-1 row by row: X[r][c] = (delta_rc - sum_{c<=t<r} L[r][t] X[t][c]) / L[r][r];
  // four lanes per column split the sum
  const int col = tid / 4, part = tid % 4;
  for (int r = 0; r < kb; ++r) {
    C acc = O::zero();
    if (col <= r && col < kb)
      for (int t = col + part; t < r; t += 4) acc = O::fma(D[r * LD + t], X[t * LD + col], acc);
    for (int o = 1; o < 4; o <<= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (part == 0 && col <= r && col < kb)
      X[r * LD + col] = O::scale(O::sub(r == col ? O::from_re(R(1)) : O::zero(), acc), rdiag[r]);
    __syncthreads();
  }
  C* Dk = Dinv + (size_t)(k0 / CNB) * CNB * CNB;
  for (int q = tid; q < CNB * CNB; q += blockDim.x) {
    const int r = q / CNB, c = q % CNB;
    Dk[q] = (r < kb && c <= r) ? X[r * LD + c] : O::zero();
  }
  if (tid == 0 && bad) atomicOr(info, 16);
}

// Panel: rows i >= k0 + kb, A[i, k0:k0+kb] <- A[i, k0:k0+kb] L_kk^-H, as the
// product with the stored inverse (one CTA per 64 rows; thread (tx, ty) owns
// rows ty*4 + a and columns tx + 16 b).
template <class C>
__global__ void __launch_bounds__(CTA_THREADS) k_dense_panel(C* A, int64_t N, int64_t ld, int k0,
                                                             const C* __restrict__ Dinv) {
  extern __shared__ unsigned char shraw[];
  using O = Ops<C>;
  constexpr int LD = CNB + 1;
  C* Pa = reinterpret_cast<C*>(shraw);   // [CNB][LD] Pa[r][t] = A[i0 + r][k0 + t]
  C* Bt = Pa + CNB * LD;                 // [CNB][LD] Bt[t][j] = conj(L_kk^-1[j][t])
  const int kb = (int)(N - k0 < CNB ? N - k0 : CNB);
  const int64_t i0 = (int64_t)k0 + kb + (int64_t)blockIdx.x * CNB;
  const C* Dk = Dinv + (size_t)(k0 / CNB) * CNB * CNB;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (int q = tid; q < CNB * CNB; q += blockDim.x) {
    const int r = q / CNB, t = q % CNB;
    Pa[r * LD + t] = (i0 + r < N && t < kb) ? A[(size_t)(i0 + r) * ld + k0 + t] : O::zero();
    Bt[t * LD + r] = O::conj(Dk[q]);
  }
  __syncthreads();
  C acc[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) acc[a][b] = O::zero();
  for (int t = 0; t < kb; ++t) {
    C av[4], bv[4];
    for (int a = 0; a < 4; ++a) av[a] = Pa[(ty * 4 + a) * LD + t];
    for (int b = 0; b < 4; ++b) bv[b] = Bt[t * LD + tx + 16 * b];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) acc[a][b] = O::fma(av[a], bv[b], acc[a][b]);
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const int64_t i = i0 + ty * 4 + a;
      const int j = tx + 16 * b;
      if (i < N && j < kb) A[(size_t)i * ld + k0 + j] = acc[a][b];
    }
}

// trailing update of one lower 64x64 tile pair: A[i][j] -= sum_t L[i][t] conj(L[j][t])
template <class C>
__global__ void __launch_bounds__(CTA_THREADS) k_dense_herk(C* A, int64_t N, int64_t ld, int k0) {
  __shared__ C Pi[CNB][17];
  __shared__ C Pj[CNB][17];
  using O = Ops<C>;
  const int kb = (int)(N - k0 < CNB ? N - k0 : CNB);
  const int64_t k1 = k0 + kb;
  int64_t t = blockIdx.x;
  int64_t bi = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) / 2.0);
  while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
  while (bi * (bi + 1) / 2 > t) --bi;
  const int64_t bj = t - bi * (bi + 1) / 2;
  const int64_t i0 = k1 + bi * CNB, j0 = k1 + bj * CNB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  C acc[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) acc[a][b] = O::zero();
  for (int t0 = 0; t0 < kb; t0 += 16) {
    for (int q = threadIdx.x; q < CNB * 16; q += blockDim.x) {
      int r = q / 16, c = q % 16;
      int64_t ii = i0 + r, jj = j0 + r;
      Pi[r][c] = (ii < N && t0 + c < kb) ? A[ii * ld + k0 + t0 + c] : O::zero();
      Pj[r][c] = (jj < N && t0 + c < kb) ? A[jj * ld + k0 + t0 + c] : O::zero();
    }
    __syncthreads();
    // thread (tx, ty) owns rows ty*4 + a and columns tx + 16 b: the 16 lanes of
    // a half-warp read 16 consecutive rows of Pj (row stride 17: distinct banks)
    for (int c = 0; c < 16; ++c) {
      C av[4], bv[4];
      for (int a = 0; a < 4; ++a) av[a] = Pi[ty * 4 + a][c];
      for (int b = 0; b < 4; ++b) bv[b] = Pj[tx + 16 * b][c];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) acc[a][b] = O::fmac(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      int64_t i = i0 + ty * 4 + a, j = j0 + tx + 16 * b;
      if (i < N && j <= i) {
        C& o = A[i * ld + j];
        o = O::sub(o, acc[a][b]);
      }
    }
}

// Blocked right-looking Cholesky A = L L^H in place (lower) of the n x n view A
// (leading dimension ld); Dinv receives the inverses of its 64 x 64 diagonal
// blocks of L (block b at Dinv + b 64^2).
template <class C>
static void dense_cholesky(C* A, int64_t n, int64_t ld, C* Dinv, int* info, cudaStream_t st) {
  const size_t sm = (size_t)2 * CNB * (CNB + 1) * sizeof(C);
  DPG_CUDA(cudaFuncSetAttribute(k_dense_diag<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  DPG_CUDA(cudaFuncSetAttribute(k_dense_panel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  for (int64_t k0 = 0; k0 < n; k0 += CNB) {
    int kb = (int)std::min<int64_t>(CNB, n - k0);
    k_dense_diag<C><<<1, CTA_THREADS, sm, st>>>(A, n, ld, (int)k0, Dinv, info);
    DPG_CHECK_LAUNCH();
    int64_t rows = n - k0 - kb;
    if (rows <= 0) break;
    k_dense_panel<C><<<(unsigned)((rows + CNB - 1) / CNB), CTA_THREADS, sm, st>>>(A, n, ld, (int)k0, Dinv);
    DPG_CHECK_LAUNCH();
    int64_t nt = (rows + CNB - 1) / CNB;
    k_dense_herk<C><<<(unsigned)(nt * (nt + 1) / 2), CTA_THREADS, 0, st>>>(A, n, ld, (int)k0);
    DPG_CHECK_LAUNCH();
  }
}

// ---------------------------------------------------------- L^-1 (blocked)
// X[kb rows, tile cols] <- Dinv_kb * X[kb rows, tile cols], one CTA per 64-column tile
template <class C>
__global__ void __launch_bounds__(CTA_THREADS) k_trinv_scale(C* X, const C* Dinv, int64_t N, int64_t ld, int kb) {
  extern __shared__ unsigned char shraw[];
  C* D = reinterpret_cast<C*>(shraw);
  C* T = D + CNB * CNB;
  using O = Ops<C>;
  const int64_t k0 = (int64_t)kb * CNB;
  const int kw = (int)(N - k0 < CNB ? N - k0 : CNB);
  const int64_t c0 = (int64_t)blockIdx.x * CNB;
  const int cw = (int)(N - c0 < CNB ? N - c0 : CNB);
  const C* Dk = Dinv + (size_t)kb * CNB * CNB;
  for (int q = threadIdx.x; q < CNB * CNB; q += blockDim.x) {
    D[q] = Dk[q];
    int r = q / CNB, c = q % CNB;
    T[q] = (r < kw && c < cw) ? X[(k0 + r) * ld + c0 + c] : O::zero();
  }
  __syncthreads();
  for (int q = threadIdx.x; q < CNB * CNB; q += blockDim.x) {
    int r = q / CNB, c = q % CNB;
    if (r >= kw || c >= cw) continue;
    C acc = O::zero();
    for (int t = 0; t <= r; ++t) acc = O::fma(D[r * CNB + t], T[t * CNB + c], acc);
    X[(k0 + r) * ld + c0 + c] = acc;
  }
}

// X[ib, jb] -= L[ib, kb] X[kb, jb] for ib > kb, jb <= kb (64x64 tiles)
template <class C>
__global__ void __launch_bounds__(CTA_THREADS) k_trinv_update(C* X, const C* L, int64_t N, int64_t ld, int kb) {
  __shared__ C La[CNB][17];
  __shared__ C Xb[16][CNB + 1];
  using O = Ops<C>;
  const int64_t k0 = (int64_t)kb * CNB;
  const int kw = (int)(N - k0 < CNB ? N - k0 : CNB);
  const int ncol = kb + 1;
  const int64_t ib = kb + 1 + blockIdx.x / ncol;
  const int64_t jb = blockIdx.x % ncol;
  const int64_t i0 = ib * CNB, j0 = jb * CNB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  C acc[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) acc[a][b] = O::zero();
  for (int t0 = 0; t0 < kw; t0 += 16) {
    for (int q = threadIdx.x; q < CNB * 16; q += blockDim.x) {
      int r = q / 16, c = q % 16;
      La[r][c] = (i0 + r < N && t0 + c < kw) ? L[(i0 + r) * ld + k0 + t0 + c] : O::zero();
      int t = q / CNB, cc = q % CNB;
      Xb[t][cc] = (t0 + t < kw && j0 + cc < N) ? X[(k0 + t0 + t) * ld + j0 + cc] : O::zero();
    }
    __syncthreads();
    for (int c = 0; c < 16; ++c) {
      C av[4], bv[4];
      for (int a = 0; a < 4; ++a) av[a] = La[ty * 4 + a][c];
      for (int b = 0; b < 4; ++b) bv[b] = Xb[c][tx + 16 * b];   // consecutive columns: distinct banks
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) acc[a][b] = O::fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      int64_t i = i0 + ty * 4 + a, j = j0 + tx + 16 * b;
      if (i < N && j < N) {
        C& o = X[i * ld + j];
        o = O::sub(o, acc[a][b]);
      }
    }
}

template <class C>
__global__ void k_identity_lower(C* X, int64_t N, int64_t ld) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N * N; q += (int64_t)gridDim.x * blockDim.x)
    X[(q / N) * ld + q % N] = (q / N == q % N) ? Ops<C>::from_re(1) : Ops<C>::zero();
}

// Lp: rows of the lower triangle of X; Up: rows of X^H (upper triangle)
template <class C>
__global__ void k_pack(const C* X, int64_t N, C* Lp, C* Up) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N * N; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = q / N, j = q % N;
    if (j > i) continue;
    C v = X[q];
    Lp[i * (i + 1) / 2 + j] = v;
    // X^H[j][i] = conj(X[i][j]) goes to row j of the upper packing at column i
    Up[j * N - j * (j - 1) / 2 + (i - j)] = Ops<C>::conj(v);
  }
}

// X = L^-1 of the n x n lower view L into the view X (both leading dimension
// ld), with the diagonal-block inverses Dinv of dense_cholesky.
template <class C>
static void dense_trinv(const C* L, C* X, int64_t n, int64_t ld, const C* Dinv, cudaStream_t st) {
  const int nb = (int)((n + CNB - 1) / CNB);
  k_identity_lower<C><<<(unsigned)std::min<int64_t>(1216, (n * n + 255) / 256), 256, 0, st>>>(X, n, ld);
  DPG_CHECK_LAUNCH();
  const size_t sms = (size_t)2 * CNB * CNB * sizeof(C);
  DPG_CUDA(cudaFuncSetAttribute(k_trinv_scale<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms));
  for (int kb = 0; kb < nb; ++kb) {
    k_trinv_scale<C><<<kb + 1, CTA_THREADS, sms, st>>>(X, Dinv, n, ld, kb);
    DPG_CHECK_LAUNCH();
    const int rows = nb - kb - 1;
    if (rows > 0) {
      k_trinv_update<C><<<(unsigned)(rows * (kb + 1)), CTA_THREADS, 0, st>>>(X, L, n, ld, kb);
      DPG_CHECK_LAUNCH();
    }
  }
}

// Complex64 products on the tensor cores (tc_gemm.cu).
void tc_configure();
size_t tc_image_bytes(int64_t rows, int64_t kc, bool is_a);
void tc_pack(void* img, const float2* src, int64_t ld, int64_t rows, int64_t kc, int mode, cudaStream_t st);
void tc_gemm(const void* Aimg, const void* Bimg, int64_t M, int64_t N, int64_t kc, float2* C, int64_t ldc,
             float alpha, float beta, int lower, int* err, int fault, cudaStream_t st);
enum { TC_A_NH = 0, TC_A_NN = 1, TC_B = 2, TC_B_TRANS = 3 };

// Panel width of the tensor-core factorisation (a multiple of 64 and of 16).
static int64_t tc_panel(int64_t N) { return N >= 4096 ? 512 : (N >= 1024 ? 256 : 128); }

// Mixed path: A = L L^H and X = L^-1 (complex64, N x N, row-major, lower
// halves) by panels of width W, right-looking.  Per panel K (rows and
// columns K0 .. K0 + W - 1), with the rows below it "2":
//   L_KK, L_KK^-1 (into X_KK)   64-wide blocked kernels on the CUDA cores
//   X_K,<K = -L_KK^-1 T_K,<K     tensor cores (T accumulated in X, below)
//   L_2K = A_2K L_KK^-H          tensor cores, in place of A_2K
//   A_22 -= L_2K L_2K^H          tensor cores, lower tiles only
//   T_2,<=K += L_2K X_K,<=K      tensor cores
// which gives X_IJ = -L_II^-1 sum_{J<=K<I} L_IK X_KJ for every block below
// the diagonal.  fault (tests): the first product issues no MMA.
static void tc_cholesky_inverse(Alloc& Al, float2* A, float2* X, int64_t N, float2* Dinv, int* info, int fault,
                                cudaStream_t st) {
  tc_configure();
  const int64_t W = tc_panel(N);
  void* Aimg = Al.get(tc_image_bytes(N, W, true));
  void* Bimg = Al.get(tc_image_bytes(N, W, false));
  DPG_CUDA(cudaMemsetAsync(X, 0, (size_t)N * N * sizeof(float2), st));
  int first = fault;
  auto gemm = [&](int64_t M, int64_t Nc, int64_t kc, float2* C, float alpha, float beta, int lower) {
    tc_gemm(Aimg, Bimg, M, Nc, kc, C, N, alpha, beta, lower, info, first, st);
    first = 0;
  };
  for (int64_t K0 = 0; K0 < N; K0 += W) {
    const int64_t kb = std::min<int64_t>(W, N - K0);
    float2* Akk = A + K0 * N + K0;
    float2* Xkk = X + K0 * N + K0;
    float2* Dk = Dinv + (K0 / CNB) * CNB * CNB;
    dense_cholesky<float2>(Akk, kb, N, Dk, info, st);
    dense_trinv<float2>(Akk, Xkk, kb, N, Dk, st);
    if (K0 > 0) {   // X_K,<K = -L_KK^-1 T_K,<K (T read into the image before it is overwritten)
      tc_pack(Aimg, Xkk, N, kb, kb, TC_A_NN, st);
      tc_pack(Bimg, X + K0 * N, N, K0, kb, TC_B_TRANS, st);
      gemm(kb, K0, kb, X + K0 * N, -1.f, 0.f, 0);
    }
    const int64_t rows = N - K0 - kb;
    if (rows <= 0) break;
    float2* A2 = A + (K0 + kb) * N + K0;   // rows below the panel, panel columns
    // L_2K = A_2K L_KK^-H
    tc_pack(Aimg, A2, N, rows, kb, TC_A_NH, st);
    tc_pack(Bimg, Xkk, N, kb, kb, TC_B, st);
    gemm(rows, kb, kb, A2, 1.f, 0.f, 0);
    // A_22 -= L_2K L_2K^H
    tc_pack(Aimg, A2, N, rows, kb, TC_A_NH, st);
    tc_pack(Bimg, A2, N, rows, kb, TC_B, st);
    gemm(rows, rows, kb, A + (K0 + kb) * N + K0 + kb, -1.f, 1.f, 1);
    // T_2,<=K += L_2K X_K,<=K
    tc_pack(Aimg, A2, N, rows, kb, TC_A_NN, st);
    tc_pack(Bimg, X + K0 * N, N, K0 + kb, kb, TC_B_TRANS, st);
    gemm(rows, K0 + kb, kb, X + (K0 + kb) * N, 1.f, 1.f, 0);
  }
  Al.release(Bimg);
  Al.release(Aimg);
}

// tensor: 0 CUDA cores, 1 tensor cores (complex64 only), 2 tensor cores whose
// first product issues no MMA (the DPGMG_FLAG_FAULT_TC_WAIT test).
template <class C>
static void coarse_factor(Alloc& A, C* dense, int64_t N, C** Lp, C** Up, int* info, int tensor, cudaStream_t st) {
  const int nb = (int)((N + CNB - 1) / CNB);
  C* Dinv = A.arr<C>((size_t)nb * CNB * CNB);
  C* X = A.arr<C>((size_t)N * N);
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (tensor) tc_cholesky_inverse(A, dense, X, N, Dinv, info, tensor == 2 ? 1 : 0, st);
  }
  if (!tensor || sizeof(C) != sizeof(float2)) {
    dense_cholesky<C>(dense, N, N, Dinv, info, st);
    dense_trinv<C>(dense, X, N, N, Dinv, st);
  }
  const int64_t np = N * (N + 1) / 2;
  *Lp = A.arr<C>((size_t)np);
  *Up = A.arr<C>((size_t)np);
  k_pack<C><<<1216, 256, 0, st>>>(X, N, *Lp, *Up);
  DPG_CHECK_LAUNCH();
  DPG_CUDA(cudaStreamSynchronize(st));
  A.release(X);
  A.release(Dinv);
}

void coarse_setup(SystemImpl& S, Level& C0, int* info, cudaStream_t st, Alloc& A) {
  const int64_t N = C0.mesh.ndof;
  C0.N0 = N;
  double2* dense = A.arr<double2>((size_t)N * N);
  DPG_CUDA(cudaMemsetAsync(dense, 0, (size_t)N * N * sizeof(double2), st));
  for (int c = 0; c < 8; ++c) {
    const unsigned slices = (unsigned)std::max(1, std::min(64, (C0.nloc * C0.nloc + 2047) / 2048));
    k_dense_scatter<<<dim3((unsigned)C0.mesh.nelem, slices), 256, 0, st>>>(dense, N, C0.E, C0.dofs, C0.nloc,
                                                                          C0.mesh.n[0], C0.mesh.n[1], c);
    DPG_CHECK_LAUNCH();
  }
  if (S.op.flags & DPGMG_FLAG_FAULT_NOT_HPD) {
    // host-made failure for the error-path tests: a negative first pivot
    static const double2 neg = make_double2(-1.0, 0.0);
    DPG_CUDA(cudaMemcpyAsync(dense, &neg, sizeof(double2), cudaMemcpyHostToDevice, st));
  }
  if (S.op.precision == DPGMG_PREC_MIXED) {
    float2* d32 = A.arr<float2>((size_t)N * N);
    k_narrow_mat<<<1216, 256, 0, st>>>(dense, d32, N * N);
    DPG_CHECK_LAUNCH();
    DPG_CUDA(cudaStreamSynchronize(st));
    A.release(dense);
    const int tc = (S.op.flags & DPGMG_FLAG_CUDA_CORES) ? 0 : ((S.op.flags & DPGMG_FLAG_FAULT_TC_WAIT) ? 2 : 1);
    coarse_factor<float2>(A, d32, N, &C0.Lp32, &C0.Up32, info, tc, st);
    A.release(d32);
  } else {
    coarse_factor<double2>(A, dense, N, &C0.Lp64, &C0.Up64, info, 0, st);
    A.release(dense);
  }
  C0.has_coarse = true;
}

// ------------------------------------------------------------------ apply
// One warp per row pair (i, N-1-i): every warp reads N+1 entries.  Four
// streaming loads per lane per step keep enough bytes in flight; the two
// accumulators take the entries in the same order as a two-load loop (a0:
// t, t + 64, ...; a1: t + 32, t + 96, ...), so the result is bitwise that
// of the plain loop the V-cycle's tolerances were measured with.
template <class C>
__device__ __forceinline__ C dot_row(const C* __restrict__ row, const C* __restrict__ v, int64_t len, int lane) {
  using O = Ops<C>;
  C a0 = O::zero(), a1 = O::zero();
  int64_t t = lane;
  for (; t + 96 < len; t += 128) {
    const C m0 = __ldcs(row + t), m1 = __ldcs(row + t + 32), m2 = __ldcs(row + t + 64), m3 = __ldcs(row + t + 96);
    a0 = O::fma(m0, v[t], a0);
    a1 = O::fma(m1, v[t + 32], a1);
    a0 = O::fma(m2, v[t + 64], a0);
    a1 = O::fma(m3, v[t + 96], a1);
  }
  for (; t + 32 < len; t += 64) {
    a0 = O::fma(__ldcs(row + t), v[t], a0);
    a1 = O::fma(__ldcs(row + t + 32), v[t + 32], a1);
  }
  if (t < len) a0 = O::fma(__ldcs(row + t), v[t], a0);
  return warp_sum_c(O::add(a0, a1));
}

template <class C>
__global__ void __launch_bounds__(256) k_trmv_lower(const C* __restrict__ Lp, int64_t N, const C* __restrict__ r,
                                                    C* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t half = (N + 1) / 2;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); w < half; w += nw) {
    const int64_t i1 = w, i2 = N - 1 - w;
    C s1 = dot_row<C>(Lp + i1 * (i1 + 1) / 2, r, i1 + 1, lane);
    if (lane == 0) y[i1] = s1;
    if (i2 != i1) {
      C s2 = dot_row<C>(Lp + i2 * (i2 + 1) / 2, r, i2 + 1, lane);
      if (lane == 0) y[i2] = s2;
    }
  }
}

template <class C>
__global__ void __launch_bounds__(256) k_trmv_upper(const C* __restrict__ Up, int64_t N, const C* __restrict__ y,
                                                    C* __restrict__ e) {
  const int lane = threadIdx.x & 31;
  const int64_t half = (N + 1) / 2;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); w < half; w += nw) {
    const int64_t j1 = w, j2 = N - 1 - w;
    C s1 = dot_row<C>(Up + j1 * N - j1 * (j1 - 1) / 2, y + j1, N - j1, lane);
    if (lane == 0) e[j1] = s1;
    if (j2 != j1) {
      C s2 = dot_row<C>(Up + j2 * N - j2 * (j2 - 1) / 2, y + j2, N - j2, lane);
      if (lane == 0) e[j2] = s2;
    }
  }
}

template <class C>
static void coarse_apply_t(const C* Lp, const C* Up, int64_t N, const C* r, C* e, C* tmp, cudaStream_t st) {
  unsigned blocks = (unsigned)std::min<int64_t>(((N + 1) / 2 + 7) / 8, 152 * 16);
  k_trmv_lower<C><<<blocks, 256, 0, st>>>(Lp, N, r, tmp);
  DPG_CHECK_LAUNCH();
  k_trmv_upper<C><<<blocks, 256, 0, st>>>(Up, N, tmp, e);
  DPG_CHECK_LAUNCH();
}

// Block forms for KB right-hand sides (vectors at stride ld): each packed
// row is read once for the KB vectors.
template <class C, int KB>
__device__ __forceinline__ void dot_row_blk(const C* __restrict__ row, const C* __restrict__ v, int64_t ld,
                                            int64_t len, int lane, C out[KB]) {
  using O = Ops<C>;
  C a[KB];
#pragma unroll
  for (int kb = 0; kb < KB; ++kb) a[kb] = O::zero();
  int64_t t = lane;
  for (; t + 32 < len; t += 64) {
    const C m0 = __ldcs(row + t), m1 = __ldcs(row + t + 32);
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) {
      a[kb] = O::fma(m0, v[kb * ld + t], a[kb]);
      a[kb] = O::fma(m1, v[kb * ld + t + 32], a[kb]);
    }
  }
  if (t < len) {
    const C m0 = __ldcs(row + t);
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) a[kb] = O::fma(m0, v[kb * ld + t], a[kb]);
  }
#pragma unroll
  for (int kb = 0; kb < KB; ++kb) out[kb] = warp_sum_c(a[kb]);
}

// UPPER = false: y = L^-1 r (packed lower rows); true: e = L^-H y (packed
// upper rows, row j starts at column j)
template <class C, int KB, bool UPPER>
__global__ void __launch_bounds__(256) k_trmv_blk(const C* __restrict__ Tp, int64_t N, const C* __restrict__ x,
                                                  C* __restrict__ y, int64_t ld) {
  const int lane = threadIdx.x & 31;
  const int64_t half = (N + 1) / 2;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); w < half; w += nw) {
    for (int side = 0; side < 2; ++side) {
      const int64_t i = side ? N - 1 - w : w;
      if (side && i == w) break;
      C s[KB];
      if (UPPER) dot_row_blk<C, KB>(Tp + i * N - i * (i - 1) / 2, x + i, ld, N - i, lane, s);
      else dot_row_blk<C, KB>(Tp + i * (i + 1) / 2, x, ld, i + 1, lane, s);
      if (lane < KB) {
        C mine = s[0];
#pragma unroll
        for (int kb = 1; kb < KB; ++kb)
          if (lane == kb) mine = s[kb];
        y[lane * ld + i] = mine;
      }
    }
  }
}

template <class C>
static void coarse_apply_blk_t(const C* Lp, const C* Up, int64_t N, const C* r, C* e, C* tmp, int K,
                               cudaStream_t st) {
  unsigned blocks = (unsigned)std::min<int64_t>(((N + 1) / 2 + 7) / 8, 152 * 16);
  for (int g = 0; g < K; g += 4) {
    const int kb = std::min(4, K - g);
    const C* rg = r + g * N;
    C* tg = tmp + g * N;
    C* eg = e + g * N;
#define DPG_TRMV_BLK(KB)                                                      \
  k_trmv_blk<C, KB, false><<<blocks, 256, 0, st>>>(Lp, N, rg, tg, N);         \
  DPG_CHECK_LAUNCH();                                                         \
  k_trmv_blk<C, KB, true><<<blocks, 256, 0, st>>>(Up, N, tg, eg, N);          \
  DPG_CHECK_LAUNCH()
    if (kb == 4) { DPG_TRMV_BLK(4); }
    else if (kb == 3) { DPG_TRMV_BLK(3); }
    else if (kb == 2) { DPG_TRMV_BLK(2); }
    else { DPG_TRMV_BLK(1); }
#undef DPG_TRMV_BLK
  }
}

// K right-hand sides at stride N0; tmp holds K * N0 values
void coarse_apply64_blk(const Level& C0, const double2* r, double2* e, double2* tmp, int K, cudaStream_t st) {
  coarse_apply_blk_t<double2>(C0.Lp64, C0.Up64, C0.N0, r, e, tmp, K, st);
}
void coarse_apply32_blk(const Level& C0, const float2* r, float2* e, float2* tmp, int K, cudaStream_t st) {
  coarse_apply_blk_t<float2>(C0.Lp32, C0.Up32, C0.N0, r, e, tmp, K, st);
}

void coarse_apply64(const Level& C0, const double2* r, double2* e, double2* tmp, cudaStream_t st) {
  coarse_apply_t<double2>(C0.Lp64, C0.Up64, C0.N0, r, e, tmp, st);
}
void coarse_apply32(const Level& C0, const float2* r, float2* e, float2* tmp, cudaStream_t st) {
  coarse_apply_t<float2>(C0.Lp32, C0.Up32, C0.N0, r, e, tmp, st);
}

}  // namespace dpgmg
