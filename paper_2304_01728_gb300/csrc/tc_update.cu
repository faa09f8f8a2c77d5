// Complex64 tile updates of the coarsest-level factorisation on the tensor
// cores (tcgen05, TF32 operands from shared memory, FP32 accumulator in TMEM).
// Used by the mixed path's coarsest factor (Sec. 4 list: direct solve on the
// initial mesh), whose work is two sequences of rank-64 updates:
//
//   HERK (blocked Cholesky):   C[i][j] -= sum_t A[i][k0+t] conj(A[j][k0+t])   (tiles with j <= i)
//   GEMM (blocked L^-1):       C[i][j] -= sum_t A[i][k0+t] B[k0+t][j]
//
// Real form.  A complex product is one real contraction over interleaved
// (re, im) pairs: with b' = (Re b, Im b) for every output column,
//   HERK   Re = <(ar, ai), b'>    Im = <(ai, -ar), b'>
//   GEMM   Re = <(ar, -ai), b'>   Im = <(ai, ar), b'>
// so one 64 x 64 complex output tile is one 128 x 64 real tile: D rows 0..63
// hold real parts, rows 64..127 imaginary parts (M = 128, N = 64).
//
// Precision (3xTF32).  Every FP32 operand value x is split into TF32 parts
// hi = rna(x), lo = rna(x - hi), and D = A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the lo*lo term is below FP32 rounding).  The products keep ~22 bits of
// each operand, close to the FP32 arithmetic of the CUDA-core kernels.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, adjacent along K at 128 B (leading byte
// offset) and along M/N at (K/4) * 128 B (stride byte offset).  One CTA of 4
// warps per output tile; the K = 64 complex columns run in two passes of 32.
#include <cstdint>

#include "internal.h"

namespace dpgmg {

namespace {

constexpr int TC_T = 64;                      // complex tile edge
constexpr int TC_KP = 64;                     // real K values per pass (32 complex)
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_A_BYTES = 128 * TC_KP * 4;   // 32 KiB
constexpr uint32_t TC_B_BYTES = 64 * TC_KP * 4;    // 16 KiB
constexpr uint32_t TC_SMEM = 2 * TC_A_BYTES + 2 * TC_B_BYTES + 1024;
constexpr int TC_HERK = 0, TC_GEMM = 1;
constexpr long long TC_WAIT_LIMIT = 1LL << 24;             // polls of one wait, at most
constexpr unsigned long long TC_WAIT_NS = 500000000ull;    // and at most 0.5 s of wall time

// byte offset of element (row r, K index k) in the canonical layout
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)(((r >> 3) * (TC_KP / 4) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor: start >> 4, leading byte offset 128,
// stride byte offset (K/4) * 128, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(((uint32_t)(TC_KP / 4) * 128u) >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// (v0, v1) at K indices (k, k + 1), k even, as TF32 hi and lo parts
__device__ __forceinline__ void store_split(unsigned char* hi, unsigned char* lo, int r, int k, float v0, float v1) {
  const float h0 = tf32_rna(v0), h1 = tf32_rna(v1);
  const uint32_t o = core_off(r, k);
  *reinterpret_cast<float2*>(hi + o) = make_float2(h0, h1);
  *reinterpret_cast<float2*>(lo + o) = make_float2(tf32_rna(v0 - h0), tf32_rna(v1 - h1));
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for the completion of mbarrier phase `parity`: gives up after
// limit_ns of wall time (or TC_WAIT_LIMIT polls)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

__global__ void __launch_bounds__(TC_THREADS) k_tc_update(float2* __restrict__ C, const float2* __restrict__ A,
                                                          const float2* __restrict__ B, int64_t N, int k0, int kw,
                                                          int mode, int kb, int* __restrict__ err, int fault) {
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  // once a wait of this factorisation has run out, later launches do nothing
  // (setup reports DPGMG_ERR_TIMEOUT); the test is uniform over the CTA and
  // comes before any TMEM allocation or barrier
  if (*reinterpret_cast<volatile int*>(err) & 32) return;

  // output tile (same enumeration as the CUDA-core kernels)
  int64_t i0, j0;
  if (mode == TC_HERK) {
    const int64_t k1 = (int64_t)k0 + kw;
    const int64_t t = blockIdx.x;
    int64_t bi = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) / 2.0);
    while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
    while (bi * (bi + 1) / 2 > t) --bi;
    const int64_t bj = t - bi * (bi + 1) / 2;
    i0 = k1 + bi * TC_T;
    j0 = k1 + bj * TC_T;
  } else {
    const int ncol = kb + 1;
    i0 = (int64_t)(kb + 1 + (int)blockIdx.x / ncol) * TC_T;
    j0 = (int64_t)((int)blockIdx.x % ncol) * TC_T;
  }

  const uint32_t raw = (uint32_t)__cvta_generic_to_shared(tc_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  unsigned char* gbase = tc_raw + (sbase - raw);
  const uint32_t sAhi = sbase, sAlo = sbase + TC_A_BYTES, sBhi = sbase + 2 * TC_A_BYTES, sBlo = sBhi + TC_B_BYTES;
  unsigned char* pAhi = gbase;
  unsigned char* pAlo = gbase + TC_A_BYTES;
  unsigned char* pBhi = gbase + 2 * TC_A_BYTES;
  unsigned char* pBlo = pBhi + TC_B_BYTES;
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  // kind::tf32, D in F32, A and B TF32 and K-major, N = 64, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_T >> 3) << 17) | ((128u >> 4) << 24);
  bool ok = true;
  int failed_pass = -1;
  for (int pass = 0; pass < 2 && ok; ++pass) {
    const int t0 = pass * (TC_KP / 2);
    constexpr int PER = TC_T * (TC_KP / 2) / TC_THREADS;   // operand values per thread
    // all global loads first (they are independent), then split and store
    float2 av[PER], bv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int q = tid + u * TC_THREADS;
      const int r = q / (TC_KP / 2), t = q % (TC_KP / 2);
      const int64_t gi = i0 + r;
      av[u] = (gi < N && t0 + t < kw) ? A[gi * N + k0 + t0 + t] : make_float2(0.f, 0.f);
      if (mode == TC_HERK) {
        const int64_t gj = j0 + r;
        bv[u] = (gj < N && t0 + t < kw) ? A[gj * N + k0 + t0 + t] : make_float2(0.f, 0.f);
      } else {
        const int tb = q / TC_T, c = q % TC_T;
        const int64_t gj = j0 + c;
        bv[u] = (gj < N && t0 + tb < kw) ? B[((int64_t)k0 + t0 + tb) * N + gj] : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int q = tid + u * TC_THREADS;
      const int r = q / (TC_KP / 2), t = q % (TC_KP / 2);
      const float2 a = av[u];
      if (mode == TC_HERK) {
        store_split(pAhi, pAlo, r, 2 * t, a.x, a.y);
        store_split(pAhi, pAlo, TC_T + r, 2 * t, a.y, -a.x);
        store_split(pBhi, pBlo, r, 2 * t, bv[u].x, bv[u].y);
      } else {
        store_split(pAhi, pAlo, r, 2 * t, a.x, -a.y);
        store_split(pAhi, pAlo, TC_T + r, 2 * t, a.y, a.x);
        const int tb = q / TC_T, c = q % TC_T;
        store_split(pBhi, pBlo, c, 2 * tb, bv[u].x, bv[u].y);
      }
    }
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0 && !fault) {   // fault (tests): issue nothing, so that the wait below runs out
#pragma unroll 1
      for (int s = 0; s < TC_KP / 8; ++s) {   // K = 8 TF32 values (32 bytes) per instruction
        const uint64_t ah = smem_desc(sAhi + 256u * s), al = smem_desc(sAlo + 256u * s);
        const uint64_t bh = smem_desc(sBhi + 256u * s), bl = smem_desc(sBlo + 256u * s);
        mma_tf32(tmem, ah, bh, idesc, (pass | s) != 0 ? 1u : 0u);
        mma_tf32(tmem, ah, bl, idesc, 1u);
        mma_tf32(tmem, al, bh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                   : "memory");
    }
    // the next pass overwrites the operands, the epilogue reads D: wait for the MMAs
    const bool done = mbar_wait(bar, (uint32_t)(pass & 1), TC_WAIT_NS);
    ok = __syncthreads_and(done) != 0;
    if (!ok) failed_pass = pass;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok && tid == 0) {
    atomicOr(err, 32);
    // MMAs issued in the failed pass may still be running: give them (and
    // their commit to the barrier) a second bounded wait before the
    // accumulator is freed and the CTA's shared memory goes away
    if (!fault) mbar_wait(bar, (uint32_t)(failed_pass & 1), 2 * TC_WAIT_NS);
  }

  float* Ds = reinterpret_cast<float*>(gbase);   // [128][65] staging of D
  if (ok) {
    const int row = warp * 32 + (tid & 31);
#pragma unroll 1
    for (int c0 = 0; c0 < TC_T; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int u = 0; u < 16; ++u) Ds[row * 65 + c0 + u] = __uint_as_float(v[u]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
  if (!ok) return;
  for (int q = tid; q < TC_T * TC_T; q += TC_THREADS) {
    const int r = q / TC_T, c = q % TC_T;
    const int64_t i = i0 + r, j = j0 + c;
    if (i < N && j < N && (mode != TC_HERK || j <= i)) {
      float2 o = C[i * N + j];
      o.x -= Ds[r * 65 + c];
      o.y -= Ds[(TC_T + r) * 65 + c];
      C[i * N + j] = o;
    }
  }
}

}  // namespace

void tc_configure() {
  DPG_CUDA(cudaFuncSetAttribute(k_tc_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
}

// Trailing update of the blocked Cholesky after panel k0 (width kw <= 64):
// every lower 64 x 64 tile of A[k0+kw:, k0+kw:].
// fault != 0 (tests): the launch issues no MMA, so its bounded waits run out.
void tc_herk_update(float2* A, int64_t N, int k0, int kw, int* err, int fault, cudaStream_t st) {
  const int64_t rows = N - k0 - kw;
  if (rows <= 0) return;
  const int64_t nt = (rows + TC_T - 1) / TC_T;
  k_tc_update<<<(unsigned)(nt * (nt + 1) / 2), TC_THREADS, TC_SMEM, st>>>(A, A, A, N, k0, kw, TC_HERK, 0, err,
                                                                          fault);
  DPG_CHECK_LAUNCH();
}

// Blocked L^-1 update for block column kb: X[ib][jb] -= L[ib][kb] X[kb][jb]
// for ib > kb, jb <= kb (64 x 64 tiles).
void tc_trinv_update(float2* X, const float2* L, int64_t N, int kb, int* err, cudaStream_t st) {
  const int nb = (int)((N + TC_T - 1) / TC_T);
  const int rows = nb - kb - 1;
  if (rows <= 0) return;
  const int k0 = kb * TC_T;
  const int kw = (int)(N - k0 < TC_T ? N - k0 : TC_T);
  k_tc_update<<<(unsigned)(rows * (kb + 1)), TC_THREADS, TC_SMEM, st>>>(X, L, X, N, k0, kw, TC_GEMM, kb, err, 0);
  DPG_CHECK_LAUNCH();
}

}  // namespace dpgmg
