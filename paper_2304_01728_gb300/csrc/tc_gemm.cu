// Complex64 matrix products on the tensor cores (tcgen05, TF32 operands from
// shared memory, FP32 accumulator in TMEM), used by the mixed path's coarsest
// factorisation (Sec. 4 list: direct solve on the initial mesh) for its
// panel solves, trailing updates and triangular-inverse updates:
//
//   C = beta C + alpha op(A) op(B),   op(A) = A (rows i, columns k),
//   op(B) = B (rows k, columns j) or B^H (rows j, columns k, conjugated),
//
// complex64 in global memory, row-major.  alpha is +-1, beta 0 or 1.
//
// Real form.  A complex product is one real contraction over interleaved
// (re, im) pairs: with b' = (Re b, Im b) per output column j,
//   C = A B^H   Re = <(ar, ai), b'>    Im = <(ai, -ar), b'>
//   C = A B     Re = <(ar, -ai), b'>   Im = <(ai, ar), b'>
// so a tile of 64 complex output rows is one 128-row real tile: D rows
// 0..63 hold real parts, rows 64..127 imaginary parts (MMA M = 128), over 128
// complex output columns (MMA N = 128).
//
// Precision (3xTF32).  Every FP32 operand value x is split into TF32 parts
// x1 = rna(x), x2 = rna(x - x1), and D accumulates a1 b1 + a1 b2 + a2 b1
// (the a2 b2 term is below FP32 rounding).  The tensor cores' FP32
// accumulation does not round to nearest: accumulated over a whole panel in
// TMEM, its bias put the 16^3 p=3 solution 2.4e-7 from the FP64 oracle's
// (with three parts and six products just the same).  Each stage of 8
// complex K values therefore accumulates into a fresh TMEM buffer that the
// epilogue warps add, rounding to nearest, into FP32 registers; the coarse
// solve is then within 1.4x of the FP32 CUDA-core factor's accuracy.
//
// Operand images.  A pack kernel writes each operand once per product into
// global memory already in the shared-memory image the MMA reads: per tile
// (64 complex rows of A as 128 real rows, or 128 complex rows of B) and per
// stage of 8 complex K values (16 TF32 values), two 8 KiB images (one per
// TF32 part) in the canonical K-major layout without swizzle (8-row x 16-byte
// core matrices, adjacent along K at 128 B, along M/N at 512 B).  The product
// kernel streams a stage of A and of B (2 x 16 KiB) into shared memory with
// two bulk asynchronous copies (cp.async.bulk, completion counted on an
// mbarrier) through a 6-stage ring, so the copies of later stages overlap the
// MMAs of the current one; one thread issues copies and MMAs, tcgen05.commit
// frees a stage, and the four warps then move D from TMEM to global memory.
// Every wait is bounded in wall time; a wait that runs out sets an error bit,
// lets the copies and MMAs already issued land (a second bounded wait), frees
// the accumulator and returns.
#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace dpgmg {

namespace {

constexpr int TG_MR = 64;                          // complex output rows per tile (MMA M = 128)
constexpr int TG_NC = 128;                         // complex output columns per tile (MMA N)
constexpr int TG_KC = 8;                           // complex K per stage
constexpr int TG_KR = 2 * TG_KC;                   // TF32 values per image row per stage
constexpr int TG_PARTS = 2;                        // TF32 parts per FP32 value
constexpr uint32_t TG_IMG = 128u * TG_KR * 4u;     // 8 KiB: one TF32 part of one tile stage
constexpr uint32_t TG_PAIR = TG_PARTS * TG_IMG;    // all parts of one operand tile stage
constexpr uint32_t TG_STAGE = 2u * TG_PAIR;        // A and B
constexpr int TG_NS = 6;                           // stages in flight
constexpr uint32_t TG_SMEM = TG_NS * TG_STAGE + 1024u;
constexpr int TG_THREADS = 160;                    // warps 0-3 drain TMEM, warp 4 issues
constexpr long long TG_WAIT_POLLS = 1LL << 24;
constexpr unsigned long long TG_WAIT_NS = 500000000ull;   // 0.5 s

enum PackMode { PACK_A_NH = 0, PACK_A_NN = 1, PACK_B = 2, PACK_B_TRANS = 3 };

// byte offset of (row r, K index k) in a stage image
__device__ __forceinline__ uint32_t img_off(int r, int k) {
  return (uint32_t)(((r >> 3) * (TG_KR / 4) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// (v.x, v.y) as TF32 parts, at byte offset o of each part image
__device__ __forceinline__ void store_parts(unsigned char* part, uint32_t o, float2 v) {
  float rx = v.x, ry = v.y;
#pragma unroll
  for (int q = 0; q < TG_PARTS; ++q) {
    const float hx = tf32_rna(rx), hy = tf32_rna(ry);
    *reinterpret_cast<float2*>(part + q * TG_IMG + o) = make_float2(hx, hy);
    rx -= hx;   // exact: hx holds the leading bits of rx
    ry -= hy;
  }
}

// One CTA per (tile, stage): the part images of that tile stage.
//   PACK_A_NH / PACK_A_NN: tile t = logical rows 64t..64t+63 of A; image rows
//     0..63 carry the real-part variant of each row, 64..127 the imaginary-part
//     variant (for op(B) = B^H or B, see above);
//   PACK_B: tile t = logical rows 128t.. of B' (the rows of B for op(B) = B^H);
//   PACK_B_TRANS: logical row j of B' = column j of B (op(B) = B), read with
//     consecutive threads on consecutive j.
// Logical entry (row, k) is src[row * ld + k] (src[k * ld + row] for
// PACK_B_TRANS); rows >= nrows and k >= kc are zero.
__global__ void __launch_bounds__(256) k_tc_pack(float* __restrict__ img, const float2* __restrict__ src,
                                                 int64_t ld, int64_t nrows, int64_t kc, int nst, int mode) {
  const int64_t t = blockIdx.x;
  const int s = blockIdx.y;
  unsigned char* part = reinterpret_cast<unsigned char*>(img) + ((size_t)t * nst + s) * TG_PAIR;
  const int64_t k0 = (int64_t)s * TG_KC;
  const bool is_a = mode == PACK_A_NH || mode == PACK_A_NN;
  const int rows = is_a ? TG_MR : 128;
  for (int q = threadIdx.x; q < rows * TG_KC; q += blockDim.x) {
    int r, kk;
    if (mode == PACK_B_TRANS) {   // consecutive threads: consecutive logical rows (source columns)
      r = q % rows;
      kk = q / rows;
    } else {                      // consecutive threads: consecutive k of one row
      r = q / TG_KC;
      kk = q % TG_KC;
    }
    const int64_t row = t * rows + r, k = k0 + kk;
    float2 v = make_float2(0.f, 0.f);
    if (row < nrows && k < kc) v = mode == PACK_B_TRANS ? src[k * ld + row] : src[row * ld + k];
    float2 p0, p1;   // values of image row r (and r + 64 for A) at K indices 2kk, 2kk + 1
    if (mode == PACK_A_NH) {
      p0 = make_float2(v.x, v.y);
      p1 = make_float2(v.y, -v.x);
    } else if (mode == PACK_A_NN) {
      p0 = make_float2(v.x, -v.y);
      p1 = make_float2(v.y, v.x);
    } else {
      p0 = v;
      p1 = v;
    }
    store_parts(part, img_off(r, 2 * kk), p0);
    if (is_a) store_parts(part, img_off(r + TG_MR, 2 * kk), p1);
  }
}

// shared-memory matrix descriptor: start >> 4, leading byte offset 128,
// stride byte offset (K / 4) x 128 B, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(((uint32_t)(TG_KR / 4) * 128u) >> 4) << 32) | (1ull << 46);
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
// limit_ns of wall time, TG_WAIT_POLLS polls, or once another CTA of the
// factorisation has reported a wait that ran out (err bit 32)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns,
                                          const int* err) {
  const unsigned long long t0 = global_ns();
  for (long long it = 0; it < TG_WAIT_POLLS; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63) {
      if (global_ns() - t0 > limit_ns) return false;
      if (err && (*reinterpret_cast<const volatile int*>(err) & 32)) return false;
    }
  }
  return false;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One CTA per (64-row, 128-column) complex output tile; tiles of the strict
// upper triangle are skipped when `lower` (C Hermitian, lower half stored).
// Warp 4 (one thread) streams the operand stages and issues the MMAs; each
// stage accumulates into a fresh TMEM buffer (two, used in turn), which warps
// 0-3 (one TMEM lane = one real output row each) drain into FP32 registers
// with round-to-nearest additions while the next stage's MMAs run.  The
// tensor cores' FP32 accumulation does not round to nearest; keeping its
// chains one stage long (2 K steps x 3 products) keeps the products as
// accurate as the CUDA cores' FMA chains.
// fault (tests): no MMA and no commit are issued, so the waits for them run out.
__global__ void __launch_bounds__(TG_THREADS) k_tc_gemm(const unsigned char* __restrict__ Aimg,
                                                        const unsigned char* __restrict__ Bimg, int64_t M, int64_t N,
                                                        int nst, float2* __restrict__ C, int64_t ldc, float alpha,
                                                        float beta, int lower, int* __restrict__ err, int fault) {
  extern __shared__ unsigned char tg_raw[];
  __shared__ __align__(8) uint64_t bar_full[TG_NS];
  __shared__ __align__(8) uint64_t bar_empty[TG_NS];
  __shared__ __align__(8) uint64_t bar_acc[2];      // MMAs of a stage done: its TMEM buffer is ready
  __shared__ __align__(8) uint64_t bar_drained[2];  // warps 0-3 have read the buffer
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntn = (N + TG_NC - 1) / TG_NC;
  const int64_t mt = blockIdx.x / ntn, nt = blockIdx.x % ntn;
  const int64_t r0 = mt * TG_MR, c0 = nt * TG_NC;
  if (lower && c0 > r0 + TG_MR - 1) return;                      // uniform over the CTA
  if (*reinterpret_cast<volatile int*>(err) & 32) return;        // an earlier wait ran out

  const uint32_t raw = (uint32_t)__cvta_generic_to_shared(tg_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  float* Ds = reinterpret_cast<float*>(tg_raw + (sbase - raw));   // epilogue staging, after the main loop
  auto sa = [](const void* p) { return (uint32_t)__cvta_generic_to_shared(p); };
  if (tid == 0) {
    for (int s = 0; s < TG_NS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bar_full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bar_empty[s])) : "memory");
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bar_acc[b])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(sa(&bar_drained[b])) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(sa(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  float acc[TG_NC];
#pragma unroll
  for (int c = 0; c < TG_NC; ++c) acc[c] = 0.f;

  if (warp == 4) {
    if (lane == 0) {
      // kind::tf32, D in F32, A and B TF32 and K-major, N = 128, M = 128
      const uint32_t idesc =
          (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TG_NC >> 3) << 17) | ((128u >> 4) << 24);
      const unsigned char* Ab = Aimg + (size_t)mt * nst * TG_PAIR;
      const unsigned char* Bb = Bimg + (size_t)nt * nst * TG_PAIR;
      auto load = [&](int ks) {
        const int s = ks % TG_NS;
        const uint32_t a = sbase + (uint32_t)s * TG_STAGE;
        mbar_expect(sa(&bar_full[s]), TG_STAGE);
        bulk_load(a, Ab + (size_t)ks * TG_PAIR, TG_PAIR, sa(&bar_full[s]));
        bulk_load(a + TG_PAIR, Bb + (size_t)ks * TG_PAIR, TG_PAIR, sa(&bar_full[s]));
      };
      bool ok = true;
      int loads = 0, landed = 0, commits = 0;
      for (; loads < nst && loads < TG_NS; ++loads) load(loads);
      for (int ks = 0; ks < nst && ok; ++ks) {
        const int s = ks % TG_NS, b = ks & 1;
        if (!mbar_wait(sa(&bar_full[s]), (uint32_t)((ks / TG_NS) & 1), TG_WAIT_NS, err)) {
          ok = false;
          break;
        }
        ++landed;
        // the buffer of stage ks - 2 must have been drained
        if (ks >= 2 && !mbar_wait(sa(&bar_drained[b]), (uint32_t)(((ks - 2) / 2) & 1), TG_WAIT_NS, err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!fault) {
          const uint32_t a = sbase + (uint32_t)s * TG_STAGE, bo = a + TG_PAIR;
          const uint32_t d = tmem + (uint32_t)(b * TG_NC);
          // (part of A, part of B) of the three products, small ones first
          constexpr int PA[3] = {1, 0, 0}, PB[3] = {0, 1, 0};
#pragma unroll
          for (int j = 0; j < TG_KR / 8; ++j) {   // K = 8 TF32 values (32 bytes) per instruction
            const uint32_t o = 256u * j;
#pragma unroll
            for (int q = 0; q < 3; ++q)
              mma_tf32(d, smem_desc(a + PA[q] * TG_IMG + o), smem_desc(bo + PB[q] * TG_IMG + o), idesc,
                       (j | q) != 0 ? 1u : 0u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           sa(&bar_empty[s]))
                       : "memory");
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           sa(&bar_acc[b]))
                       : "memory");
          ++commits;
        }
        // refill the stage read by the previous step once its MMAs are done
        if (ks >= 1 && loads < nst) {
          const int ps = (ks - 1) % TG_NS;
          if (!mbar_wait(sa(&bar_empty[ps]), (uint32_t)(((ks - 1) / TG_NS) & 1), TG_WAIT_NS, err)) {
            ok = false;
            break;
          }
          load(loads++);
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(err, 32);
        // let the copies and MMAs already issued land before the shared memory
        // and the accumulators are released
        for (int q = landed; q < loads; ++q)
          mbar_wait(sa(&bar_full[q % TG_NS]), (uint32_t)((q / TG_NS) & 1), 2 * TG_WAIT_NS, nullptr);
        if (commits > 0) {
          const int q = commits - 1;
          mbar_wait(sa(&bar_acc[q & 1]), (uint32_t)((q / 2) & 1), 2 * TG_WAIT_NS, nullptr);
        }
      }
    }
  } else {
    // warps 0-3: drain each stage's buffer into the FP32 accumulators of this lane's row
    for (int ks = 0; ks < nst; ++ks) {
      const int b = ks & 1;
      int ready = 0;
      if (lane == 0) {
        const unsigned long long t0 = global_ns();
        for (long long it = 0; it < TG_WAIT_POLLS; ++it) {
          uint32_t done;
          asm volatile(
              "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
              "selp.u32 %0, 1, 0, p;\n\t}\n"
              : "=r"(done)
              : "r"(sa(&bar_acc[b])), "r"((uint32_t)((ks / 2) & 1))
              : "memory");
          if (done) {
            ready = 1;
            break;
          }
          if ((it & 63) == 63 && (s_abort || global_ns() - t0 > 4 * TG_WAIT_NS)) break;
        }
      }
      ready = __shfl_sync(0xffffffffu, ready, 0);
      if (!ready) break;   // the issuer aborted (or never committed): nothing more to drain
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int cc = 0; cc < TG_NC; cc += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * TG_NC + cc);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[cc + u] += __uint_as_float(v[u]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(&bar_drained[b])) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
  if (s_abort) return;
  constexpr int DP = TG_NC + 1;   // staging pitch (floats): lanes of a warp hit distinct banks
  if (warp < 4) {
    const int row = warp * 32 + lane;
#pragma unroll
    for (int c = 0; c < TG_NC; ++c) Ds[row * DP + c] = acc[c];
  }
  __syncthreads();
  for (int q = tid; q < TG_MR * TG_NC; q += TG_THREADS) {
    const int i = q / TG_NC, j = q % TG_NC;
    const int64_t gi = r0 + i, gj = c0 + j;
    if (gi >= M || gj >= N || (lower && gj > gi)) continue;
    float2* o = C + gi * ldc + gj;
    float2 v = make_float2(alpha * Ds[i * DP + j], alpha * Ds[(TG_MR + i) * DP + j]);
    if (beta != 0.f) {
      const float2 c = *o;
      v.x += beta * c.x;
      v.y += beta * c.y;
    }
    *o = v;
  }
}

int stages_of(int64_t kc) { return (int)((kc + TG_KC - 1) / TG_KC); }

}  // namespace

void tc_configure() {
  DPG_CUDA(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM));
}

// bytes of the operand image of `rows` logical rows and kc complex K values
size_t tc_image_bytes(int64_t rows, int64_t kc, bool is_a) {
  const int64_t tiles = (rows + (is_a ? TG_MR : 128) - 1) / (is_a ? TG_MR : 128);
  return (size_t)std::max<int64_t>(tiles, 1) * (size_t)std::max(stages_of(kc), 1) * TG_PAIR;
}

// mode: 0 = A for op(B) = B^H, 1 = A for op(B) = B, 2 = B rows (op(B) = B^H),
// 3 = B columns (op(B) = B, src read transposed)
void tc_pack(void* img, const float2* src, int64_t ld, int64_t rows, int64_t kc, int mode, cudaStream_t st) {
  if (rows <= 0 || kc <= 0) return;
  const bool is_a = mode == PACK_A_NH || mode == PACK_A_NN;
  const int64_t tiles = (rows + (is_a ? TG_MR : 128) - 1) / (is_a ? TG_MR : 128);
  const int nst = stages_of(kc);
  k_tc_pack<<<dim3((unsigned)tiles, (unsigned)nst), 256, 0, st>>>(reinterpret_cast<float*>(img), src, ld, rows, kc,
                                                                 nst, mode);
  DPG_CHECK_LAUNCH();
}

// C (M x N, leading dimension ldc) = beta C + alpha op(A) op(B) from images
// packed with the same kc; lower: only entries j <= i are written.
void tc_gemm(const void* Aimg, const void* Bimg, int64_t M, int64_t N, int64_t kc, float2* C, int64_t ldc,
             float alpha, float beta, int lower, int* err, int fault, cudaStream_t st) {
  if (M <= 0 || N <= 0 || kc <= 0) return;
  const int64_t tiles = ((M + TG_MR - 1) / TG_MR) * ((N + TG_NC - 1) / TG_NC);
  k_tc_gemm<<<(unsigned)tiles, TG_THREADS, TG_SMEM, st>>>(reinterpret_cast<const unsigned char*>(Aimg),
                                                        reinterpret_cast<const unsigned char*>(Bimg), M, N,
                                                        stages_of(kc), C, ldc, alpha, beta, lower, err, fault);
  DPG_CHECK_LAUNCH();
}

}  // namespace dpgmg
