// Additive Schwarz smoother kernels (Sec. 3, "V-cycle and smoother"):
//   y = theta * sum_j R_j^T A_jj^-1 R_j r
// over the vertex patches of a level.  A_jj^-1 is Hermitian.
//
// Full storage (n_j x n_j blocks, rows padded to even length): one CTA per
// chunk of 32 (complex128) or 64 (complex64) columns of a patch; warp w reads
// rows k = w, w + 8, ... (coalesced), the 8 warp partials are summed in shared
// memory; y_a = sum_k conj(M[k][a]) r_k.  The chunk lists are ordered by
// decreasing patch size so that the small boundary patches fill the last wave.
//
// Half storage (lower triangle packed by rows, n_j (n_j + 1) / 2 entries):
// every stored entry is read once and used twice (row sum and mirrored
// column sum), see k_patch_apply_h.  Used for complex64 operators; patches
// up to HALF_MAX_N DOFs (the shared-memory buffers scale with n_j).
#pragma once
#include <type_traits>
#include "common.cuh"
#include "host_mesh.h"
#include "internal.h"

namespace dpgmg {

constexpr int HALF_MAX_N = 1024;

template <class C> __device__ __forceinline__ C warp_sum_s(C v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// v * i^s for s in {-1, 0, 1}: a swap of the components and one sign, exact
template <class C>
__device__ __forceinline__ C mul_i(C v, int s) {
  return s == 0 ? v : (s > 0 ? Ops<C>::mk(-v.y, v.x) : Ops<C>::mk(v.y, -v.x));
}

// conversions between the operator precision C and the vectors' type
template <class C, class V> __device__ __forceinline__ C cvt_in(V v) {
  return Ops<C>::mk((typename Ops<C>::R)v.x, (typename Ops<C>::R)v.y);
}

// patch inverses are read once per application: streaming loads (evict first)
template <class C> __device__ __forceinline__ C ld_stream(const C* p) { return __ldcs(p); }

// 16-byte asynchronous global -> shared copies (cp.async, L2 only); each thread
// later reads back only what it copied itself, after waiting on its own groups.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// acc + w r for a real w: two real FMAs instead of a complex product
template <class C>
__device__ __forceinline__ C rfma(typename Ops<C>::R w, C r, C acc) {
  if constexpr (std::is_same<C, float2>::value) return make_float2(fmaf(w, r.x, acc.x), fmaf(w, r.y, acc.y));
  else return Ops<C>::mk(::fma(w, r.x, acc.x), ::fma(w, r.y, acc.y));
}

// The work item (patch with a real packed block, first column a0, 32 PER
// columns) of k_patch_apply.  Rows have ldr = patch_ldr(n) reals (Wb = row 0);
// a lane reads 4 columns with one 16-byte copy, 8 PER lanes cover a row and a
// warp 4 / PER rows at a time (warp w: rows w 4/PER + lane / (8 PER) + 32 i).
// Each thread streams its rows through a shared-memory ring of REAL_RING
// cp.async copies, the first of them issued before the right-hand-side
// gather, so that the gather's dependent loads overlap the stream and the
// rows in flight hold no registers.  Then: shuffles combine the lanes that
// share columns, the 8 warp partials are summed in a fixed order, and the
// output phase is applied.  The start of the patch's slots passes through
// shared memory (sb), so no 64-bit value stays live across the stream.
constexpr int REAL_RING = 5;

template <class TIN, int PER>
__device__ __forceinline__ void patch_apply_real(const int32_t* __restrict__ dofs, const float* __restrict__ Wb,
                                                 const TIN* __restrict__ r, float2* __restrict__ pbuf, int64_t b,
                                                 int n, int a0, int64_t offU, float2* rj,
                                                 float2 (*part)[32 * PER + 1], int64_t* sb) {
  constexpr int LPR = 8 * PER, RPI = 4 / PER, STEP = 8 * RPI;
  __shared__ float4 ring[REAL_RING][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cg = lane % LPR, ro = lane / LPR;
  const int a = a0 + 4 * cg;   // columns a .. a + 3 lie within the padded row when a < n
  const bool act = a < n;
  const float4* W4 = reinterpret_cast<const float4*>(Wb + a);
  const int s4 = (int)(patch_ldr(n) / 4), ds = STEP * s4;   // offsets below n ldr / 4 < 2^31
  const int k0 = w * RPI + ro;
#pragma unroll
  for (int d = 0; d < REAL_RING; ++d) {
    if (act && k0 + d * STEP < n) cp_async16(&ring[d][threadIdx.x], W4 + (k0 * s4 + d * ds));
    cp_async_commit();
  }
  if (threadIdx.x == 0) *sb = b;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int32_t g = dofs[b + q];
    rj[q] = mul_i(cvt_in<float2>(r[g]), g < offU ? -1 : 0);
  }
  __syncthreads();
  float2 acc[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.f, 0.f);
  if (act) {
    const int nr = k0 < n ? (n - k0 + STEP - 1) / STEP : 0;   // this thread's rows
    const float4* src = W4 + (k0 * s4 + REAL_RING * ds);      // the next row to copy
    const float2* rp = rj + k0;
    int d = 0;
    for (int i = 0; i < nr; ++i, rp += STEP, src += ds) {
      cp_async_wait<REAL_RING - 1>();   // this thread's oldest copy (its row i) has landed
      const float4 m0 = ring[d][threadIdx.x];
      const float2 rv = *rp;
      acc[0] = rfma<float2>(m0.x, rv, acc[0]);
      acc[1] = rfma<float2>(m0.y, rv, acc[1]);
      acc[2] = rfma<float2>(m0.z, rv, acc[2]);
      acc[3] = rfma<float2>(m0.w, rv, acc[3]);
      // refill the slot with row i + REAL_RING (m0 has been read above)
      if (i + REAL_RING < nr) cp_async16(&ring[d][threadIdx.x], src);
      cp_async_commit();
      d = d + 1 == REAL_RING ? 0 : d + 1;
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, o);
      acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, o);
    }
  if (ro == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) part[w][4 * cg + c] = acc[c];
  __syncthreads();
  if (w == 0) {
    const int64_t b2 = *sb;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int c = a0 + PER * lane + u;
      if (c < n) {
        float2 s2 = part[0][PER * lane + u];
#pragma unroll
        for (int q = 1; q < 8; ++q) s2 = Ops<float2>::add(s2, part[q][PER * lane + u]);
        pbuf[b2 + c] = mul_i(s2, dofs[b2 + c] < offU ? 1 : 0);
      }
    }
  }
}

// Rows of a stored block have length ld = patch_ld(n) (even).  Work item
// (patch j, first column a0) of COLS columns; lane `lane` of warp w handles
// columns a0 + PER * lane .. + PER - 1 (PER = 1 for complex128, 2 for
// complex64: one 16-byte load per row), warps split the rows k = w, w + 8, ...
template <class C> struct PatchCols { static constexpr int per = 1; };
template <> struct PatchCols<float2> { static constexpr int per = 2; };

// A patch with rflag[j] set holds a real packed block w (A^-1[k][a] =
// w[k][a] i^(s_k - s_a), s = 1 on p-hat DOFs, global index < offU):
//   y_a = sum_k conj(A^-1[k][a]) r_k = i^(s_a) sum_k w[k][a] (i^(-s_k) r_k),
// so the gathered r carries the phase i^(-s_k), the sum is real-times-complex
// and the output the phase i^(s_a); all three phase steps are exact.
template <class C, class TIN, int PER = PatchCols<C>::per, int MINB = (PER == 2 ? 8 : 3)>
__global__ void __launch_bounds__(256, MINB) k_patch_apply(const int64_t* __restrict__ ptr, const int32_t* __restrict__ dofs,
                                                     const int64_t* __restrict__ vptr, const int2* __restrict__ chunks,
                                                     const C* __restrict__ inv, const TIN* __restrict__ r,
                                                     C* __restrict__ pbuf, const uint8_t* __restrict__ rflag,
                                                     int64_t offU) {
  extern __shared__ unsigned char shraw[];
  __shared__ C part[8][32 * PER + 1];
  C* rj = reinterpret_cast<C*>(shraw);
  using O = Ops<C>;
  const int2 ch = chunks[blockIdx.x];
  const int64_t j = ch.x;
  const int64_t b = ptr[j];
  const int n = (int)(ptr[j + 1] - b);
  if constexpr (std::is_same<C, float2>::value) {   // only complex64 inverses are packed
    if (rflag != nullptr && rflag[j] != 0) {         // uniform over the CTA
      __shared__ int64_t sb;
      patch_apply_real<TIN, PER>(dofs, reinterpret_cast<const float*>(inv + vptr[j]), r, pbuf, b, n, ch.y, offU, rj,
                                 part, &sb);
      return;
    }
  }
  const int64_t ld = patch_ld(n);
  for (int q = threadIdx.x; q < n; q += blockDim.x) rj[q] = cvt_in<C>(r[dofs[b + q]]);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int a = ch.y + PER * lane;
  C acc[PER][2];
#pragma unroll
  for (int u = 0; u < PER; ++u) acc[u][0] = acc[u][1] = O::zero();
  if (a < n) {
    const C* M = inv + vptr[j] + a;
    int k = w;
    if (PER == 2) {
      // 16-byte loads of (M[k][a], M[k][a+1]); a is even and ld even, so aligned
      const float4* M4 = reinterpret_cast<const float4*>(M);
      const int64_t s4 = ld / 2;
      for (; k + 24 < n; k += 32) {
        const float4 m0 = __ldcs(M4 + (int64_t)k * s4), m1 = __ldcs(M4 + (int64_t)(k + 8) * s4);
        const float4 m2 = __ldcs(M4 + (int64_t)(k + 16) * s4), m3 = __ldcs(M4 + (int64_t)(k + 24) * s4);
        const C r0 = rj[k], r1 = rj[k + 8], r2 = rj[k + 16], r3 = rj[k + 24];
        acc[0][0] = O::fmac(r0, Ops<C>::mk(m0.x, m0.y), acc[0][0]);
        acc[1 % PER][0] = O::fmac(r0, Ops<C>::mk(m0.z, m0.w), acc[1 % PER][0]);
        acc[0][1] = O::fmac(r1, Ops<C>::mk(m1.x, m1.y), acc[0][1]);
        acc[1 % PER][1] = O::fmac(r1, Ops<C>::mk(m1.z, m1.w), acc[1 % PER][1]);
        acc[0][0] = O::fmac(r2, Ops<C>::mk(m2.x, m2.y), acc[0][0]);
        acc[1 % PER][0] = O::fmac(r2, Ops<C>::mk(m2.z, m2.w), acc[1 % PER][0]);
        acc[0][1] = O::fmac(r3, Ops<C>::mk(m3.x, m3.y), acc[0][1]);
        acc[1 % PER][1] = O::fmac(r3, Ops<C>::mk(m3.z, m3.w), acc[1 % PER][1]);
      }
      for (; k < n; k += 8) {
        const float4 m0 = __ldcs(M4 + (int64_t)k * s4);
        acc[0][0] = O::fmac(rj[k], Ops<C>::mk(m0.x, m0.y), acc[0][0]);
        acc[1 % PER][0] = O::fmac(rj[k], Ops<C>::mk(m0.z, m0.w), acc[1 % PER][0]);
      }
    } else {
      C a2 = O::zero(), a3 = O::zero();
      for (; k + 24 < n; k += 32) {
        const C m0 = ld_stream(M + (size_t)k * ld), m1 = ld_stream(M + (size_t)(k + 8) * ld);
        const C m2 = ld_stream(M + (size_t)(k + 16) * ld), m3 = ld_stream(M + (size_t)(k + 24) * ld);
        acc[0][0] = O::fmac(rj[k], m0, acc[0][0]);
        acc[0][1] = O::fmac(rj[k + 8], m1, acc[0][1]);
        a2 = O::fmac(rj[k + 16], m2, a2);
        a3 = O::fmac(rj[k + 24], m3, a3);
      }
      for (; k < n; k += 8) acc[0][0] = O::fmac(rj[k], ld_stream(M + (size_t)k * ld), acc[0][0]);
      acc[0][0] = O::add(acc[0][0], a2);
      acc[0][1] = O::add(acc[0][1], a3);
    }
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) part[w][PER * lane + u] = O::add(acc[u][0], acc[u][1]);
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int c = ch.y + PER * lane + u;
      if (c < n) {
        C s2 = part[0][PER * lane + u];
#pragma unroll
        for (int q = 1; q < 8; ++q) s2 = O::add(s2, part[q][PER * lane + u]);
        pbuf[b + c] = s2;
      }
    }
  }
}

// work items of k_patch_apply with PER columns per lane: 32 * PER columns
inline const int2* patch_chunks(const PatchDev& P, int per, int64_t* n) {
  *n = per == 2 ? P.nchunks64 : P.nchunks;
  return per == 2 ? P.chunks64 : P.chunks;
}

// Variants of the complex64 smoother product, tuned per level at setup:
// 1 = one column per lane (32-column work items), 2 = two columns per lane
// (64-column work items, 8 CTAs per SM, 32 registers), 3 = two columns per
// lane at 6 CTAs per SM (40 registers: the real packed path then keeps its
// loads in registers).
constexpr int SMOOTH_PER2_WIDE = 3;

template <class TIN>
inline void launch_patch_apply_c64(const PatchDev& P, int variant, const float2* inv, const TIN* r, float2* pbuf,
                                   cudaStream_t st) {
  const size_t sm = (size_t)P.max_n * sizeof(float2) + 16;
  int64_t nch = 0;
  const int2* chunks = patch_chunks(P, variant == 1 ? 1 : 2, &nch);
  if (variant == SMOOTH_PER2_WIDE)
    k_patch_apply<float2, TIN, 2, 6><<<(unsigned)nch, 256, sm, st>>>(P.ptr, P.dofs, P.val_ptr, chunks, inv, r, pbuf,
                                                                     P.rflag, P.offU);
  else if (variant == 2)
    k_patch_apply<float2, TIN, 2><<<(unsigned)nch, 256, sm, st>>>(P.ptr, P.dofs, P.val_ptr, chunks, inv, r, pbuf,
                                                                  P.rflag, P.offU);
  else
    k_patch_apply<float2, TIN, 1><<<(unsigned)nch, 256, sm, st>>>(P.ptr, P.dofs, P.val_ptr, chunks, inv, r, pbuf,
                                                                  P.rflag, P.offU);
  DPG_CHECK_LAUNCH();
}

// y[g] = (accumulate ? y[g] : 0) + theta * sum_{slots of g} pbuf[slot]
template <class C, class TOUT>
__global__ void k_slot_sum(const int64_t* __restrict__ sptr, const int32_t* __restrict__ slots,
                           const C* __restrict__ pbuf, TOUT* __restrict__ y, int64_t n, double theta, int accumulate) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  C acc = Ops<C>::zero();
  for (int64_t s = sptr[g]; s < sptr[g + 1]; ++s) acc = Ops<C>::add(acc, pbuf[slots[s]]);
  acc = Ops<C>::scale(acc, (typename Ops<C>::R)theta);
  TOUT o = cvt_in<TOUT>(acc);
  y[g] = accumulate ? Ops<TOUT>::add(y[g], o) : o;
}

// ---------------------------------------------------------------- half storage
// One CTA per patch.  The packed lower triangle is cut into 32 x 32 tiles
// (I, K), K <= I; warp w takes tiles w, w + 8, ... of the list.  A tile is
// loaded with 32 coalesced row-segment loads (lane k holds column 32K + k of
// the tile's 32 rows), then
//   columns: lane k adds sum_r conj(T[r][k]) r_{32I+r} to y_{32K+k}
//            (strictly below the diagonal);
//   rows:    the 32 products T[r][k] r_{32K+k} are summed over the lanes by a
//            recursive-halving transpose-reduce (31 shuffles), after which
//            lane r holds the tile's contribution to y_{32I+r}.
// Contributions go to the warp's own shared buffer; the 8 buffers are summed
// in a fixed order, so the result is deterministic.
template <class C, class TIN>
__global__ void __launch_bounds__(256) k_patch_apply_h(const int64_t* __restrict__ ptr, const int32_t* __restrict__ dofs,
                                                       const int64_t* __restrict__ hptr, const C* __restrict__ H,
                                                       const TIN* __restrict__ r, C* __restrict__ pbuf) {
  extern __shared__ unsigned char shraw[];
  using O = Ops<C>;
  const int64_t j = blockIdx.x;
  const int64_t b = ptr[j];
  const int n = (int)(ptr[j + 1] - b);
  C* rj = reinterpret_cast<C*>(shraw);   // [n]
  C* wb = rj + n;                        // [8][n]
  for (int q = threadIdx.x; q < n; q += blockDim.x) rj[q] = cvt_in<C>(r[dofs[b + q]]);
  for (int q = threadIdx.x; q < 8 * n; q += blockDim.x) wb[q] = O::zero();
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  C* my = wb + w * n;
  const C* Hj = H + hptr[j];
  const int T = (n + 31) >> 5;
  const int ntiles = T * (T + 1) / 2;
  for (int t = w; t < ntiles; t += 8) {
    int I = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    const int K = t - I * (I + 1) / 2;
    const int k = 32 * K + lane;
    C v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int a = 32 * I + q;
      v[q] = (a < n && k <= a) ? Hj[(int64_t)a * (a + 1) / 2 + k] : O::zero();
    }
    // mirrored upper triangle: y_k += sum_r conj(M[a][k]) r_a, a = 32I + r > k
    C cacc = O::zero();
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (32 * I + q > k) cacc = O::fmac(rj[min(32 * I + q, n - 1)], v[q], cacc);
    if (k < n) my[k] = O::add(my[k], cacc);
    // row sums: v[q] <- M[a][k] r_k, then transpose-reduce over the lanes
    const C rk = (k < n) ? rj[k] : O::zero();
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = O::mul(v[q], rk);
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      const bool up = (lane & s) != 0;
#pragma unroll
      for (int i = 0; i < s; ++i) {
        const C send = up ? v[i] : v[i + s];
        C recv;
        recv.x = __shfl_xor_sync(0xffffffffu, send.x, s);
        recv.y = __shfl_xor_sync(0xffffffffu, send.y, s);
        v[i] = O::add(up ? v[i + s] : v[i], recv);
      }
    }
    const int a = 32 * I + lane;
    __syncwarp();
    if (a < n) my[a] = O::add(my[a], v[0]);
    __syncwarp();
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    C s = wb[q];
#pragma unroll
    for (int ww = 1; ww < 8; ++ww) s = O::add(s, wb[ww * n + q]);
    pbuf[b + q] = s;
  }
}

// packs the lower triangle of every full block into half storage
template <class CF, class CH>
__global__ void k_pack_half(const int64_t* __restrict__ ptr, const int64_t* __restrict__ vptr,
                            const int64_t* __restrict__ hptr, const CF* __restrict__ full, CH* __restrict__ half) {
  const int64_t j = blockIdx.x;
  const int n = (int)(ptr[j + 1] - ptr[j]);
  const CF* M = full + vptr[j];
  const int64_t ld = patch_ld(n);
  CH* Hj = half + hptr[j];
  for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += blockDim.x) {
    const int a = (int)(q / n), k = (int)(q % n);
    if (k <= a) Hj[(int64_t)a * (a + 1) / 2 + k] = cvt_in<CH>(M[a * ld + k]);
  }
}

}  // namespace dpgmg
