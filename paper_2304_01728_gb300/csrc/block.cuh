// Several right-hand sides at once (Sec. 5: loads solved together share the
// cost of reading the patches): block forms of the V-cycle kernels that
// stream stored matrices from HBM (smoother, SpMV, macro-grid condensation and
// back-substitution).  Each stored entry is read once and applied to KB
// vectors (KB <= 4 per launch), so the bytes per right-hand side fall by KB.
// Vectors of a block are stored one after another with a fixed stride; per
// vector the arithmetic is that of the single-vector kernels (no
// cross-vector reductions).
#pragma once
#include "common.cuh"
#include "host_mesh.h"
#include "internal.h"
#include "smoother.cuh"

namespace dpgmg {

constexpr int BLK_MAX = 4;   // vectors per launch of a block kernel

// pbuf[kb * ldp + slot] = A_jj^-1 (R_j r_kb) for the patch columns of one work
// item (patch j, first column a0; PER columns per lane, warps split the rows
// k = w, w + 8, ...), for kb < KB.  r_kb = r + kb * ldr.  Shared memory:
// KB * n_j values of the gathered right-hand sides.
constexpr int BLK_DEPTH = 8;   // rows in flight per thread in the block smoother

// pbuf[kb * ldp + slot] = A_jj^-1 (R_j r_kb) for the patch columns of one work
// item (patch j, first column a0; PER columns per lane, warps split the rows
// k = w, w + 8, ...), for kb < KB.  r_kb = r + kb * ldr.  Shared memory:
// KB * n_j values of the gathered right-hand sides (dynamic) and, for the
// complex64 form, a ring of BLK_DEPTH 16-byte row pieces per thread that
// cp.async fills, so that the rows in flight do not hold registers.
template <class C, class TIN, int PER, int KB>
__global__ void __launch_bounds__(256) k_patch_apply_blk(const int64_t* __restrict__ ptr,
                                                         const int32_t* __restrict__ dofs,
                                                         const int64_t* __restrict__ vptr,
                                                         const int2* __restrict__ chunks, const C* __restrict__ inv,
                                                         const TIN* __restrict__ r, int64_t ldr,
                                                         C* __restrict__ pbuf, int64_t ldp,
                                                         const uint8_t* __restrict__ rflag, int64_t offU) {
  extern __shared__ unsigned char shraw[];
  __shared__ C part[8][32 * PER + 1];
  __shared__ float4 ring[PER == 2 ? BLK_DEPTH : 1][PER == 2 ? 256 : 1];
  C* rj = reinterpret_cast<C*>(shraw);   // [KB][n]
  using O = Ops<C>;
  const int2 ch = chunks[blockIdx.x];
  const int64_t j = ch.x;
  const int64_t b = ptr[j];
  const int n = (int)(ptr[j + 1] - b);
  const int64_t ld = patch_ld(n);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int a = ch.y + PER * lane;
  const C* M = inv + vptr[j] + a;
  const bool rp = rflag != nullptr && rflag[j] != 0;   // real packed block (k_patch_apply)
  if (PER == 2 && a < n && !rp) {
    // start the first BLK_DEPTH rows of this thread (k = w + 8 d) before the gather
    const float4* M4 = reinterpret_cast<const float4*>(M);
    const int64_t s4 = ld / 2;
#pragma unroll
    for (int d = 0; d < BLK_DEPTH; ++d) {
      const int k = w + 8 * d;
      if (k < n) cp_async16(&ring[d][threadIdx.x], M4 + (int64_t)k * s4);
      cp_async_commit();
    }
  }
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int32_t g = dofs[b + q];
    const int s = rp && g < offU ? -1 : 0;
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) rj[kb * n + q] = mul_i(cvt_in<C>(r[kb * ldr + g]), s);
  }
  __syncthreads();
  C acc[KB][PER];
#pragma unroll
  for (int kb = 0; kb < KB; ++kb)
#pragma unroll
    for (int u = 0; u < PER; ++u) acc[kb][u] = O::zero();
  if (a < n && rp) {
    // real rows (two columns of a lane in one load for PER = 2), four rows in flight
    using R = typename Ops<C>::R;
    const R* Wt = reinterpret_cast<const R*>(inv + vptr[j]) + a;
    const int64_t ldw = patch_ldr(n);   // real rows
    int k = w;
    for (; k + 24 < n; k += 32) {
      C m[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        m[u] = PER == 2 ? __ldcs(reinterpret_cast<const C*>(Wt + (int64_t)(k + 8 * u) * ldw))
                        : Ops<C>::mk(__ldcs(Wt + (int64_t)(k + 8 * u) * ldw), R(0));
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          const C rv = rj[kb * n + k + 8 * u];
          acc[kb][0] = rfma<C>(m[u].x, rv, acc[kb][0]);
          if (PER == 2) acc[kb][1 % PER] = rfma<C>(m[u].y, rv, acc[kb][1 % PER]);
        }
    }
    for (; k < n; k += 8) {
      const C m0 = PER == 2 ? __ldcs(reinterpret_cast<const C*>(Wt + (int64_t)k * ldw))
                            : Ops<C>::mk(__ldcs(Wt + (int64_t)k * ldw), R(0));
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) {
        acc[kb][0] = rfma<C>(m0.x, rj[kb * n + k], acc[kb][0]);
        if (PER == 2) acc[kb][1 % PER] = rfma<C>(m0.y, rj[kb * n + k], acc[kb][1 % PER]);
      }
    }
  } else if (a < n) {
    if (PER == 2) {
      const float4* M4 = reinterpret_cast<const float4*>(M);
      const int64_t s4 = ld / 2;
      int d = 0;
      for (int k = w; k < n; k += 8) {
        cp_async_wait<BLK_DEPTH - 1>();   // this thread's oldest group (row k) has landed
        const float4 m0 = ring[d][threadIdx.x];
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          const C rv = rj[kb * n + k];
          acc[kb][0] = O::fmac(rv, Ops<C>::mk(m0.x, m0.y), acc[kb][0]);
          acc[kb][1 % PER] = O::fmac(rv, Ops<C>::mk(m0.z, m0.w), acc[kb][1 % PER]);
        }
        // refill the slot with row k + 8 BLK_DEPTH (m0 has been consumed above)
        const int kn = k + 8 * BLK_DEPTH;
        if (kn < n) cp_async16(&ring[d][threadIdx.x], M4 + (int64_t)kn * s4);
        cp_async_commit();
        d = d + 1 == BLK_DEPTH ? 0 : d + 1;
      }
      cp_async_wait<0>();
    } else {
      int k = w;
      for (; k + 24 < n; k += 32) {
        C m[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) m[u] = ld_stream(M + (size_t)(k + 8 * u) * ld);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) acc[kb][0] = O::fmac(rj[kb * n + k + 8 * u], m[u], acc[kb][0]);
      }
      for (; k < n; k += 8) {
        const C m0 = ld_stream(M + (size_t)k * ld);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) acc[kb][0] = O::fmac(rj[kb * n + k], m0, acc[kb][0]);
      }
    }
  }
#pragma unroll
  for (int kb = 0; kb < KB; ++kb) {
#pragma unroll
    for (int u = 0; u < PER; ++u) part[w][PER * lane + u] = acc[kb][u];
    __syncthreads();
    if (w == 0) {
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int c = ch.y + PER * lane + u;
        if (c < n) {
          C s2 = part[0][PER * lane + u];
#pragma unroll
          for (int q = 1; q < 8; ++q) s2 = O::add(s2, part[q][PER * lane + u]);
          pbuf[kb * ldp + b + c] = rp ? mul_i(s2, dofs[b + c] < offU ? 1 : 0) : s2;
        }
      }
    }
    __syncthreads();
  }
}

// y_kb = A x_kb (mode 0) or b_kb - A x_kb (mode 1) for kb < KB, vectors at
// stride ld.  One warp per row; each stored entry is loaded once for the KB
// vectors; the column indices of the next step are loaded one step ahead.
template <class C, int KB>
__global__ void __launch_bounds__(256) k_spmv_blk(const int32_t* __restrict__ row_ent,
                                                  const int64_t* __restrict__ ent_start,
                                                  const int64_t* __restrict__ col_ptr,
                                                  const int32_t* __restrict__ col_idx,
                                                  const int64_t* __restrict__ val_ptr, const C* __restrict__ v,
                                                  const C* __restrict__ x, const C* __restrict__ b, C* __restrict__ y,
                                                  int64_t ld, int64_t nrows, int mode,
                                                  const uint8_t* __restrict__ rent, int64_t offU) {
  using O = Ops<C>;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < nrows; row += nw) {
    const int32_t E = row_ent[row];
    C acc[KB];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) acc[kb] = O::zero();
    if (E >= 0) {
      const int64_t c0 = col_ptr[E];
      const int nnz = (int)(col_ptr[E + 1] - c0);
      const C* vals = v + val_ptr[E] + (row - ent_start[E]) * nnz;
      const int32_t* cols = col_idx + c0;
      int k = lane;
      int cA = k < nnz ? __ldg(cols + k) : 0;
      int cB = k + 32 < nnz ? __ldg(cols + k + 32) : 0;
      const bool real = rent != nullptr && rent[E] != 0;   // packed real entity (complex64 values only)
      if (real) {
        using R = typename Ops<C>::R;
        const R* a = reinterpret_cast<const R*>(v + val_ptr[E]) + (row - ent_start[E]) * nnz;
        for (; k + 32 < nnz; k += 64) {
          const R w0 = __ldcs(a + k), w1 = __ldcs(a + k + 32);
          const int sA = cA < offU ? -1 : 0, sB = cB < offU ? -1 : 0;
          C x0[KB], x1[KB];
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) {
            x0[kb] = mul_i(x[kb * ld + cA], sA);
            x1[kb] = mul_i(x[kb * ld + cB], sB);
          }
          const int kn = k + 64;
          cA = kn < nnz ? __ldg(cols + kn) : 0;
          cB = kn + 32 < nnz ? __ldg(cols + kn + 32) : 0;
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) {
            acc[kb] = rfma<C>(w0, x0[kb], acc[kb]);
            acc[kb] = rfma<C>(w1, x1[kb], acc[kb]);
          }
        }
        if (k < nnz) {
          const R w0 = __ldcs(a + k);
          const int sA = cA < offU ? -1 : 0;
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) acc[kb] = rfma<C>(w0, mul_i(x[kb * ld + cA], sA), acc[kb]);
        }
        k = nnz;   // the complex loop below has nothing left
      }
      for (; k + 32 < nnz; k += 64) {   // two columns per lane per step, indices one step ahead
        const C v0 = __ldcs(vals + k), v1 = __ldcs(vals + k + 32);
        C x0[KB], x1[KB];
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          x0[kb] = x[kb * ld + cA];
          x1[kb] = x[kb * ld + cB];
        }
        const int kn = k + 64;
        cA = kn < nnz ? __ldg(cols + kn) : 0;
        cB = kn + 32 < nnz ? __ldg(cols + kn + 32) : 0;
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          acc[kb] = O::fma(v0, x0[kb], acc[kb]);
          acc[kb] = O::fma(v1, x1[kb], acc[kb]);
        }
      }
      if (k < nnz) {
        const C v0 = __ldcs(vals + k);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) acc[kb] = O::fma(v0, x[kb * ld + cA], acc[kb]);
      }
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) {
        acc[kb] = warp_sum_s(acc[kb]);
        if (real) acc[kb] = mul_i(acc[kb], row < offU ? 1 : 0);
      }
    }
    if (lane < KB) {
      C mine = acc[0];
#pragma unroll
      for (int kb = 1; kb < KB; ++kb)
        if (lane == kb) mine = acc[kb];
      y[lane * ld + row] = mode ? O::sub(b[lane * ld + row], mine) : mine;
    }
  }
}

// y_kb[g] = (accumulate ? y_kb[g] : 0) + theta * sum_{slots of g} pbuf_kb[slot]
// for kb = blockIdx.y (y at stride ld, pbuf at stride ldp)
template <class C>
__global__ void k_slot_sum_blk(const int64_t* __restrict__ sptr, const int32_t* __restrict__ slots,
                               const C* __restrict__ pbuf, int64_t ldp, C* __restrict__ y, int64_t ld, int64_t n,
                               double theta, int accumulate) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  const C* pb = pbuf + blockIdx.y * ldp;
  C acc = Ops<C>::zero();
  for (int64_t s = sptr[g]; s < sptr[g + 1]; ++s) acc = Ops<C>::add(acc, pb[slots[s]]);
  acc = Ops<C>::scale(acc, (typename Ops<C>::R)theta);
  C* yk = y + blockIdx.y * ld;
  yk[g] = accumulate ? Ops<C>::add(yk[g], acc) : acc;
}

// Block forms of the macro-grid transfers (one CTA per coarse element K): the
// element's stored blocks Y_K (and A_II^-1 for the back-substitution) are read
// once for KB vectors at stride ld (cbuf at stride ldc).
template <class C, int KB>
__global__ void k_condense_apply_blk(int nS, int nI, const int64_t* __restrict__ Ig, const C* __restrict__ Y,
                                     const C* __restrict__ r, int64_t ld, C* __restrict__ cbuf, int64_t ldc) {
  extern __shared__ unsigned char shraw[];
  C* rI = reinterpret_cast<C*>(shraw);   // [KB][nI]
  const int64_t K = blockIdx.x;
  for (int i = threadIdx.x; i < nI; i += blockDim.x) {
    const int64_t g = Ig[K * nI + i];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) rI[kb * nI + i] = r[kb * ld + g];
  }
  __syncthreads();
  const C* YK = Y + K * (size_t)nI * nS;
  for (int a = threadIdx.x; a < nS; a += blockDim.x) {
    C acc[KB];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) acc[kb] = Ops<C>::zero();
    for (int i = 0; i < nI; ++i) {
      const C y = YK[(size_t)i * nS + a];
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) acc[kb] = Ops<C>::fmac(rI[kb * nI + i], y, acc[kb]);
    }
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) cbuf[kb * ldc + K * nS + a] = acc[kb];
  }
}

template <class C, int KB>
__global__ void k_backsub_blk(int nS, int nI, const int64_t* __restrict__ Sg, const int64_t* __restrict__ Ig,
                              const C* __restrict__ Ai, const C* __restrict__ Y, const C* __restrict__ r,
                              C* __restrict__ x, int64_t ld) {
  extern __shared__ unsigned char shraw[];
  C* rI = reinterpret_cast<C*>(shraw);   // [KB][nI]
  C* xS = rI + KB * nI;                  // [KB][nS]
  using O = Ops<C>;
  const int64_t K = blockIdx.x;
  for (int i = threadIdx.x; i < nI; i += blockDim.x) {
    const int64_t g = Ig[K * nI + i];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) rI[kb * nI + i] = r[kb * ld + g];
  }
  for (int a = threadIdx.x; a < nS; a += blockDim.x) {
    const int64_t g = Sg[K * nS + a];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) xS[kb * nS + a] = g >= 0 ? x[kb * ld + g] : O::zero();
  }
  __syncthreads();
  const C* AiK = Ai + K * (size_t)nI * nI;
  const C* YK = Y + K * (size_t)nI * nS;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = w; i < nI; i += blockDim.x >> 5) {
    C acc[KB];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) acc[kb] = O::zero();
    for (int k = lane; k < nI; k += 32) {
      const C m = AiK[(size_t)i * nI + k];
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) acc[kb] = O::fma(m, rI[kb * nI + k], acc[kb]);
    }
    for (int a = lane; a < nS; a += 32) {
      const C m = YK[(size_t)i * nS + a];
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) acc[kb] = O::fnma(m, xS[kb * nS + a], acc[kb]);
    }
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) acc[kb] = warp_sum_s(acc[kb]);
    if (lane < KB) {
      C mine = acc[0];
#pragma unroll
      for (int kb = 1; kb < KB; ++kb)
        if (lane == kb) mine = acc[kb];
      x[lane * ld + Ig[K * nI + i]] = mine;
    }
  }
}

}  // namespace dpgmg
