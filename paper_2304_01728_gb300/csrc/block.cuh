// Several right-hand sides at once (Sec. 5: loads solved together share the
// cost of reading the patches): block forms of the two products of the V-cycle
// that stream stored matrices from HBM.  Each stored entry is read once and
// applied to KB vectors (KB <= 4 per launch), so the bytes per right-hand side
// fall by KB.  Vectors of a block are stored one after another with a fixed
// stride; per vector the arithmetic and its order are those of the
// single-vector kernels' simple loops (no cross-vector reductions).
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
template <class C, class TIN, int PER, int KB>
__global__ void __launch_bounds__(256) k_patch_apply_blk(const int64_t* __restrict__ ptr,
                                                         const int32_t* __restrict__ dofs,
                                                         const int64_t* __restrict__ vptr,
                                                         const int2* __restrict__ chunks, const C* __restrict__ inv,
                                                         const TIN* __restrict__ r, int64_t ldr,
                                                         C* __restrict__ pbuf, int64_t ldp) {
  extern __shared__ unsigned char shraw[];
  __shared__ C part[8][32 * PER + 1];
  C* rj = reinterpret_cast<C*>(shraw);   // [KB][n]
  using O = Ops<C>;
  const int2 ch = chunks[blockIdx.x];
  const int64_t j = ch.x;
  const int64_t b = ptr[j];
  const int n = (int)(ptr[j + 1] - b);
  const int64_t ld = patch_ld(n);
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int32_t g = dofs[b + q];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) rj[kb * n + q] = cvt_in<C>(r[kb * ldr + g]);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int a = ch.y + PER * lane;
  C acc[KB][PER];
#pragma unroll
  for (int kb = 0; kb < KB; ++kb)
#pragma unroll
    for (int u = 0; u < PER; ++u) acc[kb][u] = O::zero();
  if (a < n) {
    const C* M = inv + vptr[j] + a;
    int k = w;
    if (PER == 2) {
      // 16-byte loads of (M[k][a], M[k][a+1]): a and ld are even
      const float4* M4 = reinterpret_cast<const float4*>(M);
      const int64_t s4 = ld / 2;
      for (; k + 8 < n; k += 16) {
        const float4 m0 = __ldcs(M4 + (int64_t)k * s4), m1 = __ldcs(M4 + (int64_t)(k + 8) * s4);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          const C r0 = rj[kb * n + k], r1 = rj[kb * n + k + 8];
          acc[kb][0] = O::fmac(r0, Ops<C>::mk(m0.x, m0.y), acc[kb][0]);
          acc[kb][1 % PER] = O::fmac(r0, Ops<C>::mk(m0.z, m0.w), acc[kb][1 % PER]);
          acc[kb][0] = O::fmac(r1, Ops<C>::mk(m1.x, m1.y), acc[kb][0]);
          acc[kb][1 % PER] = O::fmac(r1, Ops<C>::mk(m1.z, m1.w), acc[kb][1 % PER]);
        }
      }
      for (; k < n; k += 8) {
        const float4 m0 = __ldcs(M4 + (int64_t)k * s4);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          acc[kb][0] = O::fmac(rj[kb * n + k], Ops<C>::mk(m0.x, m0.y), acc[kb][0]);
          acc[kb][1 % PER] = O::fmac(rj[kb * n + k], Ops<C>::mk(m0.z, m0.w), acc[kb][1 % PER]);
        }
      }
    } else {
      for (; k + 8 < n; k += 16) {
        const C m0 = ld_stream(M + (size_t)k * ld), m1 = ld_stream(M + (size_t)(k + 8) * ld);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          acc[kb][0] = O::fmac(rj[kb * n + k], m0, acc[kb][0]);
          acc[kb][0] = O::fmac(rj[kb * n + k + 8], m1, acc[kb][0]);
        }
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
          pbuf[kb * ldp + b + c] = s2;
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
                                                  int64_t ld, int64_t nrows, int mode) {
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
      for (; k < nnz; k += 32) {
        const C v0 = __ldcs(vals + k);
        C xv[KB];
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) xv[kb] = x[kb * ld + cA];
        const int kn = k + 32;
        cA = kn < nnz ? __ldg(cols + kn) : 0;
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) acc[kb] = O::fma(v0, xv[kb], acc[kb]);
      }
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) acc[kb] = warp_sum_s(acc[kb]);
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

}  // namespace dpgmg
