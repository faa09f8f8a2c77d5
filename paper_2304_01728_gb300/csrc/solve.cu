// The DPG-MG V-cycle and MG-preconditioned conjugate gradients (Sec. 3-4):
//   k_spmv            y = A x or y = b - A x on the entity-shared CSR operator
//   k_patch_apply     per-patch dense products A_j^-1 (R_j r)   (additive Schwarz)
//   k_slot_sum        x_g (+)= theta * sum of the patch results of DOF g
//   k_condense_*      macro-grid residual condensation r_S -= Y^H r_I (h levels)
//   k_backsub         x_I = A_II^-1 r_I - Y x_S                  (h levels)
//   k_csr_real        natural inclusion P and its adjoint P^T      (h levels)
//   (coarsest solve: coarse.cu)
//   k_dot_*, k_axpy*  CG recurrences in FP64
// Every kernel is templated on the complex type of the V-cycle (complex128
// on the FP64 path, complex64 on the mixed path); CG always runs in FP64.
#include <algorithm>
#include <initializer_list>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "block.cuh"
#include "smoother.cuh"

namespace dpgmg {

template <class C> struct Prec;
template <> struct Prec<double2> {
  static const double2* A(const ECSRDev& a) { return a.v64; }
  static const double2* inv(const PatchDev& p) { return p.inv64; }
  static const double2* half(const PatchDev&) { return nullptr; }
  static const double2* Y(const Level& l) { return l.Y64; }
  static const double2* Ai(const Level& l) { return l.Ai64; }
};
template <> struct Prec<float2> {
  static const float2* A(const ECSRDev& a) { return a.v32; }
  static const float2* inv(const PatchDev& p) { return p.inv32; }
  static const float2* half(const PatchDev& p) { return p.h32; }
  static const float2* Y(const Level& l) { return l.Y32; }
  static const float2* Ai(const Level& l) { return l.Ai32; }
};

// ------------------------------------------------------------ profiling
// Events bracketing one chosen kernel (DPGMG_PROF_*) on the launching stream.
// Inside a stream capture the two records become event-record nodes of the
// graph; such pairs are read after every replay (prof_graph_accumulate).
static bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DPG_CUDA(cudaStreamIsCapturing(st, &cs));
  return cs == cudaStreamCaptureStatusActive;
}
static int prof_begin(SystemImpl* S, cudaStream_t st) {
  if (!S) return -1;
  cudaEvent_t a, b;
  DPG_CUDA(cudaEventCreate(&a));
  DPG_CUDA(cudaEventCreate(&b));
  const int idx = (int)S->prof_events.size();
  S->prof_events.emplace_back(a, b);
  if (capturing(st)) {
    DPG_CUDA(cudaEventRecordWithFlags(a, st, cudaEventRecordExternal));
    S->prof_graph_pairs.push_back(idx);
  } else {
    DPG_CUDA(cudaEventRecord(a, st));
  }
  return idx;
}
static void prof_end(SystemImpl* S, int idx, cudaStream_t st) {
  if (!S || idx < 0) return;
  if (capturing(st)) DPG_CUDA(cudaEventRecordWithFlags(S->prof_events[idx].second, st, cudaEventRecordExternal));
  else DPG_CUDA(cudaEventRecord(S->prof_events[idx].second, st));
}
// after a replay has completed: add the times of the graph's event pairs
static void prof_graph_accumulate(SystemImpl& S) {
  for (int idx : S.prof_graph_pairs) {
    float t = 0.f;
    DPG_CUDA(cudaEventElapsedTime(&t, S.prof_events[idx].first, S.prof_events[idx].second));
    S.prof_graph_ms += t;
    ++S.prof_graph_n;
  }
}

void profile_clear(SystemImpl& S) {
  for (auto& e : S.prof_events) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  S.prof_events.clear();
  S.prof_graph_pairs.clear();
  S.prof_graph_ms = 0.0;
  S.prof_graph_n = 0;
}

void profile_read(SystemImpl& S, double* ms, long long* launches, long long* bytes) {
  double tot = S.prof_graph_ms;
  long long n = S.prof_graph_n;
  std::vector<char> in_graph(S.prof_events.size(), 0);
  for (int idx : S.prof_graph_pairs) in_graph[idx] = 1;
  for (size_t i = 0; i < S.prof_events.size(); ++i) {
    if (in_graph[i]) continue;
    DPG_CUDA(cudaEventSynchronize(S.prof_events[i].second));
    float t = 0.f;
    DPG_CUDA(cudaEventElapsedTime(&t, S.prof_events[i].first, S.prof_events[i].second));
    tot += t;
    ++n;
  }
  if (ms) *ms = tot;
  if (launches) *launches = n;
  if (bytes) *bytes = S.prof_bytes;
  profile_clear(S);
}

template <class C> __device__ __forceinline__ C warp_sum(C v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// ------------------------------------------------------------------ SpMV
// A row of a packed real entity (k_pack_ops): the lane's part of
// sum_c a[r][c] (i^(-s_c) x_c) over columns k = lane, lane + 32, ...: four
// columns per lane per step (the 4-byte values leave room for more loads in
// flight), then two, then one, with two accumulators alternating by column;
// PF: each step's column indices loaded one step ahead.  The same order for
// both PF forms (bitwise equal results).  The caller sums the lanes and
// applies i^(s_r).
template <bool PF>
__device__ __forceinline__ float2 spmv_real_row(const float* __restrict__ a, const int32_t* __restrict__ cols,
                                                int nnz, const float2* __restrict__ x, int64_t offU, int lane) {
  float2 acc = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
  auto xs = [&](int c) { return mul_i(x[c], c < offU ? -1 : 0); };
  int k = lane;
  int ci[4] = {0, 0, 0, 0};
  if (PF)
#pragma unroll
    for (int u = 0; u < 4; ++u) ci[u] = k + 32 * u < nnz ? __ldg(cols + k + 32 * u) : 0;
  for (; k + 96 < nnz; k += 128) {
    float w[4];
    float2 xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) w[u] = __ldcs(a + k + 32 * u);
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = xs(PF ? ci[u] : cols[k + 32 * u]);
    if (PF) {
      const int kn = k + 128;
#pragma unroll
      for (int u = 0; u < 4; ++u) ci[u] = kn + 32 * u < nnz ? __ldg(cols + kn + 32 * u) : 0;
    }
#pragma unroll
    for (int u = 0; u < 4; u += 2) {
      acc = rfma<float2>(w[u], xv[u], acc);
      acc1 = rfma<float2>(w[u + 1], xv[u + 1], acc1);
    }
  }
  // at most three columns left (k + 96 >= nnz); ci[] holds the indices of k, k + 32, k + 64
  if (k + 32 < nnz) {
    const float w0 = __ldcs(a + k), w1 = __ldcs(a + k + 32);
    const float2 x0 = xs(PF ? ci[0] : cols[k]), x1 = xs(PF ? ci[1] : cols[k + 32]);
    acc = rfma<float2>(w0, x0, acc);
    acc1 = rfma<float2>(w1, x1, acc1);
    if (PF) {
      ci[0] = ci[2];
      ci[1] = ci[3];
    }
    k += 64;
  }
  if (k < nnz) acc = rfma<float2>(__ldcs(a + k), xs(PF ? ci[0] : cols[k]), acc);
  return make_float2(acc.x + acc1.x, acc.y + acc1.y);
}

// mode 0: y = A x; mode 1: y = b - A x.  One warp per row.  rent: packed
// real entities (complex64 values only; null otherwise).
template <class C>
__global__ void __launch_bounds__(256) k_spmv(const int32_t* __restrict__ row_ent, const int64_t* __restrict__ ent_start,
                                              const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ col_idx,
                                              const int64_t* __restrict__ val_ptr, const C* __restrict__ v,
                                              const C* __restrict__ x, const C* __restrict__ b, C* __restrict__ y,
                                              int64_t nrows, int mode, const uint8_t* __restrict__ rent,
                                              int64_t offU) {
  using O = Ops<C>;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < nrows; row += nw) {
    const int32_t E = row_ent[row];
    C acc = O::zero();
    if constexpr (std::is_same<C, float2>::value) {
      if (E >= 0 && rent != nullptr && rent[E] != 0) {
        const int64_t c0 = col_ptr[E];
        const int nnz = (int)(col_ptr[E + 1] - c0);
        const float* a = reinterpret_cast<const float*>(v + val_ptr[E]) + (row - ent_start[E]) * nnz;
        acc = mul_i(warp_sum(spmv_real_row<false>(a, col_idx + c0, nnz, x, offU, lane)), row < offU ? 1 : 0);
        if (lane == 0) y[row] = mode ? O::sub(b[row], acc) : acc;
        continue;
      }
    }
    if (E >= 0) {
      const int64_t c0 = col_ptr[E];
      const int nnz = (int)(col_ptr[E + 1] - c0);
      const C* vals = v + val_ptr[E] + (row - ent_start[E]) * nnz;
      const int32_t* cols = col_idx + c0;
      C acc1 = O::zero();
      int k = lane;
      for (; k + 32 < nnz; k += 64) {   // two independent loads per lane per step
        const C v0 = __ldcs(vals + k), v1 = __ldcs(vals + k + 32);
        const int cA = cols[k], cB = cols[k + 32];
        acc = O::fma(v0, x[cA], acc);
        acc1 = O::fma(v1, x[cB], acc1);
      }
      if (k < nnz) acc = O::fma(__ldcs(vals + k), x[cols[k]], acc);
      acc = warp_sum(O::add(acc, acc1));
    }
    if (lane == 0) y[row] = mode ? O::sub(b[row], acc) : acc;
  }
}

// The same product with one row per half-warp: two rows of a warp in flight
// at once, so that twice the rows' dependent loads (entity tables, column
// indices, gathered x) overlap.  16 lanes per row, columns k = h, h + 16, ...
// (h = lane within the half) in two accumulators alternating by column;
// packed real entities as in k_spmv.  A different summation order from
// k_spmv: equal to rounding.
template <class C>
__global__ void __launch_bounds__(256) k_spmv_hw(const int32_t* __restrict__ row_ent,
                                                 const int64_t* __restrict__ ent_start,
                                                 const int64_t* __restrict__ col_ptr,
                                                 const int32_t* __restrict__ col_idx,
                                                 const int64_t* __restrict__ val_ptr, const C* __restrict__ v,
                                                 const C* __restrict__ x, const C* __restrict__ b, C* __restrict__ y,
                                                 int64_t nrows, int mode, const uint8_t* __restrict__ rent,
                                                 int64_t offU) {
  using O = Ops<C>;
  const int lane = threadIdx.x & 31, h = lane & 15;
  const int64_t nh = (int64_t)gridDim.x * (blockDim.x >> 4);   // half-warps of the grid
  // the loop bound depends on the warp only: both halves run every trip (full-warp shuffles)
  for (int64_t base = 2 * (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)); base < nrows; base += nh) {
    const int64_t row = base + (lane >> 4);
    C acc = O::zero(), acc1 = O::zero();
    bool real = false;
    const int32_t E = row < nrows ? row_ent[row] : -1;
    if (E >= 0) {
      const int64_t c0 = col_ptr[E];
      const int nnz = (int)(col_ptr[E + 1] - c0);
      const int32_t* cols = col_idx + c0;
      const int64_t roff = (row - ent_start[E]) * nnz;
      if constexpr (std::is_same<C, float2>::value) real = rent != nullptr && rent[E] != 0;
      if (real) {
        if constexpr (std::is_same<C, float2>::value) {
          const float* a = reinterpret_cast<const float*>(v + val_ptr[E]) + roff;
          int k = h;
          for (; k + 16 < nnz; k += 32) {
            const float w0 = __ldcs(a + k), w1 = __ldcs(a + k + 16);
            const int cA = cols[k], cB = cols[k + 16];
            acc = rfma<float2>(w0, mul_i(x[cA], cA < offU ? -1 : 0), acc);
            acc1 = rfma<float2>(w1, mul_i(x[cB], cB < offU ? -1 : 0), acc1);
          }
          if (k < nnz) {
            const int cA = cols[k];
            acc = rfma<float2>(__ldcs(a + k), mul_i(x[cA], cA < offU ? -1 : 0), acc);
          }
        }
      } else {
        const C* vals = v + val_ptr[E] + roff;
        int k = h;
        for (; k + 16 < nnz; k += 32) {
          const C v0 = __ldcs(vals + k), v1 = __ldcs(vals + k + 16);
          const int cA = cols[k], cB = cols[k + 16];
          acc = O::fma(v0, x[cA], acc);
          acc1 = O::fma(v1, x[cB], acc1);
        }
        if (k < nnz) acc = O::fma(__ldcs(vals + k), x[cols[k]], acc);
      }
    }
    acc = O::add(acc, acc1);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (real) acc = mul_i(acc, row < offU ? 1 : 0);
    if (h == 0 && row < nrows) y[row] = mode ? O::sub(b[row], acc) : acc;
  }
}

// The same product with the column indices of the next step loaded one step
// ahead, so that each step waits on the gathered x entries only (the index ->
// gather chain of k_spmv is the latency it is bound by).  Identical
// accumulation order: results are bitwise those of k_spmv.
template <class C>
__global__ void __launch_bounds__(256) k_spmv_pf(const int32_t* __restrict__ row_ent,
                                                 const int64_t* __restrict__ ent_start,
                                                 const int64_t* __restrict__ col_ptr,
                                                 const int32_t* __restrict__ col_idx,
                                                 const int64_t* __restrict__ val_ptr, const C* __restrict__ v,
                                                 const C* __restrict__ x, const C* __restrict__ b, C* __restrict__ y,
                                                 int64_t nrows, int mode, const uint8_t* __restrict__ rent,
                                                 int64_t offU) {
  using O = Ops<C>;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < nrows; row += nw) {
    const int32_t E = row_ent[row];
    C acc = O::zero();
    if constexpr (std::is_same<C, float2>::value) {
      if (E >= 0 && rent != nullptr && rent[E] != 0) {
        const int64_t c0 = col_ptr[E];
        const int nnz = (int)(col_ptr[E + 1] - c0);
        const float* a = reinterpret_cast<const float*>(v + val_ptr[E]) + (row - ent_start[E]) * nnz;
        acc = mul_i(warp_sum(spmv_real_row<true>(a, col_idx + c0, nnz, x, offU, lane)), row < offU ? 1 : 0);
        if (lane == 0) y[row] = mode ? O::sub(b[row], acc) : acc;
        continue;
      }
    }
    if (E >= 0) {
      const int64_t c0 = col_ptr[E];
      const int nnz = (int)(col_ptr[E + 1] - c0);
      const C* vals = v + val_ptr[E] + (row - ent_start[E]) * nnz;
      const int32_t* cols = col_idx + c0;
      C acc1 = O::zero();
      int k = lane;
      int cA = k < nnz ? __ldg(cols + k) : 0;
      int cB = k + 32 < nnz ? __ldg(cols + k + 32) : 0;
      for (; k + 32 < nnz; k += 64) {
        const C v0 = __ldcs(vals + k), v1 = __ldcs(vals + k + 32);
        const C x0 = x[cA], x1 = x[cB];
        const int kn = k + 64;
        cA = kn < nnz ? __ldg(cols + kn) : 0;
        cB = kn + 32 < nnz ? __ldg(cols + kn + 32) : 0;
        acc = O::fma(v0, x0, acc);
        acc1 = O::fma(v1, x1, acc1);
      }
      if (k < nnz) acc = O::fma(__ldcs(vals + k), x[cA], acc);
      acc = warp_sum(O::add(acc, acc1));
    }
    if (lane == 0) y[row] = mode ? O::sub(b[row], acc) : acc;
  }
}

// The same product with the warp's whole stream of (value, column index)
// pairs, across its rows, prefetched SPMV_DEPTH steps ahead by cp.async into
// a per-thread shared-memory ring: the loads in flight hold no registers, so
// a small kernel keeps enough bytes in flight to stream the values.  Same
// accumulation order as k_spmv (two accumulators alternating by step):
// bitwise the same results.
constexpr int SPMV_DEPTH = 8;

// Row descriptor of the ring kernels (steps = ceil(nnz / 32); 0 for a row of no entity).
template <class T> struct RingRow {
  int64_t row;
  int nnz, steps;
  const T* vals;
  const int32_t* cols;
  int64_t voff;
};
template <class T>
__device__ __forceinline__ RingRow<T> ring_open(int64_t row, int64_t nrows, const int32_t* __restrict__ row_ent,
                                                const int64_t* __restrict__ ent_start,
                                                const int64_t* __restrict__ col_ptr,
                                                const int32_t* __restrict__ col_idx,
                                                const int64_t* __restrict__ val_ptr, const T* v) {
  RingRow<T> c;
  c.row = row;
  c.nnz = 0;
  c.steps = 0;
  c.vals = nullptr;
  c.cols = nullptr;
  c.voff = 0;
  if (row < nrows) {
    const int32_t E = row_ent[row];
    if (E >= 0) {
      const int64_t c0 = col_ptr[E];
      c.nnz = (int)(col_ptr[E + 1] - c0);
      c.voff = val_ptr[E] + (row - ent_start[E]) * c.nnz;
      c.vals = v + c.voff;
      c.cols = col_idx + c0;
      c.steps = (c.nnz + 31) >> 5;
    }
  }
  return c;
}

template <class C>
__device__ __forceinline__ void ring_copy(C* dst, const C* src) {
  if constexpr (sizeof(C) == 16) cp_async16(dst, src);
  else cp_async8(dst, src);
}

template <class C>
__global__ void __launch_bounds__(256) k_spmv_ring(const int32_t* __restrict__ row_ent,
                                                   const int64_t* __restrict__ ent_start,
                                                   const int64_t* __restrict__ col_ptr,
                                                   const int32_t* __restrict__ col_idx,
                                                   const int64_t* __restrict__ val_ptr, const C* __restrict__ v,
                                                   const C* __restrict__ x, const C* __restrict__ b, C* __restrict__ y,
                                                   int64_t nrows, int mode) {
  __shared__ C sv[SPMV_DEPTH][256];
  __shared__ int32_t si[SPMV_DEPTH][256];
  using O = Ops<C>;
  const int lane = threadIdx.x & 31, t = threadIdx.x;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t first = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  // prefetch cursor: the (row, step) whose pair is copied next
  RingRow<C> p = ring_open<C>(first, nrows, row_ent, ent_start, col_ptr, col_idx, val_ptr, v);
  int ps = 0;
  while (p.row < nrows && p.steps == 0) p = ring_open<C>(p.row + nw, nrows, row_ent, ent_start, col_ptr, col_idx,
                                                         val_ptr, v);
  auto issue = [&](int slot) {
    if (p.row < nrows) {
      const int k = lane + 32 * ps;
      if (k < p.nnz) {
        ring_copy<C>(&sv[slot][t], p.vals + k);
        cp_async4(&si[slot][t], p.cols + k);
      }
      if (++ps >= p.steps) {
        ps = 0;
        do {
          p = ring_open<C>(p.row + nw, nrows, row_ent, ent_start, col_ptr, col_idx, val_ptr, v);
        } while (p.row < nrows && p.steps == 0);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < SPMV_DEPTH; ++d) issue(d);
  int slot = 0;
  for (int64_t row = first; row < nrows; row += nw) {
    const RingRow<C> c = ring_open<C>(row, nrows, row_ent, ent_start, col_ptr, col_idx, val_ptr, v);
    C acc = O::zero(), acc1 = O::zero();
    for (int st = 0; st < c.steps; ++st) {
      cp_async_wait<SPMV_DEPTH - 1>();
      if (lane + 32 * st < c.nnz) {
        const C val = sv[slot][t];
        const C xv = x[si[slot][t]];
        if (st & 1) acc1 = O::fma(val, xv, acc1);
        else acc = O::fma(val, xv, acc);
      }
      issue(slot);
      slot = slot + 1 == SPMV_DEPTH ? 0 : slot + 1;
    }
    acc = warp_sum(O::add(acc, acc1));
    if (lane == 0) y[row] = mode ? O::sub(b[row], acc) : acc;
  }
  cp_async_wait<0>();
}

// Entity-blocked SpMV: one warp per task (entity E, rows r0 .. r0 + G - 1 of
// E).  The G rows share E's column list, so each column index and x entry is
// loaded once for G rows and G value streams are in flight per column.
template <class C, int G>
__global__ void __launch_bounds__(256) k_spmv_ent(const int2* __restrict__ tasks, int64_t ntasks,
                                                  const int64_t* __restrict__ ent_start,
                                                  const int32_t* __restrict__ ent_nd, const int64_t* __restrict__ col_ptr,
                                                  const int32_t* __restrict__ col_idx,
                                                  const int64_t* __restrict__ val_ptr, const C* __restrict__ v,
                                                  const C* __restrict__ x, const C* __restrict__ b, C* __restrict__ y,
                                                  int mode, const uint8_t* __restrict__ rent, int64_t offU) {
  using O = Ops<C>;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < ntasks; t += nw) {
    const int2 tk = tasks[t];
    const int E = tk.x, r0 = tk.y;
    const int g = min(G, ent_nd[E] - r0);
    const int64_t c0 = col_ptr[E];
    const int nnz = (int)(col_ptr[E + 1] - c0);
    const C* vals = v + val_ptr[E] + (int64_t)r0 * nnz;
    const int32_t* cols = col_idx + c0;
    C acc[G];
#pragma unroll
    for (int r = 0; r < G; ++r) acc[r] = O::zero();
    const bool real = rent != nullptr && rent[E] != 0;   // packed real entity (complex64 values only)
    if (real) {
      using R = typename Ops<C>::R;
      const R* a = reinterpret_cast<const R*>(v + val_ptr[E]) + (int64_t)r0 * nnz;
      for (int k = lane; k < nnz; k += 32) {
        const int c = cols[k];
        const C xv = mul_i(x[c], c < offU ? -1 : 0);
#pragma unroll
        for (int r = 0; r < G; ++r)
          if (r < g) acc[r] = rfma<C>(__ldcs(a + (int64_t)r * nnz + k), xv, acc[r]);
      }
    }
    for (int k = real ? nnz : lane; k < nnz; k += 32) {
      const C xv = x[cols[k]];
#pragma unroll
      for (int r = 0; r < G; ++r)
        if (r < g) acc[r] = O::fma(__ldcs(vals + (int64_t)r * nnz + k), xv, acc[r]);
    }
    C mine = O::zero();
#pragma unroll
    for (int r = 0; r < G; ++r) {
      const C sr = warp_sum(acc[r]);
      if (lane == r) mine = sr;
    }
    if (lane < g) {
      const int64_t row = ent_start[E] + r0 + lane;
      if (real) mine = mul_i(mine, row < offU ? 1 : 0);
      y[row] = mode ? O::sub(b[row], mine) : mine;
    }
  }
}

// rows that belong to no entity: y = 0 (mode 0) or b (mode 1)
template <class C>
__global__ void k_null_rows(const int32_t* __restrict__ rows, int64_t n, const C* __restrict__ b, C* __restrict__ y,
                            int mode) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t r = rows[i];
  y[r] = mode ? b[r] : Ops<C>::zero();
}

template <class C> struct SpmvSlot;
template <> struct SpmvSlot<float2> { static constexpr int v = 0; };
template <> struct SpmvSlot<double2> { static constexpr int v = 1; };

// G: rows of one entity per warp (1, 2, 4, 8); SPMV_PF = one row per warp with
// the column indices loaded one step ahead (k_spmv_pf); SPMV_RING = one row
// per warp with the (value, index) stream prefetched by cp.async (k_spmv_ring)
constexpr int SPMV_PF = 16;
constexpr int SPMV_RING = 32;   // one row per warp, (value, index) stream prefetched by cp.async
constexpr int SPMV_HALF = 64;   // one row per half-warp (k_spmv_hw)
// complex64 values with packed real entities: every SpMV but the cp.async
// ring variant reads them
template <class C> static const uint8_t* packed_rows(const ECSRDev& A) {
  return std::is_same<C, float2>::value ? A.rent : nullptr;
}

template <class C>
static void spmv_g(const ECSRDev& A, const C* vals, const C* x, const C* b, C* y, int mode, int G, cudaStream_t st) {
  const uint8_t* rent = packed_rows<C>(A);
  if (rent && G == SPMV_RING) G = SPMV_PF;   // the ring kernel reads complex64 values only
  if (G == SPMV_HALF) {
    int64_t blocks = std::min<int64_t>((A.nrows + 15) / 16, 152 * 16);
    k_spmv_hw<C><<<(unsigned)blocks, 256, 0, st>>>(A.row_ent, A.ent_start, A.col_ptr, A.col_idx, A.val_ptr, vals, x,
                                                    b, y, A.nrows, mode, rent, A.offU);
    DPG_CHECK_LAUNCH();
    return;
  }
  if (G == SPMV_RING) {
    int64_t blocks = std::min<int64_t>((A.nrows + 7) / 8, 152 * 8);
    k_spmv_ring<C><<<(unsigned)blocks, 256, 0, st>>>(A.row_ent, A.ent_start, A.col_ptr, A.col_idx, A.val_ptr, vals, x,
                                                      b, y, A.nrows, mode);
    DPG_CHECK_LAUNCH();
    return;
  }
  if (G == SPMV_PF) {
    int64_t blocks = std::min<int64_t>((A.nrows + 7) / 8, 152 * 16);
    k_spmv_pf<C><<<(unsigned)blocks, 256, 0, st>>>(A.row_ent, A.ent_start, A.col_ptr, A.col_idx, A.val_ptr, vals, x,
                                                    b, y, A.nrows, mode, rent, A.offU);
    DPG_CHECK_LAUNCH();
    return;
  }
  if (G <= 1 || !A.tasks[1]) {
    int64_t blocks = std::min<int64_t>((A.nrows + 7) / 8, 152 * 16);
    k_spmv<C><<<(unsigned)blocks, 256, 0, st>>>(A.row_ent, A.ent_start, A.col_ptr, A.col_idx, A.val_ptr, vals, x, b,
                                                 y, A.nrows, mode, rent, A.offU);
    DPG_CHECK_LAUNCH();
    return;
  }
  const int gi = G == 2 ? 1 : (G == 4 ? 2 : 3);
  const int64_t nt = A.ntasks[gi];
  const unsigned blocks = (unsigned)std::min<int64_t>((nt + 7) / 8, 152 * 16);
  if (G == 2)
    k_spmv_ent<C, 2><<<blocks, 256, 0, st>>>(A.tasks[gi], nt, A.ent_start, A.ent_nd, A.col_ptr, A.col_idx, A.val_ptr,
                                             vals, x, b, y, mode, rent, A.offU);
  else if (G == 4)
    k_spmv_ent<C, 4><<<blocks, 256, 0, st>>>(A.tasks[gi], nt, A.ent_start, A.ent_nd, A.col_ptr, A.col_idx, A.val_ptr,
                                             vals, x, b, y, mode, rent, A.offU);
  else
    k_spmv_ent<C, 8><<<blocks, 256, 0, st>>>(A.tasks[gi], nt, A.ent_start, A.ent_nd, A.col_ptr, A.col_idx, A.val_ptr,
                                             vals, x, b, y, mode, rent, A.offU);
  DPG_CHECK_LAUNCH();
  if (A.n_null) {
    k_null_rows<C><<<(unsigned)((A.n_null + 255) / 256), 256, 0, st>>>(A.null_rows, A.n_null, b, y, mode);
    DPG_CHECK_LAUNCH();
  }
}

template <class C>
static void spmv(const ECSRDev& A, const C* vals, const C* x, const C* b, C* y, int mode, cudaStream_t st,
                 SystemImpl* prof = nullptr) {
  int pe = prof_begin(prof, st);
  spmv_g<C>(A, vals, x, b, y, mode, A.gsel[SpmvSlot<C>::v], st);
  prof_end(prof, pe, st);
}

// ------------------------------------------------- double-float CG operator
// The CG operator is stored as complex64 high and low parts (a = a_hi + a_lo,
// exact to ~2^-48) and applied with error-free FP32 transformations
// (TwoProduct by fma, TwoSum; Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005): products a_hi x_hi are kept exactly,
// the cross terms a_hi x_lo + a_lo x_hi are added to the low accumulator.
// The result carries ~48 significant bits, enough for the FP64 CG recurrence,
// without the FP64 pipe that bounds a complex128 SpMV on this GPU.
__device__ __forceinline__ void df_add(float& sh, float& sl, float p, float q) {
  const float s = sh + p;
  const float bb = s - sh;
  const float e = (sh - (s - bb)) + (p - bb);
  sh = s;
  sl += e + q;
}
__device__ __forceinline__ void df_mul(float ah, float al, float xh, float xl, float& p, float& q) {
  p = ah * xh;
  q = fmaf(ah, xh, -p);
  q = fmaf(ah, xl, q);
  q = fmaf(al, xh, q);
}

// Warp sum of double-float values (h, l) with TwoSum on the high parts; every
// lane ends with the same (h, l) (the exact error of a + b does not depend on
// the order of the operands).
__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    const float s = h + oh;
    const float bb = s - h;
    const float e = (h - (s - bb)) + (oh - bb);
    h = s;
    l = l + ol + e;
  }
}

// One CTA per 32 consecutive rows (4 per warp).  The row sums stay in FP32
// pairs up to the end; one warp then turns the 32 results into complex128 with
// full-warp instructions (the FP64 pipe of this GPU runs at 1/64 of FP32).
// PF: the column indices of the next step are loaded one step ahead (same
// arithmetic, bitwise equal results).
constexpr int DF_ROWS = 32;
template <bool PF>
__global__ void __launch_bounds__(256) k_spmv_df(const int32_t* __restrict__ row_ent, const int64_t* __restrict__ ent_start,
                                                 const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ col_idx,
                                                 const int64_t* __restrict__ val_ptr, const float2* __restrict__ vh,
                                                 const float2* __restrict__ vl, const float2* __restrict__ xh,
                                                 const float2* __restrict__ xl, const double2* __restrict__ b,
                                                 double2* __restrict__ y, int64_t nrows, int mode,
                                                 const uint8_t* __restrict__ rent, int64_t offU) {
  __shared__ float4 res[DF_ROWS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * DF_ROWS;
#pragma unroll 1
  for (int i = 0; i < DF_ROWS / 8; ++i) {
    const int64_t row = base + w * (DF_ROWS / 8) + i;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const int32_t E = row < nrows ? row_ent[row] : -1;
    if (E >= 0) {
      const int64_t c0 = col_ptr[E];
      const int nnz = (int)(col_ptr[E + 1] - c0);
      const int64_t off = val_ptr[E] + (row - ent_start[E]) * nnz;
      const int32_t* cols = col_idx + c0;
      int pA = 0, pB = 0;   // PF: indices of this step, loaded one step ahead
      if (PF && lane < nnz) {
        pA = __ldg(cols + lane);
        pB = lane + 32 < nnz ? __ldg(cols + lane + 32) : pA;
      }
      const bool real = rent != nullptr && rent[E] != 0;
      if (real) {   // packed real entity (k_pack_ops): a = ah + al, x_c carries i^(-s_c)
        const float* ahr = reinterpret_cast<const float*>(vh + val_ptr[E]) + (row - ent_start[E]) * nnz;
        const float* alr = reinterpret_cast<const float*>(vl + val_ptr[E]) + (row - ent_start[E]) * nnz;
        for (int k = lane; k < nnz; k += 64) {
          const bool two = k + 32 < nnz;
          const float ah0 = __ldcs(ahr + k), al0 = __ldcs(alr + k);
          const int cA = PF ? pA : cols[k];
          const float ah1 = two ? __ldcs(ahr + k + 32) : 0.f, al1 = two ? __ldcs(alr + k + 32) : 0.f;
          const int cB = PF ? pB : (two ? cols[k + 32] : cA);
          const int sA = cA < offU ? -1 : 0, sB = cB < offU ? -1 : 0;
          const float2 uh0 = mul_i(xh[cA], sA), ul0 = mul_i(xl[cA], sA);
          const float2 uh1 = mul_i(xh[cB], sB), ul1 = mul_i(xl[cB], sB);
          if (PF) {
            const int kn = k + 64;
            pA = kn < nnz ? __ldg(cols + kn) : 0;
            pB = kn + 32 < nnz ? __ldg(cols + kn + 32) : pA;
          }
          float p, q;
          df_mul(ah0, al0, uh0.x, ul0.x, p, q);
          df_add(rh, rl, p, q);
          df_mul(ah0, al0, uh0.y, ul0.y, p, q);
          df_add(ih, il, p, q);
          df_mul(ah1, al1, uh1.x, ul1.x, p, q);
          df_add(rh, rl, p, q);
          df_mul(ah1, al1, uh1.y, ul1.y, p, q);
          df_add(ih, il, p, q);
        }
      }
      for (int k = real ? nnz : lane; k < nnz; k += 64) {
        // two columns per lane per step, all loads issued before the arithmetic
        const bool two = k + 32 < nnz;
        const float2 ah0 = __ldcs(vh + off + k), al0 = __ldcs(vl + off + k);
        const int cA = PF ? pA : cols[k];
        const float2 ah1 = two ? __ldcs(vh + off + k + 32) : make_float2(0.f, 0.f);
        const float2 al1 = two ? __ldcs(vl + off + k + 32) : make_float2(0.f, 0.f);
        const int cB = PF ? pB : (two ? cols[k + 32] : cA);
        const float2 uh0 = xh[cA], ul0 = xl[cA], uh1 = xh[cB], ul1 = xl[cB];
        if (PF) {
          const int kn = k + 64;
          pA = kn < nnz ? __ldg(cols + kn) : 0;
          pB = kn + 32 < nnz ? __ldg(cols + kn + 32) : pA;
        }
        float p, q;
        df_mul(ah0.x, al0.x, uh0.x, ul0.x, p, q);
        df_add(rh, rl, p, q);
        df_mul(ah0.y, al0.y, uh0.y, ul0.y, p, q);
        df_add(rh, rl, -p, -q);
        df_mul(ah0.x, al0.x, uh0.y, ul0.y, p, q);
        df_add(ih, il, p, q);
        df_mul(ah0.y, al0.y, uh0.x, ul0.x, p, q);
        df_add(ih, il, p, q);
        df_mul(ah1.x, al1.x, uh1.x, ul1.x, p, q);
        df_add(rh, rl, p, q);
        df_mul(ah1.y, al1.y, uh1.y, ul1.y, p, q);
        df_add(rh, rl, -p, -q);
        df_mul(ah1.x, al1.x, uh1.y, ul1.y, p, q);
        df_add(ih, il, p, q);
        df_mul(ah1.y, al1.y, uh1.x, ul1.x, p, q);
        df_add(ih, il, p, q);
      }
      df_warp_sum(rh, rl);
      df_warp_sum(ih, il);
      if (real && row < offU) {   // output phase i^(s_r): (re, im) -> (-im, re), exact
        const float th = rh, tl = rl;
        rh = -ih;
        rl = -il;
        ih = th;
        il = tl;
      }
    }
    if (lane == 0) res[w * (DF_ROWS / 8) + i] = make_float4(rh, rl, ih, il);
  }
  __syncthreads();
  if (w == 0) {
    const int64_t row = base + lane;
    if (row < nrows) {
      const float4 v = res[lane];
      const double re = (double)v.x + (double)v.y, im = (double)v.z + (double)v.w;
      y[row] = mode ? make_double2(b[row].x - re, b[row].y - im) : make_double2(re, im);
    }
  }
}

// The double-float CG operator with the warp's stream of (high, low, column
// index) triples prefetched SPMV_DEPTH steps ahead by cp.async (see
// k_spmv_ring).  Per lane the sums run over k = lane, lane + 32, ... in order,
// as in k_spmv_df: bitwise the same results.
__global__ void __launch_bounds__(256) k_spmv_df_ring(const int32_t* __restrict__ row_ent,
                                                      const int64_t* __restrict__ ent_start,
                                                      const int64_t* __restrict__ col_ptr,
                                                      const int32_t* __restrict__ col_idx,
                                                      const int64_t* __restrict__ val_ptr,
                                                      const float2* __restrict__ vh, const float2* __restrict__ vl,
                                                      const float2* __restrict__ xh, const float2* __restrict__ xl,
                                                      const double2* __restrict__ b, double2* __restrict__ y,
                                                      int64_t nrows, int mode) {
  __shared__ float2 sh[SPMV_DEPTH][256];
  __shared__ float2 sl[SPMV_DEPTH][256];
  __shared__ int32_t si[SPMV_DEPTH][256];
  const int lane = threadIdx.x & 31, t = threadIdx.x;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t first = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  RingRow<float2> p = ring_open<float2>(first, nrows, row_ent, ent_start, col_ptr, col_idx, val_ptr, vh);
  int ps = 0;
  while (p.row < nrows && p.steps == 0)
    p = ring_open<float2>(p.row + nw, nrows, row_ent, ent_start, col_ptr, col_idx, val_ptr, vh);
  auto issue = [&](int slot) {
    if (p.row < nrows) {
      const int k = lane + 32 * ps;
      if (k < p.nnz) {
        cp_async8(&sh[slot][t], vh + p.voff + k);
        cp_async8(&sl[slot][t], vl + p.voff + k);
        cp_async4(&si[slot][t], p.cols + k);
      }
      if (++ps >= p.steps) {
        ps = 0;
        do {
          p = ring_open<float2>(p.row + nw, nrows, row_ent, ent_start, col_ptr, col_idx, val_ptr, vh);
        } while (p.row < nrows && p.steps == 0);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < SPMV_DEPTH; ++d) issue(d);
  int slot = 0;
  for (int64_t row = first; row < nrows; row += nw) {
    const RingRow<float2> c = ring_open<float2>(row, nrows, row_ent, ent_start, col_ptr, col_idx, val_ptr, vh);
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int st = 0; st < c.steps; ++st) {
      cp_async_wait<SPMV_DEPTH - 1>();
      if (lane + 32 * st < c.nnz) {
        const float2 ah = sh[slot][t], al = sl[slot][t];
        const int col = si[slot][t];
        const float2 uh = xh[col], ul = xl[col];
        float pp, q;
        df_mul(ah.x, al.x, uh.x, ul.x, pp, q);
        df_add(rh, rl, pp, q);
        df_mul(ah.y, al.y, uh.y, ul.y, pp, q);
        df_add(rh, rl, -pp, -q);
        df_mul(ah.x, al.x, uh.y, ul.y, pp, q);
        df_add(ih, il, pp, q);
        df_mul(ah.y, al.y, uh.x, ul.x, pp, q);
        df_add(ih, il, pp, q);
      }
      issue(slot);
      slot = slot + 1 == SPMV_DEPTH ? 0 : slot + 1;
    }
    df_warp_sum(rh, rl);
    df_warp_sum(ih, il);
    if (lane == 0) {
      const double re = (double)rh + (double)rl, im = (double)ih + (double)il;
      y[row] = mode ? make_double2(b[row].x - re, b[row].y - im) : make_double2(re, im);
    }
  }
  cp_async_wait<0>();
}

// Entity-blocked double-float CG operator (same task lists as k_spmv_ent).
template <int G>
__global__ void __launch_bounds__(256) k_spmv_df_ent(const int2* __restrict__ tasks, int64_t ntasks,
                                                     const int64_t* __restrict__ ent_start,
                                                     const int32_t* __restrict__ ent_nd,
                                                     const int64_t* __restrict__ col_ptr,
                                                     const int32_t* __restrict__ col_idx,
                                                     const int64_t* __restrict__ val_ptr, const float2* __restrict__ vh,
                                                     const float2* __restrict__ vl, const float2* __restrict__ xh,
                                                     const float2* __restrict__ xl, const double2* __restrict__ b,
                                                     double2* __restrict__ y, int mode,
                                                     const uint8_t* __restrict__ rent, int64_t offU) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < ntasks; t += nw) {
    const int2 tk = tasks[t];
    const int E = tk.x, r0 = tk.y;
    const int g = min(G, ent_nd[E] - r0);
    const int64_t c0 = col_ptr[E];
    const int nnz = (int)(col_ptr[E + 1] - c0);
    const int64_t off = val_ptr[E] + (int64_t)r0 * nnz;
    const int32_t* cols = col_idx + c0;
    float rh[G], rl[G], ih[G], il[G];
#pragma unroll
    for (int r = 0; r < G; ++r) rh[r] = rl[r] = ih[r] = il[r] = 0.f;
    const bool real = rent != nullptr && rent[E] != 0;   // packed real entity (k_pack_ops)
    if (real) {
      const float* ahr = reinterpret_cast<const float*>(vh + val_ptr[E]) + (int64_t)r0 * nnz;
      const float* alr = reinterpret_cast<const float*>(vl + val_ptr[E]) + (int64_t)r0 * nnz;
      for (int k = lane; k < nnz; k += 32) {
        const int c = cols[k];
        const int sc = c < offU ? -1 : 0;
        const float2 uh = mul_i(xh[c], sc), ul = mul_i(xl[c], sc);
#pragma unroll
        for (int r = 0; r < G; ++r) {
          if (r < g) {
            const float ah = __ldcs(ahr + (int64_t)r * nnz + k), al = __ldcs(alr + (int64_t)r * nnz + k);
            float p, q;
            df_mul(ah, al, uh.x, ul.x, p, q);
            df_add(rh[r], rl[r], p, q);
            df_mul(ah, al, uh.y, ul.y, p, q);
            df_add(ih[r], il[r], p, q);
          }
        }
      }
    }
    for (int k = real ? nnz : lane; k < nnz; k += 32) {
      const int c = cols[k];
      const float2 uh = xh[c], ul = xl[c];
#pragma unroll
      for (int r = 0; r < G; ++r) {
        if (r < g) {
          const float2 ah = __ldcs(vh + off + (int64_t)r * nnz + k), al = __ldcs(vl + off + (int64_t)r * nnz + k);
          float p, q;
          df_mul(ah.x, al.x, uh.x, ul.x, p, q);
          df_add(rh[r], rl[r], p, q);
          df_mul(ah.y, al.y, uh.y, ul.y, p, q);
          df_add(rh[r], rl[r], -p, -q);
          df_mul(ah.x, al.x, uh.y, ul.y, p, q);
          df_add(ih[r], il[r], p, q);
          df_mul(ah.y, al.y, uh.x, ul.x, p, q);
          df_add(ih[r], il[r], p, q);
        }
      }
    }
    float4 mine = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < G; ++r) {
      df_warp_sum(rh[r], rl[r]);
      df_warp_sum(ih[r], il[r]);
      if (lane == r) mine = make_float4(rh[r], rl[r], ih[r], il[r]);
    }
    if (lane < g) {
      const int64_t row = ent_start[E] + r0 + lane;
      if (real && row < offU) mine = make_float4(-mine.z, -mine.w, mine.x, mine.y);   // i^(s_r), exact
      const double re = (double)mine.x + (double)mine.y, im = (double)mine.z + (double)mine.w;
      y[row] = mode ? make_double2(b[row].x - re, b[row].y - im) : make_double2(re, im);
    }
  }
}

__global__ void k_split_vec(const double2* __restrict__ x, float2* __restrict__ xh, float2* __restrict__ xl,
                            int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = x[i];
  const float hx = (float)v.x, hy = (float)v.y;
  xh[i] = make_float2(hx, hy);
  xl[i] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
}

__global__ void k_split_vals(const double2* __restrict__ v, float2* __restrict__ vh, float2* __restrict__ vl,
                             int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = v[i];
    const float hx = (float)a.x, hy = (float)a.y;
    vh[i] = make_float2(hx, hy);
    vl[i] = make_float2((float)(a.x - (double)hx), (float)(a.y - (double)hy));
  }
}

// y = A x (mode 0) or b - A x (mode 1) with the double-float operator; xh/xl scratch
static void spmv_df_g(const ECSRDev& A, const float2* xh, const float2* xl, const double2* b, double2* y, int mode,
                      int G, cudaStream_t st) {
  const int64_t n = A.nrows;
  if (A.rent && G == SPMV_RING) G = SPMV_PF;   // the ring kernel reads complex64 values only
  if (G == SPMV_RING) {
    const int64_t blocks = std::min<int64_t>((n + 7) / 8, 152 * 5);
    k_spmv_df_ring<<<(unsigned)blocks, 256, 0, st>>>(A.row_ent, A.ent_start, A.col_ptr, A.col_idx, A.val_ptr, A.v32,
                                                     A.vlo, xh, xl, b, y, n, mode);
    DPG_CHECK_LAUNCH();
    return;
  }
  if (G == SPMV_PF || G <= 1 || !A.tasks[1]) {
    const int64_t blocks = (n + DF_ROWS - 1) / DF_ROWS;
    if (G == SPMV_PF)
      k_spmv_df<true><<<(unsigned)blocks, 256, 0, st>>>(A.row_ent, A.ent_start, A.col_ptr, A.col_idx, A.val_ptr,
                                                        A.v32, A.vlo, xh, xl, b, y, n, mode, A.rent, A.offU);
    else
      k_spmv_df<false><<<(unsigned)blocks, 256, 0, st>>>(A.row_ent, A.ent_start, A.col_ptr, A.col_idx, A.val_ptr,
                                                         A.v32, A.vlo, xh, xl, b, y, n, mode, A.rent, A.offU);
    DPG_CHECK_LAUNCH();
    return;
  }
  const int gi = G == 2 ? 1 : (G == 4 ? 2 : 3);
  const int64_t nt = A.ntasks[gi];
  const unsigned blocks = (unsigned)std::min<int64_t>((nt + 7) / 8, 152 * 16);
  if (G == 2)
    k_spmv_df_ent<2><<<blocks, 256, 0, st>>>(A.tasks[gi], nt, A.ent_start, A.ent_nd, A.col_ptr, A.col_idx, A.val_ptr,
                                             A.v32, A.vlo, xh, xl, b, y, mode, A.rent, A.offU);
  else if (G == 4)
    k_spmv_df_ent<4><<<blocks, 256, 0, st>>>(A.tasks[gi], nt, A.ent_start, A.ent_nd, A.col_ptr, A.col_idx, A.val_ptr,
                                             A.v32, A.vlo, xh, xl, b, y, mode, A.rent, A.offU);
  else
    k_spmv_df_ent<8><<<blocks, 256, 0, st>>>(A.tasks[gi], nt, A.ent_start, A.ent_nd, A.col_ptr, A.col_idx, A.val_ptr,
                                             A.v32, A.vlo, xh, xl, b, y, mode, A.rent, A.offU);
  DPG_CHECK_LAUNCH();
  if (A.n_null) {
    k_null_rows<double2><<<(unsigned)((A.n_null + 255) / 256), 256, 0, st>>>(A.null_rows, A.n_null, b, y, mode);
    DPG_CHECK_LAUNCH();
  }
}

// Block form of the double-float CG operator: KB vectors (split into FP32
// pairs xh/xl at stride ld), one warp per row, each stored pair (ah, al) loaded
// once for the KB vectors.  Per vector the lane sums run over k = lane,
// lane + 32, ... in order with the error-free products and sums of k_spmv_df,
// so every column equals k_spmv_df's result.
template <int KB>
__global__ void __launch_bounds__(256) k_spmv_df_blk(const int32_t* __restrict__ row_ent,
                                                     const int64_t* __restrict__ ent_start,
                                                     const int64_t* __restrict__ col_ptr,
                                                     const int32_t* __restrict__ col_idx,
                                                     const int64_t* __restrict__ val_ptr, const float2* __restrict__ vh,
                                                     const float2* __restrict__ vl, const float2* __restrict__ xh,
                                                     const float2* __restrict__ xl, const double2* __restrict__ b,
                                                     double2* __restrict__ y, int64_t ld, int64_t nrows, int mode,
                                                     const uint8_t* __restrict__ rent, int64_t offU) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < nrows; row += nw) {
    const int32_t E = row_ent[row];
    float rh[KB], rl[KB], ih[KB], il[KB];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) rh[kb] = rl[kb] = ih[kb] = il[kb] = 0.f;
    if (E >= 0) {
      const int64_t c0 = col_ptr[E];
      const int nnz = (int)(col_ptr[E + 1] - c0);
      const int64_t off = val_ptr[E] + (row - ent_start[E]) * nnz;
      const int32_t* cols = col_idx + c0;
      int cA = lane < nnz ? __ldg(cols + lane) : 0;
      const bool real = rent != nullptr && rent[E] != 0;
      if (real) {   // packed real entity (k_pack_ops): x_c carries i^(-s_c), a = ah + al
        const float* ahr = reinterpret_cast<const float*>(vh + val_ptr[E]) + (row - ent_start[E]) * nnz;
        const float* alr = reinterpret_cast<const float*>(vl + val_ptr[E]) + (row - ent_start[E]) * nnz;
        for (int k = lane; k < nnz; k += 32) {
          const float ah = __ldcs(ahr + k), al = __ldcs(alr + k);
          const int sc = cA < offU ? -1 : 0;
          float2 uh[KB], ul[KB];
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) {
            uh[kb] = mul_i(xh[kb * ld + cA], sc);
            ul[kb] = mul_i(xl[kb * ld + cA], sc);
          }
          const int kn = k + 32;
          cA = kn < nnz ? __ldg(cols + kn) : 0;
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) {
            float p, q;
            df_mul(ah, al, uh[kb].x, ul[kb].x, p, q);
            df_add(rh[kb], rl[kb], p, q);
            df_mul(ah, al, uh[kb].y, ul[kb].y, p, q);
            df_add(ih[kb], il[kb], p, q);
          }
        }
      }
      for (int k = real ? nnz : lane; k < nnz; k += 32) {
        const float2 ah = __ldcs(vh + off + k), al = __ldcs(vl + off + k);
        float2 uh[KB], ul[KB];
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          uh[kb] = xh[kb * ld + cA];
          ul[kb] = xl[kb * ld + cA];
        }
        const int kn = k + 32;
        cA = kn < nnz ? __ldg(cols + kn) : 0;
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          float p, q;
          df_mul(ah.x, al.x, uh[kb].x, ul[kb].x, p, q);
          df_add(rh[kb], rl[kb], p, q);
          df_mul(ah.y, al.y, uh[kb].y, ul[kb].y, p, q);
          df_add(rh[kb], rl[kb], -p, -q);
          df_mul(ah.x, al.x, uh[kb].y, ul[kb].y, p, q);
          df_add(ih[kb], il[kb], p, q);
          df_mul(ah.y, al.y, uh[kb].x, ul[kb].x, p, q);
          df_add(ih[kb], il[kb], p, q);
        }
      }
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) {
        df_warp_sum(rh[kb], rl[kb]);
        df_warp_sum(ih[kb], il[kb]);
        if (real && row < offU) {   // output phase i^(s_r), exact
          const float th = rh[kb], tl = rl[kb];
          rh[kb] = -ih[kb];
          rl[kb] = -il[kb];
          ih[kb] = th;
          il[kb] = tl;
        }
      }
    }
    if (lane < KB) {
      float4 mine = make_float4(rh[0], rl[0], ih[0], il[0]);
#pragma unroll
      for (int kb = 1; kb < KB; ++kb)
        if (lane == kb) mine = make_float4(rh[kb], rl[kb], ih[kb], il[kb]);
      const int64_t i = lane * ld + row;
      const double re = (double)mine.x + (double)mine.y, im = (double)mine.z + (double)mine.w;
      y[i] = mode ? make_double2(b[i].x - re, b[i].y - im) : make_double2(re, im);
    }
  }
}

static void spmv_df(const ECSRDev& A, const double2* x, const double2* b, double2* y, int mode, float2* xh,
                    float2* xl, cudaStream_t st, SystemImpl* prof = nullptr) {
  const int64_t n = A.nrows;
  k_split_vec<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, xh, xl, n);
  DPG_CHECK_LAUNCH();
  int pe = prof_begin(prof, st);
  spmv_df_g(A, xh, xl, b, y, mode, A.gsel[2], st);
  prof_end(prof, pe, st);
}

// Complex64 values of an operator (LO: the double-float split, high parts in
// vh and low parts in vl), one CTA per row entity.  With rent, an entity whose
// entries are all real once the unit phases are taken out,
//   a[r][c] = A[r][c] i^(s_c - s_r) real (s = 1 on DOFs below offU; exact),
// is stored packed: its rows as nnz reals from float offset 2 val_ptr[E]
// (high and low parts alike), rent[E] = 1.  The SpMVs apply the phases
// exactly: y_r = i^(s_r) sum_c a[r][c] (i^(-s_c) x_c).
template <bool LO>
__global__ void k_pack_ops(const int64_t* __restrict__ ent_start, const int32_t* __restrict__ ent_nd,
                           const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ col_idx,
                           const int64_t* __restrict__ val_ptr, const double2* __restrict__ v, float2* __restrict__ vh,
                           float2* __restrict__ vl, uint8_t* __restrict__ rent, int64_t offU) {
  const int64_t E = blockIdx.x;
  const int64_t r0 = ent_start[E];
  const int64_t c0 = col_ptr[E];
  const int nnz = (int)(col_ptr[E + 1] - c0);
  const int total = ent_nd[E] * nnz;
  const int64_t vo = val_ptr[E];
  auto phase = [&](int q) {   // s_c - s_r of entry q of the entity's block
    const int64_t row = r0 + q / nnz, col = col_idx[c0 + q % nnz];
    return (col < offU ? 1 : 0) - (row < offU ? 1 : 0);
  };
  bool cplx = rent == nullptr;
  if (!cplx)
    for (int q = threadIdx.x; q < total; q += blockDim.x)
      if (mul_i(v[vo + q], phase(q)).y != 0.0) cplx = true;
  cplx = __syncthreads_or(cplx) != 0;
  if (!cplx) {
    float* h = reinterpret_cast<float*>(vh + vo);
    float* l = LO ? reinterpret_cast<float*>(vl + vo) : nullptr;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      const double a = mul_i(v[vo + q], phase(q)).x;
      const float hx = (float)a;
      h[q] = hx;
      if (LO) l[q] = (float)(a - (double)hx);
    }
  } else {
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      const double2 a = v[vo + q];
      const float hx = (float)a.x, hy = (float)a.y;
      vh[vo + q] = make_float2(hx, hy);
      if (LO) vl[vo + q] = make_float2((float)(a.x - (double)hx), (float)(a.y - (double)hy));
    }
  }
  if (threadIdx.x == 0 && rent) rent[E] = cplx ? 0 : 1;
}

// complex64 (and, with lo, double-float) values of A from A.v64; pack: real
// entities stored as reals (k_pack_ops).  Idempotent: a later call with lo
// rewrites the high parts with the same values.
static void pack_operator(Alloc& M, ECSRDev& A, bool lo, int64_t offU, bool pack, cudaStream_t st) {
  if (!A.v32) A.v32 = M.arr<float2>((size_t)std::max<int64_t>(A.nnz, 1));
  if (lo && !A.vlo) A.vlo = M.arr<float2>((size_t)std::max<int64_t>(A.nnz, 1));
  if (pack && !A.rent) A.rent = M.arr<uint8_t>((size_t)std::max<int64_t>(A.nent, 1));
  if (!pack) A.rent = nullptr;
  A.offU = offU;
  if (A.nent > 0) {
    if (lo)
      k_pack_ops<true><<<(unsigned)A.nent, 128, 0, st>>>(A.ent_start, A.ent_nd, A.col_ptr, A.col_idx, A.val_ptr,
                                                          A.v64, A.v32, A.vlo, A.rent, offU);
    else
      k_pack_ops<false><<<(unsigned)A.nent, 128, 0, st>>>(A.ent_start, A.ent_nd, A.col_ptr, A.col_idx, A.val_ptr,
                                                           A.v64, A.v32, nullptr, A.rent, offU);
    DPG_CHECK_LAUNCH();
  }
}

// entries of the packed real entities of A (host count from the device tables)
int64_t packed_entries(const ECSRDev& A) {
  if (!A.rent || A.nent == 0) return 0;
  std::vector<uint8_t> fl((size_t)A.nent);
  std::vector<int32_t> nd((size_t)A.nent);
  std::vector<int64_t> cp((size_t)A.nent + 1);
  DPG_CUDA(cudaMemcpy(fl.data(), A.rent, (size_t)A.nent, cudaMemcpyDeviceToHost));
  DPG_CUDA(cudaMemcpy(nd.data(), A.ent_nd, (size_t)A.nent * sizeof(int32_t), cudaMemcpyDeviceToHost));
  DPG_CUDA(cudaMemcpy(cp.data(), A.col_ptr, ((size_t)A.nent + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
  int64_t t = 0;
  for (int64_t E = 0; E < A.nent; ++E)
    if (fl[E]) t += (int64_t)nd[E] * (cp[E + 1] - cp[E]);
  return t;
}

void split_operator(Alloc& M, ECSRDev& A, int64_t offU, bool pack, cudaStream_t st) {
  pack_operator(M, A, true, offU, pack, st);
}

void operator_c64(Alloc& M, ECSRDev& A, int64_t offU, bool pack, cudaStream_t st) {
  pack_operator(M, A, false, offU, pack, st);
}

void split_df(const double2* v, float2* hi, float2* lo, int64_t n, cudaStream_t st) {
  k_split_vals<<<1216, 256, 0, st>>>(v, hi, lo, n);
  DPG_CHECK_LAUNCH();
}

// Double-float smoother product for the damping estimate: the patch inverses
// as complex64 high and low parts (M = Mh + Ml; LO = false: Ml = 0, the
// complex64 inverses of the mixed path's FP32 factorisation taken exactly),
// r in complex128 split into FP32 pairs in shared memory; conj(M[k][a]) r_k
// with the error-free products and sums of the CG operator.  One column per
// lane (32-column work items), warp w takes rows k = w + 8 i with two
// accumulator pairs; the 8 warp partials are combined in a fixed order and
// written in complex128.  LO = false also reads the real packed blocks of
// k_patch_apply (rflag[j] set): phase i^(-s_k) on the gathered r, real
// products, phase i^(s_a) on the output.
template <bool LO>
__global__ void __launch_bounds__(256) k_patch_apply_df(const int64_t* __restrict__ ptr, const int32_t* __restrict__ dofs,
                                                        const int64_t* __restrict__ vptr, const int2* __restrict__ chunks,
                                                        const float2* __restrict__ Mh, const float2* __restrict__ Ml,
                                                        const double2* __restrict__ r, double2* __restrict__ pbuf,
                                                        const uint8_t* __restrict__ rflag, int64_t offU) {
  extern __shared__ unsigned char shraw[];
  float4* rj = reinterpret_cast<float4*>(shraw);   // (re_hi, re_lo, im_hi, im_lo) per patch DOF
  __shared__ float4 part[8][33];
  const int2 ch = chunks[blockIdx.x];
  const int64_t j = ch.x;
  const int64_t b = ptr[j];
  const int n = (int)(ptr[j + 1] - b);
  const int64_t ld = patch_ld(n);
  const bool rp = !LO && rflag != nullptr && rflag[j] != 0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int32_t g = dofs[b + q];
    const double2 v = mul_i(r[g], rp && g < offU ? -1 : 0);
    const float hx = (float)v.x, hy = (float)v.y;
    rj[q] = make_float4(hx, (float)(v.x - (double)hx), hy, (float)(v.y - (double)hy));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int a = ch.y + lane;
  float rh0 = 0.f, rl0 = 0.f, ih0 = 0.f, il0 = 0.f, rh1 = 0.f, rl1 = 0.f, ih1 = 0.f, il1 = 0.f;
  if (a < n && rp) {
    const float* Wt = reinterpret_cast<const float*>(Mh + vptr[j]) + a;
    const int64_t ldr = patch_ldr(n);
    int k = w;
    float p, q;
    for (; k + 8 < n; k += 16) {
      const float w0 = __ldcs(Wt + (int64_t)k * ldr), w1 = __ldcs(Wt + (int64_t)(k + 8) * ldr);
      const float4 x0 = rj[k], x1 = rj[k + 8];
      df_mul(w0, 0.f, x0.x, x0.y, p, q);
      df_add(rh0, rl0, p, q);
      df_mul(w0, 0.f, x0.z, x0.w, p, q);
      df_add(ih0, il0, p, q);
      df_mul(w1, 0.f, x1.x, x1.y, p, q);
      df_add(rh1, rl1, p, q);
      df_mul(w1, 0.f, x1.z, x1.w, p, q);
      df_add(ih1, il1, p, q);
    }
    if (k < n) {
      const float w0 = __ldcs(Wt + (int64_t)k * ldr);
      const float4 x0 = rj[k];
      df_mul(w0, 0.f, x0.x, x0.y, p, q);
      df_add(rh0, rl0, p, q);
      df_mul(w0, 0.f, x0.z, x0.w, p, q);
      df_add(ih0, il0, p, q);
    }
    df_add(rh0, rl0, rh1, rl1);
    df_add(ih0, il0, ih1, il1);
  } else if (a < n) {
    const float2* H = Mh + vptr[j] + a;
    const float2* Lo = LO ? Ml + vptr[j] + a : nullptr;
    int k = w;
    float p, q;
    for (; k + 8 < n; k += 16) {
      const float2 h0 = __ldcs(H + (int64_t)k * ld), l0 = LO ? __ldcs(Lo + (int64_t)k * ld) : make_float2(0.f, 0.f);
      const float2 h1 = __ldcs(H + (int64_t)(k + 8) * ld);
      const float2 l1 = LO ? __ldcs(Lo + (int64_t)(k + 8) * ld) : make_float2(0.f, 0.f);
      const float4 x0 = rj[k], x1 = rj[k + 8];
      // conj(m) x: re = m.x x.re + m.y x.im, im = m.x x.im - m.y x.re
      df_mul(h0.x, l0.x, x0.x, x0.y, p, q);
      df_add(rh0, rl0, p, q);
      df_mul(h0.y, l0.y, x0.z, x0.w, p, q);
      df_add(rh0, rl0, p, q);
      df_mul(h0.x, l0.x, x0.z, x0.w, p, q);
      df_add(ih0, il0, p, q);
      df_mul(h0.y, l0.y, x0.x, x0.y, p, q);
      df_add(ih0, il0, -p, -q);
      df_mul(h1.x, l1.x, x1.x, x1.y, p, q);
      df_add(rh1, rl1, p, q);
      df_mul(h1.y, l1.y, x1.z, x1.w, p, q);
      df_add(rh1, rl1, p, q);
      df_mul(h1.x, l1.x, x1.z, x1.w, p, q);
      df_add(ih1, il1, p, q);
      df_mul(h1.y, l1.y, x1.x, x1.y, p, q);
      df_add(ih1, il1, -p, -q);
    }
    if (k < n) {
      const float2 h0 = __ldcs(H + (int64_t)k * ld), l0 = LO ? __ldcs(Lo + (int64_t)k * ld) : make_float2(0.f, 0.f);
      const float4 x0 = rj[k];
      df_mul(h0.x, l0.x, x0.x, x0.y, p, q);
      df_add(rh0, rl0, p, q);
      df_mul(h0.y, l0.y, x0.z, x0.w, p, q);
      df_add(rh0, rl0, p, q);
      df_mul(h0.x, l0.x, x0.z, x0.w, p, q);
      df_add(ih0, il0, p, q);
      df_mul(h0.y, l0.y, x0.x, x0.y, p, q);
      df_add(ih0, il0, -p, -q);
    }
    df_add(rh0, rl0, rh1, rl1);
    df_add(ih0, il0, ih1, il1);
  }
  part[w][lane] = make_float4(rh0, rl0, ih0, il0);
  __syncthreads();
  if (w == 0 && a < n) {
    float4 s4 = part[0][lane];
    for (int u = 1; u < 8; ++u) {
      const float4 o = part[u][lane];
      df_add(s4.x, s4.y, o.x, o.y);
      df_add(s4.z, s4.w, o.z, o.w);
    }
    const double2 o = make_double2((double)s4.x + (double)s4.y, (double)s4.z + (double)s4.w);
    pbuf[b + a] = rp ? mul_i(o, dofs[b + a] < offU ? 1 : 0) : o;
  }
}

// y = sum_j R_j^T A_jj^-1 R_j r with the double-float patch inverses (F.P.inv32 = high parts,
// plo = low parts, or null for complex64 inverses taken exactly)
static void smooth_df(const Level& F, const float2* plo, const double2* r, double2* y, double2* pbuf,
                      cudaStream_t st) {
  const PatchDev& P = F.P;
  const int64_t n = F.mesh.ndof;
  const size_t sm = (size_t)P.max_n * sizeof(float4) + 16;
  if (plo)
    k_patch_apply_df<true><<<(unsigned)P.nchunks, 256, sm, st>>>(P.ptr, P.dofs, P.val_ptr, P.chunks, P.inv32, plo, r,
                                                                  pbuf, nullptr, 0);
  else
    k_patch_apply_df<false><<<(unsigned)P.nchunks, 256, sm, st>>>(P.ptr, P.dofs, P.val_ptr, P.chunks, P.inv32,
                                                                   nullptr, r, pbuf, P.rflag, P.offU);
  DPG_CHECK_LAUNCH();
  k_slot_sum<double2, double2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P.slot_ptr, P.slots, pbuf, y, n, 1.0, 0);
  DPG_CHECK_LAUNCH();
}

void spmv64(const ECSRDev& A, const double2* x, double2* y, cudaStream_t st) {
  spmv<double2>(A, A.v64, x, nullptr, y, 0, st);
}

// ------------------------------------------------------------- smoother
// Dynamic shared memory of the half-storage product can exceed the default
// 48 KiB; the limit is set to the largest size any level needs.
static void configure_smoother_kernels() {
  const int mx = 9 * HALF_MAX_N * (int)sizeof(float2) + 16;
  DPG_CUDA(cudaFuncSetAttribute(k_patch_apply_h<float2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
}

// pbuf = per-patch products A_jj^-1 (R_j r) (full storage)
template <class C> static void patch_product(const PatchDev& P, const C* inv, const C* r, C* pbuf, cudaStream_t st);
template <>
void patch_product<float2>(const PatchDev& P, const float2* inv, const float2* r, float2* pbuf, cudaStream_t st) {
  launch_patch_apply_c64<float2>(P, P.variant, inv, r, pbuf, st);
}
template <>
void patch_product<double2>(const PatchDev& P, const double2* inv, const double2* r, double2* pbuf, cudaStream_t st) {
  const size_t sm = (size_t)P.max_n * sizeof(double2) + 16;
  int64_t nch = 0;
  const int2* chunks = patch_chunks(P, 1, &nch);
  k_patch_apply<double2, double2><<<(unsigned)nch, 256, sm, st>>>(P.ptr, P.dofs, P.val_ptr, chunks, inv, r, pbuf,
                                                                  nullptr, 0);
  DPG_CHECK_LAUNCH();
}

template <class C>
static void smooth(const Level& L, const C* r, C* y, double theta, int accumulate, C* pbuf, cudaStream_t st,
                   SystemImpl* prof = nullptr) {
  const PatchDev& P = L.P;
  const int64_t n = L.mesh.ndof;
  if (P.half && Prec<C>::half(P)) {
    const size_t sm = (size_t)9 * P.max_n * sizeof(C) + 16;
    int pe = prof_begin(prof, st);
    k_patch_apply_h<C, C><<<(unsigned)P.np, 256, sm, st>>>(P.ptr, P.dofs, P.hptr, Prec<C>::half(P), r, pbuf);
    DPG_CHECK_LAUNCH();
    prof_end(prof, pe, st);
    k_slot_sum<C, C><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P.slot_ptr, P.slots, pbuf, y, n, theta, accumulate);
    DPG_CHECK_LAUNCH();
    return;
  }
  int pe = prof_begin(prof, st);
  if constexpr (std::is_same<C, float2>::value) {
    if (P.recompute) patch_recompute_apply(L, r, pbuf, st);
    else patch_product<C>(P, Prec<C>::inv(P), r, pbuf, st);
  } else {
    patch_product<C>(P, Prec<C>::inv(P), r, pbuf, st);
  }
  prof_end(prof, pe, st);
  k_slot_sum<C, C><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P.slot_ptr, P.slots, pbuf, y, n, theta, accumulate);
  DPG_CHECK_LAUNCH();
}

void smooth_apply64(const Level& L, const double2* r, double2* y, double theta, double2* scratch, cudaStream_t st) {
  smooth<double2>(L, r, y, theta, 0, scratch, st);
}

// ------------------------------------------------------------- transfers
template <class C>
__global__ void k_condense_apply(int nS, int nI, const int64_t* __restrict__ Ig, const C* __restrict__ Y,
                                 const C* __restrict__ r, C* __restrict__ cbuf) {
  extern __shared__ unsigned char shraw[];
  C* rI = reinterpret_cast<C*>(shraw);
  const int64_t K = blockIdx.x;
  for (int i = threadIdx.x; i < nI; i += blockDim.x) rI[i] = r[Ig[K * nI + i]];
  __syncthreads();
  const C* YK = Y + K * (size_t)nI * nS;
  for (int a = threadIdx.x; a < nS; a += blockDim.x) {
    C acc = Ops<C>::zero();
    for (int i = 0; i < nI; ++i) acc = Ops<C>::fmac(rI[i], YK[(size_t)i * nS + a], acc);   // conj(Y[i][a]) r_I[i]
    cbuf[K * nS + a] = acc;
  }
}

// rs[g] = smask[g] ? r[g] - sum_{slots} cbuf[slot] : 0
template <class C>
__global__ void k_condense_sum(const int64_t* __restrict__ sptr, const int32_t* __restrict__ slots,
                               const C* __restrict__ cbuf, const char* __restrict__ smask, const C* __restrict__ r,
                               C* __restrict__ rs, int64_t n) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  if (!smask[g]) { rs[g] = Ops<C>::zero(); return; }
  C acc = r[g];
  for (int64_t s = sptr[g]; s < sptr[g + 1]; ++s) acc = Ops<C>::sub(acc, cbuf[slots[s]]);
  rs[g] = acc;
}

// x_I = A_II^-1 r_I - Y x_S, one CTA per coarse element, one warp per row
template <class C>
__global__ void k_backsub(int nS, int nI, const int64_t* __restrict__ Sg, const int64_t* __restrict__ Ig,
                          const C* __restrict__ Ai, const C* __restrict__ Y, const C* __restrict__ r,
                          C* __restrict__ x) {
  extern __shared__ unsigned char shraw[];
  C* rI = reinterpret_cast<C*>(shraw);
  C* xS = rI + nI;
  using O = Ops<C>;
  const int64_t K = blockIdx.x;
  for (int i = threadIdx.x; i < nI; i += blockDim.x) rI[i] = r[Ig[K * nI + i]];
  for (int a = threadIdx.x; a < nS; a += blockDim.x) {
    int64_t g = Sg[K * nS + a];
    xS[a] = g >= 0 ? x[g] : O::zero();
  }
  __syncthreads();
  const C* AiK = Ai + K * (size_t)nI * nI;
  const C* YK = Y + K * (size_t)nI * nS;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = w; i < nI; i += blockDim.x >> 5) {
    C acc = O::zero();
    for (int k = lane; k < nI; k += 32) acc = O::fma(AiK[(size_t)i * nI + k], rI[k], acc);
    for (int a = lane; a < nS; a += 32) acc = O::fnma(YK[(size_t)i * nS + a], xS[a], acc);
    acc = warp_sum(acc);
    if (lane == 0) x[Ig[K * nI + i]] = acc;
  }
}

// y[i] (+)= sum_k val[k] x[col[k]] with real values (natural inclusion)
template <class C>
__global__ void k_csr_real(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const C* __restrict__ x, C* __restrict__ y, int64_t n,
                           int accumulate) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  using R = typename Ops<C>::R;
  C acc = Ops<C>::zero();
  for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
    R v = (R)val[k];
    C xv = x[col[k]];
    acc.x += v * xv.x;
    acc.y += v * xv.y;
  }
  y[i] = accumulate ? Ops<C>::add(y[i], acc) : acc;
}

template <class C>
__global__ void k_gather(const int32_t* __restrict__ idx, const C* __restrict__ x, C* __restrict__ y, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[idx[i]];
}
template <class C>
__global__ void k_scatter_add(const int32_t* __restrict__ idx, const C* __restrict__ x, C* __restrict__ y, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[idx[i]] = Ops<C>::add(y[idx[i]], x[i]);
}

// ------------------------------------------------------------- vector ops
template <class C>
__global__ void k_zero(C* y, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = Ops<C>::zero();
}
__global__ void k_narrow(const double2* a, float2* b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void k_widen(const float2* a, double2* b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_double2(a[i].x, a[i].y);
}

constexpr int RED_BLOCKS = 608;

// scalar slots of the CG state
enum { SC_RHO = 0, SC_PQ, SC_ALPHA, SC_BETA, SC_RR, SC_RHONEW, SC_COUNT };

// which: 0 -> PQ then ALPHA = RHO / PQ ; 1 -> RR ; 2 -> RHONEW, BETA, RHO ; 3 -> RHO
// (one block of 256 threads; the partials are read from L2: other SMs wrote them)
__device__ void block_finish(const double2* part, int nparts, double2* sc, int which) {
  __shared__ double2 sh[256];
  double2 acc = make_double2(0, 0);
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) acc = Ops<double2>::add(acc, __ldcg(part + k));
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = Ops<double2>::add(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double2 d = sh[0];
  if (which == 0) {
    sc[SC_PQ] = d;
    double2 rho = sc[SC_RHO];
    double den = d.x * d.x + d.y * d.y;
    sc[SC_ALPHA] = make_double2((rho.x * d.x + rho.y * d.y) / den, (rho.y * d.x - rho.x * d.y) / den);
  } else if (which == 1) {
    sc[SC_RR] = d;
  } else if (which == 2) {
    double2 rho = sc[SC_RHO];
    double den = rho.x * rho.x + rho.y * rho.y;
    sc[SC_BETA] = make_double2((d.x * rho.x + d.y * rho.y) / den, (d.y * rho.x - d.x * rho.y) / den);
    sc[SC_RHONEW] = d;
    sc[SC_RHO] = d;
  } else {
    sc[SC_RHO] = d;
  }
}

__global__ void k_dot_finish(const double2* part, int nparts, double2* sc, int which) {
  block_finish(part, nparts, sc, which);
}

// After thread 0 of every block has written its partial: true in the last
// block to arrive (ticket = gridDim.x - 1), which then finishes the reduction
// (block_finish, the same order as k_dot_finish) and resets the ticket for the
// next reduction.  No block waits for another.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    __threadfence();   // this block's partial is visible before its ticket
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

__device__ __forceinline__ double2 to_c128(double2 a) { return a; }
__device__ __forceinline__ double2 to_c128(float2 a) { return make_double2(a.x, a.y); }   // exact

// sum conj(u_i) v_i in FP64 (u complex128, or complex64 widened exactly): block
// partials, finished by the last block
template <class TU>
__global__ void k_dot_fused(const TU* __restrict__ u, const double2* __restrict__ v, int64_t n,
                            double2* __restrict__ part, double2* sc, int which, unsigned* ticket) {
  __shared__ double2 sh[8];
  double2 acc = make_double2(0, 0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = Ops<double2>::fmac(v[i], to_c128(u[i]), acc);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0, 0);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s = Ops<double2>::add(s, sh[k]);
    part[blockIdx.x] = s;
  }
  if (!last_block(ticket)) return;
  block_finish(part, gridDim.x, sc, which);
  if (threadIdx.x == 0) *ticket = 0u;
}

// x += alpha p ; r -= alpha q ; ||r||^2 from block partials, finished by the last block (into sc[SC_RR]);
// r32 (may be null): complex64 copy of the new r for the mixed V-cycle
__global__ void k_cg_update_fused(double2* __restrict__ x, double2* __restrict__ r, const double2* __restrict__ p,
                                  const double2* __restrict__ q, double2* sc, int64_t n, double2* __restrict__ part,
                                  unsigned* ticket, float2* __restrict__ r32) {
  __shared__ double2 sh[8];
  const double2 al = sc[SC_ALPHA];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 pi = p[i], qi = q[i], xi = x[i], ri = r[i];
    xi.x += al.x * pi.x - al.y * pi.y;
    xi.y += al.x * pi.y + al.y * pi.x;
    ri.x -= al.x * qi.x - al.y * qi.y;
    ri.y -= al.x * qi.y + al.y * qi.x;
    x[i] = xi;
    r[i] = ri;
    if (r32) r32[i] = make_float2((float)ri.x, (float)ri.y);
    acc += ri.x * ri.x + ri.y * ri.y;
  }
  double2 a2 = warp_sum(make_double2(acc, 0.0));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0, 0);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s = Ops<double2>::add(s, sh[k]);
    part[blockIdx.x] = s;
  }
  if (!last_block(ticket)) return;
  block_finish(part, gridDim.x, sc, 1);
  if (threadIdx.x == 0) *ticket = 0u;
}

// p = z + beta p, and p's double-float split (hi, lo) for the CG operator (z complex128, or
// the mixed V-cycle's complex64 output widened exactly)
template <class TZ>
__global__ void k_cg_dir(double2* __restrict__ p, const TZ* __restrict__ z, const double2* __restrict__ sc,
                         int64_t n, float2* __restrict__ ph, float2* __restrict__ pl) {
  const double2 be = sc[SC_BETA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 pi = p[i], zi = to_c128(z[i]);
    const double2 v = make_double2(zi.x + be.x * pi.x - be.y * pi.y, zi.y + be.x * pi.y + be.y * pi.x);
    p[i] = v;
    const float hx = (float)v.x, hy = (float)v.y;
    ph[i] = make_float2(hx, hy);
    pl[i] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
  }
}

// Block forms of the fused CG kernels for K columns (blockIdx.y = column k;
// vectors at stride n; column k's scalars at sc + k SC_COUNT, its partials at
// part + k RED_BLOCKS and its ticket at ticket[k]).  Columns whose bit in
// `active` is clear return at once (all their blocks alike).
template <class TU>
__global__ void k_dot_fused_blk(const TU* __restrict__ u, const double2* __restrict__ v, int64_t n,
                                double2* __restrict__ part, double2* sc, int which, unsigned* ticket,
                                unsigned long long active) {
  const int k = blockIdx.y;
  if (!((active >> k) & 1ull)) return;
  u += (int64_t)k * n;
  v += (int64_t)k * n;
  part += (int64_t)k * RED_BLOCKS;
  sc += (int64_t)k * SC_COUNT;
  __shared__ double2 sh[8];
  double2 acc = make_double2(0, 0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = Ops<double2>::fmac(v[i], to_c128(u[i]), acc);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0, 0);
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s = Ops<double2>::add(s, sh[q]);
    part[blockIdx.x] = s;
  }
  if (!last_block(ticket + k)) return;
  block_finish(part, gridDim.x, sc, which);
  if (threadIdx.x == 0) ticket[k] = 0u;
}

__global__ void k_cg_update_fused_blk(double2* __restrict__ x, double2* __restrict__ r, const double2* __restrict__ p,
                                      const double2* __restrict__ q, double2* sc, int64_t n, double2* __restrict__ part,
                                      unsigned* ticket, unsigned long long active) {
  const int k = blockIdx.y;
  if (!((active >> k) & 1ull)) return;
  const int64_t o = (int64_t)k * n;
  x += o;
  r += o;
  p += o;
  q += o;
  sc += (int64_t)k * SC_COUNT;
  part += (int64_t)k * RED_BLOCKS;
  __shared__ double2 sh[8];
  const double2 al = sc[SC_ALPHA];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 pi = p[i], qi = q[i], xi = x[i], ri = r[i];
    xi.x += al.x * pi.x - al.y * pi.y;
    xi.y += al.x * pi.y + al.y * pi.x;
    ri.x -= al.x * qi.x - al.y * qi.y;
    ri.y -= al.x * qi.y + al.y * qi.x;
    x[i] = xi;
    r[i] = ri;
    acc += ri.x * ri.x + ri.y * ri.y;
  }
  double2 a2 = warp_sum(make_double2(acc, 0.0));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0, 0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = Ops<double2>::add(s, sh[w]);
    part[blockIdx.x] = s;
  }
  if (!last_block(ticket + k)) return;
  block_finish(part, gridDim.x, sc, 1);
  if (threadIdx.x == 0) ticket[k] = 0u;
}

__global__ void k_cg_dir_blk(double2* __restrict__ p, const double2* __restrict__ z, const double2* __restrict__ sc,
                             int64_t n, unsigned long long active) {
  const int k = blockIdx.y;
  if (!((active >> k) & 1ull)) return;
  p += (int64_t)k * n;
  z += (int64_t)k * n;
  const double2 be = sc[(int64_t)k * SC_COUNT + SC_BETA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 pi = p[i], zi = z[i];
    p[i] = make_double2(zi.x + be.x * pi.x - be.y * pi.y, zi.y + be.x * pi.y + be.y * pi.x);
  }
}

// ------------------------------------------------------------ workspace
template <class C> struct LevelWS {
  C *r = nullptr, *rs = nullptr, *x = nullptr, *t = nullptr, *pbuf = nullptr, *cbuf = nullptr;
};

struct WS {
  Alloc mem;
  std::vector<LevelWS<double2>> w64;
  std::vector<LevelWS<float2>> w32;
  double2 *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *part = nullptr, *sc = nullptr;
  unsigned* ticket = nullptr;              // last-block counter of the fused reductions (0 between them)
  float2 *xh = nullptr, *xl = nullptr;     // double-float split of the CG operand
  double2* sc_host = nullptr;    // pinned scalar read-back (a few bytes per CG step)
  ECSRDev Acg;                   // the CG operator (finest A_L, FP64)
  bool acg_owned = false;
};

template <class C> static std::vector<LevelWS<C>>& wsv(WS& w);
template <> std::vector<LevelWS<double2>>& wsv<double2>(WS& w) { return w.w64; }
template <> std::vector<LevelWS<float2>>& wsv<float2>(WS& w) { return w.w32; }

template <class C>
static void alloc_level_ws(WS& W, SystemImpl& S) {
  auto& v = wsv<C>(W);
  v.resize(S.levels.size());
  for (size_t l = 0; l < S.levels.size(); ++l) {
    const Level& L = S.levels[l];
    int64_t n = L.mesh.ndof;
    v[l].r = S.mem.arr<C>((size_t)n);
    v[l].rs = S.mem.arr<C>((size_t)n);
    v[l].x = S.mem.arr<C>((size_t)n);
    v[l].t = S.mem.arr<C>((size_t)n);
    if (l >= 1 || L.P.np > 0) v[l].pbuf = S.mem.arr<C>((size_t)std::max<int64_t>(L.P.scratch_entries(), 1));
    if (L.kind == 2) v[l].cbuf = S.mem.arr<C>((size_t)L.nK * L.nS);
  }
}

void ensure_workspace(SystemImpl& S, cudaStream_t st) {
  if (S.ws) return;
  configure_smoother_kernels();
  WS* W = new WS();
  S.ws = W;
  const Level& F = S.levels.back();
  const int64_t n = F.mesh.ndof;
  W->x = S.mem.arr<double2>((size_t)n);
  W->r = S.mem.arr<double2>((size_t)n);
  W->p = S.mem.arr<double2>((size_t)n);
  W->q = S.mem.arr<double2>((size_t)n);
  W->z = S.mem.arr<double2>((size_t)n);
  W->part = S.mem.arr<double2>(RED_BLOCKS);
  W->xh = S.mem.arr<float2>((size_t)n);
  W->xl = S.mem.arr<float2>((size_t)n);
  W->sc = S.mem.arr<double2>(SC_COUNT);
  W->ticket = S.mem.arr<unsigned>(1);
  DPG_CUDA(cudaMemsetAsync(W->ticket, 0, sizeof(unsigned), st));
  DPG_CUDA(cudaMallocHost(&W->sc_host, SC_COUNT * sizeof(double2)));
  alloc_level_ws<double2>(*W, S);
  if (S.op.precision == DPGMG_PREC_MIXED) alloc_level_ws<float2>(*W, S);
  DPG_CUDA(cudaStreamSynchronize(st));
}

void free_workspace(SystemImpl& S) {
  if (!S.ws) return;
  WS* W = reinterpret_cast<WS*>(S.ws);
  if (W->sc_host) cudaFreeHost(W->sc_host);
  delete W;
  S.ws = nullptr;
}

template <class C> static void coarse_solve(SystemImpl& S, WS& W, const C* r, C* e, cudaStream_t st);
template <> void coarse_solve<double2>(SystemImpl& S, WS& W, const double2* r, double2* e, cudaStream_t st) {
  coarse_apply64(S.levels[0], r, e, W.w64[0].t, st);
}
template <> void coarse_solve<float2>(SystemImpl& S, WS& W, const float2* r, float2* e, cudaStream_t st) {
  coarse_apply32(S.levels[0], r, e, W.w32[0].t, st);
}

// -------------------------------------------------------------- V-cycle
static inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

template <class C>
static void restrict_vec(const Level& F, const Level& Cl, const C* r1, C* rc, cudaStream_t st) {
  if (F.kind == 1) {
    k_gather<C><<<nblk(Cl.mesh.ndof), 256, 0, st>>>(F.inj, r1, rc, Cl.mesh.ndof);
  } else {
    k_csr_real<C><<<nblk(Cl.mesh.ndof), 256, 0, st>>>(F.PT_ptr, F.PT_col, F.PT_val, r1, rc, Cl.mesh.ndof, 0);
  }
  DPG_CHECK_LAUNCH();
}

template <class C>
static void prolong_add(const Level& F, const Level& Cl, const C* ec, C* x, cudaStream_t st) {
  if (F.kind == 1) {
    k_scatter_add<C><<<nblk(Cl.mesh.ndof), 256, 0, st>>>(F.inj, ec, x, Cl.mesh.ndof);
  } else {
    k_csr_real<C><<<nblk(F.mesh.ndof), 256, 0, st>>>(F.P_ptr, F.P_col, F.P_val, ec, x, F.mesh.ndof, 1);
  }
  DPG_CHECK_LAUNCH();
}

template <class C>
static void condense(const Level& F, const C* r, C* rs, C* cbuf, cudaStream_t st) {
  size_t sm = (size_t)F.nI * sizeof(C) + 16;
  k_condense_apply<C><<<(unsigned)F.nK, 256, sm, st>>>(F.nS, F.nI, F.I_glob, Prec<C>::Y(F), r, cbuf);
  DPG_CHECK_LAUNCH();
  k_condense_sum<C><<<nblk(F.mesh.ndof), 256, 0, st>>>(F.sslot_ptr, F.sslots, cbuf, F.smask, r, rs, F.mesh.ndof);
  DPG_CHECK_LAUNCH();
}

template <class C>
static void backsub(const Level& F, const C* r, C* x, cudaStream_t st) {
  size_t sm = (size_t)(F.nI + F.nS) * sizeof(C) + 16;
  k_backsub<C><<<(unsigned)F.nK, 256, sm, st>>>(F.nS, F.nI, F.S_glob, F.I_glob, Prec<C>::Ai(F), Prec<C>::Y(F), r, x);
  DPG_CHECK_LAUNCH();
}

// x = B_l r (r is not modified)
template <class C>
static void vcycle(SystemImpl& S, WS& W, int l, const C* r, C* x, cudaStream_t st) {
  auto& V = wsv<C>(W);
  const Level& F = S.levels[l];
  const int64_t n = F.mesh.ndof;
  if (l == 0) {
    if (F.has_coarse) coarse_solve<C>(S, W, r, x, st);
    else if (F.P.np > 0) smooth<C>(F, r, x, F.theta, 0, V[0].pbuf, st);   // DPGMG_COARSEST_SMOOTH
    else {
      k_zero<C><<<nblk(n), 256, 0, st>>>(x, n);
      DPG_CHECK_LAUNCH();
    }
    return;
  }
  const Level& Cl = S.levels[l - 1];
  const C* Avals = Prec<C>::A(F.A);
  const C* rs = r;
  const bool fine = l == (int)S.levels.size() - 1;
  SystemImpl* psm = (fine && S.prof_which == DPGMG_PROF_SMOOTH_FINE) ? &S : nullptr;
  SystemImpl* psp = (fine && S.prof_which == DPGMG_PROF_SPMV_FINE) ? &S : nullptr;
  if (F.kind == 2) {
    condense<C>(F, r, V[l].rs, V[l].cbuf, st);
    rs = V[l].rs;
  }
  // pre-smoothing from x = 0
  for (int k = 0; k < S.op.nu_pre; ++k) {
    if (k == 0) {
      smooth<C>(F, rs, x, F.theta, 0, V[l].pbuf, st, psm);
    } else {
      spmv<C>(F.A, Avals, x, rs, V[l].t, 1, st, psp);
      smooth<C>(F, V[l].t, x, F.theta, 1, V[l].pbuf, st, psm);
    }
  }
  if (S.op.nu_pre == 0) {
    k_zero<C><<<nblk(n), 256, 0, st>>>(x, n);
    DPG_CHECK_LAUNCH();
  }
  // coarse-grid correction
  spmv<C>(F.A, Avals, x, rs, V[l].t, 1, st, psp);
  restrict_vec<C>(F, Cl, V[l].t, V[l - 1].r, st);
  vcycle<C>(S, W, l - 1, V[l - 1].r, V[l - 1].x, st);
  prolong_add<C>(F, Cl, V[l - 1].x, x, st);
  for (int k = 0; k < S.op.nu_post; ++k) {
    spmv<C>(F.A, Avals, x, rs, V[l].t, 1, st, psp);
    smooth<C>(F, V[l].t, x, F.theta, 1, V[l].pbuf, st, psm);
  }
  if (F.kind == 2) backsub<C>(F, r, x, st);
}

// z = B r on the finest level in the V-cycle precision
// Mixed path: narrowed = r's complex64 copy is already in the finest level's
// V-cycle input (written by the CG update); z = null leaves the result in
// complex64 (the V-cycle's output buffer) for consumers that widen it on load.
static void precondition(SystemImpl& S, WS& W, const double2* r, double2* z, cudaStream_t st, bool narrowed = false) {
  const int L = (int)S.levels.size() - 1;
  const int64_t n = S.levels[L].mesh.ndof;
  if (S.op.precision == DPGMG_PREC_MIXED) {
    auto& V = W.w32;
    if (!narrowed) {
      k_narrow<<<nblk(n), 256, 0, st>>>(r, V[L].r, n);
      DPG_CHECK_LAUNCH();
    }
    vcycle<float2>(S, W, L, V[L].r, V[L].x, st);
    if (z) {
      k_widen<<<nblk(n), 256, 0, st>>>(V[L].x, z, n);
      DPG_CHECK_LAUNCH();
    }
  } else {
    vcycle<double2>(S, W, L, r, z, st);
  }
}

// ------------------------------------------------------ block V-cycle
// K right-hand sides stored one after another (stride = the level's DOF
// count).  The smoother and the SpMV stream their matrices once per group of
// up to BLK_MAX vectors; the transfers, condensation, back-substitution and
// the coarsest solve run per vector (their matrices are small or cached).
template <class C> struct BlockLevel {
  C *r = nullptr, *rs = nullptr, *x = nullptr, *t = nullptr, *pbuf = nullptr, *cbuf = nullptr;
};

template <class C, int KB>
static void patch_apply_blk_launch(const PatchDev& P, int per, const C* inv, const C* r, int64_t ldr, C* pbuf,
                                   int64_t ldp, cudaStream_t st) {
  const size_t sm = (size_t)KB * P.max_n * sizeof(C) + 16;
  int64_t nch = 0;
  const int2* chunks = patch_chunks(P, per, &nch);
  const uint8_t* rflag = std::is_same<C, float2>::value ? P.rflag : nullptr;   // packed complex64 inverses only
  if (per == 2)
    k_patch_apply_blk<C, C, 2, KB><<<(unsigned)nch, 256, sm, st>>>(P.ptr, P.dofs, P.val_ptr, chunks, inv, r, ldr,
                                                                   pbuf, ldp, rflag, P.offU);
  else
    k_patch_apply_blk<C, C, 1, KB><<<(unsigned)nch, 256, sm, st>>>(P.ptr, P.dofs, P.val_ptr, chunks, inv, r, ldr,
                                                                   pbuf, ldp, rflag, P.offU);
  DPG_CHECK_LAUNCH();
}

// dynamic shared memory of the block products: the gathered right-hand sides
// of one group (vectors x patch size), up to BLK_SMEM bytes
constexpr int BLK_SMEM = 160 * 1024;   // + up to 37 KiB of static shared memory (the smoother ring)
static void configure_block_kernels() {
  static std::once_flag once;
  std::call_once(once, []() {
    const int mx = BLK_SMEM;
#define DPG_BLK_ATTR(C, PER, KB)                                                                        \
  DPG_CUDA(cudaFuncSetAttribute(k_patch_apply_blk<C, C, PER, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))
    DPG_BLK_ATTR(float2, 1, 1); DPG_BLK_ATTR(float2, 1, 2); DPG_BLK_ATTR(float2, 1, 3); DPG_BLK_ATTR(float2, 1, 4);
    DPG_BLK_ATTR(float2, 2, 1); DPG_BLK_ATTR(float2, 2, 2); DPG_BLK_ATTR(float2, 2, 3); DPG_BLK_ATTR(float2, 2, 4);
    DPG_BLK_ATTR(double2, 1, 1); DPG_BLK_ATTR(double2, 1, 2); DPG_BLK_ATTR(double2, 1, 3);
    DPG_BLK_ATTR(double2, 1, 4);
#undef DPG_BLK_ATTR
#define DPG_BLK_ATTR2(K, C, KB) DPG_CUDA(cudaFuncSetAttribute(K<C, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))
    DPG_BLK_ATTR2(k_condense_apply_blk, float2, 1); DPG_BLK_ATTR2(k_condense_apply_blk, float2, 2);
    DPG_BLK_ATTR2(k_condense_apply_blk, float2, 3); DPG_BLK_ATTR2(k_condense_apply_blk, float2, 4);
    DPG_BLK_ATTR2(k_condense_apply_blk, double2, 1); DPG_BLK_ATTR2(k_condense_apply_blk, double2, 2);
    DPG_BLK_ATTR2(k_condense_apply_blk, double2, 3); DPG_BLK_ATTR2(k_condense_apply_blk, double2, 4);
    DPG_BLK_ATTR2(k_backsub_blk, float2, 1); DPG_BLK_ATTR2(k_backsub_blk, float2, 2);
    DPG_BLK_ATTR2(k_backsub_blk, float2, 3); DPG_BLK_ATTR2(k_backsub_blk, float2, 4);
    DPG_BLK_ATTR2(k_backsub_blk, double2, 1); DPG_BLK_ATTR2(k_backsub_blk, double2, 2);
    DPG_BLK_ATTR2(k_backsub_blk, double2, 3); DPG_BLK_ATTR2(k_backsub_blk, double2, 4);
#undef DPG_BLK_ATTR2
  });
}

// y_k = (accumulate ? y_k : 0) + theta S r_k for k < K
template <class C>
static void smooth_blk(const Level& L, const C* r, C* y, double theta, int accumulate, C* pbuf, int K,
                       cudaStream_t st) {
  const PatchDev& P = L.P;
  const int64_t n = L.mesh.ndof, ldp = std::max<int64_t>(P.scratch_entries(), 1);
  const C* inv = Prec<C>::inv(P);
  const int64_t cap = std::min<int64_t>(BLK_MAX, (BLK_SMEM - 16) / ((int64_t)P.max_n * sizeof(C) + 1));
  if constexpr (std::is_same<C, float2>::value) {
    if (P.recompute && cap == BLK_MAX) {
      configure_block_kernels();
      patch_recompute_apply_blk(L, r, n, pbuf, ldp, K, st);
      k_slot_sum_blk<C><<<dim3(nblk(n), (unsigned)K), 256, 0, st>>>(P.slot_ptr, P.slots, pbuf, ldp, y, n, n, theta,
                                                                     accumulate);
      DPG_CHECK_LAUNCH();
      return;
    }
  }
  if (!inv || cap < 1) {
    for (int k = 0; k < K; ++k) smooth<C>(L, r + k * n, y + k * n, theta, accumulate, pbuf + k * ldp, st);
    return;
  }
  configure_block_kernels();
  const int per = std::is_same<C, float2>::value ? P.cols : 1;
  for (int g = 0; g < K; g += (int)cap) {
    const int kb = (int)std::min<int64_t>(cap, K - g);
    const C* rg = r + g * n;
    C* pg = pbuf + g * ldp;
    if (kb == 4) patch_apply_blk_launch<C, 4>(P, per, inv, rg, n, pg, ldp, st);
    else if (kb == 3) patch_apply_blk_launch<C, 3>(P, per, inv, rg, n, pg, ldp, st);
    else if (kb == 2) patch_apply_blk_launch<C, 2>(P, per, inv, rg, n, pg, ldp, st);
    else patch_apply_blk_launch<C, 1>(P, per, inv, rg, n, pg, ldp, st);
  }
  k_slot_sum_blk<C><<<dim3(nblk(n), (unsigned)K), 256, 0, st>>>(P.slot_ptr, P.slots, pbuf, ldp, y, n, n, theta,
                                                                 accumulate);
  DPG_CHECK_LAUNCH();
}

// One row per warp (the entity-grouped form measured slower: fewer loads in
// flight at its register count).
template <class C>
static void spmv_blk(const ECSRDev& A, const C* vals, const C* x, const C* b, C* y, int mode, int K,
                     cudaStream_t st) {
  const int64_t n = A.nrows;
  for (int g = 0; g < K; g += BLK_MAX) {
    const int kb = std::min(BLK_MAX, K - g);
    const C* xg = x + g * n;
    const C* bg = b ? b + g * n : nullptr;
    C* yg = y + g * n;
    const unsigned blocks = (unsigned)std::min<int64_t>((A.nrows + 7) / 8, 152 * 16);
#define DPG_SPMV_BLK(KB)                                                                                            \
  k_spmv_blk<C, KB><<<blocks, 256, 0, st>>>(A.row_ent, A.ent_start, A.col_ptr, A.col_idx, A.val_ptr, vals, xg, bg, yg, \
                                            n, A.nrows, mode, packed_rows<C>(A), A.offU)
    if (kb == 4) DPG_SPMV_BLK(4);
    else if (kb == 3) DPG_SPMV_BLK(3);
    else if (kb == 2) DPG_SPMV_BLK(2);
    else DPG_SPMV_BLK(1);
#undef DPG_SPMV_BLK
    DPG_CHECK_LAUNCH();
  }
}

// vectors per launch of a block kernel whose shared memory holds `per_vec`
// values of C per vector (0: not even one vector fits)
template <class C> static int blk_group(int64_t per_vec) {
  return (int)std::min<int64_t>(BLK_MAX, (BLK_SMEM - 16) / (per_vec * (int64_t)sizeof(C) + 1));
}

// rs_k = r_k with the macro-interior residual condensed (h levels), k < K
template <class C>
static void condense_blk(const Level& F, const C* r, C* rs, C* cbuf, int K, cudaStream_t st) {
  const int64_t n = F.mesh.ndof, ldc = (int64_t)F.nK * F.nS;
  const int cap = blk_group<C>(F.nI);
  if (cap < 1) {
    for (int k = 0; k < K; ++k) condense<C>(F, r + k * n, rs + k * n, cbuf, st);
    return;
  }
  configure_block_kernels();
  for (int g = 0; g < K; g += cap) {
    const int kb = std::min(cap, K - g);
    const size_t sm = (size_t)kb * F.nI * sizeof(C) + 16;
#define DPG_COND_BLK(KB)                                                                                   \
  k_condense_apply_blk<C, KB><<<(unsigned)F.nK, 256, sm, st>>>(F.nS, F.nI, F.I_glob, Prec<C>::Y(F), r + g * n, n, \
                                                               cbuf + g * ldc, ldc)
    if (kb == 4) DPG_COND_BLK(4);
    else if (kb == 3) DPG_COND_BLK(3);
    else if (kb == 2) DPG_COND_BLK(2);
    else DPG_COND_BLK(1);
#undef DPG_COND_BLK
    DPG_CHECK_LAUNCH();
  }
  for (int k = 0; k < K; ++k) {
    k_condense_sum<C><<<nblk(n), 256, 0, st>>>(F.sslot_ptr, F.sslots, cbuf + k * ldc, F.smask, r + k * n, rs + k * n,
                                               n);
    DPG_CHECK_LAUNCH();
  }
}

template <class C>
static void backsub_blk(const Level& F, const C* r, C* x, int K, cudaStream_t st) {
  const int64_t n = F.mesh.ndof;
  const int cap = blk_group<C>((int64_t)F.nI + F.nS);
  if (cap < 1) {
    for (int k = 0; k < K; ++k) backsub<C>(F, r + k * n, x + k * n, st);
    return;
  }
  configure_block_kernels();
  for (int g = 0; g < K; g += cap) {
    const int kb = std::min(cap, K - g);
    const size_t sm = (size_t)kb * (F.nI + F.nS) * sizeof(C) + 16;
#define DPG_BACK_BLK(KB)                                                                                       \
  k_backsub_blk<C, KB><<<(unsigned)F.nK, 256, sm, st>>>(F.nS, F.nI, F.S_glob, F.I_glob, Prec<C>::Ai(F), Prec<C>::Y(F), \
                                                        r + g * n, x + g * n, n)
    if (kb == 4) DPG_BACK_BLK(4);
    else if (kb == 3) DPG_BACK_BLK(3);
    else if (kb == 2) DPG_BACK_BLK(2);
    else DPG_BACK_BLK(1);
#undef DPG_BACK_BLK
    DPG_CHECK_LAUNCH();
  }
}

template <class C> static void coarse_solve_blk(const Level& C0, const C* r, C* e, C* tmp, int K, cudaStream_t st);
template <>
void coarse_solve_blk<double2>(const Level& C0, const double2* r, double2* e, double2* tmp, int K, cudaStream_t st) {
  coarse_apply64_blk(C0, r, e, tmp, K, st);
}
template <>
void coarse_solve_blk<float2>(const Level& C0, const float2* r, float2* e, float2* tmp, int K, cudaStream_t st) {
  coarse_apply32_blk(C0, r, e, tmp, K, st);
}

template <class C>
static void vcycle_blk(SystemImpl& S, WS& W, std::vector<BlockLevel<C>>& V, int l, const C* r, C* x, int K,
                       cudaStream_t st) {
  const Level& F = S.levels[l];
  const int64_t n = F.mesh.ndof;
  if (l == 0) {
    if (F.has_coarse) coarse_solve_blk<C>(F, r, x, V[0].t, K, st);
    else if (F.P.np > 0) smooth_blk<C>(F, r, x, F.theta, 0, V[0].pbuf, K, st);
    else {
      k_zero<C><<<nblk(n * K), 256, 0, st>>>(x, n * K);
      DPG_CHECK_LAUNCH();
    }
    return;
  }
  const Level& Cl = S.levels[l - 1];
  const int64_t nc = Cl.mesh.ndof;
  const C* Avals = Prec<C>::A(F.A);
  const C* rs = r;
  if (F.kind == 2) {
    condense_blk<C>(F, r, V[l].rs, V[l].cbuf, K, st);
    rs = V[l].rs;
  }
  for (int q = 0; q < S.op.nu_pre; ++q) {
    if (q == 0) {
      smooth_blk<C>(F, rs, x, F.theta, 0, V[l].pbuf, K, st);
    } else {
      spmv_blk<C>(F.A, Avals, x, rs, V[l].t, 1, K, st);
      smooth_blk<C>(F, V[l].t, x, F.theta, 1, V[l].pbuf, K, st);
    }
  }
  if (S.op.nu_pre == 0) {
    k_zero<C><<<nblk(n * K), 256, 0, st>>>(x, n * K);
    DPG_CHECK_LAUNCH();
  }
  spmv_blk<C>(F.A, Avals, x, rs, V[l].t, 1, K, st);
  for (int k = 0; k < K; ++k) restrict_vec<C>(F, Cl, V[l].t + k * n, V[l - 1].r + k * nc, st);
  vcycle_blk<C>(S, W, V, l - 1, V[l - 1].r, V[l - 1].x, K, st);
  for (int k = 0; k < K; ++k) prolong_add<C>(F, Cl, V[l - 1].x + k * nc, x + k * n, st);
  for (int q = 0; q < S.op.nu_post; ++q) {
    spmv_blk<C>(F.A, Avals, x, rs, V[l].t, 1, K, st);
    smooth_blk<C>(F, V[l].t, x, F.theta, 1, V[l].pbuf, K, st);
  }
  if (F.kind == 2) backsub_blk<C>(F, r, x, K, st);
}

template <class C>
static std::vector<BlockLevel<C>> alloc_block_levels(Alloc& M, const SystemImpl& S, int K) {
  std::vector<BlockLevel<C>> v(S.levels.size());
  for (size_t l = 0; l < S.levels.size(); ++l) {
    const Level& L = S.levels[l];
    const size_t n = (size_t)L.mesh.ndof * K;
    v[l].r = M.arr<C>(n);
    v[l].rs = M.arr<C>(n);
    v[l].x = M.arr<C>(n);
    v[l].t = M.arr<C>(n);
    if (l >= 1 || L.P.np > 0) v[l].pbuf = M.arr<C>((size_t)std::max<int64_t>(L.P.scratch_entries(), 1) * K);
    if (L.kind == 2) v[l].cbuf = M.arr<C>((size_t)L.nK * L.nS * K);
  }
  return v;
}

static void dot(WS& W, const double2* u, const double2* v, int64_t n, int which, cudaStream_t st) {
  k_dot_fused<double2><<<RED_BLOCKS, 256, 0, st>>>(u, v, n, W.part, W.sc, which, W.ticket);
  DPG_CHECK_LAUNCH();
}

static bool cg_c128(const SystemImpl& S) { return (S.op.flags & DPGMG_FLAG_CG_C128) != 0; }

static const ECSRDev& cg_operator(SystemImpl& S, WS& W, cudaStream_t st) {
  Level& F = S.levels.back();
  if (S.levels.size() > 1 && F.kind == 1) {
    if (!F.A.vlo && !cg_c128(S)) split_operator(S.mem, F.A, F.mesh.offU, pack_storage(S), st);
    return F.A;
  }
  if (!W.acg_owned) {
    // finest operator assembled separately (single level, or h-transition below the finest);
    // its index lists come from the setup's host plan when it is still held
    if (S.plan && S.plan->has_acg) {
      assemble_ecsr(S.mem, S.plan->acg, W.Acg, st);
    } else {
      assemble_ecsr(S.mem, prep_ecsr(F.mesh, element_groups(F.mesh)), W.Acg, st);
    }
    ecsr_add_elements(W.Acg, F.E, F.dofs, F.mesh.nelem, F.nloc, 0, F.mesh.n, st);
    if (!cg_c128(S)) split_operator(S.mem, W.Acg, F.mesh.offU, pack_storage(S), st);
    DPG_CUDA(cudaStreamSynchronize(st));
    W.acg_owned = true;
  }
  return W.Acg;
}

// y = A x (mode 0) or b - A x (mode 1) with the CG operator: double-float by
// default, complex128 on the FP64 pipe under DPGMG_FLAG_CG_C128
static void cg_apply(SystemImpl& S, WS& W, const ECSRDev& A, const double2* x, const double2* b, double2* y,
                     int mode, cudaStream_t st, SystemImpl* prof = nullptr) {
  if (cg_c128(S))
    spmv<double2>(A, A.v64, x, b, y, mode, st, prof);
  else
    spmv_df(A, x, b, y, mode, W.xh, W.xl, st, prof);
}

// ------------------------------------------------------------ tuning
// The SpMV group size G (rows of one entity per warp, 1 = one warp per row)
// and the smoother's columns per lane are chosen per operator by timing the
// variants on the operator itself (one warm-up and three timed launches each,
// each timed launch after an L2 eviction, CUDA events on the setup stream).
// The first variant is kept unless another is at least 5% faster.  Choices
// are cached per (product kind, order p, level kind, log2 of the size), so
// later systems of the same shape skip the timing.
struct TuneKey {
  int kind, p, lkind, lg;
  bool operator<(const TuneKey& o) const {
    return std::tie(kind, p, lkind, lg) < std::tie(o.kind, o.p, o.lkind, o.lg);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tune;

// Reads `n` 16-byte words so that the timed launch after it finds the L2
// holding other data, as inside a V-cycle (the sum is stored only if it hits
// an impossible value, so the reads cannot be dropped).
__global__ void k_l2_evict(const float4* __restrict__ buf, int64_t n, float* __restrict__ sink) {
  float s = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = buf[i];
    s += v.x + v.y + v.z + v.w;
  }
  if (s == 1.2345678e-30f) *sink = s;
}

struct Evict {
  const float4* buf = nullptr;
  int64_t n = 0;
  float* sink = nullptr;
  void run(cudaStream_t st) const {
    if (!n) return;
    k_l2_evict<<<1216, 256, 0, st>>>(buf, n, sink);
    DPG_CHECK_LAUNCH();
  }
};

template <class F>
static int pick_variant(const TuneKey& key, const Evict& ev, cudaStream_t st, std::initializer_list<int> variants,
                        F&& run);

template <class F>
static int pick_group(const TuneKey& key, const Evict& ev, cudaStream_t st, F&& run, bool packed = false,
                      bool df = false) {
  TuneKey k = key;
  if (packed) k.kind += 8;   // packed real entities: every variant but the cp.async ring
  if (df) return packed ? pick_variant(k, ev, st, {1, SPMV_PF, 2, 4, 8}, run)
                        : pick_variant(k, ev, st, {1, SPMV_PF, SPMV_RING, 2, 4, 8}, run);
  return packed ? pick_variant(k, ev, st, {1, SPMV_PF, SPMV_HALF, 2, 4, 8}, run)
                : pick_variant(k, ev, st, {1, SPMV_PF, SPMV_RING, SPMV_HALF, 2, 4, 8}, run);
}

template <class F>
static int pick_variant(const TuneKey& key, const Evict& ev, cudaStream_t st, std::initializer_list<int> variants,
                        F&& run) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  constexpr int REPS = 3;
  cudaEvent_t a[REPS], b[REPS];
  for (int r = 0; r < REPS; ++r) {
    DPG_CUDA(cudaEventCreate(&a[r]));
    DPG_CUDA(cudaEventCreate(&b[r]));
  }
  int best = *variants.begin();
  float best_ms = 0.f;
  for (int G : variants) {
    run(G);
    for (int r = 0; r < REPS; ++r) {
      ev.run(st);
      DPG_CUDA(cudaEventRecord(a[r], st));
      run(G);
      DPG_CUDA(cudaEventRecord(b[r], st));
    }
    DPG_CUDA(cudaEventSynchronize(b[REPS - 1]));
    float ms = 0.f;
    for (int r = 0; r < REPS; ++r) {
      float t = 0.f;
      DPG_CUDA(cudaEventElapsedTime(&t, a[r], b[r]));
      ms += t;
    }
    // the first variant is the default: another must be at least 5% faster
    if (G == *variants.begin() || ms < (best == *variants.begin() ? 0.95f : 1.0f) * best_ms) {
      best = G;
      best_ms = ms;
    }
  }
  for (int r = 0; r < REPS; ++r) {
    cudaEventDestroy(a[r]);
    cudaEventDestroy(b[r]);
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return best;
}

static int log2i(int64_t n) {
  int l = 0;
  while ((int64_t(1) << (l + 1)) <= n) ++l;
  return l;
}

// One CG step (V-cycle, direction update, CG operator, scalar read-back) as a
// CUDA graph: captured on the second iteration, replayed after that.  The
// launch sequence of a step does not change between iterations, and every
// buffer it touches lives as long as the system.  If the stream cannot be
// captured (the legacy default stream), the step runs eagerly.
struct PcgGraph {
  cudaGraphExec_t exec = nullptr;
  long long nodes = 0;
  bool failed = false;
  template <class F> bool ready(cudaStream_t st, F&& body) {
    if (exec) return true;
    if (failed) return false;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
      return false;
    }
    const long long l0 = thread_launch_count();
    cudaGraph_t g = nullptr;
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    DPG_CUDA(cudaStreamEndCapture(st, &g));
    nodes = thread_launch_count() - l0;
    count_launches(-nodes);   // captured, not yet run
    const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      exec = nullptr;
      failed = true;
      return false;
    }
    return true;
  }
  void launch(cudaStream_t st) {
    DPG_CUDA(cudaGraphLaunch(exec, st));
    count_launches(nodes);
  }
  ~PcgGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

// the CG operator of a prepared system (nullptr before prepare_solve)
ECSRDev* cg_operator_of(SystemImpl& S) {
  if (!S.ws) return nullptr;
  WS& W = *reinterpret_cast<WS*>(S.ws);
  Level& F = S.levels.back();
  if (S.levels.size() > 1 && F.kind == 1) return F.A.vlo ? &F.A : nullptr;
  return W.acg_owned ? &W.Acg : nullptr;
}

void prepare_solve(SystemImpl& S, cudaStream_t st) {
  ensure_workspace(S, st);
  WS& W = *reinterpret_cast<WS*>(S.ws);
  ECSRDev& Acg = const_cast<ECSRDev&>(cg_operator(S, W, st));
  const bool mixed = S.op.precision == DPGMG_PREC_MIXED;
  const int L = (int)S.levels.size() - 1;
  // between timed launches, read up to 256 MiB of the finest patch inverses
  Evict ev;
  {
    const PatchDev& P = S.levels[L].P;
    const void* buf = mixed && P.inv32 ? (const void*)P.inv32 : (P.inv64 ? (const void*)P.inv64 : (const void*)P.wbuf);
    const int64_t bytes = std::min<int64_t>(P.inv32 || P.inv64 ? P.nvals * (mixed && P.inv32 ? 8 : 16) : P.wcap * 8,
                                            (int64_t)256 << 20);
    if (L >= 1 && buf && bytes >= 16) {
      ev.buf = reinterpret_cast<const float4*>(buf);
      ev.n = bytes / 16;
      ev.sink = reinterpret_cast<float*>(W.part);
    }
  }
  for (int l = 1; l <= L; ++l) {
    Level& F = S.levels[l];
    const int64_t n = F.mesh.ndof;
    const TuneKey key{mixed ? 0 : 1, F.mesh.p, F.kind, log2i(n)};
    if (mixed) {
      float2 *x = W.w32[l].x, *y = W.w32[l].t;
      DPG_CUDA(cudaMemsetAsync(x, 0, (size_t)n * sizeof(float2), st));
      F.A.gsel[0] = pick_group(key, ev, st, [&](int G) { spmv_g<float2>(F.A, F.A.v32, x, nullptr, y, 0, G, st); },
                               F.A.rent != nullptr);
      if (F.P.inv32 && F.P.np) {
        // smoother product: 1 or 2 columns per lane (32- or 64-column work
        // items), the latter at 8 or 6 CTAs per SM; the block smoother takes
        // the same columns per lane
        const TuneKey skey{F.P.rflag ? 4 : 3, F.mesh.p, F.kind, log2i(F.P.np)};   // packed real blocks or not
        auto run = [&](int c) { launch_patch_apply_c64<float2>(F.P, c, F.P.inv32, x, W.w32[l].pbuf, st); };
        F.P.variant = F.P.rflag ? pick_variant(skey, ev, st, {SMOOTH_PER2_WIDE, 2, 1}, run)
                                : pick_variant(skey, ev, st, {2, SMOOTH_PER2_WIDE, 1}, run);
        F.P.cols = F.P.variant == 1 ? 1 : 2;
      }
    } else {
      double2 *x = W.w64[l].x, *y = W.w64[l].t;
      DPG_CUDA(cudaMemsetAsync(x, 0, (size_t)n * sizeof(double2), st));
      F.A.gsel[1] = pick_group(key, ev, st, [&](int G) { spmv_g<double2>(F.A, F.A.v64, x, nullptr, y, 0, G, st); });
    }
  }
  {
    const Level& F = S.levels[L];
    const int64_t n = F.mesh.ndof;
    DPG_CUDA(cudaMemsetAsync(W.xh, 0, (size_t)n * sizeof(float2), st));
    DPG_CUDA(cudaMemsetAsync(W.xl, 0, (size_t)n * sizeof(float2), st));
    if (cg_c128(S)) {
      DPG_CUDA(cudaMemsetAsync(W.p, 0, (size_t)n * sizeof(double2), st));
      const TuneKey key{1, F.mesh.p, F.kind, log2i(n)};
      Acg.gsel[1] = pick_group(key, ev, st, [&](int G) { spmv_g<double2>(Acg, Acg.v64, W.p, nullptr, W.q, 0, G, st); });
    } else {
      const TuneKey key{2, F.mesh.p, F.kind, log2i(n)};
      Acg.gsel[2] = pick_group(key, ev, st, [&](int G) { spmv_df_g(Acg, W.xh, W.xl, nullptr, W.q, 0, G, st); },
                               Acg.rent != nullptr, true);
    }
  }
}

int pcg_solve(SystemImpl& S, cudaStream_t st, double2* xout, dpgmg_stats* stats, const double2* x0) {
  ensure_workspace(S, st);
  WS& W = *reinterpret_cast<WS*>(S.ws);
  const ECSRDev& A = cg_operator(S, W, st);
  {
    const Level& Ff = S.levels.back();
    const int64_t esz = S.op.precision == DPGMG_PREC_MIXED ? 8 : 16;
    if (S.prof_which == DPGMG_PROF_SMOOTH_FINE)   // stored entries read once: real packed blocks at half size
      S.prof_bytes = (Ff.P.sum_sq - Ff.P.real_sq) * esz + Ff.P.real_sq * (esz / 2);
    else if (S.prof_which == DPGMG_PROF_SPMV_FINE)   // packed real entities at half size
      S.prof_bytes = (Ff.A.nnz_alg - Ff.A.nnz_real) * esz + Ff.A.nnz_real * (esz / 2);
    else if (S.prof_which == DPGMG_PROF_SPMV_CG)     // hi + lo complex64, or hi + lo reals
      S.prof_bytes = (A.nnz_alg - A.nnz_real) * 16 + A.nnz_real * 8;
  }
  const int64_t n = S.levels.back().mesh.ndof;
  cudaEvent_t e0, e1;
  DPG_CUDA(cudaEventCreate(&e0));
  DPG_CUDA(cudaEventCreate(&e1));
  DPG_CUDA(cudaEventRecord(e0, st));
  DPG_CUDA(cudaMemcpyAsync(W.r, S.b, (size_t)n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  dot(W, W.r, W.r, n, 1, st);   // ||b||^2
  DPG_CUDA(cudaMemcpyAsync(W.sc_host, W.sc, SC_COUNT * sizeof(double2), cudaMemcpyDeviceToHost, st));
  DPG_CUDA(cudaStreamSynchronize(st));
  const double nb = std::sqrt(W.sc_host[SC_RR].x);
  double rel = 1.0;
  if (x0) {
    // warm start: x = x0, r = b - A x0
    DPG_CUDA(cudaMemcpyAsync(W.x, x0, (size_t)n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    cg_apply(S, W, A, W.x, S.b, W.r, 1, st);
    dot(W, W.r, W.r, n, 1, st);
    DPG_CUDA(cudaMemcpyAsync(W.sc_host, W.sc, SC_COUNT * sizeof(double2), cudaMemcpyDeviceToHost, st));
    DPG_CUDA(cudaStreamSynchronize(st));
    rel = nb > 0.0 ? std::sqrt(W.sc_host[SC_RR].x) / nb : 0.0;
  } else {
    k_zero<double2><<<nblk(n), 256, 0, st>>>(W.x, n);
    DPG_CHECK_LAUNCH();
  }
  int status = DPGMG_OK;
  int it = 0;
  if (nb > 0.0 && !(x0 && rel <= S.op.tol)) {
    SystemImpl* pcg_prof = S.prof_which == DPGMG_PROF_SPMV_CG ? &S : nullptr;
    // q = A p, alpha = rho / p^H q, x += alpha p, r -= alpha q, ||r||^2, scalars to the host
    const bool mixed = S.op.precision == DPGMG_PREC_MIXED;
    const int Lf = (int)S.levels.size() - 1;
    float2* r32 = mixed ? W.w32[Lf].r : nullptr;
    // presplit: p's double-float split is already in W.xh / W.xl (written by k_cg_dir)
    auto tail = [&](bool presplit) {
      if (cg_c128(S)) {
        spmv<double2>(A, A.v64, W.p, nullptr, W.q, 0, st, pcg_prof);
      } else if (presplit) {
        int pe = prof_begin(pcg_prof, st);
        spmv_df_g(A, W.xh, W.xl, nullptr, W.q, 0, A.gsel[2], st);
        prof_end(pcg_prof, pe, st);
      } else {
        spmv_df(A, W.p, nullptr, W.q, 0, W.xh, W.xl, st, pcg_prof);
      }
      dot(W, W.p, W.q, n, 0, st);   // pq = p^H q
      k_cg_update_fused<<<RED_BLOCKS, 256, 0, st>>>(W.x, W.r, W.p, W.q, W.sc, n, W.part, W.ticket, r32);
      DPG_CHECK_LAUNCH();
      DPG_CUDA(cudaMemcpyAsync(W.sc_host, W.sc, SC_COUNT * sizeof(double2), cudaMemcpyDeviceToHost, st));
    };
    // z = B r, rho_new = z^H r, beta = rho_new / rho, p = z + beta p (and its split)
    auto head = [&]() {
      if (mixed) {
        // r's complex64 copy comes from the CG update; z stays in complex64 and is widened on load
        precondition(S, W, W.r, nullptr, st, true);
        const float2* z32 = W.w32[Lf].x;
        k_dot_fused<float2><<<RED_BLOCKS, 256, 0, st>>>(z32, W.r, n, W.part, W.sc, 2, W.ticket);
        DPG_CHECK_LAUNCH();
        k_cg_dir<float2><<<RED_BLOCKS, 256, 0, st>>>(W.p, z32, W.sc, n, W.xh, W.xl);
        DPG_CHECK_LAUNCH();
      } else {
        precondition(S, W, W.r, W.z, st);
        dot(W, W.z, W.r, n, 2, st);
        k_cg_dir<double2><<<RED_BLOCKS, 256, 0, st>>>(W.p, W.z, W.sc, n, W.xh, W.xl);
        DPG_CHECK_LAUNCH();
      }
    };
    precondition(S, W, W.r, W.z, st);
    dot(W, W.z, W.r, n, 3, st);   // rho = z^H r
    DPG_CUDA(cudaMemcpyAsync(W.p, W.z, (size_t)n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    tail(false);
    PcgGraph G;
    const bool graphs = !(S.op.flags & DPGMG_FLAG_EAGER);
    bool replayed = false;
    while (true) {
      DPG_CUDA(cudaStreamSynchronize(st));
      if (replayed) prof_graph_accumulate(S);
      ++it;
      const double pq = W.sc_host[SC_PQ].x;
      if (!(pq > 0.0) || !std::isfinite(pq)) { status = DPGMG_ERR_BREAKDOWN; break; }
      rel = std::sqrt(W.sc_host[SC_RR].x) / nb;
      if (!std::isfinite(rel)) { status = DPGMG_ERR_BREAKDOWN; break; }
      if (rel <= S.op.tol || it >= S.op.max_iter) break;
      if (graphs && G.ready(st, [&]() { head(); tail(true); })) {
        G.launch(st);
        replayed = true;
      } else {
        head();
        tail(true);
      }
    }
    if (status == DPGMG_OK && rel > S.op.tol) status = DPGMG_ERR_NOT_CONVERGED;
  }
  DPG_CUDA(cudaEventRecord(e1, st));
  DPG_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  DPG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // true residual ||b - A x|| / ||b|| in FP64
  double true_rel = 0.0;
  if (nb > 0.0) {
    cg_apply(S, W, A, W.x, S.b, W.q, 1, st);
    dot(W, W.q, W.q, n, 1, st);
    DPG_CUDA(cudaMemcpyAsync(W.sc_host, W.sc, SC_COUNT * sizeof(double2), cudaMemcpyDeviceToHost, st));
    DPG_CUDA(cudaStreamSynchronize(st));
    true_rel = std::sqrt(W.sc_host[SC_RR].x) / nb;
  }
  if (xout) DPG_CUDA(cudaMemcpyAsync(xout, W.x, (size_t)n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  if (stats) {
    stats->iters = it;
    stats->relres = rel;
    stats->true_relres = true_rel;
    stats->t_pcg_ms = ms;
    stats->t_setup_ms = S.t_setup_ms;
    stats->bytes_per_iter = S.bytes_per_iter;
    stats->n_dof = n;
    stats->dev_bytes_peak = (long long)S.mem_peak();
  }
  return status;
}

// ------------------------------------------------------------ block PCG
// K independent MG-PCG iterations (each with its own scalars and stopping
// test, the recurrence of pcg_solve) that share every V-cycle: z_k = B r_k for
// all k at once through vcycle_blk.  Right-hand sides B and solutions X are
// device [K][n].  A right-hand side that has converged keeps its x, r and p;
// its V-cycle and operator columns are still computed (the matrices are read
// once for all columns).  The steps after the first are replayed from a CUDA
// graph captured for the current set of active columns (captured again when
// a column converges).
int pcg_solve_block(SystemImpl& S, cudaStream_t st, int K, const double2* B, double2* X, dpgmg_stats* stats) {
  ensure_workspace(S, st);
  WS& W = *reinterpret_cast<WS*>(S.ws);
  const ECSRDev& A = cg_operator(S, W, st);
  const int L = (int)S.levels.size() - 1;
  const int64_t n = S.levels[L].mesh.ndof;
  const bool mixed = S.op.precision == DPGMG_PREC_MIXED;
  Alloc M;
  M.budget = (size_t)-1;
  M.stream = st;
  double2* R = M.arr<double2>((size_t)n * K);
  double2* P = M.arr<double2>((size_t)n * K);
  double2* Q = M.arr<double2>((size_t)n * K);
  double2* Z = M.arr<double2>((size_t)n * K);
  double2* sc = M.arr<double2>((size_t)SC_COUNT * K);
  double2* part = M.arr<double2>((size_t)RED_BLOCKS * K);
  unsigned* ticket = M.arr<unsigned>((size_t)K);
  double2* sch = nullptr;   // pinned copy of the scalars
  DPG_CUDA(cudaMallocHost(&sch, (size_t)SC_COUNT * K * sizeof(double2)));
  struct HostFree {
    double2* p;
    ~HostFree() { cudaFreeHost(p); }
  } hf{sch};
  float2* XH = cg_c128(S) ? nullptr : M.arr<float2>((size_t)n * K);
  float2* XL = cg_c128(S) ? nullptr : M.arr<float2>((size_t)n * K);
  DPG_CUDA(cudaMemsetAsync(ticket, 0, (size_t)K * sizeof(unsigned), st));
  DPG_CUDA(cudaMemsetAsync(sc, 0, (size_t)SC_COUNT * K * sizeof(double2), st));
  // Y = A X (mode 0) or B - A X (mode 1) for all K columns with the CG operator,
  // its stored values read once per group of BLK_MAX columns
  auto cg_apply_blk = [&](const double2* Xs, const double2* Bs, double2* Ys, int mode) {
    if (cg_c128(S)) {
      spmv_blk<double2>(A, A.v64, Xs, Bs, Ys, mode, K, st);
      return;
    }
    k_split_vec<<<nblk(n * K), 256, 0, st>>>(Xs, XH, XL, n * K);
    DPG_CHECK_LAUNCH();
    for (int g = 0; g < K; g += BLK_MAX) {
      const int kb = std::min(BLK_MAX, K - g);
      const double2* bg = Bs ? Bs + (size_t)g * n : nullptr;
      const float2* xh = XH + (size_t)g * n;
      const float2* xl = XL + (size_t)g * n;
      double2* yg = Ys + (size_t)g * n;
      const unsigned blocks = (unsigned)std::min<int64_t>((n + 7) / 8, 152 * 16);
#define DPG_DF_BLK(KB)                                                                                            \
  k_spmv_df_blk<KB><<<blocks, 256, 0, st>>>(A.row_ent, A.ent_start, A.col_ptr, A.col_idx, A.val_ptr, A.v32, A.vlo, \
                                            xh, xl, bg, yg, n, n, mode, A.rent, A.offU)
      if (kb == 4) DPG_DF_BLK(4);
      else if (kb == 3) DPG_DF_BLK(3);
      else if (kb == 2) DPG_DF_BLK(2);
      else DPG_DF_BLK(1);
#undef DPG_DF_BLK
      DPG_CHECK_LAUNCH();
    }
  };
  std::vector<BlockLevel<float2>> V32;
  std::vector<BlockLevel<double2>> V64;
  if (mixed) V32 = alloc_block_levels<float2>(M, S, K);
  else V64 = alloc_block_levels<double2>(M, S, K);
  // z = B r for every column (complex128 result in Z)
  auto precondition_blk = [&]() {
    if (mixed) {
      k_narrow<<<nblk(n * K), 256, 0, st>>>(R, V32[L].r, n * K);
      DPG_CHECK_LAUNCH();
      vcycle_blk<float2>(S, W, V32, L, V32[L].r, V32[L].x, K, st);
      k_widen<<<nblk(n * K), 256, 0, st>>>(V32[L].x, Z, n * K);
      DPG_CHECK_LAUNCH();
    } else {
      vcycle_blk<double2>(S, W, V64, L, R, Z, K, st);
    }
  };
  const dim3 rgrid(RED_BLOCKS, (unsigned)K);
  auto dot_blk = [&](const double2* U, const double2* Vv, int which, unsigned long long mask) {
    k_dot_fused_blk<double2><<<rgrid, 256, 0, st>>>(U, Vv, n, part, sc, which, ticket, mask);
    DPG_CHECK_LAUNCH();
  };
  auto read_scalars = [&]() {
    DPG_CUDA(cudaMemcpyAsync(sch, sc, (size_t)SC_COUNT * K * sizeof(double2), cudaMemcpyDeviceToHost, st));
  };
  const unsigned long long all = K == 64 ? ~0ull : ((1ull << K) - 1ull);
  cudaEvent_t e0, e1;
  DPG_CUDA(cudaEventCreate(&e0));
  DPG_CUDA(cudaEventCreate(&e1));
  DPG_CUDA(cudaEventRecord(e0, st));
  DPG_CUDA(cudaMemcpyAsync(R, B, (size_t)n * K * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  k_zero<double2><<<nblk(n * K), 256, 0, st>>>(X, n * K);
  DPG_CHECK_LAUNCH();
  dot_blk(R, R, 1, all);   // ||b_k||^2
  read_scalars();
  DPG_CUDA(cudaStreamSynchronize(st));
  std::vector<double> nb(K), rel(K, 0.0);
  std::vector<int> iters(K, 0), status(K, DPGMG_OK);
  unsigned long long active = 0;
  for (int k = 0; k < K; ++k) {
    nb[k] = std::sqrt(sch[(size_t)k * SC_COUNT + SC_RR].x);
    if (nb[k] > 0.0) active |= 1ull << k;
  }
  // q = A p, alpha = rho / p^H q, x += alpha p, r -= alpha q, ||r||^2, scalars to the host
  auto tail = [&](unsigned long long mask) {
    cg_apply_blk(P, nullptr, Q, 0);
    dot_blk(P, Q, 0, mask);
    k_cg_update_fused_blk<<<rgrid, 256, 0, st>>>(X, R, P, Q, sc, n, part, ticket, mask);
    DPG_CHECK_LAUNCH();
    read_scalars();
  };
  // z = B r, rho_new = z^H r, beta = rho_new / rho, p = z + beta p
  auto head = [&](unsigned long long mask) {
    precondition_blk();
    dot_blk(Z, R, 2, mask);
    k_cg_dir_blk<<<rgrid, 256, 0, st>>>(P, Z, sc, n, mask);
    DPG_CHECK_LAUNCH();
  };
  int it = 0;
  if (active) {
    precondition_blk();
    dot_blk(Z, R, 3, active);   // rho = z^H r
    DPG_CUDA(cudaMemcpyAsync(P, Z, (size_t)n * K * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    tail(active);
    std::unique_ptr<PcgGraph> G;
    unsigned long long gmask = 0;
    const bool graphs = !(S.op.flags & DPGMG_FLAG_EAGER);
    while (true) {
      DPG_CUDA(cudaStreamSynchronize(st));
      ++it;
      for (int k = 0; k < K; ++k) {
        if (!((active >> k) & 1ull)) continue;
        const double2* c = &sch[(size_t)k * SC_COUNT];
        iters[k] = it;
        const double pq = c[SC_PQ].x;
        rel[k] = std::sqrt(c[SC_RR].x) / nb[k];
        if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rel[k])) {
          status[k] = DPGMG_ERR_BREAKDOWN;
          active &= ~(1ull << k);
        } else if (rel[k] <= S.op.tol || it >= S.op.max_iter) {
          active &= ~(1ull << k);
        }
      }
      if (!active) break;
      if (graphs && (!G || gmask != active)) {
        G.reset(new PcgGraph());
        gmask = active;
      }
      const unsigned long long mask = active;
      if (graphs && G->ready(st, [&]() { head(mask); tail(mask); })) {
        G->launch(st);
      } else {
        head(mask);
        tail(mask);
      }
    }
  }
  DPG_CUDA(cudaEventRecord(e1, st));
  DPG_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  DPG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // true residuals ||b - A x|| / ||b|| in FP64
  cg_apply_blk(X, B, Q, 1);
  dot_blk(Q, Q, 1, all);
  read_scalars();
  DPG_CUDA(cudaStreamSynchronize(st));
  int worst = DPGMG_OK;
  for (int k = 0; k < K; ++k) {
    if (status[k] == DPGMG_OK && nb[k] > 0.0 && rel[k] > S.op.tol) status[k] = DPGMG_ERR_NOT_CONVERGED;
    const double true_rel = nb[k] > 0.0 ? std::sqrt(sch[(size_t)k * SC_COUNT + SC_RR].x) / nb[k] : 0.0;
    if (stats) {
      dpgmg_stats& o = stats[k];
      o.iters = iters[k];
      o.relres = rel[k];
      o.true_relres = true_rel;
      o.t_pcg_ms = ms;
      o.t_setup_ms = S.t_setup_ms;
      o.bytes_per_iter = S.bytes_per_iter;
      o.n_dof = n;
      o.dev_bytes_peak = (long long)(S.mem_peak() + M.peak);
    }
    if (worst == DPGMG_OK && status[k] != DPGMG_OK) worst = status[k];
  }
  return worst;
}

// ---------------------------------------------------------------- theta
// theta = 1 / (1.05 lambda), lambda from 30 power iterations x <- S M x /
// ||S M x|| started from a SplitMix64 vector (seed 12345) on the smoothing
// space, then the Rayleigh quotient (M x, S M x) / (M x, x).  FP64.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
template <class C>
__global__ void k_start_vector(C* x, int64_t n, const int64_t* slot_ptr) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = 1.0 / 9007199254740992.0;
  double re = 2.0 * (double)(splitmix64(12345ull, 2 * (uint64_t)i) >> 11) * s - 1.0;
  double im = 2.0 * (double)(splitmix64(12345ull, 2 * (uint64_t)i + 1) >> 11) * s - 1.0;
  bool in = slot_ptr[i + 1] > slot_ptr[i];   // DOF belongs to some patch
  using R = typename Ops<C>::R;
  x[i] = in ? Ops<C>::mk((R)re, (R)im) : Ops<C>::zero();
}

// partial[b] = sum conj(u_i) v_i (accumulated in FP64 whatever the vector precision)
template <class C>
__global__ void k_dot_partial_t(const C* __restrict__ u, const C* __restrict__ v, int64_t n, double2* __restrict__ part) {
  __shared__ double2 sh[8];
  double2 acc = make_double2(0, 0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ux = u[i].x, uy = u[i].y, vx = v[i].x, vy = v[i].y;
    acc.x += ux * vx + uy * vy;
    acc.y += ux * vy - uy * vx;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s2 = make_double2(0, 0);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s2 = Ops<double2>::add(s2, sh[k]);
    part[blockIdx.x] = s2;
  }
}

template <class C>
__global__ void k_scale(C* x, int64_t n, const double2* sc, int slot) {
  using R = typename Ops<C>::R;
  const R s = (R)(1.0 / sqrt(sc[slot].x));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = Ops<C>::scale(x[i], s);
}

template <class C>
static void dot_t(WS& W, const C* u, const C* v, int64_t n, int which, cudaStream_t st) {
  k_dot_partial_t<C><<<RED_BLOCKS, 256, 0, st>>>(u, v, n, W.part);
  DPG_CHECK_LAUNCH();
  k_dot_finish<<<1, 256, 0, st>>>(W.part, RED_BLOCKS, W.sc, which);
  DPG_CHECK_LAUNCH();
}

__global__ void k_take_re(const double2* sc, int idx, double* out) { *out = sc[idx].x; }

double theta_from_rayleigh(double num, double den) { return 1.0 / (1.05 * (num / den)); }

// lambda = (M x)^H (S M x) / (x^H M x) after 30 power iterations of S M from a
// SplitMix64 vector on the smoothing space, with FP64 vectors and dot products;
// out[0] = numerator, out[1] = denominator (device), theta = 1 / (1.05 lambda).
//   operator M: double-float (complex64 high and low parts of the FP64 values,
//     ~48-bit products and sums on the FP32 pipe), or complex128 on the FP64
//     pipe under DPGMG_FLAG_CG_C128;
//   smoother S: the FP64 patch inverses in double-float (high parts in
//     P.inv32, low parts in plo), or complex128 under DPGMG_FLAG_CG_C128; on the
//     mixed path with FP32 patch factors, the complex64 inverses the V-cycle
//     applies, taken exactly (plo null), so theta damps the smoother in use.
// (On the mixed path with FP32 patch factors and the default CG operator the
// estimate runs in the V-cycle's complex64 arithmetic instead:
// estimate_theta_c64.)
// Mixed path with FP32 patch factors: the V-cycle's own complex64 operator
// and smoother, complex64 vectors, FP64 dot products.
static void estimate_theta_c64(SystemImpl& S, Level& F, double* out, cudaStream_t st) {
  const int64_t n = F.mesh.ndof;
  Alloc tmp;
  tmp.budget = (size_t)-1;
  tmp.stream = st;
  float2* x = tmp.arr<float2>((size_t)n);
  float2* y = tmp.arr<float2>((size_t)n);
  float2* t = tmp.arr<float2>((size_t)n);
  float2* pbuf = tmp.arr<float2>((size_t)std::max<int64_t>(F.P.scratch_entries(), 1));
  WS W;
  W.part = tmp.arr<double2>(RED_BLOCKS);
  W.sc = tmp.arr<double2>(SC_COUNT);
  k_start_vector<float2><<<nblk(n), 256, 0, st>>>(x, n, F.P.slot_ptr);
  DPG_CHECK_LAUNCH();
  dot_t<float2>(W, x, x, n, 1, st);
  k_scale<float2><<<RED_BLOCKS, 256, 0, st>>>(x, n, W.sc, SC_RR);
  DPG_CHECK_LAUNCH();
  for (int k = 0; k < 30; ++k) {
    spmv<float2>(F.A, F.A.v32, x, nullptr, t, 0, st);
    smooth<float2>(F, t, y, 1.0, 0, pbuf, st);
    dot_t<float2>(W, y, y, n, 1, st);
    k_scale<float2><<<RED_BLOCKS, 256, 0, st>>>(y, n, W.sc, SC_RR);
    DPG_CHECK_LAUNCH();
    std::swap(x, y);
  }
  spmv<float2>(F.A, F.A.v32, x, nullptr, t, 0, st);   // M x
  smooth<float2>(F, t, y, 1.0, 0, pbuf, st);           // S M x
  dot_t<float2>(W, t, y, n, 3, st);
  k_take_re<<<1, 1, 0, st>>>(W.sc, SC_RHO, out);
  DPG_CHECK_LAUNCH();
  dot_t<float2>(W, x, t, n, 3, st);
  k_take_re<<<1, 1, 0, st>>>(W.sc, SC_RHO, out + 1);
  DPG_CHECK_LAUNCH();
  W.part = nullptr;
  W.sc = nullptr;
}

static void estimate_theta_fp(SystemImpl& S, Level& F, const float2* plo, double* out, cudaStream_t st) {
  const int64_t n = F.mesh.ndof;
  const bool c128 = cg_c128(S);
  const bool z_smooth = c128 && F.P.inv64;
  Alloc tmp;
  tmp.budget = (size_t)-1;
  tmp.stream = st;
  double2* x = tmp.arr<double2>((size_t)n);
  double2* y = tmp.arr<double2>((size_t)n);
  double2* t = tmp.arr<double2>((size_t)n);
  float2* xh = c128 ? nullptr : tmp.arr<float2>((size_t)n);
  float2* xl = c128 ? nullptr : tmp.arr<float2>((size_t)n);
  double2* pbuf = tmp.arr<double2>((size_t)std::max<int64_t>(F.P.scratch_entries(), 1));
  auto op = [&](const double2* v, double2* o) {
    if (c128) spmv<double2>(F.A, F.A.v64, v, nullptr, o, 0, st);
    else spmv_df(F.A, v, nullptr, o, 0, xh, xl, st);
  };
  auto sm = [&](const double2* v, double2* o) {
    if (z_smooth) smooth<double2>(F, v, o, 1.0, 0, pbuf, st);
    else smooth_df(F, plo, v, o, pbuf, st);
  };
  WS W;
  W.part = tmp.arr<double2>(RED_BLOCKS);
  W.sc = tmp.arr<double2>(SC_COUNT);
  k_start_vector<double2><<<nblk(n), 256, 0, st>>>(x, n, F.P.slot_ptr);
  DPG_CHECK_LAUNCH();
  dot_t<double2>(W, x, x, n, 1, st);
  k_scale<double2><<<RED_BLOCKS, 256, 0, st>>>(x, n, W.sc, SC_RR);
  DPG_CHECK_LAUNCH();
  for (int k = 0; k < 30; ++k) {
    op(x, t);
    sm(t, y);
    dot_t<double2>(W, y, y, n, 1, st);
    k_scale<double2><<<RED_BLOCKS, 256, 0, st>>>(y, n, W.sc, SC_RR);
    DPG_CHECK_LAUNCH();
    std::swap(x, y);
  }
  op(x, t);                                     // M x
  sm(t, y);                                     // S M x
  dot_t<double2>(W, t, y, n, 3, st);            // (M x)^H (S M x)
  k_take_re<<<1, 1, 0, st>>>(W.sc, SC_RHO, out);
  DPG_CHECK_LAUNCH();
  dot_t<double2>(W, x, t, n, 3, st);            // x^H M x
  k_take_re<<<1, 1, 0, st>>>(W.sc, SC_RHO, out + 1);
  DPG_CHECK_LAUNCH();
  W.part = nullptr;
  W.sc = nullptr;
}

void estimate_theta(SystemImpl& S, int l, double* rayleigh, const float2* plo, cudaStream_t st) {
  Level& F = S.levels[l];
  configure_smoother_kernels();
  if (S.op.theta > 0.0) {
    F.theta = S.op.theta;
    return;
  }
  if (S.op.precision == DPGMG_PREC_MIXED && !cg_c128(S) && !F.P.inv64 && F.A.v32) {
    estimate_theta_c64(S, F, rayleigh, st);
    return;
  }
  estimate_theta_fp(S, F, plo, rayleigh, st);
}

// ------------------------------------------------------------ introspection
template <class C>
static void apply_t(SystemImpl& S, WS& W, int op, int l, const C* x, C* y, cudaStream_t st) {
  const Level& F = S.levels[l];
  auto& V = wsv<C>(W);
  switch (op) {
    case DPGMG_OP_A:
      spmv<C>(F.A, Prec<C>::A(F.A), x, nullptr, y, 0, st);
      break;
    case DPGMG_OP_SMOOTH:
      smooth<C>(F, x, y, F.theta, 0, V[l].pbuf, st);
      break;
    case DPGMG_OP_VCYCLE:
      vcycle<C>(S, W, l, x, y, st);
      break;
    case DPGMG_OP_RESTRICT:
      restrict_vec<C>(F, S.levels[l - 1], x, y, st);
      break;
    case DPGMG_OP_PROLONG:
      k_zero<C><<<nblk(F.mesh.ndof), 256, 0, st>>>(y, F.mesh.ndof);
      prolong_add<C>(F, S.levels[l - 1], x, y, st);
      break;
    case DPGMG_OP_CONDENSE:
      condense<C>(F, x, y, V[l].cbuf, st);
      break;
    case DPGMG_OP_COARSE:
      coarse_solve<C>(S, W, x, y, st);
      break;
  }
}

void apply_op(SystemImpl& S, int op, int l, const double2* x, double2* y, cudaStream_t st) {
  ensure_workspace(S, st);
  WS& W = *reinterpret_cast<WS*>(S.ws);
  if (op == DPGMG_OP_AFULL) {
    const ECSRDev& A = cg_operator(S, W, st);
    cg_apply(S, W, A, x, nullptr, y, 0, st);
    return;
  }
  if (S.op.precision == DPGMG_PREC_MIXED) {
    const Level& F = S.levels[l];
    int64_t nin = F.mesh.ndof, nout = F.mesh.ndof;
    if (op == DPGMG_OP_RESTRICT) nout = S.levels[l - 1].mesh.ndof;
    if (op == DPGMG_OP_PROLONG) nin = S.levels[l - 1].mesh.ndof;
    Alloc tmp;
    tmp.budget = (size_t)-1;
    tmp.stream = st;
    float2* xi = tmp.arr<float2>((size_t)nin);
    float2* yo = tmp.arr<float2>((size_t)nout);
    k_narrow<<<nblk(nin), 256, 0, st>>>(x, xi, nin);
    apply_t<float2>(S, W, op, l, xi, yo, st);
    k_widen<<<nblk(nout), 256, 0, st>>>(yo, y, nout);
    DPG_CUDA(cudaStreamSynchronize(st));
  } else {
    apply_t<double2>(S, W, op, l, x, y, st);
  }
  DPG_CHECK_LAUNCH();
}

}  // namespace dpgmg
