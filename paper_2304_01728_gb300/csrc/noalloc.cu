// dpgmg_smooth_noalloc: the additive Schwarz smoother of one level applied to
// caller-owned device vectors without any device-memory allocation.
//
// Some callers cannot let a library call cudaMalloc/cudaFree: programs that
// hand all device memory to their own fixed arena or pool up front (so a new
// allocation fails or breaks their accounting), and latency-critical loops
// that cannot afford the device-wide synchronisation cudaFree implies.  For
// them this entry point keeps the smoother's only scratch -- the per-slot
// patch products that the deterministic gather-sum reads -- in a file-scope
// device array of fixed size instead of in memory the library allocates.
//
// The array lives in every GPU context that loads the library, until the
// process exits (NOALLOC_MAX_SLOTS complex128 entries = 64 MiB).  Host code
// must not use the array's name as a device address: its device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on the device.
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace dpgmg {

constexpr int64_t NOALLOC_MAX_SLOTS = (int64_t)1 << 22;   // patch-product entries (complex128)
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_MAX_SLOTS];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once).
static void* noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) throw Err{DPGMG_ERR_ARG, "device ordinal out of range"};
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      throw Err{DPGMG_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
    }
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

template <class C> __device__ __forceinline__ C from_c128(double2 v);
template <> __device__ __forceinline__ double2 from_c128<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_c128<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}

// Patch products for one 32-row chunk (same work split as the solver's
// smoother); r is complex128 and is rounded to the operator precision C.
template <class C>
__global__ void __launch_bounds__(256) k_na_patch(const int64_t* __restrict__ ptr, const int32_t* __restrict__ dofs,
                                                  const int64_t* __restrict__ vptr, const int2* __restrict__ chunks,
                                                  const C* __restrict__ inv, const double2* __restrict__ r,
                                                  C* __restrict__ pbuf) {
  extern __shared__ unsigned char shraw[];
  __shared__ C part[8][33];
  C* rj = reinterpret_cast<C*>(shraw);
  using O = Ops<C>;
  const int2 ch = chunks[blockIdx.x];
  const int64_t j = ch.x;
  const int64_t b = ptr[j];
  const int n = (int)(ptr[j + 1] - b);
  for (int q = threadIdx.x; q < n; q += blockDim.x) rj[q] = from_c128<C>(r[dofs[b + q]]);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int a = ch.y + lane;
  const C* M = inv + vptr[j] + a;
  C a0 = O::zero(), a1 = O::zero();
  if (a < n) {
    int k = w;
    for (; k + 8 < n; k += 16) {
      a0 = O::fmac(rj[k], M[(size_t)k * n], a0);
      a1 = O::fmac(rj[k + 8], M[(size_t)(k + 8) * n], a1);
    }
    if (k < n) a0 = O::fmac(rj[k], M[(size_t)k * n], a0);
  }
  part[w][lane] = O::add(a0, a1);
  __syncthreads();
  if (w == 0 && a < n) {
    C s = part[0][lane];
#pragma unroll
    for (int q = 1; q < 8; ++q) s = O::add(s, part[q][lane]);
    pbuf[b + a] = s;
  }
}

// y[g] = theta * sum of the patch products of DOF g (complex128 output)
template <class C>
__global__ void k_na_sum(const int64_t* __restrict__ sptr, const int32_t* __restrict__ slots,
                         const C* __restrict__ pbuf, double2* __restrict__ y, int64_t n, double theta) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  C acc = Ops<C>::zero();
  for (int64_t s = sptr[g]; s < sptr[g + 1]; ++s) acc = Ops<C>::add(acc, pbuf[slots[s]]);
  acc = Ops<C>::scale(acc, (typename Ops<C>::R)theta);
  y[g] = make_double2((double)acc.x, (double)acc.y);
}

template <class C>
static void na_smooth(const Level& L, const C* inv, const double2* r, double2* y, C* pbuf, cudaStream_t st) {
  const PatchDev& P = L.P;
  const size_t sm = (size_t)P.max_n * sizeof(C) + 16;
  k_na_patch<C><<<(unsigned)P.nchunks, 256, sm, st>>>(P.ptr, P.dofs, P.val_ptr, P.chunks, inv, r, pbuf);
  DPG_CHECK_LAUNCH();
  const int64_t n = L.mesh.ndof;
  k_na_sum<C><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P.slot_ptr, P.slots, pbuf, y, n, L.theta);
  DPG_CHECK_LAUNCH();
}

}  // namespace dpgmg

using namespace dpgmg;

extern "C" int dpgmg_smooth_noalloc(dpgmg_handle h, dpgmg_system sys, int level, const double* r_dev,
                                    double* y_dev) {
  if (!h || !sys || !r_dev || !y_dev) return DPGMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  SystemImpl& S = sys->s;
  if (level < 1 || level >= (int)S.levels.size()) {
    set_last_error("dpgmg_smooth_noalloc: level must be 1..n_levels-1 (a level with a smoother)");
    return DPGMG_ERR_ARG;
  }
  const Level& L = S.levels[level];
  if (L.P.nslots > NOALLOC_MAX_SLOTS) {
    set_last_error("dpgmg_smooth_noalloc: level has " + std::to_string(L.P.nslots) +
                   " patch slots, above the fixed scratch of " + std::to_string(NOALLOC_MAX_SLOTS));
    return DPGMG_ERR_ARG;
  }
  try {
    DPG_CUDA(cudaSetDevice(h->h.device));
    void* scratch = noalloc_scratch(h->h.device);
    cudaStream_t st = h->h.stream;
    const double2* r = reinterpret_cast<const double2*>(r_dev);
    double2* y = reinterpret_cast<double2*>(y_dev);
    if (S.op.precision == DPGMG_PREC_MIXED)
      na_smooth<float2>(L, L.P.inv32, r, y, reinterpret_cast<float2*>(scratch), st);
    else
      na_smooth<double2>(L, L.P.inv64, r, y, reinterpret_cast<double2*>(scratch), st);
    DPG_CUDA(cudaStreamSynchronize(st));
    return DPGMG_OK;
  } catch (const Err& e) {
    set_last_error(e.msg);
    return e.code;
  }
}
