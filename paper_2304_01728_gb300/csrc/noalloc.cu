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
// looked up with cudaGetSymbolAddress, with the handle's device current, on
// every call (a cheap query), so a context the caller has reset and recreated
// in between is never given a stale address.
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "smoother.cuh"

namespace dpgmg {

constexpr int64_t NOALLOC_MAX_SLOTS = (int64_t)1 << 22;   // patch-product entries (complex128)

static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_MAX_SLOTS];

// Device address of the scratch array in the current device's context.
static void* noalloc_scratch() {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    throw Err{DPGMG_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
  }
  return p;
}

// The same smoother kernels as the solver (smoother.cuh), reading and
// writing complex128 vectors; scratch = the static array.
template <class C>
static void na_smooth(const Level& L, const C* inv_full, const C* inv_half, const double2* r, double2* y, C* scratch,
                      cudaStream_t st) {
  const PatchDev& P = L.P;
  const int64_t n = L.mesh.ndof;
  if (P.half && inv_half) {
    const int mx = 9 * HALF_MAX_N * (int)sizeof(C) + 16;
    DPG_CUDA(cudaFuncSetAttribute(k_patch_apply_h<C, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    const size_t sm = (size_t)9 * P.max_n * sizeof(C) + 16;
    k_patch_apply_h<C, double2><<<(unsigned)P.np, 256, sm, st>>>(P.ptr, P.dofs, P.hptr, inv_half, r, scratch);
  } else {
    const size_t sm = (size_t)P.max_n * sizeof(C) + 16;
    int64_t nch = 0;
    const int2* chunks = patch_chunks(P, PatchCols<C>::per, &nch);
    const uint8_t* rflag = std::is_same<C, float2>::value ? P.rflag : nullptr;   // packed complex64 inverses only
    k_patch_apply<C, double2><<<(unsigned)nch, 256, sm, st>>>(P.ptr, P.dofs, P.val_ptr, chunks, inv_full, r, scratch,
                                                              rflag, P.offU);
  }
  DPG_CHECK_LAUNCH();
  k_slot_sum<C, double2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P.slot_ptr, P.slots, scratch, y, n, L.theta, 0);
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
  if (L.P.recompute) {
    set_last_error("dpgmg_smooth_noalloc: the system recomputes its patches (no stored inverses)");
    return DPGMG_ERR_ARG;
  }
  if (L.P.scratch_entries() > NOALLOC_MAX_SLOTS) {
    set_last_error("dpgmg_smooth_noalloc: level needs " + std::to_string(L.P.scratch_entries()) +
                   " scratch entries, above the fixed scratch of " + std::to_string(NOALLOC_MAX_SLOTS));
    return DPGMG_ERR_ARG;
  }
  try {
    DPG_CUDA(cudaSetDevice(h->h.device));
    void* scratch = noalloc_scratch();
    cudaStream_t st = h->h.stream;
    const double2* r = reinterpret_cast<const double2*>(r_dev);
    double2* y = reinterpret_cast<double2*>(y_dev);
    if (S.op.precision == DPGMG_PREC_MIXED)
      na_smooth<float2>(L, L.P.inv32, L.P.h32, r, y, reinterpret_cast<float2*>(scratch), st);
    else
      na_smooth<double2>(L, L.P.inv64, nullptr, r, y, reinterpret_cast<double2*>(scratch), st);
    DPG_CUDA(cudaStreamSynchronize(st));
    return DPGMG_OK;
  } catch (const Err& e) {
    set_last_error(e.msg);
    return e.code;
  }
}
