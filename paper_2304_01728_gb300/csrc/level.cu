// DPG-MG hierarchy construction on the device (Sec. 3 of the paper):
//   * assembly of element matrices into the entity-shared CSR operator,
//   * p-transitions: restricted coarse operator = principal submatrix,
//   * h-transitions: macro-grid condensation per coarse element
//       M^K = A^K_SS - A^K_SI (A^K_II)^-1 A^K_IS     (stage one, "Prolongation")
//     and coarse operator by restriction A_c^K = I_K^T M^K I_K with the natural
//     inclusion I_K (stage two; "Alternative construction of coarse-grid
//     operators", restrict),
//   * vertex-patch blocks of the smoothing operator and their inverses
//     ("V-cycle and smoother"),
//   * the coarsest level (coarse.cu).
#include <algorithm>
#include <mutex>
#include <cstdlib>
#include <map>
#include <exception>
#include <thread>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "smoother.cuh"
#include "block.cuh"
#include "smoother.cuh"

namespace dpgmg {

// ------------------------------------------------------------ ECSR assembly
EcsrPrep prep_ecsr(const MeshL& m, const std::vector<std::vector<int64_t>>& groups) {
  EcsrPrep P;
  P.H = build_ecsr(m, groups);
  const ECSRHost& H = P.H;
  const int64_t nent = (int64_t)H.ent_start.size();
  for (int64_t E = 0; E < nent; ++E) P.max_nnz_row = std::max(P.max_nnz_row, H.col_ptr[E + 1] - H.col_ptr[E]);
  for (int gi = 1; gi <= 3; ++gi) {
    const int G = 1 << gi;
    for (int64_t E = 0; E < nent; ++E)
      for (int r0 = 0; r0 < H.ent_nd[E]; r0 += G) P.tasks[gi].push_back(make_int2((int)E, r0));
  }
  for (int64_t r = 0; r < H.nrows; ++r)
    if (H.row_ent[r] < 0) P.null_rows.push_back((int32_t)r);
  return P;
}

// Expanded column DOFs of the ECSR operator: row entity r (one warp) lists the
// DOF ranges of its column entities in order from col_ptr[r]; a warp-wide
// exclusive scan of the entities' DOF counts places each range.
__global__ void k_expand_cols(const int64_t* __restrict__ cent_ptr, const int32_t* __restrict__ col_ent,
                              const int64_t* __restrict__ col_ptr, EntRanges er, int64_t nent,
                              int32_t* __restrict__ col_idx) {
  const int lane = threadIdx.x & 31;
  const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nent) return;
  int64_t base = col_ptr[r];
  const int64_t q0 = cent_ptr[r], q1 = cent_ptr[r + 1];
  for (int64_t q = q0; q < q1; q += 32) {
    int64_t fs = 0;
    int fn = 0;
    if (q + lane < q1) er.range(col_ent[q + lane], &fs, &fn);
    int incl = fn;   // inclusive scan of the DOF counts over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    int32_t* out = col_idx + base + (incl - fn);
    for (int k = 0; k < fn; ++k) out[k] = (int32_t)(fs + k);
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
}

void assemble_ecsr(Alloc& A, const EcsrPrep& P, ECSRDev& D, cudaStream_t st) {
  const ECSRHost& H = P.H;
  D.nrows = H.nrows;
  D.nent = (int64_t)H.ent_start.size();
  D.nnz = H.nnz();
  D.nnz_alg = H.nnz_alg;
  D.row_ent = upload(A, H.row_ent, st);
  D.ent_start = upload(A, H.ent_start, st);
  D.ent_nd = upload(A, H.ent_nd, st);
  D.col_ptr = upload(A, H.col_ptr, st);
  {
    const int64_t ncols = H.col_ptr.empty() ? 0 : H.col_ptr.back();
    D.col_idx = A.arr<int32_t>((size_t)std::max<int64_t>(ncols, 1));
    if (D.nent > 0) {
      int64_t* cptr = upload(A, H.cent_ptr, st);
      int32_t* cent = upload(A, H.col_ent, st);
      k_expand_cols<<<(unsigned)((D.nent + 7) / 8), 256, 0, st>>>(cptr, cent, D.col_ptr, H.er, D.nent, D.col_idx);
      DPG_CHECK_LAUNCH();
      A.release(cent);   // stream-ordered frees: after the expansion
      A.release(cptr);
    }
  }
  D.val_ptr = upload(A, H.val_ptr, st);
  D.max_nnz_row = P.max_nnz_row;
  for (int gi = 1; gi <= 3; ++gi) {
    D.ntasks[gi] = (int64_t)P.tasks[gi].size();
    D.tasks[gi] = P.tasks[gi].empty() ? nullptr : upload(A, P.tasks[gi], st);
  }
  D.n_null = (int64_t)P.null_rows.size();
  D.null_rows = P.null_rows.empty() ? nullptr : upload(A, P.null_rows, st);
  D.v64 = A.arr<double2>((size_t)D.nnz);
  DPG_CUDA(cudaMemsetAsync(D.v64, 0, (size_t)D.nnz * sizeof(double2), st));
}

__device__ __forceinline__ int64_t ecsr_find(const ECSRDev& A, int64_t row, int64_t col) {
  int32_t E = A.row_ent[row];
  if (E < 0) return -1;
  int64_t c0 = A.col_ptr[E], c1 = A.col_ptr[E + 1];
  int64_t lo = c0, hi = c1;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (A.col_idx[mid] < col) lo = mid + 1;
    else hi = mid;
  }
  if (lo >= c1 || A.col_idx[lo] != col) return -1;
  int64_t r = row - A.ent_start[E];
  return A.val_ptr[E] + r * (c1 - c0) + (lo - c0);
}

__device__ __forceinline__ double2 widen(double2 a) { return a; }
__device__ __forceinline__ double2 widen(float2 a) { return make_double2(a.x, a.y); }   // exact

// block (e, s): slice s of element e's entries (the slices of one element are
// disjoint); TE = double2, or float2 for the mixed path's complex64 macro
// element matrices (widened exactly)
template <class TE>
__global__ void k_ecsr_add(ECSRDev A, const TE* E, const int64_t* dofs, int64_t nel, int nloc, int64_t e0,
                           int n0, int n1, int color) {
  const int64_t e = blockIdx.x;
  if (elem_color(e0 + e, n0, n1) != color) return;
  const TE* Ee = E + e * (size_t)nloc * nloc;
  const int64_t* g = dofs + e * nloc;
  for (int q = blockIdx.y * blockDim.x + threadIdx.x; q < nloc * nloc; q += gridDim.y * blockDim.x) {
    int i = q / nloc, j = q % nloc;
    int64_t gi = g[i], gj = g[j];
    if (gi < 0 || gj < 0) continue;
    int64_t pos = ecsr_find(A, gi, gj);
    if (pos < 0) continue;
    const double2 v = widen(Ee[q]);
    double2& o = A.v64[pos];
    o = make_double2(o.x + v.x, o.y + v.y);
  }
}

template <class TE>
static void ecsr_add_t(ECSRDev& D, const TE* E, const int64_t* dofs, int64_t nel, int nloc, int64_t e0,
                       const int ext[3], cudaStream_t st) {
  if (nel == 0) return;
  // one colour holds ~nel / 8 elements: slices of ~2048 entries per block keep the passes wide
  const unsigned slices = (unsigned)std::max<int64_t>(1, std::min<int64_t>(64, ((int64_t)nloc * nloc + 2047) / 2048));
  for (int c = 0; c < 8; ++c) {
    k_ecsr_add<TE><<<dim3((unsigned)nel, slices), 256, 0, st>>>(D, E, dofs, nel, nloc, e0, ext[0], ext[1], c);
    DPG_CHECK_LAUNCH();
  }
}

void ecsr_add_elements(ECSRDev& D, const double2* E, const int64_t* dofs, int64_t nel, int nloc, int64_t e0,
                       const int ext[3], cudaStream_t st) {
  ecsr_add_t<double2>(D, E, dofs, nel, nloc, e0, ext, st);
}

std::vector<std::vector<int64_t>> element_groups(const MeshL& m) {
  std::vector<std::vector<int64_t>> g(m.nelem);
  host_parallel(m.nelem, [&](int64_t lo, int64_t hi) {
    std::vector<int64_t> ent(m.loc.size());
    for (int64_t e = lo; e < hi; ++e) {
      m.elem_entities(e, ent.data());
      for (int64_t E : ent)
        if (E >= 0) g[e].push_back(E);
      std::sort(g[e].begin(), g[e].end());
      g[e].erase(std::unique(g[e].begin(), g[e].end()), g[e].end());
    }
  });
  return g;
}

static std::vector<int64_t> elem_dof_table(const MeshL& m) {
  std::vector<int64_t> d((size_t)m.nelem * m.loc.size());
  for (int64_t e = 0; e < m.nelem; ++e) m.elem_dofs(e, d.data() + e * m.loc.size());
  return d;
}

// ------------------------------------------------------------ p-transition
__global__ void k_p_restrict(const double2* Ef, double2* Ec, const int32_t* sel, int nf, int nc) {
  const int64_t e = blockIdx.x;
  for (int q = threadIdx.x; q < nc * nc; q += blockDim.x) {
    int i = q / nc, j = q % nc;
    Ec[e * (size_t)nc * nc + q] = Ef[e * (size_t)nf * nf + (size_t)sel[i] * nf + sel[j]];
  }
}

// Mixed path: patch blocks gathered as complex64 and factored in FP32 (the
// V-cycle's precision), unless DPGMG_FLAG_PATCH_FP64 asks for FP64 factors
// rounded to complex64 afterwards.
static bool patches_fp32(const SystemImpl& S) {
  return S.op.precision == DPGMG_PREC_MIXED && !(S.op.flags & DPGMG_FLAG_PATCH_FP64);
}
// Mixed path: macro condensation and restriction in complex64 (same option).
// With stored coarse operators the coarse element matrices come from the
// element stage; the macro operators and transfers are still complex64.
static bool macro_fp32(const SystemImpl& S) { return patches_fp32(S); }

// ------------------------------------------------------------ h-transition
// C = double2 (FP64 path), or float2 on the mixed path: every output of the
// macro condensation (macro element matrices, transfer blocks Y and A_II^-1,
// restricted coarse element matrices) feeds only the V-cycle, which runs in
// complex64 there; the fine element matrices are rounded on load and the
// outputs that are stored in FP64 (coarse element matrices) are widened.
template <class C>
struct MacroArgs {
  int nS, nI, nlf, nlc;
  int64_t K0;
  const double2* Ef;          // fine element matrices
  const int64_t* fdofs;       // fine element DOFs
  const int32_t* child_map;   // [8][nlf]
  int nf0, nf1;               // fine mesh extents x, y
  int nc0, nc1;               // coarse mesh extents x, y
  const C* IK;                // [nS][nlc] (real values)
  C* AK;                      // scratch [chunk][(nS+nI)^2]
  C* T1;                      // scratch [chunk][nS][nlc]
  C* MK;                      // out [chunk][nS][nS]
  C* Y;                       // out [nK][nI][nS]
  C* Ai;                      // out [nK][nI][nI]
  C* Ec;                      // scratch [chunk][nlc][nlc] (C = float2), or null: written to EcOut directly
  double2* EcOut;             // out [nK][nlc][nlc]
  int* info;
};

template <class C>
__global__ void __launch_bounds__(CTA_THREADS) k_macro(MacroArgs<C> a) {
  extern __shared__ unsigned char shm[];
  C* sh2 = reinterpret_cast<C*>(shm);
  using O = Ops<C>;
  using R = typename O::R;
  const int64_t lk = blockIdx.x;
  const int64_t K = a.K0 + lk;
  const int nS = a.nS, nI = a.nI, n = nS + nI;
  C* AK = a.AK + lk * (size_t)n * n;
  for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += blockDim.x) AK[q] = O::zero();
  __syncthreads();
  int kc[3];
  kc[0] = (int)(K % a.nc0);
  kc[1] = (int)((K / a.nc0) % a.nc1);
  kc[2] = (int)(K / ((int64_t)a.nc0 * a.nc1));
  for (int o = 0; o < 8; ++o) {
    int fc[3] = {2 * kc[0] + (o & 1), 2 * kc[1] + ((o >> 1) & 1), 2 * kc[2] + ((o >> 2) & 1)};
    int64_t fe = fc[0] + (int64_t)a.nf0 * (fc[1] + (int64_t)a.nf1 * fc[2]);
    const double2* E = a.Ef + fe * (size_t)a.nlf * a.nlf;
    const int64_t* g = a.fdofs + fe * a.nlf;
    const int32_t* cm = a.child_map + o * a.nlf;
    for (int q = threadIdx.x; q < a.nlf * a.nlf; q += blockDim.x) {
      int i = q / a.nlf, j = q % a.nlf;
      if (g[i] < 0 || g[j] < 0) continue;
      C& t = AK[(size_t)cm[i] * n + cm[j]];
      const double2 v = E[q];
      t = O::add(t, O::mk((R)v.x, (R)v.y));
    }
    __syncthreads();
  }
  // Cholesky of A_II (trailing block), Y = A_II^-1 A_IS (in place of A_IS)
  C* AII = AK + (size_t)nS * n + nS;
  int info = cta_potrf<C>(AII, nI, n, sh2);
  if (threadIdx.x == 0 && info) atomicOr(a.info, 4);
  C* AIS = AK + (size_t)nS * n;
  cta_trsm_lower<C, C>(AII, nI, n, AIS, nS, n, reinterpret_cast<char*>(sh2));
  cta_trsm_lower_h<C>(AII, nI, n, AIS, nS, n, reinterpret_cast<char*>(sh2));
  // M^K = A_SS - A_SI Y
  C* MK = a.MK + lk * (size_t)nS * nS;
  for (int q = threadIdx.x; q < nS * nS; q += blockDim.x) MK[q] = AK[(size_t)(q / nS) * n + (q % nS)];
  __syncthreads();
  cta_gemm<C>(false, nS, nS, nI, R(-1), AK + nS, n, AIS, n, R(1), MK, nS, sh2);
  // store Y and A_II^-1
  C* Y = a.Y + K * (size_t)nI * nS;
  for (int q = threadIdx.x; q < nI * nS; q += blockDim.x) Y[q] = AIS[(size_t)(q / nS) * n + (q % nS)];
  C* Ai = a.Ai + K * (size_t)nI * nI;
  for (int q = threadIdx.x; q < nI * nI; q += blockDim.x) Ai[q] = (q / nI == q % nI) ? O::from_re(R(1)) : O::zero();
  __syncthreads();
  cta_trsm_lower<C, C>(AII, nI, n, Ai, nI, nI, reinterpret_cast<char*>(sh2));
  cta_trsm_lower_h<C>(AII, nI, n, Ai, nI, nI, reinterpret_cast<char*>(sh2));
  // restriction: E_c = I_K^T (M^K I_K)
  C* T1 = a.T1 + lk * (size_t)nS * a.nlc;
  cta_gemm<C>(false, nS, a.nlc, nS, R(1), MK, nS, a.IK, a.nlc, R(0), T1, a.nlc, sh2);
  double2* Eo = a.EcOut + K * (size_t)a.nlc * a.nlc;
  if constexpr (sizeof(C) == sizeof(double2)) {
    cta_gemm<C>(true, a.nlc, a.nlc, nS, R(1), a.IK, a.nlc, T1, a.nlc, R(0), reinterpret_cast<C*>(Eo), a.nlc, sh2);
  } else {
    C* Ec = a.Ec + lk * (size_t)a.nlc * a.nlc;
    cta_gemm<C>(true, a.nlc, a.nlc, nS, R(1), a.IK, a.nlc, T1, a.nlc, R(0), Ec, a.nlc, sh2);
    __syncthreads();
    for (int q = threadIdx.x; q < a.nlc * a.nlc; q += blockDim.x) Eo[q] = widen(Ec[q]);
  }
}

template <class C>
static void macro_condense(SystemImpl& S, Level& F, Level& C_, const MacroHost& M, const int32_t* cmap, int* dinfo,
                           C* Y, C* Ai, cudaStream_t st) {
  Alloc& A = S.mem;
  std::vector<C> ik(M.IK.size());
  for (size_t i = 0; i < ik.size(); ++i) {
    ik[i].x = (typename Ops<C>::R)M.IK[i];
    ik[i].y = 0;
  }
  C* dIK = upload(A, ik, st);
  const int n = F.nS + F.nI;
  int64_t chunk = std::min<int64_t>(F.nK, 2048);
  C* AK = A.arr<C>((size_t)chunk * n * n);
  C* T1 = A.arr<C>((size_t)chunk * F.nS * C_.nloc);
  C* MK = A.arr<C>((size_t)chunk * F.nS * F.nS);
  C* Ec = sizeof(C) == sizeof(double2) ? nullptr : A.arr<C>((size_t)chunk * C_.nloc * C_.nloc);
  MacroArgs<C> a{};
  a.nS = F.nS; a.nI = F.nI; a.nlf = F.nloc; a.nlc = C_.nloc;
  a.Ef = F.E; a.fdofs = F.dofs; a.child_map = cmap;
  a.nf0 = F.mesh.n[0]; a.nf1 = F.mesh.n[1];
  a.nc0 = C_.mesh.n[0]; a.nc1 = C_.mesh.n[1];
  a.IK = dIK; a.AK = AK; a.T1 = T1; a.MK = MK;
  a.Y = Y; a.Ai = Ai; a.Ec = Ec; a.EcOut = C_.E; a.info = dinfo;
  const size_t sm = (size_t)(NB * NB + 2 * TL * NB) * sizeof(C) + 64;
  DPG_CUDA(cudaFuncSetAttribute(k_macro<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  for (int64_t K0 = 0; K0 < F.nK; K0 += chunk) {
    a.K0 = K0;
    int nb = (int)std::min<int64_t>(chunk, F.nK - K0);
    k_macro<C><<<nb, CTA_THREADS, sm, st>>>(a);
    DPG_CHECK_LAUNCH();
    ecsr_add_t<C>(F.A, MK, F.S_glob + K0 * F.nS, nb, F.nS, K0, C_.mesh.n, st);
  }
  A.release(AK);   // stream-ordered frees: after the launches above
  A.release(T1);
  A.release(MK);
  if (Ec) A.release(Ec);
  A.release(dIK);
}

// ------------------------------------------------------------------ patches
// Patch block R_j A R_j^T, read from the operator's FP64 values; C = float2
// rounds every entry to complex64 (the mixed path factors in FP32).
// The patch of CTA b is j0 + b, or order[j0 + b] when an order is given.
template <class C>
__global__ void k_patch_gather(ECSRDev A, const int64_t* ptr, const int32_t* dofs, const int64_t* vptr, C* out,
                               int64_t j0, const int64_t* order = nullptr) {
  const int64_t j = order ? order[j0 + blockIdx.x] : j0 + blockIdx.x;
  const int64_t b = ptr[j];
  const int n = (int)(ptr[j + 1] - b);
  const int ld = (int)patch_ld(n);
  C* M = out + vptr[j];
  for (int q = threadIdx.x; q < n * ld; q += blockDim.x) {
    int r = q / ld, c = q % ld;
    int64_t pos = c < n ? ecsr_find(A, dofs[b + r], dofs[b + c]) : -1;
    const double2 v = pos >= 0 ? A.v64[pos] : make_double2(0, 0);
    M[q] = Ops<C>::mk((typename Ops<C>::R)v.x, (typename Ops<C>::R)v.y);
  }
}

// Unit phases of the real form (mul_i, smoother.cuh): p-hat DOFs (global
// index < offU) carry i, u-hat DOFs carry 1.  rot(v, a, b) = conj(beta_a) v
// beta_b and its inverse unrot(x, a, b) = beta_a x conj(beta_b); multiplying
// by +-i only swaps components, so both are exact.

// In place: M (n x n) -> M^-1 via Cholesky in the scratch copy W.
// Real path: on a patch whose block is real after the unit phases are removed
// (every element touching it runs the real element path, so its entries are
// exactly phased: the test below is exact), Cholesky, triangular inverse and
// L^-H L^-1 run in real arithmetic (a quarter of the flops) and the phases
// are put back on the inverse.  Other patches take the complex path.
// CL: one patch per thread-block cluster; the cluster's CTAs share every
// dense step (Team<true>), which spreads a large patch over several SMs.
// rpack (optional, one byte per patch): a real-path patch then stores its
// inverse as the real matrix w with A^-1[r][c] = w[r][c] i^(s_r - s_c) (s = 1
// on p-hat DOFs), n rows of patch_ldr(n) reals at the start of its block, and
// sets rpack[j] = 1; a complex patch stores the complex inverse and sets 0.
// The smoother then streams half the bytes of a real patch (smoother.cuh).
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

template <class C, bool CL>
__global__ void __launch_bounds__(CTA_THREADS) k_patch_invert(const int64_t* ptr, const int32_t* pdofs,
                                                            const int64_t* vptr, C* vals, C* scratch,
                                                            const int64_t* soff, const int64_t* order, int64_t j0,
                                                            int64_t offU, int* info, uint8_t* rpack) {
  extern __shared__ unsigned char shraw[];
  C* sh = reinterpret_cast<C*>(shraw);
  Team<CL> tm;
  if constexpr (CL) {
    tm.rank = (int)cluster_rank();
    tm.n = (int)cluster_size();
  }
  const int64_t slot = blockIdx.x / tm.n;
  const int64_t j = order[j0 + slot];
  const int64_t b = ptr[j];
  const int n = (int)(ptr[j + 1] - b);
  const int ld = (int)patch_ld(n);   // stored row length; column n (if any) is padding, left 0
  C* M = vals + vptr[j];
  C* W = scratch + soff[j0 + slot];
  using R = typename Ops<C>::R;
  bool cplx = false;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    const int r = q / n, c = q % n;
    const int sr = pdofs[b + r] < offU ? 1 : 0, sc = pdofs[b + c] < offU ? 1 : 0;
    const C v = mul_i(M[(size_t)r * ld + c], sc - sr);
    if (v.y != R(0)) cplx = true;
  }
  if (!__syncthreads_or(cplx)) {
    R* Wr = reinterpret_cast<R*>(W);
    R* Mr = reinterpret_cast<R*>(M);   // L^-1 (n x n, row length n) in the block's storage
    R* shr = reinterpret_cast<R*>(shraw);
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
      const int r = q / n, c = q % n;
      if (!tm.own_row(r / TL)) continue;
      const int sr = pdofs[b + r] < offU ? 1 : 0, sc = pdofs[b + c] < offU ? 1 : 0;
      Wr[q] = mul_i(M[(size_t)r * ld + c], sc - sr).x;
    }
    tm.sync();   // every CTA has read M before any overwrites it
    int inf = cta_potrf<R, CL>(Wr, n, n, shr, tm);
    if (threadIdx.x == 0 && inf && tm.rank == 0) atomicOr(info, 8);
    for (int q = threadIdx.x; q < n * n; q += blockDim.x)
      if (tm.own_row((q / n) / TL)) Mr[q] = (q / n == q % n) ? R(1) : R(0);
    tm.sync();
    cta_trinv_lower<R, CL>(Wr, n, n, Mr, n, reinterpret_cast<char*>(shr), tm);
    tm.sync();
    cta_herk_lower_tri<R, CL>(Mr, n, n, Wr, n, shr, tm);
    tm.sync();
    if (rpack) {   // real rows of length ldr (padding columns 0) over the L^-1 copy, no longer read
      const int ldr = (int)patch_ldr(n);
      for (int q = threadIdx.x; q < n * ldr; q += blockDim.x) {
        const int r = q / ldr, c = q % ldr;
        if (tm.own_row(r / TL)) Mr[q] = c < n ? tm.ld(&Wr[(size_t)r * n + c]) : R(0);
      }
      if (threadIdx.x == 0 && tm.rank == 0) rpack[j] = 1;
      return;
    }
    for (int q = threadIdx.x; q < n * ld; q += blockDim.x) {
      const int r = q / ld, c = q % ld;
      if (!tm.own_row(r / TL)) continue;
      const int sr = pdofs[b + r] < offU ? 1 : 0, sc = c < n && pdofs[b + c] < offU ? 1 : 0;
      M[q] = c < n ? mul_i(Ops<C>::mk(tm.ld(&Wr[(size_t)r * n + c]), R(0)), sr - sc) : Ops<C>::zero();
    }
    return;
  }
  if (rpack && threadIdx.x == 0 && tm.rank == 0) rpack[j] = 0;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x)
    if (tm.own_row((q / n) / TL)) W[q] = M[(size_t)(q / n) * ld + q % n];
  tm.sync();
  int inf = cta_potrf<C, CL>(W, n, n, sh, tm);
  if (threadIdx.x == 0 && inf && tm.rank == 0) atomicOr(info, 8);
  // M = L^-1 (lower, row length ld), then W = L^-H L^-1 = A^-1, copied back into M
  for (int q = threadIdx.x; q < n * ld; q += blockDim.x)
    if (tm.own_row((q / ld) / TL)) M[q] = (q / ld == q % ld) ? Ops<C>::from_re(1) : Ops<C>::zero();
  tm.sync();
  cta_trinv_lower<C, CL>(W, n, n, M, ld, reinterpret_cast<char*>(sh), tm);
  tm.sync();
  cta_herk_lower_tri<C, CL>(M, n, ld, W, n, sh, tm);
  tm.sync();
  for (int q = threadIdx.x; q < n * ld; q += blockDim.x) {
    const int r = q / ld, c = q % ld;
    if (!tm.own_row(r / TL)) continue;
    M[q] = c < n ? tm.ld(&W[(size_t)r * n + c]) : Ops<C>::zero();
  }
}

// --------------------------------------------------------------- precision
__global__ void k_to_c64(const double2* a, float2* b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
static float2* to_c64(Alloc& A, const double2* src, int64_t n, cudaStream_t st) {
  float2* d = A.arr<float2>((size_t)std::max<int64_t>(n, 1));
  if (n > 0) {
    k_to_c64<<<1216, 256, 0, st>>>(src, d, n);
    DPG_CHECK_LAUNCH();
  }
  return d;
}

// --------------------------------------------------------------- rhs
__global__ void k_rhs(const double2* Fc, const int64_t* dofs, double2* b, int64_t nel, int nloc, int n0, int n1,
                      int color) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nel * nloc || elem_color(q / nloc, n0, n1) != color) return;
  int64_t g = dofs[q];
  if (g < 0) return;
  b[g] = make_double2(b[g].x + Fc[q].x, b[g].y + Fc[q].y);
}

void assemble_rhs(SystemImpl& S, cudaStream_t st) {
  const Level& L = S.levels.back();
  S.b = S.mem.arr<double2>((size_t)L.mesh.ndof);
  DPG_CUDA(cudaMemsetAsync(S.b, 0, (size_t)L.mesh.ndof * sizeof(double2), st));
  int64_t n = S.nelem * S.ntr;
  for (int c = 0; c < 8; ++c) {   // colour passes (see elem_color)
    k_rhs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S.Fc, L.dofs, S.b, S.nelem, (int)S.ntr, L.mesh.n[0],
                                                       L.mesh.n[1], c);
    DPG_CHECK_LAUNCH();
  }
}

// Hermitian half storage of the complex64 patch inverses halves the smoother's
// bytes, but the tiled half-storage product (k_patch_apply_h) measured 0.233 ms
// per finest application on the 16^3 p=3 workload against 0.187 ms for the
// full-storage product, so full storage is the default.
constexpr bool kHalfStorageSmoother = false;

// --------------------------------------------------------------- driver
// Invert all patch blocks in place, in chunks that bound the scratch copy.
// CTAs per patch.  A level with few large patches (the macro patches of an
// h-level) leaves most SMs idle while a handful of them factor the largest
// blocks one CTA each; a cluster of 2 or 4 CTAs per patch spreads those over
// several SMs.  Chosen so that the level has at least ~4 largest-patch shares
// per SM; DPGMG_PATCH_TEAM = 1, 2 or 4 overrides the choice.
static int patch_team(const Patches& P, int64_t max_n) {
  if (const char* e = std::getenv("DPGMG_PATCH_TEAM")) {
    const int t = std::atoi(e);
    if (t == 1 || t == 2 || t == 4) return t;
  }
  if (max_n < 96) return 1;
  int dev = 0, nsm = 0;
  DPG_CUDA(cudaGetDevice(&dev));
  DPG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  double sum = 0.0;
  for (size_t j = 0; j + 1 < P.ptr.size(); ++j) {
    const double nj = (double)(P.ptr[j + 1] - P.ptr[j]);
    sum += nj * nj * nj;
  }
  const double shares = sum / ((double)max_n * max_n * max_n);
  int t = 1;
  while (t < 4 && shares * t < 4.0 * nsm) t *= 2;
  return t;
}

template <class C>
static void invert_patches(Alloc& A, PatchDev& D, const LevelPlan& lp, C* vals, int64_t offU, int* dinfo,
                           cudaStream_t st, uint8_t* rpack = nullptr) {
  const Patches& P = lp.P;
  const size_t sm = (size_t)(NB * NB + 2 * TL * NB) * sizeof(C) + 64;
  DPG_CUDA(cudaFuncSetAttribute(k_patch_invert<C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  DPG_CUDA(cudaFuncSetAttribute(k_patch_invert<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int team = patch_team(P, D.max_n);
  cudaLaunchAttribute cattr[1];
  cattr[0].id = cudaLaunchAttributeClusterDimension;
  cattr[0].val.clusterDim.x = (unsigned)team;
  cattr[0].val.clusterDim.y = 1;
  cattr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(CTA_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cfg.attrs = cattr;
  cfg.numAttrs = 1;
  if (team > 1) {
    cfg.gridDim = dim3((unsigned)team);
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_patch_invert<C, true>, &cfg) != cudaSuccess || ncl < 1) {
      (void)cudaGetLastError();
      team = 1;
    }
  }
  const size_t one = (size_t)D.max_n * D.max_n;
  size_t cap = std::min<size_t>(std::max<size_t>(((size_t)1 << 28) / sizeof(C), one) * 4, ((size_t)2 << 30) / sizeof(C));
  cap = std::max(std::min<size_t>(cap, (size_t)D.nvals), one);
  C* scratch = A.arr<C>(cap);
  // launches of consecutive patches (largest first) whose scratch copies fit
  // `cap`; offs[q] = scratch offset of the q-th patch within its launch
  const std::vector<int64_t>& order = lp.order;
  std::vector<int64_t> offs(D.np), starts;
  for (int64_t q = 0, acc = 0; q < D.np; ++q) {
    const int64_t j = order[q];
    const int64_t nj = P.ptr[j + 1] - P.ptr[j];
    if (q == 0 || acc + nj * nj > (int64_t)cap) {
      starts.push_back(q);
      acc = 0;
    }
    offs[q] = acc;
    acc += nj * nj;
  }
  starts.push_back(D.np);
  int64_t* soff = upload(A, offs, st);
  int64_t* dorder = upload(A, order, st);
  for (size_t c = 0; c + 1 < starts.size(); ++c) {
    const int64_t j0 = starts[c], q = starts[c + 1];
    if (team == 1) {
      k_patch_invert<C, false><<<(unsigned)(q - j0), CTA_THREADS, sm, st>>>(D.ptr, D.dofs, D.val_ptr, vals, scratch,
                                                                          soff, dorder, j0, offU, dinfo, rpack);
      DPG_CHECK_LAUNCH();
    } else {
      cfg.gridDim = dim3((unsigned)((q - j0) * team));
      DPG_CUDA(cudaLaunchKernelEx(&cfg, k_patch_invert<C, true>, (const int64_t*)D.ptr, (const int32_t*)D.dofs,
                                  (const int64_t*)D.val_ptr, vals, scratch, (const int64_t*)soff,
                                  (const int64_t*)dorder, j0, offU, dinfo, rpack));
      count_launch();
    }
  }
  A.release(dorder);
  A.release(soff);
  A.release(scratch);
}


// Windows of the recompute mode (see PatchDev): consecutive patches of the
// largest-first order whose n x ld blocks fit wcap entries: a quarter of the
// level's blocks, at most 256 MiB of complex64, at least the largest block.
static void setup_recompute(Alloc& A, PatchDev& D, const LevelPlan& lp, int64_t offU, const ECSRDev& Aop,
                            int* dinfo, cudaStream_t st) {
  const Patches& P = lp.P;
  const int64_t one = D.max_n * patch_ld(D.max_n);
  D.wcap = std::max<int64_t>(one, std::min<int64_t>((D.nvals + 3) / 4, (int64_t)32 << 20));
  std::vector<int64_t> wvptr(D.np), wsoff(D.np);
  std::vector<int2> ch;
  D.wq.clear();
  D.wch.clear();
  for (int64_t q = 0, acc = 0; q < D.np; ++q) {
    const int64_t j = lp.order[q];
    const int64_t nj = P.ptr[j + 1] - P.ptr[j];
    const int64_t sz = nj * patch_ld(nj);
    if (q == 0 || acc + sz > D.wcap) {
      D.wq.push_back(q);
      D.wch.push_back((int64_t)ch.size());
      acc = 0;
    }
    wvptr[j] = acc;
    wsoff[q] = acc;   // the n x n scratch copy fits in the n x ld block's extent
    acc += sz;
    for (int64_t a0 = 0; a0 < nj; a0 += 64) ch.push_back(make_int2((int)j, (int)a0));
  }
  D.wq.push_back(D.np);
  D.wch.push_back((int64_t)ch.size());
  D.worder = upload(A, lp.order, st);
  D.wvptr = upload(A, wvptr, st);
  D.wsoff = upload(A, wsoff, st);
  D.wchunks = upload(A, ch, st);
  D.wbuf = A.arr<float2>((size_t)D.wcap);
  D.wscratch = A.arr<float2>((size_t)D.wcap);
  D.winfo = A.arr<int>(1);
  DPG_CUDA(cudaMemsetAsync(D.winfo, 0, sizeof(int), st));
  D.recompute = true;
  const size_t sm = (size_t)(NB * NB + 2 * TL * NB) * sizeof(float2) + 64;
  DPG_CUDA(cudaFuncSetAttribute(k_patch_invert<float2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  // one pass over every block now, so that a non-HPD block fails the setup
  for (size_t w = 0; w + 1 < D.wq.size(); ++w) {
    const int64_t q0 = D.wq[w], q1 = D.wq[w + 1];
    k_patch_gather<float2><<<(unsigned)(q1 - q0), 256, 0, st>>>(Aop, D.ptr, D.dofs, D.wvptr, D.wbuf, q0, D.worder);
    DPG_CHECK_LAUNCH();
    k_patch_invert<float2, false><<<(unsigned)(q1 - q0), CTA_THREADS, sm, st>>>(
        D.ptr, D.dofs, D.wvptr, D.wbuf, D.wscratch, D.wsoff, D.worder, q0, offU, dinfo, nullptr);
    DPG_CHECK_LAUNCH();
  }
}

void patch_recompute_apply(const Level& L, const float2* r, float2* pbuf, cudaStream_t st) {
  const PatchDev& D = L.P;
  const size_t smi = (size_t)(NB * NB + 2 * TL * NB) * sizeof(float2) + 64;
  const size_t sma = (size_t)D.max_n * sizeof(float2) + 16;
  for (size_t w = 0; w + 1 < D.wq.size(); ++w) {
    const int64_t q0 = D.wq[w], q1 = D.wq[w + 1];
    k_patch_gather<float2><<<(unsigned)(q1 - q0), 256, 0, st>>>(L.A, D.ptr, D.dofs, D.wvptr, D.wbuf, q0, D.worder);
    DPG_CHECK_LAUNCH();
    k_patch_invert<float2, false><<<(unsigned)(q1 - q0), CTA_THREADS, smi, st>>>(
        D.ptr, D.dofs, D.wvptr, D.wbuf, D.wscratch, D.wsoff, D.worder, q0, L.mesh.offU, D.winfo, nullptr);
    DPG_CHECK_LAUNCH();
    const int64_t c0 = D.wch[w], c1 = D.wch[w + 1];
    k_patch_apply<float2, float2, 2><<<(unsigned)(c1 - c0), 256, sma, st>>>(D.ptr, D.dofs, D.wvptr, D.wchunks + c0,
                                                                            D.wbuf, r, pbuf, nullptr, 0);
    DPG_CHECK_LAUNCH();
  }
}

// The same for K vectors (r and pbuf at strides ldr and ldp): every window is
// gathered and factored once for all K.
void patch_recompute_apply_blk(const Level& L, const float2* r, int64_t ldr, float2* pbuf, int64_t ldp, int K,
                               cudaStream_t st) {
  const PatchDev& D = L.P;
  const size_t smi = (size_t)(NB * NB + 2 * TL * NB) * sizeof(float2) + 64;
  static std::once_flag once;
  std::call_once(once, []() {
    const int mx = 160 * 1024;   // + the kernel's static shared memory (37 KiB) stays within 227 KiB
    DPG_CUDA(cudaFuncSetAttribute(k_patch_apply_blk<float2, float2, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    DPG_CUDA(cudaFuncSetAttribute(k_patch_apply_blk<float2, float2, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    DPG_CUDA(cudaFuncSetAttribute(k_patch_apply_blk<float2, float2, 2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    DPG_CUDA(cudaFuncSetAttribute(k_patch_apply_blk<float2, float2, 2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  });
  for (size_t w = 0; w + 1 < D.wq.size(); ++w) {
    const int64_t q0 = D.wq[w], q1 = D.wq[w + 1];
    k_patch_gather<float2><<<(unsigned)(q1 - q0), 256, 0, st>>>(L.A, D.ptr, D.dofs, D.wvptr, D.wbuf, q0, D.worder);
    DPG_CHECK_LAUNCH();
    k_patch_invert<float2, false><<<(unsigned)(q1 - q0), CTA_THREADS, smi, st>>>(
        D.ptr, D.dofs, D.wvptr, D.wbuf, D.wscratch, D.wsoff, D.worder, q0, L.mesh.offU, D.winfo, nullptr);
    DPG_CHECK_LAUNCH();
    const int64_t c0 = D.wch[w], c1 = D.wch[w + 1];
    for (int g = 0; g < K; g += BLK_MAX) {
      const int kb = std::min(BLK_MAX, K - g);
      const size_t sm = (size_t)kb * D.max_n * sizeof(float2) + 16;
#define DPG_RC_BLK(KB)                                                                                     \
  k_patch_apply_blk<float2, float2, 2, KB><<<(unsigned)(c1 - c0), 256, sm, st>>>(                          \
      D.ptr, D.dofs, D.wvptr, D.wchunks + c0, D.wbuf, r + (int64_t)g * ldr, ldr, pbuf + (int64_t)g * ldp, ldp, \
      nullptr, 0)
      if (kb == 4) DPG_RC_BLK(4);
      else if (kb == 3) DPG_RC_BLK(3);
      else if (kb == 2) DPG_RC_BLK(2);
      else DPG_RC_BLK(1);
#undef DPG_RC_BLK
      DPG_CHECK_LAUNCH();
    }
  }
}

static void setup_patches(SystemImpl& S, Level& F, const LevelPlan& lp, int* dinfo, cudaStream_t st) {
  Alloc& A = S.mem;
  const Patches& P = lp.P;
  PatchDev& D = F.P;
  D.np = (int64_t)P.ptr.size() - 1;
  D.nslots = (int64_t)P.dofs.size();
  D.nvals = P.val_ptr.back();
  D.max_n = lp.max_n;
  D.sum_sq = lp.sum_sq;
  D.offU = F.mesh.offU;
  D.ptr = upload(A, P.ptr, st);
  D.dofs = upload(A, P.dofs, st);
  D.val_ptr = upload(A, P.val_ptr, st);
  D.slot_ptr = upload(A, P.slot_ptr, st);
  D.slots = upload(A, P.slots, st);
  D.nchunks = (int64_t)lp.ch32.size();
  D.chunks = upload(A, lp.ch32, st);
  D.nchunks64 = (int64_t)lp.ch64.size();
  D.chunks64 = upload(A, lp.ch64, st);
  if (S.op.flags & DPGMG_FLAG_RECOMPUTE_PATCHES) {
    setup_recompute(A, D, lp, F.mesh.offU, F.A, dinfo, st);
    return;
  }
  if (patches_fp32(S)) {
    // complex64 blocks, Cholesky, triangular inverse and L^-H L^-1 in FP32; the
    // smoother and its damping estimate use exactly these inverses
    D.inv32 = A.arr<float2>((size_t)std::max<int64_t>(D.nvals, 1));
    k_patch_gather<float2><<<(unsigned)D.np, 256, 0, st>>>(F.A, D.ptr, D.dofs, D.val_ptr, D.inv32, 0);
    DPG_CHECK_LAUNCH();
    // real-path patches keep real inverses (half the smoother's bytes for them)
    if (pack_storage(S)) {
      D.rflag = A.arr<uint8_t>((size_t)std::max<int64_t>(D.np, 1));
      DPG_CUDA(cudaMemsetAsync(D.rflag, 0, (size_t)std::max<int64_t>(D.np, 1), st));
    }
    invert_patches<float2>(A, D, lp, D.inv32, F.mesh.offU, dinfo, st, D.rflag);
    return;
  }
  D.inv64 = A.arr<double2>((size_t)D.nvals);
  k_patch_gather<double2><<<(unsigned)D.np, 256, 0, st>>>(F.A, D.ptr, D.dofs, D.val_ptr, D.inv64, 0);
  DPG_CHECK_LAUNCH();
  // FP64 inverses (FP64 path, or the mixed path under DPGMG_FLAG_PATCH_FP64,
  // which rounds them to complex64 after theta is estimated)
  invert_patches<double2>(A, D, lp, D.inv64, F.mesh.offU, dinfo, st);
}

// DPGMG_COARSEST_SMOOTH on a hierarchy with more than one level: level 0 is
// smoothed (its own operator and vertex patches) instead of solved.
static bool smooth_coarsest(const SystemImpl& S) {
  return S.op.coarsest == DPGMG_COARSEST_SMOOTH && S.levels.size() > 1;
}

// Host index plan of a hierarchy (every level's integer structures); runs on
// host threads concurrently with the element stage: one per level (the levels'
// structures are independent) and one for the CG operator's lists, each of
// them spreading its larger loops over further threads.
std::shared_ptr<HostPlan> plan_host(const SystemImpl& S) {
  auto HP = std::make_shared<HostPlan>();
  const int L = (int)S.levels.size() - 1;
  HP->lv.resize(L + 1);
  std::vector<std::thread> th;
  std::vector<std::exception_ptr> errs(L + 3);
  auto guarded = [&errs](int slot, auto&& f) {
    return [&errs, slot, f]() {
      try {
        f();
      } catch (...) {
        errs[slot] = std::current_exception();
      }
    };
  };
  th.emplace_back(guarded(L + 2, [&]() { HP->fdofs = elem_dof_table(S.levels[L].mesh); }));
  if (L == 0 || S.levels[L].kind != 1) {
    HP->has_acg = true;
    th.emplace_back(guarded(L + 1, [&]() { HP->acg = prep_ecsr(S.levels[L].mesh, element_groups(S.levels[L].mesh)); }));
  }
  const int lmin = smooth_coarsest(S) ? 0 : 1;
  for (int l = L; l >= lmin; --l) th.emplace_back(guarded(l, [&S, &HP, l]() {
    const Level& F = S.levels[l];
    const Level& C = S.levels[l > 0 ? l - 1 : 0];   // level 0: the vertex patches of its own mesh
    LevelPlan& lp = HP->lv[l];
    if (l > 0) lp.cdofs = elem_dof_table(C.mesh);
    if (l == 0) {
      lp.E = prep_ecsr(F.mesh, element_groups(F.mesh));
      lp.smask.assign(F.mesh.ndof, 1);
      lp.H = 2;
    } else if (F.kind == 1) {
      p_selection(F.mesh.p, lp.sel);
      p_injection(F.mesh, C.mesh, lp.inj);
      lp.E = prep_ecsr(F.mesh, element_groups(F.mesh));
      lp.smask.assign(F.mesh.ndof, 1);
      lp.H = 2;
    } else {
      lp.M = build_macro(F.mesh, C.mesh);
      lp.E = prep_ecsr(F.mesh, lp.M.groups);
      lp.smask.assign(lp.M.smask.begin(), lp.M.smask.end());
      lp.H = 4;
    }
    lp.P = build_patches(F.mesh, lp.smask, lp.H, C.mesh.n, (S.op.flags & DPGMG_FLAG_PATCH_R2) != 0);
    const Patches& P = lp.P;
    const int64_t np = (int64_t)P.ptr.size() - 1;
    auto size_of = [&](int64_t j) { return P.ptr[j + 1] - P.ptr[j]; };
    for (int64_t j = 0; j < np; ++j) {
      lp.max_n = std::max(lp.max_n, size_of(j));
      lp.sum_sq += size_of(j) * size_of(j);
    }
    // largest patches first: the short work items of small patches end a launch
    for (int width : {32, 64}) {
      std::vector<int2>& ch = width == 32 ? lp.ch32 : lp.ch64;
      for (int64_t j = 0; j < np; ++j)
        for (int64_t a0 = 0; a0 < size_of(j); a0 += width) ch.push_back(make_int2((int)j, (int)a0));
      std::stable_sort(ch.begin(), ch.end(), [&](const int2& u, const int2& v) { return size_of(u.x) > size_of(v.x); });
    }
    lp.order.resize(np);
    for (int64_t j = 0; j < np; ++j) lp.order[j] = j;
    std::stable_sort(lp.order.begin(), lp.order.end(), [&](int64_t u, int64_t v) { return size_of(u) > size_of(v); });
  }));
  for (auto& t : th) t.join();
  for (auto& e : errs)
    if (e) std::rethrow_exception(e);
  return HP;
}

// The side stream paired with a setup stream (one per device and stream, kept
// for the life of the process): memory freed on it is reused by the next
// system set up on the same stream, which a fresh stream per system would not
// allow.
static cudaStream_t side_stream_for(cudaStream_t st) {
  static std::mutex mu;
  static std::map<std::pair<int, cudaStream_t>, cudaStream_t> streams;
  int dev = 0;
  DPG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  cudaStream_t& s = streams[{dev, st}];
  if (!s) {
    // highest priority: the factorisation is a chain of small dependent
    // launches, the patch work it overlaps is many independent CTAs
    int least = 0, greatest = 0;
    DPG_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    DPG_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest));
  }
  return s;
}

// joins the side thread on every exit path (an exception included)
struct JoinOnExit {
  std::thread t;
  ~JoinOnExit() {
    if (t.joinable()) t.join();
  }
};

void build_hierarchy(SystemImpl& S, cudaStream_t st) {
  Alloc& A = S.mem;
  const int L = (int)S.levels.size() - 1;
  const bool mixed = S.op.precision == DPGMG_PREC_MIXED;
  int* dinfo = A.arr<int>(1);
  DPG_CUDA(cudaMemsetAsync(dinfo, 0, sizeof(int), st));
  const bool dense = S.op.coarsest == DPGMG_COARSEST_CHOLESKY || L == 0 ||
                     (S.op.coarsest == DPGMG_COARSEST_SMOOTH && L == 0) ||
                     (S.op.coarsest == DPGMG_COARSEST_AUTO && S.levels[0].mesh.ndof <= 20000);
  // The coarsest factorisation (FP32/FP64 dense work) runs on a side stream from
  // a second host thread as soon as level 0's element matrices exist, overlapping
  // the patch inversion and damping estimate of level 1 (FP64, other SM pipes).
  JoinOnExit side;
  std::exception_ptr side_err;
  int* cinfo = nullptr;
  auto start_coarse = [&]() {
    int dev = 0;
    DPG_CUDA(cudaGetDevice(&dev));
    S.aux = side_stream_for(st);
    S.mem_aux.stream = S.aux;
    S.mem_aux.budget = S.mem.budget > S.mem.used ? S.mem.budget - S.mem.used : 0;
    cudaEvent_t ready;
    DPG_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    DPG_CUDA(cudaEventRecord(ready, st));
    side.t = std::thread([&S, &side_err, &cinfo, dev, ready]() {
      try {
        DPG_CUDA(cudaSetDevice(dev));
        DPG_CUDA(cudaStreamWaitEvent(S.aux, ready, 0));
        if (S.ph_ev) DPG_CUDA(cudaEventRecord(S.ph_ev[5], S.aux));
        cinfo = S.mem_aux.arr<int>(1);
        DPG_CUDA(cudaMemsetAsync(cinfo, 0, sizeof(int), S.aux));
        coarse_setup(S, S.levels[0], cinfo, S.aux, S.mem_aux);
        if (S.ph_ev) DPG_CUDA(cudaEventRecord(S.ph_ev[6], S.aux));
        DPG_CUDA(cudaStreamSynchronize(S.aux));
      } catch (...) {
        side_err = std::current_exception();
      }
      cudaEventDestroy(ready);
    });
  };
  // host index plan, built on a host thread while the element stage ran
  if (!S.plan) S.plan = S.host_plan.valid() ? S.host_plan.get() : plan_host(S);
  const HostPlan& HP = *S.plan;
  S.levels[L].dofs = upload(A, HP.fdofs, st);
  // Pass 1: every level's operator (restriction chain) and transfer data, down
  // to level 0; pass 2: smoothers and damping.  The coarsest factorisation
  // starts between the two and overlaps all of pass 2.
  for (int l = L; l >= 1; --l) {
    Level& F = S.levels[l];
    Level& C = S.levels[l - 1];
    const LevelPlan& lp = HP.lv[l];
    C.dofs = upload(A, lp.cdofs, st);
    C.nloc = (int)C.mesh.loc.size();
    C.E = A.arr<double2>((size_t)C.mesh.nelem * C.nloc * C.nloc);
    if (F.kind == 1) {
      F.inj = upload(A, lp.inj, st);
      int32_t* dsel = upload(A, lp.sel, st);
      k_p_restrict<<<(unsigned)C.mesh.nelem, 256, 0, st>>>(F.E, C.E, dsel, F.nloc, C.nloc);
      DPG_CHECK_LAUNCH();
      assemble_ecsr(A, lp.E, F.A, st);
      ecsr_add_elements(F.A, F.E, F.dofs, F.mesh.nelem, F.nloc, 0, F.mesh.n, st);
    } else {
      const MacroHost& M = lp.M;
      F.nS = M.nS;
      F.nI = M.nI;
      F.nK = C.mesh.nelem;
      F.S_glob = upload(A, M.S_glob, st);
      F.I_glob = upload(A, M.I_glob, st);
      F.P_ptr = upload(A, M.P_ptr, st);
      F.P_col = upload(A, M.P_col, st);
      F.P_val = upload(A, M.P_val, st);
      F.PT_ptr = upload(A, M.PT_ptr, st);
      F.PT_col = upload(A, M.PT_col, st);
      F.PT_val = upload(A, M.PT_val, st);
      F.sslot_ptr = upload(A, M.sslot_ptr, st);
      F.sslots = upload(A, M.sslots, st);
      F.smask = upload(A, M.smask, st);
      int32_t* cmap = upload(A, M.child_map, st);
      assemble_ecsr(A, lp.E, F.A, st);
      if (macro_fp32(S)) {
        F.Y32 = A.arr<float2>((size_t)F.nK * F.nI * F.nS);
        F.Ai32 = A.arr<float2>((size_t)F.nK * F.nI * F.nI);
        macro_condense<float2>(S, F, C, M, cmap, dinfo, F.Y32, F.Ai32, st);
      } else {
        F.Y64 = A.arr<double2>((size_t)F.nK * F.nI * F.nS);
        F.Ai64 = A.arr<double2>((size_t)F.nK * F.nI * F.nI);
        macro_condense<double2>(S, F, C, M, cmap, dinfo, F.Y64, F.Ai64, st);
      }
    }
    if (S.op.flags & DPGMG_FLAG_STORE_COARSE) {
      // "stored" coarse operator (Sec. 3): the DPG system assembled directly on
      // the coarser mesh (its own enriched test space) replaces the restriction
      DPG_CUDA(cudaStreamSynchronize(st));
      A.release(C.E);
      element_stage_level(S, C, st);
    }
  }
  const int lmin = smooth_coarsest(S) ? 0 : 1;
  if (lmin == 0) {   // level 0 smoothed: its own assembled operator
    Level& C0 = S.levels[0];
    assemble_ecsr(A, HP.lv[0].E, C0.A, st);
    ecsr_add_elements(C0.A, C0.E, C0.dofs, C0.mesh.nelem, C0.nloc, 0, C0.mesh.n, st);
  }
  if (S.ph_ev) DPG_CUDA(cudaEventRecord(S.ph_ev[2], st));
  if (L >= 1 && dense) start_coarse();
  // theta's Rayleigh quotient stays on the device until the end of the build
  double* dtheta = A.arr<double>((size_t)2 * (L + 1));
  for (int l = L; l >= lmin; --l) {
    Level& F = S.levels[l];
    const LevelPlan& lp = HP.lv[l];
    F.n_smooth = 0;
    for (char c : lp.smask) F.n_smooth += c;
    setup_patches(S, F, lp, dinfo, st);
    // double-float copies for the damping estimate; the mixed V-cycle keeps the
    // high parts (its complex64 operator and patch inverses), the CG operator
    // (finest level of a p-transition) the operator's split
    PatchDev& Pd = F.P;
    const bool keep_split = l == L && F.kind == 1;
    float2* plo = nullptr;
    const bool c128 = (S.op.flags & DPGMG_FLAG_CG_C128) != 0;
    if (!(S.op.theta > 0.0) && !c128 && patches_fp32(S)) {
      // estimate in the V-cycle's complex64 arithmetic (its operator and FP32-factored smoother)
      if (!F.A.v32) operator_c64(A, F.A, F.mesh.offU, pack_storage(S), st);
    } else if (!(S.op.theta > 0.0) && !c128) {   // double-float estimate
      Pd.inv32 = A.arr<float2>((size_t)std::max<int64_t>(Pd.nvals, 1));
      plo = A.arr<float2>((size_t)std::max<int64_t>(Pd.nvals, 1));
      split_df(Pd.inv64, Pd.inv32, plo, Pd.nvals, st);
      if (!F.A.vlo) split_operator(A, F.A, F.mesh.offU, pack_storage(S), st);
    }
    estimate_theta(S, l, dtheta + 2 * l, plo, st);
    if (plo) A.release(plo);
    if (F.A.vlo && !keep_split) {
      A.release(F.A.vlo);
      F.A.vlo = nullptr;
    }
    if (!mixed) {
      if (Pd.inv32) A.release(Pd.inv32);
      Pd.inv32 = nullptr;
      if (F.A.v32 && !keep_split) {
        A.release(F.A.v32);
        F.A.v32 = nullptr;
      }
    }
    if (mixed) {
      if (!F.A.v32) operator_c64(A, F.A, F.mesh.offU, pack_storage(S), st);
      if (kHalfStorageSmoother && Pd.max_n <= HALF_MAX_N && Pd.inv64) {
        // complex64 Hermitian half storage: lower triangles packed by rows
        std::vector<int64_t> hp(Pd.np + 1, 0), pp(Pd.np + 1);
        DPG_CUDA(cudaMemcpyAsync(pp.data(), Pd.ptr, (Pd.np + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        DPG_CUDA(cudaStreamSynchronize(st));
        for (int64_t j = 0; j < Pd.np; ++j) {
          const int64_t nj = pp[j + 1] - pp[j];
          hp[j + 1] = hp[j] + nj * (nj + 1) / 2;
        }
        Pd.nhvals = hp[Pd.np];
        Pd.hptr = upload(A, hp, st);
        Pd.h32 = A.arr<float2>((size_t)std::max<int64_t>(Pd.nhvals, 1));
        k_pack_half<double2, float2><<<(unsigned)Pd.np, 256, 0, st>>>(Pd.ptr, Pd.val_ptr, Pd.hptr, Pd.inv64, Pd.h32);
        DPG_CHECK_LAUNCH();
        Pd.half = true;
      } else if (!Pd.inv32 && Pd.inv64) {
        Pd.inv32 = to_c64(A, Pd.inv64, Pd.nvals, st);
      }
      if (Pd.inv64) A.release(Pd.inv64);   // the mixed V-cycle only reads the complex64 copy (stream-ordered free)
      Pd.inv64 = nullptr;
      if (F.kind == 2 && !F.Y32) {
        F.Y32 = to_c64(A, F.Y64, F.nK * F.nI * F.nS, st);
        F.Ai32 = to_c64(A, F.Ai64, F.nK * F.nI * F.nI, st);
      }
    }
  }
  // coarsest
  if (S.ph_ev) DPG_CUDA(cudaEventRecord(S.ph_ev[3], st));
  Level& C0 = S.levels[0];
  if (L == 0) C0.dofs = S.levels[0].dofs;
  int info = 0;
  if (side.t.joinable()) {
    side.t.join();
    if (side_err) std::rethrow_exception(side_err);
    S.ph_side = true;
    DPG_CUDA(cudaMemcpyAsync(&info, cinfo, sizeof(int), cudaMemcpyDeviceToHost, S.aux));
    DPG_CUDA(cudaStreamSynchronize(S.aux));
  } else if (dense) {
    coarse_setup(S, C0, dinfo, st, A);
  }
  if (S.ph_ev) DPG_CUDA(cudaEventRecord(S.ph_ev[4], st));
  int info_main = 0;
  std::vector<double> th((size_t)2 * (L + 1));
  DPG_CUDA(cudaMemcpyAsync(&info_main, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st));
  DPG_CUDA(cudaMemcpyAsync(th.data(), dtheta, th.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  DPG_CUDA(cudaStreamSynchronize(st));
  A.release(dtheta);
  for (int l = lmin; l <= L; ++l)
    if (!(S.op.theta > 0.0)) S.levels[l].theta = theta_from_rayleigh(th[2 * l], th[2 * l + 1]);
  info |= info_main;
  if (info & 32) throw Err{DPGMG_ERR_TIMEOUT, "tensor-core update: a bounded wait for the MMAs ran out"};
  if (info)
    throw Err{DPGMG_ERR_NOT_HPD, std::string("lost positive definiteness in:") + ((info & 4) ? " macro condensation" : "") +
                                     ((info & 8) ? " patch factorisation" : "") +
                                     ((info & 16) ? " coarsest factorisation" : "") +
                                     ((info & ~(4 | 8 | 16 | 32)) ? " other" : "")};
}

}  // namespace dpgmg
