// C ABI of the DPG-MG solver (include/dpgmg.h): handles, problem validation,
// setup / solve orchestration and introspection.  No exception crosses the
// ABI; every failure becomes a DPGMG_ERR_* status and a thread-local message.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>

#include "internal.h"


namespace dpgmg {

static thread_local std::string g_last;
void set_last_error(const std::string& m) { g_last = m; }

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;   // this thread's launches (graph capture counts)
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long thread_launch_count() { return t_launches; }

void* Alloc::get(size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (used + bytes > budget) throw Err{DPGMG_ERR_NOMEM, "device-memory budget exceeded"};
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Err{DPGMG_ERR_NOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e)};
  }
  ptrs.push_back(p);
  sizes.push_back(bytes);
  used += bytes;
  peak = std::max(peak, used);
  return p;
}

SystemImpl::~SystemImpl() { mem_aux.free_all(); }

void Alloc::release(void* p) {
  for (size_t i = 0; i < ptrs.size(); ++i)
    if (ptrs[i] == p) {
      cudaFreeAsync(p, stream);
      used -= sizes[i];
      ptrs.erase(ptrs.begin() + i);
      sizes.erase(sizes.begin() + i);
      return;
    }
}

void Alloc::free_all() {
  for (void* p : ptrs) cudaFreeAsync(p, stream);
  ptrs.clear();
  sizes.clear();
  used = 0;
}

int validate_problem(const dpgmg_problem* pb, const dpgmg_opts* op) {
  if (!pb || !op) return DPGMG_ERR_ARG;
  for (int d = 0; d < 3; ++d) {
    if (pb->n[d] < 1 || !(pb->x1[d] > pb->x0[d])) return DPGMG_ERR_ARG;
  }
  if (pb->p < 1 || pb->p > 5 || pb->dp != 1 || !(pb->omega > 0.0)) return DPGMG_ERR_ARG;
  if (pb->source < 0 || pb->source > 2) return DPGMG_ERR_ARG;
  if (pb->source == DPGMG_SRC_GAUSSIAN && !(pb->src_width > 0.0)) return DPGMG_ERR_ARG;
  if (pb->source == DPGMG_SRC_MANUFACTURED && (pb->mf_order < 1 || pb->mf_order > 8 || !pb->mf_coeffs))
    return DPGMG_ERR_ARG;
  if (pb->source == DPGMG_SRC_PLANE_WAVE) {
    double n2 = pb->wave_dir[0] * pb->wave_dir[0] + pb->wave_dir[1] * pb->wave_dir[1] + pb->wave_dir[2] * pb->wave_dir[2];
    if (!(n2 > 0.0)) return DPGMG_ERR_ARG;
  }
  if (pb->wavespeed) {
    int64_t ne = (int64_t)pb->n[0] * pb->n[1] * pb->n[2];
    for (int64_t e = 0; e < ne; ++e)
      if (!(pb->wavespeed[e] > 0.0) || !std::isfinite(pb->wavespeed[e])) return DPGMG_ERR_ARG;
  }
  if (!(op->tol > 0.0) || op->max_iter < 1 || op->nu_pre < 0 || op->nu_post < 0 || op->n_levels < 1 ||
      op->p_min < 1 || (op->precision != DPGMG_PREC_FP64 && op->precision != DPGMG_PREC_MIXED) ||
      (op->coarsest != DPGMG_COARSEST_CHOLESKY && op->coarsest != DPGMG_COARSEST_NONE &&
       op->coarsest != DPGMG_COARSEST_AUTO && op->coarsest != DPGMG_COARSEST_SMOOTH) ||
      (op->flags & ~(DPGMG_FLAG_EAGER | DPGMG_FLAG_CUDA_CORES | DPGMG_FLAG_STORE_COARSE | DPGMG_FLAG_WARM_START |
                     DPGMG_FLAG_CG_C128 | DPGMG_FLAG_PATCH_FP64 | DPGMG_FLAG_PATCH_R2 |
                     DPGMG_FLAG_RECOMPUTE_PATCHES | DPGMG_FLAG_COMPLEX_STORAGE | DPGMG_FLAG_FAULT_NOT_HPD |
                     DPGMG_FLAG_FAULT_TC_WAIT)))
    return DPGMG_ERR_ARG;
  // recompute mode: the mixed path's FP32 patch factors and complex64 damping estimate only
  if ((op->flags & DPGMG_FLAG_RECOMPUTE_PATCHES) &&
      (op->precision != DPGMG_PREC_MIXED || (op->flags & (DPGMG_FLAG_PATCH_FP64 | DPGMG_FLAG_CG_C128))))
    return DPGMG_ERR_ARG;
  if ((op->flags & DPGMG_FLAG_STORE_COARSE) && pb->wavespeed) {
    const int64_t ne = (int64_t)pb->n[0] * pb->n[1] * pb->n[2];
    for (int64_t e = 1; e < ne; ++e)
      if (pb->wavespeed[e] != pb->wavespeed[0]) return DPGMG_ERR_ARG;
  }
  return DPGMG_OK;
}

// DPGMG_COARSEST_AUTO: the dense coarsest solve is used up to this size.
constexpr double kAutoCoarsestMax = 20000.0;

// Device bytes a system needs (upper bound used for admission): everything
// resident after setup plus the largest scratch of any setup phase (the
// phases run one after another and release their scratch).
size_t estimate_bytes(const dpgmg_problem* pb, const dpgmg_opts* op) {
  const int nn[3] = {pb->n[0], pb->n[1], pb->n[2]};
  auto specs = plan_levels(nn, pb->p, op->n_levels, op->p_min);
  const bool mixed = op->precision == DPGMG_PREC_MIXED;
  const double vsz = mixed ? 8.0 : 16.0;       // V-cycle complex size
  const double x32 = mixed ? 8.0 : 0.0;        // extra complex64 copies on the mixed path
  double resident = 0.0, transient = 0.0, coarse_transient = 0.0;
  const int p = pb->p;
  const double ne = (double)nn[0] * nn[1] * nn[2];
  const double ntr = n_trace_local(p), nf = 4.0 * p * p * p;
  const double nt = std::pow(p + 2.0, 3) + 3.0 * (p + 2.0) * (p + 1.0) * (p + 1.0);
  const double m1 = nf + ntr + 1.0;
  resident += ne * (ntr * ntr + nf * (ntr + 1.0) + ntr) * 16.0;     // finest E, Yrec, Fc
  const double per = nt * nt * 8.0 + nt * m1 * 16.0 + m1 * m1 * 16.0;
  // element batch scratch, plus the load-only scratch of the element-class members (at most every
  // element) and their per-chunk blocks (chunks of <= 32 members of one class)
  const double mcols = ne + 32.0 * std::min(ne / 4.0, 4096.0);
  transient = std::max(transient, (double)element_chunk((int64_t)ne, (size_t)per) * per +
                                      ne * (nt + 1.0 + 2.0 * m1 + 2.0 * nf) * 8.0 +
                                      mcols * (nt + 2.0 * m1 + 2.0 * nf + 2.0 * ntr) * 8.0);
  double xdofs = 0.0;
  for (size_t i = 0; i < specs.size(); ++i) {
    const LevelSpec& s = specs[i];
    MeshL m;
    double a0[3] = {0, 0, 0}, a1[3] = {1, 1, 1};
    m.init(s.n, s.p, a0, a1);
    const double nel = (double)m.nelem, nl = n_trace_local(s.p), nd = (double)m.ndof;
    if (i == 0) xdofs = nd;
    if (i > 0) resident += nel * nl * nl * 16.0;                      // restricted element matrices
    resident += nel * nl * 8.0 + nd * 4.0 * (16.0 + x32) + nd * 80.0; // maps, work vectors, row indices, SpMV tasks
    const bool smooth0 = s.kind_below == 0 && op->coarsest == DPGMG_COARSEST_SMOOTH && specs.size() > 1;
    if (s.kind_below != 0 || smooth0) {
      const int q = s.p;
      const bool hlev = s.kind_below == 2;
      const double nS = 6.0 * (4.0 * (q - 1) * (q - 1) + 4.0 * (q - 1) + 1.0 + 4.0 * q * q) + 12.0 * (2.0 * (q - 1) + 1.0) + 8.0;
      const double nI = 1.0 + 6.0 * (q - 1) + 12.0 * ((q - 1.0) * (q - 1.0) + q * q);
      const double nK = nel / 8.0;
      const double nnz = hlev ? nK * nS * nS : nel * nl * nl;         // bound on stored entries
      resident += nnz * (16.0 + x32 + 4.0);                           // values (+complex64) and columns
      if (i == 0) resident += nnz * (mixed ? 8.0 : 16.0);             // double-float split of the CG operator
      int nco[3];
      for (int d = 0; d < 3; ++d) nco[d] = hlev ? s.n[d] / 2 : s.n[d];
      auto ps = patch_sizes(m, hlev, hlev ? 4 : 2, nco, (op->flags & DPGMG_FLAG_PATCH_R2) != 0);
      double nvals = 0.0, nslots = 0.0, nmax = 0.0;
      for (int64_t v : ps) {
        nvals += (double)v * (double)patch_ld(v);
        nslots += (double)v;
        nmax = std::max(nmax, (double)v);
      }
      if (op->flags & DPGMG_FLAG_RECOMPUTE_PATCHES) {
        // two window buffers instead of the stored inverses, index lists
        const double wcap = std::max(nmax * (nmax + 1.0), std::min(std::ceil(nvals / 4.0), (double)(32 << 20)));
        resident += 2.0 * wcap * 8.0 + nslots * (8.0 + 16.0 + x32) + nslots / 32.0 * 8.0 + ps.size() * 24.0;
      } else {
        resident += nvals * vsz + nslots * (8.0 + 16.0 + x32) + nslots / 32.0 * 8.0;
      }
      const double one = nmax * nmax * 16.0;
      const double cap = std::max(std::min(std::min(std::max((double)(1 << 28), one) * 4.0, (double)(2ull << 30)),
                                           nvals * 16.0), one);
      transient = std::max(transient, nvals * (16.0 + x32) + cap + nd * 48.0 + nslots * 16.0);
      // damping estimate: double-float patch inverses (high parts resident on the mixed
      // path) and operator split, vectors, slot buffer
      transient = std::max(transient, nvals * (mixed ? 24.0 : 16.0) + nnz * (mixed ? 8.0 : 16.0) + nd * 64.0 +
                                          nslots * 16.0);
      if (hlev) {
        resident += nK * (nI * nS + nI * nI) * (16.0 + x32) + nK * (nS + nI) * 8.0 + nK * nS * (16.0 + x32 + 4.0);
        const double nlc = n_trace_local(q);
        transient = std::max(transient, std::min(nK, 2048.0) * ((nS + nI) * (nS + nI) + nS * nlc + nS * nS) * 16.0);
      }
    } else if (op->coarsest == DPGMG_COARSEST_CHOLESKY || specs.size() == 1 ||
               (op->coarsest == DPGMG_COARSEST_AUTO && nd <= kAutoCoarsestMax)) {
      resident += nd * (nd + 1.0) * vsz;                              // packed L^-1 and L^-H
      // built concurrently with the level above: its scratch adds to theirs
      coarse_transient = nd * nd * (mixed ? 24.0 : 32.0) + nd * 64.0 * 16.0;
      // tensor-core operand images (two TF32 parts of a panel of up to 512
      // columns: 16 B per complex entry, twice for A's real and imaginary variants)
      if (mixed && !(op->flags & DPGMG_FLAG_CUDA_CORES)) coarse_transient += (nd + 128.0) * 512.0 * 48.0;
    }
  }
  resident += (xdofs + ne * nf) * 16.0;                              // solution outputs
  return (size_t)((resident + transient + coarse_transient) * 1.05) + ((size_t)64 << 20);
}

static void fill_bytes_per_iter(SystemImpl& S) {
  const bool mixed = S.op.precision == DPGMG_PREC_MIXED;
  const double esz = mixed ? 8.0 : 16.0;
  double b = 0;
  const Level& F = S.levels.back();
  // CG operator (FP64 as complex64 high and low parts; packed real entities half)
  int64_t cg_nnz = 0, cg_real = 0;
  if (const ECSRDev* cg = cg_operator_of(S)) {
    cg_nnz = cg->nnz_alg;
    cg_real = cg->nnz_real;
  } else if (S.levels.size() > 1 && F.kind == 1) {
    cg_nnz = F.A.nnz_alg;
  } else {
    cg_nnz = (int64_t)(F.mesh.nelem * (double)F.nloc * F.nloc * 0.8);
  }
  b += (cg_nnz - cg_real) * 16.0 + cg_real * 8.0;
  const int nu = S.op.nu_pre + S.op.nu_post;
  for (size_t l = 1; l < S.levels.size(); ++l) {
    const Level& L = S.levels[l];
    b += nu * ((double)(L.P.sum_sq - L.P.real_sq) + 0.5 * (double)L.P.real_sq) * esz;  // smoother (n_j^2 per
                                                                                      // patch, real ones half)
    b += std::max(1, nu) * ((double)(L.A.nnz_alg - L.A.nnz_real) + 0.5 * (double)L.A.nnz_real) * esz;  // SpMVs
    if (L.kind == 2) b += (double)L.nK * (2.0 * L.nI * L.nS + L.nI * L.nI) * esz; // condense + backsub
  }
  const Level& C0 = S.levels[0];
  if (C0.has_coarse) b += (double)C0.N0 * (C0.N0 + 1) * esz;                     // L^-1 and L^-H (packed)
  S.bytes_per_iter = (int64_t)b;
}

void setup_system(SystemImpl& S, const dpgmg_problem* pb, const dpgmg_opts* op, size_t budget, cudaStream_t st) {
  S.pb = *pb;
  S.op = *op;
  const int64_t ne = (int64_t)pb->n[0] * pb->n[1] * pb->n[2];
  S.wavespeed.assign(ne, 1.0);
  if (pb->wavespeed) std::copy(pb->wavespeed, pb->wavespeed + ne, S.wavespeed.begin());
  if (pb->source == DPGMG_SRC_MANUFACTURED) {
    size_t m = pb->mf_order;
    S.mf_coeffs.assign(pb->mf_coeffs, pb->mf_coeffs + 2 * 4 * m * m * m);
  }
  if (pb->u0_samples) S.u0.assign(pb->u0_samples, pb->u0_samples + 2 * boundary_point_count(pb));
  S.pb.wavespeed = nullptr;
  S.pb.mf_coeffs = nullptr;
  S.pb.u0_samples = nullptr;
  S.mem.budget = budget;
  S.mem.stream = st;
  auto specs = plan_levels(pb->n, pb->p, op->n_levels, op->p_min);
  S.levels.resize(specs.size());
  for (size_t i = 0; i < specs.size(); ++i) {
    Level& L = S.levels[specs.size() - 1 - i];
    L.mesh.init(specs[i].n, specs[i].p, pb->x0, pb->x1);
    L.kind = specs[i].kind_below;
    L.nloc = (int)L.mesh.loc.size();
  }
  struct PhaseEvents {   // destroyed on every exit path
    cudaEvent_t e[8] = {};
    ~PhaseEvents() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } ph;
  for (cudaEvent_t& x : ph.e) DPG_CUDA(cudaEventCreate(&x));
  S.ph_ev = ph.e;
  S.ph_side = false;
  struct ClearPh {
    SystemImpl& S;
    ~ClearPh() { S.ph_ev = nullptr; }
  } clear_ph{S};
  // host index plan of the hierarchy: built on a host thread during the element stage
  S.plan.reset();
  S.host_plan = std::async(std::launch::async, [&S]() { return plan_host(S); });
  struct DropPlan {   // the plan is setup-only memory; the future is drained on every exit path
    SystemImpl& S;
    ~DropPlan() {
      if (S.host_plan.valid()) S.host_plan.wait();
      S.host_plan = {};
      S.plan.reset();
    }
  } drop_plan{S};
  DPG_CUDA(cudaEventRecord(ph.e[0], st));
  element_stage(S, st);
  DPG_CUDA(cudaEventRecord(ph.e[1], st));
  build_hierarchy(S, st);   // records 2, 3, 4 (and 5, 6 on the side stream)
  assemble_rhs(S, st);
  prepare_solve(S, st);
  DPG_CUDA(cudaEventRecord(ph.e[7], st));
  DPG_CUDA(cudaEventSynchronize(ph.e[7]));
  auto span = [&](int a, int b) {
    float ms = 0.f;
    DPG_CUDA(cudaEventElapsedTime(&ms, ph.e[a], ph.e[b]));
    return (double)ms;
  };
  S.t_setup_ms = span(0, 7);
  S.t_elem_ms = span(0, 1);
  S.t_phase[0] = span(0, 1);
  S.t_phase[1] = span(1, 2);
  S.t_phase[2] = span(2, 3);
  S.t_phase[3] = S.ph_side ? span(5, 6) : 0.0;
  S.t_phase[4] = span(3, 4);
  S.t_phase[5] = span(4, 7);
  // operators and patches stored as reals (half the bytes per entry)
  for (size_t l = 1; l < S.levels.size(); ++l) S.levels[l].A.nnz_real = packed_entries(S.levels[l].A);
  if (ECSRDev* cg = cg_operator_of(S)) cg->nnz_real = packed_entries(*cg);
  for (size_t l = 1; l < S.levels.size() && S.plan; ++l) {
    PatchDev& P = S.levels[l].P;
    P.real_sq = 0;
    if (!P.rflag || P.np == 0) continue;
    std::vector<uint8_t> fl((size_t)P.np);
    DPG_CUDA(cudaMemcpy(fl.data(), P.rflag, (size_t)P.np, cudaMemcpyDeviceToHost));
    const std::vector<int64_t>& pp = S.plan->lv[l].P.ptr;
    for (int64_t j = 0; j < P.np; ++j)
      if (fl[j]) P.real_sq += (pp[j + 1] - pp[j]) * (pp[j + 1] - pp[j]);
  }
  fill_bytes_per_iter(S);
}

int64_t boundary_point_count(const dpgmg_problem* pb) {
  int64_t off[6];
  const int64_t nq = make_tables(pb->p).nql;
  return boundary_face_offsets(pb->n, off) * nq * nq;
}

}  // namespace dpgmg

using namespace dpgmg;

static int fail(const Err& e) {
  set_last_error(e.msg);
  return e.code;
}

extern "C" {

void dpgmg_default_opts(dpgmg_opts* op) {
  if (!op) return;
  op->tol = 1e-8;
  op->max_iter = 2000;
  op->nu_pre = 1;
  op->nu_post = 1;
  op->n_levels = 2;
  op->p_min = 2;
  op->precision = DPGMG_PREC_FP64;
  op->coarsest = DPGMG_COARSEST_CHOLESKY;
  op->flags = 0;
  op->theta = 0.0;
}

const char* dpgmg_strerror(int code) {
  switch (code) {
    case DPGMG_OK: return "ok";
    case DPGMG_ERR_ARG: return "invalid argument";
    case DPGMG_ERR_NOMEM: return "device memory budget exceeded";
    case DPGMG_ERR_NOT_HPD: return "factorisation lost positive definiteness";
    case DPGMG_ERR_BREAKDOWN: return "conjugate-gradient breakdown";
    case DPGMG_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case DPGMG_ERR_TIMEOUT: return "bounded device wait expired";
    case DPGMG_ERR_PENDING: return "request pending";
    case DPGMG_ERR_CUDA: return "CUDA runtime error";
    default: return "unknown status";
  }
}

const char* dpgmg_last_error(void) { return g_last.c_str(); }

int dpgmg_create(dpgmg_handle* out, int device, size_t mem_budget_bytes, void* cuda_stream) {
  if (!out) return DPGMG_ERR_ARG;
  *out = nullptr;
  try {
    int ndev = 0;
    DPG_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return DPGMG_ERR_ARG;
    DPG_CUDA(cudaSetDevice(device));
    auto* h = new (std::nothrow) dpgmg_handle_s();
    if (!h) return DPGMG_ERR_NOMEM;
    h->h.device = device;
    if (cuda_stream) {
      h->h.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
      DPG_CUDA(cudaStreamCreateWithFlags(&h->h.stream, cudaStreamNonBlocking));
      h->h.own_stream = true;
    }
    // keep freed stream-ordered memory in the process's pool between setups
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    size_t fr = 0, tot = 0;
    DPG_CUDA(cudaMemGetInfo(&fr, &tot));
    h->h.budget = mem_budget_bytes ? mem_budget_bytes : (size_t)(0.9 * fr);
    *out = h;
    return DPGMG_OK;
  } catch (const Err& e) {
    return fail(e);
  }
}

void dpgmg_destroy(dpgmg_handle h) {
  if (!h) return;
  server_shutdown(h);
  cudaSetDevice(h->h.device);
  if (h->h.own_stream) cudaStreamDestroy(h->h.stream);
  delete h;
}

int dpgmg_dof_map(const dpgmg_problem* pb, long long n_trace, int* out) {
  if (!pb || !out) return DPGMG_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (pb->n[d] < 1 || !(pb->x1[d] > pb->x0[d])) return DPGMG_ERR_ARG;
  if (pb->p < 1 || pb->p > 5) return DPGMG_ERR_ARG;
  MeshL m;
  m.init(pb->n, pb->p, pb->x0, pb->x1);
  if (n_trace != m.ndof) {
    set_last_error("dpgmg_dof_map: n_trace differs from the mesh's trace DOF count");
    return DPGMG_ERR_ARG;
  }
  const int p = pb->p;
  for (int64_t g = 0; g < m.ndof; ++g) {
    const int64_t E = m.dof_entity(g);
    int ctr[3];
    m.ent_center(E, ctr);
    int64_t st;
    int nd;
    m.ent_range(E, &st, &nd);
    const int loc = (int)(g - st);
    int kind, axis = -1, m1 = -1, m2 = -1;
    if (E < m.entE) {
      kind = 0;
    } else if (E < m.entF) {
      kind = 1;
      for (int d = 0; d < 3; ++d)
        if (ctr[d] & 1) axis = d;
      m1 = loc + 2;
    } else {
      kind = E < m.entU ? 2 : 3;
      for (int d = 0; d < 3; ++d)
        if (!(ctr[d] & 1)) axis = d;
      if (kind == 2) {
        m1 = loc % (p - 1) + 2;
        m2 = loc / (p - 1) + 2;
      } else {
        m1 = loc % p;
        m2 = loc / p;
      }
    }
    int* o = out + 7 * g;
    o[0] = kind;
    o[1] = ctr[0];
    o[2] = ctr[1];
    o[3] = ctr[2];
    o[4] = axis;
    o[5] = m1;
    o[6] = m2;
  }
  return DPGMG_OK;
}

int dpgmg_boundary_points(const dpgmg_problem* pb, long long* n_points, double* xyz) {
  if (!pb || !n_points) return DPGMG_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (pb->n[d] < 1 || !(pb->x1[d] > pb->x0[d])) return DPGMG_ERR_ARG;
  if (pb->p < 1 || pb->p > 5) return DPGMG_ERR_ARG;
  const int64_t cnt = boundary_point_count(pb);
  if (xyz) {
    if (*n_points < cnt) {
      set_last_error("dpgmg_boundary_points: capacity below the point count");
      return DPGMG_ERR_ARG;
    }
    std::vector<double> pts;
    boundary_points(pb->n, pb->x0, pb->x1, pb->p, pts);
    std::copy(pts.begin(), pts.end(), xyz);
  }
  *n_points = cnt;
  return DPGMG_OK;
}

int dpgmg_query_sizes(const dpgmg_problem* pb, const dpgmg_opts* op, long long* n_trace, long long* n_field,
                      size_t* dev_bytes) {
  int v = validate_problem(pb, op);
  if (v) return v;
  MeshL m;
  m.init(pb->n, pb->p, pb->x0, pb->x1);
  if (n_trace) *n_trace = m.ndof;
  if (n_field) *n_field = m.nelem * 4LL * pb->p * pb->p * pb->p;
  if (dev_bytes) *dev_bytes = estimate_bytes(pb, op);
  return DPGMG_OK;
}

int dpgmg_setup(dpgmg_handle h, const dpgmg_problem* pb, const dpgmg_opts* op, dpgmg_system* out) {
  if (!h || !out) return DPGMG_ERR_ARG;
  *out = nullptr;
  int v = validate_problem(pb, op);
  if (v) {
    set_last_error("invalid problem or options");
    return v;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  const size_t est = estimate_bytes(pb, op);
  size_t room = 0;
  {
    // reserve the estimate in the handle's ledger (shared with the serving loop)
    std::lock_guard<std::mutex> lg(h->ledger);
    if (h->h.used + h->h.serving + est > h->h.budget) {
      set_last_error("estimated device footprint exceeds the handle's budget (set-up systems and running requests)");
      return DPGMG_ERR_NOMEM;
    }
    room = h->h.budget - h->h.used - h->h.serving;
    h->h.used += est;
  }
  auto unreserve = [&](size_t keep) {
    {
      std::lock_guard<std::mutex> lg(h->ledger);
      h->h.used = h->h.used - std::min(h->h.used, est) + keep;
    }
    if (keep < est) server_notify(h);
  };
  auto* sys = new (std::nothrow) dpgmg_system_s();
  if (!sys) {
    unreserve(0);
    return DPGMG_ERR_NOMEM;
  }
  SystemImpl& S = sys->s;
  try {
    DPG_CUDA(cudaSetDevice(h->h.device));
    setup_system(S, pb, op, room, h->h.stream);
    unreserve(S.mem_used());
    *out = sys;
    return DPGMG_OK;
  } catch (const Err& e) {
    cudaStreamSynchronize(h->h.stream);
    profile_clear(S);
    free_workspace(S);
    delete sys;
    unreserve(0);
    return fail(e);
  } catch (const std::exception& e) {
    cudaStreamSynchronize(h->h.stream);
    free_workspace(S);
    delete sys;
    unreserve(0);
    return fail(Err{DPGMG_ERR_ARG, e.what()});
  }
}

int dpgmg_solve(dpgmg_handle h, dpgmg_system sys, void* trace_out, void* field_out, int out_is_device,
                dpgmg_stats* st) {
  if (!h || !sys) return DPGMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  SystemImpl& S = sys->s;
  try {
    DPG_CUDA(cudaSetDevice(h->h.device));
    cudaStream_t s = h->h.stream;
    const int64_t n = S.levels.back().mesh.ndof;
    const int64_t nfld = S.nelem * S.nf;
    Alloc tmp;
    tmp.budget = (size_t)-1;
    tmp.stream = s;
    double2* x = (trace_out && out_is_device) ? reinterpret_cast<double2*>(trace_out) : tmp.arr<double2>((size_t)n);
    const double2* x0 = nullptr;
    if (S.op.flags & DPGMG_FLAG_WARM_START) {
      if (!trace_out) throw Err{DPGMG_ERR_ARG, "a warm start reads its initial guess from trace_out"};
      double2* g = tmp.arr<double2>((size_t)n);
      DPG_CUDA(cudaMemcpyAsync(g, trace_out, (size_t)n * sizeof(double2),
                               out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
      x0 = g;
    }
    int status = pcg_solve(S, s, x, st, x0);
    if (field_out) {
      double2* f = out_is_device ? reinterpret_cast<double2*>(field_out) : tmp.arr<double2>((size_t)nfld);
      recover_fields(S, x, f, s);
      if (!out_is_device)
        DPG_CUDA(cudaMemcpyAsync(field_out, f, (size_t)nfld * sizeof(double2), cudaMemcpyDeviceToHost, s));
    }
    if (trace_out && !out_is_device)
      DPG_CUDA(cudaMemcpyAsync(trace_out, x, (size_t)n * sizeof(double2), cudaMemcpyDeviceToHost, s));
    DPG_CUDA(cudaStreamSynchronize(s));
    if (status != DPGMG_OK) set_last_error(dpgmg_strerror(status));
    return status;
  } catch (const Err& e) {
    return fail(e);
  }
}

int dpgmg_solve_block(dpgmg_handle h, dpgmg_system sys, int k, const void* rhs, void* trace_out, int on_device,
                      dpgmg_stats* st) {
  if (!h || !sys || !rhs || !trace_out || k < 1 || k > 64) return DPGMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  SystemImpl& S = sys->s;
  try {
    DPG_CUDA(cudaSetDevice(h->h.device));
    cudaStream_t s = h->h.stream;
    const size_t bytes = (size_t)S.levels.back().mesh.ndof * k * sizeof(double2);
    Alloc tmp;
    tmp.budget = (size_t)-1;
    tmp.stream = s;
    const double2* b = reinterpret_cast<const double2*>(rhs);
    double2* x = reinterpret_cast<double2*>(trace_out);
    if (!on_device) {
      double2* bd = tmp.arr<double2>(bytes / sizeof(double2));
      DPG_CUDA(cudaMemcpyAsync(bd, rhs, bytes, cudaMemcpyHostToDevice, s));
      b = bd;
      x = tmp.arr<double2>(bytes / sizeof(double2));
    }
    int status = pcg_solve_block(S, s, k, b, x, st);
    if (!on_device) DPG_CUDA(cudaMemcpyAsync(trace_out, x, bytes, cudaMemcpyDeviceToHost, s));
    DPG_CUDA(cudaStreamSynchronize(s));
    if (status != DPGMG_OK) set_last_error(dpgmg_strerror(status));
    return status;
  } catch (const Err& e) {
    return fail(e);
  }
}

void dpgmg_release(dpgmg_handle h, dpgmg_system sys) {
  if (!sys) return;
  if (h) {
    std::lock_guard<std::mutex> lk(h->mu);
    cudaSetDevice(h->h.device);
    cudaStreamSynchronize(h->h.stream);
    std::lock_guard<std::mutex> lg(h->ledger);
    h->h.used -= std::min(h->h.used, sys->s.mem_used());
  }
  profile_clear(sys->s);
  free_workspace(sys->s);
  delete sys;
  if (h) server_notify(h);
}

long long dpgmg_launch_count(void) { return g_launches.load(); }

int dpgmg_profile(dpgmg_handle h, dpgmg_system sys, int which) {
  if (!h || !sys || which < DPGMG_PROF_OFF || which > DPGMG_PROF_SPMV_CG) return DPGMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  sys->s.prof_which = which;
  profile_clear(sys->s);
  return DPGMG_OK;
}

int dpgmg_profile_read(dpgmg_handle h, dpgmg_system sys, double* total_ms, long long* launches,
                       long long* bytes_per_launch) {
  if (!h || !sys) return DPGMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  try {
    DPG_CUDA(cudaSetDevice(h->h.device));
    profile_read(sys->s, total_ms, launches, bytes_per_launch);
    return DPGMG_OK;
  } catch (const Err& e) {
    return fail(e);
  }
}

int dpgmg_error_indicator(dpgmg_handle h, dpgmg_system sys, const double* x, double* eta2) {
  if (!h || !sys || !x || !eta2) return DPGMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  SystemImpl& S = sys->s;
  try {
    DPG_CUDA(cudaSetDevice(h->h.device));
    cudaStream_t s = h->h.stream;
    const int64_t n = S.levels.back().mesh.ndof;
    Alloc tmp;
    tmp.budget = (size_t)-1;
    tmp.stream = s;
    double2* dx = tmp.arr<double2>((size_t)std::max<int64_t>(n, 1));
    double* de = tmp.arr<double>((size_t)std::max<int64_t>(S.nelem, 1));
    DPG_CUDA(cudaMemcpyAsync(dx, x, (size_t)n * sizeof(double2), cudaMemcpyHostToDevice, s));
    error_indicator(S, dx, de, s);
    DPG_CUDA(cudaMemcpyAsync(eta2, de, (size_t)S.nelem * sizeof(double), cudaMemcpyDeviceToHost, s));
    DPG_CUDA(cudaStreamSynchronize(s));
    return DPGMG_OK;
  } catch (const Err& e) {
    return fail(e);
  }
}

int dpgmg_setup_profile(dpgmg_handle h, dpgmg_system sys, double* element_ms, double* element_gflop,
                        double* setup_ms) {
  if (!h || !sys) return DPGMG_ERR_ARG;
  const SystemImpl& S = sys->s;
  if (element_ms) *element_ms = S.t_elem_ms;
  if (element_gflop) *element_gflop = S.elem_flops * 1e-9;
  if (setup_ms) *setup_ms = S.t_setup_ms;
  return DPGMG_OK;
}

int dpgmg_setup_phases(dpgmg_handle h, dpgmg_system sys, double* ms, int n) {
  if (!h || !sys || !ms || n < 1) return DPGMG_ERR_ARG;
  const SystemImpl& S = sys->s;
  for (int i = 0; i < n && i < DPGMG_SETUP_NPHASES; ++i) ms[i] = S.t_phase[i];
  return DPGMG_OK;
}

int dpgmg_spmv_group(dpgmg_handle h, dpgmg_system sys, int level, int set, int* group) {
  if (!h || !sys) return DPGMG_ERR_ARG;
  if (set != 0 && set != 1 && set != 2 && set != 4 && set != 8 && set != 16 && set != 32 && set != 64)
    return DPGMG_ERR_ARG;
  if (level == -1 && set == 64) return DPGMG_ERR_ARG;   // no half-warp form of the CG operator
  std::lock_guard<std::mutex> lk(h->mu);
  SystemImpl& S = sys->s;
  const int slot = S.op.precision == DPGMG_PREC_MIXED ? 0 : 1;
  int* g = nullptr;
  if (level == -1) {
    ECSRDev* A = cg_operator_of(S);
    if (!A) return DPGMG_ERR_ARG;
    g = &A->gsel[2];
  } else {
    if (level < 1 || level >= (int)S.levels.size()) return DPGMG_ERR_ARG;
    g = &S.levels[level].A.gsel[slot];
  }
  if (set) *g = set;
  if (group) *group = *g;
  return DPGMG_OK;
}

int dpgmg_level_info(dpgmg_handle h, dpgmg_system sys, int level, dpgmg_level_desc* out) {
  if (!h || !sys || !out) return DPGMG_ERR_ARG;
  SystemImpl& S = sys->s;
  if (level < 0 || level >= (int)S.levels.size()) return DPGMG_ERR_ARG;
  const Level& L = S.levels[level];
  for (int d = 0; d < 3; ++d) out->n[d] = L.mesh.n[d];
  out->p = L.mesh.p;
  out->n_dof = L.mesh.ndof;
  out->n_smooth = L.n_smooth;
  out->kind = L.kind;
  out->n_patches = L.P.np;
  out->patch_max = L.P.max_n;
  out->sum_patch_sq = L.P.sum_sq;
  out->op_nnz = L.A.nnz_alg;
  out->theta = L.theta;
  out->patch_stored = L.P.recompute ? 0 : (L.P.half ? L.P.nhvals : L.P.nvals);
  out->patch_real_sq = L.P.real_sq;
  out->op_real_nnz = L.A.nnz_real;
  return DPGMG_OK;
}

int dpgmg_element_matrix(dpgmg_handle h, dpgmg_system sys, int level, long long e, double* mat_out,
                         double* load_out) {
  if (!h || !sys || !mat_out) return DPGMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  SystemImpl& S = sys->s;
  if (level < 0 || level >= (int)S.levels.size()) return DPGMG_ERR_ARG;
  const Level& L = S.levels[level];
  if (e < 0 || e >= L.mesh.nelem) return DPGMG_ERR_ARG;
  try {
    DPG_CUDA(cudaSetDevice(h->h.device));
    cudaStream_t s = h->h.stream;
    size_t nn = (size_t)L.nloc * L.nloc;
    DPG_CUDA(cudaMemcpyAsync(mat_out, L.E + e * nn, nn * sizeof(double2), cudaMemcpyDeviceToHost, s));
    if (load_out) {
      if (level != (int)S.levels.size() - 1) return DPGMG_ERR_ARG;
      DPG_CUDA(cudaMemcpyAsync(load_out, S.Fc + e * S.ntr, S.ntr * sizeof(double2), cudaMemcpyDeviceToHost, s));
    }
    DPG_CUDA(cudaStreamSynchronize(s));
    return DPGMG_OK;
  } catch (const Err& e2) {
    return fail(e2);
  }
}

int dpgmg_rhs(dpgmg_handle h, dpgmg_system sys, double* b_out) {
  if (!h || !sys || !b_out) return DPGMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  SystemImpl& S = sys->s;
  try {
    DPG_CUDA(cudaSetDevice(h->h.device));
    size_t n = (size_t)S.levels.back().mesh.ndof;
    DPG_CUDA(cudaMemcpyAsync(b_out, S.b, n * sizeof(double2), cudaMemcpyDeviceToHost, h->h.stream));
    DPG_CUDA(cudaStreamSynchronize(h->h.stream));
    return DPGMG_OK;
  } catch (const Err& e) {
    return fail(e);
  }
}

int dpgmg_apply(dpgmg_handle h, dpgmg_system sys, int op, int level, const double* x, double* y) {
  if (!h || !sys || !x || !y) return DPGMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  SystemImpl& S = sys->s;
  const int nl = (int)S.levels.size();
  if (level < 0 || level >= nl || op < 0 || op > DPGMG_OP_AFULL) return DPGMG_ERR_ARG;
  const Level& L = S.levels[level];
  if ((op == DPGMG_OP_RESTRICT || op == DPGMG_OP_PROLONG) && level == 0) return DPGMG_ERR_ARG;
  if ((op == DPGMG_OP_A || op == DPGMG_OP_SMOOTH) && level == 0 && L.P.np == 0) return DPGMG_ERR_ARG;
  if (op == DPGMG_OP_CONDENSE && L.kind != 2) return DPGMG_ERR_ARG;
  if (op == DPGMG_OP_COARSE && (level != 0 || !L.has_coarse)) return DPGMG_ERR_ARG;
  if (op == DPGMG_OP_AFULL && level != nl - 1) return DPGMG_ERR_ARG;
  try {
    DPG_CUDA(cudaSetDevice(h->h.device));
    cudaStream_t s = h->h.stream;
    int64_t nin = L.mesh.ndof, nout = L.mesh.ndof;
    if (op == DPGMG_OP_RESTRICT) nout = S.levels[level - 1].mesh.ndof;
    if (op == DPGMG_OP_PROLONG) nin = S.levels[level - 1].mesh.ndof;
    Alloc tmp;
    tmp.budget = (size_t)-1;
    tmp.stream = s;
    double2* dx = tmp.arr<double2>((size_t)nin);
    double2* dy = tmp.arr<double2>((size_t)nout);
    DPG_CUDA(cudaMemcpyAsync(dx, x, (size_t)nin * sizeof(double2), cudaMemcpyHostToDevice, s));
    apply_op(S, op, level, dx, dy, s);
    DPG_CUDA(cudaMemcpyAsync(y, dy, (size_t)nout * sizeof(double2), cudaMemcpyDeviceToHost, s));
    DPG_CUDA(cudaStreamSynchronize(s));
    return DPGMG_OK;
  } catch (const Err& e) {
    return fail(e);
  }
}

}  // extern "C"
