// Internal declarations shared by the CUDA translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <future>
#include <mutex>
#include <string>
#include <memory>
#include <vector>

#include "../../include/dpgmg.h"
#include "host_mesh.h"

namespace dpgmg {

// ----------------------------------------------------------- error plumbing
struct Err {
  int code;
  std::string msg;
};
void set_last_error(const std::string& m);
#define DPG_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      throw ::dpgmg::Err{DPGMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
void count_launch();
void count_launches(long long n);
long long thread_launch_count();
#define DPG_CHECK_LAUNCH()            \
  do {                                \
    ::dpgmg::count_launch();          \
    DPG_CUDA(cudaGetLastError());     \
  } while (0)

// Device allocation tracked against the handle's budget.
// Stream-ordered (cudaMallocAsync / cudaFreeAsync on `stream`), so freeing
// one system never synchronises work of other streams.
struct Alloc {
  size_t budget = 0, used = 0, peak = 0;
  cudaStream_t stream = nullptr;
  std::vector<void*> ptrs;
  std::vector<size_t> sizes;
  void* get(size_t bytes);
  void release(void* p);     // free one allocation early (stream work using it must be done)
  template <class T> T* arr(size_t n) { return reinterpret_cast<T*>(get(n * sizeof(T) + 16)); }
  void free_all();
  ~Alloc() { free_all(); }
};

template <class T, class AL> T* upload(Alloc& A, const std::vector<T, AL>& h, cudaStream_t s) {
  T* d = A.arr<T>(h.size() ? h.size() : 1);
  if (!h.empty()) DPG_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return d;
}

// ----------------------------------------------------------- device structs
struct ECSRDev {
  int64_t nrows = 0, nent = 0, nnz = 0, max_nnz_row = 0;
  int64_t nnz_alg = 0;     // operator entries (algorithmic bytes count these)
  int32_t* row_ent = nullptr;
  int64_t* ent_start = nullptr;
  int32_t* ent_nd = nullptr;
  int64_t* col_ptr = nullptr;
  int32_t* col_idx = nullptr;
  int64_t* val_ptr = nullptr;
  double2* v64 = nullptr;
  float2* v32 = nullptr;   // complex64 values (= high parts of the double-float split)
  float2* vlo = nullptr;   // low parts: v64 ~ v32 + vlo (CG operator only)
  // rent[E] = 1: row entity E's rows are real once the unit phases are taken
  // out (A[r][c] = a[r][c] i^(s_r - s_c), s = 1 on DOFs below offU), and v32
  // (and vlo) hold the reals a: rows of nnz(E) reals from float offset
  // 2 val_ptr[E] (k_pack_ops).  Null: every entity complex64.
  uint8_t* rent = nullptr;
  int64_t offU = 0;
  int64_t nnz_real = 0;    // entries of the packed entities (host copy, after setup)
  // Entity-blocked SpMV work lists: tasks[i] = (entity, first row) groups of
  // G = 2^i rows of one entity (i = 1, 2, 3); rows with no entity are listed
  // in null_rows.  gsel[] is the group size chosen by the tuner for the
  // complex64, complex128 and double-float products (1 = one warp per row).
  int2* tasks[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t ntasks[4] = {0, 0, 0, 0};
  int32_t* null_rows = nullptr;
  int64_t n_null = 0;
  int gsel[3] = {1, 1, 1};
};

struct PatchDev {
  int64_t np = 0, nslots = 0, nvals = 0, max_n = 0, sum_sq = 0;
  int64_t* ptr = nullptr;
  int32_t* dofs = nullptr;
  int64_t* val_ptr = nullptr;
  int64_t* slot_ptr = nullptr;
  int32_t* slots = nullptr;
  double2* inv64 = nullptr;
  float2* inv32 = nullptr;
  int2* chunks = nullptr;      // (patch, first column) of each 32-column work item (complex128)
  int64_t nchunks = 0;
  int2* chunks64 = nullptr;    // the same for 64-column work items (complex64)
  int64_t nchunks64 = 0;
  int cols = 2;                // complex64 product: columns per lane (1 or 2), tuned at setup
  int variant = 2;             // complex64 single-vector product variant (smoother.cuh), tuned at setup
  // complex64 inverses of the mixed path: rflag[j] = 1 when patch j's block
  // holds the real matrix w (A^-1[r][c] = w[r][c] i^(s_r - s_c), s = 1 on
  // p-hat DOFs, global index < offU) as n rows of ld reals in its first half
  uint8_t* rflag = nullptr;
  int64_t offU = 0;
  int64_t real_sq = 0;         // sum of n_j^2 over the real patches (host copy, after setup)
  // Hermitian half storage (lower triangles packed by rows), used for the
  // complex64 operators of the mixed path
  bool half = false;
  int64_t nhvals = 0;
  int64_t* hptr = nullptr;     // per patch (+1): offset of its packed triangle
  float2* h32 = nullptr;
  int64_t scratch_entries() const { return nslots; }
  // DPGMG_FLAG_RECOMPUTE_PATCHES: no stored inverses; every application
  // gathers, factors (FP32) and applies the blocks window by window, a window
  // being consecutive patches of `order` (largest first) within wcap entries
  bool recompute = false;
  std::vector<int64_t> wq;       // window w = order positions [wq[w], wq[w+1])
  std::vector<int64_t> wch;      // window w's work items [wch[w], wch[w+1]) of wchunks
  int64_t wcap = 0;              // entries of the window buffer (and of its factorisation scratch)
  int64_t* worder = nullptr;     // patch order (largest first)
  int64_t* wvptr = nullptr;      // per patch: offset of its n x ld block within its window buffer
  int64_t* wsoff = nullptr;      // per order position: offset of its scratch copy
  int2* wchunks = nullptr;       // (patch, first column) of 64-column work items, window by window
  float2* wbuf = nullptr;
  float2* wscratch = nullptr;
  int* winfo = nullptr;
};

struct Level {
  MeshL mesh;
  int kind = 0;              // transition to the level below: 0 none, 1 p, 2 h
  int nloc = 0;
  double2* E = nullptr;      // element matrices [nelem][nloc][nloc]
  int64_t* dofs = nullptr;   // [nelem][nloc]
  ECSRDev A;                 // smoothing operator (A_l or macro M_l)
  PatchDev P;
  double theta = 0.0;
  int64_t n_smooth = 0;
  // p transition
  int32_t* inj = nullptr;
  // h transition
  int nS = 0, nI = 0;
  int64_t nK = 0;
  int64_t* S_glob = nullptr;
  int64_t* I_glob = nullptr;
  double2* Y64 = nullptr;    // [nK][nI][nS]   A_II^-1 A_IS
  double2* Ai64 = nullptr;   // [nK][nI][nI]   A_II^-1
  float2* Y32 = nullptr;
  float2* Ai32 = nullptr;
  int64_t *P_ptr = nullptr, *PT_ptr = nullptr, *sslot_ptr = nullptr;
  int32_t *P_col = nullptr, *PT_col = nullptr, *sslots = nullptr;
  double *P_val = nullptr, *PT_val = nullptr;
  char* smask = nullptr;
  // coarsest: packed L^-1 (rows of its lower triangle) and L^-H (rows of its upper triangle)
  int64_t N0 = 0;
  bool has_coarse = false;
  double2 *Lp64 = nullptr, *Up64 = nullptr;
  float2 *Lp32 = nullptr, *Up32 = nullptr;
};

struct Workspace;   // V-cycle work vectors (per precision)
struct Server;      // serving loop (server.cu)

struct ElemArgs;   // element-stage arguments (element.cu), kept for the error indicator

// Host side of an ECSR operator: index arrays and the SpMV work lists.
struct EcsrPrep {
  ECSRHost H;
  std::vector<int2> tasks[4];      // (entity, first row) groups of 2^i rows (i = 1, 2, 3)
  std::vector<int32_t> null_rows;  // rows with no entity
  int64_t max_nnz_row = 0;
};
EcsrPrep prep_ecsr(const MeshL& m, const std::vector<std::vector<int64_t>>& groups);
// entity lists of the elements of m (one group per element)
std::vector<std::vector<int64_t>> element_groups(const MeshL& m);

// Every host-only index structure of a hierarchy (integer bookkeeping: DOF
// maps, ECSR lists, macro transfer data, patch lists and work orders).  It
// depends on the meshes only, so setup builds it on a host thread while the
// element stage runs on the GPU; the later phases only upload and launch.
struct LevelPlan {
  std::vector<int64_t> cdofs;      // element DOFs of level l-1 (element-major)
  std::vector<int32_t> sel, inj;   // p-transition below l: local selection and injection
  MacroHost M;                     // h-transition below l: macro-element data
  EcsrPrep E;                      // level l's operator
  std::vector<char> smask;         // DOFs smoothed on level l
  int H = 2;                       // patch half-width in level-l elements
  Patches P;
  std::vector<int2> ch32, ch64;    // smoother work items of 32 / 64 rows, largest patch first
  std::vector<int64_t> order;      // inversion order, largest patch first
  int64_t max_n = 0, sum_sq = 0;
};
struct HostPlan {
  std::vector<int64_t> fdofs;      // element DOFs of the finest level
  std::vector<LevelPlan> lv;       // by level (entry 0 unused)
  bool has_acg = false;            // finest operator with element groups (CG operator), when
  EcsrPrep acg;                    // the finest level's own operator is not that
};

struct SystemImpl {
  dpgmg_problem pb;
  dpgmg_opts op;
  std::vector<double> wavespeed;
  std::vector<double> mf_coeffs;
  std::vector<double> u0;             // caller's impedance load samples (re, im), or empty
  std::vector<Level> levels;     // 0 = coarsest
  Alloc mem;
  int64_t nf = 0, ntr = 0, nelem = 0;
  double2* Yrec = nullptr;       // finest: [nelem][nf][ntr+1] K_ff^-1 [K_ft | F_f]
  double2* Fc = nullptr;         // finest: [nelem][ntr] condensed loads
  double2* b = nullptr;          // assembled right-hand side
  double t_setup_ms = 0.0;
  int64_t bytes_per_iter = 0;
  void* ws = nullptr;            // solver workspace
  double elem_flops = 0.0;       // algorithmic flops of the element stage
  double t_elem_ms = 0.0;        // its device time (events around the stage)
  // setup phase boundaries (events owned by the setup call; null outside it):
  // 0 start, 1 element stage, 2 operators, 3 smoothers, 4 after the coarsest
  // join, 5/6 coarsest factorisation start/end on the side stream, 7 end
  cudaEvent_t* ph_ev = nullptr;
  bool ph_side = false;
  std::future<std::shared_ptr<HostPlan>> host_plan;   // pending host index plan (setup only)
  std::shared_ptr<HostPlan> plan;                     // the plan, from the hierarchy build to the end of setup
  double t_phase[6] = {0, 0, 0, 0, 0, 0};
  int prof_which = 0;            // DPGMG_PROF_* being bracketed with events
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  std::vector<int> prof_graph_pairs;   // pairs recorded by a captured graph (re-read after each replay)
  double prof_graph_ms = 0.0;          // accumulated time of graph-recorded pairs
  long long prof_graph_n = 0;          // and their number of timed launches
  int64_t prof_bytes = 0;
  int coarse_blocks = 0;
  std::shared_ptr<ElemArgs> eargs;   // device tables of the element stage (resident with the system)
  // The coarsest factorisation is built on a side stream, concurrently with the
  // patch work of the level above it; its memory is tracked separately.
  cudaStream_t aux = nullptr;    // shared per setup stream, not owned
  Alloc mem_aux;
  size_t mem_used() const { return mem.used + mem_aux.used; }
  size_t mem_peak() const { return mem.peak + mem_aux.peak; }
  SystemImpl() = default;
  SystemImpl(const SystemImpl&) = delete;
  SystemImpl& operator=(const SystemImpl&) = delete;
  ~SystemImpl();
};

// Memory ledger of a handle: `used` = bytes held by systems set up with
// dpgmg_setup (reserved at the estimate during a setup), `serving` = the
// footprint estimates of the running serving requests; both under `ledger`.
struct HandleImpl {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  size_t used = 0;
  size_t serving = 0;
};

// ----------------------------------------------------------- stage entry points
// element.cu
int64_t element_chunk(int64_t nel, size_t per_elem);
void element_stage(SystemImpl& S, cudaStream_t st);
// condensed element matrices of a coarser level assembled directly on its mesh
// (the "stored" coarse operators of Sec. 3; constant wavespeed)
void element_stage_level(SystemImpl& S, Level& L, cudaStream_t st);
void recover_fields(SystemImpl& S, const double2* x, double2* fields, cudaStream_t st);
// DPG error indicator eta_K^2 of every finest element for the trace vector x (device)
void error_indicator(SystemImpl& S, const double2* x, double* eta2, cudaStream_t st);
// level.cu
void assemble_ecsr(Alloc& A, const EcsrPrep& P, ECSRDev& D, cudaStream_t st);
std::shared_ptr<HostPlan> plan_host(const SystemImpl& S);
// adds the element matrices of elements e0 .. e0 + nel - 1 of a grid with extents ext
// (colour passes: deterministic, no atomics)
void ecsr_add_elements(ECSRDev& D, const double2* E, const int64_t* dofs, int64_t nel, int nloc, int64_t e0,
                       const int ext[3], cudaStream_t st);
void build_hierarchy(SystemImpl& S, cudaStream_t st);
void assemble_rhs(SystemImpl& S, cudaStream_t st);
// coarse.cu
void coarse_setup(SystemImpl& S, Level& C0, int* info, cudaStream_t st, Alloc& A);
void coarse_apply64(const Level& C0, const double2* r, double2* e, double2* tmp, cudaStream_t st);
void coarse_apply32(const Level& C0, const float2* r, float2* e, float2* tmp, cudaStream_t st);
// y-products of the smoother in recompute mode (complex64 blocks factored in
// FP32): pbuf[slot] = A_jj^-1 (R_j r) for every patch of level L
void patch_recompute_apply(const Level& L, const float2* r, float2* pbuf, cudaStream_t st);
void patch_recompute_apply_blk(const Level& L, const float2* r, int64_t ldr, float2* pbuf, int64_t ldp, int K,
                               cudaStream_t st);
void coarse_apply64_blk(const Level& C0, const double2* r, double2* e, double2* tmp, int K, cudaStream_t st);
void coarse_apply32_blk(const Level& C0, const float2* r, float2* e, float2* tmp, int K, cudaStream_t st);
// solve.cu
// x0 (device, may be null): initial guess of the CG iteration (0 if null)
int pcg_solve(SystemImpl& S, cudaStream_t st, double2* x, dpgmg_stats* stats, const double2* x0 = nullptr);
int pcg_solve_block(SystemImpl& S, cudaStream_t st, int K, const double2* B, double2* X, dpgmg_stats* stats);
void apply_op(SystemImpl& S, int op, int level, const double2* x, double2* y, cudaStream_t st);
void ensure_workspace(SystemImpl& S, cudaStream_t st);
// CG operator split and kernel-variant tuning, run once at the end of setup
void prepare_solve(SystemImpl& S, cudaStream_t st);
ECSRDev* cg_operator_of(SystemImpl& S);
void free_workspace(SystemImpl& S);
void spmv64(const ECSRDev& A, const double2* x, double2* y, cudaStream_t st);
// enqueues the damping estimate of a level: rayleigh[0..1] (device) receive the
// numerator and denominator of lambda; theta = theta_from_rayleigh(num, den)
// (the level's operator must carry its double-float split v32 + vlo, its patch
// inverses their high parts in P.inv32 and low parts in plo)
void estimate_theta(SystemImpl& S, int level, double* rayleigh, const float2* plo, cudaStream_t st);
// double-float split of an operator's values: v32 (kept if already set) + vlo
void split_operator(Alloc& M, ECSRDev& A, int64_t offU, bool pack, cudaStream_t st);
void operator_c64(Alloc& M, ECSRDev& A, int64_t offU, bool pack, cudaStream_t st);
int64_t packed_entries(const ECSRDev& A);
// mixed path: real entities of operators and real patch inverses stored as reals
inline bool pack_storage(const SystemImpl& S) {
  return S.op.precision == DPGMG_PREC_MIXED && !(S.op.flags & DPGMG_FLAG_COMPLEX_STORAGE);
}
// hi + lo = v (complex64 parts of complex128 values)
void split_df(const double2* v, float2* hi, float2* lo, int64_t n, cudaStream_t st);
double theta_from_rayleigh(double num, double den);
void profile_read(SystemImpl& S, double* ms, long long* launches, long long* bytes);
// api.cu: validation, footprint estimate and the whole setup of one system
int validate_problem(const dpgmg_problem* pb, const dpgmg_opts* op);
size_t estimate_bytes(const dpgmg_problem* pb, const dpgmg_opts* op);
int64_t boundary_point_count(const dpgmg_problem* pb);   // points of the boundary load rule
void setup_system(SystemImpl& S, const dpgmg_problem* pb, const dpgmg_opts* op, size_t budget, cudaStream_t st);
void profile_clear(SystemImpl& S);
void smooth_apply64(const Level& L, const double2* r, double2* y, double theta, double2* scratch,
                    cudaStream_t st);

}  // namespace dpgmg

struct dpgmg_handle_s {
  dpgmg::HandleImpl h;
  std::mutex mu;       // serialises the calls on the handle
  std::mutex ledger;   // guards h.used and h.serving (innermost lock)
  dpgmg::Server* server = nullptr;
};
namespace dpgmg {
void server_shutdown(dpgmg_handle h);
// wakes the serving workers after memory was returned to the handle's ledger
void server_notify(dpgmg_handle h);
}
struct dpgmg_system_s {
  dpgmg::SystemImpl s;
};
