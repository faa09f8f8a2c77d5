// Host-side mesh, DOF numbering and multigrid index structures.
//
// Structured axis-aligned hexahedral meshes; the global trace numbering and
// element-local orderings documented in include/dpgmg.h.  Everything here is
// integer bookkeeping plus the small 1D tables of the discretisation; the
// arithmetic of the method runs in the CUDA kernels.
#pragma once
#include <cstdint>
#include <functional>
#include <memory>
#include <new>
#include <utility>
#include <vector>

namespace dpgmg {

// One element-local trace function.
struct LocFn {
  int type;        // 0 p-hat, 1 u-hat
  int idx[3];      // p-hat: H^1 indices per axis
  int d, s, a, b;  // u-hat: normal axis, side (0 low / 1 high), Legendre modes
};

std::vector<LocFn> local_trace_functions(int p);
int n_trace_local(int p);

struct MeshL {
  int n[3] = {0, 0, 0};
  int p = 0;
  double x0[3], x1[3], h[3];
  int64_t nV = 0, nEd[3], nFd[3], nFid[3], nE = 0, nF = 0, nFi = 0;
  int64_t offE = 0, offF = 0, offU = 0, ndof = 0, nelem = 0;
  // entity ids: [0,nV) vertices, [nV, nV+nE) edges, then faces (p-hat),
  // then interior faces (u-hat)
  int64_t entE = 0, entF = 0, entU = 0, nent = 0;
  std::vector<LocFn> loc;

  void init(const int nn[3], int pp, const double a[3], const double b[3]);
  static int64_t lin(const int c[3], const int64_t ext[3]) {
    return c[0] + ext[0] * (c[1] + ext[1] * (int64_t)c[2]);
  }
  void elem_coord(int64_t e, int c[3]) const {
    c[0] = (int)(e % n[0]);
    c[1] = (int)((e / n[0]) % n[1]);
    c[2] = (int)(e / ((int64_t)n[0] * n[1]));
  }
  int64_t elem_index(const int c[3]) const {
    return c[0] + (int64_t)n[0] * (c[1] + (int64_t)n[1] * c[2]);
  }
  int64_t vertex(const int c[3]) const;
  int64_t edge(int d, const int c[3]) const;    // edge index (within all edges)
  int64_t face(int d, const int c[3]) const;    // face index (within all faces)
  int64_t iface(int d, const int c[3]) const;   // interior-face rank
  bool boundary_face(int d, const int c[3]) const { return c[d] == 0 || c[d] == n[d]; }
  // global DOF of each local trace function of element e (-1 if absent)
  void elem_dofs(int64_t e, int64_t* out) const;
  // entity id of each local trace function (-1 if absent)
  void elem_entities(int64_t e, int64_t* out) const;
  // first DOF and DOF count of entity E
  void ent_range(int64_t E, int64_t* start, int* nd) const;
  // entity of a DOF, and its centre in doubled coordinates (half-element units)
  int64_t dof_entity(int64_t g) const;
  void ent_center(int64_t E, int ctr[3]) const;
  // entity at a doubled-coordinate centre (kind from parity); -1 if none
  int64_t entity_at(const int ctr[3], bool uhat) const;
};

// Level plan from the finest (n, p) (p-coarsening to p_min, then halving n).
struct LevelSpec { int n[3]; int p; int kind_below; };  // kind 0 none, 1 p, 2 h
std::vector<LevelSpec> plan_levels(const int n[3], int p, int n_levels, int p_min);

// std::allocator whose value-initialisation of trivial elements is left out
// (resize leaves them uninitialised), for large arrays that are filled in
// parallel right after their allocation.
template <class T> struct NoInitAlloc : std::allocator<T> {
  template <class U> struct rebind { using other = NoInitAlloc<U>; };
  NoInitAlloc() = default;
  template <class U> NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <class U> void construct(U* p) noexcept { ::new ((void*)p) U; }
  template <class U, class... Args> void construct(U* p, Args&&... args) {
    ::new ((void*)p) U(std::forward<Args>(args)...);
  }
};

// First DOF and DOF count of an entity from the mesh's counts alone (the same
// rule as MeshL::ent_range), for device code that expands entity lists.
struct EntRanges {
  int64_t entE, entF, entU, offE, offF, offU;
  int p;
#if defined(__CUDACC__)
  __host__ __device__
#endif
  void range(int64_t E, int64_t* start, int* nd) const {
    if (E < entE) { *start = E; *nd = 1; }
    else if (E < entF) { *start = offE + (E - entE) * (p - 1); *nd = p - 1; }
    else if (E < entU) { *start = offF + (E - entF) * (int64_t)(p - 1) * (p - 1); *nd = (p - 1) * (p - 1); }
    else { *start = offU + (E - entU) * (int64_t)p * p; *nd = p * p; }
  }
};

// Runs body(lo, hi) over contiguous ranges of [0, n) on up to 16 host threads.
void host_parallel(int64_t n, const std::function<void(int64_t, int64_t)>& body);

// Entity-shared CSR ("ECSR"): rows are grouped by entity; all rows of one
// entity share one sorted list of column DOFs.  Values of row r of entity E
// start at val_ptr[E] + (r - start(E)) * nnz_row(E).
struct ECSRHost {
  int64_t nrows = 0;                 // = ndof of the level (non-row DOFs have row_ent = -1)
  std::vector<int32_t> row_ent;      // per DOF: compact row-entity index or -1
  std::vector<int64_t> ent_start;    // per row entity: first DOF
  std::vector<int32_t> ent_nd;       // per row entity: DOF count
  std::vector<int64_t> col_ptr;      // per row entity (+1): offset in col_idx
  // column entities per row entity (sorted, distinct): col_ent[cent_ptr[E] ..
  // cent_ptr[E + 1]); the expanded column DOFs (col_ptr) are the DOF ranges of
  // these entities in order, built on the device (assemble_ecsr)
  std::vector<int64_t> cent_ptr;
  std::vector<int32_t, NoInitAlloc<int32_t>> col_ent;
  std::vector<int64_t> val_ptr;      // per row entity (+1): value offset
  int64_t nnz() const { return val_ptr.empty() ? 0 : val_ptr.back(); }
  int64_t nnz_alg = 0;               // = nnz(): entries of the operator
  EntRanges er{};                    // the mesh's entity -> DOF range rule
};
// groups: for each super-element, the list of entity ids it touches.
ECSRHost build_ecsr(const MeshL& m, const std::vector<std::vector<int64_t>>& groups);

// Vertex patches of a level's smoothing space.  Rule R1 (r2 = false): a DOF
// is in the patch of coarse vertex w when every (macro-)element adjacent to
// its entity has w as a corner.  Rule R2 (r2 = true): when w lies in the
// closure of the coarse entity carrying the DOF (its own entity on p levels,
// the macro entity on h levels); the two differ only on boundary entities.
// H = coarse element width in doubled fine units (2 on p levels, 4 on h
// levels); nco = coarse mesh extents.
struct Patches {
  std::vector<int64_t> ptr;    // per patch (+1)
  std::vector<int32_t> dofs;   // patch-major DOF lists (sorted within a patch)
  std::vector<int64_t> val_ptr;// per patch (+1): offset of the n_j x ld_j block (ld_j = patch_ld(n_j))
  std::vector<int64_t> slot_ptr; // per DOF (+1): CSR of the DOF's slots in dofs[]
  std::vector<int32_t> slots;
};
Patches build_patches(const MeshL& m, const std::vector<char>& smask, int H, const int nco[3], bool r2);
int patch_axis_span(int ctr, int H, int nco, bool r2, int W[2]);
// Row length of a stored n x n patch block: n rounded up to even, so that
// every row of a complex64 block starts on a 16-byte boundary.
#if defined(__CUDACC__)
__host__ __device__
#endif
inline int64_t patch_ld(int64_t n) { return n + (n & 1); }
// Row length of a patch block stored as real numbers (a real-path inverse of
// the mixed path, in the first half of its complex64 block): n rounded up to
// a multiple of 4, so that every row starts on a 16-byte boundary.  4 ld >= 2
// ldr, so the real rows fit in the block.
#if defined(__CUDACC__)
__host__ __device__
#endif
inline int64_t patch_ldr(int64_t n) { return (n + 3) & ~(int64_t)3; }
// Patch sizes only (same rule), for memory estimates: n_j per coarse vertex.
// macro = true selects the h-level smoothing space (fine DOFs on the coarse skeleton).
std::vector<int64_t> patch_sizes(const MeshL& m, bool macro, int H, const int nco[3], bool r2);

// Macro-grid structure of one h-transition (fine level m, coarse level mc).
struct MacroHost {
  int nS = 0, nI = 0, nloc_f = 0, nloc_c = 0;
  std::vector<int32_t> child_map;   // [8][nloc_f] -> K-local index (S first, then I)
  std::vector<int64_t> S_glob;      // [nK][nS] fine global DOF (-1 absent)
  std::vector<int64_t> I_glob;      // [nK][nI]
  std::vector<double> IK;           // [nS][nloc_c] natural inclusion (real)
  // CSR of P (fine rows) and P^T (coarse rows)
  std::vector<int64_t> P_ptr, PT_ptr;
  std::vector<int32_t> P_col, PT_col;
  std::vector<double> P_val, PT_val;
  // per fine DOF: CSR of the (K, a) slots where it is an S DOF
  std::vector<int64_t> sslot_ptr;
  std::vector<int32_t> sslots;
  std::vector<char> smask;          // fine DOF on the coarse skeleton
  std::vector<std::vector<int64_t>> groups;  // macro element -> fine entities (for ECSR)
};
MacroHost build_macro(const MeshL& mf, const MeshL& mc);

// p-transition: positions of order p-1 local functions in the order-p list,
// and the coarse -> fine DOF injection.
void p_selection(int p, std::vector<int32_t>& sel);
void p_injection(const MeshL& mf, const MeshL& mc, std::vector<int32_t>& inj);

// 1D tables for the element kernels (enriched test order pt = p + 1).
struct Tables1D {
  int p, pt, nql;
  std::vector<double> Mleg;   // [pt+1] int L_a^2 = 1/(2a+1)
  std::vector<double> D;      // [pt+1][pt+1] int L_a' L_b
  std::vector<double> S;      // [pt+1][pt+1] int L_a' L_b'
  std::vector<double> Phi;    // [p+1][pt+1] int phi_k L_b
  std::vector<double> phi_end;// [p+1][2] phi_k(0), phi_k(1)
  std::vector<double> xq, wq; // load rule: nql Gauss points / weights on [0,1]
  std::vector<double> Lq;     // [pt+1][nql] L_a at load points
};
Tables1D make_tables(int p);
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);

// Boundary faces of the box mesh in the order of the impedance-load sample
// list: sides (d, s) for d = 0, 1, 2 and s = 0 (x_d = x0_d), s = 1 (x_d =
// x1_d); within a side the faces (j1, j2) along the tangential axes t1 < t2,
// j1 fastest.  off[2d + s] = first face of side (d, s); returns the count.
int64_t boundary_face_offsets(const int n[3], int64_t off[6]);
// Physical points of the boundary load rule (nql x nql Gauss points per
// boundary face, the t1 index fastest) in the order above: xyz[3 * count].
void boundary_points(const int n[3], const double x0[3], const double x1[3], int p, std::vector<double>& xyz);

}  // namespace dpgmg
