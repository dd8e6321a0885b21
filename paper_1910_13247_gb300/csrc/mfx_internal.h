// Internal declarations of libmfx (host side and kernel launchers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>
#include <cmath>

#include "../../include/mfx.h"

namespace mfx {

constexpr int kMaxDegree = 8;
constexpr int kMaxN = kMaxDegree + 1;

// ---------------------------------------------------------------- errors
mfx_status set_error(mfx_status code, const std::string& msg);
mfx_status cuda_error(cudaError_t e, const char* where);
mfx_status host_exception();  // inside a catch handler: the current exception as a status code

// Tracing: NVTX ranges around the library's host-side phases (operator and multigrid set-up, solves,
// batch ticks, server set-up of a request), visible to ncu --nvtx and other NVTX tools; without an
// attached tool each range costs a no-op call.  Compiled out where the NVTX headers are missing.
struct TraceRange {
  explicit TraceRange(const char* name);
  ~TraceRange();
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
#define MFX_TRACE(name) ::mfx::TraceRange mfx_trace_range_(name)
#define MFX_CUDA_TRY(call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::mfx::cuda_error(e_, #call); \
  } while (0)

// ----------------------------------------------------------- 1D rules
// Gauss-Legendre points/weights on [0,1] and Gauss-Lobatto nodes on [0,1].
void gauss_legendre(int n, double* x, double* w);
void gauss_lobatto(int k, double* x);
double lagrange_value(int n, const double* nodes, int j, double x);
double lagrange_derivative(int n, const double* nodes, int j, double x);

// Tables used by the kernels for degree k with n = k + 1 Gauss points:
//   S[q][j]  = l_j(xi_q)   (GLL Lagrange basis at Gauss points)
//   D[q][p]  = L_p'(xi_q)  (derivative of the Lagrange basis on the Gauss points)
//   Sd[q][j] = l_j'(xi_q)  (derivative of the GLL basis at Gauss points)
struct BasisTables {
  int k, n;
  double gll[kMaxN], xq[kMaxN], wq[kMaxN];
  double S[kMaxN * kMaxN], D[kMaxN * kMaxN], Sd[kMaxN * kMaxN];
};
void make_basis(int k, BasisTables* t);

// ----------------------------------------------------------------- mesh
// Faces of the box with homogeneous Dirichlet conditions: bit 2d (d = 0 x, 1 y, 2 z) is the face at
// coordinate 0, bit 2d + 1 the face at the far end; the other faces are natural (Neumann) boundaries.
constexpr uint32_t kAllFaces = 0x3F;
__host__ __device__ inline bool on_dirichlet(uint32_t mask, int64_t I, int64_t J, int64_t L, int64_t Mx, int64_t My,
                                             int64_t Mz) {
  return ((mask & 1u) && I == 0) || ((mask & 2u) && I == Mx - 1) || ((mask & 4u) && J == 0) ||
         ((mask & 8u) && J == My - 1) || ((mask & 16u) && L == 0) || ((mask & 32u) && L == Mz - 1);
}

struct Mesh {
  bool structured = true;
  uint32_t dirichlet = kAllFaces;     // Dirichlet faces (bit mask above)
  int nx = 0, ny = 0, nz = 0;
  std::vector<double> vertices;       // structured lattice or coarse lattice
  std::vector<int32_t> leaves;        // octree: sorted leaves, 4 per leaf
  int max_level = 0;
};

// DoF tables of an octree mesh (host).
// Degree from which octree vmults apply hanging constraints in tensor-product form (measured on octrees
// refined twice, FP32 GDoF/s, per-node masters / tensor product: k = 2 17.2 / 13.0, k = 3 17.5 / 18.1,
// k = 4 13.5 / 19.7, k = 6 6.5 / 22.0, k = 8 (paired kernel) about 3 / 14.5)
constexpr int kTensorHangMinDegree = 3;

struct OctreeTables {
  int64_t n_cells = 0, n_dofs = 0;
  std::vector<int32_t> cell_dofs;      // n_cells x n^3
  std::vector<int32_t> constrained;    // sorted
  std::vector<int64_t> cptr;           // n_constrained + 1
  std::vector<int32_t> cmaster;
  std::vector<double> cweight;
  // tensor-product form of the hanging constraints, per cell: hface bit f (face f = 2 d + side) if the
  // face lies on a coarser neighbour's face, bits 6 + 2 f / 7 + 2 f the halves (u, v) of that coarse face
  // it covers; hedge bit e (edge e = 4 d + 2 side_v + side_u, along d) if the edge lies on a coarser
  // neighbour's edge and on no hanging face of the cell, bit 12 + e the half; hoff: start in hdofs of
  // the cell's coarse DoFs (per hanging face in f order the (k+1)^2 coarse face DoFs, u fastest, then per
  // hanging edge in e order the k+1 coarse edge DoFs; constrained coarse DoFs are -1)
  std::vector<uint32_t> hface, hedge;
  std::vector<int64_t> hoff;
  std::vector<int32_t> hdofs;
};
mfx_status octree_sort_and_check(Mesh* m);
mfx_status octree_tables(const Mesh& m, int k, OctreeTables* out);

// ------------------------------------------------------------- operator
struct DeviceArray {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace mfx

struct mfx_mesh {
  mfx::Mesh m;
};

struct mfx_op {
  int k = 0, n = 0;
  int64_t n_cells = 0, n_dofs = 0, n_constrained = 0, n_masters = 0, n_hanging = 0;
  bool structured = true;
  uint32_t dirichlet = mfx::kAllFaces;    // Dirichlet faces of the box
  bool dg = false;                        // SIPG operator (cell-major DoFs, no constraints)
  bool percell32 = false;                 // structured, k >= 6: FP32 vmult by the per-cell kernels
  double dg_h[3] = {0, 0, 0}, dg_penalty = 1.0, dg_coef = 1.0, dg_origin[3] = {0, 0, 0};
  int nx = 0, ny = 0, nz = 0;             // structured cells per direction
  int cells_per_block = 0;
  int metric_cb = 0;                  // 0: metric [cell][6][q]; > 0: [batch][6][q][metric_cb] (structured)
  int nchunk = 0;                     // structured: batches per row of cells
  int metric_cb32 = 0;                // octree FP32 metric: 0 [cell][6][q]; > 0 [cell / cb][6][q][cb]
  int f32_kernel = MFX_KERNEL_TEN_PHASE;  // structured FP32 vmult kernel (MFX_KERNEL_*)
  bool has_f64 = false, has_f32 = false;
  mfx::BasisTables basis;
  // host tables (octree) or empty (structured)
  mfx::OctreeTables tables;
  // device data
  double* d_vertices = nullptr;      // the (coarse) vertex lattice (nx+1)(ny+1)(nz+1) x 3
  int32_t* d_leaves = nullptr;       // octree: the sorted leaves, (level, i, j, l) per cell
  double* d_metric64 = nullptr;      // FP64 metric; structured operators: float pairs after creation
  float* d_metric32 = nullptr;
  // FP32 octree operators whose cells are all boxes with axes along the coordinate axes and whose
  // coefficient is constant: the metric at quadrature point q of a cell is w_q diag(D) with one D per
  // cell, stored as [cell][3] instead of the full FP32 metric (which is then not kept)
  float* d_box32 = nullptr;
  bool box32 = false;
  // k = 1 box-cell operators: the octants of the cell order (first cell of each and its 27 node entries)
  // and the cells outside them
  bool q1_split = false;
  int64_t q1_n_oct = 0, q1_n_single = 0;
  int32_t* d_q1_start = nullptr;
  int32_t* d_q1_octdofs = nullptr;
  int32_t* d_q1_single = nullptr;
  double* d_jxw = nullptr;           // n_cells x n^3 (for the right-hand side)
  int32_t* d_cell_dofs = nullptr;    // octree: encoded cell DoFs (n_cells x n^3)
  uint8_t* d_cmask = nullptr;        // octree: 1 on constrained DoFs
  int32_t* d_constrained = nullptr;  // octree
  int64_t* d_cptr = nullptr;
  int32_t* d_cmaster = nullptr;
  double* d_cweight64 = nullptr;
  float* d_cweight32 = nullptr;
  uint8_t* d_cell_hanging = nullptr; // octree: 1 if a cell touches a hanging node
  uint32_t* d_hface = nullptr;       // octree: tensor-product hanging constraints (OctreeTables::hface)
  uint32_t* d_hedge = nullptr;
  int64_t* d_hoff = nullptr;
  int32_t* d_hdofs = nullptr;
  int32_t* d_cells_plain = nullptr;  // octree, tensor-product constraints: cells without / with hanging
  int32_t* d_cells_hang = nullptr;   // faces or edges (each list runs in its own kernel instantiation)
  int64_t n_cells_plain = 0, n_cells_hang = 0;
  // diagonal set-up on cells with hanging nodes (host; cleared once the diagonal is built):
  // one quadratic form v^T A_cell v per (cell, master) pair, v = the master's column of C on the cell
  std::vector<int32_t> hang_job_cell, hang_job_master;
  std::vector<uint8_t> hang_simple;  // n_cells x n^3: 1 if the node's A_ii is its DoF's whole share
  double* d_diag64 = nullptr;
  float* d_diag32 = nullptr;
  // solver workspace (allocated at create)
  void* d_work = nullptr;
  size_t work_bytes = 0;
  double* d_scalars = nullptr;       // device scalars for reductions / solver state
  double* d_partials = nullptr;      // reduction partials
  unsigned int* d_counter = nullptr; // last-block reduction counter
  int* d_err = nullptr;              // set by a kernel whose bounded wait ran out
  int64_t bytes_device = 0;
};

namespace mfx {

// Geometry precompute (FP64) and related setup kernels (geometry.cu).
mfx_status launch_geometry(mfx_op* op, int coef_kind, const double* par, const double* coef_q,
                           cudaStream_t s);
mfx_status launch_qpoints(const mfx_op* op, double* xq, cudaStream_t s);
mfx_status launch_rhs(const mfx_op* op, const double* fq, double* b, cudaStream_t s);
mfx_status launch_diagonal(mfx_op* op, cudaStream_t s);
// Box-cell check of an octree operator's FP64 metric ([cell][6][q]): box[cell][3] = the diagonal over the
// quadrature weight, *not_box set to 1 where a cell's metric is not w_q diag(D) to 1e-12.
mfx_status launch_box_check(const mfx_op* op, float* box, int* not_box, cudaStream_t s);
// k = 1 box-cell operators (vmult_k1.cu): the octant groups of the cell order, and the FP32 vmult that
// gathers and scatters an octant group's 27 nodes once.
mfx_status build_q1_octants(mfx_op* op, cudaStream_t s);
mfx_status launch_octree_q1_box(const mfx_op* op, const float* src, float* dst, cudaStream_t s, const int32_t* skip);
mfx_status launch_distribute(const mfx_op* op, double* x, cudaStream_t s);
mfx_status launch_metric_to_pairs(mfx_op* op, int64_t entries, cudaStream_t s);
// SIPG operator (dg.cu).
// structured meshes whose FP32 vmult runs on the per-cell kernels (geometry.cu)
mfx_status launch_structured_index_tables(mfx_op* op, cudaStream_t s);
mfx_status launch_dg_vmult(const mfx_op* op, mfx_prec prec, const void* src, void* dst, cudaStream_t s,
                           const int32_t* skip);
mfx_status launch_dg_diagonal(mfx_op* op, cudaStream_t s);
mfx_status launch_dg_qpoints(const mfx_op* op, double* xq, cudaStream_t s);
mfx_status launch_dg_rhs(const mfx_op* op, const double* fq, double* b, cudaStream_t s);

int device_sm_count();

// Checked mode (validate.cu): device-side validation of an operator's index tables; on when the
// environment variable MFX_CHECKED is set to anything but "0" (read at every operator creation).
mfx_status validate_tables(const mfx_index_tables* t, int64_t* n_bad, cudaStream_t s);
mfx_status validate_operator(const mfx_op* op, int64_t* n_bad, cudaStream_t s);
bool checked_mode();

// vmult (vmult_k*.cu): one launcher per degree.
mfx_status launch_vmult(const mfx_op* op, mfx_prec prec, const void* src, void* dst, cudaStream_t s,
                        const int32_t* skip = nullptr);
template <int N>
int brick_cells_per_batch();
// FP32 octree metric layout: cells per run for the paired kernel, 0 for the per-cell kernel.
template <int N>
int octree_pair_cells();
template <int N>
int brick_cells_candidates(int* out);
int brick_cells_candidates_for_degree(int k, int* out);
template <int N>
int brick_kernel_candidates(int* out);
int brick_kernel_candidates_for_degree(int k, int* out);
template <int N>
mfx_status prepare_vmult_n(const mfx_op* op);
mfx_status prepare_vmult(const mfx_op* op);
int brick_cells_for_degree(int k);
int octree_pair_cells_for_degree(int k);
template <int N>
mfx_status launch_vmult_n(const mfx_op* op, mfx_prec prec, const void* src, void* dst, cudaStream_t s,
                          const int32_t* skip);

// vector kernels (vector.cu)
mfx_status launch_dot(const mfx_op* op, mfx_prec prec, int64_t n, const void* a, const void* b,
                      double* result, cudaStream_t s);
int reduction_blocks(int64_t n);

}  // namespace mfx
