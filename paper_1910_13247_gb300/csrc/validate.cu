// Checked mode: validation, on the device, of every index the vmult, diagonal and distribute kernels
// read from an operator's tables (the per-cell DoF and constraint-row codes, the constraint CSR, the
// tensor-product hanging tables and the cell lists).  It stands in for a memory checker: a corrupt or
// inconsistent table is reported as a count of bad entries and MFX_EMESH before any kernel indexes with
// it.  The checks read each table only at positions below its stated size and never use a checked
// value as an address.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>

#include "mfx_internal.h"

namespace mfx {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void count_bad(unsigned long long* bad, bool is_bad) {
  if (is_bad) atomicAdd(bad, 1ull);
}

// every code is a DoF in [0, n_dofs) or -1 - r for a constraint row r in [0, n_rows)
__global__ void check_cell_codes(int64_t n, const int32_t* __restrict__ codes, int64_t n_dofs, int64_t n_rows,
                                 unsigned long long* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = codes[i];
    count_bad(bad, e >= n_dofs || e < -n_rows);
  }
}

// cptr[0] = 0, non-decreasing, cptr[n_rows] = n_masters
__global__ void check_row_pointers(int64_t n_rows, const int64_t* __restrict__ cptr, int64_t n_masters,
                                   unsigned long long* bad) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= n_rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = cptr[r];
    bool b = p < 0 || p > n_masters;
    if (r == 0) b = b || p != 0;
    if (r == n_rows) b = b || p != n_masters;
    if (r < n_rows) b = b || cptr[r + 1] < p;
    count_bad(bad, b);
  }
}

// entries in [lo, hi)
__global__ void check_range(int64_t n, const int32_t* __restrict__ v, int64_t lo, int64_t hi, unsigned long long* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = v[i];
    count_bad(bad, x < lo || x >= hi);
  }
}

// per cell: only defined bits set (faces 0-5 with their halves 6-17; edges 0-11 with their halves
// 12-23, a half bit only on a hanging edge), and the cell's coarse-DoF slots inside hdofs, contiguous
// with the next cell's
__global__ void check_hanging_words(int64_t n_cells, const uint32_t* __restrict__ hface,
                                    const uint32_t* __restrict__ hedge, const int64_t* __restrict__ hoff,
                                    int64_t n_hdofs, int n, unsigned long long* bad) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_cells; c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t hf = hface[c], he = hedge[c];
    bool b = (hf >> 18) != 0u || (he >> 24) != 0u || ((he >> 12) & ~he & 0xFFFu) != 0u;
    for (int f = 0; f < 6; ++f)
      if (!(hf >> f & 1u)) b = b || ((hf >> (6 + 2 * f)) & 3u) != 0u;
    const int64_t slots = (int64_t)__popc(hf & 0x3Fu) * n * n + (int64_t)__popc(he & 0xFFFu) * n;
    const int64_t start = hoff[c];
    const int64_t end = c + 1 < n_cells ? hoff[c + 1] : n_hdofs;
    b = b || start < 0 || start + slots != end || end > n_hdofs;
    count_bad(bad, b);
  }
}

int grid_of(int64_t work) {
  const int64_t b = (work + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)device_sm_count() * 8));
}

bool env_checked() {
  const char* v = std::getenv("MFX_CHECKED");
  return v && *v && std::strcmp(v, "0") != 0;
}

}  // namespace

mfx_status validate_tables(const mfx_index_tables* t, int64_t* n_bad, cudaStream_t s) {
  if (!t || t->n_cells < 0 || t->nodes_1d < 1 || t->nodes_1d > kMaxN || t->n_dofs < 0 || t->n_rows < 0 ||
      t->n_masters < 0 || t->n_hdofs < 0 || t->n_list[0] < 0 || t->n_list[1] < 0)
    return set_error(MFX_EINVAL, "mfx_validate_tables: null descriptor or negative size");
  if ((t->n_cells > 0 && !t->cell_dofs) || (t->n_masters > 0 && !t->cmaster) || (t->n_rows > 0 && !t->cptr) ||
      (t->n_list[0] > 0 && !t->cell_list[0]) || (t->n_list[1] > 0 && !t->cell_list[1]) ||
      (t->hface && (!t->hedge || !t->hoff || (t->n_hdofs > 0 && !t->hdofs))))
    return set_error(MFX_EINVAL, "mfx_validate_tables: a table with entries has a null pointer");
  unsigned long long* d_bad = nullptr;
  MFX_CUDA_TRY(cudaMallocAsync((void**)&d_bad, sizeof(unsigned long long), s));
  cudaError_t e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), s);
  const int n = t->nodes_1d;
  if (e == cudaSuccess && t->n_cells > 0) {
    const int64_t m = t->n_cells * n * n * n;
    check_cell_codes<<<grid_of(m), kThreads, 0, s>>>(m, t->cell_dofs, t->n_dofs, t->n_rows, d_bad);
  }
  if (e == cudaSuccess && t->cptr)
    check_row_pointers<<<grid_of(t->n_rows + 1), kThreads, 0, s>>>(t->n_rows, t->cptr, t->n_masters, d_bad);
  if (e == cudaSuccess && t->n_masters > 0)
    check_range<<<grid_of(t->n_masters), kThreads, 0, s>>>(t->n_masters, t->cmaster, 0, t->n_dofs, d_bad);
  if (e == cudaSuccess && t->hface && t->n_cells > 0) {
    check_hanging_words<<<grid_of(t->n_cells), kThreads, 0, s>>>(t->n_cells, t->hface, t->hedge, t->hoff,
                                                                 t->n_hdofs, n, d_bad);
    if (t->n_hdofs > 0)
      check_range<<<grid_of(t->n_hdofs), kThreads, 0, s>>>(t->n_hdofs, t->hdofs, -1, t->n_dofs, d_bad);
  }
  for (int l = 0; l < 2 && e == cudaSuccess; ++l)
    if (t->n_list[l] > 0)
      check_range<<<grid_of(t->n_list[l]), kThreads, 0, s>>>(t->n_list[l], t->cell_list[l], 0, t->n_cells, d_bad);
  if (e == cudaSuccess) e = cudaGetLastError();
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_bad, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d_bad, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "mfx_validate_tables");
  if (n_bad) *n_bad = (int64_t)h;
  if (h) return set_error(MFX_EMESH, "index tables: " + std::to_string(h) + " entries out of range or inconsistent");
  return MFX_OK;
}

mfx_status validate_operator(const mfx_op* op, int64_t* n_bad, cudaStream_t s) {
  if (n_bad) *n_bad = 0;
  // SIPG (cell-major DoFs) and the structured row-batch kernels (lattice addresses, TMA copies clipped to
  // the vectors by their tensor maps) read no index tables
  if (op->dg || !op->d_cell_dofs) return MFX_OK;
  mfx_index_tables t;
  std::memset(&t, 0, sizeof(t));
  t.n_cells = op->n_cells;
  t.nodes_1d = op->n;
  t.n_dofs = op->n_dofs;
  t.cell_dofs = op->d_cell_dofs;
  t.cptr = op->d_cptr;
  if (op->structured) {  // lattice table of the per-cell kernels: every Dirichlet point is row 0, no masters
    t.n_rows = 1;
  } else {
    t.n_rows = op->n_constrained;
    t.n_masters = op->n_masters;
    t.cmaster = op->d_cmaster;
    if (op->d_hface) {
      t.hface = op->d_hface;
      t.hedge = op->d_hedge;
      t.hoff = op->d_hoff;
      t.hdofs = op->d_hdofs;
      t.n_hdofs = (int64_t)op->tables.hdofs.size();
    }
    t.cell_list[0] = op->d_cells_plain;
    t.n_list[0] = op->d_cells_plain ? op->n_cells_plain : 0;
    t.cell_list[1] = op->d_cells_hang;
    t.n_list[1] = op->d_cells_hang ? op->n_cells_hang : 0;
  }
  return validate_tables(&t, n_bad, s);
}

bool checked_mode() { return env_checked(); }

}  // namespace mfx

using namespace mfx;

extern "C" mfx_status mfx_validate_tables(const mfx_index_tables* tables, int64_t* n_bad, mfx_stream stream) {
  return validate_tables(tables, n_bad, (cudaStream_t)stream);
}

extern "C" mfx_status mfx_operator_validate(const mfx_op* op, int64_t* n_bad, mfx_stream stream) {
  if (!op) return set_error(MFX_EINVAL, "mfx_operator_validate: null operator");
  return validate_operator(op, n_bad, (cudaStream_t)stream);
}
