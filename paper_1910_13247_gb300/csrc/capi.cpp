// C-ABI entry points of libmfx (declared in include/mfx.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <array>
#include <map>
#include <mutex>

#include "mfx_internal.h"
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#endif

namespace mfx {

static thread_local std::string g_last_error;

mfx_status set_error(mfx_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#if __has_include(<nvtx3/nvToolsExt.h>)
TraceRange::TraceRange(const char* name) { nvtxRangePushA(name); }
TraceRange::~TraceRange() { nvtxRangePop(); }
#else
TraceRange::TraceRange(const char*) {}
TraceRange::~TraceRange() {}
#endif

// Called inside a catch handler at the C-ABI boundary: no C++ exception crosses it.
mfx_status host_exception() {
  try {
    throw;
  } catch (const std::bad_alloc&) {
    return set_error(MFX_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return set_error(MFX_EINVAL, std::string("host error: ") + e.what());
  } catch (...) {
    return set_error(MFX_EINVAL, "host error");
  }
}

mfx_status cuda_error(cudaError_t e, const char* where) {
  return set_error(MFX_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cached[dev] = v;
  }
  return cached[dev];
}

mfx_status launch_vmult(const mfx_op* op, mfx_prec prec, const void* src, void* dst, cudaStream_t s,
                        const int32_t* skip) {
  if (op->dg) return launch_dg_vmult(op, prec, src, dst, s, skip);
  switch (op->n) {
    case 2: return launch_vmult_n<2>(op, prec, src, dst, s, skip);
    case 3: return launch_vmult_n<3>(op, prec, src, dst, s, skip);
    case 4: return launch_vmult_n<4>(op, prec, src, dst, s, skip);
    case 5: return launch_vmult_n<5>(op, prec, src, dst, s, skip);
    case 6: return launch_vmult_n<6>(op, prec, src, dst, s, skip);
    case 7: return launch_vmult_n<7>(op, prec, src, dst, s, skip);
    case 8: return launch_vmult_n<8>(op, prec, src, dst, s, skip);
    case 9: return launch_vmult_n<9>(op, prec, src, dst, s, skip);
    default: return set_error(MFX_EUNSUPPORTED, "degree out of range");
  }
}

void free_workspace(mfx_op* op, cudaStream_t s);
mfx_status prepare_workspace(mfx_op* op);

mfx_status prepare_vmult(const mfx_op* op) {
  switch (op->n) {
    case 2: return prepare_vmult_n<2>(op);
    case 3: return prepare_vmult_n<3>(op);
    case 4: return prepare_vmult_n<4>(op);
    case 5: return prepare_vmult_n<5>(op);
    case 6: return prepare_vmult_n<6>(op);
    case 7: return prepare_vmult_n<7>(op);
    case 8: return prepare_vmult_n<8>(op);
    case 9: return prepare_vmult_n<9>(op);
    default: return set_error(MFX_EUNSUPPORTED, "degree out of range");
  }
}

int brick_cells_candidates_for_degree(int k, int* out) {
  switch (k + 1) {
    case 2: return brick_cells_candidates<2>(out);
    case 3: return brick_cells_candidates<3>(out);
    case 4: return brick_cells_candidates<4>(out);
    case 5: return brick_cells_candidates<5>(out);
    case 6: return brick_cells_candidates<6>(out);
    case 7: return brick_cells_candidates<7>(out);
    case 8: return brick_cells_candidates<8>(out);
    case 9: return brick_cells_candidates<9>(out);
    default: return 0;
  }
}

int brick_kernel_candidates_for_degree(int k, int* out) {
  switch (k + 1) {
    case 2: return brick_kernel_candidates<2>(out);
    case 3: return brick_kernel_candidates<3>(out);
    case 4: return brick_kernel_candidates<4>(out);
    case 5: return brick_kernel_candidates<5>(out);
    case 6: return brick_kernel_candidates<6>(out);
    case 7: return brick_kernel_candidates<7>(out);
    case 8: return brick_kernel_candidates<8>(out);
    case 9: return brick_kernel_candidates<9>(out);
    default: return 0;
  }
}

// Time the FP32 vmult of a structured operator with the metric laid out for `cb` cells per batch and
// kernel `kern`; milliseconds per application.  The metric's values do not change the time, so the
// candidates run on whatever the FP32 metric buffer holds (zeros before the geometry exists).
static mfx_status time_layout(mfx_op* op, int cb, int kern, float* x, float* y, cudaStream_t s, float* ms) {
  op->metric_cb = cb;
  op->nchunk = (op->nx + cb - 1) / cb;
  op->f32_kernel = kern;
  mfx_status st = launch_vmult(op, MFX_F32, x, y, s);  // warm-up (first launch sets kernel attributes)
  if (st != MFX_OK) return st;
  cudaEvent_t e0, e1;
  MFX_CUDA_TRY(cudaEventCreate(&e0));
  MFX_CUDA_TRY(cudaEventCreate(&e1));
  constexpr int kReps = 6;
  cudaEventRecord(e0, s);
  for (int r = 0; r < kReps && st == MFX_OK; ++r) st = launch_vmult(op, MFX_F32, x, y, s);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MFX_OK) return st;
  if (e != cudaSuccess) return cuda_error(e, "autotune timing");
  *ms = t / kReps;
  return MFX_OK;
}

// Autotuner: cells per batch and FP32 kernel for (degree, mesh size), measured once per process and
// device before the geometry is built (the geometry is then computed once, in the chosen layout).
// A requested batch size or kernel restricts the candidates to it.
static mfx_status choose_cells_per_batch(mfx_op* op, int requested, int requested_kernel, cudaStream_t s) {
  int cand[4], kcand[4];
  const int nc = brick_cells_candidates_for_degree(op->k, cand);
  const int nk = brick_kernel_candidates_for_degree(op->k, kcand);
  std::vector<std::pair<int, int>> tries;
  for (int i = 0; i < nc; ++i) {
    if (requested > 0 && cand[i] != requested) continue;
    for (int j = 0; j < nk; ++j) {
      if (requested_kernel > 0 && kcand[j] != requested_kernel) continue;
      tries.push_back({cand[i], kcand[j]});
    }
  }
  if (requested > 0 && tries.empty()) {
    bool cb_ok = false;
    for (int i = 0; i < nc; ++i) cb_ok = cb_ok || cand[i] == requested;
    if (!cb_ok) return set_error(MFX_EUNSUPPORTED, "cells_per_block not compiled for this degree");
  }
  if (tries.empty()) {
    if (requested_kernel > 0 && requested_kernel != MFX_KERNEL_TEN_PHASE)
      return set_error(MFX_EUNSUPPORTED, "structured_kernel not available for this degree");
    tries.push_back({requested > 0 ? requested : cand[0], MFX_KERNEL_TEN_PHASE});
  }
  auto take = [op](int cb, int kern) {
    op->metric_cb = cb;
    op->nchunk = (op->nx + cb - 1) / cb;
    op->f32_kernel = kern;
  };
  take(tries[0].first, tries[0].second);
  if (tries.size() < 2 || !op->has_f32) return MFX_OK;
  static std::mutex lock;
  static std::map<std::array<int64_t, 7>, std::pair<int, int>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const std::array<int64_t, 7> key = {op->k, op->nx, op->ny, op->nz, dev, requested, requested_kernel};
  {
    std::lock_guard<std::mutex> g(lock);
    auto it = cache.find(key);
    if (it != cache.end()) {
      take(it->second.first, it->second.second);
      return MFX_OK;
    }
  }
  float* x = nullptr;
  float* y = nullptr;
  MFX_CUDA_TRY(cudaMallocAsync(&x, sizeof(float) * op->n_dofs, s));
  cudaError_t e = cudaMallocAsync(&y, sizeof(float) * op->n_dofs, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(x, s);
    return cuda_error(e, "autotune vectors");
  }
  cudaMemsetAsync(x, 0, sizeof(float) * op->n_dofs, s);
  // three interleaved rounds over the candidates (a drift of the clocks hits every candidate alike);
  // the best round of each candidate decides
  std::vector<float> best_of(tries.size(), 1e30f);
  mfx_status st = MFX_OK;
  for (int round = 0; round < 3 && st == MFX_OK; ++round)
    for (size_t i = 0; i < tries.size() && st == MFX_OK; ++i) {
      float ms = 0;
      st = time_layout(op, tries[i].first, tries[i].second, x, y, s, &ms);
      if (st == MFX_OK) best_of[i] = std::min(best_of[i], ms);
    }
  std::pair<int, int> best = tries[0];
  float best_ms = 1e30f;
  for (size_t i = 0; i < tries.size(); ++i)
    if (best_of[i] < best_ms) {
      best_ms = best_of[i];
      best = tries[i];
    }
  cudaFreeAsync(x, s);
  cudaFreeAsync(y, s);
  cudaStreamSynchronize(s);
  if (st != MFX_OK) return st;
  take(best.first, best.second);
  std::lock_guard<std::mutex> g(lock);
  cache[key] = best;
  return MFX_OK;
}

int octree_pair_cells_for_degree(int k) {
  switch (k + 1) {
    case 2: return octree_pair_cells<2>();
    case 3: return octree_pair_cells<3>();
    case 4: return octree_pair_cells<4>();
    case 5: return octree_pair_cells<5>();
    case 6: return octree_pair_cells<6>();
    case 7: return octree_pair_cells<7>();
    case 8: return octree_pair_cells<8>();
    case 9: return octree_pair_cells<9>();
    default: return 0;
  }
}

int brick_cells_for_degree(int k) {
  switch (k + 1) {
    case 2: return brick_cells_per_batch<2>();
    case 3: return brick_cells_per_batch<3>();
    case 4: return brick_cells_per_batch<4>();
    case 5: return brick_cells_per_batch<5>();
    case 6: return brick_cells_per_batch<6>();
    case 7: return brick_cells_per_batch<7>();
    case 8: return brick_cells_per_batch<8>();
    case 9: return brick_cells_per_batch<9>();
    default: return 0;
  }
}

// Operator data is allocated in stream order on the creation stream (the operator is complete, and
// usable from any stream, once mfx_operator_create returns) and freed in stream order: making or
// dropping an operator never waits for the rest of the device.
// MFX_BOX_METRIC=0 in the environment keeps the full FP32 metric on box-cell octree operators (to compare
// the two forms); read at every operator creation.
static bool box_metric_enabled() {
  const char* v = std::getenv("MFX_BOX_METRIC");
  return !(v && v[0] == '0');
}

template <typename T>
static mfx_status dev_alloc(mfx_op* op, T** p, size_t count, cudaStream_t s) {
  *p = nullptr;
  if (count == 0) return MFX_OK;
  cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), s);
  if (e != cudaSuccess) {
    *p = nullptr;
    return set_error(MFX_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  op->bytes_device += (int64_t)(count * sizeof(T));
  return MFX_OK;
}

// The device's default memory pool keeps up to 16 GiB of freed operator memory for reuse instead of
// returning it at every synchronisation (the default threshold is 0), once per device and process.
static void keep_pool_memory() {
  static std::mutex lock;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> g(lock);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t threshold = (uint64_t)16 << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  }
  done.push_back(dev);
}

// Values of a host function at the operator's physical quadrature points (cell-major, q fastest, as
// mfx_quadrature_points lays them out), returned in a stream-ordered device array of n_cells n_q^3.
static mfx_status host_point_values(const mfx_op* op, mfx_point_fn f, void* user, double** out, cudaStream_t s) {
  const int64_t nq = op->n_cells * (int64_t)op->n * op->n * op->n;
  double* d = nullptr;
  *out = nullptr;
  if (cudaMallocAsync((void**)&d, sizeof(double) * 3 * std::max<int64_t>(1, nq), s) != cudaSuccess)
    return set_error(MFX_ENOMEM, "quadrature point buffer");
  std::vector<double> x((size_t)(3 * nq));
  mfx_status st = launch_qpoints(op, d, s);
  cudaError_t e = cudaSuccess;
  if (st == MFX_OK) e = cudaMemcpyAsync(x.data(), d, sizeof(double) * 3 * nq, cudaMemcpyDeviceToHost, s);
  if (st == MFX_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (st != MFX_OK || e != cudaSuccess) {
    cudaFreeAsync(d, s);
    return st != MFX_OK ? st : cuda_error(e, "quadrature points");
  }
  std::vector<double> v((size_t)nq);
  for (int64_t i = 0; i < nq; ++i) v[i] = f(&x[3 * i], user);
  e = cudaMemcpyAsync(d, v.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // v is a local buffer
  if (e != cudaSuccess) {
    cudaFreeAsync(d, s);
    return cuda_error(e, "point values upload");
  }
  *out = d;
  return MFX_OK;
}

// Lattice points of a structured mesh on no Dirichlet face.
static int64_t free_lattice_points(uint32_t dmask, int64_t Mx, int64_t My, int64_t Mz) {
  auto cnt = [](int64_t M, bool lo, bool hi) { return std::max<int64_t>(0, M - (lo ? 1 : 0) - (hi ? 1 : 0)); };
  return cnt(Mx, dmask & 1u, dmask & 2u) * cnt(My, dmask & 4u, dmask & 8u) * cnt(Mz, dmask & 16u, dmask & 32u);
}

// Frees everything in stream order on `s`; sync = wait for the whole device first (the contract of
// mfx_operator_destroy) and for the frees after.
static void destroy_op(mfx_op* op, cudaStream_t s = cudaStreamPerThread, bool sync = true) {
  if (!op) return;
  if (sync) cudaDeviceSynchronize();
  free_workspace(op, s);
  void* ptrs[] = {op->d_vertices, op->d_leaves, op->d_metric64, op->d_metric32, op->d_box32, op->d_q1_start,
                  op->d_q1_octdofs, op->d_q1_single, op->d_jxw, op->d_cell_dofs, op->d_cmask,
                  op->d_constrained, op->d_cptr, op->d_cmaster, op->d_cweight64, op->d_cweight32,
                  op->d_cell_hanging, op->d_diag64, op->d_diag32, op->d_scalars, op->d_partials, op->d_counter,
                  op->d_err, op->d_hface, op->d_hedge, op->d_hoff, op->d_hdofs, op->d_cells_plain,
                  op->d_cells_hang};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, s);
  if (sync) cudaStreamSynchronize(s);
  delete op;
}

}  // namespace mfx

using namespace mfx;

#define MFX_TRY(x)                  \
  do {                              \
    mfx_status st_ = (x);           \
    if (st_ != MFX_OK) {            \
      destroy_op(op);               \
      return st_;                   \
    }                               \
  } while (0)
#define MFX_CUDA_OP(call)                          \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      mfx_status st_ = cuda_error(e_, #call);      \
      destroy_op(op);                              \
      return st_;                                  \
    }                                              \
  } while (0)

extern "C" {

const char* mfx_last_error(void) { return g_last_error.c_str(); }
const char* mfx_version(void) { return "mfx 0.1 (sm_103a)"; }

mfx_status mfx_mesh_create_structured(mfx_mesh** out, int32_t nx, int32_t ny, int32_t nz, const double* vertices) try {
  if (!out) return set_error(MFX_EINVAL, "null output pointer");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return set_error(MFX_EINVAL, "mesh sizes must be positive");
  auto* m = new (std::nothrow) mfx_mesh();
  if (!m) return set_error(MFX_ENOMEM, "host allocation failed");
  m->m.structured = true;
  m->m.nx = nx;
  m->m.ny = ny;
  m->m.nz = nz;
  const size_t nv = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  m->m.vertices.resize(3 * nv);
  for (int l = 0; l <= nz; ++l)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        const size_t v = i + (size_t)(nx + 1) * (j + (size_t)(ny + 1) * l);
        if (vertices) {
          for (int d = 0; d < 3; ++d) m->m.vertices[3 * v + d] = vertices[3 * v + d];
        } else {
          m->m.vertices[3 * v + 0] = (double)i / nx;
          m->m.vertices[3 * v + 1] = (double)j / ny;
          m->m.vertices[3 * v + 2] = (double)l / nz;
        }
      }
  *out = m;
  return MFX_OK;
} catch (...) {
  return host_exception();
}

mfx_status mfx_mesh_create_octree(mfx_mesh** out, int32_t nx, int32_t ny, int32_t nz, const double* coarse_vertices,
                                  const int32_t* leaves, int64_t n_leaves) try {
  if (!out) return set_error(MFX_EINVAL, "null output pointer");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || !leaves || n_leaves < 1) return set_error(MFX_EINVAL, "bad octree arguments");
  mfx_mesh* m = nullptr;
  mfx_status st = mfx_mesh_create_structured(&m, nx, ny, nz, coarse_vertices);
  if (st != MFX_OK) return st;
  m->m.structured = false;
  m->m.leaves.assign(leaves, leaves + 4 * n_leaves);
  st = octree_sort_and_check(&m->m);
  if (st != MFX_OK) {
    delete m;
    return st;
  }
  *out = m;
  return MFX_OK;
} catch (...) {
  return host_exception();
}

void mfx_mesh_destroy(mfx_mesh* mesh) { delete mesh; }

mfx_status mfx_mesh_set_dirichlet(mfx_mesh* mesh, uint32_t faces) {
  if (!mesh || faces > kAllFaces) return set_error(MFX_EINVAL, "mfx_mesh_set_dirichlet: null mesh or faces > 0x3F");
  mesh->m.dirichlet = faces;
  return MFX_OK;
}

mfx_status mfx_mesh_get_dirichlet(const mfx_mesh* mesh, uint32_t* faces) {
  if (!mesh || !faces) return set_error(MFX_EINVAL, "null argument");
  *faces = mesh->m.dirichlet;
  return MFX_OK;
}

// SIPG operator (Sec. 6.1 benchmark): a structured mesh whose lattice is x_0 + (i h_x, j h_y, l h_z), a
// constant coefficient; n_cells x (k+1)^3 cell-major DoFs, no constraints, no stored geometry.
static mfx_status create_sipg(mfx_op** out, const Mesh& m, const mfx_op_desc* desc, cudaStream_t s) {
  if (!m.structured) return set_error(MFX_EUNSUPPORTED, "SIPG needs a structured mesh");
  if (desc->coef_kind != MFX_COEF_CONSTANT) return set_error(MFX_EUNSUPPORTED, "SIPG takes a constant coefficient");
  if (!(desc->coef_par[0] > 0.0)) return set_error(MFX_EINVAL, "SIPG coefficient must be positive");
  const double eta = desc->dg_penalty == 0.0 ? 1.0 : desc->dg_penalty;
  if (!(eta > 0.0)) return set_error(MFX_EINVAL, "SIPG penalty must be positive");
  const int nv[3] = {m.nx + 1, m.ny + 1, m.nz + 1};
  const double* v = m.vertices.data();
  auto vert = [&](int64_t i, int64_t j, int64_t l, int d) { return v[3 * (i + nv[0] * (j + nv[1] * l)) + d]; };
  double h[3];
  h[0] = (vert(m.nx, 0, 0, 0) - vert(0, 0, 0, 0)) / m.nx;
  h[1] = (vert(0, m.ny, 0, 1) - vert(0, 0, 0, 1)) / m.ny;
  h[2] = (vert(0, 0, m.nz, 2) - vert(0, 0, 0, 2)) / m.nz;
  if (!(h[0] > 0.0 && h[1] > 0.0 && h[2] > 0.0)) return set_error(MFX_EUNSUPPORTED, "SIPG needs a positively oriented lattice");
  const double tol = 1e-10 * std::max({h[0] * m.nx, h[1] * m.ny, h[2] * m.nz});
  for (int64_t l = 0; l < nv[2]; ++l)
    for (int64_t j = 0; j < nv[1]; ++j)
      for (int64_t i = 0; i < nv[0]; ++i) {
        const double want[3] = {vert(0, 0, 0, 0) + i * h[0], vert(0, 0, 0, 1) + j * h[1], vert(0, 0, 0, 2) + l * h[2]};
        for (int d = 0; d < 3; ++d)
          if (std::abs(vert(i, j, l, d) - want[d]) > tol)
            return set_error(MFX_EUNSUPPORTED, "SIPG needs a uniform axis-aligned lattice");
      }
  const int k = desc->degree;
  keep_pool_memory();
  mfx_op* op = new (std::nothrow) mfx_op();
  if (!op) return set_error(MFX_ENOMEM, "host allocation failed");
  op->k = k;
  op->n = k + 1;
  make_basis(k, &op->basis);
  const int prec = desc->precisions ? desc->precisions : 3;
  op->has_f64 = (prec & 1) != 0;
  op->has_f32 = (prec & 2) != 0;
  op->nx = m.nx;
  op->ny = m.ny;
  op->nz = m.nz;
  op->structured = true;
  op->dg = true;
  op->dirichlet = m.dirichlet;
  for (int d = 0; d < 3; ++d) {
    op->dg_h[d] = h[d];
    op->dg_origin[d] = vert(0, 0, 0, d);
  }
  op->dg_penalty = eta;
  op->dg_coef = desc->coef_par[0];
  op->n_cells = (int64_t)m.nx * m.ny * m.nz;
  op->n_dofs = op->n_cells * op->n * op->n * op->n;
  if (op->n_dofs >= ((int64_t)1 << 31)) {
    destroy_op(op);
    return set_error(MFX_EUNSUPPORTED, "more than 2^31 - 1 DoFs");
  }
  MFX_TRY(dev_alloc(op, &op->d_diag64, std::max<int64_t>(1, op->n_dofs), s));
  if (op->has_f32) MFX_TRY(dev_alloc(op, &op->d_diag32, std::max<int64_t>(1, op->n_dofs), s));
  MFX_TRY(dev_alloc(op, &op->d_scalars, 64, s));
  MFX_TRY(dev_alloc(op, &op->d_partials, 4096, s));
  MFX_TRY(dev_alloc(op, &op->d_counter, 16, s));
  MFX_CUDA_OP(cudaMemsetAsync(op->d_counter, 0, 16 * sizeof(unsigned int), s));
  MFX_TRY(dev_alloc(op, &op->d_err, 4, s));
  MFX_CUDA_OP(cudaMemsetAsync(op->d_err, 0, 4 * sizeof(int), s));
  MFX_TRY(launch_dg_diagonal(op, s));
  MFX_CUDA_OP(cudaStreamSynchronize(s));
  *out = op;
  return MFX_OK;
}

mfx_status mfx_operator_create(mfx_op** out, const mfx_mesh* mesh, const mfx_op_desc* desc, mfx_stream stream) try {
  MFX_TRACE("mfx_operator_create");
  if (!out || !mesh || !desc) return set_error(MFX_EINVAL, "null argument");
  *out = nullptr;
  const int k = desc->degree;
  if (k < 1 || k > kMaxDegree) return set_error(MFX_EUNSUPPORTED, "degree must be in 1..8");
  if (desc->n_q_1d != 0 && desc->n_q_1d != k + 1)
    return set_error(MFX_EUNSUPPORTED, "only n_q_1d = k + 1 is implemented");
  if (desc->coef_kind < MFX_COEF_CONSTANT || desc->coef_kind > MFX_COEF_FUNCTION)
    return set_error(MFX_EINVAL, "unknown coefficient kind");
  if (desc->coef_kind == MFX_COEF_QPOINT && !desc->coef_qpoint)
    return set_error(MFX_EINVAL, "MFX_COEF_QPOINT needs coef_qpoint");
  if (desc->coef_kind == MFX_COEF_FUNCTION && !desc->coef_fn)
    return set_error(MFX_EINVAL, "MFX_COEF_FUNCTION needs coef_fn");
  if (desc->discretization != MFX_CONTINUOUS && desc->discretization != MFX_SIPG)
    return set_error(MFX_EINVAL, "unknown discretization");
  if (desc->discretization == MFX_SIPG) return create_sipg(out, mesh->m, desc, (cudaStream_t)stream);
  cudaStream_t s = (cudaStream_t)stream;
  keep_pool_memory();
  mfx_op* op = new (std::nothrow) mfx_op();
  if (!op) return set_error(MFX_ENOMEM, "host allocation failed");
  op->k = k;
  op->n = k + 1;
  make_basis(k, &op->basis);
  const int prec = desc->precisions ? desc->precisions : 3;
  op->has_f64 = (prec & 1) != 0;
  op->has_f32 = (prec & 2) != 0;
  op->cells_per_block = desc->cells_per_block;
  const Mesh& m = mesh->m;
  op->nx = m.nx;
  op->ny = m.ny;
  op->nz = m.nz;
  op->structured = m.structured;
  op->dirichlet = m.dirichlet;
  const int n = op->n, n3 = n * n * n;
  if (m.structured) {
    op->n_cells = (int64_t)m.nx * m.ny * m.nz;
    const int64_t Mx = (int64_t)k * m.nx + 1, My = (int64_t)k * m.ny + 1, Mz = (int64_t)k * m.nz + 1;
    op->n_dofs = Mx * My * Mz;
    if (op->n_dofs >= ((int64_t)1 << 31)) {
      destroy_op(op);
      return set_error(MFX_EUNSUPPORTED, "more than 2^31 - 1 DoFs");
    }
    op->n_constrained = op->n_dofs - free_lattice_points(m.dirichlet, Mx, My, Mz);
    MFX_TRY(dev_alloc(op, &op->d_vertices, m.vertices.size(), s));
    MFX_CUDA_OP(cudaMemcpyAsync(op->d_vertices, m.vertices.data(), m.vertices.size() * sizeof(double),
                                cudaMemcpyHostToDevice, s));
    if (k >= 6 && op->has_f32) {
      // from k = 6 on the per-cell kernels beat the row-batch kernel for the FP32 vmult (k = 6 / 7 / 8
      // on 48^3 / 32^3 / 32^3 cells: 59.9 / 66.2 / 47.8 against 52.6 / 38.1 / 37.5 GDoF/s): index table
      // of the lattice (Dirichlet points as constraint rows without masters), FP32 metric per cell
      op->percell32 = true;
      MFX_TRY(dev_alloc(op, &op->d_cell_dofs, (size_t)op->n_cells * n3, s));
      MFX_TRY(dev_alloc(op, &op->d_cmask, (size_t)op->n_dofs, s));
      MFX_TRY(dev_alloc(op, &op->d_cptr, 2, s));
      MFX_TRY(dev_alloc(op, &op->d_cmaster, 1, s));
      MFX_TRY(dev_alloc(op, &op->d_cweight64, 1, s));
      MFX_TRY(dev_alloc(op, &op->d_cweight32, 1, s));
      MFX_TRY(launch_structured_index_tables(op, s));
    }
  } else {
    MFX_TRY(octree_tables(m, k, &op->tables));
    const OctreeTables& t = op->tables;
    op->n_cells = t.n_cells;
    op->n_dofs = t.n_dofs;
    op->n_constrained = (int64_t)t.constrained.size();
    op->n_masters = (int64_t)t.cmaster.size();
    for (size_t r = 0; r < t.constrained.size(); ++r)
      if (t.cptr[r + 1] > t.cptr[r]) ++op->n_hanging;
    // encoded cell DoFs: constrained -> -(row + 1)
    std::vector<int32_t> row_of(t.n_dofs, -1);
    for (size_t r = 0; r < t.constrained.size(); ++r) row_of[t.constrained[r]] = (int32_t)r;
    std::vector<int32_t> enc(t.cell_dofs.size());
    std::vector<uint8_t> cell_hang(t.n_cells, 0);
    for (size_t i = 0; i < enc.size(); ++i) {
      const int32_t d = t.cell_dofs[i];
      const int32_t r = row_of[d];
      enc[i] = r < 0 ? d : -(r + 1);
      if (r >= 0 && t.cptr[r + 1] > t.cptr[r]) cell_hang[i / n3] = 1;
    }
    // diagonal on cells with hanging nodes: one job per (cell, master of a hanging node of the cell);
    // the cell's other free nodes keep their own A_ii (flag `simple`)
    if (std::find(cell_hang.begin(), cell_hang.end(), 1) != cell_hang.end()) {
      op->hang_simple.assign(enc.size(), 1);
      std::vector<int32_t> ms;
      std::vector<int64_t> seen(t.n_dofs, -1);  // last cell that listed the DoF as a master
      for (int64_t c = 0; c < t.n_cells; ++c) {
        if (!cell_hang[c]) continue;
        ms.clear();
        for (int i = 0; i < n3; ++i) {
          const int32_t e = enc[c * n3 + i];
          if (e >= 0) continue;
          const int32_t r = -e - 1;
          for (int64_t p = t.cptr[r]; p < t.cptr[r + 1]; ++p) {
            const int32_t m = t.cmaster[p];
            if (seen[m] != c) {
              seen[m] = c;
              ms.push_back(m);
            }
          }
        }
        std::sort(ms.begin(), ms.end());
        for (int32_t m : ms) {
          op->hang_job_cell.push_back((int32_t)c);
          op->hang_job_master.push_back(m);
        }
        for (int i = 0; i < n3; ++i) {
          const int32_t e = enc[c * n3 + i];
          if (e < 0 || std::binary_search(ms.begin(), ms.end(), e)) op->hang_simple[c * n3 + i] = 0;
        }
      }
    }
    std::vector<uint8_t> mask(t.n_dofs, 0);
    for (int32_t c : t.constrained) mask[c] = 1;
    std::vector<float> w32(t.cweight.begin(), t.cweight.end());
    MFX_TRY(dev_alloc(op, &op->d_vertices, m.vertices.size(), s));
    MFX_TRY(dev_alloc(op, &op->d_leaves, m.leaves.size(), s));
    MFX_TRY(dev_alloc(op, &op->d_cell_dofs, enc.size(), s));
    MFX_TRY(dev_alloc(op, &op->d_cmask, mask.size(), s));
    MFX_TRY(dev_alloc(op, &op->d_constrained, t.constrained.size(), s));
    MFX_TRY(dev_alloc(op, &op->d_cptr, t.cptr.size(), s));
    MFX_TRY(dev_alloc(op, &op->d_cmaster, std::max<size_t>(1, t.cmaster.size()), s));
    MFX_TRY(dev_alloc(op, &op->d_cweight64, std::max<size_t>(1, t.cweight.size()), s));
    MFX_TRY(dev_alloc(op, &op->d_cweight32, std::max<size_t>(1, w32.size()), s));
    MFX_TRY(dev_alloc(op, &op->d_cell_hanging, cell_hang.size(), s));
    MFX_CUDA_OP(cudaMemcpyAsync(op->d_vertices, m.vertices.data(), m.vertices.size() * 8, cudaMemcpyHostToDevice, s));
    MFX_CUDA_OP(cudaMemcpyAsync(op->d_leaves, m.leaves.data(), m.leaves.size() * 4, cudaMemcpyHostToDevice, s));
    MFX_CUDA_OP(cudaMemcpyAsync(op->d_cell_dofs, enc.data(), enc.size() * 4, cudaMemcpyHostToDevice, s));
    MFX_CUDA_OP(cudaMemcpyAsync(op->d_cmask, mask.data(), mask.size(), cudaMemcpyHostToDevice, s));
    if (!t.constrained.empty())
      MFX_CUDA_OP(cudaMemcpyAsync(op->d_constrained, t.constrained.data(), t.constrained.size() * 4, cudaMemcpyHostToDevice, s));
    MFX_CUDA_OP(cudaMemcpyAsync(op->d_cptr, t.cptr.data(), t.cptr.size() * 8, cudaMemcpyHostToDevice, s));
    if (!t.cmaster.empty()) {
      MFX_CUDA_OP(cudaMemcpyAsync(op->d_cmaster, t.cmaster.data(), t.cmaster.size() * 4, cudaMemcpyHostToDevice, s));
      MFX_CUDA_OP(cudaMemcpyAsync(op->d_cweight64, t.cweight.data(), t.cweight.size() * 8, cudaMemcpyHostToDevice, s));
      MFX_CUDA_OP(cudaMemcpyAsync(op->d_cweight32, w32.data(), w32.size() * 4, cudaMemcpyHostToDevice, s));
    }
    MFX_CUDA_OP(cudaMemcpyAsync(op->d_cell_hanging, cell_hang.data(), cell_hang.size(), cudaMemcpyHostToDevice, s));
    // tensor-product form of the hanging constraints (used by the per-cell vmult)
    MFX_TRY(dev_alloc(op, &op->d_hface, t.hface.size(), s));
    MFX_TRY(dev_alloc(op, &op->d_hedge, t.hedge.size(), s));
    MFX_TRY(dev_alloc(op, &op->d_hoff, t.hoff.size(), s));
    MFX_TRY(dev_alloc(op, &op->d_hdofs, std::max<size_t>(1, t.hdofs.size()), s));
    MFX_CUDA_OP(cudaMemcpyAsync(op->d_hface, t.hface.data(), t.hface.size() * 4, cudaMemcpyHostToDevice, s));
    MFX_CUDA_OP(cudaMemcpyAsync(op->d_hedge, t.hedge.data(), t.hedge.size() * 4, cudaMemcpyHostToDevice, s));
    MFX_CUDA_OP(cudaMemcpyAsync(op->d_hoff, t.hoff.data(), t.hoff.size() * 8, cudaMemcpyHostToDevice, s));
    if (!t.hdofs.empty())
      MFX_CUDA_OP(cudaMemcpyAsync(op->d_hdofs, t.hdofs.data(), t.hdofs.size() * 4, cudaMemcpyHostToDevice, s));
    if (op->n_hanging > 0 && k >= kTensorHangMinDegree) {
      // the cells without hanging faces or edges run in the plain kernel, the others in the
      // tensor-product one
      std::vector<int32_t> plain, hang;
      for (int64_t c = 0; c < t.n_cells; ++c) ((t.hface[c] | t.hedge[c]) ? hang : plain).push_back((int32_t)c);
      op->n_cells_plain = (int64_t)plain.size();
      op->n_cells_hang = (int64_t)hang.size();
      MFX_TRY(dev_alloc(op, &op->d_cells_plain, std::max<size_t>(1, plain.size()), s));
      MFX_TRY(dev_alloc(op, &op->d_cells_hang, std::max<size_t>(1, hang.size()), s));
      if (!plain.empty())
        MFX_CUDA_OP(cudaMemcpyAsync(op->d_cells_plain, plain.data(), plain.size() * 4, cudaMemcpyHostToDevice, s));
      if (!hang.empty())
        MFX_CUDA_OP(cudaMemcpyAsync(op->d_cells_hang, hang.data(), hang.size() * 4, cudaMemcpyHostToDevice, s));
    }
  }
  const size_t nq = (size_t)op->n_cells * n3;
  size_t metric_entries = 6 * nq;
  if (op->structured) {
    // structured meshes: rows of cells in batches of metric_cb cells, metric interleaved per batch;
    // room for the largest layout among the compiled batch sizes (the autotuner may try each)
    int cand[4];
    const int nc = brick_cells_candidates_for_degree(k, cand);
    metric_entries = 0;
    for (int i = 0; i < nc; ++i) {
      const size_t nch = (size_t)(op->nx + cand[i] - 1) / cand[i];
      metric_entries = std::max(metric_entries, nch * op->ny * op->nz * cand[i] * 6 * n3);
    }
    op->metric_cb = cand[0];
    op->nchunk = (op->nx + cand[0] - 1) / cand[0];
  }
  // the FP64 metric is always built (geometry and diagonal are FP64); the FP32 copy on request
  size_t metric32_entries = metric_entries;
  if (!op->structured || op->percell32) {
    // octree (and per-cell structured) FP32 metric in runs of the paired kernel's batch size (the last
    // run padded)
    // (0: the per-cell kernel's [cell][6][q] layout)
    op->metric_cb32 = octree_pair_cells_for_degree(k);
    // with hanging nodes from kTensorHangMinDegree on, the per-cell kernel (tensor-product constraints)
    if (!op->structured && op->n_hanging > 0 && k >= kTensorHangMinDegree) op->metric_cb32 = 0;
    if (op->metric_cb32 > 0) {
      const size_t nb = (size_t)(op->n_cells + op->metric_cb32 - 1) / op->metric_cb32;
      metric32_entries = nb * op->metric_cb32 * 6 * n3;
    }
  }
  MFX_TRY(dev_alloc(op, &op->d_metric64, metric_entries, s));
  if (op->has_f32) MFX_TRY(dev_alloc(op, &op->d_metric32, metric32_entries, s));
  MFX_TRY(dev_alloc(op, &op->d_jxw, nq, s));
  MFX_TRY(dev_alloc(op, &op->d_diag64, std::max<int64_t>(1, op->n_dofs), s));
  if (op->has_f32) MFX_TRY(dev_alloc(op, &op->d_diag32, std::max<int64_t>(1, op->n_dofs), s));
  MFX_TRY(dev_alloc(op, &op->d_scalars, 64, s));
  MFX_TRY(dev_alloc(op, &op->d_partials, 4096, s));
  MFX_TRY(dev_alloc(op, &op->d_counter, 16, s));
  MFX_CUDA_OP(cudaMemsetAsync(op->d_counter, 0, 16 * sizeof(unsigned int), s));
  MFX_TRY(dev_alloc(op, &op->d_err, 4, s));
  MFX_CUDA_OP(cudaMemsetAsync(op->d_err, 0, 4 * sizeof(int), s));
  MFX_TRY(prepare_vmult(op));
  // a(x) from a host function: evaluated once at the physical quadrature points, then used as a
  // per-quadrature-point coefficient
  int coef_kind = desc->coef_kind;
  const double* coef_q = desc->coef_qpoint;
  double* coef_tmp = nullptr;
  if (coef_kind == MFX_COEF_FUNCTION) {
    MFX_TRY(host_point_values(op, desc->coef_fn, desc->coef_user, &coef_tmp, s));
    coef_kind = MFX_COEF_QPOINT;
    coef_q = coef_tmp;
  }
  mfx_status geo_st = MFX_OK;
  if (op->structured) {
    if (op->has_f32) MFX_CUDA_OP(cudaMemsetAsync(op->d_metric32, 0, sizeof(float) * metric32_entries, s));
    geo_st = choose_cells_per_batch(op, desc->cells_per_block, desc->structured_kernel, s);
  }
  if (geo_st == MFX_OK) geo_st = launch_geometry(op, coef_kind, desc->coef_par, coef_q, s);
  if (coef_tmp) cudaFreeAsync(coef_tmp, s);
  MFX_TRY(geo_st);
  MFX_TRY(launch_diagonal(op, s));
  // cells that are all axis-aligned boxes with a constant coefficient: the FP32 kernels take the metric
  // as one diagonal per cell (the specialised mapping for boxes parallel to the coordinate axes) — the
  // per-cell kernels (octrees; structured meshes from k = 6 on) from [cell][3], the structured row-batch
  // kernels from the first point of each line of the full FP32 metric, which they keep; not at k = 7,
  // whose FP32 kernel reads the full metric; MFX_BOX_METRIC=0 keeps the full metric everywhere
  if (!op->dg && op->has_f32 && k != 7 && box_metric_enabled()) {
    float* box = nullptr;
    int* flag = nullptr;
    MFX_TRY(dev_alloc(op, &box, (size_t)op->n_cells * 3, s));
    cudaError_t e = cudaMallocAsync((void**)&flag, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    mfx_status bst = e == cudaSuccess ? launch_box_check(op, box, flag, s) : cuda_error(e, "box metric");
    int not_box = 1;
    if (bst == MFX_OK) {
      e = cudaMemcpyAsync(&not_box, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) bst = cuda_error(e, "box metric");
    }
    if (flag) cudaFreeAsync(flag, s);
    if (bst == MFX_OK && not_box == 0 && op->structured && !op->percell32) {
      cudaFreeAsync(box, s);
      op->bytes_device -= (int64_t)((size_t)op->n_cells * 3 * sizeof(float));
      op->box32 = true;
    } else if (bst == MFX_OK && not_box == 0) {
      cudaFreeAsync(op->d_metric32, s);
      op->bytes_device -= (int64_t)(metric32_entries * sizeof(float));
      op->d_metric32 = nullptr;
      op->d_box32 = box;
      op->box32 = true;
      if (k == 1 && !op->structured) MFX_TRY(build_q1_octants(op, s));
    } else {
      cudaFreeAsync(box, s);
      op->bytes_device -= (int64_t)((size_t)op->n_cells * 3 * sizeof(float));
    }
    MFX_TRY(bst);
  }
  std::vector<int32_t>().swap(op->hang_job_cell);  // staged by the copies above: host copies no longer needed
  std::vector<int32_t>().swap(op->hang_job_master);
  std::vector<uint8_t>().swap(op->hang_simple);
  // the structured FP64 vmult works in double-float arithmetic on a pre-split metric
  if (op->structured) MFX_TRY(launch_metric_to_pairs(op, (int64_t)metric_entries, s));
  MFX_CUDA_OP(cudaStreamSynchronize(s));
  if (checked_mode()) MFX_TRY(validate_operator(op, nullptr, s));
  *out = op;
  return MFX_OK;
} catch (...) {
  return host_exception();
}

void mfx_operator_destroy(mfx_op* op) { destroy_op(op); }

mfx_status mfx_operator_release(mfx_op* op, mfx_stream stream) {
  if (!op) return set_error(MFX_EINVAL, "null operator");
  destroy_op(op, (cudaStream_t)stream, false);
  return MFX_OK;
}

mfx_status mfx_solver_prepare(mfx_op* op) {
  if (!op) return set_error(MFX_EINVAL, "null operator");
  if (!op->has_f64) return set_error(MFX_EINVAL, "solves need FP64 data");
  return prepare_workspace(op);
}

mfx_status mfx_operator_info(const mfx_op* op, mfx_op_info* info) {
  if (!op || !info) return set_error(MFX_EINVAL, "null argument");
  info->n_dofs = op->n_dofs;
  info->n_cells = op->n_cells;
  info->n_constrained = op->n_constrained;
  info->n_masters = op->n_masters;
  info->n_hanging = op->n_hanging;
  info->bytes_device = op->bytes_device + (int64_t)op->work_bytes;
  info->degree = op->k;
  info->n_q_1d = op->n;
  info->structured = op->structured ? 1 : 0;
  info->cells_per_block = op->structured ? op->metric_cb : (op->metric_cb32 > 0 ? op->metric_cb32 : 256 / (op->n * op->n));
  info->discretization = op->dg ? MFX_SIPG : MFX_CONTINUOUS;
  if (op->dg) info->cells_per_block = std::max(1, 128 / (op->n * op->n));
  info->structured_kernel = (op->structured && !op->dg && !op->percell32) ? op->f32_kernel : 0;
  info->box_metric = op->box32 ? 1 : 0;
  info->reserved = 0;
  return MFX_OK;
}

static void structured_tables(int nx, int ny, int nz, int k, uint32_t dmask, int32_t* cell_dofs,
                              int32_t* constrained, int64_t* cptr) {
  const int n = k + 1, n3 = n * n * n;
  const int64_t Mx = (int64_t)k * nx + 1, My = (int64_t)k * ny + 1, Mz = (int64_t)k * nz + 1;
  const int64_t C = (int64_t)nx * ny * nz;
  if (cell_dofs) {
    for (int64_t c = 0; c < C; ++c) {
      const int64_t cx = c % nx, cy = (c / nx) % ny, cz = c / ((int64_t)nx * ny);
      for (int i3 = 0; i3 < n; ++i3)
        for (int i2 = 0; i2 < n; ++i2)
          for (int i1 = 0; i1 < n; ++i1)
            cell_dofs[c * n3 + i1 + n * (i2 + n * i3)] =
                (int32_t)((cx * k + i1) + Mx * ((cy * k + i2) + My * (cz * k + i3)));
    }
  }
  int64_t t = 0;
  for (int64_t L = 0; L < Mz; ++L)
    for (int64_t J = 0; J < My; ++J)
      for (int64_t I = 0; I < Mx; ++I)
        if (on_dirichlet(dmask, I, J, L, Mx, My, Mz)) {
          if (constrained) constrained[t] = (int32_t)(I + Mx * (J + My * L));
          if (cptr) cptr[t] = 0;
          ++t;
        }
  if (cptr) cptr[t] = 0;
}

static void copy_tables(const OctreeTables& tb, int32_t* cell_dofs, int32_t* constrained, int64_t* cptr,
                        int32_t* cmaster, double* cweight) {
  if (cell_dofs) std::copy(tb.cell_dofs.begin(), tb.cell_dofs.end(), cell_dofs);
  if (constrained) std::copy(tb.constrained.begin(), tb.constrained.end(), constrained);
  if (cptr) std::copy(tb.cptr.begin(), tb.cptr.end(), cptr);
  if (cmaster) std::copy(tb.cmaster.begin(), tb.cmaster.end(), cmaster);
  if (cweight) std::copy(tb.cweight.begin(), tb.cweight.end(), cweight);
}

mfx_status mfx_mesh_table_sizes(const mfx_mesh* mesh, int32_t degree, int64_t* n_cells, int64_t* n_dofs,
                                int64_t* n_constrained, int64_t* n_masters) try {
  if (!mesh) return set_error(MFX_EINVAL, "null mesh");
  if (degree < 1 || degree > kMaxDegree) return set_error(MFX_EUNSUPPORTED, "degree must be in 1..8");
  const Mesh& m = mesh->m;
  int64_t C, N, NC, NM;
  if (m.structured) {
    const int64_t k = degree, Mx = k * m.nx + 1, My = k * m.ny + 1, Mz = k * m.nz + 1;
    C = (int64_t)m.nx * m.ny * m.nz;
    N = Mx * My * Mz;
    NC = N - free_lattice_points(m.dirichlet, Mx, My, Mz);
    NM = 0;
  } else {
    OctreeTables t;
    mfx_status st = octree_tables(m, degree, &t);
    if (st != MFX_OK) return st;
    C = t.n_cells;
    N = t.n_dofs;
    NC = (int64_t)t.constrained.size();
    NM = (int64_t)t.cmaster.size();
  }
  if (n_cells) *n_cells = C;
  if (n_dofs) *n_dofs = N;
  if (n_constrained) *n_constrained = NC;
  if (n_masters) *n_masters = NM;
  return MFX_OK;
} catch (...) {
  return host_exception();
}

mfx_status mfx_mesh_tables(const mfx_mesh* mesh, int32_t degree, int32_t* cell_dofs, int32_t* constrained,
                           int64_t* cptr, int32_t* cmaster, double* cweight) try {
  if (!mesh) return set_error(MFX_EINVAL, "null mesh");
  if (degree < 1 || degree > kMaxDegree) return set_error(MFX_EUNSUPPORTED, "degree must be in 1..8");
  const Mesh& m = mesh->m;
  if (m.structured) {
    structured_tables(m.nx, m.ny, m.nz, degree, m.dirichlet, cell_dofs, constrained, cptr);
    return MFX_OK;
  }
  OctreeTables t;
  mfx_status st = octree_tables(m, degree, &t);
  if (st != MFX_OK) return st;
  copy_tables(t, cell_dofs, constrained, cptr, cmaster, cweight);
  return MFX_OK;
} catch (...) {
  return host_exception();
}

mfx_status mfx_mesh_hanging_tables(const mfx_mesh* mesh, int32_t degree, uint32_t* hface, uint32_t* hedge,
                                   int64_t* hoff, int32_t* hdofs, int64_t* n_hdofs) try {
  if (!mesh) return set_error(MFX_EINVAL, "null mesh");
  if (degree < 1 || degree > kMaxDegree) return set_error(MFX_EUNSUPPORTED, "degree must be in 1..8");
  const Mesh& m = mesh->m;
  if (m.structured) {  // a structured mesh has no hanging nodes
    const int64_t C = (int64_t)m.nx * m.ny * m.nz;
    if (hface) std::fill(hface, hface + C, 0u);
    if (hedge) std::fill(hedge, hedge + C, 0u);
    if (hoff) std::fill(hoff, hoff + C, (int64_t)0);
    if (n_hdofs) *n_hdofs = 0;
    return MFX_OK;
  }
  OctreeTables t;
  mfx_status st = octree_tables(m, degree, &t);
  if (st != MFX_OK) return st;
  if (hface) std::copy(t.hface.begin(), t.hface.end(), hface);
  if (hedge) std::copy(t.hedge.begin(), t.hedge.end(), hedge);
  if (hoff) std::copy(t.hoff.begin(), t.hoff.end(), hoff);
  if (hdofs) std::copy(t.hdofs.begin(), t.hdofs.end(), hdofs);
  if (n_hdofs) *n_hdofs = (int64_t)t.hdofs.size();
  return MFX_OK;
} catch (...) {
  return host_exception();
}

mfx_status mfx_get_tables(const mfx_op* op, int32_t* cell_dofs, int32_t* constrained, int64_t* cptr,
                          int32_t* cmaster, double* cweight) {
  if (!op) return set_error(MFX_EINVAL, "null operator");
  if (op->dg) {  // cell-major DoFs, nothing constrained
    if (cell_dofs)
      for (int64_t i = 0; i < op->n_dofs; ++i) cell_dofs[i] = (int32_t)i;
    if (cptr) cptr[0] = 0;
    return MFX_OK;
  }
  if (op->structured) {
    structured_tables(op->nx, op->ny, op->nz, op->k, op->dirichlet, cell_dofs, constrained, cptr);
    return MFX_OK;
  }
  copy_tables(op->tables, cell_dofs, constrained, cptr, cmaster, cweight);
  return MFX_OK;
}

mfx_status mfx_vmult(const mfx_op* op, mfx_prec prec, const void* src, void* dst, mfx_stream stream) {
  if (!op || !src || !dst) return set_error(MFX_EINVAL, "mfx_vmult: null argument");
  if (src == dst) return set_error(MFX_EINVAL, "mfx_vmult: src and dst must not alias");
  if ((prec == MFX_F64 && !op->has_f64) || (prec == MFX_F32 && !op->has_f32) || (prec != MFX_F64 && prec != MFX_F32))
    return set_error(MFX_EINVAL, "mfx_vmult: precision not built for this operator");
  return launch_vmult(op, prec, src, dst, (cudaStream_t)stream);
}

mfx_status mfx_vmult_host(const mfx_op* op, mfx_prec prec, int32_t count, const void* const* src, void* const* dst,
                          mfx_stream stream) {
  MFX_TRACE("mfx_vmult_host");
  if (!op || count < 0 || (count > 0 && (!src || !dst))) return set_error(MFX_EINVAL, "mfx_vmult_host: bad argument");
  if ((prec == MFX_F64 && !op->has_f64) || (prec == MFX_F32 && !op->has_f32) || (prec != MFX_F64 && prec != MFX_F32))
    return set_error(MFX_EINVAL, "mfx_vmult_host: precision not built for this operator");
  if (count == 0) return MFX_OK;
  for (int32_t i = 0; i < count; ++i)
    if (!src[i] || !dst[i]) return set_error(MFX_EINVAL, "mfx_vmult_host: null vector");
  const size_t bytes = (size_t)op->n_dofs * (prec == MFX_F64 ? sizeof(double) : sizeof(float));
  // stages: upload (h2d), operator (cmp), download (d2h); buffers b = i mod 2
  cudaStream_t h2d = nullptr, cmp = nullptr, d2h = nullptr;
  cudaEvent_t ev[7] = {};
  void* buf[4] = {};  // in0, in1, out0, out1
  mfx_status st = MFX_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cmp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking);
  for (int i = 0; i < 7 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  // ev[0]: the caller's queued work; ev[1 + b]: input b uploaded; ev[3 + b]: vmult on buffers b done;
  // ev[5 + b]: output b downloaded
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h2d, ev[0], 0);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMallocAsync(&buf[i], bytes, h2d);
  if (e == cudaSuccess) e = cudaEventRecord(ev[5], h2d);  // buffers exist before any stage uses them
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cmp, ev[5], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(d2h, ev[5], 0);
  for (int32_t i = 0; i < count && e == cudaSuccess && st == MFX_OK; ++i) {
    const int b = i & 1;
    // upload i once the vmult of i - 2 has finished reading in[b]
    if (i >= 2) e = cudaStreamWaitEvent(h2d, ev[3 + b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf[b], src[i], bytes, cudaMemcpyHostToDevice, h2d);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1 + b], h2d);
    // vmult i once its input is in and the download of i - 2 has read out[b]
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cmp, ev[1 + b], 0);
    if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(cmp, ev[5 + b], 0);
    if (e == cudaSuccess) st = launch_vmult(op, prec, buf[b], buf[2 + b], cmp);
    if (e == cudaSuccess && st == MFX_OK) e = cudaEventRecord(ev[3 + b], cmp);
    // download i
    if (e == cudaSuccess && st == MFX_OK) e = cudaStreamWaitEvent(d2h, ev[3 + b], 0);
    if (e == cudaSuccess && st == MFX_OK) e = cudaMemcpyAsync(dst[i], buf[2 + b], bytes, cudaMemcpyDeviceToHost, d2h);
    if (e == cudaSuccess && st == MFX_OK) e = cudaEventRecord(ev[5 + b], d2h);
  }
  // free the staging after every stage is done, then wait for the results
  if (h2d && cmp && d2h) {
    cudaEvent_t done_cmp = ev[3], done_d2h = ev[5];
    if (cudaEventRecord(done_cmp, cmp) == cudaSuccess) cudaStreamWaitEvent(d2h, done_cmp, 0);
    if (cudaEventRecord(done_d2h, h2d) == cudaSuccess) cudaStreamWaitEvent(d2h, done_d2h, 0);
    for (int i = 0; i < 4; ++i)
      if (buf[i]) cudaFreeAsync(buf[i], d2h);
    const cudaError_t es = cudaStreamSynchronize(d2h);
    if (e == cudaSuccess) e = es;
  }
  for (int i = 0; i < 7; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (h2d) cudaStreamDestroy(h2d);
  if (cmp) cudaStreamDestroy(cmp);
  if (d2h) cudaStreamDestroy(d2h);
  if (st != MFX_OK) return st;
  if (e != cudaSuccess) return cuda_error(e, "mfx_vmult_host");
  return MFX_OK;
}

mfx_status mfx_device_check(const mfx_op* op, mfx_stream stream) {
  if (!op) return set_error(MFX_EINVAL, "null operator");
  int h = 0;
  MFX_CUDA_TRY(cudaMemcpyAsync(&h, op->d_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  MFX_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  if (h) {
    MFX_CUDA_TRY(cudaMemsetAsync(op->d_err, 0, sizeof(int), (cudaStream_t)stream));
    return set_error(MFX_ETIMEOUT, "a bounded device wait ran out (device error word was set)");
  }
  return MFX_OK;
}

mfx_status mfx_diagonal(const mfx_op* op, mfx_prec prec, void* diag, mfx_stream stream) {
  if (!op || !diag) return set_error(MFX_EINVAL, "mfx_diagonal: null argument");
  const void* srcp = prec == MFX_F64 ? (const void*)op->d_diag64 : (const void*)op->d_diag32;
  if (!srcp) return set_error(MFX_EINVAL, "mfx_diagonal: precision not built for this operator");
  const size_t bytes = (size_t)op->n_dofs * (prec == MFX_F64 ? 8 : 4);
  MFX_CUDA_TRY(cudaMemcpyAsync(diag, srcp, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return MFX_OK;
}

mfx_status mfx_quadrature_points(const mfx_op* op, double* xq, mfx_stream stream) {
  if (!op || !xq) return set_error(MFX_EINVAL, "mfx_quadrature_points: null argument");
  return launch_qpoints(op, xq, (cudaStream_t)stream);
}

mfx_status mfx_rhs(const mfx_op* op, const double* fq, double* b, mfx_stream stream) {
  if (!op || !fq || !b) return set_error(MFX_EINVAL, "mfx_rhs: null argument");
  return launch_rhs(op, fq, b, (cudaStream_t)stream);
}

mfx_status mfx_rhs_function(const mfx_op* op, mfx_point_fn f, void* user, double* b, mfx_stream stream) {
  if (!op || !f || !b) return set_error(MFX_EINVAL, "mfx_rhs_function: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  double* fq = nullptr;
  mfx_status st = host_point_values(op, f, user, &fq, s);
  if (st != MFX_OK) return st;
  st = launch_rhs(op, fq, b, s);
  cudaFreeAsync(fq, s);
  if (st == MFX_OK) MFX_CUDA_TRY(cudaStreamSynchronize(s));
  return st;
}

mfx_status mfx_mesh_transform(mfx_mesh* mesh, mfx_map_fn phi, void* user) try {
  if (!mesh || !phi) return set_error(MFX_EINVAL, "mfx_mesh_transform: null argument");
  std::vector<double>& v = mesh->m.vertices;
  for (size_t i = 0; i + 2 < v.size(); i += 3) {
    const double in[3] = {v[i], v[i + 1], v[i + 2]};
    double out[3] = {in[0], in[1], in[2]};
    phi(in, out, user);
    v[i] = out[0];
    v[i + 1] = out[1];
    v[i + 2] = out[2];
  }
  return MFX_OK;
} catch (...) {
  return host_exception();
}

mfx_status mfx_distribute(const mfx_op* op, double* x, mfx_stream stream) {
  if (!op || !x) return set_error(MFX_EINVAL, "mfx_distribute: null argument");
  if (op->dg) return MFX_OK;  // no constrained DoFs
  return launch_distribute(op, x, (cudaStream_t)stream);
}

}  // extern "C"
