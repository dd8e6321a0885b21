// Partitioned operator: the structured box split into slabs of cells along z, one part per GPU (the
// distributed path of Sec. 2.6 and Sec. 3.7: each process owns a part of the mesh and adds the
// contributions of its neighbours on the shared DoFs).
//
// A part's lattice is a contiguous slice of the global DoF vector (lexicographic numbering, z slowest),
// and the lattice plane it shares with a neighbour is a contiguous range of it (first or last `plane`
// entries).  Each part runs the ordinary operator of its own box, with the interface faces natural
// (not Dirichlet): on a shared DoF it computes the contribution of its own cells, and the sum of both
// parts' contributions is the global operator's row.  The exchange adds the neighbour's partial plane
// into the part's own (mfx_halo_accumulate), except on Dirichlet points, which are identity rows on
// both sides.  Dot products run over the DoFs a part owns (its lattice without its upper interface
// plane) and are summed over the parts by the caller (two FP64 allreduces per CG iteration).
// Communication is the caller's: NCCL, MPI, a host-side coupler of two parts on one GPU, ...
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <vector>

#include "mfx_internal.h"

// propagate a failed status
#define PART_TRY(x)                 \
  do {                              \
    mfx_status st_ = (x);           \
    if (st_ != MFX_OK) return st_;  \
  } while (0)

namespace mfx {
namespace {

// y[i] += recv[i] on the free points of a lattice plane (Mx x My, x fastest)
template <typename Real>
__global__ void halo_accumulate_kernel(int Mx, int My, uint32_t dmask, const Real* __restrict__ recv,
                                       Real* __restrict__ y) {
  const int64_t n = (int64_t)Mx * My;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(i % Mx), J = (int)(i / Mx);
    const bool d = ((dmask & 1u) && I == 0) || ((dmask & 2u) && I == Mx - 1) || ((dmask & 4u) && J == 0) ||
                   ((dmask & 8u) && J == My - 1);
    if (!d) y[i] += recv[i];
  }
}

// r = b, x = 0, z = r / D, p = z
__global__ void ppcg_init_kernel(int64_t n, const double* __restrict__ b, const double* __restrict__ D,
                                 double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                                 double* __restrict__ p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = b[i];
    r[i] = ri;
    x[i] = 0.0;
    z[i] = ri / D[i];
    p[i] = z[i];
  }
}

// x += alpha p, r -= alpha q, z = r / D
__global__ void ppcg_update_kernel(int64_t n, double alpha, const double* __restrict__ p, const double* __restrict__ q,
                                   const double* __restrict__ D, double* __restrict__ x, double* __restrict__ r,
                                   double* __restrict__ z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    z[i] = ri / D[i];
  }
}

// p = z + beta p
__global__ void ppcg_direction_kernel(int64_t n, double beta, const double* __restrict__ z, double* __restrict__ p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

int grid_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)device_sm_count() * 8));
}

int64_t plane_of(const mfx_op* op) { return (int64_t)(op->k * op->nx + 1) * (op->k * op->ny + 1); }

mfx_status accumulate(const mfx_op* op, mfx_prec prec, int side, const void* recv, void* y, cudaStream_t s) {
  const int Mx = op->k * op->nx + 1, My = op->k * op->ny + 1;
  const int64_t plane = plane_of(op);
  const int64_t off = side == 0 ? 0 : op->n_dofs - plane;
  if (prec == MFX_F64)
    halo_accumulate_kernel<double><<<grid_for(plane), 256, 0, s>>>(Mx, My, op->dirichlet, (const double*)recv,
                                                                   (double*)y + off);
  else
    halo_accumulate_kernel<float><<<grid_for(plane), 256, 0, s>>>(Mx, My, op->dirichlet, (const float*)recv,
                                                                  (float*)y + off);
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}

// v's interface planes made consistent with the neighbours': send planes out, add what comes back
mfx_status exchange_sum(const mfx_op* op, const mfx_part_info* part, const mfx_comm* comm, double* v, cudaStream_t s) {
  const int64_t plane = part->plane;
  const bool side[2] = {part->has_lo != 0, part->has_hi != 0};
  for (int d = 0; d < 2; ++d)
    if (side[d])
      MFX_CUDA_TRY(cudaMemcpyAsync(comm->send[d], d == 0 ? v : v + op->n_dofs - plane, sizeof(double) * plane,
                                   cudaMemcpyDeviceToDevice, s));
  MFX_CUDA_TRY(cudaStreamSynchronize(s));
  if (comm->exchange(comm->user) != 0) return set_error(MFX_EINVAL, "partitioned solve: exchange callback failed");
  for (int d = 0; d < 2; ++d)
    if (side[d]) PART_TRY(accumulate(op, MFX_F64, d, comm->recv[d], v, s));
  return MFX_OK;
}

mfx_status allreduce(const mfx_comm* comm, double* vals, int n) {
  if (comm->allreduce(comm->user, vals, n) != 0)
    return set_error(MFX_EINVAL, "partitioned solve: allreduce callback failed");
  return MFX_OK;
}

}  // namespace
}  // namespace mfx

using namespace mfx;

extern "C" {

mfx_status mfx_partition_box(int32_t nx, int32_t ny, int32_t nz, int32_t degree, uint32_t dirichlet, int32_t n_parts,
                             int32_t part, mfx_part_info* info) {
  if (!info || nx < 1 || ny < 1 || nz < 1) return set_error(MFX_EINVAL, "partition: null info or empty box");
  if (degree < 1 || degree > kMaxDegree) return set_error(MFX_EUNSUPPORTED, "partition: degree out of 1..8");
  if (dirichlet > 0x3Fu) return set_error(MFX_EINVAL, "partition: Dirichlet mask above 0x3F");
  if (n_parts < 1 || n_parts > nz || part < 0 || part >= n_parts)
    return set_error(MFX_EINVAL, "partition: need 1 <= n_parts <= nz and 0 <= part < n_parts");
  const int32_t base = nz / n_parts, extra = nz % n_parts;
  info->nz = base + (part < extra ? 1 : 0);
  info->cz0 = part * base + std::min(part, extra);
  info->has_lo = part > 0 ? 1 : 0;
  info->has_hi = part < n_parts - 1 ? 1 : 0;
  info->reserved = 0;
  uint32_t d = dirichlet;
  if (info->has_lo) d &= ~(uint32_t)MFX_FACE_Z0;  // interfaces are natural faces of the part's box
  if (info->has_hi) d &= ~(uint32_t)MFX_FACE_Z1;
  info->dirichlet = d;
  info->plane = (int64_t)(degree * nx + 1) * (degree * ny + 1);
  info->dof0 = info->plane * degree * (int64_t)info->cz0;
  info->n_dofs = info->plane * ((int64_t)degree * info->nz + 1);
  info->n_owned = info->n_dofs - (info->has_hi ? info->plane : 0);
  info->vertex0 = (int64_t)(nx + 1) * (ny + 1) * info->cz0;
  return MFX_OK;
}

mfx_status mfx_halo_accumulate(const mfx_op* op, mfx_prec prec, int32_t side, const void* recv, void* y,
                               mfx_stream stream) {
  if (!op || !recv || !y) return set_error(MFX_EINVAL, "halo accumulate: null argument");
  if (!op->structured || op->dg) return set_error(MFX_EUNSUPPORTED, "halo accumulate: structured continuous operators");
  if (side != 0 && side != 1) return set_error(MFX_EINVAL, "halo accumulate: side must be 0 (low z) or 1 (high z)");
  if (prec != MFX_F64 && prec != MFX_F32) return set_error(MFX_EINVAL, "halo accumulate: unknown precision");
  return accumulate(op, prec, side, recv, y, (cudaStream_t)stream);
}

mfx_status mfx_solve_partitioned(const mfx_op* op, const mfx_part_info* part, const mfx_comm* comm, const double* b,
                                 double* x, const mfx_solve_params* params, mfx_solve_stats* stats,
                                 mfx_stream stream) try {
  if (!op || !part || !comm || !b || !x || !params || !comm->exchange || !comm->allreduce)
    return set_error(MFX_EINVAL, "partitioned solve: null argument");
  if (!op->structured || op->dg || !op->has_f64)
    return set_error(MFX_EUNSUPPORTED, "partitioned solve: structured continuous operators with FP64 data");
  if (part->n_dofs != op->n_dofs || part->plane != plane_of(op) || part->dirichlet != op->dirichlet)
    return set_error(MFX_EINVAL, "partitioned solve: the part's description does not match the operator");
  for (int d = 0; d < 2; ++d)
    if ((d == 0 ? part->has_lo : part->has_hi) && (!comm->send[d] || !comm->recv[d]))
      return set_error(MFX_EINVAL, "partitioned solve: missing exchange buffer");
  MFX_TRACE("mfx_solve_partitioned");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = op->n_dofs;
  double* w = nullptr;  // D, r, z, p, q and one device scalar
  MFX_CUDA_TRY(cudaMallocAsync(&w, sizeof(double) * (5 * n + 1), s));
  double *D = w, *r = w + n, *z = w + 2 * n, *p = w + 3 * n, *q = w + 4 * n, *dres = w + 5 * n;
  auto dot = [&](const double* u, const double* v, double* out) -> mfx_status {
    PART_TRY(launch_dot(op, MFX_F64, part->n_owned, u, v, dres, s));
    MFX_CUDA_TRY(cudaMemcpyAsync(out, dres, sizeof(double), cudaMemcpyDeviceToHost, s));
    MFX_CUDA_TRY(cudaStreamSynchronize(s));
    return MFX_OK;
  };
  mfx_solve_stats st{};
  st.status = MFX_OK;
  mfx_status rc = [&]() -> mfx_status {
    // the diagonal of the global operator on the shared DoFs is the sum of both parts' diagonals
    MFX_CUDA_TRY(cudaMemcpyAsync(D, op->d_diag64, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    PART_TRY(exchange_sum(op, part, comm, D, s));
    ppcg_init_kernel<<<grid_for(n), 256, 0, s>>>(n, b, D, x, r, z, p);
    MFX_CUDA_TRY(cudaGetLastError());
    double v2[2];
    PART_TRY(dot(b, b, &v2[0]));
    PART_TRY(dot(r, z, &v2[1]));
    PART_TRY(allreduce(comm, v2, 2));
    const double bb = v2[0];
    double rz = v2[1], rr = bb;
    const double tol2 = params->tol * params->tol * bb;
    int it = 0;
    while (rr > tol2 && bb > 0.0) {
      if (it >= params->max_it) {
        st.status = MFX_NOT_CONVERGED;
        break;
      }
      PART_TRY(launch_vmult(op, MFX_F64, p, q, s));
      PART_TRY(exchange_sum(op, part, comm, q, s));
      double pq;
      PART_TRY(dot(p, q, &pq));
      PART_TRY(allreduce(comm, &pq, 1));  // first allreduce of the iteration
      if (!(pq > 0.0) || !std::isfinite(pq)) {
        st.status = MFX_BREAKDOWN;
        break;
      }
      const double alpha = rz / pq;
      ppcg_update_kernel<<<grid_for(n), 256, 0, s>>>(n, alpha, p, q, D, x, r, z);
      MFX_CUDA_TRY(cudaGetLastError());
      PART_TRY(dot(r, z, &v2[0]));
      PART_TRY(dot(r, r, &v2[1]));
      PART_TRY(allreduce(comm, v2, 2));  // second allreduce: (r, z) and (r, r) together
      const double rz_new = v2[0];
      rr = v2[1];
      ++it;
      if (!std::isfinite(rr)) {
        st.status = MFX_BREAKDOWN;
        break;
      }
      ppcg_direction_kernel<<<grid_for(n), 256, 0, s>>>(n, rz_new / rz, z, p);
      MFX_CUDA_TRY(cudaGetLastError());
      rz = rz_new;
    }
    st.iterations = it;
    st.rel_residual = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    return MFX_OK;
  }();
  cudaFreeAsync(w, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (rc != MFX_OK) return rc;
  if (e != cudaSuccess) return cuda_error(e, "partitioned solve");
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return st.status;
} catch (...) {
  return host_exception();
}

}  // extern "C"
