// vmult instantiation for degree k = 1 (n = 2 points per direction).
#include <type_traits>
#include <algorithm>
#include <vector>
#include "vmult_launch.cuh"
#include "vmult_octree_q1.cuh"

namespace mfx {
template mfx_status launch_vmult_n<2>(const mfx_op*, mfx_prec, const void*, void*, cudaStream_t,
                                           const int32_t*);
template int brick_cells_per_batch<2>();
template int octree_pair_cells<2>();
template mfx_status prepare_vmult_n<2>(const mfx_op*);
template int brick_cells_candidates<2>(int*);
template int brick_kernel_candidates<2>(int*);

// k = 1 box-cell octree operators: the octants of the cell order (setup) and the vmult launch.
mfx_status build_q1_octants(mfx_op* op, cudaStream_t s) {
  const int64_t n = op->n_cells;
  const int sms = device_sm_count();
  auto grid = [&](int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)sms * 16)); };
  uint8_t* pass = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&pass, (size_t)std::max<int64_t>(1, n), s);
  if (e != cudaSuccess) return cuda_error(e, "octant table");
  q1_window_kernel<<<grid(n), 256, 0, s>>>(n, op->d_cell_dofs, pass);
  std::vector<uint8_t> hp((size_t)n);
  e = cudaMemcpyAsync(hp.data(), pass, (size_t)n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(pass, s);
  if (e != cudaSuccess) return cuda_error(e, "octant table");
  // octant starts in ascending order, never overlapping; the other cells one by one
  std::vector<int32_t> start, single;
  start.reserve((size_t)n / 8 + 1);
  int64_t next = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (i < next) continue;
    if (hp[(size_t)i]) {
      start.push_back((int32_t)i);
      next = i + 8;
    } else {
      single.push_back((int32_t)i);
    }
  }
  op->q1_n_oct = (int64_t)start.size();
  op->q1_n_single = (int64_t)single.size();
  auto upload = [&](int32_t** d, const std::vector<int32_t>& h, size_t count) -> cudaError_t {
    *d = nullptr;
    if (count == 0) return cudaSuccess;
    cudaError_t r = cudaMallocAsync((void**)d, count * sizeof(int32_t), s);
    if (r == cudaSuccess) op->bytes_device += (int64_t)(count * sizeof(int32_t));
    if (r == cudaSuccess && !h.empty()) r = cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    return r;
  };
  e = upload(&op->d_q1_start, start, start.size());
  if (e == cudaSuccess) e = upload(&op->d_q1_single, single, single.size());
  if (e == cudaSuccess) e = upload(&op->d_q1_octdofs, {}, start.size() * 27);
  if (e == cudaSuccess && op->q1_n_oct > 0) {
    q1_octant_dofs_kernel<<<grid(op->q1_n_oct), 256, 0, s>>>(op->q1_n_oct, op->d_q1_start, op->d_cell_dofs,
                                                             op->d_q1_octdofs);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host lists are copied before they go
  if (e != cudaSuccess) return cuda_error(e, "octant table");
  op->q1_split = true;
  return MFX_OK;
}

mfx_status launch_octree_q1_box(const mfx_op* op, const float* src, float* dst, cudaStream_t s, const int32_t* skip) {
  static int bps_oct = -1, bps_single = -1;
  if (bps_oct < 0) {
    int b = 0;
    MFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, octree_q1_octant_kernel, 256, 0));
    bps_oct = b > 0 ? b : 1;
    MFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, octree_q1_single_kernel, 256, 0));
    bps_single = b > 0 ? b : 1;
  }
  VmultArgs<2, float> pa;
  fill_vmult_args<2, float>(op, &pa);
  pa.skip = skip;
  const int sms = device_sm_count();
  const int pb = (int)std::max<int64_t>(1, std::min<int64_t>((op->n_dofs + 255) / 256, (int64_t)sms * 8));
  vmult_prologue<2, float><<<pb, 256, 0, s>>>(pa, src, dst);
  OctreeQ1Args a;
  a.cell_dofs = op->d_cell_dofs;
  a.oct_start = op->d_q1_start;
  a.oct_dofs = op->d_q1_octdofs;
  a.single = op->d_q1_single;
  a.n_oct = op->q1_n_oct;
  a.n_single = op->q1_n_single;
  a.cptr = op->d_cptr;
  a.cmaster = op->d_cmaster;
  a.cweight = op->d_cweight32;
  a.box = op->d_box32;
  a.wq[0] = (float)op->basis.wq[0];
  a.wq[1] = (float)op->basis.wq[1];
  a.skip = skip;
  if (a.n_oct > 0) {
    const int64_t n_wg = (a.n_oct + 3) / 4;
    const int grid = (int)std::min<int64_t>((n_wg + 7) / 8, (int64_t)sms * bps_oct);
    octree_q1_octant_kernel<<<grid, 256, 0, s>>>(a, src, dst);
  }
  if (a.n_single > 0) {
    const int grid = (int)std::min<int64_t>((a.n_single + 255) / 256, (int64_t)sms * bps_single);
    octree_q1_single_kernel<<<grid, 256, 0, s>>>(a, src, dst);
  }
  MFX_CUDA_TRY(cudaGetLastError());
  return MFX_OK;
}
}  // namespace mfx
