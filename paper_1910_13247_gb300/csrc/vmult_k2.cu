// vmult instantiation for degree k = 2 (n = 3 points per direction).
#include <type_traits>
#include <algorithm>
#include "vmult_launch.cuh"

namespace mfx {
template mfx_status launch_vmult_n<3>(const mfx_op*, mfx_prec, const void*, void*, cudaStream_t,
                                           const int32_t*);
template int brick_cells_per_batch<3>();
template int octree_pair_cells<3>();
template mfx_status prepare_vmult_n<3>(const mfx_op*);
template int brick_cells_candidates<3>(int*);
template int brick_kernel_candidates<3>(int*);
}  // namespace mfx
