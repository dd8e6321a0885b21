// vmult instantiation for degree k = 4 (n = 5 points per direction).
#include <type_traits>
#include <algorithm>
#include "vmult_launch.cuh"

namespace mfx {
template mfx_status launch_vmult_n<5>(const mfx_op*, mfx_prec, const void*, void*, cudaStream_t,
                                           const int32_t*);
template int brick_cells_per_batch<5>();
template int octree_pair_cells<5>();
template mfx_status prepare_vmult_n<5>(const mfx_op*);
template int brick_cells_candidates<5>(int*);
template int brick_kernel_candidates<5>(int*);
}  // namespace mfx
