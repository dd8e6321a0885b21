// vmult instantiation for degree k = 6 (n = 7 points per direction).
#include <type_traits>
#include <algorithm>
#include "vmult_launch.cuh"

namespace mfx {
template mfx_status launch_vmult_n<7>(const mfx_op*, mfx_prec, const void*, void*, cudaStream_t,
                                           const int32_t*);
template int brick_cells_per_batch<7>();
template int octree_pair_cells<7>();
template mfx_status prepare_vmult_n<7>(const mfx_op*);
template int brick_cells_candidates<7>(int*);
template int brick_kernel_candidates<7>(int*);
}  // namespace mfx
