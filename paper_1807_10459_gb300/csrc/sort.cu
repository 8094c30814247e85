// sort.cu -- the library's one use of a vendor primitive: CUB's device radix
// sort of (32-bit key, int32 index) pairs, used to order samples along a
// space-filling curve before the estimator runs.  Kept in its own
// translation unit so the template instantiation compiles in parallel.
#include <cub/device/device_radix_sort.cuh>

#include "ksg_common.cuh"

namespace idtx {

cudaError_t sort_pairs_u32(void *tmp, size_t &tmp_bytes, const uint32_t *keys_in,
                           uint32_t *keys_out, const int32_t *vals_in, int32_t *vals_out, int n,
                           int end_bit, cudaStream_t stream)
{
    return cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys_out, vals_in, vals_out, n,
                                           0, end_bit, stream);
}

}  // namespace idtx
