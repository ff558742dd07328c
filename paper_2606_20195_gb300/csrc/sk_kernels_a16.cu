// 16-bit-A instantiations of the tile kernel (binary16 and bfloat16 inputs), in their own translation
// unit so that they compile in parallel with the FP32 ones.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "sk_device.cuh"
#include "sk_internal.h"
#include "sk_tile.cuh"
#include "sk_tile_kernel.cuh"

namespace sk {

template <typename TA>
static TileKernelFn pick(int32_t rule) {
  switch (rule) {
    case kRN: return tile_kernel<kRN, TA>;
    case kSR: return tile_kernel<kSR, TA>;
    case kDither: return tile_kernel<kDither, TA>;
    case kBF16: return tile_kernel<kBF16, TA>;
    default: return tile_kernel<kFP32, TA>;
  }
}

TileKernelFn tile_kernel_a16(int32_t rule, int32_t a_type) {
  if (a_type == kAF16) return pick<__half>(rule);
  if (a_type == kABF16) return pick<__nv_bfloat16>(rule);
  return nullptr;
}

}  // namespace sk
