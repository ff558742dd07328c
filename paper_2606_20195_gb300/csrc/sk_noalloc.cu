// sk_apply_noalloc: the atomic-mode sketch with its scratch in a fixed static device array, for
// callers that cannot allocate device memory (allocator callbacks, fixed-footprint services,
// applications that own all device memory). Contract and limits: include/sk.h.
#include <cuda_runtime.h>

#include "../../include/sk.h"
#include "sk_hostutil.h"
#include "sk_internal.h"

namespace sk {
sk_status noalloc_tile_launch(const sk_plan_s* p, const float* A, int64_t lda, int64_t n, void* Y, TileLaunch* L);
size_t noalloc_elem_size(const sk_plan_s* p);
void noalloc_record(sk_plan_s* p, int64_t launches, int64_t R, int32_t kernel);
sk_status noalloc_read_status(unsigned* out);
}  // namespace sk

using namespace sk;

namespace {

// 16 MiB of scratch, held by every GPU that loads this library until the process exits.
constexpr size_t kScratchBytes = (size_t)16 << 20;
constexpr size_t kStatusBytes = 256;  // status word, padded
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device. Looked up on every call (cheap), so a
// module that the driver loaded again at another address (after cudaDeviceReset, for example) is
// never addressed through a stale pointer.
sk_status scratch_address(void** out) {
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr)
    return set_error(SK_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
  *out = ptr;
  return SK_OK;
}

}  // namespace

extern "C" SK_API sk_status sk_apply_noalloc(sk_plan p, const float* A, int64_t lda, int64_t n, void* Y,
                                             void* stream) {
  clear_error();
  TileLaunch L;
  sk_status s = noalloc_tile_launch(p, A, lda, n, Y, &L);
  if (s != SK_OK) return s;
  void* base = nullptr;
  s = scratch_address(&base);
  if (s != SK_OK) return s;
  const size_t need_P = sizeof(float) * (size_t)launch_P_floats(L);
  if (kStatusBytes + need_P > kScratchBytes)
    return set_error(SK_ERR_UNSUPPORTED,
                     "sk_apply_noalloc: this size needs %zu bytes of scratch, above the %zu-byte static array; "
                     "use sk_apply",
                     kStatusBytes + need_P, kScratchBytes);
  unsigned char* b = static_cast<unsigned char*>(base);
  cudaStream_t st = (cudaStream_t)stream;
  // The array keeps the previous call's contents: clear what this call needs at zero.
  cudaError_t e = cudaMemsetAsync(Y, 0, noalloc_elem_size(p) * (size_t)(L.d * L.n), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b, 0, kStatusBytes, st);
  if (e == cudaSuccess && need_P) e = cudaMemsetAsync(b + kStatusBytes, 0, need_P, st);
  if (e != cudaSuccess) return set_error(SK_ERR_CUDA, "zeroing: %s", cudaGetErrorString(e));
  L.status = reinterpret_cast<unsigned*>(b);
  L.P = need_P ? reinterpret_cast<float*>(b + kStatusBytes) : nullptr;
  int32_t launches = 0;
  e = launch_tile(L, st, &launches);
  if (e != cudaSuccess) return set_error(SK_ERR_CUDA, "sketch kernel launch: %s", cudaGetErrorString(e));
  noalloc_record(p, launches, L.R,
                 L.glob ? SK_KERNEL_GLOBAL : L.reg ? SK_KERNEL_REGISTER : L.own ? SK_KERNEL_OWNER : SK_KERNEL_TILE);
  return SK_OK;
}

// The status word of the last no-allocation call on the current device (the first word of the
// static array; the caller synchronizes first). A symbol copy: allocates nothing.
sk_status sk::noalloc_read_status(unsigned* out) {
  *out = 0u;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_noalloc_scratch, sizeof(unsigned), 0, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(SK_ERR_CUDA, "reading the no-allocation status word: %s", cudaGetErrorString(e));
  return SK_OK;
}
