// A splat entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: for example a render loop that works
// within a fixed device-memory budget, code running where another framework
// owns the device's allocator, or code that must not pay for the device-wide
// synchronisation that cudaMalloc / cudaFree can cause.  For them,
// dr_splat_records_noalloc does the same sort-and-reduce splat as
// dr_splat_records, but its scratch lives in a fixed-size array in device
// global memory that is part of this library (every GPU that loads the
// library holds it until the process exits).
#include <mutex>

#include "../../include/diffrestore.h"
#include "dr_internal.h"

namespace dr {
namespace {

constexpr size_t kNoAllocMaxRecords = DR_NOALLOC_MAX_RECORDS;
constexpr size_t kRecBytes = kNoAllocMaxRecords * sizeof(SplatRec);
// two record buffers (the input copy and the sort's ping-pong buffer), the
// sort's histogram / offset / scan space, and one error word
constexpr size_t kSortBytes = 2 * ((256 * ((kNoAllocMaxRecords + 2047) / 2048) * 4 + 255) & ~(size_t)255) + 4096;
constexpr size_t kScratchBytes = 2 * kRecBytes + kSortBytes + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (looked up
// once per device; the host-side name of the array is not a device address).
cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace dr

extern "C" int dr_splat_records_noalloc(const void* recs, int64_t M, int32_t n_pix, double* accum,
                                        void* cuda_stream) {
  using namespace dr;
  if ((!recs && M > 0) || !accum || M < 0 || n_pix < 1) {
    set_error_message("dr_splat_records_noalloc: NULL pointer or bad size");
    return DR_ERR_INVALID_ARG;
  }
  if ((size_t)M > kNoAllocMaxRecords) {
    set_error_message("dr_splat_records_noalloc: more records than DR_NOALLOC_MAX_RECORDS (65536)");
    return DR_ERR_INVALID_ARG;
  }
  if (M == 0) return DR_OK;
  if (sort_scratch_bytes((size_t)M) > kSortBytes) {
    set_error_message("dr_splat_records_noalloc: internal scratch sizing error");
    return DR_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) {
    cudaGetLastError();
    set_error_message("dr_splat_records_noalloc: cannot locate the device scratch array");
    return DR_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  char* p = static_cast<char*>(base);
  SplatRec* a = reinterpret_cast<SplatRec*>(p);
  SplatRec* b = reinterpret_cast<SplatRec*>(p + kRecBytes);
  void* sort_scratch = p + 2 * kRecBytes;
  uint32_t* err = reinterpret_cast<uint32_t*>(p + 2 * kRecBytes + kSortBytes);
  int bits = 1;
  while (bits < 32 && (1ll << bits) < (long long)n_pix) ++bits;
  // the caller's records are inputs: sort a copy (the sort clobbers its input)
  if (cudaMemcpyAsync(a, recs, (size_t)M * sizeof(SplatRec), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess) {
    cudaGetLastError();
    set_error_message("dr_splat_records_noalloc: copy into the scratch array failed");
    return DR_ERR_CUDA;
  }
  SplatRec* sorted = sort_splat_records(a, b, (size_t)M, bits, sort_scratch, s);
  launch_segment_reduce(sorted, (size_t)M, accum, (uint32_t)n_pix, err, s);
  if (cudaGetLastError() != cudaSuccess) {
    set_error_message("dr_splat_records_noalloc: kernel launch failed");
    return DR_ERR_CUDA;
  }
  return DR_OK;
}

