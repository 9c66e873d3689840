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
#include <string>

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
constexpr size_t kErrOffset = 2 * kRecBytes + kSortBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device.  The
// host-side name of the array is not a device address.  Outside stream
// capture the address is looked up on every call (after a device reset the
// module, and with it the array, may have moved); during capture the
// address found by the last call outside capture is used, so that no module
// load happens inside a capture.
cudaError_t scratch_for_current_device(cudaStream_t s, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  } else if (!g_scratch_ptr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Copies the caller's records into the scratch array (the sort clobbers its
// input).  A record whose pixel index is >= n_pix gets the index n_pix, one
// past every pixel, so that it sorts after all valid records and the reduce
// skips it (other pixels' sums stay exact), and sets the error word.
__global__ void copy_clamp_records(const SplatRec* __restrict__ in, SplatRec* __restrict__ out, size_t n,
                                   uint32_t n_pix, uint32_t* err) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  SplatRec r = in[i];
  if (r.pix >= n_pix) {
    r.pix = n_pix;
    atomicOr(err, kErrBadIndex);
  }
  out[i] = r;
}

}  // namespace
}  // namespace dr

extern "C" int dr_splat_records_noalloc(const void* recs, int64_t M, int32_t n_pix, double* accum,
                                        void* cuda_stream) {
  using namespace dr;
  if ((!recs && M > 0) || !accum || M < 0 || n_pix < 1 || n_pix == INT32_MAX) {
    set_error_message("dr_splat_records_noalloc: NULL pointer or bad size");
    return DR_ERR_INVALID_ARG;
  }
  if ((size_t)M > kNoAllocMaxRecords) {
    set_error_message("dr_splat_records_noalloc: more records than DR_NOALLOC_MAX_RECORDS (65536)");
    return DR_ERR_INVALID_ARG;
  }
  if (sort_scratch_bytes((size_t)M) > kSortBytes) {
    set_error_message("dr_splat_records_noalloc: internal scratch sizing error");
    return DR_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  void* base = nullptr;
  if (scratch_for_current_device(s, &base) != cudaSuccess) {
    cudaGetLastError();
    set_error_message("dr_splat_records_noalloc: cannot locate the device scratch array (make the first call on "
                      "a device outside stream capture)");
    return DR_ERR_CUDA;
  }
  char* p = static_cast<char*>(base);
  SplatRec* a = reinterpret_cast<SplatRec*>(p);
  SplatRec* b = reinterpret_cast<SplatRec*>(p + kRecBytes);
  void* sort_scratch = p + 2 * kRecBytes;
  uint32_t* err = reinterpret_cast<uint32_t*>(p + kErrOffset);
  // the error word reports this call alone (dr_splat_records_noalloc_status)
  if (cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess) {
    cudaGetLastError();
    set_error_message("dr_splat_records_noalloc: clearing the error word failed");
    return DR_ERR_CUDA;
  }
  if (M == 0) return DR_OK;
  // keys 0 .. n_pix (n_pix marks a bad record)
  int bits = 1;
  while (bits < 32 && (1ll << bits) < (long long)n_pix + 1) ++bits;
  copy_clamp_records<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(static_cast<const SplatRec*>(recs), a, (size_t)M,
                                                                  (uint32_t)n_pix, err);
  SplatRec* sorted = sort_splat_records(a, b, (size_t)M, bits, sort_scratch, s);
  launch_segment_reduce(sorted, (size_t)M, accum, (uint32_t)n_pix, err, s);
  if (cudaGetLastError() != cudaSuccess) {
    set_error_message("dr_splat_records_noalloc: kernel launch failed");
    return DR_ERR_CUDA;
  }
  return DR_OK;
}

extern "C" int dr_splat_records_noalloc_status(void* cuda_stream) {
  using namespace dr;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    set_error_message("dr_splat_records_noalloc_status: not available during stream capture");
    return DR_ERR_STATE;
  }
  void* base = nullptr;
  if (scratch_for_current_device(s, &base) != cudaSuccess) {
    cudaGetLastError();
    set_error_message("dr_splat_records_noalloc_status: cannot locate the device scratch array");
    return DR_ERR_CUDA;
  }
  uint32_t flags = 0;
  cudaError_t e = cudaMemcpyAsync(&flags, static_cast<char*>(base) + kErrOffset, sizeof(flags),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error_message((std::string("dr_splat_records_noalloc_status: ") + cudaGetErrorString(e)).c_str());
    return DR_ERR_CUDA;
  }
  if (flags) {
    set_error_message("dr_splat_records_noalloc: a record's pixel index was >= n_pix (the record was skipped)");
    return DR_ERR_DEVICE_CHECK;
  }
  return DR_OK;
}
