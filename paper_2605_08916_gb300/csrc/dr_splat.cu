// Atomic-free, deterministic splatting of the ergodic-average contributions
// into the FP64 image, and Resolve (Alg. 3).
//
// The paper atomically adds dt * f / p into an accumulation buffer per chain
// (Alg. 1, Accumulate).  Here every chain-step emits a 16-B record
// (pixel, rgb); a batch of records is sorted by pixel with a stable LSD radix
// sort (8-bit digits; per-tile digit histograms in shared memory, a
// device-wide exclusive scan, and a stable scatter that ranks equal digits
// with warp match-any) and then reduced per pixel in FP64 by one writer per
// pixel.  The sum order is the records' (step, chain) order, so the image is
// bit-reproducible and equals a sequential FP64 sum of the same records.
#include "dr_internal.h"

namespace dr {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kScanThreads = 1024;
constexpr int kScanChunk = 2048;

DR_D uint32_t rec_key(const SplatRec& r) { return r.pix; }
DR_D uint32_t rec_key(const uint2& r) { return r.x; }

template <class R>
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const R* __restrict__ in, size_t n, int shift,
                                                                  uint32_t* __restrict__ hist, int ntiles) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const size_t base = (size_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const size_t i = base + (size_t)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(rec_key(in[i]) >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one 8-bit digit pass.  Each block ranks its tile of
// kSortTile elements (rounds of 256: warp match-any ranks equal digits, a
// per-digit prefix over the warps orders the warps), places the tile in
// shared memory in (digit, input) order, and then writes it out in that
// order: the elements of one digit leave the block as one contiguous run, so
// the global stores are coalesced.  The output is the same stable
// permutation as placing each element directly.
template <class R>
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const R* __restrict__ in, R* __restrict__ out,
                                                                     size_t n, int shift,
                                                                     const uint32_t* __restrict__ offs, int ntiles) {
  __shared__ uint32_t run[256];     // elements of each digit ranked so far in this tile
  __shared__ uint32_t whist[kSortThreads / 32][256];
  __shared__ uint32_t dstart[256];  // first position of each digit in the staged tile
  __shared__ uint32_t gbase[256];   // where this tile's run of each digit goes
  __shared__ uint32_t wsum[kSortThreads / 32];
  __shared__ R stage[kSortTile];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  run[threadIdx.x] = 0;
  gbase[threadIdx.x] = offs[(size_t)threadIdx.x * ntiles + blockIdx.x];
  const size_t base = (size_t)blockIdx.x * kSortTile;
  const uint32_t lt_mask = (1u << lane) - 1u;
  R v[kSortItems];
  uint32_t dg[kSortItems], pos[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const size_t i = base + (size_t)r * kSortThreads + threadIdx.x;
    dg[r] = 256;
    if (i < n) {
      v[r] = in[i];
      dg[r] = (rec_key(v[r]) >> shift) & 255u;
    }
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) whist[w][threadIdx.x] = 0;
    __syncthreads();
    const uint32_t peers = __match_any_sync(0xffffffffu, dg[r]);
    const uint32_t rank = __popc(peers & lt_mask);
    if (dg[r] < 256 && lane == __ffs(peers) - 1) whist[warp][dg[r]] = __popc(peers);
    __syncthreads();
    {
      uint32_t acc = run[threadIdx.x];
#pragma unroll
      for (int w = 0; w < kSortThreads / 32; ++w) {
        const uint32_t c = whist[w][threadIdx.x];
        whist[w][threadIdx.x] = acc;
        acc += c;
      }
      run[threadIdx.x] = acc;
    }
    __syncthreads();
    pos[r] = dg[r] < 256 ? whist[warp][dg[r]] + rank : 0u;
    __syncthreads();
  }
  // dstart = exclusive prefix of the tile's digit counts
  {
    const uint32_t c = run[threadIdx.x];
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    dstart[threadIdx.x] = before + x - c;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r)
    if (dg[r] < 256) stage[dstart[dg[r]] + pos[r]] = v[r];
  __syncthreads();
  const size_t left = n - base;
  const int cnt = left < (size_t)kSortTile ? (int)left : kSortTile;
  for (int q = threadIdx.x; q < cnt; q += kSortThreads) {
    const R e = stage[q];
    const uint32_t d = (rec_key(e) >> shift) & 255u;
    out[gbase[d] + ((uint32_t)q - dstart[d])] = e;
  }
}

// ---------------- device-wide exclusive scan of uint32 (reduce, scan sums, scan chunks)
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh, uint32_t* total) {
  // kScanThreads threads; sh has kScanThreads / 32 entries
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  const uint32_t warp_off = warp == 0 ? 0u : sh[warp - 1];
  *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t* __restrict__ in, size_t n,
                                                                   uint32_t* __restrict__ sums) {
  __shared__ uint32_t sh[32];
  const size_t base = (size_t)blockIdx.x * kScanChunk;
  uint32_t v = 0;
  for (int k = 0; k < kScanChunk / kScanThreads; ++k) {
    const size_t i = base + (size_t)k * kScanThreads + threadIdx.x;
    if (i < n) v += in[i];
  }
  uint32_t total;
  block_exclusive_scan(v, sh, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint32_t* __restrict__ sums, int nchunks) {
  __shared__ uint32_t sh[32];
  uint32_t carry = 0;
  for (int base = 0; base < nchunks; base += kScanThreads) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < nchunks ? sums[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(v, sh, &total);
    if (i < nchunks) sums[i] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_chunks_kernel(const uint32_t* __restrict__ in, size_t n,
                                                                   const uint32_t* __restrict__ sums,
                                                                   uint32_t* __restrict__ out) {
  __shared__ uint32_t sh[32];
  const size_t base = (size_t)blockIdx.x * kScanChunk;
  uint32_t carry = sums[blockIdx.x];
  for (int k = 0; k < kScanChunk / kScanThreads; ++k) {
    const size_t i = base + (size_t)k * kScanThreads + threadIdx.x;
    const uint32_t v = i < n ? in[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(v, sh, &total);
    if (i < n) out[i] = carry + ex;
    carry += total;
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct SortScratch {
  uint32_t* hist;
  uint32_t* offs;
  uint32_t* sums;
  int ntiles;
  size_t nhist;
  int nchunks;
};

SortScratch carve(void* scratch, size_t n) {
  SortScratch s;
  s.ntiles = (int)((n + kSortTile - 1) / kSortTile);
  if (s.ntiles < 1) s.ntiles = 1;
  s.nhist = (size_t)256 * s.ntiles;
  s.nchunks = (int)((s.nhist + kScanChunk - 1) / kScanChunk);
  char* p = static_cast<char*>(scratch);
  s.hist = reinterpret_cast<uint32_t*>(p);
  p += align256(s.nhist * 4);
  s.offs = reinterpret_cast<uint32_t*>(p);
  p += align256(s.nhist * 4);
  s.sums = reinterpret_cast<uint32_t*>(p);
  return s;
}

template <class R>
R* radix_sort(R* in, R* out, size_t n, int bits, void* scratch, cudaStream_t st) {
  if (n == 0) return in;
  SortScratch s = carve(scratch, n);
  R* src = in;
  R* dst = out;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<R><<<s.ntiles, kSortThreads, 0, st>>>(src, n, shift, s.hist, s.ntiles);
    scan_reduce_kernel<<<s.nchunks, kScanThreads, 0, st>>>(s.hist, s.nhist, s.sums);
    scan_sums_kernel<<<1, kScanThreads, 0, st>>>(s.sums, s.nchunks);
    scan_chunks_kernel<<<s.nchunks, kScanThreads, 0, st>>>(s.hist, s.nhist, s.sums, s.offs);
    radix_scatter_kernel<R><<<s.ntiles, kSortThreads, 0, st>>>(src, dst, n, shift, s.offs, s.ntiles);
    R* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

// A float's value as a double, built from its bits on the integer pipes
// (the FP64 pipe is narrow on this GPU and the reduce is bound by it).
// Exact: every float is a double.  Zero, subnormal, infinite and NaN inputs
// take the hardware conversion.
DR_D double float_to_double_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                                  ((unsigned long long)(e + 896u) << 52) |  // exponent bias 1023 - 127
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// r += v in FP64, skipping v == 0: adding a zero leaves an FP64 sum that
// starts at +0 unchanged, so the result is the plain sequential sum's.
DR_D void add_nonzero(double& r, float v) {
  if (v != 0.0f) r += float_to_double_bits(v);
}

__global__ void segment_reduce_kernel(const SplatRec* __restrict__ s, size_t n, double* __restrict__ accum,
                                      uint32_t n_pix, uint32_t* err) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t pix = s[i].pix;
  if (i > 0 && s[i - 1].pix == pix) return;
  if (pix >= n_pix) {
    atomicOr(err, kErrBadIndex);
    return;
  }
  double r = 0.0, g = 0.0, b = 0.0;
  for (size_t k = i; k < n; ++k) {
    const SplatRec q = s[k];
    if (q.pix != pix) break;
    add_nonzero(r, q.r);
    add_nonzero(g, q.g);
    add_nonzero(b, q.b);
  }
  accum[(size_t)pix * 3 + 0] += r;
  accum[(size_t)pix * 3 + 1] += g;
  accum[(size_t)pix * 3 + 2] += b;
}

__global__ void resolve_kernel(const double* __restrict__ accum, size_t n,
                               const unsigned long long* __restrict__ tour_count, double k0, float* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long tc = *tour_count;
  out[i] = tc == 0ull ? 0.0f : (float)(k0 / (double)tc * accum[i]);
}

__global__ void resolve_count_kernel(const double* __restrict__ accum, size_t n, unsigned long long tc, double k0,
                                     float* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = tc == 0ull ? 0.0f : (float)(k0 / (double)tc * accum[i]);
}

}  // namespace

size_t sort_scratch_bytes(size_t n) {
  size_t ntiles = (n + kSortTile - 1) / kSortTile;
  if (ntiles < 1) ntiles = 1;
  const size_t nhist = 256 * ntiles;
  const size_t nchunks = (nhist + kScanChunk - 1) / kScanChunk;
  return 2 * align256(nhist * 4) + align256(nchunks * 4);
}

size_t scan_scratch_bytes(size_t n) { return align256(((n + kScanChunk - 1) / kScanChunk + 1) * 4); }

void launch_exclusive_scan(const uint32_t* in, uint32_t* out, size_t n, void* scratch, cudaStream_t s) {
  if (n == 0) return;
  const int nchunks = (int)((n + kScanChunk - 1) / kScanChunk);
  uint32_t* sums = static_cast<uint32_t*>(scratch);
  scan_reduce_kernel<<<nchunks, kScanThreads, 0, s>>>(in, n, sums);
  scan_sums_kernel<<<1, kScanThreads, 0, s>>>(sums, nchunks);
  scan_chunks_kernel<<<nchunks, kScanThreads, 0, s>>>(in, n, sums, out);
}

SplatRec* sort_splat_records(SplatRec* in, SplatRec* out, size_t n, int bits, void* scratch, cudaStream_t s) {
  return radix_sort<SplatRec>(in, out, n, bits, scratch, s);
}

uint2* sort_pairs(uint2* in, uint2* out, size_t n, int bits, void* scratch, cudaStream_t s) {
  return radix_sort<uint2>(in, out, n, bits, scratch, s);
}

void launch_segment_reduce(const SplatRec* sorted, size_t n, double* accum, uint32_t n_pix, uint32_t* err,
                           cudaStream_t s) {
  if (n == 0) return;
  segment_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sorted, n, accum, n_pix, err);
}

void launch_resolve(const double* accum, size_t n, const unsigned long long* tour_count, double k0, float* out,
                    cudaStream_t s) {
  if (n == 0) return;
  resolve_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(accum, n, tour_count, k0, out);
}

void launch_resolve_count(const double* accum, size_t n, unsigned long long tour_count, double k0, float* out,
                          cudaStream_t s) {
  if (n == 0) return;
  resolve_count_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(accum, n, tour_count, k0, out);
}

}  // namespace dr
