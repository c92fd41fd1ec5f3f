// Tile binning: device-wide scans, the stable LSD radix sort of 32-bit keys,
// duplication of each visible (view, Gaussian) record into its tiles and the
// per-tile [start, end) ranges.
//
// Order of the (tile, Gaussian) list (the front-to-back order of Sec. 4.3):
// records are first sorted by centre depth (stable, so equal depths keep the
// ascending (view, Gaussian) index), duplicated in that order, and then
// stably sorted by global tile id.  Within a tile the list is therefore in
// ascending (depth, Gaussian index) order, and only ceil(log2 tiles) key bits
// are sorted per pair instead of tile+depth bits.
#include "common.cuh"

namespace ocgs {
namespace {

constexpr int kBlock = 256;
constexpr int kItems = 16;
constexpr int kChunk = kBlock * kItems;  // items per block in scans and sort passes
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// ------------------------------------------------------------------ scan
template <typename T>
__global__ void __launch_bounds__(kBlock) scan_reduce_kernel(const T* __restrict__ in, uint32_t n,
                                                             T* __restrict__ block_sums) {
  __shared__ T warp_sums[kBlock / 32];
  const uint32_t base = blockIdx.x * kChunk;
  T s = 0;
#pragma unroll 4
  for (int j = 0; j < kItems; ++j) {
    const uint32_t k = base + j * kBlock + threadIdx.x;
    if (k < n) s += in[k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_sums[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = 0;
    for (int w = 0; w < kBlock / 32; ++w) t += warp_sums[w];
    block_sums[blockIdx.x] = t;
  }
}

// exclusive scan of one chunk per block, each warp owning a contiguous 32*kItems slice
template <typename T>
__global__ void __launch_bounds__(kBlock) scan_chunk_kernel(const T* in, T* out, uint32_t n,
                                                            const T* __restrict__ block_offsets,
                                                            T* __restrict__ d_total) {
  __shared__ T warp_tot[kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wbase = blockIdx.x * kChunk + warp * 32 * kItems;
  T vals[kItems];
  T run = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t k = wbase + j * 32 + lane;
    const T x = k < n ? in[k] : T(0);
    const T inc = warp_inclusive_scan<T>(x, lane);
    vals[j] = run + inc - x;  // exclusive within the warp slice
    run += __shfl_sync(kFull, inc, 31);
  }
  if (lane == 0) warp_tot[warp] = run;
  __syncthreads();
  T off = block_offsets ? block_offsets[blockIdx.x] : T(0);
  T tot = 0;
  for (int w = 0; w < kBlock / 32; ++w) {
    if (w < warp) off += warp_tot[w];
    tot += warp_tot[w];
  }
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t k = wbase + j * 32 + lane;
    if (k < n) out[k] = off + vals[j];
  }
  if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    const T first = block_offsets ? block_offsets[blockIdx.x] : T(0);
    *d_total = first + tot;
  }
}

template <typename T>
size_t scan_levels_bytes(uint32_t n) {
  size_t bytes = 0;
  while (n > (uint32_t)kChunk) {
    n = (n + kChunk - 1) / kChunk;
    bytes += ((size_t)n * sizeof(T) + 255) & ~(size_t)255;
  }
  return bytes;
}

template <typename T>
cudaError_t scan_exclusive(const T* in, T* out, uint32_t n, T* d_total, char* scratch, cudaStream_t s) {
  if (n == 0) {
    if (d_total) return cudaMemsetAsync(d_total, 0, sizeof(T), s);
    return cudaSuccess;
  }
  const uint32_t nb = (n + kChunk - 1) / kChunk;
  if (nb == 1) {
    scan_chunk_kernel<T><<<1, kBlock, 0, s>>>(in, out, n, nullptr, d_total);
    return launched();
  }
  T* sums = reinterpret_cast<T*>(scratch);
  char* rest = scratch + (((size_t)nb * sizeof(T) + 255) & ~(size_t)255);
  scan_reduce_kernel<T><<<nb, kBlock, 0, s>>>(in, n, sums);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  e = scan_exclusive<T>(sums, sums, nb, nullptr, rest, s);  // in place over the block sums
  if (e != cudaSuccess) return e;
  scan_chunk_kernel<T><<<nb, kBlock, 0, s>>>(in, out, n, sums, d_total);
  return launched();
}

// ------------------------------------------------------------------ radix sort
constexpr int kMaxRadix = 256;

__global__ void __launch_bounds__(kBlock) radix_upsweep_kernel(const uint32_t* __restrict__ keys,
                                                               uint32_t n, int shift, uint32_t mask,
                                                               uint32_t* __restrict__ counts,
                                                               uint32_t n_blocks) {
  __shared__ uint32_t hist[kMaxRadix + 1];
  const int R = (int)mask + 1;
  for (int i = threadIdx.x; i <= R; i += kBlock) hist[i] = 0;
  __syncthreads();
  const uint32_t base = blockIdx.x * kChunk;
  const int lane = threadIdx.x & 31;
#pragma unroll 4
  for (int j = 0; j < kItems; ++j) {
    const uint32_t k = base + j * kBlock + threadIdx.x;
    const uint32_t d = k < n ? ((keys[k] >> shift) & mask) : (uint32_t)R;
    const unsigned peers = __match_any_sync(kFull, d);
    if (lane == __ffs(peers) - 1) atomicAdd(&hist[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < R; i += kBlock) counts[(size_t)i * n_blocks + blockIdx.x] = hist[i];
}

// stable scatter: items of a block are ranked in their original order (round j
// covers items j*kBlock .. j*kBlock+kBlock-1, warps in order, lanes in order)
__global__ void __launch_bounds__(kBlock) radix_scatter_kernel(const uint32_t* __restrict__ keys_in,
                                                               const uint32_t* __restrict__ vals_in,
                                                               uint32_t* __restrict__ keys_out,
                                                               uint32_t* __restrict__ vals_out,
                                                               uint32_t n, int shift, uint32_t mask,
                                                               const uint32_t* __restrict__ offsets,
                                                               uint32_t n_blocks) {
  constexpr int NW = kBlock / 32;
  __shared__ uint32_t base[kMaxRadix];
  __shared__ uint32_t whist[NW][kMaxRadix + 1];
  const int R = (int)mask + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < R; i += kBlock) base[i] = offsets[(size_t)i * n_blocks + blockIdx.x];
  const uint32_t blk = blockIdx.x * kChunk;
  const unsigned lt = (1u << lane) - 1u;
  for (int j = 0; j < kItems; ++j) {
    const uint32_t k = blk + j * kBlock + threadIdx.x;
    const bool valid = k < n;
    const uint32_t key = valid ? keys_in[k] : 0u;
    const uint32_t val = valid ? vals_in[k] : 0u;
    const uint32_t d = valid ? ((key >> shift) & mask) : (uint32_t)R;
    for (int i = lane; i <= R; i += 32) whist[warp][i] = 0;
    __syncwarp();
    const unsigned peers = __match_any_sync(kFull, d);
    const uint32_t rank = __popc(peers & lt);
    if (rank == 0) whist[warp][d] = __popc(peers);
    __syncthreads();
    uint32_t run = 0;
    if (threadIdx.x < R) {
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = whist[w][threadIdx.x];
        whist[w][threadIdx.x] = run;
        run += c;
      }
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = base[d] + whist[warp][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
    __syncthreads();
    if (threadIdx.x < R) base[threadIdx.x] += run;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ binning helpers
__global__ void gather_counts_kernel(const uint32_t* __restrict__ order, const int32_t* __restrict__ ntiles,
                                     uint64_t* __restrict__ counts, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) counts[i] = (uint64_t)ntiles[order[i]];
}

__global__ void iota_kernel(uint32_t* v, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i;
}

// last item whose exclusive offset is <= k (items with a zero count only occur at the tail)
__device__ __forceinline__ uint32_t find_item(const uint64_t* off, uint32_t n, uint64_t k) {
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo + 1) >> 1);
    if (off[mid] <= k) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int kDupPerBlock = kChunk;  // outputs per block

__global__ void __launch_bounds__(kBlock) duplicate_kernel(const uint32_t* __restrict__ order,
                                                           const uint64_t* __restrict__ offsets,
                                                           uint32_t n_items, const int4* __restrict__ rect,
                                                           const DevCam* __restrict__ cams, int64_t n_gauss,
                                                           uint32_t n_pairs, uint32_t* __restrict__ keys,
                                                           uint32_t* __restrict__ vals, int* __restrict__ status) {
  __shared__ uint64_t s_off[kDupPerBlock + 1];
  __shared__ uint32_t s_range[2];
  const uint64_t k0 = (uint64_t)blockIdx.x * kDupPerBlock;
  const uint64_t k1 = (k0 + kDupPerBlock < (uint64_t)n_pairs) ? k0 + kDupPerBlock : (uint64_t)n_pairs;
  if (threadIdx.x == 0) {
    s_range[0] = find_item(offsets, n_items, k0);
    s_range[1] = find_item(offsets, n_items, k1 - 1);
  }
  __syncthreads();
  const uint32_t i0 = s_range[0], i1 = s_range[1];
  // every item in range has >= 1 pair (zero-count records sort to the tail), so m <= kDupPerBlock
  const uint32_t m = i1 - i0 + 1;
  if (m > (uint32_t)kDupPerBlock) {
    if (threadIdx.x == 0) atomicOr(status, kStatusCapacity);
    return;
  }
  for (uint32_t t = threadIdx.x; t < m; t += kBlock) s_off[t] = offsets[i0 + t];
  __syncthreads();
  for (uint64_t k = k0 + threadIdx.x; k < k1; k += kBlock) {
    uint32_t lo = 0, hi = m - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= k) lo = mid; else hi = mid - 1;
    }
    const uint32_t rec_idx = order[i0 + lo];
    const uint32_t local = (uint32_t)(k - s_off[lo]);
    const int4 rc = rect[rec_idx];
    const int view = (int)(rec_idx / (uint64_t)n_gauss);
    const int w = rc.z - rc.x + 1;
    const int tx = rc.x + (int)(local % (uint32_t)w);
    const int ty = rc.y + (int)(local / (uint32_t)w);
    const DevCam& cam = cams[view];
    keys[k] = (uint32_t)(cam.tile_offset + ty * cam.tiles_x + tx);
    vals[k] = rec_idx;
  }
}

__global__ void tile_ranges_kernel(const uint32_t* __restrict__ keys, uint32_t n, uint2* __restrict__ ranges) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t t = keys[k];
  if (k == 0 || keys[k - 1] != t) ranges[t].x = k;
  if (k == n - 1 || keys[k + 1] != t) ranges[t].y = k + 1;
}

// work key for the persistent queue: heaviest tiles first (descending pair count)
__global__ void tile_work_kernel(const uint2* __restrict__ ranges, uint32_t n, uint32_t* __restrict__ work_key,
                                 uint32_t* __restrict__ ids) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint2 r = ranges[t];
  work_key[t] = 0xffffffffu - (r.y - r.x);
  ids[t] = t;
}

}  // namespace

size_t scan_scratch_bytes(uint32_t n) { return scan_levels_bytes<uint64_t>(n) + 256; }

cudaError_t scan_exclusive_u64(const uint64_t* in, uint64_t* out, uint32_t n, uint64_t* d_total,
                               void* scratch, cudaStream_t s) {
  return scan_exclusive<uint64_t>(in, out, n, d_total, static_cast<char*>(scratch), s);
}

cudaError_t scan_exclusive_u32(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* d_total,
                               void* scratch, cudaStream_t s) {
  return scan_exclusive<uint32_t>(in, out, n, d_total, static_cast<char*>(scratch), s);
}

size_t radix_scratch_bytes(uint32_t n) {
  const uint32_t nb = (n + kChunk - 1) / kChunk;
  const size_t counts = (size_t)kMaxRadix * nb;
  const size_t cbytes = (counts * sizeof(uint32_t) + 255) & ~(size_t)255;
  return cbytes + scan_levels_bytes<uint32_t>((uint32_t)counts) + 256;
}

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                             uint32_t n, int n_bits, void* scratch, bool* result_in_alt, cudaStream_t s) {
  *result_in_alt = false;
  if (n <= 1 || n_bits <= 0) return cudaSuccess;
  const uint32_t nb = (n + kChunk - 1) / kChunk;
  const int passes = (n_bits + 7) / 8;
  const int digit = (n_bits + passes - 1) / passes;  // balanced digit width <= 8
  uint32_t* counts = static_cast<uint32_t*>(scratch);
  const size_t cbytes = ((size_t)kMaxRadix * nb * sizeof(uint32_t) + 255) & ~(size_t)255;
  char* scan_scratch = static_cast<char*>(scratch) + cbytes;
  uint32_t *kin = keys, *vin = vals, *kout = keys_alt, *vout = vals_alt;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * digit;
    const int width = min(digit, n_bits - shift);
    const uint32_t mask = (1u << width) - 1u;
    radix_upsweep_kernel<<<nb, kBlock, 0, s>>>(kin, n, shift, mask, counts, nb);
    cudaError_t e = launched();
    if (e != cudaSuccess) return e;
    e = scan_exclusive<uint32_t>(counts, counts, (mask + 1) * nb, nullptr, scan_scratch, s);
    if (e != cudaSuccess) return e;
    radix_scatter_kernel<<<nb, kBlock, 0, s>>>(kin, vin, kout, vout, n, shift, mask, counts, nb);
    e = launched();
    if (e != cudaSuccess) return e;
    uint32_t* t = kin; kin = kout; kout = t;
    t = vin; vin = vout; vout = t;
    *result_in_alt = !*result_in_alt;
  }
  return cudaSuccess;
}

cudaError_t launch_gather_counts(const uint32_t* order, const int32_t* ntiles, uint64_t* counts,
                                 uint32_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  gather_counts_kernel<<<(n + 255) / 256, 256, 0, s>>>(order, ntiles, counts, n);
  return launched();
}

cudaError_t launch_iota(uint32_t* v, uint32_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  iota_kernel<<<(n + 255) / 256, 256, 0, s>>>(v, n);
  return launched();
}

cudaError_t launch_duplicate(const uint32_t* order, const uint64_t* offsets, uint32_t n_items,
                             const int4* rect, const DevCam* cams, int64_t n_gauss, uint32_t n_pairs,
                             uint32_t* keys, uint32_t* vals, int* status, cudaStream_t s) {
  if (n_pairs == 0) return cudaSuccess;
  const uint32_t nb = (n_pairs + kDupPerBlock - 1) / kDupPerBlock;
  duplicate_kernel<<<nb, kBlock, 0, s>>>(order, offsets, n_items, rect, cams, n_gauss, n_pairs, keys, vals, status);
  return launched();
}

cudaError_t launch_tile_ranges(const uint32_t* keys, uint32_t n_pairs, uint2* ranges, cudaStream_t s) {
  if (n_pairs == 0) return cudaSuccess;
  tile_ranges_kernel<<<(n_pairs + 255) / 256, 256, 0, s>>>(keys, n_pairs, ranges);
  return launched();
}

cudaError_t launch_tile_order(const uint2* ranges, uint32_t n_tiles, uint32_t* work_key,
                              uint32_t* tile_ids, cudaStream_t s) {
  if (n_tiles == 0) return cudaSuccess;
  tile_work_kernel<<<(n_tiles + 255) / 256, 256, 0, s>>>(ranges, n_tiles, work_key, tile_ids);
  return launched();
}

}  // namespace ocgs
