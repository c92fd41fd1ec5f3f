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

// Lanes of the warp whose digit equals this lane's, from one ballot per bit
// (bits = digit width + 1: the extra bit marks out-of-range items).
__device__ __forceinline__ unsigned digit_peers(uint32_t d, int bits) {
  unsigned peers = kFull;
  for (int b = 0; b < bits; ++b) {
    const bool set = (d >> b) & 1u;
    const unsigned bal = __ballot_sync(kFull, set);
    peers &= set ? bal : ~bal;
  }
  return peers;
}

__global__ void __launch_bounds__(kBlock) radix_upsweep_kernel(const uint32_t* __restrict__ keys,
                                                               uint32_t n, int shift, uint32_t mask,
                                                               uint32_t* __restrict__ counts,
                                                               uint32_t n_blocks) {
  constexpr int NW = kBlock / 32;
  __shared__ uint32_t whist[NW][kMaxRadix + 1];
  const int R = (int)mask + 1;
  const int bits = __popc(mask) + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = lane; i <= R; i += 32) whist[warp][i] = 0;
  __syncwarp();
  const uint32_t wbase = blockIdx.x * kChunk + warp * 32 * kItems;
  uint32_t key[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t k = wbase + j * 32 + lane;
    key[j] = k < n ? keys[k] : 0u;
  }
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t k = wbase + j * 32 + lane;
    const uint32_t d = k < n ? ((key[j] >> shift) & mask) : (uint32_t)R;
    const unsigned peers = digit_peers(d, bits);
    if (lane == __ffs(peers) - 1) whist[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < R; i += kBlock) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) t += whist[w][i];
    counts[(size_t)i * n_blocks + blockIdx.x] = t;
  }
}

// Stable scatter of one pass.  Warp w of the block owns the contiguous slice
// [w*32*kItems, (w+1)*32*kItems) of the block's chunk and ranks its items in
// their original order (round j covers the slice's items j*32 .. j*32+31)
// with a running per-warp count of every digit.  The block then orders its
// whole chunk by digit in shared memory and writes it out in digit runs, so
// the global stores are coalesced.
__global__ void __launch_bounds__(kBlock) radix_scatter_kernel(const uint32_t* __restrict__ keys_in,
                                                               const uint32_t* __restrict__ vals_in,
                                                               uint32_t* __restrict__ keys_out,
                                                               uint32_t* __restrict__ vals_out,
                                                               uint32_t n, int shift, uint32_t mask,
                                                               const uint32_t* __restrict__ offsets,
                                                               uint32_t n_blocks) {
  constexpr int NW = kBlock / 32;
  __shared__ uint32_t whist[NW][kMaxRadix + 1];
  __shared__ uint32_t dstart[kMaxRadix];
  __shared__ uint32_t gbase[kMaxRadix];
  __shared__ uint32_t wsum[NW];
  __shared__ uint32_t sk[kChunk];
  __shared__ uint32_t sv[kChunk];
  const int R = (int)mask + 1;
  const int bits = __popc(mask) + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = lane; i <= R; i += 32) whist[warp][i] = 0;
  for (int i = threadIdx.x; i < R; i += kBlock) gbase[i] = offsets[(size_t)i * n_blocks + blockIdx.x];
  __syncwarp();
  const uint32_t wbase = blockIdx.x * kChunk + warp * 32 * kItems;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t key[kItems], val[kItems], rank[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t k = wbase + j * 32 + lane;
    const bool valid = k < n;
    key[j] = valid ? keys_in[k] : 0u;
    val[j] = valid ? vals_in[k] : 0u;
  }
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t k = wbase + j * 32 + lane;
    const uint32_t d = k < n ? ((key[j] >> shift) & mask) : (uint32_t)R;
    const unsigned peers = digit_peers(d, bits);
    const int leader = __ffs(peers) - 1;
    uint32_t before = 0;
    if (lane == leader) before = whist[warp][d];
    before = __shfl_sync(peers, before, leader);
    rank[j] = before + __popc(peers & lt);
    if (lane == leader) whist[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: offsets of the warps inside the digit, and the digit's total
  uint32_t tot = 0;
  if (threadIdx.x < R) {
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = whist[w][threadIdx.x];
      whist[w][threadIdx.x] = tot;
      tot += c;
    }
  }
  // exclusive scan of the digit totals across the block (digit = thread index)
  uint32_t inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t carry = 0;
  for (int w = 0; w < warp; ++w) carry += wsum[w];
  if (threadIdx.x < R) dstart[threadIdx.x] = carry + inc - tot;
  __syncthreads();
  const uint32_t n_here = (n - blockIdx.x * kChunk < (uint32_t)kChunk) ? n - blockIdx.x * kChunk : (uint32_t)kChunk;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t k = wbase + j * 32 + lane;
    if (k < n) {
      const uint32_t d = (key[j] >> shift) & mask;
      const uint32_t lp = dstart[d] + whist[warp][d] + rank[j];
      sk[lp] = key[j];
      sv[lp] = val[j];
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n_here; i += kBlock) {
    const uint32_t kk = sk[i];
    const uint32_t d = (kk >> shift) & mask;
    const uint32_t pos = gbase[d] + (i - dstart[d]);
    keys_out[pos] = kk;
    vals_out[pos] = sv[i];
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

// Pixel-centre rectangle of tile (tx, ty) of a view, clipped to the image.
__device__ __forceinline__ void tile_rect(const DevCam& cam, int tw, int th, int tx, int ty, float* x0, float* x1,
                                          float* y0, float* y1) {
  *x0 = (float)(tx * tw) + 0.5f;
  *x1 = (float)(min((tx + 1) * tw, cam.W) - 1) + 0.5f;
  *y0 = (float)(ty * th) + 0.5f;
  *y1 = (float)(min((ty + 1) * th, cam.H) - 1) + 0.5f;
}

constexpr int kWarpsPerBlock = 8;
constexpr int kSmallRect = 32;  // records with at most this many candidate tiles keep a bit mask

// The (record, candidate tile) items of the 32 records of a warp are walked as
// one flat list, 32 items per step, so that a record with many candidate
// tiles does not leave the other lanes idle.  Items of one record occupy
// consecutive lanes of a step (a "segment"); the first lane of each segment
// accounts for the whole segment, so no two lanes update the same record.
struct WarpItems {
  int incl[32];  // inclusive prefix of the candidate counts
  int4 rc[32];
  int view[32];
};

__device__ __forceinline__ int item_record(const int* incl, int q) {
  int lo = 0, hi = 31;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (incl[mid] > q) hi = mid; else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ unsigned lanes_le(int lane) { return lane == 31 ? kFull : ((2u << lane) - 1u); }

__global__ void __launch_bounds__(32 * kWarpsPerBlock) tile_count_kernel(
    const RecPtrs rec, const int4* __restrict__ rect, const DevCam* __restrict__ cams, int64_t n_gauss,
    uint32_t n_rec, int tw, int th, int32_t* __restrict__ ntiles, uint32_t* __restrict__ tmask,
    uint32_t* __restrict__ depth_key) {
  __shared__ WarpItems s_it[kWarpsPerBlock];
  __shared__ SupportConic s_k[kWarpsPerBlock][32];
  __shared__ int s_cnt[kWarpsPerBlock][32];
  __shared__ uint32_t s_bits[kWarpsPerBlock][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t r = (blockIdx.x * kWarpsPerBlock + warp) * 32u + lane;
  int4 rc = make_int4(0, 0, -1, -1);
  if (r < n_rec) rc = rect[r];
  const int n = (rc.z < rc.x) ? 0 : (rc.z - rc.x + 1) * (rc.w - rc.y + 1);
  if (n > 0) {
    const float4 g0 = rec.g0[r];
    s_k[warp][lane] = support_conic(g0, rec.g1[r], rec.g2[r], support_rho(g0.z));
  }
  WarpItems& it = s_it[warp];
  it.rc[lane] = rc;
  it.view[lane] = (int)(r / (uint64_t)n_gauss);
  s_cnt[warp][lane] = 0;
  s_bits[warp][lane] = 0u;
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  it.incl[lane] = incl;
  const int total = __shfl_sync(kFull, incl, 31);
  __syncwarp();
  for (int q0 = 0; q0 < total; q0 += 32) {
    const int q = q0 + lane;
    const bool valid = q < total;
    int ri = 0, t = 0;
    bool hit = false;
    if (valid) {
      ri = item_record(it.incl, q);
      const int4 c = it.rc[ri];
      const int w = c.z - c.x + 1;
      t = q - (it.incl[ri] - w * (c.w - c.y + 1));
      const DevCam& cam = cams[it.view[ri]];
      float x0, x1, y0, y1;
      tile_rect(cam, tw, th, c.x + t % w, c.y + t / w, &x0, &x1, &y0, &y1);
      hit = conic_touches(s_k[warp][ri], x0, x1, y0, y1);
    }
    const bool head = valid && (t == 0 || lane == 0);
    const unsigned heads = __ballot_sync(kFull, head);
    const unsigned hitm = __ballot_sync(kFull, hit);
    if (head) {
      const unsigned later = heads & ~lanes_le(lane);
      const int end = later ? __ffs(later) - 1 : 32;
      const unsigned seg = (end == 32 ? kFull : ((1u << end) - 1u)) & ~((1u << lane) - 1u);
      const unsigned sh = hitm & seg;
      s_cnt[warp][ri] += __popc(sh);
      const int4 c = it.rc[ri];
      if ((c.z - c.x + 1) * (c.w - c.y + 1) <= kSmallRect) s_bits[warp][ri] |= (sh >> lane) << t;
    }
    __syncwarp();
  }
  if (r < n_rec) {
    const int cnt = s_cnt[warp][lane];
    ntiles[r] = cnt;
    tmask[r] = s_bits[warp][lane];
    if (cnt == 0) depth_key[r] = 0xffffffffu;
  }
}

// roff[order[i]] = offsets[i]: each record's first pair slot, in record order.
__global__ void scatter_offsets_kernel(const uint32_t* __restrict__ order, const uint64_t* __restrict__ offsets,
                                       uint32_t n, uint64_t* __restrict__ roff) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) roff[order[i]] = offsets[i];
}

// Same flat walk as the count, in record order: a small record takes its hits
// from the count-pass mask, a large one repeats the test.  The k-th kept tile
// of a record goes to roff[record] + k (kept tiles in rectangle order).
__global__ void __launch_bounds__(32 * kWarpsPerBlock) duplicate_kernel(
    const uint64_t* __restrict__ roff, const int32_t* __restrict__ ntiles, uint32_t n_rec,
    const int4* __restrict__ rect, const uint32_t* __restrict__ tmask, const RecPtrs rec,
    const DevCam* __restrict__ cams, int64_t n_gauss, int tw, int th, uint32_t n_pairs, uint32_t* __restrict__ keys,
    uint32_t* __restrict__ vals) {
  __shared__ WarpItems s_it[kWarpsPerBlock];
  __shared__ SupportConic s_k[kWarpsPerBlock][32];
  __shared__ uint64_t s_o[kWarpsPerBlock][32];
  __shared__ uint32_t s_bits[kWarpsPerBlock][32];
  __shared__ uint32_t s_run[kWarpsPerBlock][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t r = (blockIdx.x * kWarpsPerBlock + warp) * 32u + lane;
  int4 rc = make_int4(0, 0, -1, -1);
  int n = 0;
  if (r < n_rec && ntiles[r] > 0) {
    rc = rect[r];
    n = (rc.z - rc.x + 1) * (rc.w - rc.y + 1);
    s_o[warp][lane] = roff[r];
    if (n <= kSmallRect) {
      s_bits[warp][lane] = tmask[r];
    } else {
      const float4 g0 = rec.g0[r];
      s_k[warp][lane] = support_conic(g0, rec.g1[r], rec.g2[r], support_rho(g0.z));
    }
  }
  WarpItems& it = s_it[warp];
  it.rc[lane] = rc;
  it.view[lane] = (int)(r / (uint64_t)n_gauss);
  s_run[warp][lane] = 0u;
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  it.incl[lane] = incl;
  const int total = __shfl_sync(kFull, incl, 31);
  const uint32_t rbase = r - lane;
  __syncwarp();
  for (int q0 = 0; q0 < total; q0 += 32) {
    const int q = q0 + lane;
    const bool valid = q < total;
    int ri = 0, t = 0, tx = 0, ty = 0;
    bool hit = false;
    const DevCam* cam = cams;
    if (valid) {
      ri = item_record(it.incl, q);
      const int4 c = it.rc[ri];
      const int w = c.z - c.x + 1;
      const int nr = w * (c.w - c.y + 1);
      t = q - (it.incl[ri] - nr);
      tx = c.x + t % w;
      ty = c.y + t / w;
      cam = &cams[it.view[ri]];
      if (nr <= kSmallRect) {
        hit = (s_bits[warp][ri] >> t) & 1u;
      } else {
        float x0, x1, y0, y1;
        tile_rect(*cam, tw, th, tx, ty, &x0, &x1, &y0, &y1);
        hit = conic_touches(s_k[warp][ri], x0, x1, y0, y1);
      }
    }
    const bool head = valid && (t == 0 || lane == 0);
    const unsigned heads = __ballot_sync(kFull, head);
    const unsigned hitm = __ballot_sync(kFull, hit);
    const int h = 31 - __clz(heads & lanes_le(lane));  // first lane of this lane's segment
    if (hit) {
      const uint64_t pos = s_o[warp][ri] + s_run[warp][ri] + __popc(hitm & lt & ~((1u << h) - 1u));
      if (pos < n_pairs) {
        keys[pos] = (uint32_t)(cam->tile_offset + ty * cam->tiles_x + tx);
        vals[pos] = rbase + (uint32_t)ri;
      }
    }
    __syncwarp();
    if (head) {
      const unsigned later = heads & ~lanes_le(lane);
      const int end = later ? __ffs(later) - 1 : 32;
      const unsigned seg = (end == 32 ? kFull : ((1u << end) - 1u)) & ~((1u << lane) - 1u);
      s_run[warp][ri] += __popc(hitm & seg);
    }
    __syncwarp();
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

cudaError_t launch_tile_count(const RecPtrs rec, const int4* rect, const DevCam* cams, int64_t n_gauss,
                              uint32_t n_rec, int tile_w, int tile_h, int32_t* ntiles, uint32_t* tmask,
                              uint32_t* depth_key, cudaStream_t s) {
  if (n_rec == 0) return cudaSuccess;
  const uint32_t per_block = 32u * kWarpsPerBlock;
  tile_count_kernel<<<(n_rec + per_block - 1) / per_block, 32 * kWarpsPerBlock, 0, s>>>(
      rec, rect, cams, n_gauss, n_rec, tile_w, tile_h, ntiles, tmask, depth_key);
  return launched();
}

cudaError_t launch_duplicate(const uint32_t* order, const uint64_t* offsets, uint64_t* roff, uint32_t n_rec,
                             const int32_t* ntiles, const int4* rect, const uint32_t* tmask, const RecPtrs rec,
                             const DevCam* cams, int64_t n_gauss, int tile_w, int tile_h, uint32_t n_pairs,
                             uint32_t* keys, uint32_t* vals, cudaStream_t s) {
  if (n_pairs == 0 || n_rec == 0) return cudaSuccess;
  scatter_offsets_kernel<<<(n_rec + 255) / 256, 256, 0, s>>>(order, offsets, n_rec, roff);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  const uint32_t per_block = 32u * kWarpsPerBlock;
  duplicate_kernel<<<(n_rec + per_block - 1) / per_block, 32 * kWarpsPerBlock, 0, s>>>(
      roff, ntiles, n_rec, rect, tmask, rec, cams, n_gauss, tile_w, tile_h, n_pairs, keys, vals);
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
