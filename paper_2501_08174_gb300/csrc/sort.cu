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
                                                               uint32_t n_blocks, const uint32_t* __restrict__ d_n) {
  constexpr int NW = kBlock / 32;
  __shared__ uint32_t whist[NW][kMaxRadix + 1];
  if (d_n) n = min(n, *d_n);  // device-side count (capacity launches)
  const int R = (int)mask + 1;
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
    if (k < n) atomicAdd(&whist[warp][(key[j] >> shift) & mask], 1u);
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
// vals_in NULL: the values are the items' indices
__global__ void __launch_bounds__(kBlock) radix_scatter_kernel(const uint32_t* __restrict__ keys_in,
                                                               const uint32_t* __restrict__ vals_in,
                                                               uint32_t* __restrict__ keys_out,
                                                               uint32_t* __restrict__ vals_out,
                                                               uint32_t n, int shift, uint32_t mask,
                                                               const uint32_t* __restrict__ offsets,
                                                               uint32_t n_blocks, const uint32_t* __restrict__ d_n) {
  constexpr int NW = kBlock / 32;
  if (d_n) n = min(n, *d_n);  // device-side count (capacity launches)
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
    val[j] = valid ? (vals_in ? vals_in[k] : k) : 0u;  // no values: the item's index
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
  const uint32_t n_here = (blockIdx.x * kChunk >= n) ? 0u
                          : ((n - blockIdx.x * kChunk < (uint32_t)kChunk) ? n - blockIdx.x * kChunk : (uint32_t)kChunk);
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

constexpr int kThreads = 256;
// a record with at most this many candidate rows is a small one: its row runs are
// kept in shared memory and its tiles written in the warp-flat list
constexpr int kSmallRows = 16;

__device__ __forceinline__ int row_count(const RowRuns& rr) {
  return max(0, rr.a1 - rr.a0 + 1) + max(0, rr.b1 - rr.b0 + 1);
}

// What a lane knows of its record for the rows of that record that other lanes
// of its warp evaluate: the support conic, the candidate tile rectangle and the view.
struct RowOwner {
  SupportConic k;
  int4 rc;
  int tile_offset, tiles_x, W, H;
};

// The candidate tile rows of the warp's 32 records, flattened over the lanes:
// f(ri, ty) runs once for every row ty of record ri, 32 rows at a time, so
// records with many rows no longer leave the lanes of small ones idle.
// nrows: the rows of this lane's record (0 for none); s_own[lane] must hold it.
template <class F>
__device__ __forceinline__ void for_warp_rows(int nrows, int lane, int* s_incl, const RowOwner* s_own, F f) {
  const int incl = warp_inclusive_scan<int>(nrows, lane);
  s_incl[lane] = incl;
  const int total = __shfl_sync(kFull, incl, 31);
  __syncwarp();
  for (int q0 = 0; q0 < total; q0 += 32) {
    const int q = q0 + lane;
    if (q < total) {
      int lo = 0, hi = 31;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_incl[mid] > q) hi = mid; else lo = mid + 1;
      }
      const int excl = lo > 0 ? s_incl[lo - 1] : 0;
      f(lo, s_own[lo].rc.y + (q - excl));
    }
  }
  __syncwarp();
}

// Exact tile count of each record: one closed-form coverage computation per
// candidate tile row, the rows of a warp's 32 records spread over its lanes.
__global__ void __launch_bounds__(kThreads) tile_count_kernel(const float4* __restrict__ bin,
                                                              const DevCam* __restrict__ cams, int64_t n_gauss,
                                                              uint32_t n_rec, int tw, int th,
                                                              int32_t* __restrict__ ntiles,
                                                              uint32_t* __restrict__ depth_key) {
  __shared__ RowOwner s_own[kThreads / 32][32];
  __shared__ int s_incl[kThreads / 32][32], s_cnt[kThreads / 32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t r = blockIdx.x * kThreads + threadIdx.x;
  int nrows = 0;
  if (r < n_rec) {
    const BinView b = load_bin(bin, r);
    if (b.rc.z >= b.rc.x) {
      const DevCam& cam = cams[view_of_record(r, n_gauss)];
      s_own[warp][lane] = RowOwner{support_conic(b.g0, b.g1, b.g2, b.rb), b.rc, cam.tile_offset, cam.tiles_x,
                                   cam.W, cam.H};
      nrows = b.rc.w - b.rc.y + 1;
    }
  }
  s_cnt[warp][lane] = 0;
  // the rows of the warp's records, spread over the lanes
  for_warp_rows(nrows, lane, s_incl[warp], s_own[warp], [&](int ri, int ty) {
    const RowOwner& o = s_own[warp][ri];
    const int c = row_count(row_runs(o.k, ty, tw, th, o.W, o.H, o.rc));
    if (c) atomicAdd(&s_cnt[warp][ri], c);
  });
  if (r < n_rec) {
    const int cnt = s_cnt[warp][lane];
    ntiles[r] = cnt;
    if (cnt == 0) depth_key[r] = 0xffffffffu;
  }
}

__device__ __forceinline__ uint64_t write_runs(const RowRuns& rr, uint32_t rowbase, uint32_t r, uint64_t pos,
                                               uint64_t stop, uint32_t* __restrict__ keys,
                                               uint32_t* __restrict__ vals) {
  for (int tx = rr.a0; tx <= rr.a1; ++tx, ++pos)
    if (pos < stop) { keys[pos] = rowbase + tx; vals[pos] = r; }
  for (int tx = rr.b0; tx <= rr.b1; ++tx, ++pos)
    if (pos < stop) { keys[pos] = rowbase + tx; vals[pos] = r; }
  return pos;
}

// The (tile, record) pairs, written in depth order: entry i of the depth
// order (record order[i]) writes its tiles from offsets[i] on, rows in order
// and tiles left to right, so the runs of consecutive entries are adjacent and
// a warp's stores are contiguous.  The row runs of the entries that span few
// rows are computed with those rows spread over the warp; the warp then writes
// all those entries' tiles as one flat list, 32 consecutive slots per step.  The
// rows of an entry with many rows are shared out over the warp, with a warp scan
// of the row counts.
constexpr int kDupThreads = 128;
constexpr int kWarpsPerBlock = kDupThreads / 32;

__global__ void __launch_bounds__(kDupThreads) duplicate_kernel(
    const uint32_t* __restrict__ order, const uint64_t* __restrict__ offsets, const uint64_t* __restrict__ total,
    uint32_t n_rec, const float4* __restrict__ bin, const DevCam* __restrict__ cams, int64_t n_gauss, int tw, int th,
    uint32_t n_pairs, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  __shared__ short4 s_runs[kWarpsPerBlock][kSmallRows][32];  // [row][lane]: lanes in distinct banks
  __shared__ int s_incl[kWarpsPerBlock][32];
  __shared__ uint32_t s_rowbase[kWarpsPerBlock][32];  // tile id of (first row, column 0)
  __shared__ uint32_t s_tilesx[kWarpsPerBlock][32];
  __shared__ uint32_t s_pos[kWarpsPerBlock][32];
  __shared__ uint32_t s_rec[kWarpsPerBlock][32];
  __shared__ RowOwner s_own[kWarpsPerBlock][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t i = blockIdx.x * kDupThreads + threadIdx.x;
  uint32_t r = 0;
  int cnt = 0;
  BinView bv;
  bv.rc = make_int4(0, 0, -1, -1);
  uint64_t o = 0;
  if (i < n_rec) {
    o = offsets[i];
    r = order[i];
  }
  // this entry's count: the next entry's offset (or the total) minus its own
  uint64_t o_next = __shfl_down_sync(kFull, o, 1);
  if (lane == 31 || i + 1 >= n_rec) o_next = (i + 1 < n_rec) ? offsets[i + 1] : *total;
  if (i < n_rec && o < (uint64_t)n_pairs) {  // entries past a capacity write nothing
    cnt = (int)(o_next - o);
    if (cnt > 0) bv = load_bin(bin, r);
  }
  const int4 rc = bv.rc;
  const bool small = cnt > 0 && (rc.w - rc.y + 1) <= kSmallRows;
  if (small) {
    const DevCam& cam = cams[view_of_record(r, n_gauss)];
    s_own[warp][lane] = RowOwner{support_conic(bv.g0, bv.g1, bv.g2, bv.rb), rc, cam.tile_offset, cam.tiles_x, cam.W,
                                 cam.H};
    s_rowbase[warp][lane] = (uint32_t)(cam.tile_offset + rc.y * cam.tiles_x);
    s_tilesx[warp][lane] = (uint32_t)cam.tiles_x;
    s_pos[warp][lane] = (uint32_t)o;
    s_rec[warp][lane] = r;
  }
  // the row runs of the small entries, the rows spread over the warp
  for_warp_rows(small ? rc.w - rc.y + 1 : 0, lane, s_incl[warp], s_own[warp], [&](int ri, int ty) {
    const RowOwner& ow = s_own[warp][ri];
    const RowRuns rr = row_runs(ow.k, ty, tw, th, ow.W, ow.H, ow.rc);
    s_runs[warp][ty - ow.rc.y][ri] = make_short4((short)rr.a0, (short)rr.a1, (short)rr.b0, (short)rr.b1);
  });
  // flat walk over the small entries' tiles
  const int scnt = small ? cnt : 0;
  int incl = scnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += t;
  }
  s_incl[warp][lane] = incl;
  const int all = __shfl_sync(kFull, incl, 31);
  __syncwarp();
  for (int q0 = 0; q0 < all; q0 += 32) {
    const int q = q0 + lane;
    if (q < all) {
      int lo = 0, hi = 31;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_incl[warp][mid] > q) hi = mid; else lo = mid + 1;
      }
      const int ri = lo;
      const int excl = ri > 0 ? s_incl[warp][ri - 1] : 0;  // tiles of the warp's earlier small entries
      int kth = q - excl;
      int tx = -1, row = 0;
      for (; row < kSmallRows; ++row) {
        const short4 ru = s_runs[warp][row][ri];
        const int la = max(0, (int)ru.y - (int)ru.x + 1), lb = max(0, (int)ru.w - (int)ru.z + 1);
        if (kth < la) { tx = ru.x + kth; break; }
        kth -= la;
        if (kth < lb) { tx = ru.z + kth; break; }
        kth -= lb;
      }
      const uint32_t pos = s_pos[warp][ri] + (uint32_t)(q - excl);
      if (tx >= 0 && pos < n_pairs) {
        keys[pos] = s_rowbase[warp][ri] + (uint32_t)row * s_tilesx[warp][ri] + (uint32_t)tx;
        vals[pos] = s_rec[warp][ri];
      }
    }
  }
  unsigned big = __ballot_sync(kFull, cnt > 0 && !small);
  while (big) {
    const int src = __ffs(big) - 1;
    big &= big - 1u;
    const uint32_t rr = __shfl_sync(kFull, r, src);
    const uint64_t oo = __shfl_sync(kFull, o, src);
    const int bcnt = __shfl_sync(kFull, cnt, src);
    const BinView bb = load_bin(bin, rr);
    const int4 bc = bb.rc;
    const DevCam& cam = cams[view_of_record(rr, n_gauss)];
    const SupportConic k = support_conic(bb.g0, bb.g1, bb.g2, bb.rb);
    const uint64_t stop = min(oo + (uint64_t)bcnt, (uint64_t)n_pairs);
    uint64_t base = oo;
    for (int row0 = bc.y; row0 <= bc.w; row0 += 32) {
      const int ty = row0 + lane;
      RowRuns runs{1, 0, 1, 0};
      int c = 0;
      if (ty <= bc.w) {
        runs = row_runs(k, ty, tw, th, cam.W, cam.H, bc);
        c = row_count(runs);
      }
      int inc = c;
#pragma unroll
      for (int s2 = 1; s2 < 32; s2 <<= 1) {
        const int t = __shfl_up_sync(kFull, inc, s2);
        if (lane >= s2) inc += t;
      }
      if (c > 0)
        write_runs(runs, (uint32_t)(cam.tile_offset + ty * cam.tiles_x), rr, base + (uint64_t)(inc - c), stop, keys,
                   vals);
      base += (uint64_t)__shfl_sync(kFull, inc, 31);
    }
  }
}

// [start, end) of every tile in the sorted keys: each thread takes 4
// consecutive keys with one 16-byte load and finds their neighbours across
// lanes with shuffles (the warp's two outer neighbours come from memory).
__global__ void tile_ranges_kernel(const uint32_t* __restrict__ keys, uint32_t n, uint2* __restrict__ ranges,
                                   const uint32_t* __restrict__ d_n) {
  if (d_n) n = min(n, *d_n);
  const int lane = threadIdx.x & 31;
  const uint32_t groups = (n + 3) / 4;
  for (uint32_t base = blockIdx.x * blockDim.x; base < groups; base += gridDim.x * blockDim.x) {
    const uint32_t i0 = (base + threadIdx.x) * 4;
    uint32_t k[4];
    if (i0 + 3 < n) {
      const uint4 v = *reinterpret_cast<const uint4*>(keys + i0);
      k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? keys[i0 + j] : 0xffffffffu;
    }
    uint32_t prev = __shfl_up_sync(kFull, k[3], 1);
    uint32_t next = __shfl_down_sync(kFull, k[0], 1);
    if (lane == 0 && i0 > 0 && i0 <= n) prev = keys[i0 - 1];
    if (lane == 31 && i0 + 4 < n) next = keys[i0 + 4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t idx = i0 + j;
      if (idx < n) {
        const uint32_t p = j ? k[j - 1] : prev;
        const uint32_t q = j < 3 ? k[j + 1] : next;
        if (idx == 0 || p != k[j]) ranges[k[j]].x = idx;
        if (idx == n - 1 || q != k[j]) ranges[k[j]].y = idx + 1;
      }
    }
  }
}

// work key for the persistent queue: heaviest tiles first (descending log-scale
// pair count, one 8-bit radix pass)
__global__ void tile_work_kernel(const uint2* __restrict__ ranges, const uint2* __restrict__ ranges2, uint32_t n,
                                 uint32_t* __restrict__ work_key, uint32_t* __restrict__ ids) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint2 r = ranges[t];
  uint32_t len = r.y - r.x;
  if (ranges2) len += ranges2[t].y - ranges2[t].x;
  work_key[t] = queue_key(len);
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
                             uint32_t n, int n_bits, void* scratch, bool* result_in_alt, cudaStream_t s,
                             const uint32_t* d_n, bool index_vals) {
  *result_in_alt = false;
  if (n <= 1 || n_bits <= 0) {
    if (index_vals && n > 0) {  // nothing to sort: the values are the indices
      launch_iota(vals, n, s);
      return launched();
    }
    return cudaSuccess;
  }
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
    radix_upsweep_kernel<<<nb, kBlock, 0, s>>>(kin, n, shift, mask, counts, nb, d_n);
    cudaError_t e = launched();
    if (e != cudaSuccess) return e;
    e = scan_exclusive<uint32_t>(counts, counts, (mask + 1) * nb, nullptr, scan_scratch, s);
    if (e != cudaSuccess) return e;
    radix_scatter_kernel<<<nb, kBlock, 0, s>>>(kin, p == 0 && index_vals ? nullptr : vin, kout, vout, n, shift,
                                               mask, counts, nb, d_n);
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

cudaError_t launch_tile_count(const float4* bin, const DevCam* cams, int64_t n_gauss, uint32_t n_rec, int tile_w,
                              int tile_h, int32_t* ntiles, uint32_t* depth_key, cudaStream_t s) {
  if (n_rec == 0) return cudaSuccess;
  tile_count_kernel<<<(n_rec + kThreads - 1) / kThreads, kThreads, 0, s>>>(bin, cams, n_gauss, n_rec, tile_w, tile_h,
                                                                           ntiles, depth_key);
  return launched();
}

cudaError_t launch_duplicate(const uint32_t* order, const uint64_t* offsets, const uint64_t* total, uint32_t n_rec,
                             const float4* bin, const DevCam* cams, int64_t n_gauss, int tile_w, int tile_h,
                             uint32_t n_pairs, uint32_t* keys, uint32_t* vals, cudaStream_t s) {
  if (n_pairs == 0 || n_rec == 0) return cudaSuccess;
  duplicate_kernel<<<(n_rec + kDupThreads - 1) / kDupThreads, kDupThreads, 0, s>>>(
      order, offsets, total, n_rec, bin, cams, n_gauss, tile_w, tile_h, n_pairs, keys, vals);
  return launched();
}

cudaError_t launch_tile_ranges(const uint32_t* keys, uint32_t n_pairs, uint2* ranges, cudaStream_t s,
                               const uint32_t* d_n) {
  if (n_pairs == 0) return cudaSuccess;
  const uint32_t blocks = (n_pairs / 4 + 256) / 256;
  tile_ranges_kernel<<<blocks < 152u * 16u ? blocks : 152u * 16u, 256, 0, s>>>(keys, n_pairs, ranges, d_n);
  return launched();
}

cudaError_t launch_tile_order(const uint2* ranges, uint32_t n_tiles, uint32_t* work_key, uint32_t* tile_ids,
                              cudaStream_t s, const uint2* ranges2) {
  if (n_tiles == 0) return cudaSuccess;
  tile_work_kernel<<<(n_tiles + 255) / 256, 256, 0, s>>>(ranges, ranges2, n_tiles, work_key, tile_ids);
  return launched();
}

}  // namespace ocgs

namespace ocgs {
namespace {
__global__ void clamp_count_kernel(const uint64_t* __restrict__ total, uint32_t cap, uint32_t* __restrict__ n32,
                                   int* __restrict__ status) {
  const uint64_t t = *total;
  *n32 = (uint32_t)(t < (uint64_t)cap ? t : (uint64_t)cap);
  if (t > (uint64_t)cap) atomicOr(status, kStatusCapacity);
}
}  // namespace

cudaError_t launch_clamp_count(const uint64_t* total, uint32_t cap, uint32_t* n32, int* status, cudaStream_t s) {
  clamp_count_kernel<<<1, 1, 0, s>>>(total, cap, n32, status);
  return launched();
}

}  // namespace ocgs

// ------------------------------------------------------------------ two-pass binning
// The first pass bins only the records at the front of the depth order; the
// tiles whose pixels all stop inside that prefix (the front-to-back walk of
// Sec. 4.3 ends when T falls below its bound) are final.  The second pass bins
// the records behind the front, but only into the tiles still open, and those
// tiles continue from where the first pass stopped.  Each tile's list is the
// one a single pass builds (records in depth order), split in two segments.
namespace ocgs {
namespace {

__device__ __forceinline__ int4 bin_rect(const float4 b2) {
  const uint32_t xy = __float_as_uint(b2.z), zw = __float_as_uint(b2.w);
  return make_int4((int)(int16_t)(xy & 0xffffu), (int)(int16_t)(xy >> 16), (int)(int16_t)(zw & 0xffffu),
                   (int)(int16_t)(zw >> 16));
}

// open tiles among [rowbase + x0, rowbase + x1] from the exclusive prefix P of the open flags
__device__ __forceinline__ int open_in(const uint32_t* __restrict__ P, uint32_t rowbase, int x0, int x1) {
  return x1 < x0 ? 0 : (int)(P[rowbase + (uint32_t)x1 + 1u] - P[rowbase + (uint32_t)x0]);
}

constexpr int kFlatWarps = kThreads / 32;

__global__ void __launch_bounds__(kThreads) tile_count_sorted_kernel(const uint32_t* __restrict__ order, uint32_t n,
                                                                     const float4* __restrict__ bin,
                                                                     const DevCam* __restrict__ cams, int64_t n_gauss,
                                                                     int tw, int th, int32_t* __restrict__ ntiles,
                                                                     uint64_t* __restrict__ counts) {
  __shared__ RowOwner s_own[kFlatWarps][32];
  __shared__ int s_incl[kFlatWarps][32], s_cnt[kFlatWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
  uint32_t r = 0;
  int nrows = 0;
  if (i < n) {
    r = order[i];
    const BinView b = load_bin(bin, r);
    if (b.rc.z >= b.rc.x) {
      const DevCam& cam = cams[view_of_record(r, n_gauss)];
      s_own[warp][lane] = RowOwner{support_conic(b.g0, b.g1, b.g2, b.rb), b.rc, cam.tile_offset, cam.tiles_x,
                                   cam.W, cam.H};
      nrows = b.rc.w - b.rc.y + 1;
    }
  }
  s_cnt[warp][lane] = 0;
  for_warp_rows(nrows, lane, s_incl[warp], s_own[warp], [&](int ri, int ty) {
    const RowOwner& o = s_own[warp][ri];
    const int c = row_count(row_runs(o.k, ty, tw, th, o.W, o.H, o.rc));
    if (c) atomicAdd(&s_cnt[warp][ri], c);
  });
  if (i < n) {
    const int cnt = s_cnt[warp][lane];
    ntiles[r] = cnt;
    counts[i] = (uint64_t)cnt;
  }
}

// number of entries of an ascending array below key: a 32-way search by one warp
// (each round probes 32 evenly spaced entries of the bracket [lo, hi] that holds
// the answer and keeps the stretch between the last probe below key and the next)
__global__ void count_below_kernel(const uint32_t* __restrict__ sorted_keys, uint32_t n, uint32_t key,
                                   uint32_t* __restrict__ out) {
  const uint32_t lane = threadIdx.x;
  uint32_t lo = 0, hi = n;
  while (hi - lo > 32u) {
    const uint32_t step = (hi - lo + 31u) / 32u;
    const uint32_t pos = lo + lane * step;
    const int c = __popc(__ballot_sync(kFull, pos < hi && sorted_keys[pos] < key));
    const uint32_t nhi = min(hi, lo + (uint32_t)c * step);
    lo = c > 0 ? lo + (uint32_t)(c - 1) * step + 1u : lo;
    hi = nhi;
  }
  const uint32_t pos = lo + lane;
  const int c = __popc(__ballot_sync(kFull, pos < hi && sorted_keys[pos] < key));
  if (lane == 0) *out = lo + (uint32_t)c;
}

// Second pass, step 1: flag the entries (records behind the front, in depth
// order) whose candidate rectangle holds an open tile (row sums of the open
// flags from their prefix P, all rows loaded independently).
__global__ void __launch_bounds__(kThreads) open_candidate_kernel(const uint32_t* __restrict__ order, uint32_t n,
                                                                  const float4* __restrict__ bin,
                                                                  const DevCam* __restrict__ cams, int64_t n_gauss,
                                                                  const uint32_t* __restrict__ P,
                                                                  uint32_t* __restrict__ flag) {
  const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const uint32_t r = order[i];
  const int4 rc = bin_rect(bin[3 * (size_t)r + 2]);
  int cand = 0;
  if (rc.z >= rc.x) {
    const DevCam& cam = cams[view_of_record(r, n_gauss)];
    const uint32_t base = (uint32_t)(cam.tile_offset + rc.y * cam.tiles_x);
    for (int ty = rc.y; ty <= rc.w; ++ty)
      cand += open_in(P, base + (uint32_t)((ty - rc.y) * cam.tiles_x), rc.x, rc.z);
  }
  flag[i] = cand > 0 ? 1u : 0u;
}

// step 2: the flagged entries' records, in depth order (pos: exclusive scan of the flags)
__global__ void compact_candidates_kernel(const uint32_t* __restrict__ order, uint32_t n,
                                          const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                                          uint32_t* __restrict__ cand) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) cand[pos[i]] = order[i];
}

// step 3: open tiles reached by each candidate (counts[c] = 0 for c >= *n_cand)
__global__ void __launch_bounds__(kThreads) open_count_kernel(const uint32_t* __restrict__ cand, uint32_t n,
                                                              const uint32_t* __restrict__ n_cand,
                                                              const float4* __restrict__ bin,
                                                              const DevCam* __restrict__ cams, int64_t n_gauss,
                                                              int tw, int th, const uint32_t* __restrict__ P,
                                                              uint64_t* __restrict__ counts) {
  __shared__ RowOwner s_own[kFlatWarps][32];
  __shared__ int s_incl[kFlatWarps][32], s_cnt[kFlatWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t c = blockIdx.x * kThreads + threadIdx.x;
  const uint32_t nc = min(n, *n_cand);
  int nrows = 0;
  if (c < nc) {
    const uint32_t r = cand[c];
    const BinView b = load_bin(bin, r);
    const DevCam& cam = cams[view_of_record(r, n_gauss)];
    s_own[warp][lane] = RowOwner{support_conic(b.g0, b.g1, b.g2, b.rb), b.rc, cam.tile_offset, cam.tiles_x,
                                 cam.W, cam.H};
    nrows = max(0, b.rc.w - b.rc.y + 1);
  }
  s_cnt[warp][lane] = 0;
  for_warp_rows(nrows, lane, s_incl[warp], s_own[warp], [&](int ri, int ty) {
    const RowOwner& o = s_own[warp][ri];
    const RowRuns rr = row_runs(o.k, ty, tw, th, o.W, o.H, o.rc);
    const uint32_t rowbase = (uint32_t)(o.tile_offset + ty * o.tiles_x);
    const int cnt = open_in(P, rowbase, rr.a0, rr.a1) + open_in(P, rowbase, rr.b0, rr.b1);
    if (cnt) atomicAdd(&s_cnt[warp][ri], cnt);
  });
  if (c < n) counts[c] = (uint64_t)s_cnt[warp][lane];
}

// The open tiles, compacted in ascending id: open_ids[P[t]] = t for every open tile t.
__global__ void open_ids_kernel(const uint32_t* __restrict__ open, const uint32_t* __restrict__ P, uint32_t n,
                                uint32_t* __restrict__ open_ids) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && open[t]) open_ids[P[t]] = t;
}

// The open tiles of the run [x0, x1] of a tile row are the contiguous slice
// open_ids[P[rowbase + x0], P[rowbase + x1 + 1]) of the compacted open ids.
struct OpenSlice {
  uint32_t start;
  int count;
};
__device__ __forceinline__ OpenSlice open_slice(const uint32_t* __restrict__ P, uint32_t rowbase, int x0, int x1) {
  if (x1 < x0) return OpenSlice{0u, 0};
  const uint32_t a = P[rowbase + (uint32_t)x0];
  return OpenSlice{a, (int)(P[rowbase + (uint32_t)x1 + 1u] - a)};
}

constexpr int kOpenThreads = 128;
constexpr int kOpenWarps = kOpenThreads / 32;

// step 4, the second-pass pairs in depth order: candidate i writes its open
// tiles from offsets[i] on (rows in order, tiles left to right), each run's open
// tiles being a slice of open_ids.  A lane finds the slices of its candidate
// when it spans few rows and the warp writes all those candidates' tiles as one
// flat list, 32 consecutive slots per step; the rows of a taller candidate are
// shared out over the warp.
__global__ void __launch_bounds__(kOpenThreads) duplicate_open_kernel(
    const uint32_t* __restrict__ order, const uint64_t* __restrict__ offsets, const uint64_t* __restrict__ total,
    uint32_t n_rec, const uint32_t* __restrict__ n_cand, const float4* __restrict__ bin,
    const DevCam* __restrict__ cams, int64_t n_gauss, int tw, int th, const uint32_t* __restrict__ open_ids,
    const uint32_t* __restrict__ P, uint32_t n_pairs, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  __shared__ uint32_t s_sa[kOpenWarps][kSmallRows][32], s_sb[kOpenWarps][kSmallRows][32];  // [row][lane]
  __shared__ uint32_t s_cnt[kOpenWarps][kSmallRows][32];  // open tiles of the two runs: a | b << 16
  __shared__ int s_incl[kOpenWarps][32];
  __shared__ uint32_t s_pos[kOpenWarps][32];
  __shared__ uint32_t s_rec[kOpenWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t i = blockIdx.x * kOpenThreads + threadIdx.x;
  n_rec = min(n_rec, *n_cand);
  uint32_t r = 0;
  uint64_t o = 0;
  if (i < n_rec) {
    o = offsets[i];
    r = order[i];
  }
  uint64_t o_next = __shfl_down_sync(kFull, o, 1);
  if (lane == 31 || i + 1 >= n_rec) o_next = (i + 1 < n_rec) ? offsets[i + 1] : *total;
  int cnt = 0;
  int4 rc = make_int4(0, 0, -1, -1);
  if (i < n_rec && o < (uint64_t)n_pairs) {  // entries past a capacity write nothing
    cnt = (int)(o_next - o);
    if (cnt > 0) rc = bin_rect(bin[3 * (size_t)r + 2]);
  }
  const bool small = cnt > 0 && (rc.w - rc.y + 1) <= kSmallRows;
  if (small) {
    // a lane finds its candidate's slices (the rows spread over the warp measured slower
    // here, the candidates behind the front spanning few rows)
    const BinView b = load_bin(bin, r);
    const DevCam& cam = cams[view_of_record(r, n_gauss)];
    const SupportConic k = support_conic(b.g0, b.g1, b.g2, b.rb);
    for (int ty = rc.y; ty <= rc.w; ++ty) {
      const RowRuns rr = row_runs(k, ty, tw, th, cam.W, cam.H, rc);
      const uint32_t rowbase = (uint32_t)(cam.tile_offset + ty * cam.tiles_x);
      const OpenSlice sa = open_slice(P, rowbase, rr.a0, rr.a1), sb = open_slice(P, rowbase, rr.b0, rr.b1);
      s_sa[warp][ty - rc.y][lane] = sa.start;
      s_sb[warp][ty - rc.y][lane] = sb.start;
      s_cnt[warp][ty - rc.y][lane] = (uint32_t)sa.count | ((uint32_t)sb.count << 16);
    }
    s_pos[warp][lane] = (uint32_t)o;
    s_rec[warp][lane] = r;
  }
  // flat walk over the small candidates' open tiles
  const int scnt = small ? cnt : 0;
  int incl = scnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += t;
  }
  s_incl[warp][lane] = incl;
  const int all = __shfl_sync(kFull, incl, 31);
  __syncwarp();
  for (int q0 = 0; q0 < all; q0 += 32) {
    const int q = q0 + lane;
    if (q < all) {
      int lo = 0, hi = 31;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_incl[warp][mid] > q) hi = mid; else lo = mid + 1;
      }
      const int ri = lo;
      const int excl = ri > 0 ? s_incl[warp][ri - 1] : 0;  // tiles of the warp's earlier small candidates
      int kth = q - excl;
      uint32_t slot = 0xffffffffu;
      for (int row = 0; row < kSmallRows; ++row) {
        const uint32_t c = s_cnt[warp][row][ri];
        const int la = (int)(c & 0xffffu), lb = (int)(c >> 16);
        if (kth < la) { slot = s_sa[warp][row][ri] + (uint32_t)kth; break; }
        kth -= la;
        if (kth < lb) { slot = s_sb[warp][row][ri] + (uint32_t)kth; break; }
        kth -= lb;
      }
      const uint32_t pos = s_pos[warp][ri] + (uint32_t)(q - excl);
      if (slot != 0xffffffffu && pos < n_pairs) {
        keys[pos] = open_ids[slot];
        vals[pos] = s_rec[warp][ri];
      }
    }
  }
  unsigned big = __ballot_sync(kFull, cnt > 0 && !small);
  while (big) {
    const int src = __ffs(big) - 1;
    big &= big - 1u;
    const uint32_t rr = __shfl_sync(kFull, r, src);
    const uint64_t oo = __shfl_sync(kFull, o, src);
    const int bcnt = __shfl_sync(kFull, cnt, src);
    const BinView bb = load_bin(bin, rr);
    const int4 bc = bb.rc;
    const DevCam& cam = cams[view_of_record(rr, n_gauss)];
    const SupportConic k = support_conic(bb.g0, bb.g1, bb.g2, bb.rb);
    const uint64_t stop = min(oo + (uint64_t)bcnt, (uint64_t)n_pairs);
    uint64_t base = oo;
    for (int row0 = bc.y; row0 <= bc.w; row0 += 32) {
      const int ty = row0 + lane;
      OpenSlice sa{0u, 0}, sb{0u, 0};
      if (ty <= bc.w) {
        const RowRuns runs = row_runs(k, ty, tw, th, cam.W, cam.H, bc);
        const uint32_t rowbase = (uint32_t)(cam.tile_offset + ty * cam.tiles_x);
        sa = open_slice(P, rowbase, runs.a0, runs.a1);
        sb = open_slice(P, rowbase, runs.b0, runs.b1);
      }
      const int c = sa.count + sb.count;
      int inc = c;
#pragma unroll
      for (int s2 = 1; s2 < 32; s2 <<= 1) {
        const int t = __shfl_up_sync(kFull, inc, s2);
        if (lane >= s2) inc += t;
      }
      uint64_t pos = base + (uint64_t)(inc - c);
      for (int j = 0; j < sa.count; ++j, ++pos)
        if (pos < stop) { keys[pos] = open_ids[sa.start + (uint32_t)j]; vals[pos] = rr; }
      for (int j = 0; j < sb.count; ++j, ++pos)
        if (pos < stop) { keys[pos] = open_ids[sb.start + (uint32_t)j]; vals[pos] = rr; }
      base += (uint64_t)__shfl_sync(kFull, inc, 31);
    }
  }
}

// The second pass's queue: tiles with a second-pass segment, longest first (log scale),
// every other tile last; n_again counts the former.
__global__ void second_queue_kernel(const uint2* __restrict__ ranges2, uint32_t n_tiles,
                                    uint32_t* __restrict__ work_key, uint32_t* __restrict__ ids,
                                    uint32_t* __restrict__ n_again) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  const uint2 r2 = ranges2[t];
  const uint32_t len = r2.y - r2.x;
  if (len) atomicAdd(n_again, 1u);
  work_key[t] = queue_key(len);
  ids[t] = t;
}

}  // namespace

cudaError_t launch_tile_count_sorted(const uint32_t* order, uint32_t n, const float4* bin, const DevCam* cams,
                                     int64_t n_gauss, int tile_w, int tile_h, int32_t* ntiles, uint64_t* counts,
                                     cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  tile_count_sorted_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(order, n, bin, cams, n_gauss, tile_w,
                                                                              tile_h, ntiles, counts);
  return launched();
}

cudaError_t launch_count_below(const uint32_t* sorted_keys, uint32_t n, uint32_t key, uint32_t* out,
                               cudaStream_t s) {
  count_below_kernel<<<1, 32, 0, s>>>(sorted_keys, n, key, out);
  return launched();
}

cudaError_t launch_open_candidates(const uint32_t* order, uint32_t n, const float4* bin, const DevCam* cams,
                                   int64_t n_gauss, const uint32_t* open_prefix, uint32_t* flag, uint32_t* pos,
                                   uint32_t* cand, uint32_t* n_cand, void* scratch, cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(n_cand, 0, sizeof(uint32_t), s);
  open_candidate_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(order, n, bin, cams, n_gauss,
                                                                           open_prefix, flag);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  e = scan_exclusive<uint32_t>(flag, pos, n, n_cand, static_cast<char*>(scratch), s);
  if (e != cudaSuccess) return e;
  compact_candidates_kernel<<<(n + 255) / 256, 256, 0, s>>>(order, n, flag, pos, cand);
  return launched();
}

cudaError_t launch_open_count(const uint32_t* cand, uint32_t n, const uint32_t* n_cand, const float4* bin,
                              const DevCam* cams, int64_t n_gauss, int tile_w, int tile_h,
                              const uint32_t* open_prefix, uint64_t* counts, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  open_count_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(cand, n, n_cand, bin, cams, n_gauss, tile_w,
                                                                       tile_h, open_prefix, counts);
  return launched();
}

cudaError_t launch_duplicate_open(const uint32_t* cand, const uint64_t* offsets, const uint64_t* total,
                                  uint32_t n_rec, const uint32_t* n_cand, const float4* bin, const DevCam* cams,
                                  int64_t n_gauss, int tile_w, int tile_h, const uint32_t* open,
                                  const uint32_t* open_prefix, uint32_t n_tiles, uint32_t* open_ids, uint32_t n_pairs,
                                  uint32_t* keys, uint32_t* vals, cudaStream_t s) {
  if (n_pairs == 0 || n_rec == 0) return cudaSuccess;
  open_ids_kernel<<<(n_tiles + 255) / 256, 256, 0, s>>>(open, open_prefix, n_tiles, open_ids);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  duplicate_open_kernel<<<(n_rec + kOpenThreads - 1) / kOpenThreads, kOpenThreads, 0, s>>>(
      cand, offsets, total, n_rec, n_cand, bin, cams, n_gauss, tile_w, tile_h, open_ids, open_prefix, n_pairs, keys,
      vals);
  return launched();
}

cudaError_t launch_second_queue(const uint2* ranges2, uint32_t n_tiles, uint32_t* work_key, uint32_t* ids,
                                uint32_t* n_again, cudaStream_t s) {
  if (n_tiles == 0) return cudaSuccess;
  second_queue_kernel<<<(n_tiles + 255) / 256, 256, 0, s>>>(ranges2, n_tiles, work_key, ids, n_again);
  return launched();
}

}  // namespace ocgs
