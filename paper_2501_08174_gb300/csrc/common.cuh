// Internal definitions shared by the CUDA translation units of libocgs.
//
// Record layout of one (view, Gaussian) pair, written by the preprocess kernel
// and read by the rasterizers (structure of arrays, one float4 per array):
//   g0 = (c_x, c_y, o, z_c)      projected centre [px], opacity, centre depth
//   g1 = (A00, A01, A10, A11)    numerator of the ray-splat hit (u, v)
//   g2 = (e0, e1, e2, zD)        denominator coefficients and zD = z_c * e0
//   a0 = (r, g, b, n_x)          colour and camera-frame normal
//   a1 = (n_y, n_z)
// For a pixel centre x with (dx, dy) = x - c the ray-splat intersection of
// 2DGS (planes x = const and y = const pulled back through the surfel's
// splat-to-pixel matrix, then crossed) reduces to the projective map
//   u = (A00 dx + A01 dy) / den,  v = (A10 dx + A11 dy) / den,
//   den = e0 + e1 dx + e2 dy,  z_hit = zD / den,
// which is the same intersection written about the projected centre so that
// no large pixel coordinates cancel in float32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace ocgs {

constexpr float kRhoCut = 9.0f;            // support cut-off rho <= 9 (3 sigma)
constexpr float kAlphaMin = 1.0f / 255.0f;  // skip below this opacity
constexpr float kAlphaMax = 0.99f;          // opacity clamp
// Opacity below which the 0.99 clamp of alpha never applies: G = exp(-rho/2) <= 1
// for rho >= 0 (the base-2 exponential's relative error is about 2^-22), so o G <
// 0.989 (1 + 2^-20) < 0.99.  The backward takes a clamp-free path for such a
// record, whose alpha = o (blended ? G : 0) equals the clamped form bit for bit.
constexpr float kNoClampO = 0.989f;
constexpr float kTEps = 1e-4f;              // stop when T (1 - alpha) would fall below this
constexpr float kInvSigmaF2 = 2.0f;         // 1 / sigma_f^2 of the screen low-pass filter (sigma_f^2 = 1/2 px^2)

// status bits raised on the device, read back by the host
constexpr int kStatusNonFinite = 1;
constexpr int kStatusCapacity = 2;
constexpr int kStatusTimeout = 4;

struct DevCam {
  float R[9];        // world->camera rotation, row-major
  float t[3];
  float fx, fy, cx, cy;
  float campos[3];   // camera centre in world coordinates
  float near_plane;
  int W, H;
  int tiles_x, tiles_y;
  int tile_offset;   // first global tile id of this view
  int cover_rect;    // 1: the binning takes every tile of a record's screen rectangle (no support test)
  long long pix_offset;  // first pixel of this view in the concatenated images
};

struct RecPtrs {
  float4* g0;
  float4* g1;
  float4* g2;
  float4* a0;
  float4* a1;  // (n_y, n_z, lowest, highest pixel-centre row the support reaches)
};

struct ImgPtrs {
  float* rgb;
  float* alpha;
  float* depth;
  float* normal;
  float* depth2;  // sum w z^2, optional
};

struct GaussPtrs {
  const float* xyz;
  const float* quat;
  const float* scale;
  const float* opacity;
  const float* sh;
};

struct GaussOut {
  float* xyz;
  float* quat;
  float* scale;
  float* opacity;
  float* sh;
};

// number of float slots of one record gradient (18 used, padded to 5 float4)
constexpr int kGradStride = 20;
// The first kGradSlotsRGB slots are the ones a loss on colour and opacity alone
// reaches; the depth and normal cotangents add the last five.
// The colour slots r, g, b share the third float4 (slots 8..11), so the colour's
// chain rule reads them with one aligned 16-byte load.
enum GradSlot {
  kGcx = 0, kGcy, kGo, kGA00, kGA01, kGA10, kGA11, kGe0, kGr, kGg, kGb, kGe1, kGe2,
  kGzc, kGzD, kGnx, kGny, kGnz
};
static_assert(kGr % 4 == 0 && kGb / 4 == kGr / 4, "colour slots in one float4");
constexpr int kGradSlotsRGB = 13;
constexpr int kGradSlots = 18;

__device__ __forceinline__ bool finitef(float x) { return isfinite(x); }

// Support bound in rho of a surfel of opacity o: the 3-sigma cut, tightened to
// where o exp(-rho/2) can still reach 1/255 (with a margin, so that no pixel
// that FP32 would blend lies outside).  Used for the screen box and tile test.
__device__ __forceinline__ float support_rho(float o) {
  return fminf(kRhoCut, __fadd_rn(__fmul_rn(2.0f, __logf(__fmul_rn(255.0f, o))), 1e-3f));
}

// sqrt from the approximate reciprocal square root (the coverage test below
// carries margins far above its error; every caller uses the same function).
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.f ? __fmul_rn(x, rsqrtf(x)) : 0.f; }

// Screen support of a record, {rho <= rb} grown by 0.1 % (+1e-3) in rho:
//  * the filter disc |x - c|^2 <= r2f, and
//  * the projected surfel disc, the ellipse
//      (A00 dx + A01 dy)^2 + (A10 dx + A11 dy)^2 <= rt (e0 + e1 dx + e2 dy)^2
//    in (dx, dy) = x - c, written a dx^2 + 2 b dx dy + c dy^2 + 2 d dx + 2 e dy + f <= 0
//    and, about its centre m, a u^2 + 2 b u v + c v^2 <= kappa.
struct SupportConic {
  float cx, cy, r2f;
  float a, b, c;
  float mx, my, kappa, det;
  float umax, vmax, vstar;  // x half-extent, y half-extent, v of the rightmost point
  bool ellipse;             // a > 0, det > 0, kappa > 0 and finite
};

__device__ __forceinline__ SupportConic support_conic(const float4 g0, const float4 g1, const float4 g2, float rb) {
  SupportConic k;
  const float rt = __fadd_rn(__fmul_rn(rb, 1.001f), 1e-3f);
  k.cx = g0.x;
  k.cy = g0.y;
  k.r2f = __fmul_rn(0.5f, rt);
  k.a = __fsub_rn(__fmaf_rn(g1.x, g1.x, __fmul_rn(g1.z, g1.z)), __fmul_rn(rt, __fmul_rn(g2.y, g2.y)));
  k.b = __fsub_rn(__fmaf_rn(g1.x, g1.y, __fmul_rn(g1.z, g1.w)), __fmul_rn(rt, __fmul_rn(g2.y, g2.z)));
  k.c = __fsub_rn(__fmaf_rn(g1.y, g1.y, __fmul_rn(g1.w, g1.w)), __fmul_rn(rt, __fmul_rn(g2.z, g2.z)));
  // With p = (A00, A10) and q = (A01, A11), the columns of the map, and w = e1 q - e2 p,
  // Lagrange's identity gives det = a c - b^2 = (A00 A11 - A01 A10)^2 - rt |w|^2, the
  // centre m = rt e0 (q.w, -p.w) / det and kappa = rt e0 (e0 + e1 mx + e2 my).  These
  // forms keep their accuracy for a thin ellipse (an almost edge-on surfel), where the
  // product form a c - b^2 cancels to a few correct digits and shrinks the support.
  const float D = __fmaf_rn(g1.x, g1.w, -__fmul_rn(g1.y, g1.z));
  const float wx = __fmaf_rn(g2.y, g1.y, -__fmul_rn(g2.z, g1.x));
  const float wy = __fmaf_rn(g2.y, g1.w, -__fmul_rn(g2.z, g1.z));
  k.det = __fsub_rn(__fmul_rn(D, D), __fmul_rn(rt, __fmaf_rn(wx, wx, __fmul_rn(wy, wy))));
  const float s = __fmul_rn(rt, g2.x);
  k.mx = __fdividef(__fmul_rn(s, __fmaf_rn(g1.y, wx, __fmul_rn(g1.w, wy))), k.det);
  k.my = -__fdividef(__fmul_rn(s, __fmaf_rn(g1.x, wx, __fmul_rn(g1.z, wy))), k.det);
  k.kappa = __fmul_rn(s, __fmaf_rn(g2.z, k.my, __fmaf_rn(g2.y, k.mx, g2.x)));
  k.ellipse = k.a > 0.f && k.det > 0.f && k.kappa > 0.f && isfinite(k.mx) && isfinite(k.my) &&
              isfinite(k.kappa) && isfinite(k.det);
  k.umax = k.vmax = k.vstar = 0.f;
  if (k.ellipse) {
    k.umax = fast_sqrt(__fdividef(__fmul_rn(k.kappa, k.c), k.det));
    k.vmax = fast_sqrt(__fdividef(__fmul_rn(k.kappa, k.a), k.det));
    k.vstar = __fdividef(-__fmul_rn(k.b, k.umax), k.c);
  }
  return k;
}

// The x extent (absolute pixel coordinates) of the support within the band
// y in [y0, y1]: up to two intervals [lo0, hi0] (ellipse) and [lo1, hi1]
// (filter disc); an empty interval has lo > hi.  Each end carries a margin of
// 0.02 px plus 2e-6 of its magnitude for the FP32 roots.
struct RowSpan {
  float lo0, hi0, lo1, hi1;
};

__device__ __forceinline__ float ellipse_u(const SupportConic& k, float v, float sgn) {
  const float disc = fmaxf(0.f, __fsub_rn(__fmul_rn(k.a, k.kappa), __fmul_rn(k.det, __fmul_rn(v, v))));
  return __fdividef(__fmaf_rn(sgn, fast_sqrt(disc), -__fmul_rn(k.b, v)), k.a);
}

__device__ __forceinline__ RowSpan support_row_span(const SupportConic& k, float y0, float y1, float full_lo,
                                                    float full_hi) {
  RowSpan s;
  s.lo0 = 1.f; s.hi0 = 0.f; s.lo1 = 1.f; s.hi1 = 0.f;
  const float Y0 = __fsub_rn(y0, k.cy) - 0.02f, Y1 = __fsub_rn(y1, k.cy) + 0.02f;
  if (k.ellipse) {
    const float vlo = fmaxf(__fsub_rn(Y0, k.my), -k.vmax), vhi = fminf(__fsub_rn(Y1, k.my), k.vmax);
    if (vlo <= vhi) {
      const float hi = (k.vstar >= vlo && k.vstar <= vhi) ? k.umax
                                                          : fmaxf(ellipse_u(k, vlo, 1.f), ellipse_u(k, vhi, 1.f));
      const float lo = (-k.vstar >= vlo && -k.vstar <= vhi) ? -k.umax
                                                            : fminf(ellipse_u(k, vlo, -1.f), ellipse_u(k, vhi, -1.f));
      const float xl = __fadd_rn(__fadd_rn(k.cx, k.mx), lo), xh = __fadd_rn(__fadd_rn(k.cx, k.mx), hi);
      s.lo0 = xl - (0.02f + 2e-6f * fabsf(xl));
      s.hi0 = xh + (0.02f + 2e-6f * fabsf(xh));
    }
  } else {
    s.lo0 = full_lo;  // not a proper ellipse in FP32: keep the whole candidate row
    s.hi0 = full_hi;
  }
  const float yc = fminf(fmaxf(0.f, Y0), Y1);
  const float rem = __fsub_rn(k.r2f, __fmul_rn(yc, yc));
  if (rem >= 0.f) {
    const float hw = fast_sqrt(rem);
    const float xl = __fsub_rn(k.cx, hw), xh = __fadd_rn(k.cx, hw);
    s.lo1 = xl - (0.02f + 2e-6f * fabsf(xl));
    s.hi1 = xh + (0.02f + 2e-6f * fabsf(xh));
  }
  return s;
}

// Pixel-centre rows [lo, hi] the support can reach (a superset of every band
// support_row_span finds non-empty): the filter disc and, when the support is a
// proper ellipse in FP32, the ellipse, padded by 0.1 px (0.02 px more than the
// row spans' own margin, for the rounding of the rearranged bounds) plus 1e-5 of
// their magnitude; the whole column otherwise.
__device__ __forceinline__ float2 support_rows(const float4 g0, const float4 g1, const float4 g2, float rb) {
  const SupportConic k = support_conic(g0, g1, g2, rb);
  const float rf = fast_sqrt(k.r2f);
  float lo = __fsub_rn(k.cy, rf), hi = __fadd_rn(k.cy, rf);
  if (k.ellipse) {
    const float c = __fadd_rn(k.cy, k.my);
    lo = fminf(lo, __fsub_rn(c, k.vmax));
    hi = fmaxf(hi, __fadd_rn(c, k.vmax));
  } else {
    lo = -INFINITY;
    hi = INFINITY;
  }
  const float pad = 0.1f + 1e-5f * fmaxf(fabsf(lo), fabsf(hi));
  return make_float2(lo - pad, hi + pad);
}

// Tiles [t0, t1] of a row whose pixel-centre columns i (centre i + 0.5) meet
// [lo, hi], clipped to the candidate tiles [c0, c1]; t0 > t1 if none.
__device__ __forceinline__ void span_tiles(float lo, float hi, int tw, int W, int c0, int c1, int* t0, int* t1) {
  *t0 = 1;
  *t1 = 0;
  if (!(lo <= hi)) return;
  const float ilo = fmaxf(ceilf(lo - 0.5f), 0.f), ihi = fminf(floorf(hi - 0.5f), (float)(W - 1));
  if (ilo > ihi) return;
  *t0 = max((int)ilo / tw, c0);
  *t1 = min((int)ihi / tw, c1);
}

// 8-bit log-scale code of a tile's pair count, 16 steps per octave: the
// persistent queues only need the heaviest tiles roughly first, and one 8-bit
// radix pass orders them (0 for an empty tile, increasing with the count).
__device__ __forceinline__ uint32_t work_code(uint32_t len) {
  const uint32_t x = min(len, 32767u) + 1u;
  const uint32_t e = 31u - (uint32_t)__clz(x);
  const uint32_t m = e >= 4u ? (x >> (e - 4u)) & 15u : (x << (4u - e)) & 15u;
  return e * 16u + m;
}

#ifndef OCGS_QUEUE_DROP
#define OCGS_QUEUE_DROP 4
#endif
// an empty tile (code 0) must stay behind every non-empty one (codes >= 16)
static_assert(OCGS_QUEUE_DROP >= 0 && OCGS_QUEUE_DROP <= 4, "queue key bits");
// Radix key of a tile in a persistent queue: heaviest first.  The low
// OCGS_QUEUE_DROP bits of the code are dropped (4: whole octaves of the pair
// count), so that the tiles of one weight class keep their id order (view by
// view, row by row) and neighbouring tiles, which share records, run close
// together in time.  On 500k surfels x 16 views this halved the backward's
// DRAM reads (3.53 -> 1.92 GB per launch) against the exact 8-bit code.
__device__ __forceinline__ uint32_t queue_key(uint32_t len) {
  return 255u - (work_code(len) & ~((1u << OCGS_QUEUE_DROP) - 1u));
}

// Tile runs of one row of a record's candidate rectangle: the union of the
// runs of the two intervals, as at most two disjoint runs in increasing order.
struct RowRuns {
  int a0, a1, b0, b1;  // run a = [a0, a1], run b = [b0, b1] (empty if start > end)
};

__device__ __forceinline__ RowRuns row_runs(const SupportConic& k, int ty, int tw, int th, int W, int H,
                                            const int4 rc) {
  const float y0 = (float)(ty * th) + 0.5f;
  const float y1 = (float)(min((ty + 1) * th, H) - 1) + 0.5f;
  const float full_lo = (float)(rc.x * tw) + 0.5f, full_hi = (float)(min((rc.z + 1) * tw, W) - 1) + 0.5f;
  const RowSpan sp = support_row_span(k, y0, y1, full_lo, full_hi);
  int p0, p1, q0, q1;
  span_tiles(sp.lo0, sp.hi0, tw, W, rc.x, rc.z, &p0, &p1);
  span_tiles(sp.lo1, sp.hi1, tw, W, rc.x, rc.z, &q0, &q1);
  RowRuns r;
  if (p0 > p1) { p0 = q0; p1 = q1; q0 = 1; q1 = 0; }
  if (q0 > q1) {
    r.a0 = p0; r.a1 = p1; r.b0 = 1; r.b1 = 0;
  } else if (q0 > p1 + 1 || p0 > q1 + 1) {  // disjoint: order them
    if (p0 < q0) { r.a0 = p0; r.a1 = p1; r.b0 = q0; r.b1 = q1; }
    else { r.a0 = q0; r.a1 = q1; r.b0 = p0; r.b1 = p1; }
  } else {  // overlapping or adjacent: merge
    r.a0 = min(p0, q0); r.a1 = max(p1, q1); r.b0 = 1; r.b1 = 0;
  }
  return r;
}

// Binning record of one (view, surfel), 48 contiguous bytes (3 float4) so that
// the depth-ordered gather of the binning fetches one span per record:
//   b0 = (cx, cy, rb, A00), b1 = (A01, A10, A11, e0),
//   b2 = (e1, e2, rect x | y << 16, rect z | w << 16)   (tile rect as int16)
// with rb = support_rho(o), the bound the rasterizers derive from the opacity.
struct BinView {
  float4 g0, g1, g2;  // centre / matrix / denominator terms as the record keeps them
  float rb;
  int4 rc;
};

__device__ __forceinline__ uint32_t pack_i16x2(int lo, int hi) {
  return (uint32_t)(uint16_t)(int16_t)lo | ((uint32_t)(uint16_t)(int16_t)hi << 16);
}

__device__ __forceinline__ BinView load_bin(const float4* __restrict__ bin, uint32_t r) {
  const float4* p = bin + 3 * (size_t)r;
  const float4 b0 = p[0], b1 = p[1], b2 = p[2];
  BinView v;
  v.g0 = make_float4(b0.x, b0.y, 0.f, 0.f);
  v.g1 = make_float4(b0.w, b1.x, b1.y, b1.z);
  v.g2 = make_float4(b1.w, b2.x, b2.y, 0.f);
  v.rb = b0.z;
  const uint32_t xy = __float_as_uint(b2.z), zw = __float_as_uint(b2.w);
  v.rc = make_int4((int)(int16_t)(xy & 0xffffu), (int)(int16_t)(xy >> 16), (int)(int16_t)(zw & 0xffffu),
                   (int)(int16_t)(zw >> 16));
  return v;
}

// view of a (view, Gaussian) record index r = v N + i (record indices fit 32 bits, so
// a 32-bit division does)
__device__ __forceinline__ int view_of_record(uint32_t r, int64_t n_gauss) {
  return (int)(r / (uint32_t)n_gauss);
}

// first global tile id -> view, by binary search over V+1 prefix offsets
__device__ __forceinline__ int view_of_tile(const int* tile_prefix, int n_views, int tile) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_prefix[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace ocgs

// ----------------------------------------------------------------------------- host-side launch helpers
namespace ocgs {

// process-wide count of kernels launched by this library (read by ocgs_kernel_launches)
extern std::atomic<long long> g_kernel_launches;
inline cudaError_t launched() {
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_preprocess(const GaussPtrs& g, int64_t n, int sh_degree, const DevCam* cams,
                              int n_views, int tile_w, int tile_h, RecPtrs rec, int32_t* ntiles,
                              float4* bin, uint32_t* depth_key, int* status, cudaStream_t s);

// EWA projection of 3D Gaussians (scale [n,3]) into the same record format
cudaError_t launch_preprocess_ewa(const GaussPtrs& g, int64_t n, int sh_degree, const DevCam* cams, int n_views,
                                  int tile_w, int tile_h, RecPtrs rec, int32_t* ntiles, float4* bin,
                                  uint32_t* depth_key, int* status, cudaStream_t s);
cudaError_t launch_preprocess_backward(const GaussPtrs& g, int64_t n, int sh_degree,
                                       const DevCam* cams, int n_views, const float* grad_rec,
                                       const int32_t* ntiles, GaussOut out, cudaStream_t s);

// stable LSD radix sort of (key, value) 32-bit pairs on key bits [0, n_bits)
// in ping-pong buffers; returns in *result_in_alt whether the sorted data ended
// in the alternate buffers.  scratch must hold radix_scratch_bytes(n) bytes.
size_t radix_scratch_bytes(uint32_t n);
// d_n (optional): device-side item count, read by the kernels and clamped to n
// (n sizes the launch: a capacity).  index_vals: the values are 0, 1, ..., n - 1 (the
// first pass generates them instead of reading vals, which need not be initialised)
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                             uint32_t n, int n_bits, void* scratch, bool* result_in_alt,
                             cudaStream_t s, const uint32_t* d_n = nullptr, bool index_vals = false);

// exclusive scan of n uint64 values (in may equal out); the total is written to *d_total.
size_t scan_scratch_bytes(uint32_t n);
cudaError_t scan_exclusive_u64(const uint64_t* in, uint64_t* out, uint32_t n, uint64_t* d_total,
                               void* scratch, cudaStream_t s);
cudaError_t scan_exclusive_u32(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* d_total,
                               void* scratch, cudaStream_t s);

cudaError_t launch_gather_counts(const uint32_t* order, const int32_t* ntiles, uint64_t* counts,
                                 uint32_t n, cudaStream_t s);
cudaError_t launch_iota(uint32_t* v, uint32_t n, cudaStream_t s);
// exact tile counts: ntiles[r] = tiles of rect[r] the record's support reaches
// (row_runs); a record with none gets depth key 0xffffffff so that it sorts to
// the tail
cudaError_t launch_tile_count(const float4* bin, const DevCam* cams, int64_t n_gauss, uint32_t n_rec, int tile_w,
                              int tile_h, int32_t* ntiles, uint32_t* depth_key, cudaStream_t s);
// write the (tile, record) pairs in depth order: offsets [n_rec] are the
// exclusive scan of the tile counts taken in depth order (order), total their
// sum (device); pairs at or past n_pairs are dropped
cudaError_t launch_duplicate(const uint32_t* order, const uint64_t* offsets, const uint64_t* total, uint32_t n_rec,
                             const float4* bin, const DevCam* cams, int64_t n_gauss, int tile_w, int tile_h,
                             uint32_t n_pairs, uint32_t* keys, uint32_t* vals, cudaStream_t s);
cudaError_t launch_tile_ranges(const uint32_t* keys, uint32_t n_pairs, uint2* ranges, cudaStream_t s,
                               const uint32_t* d_n = nullptr);
// n32 = min(*total, cap); raises kStatusCapacity when *total > cap
cudaError_t launch_clamp_count(const uint64_t* total, uint32_t cap, uint32_t* n32, int* status, cudaStream_t s);
// Work keys of the persistent queue: heaviest tiles first over all views, by octave
// of the pair count (queue_key; ranges2: an optional second segment of each tile's
// list, counted with the first), sorted with one 8-bit radix pass.  A strict
// view-by-view order left SMs idle at the end of each launch, each view's heavy tiles
// starting late (backward active warps 15.6 -> 14.6 per SM on a 4-view case).
cudaError_t launch_tile_order(const uint2* ranges, uint32_t n_tiles, uint32_t* work_key, uint32_t* tile_ids,
                              cudaStream_t s, const uint2* ranges2 = nullptr);

// Two-pass binning (front records first, then the records behind them into the tiles left open):
// exact tile counts of the first n entries of the depth order (counts[i], and ntiles[order[i]])
cudaError_t launch_tile_count_sorted(const uint32_t* order, uint32_t n, const float4* bin, const DevCam* cams,
                                     int64_t n_gauss, int tile_w, int tile_h, int32_t* ntiles, uint64_t* counts,
                                     cudaStream_t s);
// *out = number of entries of the ascending sorted_keys[n] below key
cudaError_t launch_count_below(const uint32_t* sorted_keys, uint32_t n, uint32_t key, uint32_t* out,
                               cudaStream_t s);
// Second pass over the n entries behind the front (order: their records in depth order).
// open_prefix [n_tiles + 1] is the exclusive prefix sum of the 0/1 open flags.
// Candidates (a screen box holding an open tile), compacted in depth order into
// cand[*n_cand]; flag and pos are [n] scratch, scratch holds scan_scratch_bytes(n).
cudaError_t launch_open_candidates(const uint32_t* order, uint32_t n, const float4* bin, const DevCam* cams,
                                   int64_t n_gauss, const uint32_t* open_prefix, uint32_t* flag, uint32_t* pos,
                                   uint32_t* cand, uint32_t* n_cand, void* scratch, cudaStream_t s);
// counts[c] = open tiles reached by candidate c (0 for c >= *n_cand; counts is [n])
cudaError_t launch_open_count(const uint32_t* cand, uint32_t n, const uint32_t* n_cand, const float4* bin,
                              const DevCam* cams, int64_t n_gauss, int tile_w, int tile_h,
                              const uint32_t* open_prefix, uint64_t* counts, cudaStream_t s);
// the (open tile, record) pairs of the candidates, in depth order, from the scan of those counts
// (open_ids: scratch of n_tiles ids, filled with the compacted open tiles first)
cudaError_t launch_duplicate_open(const uint32_t* cand, const uint64_t* offsets, const uint64_t* total,
                                  uint32_t n_rec, const uint32_t* n_cand, const float4* bin, const DevCam* cams,
                                  int64_t n_gauss, int tile_w, int tile_h, const uint32_t* open,
                                  const uint32_t* open_prefix, uint32_t n_tiles, uint32_t* open_ids, uint32_t n_pairs,
                                  uint32_t* keys, uint32_t* vals, cudaStream_t s);
// the second pass's queue: tiles with a non-empty ranges2 first (longest first);
// n_again (zeroed by the caller) counts them
cudaError_t launch_second_queue(const uint2* ranges2, uint32_t n_tiles, uint32_t* work_key, uint32_t* ids,
                                uint32_t* n_again, cudaStream_t s);

struct RasterArgs {
  int ewa;  // records are projected 3D Gaussians (preprocess_ewa)
  const DevCam* cams;
  const int* tile_prefix;   // [V+1]
  int n_views;
  int64_t n_gauss;
  uint32_t n_tiles;
  const uint2* ranges;
  const uint32_t* vals;     // sorted record indices
  RecPtrs rec;
  ImgPtrs out;
  float* t_final;           // NULL: the pass keeps no backward state
  uint32_t* last;
  float* score;
  const uint32_t* tile_order;  // persistent: tiles in work order (NULL = natural)
  uint32_t* queue;             // persistent: global tile counter (zeroed)
  int persistent_ctas;         // 0 = one CTA per tile
  const uint32_t* n_queue;     // persistent: device-side queue length (NULL = n_tiles)
  // Two-pass rendering.  First pass: open[t] is set to 1 for each tile with a
  // pixel still running at the end of its list, and done[pixel] records which
  // pixels have stopped.  Second pass: prior[t] is the tile's first-pass range;
  // the tile continues where that list ended (position prior.y - prior.x) from
  // the first pass's images, t_final, last and done.
  uint32_t* open;
  uint8_t* done;
  const uint2* prior;
};
// ppt: pixels per thread (vertically adjacent): 1 or 2, and 4 for 16-wide tiles;
// batch: records a warp stages per batch (32; also 16 and 64 for the 16-wide
// shapes with 2 or 4 pixels per thread, see OCGS_RASTER_SHAPES)
cudaError_t launch_raster_forward(const RasterArgs& a, int tile_w, int tile_h, int ppt, int batch, bool write_image,
                                  cudaStream_t s);

struct RasterBwdArgs {
  const DevCam* cams;
  const int* tile_prefix;
  int n_views;
  int64_t n_gauss;
  uint32_t n_tiles;
  const uint2* ranges;
  const uint32_t* vals;
  const uint2* ranges2;     // two-pass renders: the second segment of each tile's list (NULL: none)
  const uint32_t* vals2;
  RecPtrs rec;
  const float* t_final;
  const uint32_t* last;
  ImgPtrs d_out;            // cotangents, NULL planes = 0
  float* grad_rec;          // [V*N][kGradStride], zeroed
  const uint32_t* tile_order;
  uint32_t* queue;
  int persistent_ctas;
};
cudaError_t launch_raster_backward(const RasterBwdArgs& a, int tile_w, int tile_h, int ppt, int batch,
                                   cudaStream_t s);
// sum of the per-pixel blended-prefix lengths (the pairs both passes must evaluate)
cudaError_t launch_sum_u32(const uint32_t* v, int64_t n, unsigned long long* out, cudaStream_t s);

cudaError_t launch_background_loss(const float* alpha, const uint8_t* mask, const DevCam* cams,
                                   int n_views, const int* block_prefix, int n_blocks, float gamma,
                                   double* partial, double* loss, float* d_alpha, cudaStream_t s);
constexpr int kLossBlockPixels = 4096;

// Packed FP32x2 arithmetic: pfma / pmul / padd round each lane as the scalar
// operation does, so a pair gives two scalar results bit for bit whether it runs
// on the packed instructions of sm_100+ (__ffma2_rn, ...) or, with
// -DOCGS_SCALAR_PAIRS, as two scalar ones (measured 9-10 % slower in both
// rasterizers on 500k surfels x 16 views).
#ifdef OCGS_SCALAR_PAIRS
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
  return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
}
#else
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
#endif
__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }

// Float32 sums with the rounding error kept (FP64 runs at a small fraction of the
// FP32 rate on this part): Knuth's TwoSum gives s + err = a + b exactly, and a
// compensated sum adds each term to hi and collects the rounding errors in lo, so
// hi + lo carries about twice the float precision.  The loss kernels accumulate
// per thread this way and reduce the pairs to one FP64 partial per block.
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
struct CompSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    float err;
    hi = two_sum(hi, x, err);
    lo = __fadd_rn(lo, err);
  }
  // a term known as a float pair x + y (y far below x)
  __device__ __forceinline__ void add(float x, float y) {
    add(x);
    lo = __fadd_rn(lo, y);
  }
};

// Block totals of NV compensated sums per thread, in a fixed order: each warp's
// shuffle tree merges the pairs with two_sum, then thread 0 adds the warps' pairs
// in order in FP64.  Every thread of the NT-thread block calls it; out is written
// by thread 0.
template <int NT, int NV>
__device__ __forceinline__ void block_comp_sums(CompSum (&c)[NV], double* out) {
  static_assert(NT % 32 == 0, "whole warps");
  __shared__ float2 s_w[NT / 32][NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h = __shfl_down_sync(0xffffffffu, c[k].hi, o);
      const float l = __shfl_down_sync(0xffffffffu, c[k].lo, o);
      float err;
      c[k].hi = two_sum(c[k].hi, h, err);
      c[k].lo = __fadd_rn(__fadd_rn(c[k].lo, l), err);
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) s_w[threadIdx.x >> 5][k] = make_float2(c[k].hi, c[k].lo);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += (double)s_w[w][k].x + (double)s_w[w][k].y;
      out[k] = t;
    }
  }
}

// Per-view totals of per-block FP64 partial sums: one CTA of kViewSumThreads per
// view (blockIdx.x = view) adds NV values per block, partial[NV b + k] for the
// view's blocks [b0, b1), in a fixed order (each thread a strided run of blocks,
// then each warp's xor tree, then the warps in order), so the totals are the
// same from run to run.  The result is valid in thread 0.
constexpr int kViewSumThreads = 128;
template <int NV>
__device__ __forceinline__ void view_block_sums(const double* __restrict__ partial, int b0, int b1, double* out) {
  __shared__ double s_w[kViewSumThreads / 32][NV];
  double t[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) t[k] = 0.0;
  for (int b = b0 + (int)threadIdx.x; b < b1; b += kViewSumThreads) {
#pragma unroll
    for (int k = 0; k < NV; ++k) t[k] += partial[(int64_t)NV * b + k];
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) s_w[threadIdx.x >> 5][k] = t[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = 0.0;
      for (int w = 0; w < kViewSumThreads / 32; ++w) a += s_w[w][k];
      out[k] = a;
    }
  }
}
cudaError_t launch_masked_l1(const float* rgb, const float* target, const uint8_t* mask, const DevCam* cams,
                             int n_views, const int* block_prefix, int n_blocks, float weight, double* partial,
                             double* loss, float* d_rgb, cudaStream_t s);

cudaError_t launch_prune_flags(const float* score, uint32_t n, float threshold, uint32_t* keep,
                               uint32_t* border, cudaStream_t s);
cudaError_t launch_prune_compact(const GaussPtrs& in, uint32_t n, int sh_degree, const uint32_t* keep,
                                 const uint32_t* keep_pos, const uint32_t* border,
                                 const uint32_t* border_pos, GaussOut out, int64_t* border_idx,
                                 int64_t border_cap, cudaStream_t s);

// Adam (adam.cu): one segment per parameter array
struct AdamSeg {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t count;  // floats
  float lr;
  int vector;     // all four pointers 16-byte aligned
};
struct AdamArgs {
  AdamSeg seg[5];
  float beta1, beta2, one_m_beta1, one_m_beta2, inv_bc1, inv_bc2, eps;
  int* status;
};
cudaError_t launch_adam(const AdamArgs& a, int sm_count, cudaStream_t s);

// SSIM / PSNR (ssim.cu).  SSIM works on 32x32 output tiles per view:
// tile_prefix [n_views + 1] counts ssim_tiles(W, H) per view; partial holds 3
// doubles per tile; gmap 9 planes of p_total floats (only when d_rgb is given).
int ssim_tiles(int width, int height);
cudaError_t launch_ssim(const float* rgb, const float* target, const uint8_t* mask, const DevCam* cams, int n_views,
                        const int* tile_prefix, int n_tiles, int64_t p_total, float weight, double* partial,
                        float* gmap, double* ssim, double* ssim_masked, float* d_rgb, cudaStream_t s);
// 2DGS regularisers (regularisers.cu), over the loss blocks; partial holds one
// double per block; gmap 6 floats per pixel (normal consistency, with adjoints)
cudaError_t launch_depth_distortion(const float* alpha, const float* depth, const float* depth2, const DevCam* cams,
                                    int n_views, const int* block_prefix, int n_blocks, float weight,
                                    double* partial, double* loss, float* d_alpha, float* d_depth, float* d_depth2,
                                    cudaStream_t s);
cudaError_t launch_normal_consistency(const float* alpha, const float* depth, const float* normal, const DevCam* cams,
                                      int n_views, const int* block_prefix, int n_blocks, float weight, float a_min,
                                      double* partial, float* gmap, double* loss, float* d_alpha, float* d_depth,
                                      float* d_normal, cudaStream_t s);
// PSNR over the loss blocks (kLossBlockPixels per block); partial holds 2 doubles per block
cudaError_t launch_masked_psnr(const float* rgb, const float* target, const uint8_t* mask, const DevCam* cams,
                               int n_views, const int* block_prefix, int n_blocks, double max_i, double* partial,
                               double* psnr, cudaStream_t s);

}  // namespace ocgs
