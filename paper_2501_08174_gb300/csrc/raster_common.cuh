// Definitions shared by the forward (raster_fwd.cu) and backward
// (raster_bwd.cu) tile rasterizers: the warp's band of a tile, the evaluation
// of one surfel at two pixel centres of a column, and the launch shapes.
//
// Both passes evaluate a (pixel, surfel) candidate with the same explicitly
// rounded intrinsics, so that the backward replays every decision of the
// forward (skip, clamp, stop, surfel/filter branch) bit for bit, and the value
// at a pixel depends neither on the tile shape nor on how many pixels a
// thread owns.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace ocgs {
namespace raster {

constexpr unsigned kFull = 0xffffffffu;
// Warps per CTA.  Each warp owns one band of full tile rows (32 threads x PPT
// pixels) and walks its tile's list on its own: its own queue slot, its own
// shared-memory batches, no CTA barrier.
constexpr int kBlockWarps = 4;

// Records a warp stages in shared memory per batch: 16, 32 or 64 (the
// Gaussians-per-batch option).  32 lanes load one record each per staging
// round; 64 takes two rounds, 16 loads with half the lanes.
template <int BATCH>
struct Batch {
  static_assert(BATCH == 16 || BATCH == 32 || BATCH == 64, "batch size");
  static constexpr int kRounds = BATCH > 32 ? BATCH / 32 : 1;
  static constexpr int kLanes = BATCH < 32 ? BATCH : 32;
};

#ifdef OCGS_COUNT
// diagnostic build only: counters of warp iterations and evaluated (lane, pixel) pairs,
// one array per translation unit (g_diag, defined by each rasterizer file)
#define OCGS_DIAG(slot, v) atomicAdd(&g_diag[slot], (unsigned long long)(v))
#else
#define OCGS_DIAG(slot, v)
#endif

// The band of a warp: its pixel rows of the tile (32 threads x PPT rows) and
// the tile's columns, as pixel-centre bounds clipped to the image.
template <int TW, int TH, int PPT>
__device__ __forceinline__ float4 warp_band(const DevCam& cam, int local, int wt) {
  constexpr int kRows = (32 / TW) * PPT;
  const int x0 = (local % cam.tiles_x) * TW, y0 = (local / cam.tiles_x) * TH + ((wt * 32) / TW) * PPT;
  return make_float4((float)x0 + 0.5f, (float)(min(x0 + TW, cam.W) - 1) + 0.5f, (float)y0 + 0.5f,
                     (float)(min(y0 + kRows, cam.H) - 1) + 0.5f);
}

// CTAs of BW independent warps: persistent_ctas counts tile-sized CTAs
// (TW*TH/PPT threads), converted to the same number of warps
template <int TW, int TH, int PPT, int BW = kBlockWarps>
unsigned warp_grid(int persistent_ctas, uint32_t n_tiles) {
  constexpr uint64_t WPT = TW * TH / PPT / 32;
  const uint64_t warps = (persistent_ctas ? (uint64_t)persistent_ctas : (uint64_t)n_tiles) * WPT;
  return (unsigned)((warps + BW - 1) / BW);
}

// ----------------------------------------------------------------------------- one surfel at two pixels
// The ray-splat map of a record about its projected centre (see common.cuh):
// for (dx, dy) = x - c, u = (A00 dx + A01 dy) / den, v = (A10 dx + A11 dy) / den,
// den = e0 + e1 dx + e2 dy.  The terms that depend only on the pixel column
// are computed once per entry and thread.
struct SplatColumn {
  float dx, ux, vx, ex, dx2;
};

__device__ __forceinline__ SplatColumn splat_column(const float4 g0, const float4 g1, const float4 g2, float px) {
  SplatColumn c;
  c.dx = __fsub_rn(px, g0.x);
  c.ux = __fmul_rn(g1.x, c.dx);
  c.vx = __fmul_rn(g1.z, c.dx);
  c.ex = __fmaf_rn(g2.y, c.dx, g2.x);
  c.dx2 = __fmul_rn(c.dx, c.dx);
  return c;
}

// Two pixels of one column (rows py.x and py.y) are evaluated together as a
// pair with the packed FP32x2 helpers pfma / pmul / padd of common.cuh (each
// lane rounded as the scalar operation), so a pair gives the two scalar results
// bit for bit.
__device__ __forceinline__ float lane2(float2 v, int i) { return i ? v.y : v.x; }
__device__ __forceinline__ void set_lane2(float2& v, int i, float x) {
  if (i) v.y = x;
  else v.x = x;
}

// rb: the record's blend bound in rho.  A candidate is blended only where rho <= 9
// (the 3-sigma cut) and alpha = o exp(-rho/2) >= 1/255, i.e. rho <= 2 ln(255 o); both
// tests are the one comparison rho <= min(9, 2 ln(255 o)), computed once per record.
// Evaluated in float32 it can differ from the alpha test only where alpha is within a
// few ulps of 1/255.
__device__ __forceinline__ float blend_rho(float o) {
  return fminf(kRhoCut, __fmul_rn(2.0f, __logf(__fmul_rn(255.0f, o))));
}

// The evaluation is split so that a thread computes the cheap terms of all its pixels
// as straight-line code (head) before the rest (tail).
struct SplatHead2 {
  float2 dy, un, vn, den, rho2, q;
};

__device__ __forceinline__ SplatHead2 splat_head2(const float4 g0, const float4 g1, const float4 g2,
                                                  const SplatColumn& c, float2 py) {
  SplatHead2 h;
  h.dy = padd(py, bc2(-g0.y));
  h.un = pfma(bc2(g1.y), h.dy, bc2(c.ux));
  h.vn = pfma(bc2(g1.w), h.dy, bc2(c.vx));
  h.den = pfma(bc2(g2.z), h.dy, bc2(c.ex));
  h.rho2 = pmul(bc2(kInvSigmaF2), pfma(h.dy, h.dy, bc2(c.dx2)));
  h.q = pfma(h.un, h.un, pmul(h.vn, h.vn));
  return h;
}

// A cheap superset of the pixels a candidate can blend: the surfel term within the
// blend bound (u^2 + v^2 <= rb, tested as q <= rb den^2 with a relative margin that
// covers the rounding of rho3 = q / den^2) or the filter term within it.  Only used
// to skip an entry no pixel of the band can blend; the blend decision itself is
// taken in splat_tail2.
__device__ __forceinline__ bool may_blend(const SplatHead2& h, float rb, bool live0, bool live1) {
  const float2 lim = pmul(bc2(__fmul_rn(rb, 1.0001f)), pmul(h.den, h.den));
  return (live0 && (h.q.x <= lim.x || h.rho2.x <= rb)) || (live1 && (h.q.y <= lim.y || h.rho2.y <= rb));
}

// exp(-rho / 2) = 2^(rho * (-1 / (2 ln 2))): one multiply and the base-2 exponential of
// the special-function unit (PTX ex2.approx, relative error about 2^-22; results below
// 2^-126, where rho > 174, flush to 0, far outside every support bound).
constexpr float kNegHalfLog2e = -0.721347520444481703680f;
__device__ __forceinline__ float exp2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct SplatEval2 {
  float2 r, rho3;   // 1 / den and the surfel rho (FINITE: zeroed where the filter term won)
  float2 Gc;        // dalpha/do: G where the candidate blends below the 0.99 clamp, else 0
  float2 alpha;     // the blended opacity min(0.99, o G), 0 where the candidate is skipped
  float2 z;         // depth of the hit (surfel term) or of the centre (filter term)
  bool surf[2];     // the surfel term won the min (else the screen filter)
  bool ok[2];       // live and rho <= rb (within 3 sigma, alpha >= 1/255): blended unless the pixel stops
};

// rho = min(rho3, rho2), rho3 = (u^2 + v^2) = q / den^2: the surfel term wins where
// rho3 <= rho2 (with den = 0, rho3 is +inf or NaN and the filter term wins).
// live[i]: the pixel still composites (forward) or lies before its last blended
// entry (backward); EWA: a projected 3D Gaussian, rho = q (constant denominator,
// the screen filter already folded into its covariance), blended only where q <= rb.
// FINITE (backward): r and rho3 are zeroed where the filter term won, so that
// products the backward masks with zero stay finite (the forward reads z only).
// A skipped candidate gets alpha = 0 (T (1 - 0) = T and w = 0 exactly) and
// Gc = 0, which zeroes every term of its adjoint without further masks.
// CLAMP = false (backward): the record's o < kNoClampO, so alpha never reaches
// the clamp (see kNoClampO).
template <bool FINITE, bool EWA = false, bool CLAMP = true>
__device__ __forceinline__ SplatEval2 splat_tail2(const float4 g0, const float4 g2, const SplatHead2& h, float rb,
                                                  bool live0, bool live1) {
  SplatEval2 e;
  const float2 r = EWA ? bc2(1.0f) : make_float2(__fdividef(1.0f, h.den.x), __fdividef(1.0f, h.den.y));
  const float2 r3 = EWA ? h.q : pmul(h.q, pmul(r, r));
  e.surf[0] = EWA || r3.x <= h.rho2.x;
  e.surf[1] = EWA || r3.y <= h.rho2.y;
  if (FINITE) {
    e.r = make_float2(e.surf[0] ? r.x : 0.0f, e.surf[1] ? r.y : 0.0f);
    e.rho3 = make_float2(e.surf[0] ? r3.x : 0.0f, e.surf[1] ? r3.y : 0.0f);
  } else {
    e.r = r;
    e.rho3 = r3;
  }
  const float2 rho = make_float2(e.surf[0] ? r3.x : h.rho2.x, e.surf[1] ? r3.y : h.rho2.y);
  const float2 ex = pmul(bc2(kNegHalfLog2e), rho);
  const float2 G = make_float2(exp2_approx(ex.x), exp2_approx(ex.y));
  const float2 oG = pmul(bc2(g0.z), G);
  e.ok[0] = live0 && (rho.x <= rb);
  e.ok[1] = live1 && (rho.y <= rb);
  if (CLAMP) {
    e.alpha = make_float2(e.ok[0] ? fminf(kAlphaMax, oG.x) : 0.0f, e.ok[1] ? fminf(kAlphaMax, oG.y) : 0.0f);
    if (FINITE)
      e.Gc = make_float2(e.ok[0] && oG.x < kAlphaMax ? G.x : 0.0f, e.ok[1] && oG.y < kAlphaMax ? G.y : 0.0f);
  } else {
    e.Gc = make_float2(e.ok[0] ? G.x : 0.0f, e.ok[1] ? G.y : 0.0f);
    e.alpha = pmul(bc2(g0.z), e.Gc);  // o G where blended, o 0 = 0 elsewhere
  }
  const float2 zs = pmul(bc2(g2.w), e.r);
  e.z = make_float2(e.surf[0] ? zs.x : g0.w, e.surf[1] ? zs.y : g0.w);
  return e;
}

}  // namespace raster

// ----------------------------------------------------------------------------- launch shapes
// The tile shapes and pixels per thread the rasterizers are built for, with
// the batch sizes each shape offers (every shape has 32; the 16-wide shapes
// also 16 and 64).
#define OCGS_RASTER_SHAPES(X)                                                             \
  X(16, 16, 1, 32) X(16, 16, 2, 32) X(16, 16, 4, 32) X(16, 8, 1, 32) X(16, 8, 2, 32)     \
  X(16, 8, 4, 32) X(8, 8, 1, 32) X(8, 8, 2, 32) X(32, 8, 1, 32) X(32, 8, 2, 32)           \
  X(16, 16, 2, 16) X(16, 16, 4, 16) X(16, 8, 4, 16) X(16, 16, 2, 64) X(16, 16, 4, 64) X(16, 8, 4, 64)

}  // namespace ocgs
