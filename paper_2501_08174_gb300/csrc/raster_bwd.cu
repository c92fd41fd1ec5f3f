// Backward tile rasterizer: the reverse-order adjoint of the front-to-back
// compositing (the backpropagation through the rasterizer of Sec. 3.2).
//
// The backward walks each tile's list back to front from each pixel's last
// blended entry, recovering the transmittance T_i = T_{i+1} / (1 - alpha_i)
// from the stored final transmittance, so nothing per (pixel, Gaussian) is
// stored between the passes.  Per-Gaussian gradients are summed over the
// thread's pixels, reduced over the warp, gathered per batch in the warp's
// shared memory and added to global memory with one vector atomic per 4
// values, entry and warp.  The warp reduction of the 15 sums of a colour and
// opacity loss goes through shared memory (each lane writes its sums, then
// 30 lanes each add 16 of them and pair up with one shuffle); the 20 sums
// with depth and normal cotangents use a halving transpose of shuffles.
//
// Terms that are linear in per-entry or per-column constants are summed before
// they are multiplied: a thread sums the pixel terms of its column and scales
// the sums by the column offset dx once per entry, and the centre gradient's
// share through (u, v, den) is formed from the warp totals of the u, v and den
// terms when the batch is flushed.
#include "raster_common.cuh"

namespace ocgs {
namespace {
using namespace raster;

#ifdef OCGS_COUNT
__device__ unsigned long long g_diag[8];
#endif

// Resident warps per SM the compiler is asked to fit (caps registers per thread):
// 20 leaves 96 registers (4 bytes spilled), measured 1.4 % faster than 16 at 119
// registers on 500k surfels x 16 views
#ifndef OCGS_BWD_WARPS
#define OCGS_BWD_WARPS 20
#endif
// With depth and normal cotangents: 16 resident warps leave 128 registers (no spill;
// 20 would spill 176 bytes), measured 4.7 % faster than 12 at 151 registers on the
// 1M-surfel, 64-view iteration
#ifndef OCGS_BWD_WARPS_GEO
#define OCGS_BWD_WARPS_GEO 16
#endif
// warps per CTA of the backward (the resident-warp targets are multiples of it)
#ifndef OCGS_BWD_BLOCK_WARPS
#define OCGS_BWD_BLOCK_WARPS 4
#endif
constexpr int kBW = OCGS_BWD_BLOCK_WARPS;
static_assert(OCGS_BWD_WARPS % kBW == 0 && OCGS_BWD_WARPS_GEO % kBW == 0, "resident warps per CTA");

// One halving step of a warp transpose-reduction: lanes with bit OFF clear keep
// the first ceil(C/2) of their C values, the others keep the rest, and each
// adds the partner's copy of what it keeps.  After the steps for OFF = 16..1
// every lane holds the warp total of one slot: C + C/2 + ... shuffles in all
// instead of 5 C for independent butterflies.
template <int C, int OFF>
__device__ __forceinline__ void halve(float* v, int lane, int& base, int& real) {
  constexpr int KEEP = (C + 1) / 2;
  const bool upper = (lane & OFF) != 0;
#pragma unroll
  for (int i = 0; i < KEEP; ++i) {
    const float lo = v[i];
    const float hi = (KEEP + i < C) ? v[KEEP + i] : 0.f;
    const float got = __shfl_xor_sync(kFull, upper ? lo : hi, OFF);
    v[i] = (upper ? hi : lo) + got;
  }
  if (upper) {
    base += KEEP;
    real -= KEEP;
  } else if (real > KEEP) {
    real = KEEP;
  }
}

// Warp sum of the 20 sums; returns the one this lane holds (or -1).
__device__ __forceinline__ int warp_reduce20(float* v, int lane) {
  int base = 0, real = 20;
  halve<20, 16>(v, lane, base, real);
  halve<10, 8>(v, lane, base, real);
  halve<5, 4>(v, lane, base, real);
  halve<3, 2>(v, lane, base, real);
  halve<2, 1>(v, lane, base, real);
  return real >= 1 ? base : -1;
}

// Two sums beside the gradient slots, kept in the row's padding until the
// flush: the totals of the u and v terms, 2 dL/drho (u, v) / den^2, from
// which the flush forms the centre gradient's share through (u, v, den).
constexpr int kSumU = 18, kSumV = 19;
static_assert(kSumV < kGradStride && kGradSlots <= kSumU, "sums in the row padding");

// Sums of the 15-sum path in the order of the reduction buffer: the 13 slots,
// then the u and v totals.
constexpr int kRedSums = kGradSlotsRGB + 2;
__device__ __forceinline__ int red_target(int q) { return q < kGradSlotsRGB ? q : kSumU + (q - kGradSlotsRGB); }

// Row of one lane in the reduction buffer of the 15-sum path: 15 float2 (the
// two pixel lanes of the packed sums, not yet added).  15 is odd, so the
// 16-lane phases of the 64-bit stores (lane L writes row L) and of the 64-bit
// loads (lane L reads sum L & 15 of rows 16 (L >> 4) + i) hit distinct banks.
constexpr int kRedRow = kRedSums;
// sum 15 of the last row is read (and ignored) by lanes 15 and 31
constexpr int kRedSize = 32 * kRedRow + 1;

// Slots accumulated with the opposite sign (flipped when the lanes are summed).
__device__ __forceinline__ bool negated_slot(int q) { return q == kGe0 || q == kGe1 || q == kGe2; }

// GEO: a depth, depth2 or normal cotangent is given; without one the depth and
// normal terms of the adjoint are zero and are not evaluated (13 slots instead
// of 18, 15 sums instead of 20).
template <int TW, int TH, int PPT, int BATCH, bool GEO>
__global__ void __launch_bounds__(kBW * 32, (GEO ? OCGS_BWD_WARPS_GEO : OCGS_BWD_WARPS) / kBW)
    raster_bwd_kernel(const RasterBwdArgs a) {
  constexpr int WPT = TW * TH / PPT / 32;  // warps per tile: each owns a band of full tile rows
  constexpr int ROWS = BATCH > 32 ? BATCH / 32 : 1;  // gradient rows of a batch each lane flushes
  using B = Batch<BATCH>;
  __shared__ float4 s_g0[kBW][BATCH], s_g1[kBW][BATCH], s_g2[kBW][BATCH],
      s_a0[kBW][BATCH];
  __shared__ float2 s_a1[kBW][BATCH];
  __shared__ uint32_t s_idx[kBW][BATCH];
  __shared__ int s_q[kBW][BATCH];  // list position of each kept entry
  __shared__ __align__(16) float s_grad[kBW][BATCH * kGradStride];  // per-batch gradient sums of each entry
  __shared__ float s_rb[kBW][BATCH];
  __shared__ __align__(16) float2 s_red[kBW][GEO ? 1 : kRedSize];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    if (r * 32 + lane < BATCH) {  // a batch of 16 has rows for half the lanes
      float* row = &s_grad[wib][(r * 32 + lane) * kGradStride];
#pragma unroll
      for (int q = 0; q < kGradStride; ++q) row[q] = 0.f;
    }
  }
  // the sum this lane adds up in the 15-sum reduction, its sign and its place in the row
  const int red_slot = lane & 15;
  const float red_sign = negated_slot(red_slot) ? -1.f : 1.f;
  const int red_dst = red_target(red_slot);
  const uint32_t n_units = a.n_tiles * (uint32_t)WPT;
  for (uint32_t it = 0;; ++it) {
    // work unit: one warp's band of one tile; the warps run independently
    uint32_t unit;
    if (a.persistent_ctas) {
      uint32_t u = 0;
      if (lane == 0) u = atomicAdd(a.queue, 1u);
      unit = __shfl_sync(kFull, u, 0);
      if (unit >= n_units) break;
    } else {
      if (it > 0) break;
      unit = blockIdx.x * kBW + wib;
      if (unit >= n_units) break;
    }
    uint32_t tile = unit / WPT;
    if (a.persistent_ctas && a.tile_order) tile = a.tile_order[tile];
    const int tid = (int)(unit % WPT) * 32 + lane;  // thread of the tile
    const int lx = tid % TW, ly0 = (tid / TW) * PPT;
    const int v = view_of_tile(a.tile_prefix, a.n_views, (int)tile);
    const DevCam& cam = a.cams[v];
    const int local = (int)tile - cam.tile_offset;
    const int px = (local % cam.tiles_x) * TW + lx;
    const int py0 = (local / cam.tiles_x) * TH + ly0;
    const float pxf = (float)px + 0.5f;
    const uint2 rg1 = a.ranges[tile];
    const uint32_t start = rg1.x;
    // a two-pass list continues in the second segment after its first rg1.y - rg1.x entries
    const uint32_t len1 = a.ranges2 ? rg1.y - rg1.x : 0xffffffffu;
    const uint32_t start2 = a.ranges2 ? a.ranges2[tile].x : 0u;
    // pixel k of this thread is lane (k & 1) of pair k / 2 (an odd PPT leaves an idle lane)
    constexpr int NP = (PPT + 1) / 2;
    float2 T[NP], gAT[NP], S[NP];
    float2 gC0[NP], gC1[NP], gC2[NP], gD[NP], gN0[NP], gN1[NP], gN2[NP], gQ[NP];
    uint32_t last[2 * NP];
    uint32_t thread_last = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      T[p] = bc2(1.f);
      gAT[p] = bc2(0.f);
      S[p] = bc2(0.f);  // sum over later blended entries of w * (gC.rgb + gD z + gN.n)
      gC0[p] = gC1[p] = gC2[p] = gD[p] = gN0[p] = gN1[p] = gN2[p] = gQ[p] = bc2(0.f);
    }
#pragma unroll
    for (int k = 0; k < 2 * NP; ++k) {
      last[k] = 0u;
      const int py = py0 + k;
      const int p = k >> 1, i = k & 1;
      if (k < PPT && px < cam.W && py < cam.H) {
        const int64_t pix = cam.pix_offset + (int64_t)py * cam.W + px;
        const float Tf = a.t_final[pix];
        set_lane2(T[p], i, Tf);
        last[k] = a.last[pix];
        if (a.d_out.rgb) {
          set_lane2(gC0[p], i, a.d_out.rgb[3 * pix]);
          set_lane2(gC1[p], i, a.d_out.rgb[3 * pix + 1]);
          set_lane2(gC2[p], i, a.d_out.rgb[3 * pix + 2]);
        }
        if (a.d_out.alpha) set_lane2(gAT[p], i, a.d_out.alpha[pix] * Tf);
        if (GEO && a.d_out.depth) set_lane2(gD[p], i, a.d_out.depth[pix]);
        if (GEO && a.d_out.depth2) set_lane2(gQ[p], i, a.d_out.depth2[pix]);
        if (GEO && a.d_out.normal) {
          set_lane2(gN0[p], i, a.d_out.normal[3 * pix]);
          set_lane2(gN1[p], i, a.d_out.normal[3 * pix + 1]);
          set_lane2(gN2[p], i, a.d_out.normal[3 * pix + 2]);
        }
        thread_last = max(thread_last, last[k]);
      }
    }
    // entries at or beyond the warp's largest last index are idle for every lane
    const int warp_last = (int)__reduce_max_sync(kFull, thread_last);
    const float4 band = warp_band<TW, TH, PPT>(cam, local, (int)(unit % WPT));
    for (int bend = warp_last; bend > 0; bend -= BATCH) {
      const int bstart = max(0, bend - BATCH);
      __syncwarp();  // the previous batch is consumed and flushed
      // a batch of the list, ending at bend; keep (in order) the entries whose rows meet the band
      int cnt = 0;
#pragma unroll
      for (int r = 0; r < B::kRounds; ++r) {
        const int q = bstart + r * 32 + lane;
        bool keep = false;
        uint32_t idx = 0;
        float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < B::kLanes && q < bend) {
          idx = (uint32_t)q < len1 ? a.vals[start + q] : a.vals2[start2 + ((uint32_t)q - len1)];
          a1 = a.rec.a1[idx];
          keep = a1.w >= band.z && a1.z <= band.w;
        }
        const unsigned km = __ballot_sync(kFull, keep);
        if (keep) {
          const int slot = cnt + __popc(km & lt);
          const float4 g0 = a.rec.g0[idx];
          s_g0[wib][slot] = g0;
          s_g1[wib][slot] = a.rec.g1[idx];
          s_g2[wib][slot] = a.rec.g2[idx];
          s_a0[wib][slot] = a.rec.a0[idx];
          s_a1[wib][slot] = make_float2(a1.x, a1.y);
          s_rb[wib][slot] = blend_rho(g0.z);
          s_idx[wib][slot] = idx;
          s_q[wib][slot] = q;
        }
        cnt += __popc(km);
      }
      __syncwarp();
      for (int j = cnt - 1; j >= 0; --j) {
        const int jj = s_q[wib][j];
#ifdef OCGS_COUNT
        if (lane == 0) OCGS_DIAG(2, 1);
#endif
        // every entry of the walk lies before warp_last, so some lane has jj < its
        // last index; the support test of all pixels runs as straight-line code
        const float4 g0 = s_g0[wib][j], g1 = s_g1[wib][j], g2 = s_g2[wib][j];
        const float rb = s_rb[wib][j];
        const SplatColumn col = splat_column(g0, g1, g2, pxf);
        SplatHead2 hd[NP];
        bool live[2 * NP];
        bool any = false;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float2 py = make_float2((float)(py0 + 2 * p) + 0.5f, (float)(py0 + 2 * p + 1) + 0.5f);
          hd[p] = splat_head2(g0, g1, g2, col, py);
          live[2 * p] = jj < (int)last[2 * p];
          live[2 * p + 1] = jj < (int)last[2 * p + 1];
          any = any || may_blend(hd[p], rb, live[2 * p], live[2 * p + 1]);
        }
        if (!__any_sync(kFull, any)) continue;  // the support misses every pixel of the band
#ifdef OCGS_COUNT
        if (lane == 0) OCGS_DIAG(5, 1);  // entries evaluated in full
#endif
        const float4 ap = s_a0[wib][j];
        const float2 an = s_a1[wib][j];
        const float2 no = bc2(-g0.z);  // 2 dalpha/drho = -alpha = -o G
        // this thread's sums (one lane per pixel of a pair): the slots of the
        // record gradient, and the u and v totals in kSumU, kSumV.  The dx-scaled
        // slots (A00, A10, e1, and the filter term of cx) hold their pixel sums
        // until the column offset is applied after the pairs.
        float2 acc[kGradStride];
#pragma unroll
        for (int q = 0; q < kGradStride; ++q) acc[q] = bc2(0.f);
        bool contrib = false;
        // no per-pair branch: a candidate that is not blended has alpha = 0 and
        // Gc = 0, which makes its weight and every term of its adjoint exactly 0
        auto pairs = [&](auto clamp) {
          constexpr bool CLAMP = decltype(clamp)::value;
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const SplatEval2 e = splat_tail2<true, false, CLAMP>(g0, g2, hd[p], rb, live[2 * p], live[2 * p + 1]);
            contrib = contrib || e.ok[0] || e.ok[1];
#ifdef OCGS_COUNT
            OCGS_DIAG(6, (e.ok[0] ? 1 : 0) + (e.ok[1] ? 1 : 0));  // (pixel, entry) blends
#endif
            // undo the entry: T before it, its weight, and dL/dalpha
            const float2 om = pfma(e.alpha, bc2(-1.f), bc2(1.f));  // 1 - alpha
            const float2 inv = make_float2(__fdividef(1.f, om.x), __fdividef(1.f, om.y));
            const float2 Ti = pmul(T[p], inv);
            const float2 w = pmul(e.alpha, Ti);
            float2 F = pmul(gC0[p], bc2(ap.x));
            F = pfma(gC1[p], bc2(ap.y), F);
            F = pfma(gC2[p], bc2(ap.z), F);
            if (GEO) {
              F = pfma(gD[p], e.z, F);
              F = pfma(pmul(gQ[p], e.z), e.z, F);  // d(sum w z^2)/dw = z^2
              F = pfma(gN0[p], bc2(ap.w), F);
              F = pfma(gN1[p], bc2(an.x), F);
              F = pfma(gN2[p], bc2(an.y), F);
            }
            // dL/dalpha = T_i F + (gAT - S) / (1 - alpha)
            const float2 ga = pfma(Ti, F, pmul(pfma(S[p], bc2(-1.f), gAT[p]), inv));
            S[p] = pfma(w, F, S[p]);
            // a skipped candidate has alpha = 0, and the fast reciprocal of 1 - 0 is exactly 1
            // on this GPU (checked at 1, 2 and 0.5), so T passes through it unchanged
            T[p] = Ti;
            acc[kGr] = pfma(gC0[p], w, acc[kGr]);
            acc[kGg] = pfma(gC1[p], w, acc[kGg]);
            acc[kGb] = pfma(gC2[p], w, acc[kGb]);
            if (GEO) {
              acc[kGnx] = pfma(gN0[p], w, acc[kGnx]);
              acc[kGny] = pfma(gN1[p], w, acc[kGny]);
              acc[kGnz] = pfma(gN2[p], w, acc[kGnz]);
            }
            // alpha = o G below the clamp: dalpha/do = G, dalpha/drho = -o G / 2
            // (Gc is 0 at the clamp and for skipped candidates); gs2 = 2 dL/drho
            const float2 gop = pmul(ga, e.Gc);
            acc[kGo] = padd(acc[kGo], gop);
            const float2 gs2 = pmul(gop, no);
            // rho and depth came from the surfel's (u, v) where it won the min, from the
            // screen-space filter elsewhere.  e.r and e.rho3 are 0 where the filter won,
            // so the surfel terms below vanish there without a mask.
            const float2 gf2 = make_float2(e.surf[0] ? 0.f : gs2.x, e.surf[1] ? 0.f : gs2.y);
            float2 gzs = bc2(0.f);
            if (GEO) {
              // d/dz of w (gD z + gQ z^2)
              const float2 gz = pmul(pfma(pmul(bc2(2.f), gQ[p]), e.z, gD[p]), w);
              gzs = make_float2(e.surf[0] ? gz.x : 0.f, e.surf[1] ? gz.y : 0.f);
              acc[kGzc] = padd(acc[kGzc], pfma(gzs, bc2(-1.f), gz));
              acc[kGzD] = pfma(gzs, e.r, acc[kGzD]);
            }
            // 2 grho / den^2, shared by the u, v and den terms (rho3 = q / den^2)
            const float2 t = pmul(gs2, pmul(e.r, e.r));
            const float2 gun = pmul(t, hd[p].un);
            const float2 gvn = pmul(t, hd[p].vn);
            // -dL/dden = (2 grho rho3 + gz z) / den; the e slots accumulate negated and
            // are flipped when the lanes are summed
            const float2 ngden = GEO ? pmul(pfma(gs2, e.rho3, pmul(gzs, e.z)), e.r)
                                     : pmul(t, pmul(hd[p].q, e.r));
            acc[kSumU] = padd(acc[kSumU], gun);
            acc[kSumV] = padd(acc[kSumV], gvn);
            acc[kGA01] = pfma(gun, hd[p].dy, acc[kGA01]);
            acc[kGA11] = pfma(gvn, hd[p].dy, acc[kGA11]);
            acc[kGe0] = padd(acc[kGe0], ngden);
            acc[kGe2] = pfma(ngden, hd[p].dy, acc[kGe2]);
            // the filter term: d rho2 / d(c) = -4 (x - c) with rho2 = 2 |x - c|^2 (the
            // factor -2 and dx are applied later)
            acc[kGcx] = padd(acc[kGcx], gf2);
            acc[kGcy] = pfma(gf2, hd[p].dy, acc[kGcy]);
          }
        };
        if (g0.z < kNoClampO) pairs(std::false_type{});
        else pairs(std::true_type{});
        if (!__any_sync(kFull, contrib)) continue;  // no pixel of the band blends it
#ifdef OCGS_COUNT
        if (lane == 0) OCGS_DIAG(3, 1);
        OCGS_DIAG(4, contrib ? 1 : 0);
#endif
        // the column offset of this thread's pixels
        const float2 dx = bc2(col.dx);
        acc[kGA00] = pmul(acc[kSumU], dx);
        acc[kGA10] = pmul(acc[kSumV], dx);
        acc[kGe1] = pmul(acc[kGe0], dx);
        acc[kGcx] = pmul(acc[kGcx], dx);
        if (GEO) {
          float gr[kGradStride];
#pragma unroll
          for (int q = 0; q < kGradStride; ++q)
            gr[q] = negated_slot(q) ? -__fadd_rn(acc[q].x, acc[q].y) : __fadd_rn(acc[q].x, acc[q].y);
          const int slot = warp_reduce20(gr, lane);
          if (slot >= 0) s_grad[wib][j * kGradStride + slot] = gr[0];  // one lane per slot
        } else {
          // through shared memory: lane L's row holds its 15 packed sums; lane L then adds
          // sum L & 15 over the rows 16 (L >> 4) .. 16 (L >> 4) + 15, both pixel lanes
          float2* red = s_red[wib];
#pragma unroll
          for (int q = 0; q < kRedSums; ++q) red[lane * kRedRow + q] = acc[red_target(q)];
          __syncwarp();
          // four independent partial sums keep the dependent chain short
          const float2* col = red + (lane >> 4) * 16 * kRedRow + red_slot;
          float2 s4[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) s4[i] = col[i * kRedRow];
#pragma unroll
          for (int i = 4; i < 16; ++i) s4[i & 3] = padd(s4[i & 3], col[i * kRedRow]);
          const float2 sum = padd(padd(s4[0], s4[1]), padd(s4[2], s4[3]));
          float tot = __fadd_rn(sum.x, sum.y);
          tot = __fadd_rn(tot, __shfl_xor_sync(kFull, tot, 16));
          if (lane < kRedSums) s_grad[wib][j * kGradStride + red_dst] = tot * red_sign;
          __syncwarp();  // the rows are read before the next entry writes them
        }
      }
      // flush the batch: complete the centre gradient, then one vector atomic per
      // 4 slots and entry for the warp
      __syncwarp();
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const int e = r * 32 + lane;
        if (e < cnt) {
          float* rs = &s_grad[wib][e * kGradStride];
          // dL/dc = -2 x the filter sums, minus the totals of dL/du, dL/dv and dL/dden times
          // the coefficients with which x - c enters u, v and den (g1.x, g1.z, g2.y for the
          // x offset; g1.y, g1.w, g2.z for y); the e0 slot holds the dL/dden total
          const float4 g1 = s_g1[wib][e], g2 = s_g2[wib][e];
          const float su = rs[kSumU], sv = rs[kSumV], se = rs[kGe0];
          rs[kGcx] = -2.f * rs[kGcx] - g2.y * se - g1.z * sv - g1.x * su;
          rs[kGcy] = -2.f * rs[kGcy] - g2.z * se - g1.w * sv - g1.y * su;
          rs[kSumU] = 0.f;
          rs[kSumV] = 0.f;
          float4* row = reinterpret_cast<float4*>(rs);
          float4* dst = reinterpret_cast<float4*>(a.grad_rec + (size_t)s_idx[wib][e] * kGradStride);
#pragma unroll
          for (int q = 0; q < kGradStride / 4; ++q) {
            const float4 g4 = row[q];
            if (g4.x != 0.f || g4.y != 0.f || g4.z != 0.f || g4.w != 0.f) {
              atomicAdd(dst + q, g4);
              row[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
          }
        }
      }
    }
  }
}

template <int TW, int TH, int PPT, int BATCH>
cudaError_t bwd_dispatch(const RasterBwdArgs& a, cudaStream_t s) {
  const unsigned grid = warp_grid<TW, TH, PPT, kBW>(a.persistent_ctas, a.n_tiles);
  if (grid == 0) return cudaSuccess;
  if (a.d_out.depth || a.d_out.normal || a.d_out.depth2)
    raster_bwd_kernel<TW, TH, PPT, BATCH, true><<<grid, kBW * 32, 0, s>>>(a);
  else raster_bwd_kernel<TW, TH, PPT, BATCH, false><<<grid, kBW * 32, 0, s>>>(a);
  return launched();
}

}  // namespace

#ifdef OCGS_COUNT
extern "C" int ocgs_diag_read_bwd(unsigned long long* out, int reset) {
  cudaMemcpyFromSymbol(out, g_diag, sizeof(g_diag));
  if (reset) {
    unsigned long long z[8] = {0};
    cudaMemcpyToSymbol(g_diag, z, sizeof(z));
  }
  return 0;
}
#endif

cudaError_t launch_raster_backward(const RasterBwdArgs& a, int tile_w, int tile_h, int ppt, int batch,
                                   cudaStream_t s) {
#define OCGS_BWD(W, H, K, BT) \
  if (tile_w == W && tile_h == H && ppt == K && batch == BT) return bwd_dispatch<W, H, K, BT>(a, s);
  OCGS_RASTER_SHAPES(OCGS_BWD)
#undef OCGS_BWD
  return cudaErrorInvalidValue;
}

}  // namespace ocgs
