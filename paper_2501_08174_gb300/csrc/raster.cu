// Tile rasterizer: front-to-back compositing (forward) and its reverse-order
// adjoint (backward).
//
// A warp owns one band of a screen tile (32 threads x PPT vertically adjacent
// pixels each: full tile rows) and walks the tile's sorted (depth, Gaussian)
// list on its own, with no CTA barrier: its own slot of the persistent queue,
// its own shared-memory batches of one record per lane.  Every lane evaluates
// the batch against its pixel centres, so one shared-memory read of a record
// (and, in the backward, one warp reduction of its gradient) serves PPT
// pixels; the forward first drops, in order, the entries whose support misses
// the band.  Compositing of a pixel stops at the first blended candidate that
// would bring its transmittance below 1e-4 (Sec. 4.3: rendering ends once the
// pixel reaches an opacity close to 1), and a warp stops once all its pixels
// have stopped.  The forward optionally records, for each Gaussian, the max
// blending weight over the pixels where it was blended (the per-Gaussian
// visibility record that Sec. 4.3 and Sec. 5.1 keep while colours accumulate),
// with one warp max-reduction and at most one atomic per warp.
//
// The backward walks the same list back to front from each pixel's last
// blended entry, recovering the transmittance T_i = T_{i+1} / (1 - alpha_i)
// from the stored final transmittance, so nothing per (pixel, Gaussian) is
// stored between the passes.  Per-Gaussian gradients are summed over the
// thread's pixels, reduced over the warp with a halving transpose (about 20
// shuffles for 18 values), gathered per batch in the warp's shared memory and
// added to global memory with one vector atomic per 4 values, entry and warp.
#include "common.cuh"

namespace ocgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// Warps per CTA.  Each warp owns one band of full tile rows (32 threads x PPT
// pixels) and walks its tile's list on its own: its own queue slot, its own
// shared-memory batches, no CTA barrier.
constexpr int kBlockWarps = 4;

#ifdef OCGS_COUNT
// diagnostic build only: warp iterations and evaluated (lane, pixel) pairs
__device__ unsigned long long g_diag[8];
#define OCGS_DIAG(slot, v) atomicAdd(&g_diag[slot], (unsigned long long)(v))
#else
#define OCGS_DIAG(slot, v)
#endif

// Resident warps per SM the compiler is asked to fit (caps registers per thread);
// the forward with the Q plane and the backward with depth and normal
// cotangents keep more registers.
#ifndef OCGS_FWD_WARPS
#define OCGS_FWD_WARPS 24
#endif
#ifndef OCGS_FWD_WARPS_Q2
#define OCGS_FWD_WARPS_Q2 20
#endif
#ifndef OCGS_BWD_WARPS
#define OCGS_BWD_WARPS 16
#endif
#ifndef OCGS_BWD_WARPS_GEO
#define OCGS_BWD_WARPS_GEO 12
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

// Q2: also accumulate Q = sum w z^2 (the depth distortion's third plane)
// EWA: the records are projected 3D Gaussians (the 3DGS variant of Appendix B)
template <int TW, int TH, int PPT, bool IMG, bool SCORE, bool Q2, bool EWA>
__global__ void __launch_bounds__(kBlockWarps * 32, (Q2 ? OCGS_FWD_WARPS_Q2 : OCGS_FWD_WARPS) / kBlockWarps)
    raster_fwd_kernel(const RasterArgs a) {
  constexpr int WPT = TW * TH / PPT / 32;  // warps per tile: each owns a band of full tile rows
  __shared__ float4 s_g0[kBlockWarps][32], s_g1[kBlockWarps][32], s_g2[kBlockWarps][32], s_a0[kBlockWarps][32];
  __shared__ float2 s_a1[kBlockWarps][32];
  __shared__ uint32_t s_gid[kBlockWarps][32];
  __shared__ uint32_t s_pos[kBlockWarps][32];  // list index of each kept entry
  __shared__ float s_rb[kBlockWarps][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t n_units = (a.n_queue ? *a.n_queue : a.n_tiles) * (uint32_t)WPT;
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
      unit = blockIdx.x * kBlockWarps + wib;
      if (unit >= n_units) break;
    }
    uint32_t tile = unit / WPT;
    if (a.persistent_ctas && a.tile_order) tile = a.tile_order[tile];
    const int tid = (int)(unit % WPT) * 32 + lane;  // thread of the tile
    const int lx = tid % TW, ly0 = (tid / TW) * PPT;  // this thread's column and first of PPT rows
    const int v = view_of_tile(a.tile_prefix, a.n_views, (int)tile);
    const DevCam& cam = a.cams[v];
    const int local = (int)tile - cam.tile_offset;
    const int px = (local % cam.tiles_x) * TW + lx;
    const int py0 = (local / cam.tiles_x) * TH + ly0;
    const float pxf = (float)px + 0.5f;
    const uint2 rg = a.ranges[tile];
    const uint32_t start = rg.x, end = rg.y;
    const int64_t gbase = (int64_t)v * a.n_gauss;
    // pixel k of this thread is lane (k & 1) of pair k / 2; an odd PPT leaves a
    // dummy lane that starts done
    constexpr int NP = (PPT + 1) / 2;
    float2 T[NP], c0[NP], c1[NP], c2[NP], dep[NP], n0[NP], n1[NP], n2[NP], qz[NP];
    uint32_t last[2 * NP];
    bool done[2 * NP];
    bool alldone = true;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      T[p] = bc2(1.f);
      c0[p] = c1[p] = c2[p] = dep[p] = n0[p] = n1[p] = n2[p] = qz[p] = bc2(0.f);
    }
#pragma unroll
    for (int k = 0; k < 2 * NP; ++k) {
      last[k] = 0u;
      done[k] = !(k < PPT && px < cam.W && py0 + k < cam.H);
    }
    uint32_t pos0 = 0u;  // list position before this pass's first entry
    if (a.prior) {
      // second pass: continue each pixel from the end of the tile's first-pass list
      const uint2 pr = a.prior[tile];
      pos0 = pr.y - pr.x;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (!done[k]) {
          const int64_t pix = cam.pix_offset + (int64_t)(py0 + k) * cam.W + px;
          const int p = k >> 1, i = k & 1;
          set_lane2(T[p], i, a.t_final[pix]);
          if (IMG) {
            set_lane2(c0[p], i, a.out.rgb[3 * pix]);
            set_lane2(c1[p], i, a.out.rgb[3 * pix + 1]);
            set_lane2(c2[p], i, a.out.rgb[3 * pix + 2]);
            set_lane2(dep[p], i, a.out.depth[pix]);
            if (Q2) set_lane2(qz[p], i, a.out.depth2[pix]);
            set_lane2(n0[p], i, a.out.normal[3 * pix]);
            set_lane2(n1[p], i, a.out.normal[3 * pix + 1]);
            set_lane2(n2[p], i, a.out.normal[3 * pix + 2]);
          }
          if (a.last) last[k] = a.last[pix];
          done[k] = a.done[pix] != 0;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 2 * NP; ++k) alldone = alldone && done[k];
    const float4 band = warp_band<TW, TH, PPT>(cam, local, (int)(unit % WPT));
    for (uint32_t b0 = start; b0 < end; b0 += 32) {
      if (__all_sync(kFull, alldone)) break;
      const uint32_t kk = b0 + lane;
      // a batch of the list; keep (in order) the entries whose rows meet this warp's band
      bool keep = false;
      uint32_t idx = 0;
      if (kk < end) {
        idx = a.vals[kk];
        const float4 a1 = a.rec.a1[idx];
        keep = a1.w >= band.z && a1.z <= band.w;
      }
      const unsigned km = __ballot_sync(kFull, keep);
      const int slot = __popc(km & lt);
      __syncwarp();  // the previous batch is consumed
      if (keep) {
        const float4 g0 = a.rec.g0[idx];
        s_g0[wib][slot] = g0;
        s_g1[wib][slot] = a.rec.g1[idx];
        s_g2[wib][slot] = a.rec.g2[idx];
        if (IMG) {
          const float4 a1 = a.rec.a1[idx];
          s_a0[wib][slot] = a.rec.a0[idx];
          s_a1[wib][slot] = make_float2(a1.x, a1.y);
        }
        s_rb[wib][slot] = support_rho(g0.z);
        s_pos[wib][slot] = kk;
        if (SCORE) s_gid[wib][slot] = (uint32_t)((int64_t)idx - gbase);
      }
      __syncwarp();
      const int cnt = __popc(km);
      for (int j = 0; j < cnt; ++j) {
        if ((j & 7) == 0 && __all_sync(kFull, alldone)) break;
        float wmax = 0.f;
#ifdef OCGS_COUNT
        if (lane == 0) OCGS_DIAG(0, 1);
        {
          int act = 0;
#pragma unroll
          for (int k = 0; k < 2 * NP; ++k) act += done[k] ? 0 : 1;
          OCGS_DIAG(1, act);
        }
#endif
        if (!alldone) {
          const float4 g0 = s_g0[wib][j], g1 = s_g1[wib][j], g2 = s_g2[wib][j];
          const float rb = s_rb[wib][j];
          const SplatColumn col = splat_column(g0, g1, g2, pxf);
          float4 ap = make_float4(0.f, 0.f, 0.f, 0.f);
          float2 an = make_float2(0.f, 0.f);
          if (IMG) {
            ap = s_a0[wib][j];
            an = s_a1[wib][j];
          }
          const uint32_t pos = pos0 + s_pos[wib][j] - start + 1u;
          // every pair is evaluated without a per-pair branch: lanes that do not
          // blend are masked to exact zeros below, and straight-line code lets the
          // pairs' dependency chains interleave
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const int k0 = 2 * p, k1 = 2 * p + 1;
            const float2 py = make_float2((float)(py0 + k0) + 0.5f, (float)(py0 + k1) + 0.5f);
            SplatHead2 h = splat_head2<EWA>(g0, g1, g2, col, py, rb);
            // a surfel pixel outside the support bound fails the tail's rho <= rb test
            // on its own (rho is then the filter term rho2 > rb), so the head's pass
            // flag only needs the stop state here; the EWA support is in3 alone
            h.pass[0] = (EWA ? h.pass[0] : true) && !done[k0];
            h.pass[1] = (EWA ? h.pass[1] : true) && !done[k1];
            const SplatEval2 e = splat_tail2<false, EWA>(g0, g2, h, rb);
            // lanes that do not blend take alpha 0: T (1 - 0) = T and w = 0 exactly
            const float2 a2 = make_float2(e.ok[0] ? e.alpha.x : 0.f, e.ok[1] ? e.alpha.y : 0.f);
            float2 Tn = __fmul2_rn(T[p], __ffma2_rn(a2, bc2(-1.f), bc2(1.f)));  // T (1 - alpha)
            float2 w = __fmul2_rn(a2, T[p]);
            const uint32_t l0 = last[k0], l1 = last[k1];
            if (e.ok[0]) last[k0] = pos;
            if (e.ok[1]) last[k1] = pos;
            if (Tn.x < kTEps || Tn.y < kTEps) {
              // rare: an entry that would take T below kTEps ends the pixel unblended
              if (Tn.x < kTEps) { done[k0] = true; w.x = 0.f; Tn.x = T[p].x; last[k0] = l0; }
              if (Tn.y < kTEps) { done[k1] = true; w.y = 0.f; Tn.y = T[p].y; last[k1] = l1; }
            }
            if (IMG) {
              c0[p] = __ffma2_rn(w, bc2(ap.x), c0[p]);
              c1[p] = __ffma2_rn(w, bc2(ap.y), c1[p]);
              c2[p] = __ffma2_rn(w, bc2(ap.z), c2[p]);
              dep[p] = __ffma2_rn(w, e.z, dep[p]);
              if (Q2) qz[p] = __ffma2_rn(__fmul2_rn(w, e.z), e.z, qz[p]);
              n0[p] = __ffma2_rn(w, bc2(ap.w), n0[p]);
              n1[p] = __ffma2_rn(w, bc2(an.x), n1[p]);
              n2[p] = __ffma2_rn(w, bc2(an.y), n2[p]);
            }
            T[p] = Tn;
            wmax = fmaxf(wmax, fmaxf(w.x, w.y));
          }
          alldone = true;
#pragma unroll
          for (int k = 0; k < 2 * NP; ++k) alldone = alldone && done[k];
        }
        if (SCORE) {
          // one global max per entry and warp (non-negative floats order like their bits)
          const unsigned m = __reduce_max_sync(kFull, __float_as_uint(wmax));
          if (lane == 0 && m != 0u) atomicMax(reinterpret_cast<unsigned*>(a.score) + s_gid[wib][j], m);
        }
      }
    }
    if (a.open) {
      // the tile stays open if a pixel of any of its warps has not stopped within its list
      if (__any_sync(kFull, !alldone) && lane == 0) a.open[tile] = 1u;
      if (!IMG) {
        // a pass without images keeps only what the continuation needs: T and the stop flags
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (px < cam.W && py0 + k < cam.H) {
            const int64_t pix = cam.pix_offset + (int64_t)(py0 + k) * cam.W + px;
            a.t_final[pix] = lane2(T[k >> 1], k & 1);
            a.done[pix] = done[k] ? 1 : 0;
          }
        }
      }
    }
    if (IMG) {
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const int py = py0 + k;
        const int p = k >> 1, i = k & 1;
        if (px < cam.W && py < cam.H) {
          const int64_t pix = cam.pix_offset + (int64_t)py * cam.W + px;
          const float Tk = lane2(T[p], i);
          a.out.rgb[3 * pix + 0] = lane2(c0[p], i);
          a.out.rgb[3 * pix + 1] = lane2(c1[p], i);
          a.out.rgb[3 * pix + 2] = lane2(c2[p], i);
          a.out.alpha[pix] = 1.f - Tk;
          a.out.depth[pix] = lane2(dep[p], i);
          if (Q2) a.out.depth2[pix] = lane2(qz[p], i);
          a.out.normal[3 * pix + 0] = lane2(n0[p], i);
          a.out.normal[3 * pix + 1] = lane2(n1[p], i);
          a.out.normal[3 * pix + 2] = lane2(n2[p], i);
          if (a.t_final) {  // the backward's state, when the pass keeps it
            a.t_final[pix] = Tk;
            a.last[pix] = last[k];
          }
          if (a.open) a.done[pix] = done[k] ? 1 : 0;
        }
      }
    }
  }
}

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

// Warp sum of C gradient slots (18, or 13 without depth and normal cotangents);
// returns the slot this lane holds (or -1).
template <int C>
__device__ __forceinline__ int warp_reduce(float* v, int lane) {
  static_assert(C == 18 || C == 13, "slot count");
  int base = 0, real = C;
  if (C == 18) {
    halve<18, 16>(v, lane, base, real);
    halve<9, 8>(v, lane, base, real);
    halve<5, 4>(v, lane, base, real);
    halve<3, 2>(v, lane, base, real);
    halve<2, 1>(v, lane, base, real);
  } else {
    halve<13, 16>(v, lane, base, real);
    halve<7, 8>(v, lane, base, real);
    halve<4, 4>(v, lane, base, real);
    halve<2, 2>(v, lane, base, real);
    halve<1, 1>(v, lane, base, real);
  }
  return real >= 1 ? base : -1;
}

// GEO: a depth, depth2 or normal cotangent is given; without one the depth and
// normal terms of the adjoint are zero and are not evaluated (13 slots instead
// of 18).
template <int TW, int TH, int PPT, bool GEO>
__global__ void __launch_bounds__(kBlockWarps * 32, (GEO ? OCGS_BWD_WARPS_GEO : OCGS_BWD_WARPS) / kBlockWarps) raster_bwd_kernel(const RasterBwdArgs a) {
  constexpr int WPT = TW * TH / PPT / 32;  // warps per tile: each owns a band of full tile rows
  constexpr int NG = GEO ? kGradSlots : kGradSlotsRGB;
  __shared__ float4 s_g0[kBlockWarps][32], s_g1[kBlockWarps][32], s_g2[kBlockWarps][32], s_a0[kBlockWarps][32];
  __shared__ float2 s_a1[kBlockWarps][32];
  __shared__ uint32_t s_idx[kBlockWarps][32];
  __shared__ int s_q[kBlockWarps][32];  // list position of each kept entry
  __shared__ __align__(16) float s_grad[kBlockWarps][32 * kGradStride];  // per-batch gradient sums of each entry
  __shared__ float s_rb[kBlockWarps][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  float* const grow = &s_grad[wib][lane * kGradStride];  // this lane's entry row of a batch
#pragma unroll
  for (int q = 0; q < kGradStride; ++q) grow[q] = 0.f;
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
      unit = blockIdx.x * kBlockWarps + wib;
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
    const int warp_last = (int)__reduce_max_sync(kFull, thread_last);  // entries beyond it are idle for this warp
    const float4 band = warp_band<TW, TH, PPT>(cam, local, (int)(unit % WPT));
    for (int bend = warp_last; bend > 0; bend -= 32) {
      const int bstart = max(0, bend - 32);
      // a batch of the list, ending at bend; keep (in order) the entries whose rows meet the band
      bool keep = false;
      uint32_t idx = 0;
      float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (bstart + lane < bend) {
        const uint32_t q = (uint32_t)(bstart + lane);
        idx = q < len1 ? a.vals[start + q] : a.vals2[start2 + (q - len1)];
        a1 = a.rec.a1[idx];
        keep = a1.w >= band.z && a1.z <= band.w;
      }
      const unsigned km = __ballot_sync(kFull, keep);
      const int slot = __popc(km & lt);
      __syncwarp();  // the previous batch is consumed and flushed
      if (keep) {
        const float4 g0 = a.rec.g0[idx];
        s_g0[wib][slot] = g0;
        s_g1[wib][slot] = a.rec.g1[idx];
        s_g2[wib][slot] = a.rec.g2[idx];
        s_a0[wib][slot] = a.rec.a0[idx];
        s_a1[wib][slot] = make_float2(a1.x, a1.y);
        s_rb[wib][slot] = support_rho(g0.z);
        s_idx[wib][slot] = idx;
        s_q[wib][slot] = bstart + lane;
      }
      __syncwarp();
      const int cnt = __popc(km);
      for (int j = cnt - 1; j >= 0; --j) {
        const int jj = s_q[wib][j];
        float gr[kGradSlots];
#pragma unroll
        for (int q = 0; q < NG; ++q) gr[q] = 0.f;
        bool contrib = false;
#ifdef OCGS_COUNT
        if (lane == 0) OCGS_DIAG(2, 1);
#endif
        if (jj < (int)thread_last) {
          const float4 g0 = s_g0[wib][j], g1 = s_g1[wib][j], g2 = s_g2[wib][j];
          const float rb = s_rb[wib][j];
          const SplatColumn col = splat_column(g0, g1, g2, pxf);
          SplatHead2 hd[NP];
          bool any = false;
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const float2 py = make_float2((float)(py0 + 2 * p) + 0.5f, (float)(py0 + 2 * p + 1) + 0.5f);
            hd[p] = splat_head2(g0, g1, g2, col, py, rb);
            hd[p].pass[0] = hd[p].pass[0] && jj < (int)last[2 * p];
            hd[p].pass[1] = hd[p].pass[1] && jj < (int)last[2 * p + 1];
            any = any || hd[p].pass[0] || hd[p].pass[1];
          }
          if (any) {
            const float4 ap = s_a0[wib][j];
            const float2 an = s_a1[wib][j];
            const float2 dx = bc2(col.dx);
            const float2 ng2y = bc2(-g2.y), ng2z = bc2(-g2.z);
            float2 acc[kGradSlots];  // this thread's sums (first NG used), one lane per pixel of a pair
#pragma unroll
            for (int q = 0; q < NG; ++q) acc[q] = bc2(0.f);
            // no per-pair branch (see the forward): a pair without a blended pixel
            // adds exact zeros
#pragma unroll
            for (int p = 0; p < NP; ++p) {
              const SplatEval2 e = splat_tail2<true>(g0, g2, hd[p], rb);
              const bool ok0 = e.ok[0], ok1 = e.ok[1];
              contrib = contrib || ok0 || ok1;
              // undo the entry: T before it, its weight, and dL/dalpha (lanes that did
              // not blend get zero weight and zero dL/dalpha, which zeroes every term)
              const float2 om = __ffma2_rn(e.alpha, bc2(-1.f), bc2(1.f));  // 1 - alpha
              const float2 inv = make_float2(__fdividef(1.f, om.x), __fdividef(1.f, om.y));
              const float2 Ti = __fmul2_rn(T[p], inv);
              const float2 w = __fmul2_rn(e.alpha, Ti);
              float2 F = __fmul2_rn(gC0[p], bc2(ap.x));
              F = __ffma2_rn(gC1[p], bc2(ap.y), F);
              F = __ffma2_rn(gC2[p], bc2(ap.z), F);
              if (GEO) {
                F = __ffma2_rn(gD[p], e.z, F);
                F = __ffma2_rn(__fmul2_rn(gQ[p], e.z), e.z, F);  // d(sum w z^2)/dw = z^2
                F = __ffma2_rn(gN0[p], bc2(ap.w), F);
                F = __ffma2_rn(gN1[p], bc2(an.x), F);
                F = __ffma2_rn(gN2[p], bc2(an.y), F);
              }
              // dL/dalpha = T_i F + (gAT - S) / (1 - alpha)
              const float2 galpha = __ffma2_rn(Ti, F, __fmul2_rn(__ffma2_rn(S[p], bc2(-1.f), gAT[p]), inv));
              const float2 wm = make_float2(ok0 ? w.x : 0.f, ok1 ? w.y : 0.f);
              const float2 ga = make_float2(ok0 ? galpha.x : 0.f, ok1 ? galpha.y : 0.f);
              S[p] = __ffma2_rn(wm, F, S[p]);
              T[p] = make_float2(ok0 ? Ti.x : T[p].x, ok1 ? Ti.y : T[p].y);
              acc[kGr] = __ffma2_rn(gC0[p], wm, acc[kGr]);
              acc[kGg] = __ffma2_rn(gC1[p], wm, acc[kGg]);
              acc[kGb] = __ffma2_rn(gC2[p], wm, acc[kGb]);
              if (GEO) {
                acc[kGnx] = __ffma2_rn(gN0[p], wm, acc[kGnx]);
                acc[kGny] = __ffma2_rn(gN1[p], wm, acc[kGny]);
                acc[kGnz] = __ffma2_rn(gN2[p], wm, acc[kGnz]);
              }
              // alpha = o G below the 0.99 clamp; at the clamp nothing flows to rho or o
              const bool un0 = e.oG.x < kAlphaMax, un1 = e.oG.y < kAlphaMax;
              const float2 grr = __fmul2_rn(__fmul2_rn(bc2(-0.5f), ga), e.alpha);
              const float2 grho = make_float2(un0 ? grr.x : 0.f, un1 ? grr.y : 0.f);
              const float2 gop = __fmul2_rn(ga, e.G);
              acc[kGo] = __fadd2_rn(acc[kGo], make_float2(un0 ? gop.x : 0.f, un1 ? gop.y : 0.f));
              // rho and depth came from the surfel's (u, v) where it won the min, from the
              // screen-space filter elsewhere: split the cotangents between the two
              const bool s0 = e.surf[0], s1 = e.surf[1];
              const float2 grs = make_float2(s0 ? grho.x : 0.f, s1 ? grho.y : 0.f);
              const float2 grf = __ffma2_rn(grs, bc2(-1.f), grho);  // grho where the filter won, else 0
              float2 gzs = bc2(0.f);
              if (GEO) {
                // d/dz of w (gD z + gQ z^2)
                const float2 gz = __fmul2_rn(__ffma2_rn(__fmul2_rn(bc2(2.f), gQ[p]), e.z, gD[p]), wm);
                gzs = make_float2(s0 ? gz.x : 0.f, s1 ? gz.y : 0.f);
                acc[kGzc] = __fadd2_rn(acc[kGzc], __ffma2_rn(gzs, bc2(-1.f), gz));
                acc[kGzD] = __ffma2_rn(gzs, e.r, acc[kGzD]);
              }
              const float2 r2 = __fmul2_rn(e.r, e.r);
              const float2 gs2 = __fmul2_rn(grs, bc2(2.f));
              const float2 gun = __fmul2_rn(__fmul2_rn(gs2, hd[p].un), r2);
              const float2 gvn = __fmul2_rn(__fmul2_rn(gs2, hd[p].vn), r2);
              // -dL/dden = (2 grho rho3 + gz z) / den; the e slots and c slots below
              // accumulate negated and are flipped when the lanes are summed
              const float2 ngden = GEO ? __fmul2_rn(__ffma2_rn(gs2, e.rho3, __fmul2_rn(gzs, e.z)), e.r)
                                       : __fmul2_rn(__fmul2_rn(gs2, e.rho3), e.r);
              const float2 gdxs = __ffma2_rn(ngden, ng2y, __ffma2_rn(gvn, bc2(g1.z), __fmul2_rn(gun, bc2(g1.x))));
              const float2 gdys = __ffma2_rn(ngden, ng2z, __ffma2_rn(gvn, bc2(g1.w), __fmul2_rn(gun, bc2(g1.y))));
              acc[kGA00] = __ffma2_rn(gun, dx, acc[kGA00]);
              acc[kGA01] = __ffma2_rn(gun, hd[p].dy, acc[kGA01]);
              acc[kGA10] = __ffma2_rn(gvn, dx, acc[kGA10]);
              acc[kGA11] = __ffma2_rn(gvn, hd[p].dy, acc[kGA11]);
              acc[kGe0] = __fadd2_rn(acc[kGe0], ngden);
              acc[kGe1] = __ffma2_rn(ngden, dx, acc[kGe1]);
              acc[kGe2] = __ffma2_rn(ngden, hd[p].dy, acc[kGe2]);
              const float2 gf4 = __fmul2_rn(grf, bc2(4.f));
              acc[kGcx] = __fadd2_rn(acc[kGcx], __ffma2_rn(gf4, dx, gdxs));
              acc[kGcy] = __fadd2_rn(acc[kGcy], __ffma2_rn(gf4, hd[p].dy, gdys));
            }
#pragma unroll
            for (int q = 0; q < NG; ++q) {
              const bool negated = q == kGcx || q == kGcy || q == kGe0 || q == kGe1 || q == kGe2;
              gr[q] = negated ? -__fadd_rn(acc[q].x, acc[q].y) : __fadd_rn(acc[q].x, acc[q].y);
            }
          }
        }
        if (__any_sync(kFull, contrib)) {
#ifdef OCGS_COUNT
          if (lane == 0) OCGS_DIAG(3, 1);
          OCGS_DIAG(4, contrib ? 1 : 0);
          {
            const int nc = __popc(__ballot_sync(kFull, contrib));
            if (lane == 0) OCGS_DIAG(nc == 1 ? 5 : (nc <= 8 ? 6 : (nc >= 24 ? 7 : 0)), nc == 1 || nc <= 8 || nc >= 24 ? 1 : 0);
          }
#endif
          const int slot = warp_reduce<NG>(gr, lane);
          if (slot >= 0) s_grad[wib][j * kGradStride + slot] = gr[0];  // one lane per slot
        }
      }
      // flush the batch: one vector atomic per 4 slots and entry for the warp
      __syncwarp();
      if (lane < cnt) {
        float4* row = reinterpret_cast<float4*>(grow);
        float4* dst = reinterpret_cast<float4*>(a.grad_rec + (size_t)s_idx[wib][lane] * kGradStride);
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

// CTAs of kBlockWarps independent warps: persistent_ctas counts tile-sized CTAs
// (TW*TH/PPT threads), converted to the same number of warps
template <int TW, int TH, int PPT>
unsigned warp_grid(int persistent_ctas, uint32_t n_tiles) {
  constexpr uint64_t WPT = TW * TH / PPT / 32;
  const uint64_t warps = (persistent_ctas ? (uint64_t)persistent_ctas : (uint64_t)n_tiles) * WPT;
  return (unsigned)((warps + kBlockWarps - 1) / kBlockWarps);
}

template <int TW, int TH, int PPT>
cudaError_t fwd_dispatch(const RasterArgs& a, bool img, cudaStream_t s) {
  const unsigned grid = warp_grid<TW, TH, PPT>(a.persistent_ctas, a.n_tiles);
  if (grid == 0) return cudaSuccess;
  constexpr int NT = kBlockWarps * 32;
  const bool score = a.score != nullptr;
  const bool q2 = img && a.out.depth2 != nullptr;
  if (a.ewa) {
    if (img && score) raster_fwd_kernel<TW, TH, PPT, true, true, false, true><<<grid, NT, 0, s>>>(a);
    else if (img) raster_fwd_kernel<TW, TH, PPT, true, false, false, true><<<grid, NT, 0, s>>>(a);
    else if (score) raster_fwd_kernel<TW, TH, PPT, false, true, false, true><<<grid, NT, 0, s>>>(a);
    else return cudaSuccess;
  } else if (img && score && q2) raster_fwd_kernel<TW, TH, PPT, true, true, true, false><<<grid, NT, 0, s>>>(a);
  else if (img && q2) raster_fwd_kernel<TW, TH, PPT, true, false, true, false><<<grid, NT, 0, s>>>(a);
  else if (img && score) raster_fwd_kernel<TW, TH, PPT, true, true, false, false><<<grid, NT, 0, s>>>(a);
  else if (img) raster_fwd_kernel<TW, TH, PPT, true, false, false, false><<<grid, NT, 0, s>>>(a);
  else if (score) raster_fwd_kernel<TW, TH, PPT, false, true, false, false><<<grid, NT, 0, s>>>(a);
  else return cudaSuccess;
  return launched();
}

template <int TW, int TH, int PPT>
cudaError_t bwd_dispatch(const RasterBwdArgs& a, cudaStream_t s) {
  const unsigned grid = warp_grid<TW, TH, PPT>(a.persistent_ctas, a.n_tiles);
  if (grid == 0) return cudaSuccess;
  if (a.d_out.depth || a.d_out.normal || a.d_out.depth2)
    raster_bwd_kernel<TW, TH, PPT, true><<<grid, kBlockWarps * 32, 0, s>>>(a);
  else raster_bwd_kernel<TW, TH, PPT, false><<<grid, kBlockWarps * 32, 0, s>>>(a);
  return launched();
}

__global__ void sum_u32_kernel(const uint32_t* __restrict__ v, int64_t n, unsigned long long* __restrict__ out) {
  unsigned long long acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += v[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

}  // namespace

#ifdef OCGS_COUNT
extern "C" int ocgs_diag_read(unsigned long long* out, int reset) {
  cudaMemcpyFromSymbol(out, g_diag, sizeof(g_diag));
  if (reset) {
    unsigned long long z[8] = {0};
    cudaMemcpyToSymbol(g_diag, z, sizeof(z));
  }
  return 0;
}
#endif

cudaError_t launch_sum_u32(const uint32_t* v, int64_t n, unsigned long long* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess || n == 0) return e;
  sum_u32_kernel<<<304, 256, 0, s>>>(v, n, out);
  return launched();
}

cudaError_t launch_raster_forward(const RasterArgs& a, int tile_w, int tile_h, int ppt, bool write_image,
                                  cudaStream_t s) {
#define OCGS_FWD(W, H, K) \
  if (tile_w == W && tile_h == H && ppt == K) return fwd_dispatch<W, H, K>(a, write_image, s);
  OCGS_FWD(16, 16, 1) OCGS_FWD(16, 16, 2) OCGS_FWD(16, 16, 4)
  OCGS_FWD(16, 8, 1) OCGS_FWD(16, 8, 2) OCGS_FWD(16, 8, 4)
  OCGS_FWD(8, 8, 1) OCGS_FWD(8, 8, 2)
  OCGS_FWD(32, 8, 1) OCGS_FWD(32, 8, 2)
#undef OCGS_FWD
  return cudaErrorInvalidValue;
}

cudaError_t launch_raster_backward(const RasterBwdArgs& a, int tile_w, int tile_h, int ppt, cudaStream_t s) {
#define OCGS_BWD(W, H, K) \
  if (tile_w == W && tile_h == H && ppt == K) return bwd_dispatch<W, H, K>(a, s);
  OCGS_BWD(16, 16, 1) OCGS_BWD(16, 16, 2) OCGS_BWD(16, 16, 4)
  OCGS_BWD(16, 8, 1) OCGS_BWD(16, 8, 2) OCGS_BWD(16, 8, 4)
  OCGS_BWD(8, 8, 1) OCGS_BWD(8, 8, 2)
  OCGS_BWD(32, 8, 1) OCGS_BWD(32, 8, 2)
#undef OCGS_BWD
  return cudaErrorInvalidValue;
}

}  // namespace ocgs
