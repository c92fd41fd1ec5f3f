// Forward tile rasterizer: front-to-back compositing (Sec. 4.3) with the
// optional per-Gaussian contribution record (Sec. 4.3, Sec. 5.1).
//
// A warp owns one band of a screen tile (32 threads x PPT vertically adjacent
// pixels each: full tile rows) and walks the tile's sorted (depth, Gaussian)
// list on its own, with no CTA barrier: its own slot of the persistent queue,
// its own shared-memory batches of BATCH records.  Every lane evaluates the
// batch against its pixel centres, so one shared-memory read of a record
// serves PPT pixels; the batch staging first drops, in order, the entries
// whose support misses the band's rows.  Compositing of a pixel stops at the
// first blended candidate that would bring its transmittance below 1e-4
// (rendering ends once the pixel reaches an opacity close to 1), and a warp
// stops once all its pixels have stopped.  The forward optionally records, for
// each Gaussian, the max blending weight over the pixels where it was blended
// (the per-Gaussian visibility record kept while colours accumulate), with
// one warp max-reduction and at most one atomic per warp and entry.
#include "raster_common.cuh"

namespace ocgs {
namespace {
using namespace raster;

#ifdef OCGS_COUNT
__device__ unsigned long long g_diag[8];
#endif

// Resident warps per SM the compiler is asked to fit (caps registers per
// thread): 20 leaves 96 registers, enough for the image planes without spills
// (24 warps at 80 registers spill about 60 bytes and measured 1.5 % slower).
#ifndef OCGS_FWD_WARPS
#define OCGS_FWD_WARPS 20
#endif
#ifndef OCGS_FWD_WARPS_Q2
#define OCGS_FWD_WARPS_Q2 20
#endif

// Q2: also accumulate Q = sum w z^2 (the depth distortion's third plane)
// EWA: the records are projected 3D Gaussians (the 3DGS variant of Appendix B)
template <int TW, int TH, int PPT, int BATCH, bool IMG, bool SCORE, bool Q2, bool EWA>
__global__ void __launch_bounds__(kBlockWarps * 32, (Q2 ? OCGS_FWD_WARPS_Q2 : OCGS_FWD_WARPS) / kBlockWarps)
    raster_fwd_kernel(const RasterArgs a) {
  constexpr int WPT = TW * TH / PPT / 32;  // warps per tile: each owns a band of full tile rows
  using B = Batch<BATCH>;
  __shared__ float4 s_g0[kBlockWarps][BATCH], s_g1[kBlockWarps][BATCH], s_g2[kBlockWarps][BATCH],
      s_a0[kBlockWarps][IMG ? BATCH : 1];
  __shared__ float2 s_a1[kBlockWarps][IMG ? BATCH : 1];
  __shared__ uint32_t s_gid[kBlockWarps][SCORE ? BATCH : 1];
  __shared__ uint32_t s_pos[kBlockWarps][BATCH];  // list index of each kept entry
  __shared__ float s_rb[kBlockWarps][BATCH];
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
    for (uint32_t b0 = start; b0 < end; b0 += BATCH) {
      if (__all_sync(kFull, alldone)) break;
      __syncwarp();  // the previous batch is consumed
      // a batch of the list; keep (in order) the entries whose rows meet this warp's band
      int cnt = 0;
#pragma unroll
      for (int r = 0; r < B::kRounds; ++r) {
        const uint32_t kk = b0 + (uint32_t)(r * 32 + lane);
        bool keep = false;
        uint32_t idx = 0;
        float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < B::kLanes && kk < end) {
          idx = a.vals[kk];
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
          if (IMG) {
            s_a0[wib][slot] = a.rec.a0[idx];
            s_a1[wib][slot] = make_float2(a1.x, a1.y);
          }
          s_rb[wib][slot] = blend_rho(g0.z);
          s_pos[wib][slot] = kk;
          if (SCORE) s_gid[wib][slot] = (uint32_t)((int64_t)idx - gbase);
        }
        cnt += __popc(km);
      }
      __syncwarp();
      for (int j = 0; j < cnt; ++j) {
        if ((j & 7) == 0 && j > 0 && __all_sync(kFull, alldone)) break;
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
          // every pair is evaluated without a per-pair branch: a candidate that is
          // not blended has alpha = 0 (T (1 - 0) = T, w = 0 exactly), and
          // straight-line code lets the pairs' dependency chains interleave
          bool stopped = false;
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const int k0 = 2 * p, k1 = 2 * p + 1;
            const float2 py = make_float2((float)(py0 + k0) + 0.5f, (float)(py0 + k1) + 0.5f);
            const SplatHead2 h = splat_head2(g0, g1, g2, col, py);
            const SplatEval2 e = splat_tail2<false, EWA>(g0, g2, h, rb, !done[k0], !done[k1]);
            float2 Tn = pmul(T[p], pfma(e.alpha, bc2(-1.f), bc2(1.f)));  // T (1 - alpha)
            float2 w = pmul(e.alpha, T[p]);
            const uint32_t l0 = last[k0], l1 = last[k1];
            if (e.ok[0]) last[k0] = pos;
            if (e.ok[1]) last[k1] = pos;
            if (fminf(Tn.x, Tn.y) < kTEps) {
              // rare: an entry that would take T below kTEps ends the pixel unblended
              if (Tn.x < kTEps) { done[k0] = true; w.x = 0.f; Tn.x = T[p].x; last[k0] = l0; }
              if (Tn.y < kTEps) { done[k1] = true; w.y = 0.f; Tn.y = T[p].y; last[k1] = l1; }
              stopped = true;
            }
            if (IMG) {
              c0[p] = pfma(w, bc2(ap.x), c0[p]);
              c1[p] = pfma(w, bc2(ap.y), c1[p]);
              c2[p] = pfma(w, bc2(ap.z), c2[p]);
              dep[p] = pfma(w, e.z, dep[p]);
              if (Q2) qz[p] = pfma(pmul(w, e.z), e.z, qz[p]);
              n0[p] = pfma(w, bc2(ap.w), n0[p]);
              n1[p] = pfma(w, bc2(an.x), n1[p]);
              n2[p] = pfma(w, bc2(an.y), n2[p]);
            }
            T[p] = Tn;
            if (SCORE) wmax = fmaxf(wmax, fmaxf(w.x, w.y));
#ifdef OCGS_COUNT
            OCGS_DIAG(2, (w.x > 0.f ? 1 : 0) + (w.y > 0.f ? 1 : 0));  // (pixel, entry) blends
#endif
          }
          if (stopped) {  // done only changes when a pixel stops
            alldone = true;
#pragma unroll
            for (int k = 0; k < 2 * NP; ++k) alldone = alldone && done[k];
          }
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

template <int TW, int TH, int PPT, int BATCH>
cudaError_t fwd_dispatch(const RasterArgs& a, bool img, cudaStream_t s) {
  const unsigned grid = warp_grid<TW, TH, PPT>(a.persistent_ctas, a.n_tiles);
  if (grid == 0) return cudaSuccess;
  constexpr int NT = kBlockWarps * 32;
  const bool score = a.score != nullptr;
  const bool q2 = img && a.out.depth2 != nullptr;
  if (a.ewa) {
    if (img && score) raster_fwd_kernel<TW, TH, PPT, BATCH, true, true, false, true><<<grid, NT, 0, s>>>(a);
    else if (img) raster_fwd_kernel<TW, TH, PPT, BATCH, true, false, false, true><<<grid, NT, 0, s>>>(a);
    else if (score) raster_fwd_kernel<TW, TH, PPT, BATCH, false, true, false, true><<<grid, NT, 0, s>>>(a);
    else return cudaSuccess;
  } else if (img && score && q2) raster_fwd_kernel<TW, TH, PPT, BATCH, true, true, true, false><<<grid, NT, 0, s>>>(a);
  else if (img && q2) raster_fwd_kernel<TW, TH, PPT, BATCH, true, false, true, false><<<grid, NT, 0, s>>>(a);
  else if (img && score) raster_fwd_kernel<TW, TH, PPT, BATCH, true, true, false, false><<<grid, NT, 0, s>>>(a);
  else if (img) raster_fwd_kernel<TW, TH, PPT, BATCH, true, false, false, false><<<grid, NT, 0, s>>>(a);
  else if (score) raster_fwd_kernel<TW, TH, PPT, BATCH, false, true, false, false><<<grid, NT, 0, s>>>(a);
  else return cudaSuccess;
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

cudaError_t launch_raster_forward(const RasterArgs& a, int tile_w, int tile_h, int ppt, int batch, bool write_image,
                                  cudaStream_t s) {
#define OCGS_FWD(W, H, K, BT) \
  if (tile_w == W && tile_h == H && ppt == K && batch == BT) return fwd_dispatch<W, H, K, BT>(a, write_image, s);
  OCGS_RASTER_SHAPES(OCGS_FWD)
#undef OCGS_FWD
  return cudaErrorInvalidValue;
}

}  // namespace ocgs
