// Tile rasterizer: front-to-back compositing (forward) and its reverse-order
// adjoint (backward).
//
// One CTA owns one screen tile (one thread per pixel).  The tile's sorted
// (depth, Gaussian) list is streamed through shared memory in batches of one
// record per thread; every thread then evaluates the batch against its pixel
// centre.  Compositing of a pixel stops at the first blended candidate that
// would bring its transmittance below 1e-4 (Sec. 4.3: rendering ends once the
// pixel reaches an opacity close to 1), warps stop once all their pixels have
// stopped, and the CTA stops once every pixel has.  The forward optionally
// records, for each Gaussian, the max blending weight over the pixels where it
// was blended (the per-Gaussian visibility record that Sec. 4.3 and Sec. 5.1
// keep while colours accumulate), with one warp max-reduction and at most one
// atomic per warp.
//
// The backward walks the same list back to front from each pixel's last
// blended entry, recovering the transmittance T_i = T_{i+1} / (1 - alpha_i)
// from the stored final transmittance, so nothing per (pixel, Gaussian) is
// stored between the passes.  Per-Gaussian gradients are reduced over the warp
// with shuffles before one atomic add per slot and warp.
#include "common.cuh"

namespace ocgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int TW, int TH, bool IMG, bool SCORE>
__global__ void __launch_bounds__(TW * TH) raster_fwd_kernel(const RasterArgs a) {
  constexpr int BS = TW * TH;
  __shared__ float4 s_g0[BS], s_g1[BS], s_g2[BS], s_a0[BS];
  __shared__ float2 s_a1[BS];
  __shared__ uint32_t s_gid[BS];
  __shared__ uint32_t s_tile;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int lx = tid % TW, ly = tid / TW;
  for (uint32_t it = 0;; ++it) {
    uint32_t tile;
    if (a.persistent_ctas) {
      __syncthreads();
      if (tid == 0) s_tile = atomicAdd(a.queue, 1u);
      __syncthreads();
      tile = s_tile;
      if (tile >= a.n_tiles) break;
      if (a.tile_order) tile = a.tile_order[tile];
    } else {
      if (it > 0) break;
      tile = blockIdx.x;
    }
    const int v = view_of_tile(a.tile_prefix, a.n_views, (int)tile);
    const DevCam& cam = a.cams[v];
    const int local = (int)tile - cam.tile_offset;
    const int px = (local % cam.tiles_x) * TW + lx;
    const int py = (local / cam.tiles_x) * TH + ly;
    const bool inside = px < cam.W && py < cam.H;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const uint2 rg = a.ranges[tile];
    const uint32_t start = rg.x, end = rg.y;
    const int64_t gbase = (int64_t)v * a.n_gauss;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, dep = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    for (uint32_t b0 = start; b0 < end; b0 += BS) {
      if (__syncthreads_count(!done) == 0) break;
      const uint32_t k = b0 + tid;
      if (k < end) {
        const uint32_t idx = a.vals[k];
        s_g0[tid] = a.rec.g0[idx];
        s_g1[tid] = a.rec.g1[idx];
        s_g2[tid] = a.rec.g2[idx];
        s_a0[tid] = a.rec.a0[idx];
        s_a1[tid] = a.rec.a1[idx];
        if (SCORE) s_gid[tid] = (uint32_t)((int64_t)idx - gbase);
      }
      __syncthreads();
      const int cnt = (end - b0 < (uint32_t)BS) ? (int)(end - b0) : BS;
      for (int j = 0; j < cnt; ++j) {
        if (__all_sync(kFull, done)) break;
        float w = 0.f;
        if (!done) {
          const SplatEval e = eval_splat(s_g0[j], s_g1[j], s_g2[j], pxf, pyf);
          if (e.ok) {
            const float Tn = T * (1.f - e.alpha);
            if (Tn < kTEps) {
              done = true;
            } else {
              w = e.alpha * T;
              if (IMG) {
                const float4 ap = s_a0[j];
                const float2 an = s_a1[j];
                c0 += w * ap.x; c1 += w * ap.y; c2 += w * ap.z;
                dep += w * e.z;
                n0 += w * ap.w; n1 += w * an.x; n2 += w * an.y;
              }
              T = Tn;
              last = b0 + (uint32_t)j - start + 1u;
            }
          }
        }
        if (SCORE) {
          const unsigned m = __reduce_max_sync(kFull, __float_as_uint(w));
          if (lane == 0 && m != 0u) atomicMax(reinterpret_cast<unsigned*>(a.score) + s_gid[j], m);
        }
      }
    }
    if (IMG && inside) {
      const int64_t pix = cam.pix_offset + (int64_t)py * cam.W + px;
      a.out.rgb[3 * pix + 0] = c0;
      a.out.rgb[3 * pix + 1] = c1;
      a.out.rgb[3 * pix + 2] = c2;
      a.out.alpha[pix] = 1.f - T;
      a.out.depth[pix] = dep;
      a.out.normal[3 * pix + 0] = n0;
      a.out.normal[3 * pix + 1] = n1;
      a.out.normal[3 * pix + 2] = n2;
      a.t_final[pix] = T;
      a.last[pix] = last;
    }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) raster_bwd_kernel(const RasterBwdArgs a) {
  constexpr int BS = TW * TH;
  constexpr int NG = 18;
  __shared__ float4 s_g0[BS], s_g1[BS], s_g2[BS], s_a0[BS];
  __shared__ float2 s_a1[BS];
  __shared__ uint32_t s_idx[BS];
  __shared__ uint32_t s_tile, s_max;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int lx = tid % TW, ly = tid / TW;
  for (uint32_t it = 0;; ++it) {
    uint32_t tile;
    if (a.persistent_ctas) {
      __syncthreads();
      if (tid == 0) s_tile = atomicAdd(a.queue, 1u);
      __syncthreads();
      tile = s_tile;
      if (tile >= a.n_tiles) break;
      if (a.tile_order) tile = a.tile_order[tile];
    } else {
      if (it > 0) break;
      tile = blockIdx.x;
    }
    const int v = view_of_tile(a.tile_prefix, a.n_views, (int)tile);
    const DevCam& cam = a.cams[v];
    const int local = (int)tile - cam.tile_offset;
    const int px = (local % cam.tiles_x) * TW + lx;
    const int py = (local / cam.tiles_x) * TH + ly;
    const bool inside = px < cam.W && py < cam.H;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const uint32_t start = a.ranges[tile].x;
    float T = 1.f, Tf = 1.f;
    uint32_t my_last = 0;
    float gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gA = 0.f, gD = 0.f, gN0 = 0.f, gN1 = 0.f, gN2 = 0.f;
    if (inside) {
      const int64_t pix = cam.pix_offset + (int64_t)py * cam.W + px;
      Tf = a.t_final[pix];
      T = Tf;
      my_last = a.last[pix];
      if (a.d_out.rgb) { gC0 = a.d_out.rgb[3 * pix]; gC1 = a.d_out.rgb[3 * pix + 1]; gC2 = a.d_out.rgb[3 * pix + 2]; }
      if (a.d_out.alpha) gA = a.d_out.alpha[pix];
      if (a.d_out.depth) gD = a.d_out.depth[pix];
      if (a.d_out.normal) { gN0 = a.d_out.normal[3 * pix]; gN1 = a.d_out.normal[3 * pix + 1]; gN2 = a.d_out.normal[3 * pix + 2]; }
    }
    __syncthreads();
    if (tid == 0) s_max = 0u;
    __syncthreads();
    if (my_last) atomicMax(&s_max, my_last);
    __syncthreads();
    const int max_last = (int)s_max;
    float S = 0.f;  // sum over later blended entries of w * (gC.rgb + gD z + gN.n)
    const float gAT = gA * Tf;
    for (int bend = max_last; bend > 0; bend -= BS) {
      const int bstart = max(0, bend - BS);
      __syncthreads();
      if (bstart + tid < bend) {
        const uint32_t idx = a.vals[start + (uint32_t)(bstart + tid)];
        s_g0[tid] = a.rec.g0[idx];
        s_g1[tid] = a.rec.g1[idx];
        s_g2[tid] = a.rec.g2[idx];
        s_a0[tid] = a.rec.a0[idx];
        s_a1[tid] = a.rec.a1[idx];
        s_idx[tid] = idx;
      }
      __syncthreads();
      for (int j = bend - 1 - bstart; j >= 0; --j) {
        const int jj = bstart + j;
        float gr[NG];
#pragma unroll
        for (int q = 0; q < NG; ++q) gr[q] = 0.f;
        bool contrib = false;
        if (jj < (int)my_last) {
          const float4 g1 = s_g1[j], g2 = s_g2[j];
          const SplatEval e = eval_splat(s_g0[j], g1, g2, pxf, pyf);
          if (e.ok) {
            contrib = true;
            const float4 ap = s_a0[j];
            const float2 an = s_a1[j];
            const float inv = 1.f / (1.f - e.alpha);
            const float Ti = T * inv;
            const float w = e.alpha * Ti;
            const float F = gC0 * ap.x + gC1 * ap.y + gC2 * ap.z + gD * e.z + gN0 * ap.w + gN1 * an.x +
                            gN2 * an.y;
            const float galpha = Ti * F - (S - gAT) * inv;
            S += w * F;
            T = Ti;
            gr[kGr] = gC0 * w; gr[kGg] = gC1 * w; gr[kGb] = gC2 * w;
            gr[kGnx] = gN0 * w; gr[kGny] = gN1 * w; gr[kGnz] = gN2 * w;
            const float gz = gD * w;
            const bool unclamped = e.oG < kAlphaMax;
            const float grho = unclamped ? -0.5f * galpha * e.alpha : 0.f;
            gr[kGo] = unclamped ? galpha * e.G : 0.f;
            float gdx, gdy;
            if (e.surf) {
              const float r2 = e.r * e.r;
              const float gun = grho * 2.f * e.un * r2;
              const float gvn = grho * 2.f * e.vn * r2;
              const float gden = -grho * 2.f * e.rho3 * e.r - gz * e.z * e.r;
              gr[kGzD] = gz * e.r;
              gdx = gun * g1.x + gvn * g1.z + gden * g2.y;
              gdy = gun * g1.y + gvn * g1.w + gden * g2.z;
              gr[kGA00] = gun * e.dx; gr[kGA01] = gun * e.dy;
              gr[kGA10] = gvn * e.dx; gr[kGA11] = gvn * e.dy;
              gr[kGe0] = gden; gr[kGe1] = gden * e.dx; gr[kGe2] = gden * e.dy;
            } else {
              gdx = grho * 4.f * e.dx;
              gdy = grho * 4.f * e.dy;
              gr[kGzc] = gz;
            }
            gr[kGcx] = -gdx;
            gr[kGcy] = -gdy;
          }
        }
        if (__any_sync(kFull, contrib)) {
#pragma unroll
          for (int q = 0; q < NG; ++q) gr[q] = warp_sum(gr[q]);
          if (lane == 0) {
            float* dst = a.grad_rec + (size_t)s_idx[j] * kGradStride;
#pragma unroll
            for (int q = 0; q < NG; ++q)
              if (gr[q] != 0.f) atomicAdd(dst + q, gr[q]);
          }
        }
      }
    }
  }
}

template <int TW, int TH>
cudaError_t fwd_dispatch(const RasterArgs& a, bool img, cudaStream_t s) {
  const unsigned grid = a.persistent_ctas ? (unsigned)a.persistent_ctas : a.n_tiles;
  if (grid == 0) return cudaSuccess;
  const bool score = a.score != nullptr;
  if (img && score) raster_fwd_kernel<TW, TH, true, true><<<grid, TW * TH, 0, s>>>(a);
  else if (img) raster_fwd_kernel<TW, TH, true, false><<<grid, TW * TH, 0, s>>>(a);
  else if (score) raster_fwd_kernel<TW, TH, false, true><<<grid, TW * TH, 0, s>>>(a);
  else return cudaSuccess;
  return launched();
}

template <int TW, int TH>
cudaError_t bwd_dispatch(const RasterBwdArgs& a, cudaStream_t s) {
  const unsigned grid = a.persistent_ctas ? (unsigned)a.persistent_ctas : a.n_tiles;
  if (grid == 0) return cudaSuccess;
  raster_bwd_kernel<TW, TH><<<grid, TW * TH, 0, s>>>(a);
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

cudaError_t launch_sum_u32(const uint32_t* v, int64_t n, unsigned long long* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess || n == 0) return e;
  sum_u32_kernel<<<304, 256, 0, s>>>(v, n, out);
  return launched();
}

cudaError_t launch_raster_forward(const RasterArgs& a, int tile_w, int tile_h, bool write_image,
                                  cudaStream_t s) {
  if (tile_w == 16 && tile_h == 16) return fwd_dispatch<16, 16>(a, write_image, s);
  if (tile_w == 16 && tile_h == 8) return fwd_dispatch<16, 8>(a, write_image, s);
  if (tile_w == 8 && tile_h == 8) return fwd_dispatch<8, 8>(a, write_image, s);
  if (tile_w == 32 && tile_h == 8) return fwd_dispatch<32, 8>(a, write_image, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_raster_backward(const RasterBwdArgs& a, int tile_w, int tile_h, cudaStream_t s) {
  if (tile_w == 16 && tile_h == 16) return bwd_dispatch<16, 16>(a, s);
  if (tile_w == 16 && tile_h == 8) return bwd_dispatch<16, 8>(a, s);
  if (tile_w == 8 && tile_h == 8) return bwd_dispatch<8, 8>(a, s);
  if (tile_w == 32 && tile_h == 8) return bwd_dispatch<32, 8>(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace ocgs
