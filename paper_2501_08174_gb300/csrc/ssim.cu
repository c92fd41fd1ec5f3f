// SSIM of masked images and masked PSNR (Sec. 5), and the D-SSIM part of the
// photometric loss that Eq. 2 evaluates on masked images.
//
// SSIM statistics are windowed means under an 11x11 Gaussian window of sigma
// 1.5, zero outside the image; the window is separable, so every block stages
// a 42x42 patch (its 32x32 output tile plus a 5-pixel halo) of one channel of
// both masked images in shared memory and applies the 11 taps along rows, then
// columns, each thread producing 4 neighbouring outputs from one 14-value
// window so that a staged value is read once per 4 outputs.  The statistics
// pass filters (x1, x2) and (x1^2, x2^2) as packed FP32x2 pairs, one packed FMA
// per tap for two planes (each lane rounded as the scalar tap).
// The adjoint of the mean SSIM needs, at every pixel q,
//     sum_p dS(p)/dE[x2](p) G(p-q) + 2 x2(q) sum_p dS(p)/dE[x2^2](p) G(p-q)
//                                 +   x1(q) sum_p dS(p)/dE[x1 x2](p) G(p-q),
// i.e. the same window applied to three per-pixel maps, which the first pass
// writes and the second blurs.
#include "common.cuh"

#include <cmath>

namespace ocgs {
namespace {

constexpr int kT = 32;               // output tile side
constexpr int kR = 5;                // window radius
constexpr int kP = kT + 2 * kR;      // staged patch side (42)
constexpr int kSeg = 4;              // outputs per thread along a row (first pass) or column (second)
constexpr int kThreadsSsim = 256;
constexpr int kTaps = 2 * kR + 1;
constexpr int kRowItems = kP * (kT / kSeg);  // row segments of one plane (336)
constexpr int kPatchLoads = (kP * kP + kThreadsSsim - 1) / kThreadsSsim;  // patch values per thread (7)
constexpr int kLoadGroup = 4;        // patch values a thread of the statistics pass loads at once
constexpr float kC1 = 0.0001f;       // (0.01)^2
constexpr float kC2 = 0.0009f;       // (0.03)^2

struct Window {
  float w[kTaps];
};

__device__ __forceinline__ void tile_origin(const int* prefix, int n_views, const DevCam* cams, int* v, int* x0,
                                            int* y0) {
  const int b = blockIdx.x;
  *v = view_of_tile(prefix, n_views, b);
  const DevCam& cam = cams[*v];
  const int local = b - prefix[*v];
  const int tx = (cam.W + kT - 1) / kT;
  *x0 = (local % tx) * kT;
  *y0 = (local / tx) * kT;
}

// kSeg consecutive outputs of an 11-tap window over 14 inputs
__device__ __forceinline__ void taps4(const float (&in)[kSeg + 2 * kR], const Window& win, float (&out)[kSeg]) {
#pragma unroll
  for (int k = 0; k < kSeg; ++k) {
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < kTaps; ++t) acc = __fmaf_rn(win.w[t], in[k + t], acc);
    out[k] = acc;
  }
}

// the same window over pairs of planes, one packed FP32x2 FMA per tap (each lane
// rounded as taps4 rounds it)
__device__ __forceinline__ void taps4x2(const float2 (&in)[kSeg + 2 * kR], const Window& win, float2 (&out)[kSeg]) {
#pragma unroll
  for (int k = 0; k < kSeg; ++k) {
    float2 acc = bc2(0.f);
#pragma unroll
    for (int t = 0; t < kTaps; ++t) acc = pfma(bc2(win.w[t]), in[k + t], acc);
    out[k] = acc;
  }
}

// partial[3 b + k]: k = 0 sum of S over the tile's values, 1 sum over its mask
// values, 2 number of mask values.  gmap (or NULL): planes [9][P_total], plane
// 3 c + j holds, for channel c, j = 0 dS/dE[x2], 1 dS/dE[x2^2], 2 dS/dE[x1 x2].
__global__ void __launch_bounds__(kThreadsSsim, 4) ssim_stats_kernel(
    const float* __restrict__ rgb, const float* __restrict__ target, const uint8_t* __restrict__ mask,
    const DevCam* __restrict__ cams, int n_views, const int* __restrict__ prefix, const Window win,
    int64_t p_total, double* __restrict__ partial, float* __restrict__ gmap) {
  __shared__ float2 sx[kP][kP + 1];               // (masked target x1, masked render x2) of one channel
  // row-windowed (x1, x2), (x1^2, x2^2) as packed pairs, and x1 x2
  __shared__ __align__(16) float2 h01[kP][kT], h23[kP][kT];
  __shared__ __align__(16) float h4[kP][kT];
  __shared__ int s_cnt[kThreadsSsim / 32];
  int v, x0, y0;
  tile_origin(prefix, n_views, cams, &v, &x0, &y0);
  const DevCam& cam = cams[v];
  const int tid = threadIdx.x;
  const int col = tid % kT, r0 = (tid / kT) * kSeg;  // second pass: 4 rows of one column
  CompSum sums[2];  // S over all values, S over the mask values
  int cnt = 0;      // mask values
  for (int c = 0; c < 3; ++c) {
    if (c > 0) __syncthreads();  // the previous channel's second pass is done with sx and h
    // the patch in groups of kLoadGroup values per thread, each group's loads issued
    // before the first is used (the memory latency is paid per group, not per value)
#pragma unroll
    for (int j0 = 0; j0 < kPatchLoads; j0 += kLoadGroup) {
      float lt[kLoadGroup], lr[kLoadGroup];
      bool lm[kLoadGroup];
#pragma unroll
      for (int u = 0; u < kLoadGroup; ++u) {
        const int i = tid + (j0 + u) * kThreadsSsim;
        const int py = i / kP, px = i % kP;
        const int gy = y0 - kR + py, gx = x0 - kR + px;
        lt[u] = lr[u] = 0.f;
        lm[u] = false;
        if (j0 + u < kPatchLoads && i < kP * kP && gy >= 0 && gy < cam.H && gx >= 0 && gx < cam.W) {
          const int64_t q = cam.pix_offset + (int64_t)gy * cam.W + gx;
          lm[u] = mask[q] != 0;
          lt[u] = target[3 * q + c];
          lr[u] = rgb[3 * q + c];
        }
      }
#pragma unroll
      for (int u = 0; u < kLoadGroup; ++u) {
        const int i = tid + (j0 + u) * kThreadsSsim;
        if (j0 + u < kPatchLoads && i < kP * kP)
          sx[i / kP][i % kP] = lm[u] ? make_float2(lt[u], lr[u]) : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    for (int i = tid; i < kRowItems; i += kThreadsSsim) {
      const int r = i / (kT / kSeg), x = (i % (kT / kSeg)) * kSeg;
      float2 in2[kSeg + 2 * kR], sq2[kSeg + 2 * kR];
      float x12[kSeg + 2 * kR];
#pragma unroll
      for (int t = 0; t < kSeg + 2 * kR; ++t) {
        const float2 q = sx[r][x + t];
        in2[t] = q;
        sq2[t] = pmul(q, q);
        x12[t] = __fmul_rn(q.x, q.y);
      }
      float2 o2[kSeg];
      float o[kSeg];
      taps4x2(in2, win, o2);
      *reinterpret_cast<float4*>(&h01[r][x]) = make_float4(o2[0].x, o2[0].y, o2[1].x, o2[1].y);
      *reinterpret_cast<float4*>(&h01[r][x + 2]) = make_float4(o2[2].x, o2[2].y, o2[3].x, o2[3].y);
      taps4x2(sq2, win, o2);
      *reinterpret_cast<float4*>(&h23[r][x]) = make_float4(o2[0].x, o2[0].y, o2[1].x, o2[1].y);
      *reinterpret_cast<float4*>(&h23[r][x + 2]) = make_float4(o2[2].x, o2[2].y, o2[3].x, o2[3].y);
      taps4(x12, win, o);
      *reinterpret_cast<float4*>(&h4[r][x]) = make_float4(o[0], o[1], o[2], o[3]);
    }
    __syncthreads();
    float st[5][kSeg];  // windowed x1, x2, x1^2, x2^2, x1 x2
    {
      float2 in2[kSeg + 2 * kR], o2[kSeg];
#pragma unroll
      for (int t = 0; t < kSeg + 2 * kR; ++t) in2[t] = h01[r0 + t][col];
      taps4x2(in2, win, o2);
#pragma unroll
      for (int k = 0; k < kSeg; ++k) {
        st[0][k] = o2[k].x;
        st[1][k] = o2[k].y;
      }
#pragma unroll
      for (int t = 0; t < kSeg + 2 * kR; ++t) in2[t] = h23[r0 + t][col];
      taps4x2(in2, win, o2);
#pragma unroll
      for (int k = 0; k < kSeg; ++k) {
        st[2][k] = o2[k].x;
        st[3][k] = o2[k].y;
      }
      float in[kSeg + 2 * kR];
#pragma unroll
      for (int t = 0; t < kSeg + 2 * kR; ++t) in[t] = h4[r0 + t][col];
      taps4(in, win, st[4]);
    }
#pragma unroll
    for (int k = 0; k < kSeg; ++k) {
      const int gx = x0 + col, gy = y0 + r0 + k;
      if (gx >= cam.W || gy >= cam.H) continue;
      const int64_t p = cam.pix_offset + (int64_t)gy * cam.W + gx;
      const bool m = mask[p] != 0;
      const float mu1 = st[0][k], mu2 = st[1][k];
      const float v11 = st[2][k] - mu1 * mu1, v22 = st[3][k] - mu2 * mu2, v12 = st[4][k] - mu1 * mu2;
      const float n1 = 2.f * mu1 * mu2 + kC1, n2 = 2.f * v12 + kC2;
      const float d1 = mu1 * mu1 + mu2 * mu2 + kC1, d2 = v11 + v22 + kC2;
      const float inv = 1.f / (d1 * d2);
      const float S = n1 * n2 * inv;
      sums[0].add(S);
      if (m) {
        sums[1].add(S);
        ++cnt;
      }
      if (gmap) {
        // partial derivatives at fixed (mu, sigma), then through sigma22 = E[x2^2] - mu2^2
        // and sigma12 = E[x1 x2] - mu1 mu2 onto the three windowed means of x2
        const float dmu2 = 2.f * mu1 * n2 * inv - S * 2.f * mu2 / d1;
        const float dv22 = -S / d2;
        const float dv12 = 2.f * n1 * inv;
        gmap[(3 * c) * p_total + p] = dmu2 - 2.f * mu2 * dv22 - mu1 * dv12;
        gmap[(3 * c + 1) * p_total + p] = dv22;
        gmap[(3 * c + 2) * p_total + p] = dv12;
      }
    }
  }
  // block sums in a fixed order; the barrier inside block_comp_sums publishes s_cnt
  const int wc = __reduce_add_sync(0xffffffffu, cnt);
  if ((tid & 31) == 0) s_cnt[tid >> 5] = wc;
  block_comp_sums<kThreadsSsim, 2>(sums, partial + 3 * blockIdx.x);
  if (tid == 0) {
    int t = 0;
    for (int w = 0; w < kThreadsSsim / 32; ++w) t += s_cnt[w];
    partial[3 * blockIdx.x + 2] = (double)t;
  }
}

// d_rgb(q) += coef_v M(q) [G*a + 2 x2 G*b + x1 G*c](q), coef_v = -weight / (3 h w)
__global__ void __launch_bounds__(kThreadsSsim) ssim_grad_kernel(
    const float* __restrict__ rgb, const float* __restrict__ target, const uint8_t* __restrict__ mask,
    const DevCam* __restrict__ cams, int n_views, const int* __restrict__ prefix, const Window win,
    int64_t p_total, const float* __restrict__ gmap, float weight, float* __restrict__ d_rgb) {
  __shared__ float sg[3][kP][kP + 1];
  __shared__ __align__(16) float h[3][kP][kT];
  int v, x0, y0;
  tile_origin(prefix, n_views, cams, &v, &x0, &y0);
  const DevCam& cam = cams[v];
  const int tid = threadIdx.x;
  const int col = tid % kT, r0 = (tid / kT) * kSeg;
  const float coef = -weight / (3.f * (float)cam.W * (float)cam.H);
  for (int c = 0; c < 3; ++c) {
    if (c > 0) __syncthreads();
    // each plane's patch in one group: its loads in flight together, then the stores
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float lv[kPatchLoads];
#pragma unroll
      for (int k = 0; k < kPatchLoads; ++k) {
        const int i = tid + k * kThreadsSsim;
        const int py = i / kP, px = i % kP;
        const int gy = y0 - kR + py, gx = x0 - kR + px;
        lv[k] = 0.f;
        if (i < kP * kP && gy >= 0 && gy < cam.H && gx >= 0 && gx < cam.W)
          lv[k] = gmap[(3 * c + j) * p_total + cam.pix_offset + (int64_t)gy * cam.W + gx];
      }
#pragma unroll
      for (int k = 0; k < kPatchLoads; ++k) {
        const int i = tid + k * kThreadsSsim;
        if (i < kP * kP) sg[j][i / kP][i % kP] = lv[k];
      }
    }
    __syncthreads();
    for (int i = tid; i < 3 * kRowItems; i += kThreadsSsim) {
      const int j = i / kRowItems, rem = i % kRowItems;
      const int r = rem / (kT / kSeg), x = (rem % (kT / kSeg)) * kSeg;
      float in[kSeg + 2 * kR], o[kSeg];
#pragma unroll
      for (int t = 0; t < kSeg + 2 * kR; ++t) in[t] = sg[j][r][x + t];
      taps4(in, win, o);
      *reinterpret_cast<float4*>(&h[j][r][x]) = make_float4(o[0], o[1], o[2], o[3]);
    }
    __syncthreads();
    float g[3][kSeg];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float in[kSeg + 2 * kR];
#pragma unroll
      for (int t = 0; t < kSeg + 2 * kR; ++t) in[t] = h[j][r0 + t][col];
      taps4(in, win, g[j]);
    }
    // x2 = R M: no gradient where M = 0 (the loads of the 4 outputs are issued together)
    bool om[kSeg];
    float o1[kSeg], o2[kSeg], od[kSeg];
#pragma unroll
    for (int k = 0; k < kSeg; ++k) {
      const int gx = x0 + col, gy = y0 + r0 + k;
      om[k] = false;
      o1[k] = o2[k] = od[k] = 0.f;
      if (gx < cam.W && gy < cam.H) {
        const int64_t p = cam.pix_offset + (int64_t)gy * cam.W + gx;
        om[k] = mask[p] != 0;
        o1[k] = target[3 * p + c];
        o2[k] = rgb[3 * p + c];
        od[k] = d_rgb[3 * p + c];
      }
    }
#pragma unroll
    for (int k = 0; k < kSeg; ++k) {
      if (!om[k]) continue;
      const int64_t p = cam.pix_offset + (int64_t)(y0 + r0 + k) * cam.W + (x0 + col);
      d_rgb[3 * p + c] = od[k] + coef * (g[0][k] + 2.f * o2[k] * g[1][k] + o1[k] * g[2][k]);
    }
  }
}

// out[v]: k = 0 -> mean over all values, 1 -> mean over mask values (NaN if none)
// one CTA per view
__global__ void __launch_bounds__(kViewSumThreads) ssim_final_kernel(const double* __restrict__ partial,
                                                                    const int* __restrict__ prefix,
                                                                    const DevCam* __restrict__ cams,
                                                                    double* __restrict__ ssim,
                                                                    double* __restrict__ ssim_masked) {
  const int v = blockIdx.x;
  double t[3];
  view_block_sums<3>(partial, prefix[v], prefix[v + 1], t);
  if (threadIdx.x != 0) return;
  ssim[v] = t[0] / (3.0 * (double)cams[v].W * (double)cams[v].H);
  if (ssim_masked) ssim_masked[v] = t[2] > 0.0 ? t[1] / t[2] : __longlong_as_double(0x7ff8000000000000ll);
}

// partial[2 b]: sum of squared masked differences, partial[2 b + 1]: mask values
__global__ void __launch_bounds__(256) psnr_partial_kernel(const float* __restrict__ rgb,
                                                           const float* __restrict__ target,
                                                           const uint8_t* __restrict__ mask,
                                                           const DevCam* __restrict__ cams, int n_views,
                                                           const int* __restrict__ block_prefix,
                                                           double* __restrict__ partial) {
  __shared__ double red[2][8];
  const int b = blockIdx.x;
  const int v = view_of_tile(block_prefix, n_views, b);
  const DevCam& cam = cams[v];
  const int64_t npix = (int64_t)cam.W * cam.H;
  const int64_t lo = (int64_t)(b - block_prefix[v]) * kLossBlockPixels;
  const int64_t hi = (lo + kLossBlockPixels < npix) ? lo + kLossBlockPixels : npix;
  double se = 0.0, n = 0.0;
  for (int64_t k = lo + threadIdx.x; k < hi; k += 256) {
    const int64_t p = cam.pix_offset + k;
    if (!mask[p]) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double d = (double)target[3 * p + c] - (double)rgb[3 * p + c];
      se += d * d;
    }
    n += 3.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_down_sync(0xffffffffu, se, o);
    n += __shfl_down_sync(0xffffffffu, n, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = se;
    red[1][threadIdx.x >> 5] = n;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
    partial[2 * b + threadIdx.x] = t;
  }
}

// one CTA per view
__global__ void __launch_bounds__(kViewSumThreads) psnr_final_kernel(const double* __restrict__ partial,
                                                                    const int* __restrict__ block_prefix,
                                                                    double max_i, double* __restrict__ psnr) {
  const int v = blockIdx.x;
  double t[2];
  view_block_sums<2>(partial, block_prefix[v], block_prefix[v + 1], t);
  if (threadIdx.x != 0) return;
  const double se = t[0], n = t[1];
  if (n == 0.0) psnr[v] = __longlong_as_double(0x7ff8000000000000ll);
  else if (se == 0.0) psnr[v] = __longlong_as_double(0x7ff0000000000000ll);
  else psnr[v] = 20.0 * log10(max_i / sqrt(se / n));
}

Window make_window() {
  Window w;
  double g[2 * kR + 1], s = 0.0;
  for (int t = -kR; t <= kR; ++t) {
    g[t + kR] = std::exp(-(double)(t * t) / (2.0 * 1.5 * 1.5));
    s += g[t + kR];
  }
  for (int t = 0; t <= 2 * kR; ++t) w.w[t] = (float)(g[t] / s);
  return w;
}

}  // namespace

int ssim_tiles(int width, int height) { return ((width + kT - 1) / kT) * ((height + kT - 1) / kT); }

cudaError_t launch_ssim(const float* rgb, const float* target, const uint8_t* mask, const DevCam* cams, int n_views,
                        const int* tile_prefix, int n_tiles, int64_t p_total, float weight, double* partial,
                        float* gmap, double* ssim, double* ssim_masked, float* d_rgb, cudaStream_t s) {
  if (n_tiles == 0) return cudaSuccess;
  const Window w = make_window();
  ssim_stats_kernel<<<n_tiles, kThreadsSsim, 0, s>>>(rgb, target, mask, cams, n_views, tile_prefix, w, p_total,
                                                     partial, d_rgb ? gmap : nullptr);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  ssim_final_kernel<<<n_views, kViewSumThreads, 0, s>>>(partial, tile_prefix, cams, ssim, ssim_masked);
  e = launched();
  if (e != cudaSuccess || !d_rgb) return e;
  ssim_grad_kernel<<<n_tiles, kThreadsSsim, 0, s>>>(rgb, target, mask, cams, n_views, tile_prefix, w, p_total, gmap,
                                                    weight, d_rgb);
  return launched();
}

cudaError_t launch_masked_psnr(const float* rgb, const float* target, const uint8_t* mask, const DevCam* cams,
                               int n_views, const int* block_prefix, int n_blocks, double max_i, double* partial,
                               double* psnr, cudaStream_t s) {
  if (n_blocks > 0) {
    psnr_partial_kernel<<<n_blocks, 256, 0, s>>>(rgb, target, mask, cams, n_views, block_prefix, partial);
    cudaError_t e = launched();
    if (e != cudaSuccess) return e;
  }
  psnr_final_kernel<<<n_views, kViewSumThreads, 0, s>>>(partial, block_prefix, max_i, psnr);
  return launched();
}

}  // namespace ocgs
