// SSIM of masked images and masked PSNR (Sec. 5), and the D-SSIM part of the
// photometric loss that Eq. 2 evaluates on masked images.
//
// SSIM statistics are windowed means under an 11x11 Gaussian window of sigma
// 1.5, zero outside the image; the window is separable, so every block stages
// a 26x26 patch (its 16x16 output tile plus a 5-pixel halo) of both masked
// images in shared memory and applies the 11 taps along rows, then columns.
// The adjoint of the mean SSIM needs, at every pixel q,
//     sum_p dS(p)/dE[x2](p) G(p-q) + 2 x2(q) sum_p dS(p)/dE[x2^2](p) G(p-q)
//                                 +   x1(q) sum_p dS(p)/dE[x1 x2](p) G(p-q),
// i.e. the same window applied to three per-pixel maps, which the first pass
// writes and the second blurs.
#include "common.cuh"

#include <cmath>

namespace ocgs {
namespace {

constexpr int kT = 16;               // output tile side
constexpr int kR = 5;                // window radius
constexpr int kP = kT + 2 * kR;      // staged patch side (26)
constexpr int kThreadsSsim = kT * kT;
constexpr float kC1 = 0.0001f;       // (0.01)^2
constexpr float kC2 = 0.0009f;       // (0.03)^2

struct Window {
  float w[2 * kR + 1];
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

// partial[3 b + k]: k = 0 sum of S over the tile's values, 1 sum over its mask
// values, 2 number of mask values.  gmap [P,3,3] (or NULL): per pixel and
// channel, dS/dE[x2], dS/dE[x2^2], dS/dE[x1 x2].
__global__ void __launch_bounds__(kThreadsSsim) ssim_stats_kernel(
    const float* __restrict__ rgb, const float* __restrict__ target, const uint8_t* __restrict__ mask,
    const DevCam* __restrict__ cams, int n_views, const int* __restrict__ prefix, const Window win,
    double* __restrict__ partial, float* __restrict__ gmap) {
  __shared__ float s1[3][kP][kP + 1], s2[3][kP][kP + 1];  // masked target x1, masked render x2
  __shared__ float h[5][kP][kT + 1];
  __shared__ double red[3][kThreadsSsim / 32];
  int v, x0, y0;
  tile_origin(prefix, n_views, cams, &v, &x0, &y0);
  const DevCam& cam = cams[v];
  const int tid = threadIdx.x;
  for (int i = tid; i < kP * kP; i += kThreadsSsim) {
    const int py = i / kP, px = i % kP;
    const int gy = y0 - kR + py, gx = x0 - kR + px;
    float a[3] = {0.f, 0.f, 0.f}, b[3] = {0.f, 0.f, 0.f};
    if (gy >= 0 && gy < cam.H && gx >= 0 && gx < cam.W) {
      const int64_t p = cam.pix_offset + (int64_t)gy * cam.W + gx;
      if (mask[p]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          a[c] = target[3 * p + c];
          b[c] = rgb[3 * p + c];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s1[c][py][px] = a[c];
      s2[c][py][px] = b[c];
    }
  }
  const int tx = tid % kT, ty = tid / kT;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool inside = gx < cam.W && gy < cam.H;
  const int64_t p = cam.pix_offset + (int64_t)gy * cam.W + gx;
  const bool m = inside && mask[p];
  double sum_all = 0.0, sum_m = 0.0;
  for (int c = 0; c < 3; ++c) {
    __syncthreads();
    for (int i = tid; i < kP * kT; i += kThreadsSsim) {
      const int r = i / kT, j = i % kT;
      float m1 = 0.f, m2 = 0.f, e11 = 0.f, e22 = 0.f, e12 = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kR; ++t) {
        const float a = s1[c][r][j + t], b = s2[c][r][j + t], w = win.w[t];
        m1 = __fmaf_rn(w, a, m1);
        m2 = __fmaf_rn(w, b, m2);
        e11 = __fmaf_rn(w, a * a, e11);
        e22 = __fmaf_rn(w, b * b, e22);
        e12 = __fmaf_rn(w, a * b, e12);
      }
      h[0][r][j] = m1;
      h[1][r][j] = m2;
      h[2][r][j] = e11;
      h[3][r][j] = e22;
      h[4][r][j] = e12;
    }
    __syncthreads();
    if (inside) {
      float mu1 = 0.f, mu2 = 0.f, e11 = 0.f, e22 = 0.f, e12 = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kR; ++t) {
        const float w = win.w[t];
        mu1 = __fmaf_rn(w, h[0][ty + t][tx], mu1);
        mu2 = __fmaf_rn(w, h[1][ty + t][tx], mu2);
        e11 = __fmaf_rn(w, h[2][ty + t][tx], e11);
        e22 = __fmaf_rn(w, h[3][ty + t][tx], e22);
        e12 = __fmaf_rn(w, h[4][ty + t][tx], e12);
      }
      const float v11 = e11 - mu1 * mu1, v22 = e22 - mu2 * mu2, v12 = e12 - mu1 * mu2;
      const float n1 = 2.f * mu1 * mu2 + kC1, n2 = 2.f * v12 + kC2;
      const float d1 = mu1 * mu1 + mu2 * mu2 + kC1, d2 = v11 + v22 + kC2;
      const float inv = 1.f / (d1 * d2);
      const float S = n1 * n2 * inv;
      sum_all += (double)S;
      if (m) sum_m += (double)S;
      if (gmap) {
        // partial derivatives at fixed (mu, sigma), then through sigma22 = E[x2^2] - mu2^2
        // and sigma12 = E[x1 x2] - mu1 mu2 onto the three windowed means of x2
        const float dmu2 = 2.f * mu1 * n2 * inv - S * 2.f * mu2 / d1;
        const float dv22 = -S / d2;
        const float dv12 = 2.f * n1 * inv;
        float* gm = gmap + 9 * p + 3 * c;
        gm[0] = dmu2 - 2.f * mu2 * dv22 - mu1 * dv12;
        gm[1] = dv22;
        gm[2] = dv12;
      }
    }
  }
  // block sums (fixed order: warp shuffles, then warps in order)
  double cnt = m ? 3.0 : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum_all += __shfl_down_sync(0xffffffffu, sum_all, o);
    sum_m += __shfl_down_sync(0xffffffffu, sum_m, o);
    cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = sum_all;
    red[1][tid >> 5] = sum_m;
    red[2][tid >> 5] = cnt;
  }
  __syncthreads();
  if (tid < 3) {
    double t = 0.0;
    for (int w = 0; w < kThreadsSsim / 32; ++w) t += red[tid][w];
    partial[3 * blockIdx.x + tid] = t;
  }
}

// d_rgb(q) += coef_v M(q) [G*a + 2 x2 G*b + x1 G*c](q), coef_v = -weight / (3 h w)
__global__ void __launch_bounds__(kThreadsSsim) ssim_grad_kernel(
    const float* __restrict__ rgb, const float* __restrict__ target, const uint8_t* __restrict__ mask,
    const DevCam* __restrict__ cams, int n_views, const int* __restrict__ prefix, const Window win,
    const float* __restrict__ gmap, float weight, float* __restrict__ d_rgb) {
  __shared__ float sg[9][kP][kP + 1];
  __shared__ float h[9][kP][kT + 1];
  int v, x0, y0;
  tile_origin(prefix, n_views, cams, &v, &x0, &y0);
  const DevCam& cam = cams[v];
  const int tid = threadIdx.x;
  for (int i = tid; i < kP * kP; i += kThreadsSsim) {
    const int py = i / kP, px = i % kP;
    const int gy = y0 - kR + py, gx = x0 - kR + px;
    const bool in = gy >= 0 && gy < cam.H && gx >= 0 && gx < cam.W;
    const int64_t p = cam.pix_offset + (int64_t)gy * cam.W + gx;
#pragma unroll
    for (int k = 0; k < 9; ++k) sg[k][py][px] = in ? gmap[9 * p + k] : 0.f;
  }
  __syncthreads();
  for (int i = tid; i < kP * kT; i += kThreadsSsim) {
    const int r = i / kT, j = i % kT;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float acc = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kR; ++t) acc = __fmaf_rn(win.w[t], sg[k][r][j + t], acc);
      h[k][r][j] = acc;
    }
  }
  __syncthreads();
  const int tx = tid % kT, ty = tid / kT;
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx >= cam.W || gy >= cam.H) return;
  const int64_t p = cam.pix_offset + (int64_t)gy * cam.W + gx;
  if (!mask[p]) return;  // x2 = R M: no gradient where M = 0
  const float coef = -weight / (3.f * (float)cam.W * (float)cam.H);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float ga = 0.f, gb = 0.f, gc = 0.f;
#pragma unroll
    for (int t = 0; t <= 2 * kR; ++t) {
      const float w = win.w[t];
      ga = __fmaf_rn(w, h[3 * c][ty + t][tx], ga);
      gb = __fmaf_rn(w, h[3 * c + 1][ty + t][tx], gb);
      gc = __fmaf_rn(w, h[3 * c + 2][ty + t][tx], gc);
    }
    const float x1 = target[3 * p + c], x2 = rgb[3 * p + c];
    d_rgb[3 * p + c] += coef * (ga + 2.f * x2 * gb + x1 * gc);
  }
}

// out[v]: k = 0 -> mean over all values, 1 -> mean over mask values (NaN if none)
__global__ void ssim_final_kernel(const double* __restrict__ partial, const int* __restrict__ prefix,
                                  const DevCam* __restrict__ cams, int n_views, double* __restrict__ ssim,
                                  double* __restrict__ ssim_masked) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  double a = 0.0, m = 0.0, n = 0.0;
  for (int b = prefix[v]; b < prefix[v + 1]; ++b) {
    a += partial[3 * b];
    m += partial[3 * b + 1];
    n += partial[3 * b + 2];
  }
  ssim[v] = a / (3.0 * (double)cams[v].W * (double)cams[v].H);
  if (ssim_masked) ssim_masked[v] = n > 0.0 ? m / n : __longlong_as_double(0x7ff8000000000000ll);
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

__global__ void psnr_final_kernel(const double* __restrict__ partial, const int* __restrict__ block_prefix,
                                  int n_views, double max_i, double* __restrict__ psnr) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  double se = 0.0, n = 0.0;
  for (int b = block_prefix[v]; b < block_prefix[v + 1]; ++b) {
    se += partial[2 * b];
    n += partial[2 * b + 1];
  }
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
                        const int* tile_prefix, int n_tiles, float weight, double* partial, float* gmap,
                        double* ssim, double* ssim_masked, float* d_rgb, cudaStream_t s) {
  if (n_tiles == 0) return cudaSuccess;
  const Window w = make_window();
  ssim_stats_kernel<<<n_tiles, kThreadsSsim, 0, s>>>(rgb, target, mask, cams, n_views, tile_prefix, w, partial,
                                                     d_rgb ? gmap : nullptr);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  ssim_final_kernel<<<(n_views + 127) / 128, 128, 0, s>>>(partial, tile_prefix, cams, n_views, ssim, ssim_masked);
  e = launched();
  if (e != cudaSuccess || !d_rgb) return e;
  ssim_grad_kernel<<<n_tiles, kThreadsSsim, 0, s>>>(rgb, target, mask, cams, n_views, tile_prefix, w, gmap, weight,
                                                    d_rgb);
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
  psnr_final_kernel<<<(n_views + 127) / 128, 128, 0, s>>>(partial, block_prefix, n_views, max_i, psnr);
  return launched();
}

}  // namespace ocgs
