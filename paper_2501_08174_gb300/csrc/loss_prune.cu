// Background loss (Eq. 1) with its fused adjoint, and the pruning keep-set
// compaction (Sec. 4.3).
#include "common.cuh"

namespace ocgs {
namespace {

constexpr int kLossThreads = 256;

// Each block reduces kLossBlockPixels pixels of one view in FP64, in a fixed
// order, and writes one partial sum; a second pass adds the partials of a view
// in block order, so the loss is bitwise reproducible.
__global__ void __launch_bounds__(kLossThreads) bg_loss_partial_kernel(
    const float* __restrict__ alpha, const uint8_t* __restrict__ mask, const DevCam* __restrict__ cams,
    int n_views, const int* __restrict__ block_prefix, float gamma, double* __restrict__ partial,
    float* __restrict__ d_alpha) {
  __shared__ double warp_part[kLossThreads / 32];
  const int b = blockIdx.x;
  const int v = view_of_tile(block_prefix, n_views, b);
  const DevCam& cam = cams[v];
  const int64_t npix = (int64_t)cam.W * cam.H;
  const int64_t lo = (int64_t)(b - block_prefix[v]) * kLossBlockPixels;
  const int64_t hi = (lo + kLossBlockPixels < npix) ? lo + kLossBlockPixels : npix;
  const float g = gamma / (float)npix;
  double acc = 0.0;
  for (int64_t k = lo + threadIdx.x; k < hi; k += kLossThreads) {
    const int64_t p = cam.pix_offset + k;
    const float bg = mask[p] ? 0.f : 1.f;
    acc += (double)alpha[p] * (double)bg;
    if (d_alpha) d_alpha[p] += g * bg;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLossThreads / 32; ++w) t += warp_part[w];
    partial[b] = t;
  }
}

// Masked L1 (Eq. 2, L1 part): |I M - R M| summed in FP64 per block, with the
// adjoint weight * sign(R - I) * M / (3 h w) added into d_rgb.
__global__ void __launch_bounds__(kLossThreads) l1_partial_kernel(
    const float* __restrict__ rgb, const float* __restrict__ target, const uint8_t* __restrict__ mask,
    const DevCam* __restrict__ cams, int n_views, const int* __restrict__ block_prefix, float weight,
    double* __restrict__ partial, float* __restrict__ d_rgb) {
  __shared__ double warp_part[kLossThreads / 32];
  const int b = blockIdx.x;
  const int v = view_of_tile(block_prefix, n_views, b);
  const DevCam& cam = cams[v];
  const int64_t npix = (int64_t)cam.W * cam.H;
  const int64_t lo = (int64_t)(b - block_prefix[v]) * kLossBlockPixels;
  const int64_t hi = (lo + kLossBlockPixels < npix) ? lo + kLossBlockPixels : npix;
  const float g = weight / (3.0f * (float)npix);
  double acc = 0.0;
  for (int64_t k = lo + threadIdx.x; k < hi; k += kLossThreads) {
    const int64_t p = cam.pix_offset + k;
    if (!mask[p]) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float d = rgb[3 * p + c] - target[3 * p + c];
      acc += fabs((double)d);
      if (d_rgb) d_rgb[3 * p + c] += d > 0.f ? g : (d < 0.f ? -g : 0.f);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLossThreads / 32; ++w) t += warp_part[w];
    partial[b] = t;
  }
}

__global__ void bg_loss_final_kernel(const double* __restrict__ partial, const int* __restrict__ block_prefix,
                                     const DevCam* __restrict__ cams, int n_views, double* __restrict__ loss) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  double t = 0.0;
  for (int b = block_prefix[v]; b < block_prefix[v + 1]; ++b) t += partial[b];
  loss[v] = t / ((double)cams[v].W * (double)cams[v].H);
}

__global__ void scale_kernel(double* __restrict__ x, int n, double f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= f;
}

__global__ void prune_flags_kernel(const float* __restrict__ score, uint32_t n, float tau,
                                   uint32_t* __restrict__ keep, uint32_t* __restrict__ border) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float s = score[i];
  keep[i] = s > tau ? 1u : 0u;
  border[i] = fabsf(s - tau) <= 1e-6f ? 1u : 0u;
}

__global__ void prune_compact_kernel(GaussPtrs in, uint32_t n, int k3, const uint32_t* __restrict__ keep,
                                     const uint32_t* __restrict__ keep_pos, const uint32_t* __restrict__ border,
                                     const uint32_t* __restrict__ border_pos, GaussOut out,
                                     int64_t* __restrict__ border_idx, int64_t border_cap) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (keep[i]) {
    const int64_t j = keep_pos[i];
    out.xyz[3 * j + 0] = in.xyz[3 * (int64_t)i + 0];
    out.xyz[3 * j + 1] = in.xyz[3 * (int64_t)i + 1];
    out.xyz[3 * j + 2] = in.xyz[3 * (int64_t)i + 2];
    reinterpret_cast<float4*>(out.quat)[j] = reinterpret_cast<const float4*>(in.quat)[i];
    reinterpret_cast<float2*>(out.scale)[j] = reinterpret_cast<const float2*>(in.scale)[i];
    out.opacity[j] = in.opacity[i];
    for (int k = 0; k < k3; ++k) out.sh[j * k3 + k] = in.sh[(int64_t)i * k3 + k];
  }
  if (border_idx && border[i]) {
    const int64_t j = border_pos[i];
    if (j < border_cap) border_idx[j] = i;
  }
}

}  // namespace

cudaError_t launch_background_loss(const float* alpha, const uint8_t* mask, const DevCam* cams,
                                   int n_views, const int* block_prefix, int n_blocks, float gamma,
                                   double* partial, double* loss, float* d_alpha, cudaStream_t s) {
  if (n_blocks > 0) {
    bg_loss_partial_kernel<<<n_blocks, kLossThreads, 0, s>>>(alpha, mask, cams, n_views, block_prefix,
                                                             gamma, partial, d_alpha);
    cudaError_t e = launched();
    if (e != cudaSuccess) return e;
  }
  bg_loss_final_kernel<<<(n_views + 127) / 128, 128, 0, s>>>(partial, block_prefix, cams, n_views, loss);
  return launched();
}

cudaError_t launch_masked_l1(const float* rgb, const float* target, const uint8_t* mask, const DevCam* cams,
                             int n_views, const int* block_prefix, int n_blocks, float weight, double* partial,
                             double* loss, float* d_rgb, cudaStream_t s) {
  if (n_blocks > 0) {
    l1_partial_kernel<<<n_blocks, kLossThreads, 0, s>>>(rgb, target, mask, cams, n_views, block_prefix, weight,
                                                        partial, d_rgb);
    cudaError_t e = launched();
    if (e != cudaSuccess) return e;
  }
  // the final pass divides by h*w; the L1 mean is over 3*h*w values
  bg_loss_final_kernel<<<(n_views + 127) / 128, 128, 0, s>>>(partial, block_prefix, cams, n_views, loss);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  scale_kernel<<<(n_views + 127) / 128, 128, 0, s>>>(loss, n_views, 1.0 / 3.0);
  return launched();
}

cudaError_t launch_prune_flags(const float* score, uint32_t n, float threshold, uint32_t* keep,
                               uint32_t* border, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  prune_flags_kernel<<<(n + 255) / 256, 256, 0, s>>>(score, n, threshold, keep, border);
  return launched();
}

cudaError_t launch_prune_compact(const GaussPtrs& in, uint32_t n, int sh_degree, const uint32_t* keep,
                                 const uint32_t* keep_pos, const uint32_t* border,
                                 const uint32_t* border_pos, GaussOut out, int64_t* border_idx,
                                 int64_t border_cap, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int k3 = 3 * (sh_degree + 1) * (sh_degree + 1);
  prune_compact_kernel<<<(n + 255) / 256, 256, 0, s>>>(in, n, k3, keep, keep_pos, border, border_pos, out,
                                                       border_idx, border_cap);
  return launched();
}

}  // namespace ocgs
