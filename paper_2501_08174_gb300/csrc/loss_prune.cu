// Background loss (Eq. 1) with its fused adjoint, and the pruning keep-set
// compaction (Sec. 4.3).
#include "common.cuh"
#include "ocgs.h"

#include <cmath>
#include <cstring>
#include <mutex>

namespace ocgs {
namespace {

constexpr int kLossThreads = 256;

// Each block reduces kLossBlockPixels pixels of one view, in a fixed order
// (compensated float32 sums per thread, merged into one FP64 partial per block),
// and a second pass adds the partials of a view in block order, so the loss is
// bitwise reproducible.
__global__ void __launch_bounds__(kLossThreads) bg_loss_partial_kernel(
    const float* __restrict__ alpha, const uint8_t* __restrict__ mask, const DevCam* __restrict__ cams,
    int n_views, const int* __restrict__ block_prefix, float gamma, double* __restrict__ partial,
    float* __restrict__ d_alpha) {
  const int b = blockIdx.x;
  const int v = view_of_tile(block_prefix, n_views, b);
  const DevCam& cam = cams[v];
  const int64_t npix = (int64_t)cam.W * cam.H;
  const int64_t lo = (int64_t)(b - block_prefix[v]) * kLossBlockPixels;
  const int64_t hi = (lo + kLossBlockPixels < npix) ? lo + kLossBlockPixels : npix;
  const float g = gamma / (float)npix;
  CompSum acc[1];
  for (int64_t k = lo + threadIdx.x; k < hi; k += kLossThreads) {
    const int64_t p = cam.pix_offset + k;
    const float bg = mask[p] ? 0.f : 1.f;
    acc[0].add(alpha[p] * bg);  // alpha (1 - M) is exact
    if (d_alpha) d_alpha[p] += g * bg;
  }
  block_comp_sums<kLossThreads, 1>(acc, partial + b);
}

// Masked L1 (Eq. 2, L1 part): |I M - R M| summed per block, with the adjoint
// weight * sign(R - I) * M / (3 h w) added into d_rgb.  Each difference is
// taken exactly as a float pair (TwoSum: R - I = d + e, |e| <= ulp(d) / 2, so
// |R - I| = |d| + sign(d) e) and summed with compensation, so the loss differs
// from the exact one by rounding far below float precision; the sign of d is
// the sign of the exact difference (d = 0 only when R = I).
__global__ void __launch_bounds__(kLossThreads) l1_partial_kernel(
    const float* __restrict__ rgb, const float* __restrict__ target, const uint8_t* __restrict__ mask,
    const DevCam* __restrict__ cams, int n_views, const int* __restrict__ block_prefix, float weight,
    double* __restrict__ partial, float* __restrict__ d_rgb) {
  const int b = blockIdx.x;
  const int v = view_of_tile(block_prefix, n_views, b);
  const DevCam& cam = cams[v];
  const int64_t npix = (int64_t)cam.W * cam.H;
  const int64_t lo = (int64_t)(b - block_prefix[v]) * kLossBlockPixels;
  const int64_t hi = (lo + kLossBlockPixels < npix) ? lo + kLossBlockPixels : npix;
  const float g = weight / (3.0f * (float)npix);
  CompSum acc[1];
  for (int64_t k = lo + threadIdx.x; k < hi; k += kLossThreads) {
    const int64_t p = cam.pix_offset + k;
    if (!mask[p]) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float e;
      const float d = two_sum(rgb[3 * p + c], -target[3 * p + c], e);
      acc[0].add(fabsf(d), d > 0.f ? e : -e);
      if (d_rgb) d_rgb[3 * p + c] += d > 0.f ? g : (d < 0.f ? -g : 0.f);
    }
  }
  block_comp_sums<kLossThreads, 1>(acc, partial + b);
}

// one CTA per view
__global__ void __launch_bounds__(kViewSumThreads) bg_loss_final_kernel(const double* __restrict__ partial,
                                                                       const int* __restrict__ block_prefix,
                                                                       const DevCam* __restrict__ cams,
                                                                       double* __restrict__ loss) {
  const int v = blockIdx.x;
  double t;
  view_block_sums<1>(partial, block_prefix[v], block_prefix[v + 1], &t);
  if (threadIdx.x == 0) loss[v] = t / ((double)cams[v].W * (double)cams[v].H);
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
  bg_loss_final_kernel<<<n_views, kViewSumThreads, 0, s>>>(partial, block_prefix, cams, loss);
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
  bg_loss_final_kernel<<<n_views, kViewSumThreads, 0, s>>>(partial, block_prefix, cams, loss);
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

// ----------------------------------------------------------------------------- allocation-free background loss
//
// ocgs_background_loss_noalloc computes exactly what ocgs_background_loss
// computes, with the same kernels, but needs no context and allocates no
// device memory: its scratch (the per-block FP64 partial sums, the view table
// and the block prefix) lives in one file-scope device array of fixed size,
// which every GPU that loads this library holds until the process exits.
// Host code cannot hand that array to a kernel by name (in host code the name
// is only a stand-in), so the first call on each device, with that device
// current, looks its device address up with cudaGetSymbolAddress and keeps it.
// The view sizes travel to the device as a kernel argument (copied by value
// at launch), and a one-block kernel writes the view table and the block
// prefix into the array, so no host buffer is read after the call returns.
namespace {

constexpr int kNoAllocMaxViews = 1024;
constexpr int kNoAllocMaxBlocks = 65536;  // 65536 blocks x 4096 pixels = 268,435,456 pixels per call
constexpr size_t kNoAllocPartialBytes = sizeof(double) * kNoAllocMaxBlocks;
constexpr size_t kNoAllocCamOffset = kNoAllocPartialBytes;
constexpr size_t kNoAllocCamBytes = ((sizeof(ocgs::DevCam) * kNoAllocMaxViews) + 255) & ~(size_t)255;
constexpr size_t kNoAllocPrefixOffset = kNoAllocCamOffset + kNoAllocCamBytes;
constexpr size_t kNoAllocBytes = kNoAllocPrefixOffset + sizeof(int) * (kNoAllocMaxViews + 1);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// width and height of every view (each at most 16384), passed by value
struct NoAllocViews {
  uint16_t w[kNoAllocMaxViews];
  uint16_t h[kNoAllocMaxViews];
};

// One block of kNoAllocMaxViews threads: thread v fills the view table entry of
// view v (size and first pixel) and the block prefix (first loss block of v).
__global__ void __launch_bounds__(kNoAllocMaxViews) noalloc_setup_kernel(const NoAllocViews views, int n_views,
                                                                         ocgs::DevCam* __restrict__ cams,
                                                                         int* __restrict__ prefix) {
  __shared__ long long s_pix[kNoAllocMaxViews];
  __shared__ int s_blk[kNoAllocMaxViews];
  const int v = threadIdx.x;
  const long long np = v < n_views ? (long long)views.w[v] * views.h[v] : 0;
  s_pix[v] = np;
  s_blk[v] = (int)((np + ocgs::kLossBlockPixels - 1) / ocgs::kLossBlockPixels);
  __syncthreads();
  // inclusive Hillis-Steele scan over the views
  for (int o = 1; o < kNoAllocMaxViews; o <<= 1) {
    const long long pp = v >= o ? s_pix[v - o] : 0;
    const int bb = v >= o ? s_blk[v - o] : 0;
    __syncthreads();
    s_pix[v] += pp;
    s_blk[v] += bb;
    __syncthreads();
  }
  if (v < n_views) {
    ocgs::DevCam d;
    memset(&d, 0, sizeof(d));
    d.W = views.w[v];
    d.H = views.h[v];
    d.pix_offset = s_pix[v] - np;
    cams[v] = d;
    prefix[v] = s_blk[v] - (int)((np + ocgs::kLossBlockPixels - 1) / ocgs::kLossBlockPixels);
  }
  if (v == n_views - 1) prefix[n_views] = s_blk[v];
}

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_addr[kNoAllocMaxDevices];  // device address of the array, per device

}  // namespace

extern "C" ocgs_status ocgs_background_loss_noalloc(const float* alpha, const uint8_t* mask,
                                                    const ocgs_camera* cams, int32_t n_views, float gamma,
                                                    double* loss, float* d_alpha, void* stream) {
  if (!alpha || !mask || !loss || !cams) return OCGS_ERR_ARG;
  if (n_views < 1) return OCGS_ERR_ARG;
  if (n_views > kNoAllocMaxViews) return OCGS_ERR_CAPACITY;  // beyond the static view table
  if (!std::isfinite(gamma)) return OCGS_ERR_ARG;
  NoAllocViews views;
  int64_t blocks = 0;
  for (int v = 0; v < n_views; ++v) {
    if (cams[v].width < 1 || cams[v].height < 1 || cams[v].width > 16384 || cams[v].height > 16384)
      return OCGS_ERR_ARG;
    const int64_t np = (int64_t)cams[v].width * cams[v].height;
    blocks += (np + ocgs::kLossBlockPixels - 1) / ocgs::kLossBlockPixels;
    views.w[v] = (uint16_t)cams[v].width;
    views.h[v] = (uint16_t)cams[v].height;
  }
  if (blocks > kNoAllocMaxBlocks) return OCGS_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OCGS_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return OCGS_ERR_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return OCGS_ERR_CUDA;
      g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_noalloc_addr[dev];
  }
  ocgs::DevCam* d_cams = reinterpret_cast<ocgs::DevCam*>(base + kNoAllocCamOffset);
  int* d_prefix = reinterpret_cast<int*>(base + kNoAllocPrefixOffset);
  double* d_partial = reinterpret_cast<double*>(base);
  noalloc_setup_kernel<<<1, kNoAllocMaxViews, 0, s>>>(views, n_views, d_cams, d_prefix);
  if (ocgs::launched() != cudaSuccess) return OCGS_ERR_CUDA;
  if (ocgs::launch_background_loss(alpha, mask, d_cams, n_views, d_prefix, (int)blocks, gamma, d_partial, loss,
                                   d_alpha, s) != cudaSuccess)
    return OCGS_ERR_CUDA;
  return OCGS_OK;
}
