// The 2DGS regularisers that Eq. 3 adds to the loss, on the composited planes of
// every view:
//  * depth distortion: per pixel sum_{i,j} w_i w_j (z_i - z_j)^2 = 2 (A Q - D^2),
//    from A = sum w, D = sum w z and Q = sum w z^2; mean over the view's pixels;
//  * normal consistency: per pixel sum_i w_i (1 - n_i . N) = A - N . N_r, with N_r
//    = sum w n and N the unit normal of the expected-depth surface, from central
//    differences of the camera-frame points P = (D / A) ray at the four
//    neighbours, turned towards the camera; counted where the pixel and its four
//    neighbours lie inside the image and have A > a_min; summed and divided by h w.
// Both adjoints are written as cotangents of the planes, which the backward
// rasterizer takes.  Every pixel writes only its own entries: the normal
// consistency's stencil adjoint goes through a per-pixel map that a second pass
// gathers.
#include "common.cuh"

namespace ocgs {
namespace {

constexpr int kRegThreads = 256;
constexpr int kNcUnroll = 2;  // pixels per thread whose stencil loads are in flight together

struct Block {
  int v;
  int64_t lo, hi;  // pixels [lo, hi) of view v
};

__device__ __forceinline__ Block loss_block(const int* block_prefix, int n_views, const DevCam* cams) {
  Block b;
  b.v = view_of_tile(block_prefix, n_views, blockIdx.x);
  const DevCam& cam = cams[b.v];
  const int64_t npix = (int64_t)cam.W * cam.H;
  b.lo = (int64_t)(blockIdx.x - block_prefix[b.v]) * kLossBlockPixels;
  b.hi = (b.lo + kLossBlockPixels < npix) ? b.lo + kLossBlockPixels : npix;
  return b;
}

// a * b exactly, as the float pair p + e (FMA: e = a b - p)
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
  const float p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
  return p;
}

__global__ void __launch_bounds__(kRegThreads) depth_distortion_kernel(
    const float* __restrict__ alpha, const float* __restrict__ depth, const float* __restrict__ depth2,
    const DevCam* __restrict__ cams, int n_views, const int* __restrict__ block_prefix, float weight,
    double* __restrict__ partial, float* __restrict__ d_alpha, float* __restrict__ d_depth,
    float* __restrict__ d_depth2) {
  const Block b = loss_block(block_prefix, n_views, cams);
  const DevCam& cam = cams[b.v];
  const float k = weight / ((float)cam.W * (float)cam.H);
  CompSum acc[1];
  for (int64_t i = b.lo + threadIdx.x; i < b.hi; i += kRegThreads) {
    const int64_t p = cam.pix_offset + i;
    const float A = alpha[p], D = depth[p], Q = depth2[p];
    // A Q - D^2 from the exact products, so that its cancellation (the blended depths
    // close together) costs no accuracy: (aq + ea) - (dd + ed), the leading difference
    // kept exactly by two_sum
    float ea, ed, es;
    const float aq = two_prod(A, Q, ea), dd = two_prod(D, D, ed);
    const float s0 = two_sum(aq, -dd, es);
    acc[0].add(2.f * s0, 2.f * __fadd_rn(es, __fsub_rn(ea, ed)));
    if (d_alpha) {
      d_alpha[p] += k * 2.f * Q;
      d_depth[p] += k * -4.f * D;
      d_depth2[p] += k * 2.f * A;
    }
  }
  block_comp_sums<kRegThreads, 1>(acc, partial + blockIdx.x);
}

struct Pt {
  float3 P;
  bool ok;
};

// The camera-frame point of pixel (x, y) from its alpha A and depth D (A = NaN
// outside the image): P = (D / A) ray, counted where A > a_min.
__device__ __forceinline__ Pt surface_point(float A, float D, const DevCam& cam, int x, int y, float a_min) {
  Pt r;
  r.ok = false;
  r.P = make_float3(0.f, 0.f, 0.f);
  if (!(A > a_min)) return r;
  const float d = D / A;
  r.P = make_float3(d * (((float)x + 0.5f - cam.cx) / cam.fx), d * (((float)y + 0.5f - cam.cy) / cam.fy), d);
  r.ok = true;
  return r;
}

// Alpha and depth of the five stencil pixels (centre, x + 1, x - 1, y + 1, y - 1) of
// pixel (x, y) and its accumulated normal, NaN alpha outside the image.
struct Stencil {
  float A[5], D[5];
  float3 Nr;
};
__host__ __device__ constexpr int stencil_dx(int j) { return (j == 1) - (j == 2); }
__host__ __device__ constexpr int stencil_dy(int j) { return (j == 3) - (j == 4); }

__device__ __forceinline__ void load_stencil(const float* __restrict__ alpha, const float* __restrict__ depth,
                                             const float* __restrict__ normal, const DevCam& cam, int x, int y,
                                             Stencil& st) {
  const int64_t p = cam.pix_offset + (int64_t)y * cam.W + x;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int xx = x + stencil_dx(j), yy = y + stencil_dy(j);
    st.A[j] = __int_as_float(0x7fc00000);
    st.D[j] = 0.f;
    if (xx >= 0 && xx < cam.W && yy >= 0 && yy < cam.H) {
      const int64_t q = p + stencil_dx(j) + (int64_t)stencil_dy(j) * cam.W;
      st.A[j] = alpha[q];
      st.D[j] = depth[q];
    }
  }
  st.Nr = make_float3(normal[3 * p], normal[3 * p + 1], normal[3 * p + 2]);
}

__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// gmap [P][6] (or NULL): d(weight term)/d(dx) and d/d(dy) of the pixel's central differences
__global__ void __launch_bounds__(kRegThreads, 4) normal_consistency_kernel(
    const float* __restrict__ alpha, const float* __restrict__ depth, const float* __restrict__ normal,
    const DevCam* __restrict__ cams, int n_views, const int* __restrict__ block_prefix, float weight, float a_min,
    double* __restrict__ partial, float* __restrict__ gmap, float* __restrict__ d_alpha,
    float* __restrict__ d_normal) {
  const Block b = loss_block(block_prefix, n_views, cams);
  const DevCam& cam = cams[b.v];
  const float k = weight / ((float)cam.W * (float)cam.H);
  CompSum acc[1];
  // kNcUnroll pixels per round, every load of the round issued before any is used
  for (int64_t i0 = b.lo + threadIdx.x; i0 < b.hi; i0 += kNcUnroll * kRegThreads) {
    Stencil st[kNcUnroll];
#pragma unroll
    for (int u = 0; u < kNcUnroll; ++u) {
      const int64_t i = i0 + u * kRegThreads;
      if (i < b.hi) load_stencil(alpha, depth, normal, cam, (int)(i % cam.W), (int)(i / cam.W), st[u]);
    }
#pragma unroll
    for (int u = 0; u < kNcUnroll; ++u) {
      const int64_t i = i0 + u * kRegThreads;
      if (i >= b.hi) break;
      const int64_t p = cam.pix_offset + i;
      const int x = (int)(i % cam.W), y = (int)(i / cam.W);
      float g6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const Pt c = surface_point(st[u].A[0], st[u].D[0], cam, x, y, a_min);
      const Pt xp = surface_point(st[u].A[1], st[u].D[1], cam, x + 1, y, a_min);
      const Pt xm = surface_point(st[u].A[2], st[u].D[2], cam, x - 1, y, a_min);
      const Pt yp = surface_point(st[u].A[3], st[u].D[3], cam, x, y + 1, a_min);
      const Pt ym = surface_point(st[u].A[4], st[u].D[4], cam, x, y - 1, a_min);
      if (c.ok && xp.ok && xm.ok && yp.ok && ym.ok) {
        const float3 dx = sub3(xp.P, xm.P), dy = sub3(yp.P, ym.P);
        const float3 cr = cross3(dx, dy);
        const float len = sqrtf(dot3(cr, cr));
        if (len > 0.f) {
          const float3 ch = make_float3(cr.x / len, cr.y / len, cr.z / len);
          const float s = dot3(ch, c.P) > 0.f ? -1.f : 1.f;  // turned towards the camera
          const float3 N = make_float3(s * ch.x, s * ch.y, s * ch.z);
          const float3 Nr = st[u].Nr;
          const float A = st[u].A[0];
          float e;
          const float t = two_sum(A, -dot3(N, Nr), e);  // A - N . N_r exactly
          acc[0].add(t, e);
          if (gmap) {
            d_alpha[p] += k;
            d_normal[3 * p] -= k * N.x;
            d_normal[3 * p + 1] -= k * N.y;
            d_normal[3 * p + 2] -= k * N.z;
            // term depends on cr through N = s cr / |cr|: g_cr = s (I - ch ch^T) g_N / |cr|, g_N = -k Nr
            const float3 gN = make_float3(-k * Nr.x, -k * Nr.y, -k * Nr.z);
            const float pr = dot3(ch, gN);
            const float3 gc = make_float3(s * (gN.x - ch.x * pr) / len, s * (gN.y - ch.y * pr) / len,
                                          s * (gN.z - ch.z * pr) / len);
            const float3 gdx = cross3(dy, gc), gdy = cross3(gc, dx);  // d(gc . (dx x dy))
            g6[0] = gdx.x; g6[1] = gdx.y; g6[2] = gdx.z;
            g6[3] = gdy.x; g6[4] = gdy.y; g6[5] = gdy.z;
          }
        }
      }
      if (gmap) {
#pragma unroll
        for (int j = 0; j < 6; ++j) gmap[6 * p + j] = g6[j];
      }
    }
  }
  block_comp_sums<kRegThreads, 1>(acc, partial + blockIdx.x);
}

// point gradient of pixel q: it is the x+1 point of q - x, the x-1 point of
// q + x, the y+1 point of q - W and the y-1 point of q + W; then P = (D / A) ray
__global__ void __launch_bounds__(kRegThreads, 4) normal_consistency_gather_kernel(
    const float* __restrict__ alpha, const float* __restrict__ depth, const DevCam* __restrict__ cams, int n_views,
    const int* __restrict__ block_prefix, float a_min, const float* __restrict__ gmap, float* __restrict__ d_alpha,
    float* __restrict__ d_depth) {
  const Block b = loss_block(block_prefix, n_views, cams);
  const DevCam& cam = cams[b.v];
  // kNcUnroll pixels per round: their alphas and depths are loaded together, then the
  // neighbours' map entries of the counted ones, then the sums
  for (int64_t i0 = b.lo + threadIdx.x; i0 < b.hi; i0 += kNcUnroll * kRegThreads) {
    float A[kNcUnroll], D[kNcUnroll];
#pragma unroll
    for (int u = 0; u < kNcUnroll; ++u) {
      const int64_t i = i0 + u * kRegThreads;
      A[u] = 0.f;
      D[u] = 0.f;
      if (i < b.hi) {
        A[u] = alpha[cam.pix_offset + i];
        D[u] = depth[cam.pix_offset + i];
      }
    }
    float m[kNcUnroll][12];  // x-1, x+1 (their dx terms), y-1, y+1 (their dy terms)
#pragma unroll
    for (int u = 0; u < kNcUnroll; ++u) {
      const int64_t i = i0 + u * kRegThreads;
#pragma unroll
      for (int j = 0; j < 12; ++j) m[u][j] = 0.f;
      if (i < b.hi && A[u] > a_min) {  // else not a point of any counted stencil
        const int64_t q = cam.pix_offset + i;
        const int x = (int)(i % cam.W), y = (int)(i / cam.W);
        const int64_t nb[4] = {q - 1, q + 1, q - cam.W, q + cam.W};
        const bool in[4] = {x > 0, x + 1 < cam.W, y > 0, y + 1 < cam.H};
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          if (in[n]) {
            const float* e = gmap + 6 * nb[n] + (n < 2 ? 0 : 3);
            m[u][3 * n] = e[0];
            m[u][3 * n + 1] = e[1];
            m[u][3 * n + 2] = e[2];
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kNcUnroll; ++u) {
      const int64_t i = i0 + u * kRegThreads;
      if (i >= b.hi || !(A[u] > a_min)) continue;
      const int64_t q = cam.pix_offset + i;
      const int x = (int)(i % cam.W), y = (int)(i / cam.W);
      // the same sums as term by term over the present neighbours (an absent one adds +0)
      float3 g = make_float3(0.f, 0.f, 0.f);
      g.x += m[u][0]; g.y += m[u][1]; g.z += m[u][2];
      g.x -= m[u][3]; g.y -= m[u][4]; g.z -= m[u][5];
      g.x += m[u][6]; g.y += m[u][7]; g.z += m[u][8];
      g.x -= m[u][9]; g.y -= m[u][10]; g.z -= m[u][11];
      const float3 ray = make_float3(((float)x + 0.5f - cam.cx) / cam.fx, ((float)y + 0.5f - cam.cy) / cam.fy, 1.f);
      const float gr = dot3(g, ray);
      d_depth[q] += gr / A[u];
      d_alpha[q] -= gr * D[u] / (A[u] * A[u]);
    }
  }
}

// one CTA per view
__global__ void __launch_bounds__(kViewSumThreads) reg_final_kernel(const double* __restrict__ partial,
                                                                   const int* __restrict__ block_prefix,
                                                                   const DevCam* __restrict__ cams,
                                                                   double* __restrict__ loss) {
  const int v = blockIdx.x;
  double t;
  view_block_sums<1>(partial, block_prefix[v], block_prefix[v + 1], &t);
  if (threadIdx.x == 0) loss[v] = t / ((double)cams[v].W * (double)cams[v].H);
}

}  // namespace

cudaError_t launch_depth_distortion(const float* alpha, const float* depth, const float* depth2, const DevCam* cams,
                                    int n_views, const int* block_prefix, int n_blocks, float weight,
                                    double* partial, double* loss, float* d_alpha, float* d_depth, float* d_depth2,
                                    cudaStream_t s) {
  if (n_blocks > 0) {
    depth_distortion_kernel<<<n_blocks, kRegThreads, 0, s>>>(alpha, depth, depth2, cams, n_views, block_prefix,
                                                             weight, partial, d_alpha, d_depth, d_depth2);
    cudaError_t e = launched();
    if (e != cudaSuccess) return e;
  }
  reg_final_kernel<<<n_views, kViewSumThreads, 0, s>>>(partial, block_prefix, cams, loss);
  return launched();
}

cudaError_t launch_normal_consistency(const float* alpha, const float* depth, const float* normal, const DevCam* cams,
                                      int n_views, const int* block_prefix, int n_blocks, float weight, float a_min,
                                      double* partial, float* gmap, double* loss, float* d_alpha, float* d_depth,
                                      float* d_normal, cudaStream_t s) {
  if (n_blocks > 0) {
    normal_consistency_kernel<<<n_blocks, kRegThreads, 0, s>>>(alpha, depth, normal, cams, n_views, block_prefix,
                                                               weight, a_min, partial, d_alpha ? gmap : nullptr,
                                                               d_alpha, d_normal);
    cudaError_t e = launched();
    if (e != cudaSuccess) return e;
    if (d_alpha) {
      normal_consistency_gather_kernel<<<n_blocks, kRegThreads, 0, s>>>(alpha, depth, cams, n_views, block_prefix,
                                                                        a_min, gmap, d_alpha, d_depth);
      e = launched();
      if (e != cudaSuccess) return e;
    }
  }
  reg_final_kernel<<<n_views, kViewSumThreads, 0, s>>>(partial, block_prefix, cams, loss);
  return launched();
}

}  // namespace ocgs
