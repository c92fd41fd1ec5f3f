// Surfel projection (forward) and its chain rule (backward).
//
// One thread per Gaussian loops over the views of the call, so the 232-byte
// parameter record is read from HBM once per call and not once per view.
// Forward (per view): cull, the 2DGS splat-to-pixel homography written about
// the projected centre, a conservative screen box of the support, the tile
// rectangle, the camera-facing normal and the view-dependent SH colour.
#include "common.cuh"

namespace ocgs {
namespace {

// Real spherical harmonics with the Condon-Shortley phase, m = -l..l, evaluated
// at a unit direction.  Constants are the closed-form normalisations:
//   1/(2 sqrt(pi)); sqrt(3/(4pi)); sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4;
//   sqrt(70/pi)/8, sqrt(105/pi)/2, sqrt(42/pi)/8, sqrt(7/pi)/4, sqrt(105/pi)/4.
constexpr float kY0 = 0.28209479177387814f;
constexpr float kY1 = 0.48860251190291992f;
constexpr float kY2a = 1.09254843059207907f;
constexpr float kY2b = 0.31539156525252005f;
constexpr float kY2c = 0.54627421529603953f;
constexpr float kY3a = 0.59004358992664352f;
constexpr float kY3b = 2.89061144264055405f;
constexpr float kY3c = 0.45704579946446572f;
constexpr float kY3d = 0.37317633259011540f;
constexpr float kY3e = 1.44530572132027702f;

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = kY0;
  if (DEG >= 1) {
    Y[1] = -kY1 * y;
    Y[2] = kY1 * z;
    Y[3] = -kY1 * x;
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kY2a * x * y;
    Y[5] = -kY2a * y * z;
    Y[6] = kY2b * (2.0f * zz - xx - yy);
    Y[7] = -kY2a * x * z;
    Y[8] = kY2c * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -kY3a * y * (3.0f * xx - yy);
      Y[10] = kY3b * x * y * z;
      Y[11] = -kY3c * y * (4.0f * zz - xx - yy);
      Y[12] = kY3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
      Y[13] = -kY3c * x * (4.0f * zz - xx - yy);
      Y[14] = kY3e * z * (xx - yy);
      Y[15] = -kY3a * x * (xx - 3.0f * yy);
    }
  }
}

// g = sum_k beta_k * grad Y_k(x, y, z) (gradient of the polynomials)
template <int DEG>
__device__ __forceinline__ float3 sh_basis_vjp(float x, float y, float z, const float* b) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (DEG >= 1) {
    gy += -kY1 * b[1];
    gz += kY1 * b[2];
    gx += -kY1 * b[3];
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += kY2a * y * b[4];
    gy += kY2a * x * b[4];
    gy += -kY2a * z * b[5];
    gz += -kY2a * y * b[5];
    gx += -2.f * kY2b * x * b[6];
    gy += -2.f * kY2b * y * b[6];
    gz += 4.f * kY2b * z * b[6];
    gx += -kY2a * z * b[7];
    gz += -kY2a * x * b[7];
    gx += 2.f * kY2c * x * b[8];
    gy += -2.f * kY2c * y * b[8];
    if (DEG >= 3) {
      gx += -6.f * kY3a * x * y * b[9];
      gy += -kY3a * (3.f * xx - 3.f * yy) * b[9];
      gx += kY3b * y * z * b[10];
      gy += kY3b * x * z * b[10];
      gz += kY3b * x * y * b[10];
      gx += 2.f * kY3c * x * y * b[11];
      gy += -kY3c * (4.f * zz - xx - 3.f * yy) * b[11];
      gz += -8.f * kY3c * y * z * b[11];
      gx += -6.f * kY3d * x * z * b[12];
      gy += -6.f * kY3d * y * z * b[12];
      gz += kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * b[12];
      gx += -kY3c * (4.f * zz - 3.f * xx - yy) * b[13];
      gy += 2.f * kY3c * x * y * b[13];
      gz += -8.f * kY3c * x * z * b[13];
      gx += 2.f * kY3e * x * z * b[14];
      gy += -2.f * kY3e * y * z * b[14];
      gz += kY3e * (xx - yy) * b[14];
      gx += -kY3a * (3.f * xx - 3.f * yy) * b[15];
      gy += 6.f * kY3a * x * y * b[15];
    }
  }
  return make_float3(gx, gy, gz);
}

struct Frame {
  float qn[4];   // normalised quaternion (w, x, y, z)
  float inv_norm;
  float tu[3], tv[3], tw[3];
};

__device__ __forceinline__ Frame make_frame(float4 q) {
  Frame f;
  const float nn = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  f.inv_norm = rsqrtf(nn);
  const float w = q.x * f.inv_norm, x = q.y * f.inv_norm, y = q.z * f.inv_norm, z = q.w * f.inv_norm;
  f.qn[0] = w; f.qn[1] = x; f.qn[2] = y; f.qn[3] = z;
  // columns of the rotation matrix of (w, x, y, z)
  f.tu[0] = 1.f - 2.f * (y * y + z * z);
  f.tu[1] = 2.f * (x * y + w * z);
  f.tu[2] = 2.f * (x * z - w * y);
  f.tv[0] = 2.f * (x * y - w * z);
  f.tv[1] = 1.f - 2.f * (x * x + z * z);
  f.tv[2] = 2.f * (y * z + w * x);
  f.tw[0] = 2.f * (x * z + w * y);
  f.tw[1] = 2.f * (y * z - w * x);
  f.tw[2] = 1.f - 2.f * (x * x + y * y);
  return f;
}

// Sort key of the front-to-back order: the centre depth R_2 . X + t_z of the float32 camera
// and centre, evaluated as accurately as in twice the precision and rounded once to float32
// (the compensated dot product Dot2 of Ogita, Rump and Oishi, 2005): each product is split
// exactly into p + e with e = fma(a, b, -p), the running sum is kept exact with Knuth's
// TwoSum, and the collected errors are added before the one final rounding.  The key is
// then the depth rounded to float32 (up to cases within about 1e-4 ulp of a rounding
// midpoint), independent of how the float32 geometry below is contracted; positive for
// every record that is not culled, so the bit pattern orders like the value.
__device__ __forceinline__ uint32_t depth_key_of(const DevCam& cam, const float* X) {
  float s = cam.t[2], c = 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float p = __fmul_rn(cam.R[6 + j], X[j]);
    const float e = __fmaf_rn(cam.R[6 + j], X[j], -p);  // R X = p + e exactly
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));  // s + p = t + err exactly
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
  }
  return __float_as_uint(__fadd_rn(s, c));
}

__device__ __forceinline__ void rot3(const float* R, const float* a, float* o) {
  o[0] = R[0] * a[0] + R[1] * a[1] + R[2] * a[2];
  o[1] = R[3] * a[0] + R[4] * a[1] + R[5] * a[2];
  o[2] = R[6] * a[0] + R[7] * a[1] + R[8] * a[2];
}
__device__ __forceinline__ void rot3T(const float* R, const float* a, float* o) {
  o[0] = R[0] * a[0] + R[3] * a[1] + R[6] * a[2];
  o[1] = R[1] * a[0] + R[4] * a[1] + R[7] * a[2];
  o[2] = R[2] * a[0] + R[5] * a[1] + R[8] * a[2];
}

// Camera-frame quantities of one Gaussian in one view, shared by both passes.
struct ViewGeom {
  float p[3];       // centre
  float U[3], V[3];  // scaled tangent axes
  float n[3];       // camera-facing normal
  float nsign;      // +1 or -1 (flip applied to R t_w)
  float iz, pxn, pyn;
  float a, b, c, d;  // centred homography entries
};

__device__ __forceinline__ void view_geom(const DevCam& cam, const float* X, const Frame& f, float su,
                                          float sv, ViewGeom& G) {
  float tmp[3];
  rot3(cam.R, X, G.p);
  G.p[0] += cam.t[0]; G.p[1] += cam.t[1]; G.p[2] += cam.t[2];
  rot3(cam.R, f.tu, tmp);
  G.U[0] = su * tmp[0]; G.U[1] = su * tmp[1]; G.U[2] = su * tmp[2];
  rot3(cam.R, f.tv, tmp);
  G.V[0] = sv * tmp[0]; G.V[1] = sv * tmp[1]; G.V[2] = sv * tmp[2];
  rot3(cam.R, f.tw, G.n);
  const float dot = __fmaf_rn(G.n[2], G.p[2], __fmaf_rn(G.n[1], G.p[1], __fmul_rn(G.n[0], G.p[0])));
  G.nsign = dot > 0.f ? -1.f : 1.f;
  G.n[0] *= G.nsign; G.n[1] *= G.nsign; G.n[2] *= G.nsign;
  G.iz = 1.0f / G.p[2];
  G.pxn = G.p[0] * G.iz;
  G.pyn = G.p[1] * G.iz;
  G.a = cam.fx * (G.U[0] - G.U[2] * G.pxn);
  G.b = cam.fx * (G.V[0] - G.V[2] * G.pxn);
  G.c = cam.fy * (G.U[1] - G.U[2] * G.pyn);
  G.d = cam.fy * (G.V[1] - G.V[2] * G.pyn);
}

template <int DEG>
__device__ __forceinline__ void view_colour(const DevCam& cam, const float* X, const float* sh,
                                            float* dirn, float* dlen, float* raw) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  float dv[3] = {X[0] - cam.campos[0], X[1] - cam.campos[1], X[2] - cam.campos[2]};
  const float len = sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  const float il = 1.0f / len;
  dirn[0] = dv[0] * il; dirn[1] = dv[1] * il; dirn[2] = dv[2] * il;
  *dlen = len;
  float Y[K];
  sh_basis<DEG>(dirn[0], dirn[1], dirn[2], Y);
  float r0 = 0.5f, r1 = 0.5f, r2 = 0.5f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    r0 += Y[k] * sh[3 * k + 0];
    r1 += Y[k] * sh[3 * k + 1];
    r2 += Y[k] * sh[3 * k + 2];
  }
  raw[0] = r0; raw[1] = r1; raw[2] = r2;
}

__device__ __forceinline__ float project_x(const DevCam& cam, float X, float Z) { return cam.fx * X / Z + cam.cx; }
__device__ __forceinline__ float project_y(const DevCam& cam, float Y, float Z) { return cam.fy * Y / Z + cam.cy; }

// ----------------------------------------------------------------------------- SH staging
// A block's SH coefficients (NF = 3K floats per Gaussian, NF x 4 bytes apart) are
// one contiguous span of the array: they are moved between global and shared
// memory with coalesced loads and stores, and each thread reads or writes its own
// NF floats in shared memory.  When NF is a multiple of 4 the rows are float4 rows
// whose stride in float4 is odd (conflict-free 16-byte accesses by 8 threads per
// phase); otherwise float rows of odd stride.
constexpr int kPreThreads = 128;
// views whose cameras the projection kernels keep in shared memory (more are read from global)
constexpr int kSmemCams = 64;

// Copies the views' cameras to s_cams when they fit (the caller's next block barrier
// publishes them) and returns where the view loop reads them from.
__device__ __forceinline__ const DevCam* stage_cams(const DevCam* __restrict__ cams, int n_views, DevCam* s_cams) {
  if (n_views > kSmemCams) return cams;
  const int words = n_views * (int)(sizeof(DevCam) / sizeof(int));
  for (int w = threadIdx.x; w < words; w += blockDim.x)
    reinterpret_cast<int*>(s_cams)[w] = reinterpret_cast<const int*>(cams)[w];
  return s_cams;
}

template <int NF>
struct ShRows {
  static constexpr bool kVec = NF % 4 == 0;
  static constexpr int kStride = kVec ? 4 * ((NF / 4) | 1) : (NF | 1);  // floats per row
  static constexpr int kFloats = kPreThreads * kStride;
  // position in shared memory of float f of the block's span
  __device__ static __forceinline__ int at(int f) { return (f / NF) * kStride + f % NF; }
};

// loads the block's span of src into its rows (all threads; ends with a barrier)
template <int NF>
__device__ __forceinline__ void sh_rows_load(const float* __restrict__ src, int64_t n, float* rows) {
  using L = ShRows<NF>;
  const int64_t i0 = (int64_t)blockIdx.x * kPreThreads;
  const int total = (int)min((int64_t)kPreThreads, n - i0) * NF;
  const float* base = src + i0 * NF;
  if (L::kVec && (reinterpret_cast<uintptr_t>(base) & 15u) == 0) {
    for (int j = threadIdx.x; 4 * j < total; j += kPreThreads)  // total is a multiple of 4 here
      *reinterpret_cast<float4*>(rows + L::at(4 * j)) = reinterpret_cast<const float4*>(base)[j];
  } else {
    for (int f = threadIdx.x; f < total; f += kPreThreads) rows[L::at(f)] = base[f];
  }
  __syncthreads();
}

// this thread's row
template <int NF>
__device__ __forceinline__ void sh_row_read(const float* rows, float* v) {
  using L = ShRows<NF>;
  const float* r = rows + threadIdx.x * L::kStride;
  if constexpr (L::kVec) {
#pragma unroll
    for (int m = 0; m < NF / 4; ++m) {
      const float4 a = reinterpret_cast<const float4*>(r)[m];
      v[4 * m] = a.x;
      v[4 * m + 1] = a.y;
      v[4 * m + 2] = a.z;
      v[4 * m + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < NF; ++k) v[k] = r[k];
  }
}

template <int NF>
__device__ __forceinline__ void sh_row_write(float* rows, const float* v) {
  using L = ShRows<NF>;
  float* r = rows + threadIdx.x * L::kStride;
  if constexpr (L::kVec) {
#pragma unroll
    for (int m = 0; m < NF / 4; ++m)
      reinterpret_cast<float4*>(r)[m] = make_float4(v[4 * m], v[4 * m + 1], v[4 * m + 2], v[4 * m + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < NF; ++k) r[k] = v[k];
  }
}

// adds the block's rows to its span of dst (all threads; starts with a barrier)
template <int NF>
__device__ __forceinline__ void sh_rows_add(float* __restrict__ dst, int64_t n, const float* rows) {
  using L = ShRows<NF>;
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * kPreThreads;
  const int total = (int)min((int64_t)kPreThreads, n - i0) * NF;
  float* base = dst + i0 * NF;
  if (L::kVec && (reinterpret_cast<uintptr_t>(base) & 15u) == 0) {
    for (int j = threadIdx.x; 4 * j < total; j += kPreThreads) {
      float4 v = reinterpret_cast<float4*>(base)[j];
      const float4 a = *reinterpret_cast<const float4*>(rows + L::at(4 * j));
      v.x += a.x;
      v.y += a.y;
      v.z += a.z;
      v.w += a.w;
      reinterpret_cast<float4*>(base)[j] = v;
    }
  } else {
    for (int f = threadIdx.x; f < total; f += kPreThreads) base[f] += rows[L::at(f)];
  }
}

template <int DEG>
__global__ void __launch_bounds__(128) preprocess_kernel(GaussPtrs g, int64_t n,
                                                         const DevCam* __restrict__ cams, int n_views,
                                                         int tile_w, int tile_h, RecPtrs rec,
                                                         int32_t* __restrict__ ntiles,
                                                         float4* __restrict__ bin,
                                                         uint32_t* __restrict__ depth_key,
                                                         int* __restrict__ status) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ __align__(16) float s_rows[ShRows<3 * K>::kFloats];
  __shared__ DevCam s_cams[kSmemCams];
  const DevCam* vcams = stage_cams(cams, n_views, s_cams);
  sh_rows_load<3 * K>(g.sh, n, s_rows);  // its barrier also publishes s_cams
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float X[3] = {g.xyz[3 * i], g.xyz[3 * i + 1], g.xyz[3 * i + 2]};
  const float4 q = reinterpret_cast<const float4*>(g.quat)[i];
  const float2 s = reinterpret_cast<const float2*>(g.scale)[i];
  const float o = g.opacity[i];
  float sh[3 * K];
  sh_row_read<3 * K>(s_rows, sh);
  bool finite = finitef(X[0]) && finitef(X[1]) && finitef(X[2]) && finitef(q.x) && finitef(q.y) &&
                finitef(q.z) && finitef(q.w) && finitef(s.x) && finitef(s.y) && finitef(o);
#pragma unroll
  for (int k = 0; k < 3 * K; ++k) finite = finite && finitef(sh[k]);
  const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  if (!finite) atomicOr(status, kStatusNonFinite);
  const bool bad = !finite || !(qn2 > 0.f) || !(s.x > 0.f) || !(s.y > 0.f) || !(o >= kAlphaMin);
  const Frame f = make_frame(q);
  // support bound in rho: the 3-sigma cut, tightened where o exp(-rho/2) < 1/255 anyway
  const float rho_b = bad ? 0.f : support_rho(o);
  const float kq = sqrtf(fmaxf(rho_b, 0.f));
  const float rf = sqrtf(0.5f * fmaxf(rho_b, 0.f));

  for (int v = 0; v < n_views; ++v) {
    const DevCam& cam = vcams[v];
    const int64_t idx = (int64_t)v * n + i;
    bool culled = bad;
    ViewGeom G;
    view_geom(cam, X, f, s.x, s.y, G);
    const float zmin = G.p[2] - 3.0f * (fabsf(G.U[2]) + fabsf(G.V[2]));
    culled = culled || !(zmin > cam.near_plane);
    int4 rc = make_int4(0, 0, -1, -1);
    if (!culled) {
      // screen box: corners of the support square (all in front of the camera), union the filter disc
      float xmin = 3.4e38f, xmax = -3.4e38f, ymin = 3.4e38f, ymax = -3.4e38f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float s1 = (c & 1) ? kq : -kq, s2 = (c & 2) ? kq : -kq;
        const float PX = G.p[0] + s1 * G.U[0] + s2 * G.V[0];
        const float PY = G.p[1] + s1 * G.U[1] + s2 * G.V[1];
        const float PZ = G.p[2] + s1 * G.U[2] + s2 * G.V[2];
        const float x = project_x(cam, PX, PZ), y = project_y(cam, PY, PZ);
        xmin = fminf(xmin, x); xmax = fmaxf(xmax, x);
        ymin = fminf(ymin, y); ymax = fmaxf(ymax, y);
      }
      const float ccx = cam.fx * G.pxn + cam.cx, ccy = cam.fy * G.pyn + cam.cy;
      xmin = fminf(xmin, ccx - rf); xmax = fmaxf(xmax, ccx + rf);
      ymin = fminf(ymin, ccy - rf); ymax = fmaxf(ymax, ccy + rf);
      const float padx = 0.05f + 1e-5f * (fabsf(xmin) + fabsf(xmax));
      const float pady = 0.05f + 1e-5f * (fabsf(ymin) + fabsf(ymax));
      // pixel columns whose centre i + 0.5 lies in [xmin, xmax]
      const float lo_x = fmaxf(ceilf(xmin - padx - 0.5f), 0.f);
      const float hi_x = fminf(floorf(xmax + padx - 0.5f), (float)(cam.W - 1));
      const float lo_y = fmaxf(ceilf(ymin - pady - 0.5f), 0.f);
      const float hi_y = fminf(floorf(ymax + pady - 0.5f), (float)(cam.H - 1));
      if (lo_x <= hi_x && lo_y <= hi_y) {
        rc = make_int4((int)lo_x / tile_w, (int)lo_y / tile_h, (int)hi_x / tile_w, (int)hi_y / tile_h);
      } else {
        culled = true;
      }
    }
    if (culled) {
      ntiles[idx] = 0;
      depth_key[idx] = 0xffffffffu;
      bin[3 * idx + 2] = make_float4(0.f, 0.f, __uint_as_float(pack_i16x2(0, 0)), __uint_as_float(pack_i16x2(-1, -1)));
      continue;
    }
    ntiles[idx] = (rc.z - rc.x + 1) * (rc.w - rc.y + 1);
    depth_key[idx] = depth_key_of(cam, X);
    const float pz = G.p[2];
    const float e0 = G.a * G.d - G.b * G.c;
    const float e1 = G.V[2] * G.c - G.U[2] * G.d;
    const float e2 = G.U[2] * G.b - G.V[2] * G.a;
    float dirn[3], dlen, raw[3];
    view_colour<DEG>(cam, X, sh, dirn, &dlen, raw);
    const float4 g0 = make_float4(cam.fx * G.pxn + cam.cx, cam.fy * G.pyn + cam.cy, o, pz);
    const float4 g1 = make_float4(pz * G.d, -pz * G.b, -pz * G.c, pz * G.a);
    rec.g0[idx] = g0;
    rec.g1[idx] = g1;
    rec.g2[idx] = make_float4(e0, e1, e2, pz * e0);
    // the support bound the binning and the rasterizers' row test see; unbounded (every
    // tile and row of the screen rectangle) when the view checks the support test
    const float rb_bin = cam.cover_rect ? INFINITY : rho_b;
    bin[3 * idx] = make_float4(g0.x, g0.y, rb_bin, g1.x);
    bin[3 * idx + 1] = make_float4(g1.y, g1.z, g1.w, e0);
    bin[3 * idx + 2] = make_float4(e1, e2, __uint_as_float(pack_i16x2(rc.x, rc.y)),
                                   __uint_as_float(pack_i16x2(rc.z, rc.w)));
    rec.a0[idx] = make_float4(fmaxf(raw[0], 0.f), fmaxf(raw[1], 0.f), fmaxf(raw[2], 0.f), G.n[0]);
    const float4 g2 = make_float4(e0, e1, e2, pz * e0);
    const float2 rows = support_rows(g0, g1, g2, rb_bin);
    rec.a1[idx] = make_float4(G.n[1], G.n[2], rows.x, rows.y);
  }
}

template <int DEG>
__global__ void __launch_bounds__(128) preprocess_bwd_kernel(GaussPtrs g, int64_t n,
                                                             const DevCam* __restrict__ cams,
                                                             int n_views,
                                                             const float* __restrict__ grad_rec,
                                                             const int32_t* __restrict__ ntiles,
                                                             GaussOut out) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ __align__(16) float s_rows[ShRows<3 * K>::kFloats];
  // the views' cameras in shared memory (short-latency reads in the view loop)
  __shared__ DevCam s_cams[kSmemCams];
  const DevCam* vcams = stage_cams(cams, n_views, s_cams);
  sh_rows_load<3 * K>(g.sh, n, s_rows);  // its barrier also publishes s_cams
  // every thread reaches the block's final exchange of SH gradients: a thread past
  // the end recomputes the last Gaussian and writes nothing
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i0 < n;
  const int64_t i = active ? i0 : n - 1;
  float X[3] = {g.xyz[3 * i], g.xyz[3 * i + 1], g.xyz[3 * i + 2]};
  const float4 q = reinterpret_cast<const float4*>(g.quat)[i];
  const float2 s = reinterpret_cast<const float2*>(g.scale)[i];
  float sh[3 * K];
  sh_row_read<3 * K>(s_rows, sh);
  const Frame f = make_frame(q);

  float gX[3] = {0.f, 0.f, 0.f};
  float gtu[3] = {0.f, 0.f, 0.f}, gtv[3] = {0.f, 0.f, 0.f}, gtw[3] = {0.f, 0.f, 0.f};
  float gsu = 0.f, gsv = 0.f, go = 0.f;
  float gsh[3 * K];
#pragma unroll
  for (int k = 0; k < 3 * K; ++k) gsh[k] = 0.f;

  // the tile counts and record gradients of the next two views are requested before
  // the current view is processed, so their memory latency overlaps its arithmetic
  constexpr int NQ = kGradStride / 4;
  int nt_next = 0, nt_next2 = 0;
  float4 g_next[NQ], g_next2[NQ];
  auto request = [&](int v, int& nt, float4* gv) {
    const int64_t idx = (int64_t)v * n + i;
    nt = ntiles[idx];
    const float4* gr4 = reinterpret_cast<const float4*>(grad_rec + idx * kGradStride);
#pragma unroll
    for (int q = 0; q < NQ; ++q) gv[q] = gr4[q];
  };
  if (n_views > 0) request(0, nt_next, g_next);
  if (n_views > 1) request(1, nt_next2, g_next2);
  for (int v = 0; v < n_views; ++v) {
    const int nt = nt_next;
    float gq[kGradStride];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      gq[4 * q] = g_next[q].x;
      gq[4 * q + 1] = g_next[q].y;
      gq[4 * q + 2] = g_next[q].z;
      gq[4 * q + 3] = g_next[q].w;
      g_next[q] = g_next2[q];
    }
    nt_next = nt_next2;
    if (v + 2 < n_views) request(v + 2, nt_next2, g_next2);
    if (nt == 0) continue;
    const DevCam& cam = vcams[v];
    const float g_cx = gq[kGcx], g_cy = gq[kGcy], g_o = gq[kGo], g_zc = gq[kGzc];
    const float gA00 = gq[kGA00], gA01 = gq[kGA01], gA10 = gq[kGA10], gA11 = gq[kGA11];
    float ge0 = gq[kGe0];
    const float ge1 = gq[kGe1], ge2 = gq[kGe2], gzD = gq[kGzD];
    const float grgb[3] = {gq[kGr], gq[kGg], gq[kGb]};
    const float gn[3] = {gq[kGnx], gq[kGny], gq[kGnz]};
    go += g_o;

    ViewGeom G;
    view_geom(cam, X, f, s.x, s.y, G);
    const float pz = G.p[2];
    const float e0 = G.a * G.d - G.b * G.c;
    // zD = pz e0 ; A = pz [d, -b; -c, a] ; e0 = ad - bc ; e1 = Vz c - Uz d ; e2 = Uz b - Vz a
    float gpz = gzD * e0 + g_zc + gA00 * G.d - gA01 * G.b - gA10 * G.c + gA11 * G.a;
    ge0 += gzD * pz;
    float ga = gA11 * pz + ge0 * G.d - ge2 * G.V[2];
    float gb = -gA01 * pz - ge0 * G.c + ge2 * G.U[2];
    float gc = -gA10 * pz - ge0 * G.b + ge1 * G.V[2];
    float gd = gA00 * pz + ge0 * G.a - ge1 * G.U[2];
    float gU[3] = {0.f, 0.f, 0.f}, gV[3] = {0.f, 0.f, 0.f};
    gU[2] += -ge1 * G.d + ge2 * G.b;
    gV[2] += ge1 * G.c - ge2 * G.a;
    // centre c = (fx pxn + cx, fy pyn + cy)
    float gpxn = g_cx * cam.fx, gpyn = g_cy * cam.fy;
    // a = fx (Ux - Uz pxn), b = fx (Vx - Vz pxn), c = fy (Uy - Uz pyn), d = fy (Vy - Vz pyn)
    gU[0] += cam.fx * ga;
    gU[2] -= cam.fx * G.pxn * ga;
    gpxn -= cam.fx * G.U[2] * ga;
    gV[0] += cam.fx * gb;
    gV[2] -= cam.fx * G.pxn * gb;
    gpxn -= cam.fx * G.V[2] * gb;
    gU[1] += cam.fy * gc;
    gU[2] -= cam.fy * G.pyn * gc;
    gpyn -= cam.fy * G.U[2] * gc;
    gV[1] += cam.fy * gd;
    gV[2] -= cam.fy * G.pyn * gd;
    gpyn -= cam.fy * G.V[2] * gd;
    // pxn = px / pz, pyn = py / pz
    float gp[3];
    gp[0] = gpxn * G.iz;
    gp[1] = gpyn * G.iz;
    gp[2] = gpz - (gpxn * G.pxn + gpyn * G.pyn) * G.iz;
    // p = R X + t ; U = su R tu ; V = sv R tv ; n = nsign R tw
    float tmp[3];
    rot3T(cam.R, gp, tmp);
    gX[0] += tmp[0]; gX[1] += tmp[1]; gX[2] += tmp[2];
    rot3T(cam.R, gU, tmp);
    gsu += tmp[0] * f.tu[0] + tmp[1] * f.tu[1] + tmp[2] * f.tu[2];
    gtu[0] += s.x * tmp[0]; gtu[1] += s.x * tmp[1]; gtu[2] += s.x * tmp[2];
    rot3T(cam.R, gV, tmp);
    gsv += tmp[0] * f.tv[0] + tmp[1] * f.tv[1] + tmp[2] * f.tv[2];
    gtv[0] += s.y * tmp[0]; gtv[1] += s.y * tmp[1]; gtv[2] += s.y * tmp[2];
    rot3T(cam.R, gn, tmp);
    gtw[0] += G.nsign * tmp[0]; gtw[1] += G.nsign * tmp[1]; gtw[2] += G.nsign * tmp[2];
    // colour: rgb = max(0, sum_k sh_k Y_k(dir) + 0.5), dir = normalize(X - campos)
    float dirn[3], dlen, raw[3];
    view_colour<DEG>(cam, X, sh, dirn, &dlen, raw);
    const float graw[3] = {raw[0] > 0.f ? grgb[0] : 0.f, raw[1] > 0.f ? grgb[1] : 0.f,
                           raw[2] > 0.f ? grgb[2] : 0.f};
    float Y[K], beta[K];
    sh_basis<DEG>(dirn[0], dirn[1], dirn[2], Y);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      gsh[3 * k + 0] += graw[0] * Y[k];
      gsh[3 * k + 1] += graw[1] * Y[k];
      gsh[3 * k + 2] += graw[2] * Y[k];
      beta[k] = graw[0] * sh[3 * k] + graw[1] * sh[3 * k + 1] + graw[2] * sh[3 * k + 2];
    }
    if (DEG > 0) {
      const float3 gdn = sh_basis_vjp<DEG>(dirn[0], dirn[1], dirn[2], beta);
      const float dp = gdn.x * dirn[0] + gdn.y * dirn[1] + gdn.z * dirn[2];
      const float il = 1.0f / dlen;
      gX[0] += (gdn.x - dp * dirn[0]) * il;
      gX[1] += (gdn.y - dp * dirn[1]) * il;
      gX[2] += (gdn.z - dp * dirn[2]) * il;
    }
  }
  // rotation columns -> normalised quaternion -> raw quaternion
  // G = dL/dR with columns (gtu, gtv, gtw): G_rc = column c, row r
  const float G00 = gtu[0], G10 = gtu[1], G20 = gtu[2];
  const float G01 = gtv[0], G11 = gtv[1], G21 = gtv[2];
  const float G02 = gtw[0], G12 = gtw[1], G22 = gtw[2];
  const float w = f.qn[0], x = f.qn[1], y = f.qn[2], z = f.qn[3];
  const float gw = 2.f * (-z * G01 + y * G02 + z * G10 - x * G12 - y * G20 + x * G21);
  const float gx = 2.f * (y * G01 + z * G02 + y * G10 - 2.f * x * G11 - w * G12 + z * G20 + w * G21 -
                          2.f * x * G22);
  const float gy = 2.f * (-2.f * y * G00 + x * G01 + w * G02 + x * G10 + z * G12 - w * G20 + z * G21 -
                          2.f * y * G22);
  const float gz = 2.f * (-2.f * z * G00 - w * G01 + x * G02 + w * G10 - 2.f * z * G11 + y * G12 +
                          x * G20 + y * G21);
  const float dotq = gw * w + gx * x + gy * y + gz * z;
  const float in = f.inv_norm;
  if (active) {
    out.xyz[3 * i + 0] += gX[0];
    out.xyz[3 * i + 1] += gX[1];
    out.xyz[3 * i + 2] += gX[2];
    out.quat[4 * i + 0] += (gw - w * dotq) * in;
    out.quat[4 * i + 1] += (gx - x * dotq) * in;
    out.quat[4 * i + 2] += (gy - y * dotq) * in;
    out.quat[4 * i + 3] += (gz - z * dotq) * in;
    out.scale[2 * i + 0] += gsu;
    out.scale[2 * i + 1] += gsv;
    out.opacity[i] += go;
  }
  // the SH gradients leave through this thread's row (only it has read that row) and
  // are added to the output with coalesced accesses
  sh_row_write<3 * K>(s_rows, gsh);
  sh_rows_add<3 * K>(out.sh, n, s_rows);
}

// EWA projection of 3D Gaussians, for the 3DGS variant of the pruning record
// (Appendix B).  The image covariance is J W Sigma W^T J^T + 0.3 I, Sigma =
// R diag(s^2) R^T, J the Jacobian of the pinhole projection at the camera-frame
// mean and 0.3 px^2 the 3DGS screen-space low-pass.  The record is written in the
// surfel record's form: centre, u = M00 dx + M01 dy, v = M11 dy with M^T M the
// inverse covariance (so u^2 + v^2 is the Mahalanobis distance), a constant
// denominator (e = (1, 0, 0)) and the centre depth; binning, sorting and the
// contribution record then run unchanged, and the rasterizer's EWA flag leaves
// out the screen filter, which the dilation already contains.  Scales are [n,3].
template <int DEG>
__global__ void __launch_bounds__(128) preprocess_ewa_kernel(GaussPtrs g, int64_t n,
                                                             const DevCam* __restrict__ cams, int n_views,
                                                             int tile_w, int tile_h, RecPtrs rec,
                                                             int32_t* __restrict__ ntiles,
                                                             float4* __restrict__ bin,
                                                             uint32_t* __restrict__ depth_key,
                                                             int* __restrict__ status) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ __align__(16) float s_rows[ShRows<3 * K>::kFloats];
  __shared__ DevCam s_cams[kSmemCams];
  const DevCam* vcams = stage_cams(cams, n_views, s_cams);
  sh_rows_load<3 * K>(g.sh, n, s_rows);  // its barrier also publishes s_cams
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float X[3] = {g.xyz[3 * i], g.xyz[3 * i + 1], g.xyz[3 * i + 2]};
  const float4 q = reinterpret_cast<const float4*>(g.quat)[i];
  const float s3[3] = {g.scale[3 * i], g.scale[3 * i + 1], g.scale[3 * i + 2]};
  const float o = g.opacity[i];
  float sh[3 * K];
  bool finite = finitef(X[0]) && finitef(X[1]) && finitef(X[2]) && finitef(q.x) && finitef(q.y) &&
                finitef(q.z) && finitef(q.w) && finitef(s3[0]) && finitef(s3[1]) && finitef(s3[2]) && finitef(o);
#pragma unroll
  for (int k = 0; k < 3 * K; ++k) {
    sh[k] = s_rows[threadIdx.x * ShRows<3 * K>::kStride + k];
    finite = finite && finitef(sh[k]);
  }
  const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  if (!finite) atomicOr(status, kStatusNonFinite);
  const bool bad = !finite || !(qn2 > 0.f) || !(s3[0] > 0.f) || !(s3[1] > 0.f) || !(s3[2] > 0.f) ||
                   !(o >= kAlphaMin);
  const Frame f = make_frame(q);
  // world-frame 3D covariance (symmetric: xx xy xz yy yz zz)
  const float v0 = s3[0] * s3[0], v1 = s3[1] * s3[1], v2 = s3[2] * s3[2];
  float S[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) S[r][c] = v0 * f.tu[r] * f.tu[c] + v1 * f.tv[r] * f.tv[c] + v2 * f.tw[r] * f.tw[c];
  const float rho_b = bad ? 0.f : support_rho(o);

  for (int v = 0; v < n_views; ++v) {
    const DevCam& cam = vcams[v];
    const int64_t idx = (int64_t)v * n + i;
    float t[3];
    rot3(cam.R, X, t);
    t[0] += cam.t[0]; t[1] += cam.t[1]; t[2] += cam.t[2];
    bool culled = bad || !(t[2] > cam.near_plane);
    int4 rc = make_int4(0, 0, -1, -1);
    float m00 = 0.f, m01 = 0.f, m11 = 0.f, ccx = 0.f, ccy = 0.f;
    if (!culled) {
      const float iz = 1.0f / t[2];
      // T = J W (2 x 3): rows of the Jacobian times the camera rotation
      const float j0[3] = {cam.fx * iz, 0.f, -cam.fx * t[0] * iz * iz};
      const float j1[3] = {0.f, cam.fy * iz, -cam.fy * t[1] * iz * iz};
      float T0[3], T1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T0[c] = j0[0] * cam.R[c] + j0[1] * cam.R[3 + c] + j0[2] * cam.R[6 + c];
        T1[c] = j1[0] * cam.R[c] + j1[1] * cam.R[3 + c] + j1[2] * cam.R[6 + c];
      }
      float ST0[3], ST1[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        ST0[r] = S[r][0] * T0[0] + S[r][1] * T0[1] + S[r][2] * T0[2];
        ST1[r] = S[r][0] * T1[0] + S[r][1] * T1[1] + S[r][2] * T1[2];
      }
      const float a = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + 0.3f;
      const float b = T0[0] * ST1[0] + T0[1] * ST1[1] + T0[2] * ST1[2];
      const float c = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + 0.3f;
      const float det = a * c - b * b;
      if (!(det > 0.f) || !isfinite(det)) {
        culled = true;
      } else {
        const float A = c / det, B = -b / det;  // conic [[A, B], [B, C]], C = a / det
        m00 = sqrtf(A);
        m01 = B / m00;
        m11 = 1.0f / sqrtf(c);  // m11^2 = C - m01^2 = C - B^2 / A = 1 / c
        ccx = cam.fx * t[0] * iz + cam.cx;
        ccy = cam.fy * t[1] * iz + cam.cy;
        // {d^T conic d <= rb} lies in the disc of radius sqrt(rb * lambda_max(cov))
        const float mid = 0.5f * (a + c);
        const float lmax = mid + sqrtf(fmaxf(0.25f * (a - c) * (a - c) + b * b, 0.f));
        const float rad = sqrtf(rho_b * lmax) * 1.001f + 0.05f;
        const float lo_x = fmaxf(ceilf(ccx - rad - 0.5f), 0.f), hi_x = fminf(floorf(ccx + rad - 0.5f), (float)(cam.W - 1));
        const float lo_y = fmaxf(ceilf(ccy - rad - 0.5f), 0.f), hi_y = fminf(floorf(ccy + rad - 0.5f), (float)(cam.H - 1));
        if (lo_x <= hi_x && lo_y <= hi_y)
          rc = make_int4((int)lo_x / tile_w, (int)lo_y / tile_h, (int)hi_x / tile_w, (int)hi_y / tile_h);
        else
          culled = true;
      }
    }
    if (culled) {
      ntiles[idx] = 0;
      depth_key[idx] = 0xffffffffu;
      bin[3 * idx + 2] = make_float4(0.f, 0.f, __uint_as_float(pack_i16x2(0, 0)), __uint_as_float(pack_i16x2(-1, -1)));
      continue;
    }
    ntiles[idx] = (rc.z - rc.x + 1) * (rc.w - rc.y + 1);
    depth_key[idx] = depth_key_of(cam, X);
    float dirn[3], dlen, raw[3];
    view_colour<DEG>(cam, X, sh, dirn, &dlen, raw);
    const float4 g0 = make_float4(ccx, ccy, o, t[2]);
    const float4 g1 = make_float4(m00, m01, 0.f, m11);
    rec.g0[idx] = g0;
    rec.g1[idx] = g1;
    rec.g2[idx] = make_float4(1.f, 0.f, 0.f, t[2]);
    rec.a0[idx] = make_float4(fmaxf(raw[0], 0.f), fmaxf(raw[1], 0.f), fmaxf(raw[2], 0.f), 0.f);
    const float rb_bin = cam.cover_rect ? INFINITY : rho_b;  // as in the surfel projection
    const float2 rows = support_rows(g0, g1, make_float4(1.f, 0.f, 0.f, t[2]), rb_bin);
    rec.a1[idx] = make_float4(0.f, 0.f, rows.x, rows.y);
    bin[3 * idx] = make_float4(g0.x, g0.y, rb_bin, g1.x);
    bin[3 * idx + 1] = make_float4(g1.y, g1.z, g1.w, 1.f);
    bin[3 * idx + 2] = make_float4(0.f, 0.f, __uint_as_float(pack_i16x2(rc.x, rc.y)),
                                   __uint_as_float(pack_i16x2(rc.z, rc.w)));
  }
}

}  // namespace

cudaError_t launch_preprocess(const GaussPtrs& g, int64_t n, int sh_degree, const DevCam* cams,
                              int n_views, int tile_w, int tile_h, RecPtrs rec, int32_t* ntiles,
                              float4* bin, uint32_t* depth_key, int* status, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int bs = kPreThreads;
  const unsigned grid = (unsigned)((n + bs - 1) / bs);
  switch (sh_degree) {
    case 0: preprocess_kernel<0><<<grid, bs, 0, s>>>(g, n, cams, n_views, tile_w, tile_h, rec, ntiles, bin, depth_key, status); break;
    case 1: preprocess_kernel<1><<<grid, bs, 0, s>>>(g, n, cams, n_views, tile_w, tile_h, rec, ntiles, bin, depth_key, status); break;
    case 2: preprocess_kernel<2><<<grid, bs, 0, s>>>(g, n, cams, n_views, tile_w, tile_h, rec, ntiles, bin, depth_key, status); break;
    default: preprocess_kernel<3><<<grid, bs, 0, s>>>(g, n, cams, n_views, tile_w, tile_h, rec, ntiles, bin, depth_key, status); break;
  }
  return launched();
}

cudaError_t launch_preprocess_backward(const GaussPtrs& g, int64_t n, int sh_degree,
                                       const DevCam* cams, int n_views, const float* grad_rec,
                                       const int32_t* ntiles, GaussOut out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int bs = kPreThreads;
  const unsigned grid = (unsigned)((n + bs - 1) / bs);
  switch (sh_degree) {
    case 0: preprocess_bwd_kernel<0><<<grid, bs, 0, s>>>(g, n, cams, n_views, grad_rec, ntiles, out); break;
    case 1: preprocess_bwd_kernel<1><<<grid, bs, 0, s>>>(g, n, cams, n_views, grad_rec, ntiles, out); break;
    case 2: preprocess_bwd_kernel<2><<<grid, bs, 0, s>>>(g, n, cams, n_views, grad_rec, ntiles, out); break;
    default: preprocess_bwd_kernel<3><<<grid, bs, 0, s>>>(g, n, cams, n_views, grad_rec, ntiles, out); break;
  }
  return launched();
}

}  // namespace ocgs

namespace ocgs {
cudaError_t launch_preprocess_ewa(const GaussPtrs& g, int64_t n, int sh_degree, const DevCam* cams, int n_views,
                                  int tile_w, int tile_h, RecPtrs rec, int32_t* ntiles, float4* bin,
                                  uint32_t* depth_key, int* status, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int bs = kPreThreads;
  const unsigned grid = (unsigned)((n + bs - 1) / bs);
  switch (sh_degree) {
    case 0: preprocess_ewa_kernel<0><<<grid, bs, 0, s>>>(g, n, cams, n_views, tile_w, tile_h, rec, ntiles, bin, depth_key, status); break;
    case 1: preprocess_ewa_kernel<1><<<grid, bs, 0, s>>>(g, n, cams, n_views, tile_w, tile_h, rec, ntiles, bin, depth_key, status); break;
    case 2: preprocess_ewa_kernel<2><<<grid, bs, 0, s>>>(g, n, cams, n_views, tile_w, tile_h, rec, ntiles, bin, depth_key, status); break;
    default: preprocess_ewa_kernel<3><<<grid, bs, 0, s>>>(g, n, cams, n_views, tile_w, tile_h, rec, ntiles, bin, depth_key, status); break;
  }
  return launched();
}
}  // namespace ocgs
