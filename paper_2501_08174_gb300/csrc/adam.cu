// Fused Adam update of the five parameter arrays (Kingma & Ba, 2015,
// Algorithm 1), the optimiser of the 2DGS training the method keeps (Sec. 5.1).
// One launch: grid.y selects the array, grid.x strides over its elements with
// 16-byte vector accesses where all four arrays of the parameter allow them.
// HBM-bound: 4 loads and 3 stores of 4 bytes per element.
#include "common.cuh"

namespace ocgs {
namespace {

constexpr int kAdamThreads = 256;

__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr, const AdamArgs& a) {
  m = __fmaf_rn(a.beta1, m, __fmul_rn(a.one_m_beta1, g));
  v = __fmaf_rn(a.beta2, v, __fmul_rn(a.one_m_beta2, __fmul_rn(g, g)));
  const float mhat = __fmul_rn(m, a.inv_bc1);  // m / (1 - beta1^t)
  const float vhat = __fmul_rn(v, a.inv_bc2);  // v / (1 - beta2^t)
  p = __fsub_rn(p, __fdiv_rn(__fmul_rn(lr, mhat), __fadd_rn(__fsqrt_rn(vhat), a.eps)));
}

__global__ void __launch_bounds__(kAdamThreads) adam_kernel(const AdamArgs a) {
  const AdamSeg sg = a.seg[blockIdx.y];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  int64_t head = 0;
  if (sg.vector) {
    const int64_t n4 = sg.count / 4;
    float4* p4 = reinterpret_cast<float4*>(sg.p);
    const float4* g4 = reinterpret_cast<const float4*>(sg.g);
    float4* m4 = reinterpret_cast<float4*>(sg.m);
    float4* v4 = reinterpret_cast<float4*>(sg.v);
    for (int64_t i = i0; i < n4; i += stride) {
      float4 p = p4[i], m = m4[i], v = v4[i];
      const float4 g = g4[i];
      adam1(p.x, g.x, m.x, v.x, sg.lr, a);
      adam1(p.y, g.y, m.y, v.y, sg.lr, a);
      adam1(p.z, g.z, m.z, v.z, sg.lr, a);
      adam1(p.w, g.w, m.w, v.w, sg.lr, a);
      bad = bad || !(isfinite(g.x) && isfinite(g.y) && isfinite(g.z) && isfinite(g.w));
      p4[i] = p;
      m4[i] = m;
      v4[i] = v;
    }
    head = n4 * 4;
  }
  for (int64_t i = head + i0; i < sg.count; i += stride) {
    float p = sg.p[i], m = sg.m[i], v = sg.v[i];
    const float g = sg.g[i];
    adam1(p, g, m, v, sg.lr, a);
    bad = bad || !isfinite(g);
    sg.p[i] = p;
    sg.m[i] = m;
    sg.v[i] = v;
  }
  if (bad) atomicOr(a.status, kStatusNonFinite);
}

}  // namespace

cudaError_t launch_adam(const AdamArgs& a, int sm_count, cudaStream_t s) {
  int64_t most = 0;
  for (int k = 0; k < 5; ++k) most = a.seg[k].count > most ? a.seg[k].count : most;
  if (most == 0) return cudaSuccess;
  const int64_t want = (most / 4 + kAdamThreads - 1) / kAdamThreads;
  const int64_t cap = (int64_t)sm_count * 8;  // 8 blocks of 256 per SM, grid-stride beyond
  const unsigned gx = (unsigned)(want < 1 ? 1 : (want > cap ? cap : want));
  adam_kernel<<<dim3(gx, 5), kAdamThreads, 0, s>>>(a);
  return launched();
}

}  // namespace ocgs
