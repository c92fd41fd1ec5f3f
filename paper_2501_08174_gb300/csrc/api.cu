// Host runtime of libocgs: the C ABI declared in include/ocgs.h.
//
// A context binds one device and one stream and owns a stream-ordered memory
// pool (cudaMallocFromPoolAsync) that keeps freed blocks for reuse, so the
// per-call buffers (records, keys, pairs) cost no driver allocation after the
// first call of a given size.  Every call validates its arguments on the host
// before any launch; device-side conditions (non-finite parameters) are
// raised in a status word that the synchronising calls read back.
#include "ocgs.h"
#include "common.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

using namespace ocgs;

std::atomic<long long> ocgs::g_kernel_launches{0};

struct ocgs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  ocgs_options opts{16, 16, 0, 2, 0.f, 32};
  int cover_rect = 0;  // ocgs_set_coverage
  ocgs_stats stats{};
  std::string err;
  int* d_status = nullptr;
  uint64_t* d_scalar = nullptr;   // [4]
  uint64_t* h_scalar = nullptr;   // pinned [4]
  int sm_count = 0;
  // built-in stage profiler: event pairs recorded on the stream around each stage
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_stage;
  size_t ev_used = 0;
  double prof_ms[16] = {0};
  int64_t prof_n[16] = {0};
};

struct ocgs_fwd_state {
  ocgs_ctx* ctx = nullptr;
  int V = 0;
  int64_t N = 0;
  int deg = 0;
  int64_t P = 0;
  uint32_t K = 0;
  uint32_t n_tiles = 0;
  int tile_w = 16, tile_h = 16, ppt = 1, batch = 32;
  int persistent = 0;
  DevCam* d_cams = nullptr;
  int* d_tile_prefix = nullptr;
  RecPtrs rec{};
  int32_t* ntiles = nullptr;
  uint32_t* vals = nullptr;
  uint2* ranges = nullptr;
  uint2* ranges2 = nullptr;   // two-pass renders: second segment of each tile's list
  uint32_t* vals2 = nullptr;
  float* t_final = nullptr;
  uint32_t* last = nullptr;
  uint32_t* tile_order = nullptr;
  std::vector<void*> allocs;
};

namespace {

const char* kStatusNames[] = {"OCGS_OK",      "OCGS_ERR_ARG",       "OCGS_ERR_OOM",      "OCGS_ERR_CUDA",
                              "OCGS_ERR_TIMEOUT", "OCGS_ERR_NONFINITE", "OCGS_ERR_CAPACITY", "OCGS_ERR_STATE"};

ocgs_status set_err(ocgs_ctx* ctx, ocgs_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

ocgs_status cuda_err(ocgs_ctx* ctx, cudaError_t e, const char* what) {
  const ocgs_status s = (e == cudaErrorMemoryAllocation) ? OCGS_ERR_OOM : OCGS_ERR_CUDA;
  return set_err(ctx, s, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call);   \
  } while (0)

// Stream-ordered allocations of one call; freed (stream-ordered) on scope
// exit unless handed over to a forward state.
struct Arena {
  ocgs_ctx* ctx;
  std::vector<void*> ptrs;
  explicit Arena(ocgs_ctx* c) : ctx(c) {}
  ~Arena() {
    for (void* p : ptrs) cudaFreeAsync(p, ctx->stream);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
    void* q = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&q, (bytes + 255) & ~(size_t)255, ctx->pool, ctx->stream);
    if (e != cudaSuccess) return e;
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaSuccess;
  }
  void release_to(std::vector<void*>& dst) {
    dst.insert(dst.end(), ptrs.begin(), ptrs.end());
    ptrs.clear();
  }
};

// Records a CUDA event pair around one stage when the profiler is on.
struct StageTimer {
  ocgs_ctx* ctx;
  int slot = -1;
  StageTimer(ocgs_ctx* c, int stage) : ctx(c) {
    if (!ctx->prof) return;
    if (2 * ctx->ev_used + 2 > ctx->ev.size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return;
      if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
      ctx->ev.push_back(a);
      ctx->ev.push_back(b);
      ctx->ev_stage.push_back(0);
    }
    slot = (int)ctx->ev_used++;
    ctx->ev_stage[slot] = stage;
    cudaEventRecord(ctx->ev[2 * slot], ctx->stream);
  }
  void stop() {
    if (slot >= 0) cudaEventRecord(ctx->ev[2 * slot + 1], ctx->stream);
    slot = -1;
  }
  ~StageTimer() { stop(); }
};

bool finite_f(float x) { return std::isfinite(x); }

ocgs_status check_gaussians(ocgs_ctx* ctx, const ocgs_gaussians* g) {
  if (!g) return set_err(ctx, OCGS_ERR_ARG, "gaussians is NULL");
  if (g->n < 0) return set_err(ctx, OCGS_ERR_ARG, "gaussians.n < 0");
  if (g->sh_degree < 0 || g->sh_degree > 3) return set_err(ctx, OCGS_ERR_ARG, "sh_degree must be 0..3");
  if (g->n > 0 && (!g->xyz || !g->quat || !g->scale || !g->opacity || !g->sh))
    return set_err(ctx, OCGS_ERR_ARG, "a Gaussian parameter pointer is NULL");
  if (g->n > 0 && ((uintptr_t)g->quat % 16 || (uintptr_t)g->scale % 8))
    return set_err(ctx, OCGS_ERR_ARG, "quat must be 16-byte and scale 8-byte aligned");
  return OCGS_OK;
}

ocgs_status check_cameras(ocgs_ctx* ctx, const ocgs_camera* cams, int n_views) {
  if (!cams) return set_err(ctx, OCGS_ERR_ARG, "cams is NULL");
  if (n_views < 1 || n_views > 4096) return set_err(ctx, OCGS_ERR_ARG, "n_views must be 1..4096");
  for (int v = 0; v < n_views; ++v) {
    const ocgs_camera& c = cams[v];
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384)
      return set_err(ctx, OCGS_ERR_ARG, "camera " + std::to_string(v) + ": width/height must be 1..16384");
    if (!(c.near_plane > 0.f) || !finite_f(c.near_plane))
      return set_err(ctx, OCGS_ERR_ARG, "camera " + std::to_string(v) + ": near_plane must be > 0");
    if (!finite_f(c.fx) || !finite_f(c.fy) || !finite_f(c.cx) || !finite_f(c.cy) || !(c.fx > 0.f) || !(c.fy > 0.f))
      return set_err(ctx, OCGS_ERR_ARG, "camera " + std::to_string(v) + ": bad intrinsics");
    for (int k = 0; k < 16; ++k)
      if (!finite_f(c.viewmat[k])) return set_err(ctx, OCGS_ERR_ARG, "camera " + std::to_string(v) + ": non-finite viewmat");
  }
  return OCGS_OK;
}

struct CamPlan {
  std::vector<DevCam> cams;
  std::vector<int> tile_prefix;  // V+1
  int64_t P = 0;
  int64_t tiles = 0;
};

CamPlan plan_cameras(const ocgs_camera* cams, int V, int tw, int th, int cover_rect) {
  CamPlan pl;
  pl.cams.resize(V);
  pl.tile_prefix.resize(V + 1);
  int64_t tiles = 0, pix = 0;
  for (int v = 0; v < V; ++v) {
    const ocgs_camera& c = cams[v];
    DevCam& d = pl.cams[v];
    std::memset(&d, 0, sizeof(d));
    for (int r = 0; r < 3; ++r) {
      for (int k = 0; k < 3; ++k) d.R[3 * r + k] = c.viewmat[4 * r + k];
      d.t[r] = c.viewmat[4 * r + 3];
    }
    // camera centre = -R^T t
    for (int k = 0; k < 3; ++k)
      d.campos[k] = -(d.R[k] * d.t[0] + d.R[3 + k] * d.t[1] + d.R[6 + k] * d.t[2]);
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
    d.near_plane = c.near_plane;
    d.W = c.width; d.H = c.height;
    d.tiles_x = (c.width + tw - 1) / tw;
    d.tiles_y = (c.height + th - 1) / th;
    d.tile_offset = (int)tiles;
    d.cover_rect = cover_rect;
    d.pix_offset = pix;
    pl.tile_prefix[v] = (int)tiles;
    tiles += (int64_t)d.tiles_x * d.tiles_y;
    pix += (int64_t)c.width * c.height;
  }
  pl.tile_prefix[V] = (int)tiles;
  pl.P = pix;
  pl.tiles = tiles;
  return pl;
}

int bits_for(uint64_t n) {  // bits needed to represent values 0..n-1
  int b = 0;
  while (n > 1 && (1ull << b) < n) ++b;
  return b;
}

struct LossPlan {
  std::vector<DevCam> cams;
  std::vector<int> prefix;  // loss blocks per view, prefix sums
  int blocks = 0;
};

ocgs_status plan_loss(ocgs_ctx* ctx, const ocgs_camera* cams, int n_views, LossPlan* lp) {
  if (!cams || n_views < 1 || n_views > 4096) return set_err(ctx, OCGS_ERR_ARG, "bad cameras");
  lp->cams.assign(n_views, DevCam{});
  lp->prefix.assign(n_views + 1, 0);
  int64_t pix = 0;
  int blocks = 0;
  for (int v = 0; v < n_views; ++v) {
    if (cams[v].width < 1 || cams[v].height < 1 || cams[v].width > 16384 || cams[v].height > 16384)
      return set_err(ctx, OCGS_ERR_ARG, "camera width/height must be 1..16384");
    DevCam& d = lp->cams[v];
    std::memset(&d, 0, sizeof(DevCam));
    d.W = cams[v].width;
    d.H = cams[v].height;
    d.fx = cams[v].fx;
    d.fy = cams[v].fy;
    d.cx = cams[v].cx;
    d.cy = cams[v].cy;
    d.pix_offset = pix;
    const int64_t np = (int64_t)cams[v].width * cams[v].height;
    lp->prefix[v] = blocks;
    blocks += (int)((np + kLossBlockPixels - 1) / kLossBlockPixels);
    pix += np;
  }
  lp->prefix[n_views] = blocks;
  lp->blocks = blocks;
  return OCGS_OK;
}

ocgs_status read_status(ocgs_ctx* ctx, int* status) {
  CK(cudaMemcpyAsync(ctx->h_scalar + 3, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *status = *reinterpret_cast<int*>(ctx->h_scalar + 3);
  return OCGS_OK;
}

bool valid_tile(int tw, int th, int ppt, int batch) {
  const bool shape = (tw == 16 && th == 16) || (tw == 16 && th == 8) || (tw == 8 && th == 8) || (tw == 32 && th == 8);
  if (!(shape && (ppt == 1 || ppt == 2 || (ppt == 4 && tw == 16 && (th == 16 || th == 8))))) return false;
  // the shapes built with other batch sizes (OCGS_RASTER_SHAPES)
  const bool small_big = tw == 16 && ((th == 16 && (ppt == 2 || ppt == 4)) || (th == 8 && ppt == 4));
  return batch == 32 || ((batch == 16 || batch == 64) && small_big);
}

GaussPtrs gptrs(const ocgs_gaussians* g) { return GaussPtrs{g->xyz, g->quat, g->scale, g->opacity, g->sh}; }

void free_state(ocgs_fwd_state* st) {
  for (void* p : st->allocs) cudaFreeAsync(p, st->ctx->stream);
  st->allocs.clear();
}

// The forward pipeline shared by ocgs_render and ocgs_accumulate_contribution:
// preprocess, depth sort, duplication, tile sort, ranges, rasterization.
ocgs_status forward_pass(ocgs_ctx* ctx, const ocgs_gaussians* g, const ocgs_camera* cams, int V,
                         const ocgs_image* out, float* score, ocgs_fwd_state* st, bool keep_state,
                         bool ewa = false) {
  const int tw = ctx->opts.tile_w, th = ctx->opts.tile_h;
  const int64_t N = g->n;
  CamPlan pl = plan_cameras(cams, V, tw, th, ctx->cover_rect);
  if ((uint64_t)N * (uint64_t)V >= 0xffffffffull)
    return set_err(ctx, OCGS_ERR_CAPACITY, "n_views * n exceeds 2^32 - 1 records");
  if (pl.tiles >= (int64_t)INT32_MAX) return set_err(ctx, OCGS_ERR_CAPACITY, "too many tiles");
  const uint32_t VN = (uint32_t)(N * V);
  cudaStream_t s = ctx->stream;
  Arena keep(ctx), tmp(ctx);

  st->ctx = ctx; st->V = V; st->N = N; st->deg = g->sh_degree; st->P = pl.P;
  st->n_tiles = (uint32_t)pl.tiles; st->tile_w = tw; st->tile_h = th; st->ppt = ctx->opts.pixels_per_thread;
  st->batch = ctx->opts.batch;
  st->persistent = ctx->opts.persistent;
  CK(keep.alloc(&st->d_cams, V));
  CK(keep.alloc(&st->d_tile_prefix, V + 1));
  CK(cudaMemcpyAsync(st->d_cams, pl.cams.data(), sizeof(DevCam) * V, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(st->d_tile_prefix, pl.tile_prefix.data(), sizeof(int) * (V + 1), cudaMemcpyHostToDevice, s));
  CK(keep.alloc(&st->rec.g0, VN));
  CK(keep.alloc(&st->rec.g1, VN));
  CK(keep.alloc(&st->rec.g2, VN));
  CK(keep.alloc(&st->rec.a0, VN));
  CK(keep.alloc(&st->rec.a1, VN));
  CK(keep.alloc(&st->ntiles, VN));
  CK(keep.alloc(&st->ranges, pl.tiles));
  CK(keep.alloc(&st->t_final, keep_state ? pl.P : 1));
  CK(keep.alloc(&st->last, keep_state ? pl.P : 1));
  float4* bin;
  uint32_t *dkey, *order, *dkey_alt, *order_alt;
  uint64_t* counts;
  CK(tmp.alloc(&bin, 3 * (size_t)VN));
  CK(tmp.alloc(&dkey, VN));
  CK(tmp.alloc(&order, VN));
  CK(tmp.alloc(&dkey_alt, VN));
  CK(tmp.alloc(&order_alt, VN));
  CK(tmp.alloc(&counts, VN));
  char* scratch;
  const size_t sbytes = std::max(radix_scratch_bytes(VN), scan_scratch_bytes(VN));
  CK(tmp.alloc(&scratch, sbytes));
  CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s));
  CK(cudaMemsetAsync(st->ranges, 0, sizeof(uint2) * pl.tiles, s));

  {
    StageTimer t(ctx, OCGS_STAGE_PREPROCESS);
    if (ewa)
      CK(launch_preprocess_ewa(gptrs(g), N, g->sh_degree, st->d_cams, V, tw, th, st->rec, st->ntiles, bin, dkey,
                               ctx->d_status, s));
    else
      CK(launch_preprocess(gptrs(g), N, g->sh_degree, st->d_cams, V, tw, th, st->rec, st->ntiles, bin, dkey,
                           ctx->d_status, s));
  }
  int status = 0;
  uint32_t K = 0;
  // two passes need something to continue: images, or the contribution score
  const bool two_pass = (out != nullptr || score != nullptr) && st->persistent && ctx->opts.front_fraction > 0.f &&
                        VN > 0;
  if (!two_pass) {
    {
      StageTimer t(ctx, OCGS_STAGE_BINNING);
      CK(launch_tile_count(bin, st->d_cams, N, VN, tw, th, st->ntiles, dkey, s));
    }
    bool alt = false;
    {
      StageTimer t(ctx, OCGS_STAGE_DEPTH_SORT);
      CK(radix_sort_pairs(dkey, order, dkey_alt, order_alt, VN, 32, scratch, &alt, s, nullptr, true));
    }
    uint32_t* sorted = alt ? order_alt : order;
    {
      StageTimer t(ctx, OCGS_STAGE_BINNING);
      CK(launch_gather_counts(sorted, st->ntiles, counts, VN, s));
      CK(scan_exclusive_u64(counts, counts, VN, ctx->d_scalar, scratch, s));
    }
    CK(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    ocgs_status rs = read_status(ctx, &status);
    if (rs != OCGS_OK) return rs;
    const uint64_t K64 = VN ? ctx->h_scalar[0] : 0;
    if (K64 > (uint64_t)INT32_MAX)
      return set_err(ctx, OCGS_ERR_CAPACITY, "more than 2^31-1 (tile, Gaussian) pairs; split the views");
    K = (uint32_t)K64;
    st->K = K;

    uint32_t *pkey, *pval, *pkey_alt, *pval_alt;
    CK(tmp.alloc(&pkey, K));
    CK(keep.alloc(&pval, K));
    CK(tmp.alloc(&pkey_alt, K));
    CK(keep.alloc(&pval_alt, K));
    char* pscratch;
    CK(tmp.alloc(&pscratch, radix_scratch_bytes(K)));
    {
      StageTimer t(ctx, OCGS_STAGE_BINNING);
      CK(launch_duplicate(sorted, counts, reinterpret_cast<const uint64_t*>(ctx->d_scalar), VN, bin, st->d_cams,
                          N, tw, th, K, pkey, pval, s));
    }
    const int tbits = bits_for((uint64_t)pl.tiles);
    bool palt = false;
    {
      StageTimer t(ctx, OCGS_STAGE_TILE_SORT);
      CK(radix_sort_pairs(pkey, pval, pkey_alt, pval_alt, K, tbits, pscratch, &palt, s));
    }
    uint32_t* skey = palt ? pkey_alt : pkey;
    st->vals = palt ? pval_alt : pval;
    {
      StageTimer t(ctx, OCGS_STAGE_BINNING);
      CK(launch_tile_ranges(skey, K, st->ranges, s));
    }

    uint32_t* queue = nullptr;
    st->tile_order = nullptr;
    if (st->persistent) {
      CK(tmp.alloc(&queue, 1));
      CK(cudaMemsetAsync(queue, 0, sizeof(uint32_t), s));
      uint32_t *wk, *ids, *wk_alt, *ids_alt;
      CK(tmp.alloc(&wk, pl.tiles));
      CK(keep.alloc(&ids, pl.tiles));
      CK(tmp.alloc(&wk_alt, pl.tiles));
      CK(keep.alloc(&ids_alt, pl.tiles));
      char* tscratch;
      CK(tmp.alloc(&tscratch, radix_scratch_bytes((uint32_t)pl.tiles)));
      CK(launch_tile_order(st->ranges, (uint32_t)pl.tiles, wk, ids, s));
      bool talt = false;
      CK(radix_sort_pairs(wk, ids, wk_alt, ids_alt, (uint32_t)pl.tiles, 8, tscratch, &talt, s));
      st->tile_order = talt ? ids_alt : ids;
    }

    RasterArgs ra{};
    ra.ewa = ewa ? 1 : 0;
    ra.cams = st->d_cams;
    ra.tile_prefix = st->d_tile_prefix;
    ra.n_views = V;
    ra.n_gauss = N;
    ra.n_tiles = (uint32_t)pl.tiles;
    ra.ranges = st->ranges;
    ra.vals = st->vals;
    ra.rec = st->rec;
    if (out) ra.out = ImgPtrs{out->rgb, out->alpha, out->depth, out->normal, out->depth2};
    ra.t_final = keep_state ? st->t_final : nullptr;  // no state kept: nothing to write
    ra.last = keep_state ? st->last : nullptr;
    ra.score = score;
    ra.tile_order = st->tile_order;
    ra.queue = queue;
    ra.persistent_ctas = st->persistent ? ctx->sm_count * (2048 * st->ppt / (tw * th)) : 0;
    {
      StageTimer t(ctx, OCGS_STAGE_RASTER_FWD);
      CK(launch_raster_forward(ra, tw, th, st->ppt, st->batch, out != nullptr, s));
    }

  } else {
    // Two passes.  The front of the depth order is binned and rendered first.
    // Each tile with a pixel still running at the end of that prefix is then
    // binned with the records behind the front and continues from the state
    // the first pass left (T, the sums, the last blended position, the stop
    // flags): every pixel walks the same list, in the same order, as in one pass.
    bool alt = false;
    {
      StageTimer t(ctx, OCGS_STAGE_DEPTH_SORT);
      CK(radix_sort_pairs(dkey, order, dkey_alt, order_alt, VN, 32, scratch, &alt, s, nullptr, true));
    }
    uint32_t* sorted = alt ? order_alt : order;
    const uint32_t* skeys = alt ? dkey_alt : dkey;
    const double front = std::ceil((double)ctx->opts.front_fraction * (double)VN);
    const uint32_t M = (uint32_t)std::min<double>((double)VN, std::max(1.0, front));
    uint32_t* d_valid = reinterpret_cast<uint32_t*>(ctx->d_scalar + 4);
    {
      StageTimer t(ctx, OCGS_STAGE_BINNING);
      CK(launch_tile_count_sorted(sorted, M, bin, st->d_cams, N, tw, th, st->ntiles, counts, s));
      CK(scan_exclusive_u64(counts, counts, M, ctx->d_scalar, scratch, s));
      CK(launch_count_below(skeys, VN, 0xffffffffu, d_valid, s));  // records with a non-empty screen box
    }
    CK(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, 5 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    ocgs_status rs = read_status(ctx, &status);
    if (rs != OCGS_OK) return rs;
    const uint64_t K1_64 = ctx->h_scalar[0];
    const uint32_t n_valid = *reinterpret_cast<const uint32_t*>(ctx->h_scalar + 4);
    if (K1_64 > (uint64_t)INT32_MAX)
      return set_err(ctx, OCGS_ERR_CAPACITY, "more than 2^31-1 (tile, Gaussian) pairs; split the views");
    const uint32_t K1 = (uint32_t)K1_64;
    const bool second = M < n_valid;  // records behind the front remain
    const int tbits = bits_for((uint64_t)pl.tiles);
    const uint32_t n_t = (uint32_t)pl.tiles;

    uint32_t *pkey, *pval, *pkey_alt, *pval_alt;
    CK(tmp.alloc(&pkey, K1));
    CK(keep.alloc(&pval, K1));
    CK(tmp.alloc(&pkey_alt, K1));
    CK(keep.alloc(&pval_alt, K1));
    char* pscratch;
    CK(tmp.alloc(&pscratch, radix_scratch_bytes(K1)));
    {
      StageTimer t(ctx, OCGS_STAGE_BINNING);
      CK(launch_duplicate(sorted, counts, reinterpret_cast<const uint64_t*>(ctx->d_scalar), M, bin, st->d_cams, N,
                          tw, th, K1, pkey, pval, s));
    }
    bool palt = false;
    {
      StageTimer t(ctx, OCGS_STAGE_TILE_SORT);
      CK(radix_sort_pairs(pkey, pval, pkey_alt, pval_alt, K1, tbits, pscratch, &palt, s));
    }
    st->vals = palt ? pval_alt : pval;
    {
      StageTimer t(ctx, OCGS_STAGE_BINNING);
      CK(launch_tile_ranges(palt ? pkey_alt : pkey, K1, st->ranges, s));
    }
    uint32_t *queue, *wk, *ids, *wk_alt, *ids_alt;
    CK(tmp.alloc(&queue, 1));
    CK(tmp.alloc(&wk, n_t));
    CK(tmp.alloc(&ids, n_t));
    CK(tmp.alloc(&wk_alt, n_t));
    CK(tmp.alloc(&ids_alt, n_t));
    char* tscratch;
    CK(tmp.alloc(&tscratch, std::max(radix_scratch_bytes(n_t), scan_scratch_bytes(n_t + 1))));
    CK(cudaMemsetAsync(queue, 0, sizeof(uint32_t), s));
    CK(launch_tile_order(st->ranges, n_t, wk, ids, s));
    bool talt = false;
    CK(radix_sort_pairs(wk, ids, wk_alt, ids_alt, n_t, 8, tscratch, &talt, s));
    // the first pass leaves each pixel's state for the second: T and the last
    // blended position (the kept state, or scratch), the stop flags, the open tiles
    const bool img = out != nullptr;
    float* t_fin = keep_state && img ? st->t_final : nullptr;
    uint32_t* lst = keep_state && img ? st->last : nullptr;
    uint32_t* open = nullptr;
    uint8_t* done = nullptr;
    if (second) {
      if (!t_fin) CK(tmp.alloc(&t_fin, pl.P));
      if (!lst && img) CK(tmp.alloc(&lst, pl.P));
      CK(tmp.alloc(&open, n_t));
      CK(tmp.alloc(&done, pl.P));
      CK(cudaMemsetAsync(open, 0, sizeof(uint32_t) * n_t, s));
    }
    RasterArgs ra{};
    ra.ewa = ewa ? 1 : 0;
    ra.cams = st->d_cams;
    ra.tile_prefix = st->d_tile_prefix;
    ra.n_views = V;
    ra.n_gauss = N;
    ra.n_tiles = n_t;
    ra.ranges = st->ranges;
    ra.vals = st->vals;
    ra.rec = st->rec;
    if (img) ra.out = ImgPtrs{out->rgb, out->alpha, out->depth, out->normal, out->depth2};
    ra.t_final = t_fin;
    ra.last = lst;
    ra.score = score;
    ra.tile_order = talt ? ids_alt : ids;
    ra.queue = queue;
    ra.persistent_ctas = ctx->sm_count * (2048 * st->ppt / (tw * th));
    ra.open = open;
    ra.done = done;
    {
      StageTimer t(ctx, OCGS_STAGE_RASTER_FWD);
      CK(launch_raster_forward(ra, tw, th, st->ppt, st->batch, img, s));
    }
    uint32_t K2 = 0;
    uint32_t* P = nullptr;
    const uint32_t n_back = second ? n_valid - M : 0u;  // records behind the front
    // candidates of the second pass: the sorted order's first M entries are no longer
    // needed, nor are the depth keys (flag and position scratch)
    uint32_t* cand = order == sorted ? order_alt : order;
    uint32_t* n_cand = reinterpret_cast<uint32_t*>(ctx->d_scalar + 7);
    if (second) {
      CK(tmp.alloc(&P, (size_t)n_t + 1));
      {
        StageTimer t(ctx, OCGS_STAGE_BINNING);
        CK(scan_exclusive_u32(open, P, n_t, P + n_t, tscratch, s));
        // the records behind the front whose screen box meets an open tile, then their exact counts
        CK(launch_open_candidates(sorted + M, n_back, bin, st->d_cams, N, P, dkey, dkey_alt, cand, n_cand, scratch,
                                  s));
        CK(launch_open_count(cand, n_back, n_cand, bin, st->d_cams, N, tw, th, P, counts, s));
        CK(scan_exclusive_u64(counts, counts, n_back, ctx->d_scalar + 5, scratch, s));
      }
      CK(cudaMemcpyAsync(ctx->h_scalar + 5, ctx->d_scalar + 5, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      const uint64_t K2_64 = ctx->h_scalar[5];
      if ((uint64_t)K1 + K2_64 > (uint64_t)INT32_MAX)
        return set_err(ctx, OCGS_ERR_CAPACITY, "more than 2^31-1 (tile, Gaussian) pairs; split the views");
      K2 = (uint32_t)K2_64;
    }
    if (K2) {
      uint32_t *qkey, *qval, *qkey_alt, *qval_alt;
      CK(tmp.alloc(&qkey, K2));
      CK(keep.alloc(&qval, K2));
      CK(tmp.alloc(&qkey_alt, K2));
      CK(keep.alloc(&qval_alt, K2));
      char* qscratch;
      CK(tmp.alloc(&qscratch, radix_scratch_bytes(K2)));
      CK(keep.alloc(&st->ranges2, n_t));
      CK(cudaMemsetAsync(st->ranges2, 0, sizeof(uint2) * n_t, s));
      {
        StageTimer t(ctx, OCGS_STAGE_BINNING);
        uint32_t* open_ids;
        CK(tmp.alloc(&open_ids, n_t));
        CK(launch_duplicate_open(cand, counts, ctx->d_scalar + 5, n_back, n_cand, bin, st->d_cams, N, tw, th, open,
                                 P, n_t, open_ids, K2, qkey, qval, s));
      }
      bool qalt = false;
      {
        StageTimer t(ctx, OCGS_STAGE_TILE_SORT);
        CK(radix_sort_pairs(qkey, qval, qkey_alt, qval_alt, K2, tbits, qscratch, &qalt, s));
      }
      st->vals2 = qalt ? qval_alt : qval;
      uint32_t* n_again = reinterpret_cast<uint32_t*>(ctx->d_scalar + 6);
      {
        StageTimer t(ctx, OCGS_STAGE_BINNING);
        CK(launch_tile_ranges(qalt ? qkey_alt : qkey, K2, st->ranges2, s));
        CK(cudaMemsetAsync(n_again, 0, sizeof(uint32_t), s));
        CK(launch_second_queue(st->ranges2, n_t, wk, ids, n_again, s));
        CK(radix_sort_pairs(wk, ids, wk_alt, ids_alt, n_t, 8, tscratch, &talt, s));
      }
      RasterArgs rb = ra;
      rb.ranges = st->ranges2;
      rb.vals = st->vals2;
      rb.prior = st->ranges;
      rb.tile_order = talt ? ids_alt : ids;
      rb.n_queue = n_again;
      rb.open = nullptr;
      CK(cudaMemsetAsync(queue, 0, sizeof(uint32_t), s));
      {
        StageTimer t(ctx, OCGS_STAGE_RASTER_FWD);
        CK(launch_raster_forward(rb, tw, th, st->ppt, st->batch, img, s));
      }
    }
    K = K1 + K2;
    st->K = K;
    if (keep_state) {
      // the backward's work order: longest complete lists first
      uint32_t *bids, *bids_alt;
      CK(keep.alloc(&bids, n_t));
      CK(keep.alloc(&bids_alt, n_t));
      CK(launch_tile_order(st->ranges, n_t, wk, bids, s, st->ranges2));
      bool balt = false;
      CK(radix_sort_pairs(wk, bids, wk_alt, bids_alt, n_t, 8, tscratch, &balt, s));
      st->tile_order = balt ? bids_alt : bids;
    }
  }

  ctx->stats.n_gaussians = N;
  ctx->stats.n_views = V;
  ctx->stats.n_pixels = pl.P;
  ctx->stats.n_pairs = K;
  ctx->stats.n_tiles = pl.tiles;
  ctx->stats.tile_w = tw;
  ctx->stats.tile_h = th;
  ctx->stats.n_visible = -1;
  if (keep_state) keep.release_to(st->allocs);
  if (status & kStatusNonFinite)
    return set_err(ctx, OCGS_ERR_NONFINITE, "non-finite Gaussian parameters (those Gaussians were not rendered)");
  return OCGS_OK;
}

// Buffers of one pruning-sweep chunk with a fixed pair capacity: everything a
// forward pass needs, allocated once, so that the pass can be enqueued without
// allocation, host copy or host synchronisation (and hence captured).
struct SweepWs {
  RecPtrs rec{};
  int32_t* ntiles = nullptr;
  uint2* ranges = nullptr;
  float4* bin = nullptr;
  uint32_t *dkey = nullptr, *order = nullptr, *dkey_alt = nullptr, *order_alt = nullptr;
  uint64_t *counts = nullptr, *total = nullptr;
  uint32_t* n32 = nullptr;
  char *scratch = nullptr, *pscratch = nullptr, *tscratch = nullptr;
  uint32_t *pkey = nullptr, *pval = nullptr, *pkey_alt = nullptr, *pval_alt = nullptr;
  uint32_t *queue = nullptr, *wk = nullptr, *ids = nullptr, *wk_alt = nullptr, *ids_alt = nullptr;
  float* t_final = nullptr;
  uint32_t* last = nullptr;
  uint32_t vn_max = 0, cap = 0;
  int64_t tiles_max = 0;
};

cudaError_t alloc_sweep_ws(Arena& a, SweepWs& w, uint32_t vn_max, int64_t tiles_max, uint32_t cap) {
  w.vn_max = vn_max;
  w.tiles_max = tiles_max;
  w.cap = cap;
  cudaError_t e = cudaSuccess;
#define OCGS_A(ptr, n) if (e == cudaSuccess) e = a.alloc(&(ptr), (size_t)(n))
  OCGS_A(w.rec.g0, vn_max); OCGS_A(w.rec.g1, vn_max); OCGS_A(w.rec.g2, vn_max);
  OCGS_A(w.rec.a0, vn_max); OCGS_A(w.rec.a1, vn_max);
  OCGS_A(w.ntiles, vn_max); OCGS_A(w.ranges, tiles_max); OCGS_A(w.bin, 3 * (size_t)vn_max);
  OCGS_A(w.dkey, vn_max); OCGS_A(w.order, vn_max); OCGS_A(w.dkey_alt, vn_max); OCGS_A(w.order_alt, vn_max);
  OCGS_A(w.counts, vn_max); OCGS_A(w.total, 1); OCGS_A(w.n32, 1);
  OCGS_A(w.scratch, std::max(radix_scratch_bytes(vn_max), scan_scratch_bytes(vn_max)));
  OCGS_A(w.pkey, cap); OCGS_A(w.pval, cap); OCGS_A(w.pkey_alt, cap); OCGS_A(w.pval_alt, cap);
  OCGS_A(w.pscratch, radix_scratch_bytes(cap));
  OCGS_A(w.queue, 1); OCGS_A(w.wk, tiles_max); OCGS_A(w.ids, tiles_max); OCGS_A(w.wk_alt, tiles_max);
  OCGS_A(w.ids_alt, tiles_max); OCGS_A(w.tscratch, radix_scratch_bytes((uint32_t)tiles_max));
  OCGS_A(w.t_final, 1); OCGS_A(w.last, 1);
#undef OCGS_A
  return e;
}

// One chunk of the pruning sweep (V <= 16 views) in capacity mode: the pair
// count stays on the device (clamped to w.cap; an overflow raises the status
// word's capacity bit and the result must then be discarded).
ocgs_status enqueue_sweep_chunk(ocgs_ctx* ctx, const ocgs_gaussians* g, int V, const DevCam* d_cams,
                                const int* d_prefix, int64_t n_tiles, SweepWs& w, float* score, cudaStream_t s) {
  const int tw = ctx->opts.tile_w, th = ctx->opts.tile_h, ppt = ctx->opts.pixels_per_thread;
  const int64_t N = g->n;
  const uint32_t VN = (uint32_t)(N * V);
  CK(cudaMemsetAsync(w.ranges, 0, sizeof(uint2) * n_tiles, s));
  CK(launch_preprocess(gptrs(g), N, g->sh_degree, d_cams, V, tw, th, w.rec, w.ntiles, w.bin, w.dkey, ctx->d_status,
                       s));
  CK(launch_tile_count(w.bin, d_cams, N, VN, tw, th, w.ntiles, w.dkey, s));
  bool alt = false;
  CK(radix_sort_pairs(w.dkey, w.order, w.dkey_alt, w.order_alt, VN, 32, w.scratch, &alt, s, nullptr, true));
  uint32_t* sorted = alt ? w.order_alt : w.order;
  CK(launch_gather_counts(sorted, w.ntiles, w.counts, VN, s));
  CK(scan_exclusive_u64(w.counts, w.counts, VN, w.total, w.scratch, s));
  CK(launch_clamp_count(w.total, w.cap, w.n32, ctx->d_status, s));
  CK(launch_duplicate(sorted, w.counts, w.total, VN, w.bin, d_cams, N, tw, th, w.cap, w.pkey, w.pval, s));
  bool palt = false;
  CK(radix_sort_pairs(w.pkey, w.pval, w.pkey_alt, w.pval_alt, w.cap, bits_for((uint64_t)n_tiles), w.pscratch, &palt,
                      s, w.n32));
  uint32_t* skey = palt ? w.pkey_alt : w.pkey;
  uint32_t* svals = palt ? w.pval_alt : w.pval;
  CK(launch_tile_ranges(skey, w.cap, w.ranges, s, w.n32));
  RasterArgs ra{};
  ra.cams = d_cams;
  ra.tile_prefix = d_prefix;
  ra.n_views = V;
  ra.n_gauss = N;
  ra.n_tiles = (uint32_t)n_tiles;
  ra.ranges = w.ranges;
  ra.vals = svals;
  ra.rec = w.rec;
  ra.t_final = w.t_final;
  ra.last = w.last;
  ra.score = score;
  if (ctx->opts.persistent) {
    CK(cudaMemsetAsync(w.queue, 0, sizeof(uint32_t), s));
    CK(launch_tile_order(w.ranges, (uint32_t)n_tiles, w.wk, w.ids, s));
    bool talt = false;
    CK(radix_sort_pairs(w.wk, w.ids, w.wk_alt, w.ids_alt, (uint32_t)n_tiles, 8, w.tscratch, &talt, s));
    ra.tile_order = talt ? w.ids_alt : w.ids;
    ra.queue = w.queue;
    ra.persistent_ctas = ctx->sm_count * (2048 * ppt / (tw * th));
  }
  CK(launch_raster_forward(ra, tw, th, ppt, ctx->opts.batch, false, s));
  return OCGS_OK;
}

}  // namespace

extern "C" {

const char* ocgs_status_str(ocgs_status s) {
  const int i = (int)s;
  if (i < 0 || i >= (int)(sizeof(kStatusNames) / sizeof(kStatusNames[0]))) return "OCGS_ERR_UNKNOWN";
  return kStatusNames[i];
}

const char* ocgs_last_error(const ocgs_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int32_t ocgs_abi_version(void) { return OCGS_ABI_VERSION; }

ocgs_status ocgs_create(ocgs_ctx** out, int32_t device, void* stream) {
  if (!out) return OCGS_ERR_ARG;
  *out = nullptr;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0) return OCGS_ERR_CUDA;
  if (device < 0 || device >= n_dev) return OCGS_ERR_ARG;
  ocgs_ctx* ctx = new ocgs_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return OCGS_ERR_CUDA; }
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) { delete ctx; return OCGS_ERR_CUDA; }
  uint64_t thr = UINT64_MAX;
  cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  if (cudaMalloc(&ctx->d_status, 256) != cudaSuccess || cudaMalloc(&ctx->d_scalar, 256) != cudaSuccess ||
      cudaHostAlloc(&ctx->h_scalar, 256, cudaHostAllocDefault) != cudaSuccess) {
    ocgs_destroy(ctx);
    return OCGS_ERR_OOM;
  }
  cudaMemset(ctx->d_status, 0, 256);
  *out = ctx;
  return OCGS_OK;
}

ocgs_status ocgs_destroy(ocgs_ctx* ctx) {
  if (!ctx) return OCGS_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_scalar) cudaFree(ctx->d_scalar);
  if (ctx->h_scalar) cudaFreeHost(ctx->h_scalar);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  delete ctx;
  return OCGS_OK;
}

ocgs_status ocgs_set_stream(ocgs_ctx* ctx, void* stream) {
  if (!ctx) return OCGS_ERR_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return OCGS_OK;
}

ocgs_status ocgs_set_options(ocgs_ctx* ctx, const ocgs_options* o) {
  if (!ctx || !o) return OCGS_ERR_ARG;
  const int ppt = o->pixels_per_thread == 0 ? 2 : o->pixels_per_thread;
  const int batch = o->batch == 0 ? 32 : o->batch;
  if (!valid_tile(o->tile_w, o->tile_h, ppt, 32))
    return set_err(ctx, OCGS_ERR_ARG, "tile must be 16x16, 16x8, 8x8 or 32x8 with 1 or 2 pixels per thread (4 for 16x16 and 16x8)");
  if (!valid_tile(o->tile_w, o->tile_h, ppt, batch))
    return set_err(ctx, OCGS_ERR_ARG, "batch must be 32, or 16 or 64 with 16x16 tiles and 2 or 4 pixels per thread "
                                      "or 16x8 tiles and 4");
  if (!(o->front_fraction >= 0.f && o->front_fraction <= 1.f))
    return set_err(ctx, OCGS_ERR_ARG, "front_fraction must lie in [0, 1]");
  ctx->opts = *o;
  ctx->opts.pixels_per_thread = ppt;
  ctx->opts.batch = batch;
  return OCGS_OK;
}

ocgs_status ocgs_set_coverage(ocgs_ctx* ctx, int32_t rect) {
  if (!ctx || (rect != 0 && rect != 1)) return OCGS_ERR_ARG;
  ctx->cover_rect = rect;
  return OCGS_OK;
}

ocgs_status ocgs_get_options(const ocgs_ctx* ctx, ocgs_options* o) {
  if (!ctx || !o) return OCGS_ERR_ARG;
  *o = ctx->opts;
  return OCGS_OK;
}

ocgs_status ocgs_get_stats(const ocgs_ctx* ctx, ocgs_stats* s) {
  if (!ctx || !s) return OCGS_ERR_ARG;
  *s = ctx->stats;
  return OCGS_OK;
}

ocgs_status ocgs_sync(ocgs_ctx* ctx) {
  if (!ctx) return OCGS_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  int status = 0;
  ocgs_status r = read_status(ctx, &status);
  if (r != OCGS_OK) return r;
  CK(cudaGetLastError());
  if (status & kStatusCapacity)
    return set_err(ctx, OCGS_ERR_CAPACITY, "more (tile, Gaussian) pairs than a captured graph's capacity; re-create it");
  if (status & kStatusNonFinite)
    return set_err(ctx, OCGS_ERR_NONFINITE, "non-finite Gaussian parameters or optimiser gradients");
  if (status & kStatusTimeout) return set_err(ctx, OCGS_ERR_TIMEOUT, "a bounded device wait gave up");
  return OCGS_OK;
}

ocgs_status ocgs_render(ocgs_ctx* ctx, const ocgs_gaussians* g, const ocgs_camera* cams, int32_t n_views,
                        const ocgs_image* out, float* score, ocgs_fwd_state** state) {
  if (!ctx) return OCGS_ERR_ARG;
  ocgs_status r = check_gaussians(ctx, g);
  if (r != OCGS_OK) return r;
  r = check_cameras(ctx, cams, n_views);
  if (r != OCGS_OK) return r;
  if (!out || !out->rgb || !out->alpha || !out->depth || !out->normal)
    return set_err(ctx, OCGS_ERR_ARG, "every output image pointer must be non-NULL");
  CK(cudaSetDevice(ctx->device));
  if (state) *state = nullptr;
  ocgs_fwd_state* st = new ocgs_fwd_state();
  r = forward_pass(ctx, g, cams, n_views, out, score, st, true);
  if (r != OCGS_OK && r != OCGS_ERR_NONFINITE) {
    free_state(st);
    delete st;
    return r;
  }
  if (state) {
    *state = st;
  } else {
    free_state(st);
    delete st;
  }
  return r;
}

ocgs_status ocgs_render_backward(ocgs_ctx* ctx, const ocgs_fwd_state* st, const ocgs_gaussians* g,
                                 const ocgs_image* d_out, const ocgs_gaussians_out* d_params) {
  if (!ctx) return OCGS_ERR_ARG;
  if (!st || st->ctx != ctx) return set_err(ctx, OCGS_ERR_STATE, "forward state missing or from another context");
  ocgs_status r = check_gaussians(ctx, g);
  if (r != OCGS_OK) return r;
  if (g->n != st->N || g->sh_degree != st->deg)
    return set_err(ctx, OCGS_ERR_ARG, "gaussians differ from the forward call (n or sh_degree)");
  if (!d_out) return set_err(ctx, OCGS_ERR_ARG, "d_out is NULL");
  if (!d_params || (st->N > 0 && (!d_params->xyz || !d_params->quat || !d_params->scale || !d_params->opacity ||
                                  !d_params->sh)))
    return set_err(ctx, OCGS_ERR_ARG, "a gradient pointer is NULL");
  if (st->N == 0) return OCGS_OK;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  Arena tmp(ctx);
  const uint64_t VN = (uint64_t)st->N * st->V;
  float* grad_rec;
  CK(tmp.alloc(&grad_rec, VN * kGradStride));
  StageTimer t_bwd(ctx, OCGS_STAGE_RASTER_BWD);
  CK(cudaMemsetAsync(grad_rec, 0, VN * kGradStride * sizeof(float), s));
  RasterBwdArgs ba{};
  ba.cams = st->d_cams;
  ba.tile_prefix = st->d_tile_prefix;
  ba.n_views = st->V;
  ba.n_gauss = st->N;
  ba.n_tiles = st->n_tiles;
  ba.ranges = st->ranges;
  ba.vals = st->vals;
  ba.ranges2 = st->ranges2;
  ba.vals2 = st->vals2;
  ba.rec = st->rec;
  ba.t_final = st->t_final;
  ba.last = st->last;
  ba.d_out = ImgPtrs{d_out->rgb, d_out->alpha, d_out->depth, d_out->normal, d_out->depth2};
  ba.grad_rec = grad_rec;
  ba.tile_order = st->tile_order;
  uint32_t* queue = nullptr;
  if (st->persistent) {
    CK(tmp.alloc(&queue, 1));
    CK(cudaMemsetAsync(queue, 0, sizeof(uint32_t), s));
    ba.persistent_ctas = ctx->sm_count * (2048 * st->ppt / (st->tile_w * st->tile_h));
  }
  ba.queue = queue;
  CK(launch_raster_backward(ba, st->tile_w, st->tile_h, st->ppt, st->batch, s));
  t_bwd.stop();
  GaussOut go{d_params->xyz, d_params->quat, d_params->scale, d_params->opacity, d_params->sh};
  {
    StageTimer t(ctx, OCGS_STAGE_PREPROCESS_BWD);
    CK(launch_preprocess_backward(gptrs(g), st->N, st->deg, st->d_cams, st->V, grad_rec, st->ntiles, go, s));
  }
  return OCGS_OK;
}

ocgs_status ocgs_state_release(ocgs_ctx* ctx, ocgs_fwd_state* st) {
  if (!ctx || !st) return OCGS_ERR_ARG;
  if (st->ctx != ctx) return set_err(ctx, OCGS_ERR_STATE, "state from another context");
  cudaSetDevice(ctx->device);
  free_state(st);
  delete st;
  return OCGS_OK;
}

ocgs_status ocgs_background_loss(ocgs_ctx* ctx, const float* alpha, const uint8_t* mask,
                                 const ocgs_camera* cams, int32_t n_views, float gamma, double* loss,
                                 float* d_alpha) {
  if (!ctx) return OCGS_ERR_ARG;
  if (!alpha || !mask || !loss) return set_err(ctx, OCGS_ERR_ARG, "alpha, mask and loss must be non-NULL");
  if (!std::isfinite(gamma)) return set_err(ctx, OCGS_ERR_ARG, "gamma must be finite");
  LossPlan lp;
  ocgs_status r = plan_loss(ctx, cams, n_views, &lp);
  if (r != OCGS_OK) return r;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  Arena tmp(ctx);
  DevCam* d_cams;
  int* d_prefix;
  double* partial;
  CK(tmp.alloc(&d_cams, n_views));
  CK(tmp.alloc(&d_prefix, n_views + 1));
  CK(tmp.alloc(&partial, lp.blocks));
  StageTimer t(ctx, OCGS_STAGE_LOSS);
  CK(cudaMemcpyAsync(d_cams, lp.cams.data(), sizeof(DevCam) * n_views, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_prefix, lp.prefix.data(), sizeof(int) * (n_views + 1), cudaMemcpyHostToDevice, s));
  CK(launch_background_loss(alpha, mask, d_cams, n_views, d_prefix, lp.blocks, gamma, partial, loss, d_alpha, s));
  return OCGS_OK;
}

ocgs_status ocgs_masked_l1(ocgs_ctx* ctx, const float* rgb, const float* target, const uint8_t* mask,
                           const ocgs_camera* cams, int32_t n_views, float weight, double* loss, float* d_rgb) {
  if (!ctx) return OCGS_ERR_ARG;
  if (!rgb || !target || !mask || !loss) return set_err(ctx, OCGS_ERR_ARG, "rgb, target, mask and loss must be non-NULL");
  if (!std::isfinite(weight)) return set_err(ctx, OCGS_ERR_ARG, "weight must be finite");
  LossPlan lp;
  ocgs_status r = plan_loss(ctx, cams, n_views, &lp);
  if (r != OCGS_OK) return r;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  Arena tmp(ctx);
  DevCam* d_cams;
  int* d_prefix;
  double* partial;
  CK(tmp.alloc(&d_cams, n_views));
  CK(tmp.alloc(&d_prefix, n_views + 1));
  CK(tmp.alloc(&partial, lp.blocks));
  StageTimer t(ctx, OCGS_STAGE_LOSS);
  CK(cudaMemcpyAsync(d_cams, lp.cams.data(), sizeof(DevCam) * n_views, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_prefix, lp.prefix.data(), sizeof(int) * (n_views + 1), cudaMemcpyHostToDevice, s));
  CK(launch_masked_l1(rgb, target, mask, d_cams, n_views, d_prefix, lp.blocks, weight, partial, loss, d_rgb, s));
  return OCGS_OK;
}

ocgs_status ocgs_ssim(ocgs_ctx* ctx, const float* rgb, const float* target, const uint8_t* mask,
                      const ocgs_camera* cams, int32_t n_views, float weight, double* ssim, double* ssim_masked,
                      float* d_rgb) {
  if (!ctx) return OCGS_ERR_ARG;
  if (!rgb || !target || !mask || !ssim) return set_err(ctx, OCGS_ERR_ARG, "rgb, target, mask and ssim must be non-NULL");
  if (!std::isfinite(weight)) return set_err(ctx, OCGS_ERR_ARG, "weight must be finite");
  LossPlan lp;
  ocgs_status r = plan_loss(ctx, cams, n_views, &lp);
  if (r != OCGS_OK) return r;
  std::vector<int> prefix(n_views + 1, 0);
  int64_t P = 0;
  for (int v = 0; v < n_views; ++v) {
    prefix[v + 1] = prefix[v] + ssim_tiles(lp.cams[v].W, lp.cams[v].H);
    P += (int64_t)lp.cams[v].W * lp.cams[v].H;
  }
  const int tiles = prefix[n_views];
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  Arena tmp(ctx);
  DevCam* d_cams;
  int* d_prefix;
  double* partial;
  float* gmap = nullptr;
  CK(tmp.alloc(&d_cams, n_views));
  CK(tmp.alloc(&d_prefix, n_views + 1));
  CK(tmp.alloc(&partial, 3 * (size_t)tiles));
  if (d_rgb) CK(tmp.alloc(&gmap, 9 * (size_t)P));
  StageTimer t(ctx, OCGS_STAGE_LOSS);
  CK(cudaMemcpyAsync(d_cams, lp.cams.data(), sizeof(DevCam) * n_views, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_prefix, prefix.data(), sizeof(int) * (n_views + 1), cudaMemcpyHostToDevice, s));
  CK(launch_ssim(rgb, target, mask, d_cams, n_views, d_prefix, tiles, P, weight, partial, gmap, ssim, ssim_masked,
                 d_rgb, s));
  return OCGS_OK;
}

ocgs_status ocgs_masked_psnr(ocgs_ctx* ctx, const float* rgb, const float* target, const uint8_t* mask,
                             const ocgs_camera* cams, int32_t n_views, float max_i, double* psnr) {
  if (!ctx) return OCGS_ERR_ARG;
  if (!rgb || !target || !mask || !psnr) return set_err(ctx, OCGS_ERR_ARG, "rgb, target, mask and psnr must be non-NULL");
  if (!(std::isfinite(max_i) && max_i > 0.f)) return set_err(ctx, OCGS_ERR_ARG, "max_i must be finite and > 0");
  LossPlan lp;
  ocgs_status r = plan_loss(ctx, cams, n_views, &lp);
  if (r != OCGS_OK) return r;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  Arena tmp(ctx);
  DevCam* d_cams;
  int* d_prefix;
  double* partial;
  CK(tmp.alloc(&d_cams, n_views));
  CK(tmp.alloc(&d_prefix, n_views + 1));
  CK(tmp.alloc(&partial, 2 * (size_t)lp.blocks));
  StageTimer t(ctx, OCGS_STAGE_LOSS);
  CK(cudaMemcpyAsync(d_cams, lp.cams.data(), sizeof(DevCam) * n_views, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_prefix, lp.prefix.data(), sizeof(int) * (n_views + 1), cudaMemcpyHostToDevice, s));
  CK(launch_masked_psnr(rgb, target, mask, d_cams, n_views, d_prefix, lp.blocks, (double)max_i, partial, psnr, s));
  return OCGS_OK;
}

ocgs_status ocgs_depth_distortion(ocgs_ctx* ctx, const float* alpha, const float* depth, const float* depth2,
                                  const ocgs_camera* cams, int32_t n_views, float weight, double* loss, float* d_alpha,
                                  float* d_depth, float* d_depth2) {
  if (!ctx) return OCGS_ERR_ARG;
  if (!alpha || !depth || !depth2 || !loss) return set_err(ctx, OCGS_ERR_ARG, "alpha, depth, depth2 and loss must be non-NULL");
  if ((d_alpha != nullptr) != (d_depth != nullptr) || (d_alpha != nullptr) != (d_depth2 != nullptr))
    return set_err(ctx, OCGS_ERR_ARG, "d_alpha, d_depth and d_depth2 must all be given or all be NULL");
  if (!std::isfinite(weight)) return set_err(ctx, OCGS_ERR_ARG, "weight must be finite");
  LossPlan lp;
  ocgs_status r = plan_loss(ctx, cams, n_views, &lp);
  if (r != OCGS_OK) return r;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  Arena tmp(ctx);
  DevCam* d_cams;
  int* d_prefix;
  double* partial;
  CK(tmp.alloc(&d_cams, n_views));
  CK(tmp.alloc(&d_prefix, n_views + 1));
  CK(tmp.alloc(&partial, lp.blocks));
  StageTimer t(ctx, OCGS_STAGE_LOSS);
  CK(cudaMemcpyAsync(d_cams, lp.cams.data(), sizeof(DevCam) * n_views, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_prefix, lp.prefix.data(), sizeof(int) * (n_views + 1), cudaMemcpyHostToDevice, s));
  CK(launch_depth_distortion(alpha, depth, depth2, d_cams, n_views, d_prefix, lp.blocks, weight, partial, loss,
                             d_alpha, d_depth, d_depth2, s));
  return OCGS_OK;
}

ocgs_status ocgs_normal_consistency(ocgs_ctx* ctx, const float* alpha, const float* depth, const float* normal,
                                    const ocgs_camera* cams, int32_t n_views, float weight, float a_min, double* loss,
                                    float* d_alpha, float* d_depth, float* d_normal) {
  if (!ctx) return OCGS_ERR_ARG;
  if (!alpha || !depth || !normal || !loss) return set_err(ctx, OCGS_ERR_ARG, "alpha, depth, normal and loss must be non-NULL");
  if ((d_alpha != nullptr) != (d_depth != nullptr) || (d_alpha != nullptr) != (d_normal != nullptr))
    return set_err(ctx, OCGS_ERR_ARG, "d_alpha, d_depth and d_normal must all be given or all be NULL");
  if (!std::isfinite(weight) || !std::isfinite(a_min) || a_min < 0.f)
    return set_err(ctx, OCGS_ERR_ARG, "weight must be finite and a_min finite and >= 0");
  LossPlan lp;
  ocgs_status r = plan_loss(ctx, cams, n_views, &lp);
  if (r != OCGS_OK) return r;
  int64_t P = 0;
  for (int v = 0; v < n_views; ++v) {
    if (!(cams[v].fx > 0.f && cams[v].fy > 0.f) || !std::isfinite(cams[v].cx) || !std::isfinite(cams[v].cy))
      return set_err(ctx, OCGS_ERR_ARG, "camera intrinsics must be finite with fx, fy > 0");
    P += (int64_t)cams[v].width * cams[v].height;
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  Arena tmp(ctx);
  DevCam* d_cams;
  int* d_prefix;
  double* partial;
  float* gmap = nullptr;
  CK(tmp.alloc(&d_cams, n_views));
  CK(tmp.alloc(&d_prefix, n_views + 1));
  CK(tmp.alloc(&partial, lp.blocks));
  if (d_alpha) CK(tmp.alloc(&gmap, 6 * (size_t)P));
  StageTimer t(ctx, OCGS_STAGE_LOSS);
  CK(cudaMemcpyAsync(d_cams, lp.cams.data(), sizeof(DevCam) * n_views, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_prefix, lp.prefix.data(), sizeof(int) * (n_views + 1), cudaMemcpyHostToDevice, s));
  CK(launch_normal_consistency(alpha, depth, normal, d_cams, n_views, d_prefix, lp.blocks, weight, a_min, partial,
                               gmap, loss, d_alpha, d_depth, d_normal, s));
  return OCGS_OK;
}

ocgs_status ocgs_state_query(ocgs_ctx* ctx, const ocgs_fwd_state* st, ocgs_state_info* info) {
  if (!ctx || !info) return OCGS_ERR_ARG;
  if (!st || st->ctx != ctx) return set_err(ctx, OCGS_ERR_STATE, "forward state missing or from another context");
  CK(cudaSetDevice(ctx->device));
  unsigned long long* d = reinterpret_cast<unsigned long long*>(ctx->d_scalar) + 2;
  CK(launch_sum_u32(st->last, st->P, d, ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_scalar + 2, d, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  info->n_pairs = st->K;
  info->n_pixels = st->P;
  info->n_tiles = st->n_tiles;
  info->n_views = st->V;
  info->n_evals = (int64_t)ctx->h_scalar[2];
  return OCGS_OK;
}

int64_t ocgs_kernel_launches(void) { return (int64_t)g_kernel_launches.load(); }

ocgs_status ocgs_profile_enable(ocgs_ctx* ctx, int32_t enable) {
  if (!ctx) return OCGS_ERR_ARG;
  if (ctx->prof || enable) CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof = enable != 0;
  ctx->ev_used = 0;
  for (int i = 0; i < 16; ++i) { ctx->prof_ms[i] = 0.0; ctx->prof_n[i] = 0; }
  return OCGS_OK;
}

ocgs_status ocgs_profile_read(ocgs_ctx* ctx, ocgs_profile* out) {
  if (!ctx || !out) return OCGS_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
    ctx->prof_ms[ctx->ev_stage[i]] += ms;
    ctx->prof_n[ctx->ev_stage[i]] += 1;
  }
  ctx->ev_used = 0;
  for (int i = 0; i < 16; ++i) { out->ms[i] = ctx->prof_ms[i]; out->launches[i] = ctx->prof_n[i]; }
  return OCGS_OK;
}

ocgs_status ocgs_accumulate_contribution(ocgs_ctx* ctx, const ocgs_gaussians* g, const ocgs_camera* cams,
                                         int32_t n_views, float* score) {
  if (!ctx) return OCGS_ERR_ARG;
  ocgs_status r = check_gaussians(ctx, g);
  if (r != OCGS_OK) return r;
  r = check_cameras(ctx, cams, n_views);
  if (r != OCGS_OK) return r;
  if (!score && g->n > 0) return set_err(ctx, OCGS_ERR_ARG, "score is NULL");
  if (g->n == 0) return OCGS_OK;
  CK(cudaSetDevice(ctx->device));
  // views are swept in chunks so that one chunk's pairs stay well inside the 2^31 limit
  const int chunk = 16;
  ocgs_status worst = OCGS_OK;
  int64_t pairs = 0;
  for (int v0 = 0; v0 < n_views; v0 += chunk) {
    const int nv = std::min(chunk, n_views - v0);
    ocgs_fwd_state st;
    r = forward_pass(ctx, g, cams + v0, nv, nullptr, score, &st, false);
    pairs += ctx->stats.n_pairs;
    if (r == OCGS_ERR_NONFINITE) worst = r;
    else if (r != OCGS_OK) return r;
  }
  ctx->stats.n_views = n_views;
  ctx->stats.n_pairs = pairs;
  return worst;
}

// The 3DGS variant of the pruning record (Appendix B): 3D Gaussians whose scale has
// three entries; the record format is the surfel one, so the pipeline is shared.
static ocgs_status check_gaussians3d(ocgs_ctx* ctx, const ocgs_gaussians3d* g, ocgs_gaussians* as2d) {
  if (!g) return set_err(ctx, OCGS_ERR_ARG, "gaussians is NULL");
  if (g->n < 0) return set_err(ctx, OCGS_ERR_ARG, "gaussians.n < 0");
  if (g->sh_degree < 0 || g->sh_degree > 3) return set_err(ctx, OCGS_ERR_ARG, "sh_degree must be 0..3");
  if (g->n > 0 && (!g->xyz || !g->quat || !g->scale || !g->opacity || !g->sh))
    return set_err(ctx, OCGS_ERR_ARG, "a Gaussian parameter pointer is NULL");
  if (g->n > 0 && (uintptr_t)g->quat % 16) return set_err(ctx, OCGS_ERR_ARG, "quat must be 16-byte aligned");
  *as2d = ocgs_gaussians{g->xyz, g->quat, g->scale, g->opacity, g->sh, g->n, g->sh_degree, 0};
  return OCGS_OK;
}

ocgs_status ocgs_render_3d(ocgs_ctx* ctx, const ocgs_gaussians3d* g, const ocgs_camera* cams, int32_t n_views,
                           const ocgs_image* out, float* score) {
  if (!ctx) return OCGS_ERR_ARG;
  ocgs_gaussians g2;
  ocgs_status r = check_gaussians3d(ctx, g, &g2);
  if (r != OCGS_OK) return r;
  r = check_cameras(ctx, cams, n_views);
  if (r != OCGS_OK) return r;
  if (!out || !out->rgb || !out->alpha || !out->depth || !out->normal)
    return set_err(ctx, OCGS_ERR_ARG, "rgb, alpha, depth and normal must be non-NULL");
  if (out->depth2) return set_err(ctx, OCGS_ERR_ARG, "the 3DGS variant has no depth2 plane");
  CK(cudaSetDevice(ctx->device));
  ocgs_fwd_state st;
  r = forward_pass(ctx, &g2, cams, n_views, out, score, &st, false, true);
  free_state(&st);
  return r;
}

ocgs_status ocgs_accumulate_contribution_3d(ocgs_ctx* ctx, const ocgs_gaussians3d* g, const ocgs_camera* cams,
                                            int32_t n_views, float* score) {
  if (!ctx) return OCGS_ERR_ARG;
  ocgs_gaussians g2;
  ocgs_status r = check_gaussians3d(ctx, g, &g2);
  if (r != OCGS_OK) return r;
  r = check_cameras(ctx, cams, n_views);
  if (r != OCGS_OK) return r;
  if (!score && g->n > 0) return set_err(ctx, OCGS_ERR_ARG, "score is NULL");
  if (g->n == 0) return OCGS_OK;
  CK(cudaSetDevice(ctx->device));
  const int chunk = 16;
  ocgs_status worst = OCGS_OK;
  for (int v0 = 0; v0 < n_views; v0 += chunk) {
    const int nv = std::min(chunk, n_views - v0);
    ocgs_fwd_state st;
    r = forward_pass(ctx, &g2, cams + v0, nv, nullptr, score, &st, false, true);
    free_state(&st);
    if (r == OCGS_ERR_NONFINITE) worst = r;
    else if (r != OCGS_OK) return r;
  }
  return worst;
}

ocgs_status ocgs_prune(ocgs_ctx* ctx, const float* score, float threshold, const ocgs_gaussians* in,
                       const ocgs_gaussians_out* out, int64_t* n_kept, int64_t* borderline,
                       int64_t borderline_cap, int64_t* n_borderline) {
  if (!ctx) return OCGS_ERR_ARG;
  ocgs_status r = check_gaussians(ctx, in);
  if (r != OCGS_OK) return r;
  if (!n_kept || !n_borderline) return set_err(ctx, OCGS_ERR_ARG, "n_kept and n_borderline must be non-NULL");
  if (!std::isfinite(threshold)) return set_err(ctx, OCGS_ERR_ARG, "threshold must be finite");
  if (in->n > 0 && (!score || !out || !out->xyz || !out->quat || !out->scale || !out->opacity || !out->sh))
    return set_err(ctx, OCGS_ERR_ARG, "score and every output pointer must be non-NULL");
  if (borderline_cap < 0 || (borderline_cap > 0 && !borderline))
    return set_err(ctx, OCGS_ERR_ARG, "bad borderline buffer");
  if (in->n >= (int64_t)0xffffffffll) return set_err(ctx, OCGS_ERR_CAPACITY, "n too large");
  *n_kept = 0;
  *n_borderline = 0;
  if (in->n == 0) return OCGS_OK;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const uint32_t n = (uint32_t)in->n;
  Arena tmp(ctx);
  uint32_t *keep, *keep_pos, *border, *border_pos;
  CK(tmp.alloc(&keep, n));
  CK(tmp.alloc(&keep_pos, n));
  CK(tmp.alloc(&border, n));
  CK(tmp.alloc(&border_pos, n));
  char* scratch;
  CK(tmp.alloc(&scratch, scan_scratch_bytes(n)));
  uint32_t* totals = reinterpret_cast<uint32_t*>(ctx->d_scalar);
  StageTimer t(ctx, OCGS_STAGE_PRUNE);
  CK(launch_prune_flags(score, n, threshold, keep, border, s));
  CK(scan_exclusive_u32(keep, keep_pos, n, totals, scratch, s));
  CK(scan_exclusive_u32(border, border_pos, n, totals + 1, scratch, s));
  GaussOut go{out->xyz, out->quat, out->scale, out->opacity, out->sh};
  CK(launch_prune_compact(gptrs(in), n, in->sh_degree, keep, keep_pos, border, border_pos, go,
                          borderline_cap > 0 ? borderline : nullptr, borderline_cap, s));
  t.stop();
  CK(cudaMemcpyAsync(ctx->h_scalar, totals, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const uint32_t* h = reinterpret_cast<const uint32_t*>(ctx->h_scalar);
  *n_kept = h[0];
  *n_borderline = h[1];
  return OCGS_OK;
}

ocgs_status ocgs_adam_step(ocgs_ctx* ctx, const ocgs_gaussians* grads, const ocgs_gaussians_out* params,
                           const ocgs_gaussians_out* m, const ocgs_gaussians_out* v, const ocgs_adam_config* cfg) {
  if (!ctx) return OCGS_ERR_ARG;
  if (!grads || !params || !m || !v || !cfg) return set_err(ctx, OCGS_ERR_ARG, "a required argument is NULL");
  if (grads->n < 0) return set_err(ctx, OCGS_ERR_ARG, "grads.n < 0");
  if (grads->sh_degree < 0 || grads->sh_degree > 3) return set_err(ctx, OCGS_ERR_ARG, "sh_degree must be 0..3");
  if (!(cfg->beta1 >= 0.0 && cfg->beta1 < 1.0 && cfg->beta2 >= 0.0 && cfg->beta2 < 1.0))
    return set_err(ctx, OCGS_ERR_ARG, "beta1 and beta2 must lie in [0, 1)");
  if (!(std::isfinite(cfg->eps) && cfg->eps > 0.0 && (float)cfg->eps > 0.f))
    return set_err(ctx, OCGS_ERR_ARG, "eps must be finite and > 0 in single precision");
  for (int k = 0; k < 5; ++k)
    if (!std::isfinite(cfg->lr[k]) || !std::isfinite((float)cfg->lr[k]))
      return set_err(ctx, OCGS_ERR_ARG, "learning rates must be finite in single precision");
  if (cfg->step < 1) return set_err(ctx, OCGS_ERR_ARG, "step must be >= 1");
  if (grads->n == 0) return OCGS_OK;
  const int64_t n = grads->n;
  const int64_t K = (int64_t)(grads->sh_degree + 1) * (grads->sh_degree + 1);
  const float* g[5] = {grads->xyz, grads->quat, grads->scale, grads->opacity, grads->sh};
  float* p[5] = {params->xyz, params->quat, params->scale, params->opacity, params->sh};
  float* mm[5] = {m->xyz, m->quat, m->scale, m->opacity, m->sh};
  float* vv[5] = {v->xyz, v->quat, v->scale, v->opacity, v->sh};
  const int64_t count[5] = {3 * n, 4 * n, 2 * n, n, 3 * K * n};
  AdamArgs a;
  for (int k = 0; k < 5; ++k) {
    if (!g[k] || !p[k] || !mm[k] || !vv[k]) return set_err(ctx, OCGS_ERR_ARG, "a parameter, gradient or moment pointer is NULL");
    const uintptr_t all = (uintptr_t)g[k] | (uintptr_t)p[k] | (uintptr_t)mm[k] | (uintptr_t)vv[k];
    if (all % 4) return set_err(ctx, OCGS_ERR_ARG, "arrays must be 4-byte aligned");
    a.seg[k] = AdamSeg{p[k], g[k], mm[k], vv[k], count[k], (float)cfg->lr[k], all % 16 == 0 ? 1 : 0};
  }
  // bias corrections 1 - beta^t in double, then single precision factors
  const double bc1 = 1.0 - std::pow(cfg->beta1, (double)cfg->step);
  const double bc2 = 1.0 - std::pow(cfg->beta2, (double)cfg->step);
  if (!(bc1 > 0.0 && bc2 > 0.0)) return set_err(ctx, OCGS_ERR_ARG, "bias correction 1 - beta^t is zero");
  a.beta1 = (float)cfg->beta1;
  a.beta2 = (float)cfg->beta2;
  a.one_m_beta1 = (float)(1.0 - cfg->beta1);
  a.one_m_beta2 = (float)(1.0 - cfg->beta2);
  a.inv_bc1 = (float)(1.0 / bc1);
  a.inv_bc2 = (float)(1.0 / bc2);
  a.eps = (float)cfg->eps;
  a.status = ctx->d_status;
  CK(cudaSetDevice(ctx->device));
  StageTimer t(ctx, OCGS_STAGE_ADAM);
  CK(launch_adam(a, ctx->sm_count, ctx->stream));
  return OCGS_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- autotuner
namespace {

int log2_bucket(int64_t x) {
  int b = 0;
  while (x > 1) { x >>= 1; ++b; }
  return b;
}

std::string tune_key(ocgs_ctx* ctx, const ocgs_gaussians* g, const ocgs_camera* cams, int V) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, ctx->device);
  int64_t pix = 0;
  for (int v = 0; v < V; ++v) pix += (int64_t)cams[v].width * cams[v].height;
  std::ostringstream os;
  std::string name(prop.name);
  for (char& c : name) if (c == ' ') c = '_';
  os << "v2/" << name << "/sm" << prop.multiProcessorCount << "/deg" << g->sh_degree << "/v" << V << "/n2^"
     << log2_bucket(g->n) << "/p2^" << log2_bucket(pix);
  return os.str();
}

}  // namespace

extern "C" ocgs_status ocgs_autotune(ocgs_ctx* ctx, const ocgs_gaussians* g, const ocgs_camera* cams,
                                     int32_t n_views, const char* cache_path, ocgs_tune_result* result) {
  if (!ctx || !result) return OCGS_ERR_ARG;
  ocgs_status r = check_gaussians(ctx, g);
  if (r != OCGS_OK) return r;
  r = check_cameras(ctx, cams, n_views);
  if (r != OCGS_OK) return r;
  CK(cudaSetDevice(ctx->device));
  std::memset(result, 0, sizeof(*result));
  const std::string key = tune_key(ctx, g, cams, n_views);
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string k;
      ocgs_options o{};
      double ms = 0.0;
      if ((ls >> k >> o.tile_w >> o.tile_h >> o.pixels_per_thread >> o.persistent >> o.front_fraction >> o.batch >>
           ms) &&
          k == key && ocgs_set_options(ctx, &o) == OCGS_OK) {
        result->best = ctx->opts;
        result->best_ms = ms;
        result->from_cache = 1;
      }
    }
    if (result->from_cache) return OCGS_OK;
  }
  // buffers for the timed passes: the images, a contribution score and the
  // colour and opacity cotangents of a training step (dL/dC = dL/dA = 1)
  int64_t P = 0;
  for (int v = 0; v < n_views; ++v) P += (int64_t)cams[v].width * cams[v].height;
  const int64_t N = g->n;
  const int64_t K3 = 3 * (int64_t)(g->sh_degree + 1) * (g->sh_degree + 1);
  cudaStream_t s = ctx->stream;
  Arena tmp(ctx);
  float *img, *ones, *grad, *score;
  CK(tmp.alloc(&img, (size_t)P * 8));
  CK(tmp.alloc(&ones, (size_t)P * 4));
  CK(tmp.alloc(&grad, (size_t)N * (10 + K3)));
  CK(tmp.alloc(&score, (size_t)std::max<int64_t>(N, 1)));
  std::vector<float> h_ones(1 << 16, 1.0f);
  for (int64_t off = 0; off < 4 * P; off += (int64_t)h_ones.size()) {
    const int64_t n = std::min<int64_t>((int64_t)h_ones.size(), 4 * P - off);
    CK(cudaMemcpyAsync(ones + off, h_ones.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s));
  }
  const ocgs_image out{img, img + 3 * P, img + 4 * P, img + 5 * P, nullptr};
  const ocgs_image d_out{ones, ones + 3 * P, nullptr, nullptr, nullptr};
  const ocgs_gaussians_out dp{grad, grad + 3 * N, grad + 7 * N, grad + 9 * N, grad + 10 * N};
  const ocgs_options saved = ctx->opts;
  const bool prof = ctx->prof;
  ctx->prof = false;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  ocgs_status status = OCGS_OK;
  // ms of one render + backward with options o (once untimed, twice timed), or < 0.  A
  // candidate whose pair count exceeds the capacity of one render (small tiles in one pass)
  // is infeasible for this workload and skipped.
  auto time_options = [&](const ocgs_options& o) -> double {
    if (status != OCGS_OK || ocgs_set_options(ctx, &o) != OCGS_OK) return -1.0;
    for (int rep = 0; rep < 3 && status == OCGS_OK; ++rep) {
      if (rep == 1) cudaEventRecord(e0, s);
      ocgs_fwd_state* st = nullptr;
      status = ocgs_render(ctx, g, cams, n_views, &out, score, &st);
      if (status == OCGS_ERR_NONFINITE) status = OCGS_OK;
      if (status == OCGS_OK) status = ocgs_render_backward(ctx, st, g, &d_out, &dp);
      if (st) ocgs_state_release(ctx, st);
    }
    if (status == OCGS_ERR_CAPACITY) {
      status = OCGS_OK;
      return -1.0;
    }
    if (status != OCGS_OK) return -1.0;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    result->n_tried++;
    return ms / 2.0;
  };
  double best = 1e30;
  ocgs_options best_opts = saved;
  auto consider = [&](const ocgs_options& o) {
    const double ms = time_options(o);
    if (ms >= 0.0 && ms < best) {
      best = ms;
      best_opts = ctx->opts;
    }
  };
  // 1. tile shape, pixels per thread and persistence at the context's split and 32 per batch
  const int shapes[][3] = {{16, 16, 4}, {16, 16, 2}, {16, 8, 4}, {16, 8, 2}, {8, 8, 2}, {32, 8, 2}, {16, 16, 1}};
  for (const auto& sh : shapes)
    for (int pers = 0; pers <= 1; ++pers) consider(ocgs_options{sh[0], sh[1], pers, sh[2], saved.front_fraction, 32});
  // 2. the two-pass split, for a persistent choice (the only renders that use it)
  if (status == OCGS_OK && best_opts.persistent) {
    const ocgs_options base = best_opts;
    for (float f : {0.0f, 0.05f, 0.1f, 0.2f})
      if (f != base.front_fraction) consider(ocgs_options{base.tile_w, base.tile_h, 1, base.pixels_per_thread, f, 32});
  }
  // 3. Gaussians per batch, where the chosen shape offers more than 32
  if (status == OCGS_OK) {
    const ocgs_options base = best_opts;
    for (int b : {16, 64})
      if (valid_tile(base.tile_w, base.tile_h, base.pixels_per_thread, b))
        consider(ocgs_options{base.tile_w, base.tile_h, base.persistent, base.pixels_per_thread, base.front_fraction, b});
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->prof = prof;
  if (status != OCGS_OK) {
    ctx->opts = saved;
    return status;
  }
  ctx->opts = best_opts;
  result->best = best_opts;
  result->best_ms = best;
  if (cache_path) {
    std::ofstream outf(cache_path, std::ios::app);
    outf << key << " " << best_opts.tile_w << " " << best_opts.tile_h << " " << best_opts.pixels_per_thread << " "
         << best_opts.persistent << " " << best_opts.front_fraction << " " << best_opts.batch << " " << best << "\n";
  }
  return OCGS_OK;
}

// ----------------------------------------------------------------------------- captured pruning sweep
struct ocgs_graph {
  ocgs_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> allocs;
  int64_t n_kernels = 0;
};

extern "C" ocgs_status ocgs_contribution_graph_create(ocgs_ctx* ctx, const ocgs_gaussians* g,
                                                      const ocgs_camera* cams, int32_t n_views, float* score,
                                                      float headroom, ocgs_graph** out) {
  if (!ctx || !out) return OCGS_ERR_ARG;
  *out = nullptr;
  ocgs_status r = check_gaussians(ctx, g);
  if (r != OCGS_OK) return r;
  r = check_cameras(ctx, cams, n_views);
  if (r != OCGS_OK) return r;
  if (!score || g->n == 0) return set_err(ctx, OCGS_ERR_ARG, "score must be non-NULL and n > 0");
  if (!(headroom >= 1.f) || !std::isfinite(headroom)) return set_err(ctx, OCGS_ERR_ARG, "headroom must be >= 1");
  CK(cudaSetDevice(ctx->device));
  const int chunk = 16;
  const int tw = ctx->opts.tile_w, th = ctx->opts.tile_h;
  // measure the pair count of every chunk with the eager path
  uint64_t kmax = 0;
  int64_t tiles_max = 0;
  std::vector<CamPlan> plans;
  for (int v0 = 0; v0 < n_views; v0 += chunk) {
    const int nv = std::min(chunk, n_views - v0);
    ocgs_fwd_state st;
    r = forward_pass(ctx, g, cams + v0, nv, nullptr, nullptr, &st, false);
    if (r != OCGS_OK && r != OCGS_ERR_NONFINITE) return r;
    kmax = std::max<uint64_t>(kmax, (uint64_t)ctx->stats.n_pairs);
    plans.push_back(plan_cameras(cams + v0, nv, tw, th, ctx->cover_rect));
    tiles_max = std::max<int64_t>(tiles_max, plans.back().tiles);
  }
  const double capd = (double)kmax * (double)headroom + 4096.0;
  if (capd > (double)INT32_MAX) return set_err(ctx, OCGS_ERR_CAPACITY, "pair capacity above 2^31-1");
  const uint32_t cap = (uint32_t)capd;
  ocgs_graph* gr = new ocgs_graph();
  gr->ctx = ctx;
  Arena a(ctx);
  SweepWs w;
  cudaError_t e = alloc_sweep_ws(a, w, (uint32_t)(g->n * std::min(chunk, n_views)), tiles_max, cap);
  std::vector<DevCam*> dc(plans.size());
  std::vector<int*> dp(plans.size());
  for (size_t c = 0; c < plans.size() && e == cudaSuccess; ++c) {
    const int nv = (int)plans[c].cams.size();
    e = a.alloc(&dc[c], nv);
    if (e == cudaSuccess) e = a.alloc(&dp[c], nv + 1);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dc[c], plans[c].cams.data(), sizeof(DevCam) * nv, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dp[c], plans[c].tile_prefix.data(), sizeof(int) * (nv + 1), cudaMemcpyHostToDevice,
                          ctx->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    delete gr;
    return cuda_err(ctx, e, "graph workspace");
  }
  // capture on a private stream (the context stream may be the legacy default stream)
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const bool prof = ctx->prof;
  ctx->prof = false;
  const long long launches0 = g_kernel_launches.load();
  r = OCGS_OK;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(score, 0, sizeof(float) * g->n, cs);
    for (size_t c = 0; c < plans.size() && e == cudaSuccess && r == OCGS_OK; ++c)
      r = enqueue_sweep_chunk(ctx, g, (int)plans[c].cams.size(), dc[c], dp[c], plans[c].tiles, w, score, cs);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &gr->graph);
    if (e == cudaSuccess) e = e2;
  }
  ctx->prof = prof;
  gr->n_kernels = g_kernel_launches.load() - launches0;
  g_kernel_launches -= gr->n_kernels;  // counted when launched, not when captured
  cudaStreamDestroy(cs);
  if (e == cudaSuccess && r == OCGS_OK) e = cudaGraphInstantiate(&gr->exec, gr->graph, 0);
  if (e != cudaSuccess || r != OCGS_OK) {
    if (gr->graph) cudaGraphDestroy(gr->graph);
    delete gr;
    return r != OCGS_OK ? r : cuda_err(ctx, e, "graph capture");
  }
  a.release_to(gr->allocs);
  *out = gr;
  return OCGS_OK;
}

extern "C" ocgs_status ocgs_graph_launch(ocgs_ctx* ctx, ocgs_graph* gr) {
  if (!ctx || !gr || gr->ctx != ctx) return OCGS_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaGraphLaunch(gr->exec, ctx->stream));
  g_kernel_launches += gr->n_kernels;
  return OCGS_OK;
}

extern "C" ocgs_status ocgs_graph_destroy(ocgs_ctx* ctx, ocgs_graph* gr) {
  if (!ctx || !gr || gr->ctx != ctx) return OCGS_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  for (void* p : gr->allocs) cudaFreeAsync(p, ctx->stream);
  delete gr;
  return OCGS_OK;
}
