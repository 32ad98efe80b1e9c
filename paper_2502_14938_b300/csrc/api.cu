// Host side of the C ABI (include/gsc.h, include/gsc_debug.h): context,
// model upload, cameras, the per-frame launch sequence (replayed as a CUDA
// graph), capacity growth and the debug read-backs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gsc.h"
#include "gsc_debug.h"
#include "gsc_internal.cuh"

using namespace gsc;

namespace {

constexpr int NSLOT = 4;  // pinned FrameIn ring

// NVTX range over a scope (a no-op unless a profiler attaches a tool); the
// frame's stages are named "gsc.<stage>" so a profiler can select their
// kernels (eager launches) or the launches that record them (graph capture).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct ModelHost {
  uint32_t n = 0;
  DevBuf px, py, pz, level, lod_r, feat, offs, scale, w32, feat_bf16, w_tc, feat_fp8, w_tc8;
  ModelDev dev{};
};

struct Counters {  // tail of FrameDev read back after a frame
  uint32_t vis_count[MAXV];
  uint32_t item_base[MAXV + 1];
  uint32_t rec_base[MAXV + 1];
  uint32_t n_items, n_records;
  uint32_t n_valid, n_pairs, n_pairs_used, err;
  uint32_t n_records_need;
  uint32_t n_big;
  uint32_t n_derived;
  uint32_t cache_depth;
};

}  // namespace

struct gsc_ctx {
  gsc_config cfg{};
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t ev_slot[NSLOT] = {};
  cudaEvent_t ev_stage[9] = {};
  int device = 0, n_sm = 148;
  std::string err;
  std::vector<ModelHost> models;
  ModelDev* d_models = nullptr;
  std::vector<gsc_camera> cams;
  bool cams_set = false;
  FrameIn* h_fin[NSLOT] = {};
  int slot = 0;
  FrameIn* d_fin = nullptr;
  FrameDev* d_fd = nullptr;
  Counters* h_cnt = nullptr;
  bool pending = false;  // an asynchronous frame whose counters were not checked yet
  // buffers
  uint32_t vis_cap = 0, n_vis_slots = 0;
  uint32_t* d_vis_buf = nullptr;
  uint32_t** d_vis_tab = nullptr;
  uint8_t* d_eye_buf = nullptr;   // exact stereo views: eye mask per visible anchor (same slots)
  uint8_t** d_eye_tab = nullptr;
  float* d_dbg_buf = nullptr;
  float** d_dbg_tab = nullptr;
  uint32_t rec_cap = 0;
  Records rec{};
  uint32_t *s1k0 = nullptr, *s1v0 = nullptr, *s1k1 = nullptr, *s1v1 = nullptr, *offs = nullptr, *big = nullptr;
  uint32_t *s1k2 = nullptr, *s1v2 = nullptr;  // the depth sort's result
  float4* attrs = nullptr;  // derived attributes, 3 float4 per Gaussian in frame item order
  float* unfused = nullptr;  // GSC_FLAG_UNFUSED: the operators' intermediate tensors
  size_t unfused_items = 0;
  uint32_t pair_cap = 0;
  uint32_t *pk0 = nullptr, *pv0 = nullptr, *pk1 = nullptr, *pv1 = nullptr;
  uint32_t ranges_cap = 0;
  uint2* ranges = nullptr;
  SortBufs sb{};
  uint32_t status_tiles = 0;  // sort look-back tiles allocated
  uint32_t scan_tiles = 0;    // scan look-back words allocated
  uint32_t* cull_masks = nullptr;  // the cull's keep masks [views][mask words] and tile counts [views][tiles]
  uint32_t* cull_cnt = nullptr;
  uint32_t cull_mask_stride = 0, cull_cnt_stride = 0, cull_views = 0;
  unsigned long long* st_scan = nullptr;
  // results of the last frame's sequence
  uint32_t* order_out = nullptr;  // records in depth order
  uint32_t* pkeys_out = nullptr;
  uint32_t* pvals_out = nullptr;
  // host-output images
  float* d_T[MAXV] = {};
  size_t d_T_bytes[MAXV] = {};
  // graph
  cudaGraphExec_t gexec = nullptr;
  bool graph_valid = false;
  bool replay_next = false;  // next enqueue re-renders a cached frame without new cache decisions
  // frame shape (host-known)
  uint32_t total_tiles = 0, tile_bits = 1;
  std::vector<int> models_used;
  uint32_t spin_limit = 1u << 20;
  bool timing = false;
  // caches of derived Gaussians, one per derivation view (Sec. 4)
  int n_caches = 0;
  CacheDev h_caches[MAX_CACHES] = {};
  uint32_t cache_na[MAX_CACHES] = {};  // anchors of each cache's model
  CacheDev* d_caches = nullptr;
  // reuse predictor: float32 master weights and their bfloat16 rounding
  float* rw_theta = nullptr;
  float* rw_w = nullptr;
  bool reuse_set = false;
  float4* attrs_fresh = nullptr;  // collection: every visible anchor derived afresh
  // per-frame tables: decoder view set per model, projection table
  DViewSet* d_tabs = nullptr;
  ProjTab* d_ptab = nullptr;
  // pipelined host frames: two device image sets, a copy stream
  void* d_hbuf[2][MAXV] = {};
  size_t d_hbuf_bytes[2][MAXV] = {};
  cudaStream_t copy_stream = nullptr;
  // second branch of the frame graph: the plan and the frame tables run
  // beside the cache's scan and assignment (ev_fork / ev_join)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_rendered[2] = {}, ev_copied[2] = {};
  int hslot = 0;
  bool hpending[2] = {false, false};
  bool keep_err = false;  // the frame being enqueued is one nobody waits for (pipelined host / no stats)
  bool async_since_sync = false;  // frames without statistics were enqueued since the last synchronising call
};

namespace {

int fail(gsc_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(ctx, e_ == cudaErrorMemoryAllocation ? GSC_ERR_OOM : GSC_ERR_CUDA, \
                                       "%s: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

template <typename T>
int dalloc(gsc_ctx* ctx, T** p, size_t count) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) return GSC_OK;
  CK(cudaMalloc((void**)p, count * sizeof(T)));
  return GSC_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

int upload(gsc_ctx* ctx, DevBuf& b, const void* src, size_t bytes) {
  dfree(b.p);
  b.p = nullptr;
  b.bytes = bytes;
  if (bytes == 0) return GSC_OK;
  CK(cudaMalloc(&b.p, bytes));
  CK(cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice));
  return GSC_OK;
}

bool finite_all(const float* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

void invalidate_graph(gsc_ctx* ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
  ctx->graph_valid = false;
}

uint32_t models_max_n(const gsc_ctx* ctx) {
  uint32_t m = 0;
  for (const auto& mh : ctx->models) m = std::max(m, mh.n);
  return m;
}

int ensure_status(gsc_ctx* ctx) {
  // sort tiles hold 2048 or 4096 keys (256 or 512 digit words each); scan tiles
  // 1024 elements (the pair offsets run over records, a cache's scan over
  // its lines and the visible anchors, the standalone scan over up to the
  // pair capacity)
  const uint32_t lines = std::max<uint32_t>(ctx->cfg.cache_gaussians / K, 1u);
  const uint32_t need = std::max((ctx->rec_cap + 2047u) / 2048u, (ctx->pair_cap + 2047u) / 2048u) + 1u;
  const uint32_t need_scan = std::max({(ctx->rec_cap + 1023u) / 1024u, (ctx->pair_cap + 1023u) / 1024u,
                                       (ctx->vis_cap + lines + 1023u) / 1024u}) + 1u;
  if (need > ctx->status_tiles) {
    int r = dalloc(ctx, &ctx->sb.status, (size_t)need * 512);  // up to 512 digit words per tile
    if (r) return r;
    CK(cudaMemset(ctx->sb.status, 0, (size_t)need * 512 * sizeof(unsigned long long)));
    ctx->status_tiles = need;
  }
  if (need_scan > ctx->scan_tiles) {
    int r = dalloc(ctx, &ctx->st_scan, (size_t)need_scan);
    if (r) return r;
    CK(cudaMemset(ctx->st_scan, 0, (size_t)need_scan * sizeof(unsigned long long)));
    ctx->scan_tiles = need_scan;
  }
  const uint32_t mw = cull_mask_words(models_max_n(ctx)), ct = cull_tiles(models_max_n(ctx));
  const uint32_t views = std::max<uint32_t>(ctx->n_vis_slots, 1u);
  if (mw > ctx->cull_mask_stride || ct > ctx->cull_cnt_stride || views > ctx->cull_views) {
    const uint32_t mws = std::max(mw, ctx->cull_mask_stride), cts = std::max(ct, ctx->cull_cnt_stride);
    const uint32_t vs = std::max(views, ctx->cull_views);
    int r;
    if ((r = dalloc(ctx, &ctx->cull_masks, (size_t)mws * vs)) || (r = dalloc(ctx, &ctx->cull_cnt, (size_t)cts * vs)))
      return r;
    ctx->cull_mask_stride = mws;
    ctx->cull_cnt_stride = cts;
    ctx->cull_views = vs;
    invalidate_graph(ctx);
  }
  return GSC_OK;
}

int alloc_records(gsc_ctx* ctx, uint32_t cap) {
  int r;
  if ((r = dalloc(ctx, &ctx->rec.geo, cap)) || (r = dalloc(ctx, &ctx->rec.cop, cap)) ||
      (r = dalloc(ctx, &ctx->rec.col, cap)) || (r = dalloc(ctx, &ctx->rec.aux, cap)) ||
      (r = dalloc(ctx, &ctx->rec.key, cap)) ||
      (r = dalloc(ctx, &ctx->rec.cnt, cap)) || (r = dalloc(ctx, &ctx->s1k0, cap)) ||
      (r = dalloc(ctx, &ctx->s1v0, cap)) || (r = dalloc(ctx, &ctx->s1k1, cap)) ||
      (r = dalloc(ctx, &ctx->s1v1, cap)) || (r = dalloc(ctx, &ctx->s1k2, cap)) || (r = dalloc(ctx, &ctx->s1v2, cap)) ||
      (r = dalloc(ctx, &ctx->offs, cap)) || (r = dalloc(ctx, &ctx->big, cap)) ||
      (r = dalloc(ctx, &ctx->attrs, (size_t)cap * 3)))
    return r;
  if ((ctx->cfg.flags & GSC_FLAG_REUSE_COLLECT) && (r = dalloc(ctx, &ctx->attrs_fresh, (size_t)cap * 3))) return r;
  ctx->rec_cap = cap;
  invalidate_graph(ctx);
  return ensure_status(ctx);
}

int alloc_pairs(gsc_ctx* ctx, uint32_t cap) {
  int r;
  if ((r = dalloc(ctx, &ctx->pk0, cap)) || (r = dalloc(ctx, &ctx->pv0, cap)) || (r = dalloc(ctx, &ctx->pk1, cap)) ||
      (r = dalloc(ctx, &ctx->pv1, cap)))
    return r;
  ctx->pair_cap = cap;
  invalidate_graph(ctx);
  return ensure_status(ctx);
}

// Blend tilings: a lane owns 4 pixels of one column and a warp 32 / tile_w
// column strips; powers of two keep the coverage arithmetic exact.
bool tiling_ok(uint32_t tw, uint32_t th, uint32_t bps) {
  if (tw != 8 && tw != 16 && tw != 32) return false;
  if (th == 0 || (th & (th - 1)) != 0) return false;
  const uint32_t npx = tw * th;
  if (npx < 128 || npx > 1024 || th % ((32 / tw) * 4) != 0) return false;
  return bps <= 32;
}

// Tile count, tile-key bits and the range table for the current cameras and tiling.
int retile(gsc_ctx* ctx) {
  uint32_t tiles = 0;
  for (const auto& c : ctx->cams)
    tiles += ((c.width + ctx->cfg.tile_w - 1) / ctx->cfg.tile_w) * ((c.height + ctx->cfg.tile_h - 1) / ctx->cfg.tile_h);
  ctx->total_tiles = tiles;
  uint32_t bits = 1;
  while ((1u << bits) < tiles && bits < 31) ++bits;
  ctx->tile_bits = bits;
  if (tiles > ctx->ranges_cap) {
    int r = dalloc(ctx, &ctx->ranges, tiles);
    if (r) return r;
    ctx->ranges_cap = tiles;
  }
  invalidate_graph(ctx);
  return GSC_OK;
}

// ------------------------------------------------------------------ caches (Sec. 4)
void free_cache(CacheDev& c) {
  void* p[] = {c.slot_of, c.slot_anchor, c.slot_frame, c.slot_attr, c.vstat, c.flags, c.ranks,
               c.free_list, c.miss, c.state, c.slot_dir, c.cz, c.clab};
  for (void* q : p) dfree(q);
  c = CacheDev{};
}

// Empty cache: no anchor has a line, every line unused, t = 0, depth = D_max.
int init_cache(gsc_ctx* ctx, CacheDev& c, uint32_t n_anchors) {
  if (n_anchors) CK(cudaMemset(c.slot_of, 0xFF, (size_t)n_anchors * 4));
  CK(cudaMemset(c.slot_anchor, 0xFF, (size_t)c.S * 4));
  CK(cudaMemset(c.slot_frame, 0, (size_t)c.S * 4));
  uint32_t st[CS_WORDS] = {0};
  st[CS_DEPTH] = ctx->cfg.max_depth;
  st[CS_DMAX] = ctx->cfg.max_depth;
  st[CS_GUIDE] = ctx->cfg.depth_guide;
  st[CS_S] = c.S;
  CK(cudaMemcpy(c.state, st, sizeof st, cudaMemcpyHostToDevice));
  return GSC_OK;
}

// One cache per derivation view of the current cameras (the views are found
// as prepare_frame_cameras finds them: a stereo pair under stereo_unify is one view).
int setup_caches(gsc_ctx* ctx) {
  for (int i = 0; i < ctx->n_caches; ++i) free_cache(ctx->h_caches[i]);
  ctx->n_caches = 0;
  if (ctx->cfg.reuse == GSC_REUSE_OFF) return GSC_OK;
  const size_t n = ctx->cams.size();
  std::vector<int> dof(n, -1);
  std::vector<uint32_t> dv_model;
  for (size_t c = 0; c < n; ++c) {
    if (dof[c] >= 0) continue;
    const int p = ctx->cams[c].stereo_partner;
    const bool pair = ctx->cfg.stereo_unify && p > (int)c && p < (int)n && ctx->cams[p].stereo_partner == (int)c;
    dof[c] = (int)dv_model.size();
    if (pair) dof[p] = (int)dv_model.size();
    dv_model.push_back(ctx->cams[c].model_id);
  }
  if (dv_model.size() > (size_t)MAX_CACHES)
    return fail(ctx, GSC_ERR_INVALID_ARG, "at most %d derivation views with a cache", MAX_CACHES);
  const uint32_t S = std::max<uint32_t>(ctx->cfg.cache_gaussians / K, 1u);
  const uint32_t vcap = ctx->vis_cap;
  for (size_t d = 0; d < dv_model.size(); ++d) {
    CacheDev& c = ctx->h_caches[d];
    const uint32_t na = ctx->models[dv_model[d]].n;
    c.S = S;
    c.active = 1;
    int r;
    if ((r = dalloc(ctx, &c.slot_of, std::max(na, 1u))) || (r = dalloc(ctx, &c.slot_anchor, S)) ||
        (r = dalloc(ctx, &c.slot_frame, S)) || (r = dalloc(ctx, &c.slot_attr, (size_t)S * K * 3)) ||
        (r = dalloc(ctx, &c.vstat, vcap)) || (r = dalloc(ctx, &c.flags, (size_t)S + vcap)) ||
        (r = dalloc(ctx, &c.ranks, (size_t)S + vcap)) || (r = dalloc(ctx, &c.free_list, S)) ||
        (r = dalloc(ctx, &c.miss, vcap)) ||
        (r = dalloc(ctx, &c.state, CS_WORDS)) || (r = dalloc(ctx, &c.slot_dir, S)))
      return r;
    if ((ctx->cfg.flags & GSC_FLAG_REUSE_COLLECT) &&
        ((r = dalloc(ctx, &c.cz, (size_t)vcap * 36)) || (r = dalloc(ctx, &c.clab, vcap))))
      return r;
    if ((r = init_cache(ctx, c, na))) return r;
    ctx->cache_na[d] = na;
    ctx->n_caches = (int)d + 1;
  }
  if (!ctx->d_caches) CK(cudaMalloc((void**)&ctx->d_caches, sizeof(CacheDev) * MAX_CACHES));
  CK(cudaMemcpy(ctx->d_caches, ctx->h_caches, sizeof(CacheDev) * MAX_CACHES, cudaMemcpyHostToDevice));
  return GSC_OK;
}

// The launch sequence of one frame (everything after the FrameIn upload).
// replay: the frame is being rendered again after a buffer grew.  Its cache
// decisions (hit / line / miss lists, the next reuse depth) were taken and
// committed by the first attempt, and derivation rewrites the same lines
// with the same values, so the cache kernels are left out and the policy
// only restates the frame's counts.
void enqueue_sequence(gsc_ctx* ctx, bool replay = false) {
  cudaStream_t s = ctx->stream;
  FrameDev* fd = ctx->d_fd;
  const bool tm = ctx->timing;
  NvtxRange frame_range("gsc.frame");
  if (tm) cudaEventRecord(ctx->ev_stage[0], s);
  nvtxRangePushA("gsc.cull_cache");
  launch_frame_begin(fd, ctx->d_fin, replay ? nullptr : ctx->d_caches, replay ? 0 : ctx->n_caches, ctx->ranges,
                     ctx->total_tiles, s);
  CacheDev* caches = ctx->n_caches ? ctx->d_caches : nullptr;
  const bool learned = ctx->cfg.reuse == GSC_REUSE_LEARNED;
  // The cull's write pass probes the caches by the depth rule as it writes
  // the ids (with a model without anchors, whose cull launches nothing, the
  // probe kernel runs instead)
  bool fuse = !ctx->models_used.empty();
  for (int m : ctx->models_used) fuse = fuse && ctx->models[m].dev.n > 0;
  const bool probed = fuse && caches && !replay && !learned;
  CullProbe probe{probed ? caches : nullptr};
  for (int m : ctx->models_used)
    launch_cull(ctx->d_models, &ctx->models[m].dev, m, fd, ctx->d_vis_tab, ctx->d_eye_tab, ctx->cull_masks,
                ctx->cull_cnt, ctx->cull_mask_stride, ctx->cull_cnt_stride, probe, s);
  const bool collect = caches && (ctx->cfg.flags & GSC_FLAG_REUSE_COLLECT) && !replay;
  const bool tc = ctx->cfg.precision != GSC_PREC_FP32, fp8 = ctx->cfg.precision == GSC_PREC_FP8;
  if (probed && !collect) {
    // the cache decisions are taken: the plan and the frame tables (one warp
    // each) run on a second branch beside the scan and assignment of the
    // free lines, which they do not read (the plan adds to n_derived, the
    // assignment subtracts the hits from it)
    cudaEventRecord(ctx->ev_fork, s);
    cudaStreamWaitEvent(ctx->aux_stream, ctx->ev_fork, 0);
    launch_plan(fd, ctx->rec_cap, ctx->aux_stream);
    launch_tables(fd, caches, ctx->d_eye_tab, ctx->d_tabs, ctx->d_ptab, (int)ctx->models.size(), ctx->aux_stream);
    cudaEventRecord(ctx->ev_join, ctx->aux_stream);
    launch_cache_frame(ctx->d_caches, ctx->h_caches, ctx->n_caches, fd, ctx->d_vis_tab, ctx->d_models, ctx->rw_w,
                       learned, nullptr, ctx->st_scan, ctx->n_sm, s, probed);
    cudaStreamWaitEvent(s, ctx->ev_join, 0);
  } else {
    launch_plan(fd, ctx->rec_cap, s);
    if (collect)  // fresh attributes of every visible anchor, for the labels
      for (int m : ctx->models_used)
        if (tc)
          launch_derive_tc(ctx->d_models, m, fd, ctx->d_vis_tab, ctx->attrs_fresh, nullptr, nullptr, nullptr,
                           fp8, ctx->n_sm, s);
        else
          launch_derive_f32(ctx->d_models, m, fd, ctx->d_vis_tab, ctx->attrs_fresh, nullptr, nullptr, nullptr,
                            ctx->n_sm, s);
    if (caches && !replay)
      launch_cache_frame(ctx->d_caches, ctx->h_caches, ctx->n_caches, fd, ctx->d_vis_tab, ctx->d_models, ctx->rw_w,
                         learned, collect ? ctx->attrs_fresh : nullptr, ctx->st_scan, ctx->n_sm, s, probed);
    launch_tables(fd, caches, ctx->d_eye_tab, ctx->d_tabs, ctx->d_ptab, (int)ctx->models.size(), s);
  }
  if (tm) cudaEventRecord(ctx->ev_stage[1], s);
  nvtxRangePop();
  nvtxRangePushA("gsc.derive_project");
  for (int m : ctx->models_used)
    if (tc)
      launch_derive_tc(ctx->d_models, m, fd, ctx->d_vis_tab, ctx->attrs, ctx->d_dbg_tab, caches, ctx->d_tabs,
                       fp8, ctx->n_sm, s);
    else if (ctx->cfg.flags & GSC_FLAG_UNFUSED)
      launch_derive_unfused(ctx->d_models, &ctx->models[m].dev, m, fd, ctx->d_vis_tab, ctx->attrs, ctx->d_dbg_tab,
                            ctx->d_tabs, ctx->unfused, ctx->unfused_items, ctx->n_sm, s);
    else
      launch_derive_f32(ctx->d_models, m, fd, ctx->d_vis_tab, ctx->attrs, ctx->d_dbg_tab, caches, ctx->d_tabs,
                        ctx->n_sm, s);
  launch_project(ctx->d_models, fd, ctx->d_vis_tab, ctx->attrs, caches, ctx->rec, ctx->d_ptab, ctx->n_sm, s);
  if (caches && replay) launch_cache_replay_counts(ctx->d_caches, ctx->n_caches, fd, s);
  if (tm) cudaEventRecord(ctx->ev_stage[2], s);
  nvtxRangePop();
  nvtxRangePushA("gsc.sort_keygen");
  launch_depth_sort(ctx->rec.key, ctx->s1k0, ctx->s1v0, ctx->s1k1, ctx->s1v1, ctx->s1k2, ctx->s1v2, &fd->n_records,
                    &fd->n_valid, SLOT_SORT1, fd, ctx->sb, fd->hist_depth, ctx->n_sm, s);
  const uint32_t* ov = ctx->s1v2;
  ctx->order_out = ctx->s1v2;
  if (tm) cudaEventRecord(ctx->ev_stage[3], s);
  launch_scan_u32(ctx->rec.cnt, ov, &fd->n_valid, ctx->offs, &fd->n_pairs, ctx->st_scan, fd, SLOT_SCAN, ctx->n_sm, s,
                  nullptr, 0, ctx->big, &fd->n_big, KG_SMALL);
  launch_keygen(fd, ctx->rec, ov, ctx->offs, ctx->pk0, ctx->pv0, ctx->pair_cap, ctx->big, ctx->n_sm, s);
  if (tm) cudaEventRecord(ctx->ev_stage[4], s);
  uint32_t *pk = nullptr, *pv = nullptr;
  launch_sort_impl(ctx->pk0, ctx->pv0, ctx->pk1, ctx->pv1, ctx->pk0, ctx->pv0, &fd->n_pairs_used, nullptr,
                   (int)ctx->tile_bits, 0, SLOT_SORT2, fd, ctx->sb, ctx->n_sm, s, &pk, &pv, 16,
                   fd->hist_tile);
  ctx->pkeys_out = pk;
  ctx->pvals_out = pv;
  if (tm) cudaEventRecord(ctx->ev_stage[5], s);
  launch_ranges(fd, pk, ctx->ranges, ctx->n_sm, s);
  if (tm) cudaEventRecord(ctx->ev_stage[6], s);
  nvtxRangePop();
  nvtxRangePushA("gsc.blend");
  launch_blend(fd, ctx->ranges, pv, ctx->rec, ctx->d_fin, ctx->total_tiles, ctx->cfg.tile_w * ctx->cfg.tile_h,
               ctx->cfg.blocks_per_sm, (ctx->cfg.flags & GSC_FLAG_BLEND_WORK) != 0, ctx->n_sm, s);
  if (tm) cudaEventRecord(ctx->ev_stage[7], s);
  nvtxRangePop();
}

int build_graph(gsc_ctx* ctx) {
  invalidate_graph(ctx);
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  enqueue_sequence(ctx);
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  if (e != cudaSuccess) return fail(ctx, GSC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&ctx->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, GSC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  ctx->graph_valid = true;
  return GSC_OK;
}

// ------------------------------------------------------------------ cameras (host, float64)
// Camera constants and the unified camera of each stereo pair (Eq. 5-6) are
// scalar float64 work per frame, done here rather than on the GPU, whose
// float64 rate would put a long dependency chain at the head of every frame.
// Every operation is written out in a fixed order and this file is compiled
// without floating-point contraction, so the results are those of the same
// sequence of IEEE double operations anywhere.

// Camera centre p = -R^T t.
void center64(const float* R, const float* t, double* p) {
  for (int i = 0; i < 3; ++i) {
    double s = (double)R[i] * (double)t[0];
    s = s + (double)R[3 + i] * (double)t[1];
    s = s + (double)R[6 + i] * (double)t[2];
    p[i] = -s;
  }
}

struct HostCam {
  float R[9], t[3];
  float fx, fy, cx, cy, znear;
  int W, H, model;
};

HostCam host_cam(const gsc_camera& c) {
  HostCam h;
  std::memcpy(h.R, c.R, sizeof h.R);
  std::memcpy(h.t, c.t, sizeof h.t);
  h.fx = c.fx; h.fy = c.fy; h.cx = c.cx; h.cy = c.cy; h.znear = c.znear;
  h.W = (int)c.width; h.H = (int)c.height; h.model = (int)c.model_id;
  return h;
}

// Derived constants: double-float centre (pc, pc_lo), dt = t + R pc (what
// R (x - pc) misses of R x + t when the float32 R is not exactly
// orthonormal), guard-band tangents 1.3 (W/2)/fx and 1.3 (H/2)/fy in
// float32, tile counts.
void fill_camdev(CamDev& c, const HostCam& in, uint32_t tile_w, uint32_t tile_h) {
  std::memset(&c, 0, sizeof c);
  for (int i = 0; i < 9; ++i) c.R[i] = in.R[i];
  for (int i = 0; i < 3; ++i) c.t[i] = in.t[i];
  c.fx = in.fx; c.fy = in.fy; c.cx = in.cx; c.cy = in.cy;
  c.W = in.W; c.H = in.H; c.znear = in.znear;
  c.model = in.model;
  double p[3];
  center64(c.R, c.t, p);
  for (int i = 0; i < 3; ++i) {
    c.pc[i] = (float)p[i];
    c.pc_lo[i] = (float)(p[i] - (double)c.pc[i]);
  }
  for (int i = 0; i < 3; ++i) {
    double s = (double)c.t[i];
    for (int k = 0; k < 3; ++k) s = s + (double)c.R[3 * i + k] * p[k];
    c.dt[i] = (float)s;
  }
  const float half_w = 0.5f * (float)c.W, half_h = 0.5f * (float)c.H;
  c.gx = 1.3f * (half_w / c.fx);
  c.gy = 1.3f * (half_h / c.fy);
  c.ntx = (c.W + (int)tile_w - 1) / (int)tile_w;
  c.nty = (c.H + (int)tile_h - 1) / (int)tile_h;
}

// Unified camera of a stereo pair (Eq. 5-6): d_u = normalised mean forward
// axis; p_u = mean centre - d_u |p1 - p2| / (2 tan(theta/2)) with
// 2 tan(theta/2) = W / fx (horizontal field of view); right/down axes from
// the mean down axis orthogonalised against d_u; rounded once to float32.
HostCam unified_camera(const HostCam& L, const HostCam& Rr) {
  double p1[3], p2[3];
  center64(L.R, L.t, p1);
  center64(Rr.R, Rr.t, p2);
  double d[3], y[3], pm[3];
  for (int i = 0; i < 3; ++i) {
    d[i] = ((double)L.R[6 + i] + (double)Rr.R[6 + i]) * 0.5;
    y[i] = ((double)L.R[3 + i] + (double)Rr.R[3 + i]) * 0.5;
    pm[i] = (p1[i] + p2[i]) * 0.5;
  }
  const double dn = std::sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
  double du[3];
  for (int i = 0; i < 3; ++i) du[i] = d[i] / dn;
  const double bx = p1[0] - p2[0], by = p1[1] - p2[1], bz = p1[2] - p2[2];
  const double b = std::sqrt((bx * bx + by * by) + bz * bz);
  const double back = (b * (double)L.fx) / (double)L.W;
  double pu[3];
  for (int i = 0; i < 3; ++i) pu[i] = pm[i] - du[i] * back;
  const double xr[3] = {y[1] * du[2] - y[2] * du[1], y[2] * du[0] - y[0] * du[2], y[0] * du[1] - y[1] * du[0]};
  const double xn = std::sqrt((xr[0] * xr[0] + xr[1] * xr[1]) + xr[2] * xr[2]);
  double xu[3];
  for (int i = 0; i < 3; ++i) xu[i] = xr[i] / xn;
  const double yu[3] = {du[1] * xu[2] - du[2] * xu[1], du[2] * xu[0] - du[0] * xu[2], du[0] * xu[1] - du[1] * xu[0]};
  const double Ru[9] = {xu[0], xu[1], xu[2], yu[0], yu[1], yu[2], du[0], du[1], du[2]};
  HostCam U = L;
  for (int i = 0; i < 9; ++i) U.R[i] = (float)Ru[i];
  for (int r = 0; r < 3; ++r) {
    double s = Ru[r * 3 + 0] * pu[0];
    s = s + Ru[r * 3 + 1] * pu[1];
    s = s + Ru[r * 3 + 2] * pu[2];
    U.t[r] = (float)(-s);
  }
  return U;
}

// Cameras, tile bases and derivation views of the current frame into F.
void prepare_frame_cameras(const gsc_ctx* ctx, FrameIn& F) {
  const uint32_t nc = (uint32_t)ctx->cams.size();
  const uint32_t tw = ctx->cfg.tile_w, th = ctx->cfg.tile_h;
  F.n_cams = nc;
  uint32_t tb = 0;
  for (uint32_t c = 0; c < nc; ++c) {
    fill_camdev(F.cam[c], host_cam(ctx->cams[c]), tw, th);
    F.cam[c].tile_base = tb;
    tb += (uint32_t)(F.cam[c].ntx * F.cam[c].nty);
  }
  F.total_tiles = tb;
  uint32_t bits = 1;
  while ((1u << bits) < tb && bits < 31) ++bits;
  F.tile_bits = bits;
  // the depth sort's base: bits of the smallest near plane (positive floats
  // order as their bits, and every valid depth exceeds its camera's plane)
  float zmin = nc ? F.cam[0].znear : 1.f;
  for (uint32_t c = 1; c < nc; ++c) zmin = std::min(zmin, F.cam[c].znear);
  std::memcpy(&F.depth_base, &zmin, 4);
  uint32_t nd = 0;
  for (uint32_t c = 0; c < nc; ++c) F.dview_of_cam[c] = -1;
  for (uint32_t c = 0; c < nc; ++c) {
    if (F.dview_of_cam[c] >= 0) continue;
    const int p = ctx->cams[c].stereo_partner;
    const bool pair = ctx->cfg.stereo_unify && p > (int)c && p < (int)nc && ctx->cams[p].stereo_partner == (int)c;
    if (pair) {
      fill_camdev(F.dcam[nd], unified_camera(host_cam(ctx->cams[c]), host_cam(ctx->cams[p])), tw, th);
      F.dcam[nd].tile_base = F.cam[c].tile_base;
      F.dview_of_cam[p] = (int)nd;
    } else {
      F.dcam[nd] = F.cam[c];
    }
    F.dview_cam[nd][0] = (int)c;
    F.dview_cam[nd][1] = pair ? p : -1;
    F.dview_exact[nd] = pair && ctx->cfg.stereo_unify == GSC_STEREO_EXACT ? 1 : 0;
    F.dview_of_cam[c] = (int)nd;
    ++nd;
  }
  F.n_dviews = nd;
}

// Upload the frame description into the next pinned slot and enqueue the
// frame.  out_rgb / out_T are device pointers per camera.
int enqueue_frame(gsc_ctx* ctx, void* const* out_rgb, float* const* out_T) {
  const int sl = ctx->slot;
  ctx->slot = (ctx->slot + 1) % NSLOT;
  CK(cudaEventSynchronize(ctx->ev_slot[sl]));
  FrameIn* F = ctx->h_fin[sl];
  std::memset(F, 0, sizeof(FrameIn));
  prepare_frame_cameras(ctx, *F);
  F->tile_w = ctx->cfg.tile_w;
  F->tile_h = ctx->cfg.tile_h;
  F->out_format = ctx->cfg.out_format;
  F->keep_err = ctx->keep_err ? 1u : 0u;
  F->cap_vis = ctx->vis_cap;
  F->cap_rec = ctx->rec_cap;
  F->cap_pairs = ctx->pair_cap;
  F->spin_limit = ctx->spin_limit;
  for (int i = 0; i < 3; ++i) F->bg[i] = ctx->cfg.bg[i];
  for (size_t i = 0; i < ctx->cams.size(); ++i) {
    F->out_rgb[i] = (unsigned long long)(uintptr_t)out_rgb[i];
    F->out_T[i] = (unsigned long long)(uintptr_t)(out_T ? out_T[i] : nullptr);
  }
  CK(cudaEventRecord(ctx->ev_in, ctx->user_stream));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
  CK(cudaMemcpyAsync(ctx->d_fin, F, sizeof(FrameIn), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaEventRecord(ctx->ev_slot[sl], ctx->stream));
  if (ctx->replay_next) {
    ctx->replay_next = false;
    enqueue_sequence(ctx, true);
    CK(cudaGetLastError());
  } else if (ctx->cfg.use_graph && !ctx->timing) {
    if (!ctx->graph_valid) {
      int r = build_graph(ctx);
      if (r) return r;
    }
    CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
  } else {
    enqueue_sequence(ctx);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(ctx->h_cnt, &ctx->d_fd->vis_count[0], sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaEventRecord(ctx->ev_out, ctx->stream));
  CK(cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0));
  ctx->pending = true;
  return GSC_OK;
}

// Wait for the last frame and turn its counters into a status.  Grows a
// buffer that overflowed (returns GSC_ERR_CAPACITY so the caller re-renders).
int finish_frame(gsc_ctx* ctx) {
  CK(cudaEventSynchronize(ctx->ev_out));
  ctx->pending = false;
  const Counters& c = *ctx->h_cnt;
  if (c.err & ERR_TIMEOUT) return fail(ctx, GSC_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (c.err & ERR_BOUNDS) return fail(ctx, GSC_ERR_INTERNAL, "a bounds-checked store was out of range");
  if (c.err & ERR_REC_OVERFLOW) {
    // grow to the frame's requirement plus headroom, at most the worst case
    unsigned long long worst = 0;
    for (const auto& cam : ctx->cams) worst += (unsigned long long)K * ctx->models[cam.model_id].n;
    unsigned long long need = (unsigned long long)c.n_records_need + c.n_records_need / 2 + 1024;
    need = std::min<unsigned long long>(std::min(need, worst), 0x3FFFFFFFull);
    int r = alloc_records(ctx, (uint32_t)need);
    if (r) return r;
    return fail(ctx, GSC_ERR_CAPACITY, "record buffer grown to %u", ctx->rec_cap);
  }
  if (c.err & ERR_PAIR_OVERFLOW) {
    unsigned long long need = (unsigned long long)c.n_pairs + c.n_pairs / 4 + 1024;
    need = std::min<unsigned long long>(need, 0x3FFFFFFFull);
    int r = alloc_pairs(ctx, (uint32_t)need);
    if (r) return r;
    return fail(ctx, GSC_ERR_CAPACITY, "pair buffer grown to %u", ctx->pair_cap);
  }
  return GSC_OK;
}

void fill_stats(gsc_ctx* ctx, gsc_frame_stats* st) {
  const Counters& c = *ctx->h_cnt;
  std::memset(st, 0, sizeof(*st));
  uint64_t vis = 0;
  for (uint32_t d = 0; d < MAXV; ++d) vis += c.vis_count[d];
  st->visible_anchors = vis;
  st->derived_anchors = c.n_derived;
  st->records = c.n_records;
  st->valid_records = c.n_valid;
  st->pairs = c.n_pairs;
  st->cache_depth = ctx->n_caches ? c.cache_depth : 0;
  st->error_flags = c.err;
  if (ctx->timing) {
    float tot = 0.f;
    for (int i = 0; i < 7; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ctx->ev_stage[i], ctx->ev_stage[i + 1]);
      st->ms_stage[i] = ms;
      tot += ms;
    }
    st->ms_stage[7] = tot;
  }
}

// Errors of frames nobody waited for (pipelined host frames, frames without
// statistics): a timeout, or an overflow, after which the buffers are grown
// to what those frames asked for; their images are invalid.
int take_sticky_error(gsc_ctx* ctx) {
  uint32_t e[3] = {0, 0, 0};  // err_sticky, need_sticky[0..1]
  static_assert(offsetof(FrameDev, need_sticky) == offsetof(FrameDev, err_sticky) + 4, "sticky words");
  CK(cudaMemcpy(e, &ctx->d_fd->err_sticky, sizeof e, cudaMemcpyDeviceToHost));
  if (!e[0]) return GSC_OK;
  CK(cudaMemset(&ctx->d_fd->err_sticky, 0, sizeof e));
  if (e[0] & ERR_TIMEOUT) return fail(ctx, GSC_ERR_TIMEOUT, "a bounded device-side wait gave up in an unwaited frame");
  if (e[0] & ERR_REC_OVERFLOW) {
    unsigned long long worst = 0;
    for (const auto& cam : ctx->cams) worst += (unsigned long long)K * ctx->models[cam.model_id].n;
    unsigned long long need = (unsigned long long)e[1] + e[1] / 2 + 1024;
    need = std::min<unsigned long long>(std::min(need, worst), 0x3FFFFFFFull);
    if (need > ctx->rec_cap) {
      int r = alloc_records(ctx, (uint32_t)need);
      if (r) return r;
    }
  }
  if (e[0] & ERR_PAIR_OVERFLOW) {
    unsigned long long need = (unsigned long long)e[2] + e[2] / 4 + 1024;
    need = std::min<unsigned long long>(need, 0x3FFFFFFFull);
    if (need > ctx->pair_cap) {
      int r = alloc_pairs(ctx, (uint32_t)need);
      if (r) return r;
    }
  }
  return fail(ctx, GSC_ERR_CAPACITY, "an unwaited frame overflowed a buffer (its images are invalid); buffers grown "
                                     "to %u records, %u pairs", ctx->rec_cap, ctx->pair_cap);
}

int render_impl(gsc_ctx* ctx, void* const* out_dev, float* const* out_T, gsc_frame_stats* stats, bool sync) {
  if (!ctx->cams_set) return fail(ctx, GSC_ERR_STATE, "gsc_set_cameras must come first");
  if (ctx->cfg.reuse == GSC_REUSE_LEARNED && !ctx->reuse_set)
    return fail(ctx, GSC_ERR_STATE, "the learned reuse form needs predictor weights (gsc_reuse_set_weights)");
  if (sync && (ctx->pending || ctx->async_since_sync)) {
    // report the problems of earlier frames rendered without statistics
    // (each kept its error bits on the device) before starting this one
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->pending = false;
    ctx->async_since_sync = false;
    int r = take_sticky_error(ctx);
    if (r) return r;
  }
  for (int attempt = 0; attempt < 4; ++attempt) {
    ctx->keep_err = !sync;
    int r = enqueue_frame(ctx, out_dev, out_T);
    ctx->keep_err = false;
    if (r) return r;
    if (!sync) {
      ctx->async_since_sync = true;
      return GSC_OK;
    }
    r = finish_frame(ctx);
    if (r == GSC_ERR_CAPACITY) {  // grown: render the frame again
      ctx->replay_next = ctx->n_caches > 0;
      continue;
    }
    if (r) return r;
    if (stats) fill_stats(ctx, stats);
    ctx->err.clear();
    return GSC_OK;
  }
  return fail(ctx, GSC_ERR_CAPACITY, "capacity still insufficient after growth");
}

}  // namespace

extern "C" {

void gsc_default_config(gsc_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->max_views = 2;
  cfg->precision = GSC_PREC_FP32;
  cfg->reuse = GSC_REUSE_OFF;
  cfg->stereo_unify = 0;
  cfg->cache_gaussians = 4u << 20;
  cfg->max_depth = 10;
  cfg->tile_w = 16;
  cfg->tile_h = 16;
  cfg->pair_capacity = 16u << 20;
  cfg->use_graph = 1;
}

int gsc_version(void) { return GSC_VERSION; }

int gsc_create(gsc_ctx** out, const gsc_config* cfg_in, void* cuda_stream) {
  if (!out) return GSC_ERR_INVALID_ARG;
  *out = nullptr;
  gsc_config cfg;
  if (cfg_in) cfg = *cfg_in; else gsc_default_config(&cfg);
  if (cfg.tile_w == 0) cfg.tile_w = 16;
  if (cfg.tile_h == 0) cfg.tile_h = 16;
  if (cfg.max_depth == 0) cfg.max_depth = 10;
  if (cfg.cache_gaussians == 0) cfg.cache_gaussians = 4u << 20;
  if (cfg.pair_capacity == 0) cfg.pair_capacity = 16u << 20;
  if (cfg.max_views == 0 || cfg.max_views > GSC_MAX_VIEWS) return GSC_ERR_INVALID_ARG;
  if (!tiling_ok(cfg.tile_w, cfg.tile_h, cfg.blocks_per_sm)) return GSC_ERR_INVALID_ARG;
  if (cfg.out_format > GSC_OUT_RGBA8) return GSC_ERR_INVALID_ARG;
  if (cfg.depth_guide > GSC_GUIDE_STAGED) return GSC_ERR_INVALID_ARG;
  if (cfg.precision > GSC_PREC_FP8 || cfg.reuse > GSC_REUSE_LEARNED) return GSC_ERR_INVALID_ARG;
  if ((cfg.flags & GSC_FLAG_UNFUSED) && cfg.precision != GSC_PREC_FP32) return GSC_ERR_INVALID_ARG;
  if (cfg.stereo_unify > GSC_STEREO_EXACT) return GSC_ERR_INVALID_ARG;
  if ((cfg.flags & GSC_FLAG_REUSE_COLLECT) && cfg.reuse == GSC_REUSE_OFF) return GSC_ERR_INVALID_ARG;
  if (cfg.pair_capacity > 0x3FFFFFFFull) cfg.pair_capacity = 0x3FFFFFFFull;

  gsc_ctx* ctx = new (std::nothrow) gsc_ctx();
  if (!ctx) return GSC_ERR_OOM;
  ctx->cfg = cfg;
  ctx->timing = (cfg.flags & GSC_FLAG_TIMING) != 0;
  ctx->user_stream = (cudaStream_t)cuda_stream;
  auto bail = [&](int code) {
    gsc_destroy(ctx);
    return code;
  };
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(GSC_ERR_CUDA);
  if (prepare_derive_f32() != cudaSuccess || prepare_derive_tc() != cudaSuccess || prepare_sort() != cudaSuccess)
    return bail(GSC_ERR_CUDA);
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (cudaMalloc((void**)&ctx->d_tabs, dview_set_bytes() * MAX_MODELS) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_ptab, proj_tab_bytes()) != cudaSuccess)
    return bail(GSC_ERR_OOM);
  if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(GSC_ERR_CUDA);
  if (cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return bail(GSC_ERR_CUDA);
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreateWithFlags(&ctx->ev_rendered[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_copied[i], cudaEventDisableTiming) != cudaSuccess)
      return bail(GSC_ERR_CUDA);
  if (cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return bail(GSC_ERR_CUDA);
  for (int i = 0; i < NSLOT; ++i) {
    if (cudaEventCreateWithFlags(&ctx->ev_slot[i], cudaEventDisableTiming) != cudaSuccess) return bail(GSC_ERR_CUDA);
    if (cudaMallocHost((void**)&ctx->h_fin[i], sizeof(FrameIn)) != cudaSuccess) return bail(GSC_ERR_OOM);
  }
  for (int i = 0; i < 9; ++i)
    if (cudaEventCreate(&ctx->ev_stage[i]) != cudaSuccess) return bail(GSC_ERR_CUDA);
  if (cudaMallocHost((void**)&ctx->h_cnt, sizeof(Counters)) != cudaSuccess) return bail(GSC_ERR_OOM);
  std::memset(ctx->h_cnt, 0, sizeof(Counters));
  if (cudaMalloc((void**)&ctx->d_fin, sizeof(FrameIn)) != cudaSuccess) return bail(GSC_ERR_OOM);
  if (cudaMalloc((void**)&ctx->d_fd, sizeof(FrameDev)) != cudaSuccess) return bail(GSC_ERR_OOM);
  if (cudaMemset(ctx->d_fd, 0, sizeof(FrameDev)) != cudaSuccess) return bail(GSC_ERR_CUDA);
  if (cudaMalloc((void**)&ctx->d_models, sizeof(ModelDev) * MAX_MODELS) != cudaSuccess) return bail(GSC_ERR_OOM);
  if (cudaMalloc((void**)&ctx->d_vis_tab, sizeof(uint32_t*) * MAXV) != cudaSuccess) return bail(GSC_ERR_OOM);
  if (cudaMalloc((void**)&ctx->d_eye_tab, sizeof(uint8_t*) * MAXV) != cudaSuccess) return bail(GSC_ERR_OOM);
  if (cudaMemset(ctx->d_eye_tab, 0, sizeof(uint8_t*) * MAXV) != cudaSuccess) return bail(GSC_ERR_CUDA);
  if (cudaMalloc((void**)&ctx->sb.hist, sizeof(uint32_t) * 4 * 256) != cudaSuccess) return bail(GSC_ERR_OOM);
  if (alloc_pairs(ctx, (uint32_t)cfg.pair_capacity) != GSC_OK) return bail(GSC_ERR_OOM);
  *out = ctx;
  return GSC_OK;
}

void gsc_destroy(gsc_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  invalidate_graph(ctx);
  for (auto& m : ctx->models) {
    dfree(m.px.p); dfree(m.py.p); dfree(m.pz.p); dfree(m.level.p); dfree(m.lod_r.p);
    dfree(m.feat.p); dfree(m.offs.p); dfree(m.scale.p); dfree(m.w32.p);
    dfree(m.feat_bf16.p); dfree(m.w_tc.p); dfree(m.feat_fp8.p); dfree(m.w_tc8.p);
  }
  void* bufs[] = {ctx->d_models, ctx->d_vis_buf, ctx->d_vis_tab, ctx->d_eye_buf, ctx->d_eye_tab, ctx->d_dbg_buf, ctx->d_dbg_tab, ctx->rec.geo,
                  ctx->rec.cop, ctx->rec.col, ctx->rec.aux, ctx->rec.key, ctx->rec.cnt, ctx->s1k0, ctx->s1v0, ctx->s1k1,
                  ctx->s1v1, ctx->s1k2, ctx->s1v2, ctx->offs, ctx->big, ctx->pk0, ctx->pv0, ctx->pk1, ctx->pv1, ctx->ranges, ctx->sb.hist,
                  ctx->sb.status, ctx->cull_masks, ctx->cull_cnt, ctx->st_scan, ctx->d_fin, ctx->d_fd, ctx->attrs,
                  ctx->attrs_fresh, ctx->rw_theta, ctx->rw_w, ctx->d_tabs, ctx->d_ptab, ctx->unfused};
  for (void* p : bufs) dfree(p);
  for (int i = 0; i < ctx->n_caches; ++i) free_cache(ctx->h_caches[i]);
  dfree(ctx->d_caches);
  for (int i = 0; i < MAXV; ++i) {
    dfree(ctx->d_T[i]);
  }
  for (int i = 0; i < NSLOT; ++i) {
    if (ctx->h_fin[i]) cudaFreeHost(ctx->h_fin[i]);
    if (ctx->ev_slot[i]) cudaEventDestroy(ctx->ev_slot[i]);
  }
  for (int i = 0; i < 9; ++i)
    if (ctx->ev_stage[i]) cudaEventDestroy(ctx->ev_stage[i]);
  if (ctx->h_cnt) cudaFreeHost(ctx->h_cnt);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  for (int i = 0; i < 2; ++i) {
    if (ctx->ev_rendered[i]) cudaEventDestroy(ctx->ev_rendered[i]);
    if (ctx->ev_copied[i]) cudaEventDestroy(ctx->ev_copied[i]);
    for (int v = 0; v < MAXV; ++v) dfree(ctx->d_hbuf[i][v]);
  }
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* gsc_last_error(const gsc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int gsc_load_model(gsc_ctx* ctx, const gsc_model_desc* d, uint32_t* model_id_out) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!d || !model_id_out) return fail(ctx, GSC_ERR_INVALID_ARG, "null argument");
  if (d->feat_dim != FDIM || d->k != K || d->hidden != HID)
    return fail(ctx, GSC_ERR_INVALID_ARG, "unsupported dims (feat %u, k %u, hidden %u)", d->feat_dim, d->k, d->hidden);
  if (ctx->models.size() >= MAX_MODELS) return fail(ctx, GSC_ERR_INVALID_ARG, "at most %d models", MAX_MODELS);
  if (d->n_anchors > (1u << 28)) return fail(ctx, GSC_ERR_INVALID_ARG, "too many anchors");
  if (d->n_levels == 0 || d->n_levels > 32) return fail(ctx, GSC_ERR_INVALID_ARG, "n_levels must be 1..32");
  const size_t n = d->n_anchors;
  if (n > 0 && (!d->pos || !d->feat || !d->offset || !d->scale || !d->level))
    return fail(ctx, GSC_ERR_INVALID_ARG, "null model array");
  for (int h = 0; h < 3; ++h)
    if (!d->W1[h] || !d->b1[h] || !d->W2[h] || !d->b2[h]) return fail(ctx, GSC_ERR_INVALID_ARG, "null MLP weights");
  if (n > 0 && !finite_all(d->pos, 3 * n)) return fail(ctx, GSC_ERR_INVALID_ARG, "non-finite anchor position");
  if (!(d->lod_dmax >= 0.f) || !std::isfinite(d->lod_dmax)) return fail(ctx, GSC_ERR_INVALID_ARG, "bad lod_dmax");
  for (size_t i = 0; i < n; ++i)
    if (d->level[i] >= d->n_levels) return fail(ctx, GSC_ERR_INVALID_ARG, "level >= n_levels at anchor %zu", i);
  if (!(d->lod_blend >= 0.f) || !(d->lod_blend <= 32.f)) return fail(ctx, GSC_ERR_INVALID_ARG, "bad lod_blend");
  if (d->level_offset)
    for (size_t i = 0; i < n; ++i)
      if (!(std::fabs(d->level_offset[i]) <= 8.f))
        return fail(ctx, GSC_ERR_INVALID_ARG, "level offset not finite or beyond 8 levels at anchor %zu", i);
  ModelHost mh;
  mh.n = (uint32_t)n;
  std::vector<float> xs(n), ys(n), zs(n);
  for (size_t i = 0; i < n; ++i) {
    xs[i] = d->pos[3 * i];
    ys[i] = d->pos[3 * i + 1];
    zs[i] = d->pos[3 * i + 2];
  }
  // packed float32 weights
  std::vector<float> w(W_FLOATS, 0.f);
  const int outd[3] = {K, 3 * K, 7 * K};
  const int obase[3] = {0, K, 4 * K};
  for (int h = 0; h < 3; ++h) {
    for (int c = 0; c < IN; ++c)
      for (int o = 0; o < HID; ++o) w[WOFF_W1 + c * NH + h * HID + o] = d->W1[h][c * HID + o];
    for (int o = 0; o < HID; ++o) w[WOFF_B1 + h * HID + o] = d->b1[h][o];
    for (int o = 0; o < outd[h]; ++o) {
      for (int c = 0; c < HID; ++c) w[WOFF_W2T + (obase[h] + o) * HID + c] = d->W2[h][c * outd[h] + o];
      w[WOFF_B2 + obase[h] + o] = d->b2[h][o];
    }
  }
  int r;
  // Octree-GS level selection: per-anchor switching radius r_a, level 0
  // always drawn (+inf), r_a = d_max 2^(Delta_a - l) rounded once to float32.
  const bool octree = d->level_offset != nullptr || d->lod_blend > 0.f;
  if (octree) {
    std::vector<float> rad(n);
    for (size_t i = 0; i < n; ++i) {
      const int l = d->level[i];
      const double delta = d->level_offset ? (double)d->level_offset[i] : 0.0;
      rad[i] = l == 0 ? INFINITY : (float)std::ldexp((double)d->lod_dmax * std::exp2(delta), -l);
    }
    if ((r = upload(ctx, mh.lod_r, rad.data(), n * 4))) return r;
  }
  if ((r = upload(ctx, mh.px, xs.data(), n * 4)) || (r = upload(ctx, mh.py, ys.data(), n * 4)) ||
      (r = upload(ctx, mh.pz, zs.data(), n * 4)) || (r = upload(ctx, mh.level, d->level, n)) ||
      (r = upload(ctx, mh.feat, d->feat, n * FDIM * 4)) || (r = upload(ctx, mh.offs, d->offset, n * K * 3 * 4)) ||
      (r = upload(ctx, mh.scale, d->scale, n * 4)) || (r = upload(ctx, mh.w32, w.data(), w.size() * 4)))
    return r;
  // tensor-core forms: bf16 features (converted on the device) and the weight image
  std::vector<uint8_t> img;
  pack_tc_weights(d->W1, d->b1, d->W2, d->b2, img);
  if ((r = upload(ctx, mh.w_tc, img.data(), img.size()))) return r;
  mh.feat_bf16.bytes = n * FDIM * 2;
  if (n) {
    CK(cudaMalloc(&mh.feat_bf16.p, mh.feat_bf16.bytes));
    launch_to_bf16((const float*)mh.feat.p, mh.feat_bf16.p, n * FDIM, ctx->stream);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
  }
  mh.dev.feat_bf16 = mh.feat_bf16.p;
  mh.dev.w_tc = mh.w_tc.p;
  mh.dev.fp8_inv_sx = 1.f;
  if (ctx->cfg.precision == GSC_PREC_FP8) {  // e4m3 features and weight image with per-tensor scales
    const Fp8Scales sc = fp8_scales(d->feat, n, d->W1, d->b1, d->W2);
    mh.dev.fp8_inv_sx = 1.0f / sc.sx;
    mh.w_tc8.bytes = TC8_IMAGE_BYTES;
    CK(cudaMalloc(&mh.w_tc8.p, mh.w_tc8.bytes));
    CK(make_tc8_image(d->W1, d->b1, d->W2, d->b2, sc, mh.w_tc8.p, ctx->stream));
    mh.feat_fp8.bytes = n * FDIM;
    if (n) {
      CK(cudaMalloc(&mh.feat_fp8.p, mh.feat_fp8.bytes));
      launch_to_e4m3((const float*)mh.feat.p, 1.0f / sc.sx, mh.feat_fp8.p, n * FDIM, ctx->stream);
      CK(cudaStreamSynchronize(ctx->stream));
      CK(cudaGetLastError());
    }
    mh.dev.feat_fp8 = mh.feat_fp8.p;
    mh.dev.w_tc8 = mh.w_tc8.p;
  }
  mh.dev.n = mh.n;
  mh.dev.n_levels = d->n_levels;
  mh.dev.lod_dmax = d->lod_dmax;
  mh.dev.px = (const float*)mh.px.p;
  mh.dev.py = (const float*)mh.py.p;
  mh.dev.pz = (const float*)mh.pz.p;
  mh.dev.level = (const uint8_t*)mh.level.p;
  mh.dev.lod_r = octree ? (const float*)mh.lod_r.p : nullptr;
  mh.dev.lod_beta = d->lod_blend;
  mh.dev.feat = (const float4*)mh.feat.p;
  mh.dev.offs = (const float*)mh.offs.p;
  mh.dev.scale = (const float*)mh.scale.p;
  mh.dev.w32 = (const float*)mh.w32.p;
  const uint32_t id = (uint32_t)ctx->models.size();
  CK(cudaMemcpy(ctx->d_models + id, &mh.dev, sizeof(ModelDev), cudaMemcpyHostToDevice));
  ctx->models.push_back(mh);
  *model_id_out = id;
  ctx->cams_set = false;  // buffers are sized at the next gsc_set_cameras
  invalidate_graph(ctx);
  ctx->err.clear();
  return GSC_OK;
}

int gsc_set_cameras(gsc_ctx* ctx, const gsc_camera* cams, uint32_t n) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!cams || n == 0) return fail(ctx, GSC_ERR_INVALID_ARG, "no cameras");
  if (n > ctx->cfg.max_views) return fail(ctx, GSC_ERR_INVALID_ARG, "%u cameras > max_views %u", n, ctx->cfg.max_views);
  uint32_t per_model[MAX_MODELS] = {0};
  for (uint32_t i = 0; i < n; ++i) {
    const gsc_camera& c = cams[i];
    if (c.model_id >= ctx->models.size()) return fail(ctx, GSC_ERR_INVALID_ARG, "camera %u: unknown model", i);
    if (c.width == 0 || c.height == 0 || c.width > 16384 || c.height > 16384)
      return fail(ctx, GSC_ERR_INVALID_ARG, "camera %u: bad size", i);
    if (!(c.fx > 0.f) || !(c.fy > 0.f) || !(c.znear > 0.f) || !finite_all(c.R, 9) || !finite_all(c.t, 3) ||
        !std::isfinite(c.cx) || !std::isfinite(c.cy))
      return fail(ctx, GSC_ERR_INVALID_ARG, "camera %u: bad intrinsics or pose", i);
    if (c.stereo_partner >= 0) {
      const uint32_t p = (uint32_t)c.stereo_partner;
      if (p >= n || p == i || cams[p].stereo_partner != (int32_t)i)
        return fail(ctx, GSC_ERR_INVALID_ARG, "camera %u: stereo partner must reference back", i);
      if (cams[p].model_id != c.model_id || cams[p].width != c.width || cams[p].height != c.height ||
          cams[p].fx != c.fx || cams[p].fy != c.fy)
        return fail(ctx, GSC_ERR_INVALID_ARG, "camera %u: stereo partner must share model and intrinsics", i);
    }
    const bool second_eye = ctx->cfg.stereo_unify && c.stereo_partner >= 0 && (uint32_t)c.stereo_partner < i;
    if (!second_eye) per_model[c.model_id]++;
  }
  // shape of the frame
  bool shape_same = ctx->cams.size() == n;
  for (uint32_t i = 0; shape_same && i < n; ++i) {
    const gsc_camera& a = ctx->cams[i];
    const gsc_camera& b = cams[i];
    shape_same = a.width == b.width && a.height == b.height && a.model_id == b.model_id &&
                 a.stereo_partner == b.stereo_partner;
  }
  ctx->cams.assign(cams, cams + n);
  if (shape_same && ctx->cams_set) return GSC_OK;
  invalidate_graph(ctx);
  ctx->models_used.clear();
  for (uint32_t m = 0; m < MAX_MODELS; ++m)
    if (per_model[m]) ctx->models_used.push_back((int)m);
  int r;
  if ((r = retile(ctx))) return r;
  // visible-id lists: one slot per derivation view, each sized for the largest model
  const uint32_t vcap = std::max<uint32_t>(models_max_n(ctx), 1u);
  if (vcap > ctx->vis_cap || n > ctx->n_vis_slots) {
    const uint32_t slots = std::max(n, ctx->n_vis_slots);
    if ((r = dalloc(ctx, &ctx->d_vis_buf, (size_t)vcap * slots))) return r;
    std::vector<uint32_t*> tab(MAXV, nullptr);
    for (uint32_t i = 0; i < slots; ++i) tab[i] = ctx->d_vis_buf + (size_t)vcap * i;
    CK(cudaMemcpy(ctx->d_vis_tab, tab.data(), sizeof(uint32_t*) * MAXV, cudaMemcpyHostToDevice));
    if ((r = dalloc(ctx, &ctx->d_eye_buf, (size_t)vcap * slots))) return r;
    std::vector<uint8_t*> etab(MAXV, nullptr);
    for (uint32_t i = 0; i < slots; ++i) etab[i] = ctx->d_eye_buf + (size_t)vcap * i;
    CK(cudaMemcpy(ctx->d_eye_tab, etab.data(), sizeof(uint8_t*) * MAXV, cudaMemcpyHostToDevice));
    ctx->vis_cap = vcap;
    ctx->n_vis_slots = slots;
    if (ctx->cfg.flags & GSC_FLAG_DEBUG_ATTRS) {
      if ((r = dalloc(ctx, &ctx->d_dbg_buf, (size_t)vcap * slots * K * 11))) return r;
      std::vector<float*> dt(MAXV, nullptr);
      for (uint32_t i = 0; i < slots; ++i) dt[i] = ctx->d_dbg_buf + (size_t)vcap * K * 11 * i;
      if (!ctx->d_dbg_tab) CK(cudaMalloc((void**)&ctx->d_dbg_tab, sizeof(float*) * MAXV));
      CK(cudaMemcpy(ctx->d_dbg_tab, dt.data(), sizeof(float*) * MAXV, cudaMemcpyHostToDevice));
    }
  }
  // unfused decoder: intermediate tensors for every visible anchor of every view
  if (ctx->cfg.flags & GSC_FLAG_UNFUSED) {
    const size_t items = (size_t)ctx->vis_cap * ctx->n_vis_slots;
    if (items > ctx->unfused_items) {
      if ((r = dalloc(ctx, &ctx->unfused, unfused_scratch_floats(items)))) return r;
      ctx->unfused_items = items;
      invalidate_graph(ctx);
    }
  }
  // caches of derived Gaussians (reuse forms): fresh for a new camera layout
  if ((r = setup_caches(ctx))) return r;
  // records: worst case (every anchor visible), capped at 8M then grown on demand
  unsigned long long worst = 0;
  for (const auto& c : ctx->cams) worst += (unsigned long long)K * ctx->models[c.model_id].n;
  const uint32_t want = (uint32_t)std::min<unsigned long long>(std::max<unsigned long long>(worst, 1024ull), 8ull << 20);
  if (want > ctx->rec_cap) {
    if ((r = alloc_records(ctx, want))) return r;
  }
  if ((r = ensure_status(ctx))) return r;
  ctx->cams_set = true;
  ctx->err.clear();
  return GSC_OK;
}

int gsc_render_frame(gsc_ctx* ctx, void* const* out_rgb, gsc_frame_stats* stats) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!out_rgb) return fail(ctx, GSC_ERR_INVALID_ARG, "null output table");
  for (size_t i = 0; i < ctx->cams.size(); ++i)
    if (!out_rgb[i]) return fail(ctx, GSC_ERR_INVALID_ARG, "null output image %zu", i);
  float* Ts[MAXV] = {};
  if (ctx->cfg.flags & GSC_FLAG_DEBUG_T) {
    for (size_t i = 0; i < ctx->cams.size(); ++i) {
      const size_t b = (size_t)ctx->cams[i].width * ctx->cams[i].height * 4;
      if (ctx->d_T_bytes[i] < b) {
        dfree(ctx->d_T[i]);
        ctx->d_T[i] = nullptr;
        CK(cudaMalloc((void**)&ctx->d_T[i], b));
        ctx->d_T_bytes[i] = b;
      }
      Ts[i] = ctx->d_T[i];
    }
  }
  return render_impl(ctx, out_rgb, (ctx->cfg.flags & GSC_FLAG_DEBUG_T) ? Ts : nullptr, stats, stats != nullptr);
}

namespace {
size_t image_bytes(const gsc_ctx* ctx, size_t i) {
  const size_t px = (size_t)ctx->cams[i].width * ctx->cams[i].height;
  return px * (ctx->cfg.out_format == GSC_OUT_RGBA8 ? 4 : 12);
}

// Device image set `set` sized for the current cameras.
int ensure_host_images(gsc_ctx* ctx, int set, void** outs) {
  for (size_t i = 0; i < ctx->cams.size(); ++i) {
    const size_t b = image_bytes(ctx, i);
    if (ctx->d_hbuf_bytes[set][i] < b) {
      dfree(ctx->d_hbuf[set][i]);
      ctx->d_hbuf[set][i] = nullptr;
      CK(cudaMalloc(&ctx->d_hbuf[set][i], b));
      ctx->d_hbuf_bytes[set][i] = b;
    }
    outs[i] = ctx->d_hbuf[set][i];
  }
  return GSC_OK;
}

}  // namespace

int gsc_render_frame_host(gsc_ctx* ctx, void* const* out_rgb, gsc_frame_stats* stats) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!out_rgb) return fail(ctx, GSC_ERR_INVALID_ARG, "null output table");
  if (!ctx->cams_set) return fail(ctx, GSC_ERR_STATE, "gsc_set_cameras must come first");
  for (size_t i = 0; i < ctx->cams.size(); ++i)
    if (!out_rgb[i]) return fail(ctx, GSC_ERR_INVALID_ARG, "null output image %zu", i);
  int r = gsc_wait_host(ctx);
  if (r) return r;
  void* outs[MAXV] = {};
  if ((r = ensure_host_images(ctx, 0, outs))) return r;
  gsc_frame_stats tmp;
  r = render_impl(ctx, outs, nullptr, stats ? stats : &tmp, true);
  if (r) return r;
  for (size_t i = 0; i < ctx->cams.size(); ++i)
    CK(cudaMemcpyAsync(out_rgb[i], outs[i], image_bytes(ctx, i), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return GSC_OK;
}

int gsc_render_frame_host_async(gsc_ctx* ctx, void* const* out) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!out) return fail(ctx, GSC_ERR_INVALID_ARG, "null output table");
  if (!ctx->cams_set) return fail(ctx, GSC_ERR_STATE, "gsc_set_cameras must come first");
  for (size_t i = 0; i < ctx->cams.size(); ++i)
    if (!out[i]) return fail(ctx, GSC_ERR_INVALID_ARG, "null output image %zu", i);
  if (ctx->cfg.reuse == GSC_REUSE_LEARNED && !ctx->reuse_set)
    return fail(ctx, GSC_ERR_STATE, "the learned reuse form needs predictor weights (gsc_reuse_set_weights)");
  const int set = ctx->hslot;
  ctx->hslot ^= 1;
  if (ctx->hpending[set]) {  // the copy of the frame two back still reads this set
    CK(cudaEventSynchronize(ctx->ev_copied[set]));
    ctx->hpending[set] = false;
  }
  void* outs[MAXV] = {};
  int r = ensure_host_images(ctx, set, outs);
  if (r) return r;
  ctx->pending = false;  // errors of pipelined frames are collected by gsc_wait_host
  ctx->keep_err = true;
  r = enqueue_frame(ctx, outs, nullptr);
  ctx->keep_err = false;
  if (r) return r;
  CK(cudaEventRecord(ctx->ev_rendered[set], ctx->stream));
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_rendered[set], 0));
  for (size_t i = 0; i < ctx->cams.size(); ++i)
    CK(cudaMemcpyAsync(out[i], outs[i], image_bytes(ctx, i), cudaMemcpyDeviceToHost, ctx->copy_stream));
  CK(cudaEventRecord(ctx->ev_copied[set], ctx->copy_stream));
  ctx->hpending[set] = true;
  ctx->pending = false;
  return GSC_OK;
}

int gsc_wait_host(gsc_ctx* ctx) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  bool any = false;
  for (int set = 0; set < 2; ++set)
    if (ctx->hpending[set]) {
      CK(cudaEventSynchronize(ctx->ev_copied[set]));
      ctx->hpending[set] = false;
      any = true;
    }
  if (!any) return GSC_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  return take_sticky_error(ctx);
}

static int dbg_sync(gsc_ctx* ctx);
static int dbg_copy(gsc_ctx* ctx, void* dst, const void* src, uint64_t count, uint64_t cap, size_t elem);

int gsc_set_tiling(gsc_ctx* ctx, uint32_t tile_w, uint32_t tile_h, uint32_t blocks_per_sm) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!tiling_ok(tile_w, tile_h, blocks_per_sm))
    return fail(ctx, GSC_ERR_INVALID_ARG, "unsupported tiling %ux%u, %u blocks/SM", tile_w, tile_h, blocks_per_sm);
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->cfg.tile_w = tile_w;
  ctx->cfg.tile_h = tile_h;
  ctx->cfg.blocks_per_sm = blocks_per_sm;
  if (ctx->cams_set) {
    int r = retile(ctx);
    if (r) return r;
  }
  ctx->err.clear();
  return GSC_OK;
}

// ------------------------------------------------------------------ reuse predictor (K12)
int gsc_reuse_set_weights(gsc_ctx* ctx, const float* params, uint32_t n_params) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!params || n_params != GSC_REUSE_NPARAM)
    return fail(ctx, GSC_ERR_INVALID_ARG, "predictor takes %d parameters", GSC_REUSE_NPARAM);
  if (!finite_all(params, n_params)) return fail(ctx, GSC_ERR_INVALID_ARG, "non-finite predictor parameter");
  CK(cudaStreamSynchronize(ctx->stream));
  int r;
  if (!ctx->rw_theta && ((r = dalloc(ctx, &ctx->rw_theta, GSC_REUSE_NPARAM)) ||
                         (r = dalloc(ctx, &ctx->rw_w, GSC_REUSE_NPARAM))))
    return r;
  CK(cudaMemcpy(ctx->rw_theta, params, sizeof(float) * GSC_REUSE_NPARAM, cudaMemcpyHostToDevice));
  launch_reuse_round(ctx->rw_theta, ctx->rw_w, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->reuse_set = true;
  ctx->err.clear();
  return GSC_OK;
}

int gsc_reuse_get_weights(gsc_ctx* ctx, float* params, uint32_t n_params) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!params || n_params != GSC_REUSE_NPARAM)
    return fail(ctx, GSC_ERR_INVALID_ARG, "predictor takes %d parameters", GSC_REUSE_NPARAM);
  if (!ctx->reuse_set) return fail(ctx, GSC_ERR_STATE, "no predictor weights");
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(params, ctx->rw_theta, sizeof(float) * GSC_REUSE_NPARAM, cudaMemcpyDeviceToHost));
  return GSC_OK;
}

int gsc_reuse_collect(gsc_ctx* ctx, uint32_t dview, float* z, uint8_t* label, uint32_t* vis_index, uint64_t cap,
                      uint64_t* n) {
  if (!ctx || !n) return GSC_ERR_INVALID_ARG;
  if (!(ctx->cfg.flags & GSC_FLAG_REUSE_COLLECT) || ctx->n_caches == 0)
    return fail(ctx, GSC_ERR_STATE, "collection needs a cached form created with GSC_FLAG_REUSE_COLLECT");
  if (ctx->pending) {
    int r = finish_frame(ctx);
    if (r) return r;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (dview >= (uint32_t)ctx->n_caches) return fail(ctx, GSC_ERR_INVALID_ARG, "no cache for view %u", dview);
  const uint32_t V = ctx->h_cnt->vis_count[dview];
  std::vector<uint8_t> lab(V);
  if (V) CK(cudaMemcpy(lab.data(), ctx->h_caches[dview].clab, V, cudaMemcpyDeviceToHost));
  uint64_t cnt = 0;
  for (uint32_t i = 0; i < V; ++i) cnt += lab[i] != 255;
  *n = cnt;
  if (!z && !label && !vis_index) return GSC_OK;
  std::vector<float> zz;
  if (z) {
    zz.resize((size_t)V * 36);
    if (V) CK(cudaMemcpy(zz.data(), ctx->h_caches[dview].cz, zz.size() * 4, cudaMemcpyDeviceToHost));
  }
  uint64_t o = 0;
  for (uint32_t i = 0; i < V && o < cap; ++i) {
    if (lab[i] == 255) continue;
    if (z) std::memcpy(z + o * 36, zz.data() + (size_t)i * 36, 36 * 4);
    if (label) label[o] = lab[i];
    if (vis_index) vis_index[o] = i;
    ++o;
  }
  return GSC_OK;
}

namespace {
uint64_t splitmix64_next(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct TrainBufs {
  float *Z = nullptr, *Y = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *part = nullptr, *loss = nullptr;
  uint32_t *order = nullptr, *ctl = nullptr;
  ~TrainBufs() {
    void* p[] = {Z, Y, m, v, grad, part, loss, order, ctl};
    for (void* q : p) dfree(q);
  }
};

int reuse_upload(gsc_ctx* ctx, TrainBufs& B, const float* z, const uint8_t* y, uint64_t n, uint32_t epochs,
                 uint32_t batch, const uint32_t* order, uint64_t seed, ReuseTrain& T) {
  int r;
  if ((r = dalloc(ctx, &B.Z, (size_t)n * 36)) || (r = dalloc(ctx, &B.Y, (size_t)n)) ||
      (r = dalloc(ctx, &B.order, (size_t)n * epochs)) || (r = dalloc(ctx, &B.m, GSC_REUSE_NPARAM)) ||
      (r = dalloc(ctx, &B.v, GSC_REUSE_NPARAM)) || (r = dalloc(ctx, &B.grad, GSC_REUSE_NPARAM)) ||
      (r = dalloc(ctx, &B.part, (size_t)reuse_blocks(batch) * (GSC_REUSE_NPARAM + 1))) ||
      (r = dalloc(ctx, &B.loss, epochs)) || (r = dalloc(ctx, &B.ctl, 2)))
    return r;
  std::vector<float> yf(n);
  for (uint64_t i = 0; i < n; ++i) {
    if (y[i] > 1) return fail(ctx, GSC_ERR_INVALID_ARG, "label %llu is %u (0 or 1 expected)", (unsigned long long)i, y[i]);
    yf[i] = (float)y[i];
  }
  if (!finite_all(z, (size_t)n * 36)) return fail(ctx, GSC_ERR_INVALID_ARG, "non-finite predictor input");
  std::vector<uint32_t> ord((size_t)n * epochs);
  if (order) {
    for (size_t i = 0; i < ord.size(); ++i) {
      if (order[i] >= n) return fail(ctx, GSC_ERR_INVALID_ARG, "order[%zu] out of range", i);
      ord[i] = order[i];
    }
  } else {  // a Fisher-Yates shuffle per epoch from SplitMix64(seed)
    uint64_t st = seed;
    for (uint32_t e = 0; e < epochs; ++e) {
      uint32_t* o = ord.data() + (size_t)e * n;
      for (uint64_t i = 0; i < n; ++i) o[i] = (uint32_t)i;
      for (uint64_t i = n - 1; i > 0; --i) std::swap(o[i], o[splitmix64_next(st) % (i + 1)]);
    }
  }
  CK(cudaMemcpy(B.Z, z, (size_t)n * 36 * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.Y, yf.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.order, ord.data(), ord.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemset(B.m, 0, GSC_REUSE_NPARAM * 4));
  CK(cudaMemset(B.v, 0, GSC_REUSE_NPARAM * 4));
  CK(cudaMemset(B.loss, 0, (size_t)epochs * 4));
  CK(cudaMemset(B.ctl, 0, 8));
  T = ReuseTrain{B.Z, B.Y, B.order, ctx->rw_theta, ctx->rw_w, B.m, B.v, B.grad, B.part, B.loss, B.ctl};
  return GSC_OK;
}
}  // namespace

int gsc_reuse_train(gsc_ctx* ctx, const float* z, const uint8_t* y, uint64_t n, uint32_t epochs, uint32_t batch,
                    float lr, uint64_t seed, const uint32_t* order, float* epoch_loss) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!z || !y || n == 0 || n > (1ull << 26) || epochs == 0 || batch == 0 || !(lr > 0.f) || !std::isfinite(lr) ||
      n * (uint64_t)epochs > (1ull << 31))
    return fail(ctx, GSC_ERR_INVALID_ARG, "bad training arguments");
  if (!ctx->reuse_set) return fail(ctx, GSC_ERR_STATE, "set initial predictor weights first");
  if (ctx->pending) {
    int r = finish_frame(ctx);
    if (r) return r;
  }
  batch = (uint32_t)std::min<uint64_t>(batch, n);
  TrainBufs B;
  ReuseTrain T{};
  int r = reuse_upload(ctx, B, z, y, n, epochs, batch, order, seed, T);
  if (r) return r;
  // one epoch as a graph: every mini-batch's fwd/bwd, reduce and Adam step
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  for (uint64_t b0 = 0; b0 < n; b0 += batch) {
    const uint32_t nb = (uint32_t)std::min<uint64_t>(batch, n - b0);
    launch_reuse_batch(T, (uint32_t)n, (uint32_t)b0, nb, lr, 1.0f / (float)n, ctx->stream);
  }
  launch_reuse_epoch_end(T, ctx->stream);
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  if (e != cudaSuccess) return fail(ctx, GSC_ERR_CUDA, "training graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, GSC_ERR_CUDA, "training graph instantiate: %s", cudaGetErrorString(e));
  for (uint32_t ep = 0; ep < epochs && e == cudaSuccess; ++ep) e = cudaGraphLaunch(ge, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaGraphExecDestroy(ge);
  if (e != cudaSuccess) return fail(ctx, GSC_ERR_CUDA, "training: %s", cudaGetErrorString(e));
  if (epoch_loss) CK(cudaMemcpy(epoch_loss, B.loss, (size_t)epochs * 4, cudaMemcpyDeviceToHost));
  ctx->err.clear();
  return GSC_OK;
}

int gsc_debug_frame_upload_bytes(void) { return (int)sizeof(FrameIn); }

int gsc_debug_reuse_grad(gsc_ctx* ctx, const float* z, const uint8_t* y, uint64_t n, float* grad, float* loss) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!z || !y || !grad || n == 0 || n > (1ull << 24)) return fail(ctx, GSC_ERR_INVALID_ARG, "bad arguments");
  if (!ctx->reuse_set) return fail(ctx, GSC_ERR_STATE, "set predictor weights first");
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<uint32_t> ident(n);
  for (uint64_t i = 0; i < n; ++i) ident[i] = (uint32_t)i;
  TrainBufs B;
  ReuseTrain T{};
  int r = reuse_upload(ctx, B, z, y, n, 1, (uint32_t)n, ident.data(), 0, T);
  if (r) return r;
  launch_reuse_batch(T, (uint32_t)n, 0, (uint32_t)n, 0.f, 1.0f / (float)n, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(grad, B.grad, GSC_REUSE_NPARAM * 4, cudaMemcpyDeviceToHost));
  if (loss) CK(cudaMemcpy(loss, B.loss, 4, cudaMemcpyDeviceToHost));
  return GSC_OK;
}

int gsc_cache_reset(gsc_ctx* ctx) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < ctx->n_caches; ++i) {
    int r = init_cache(ctx, ctx->h_caches[i], ctx->cache_na[i]);
    if (r) return r;
  }
  ctx->err.clear();
  return GSC_OK;
}

int gsc_debug_cache(gsc_ctx* ctx, uint32_t d, uint32_t* vstat, uint64_t cap, uint64_t* n, uint32_t* state8) {
  int r = dbg_sync(ctx);
  if (r) return r;
  if (d >= (uint32_t)ctx->n_caches || !n) return fail(ctx, GSC_ERR_INVALID_ARG, "no cache for view %u", d);
  const CacheDev& c = ctx->h_caches[d];
  uint32_t st[CS_WORDS];
  CK(cudaMemcpy(st, c.state, sizeof st, cudaMemcpyDeviceToHost));
  static_assert(CS_S == 7, "the 8 documented state words are CS_T .. CS_S");
  if (state8)
    for (int i = 0; i <= CS_S; ++i) state8[i] = st[i];
  *n = st[CS_VIS];
  return dbg_copy(ctx, vstat, c.vstat, st[CS_VIS], cap, 4);
}

int gsc_synchronize(gsc_ctx* ctx) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  if (!ctx->pending && !ctx->async_since_sync) return GSC_OK;
  ctx->pending = false;
  ctx->async_since_sync = false;
  return take_sticky_error(ctx);
}

// ------------------------------------------------------------------ debug exports
static int dbg_sync(gsc_ctx* ctx) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  return GSC_OK;
}

static int dbg_copy(gsc_ctx* ctx, void* dst, const void* src, uint64_t count, uint64_t cap, size_t elem) {
  const uint64_t m = std::min(count, cap);
  if (m && dst) CK(cudaMemcpy(dst, src, m * elem, cudaMemcpyDeviceToHost));
  return GSC_OK;
}

int gsc_debug_visible(gsc_ctx* ctx, uint32_t d, uint32_t* ids, uint64_t cap, uint64_t* n) {
  int r = dbg_sync(ctx);
  if (r) return r;
  if (d >= MAXV || !n) return fail(ctx, GSC_ERR_INVALID_ARG, "bad view");
  uint32_t cnt = ctx->h_cnt->vis_count[d];
  *n = cnt;
  if (!ctx->d_vis_buf || d >= ctx->n_vis_slots) return cnt ? GSC_ERR_STATE : GSC_OK;
  return dbg_copy(ctx, ids, ctx->d_vis_buf + (size_t)ctx->vis_cap * d, cnt, cap, 4);
}

int gsc_debug_visible_eyes(gsc_ctx* ctx, uint32_t d, uint8_t* eyes, uint64_t cap, uint64_t* n) {
  int r = dbg_sync(ctx);
  if (r) return r;
  if (d >= MAXV || !n) return fail(ctx, GSC_ERR_INVALID_ARG, "bad view");
  uint32_t cnt = ctx->h_cnt->vis_count[d];
  *n = cnt;
  if (!ctx->d_eye_buf || d >= ctx->n_vis_slots) return cnt ? GSC_ERR_STATE : GSC_OK;
  return dbg_copy(ctx, eyes, ctx->d_eye_buf + (size_t)ctx->vis_cap * d, cnt, cap, 1);
}

int gsc_debug_dviews(gsc_ctx* ctx, uint32_t* n_dviews, int32_t* first_cam) {
  int r = dbg_sync(ctx);
  if (r) return r;
  FrameDev* h = (FrameDev*)malloc(sizeof(FrameDev));
  if (!h) return GSC_ERR_OOM;
  cudaError_t e = cudaMemcpy(h, ctx->d_fd, sizeof(FrameDev), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    free(h);
    return fail(ctx, GSC_ERR_CUDA, "%s", cudaGetErrorString(e));
  }
  if (n_dviews) *n_dviews = h->n_dviews;
  if (first_cam)
    for (int i = 0; i < MAXV; ++i) first_cam[i] = i < (int)h->n_dviews ? h->dview_cam[i][0] : -1;
  free(h);
  return GSC_OK;
}

int gsc_debug_attrs(gsc_ctx* ctx, uint32_t d, float* attrs, uint64_t cap, uint64_t* n) {
  int r = dbg_sync(ctx);
  if (r) return r;
  if (!(ctx->cfg.flags & GSC_FLAG_DEBUG_ATTRS) || !ctx->d_dbg_buf)
    return fail(ctx, GSC_ERR_STATE, "context was created without GSC_FLAG_DEBUG_ATTRS");
  if (d >= ctx->n_vis_slots || !n) return fail(ctx, GSC_ERR_INVALID_ARG, "bad view");
  const uint32_t cnt = ctx->h_cnt->vis_count[d];
  *n = cnt;
  return dbg_copy(ctx, attrs, ctx->d_dbg_buf + (size_t)ctx->vis_cap * K * 11 * d, cnt, cap, sizeof(float) * K * 11);
}

int gsc_debug_records(gsc_ctx* ctx, float* rec12, uint32_t* depth_key, uint32_t* tile_count, uint64_t cap,
                      uint64_t* n) {
  int r = dbg_sync(ctx);
  if (r) return r;
  if (!n) return GSC_ERR_INVALID_ARG;
  const uint32_t cnt = ctx->h_cnt->n_records;
  *n = cnt;
  const uint64_t m = std::min<uint64_t>(cnt, cap);
  if (m == 0) return GSC_OK;
  // records that cover no tile hold only their (invalid) key on the device:
  // report them with zero geometry, their camera and a count of 0
  std::vector<uint32_t> keys(m);
  CK(cudaMemcpy(keys.data(), ctx->rec.key, m * 4, cudaMemcpyDeviceToHost));
  const Counters& hc = *ctx->h_cnt;
  auto camera_of = [&](uint64_t i) {
    uint32_t c = 0;
    while (c + 1 < ctx->cams.size() && i >= hc.rec_base[c + 1]) ++c;
    return c;
  };
  if (rec12) {
    std::vector<float4> g(m), c(m), o(m);
    CK(cudaMemcpy(g.data(), ctx->rec.geo, m * 16, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(c.data(), ctx->rec.cop, m * 16, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(o.data(), ctx->rec.col, m * 16, cudaMemcpyDeviceToHost));
    for (uint64_t i = 0; i < m; ++i) {
      float* q = rec12 + i * 12;
      if (keys[i] == INVALID_KEY) {
        for (int u = 0; u < 11; ++u) q[u] = 0.f;
        const uint32_t bits = camera_of(i);
        std::memcpy(&q[11], &bits, 4);
        continue;
      }
      q[0] = g[i].x; q[1] = g[i].y; q[2] = g[i].z; q[3] = g[i].w;
      q[4] = c[i].x; q[5] = c[i].y; q[6] = c[i].z; q[7] = c[i].w;
      q[8] = o[i].x; q[9] = o[i].y; q[10] = o[i].z; q[11] = o[i].w;
    }
  }
  if (depth_key) std::memcpy(depth_key, keys.data(), m * 4);
  if (tile_count) {
    CK(cudaMemcpy(tile_count, ctx->rec.cnt, m * 4, cudaMemcpyDeviceToHost));
    for (uint64_t i = 0; i < m; ++i)
      if (keys[i] == INVALID_KEY) tile_count[i] = 0;
  }
  return GSC_OK;
}

int gsc_debug_pairs(gsc_ctx* ctx, uint32_t* keys, uint32_t* vals, uint64_t cap, uint64_t* n) {
  int r = dbg_sync(ctx);
  if (r) return r;
  if (!n) return GSC_ERR_INVALID_ARG;
  const uint32_t cnt = ctx->h_cnt->n_pairs_used;
  *n = cnt;
  if ((r = dbg_copy(ctx, keys, ctx->pkeys_out, cnt, cap, 4))) return r;
  return dbg_copy(ctx, vals, ctx->pvals_out, cnt, cap, 4);
}

int gsc_debug_depth_order(gsc_ctx* ctx, uint32_t* vals, uint64_t cap, uint64_t* n) {
  int r = dbg_sync(ctx);
  if (r) return r;
  if (!n) return GSC_ERR_INVALID_ARG;
  const uint32_t cnt = ctx->h_cnt->n_valid;
  *n = cnt;
  return dbg_copy(ctx, vals, ctx->order_out, cnt, cap, 4);
}

int gsc_debug_ranges(gsc_ctx* ctx, uint32_t* ranges, uint64_t cap, uint64_t* n) {
  int r = dbg_sync(ctx);
  if (r) return r;
  if (!n) return GSC_ERR_INVALID_ARG;
  *n = ctx->total_tiles;
  return dbg_copy(ctx, ranges, ctx->ranges, ctx->total_tiles, cap, 8);
}

int gsc_debug_final_T(gsc_ctx* ctx, uint32_t v, float* T, uint64_t cap, uint64_t* n) {
  int r = dbg_sync(ctx);
  if (r) return r;
  if (!(ctx->cfg.flags & GSC_FLAG_DEBUG_T)) return fail(ctx, GSC_ERR_STATE, "context was created without GSC_FLAG_DEBUG_T");
  if (v >= ctx->cams.size() || !n) return fail(ctx, GSC_ERR_INVALID_ARG, "bad camera");
  const uint64_t cnt = (uint64_t)ctx->cams[v].width * ctx->cams[v].height;
  *n = cnt;
  return dbg_copy(ctx, T, ctx->d_T[v], cnt, cap, 4);
}

int gsc_debug_blend_work(gsc_ctx* ctx, uint64_t* work) {
  int r = dbg_sync(ctx);
  if (r) return r;
  if (!(ctx->cfg.flags & GSC_FLAG_BLEND_WORK)) return fail(ctx, GSC_ERR_STATE, "context was created without GSC_FLAG_BLEND_WORK");
  if (!work) return fail(ctx, GSC_ERR_INVALID_ARG, "null output");
  unsigned long long w[2];
  CK(cudaMemcpy(w, ctx->d_fd->blend_work, sizeof(w), cudaMemcpyDeviceToHost));
  work[0] = w[0];
  work[1] = w[1];
  return GSC_OK;
}

int gsc_debug_set_spin_limit(gsc_ctx* ctx, uint32_t limit) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  ctx->spin_limit = limit;
  return GSC_OK;
}

int gsc_debug_sort_pairs(gsc_ctx* ctx, uint32_t* keys, uint32_t* vals, uint64_t n, uint32_t bits) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!keys || !vals || bits == 0 || bits > 32 || n > 0x3FFFFFFFull) return fail(ctx, GSC_ERR_INVALID_ARG, "bad sort args");
  if (n == 0) return GSC_OK;
  if (n > ctx->pair_cap) {
    int r = alloc_pairs(ctx, (uint32_t)n);
    if (r) return r;
  }
  int r = ensure_status(ctx);
  if (r) return r;
  uint32_t* d_n = nullptr;
  CK(cudaMalloc((void**)&d_n, 4));
  const uint32_t n32 = (uint32_t)n;
  CK(cudaMemcpy(d_n, &n32, 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->pk0, keys, n * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->pv0, vals, n * 4, cudaMemcpyHostToDevice));
  launch_bump_epoch(ctx->d_fd, ctx->spin_limit, ctx->stream);
  uint32_t *ok = nullptr, *ov = nullptr;
  launch_sort_impl(ctx->pk0, ctx->pv0, ctx->pk1, ctx->pv1, ctx->pk0, ctx->pv0, d_n, nullptr, (int)bits, 0, SLOT_SORT2,
                   ctx->d_fd, ctx->sb, ctx->n_sm, ctx->stream, &ok, &ov, 16);
  CK(cudaStreamSynchronize(ctx->stream));
  uint32_t err = 0;
  CK(cudaMemcpy(&err, &ctx->d_fd->err, 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(keys, ok, n * 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(vals, ov, n * 4, cudaMemcpyDeviceToHost));
  cudaFree(d_n);
  invalidate_graph(ctx);
  if (err & ERR_TIMEOUT) return fail(ctx, GSC_ERR_TIMEOUT, "a bounded device-side wait gave up");
  return GSC_OK;
}

int gsc_debug_wait_timeout(gsc_ctx* ctx, uint32_t spin_limit) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  launch_bump_epoch(ctx->d_fd, spin_limit, ctx->stream);
  launch_wait_probe(ctx->d_fd, ctx->st_scan, ctx->stream);
  CK(cudaStreamSynchronize(ctx->stream));
  uint32_t err = 0;
  CK(cudaMemcpy(&err, &ctx->d_fd->err, 4, cudaMemcpyDeviceToHost));
  if (err & ERR_TIMEOUT) return fail(ctx, GSC_ERR_TIMEOUT, "a bounded device-side wait gave up");
  return fail(ctx, GSC_ERR_INTERNAL, "the probe's wait did not time out");
}

int gsc_debug_scan(gsc_ctx* ctx, uint32_t* vals, uint64_t n, uint64_t* total) {
  if (!ctx) return GSC_ERR_INVALID_ARG;
  if (!vals || !total || n > 0x3FFFFFFFull) return fail(ctx, GSC_ERR_INVALID_ARG, "bad scan args");
  *total = 0;
  if (n == 0) return GSC_OK;
  if (n > ctx->pair_cap) {
    int r = alloc_pairs(ctx, (uint32_t)n);
    if (r) return r;
  }
  int r = ensure_status(ctx);
  if (r) return r;
  uint32_t* d_n = nullptr;
  CK(cudaMalloc((void**)&d_n, 8));
  const uint32_t n32 = (uint32_t)n;
  CK(cudaMemcpy(d_n, &n32, 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->pk0, vals, n * 4, cudaMemcpyHostToDevice));
  launch_bump_epoch(ctx->d_fd, ctx->spin_limit, ctx->stream);
  launch_scan_u32(ctx->pk0, nullptr, d_n, ctx->pk1, d_n + 1, ctx->st_scan, ctx->d_fd, SLOT_SCAN, ctx->n_sm, ctx->stream);
  CK(cudaStreamSynchronize(ctx->stream));
  uint32_t tot = 0, err = 0;
  CK(cudaMemcpy(&tot, d_n + 1, 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&err, &ctx->d_fd->err, 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(vals, ctx->pk1, n * 4, cudaMemcpyDeviceToHost));
  cudaFree(d_n);
  *total = tot;
  if (err & ERR_TIMEOUT) return fail(ctx, GSC_ERR_TIMEOUT, "a bounded device-side wait gave up");
  return GSC_OK;
}

}  // extern "C"
