// zq_api.cu -- the C ABI declared in include/zq.h.
#include <algorithm>
#include <cstring>
#include <new>

#include "zq_internal.cuh"

using zq::Ctx;

struct zq_ctx {
  Ctx c;
};

namespace {

template <typename T>
zq_status grow(T** p, int64_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (count <= 0) count = 1;
  if (cudaMalloc(reinterpret_cast<void**>(p), (size_t)count * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    return ZQ_ENOMEM;
  }
  return ZQ_OK;
}

void free_all(Ctx& c) {
  void* ps[] = {c.off, c.small_d, c.fused_bin_start, c.fused_bin_bodies, c.bead_body, c.aabb, c.body_q, c.count_tab, c.count_tab2, c.root, c.key, c.skey, c.perm,
                c.key_tmp, c.perm_tmp, c.sort_hist, c.lcp, c.cl, c.cr, c.first, c.cnt, c.height,
                c.roff, c.scan_tmp, c.counters, c.sid, c.slot_of, c.sc,
                c.sheight, c.bstart, c.bhist, c.st64, c.rec64, c.rec32, c.x64, c.x32, c.x64b, c.x32b, c.stage, c.ord,
                c.pos_of, c.pnode, c.pc, c.proff, c.ph, c.prw, c.seg, c.seg_r, c.topv,
                c.top_cnt, c.nseg, c.srw, c.xblk};
  for (void* p : ps)
    if (p) cudaFree(p);
  Ctx fresh;
  fresh.device = c.device;
  fresh.stream = c.stream;
  fresh.num_sms = c.num_sms;
  fresh.launches = c.launches;
  c = fresh;
}

void destroy_streams(Ctx& c) {
  for (int i = 0; i < 4; ++i) {
    if (c.side[i]) {
      cudaStreamSynchronize(c.side[i]);
      cudaStreamDestroy(c.side[i]);
    }
    if (c.join_ev[i]) cudaEventDestroy(c.join_ev[i]);
    c.side[i] = nullptr;
    c.join_ev[i] = nullptr;
  }
  if (c.fork_ev) cudaEventDestroy(c.fork_ev);
  c.fork_ev = nullptr;
}

#define ZQ_TRY(expr)                  \
  do {                                \
    zq_status _s = (expr);            \
    if (_s != ZQ_OK) return _s;       \
  } while (0)

zq_status ensure_capacity(Ctx& c, int64_t N, int64_t m, int64_t hist_words) {
  if (N > c.cap_N || m > c.cap_m) {
    const int64_t nodes = N;  // >= N - m
    ZQ_TRY(grow(&c.off, m + 1));
    ZQ_TRY(grow(&c.small_d, m));
    ZQ_TRY(grow(&c.fused_bin_start, m + 1));
    ZQ_TRY(grow(&c.fused_bin_bodies, m));
    ZQ_TRY(grow(&c.bead_body, N));
    ZQ_TRY(grow(&c.aabb, 6 * m));
    ZQ_TRY(grow(&c.body_q, 3 * m));
    ZQ_TRY(grow(&c.root, m));
    ZQ_TRY(grow(&c.key, N));
    ZQ_TRY(grow(&c.skey, N));
    ZQ_TRY(grow(&c.perm, N));
    ZQ_TRY(grow(&c.key_tmp, N));
    ZQ_TRY(grow(&c.perm_tmp, N));
    ZQ_TRY(grow(&c.lcp, nodes));
    ZQ_TRY(grow(&c.cl, nodes));
    ZQ_TRY(grow(&c.cr, nodes));
    ZQ_TRY(grow(&c.first, nodes));
    ZQ_TRY(grow(&c.cnt, nodes));
    ZQ_TRY(grow(&c.height, nodes));
    ZQ_TRY(grow(&c.roff, nodes));
    ZQ_TRY(grow(&c.scan_tmp, zq::scan_tmp_words(nodes)));
    ZQ_TRY(grow(&c.counters, 4));
    if (!c.count_tab) {
      ZQ_TRY(grow(&c.count_tab, 2 * zq::kCountTab));
      ZQ_TRY(grow(&c.count_tab2, 2 * zq::kCountTab));
      ZQ_TRY(zq::launch_count_table(c));
      ZQ_TRY(zq::launch_count_table_dd(c));
    }
    ZQ_TRY(grow(&c.sid, nodes));
    ZQ_TRY(grow(&c.slot_of, nodes));
    ZQ_TRY(grow(&c.sc, nodes));
    ZQ_TRY(grow(&c.sheight, nodes));
    ZQ_TRY(grow(&c.bstart, zq::kMaxBuckets + 1));
    ZQ_TRY(grow(&c.bhist, zq::bucket_hist_words(nodes)));
    ZQ_TRY(grow(&c.st64, nodes * zq::kState));
    ZQ_TRY(grow(&c.rec64, nodes * zq::kRecMax));
    ZQ_TRY(grow(&c.rec32, nodes * zq::kRecMax));
    ZQ_TRY(grow(&c.x64, nodes * 6));
    ZQ_TRY(grow(&c.x32, nodes * 6));
    ZQ_TRY(grow(&c.x64b, nodes * 6));
    ZQ_TRY(grow(&c.x32b, nodes * 6));
    ZQ_TRY(grow(&c.pos_of, nodes));
    ZQ_TRY(grow(&c.pnode, nodes));
    ZQ_TRY(grow(&c.pc, nodes));
    ZQ_TRY(grow(&c.proff, nodes));
    ZQ_TRY(grow(&c.ph, nodes));
    ZQ_TRY(grow(&c.prw, nodes + 1));
    ZQ_TRY(grow(&c.seg, nodes));
    ZQ_TRY(grow(&c.seg_r, nodes));
    ZQ_TRY(grow(&c.topv, nodes));
    ZQ_TRY(grow(&c.top_cnt, m));
    ZQ_TRY(grow(&c.nseg, 2));
    ZQ_TRY(grow(&c.srw, nodes));
    ZQ_CUDA_TRY(cudaMemsetAsync(c.counters, 0, 4 * sizeof(int32_t), c.stream));
    c.cap_N = N;
    c.cap_m = m;
  }
  if (hist_words > c.sort_hist_cap) {
    ZQ_TRY(grow(&c.sort_hist, hist_words));
    c.sort_hist_cap = hist_words;
  }
  return ZQ_OK;
}

}  // namespace

extern "C" {

const char* zq_status_string(zq_status s) {
  switch (s) {
    case ZQ_OK: return "ok";
    case ZQ_EINVAL: return "invalid argument";
    case ZQ_ENOMEM: return "device allocation failed";
    case ZQ_ECUDA: return "CUDA error";
    case ZQ_ESTATE: return "call out of order";
    case ZQ_ENONFINITE: return "non-finite coordinate";
    case ZQ_WDEGENERATE: return "degenerate node (coincident or collinear beads)";
  }
  return "unknown status";
}

zq_status zq_create(zq_ctx** ctx, int device, void* cuda_stream) {
  if (!ctx) return ZQ_EINVAL;
  *ctx = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return ZQ_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return ZQ_ECUDA;
  zq_ctx* h = new (std::nothrow) zq_ctx();
  if (!h) return ZQ_ENOMEM;
  h->c.device = device;
  h->c.stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaDeviceGetAttribute(&h->c.num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete h;
    return ZQ_ECUDA;
  }
  // Side stream priorities: 0 runs zq_pipeline's downward sweep, which
  // follows the transform build on the step's critical path (highest);
  // 1 runs the early upward sweep beside the build's latency-bound upper
  // heights (lowest); 2 and 3 the default.
  int prio_low = 0, prio_high = 0;
  bool ok = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->c.fork_ev, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < 4 && ok; ++i) {
    const int prio = i == 0 ? prio_high : (i == 1 ? prio_low : 0);
    ok = cudaStreamCreateWithPriority(&h->c.side[i], cudaStreamNonBlocking, prio) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->c.join_ev[i], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    destroy_streams(h->c);
    delete h;
    return ZQ_ECUDA;
  }
  *ctx = h;
  return ZQ_OK;
}

zq_status zq_destroy(zq_ctx* ctx) {
  if (!ctx) return ZQ_EINVAL;
  cudaSetDevice(ctx->c.device);
  cudaStreamSynchronize(ctx->c.stream);
  if (ctx->c.gexec) cudaGraphExecDestroy(ctx->c.gexec);
  ctx->c.gexec = nullptr;
  destroy_streams(ctx->c);
  free_all(ctx->c);
  delete ctx;
  return ZQ_OK;
}

// The tree of m bodies; with schedules, also the segment and bucket
// schedules of the level build and the separate sweeps (the fused step of
// zq_pipeline needs neither; zq_build_transforms makes them when missing).
static zq_status build_tree_impl(zq_ctx* ctx, int64_t m, const int64_t* off, const double* x, const double* y,
                                 const double* z, int32_t level_cut, bool schedules) {
  if (!ctx || !off || !x || !y || !z || m < 1) return ZQ_EINVAL;
  if (level_cut == 0) level_cut = zq::kDefaultCut;
  if (level_cut < 1 || level_cut > zq::kMaxCut) return ZQ_EINVAL;
  if (off[0] != 0) return ZQ_EINVAL;
  int64_t max_big = 0;
  for (int64_t j = 0; j < m; ++j) {
    const int64_t n = off[j + 1] - off[j];
    if (n < 3 || n > INT32_MAX) return ZQ_EINVAL;
    if (n > zq::kSmallSortMax && n > max_big) max_big = n;
  }
  const int64_t N = off[m];
  if (N > zq::kMaxBeads) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  // Same bodies and level cut as the previous tree: reuse the launch plan (no
  // host synchronisation, so the call can be captured in a CUDA graph).
  if (c.have_tree && m == c.m && level_cut == c.cut &&
      std::equal(off, off + m + 1, c.off_h.begin())) {
    c.have_xform = false;
    ZQ_TRY(zq::launch_tree(c, x, y, z, schedules));
    return ZQ_OK;
  }
  const int64_t hist_words = zq::sort_hist_words(max_big);
  ++c.plan_gen;  // a new plan, possibly new buffers: captured steps are stale
  ZQ_TRY(ensure_capacity(c, N, m, hist_words));
  c.N = N;
  c.m = m;
  c.nodes = N - m;
  c.R = 3 * N - 6 * m;
  c.cut = level_cut;
  c.have_tree = false;
  c.have_xform = false;
  c.off_h.assign(off, off + m + 1);
  c.small_bodies.clear();
  c.big_bodies.clear();
  c.max_small = 0;
  {
    std::vector<int32_t> cls[4];
    for (int64_t j = 0; j < m; ++j) {
      const int64_t n = off[j + 1] - off[j];
      if (n <= zq::kSmallSortMax) {
        cls[zq::small_tree_class(n)].push_back((int32_t)j);
        if (n > c.max_small) c.max_small = (int32_t)n;
      } else {
        c.big_bodies.push_back((int32_t)j);
      }
    }
    for (int k = 0; k < 4; ++k) {
      c.small_class_start[k] = (int)c.small_bodies.size();
      c.small_bodies.insert(c.small_bodies.end(), cls[k].begin(), cls[k].end());
    }
    c.small_class_start[4] = (int)c.small_bodies.size();
    // the fused step's blocks: bodies largest first (ties by id), each to
    // the block with the fewest nodes so far; four blocks per SM
    std::vector<int32_t> order((size_t)m);
    for (int64_t j = 0; j < m; ++j) order[(size_t)j] = (int32_t)j;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    c.fused_bins = (int32_t)std::min<int64_t>((int64_t)c.num_sms * 4, m);
    std::vector<std::vector<int32_t>> bins((size_t)c.fused_bins);
    std::vector<std::pair<int64_t, int32_t>> heap;  // (nodes, bin), min-heap
    for (int32_t b = 0; b < c.fused_bins; ++b) heap.push_back({0, b});
    auto later = [](const std::pair<int64_t, int32_t>& x, const std::pair<int64_t, int32_t>& y) { return x > y; };
    for (const int32_t j : order) {
      std::pop_heap(heap.begin(), heap.end(), later);
      auto& top = heap.back();
      bins[(size_t)top.second].push_back(j);
      top.first += off[j + 1] - off[j] - 1;
      std::push_heap(heap.begin(), heap.end(), later);
    }
    c.fused_bins_h.assign(1, 0);
    for (const auto& bin : bins) c.fused_bins_h.push_back(c.fused_bins_h.back() + (int32_t)bin.size());
    for (const auto& bin : bins) c.fused_bins_h.insert(c.fused_bins_h.end(), bin.begin(), bin.end());
  }
  ZQ_CUDA_TRY(cudaMemcpyAsync(c.off, off, (m + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
  if (!c.small_bodies.empty())
    ZQ_CUDA_TRY(cudaMemcpyAsync(c.small_d, c.small_bodies.data(), c.small_bodies.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, c.stream));
  ZQ_CUDA_TRY(cudaMemcpyAsync(c.fused_bin_start, c.fused_bins_h.data(), (c.fused_bins + 1) * sizeof(int32_t),
                              cudaMemcpyHostToDevice, c.stream));
  ZQ_CUDA_TRY(cudaMemcpyAsync(c.fused_bin_bodies, c.fused_bins_h.data() + c.fused_bins + 1, m * sizeof(int32_t),
                              cudaMemcpyHostToDevice, c.stream));
  // the host vectors are read by the copies above: keep them alive until then
  ZQ_CUDA_TRY(cudaStreamSynchronize(c.stream));
  ZQ_TRY(zq::launch_bead_body(c));
  ZQ_TRY(zq::launch_tree(c, x, y, z, schedules));
  c.have_tree = true;
  return ZQ_OK;
}

zq_status zq_build_tree_batched(zq_ctx* ctx, int64_t m, const int64_t* off, const double* x,
                                const double* y, const double* z, int32_t level_cut) {
  return build_tree_impl(ctx, m, off, x, y, z, level_cut, true);
}

zq_status zq_build_tree(zq_ctx* ctx, int64_t n, const double* x, const double* y, const double* z,
                        int32_t level_cut) {
  const int64_t off[2] = {0, n};
  return zq_build_tree_batched(ctx, 1, off, x, y, z, level_cut);
}

zq_status zq_build_transforms(zq_ctx* ctx, const double* x, const double* y, const double* z) {
  if (!ctx || !x || !y || !z) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  if (!c.have_tree) return ZQ_ESTATE;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  if (!c.have_sched) ZQ_TRY(zq::launch_schedules(c));  // the tree came from a fused step
  ZQ_TRY(zq::launch_build(c, x, y, z, 3));
  c.have_xform = true;
  c.have64 = c.have32 = true;
  return ZQ_OK;
}

zq_status zq_apply_Q(zq_ctx* ctx, zq_prec prec, int64_t k, const void* v, int64_t ldv, void* out,
                     int64_t ldo) {
  if (!ctx || !v || !out || k < 1) return ZQ_EINVAL;
  if (prec != ZQ_FP32 && prec != ZQ_FP64) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  if (!c.have_xform || !(prec == ZQ_FP64 ? c.have64 : c.have32)) return ZQ_ESTATE;
  if (ldv < 3 * c.N || ldo < c.R) return ZQ_EINVAL;
  const size_t es = prec == ZQ_FP64 ? sizeof(double) : sizeof(float);
  for (int64_t col = 0; col < k; ++col) {
    const char* vi = static_cast<const char*>(v) + (size_t)col * ldv * es;
    char* oi = static_cast<char*>(out) + (size_t)col * ldo * es;
    ZQ_TRY(zq::launch_apply_Q(c, prec, vi, ldv, oi));
  }
  return ZQ_OK;
}

zq_status zq_apply_Q_full(zq_ctx* ctx, zq_prec prec, const void* v, void* out, void* root) {
  if (!ctx || !v || !out || !root) return ZQ_EINVAL;
  if (prec != ZQ_FP32 && prec != ZQ_FP64) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  if (!c.have_xform || !(prec == ZQ_FP64 ? c.have64 : c.have32)) return ZQ_ESTATE;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  return zq::launch_apply_Q(c, prec, v, 3 * c.N, out, root);
}

zq_status zq_apply_QT_full(zq_ctx* ctx, zq_prec prec, const void* w, const void* root, void* out) {
  if (!ctx || !w || !out || !root) return ZQ_EINVAL;
  if (prec != ZQ_FP32 && prec != ZQ_FP64) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  if (!c.have_xform || !(prec == ZQ_FP64 ? c.have64 : c.have32)) return ZQ_ESTATE;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  return zq::launch_apply_QT(c, prec, w, out, 3 * c.N, root);
}

zq_status zq_qgen_nnz(zq_ctx* ctx, int64_t* nnz) {
  if (!ctx || !nnz) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  if (!c.have_tree) return ZQ_ESTATE;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  return zq::launch_qgen_nnz(c, nnz);
}

zq_status zq_qgen(zq_ctx* ctx, zq_prec prec, int64_t* row_ptr, int32_t* col, void* val, void* uz) {
  if (!ctx || !row_ptr || !col || !val) return ZQ_EINVAL;
  if (prec != ZQ_FP32 && prec != ZQ_FP64) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  if (!c.have_xform || !(prec == ZQ_FP64 ? c.have64 : c.have32)) return ZQ_ESTATE;
  if (3 * c.N > INT32_MAX) return ZQ_EINVAL;  // column indices are int32
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  return zq::launch_qgen(c, prec, row_ptr, col, val, uz);
}

zq_status zq_reserve_block(zq_ctx* ctx, zq_prec prec, int64_t k_max) {
  if (!ctx || k_max < 1) return ZQ_EINVAL;
  if (prec < ZQ_FP64 || prec > ZQ_BF16_TC) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  if (!c.have_tree) return ZQ_ESTATE;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  const int64_t es = prec == ZQ_FP64 ? 8 : 4;
  const int64_t bytes = c.nodes * 6 * k_max * es;
  if (bytes > c.xblk_bytes) {
    if (c.xblk) cudaFree(c.xblk);
    c.xblk = nullptr;
    c.xblk_bytes = 0;
    if (cudaMalloc(&c.xblk, (size_t)bytes) != cudaSuccess) {
      c.xblk = nullptr;
      return ZQ_ENOMEM;
    }
    c.xblk_bytes = bytes;
  }
  return ZQ_OK;
}

static zq_status apply_block(zq_ctx* ctx, bool up, zq_prec prec, int64_t k, const void* in, void* out) {
  if (!ctx || !in || !out || k < 1 || k > (1 << 20)) return ZQ_EINVAL;
  if (prec < ZQ_FP64 || prec > ZQ_BF16_TC) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  if (!c.have_xform || !(prec == ZQ_FP64 ? c.have64 : c.have32)) return ZQ_ESTATE;
  const int64_t es = prec == ZQ_FP64 ? 8 : 4;
  if (c.nodes * 6 * k * es > c.xblk_bytes) return ZQ_ESTATE;
  return zq::launch_apply_block(c, up, prec, k, in, out);
}

zq_status zq_apply_Q_block(zq_ctx* ctx, zq_prec prec, int64_t k, const void* V, void* out) {
  return apply_block(ctx, true, prec, k, V, out);
}

zq_status zq_apply_QT_block(zq_ctx* ctx, zq_prec prec, int64_t k, const void* W, void* out) {
  return apply_block(ctx, false, prec, k, W, out);
}

zq_status zq_apply_QT(zq_ctx* ctx, zq_prec prec, int64_t k, const void* w, int64_t ldw, void* out,
                      int64_t ldo) {
  if (!ctx || !w || !out || k < 1) return ZQ_EINVAL;
  if (prec != ZQ_FP32 && prec != ZQ_FP64) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  if (!c.have_xform || !(prec == ZQ_FP64 ? c.have64 : c.have32)) return ZQ_ESTATE;
  if (ldw < c.R || ldo < 3 * c.N) return ZQ_EINVAL;
  const size_t es = prec == ZQ_FP64 ? sizeof(double) : sizeof(float);
  for (int64_t col = 0; col < k; ++col) {
    const char* wi = static_cast<const char*>(w) + (size_t)col * ldw * es;
    char* oi = static_cast<char*>(out) + (size_t)col * ldo * es;
    ZQ_TRY(zq::launch_apply_QT(c, prec, wi, oi, ldo));
  }
  return ZQ_OK;
}

// Q~ v and/or Q~^T w (null pairs skipped), with optional per-body rotations.
// With both, the two products are independent: Q~^T w runs on a side
// stream (with its own scratch) while Q~ v runs on the context stream,
// joined after.
static zq_status apply_two(zq_ctx* ctx, zq_prec prec, const double* rot, const void* v, void* qv, const void* w,
                           void* qtw) {
  if (!ctx) return ZQ_EINVAL;
  if ((v == nullptr) != (qv == nullptr) || (w == nullptr) != (qtw == nullptr) || (!v && !w)) return ZQ_EINVAL;
  if (prec != ZQ_FP32 && prec != ZQ_FP64) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  if (!c.have_xform || !(prec == ZQ_FP64 ? c.have64 : c.have32)) return ZQ_ESTATE;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  if (!v) return zq::launch_apply_QT(c, prec, w, qtw, 3 * c.N, nullptr, rot);
  if (!w) return zq::launch_apply_Q(c, prec, v, 3 * c.N, qv, nullptr, rot);
  ZQ_CUDA_TRY(cudaEventRecord(c.fork_ev, c.stream));
  ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[0], c.fork_ev, 0));
  ZQ_TRY(zq::launch_apply_Q(c, prec, v, 3 * c.N, qv, nullptr, rot));
  cudaStream_t main = c.stream;
  std::swap(c.x32, c.x32b);
  std::swap(c.x64, c.x64b);
  c.stream = c.side[0];
  const zq_status st = zq::launch_apply_QT(c, prec, w, qtw, 3 * c.N, nullptr, rot);
  c.stream = main;
  std::swap(c.x32, c.x32b);
  std::swap(c.x64, c.x64b);
  ZQ_TRY(st);
  ZQ_CUDA_TRY(cudaEventRecord(c.join_ev[0], c.side[0]));
  ZQ_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev[0], 0));
  return ZQ_OK;
}

zq_status zq_apply_pair(zq_ctx* ctx, zq_prec prec, const void* v, void* qv, const void* w, void* qtw) {
  if (!v || !w) return ZQ_EINVAL;
  return apply_two(ctx, prec, nullptr, v, qv, w, qtw);
}

zq_status zq_apply_rotated(zq_ctx* ctx, zq_prec prec, const double* R, const void* v, void* qv, const void* w,
                           void* qtw) {
  if (!R) return ZQ_EINVAL;
  return apply_two(ctx, prec, R, v, qv, w, qtw);
}

// zq_pipeline with both products and the vectors in the caller's order:
// 0 = the sweeps gather v and scatter Q~^T w through perm themselves;
// 1 = v is gathered into the tree's order on a side stream next to the
// transform build, so the upward sweep reads contiguous planes;
// 2 = as 1, and the downward sweep also writes in tree order, brought back to
// the caller's order by a separate gather after it (through the inverse
// permutation that the first gather writes).
constexpr int kPipeOrder = 2;

// scratch: v in tree order, Q~^T w in tree order (mode 2), inverse permutation
static int64_t pipe_order_planes(int64_t N, size_t es) {
  return (kPipeOrder == 2 ? 2 : 1) * 3 * N * (int64_t)es;
}

static int64_t pipe_order_bytes(int64_t N, size_t es) {
  return pipe_order_planes(N, es) + N * (int64_t)sizeof(int32_t);
}

static bool pipe_reorders(const Ctx& c, const void* v, const void* w) {
  return kPipeOrder > 0 && v && w && !c.tree_order && !c.fused_step;
}

// Every body small enough for the fused step (one thread block per body).
static bool bodies_fit_fused(int64_t m, const int64_t* off) {
  for (int64_t j = 0; j < m; ++j)
    if (off[j + 1] - off[j] > zq::kSmallSortMax) return false;
  return true;
}

static zq_status pipeline_body(zq_ctx* ctx, zq_prec prec, int64_t m, const int64_t* off, const double* x,
                               const double* y, const double* z, const void* v, void* qv, const void* w,
                               void* qtw, int32_t level_cut, int32_t flags) {
  if (!ctx || !off || !x || !y || !z || m < 1) return ZQ_EINVAL;
  if (prec != ZQ_FP32 && prec != ZQ_FP64) return ZQ_EINVAL;
  if ((v == nullptr) != (qv == nullptr) || (w == nullptr) != (qtw == nullptr)) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  c.time_started = false;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  const bool host = (flags & ZQ_HOST_BUFFERS) != 0;
  const bool keep = (flags & ZQ_KEEP_TREE) != 0;
  if (keep && (!c.have_tree || m != c.m || !std::equal(off, off + m + 1, c.off_h.begin())))
    return ZQ_ESTATE;
  const int64_t N = off[m], R = 3 * N - 6 * m;
  const size_t es = prec == ZQ_FP64 ? sizeof(double) : sizeof(float);
  const bool reorder = pipe_reorders(c, v, w);
  if (reorder && pipe_order_bytes(N, es) > c.ord_cap) {
    ++c.plan_gen;
    if (c.ord) cudaFree(c.ord);
    c.ord = nullptr;
    c.ord_cap = 0;
    if (cudaMalloc(&c.ord, (size_t)pipe_order_bytes(N, es)) != cudaSuccess) return ZQ_ENOMEM;
    c.ord_cap = pipe_order_bytes(N, es);
  }
  const double *dx = x, *dy = y, *dz = z;
  const void *dv = v, *dw = w;
  void *dqv = qv, *dqtw = qtw;
  if (host) {
    // staging layout: x y z (N doubles each) | v (3N) | qtw (3N) | w (R) | qv (R)
    const int64_t bytes = 3 * N * 8 + (int64_t)es * (6 * N + 2 * R);
    if (bytes > c.stage_cap) {
      ++c.plan_gen;
      if (c.stage) cudaFree(c.stage);
      c.stage = nullptr;
      c.stage_cap = 0;
      if (cudaMalloc(&c.stage, (size_t)bytes) != cudaSuccess) return ZQ_ENOMEM;
      c.stage_cap = bytes;
    }
    char* p = static_cast<char*>(c.stage);
    double* sx = reinterpret_cast<double*>(p);
    double* sy = sx + N;
    double* sz = sy + N;
    char* sv = reinterpret_cast<char*>(sz + N);
    char* sqtw = sv + 3 * N * es;
    char* sw = sqtw + 3 * N * es;
    char* sqv = sw + R * es;
    // coordinates first on the context stream (the tree needs them); the
    // vectors after them on a side stream, overlapping the tree and the
    // transforms, joined before the sweeps.  Forking after the coordinate
    // copies keeps the vectors from sharing the host link with them (the
    // tree would wait for both).
    ZQ_CUDA_TRY(cudaMemcpyAsync(sx, x, N * 8, cudaMemcpyHostToDevice, c.stream));
    ZQ_CUDA_TRY(cudaMemcpyAsync(sy, y, N * 8, cudaMemcpyHostToDevice, c.stream));
    ZQ_CUDA_TRY(cudaMemcpyAsync(sz, z, N * 8, cudaMemcpyHostToDevice, c.stream));
    ZQ_CUDA_TRY(cudaEventRecord(c.fork_ev, c.stream));
    ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[3], c.fork_ev, 0));
    if (v) ZQ_CUDA_TRY(cudaMemcpyAsync(sv, v, 3 * N * es, cudaMemcpyHostToDevice, c.side[3]));
    if (w) ZQ_CUDA_TRY(cudaMemcpyAsync(sw, w, R * es, cudaMemcpyHostToDevice, c.side[3]));
    ZQ_CUDA_TRY(cudaEventRecord(c.join_ev[3], c.side[3]));
    dx = sx; dy = sy; dz = sz;
    dv = v ? sv : nullptr;
    dw = w ? sw : nullptr;
    dqv = qv ? sqv : nullptr;
    dqtw = qtw ? sqtw : nullptr;
  }
  const bool fused = c.fused_step && bodies_fit_fused(m, off);
  if (!keep) ZQ_TRY(build_tree_impl(ctx, m, off, dx, dy, dz, level_cut, !fused));
  if (fused) {
    // transforms and both products of every body in one launch; the
    // separate products need zq_build_transforms afterwards (other layout)
    if (host) ZQ_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev[3], 0));  // the vectors are in
    ZQ_TRY(zq::launch_fused_step(c, prec, dx, dy, dz, dv, dqv, dw, dqtw));
    c.have_xform = false;
    c.have64 = c.have32 = false;
    if (host) {
      if (qv) ZQ_CUDA_TRY(cudaMemcpyAsync(qv, dqv, R * es, cudaMemcpyDeviceToHost, c.stream));
      if (qtw) ZQ_CUDA_TRY(cudaMemcpyAsync(qtw, dqtw, 3 * N * es, cudaMemcpyDeviceToHost, c.stream));
    }
    return ZQ_OK;
  }
  // v into the tree's order on a side stream, next to the transform build
  // (it needs the tree's perm and, from host buffers, the copied v)
  char* vt = reorder ? static_cast<char*>(c.ord) : nullptr;
  char* qtt = reorder && kPipeOrder == 2 ? vt + 3 * N * es : nullptr;
  int32_t* iperm = reorder ? reinterpret_cast<int32_t*>(vt + pipe_order_planes(N, es)) : nullptr;
  if (reorder) {
    ZQ_CUDA_TRY(cudaEventRecord(c.fork_ev, c.stream));
    ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[2], c.fork_ev, 0));
    if (host) ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[2], c.join_ev[3], 0));
    cudaStream_t main = c.stream;
    c.stream = c.side[2];
    const zq_status st = zq::launch_to_tree(c, prec, dv, vt, iperm);
    c.stream = main;
    ZQ_TRY(st);
    ZQ_CUDA_TRY(cudaEventRecord(c.join_ev[2], c.side[2]));
  }
  // The upward sweep starts early: the segments whose nodes all lie at or
  // below the level cut need only the level launches of the build, so they
  // are swept on a side stream while the nodes above the cut (a few long
  // dependent chains per body) are built; the other segments and the top
  // nodes follow the build.
  const bool early_up = dv != nullptr;
  auto sweep_up_early = [&]() -> zq_status {
    ZQ_CUDA_TRY(cudaEventRecord(c.fork_ev, c.stream));
    ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[1], c.fork_ev, 0));
    if (reorder) ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[1], c.join_ev[2], 0));  // v in tree order
    if (host) ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[1], c.join_ev[3], 0));     // v copied in
    cudaStream_t main = c.stream;
    const bool saved = c.tree_order;
    c.stream = c.side[1];
    c.tree_order = saved || reorder;
    const zq_status st = zq::launch_apply_Q(c, prec, reorder ? vt : dv, 3 * N, dqv, nullptr, nullptr, 1);
    c.tree_order = saved;
    c.stream = main;
    ZQ_TRY(st);
    ZQ_CUDA_TRY(cudaEventRecord(c.join_ev[1], c.side[1]));
    return ZQ_OK;
  };
  // the two sweeps of the step, each on the stream current at its call
  auto sweep_up = [&]() -> zq_status {
    if (reorder) ZQ_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev[2], 0));
    if (early_up) ZQ_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev[1], 0));
    const bool saved = c.tree_order;
    c.tree_order = saved || reorder;
    const zq_status st =
        zq::launch_apply_Q(c, prec, reorder ? vt : dv, 3 * N, dqv, nullptr, nullptr, early_up ? 2 : 0);
    c.tree_order = saved;
    return st;
  };
  auto sweep_down = [&]() -> zq_status {
    const bool saved = c.tree_order;
    c.tree_order = saved || qtt != nullptr;
    zq_status st = zq::launch_apply_QT(c, prec, dw, qtt ? qtt : dqtw, 3 * N);
    c.tree_order = saved;
    if (st == ZQ_OK && qtt) {
      // the inverse permutation comes from the gather into tree order
      ZQ_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev[2], 0));
      st = zq::launch_from_tree(c, prec, qtt, dqtw, iperm);
    }
    return st;
  };
  // only the records of the precision the sweeps use
  if (early_up) ZQ_TRY(zq::launch_build(c, dx, dy, dz, prec == ZQ_FP64 ? 1 : 2, sweep_up_early));
  else ZQ_TRY(zq::launch_build(c, dx, dy, dz, prec == ZQ_FP64 ? 1 : 2));
  c.have_xform = true;
  c.have64 = prec == ZQ_FP64;
  c.have32 = prec == ZQ_FP32;
  if (host) ZQ_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev[3], 0));  // the vectors are in
  if (dv && dw && host) {
    // host buffers: the sweeps one after the other (together they take as
    // long as run concurrently), so that qv goes back over the host link
    // while Q~^T w runs instead of both results going back at the end
    ZQ_TRY(sweep_up());
    ZQ_CUDA_TRY(cudaEventRecord(c.fork_ev, c.stream));
    ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[3], c.fork_ev, 0));
    ZQ_CUDA_TRY(cudaMemcpyAsync(qv, dqv, R * es, cudaMemcpyDeviceToHost, c.side[3]));
    ZQ_CUDA_TRY(cudaEventRecord(c.join_ev[3], c.side[3]));
    ZQ_TRY(sweep_down());
    ZQ_CUDA_TRY(cudaMemcpyAsync(qtw, dqtw, 3 * N * es, cudaMemcpyDeviceToHost, c.stream));
    ZQ_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev[3], 0));
  } else if (dv && dw) {
    // Q~v on the context stream, Q~^T w concurrently on a side stream
    ZQ_CUDA_TRY(cudaEventRecord(c.fork_ev, c.stream));
    ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[0], c.fork_ev, 0));
    ZQ_TRY(sweep_up());
    cudaStream_t main = c.stream;
    std::swap(c.x32, c.x32b);
    std::swap(c.x64, c.x64b);
    c.stream = c.side[0];
    const zq_status st = sweep_down();
    c.stream = main;
    std::swap(c.x32, c.x32b);
    std::swap(c.x64, c.x64b);
    ZQ_TRY(st);
    ZQ_CUDA_TRY(cudaEventRecord(c.join_ev[0], c.side[0]));
    ZQ_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev[0], 0));
  } else {
    if (dv) ZQ_TRY(sweep_up());  // joins the early part of the sweep
    if (dw) ZQ_TRY(zq_apply_QT(ctx, prec, 1, dw, R, dqtw, 3 * N));
    if (host) {
      if (qv) ZQ_CUDA_TRY(cudaMemcpyAsync(qv, dqv, R * es, cudaMemcpyDeviceToHost, c.stream));
      if (qtw) ZQ_CUDA_TRY(cudaMemcpyAsync(qtw, dqtw, 3 * N * es, cudaMemcpyDeviceToHost, c.stream));
    }
  }
  return ZQ_OK;
}

zq_status zq_time_kernel(zq_ctx* ctx, const char* name, void* start_event, void* stop_event) {
  if (!ctx) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  if (!name) {
    c.time_name[0] = 0;
    c.time_ev0 = c.time_ev1 = nullptr;
    return ZQ_OK;
  }
  if (!start_event || !stop_event || std::strlen(name) >= sizeof(c.time_name)) return ZQ_EINVAL;
  std::strncpy(c.time_name, name, sizeof(c.time_name) - 1);
  c.time_ev0 = static_cast<cudaEvent_t>(start_event);
  c.time_ev1 = static_cast<cudaEvent_t>(stop_event);
  return ZQ_OK;
}

zq_status zq_set_vector_order(zq_ctx* ctx, zq_vector_order order) {
  if (!ctx || (order != ZQ_ORDER_CALLER && order != ZQ_ORDER_TREE)) return ZQ_EINVAL;
  ctx->c.tree_order = order == ZQ_ORDER_TREE;
  return ZQ_OK;
}

zq_status zq_set_step_schedule(zq_ctx* ctx, zq_step_schedule schedule) {
  if (!ctx || (schedule != ZQ_STEP_LEVELS && schedule != ZQ_STEP_FUSED)) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  if (c.fused_step != (schedule == ZQ_STEP_FUSED)) ++c.plan_gen;  // a captured step is stale
  c.fused_step = schedule == ZQ_STEP_FUSED;
  return ZQ_OK;
}

zq_status zq_set_build_arith(zq_ctx* ctx, zq_build_arith arith) {
  if (!ctx || (arith != ZQ_BUILD_DD && arith != ZQ_BUILD_FP64)) return ZQ_EINVAL;
  ctx->c.build_dd = arith == ZQ_BUILD_DD;
  return ZQ_OK;
}

zq_status zq_launch_count(const zq_ctx* ctx, int64_t* launches) {
  if (!ctx || !launches) return ZQ_EINVAL;
  *launches = ctx->c.launches;
  return ZQ_OK;
}

zq_status zq_sync(zq_ctx* ctx) {
  if (!ctx) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  ZQ_CUDA_TRY(cudaStreamSynchronize(c.stream));
  ZQ_CUDA_TRY(cudaGetLastError());
  if (!c.counters) return ZQ_OK;
  int32_t err = 0;
  ZQ_CUDA_TRY(cudaMemcpy(&err, c.counters + 2, sizeof(int32_t), cudaMemcpyDeviceToHost));
  ZQ_CUDA_TRY(cudaMemset(c.counters + 2, 0, sizeof(int32_t)));
  if (err & zq::kErrNonFinite) return ZQ_ENONFINITE;
  if (err & zq::kErrDegenerate) return ZQ_WDEGENERATE;
  return ZQ_OK;
}

zq_status zq_sizes(const zq_ctx* ctx, int64_t* N, int64_t* m, int64_t* R, int64_t* nodes) {
  if (!ctx) return ZQ_EINVAL;
  const Ctx& c = ctx->c;
  if (!c.have_tree) return ZQ_ESTATE;
  if (N) *N = c.N;
  if (m) *m = c.m;
  if (R) *R = c.R;
  if (nodes) *nodes = c.nodes;
  return ZQ_OK;
}

zq_status zq_get_tree(zq_ctx* ctx, int32_t* perm, int32_t* left, int32_t* right, int32_t* first,
                      int32_t* count, int32_t* height, int32_t* roff) {
  if (!ctx) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  if (!c.have_tree) return ZQ_ESTATE;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  ZQ_CUDA_TRY(cudaStreamSynchronize(c.stream));
  const size_t nb = (size_t)c.nodes * sizeof(int32_t);
  if (perm) ZQ_CUDA_TRY(cudaMemcpy(perm, c.perm, c.N * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (left) ZQ_CUDA_TRY(cudaMemcpy(left, c.cl, nb, cudaMemcpyDeviceToHost));
  if (right) ZQ_CUDA_TRY(cudaMemcpy(right, c.cr, nb, cudaMemcpyDeviceToHost));
  if (first) ZQ_CUDA_TRY(cudaMemcpy(first, c.first, nb, cudaMemcpyDeviceToHost));
  if (count) ZQ_CUDA_TRY(cudaMemcpy(count, c.cnt, nb, cudaMemcpyDeviceToHost));
  if (roff) ZQ_CUDA_TRY(cudaMemcpy(roff, c.roff, nb, cudaMemcpyDeviceToHost));
  if (height) {
    std::vector<uint8_t> h((size_t)c.nodes);
    ZQ_CUDA_TRY(cudaMemcpy(h.data(), c.height, (size_t)c.nodes, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < c.nodes; ++i) height[i] = h[(size_t)i];
  }
  return ZQ_OK;
}

// Row offsets of the two layouts of Q~ (Sec. 3).  In-order: a running sum
// of the node sizes by id.  Pre-order, the recursive [Residue_p;
// diag(Q~_x, Q~_y)]: a depth-first walk from each body's root that numbers
// a node before its left subtree and the left subtree before the right one.
zq_status zq_residue_offsets(int64_t m, const int64_t* off, const int32_t* left, const int32_t* right,
                             zq_row_order order, int64_t* node_off, int64_t* body_off) {
  if (m < 1 || !off || !left || !right || !node_off) return ZQ_EINVAL;
  if (order != ZQ_ROWS_INORDER && order != ZQ_ROWS_PREORDER) return ZQ_EINVAL;
  if (off[0] != 0) return ZQ_EINVAL;
  for (int64_t j = 0; j < m; ++j)
    if (off[j + 1] - off[j] < 3 || off[j + 1] > zq::kMaxBeads) return ZQ_EINVAL;
  auto rows = [&](int64_t q) -> int64_t { return 3 * ((left[q] >= 0) + (right[q] >= 0)); };
  // every child inside its body, every internal node the child of at most one node
  std::vector<uint8_t> is_child((size_t)(off[m] - m), 0);
  for (int64_t j = 0; j < m; ++j) {
    const int64_t nb = off[j] - j, ne = off[j + 1] - j - 1;
    for (int64_t q = nb; q < ne; ++q) {
      for (const int32_t code : {left[q], right[q]}) {
        if (code >= 0) {
          if (code < nb || code >= ne || code == q || is_child[(size_t)code]) return ZQ_EINVAL;
          is_child[(size_t)code] = 1;
        } else {
          const int64_t pos = -1 - (int64_t)code;
          if (pos < off[j] || pos >= off[j + 1]) return ZQ_EINVAL;
        }
      }
    }
  }
  // one tree per body: a single root from which every node is reached (the
  // walk visits each node once: no node has two parents); the walk is the
  // pre-order numbering, the in-order one is by id
  std::vector<int32_t> stack;
  for (int64_t j = 0; j < m; ++j) {
    const int64_t nb = off[j] - j, ne = off[j + 1] - j - 1;
    const int64_t base = 3 * off[j] - 6 * j;
    int64_t root = -1;
    for (int64_t q = nb; q < ne; ++q) {
      if (is_child[(size_t)q]) continue;
      if (root >= 0) return ZQ_EINVAL;  // two roots
      root = q;
    }
    if (root < 0) return ZQ_EINVAL;
    int64_t acc = base, reached = 0;
    stack.assign(1, (int32_t)root);
    while (!stack.empty()) {
      const int32_t q = stack.back();
      stack.pop_back();
      if (order == ZQ_ROWS_PREORDER) node_off[q] = acc;
      acc += rows(q);
      ++reached;
      if (right[q] >= 0) stack.push_back(right[q]);
      if (left[q] >= 0) stack.push_back(left[q]);  // the left subtree first
    }
    if (reached != ne - nb) return ZQ_EINVAL;
    if (order == ZQ_ROWS_INORDER) {
      acc = base;
      for (int64_t q = nb; q < ne; ++q) {
        node_off[q] = acc;
        acc += rows(q);
      }
    }
  }
  if (body_off)
    for (int64_t j = 0; j <= m; ++j) body_off[j] = 3 * off[j] - 6 * j;
  return ZQ_OK;
}

zq_status zq_get_residue_offsets(zq_ctx* ctx, zq_row_order order, int64_t* node_off, int64_t* body_off) {
  if (!ctx || !node_off) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  if (!c.have_tree) return ZQ_ESTATE;
  std::vector<int32_t> l((size_t)c.nodes), r((size_t)c.nodes);
  ZQ_TRY(zq_get_tree(ctx, nullptr, l.data(), r.data(), nullptr, nullptr, nullptr, nullptr));
  return zq_residue_offsets(c.m, c.off_h.data(), l.data(), r.data(), order, node_off, body_off);
}

zq_status zq_get_nodes(zq_ctx* ctx, double* centroid, double* T22) {
  if (!ctx) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  if (!c.have_xform) return ZQ_ESTATE;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  ZQ_CUDA_TRY(cudaStreamSynchronize(c.stream));
  std::vector<double> st((size_t)c.nodes * zq::kState);
  std::vector<int32_t> slot((size_t)c.nodes);
  ZQ_CUDA_TRY(cudaMemcpy(st.data(), c.st64, st.size() * sizeof(double), cudaMemcpyDeviceToHost));
  ZQ_CUDA_TRY(cudaMemcpy(slot.data(), c.slot_of, slot.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
  for (int64_t q = 0; q < c.nodes; ++q) {
    const double* s = st.data() + (size_t)slot[(size_t)q] * zq::kState;
    double v[9];
    for (int a = 0; a < 9; ++a) {
      if (c.st_is_dd && a >= 3) {  // T22: a double-single pair in the 8-byte word
        float hl[2];
        std::memcpy(hl, s + a, sizeof(hl));
        v[a] = (double)hl[0] + (double)hl[1];
      } else {
        v[a] = s[a];
      }
    }
    if (centroid)
      for (int a = 0; a < 3; ++a) centroid[3 * q + a] = v[a];
    if (T22)
      for (int a = 0; a < 6; ++a) T22[6 * q + a] = v[3 + a];
  }
  return ZQ_OK;
}

zq_status zq_get_records(zq_ctx* ctx, double* rec) {
  if (!ctx || !rec) return ZQ_EINVAL;
  Ctx& c = ctx->c;
  if (!c.have_xform || !c.have64) return ZQ_ESTATE;
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  ZQ_CUDA_TRY(cudaStreamSynchronize(c.stream));
  const size_t nodes = (size_t)c.nodes;
  std::vector<uint32_t> prw(nodes + 1);
  std::vector<int32_t> pnode(nodes);
  std::vector<int2> pc(nodes);
  ZQ_CUDA_TRY(cudaMemcpy(prw.data(), c.prw, (nodes + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  ZQ_CUDA_TRY(cudaMemcpy(pnode.data(), c.pnode, nodes * sizeof(int32_t), cudaMemcpyDeviceToHost));
  ZQ_CUDA_TRY(cudaMemcpy(pc.data(), c.pc, nodes * sizeof(int2), cudaMemcpyDeviceToHost));
  std::vector<double> cr((size_t)prw[nodes] * 4);
  ZQ_CUDA_TRY(cudaMemcpy(cr.data(), c.rec64, cr.size() * sizeof(double), cudaMemcpyDeviceToHost));
  // compact (by position) -> dense documented layout (by node id)
  static const int rows6[3][3] = {{4, 5, -1}, {3, 4, 5}, {3, 4, 5}};
  static const int rows9[3][6] = {{3, 7, 8, -1, -1, -1}, {3, 4, 6, 7, 8, -1}, {3, 4, 5, 6, 7, 8}};
  static const int off6[3] = {5, 7, 10}, off9[3] = {5, 8, 13};
  for (size_t p = 0; p < nodes; ++p) {
    const int type = (pc[p].x >= 0) + (pc[p].y >= 0);
    const double* r = cr.data() + (size_t)prw[p] * 4;
    double* d = rec + (size_t)pnode[p] * zq::kRec;
    for (int i = 0; i < zq::kRec; ++i) d[i] = 0.0;
    d[0] = r[0];
    d[1] = r[1];
    if (type == 0) {
      for (int i = 0; i < 9; ++i) d[5 + i] = r[2 + i];
      continue;
    }
    const int k = type == 1 ? 6 : 9;
    for (int j = 0; j < 3; ++j) d[2 + j] = r[2 + j];
    int tail_at = 5;
    for (int j = 0; j < 3; ++j) {
      const int nv = type == 1 ? (j == 0 ? 2 : 3) : (j == 0 ? 3 : (j == 1 ? 5 : 6));
      for (int i = 0; i < nv; ++i) {
        const int row = type == 1 ? rows6[j][i] : rows9[j][i];
        d[tail_at + row - j - 1] = r[(type == 1 ? off6[j] : off9[j]) + i];
      }
      tail_at += k - 1 - j;
    }
  }
  return ZQ_OK;
}

}  // extern "C"

// ZQ_GRAPH: the step is captured once as a CUDA graph and replayed while
// the arguments and the plan are unchanged.  A call that would plan (new
// bodies, level cut or buffers) runs directly; the next one captures.
zq_status zq_pipeline(zq_ctx* ctx, zq_prec prec, int64_t m, const int64_t* off, const double* x,
                      const double* y, const double* z, const void* v, void* qv, const void* w,
                      void* qtw, int32_t level_cut, int32_t flags) {
  if (!(flags & ZQ_GRAPH) || !ctx) return pipeline_body(ctx, prec, m, off, x, y, z, v, qv, w, qtw, level_cut, flags);
  flags &= ~ZQ_GRAPH;
  Ctx& c = ctx->c;
  // the legacy default stream cannot be captured
  if (!c.stream || !off || m < 1) return pipeline_body(ctx, prec, m, off, x, y, z, v, qv, w, qtw, level_cut, flags);
  const int32_t cut = level_cut == 0 ? zq::kDefaultCut : level_cut;
  std::vector<uintptr_t> key = {(uintptr_t)prec, (uintptr_t)m, (uintptr_t)cut, (uintptr_t)flags,
                                (uintptr_t)c.build_dd, (uintptr_t)c.tree_order, (uintptr_t)c.fused_step,
                                (uintptr_t)x, (uintptr_t)y,
                                (uintptr_t)z, (uintptr_t)v,
                                (uintptr_t)qv, (uintptr_t)w, (uintptr_t)qtw};
  key.insert(key.end(), off, off + m + 1);
  // the kernel-timing hook is part of the captured step
  key.push_back((uintptr_t)c.time_ev0);
  key.push_back((uintptr_t)c.time_ev1);
  for (const char* t = c.time_name; *t; ++t) key.push_back((uintptr_t)(unsigned char)*t);
  ZQ_CUDA_TRY(cudaSetDevice(c.device));
  const bool warm = c.have_tree && m == c.m && cut == c.cut && std::equal(off, off + m + 1, c.off_h.begin());
  const int64_t N = off[m], R = 3 * N - 6 * m;
  const int64_t stage_bytes = 3 * N * 8 + (int64_t)(prec == ZQ_FP64 ? 8 : 4) * (6 * N + 2 * R);
  const bool staged = (!(flags & ZQ_HOST_BUFFERS) || stage_bytes <= c.stage_cap) &&
                      (!pipe_reorders(c, v, w) || pipe_order_bytes(N, prec == ZQ_FP64 ? 8 : 4) <= c.ord_cap);
  key.push_back((uintptr_t)c.plan_gen);
  if (c.gexec && warm && staged && key == c.gkey) {
    c.time_started = false;
    ZQ_CUDA_TRY(cudaGraphLaunch(c.gexec, c.stream));
    c.launches += c.glaunches;
    c.have_xform = true;
    c.have64 = prec == ZQ_FP64;
    c.have32 = prec == ZQ_FP32;
    return ZQ_OK;
  }
  if (!warm || !staged) return pipeline_body(ctx, prec, m, off, x, y, z, v, qv, w, qtw, level_cut, flags);
  // capture this call's work (nothing runs until the launch below)
  ZQ_CUDA_TRY(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
  const int64_t l0 = c.launches;
  const zq_status st = pipeline_body(ctx, prec, m, off, x, y, z, v, qv, w, qtw, level_cut, flags);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c.stream, &g);
  if (st != ZQ_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != ZQ_OK ? st : ZQ_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return ZQ_ECUDA;
  if (c.gexec) cudaGraphExecDestroy(c.gexec);
  c.gexec = ex;
  c.gkey = key;
  c.glaunches = c.launches - l0;
  ZQ_CUDA_TRY(cudaGraphLaunch(c.gexec, c.stream));
  return ZQ_OK;
}
