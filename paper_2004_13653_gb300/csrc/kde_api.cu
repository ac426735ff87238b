// C ABI entry points: argument validation, workspace ownership, host-buffer
// staging, path dispatch and error reporting.  Every arithmetic step runs in
// the kernels of the other translation units.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "kde_internal.cuh"

namespace kde {

std::atomic<int64_t> g_launches{0};
void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {

thread_local char g_err[512] = "";
// the stream kde_grid() runs on, per calling thread (kde_set_stream)
thread_local void* g_plain_stream = nullptr;

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(KDE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define KDE_CUDA(call, what)                 \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// ------------------------------------------------------------- workspace

constexpr int kMaxDevices = 64;
std::mutex g_ws_mu;
void* g_ws_ptr[kMaxDevices] = {};
size_t g_ws_bytes[kMaxDevices] = {};

// Library-owned workspace of at least `need` bytes on the current device.
// Growing it frees the old block (cudaFree waits for the device to idle).
int library_workspace(size_t need, void** out) {
  int dev = 0;
  KDE_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(KDE_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_ws_mu);
  if (g_ws_bytes[dev] < need) {
    if (g_ws_ptr[dev]) {
      cudaFree(g_ws_ptr[dev]);
      g_ws_ptr[dev] = nullptr;
      g_ws_bytes[dev] = 0;
    }
    size_t bytes = need + need / 4;
    bytes = (bytes + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(KDE_ENOMEM, "cudaMalloc of %zu workspace bytes failed: %s", bytes,
                  cudaGetErrorString(e));
    }
    g_ws_ptr[dev] = p;
    g_ws_bytes[dev] = bytes;
  }
  *out = g_ws_ptr[dev];
  return KDE_OK;
}

// A second stream per device, at the lowest priority, for work that overlaps
// the tensor-core contraction (created on first use, kept until release).
cudaStream_t g_side[kMaxDevices] = {};

int side_stream(cudaStream_t* out) {
  int dev = 0;
  KDE_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(KDE_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_ws_mu);
  if (!g_side[dev]) {
    int least = 0, greatest = 0;
    KDE_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priority range");
    KDE_CUDA(cudaStreamCreateWithPriority(&g_side[dev], cudaStreamNonBlocking, least),
             "create the side stream");
  }
  *out = g_side[dev];
  return KDE_OK;
}

// 0: device or managed memory, 1: host memory (pinned or pageable)
int memory_kind(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 0 : 1;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// The radial Gaussian is the product Gaussian (exp(-|u|^2/2) factorises).
int kid_of(const kde_args* a) {
  return a->kernel_id == kRadial + KDE_GAUSSIAN ? KDE_GAUSSIAN : a->kernel_id;
}

int validate(const kde_args* a, const kde_opts* o) {
  if (!a) return fail(KDE_EINVAL, "args is NULL");
  if (a->n < 0) return fail(KDE_EINVAL, "n = %lld is negative", (long long)a->n);
  if (a->n > 0 && !a->points) return fail(KDE_EINVAL, "points is NULL with n > 0");
  if (!a->out) return fail(KDE_EINVAL, "out is NULL");
  if (a->nx <= 0 || a->ny <= 0) return fail(KDE_EINVAL, "grid %d x %d is empty", a->nx, a->ny);
  if ((int64_t)a->nx * (int64_t)a->ny >= (int64_t)1 << 31)
    return fail(KDE_EINVAL, "grid %d x %d has 2^31 cells or more", a->nx, a->ny);
  if (!(a->cell > 0) || !isfinite(a->cell)) return fail(KDE_EINVAL, "cell must be positive and finite");
  if (!(a->h > 0) || !isfinite(a->h)) return fail(KDE_EINVAL, "h must be positive and finite");
  if (!isfinite(a->origin_x) || !isfinite(a->origin_y))
    return fail(KDE_EINVAL, "grid origin must be finite");
  if (a->kernel_id < 0 || a->kernel_id > 15)
    return fail(KDE_EINVAL, "kernel_id %d is neither a Table 1 kernel (0..7) nor a radial one (8..15)",
                a->kernel_id);
  if (a->n > ((int64_t)1 << 31))
    return fail(KDE_EINVAL, "n = %lld exceeds 2^31 points per instance", (long long)a->n);
  // the kernels read points as double2 and write out as float
  if (a->points && (reinterpret_cast<uintptr_t>(a->points) & 15))
    return fail(KDE_EINVAL, "points must be 16-byte aligned");
  if (a->weights && (reinterpret_cast<uintptr_t>(a->weights) & 3))
    return fail(KDE_EINVAL, "weights must be 4-byte aligned");
  if (reinterpret_cast<uintptr_t>(a->out) & 3) return fail(KDE_EINVAL, "out must be 4-byte aligned");
  if (o) {
    if (o->path < KDE_PATH_AUTO || o->path > KDE_PATH_CUTOFF)
      return fail(KDE_EINVAL, "unknown path %d", o->path);
    if ((o->path == KDE_PATH_TC_FP16 || o->path == KDE_PATH_TC_SPLIT16) &&
        kid_of(a) != KDE_GAUSSIAN)
      return fail(KDE_ENOTSUP, "tensor-core paths need the Gaussian kernel");
    if (o->path == KDE_PATH_CUTOFF && kid_of(a) == KDE_GAUSSIAN)
      return fail(KDE_ENOTSUP, "the cutoff path needs a compact-support kernel");
    if (o->path == KDE_PATH_SIMT_FP32 && kid_of(a) >= kRadial)
      return fail(KDE_ENOTSUP, "radial compact kernels run on the cutoff path");
    if (o->split_k < 0 || o->split_k > 1024) return fail(KDE_EINVAL, "split_k out of range");
    if (o->k_chunk < 0 || (o->k_chunk % 32) != 0 || (o->k_chunk > 0 && o->k_chunk < 64))
      return fail(KDE_EINVAL, "k_chunk must be 0 or a multiple of 32 of at least 64");
    if (o->tile_n != 0 && o->tile_n != 128 && o->tile_n != 256)
      return fail(KDE_EINVAL, "tile_n must be 0, 128 or 256");
    if (o->stage_points != 0 && o->stage_points != 32 && o->stage_points != 64)
      return fail(KDE_EINVAL, "stage_points must be 0, 32 or 64");
    if (o->max_ctas < 0) return fail(KDE_EINVAL, "max_ctas must be >= 0");
    if (o->workspace && o->workspace_bytes == 0)
      return fail(KDE_EINVAL, "workspace given with zero size");
    if ((o->flags & KDE_FLAG_LONLAT) && !(fabs(o->lat0_deg) < 90.0))
      return fail(KDE_EINVAL, "KDE_FLAG_LONLAT needs a standard latitude in (-90, 90)");
  }
  return KDE_OK;
}

int resolve_path(const kde_args* a, const kde_opts* o) {
  int path = o ? o->path : KDE_PATH_AUTO;
  if (path == KDE_PATH_AUTO)
    path = kid_of(a) == KDE_GAUSSIAN ? KDE_PATH_TC_SPLIT16 : KDE_PATH_CUTOFF;
  return path;
}

bool is_tc(int path) { return path == KDE_PATH_TC_FP16 || path == KDE_PATH_TC_SPLIT16; }

// Point-range splits for one persistent tensor-core density: the fewest
// splits whose work items fill the CTAs' waves within ~3%, keeping at least
// 256 points per split.
int choose_tc_splits(int64_t tiles, int ctas, int64_t n_pad) {
  const int64_t max_s = std::max<int64_t>(1, std::min<int64_t>(64, n_pad / 256));
  int best = 1;
  double best_waste = 1e30;
  for (int64_t s = 1; s <= max_s; ++s) {
    const int64_t items = tiles * s;
    const int64_t waves = (items + ctas - 1) / ctas;
    const double waste = (double)(waves * ctas) / (double)items;
    if (waste < best_waste - 0.03) {
      best_waste = waste;
      best = (int)s;
    }
  }
  return best;
}

int sm_count() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  return sms > 0 ? sms : 152;
}

struct InstPlan {
  int path;
  int splits;
  int64_t n_pad, prep_begin;
  size_t off_gxt, off_gyt, off_part, off_run;  // off_run: SIMT running sums
  // tensor-core path: the instance's tile family and accumulator chunk
  int fam, k_chunk, split_req;
  int tiles_m, tiles_n, items;
  int64_t per_split;
  // cutoff path, and the bin sort of block-sparse tensor-core instances
  CutoffGeom geo;
  int bin_begin;
  int obx, oby, out_begin;  // cutoff: output blocks of kCutoffBin cells, first CTA
  int64_t cut_begin;
  int tile_begin;  // block-sparse: first tile in the batch's tile numbering
};

// Block-sparse skipping: reach of a Gaussian operand in prepared units
// (h sqrt(2 ln 2)).  2^(15 - 6.45^2) < 2^-26.6, which rounds to zero in FP16
// (hi and lo alike); the margin over the exact bound sqrt(41) = 6.403 covers
// the FP32 rounding of the offsets and of ex2.approx.
constexpr double kSparseReach = 6.45;

// The adjoint takes the tensor-core contractions when the window kernel's
// cells per point exceed this fraction of the grid padded to 256-cell tiles
// (measured on 1M points x 1024^2: the contractions take 6.2 ms at every h,
// the window 5.7 ms at h = 5.1 cells and 26 ms at h = 8.2 cells, about 1 ns
// per window cell and point).
constexpr double kAdjointTcRatio = 0.006;

// Tensor-core instances that share a tile shape and pipeline stage: one
// persistent launch over their work items.
struct TcFamily {
  TcPlan plan;
  std::vector<int> order;  // instances, most expensive items first
  int items = 0;
  int tab_begin = 0;       // first entry of the family in the TC table
  // CTA-pair batches: each pair's items (offsets, then item indices), from a
  // longest-processing-time-first assignment; empty = round robin
  std::vector<uint32_t> sched;
  size_t off_sched = 0;
};

// Longest processing time first: the items, longest first, each to the CTA
// pair with the least work so far; returns offsets[clusters + 1] followed by
// the item indices of each pair in the order it takes them.  cost[i] is the
// item's length in pipeline stages plus a fixed cost for its final drain.
std::vector<uint32_t> lpt_schedule(const std::vector<int64_t>& cost, int clusters) {
  const int n = (int)cost.size();
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<std::vector<uint32_t>> per(clusters);
  std::vector<std::pair<int64_t, int>> heap;  // (load, pair), smallest load on top
  for (int c = 0; c < clusters; ++c) heap.push_back({0, c});
  auto cmp = [](const std::pair<int64_t, int>& a, const std::pair<int64_t, int>& b) {
    return a.first != b.first ? a.first > b.first : a.second > b.second;
  };
  std::make_heap(heap.begin(), heap.end(), cmp);
  for (int i : idx) {
    std::pop_heap(heap.begin(), heap.end(), cmp);
    auto& top = heap.back();
    per[top.second].push_back((uint32_t)i);
    top.first += cost[i];
    std::push_heap(heap.begin(), heap.end(), cmp);
  }
  std::vector<uint32_t> t(clusters + 1);
  t[0] = 0;
  for (int c = 0; c < clusters; ++c) t[c + 1] = t[c] + (uint32_t)per[c].size();
  for (int c = 0; c < clusters; ++c) t.insert(t.end(), per[c].begin(), per[c].end());
  return t;
}

struct BatchPlan {
  int count;
  std::vector<InstPlan> in;
  TcPlan tc;                  // the call's default plan (and the block-sparse one)
  std::vector<TcFamily> fam;  // tensor-core families, in launch order
  std::vector<int> tc_order;  // TC instances: the families' orders concatenated
  int n_tc = 0, n_cut = 0, n_simt = 0, n_reduce = 0, tc_items = 0, max_side = 1;
  int64_t total_pad = 0, cut_m = 0, total_bins = 0, reduce_cells = 0, cut_bins = 0;
  int64_t cut_slice_bins = 0;  // output blocks of cutoff instances that split heavy blocks
  bool sparse = false;  // block-sparse tensor-core instances
  int tiles_total = 0, piece_len = 0, max_pieces = 0;
  size_t off_sp_total = 0, off_sp_np = 0, off_sp_pb = 0, off_sp_nf = 0, off_sp_fb = 0,
         off_sp_tail = 0, off_sp_temp = 0, off_sp_part = 0;
  CutoffSizes cz;
  bool host_pts = false, host_w = false, host_out = false;
  size_t off_scal, off_pts, off_wts, off_tab_prep, off_tab_tc, off_tab_cut, off_tab_red;
  size_t off_co_keys[2], off_co_vals[2], off_co_hist, off_co_start,
      off_co_spts, off_co_sw, off_co_order, off_co_totals, off_co_ranges, off_co_ocount, off_hxy,
      off_hw,
      off_hout, total;
};

int make_plan(const kde_args* A, int count, const kde_opts* o, const kde_tiling* tiles,
              bool probe_memory, BatchPlan* P) {
  P->count = count;
  P->in.assign(count, InstPlan());
  const int sms = sm_count();
  const int ctas = (o && o->max_ctas > 0) ? std::min(o->max_ctas, sms) : sms;
  int tc_split16 = -1;
  for (int k = 0; k < count; ++k) {
    const kde_args* a = &A[k];
    InstPlan& I = P->in[k];
    I.path = resolve_path(a, o);
    if (is_tc(I.path)) {
      const int s16 = I.path == KDE_PATH_TC_SPLIT16;
      if (tc_split16 >= 0 && tc_split16 != s16)
        return fail(KDE_ENOTSUP, "one batch cannot mix FP16 and split-FP16 tensor paths");
      tc_split16 = s16;
    }
    I.n_pad = std::max<int64_t>(512, (a->n + 511) / 512 * 512);
    I.prep_begin = P->total_pad;
    P->total_pad += I.n_pad;
    P->max_side = std::max({P->max_side, a->nx, a->ny});
  }
  if (count == 1 && probe_memory) {
    const kde_args* a = &A[0];
    P->host_pts = a->n > 0 && memory_kind(a->points) == 1;
    P->host_w = a->n > 0 && a->weights && memory_kind(a->weights) == 1;
    P->host_out = memory_kind(a->out) == 1;
  } else if (probe_memory) {
    for (int k = 0; k < count; ++k)
      if ((A[k].n > 0 && memory_kind(A[k].points) != 0) ||
          (A[k].weights && memory_kind(A[k].weights) != 0) || memory_kind(A[k].out) != 0)
        return fail(KDE_EINVAL, "instance %d: batched calls need device pointers", k);
  }

  // tensor-core plan shared by every TC instance of the batch
  TcPlan& t = P->tc;
  t.split16 = tc_split16 == 1;
  t.tile_n = (o && o->tile_n) ? o->tile_n : 256;
  if (count == 1 && !(o && o->tile_n)) t.tile_n = A[0].ny <= 128 ? 128 : 256;
  // the tensor core's FP32 accumulation loses accuracy with every MMA step it
  // adds into a large sum, so split-FP16 drains its accumulators often
  // (512-point chunks are ~5% faster on CTA pairs but reach 1e-5 on a dense
  // batched instance)
  t.k_chunk = (o && o->k_chunk) ? o->k_chunk : (t.split16 ? 256 : 1024);
  // 64-point stages (128-byte rows): fewer barrier round trips per point
  // outweigh the deeper pipeline 32-point stages would allow
  t.stage_points = (o && o->stage_points) ? o->stage_points : 64;
  t.ctas = ctas;
  t.skip_zero = (o && (o->flags & KDE_FLAG_SKIP_ZERO)) ? 1 : 0;
  t.splits = 1;
  // CTA pairs (256 x 256 tiles, cta_group::2) halve each SM's operand reads
  // per MMA; they are the default with 256-wide tiles (20M points x 4096^2:
  // split-FP16 1223 ms, FP16 885 ms on pairs against 1186 ms on one CTA)
  // block-sparse skipping runs on CTA pairs
  const bool want_sparse = t.skip_zero && tc_split16 >= 0;
  const bool want_pair = o && ((o->flags & KDE_FLAG_CTA_PAIR) || want_sparse);
  const bool no_pair = o && (o->flags & KDE_FLAG_ONE_CTA);
  if (want_sparse && no_pair)
    return fail(KDE_ENOTSUP, "KDE_FLAG_SKIP_ZERO runs on CTA pairs; KDE_FLAG_ONE_CTA excludes it");
  if (want_pair && no_pair) return fail(KDE_EINVAL, "KDE_FLAG_CTA_PAIR and KDE_FLAG_ONE_CTA conflict");
  if (want_pair) {
    if ((o->tile_n && o->tile_n != 256) || (o->stage_points && o->stage_points != 64))
      return fail(KDE_EINVAL, "CTA-pair tiles are 256 x 256 with 64-point stages");
    t.tile_n = 256;
    t.stage_points = 64;
  }
  const bool pair_ok = t.tile_n == 256 && t.stage_points == 64 && ctas >= 2;
  if (want_pair && !pair_ok)
    return fail(KDE_EINVAL, "CTA-pair tiles need tile_n 256, 64-point stages and two CTAs");
  t.pair = want_pair || (!no_pair && pair_ok) ? 1 : 0;
  P->sparse = want_sparse;

  if (tc_split16 >= 0 && (t.k_chunk % t.stage_points || t.k_chunk < 2 * t.stage_points))
    return fail(KDE_EINVAL, "k_chunk %d must be a multiple of, and at least twice, the %d-point stage",
                t.k_chunk, t.stage_points);

  // tile families: the call's plan, changed per instance by its tiling; the
  // instances of one family share a persistent launch
  for (int k = 0; k < count; ++k) {
    InstPlan& I = P->in[k];
    I.fam = -1;
    I.split_req = o ? o->split_k : 0;
    if (!is_tc(I.path)) continue;
    TcPlan f = t;
    int kc = t.k_chunk;
    if (tiles) {
      const kde_tiling& ti = tiles[k];
      if ((ti.tile_n != 0 && ti.tile_n != 128 && ti.tile_n != 256) ||
          (ti.stage_points != 0 && ti.stage_points != 32 && ti.stage_points != 64) ||
          ti.k_chunk < 0 || (ti.k_chunk % 32) != 0 || ti.split_k < 0 || ti.split_k > 1024 ||
          (ti.flags & ~(KDE_FLAG_CTA_PAIR | KDE_FLAG_ONE_CTA)) ||
          ((ti.flags & KDE_FLAG_CTA_PAIR) && (ti.flags & KDE_FLAG_ONE_CTA)))
        return fail(KDE_EINVAL, "instance %d: invalid tiling", k);
      if (P->sparse) {
        if ((ti.flags & KDE_FLAG_ONE_CTA) || (ti.tile_n && ti.tile_n != 256) ||
            (ti.stage_points && ti.stage_points != 64))
          return fail(KDE_ENOTSUP, "instance %d: block-sparse skipping runs on 256 x 256 CTA-pair "
                      "tiles with 64-point stages", k);
      } else {
        if (ti.tile_n) f.tile_n = ti.tile_n;
        if (ti.stage_points) f.stage_points = ti.stage_points;
        const bool can_pair = f.tile_n == 256 && f.stage_points == 64 && ctas >= 2;
        if (ti.flags & KDE_FLAG_CTA_PAIR) {
          if (!can_pair)
            return fail(KDE_EINVAL, "instance %d: CTA-pair tiles need tile_n 256, 64-point stages "
                        "and two CTAs", k);
          f.pair = 1;
        } else if (ti.flags & KDE_FLAG_ONE_CTA) {
          f.pair = 0;
        } else {
          f.pair = t.pair && can_pair ? 1 : 0;
        }
      }
      if (ti.k_chunk) kc = ti.k_chunk;
      if (ti.split_k) I.split_req = ti.split_k;
      if (kc % f.stage_points || kc < 2 * f.stage_points)
        return fail(KDE_EINVAL, "instance %d: k_chunk %d must be a multiple of, and at least "
                    "twice, the %d-point stage", k, kc, f.stage_points);
    }
    I.k_chunk = kc;
    for (int q = 0; q < (int)P->fam.size() && I.fam < 0; ++q) {
      const TcPlan& g = P->fam[q].plan;
      if (g.pair == f.pair && g.tile_n == f.tile_n && g.stage_points == f.stage_points) I.fam = q;
    }
    if (I.fam < 0) {
      I.fam = (int)P->fam.size();
      P->fam.push_back(TcFamily());
      P->fam.back().plan = f;
    }
  }

  // per-path work decomposition
  std::vector<double> fam_cost(P->fam.size(), 0.0);
  for (int k = 0; k < count; ++k) {
    const kde_args* a = &A[k];
    InstPlan& I = P->in[k];
    if (is_tc(I.path)) {
      const TcPlan& f = P->fam[I.fam].plan;
      const int tile_m = f.pair ? 256 : 128;
      I.tiles_m = (a->nx + tile_m - 1) / tile_m;
      I.tiles_n = (a->ny + f.tile_n - 1) / f.tile_n;
      fam_cost[I.fam] += (double)I.tiles_m * I.tiles_n * (double)I.n_pad;
    }
  }
  for (int k = 0; k < count; ++k) {
    const kde_args* a = &A[k];
    InstPlan& I = P->in[k];
    int splits = I.split_req;
    if (I.path == KDE_PATH_SIMT_FP32) {
      if (splits == 0) {
        const int64_t tiles = (int64_t)((a->nx + 127) / 128) * ((a->ny + 63) / 64);
        const int64_t want = (6 * (int64_t)sms + tiles - 1) / tiles;
        const int64_t maxs = std::max<int64_t>(1, I.n_pad / 4096);
        splits = (int)std::max<int64_t>(1, std::min<int64_t>({want, maxs, 64}));
      }
      ++P->n_simt;
    } else if (is_tc(I.path) && P->sparse) {
      // block-sparse: the work list is built on the device; no point splits
      splits = 1;
      I.per_split = I.n_pad;
      I.items = 0;
      P->fam[I.fam].order.push_back(k);
      ++P->n_tc;
    } else if (is_tc(I.path)) {
      const TcPlan& f = P->fam[I.fam].plan;
      const int units = f.pair ? ctas / 2 : ctas;
      const int64_t tiles = (int64_t)I.tiles_m * I.tiles_n;
      if (splits == 0) {
        if (count == 1) {
          splits = choose_tc_splits(tiles, units, I.n_pad);
        } else {
          // items of about a sixth of each CTA's (pair's) share of the family
          const double target_item = fam_cost[I.fam] / (double)units / 6.0;
          const double want = std::ceil((double)I.n_pad / std::max(target_item, 1.0));
          splits = (int)std::max(1.0, std::min({want, 64.0, (double)(I.n_pad / 256)}));
        }
      }
      const int64_t ks = f.stage_points;
      I.per_split = ((I.n_pad + splits - 1) / splits + ks - 1) / ks * ks;
      I.items = (int)(tiles * splits);
      P->fam[I.fam].order.push_back(k);
      ++P->n_tc;
    } else {  // cutoff
      splits = 1;
      I.geo = cutoff_geometry(a->nx, a->ny, a->cell / a->h, 1.0,
                              cutoff_sort_bin(a->nx, a->ny, a->h / a->cell));
      I.bin_begin = (int)P->total_bins;
      P->total_bins += I.geo.nbins;
      I.obx = (a->nx + kCutoffBin - 1) / kCutoffBin;
      I.oby = (a->ny + kCutoffBin - 1) / kCutoffBin;
      I.out_begin = (int)P->cut_bins;
      P->cut_bins += (int64_t)I.obx * I.oby;
      if (I.geo.bin == 4) P->cut_slice_bins += (int64_t)I.obx * I.oby;
      I.cut_begin = P->cut_m;
      P->cut_m += I.n_pad;
      ++P->n_cut;
    }
    I.splits = std::max(splits, 1);
    if (I.splits > 1) {
      ++P->n_reduce;
      P->reduce_cells += (int64_t)a->nx * a->ny;
    }
  }
  // most expensive work items first within each family, so round-robin CTAs
  // balance; the TC table holds the families one after the other
  for (TcFamily& f : P->fam) {
    std::stable_sort(f.order.begin(), f.order.end(), [&](int x, int y) {
      return P->in[x].per_split > P->in[y].per_split;
    });
    f.tab_begin = (int)P->tc_order.size();
    for (int k : f.order) {
      P->tc_order.push_back(k);
      f.items += P->in[k].items;
    }
  }
  if (P->sparse) {
    // bins of the block-sparse instances follow the cutoff bins in the sort
    double est = 0.0;
    int64_t bound = 0;
    for (int k : P->tc_order) {
      const kde_args* a = &A[k];
      InstPlan& I = P->in[k];
      const double cs = a->cell * kernel_sigma(KDE_GAUSSIAN, a->h);
      I.geo = cutoff_geometry(a->nx, a->ny, cs, kSparseReach, kSparseBin);
      I.bin_begin = (int)P->total_bins;
      P->total_bins += I.geo.nbins;
      I.cut_begin = P->cut_m;
      P->cut_m += I.n_pad;
      I.tile_begin = P->tiles_total;
      P->tiles_total += I.tiles_m * I.tiles_n;
      est += 1.5 * (double)I.n_pad;
    }
    // pieces of about an eighth of each CTA pair's share, in whole drain chunks
    const int clusters = std::max(1, ctas / 2);
    int64_t L = (int64_t)(est / (8.0 * clusters));
    L = std::max<int64_t>(2048, std::min<int64_t>(kSparseMaxPiece, L));
    L = (L + t.k_chunk - 1) / t.k_chunk * t.k_chunk;
    P->piece_len = (int)L;
    for (int k : P->tc_order) {
      const kde_args* a = &A[k];
      const InstPlan& I = P->in[k];
      // a bin lies within reach of at most `per_axis` tiles along each axis
      const double rc = kSparseReach / (a->cell * kernel_sigma(KDE_GAUSSIAN, a->h));
      const int64_t per_axis = (int64_t)std::ceil((288.0 + 2.0 * rc) / 256.0) + 1;
      const int64_t tiles = (int64_t)I.tiles_m * I.tiles_n;
      const int64_t reach_tiles = std::min(per_axis * per_axis, tiles);
      bound += (I.n_pad * reach_tiles + L - 1) / L + tiles;
    }
    if (bound > (1 << 24) || P->tiles_total > (1 << 26))
      return fail(KDE_EINVAL, "block-sparse work list too large (%lld pieces)", (long long)bound);
    P->max_pieces = (int)bound;
  }
  if (P->total_bins >= ((int64_t)1 << 31)) return fail(KDE_EINVAL, "too many bins in one batch");
  if (P->cut_m >= ((int64_t)1 << 32)) return fail(KDE_EINVAL, "too many points to sort in one batch");
  for (int k : P->tc_order) P->tc_items += P->in[k].items;
  if ((int64_t)P->tc_items > 0x7fffffff) return fail(KDE_EINVAL, "too many work items");
  // batches on CTA pairs: balance the pairs' work with a host-side schedule
  // (items of different instances differ in length; round robin left the last
  // pair finishing 7% after the mean on the 256-instance batch)
  if (count > 1 && !P->sparse) {
    for (TcFamily& f : P->fam) {
      if (!f.plan.pair || f.items < 2) continue;
      std::vector<int64_t> cost;
      cost.reserve(f.items);
      for (int k : f.order) {
        const InstPlan& I = P->in[k];
        const int64_t per_tile = (int64_t)I.tiles_m * I.tiles_n;
        for (int local = 0; local < I.items; ++local) {
          const int64_t s = local / per_tile;
          const int64_t len = std::min<int64_t>(I.per_split, I.n_pad - s * I.per_split);
          cost.push_back(std::max<int64_t>(len, 0) / f.plan.stage_points + 4);
        }
      }
      f.sched = lpt_schedule(cost, pair_clusters(f.plan, f.items));
    }
  }
  if (P->sparse && P->fam.size() > 1) return fail(KDE_EINVAL, "block-sparse batch with two tilings");
  P->cz = cutoff_sizes(P->cut_m, P->total_bins);

  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = align256(off + bytes); return r; };
  P->off_scal = take(sizeof(CallScalars) * (size_t)(count + 1));
  P->off_pts = take(sizeof(float4) * (size_t)P->total_pad);
  P->off_wts = take(sizeof(float) * (size_t)P->total_pad);
  P->off_tab_prep = take(sizeof(PrepInst) * (size_t)count);
  P->off_tab_tc = take(sizeof(TcInst) * (size_t)std::max(P->n_tc, 1));
  P->off_tab_cut = take(sizeof(CutInst) * (size_t)std::max(P->n_cut + (P->sparse ? P->n_tc : 0), 1));
  P->off_tab_red = take(sizeof(ReduceInst) * (size_t)std::max(P->n_reduce, 1));
  for (TcFamily& f : P->fam)
    if (!f.sched.empty()) f.off_sched = take(sizeof(uint32_t) * f.sched.size());
  for (int k = 0; k < count; ++k) {
    InstPlan& I = P->in[k];
    I.off_gxt = take(sizeof(float2) * (size_t)A[k].nx);
    I.off_gyt = take(sizeof(float2) * (size_t)A[k].ny);
    I.off_part = I.splits > 1 ? take(sizeof(float) * (size_t)A[k].nx * A[k].ny * I.splits) : 0;
    I.off_run = I.path == KDE_PATH_SIMT_FP32 ? take(simt_scratch_bytes(A[k].nx, A[k].ny, I.splits))
                                             : 0;
  }
  if (P->n_cut || P->sparse) {
    const size_t u = sizeof(uint32_t);
    for (int k = 0; k < 2; ++k) {
      P->off_co_keys[k] = take(u * (size_t)P->cut_m);
      P->off_co_vals[k] = take(u * (size_t)P->cut_m);
    }
    P->off_co_hist = take(u * P->cz.hist_words);
    P->off_co_start = take(u * ((size_t)P->total_bins + 1));
    P->off_co_spts = take(sizeof(float4) * (size_t)P->cut_m);
    P->off_co_sw = take(sizeof(float) * (size_t)P->cut_m);
    P->off_co_order = take(u * (size_t)std::max<int64_t>(P->cut_bins, 1));
    P->off_co_totals = take(u * (size_t)std::max<int64_t>(P->cut_bins, 1));
    P->off_co_ranges = take(sizeof(int4) * (size_t)std::max<int64_t>(P->cut_bins, 1));
    P->off_co_ocount = take(u * kCutOcountWords);
  }
  if (P->sparse) {
    const size_t u = sizeof(uint32_t);
    P->off_sp_total = take(u * (size_t)P->tiles_total);
    P->off_sp_np = take(u * ((size_t)P->tiles_total + 1));
    P->off_sp_pb = take(u * ((size_t)P->tiles_total + 1));
    P->off_sp_nf = take(u * ((size_t)P->tiles_total + 1));
    P->off_sp_fb = take(u * ((size_t)P->tiles_total + 1));
    P->off_sp_tail = take(u * (size_t)P->tiles_total);
    P->off_sp_temp = take(u * sparse_scan_words(P->tiles_total));
    P->off_sp_part = take(sizeof(float) * 65536 * (size_t)P->max_pieces);
  }
  P->off_hxy = take(P->host_pts ? sizeof(double) * 2 * (size_t)A[0].n : 0);
  P->off_hw = take(P->host_w ? sizeof(float) * (size_t)A[0].n : 0);
  P->off_hout = take(P->host_out ? sizeof(float) * (size_t)A[0].nx * A[0].ny : 0);
  P->total = off;
  return KDE_OK;
}

cudaStream_t stream_of(const kde_opts* o) {
  return o ? reinterpret_cast<cudaStream_t>(o->stream) : (cudaStream_t)0;
}

int acquire_workspace(const kde_opts* o, size_t need, cudaStream_t s, void** ws) {
  if (o && o->workspace) {
    if (o->workspace_bytes < need)
      return fail(KDE_ENOMEM, "caller workspace has %zu bytes, %zu needed", o->workspace_bytes, need);
    *ws = o->workspace;
    return KDE_OK;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_ws_mu);
    if (dev < 0 || dev >= kMaxDevices || g_ws_bytes[dev] < need)
      return fail(KDE_ENOMEM, "the workspace must hold %zu bytes before stream capture "
                  "(make the same call once outside capture, or pass opts->workspace)", need);
    *ws = g_ws_ptr[dev];
    return KDE_OK;
  }
  cudaGetLastError();
  return library_workspace(need, ws);
}

// The bin-key kernel's FP32 constants of a sort instance (set after its
// geometry and reach).
void set_key_constants(CutInst& q) {
  q.key_lo = (float)-q.range_reach;
  q.key_hx = (float)(q.ext_x - q.reach + q.range_reach);
  q.key_hy = (float)(q.ext_y - q.reach + q.range_reach);
  q.key_inv = (float)q.inv_binw;
}

// Plan, lay out, upload and launch every instance of a batch on one stream.
int run_batch(const kde_args* A, int count, const kde_opts* o, const kde_tiling* tiles,
              bool force_sync) {
  for (int k = 0; k < count; ++k) {
    int rc = validate(&A[k], o);
    if (rc) return rc;
  }
  BatchPlan P;
  int rc = make_plan(A, count, o, tiles, true, &P);
  if (rc) return rc;
  cudaStream_t s = stream_of(o);
  // host output makes the call wait for its copy back, unless the caller
  // asked for the asynchronous host mode (and then synchronises the stream)
  const bool host_async = o && (o->flags & KDE_FLAG_HOST_ASYNC);
  const bool sync = force_sync || (o && (o->flags & KDE_FLAG_SYNC)) || (P.host_out && !host_async);
  void* wsv = nullptr;
  rc = acquire_workspace(o, P.total, s, &wsv);
  if (rc) return rc;
  char* base = static_cast<char*>(wsv);
  CallScalars* scal = reinterpret_cast<CallScalars*>(base + P.off_scal);
  CallScalars* batch_scal = scal + count;
  float4* pts = reinterpret_cast<float4*>(base + P.off_pts);
  float* wts = reinterpret_cast<float*>(base + P.off_wts);

  KDE_CUDA(cudaMemsetAsync(scal, 0, sizeof(CallScalars) * (size_t)(count + 1), s), "clear scalars");
  const double* xy0 = A[0].points;
  const float* w0 = A[0].weights;
  if (P.host_pts) {
    double* d = reinterpret_cast<double*>(base + P.off_hxy);
    KDE_CUDA(cudaMemcpyAsync(d, xy0, sizeof(double) * 2 * A[0].n, cudaMemcpyHostToDevice, s),
             "copy points to device");
    xy0 = d;
  }
  if (P.host_w) {
    float* d = reinterpret_cast<float*>(base + P.off_hw);
    KDE_CUDA(cudaMemcpyAsync(d, w0, sizeof(float) * A[0].n, cudaMemcpyHostToDevice, s),
             "copy weights to device");
    w0 = d;
  }

  // ---- tables
  std::vector<PrepInst> prep(count, PrepInst{});
  const bool lonlat = o && (o->flags & KDE_FLAG_LONLAT);
  const MercParams merc = lonlat ? mercator_params(o->lat0_deg) : MercParams{};
  std::vector<TcInst> tct;
  std::vector<CutInst> cut;
  std::vector<ReduceInst> red;
  std::vector<float*> out_dev(count);
  for (int k = 0; k < count; ++k) {
    const kde_args* a = &A[k];
    const InstPlan& I = P.in[k];
    out_dev[k] = (k == 0 && P.host_out) ? reinterpret_cast<float*>(base + P.off_hout) : a->out;
    PrepInst& q = prep[k];
    q.xy = k == 0 ? xy0 : a->points;
    q.w = k == 0 ? w0 : a->weights;
    q.pts = pts + I.prep_begin;
    q.wts = wts + I.prep_begin;
    q.gxt = reinterpret_cast<float2*>(base + I.off_gxt);
    q.gyt = reinterpret_cast<float2*>(base + I.off_gyt);
    q.scal = scal + k;
    q.n = a->n;
    q.n_pad = I.n_pad;
    q.begin = I.prep_begin;
    q.ox = a->origin_x;
    q.oy = a->origin_y;
    q.sigma = kernel_sigma(kid_of(a), a->h);
    q.cell_sigma = a->cell * q.sigma;
    q.nx = a->nx;
    q.ny = a->ny;
    q.lonlat = lonlat ? 1 : 0;
    q.merc = merc;
  }
  auto part_of = [&](int k) {
    return P.in[k].splits > 1 ? reinterpret_cast<float*>(base + P.in[k].off_part) : out_dev[k];
  };
  auto compact_scale = [&](int k) {
    const int kid = kid_of(&A[k]);
    const double c1 = kernel_const_1d(kid);
    const double c = kid >= kRadial ? kernel_const_radial(kid - kRadial) : c1 * c1;
    return A[k].n > 0 ? (float)(c / ((double)A[k].n * A[k].h * A[k].h)) : 0.0f;
  };
  int item_begin = 0;
  for (int k : P.tc_order) {
    const kde_args* a = &A[k];
    const InstPlan& I = P.in[k];
    const TcFamily& fam = P.fam[I.fam];
    if (k == fam.order.front()) item_begin = 0;  // each family numbers its own items
    TcInst q;
    q.pts = prep[k].pts;
    q.wts = prep[k].wts;
    q.gxt = prep[k].gxt;
    q.gyt = prep[k].gyt;
    q.scal = scal + k;
    q.part = part_of(k);
    q.n_pad = I.n_pad;
    q.per_split = I.per_split;
    q.nx = a->nx;
    q.ny = a->ny;
    q.tiles_m = I.tiles_m;
    q.tiles_n = I.tiles_n;
    q.splits = I.splits;
    q.item_begin = item_begin;
    q.chunk_stages = I.k_chunk / fam.plan.stage_points;
    // c = 2^-30 / (2 pi N h^2); the kernel multiplies by max |w|
    q.base_scale = a->n > 0 ? (float)(0x1p-30 / (2.0 * 3.14159265358979323846 * (double)a->n *
                                                 a->h * a->h))
                            : 0.0f;
    q.start = nullptr;
    q.cs = q.reach = q.inv_binw = q.range_reach = 0.0;
    q.nbx = q.nby = q.bin_begin = q.tile_begin = 0;
    if (P.sparse) {  // points in bin order; the sparse reduce writes the output
      q.pts = reinterpret_cast<const float4*>(base + P.off_co_spts);
      q.wts = reinterpret_cast<const float*>(base + P.off_co_sw);
      q.part = out_dev[k];
      q.start = reinterpret_cast<const uint32_t*>(base + P.off_co_start);
      q.cs = prep[k].cell_sigma;
      q.reach = kSparseReach;
      q.range_reach = range_reach(kSparseReach, I.geo);
      q.inv_binw = I.geo.inv_binw;
      q.nbx = I.geo.nbx;
      q.nby = I.geo.nby;
      q.bin_begin = I.bin_begin;
      q.tile_begin = I.tile_begin;
    }
    item_begin += I.items;
    tct.push_back(q);
  }
  for (int k = 0; k < count; ++k) {
    const InstPlan& I = P.in[k];
    if (I.path == KDE_PATH_CUTOFF) {
      CutInst q = {};
      q.gxt = prep[k].gxt;
      q.gyt = prep[k].gyt;
      q.out = out_dev[k];
      q.n = A[k].n;
      q.n_pad = I.n_pad;
      q.prep_begin = I.prep_begin;
      q.cut_begin = I.cut_begin;
      q.inv_binw = I.geo.inv_binw;
      q.ext_x = I.geo.ext_x;
      q.ext_y = I.geo.ext_y;
      q.reach = 1.0;
      q.range_reach = range_reach(1.0, I.geo);
      set_key_constants(q);
      q.cs = A[k].cell / A[k].h;
      q.nbx = I.geo.nbx;
      q.nby = I.geo.nby;
      q.bin_begin = I.bin_begin;
      q.obx = I.obx;
      q.oby = I.oby;
      q.out_begin = I.out_begin;
      q.nx = A[k].nx;
      q.ny = A[k].ny;
      q.kid = kid_of(&A[k]);
      q.scale = compact_scale(k);
      q.slice = I.geo.bin == 4;
      cut.push_back(q);
    }
    if (I.splits > 1) {
      ReduceInst q;
      q.part = part_of(k);
      q.out = out_dev[k];
      q.cells = (int64_t)A[k].nx * A[k].ny;
      q.begin = red.empty() ? 0 : red.back().begin + red.back().cells;
      q.splits = I.splits;
      red.push_back(q);
    }
  }
  const int n_cut_only = (int)cut.size();
  if (P.sparse) {  // bin-sort entries of the block-sparse instances, after the cutoff ones
    for (int k : P.tc_order) {
      const InstPlan& I = P.in[k];
      CutInst q = {};
      q.gxt = prep[k].gxt;
      q.gyt = prep[k].gyt;
      q.out = out_dev[k];
      q.n = A[k].n;
      q.n_pad = I.n_pad;
      q.prep_begin = I.prep_begin;
      q.cut_begin = I.cut_begin;
      q.inv_binw = I.geo.inv_binw;
      q.ext_x = I.geo.ext_x;
      q.ext_y = I.geo.ext_y;
      q.reach = kSparseReach;
      q.range_reach = range_reach(kSparseReach, I.geo);
      q.cs = A[k].cell * kernel_sigma(KDE_GAUSSIAN, A[k].h);
      set_key_constants(q);
      q.nbx = I.geo.nbx;
      q.nby = I.geo.nby;
      q.bin_begin = I.bin_begin;
      q.nx = A[k].nx;
      q.ny = A[k].ny;
      q.kid = KDE_GAUSSIAN;
      cut.push_back(q);
    }
    // cut_begin must increase along the table for the key kernel's search
    std::stable_sort(cut.begin() + n_cut_only, cut.end(),
                     [](const CutInst& x, const CutInst& y) { return x.cut_begin < y.cut_begin; });
  }
  PrepInst* d_prep = reinterpret_cast<PrepInst*>(base + P.off_tab_prep);
  TcInst* d_tc = reinterpret_cast<TcInst*>(base + P.off_tab_tc);
  CutInst* d_cut = reinterpret_cast<CutInst*>(base + P.off_tab_cut);
  ReduceInst* d_red = reinterpret_cast<ReduceInst*>(base + P.off_tab_red);
  KDE_CUDA(launch_upload(prep.data(), sizeof(PrepInst) * prep.size(), d_prep, s), "upload tables");
  if (!tct.empty())
    KDE_CUDA(launch_upload(tct.data(), sizeof(TcInst) * tct.size(), d_tc, s), "upload tables");
  if (!cut.empty())
    KDE_CUDA(launch_upload(cut.data(), sizeof(CutInst) * cut.size(), d_cut, s), "upload tables");
  if (!red.empty())
    KDE_CUDA(launch_upload(red.data(), sizeof(ReduceInst) * red.size(), d_red, s), "upload tables");
  for (const TcFamily& f : P.fam)
    if (!f.sched.empty())
      KDE_CUDA(launch_upload(f.sched.data(), sizeof(uint32_t) * f.sched.size(), base + f.off_sched,
                             s),
               "upload schedule");

  // ---- launches
  KDE_CUDA(launch_prepare(d_prep, count, P.total_pad, P.max_side, s), "prepare points");
  cudaEvent_t* ev = o ? static_cast<cudaEvent_t*>(o->timing_events) : nullptr;
  if (ev) KDE_CUDA(cudaEventRecord(ev[0], s), "record start event");
  CutoffScratch cs;
  if (P.n_cut || P.sparse) {
    for (int k = 0; k < 2; ++k) {
      cs.keys[k] = reinterpret_cast<uint32_t*>(base + P.off_co_keys[k]);
      cs.vals[k] = reinterpret_cast<uint32_t*>(base + P.off_co_vals[k]);
    }
    cs.hist = reinterpret_cast<uint32_t*>(base + P.off_co_hist);
    cs.start = reinterpret_cast<uint32_t*>(base + P.off_co_start);
    cs.spts = reinterpret_cast<float4*>(base + P.off_co_spts);
    cs.sw = reinterpret_cast<float*>(base + P.off_co_sw);
    cs.order = reinterpret_cast<uint32_t*>(base + P.off_co_order);
    cs.totals = reinterpret_cast<uint32_t*>(base + P.off_co_totals);
    cs.ranges = reinterpret_cast<int4*>(base + P.off_co_ranges);
    cs.ocount = reinterpret_cast<uint32_t*>(base + P.off_co_ocount);
    cs.err = batch_scal;
  }
  // The compact instances (sort and gather) overlap the tensor-core
  // contraction on the side stream when no block-sparse instance needs the
  // sort first: the contraction is enqueued first, its CTAs take every SM,
  // the small sort kernels fit beside them and the gather fills the SMs its
  // tail frees.  They write disjoint buffers, so results do not change.
  const bool overlap = P.n_cut && P.n_tc && !P.sparse;
  cudaStream_t s2 = s;
  cudaEvent_t fork = nullptr, join = nullptr;
  struct EventGuard {
    cudaEvent_t* e[2];
    ~EventGuard() {
      for (cudaEvent_t* x : e)
        if (*x) cudaEventDestroy(*x);
    }
  } guard{{&fork, &join}};
  if (overlap) {
    if (int rc = side_stream(&s2)) return rc;
    KDE_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "create event");
    KDE_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming), "create event");
    KDE_CUDA(cudaEventRecord(fork, s), "fork to the side stream");
  }
  if ((P.n_cut || P.sparse) && !overlap)
    KDE_CUDA(launch_bin_sort(d_cut, (int)cut.size(), P.cut_m, P.total_bins, pts, wts, P.cz, cs, s),
             "bin sort");
  if (P.n_tc && P.sparse) {
    SparseCtl sp;
    sp.piece_begin = reinterpret_cast<const uint32_t*>(base + P.off_sp_pb);
    sp.full_begin = reinterpret_cast<const uint32_t*>(base + P.off_sp_fb);
    sp.tail_tile = reinterpret_cast<const uint32_t*>(base + P.off_sp_tail);
    sp.tile_total = reinterpret_cast<const uint32_t*>(base + P.off_sp_total);
    sp.part = reinterpret_cast<float*>(base + P.off_sp_part);
    sp.tiles_total = P.tiles_total;
    sp.piece_len = P.piece_len;
    sp.max_pieces = P.max_pieces;
    KDE_CUDA(launch_sparse_plan(d_tc, P.n_tc, sp, reinterpret_cast<uint32_t*>(base + P.off_sp_np),
                                reinterpret_cast<uint32_t*>(base + P.off_sp_nf),
                                reinterpret_cast<uint32_t*>(base + P.off_sp_temp), batch_scal, s),
             "block-sparse work list");
    KDE_CUDA(launch_tc_pair(P.fam[0].plan, d_tc, P.n_tc, 0, &sp, nullptr, batch_scal, s),
             "block-sparse tensor-core contraction");
    KDE_CUDA(launch_sparse_reduce(d_tc, P.n_tc, sp, s), "block-sparse reduce");
  } else if (P.n_tc) {
    for (const TcFamily& f : P.fam) {  // one persistent launch per tile family
      if (f.items < 1) continue;
      const int nf = (int)f.order.size();
      const uint32_t* sched =
          f.sched.empty() ? nullptr : reinterpret_cast<const uint32_t*>(base + f.off_sched);
      KDE_CUDA(f.plan.pair ? launch_tc_pair(f.plan, d_tc + f.tab_begin, nf, f.items, nullptr, sched,
                                            batch_scal, s)
                           : launch_tc(f.plan, d_tc + f.tab_begin, nf, f.items, batch_scal, s),
               "tensor-core contraction");
    }
  }
  for (int k = 0; k < count; ++k) {
    const InstPlan& I = P.in[k];
    if (I.path != KDE_PATH_SIMT_FP32) continue;
    KDE_CUDA(launch_simt(kid_of(&A[k]), prep[k].pts, prep[k].wts, I.n_pad, prep[k].gxt,
                         prep[k].gyt, A[k].nx, A[k].ny, I.splits, compact_scale(k),
                         reinterpret_cast<float2*>(base + I.off_run), part_of(k), s),
             "SIMT direct sum");
  }
  if (overlap) {
    KDE_CUDA(cudaStreamWaitEvent(s2, fork, 0), "side stream waits for the prepared points");
    KDE_CUDA(launch_bin_sort(d_cut, (int)cut.size(), P.cut_m, P.total_bins, pts, wts, P.cz, cs, s2),
             "bin sort");
    KDE_CUDA(launch_cutoff_eval(d_cut, n_cut_only, P.cut_bins, P.cut_slice_bins, cs, s2),
             "cutoff evaluation");
    KDE_CUDA(cudaEventRecord(join, s2), "join from the side stream");
    KDE_CUDA(cudaStreamWaitEvent(s, join, 0), "join the side stream");
  } else if (P.n_cut) {
    KDE_CUDA(launch_cutoff_eval(d_cut, n_cut_only, P.cut_bins, P.cut_slice_bins, cs, s),
             "cutoff evaluation");
  }
  if (ev) KDE_CUDA(cudaEventRecord(ev[1], s), "record end event");
  if (P.n_reduce) KDE_CUDA(launch_reduce(d_red, P.n_reduce, P.reduce_cells, s), "split-K reduce");
  if (P.host_out)
    KDE_CUDA(cudaMemcpyAsync(A[0].out, out_dev[0], sizeof(float) * A[0].nx * A[0].ny,
                             cudaMemcpyDeviceToHost, s),
             "copy result to host");
  if (sync) {
    std::vector<CallScalars> hs(count + 1);
    KDE_CUDA(cudaMemcpyAsync(hs.data(), scal, sizeof(CallScalars) * (count + 1),
                             cudaMemcpyDeviceToHost, s),
             "read status");
    KDE_CUDA(cudaStreamSynchronize(s), "synchronize");
    for (int k = 0; k <= count; ++k) {
      const int err = hs[k].err;
      if (err & kErrTimeout)
        return fail(KDE_ETIMEOUT, "a device-side wait gave up (role %d)", hs[k].timeout_where);
      if (err & kErrNonFinite)
        return fail(KDE_EDATA, "instance %d: non-finite coordinate or weight", k);
      if (err) return fail(KDE_ECUDA, "device error word 0x%x", err);
    }
  }
  g_err[0] = 0;
  return KDE_OK;
}

}  // namespace

void set_error_message(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg ? msg : ""); }

}  // namespace kde

using namespace kde;

extern "C" {

void kde_default_opts(kde_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->path = KDE_PATH_AUTO;
}

int kde_grid(const double* points, const float* weights, int64_t n, const double grid_origin[2],
             double cell, int nx, int ny, double h, int kernel_id, float* out) {
  if (!grid_origin) return fail(KDE_EINVAL, "grid_origin is NULL");
  kde_args a;
  a.points = points;
  a.weights = weights;
  a.n = n;
  a.origin_x = grid_origin[0];
  a.origin_y = grid_origin[1];
  a.cell = cell;
  a.nx = nx;
  a.ny = ny;
  a.h = h;
  a.kernel_id = kernel_id;
  a.out = out;
  kde_opts o;
  kde_default_opts(&o);
  o.stream = g_plain_stream;
  return run_batch(&a, 1, &o, nullptr, true);
}

void kde_set_stream(void* stream) { g_plain_stream = stream; }

int kde_grid_ex(const kde_args* a, const kde_opts* opts) {
  if (!a) return fail(KDE_EINVAL, "args is NULL");
  return run_batch(a, 1, opts, nullptr, false);
}

int kde_workspace_size(const kde_args* a, const kde_opts* opts, size_t* bytes) {
  if (!bytes) return fail(KDE_EINVAL, "bytes is NULL");
  int rc = validate(a, opts);
  if (rc) return rc;
  BatchPlan pl;
  rc = make_plan(a, 1, opts, nullptr, true, &pl);
  if (rc) return rc;
  *bytes = pl.total;
  return KDE_OK;
}

int kde_project_mercator(const double* lonlat_deg, int64_t n, double lat0_deg, double* xy_out,
                         void* stream) {
  if (n < 0) return fail(KDE_EINVAL, "n = %lld is negative", (long long)n);
  if (!(fabs(lat0_deg) < 90.0)) return fail(KDE_EINVAL, "standard latitude must be in (-90, 90)");
  if (n == 0) return KDE_OK;
  if (!lonlat_deg || !xy_out) return fail(KDE_EINVAL, "null pointer");
  if ((reinterpret_cast<uintptr_t>(lonlat_deg) | reinterpret_cast<uintptr_t>(xy_out)) & 15)
    return fail(KDE_EINVAL, "lon/lat and output must be 16-byte aligned");
  if (memory_kind(lonlat_deg) != 0 || memory_kind(xy_out) != 0)
    return fail(KDE_EINVAL, "kde_project_mercator needs device pointers");
  KDE_CUDA(launch_mercator(lonlat_deg, n, lat0_deg, xy_out, reinterpret_cast<cudaStream_t>(stream)),
           "Mercator projection");
  g_err[0] = 0;
  return KDE_OK;
}

int kde_grid_batched(const kde_args* inst, int count, const kde_opts* opts) {
  if (!inst || count < 0) return fail(KDE_EINVAL, "inst is NULL or count < 0");
  for (int b = 0; b < count; b += kMaxBatch) {
    const int c = std::min(kMaxBatch, count - b);
    const int rc = run_batch(inst + b, c, opts, nullptr, false);
    if (rc) return rc;
  }
  if (opts && (opts->flags & KDE_FLAG_SYNC) && count == 0) g_err[0] = 0;
  return KDE_OK;
}

int kde_grid_batched_tiled(const kde_args* inst, const kde_tiling* tiles, int count,
                           const kde_opts* opts) {
  if (!inst || count < 0) return fail(KDE_EINVAL, "inst is NULL or count < 0");
  for (int b = 0; b < count; b += kMaxBatch) {
    const int c = std::min(kMaxBatch, count - b);
    const int rc = run_batch(inst + b, c, opts, tiles ? tiles + b : nullptr, false);
    if (rc) return rc;
  }
  if (opts && (opts->flags & KDE_FLAG_SYNC) && count == 0) g_err[0] = 0;
  return KDE_OK;
}

int kde_grid_backward(const kde_args* a, const float* grad_out, float* grad_points,
                      float* grad_weights, double* grad_h, const kde_opts* opts) {
  int rc = validate(a, opts);
  if (rc) return rc;
  if (kid_of(a) != KDE_GAUSSIAN)
    return fail(KDE_ENOTSUP, "the adjoint is implemented for the Gaussian kernel");
  if (!grad_out || (a->n > 0 && !grad_points))
    return fail(KDE_EINVAL, "grad_out and grad_points are required");
  if (a->n > 0 && (memory_kind(a->points) != 0 || (a->weights && memory_kind(a->weights) != 0) ||
                   memory_kind(grad_points) != 0 ||
                   (grad_weights && memory_kind(grad_weights) != 0)))
    return fail(KDE_EINVAL, "kde_grid_backward needs device pointers");
  if (memory_kind(grad_out) != 0) return fail(KDE_EINVAL, "grad_out must be device memory");
  if ((reinterpret_cast<uintptr_t>(grad_points) & 7) || (reinterpret_cast<uintptr_t>(grad_out) & 3))
    return fail(KDE_EINVAL, "misaligned gradient buffer");
  cudaStream_t s = stream_of(opts);
  if (a->n == 0) {
    if (grad_h) *grad_h = 0.0;
    g_err[0] = 0;
    return KDE_OK;
  }
  const int64_t n_pad = (a->n + 511) / 512 * 512;
  // Window kernel or the two tensor-core contractions: the window sums about
  // (16 h / cell)^2 cells per point on the FP32 pipes, the contractions
  // nx ny cells per point (twice, three FP16 products) on the tensor cores.
  const int path = opts ? opts->path : KDE_PATH_AUTO;
  bool use_tc = path == KDE_PATH_TC_SPLIT16 || path == KDE_PATH_TC_FP16;
  if (path == KDE_PATH_AUTO) {
    const double R = std::ceil(8.0 * a->h / a->cell);
    const double win = std::min(2.0 * R + 1.0, (double)a->nx) * std::min(2.0 * R + 1.0, (double)a->ny);
    const double nxp = std::ceil(a->nx / 256.0) * 256.0, nyp = std::ceil(a->ny / 256.0) * 256.0;
    use_tc = win > kAdjointTcRatio * nxp * nyp;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = align256(off + bytes); return r; };
  const size_t o_scal = take(sizeof(CallScalars));
  const size_t o_tab = take(sizeof(PrepInst));
  const size_t o_pts = take(sizeof(float4) * n_pad);
  const size_t o_wts = take(sizeof(float) * n_pad);
  const size_t o_gxt = take(sizeof(float2) * a->nx);
  const size_t o_gyt = take(sizeof(float2) * a->ny);
  const size_t o_ht = take(sizeof(double) * a->n);
  const size_t o_lt = take(sizeof(double) * a->n);
  const size_t o_part = take(sizeof(double) * 2 * sum_partials(a->n));
  const size_t o_res = take(sizeof(double) * 2);
  const size_t o_tc = take(use_tc ? adjoint_tc_workspace(a->nx, a->ny) : 0);
  void* wsv = nullptr;
  rc = acquire_workspace(opts, off, s, &wsv);
  if (rc) return rc;
  char* base = static_cast<char*>(wsv);
  PrepInst q = {};
  q.xy = a->points;
  q.w = a->weights;
  q.pts = reinterpret_cast<float4*>(base + o_pts);
  q.wts = reinterpret_cast<float*>(base + o_wts);
  q.gxt = reinterpret_cast<float2*>(base + o_gxt);
  q.gyt = reinterpret_cast<float2*>(base + o_gyt);
  q.scal = reinterpret_cast<CallScalars*>(base + o_scal);
  q.n = a->n;
  q.n_pad = n_pad;
  q.begin = 0;
  q.ox = a->origin_x;
  q.oy = a->origin_y;
  // offsets in bandwidths (window kernel) or in h sqrt(2 ln 2) (contractions)
  q.sigma = use_tc ? kernel_sigma(KDE_GAUSSIAN, a->h) : 1.0 / a->h;
  q.cell_sigma = a->cell * q.sigma;
  q.nx = a->nx;
  q.ny = a->ny;
  double* ht = reinterpret_cast<double*>(base + o_ht);
  double* lt = reinterpret_cast<double*>(base + o_lt);
  double* part = reinterpret_cast<double*>(base + o_part);
  double* res = reinterpret_cast<double*>(base + o_res);
  KDE_CUDA(cudaMemsetAsync(q.scal, 0, sizeof(CallScalars), s), "clear scalars");
  KDE_CUDA(launch_upload(&q, sizeof(q), base + o_tab, s), "upload tables");
  KDE_CUDA(launch_prepare(reinterpret_cast<PrepInst*>(base + o_tab), 1, n_pad,
                          std::max(a->nx, a->ny), s),
           "prepare points");
  if (use_tc) {
    const int sms = sm_count();
    const int ctas = (opts && opts->max_ctas > 0) ? std::min(opts->max_ctas, sms) : sms;
    KDE_CUDA(launch_adjoint_gauss_tc(q.pts, q.wts, a->n, grad_out, q.gxt, q.gyt, a->nx, a->ny,
                                     a->cell, a->h, grad_points, grad_weights, ht, lt,
                                     base + o_tc, ctas, s),
             "adjoint contractions");
  } else {
    KDE_CUDA(launch_adjoint_gauss(q.pts, q.wts, a->n, grad_out, q.gxt, q.gyt, a->nx, a->ny,
                                  a->cell, a->h, grad_points, grad_weights, ht, lt, s),
             "adjoint");
  }
  const bool sync = grad_h || (opts && (opts->flags & KDE_FLAG_SYNC));
  if (grad_h) {
    const size_t np = sum_partials(a->n);
    KDE_CUDA(launch_sum(ht, a->n, part, res, s), "sum");
    KDE_CUDA(launch_sum(lt, a->n, part + np, res + 1, s), "sum");
  }
  if (sync) {
    double hres[2] = {0.0, 0.0};
    int err = 0, err_tc = 0, where = 0;
    if (grad_h)
      KDE_CUDA(cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, s), "read result");
    KDE_CUDA(cudaMemcpyAsync(&err, &q.scal->err, sizeof(int), cudaMemcpyDeviceToHost, s),
             "read status");
    if (use_tc) {
      const CallScalars* ts = reinterpret_cast<const CallScalars*>(base + o_tc);
      KDE_CUDA(cudaMemcpyAsync(&err_tc, &ts->err, sizeof(int), cudaMemcpyDeviceToHost, s),
               "read status");
      KDE_CUDA(cudaMemcpyAsync(&where, &ts->timeout_where, sizeof(int), cudaMemcpyDeviceToHost, s),
               "read status");
    }
    KDE_CUDA(cudaStreamSynchronize(s), "synchronize");
    if (err & kErrNonFinite) return fail(KDE_EDATA, "non-finite coordinate or weight");
    if (err_tc & kErrTimeout)
      return fail(KDE_ETIMEOUT, "a device-side wait of the adjoint gave up (role %d)", where);
    // dL/dh = -(2/h) sum G F + sum_p h-terms, with sum G F = sum_p w_p dL/dw_p
    if (grad_h) *grad_h = -2.0 / a->h * hres[1] + hres[0];
  }
  g_err[0] = 0;
  return KDE_OK;
}

int kde_lscv_grid(const kde_args* a, const float* F, double* loss, float* grad_F,
                  float* grad_w_direct, float* grad_points_direct, double* grad_h_direct,
                  const kde_opts* opts) {
  if (!a) return fail(KDE_EINVAL, "args is NULL");
  kde_args chk = *a;
  if (!chk.out) chk.out = const_cast<float*>(F);  // out is not used here
  int rc = validate(&chk, opts);
  if (rc) return rc;
  if (kid_of(a) != KDE_GAUSSIAN)
    return fail(KDE_ENOTSUP, "the LSCV loss is implemented for the Gaussian kernel");
  if (!F || !loss) return fail(KDE_EINVAL, "F and loss are required");
  if (memory_kind(F) != 0 || (grad_F && memory_kind(grad_F) != 0) ||
      (a->n > 0 && (memory_kind(a->points) != 0 ||
                    (a->weights && memory_kind(a->weights) != 0) ||
                    (grad_w_direct && memory_kind(grad_w_direct) != 0) ||
                    (grad_points_direct && memory_kind(grad_points_direct) != 0))))
    return fail(KDE_EINVAL, "kde_lscv_grid needs device pointers");
  cudaStream_t s = stream_of(opts);
  const int64_t n = a->n;
  const int64_t n_pad = std::max<int64_t>(512, (n + 511) / 512 * 512);
  const int sq_blocks = 152 * 4;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = align256(off + bytes); return r; };
  const size_t o_scal = take(sizeof(CallScalars));
  const size_t o_tab = take(sizeof(PrepInst));
  const size_t o_pts = take(sizeof(float4) * n_pad);
  const size_t o_wts = take(sizeof(float) * n_pad);
  const size_t o_gxt = take(sizeof(float2) * a->nx);
  const size_t o_gyt = take(sizeof(float2) * a->ny);
  const size_t o_loo = take(sizeof(double) * std::max<int64_t>(n, 1));
  const size_t o_hd = take(sizeof(double) * std::max<int64_t>(n, 1));
  const size_t o_sq = take(sizeof(double) * sq_blocks);
  const size_t o_gd = take(grad_F ? sizeof(double) * (size_t)a->nx * a->ny : 0);
  const size_t o_part = take(sizeof(double) * 3 * (sum_partials(std::max<int64_t>(n, sq_blocks)) + 1));
  const size_t o_res = take(sizeof(double) * 4);
  void* wsv = nullptr;
  rc = acquire_workspace(opts, off, s, &wsv);
  if (rc) return rc;
  char* base = static_cast<char*>(wsv);
  PrepInst q = {};
  q.xy = a->points;
  q.w = a->weights;
  q.pts = reinterpret_cast<float4*>(base + o_pts);
  q.wts = reinterpret_cast<float*>(base + o_wts);
  q.gxt = reinterpret_cast<float2*>(base + o_gxt);
  q.gyt = reinterpret_cast<float2*>(base + o_gyt);
  q.scal = reinterpret_cast<CallScalars*>(base + o_scal);
  q.n = n;
  q.n_pad = n_pad;
  q.begin = 0;
  q.ox = a->origin_x;
  q.oy = a->origin_y;
  q.sigma = 1.0 / a->h;
  q.cell_sigma = a->cell / a->h;
  q.nx = a->nx;
  q.ny = a->ny;
  double* loo = reinterpret_cast<double*>(base + o_loo);
  double* hd = reinterpret_cast<double*>(base + o_hd);
  double* sq = reinterpret_cast<double*>(base + o_sq);
  double* part = reinterpret_cast<double*>(base + o_part);
  double* res = reinterpret_cast<double*>(base + o_res);
  const size_t np = sum_partials(std::max<int64_t>(n, sq_blocks)) + 1;
  KDE_CUDA(cudaMemsetAsync(q.scal, 0, sizeof(CallScalars), s), "clear scalars");
  KDE_CUDA(cudaMemsetAsync(res, 0, sizeof(double) * 4, s), "clear results");
  KDE_CUDA(launch_upload(&q, sizeof(q), base + o_tab, s), "upload tables");
  KDE_CUDA(launch_prepare(reinterpret_cast<PrepInst*>(base + o_tab), 1, n_pad,
                          std::max(a->nx, a->ny), s),
           "prepare points");
  KDE_CUDA(launch_lscv(q.pts, q.wts, n, F, a->nx, a->ny, a->cell, a->h,
                       grad_F ? reinterpret_cast<double*>(base + o_gd) : nullptr, grad_F,
                       grad_w_direct, grad_points_direct, sq, sq_blocks, loo, hd, s),
           "LSCV");
  KDE_CUDA(launch_sum(sq, sq_blocks, part, res, s), "sum");
  if (n > 0) {
    KDE_CUDA(launch_sum(loo, n, part + np, res + 1, s), "sum");
    KDE_CUDA(launch_sum(hd, n, part + 2 * np, res + 2, s), "sum");
  }
  double hres[4];
  int err = 0;
  KDE_CUDA(cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, s), "read result");
  KDE_CUDA(cudaMemcpyAsync(&err, &q.scal->err, sizeof(int), cudaMemcpyDeviceToHost, s),
           "read status");
  KDE_CUDA(cudaStreamSynchronize(s), "synchronize");
  if (err & kErrNonFinite) return fail(KDE_EDATA, "non-finite coordinate or weight");
  const double N = (double)std::max<int64_t>(n, 1);
  // L = cell^2 sum F^2 - (2/N) sum_p w_p bilerp(F - F_p, x_p)
  *loss = a->cell * a->cell * hres[0] - 2.0 / N * hres[1];
  // the direct dependence on h is through each point's own term F_p
  if (grad_h_direct) *grad_h_direct += 2.0 / N * hres[2];
  g_err[0] = 0;
  return KDE_OK;
}

const char* kde_last_error(void) { return g_err; }

int kde_release(void) {
  std::lock_guard<std::mutex> lock(g_ws_mu);
  int prev = 0;
  cudaGetDevice(&prev);
  for (int d = 0; d < kMaxDevices; ++d) {
    if (g_ws_ptr[d]) {
      cudaSetDevice(d);
      cudaFree(g_ws_ptr[d]);
      g_ws_ptr[d] = nullptr;
      g_ws_bytes[d] = 0;
    }
    if (g_side[d]) {
      cudaSetDevice(d);
      cudaStreamDestroy(g_side[d]);
      g_side[d] = nullptr;
    }
  }
  cudaSetDevice(prev);
  cudaGetLastError();
  return KDE_OK;
}

int64_t kde_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int kde_grid_binned(const double* points, const int64_t* traj_offsets, int64_t ntraj, int64_t n,
                    const double grid_origin[2], double cell, int nx, int ny, double h,
                    int kernel_id, int window, int interpolate, int32_t* counts_out, float* out,
                    int64_t* interpolated, const kde_opts* opts) {
  if (!grid_origin) return fail(KDE_EINVAL, "grid_origin is NULL");
  kde_args a;
  a.points = points;
  a.weights = nullptr;
  a.n = n;
  a.origin_x = grid_origin[0];
  a.origin_y = grid_origin[1];
  a.cell = cell;
  a.nx = nx;
  a.ny = ny;
  a.h = h;
  a.kernel_id = kernel_id;
  a.out = out;
  int rc = validate(&a, nullptr);
  if (rc) return rc;
  if (kernel_id > 7) return fail(KDE_EINVAL, "the binned estimator takes the Table 1 kernels (0..7)");
  if (traj_offsets && ntraj < 1) return fail(KDE_EINVAL, "ntraj must be >= 1 with offsets");
  if (ny > 64 * 65535) return fail(KDE_EINVAL, "ny = %d exceeds 4194240 rows", ny);
  if (window < 0 || (window > 0 && ((window & 1) == 0 || window > 255)))
    return fail(KDE_EINVAL, "window must be 0 (automatic) or odd and <= 255");
  if ((n > 0 && memory_kind(points) != 0) || memory_kind(out) != 0 ||
      (traj_offsets && memory_kind(traj_offsets) != 0) ||
      (counts_out && memory_kind(counts_out) != 0))
    return fail(KDE_EINVAL, "kde_grid_binned needs device pointers");
  if ((traj_offsets && (reinterpret_cast<uintptr_t>(traj_offsets) & 7)) ||
      (counts_out && (reinterpret_cast<uintptr_t>(counts_out) & 3)))
    return fail(KDE_EINVAL, "misaligned offsets or counts");
  cudaStream_t s = stream_of(opts);
  const int64_t cells = (int64_t)nx * ny;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = align256(off + bytes); return r; };
  const size_t o_added = take(sizeof(unsigned long long));
  const size_t o_counts = take(counts_out ? 0 : sizeof(int) * (size_t)cells);
  const size_t o_rows = take(sizeof(float) * (size_t)cells);
  void* wsv = nullptr;
  rc = acquire_workspace(opts, off, s, &wsv);
  if (rc) return rc;
  char* base = static_cast<char*>(wsv);
  int* counts = counts_out ? reinterpret_cast<int*>(counts_out) : reinterpret_cast<int*>(base + o_counts);
  unsigned long long* added = reinterpret_cast<unsigned long long*>(base + o_added);
  const int win = binned_window(kernel_id, h, cell, window);
  KDE_CUDA(launch_binned(points, n, traj_offsets, ntraj, grid_origin[0], grid_origin[1], cell, nx,
                         ny, h, kernel_id, win, interpolate, counts,
                         reinterpret_cast<float*>(base + o_rows), added, out, s),
           "binned estimator");
  if (interpolated || (opts && (opts->flags & KDE_FLAG_SYNC))) {
    unsigned long long hv = 0;
    KDE_CUDA(cudaMemcpyAsync(&hv, added, sizeof(hv), cudaMemcpyDeviceToHost, s), "read count");
    KDE_CUDA(cudaStreamSynchronize(s), "synchronize");
    if (interpolated) *interpolated = (int64_t)hv;
  }
  g_err[0] = 0;
  return KDE_OK;
}

int kde_dp_simplify(const double* points, const int64_t* traj_offsets, int64_t ntraj, int64_t n,
                    double eps, uint8_t* keep, double* out_points, int64_t* out_offsets,
                    int64_t* n_kept, int* iterations, const kde_opts* opts) {
  if (n < 0 || n >= ((int64_t)1 << 31) - 1)
    return fail(KDE_EINVAL, "n = %lld must be in [0, 2^31 - 1)", (long long)n);
  if (n > 0 && (!points || !keep)) return fail(KDE_EINVAL, "points or keep is NULL with n > 0");
  if (!(eps >= 0.0) || !isfinite(eps)) return fail(KDE_EINVAL, "eps must be finite and >= 0");
  if (traj_offsets && ntraj < 1) return fail(KDE_EINVAL, "ntraj must be >= 1 with offsets");
  if (out_offsets && !traj_offsets && ntraj != 1)
    return fail(KDE_EINVAL, "out_offsets without traj_offsets needs ntraj = 1");
  if (!traj_offsets) ntraj = 1;
  if ((points && (reinterpret_cast<uintptr_t>(points) & 15)) ||
      (out_points && (reinterpret_cast<uintptr_t>(out_points) & 15)) ||
      (traj_offsets && (reinterpret_cast<uintptr_t>(traj_offsets) & 7)) ||
      (out_offsets && (reinterpret_cast<uintptr_t>(out_offsets) & 7)))
    return fail(KDE_EINVAL, "points must be 16-byte and offsets 8-byte aligned");
  const void* dev_ptrs[] = {points, keep, out_points, traj_offsets, out_offsets};
  for (const void* q : dev_ptrs)
    if (q && n > 0 && memory_kind(q) != 0)
      return fail(KDE_EINVAL, "kde_dp_simplify needs device pointers");
  cudaStream_t s = stream_of(opts);
  const size_t need = align256(sizeof(CallScalars)) + dp_workspace_bytes(n);
  void* wsv = nullptr;
  int rc = acquire_workspace(opts, need, s, &wsv);
  if (rc) return rc;
  CallScalars* scal = static_cast<CallScalars*>(wsv);
  KDE_CUDA(cudaMemsetAsync(scal, 0, sizeof(CallScalars), s), "clear scalars");
  int64_t kept = 0;
  int its = 0;
  KDE_CUDA(launch_dp(points, n, traj_offsets, ntraj, eps, keep, out_points, out_offsets,
                     static_cast<char*>(wsv) + align256(sizeof(CallScalars)), scal, &kept, &its, s),
           "Douglas-Peucker");
  CallScalars hs;
  KDE_CUDA(cudaMemcpyAsync(&hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s), "read status");
  KDE_CUDA(cudaStreamSynchronize(s), "synchronize");
  if (hs.err & kErrNonFinite) return fail(KDE_EDATA, "non-finite coordinate");
  if (hs.err & kErrBadArg) return fail(KDE_EINVAL, "traj_offsets must rise from 0 to n");
  if (n_kept) *n_kept = kept;
  if (iterations) *iterations = its;
  g_err[0] = 0;
  return KDE_OK;
}

int kde_diag_wait_timeout(int64_t limit_ns, void* stream) {
  if (limit_ns < 1000 || limit_ns > 2000000000ll)
    return fail(KDE_EINVAL, "limit_ns must be in [1 us, 2 s]");
  void* ws = nullptr;
  int rc = library_workspace(sizeof(CallScalars), &ws);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CallScalars* scal = static_cast<CallScalars*>(ws);
  KDE_CUDA(cudaMemsetAsync(scal, 0, sizeof(CallScalars), s), "clear scalars");
  KDE_CUDA(launch_wait_timeout(scal, (uint64_t)limit_ns, s), "timeout diagnostic");
  CallScalars hs;
  KDE_CUDA(cudaMemcpyAsync(&hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s), "read status");
  KDE_CUDA(cudaStreamSynchronize(s), "synchronize");
  if (hs.err & kErrTimeout)
    return fail(KDE_ETIMEOUT, "a device-side wait gave up (role %d)", hs.timeout_where);
  g_err[0] = 0;
  return KDE_OK;
}

int kde_diag_sort_wait_timeout(int64_t limit_ns, void* stream) {
  if (limit_ns < 1000 || limit_ns > 2000000000ll)
    return fail(KDE_EINVAL, "limit_ns must be in [1 us, 2 s]");
  void* ws = nullptr;
  const size_t o_buf = align256(sizeof(CallScalars));
  int rc = library_workspace(o_buf + sizeof(uint32_t) * lookback_probe_words(), &ws);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CallScalars* scal = static_cast<CallScalars*>(ws);
  uint32_t* buf = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + o_buf);
  KDE_CUDA(cudaMemsetAsync(scal, 0, sizeof(CallScalars), s), "clear scalars");
  KDE_CUDA(launch_lookback_timeout_probe(buf, scal, (uint64_t)limit_ns, s), "look-back diagnostic");
  CallScalars hs;
  KDE_CUDA(cudaMemcpyAsync(&hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s), "read status");
  KDE_CUDA(cudaStreamSynchronize(s), "synchronize");
  if (hs.err & kErrTimeout)
    return fail(KDE_ETIMEOUT, "a device-side wait gave up (role %d)", hs.timeout_where);
  g_err[0] = 0;
  return KDE_OK;
}

int kde_diag_peak_rates(double* rates, void* stream) {
  if (!rates) return fail(KDE_EINVAL, "null pointer");
  void* ws = nullptr;
  int rc = library_workspace(sizeof(CallScalars) + 256 * sizeof(float), &ws);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CallScalars* scal = static_cast<CallScalars*>(ws);
  float* sink = reinterpret_cast<float*>(static_cast<char*>(ws) + sizeof(CallScalars));
  KDE_CUDA(cudaMemsetAsync(scal, 0, sizeof(CallScalars), s), "clear scalars");
  double r[3] = {0.0, 0.0, 0.0};
  KDE_CUDA(run_peak_probes(sm_count(), scal, sink, r, s), "peak probes");
  CallScalars hs;
  KDE_CUDA(cudaMemcpyAsync(&hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s), "read status");
  KDE_CUDA(cudaStreamSynchronize(s), "synchronize");
  if (hs.err & kErrTimeout)
    return fail(KDE_ETIMEOUT, "a device-side wait gave up (role %d)", hs.timeout_where);
  for (int k = 0; k < 3; ++k) rates[k] = r[k];
  g_err[0] = 0;
  return KDE_OK;
}

int kde_diag_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, int per_block,
                            void* stream) {
  if (n < 0 || per_block < 1 || per_block > 2048)
    return fail(KDE_EINVAL, "n must be >= 0 and per_block in [1, 2048]");
  if (n == 0) return KDE_OK;
  if (!in || !out) return fail(KDE_EINVAL, "null pointer");
  if (memory_kind(in) != 0 || memory_kind(out) != 0)
    return fail(KDE_EINVAL, "kde_diag_exclusive_scan needs device pointers");
  void* ws = nullptr;
  int rc = library_workspace(sizeof(uint32_t) * (scan_temp_words(n, per_block) + 64), &ws);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  KDE_CUDA(launch_exclusive_scan(in, out, n, per_block, static_cast<uint32_t*>(ws), s),
           "exclusive scan");
  KDE_CUDA(cudaStreamSynchronize(s), "synchronize");
  g_err[0] = 0;
  return KDE_OK;
}

const char* kde_version(void) { return "kde-gb300 0.1 (sm_103a)"; }

}  // extern "C"
