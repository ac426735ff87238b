// C ABI entry points: argument validation, workspace ownership, host-buffer
// staging, path dispatch and error reporting.  Every arithmetic step runs in
// the kernels of the other translation units.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "kde_internal.cuh"

namespace kde {

std::atomic<int64_t> g_launches{0};
void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {

thread_local char g_err[512] = "";

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

struct Plan {
  int path;
  int splits;
  int64_t n_pad;
  bool host_pts, host_w, host_out;
  TcPlan tc;
  CutoffPlan co;
  // byte offsets into the workspace
  size_t off_scal, off_pts, off_wts, off_gxt, off_gyt, off_part, off_hxy, off_hw, off_hout, total;
  size_t off_co_keys[2], off_co_vals[2], off_co_hist, off_co_hscan, off_co_stemp, off_co_start,
      off_co_spts, off_co_sw;
};

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
  if (a->kernel_id < 0 || a->kernel_id > 7)
    return fail(KDE_EINVAL, "kernel_id %d is not a Table 1 kernel (0..7)", a->kernel_id);
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
        a->kernel_id != KDE_GAUSSIAN)
      return fail(KDE_ENOTSUP, "tensor-core paths need the Gaussian kernel");
    if (o->path == KDE_PATH_CUTOFF && a->kernel_id == KDE_GAUSSIAN)
      return fail(KDE_ENOTSUP, "the cutoff path needs a compact-support kernel");
    if (o->split_k < 0 || o->split_k > 1024) return fail(KDE_EINVAL, "split_k out of range");
    if (o->k_chunk < 0 || (o->k_chunk % 32) != 0 || (o->k_chunk > 0 && o->k_chunk < 64))
      return fail(KDE_EINVAL, "k_chunk must be 0 or a multiple of 32 of at least 64");
    if (o->tile_n != 0 && o->tile_n != 128 && o->tile_n != 256)
      return fail(KDE_EINVAL, "tile_n must be 0, 128 or 256");
    if (o->stage_points != 0 && o->stage_points != 32 && o->stage_points != 64)
      return fail(KDE_EINVAL, "stage_points must be 0, 32 or 64");
    if (o->workspace && o->workspace_bytes == 0)
      return fail(KDE_EINVAL, "workspace given with zero size");
  }
  return KDE_OK;
}

int resolve_path(const kde_args* a, const kde_opts* o) {
  int path = o ? o->path : KDE_PATH_AUTO;
  if (path == KDE_PATH_AUTO)
    path = a->kernel_id == KDE_GAUSSIAN ? KDE_PATH_TC_SPLIT16 : KDE_PATH_CUTOFF;
  return path;
}

// Point-range splits for the persistent tensor-core kernel: the fewest
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

int make_plan(const kde_args* a, const kde_opts* o, bool probe_memory, Plan* p) {
  memset(p, 0, sizeof(*p));
  p->path = resolve_path(a, o);
  const int64_t n = a->n;
  p->n_pad = std::max<int64_t>(512, (n + 511) / 512 * 512);
  const int64_t cells = (int64_t)a->nx * a->ny;
  if (probe_memory) {
    p->host_pts = n > 0 && memory_kind(a->points) == 1;
    p->host_w = n > 0 && a->weights && memory_kind(a->weights) == 1;
    p->host_out = memory_kind(a->out) == 1;
  }
  const int sms = sm_count();
  int splits = o ? o->split_k : 0;
  if (p->path == KDE_PATH_SIMT_FP32) {
    if (splits == 0) {
      const int64_t tiles = (int64_t)((a->nx + 127) / 128) * ((a->ny + 63) / 64);
      const int64_t want = (6 * (int64_t)sms + tiles - 1) / tiles;
      const int64_t maxs = std::max<int64_t>(1, p->n_pad / 4096);
      splits = (int)std::max<int64_t>(1, std::min<int64_t>({want, maxs, 64}));
    }
  } else if (p->path == KDE_PATH_TC_FP16 || p->path == KDE_PATH_TC_SPLIT16) {
    TcPlan& t = p->tc;
    t.tile_n = (o && o->tile_n) ? o->tile_n : (a->ny <= 128 ? 128 : 256);
    t.split16 = p->path == KDE_PATH_TC_SPLIT16;
    // the tensor core's FP32 accumulation loses accuracy with every MMA step it
    // adds into a large sum, so split-FP16 drains its accumulators often
    t.k_chunk = (o && o->k_chunk) ? o->k_chunk : (t.split16 ? 256 : 1024);
    t.ctas = (o && o->max_ctas > 0) ? std::min(o->max_ctas, sms) : sms;
    t.skip_zero = (o && (o->flags & KDE_FLAG_SKIP_ZERO)) ? 1 : 0;
    // 64-point stages (128-byte rows): fewer barrier round trips per point
    // outweigh the deeper pipeline 32-point stages would allow
    t.stage_points = (o && o->stage_points) ? o->stage_points : 64;
    // two accumulator halves drained half a chunk apart need two stages per chunk
    if (t.k_chunk % t.stage_points || t.k_chunk < 2 * t.stage_points)
      return fail(KDE_EINVAL, "k_chunk %d must be a multiple of, and at least twice, the %d-point stage",
                  t.k_chunk, t.stage_points);
    const int64_t tiles = (int64_t)((a->nx + 127) / 128) * ((a->ny + t.tile_n - 1) / t.tile_n);
    if (splits == 0) splits = choose_tc_splits(tiles, t.ctas, p->n_pad);
    t.splits = splits;
  } else {
    splits = std::max(splits, 1);
  }
  p->splits = splits;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = align256(off + bytes); return r; };
  p->off_scal = take(sizeof(CallScalars));
  p->off_pts = take(sizeof(float4) * (size_t)p->n_pad);
  p->off_wts = take(sizeof(float) * (size_t)p->n_pad);
  p->off_gxt = take(sizeof(float2) * (size_t)a->nx);
  p->off_gyt = take(sizeof(float2) * (size_t)a->ny);
  p->off_part = take(p->splits > 1 ? sizeof(float) * (size_t)cells * p->splits : 0);
  p->off_hxy = take(p->host_pts ? sizeof(double) * 2 * (size_t)n : 0);
  p->off_hw = take(p->host_w ? sizeof(float) * (size_t)n : 0);
  p->off_hout = take(p->host_out ? sizeof(float) * (size_t)cells : 0);
  if (p->path == KDE_PATH_CUTOFF) {
    p->co = plan_cutoff(a->nx, a->ny, a->cell, a->h, p->n_pad);
    const size_t u = sizeof(uint32_t);
    for (int k = 0; k < 2; ++k) {
      p->off_co_keys[k] = take(u * (size_t)p->n_pad);
      p->off_co_vals[k] = take(u * (size_t)p->n_pad);
    }
    p->off_co_hist = take(u * p->co.hist_words);
    p->off_co_hscan = take(u * p->co.hist_words);
    p->off_co_stemp = take(u * (p->co.scan_words + 64));
    p->off_co_start = take(u * ((size_t)p->co.nbins + 1));
    p->off_co_spts = take(sizeof(float4) * (size_t)p->n_pad);
    p->off_co_sw = take(sizeof(float) * (size_t)p->n_pad);
  }
  p->total = off;
  return KDE_OK;
}

cudaStream_t stream_of(const kde_opts* o) {
  return o ? reinterpret_cast<cudaStream_t>(o->stream) : (cudaStream_t)0;
}

int run_grid(const kde_args* a, const kde_opts* o, bool force_sync) {
  int rc = validate(a, o);
  if (rc) return rc;
  Plan pl;
  rc = make_plan(a, o, true, &pl);
  if (rc) return rc;
  cudaStream_t s = stream_of(o);
  const bool sync = force_sync || (o && (o->flags & KDE_FLAG_SYNC)) || pl.host_out;
  const int64_t cells = (int64_t)a->nx * a->ny;

  void* ws = nullptr;
  if (o && o->workspace) {
    if (o->workspace_bytes < pl.total)
      return fail(KDE_ENOMEM, "caller workspace has %zu bytes, %zu needed", o->workspace_bytes,
                  pl.total);
    ws = o->workspace;
  } else {
    rc = library_workspace(pl.total, &ws);
    if (rc) return rc;
  }
  char* base = static_cast<char*>(ws);
  CallScalars* scal = reinterpret_cast<CallScalars*>(base + pl.off_scal);
  float* out_dev = pl.host_out ? reinterpret_cast<float*>(base + pl.off_hout) : a->out;

  KDE_CUDA(cudaMemsetAsync(scal, 0, sizeof(CallScalars), s), "clear scalars");
  if (a->n == 0) {
    KDE_CUDA(cudaMemsetAsync(out_dev, 0, sizeof(float) * cells, s), "zero output");
  } else {
    const double* xy = a->points;
    const float* w = a->weights;
    if (pl.host_pts) {
      double* d = reinterpret_cast<double*>(base + pl.off_hxy);
      KDE_CUDA(cudaMemcpyAsync(d, xy, sizeof(double) * 2 * a->n, cudaMemcpyHostToDevice, s),
               "copy points to device");
      xy = d;
    }
    if (pl.host_w) {
      float* d = reinterpret_cast<float*>(base + pl.off_hw);
      KDE_CUDA(cudaMemcpyAsync(d, w, sizeof(float) * a->n, cudaMemcpyHostToDevice, s),
               "copy weights to device");
      w = d;
    }
    float4* pts = reinterpret_cast<float4*>(base + pl.off_pts);
    float* wts = reinterpret_cast<float*>(base + pl.off_wts);
    float2* gxt = reinterpret_cast<float2*>(base + pl.off_gxt);
    float2* gyt = reinterpret_cast<float2*>(base + pl.off_gyt);
    const double sigma = kernel_sigma(a->kernel_id, a->h);
    KDE_CUDA(launch_prepare(xy, w, a->n, pl.n_pad, a->origin_x, a->origin_y, sigma, pts, wts, scal, s),
             "prepare points");
    KDE_CUDA(launch_grid_tables(a->nx, a->ny, a->cell, sigma, gxt, gyt, s), "grid tables");
    const double c1 = kernel_const_1d(a->kernel_id);
    const float scale = (float)(c1 * c1 / ((double)a->n * a->h * a->h));
    float* part = pl.splits > 1 ? reinterpret_cast<float*>(base + pl.off_part) : out_dev;
    cudaEvent_t* ev = o ? static_cast<cudaEvent_t*>(o->timing_events) : nullptr;
    if (ev) KDE_CUDA(cudaEventRecord(ev[0], s), "record start event");
    switch (pl.path) {
      case KDE_PATH_SIMT_FP32:
        KDE_CUDA(launch_simt(a->kernel_id, pts, wts, pl.n_pad, gxt, gyt, a->nx, a->ny, pl.splits,
                             scale, part, s),
                 "SIMT direct sum");
        break;
      case KDE_PATH_TC_FP16:
      case KDE_PATH_TC_SPLIT16: {
        // c = 2^-30 / (2 pi N h^2); the kernel multiplies by max |w|
        const double base = 0x1p-30 / (2.0 * 3.14159265358979323846 * (double)a->n * a->h * a->h);
        KDE_CUDA(launch_tc(pl.tc, pts, wts, pl.n_pad, gxt, gyt, a->nx, a->ny, (float)base, scal,
                           part, scal, s),
                 "tensor-core contraction");
        break;
      }
      case KDE_PATH_CUTOFF: {
        CutoffScratch cs;
        for (int k = 0; k < 2; ++k) {
          cs.keys[k] = reinterpret_cast<uint32_t*>(base + pl.off_co_keys[k]);
          cs.vals[k] = reinterpret_cast<uint32_t*>(base + pl.off_co_vals[k]);
        }
        cs.hist = reinterpret_cast<uint32_t*>(base + pl.off_co_hist);
        cs.hist_scan = reinterpret_cast<uint32_t*>(base + pl.off_co_hscan);
        cs.scan_temp = reinterpret_cast<uint32_t*>(base + pl.off_co_stemp);
        cs.start = reinterpret_cast<uint32_t*>(base + pl.off_co_start);
        cs.spts = reinterpret_cast<float4*>(base + pl.off_co_spts);
        cs.sw = reinterpret_cast<float*>(base + pl.off_co_sw);
        KDE_CUDA(launch_cutoff(a->kernel_id, pl.co, pts, wts, a->n, pl.n_pad, a->cell, a->h, gxt,
                               gyt, a->nx, a->ny, scale, cs, part, s),
                 "cutoff evaluation");
        break;
      }
      default:
        return fail(KDE_ENOTSUP, "path %d is not available in this build", pl.path);
    }
    if (ev) KDE_CUDA(cudaEventRecord(ev[1], s), "record end event");
    if (pl.splits > 1)
      KDE_CUDA(launch_reduce_splits(part, pl.splits, cells, out_dev, s), "split-K reduce");
  }
  if (pl.host_out)
    KDE_CUDA(cudaMemcpyAsync(a->out, out_dev, sizeof(float) * cells, cudaMemcpyDeviceToHost, s),
             "copy result to host");
  if (sync) {
    CallScalars hs;
    KDE_CUDA(cudaMemcpyAsync(&hs, scal, sizeof(int) * 3, cudaMemcpyDeviceToHost, s), "read status");
    KDE_CUDA(cudaStreamSynchronize(s), "synchronize");
    if (hs.err & kErrTimeout)
      return fail(KDE_ETIMEOUT, "a device-side wait gave up (role %d)", hs.timeout_where);
    if (hs.err & kErrNonFinite) return fail(KDE_EDATA, "non-finite coordinate or weight");
    if (hs.err & kErrNegWeight)
      return fail(KDE_EDATA, "the tensor-core paths need non-negative weights");
    if (hs.err) return fail(KDE_ECUDA, "device error word 0x%x", hs.err);
  }
  g_err[0] = 0;
  return KDE_OK;
}

}  // namespace
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
  return run_grid(&a, &o, true);
}

int kde_grid_ex(const kde_args* a, const kde_opts* opts) { return run_grid(a, opts, false); }

int kde_workspace_size(const kde_args* a, const kde_opts* opts, size_t* bytes) {
  if (!bytes) return fail(KDE_EINVAL, "bytes is NULL");
  int rc = validate(a, opts);
  if (rc) return rc;
  Plan pl;
  rc = make_plan(a, opts, true, &pl);
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
  (void)inst;
  (void)count;
  (void)opts;
  return fail(KDE_ENOTSUP, "kde_grid_batched is not available in this build");
}

int kde_grid_backward(const kde_args* a, const float* grad_out, float* grad_points,
                      float* grad_weights, double* grad_h, const kde_opts* opts) {
  (void)a;
  (void)grad_out;
  (void)grad_points;
  (void)grad_weights;
  (void)grad_h;
  (void)opts;
  return fail(KDE_ENOTSUP, "kde_grid_backward is not available in this build");
}

int kde_lscv_grid(const kde_args* a, const float* F, double* loss, float* grad_F,
                  float* grad_w_direct, float* grad_points_direct, double* grad_h_direct,
                  const kde_opts* opts) {
  (void)a;
  (void)F;
  (void)loss;
  (void)grad_F;
  (void)grad_w_direct;
  (void)grad_points_direct;
  (void)grad_h_direct;
  (void)opts;
  return fail(KDE_ENOTSUP, "kde_lscv_grid is not available in this build");
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
  }
  cudaSetDevice(prev);
  cudaGetLastError();
  return KDE_OK;
}

int64_t kde_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

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
