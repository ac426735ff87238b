// kde_grid_noalloc: the FP32 SIMT density for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc: code running inside a stream capture
// that forbids allocation, real-time loops that may not block on the
// allocator, plugins whose host application owns every device allocation, or
// processes whose memory budget is fixed up front.  This entry point
// therefore allocates nothing.  Its scratch (prepared points, cell-centre
// tables and status words) lives in one file-scope device array of fixed size,
// reserved on every GPU that loads the library for as long as the process
// lives.  The caller still provides the points, the weights and the output.
//
// Limits and rules:
//   * the scratch holds kNoAllocScratchBytes; inputs needing more are rejected
//     with KDE_EINVAL before any launch (the point count is checked before any
//     size is computed from it, so no size can wrap around);
//   * every call on a device shares the array and it keeps the last call's
//     contents: the status words are cleared at the start of each call, and
//     calls that overlap on the GPU (different streams, or host threads that
//     do not serialise) race on it;
//   * the array's device address is looked up once per device ordinal, on the
//     first call made with that device current, and kept for the life of the
//     process; make that first call before any stream capture.  A device
//     reset (cudaDeviceReset) or a non-primary driver context invalidates the
//     kept address, so neither is supported.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "kde_internal.cuh"

namespace kde {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;  // 8 MiB per device
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDev = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDev] = {};

int noalloc_fail(int code, const char* msg) {
  set_error_message(msg);
  return code;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// Where each part of one call lives in the scratch.
struct NoAllocLayout {
  int64_t n_pad;
  size_t off_scal, off_tab, off_pts, off_wts, off_gxt, off_gyt, need;
};

// Most points the scratch can hold (20 bytes each: a float4 and a weight).
constexpr int64_t kNoAllocMaxPoints = (int64_t)(kNoAllocScratchBytes / 20);

// The scratch layout for n points on an nx x ny grid (host only).  Returns
// false, without forming any offset, when n alone exceeds the scratch, so no
// size computed here can wrap around; otherwise L->need says whether the
// whole layout fits.
bool noalloc_layout(int64_t n, int nx, int ny, NoAllocLayout* L) {
  if (n < 0 || n > kNoAllocMaxPoints || nx <= 0 || ny <= 0) return false;
  L->n_pad = n < 512 ? 512 : (n + 511) / 512 * 512;
  L->off_scal = 0;
  L->off_tab = up256(L->off_scal + sizeof(CallScalars));
  L->off_pts = up256(L->off_tab + sizeof(PrepInst));
  L->off_wts = up256(L->off_pts + sizeof(float4) * (size_t)L->n_pad);
  L->off_gxt = up256(L->off_wts + sizeof(float) * (size_t)L->n_pad);
  L->off_gyt = up256(L->off_gxt + sizeof(float2) * (size_t)nx);
  L->need = up256(L->off_gyt + sizeof(float2) * (size_t)ny);
  return true;
}

bool device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device address of the static scratch on the current device (set up once per
// device: the symbol's name in host code is not a device address).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
    return noalloc_fail(KDE_ECUDA, "kde_grid_noalloc: no current CUDA device");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(KDE_ECUDA, "kde_grid_noalloc: cudaGetSymbolAddress of the scratch failed");
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return KDE_OK;
}

}  // namespace

}  // namespace kde

using namespace kde;

extern "C" int kde_grid_noalloc(const double* points, const float* weights, int64_t n,
                                const double grid_origin[2], double cell, int nx, int ny,
                                double h, int kernel_id, float* out, void* stream) {
  set_error_message("");
  if (n < 0 || (n > 0 && !points) || !out || !grid_origin)
    return noalloc_fail(KDE_EINVAL, "kde_grid_noalloc: null pointer or negative n");
  if (nx <= 0 || ny <= 0 || (int64_t)nx * ny >= ((int64_t)1 << 31))
    return noalloc_fail(KDE_EINVAL, "kde_grid_noalloc: grid size out of range");
  if (!(cell > 0) || !isfinite(cell) || !(h > 0) || !isfinite(h) || !isfinite(grid_origin[0]) ||
      !isfinite(grid_origin[1]))
    return noalloc_fail(KDE_EINVAL, "kde_grid_noalloc: cell, h and origin must be finite, "
                                    "cell and h positive");
  // the radial Gaussian is the product Gaussian; the radial compact kernels
  // need the cutoff path, which this entry point does not run
  if (kernel_id == kRadial + KDE_GAUSSIAN) kernel_id = KDE_GAUSSIAN;
  if (kernel_id < 0 || kernel_id > 7)
    return noalloc_fail(KDE_EINVAL, "kde_grid_noalloc: kernel_id is not a Table 1 kernel "
                                    "(0..7) or the radial Gaussian (14)");
  if ((points && (reinterpret_cast<uintptr_t>(points) & 15)) ||
      (weights && (reinterpret_cast<uintptr_t>(weights) & 3)) ||
      (reinterpret_cast<uintptr_t>(out) & 3))
    return noalloc_fail(KDE_EINVAL, "kde_grid_noalloc: misaligned pointer");
  NoAllocLayout L;
  if (!noalloc_layout(n, nx, ny, &L) || L.need > kNoAllocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "kde_grid_noalloc: %lld points on a %d x %d grid exceed the static maximum of %zu "
             "bytes of scratch (at most %lld points, fewer on large grids)",
             (long long)n, nx, ny, kNoAllocScratchBytes, (long long)kNoAllocMaxPoints);
    return noalloc_fail(KDE_EINVAL, msg);
  }
  if ((n > 0 && !device_pointer(points)) || (n > 0 && weights && !device_pointer(weights)) ||
      !device_pointer(out))
    return noalloc_fail(KDE_EINVAL, "kde_grid_noalloc: points, weights and out must be device memory");

  const int64_t n_pad = L.n_pad;
  const size_t off_scal = L.off_scal, off_tab = L.off_tab, off_pts = L.off_pts,
               off_wts = L.off_wts, off_gxt = L.off_gxt, off_gyt = L.off_gyt;
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  char* base = static_cast<char*>(scratch);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  PrepInst q = {};
  q.xy = points;
  q.w = weights;
  q.pts = reinterpret_cast<float4*>(base + off_pts);
  q.wts = reinterpret_cast<float*>(base + off_wts);
  q.gxt = reinterpret_cast<float2*>(base + off_gxt);
  q.gyt = reinterpret_cast<float2*>(base + off_gyt);
  q.scal = reinterpret_cast<CallScalars*>(base + off_scal);
  q.n = n;
  q.n_pad = n_pad;
  q.begin = 0;
  q.ox = grid_origin[0];
  q.oy = grid_origin[1];
  q.sigma = kernel_sigma(kernel_id, h);
  q.cell_sigma = cell * q.sigma;
  q.nx = nx;
  q.ny = ny;
  const double c1 = kernel_const_1d(kernel_id);
  const float scale = n > 0 ? (float)(c1 * c1 / ((double)n * h * h)) : 0.0f;

  cudaError_t e = cudaMemsetAsync(q.scal, 0, sizeof(CallScalars), s);
  if (e == cudaSuccess)
    e = launch_upload(&q, sizeof(q), base + off_tab, s);
  if (e == cudaSuccess)
    e = launch_prepare(reinterpret_cast<const PrepInst*>(base + off_tab), 1, n_pad,
                       nx > ny ? nx : ny, s);
  if (e == cudaSuccess)  // one point split: the kernel writes `out` directly
    e = launch_simt(kernel_id, q.pts, q.wts, n_pad, q.gxt, q.gyt, nx, ny, 1, scale, nullptr, out, s);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "kde_grid_noalloc: %s", cudaGetErrorString(e));
    return noalloc_fail(KDE_ECUDA, msg);
  }
  return KDE_OK;
}
