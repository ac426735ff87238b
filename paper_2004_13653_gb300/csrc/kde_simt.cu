// Path (a): FP32 direct sum on the CUDA cores, any Table 1 kernel.
//
// Every Table 1 kernel is a product f(s,t) = k(s) k(t) (Sec. III-C).  A CTA
// owns 128 x 64 cells; for each batch of 32 points it first tabulates the
// 128 x-factors and 64 (weighted) y-factors of every point in shared memory,
// each evaluated once, then every thread accumulates the outer products of its
// 8 x 8 cells (columns 4t..4t+3 and 64+4t..64+4t+3, eight consecutive rows):
// per point two 16-byte reads of each table and 64 FMAs.  The tables are
// double-buffered, so one barrier per batch separates a batch's tabulation
// from its use; each point's table reads are issued while the previous
// point's FMAs run, and the next batch's points are loaded into registers
// while the current batch is accumulated.  Points arrive in tiles of 256;
// each thread sums one tile in registers and adds that partial into a
// (hi, lo) running sum (in global scratch, or in shared memory for callers
// without scratch) with an error-free two-sum, so the result does not degrade
// with the number of points a cell sees.  The factors and the order of every sum are
// those of a thread that evaluates its own factors, so the result does not
// depend on the tabulation.
#include "kde_internal.cuh"
#include "kernel_factors.cuh"

namespace kde {
namespace {

constexpr int kThreads = 128;  // 16 (x) x 8 (y) threads, 8 x 8 cells each
constexpr int kTileX = 128;    // cells along x per CTA
constexpr int kTileY = 64;     // cells along y per CTA
constexpr int kPtsTile = 256;  // points per register partial (two-sum cadence)
constexpr int kBatch = 32;     // points per factor table
constexpr int kTable = kBatch * (kTileX + kTileY);  // floats per table buffer

struct TableRow {
  float4 xa, xb, ya, yb;
};

__device__ __forceinline__ TableRow table_row(const float* KX, const float* KY, int q, int tx,
                                              int ty) {
  // columns 4tx.. and 64+4tx..: a half-warp reads 256 contiguous bytes
  TableRow r;
  r.xa = *reinterpret_cast<const float4*>(KX + q * kTileX + tx * 4);
  r.xb = *reinterpret_cast<const float4*>(KX + q * kTileX + 64 + tx * 4);
  r.ya = *reinterpret_cast<const float4*>(KY + q * kTileY + ty * 8);
  r.yb = *reinterpret_cast<const float4*>(KY + q * kTileY + ty * 8 + 4);
  return r;
}

// GRUN: the (hi, lo) running sums live in global scratch (64 KB per CTA,
// touched once per 256 points, so they stay in L2), which leaves shared
// memory to the tables and three CTAs per SM; otherwise in shared memory (two
// CTAs per SM, for callers that give no scratch).
template <int KID, bool GRUN>
__global__ void __launch_bounds__(kThreads, GRUN ? 3 : 2)
    k_simt(const float4* __restrict__ pts, const float* __restrict__ wts, int64_t n_pad,
           int64_t per_split, const float2* __restrict__ gxt, const float2* __restrict__ gyt,
           int nx, int ny, float scale, float2* __restrict__ grun, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* tables = reinterpret_cast<float*>(smem);                        // [2][kTable]
  const int tid = threadIdx.x, lane = tid & 31;
  const int tx = tid & 15, ty = tid >> 4;
  const int cx0 = blockIdx.x * kTileX, cy0 = blockIdx.y * kTileY;
  // running sum of cell c = b * 8 + a of this thread: run[c * kThreads]
  float2* run;
  if (GRUN) {
    const int64_t cta = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    run = grun + cta * 64 * kThreads + tid;
  } else {
    run = reinterpret_cast<float2*>(tables + 2 * kTable) + tid;  // [64][kThreads]
  }
  float* dst = part + (int64_t)blockIdx.z * nx * ny;
  auto cell = [&](int b, int a, int& x, int& y) {
    y = cy0 + ty * 8 + b;
    x = cx0 + (a < 4 ? tx * 4 + a : 64 + tx * 4 + a - 4);
  };

  const int64_t p_begin = (int64_t)blockIdx.z * per_split;
  int64_t p_end = p_begin + per_split;
  if (p_end > n_pad) p_end = n_pad;
  if (p_begin >= p_end) {  // no points in this split: a zero partial
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        int x, y;
        cell(b, a, x, y);
        if (x < nx && y < ny) dst[(int64_t)y * nx + x] = 0.f;
      }
    return;
  }
  // factor roles: x column tid; y row frow for points fq0 .. fq0 + kBatch/2 - 1
  static_assert(kThreads == kTileX && kThreads == 2 * kTileY, "factor roles");
  static_assert(kPtsTile % kBatch == 0 && kBatch == 32, "one point per lane per batch");
  const float2 gxr = gxt[min(cx0 + tid, nx - 1)];
  const int frow = tid & (kTileY - 1), fq0 = (tid / kTileY) * (kBatch / 2);
  const float2 gyr = gyt[min(cy0 + frow, ny - 1)];

  // Every warp holds the points of the next batch in registers, one per
  // lane, loaded while the current batch is accumulated (the global-memory
  // latency hides behind a whole batch); the tabulation broadcasts them with
  // shuffles.
  float4 nP;
  float nW;
  auto fetch = [&](int64_t first) {
    const int64_t p = first + lane;
    const bool in = p < p_end;
    nP = in ? pts[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    nW = in ? wts[p] : 0.f;
  };
  fetch(p_begin);

  int buf = 0;
  for (int64_t base = p_begin; base < p_end; base += kPtsTile) {
    float acc[8][8];
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int a = 0; a < 8; ++a) acc[b][a] = 0.f;

    for (int bb = 0; bb < kPtsTile; bb += kBatch, buf ^= 1) {
      float* KX = tables + buf * kTable;  // [kBatch][kTileX]
      float* KY = KX + kBatch * kTileX;   // [kBatch][kTileY]
      const float4 P = nP;
      const float W = nW;
      // This buffer was last read two batches ago, before the barrier of the
      // previous batch, which every thread has passed.
#pragma unroll 8
      for (int q = 0; q < kBatch; ++q) {
        const float px = __shfl_sync(0xffffffffu, P.x, q), pxl = __shfl_sync(0xffffffffu, P.y, q);
        KX[q * kTileX + tid] = kfactor<KID>((gxr.x - px) + (gxr.y - pxl));
      }
#pragma unroll 8
      for (int k = 0; k < kBatch / 2; ++k) {
        const int q = fq0 + k;
        const float py = __shfl_sync(0xffffffffu, P.z, q), pyl = __shfl_sync(0xffffffffu, P.w, q);
        const float w = __shfl_sync(0xffffffffu, W, q);
        KY[q * kTileY + frow] = w * kfactor<KID>((gyr.x - py) + (gyr.y - pyl));
      }
      __syncthreads();
      fetch(base + bb + kBatch);
      TableRow cur = table_row(KX, KY, 0, tx, ty);
#pragma unroll 4
      for (int q = 0; q < kBatch; ++q) {
        TableRow nxt = cur;
        if (q + 1 < kBatch) nxt = table_row(KX, KY, q + 1, tx, ty);
        const float kx[8] = {cur.xa.x, cur.xa.y, cur.xa.z, cur.xa.w,
                             cur.xb.x, cur.xb.y, cur.xb.z, cur.xb.w};
        const float ky[8] = {cur.ya.x, cur.ya.y, cur.ya.z, cur.ya.w,
                             cur.yb.x, cur.yb.y, cur.yb.z, cur.yb.w};
#pragma unroll
        for (int b = 0; b < 8; ++b)
#pragma unroll
          for (int a = 0; a < 8; ++a) acc[b][a] = fmaf(kx[a], ky[b], acc[b][a]);
        cur = nxt;
      }
    }
    // this tile's partials into the running sums; after the last tile the
    // sums are the cells' results
    const bool first = base == p_begin, last = base + kPtsTile >= p_end;
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        float2 r = first ? make_float2(0.f, 0.f) : run[(b * 8 + a) * kThreads];
        two_sum_acc(r, acc[b][a]);
        if (last) {
          int x, y;
          cell(b, a, x, y);
          if (x < nx && y < ny) dst[(int64_t)y * nx + x] = (r.x + r.y) * scale;
        } else {
          run[(b * 8 + a) * kThreads] = r;
        }
      }
  }
}

// 48 KB of tables (+ 64 KB of running sums without global scratch)
constexpr size_t kSmemTables = 2 * kTable * sizeof(float);
constexpr size_t kSmemRun = 64 * kThreads * sizeof(float2);

template <int KID, bool GRUN>
cudaError_t launch_kid(const float4* pts, const float* wts, int64_t n_pad, const float2* gxt,
                       const float2* gyt, int nx, int ny, int splits, float scale, float2* grun,
                       float* part, cudaStream_t s) {
  const size_t smem = GRUN ? kSmemTables : kSmemTables + kSmemRun;
  // per-device attribute; cheap, so set on every launch
  cudaError_t e = cudaFuncSetAttribute(k_simt<KID, GRUN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t per = (n_pad + splits - 1) / splits;
  per = (per + kPtsTile - 1) / kPtsTile * kPtsTile;
  if (per < kPtsTile) per = kPtsTile;
  dim3 grid((nx + kTileX - 1) / kTileX, (ny + kTileY - 1) / kTileY, splits);
  k_simt<KID, GRUN><<<grid, kThreads, smem, s>>>(pts, wts, n_pad, per, gxt, gyt, nx, ny, scale,
                                                 grun, part);
  note_launches(1);
  return cudaGetLastError();
}

template <int KID>
cudaError_t launch_kid(const float4* pts, const float* wts, int64_t n_pad, const float2* gxt,
                       const float2* gyt, int nx, int ny, int splits, float scale, float2* grun,
                       float* part, cudaStream_t s) {
  return grun ? launch_kid<KID, true>(pts, wts, n_pad, gxt, gyt, nx, ny, splits, scale, grun,
                                      part, s)
              : launch_kid<KID, false>(pts, wts, n_pad, gxt, gyt, nx, ny, splits, scale, grun,
                                       part, s);
}

}  // namespace

size_t simt_scratch_bytes(int nx, int ny, int splits) {
  return (size_t)((nx + kTileX - 1) / kTileX) * ((ny + kTileY - 1) / kTileY) * splits * kSmemRun;
}

cudaError_t launch_simt(int kid, const float4* pts, const float* wts, int64_t n_pad,
                        const float2* gxt, const float2* gyt, int nx, int ny, int splits,
                        float scale, float2* scratch, float* part, cudaStream_t s) {
  switch (kid) {
#define KDE_CASE(K) \
  case K:           \
    return launch_kid<K>(pts, wts, n_pad, gxt, gyt, nx, ny, splits, scale, scratch, part, s);
    KDE_CASE(KDE_UNIFORM)
    KDE_CASE(KDE_TRIANGULAR)
    KDE_CASE(KDE_EPANECHNIKOV)
    KDE_CASE(KDE_QUARTIC)
    KDE_CASE(KDE_TRIWEIGHT)
    KDE_CASE(KDE_TRICUBE)
    KDE_CASE(KDE_GAUSSIAN)
    KDE_CASE(KDE_COSINE)
#undef KDE_CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace kde
