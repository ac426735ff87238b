// Path (c): the compact kernels of Table 1 evaluated over their support only.
//
// With the indicator of Eq. 8 a point contributes to the cells within one
// bandwidth of it.  The grid is cut into 32x32-cell bins; every point gets the
// key of its bin (points farther than a bandwidth outside the grid are
// dropped), the (key, index) pairs are sorted with a stable LSD radix sort,
// and each output bin is then computed by one CTA that reads the points of
// the bins within reach, in sorted order, a batch of 64 at a time: for each
// batch the CTA tabulates the x and y kernel factors of its 32 columns and 32
// rows in shared memory, and each thread adds the outer products into its
// four cells.  Nothing is accumulated with atomics, and the order of every
// sum is fixed, so results are reproducible bit for bit.
#include "kde_internal.cuh"
#include "kernel_factors.cuh"

namespace kde {
namespace {

constexpr int kBin = 32;            // cells per bin side (= output tile side)
constexpr int kSortThreads = 256;   // 8 warps
constexpr int kSortRounds = 8;      // 32-element rounds per warp
constexpr int kSortChunk = kSortThreads * kSortRounds;  // 2048 keys per block
constexpr int kBatch = 64;          // points per shared-memory batch

// Bin key of each point (centred, scaled by 1/h): key = by * nbx + bx, or
// nbins for padding and for points that cannot reach the grid.
__global__ void k_bin_keys(const float4* __restrict__ pts, int64_t n, int64_t n_pad,
                           double inv_binw, double ext_x, double ext_y, int nbx, int nby,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const uint32_t nbins = (uint32_t)nbx * nby;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += stride) {
    uint32_t key = nbins;
    if (p < n) {
      const float4 q = pts[p];
      const double X = (double)q.x + (double)q.y, Y = (double)q.z + (double)q.w;
      // a point reaches the grid only if it lies within one bandwidth (+ a cell) of it
      if (X >= -1.0 && Y >= -1.0 && X <= ext_x && Y <= ext_y) {
        const int bx = min(max((int)floor(X * inv_binw), 0), nbx - 1);
        const int by = min(max((int)floor(Y * inv_binw), 0), nby - 1);
        key = (uint32_t)by * nbx + bx;
      }
    }
    keys[p] = key;
    vals[p] = (uint32_t)p;
  }
}

// Rank of each key's digit among equal digits earlier in this block's chunk:
// each warp walks its 256 keys in rounds of 32, peers found with match_any,
// per-warp digit counts kept in shared memory.  Deterministic.
__device__ __forceinline__ void rank_digits(const uint32_t* __restrict__ keys, int64_t m,
                                            int64_t base, int shift,
                                            uint32_t (*cnt)[256], uint32_t (&digit)[kSortRounds],
                                            uint32_t (&rank)[kSortRounds]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t e = base + (int64_t)warp * 32 * kSortRounds + r * 32 + lane;
    const bool valid = e < m;
    const uint32_t d = valid ? (keys[e] >> shift) & 255u : 0u;
    const uint32_t active = __ballot_sync(0xffffffffu, valid);
    uint32_t peers = 0, old = 0;
    if (valid) {
      peers = __match_any_sync(active, d);
      old = cnt[warp][d];
    }
    __syncwarp();
    if (valid && lane == 31 - __clz(peers)) cnt[warp][d] = old + __popc(peers);
    __syncwarp();
    digit[r] = valid ? d : 0xffffffffu;
    rank[r] = old + __popc(peers & lt);
  }
}

__global__ void __launch_bounds__(kSortThreads)
    k_radix_count(const uint32_t* __restrict__ keys, int64_t m, int shift, int nchunks,
                  uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[kSortThreads / 32][256];
  for (int i = threadIdx.x; i < (kSortThreads / 32) * 256; i += kSortThreads) (&cnt[0][0])[i] = 0;
  __syncthreads();
  uint32_t digit[kSortRounds], rank[kSortRounds];
  rank_digits(keys, m, (int64_t)blockIdx.x * kSortChunk, shift, cnt, digit, rank);
  __syncthreads();
  const int d = threadIdx.x;  // 256 threads, one digit each
  uint32_t sum = 0;
  for (int w = 0; w < kSortThreads / 32; ++w) sum += cnt[w][d];
  hist[(int64_t)d * nchunks + blockIdx.x] = sum;
}

__global__ void __launch_bounds__(kSortThreads)
    k_radix_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                    int64_t m, int shift, int nchunks, const uint32_t* __restrict__ offs,
                    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
  __shared__ uint32_t cnt[kSortThreads / 32][256];
  for (int i = threadIdx.x; i < (kSortThreads / 32) * 256; i += kSortThreads) (&cnt[0][0])[i] = 0;
  __syncthreads();
  uint32_t digit[kSortRounds], rank[kSortRounds];
  const int64_t base = (int64_t)blockIdx.x * kSortChunk;
  rank_digits(keys, m, base, shift, cnt, digit, rank);
  __syncthreads();
  {  // exclusive prefix of the per-warp counts, per digit
    const int d = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) {
      const uint32_t c = cnt[w][d];
      cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    if (digit[r] == 0xffffffffu) continue;
    const int64_t e = base + (int64_t)warp * 32 * kSortRounds + r * 32 + lane;
    const uint32_t pos =
        offs[(int64_t)digit[r] * nchunks + blockIdx.x] + cnt[warp][digit[r]] + rank[r];
    keys_out[pos] = keys[e];
    vals_out[pos] = vals[e];
  }
}

// start[k] = first position whose key >= k in the sorted keys (k = 0..nbins).
__global__ void k_bin_bounds(const uint32_t* __restrict__ skeys, int64_t m, int nbins,
                             uint32_t* __restrict__ start) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > nbins) return;
  int64_t lo = 0, hi = m;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (skeys[mid] < (uint32_t)k) lo = mid + 1; else hi = mid;
  }
  start[k] = (uint32_t)lo;
}

__global__ void k_permute(const float4* __restrict__ pts, const float* __restrict__ wts,
                          const uint32_t* __restrict__ order, int64_t count,
                          float4* __restrict__ pts_out, float* __restrict__ w_out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const uint32_t src = order[i];
    pts_out[i] = pts[src];
    w_out[i] = wts[src];
  }
}

// One CTA per 32x32 output bin; thread (cx, 4 rows).
template <int KID>
__global__ void __launch_bounds__(256)
    k_cutoff(const float4* __restrict__ P, const float* __restrict__ W,
             const uint32_t* __restrict__ start, int nbx, int nby, int R,
             const float2* __restrict__ gxt, const float2* __restrict__ gyt, int nx, int ny,
             float scale, float* __restrict__ out) {
  __shared__ float4 sP[kBatch];
  __shared__ float sW[kBatch];
  __shared__ __align__(16) float KX[kBatch][kBin];
  __shared__ __align__(16) float KY[kBatch][kBin];
  __shared__ float2 sgx[kBin], sgy[kBin];
  const int bx = blockIdx.x, by = blockIdx.y;
  const int x0 = bx * kBin, y0 = by * kBin;
  const int t = threadIdx.x;
  const int cx = t & 31, cy0 = (t >> 5) * 4;
  if (t < kBin) sgx[t] = gxt[min(x0 + t, nx - 1)];
  else if (t < 2 * kBin) sgy[t - kBin] = gyt[min(y0 + t - kBin, ny - 1)];
  float2 run[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) run[r] = make_float2(0.f, 0.f);
  // evaluation role: point c = t / 4, eight columns / rows starting at j0
  const int ec = t >> 2, ej0 = (t & 3) * 8;

  for (int qy = max(by - R, 0); qy <= min(by + R, nby - 1); ++qy) {
    const int qx0 = max(bx - R, 0), qx1 = min(bx + R, nbx - 1);
    const uint32_t s = start[qy * nbx + qx0], e = start[qy * nbx + qx1 + 1];
    for (uint32_t b = s; b < e; b += kBatch) {
      const int cnt = (int)min((uint32_t)kBatch, e - b);
      __syncthreads();  // previous batch fully consumed
      if (t < cnt) {
        sP[t] = P[b + t];
        sW[t] = W[b + t];
      }
      __syncthreads();
      if (ec < cnt) {
        const float4 p = sP[ec];
        const float w = sW[ec];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float2 gx = sgx[ej0 + j], gy = sgy[ej0 + j];
          KX[ec][ej0 + j] = kfactor<KID>((gx.x - p.x) + (gx.y - p.y));
          KY[ec][ej0 + j] = w * kfactor<KID>((gy.x - p.z) + (gy.y - p.w));
        }
      }
      __syncthreads();
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int c = 0; c < cnt; ++c) {
        const float kx = KX[c][cx];
        const float4 ky = *reinterpret_cast<const float4*>(&KY[c][cy0]);
        acc[0] = fmaf(kx, ky.x, acc[0]);
        acc[1] = fmaf(kx, ky.y, acc[1]);
        acc[2] = fmaf(kx, ky.z, acc[2]);
        acc[3] = fmaf(kx, ky.w, acc[3]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) two_sum_acc(run[r], acc[r]);
    }
  }
  const int x = x0 + cx;
  if (x < nx) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int y = y0 + cy0 + r;
      if (y < ny) out[(int64_t)y * nx + x] = (run[r].x + run[r].y) * scale;
    }
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace

CutoffPlan plan_cutoff(int nx, int ny, double cell, double h, int64_t n_pad) {
  CutoffPlan c;
  c.nbx = (nx + kBin - 1) / kBin;
  c.nby = (ny + kBin - 1) / kBin;
  c.nbins = c.nbx * c.nby;
  // bins a point can reach: its support (h) plus half a cell, in 32-cell bins
  c.R = (int)ceil((h / cell + 1.0) / kBin);
  c.nchunks = (int)((n_pad + kSortChunk - 1) / kSortChunk);
  int bits = 1;
  while ((1ll << bits) <= (long long)c.nbins) ++bits;  // keys 0..nbins
  c.passes = (bits + 7) / 8;
  c.hist_words = (size_t)256 * c.nchunks;
  c.scan_words = scan_temp_words((int64_t)c.hist_words, 2048);
  return c;
}

cudaError_t launch_cutoff(int kid, const CutoffPlan& c, const float4* pts, const float* wts,
                          int64_t n, int64_t n_pad, double cell, double h, const float2* gxt,
                          const float2* gyt, int nx, int ny, float scale, CutoffScratch ws,
                          float* out, cudaStream_t s) {
  const double cell_s = cell / h;  // cell side in bandwidths
  k_bin_keys<<<grid_for(n_pad), 256, 0, s>>>(pts, n, n_pad, 1.0 / (kBin * cell_s),
                                             nx * cell_s + 1.0, ny * cell_s + 1.0, c.nbx, c.nby,
                                             ws.keys[0], ws.vals[0]);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int cur = 0;
  for (int pass = 0; pass < c.passes; ++pass) {
    const int shift = 8 * pass;
    k_radix_count<<<c.nchunks, kSortThreads, 0, s>>>(ws.keys[cur], n_pad, shift, c.nchunks, ws.hist);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_exclusive_scan(ws.hist, ws.hist_scan, (int64_t)c.hist_words, 2048, ws.scan_temp, s);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<c.nchunks, kSortThreads, 0, s>>>(ws.keys[cur], ws.vals[cur], n_pad, shift,
                                                        c.nchunks, ws.hist_scan, ws.keys[cur ^ 1],
                                                        ws.vals[cur ^ 1]);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cur ^= 1;
  }
  k_bin_bounds<<<(c.nbins + 1 + 255) / 256, 256, 0, s>>>(ws.keys[cur], n_pad, c.nbins, ws.start);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // only points that reach the grid are gathered: the first start[nbins] of the order
  k_permute<<<grid_for(n_pad), 256, 0, s>>>(pts, wts, ws.vals[cur], n_pad, ws.spts, ws.sw);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  dim3 grid(c.nbx, c.nby);
  switch (kid) {
#define KDE_CASE(K)                                                                              \
  case K:                                                                                        \
    k_cutoff<K><<<grid, 256, 0, s>>>(ws.spts, ws.sw, ws.start, c.nbx, c.nby, c.R, gxt, gyt, nx, \
                                     ny, scale, out);                                            \
    break;
    KDE_CASE(KDE_UNIFORM)
    KDE_CASE(KDE_TRIANGULAR)
    KDE_CASE(KDE_EPANECHNIKOV)
    KDE_CASE(KDE_QUARTIC)
    KDE_CASE(KDE_TRIWEIGHT)
    KDE_CASE(KDE_TRICUBE)
    KDE_CASE(KDE_COSINE)
#undef KDE_CASE
    default:
      return cudaErrorInvalidValue;
  }
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace kde
