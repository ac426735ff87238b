// Path (c): the compact kernels of Table 1 evaluated over their support only.
//
// With the indicator of Eq. 8 a point contributes to the cells within one
// bandwidth of it.  Every point gets the key of its sort bin (4, 8 or 16
// cells a side, chosen from the bandwidth; points farther than a bandwidth
// outside the grid are dropped), the (key, index) pairs are sorted with a
// stable LSD radix sort, and each 16x16-cell output block is then computed by
// one CTA that reads the points of the sort bins within reach of its cells,
// in sorted order: its eight warps take 32-point batches in turn, tabulate
// the x and y kernel factors of the block's 16 columns and 16 rows in shared
// memory, and each thread adds the outer products into its eight cells.  The
// blocks run heaviest first.  Nothing is accumulated with atomics, and the
// order of every sum is fixed, so results are reproducible bit for bit.  The
// same sort, with 32-cell bins and a wider reach, orders the points of the
// block-sparse tensor-core path.
#include "kde_internal.cuh"
#include "kernel_factors.cuh"

namespace kde {
namespace {

constexpr int kBin = kCutoffBin;    // cells per output block side
constexpr int kGroupThreads = 32;   // a point group is one warp: 8 cells per thread
constexpr int kGroups = 8;          // point groups per CTA (one output block)
constexpr int kSortThreads = 256;   // 8 warps
constexpr int kSortRounds = 8;      // 32-element rounds per warp
constexpr int kSortChunk = kSortThreads * kSortRounds;  // 2048 keys per block
constexpr int kBatch = 32;          // points per shared-memory batch (one per lane)

template <class T>
__device__ __forceinline__ int find_by(const T* tab, int ninst, int64_t v, int64_t T::*field) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].*field <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Bin key of each point of every instance (points centred and scaled):
// key = bin_begin + by * nbx + bx, or total_bins for padding and for points
// that cannot reach their grid.  vals = the point's index in the prepared
// arrays.
__global__ void k_bin_keys(const CutInst* __restrict__ tab, int ninst, int64_t m,
                           const float4* __restrict__ prepared, uint32_t total_bins,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < m; g += stride) {
    const CutInst& I = tab[find_by(tab, ninst, g, &CutInst::cut_begin)];
    const int64_t p = g - I.cut_begin;
    uint32_t key = total_bins;
    if (p < I.n) {
      // FP32 throughout (FP64 is slow here): the keys can be one bin off near
      // a bin edge, which the ranges' widened reach covers
      const float4 q = prepared[I.prep_begin + p];
      const float X = q.x + q.y, Y = q.z + q.w;
      // a point reaches the grid only if it lies within the reach of it
      if (X >= I.key_lo && Y >= I.key_lo && X <= I.key_hx && Y <= I.key_hy) {
        const int bx = min(max((int)floorf(X * I.key_inv), 0), I.nbx - 1);
        const int by = min(max((int)floorf(Y * I.key_inv), 0), I.nby - 1);
        key = (uint32_t)I.bin_begin + (uint32_t)by * I.nbx + bx;
      }
    }
    keys[g] = key;
    vals[g] = (uint32_t)(I.prep_begin + p);
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


// Accumulate one batch's outer products into a thread's eight cells (columns
// cx, cx+1, rows cy0..cy0+3; acc[2 r + c]): product kernels from tabulated
// factors, radial kernels from tabulated squared offsets and the profile per
// pair.  Per point one 8-byte and one 16-byte table read feed eight FMAs.
template <int KID, bool RADIAL>
__device__ __forceinline__ void accumulate(const float (*KX)[kBin], const float (*KY)[kBin],
                                           const float* sW, int cnt, int cx, int cy0,
                                           float (&acc)[8]) {
  int c = 0;
  if (!RADIAL) {  // two points per step so their table reads are in flight together
    for (; c + 2 <= cnt; c += 2) {
      float2 kx[2];
      float4 ky[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        kx[u] = *reinterpret_cast<const float2*>(&KX[c + u][cx]);
        ky[u] = *reinterpret_cast<const float4*>(&KY[c + u][cy0]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float y[4] = {ky[u].x, ky[u].y, ky[u].z, ky[u].w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          acc[2 * r] = fmaf(kx[u].x, y[r], acc[2 * r]);
          acc[2 * r + 1] = fmaf(kx[u].y, y[r], acc[2 * r + 1]);
        }
      }
    }
  }
  for (; c < cnt; ++c) {
    const float2 kx = *reinterpret_cast<const float2*>(&KX[c][cx]);
    const float4 ky4 = *reinterpret_cast<const float4*>(&KY[c][cy0]);
    const float y[4] = {ky4.x, ky4.y, ky4.z, ky4.w};
    if (RADIAL) {
      const float w = sW[c];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        acc[2 * r] = fmaf(w, kradial<KID>(kx.x + y[r]), acc[2 * r]);
        acc[2 * r + 1] = fmaf(w, kradial<KID>(kx.y + y[r]), acc[2 * r + 1]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        acc[2 * r] = fmaf(kx.x, y[r], acc[2 * r]);
        acc[2 * r + 1] = fmaf(kx.y, y[r], acc[2 * r + 1]);
      }
    }
  }
}

// The sort bins whose points can reach output block (bx, by), with the
// widened reach: the points left out have |u| or |v| above 1 in FP32 too, so
// their factors are exactly zero, and those whose FP32 key put them a bin
// further are still in.
__device__ __forceinline__ BinRange output_block_bins(const CutInst& I, int bx, int by) {
  return block_bins(I.cs, I.range_reach, I.inv_binw, I.nbx, I.nby, bx * kBin, by * kBin, kBin);
}

// The instance of global output block blk, and the block's position in it.
__device__ __forceinline__ const CutInst& output_block(const CutInst* __restrict__ tab, int ninst,
                                                       int blk, int& bx, int& by) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].out_begin <= blk) lo = mid; else hi = mid - 1;
  }
  const CutInst& I = tab[lo];
  const int local = blk - I.out_begin;
  bx = local % I.obx;
  by = local / I.obx;
  return I;
}

// Weight class of a block from the points within its reach (larger is
// heavier): two classes per power of two.
__device__ __forceinline__ int weight_key(uint32_t total) {
  if (total == 0) return 0;
  const int b = 31 - __clz(total);
  return 1 + 2 * b + (b >= 1 ? (int)((total >> (b - 1)) & 1u) : 0);
}

// Points within reach of each output block, and the count of blocks per
// weight class.  The rows' runs are read two at a time so their loads overlap.
__global__ void k_cut_block_totals(const CutInst* __restrict__ tab, int ninst,
                                   const uint32_t* __restrict__ start, int nblocks,
                                   uint32_t* __restrict__ totals, uint32_t* __restrict__ ocount) {
  const int blk = blockIdx.x * blockDim.x + threadIdx.x;
  if (blk >= nblocks) return;
  int bx, by;
  const CutInst& I = output_block(tab, ninst, blk, bx, by);
  const BinRange br = output_block_bins(I, bx, by);
  uint32_t total = 0;
  if (!range_empty(br)) {
    int r = br.lo_by;
    for (; r + 1 <= br.hi_by; r += 2) {
      const uint32_t* a = start + I.bin_begin + r * I.nbx;
      const uint32_t* b = a + I.nbx;
      const uint32_t a0 = __ldg(a + br.lo_bx), a1 = __ldg(a + br.hi_bx + 1);
      const uint32_t b0 = __ldg(b + br.lo_bx), b1 = __ldg(b + br.hi_bx + 1);
      total += (a1 - a0) + (b1 - b0);
    }
    if (r <= br.hi_by) {
      const uint32_t* a = start + I.bin_begin + r * I.nbx;
      total += __ldg(a + br.hi_bx + 1) - __ldg(a + br.lo_bx);
    }
  }
  totals[blk] = total;
  atomicAdd(&ocount[weight_key(total)], 1u);
}

// The output blocks in decreasing weight class (a counting sort; within a
// class the order is whatever the atomics give).  Each block computes only its
// own cells, so the order changes the schedule, never a result: the heaviest
// blocks (dense clusters) start first instead of wherever raster order puts
// them.
__global__ void k_cut_order_scatter(const uint32_t* __restrict__ totals, int nblocks,
                                    uint32_t* __restrict__ ocount, uint32_t* __restrict__ order) {
  __shared__ uint32_t first[kCutOrderKeys];
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int k = kCutOrderKeys - 1; k >= 0; --k) {
      first[k] = acc;
      acc += ocount[k];
    }
  }
  __syncthreads();
  const int blk = blockIdx.x * blockDim.x + threadIdx.x;
  if (blk >= nblocks) return;
  const int key = weight_key(__ldg(totals + blk));
  order[first[key] + atomicAdd(&ocount[kCutOrderKeys + key], 1u)] = (uint32_t)blk;
}

// Shared-memory tables of one point group.
struct GroupTables {
  float4 P[kBatch];
  float W[kBatch];
  __align__(16) float KX[kBatch][kBin];
  __align__(16) float KY[kBatch][kBin];
};

// The block's work, for one kernel.  The points that can reach the block are
// the runs of the sort bins in its range, one run per bin row; their
// concatenation is cut into kBatch-point batches, and warp g of the CTA takes
// batches g, g+G, g+2G, ... (fetching the next while computing the current;
// the warp synchronises only itself) and ends with the two-sum of its eight
// cells in run.
template <int KID, bool RADIAL>
__device__ __forceinline__ void cutoff_group(const CutInst& I, const float4* __restrict__ P,
                                             const float* __restrict__ W,
                                             const uint32_t* __restrict__ start, int bx, int by,
                                             int64_t total, int g, int lane, GroupTables& T,
                                             float2 (&run)[8]) {
  const int nx = I.nx, ny = I.ny;
  const int x0 = bx * kBin, y0 = by * kBin;
  const int cx = 2 * (lane & 7), cy0 = 4 * (lane >> 3);
  // table role: column (and row) ej for the points of one parity, c = 2k + half
  constexpr int kEvalPts = kBatch * kBin / kGroupThreads;
  static_assert(kGroupThreads == 2 * kBin && kBatch == kGroupThreads, "table roles");
  const int ej = lane & (kBin - 1), half = lane >> 4;
  const float2 gxe = I.gxt[min(x0 + ej, nx - 1)];
  const float2 gye = I.gyt[min(y0 + ej, ny - 1)];
  if (total == 0) return;
  const BinRange br = output_block_bins(I, bx, by);
  RunCursor cur;
  cur.init(start, I.bin_begin, I.nbx, br);
  constexpr int64_t kStride = (int64_t)kGroups * kBatch;
  int64_t v = (int64_t)g * kBatch + lane;  // this lane's point of the warp's current batch
  float4 pf = make_float4(0.f, 0.f, 0.f, 0.f);
  float wf = 0.f;
  if (v < total) {
    const int64_t p = cur.map(v);
    pf = P[p];
    wf = W[p];
  }
  for (int64_t b0 = (int64_t)g * kBatch; b0 < total; b0 += kStride, v += kStride) {
    const int cnt = (int)min((int64_t)kBatch, total - b0);
    __syncwarp();  // the warp's previous batch is consumed
    if (lane < cnt) {
      T.P[lane] = pf;
      T.W[lane] = wf;
    }
    __syncwarp();
    if (v + kStride < total) {  // next batch, in flight
      const int64_t p = cur.map(v + kStride);
      pf = P[p];
      wf = W[p];
    }
    // the two half-warps write rows 2k and 2k+1: conflict-free
#pragma unroll 4
    for (int k = 0; k < kEvalPts; ++k) {
      const int c = 2 * k + half;
      if (c < cnt) {
        const float4 p = T.P[c];
        const float u = (gxe.x - p.x) + (gxe.y - p.y), w = (gye.x - p.z) + (gye.y - p.w);
        if (RADIAL) {
          T.KX[c][ej] = u * u;
          T.KY[c][ej] = w * w;
        } else {
          T.KX[c][ej] = kfactor<KID>(u);
          T.KY[c][ej] = T.W[c] * kfactor<KID>(w);
        }
      }
    }
    __syncwarp();
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    accumulate<KID, RADIAL>(T.KX, T.KY, T.W, cnt, cx, cy0, acc);
#pragma unroll
    for (int r = 0; r < 8; ++r) two_sum_acc(run[r], acc[r]);
  }
}

// One CTA per 16x16-cell output block of some instance (the order list maps
// CTAs to blocks, heaviest first), kGroups one-warp point groups: a dense
// block's points are shared out over the groups, whose (hi, lo) sums are
// added in group order at the end, so results are reproducible.  Blocks of 16
// cells spread a dense region over many CTAs; the finer sort bins keep the
// points a block reads close to those its cells' supports actually reach.
__global__ void __launch_bounds__(kGroups * kGroupThreads)
    k_cutoff(const CutInst* __restrict__ tab, int ninst, const float4* __restrict__ P,
             const float* __restrict__ W, const uint32_t* __restrict__ start,
             const uint32_t* __restrict__ order, const uint32_t* __restrict__ totals) {
  // the groups' tables; after every group is done, their partial sums
  constexpr size_t kTablesBytes = sizeof(GroupTables) * kGroups;
  constexpr size_t kPartBytes = sizeof(float2) * kGroups * kGroupThreads * 8;
  __shared__ __align__(16) unsigned char smem[kTablesBytes > kPartBytes ? kTablesBytes
                                                                        : kPartBytes];
  GroupTables* tables = reinterpret_cast<GroupTables*>(smem);
  float2 (*part)[kGroupThreads][8] = reinterpret_cast<float2 (*)[kGroupThreads][8]>(smem);
  int bx, by;
  const int blk = (int)__ldg(order + blockIdx.x);
  const CutInst& I = output_block(tab, ninst, blk, bx, by);
  const int64_t total = __ldg(totals + blk);
  const int g = threadIdx.x / kGroupThreads, lane = threadIdx.x % kGroupThreads;
  float2 run[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) run[r] = make_float2(0.f, 0.f);
  GroupTables& T = tables[g];
  switch (I.kid) {
#define KDE_CUT(K)                                                                      \
  case K:                                                                               \
    cutoff_group<K, false>(I, P, W, start, bx, by, total, g, lane, T, run);             \
    break;                                                                              \
  case kRadial + K:                                                                     \
    cutoff_group<K, true>(I, P, W, start, bx, by, total, g, lane, T, run);              \
    break;
    KDE_CUT(KDE_UNIFORM)
    KDE_CUT(KDE_TRIANGULAR)
    KDE_CUT(KDE_EPANECHNIKOV)
    KDE_CUT(KDE_QUARTIC)
    KDE_CUT(KDE_TRIWEIGHT)
    KDE_CUT(KDE_TRICUBE)
    KDE_CUT(KDE_COSINE)
#undef KDE_CUT
    default: break;
  }
  __syncthreads();  // every group is done with its tables
#pragma unroll
  for (int r = 0; r < 8; ++r) part[g][lane][r] = run[r];
  __syncthreads();
  if (g == 0) {
    const int cx = 2 * (lane & 7), cy0 = 4 * (lane >> 3);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      float2 sum = part[0][lane][r];
      for (int h = 1; h < kGroups; ++h) {
        const float2 o = part[h][lane][r];
        two_sum_acc(sum, o.x);
        sum.y += o.y;
      }
      const int x = bx * kBin + cx + (r & 1), y = by * kBin + cy0 + (r >> 1);
      if (x < I.nx && y < I.ny) I.out[(int64_t)y * I.nx + x] = (sum.x + sum.y) * I.scale;
    }
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace

CutoffGeom cutoff_geometry(int nx, int ny, double cs, double reach, int bin) {
  CutoffGeom g;
  g.bin = bin;
  g.nbx = (nx + bin - 1) / bin;
  g.nby = (ny + bin - 1) / bin;
  g.nbins = g.nbx * g.nby;
  g.inv_binw = 1.0 / (bin * cs);
  g.ext_x = nx * cs + reach;
  g.ext_y = ny * cs + reach;
  return g;
}

int cutoff_sort_bin(int nx, int ny, double reach_cells) {
  // an output block reads about (16 + 2 reach + bin)^2 cells' points, of which
  // (16 + 2 reach)^2 can reach it; finer bins mean more bins to sort
  int bin = reach_cells <= 6.0 ? 4 : reach_cells <= 16.0 ? 8 : 16;
  while (bin < 64 && ((int64_t)(nx + bin - 1) / bin) * ((ny + bin - 1) / bin) > (1 << 24)) bin *= 2;
  return bin;
}

CutoffSizes cutoff_sizes(int64_t m, int64_t total_bins) {
  CutoffSizes z;
  z.nchunks = (int)((m + kSortChunk - 1) / kSortChunk);
  int bits = 1;
  while ((1ll << bits) <= (long long)total_bins) ++bits;  // keys 0..total_bins
  z.passes = (bits + 7) / 8;
  z.hist_words = (size_t)256 * z.nchunks;
  z.scan_words = scan_temp_words((int64_t)z.hist_words, 2048);
  return z;
}

cudaError_t launch_bin_sort(const CutInst* tab, int ninst, int64_t m, int64_t total_bins,
                            const float4* prepared, const float* prepared_w, const CutoffSizes& z,
                            CutoffScratch ws, cudaStream_t s) {
  if (ninst <= 0 || m <= 0) return cudaSuccess;
  k_bin_keys<<<grid_for(m), 256, 0, s>>>(tab, ninst, m, prepared, (uint32_t)total_bins,
                                         ws.keys[0], ws.vals[0]);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int cur = 0;
  for (int pass = 0; pass < z.passes; ++pass) {
    const int shift = 8 * pass;
    k_radix_count<<<z.nchunks, kSortThreads, 0, s>>>(ws.keys[cur], m, shift, z.nchunks, ws.hist);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_exclusive_scan(ws.hist, ws.hist_scan, (int64_t)z.hist_words, 2048, ws.scan_temp, s);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<z.nchunks, kSortThreads, 0, s>>>(ws.keys[cur], ws.vals[cur], m, shift,
                                                        z.nchunks, ws.hist_scan, ws.keys[cur ^ 1],
                                                        ws.vals[cur ^ 1]);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cur ^= 1;
  }
  k_bin_bounds<<<(int)((total_bins + 1 + 255) / 256), 256, 0, s>>>(ws.keys[cur], m,
                                                                   (int)total_bins, ws.start);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_permute<<<grid_for(m), 256, 0, s>>>(prepared, prepared_w, ws.vals[cur], m, ws.spts, ws.sw);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_cutoff_eval(const CutInst* tab, int ninst, int64_t cut_bins,
                               const CutoffScratch& ws, cudaStream_t s) {
  if (ninst <= 0 || cut_bins <= 0) return cudaSuccess;
  if (cut_bins > 0x7fffffff) return cudaErrorInvalidValue;
  const int nb = (int)cut_bins, grid = (nb + 255) / 256;
  cudaError_t e = cudaMemsetAsync(ws.ocount, 0, sizeof(uint32_t) * 2 * kCutOrderKeys, s);
  if (e != cudaSuccess) return e;
  k_cut_block_totals<<<grid, 256, 0, s>>>(tab, ninst, ws.start, nb, ws.totals, ws.ocount);
  k_cut_order_scatter<<<grid, 256, 0, s>>>(ws.totals, nb, ws.ocount, ws.order);
  k_cutoff<<<(unsigned)nb, kGroups * kGroupThreads, 0, s>>>(tab, ninst, ws.spts, ws.sw,
                                                             ws.start, ws.order, ws.totals);
  note_launches(3);
  return cudaGetLastError();
}

}  // namespace kde
