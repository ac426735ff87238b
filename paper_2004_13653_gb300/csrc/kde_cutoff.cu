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
// blocks run heaviest first; a block with thousands of points within reach is
// split into four row slices, one CTA each, and light blocks share a CTA two
// at a time, four warps each.  Nothing is accumulated with atomics, and the
// order of every sum is fixed, so results are reproducible bit for bit.  The
// same sort, with 32-cell bins and a wider reach, orders the points of the
// block-sparse tensor-core path.
#include "kde_internal.cuh"
#include "kernel_factors.cuh"
#include "tc_ptx.cuh"

namespace kde {
namespace {

constexpr int kBin = kCutoffBin;    // cells per output block side
constexpr int kGroupThreads = 32;   // a point group is one warp: 8 cells per thread
constexpr int kGroups = 8;          // point groups per CTA (one output block)
constexpr int kSortThreads = 512;   // 16 warps
constexpr int kSortRounds = 8;      // 32-element rounds per warp
constexpr int kSortChunk = kSortThreads * kSortRounds;  // 4096 keys per block
constexpr int kMaxPasses = 4;     // 8-bit digits of 32-bit keys
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

// Radix buckets per pass: the 256 values of an 8-bit digit, then one bucket
// for keys with a bit set at or above `top` = 8 x passes.  Only the key that
// marks padding and unreachable points (total_bins) can have one, when it
// needs a bit more than every valid key; it then sorts after every digit in
// each pass, so the valid keys alone decide the number of passes.
constexpr int kDigits = 257;
static_assert(kSortThreads >= kDigits, "one thread per radix bucket in the look-back");

__device__ __forceinline__ uint32_t radix_digit(uint32_t key, int shift, int top) {
  return (top < 32 && (key >> top) != 0u) ? 256u : (key >> shift) & 255u;
}

// Bin key of each point of every instance (points centred and scaled):
// key = bin_begin + by * nbx + bx, or total_bins for padding and for points
// that cannot reach their grid.  vals = the point's index in the prepared
// arrays.  Each CTA also counts the digits of every radix pass of its keys
// (lanes that share a digit add once) and adds them to the per-pass
// histograms ghist[pass][kDigits].
__global__ void __launch_bounds__(256)
    k_bin_keys(const CutInst* __restrict__ tab, int ninst, int64_t m,
               const float4* __restrict__ prepared, uint32_t total_bins, int passes,
               uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
               uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[kMaxPasses][kDigits];
  for (int i = threadIdx.x; i < kMaxPasses * kDigits; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  // warp-uniform trip count, so every lane takes part in the matches
  for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); g0 < m; g0 += stride) {
    const int64_t g = g0 + lane;
    const bool valid = g < m;
    uint32_t key = total_bins;
    if (valid) {
      const CutInst& I = tab[find_by(tab, ninst, g, &CutInst::cut_begin)];
      const int64_t p = g - I.cut_begin;
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
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    for (int pass = 0; pass < passes; ++pass) {
      const uint32_t d = radix_digit(key, 8 * pass, 8 * passes);
      const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 0xffffffffu) & act;
      if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[pass][d], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kDigits; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&ghist[i], c);
  }
}

// Rank of each key's digit among equal digits earlier in this block's chunk:
// each warp walks its 256 keys (kv, loaded beforehand) in rounds of 32, peers
// found with match_any, per-warp digit counts kept in shared memory.
// Deterministic.
__device__ __forceinline__ void rank_digits(const uint32_t (&kv)[kSortRounds], int64_t m,
                                            int64_t base, int shift, int top,
                                            uint32_t (*cnt)[kDigits], uint32_t (&digit)[kSortRounds],
                                            uint32_t (&rank)[kSortRounds]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t e = base + (int64_t)warp * 32 * kSortRounds + r * 32 + lane;
    const bool valid = e < m;
    const uint32_t d = valid ? radix_digit(kv[r], shift, top) : 0u;
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

// Look-back status of one (chunk, digit) of a radix pass: bits 61-63 the pass
// number plus one (0 or another pass: not yet published by this pass), bit 60
// set when the value is the inclusive prefix over chunks 0..c, clear when it
// is the chunk's own count; bits 0-39 the value.
constexpr unsigned long long kStatusIncl = 1ull << 60;
constexpr unsigned long long kStatusValue = (1ull << 40) - 1;
constexpr int kRoleLookback = 31;  // timeout role id of the look-back wait

__device__ __forceinline__ unsigned long long status_word(int pass, bool incl, uint64_t v) {
  return ((unsigned long long)(pass + 1) << 61) | (incl ? kStatusIncl : 0ull) | v;
}

// One stable counting pass over 8 bits of the keys and the bucket above them
// (`top` = 8 x passes; Merrill and Garland's
// single-pass prefix scan with decoupled look-back, applied per digit).  CTAs
// take 4096-key chunks in the order they start (a counter), so every chunk a
// CTA waits for belongs to a CTA that is already running.  Each CTA ranks its
// keys per digit (stable: warps in order, lanes in order), publishes its
// per-digit counts, then walks back over earlier chunks until it meets an
// inclusive prefix, publishes its own inclusive prefix and scatters: position
// = (keys of smaller digits) + (same digit in earlier chunks) + rank.  The
// last pass writes the permuted points and weights instead of the indices.
// A wait that does not end within the limit records a timeout in err; the
// positions are then bounded, not correct.
__global__ void __launch_bounds__(kSortThreads)
    k_radix_pass(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t m,
                 int pass, int top, const uint32_t* __restrict__ ghist,
                 uint32_t* __restrict__ chunk_ctr,
                 unsigned long long* __restrict__ status, uint32_t* __restrict__ keys_out,
                 uint32_t* __restrict__ vals_out, const float4* __restrict__ prepared,
                 const float* __restrict__ wts, float4* __restrict__ spts, float* __restrict__ sw,
                 int last, CallScalars* __restrict__ err, uint64_t limit_ns) {
  __shared__ uint32_t cnt[kSortThreads / 32][kDigits];
  __shared__ uint32_t base[kDigits];
  __shared__ uint32_t wsum[kSortThreads / 32];
  __shared__ uint32_t chunk_s;
  if (threadIdx.x == 0) chunk_s = atomicAdd(&chunk_ctr[pass], 1u);
  for (int i = threadIdx.x; i < (kSortThreads / 32) * kDigits; i += kSortThreads)
    (&cnt[0][0])[i] = 0;
  __syncthreads();
  const uint32_t chunk = chunk_s;
  const int shift = 8 * pass;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e0 = (int64_t)chunk * kSortChunk + (int64_t)warp * 32 * kSortRounds + lane;
  // every key and index of this thread in flight at once
  uint32_t kv[kSortRounds], vv[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t e = e0 + r * 32;
    kv[r] = e < m ? keys[e] : 0u;
    vv[r] = e < m ? vals[e] : 0u;
  }
  uint32_t digit[kSortRounds], rank[kSortRounds];
  rank_digits(kv, m, (int64_t)chunk * kSortChunk, shift, top, cnt, digit, rank);
  __syncthreads();
  // the first kDigits threads own one bucket each
  const bool dig = threadIdx.x < kDigits;
  const int d = dig ? (int)threadIdx.x : 0;
  uint32_t total = 0;
  if (dig) {
    for (int w = 0; w < kSortThreads / 32; ++w) {
      const uint32_t c = cnt[w][d];
      cnt[w][d] = total;  // exclusive prefix over the warps
      total += c;
    }
  }
  volatile unsigned long long* st = status + (size_t)chunk * kDigits + d;
  if (dig) *st = status_word(pass, chunk == 0, total);
  uint64_t excl = 0;
  if (dig && chunk > 0) {
    // four earlier chunks per step, their words loaded together; the walk
    // ends at the first inclusive prefix (chunk 0 publishes one at once)
    constexpr int kLook = 4;
    const uint64_t t0 = tc::globaltimer_ns();
    int64_t c = (int64_t)chunk - 1;
    for (uint32_t it = 1;; ++it) {
      unsigned long long v[kLook];
#pragma unroll
      for (int j = 0; j < kLook; ++j)
        v[j] = c - j >= 0
                   ? *(volatile unsigned long long*)(status + (size_t)(c - j) * kDigits + d)
                   : 0ull;
      bool done = false;
      int j = 0;
      for (; j < kLook; ++j) {
        if ((int)(v[j] >> 61) != pass + 1) break;  // not yet published
        excl += v[j] & kStatusValue;
        if (v[j] & kStatusIncl) {
          done = true;
          break;
        }
      }
      if (done) break;
      c -= j;
      if (j == 0 && (it & 63) == 0 &&
          (tc::globaltimer_ns() - t0 > limit_ns || it > (1u << 30))) {
        if (atomicOr(&err->err, kErrTimeout | kErrSortTimeout) == 0)
          atomicExch(&err->timeout_where, kRoleLookback);
        break;
      }
    }
    *st = status_word(pass, true, excl + total);
  }
  // keys of smaller digits: exclusive scan of this pass's histogram
  const uint32_t gh = dig ? ghist[pass * kDigits + d] : 0u;
  uint32_t inc = gh;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  if (dig) base[d] = before + inc - gh + (uint32_t)excl;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    if (digit[r] == 0xffffffffu) continue;
    const uint32_t pos = base[digit[r]] + cnt[warp][digit[r]] + rank[r];
    if (pos >= m) continue;  // only after a timed-out wait
    keys_out[pos] = kv[r];
    const uint32_t v = vv[r];
    if (last) {
      spts[pos] = prepared[v];
      sw[pos] = wts[v];
    } else {
      vals_out[pos] = v;
    }
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


// Accumulate one batch's outer products into a thread's cells: columns cx,
// cx+1 of RPL rows from cy0 (acc[2 r + c]); RPL = 4 for a whole 16-row
// block, 1 for a 4-row slice of a heavy block.  Product kernels from
// tabulated factors, radial kernels from tabulated squared offsets and the
// profile per pair.  Per point one 8-byte and one 4*RPL-byte table read feed
// 2*RPL FMAs.
template <int KID, bool RADIAL, int RPL>
__device__ __forceinline__ void accumulate(const float (*KX)[kBin], const float (*KY)[kBin],
                                           const float* sW, int cnt, int cx, int cy0,
                                           float (&acc)[2 * RPL]) {
  static_assert(RPL == 4 || RPL == 1, "rows per lane");
  auto load_y = [&](int c, float (&y)[RPL]) {
    if constexpr (RPL == 4) {
      const float4 v = *reinterpret_cast<const float4*>(&KY[c][cy0]);
      y[0] = v.x;
      y[1] = v.y;
      y[2] = v.z;
      y[3] = v.w;
    } else {
      y[0] = KY[c][cy0];
    }
  };
  int c = 0;
  if (!RADIAL) {  // two points per step so their table reads are in flight together
    for (; c + 2 <= cnt; c += 2) {
      float2 kx[2];
      float y[2][RPL];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        kx[u] = *reinterpret_cast<const float2*>(&KX[c + u][cx]);
        load_y(c + u, y[u]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          acc[2 * r] = fmaf(kx[u].x, y[u][r], acc[2 * r]);
          acc[2 * r + 1] = fmaf(kx[u].y, y[u][r], acc[2 * r + 1]);
        }
      }
    }
  }
  for (; c < cnt; ++c) {
    const float2 kx = *reinterpret_cast<const float2*>(&KX[c][cx]);
    float y[RPL];
    load_y(c, y);
    if (RADIAL) {
      const float w = sW[c];
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        acc[2 * r] = fmaf(w, kradial<KID>(kx.x + y[r]), acc[2 * r]);
        acc[2 * r + 1] = fmaf(w, kradial<KID>(kx.y + y[r]), acc[2 * r + 1]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
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

// Blocks with at least 4096 points within reach (weight class 25 and up) of
// an instance whose supports allow it are computed as four items of four rows
// each, so a dense cluster's block is spread over four CTAs instead of
// holding one for the whole launch; their order keys sit above all others, so
// they come first.  The split depends only on the block's own point count
// and its instance, so a block is computed the same way in every run and in a
// batch as on its own.
constexpr int kHeavyKey = 25;  // weight_key(4096)
// Blocks with fewer than 192 points within reach (weight class 15 and below,
// empty blocks included) are computed two to a CTA, four point groups each:
// eight groups would leave most of their warps without a batch.  Like the
// split of heavy blocks, this depends only on the block's own count.
constexpr int kLightKey = 15;  // weight_key(191)
__device__ __forceinline__ int order_key(const CutInst& I, uint32_t total) {
  const int k = weight_key(total);
  return I.slice && k >= kHeavyKey ? kCutOrderClasses + k : k;
}

// Points within reach of each output block, the block's range of sort bins
// (found once here, in FP64, so the gather itself needs no FP64), and the
// count of blocks per weight class.  The rows' runs are read two at a time so
// their loads overlap.
__global__ void k_cut_block_totals(const CutInst* __restrict__ tab, int ninst,
                                   const uint32_t* __restrict__ start, int nblocks,
                                   uint32_t* __restrict__ totals, int4* __restrict__ ranges,
                                   uint32_t* __restrict__ ocount) {
  const int blk = blockIdx.x * blockDim.x + threadIdx.x;
  if (blk >= nblocks) return;
  int bx, by;
  const CutInst& I = output_block(tab, ninst, blk, bx, by);
  const BinRange br = output_block_bins(I, bx, by);
  ranges[blk] = make_int4(br.lo_bx, br.hi_bx, br.lo_by, br.hi_by);
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
  atomicAdd(&ocount[order_key(I, total)], 1u);
}

// The output blocks in decreasing weight class (a counting sort; within a
// class the order is whatever the atomics give).  Each block computes only its
// own cells, so the order changes the schedule, never a result: the heaviest
// blocks (dense clusters) start first instead of wherever raster order puts
// them.
__global__ void k_cut_order_scatter(const CutInst* __restrict__ tab, int ninst,
                                    const uint32_t* __restrict__ totals, int nblocks,
                                    uint32_t* __restrict__ ocount, uint32_t* __restrict__ order) {
  __shared__ uint32_t first[kCutOrderKeys];
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int k = kCutOrderKeys - 1; k >= 0; --k) {
      first[k] = acc;
      acc += ocount[k];
    }
    // the blocks to be split into slices come first and the light ones last;
    // the gather needs the count of the first and the position of the second
    if (blockIdx.x == 0) {
      ocount[2 * kCutOrderKeys] = first[kCutOrderClasses - 1];
      ocount[2 * kCutOrderKeys + 1] = first[kLightKey];
    }
  }
  __syncthreads();
  const int blk = blockIdx.x * blockDim.x + threadIdx.x;
  if (blk >= nblocks) return;
  int bx, by;
  const int key = order_key(output_block(tab, ninst, blk, bx, by), __ldg(totals + blk));
  order[first[key] + atomicAdd(&ocount[kCutOrderKeys + key], 1u)] = (uint32_t)blk;
}

// The RunCursor walk with 32-bit positions (a block's or slice's reach list
// and the sorted points number fewer than 2^32): fewer registers in the
// gather, whose occupancy its register count sets.
struct RunCursor32 {
  const uint32_t* row;  // start + row0 + by * nbx
  int nbx, lo_bx, hi_bx, by, hi_by;
  uint32_t vr, ra, rb;
  __device__ __forceinline__ void load_run() {
    ra = __ldg(row + lo_bx);
    rb = __ldg(row + hi_bx + 1);
  }
  __device__ __forceinline__ void init(const uint32_t* start, int row0, int nbx_,
                                       const BinRange& br) {
    nbx = nbx_;
    lo_bx = br.lo_bx;
    hi_bx = br.hi_bx;
    by = br.lo_by;
    hi_by = br.hi_by;
    row = start + row0 + by * nbx;
    vr = 0;
    load_run();
  }
  // index of position v (v below the range's total, not decreasing)
  __device__ __forceinline__ uint32_t map(uint32_t v) {
    while (v >= vr + (rb - ra) && by < hi_by) {
      vr += rb - ra;
      ++by;
      row += nbx;
      load_run();
    }
    return ra + (v - vr);
  }
};

// Shared-memory tables of one point group.
struct GroupTables {
  float4 P[kBatch];
  float W[kBatch];
  __align__(16) float KX[kBatch][kBin];
  __align__(16) float KY[kBatch][kBin];
};

constexpr int kSliceRows = 4;
// dynamic shared memory of the gather: the groups' tables, then their running sums
constexpr size_t kCutTablesBytes = sizeof(GroupTables) * kGroups;
constexpr size_t kCutSmemBytes = kCutTablesBytes + sizeof(float2) * kGroups * 8 * kGroupThreads;
constexpr int kSlices = kBin / kSliceRows;  // items per heavy block

// The work of one item, for one kernel: rows y_off..y_off + 4 RPL - 1 of the
// block (RPL = 4: all 16 rows; RPL = 1: a 4-row slice).  The points that can
// reach those rows are the runs of the sort bins in range br, one run per bin
// row; their concatenation is cut into kBatch-point batches, and group g of
// the block's NG takes batches g, g+NG, g+2NG, ... (fetching the next while computing
// the current; the warp synchronises only itself) and adds each batch into
// the (hi, lo) running sums of its cells with a two-sum; the running sums
// live in shared memory (run[r * 32] for cell r of this lane), which keeps
// the kernel at 64 registers and four CTAs per SM.
template <int KID, bool RADIAL, int RPL, int NG>
__device__ __forceinline__ void cutoff_group(const CutInst& I, const float4* __restrict__ P,
                                             const float* __restrict__ W,
                                             const uint32_t* __restrict__ start, int bx, int by,
                                             int y_off, const BinRange& br, int64_t total, int g,
                                             int lane, GroupTables& T, float2* run) {
  const int nx = I.nx, ny = I.ny;
  const int x0 = bx * kBin, y0 = by * kBin;
  const int cx = 2 * (lane & 7), cy0 = y_off + RPL * (lane >> 3);
  // table role: column (and row) ej for the points of one parity, c = 2k + half
  constexpr int kEvalPts = kBatch * kBin / kGroupThreads;
  static_assert(kGroupThreads == 2 * kBin && kBatch == kGroupThreads, "table roles");
  const int ej = lane & (kBin - 1), half = lane >> 4;
  const float2 gxe = I.gxt[min(x0 + ej, nx - 1)];
  const float2 gye = I.gyt[min(y0 + ej, ny - 1)];
  if (total == 0) return;
  RunCursor32 cur;
  cur.init(start, I.bin_begin, I.nbx, br);
  constexpr uint32_t kStride = NG * kBatch;
  const uint32_t total32 = (uint32_t)total;
  uint32_t v = g * kBatch + lane;  // this lane's point of the warp's current batch
  float4 pf = make_float4(0.f, 0.f, 0.f, 0.f);
  float wf = 0.f;
  if (v < total32) {
    const uint32_t p = cur.map(v);
    pf = P[p];
    wf = W[p];
  }
  for (uint32_t b0 = g * kBatch; b0 < total32; b0 += kStride, v += kStride) {
    const int cnt = (int)min((uint32_t)kBatch, total32 - b0);
    __syncwarp();  // the warp's previous batch is consumed
    if (lane < cnt) {
      T.P[lane] = pf;
      T.W[lane] = wf;
    }
    __syncwarp();
    if (v + kStride < total32) {  // next batch, in flight
      const uint32_t p = cur.map(v + kStride);
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
    float acc[2 * RPL];
#pragma unroll
    for (int r = 0; r < 2 * RPL; ++r) acc[r] = 0.f;
    accumulate<KID, RADIAL, RPL>(T.KX, T.KY, T.W, cnt, cx, cy0, acc);
#pragma unroll
    for (int r = 0; r < 2 * RPL; ++r) {
      float2 x = run[r * kGroupThreads];
      two_sum_acc(x, acc[r]);
      run[r * kGroupThreads] = x;
    }
  }
}

// Points of the sort bins in range br (the runs of its bin rows).
__device__ __forceinline__ uint32_t range_total(const uint32_t* __restrict__ start, int row0,
                                                int nbx, const BinRange& br) {
  uint32_t total = 0;
  if (range_empty(br)) return 0;
  for (int r = br.lo_by; r <= br.hi_by; ++r) {
    const uint32_t* a = start + row0 + r * nbx;
    total += __ldg(a + br.hi_bx + 1) - __ldg(a + br.lo_bx);
  }
  return total;
}

template <int RPL, int NG>
__device__ __forceinline__ void group_dispatch(const CutInst& I, const float4* __restrict__ P,
                                               const float* __restrict__ W,
                                               const uint32_t* __restrict__ start, int bx, int by,
                                               int y_off, const BinRange& br, int64_t total, int g,
                                               int lane, GroupTables& T, float2* run) {
  switch (I.kid) {
#define KDE_CUT(K)                                                                       \
  case K:                                                                                \
    cutoff_group<K, false, RPL, NG>(I, P, W, start, bx, by, y_off, br, total, g, lane, T, run); \
    break;                                                                               \
  case kRadial + K:                                                                      \
    cutoff_group<K, true, RPL, NG>(I, P, W, start, bx, by, y_off, br, total, g, lane, T, run); \
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
}

// One CTA of kGroups one-warp point groups per item: first the four slices of
// every heavy block, then the other blocks, each in the order list's
// heaviest-first order, and last the light blocks two at a time, groups 0-3
// on the first and 4-7 on the second (CTAs past the last item return at once).  A whole
// block's eight cells per thread, or a slice's two, are summed over the groups
// in group order at the end, so every cell is computed by one CTA in a fixed
// order and results are reproducible bit for bit.  Blocks of 16 cells spread a
// dense region over many CTAs; the finer sort bins keep the points an item
// reads close to those its cells' supports actually reach.
__global__ void __launch_bounds__(kGroups * kGroupThreads)
    k_cutoff(const CutInst* __restrict__ tab, int ninst, const float4* __restrict__ P,
             const float* __restrict__ W, const uint32_t* __restrict__ start,
             const uint32_t* __restrict__ order, const uint32_t* __restrict__ totals,
             const int4* __restrict__ ranges, const uint32_t* __restrict__ heavy_count,
             int nblocks, const CallScalars* __restrict__ err) {
  // the groups' tables, then their running sums (cell r of lane l of group g
  // at part[g][r][l])
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int4 s_rg[2];
  __shared__ uint32_t s_total[2];
  __shared__ int s_blk[2];
  GroupTables* tables = reinterpret_cast<GroupTables*>(smem);
  float2 (*part)[8][kGroupThreads] =
      reinterpret_cast<float2 (*)[8][kGroupThreads]>(smem + kCutTablesBytes);
  const int g = threadIdx.x / kGroupThreads, lane = threadIdx.x % kGroupThreads;
  GroupTables& T = tables[g];
  // after a timed-out sort the bin starts may not rise, and positions taken
  // from them could leave the sorted points: compute nothing (the call
  // reports the timeout)
  if (*reinterpret_cast<const volatile int*>(&err->err) & kErrSortTimeout) return;
  const int64_t heavy = __ldg(heavy_count);
  const int64_t light = __ldg(heavy_count + 1);  // order position of the first light block
  const int64_t singles = kSlices * heavy + (light - heavy);
  const int64_t item = blockIdx.x;
  if (item >= singles + ((int64_t)nblocks - light + 1) / 2) return;
  if (item >= singles) {
    // two light blocks: half h = g / 4 takes the block at order position
    // light + 2 (item - singles) + h with its four groups
    const int half = g >> 2, gh = g & 3;
    const int64_t pos = light + 2 * (item - singles) + half;
    const bool has = pos < nblocks;
    if (has && gh == 0 && lane == 0) {
      const int blk = (int)__ldg(order + pos);
      s_blk[half] = blk;
      s_rg[half] = __ldg(ranges + blk);
      s_total[half] = __ldg(totals + blk);
    }
    __syncthreads();
    if (has) {
      int bx, by;
      const CutInst& I = output_block(tab, ninst, s_blk[half], bx, by);
      const int4 rg = s_rg[half];
      const BinRange br = {rg.x, rg.y, rg.z, rg.w};
#pragma unroll
      for (int r = 0; r < 8; ++r) part[g][r][lane] = make_float2(0.f, 0.f);
      group_dispatch<4, 4>(I, P, W, start, bx, by, 0, br, s_total[half], gh, lane, T,
                           &part[g][0][lane]);
    }
    __syncthreads();  // every group's running sums are final
    if (has) {
      // group gh of the half combines cells 2 gh and 2 gh + 1 of every
      // thread's eight over the half's four groups, in order
      int bx, by;
      const CutInst& I = output_block(tab, ninst, s_blk[half], bx, by);
      const int cx = 2 * (lane & 7), cy0 = 4 * (lane >> 3);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int r = 2 * gh + rr;
        float2 sum = part[4 * half][r][lane];
#pragma unroll
        for (int h = 1; h < 4; ++h) {
          const float2 o = part[4 * half + h][r][lane];
          two_sum_acc(sum, o.x);
          sum.y += o.y;
        }
        const int x = bx * kBin + cx + (r & 1), y = by * kBin + cy0 + (r >> 1);
        if (x < I.nx && y < I.ny) I.out[(int64_t)y * I.nx + x] = (sum.x + sum.y) * I.scale;
      }
    }
    return;
  }
  {
    int64_t pos;
    int slice;
    if (item < kSlices * heavy) {
      pos = item / kSlices;
      slice = (int)(item % kSlices);
    } else {
      pos = heavy + (item - kSlices * heavy);
      slice = -1;
    }
    const int blk = (int)__ldg(order + pos);
    int bx, by;
    const CutInst& I = output_block(tab, ninst, blk, bx, by);
    if (threadIdx.x == 0) {
      if (slice < 0) {
        s_rg[0] = __ldg(ranges + blk);
        s_total[0] = __ldg(totals + blk);
      } else {  // the slice's own bin range and point count
        const BinRange b = block_bins_rect(I.cs, I.range_reach, I.inv_binw, I.nbx, I.nby,
                                           bx * kBin, by * kBin + slice * kSliceRows, kBin,
                                           kSliceRows);
        s_rg[0] = make_int4(b.lo_bx, b.hi_bx, b.lo_by, b.hi_by);
        s_total[0] = range_total(start, I.bin_begin, I.nbx, b);
      }
    }
    __syncthreads();
    const int4 rg = s_rg[0];
    const BinRange br = {rg.x, rg.y, rg.z, rg.w};
    const int64_t total = s_total[0];
    if (slice < 0) {
#pragma unroll
      for (int r = 0; r < 8; ++r) part[g][r][lane] = make_float2(0.f, 0.f);
      group_dispatch<4, kGroups>(I, P, W, start, bx, by, 0, br, total, g, lane, T,
                                 &part[g][0][lane]);
      __syncthreads();  // every group's running sums are final
      // group g combines cell r = g of every thread's eight, over the groups in
      // order (the same order for every block and run)
      static_assert(kGroups == 8, "one cell of eight per group");
      const int r = g;
      const int cx = 2 * (lane & 7), cy0 = 4 * (lane >> 3);
      float2 sum = part[0][r][lane];
#pragma unroll
      for (int h = 1; h < kGroups; ++h) {
        const float2 o = part[h][r][lane];
        two_sum_acc(sum, o.x);
        sum.y += o.y;
      }
      const int x = bx * kBin + cx + (r & 1), y = by * kBin + cy0 + (r >> 1);
      if (x < I.nx && y < I.ny) I.out[(int64_t)y * I.nx + x] = (sum.x + sum.y) * I.scale;
    } else {
      part[g][0][lane] = make_float2(0.f, 0.f);
      part[g][1][lane] = make_float2(0.f, 0.f);
      group_dispatch<1, kGroups>(I, P, W, start, bx, by, slice * kSliceRows, br, total, g, lane, T,
                        &part[g][0][lane]);
      __syncthreads();
      if (threadIdx.x < 2 * kGroupThreads) {  // 64 cells, one thread each
        const int l = threadIdx.x >> 1, r = threadIdx.x & 1;
        float2 sum = part[0][r][l];
#pragma unroll
        for (int h = 1; h < kGroups; ++h) {
          const float2 o = part[h][r][l];
          two_sum_acc(sum, o.x);
          sum.y += o.y;
        }
        const int x = bx * kBin + 2 * (l & 7) + r, y = by * kBin + slice * kSliceRows + (l >> 3);
        if (x < I.nx && y < I.ny) I.out[(int64_t)y * I.nx + x] = (sum.x + sum.y) * I.scale;
      }
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
  // the valid keys 0..total_bins - 1 set the passes; the marker total_bins
  // takes the bucket above the digits where it needs one more bit
  int bits = 1;
  while ((1ll << bits) < (long long)total_bins) ++bits;
  z.passes = (bits + 7) / 8;
  // look-back status (one 64-bit word per chunk and bucket), the per-pass
  // bucket histograms and the per-pass chunk counters, cleared together
  z.hist_words = (size_t)2 * kDigits * z.nchunks + (size_t)kMaxPasses * kDigits + kMaxPasses;
  return z;
}

cudaError_t launch_bin_sort(const CutInst* tab, int ninst, int64_t m, int64_t total_bins,
                            const float4* prepared, const float* prepared_w, const CutoffSizes& z,
                            CutoffScratch ws, cudaStream_t s) {
  if (ninst <= 0 || m <= 0) return cudaSuccess;
  if (z.passes < 1 || z.passes > kMaxPasses) return cudaErrorInvalidValue;
  unsigned long long* status = reinterpret_cast<unsigned long long*>(ws.hist);
  uint32_t* ghist = ws.hist + (size_t)2 * kDigits * z.nchunks;
  uint32_t* chunk_ctr = ghist + kMaxPasses * kDigits;
  cudaError_t e = cudaMemsetAsync(ws.hist, 0, sizeof(uint32_t) * z.hist_words, s);
  if (e != cudaSuccess) return e;
  k_bin_keys<<<grid_for(m), 256, 0, s>>>(tab, ninst, m, prepared, (uint32_t)total_bins, z.passes,
                                         ws.keys[0], ws.vals[0], ghist);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int cur = 0;
  for (int pass = 0; pass < z.passes; ++pass) {
    const int last = pass == z.passes - 1;
    k_radix_pass<<<z.nchunks, kSortThreads, 0, s>>>(ws.keys[cur], ws.vals[cur], m, pass,
                                                    8 * z.passes, ghist, chunk_ctr, status,
                                                    ws.keys[cur ^ 1],
                                                    ws.vals[cur ^ 1], prepared, prepared_w, ws.spts,
                                                    ws.sw, last, ws.err, tc::kWaitLimitNs);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cur ^= 1;
  }
  k_bin_bounds<<<(int)((total_bins + 1 + 255) / 256), 256, 0, s>>>(ws.keys[cur], m,
                                                                   (int)total_bins, ws.start);
  note_launches(1);
  return cudaGetLastError();
}

size_t lookback_probe_words() {
  return 4 * 2 * kSortChunk + 2 * 2 * kDigits + kDigits + kMaxPasses;
}

cudaError_t launch_lookback_timeout_probe(uint32_t* buf, CallScalars* err, uint64_t limit_ns,
                                          cudaStream_t s) {
  // zero keys in two chunks; the chunk counter starts at 1, so the one
  // CTA takes chunk 1 and waits for a chunk 0 that never publishes
  constexpr int64_t m = 2 * kSortChunk;
  uint32_t* keys = buf;
  uint32_t* vals = keys + m;
  uint32_t* keys_out = vals + m;
  uint32_t* vals_out = keys_out + m;
  unsigned long long* status = reinterpret_cast<unsigned long long*>(vals_out + m);
  uint32_t* ghist = reinterpret_cast<uint32_t*>(status + 2 * kDigits);
  uint32_t* chunk_ctr = ghist + kDigits;
  cudaError_t e = cudaMemsetAsync(buf, 0, sizeof(uint32_t) * lookback_probe_words(), s);
  if (e != cudaSuccess) return e;
  const uint32_t one = 1;
  // a kernel-parameter write keeps the probe free of host-to-device copies
  e = launch_upload(&one, sizeof(one), chunk_ctr, s);
  if (e != cudaSuccess) return e;
  k_radix_pass<<<1, kSortThreads, 0, s>>>(keys, vals, m, 0, 8, ghist, chunk_ctr, status, keys_out,
                                          vals_out, nullptr, nullptr, nullptr, nullptr, 0, err,
                                          limit_ns);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_cutoff_eval(const CutInst* tab, int ninst, int64_t cut_bins, int64_t slice_bins,
                               const CutoffScratch& ws, cudaStream_t s) {
  if (ninst <= 0 || cut_bins <= 0) return cudaSuccess;
  if (cut_bins > 0x7fffffff || !ws.err) return cudaErrorInvalidValue;
  const int nb = (int)cut_bins, grid = (nb + 255) / 256;
  // per-key counts and cursors of the order, then the gather's item counter
  cudaError_t e = cudaMemsetAsync(ws.ocount, 0, sizeof(uint32_t) * kCutOcountWords, s);
  if (e != cudaSuccess) return e;
  k_cut_block_totals<<<grid, 256, 0, s>>>(tab, ninst, ws.start, nb, ws.totals, ws.ranges,
                                          ws.ocount);
  k_cut_order_scatter<<<grid, 256, 0, s>>>(tab, ninst, ws.totals, nb, ws.ocount, ws.order);
  // one CTA per item: every block, plus three more slices for each block of a
  // slicing instance that may turn out heavy
  const int64_t ctas = (int64_t)nb + (int64_t)(kSlices - 1) * slice_bins;
  if (ctas > 0x7fffffff) return cudaErrorInvalidValue;
  if ((e = cudaFuncSetAttribute(k_cutoff, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kCutSmemBytes)) != cudaSuccess)
    return e;
  k_cutoff<<<(unsigned)ctas, kGroups * kGroupThreads, kCutSmemBytes, s>>>(
      tab, ninst, ws.spts, ws.sw, ws.start, ws.order, ws.totals, ws.ranges,
      ws.ocount + 2 * kCutOrderKeys, nb, ws.err);
  note_launches(3);
  return cudaGetLastError();
}

}  // namespace kde
