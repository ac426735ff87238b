// Block-sparse skipping for the Gaussian tensor-core path.
//
// In the factorisation F = c A B^T the operands are A[i,p] = 2^(15 - u^2) and
// B[j,p] = (w_p / w_max) 2^(15 - v^2) in FP16 (hi and lo parts for
// split-FP16), u and v the offsets between cell centre and point in units of
// h sqrt(2 ln 2) (the separable Gaussian of Table 1).  Beyond |u| = 6.45 the
// exact value is below 2^-26.6, so both FP16 parts round to zero: such a
// point contributes exactly nothing to any cell of a tile that lies that far
// from it along x or along y.  Skipping those (tile, point) pairs therefore
// changes no product, only which zeros are added.
//
// The points are sorted into 32 x 32-cell bins (the cutoff path's stable
// radix sort, with that reach); a 256 x 256 tile then needs only the bins
// within reach, i.e. one contiguous run of sorted points per bin row.  This
// file builds the work list (points per tile, cut into pieces of a fixed
// length, and the exclusive scan of the pieces per tile) and sums each
// tile's piece partials, in piece order, into the output.  The pieces of a
// tile all hold piece_len points except its last; the schedule lists the full
// pieces first and then the last pieces by decreasing length, so that dealing
// them to the CTA pairs in snake order balances the pairs' work.
#include "kde_internal.cuh"

namespace kde {
namespace {

__device__ __forceinline__ int inst_of_tile(const TcInst* __restrict__ tab, int ninst, int t) {
  int a = 0, b = ninst - 1;
  while (a < b) {
    const int mid = (a + b + 1) >> 1;
    if (tab[mid].tile_begin <= t) a = mid; else b = mid - 1;
  }
  return a;
}

// One thread per tile: the points its bin rows hold, its piece count and its
// count of full pieces.  npieces and nfull have tiles_total + 1 entries; the
// last are zero so that the exclusive scans end with the totals.
__global__ void k_sparse_totals(const TcInst* __restrict__ tab, int ninst, SparseCtl sp,
                                uint32_t* __restrict__ tile_total, uint32_t* __restrict__ npieces,
                                uint32_t* __restrict__ nfull) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > sp.tiles_total) return;
  if (t == sp.tiles_total) {
    npieces[t] = 0;
    nfull[t] = 0;
    return;
  }
  const TcInst& I = tab[inst_of_tile(tab, ninst, t)];
  const int local = t - I.tile_begin;
  const int tm = local % I.tiles_m, tn = local / I.tiles_m;
  const BinRange br = tile_bins(I.cs, I.range_reach, I.inv_binw, I.nbx, I.nby, tm, tn);
  uint64_t total = 0;
  for (int by = br.lo_by; br.lo_bx <= br.hi_bx && by <= br.hi_by; ++by) {
    const int row = I.bin_begin + by * I.nbx;
    total += I.start[row + br.hi_bx + 1] - I.start[row + br.lo_bx];
  }
  tile_total[t] = (uint32_t)total;
  npieces[t] = (uint32_t)((total + sp.piece_len - 1) / sp.piece_len);
  nfull[t] = (uint32_t)(total / sp.piece_len);
}

// Lists the tiles whose last piece is short, longest first: a counting sort
// on the piece's length in 512 classes (64-point MMA stages for the longest
// pieces the planner makes; one CTA; the order among tails of the same class
// is whatever the atomics give, which changes no result).
constexpr int kTailClasses = 512;
constexpr int kTailKeys = kTailClasses + 1;  // keys 1 .. kTailClasses
constexpr int kTailThreads = 1024;
static_assert(kTailKeys <= kTailThreads, "one key per thread in the scan");

// class of a short piece of rem points, 1 <= rem < L
__device__ __forceinline__ int tail_key(uint32_t rem, uint32_t L) {
  return 1 + (int)(((uint64_t)(rem - 1) * kTailClasses) / L);
}

__global__ void __launch_bounds__(kTailThreads) k_sparse_tails(SparseCtl sp) {
  __shared__ uint32_t cnt[kTailKeys];
  __shared__ uint32_t warp_sum[kTailThreads / 32];
  const int tid = threadIdx.x;
  const uint32_t L = (uint32_t)sp.piece_len;
  if (tid < kTailKeys) cnt[tid] = 0;
  __syncthreads();
  for (int t = tid; t < sp.tiles_total; t += kTailThreads) {
    const uint32_t rem = __ldg(sp.tile_total + t) % L;
    if (rem) atomicAdd(&cnt[tail_key(rem, L)], 1u);
  }
  __syncthreads();
  // exclusive scan with the longest key first: thread r holds key kTailKeys-1-r
  const int key = kTailKeys - 1 - tid;
  const uint32_t c = tid < kTailKeys ? cnt[key] : 0u;
  uint32_t v = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
    if ((tid & 31) >= o) v += n;
  }
  if ((tid & 31) == 31) warp_sum[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    uint32_t w = warp_sum[tid];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t n = __shfl_up_sync(0xffffffffu, w, o);
      if (tid >= o) w += n;
    }
    warp_sum[tid] = w;  // inclusive over warps
  }
  __syncthreads();
  const uint32_t before = v - c + ((tid >> 5) ? warp_sum[(tid >> 5) - 1] : 0u);
  __syncthreads();
  if (tid < kTailKeys) cnt[key] = before;  // now the cursor of each key
  __syncthreads();
  uint32_t* tail = const_cast<uint32_t*>(sp.tail_tile);
  for (int t = tid; t < sp.tiles_total; t += kTailThreads) {
    const uint32_t rem = __ldg(sp.tile_total + t) % L;
    if (rem) tail[atomicAdd(&cnt[tail_key(rem, L)], 1u)] = t;
  }
}

// out cell (i, j) of tile t = sum over the tile's pieces, in order.  Grid:
// (tiles, 16); thread = local column i, 16 local rows per block.
__global__ void __launch_bounds__(256)
    k_sparse_reduce(const TcInst* __restrict__ tab, int ninst, SparseCtl sp) {
  const int t = blockIdx.x;
  const TcInst& I = tab[inst_of_tile(tab, ninst, t)];
  const int local = t - I.tile_begin;
  const int tm = local % I.tiles_m, tn = local / I.tiles_m;
  const int il = threadIdx.x, i = tm * 256 + il;
  if (i >= I.nx) return;
  const int p0 = min((int)sp.piece_begin[t], sp.max_pieces);
  const int p1 = min((int)sp.piece_begin[t + 1], sp.max_pieces);
  for (int jl = blockIdx.y * 16; jl < blockIdx.y * 16 + 16; ++jl) {
    const int j = tn * 256 + jl;
    if (j >= I.ny) break;
    float acc = 0.f;
    for (int p = p0; p < p1; ++p) acc += sp.part[(int64_t)p * 65536 + jl * 256 + il];
    I.part[(int64_t)j * I.nx + i] = acc;
  }
}

}  // namespace

size_t sparse_scan_words(int tiles_total) {
  return scan_temp_words((int64_t)tiles_total + 1, 2048) + 64;
}

cudaError_t launch_sparse_plan(const TcInst* tab, int ninst, const SparseCtl& sp,
                               uint32_t* npieces, uint32_t* nfull, uint32_t* scan_temp,
                               CallScalars* err, cudaStream_t s) {
  (void)err;
  if (sp.piece_len <= 0) return cudaErrorInvalidValue;
  const int m = sp.tiles_total + 1;
  k_sparse_totals<<<(m + 255) / 256, 256, 0, s>>>(
      tab, ninst, sp, const_cast<uint32_t*>(sp.tile_total), npieces, nfull);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_exclusive_scan(npieces, const_cast<uint32_t*>(sp.piece_begin), m, 2048, scan_temp, s);
  if (e != cudaSuccess) return e;
  e = launch_exclusive_scan(nfull, const_cast<uint32_t*>(sp.full_begin), m, 2048, scan_temp, s);
  if (e != cudaSuccess) return e;
  k_sparse_tails<<<1, kTailThreads, 0, s>>>(sp);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sparse_reduce(const TcInst* tab, int ninst, const SparseCtl& sp,
                                 cudaStream_t s) {
  k_sparse_reduce<<<dim3(sp.tiles_total, 16), 256, 0, s>>>(tab, ninst, sp);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace kde
