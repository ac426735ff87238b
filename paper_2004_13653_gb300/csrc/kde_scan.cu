// Exclusive prefix sum over an array of unsigned counts, across many blocks.
//
// The multi-block scheme of Sec. IV-A ("Scan Algorithm"): every block scans
// its own piece, the per-block totals are collected and scanned in turn
// (recursively, until one block holds them all), and a propagation pass adds
// each block's scanned total to all of its elements.  The total that a block
// contributes is the sum of all its inputs -- including its last element -- so
// the propagation is correct where adding a block's last *scanned* value
// would drop that element (the pitfall the paper's note on the scan
// describes).  Within a block the scan is a per-thread sequential scan of a
// few consecutive elements followed by a warp-shuffle scan of the per-thread
// totals.
#include "kde_internal.cuh"

namespace kde {
namespace {

constexpr int kScanThreads = 256;

// Scan `per_block` elements per block; writes block totals to sums (if any).
__global__ void k_scan_blocks(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                              int64_t m, int per_block, uint32_t* __restrict__ sums) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * per_block;
  const int per_thread = (per_block + kScanThreads - 1) / kScanThreads;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t first = base + (int64_t)t * per_thread;
  const int64_t block_end = min(base + (int64_t)per_block, m);
  uint32_t vals[8];
  uint32_t tot = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t e = first + k;
    const uint32_t v = (k < per_thread && e < block_end) ? in[e] : 0u;
    vals[k] = tot;  // exclusive within the thread
    tot += v;
  }
  // exclusive scan of thread totals: warp shuffles, then across warps
  uint32_t incl = tot;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  uint32_t warp_off = 0, block_tot = 0;
  for (int w = 0; w < kScanThreads / 32; ++w) {
    if (w < warp) warp_off += warp_tot[w];
    block_tot += warp_tot[w];
  }
  const uint32_t off = warp_off + incl - tot;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t e = first + k;
    if (k < per_thread && e < block_end) out[e] = off + vals[k];
  }
  if (sums && t == 0) sums[blockIdx.x] = block_tot;
}

// Propagation: add each block's scanned total to its elements.
__global__ void k_scan_propagate(uint32_t* __restrict__ out, int64_t m, int per_block,
                                 const uint32_t* __restrict__ scanned_sums) {
  const uint32_t add = scanned_sums[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * per_block;
  for (int k = threadIdx.x; k < per_block; k += blockDim.x) {
    const int64_t e = base + k;
    if (e < m) out[e] += add;
  }
}

}  // namespace

size_t scan_temp_words(int64_t m, int per_block) {
  size_t words = 0;
  while (m > per_block) {
    const int64_t nb = (m + per_block - 1) / per_block;
    words += 2 * (size_t)nb + 64;
    m = nb;
  }
  return words;
}

cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t m, int per_block,
                                  uint32_t* temp, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  if (per_block < 1 || per_block > kScanThreads * 8) return cudaErrorInvalidValue;
  const int64_t nb = (m + per_block - 1) / per_block;
  if (nb > 0x7fffffff) return cudaErrorInvalidValue;
  if (nb == 1) {
    k_scan_blocks<<<1, kScanThreads, 0, s>>>(in, out, m, per_block, nullptr);
    note_launches(1);
    return cudaGetLastError();
  }
  uint32_t* sums = temp;
  uint32_t* sums_scanned = temp + nb;
  uint32_t* next = temp + 2 * nb + 64;
  k_scan_blocks<<<(int)nb, kScanThreads, 0, s>>>(in, out, m, per_block, sums);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_exclusive_scan(sums, sums_scanned, nb, per_block, next, s);
  if (e != cudaSuccess) return e;
  k_scan_propagate<<<(int)nb, kScanThreads, 0, s>>>(out, m, per_block, sums_scanned);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace kde
