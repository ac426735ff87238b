// Split-K reduction: the point range of a density is cut into S slices that
// are summed into S partial grids; this adds them in the fixed order
// s = 0, 1, ..., S-1 so the result does not depend on scheduling.  One launch
// serves every instance of a batch (flattened cell index, instance found by
// binary search on the table's begin).
#include "kde_internal.cuh"

namespace kde {
namespace {

__global__ void k_reduce(const ReduceInst* __restrict__ tab, int ninst, int64_t total) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tab[mid].begin <= g) lo = mid; else hi = mid - 1;
    }
    const ReduceInst& I = tab[lo];
    const int64_t c = g - I.begin;
    float acc = I.part[c];
    for (int s = 1; s < I.splits; ++s) acc += I.part[(int64_t)s * I.cells + c];
    I.out[c] = acc;
  }
}

}  // namespace

cudaError_t launch_reduce(const ReduceInst* tab, int ninst, int64_t total_cells, cudaStream_t s) {
  if (ninst <= 0 || total_cells <= 0) return cudaSuccess;
  int64_t blocks = (total_cells + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_reduce<<<(int)blocks, 256, 0, s>>>(tab, ninst, total_cells);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace kde
