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
// tile's piece partials, in piece order, into the output.
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

// One thread per tile: the points its bin rows hold, and its piece count.
// npieces has tiles_total + 1 entries; the last is zero so that the exclusive
// scan ends with the total.
__global__ void k_sparse_totals(const TcInst* __restrict__ tab, int ninst, SparseCtl sp,
                                uint32_t* __restrict__ tile_total, uint32_t* __restrict__ npieces) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > sp.tiles_total) return;
  if (t == sp.tiles_total) {
    npieces[t] = 0;
    return;
  }
  const TcInst& I = tab[inst_of_tile(tab, ninst, t)];
  const int local = t - I.tile_begin;
  const int tm = local % I.tiles_m, tn = local / I.tiles_m;
  const BinRange br = tile_bins(I.cs, I.reach, I.inv_binw, I.nbx, I.nby, tm, tn);
  uint64_t total = 0;
  for (int by = br.lo_by; br.lo_bx <= br.hi_bx && by <= br.hi_by; ++by) {
    const int row = I.bin_begin + by * I.nbx;
    total += I.start[row + br.hi_bx + 1] - I.start[row + br.lo_bx];
  }
  tile_total[t] = (uint32_t)total;
  npieces[t] = (uint32_t)((total + sp.piece_len - 1) / sp.piece_len);
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
                               uint32_t* npieces, uint32_t* scan_temp, CallScalars* err,
                               cudaStream_t s) {
  (void)err;
  const int m = sp.tiles_total + 1;
  k_sparse_totals<<<(m + 255) / 256, 256, 0, s>>>(tab, ninst, sp,
                                                  const_cast<uint32_t*>(sp.tile_total), npieces);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_exclusive_scan(npieces, const_cast<uint32_t*>(sp.piece_begin), m, 2048, scan_temp,
                               s);
}

cudaError_t launch_sparse_reduce(const TcInst* tab, int ninst, const SparseCtl& sp,
                                 cudaStream_t s) {
  k_sparse_reduce<<<dim3(sp.tiles_total, 16), 256, 0, s>>>(tab, ninst, sp);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace kde
