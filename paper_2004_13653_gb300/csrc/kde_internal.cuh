// Internal declarations shared by the library's translation units.
//
// Data layout in HBM (one call):
//   pts   float4[n_pad]  (x_hi, x_lo, y_hi, y_lo): centred, scaled coordinates
//                         X = (x - ox) * sigma split into two floats (hi + lo)
//   wts   float[n_pad]   weights (padding = 0)
//   gxt   float2[nx]     (hi, lo) of (i + 1/2) * cell * sigma
//   gyt   float2[ny]     (hi, lo) of (j + 1/2) * cell * sigma
//   part  float[S][ny][nx] split-K partial sums (S = 1: the output itself)
//   scal  CallScalars    device error word and |w| maximum
// sigma = 1/h for the compact kernels (offsets in bandwidths) and
// 1/(h sqrt(2 ln 2)) for the Gaussian, whose factor is then 2^(-u^2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kde.h"
#include "kde_diag.h"

namespace kde {

constexpr int kErrTimeout = 1;    // a bounded device-side wait gave up
constexpr int kErrNonFinite = 2;  // non-finite coordinate or weight
constexpr int kErrBadArg = 4;     // a kernel saw an impossible argument
constexpr int kErrNegWeight = 8;  // negative weight on a tensor-core path

struct CallScalars {
  int err;            // OR of kErr* bits
  unsigned wmax_bits; // bit pattern of max |w| (non-negative floats order as ints)
  int timeout_where;  // role id of the first wait that gave up
  int pad[61];        // keep the struct 256 bytes
};

// One factor k(s) of each Table 1 kernel without its constant; the constant
// squared and 1/(N h^2) are applied once to the sum.
__host__ __device__ inline double kernel_const_1d(int kid) {
  switch (kid) {
    case KDE_UNIFORM: return 0.5;
    case KDE_TRIANGULAR: return 1.0;
    case KDE_EPANECHNIKOV: return 0.75;
    case KDE_QUARTIC: return 15.0 / 16.0;
    case KDE_TRIWEIGHT: return 35.0 / 32.0;
    case KDE_TRICUBE: return 70.0 / 81.0;
    case KDE_GAUSSIAN: return 0.398942280401432677939946059934;  // 1/sqrt(2 pi)
    case KDE_COSINE: return 0.785398163397448309615660845820;    // pi/4
  }
  return 0.0;
}

// Coordinate scale sigma for a kernel and bandwidth.
inline double kernel_sigma(int kid, double h) {
  // Gaussian: exp(-s^2/2) = 2^(-u^2) with u = s / sqrt(2 ln 2)
  return kid == KDE_GAUSSIAN ? 1.0 / (h * 1.17741002251547469101) : 1.0 / h;
}

// -------------------------------------------------------------- launches
// All launch helpers enqueue on `s`, add the number of kernels they launched
// to the process-wide counter, and return the launch status.

void note_launches(int k);

cudaError_t launch_mercator(const double* lonlat, int64_t n, double lat0_deg, double* xy,
                            cudaStream_t s);

cudaError_t launch_prepare(const double* xy, const float* w, int64_t n, int64_t n_pad,
                           double ox, double oy, double sigma, float4* pts, float* wts,
                           CallScalars* scal, cudaStream_t s);

cudaError_t launch_grid_tables(int nx, int ny, double cell, double sigma, float2* gxt,
                               float2* gyt, cudaStream_t s);

// Path (a): FP32 SIMT direct sum into part[S][ny][nx] (scaled).
cudaError_t launch_simt(int kid, const float4* pts, const float* wts, int64_t n_pad,
                        const float2* gxt, const float2* gyt, int nx, int ny, int splits,
                        float scale, float* part, cudaStream_t s);

// Sum S partial grids in fixed order (s = 0, 1, ...) into out.
cudaError_t launch_reduce_splits(const float* part, int splits, int64_t cells, float* out,
                                 cudaStream_t s);

// Exclusive scan of m counts, `per_block` (<= 2048) per block, multi-block
// with propagation; temp needs scan_temp_words(m, per_block) words.
size_t scan_temp_words(int64_t m, int per_block);
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t m, int per_block,
                                  uint32_t* temp, cudaStream_t s);

// Path (c): binned cutoff evaluation of the compact kernels.
struct CutoffPlan {
  int nbx, nby, nbins;  // 32x32-cell bins
  int R;                // bins within reach of a point, per direction
  int nchunks;          // radix-sort blocks of 2048 keys
  int passes;           // 8-bit radix passes
  size_t hist_words, scan_words;
};
struct CutoffScratch {
  uint32_t* keys[2];
  uint32_t* vals[2];
  uint32_t* hist;
  uint32_t* hist_scan;
  uint32_t* scan_temp;
  uint32_t* start;  // [nbins + 1]
  float4* spts;     // points in bin order
  float* sw;
};
CutoffPlan plan_cutoff(int nx, int ny, double cell, double h, int64_t n_pad);
cudaError_t launch_cutoff(int kid, const CutoffPlan& c, const float4* pts, const float* wts,
                          int64_t n, int64_t n_pad, double cell, double h, const float2* gxt,
                          const float2* gyt, int nx, int ny, float scale, CutoffScratch ws,
                          float* out, cudaStream_t s);

// Path (b): Gaussian as a tcgen05 contraction.
struct TcPlan {
  int tile_n;      // 128 or 256 grid rows (y) per tile; tile_m is 128 (x)
  int split16;     // 0: single FP16, 1: hi/lo split (three products)
  int splits;      // point-range splits S (partials in part[S])
  int k_chunk;     // points per TMEM accumulator drain (multiple of 64)
  int ctas;        // persistent CTAs
  int skip_zero;   // skip (tile, stage) pairs whose operands are all zero
  int stage_points;  // 32 or 64 points per pipeline stage
};
size_t tc_smem_bytes(const TcPlan& p);
cudaError_t launch_tc(const TcPlan& plan, const float4* pts, const float* wts, int64_t n_pad,
                      const float2* gxt, const float2* gyt, int nx, int ny, float scale,
                      const CallScalars* scal_in, float* part, CallScalars* scal,
                      cudaStream_t s);

}  // namespace kde
