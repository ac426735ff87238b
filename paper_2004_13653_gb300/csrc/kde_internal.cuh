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
// the bin sort's look-back gave up (set with kErrTimeout): the sorted order and
// the bin starts are then not trusted, and the kernels that walk the sorted
// points (the cutoff gather, the block-sparse contraction) skip their work;
// only the sort sets it, in a launch before theirs, so every CTA of theirs
// reads the same value
constexpr int kErrSortTimeout = 8;

struct CallScalars {
  int err;            // OR of kErr* bits
  unsigned wmax_bits; // bit pattern of max |w| (non-negative floats order as ints)
  int timeout_where;  // role id of the first wait that gave up
  int negw;           // nonzero when some weight is negative
  int pad[60];        // keep the struct 256 bytes
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

// Kernel ids 8..15: radial variants K(u) = c k(|u|) of the Table 1 kernels
// on the unit disk; c makes K integrate to one over the plane.
constexpr int kRadial = 8;
__host__ __device__ inline double kernel_const_radial(int kid) {
  constexpr double pi = 3.14159265358979323846;
  switch (kid) {
    case KDE_UNIFORM: return 1.0 / pi;                 // int_0^1 r dr = 1/2
    case KDE_TRIANGULAR: return 3.0 / pi;              // int r (1-r) = 1/6
    case KDE_EPANECHNIKOV: return 2.0 / pi;            // int r (1-r^2) = 1/4
    case KDE_QUARTIC: return 3.0 / pi;                 // int r (1-r^2)^2 = 1/6
    case KDE_TRIWEIGHT: return 4.0 / pi;               // int r (1-r^2)^3 = 1/8
    case KDE_TRICUBE: return 220.0 / (81.0 * pi);      // int r (1-r^3)^3 = 81/440
    case KDE_GAUSSIAN: return 1.0 / (2.0 * pi);
    case KDE_COSINE: return pi / (4.0 * pi - 8.0);     // int r cos(pi r/2) = 2/pi - 4/pi^2
  }
  return 0.0;
}

// Coordinate scale sigma for a kernel and bandwidth.
inline double kernel_sigma(int kid, double h) {
  // Gaussian: exp(-s^2/2) = 2^(-u^2) with u = s / sqrt(2 ln 2)
  return kid == KDE_GAUSSIAN ? 1.0 / (h * 1.17741002251547469101) : 1.0 / h;
}

// ------------------------------------------------------- instance tables
// Every launch is driven by a table of per-instance descriptors that lives in
// the workspace; a single density is a batch of one.  Tables are written by
// launch_upload (a kernel whose parameters carry the bytes), so a whole call
// can be captured in a CUDA graph.

constexpr int kMaxBatch = 256;  // instances per batched launch

// Eq. 1-4 at one standard latitude phi0, set up on the host (kde_prep.cu):
// x = lambda r0, y = r0 q(phi); near phi0 (|phi - phi0| <= range) y is the
// Taylor series of q about phi0 (y0 + c1 d + c2 d^2 in FP64, orders 3..7 in
// FP32), elsewhere the closed form with eccentricity e.
struct MercParams {
  double r0, kx, phi0, y0, c1, c2, range, e;
  float c[5];
};
// Parameters of the projection at standard latitude lat0_deg (|lat0| < 90).
MercParams mercator_params(double lat0_deg);

struct PrepInst {
  const double* xy;  // caller's points (device): metres, or (lon, lat) degrees when lonlat
  const float* w;    // caller's weights (device) or null
  float4* pts;       // prepared points, n_pad entries
  float* wts;
  float2* gxt;
  float2* gyt;
  CallScalars* scal;
  int64_t n, n_pad, begin;  // begin: offset in the flattened n_pad space
  double ox, oy, sigma, cell_sigma;
  int nx, ny;
  int lonlat;       // 1: xy holds (lon, lat) degrees, projected here with merc
  MercParams merc;
};

struct TcInst {
  const float4* pts;
  const float* wts;
  const float2* gxt;
  const float2* gyt;
  const CallScalars* scal;  // holds max |w| of the instance
  float* part;              // [splits][ny][nx]; with block-sparse skipping: the output
  int64_t n_pad, per_split;
  int nx, ny, tiles_m, tiles_n, splits, item_begin, chunk_stages;
  float base_scale;  // 2^-30 / (2 pi N h^2); times max |w|
  // block-sparse skipping (pts / wts then hold the points in bin order)
  const uint32_t* start;  // bin starts of the shared sort
  double cs, reach, inv_binw;  // cell and reach in prepared units, 1 / bin width
  double range_reach;          // reach plus the bin keys' FP32 rounding margin (ranges use it)
  int nbx, nby, bin_begin, tile_begin;
};

// Points of bin rows lo_by..hi_by, columns lo_bx..hi_bx can reach the block
// of w x h cells whose first cell is (cx0, cy0): every other point lies
// farther than `reach` (prepared units) from each of the block's cell centres
// along x or along y.  Used by the kernels that plan work and those that do it,
// so the two agree bit for bit.  An empty range has lo > hi.
struct BinRange {
  int lo_bx, hi_bx, lo_by, hi_by;
};
__host__ __device__ inline BinRange block_bins_rect(double cs, double reach, double inv_binw,
                                                    int nbx, int nby, int cx0, int cy0, int w,
                                                    int h) {
  BinRange r;
  const double x0 = ((double)cx0 + 0.5) * cs - reach, x1 = ((double)cx0 + w - 0.5) * cs + reach;
  const double y0 = ((double)cy0 + 0.5) * cs - reach, y1 = ((double)cy0 + h - 0.5) * cs + reach;
  r.lo_bx = (int)fmin((double)nbx, fmax(0.0, floor(x0 * inv_binw)));
  r.hi_bx = (int)fmin((double)(nbx - 1), floor(x1 * inv_binw));
  r.lo_by = (int)fmin((double)nby, fmax(0.0, floor(y0 * inv_binw)));
  r.hi_by = (int)fmin((double)(nby - 1), floor(y1 * inv_binw));
  return r;
}
// the same for a block of side x side cells
__host__ __device__ inline BinRange block_bins(double cs, double reach, double inv_binw, int nbx,
                                               int nby, int cx0, int cy0, int side) {
  return block_bins_rect(cs, reach, inv_binw, nbx, nby, cx0, cy0, side, side);
}
// the 256 x 256 tile (tm, tn) of the tensor-core paths
__host__ __device__ inline BinRange tile_bins(double cs, double reach, double inv_binw, int nbx,
                                              int nby, int tm, int tn) {
  return block_bins(cs, reach, inv_binw, nbx, nby, tm * 256, tn * 256, 256);
}

// Walks the bin-row runs of a block's range (the points of bins lo_bx..hi_bx
// of each row, contiguous in the sorted order) in increasing position order
// and maps a position of their concatenation to an index of the sorted
// points.  Positions must not decrease from call to call.
struct RunCursor {
  const uint32_t* start;
  int row0, nbx, lo_bx, hi_bx, by, hi_by;
  int64_t vr;         // position of the current run's first point
  uint32_t ra, rb;    // the current run in the sorted points
  __device__ __forceinline__ void load_run() {
    const int row = row0 + by * nbx;
    ra = __ldg(start + row + lo_bx);
    rb = __ldg(start + row + hi_bx + 1);
  }
  // start: bin starts of the sort; row0: first bin of the instance; the range
  // must not be empty
  __device__ __forceinline__ void init(const uint32_t* start_, int row0_, int nbx_,
                                       const BinRange& br) {
    start = start_;
    row0 = row0_;
    nbx = nbx_;
    lo_bx = br.lo_bx;
    hi_bx = br.hi_bx;
    by = br.lo_by;
    hi_by = br.hi_by;
    vr = 0;
    load_run();
  }
  // index of position v (v below the range's total)
  __device__ __forceinline__ int64_t map(int64_t v) {
    while (v >= vr + (int64_t)(rb - ra) && by < hi_by) {
      vr += rb - ra;
      ++by;
      load_run();
    }
    return (int64_t)ra + (v - vr);
  }
};
__host__ __device__ inline bool range_empty(const BinRange& br) {
  return br.lo_bx > br.hi_bx || br.lo_by > br.hi_by;
}

// Work list of the block-sparse contraction: each tile's points (its bin
// rows' runs, concatenated) cut into pieces of piece_len points; piece p of
// a tile has id piece_begin[tile] + p and owns partial tile `id` of `part`
// (256 x 256 floats, [j_local][i_local]).  The contraction takes the pieces
// in schedule order: first every full piece (tile by tile), then the
// shorter last pieces, longest first (tail_tile), dealt to the CTA pairs in
// snake order so their loads come out even.  The schedule decides only
// which CTA pair computes a piece, never what is summed or in which order.
struct SparseCtl {
  const uint32_t* piece_begin;  // [tiles_total + 1], exclusive scan of pieces per tile
  const uint32_t* full_begin;   // [tiles_total + 1], exclusive scan of full pieces per tile
  const uint32_t* tail_tile;    // [tiles_total] tiles with a short last piece, longest first
  const uint32_t* tile_total;   // [tiles_total] points that can reach each tile
  float* part;                  // [max_pieces][256][256]
  int tiles_total, piece_len, max_pieces;
};
// Longest piece the planner makes.
constexpr int kSparseMaxPiece = 32768;

// An instance of the bin sort (cutoff or block-sparse) and, for the cutoff
// path, of its evaluation.  Sort bins: nbx x nby bins of `bin` cells, keys
// from bin_begin; output blocks (cutoff): obx x oby blocks of kCutoffBin
// cells, CTAs from out_begin.
struct CutInst {
  const float2* gxt;
  const float2* gyt;
  float* out;
  int64_t n, n_pad, prep_begin, cut_begin;  // point ranges (prepared / cutoff spaces)
  double inv_binw, ext_x, ext_y, reach, cs; // reach: support radius, cs: cell side (prepared units)
  // reach widened by more than the FP32 rounding of the bin keys: every range
  // of bins (and the keys' reach test) uses it, so a point whose key landed
  // one bin off is still read by every block it can reach; the extra points
  // contribute exact zeros
  double range_reach;
  // the keys' FP32 constants: accepted coordinates [key_lo, key_hx] x
  // [key_lo, key_hy], 1 / bin width
  float key_lo, key_hx, key_hy, key_inv;
  int nbx, nby, bin_begin, nx, ny, kid;
  int obx, oby, out_begin;
  float scale;
  // heavy output blocks (4096 or more points within reach) are computed as
  // four 4-row slices: set for supports of at most 6 cells (4-cell sort bins),
  // where a slice reads about half of the block's points
  int slice;
};

struct ReduceInst {
  const float* part;
  float* out;
  int64_t cells, begin;  // begin: offset in the flattened cell space
  int splits;
};

// Write `bytes` host bytes to device memory `dst` in stream order (kernel
// launches carrying the bytes as parameters; capturable).
cudaError_t launch_upload(const void* bytes, size_t nbytes, void* dst, cudaStream_t s);

// -------------------------------------------------------------- launches
// All launch helpers enqueue on `s`, add the number of kernels they launched
// to the process-wide counter, and return the launch status.

void note_launches(int k);

// Set the calling thread's kde_last_error() message.
void set_error_message(const char* msg);

cudaError_t launch_mercator(const double* lonlat, int64_t n, double lat0_deg, double* xy,
                            cudaStream_t s);

// Centre / scale / split every instance's points and build its grid tables.
cudaError_t launch_prepare(const PrepInst* tab, int ninst, int64_t total_pad, int max_side,
                           cudaStream_t s);

// Path (a): FP32 SIMT direct sum into part[S][ny][nx] (scaled).
// scratch: simt_scratch_bytes(nx, ny, splits) of device memory for the
// running sums, or nullptr to keep them in shared memory (fewer CTAs per SM).
size_t simt_scratch_bytes(int nx, int ny, int splits);
cudaError_t launch_simt(int kid, const float4* pts, const float* wts, int64_t n_pad,
                        const float2* gxt, const float2* gyt, int nx, int ny, int splits,
                        float scale, float2* scratch, float* part, cudaStream_t s);

// Sum each instance's S partial grids in fixed order (s = 0, 1, ...).
cudaError_t launch_reduce(const ReduceInst* tab, int ninst, int64_t total_cells, cudaStream_t s);

// Exclusive scan of m counts, `per_block` (<= 2048) per block, multi-block
// with propagation; temp needs scan_temp_words(m, per_block) words.
size_t scan_temp_words(int64_t m, int per_block);
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t m, int per_block,
                                  uint32_t* temp, cudaStream_t s);

// Path (c): binned cutoff evaluation of the compact kernels.
struct CutoffGeom {
  int nbx, nby, nbins, bin;
  double inv_binw, ext_x, ext_y;
};
// Block sides in cells: the cutoff path's output blocks (one CTA each), and
// the block-sparse tensor-core work list's sort bins.
constexpr int kCutoffBin = 16;
constexpr int kSparseBin = 32;
// Sort bins of `bin` cells; cs: cell side in prepared units; reach: support
// radius in prepared units.
CutoffGeom cutoff_geometry(int nx, int ny, double cs, double reach, int bin);
// The reach the bin ranges use: the keys are computed in FP32 from the hi/lo
// coordinates, within 3 units of 2^-24 of the coordinate's magnitude (at most
// the geometry's extent) of the exact position; the margin is 8 such units
// plus a millionth of a bandwidth.
inline double range_reach(double reach, const CutoffGeom& g) {
  const double ext = g.ext_x > g.ext_y ? g.ext_x : g.ext_y;
  return reach + 1e-6 + 8.0 * 0x1p-24 * ext;
}
// The cutoff path's sort-bin side for a support of reach_cells cells: small
// enough that an output block reads little beyond its support's reach, large
// enough that the number of bins stays bounded.
int cutoff_sort_bin(int nx, int ny, double reach_cells);
struct CutoffScratch {
  uint32_t* keys[2];
  uint32_t* vals[2];
  uint32_t* hist;   // [hist_words] the sort's look-back status, digit histograms, counters
  uint32_t* start;  // [total bins + 1]
  float4* spts;     // points in bin order
  float* sw;
  uint32_t* order;  // [cutoff output blocks] the blocks, heaviest first
  uint32_t* totals; // [cutoff output blocks] points within reach of each block
  int4* ranges;     // [cutoff output blocks] each block's sort-bin range (BinRange)
  uint32_t* ocount; // [kCutOcountWords] per-key block counts and cursors, blocks to split,
                    // position of the first light block
  CallScalars* err; // where a timed-out wait of the sort's look-back is recorded
};
// Weight classes of the cutoff path's output blocks (by points within reach:
// 66 classes, and the same again above them for the heavy blocks the gather
// splits into row slices); the ocount scratch holds their counts, their
// cursors and the number of blocks to be split.
constexpr int kCutOrderClasses = 66;
constexpr int kCutOrderKeys = 2 * kCutOrderClasses;
constexpr int kCutOcountWords = 2 * kCutOrderKeys + 2;
struct CutoffSizes {
  int nchunks, passes;
  size_t hist_words;
};
CutoffSizes cutoff_sizes(int64_t m, int64_t total_bins);
// Keys, stable radix sort, bin starts and the permuted points for every
// instance of `tab` (cutoff instances and block-sparse tensor-core instances).
// One kernel computes the keys and the digit histograms of every pass; each
// 8-bit pass is then one kernel whose chunk offsets come from a decoupled
// look-back (bounded waits, recorded in ws.err); the last pass writes the
// permuted points.  ws.hist holds z.hist_words words of look-back state.
cudaError_t launch_bin_sort(const CutInst* tab, int ninst, int64_t m, int64_t total_bins,
                            const float4* prepared, const float* prepared_w, const CutoffSizes& z,
                            CutoffScratch ws, cudaStream_t s);
// The bounded wait of the sort's look-back, made to run out: one radix pass
// over two chunks of zero keys runs as the second chunk while the first never
// publishes, so it gives up after limit_ns and records a timeout (role 31) in
// err.  buf: lookback_probe_words() words of device memory.
size_t lookback_probe_words();
cudaError_t launch_lookback_timeout_probe(uint32_t* buf, CallScalars* err, uint64_t limit_ns,
                                          cudaStream_t s);
// The cutoff evaluation of the first ninst instances (output blocks
// 0..cut_bins-1, of which slice_bins belong to instances with CutInst::slice
// set): one CTA per block, or per 4-row slice of a heavy block.
cudaError_t launch_cutoff_eval(const CutInst* tab, int ninst, int64_t cut_bins, int64_t slice_bins,
                               const CutoffScratch& ws, cudaStream_t s);

// Adjoint of the Gaussian density (points prepared with sigma = 1/h) and the
// grid LSCV loss.  hterm / lterm: per-point FP64 terms of dL/dh.
cudaError_t launch_adjoint_gauss(const float4* pts, const float* wts, int64_t n, const float* G,
                                 const float2* gxt, const float2* gyt, int nx, int ny,
                                 double cell, double h, float* grad_xy, float* grad_w,
                                 double* hterm, double* lterm, cudaStream_t s);
// The same adjoint as two tcgen05 contractions (points prepared in the
// Gaussian's units, sigma = 1/(h sqrt(2 ln 2)), and their cell tables):
// U = G B and V = G^T A with the points' operands generated on chip.  ws:
// adjoint_tc_workspace(nx, ny) bytes (the cotangent's FP16 tiles and a status
// word); errors of its waits are recorded in ws's CallScalars.
size_t adjoint_tc_workspace(int nx, int ny);
cudaError_t launch_adjoint_gauss_tc(const float4* pts, const float* wts, int64_t n, const float* G,
                                    const float2* gxt, const float2* gyt, int nx, int ny,
                                    double cell, double h, float* grad_xy, float* grad_w,
                                    double* hterm, double* lterm, void* ws, int max_ctas,
                                    cudaStream_t s);
// Gd: FP64 scratch for the cotangent (cells), G: FP32 cotangent out; loo and
// hdir: per-point leave-one-out terms and direct dL/dh terms (sum hdir * 2/N).
cudaError_t launch_lscv(const float4* pts, const float* wts, int64_t n, const float* F, int nx,
                        int ny, double cell, double h, double* Gd, float* G, float* gw_direct,
                        float* gxy_direct, double* sq_part, int sq_blocks, double* loo,
                        double* hdir, cudaStream_t s);
// Fixed-order sum of n doubles into *result (device); partial needs
// sum_partials(n) doubles.
size_t sum_partials(int64_t n);
cudaError_t launch_sum(const double* v, int64_t n, double* partial, double* result,
                       cudaStream_t s);

// The paper's binned estimator: count matrix with interpolation (Algorithm 3)
// and the separable window x window convolution of Eq. 7.
int binned_window(int kid, double h, double cell, int window);
cudaError_t launch_binned(const double* xy, int64_t n, const int64_t* off, int64_t ntraj,
                          double ox, double oy, double cell, int nx, int ny, double h, int kid,
                          int window, int interpolate, int* counts, float* rowbuf,
                          unsigned long long* added, float* out, cudaStream_t s);

// Douglas-Peucker compression of every trajectory (level-synchronous;
// synchronous on `s`).  ws: dp_workspace_bytes(n) bytes.
size_t dp_workspace_bytes(int64_t n);
cudaError_t launch_dp(const double* xy, int64_t n, const int64_t* off, int64_t ntraj, double eps,
                      uint8_t* keep, double* out_xy, int64_t* out_off, void* ws,
                      CallScalars* scal, int64_t* n_kept, int* iterations, cudaStream_t s);

// Path (b): Gaussian as a tcgen05 contraction.
struct TcPlan {
  int tile_n;        // 128 or 256 grid rows (y) per tile; tile_m is 128 (x)
  int split16;       // 0: single FP16, 1: hi/lo split (three products)
  int splits;        // point-range splits S (partials in part[S])
  int k_chunk;       // points per TMEM accumulator drain
  int ctas;          // persistent CTAs
  int skip_zero;     // skip (tile, stage) pairs whose operands are all zero
  int stage_points;  // 32 or 64 points per pipeline stage
  int pair;          // 1: 256 x 256 tiles on CTA pairs (cta_group::2)
};
size_t tc_smem_bytes(const TcPlan& p);
// Diagnostic: one wait that times out after limit_ns (sets kErrTimeout).
cudaError_t launch_wait_timeout(CallScalars* scal, uint64_t limit_ns, cudaStream_t s);
// Diagnostic: measured tcgen05 FP16 rates (pairs, single CTAs; TFLOP/s) and
// the ex2 rate (1e12 per second) in rates[0..2].  sink: device, 256 floats.
cudaError_t run_peak_probes(int sms, CallScalars* scal, float* sink, double* rates,
                            cudaStream_t s);
// One persistent launch over the work items of every instance in `tab`.
cudaError_t launch_tc(const TcPlan& plan, const TcInst* tab, int ninst, int n_items,
                      CallScalars* err, cudaStream_t s);
// The same on CTA pairs (tiles_m / tiles_n of the table count 256-cell tiles).
// With sp != nullptr the work items are the pieces of the block-sparse work
// list (their count is read on the device).  sched (device, or nullptr for
// round robin): the items of each of the pair_clusters() CTA pairs, as
// offsets[clusters + 1] followed by the item indices.
int pair_clusters(const TcPlan& plan, int n_items);
cudaError_t launch_tc_pair(const TcPlan& plan, const TcInst* tab, int ninst, int n_items,
                           const SparseCtl* sp, const uint32_t* sched, CallScalars* err,
                           cudaStream_t s);
// Block-sparse work list: tile totals, pieces and full pieces per tile and
// their exclusive scans, the tail pieces ordered longest first.  npieces and
// nfull are [tiles_total + 1] scratch words.
size_t sparse_scan_words(int tiles_total);
cudaError_t launch_sparse_plan(const TcInst* tab, int ninst, const SparseCtl& sp,
                               uint32_t* npieces, uint32_t* nfull, uint32_t* scan_temp,
                               CallScalars* err, cudaStream_t s);
// Sum each tile's piece partials in order into the instance outputs.
cudaError_t launch_sparse_reduce(const TcInst* tab, int ninst, const SparseCtl& sp,
                                 cudaStream_t s);

}  // namespace kde
