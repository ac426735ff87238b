/*
 * kde.h — C ABI of the GB300 (sm_103a) kernel-density-on-a-grid library.
 *
 * The library computes the vessel-density surface of arXiv 2004.13653,
 * Sec. III-C (Eq. 7, Table 1), read as the direct sum over points
 *
 *     F[j*nx + i] = 1/(N h^2) * sum_p w_p * k((gx_i - x_p)/h) * k((gy_j - y_p)/h)
 *
 * at the cell centres gx_i = ox + (i + 1/2) cell, gy_j = oy + (j + 1/2) cell,
 * where k is one factor of a Table 1 product kernel f(s,t) = k(s) k(t) with
 * support |s| <= 1 (Eq. 8, s measured in bandwidths h), N is the number of
 * points (not the weight sum) and (x_p, y_p) are projected metres (Sec. III-A).
 *
 * Conventions shared by every entry point:
 *   - Return value: KDE_OK (0) or a negative KDE_E* code; kde_last_error()
 *     then holds a message for the calling thread.
 *   - Ownership: the caller owns every buffer it passes.  The library owns one
 *     internal device workspace per device (grown on demand with cudaMalloc,
 *     freed by kde_release()) unless the caller passes its own in kde_opts.
 *   - Memory spaces: "device" pointers must be CUDA device (or managed)
 *     memory; kde_grid / kde_grid_ex also accept host pointers for points,
 *     weights and out, which are then copied through the workspace.
 *   - Streams: kde_grid_ex and friends enqueue on opts->stream (a
 *     cudaStream_t; NULL = the legacy default stream) and return without
 *     waiting unless KDE_FLAG_SYNC is set.  kde_grid() always waits.
 *     Calls that use the library's workspace are ordered only by their
 *     streams: calls in flight at the same time on different streams of one
 *     device (from one host thread or several) must each pass their own
 *     workspace in kde_opts; on one stream, or on streams the caller orders
 *     with events, the library's workspace is safe.
 *   - Layout: points are interleaved (x0, y0, x1, y1, ...) FP64 metres;
 *     weights are FP32 (NULL = all ones); out is FP32 row-major [ny][nx]
 *     with out[j*nx + i] and is overwritten.
 */
#ifndef KDE_GB300_KDE_H
#define KDE_GB300_KDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define KDE_OK 0
#define KDE_EINVAL (-1)   /* bad argument (null, size, h, kernel id, ...)   */
#define KDE_ENOMEM (-2)   /* workspace allocation failed or too small       */
#define KDE_ECUDA (-3)    /* CUDA runtime / launch error                    */
#define KDE_ETIMEOUT (-4) /* a bounded device-side wait gave up             */
#define KDE_ENOTSUP (-5)  /* combination not supported (e.g. TC + compact)  */
#define KDE_EDATA (-6)    /* non-finite coordinate or weight (sync calls)   */

/* ---- kernels: Table 1 of the paper, in its row order -------------------- */
typedef enum {
  KDE_UNIFORM = 0,      /* k(s) = 1/2                       I(s)            */
  KDE_TRIANGULAR = 1,   /* k(s) = 1 - |s|                   I(s)            */
  KDE_EPANECHNIKOV = 2, /* k(s) = 3/4 (1 - s^2)             I(s)            */
  KDE_QUARTIC = 3,      /* k(s) = 15/16 (1 - s^2)^2         I(s)            */
  KDE_TRIWEIGHT = 4,    /* k(s) = 35/32 (1 - s^2)^3         I(s)            */
  KDE_TRICUBE = 5,      /* k(s) = 70/81 (1 - |s|^3)^3       I(s)            */
  KDE_GAUSSIAN = 6,     /* k(s) = exp(-s^2/2) / sqrt(2 pi)                  */
  KDE_COSINE = 7,       /* k(s) = pi/4 cos(pi s / 2)        I(s)            */
  /* Radial variants K(u) = c k~(|u|) on the unit disk (id = 8 + Table 1 id;
   * k~ the Table 1 profile without its constant, c = 1/(2 pi int r k~ dr) so
   * that K integrates to one).  They run on the cutoff path; the radial
   * Gaussian equals the product Gaussian and runs wherever KDE_GAUSSIAN does. */
  KDE_RADIAL_UNIFORM = 8,       /* c = 1/pi                                  */
  KDE_RADIAL_TRIANGULAR = 9,    /* c = 3/pi                                  */
  KDE_RADIAL_EPANECHNIKOV = 10, /* c = 2/pi                                  */
  KDE_RADIAL_QUARTIC = 11,      /* c = 3/pi                                  */
  KDE_RADIAL_TRIWEIGHT = 12,    /* c = 4/pi                                  */
  KDE_RADIAL_TRICUBE = 13,      /* c = 220/(81 pi)                           */
  KDE_RADIAL_GAUSSIAN = 14,     /* = KDE_GAUSSIAN                            */
  KDE_RADIAL_COSINE = 15        /* c = pi/(4 pi - 8)                         */
} kde_kernel;

/* ---- evaluation paths --------------------------------------------------- */
typedef enum {
  KDE_PATH_AUTO = 0,       /* Gaussian -> TC_SPLIT16, compact -> CUTOFF       */
  KDE_PATH_SIMT_FP32 = 1,  /* FP32 direct sum on the CUDA cores (Table 1)    */
  KDE_PATH_TC_FP16 = 2,    /* Gaussian as F = A B^T on tcgen05, FP16 operands */
  KDE_PATH_TC_SPLIT16 = 3, /* same, hi/lo FP16 operands, three products       */
  KDE_PATH_CUTOFF = 4      /* binned gather over the compact support          */
} kde_path;

#define KDE_FLAG_SYNC 1u         /* wait for completion and check device flags */
#define KDE_FLAG_SKIP_ZERO 2u    /* TC paths: block-sparse skipping. Points are */
                                 /* sorted into 32x32-cell bins and each 256x256*/
                                 /* tile reads only the bins within 6.45        */
                                 /* h sqrt(2 ln 2) (~7.6 h) of it; beyond that  */
                                 /* every FP16 operand is exactly zero, so no   */
                                 /* product changes (Table 1 Gaussian).  Runs   */
                                 /* on CTA pairs (KDE_ENOTSUP with ONE_CTA).    */
                                 /* Workspace grows by the piece partials.      */
#define KDE_FLAG_CTA_PAIR 4u     /* TC paths: 256x256 tiles on pairs of CTAs    */
                                 /* (tcgen05 cta_group::2); the default with    */
                                 /* 256-wide tiles                              */
#define KDE_FLAG_ONE_CTA 8u      /* TC paths: 128xN tiles on single CTAs        */
#define KDE_FLAG_LONLAT 16u      /* points are (lon, lat) in degrees: the call  */
                                 /* projects them with Eq. 1-4 (as            */
                                 /* kde_project_mercator at opts->lat0_deg)    */
                                 /* while centring them; origin, cell and h    */
                                 /* stay in projected metres                   */
#define KDE_FLAG_HOST_ASYNC 32u  /* with host buffers: return once the copies  */
                                 /* and kernels are queued on opts->stream     */
                                 /* instead of waiting for the result. The     */
                                 /* host buffers must stay valid and unchanged */
                                 /* until the stream has passed the call (and  */
                                 /* be pinned for the copies to overlap other  */
                                 /* work); out is valid after the caller       */
                                 /* synchronises the stream; device-side data  */
                                 /* errors are then not reported               */

typedef struct kde_args {
  const double* points; /* [2n] interleaved x,y metres (device or host)      */
  const float* weights; /* [n] or NULL for unit weights (device or host)     */
  int64_t n;            /* number of points N, >= 0                          */
  double origin_x;      /* lower-left corner of cell (0,0), metres           */
  double origin_y;
  double cell;          /* cell side, metres, > 0                            */
  int32_t nx, ny;       /* grid size, > 0, nx*ny < 2^31                      */
  double h;             /* bandwidth, metres, > 0 and finite                 */
  int32_t kernel_id;    /* kde_kernel                                        */
  float* out;           /* [ny*nx] result (device or host)                   */
} kde_args;

typedef struct kde_opts {
  int32_t path;           /* kde_path                                        */
  uint32_t flags;         /* KDE_FLAG_*                                      */
  void* stream;           /* cudaStream_t, NULL = legacy default stream      */
  void* workspace;        /* optional caller-owned device scratch ...        */
  size_t workspace_bytes; /* ... of at least kde_workspace_size() bytes      */
  int32_t split_k;        /* point-range splits, 0 = automatic               */
  int32_t k_chunk;        /* TC paths: points per accumulator drain, 0=auto  */
  int32_t tile_n;         /* TC paths: 128 or 256 grid rows per tile, 0=auto */
  int32_t max_ctas;       /* cap on resident CTAs (0 = one per SM)           */
  void* timing_events;    /* optional cudaEvent_t[2]: recorded on the stream */
                          /* right before / after the dominant kernel       */
  int32_t stage_points;   /* TC paths: 32 or 64 points per pipeline stage,  */
                          /* 0 = automatic                                  */
  double lat0_deg;        /* KDE_FLAG_LONLAT: standard latitude phi0 of     */
                          /* Eq. 1-4, in (-90, 90) degrees                  */
} kde_opts;

/* Fill *o with the defaults (AUTO path, legacy stream, library workspace). */
void kde_default_opts(kde_opts* o);

/*
 * kde_grid — the density of Sec. III-C (Eq. 7 read as a direct sum over
 * points, Table 1 kernels, Eq. 8 indicator) at the nx*ny cell centres.
 * points/weights/out may be device or host memory.  Runs on the calling
 * thread's kde_set_stream() stream (the legacy default stream unless set)
 * with the AUTO path and returns after completion.
 * Errors: KDE_EINVAL (null points with n > 0, null out, n < 0, nx/ny <= 0,
 * nx*ny >= 2^31, cell or h not positive and finite, unknown kernel_id,
 * non-finite origin), KDE_EDATA (a non-finite coordinate or weight),
 * KDE_ENOMEM, KDE_ECUDA, KDE_ETIMEOUT.  n = 0 writes zeros.
 */
int kde_grid(const double* points, const float* weights, int64_t n,
             const double grid_origin[2], double cell, int nx, int ny,
             double h, int kernel_id, float* out);

/* kde_set_stream — the CUDA stream (a cudaStream_t; NULL = the legacy
 * default stream, the initial setting) that kde_grid() runs on and waits for,
 * for the calling host thread only (Sec. III-C's density computed by
 * kde_grid as above; the stream is plumbing, without a counterpart in the
 * paper).  The stream must stay valid while kde_grid() calls use it.
 * kde_grid_ex and the other entry points take their stream from kde_opts. */
void kde_set_stream(void* stream);

/* kde_grid with explicit path, stream, workspace and tiling (Sec. III-C,
 * Eq. 7 / Table 1).  Asynchronous on opts->stream unless KDE_FLAG_SYNC.
 * opts may be NULL (defaults).  KDE_ENOTSUP for a TC path with a
 * non-Gaussian kernel (only the Gaussian row of Table 1 is separable into
 * exponential factors that a matrix product can sum). */
int kde_grid_ex(const kde_args* a, const kde_opts* opts);

/* Bytes of device workspace kde_grid_ex needs for these arguments/options
 * (for callers that pass their own workspace). */
int kde_workspace_size(const kde_args* a, const kde_opts* opts, size_t* bytes);

/*
 * kde_project_mercator — Sec. III-A, Eq. 1-4: (lon, lat) in degrees to
 * Mercator metres with r0 = a cos(phi0)/sqrt(1 - e^2 sin^2 phi0),
 * q = ln tan(pi/4 + phi/2) + (e/2) ln((1 - e sin phi)/(1 + e sin phi)),
 * x = lambda r0, y = q r0 (lambda in radians), WGS84 a = 6378137 m,
 * e^2 = 0.00669437999014.  lonlat_deg and xy_out: device, [2n] interleaved
 * FP64 (may alias).  FP64 throughout.  Asynchronous on stream.
 * Errors: KDE_EINVAL (n < 0, null or host pointers, |lat0| >= 90).
 */
int kde_project_mercator(const double* lonlat_deg, int64_t n, double lat0_deg,
                         double* xy_out, void* stream);

/*
 * kde_grid_batched — many independent densities (each one Sec. III-C, Eq. 7
 * with its own points, grid, h and kernel) in one persistent launch whose
 * work list spans all instances; the merged-buffer idea of Sec. IV-C-1
 * (all trajectories in one allocation with a length table) applied to
 * instances.  All pointers in inst[] must be device memory.  Each instance
 * runs the path AUTO would choose (Gaussian: split-FP16 tensor path,
 * compact kernels: binned cutoff path) unless opts->path forces
 * KDE_PATH_SIMT_FP32.  Asynchronous on opts->stream unless KDE_FLAG_SYNC;
 * graph-capturable when the workspace is already large enough (call once
 * outside capture, or pass opts->workspace).  When a batch holds both
 * Gaussian and compact instances (and no block-sparse ones), the compact
 * instances run on a library-owned low-priority stream forked from and joined
 * back to opts->stream by events, so they overlap the tensor-core
 * contraction; the call stays ordered on opts->stream as a whole.
 */
int kde_grid_batched(const kde_args* inst, int count, const kde_opts* opts);

/* Per-instance tiling of a tensor-core density in kde_grid_batched_tiled
 * (every field 0 = the call's own choice, as in kde_opts). */
typedef struct kde_tiling {
  int32_t tile_n;       /* 128 or 256 grid rows (y) per tile                 */
  int32_t k_chunk;      /* points per accumulator drain (multiple of 32, at  */
                        /* least twice the stage)                            */
  int32_t split_k;      /* point-range splits, 0..1024                       */
  int32_t stage_points; /* 32 or 64 points per pipeline stage                */
  uint32_t flags;       /* KDE_FLAG_CTA_PAIR (256 x 256 tiles on CTA pairs), */
                        /* KDE_FLAG_ONE_CTA (128 x tile_n tiles), or 0       */
} kde_tiling;

/*
 * kde_grid_batched_tiled — kde_grid_batched with a tiling per instance
 * (tiles[k] for inst[k]; NULL = kde_grid_batched), for instance the one an
 * autotuner measured best for that instance's class.  Tensor-core instances
 * that end up with the same tile shape and stage form one family; each family
 * is one persistent launch over its instances' work items (all in stream
 * order, still one call and capturable the same way).  The tiling is ignored
 * for non-tensor-core instances.  Errors as kde_grid_batched, plus KDE_EINVAL
 * for an invalid tiling and KDE_ENOTSUP for a one-CTA tiling with
 * KDE_FLAG_SKIP_ZERO.
 */
int kde_grid_batched_tiled(const kde_args* inst, const kde_tiling* tiles, int count,
                           const kde_opts* opts);

/*
 * kde_grid_backward — adjoint of the Gaussian density (Sec. III-C, Eq. 7
 * with the Gaussian row of Table 1).  Given G = dL/dF (device, [ny*nx]
 * FP32), writes dL/dpoints (device, [2n] FP32, interleaved), dL/dweights
 * (device [n] FP32, or NULL) and dL/dh (host double, or NULL):
 *   dL/dw_p = c sum_ij G_ij A_ip B_jp,
 *   dL/dx_p = c w_p sum_ij G_ij (gx_i - x_p)/h^2 A_ip B_jp (same for y),
 *   dL/dh   = -(2/h) sum_ij G_ij F_ij + c sum_p w_p sum_ij G_ij r^2/h^3 A B,
 * c = 1/(2 pi N h^2), A, B the 1-D Gaussian factors, recomputed on the fly.
 * Two forms: a window kernel that sums each point's +-8h window on the FP32
 * pipes (opts->path KDE_PATH_SIMT_FP32), and, for wide bandwidths, two
 * tcgen05 contractions U = G B and V = G^T A (split-FP16, three products;
 * KDE_PATH_TC_SPLIT16 or KDE_PATH_TC_FP16) whose epilogues fold U and V
 * into the per-point sums.  KDE_PATH_AUTO takes the contractions when the
 * window covers more than 0.6% of the grid padded to 256-cell tiles.
 * Requires a->points on the device and kernel_id == KDE_GAUSSIAN.  dL/dh
 * makes the call synchronous (and reports KDE_ETIMEOUT from the
 * contractions' bounded waits).
 */
int kde_grid_backward(const kde_args* a, const float* grad_out,
                      float* grad_points, float* grad_weights, double* grad_h,
                      const kde_opts* opts);

/*
 * kde_lscv_grid — least-squares cross-validation loss of the Gaussian
 * density on the grid (the paper chooses the bandwidth by eye, Sec. V-D;
 * this is its quantitative counterpart):
 *   L = cell^2 sum F^2 - (2/N) sum_p w_p bilerp(F - F_p, x_p),
 * F_p = w_p K(|g - x_p|/h)/(N h^2) point p's own term at the cell centres g
 * (K(u) = exp(-u^2/2)/(2 pi)), bilerp = bilinear interpolation between cell
 * centres with zero outside the grid; bilerp(F - F_p, x_p) is the
 * leave-one-out density at x_p interpolated from the grid.  F: device
 * [ny*nx] (as computed by kde_grid_ex for the same arguments).  Writes the loss to *loss (host),
 * dL/dF to grad_F (device [ny*nx], FP32), and the loss's direct partial
 * derivatives w.r.t. w_p and x_p (not through F) to grad_w_direct (device
 * [n]) and grad_points_direct (device [2n]); either may be NULL.  The
 * direct partial w.r.t. h is added to *grad_h_direct (host) when non-NULL.
 * Synchronous.
 */
int kde_lscv_grid(const kde_args* a, const float* F, double* loss,
                  float* grad_F, float* grad_w_direct,
                  float* grad_points_direct, double* grad_h_direct,
                  const kde_opts* opts);

/*
 * kde_grid_binned — the paper's own estimator (Sec. IV-B): the fixes are
 * projected onto the count matrix M_D (Algorithm 3; cell = floor((x - o) /
 * cell), fixes outside the grid are dropped), cells skipped between
 * consecutive fixes of one trajectory are added by linear interpolation
 * (Eq. InterX / InterY: round(i + c/c_max di), c = 1..c_max-1, when both
 * fixes are inside the grid and interpolate != 0), and M_D is convolved with
 * the window x window stencil f(s,t) = k(s cell/h) k(t cell/h) / (N h^2) of a
 * Table 1 kernel (Eq. 7, N = n fixes).  window: odd, <= 255, or 0 for the
 * compact support (2 floor(h/cell) + 1) or +-4 h for the Gaussian.  points:
 * device [2n] interleaved metres; traj_offsets: device [ntraj+1] trajectory
 * boundaries, or NULL for one trajectory; counts_out: device [ny*nx] int32
 * (optional); out: device [ny*nx] FP32; interpolated: host (optional, makes
 * the call synchronous) = number of interpolated cells added.  The counts are
 * exact integers (identical to a CPU evaluation); the convolution is FP32.
 * Errors: KDE_EINVAL (as kde_grid, plus window, offsets, host pointers).
 */
int kde_grid_binned(const double* points, const int64_t* traj_offsets, int64_t ntraj,
                    int64_t n, const double grid_origin[2], double cell, int nx, int ny,
                    double h, int kernel_id, int window, int interpolate, int32_t* counts_out,
                    float* out, int64_t* interpolated, const kde_opts* opts);

/*
 * kde_dp_simplify — Douglas-Peucker compression of vessel trajectories
 * (Sec. III-B, Eq. 9), computed level-synchronously as in Sec. IV-A: all
 * curve segments of all trajectories are split in the same iteration.  Both
 * ends of every trajectory are kept; a segment is split at the point of
 * largest VED (the first one on ties) when that VED is larger than eps; the
 * VED is the distance to the line through the segment's ends, or to its start
 * when both ends coincide.  The VED is evaluated in FP64 with every operation
 * rounded as written, so the kept set equals a sequential FP64 evaluation.
 * points: device [2n] interleaved metres (16-byte aligned); traj_offsets:
 * device [ntraj+1] rising from 0 to n, or NULL for one trajectory; eps >= 0
 * metres; keep: device [n] (1 = kept); out_points: device [2n] or NULL,
 * receives the kept points in order; out_offsets: device [ntraj+1] or NULL,
 * the trajectories' bounds in out_points; n_kept, iterations: host, optional.
 * Synchronous: every iteration runs inside one cooperative launch (the loop
 * ends on the device when an iteration keeps no point), and the call reads
 * the iteration count and the kept count back once.  Errors: KDE_EINVAL (n,
 * eps, pointers, alignment, offsets that do not rise from 0 to n), KDE_EDATA
 * (non-finite coordinate), KDE_ECUDA (the device cannot hold the cooperative
 * launch's CTAs at once).
 */
int kde_dp_simplify(const double* points, const int64_t* traj_offsets, int64_t ntraj,
                    int64_t n, double eps, uint8_t* keep, double* out_points,
                    int64_t* out_offsets, int64_t* n_kept, int* iterations,
                    const kde_opts* opts);

/*
 * kde_grid_noalloc — the FP32 SIMT density (path KDE_PATH_SIMT_FP32, one
 * point split) without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory
 * (a stream capture that forbids allocation, a real-time loop that must not
 * block on the allocator, a plugin whose host owns all device memory, a fixed
 * memory budget).  Its scratch is one static device array of 8 MiB per GPU,
 * reserved while the library is loaded; inputs needing more scratch (about
 * 400,000 points on a small grid; 20 bytes per point plus 8 per grid row and
 * column) are rejected with KDE_EINVAL before anything is launched.
 * kernel_id: a Table 1 kernel (0..7) or the radial Gaussian (14, the same
 * density as KDE_GAUSSIAN).  points, weights (or NULL) and out are device
 * memory, laid out as for kde_grid.  Asynchronous on `stream` (a
 * cudaStream_t, NULL = legacy default stream); non-finite inputs are not
 * reported.  Every call on a device shares the scratch and it keeps the last
 * call's contents: calls that overlap on the GPU race.  The first call on a
 * device looks up the scratch's device address and keeps it for the life of
 * the process; make that call before any stream capture.  A device reset
 * (cudaDeviceReset) or a non-primary driver context invalidates the kept
 * address and is not supported.  Errors: KDE_EINVAL, KDE_ECUDA.
 */
int kde_grid_noalloc(const double* points, const float* weights, int64_t n,
                     const double grid_origin[2], double cell, int nx, int ny, double h,
                     int kernel_id, float* out, void* stream);

/* Message for the last failing call on this thread ("" if none). */
const char* kde_last_error(void);

/* Free the library's workspaces on every device (safe to call any time no
 * call is in flight). */
int kde_release(void);

/* Number of kernels the library has launched in this process (all
 * devices, all entry points); a diagnostic for counting launches. */
int64_t kde_launch_count(void);

/* Library version string. */
const char* kde_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KDE_GB300_KDE_H */
