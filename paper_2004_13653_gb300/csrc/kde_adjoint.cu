// Adjoint of the Gaussian density and the grid LSCV loss.
//
// Density (Sec. III-C, Eq. 7 read as a direct sum, Gaussian row of Table 1):
//   F_ij = c sum_p w_p A_ip B_jp,  A_ip = exp(-s_ip^2/2), B_jp = exp(-t_jp^2/2),
//   s_ip = (gx_i - x_p)/h, t_jp = (gy_j - y_p)/h, c = 1/(2 pi N h^2).
// For a cotangent G = dL/dF:
//   dL/dw_p = c sum_ij G_ij A_ip B_jp
//   dL/dx_p = c w_p / h sum_ij G_ij s_ip A_ip B_jp     (dA/dx_p = A s / h)
//   dL/dy_p = c w_p / h sum_ij G_ij t_jp A_ip B_jp
//   dL/dh   = -(2/h) sum_ij G_ij F_ij + c/h sum_p w_p sum_ij G_ij (s^2 + t^2) A B
// and sum_ij G_ij F_ij = sum_p w_p dL/dw_p, so F itself is not needed.
//
// One warp per point in turn, over batches of 32 points: lanes take the
// columns of the point's window (for a window of at most 16 columns, groups
// of lanes take alternate rows), the rows are walked in order, and the four
// sums are reduced across the warp in a fixed order (reproducible).  The sum
// over a window is separable: per row, three FMAs per cell form sum G A,
// sum G s A and sum G s^2 A, which the row's B and t then weight.  The window
// itself (FP64) is found once per point, by the lane that later writes the
// point's results; the batch's points, windows and sums pass between the
// lanes through shared memory.  The window spans +-8 bandwidths (clamped to
// the grid): beyond it every term is below exp(-32) of the largest, far under
// the accuracy of the FP32 sums.
#include "kde_internal.cuh"
#include "kernel_factors.cuh"

namespace kde {
namespace {

constexpr float kLog2e = 1.44269504088896340736f;

__device__ __forceinline__ float gauss(float s) { return ex2_approx(-0.5f * kLog2e * s * s); }

// COLS: window columns a lane keeps in registers per block of 32 * COLS
// columns (the host picks the smallest power of two that covers the window).
// A window of at most 16 columns takes 2^sub_log2 >= its width lanes per row
// and 32 / 2^sub_log2 rows at a time (sub_log2 = 5 otherwise).  The launch
// bounds are the blocks per SM each COLS fits without spilling registers.
template <int COLS>
__global__ void __launch_bounds__(256, COLS == 1 ? 5 : (COLS == 2 ? 4 : (COLS == 4 ? 3 : 1)))
    k_adjoint_gauss(const float4* __restrict__ pts, const float* __restrict__ wts, int64_t n,
                    const float* __restrict__ G, const float2* __restrict__ gxt,
                    const float2* __restrict__ gyt, int nx, int ny, double cell_s, int R,
                    int sub_log2, float c, float inv_h, float* __restrict__ grad_xy,
                    float* __restrict__ grad_w, double* __restrict__ hterm,
                    double* __restrict__ lterm) {
  // per warp: the batch's points, windows and reduced sums (one slot per point)
  __shared__ float4 sP[8][32];
  __shared__ int4 sWin[8][32];
  __shared__ float4 sSum[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // lanes in groups of 2^sub_log2 over the columns; group g takes rows g, g + ng, ...
  const int ci = lane & ((1 << sub_log2) - 1), rg = lane >> sub_log2, ng = 32 >> sub_log2;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t pb = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; pb < n;
       pb += warps * 32) {
    // Lane l prepares point pb + l: its window of cells within R of its cell
    // (X, Y in bandwidths).  This is the FP64 part, so it runs once per point
    // instead of once per lane of the warp.
    const int64_t pl = pb + lane;
    if (pl < n) {
      const float4 P = pts[pl];
      const double X = (double)P.x + (double)P.y, Y = (double)P.z + (double)P.w;
      const int ic = (int)floor(X / cell_s), jc = (int)floor(Y / cell_s);
      sP[wib][lane] = P;
      sWin[wib][lane] = make_int4(max(ic - R, 0), min(ic + R, nx - 1), max(jc - R, 0),
                                  min(jc + R, ny - 1));
    }
    __syncwarp();
    const int cnt = n - pb < 32 ? (int)(n - pb) : 32;
    for (int q = 0; q < cnt; ++q) {
      const float4 P = sP[wib][q];
      const int4 win = sWin[wib][q];
      const int i0 = win.x, i1 = win.y, j0 = win.z, j1 = win.w;
      float aw = 0.f, ax = 0.f, ay = 0.f, ah = 0.f;
      if (i0 <= i1 && j0 <= j1) {
        for (int ib = i0; ib <= i1; ib += 32 * COLS) {
          // per column: A, s A and s^2 A (zero outside the window)
          float A[COLS], SA[COLS], S2A[COLS];
          int col[COLS];
#pragma unroll
          for (int k = 0; k < COLS; ++k) {
            const int i = ib + ci + 32 * k;
            col[k] = i <= i1 ? i : -1;
            const float2 g = gxt[min(i, nx - 1)];
            const float S = (g.x - P.x) + (g.y - P.y);
            A[k] = col[k] >= 0 ? gauss(S) : 0.f;
            SA[k] = S * A[k];
            S2A[k] = S * SA[k];
          }
          // Rows in order, four per iteration so their loads are in flight
          // together.  The window sum is separable: with the lane's row sums
          // u = sum G A, v = sum G s A, x = sum G s^2 A,
          //   w += B u,  x_p += B v,  y_p += t B u,  h += B x + t^2 B u.
#pragma unroll 4
          for (int j = j0 + rg; j <= j1; j += ng) {
            const float2 g = gyt[j];
            const float t = (g.x - P.z) + (g.y - P.w);
            const float B = gauss(t);
            const float* Grow = G + (int64_t)j * nx;
            float u = 0.f, v = 0.f, x = 0.f;
#pragma unroll
            for (int k = 0; k < COLS; ++k) {
              const float Gv = col[k] >= 0 ? __ldg(Grow + col[k]) : 0.f;
              u = fmaf(Gv, A[k], u);
              v = fmaf(Gv, SA[k], v);
              x = fmaf(Gv, S2A[k], x);
            }
            const float Bu = B * u;
            aw += Bu;
            ax = fmaf(B, v, ax);
            ay = fmaf(t, Bu, ay);
            ah = fmaf(B, x, fmaf(t * t, Bu, ah));
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        aw += __shfl_xor_sync(0xffffffffu, aw, o);
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        ah += __shfl_xor_sync(0xffffffffu, ah, o);
      }
      if (lane == 0) sSum[wib][q] = make_float4(aw, ax, ay, ah);
    }
    __syncwarp();
    if (pl < n) {
      const float w = wts[pl];
      const float4 r = sSum[wib][lane];
      const float gw = c * r.x;
      if (grad_w) grad_w[pl] = gw;
      grad_xy[2 * pl] = c * w * inv_h * r.y;
      grad_xy[2 * pl + 1] = c * w * inv_h * r.z;
      hterm[pl] = (double)c * w * inv_h * r.w;
      lterm[pl] = (double)w * gw;
    }
    __syncwarp();
  }
}

// Fixed-order block sums of a double array: partial[b] = sum of block b's slice.
__global__ void k_sum_blocks(const double* __restrict__ v, int64_t n, int64_t per_block,
                             double* __restrict__ partial) {
  __shared__ double sh[256];
  const int64_t b0 = (int64_t)blockIdx.x * per_block;
  const int64_t b1 = min(b0 + per_block, n);
  double acc = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) acc += v[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// ----------------------------------------------------------------- LSCV

// Gd = 2 cell^2 F; per-block partial sums of F^2 (FP64).
__global__ void k_lscv_grid(const float* __restrict__ F, int64_t cells, double two_cell2,
                            double* __restrict__ G, double* __restrict__ sq_part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cells;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float f = F[q];
    if (G) G[q] = two_cell2 * f;
    acc += (double)f * f;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) sq_part[blockIdx.x] = sh[0];
}

// Per point: the leave-one-out term w_p bilerp(F - F_p, x_p) (the bilinear
// sample of F between cell centres, zero outside, minus the same sample of
// the point's own term F_p = w_p S, S = exp(-r^2/2h^2)/(2 pi N h^2)), the
// loss's direct partials (through the bilinear weights, w_p and F_p), and the
// scatter of -(2/N) w_p beta into the FP64 cotangent (atomic adds; in FP64
// their order does not show in the FP32 result).  FP64 throughout.
__global__ void k_lscv_points(const float4* __restrict__ pts, const float* __restrict__ wts,
                              int64_t n, const float* __restrict__ F, int nx, int ny,
                              double cells_per_h, double cell_h, double inv_cell, double inv_h,
                              double inv_N, double self_term, double* __restrict__ G,
                              float* __restrict__ gw_direct, float* __restrict__ gxy_direct,
                              double* __restrict__ loo, double* __restrict__ hdir) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const float4 P = pts[p];
    const double w = wts[p];
    const double X = (double)P.x + (double)P.y, Y = (double)P.z + (double)P.w;  // in h
    const double fx = X * cells_per_h - 0.5;
    const double fy = Y * cells_per_h - 0.5;
    const double fi = floor(fx), fj = floor(fy);
    const double ax = fx - fi, ay = fy - fj;
    double v = 0.0, sv = 0.0, dvx = 0.0, dvy = 0.0, dsx = 0.0, dsy = 0.0, sh = 0.0;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const double ii = fi + a, jj = fj + b;
        if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
        const int64_t q = (int64_t)jj * nx + (int64_t)ii;
        const double wx = a ? ax : 1.0 - ax, wy = b ? ay : 1.0 - ay, ww = wx * wy;
        const double ex = (a ? 1.0 : -1.0) * wy * inv_cell;  // d(wx wy)/dx_p
        const double ey = (b ? 1.0 : -1.0) * wx * inv_cell;
        const double dx = (ii + 0.5) * cell_h - X, dy = (jj + 0.5) * cell_h - Y;  // in h
        const double r2 = dx * dx + dy * dy;
        const double S = self_term * exp(-0.5 * r2);
        const double f = F[q];
        v += ww * f;
        sv += ww * S;
        dvx += ex * f;
        dvy += ey * f;
        dsx += ex * S + ww * S * dx * inv_h;
        dsy += ey * S + ww * S * dy * inv_h;
        sh += ww * S * (r2 - 2.0) * inv_h;
        if (G) atomicAdd(&G[q], -2.0 * inv_N * w * ww);
      }
    if (gw_direct) gw_direct[p] = (float)(-2.0 * inv_N * (v - 2.0 * w * sv));
    if (gxy_direct) {
      gxy_direct[2 * p] = (float)(-2.0 * inv_N * w * (dvx - w * dsx));
      gxy_direct[2 * p + 1] = (float)(-2.0 * inv_N * w * (dvy - w * dsy));
    }
    loo[p] = w * (v - w * sv);
    hdir[p] = w * w * sh;
  }
}

__global__ void k_to_float(const double* __restrict__ src, int64_t n, float* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride)
    dst[q] = (float)src[q];
}

int grid_blocks(int64_t n, int threads, int cap) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

}  // namespace

size_t sum_partials(int64_t n) { return (size_t)((n + 65535) / 65536) + 1; }

cudaError_t launch_sum(const double* v, int64_t n, double* partial, double* result,
                       cudaStream_t s) {
  const int64_t per = 65536;
  const int nb = (int)std::max<int64_t>(1, (n + per - 1) / per);
  k_sum_blocks<<<nb, 256, 0, s>>>(v, n, per, partial);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_blocks<<<1, 256, 0, s>>>(partial, nb, nb, result);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_gauss(const float4* pts, const float* wts, int64_t n, const float* G,
                                 const float2* gxt, const float2* gyt, int nx, int ny,
                                 double cell, double h, float* grad_xy, float* grad_w,
                                 double* hterm, double* lterm, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int R = (int)ceil(8.0 * h / cell) + 1;
  const float c = (float)(1.0 / (2.0 * 3.14159265358979323846 * (double)n * h * h));
  const int width = 2 * R + 1;
  const int blocks = grid_blocks((n + 31) / 32 * 32, 256, 152 * 64);  // a warp per 32 points
  int sub_log2 = 0;
  while ((1 << sub_log2) < width && sub_log2 < 5) ++sub_log2;
#define KDE_ADJ(C)                                                                          \
  k_adjoint_gauss<C><<<blocks, 256, 0, s>>>(pts, wts, n, G, gxt, gyt, nx, ny, cell / h, R,    \
                                            C == 1 ? sub_log2 : 5, c, (float)(1.0 / h),     \
                                            grad_xy, grad_w, hterm, lterm)
  if (width <= 32) KDE_ADJ(1);
  else if (width <= 64) KDE_ADJ(2);
  else if (width <= 128) KDE_ADJ(4);
  else KDE_ADJ(8);
#undef KDE_ADJ
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_lscv(const float4* pts, const float* wts, int64_t n, const float* F, int nx,
                        int ny, double cell, double h, double* Gd, float* G, float* gw_direct,
                        float* gxy_direct, double* sq_part, int sq_blocks, double* loo,
                        double* hdir, cudaStream_t s) {
  const int64_t cells = (int64_t)nx * ny;
  k_lscv_grid<<<sq_blocks, 256, 0, s>>>(F, cells, 2.0 * cell * cell, Gd, sq_part);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (n > 0) {
    const double self = 1.0 / (2.0 * 3.14159265358979323846) / ((double)n * h * h);
    k_lscv_points<<<grid_blocks(n, 256, 152 * 16), 256, 0, s>>>(
        pts, wts, n, F, nx, ny, h / cell, cell / h, 1.0 / cell, 1.0 / h, 1.0 / (double)n, self,
        Gd, gw_direct, gxy_direct, loo, hdir);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (G) {
    k_to_float<<<grid_blocks(cells, 256, 152 * 16), 256, 0, s>>>(Gd, cells, G);
    note_launches(1);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace kde
