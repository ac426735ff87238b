// The paper's own GPU estimator (Sec. IV-B): the fixes are projected onto the
// count matrix M_D with integer atomic adds (Algorithm 3), cells skipped
// between consecutive fixes of one trajectory are filled by linear
// interpolation (Eq. InterX / InterY), and M_D is convolved with a
// window x window stencil of a Table 1 kernel (Eq. 7).
//
// Counting: one thread per fix; the cell index is floor((x - o) / cell) with
// the FP64 division correctly rounded (a multiply by 1/cell decides it except
// within rounding distance of a cell edge), and the interpolated cells are
// floor(i + (c/c_max) di + 1/2) with c = 1..c_max-1, evaluated with
// explicitly rounded FP64 operations (no fused multiply-add), so the counts
// are bit-identical to a CPU evaluation.
// Integer atomics make the counts independent of scheduling.
//
// Convolution: the Table 1 kernels are products, so the 2-D stencil
// f(s,t) = k(s cell/h) k(t cell/h) / (N h^2) is applied as a row pass and a
// column pass; each pass stages a tile plus its halo in shared memory and
// keeps the 1-D stencil in registers.
#include <math.h>

#include "kde_internal.cuh"

namespace kde {
namespace {

constexpr int kMaxHalf = 127;  // window half-width limit (window <= 255)

// floor((v - o) / d) with the FP64 division correctly rounded, or -1 outside
// [0, n).  FP64 division is costly on this GPU, so the quotient is first
// taken as (v - o) * inv_d (inv_d = 1/d rounded): that product is within
// 3 ulp of the exact quotient, the rounded division within half an ulp, so
// unless the product lies within 4e-15 relative of an integer both have the
// same floor; only those rare cases divide.
__device__ __forceinline__ int64_t cell_index(double v, double o, double d, double inv_d, int n) {
  const double t = __dsub_rn(v, o);
  const double q = __dmul_rn(t, inv_d);
  double f = floor(q);
  const double frac = q - f;  // exact for |q| < 2^52
  if (!(fmin(frac, 1.0 - frac) > 4e-15 * fmax(fabs(q), 1.0)))
    f = floor(__ddiv_rn(t, d));
  if (!(f >= 0.0) || f >= (double)n) return -1;
  return (int64_t)f;
}

__global__ void k_count(const double* __restrict__ xy, int64_t n,
                        const int64_t* __restrict__ off, int64_t ntraj, double ox, double oy,
                        double cell, double inv_cell, int nx, int ny, int interpolate,
                        int* __restrict__ counts, unsigned long long* __restrict__ added) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long my_added = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const int64_t i = cell_index(xy[2 * p], ox, cell, inv_cell, nx);
    const int64_t j = cell_index(xy[2 * p + 1], oy, cell, inv_cell, ny);
    if (i < 0 || j < 0) continue;
    atomicAdd(&counts[j * nx + i], 1);
    if (!interpolate || p + 1 >= n) continue;
    // the fix's trajectory: the last k with off[k] <= p
    int64_t next_start = n;
    if (off) {
      int64_t lo = 0, hi = ntraj - 1;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= p) lo = mid; else hi = mid - 1;
      }
      next_start = off[lo + 1];
    }
    if (p + 1 >= next_start) continue;
    const int64_t i1 = cell_index(xy[2 * p + 2], ox, cell, inv_cell, nx);
    const int64_t j1 = cell_index(xy[2 * p + 3], oy, cell, inv_cell, ny);
    if (i1 < 0 || j1 < 0) continue;
    const int64_t di = i1 - i, dj = j1 - j;
    const int64_t adi = di < 0 ? -di : di, adj = dj < 0 ? -dj : dj;
    const int64_t cmax = adi > adj ? adi : adj;
    for (int64_t c = 1; c < cmax; ++c) {
      const double t = __ddiv_rn((double)c, (double)cmax);
      const int64_t ic = (int64_t)floor(__dadd_rn(__dadd_rn((double)i, __dmul_rn(t, (double)di)), 0.5));
      const int64_t jc = (int64_t)floor(__dadd_rn(__dadd_rn((double)j, __dmul_rn(t, (double)dj)), 0.5));
      atomicAdd(&counts[jc * nx + ic], 1);
      ++my_added;
    }
  }
  if (my_added) atomicAdd(added, my_added);
}

struct Stencil {
  float k[2 * kMaxHalf + 1];
};

constexpr int kTile = 128;     // outputs per block of the row pass
constexpr int kColTile = 64;   // rows per block of the column pass (static smem < 48 KB)

// Row pass: R(i, j) = sum_s k_s M(i - s, j) (cells outside the grid are zero).
// Rows are strided over gridDim.y (which is capped at 65535).
__global__ void k_conv_rows(const int* __restrict__ counts, int nx, int ny, int a,
                            const __grid_constant__ Stencil st, float* __restrict__ R) {
  __shared__ float line[kTile + 2 * kMaxHalf];
  const int i0 = blockIdx.x * kTile;
  for (int j = blockIdx.y; j < ny; j += gridDim.y) {
    for (int t = threadIdx.x; t < kTile + 2 * a; t += blockDim.x) {
      const int i = i0 - a + t;
      line[t] = (i >= 0 && i < nx) ? (float)counts[(int64_t)j * nx + i] : 0.f;
    }
    __syncthreads();
    const int i = i0 + threadIdx.x;
    if (threadIdx.x < kTile && i < nx) {
      float acc = 0.f;
      for (int s = -a; s <= a; ++s) acc = fmaf(st.k[s + a], line[threadIdx.x + a - s], acc);
      R[(int64_t)j * nx + i] = acc;
    }
    __syncthreads();
  }
}

// Column pass: out(i, j) = norm sum_t k_t R(i, j - t); block = 32 columns x
// kColTile rows, each thread walks its column.
__global__ void k_conv_cols(const float* __restrict__ R, int nx, int ny, int a,
                            const __grid_constant__ Stencil st, float norm,
                            float* __restrict__ out) {
  __shared__ float col[kColTile + 2 * kMaxHalf][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * kColTile;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int r = ty; r < kColTile + 2 * a; r += 8) {
    const int j = j0 - a + r, i = i0 + tx;
    col[r][tx] = (j >= 0 && j < ny && i < nx) ? R[(int64_t)j * nx + i] : 0.f;
  }
  __syncthreads();
  const int i = i0 + tx;
  if (i >= nx) return;
  for (int r = ty; r < kColTile; r += 8) {
    const int j = j0 + r;
    if (j >= ny) break;
    float acc = 0.f;
    for (int t = -a; t <= a; ++t) acc = fmaf(st.k[t + a], col[r + a - t][tx], acc);
    out[(int64_t)j * nx + i] = acc * norm;
  }
}

// One factor k(s) of a Table 1 kernel with its constant, in double (host side).
double table1_factor(int kid, double s) {
  const double a = fabs(s);
  const bool in = a <= 1.0;
  switch (kid) {
    case KDE_UNIFORM: return in ? 0.5 : 0.0;
    case KDE_TRIANGULAR: return in ? 1.0 - a : 0.0;
    case KDE_EPANECHNIKOV: return in ? 0.75 * (1.0 - s * s) : 0.0;
    case KDE_QUARTIC: return in ? 15.0 / 16.0 * (1.0 - s * s) * (1.0 - s * s) : 0.0;
    case KDE_TRIWEIGHT: {
      const double u = 1.0 - s * s;
      return in ? 35.0 / 32.0 * u * u * u : 0.0;
    }
    case KDE_TRICUBE: {
      const double u = 1.0 - a * a * a;
      return in ? 70.0 / 81.0 * u * u * u : 0.0;
    }
    case KDE_GAUSSIAN: return kernel_const_1d(KDE_GAUSSIAN) * exp(-0.5 * s * s);
    default: return in ? kernel_const_1d(KDE_COSINE) * cos(1.5707963267948966 * s) : 0.0;
  }
}

}  // namespace

int binned_window(int kid, double h, double cell, int window) {
  if (window > 0) return window;
  const double r = h / cell;
  const int a = kid == KDE_GAUSSIAN ? (int)ceil(4.0 * r) : (int)floor(r);
  return 2 * (a < kMaxHalf ? a : kMaxHalf) + 1;
}

cudaError_t launch_binned(const double* xy, int64_t n, const int64_t* off, int64_t ntraj,
                          double ox, double oy, double cell, int nx, int ny, double h, int kid,
                          int window, int interpolate, int* counts, float* rowbuf,
                          unsigned long long* added, float* out, cudaStream_t s) {
  const int a = (window - 1) / 2;
  if (window < 1 || (window & 1) == 0 || a > kMaxHalf) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)nx * ny, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(added, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_count<<<(int)blocks, 256, 0, s>>>(xy, n, off, ntraj, ox, oy, cell, 1.0 / cell, nx, ny,
                                        interpolate, counts, added);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  Stencil st;
  for (int t = -a; t <= a; ++t) st.k[t + a] = (float)table1_factor(kid, t * cell / h);
  const float norm = n > 0 ? (float)(1.0 / ((double)n * h * h)) : 0.0f;
  k_conv_rows<<<dim3((nx + kTile - 1) / kTile, ny < 65535 ? ny : 65535), kTile, 0, s>>>(
      counts, nx, ny, a, st, rowbuf);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_conv_cols<<<dim3((nx + 31) / 32, (ny + kColTile - 1) / kColTile), 256, 0, s>>>(
      rowbuf, nx, ny, a, st, norm, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace kde
