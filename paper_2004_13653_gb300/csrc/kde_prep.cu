// Steps before the density sum: the Mercator projection (Sec. III-A, Eq. 1-4)
// and the centring of the points and cell centres against the grid origin
// (the x - x_min of Eq. 5-6), both in FP64, followed by the split of each
// centred, scaled coordinate into two FP32 numbers hi + lo.  These are the
// only FP64 steps of the library: the projected coordinates are ~1e7 m and
// their differences must be resolved to millimetres.
#include "kde_internal.cuh"

namespace kde {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kWgs84A = 6378137.0;
constexpr double kWgs84E2 = 0.00669437999014;

// Eq. 1-4: x = lambda r0, y = q r0 with the isometric latitude q.
__global__ void k_mercator(const double* __restrict__ lonlat, int64_t n, double r0, double e,
                           double* __restrict__ xy) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const double2 ll = reinterpret_cast<const double2*>(lonlat)[p];
    const double lam = ll.x * (kPi / 180.0);
    const double phi = ll.y * (kPi / 180.0);
    const double es = e * sin(phi);
    const double q = log(tan(0.25 * kPi + 0.5 * phi)) + 0.5 * e * log((1.0 - es) / (1.0 + es));
    reinterpret_cast<double2*>(xy)[p] = make_double2(lam * r0, q * r0);
  }
}

__device__ __forceinline__ float2 split_hi_lo(double v) {
  const float hi = __double2float_rn(v);
  const float lo = __double2float_rn(v - (double)hi);
  return make_float2(hi, lo);
}

// Centre, scale, split; weights copied (unit when w == NULL); padding zeroed;
// max |w| reduced for the tensor path's operand scaling.
__global__ void k_prepare(const double* __restrict__ xy, const float* __restrict__ w, int64_t n,
                          int64_t n_pad, double ox, double oy, double sigma,
                          float4* __restrict__ pts, float* __restrict__ wts,
                          CallScalars* __restrict__ scal) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned wbits = 0;
  bool bad = false;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += stride) {
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    float wv = 0.f;
    if (p < n) {
      const double2 v = reinterpret_cast<const double2*>(xy)[p];
      const double X = (v.x - ox) * sigma;
      const double Y = (v.y - oy) * sigma;
      wv = w ? w[p] : 1.0f;
      if (isfinite(X) && isfinite(Y) && isfinite(wv)) {
        const float2 sx = split_hi_lo(X), sy = split_hi_lo(Y);
        r = make_float4(sx.x, sx.y, sy.x, sy.y);
        wbits = max(wbits, __float_as_uint(fabsf(wv)));
      } else {
        bad = true;
        wv = 0.f;
      }
    }
    pts[p] = r;
    wts[p] = wv;
  }
  // warp-level max, one atomic per warp
  for (int o = 16; o > 0; o >>= 1) wbits = max(wbits, __shfl_xor_sync(0xffffffffu, wbits, o));
  const unsigned anybad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (wbits) atomicMax(&scal->wmax_bits, wbits);
    if (anybad) atomicOr(&scal->err, kErrNonFinite);
  }
}

__global__ void k_grid_tables(int nx, int ny, double cell_sigma, float2* __restrict__ gxt,
                              float2* __restrict__ gyt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nx) gxt[t] = split_hi_lo(((double)t + 0.5) * cell_sigma);
  if (t < ny) gyt[t] = split_hi_lo(((double)t + 0.5) * cell_sigma);
}

int blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

}  // namespace

cudaError_t launch_mercator(const double* lonlat, int64_t n, double lat0_deg, double* xy,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const double phi0 = lat0_deg * (kPi / 180.0);
  const double r0 = kWgs84A * cos(phi0) / sqrt(1.0 - kWgs84E2 * sin(phi0) * sin(phi0));
  k_mercator<<<blocks_for(n, 256), 256, 0, s>>>(lonlat, n, r0, sqrt(kWgs84E2), xy);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_prepare(const double* xy, const float* w, int64_t n, int64_t n_pad,
                           double ox, double oy, double sigma, float4* pts, float* wts,
                           CallScalars* scal, cudaStream_t s) {
  if (n_pad <= 0) return cudaSuccess;
  k_prepare<<<blocks_for(n_pad, 256), 256, 0, s>>>(xy, w, n, n_pad, ox, oy, sigma, pts, wts,
                                                    scal);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_grid_tables(int nx, int ny, double cell, double sigma, float2* gxt,
                               float2* gyt, cudaStream_t s) {
  const int m = nx > ny ? nx : ny;
  k_grid_tables<<<(m + 255) / 256, 256, 0, s>>>(nx, ny, cell * sigma, gxt, gyt);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace kde
