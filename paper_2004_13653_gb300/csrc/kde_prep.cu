// Steps before the density sum: the Mercator projection (Sec. III-A, Eq. 1-4)
// and the centring of the points and cell centres against the grid origin
// (the x - x_min of Eq. 5-6), both in FP64, followed by the split of each
// centred, scaled coordinate into two FP32 numbers hi + lo.  These are the
// only FP64 steps of the library: the projected coordinates are ~1e7 m and
// their differences must be resolved to millimetres.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "kde_internal.cuh"

namespace kde {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kWgs84A = 6378137.0;
constexpr double kWgs84E2 = 0.00669437999014;

// Eq. 1-4: x = lambda r0, y = q r0 with the isometric latitude q.  Near the
// standard latitude phi0 (|phi - phi0| <= m.range) y comes from the
// Taylor series of q about phi0: the constant, linear and quadratic terms in
// FP64, the terms of order 3..7 (a few metres at most) in FP32.  Elsewhere the
// closed form is evaluated in FP64.  GB300's FP64 rate makes the closed form
// (two logarithms, a tangent and a sine per point) the slow part.
// MercParams: kx = r0 pi/180; y0 = r0 q(phi0); c_k = r0 q^(k)(phi0)/k!
// (c[] holds c3 .. c7); range: |phi - phi0| up to which the series is used.
using MercSeries = MercParams;

__device__ __forceinline__ double2 mercator_xy(double2 ll, const MercParams& m) {
  const double phi = ll.y * (kPi / 180.0);
  const double d = phi - m.phi0;
  double y;
  if (fabs(d) <= m.range) {
    const float df = (float)d;
    float t = m.c[4];
    t = fmaf(t, df, m.c[3]);
    t = fmaf(t, df, m.c[2]);
    t = fmaf(t, df, m.c[1]);
    t = fmaf(t, df, m.c[0]);
    y = fma(m.c2, d * d, fma(m.c1, d, m.y0)) + (double)(t * (df * df * df));
  } else {
    const double es = m.e * sin(phi);
    const double q = log(tan(0.25 * kPi + 0.5 * phi)) + 0.5 * m.e * log((1.0 - es) / (1.0 + es));
    y = q * m.r0;
  }
  return make_double2(ll.x * m.kx, y);
}

__global__ void k_mercator(const double* __restrict__ lonlat, int64_t n,
                           const __grid_constant__ MercParams m, double* __restrict__ xy) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
    reinterpret_cast<double2*>(xy)[p] =
        mercator_xy(reinterpret_cast<const double2*>(lonlat)[p], m);
}

// Truncated power series in d (order kOrd) on the host.
constexpr int kOrd = 8;
struct Series {
  double a[kOrd + 1];
};
Series series_mul(const Series& x, const Series& y) {
  Series r = {};
  for (int i = 0; i <= kOrd; ++i)
    for (int j = 0; i + j <= kOrd; ++j) r.a[i + j] += x.a[i] * y.a[j];
  return r;
}
Series series_recip(const Series& x) {  // x.a[0] != 0
  Series r = {};
  r.a[0] = 1.0 / x.a[0];
  for (int k = 1; k <= kOrd; ++k) {
    double s = 0.0;
    for (int j = 1; j <= k; ++j) s += x.a[j] * r.a[k - j];
    r.a[k] = -s / x.a[0];
  }
  return r;
}

// Taylor coefficients of q(phi0 + d) - q(phi0) from
// q'(phi) = (1 - e^2) / ((1 - e^2 sin^2 phi) cos phi), integrated term by term.
MercSeries mercator_series(double phi0, double r0, double e2) {
  Series sd = {}, cd = {};  // sin d, cos d
  double f = 1.0;
  for (int k = 0; k <= kOrd; ++k) {
    if (k > 0) f /= k;
    const double v = f * ((k / 2) % 2 ? -1.0 : 1.0);
    if (k % 2) sd.a[k] = v; else cd.a[k] = v;
  }
  Series sn = {}, cs = {};  // sin(phi0 + d), cos(phi0 + d)
  for (int k = 0; k <= kOrd; ++k) {
    sn.a[k] = sin(phi0) * cd.a[k] + cos(phi0) * sd.a[k];
    cs.a[k] = cos(phi0) * cd.a[k] - sin(phi0) * sd.a[k];
  }
  Series den = series_mul(sn, sn);
  for (int k = 0; k <= kOrd; ++k) den.a[k] = (k == 0 ? 1.0 : 0.0) - e2 * den.a[k];
  den = series_mul(den, cs);
  const Series qp = series_recip(den);  // q'/(1 - e^2)
  MercSeries m;
  const double e = sqrt(e2);
  const double s0 = sin(phi0);
  m.r0 = r0;
  m.kx = r0 * (kPi / 180.0);
  m.phi0 = phi0;
  m.y0 = r0 * (log(tan(0.25 * kPi + 0.5 * phi0)) + 0.5 * e * log((1.0 - e * s0) / (1.0 + e * s0)));
  m.c1 = r0 * (1.0 - e2) * qp.a[0];
  m.c2 = r0 * (1.0 - e2) * qp.a[1] / 2.0;
  for (int k = 3; k <= 7; ++k) m.c[k - 3] = (float)(r0 * (1.0 - e2) * qp.a[k - 1] / k);
  // range: the FP32 rounding of the order-3 term plus the first omitted term
  // stay below 2e-7 m (at most 0.01 rad, ~64 km of latitude)
  const double c3 = fabs(r0 * (1.0 - e2) * qp.a[2] / 3), c8 = fabs(r0 * (1.0 - e2) * qp.a[7] / 8);
  m.range = 0.01;
  while (m.range > 1e-4 && c3 * pow(m.range, 3) * 1.2e-7 + c8 * pow(m.range, 8) > 2e-7)
    m.range *= 0.9;
  m.e = e;
  return m;
}

__device__ __forceinline__ float2 split_hi_lo(double v) {
  const float hi = __double2float_rn(v);
  const float lo = __double2float_rn(v - (double)hi);
  return make_float2(hi, lo);
}

// Instance of flattened index p: the last entry whose begin <= p.
template <class T>
__device__ __forceinline__ int find_instance(const T* tab, int ninst, int64_t p) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].begin <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Centre, scale, split; weights copied (unit when w == NULL); padding zeroed;
// max |w| reduced per instance for the tensor path's operand scaling.  Every
// instance's n_pad is a multiple of 512, so a warp never straddles two.
__global__ void k_prepare(const PrepInst* __restrict__ tab, int ninst, int64_t total) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const PrepInst& I = tab[find_instance(tab, ninst, g)];
    const int64_t p = g - I.begin;
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    float wv = 0.f;
    bool bad = false;
    unsigned wbits = 0;
    if (p < I.n) {
      double2 v = reinterpret_cast<const double2*>(I.xy)[p];
      if (I.lonlat) v = mercator_xy(v, I.merc);  // Eq. 1-4 fused into the centring
      const double X = (v.x - I.ox) * I.sigma;
      const double Y = (v.y - I.oy) * I.sigma;
      wv = I.w ? I.w[p] : 1.0f;
      if (isfinite(X) && isfinite(Y) && isfinite(wv)) {
        const float2 sx = split_hi_lo(X), sy = split_hi_lo(Y);
        r = make_float4(sx.x, sx.y, sy.x, sy.y);
        wbits = __float_as_uint(fabsf(wv));
      } else {
        bad = true;
        wv = 0.f;
      }
    }
    I.pts[p] = r;
    I.wts[p] = wv;
    // warp-level max, one atomic per warp (all lanes share the instance)
    for (int o = 16; o > 0; o >>= 1) wbits = max(wbits, __shfl_xor_sync(0xffffffffu, wbits, o));
    const unsigned anybad = __any_sync(0xffffffffu, bad);
    const unsigned anyneg = __any_sync(0xffffffffu, wv < 0.f);
    if ((threadIdx.x & 31) == 0) {
      if (wbits) atomicMax(&I.scal->wmax_bits, wbits);
      if (anybad) atomicOr(&I.scal->err, kErrNonFinite);
      if (anyneg) atomicOr(&I.scal->negw, 1);
    }
  }
}

// Cell-centre tables: blockIdx.y = instance.
__global__ void k_grid_tables(const PrepInst* __restrict__ tab) {
  const PrepInst& I = tab[blockIdx.y];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < max(I.nx, I.ny);
       t += gridDim.x * blockDim.x) {
    if (t < I.nx) I.gxt[t] = split_hi_lo(((double)t + 0.5) * I.cell_sigma);
    if (t < I.ny) I.gyt[t] = split_hi_lo(((double)t + 0.5) * I.cell_sigma);
  }
}

constexpr int kBlobBytes = 31 * 1024;
struct Blob {
  unsigned char bytes[kBlobBytes];
};

__global__ void k_upload(const __grid_constant__ Blob blob, int nbytes, unsigned char* dst) {
  for (int i = threadIdx.x; i < nbytes; i += blockDim.x) dst[i] = blob.bytes[i];
}

int blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

}  // namespace

MercParams mercator_params(double lat0_deg) {
  const double phi0 = lat0_deg * (kPi / 180.0);
  const double r0 = kWgs84A * cos(phi0) / sqrt(1.0 - kWgs84E2 * sin(phi0) * sin(phi0));
  return mercator_series(phi0, r0, kWgs84E2);
}

cudaError_t launch_mercator(const double* lonlat, int64_t n, double lat0_deg, double* xy,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const MercParams m = mercator_params(lat0_deg);
  k_mercator<<<blocks_for(n, 256), 256, 0, s>>>(lonlat, n, m, xy);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_prepare(const PrepInst* tab, int ninst, int64_t total_pad, int max_side,
                           cudaStream_t s) {
  if (ninst <= 0) return cudaSuccess;
  if (total_pad > 0) {
    k_prepare<<<blocks_for(total_pad, 256), 256, 0, s>>>(tab, ninst, total_pad);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  dim3 grid((max_side + 255) / 256, ninst);
  k_grid_tables<<<grid, 256, 0, s>>>(tab);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_upload(const void* bytes, size_t nbytes, void* dst, cudaStream_t s) {
  static Blob blob;  // staging for the launch parameters (copied at launch)
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  const unsigned char* src = static_cast<const unsigned char*>(bytes);
  for (size_t off = 0; off < nbytes; off += kBlobBytes) {
    const int len = (int)std::min<size_t>(kBlobBytes, nbytes - off);
    memcpy(blob.bytes, src + off, len);
    k_upload<<<1, 256, 0, s>>>(blob, len, static_cast<unsigned char*>(dst) + off);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace kde
