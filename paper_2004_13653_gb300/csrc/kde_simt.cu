// Path (a): FP32 direct sum on the CUDA cores, any Table 1 kernel.
//
// Every Table 1 kernel is a product f(s,t) = k(s) k(t) (Sec. III-C), so a
// thread that owns an 8x8 block of cells evaluates 8 x-factors and 8
// y-factors per point and accumulates their outer product: 16 kernel
// evaluations and 64 FMAs per point instead of 64 evaluations.  Points are
// staged in shared memory in tiles of 256 (coalesced float4 loads, then
// broadcast reads).  Each thread sums one tile of points in registers and
// adds that partial into a (hi, lo) running sum in shared memory with an
// error-free two-sum, so the result does not degrade with the number of
// points a cell sees.
#include "kde_internal.cuh"
#include "kernel_factors.cuh"

namespace kde {
namespace {

constexpr int kThreads = 128;  // 16 (x) x 8 (y) threads
constexpr int kTileX = 128;    // cells along x per CTA (16 threads x 8, stride 16)
constexpr int kTileY = 64;     // cells along y per CTA (8 threads x 8, stride 8)
constexpr int kPtsTile = 256;  // points per shared-memory tile

template <int KID>
__global__ void __launch_bounds__(kThreads, 3)
    k_simt(const float4* __restrict__ pts, const float* __restrict__ wts, int64_t n_pad,
           int64_t per_split, const float2* __restrict__ gxt, const float2* __restrict__ gyt,
           int nx, int ny, float scale, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* sp = reinterpret_cast<float4*>(smem);                       // [kPtsTile]
  float* sw = reinterpret_cast<float*>(sp + kPtsTile);                // [kPtsTile]
  float2* run = reinterpret_cast<float2*>(sw + kPtsTile);             // [64][kThreads]

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int x0 = blockIdx.x * kTileX + tx;
  const int y0 = blockIdx.y * kTileY + ty;

  float gxh[8], gxl[8], gyh[8], gyl[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int x = min(x0 + 16 * a, nx - 1);
    const float2 g = gxt[x];
    gxh[a] = g.x;
    gxl[a] = g.y;
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int y = min(y0 + 8 * b, ny - 1);
    const float2 g = gyt[y];
    gyh[b] = g.x;
    gyl[b] = g.y;
  }
#pragma unroll
  for (int c = 0; c < 64; ++c) run[c * kThreads + tid] = make_float2(0.f, 0.f);

  const int64_t p_begin = (int64_t)blockIdx.z * per_split;
  int64_t p_end = p_begin + per_split;
  if (p_end > n_pad) p_end = n_pad;

  for (int64_t base = p_begin; base < p_end; base += kPtsTile) {
    __syncthreads();
    for (int q = tid; q < kPtsTile; q += kThreads) {
      const int64_t p = base + q;
      if (p < p_end) {
        sp[q] = pts[p];
        sw[q] = wts[p];
      } else {
        sp[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        sw[q] = 0.f;
      }
    }
    __syncthreads();

    float acc[8][8];
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int a = 0; a < 8; ++a) acc[b][a] = 0.f;

#pragma unroll 1
    for (int q = 0; q < kPtsTile; ++q) {
      const float4 P = sp[q];
      const float wq = sw[q];
      float kx[8], ky[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) kx[a] = kfactor<KID>((gxh[a] - P.x) + (gxl[a] - P.y));
#pragma unroll
      for (int b = 0; b < 8; ++b) ky[b] = wq * kfactor<KID>((gyh[b] - P.z) + (gyl[b] - P.w));
#pragma unroll
      for (int b = 0; b < 8; ++b)
#pragma unroll
        for (int a = 0; a < 8; ++a) acc[b][a] = fmaf(kx[a], ky[b], acc[b][a]);
    }
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        float2 r = run[(b * 8 + a) * kThreads + tid];
        two_sum_acc(r, acc[b][a]);
        run[(b * 8 + a) * kThreads + tid] = r;
      }
  }

  float* dst = part + (int64_t)blockIdx.z * nx * ny;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int y = y0 + 8 * b;
    if (y >= ny) continue;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int x = x0 + 16 * a;
      if (x >= nx) continue;
      const float2 r = run[(b * 8 + a) * kThreads + tid];
      dst[(int64_t)y * nx + x] = (r.x + r.y) * scale;
    }
  }
}

constexpr size_t kSmem = kPtsTile * (sizeof(float4) + sizeof(float)) +
                         64 * kThreads * sizeof(float2);

template <int KID>
cudaError_t launch_kid(const float4* pts, const float* wts, int64_t n_pad, const float2* gxt,
                       const float2* gyt, int nx, int ny, int splits, float scale, float* part,
                       cudaStream_t s) {
  // per-device attribute; cheap, so set on every launch
  cudaError_t e = cudaFuncSetAttribute(k_simt<KID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmem);
  if (e != cudaSuccess) return e;
  int64_t per = (n_pad + splits - 1) / splits;
  per = (per + kPtsTile - 1) / kPtsTile * kPtsTile;
  if (per < kPtsTile) per = kPtsTile;
  dim3 grid((nx + kTileX - 1) / kTileX, (ny + kTileY - 1) / kTileY, splits);
  k_simt<KID><<<grid, kThreads, kSmem, s>>>(pts, wts, n_pad, per, gxt, gyt, nx, ny, scale, part);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_simt(int kid, const float4* pts, const float* wts, int64_t n_pad,
                        const float2* gxt, const float2* gyt, int nx, int ny, int splits,
                        float scale, float* part, cudaStream_t s) {
  switch (kid) {
#define KDE_CASE(K) \
  case K:           \
    return launch_kid<K>(pts, wts, n_pad, gxt, gyt, nx, ny, splits, scale, part, s);
    KDE_CASE(KDE_UNIFORM)
    KDE_CASE(KDE_TRIANGULAR)
    KDE_CASE(KDE_EPANECHNIKOV)
    KDE_CASE(KDE_QUARTIC)
    KDE_CASE(KDE_TRIWEIGHT)
    KDE_CASE(KDE_TRICUBE)
    KDE_CASE(KDE_GAUSSIAN)
    KDE_CASE(KDE_COSINE)
#undef KDE_CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace kde
