// Throughput probes behind the rooflines: the tcgen05 FP16 MMA rate (CTA
// pairs, M = 256, N = 256, K = 16, and single CTAs, M = 128, N = 256) with
// the operands already in shared memory, and the MUFU ex2 rate.  They run at
// whatever clock the GPU is at, so a kernel's fraction of them compares like
// with like (the cuBLAS figure the bench also reports is taken under the power
// cap, at a lower clock).
#include <algorithm>

#include "kde_internal.cuh"
#include "tc_ptx.cuh"

namespace kde {
namespace {

using namespace tc;

// A: 128 rows of 64 FP16 (128 bytes); B: up to 256 such rows (single CTA,
// N = 256; a pair reads 128 rows of B in each CTA).
constexpr int kProbeABytes = 128 * 128;
constexpr int kProbeOperandBytes = kProbeABytes + 256 * 128;
constexpr int kProbeSmem = 160 * 1024;  // keeps one CTA per SM

// MMAs on zeroed, 128-byte-swizzled operands into two alternating
// accumulators; one thread issues them, the CTA waits (bounded) for the last.
template <bool PAIR>
__global__ void __launch_bounds__(128, 1) k_peak_mma(int iters, CallScalars* scal) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* done = reinterpret_cast<uint64_t*>(smem + kProbeOperandBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kProbeOperandBytes + 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kProbeOperandBytes + 12);
  for (int i = threadIdx.x; i < kProbeOperandBytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(done, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  if (threadIdx.x < 32) {
    if (PAIR) tmem_alloc_pair(tmem_slot, 512);
    else tmem_alloc(tmem_slot, 512);
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const bool issuer = threadIdx.x == 0 && (!PAIR || cluster_rank() == 0);
  if (issuer) {
    const uint32_t base = smem_u32(smem);
    const uint64_t da = desc_swz(base, 2u, 1024u);
    const uint64_t db = desc_swz(base + kProbeABytes, 2u, 1024u);
    constexpr uint32_t idesc = PAIR ? idesc_f16_f32(256, 256) : idesc_f16_f32(128, 256);
    for (int it = 0; it < iters; ++it) {
      const uint32_t d = tmem + ((it >> 2) & 1) * 256u;
      const uint64_t dk = (uint64_t)(2 * (it & 3));
      if (PAIR) mma_f16_pair(d, da + dk, db + dk, idesc, (it & 3) ? 1u : 0u);
      else mma_f16(d, da + dk, db + dk, idesc, (it & 3) ? 1u : 0u);
    }
    if (PAIR) mma_commit_pair(done);
    else mma_commit(done);
  }
  if (threadIdx.x == 0) mbar_wait(done, 0, abort_flag, scal, 31, /*honour_abort=*/false);
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync_all();
  if (threadIdx.x < 32) {
    tc_fence_after();
    if (PAIR) tmem_dealloc_pair(tmem, 512);
    else tmem_dealloc(tmem, 512);
  }
}

// Eight independent chains of ex2 per thread: v <- 2^-v maps (0, 1] into
// [1/2, 1), so the chains stay finite.
__global__ void __launch_bounds__(256) k_peak_ex2(int iters, float* sink) {
  float v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = 0.5f + 0.001f * (float)((threadIdx.x + k) & 255);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = ex2_neg(v[k]);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += v[k];
  if (s == 12345.f) sink[threadIdx.x] = s;  // keeps the chains live
}

template <class F>
int time_ms(F launch, cudaStream_t s, float* ms) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return -1;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return -1;
  }
  int rc = 0;
  if (cudaEventRecord(a, s) != cudaSuccess || launch() != cudaSuccess ||
      cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
      cudaEventElapsedTime(ms, a, b) != cudaSuccess)
    rc = -1;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

}  // namespace

// rates: [0] TFLOP/s of FP16 MMAs on CTA pairs, [1] on single CTAs,
// [2] ex2 results per second (1e12).  scal: a zeroed CallScalars in device
// memory (a wait that gives up sets kErrTimeout there).
cudaError_t run_peak_probes(int sms, CallScalars* scal, float* sink, double* rates,
                            cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_peak_mma<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_peak_mma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kProbeSmem);
  if (e != cudaSuccess) return e;
  auto failed = []() {
    const cudaError_t last = cudaGetLastError();
    return last != cudaSuccess ? last : cudaErrorUnknown;
  };
  const int clusters = std::max(1, sms / 2);
  const int iters = 1 << 16;
  for (int pass = 0; pass < 2; ++pass) {  // the first pass warms the clocks up
    float ms = 0.f;
    auto pair = [&]() {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(2 * clusters);
      cfg.blockDim = dim3(128);
      cfg.dynamicSmemBytes = kProbeSmem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      note_launches(1);
      return cudaLaunchKernelEx(&cfg, k_peak_mma<true>, iters, scal);
    };
    if (time_ms(pair, s, &ms)) return failed();
    rates[0] = 2.0 * 256 * 256 * 16 * (double)iters * clusters / (ms * 1e-3) / 1e12;
    auto one = [&]() {
      k_peak_mma<false><<<sms, 128, kProbeSmem, s>>>(iters, scal);
      note_launches(1);
      return cudaGetLastError();
    };
    if (time_ms(one, s, &ms)) return failed();
    rates[1] = 2.0 * 128 * 256 * 16 * (double)iters * sms / (ms * 1e-3) / 1e12;
    const int ex_iters = 1 << 14, blocks = sms * 8;
    auto ex2 = [&]() {
      k_peak_ex2<<<blocks, 256, 0, s>>>(ex_iters, sink);
      note_launches(1);
      return cudaGetLastError();
    };
    if (time_ms(ex2, s, &ms)) return failed();
    rates[2] = 8.0 * ex_iters * 256.0 * blocks / (ms * 1e-3) / 1e12;
  }
  return cudaSuccess;
}

}  // namespace kde
