// Split-K reduction: the point range of one density is cut into S slices that
// are summed into S partial grids; this adds them in the fixed order
// s = 0, 1, ..., S-1 so the result does not depend on scheduling.
#include "kde_internal.cuh"

namespace kde {
namespace {

__global__ void k_reduce_splits(const float* __restrict__ part, int splits, int64_t cells,
                                bool vec, float* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; c < cells; c += stride) {
    if (vec && c + 3 < cells) {
      float4 acc = reinterpret_cast<const float4*>(part + c)[0];
      for (int s = 1; s < splits; ++s) {
        const float4 v = reinterpret_cast<const float4*>(part + (int64_t)s * cells + c)[0];
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
      }
      reinterpret_cast<float4*>(out + c)[0] = acc;
    } else {
      for (int64_t e = c; e < c + 4 && e < cells; ++e) {
        float acc = part[e];
        for (int s = 1; s < splits; ++s) acc += part[(int64_t)s * cells + e];
        out[e] = acc;
      }
    }
  }
}

}  // namespace

cudaError_t launch_reduce_splits(const float* part, int splits, int64_t cells, float* out,
                                 cudaStream_t s) {
  if (cells <= 0) return cudaSuccess;
  int64_t blocks = (cells / 4 + 255) / 256 + 1;
  if (blocks > 152 * 8) blocks = 152 * 8;
  // float4 accesses only when every row start is 16-byte aligned
  const bool vec = (cells % 4) == 0 && (reinterpret_cast<uintptr_t>(part) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(out) % 16) == 0;
  k_reduce_splits<<<(int)blocks, 256, 0, s>>>(part, splits, cells, vec, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace kde
