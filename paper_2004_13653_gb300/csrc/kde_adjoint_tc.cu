// Adjoint of the Gaussian density as two tcgen05 contractions (Eq. 7 with
// the Gaussian row of Table 1), the form for wide bandwidths.
//
// With A_ip = 2^(-u_ip^2), B_jp = 2^(-v_jp^2) (u, v: offsets of cell and
// point in units of h sqrt(2 ln 2)) and a cotangent G = dL/dF,
//   U_ip = sum_j G_ij B_jp   (contraction 1, over the y cells)
//   V_jp = sum_i G_ij A_ip   (contraction 2, over the x cells)
//   dL/dw_p = c sum_i A_ip U_ip
//   dL/dx_p = c w_p sqrt(2 ln 2)/h sum_i u_ip A_ip U_ip
//   dL/dy_p = c w_p sqrt(2 ln 2)/h sum_j v_jp B_jp V_jp
//   h-term  = c w_p (2 ln 2)/h [sum_i u^2 A U + sum_j v^2 B V]
// (c = 1/(2 pi N h^2)).  Each contraction is D[p, n] = sum_k E[p, k] T[n, k]
// with M = 128 points per tile (TMEM lanes), N = 256 cells of the
// accumulated axis per accumulator (TMEM columns) and K = the other axis, 64
// cells per stage:
//   - E (the generated operand, rows = points): 2^(15 - (g_k - y_p)^2) for
//     contraction 1 (2^(15 - (g_k - x_p)^2) for 2), made by producer warps
//     in shared memory as FP16 hi/lo, as the forward makes its operands;
//   - T (rows = cells of the accumulated axis): the cotangent, scaled by a
//     power of two so its largest entry is near 2^14, split into FP16 hi/lo
//     and laid out beforehand in global memory exactly as a stage wants it in
//     shared memory (128-byte swizzled K-major rows), so one bulk copy (async
//     proxy, completing on an mbarrier) moves each stage's 64 KB;
//   - three FP16 MMAs per K step (hi*hi, hi*lo, lo*hi), FP32 accumulation in
//     TMEM; two accumulators alternate between consecutive N tiles, so the
//     MMAs never wait for the epilogue;
//   - the epilogue regenerates the factor of the accumulated axis for each of
//     its cells and folds U (or V) into three per-point sums, so neither U
//     nor V ever leaves the SM.
// The work is N_pad * nx_pad * ny_pad multiply-adds per contraction, against
// N * (16 h / cell)^2 cells for the window kernel of kde_adjoint.cu: the
// library takes this form when the window is the larger.
#include <cuda_fp16.h>

#include <algorithm>

#include "kde_internal.cuh"
#include "tc_ptx.cuh"

namespace kde {
namespace {

using namespace tc;

constexpr int kM = 128;       // points per tile (TMEM lanes)
constexpr int kN = 256;       // cells of the accumulated axis per accumulator
constexpr int kK = 64;        // cells of the contracted axis per stage
constexpr int kStages = 2;
constexpr int kRowBytes = 2 * kK;                         // 64 FP16 per operand row
constexpr int kEBytes = kM * kRowBytes;                   // 16 KB per part
constexpr int kTBytes = kN * kRowBytes;                   // 32 KB per part
constexpr int kStageBytes = 2 * (kEBytes + kTBytes);      // hi and lo: 96 KB
constexpr int kWarps = 14;    // 0 MMA, 1 bulk loader, 2-9 epilogue, 10-13 producers
constexpr int kThreads = 32 * kWarps;
constexpr int kFirstEpiWarp = 2, kEpiWarps = 8, kFirstProducerWarp = 10;
constexpr uint32_t kIdesc = idesc_f16_f32(kM, kN);
constexpr int kOffBars = kStages * kStageBytes;
constexpr int kNumBars = 3 * kStages + 4 + 1;
constexpr int kOffComb = kOffBars + kNumBars * 8;         // [4][32][3] doubles
constexpr int kOffMisc = kOffComb + 4 * 32 * 3 * 8;
constexpr int kSmemBytes = kOffMisc + 64 + 1024;
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
constexpr int kBarEpi = 1;    // named barrier of the epilogue warps

enum Role : int { kRoleMma = 21, kRoleLoader = 22, kRoleEpilogue = 23, kRoleProducer = 24 };

struct AdjTcArgs {
  const float4* pts;        // prepared points (Gaussian units), n_pad entries
  const float* wts;
  int64_t n;
  const unsigned char* tiles;  // [n_tiles][n_stages][part][kN rows][128 B]
  const float2* acc_tab;    // cell centres of the accumulated axis (hi, lo)
  const float2* k_tab;      // cell centres of the contracted axis
  int acc_cells, k_cells, n_tiles, n_stages;
  float cs;                 // cell side in prepared units
  int axis;                 // 0: x accumulated (dL/dw, dL/dx, h), 1: y (dL/dy, h)
  const CallScalars* gscal; // wmax_bits: max |G|
  double c;                 // 1/(2 pi N h^2)
  double k_xy, k_h;         // sqrt(2 ln 2)/h and 2 ln 2/h
  float* grad_xy;
  float* grad_w;
  double* hterm;
  double* lterm;
};

// The power of two the cotangent is scaled by before the FP16 split.
__host__ __device__ inline int g_exponent(unsigned gmax_bits) {
  if (gmax_bits == 0u || gmax_bits >= 0x7f800000u) return 0;
  const int e = (int)((gmax_bits >> 23) & 0xff) - 127;  // floor(log2 max|G|)
  return max(-100, min(100, 13 - e));
}

// max |G| into gscal->wmax_bits (non-negative floats order as unsigned ints).
__global__ void k_abs_max(const float* __restrict__ G, int64_t cells, CallScalars* gscal) {
  unsigned m = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cells; q += stride) {
    const float v = fabsf(G[q]);
    if (v == v) m = max(m, __float_as_uint(v));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(&gscal->wmax_bits, m);
}

// The cotangent as the contraction's T operand: tile (nt, ks) holds rows
// n = nt kN + r (accumulated axis) and columns k = ks kK + e (contracted
// axis) of G scaled by 2^s, hi (11 significant bits, exact in FP16) and lo =
// the rest, each part kN rows of 128 bytes with the 16-byte chunks of row r
// at chunk ^ (r & 7) (the tensor core's 128-byte swizzle).  Cells outside
// the grid are zero.  One thread per (tile, stage, row, chunk).
__global__ void k_tile_cotangent(const float* __restrict__ G, int nx, int ny, int axis,
                                 int n_tiles, int n_stages, const CallScalars* __restrict__ gscal,
                                 unsigned char* __restrict__ tiles) {
  const int64_t total = (int64_t)n_tiles * n_stages * kN * 8;
  const float scale = ldexpf(1.0f, g_exponent(gscal->wmax_bits));
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const int chunk = (int)(q & 7);
    const int r = (int)((q >> 3) % kN);
    const int64_t ts = q / (8 * kN);  // tile * n_stages + stage
    const int ks = (int)(ts % n_stages), nt = (int)(ts / n_stages);
    const int row = nt * kN + r;
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int e2 = 0; e2 < 4; ++e2) {
      float v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int col = ks * kK + chunk * 8 + 2 * e2 + h;
        // axis 0: rows are x cells i, columns y cells j; axis 1 the reverse
        const int i = axis == 0 ? row : col, j = axis == 0 ? col : row;
        v[h] = (i < nx && j < ny) ? G[(int64_t)j * nx + i] * scale : 0.0f;
      }
      const float h0 = __uint_as_float(__float_as_uint(v[0]) & 0xFFFFE000u);
      const float h1 = __uint_as_float(__float_as_uint(v[1]) & 0xFFFFE000u);
      const __half2 hh = __floats2half2_rn(h0, h1);
      const __half2 ll = __floats2half2_rn(v[0] - h0, v[1] - h1);
      hw[e2] = *reinterpret_cast<const uint32_t*>(&hh);
      lw[e2] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    unsigned char* base = tiles + ts * (2 * (int64_t)kTBytes) + (int64_t)r * kRowBytes +
                          ((chunk ^ (r & 7)) << 4);
    *reinterpret_cast<uint4*>(base) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(base + kTBytes) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

// One persistent CTA per SM; work item = a tile of 128 points, which the CTA
// takes through every N tile of the accumulated axis (n_tiles) and, for each,
// every K stage of the contracted axis (n_stages).  Roles: warp 0 issues the
// MMAs (one thread), warp 1 the stage bulk copies, warps 2-9 drain the
// accumulators into per-point sums (two warps per TMEM lane quadrant, 128
// columns each), warps 10-13 generate the points' operand rows.
__global__ void __launch_bounds__(kThreads, 1)
    k_adjoint_tc(const __grid_constant__ AdjTcArgs a, CallScalars* __restrict__ scal) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBars);
  uint64_t* full_e = bars;                // [kStages] producers -> MMA
  uint64_t* full_t = bars + kStages;      // [kStages] bulk copy -> MMA (transaction bytes)
  uint64_t* empty = bars + 2 * kStages;   // [kStages] MMA -> producers and loader
  uint64_t* accfull = bars + 3 * kStages; // [2] MMA -> epilogue
  uint64_t* accempty = accfull + 2;       // [2] epilogue -> MMA
  uint64_t* mmadone = accempty + 2;
  double* comb = reinterpret_cast<double*>(smem + kOffComb);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kOffMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_items = (int)((a.n + kM - 1) / kM);
  const int stages_per_item = a.n_tiles * a.n_stages;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_e[s], 4);
      mbar_init(&full_t[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], kEpiWarps);
    }
    mbar_init(mmadone, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // -------------------------------------------------------------- MMA issue
    if (lane == 0) {
      uint32_t g = 0, mc = 0;
      bool ok = true;
      const uint32_t sbase = smem_u32(smem);
      for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
        for (int nt = 0; ok && nt < a.n_tiles; ++nt, ++mc) {
          const uint32_t b = mc & 1u;
          if (!(ok = mbar_wait(&accempty[b], ((mc >> 1) & 1u) ^ 1u, abort_flag, scal, kRoleMma)))
            break;
          tc_fence_after();
          const uint32_t acc = tmem_base + b * 256u;
          for (int ks = 0; ks < a.n_stages; ++ks, ++g) {
            const uint32_t s = g % kStages, ph = (g / kStages) & 1u;
            if (!(ok = mbar_wait(&full_e[s], ph, abort_flag, scal, kRoleMma))) break;
            if (!(ok = mbar_wait(&full_t[s], ph, abort_flag, scal, kRoleMma))) break;
            tc_fence_after();
            const uint32_t st = sbase + s * kStageBytes;
            const uint64_t ehi = desc_swz(st, 2u, 1024u), elo = desc_swz(st + kEBytes, 2u, 1024u);
            const uint64_t thi = desc_swz(st + 2 * kEBytes, 2u, 1024u);
            const uint64_t tlo = desc_swz(st + 2 * kEBytes + kTBytes, 2u, 1024u);
#pragma unroll
            for (int k = 0; k < kK / 16; ++k) {
              const uint64_t dk = (uint64_t)(2 * k);
              mma_f16(acc, ehi + dk, thi + dk, kIdesc, (ks == 0 && k == 0) ? 0u : 1u);
              mma_f16(acc, ehi + dk, tlo + dk, kIdesc, 1u);
              mma_f16(acc, elo + dk, thi + dk, kIdesc, 1u);
            }
            mma_commit(&empty[s]);
          }
          if (!ok) break;
          mma_commit(&accfull[b]);
        }
      }
      mma_commit(mmadone);
      mbar_wait(mmadone, 0, abort_flag, scal, kRoleMma, /*honour_abort=*/false);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------- stage bulk copies of T
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
        for (int q = 0; ok && q < stages_per_item; ++q, ++g) {
          const uint32_t s = g % kStages;
          if (!(ok = mbar_wait(&empty[s], ((g / kStages) & 1u) ^ 1u, abort_flag, scal,
                               kRoleLoader)))
            break;
          // tile (nt, ks) = q, hi and lo contiguous: 64 KB
          mbar_arrive_expect_tx(&full_t[s], 2 * kTBytes);
          bulk_g2s(smem + s * kStageBytes + 2 * kEBytes, a.tiles + (int64_t)q * 2 * kTBytes,
                   2 * kTBytes, &full_t[s]);
        }
      }
    }
    __syncwarp();
  } else if (warp < kFirstProducerWarp) {
    // --------------------------------------------------------------- epilogue
    const int q = warp & 3, colh = (warp - kFirstEpiWarp) >> 2;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    // The eight warps meet at a named barrier once per item, so none of them
    // leaves the item loop early: after a failed wait they skip the work.
    uint32_t dc = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
      const int64_t p = (int64_t)it * kM + q * 32 + lane;
      const float4 P = a.pts[p];  // n_pad is a multiple of 512: in bounds
      // the point's coordinate along the accumulated axis (hi, lo)
      const float ph = a.axis == 0 ? P.x : P.z, pl = a.axis == 0 ? P.y : P.w;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int nt = 0; nt < a.n_tiles; ++nt, ++dc) {
        const uint32_t b = dc & 1u;
        if (ok) ok = mbar_wait(&accfull[b], (dc >> 1) & 1u, abort_flag, scal, kRoleEpilogue);
        if (!ok) continue;
        tc_fence_after();
        const int c0 = nt * kN + colh * 128;  // first cell of this thread's 128 columns
        // offsets u = (cell - point) in prepared units, recentred on cell c0
        const float2 g0 = a.acc_tab[min(c0, a.acc_cells - 1)];
        const float r = (ph - g0.x) + (pl - g0.y) - (float)(c0 - min(c0, a.acc_cells - 1)) * a.cs;
        float t0 = 0.f, t1 = 0.f, t2 = 0.f;
        const uint32_t acc = tmem_base + b * 256u + lane_off + colh * 128;
#pragma unroll 1
        for (int cb = 0; cb < 8; ++cb) {
          uint32_t d[16];
          tmem_ld16_async(acc + cb * 16, d);
          tmem_wait_ld();
          if (cb == 7) {  // every column is in registers: release the accumulator
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[b]);
          }
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float u = (float)(cb * 16 + e) * a.cs - r;
            const float f = ex2_neg(u * u) * __uint_as_float(d[e]);
            t0 += f;
            t1 = fmaf(u, f, t1);
            t2 = fmaf(u * u, f, t2);
          }
        }
        s0 += t0;
        s1 += t1;
        s2 += t2;
      }
      // the two column halves of each point, added in a fixed order
      if (colh == 1) {
        comb[(q * 32 + lane) * 3 + 0] = s0;
        comb[(q * 32 + lane) * 3 + 1] = s1;
        comb[(q * 32 + lane) * 3 + 2] = s2;
      }
      named_sync(kBarEpi, 32 * kEpiWarps);
      if (ok && colh == 0 && p < a.n) {
        s0 += comb[(q * 32 + lane) * 3 + 0];
        s1 += comb[(q * 32 + lane) * 3 + 1];
        s2 += comb[(q * 32 + lane) * 3 + 2];
        // D carries 2^15 (the generated operand) and 2^s (the cotangent)
        const double k = a.c * ldexp(1.0, -15 - g_exponent(a.gscal->wmax_bits));
        const double w = a.wts[p];
        if (a.axis == 0) {
          const double gw = k * s0;
          if (a.grad_w) a.grad_w[p] = (float)gw;
          a.grad_xy[2 * p] = (float)(k * w * a.k_xy * s1);
          a.hterm[p] = k * w * a.k_h * s2;
          a.lterm[p] = w * gw;
        } else {
          a.grad_xy[2 * p + 1] = (float)(k * w * a.k_xy * s1);
          a.hterm[p] += k * w * a.k_h * s2;
        }
      }
      named_sync(kBarEpi, 32 * kEpiWarps);  // comb is free for the next item
    }
    if (!ok && lane == 0) *abort_flag = 1;
  } else {
    // -------------------------------------------------- point operand rows
    const int t = threadIdx.x - kFirstProducerWarp * 32;  // row = point of the tile
    uint32_t g = 0;
    bool ok = true;
    for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
      const float4 P = a.pts[(int64_t)it * kM + t];
      // coordinate along the contracted axis (hi, lo)
      const float ph = a.axis == 0 ? P.z : P.x, pl = a.axis == 0 ? P.w : P.y;
      for (int q = 0; ok && q < stages_per_item; ++q, ++g) {
        const uint32_t s = g % kStages;
        if (!(ok = mbar_wait(&empty[s], ((g / kStages) & 1u) ^ 1u, abort_flag, scal,
                             kRoleProducer)))
          break;
        const int k0 = (q % a.n_stages) * kK;  // first contracted cell of the stage
        const float2 g0 = a.k_tab[min(k0, a.k_cells - 1)];
        // v_e = (cell k0 + e) - point, recentred on cell k0
        const float r = (ph - g0.x) + (pl - g0.y) - (float)(k0 - min(k0, a.k_cells - 1)) * a.cs;
        unsigned char* row = smem + s * kStageBytes + t * kRowBytes;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int e2 = 0; e2 < 4; ++e2) {
            const float v0 = (float)(c * 8 + 2 * e2) * a.cs - r;
            const float v1 = v0 + a.cs;
            const float2 y = fma2(make_float2(v0, v1), make_float2(v0, v1),
                                  make_float2(-15.f, -15.f));
            const float x0 = ex2_neg(y.x), x1 = ex2_neg(y.y);
            const float h0 = __uint_as_float(__float_as_uint(x0) & 0xFFFFE000u);
            const float h1 = __uint_as_float(__float_as_uint(x1) & 0xFFFFE000u);
            const float2 l = sub2(make_float2(x0, x1), make_float2(h0, h1));
            const __half2 hh = __floats2half2_rn(h0, h1);
            const __half2 ll = __floats2half2_rn(l.x, l.y);
            hw[e2] = *reinterpret_cast<const uint32_t*>(&hh);
            lw[e2] = *reinterpret_cast<const uint32_t*>(&ll);
          }
          const int off = (c ^ (t & 7)) << 4;
          *reinterpret_cast<uint4*>(row + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(row + kEBytes + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_e[s]);
      }
    }
    if (!ok && lane == 0) *abort_flag = 1;
  }

  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

int blocks_for_tc(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace

size_t adjoint_tc_workspace(int nx, int ny) {
  const size_t tx = (size_t)((nx + kN - 1) / kN) * ((ny + kK - 1) / kK);  // contraction 1
  const size_t ty = (size_t)((ny + kN - 1) / kN) * ((nx + kK - 1) / kK);  // contraction 2
  return 256 + (tx + ty) * 2 * kTBytes;
}

cudaError_t launch_adjoint_gauss_tc(const float4* pts, const float* wts, int64_t n, const float* G,
                                    const float2* gxt, const float2* gyt, int nx, int ny,
                                    double cell, double h, float* grad_xy, float* grad_w,
                                    double* hterm, double* lterm, void* ws, int max_ctas,
                                    cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_adjoint_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes);
  if (e != cudaSuccess) return e;
  CallScalars* gscal = static_cast<CallScalars*>(ws);
  unsigned char* tiles1 = static_cast<unsigned char*>(ws) + 256;
  const int nt1 = (nx + kN - 1) / kN, ns1 = (ny + kK - 1) / kK;
  const int nt2 = (ny + kN - 1) / kN, ns2 = (nx + kK - 1) / kK;
  unsigned char* tiles2 = tiles1 + (size_t)nt1 * ns1 * 2 * kTBytes;
  const int64_t cells = (int64_t)nx * ny;
  if ((e = cudaMemsetAsync(gscal, 0, sizeof(CallScalars), s)) != cudaSuccess) return e;
  k_abs_max<<<blocks_for_tc(cells), 256, 0, s>>>(G, cells, gscal);
  k_tile_cotangent<<<blocks_for_tc((int64_t)nt1 * ns1 * kN * 8), 256, 0, s>>>(
      G, nx, ny, 0, nt1, ns1, gscal, tiles1);
  k_tile_cotangent<<<blocks_for_tc((int64_t)nt2 * ns2 * kN * 8), 256, 0, s>>>(
      G, nx, ny, 1, nt2, ns2, gscal, tiles2);
  note_launches(3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const double sigma = 1.0 / (h * 1.17741002251547469101);  // Gaussian prepared units
  AdjTcArgs a = {};
  a.pts = pts;
  a.wts = wts;
  a.n = n;
  a.cs = (float)(cell * sigma);
  a.gscal = gscal;
  a.c = 1.0 / (2.0 * 3.14159265358979323846 * (double)n * h * h);
  a.k_xy = 1.17741002251547469101 / h;  // sqrt(2 ln 2) / h
  a.k_h = 1.38629436111989061883 / h;   // 2 ln 2 / h
  a.grad_xy = grad_xy;
  a.grad_w = grad_w;
  a.hterm = hterm;
  a.lterm = lterm;
  const int items = (int)((n + kM - 1) / kM);
  const int grid = std::max(1, std::min(items, max_ctas));
  for (int axis = 0; axis < 2; ++axis) {
    a.axis = axis;
    a.tiles = axis == 0 ? tiles1 : tiles2;
    a.acc_tab = axis == 0 ? gxt : gyt;
    a.k_tab = axis == 0 ? gyt : gxt;
    a.acc_cells = axis == 0 ? nx : ny;
    a.k_cells = axis == 0 ? ny : nx;
    a.n_tiles = axis == 0 ? nt1 : nt2;
    a.n_stages = axis == 0 ? ns1 : ns2;
    k_adjoint_tc<<<grid, kThreads, kSmemBytes, s>>>(a, gscal);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace kde
