// Path (b): the Gaussian density as a tensor-core contraction.
//
// The Gaussian row of Table 1 factorises, exp(-(s^2+t^2)/2) = exp(-s^2/2)
// exp(-t^2/2), so the direct sum of Eq. 7 over points is a matrix product
//     F[i,j] = c * sum_p A[i,p] B[j,p],
//     A[i,p] = 2^(15 - u_ip^2),   B[j,p] = (w_p / w_max) 2^(15 - v_jp^2),
// u, v = offsets in units of h sqrt(2 ln 2), c = w_max 2^-30 / (2 pi N h^2)
// (the 2^15 factors keep the FP16 operands in the normal range).
//
// One persistent CTA per SM computes 128 x BN output tiles (x index i along
// TMEM lanes, y index j along TMEM columns) for a range of points:
//   warp 0      one thread issues tcgen05.mma (FP16 x FP16 -> FP32 in TMEM)
//   warp 1      loads 64 points per stage and re-centres them on the tile
//   warps 2-5   epilogue: TMEM -> registers -> partial grid in global memory
//   warps 6..   producers: one warp per 32 operand rows; each thread writes
//               a share of the chunks of up to four rows, as FP16 (or hi + lo
//               FP16 pairs) in the swizzled K-major layout the MMA reads.
// A and B never exist in global memory.  The FP32 accumulator is drained
// every k_chunk points into the partial grid (double-buffered in TMEM) so the
// tensor core never adds more than k_chunk/16 products into one FP32 value.
// In split mode each operand is hi + lo with hi = fp16(v), lo = fp16(v - hi)
// and the MMA sums A_hi B_hi + A_hi B_lo + A_lo B_hi (about 22 bits).
#include <cuda_fp16.h>

#include <algorithm>

#include "kde_internal.cuh"
#include "tc_ptx.cuh"

namespace kde {
namespace {

using namespace tc;

constexpr int kBM = 128;    // grid x-cells per tile (TMEM lanes)
constexpr int kPS = 8;      // depth of the point-parameter ring
constexpr int kGroup = 4;   // stages the loader fetches at once

enum Role : int { kRoleMma = 1, kRoleLoader = 2, kRoleEpilogue = 3, kRoleProducer = 4 };

// KS points per pipeline stage: one operand row of KS FP16 values, stored
// K-major with the 128-byte (KS = 64) or 64-byte (KS = 32) swizzle.
template <int BN, bool SPLIT, int KS>
struct Cfg {
  static constexpr int kKS = KS;
  static constexpr int kRowBytes = 2 * KS;
  static constexpr int kChunks = KS / 8;                  // 16-byte chunks per row
  static constexpr int kSwzShift = KS == 64 ? 0 : 1;      // row bits that permute chunks
  static constexpr uint32_t kLayout = KS == 64 ? 2u : 4u; // 128B / 64B swizzle
  static constexpr uint32_t kSbo = 8 * kRowBytes;         // 8-row atom stride
  static constexpr int kHN = BN / 2;  // N of one accumulator half
  static constexpr int kABytes = kBM * kRowBytes;
  static constexpr int kBBytes = BN * kRowBytes;
  static constexpr int kParts = SPLIT ? 2 : 1;
  static constexpr int kStageBytes = kParts * (kABytes + kBBytes);
  static constexpr int kStages = (192 * 1024) / kStageBytes;
  static constexpr int kProducers = kBM + BN;  // operand rows (one producer thread per row)
  static constexpr int kProducerWarps = kProducers / 32;
  // rows per producer thread: a block of 32 * RPT rows is written by RPT
  // warps, each taking kChunks / RPT of the row's chunks
  static constexpr int kRowsPerThread =
      (kProducers % 128 == 0 && kChunks % 4 == 0) ? 4 : (kProducers % 64 == 0 && kChunks % 2 == 0) ? 2 : 1;
  static constexpr int kThreads = 32 * (6 + kProducerWarps);
  // TMEM: accumulator halves in columns [0, BN), running sums in [BN, 2 BN)
  static constexpr uint32_t kTmemCols = 2 * BN;
  static constexpr uint32_t kIdescHalf = idesc_f16_f32(kBM, kHN);
  static constexpr uint32_t kIdescFull = idesc_f16_f32(kBM, BN);
  // shared-memory map (offsets from a 1024-byte aligned base)
  static constexpr int kOffA = 0;                               // A_hi [, A_lo]
  static constexpr int kOffB = kParts * kABytes;                // B_hi [, B_lo]
  static constexpr int kOffParams = kStages * kStageBytes;      // float[kPS][4][kKS]
  static constexpr int kOffBars = kOffParams + kPS * 4 * kKS * 4;
  static constexpr int kNumBars = 2 * kStages + 2 * kPS + 4 + 1;
  static constexpr int kOffMisc = kOffBars + kNumBars * 8;      // tmem slot, abort flag
  static constexpr int kSmemBytes = kOffMisc + 64 + 1024;       // + alignment slack
  static_assert(kStages >= 2, "pipeline needs two stages");
  static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
};

struct Item {
  const TcInst* I;  // the instance the item belongs to
  int tm, tn, s;
  int64_t k_begin;
  int nst;  // stages of KS points
};

// Work item `it` of the whole launch: instance found by binary search on the
// table's item_begin, then (x tile, y tile, point split) within it.
__device__ __forceinline__ Item item_of(const TcInst* __restrict__ tab, int ninst, int it,
                                        int ks) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].item_begin <= it) lo = mid; else hi = mid - 1;
  }
  Item r;
  r.I = tab + lo;
  const int local = it - r.I->item_begin;
  r.tm = local % r.I->tiles_m;
  const int rest = local / r.I->tiles_m;
  r.tn = rest % r.I->tiles_n;
  r.s = rest / r.I->tiles_n;
  r.k_begin = (int64_t)r.s * r.I->per_split;
  int64_t k_end = r.k_begin + r.I->per_split;
  if (k_end > r.I->n_pad) k_end = r.I->n_pad;
  r.nst = k_end > r.k_begin ? (int)((k_end - r.k_begin) / ks) : 0;
  return r;
}

// Accumulator half h restarts every C stages, half 1 offset by C/2, so the
// two halves are never drained at the same time (except at an item's end)
// and the tensor core keeps working on one half while the other drains.
__device__ __forceinline__ bool chunk_starts(int h, int st, int C) {
  if (st == 0) return true;
  const int off = h ? C / 2 : 0;
  return st >= off && (st - off) % C == 0;
}
__device__ __forceinline__ int next_boundary(int h, int cs, int C) {
  if (h == 0) return (cs / C + 1) * C;
  return cs < C / 2 ? C / 2 : cs + C;
}

template <int BN, bool SPLIT, int KS>
__global__ void __launch_bounds__(Cfg<BN, SPLIT, KS>::kThreads, 1)
    k_tc(const TcInst* __restrict__ tab, int ninst, int n_items, CallScalars* __restrict__ scal) {
  using C = Cfg<BN, SPLIT, KS>;
  constexpr int HN = C::kHN;
  constexpr int kKS = KS;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // align in the shared window by pointer arithmetic on the shared array, so
  // the compiler keeps the shared address space (LDS/STS, not generic LD/ST)
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float* params = reinterpret_cast<float*>(smem + C::kOffParams);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kOffBars);
  uint64_t* full = bars;                       // [kStages] producers -> MMA
  uint64_t* empty = bars + C::kStages;         // [kStages] MMA -> producers
  uint64_t* pfull = bars + 2 * C::kStages;     // [kPS] loader -> producers
  uint64_t* pempty = pfull + kPS;              // [kPS] producers -> loader
  uint64_t* accfull = pempty + kPS;            // [2] MMA -> epilogue, per half
  uint64_t* accempty = accfull + 2;            // [2] epilogue -> MMA, per half
  uint64_t* mmadone = accempty + 2;            // [1] final drain of the MMA pipe
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kOffMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kOffMisc + 4);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], C::kProducerWarps);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < kPS; ++s) {
      mbar_init(&pfull[s], 32);
      mbar_init(&pempty[s], C::kProducerWarps);
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(&accfull[h], 1);
      mbar_init(&accempty[h], 128);
    }
    mbar_init(mmadone, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(tmem_slot, C::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      uint32_t g = 0;
      uint32_t mc[2] = {0, 0};
      bool ok = true;
      const uint32_t smem_base = smem_u32(smem);
      for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
        const Item itm = item_of(tab, ninst, it, kKS);
        const int CS = itm.I->chunk_stages;
        for (int st = 0; ok && st < itm.nst; ++st, ++g) {
          const uint32_t s = g % C::kStages;
          if (!(ok = mbar_wait(&full[s], (g / C::kStages) & 1, abort_flag, scal, kRoleMma))) break;
          tc_fence_after();
          const uint32_t a0 = smem_base + s * C::kStageBytes + C::kOffA;
          const uint32_t b0 = smem_base + s * C::kStageBytes + C::kOffB;
          const uint64_t ahi = desc_swz(a0, C::kLayout, C::kSbo);
          const uint64_t alo = desc_swz(a0 + C::kABytes, C::kLayout, C::kSbo);
          const bool f0 = chunk_starts(0, st, CS), f1 = chunk_starts(1, st, CS);
          if (f0 && f1) {
            // first stage of an item: both halves start fresh, one N = BN MMA
            for (int h = 0; ok && h < 2; ++h) {
              if (!(ok = mbar_wait(&accempty[h], (mc[h] & 1) ^ 1, abort_flag, scal, kRoleMma))) break;
              ++mc[h];
            }
            if (!ok) break;
            tc_fence_after();
          }
          if (f0 != f1) {
            // one half restarts: issue the other half's whole stage first so the
            // tensor core works while the epilogue drains the restarting half
#pragma unroll
            for (int o = 0; o < 2; ++o) {
              const int h = (o == 0) ? (f0 ? 1 : 0) : (f0 ? 0 : 1);
              const bool fresh = o == 1;
              if (fresh) {
                if (!(ok = mbar_wait(&accempty[h], (mc[h] & 1) ^ 1, abort_flag, scal, kRoleMma))) break;
                ++mc[h];
                tc_fence_after();
              }
              const uint32_t d_tmem = tmem_base + h * HN;
              const uint32_t bh = b0 + h * HN * C::kRowBytes;  // rows [h HN, (h+1) HN) of B
              const uint64_t bhi = desc_swz(bh, C::kLayout, C::kSbo);
              const uint64_t blo = desc_swz(bh + C::kBBytes, C::kLayout, C::kSbo);
#pragma unroll
              for (int k = 0; k < kKS / 16; ++k) {
                const uint32_t acc = (fresh && k == 0) ? 0u : 1u;
                const uint64_t dk = (uint64_t)(2 * k);  // +32 bytes in the start-address field
                mma_f16(d_tmem, ahi + dk, bhi + dk, C::kIdescHalf, acc);
                if (SPLIT) {
                  mma_f16(d_tmem, ahi + dk, blo + dk, C::kIdescHalf, 1u);
                  mma_f16(d_tmem, alo + dk, bhi + dk, C::kIdescHalf, 1u);
                }
              }
            }
          } else {
            // both halves continue (or both start): the halves are adjacent TMEM
            // columns, so one N = BN MMA covers them
            const uint64_t bhi = desc_swz(b0, C::kLayout, C::kSbo);
            const uint64_t blo = desc_swz(b0 + C::kBBytes, C::kLayout, C::kSbo);
#pragma unroll
            for (int k = 0; k < kKS / 16; ++k) {
              const uint32_t acc = (f0 && k == 0) ? 0u : 1u;
              const uint64_t dk = (uint64_t)(2 * k);
              mma_f16(tmem_base, ahi + dk, bhi + dk, C::kIdescFull, acc);
              if (SPLIT) {
                mma_f16(tmem_base, ahi + dk, blo + dk, C::kIdescFull, 1u);
                mma_f16(tmem_base, alo + dk, bhi + dk, C::kIdescFull, 1u);
              }
            }
          }
          if (!ok) break;
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (st + 1 == itm.nst || chunk_starts(h, st + 1, CS)) mma_commit(&accfull[h]);
          if (!ok) break;
          mma_commit(&empty[s]);
        }
      }
      // every issued MMA must finish before TMEM is released
      mma_commit(mmadone);
      mbar_wait(mmadone, 0, abort_flag, scal, kRoleMma, /*honour_abort=*/false);
    }
    __syncwarp();
  } else if (warp == 1) {
    // --------------------------------------------------------- point loader
    uint32_t g = 0;
    bool ok = true;
    for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
      const Item itm = item_of(tab, ninst, it, kKS);
      const TcInst& I = *itm.I;
      const float wmax = __uint_as_float(I.scal->wmax_bits);
      const float inv_wmax = wmax > 0.f ? 1.0f / wmax : 1.0f;
      const float2 cx = I.gxt[min(itm.tm * kBM + kBM / 2, I.nx - 1)];
      const float2 cy = I.gyt[min(itm.tn * BN + BN / 2, I.ny - 1)];
      const float4* __restrict__ pts = I.pts;
      const float* __restrict__ wts = I.wts;
      for (int st = 0; ok && st < itm.nst; st += kGroup) {
        const int ng = min(kGroup, itm.nst - st);
        constexpr int kPer = kKS / 32;  // points per lane per stage
        float4 P[kGroup][kPer];
        float W[kGroup][kPer];
#pragma unroll
        for (int u = 0; u < kGroup; ++u)
#pragma unroll
          for (int hh = 0; hh < kPer; ++hh)
            if (u < ng) {
              const int64_t p = itm.k_begin + (int64_t)(st + u) * kKS + lane + 32 * hh;
              P[u][hh] = __ldg(pts + p);
              W[u][hh] = __ldg(wts + p);
            }
#pragma unroll
        for (int u = 0; u < kGroup; ++u) {
          if (u >= ng) break;
          const uint32_t ps = g % kPS;
          if (!(ok = mbar_wait(&pempty[ps], ((g / kPS) & 1) ^ 1, abort_flag, scal, kRoleLoader)))
            break;
          float* prm = params + ps * 4 * kKS;
#pragma unroll
          for (int hh = 0; hh < kPer; ++hh) {
            const int e = lane + 32 * hh;
            const float4 q = P[u][hh];
            prm[e] = (q.x - cx.x) + (q.y - cx.y);
            prm[kKS + e] = (q.z - cy.x) + (q.w - cy.y);
            const float w = W[u][hh];
            // |B| = (|w| / w_max) 2^(15 - v^2) = 2^(cb - v^2); w = 0 gives cb = -inf,
            // B = 0; the sign of w is kept as a sign bit to apply to B
            prm[2 * kKS + e] = w != 0.f ? 15.0f + log2f(fabsf(w) * inv_wmax) : -INFINITY;
            reinterpret_cast<uint32_t*>(prm)[3 * kKS + e] = w < 0.f ? 0x80000000u : 0u;
          }
          mbar_arrive(&pfull[ps]);
          ++g;
        }
      }
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    uint32_t dc0 = 0, dc1 = 0;
    bool ok = true;
    for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
      const Item itm = item_of(tab, ninst, it, kKS);
      const TcInst& I = *itm.I;
      const int nx = I.nx, ny = I.ny, CS = I.chunk_stages;
      const float wmax = __uint_as_float(I.scal->wmax_bits);
      const float scale = I.base_scale * (wmax > 0.f ? wmax : 1.0f);
      const int i = itm.tm * kBM + q * 32 + lane;
      const int j0 = itm.tn * BN;
      float* slot = I.part + (int64_t)itm.s * nx * ny;
      if (itm.nst == 0) {
        if (i < nx)
          for (int c = 0; c < BN && j0 + c < ny; ++c) slot[(int64_t)(j0 + c) * nx + i] = 0.f;
        continue;
      }
      int cs0 = 0, cs1 = 0;
      bool done0 = false, done1 = false, first0 = true, first1 = true;
      while (ok && !(done0 && done1)) {
        // next drain in commit order: earliest chunk end, half 0 first on ties
        const int e0 = done0 ? 0x7fffffff : min(next_boundary(0, cs0, CS), itm.nst) - 1;
        const int e1 = done1 ? 0x7fffffff : min(next_boundary(1, cs1, CS), itm.nst) - 1;
        const int h = e0 <= e1 ? 0 : 1;
        const int eh = h ? e1 : e0;
        const bool first = h ? first1 : first0;
        const bool final = eh == itm.nst - 1;
        const uint32_t parity = (h ? dc1 : dc0) & 1;
        if (!(ok = mbar_wait(&accfull[h], parity, abort_flag, scal, kRoleEpilogue))) break;
        if (h) ++dc1; else ++dc0;
        tc_fence_after();
        const uint32_t acc_col = tmem_base + lane_off + h * HN;
        const uint32_t run_col = tmem_base + lane_off + BN + h * HN;
        // 32-column slices, both loads in flight together; the half is
        // released to the MMA as soon as its last slice is in registers
#pragma unroll 1
        for (int cb = 0; cb < HN / 32; ++cb) {
          uint32_t ra[32], rr[32];
          tmem_ld32_async(acc_col + cb * 32, ra);
          if (!first) tmem_ld32_async(run_col + cb * 32, rr);
          tmem_wait_ld();
          if (cb == HN / 32 - 1) {
            tc_fence_before();
            mbar_arrive(&accempty[h]);
          }
          float a[32];
#pragma unroll
          for (int c = 0; c < 32; ++c) a[c] = __uint_as_float(ra[c]);
          if (!first) {
#pragma unroll
            for (int c = 0; c < 32; ++c) a[c] += __uint_as_float(rr[c]);
          }
          if (final) {
            if (i < nx) {
#pragma unroll
              for (int c = 0; c < 32; ++c) {
                const int j = j0 + h * HN + cb * 32 + c;
                if (j < ny) slot[(int64_t)j * nx + i] = a[c] * scale;
              }
            }
          } else {
            tmem_st32(run_col + cb * 32, a);
          }
        }
        // the running sum's stores complete before this thread's next loads
        if (!final) tmem_wait_st();
        if (h) {
          if (final) done1 = true; else { cs1 = eh + 1; first1 = false; }
        } else {
          if (final) done0 = true; else { cs0 = eh + 1; first0 = false; }
        }
      }
    }
  } else {
    // ------------------------------------------------------------ producers
    // Rows come in blocks of 32 * RPT (A rows first, then B rows); the RPT
    // warps of a block split its chunks, and lane l writes rows l + 32 k.  A
    // thread reuses each broadcast load of a chunk's point parameters for
    // its RPT rows, which keeps these loads a small share of the shared-
    // memory bandwidth the operand stores and the tensor core's reads take.
    constexpr int RPT = C::kRowsPerThread, CPT = C::kChunks / RPT;
    const int pw = warp - 6;
    const int rowblock = pw / RPT, cset = pw % RPT;
    const int row_first = rowblock * 32 * RPT;  // in A rows, then B rows
    const bool isA = row_first < kBM;           // warp-uniform
    const int r0 = (isA ? row_first : row_first - kBM) + lane;
    const int lo_off = isA ? C::kABytes : C::kBBytes;
    uint32_t g = 0;
    bool ok = true;
    for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
      const Item itm = item_of(tab, ninst, it, kKS);
      const TcInst& I = *itm.I;
      const bool signs = !isA && I.scal->negw != 0;
      float gv[RPT];
      {
        const float2* tab_g = isA ? I.gxt : I.gyt;
        const int base = isA ? itm.tm * kBM : itm.tn * BN;
        const int half = isA ? kBM / 2 : BN / 2;
        const int n_g = isA ? I.nx : I.ny;
        const float2 c = tab_g[min(base + half, n_g - 1)];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          const float2 v = tab_g[min(base + r0 + 32 * k, n_g - 1)];
          gv[k] = (v.x - c.x) + (v.y - c.y);
        }
      }
      for (int st = 0; st < itm.nst; ++st, ++g) {
        const uint32_t s = g % C::kStages, ps = g % kPS;
        if (!(ok = mbar_wait(&pfull[ps], (g / kPS) & 1, abort_flag, scal, kRoleProducer))) break;
        if (!(ok = mbar_wait(&empty[s], ((g / C::kStages) & 1) ^ 1, abort_flag, scal, kRoleProducer)))
          break;
        unsigned char* row0 =
            smem + s * C::kStageBytes + (isA ? C::kOffA : C::kOffB) + r0 * C::kRowBytes;
        const float4* crd = reinterpret_cast<const float4*>(params + ps * 4 * kKS + (isA ? 0 : kKS));
        const float4* cbv = reinterpret_cast<const float4*>(params + ps * 4 * kKS + 2 * kKS);
        const uint4* sgn = reinterpret_cast<const uint4*>(params + ps * 4 * kKS + 3 * kKS);
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
          const int c = cset * CPT + cc;
          const float4 p0 = crd[2 * c], p1 = crd[2 * c + 1];
          float4 c0 = make_float4(15.f, 15.f, 15.f, 15.f), c1 = c0;
          if (!isA) {
            c0 = cbv[2 * c];
            c1 = cbv[2 * c + 1];
          }
          const float pc[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
          const float ce[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
          uint32_t sb[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
          if (signs) {  // negative weights: B takes the weight's sign
            const uint4 s0 = sgn[2 * c], s1 = sgn[2 * c + 1];
            sb[0] = s0.x; sb[1] = s0.y; sb[2] = s0.z; sb[3] = s0.w;
            sb[4] = s1.x; sb[5] = s1.y; sb[6] = s1.z; sb[7] = s1.w;
          }
          // rows lane + 32 k share the swizzle phase of row lane
          const int off = (c ^ ((lane >> C::kSwzShift) & (C::kChunks - 1))) << 4;
#pragma unroll
          for (int k = 0; k < RPT; ++k) {
            float v[8];
#pragma unroll
            for (int e2 = 0; e2 < 8; ++e2) {
              const float u = gv[k] - pc[e2];
              asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(v[e2]) : "f"(fmaf(-u, u, ce[e2])));
              if (signs) v[e2] = __uint_as_float(__float_as_uint(v[e2]) ^ sb[e2]);
            }
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
              if (SPLIT) {
                // hi keeps 11 significant bits (exact in FP16), lo = v - hi exactly
                const float h0 = __uint_as_float(__float_as_uint(v[2 * e2]) & 0xFFFFE000u);
                const float h1 = __uint_as_float(__float_as_uint(v[2 * e2 + 1]) & 0xFFFFE000u);
                const __half2 hh = __floats2half2_rn(h0, h1);
                const __half2 ll = __floats2half2_rn(v[2 * e2] - h0, v[2 * e2 + 1] - h1);
                hw[e2] = *reinterpret_cast<const uint32_t*>(&hh);
                lw[e2] = *reinterpret_cast<const uint32_t*>(&ll);
              } else {
                const __half2 hh = __floats2half2_rn(v[2 * e2], v[2 * e2 + 1]);
                hw[e2] = *reinterpret_cast<const uint32_t*>(&hh);
              }
            }
            unsigned char* row = row0 + 32 * k * C::kRowBytes;
            *reinterpret_cast<uint4*>(row + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            if (SPLIT)
              *reinterpret_cast<uint4*>(row + lo_off + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
        // each writer makes its stores visible to the tensor core's proxy; the
        // warp then signals once (__syncwarp orders the lanes' writes first)
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&full[s]);
          mbar_arrive(&pempty[ps]);
        }
      }
    }
  }

  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, C::kTmemCols);
  }
}

template <int BN, bool SPLIT, int KS>
cudaError_t launch_cfg(const TcPlan& p, const TcInst* tab, int ninst, int n_items,
                       CallScalars* err, cudaStream_t s) {
  using C = Cfg<BN, SPLIT, KS>;
  cudaError_t e = cudaFuncSetAttribute(k_tc<BN, SPLIT, KS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
  if (e != cudaSuccess) return e;
  const int grid = std::min(n_items, p.ctas);
  k_tc<BN, SPLIT, KS><<<grid, C::kThreads, C::kSmemBytes, s>>>(tab, ninst, n_items, err);
  note_launches(1);
  return cudaGetLastError();
}

template <int BN, bool SPLIT>
cudaError_t launch_ks(const TcPlan& p, const TcInst* tab, int ninst, int n_items,
                      CallScalars* err, cudaStream_t s) {
  if (p.stage_points == 32) return launch_cfg<BN, SPLIT, 32>(p, tab, ninst, n_items, err, s);
  if (p.stage_points == 64) return launch_cfg<BN, SPLIT, 64>(p, tab, ninst, n_items, err, s);
  return cudaErrorInvalidValue;
}

// A wait on an mbarrier that nothing signals, bounded by limit_ns: exercises
// the timeout path of the pipelines' waits (records kErrTimeout, returns).
__global__ void k_wait_timeout(CallScalars* scal, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    mbar_init_fence();
  }
  __syncthreads();
  mbar_wait(&bar, 0, &abort_flag, scal, 99, /*honour_abort=*/true, limit_ns);
}

}  // namespace

cudaError_t launch_wait_timeout(CallScalars* scal, uint64_t limit_ns, cudaStream_t s) {
  k_wait_timeout<<<1, 32, 0, s>>>(scal, limit_ns);
  note_launches(1);
  return cudaGetLastError();
}

size_t tc_smem_bytes(const TcPlan& p) {
  if (p.tile_n == 256)
    return p.split16 ? Cfg<256, true, 64>::kSmemBytes : Cfg<256, false, 64>::kSmemBytes;
  return p.split16 ? Cfg<128, true, 64>::kSmemBytes : Cfg<128, false, 64>::kSmemBytes;
}

cudaError_t launch_tc(const TcPlan& plan, const TcInst* tab, int ninst, int n_items,
                      CallScalars* err, cudaStream_t s) {
  if (ninst < 1 || n_items < 1 || plan.ctas < 1) return cudaErrorInvalidValue;
  if (plan.tile_n == 256)
    return plan.split16 ? launch_ks<256, true>(plan, tab, ninst, n_items, err, s)
                        : launch_ks<256, false>(plan, tab, ninst, n_items, err, s);
  if (plan.tile_n == 128)
    return plan.split16 ? launch_ks<128, true>(plan, tab, ninst, n_items, err, s)
                        : launch_ks<128, false>(plan, tab, ninst, n_items, err, s);
  return cudaErrorInvalidValue;
}

}  // namespace kde
