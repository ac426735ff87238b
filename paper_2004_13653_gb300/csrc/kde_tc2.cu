// Path (b) on CTA pairs: the Gaussian density as a tcgen05 contraction with
// cta_group::2, one 256 x 256 output tile per pair of CTAs (a cluster of 2).
//
// The factorisation is the one of kde_tc.cu (A[i,p] = 2^(15-u^2),
// B[j,p] = (w_p/w_max) 2^(15-v^2), F = c A B^T).  In a pair, each CTA
// generates only its own 128 rows of A (x cells) and 128 rows of B (y cells)
// per stage, and the leader CTA issues M = 256 MMAs that read A and B from
// both CTAs' shared memory and write each CTA's 128 rows of D into its own
// TMEM.  Per output pair this generates a third fewer exponentials than one
// CTA with a 128 x 256 tile, and each SM's shared memory serves half of B.
//
// Roles in each CTA: warp 0 (leader CTA, one thread) issues the MMAs; warp 1
// loads and re-centres points; warps 2-9 drain this CTA's TMEM (two warps per
// lane quadrant, 128 columns each); warps 10-17 generate operand rows.
// Producers of both CTAs signal the leader's stage barriers; MMA completion is
// multicast to both CTAs; both CTAs' epilogues signal the leader when the
// accumulator is free again.
//
// Accumulator: one N = 256 accumulator in TMEM columns [0, 256) (column j is
// y cell j of the tile: CTA 0 supplies B rows 0-127, CTA 1 rows 128-255),
// drained every chunk into a running sum in columns [256, 512) while the
// tensor core waits.  N = 256 MMAs keep each SM's operand reads at 8 KB per
// 128 cycles.
#include <cuda_fp16.h>

#include <algorithm>

#include "kde_internal.cuh"
#include "tc_ptx.cuh"

namespace kde {
namespace {

using namespace tc;

constexpr int kRows = 128;  // A rows and B rows each CTA of the pair generates
constexpr int kKS = 64;     // points per stage
constexpr int kPS = 8;      // point-parameter ring depth
constexpr int kGroup = 4;   // stages the loader fetches at once

enum Role : int { kRoleMma = 11, kRoleLoader = 12, kRoleEpilogue = 13, kRoleProducer = 14 };

template <bool SPLIT, bool SPARSE>
struct PairCfg {
  static constexpr int kRowBytes = 2 * kKS;
  static constexpr int kABytes = kRows * kRowBytes;
  static constexpr int kBBytes = kRows * kRowBytes;
  static constexpr int kParts = SPLIT ? 2 : 1;
  static constexpr int kStageBytes = kParts * (kABytes + kBBytes);
  static constexpr int kStages = (192 * 1024) / kStageBytes;
  // producer threads per operand row, each taking 64 / kPerRow points of a
  // stage (one: 576 threads, which leaves the epilogue the registers for
  // 32-column drain slices)
  static constexpr int kPerRow = 1;
  static constexpr int kProducers = 2 * kRows * kPerRow;
  static constexpr int kProducerWarps = kProducers / 32;
  static constexpr int kEpiWarps = 8;
  static constexpr int kFirstProducerWarp = 2 + kEpiWarps;
  static constexpr int kThreads = 32 * (kFirstProducerWarp + kProducerWarps);
  static constexpr uint32_t kTmemCols = 512;
  static constexpr uint32_t kIdesc = idesc_f16_f32(256, 256);
  static constexpr int kOffA = 0;
  static constexpr int kOffB = kParts * kABytes;
  static constexpr int kOffParams = kStages * kStageBytes;
  static constexpr int kOffBars = kOffParams + kPS * 3 * kKS * 4;
  static constexpr int kNumBars = 2 * kStages + 2 * kPS + 2 + 1;
  static constexpr int kOffMisc = kOffBars + kNumBars * 8;
  static constexpr int kSmemBytes = kOffMisc + 64 + 1024;
  static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
};

struct Item {
  const TcInst* I;
  int tm, tn, s;
  int64_t k_begin;  // dense: first point; sparse: first position in the tile's runs
  int nst;
  int64_t slot;     // sparse: the piece's partial tile
  int64_t vend;     // sparse: end position in the tile's runs
};

__device__ __forceinline__ Item pair_item(const TcInst* __restrict__ tab, int ninst, int it) {
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
  r.nst = k_end > r.k_begin ? (int)((k_end - r.k_begin) / kKS) : 0;
  r.slot = 0;
  r.vend = k_end;
  return r;
}

// Block-sparse work item at schedule position `pos`: full pieces first (tile
// by tile), then the tiles' short last pieces, longest first.  Returns the
// tile, the piece's range of positions in the concatenation of the tile's
// bin-row runs, and the piece id (its partial slot).
__device__ __forceinline__ Item sparse_item(const TcInst* __restrict__ tab, int ninst,
                                            const SparseCtl& sp, int pos) {
  const int n_full = (int)__ldg(sp.full_begin + sp.tiles_total);
  int t, p;
  if (pos < n_full) {
    int lo = 0, hi = sp.tiles_total - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((int)__ldg(sp.full_begin + mid) <= pos) lo = mid; else hi = mid - 1;
    }
    t = lo;
    p = pos - (int)__ldg(sp.full_begin + t);
  } else {
    t = (int)__ldg(sp.tail_tile + (pos - n_full));
    p = (int)(__ldg(sp.piece_begin + t + 1) - __ldg(sp.piece_begin + t)) - 1;
  }
  const int it = (int)__ldg(sp.piece_begin + t) + p;
  int a = 0, b = ninst - 1;
  while (a < b) {
    const int mid = (a + b + 1) >> 1;
    if (tab[mid].tile_begin <= t) a = mid; else b = mid - 1;
  }
  Item r;
  r.I = tab + a;
  const int local = t - r.I->tile_begin;
  r.tm = local % r.I->tiles_m;
  r.tn = local / r.I->tiles_m;
  r.s = 0;
  r.k_begin = (int64_t)p * sp.piece_len;
  const int64_t total = __ldg(sp.tile_total + t);
  r.vend = min(total, r.k_begin + (int64_t)sp.piece_len);
  r.nst = r.vend > r.k_begin ? (int)((r.vend - r.k_begin + kKS - 1) / kKS) : 0;
  r.slot = it;
  return r;
}

template <bool SPARSE>
__device__ __forceinline__ Item get_item(const TcInst* __restrict__ tab, int ninst,
                                         const SparseCtl& sp, int it) {
  if (SPARSE) return sparse_item(tab, ninst, sp, it);
  return pair_item(tab, ninst, it);
}

// Schedule position of CTA pair c (of nc) in round r.  Dense items go round
// robin; block-sparse items are listed longest first and are dealt in snake
// order (forward in even rounds, backward in odd ones), so that the pairs'
// sums of piece lengths come out nearly equal.  Every role of both CTAs
// walks the same sequence.
template <bool SPARSE>
__device__ __forceinline__ int sched_pos(int r, int c, int nc) {
  return r * nc + ((SPARSE && (r & 1)) ? nc - 1 - c : c);
}

template <bool SPLIT, bool SPARSE>
__global__ void __launch_bounds__(PairCfg<SPLIT, SPARSE>::kThreads, 1)
    k_tc_pair(const TcInst* __restrict__ tab, int ninst, int n_items_arg,
              const __grid_constant__ SparseCtl sp, CallScalars* __restrict__ scal) {
  using C = PairCfg<SPLIT, SPARSE>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float* params = reinterpret_cast<float*>(smem + C::kOffParams);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kOffBars);
  uint64_t* full = bars;                    // [kStages] producers (both CTAs) -> leader MMA
  uint64_t* empty = bars + C::kStages;      // [kStages] MMA -> producers (multicast)
  uint64_t* pfull = bars + 2 * C::kStages;  // [kPS] loader -> producers
  uint64_t* pempty = pfull + kPS;           // [kPS] producers -> loader
  uint64_t* accfull = pempty + kPS;         // [1] MMA -> epilogues (multicast)
  uint64_t* accempty = accfull + 1;         // [1] epilogues (both CTAs) -> leader MMA
  uint64_t* mmadone = accempty + 1;         // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kOffMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kOffMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int n_items = n_items_arg;
  if (SPARSE) {  // the work list was built on the device by the preceding launches
    const int listed = (int)__ldg(sp.piece_begin + sp.tiles_total);
    // a list longer than the partial buffer is an error: no piece is computed
    n_items = listed > sp.max_pieces ? 0 : listed;
    if (listed > sp.max_pieces && blockIdx.x == 0 && threadIdx.x == 0)
      atomicOr(&scal->err, kErrBadArg);
  }
  const uint32_t rank = cluster_rank();
  const uint32_t peer = rank ^ 1u;
  const int cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;
  auto propagate_abort = [&]() {
    store_cluster_u32(map_to_rank(smem_u32((const void*)abort_flag), peer), 1u);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 2 * C::kProducerWarps);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < kPS; ++s) {
      mbar_init(&pfull[s], 32);
      mbar_init(&pempty[s], C::kProducerWarps);
    }
    mbar_init(accfull, 1);
    mbar_init(accempty, 2 * C::kEpiWarps);
    mbar_init(mmadone, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc_pair(tmem_slot, C::kTmemCols);
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers initialised, TMEM allocated in both
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------- MMA issue (leader only)
    if (rank == 0 && lane == 0) {
      uint32_t g = 0, mc = 0;
      bool ok = true;
      const uint32_t smem_base = smem_u32(smem);
      for (int rd = 0, it = sched_pos<SPARSE>(0, cluster, n_clusters); ok && it < n_items;
           it = sched_pos<SPARSE>(++rd, cluster, n_clusters)) {
        const Item itm = get_item<SPARSE>(tab, ninst, sp, it);
        const int CS = itm.I->chunk_stages;
        for (int st = 0; ok && st < itm.nst; ++st, ++g) {
          const bool fresh = st % CS == 0;
          if (fresh) {  // the epilogues of both CTAs have drained the accumulator
            if (!(ok = mbar_wait_cluster(accempty, (mc & 1) ^ 1, abort_flag, scal, kRoleMma))) break;
            ++mc;
            tc_fence_after();
          }
          const uint32_t s = g % C::kStages;
          if (!(ok = mbar_wait_cluster(&full[s], (g / C::kStages) & 1, abort_flag, scal, kRoleMma)))
            break;
          tc_fence_after();
          const uint32_t a0 = smem_base + s * C::kStageBytes + C::kOffA;
          const uint32_t b0 = smem_base + s * C::kStageBytes + C::kOffB;
          const uint64_t ahi = desc_swz(a0, 2u, 1024u), alo = desc_swz(a0 + C::kABytes, 2u, 1024u);
          const uint64_t bhi = desc_swz(b0, 2u, 1024u), blo = desc_swz(b0 + C::kBBytes, 2u, 1024u);
#pragma unroll
          for (int k = 0; k < kKS / 16; ++k) {
            const uint32_t acc = (fresh && k == 0) ? 0u : 1u;
            const uint64_t dk = (uint64_t)(2 * k);
            mma_f16_pair(tmem_base, ahi + dk, bhi + dk, C::kIdesc, acc);
            if (SPLIT) {
              mma_f16_pair(tmem_base, ahi + dk, blo + dk, C::kIdesc, 1u);
              mma_f16_pair(tmem_base, alo + dk, bhi + dk, C::kIdesc, 1u);
            }
          }
          mma_commit_pair(&empty[s]);
          if (st + 1 == itm.nst || (st + 1) % CS == 0) mma_commit_pair(accfull);
        }
      }
      if (!ok) propagate_abort();
      mma_commit_pair(mmadone);
      mbar_wait(mmadone, 0, abort_flag, scal, kRoleMma, /*honour_abort=*/false);
    }
    __syncwarp();
  } else if (warp == 1) {
    // --------------------------------------------------------- point loader
    uint32_t g = 0;
    bool ok = true, negative = false;
    for (int rd = 0, it = sched_pos<SPARSE>(0, cluster, n_clusters); ok && it < n_items;
         it = sched_pos<SPARSE>(++rd, cluster, n_clusters)) {
      const Item itm = get_item<SPARSE>(tab, ninst, sp, it);
      const TcInst& I = *itm.I;
      const float wmax = __uint_as_float(I.scal->wmax_bits);
      const float inv_wmax = wmax > 0.f ? 1.0f / wmax : 1.0f;
      const float2 cx = I.gxt[min(itm.tm * 256 + (int)rank * kRows + kRows / 2, I.nx - 1)];
      const float2 cy = I.gyt[min(itm.tn * 256 + (int)rank * kRows + kRows / 2, I.ny - 1)];
      RunCursor cur;
      if (SPARSE)  // items exist only for tiles whose range holds points
        cur.init(I.start, I.bin_begin, I.nbx,
                 tile_bins(I.cs, I.range_reach, I.inv_binw, I.nbx, I.nby, itm.tm, itm.tn));
      for (int st = 0; ok && st < itm.nst; st += kGroup) {
        const int ng = min(kGroup, itm.nst - st);
        float4 P[kGroup][2];
        float W[kGroup][2];
#pragma unroll
        for (int u = 0; u < kGroup; ++u)
#pragma unroll
          for (int hh = 0; hh < 2; ++hh)
            if (u < ng) {
              const int64_t v = itm.k_begin + (int64_t)(st + u) * kKS + lane + 32 * hh;
              if (!SPARSE) {
                P[u][hh] = __ldg(I.pts + v);
                W[u][hh] = __ldg(I.wts + v);
              } else if (v < itm.vend) {
                const int64_t p = cur.map(v);
                P[u][hh] = __ldg(I.pts + p);
                W[u][hh] = __ldg(I.wts + p);
              } else {  // past the piece: a zero-weight point (B = 0)
                P[u][hh] = make_float4(0.f, 0.f, 0.f, 0.f);
                W[u][hh] = 0.f;
              }
            }
#pragma unroll
        for (int u = 0; u < kGroup; ++u) {
          if (u >= ng) break;
          const uint32_t ps = g % kPS;
          if (!(ok = mbar_wait(&pempty[ps], ((g / kPS) & 1) ^ 1, abort_flag, scal, kRoleLoader)))
            break;
          float* prm = params + ps * 3 * kKS;
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int e = lane + 32 * hh;
            const float4 q = P[u][hh];
            prm[e] = (q.x - cx.x) + (q.y - cx.y);
            prm[kKS + e] = (q.z - cy.x) + (q.w - cy.y);
            const float w = W[u][hh];
            negative |= w < 0.f;
            prm[2 * kKS + e] = w > 0.f ? 15.0f + log2f(w * inv_wmax) : -INFINITY;
          }
          mbar_arrive(&pfull[ps]);
          ++g;
        }
      }
    }
    if (!ok && lane == 0) propagate_abort();
    if (__any_sync(0xffffffffu, negative) && lane == 0) atomicOr(&scal->err, kErrNegWeight);
  } else if (warp < C::kFirstProducerWarp) {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;                         // TMEM lane quadrant
    const int colh = (warp - 2) >> 2;               // which 128 columns
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const uint32_t accempty_leader = map_to_rank(smem_u32(accempty), 0);
    uint32_t dc = 0;
    bool ok = true;
    for (int rd = 0, it = sched_pos<SPARSE>(0, cluster, n_clusters); ok && it < n_items;
         it = sched_pos<SPARSE>(++rd, cluster, n_clusters)) {
      const Item itm = get_item<SPARSE>(tab, ninst, sp, it);
      const TcInst& I = *itm.I;
      const int nx = I.nx, ny = I.ny, CS = I.chunk_stages;
      const float wmax = __uint_as_float(I.scal->wmax_bits);
      const float scale = I.base_scale * (wmax > 0.f ? wmax : 1.0f);
      const int i = itm.tm * 256 + (int)rank * kRows + q * 32 + lane;
      const int j0 = itm.tn * 256 + colh * 128;
      float* slot = I.part + (int64_t)itm.s * nx * ny;
      // sparse: the piece's own 256 x 256 partial, [j_local][i_local]
      float* piece = SPARSE ? sp.part + itm.slot * 65536 + (int64_t)(colh * 128) * 256 +
                                  (int)rank * kRows + q * 32 + lane
                            : nullptr;
      if (!SPARSE && itm.nst == 0) {
        if (i < nx)
          for (int c = 0; c < 128 && j0 + c < ny; ++c) slot[(int64_t)(j0 + c) * nx + i] = 0.f;
        continue;
      }
      const int nchunks = (itm.nst + CS - 1) / CS;
      for (int ch = 0; ok && ch < nchunks; ++ch, ++dc) {
        const bool first = ch == 0, final = ch == nchunks - 1;
        if (!(ok = mbar_wait(accfull, dc & 1, abort_flag, scal, kRoleEpilogue))) break;
        tc_fence_after();
        const uint32_t acc_col = tmem_base + lane_off + colh * 128;
        const uint32_t run_col = acc_col + 256;
        // 32-column slices, the accumulator and running-sum loads in flight
        // together; the accumulator is released as soon as its last slice is
        // in registers (the MMAs never touch the running sum's columns)
#pragma unroll 1
        for (int cb = 0; cb < 4; ++cb) {
          uint32_t ra[32], rr[32];
          tmem_ld32_async(acc_col + cb * 32, ra);
          if (!first) tmem_ld32_async(run_col + cb * 32, rr);
          tmem_wait_ld();
          if (cb == 3) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(accempty_leader);
          }
          float a[32];
#pragma unroll
          for (int c = 0; c < 32; ++c) a[c] = __uint_as_float(ra[c]);
          if (!first) {
#pragma unroll
            for (int c = 0; c < 32; ++c) a[c] += __uint_as_float(rr[c]);
          }
          if (final && SPARSE) {
#pragma unroll
            for (int c = 0; c < 32; ++c) piece[(cb * 32 + c) * 256] = a[c] * scale;
          } else if (final) {
            if (i < nx) {
#pragma unroll
              for (int c = 0; c < 32; ++c) {
                const int j = j0 + cb * 32 + c;
                if (j < ny) slot[(int64_t)j * nx + i] = a[c] * scale;
              }
            }
          } else {
            tmem_st32(run_col + cb * 32, a);
          }
        }
        // the running sum's stores complete before this thread's next loads
        if (!final) tmem_wait_st();
      }
    }
    if (!ok && lane == 0) propagate_abort();
  } else {
    // ------------------------------------------------------------ producers
    const int t = threadIdx.x - C::kFirstProducerWarp * 32;
    const bool isA = t < kRows * C::kPerRow;  // warp-uniform
    const int tl = isA ? t : t - kRows * C::kPerRow;
    const int r = tl % kRows;
    const int chunk0 = (tl / kRows) * (8 / C::kPerRow);  // first 8-point chunk of this thread
    const int lo_off = isA ? C::kABytes : C::kBBytes;
    uint32_t full_leader[C::kStages];
#pragma unroll
    for (int s = 0; s < C::kStages; ++s) full_leader[s] = map_to_rank(smem_u32(&full[s]), 0);
    uint32_t g = 0;
    bool ok = true;
    for (int rd = 0, it = sched_pos<SPARSE>(0, cluster, n_clusters); ok && it < n_items;
         it = sched_pos<SPARSE>(++rd, cluster, n_clusters)) {
      const Item itm = get_item<SPARSE>(tab, ninst, sp, it);
      const TcInst& I = *itm.I;
      float gv;
      if (isA) {
        const int base = itm.tm * 256 + (int)rank * kRows;
        const float2 c = I.gxt[min(base + kRows / 2, I.nx - 1)];
        const float2 v = I.gxt[min(base + r, I.nx - 1)];
        gv = (v.x - c.x) + (v.y - c.y);
      } else {
        const int base = itm.tn * 256 + (int)rank * kRows;
        const float2 c = I.gyt[min(base + kRows / 2, I.ny - 1)];
        const float2 v = I.gyt[min(base + r, I.ny - 1)];
        gv = (v.x - c.x) + (v.y - c.y);
      }
      for (int st = 0; st < itm.nst; ++st, ++g) {
        const uint32_t s = g % C::kStages, ps = g % kPS;
        if (!(ok = mbar_wait(&pfull[ps], (g / kPS) & 1, abort_flag, scal, kRoleProducer))) break;
        if (!(ok = mbar_wait(&empty[s], ((g / C::kStages) & 1) ^ 1, abort_flag, scal,
                             kRoleProducer)))
          break;
        unsigned char* hi_row =
            smem + s * C::kStageBytes + (isA ? C::kOffA : C::kOffB) + r * C::kRowBytes;
        const float4* crd = reinterpret_cast<const float4*>(params + ps * 3 * kKS + (isA ? 0 : kKS));
        const float4* cbv = reinterpret_cast<const float4*>(params + ps * 3 * kKS + 2 * kKS);
#pragma unroll
        for (int c = chunk0; c < chunk0 + 8 / C::kPerRow; ++c) {
          const float4 p0 = crd[2 * c], p1 = crd[2 * c + 1];
          float4 c0 = make_float4(15.f, 15.f, 15.f, 15.f), c1 = c0;
          if (!isA) {
            c0 = cbv[2 * c];
            c1 = cbv[2 * c + 1];
          }
          const float pc[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
          const float ce[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
          float v[8];
#pragma unroll
          for (int e2 = 0; e2 < 8; ++e2) {
            const float u = gv - pc[e2];
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(v[e2]) : "f"(fmaf(-u, u, ce[e2])));
          }
          const int off = (c ^ (r & 7)) << 4;
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int e2 = 0; e2 < 4; ++e2) {
            if (SPLIT) {
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
          *reinterpret_cast<uint4*>(hi_row + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          if (SPLIT)
            *reinterpret_cast<uint4*>(hi_row + lo_off + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        // each writer orders its stores to this CTA's shared memory before
        // the tensor core's (async-proxy) reads of it, then the warp signals
        // the leader's stage barrier once
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive_cluster(full_leader[s]);
          mbar_arrive(&pempty[ps]);
        }
      }
    }
    if (!ok && lane == 0) propagate_abort();
  }

  __syncwarp();
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // the leader's MMAs are done; no CTA touches the other any more
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, C::kTmemCols);
  }
}

template <bool SPLIT, bool SPARSE>
cudaError_t launch_pair(const TcPlan& p, const TcInst* tab, int ninst, int n_items,
                        const SparseCtl& sp, CallScalars* err, cudaStream_t s) {
  using C = PairCfg<SPLIT, SPARSE>;
  cudaError_t e = cudaFuncSetAttribute(k_tc_pair<SPLIT, SPARSE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
  if (e != cudaSuccess) return e;
  // the sparse work list's length is known only on the device
  const int clusters = SPARSE ? std::max(1, p.ctas / 2) : std::max(1, std::min(n_items, p.ctas / 2));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * clusters);
  cfg.blockDim = dim3(C::kThreads);
  cfg.dynamicSmemBytes = C::kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_tc_pair<SPLIT, SPARSE>, tab, ninst, n_items, sp, err);
  note_launches(1);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_pair(const TcPlan& plan, const TcInst* tab, int ninst, int n_items,
                           const SparseCtl* sp, CallScalars* err, cudaStream_t s) {
  if (ninst < 1 || plan.ctas < 2 || plan.stage_points != kKS) return cudaErrorInvalidValue;
  if (sp) {
    if (sp->tiles_total < 1 || sp->piece_len < kKS || sp->piece_len % kKS) return cudaErrorInvalidValue;
    return plan.split16 ? launch_pair<true, true>(plan, tab, ninst, 0, *sp, err, s)
                        : launch_pair<false, true>(plan, tab, ninst, 0, *sp, err, s);
  }
  if (n_items < 1) return cudaErrorInvalidValue;
  const SparseCtl none = {};
  return plan.split16 ? launch_pair<true, false>(plan, tab, ninst, n_items, none, err, s)
                      : launch_pair<false, false>(plan, tab, ninst, n_items, none, err, s);
}

}  // namespace kde
