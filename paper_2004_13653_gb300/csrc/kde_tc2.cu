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
// Roles, by warpgroup (setmaxnreg divides the registers per warpgroup):
//   WG0   warp 0: MMA issue (leader CTA, one thread); warp 1: loads and
//         re-centres the points of each stage; warp 2: signals each finished
//         stage to the leader (one cluster arrive per CTA and stage); warp 3
//         idles.  48 registers.
//   WG1-2 warps 4-11: epilogue.  Each thread owns one TMEM lane (an x cell)
//         and 128 of the tile's 256 y cells, and keeps their running sums in
//         its registers (168 registers).
//   WG3-4 warps 12-19: operand producers, four per operand; each thread
//         writes a quarter of four A or B rows (48 registers).
//
// Accumulators: two N = 256 FP32 accumulators fill TMEM's 512 columns.  The
// MMAs of chunk c (k_chunk points) accumulate into accumulator c mod 2 while
// the epilogues add chunk c - 1 into their registers, so the tensor core does
// not wait for a drain.  Chunks stay short because the tensor core's FP32
// accumulation loses accuracy with every MMA step it adds into a large sum;
// the running sums add the chunks with IEEE FP32 adds.
//
// Stage hand-off: each producer orders its shared-memory stores before the
// tensor core's (async-proxy) reads with fence.proxy.async and arrives on a
// named barrier without waiting; the signalling warp waits on that barrier
// and makes one cluster-scope release arrive on the leader's stage barrier.
// The barrier's id follows the stage slot, so a producer can reach the same
// id again only after the MMAs have consumed that slot, i.e. after the
// barrier completed.
//
// Weights enter B as log2(|w|/w_max) in the exponent; an instance with a
// negative weight (flagged by the prepare kernel) also gets each B value's
// sign, applied to the packed FP16 hi/lo words.
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
constexpr int kGroup = 1;   // stages the loader fetches at once

// parameter ring slot: A coordinates, B coordinates, B exponent offsets
// (-(15 + log2(|w|/w_max)), +inf for w = 0), B sign words of point pairs
constexpr int kPrmA = 0, kPrmB = kKS, kPrmN = 2 * kKS, kPrmS = 3 * kKS;
constexpr int kPrmFloats = 3 * kKS + kKS / 2;

// warp roles and register budgets (see the file comment)
constexpr int kWarps = 20;
constexpr int kThreads = 32 * kWarps;
constexpr int kWarpMma = 0, kWarpLoader = 1, kWarpSignal = 2;
constexpr int kFirstEpiWarp = 4, kEpiWarps = 8;
constexpr int kFirstProducerWarp = 12, kProducerWarps = 8;
constexpr int kRowsPerThread = kRows / 32;  // operand rows per producer thread
constexpr int kRegsLaunch = 96;  // 640 threads: at most 65536 / 640 = 102, allocated in 8s
constexpr int kRegsCtl = 48, kRegsEpi = 168, kRegsProd = 48;
static_assert(128 * kRegsCtl + 256 * kRegsEpi + 256 * kRegsProd <= kThreads * kRegsLaunch,
              "the warpgroups' register budgets exceed the block's pool");
constexpr int kBarProducers = 1;  // named barriers 1..kStages: producers -> signal warp

enum Role : int {
  kRoleMma = 11, kRoleLoader = 12, kRoleEpilogue = 13, kRoleProducer = 14, kRoleSignal = 15
};

template <bool SPLIT, bool SPARSE>
struct PairCfg {
  static constexpr int kRowBytes = 2 * kKS;
  static constexpr int kABytes = kRows * kRowBytes;
  static constexpr int kBBytes = kRows * kRowBytes;
  static constexpr int kParts = SPLIT ? 2 : 1;
  static constexpr int kStageBytes = kParts * (kABytes + kBBytes);
  static constexpr int kStages = (192 * 1024) / kStageBytes;
  static constexpr uint32_t kTmemCols = 512;
  static constexpr uint32_t kIdesc = idesc_f16_f32(256, 256);
  static constexpr int kOffA = 0;
  static constexpr int kOffB = kParts * kABytes;
  static constexpr int kOffParams = kStages * kStageBytes;
  static constexpr int kOffBars = kOffParams + kPS * kPrmFloats * 4;
  static constexpr int kNumBars = 2 * kStages + 2 * kPS + 2 + 2 + 1;
  static constexpr int kOffMisc = kOffBars + kNumBars * 8;
  static constexpr int kSmemBytes = kOffMisc + 64 + 1024;
  static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
  static_assert(kBarProducers + kStages <= 16, "named barrier ids");
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
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_pair(const TcInst* __restrict__ tab, int ninst, int n_items_arg,
              const __grid_constant__ SparseCtl sp, const uint32_t* __restrict__ sched,
              CallScalars* __restrict__ scal) {
  using C = PairCfg<SPLIT, SPARSE>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float* params = reinterpret_cast<float*>(smem + C::kOffParams);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kOffBars);
  uint64_t* full = bars;                    // [kStages] signal warps (both CTAs) -> leader MMA
  uint64_t* empty = bars + C::kStages;      // [kStages] MMA -> producers (multicast)
  uint64_t* pfull = bars + 2 * C::kStages;  // [kPS] loader -> producers
  uint64_t* pempty = pfull + kPS;           // [kPS] signal warp -> loader
  uint64_t* accfull = pempty + kPS;         // [2] MMA -> epilogues (multicast)
  uint64_t* accempty = accfull + 2;         // [2] epilogues (both CTAs) -> leader MMA
  uint64_t* mmadone = accempty + 2;         // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kOffMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kOffMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int n_items = n_items_arg;
  if (SPARSE) {  // the work list was built on the device by the preceding launches
    const int listed = (int)__ldg(sp.piece_begin + sp.tiles_total);
    // a list longer than the partial buffer is an error: no piece is computed.
    // So is a timed-out bin sort (the pieces' positions come from its bin
    // starts); only the sort, an earlier launch, sets that bit, so both CTAs
    // of a pair read the same value and agree on their (empty) list
    const bool sort_failed =
        *reinterpret_cast<const volatile int*>(&scal->err) & kErrSortTimeout;
    n_items = listed > sp.max_pieces || sort_failed ? 0 : listed;
    if (listed > sp.max_pieces && blockIdx.x == 0 && threadIdx.x == 0)
      atomicOr(&scal->err, kErrBadArg);
  }
  const uint32_t rank = cluster_rank();
  const uint32_t peer = rank ^ 1u;
  const int cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;
  auto propagate_abort = [&]() {
    store_cluster_u32(map_to_rank(smem_u32((const void*)abort_flag), peer), 1u);
  };
  // The item at position k of this CTA pair's list, -1 past its end: from the
  // host's schedule table when there is one (offsets[n_clusters + 1], then
  // the items), else round robin (snake order for block-sparse pieces).
  // Every role of both CTAs walks the same list.
  auto item_at = [&](int k) -> int {
    if (sched) {
      const uint32_t a = __ldg(sched + cluster), b = __ldg(sched + cluster + 1);
      return a + (uint32_t)k < b ? (int)__ldg(sched + n_clusters + 1 + a + k) : -1;
    }
    const int it = sched_pos<SPARSE>(k, cluster, n_clusters);
    return it < n_items ? it : -1;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 2);  // one signal-warp arrive per CTA of the pair
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < kPS; ++s) {
      mbar_init(&pfull[s], 32);
      mbar_init(&pempty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 2 * kEpiWarps);
    }
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

  if (warp < kFirstEpiWarp) {
    regs_dec<kRegsCtl>();
    if (warp == kWarpMma) {
      // ----------------------------------------------- MMA issue (leader only)
      if (rank == 0 && lane == 0) {
        uint32_t g = 0, mc = 0;
        bool ok = true;
        const uint32_t smem_base = smem_u32(smem);
        for (int rd = 0, it = item_at(0); ok && it >= 0; it = item_at(++rd)) {
          const Item itm = get_item<SPARSE>(tab, ninst, sp, it);
          const int CS = itm.I->chunk_stages;
          uint32_t acc_addr = tmem_base;
          for (int st = 0; ok && st < itm.nst; ++st, ++g) {
            const bool fresh = st % CS == 0;
            if (fresh) {  // both CTAs' epilogues have taken this accumulator's last chunk
              const uint32_t b = mc & 1u;
              if (!(ok = mbar_wait_cluster(&accempty[b], ((mc >> 1) & 1u) ^ 1u, abort_flag, scal,
                                           kRoleMma)))
                break;
              tc_fence_after();
              acc_addr = tmem_base + b * 256u;
            }
            const uint32_t s = g % C::kStages;
            if (!(ok = mbar_wait_cluster(&full[s], (g / C::kStages) & 1, abort_flag, scal,
                                         kRoleMma)))
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
              mma_f16_pair(acc_addr, ahi + dk, bhi + dk, C::kIdesc, acc);
              if (SPLIT) {
                mma_f16_pair(acc_addr, ahi + dk, blo + dk, C::kIdesc, 1u);
                mma_f16_pair(acc_addr, alo + dk, bhi + dk, C::kIdesc, 1u);
              }
            }
            mma_commit_pair(&empty[s]);
            if (st + 1 == itm.nst || (st + 1) % CS == 0) {
              mma_commit_pair(&accfull[mc & 1u]);
              ++mc;
            }
          }
        }
        if (!ok) propagate_abort();
        mma_commit_pair(mmadone);
        mbar_wait(mmadone, 0, abort_flag, scal, kRoleMma, /*honour_abort=*/false);
      }
      __syncwarp();
    } else if (warp == kWarpLoader) {
      // ------------------------------------------------------- point loader
      uint32_t g = 0;
      bool ok = true;
      for (int rd = 0, it = item_at(0); ok && it >= 0; it = item_at(++rd)) {
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
            float* prm = params + ps * kPrmFloats;
            uint32_t neg[2];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const int e = lane + 32 * hh;
              const float4 q = P[u][hh];
              prm[kPrmA + e] = (q.x - cx.x) + (q.y - cx.y);
              prm[kPrmB + e] = (q.z - cy.x) + (q.w - cy.y);
              const float w = W[u][hh];
              neg[hh] = w < 0.f ? 1u : 0u;
              prm[kPrmN + e] = w != 0.f ? -(15.0f + log2f(fabsf(w) * inv_wmax)) : INFINITY;
            }
            // sign word of points (2 lane, 2 lane + 1): bit 15 and bit 31, the
            // sign bits of their packed FP16 halves
            const int src = (2 * lane) & 31;
            const uint32_t h = lane < 16 ? 0u : 1u;
            const uint32_t s_lo = __shfl_sync(0xffffffffu, neg[0], src) |
                                  (__shfl_sync(0xffffffffu, neg[1], src) << 1);
            const uint32_t s_hi = __shfl_sync(0xffffffffu, neg[0], src + 1) |
                                  (__shfl_sync(0xffffffffu, neg[1], src + 1) << 1);
            reinterpret_cast<uint32_t*>(prm + kPrmS)[lane] =
                (((s_lo >> h) & 1u) << 15) | (((s_hi >> h) & 1u) << 31);
            mbar_arrive(&pfull[ps]);
            ++g;
          }
        }
      }
      if (!ok && lane == 0) propagate_abort();
    } else if (warp == kWarpSignal) {
      // ------------------------------------------- stage hand-off to the MMA
      // It takes part in every stage's barrier, aborted or not, because the
      // producers arrive at every stage's barrier whatever happens.
      const uint32_t full_leader0 = map_to_rank(smem_u32(&full[0]), 0);
      uint32_t g = 0;
      for (int rd = 0, it = item_at(0); it >= 0; it = item_at(++rd)) {
        const Item itm = get_item<SPARSE>(tab, ninst, sp, it);
        for (int st = 0; st < itm.nst; ++st, ++g) {
          const uint32_t s = g % C::kStages;
          // every producer of this CTA has fenced and arrived for stage g
          named_sync(kBarProducers + (int)s, 32 * (kProducerWarps + 1));
          if (lane == 0 && !*abort_flag) {
            mbar_arrive_cluster(full_leader0 + 8u * s);
            mbar_arrive(&pempty[g % kPS]);
          }
          __syncwarp();
        }
      }
    }
  } else if (warp < kFirstProducerWarp) {
    // ------------------------------------------------------------- epilogue
    regs_inc<kRegsEpi>();
    const int q = warp & 3;                         // TMEM lane quadrant
    const int colh = (warp - kFirstEpiWarp) >> 2;   // which 128 columns
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const uint32_t accempty_leader0 = map_to_rank(smem_u32(&accempty[0]), 0);
    uint32_t dc = 0;
    bool ok = true;
    for (int rd = 0, it = item_at(0); ok && it >= 0; it = item_at(++rd)) {
      const Item itm = get_item<SPARSE>(tab, ninst, sp, it);
      const TcInst& I = *itm.I;
      const int nx = I.nx, ny = I.ny, CS = I.chunk_stages;
      const float wmax = __uint_as_float(I.scal->wmax_bits);
      const float scale = I.base_scale * (wmax > 0.f ? wmax : 1.0f);
      const int i = itm.tm * 256 + (int)rank * kRows + q * 32 + lane;
      const int j0 = itm.tn * 256 + colh * 128;
      float* slot = I.part + (int64_t)itm.s * nx * ny;
      float* piece = SPARSE ? sp.part + itm.slot * 65536 + (int64_t)(colh * 128) * 256 +
                                  (int)rank * kRows + q * 32 + lane
                            : nullptr;
      if (itm.nst == 0) {  // no points in this item's range: its sums are zero
        if (SPARSE)
          for (int c = 0; c < 128; ++c) piece[c * 256] = 0.f;
        else if (i < nx)
          for (int c = 0; c < 128 && j0 + c < ny; ++c) slot[(int64_t)(j0 + c) * nx + i] = 0.f;
        continue;
      }
      float run[128];
      const int nchunks = (itm.nst + CS - 1) / CS;
      for (int ch = 0; ok && ch < nchunks; ++ch, ++dc) {
        const uint32_t b = dc & 1u;
        if (!(ok = mbar_wait(&accfull[b], (dc >> 1) & 1u, abort_flag, scal, kRoleEpilogue))) break;
        tc_fence_after();
        const uint32_t acc_col = tmem_base + b * 256u + lane_off + colh * 128;
#pragma unroll
        for (int cb = 0; cb < 16; ++cb) {
          uint32_t ra[8];
          tmem_ld8_async(acc_col + cb * 8, ra);
          tmem_wait_ld();
          if (ch == 0) {
#pragma unroll
            for (int c = 0; c < 8; ++c) run[cb * 8 + c] = __uint_as_float(ra[c]);
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) run[cb * 8 + c] += __uint_as_float(ra[c]);
          }
        }
        // the accumulator is read: the MMAs of chunk dc + 2 may overwrite it
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(accempty_leader0 + 8u * b);
      }
      if (!ok) break;
      if (SPARSE) {  // the piece's own 256 x 256 partial, [j_local][i_local]
#pragma unroll
        for (int c = 0; c < 128; ++c) piece[c * 256] = run[c] * scale;
      } else if (i < nx) {
#pragma unroll
        for (int c = 0; c < 128; ++c)
          if (j0 + c < ny) slot[(int64_t)(j0 + c) * nx + i] = run[c] * scale;
      }
    }
    if (!ok && lane == 0) propagate_abort();
  } else {
    // ------------------------------------------------------------ producers
    // Four warps per operand; lane l of warp k of a group writes rows l,
    // l + 32, l + 64, l + 96 in chunks 2k and 2k + 1.  A thread reuses each
    // broadcast load of a chunk's point parameters for its four rows, which
    // keeps these loads a small share of the shared-memory bandwidth the
    // tensor core's operand reads and the operand stores already take.
    regs_dec<kRegsProd>();
    const int pw = warp - kFirstProducerWarp;
    const bool isA = pw < kProducerWarps / 2;  // warp-uniform
    const int c0 = 2 * (pw & 3);
    const int lo_off = isA ? C::kABytes : C::kBBytes;
    uint32_t g = 0;
    bool ok = true;
    // every stage ends with an arrive at its barrier, also after an abort
    // (then without waiting or storing), so the signalling warp never waits
    // on a barrier that cannot complete
    for (int rd = 0, it = item_at(0); it >= 0; it = item_at(++rd)) {
      const Item itm = get_item<SPARSE>(tab, ninst, sp, it);
      const TcInst& I = *itm.I;
      const bool signs = !isA && I.scal->negw != 0;
      float ngv[kRowsPerThread];  // minus the rows' cell coordinates
      {
        const int base = (isA ? itm.tm : itm.tn) * 256 + (int)rank * kRows;
        const float2* tab_g = isA ? I.gxt : I.gyt;
        const int n_g = isA ? I.nx : I.ny;
        const float2 c = tab_g[min(base + kRows / 2, n_g - 1)];
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) {
          const float2 v = tab_g[min(base + k * 32 + lane, n_g - 1)];
          ngv[k] = -((v.x - c.x) + (v.y - c.y));
        }
      }
      for (int st = 0; st < itm.nst; ++st, ++g) {
        const uint32_t s = g % C::kStages, ps = g % kPS;
        if (ok) ok = mbar_wait(&pfull[ps], (g / kPS) & 1, abort_flag, scal, kRoleProducer);
        if (ok)
          ok = mbar_wait(&empty[s], ((g / C::kStages) & 1) ^ 1, abort_flag, scal, kRoleProducer);
        if (!ok) {
          named_arrive(kBarProducers + (int)s, 32 * (kProducerWarps + 1));
          continue;
        }
        unsigned char* row0 =
            smem + s * C::kStageBytes + (isA ? C::kOffA : C::kOffB) + lane * C::kRowBytes;
        const float* prm = params + ps * kPrmFloats;
        const float4* crd = reinterpret_cast<const float4*>(prm + (isA ? kPrmA : kPrmB));
        const float4* nce = reinterpret_cast<const float4*>(prm + kPrmN);
        const uint4* sgn = reinterpret_cast<const uint4*>(prm + kPrmS);
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int c = c0 + cc;
          const float4 p0 = crd[2 * c], p1 = crd[2 * c + 1];
          float4 n0 = make_float4(-15.f, -15.f, -15.f, -15.f), n1 = n0;
          if (!isA) {
            n0 = nce[2 * c];
            n1 = nce[2 * c + 1];
          }
          uint4 sg = make_uint4(0u, 0u, 0u, 0u);
          if (signs) sg = sgn[c];
          const float2 P2[4] = {make_float2(p0.x, p0.y), make_float2(p0.z, p0.w),
                                make_float2(p1.x, p1.y), make_float2(p1.z, p1.w)};
          const float2 N2[4] = {make_float2(n0.x, n0.y), make_float2(n0.z, n0.w),
                                make_float2(n1.x, n1.y), make_float2(n1.z, n1.w)};
          // rows lane + 32 k share the swizzle phase lane & 7
          const int off = (c ^ (lane & 7)) << 4;
#pragma unroll
          for (int k = 0; k < kRowsPerThread; ++k) {
            const float2 ng2 = make_float2(ngv[k], ngv[k]);
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
              const float2 u = add2(P2[e2], ng2);     // point - cell, in units of h sqrt(2 ln 2)
              const float2 y = fma2(u, u, N2[e2]);    // u^2 - exponent offset
              const float v0 = ex2_neg(y.x), v1 = ex2_neg(y.y);
              if (SPLIT) {
                // hi = v with 11 significant bits (exact in FP16), lo = v - hi
                const float h0 = __uint_as_float(__float_as_uint(v0) & 0xFFFFE000u);
                const float h1 = __uint_as_float(__float_as_uint(v1) & 0xFFFFE000u);
                const float2 l = sub2(make_float2(v0, v1), make_float2(h0, h1));
                const __half2 hh = __floats2half2_rn(h0, h1);
                const __half2 ll = __floats2half2_rn(l.x, l.y);
                hw[e2] = *reinterpret_cast<const uint32_t*>(&hh);
                lw[e2] = *reinterpret_cast<const uint32_t*>(&ll);
              } else {
                const __half2 hh = __floats2half2_rn(v0, v1);
                hw[e2] = *reinterpret_cast<const uint32_t*>(&hh);
              }
            }
            if (signs) {  // negative weights: flip the FP16 sign bits of those points
              hw[0] ^= sg.x; hw[1] ^= sg.y; hw[2] ^= sg.z; hw[3] ^= sg.w;
              if (SPLIT) {
                lw[0] ^= sg.x; lw[1] ^= sg.y; lw[2] ^= sg.z; lw[3] ^= sg.w;
              }
            }
            unsigned char* row = row0 + k * 32 * C::kRowBytes;
            *reinterpret_cast<uint4*>(row + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            if (SPLIT)
              *reinterpret_cast<uint4*>(row + lo_off + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
        // order this thread's stores before the tensor core's reads of them,
        // then hand the stage to the signalling warp without waiting
        fence_proxy_async_smem();
        named_arrive(kBarProducers + (int)s, 32 * (kProducerWarps + 1));
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

}  // namespace

int pair_clusters(const TcPlan& plan, int n_items);

namespace {

template <bool SPLIT, bool SPARSE>
cudaError_t launch_pair(const TcPlan& p, const TcInst* tab, int ninst, int n_items,
                        const SparseCtl& sp, const uint32_t* sched, CallScalars* err,
                        cudaStream_t s) {
  using C = PairCfg<SPLIT, SPARSE>;
  // setmaxnreg draws on the registers the block was launched with: refuse a
  // build whose launch register count would not hold the warpgroups' budgets
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_tc_pair<SPLIT, SPARSE>);
  if (e != cudaSuccess) return e;
  if ((fa.numRegs + 7) / 8 * 8 < kRegsLaunch) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(k_tc_pair<SPLIT, SPARSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           C::kSmemBytes);
  if (e != cudaSuccess) return e;
  // the sparse work list's length is known only on the device
  const int clusters = SPARSE ? std::max(1, p.ctas / 2) : pair_clusters(p, n_items);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * clusters);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = C::kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_tc_pair<SPLIT, SPARSE>, tab, ninst, n_items, sp, sched, err);
  note_launches(1);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

int pair_clusters(const TcPlan& plan, int n_items) {
  return std::max(1, std::min(n_items, plan.ctas / 2));
}

cudaError_t launch_tc_pair(const TcPlan& plan, const TcInst* tab, int ninst, int n_items,
                           const SparseCtl* sp, const uint32_t* sched, CallScalars* err,
                           cudaStream_t s) {
  if (ninst < 1 || plan.ctas < 2 || plan.stage_points != kKS) return cudaErrorInvalidValue;
  if (sp) {
    if (sp->tiles_total < 1 || sp->piece_len < kKS || sp->piece_len % kKS) return cudaErrorInvalidValue;
    return plan.split16 ? launch_pair<true, true>(plan, tab, ninst, 0, *sp, nullptr, err, s)
                        : launch_pair<false, true>(plan, tab, ninst, 0, *sp, nullptr, err, s);
  }
  if (n_items < 1) return cudaErrorInvalidValue;
  const SparseCtl none = {};
  return plan.split16 ? launch_pair<true, false>(plan, tab, ninst, n_items, none, sched, err, s)
                      : launch_pair<false, false>(plan, tab, ninst, n_items, none, sched, err, s);
}

}  // namespace kde
