// Douglas-Peucker compression of the trajectories (Sec. III-B), in the
// level-synchronous form of Sec. IV-A: every curve segment of every
// trajectory is processed in the same iteration, so the recursion of the
// textbook algorithm becomes a loop over tree levels.
//
// Each point carries the two ends (s, e) of the segment it lies in, which
// plays the part of the paper's label set Lp, and each segment's length
// |e - s| is kept at its start index.  Eq. 9's VED is |cross| / length, and for
// one segment the correctly rounded quotient never decreases when the cross
// product grows, so the steps work on the cross product and divide only where
// the result could depend on it.  One iteration:
//   1. ved   : the cross product of every open point with its segment; its
//              maximum per segment by a segmented max over each warp's lanes
//              and one 64-bit atomicMax per run (non-negative doubles order
//              like their bit patterns);
//   2. arg   : the segment's largest VED is the maximum cross product divided
//              by the length; the points whose cross product is within 1e-15
//              of the maximum (no other can tie after rounding) compute their
//              VED exactly, and the first one equal to that largest VED, if it
//              exceeds eps, is the split (atomicMin) -- the tie rule of the
//              sequential algorithm;
//   3. split : that point is kept and records the lengths of the two segments
//              it starts and ends; the others move their s or e to it (the
//              label update of Eq. 11); segments with nothing above eps are
//              closed.  The per-segment slots of the next iteration
//              (double-buffered) are cleared here.
// The loop ends when an iteration keeps no point.  All iterations run in one
// cooperative launch: the three steps are phases of a persistent kernel
// separated by grid-wide barriers, and the count of points kept in an
// iteration is read on the device, so no level costs a host round trip.
// The VED is evaluated with
// explicitly rounded FP64 operations in the order of Eq. 9, so every
// comparison -- and therefore the kept set -- is identical to a sequential
// FP64 evaluation.  The kept points are then compacted with the Sec. IV-A
// exclusive scan.
#include <cooperative_groups.h>

#include "kde_internal.cuh"

namespace kde {
namespace {

namespace cg = cooperative_groups;

constexpr uint8_t kKept = 1, kDone = 2;
constexpr uint32_t kNoArg = 0xffffffffu;

// |e - s|, rounded as Eq. 9 is evaluated
__device__ __forceinline__ double seg_len(double2 a, double2 b) {
  const double dx = __dsub_rn(b.x, a.x), dy = __dsub_rn(b.y, a.y);
  return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}
// The numerator of Eq. 9, |(p - s) x (e - s)| -- or, for a segment of zero
// length, the distance |p - s| itself (the VED then).
__device__ __forceinline__ double ved_num(double2 q, double2 a, double2 b, double len) {
  const double vx = __dsub_rn(q.x, a.x), vy = __dsub_rn(q.y, a.y);
  if (len == 0.0) return __dsqrt_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)));
  const double dx = __dsub_rn(b.x, a.x), dy = __dsub_rn(b.y, a.y);
  return fabs(__dsub_rn(__dmul_rn(vx, dy), __dmul_rn(vy, dx)));
}
// The VED from its numerator.
__device__ __forceinline__ double ved_of(double num, double len) {
  return len == 0.0 ? num : __ddiv_rn(num, len);
}

// Trajectory bounds of point p: the last k with off[k] <= p; bounds clamped to
// [0, n] so that malformed offsets cannot index outside the points.
__device__ __forceinline__ void traj_bounds(const int64_t* __restrict__ off, int64_t ntraj,
                                            int64_t n, int64_t p, int64_t& a, int64_t& b) {
  if (!off) {
    a = 0;
    b = n;
    return;
  }
  int64_t lo = 0, hi = ntraj - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid; else hi = mid - 1;
  }
  a = min(max(off[lo], (int64_t)0), n);
  b = min(max(off[lo + 1], a), n);
}

__global__ void k_dp_init(const double2* __restrict__ xy, int64_t n,
                          const int64_t* __restrict__ off, int64_t ntraj, int32_t* __restrict__ s,
                          int32_t* __restrict__ e, uint8_t* __restrict__ flag,
                          unsigned long long* __restrict__ segmax, uint32_t* __restrict__ segarg,
                          double* __restrict__ seglen, CallScalars* __restrict__ scal) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    int64_t a, b;
    traj_bounds(off, ntraj, n, p, a, b);
    const double2 q = xy[p];
    bool bad = !(isfinite(q.x) && isfinite(q.y));
    if (!(a <= p && p < b)) {  // offsets do not cover p: a trajectory of its own
      bad = true;
      a = p;
      b = p + 1;
    }
    s[p] = (int32_t)a;
    e[p] = (int32_t)(b - 1);
    flag[p] = (p == a || p == b - 1 || bad) ? kKept : 0;
    if (p == a) seglen[p] = seg_len(q, xy[b - 1]);
    segmax[p] = 0ull;
    segmax[n + p] = 0ull;
    segarg[p] = kNoArg;
    segarg[n + p] = kNoArg;
    if (bad) atomicOr(&scal->err, kErrNonFinite);
  }
  if (off && blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[ntraj] != n))
    atomicOr(&scal->err, kErrBadArg);
}

// Step 1.  Lanes of a warp hold consecutive points, so equal segment starts
// form runs of lanes: a shuffle scan takes each run's maximum and its last
// lane issues the atomic.
__device__ __forceinline__ void dp_ved(const double2* __restrict__ xy, int64_t n,
                                       const int32_t* __restrict__ s, const int32_t* __restrict__ e,
                                       const uint8_t* __restrict__ flag,
                                       const double* __restrict__ seglen, double* __restrict__ num,
                                       unsigned long long* __restrict__ segmax) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t p = base + threadIdx.x;
    int64_t key = -1 - lane;  // lanes without a candidate never join a run
    unsigned long long v = 0ull;
    if (p < n && !(flag[p] & (kKept | kDone))) {
      const int32_t sp = s[p], ep = e[p];
      const double c = ved_num(xy[p], xy[sp], xy[ep], seglen[sp]);
      num[p] = c;
      key = sp;
      v = (unsigned long long)__double_as_longlong(c);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long vo = __shfl_up_sync(0xffffffffu, v, o);
      const int64_t ko = __shfl_up_sync(0xffffffffu, key, o);
      if (lane >= o && ko == key && vo > v) v = vo;
    }
    const int64_t knext = __shfl_down_sync(0xffffffffu, key, 1);
    const bool last = lane == 31 || knext != key;
    if (last && key >= 0 && v != 0ull) atomicMax(&segmax[key], v);
  }
}

// Step 2: the first point of each segment whose VED equals the segment's
// largest, when that exceeds eps.  A cross product below (1 - 1e-15) times the
// largest one gives a VED strictly below the largest after rounding (the
// division is correctly rounded and monotone), so only the others divide.
__device__ __forceinline__ void dp_arg(int64_t n, double eps, const int32_t* __restrict__ s,
                                       const uint8_t* __restrict__ flag,
                                       const double* __restrict__ seglen,
                                       const double* __restrict__ num,
                                       const unsigned long long* __restrict__ segmax,
                                       uint32_t* __restrict__ segarg) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    if (flag[p] & (kKept | kDone)) continue;
    const int32_t sp = s[p];
    const double cmax = __longlong_as_double((long long)segmax[sp]);
    const double c = num[p];
    if (!(c >= __dmul_rn(cmax, 1.0 - 1e-15))) continue;
    const double len = seglen[sp];
    const double dmax = cmax == 0.0 ? 0.0 : ved_of(cmax, len);
    const double d = c == cmax ? dmax : ved_of(c, len);
    if (dmax > eps && d == dmax) atomicMin(&segarg[sp], (uint32_t)p);
  }
}

// Step 3: keep the split points, move the others' segment ends, close the
// segments without a split, clear the next iteration's slots.
__device__ __forceinline__ void dp_split(const double2* __restrict__ xy, int64_t n,
                                         int32_t* __restrict__ s, int32_t* __restrict__ e,
                                         uint8_t* __restrict__ flag,
                                         const uint32_t* __restrict__ segarg,
                                         double* __restrict__ seglen,
                                         unsigned long long* __restrict__ segmax_next,
                                         uint32_t* __restrict__ segarg_next,
                                         unsigned long long* __restrict__ kept_now) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long mine = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const uint8_t f = flag[p];
    if (f & (kKept | kDone)) continue;
    int32_t sp = s[p];
    const uint32_t k = segarg[sp];
    if (k == kNoArg) {
      flag[p] = f | kDone;
      continue;
    }
    if ((int64_t)k == p) {  // the lengths of the segments [s, p] and [p, e]
      flag[p] = kKept;
      const double2 q = xy[p];
      seglen[sp] = seg_len(xy[sp], q);
      seglen[p] = seg_len(q, xy[e[p]]);
      ++mine;
      continue;
    }
    if (p < (int64_t)k) e[p] = (int32_t)k;
    else s[p] = sp = (int32_t)k;
    segmax_next[sp] = 0ull;
    segarg_next[sp] = kNoArg;
  }
  if (mine) atomicAdd(kept_now, mine);
}

// Every iteration of the level loop in one cooperative launch (all CTAs
// resident).  counter[it & 1] counts the points iteration `it` keeps; the
// other slot is cleared after the first barrier of the iteration, when every
// CTA has read the previous iteration's count.  Each CTA leaves the loop on
// the same count, so all take the same barriers.  Every iteration keeps at
// least one point or ends the loop, so n + 1 iterations bound it.
__global__ void __launch_bounds__(256)
    k_dp_levels(const double2* __restrict__ xy, int64_t n, double eps, int32_t* __restrict__ s,
                int32_t* __restrict__ e, uint8_t* __restrict__ flag, double* __restrict__ num,
                double* __restrict__ seglen, unsigned long long* __restrict__ segmax,
                uint32_t* __restrict__ segarg, unsigned long long* __restrict__ counter,
                int* __restrict__ iterations) {
  cg::grid_group grid = cg::this_grid();
  __shared__ unsigned long long kept;
  int64_t it = 0;
  for (; it <= n; ++it) {
    const int b = (int)(it & 1);
    dp_ved(xy, n, s, e, flag, seglen, num, segmax + b * n);
    grid.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) counter[b ^ 1] = 0ull;
    dp_arg(n, eps, s, flag, seglen, num, segmax + b * n, segarg + b * n);
    grid.sync();
    dp_split(xy, n, s, e, flag, segarg + b * n, seglen, segmax + (b ^ 1) * n,
             segarg + (b ^ 1) * n, counter + b);
    grid.sync();
    if (threadIdx.x == 0) kept = __ldcg(counter + b);
    __syncthreads();
    const bool done = kept == 0ull;
    __syncthreads();  // `kept` is rewritten in the next iteration
    if (done) {
      ++it;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *iterations = (int)it;
}

__global__ void k_dp_flags(const uint8_t* __restrict__ flag, int64_t n,
                           uint32_t* __restrict__ kept32, uint8_t* __restrict__ keep) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= n; p += stride) {
    const uint32_t k = p < n ? (flag[p] & kKept) : 0u;
    kept32[p] = k;
    if (p < n) keep[p] = (uint8_t)k;
  }
}

__global__ void k_dp_compact(const double2* __restrict__ xy, int64_t n,
                             const uint32_t* __restrict__ kept32, const uint32_t* __restrict__ pos,
                             double2* __restrict__ out, const int64_t* __restrict__ off,
                             int64_t ntraj, int64_t* __restrict__ out_off) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
    if (out && kept32[p]) out[pos[p]] = xy[p];
  if (out_off)
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= ntraj; k += stride) {
      const int64_t o = off ? min(max(off[k], (int64_t)0), n) : (k == 0 ? 0 : n);
      out_off[k] = pos[o];
    }
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

}  // namespace

size_t dp_workspace_bytes(int64_t n) {
  const size_t m = (size_t)n + 1;
  return 256 * 14 + m * (4 + 4 + 1 + 16 + 8 + 8 + 8 + 4 + 4) +
         4 * (scan_temp_words((int64_t)m, 2048) + 64);
}

cudaError_t launch_dp(const double* xy, int64_t n, const int64_t* off, int64_t ntraj, double eps,
                      uint8_t* keep, double* out_xy, int64_t* out_off, void* ws,
                      CallScalars* scal, int64_t* n_kept, int* iterations, cudaStream_t st) {
  const size_t m = (size_t)n + 1;
  char* w = static_cast<char*>(ws);
  size_t o = 0;
  auto take = [&](size_t bytes) { char* r = w + o; o = (o + bytes + 255) & ~(size_t)255; return r; };
  int32_t* s = reinterpret_cast<int32_t*>(take(4 * m));
  int32_t* e = reinterpret_cast<int32_t*>(take(4 * m));
  uint8_t* flag = reinterpret_cast<uint8_t*>(take(m));
  unsigned long long* segmax = reinterpret_cast<unsigned long long*>(take(16 * m));
  double* num = reinterpret_cast<double*>(take(8 * m));
  double* seglen = reinterpret_cast<double*>(take(8 * m));
  uint32_t* segarg = reinterpret_cast<uint32_t*>(take(8 * m));
  uint32_t* kept32 = reinterpret_cast<uint32_t*>(take(4 * m));
  uint32_t* pos = reinterpret_cast<uint32_t*>(take(4 * m));
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(take(16));
  int* iters_dev = reinterpret_cast<int*>(take(sizeof(int)));
  uint32_t* scan_temp = reinterpret_cast<uint32_t*>(take(4 * (scan_temp_words((int64_t)m, 2048) + 64)));
  const double2* P = reinterpret_cast<const double2*>(xy);
  const int g = grid_for(n);
  cudaError_t err = cudaSuccess;
  int it = 0;
  if (n > 0) {
    k_dp_init<<<g, 256, 0, st>>>(P, n, off, ntraj, s, e, flag, segmax, segarg, seglen, scal);
    note_launches(1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(counter, 0, 16, st)) != cudaSuccess) return err;
    // all CTAs of the cooperative launch must be resident at once
    int dev = 0, per_sm = 0, sms = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dp_levels, 256, 0)) !=
        cudaSuccess)
      return err;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    // up to four CTAs per SM: enough warps for the memory phases, few CTAs
    // at each barrier
    const int gl = (int)std::min<int64_t>((int64_t)std::min(per_sm, 4) * sms, (n + 255) / 256);
    void* args[] = {(void*)&P, (void*)&n, (void*)&eps, (void*)&s, (void*)&e, (void*)&flag,
                    (void*)&num, (void*)&seglen, (void*)&segmax, (void*)&segarg,
                    (void*)&counter, (void*)&iters_dev};
    err = cudaLaunchCooperativeKernel((const void*)k_dp_levels, dim3(gl), dim3(256), args, 0, st);
    note_launches(1);
    if (err != cudaSuccess) return err;
    if ((err = cudaMemcpyAsync(&it, iters_dev, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return err;
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;
  }
  if (iterations) *iterations = it;
  k_dp_flags<<<grid_for(n + 1), 256, 0, st>>>(flag, n, kept32, keep);
  note_launches(1);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if ((err = launch_exclusive_scan(kept32, pos, (int64_t)m, 2048, scan_temp, st)) != cudaSuccess)
    return err;
  if (out_xy || out_off) {
    k_dp_compact<<<grid_for(std::max<int64_t>(n, ntraj + 1)), 256, 0, st>>>(
        P, n, kept32, pos, reinterpret_cast<double2*>(out_xy), off, ntraj, out_off);
    note_launches(1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  if (n_kept) {
    uint32_t total = 0;
    if ((err = cudaMemcpyAsync(&total, pos + n, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return err;
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;
    *n_kept = total;
  }
  return cudaSuccess;
}

}  // namespace kde
