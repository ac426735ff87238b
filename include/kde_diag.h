/*
 * kde_diag.h — diagnostic entry points of the KDE library (building blocks
 * exposed so they can be checked against the paper on their own).
 */
#ifndef KDE_GB300_KDE_DIAG_H
#define KDE_GB300_KDE_DIAG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * kde_diag_exclusive_scan — the multi-block exclusive prefix sum of
 * arXiv 2004.13653, Sec. IV-A ("Scan Algorithm"): each block of `per_block`
 * elements is scanned, the block totals are scanned in turn (recursively) and
 * propagated to the following blocks.  The block-sparse work list and the
 * Douglas-Peucker compaction use it.  in, out: device, [n] uint32 (must not
 * alias); per_block in [1, 2048] (small values reproduce the paper's worked
 * example with four-element blocks).  Synchronous; uses the library
 * workspace.  Errors: KDE_EINVAL (n < 0, per_block out of range, null or host
 * pointers), KDE_ENOMEM, KDE_ECUDA.
 */
int kde_diag_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, int per_block,
                            void* stream);

/*
 * kde_diag_wait_timeout — exercises the bounded device-side waits that every
 * pipeline of the library uses between its producer, MMA and epilogue roles
 * (no counterpart in the paper, which has no such pipelines): one kernel
 * waits on a barrier nothing signals, gives up after limit_ns nanoseconds,
 * records the timeout and returns, leaving the context usable.  Returns
 * KDE_ETIMEOUT (the expected outcome), or KDE_EINVAL for a limit outside
 * [1 us, 2 s].  Synchronous.
 */
int kde_diag_wait_timeout(int64_t limit_ns, void* stream);

/*
 * kde_diag_sort_wait_timeout — exercises the bounded wait of the bin sort's
 * look-back (no counterpart in the paper; the sort orders the points of the
 * cutoff path, Sec. III-C with Eq. 8, and of the block-sparse path): one
 * radix pass over two chunks of zero keys runs as the second while the
 * first never publishes its counts, so the pass gives up after limit_ns
 * nanoseconds, records the timeout (role 31), keeps every position it writes
 * inside its buffers and returns, leaving the context usable.  Returns
 * KDE_ETIMEOUT (the expected outcome), or KDE_EINVAL for a limit outside
 * [1 us, 2 s].  Synchronous; uses the library workspace.
 */
int kde_diag_sort_wait_timeout(int64_t limit_ns, void* stream);

/*
 * kde_diag_peak_rates — measures, at the clock the GPU runs at, the rates the
 * rooflines of the tensor-core and exp-bound kernels are set against (no
 * counterpart in the paper): rates[0] = tcgen05 kind::f16 MMAs on CTA pairs
 * (M = 256, N = 256, K = 16, operands resident in shared memory), TFLOP/s;
 * rates[1] = the same on single CTAs (M = 128, N = 256); rates[2] = MUFU
 * ex2.approx results per second, in units of 1e12.  rates: host, [3] double,
 * written only on success.  Each probe runs for a few milliseconds on every
 * SM, twice (the first pass warms the clocks up).  Synchronous; uses the
 * library workspace.  Errors: KDE_EINVAL (null rates), KDE_ENOMEM, KDE_ECUDA,
 * KDE_ETIMEOUT (a bounded device-side wait gave up).
 */
int kde_diag_peak_rates(double* rates, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KDE_GB300_KDE_DIAG_H */
