/*
 * rsb_test.h — measurement and test hooks of librsb.  They are not part of the
 * method and not needed to partition a mesh: kernel timing for the bandwidth
 * roofline of the benchmark, and a switch that drives the failure path of the
 * bounded device waits in tests.  The method's calls are in rsb.h.
 */
#ifndef RSB_TEST_H
#define RSB_TEST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Kernel timing for bandwidth accounting (not part of the method).
 * rsb_profile_begin(family) makes the following calls bracket every launch of
 * one kernel family (or of every family, RSB_PROF_ALL) with CUDA events on the
 * library's stream and add up the algorithmic bytes of each launch;
 * rsb_profile_end() returns the totals over the timed families and switches
 * timing off; rsb_profile_read() then gives one family's totals.  Families:
 *   1 Lanczos SpMV: k_lz_a1 (FP32 step D1) or the fused k_lz_a (FP64 step A)
 *   2 FP32 step D3 (both updates + norm, k_lz_d3) or FP64 step B (update +
 *     second Gram-Schmidt dots, k_lz_b)
 *   3 FP64 step C (update + norm, k_lz_c)
 *   4 CG Laplacian action (inverse iteration)
 *   5 Laplacian action of rsb_laplacian_bench
 *   6 the persistent Lanczos kernels (bytes of all of their phases)
 *   7 FP32 step D2 (dots of v_j and z with the basis, k_lz_d2)
 *   8 the AMG V-cycles of the flexible CG (time only)
 * Bytes count 4 B per stored SELL entry (padding included), every vector
 * element read or written once, and FP64 deflation vectors.  The event
 * records add a few microseconds per launch, so profiled calls run slower.
 */
#define RSB_PROF_ALL (-1)
void rsb_profile_begin(int family);
void rsb_profile_end(double *ms_total, int64_t *launches, double *bytes_total);
void rsb_profile_read(int family, double *ms, int64_t *launches, double *bytes);

/*
 * Failure-path test hook (not part of the method).  While on != 0, the
 * persistent launch modes (use_graph 2 and 3) start their grid barrier from a
 * corrupted arrival count, so no CTA sees the last arrival: every bounded wait
 * runs out (4 s of the GPU's global timer), the kernel ends, and the call
 * returns RSB_ETIMEOUT.  Nothing faults or hangs; the next call with the hook
 * off starts from a clean barrier.  Process-wide, not thread-safe; for tests.
 */
void rsb_test_poison_barrier(int on);

#ifdef __cplusplus
}
#endif

#endif /* RSB_TEST_H */
