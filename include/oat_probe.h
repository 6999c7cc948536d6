/*
 * Diagnostics of liboat.so: a memory-bandwidth probe, used by the benchmark to measure the
 * on-chip roofline it reports (the L2 read bandwidth is not among the measured peaks), and
 * the sample positions the filtered backprojection computes, for measuring their accuracy.
 */
#ifndef OAT_PROBE_H
#define OAT_PROBE_H

#include "oat.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Reads the device buffer d_buf (n_bytes, a multiple of 16, 16-byte aligned) reps times with
 * 16-byte loads (cached in L2 only) spread over every SM.  The loads feed a sum that decides
 * whether anything is written to *d_sink (one float, device memory; in practice it never is),
 * so that none of them can be dropped.  With a buffer that fits
 * in L2 and is already resident there, bytes / time is the L2 read bandwidth.  Asynchronous on
 * `stream`; allocates nothing.  Returns OAT_ERR_INVALID_ARG for a bad size or pointer.
 */
int oat_probe_read(const void *d_buf, long long n_bytes, int reps, float *d_sink, void *stream);

/*
 * The fractional sample index k~ = (|r_q - r_n| / c - t_min) / dt of Eqs. linearint and disfbp
 * (Sec. III.C) exactly as oat_fbp computes it in FP32 (from its brick-centre distance in float
 * pairs plus the node's FP32 offset), for n (node, transducer) pairs.  This is the estimate
 * before oat_fbp's double-precision resolution of values within its guard band of an integer:
 * its error against the definition must stay well inside that band.
 *   d_nodes        device, int [n][3]: (ix, iy, iz) node indices (any integers: only arithmetic)
 *   d_transducers  device, int [n]: transducer indices
 *   d_out          device, double [n]: k~ as oat_fbp holds it (integer part plus FP32 fraction,
 *                  converted exactly); NaN where the transducer index is outside 0 .. Q-1
 * Asynchronous on `stream`; allocates nothing; needs no FBP weights.  n = 0 does nothing.
 * Errors: OAT_ERR_INVALID_ARG (NULL plan, n < 0, NULL buffer with n > 0), OAT_ERR_CUDA.
 */
int oat_fbp_sample_positions(oat_plan plan, const int *d_nodes, const int *d_transducers, int n, double *d_out,
                             void *stream);

#ifdef __cplusplus
}
#endif

#endif
