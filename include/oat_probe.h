/*
 * Memory-bandwidth probe of liboat.so, used by the benchmark to measure the on-chip roofline it
 * reports (the L2 read bandwidth is not among the measured peaks).
 */
#ifndef OAT_PROBE_H
#define OAT_PROBE_H

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

#ifdef __cplusplus
}
#endif

#endif
