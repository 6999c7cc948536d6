/*
 * oat_recon.h - C ABI of the device kernels behind the penalised least-squares reconstruction
 *
 *     alpha* = argmin_{alpha >= 0}  1/2 || H alpha - u ||^2 + mu TV(alpha)
 *
 * solved with FISTA (Beck and Teboulle, 2009).  The objective is the PLS objective of
 * Sec. IV.A (Eq. PLSObjFuncInt) with a total-variation penalty in place of the quadratic
 * smoothness penalty of Sec. IV.B; the paper solves it with linear conjugate gradients and
 * names fast-converging optimisation algorithms (its reference to FISTA) as the way to fewer
 * iterations in Sec. V.  H and H^T come from oat.h; these entry points are the remaining
 * vector and proximal steps, so that one FISTA iteration runs entirely in this library's
 * kernels.  Reductions are accumulated in double precision.
 *
 * Conventions: all pointers are device pointers (16-byte aligned), arrays contiguous, float32
 * unless stated; `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 * every call only enqueues work and allocates nothing.  Return OAT_OK or OAT_ERR_INVALID_ARG /
 * OAT_ERR_CUDA (oat_last_error() has the message).
 * TV(x) = sum_n || (x_{n+e_x} - x_n, x_{n+e_y} - x_n, x_{n+e_z} - x_n) ||_2 (isotropic, forward
 * differences, zero difference across the far boundary of each axis).
 */
#ifndef OAT_RECON_H
#define OAT_RECON_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * FISTA data-space step.  With hx = H alpha_k and hx_prev = H alpha_{k-1}:
 *   r = (1 + beta) hx - beta hx_prev - u        (= H y_{k+1} - u by linearity of H)
 *   acc[0] += sum (hx - u)^2,  acc[1] += sum u^2   (double; caller zeroes acc)
 * hx_prev may equal hx (beta ignored then).  r may alias hx_prev.  n elements.
 * The measured data u are stored as u_dtype (OAT_F32, OAT_F16 or OAT_BF16, oat.h) and read
 * exactly; everything else is float32.  Returns OAT_ERR_INVALID_ARG for a bad size, dtype or
 * pointer (float pointers must be 16-byte aligned).
 */
int oat_fista_residual(long long n, const float *hx, const float *hx_prev, const void *u, int u_dtype, float beta,
                       float *r, double *acc, void *stream);

/*
 * Proximal map of lam * TV plus the constraint x >= 0 at z - step * g (the FISTA gradient
 * step fused in):  out = argmin_{x >= 0} 1/2 ||x - (z - step g)||^2 + lam TV(x),
 * computed by `iters` iterations of the fast gradient projection on the dual (Beck and
 * Teboulle, 2009, FGP).  g may be NULL (pure proximal map of z).
 * Volumes [nz][ny][nx]; work: caller-owned device scratch of 7 * nx * ny * nz floats.
 */
int oat_tv_prox(int nx, int ny, int nz, const float *z, const float *g, float step, float lam, int iters,
                float *out, float *work, void *stream);

/* y = a + beta (a - a_prev), n elements (y may alias a_prev). */
int oat_fista_momentum(long long n, const float *a, const float *a_prev, float beta, float *y, void *stream);

/* acc[0] += sum x_i y_i in double (caller zeroes acc). */
int oat_dot(long long n, const float *x, const float *y, double *acc, void *stream);

/* acc[0] += TV(x) in double (caller zeroes acc); volume [nz][ny][nx]. */
int oat_tv_value(int nx, int ny, int nz, const float *x, double *acc, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* OAT_RECON_H */
