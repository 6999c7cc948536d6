/*
 * oat_sph.h - C ABI of the spherical-voxel imaging model H_sph and its adjoint (Sec. II.B,
 * Eqs. basissph, coeffsph, dis_sph, p0f, ddmodelsp, sphbwd), for point transducers.
 *
 * The object is a set of uniform spheres of diameter Delta_s centred on the grid nodes r_n with
 * coefficients alpha_n (the mean of the object over each sphere), and the data are L temporal
 * frequency samples of the pressure at each transducer q:
 *
 *   u_{q,l} = p0(f_l) sum_n alpha_n exp(-j 2 pi f_l d_qn / c) / (2 pi d_qn),   d_qn = |r_q - r_n|,
 *   p0(f)  = -j (Gamma c / f) [ Delta_s / (2 c) cos(pi f Delta_s / c)
 *                               - sin(pi f Delta_s / c) / (2 pi f) ] h_e(f),
 *
 * (Gamma = beta c^2 / C_p; h_e the transducer's electric response, 1 if not given), and the adjoint
 * for real alpha and the inner product Re <u, v>:
 *
 *   alpha'_n = Re sum_q sum_l u_{q,l} conj(p0(f_l)) exp(+j 2 pi f_l d_qn / c) / (2 pi d_qn).
 *
 * The frequencies are uniformly spaced, f_l = f0 + l df (l = 0 .. L-1), all > 0.  Sums are
 * direct (every voxel, transducer and frequency).  Phases are formed in float-pair arithmetic
 * from the exact distance, so that they keep about 1e-10 cycle at any distance; exponentials
 * of consecutive frequencies come from a complex rotation started from an exact value every few
 * frequencies.  Accumulation is FP32 with compensation; p0 is applied in double precision.
 *
 * Conventions: device pointers 16-byte aligned, arrays contiguous; alpha is float32
 * [nz][ny][nx] (x fastest, the node layout of oat.h); u is complex float32 [Q][L] stored as
 * interleaved (re, im) float pairs; `stream` is a cudaStream_t passed as void* (NULL = legacy
 * default stream).  Return OAT_OK or a negative OAT_ERR_* code of oat.h (oat_last_error() has
 * the message).
 */
#ifndef OAT_SPH_H
#define OAT_SPH_H

#include "oat.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oat_sph_s *oat_sph;

/*
 * Creates the operator on `device`.  From geom it uses nx, ny, nz, spacing_mm, origin_mm,
 * n_transducers, positions_mm, c_mm_per_us and gruneisen (copied; the time-sampling fields,
 * data_dtype, apply_d and lattice_weights are ignored).  Every transducer must lie at least
 * Delta_s / 2 from every node (outside every spherical voxel).
 * 1 <= n_freq = L <= 12800 (the adjoint stages transducer rows of v in shared memory),
 * f0_mhz > 0, df_mhz >= 0 (> 0 when L > 1); eir: NULL, or a host array of
 * [L][2] doubles (re, im) of h_e(f_l), copied.
 * Allocates the transducer table, p0, a [Q][L] complex scratch of the adjoint and the forward's
 * per-slab totals (the voxels are split into slabs so that few transducers still fill the GPU;
 * [n_slab][Q][L] double pairs, at most 1 GiB).
 * Errors: OAT_ERR_INVALID_ARG (NULL, sizes, non-finite values, a transducer inside a voxel),
 *         OAT_ERR_OOM, OAT_ERR_CUDA.
 */
int oat_sph_create(const oat_geometry *geom, int n_freq, double f0_mhz, double df_mhz, const double *eir, int device,
                   oat_sph *out);

/* u = H_sph alpha: d_alpha float32 [nz][ny][nx] -> d_u complex float32 [Q][L] (overwritten).
 * Asynchronous on `stream`; allocates nothing. */
int oat_sph_project(oat_sph op, const float *d_alpha, float *d_u, void *stream);

/* alpha' = H_sph^T u: d_u complex float32 [Q][L] -> d_alpha float32 [nz][ny][nx] (overwritten).
 * Asynchronous on `stream`; allocates nothing; uses the operator's scratch, so calls on one
 * operator must not overlap (order them on one stream). */
int oat_sph_backproject(oat_sph op, const float *d_u, float *d_alpha, void *stream);

/* Frees the operator (synchronises its device).  NULL is a no-op. */
int oat_sph_destroy(oat_sph op);

#ifdef __cplusplus
}
#endif

#endif
