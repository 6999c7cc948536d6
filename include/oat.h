/*
 * oat.h - C ABI of the GB300 (sm_103a) projector / backprojector pair of the
 * interpolation-based discrete imaging model of three-dimensional optoacoustic tomography.
 *
 *   H   = D G         forward model, Sec. II.B: G is the discrete spherical Radon transform
 *                     of the trilinearly interpolated volume (Eq. dis_srt, Appendix), D the
 *                     temporal difference operator (Eq. dis_g2p).  Point-like transducers,
 *                     no EIR (H^e = identity).
 *   H^T = G^T D^T     its exact adjoint (Sec. II.B, "Adjoints of the system matrices").
 *
 * Every entry point is extern "C", takes plain host or device pointers and sizes, and
 * returns an int status: OAT_OK (0) or one of the negative OAT_ERR_* codes below, with a
 * human-readable message available from oat_last_error() on the calling thread.
 *
 * Layouts (all arrays contiguous, row-major, 16-byte aligned device pointers):
 *   volume  float32 [nz][ny][nx]   node (ix, iy, iz) at origin_mm + spacing_mm * (ix, iy, iz)
 *   data    [Q][K] in the plan's data_dtype (float32, float16 or bfloat16), time fastest;
 *           sample k of transducer q is at t_k = t_min_us + k / fs_mhz
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All
 * compute calls only enqueue work on that stream and return; they allocate no memory
 * (the plan owns every table and scratch buffer it needs).  Launch errors are reported by
 * the call; errors of the kernels themselves surface at the caller's next synchronisation.
 * One plan must not be used by two calls that overlap on the GPU (they share scratch).
 */
#ifndef OAT_H
#define OAT_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define OAT_OK               0
#define OAT_ERR_INVALID_ARG (-1)   /* NULL pointer, bad size, misaligned buffer, bad enum */
#define OAT_ERR_GEOMETRY    (-2)   /* geometry that the model does not admit (see below) */
#define OAT_ERR_CUDA        (-3)   /* a CUDA runtime call or a kernel launch failed      */
#define OAT_ERR_OOM         (-4)   /* device allocation failed during plan creation      */
#define OAT_ERR_UNSUPPORTED (-5)   /* valid request this build does not implement        */

/* ---- data storage types (the type of u / y; interpolation and sums are FP32) ------ */
#define OAT_F32  0
#define OAT_F16  1
#define OAT_BF16 2

/* ---- shell-lattice point weights (oat_geometry.lattice_weights) ------------------- */
#define OAT_LATTICE_UNIFORM    0
#define OAT_LATTICE_EXACT_AREA 1

typedef struct oat_plan_s *oat_plan;

/*
 * Measurement geometry and grid (Sec. III.A).  Everything is copied at plan creation.
 *   nx, ny, nz          node counts, each >= 1, nx*ny*nz < 2^31
 *   spacing_mm          grid spacing Delta_s > 0; also the lattice spacing on the shells
 *   origin_mm           position of node (0,0,0)
 *   n_transducers       Q >= 1
 *   positions_mm        HOST pointer to [Q][3] doubles: point-like transducer positions; the
 *                       measurement sphere and the support sphere are centred at (0,0,0)
 *   n_samples           K >= 1 (>= 3 when apply_d)
 *   fs_mhz              sampling rate, Delta_t = 1 / fs_mhz microseconds
 *   t_min_us            time of sample 0 (>= 0)
 *   c_mm_per_us         speed of sound c_0 > 0
 *   support_radius_mm   R, radius of the origin-centred sphere containing the object; <= 0
 *                       selects the sphere enclosing the node cuboid grown by one spacing
 *   gruneisen           Gamma = beta c^2 / C_p (finite), scales D; D = Gamma/(8 pi c^2 dt^2)(...)
 *   data_dtype          OAT_F32, OAT_F16 or OAT_BF16: storage of u (project) and y (backproject)
 *   apply_d             1: H = D G (the model); 0: G only (the spherical Radon transform)
 *   lattice_weights     weight of each shell-lattice point in G (Eq. dis_srt):
 *                       OAT_LATTICE_UNIFORM (0): Delta_s^2 for every point (the Appendix);
 *                       OAT_LATTICE_EXACT_AREA (1): the area of its ring's strip of the shell
 *                       shared by the ring's N_j points, Delta_s 2 pi rho sin(theta_i) / N_j,
 *                       which removes the bias of rounding 2 pi / dphi_i down to N_j.  The
 *                       lattice itself is the same; G^T uses the same weights.
 */
typedef struct {
    int nx, ny, nz;
    double spacing_mm;
    double origin_mm[3];
    int n_transducers;
    const double *positions_mm;
    int n_samples;
    double fs_mhz;
    double t_min_us;
    double c_mm_per_us;
    double support_radius_mm;
    double gruneisen;
    int data_dtype;
    int apply_d;
    int lattice_weights;
} oat_geometry;

/* Sizes and counts of a plan (oat_plan_query). */
typedef struct {
    long long n_radius_classes;   /* distinct |r_q| values; lattice tables are per class   */
    long long n_rings;            /* ring records (class, k, i) in the lattice tables       */
    long long points_ball;        /* lattice points of one application of G (all q, k)      */
    long long points_grid;        /* of those, points with a stencil node in the grid, i.e.
                                     the interpolations that can be non-zero; -1 unless the
                                     query asked for the count                              */
    long long table_bytes;        /* device bytes of geometry / lattice tables              */
    long long scratch_bytes;      /* device bytes of scratch owned by the plan              */
    long long work_items;         /* thread-block work items of one projection              */
} oat_stats;

/*
 * Create a plan on CUDA device `device` (the caller's current device is restored).
 * Builds, in FP64 on the host, the local frame of every transducer and the shell lattice of
 * every (radius class, sample): theta_i = i dtheta, i < N_i = floor(theta_max / dtheta),
 * phi_j = j dphi_i, j < N_j = floor(2 pi / dphi_i), dtheta = Delta_s / (c t_k),
 * dphi_i = Delta_s / (c t_k sin theta_i), theta_max from the support sphere (Appendix,
 * Eqs. srtlocal and srtdislocal); then uploads them and allocates the plan's scratch.
 * Errors: OAT_ERR_INVALID_ARG (NULL, sizes, enums, non-finite numbers),
 *         OAT_ERR_GEOMETRY (a transducer at |r_q| <= R, or no lattice point at all),
 *         OAT_ERR_OOM, OAT_ERR_CUDA.  On error *out is set to NULL.
 */
int oat_plan_create(const oat_geometry *geom, int device, oat_plan *out);

/* Release a plan and its device memory (after the work using it has completed).
 * NULL is accepted. */
int oat_plan_destroy(oat_plan plan);

/*
 * u = H alpha (or G alpha when apply_d = 0)  -- Eqs. dis_srt and dis_g2p.
 *   d_vol   device, float32 [nz][ny][nx], read only
 *   d_data  device, [Q][K] of data_dtype, fully overwritten
 * D rows 0 and K-1 are zero; a D term whose tau_k = t_k / dt is <= 0 is zero.  The lattice
 * points carry the plan's lattice_weights; with a transducer response set (oat_plan_set_eir)
 * the result is H^e D G alpha (H^e G alpha without D).
 * Errors: OAT_ERR_INVALID_ARG (NULL plan or pointer, pointer not 16-byte aligned),
 *         OAT_ERR_CUDA (launch failure).
 */
int oat_project(oat_plan plan, const float *d_vol, void *d_data, void *stream);

/*
 * alpha' = H^T y (or G^T y when apply_d = 0)  -- the adjoints of Sec. II.B.  Exact transpose
 * of oat_project: the same FP32 lattice points, the same interpolation and lattice weights; D^T
 * is the exact transpose of D including its zero boundary rows; with a transducer response set,
 * H^e^T is applied first.  Computed brick by brick: each brick of
 * voxels sums the weighted lattice points that fall in its cells as exact fixed-point integers,
 * so there are no floating-point atomics and the result does not depend on execution order.
 * The fixed-point unit adapts to the data: transducers are taken in passes whose largest
 * |D^T y| lie within a factor 2^8 of each other, each pass rounds its contributions to 30 bits
 * of its own largest |D^T y| and folds, exactly, into a finer 64-bit per-voxel unit; a spike or
 * an outlier transducer row therefore costs no precision in the other rows.
 *   d_data  device, [Q][K] of data_dtype, read only
 *   d_vol   device, float32 [nz][ny][nx], fully overwritten
 * Errors: as oat_project.
 */
int oat_backproject(oat_plan plan, const void *d_data, float *d_vol, void *stream);

/*
 * alpha' = H^T y exactly as oat_backproject, for callers that cannot allocate device memory at
 * the time of the call: the backprojector's per-voxel scratch (a 64-bit accumulator per voxel and
 * one max|D^T y| word) is taken from an array of this library in static device memory instead of
 * the plan's scratch, and the call allocates nothing (no cudaMalloc or cudaFree, no allocating
 * library call).  The per-transducer maxima of |D^T y| still use the plan's own scratch, which
 * oat_plan_create allocated.  This entry point has no counterpart in the paper.
 *   Limit: nx * ny * nz <= 2,097,152 voxels (the array holds 16 MiB + 256 bytes on every GPU
 *          that loads the library, until the process exits); larger volumes return
 *          OAT_ERR_INVALID_ARG.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *   that device current and keeps it for the life of the process; make that first call before
 *   any stream capture.  The kept address does not survive cudaDeviceReset on that device: do
 *   not call this entry point again in a process that has reset the device.
 *   All calls share the array and each clears what it needs at its start, so two calls whose
 *   work overlaps on the GPU (on different streams, or from different plans) race and give wrong
 *   results; order them.
 * Arguments, layouts and other errors as oat_backproject.
 */
int oat_backproject_noalloc(oat_plan plan, const void *d_data, float *d_vol, void *stream);

/*
 * Filtered backprojection (Sec. III.C, Eqs. linearint and disfbp): for every node n,
 *   alpha_n = -1 / (pi Gamma c dt) * sum_q w_q { 0.5 (p_{q,k+1} - p_{q,k})
 *                                   + [p_{q,k} + (k~ - k)(p_{q,k+1} - p_{q,k})] / (k~ + t_min/dt) },
 *   k~ = (|r_q - r_n| / c - t_min) / dt, k = floor(k~)
 * (the same sum as the paper's Eq. disfbp), samples outside 0 .. K-1 counting as zero.
 * The sum is discontinuous where k~ crosses an integer; the kernel reads the pair k, k + 1 of the
 * exact k~: k~ is formed in FP32 (good to about 2e-6 grid units of distance) and recomputed in
 * double precision wherever it lies within 1e-5 (ds / (c dt) + 1) samples of an integer.
 *
 * oat_plan_set_fbp_weights: w_q, one per transducer (host array of n_transducers doubles; for a
 *   spherical scan, the patch area over the sphere radius, R^s dtheta dphi sin theta_q).  Copied
 *   into the plan (synchronous); required before oat_fbp.
 * oat_fbp: d_data [Q][K] in the plan's data dtype -> d_vol [nz][ny][nx] float32 (overwritten);
 *   asynchronous on `stream`, allocates nothing.  Both 16-byte aligned.
 * Errors: OAT_ERR_INVALID_ARG (NULL, misaligned, non-finite weight, weights not set),
 *         OAT_ERR_CUDA.
 */
int oat_plan_set_fbp_weights(oat_plan plan, const double *weights);
int oat_fbp(oat_plan plan, const void *d_data, float *d_vol, void *stream);

/*
 * Transducer response (Sec. II.B, Eq. EIR): the full model H = H^e D G, with
 *   [H^e p]_{q,k} = sum_{kappa=0}^{K-1} h_{k-1-kappa} p_{q,kappa},
 *   h_m = dt h^e(m dt) for m = first_index .. first_index + n_taps - 1, zero elsewhere,
 * and its adjoint H^T = G^T D^T H^e^T with [H^e^T u]_{q,k} = sum_kappa h_{kappa-1-k} u_{q,kappa}
 * (sums over the record 0 .. K-1 only).  Once set, oat_project returns H^e D G alpha (D G alpha
 * kept in double precision in shared memory, the convolution in double, one rounding to the data
 * dtype) and oat_backproject / oat_backproject_noalloc compute z = H^e^T y in double from the
 * stored y, rounded once to float32 into a plan-owned [Q][K] buffer that the voxel gather reads.
 *
 * oat_plan_set_eir: h host array of n_taps doubles (copied; synchronous); n_taps = 0 removes the
 *   response (h may then be NULL).  The first call allocates the float32 [Q][K] buffer
 *   (Q K 4 bytes, counted in oat_stats.scratch_bytes), kept until oat_plan_destroy; later calls
 *   allocate only the tap array.  Calls must not overlap with the plan's work in flight.
 *   With a response set, oat_backproject / oat_backproject_noalloc on one plan share that
 *   buffer: order them (one stream).
 * Errors: OAT_ERR_INVALID_ARG (NULL plan, n_taps < 0, NULL h with n_taps > 0, non-finite tap,
 *         |first_index| > 2^30, (n_samples + n_taps) doubles above a block's shared memory),
 *         OAT_ERR_OOM, OAT_ERR_CUDA.
 */
int oat_plan_set_eir(oat_plan plan, const double *h, int n_taps, int first_index);

/*
 * Fill *stats.  With count_grid_points != 0 the call also counts, on the device and
 * synchronously (on the legacy default stream), the lattice points whose interpolation
 * stencil touches the grid, the unit of work of the throughput metric.
 * Errors: OAT_ERR_INVALID_ARG, OAT_ERR_CUDA.
 */
int oat_plan_query(oat_plan plan, int count_grid_points, oat_stats *stats);

/*
 * Kernel timing for measurement.  With enable != 0 every later oat_project and
 * oat_backproject records a pair of CUDA events on the caller's stream around its main
 * kernel (the shell gather of G, the voxel gather of G^T; oat_fbp likewise).
 * oat_plan_kernel_time() synchronises on those events and returns the summed milliseconds and
 * the number of launches for which = 0 (G), 1 (G^T) or 2 (FBP) since the last reset
 * (reset != 0 clears them).
 * At most 4096 launches are recorded per kernel between resets; later ones are not timed.
 * Errors: OAT_ERR_INVALID_ARG, OAT_ERR_CUDA.
 */
int oat_plan_set_profiling(oat_plan plan, int enable);
int oat_plan_kernel_time(oat_plan plan, int which, int reset, double *ms, long long *launches);

/* Message of the last failing call on this thread ("" if none). */
const char *oat_last_error(void);

/* ABI version (major * 10000 + minor * 100 + patch). */
int oat_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OAT_H */
