/*
 * oat_unet.h - C ABI of the kernels of the learned warm start for the PLS-TV reconstruction:
 * a small 3-D U-Net (3 levels, 16 / 32 / 64 channels) that maps the backprojection H^T y to an
 * initial estimate.  This layer has no counterpart in the paper; it feeds x_0 to the FISTA
 * solver of oat_recon.h, which still decides the result.
 *
 * Tensors: BF16 activations, channels last x[z][y][x][c]; convolution weights BF16
 * w[tap][cout][cin], tap = (dz * 3 + dy) * 3 + dx for offsets (dz - 1, dy - 1, dx - 1), zero
 * padding; biases, gradients of weights, optimiser state and the head in FP32.  All pointers are
 * device pointers with at least 4-byte alignment; `stream` is a cudaStream_t as void*; calls
 * only enqueue work.  Return OAT_OK or OAT_ERR_INVALID_ARG / OAT_ERR_CUDA.
 */
#ifndef OAT_UNET_H
#define OAT_UNET_H

#ifdef __cplusplus
extern "C" {
#endif

/* y = act(b + conv3x3x3(x, w)) on the 5th-generation tensor cores: tcgen05.mma, BF16 in, FP32
 * accumulation in tensor memory, BF16 out; operands staged in shared memory by TMA.
 * cin a multiple of 16 up to 96, cout 16, 32, 48, 64 or 96; relu != 0 applies max(0, .); bias
 * may be NULL.  x, w and y must be 16-byte aligned (OAT_ERR_INVALID_ARG otherwise). */
int oat_conv3d_bf16(int nx, int ny, int nz, int cin, int cout, const void *x, const void *w, const float *bias, int relu,
                    void *y, void *stream);

/* Synchronous status of the tensor-core convolutions launched so far: OAT_OK, or OAT_ERR_CUDA if
 * one of them gave up waiting on its copy / MMA pipeline (a bounded wait ran out, about a second;
 * its output is then undefined).  Reading the status clears it. */
int oat_unet_check(void);

/* wf[tap][ci][co] = w[26 - tap][co][ci]: with it, oat_conv3d_bf16(g, wf) is the input gradient. */
int oat_conv3d_flip_weights(int cin, int cout, const void *w, void *wf, void *stream);

/* dw[tap][co][ci] += sum_v g[v][co] x[v + off(tap)][ci];  db[co] += sum_v g[v][co] (db may be
 * NULL).  On the tensor cores (tcgen05.mma, BF16 in, FP32 accumulation in tensor memory), the
 * voxels split over blocks whose partial sums are added in a fixed order: no floating-point atomics,
 * the same result on every run.  cin a multiple of 16 up to 96, cout a multiple of 8 up to 128;
 * x and g 16-byte aligned.  The partial sums live in a static device array of this library (8 MB on
 * every GPU that loads it): weight-gradient calls whose work overlaps on the GPU (different
 * streams) race on it; order them. */
int oat_conv3d_wgrad(int nx, int ny, int nz, int cin, int cout, const void *x, const void *g, float *dw, float *db,
                     void *stream);

/* c = a + b, n BF16 elements (FP32 add). */
int oat_add_bf16(long long n, const void *a, const void *b, void *c, void *stream);

/* g = dout * (act > 0), n elements. */
int oat_relu_grad(long long n, const void *act, const void *dout, void *g, void *stream);

/* 2x2x2 average pooling of x (input sizes nx, ny, nz, even) into y; with backward != 0, x is the
 * gradient of the pooled tensor and y receives the gradient of the input. */
int oat_avgpool2(int nx, int ny, int nz, int c, const void *x, void *y, int backward, void *stream);

/* Nearest 2x upsampling of x (sizes nx, ny, nz, c channels) into channels [c0, c0 + c) of y
 * (ctot channels); with backward != 0, x is the gradient of y (ctot channels, read at [c0, c0+c))
 * and y receives the gradient of the low-resolution tensor (c channels). */
int oat_upsample2(int nx, int ny, int nz, int c, const void *x, int ctot, int c0, void *y, int backward, void *stream);

/* dst[v][d0 + i] = src[v][s0 + i], i < c (channel concatenation and its adjoint). */
int oat_copy_channels(long long nvox, int c, const void *src, int cs, int s0, void *dst, int cd, int d0, void *stream);

/* x[v][0] = scale * v[v], x[v][1..15] = 0 (FP32 volume to the 16-channel BF16 input). */
int oat_pack_input(long long nvox, const float *v, float scale, void *x, void *stream);

/* 1x1x1 head: out[v] = b[0] + sum_c w[c] f[v][c] (FP32 out), and its gradient (dw, db accumulate). */
int oat_head(long long nvox, int c, const void *f, const float *w, const float *b, float *out, void *stream);
int oat_head_grad(long long nvox, int c, const void *f, const float *w, const float *dout, void *df, float *dw, float *db,
                  void *stream);

/* loss[0] += mean (p - t)^2 (double); grad = 2 (p - t) / n. */
int oat_mse(long long n, const float *pred, const float *target, float *grad, double *loss, void *stream);

/* Adam step (bias-corrected, step >= 1) on FP32 parameters p with gradient g and moments m, v;
 * refreshes the BF16 copy pbf16 when not NULL. */
int oat_adam(long long n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps, int step,
             void *pbf16, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* OAT_UNET_H */
