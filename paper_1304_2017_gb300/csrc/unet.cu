// Kernels of the learned warm start: a small 3-D U-Net on BF16 activations (include/oat_unet.h).
//
// Activations are BF16, channels last: x[z][y][x][c].  Convolution weights are BF16
// w[tap][cout][cin], tap = (dz * 3 + dy) * 3 + dx for offsets (dz - 1, dy - 1, dx - 1), zero
// padding ('same').
//
// The convolution itself (oat_conv3d_bf16) runs on the 5th-generation tensor cores in
// conv_tc.cu.  The input gradient of a 'same' 3x3x3 convolution is the same convolution of the
// output gradient with the kernel flipped in space and transposed in channels, so the same kernel
// serves the backward pass (k_flip_weights builds that kernel).
// The weight and bias gradients (oat_conv3d_wgrad) also run on the tensor cores (conv_tc.cu), with a
// fixed-order reduction over voxel splits.
#include <cuda_bf16.h>

#include <cmath>
#include <string>

#include "../../include/oat_unet.h"
#include "oat_internal.h"

namespace oat {

typedef __nv_bfloat16 bf16;

// wf[tap][ci][co] = w[26 - tap][co][ci]: kernel of the input gradient
__global__ void k_flip_weights(int cin, int cout, const bf16 *__restrict__ w, bf16 *__restrict__ wf) {
    const int n = 27 * cin * cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int co = i % cout, ci = (i / cout) % cin, tap = i / (cout * cin);
        wf[i] = w[((size_t)(26 - tap) * cout + co) * cin + ci];
    }
}

// c = a + b (BF16, FP32 add)
__global__ void k_add_bf16(long long n, const bf16 *__restrict__ a, const bf16 *__restrict__ b, bf16 *c) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c[i] = __float2bfloat16(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

// g = dout * (act > 0)
__global__ void k_relu_grad(long long n, const bf16 *__restrict__ act, const bf16 *__restrict__ dout, bf16 *g) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        g[i] = __bfloat162float(act[i]) > 0.f ? dout[i] : __float2bfloat16(0.f);
}

// 2x2x2 average pooling (channels last); nx, ny, nz of the input, even
__global__ void k_avgpool2(int nx, int ny, int nz, int c, const bf16 *__restrict__ x, bf16 *__restrict__ y) {
    const int mx = nx / 2, my = ny / 2, mz = nz / 2;
    const long long n = (long long)mx * my * mz * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        const long long v = i / c;
        const int xx = (int)(v % mx), yy = (int)((v / mx) % my), zz = (int)(v / ((long long)mx * my));
        float s = 0.f;
        for (int d = 0; d < 8; ++d)
            s += __bfloat162float(x[((((long long)(2 * zz + (d >> 2)) * ny + 2 * yy + ((d >> 1) & 1)) * nx + 2 * xx + (d & 1))) * c + ch]);
        y[i] = __float2bfloat16(0.125f * s);
    }
}

// adjoint of avgpool2: dx = dy / 8 spread over the 2x2x2 block
__global__ void k_avgpool2_grad(int nx, int ny, int nz, int c, const bf16 *__restrict__ dy, bf16 *__restrict__ dx) {
    const long long n = (long long)nx * ny * nz * c;
    const int mx = nx / 2, my = ny / 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        const long long v = i / c;
        const int xx = (int)(v % nx), yy = (int)((v / nx) % ny), zz = (int)(v / ((long long)nx * ny));
        dx[i] = __float2bfloat16(0.125f * __bfloat162float(dy[(((long long)(zz / 2) * my + yy / 2) * mx + xx / 2) * c + ch]));
    }
}

// nearest 2x upsampling of x (nx, ny, nz: input sizes) into channels [c0, c0 + c) of y (ctot channels)
__global__ void k_upsample2(int nx, int ny, int nz, int c, const bf16 *__restrict__ x, int ctot, int c0, bf16 *__restrict__ y) {
    const int ox = 2 * nx, oy = 2 * ny, oz = 2 * nz;
    const long long n = (long long)ox * oy * oz * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        const long long v = i / c;
        const int xx = (int)(v % ox), yy = (int)((v / ox) % oy), zz = (int)(v / ((long long)ox * oy));
        y[v * ctot + c0 + ch] = x[(((long long)(zz / 2) * ny + yy / 2) * nx + xx / 2) * c + ch];
    }
}

// adjoint of upsample2: dx = sum over the 2x2x2 children of channels [c0, c0 + c) of dy
__global__ void k_upsample2_grad(int nx, int ny, int nz, int c, const bf16 *__restrict__ dy, int ctot, int c0,
                                 bf16 *__restrict__ dx) {
    const long long n = (long long)nx * ny * nz * c;
    const int ox = 2 * nx, oy = 2 * ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        const long long v = i / c;
        const int xx = (int)(v % nx), yy = (int)((v / nx) % ny), zz = (int)(v / ((long long)nx * ny));
        float s = 0.f;
        for (int d = 0; d < 8; ++d)
            s += __bfloat162float(dy[((((long long)(2 * zz + (d >> 2)) * oy + 2 * yy + ((d >> 1) & 1)) * ox + 2 * xx + (d & 1))) * ctot + c0 + ch]);
        dx[i] = __float2bfloat16(s);
    }
}

// copy channels [s0, s0 + c) of src (cs channels) to channels [d0, d0 + c) of dst (cd channels)
__global__ void k_copy_channels(long long nvox, int c, const bf16 *__restrict__ src, int cs, int s0, bf16 *__restrict__ dst,
                                int cd, int d0) {
    const long long n = nvox * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / c;
        const int ch = (int)(i % c);
        dst[v * cd + d0 + ch] = src[v * cs + s0 + ch];
    }
}

// pack a float32 volume scaled by s into channel 0 of a 16-channel BF16 tensor (others zero)
__global__ void k_pack_input(long long nvox, const float *__restrict__ v, float s, bf16 *__restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvox * 16; i += (long long)gridDim.x * blockDim.x)
        x[i] = (i % 16 == 0) ? __float2bfloat16(v[i / 16] * s) : __float2bfloat16(0.f);
}

// 1x1x1 head: out[v] = b + sum_c w[c] feat[v][c] (float32 out)
__global__ void k_head(long long nvox, int c, const bf16 *__restrict__ f, const float *__restrict__ w, const float *__restrict__ b,
                       float *out) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        float s = b[0];
        for (int ch = 0; ch < c; ++ch) s = fmaf(w[ch], __bfloat162float(f[v * c + ch]), s);
        out[v] = s;
    }
}

// head backward: df[v][c] = dout[v] w[c]; dw[c] += sum_v dout[v] f[v][c]; db += sum dout
__global__ void k_head_grad(long long nvox, int c, const bf16 *__restrict__ f, const float *__restrict__ w,
                            const float *__restrict__ dout, bf16 *df, float *dw, float *db) {
    float acc[64];
    for (int ch = 0; ch < c; ++ch) acc[ch] = 0.f;
    float bacc = 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        const float d = dout[v];
        bacc += d;
        for (int ch = 0; ch < c; ++ch) {
            acc[ch] = fmaf(d, __bfloat162float(f[v * c + ch]), acc[ch]);
            df[v * c + ch] = __float2bfloat16(d * w[ch]);
        }
    }
    for (int ch = 0; ch < c; ++ch) {
        float s = acc[ch];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0 && s != 0.f) atomicAdd(dw + ch, s);
    }
    for (int o = 16; o > 0; o >>= 1) bacc += __shfl_xor_sync(0xffffffffu, bacc, o);
    if ((threadIdx.x & 31) == 0 && bacc != 0.f) atomicAdd(db, bacc);
}

// loss += sum (p - t)^2 / n (double); grad = 2 (p - t) / n
__global__ void k_mse(long long n, const float *__restrict__ p, const float *__restrict__ t, float *grad, double *loss) {
    double s = 0.0;
    const float inv = 2.f / (float)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = p[i] - t[i];
        s += (double)d * d;
        grad[i] = inv * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(loss, s / (double)n);
}

// Adam on FP32 master weights; refreshes the BF16 copy (if any)
__global__ void k_adam(long long n, float *p, const float *__restrict__ g, float *m, float *v, float lr, float b1, float b2,
                       float eps, float c1, float c2, bf16 *pb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi; v[i] = vi;
        const float w = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = w;
        if (pb) pb[i] = __float2bfloat16(w);
    }
}

static unsigned grid1(long long n) {
    return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 16LL * current_sm_count()));
}

static int launched(const char *what) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace oat

using namespace oat;

extern "C" {

int oat_conv3d_bf16(int nx, int ny, int nz, int cin, int cout, const void *x, const void *w, const float *bias, int relu,
                    void *y, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || cin < 16 || cin > 96 || cin % 16 || !x || !w || !y ||
        (cout != 16 && cout != 32 && cout != 48 && cout != 64 && cout != 96))
        return set_error(OAT_ERR_INVALID_ARG, "oat_conv3d_bf16: need cin a multiple of 16 up to 96, cout in {16, 32, 48, 64, 96}");
    return launch_conv3d_tc(nx, ny, nz, cin, cout, x, w, bias, relu, y, (cudaStream_t)stream);
}

int oat_unet_check(void) { return conv_tc_check(); }

int oat_conv3d_flip_weights(int cin, int cout, const void *w, void *wf, void *stream) {
    if (cin < 1 || cout < 1 || !w || !wf) return set_error(OAT_ERR_INVALID_ARG, "oat_conv3d_flip_weights: bad arguments");
    k_flip_weights<<<grid1(27LL * cin * cout), 256, 0, (cudaStream_t)stream>>>(cin, cout, (const bf16 *)w, (bf16 *)wf);
    return launched("oat_conv3d_flip_weights");
}

int oat_conv3d_wgrad(int nx, int ny, int nz, int cin, int cout, const void *x, const void *g, float *dw, float *db,
                     void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || cin < 16 || cin > 96 || cin % 16 || cout < 8 || cout > 128 || cout % 8 || !x ||
        !g || !dw)
        return set_error(OAT_ERR_INVALID_ARG, "oat_conv3d_wgrad: need cin a multiple of 16 up to 96, cout a multiple of 8 up to 128");
    return launch_wgrad_tc(nx, ny, nz, cin, cout, x, g, dw, db, (cudaStream_t)stream);
}

int oat_add_bf16(long long n, const void *a, const void *b, void *c, void *stream) {
    if (n < 0 || !a || !b || !c) return set_error(OAT_ERR_INVALID_ARG, "oat_add_bf16: bad arguments");
    k_add_bf16<<<grid1(n), 256, 0, (cudaStream_t)stream>>>(n, (const bf16 *)a, (const bf16 *)b, (bf16 *)c);
    return launched("oat_add_bf16");
}

int oat_relu_grad(long long n, const void *act, const void *dout, void *g, void *stream) {
    if (n < 0 || !act || !dout || !g) return set_error(OAT_ERR_INVALID_ARG, "oat_relu_grad: bad arguments");
    k_relu_grad<<<grid1(n), 256, 0, (cudaStream_t)stream>>>(n, (const bf16 *)act, (const bf16 *)dout, (bf16 *)g);
    return launched("oat_relu_grad");
}

int oat_avgpool2(int nx, int ny, int nz, int c, const void *x, void *y, int backward, void *stream) {
    if (nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 || nz % 2 || c < 1 || !x || !y)
        return set_error(OAT_ERR_INVALID_ARG, "oat_avgpool2: even sizes required");
    cudaStream_t s = (cudaStream_t)stream;
    if (!backward) k_avgpool2<<<grid1((long long)nx * ny * nz * c / 8), 256, 0, s>>>(nx, ny, nz, c, (const bf16 *)x, (bf16 *)y);
    else k_avgpool2_grad<<<grid1((long long)nx * ny * nz * c), 256, 0, s>>>(nx, ny, nz, c, (const bf16 *)x, (bf16 *)y);
    return launched("oat_avgpool2");
}

int oat_upsample2(int nx, int ny, int nz, int c, const void *x, int ctot, int c0, void *y, int backward, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || c < 1 || c0 < 0 || c0 + c > ctot || !x || !y)
        return set_error(OAT_ERR_INVALID_ARG, "oat_upsample2: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (!backward) k_upsample2<<<grid1(8LL * nx * ny * nz * c), 256, 0, s>>>(nx, ny, nz, c, (const bf16 *)x, ctot, c0, (bf16 *)y);
    else k_upsample2_grad<<<grid1((long long)nx * ny * nz * c), 256, 0, s>>>(nx, ny, nz, c, (const bf16 *)x, ctot, c0, (bf16 *)y);
    return launched("oat_upsample2");
}

int oat_copy_channels(long long nvox, int c, const void *src, int cs, int s0, void *dst, int cd, int d0, void *stream) {
    if (nvox < 0 || c < 1 || s0 + c > cs || d0 + c > cd || !src || !dst) return set_error(OAT_ERR_INVALID_ARG, "oat_copy_channels");
    k_copy_channels<<<grid1(nvox * c), 256, 0, (cudaStream_t)stream>>>(nvox, c, (const bf16 *)src, cs, s0, (bf16 *)dst, cd, d0);
    return launched("oat_copy_channels");
}

int oat_pack_input(long long nvox, const float *v, float scale, void *x, void *stream) {
    if (nvox < 0 || !v || !x) return set_error(OAT_ERR_INVALID_ARG, "oat_pack_input");
    k_pack_input<<<grid1(nvox * 16), 256, 0, (cudaStream_t)stream>>>(nvox, v, scale, (bf16 *)x);
    return launched("oat_pack_input");
}

int oat_head(long long nvox, int c, const void *f, const float *w, const float *b, float *out, void *stream) {
    if (nvox < 0 || c < 1 || c > 64 || !f || !w || !b || !out) return set_error(OAT_ERR_INVALID_ARG, "oat_head");
    k_head<<<grid1(nvox), 256, 0, (cudaStream_t)stream>>>(nvox, c, (const bf16 *)f, w, b, out);
    return launched("oat_head");
}

int oat_head_grad(long long nvox, int c, const void *f, const float *w, const float *dout, void *df, float *dw, float *db,
                  void *stream) {
    if (nvox < 0 || c < 1 || c > 64 || !f || !w || !dout || !df || !dw || !db) return set_error(OAT_ERR_INVALID_ARG, "oat_head_grad");
    k_head_grad<<<grid1(nvox), 256, 0, (cudaStream_t)stream>>>(nvox, c, (const bf16 *)f, w, dout, (bf16 *)df, dw, db);
    return launched("oat_head_grad");
}

int oat_mse(long long n, const float *pred, const float *target, float *grad, double *loss, void *stream) {
    if (n < 1 || !pred || !target || !grad || !loss) return set_error(OAT_ERR_INVALID_ARG, "oat_mse");
    k_mse<<<grid1(n), 256, 0, (cudaStream_t)stream>>>(n, pred, target, grad, loss);
    return launched("oat_mse");
}

int oat_adam(long long n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps, int step,
             void *pbf16, void *stream) {
    if (n < 0 || !p || !g || !m || !v || step < 1) return set_error(OAT_ERR_INVALID_ARG, "oat_adam");
    const float c1 = 1.f / (1.f - powf(b1, (float)step)), c2 = 1.f / (1.f - powf(b2, (float)step));
    k_adam<<<grid1(n), 256, 0, (cudaStream_t)stream>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2, (bf16 *)pbf16);
    return launched("oat_adam");
}

}  // extern "C"
