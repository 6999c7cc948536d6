// Vector and proximal kernels of the FISTA-TV reconstruction (include/oat_recon.h).
//
// TV prox with non-negativity by the fast gradient projection on the dual problem (Beck and
// Teboulle, 2009): for the dual field p (three components per voxel, |p_n| <= 1),
//   x(p)  = max(0, z - lam grad^T p)
//   p    <- Proj_{|.|<=1}( r + grad x(r) / (12 lam) )        (12 >= ||grad||^2 in 3-D)
//   r    <- p_new + (t_k - 1)/t_{k+1} (p_new - p_old)
// with grad the forward difference (zero across the far boundary) and
//   (grad^T r)_n = sum_d ( [n_d > 0] r_d[n - e_d] - [n_d < N_d - 1] r_d[n] ).
// Reductions: warp shuffles, a shared-memory block sum, one double atomic per block.
#include <cmath>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/oat_recon.h"
#include "oat_internal.h"

namespace oat {

constexpr int kRThreads = 256;

__device__ __forceinline__ void block_add(double v, double *out) {
    __shared__ double red[kRThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < kRThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && v != 0.0) atomicAdd(out, v);
    }
}

template <int DT>
__device__ __forceinline__ float load_u(const void *u, long long i) {
    if (DT == OAT_F32) return ((const float *)u)[i];
    if (DT == OAT_F16) return __half2float(((const __half *)u)[i]);
    return __bfloat162float(((const __nv_bfloat16 *)u)[i]);
}

template <int DT>
__global__ void __launch_bounds__(kRThreads) k_fista_residual(long long n, const float *__restrict__ hx,
                                                              const float *__restrict__ hp, const void *__restrict__ u,
                                                              float beta, float *r, double *acc) {
    double s0 = 0.0, s1 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float h = hx[i], uu = load_u<DT>(u, i);
        const float prev = hp[i];
        const double d = (double)h - (double)uu;
        s0 += d * d;
        s1 += (double)uu * uu;
        r[i] = fmaf(beta, h - prev, h) - uu;
    }
    block_add(s0, acc);
    block_add(s1, acc + 1);
}

__global__ void __launch_bounds__(kRThreads) k_dot(long long n, const float *__restrict__ x, const float *__restrict__ y,
                                                   double *acc) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += (double)x[i] * (double)y[i];
    block_add(s, acc);
}

__global__ void k_momentum(long long n, const float *__restrict__ a, const float *ap, float beta, float *y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = a[i];
        y[i] = fmaf(beta, v - ap[i], v);
    }
}

struct Vol {
    int nx, ny, nz;
    long long N;
};

// x_n = max(0, z_n - step g_n - lam (grad^T q)_n)
__global__ void k_tv_primal(Vol v, const float *__restrict__ z, const float *__restrict__ g, float step, float lam,
                            const float *__restrict__ q, float *__restrict__ x) {
    const float *qx = q, *qy = q + v.N, *qz = q + 2 * v.N;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < v.N; n += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(n % v.nx), iy = (int)((n / v.nx) % v.ny), iz = (int)(n / ((long long)v.nx * v.ny));
        float dt = 0.f;
        if (ix > 0) dt += qx[n - 1];
        if (ix < v.nx - 1) dt -= qx[n];
        if (iy > 0) dt += qy[n - v.nx];
        if (iy < v.ny - 1) dt -= qy[n];
        if (iz > 0) dt += qz[n - (long long)v.nx * v.ny];
        if (iz < v.nz - 1) dt -= qz[n];
        float zz = z[n];
        if (g) zz = fmaf(-step, g[n], zz);
        x[n] = fmaxf(0.f, fmaf(-lam, dt, zz));
    }
}

// p <- Proj(r + grad x / (12 lam)); r <- p + mom (p - p_old)
__global__ void k_tv_dual(Vol v, const float *__restrict__ x, float inv12lam, float mom, float *p, float *r) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < v.N; n += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(n % v.nx), iy = (int)((n / v.nx) % v.ny), iz = (int)(n / ((long long)v.nx * v.ny));
        const float xc = x[n];
        const float gx = ix < v.nx - 1 ? x[n + 1] - xc : 0.f;
        const float gy = iy < v.ny - 1 ? x[n + v.nx] - xc : 0.f;
        const float gz = iz < v.nz - 1 ? x[n + (long long)v.nx * v.ny] - xc : 0.f;
        float a = fmaf(inv12lam, gx, r[n]), b = fmaf(inv12lam, gy, r[n + v.N]), c = fmaf(inv12lam, gz, r[n + 2 * v.N]);
        const float nrm = sqrtf(a * a + b * b + c * c);
        if (nrm > 1.f) { const float s = 1.f / nrm; a *= s; b *= s; c *= s; }
        const float pa = p[n], pb = p[n + v.N], pc = p[n + 2 * v.N];
        p[n] = a; p[n + v.N] = b; p[n + 2 * v.N] = c;
        r[n] = fmaf(mom, a - pa, a); r[n + v.N] = fmaf(mom, b - pb, b); r[n + 2 * v.N] = fmaf(mom, c - pc, c);
    }
}

__global__ void __launch_bounds__(kRThreads) k_tv_value(Vol v, const float *__restrict__ x, double *acc) {
    double s = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < v.N; n += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(n % v.nx), iy = (int)((n / v.nx) % v.ny), iz = (int)(n / ((long long)v.nx * v.ny));
        const float xc = x[n];
        const float gx = ix < v.nx - 1 ? x[n + 1] - xc : 0.f;
        const float gy = iy < v.ny - 1 ? x[n + v.nx] - xc : 0.f;
        const float gz = iz < v.nz - 1 ? x[n + (long long)v.nx * v.ny] - xc : 0.f;
        s += sqrt((double)gx * gx + (double)gy * gy + (double)gz * gz);
    }
    block_add(s, acc);
}

static unsigned grid_for(long long n) {
    return (unsigned)std::max<long long>(1, std::min<long long>((n + kRThreads - 1) / kRThreads, 8LL * current_sm_count()));
}

static bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace oat

using namespace oat;

extern "C" {

int oat_fista_residual(long long n, const float *hx, const float *hx_prev, const void *u, int u_dtype, float beta,
                       float *r, double *acc, void *stream) {
    if (n < 0 || !hx || !hx_prev || !u || !r || !acc || !al16(hx) || !al16(hx_prev) || !al16(u) || !al16(r) ||
        (u_dtype != OAT_F32 && u_dtype != OAT_F16 && u_dtype != OAT_BF16))
        return set_error(OAT_ERR_INVALID_ARG, "oat_fista_residual: bad size, dtype or pointer");
    if (n == 0) return OAT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (u_dtype == OAT_F32) k_fista_residual<OAT_F32><<<grid_for(n), kRThreads, 0, s>>>(n, hx, hx_prev, u, beta, r, acc);
    else if (u_dtype == OAT_F16) k_fista_residual<OAT_F16><<<grid_for(n), kRThreads, 0, s>>>(n, hx, hx_prev, u, beta, r, acc);
    else k_fista_residual<OAT_BF16><<<grid_for(n), kRThreads, 0, s>>>(n, hx, hx_prev, u, beta, r, acc);
    return check_launch("oat_fista_residual");
}

int oat_dot(long long n, const float *x, const float *y, double *acc, void *stream) {
    if (n < 0 || !x || !y || !acc) return set_error(OAT_ERR_INVALID_ARG, "oat_dot: bad size or pointer");
    if (n == 0) return OAT_OK;
    k_dot<<<grid_for(n), kRThreads, 0, (cudaStream_t)stream>>>(n, x, y, acc);
    return check_launch("oat_dot");
}

int oat_fista_momentum(long long n, const float *a, const float *a_prev, float beta, float *y, void *stream) {
    if (n < 0 || !a || !a_prev || !y) return set_error(OAT_ERR_INVALID_ARG, "oat_fista_momentum: bad size or pointer");
    if (n == 0) return OAT_OK;
    k_momentum<<<grid_for(n), kRThreads, 0, (cudaStream_t)stream>>>(n, a, a_prev, beta, y);
    return check_launch("oat_fista_momentum");
}

int oat_tv_prox(int nx, int ny, int nz, const float *z, const float *g, float step, float lam, int iters,
                float *out, float *work, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || iters < 0 || !z || !out || !work || !(lam >= 0.f) || !std::isfinite(step))
        return set_error(OAT_ERR_INVALID_ARG, "oat_tv_prox: bad size, weight or pointer");
    Vol v{nx, ny, nz, (long long)nx * ny * nz};
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = grid_for(v.N);
    if (lam == 0.f || iters == 0) {   // projection onto x >= 0 of the gradient step only
        cudaMemsetAsync(work, 0, sizeof(float) * 3 * v.N, s);
        k_tv_primal<<<grid, kRThreads, 0, s>>>(v, z, g, step, 0.f, work, out);
        return check_launch("oat_tv_prox");
    }
    float *p = work, *r = work + 3 * v.N, *x = work + 6 * v.N;
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(float) * 6 * v.N, s);
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_tv_prox: ") + cudaGetErrorString(e));
    double t = 1.0;
    const float inv = 1.f / (12.f * lam);
    for (int it = 0; it < iters; ++it) {
        k_tv_primal<<<grid, kRThreads, 0, s>>>(v, z, g, step, lam, r, x);
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        k_tv_dual<<<grid, kRThreads, 0, s>>>(v, x, inv, (float)((t - 1.0) / tn), p, r);
        t = tn;
    }
    k_tv_primal<<<grid, kRThreads, 0, s>>>(v, z, g, step, lam, p, out);
    return check_launch("oat_tv_prox");
}

int oat_tv_value(int nx, int ny, int nz, const float *x, double *acc, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !x || !acc) return set_error(OAT_ERR_INVALID_ARG, "oat_tv_value: bad size or pointer");
    Vol v{nx, ny, nz, (long long)nx * ny * nz};
    k_tv_value<<<grid_for(v.N), kRThreads, 0, (cudaStream_t)stream>>>(v, x, acc);
    return check_launch("oat_tv_value");
}

}  // extern "C"
