// Transducer response H^e (Sec. II.B, Eq. EIR) in the data space, one thread block per transducer
// row.  With taps h_m (m = m0 .. m0 + n - 1, zero elsewhere):
//
// k_apply_d_eir  the projector's epilogue when a response is set: s_j = (D g)_j (or g_j) in FP64
//                from the exact fixed-point sums of G into shared memory, then
//                u_k = sum_m h_m s_{k-1-m} over the window in FP64, one rounding to the storage
//                type (replaces k_apply_d_fix).
// k_eir_t        the backprojector's prologue: z_k = sum_m h_m y_{k+1+m} over the window (the
//                exact transpose), in FP64 from the stored y, one rounding to float32; the
//                voxel gather then reads z.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <string>

#include "brick.cuh"

namespace oat {

constexpr int kEirThreads = 256;

template <int DT>
__device__ __forceinline__ void store_eir(void *out, size_t i, float v) {
    if (DT == OAT_F32) ((float *)out)[i] = v;
    else if (DT == OAT_F16) ((__half *)out)[i] = __float2half_rn(v);
    else ((__nv_bfloat16 *)out)[i] = __float2bfloat16_rn(v);
}

template <int DT>
__device__ __forceinline__ double load_eir(const void *y, size_t i) {
    if (DT == OAT_F32) return (double)((const float *)y)[i];
    else if (DT == OAT_F16) return (double)__half2float(((const __half *)y)[i]);
    else return (double)__bfloat162float(((const __nv_bfloat16 *)y)[i]);
}

template <int DT, bool APPLY_D>
__global__ void __launch_bounds__(kEirThreads) k_apply_d_eir(const long long *__restrict__ gacc,
                                                              const double *__restrict__ wD, const double *__restrict__ h,
                                                              int nh, int m0, void *out, int K, const unsigned int *amax,
                                                              double bound_pts, double ds2) {
    extern __shared__ double sm[];
    double *srow = sm, *sh = sm + K;
    const double unit = ds2 / pow2_scale(bound_pts * (double)__uint_as_float(*amax), 61);
    const size_t base = (size_t)blockIdx.x * K;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        double v;
        if (!APPLY_D) v = (double)gacc[base + j] * unit;
        else if (j < 1 || j > K - 2) v = 0.0;
        else v = wD[j + 1] * ((double)gacc[base + j + 1] * unit) - wD[j - 1] * ((double)gacc[base + j - 1] * unit);
        srow[j] = v;
    }
    for (int i = threadIdx.x; i < nh; i += blockDim.x) sh[i] = h[i];
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < nh; ++i) {
            const int j = k - 1 - (m0 + i);
            if (j >= 0 && j < K) acc = fma(sh[i], srow[j], acc);
        }
        store_eir<DT>(out, base + k, (float)acc);
    }
}

template <int DT>
__global__ void __launch_bounds__(kEirThreads) k_eir_t(const void *__restrict__ y, const double *__restrict__ h,
                                                        int nh, int m0, float *__restrict__ z, int K) {
    extern __shared__ double sm[];
    double *srow = sm, *sh = sm + K;
    const size_t base = (size_t)blockIdx.x * K;
    for (int j = threadIdx.x; j < K; j += blockDim.x) srow[j] = load_eir<DT>(y, base + j);
    for (int i = threadIdx.x; i < nh; i += blockDim.x) sh[i] = h[i];
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < nh; ++i) {
            const int j = k + 1 + m0 + i;
            if (j >= 0 && j < K) acc = fma(sh[i], srow[j], acc);
        }
        z[base + k] = (float)acc;
    }
}

size_t eir_smem_bytes(const Plan &p) { return sizeof(double) * ((size_t)p.K + (size_t)p.eir_n); }

int set_eir_attributes(const Plan &p) {
    const int bytes = (int)eir_smem_bytes(p);
    cudaError_t e = cudaSuccess;
#define OAT_ATTR(K_) if (e == cudaSuccess) e = cudaFuncSetAttribute(K_, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
    OAT_ATTR((k_apply_d_eir<OAT_F32, true>)); OAT_ATTR((k_apply_d_eir<OAT_F16, true>)); OAT_ATTR((k_apply_d_eir<OAT_BF16, true>));
    OAT_ATTR((k_apply_d_eir<OAT_F32, false>)); OAT_ATTR((k_apply_d_eir<OAT_F16, false>)); OAT_ATTR((k_apply_d_eir<OAT_BF16, false>));
    OAT_ATTR(k_eir_t<OAT_F32>); OAT_ATTR(k_eir_t<OAT_F16>); OAT_ATTR(k_eir_t<OAT_BF16>);
#undef OAT_ATTR
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("oat_plan_set_eir: ") + cudaGetErrorString(e));
}

int launch_apply_d_eir(Plan &p, void *data, cudaStream_t s) {
    const size_t smem = eir_smem_bytes(p);
    const double bp = p.fwd_bound, ds2 = p.g.spacing_mm * p.g.spacing_mm;
    const long long *g = (const long long *)p.d_gacc;
    const int dt = p.g.data_dtype;
#define OAT_EIR(DTV, AD) k_apply_d_eir<DTV, AD><<<(unsigned)p.Q, kEirThreads, smem, s>>>( \
        g, p.t.wD64, p.d_eir, p.eir_n, p.eir_m0, data, p.K, p.d_amax, bp, ds2)
    if (p.g.apply_d) {
        if (dt == OAT_F32) OAT_EIR(OAT_F32, true); else if (dt == OAT_F16) OAT_EIR(OAT_F16, true); else OAT_EIR(OAT_BF16, true);
    } else {
        if (dt == OAT_F32) OAT_EIR(OAT_F32, false); else if (dt == OAT_F16) OAT_EIR(OAT_F16, false); else OAT_EIR(OAT_BF16, false);
    }
#undef OAT_EIR
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("oat_project: k_apply_d_eir: ") + cudaGetErrorString(e));
}

int launch_eir_t(Plan &p, const void *y, float *z, cudaStream_t s) {
    const size_t smem = eir_smem_bytes(p);
    switch (p.g.data_dtype) {
        case OAT_F32: k_eir_t<OAT_F32><<<(unsigned)p.Q, kEirThreads, smem, s>>>(y, p.d_eir, p.eir_n, p.eir_m0, z, p.K); break;
        case OAT_F16: k_eir_t<OAT_F16><<<(unsigned)p.Q, kEirThreads, smem, s>>>(y, p.d_eir, p.eir_n, p.eir_m0, z, p.K); break;
        default: k_eir_t<OAT_BF16><<<(unsigned)p.Q, kEirThreads, smem, s>>>(y, p.d_eir, p.eir_n, p.eir_m0, z, p.K); break;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("oat_backproject: k_eir_t: ") + cudaGetErrorString(e));
}

}  // namespace oat
