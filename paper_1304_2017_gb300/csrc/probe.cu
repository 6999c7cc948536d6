// Read-bandwidth probe (include/oat_probe.h): grid-stride 16-byte loads, four independent sums
// per thread to keep many loads in flight, one atomic per block so nothing is dead code.
#include <cstdint>
#include <string>

#include "../../include/oat_probe.h"
#include "oat_internal.h"

namespace oat {

__global__ void __launch_bounds__(512) k_probe_read(const float4 *__restrict__ buf, long long n4, int reps,
                                                    float *sink) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n4; i += 4 * stride) {
            const float4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const float4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            s0 += a.x + a.y + a.z + a.w;
            s1 += b.x + b.y + b.z + b.w;
            s2 += c.x + c.y + c.z + c.w;
            s3 += d.x + d.y + d.z + d.w;
        }
        for (; i < n4; i += stride) {
            const float4 a = __ldcg(buf + i);
            s0 += a.x + a.y + a.z + a.w;
        }
    }
    float s = (s0 + s1) + (s2 + s3);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s == 12345.678f) atomicAdd(sink, s);   // never true in practice
}

}  // namespace oat

using namespace oat;

extern "C" int oat_probe_read(const void *d_buf, long long n_bytes, int reps, float *d_sink, void *stream) {
    if (!d_buf || !d_sink || n_bytes <= 0 || (n_bytes & 15) || ((uintptr_t)d_buf & 15) || reps < 1)
        return set_error(OAT_ERR_INVALID_ARG, "oat_probe_read: bad size or pointer");
    k_probe_read<<<(unsigned)(4 * current_sm_count()), 512, 0, (cudaStream_t)stream>>>((const float4 *)d_buf, n_bytes / 16, reps, d_sink);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("oat_probe_read: ") + cudaGetErrorString(e));
}
