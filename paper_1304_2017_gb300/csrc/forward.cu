// Projector u = D G alpha (Eqs. dis_srt and dis_g2p).
//
// k_shell_gather: one thread block per work item (radius class c, sample k, up to kT
// transducers of class c).  All transducers of a class share the shell lattice of sample k in
// local coordinates, so each lattice point's (cos phi_j, sin phi_j) is computed once and
// reused for the kT transducers.  Warps take rings, lanes take points along a ring; every
// point is a trilinear gather from the L2-resident volume.  Per-lane per-ring sums are folded
// into compensated per-thread totals, then reduced across the block.  Output: g [Q][K] scratch.
//
// k_apply_d: u_k = C_D (g_{k+1}/tau_{k+1} - g_{k-1}/tau_{k-1}) for 1 <= k <= K-2, 0 otherwise
// (or u = g without D), stored as float32 / float16 / bfloat16.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "oat_internal.h"

namespace oat {

constexpr int kT = 8;          // transducers per work item (matches the plan's tiling)
constexpr int kWarps = 8;      // warps per block

struct FwdArgs {
    DevTables t;
    const float *vol;
    double *g;
    int nx, ny, nz, K;
    float O[3];
    float ds2;
};

__global__ void __launch_bounds__(kWarps * 32) k_shell_gather(FwdArgs a) {
    const int4 it = a.t.items[blockIdx.x];
    const int cls = it.x, k = it.y, q0 = it.z, nq = it.w;
    __shared__ float sE[kT][9];
    __shared__ float sRed[kWarps][kT][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < kT * 9) {
        int t = threadIdx.x / 9, c = threadIdx.x % 9;
        float v = 0.f;
        if (t < nq) {
            const Xdcr &x = a.t.xd[a.t.qlist[q0 + t]];
            v = c < 3 ? x.ex[c] : (c < 6 ? x.ey[c - 3] : x.ez[c - 6]);
        }
        sE[t][c] = v;
    }
    __syncthreads();

    const int off = a.t.ring_off[cls * a.K + k];
    const int nr = a.t.ring_cnt[cls * a.K + k];
    // box of points whose stencil can touch the grid: P in [-1, n) per axis
    const float bx = (float)a.nx, by = (float)a.ny, bz = (float)a.nz;
    float tot[kT], err[kT];
#pragma unroll
    for (int t = 0; t < kT; ++t) { tot[t] = 0.f; err[t] = 0.f; }

    for (int i = warp; i < nr; i += kWarps) {
        const Ring r = a.t.rings[off + i];
        if (r.nj == 0) continue;
        float3 B[kT];
#pragma unroll
        for (int t = 0; t < kT; ++t) B[t] = ring_base(a.O, &sE[t][6], r.h);
        float racc[kT];
#pragma unroll
        for (int t = 0; t < kT; ++t) racc[t] = 0.f;
        for (int j0 = 0; j0 < r.nj; j0 += 32) {
            // Chunk of (up to) 32 consecutive points: lane t < nq tests whether the chunk can
            // reach the grid for transducer t (centre point within half the chunk's arc length,
            // plus one spacing, of the box); chunks that cannot are skipped for that transducer.
            const int jn = min(32, r.nj - j0);
            unsigned act;
            {
                const float half = 0.5f * (float)(jn - 1) + 1.0f;
                const float phc = (float)j0 * r.dphi + 0.5f * (float)(jn - 1) * r.dphi;
                float sc, cc;
                sincosf(phc, &sc, &cc);
                bool hit = false;
                if (lane < nq) {
                    const int l = lane & (kT - 1);
                    const float3 C = ring_point(ring_base(a.O, &sE[l][6], r.h), &sE[l][0], &sE[l][3], r.a * cc, r.a * sc);
                    const float dx = fmaxf(fmaxf(-1.f - C.x, C.x - bx), 0.f);
                    const float dy = fmaxf(fmaxf(-1.f - C.y, C.y - by), 0.f);
                    const float dz = fmaxf(fmaxf(-1.f - C.z, C.z - bz), 0.f);
                    hit = dx * dx + dy * dy + dz * dz <= half * half;
                }
                act = __ballot_sync(0xffffffffu, hit);
            }
            if (act == 0u) continue;
            const int j = j0 + lane;
            if (j < r.nj) {
                float u, v;
                ring_uv(r, j, u, v);
#pragma unroll
                for (int t = 0; t < kT; ++t) {
                    if (act & (1u << t)) {
                        float3 P = ring_point(B[t], &sE[t][0], &sE[t][3], u, v);
                        racc[t] += trilinear(a.vol, a.nx, a.ny, a.nz, P);
                    }
                }
            }
        }
#pragma unroll
        for (int t = 0; t < kT; ++t) kadd(tot[t], err[t], racc[t]);
    }

    // block reduction of (tot + err) per transducer: warp shuffle, then across warps
#pragma unroll
    for (int t = 0; t < kT; ++t) {
        float s = tot[t], e = err[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float s2 = __shfl_xor_sync(0xffffffffu, s, o);
            float e2 = __shfl_xor_sync(0xffffffffu, e, o);
            kadd(s, e, s2);
            e += e2;
        }
        if (lane == 0) { sRed[warp][t][0] = s; sRed[warp][t][1] = e; }
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        const int t = threadIdx.x;
        float s = 0.f, e = 0.f;
        for (int w = 0; w < kWarps; ++w) { kadd(s, e, sRed[w][t][0]); e += sRed[w][t][1]; }
        const int q = a.t.qlist[q0 + t];
        a.g[(size_t)q * a.K + k] = (double)a.ds2 * ((double)s + (double)e);
    }
}

template <int DT>
__device__ __forceinline__ void store_data(void *out, size_t i, float v) {
    if (DT == OAT_F32) ((float *)out)[i] = v;
    else if (DT == OAT_F16) ((__half *)out)[i] = __float2half_rn(v);
    else ((__nv_bfloat16 *)out)[i] = __float2bfloat16_rn(v);
}

// D in double precision on the FP64 sums of G (the difference of neighbouring samples
// cancels by one to three digits), one rounding to the storage type at the end.
template <int DT, bool APPLY_D>
__global__ void k_apply_d(const double *__restrict__ g, const double *__restrict__ wD, void *out, int Q, int K) {
    const size_t n = (size_t)Q * K;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % K);
        double v;
        if (!APPLY_D) v = g[idx];
        else if (k < 1 || k > K - 2) v = 0.0;
        else v = wD[k + 1] * g[idx + 1] - wD[k - 1] * g[idx - 1];
        store_data<DT>(out, idx, (float)v);
    }
}

// G alpha without D into the plan's g scratch (also used by the grid-point counter below).
static int enqueue_G(Plan &p, const float *vol, cudaStream_t s) {
    FwdArgs a;
    a.t = p.t; a.vol = vol; a.g = p.d_g;
    a.nx = p.nx; a.ny = p.ny; a.nz = p.nz; a.K = p.K;
    for (int d = 0; d < 3; ++d) a.O[d] = p.O[d];
    a.ds2 = p.ds2;
    cudaError_t e = cudaMemsetAsync(p.d_g, 0, sizeof(double) * (size_t)p.Q * p.K, s);
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_project: memset: ") + cudaGetErrorString(e));
    const bool prof = p.profiling && p.ev_used[0] + 2 <= (int)p.ev[0].size();
    if (prof) cudaEventRecord(p.ev[0][p.ev_used[0]], s);
    k_shell_gather<<<(unsigned)p.n_items, kWarps * 32, 0, s>>>(a);
    if (prof) { cudaEventRecord(p.ev[0][p.ev_used[0] + 1], s); p.ev_used[0] += 2; }
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_project: k_shell_gather: ") + cudaGetErrorString(e));
    return OAT_OK;
}

int launch_project(Plan &p, const float *vol, void *data, cudaStream_t s) {
    int rc = enqueue_G(p, vol, s);
    if (rc != OAT_OK) return rc;
    const size_t n = (size_t)p.Q * p.K;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
    const int dt = p.g.data_dtype;
    if (p.g.apply_d) {
        if (dt == OAT_F32) k_apply_d<OAT_F32, true><<<blocks, 256, 0, s>>>(p.d_g, p.t.wD64, data, p.Q, p.K);
        else if (dt == OAT_F16) k_apply_d<OAT_F16, true><<<blocks, 256, 0, s>>>(p.d_g, p.t.wD64, data, p.Q, p.K);
        else k_apply_d<OAT_BF16, true><<<blocks, 256, 0, s>>>(p.d_g, p.t.wD64, data, p.Q, p.K);
    } else {
        if (dt == OAT_F32) k_apply_d<OAT_F32, false><<<blocks, 256, 0, s>>>(p.d_g, p.t.wD64, data, p.Q, p.K);
        else if (dt == OAT_F16) k_apply_d<OAT_F16, false><<<blocks, 256, 0, s>>>(p.d_g, p.t.wD64, data, p.Q, p.K);
        else k_apply_d<OAT_BF16, false><<<blocks, 256, 0, s>>>(p.d_g, p.t.wD64, data, p.Q, p.K);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_project: k_apply_d: ") + cudaGetErrorString(e));
    return OAT_OK;
}

// ---------------------------------------------------------------------------- point counting

__global__ void __launch_bounds__(kWarps * 32) k_count(FwdArgs a, unsigned long long *count) {
    const int4 it = a.t.items[blockIdx.x];
    const int cls = it.x, k = it.y, q0 = it.z, nq = it.w;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int off = a.t.ring_off[cls * a.K + k];
    const int nr = a.t.ring_cnt[cls * a.K + k];
    unsigned long long n = 0;
    for (int t = 0; t < nq; ++t) {
        const Xdcr &x = a.t.xd[a.t.qlist[q0 + t]];
        for (int i = warp; i < nr; i += kWarps) {
            const Ring r = a.t.rings[off + i];
            float3 B = ring_base(a.O, x.ez, r.h);
            for (int j = lane; j < r.nj; j += 32) {
                float u, v;
                ring_uv(r, j, u, v);
                float3 P = ring_point(B, x.ex, x.ey, u, v);
                n += (P.x >= -1.f && P.x < (float)a.nx && P.y >= -1.f && P.y < (float)a.ny && P.z >= -1.f &&
                      P.z < (float)a.nz);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0 && n) atomicAdd(count, n);
}

int count_grid_points(Plan &p, long long *out) {
    FwdArgs a;
    a.t = p.t; a.vol = nullptr; a.g = nullptr;
    a.nx = p.nx; a.ny = p.ny; a.nz = p.nz; a.K = p.K;
    for (int d = 0; d < 3; ++d) a.O[d] = p.O[d];
    a.ds2 = p.ds2;
    unsigned long long *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long));
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_plan_query: ") + cudaGetErrorString(e));
    cudaMemset(d, 0, sizeof(unsigned long long));
    k_count<<<(unsigned)p.n_items, kWarps * 32>>>(a, d);
    unsigned long long h = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_plan_query: count: ") + cudaGetErrorString(e));
    *out = (long long)h;
    return OAT_OK;
}

}  // namespace oat
