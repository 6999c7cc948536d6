// Projector u = D G alpha (Eqs. dis_srt and dis_g2p).
//
// k_brick_gather   G alpha as 64-bit fixed-point sums [Q][K]: per-brick shell gather (below).
// k_apply_d_fix    u_k = C_D (g_{k+1}/tau_{k+1} - g_{k-1}/tau_{k-1}) for 1 <= k <= K-2, 0 at the
//                  ends (or u = g without D) in double precision -- the difference of
//                  neighbouring samples cancels by one to three digits -- with one rounding to
//                  float32 / float16 / bfloat16 at the end.
// k_absmax         max |x| of a buffer (the projector's fixed-point unit).
// k_brick_gather<COUNT>  lattice points whose stencil touches the grid (oat_plan_query).
// k_brick_gather<AREA>   the same gather with each point's value scaled by its ring's
//                  exact-strip-area weight factor (OAT_LATTICE_EXACT_AREA).
// With a transducer response set, eir.cu's k_apply_d_eir replaces k_apply_d_fix.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "brick.cuh"
#include <cstdlib>

namespace oat {

__global__ void k_absmax(const void *__restrict__ x, size_t n, int dtype, unsigned int *out) {
    float m = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float v;
        if (dtype == OAT_F32) v = ((const float *)x)[i];
        else if (dtype == OAT_F16) v = __half2float(((const __half *)x)[i]);
        else v = __bfloat162float(((const __nv_bfloat16 *)x)[i]);
        v = fabsf(v);
        m = (v > m || v != v) ? v : m;   // NaN wins, making the scale 1
    }
    for (int o = 16; o > 0; o >>= 1) {
        float w = __shfl_xor_sync(0xffffffffu, m, o);
        m = (w > m || w != w) ? w : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

template <int DT>
__device__ __forceinline__ void store_data(void *out, size_t i, float v) {
    if (DT == OAT_F32) ((float *)out)[i] = v;
    else if (DT == OAT_F16) ((__half *)out)[i] = __float2half_rn(v);
    else ((__nv_bfloat16 *)out)[i] = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------------------- bricks
// k_brick_gather: one block per work item (brick of kBF^3 cells, range of transducers).  The
// brick's (kBF+1)^3 nodes are staged in shared memory (zero outside the grid).  A warp takes one
// unit (a transducer and kShells consecutive shells) at a time; one lane per ring computes the
// ring's azimuth window clipped to the brick, one lane per anchor segment computes its anchor,
// the candidates are spread evenly over the lanes (brick.cuh), and each point whose cell lies
// in the brick is interpolated from shared memory.  Candidate chunks hold one shell each, in
// shell order; every lane keeps a compensated FP32 sum of the current shell, which is summed over
// the warp and added to g[q][k] as a 64-bit fixed-point integer (one atomic per shell and unit)
// when the shell changes.  Integer addition makes the result independent of the order in which
// bricks finish.
constexpr int kFwdThreads = 1024;

struct FwdArgs {
    DevTables t;
    const float *vol;
    unsigned long long *gacc;     // [Q][K] fixed-point sums
    const unsigned int *amax;     // bits of max |alpha|
    int nx, ny, nz, K, Q;
    int nb[3], bs[3];
    int qchunk, kspan;
    float O[3], O_lo[3];
    float R0, dR;
    double bound_pts;             // max sum of the point weights (over Delta_s^2) of one shell
    unsigned long long *count;    // COUNT mode: owned lattice points
};

// The warp's compensated sums (s, e), summed over the lanes, rounded to the fixed-point unit
// 1 / scale and added to *dst by lane 0 (integer addition: exact and order-independent).
__device__ __forceinline__ void flush_shell(float s, float e, double scale, int lane, unsigned long long *dst) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
        kadd(s, e, s2);
        e += e2;
    }
    if (lane == 0) {
        const long long v = __double2ll_rn(((double)s + (double)e) * scale);
        if (v != 0) atomicAdd(dst, (unsigned long long)v);
    }
}

// Trilinear interpolation (Eq. expfunI) at weights w of the cell whose first node is sp (node
// strides 1, S1, S2): x-lerps of the (z, z + 1) corner pairs side by side, then the y-lerps of
// the two z planes side by side, then z.  Each lerp is fma(w, b - a, a), as a scalar evaluation
// would round it.
template <int S1, int S2>
__device__ __forceinline__ float trilinear(const float *sp, const float w[3]) {
    const f32x2 M1 = pk2(-1.f, -1.f);
    const f32x2 A0 = pk2(sp[0], sp[S2]), A1 = pk2(sp[1], sp[S2 + 1]);
    const f32x2 B0 = pk2(sp[S1], sp[S2 + S1]), B1 = pk2(sp[S1 + 1], sp[S2 + S1 + 1]);
    const f32x2 WX = pk2(w[0], w[0]);
    const f32x2 CA = fma2(WX, fma2(A0, M1, A1), A0);   // (c00, c10)
    const f32x2 CB = fma2(WX, fma2(B0, M1, B1), B0);   // (c01, c11)
    const f32x2 E = fma2(pk2(w[1], w[1]), fma2(CA, M1, CB), CA);
    float e0, e1;
    upk2(E, e0, e1);
    return fmaf(w[2], e1 - e0, e0);
}

// COUNT: instead of interpolating, count the points each brick owns (the bricks tile the cells
// [-1, n-1]^3, so the total is the number of lattice points whose stencil touches the grid).
template <int B, bool COUNT, bool AREA>
__global__ void __launch_bounds__(kFwdThreads, 1) k_brick_gather(FwdArgs a) {
    extern __shared__ float sv[];   // (B+1)^3 nodes of the brick, then the warps' segment slots
    constexpr int S1 = B + 1, S2 = (B + 1) * (B + 1), NN = (B + 1) * (B + 1) * (B + 1);
    constexpr int NNp = NN + ((NN & 3) ? 4 - (NN & 3) : 0);
    SegSlot *slots = (SegSlot *)(sv + NNp);
    BrickView *views = (BrickView *)(slots + kFwdThreads);
    const int nqc = (a.Q + a.qchunk - 1) / a.qchunk;
    const int brick = blockIdx.x / nqc;
    const int q0 = (blockIdx.x % nqc) * a.qchunk;
    const int q1 = min(a.Q, q0 + a.qchunk);
    int L[3], E[3];
    {
        const int n[3] = {a.nx, a.ny, a.nz};
        brick_box(brick, a.nb, a.bs, n, L, E);
    }
    for (int idx = threadIdx.x; idx < (COUNT ? 0 : NN); idx += blockDim.x) {
        const int x = idx % S1 + L[0], y = (idx / S1) % S1 + L[1], z = idx / S2 + L[2];
        float val = 0.f;
        if (x >= 0 && x < a.nx && y >= 0 && y < a.ny && z >= 0 && z < a.nz) val = __ldg(a.vol + ((size_t)z * a.ny + y) * a.nx + x);
        sv[idx] = val;
    }
    __syncthreads();

    // brick centre c, cell box [blo, bhi) and bounding-sphere radius rb: block-shared constants
    __shared__ float c[3], blo[3], bhi[3], rbs[2];
    __shared__ int s_next;   // next unit to take (the first nwarps are taken by the warps' indices)
    if (threadIdx.x == 0) s_next = blockDim.x >> 5;
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        c[d] = L[d] + 0.5f * E[d];
        blo[d] = (float)L[d];
        bhi[d] = (float)(L[d] + E[d]);
        if (d == 0) {
            rbs[0] = 0.5f * sqrtf((float)(E[0] * E[0] + E[1] * E[1] + E[2] * E[2])) + 0.05f;
            rbs[1] = rbs[0] * rbs[0];
        }
    }
    __syncthreads();
    const float &rb = rbs[0], &rb2 = rbs[1];
    const double scale = COUNT ? 1.0 : pow2_scale(a.bound_pts * (double)__uint_as_float(*a.amax), 61);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long owned = 0;   // COUNT mode
    SegSlot *ws = slots + warp * 32;
    const int nkg = (a.kspan + kShells - 1) / kShells;
    const int units = (q1 - q0) * nkg;
    int vq = -1;
    BrickView &v = views[warp];   // the current transducer's view of the brick (shared, per warp)
    float ex[3], ey[3];

    for (int u = warp; u < units; u = next_unit(&s_next, lane)) {
        const int q = q0 + u / nkg;
        if (q != vq) {
            __syncwarp();
            if (lane == 0) brick_view(a.t.xd[q], a.O, c, rb, a.R0, a.dR, a.K, v);
            __syncwarp();
#pragma unroll
            for (int d = 0; d < 3; ++d) { ex[d] = v.ex[d]; ey[d] = v.ey[d]; }
            vq = q;
        }
        const int kb = v.k0 + (u % nkg) * kShells;
        if (kb > v.k1) continue;
        int n = 0, gbase = 0;
        if (lane < kShells && kb + lane <= v.k1) {
            const int k = kb + lane, ck = v.cls * a.K + k;
            int ilo, ihi;
            if (shell_ring_range(v, __ldg(a.t.Rk + k), __ldg(a.t.ring_cnt + ck), rb2, ilo, ihi)) {
                n = ihi - ilo + 1;
                gbase = __ldg(a.t.ring_off + ck) + ilo;
            }
        }
        int p0, p1, p2;
        const int T = unit_shells(n, lane, p0, p1, p2);
        if (T == 0) continue;
        // chunks hold one shell each (in shell order): a Kahan-compensated FP32 sum per lane (sum
        // acc, compensation kc: the sum is acc - kc), reduced over the warp with compensation and
        // added as a fixed-point integer when the shell changes.  H is a difference of neighbouring
        // shell sums (D), which cancels by up to a few digits, so the sums keep more than FP32.
        float acc = 0.f, kc = 0.f;
        int cur = -1;
        for (int ib = 0; ib < T; ib += 32) {
            int shell;
            const int gidx = unit_ring(ib + lane, T, p0, p1, p2, gbase, shell);
            int wa0, wna, wb0, wnb, sincl;
            const int S = ring_windows(v, a.t.rings, gidx, a.O, rb2, blo, bhi, lane, wa0, wna, wb0, wnb, sincl);
            for (int sc = 0, used = 0; sc < S; sc += used) {
                int my_start, csh;
                const int total = segment_chunk<true>(a.t.xd + q, a.t.rings, a.t.anchors, AREA ? a.t.ring_w : nullptr, gidx, shell, a.O, a.O_lo, L,
                                                      sc, S, lane, wa0, wna, wb0, wnb, sincl, ws, my_start, used, csh);
                if (csh != cur) {
                    if (!COUNT && cur >= 0) flush_shell(acc, -kc, scale, lane, a.gacc + (size_t)q * a.K + kb + cur);
                    acc = 0.f; kc = 0.f; cur = csh;
                }
                for (int f = 0; f < total; f += 32) {
                    int lc[3];
                    float w[3], wr;
                    if (segment_point(ws, f, lane, my_start, total, ex, ey, lc, w, wr) < 0) continue;
                    if ((unsigned)lc[0] < (unsigned)E[0] && (unsigned)lc[1] < (unsigned)E[1] && (unsigned)lc[2] < (unsigned)E[2]) {
                        if (COUNT) { ++owned; continue; }
                        const float *sp = sv + lc[2] * S2 + lc[1] * S1 + lc[0];
                        const float v = trilinear<S1, S2>(sp, w);
                        const float y = __fsub_rn(AREA ? wr * v : v, kc);
                        const float t = __fadd_rn(acc, y);
                        kc = __fsub_rn(__fsub_rn(t, acc), y);
                        acc = t;
                    }
                }
                __syncwarp();
            }
        }
        if (!COUNT && cur >= 0) flush_shell(acc, -kc, scale, lane, a.gacc + (size_t)q * a.K + kb + cur);
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) owned += __shfl_xor_sync(0xffffffffu, owned, o);
        if (lane == 0 && owned) atomicAdd(a.count, owned);
    }
}

// D in double on the exact fixed-point sums of G; one rounding to the storage type.
template <int DT, bool APPLY_D>
__global__ void k_apply_d_fix(const long long *__restrict__ gacc, const double *__restrict__ wD, void *out, int Q, int K,
                              const unsigned int *amax, double bound_pts, double ds2) {
    const double unit = ds2 / pow2_scale(bound_pts * (double)__uint_as_float(*amax), 61);
    const size_t n = (size_t)Q * K;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % K);
        double val;
        if (!APPLY_D) val = (double)gacc[idx] * unit;
        else if (k < 1 || k > K - 2) val = 0.0;
        else val = wD[k + 1] * ((double)gacc[idx + 1] * unit) - wD[k - 1] * ((double)gacc[idx - 1] * unit);
        store_data<DT>(out, idx, (float)val);
    }
}

size_t forward_smem_bytes() {
    const size_t nn = (size_t)(kBF + 1) * (kBF + 1) * (kBF + 1);
    return sizeof(float) * (nn + ((nn & 3) ? 4 - (nn & 3) : 0)) + sizeof(SegSlot) * kFwdThreads +
           sizeof(BrickView) * (kFwdThreads / 32);
}

int set_forward_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_brick_gather<kBF, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)forward_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_brick_gather<kBF, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)forward_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_brick_gather<kBF, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)forward_smem_bytes());
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
}

static void fill_forward_args(const Plan &p, const float *vol, FwdArgs &a) {
    a.t = p.t; a.vol = vol;
    a.gacc = (unsigned long long *)p.d_gacc;
    a.amax = p.d_amax;
    a.nx = p.nx; a.ny = p.ny; a.nz = p.nz; a.K = p.K; a.Q = p.Q;
    for (int d = 0; d < 3; ++d) { a.nb[d] = p.fwd.nb[d]; a.bs[d] = p.fwd.bs[d]; a.O[d] = p.O[d]; a.O_lo[d] = p.O_lo[d]; }
    a.qchunk = p.fwd.qchunk; a.kspan = p.fwd.kspan;
    a.R0 = p.R0; a.dR = p.dR;
    a.bound_pts = p.fwd_bound;
    a.count = nullptr;
}

int launch_project(Plan &p, const float *vol, void *data, cudaStream_t s) {
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    cudaError_t e = cudaMemsetAsync(p.d_amax, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.d_gacc, 0, sizeof(long long) * (size_t)p.Q * p.K, s);
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_project: memset: ") + cudaGetErrorString(e));
    k_absmax<<<(unsigned)std::min<size_t>((N + 255) / 256, (size_t)p.n_sm * 8), 256, 0, s>>>(vol, N, OAT_F32, p.d_amax);
    FwdArgs a;
    fill_forward_args(p, vol, a);
    const bool prof = p.profiling && p.ev_used[0] + 2 <= (int)p.ev[0].size();
    if (prof) cudaEventRecord(p.ev[0][p.ev_used[0]], s);
    if (p.area) k_brick_gather<kBF, false, true><<<(unsigned)p.fwd.items, kFwdThreads, p.fwd.smem, s>>>(a);
    else k_brick_gather<kBF, false, false><<<(unsigned)p.fwd.items, kFwdThreads, p.fwd.smem, s>>>(a);
    if (prof) { cudaEventRecord(p.ev[0][p.ev_used[0] + 1], s); p.ev_used[0] += 2; }
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_project: k_brick_gather: ") + cudaGetErrorString(e));
    if (p.eir_n > 0) return launch_apply_d_eir(p, data, s);
    const size_t n = (size_t)p.Q * p.K;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)p.n_sm * 16);
    const int dt = p.g.data_dtype;
    const double bp = p.fwd_bound, ds2 = p.g.spacing_mm * p.g.spacing_mm;
    const long long *g = (const long long *)p.d_gacc;
#define OAT_APPLY(DTV, AD) k_apply_d_fix<DTV, AD><<<blocks, 256, 0, s>>>(g, p.t.wD64, data, p.Q, p.K, p.d_amax, bp, ds2)
    if (p.g.apply_d) {
        if (dt == OAT_F32) OAT_APPLY(OAT_F32, true); else if (dt == OAT_F16) OAT_APPLY(OAT_F16, true); else OAT_APPLY(OAT_BF16, true);
    } else {
        if (dt == OAT_F32) OAT_APPLY(OAT_F32, false); else if (dt == OAT_F16) OAT_APPLY(OAT_F16, false); else OAT_APPLY(OAT_BF16, false);
    }
#undef OAT_APPLY
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_project: k_apply_d: ") + cudaGetErrorString(e));
    return OAT_OK;
}

// ---------------------------------------------------------------------------- point counting

// Lattice points whose stencil touches the grid: the projector's enumeration in COUNT mode.
int count_grid_points(Plan &p, long long *out) {
    FwdArgs a;
    fill_forward_args(p, nullptr, a);
    a.count = p.d_count;
    cudaError_t e = cudaMemset(p.d_count, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) {
        k_brick_gather<kBF, true, false><<<(unsigned)p.fwd.items, kFwdThreads, p.fwd.smem>>>(a);
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, p.d_count, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_plan_query: count: ") + cudaGetErrorString(e));
    *out = (long long)h;
    return OAT_OK;
}

}  // namespace oat
