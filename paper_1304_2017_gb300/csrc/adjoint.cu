// Backprojector alpha' = G^T D^T y (adjoints of Eqs. dis_srt and dis_g2p), no floating-point
// atomics.
//
// A lattice point P of (q, k) contributes Delta_s^2 g'_{q,k} psi_n(P) to the eight nodes n of
// the cell floor(P) (Eq. expfunI), with g'_{q,k} = (C_D / tau_k)(m_{k-1} y_{k-1} -
// m_{k+1} y_{k+1}), m_j = [1 <= j <= K-2] (the exact transpose of the projector's D), read
// straight from y.
//
// k_brick_gather_t  one thread block per brick of kBA^3 cells (and range of transducers).  The
//                   block walks, transducer by transducer, the lattice points that can lie in
//                   the brick (brick.cuh), evaluates each with the lattice-point functions shared
//                   with the projector (oat_internal.h), and for the points whose cell lies in
//                   the brick adds the
//                   eight weights w_c g'_{q,k}, rounded to the pass's fixed-point unit, to the
//                   brick's (kBA+1)^3 node sums with 32-bit integer shared-memory atomics.
//                   Integer addition is exact and associative, so the sums do not depend on the
//                   order of the points.  After each bounded pass of transducers the node sums
//                   are folded, exactly, into the volume's 64-bit accumulator (integer global
//                   atomics: the nodes on brick faces are shared with neighbouring bricks).
// Fixed-point units.  k_gprime_rowmax first takes, per transducer q, M_q = max |g'_{q,k}| over
// the samples whose shells can reach the grid.  A pass over transducers Q_p uses the unit
// 2^-e_p with e_p chosen so that every contribution |w g'| <= max_{q in Q_p} M_q maps to at most
// 2^30 units: each pass keeps 30 bits relative to its own data, so a spike or a
// wide-dynamic-range record in one pass costs no precision in the others.  The volume
// accumulator's unit 2^-e_g is finer (e_g >= e_p: a pass folds in by an exact left shift); it
// is chosen from the largest M_q and the plan's bound on the contributions one node can
// receive, so that no 64-bit sum can overflow.
// k_finish_t        alpha'_n = sum_n 2^-e_g Delta_s^2 as float32: every voxel written once.
// AREA instances scale each point's g' by its ring's exact-strip-area weight factor.  With a transducer response set, eir.cu's k_eir_t
// first forms z = H^e^T y and the gather reads z as float32 data.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "brick.cuh"

#include <mutex>
#include <string>

namespace oat {

constexpr int kAdjThreads = 1024;

struct AdjArgs {
    DevTables t;
    const void *y;
    unsigned long long *vacc;     // [N] fixed-point node sums
    const float *rowmax;          // [Q] M_q = max |g'_{q,k}| over the shells that reach the grid
    const unsigned int *amax;     // bits of max_q M_q
    int nx, ny, nz, K, Q;
    int nb[3], bs[3];
    int qchunk, kspan, qpass;
    float O[3], O_lo[3];
    float R0, dR;
    float wfac;                   // bound of a point's lattice-weight factor (1 with uniform weights)
    int fbits;                    // the volume accumulator holds max M_q wfac as 2^fbits units at most
    int apply_d;
};

// Exponent e such that |x| 2^e <= 2^bits for every |x| <= bound (bound = m 2^ex, m in [0.5, 1),
// e = bits - ex); 0 when bound is zero or not finite.
__host__ __device__ __forceinline__ int pow2_exp(double bound, int bits) {
    if (!(bound > 0.0) || !(bound < 1e300)) return 0;
    int ex;
    frexp(bound, &ex);
    return bits - ex;
}

// Exponent of the volume accumulator's unit: every contribution, in that unit, is at most 2^fbits.
__device__ __forceinline__ int volume_exp(const unsigned int *amax, float wfac, int fbits) {
    return pow2_exp((double)__uint_as_float(*amax) * (double)wfac, fbits);
}

template <int DT>
__device__ __forceinline__ float load_data(const void *p, size_t i) {
    if (DT == OAT_F32) return __ldg((const float *)p + i);
    else if (DT == OAT_F16) return __half2float(((const __half *)p)[i]);
    else return __bfloat162float(((const __nv_bfloat16 *)p)[i]);
}

// g'_{q,k}: D^T y (exact transpose of the projector's D, masked rows 0 and K-1), or y itself.
template <int DT>
__device__ __forceinline__ float gprime(const AdjArgs &a, int q, int k) {
    const size_t base = (size_t)q * a.K;
    if (!a.apply_d) return load_data<DT>(a.y, base + k);
    const float w = __ldg(a.t.wD + k);
    if (w == 0.f) return 0.f;
    float lo = (k - 1 >= 1 && k - 1 <= a.K - 2) ? load_data<DT>(a.y, base + k - 1) : 0.f;
    float hi = (k + 1 >= 1 && k + 1 <= a.K - 2) ? load_data<DT>(a.y, base + k + 1) : 0.f;
    return w * (lo - hi);
}

// M_q = max |g'_{q,k}| over the samples kr[q].x .. kr[q].y (the shells that can reach the grid,
// from the plan), computed with the gather's own gprime so that every g' the gather uses is
// bounded by it; max_q M_q into *amax (NaN wins: its unit then becomes 1).  One warp per row.
template <int DT>
__global__ void k_gprime_rowmax(AdjArgs a, const int2 *__restrict__ kr, float *rowmax, unsigned int *amax) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    float wmax = 0.f;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < a.Q; q += warps) {
        const int2 r = __ldg(kr + q);
        float m = 0.f;
        for (int k = r.x + lane; k <= r.y; k += 32) {
            const float v = fabsf(gprime<DT>(a, q, k));
            m = (v > m || v != v) ? v : m;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float w = __shfl_xor_sync(0xffffffffu, m, o);
            m = (w > m || w != w) ? w : m;
        }
        if (lane == 0) rowmax[q] = m;
        wmax = (m > wmax || m != m) ? m : wmax;
    }
    if (lane == 0) atomicMax(amax, __float_as_uint(wmax));
}

// Node sums of one pass live in shared memory as two 32-bit integer halves of the
// fixed-point value v (|v| <= 2^30): hi = v >> 15 (arithmetic) and lo = v & 0x7fff, each added
// with a native 32-bit integer atomic.  A pass is bounded so that neither half can overflow
// (at most 2^15 contributions per node); the halves are then folded into the 64-bit volume
// accumulator and cleared.
__device__ __forceinline__ void sadd(int *hi, unsigned int *lo, int idx, float x) {
    const int v = __float2int_rn(x);
    atomicAdd(hi + idx, v >> 15);
    atomicAdd(lo + idx, (unsigned int)(v & 0x7fff));
}

// Node layout of the brick's (B+1)^3 node sums: x stride 1, y stride S1, z stride S2, with S2
// padded so that the 32 lanes' scatters, which follow rings in arbitrary directions, spread
// over the banks.  Simulated on lattice-point warps of the 256^3 workload (the same address in
// several lanes counts as a conflict, as the measured wavefronts per atomic, 3.2, show): about
// 3.1-3.2 bank wavefronts per atomic with the padding against 3.5 without; among paddings that
// simulate alike, 19 (S2 = 644 at B = 24) timed 0.5 % faster than 13.
template <int B>
struct NodeLayout {
    static constexpr int S1 = B + 1;
    static constexpr int S2 = S1 * (B + 1) + 19;
    static constexpr int NN = S2 * (B + 1);
    static constexpr int NN2 = 2 * NN + ((2 * NN) & 3 ? 4 - ((2 * NN) & 3) : 0);
};

// Scatter one owned point (cell-local weights wx, wy, wz; first node b in the low 16 bits of
// e.w, the point's shell s within the unit above them) with value wg[s].
// The eight weights are the products (g uz_or_wz) uy_or_wy ux_or_wx in that order, formed in
// packed FP32 pairs.
template <int S1, int S2>
__device__ __forceinline__ void scatter8(int *shi, unsigned int *slo, float4 e, const float *wg, float wr = 1.f) {
    const float wx = e.x, wy = e.y, wz = e.z;
    const int bs = __float_as_int(e.w);
    const int b = bs & 0xffff;
    const float gq = wg[bs >> 16] * wr;
    const float ux = 1.f - wx, uy = 1.f - wy, uz = 1.f - wz;
    const f32x2 Z = mul2(pk2(gq, gq), pk2(uz, wz));          // (g uz, g wz)
    const f32x2 Y0 = mul2(Z, pk2(uy, uy)), Y1 = mul2(Z, pk2(wy, wy));
    float g00, g10, g01, g11;
    upk2(Y0, g00, g10);
    upk2(Y1, g01, g11);
    const f32x2 X = pk2(ux, wx);
    float v0, v1;
    upk2(mul2(pk2(g00, g00), X), v0, v1);
    sadd(shi, slo, b, v0);           sadd(shi, slo, b + 1, v1);
    upk2(mul2(pk2(g01, g01), X), v0, v1);
    sadd(shi, slo, b + S1, v0);      sadd(shi, slo, b + S1 + 1, v1);
    upk2(mul2(pk2(g10, g10), X), v0, v1);
    sadd(shi, slo, b + S2, v0);      sadd(shi, slo, b + S2 + 1, v1);
    upk2(mul2(pk2(g11, g11), X), v0, v1);
    sadd(shi, slo, b + S2 + S1, v0); sadd(shi, slo, b + S2 + S1 + 1, v1);
}

template <int B, int DT, bool AREA>
__global__ void __launch_bounds__(kAdjThreads, 1) k_brick_gather_t(AdjArgs a) {
    extern __shared__ int shi[];   // node-sum high halves, low halves, segment slots, views
    using NL = NodeLayout<B>;
    constexpr int S1 = NL::S1, S2 = NL::S2, NN = NL::NN, NN2 = NL::NN2;
    unsigned int *slo = (unsigned int *)(shi + NN);
    SegSlot *slots = (SegSlot *)(shi + NN2);
    BrickView *views = (BrickView *)(slots + kAdjThreads);
    const int nqc = (a.Q + a.qchunk - 1) / a.qchunk;
    const int brick = blockIdx.x / nqc;
    const int q0 = (blockIdx.x % nqc) * a.qchunk;
    const int q1 = min(a.Q, q0 + a.qchunk);
    int L[3], E[3];
    {
        const int n[3] = {a.nx, a.ny, a.nz};
        brick_box(brick, a.nb, a.bs, n, L, E);
    }
    for (int idx = threadIdx.x; idx < NN; idx += blockDim.x) { shi[idx] = 0; slo[idx] = 0u; }
    __syncthreads();

    // bounding sphere and box of the brick's cells [L, L + E)
    // brick centre c, cell box [blo, bhi) and bounding-sphere radius rb: block-shared constants
    __shared__ float c[3], blo[3], bhi[3], rbs[2];
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
    __shared__ struct { float scale; int qe; long long fold; } s_pass;   // the current pass: unit, end
    __shared__ int s_next;   // next unit of the pass to take (the first nwarps by the warps' indices)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    SegSlot *ws = slots + warp * 32;
    __shared__ float s_wg[kAdjThreads / 32][kShells];
    float *wg = s_wg[warp];

    int qe = q0;   // end of the current pass, read from s_pass right after the pass's first barrier
    for (int qp = q0; qp < q1; qp = qe) {
        // the pass: at most qpass transducers from qp on, ended early before a transducer whose
        // max |g'| would spread the pass's maxima by more than 2^8, so that every transducer's
        // contributions keep at least 22 bits of its own maximum (a spike or an outlier row gets
        // a pass of its own).  Its unit 2^-ep: contributions |w g'| <= max_{q in pass} M_q wfac
        // map to at most 2^30 units; never finer than the volume accumulator's unit 2^-eg, so that
        // the pass folds in exactly (ep in [-113, 126], so 2^ep is a normal float).
        if (warp == 0) {
            const int n = min(a.qpass, q1 - qp);
            float hi = 0.f, lo = __int_as_float(0x7f800000);   // running max and least positive max
            int cut = n;
            for (int base = 0; base < n; base += 32) {
                const int i = base + lane;
                float v = i < n ? __ldg(a.rowmax + qp + i) : 0.f;
                if (v != v) v = __int_as_float(0x7f800000);   // NaN rows: alone in their pass
                float vh = v, vl = v > 0.f ? v : __int_as_float(0x7f800000);
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float th = __shfl_up_sync(0xffffffffu, vh, o), tl = __shfl_up_sync(0xffffffffu, vl, o);
                    if (lane >= o) { vh = fmaxf(vh, th); vl = fminf(vl, tl); }
                }
                vh = fmaxf(vh, hi);
                vl = fminf(vl, lo);
                const unsigned bad = __ballot_sync(0xffffffffu, i < n && vh > 256.f * vl);
                if (bad) {
                    cut = max(1, base + __ffs(bad) - 1);
                    break;
                }
                hi = __shfl_sync(0xffffffffu, vh, 31);
                lo = __shfl_sync(0xffffffffu, vl, 31);
            }
            float m = 0.f;
            for (int q = qp + lane; q < qp + cut; q += 32) {
                const float v = __ldg(a.rowmax + q);
                m = (v > m || v != v) ? v : m;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float w = __shfl_xor_sync(0xffffffffu, m, o);
                m = (w > m || w != w) ? w : m;
            }
            if (lane == 0) {
                const int eg = volume_exp(a.amax, a.wfac, a.fbits);
                const int ep = min(126, m > 0.f ? min(eg, pow2_exp((double)m * (double)a.wfac, 30)) : eg);
                s_pass.scale = ldexpf(1.f, ep);
                s_pass.fold = eg - ep < 63 ? (1LL << (eg - ep)) : 0;   // a larger shift meets only zero sums
                s_pass.qe = qp + cut;
                s_next = nwarps;
            }
        }
        __syncthreads();
        qe = s_pass.qe;   // s_pass is rewritten only after the barrier that ends this pass
        const int nkg = (a.kspan + kShells - 1) / kShells;
        const int units = (qe - qp) * nkg;
        int vq = -1;
        BrickView &v = views[warp];   // the current transducer's view of the brick (shared, per warp)
        float ex[3], ey[3];
        for (int u = warp; u < units; u = next_unit(&s_next, lane)) {
            const int q = qp + u / nkg;
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
            // lanes 0..kShells-1: one shell each (skipped where g' is zero)
            int n = 0, gbase = 0;
            float gs = 0.f;
            if (lane < kShells && kb + lane <= v.k1) {
                const int k = kb + lane, ck = v.cls * a.K + k;
                int ilo, ihi;
                if (shell_ring_range(v, __ldg(a.t.Rk + k), __ldg(a.t.ring_cnt + ck), rb2, ilo, ihi)) {
                    gs = gprime<DT>(a, q, k) * s_pass.scale;
                    if (gs != 0.f) {
                        n = ihi - ilo + 1;
                        gbase = __ldg(a.t.ring_off + ck) + ilo;
                    }
                }
            }
            int p0, p1, p2;
            const int T = unit_shells(n, lane, p0, p1, p2);
            if (T == 0) continue;
            __syncwarp();
            if (lane < kShells) wg[lane] = gs;   // g' of the unit's shells, read by scatter8
            __syncwarp();
            for (int ib = 0; ib < T; ib += 32) {
                int shell;
                const int gidx = unit_ring(ib + lane, T, p0, p1, p2, gbase, shell);
                int wa0, wna, wb0, wnb, sincl;
                const int S = ring_windows(v, a.t.rings, gidx, a.O, rb2, blo, bhi, lane, wa0, wna, wb0, wnb, sincl);
                for (int sc = 0, used = 0; sc < S; sc += used) {
                    int my_start, csh;
                    const int total = segment_chunk<false>(a.t.xd + q, a.t.rings, a.t.anchors, AREA ? a.t.ring_w : nullptr,
                                                           gidx, shell, a.O, a.O_lo,
                                                           L, sc, S, lane, wa0, wna, wb0, wnb, sincl, ws, my_start, used,
                                                           csh);
                    for (int f = 0; f < total; f += 32) {
                        int lc[3];
                        float w[3], wr;
                        bool own = false;
                        float4 ent;
                        const int sh = segment_point(ws, f, lane, my_start, total, ex, ey, lc, w, wr);
                        if (sh >= 0) {
                            own = (unsigned)lc[0] < (unsigned)E[0] && (unsigned)lc[1] < (unsigned)E[1] &&
                                  (unsigned)lc[2] < (unsigned)E[2];
                            ent = make_float4(w[0], w[1], w[2], __int_as_float((lc[2] * S2 + lc[1] * S1 + lc[0]) | (sh << 16)));
                        }
                        // each lane scatters its own point (about 93 % of the candidates are
                        // owned; a per-warp queue that kept every lane of the scatter busy cost
                        // more in its shared stores, loads and bookkeeping: measured 10 % slower)
                        if (own) scatter8<S1, S2>(shi, slo, ent, wg, AREA ? wr : 1.f);
                    }
                    __syncwarp();
                }
            }
            __syncwarp();
        }
        __syncthreads();
        // fold the pass into the 64-bit volume accumulator (nodes on brick faces are shared
        // with neighbouring bricks: integer atomics)
        for (int idx = threadIdx.x; idx < NN; idx += blockDim.x) {
            const int hi = shi[idx];
            const unsigned int lo = slo[idx];
            if (hi != 0 || lo != 0u) {
                shi[idx] = 0; slo[idx] = 0u;
                const int lz = idx / S2, r = idx - lz * S2, ly = r / S1;
                const int x = r - ly * S1 + L[0], y = ly + L[1], z = lz + L[2];
                if (x >= 0 && x < a.nx && y >= 0 && y < a.ny && z >= 0 && z < a.nz) {
                    // the pass's sum in the volume's unit: exact (eg >= ep)
                    const long long vv = ((long long)hi * 32768LL + (long long)lo) * s_pass.fold;
                    atomicAdd(a.vacc + ((size_t)z * a.ny + y) * a.nx + x, (unsigned long long)vv);
                }
            }
        }
        __syncthreads();
    }
}

__global__ void k_finish_t(const long long *__restrict__ vacc, float *__restrict__ vol, size_t n,
                           const unsigned int *amax, float wfac, int fbits, double ds2) {
    const double unit = ldexp(ds2, -volume_exp(amax, wfac, fbits));
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        vol[i] = (float)((double)vacc[i] * unit);
}

static int backproject_with(Plan &p, const void *data, float *vol, cudaStream_t s, long long *vacc, unsigned int *amax) {
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(vacc, 0, sizeof(long long) * N, s);
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_backproject: memset: ") + cudaGetErrorString(e));
    // with a transducer response the gather reads z = H^e^T y (float32) instead of y
    int dtype = p.g.data_dtype;
    if (p.eir_n > 0) {
        const int rc = launch_eir_t(p, data, p.d_eir_z, s);
        if (rc != OAT_OK) return rc;
        data = p.d_eir_z;
        dtype = OAT_F32;
    }
    AdjArgs a;
    a.t = p.t; a.y = data;
    a.vacc = (unsigned long long *)vacc;
    a.rowmax = p.d_rowmax;
    a.amax = amax;
    a.nx = p.nx; a.ny = p.ny; a.nz = p.nz; a.K = p.K; a.Q = p.Q;
    for (int d = 0; d < 3; ++d) { a.nb[d] = p.adj.nb[d]; a.bs[d] = p.adj.bs[d]; a.O[d] = p.O[d]; a.O_lo[d] = p.O_lo[d]; }
    a.qchunk = p.adj.qchunk; a.kspan = p.adj.kspan; a.qpass = p.adj_qpass;
    a.R0 = p.R0; a.dR = p.dR;
    a.wfac = p.adj_wfac;
    a.fbits = p.adj_fbits;
    a.apply_d = p.g.apply_d;
    {
        // per-transducer max |g'| (the passes' units) and its maximum (the volume's unit)
        const unsigned rb = (unsigned)std::min<long long>(((long long)p.Q + 7) / 8, (long long)p.n_sm * 16);
        float *rm = p.d_rowmax;
        const int2 *kr = p.d_krange;
        switch (dtype) {
            case OAT_F32: k_gprime_rowmax<OAT_F32><<<rb, 256, 0, s>>>(a, kr, rm, amax); break;
            case OAT_F16: k_gprime_rowmax<OAT_F16><<<rb, 256, 0, s>>>(a, kr, rm, amax); break;
            default: k_gprime_rowmax<OAT_BF16><<<rb, 256, 0, s>>>(a, kr, rm, amax); break;
        }
    }
    const bool prof = p.profiling && p.ev_used[1] + 2 <= (int)p.ev[1].size();
    if (prof) cudaEventRecord(p.ev[1][p.ev_used[1]], s);
    const unsigned grid = (unsigned)p.adj.items;
#define OAT_GT(DTV, AR) k_brick_gather_t<kBA, DTV, AR><<<grid, kAdjThreads, p.adj.smem, s>>>(a)
    if (p.area) {
        switch (dtype) {
            case OAT_F32: OAT_GT(OAT_F32, true); break;
            case OAT_F16: OAT_GT(OAT_F16, true); break;
            default: OAT_GT(OAT_BF16, true); break;
        }
    } else {
        switch (dtype) {
            case OAT_F32: OAT_GT(OAT_F32, false); break;
            case OAT_F16: OAT_GT(OAT_F16, false); break;
            default: OAT_GT(OAT_BF16, false); break;
        }
    }
#undef OAT_GT
    if (prof) { cudaEventRecord(p.ev[1][p.ev_used[1] + 1], s); p.ev_used[1] += 2; }
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_backproject: k_brick_gather_t: ") + cudaGetErrorString(e));
    k_finish_t<<<(unsigned)std::min<size_t>((N + 255) / 256, (size_t)p.n_sm * 16), 256, 0, s>>>(
        (const long long *)vacc, vol, N, amax, p.adj_wfac, p.adj_fbits, p.g.spacing_mm * p.g.spacing_mm);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_backproject: k_finish_t: ") + cudaGetErrorString(e));
    return OAT_OK;
}

int launch_backproject(Plan &p, const void *data, float *vol, cudaStream_t s) {
    return backproject_with(p, data, vol, s, p.d_vacc, p.d_amax + 1);
}

// ---------------------------------------------------------------------------------------------
// Backprojection without any allocation.  Some callers cannot allocate device memory at the
// time they need H^T (for example code running inside a pool-managed or graph-building context
// that forbids cudaMalloc, or a host framework that hands out only the buffers it owns).  For
// them the scratch of the backprojector -- the 64-bit node accumulator and the max|g'| word -- is a
// file-scope array in device memory, sized for volumes of at most kStaticVoxels voxels.  The
// array exists on every GPU that loads this library, until the process exits.
constexpr size_t kStaticVoxels = size_t(1) << 21;          // 2,097,152 voxels (e.g. 128^3)
constexpr size_t kStaticHeader = 32;                       // 256 bytes: max|g'| bit pattern
static __device__ __align__(256) unsigned long long g_static_scratch[kStaticHeader + kStaticVoxels];

static std::mutex g_static_mu;
static void *g_static_addr[256] = {};

// Device address of the array on device dev (dev current); looked up once per device.
static int static_scratch(int dev, void **out) {
    if (dev < 0 || dev >= 256) return set_error(OAT_ERR_INVALID_ARG, "oat_backproject_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr)
            return set_error(OAT_ERR_CUDA, std::string("oat_backproject_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_static_addr[dev] = ptr;
    }
    *out = g_static_addr[dev];
    return OAT_OK;
}

int launch_backproject_static(Plan &p, const void *data, float *vol, cudaStream_t s) {
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    if (N > kStaticVoxels)
        return set_error(OAT_ERR_INVALID_ARG, "oat_backproject_noalloc: volume of " + std::to_string(N) +
                                                  " voxels exceeds the static scratch limit of " +
                                                  std::to_string(kStaticVoxels) + " voxels");
    void *base = nullptr;
    int rc = static_scratch(p.device, &base);
    if (rc != OAT_OK) return rc;
    unsigned long long *w = (unsigned long long *)base;
    return backproject_with(p, data, vol, s, (long long *)(w + kStaticHeader), (unsigned int *)w);
}

size_t adjoint_smem_bytes(bool area) {
    (void)area;
    return sizeof(int) * NodeLayout<kBA>::NN2 + sizeof(SegSlot) * kAdjThreads + sizeof(BrickView) * (kAdjThreads / 32);
}

int set_adjoint_attributes() {
    const int b0 = (int)adjoint_smem_bytes(false), b1 = (int)adjoint_smem_bytes(true);
    cudaError_t e = cudaSuccess;
#define OAT_ATTR(DTV, AR, BYTES) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_brick_gather_t<kBA, DTV, AR>, cudaFuncAttributeMaxDynamicSharedMemorySize, BYTES)
    OAT_ATTR(OAT_F32, false, b0); OAT_ATTR(OAT_F16, false, b0); OAT_ATTR(OAT_BF16, false, b0);
    OAT_ATTR(OAT_F32, true, b1); OAT_ATTR(OAT_F16, true, b1); OAT_ATTR(OAT_BF16, true, b1);
#undef OAT_ATTR
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
}

}  // namespace oat
