// Spherical-voxel imaging model H_sph and its adjoint (include/oat_sph.h; Sec. II.B, Eqs. dis_sph,
// p0f, sphbwd) for point transducers, as direct sums over voxels x transducers x frequencies.
//
// Phases.  The phase of term (q, n, l) in cycles is f_l d_qn / c, up to a few hundred cycles,
// and the interpolation-free model needs it to about 1e-7 cycle.  The distance d_qn is formed in
// float-pair arithmetic from the node index and the transducer position in index units (both
// exact pairs), tau = d / c likewise, and f tau as a pair product whose integer part is dropped
// exactly: the fraction keeps ~1e-10 cycle whatever the distance.  Consecutive frequencies then
// differ by the rotation z = exp(-+j 2 pi df tau) (from sincospif, ~1 ulp), applied with one
// complex multiply per term (the forward takes two of its three steps per run by the three-term
// recurrence E_{k+1} = 2 cos(theta) E_k - E_{k-1} instead); every run of rotations starts from a
// directly evaluated phase.
//
// k_sph_fwd  one warp per (transducer, run of 256 frequencies, slab of voxels), 8 consecutive
//            frequencies per lane; the warp walks its slab 32 voxels at a time: lane j forms voxel
//            j's distance, weight alpha / (2 pi d) and z, the warp shares them by shuffles, and
//            every lane adds the voxel's 8 terms.  Sums: FP32 over 128 voxels, then compensated
//            (two-sum) into the slab total, written in double.  The slab count is chosen so that
//            the grid fills the GPU many times over whatever the transducer count.
// k_sph_reduce  sum of the slab totals in double, times p0 (double), rounded to float32.
// k_sph_conj v = u conj(p0) in double, rounded to float32 (the adjoint's input).
// k_sph_bwd  one thread per two consecutive voxels; transducer rows of v staged in shared
//            memory; per (voxel, transducer) the sum over frequencies runs in FP32 with an exact
//            phase every 32 frequencies, is weighted by 1 / (2 pi d) and added with
//            compensation.  Every voxel is written once: no atomics.
#include <cmath>
#include <string>
#include <vector>

#include "oat_internal.h"
#include "../../include/oat_sph.h"

namespace oat {

struct SphPlan {
    int device = 0;
    int nx = 0, ny = 0, nz = 0;
    long long N = 0;
    int Q = 0, L = 0, nseg = 0, qtile = 1;
    int n_slab = 1;                     // voxel slabs of the forward
    long long slab = 0;                 // voxels per slab (multiple of 32)
    size_t bwd_smem = 0;
    float sig_hi = 0.f, sig_lo = 0.f;   // Delta_s / c (microseconds per index unit) as a pair
    float df_hi = 0.f, df_lo = 0.f;     // frequency step (MHz) as a pair
    float inv2pids = 0.f;               // 1 / (2 pi Delta_s)
    float4 *d_xd = nullptr;             // [2Q]: (T hi xyz, 0), (T lo xyz, 0); T = (r_q - origin) / Delta_s
    float2 *d_freq = nullptr;           // [L]: f_l as (hi, lo)
    double2 *d_p0 = nullptr;            // [L]: p0(f_l)
    float2 *d_v = nullptr;              // [Q][L] scratch of the adjoint
    double2 *d_part = nullptr;          // [n_slab][Q][L] slab totals of the forward
};

namespace {

constexpr int kSphF = 8;                  // frequencies per lane (forward)
constexpr int kSphSeg = 32 * kSphF;       // frequencies per warp task (forward)
constexpr int kSphFwdThreads = 256;
constexpr int kSphBwdThreads = 256;       // two voxels per thread
constexpr int kSphAnchor = 32;            // adjoint: direct phase every 32 frequencies
constexpr float kTwoPi = 6.28318530717958647692f;

struct SphArgs {
    const float4 *xd;
    const float2 *freq;
    const double2 *p0;
    const float *alpha;
    float2 *u;
    double2 *part;
    const float2 *v;
    float *out;
    int nx, ny, nz, Q, L, nseg, qtile;
    long long N, slab;
    float sig_hi, sig_lo, df_hi, df_lo, inv2pids;
};

// Packed FP32 pairs (f32x2, pk2, upk2, add2, mul2, fma2) come from oat_internal.h.

// (ph + pl) ~ (ah + al)(bh + bl), the product's rounding error from an FMA, al bl dropped.
__device__ __forceinline__ void pmul(float ah, float al, float bh, float bl, float &ph, float &pl) {
    ph = __fmul_rn(ah, bh);
    pl = fmaf(ah, bl, fmaf(al, bh, fmaf(ah, bh, -ph)));
}

// ph + pl minus its nearest integer (ph - rint(ph) is exact for |ph| < 2^23).
__device__ __forceinline__ float pfrac(float ph, float pl) { return __fadd_rn(__fsub_rn(ph, rintf(ph)), pl); }

// Distance from node (x, y, z) (exact small integers) to the transducer T = th + tl, index units,
// as dh + dl: |v|^2 summed as a pair, one Newton step on the square root.
__device__ __forceinline__ void sph_dist(float x, float y, float z, const float4 &th, const float4 &tl, float &dh,
                                         float &dl) {
    const float c[3] = {x, y, z}, h[3] = {th.x, th.y, th.z}, l[3] = {tl.x, tl.y, tl.z};
    float S = 0.f, E = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float s, e;
        two_sum(c[d], -h[d], s, e);
        e = __fsub_rn(e, l[d]);
        const float p = __fmul_rn(s, s);
        const float pe = fmaf(__fmul_rn(2.f, s), e, fmaf(s, s, -p));
        float t;
        two_sum(S, p, S, t);
        E = __fadd_rn(E, __fadd_rn(t, pe));
    }
    dh = sqrtf(S);
    const float r = __fmul_rn(dh, dh), re = fmaf(dh, dh, -r);
    dl = __fdiv_rn(__fadd_rn(__fsub_rn(__fsub_rn(S, r), re), E), __fmul_rn(2.f, dh));
}

__global__ void __launch_bounds__(kSphFwdThreads, 3) k_sph_fwd(SphArgs a) {
    const int lane = threadIdx.x & 31;
    const int task = blockIdx.x * (kSphFwdThreads / 32) + (threadIdx.x >> 5);
    if (task >= a.Q * a.nseg) return;   // whole warps only; the kernel has no block barrier
    const long long v0 = (long long)blockIdx.y * a.slab, v1 = min(a.N, v0 + a.slab);
    const int q = task / a.nseg;
    const int l0 = (task - q * a.nseg) * kSphSeg + lane * kSphF;
    const float2 f0 = __ldg(a.freq + min(l0, a.L - 1));   // lanes past L compute but never store
    static_assert(kSphF == 8, "the packed loop pairs frequencies k and k + 4");
    float Sr[kSphF], Si[kSphF], Cr[kSphF], Ci[kSphF];
    f32x2 T2r[kSphF / 2], T2i[kSphF / 2];   // (frequency k, frequency k + 4) partial sums
#pragma unroll
    for (int k = 0; k < kSphF; ++k) { Sr[k] = Si[k] = Cr[k] = Ci[k] = 0.f; }
#pragma unroll
    for (int k = 0; k < kSphF / 2; ++k) { T2r[k] = 0ull; T2i[k] = 0ull; }
    // this lane's voxel of the current chunk of 32
    int ix, iy, iz;
    {
        const long long n = v0 + lane, nxy = (long long)a.nx * a.ny;
        ix = (int)(n % a.nx); iy = (int)((n / a.nx) % a.ny); iz = (int)(n / nxy);
    }
    int chunk = 0;
    for (long long base = v0; base < v1; base += 32, ++chunk) {
        float tauh = 0.f, taul = 0.f, w = 0.f, zr = 1.f, zi = 0.f, z4r = 1.f, z4i = 0.f;
        if (base + lane < v1) {
            const float al = __ldg(a.alpha + base + lane);
            const float4 th = __ldg(a.xd + 2 * q), tl = __ldg(a.xd + 2 * q + 1);   // L1 hits
            float dh, dl;
            sph_dist((float)ix, (float)iy, (float)iz, th, tl, dh, dl);
            pmul(dh, dl, a.sig_hi, a.sig_lo, tauh, taul);
            w = __fdiv_rn(__fmul_rn(al, a.inv2pids), dh);          // alpha / (2 pi d)
            float ph, pl, s, c;
            pmul(a.df_hi, a.df_lo, tauh, taul, ph, pl);
            sincospif(2.f * pfrac(ph, pl), &s, &c);
            zr = c; zi = -s;                                        // exp(-j 2 pi df tau)
            pmul(4.f * a.df_hi, 4.f * a.df_lo, tauh, taul, ph, pl);
            sincospif(2.f * pfrac(ph, pl), &s, &c);
            z4r = c; z4i = -s;                                      // exp(-j 2 pi 4 df tau)
        }
        ix += 32;
        while (ix >= a.nx) {
            ix -= a.nx;
            if (++iy >= a.ny) { iy = 0; ++iz; }
        }
        for (int j = 0; j < 32; ++j) {
            const float vth = __shfl_sync(0xffffffffu, tauh, j), vtl = __shfl_sync(0xffffffffu, taul, j);
            const float vw = __shfl_sync(0xffffffffu, w, j);
            const float vzr = __shfl_sync(0xffffffffu, zr, j), vzi = __shfl_sync(0xffffffffu, zi, j);
            const float v4r = __shfl_sync(0xffffffffu, z4r, j), v4i = __shfl_sync(0xffffffffu, z4i, j);
            float ph, pl, s, c;
            pmul(f0.x, f0.y, vth, vtl, ph, pl);
            __sincosf(kTwoPi * pfrac(ph, pl), &s, &c);
            const float er0 = vw * c, ei0 = -vw * s;                 // w exp(-j 2 pi f_l0 tau)
            const float er4 = fmaf(er0, v4r, -ei0 * v4i), ei4 = fmaf(er0, v4i, ei0 * v4r);   // ... f_l0+4
            // frequencies k and k + 4 side by side.  E_1 = E_0 z by one packed complex rotation;
            // then E_{k+1} = 2 cos(theta) E_k - E_{k-1} (z = exp(-j theta), so E_{k+1} + E_{k-1} =
            // (z + 1/z) E_k), two scalar FMAs with a negated addend per step and component: half
            // the FMA-pipe work of a complex rotation, on a pipe that bounds this kernel.  Over
            // two steps its rounding stays within a few ulp of |E|.
            static_assert(kSphF / 2 == 4, "E_0 .. E_3 below");
            const f32x2 Er = pk2(er0, er4), Ei = pk2(ei0, ei4);
            const f32x2 Zr = pk2(vzr, vzr), Zi = pk2(vzi, vzi), NZi = pk2(-vzi, -vzi);
            T2r[0] = add2(T2r[0], Er); T2i[0] = add2(T2i[0], Ei);
            const f32x2 E1r = fma2(Er, Zr, mul2(Ei, NZi));
            const f32x2 E1i = fma2(Er, Zi, mul2(Ei, Zr));
            T2r[1] = add2(T2r[1], E1r); T2i[1] = add2(T2i[1], E1i);
            const float c2 = 2.f * vzr;
            float a0r, a4r, a0i, a4i, b0r, b4r, b0i, b4i;
            upk2(Er, a0r, a4r); upk2(Ei, a0i, a4i); upk2(E1r, b0r, b4r); upk2(E1i, b0i, b4i);
            const float c0r = fmaf(c2, b0r, -a0r), c4r = fmaf(c2, b4r, -a4r);
            const float c0i = fmaf(c2, b0i, -a0i), c4i = fmaf(c2, b4i, -a4i);
            T2r[2] = add2(T2r[2], pk2(c0r, c4r)); T2i[2] = add2(T2i[2], pk2(c0i, c4i));
            const float d0r = fmaf(c2, c0r, -b0r), d4r = fmaf(c2, c4r, -b4r);
            const float d0i = fmaf(c2, c0i, -b0i), d4i = fmaf(c2, c4i, -b4i);
            T2r[3] = add2(T2r[3], pk2(d0r, d4r)); T2i[3] = add2(T2i[3], pk2(d0i, d4i));
        }
        if ((chunk & 3) == 3 || base + 32 >= v1) {
#pragma unroll
            for (int k = 0; k < kSphF / 2; ++k) {
                float lo, hi, e;
                upk2(T2r[k], lo, hi);
                two_sum(Sr[k], lo, Sr[k], e); Cr[k] += e;
                two_sum(Sr[k + 4], hi, Sr[k + 4], e); Cr[k + 4] += e;
                upk2(T2i[k], lo, hi);
                two_sum(Si[k], lo, Si[k], e); Ci[k] += e;
                two_sum(Si[k + 4], hi, Si[k + 4], e); Ci[k + 4] += e;
                T2r[k] = 0ull; T2i[k] = 0ull;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kSphF; ++k) {
        const int l = l0 + k;
        if (l < a.L)
            a.part[((size_t)blockIdx.y * a.Q + q) * a.L + l] =
                make_double2((double)Sr[k] + (double)Cr[k], (double)Si[k] + (double)Ci[k]);
    }
}

__global__ void k_sph_reduce(const double2 *__restrict__ part, const double2 *__restrict__ p0, float2 *__restrict__ u,
                             long long n, int L, int n_slab) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int b = 0; b < n_slab; ++b) {
            const double2 t = part[(size_t)b * n + i];
            sr += t.x; si += t.y;
        }
        const double2 p = p0[i % L];
        u[i] = make_float2((float)(p.x * sr - p.y * si), (float)(p.x * si + p.y * sr));
    }
}

__global__ void k_sph_conj(const float2 *__restrict__ u, const double2 *__restrict__ p0, float2 *__restrict__ v,
                           long long n, int L) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 x = u[i];
        const double2 p = p0[i % L];
        v[i] = make_float2((float)((double)x.x * p.x + (double)x.y * p.y), (float)((double)x.y * p.x - (double)x.x * p.y));
    }
}

__global__ void __launch_bounds__(kSphBwdThreads) k_sph_bwd(SphArgs a) {
    extern __shared__ ulonglong2 sv[];   // [qtile][L]: (v_re, v_re), (-v_im, -v_im) as packed pairs
    const long long n0 = ((long long)blockIdx.x * kSphBwdThreads + threadIdx.x) * 2;
    float px[2], py[2], pz[2];
    bool ok[2];
    const long long nxy = (long long)a.nx * a.ny;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const long long n = n0 + v;
        ok[v] = n < a.N;
        const long long m = ok[v] ? n : 0;
        px[v] = (float)(m % a.nx);
        py[v] = (float)((m / a.nx) % a.ny);
        pz[v] = (float)(m / nxy);
    }
    float S[2] = {0.f, 0.f}, C[2] = {0.f, 0.f};
    for (int q0 = 0; q0 < a.Q; q0 += a.qtile) {
        const int nq = min(a.qtile, a.Q - q0);
        __syncthreads();
        const float2 *src = a.v + (size_t)q0 * a.L;
        for (int i = threadIdx.x; i < nq * a.L; i += blockDim.x) {
            const float2 y = src[i];
            ulonglong2 t;
            t.x = pk2(y.x, y.x);
            t.y = pk2(-y.y, -y.y);
            sv[i] = t;
        }
        __syncthreads();
        for (int t = 0; t < nq; ++t) {
            const int q = q0 + t;
            const float4 th = __ldg(a.xd + 2 * q), tl = __ldg(a.xd + 2 * q + 1);
            float tauh[2], taul[2], w[2], zr[2], zi[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                float dh, dl, ph, pl, s, c;
                sph_dist(px[v], py[v], pz[v], th, tl, dh, dl);
                pmul(dh, dl, a.sig_hi, a.sig_lo, tauh[v], taul[v]);
                w[v] = __fdiv_rn(a.inv2pids, dh);                    // 1 / (2 pi d)
                pmul(a.df_hi, a.df_lo, tauh[v], taul[v], ph, pl);
                sincospif(2.f * pfrac(ph, pl), &s, &c);
                zr[v] = c; zi[v] = s;                                 // exp(+j 2 pi df tau)
            }
            // the two voxels side by side in packed pairs
            const f32x2 Zr = pk2(zr[0], zr[1]), Zi = pk2(zi[0], zi[1]), NZi = pk2(-zi[0], -zi[1]);
            f32x2 acc = 0ull;
            const ulonglong2 *row = sv + t * a.L;
            for (int la = 0; la < a.L; la += kSphAnchor) {
                const float2 fa = __ldg(a.freq + la);
                float er[2], ei[2];
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    float ph, pl, s, c;
                    pmul(fa.x, fa.y, tauh[v], taul[v], ph, pl);
                    __sincosf(kTwoPi * pfrac(ph, pl), &s, &c);
                    er[v] = c; ei[v] = s;                             // exp(+j 2 pi f_la tau)
                }
                f32x2 Er = pk2(er[0], er[1]), Ei = pk2(ei[0], ei[1]);
                const int cnt = min(kSphAnchor, a.L - la);
                const ulonglong2 *rv = row + la;
                // Re(v e) = v_re e_re - v_im e_im; e <- e z
#define OAT_SPH_STEP(Y)                                        \
    {                                                          \
        acc = fma2((Y).x, Er, acc);                            \
        acc = fma2((Y).y, Ei, acc);                            \
        const f32x2 nr = fma2(Er, Zr, mul2(Ei, NZi));          \
        Ei = fma2(Er, Zi, mul2(Ei, Zr));                       \
        Er = nr;                                               \
    }
                if (cnt == kSphAnchor) {
#pragma unroll 8
                    for (int k = 0; k < kSphAnchor; ++k) OAT_SPH_STEP(rv[k])
                } else {
                    for (int k = 0; k < cnt; ++k) OAT_SPH_STEP(rv[k])
                }
#undef OAT_SPH_STEP
            }
            float acc0, acc1;
            upk2(acc, acc0, acc1);
            const float accv[2] = {acc0, acc1};
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                float e;
                two_sum(S[v], w[v] * accv[v], S[v], e);
                C[v] += e;
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 2; ++v)
        if (ok[v]) a.out[n0 + v] = S[v] + C[v];
}

SphArgs sph_args(const SphPlan &p) {
    SphArgs a{};
    a.xd = p.d_xd; a.freq = p.d_freq; a.p0 = p.d_p0;
    a.nx = p.nx; a.ny = p.ny; a.nz = p.nz; a.Q = p.Q; a.L = p.L; a.nseg = p.nseg; a.qtile = p.qtile;
    a.N = p.N; a.slab = p.slab;
    a.sig_hi = p.sig_hi; a.sig_lo = p.sig_lo; a.df_hi = p.df_hi; a.df_lo = p.df_lo; a.inv2pids = p.inv2pids;
    return a;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

void pair_split(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

void sph_free(SphPlan *p) {
    if (!p) return;
    if (p->d_xd) cudaFree(p->d_xd);
    if (p->d_freq) cudaFree(p->d_freq);
    if (p->d_p0) cudaFree(p->d_p0);
    if (p->d_v) cudaFree(p->d_v);
    if (p->d_part) cudaFree(p->d_part);
    delete p;
}

struct SphDevice {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit SphDevice(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) err = cudaSetDevice(dev);
    }
    ~SphDevice() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace oat

using namespace oat;

extern "C" {

int oat_sph_create(const oat_geometry *geom, int n_freq, double f0_mhz, double df_mhz, const double *eir, int device,
                   oat_sph *out) {
    if (!out) return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: out is NULL");
    *out = nullptr;
    if (!geom || !geom->positions_mm) return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: NULL geometry or positions");
    const oat_geometry &g = *geom;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1 || (long long)g.nx * g.ny * g.nz >= (1LL << 31))
        return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: grid sizes must be >= 1 with nx*ny*nz < 2^31");
    if (!(g.spacing_mm > 0.0) || !std::isfinite(g.spacing_mm) || !(g.c_mm_per_us > 0.0) ||
        !std::isfinite(g.c_mm_per_us) || !std::isfinite(g.gruneisen))
        return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: spacing, speed of sound and Gruneisen must be finite, "
                                              "spacing and speed > 0");
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(g.origin_mm[d])) return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: non-finite origin");
    if (g.n_transducers < 1) return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: n_transducers must be >= 1");
    if (n_freq < 1 || n_freq > 12800) return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: n_freq must be in 1 .. 12800");
    if (!(f0_mhz > 0.0) || !std::isfinite(f0_mhz) || !(df_mhz >= 0.0) || !std::isfinite(df_mhz) ||
        (n_freq > 1 && !(df_mhz > 0.0)) || !std::isfinite(f0_mhz + (n_freq - 1) * df_mhz))
        return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: need f0 > 0 and df > 0 (df >= 0 for one frequency)");
    if (eir)
        for (int i = 0; i < 2 * n_freq; ++i)
            if (!std::isfinite(eir[i])) return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: non-finite EIR value");
    const int Q = g.n_transducers, L = n_freq;
    const double ds = g.spacing_mm, c = g.c_mm_per_us;
    const int n[3] = {g.nx, g.ny, g.nz};
    std::vector<float4> xd(2 * (size_t)Q);
    for (int q = 0; q < Q; ++q) {
        const double *r = g.positions_mm + 3 * (size_t)q;
        double T[3], d2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            if (!std::isfinite(r[d])) return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: non-finite position");
            T[d] = (r[d] - g.origin_mm[d]) / ds;
            const double nearest = std::min<double>(std::max<double>(std::nearbyint(T[d]), 0.0), n[d] - 1);
            d2 += (T[d] - nearest) * (T[d] - nearest);
        }
        if (d2 < 0.25)
            return set_error(OAT_ERR_INVALID_ARG, "oat_sph_create: transducer " + std::to_string(q) +
                                                      " lies inside a spherical voxel (closer than Delta_s / 2 to a node)");
        float h[3], l[3];
        for (int d = 0; d < 3; ++d) pair_split(T[d], h[d], l[d]);
        xd[2 * (size_t)q] = make_float4(h[0], h[1], h[2], 0.f);
        xd[2 * (size_t)q + 1] = make_float4(l[0], l[1], l[2], 0.f);
    }
    std::vector<float2> freq(L);
    std::vector<double2> p0(L);
    for (int l = 0; l < L; ++l) {
        const double f = f0_mhz + l * df_mhz;
        float fh, fl;
        pair_split(f, fh, fl);
        freq[l] = make_float2(fh, fl);
        // Eq. p0f with beta c^3 / C_p = Gamma c: -j (Gamma c / f)[ds/(2c) cos x - sin x / (2 pi f)], x = pi f ds / c
        const double x = M_PI * f * ds / c;
        const double b = (g.gruneisen * c / f) * (ds / (2.0 * c) * std::cos(x) - std::sin(x) / (2.0 * M_PI * f));
        double re = 0.0, im = -b;
        if (eir) {
            const double er = eir[2 * l], ei = eir[2 * l + 1];
            const double r2 = re * er - im * ei, i2 = re * ei + im * er;
            re = r2; im = i2;
        }
        p0[l] = make_double2(re, im);
    }
    SphPlan *p = new SphPlan;
    p->device = device;
    p->nx = g.nx; p->ny = g.ny; p->nz = g.nz;
    p->N = (long long)g.nx * g.ny * g.nz;
    p->Q = Q; p->L = L;
    p->nseg = (L + kSphSeg - 1) / kSphSeg;
    p->qtile = std::max(1, std::min(64, 32768 / (int)(sizeof(ulonglong2) * L)));
    p->bwd_smem = sizeof(ulonglong2) * (size_t)p->qtile * L;
    pair_split(ds / c, p->sig_hi, p->sig_lo);
    pair_split(df_mhz, p->df_hi, p->df_lo);
    p->inv2pids = (float)(1.0 / (2.0 * M_PI * ds));
    SphDevice dg(device);
    if (dg.err != cudaSuccess) {
        delete p;
        return set_error(OAT_ERR_CUDA, std::string("oat_sph_create: cudaSetDevice: ") + cudaGetErrorString(dg.err));
    }
    cudaError_t e = cudaSuccess;
    const char *what = "";
    auto step = [&](cudaError_t r, const char *w) {
        if (e == cudaSuccess && r != cudaSuccess) { e = r; what = w; }
    };
    // forward slabs: enough (warp task, slab) work items for about 16 waves of resident blocks,
    // slabs of at least 8192 voxels, slab totals within 1 GiB
    {
        int sms = 1, per_sm = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sph_fwd, kSphFwdThreads, 0);
        const long long tasks = (long long)Q * p->nseg;
        const long long want_warps = 16LL * sms * std::max(per_sm, 1) * (kSphFwdThreads / 32);
        long long ns = (want_warps + tasks - 1) / tasks;
        ns = std::min(ns, std::max(1LL, p->N / 8192));
        ns = std::min(ns, 65535LL);
        ns = std::min(ns, std::max(1LL, (1LL << 30) / (long long)(sizeof(double2) * (size_t)Q * L)));
        p->slab = ((p->N + ns - 1) / ns + 31) / 32 * 32;
        p->n_slab = (int)((p->N + p->slab - 1) / p->slab);
        cudaGetLastError();
    }
    step(cudaMalloc(&p->d_xd, sizeof(float4) * xd.size()), "cudaMalloc(transducers)");
    if (e == cudaSuccess)
        step(cudaMalloc(&p->d_part, sizeof(double2) * (size_t)p->n_slab * Q * L), "cudaMalloc(forward slab totals)");
    if (e == cudaSuccess) step(cudaMalloc(&p->d_freq, sizeof(float2) * L), "cudaMalloc(frequencies)");
    if (e == cudaSuccess) step(cudaMalloc(&p->d_p0, sizeof(double2) * L), "cudaMalloc(p0)");
    if (e == cudaSuccess) step(cudaMalloc(&p->d_v, sizeof(float2) * (size_t)Q * L), "cudaMalloc(adjoint scratch)");
    if (e == cudaSuccess) step(cudaMemcpy(p->d_xd, xd.data(), sizeof(float4) * xd.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
    if (e == cudaSuccess) step(cudaMemcpy(p->d_freq, freq.data(), sizeof(float2) * L, cudaMemcpyHostToDevice), "cudaMemcpy");
    if (e == cudaSuccess) step(cudaMemcpy(p->d_p0, p0.data(), sizeof(double2) * L, cudaMemcpyHostToDevice), "cudaMemcpy");
    if (e == cudaSuccess)
        step(cudaFuncSetAttribute(k_sph_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->bwd_smem),
             "cudaFuncSetAttribute");
    if (e != cudaSuccess) {
        const int code = e == cudaErrorMemoryAllocation ? OAT_ERR_OOM : OAT_ERR_CUDA;
        sph_free(p);
        cudaGetLastError();
        return set_error(code, std::string("oat_sph_create: ") + what + ": " + cudaGetErrorString(e));
    }
    *out = reinterpret_cast<oat_sph>(p);
    return OAT_OK;
}

int oat_sph_project(oat_sph op, const float *d_alpha, float *d_u, void *stream) {
    SphPlan *p = reinterpret_cast<SphPlan *>(op);
    if (!p || !d_alpha || !d_u) return set_error(OAT_ERR_INVALID_ARG, "oat_sph_project: NULL operator or buffer");
    if (!aligned16(d_alpha) || !aligned16(d_u))
        return set_error(OAT_ERR_INVALID_ARG, "oat_sph_project: buffers must be 16-byte aligned");
    SphDevice dg(p->device);
    if (dg.err != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_sph_project: ") + cudaGetErrorString(dg.err));
    SphArgs a = sph_args(*p);
    a.alpha = d_alpha;
    a.part = p->d_part;
    const cudaStream_t s = (cudaStream_t)stream;
    const long long warps = (long long)p->Q * p->nseg;
    const dim3 grid((unsigned)((warps + kSphFwdThreads / 32 - 1) / (kSphFwdThreads / 32)), (unsigned)p->n_slab);
    k_sph_fwd<<<grid, kSphFwdThreads, 0, s>>>(a);
    const long long M = (long long)p->Q * p->L;
    k_sph_reduce<<<(unsigned)std::min<long long>((M + 255) / 256, 8LL * current_sm_count()), 256, 0, s>>>(
        p->d_part, p->d_p0, reinterpret_cast<float2 *>(d_u), M, p->L, p->n_slab);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("oat_sph_project: ") + cudaGetErrorString(e));
}

int oat_sph_backproject(oat_sph op, const float *d_u, float *d_alpha, void *stream) {
    SphPlan *p = reinterpret_cast<SphPlan *>(op);
    if (!p || !d_alpha || !d_u) return set_error(OAT_ERR_INVALID_ARG, "oat_sph_backproject: NULL operator or buffer");
    if (!aligned16(d_alpha) || !aligned16(d_u))
        return set_error(OAT_ERR_INVALID_ARG, "oat_sph_backproject: buffers must be 16-byte aligned");
    SphDevice dg(p->device);
    if (dg.err != cudaSuccess)
        return set_error(OAT_ERR_CUDA, std::string("oat_sph_backproject: ") + cudaGetErrorString(dg.err));
    const cudaStream_t s = (cudaStream_t)stream;
    const long long M = (long long)p->Q * p->L;
    k_sph_conj<<<(unsigned)std::min<long long>((M + 255) / 256, 8LL * current_sm_count()), 256, 0, s>>>(
        reinterpret_cast<const float2 *>(d_u), p->d_p0, p->d_v, M, p->L);
    SphArgs a = sph_args(*p);
    a.v = p->d_v;
    a.out = d_alpha;
    const unsigned blocks = (unsigned)((p->N + 2 * kSphBwdThreads - 1) / (2 * kSphBwdThreads));
    k_sph_bwd<<<blocks, kSphBwdThreads, p->bwd_smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK
                            : set_error(OAT_ERR_CUDA, std::string("oat_sph_backproject: ") + cudaGetErrorString(e));
}

int oat_sph_destroy(oat_sph op) {
    SphPlan *p = reinterpret_cast<SphPlan *>(op);
    if (!p) return OAT_OK;
    SphDevice dg(p->device);
    cudaDeviceSynchronize();
    sph_free(p);
    return OAT_OK;
}

}  // extern "C"
