// Filtered backprojection (include/oat.h, Sec. III.C, Eq. disfbp): a per-voxel gather over all
// transducers with two-tap linear interpolation in time and the first difference for dp/dt.
//
// k_fbp  one thread block per brick of 8^3 voxels, two voxels per thread (z and z + 4, whose
//        terms run side by side in packed FP32 pairs).  Transducers come in
//        tiles of 256 through shared memory; for each (brick, transducer) one thread computes,
//        in float-pair arithmetic, the distance D from the transducer to the brick centre and
//        the fractional sample index K = D ds / (c dt) - t_min / dt split into an integer and an
//        FP32 fraction.  A voxel at offset delta from the centre is at distance D + dD with
//          dD = (2 D u.delta + |delta|^2) / (D + sqrt(D^2 + 2 D u.delta + |delta|^2))
//        (u the unit vector from the transducer to the centre): every FP32 quantity stays
//        small, so k~ = K + dD ds / (c dt) is good to about 2e-6 grid units of distance (worst
//        case; 2.5e-7 rms), measured against FP64 through oat_fbp_sample_positions: the roundings of
//        the FP32 offset terms dominate, not the SFU square root and reciprocal (a Newton step on
//        each changed nothing measurable).  Per term, with w = k~ - k and
//        tau = k~ + t_min / dt,
//          {..} = 0.5 (p_{k+1} - p_k) + (p_k + w (p_{k+1} - p_k)) / tau
//        (the braces of Eq. disfbp rewritten), summed with compensation over a tile and in
//        double across tiles; every voxel is written once.  Tiles whose sample windows lie
//        inside the record (the usual case) skip the per-sample bounds tests.
//        Eq. disfbp is discontinuous where k~ crosses an integer (the sample pair k, k + 1
//        changes), so the pair must be the one the exact k~ selects.  Where the FP32 weight
//        w = k~ - k is within a guard band of 0 or 1 -- g = 1e-5 (ds / (c dt) + 1) samples, at
//        least four times the FP32 error bound of k~ -- the pair and the weight are taken from
//        k~ recomputed in double precision from the node index and the transducer position (the
//        definition of Eq. linearint).  Outside the band the FP32 floor equals the exact one.
//        The band holds about 2g of the pairs (1e-4 at the 256^3 / 65 mm scan).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <string>

#include "oat_internal.h"

namespace oat {

constexpr int kFbpB = 8;
constexpr int kFbpThreads = kFbpB * kFbpB * kFbpB / 2;   // two voxels per thread
constexpr int kFbpTile = 256;                           // transducers per tile, one per thread

static_assert(kFbpTile == kFbpThreads, "one transducer set-up per thread and tile");

struct FbpArgs {
    const float4 *xd;            // [2Q]: (T hi, w), (T lo, 0); T in index units from node (0,0,0)
    const void *p;               // [Q][K]
    float *vol;                  // [nz][ny][nx]
    int nx, ny, nz, K, Q;
    int bx, by;                  // bricks along x and y
    float sk_hi, sk_lo;          // ds / (c dt): index units -> samples, as a float pair
    float t0_hi, t0_lo;          // t_min / dt as a float pair
    int R, W;                    // staged sample windows: offset R, width W = 2 R + 1
    double scale;                // -1 / (pi Gamma c dt)
    double sk64, t0_64;          // ds / (c dt) and t_min / dt in double (exact sample positions)
    float guard;                 // half-width of the band around integers resolved in double
};

// Per (brick, transducer): unit vector u, distance D (index units), integer and fractional part
// of the sample index at the brick centre, tau at the centre, weight.
struct __align__(16) FbpQ {
    float ux, uy, uz, D;
    int kint;
    float kfrac, tau, w;
};

template <int DT>
struct DataT;
template <>
struct DataT<OAT_F32> { using T = float; };
template <>
struct DataT<OAT_F16> { using T = __half; };
template <>
struct DataT<OAT_BF16> { using T = __nv_bfloat16; };

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ FbpQ fbp_setup(const FbpArgs &a, int q, float cx, float cy, float cz) {
    const float4 hi = __ldg(a.xd + 2 * q), lo = __ldg(a.xd + 2 * q + 1);
    const float c[3] = {cx, cy, cz}, th[3] = {hi.x, hi.y, hi.z}, tl[3] = {lo.x, lo.y, lo.z};
    // v = c - T and S + E = |v|^2, float pairs
    float vh[3], S = 0.f, E = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float s, e;
        two_sum(c[d], -th[d], s, e);
        e = __fsub_rn(e, tl[d]);
        vh[d] = s;
        const float pp = __fmul_rn(s, s);
        const float pe = fmaf(__fmul_rn(2.f, s), e, fmaf(s, s, -pp));
        float t;
        two_sum(S, pp, S, t);
        E = __fadd_rn(E, __fadd_rn(t, pe));
    }
    // D = sqrt(S + E) as D0 + corr (one Newton step in float pairs)
    const float D0 = sqrtf(S);
    const float r = __fmul_rn(D0, D0), re = fmaf(D0, D0, -r);
    const float corr = __fdiv_rn(__fadd_rn(__fsub_rn(__fsub_rn(S, r), re), E), __fmul_rn(2.f, D0));
    // K = D sk - t0
    const float kp = __fmul_rn(D0, a.sk_hi);
    const float kpe = fmaf(corr, a.sk_hi, fmaf(D0, a.sk_lo, fmaf(D0, a.sk_hi, -kp)));
    float ks, ke;
    two_sum(kp, -a.t0_hi, ks, ke);
    ke = __fadd_rn(ke, __fsub_rn(kpe, a.t0_lo));
    const float fl = floorf(ks);
    FbpQ o;
    const float inv = __fdiv_rn(1.f, D0);
    o.ux = __fmul_rn(vh[0], inv); o.uy = __fmul_rn(vh[1], inv); o.uz = __fmul_rn(vh[2], inv);
    o.D = D0;
    o.kint = (int)fl;
    o.kfrac = __fadd_rn(__fsub_rn(ks, fl), ke);
    o.tau = __fadd_rn(kp, kpe);
    o.w = hi.w;
    if (!(D0 > 1e-3f) || !(D0 < 1e30f)) {
        // a transducer at the brick centre (the formula is singular there) or a non-finite
        // position: no contribution, and finite values so that every sample index stays in
        // its window
        o.ux = o.uy = o.uz = 0.f; o.D = 1.f; o.kint = 0; o.kfrac = 0.f; o.tau = 1.f; o.w = 0.f;
    }
    return o;
}

// Exact floor of |x| < 2^22 as an integer without a conversion instruction: x + 1.5 2^23 puts
// the integer in the low mantissa bits (fk is already integral, so the sum is exact).
__device__ __forceinline__ int int_of_integral(float fk) { return __float_as_int(fk + 12582912.f) - 0x4B400000; }

// Sample positions of two voxels at offsets (dx, dy, dz0|1) from the brick centre, |delta|^2 =
// dd0|1 (packed DZ, DD; dx, dy, dz are half-integers, so DD is exact): the distance change
// DDD = |r_q - r_n| - D (grid units) and KF = k~ - Q.kint, per voxel with the one-voxel form's
// operations and rounding.  The only place the kernel forms k~ (oat_fbp_sample_positions reads
// it through this function too).
__device__ __forceinline__ void fbp_kpos(const FbpQ &Q, float dx, float dy, f32x2 DZ, f32x2 DD, float sk, f32x2 &DDD,
                                         f32x2 &KF) {
    const float c = fmaf(Q.uy, dy, Q.ux * dx);
    const f32x2 UD = fma2(pk2(Q.uz, Q.uz), DZ, pk2(c, c));
    const float td = 2.f * Q.D;
    const f32x2 TT = fma2(pk2(td, td), UD, DD);
    const f32x2 DQ = pk2(Q.D, Q.D);
    const f32x2 S2 = fma2(DQ, DQ, TT);
    float s2a, s2b;
    upk2(S2, s2a, s2b);
    const f32x2 DEN = add2(DQ, mul2(S2, pk2(rsqrtf(s2a), rsqrtf(s2b))));
    float dna, dnb;
    upk2(DEN, dna, dnb);
    DDD = mul2(TT, pk2(__fdividef(1.f, dna), __fdividef(1.f, dnb)));   // distance - D
    KF = fma2(DDD, pk2(sk, sk), pk2(Q.kfrac, Q.kfrac));
}

// Sample position k~ - kint of node (ix, iy, iz) for transducer q in double precision: the
// distance from the node to the transducer (index units, T = hi + lo exactly) times ds / (c dt),
// minus t_min / dt (Eq. linearint).  Called only for pairs in the guard band.
__device__ __noinline__ double fbp_kexact(const float4 *__restrict__ xd, double sk64, double t0_64, int q, int ix,
                                          int iy, int iz, int kint) {
    const float4 hi = __ldg(xd + 2 * q), lo = __ldg(xd + 2 * q + 1);
    const double vx = (double)ix - ((double)hi.x + (double)lo.x);
    const double vy = (double)iy - ((double)hi.y + (double)lo.y);
    const double vz = (double)iz - ((double)hi.z + (double)lo.z);
    const double d = sqrt(fma(vx, vx, fma(vy, vy, vz * vz)));
    return fma(d, sk64, -t0_64) - (double)kint;
}

// Replaces the floor fk and the weight w = k~ - fk of a pair in the guard band by those of the
// exact sample position.
// The exact floor differs from the FP32 one by at most one inside the band; anything else (a
// transducer the set-up marked as contributing nothing -- its weight is zero and its FP32 values
// are placeholders --, a non-finite position) keeps the FP32 values, whose sample indices are
// known to lie in the kernel's window.
__device__ __forceinline__ void fbp_resolve(const FbpArgs &a, int q, int ix, int iy, int iz, int kint, float &fk,
                                            float &w) {
    const double ke = fbp_kexact(a.xd, a.sk64, a.t0_64, q, ix, iy, iz, kint);
    const double fe = floor(ke);
    if (fabs(fe - (double)fk) <= 1.0) {
        fk = (float)fe;
        w = (float)(ke - fe);
    }
}

// The (voxel, transducer) terms of two voxels at offsets (dx, dy, dz0|1) from the brick centre
// (packed DZ, DD): w_q {..} of Eq. disfbp for each, packed.  Per voxel the
// operations and their rounding are those of the one-voxel form: distance change dD, sample
// position k~, two-tap interpolation and first difference.  CHECK: samples outside 0 .. K-1
// count as zero (else every sample read is known to be inside).  STAGED: row is the brick's
// window of this transducer's samples in shared memory, sample kint - R + j at j (zero outside
// the record), so that sample k reads row[k - kint + R].
// A voxel whose k~ lies in the guard band takes its pair and weight from fbp_resolve
// (transducer q; the voxels are nodes (ix, iy, iz0) and (ix, iy, iz0 + 4)).
template <int MODE, typename T>
__device__ __forceinline__ f32x2 fbp_pair(const FbpArgs &a, int q, int ix, int iy, int iz0, const FbpQ &Q,
                                          const T *row, int K, float dx, float dy, f32x2 DZ, f32x2 DD, float sk,
                                          int R) {
    constexpr bool CHECK = MODE == 1, STAGED = MODE == 2;
    f32x2 DDD, KF;
    fbp_kpos(Q, dx, dy, DZ, DD, sk, DDD, KF);
    const f32x2 SK = pk2(sk, sk);
    float kfa, kfb;
    upk2(KF, kfa, kfb);
    float fka = floorf(kfa), fkb = floorf(kfb);
    const f32x2 M1 = pk2(-1.f, -1.f);
    f32x2 WGT = fma2(pk2(fka, fkb), M1, KF);                       // k~ - k
    {
        // |w - 1/2| > 1/2 - g: the weight is within g of 0 or 1, k~ within g of an integer
        float ua, ub;
        upk2(add2(WGT, pk2(-0.5f, -0.5f)), ua, ub);
        const float lim = 0.5f - a.guard;
        if (fmaxf(fabsf(ua), fabsf(ub)) > lim) {
            float wa, wb;
            upk2(WGT, wa, wb);
            if (fabsf(ua) > lim) fbp_resolve(a, q, ix, iy, iz0, Q.kint, fka, wa);
            if (fabsf(ub) > lim) fbp_resolve(a, q, ix, iy, iz0 + 4, Q.kint, fkb, wb);
            WGT = pk2(wa, wb);
        }
    }
    const int ka = (STAGED ? R : Q.kint) + int_of_integral(fka), kb = (STAGED ? R : Q.kint) + int_of_integral(fkb);
    const f32x2 TAU = fma2(DDD, SK, pk2(Q.tau, Q.tau));
    float p0a, p1a, p0b, p1b;
    if (CHECK) {
        p0a = (ka >= 0 && ka < K) ? to_f(row[ka]) : 0.f;
        p1a = (ka + 1 >= 0 && ka + 1 < K) ? to_f(row[ka + 1]) : 0.f;
        p0b = (kb >= 0 && kb < K) ? to_f(row[kb]) : 0.f;
        p1b = (kb + 1 >= 0 && kb + 1 < K) ? to_f(row[kb + 1]) : 0.f;
    } else {
        p0a = to_f(row[ka]); p1a = to_f(row[ka + 1]);
        p0b = to_f(row[kb]); p1b = to_f(row[kb + 1]);
    }
    const f32x2 P0 = pk2(p0a, p0b);
    const f32x2 DP = fma2(P0, M1, pk2(p1a, p1b));                  // p_{k+1} - p_k
    float ta, tb;
    upk2(TAU, ta, tb);
    const f32x2 IT = pk2(__fdividef(1.f, ta), __fdividef(1.f, tb));
    const f32x2 BR = fma2(fma2(WGT, DP, P0), IT, mul2(pk2(0.5f, 0.5f), DP));
    return mul2(pk2(Q.w, Q.w), BR);
}

template <int DT, bool STAGED>
__global__ void __launch_bounds__(kFbpThreads) k_fbp(FbpArgs a) {
    using T = typename DataT<DT>::T;
    __shared__ FbpQ tq[kFbpTile];
    extern __shared__ float swin[];   // STAGED: [kFbpTile][W] sample windows
    const int b = blockIdx.x;
    const int bx = b % a.bx, by = (b / a.bx) % a.by, bz = b / (a.bx * a.by);
    const int lx = threadIdx.x & 7, ly = (threadIdx.x >> 3) & 7, lz = threadIdx.x >> 6;   // lz 0..3; + 4
    const int ix = bx * kFbpB + lx, iy = by * kFbpB + ly, iz = bz * kFbpB + lz;
    const float cx = bx * kFbpB + 3.5f, cy = by * kFbpB + 3.5f, cz = bz * kFbpB + 3.5f;
    const float dx = lx - 3.5f, dy = ly - 3.5f, dz0 = lz - 3.5f, dz1 = lz + 0.5f;
    const float dxy = dx * dx + dy * dy;
    const f32x2 DZ = pk2(dz0, dz1), DD = pk2(dxy + dz0 * dz0, dxy + dz1 * dz1);
    const float sk = a.sk_hi;
    // every voxel of the brick is within rb of the centre: its sample index is within rb sk
    // (plus rounding) of the centre's
    const float reach = (3.5f * 1.7320509f + 0.01f) * sk + 1.f;
    double total0 = 0.0, total1 = 0.0;
    for (int q0 = 0; q0 < a.Q; q0 += kFbpTile) {
        const int nt = min(kFbpTile, a.Q - q0);
        __syncthreads();
        bool inside = true;
        if (threadIdx.x < nt) {
            const FbpQ Q = fbp_setup(a, q0 + threadIdx.x, cx, cy, cz);
            tq[threadIdx.x] = Q;
            const float lo = (float)Q.kint + Q.kfrac - reach, hi = (float)Q.kint + Q.kfrac + reach;
            inside = lo >= 0.f && hi <= (float)(a.K - 2);
        }
        const bool all_inside = __syncthreads_and(inside);
        const T *row = (const T *)a.p + (size_t)q0 * a.K;
        if (STAGED) {
            // each warp copies whole windows: rows t = warp, warp + 8, ...; lanes along the row
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            for (int t = warp; t < nt; t += kFbpThreads / 32) {
                const int k0 = tq[t].kint - a.R;
                const T *src = row + (size_t)t * a.K;
                for (int j = lane; j < a.W; j += 32) {
                    const int k = k0 + j;
                    swin[t * a.W + j] = (k >= 0 && k < a.K) ? to_f(src[k]) : 0.f;
                }
            }
            __syncthreads();
        }
        // compensated (Kahan) sums of the tile's terms, both voxels at once
        f32x2 S = 0ull, C = 0ull;
        const f32x2 M1 = pk2(-1.f, -1.f);
#define OAT_FBP_ACC(X)                                 \
    {                                                  \
        const f32x2 y_ = fma2(C, M1, (X));             \
        const f32x2 t_ = add2(S, y_);                  \
        C = fma2(y_, M1, fma2(S, M1, t_));             \
        S = t_;                                        \
    }
        if (STAGED) {
            for (int t = 0; t < nt; ++t)
                OAT_FBP_ACC((fbp_pair<2>(a, q0 + t, ix, iy, iz, tq[t], swin + t * a.W, a.K, dx, dy, DZ, DD, sk, a.R)))
        } else if (all_inside) {
            for (int t = 0; t < nt; ++t, row += a.K)
                OAT_FBP_ACC((fbp_pair<0>(a, q0 + t, ix, iy, iz, tq[t], row, a.K, dx, dy, DZ, DD, sk, 0)))
        } else {
            for (int t = 0; t < nt; ++t, row += a.K)
                OAT_FBP_ACC((fbp_pair<1>(a, q0 + t, ix, iy, iz, tq[t], row, a.K, dx, dy, DZ, DD, sk, 0)))
        }
#undef OAT_FBP_ACC
        float s0, s1, c0, c1;
        upk2(S, s0, s1);
        upk2(C, c0, c1);
        total0 += (double)s0 - (double)c0;
        total1 += (double)s1 - (double)c1;
    }
    if (ix < a.nx && iy < a.ny) {
        if (iz < a.nz) a.vol[((size_t)iz * a.ny + iy) * a.nx + ix] = (float)(total0 * a.scale);
        if (iz + 4 < a.nz) a.vol[((size_t)(iz + 4) * a.ny + iy) * a.nx + ix] = (float)(total1 * a.scale);
    }
}

// k~ of (node, transducer) pairs exactly as k_fbp forms it: the node's brick centre and offset,
// fbp_setup for the transducer, then fbp_kpos (the node in the first of the two packed lanes).
// out[i] = kint + KF in double (exact); NaN for a transducer index outside 0 .. Q-1.
__global__ void k_fbp_kpos(FbpArgs a, const int *__restrict__ nodes, const int *__restrict__ qs, int n, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ix = nodes[3 * i], iy = nodes[3 * i + 1], iz = nodes[3 * i + 2], q = qs[i];
    if (q < 0 || q >= a.Q) { out[i] = __longlong_as_double(0x7ff8000000000000LL); return; }
    const int bx = ix >= 0 ? ix / kFbpB : -((-ix + kFbpB - 1) / kFbpB);
    const int by = iy >= 0 ? iy / kFbpB : -((-iy + kFbpB - 1) / kFbpB);
    const int bz = iz >= 0 ? iz / kFbpB : -((-iz + kFbpB - 1) / kFbpB);
    const FbpQ Q = fbp_setup(a, q, bx * kFbpB + 3.5f, by * kFbpB + 3.5f, bz * kFbpB + 3.5f);
    const float dx = (ix - bx * kFbpB) - 3.5f, dy = (iy - by * kFbpB) - 3.5f, dz = (iz - bz * kFbpB) - 3.5f;
    const float dxy = dx * dx + dy * dy, dd = dxy + dz * dz;
    f32x2 DDD, KF;
    fbp_kpos(Q, dx, dy, pk2(dz, dz), pk2(dd, dd), a.sk_hi, DDD, KF);
    float kf, kf2;
    upk2(KF, kf, kf2);
    out[i] = (double)Q.kint + (double)kf;
}

// Half-width of the guard band in samples for sk = ds / (c dt) samples per grid unit: 1e-5 grid
// units of distance plus 1e-5 samples, at least four times the FP32 error of k~ (measured at most
// 2.2e-6 grid units of distance, FP32 rounding of the fraction included).
static double fbp_guard(double sk) { return 1e-5 * (sk + 1.0); }

static void fbp_args(const Plan &p, FbpArgs &a) {
    a.xd = p.d_fbp;
    a.nx = p.nx; a.ny = p.ny; a.nz = p.nz; a.K = p.K; a.Q = p.Q;
    a.bx = (p.nx + kFbpB - 1) / kFbpB; a.by = (p.ny + kFbpB - 1) / kFbpB;
    const double sk = p.g.spacing_mm / (p.g.c_mm_per_us * p.dt), t0 = p.g.t_min_us / p.dt;
    a.sk_hi = (float)sk; a.sk_lo = (float)(sk - (double)a.sk_hi);
    a.t0_hi = (float)t0; a.t0_lo = (float)(t0 - (double)a.t0_hi);
    a.scale = -1.0 / (M_PI * p.g.gruneisen * p.g.c_mm_per_us * p.dt);
    a.sk64 = sk; a.t0_64 = t0;
    a.guard = (float)fbp_guard(sk);
}

int launch_fbp_kpos(Plan &p, const int *nodes, const int *qs, int n, double *out, cudaStream_t s) {
    if (n == 0) return OAT_OK;
    FbpArgs a;
    fbp_args(p, a);
    a.p = nullptr; a.vol = nullptr; a.R = 0; a.W = 0;
    k_fbp_kpos<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, nodes, qs, n, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("oat_fbp_sample_positions: ") + cudaGetErrorString(e));
}

int launch_fbp(Plan &p, const void *data, float *vol, cudaStream_t s) {
    FbpArgs a;
    fbp_args(p, a);
    a.p = data; a.vol = vol;
    const int bz = (p.nz + kFbpB - 1) / kFbpB;
    const double sk = p.g.spacing_mm / (p.g.c_mm_per_us * p.dt);
    const unsigned blocks = (unsigned)((size_t)a.bx * a.by * bz);
    // every voxel of a brick lies within 3.5 sqrt(3) grid units of its centre, so its sample
    // index is within that times sk of the centre's (the kernel's reach, plus a margin): the
    // samples any brick reads for one transducer lie in kint - R .. kint + R
    const double reach = (3.5 * std::sqrt(3.0) + 0.01) * sk + 1.0;
    a.R = (int)std::ceil(reach) + 1;
    a.W = 2 * a.R + 1;
    const size_t win_bytes = sizeof(float) * (size_t)kFbpTile * a.W;
    bool staged = win_bytes <= 96 * 1024;   // else the direct (L2) reads
    if (staged) {
        cudaError_t ea = cudaSuccess;
        switch (p.g.data_dtype) {
            case OAT_F32: ea = cudaFuncSetAttribute(k_fbp<OAT_F32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_bytes); break;
            case OAT_F16: ea = cudaFuncSetAttribute(k_fbp<OAT_F16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_bytes); break;
            default: ea = cudaFuncSetAttribute(k_fbp<OAT_BF16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_bytes); break;
        }
        if (ea != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_fbp: cudaFuncSetAttribute: ") + cudaGetErrorString(ea));
    }
    const bool prof = p.profiling && p.ev_used[2] + 2 <= (int)p.ev[2].size();
    if (prof) cudaEventRecord(p.ev[2][p.ev_used[2]], s);
    const size_t sm = staged ? win_bytes : 0;
#define OAT_FBP_LAUNCH(DTV)                                                                     \
    (staged ? k_fbp<DTV, true><<<blocks, kFbpThreads, sm, s>>>(a) : k_fbp<DTV, false><<<blocks, kFbpThreads, 0, s>>>(a))
    switch (p.g.data_dtype) {
        case OAT_F32: OAT_FBP_LAUNCH(OAT_F32); break;
        case OAT_F16: OAT_FBP_LAUNCH(OAT_F16); break;
        default: OAT_FBP_LAUNCH(OAT_BF16); break;
    }
#undef OAT_FBP_LAUNCH
    if (prof) { cudaEventRecord(p.ev[2][p.ev_used[2] + 1], s); p.ev_used[2] += 2; }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("oat_fbp: k_fbp: ") + cudaGetErrorString(e));
}

}  // namespace oat
