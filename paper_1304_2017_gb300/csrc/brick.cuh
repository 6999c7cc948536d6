// Brick enumeration shared by the projector and the backprojector.
//
// The cell range [-1, n-1]^3 (cell m = [m, m+1)^3 in grid-index units; cells -1 and n-1 hold
// the points whose stencil is half outside the grid) is tiled by bricks of B^3 cells.  A
// lattice point belongs to the brick containing floor(P).  For one brick and one transducer
// the lattice points that can lie in the brick are found through the brick's bounding sphere
// (centre c, radius rb):
//   shells   |rho_k - |c - r_q|| <= rb                                (triangle inequality)
//   rings    |theta_i - theta_c| <= gamma_k, the half-angle of the cone through the circle in
//            which shell k cuts the sphere
//   points   the azimuth window in which the ring is within rb of c (exact point-to-ring
//            distance); up to two index ranges because phi wraps at 2 pi.
// All windows carry a small margin; every candidate is then tested exactly with floor(P), so
// the windows only need to be conservative.
#pragma once

#include "oat_internal.h"

namespace oat {

constexpr float kTwoPiF = 6.28318530717958647692f;

// Brick seen from one transducer (local frame of the transducer, index units).
struct __align__(16) BrickView {
    float ex[3], ey[3], ez[3];
    float wz0;     // (c - O) . e_z : axial coordinate of the centre about the global origin
    float rw;      // distance of the centre from the transducer axis
    float d;       // distance of the centre from the transducer
    float thc;     // polar angle of the centre (from e_z)
    float phc;     // azimuth of the centre in [0, 2 pi)
    float m[3];    // |(e_x[d], e_y[d])|: a ring of radius a moves coordinate d by a m[d] cos(phi - psi[d])
    float psi[3];
    int cls, k0, k1;
};

__device__ __forceinline__ void brick_view(const Xdcr &x, const float O[3], const float c[3], float rb, float R0,
                                           float dR, int K, BrickView &v) {
#pragma unroll
    for (int d = 0; d < 3; ++d) { v.ex[d] = x.ex[d]; v.ey[d] = x.ey[d]; v.ez[d] = x.ez[d]; }
    const float c0 = c[0] - O[0], c1 = c[1] - O[1], c2 = c[2] - O[2];
    const float vx = c0 * x.ex[0] + c1 * x.ex[1] + c2 * x.ex[2];
    const float vy = c0 * x.ey[0] + c1 * x.ey[1] + c2 * x.ey[2];
    v.wz0 = c0 * x.ez[0] + c1 * x.ez[1] + c2 * x.ez[2];
    const float vz = v.wz0 + x.dist;
    const float rw2 = vx * vx + vy * vy;
    v.rw = sqrtf(rw2);
    v.d = sqrtf(rw2 + vz * vz);
    v.k0 = max(0, (int)ceilf((v.d - rb - R0) / dR));
    v.k1 = min(K - 1, (int)floorf((v.d + rb - R0) / dR));
    v.thc = atan2f(v.rw, vz);
    float ph = atan2f(vy, vx);
    v.phc = ph < 0.f ? ph + kTwoPiF : ph;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        v.m[d] = sqrtf(x.ex[d] * x.ex[d] + x.ey[d] * x.ey[d]);
        v.psi[d] = atan2f(x.ey[d], x.ex[d]);
    }
    v.cls = x.cls;
}

// Rings of shell k (radius Rk, nr rings) that can meet the bounding sphere.
__device__ __forceinline__ bool shell_ring_range(const BrickView &v, float Rk, int nr, float rb2, int &ilo, int &ihi) {
    if (nr <= 1) return false;
    const float dd = Rk - v.d;
    const float s2 = __fdividef(rb2 - dd * dd, 4.f * Rk * v.d);   // sin^2(gamma / 2)
    if (!(s2 > 0.f)) return false;
    const float gam = s2 >= 1.f ? 3.14159265f : 2.f * asinf(sqrtf(s2));
    ilo = max(1, (int)ceilf(Rk * (v.thc - gam) - 0.01f));
    ihi = min(nr - 1, (int)floorf(Rk * (v.thc + gam) + 0.01f));
    return ilo <= ihi;
}

// arccos(x), |x| <= 1, by Hastings' approximation (Abramowitz and Stegun, Handbook of
// Mathematical Functions, 4.4.45): acos(x) ~ sqrt(1 - x) (a0 + a1 x + a2 x^2 + a3 x^3) on [0, 1]
// and pi - acos(-x) below 0; absolute error below 7e-5 rad.  Used only for the azimuth windows,
// whose 2e-3 rad margins cover it.
__device__ __forceinline__ float acos_window(float x) {
    const float ax = fminf(fabsf(x), 1.f);
    float p = fmaf(ax, -0.0187293f, 0.0742610f);
    p = fmaf(ax, p, -0.2121144f);
    p = fmaf(ax, p, 1.5707288f);
    const float t = fmaxf(1.f - ax, 1e-30f);
    const float r = t * rsqrtf(t) * p;
    return x < 0.f ? 3.14159265f - r : r;
}

// Azimuth index ranges [a0, a1] and [b0, b1] (either may be empty, lo > hi; b holds the part
// past 2 pi) of ring r (centre C) whose points can lie in the box lo <= P < hi: the window
// |phi - phi_c| <= 2 asin(sqrt(rem / (4 a r_w))) in which the ring is within rb of the brick
// centre (exact point-to-ring distance), shrunk axis by axis to the hull of the azimuths at
// which the ring's coordinate d = C_d + a m_d cos(phi - psi_d) lies in [lo_d, hi_d] (two arcs
// per axis from two arccosines; their hull inside the window keeps the window one interval).
// Margins of 1e-3 grid units and 2e-3 rad keep it conservative (the arccosines come from
// acos_window, the reciprocals from the approximate division, 2 ulp); candidates are then tested
// exactly with their cells.
__device__ __forceinline__ bool ring_box_ranges(const BrickView &v, const Ring &r, float3 C, float rb2,
                                                const float lo[3], const float hi[3], int &a0, int &a1, int &b0,
                                                int &b1) {
    a0 = 0; a1 = -1; b0 = 0; b1 = -1;
    if (r.nj == 0) return false;
    const float dz = v.wz0 - r.h;
    const float dr = v.rw - r.a;
    const float rem = rb2 - dz * dz - dr * dr;
    if (!(rem > 0.f)) return false;
    const float den = 4.f * r.a * v.rw;
    float w0 = 0.f, w1 = kTwoPiF;
    if (den > 1e-12f && rem < den) {
        const float delta = acos_window(1.f - 2.f * (rem / den)) + 2e-3f;   // 2 asin(sqrt(rem / den))
        if (delta < 3.1f) { w0 = v.phc - delta; w1 = v.phc + delta; }
    }
    const float Cd[3] = {C.x, C.y, C.z};
    constexpr float kPi = 3.14159265358979f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float M = r.a * v.m[d];
        if (M < 1e-4f) {
            if (Cd[d] < lo[d] - M - 1e-3f || Cd[d] > hi[d] + M + 1e-3f) return false;
            continue;
        }
        const float inv = __fdividef(1.f, M);
        const float cl = (lo[d] - 1e-3f - Cd[d]) * inv, ch = (hi[d] + 1e-3f - Cd[d]) * inv;
        if (ch < -1.f || cl > 1.f) return false;
        if (cl <= -1.f && ch >= 1.f) continue;
        const float ah = ch >= 1.f ? 0.f : acos_window(ch);
        const float al = cl <= -1.f ? kPi : acos_window(cl);
        const float sh = kTwoPiF * floorf((w0 - v.psi[d] + kPi) * (1.f / kTwoPiF));
        const float x0 = w0 - v.psi[d] - sh, x1 = w1 - v.psi[d] - sh;   // x0 in [-pi, pi)
        float hl = 1e30f, hh = -1e30f;
        const float p0[4] = {-al, ah, kTwoPiF - al, kTwoPiF + ah};
        const float p1[4] = {-ah, al, kTwoPiF - ah, kTwoPiF + al};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float l = fmaxf(p0[s], x0), h = fminf(p1[s], x1);
            if (l <= h) { hl = fminf(hl, l); hh = fmaxf(hh, h); }
        }
        if (hl > hh) return false;
        w0 = hl + v.psi[d] + sh;
        w1 = hh + v.psi[d] + sh;
    }
    w0 -= 2e-3f; w1 += 2e-3f;
    if (w1 - w0 >= kTwoPiF - 1e-6f) { a1 = r.nj - 1; return true; }
    const float sh = kTwoPiF * floorf(w0 * (1.f / kTwoPiF));
    w0 -= sh; w1 -= sh;   // w0 in [0, 2 pi)
    const float inv = __fdividef(1.f, r.dphi);
    a0 = max(0, (int)ceilf(w0 * inv));
    a1 = min(r.nj - 1, (int)floorf(w1 * inv));
    if (w1 >= kTwoPiF) {
        b0 = 0;
        b1 = min(r.nj - 1, (int)floorf((w1 - kTwoPiF) * inv));
    }
    return true;
}

// ---------------------------------------------------------------------------- candidates
// A warp enumerates the candidates of one unit -- a transducer and kShells consecutive shells --
// in three levels:
//   rings     the units' rings, flattened over its shells, one lane per ring: the ring's azimuth
//             windows clipped to the brick (ring_windows);
//   segments  the part of a window that shares one anchor (j >> ash): up to 32 points.  One lane
//             per segment computes the anchor and fills a slot (segment_chunk);
//   points    the segments' points spread evenly over the lanes (segment_point).
constexpr int kShells = 4;

// Shells of a unit: lane s < kShells takes shell kb + s (if <= k1 and its rings can meet the
// brick's bounding sphere): first ring gbase (in the ring table) and ring count n.  Returns the
// unit's ring count; p0..p2 = inclusive prefixes of the ring counts of shells 0..2.
// Warp-collective.
__device__ __forceinline__ int unit_shells(int n, int lane, int &p0, int &p1, int &p2) {
    int incl = n;
#pragma unroll
    for (int o = 1; o < kShells; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    p0 = __shfl_sync(0xffffffffu, incl, 0);
    p1 = __shfl_sync(0xffffffffu, incl, 1);
    p2 = __shfl_sync(0xffffffffu, incl, 2);
    return __shfl_sync(0xffffffffu, incl, kShells - 1);
}

// Ring fi of a unit's flattened list: its shell s and its index in the ring table (-1 past the
// end T).  gbase: lane s holds shell s's first ring.  Warp-collective.
__device__ __forceinline__ int unit_ring(int fi, int T, int p0, int p1, int p2, int gbase, int &s) {
    s = (fi >= p0) + (fi >= p1) + (fi >= p2);
    const int before = s == 0 ? 0 : (s == 1 ? p0 : (s == 2 ? p1 : p2));
    const int g = __shfl_sync(0xffffffffu, gbase, s) + (fi - before);
    return fi < T ? g : -1;
}

// One anchor segment of a warp's chunk.
struct __align__(16) SegSlot {
    float f[3];          // anchor fraction A - I
    int I[3];            // anchor cell I, relative to the brick's lowest cell L
    float xa, ya;        // anchor local coordinates (hi parts)
    float dphi, dphi_lo;
    int mp;              // m = j - j_A of the segment's first point | shell << 6 |
                         // position of that point in the chunk's candidate list << 8
    float w;             // the ring's point weight over Delta_s^2 (1 with uniform weights)
};

// Anchor segments (runs of points sharing an anchor, anchors every 2^sh points) of the index
// range lo .. lo + n - 1.
__device__ __forceinline__ int anchor_segments(int lo, int n, int sh) {
    return n > 0 ? ((lo + n - 1) >> sh) - (lo >> sh) + 1 : 0;
}

// Lane's ring gidx (none if < 0): its windows [wa0, wa0 + wna) and [wb0, wb0 + wnb) clipped to
// the brick, and the inclusive prefix over lanes of their anchor segments.  Returns the batch's
// segment count.  Warp-collective.
__device__ __forceinline__ int ring_windows(const BrickView &v, const Ring *__restrict__ rings, int gidx,
                                            const float O[3], float rb2, const float blo[3], const float bhi[3],
                                            int lane, int &wa0, int &wna, int &wb0, int &wnb, int &sincl) {
    int a0 = 0, a1 = -1, b0 = 0, b1 = -1, sh = 0;
    if (gidx >= 0) {
        const Ring r = rings[gidx];
        ring_box_ranges(v, r, ring_base(O, v.ez, r.h), rb2, blo, bhi, a0, a1, b0, b1);
        sh = r.ash;
    }
    wa0 = a0; wna = max(0, a1 - a0 + 1);
    wb0 = b0; wnb = max(0, b1 - b0 + 1);
    int incl = anchor_segments(wa0, wna, sh) + anchor_segments(wb0, wnb, sh);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    sincl = incl;
    return __shfl_sync(0xffffffffu, incl, 31);
}

// Segments sc .. sc + 31 of the batch, one per lane: anchor and slot ws[lane].  Returns the
// chunk's number of candidates; my_start = first candidate of slot `lane` (INT_MAX if none);
// used = segments taken.  With ONE_SHELL the chunk stops before the first segment of another
// shell than segment sc's (segments come in shell order), so that every candidate of the chunk
// has shell cshell.  Warp-collective.
template <bool ONE_SHELL>
__device__ __forceinline__ int segment_chunk(const Xdcr *__restrict__ xq, const Ring *__restrict__ rings,
                                             const float4 *__restrict__ anchors, const float *__restrict__ ring_w,
                                             int gidx, int shell,
                                             const float Oh[3], const float Ol[3], const int L[3], int sc, int S,
                                             int lane, int wa0, int wna, int wb0, int wnb, int sincl, SegSlot *ws,
                                             int &my_start, int &used, int &cshell) {
    const int g = sc + lane;
    // owning ring lane: the number of lanes whose inclusive prefix is <= g
    int r = 0;
#pragma unroll
    for (int b = 16; b >= 1; b >>= 1) {
        const int sv = __shfl_sync(0xffffffffu, sincl, r + b - 1);
        if (sv <= g) r += b;
    }
    const int ra0 = __shfl_sync(0xffffffffu, wa0, r), rna = __shfl_sync(0xffffffffu, wna, r);
    const int rb0 = __shfl_sync(0xffffffffu, wb0, r), rnb = __shfl_sync(0xffffffffu, wnb, r);
    const int rincl = __shfl_sync(0xffffffffu, sincl, r);
    const int rg_idx = __shfl_sync(0xffffffffu, gidx, r), rshell = __shfl_sync(0xffffffffu, shell, r);
    bool take = g < S;
    cshell = __shfl_sync(0xffffffffu, rshell, 0);
    if (ONE_SHELL) take = take && rshell == cshell;
    used = __popc(__ballot_sync(0xffffffffu, take));
    int cnt = 0, j0 = 0, t = 0, sh = 0;
    if (take) {
        sh = __ldg(&rings[rg_idx].ash);
        const int nsa = anchor_segments(ra0, rna, sh), nsb = anchor_segments(rb0, rnb, sh);
        const int sg = g - (rincl - nsa - nsb);
        int lo, hi;
        if (sg < nsa) { t = (ra0 >> sh) + sg; lo = ra0; hi = ra0 + rna - 1; }
        else { t = (rb0 >> sh) + (sg - nsa); lo = rb0; hi = rb0 + rnb - 1; }
        j0 = max(lo, t << sh);
        cnt = min(hi, (t << sh) + (1 << sh) - 1) - j0 + 1;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (cnt > 0) {
        const Ring rg = rings[rg_idx];
        const float4 xy = __ldg(anchors + rg.aoff + t);
        int I[3];
        float fr[3];
        anchor_point(Oh, Ol, *xq, rg.h, rg.h_lo, xy, I, fr);
        SegSlot &sl = ws[lane];
#pragma unroll
        for (int d = 0; d < 3; ++d) { sl.f[d] = fr[d]; sl.I[d] = I[d] - L[d]; }
        sl.xa = xy.x; sl.ya = xy.z;
        sl.dphi = rg.dphi; sl.dphi_lo = rg.dphi_lo;
        sl.mp = (j0 - (t << sh)) | (rshell << 6) | ((incl - cnt) << 8);
        sl.w = ring_w ? __ldg(ring_w + rg_idx) : 1.f;
    }
    my_start = cnt > 0 ? incl - cnt : 0x7fffffff;
    __syncwarp();
    return __shfl_sync(0xffffffffu, incl, 31);
}

// Candidate f + lane of a chunk: its cell relative to the brick's lowest cell (lc), its position
// in that cell (w), its ring's weight factor (wr) and its shell within the unit (returned; -1
// for lanes past the end of the list), through the shared lattice-point functions (ex, ey: the
// transducer's frame, hi parts).  Warp-collective.
__device__ __forceinline__ int segment_point(const SegSlot *ws, int f, int lane, int my_start, int total,
                                             const float ex[3], const float ey[3], int lc[3], float w[3],
                                             float &wr) {
    const int before = __popc(__ballot_sync(0xffffffffu, my_start <= f));
    const unsigned inside =
        __reduce_or_sync(0xffffffffu, (my_start > f && my_start < f + 32) ? (1u << (my_start - f)) : 0u);
    const int cidx = f + lane;
    if (cidx >= total) return -1;
    const SegSlot &sl = ws[before - 1 + __popc(inside & ((2u << lane) - 1u))];
    const int mp = sl.mp;
    const float3 R = anchor_offset(sl.f, sl.xa, sl.ya, ex, ey, sl.dphi, sl.dphi_lo, (mp & 31) + (cidx - (mp >> 8)));
    const float fx = floorf(R.x), fy = floorf(R.y), fz = floorf(R.z);
    lc[0] = sl.I[0] + (int)fx; lc[1] = sl.I[1] + (int)fy; lc[2] = sl.I[2] + (int)fz;
    w[0] = __fsub_rn(R.x, fx); w[1] = __fsub_rn(R.y, fy); w[2] = __fsub_rn(R.z, fz);
    wr = sl.w;
    return (mp >> 6) & 3;
}

// Next unit of a warp: the warps of a block take units from a shared counter, so that a warp
// that finishes its units early takes more (the units' sizes differ by an order of magnitude
// between the edge and the middle of a brick's shell range).  Warp-collective.
__device__ __forceinline__ int next_unit(int *counter, int lane) {
    int u = 0;
    if (lane == 0) u = atomicAdd(counter, 1);
    return __shfl_sync(0xffffffffu, u, 0);
}

// Lowest cell L and cell counts E (<= bs) of brick id in a grid of nb[3] bricks (x fastest)
// tiling the cells [-1, n-1] of each axis.
__device__ __forceinline__ void brick_box(int id, const int nb[3], const int bs[3], const int n[3], int L[3], int E[3]) {
    const int b[3] = {id % nb[0], (id / nb[0]) % nb[1], id / (nb[0] * nb[1])};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        L[d] = -1 + bs[d] * b[d];
        E[d] = min(bs[d], n[d] - L[d]);
    }
}

// Power-of-two scale 2^e with |x * 2^e| <= 2^bits for every |x| <= bound (1 if bound is zero or
// not finite).  Sums are accumulated as integers in this fixed-point unit: integer addition is
// exact and associative, so the result does not depend on the order of the contributions.
__host__ __device__ __forceinline__ double pow2_scale(double bound, int bits) {
    if (!(bound > 0.0) || !(bound < 1e300)) return 1.0;
    int e = bits - (int)ceil(log2(bound));
    return ldexp(1.0, e);
}

}  // namespace oat
