// Internal plan layout and the device-side lattice / interpolation helpers shared by the
// projector and the backprojector.  Both directions call the same __device__ functions, so
// a lattice point has bit-identical FP32 coordinates in H and in H^T, which makes the two
// kernels exact transposes of each other up to summation order.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/oat.h"

namespace oat {

// One ring (radius class c, sample k, polar index i) of the shell lattice, in grid-index
// units (1 = Delta_s).  With rho_k = c t_k, theta_i = i dtheta, |r_q| = |transducer|:
//   h    = (rho_k cos theta_i - |r_q|) / Delta_s   axial offset of the ring centre from the
//                                                  global origin along the frame's e_z
//   a    = rho_k sin theta_i / Delta_s             ring radius
//   dphi = Delta_s / (rho_k sin theta_i)           azimuthal step (radians)
//   nj   = floor(2 pi / dphi)                      number of points on the ring
// The lattice point (k, i, j) of transducer q sits at
//   P = O + h e_z + a (cos(j dphi) e_x + sin(j dphi) e_y)     (index units)
// where O = -origin / Delta_s is the global origin in index coordinates and
// (e_x, e_y, e_z) is the transducer's local frame (Appendix).
//
// h and dphi are also kept as unevaluated sums of two floats (hi + lo, |lo| <= ulp(hi) / 2),
// for the anchors below.  The ring's anchors sit every 2^ash points, ash the largest value <= 5
// with 2^ash dphi <= 1 (so that a point is at most 1 rad of azimuth from its anchor): anchor t
// is the point j = t 2^ash, its local coordinates (a cos(j dphi), a sin(j dphi)) are table entry
// aoff + t, also as float pairs.
constexpr int kMaxAnchorShift = 5;                   // at most 32 points per anchor

struct __align__(16) Ring {
    float h, a, dphi;
    int nj;
    float h_lo, dphi_lo;
    int aoff;                 // first anchor of the ring in the anchor table
    int ash;                  // anchor spacing 2^ash points (0 .. 5)
};

// Per-transducer record: local frame (float pairs hi + lo) and |r_q| / Delta_s, radius class.
struct __align__(16) Xdcr {
    float ex[3], ey[3], ez[3];
    float ex_lo[3], ey_lo[3], ez_lo[3];
    float dist;   // |r_q| / Delta_s
    int cls;
    int pad[3];
};

struct DevTables {
    const Ring *rings;        // all rings, grouped by (class, k)
    const int *ring_off;      // [n_cls * K] first ring of (class, k)
    const int *ring_cnt;      // [n_cls * K] N_i(class, k)
    const Xdcr *xd;           // [Q]
    const int *qlist;         // transducers sorted by class
    const float4 *anchors;    // (x hi, x lo, y hi, y lo) local coordinates of every anchor
    const float *Rk;          // [K] rho_k / Delta_s (may be <= 0)
    const float *wD;          // [K] C_D / tau_k, 0 where tau_k <= 0
    const double *wD64;       // [K] the same in double (forward D)
    const float *ring_w;      // [rings] point weight / Delta_s^2 (exact strip areas); null: 1
};

// Brick tiling of the cell range [-1, n-1]^3 for one direction: nb bricks per axis of bs cells
// (bs <= the kernel's compile-time brick edge), work items = bricks x transducer chunks.
struct BrickCfg {
    int nb[3] = {1, 1, 1};
    int bs[3] = {1, 1, 1};
    int qchunk = 1;
    int kspan = 1;          // upper bound of the shells crossing one brick
    long long items = 0;
    size_t smem = 0;
};

constexpr int kBF = 34;     // projector brick edge: (kBF+1)^3 float nodes in shared memory
constexpr int kBA = 24;     // backprojector brick edge: (kBA+1)^3 pairs of 32-bit node-sum halves in shared memory

struct Plan {
    oat_geometry g{};
    std::vector<double> pos;
    int device = 0;
    int Q = 0, K = 0, n_cls = 0;
    int nx = 0, ny = 0, nz = 0;
    double R = 0, dt = 0, cd = 0;
    float O[3] = {0, 0, 0};      // -origin / Delta_s (hi part)
    float O_lo[3] = {0, 0, 0};   // its lo part
    float ds2 = 0;               // Delta_s^2
    float R0 = 0, dR = 0;        // rho_0 / Delta_s and c dt / Delta_s
    long long n_rings = 0, n_anchors = 0, points_ball = 0;
    long long max_shell_points = 0;   // largest N_i-ring lattice of one shell (fixed-point bound)
    bool area = false;                // exact strip-area point weights (ring_w)
    double fwd_bound = 0.0;           // max over shells of the sum of point weights / Delta_s^2
    float adj_wfac = 1.f;             // bound of a point's weight factor in G^T (exact areas; else 1)
    int adj_fbits = 30;               // G^T volume accumulator: a contribution is <= 2^adj_fbits units
    int adj_qpass = 1;                // transducers per backprojector pass (bounds the 32-bit halves)
    int n_sm = 0;                     // streaming multiprocessors of the plan's device (grid sizes)
    BrickCfg fwd, adj;                 // brick tilings of the projector and the backprojector
    long long table_bytes = 0, scratch_bytes = 0;
    std::vector<long long> cls_points;   // [n_cls * K] points per (class, k)

    // device memory
    void *d_tables = nullptr;   // one allocation holding every table
    DevTables t{};
    long long *d_gacc = nullptr;     // [Q][K] scratch: fixed-point sums of G alpha
    long long *d_vacc = nullptr;     // [nz][ny][nx] scratch: fixed-point node sums of G^T g'
    unsigned int *d_amax = nullptr;  // [2] scratch: max|alpha| and max|g'| bit patterns
    float *d_rowmax = nullptr;       // [Q] scratch: per-transducer max |g'| of the backprojector
    const int2 *d_krange = nullptr;  // [Q] (in the tables) samples whose shells can reach the grid
    unsigned long long *d_count = nullptr;  // point counter of oat_plan_query

    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> ev[3];       // [G, G^T, FBP]
    int ev_used[3] = {0, 0, 0};
    double ms_acc[3] = {0, 0, 0};
    long long launches[3] = {0, 0, 0};

    // filtered backprojection: per transducer (T hi xyz, weight) and (T lo xyz, 0), T the
    // position in index units relative to node (0,0,0) as a float pair
    float4 *d_fbp = nullptr;
    std::vector<float4> fbp_host;
    bool fbp_weights = false;

    // transducer response H^e: taps h_m for m = eir_m0 .. eir_m0 + eir_n - 1 (none when
    // eir_n == 0) and the float32 [Q][K] buffer that holds H^e^T y for the backprojector
    double *d_eir = nullptr;
    float *d_eir_z = nullptr;
    int eir_n = 0, eir_m0 = 0;
};

// status helpers (abi.cpp)
int set_error(int code, const std::string &msg);
// SM count of the current device (looked up once per device; 1 if the query fails)
int current_sm_count();

// kernels' host launchers (forward.cu, adjoint.cu)
int launch_project(Plan &p, const float *vol, void *data, cudaStream_t s);
int launch_backproject(Plan &p, const void *data, float *vol, cudaStream_t s);
int launch_backproject_static(Plan &p, const void *data, float *vol, cudaStream_t s);
int count_grid_points(Plan &p, long long *out);

// transducer response (eir.cu)
size_t eir_smem_bytes(const Plan &p);
int set_eir_attributes(const Plan &p);
int launch_apply_d_eir(Plan &p, void *data, cudaStream_t s);
int launch_eir_t(Plan &p, const void *y, float *z, cudaStream_t s);
int launch_fbp(Plan &p, const void *data, float *vol, cudaStream_t s);
int launch_fbp_kpos(Plan &p, const int *nodes, const int *qs, int n, double *out, cudaStream_t s);

// tensor-core convolution of the learned warm start (conv_tc.cu)
int launch_conv3d_tc(int nx, int ny, int nz, int cin, int cout, const void *x, const void *w, const float *bias, int relu,
                     void *y, cudaStream_t s);
int launch_wgrad_tc(int nx, int ny, int nz, int cin, int cout, const void *x, const void *g, float *dw, float *db,
                    cudaStream_t s);
int conv_tc_check();
int set_adjoint_attributes();
int set_forward_attributes();
size_t forward_smem_bytes();
size_t adjoint_smem_bytes(bool area);

constexpr int kMaxEvents = 4096;

}  // namespace oat

// ------------------------------------------------------------------------------------------
// Device helpers
// ------------------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace oat {

// ---------------------------------------------------------------------------- lattice points
// Every kernel computes lattice point (q, k, i, j) with the functions below, operation for
// operation, so that a point has the same cell and the same weights in H and in H^T and in
// every brick that looks at it.
//
// FP32 coordinates of magnitude |O| + |h| + a (several hundred grid units when the scanner is
// far from the grid) would carry rounding errors of ~1e-5 cells.  Instead each point is taken
// relative to its ring's anchor j_A = 32 floor(j / 32):
//   anchor  A = O + h e_z + x_A e_x + y_A e_y   in float-pair arithmetic (about 44 bits), split
//           into its cell I = floor(A) and fraction f = A - I;
//   point   P - I = f + dx e_x + dy e_y, with (dx, dy) the change of the local coordinates from
//           the anchor to point j: a rotation by delta = (j - j_A) dphi,
//             dx = x_A (cos delta - 1) - y_A sin delta,  dy = y_A (cos delta - 1) + x_A sin delta,
//           in FP32 (|dx|, |dy| <= 32 grid units).
// The cell of P is I + floor(P - I): it depends only on (q, k, i, j).

// s + e = a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s + e) += (xh + xl)(yh + yl), dropping xl yl: the product's rounding error comes from an FMA.
__device__ __forceinline__ void pair_madd(float xh, float xl, float yh, float yl, float &s, float &e) {
    const float p = __fmul_rn(xh, yh);
    const float pe = fmaf(xl, yh, fmaf(xh, yl, fmaf(xh, yh, -p)));
    float t;
    two_sum(s, p, s, t);
    e = __fadd_rn(e, __fadd_rn(t, pe));
}

// Anchor of a ring for transducer x: local coordinates xy = (x hi, x lo, y hi, y lo), ring axial
// offset (hh, hl); O = (Oh, Ol).  Returns the cell I and the fraction f (f may leave [0, 1) by
// the size of the pair's low part).
__device__ __forceinline__ void anchor_point(const float Oh[3], const float Ol[3], const Xdcr &x, float hh, float hl,
                                             float4 xy, int I[3], float f[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float s = Oh[d], e = Ol[d];
        pair_madd(hh, hl, x.ez[d], x.ez_lo[d], s, e);
        pair_madd(xy.x, xy.y, x.ex[d], x.ex_lo[d], s, e);
        pair_madd(xy.z, xy.w, x.ey[d], x.ey_lo[d], s, e);
        const float fl = floorf(s);
        I[d] = (int)fl;
        f[d] = __fadd_rn(__fsub_rn(s, fl), e);
    }
}

// Two floats in one 64-bit register for the packed FP32 instructions of sm_100+: add / mul /
// fma .rn.f32x2 round like their scalar forms, lane by lane, so a packed evaluation gives the
// bits of the scalar one at about half the issued instructions.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 r, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Point m = j - j_A (0 <= m < 2^ash <= 32) of a ring relative to its anchor's cell: P - I.
// (xa, ya): the anchor's local coordinates (hi parts).  The rotation delta = m dphi (|delta| <=
// 1 by the choice of the anchor spacing) enters through sin(delta) and cos(delta) - 1 from their
// Taylor series through delta^11 and delta^12 (the first omitted terms are below 2e-10), Horner
// form in FP32 (scalar FMAs, whose coefficients are instruction immediates).  Then
//   dx = x_A (cos delta - 1) - y_A sin delta,  dy = y_A (cos delta - 1) + x_A sin delta,
//   P - I = f + dx e_x + dy e_y.
__device__ __forceinline__ float3 anchor_offset(const float f[3], float xa, float ya, const float ex[3],
                                                const float ey[3], float dphi, float dphi_lo, int m) {
    const float mf = __int2float_rn(m);
    const float d = fmaf(mf, dphi_lo, __fmul_rn(mf, dphi));
    const float d2 = __fmul_rn(d, d);
    // sin series (coefficients of delta^11 down to delta^3) and cos series (delta^12 .. delta^4)
    const float ps = fmaf(d2, fmaf(d2, fmaf(d2, fmaf(d2, (float)(-1.0 / 39916800.0), (float)(1.0 / 362880.0)),
                                        (float)(-1.0 / 5040.0)), (float)(1.0 / 120.0)), (float)(-1.0 / 6.0));
    const float pc = fmaf(d2, fmaf(d2, fmaf(d2, fmaf(d2, (float)(1.0 / 479001600.0), (float)(-1.0 / 3628800.0)),
                                        (float)(1.0 / 40320.0)), (float)(-1.0 / 720.0)), (float)(1.0 / 24.0));
    const float sd = fmaf(__fmul_rn(d, d2), ps, d);
    const float cm = __fmul_rn(d2, fmaf(d2, pc, -0.5f));
    // (dx, dy) = (xa cm - ya sd, ya cm + xa sd)
    const f32x2 DXY = fma2(pk2(-ya, xa), pk2(sd, sd), mul2(pk2(xa, ya), pk2(cm, cm)));
    float dx, dy;
    upk2(DXY, dx, dy);
    f32x2 R01 = fma2(pk2(dx, dx), pk2(ex[0], ex[1]), pk2(f[0], f[1]));
    R01 = fma2(pk2(dy, dy), pk2(ey[0], ey[1]), R01);
    float r0, r1;
    upk2(R01, r0, r1);
    return make_float3(r0, r1, fmaf(dy, ey[2], fmaf(dx, ex[2], f[2])));
}

// Approximate ring centre B = O + h e_z in FP32 (azimuth windows only, which carry margins).
__device__ __forceinline__ float3 ring_base(const float O[3], const float ez[3], float h) {
    return make_float3(fmaf(h, ez[0], O[0]), fmaf(h, ez[1], O[1]), fmaf(h, ez[2], O[2]));
}

__device__ __forceinline__ float lerp1(float a, float b, float w) { return fmaf(w, b - a, a); }

// Neumaier compensated accumulation: (s, e) += x.
__device__ __forceinline__ void kadd(float &s, float &e, float x) {
    float t = s + x;
    e += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

}  // namespace oat
#endif
