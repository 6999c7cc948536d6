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
struct Ring {
    float h, a, dphi;
    int nj;
};

// Per-transducer record: local frame and |r_q| / Delta_s, and its radius class.
struct Xdcr {
    float ex[3], ey[3], ez[3];
    float dist;   // |r_q| / Delta_s
    int cls;
    int pad[2];
};

struct DevTables {
    const Ring *rings;        // all rings, grouped by (class, k)
    const int *ring_off;      // [n_cls * K] first ring of (class, k)
    const int *ring_cnt;      // [n_cls * K] N_i(class, k)
    const Xdcr *xd;           // [Q]
    const int *qlist;         // transducers sorted by class
    const int4 *items;        // forward work items (class, k, first in qlist, count)
    const float *Rk;          // [K] rho_k / Delta_s (may be <= 0)
    const float *wD;          // [K] C_D / tau_k, 0 where tau_k <= 0
    const double *wD64;       // [K] the same in double (forward D)
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

constexpr int kBF = 32;     // projector brick edge: (kBF+1)^3 float nodes in shared memory
constexpr int kBA = 24;     // backprojector brick edge: (kBA+1)^3 pairs of 32-bit node-sum halves in shared memory

struct Plan {
    oat_geometry g{};
    std::vector<double> pos;
    int device = 0;
    int Q = 0, K = 0, n_cls = 0;
    int nx = 0, ny = 0, nz = 0;
    double R = 0, dt = 0, cd = 0;
    float O[3] = {0, 0, 0};      // -origin / Delta_s
    float ds2 = 0;               // Delta_s^2
    float R0 = 0, dR = 0;        // rho_0 / Delta_s and c dt / Delta_s
    long long n_rings = 0, points_ball = 0, n_items = 0;
    long long max_shell_points = 0;   // largest N_i-ring lattice of one shell (fixed-point bound)
    float gscale = 1.f;               // max |g'| / max |y|: 2 max_k C_D/tau_k with D, 1 without
    int adj_qpass = 1;                // transducers per backprojector pass (bounds the 32-bit halves)
    BrickCfg fwd, adj;                 // brick tilings of the projector and the backprojector
    bool fwd_radial = false;           // projector kernel: radial lanes or bricks
    const int4 *d_ritems = nullptr;    // radial work items (class, first shell, first in qlist, count)
    long long n_ritems = 0;
    long long table_bytes = 0, scratch_bytes = 0;
    std::vector<long long> cls_points;   // [n_cls * K] points per (class, k)

    // device memory
    void *d_tables = nullptr;   // one allocation holding every table
    DevTables t{};
    long long *d_gacc = nullptr;     // [Q][K] scratch: fixed-point sums of G alpha
    long long *d_vacc = nullptr;     // [nz][ny][nx] scratch: fixed-point node sums of G^T g'
    unsigned int *d_amax = nullptr;  // [2] scratch: max|alpha| and max|y| bit patterns
    unsigned long long *d_count = nullptr;  // point counter of oat_plan_query

    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> ev[2];
    int ev_used[2] = {0, 0};
    double ms_acc[2] = {0, 0};
    long long launches[2] = {0, 0};
};

// status helpers (abi.cpp)
int set_error(int code, const std::string &msg);

// kernels' host launchers (forward.cu, adjoint.cu)
int launch_project(Plan &p, const float *vol, void *data, cudaStream_t s);
int launch_backproject(Plan &p, const void *data, float *vol, cudaStream_t s);
int launch_backproject_static(Plan &p, const void *data, float *vol, cudaStream_t s);
int count_grid_points(Plan &p, long long *out);
int set_adjoint_attributes();
int set_forward_attributes();
size_t forward_smem_bytes();
size_t adjoint_smem_bytes();

constexpr int kMaxEvents = 4096;

}  // namespace oat

// ------------------------------------------------------------------------------------------
// Device helpers
// ------------------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace oat {

// (u, v) = a (cos phi_j, sin phi_j), phi_j = j * dphi in FP32.  Explicitly rounded so that
// every kernel evaluates exactly the same values.
__device__ __forceinline__ void ring_uv(float a, float dphi, int j, float &u, float &v) {
    float phi = __fmul_rn(__int2float_rn(j), dphi);
    float s, c;
    sincosf(phi, &s, &c);
    u = __fmul_rn(a, c);
    v = __fmul_rn(a, s);
}

__device__ __forceinline__ void ring_uv(const Ring &r, int j, float &u, float &v) { ring_uv(r.a, r.dphi, j, u, v); }

// Ring centre in index coordinates for one transducer: B = O + h e_z.
__device__ __forceinline__ float3 ring_base(const float O[3], const float ez[3], float h) {
    return make_float3(fmaf(h, ez[0], O[0]), fmaf(h, ez[1], O[1]), fmaf(h, ez[2], O[2]));
}

// Lattice point P = B + u e_x + v e_y (index coordinates), fused multiply-adds in a fixed order.
__device__ __forceinline__ float3 ring_point(float3 B, const float ex[3], const float ey[3], float u, float v) {
    return make_float3(fmaf(v, ey[0], fmaf(u, ex[0], B.x)),
                       fmaf(v, ey[1], fmaf(u, ex[1], B.y)),
                       fmaf(v, ey[2], fmaf(u, ex[2], B.z)));
}

__device__ __forceinline__ float lerp1(float a, float b, float w) { return fmaf(w, b - a, a); }

// sum_n alpha_n psi_n(P): trilinear interpolation with the nodes outside the grid absent
// (Eq. expfunI).
__device__ __forceinline__ float trilinear(const float *__restrict__ vol, int nx, int ny, int nz, float3 P) {
    float fx = floorf(P.x), fy = floorf(P.y), fz = floorf(P.z);
    int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    // all eight nodes outside (also rejects NaN: comparisons are false)
    if (!(ix >= -1 && ix < nx && iy >= -1 && iy < ny && iz >= -1 && iz < nz)) return 0.f;
    float wx = P.x - fx, wy = P.y - fy, wz = P.z - fz;
    const int sy = nx, sz = nx * ny;
    float v000, v001, v010, v011, v100, v101, v110, v111;
    if (ix >= 0 && ix < nx - 1 && iy >= 0 && iy < ny - 1 && iz >= 0 && iz < nz - 1) {
        const float *b = vol + (iz * ny + iy) * nx + ix;
        v000 = __ldg(b);          v001 = __ldg(b + 1);
        v010 = __ldg(b + sy);     v011 = __ldg(b + sy + 1);
        v100 = __ldg(b + sz);     v101 = __ldg(b + sz + 1);
        v110 = __ldg(b + sz + sy); v111 = __ldg(b + sz + sy + 1);
    } else {
        bool x0 = ix >= 0, x1 = ix + 1 < nx, y0 = iy >= 0, y1 = iy + 1 < ny, z0 = iz >= 0, z1 = iz + 1 < nz;
        auto at = [&](bool ok, int x, int y, int z) -> float {
            return ok ? __ldg(vol + (z * ny + y) * nx + x) : 0.f;
        };
        v000 = at(z0 && y0 && x0, ix, iy, iz);         v001 = at(z0 && y0 && x1, ix + 1, iy, iz);
        v010 = at(z0 && y1 && x0, ix, iy + 1, iz);     v011 = at(z0 && y1 && x1, ix + 1, iy + 1, iz);
        v100 = at(z1 && y0 && x0, ix, iy, iz + 1);     v101 = at(z1 && y0 && x1, ix + 1, iy, iz + 1);
        v110 = at(z1 && y1 && x0, ix, iy + 1, iz + 1); v111 = at(z1 && y1 && x1, ix + 1, iy + 1, iz + 1);
    }
    float c00 = lerp1(v000, v001, wx), c01 = lerp1(v010, v011, wx);
    float c10 = lerp1(v100, v101, wx), c11 = lerp1(v110, v111, wx);
    float c0 = lerp1(c00, c01, wy), c1 = lerp1(c10, c11, wy);
    return lerp1(c0, c1, wz);
}

// Neumaier compensated accumulation: (s, e) += x.
__device__ __forceinline__ void kadd(float &s, float &e, float x) {
    float t = s + x;
    e += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

}  // namespace oat
#endif
