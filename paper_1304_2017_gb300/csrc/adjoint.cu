// Backprojector alpha' = G^T D^T y as a gather per voxel, no floating-point atomics.
//
// A lattice point P of (q, k) contributes Delta_s^2 g'_{q,k} psi_n(P) to the eight nodes n of
// the cell m = floor(P) that contains it (Eq. expfunI; adjoint of Eq. dis_srt).  Points are
// partitioned by their cell, so:
//
// k_cell_gather: one thread per cell m in [-1, n-1]^3.  For every transducer q the thread
//   enumerates the lattice points that can lie in its cell -- shells k whose radius is within
//   the cell's circumscribed radius of the cell centre, rings i of those shells whose polar
//   angle is within the angle the cell subtends, and on each ring the azimuth window whose
//   points are within that radius (exact point-to-ring-distance condition) -- evaluates each
//   candidate with the SAME FP32 lattice-point function as the projector, keeps those with
//   floor(P) == m, and accumulates the eight trilinear weights times g'_{q,k} into eight
//   per-corner partial sums held in registers.  g'_{q,k} = (C_D / tau_k)(m_{k-1} y_{k-1} -
//   m_{k+1} y_{k+1}) is read straight from y (D^T fused into the input read).
//   Output: per-cell corner partials, scratch [cells][8].
//
// k_combine: each node sums the partials of its eight adjacent cells (written once).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "oat_internal.h"

namespace oat {

struct AdjArgs {
    DevTables t;
    const void *y;
    float *part;
    int nx, ny, nz, K, Q;
    float O[3];
    float R0, dR;
    float ds2;
    int apply_d;
};

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

constexpr float kCellR = 0.8700f;        // > sqrt(3)/2: circumscribed radius of a unit cell + margin
constexpr float kTwoPi = 6.28318530717958647692f;

template <int DT>
__global__ void __launch_bounds__(128) k_cell_gather(AdjArgs a) {
    const int cx = a.nx + 1, cy = a.ny + 1, cz = a.nz + 1;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= cx * cy * cz) return;
    const int mx = cell % cx - 1, my = (cell / cx) % cy - 1, mz = cell / (cx * cy) - 1;
    // cell centre relative to the global origin, index units
    const float Xg0 = (float)mx + 0.5f - a.O[0], Xg1 = (float)my + 0.5f - a.O[1], Xg2 = (float)mz + 0.5f - a.O[2];
    const float rc2 = kCellR * kCellR;

    float acc[8], outer[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) { acc[c] = 0.f; outer[c] = 0.f; }

    for (int q = 0; q < a.Q; ++q) {
        const Xdcr &x = a.t.xd[q];
        // cell centre in the transducer's local frame (transducer at the local origin)
        const float vx = Xg0 * x.ex[0] + Xg1 * x.ex[1] + Xg2 * x.ex[2];
        const float vy = Xg0 * x.ey[0] + Xg1 * x.ey[1] + Xg2 * x.ey[2];
        const float vz0 = Xg0 * x.ez[0] + Xg1 * x.ez[1] + Xg2 * x.ez[2];
        const float vz = vz0 + x.dist;
        const float rv2 = vx * vx + vy * vy;
        const float d = sqrtf(rv2 + vz * vz);
        int klo = (int)ceilf((d - kCellR - a.R0) / a.dR);
        int khi = (int)floorf((d + kCellR - a.R0) / a.dR);
        klo = max(klo, 0);
        khi = min(khi, a.K - 1);
        if (klo <= khi) {
            const float rv = sqrtf(rv2);
            const float thc = atan2f(rv, vz);
            float phc = atan2f(vy, vx);
            if (phc < 0.f) phc += kTwoPi;
            const int cbase = x.cls * a.K;
            for (int k = klo; k <= khi; ++k) {
                const int nr = __ldg(a.t.ring_cnt + cbase + k);
                if (nr <= 1) continue;
                const float Rk = __ldg(a.t.Rk + k);
                // half-angle of the cone through the shell-ball intersection: sin^2(gam/2)
                const float dd = Rk - d;
                const float s2 = (rc2 - dd * dd) / (4.f * Rk * d);
                if (!(s2 > 0.f)) continue;
                const float gam = s2 >= 1.f ? 3.14159265f : 2.f * asinf(sqrtf(s2));
                const int ilo = max(1, (int)ceilf(Rk * (thc - gam) - 1e-3f));
                const int ihi = min(nr - 1, (int)floorf(Rk * (thc + gam) + 1e-3f));
                if (ilo > ihi) continue;
                const float gp = gprime<DT>(a, q, k);
                if (gp == 0.f) continue;
                const int off = __ldg(a.t.ring_off + cbase + k);
                for (int i = ilo; i <= ihi; ++i) {
                    const Ring r = a.t.rings[off + i];
                    if (r.nj == 0) continue;
                    // distance from the cell centre to a ring point at azimuth phi:
                    // dz^2 + (rv - a)^2 + 4 a rv sin^2((phi - phc)/2) <= rc^2
                    const float dz = vz0 - r.h;
                    const float dr = rv - r.a;
                    const float rem = rc2 - dz * dz - dr * dr;
                    if (!(rem > 0.f)) continue;
                    int jlo0, jhi0;
                    bool all = false;
                    const float den = 4.f * r.a * rv;
                    float delta = 0.f;
                    if (!(den > 1e-12f) || rem >= den) all = true;
                    else {
                        delta = 2.f * asinf(sqrtf(rem / den)) + 2e-3f;
                        if (delta >= 3.1f) all = true;
                    }
                    const float3 B = ring_base(a.O, x.ez, r.h);
                    for (int sh = -1; sh <= 1; ++sh) {
                        if (all) {
                            if (sh != 0) continue;
                            jlo0 = 0; jhi0 = r.nj - 1;
                        } else {
                            const float c0 = phc + sh * kTwoPi;
                            jlo0 = max(0, (int)ceilf((c0 - delta) / r.dphi));
                            jhi0 = min(r.nj - 1, (int)floorf((c0 + delta) / r.dphi));
                        }
                        for (int j = jlo0; j <= jhi0; ++j) {
                            float u, v;
                            ring_uv(r, j, u, v);
                            const float3 P = ring_point(B, x.ex, x.ey, u, v);
                            const float fx = floorf(P.x), fy = floorf(P.y), fz = floorf(P.z);
                            if ((int)fx != mx || (int)fy != my || (int)fz != mz) continue;
                            const float wx = P.x - fx, wy = P.y - fy, wz = P.z - fz;
                            const float ux = 1.f - wx, uy = 1.f - wy, uz = 1.f - wz;
                            const float g00 = gp * uz * uy, g01 = gp * uz * wy, g10 = gp * wz * uy, g11 = gp * wz * wy;
                            acc[0] = fmaf(g00, ux, acc[0]); acc[1] = fmaf(g00, wx, acc[1]);
                            acc[2] = fmaf(g01, ux, acc[2]); acc[3] = fmaf(g01, wx, acc[3]);
                            acc[4] = fmaf(g10, ux, acc[4]); acc[5] = fmaf(g10, wx, acc[5]);
                            acc[6] = fmaf(g11, ux, acc[6]); acc[7] = fmaf(g11, wx, acc[7]);
                        }
                    }
                }
            }
        }
        if ((q & 31) == 31) {
#pragma unroll
            for (int c = 0; c < 8; ++c) { outer[c] += acc[c]; acc[c] = 0.f; }
        }
    }
    float4 *o = reinterpret_cast<float4 *>(a.part + (size_t)cell * 8);
    o[0] = make_float4(a.ds2 * (outer[0] + acc[0]), a.ds2 * (outer[1] + acc[1]), a.ds2 * (outer[2] + acc[2]),
                       a.ds2 * (outer[3] + acc[3]));
    o[1] = make_float4(a.ds2 * (outer[4] + acc[4]), a.ds2 * (outer[5] + acc[5]), a.ds2 * (outer[6] + acc[6]),
                       a.ds2 * (outer[7] + acc[7]));
}

// node n = sum over its eight cells m = n - c of corner c of m; corner index (dz, dy, dx) bits.
__global__ void k_combine(const float *__restrict__ part, float *__restrict__ vol, int nx, int ny, int nz) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nx * ny * nz) return;
    const int ix = n % nx, iy = (n / nx) % ny, iz = n / (nx * ny);
    const int cx = nx + 1, cy = ny + 1;
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const int m = ((iz - dz + 1) * cy + (iy - dy + 1)) * cx + (ix - dx + 1);
        s += __ldg(part + (size_t)m * 8 + c);
    }
    vol[n] = s;
}

int launch_backproject(Plan &p, const void *data, float *vol, cudaStream_t s) {
    AdjArgs a;
    a.t = p.t; a.y = data; a.part = p.d_part;
    a.nx = p.nx; a.ny = p.ny; a.nz = p.nz; a.K = p.K; a.Q = p.Q;
    for (int d = 0; d < 3; ++d) a.O[d] = p.O[d];
    a.R0 = p.R0; a.dR = p.dR; a.ds2 = p.ds2; a.apply_d = p.g.apply_d;
    const long long cells = (long long)(p.nx + 1) * (p.ny + 1) * (p.nz + 1);
    const unsigned blocks = (unsigned)((cells + 127) / 128);
    const bool prof = p.profiling && p.ev_used[1] + 2 <= (int)p.ev[1].size();
    if (prof) cudaEventRecord(p.ev[1][p.ev_used[1]], s);
    switch (p.g.data_dtype) {
        case OAT_F32: k_cell_gather<OAT_F32><<<blocks, 128, 0, s>>>(a); break;
        case OAT_F16: k_cell_gather<OAT_F16><<<blocks, 128, 0, s>>>(a); break;
        default: k_cell_gather<OAT_BF16><<<blocks, 128, 0, s>>>(a); break;
    }
    if (prof) { cudaEventRecord(p.ev[1][p.ev_used[1] + 1], s); p.ev_used[1] += 2; }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_backproject: k_cell_gather: ") + cudaGetErrorString(e));
    const long long N = (long long)p.nx * p.ny * p.nz;
    k_combine<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(p.d_part, vol, p.nx, p.ny, p.nz);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_backproject: k_combine: ") + cudaGetErrorString(e));
    return OAT_OK;
}

}  // namespace oat
