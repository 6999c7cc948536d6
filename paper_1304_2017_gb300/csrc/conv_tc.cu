// 3x3x3 'same' convolution of the learned warm start on the 5th-generation tensor cores
// (include/oat_unet.h, oat_conv3d_bf16): tcgen05.mma with the accumulator in tensor memory, both
// operands staged in shared memory by TMA (cp.async.bulk.tensor), an mbarrier pipeline between
// the copy thread and the MMA thread.
//
// Implicit GEMM per tile of M = 128 output voxels (bx consecutive voxels along x times by rows
// along y, bx by <= 128, at one z): D[m][co] = sum_tap sum_ci A_tap[m][ci] B_tap[co][ci] with
// A_tap[m][ci] = x[z + dz][y + dy][x + dx][ci] (zero outside the grid: the TMA fill) and
// B_tap[co][ci] = w[tap][co][ci].  Both operands are K-major with K = the input channels, in the
// no-swizzle core-matrix layout: a core matrix is 8 rows of 16 bytes (8 channels), rows 16 bytes
// apart; the 8-row groups follow each other (stride 128 bytes, SBO); the 8-channel groups are
// LBO apart (A: bx by rounded up to 8, times 16 bytes; B: cout 16 bytes), every group starting on
// a 128-byte boundary as the tensor copies require.  One TMA box per 8-channel group writes exactly
// that layout: box (8 channels, bx, by, 1) of the activations, (8 channels, cout, 1) of the
// weights.  Each tap is one pipeline stage: cin / 16 MMAs of 128 x cout x 16 (BF16 in, FP32
// accumulation), accumulating into cout TMEM columns.
//
// Roles: thread 0 issues the copies, thread 32 the MMAs; warp 0 allocates and frees the TMEM
// columns; all four warps read the accumulator back (tcgen05.ld, warp w owns TMEM lanes
// 32w .. 32w + 31, i.e. tile rows), add the bias, apply the ReLU and store BF16 channels-last.
//
// Every wait on an mbarrier is bounded (about a second of SM clock); a wait that runs out sets
// g_tc_error, lets the other roles stop, waits (bounded) for the copies and MMAs already issued,
// frees the TMEM and returns.  oat_unet_check() reports the flag to the host.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/oat_unet.h"
#include "oat_internal.h"

namespace oat {

typedef __nv_bfloat16 bf16;

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;          // tile rows = TMEM lanes
constexpr int kTcStages = 4;
constexpr int kTcCols = 128;       // TMEM columns allocated (>= cout, a power of two)
constexpr long long kWaitCycles = 2000000000LL;

__device__ unsigned int g_tc_error;   // 1: an mbarrier wait ran out

struct ConvTcArgs {
    int nx, ny, nz, cin, cout;
    int bx, by, tiles_x, tiles_y;
    const float *bias;
    int relu;
    bf16 *y;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity to complete; false if it did not in time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
        __nanosleep(32);
    }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M / N) byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_tc(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_conv3d_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, ConvTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full_bar[kTcStages], empty_bar[kTcStages], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort, s_issued, s_waited;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cin = a.cin, cout = a.cout, m_used = a.bx * a.by;
    const uint32_t a_bytes = (uint32_t)kTcM * cin * 2, b_bytes = (uint32_t)cout * cin * 2;
    const uint32_t stage_bytes = (a_bytes + b_bytes + 1023u) & ~1023u;
    // 8-channel groups of the tile: the TMA writes bx by rows of 16 bytes per group; groups start
    // on 128-byte boundaries (a tensor copy's shared-memory destination must be 128-byte aligned),
    // so the group stride is the row count rounded up to 8 rows
    const uint32_t lbo_a = (uint32_t)((m_used + 7) & ~7) * 16u, lbo_b = (uint32_t)cout * 16u;
    const uint32_t tx_bytes = (uint32_t)(m_used + cout) * cin * 2u;
    int tile = blockIdx.x;
    const int tx = tile % a.tiles_x;
    tile /= a.tiles_x;
    const int ty = tile % a.tiles_y, tz = tile / a.tiles_y;
    const int x0 = tx * a.bx, y0 = ty * a.by;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&done_bar), 1);
        s_abort = 0; s_issued = 0; s_waited = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t sbase = (smem_u32(smem) + 1023u) & ~1023u;   // stages on 1 KB boundaries

    if (threadIdx.x == 0) {
        // copies: stage s <- tap t
        for (int t = 0; t < 27; ++t) {
            const int s = t % kTcStages;
            if (t >= kTcStages && !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)((t / kTcStages - 1) & 1))) {
                atomicOr(&g_tc_error, 1u);
                s_abort = 1;
                break;
            }
            if (*(volatile int *)&s_abort) break;
            const uint32_t bar = smem_u32(&full_bar[s]);
            const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_bytes;
            mbar_expect_tx(bar, tx_bytes);
            const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
            for (int cc = 0; cc < cin / 8; ++cc) {
                tma_load_4d(sa + cc * lbo_a, &mapA, cc * 8, x0 + dx, y0 + dy, tz + dz, bar);
                tma_load_3d(sb + cc * lbo_b, &mapB, cc * 8, 0, t, bar);
            }
            s_issued = t + 1;
        }
    } else if (threadIdx.x == 32) {
        // MMAs: cin / 16 per tap into the TMEM accumulator
        const uint32_t idesc = idesc_bf16(kTcM, cout);
        int t = 0;
        for (; t < 27; ++t) {
            const int s = t % kTcStages;
            if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((t / kTcStages) & 1))) {
                atomicOr(&g_tc_error, 1u);
                s_abort = 1;
                break;
            }
            s_waited = t + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_bytes;
            for (int j = 0; j < cin / 16; ++j) {
                const uint64_t da = smem_desc(sa + 2u * j * lbo_a, lbo_a, 128u);
                const uint64_t db = smem_desc(sb + 2u * j * lbo_b, lbo_b, 128u);
                mma_bf16_tc(tmem, da, db, idesc, (t > 0 || j > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(&empty_bar[s]));   // the stage is free once these MMAs are done
        }
        mma_commit(smem_u32(&done_bar));           // all MMAs issued so far are done
    }
    __syncwarp();

    // epilogue: TMEM lanes 32 warp .. + 31 are tile rows; bias, ReLU, BF16 store
    const bool ok = mbar_wait(smem_u32(&done_bar), 0u);
    if (!ok) {
        atomicOr(&g_tc_error, 1u);
        s_abort = 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // tcgen05.ld is warp-collective: the warp reads the accumulator only if all its lanes can
    if (__all_sync(0xffffffffu, ok && !*(volatile int *)&s_abort)) {
        const int m = warp * 32 + lane;
        const int xl = m % a.bx, yl = m / a.bx;
        const int xg = x0 + xl, yg = y0 + yl;
        const bool valid = m < m_used && xg < a.nx && yg < a.ny;
        bf16 *dst = a.y + ((((size_t)tz * a.ny + yg) * a.nx + xg) * cout);
        for (int c = 0; c < cout; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);   // warp-collective
            if (valid) {
                __align__(16) __nv_bfloat162 o[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float v0 = v[2 * i] + (a.bias ? __ldg(a.bias + c + 2 * i) : 0.f);
                    float v1 = v[2 * i + 1] + (a.bias ? __ldg(a.bias + c + 2 * i + 1) : 0.f);
                    if (a.relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                    o[i] = __floats2bfloat162_rn(v0, v1);
                }
                uint4 *d4 = reinterpret_cast<uint4 *>(dst + c);
                d4[0] = *reinterpret_cast<const uint4 *>(&o[0]);
                d4[1] = *reinterpret_cast<const uint4 *>(&o[4]);
            }
        }
    }
    // after an abort: wait (bounded) for the copies issued but not consumed, so that nothing
    // writes into this block's shared memory after it exits
    __syncthreads();
    if (threadIdx.x == 0 && s_abort) {
        for (int t = s_waited; t < s_issued; ++t)
            mbar_wait(smem_u32(&full_bar[t % kTcStages]), (uint32_t)((t / kTcStages) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
}

// ----------------------------------------------------------------------- weight gradient
// dW[tap][co][ci] = sum_v g[v][co] x[v + off(tap)][ci] and db[co] = sum_v g[v][co] on the tensor
// cores: per tap a GEMM with M = co (128 rows, those >= cout zero), N = ci plus one column of ones
// (its result is the bias gradient: the voxels' g rows are zero outside the grid), K = voxels in
// chunks of one x-run of up to 128 voxels.  Both operands are MN-major as the activations are
// stored (8 channels contiguous per voxel): a TMA box (8 channels, bx voxels) is one column of
// core matrices along K (8-row groups 128 bytes apart, LBO) and the 8-channel groups follow at
// 2048 bytes (SBO).  Rows a box does not write stay zero (the buffers are cleared once), so
// chunks shorter than the 16-voxel MMA step add nothing.  Block (tap, split) sums the chunks
// split, split + S, ... in TMEM and writes its partial to g_wgrad_ws; k_wgrad_reduce then adds the
// splits in a fixed order: no floating-point atomics, the same result on every run.
constexpr int kWgStages = 3;
constexpr int kWgSplitMax = 8;
constexpr int kWgGroupBytes = 2048;                 // 128 voxel rows x 16 bytes
constexpr size_t kWgWsFloats = (size_t)27 * kWgSplitMax * 96 * 97;
__device__ float g_wgrad_ws[kWgWsFloats];         // partial dW and db of every (tap, split)

struct WgArgs {
    int nx, ny, nz, cin, cout;
    int bx, tiles_x, splits;
    long long nchunks;
};

__global__ void __launch_bounds__(kTcThreads, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap mapG, const __grid_constant__ CUtensorMap mapX, WgArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full_bar[kWgStages], empty_bar[kWgStages], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cin = a.cin, cout = a.cout;
    const int tap = blockIdx.x / a.splits, split = blockIdx.x % a.splits;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int n_groups_b = cin / 8 + 2;                       // x channels, the ones column, zeros
    const uint32_t a_region = 16u * kWgGroupBytes, b_region = (uint32_t)n_groups_b * kWgGroupBytes;
    const uint32_t stage_bytes = a_region + b_region;
    const uint32_t tx_bytes = (uint32_t)(cout / 8 + cin / 8) * a.bx * 16u;
    const int ksteps = (a.bx + 15) / 16;
    const long long my_chunks = a.nchunks > split ? (a.nchunks - split + a.splits - 1) / a.splits : 0;
    const uint32_t sbase = (smem_u32(smem) + 1023u) & ~1023u;
    unsigned char *sgen = smem + (sbase - smem_u32(smem));

    // clear every stage (rows no box writes must be zero) and set the ones column of B
    for (uint32_t i = threadIdx.x * 16u; i < stage_bytes * kWgStages; i += kTcThreads * 16u)
        *reinterpret_cast<uint4 *>(sgen + i) = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    for (int i = threadIdx.x; i < kWgStages * 128; i += kTcThreads) {
        const int st = i / 128, v = i % 128;
        *reinterpret_cast<unsigned short *>(sgen + st * stage_bytes + a_region + (cin / 8) * kWgGroupBytes + v * 16) =
            (unsigned short)0x3F80;   // bf16 1.0
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
    if (threadIdx.x == 0) {
        for (int st = 0; st < kWgStages; ++st) {
            mbar_init(smem_u32(&full_bar[st]), 1);
            mbar_init(smem_u32(&empty_bar[st]), 1);
        }
        mbar_init(smem_u32(&done_bar), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    long long issued = 0, waited = 0;

    if (threadIdx.x == 0) {
        for (long long i = 0; i < my_chunks; ++i) {
            const int st = (int)(i % kWgStages);
            if (i >= kWgStages && !mbar_wait(smem_u32(&empty_bar[st]), (uint32_t)((i / kWgStages - 1) & 1))) {
                atomicOr(&g_tc_error, 1u);
                s_abort = 1;
                break;
            }
            if (*(volatile int *)&s_abort) break;
            const long long c = split + i * a.splits;
            const int xt = (int)(c % a.tiles_x);
            const long long r = c / a.tiles_x;
            const int yy = (int)(r % a.ny), zz = (int)(r / a.ny), x0 = xt * a.bx;
            const uint32_t bar = smem_u32(&full_bar[st]);
            const uint32_t sa = sbase + st * stage_bytes, sb = sa + a_region;
            mbar_expect_tx(bar, tx_bytes);
            for (int gi = 0; gi < cout / 8; ++gi) tma_load_4d(sa + gi * kWgGroupBytes, &mapG, gi * 8, x0, yy, zz, bar);
            for (int gi = 0; gi < cin / 8; ++gi)
                tma_load_4d(sb + gi * kWgGroupBytes, &mapX, gi * 8, x0 + dx, yy + dy, zz + dz, bar);
            issued = i + 1;
        }
    } else if (threadIdx.x == 32) {
        // A and B MN-major (bits 15, 16), N = cin + 16
        const uint32_t idesc = idesc_bf16(128, cin + 16) | (1u << 15) | (1u << 16);
        for (long long i = 0; i < my_chunks; ++i) {
            const int st = (int)(i % kWgStages);
            if (!mbar_wait(smem_u32(&full_bar[st]), (uint32_t)((i / kWgStages) & 1))) {
                atomicOr(&g_tc_error, 1u);
                s_abort = 1;
                break;
            }
            waited = i + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = sbase + st * stage_bytes, sb = sa + a_region;
            for (int j = 0; j < ksteps; ++j) {
                const uint64_t da = smem_desc(sa + 256u * j, 128u, (uint32_t)kWgGroupBytes);
                const uint64_t db = smem_desc(sb + 256u * j, 128u, (uint32_t)kWgGroupBytes);
                mma_bf16_tc(tmem, da, db, idesc, (i > 0 || j > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(&empty_bar[st]));
        }
        mma_commit(smem_u32(&done_bar));
    }
    __syncwarp();

    const bool ok = mbar_wait(smem_u32(&done_bar), 0u);
    if (!ok) {
        atomicOr(&g_tc_error, 1u);
        s_abort = 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__all_sync(0xffffffffu, ok && !*(volatile int *)&s_abort)) {
        const int co = warp * 32 + lane;
        float *dst = g_wgrad_ws + (((size_t)tap * a.splits + split) * cout + (co < cout ? co : 0)) * (cin + 1);
        for (int c = 0; c < cin + 16; c += 16) {
            float v[16];
            if (my_chunks > 0) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);   // warp-collective
            else {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.f;
            }
            if (co < cout) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (c + i <= cin) dst[c + i] = v[i];   // column cin: the bias gradient
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_abort) {
        for (long long t = waited; t < issued; ++t)
            mbar_wait(smem_u32(&full_bar[t % kWgStages]), (uint32_t)((t / kWgStages) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
}

// dw[tap][co][ci] += sum_s partial[tap][s][co][ci] and db[co] += sum_s partial[13][s][co][cin], the
// splits in order.
__global__ void k_wgrad_reduce(int cin, int cout, int splits, float *dw, float *db) {
    const int n = 27 * cout * cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int tap = i / (cout * cin), r = i % (cout * cin), co = r / cin, ci = r % cin;
        float s = 0.f;
        for (int k = 0; k < splits; ++k) s += g_wgrad_ws[(((size_t)tap * splits + k) * cout + co) * (cin + 1) + ci];
        dw[i] += s;
        if (db && tap == 13 && ci == 0) {
            float b = 0.f;
            for (int k = 0; k < splits; ++k) b += g_wgrad_ws[(((size_t)13 * splits + k) * cout + co) * (cin + 1) + cin];
            db[co] += b;
        }
    }
}

// ------------------------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    });
    return fn;
}

// Dynamic shared memory of a block: the stages plus alignment slack, and at least 60 KB so that at
// most three blocks share an SM (3 x 128 of its 512 TMEM columns: tcgen05.alloc never waits).
size_t conv_tc_smem_bytes(int cin, int cout) {
    const size_t stage = ((size_t)kTcM * cin * 2 + (size_t)cout * cin * 2 + 1023) & ~(size_t)1023;
    const size_t need = stage * kTcStages + 1024;
    return need < 60 * 1024 ? 60 * 1024 : need;
}

int launch_conv3d_tc(int nx, int ny, int nz, int cin, int cout, const void *x, const void *w, const float *bias, int relu,
                     void *y, cudaStream_t s) {
    if (((uintptr_t)x & 15) || ((uintptr_t)w & 15) || ((uintptr_t)y & 15))
        return set_error(OAT_ERR_INVALID_ARG, "oat_conv3d_bf16: x, w and y must be 16-byte aligned");
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(OAT_ERR_CUDA, "oat_conv3d_bf16: cuTensorMapEncodeTiled is not available");
    ConvTcArgs a;
    a.nx = nx; a.ny = ny; a.nz = nz; a.cin = cin; a.cout = cout;
    a.bx = nx < kTcM ? nx : kTcM;
    a.by = kTcM / a.bx;
    if (a.by > ny) a.by = ny;
    a.tiles_x = (nx + a.bx - 1) / a.bx;
    a.tiles_y = (ny + a.by - 1) / a.by;
    a.bias = bias; a.relu = relu; a.y = (bf16 *)y;
    const long long tiles = (long long)a.tiles_x * a.tiles_y * nz;
    if (tiles > 0x7fffffffLL) return set_error(OAT_ERR_INVALID_ARG, "oat_conv3d_bf16: volume too large");

    // activations x[z][y][x][c]: dims (c, x, y, z), box (8, bx, by, 1); zero fill outside
    CUtensorMap mA, mB;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)cin, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
        const cuuint64_t strides[3] = {(cuuint64_t)cin * 2, (cuuint64_t)nx * cin * 2, (cuuint64_t)ny * nx * cin * 2};
        const cuuint32_t box[4] = {8, (cuuint32_t)a.bx, (cuuint32_t)a.by, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        CUresult r = enc(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(x), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return set_error(OAT_ERR_CUDA, "oat_conv3d_bf16: tensor map of the activations: error " + std::to_string((int)r));
    }
    // weights w[tap][co][ci]: dims (ci, co, tap), box (8, cout, 1)
    {
        const cuuint64_t dims[3] = {(cuuint64_t)cin, (cuuint64_t)cout, 27};
        const cuuint64_t strides[2] = {(cuuint64_t)cin * 2, (cuuint64_t)cout * cin * 2};
        const cuuint32_t box[3] = {8, (cuuint32_t)cout, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(w), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return set_error(OAT_ERR_CUDA, "oat_conv3d_bf16: tensor map of the weights: error " + std::to_string((int)r));
    }
    const size_t smem = conv_tc_smem_bytes(cin, cout);
    cudaError_t e = cudaFuncSetAttribute(k_conv3d_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_conv3d_bf16: ") + cudaGetErrorString(e));
    k_conv3d_tc<<<(unsigned)tiles, kTcThreads, smem, s>>>(mA, mB, a);
    e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("oat_conv3d_bf16: ") + cudaGetErrorString(e));
}

int launch_wgrad_tc(int nx, int ny, int nz, int cin, int cout, const void *x, const void *g, float *dw, float *db,
                    cudaStream_t s) {
    if (((uintptr_t)x & 15) || ((uintptr_t)g & 15))
        return set_error(OAT_ERR_INVALID_ARG, "oat_conv3d_wgrad: x and g must be 16-byte aligned");
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(OAT_ERR_CUDA, "oat_conv3d_wgrad: cuTensorMapEncodeTiled is not available");
    WgArgs a;
    a.nx = nx; a.ny = ny; a.nz = nz; a.cin = cin; a.cout = cout;
    a.bx = nx < 128 ? nx : 128;
    a.tiles_x = (nx + a.bx - 1) / a.bx;
    a.nchunks = (long long)a.tiles_x * ny * nz;
    // voxel splits per tap: about one block per SM in all, within the workspace
    int splits = current_sm_count() / 27;
    if (splits < 1) splits = 1;
    if (splits > kWgSplitMax) splits = kWgSplitMax;
    while (splits > 1 && (size_t)27 * splits * cout * (cin + 1) > kWgWsFloats) --splits;
    if ((long long)splits > a.nchunks) splits = (int)std::max(1LL, a.nchunks);
    a.splits = splits;
    CUtensorMap mG, mX;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    {
        const cuuint64_t dims[4] = {(cuuint64_t)cout, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
        const cuuint64_t strides[3] = {(cuuint64_t)cout * 2, (cuuint64_t)nx * cout * 2, (cuuint64_t)ny * nx * cout * 2};
        const cuuint32_t box[4] = {8, (cuuint32_t)a.bx, 1, 1};
        CUresult r = enc(&mG, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(g), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return set_error(OAT_ERR_CUDA, "oat_conv3d_wgrad: tensor map of the gradient: error " + std::to_string((int)r));
    }
    {
        const cuuint64_t dims[4] = {(cuuint64_t)cin, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
        const cuuint64_t strides[3] = {(cuuint64_t)cin * 2, (cuuint64_t)nx * cin * 2, (cuuint64_t)ny * nx * cin * 2};
        const cuuint32_t box[4] = {8, (cuuint32_t)a.bx, 1, 1};
        CUresult r = enc(&mX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(x), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return set_error(OAT_ERR_CUDA, "oat_conv3d_wgrad: tensor map of the activations: error " + std::to_string((int)r));
    }
    const size_t smem = (size_t)kWgStages * (16 + cin / 8 + 2) * kWgGroupBytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_conv3d_wgrad: ") + cudaGetErrorString(e));
    k_wgrad_tc<<<(unsigned)(27 * splits), kTcThreads, smem, s>>>(mG, mX, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_conv3d_wgrad: ") + cudaGetErrorString(e));
    const int n = 27 * cout * cin;
    k_wgrad_reduce<<<(unsigned)std::min(1024, (n + 255) / 256), 256, 0, s>>>(cin, cout, splits, dw, db);
    e = cudaGetLastError();
    return e == cudaSuccess ? OAT_OK : set_error(OAT_ERR_CUDA, std::string("oat_conv3d_wgrad: ") + cudaGetErrorString(e));
}

int conv_tc_check() {
    unsigned int flag = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&flag, g_tc_error, sizeof(flag));
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_unet_check: ") + cudaGetErrorString(e));
    if (flag) {
        const unsigned int zero = 0;
        cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(zero));
        return set_error(OAT_ERR_CUDA, "oat_unet_check: a tensor-core convolution timed out waiting on its pipeline");
    }
    return OAT_OK;
}

}  // namespace oat
