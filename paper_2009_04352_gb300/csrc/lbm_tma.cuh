// Row-pipelined form of the fused step for nx a multiple of 64.
//
// Work unit: one (y, z) row of nx cells, processed by one CTA of NW warps, two
// cells per lane. Each CTA owns a ring of S shared-memory stages; a stage holds
// the 19 source rows its output row gathers from (the z/y shifts and the wall
// reflection -- mirror or opposite slot, lbm_device.cuh -- are the choice of
// the source row). Lanes 0..18 of warp 0 issue one bulk copy (cp.async.bulk)
// per population row, with completion counted on the stage's "full" mbarrier;
// every warp computes its cells from shared memory, where the x-shift of the
// streaming step and its periodic wrap are an index offset, then arrives on
// the stage's "empty" mbarrier so that warp 0 can refill it. Rows are whole, so
// every byte copied is used exactly once. The copies of the next S-1 rows are
// in flight while the CTA computes the current one, so DRAM latency is covered
// by the ring rather than by occupancy. Every wait on an mbarrier is bounded
// by the launch's wait limit: on timeout the warp sets the error flag; warp 0
// also waits for the copies it still has in flight before returning, bounded
// by the fixed WAIT_CYCLES whatever the launch's limit, so that no copy can
// land in shared memory after its CTA has exited.
#pragma once

#include "lbm_pair.cuh"

namespace lbm {

constexpr long long WAIT_CYCLES = 1LL << 32;   // ~2 s at 2 GHz: default limit, and the drain limit
constexpr int ROW_MAX_STAGES = 4;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Non-blocking test of phase `parity` (test_wait returns at once; try_wait
// may suspend the thread for a hardware-chosen time, which would let a short
// wait limit pass unnoticed).
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Warp-uniform wait for phase `parity` of the barrier, given up after `limit`
// clock cycles (returns false). Polls with a short sleep between tests, so a
// waiting warp takes few issue slots from the warps that compute.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, long long limit)
{
    if (__all_sync(0xffffffffu, mbar_test(bar, parity))) return true;
    const long long t0 = clock64();
    for (;;) {
        const long long dt = __shfl_sync(0xffffffffu, clock64() - t0, 0);
        if (dt > limit) return false;
        __nanosleep(20);
        if (__all_sync(0xffffffffu, mbar_test(bar, parity))) return true;
    }
}

template <typename T> __device__ __forceinline__ float lds1(const T *p);
template <> __device__ __forceinline__ float lds1<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float lds1<__half>(const __half *p) { return __half2float(*p); }

template <typename T> __device__ __forceinline__ float2 lds2(const T *p);
template <> __device__ __forceinline__ float2 lds2<float>(const float *p) { return *reinterpret_cast<const float2 *>(p); }
template <> __device__ __forceinline__ float2 lds2<__half>(const __half *p)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Shared memory of the row kernel: 2 * S mbarriers in the first 128 bytes,
// then S stages of 19 rows of nx elements.
template <typename T> __host__ __device__ inline int rows_smem_bytes(int nx, int stages)
{
    return 128 + stages * Q * nx * (int)sizeof(T);
}

// Lane a (< 19) of the producer warp copies the source row of population a
// for output row (y, z) into the stage.
template <typename T>
__device__ __forceinline__ void issue_row(const T *__restrict__ src, const Geom &g, int wall, int y, int z, int a,
                                          T *stage, uint32_t bar)
{
    const int ey = ey_of(a), ez = ez_of(a);
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
    int slot = a, ys = y - ey, zs = ez == 1 ? zm : (ez == -1 ? zp : z);
    const bool crosses = (y == 0 && ey == 1) || (y == g.ny - 1 && ey == -1);
    if (crosses) {
        ys = y;
        if (bb_map(wall)) {
            slot = opp_of(a);
            zs = z;
        } else {
            slot = mirror_of(a);
        }
    }
    const T *row = src + (long long)slot * g.plane + ((long long)zs * g.ny + ys) * g.sx;
    bulk_load(smem_addr(stage + (long long)a * g.nx), row, (uint32_t)(g.nx * sizeof(T)), bar);
}

// Populations of the pair (x0, x0 + 1) from a staged row set.
template <typename T>
__device__ __forceinline__ void read_rows(const T *stage, int nx, int wall, int y, int ny, int x0, float2 (&f)[Q])
{
    const bool bottom = y == 0, top = y == ny - 1;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const T *b = stage + (long long)a * nx;
        const int ex = ex_of(a), ey = ey_of(a);
        const bool bb_cross = bb_map(wall) && ((bottom && ey == 1) || (top && ey == -1));
        if (ex == 0 || bb_cross) {
            f[a] = lds2<T>(b + x0);
        } else if (ex == 1) {   // cells read x - 1
            f[a] = make_float2(lds1<T>(b + (x0 == 0 ? nx - 1 : x0 - 1)), lds1<T>(b + x0));
        } else {                // cells read x + 1
            f[a] = make_float2(lds1<T>(b + x0 + 1), lds1<T>(b + (x0 + 2 == nx ? 0 : x0 + 2)));
        }
    }
}

template <typename T, bool STATS, int NW, int COLL = COLL_BGK>
__global__ void __launch_bounds__(NW * 32, 16 / NW) k_step_rows(const T *__restrict__ src, T *__restrict__ dst, Geom g, Phys p,
                                                      float *__restrict__ tw_out, double *__restrict__ part,
                                                      int *__restrict__ err, int S, long long wait_limit)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + ROW_MAX_STAGES;
    T *ring = reinterpret_cast<T *>(smem + 128);
    const long long stage_elems = (long long)Q * g.nx;

    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(smem_addr(full + st), 1);
            mbar_init(smem_addr(empty + st), NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const long long nrows = (long long)g.ny * g.nz;
    const long long mine = blockIdx.x < nrows ? (nrows - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const uint32_t row_bytes = (uint32_t)(stage_elems * sizeof(T));

    auto issue = [&](long long k) {   // warp 0 only
        const long long r = blockIdx.x + k * gridDim.x;
        const int st = (int)(k % S);
        if (lane == 0) mbar_arrive_expect_tx(smem_addr(full + st), row_bytes);
        __syncwarp();
        if (lane < Q)
            issue_row<T>(src, g, p.wall, (int)(r % g.ny), (int)(r / g.ny), lane, ring + st * stage_elems,
                         smem_addr(full + st));
    };

    if (warp == 0)
        for (long long k = 0; k < S - 1 && k < mine; ++k) issue(k);

    for (long long i = 0; i < mine; ++i) {
        if (warp == 0) {
            const long long ahead = i + S - 1;
            if (ahead < mine) {
                const int st = (int)(ahead % S);
                if (ahead >= S && !warp_wait(smem_addr(empty + st), (uint32_t)(((ahead / S) - 1) & 1), wait_limit)) {
                    if (lane == 0) atomicExch(err, 1);
                    for (long long k = i; k < ahead; ++k)   // copies still in flight
                        warp_wait(smem_addr(full + k % S), (uint32_t)((k / S) & 1), WAIT_CYCLES);
                    return;
                }
                issue(ahead);
            }
        }
        const int st = (int)(i % S);
        if (!warp_wait(smem_addr(full + st), (uint32_t)((i / S) & 1), wait_limit)) {
            if (lane == 0) atomicExch(err, 1);
            if (warp == 0) {
                const long long last = (i + S - 1 < mine ? i + S - 1 : mine - 1);
                for (long long k = i; k <= last; ++k)
                    warp_wait(smem_addr(full + k % S), (uint32_t)((k / S) & 1), WAIT_CYCLES);
            }
            return;
        }
        const long long r = blockIdx.x + i * gridDim.x;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        const bool wall_row = y == 0 || y == g.ny - 1;
        const T *stage = ring + st * stage_elems;
        float v[K_ACC];
        if (STATS) stats_zero(v);
        for (int x0 = 2 * (warp * 32 + lane); x0 < g.nx; x0 += 64 * NW) {
            float2 f[Q];
            read_rows<T>(stage, g.nx, p.wall, y, g.ny, x0, f);
            const PairState c = collide_pair<COLL, sizeof(T) == 4>(f, p, row_smag(p, y, g.ny));
            float2 twx = bc(0.f), twz = bc(0.f);
            if (wall_row) {
                float fa[Q], fb[Q];
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    fa[a] = f[a].x;
                    fb[a] = f[a].y;
                }
                const CellState ca{c.rho.x, c.ux.x, c.uy.x, c.uz.x}, cb{c.rho.y, c.ux.y, c.uy.y, c.uz.y};
                wall_layer(fa, ca, p, y == 0, 0xffffffffu, twx.x, twz.x);
                wall_layer(fb, cb, p, y == 0, 0xffffffffu, twx.y, twz.y);
#pragma unroll
                for (int a = 0; a < Q; ++a) f[a] = make_float2(fa[a], fb[a]);
                float4 *t = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(tw_out) +
                                                       ((long long)((y == 0 ? 0 : 1) * g.nz + z) * g.nx + x0));
                *t = make_float4(twx.x, twz.x, twx.y, twz.y);
            }
            T *d = dst + ((long long)z * g.ny + y) * g.sx + x0;
#pragma unroll
            for (int a = 0; a < Q; ++a) st2<T>(d + a * g.plane, f[a]);
            if (STATS) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    stats_cell(v, h ? c.rho.y : c.rho.x, h ? c.ux.y : c.ux.x, h ? c.uy.y : c.uy.x,
                               h ? c.uz.y : c.uz.x, h ? twx.y : twx.x, h ? twz.y : twz.x, wall_row);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(empty + st));
        if (STATS) {
            // warp sums in FP32 (stats_block_store of lbm_kernels.cuh explains
            // why); lane 2k holds sum k, lane 30 the cell count
            const float w = warp_stats_reduce(v);
            const float cnt = __shfl_sync(0xffffffffu, w, 2 * K_PART);
            if (!(lane & 1) && (lane >> 1) < K_PART)
                part[(((long long)y * g.nz + z) * NW + warp) * K_PART + (lane >> 1)] =
                    lane == 0 ? (double)w + (double)cnt : (double)w;
        }
    }
}

}  // namespace lbm
