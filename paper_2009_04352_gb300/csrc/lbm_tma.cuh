// Warp-pipelined form of the fused step for nx a multiple of 64.
//
// Work unit: a segment of 64 cells of one (y, z) row, two cells per lane.
// Each warp owns a private ring of STAGES shared-memory buffers. For every
// segment it will process, lanes 0..18 each issue the bulk copies
// (cp.async.bulk, completion counted on the stage's mbarrier) of one source
// population row: the 64 cells plus a 16-byte halo on each side, taken with
// the periodic wrap at the row ends. The x-shift of the streaming step is then
// an index offset in shared memory, and the z/y shifts and the wall reflection
// (mirror or opposite slot, lbm_device.cuh) are the choice of the source row.
// The copies of the next STAGES-1 segments are in flight while the warp
// computes the current one, so DRAM latency is covered by the ring rather than
// by occupancy. Every wait on an mbarrier is bounded: on timeout the warp sets
// the error flag, waits (bounded) for its copies still in flight and returns.
#pragma once

#include "lbm_pair.cuh"

namespace lbm {

constexpr int SEG = 64;          // cells per segment (two per lane)
constexpr int TMA_WARPS = 4;     // warps per CTA
constexpr int TMA_STAGES = 3;    // segments per warp ring
constexpr long long WAIT_CYCLES = 1LL << 32;   // ~2 s at 2 GHz

template <typename T> __host__ __device__ constexpr int halo() { return 16 / (int)sizeof(T); }
template <typename T> __host__ __device__ constexpr int seg_len() { return SEG + 2 * halo<T>(); }
template <typename T> __host__ __device__ constexpr int stage_elems() { return Q * seg_len<T>(); }

// dynamic shared memory per CTA: mbarriers (128 bytes reserved) then buffers
template <typename T> __host__ __device__ constexpr int tma_smem_bytes()
{
    return 128 + TMA_WARPS * TMA_STAGES * stage_elems<T>() * (int)sizeof(T);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
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

// Warp-uniform bounded wait for phase `parity` of the barrier.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity)
{
    if (__all_sync(0xffffffffu, mbar_test(bar, parity))) return true;
    const long long t0 = clock64();
    for (;;) {
        if (__all_sync(0xffffffffu, mbar_test(bar, parity))) return true;
        const long long dt = __shfl_sync(0xffffffffu, clock64() - t0, 0);
        if (dt > WAIT_CYCLES) return false;
    }
}

struct Seg {
    int y, z, x0;
};

__device__ __forceinline__ Seg seg_of(const Geom &g, long long s)
{
    const int nsx = g.nx / SEG;
    const long long r = s / nsx;
    Seg q;
    q.x0 = (int)(s - r * nsx) * SEG;
    q.y = (int)(r % g.ny);
    q.z = (int)(r / g.ny);
    return q;
}

// Lane a (< 19) issues the copies of population a of segment q into buf.
template <typename T>
__device__ __forceinline__ void issue_population(const T *__restrict__ src, const Geom &g, int wall, const Seg &q, int a,
                                                 T *buf, uint32_t bar)
{
    constexpr int H = halo<T>();
    const int ex = ex_of(a), ey = ey_of(a), ez = ez_of(a);
    (void)ex;
    const int zm = q.z == 0 ? g.nz - 1 : q.z - 1, zp = q.z == g.nz - 1 ? 0 : q.z + 1;
    int slot = a, ys = q.y - ey, zs = ez == 1 ? zm : (ez == -1 ? zp : q.z);
    const bool crosses = (q.y == 0 && ey == 1) || (q.y == g.ny - 1 && ey == -1);
    if (crosses) {
        ys = q.y;
        if (wall == WALL_BB) {
            slot = opp_of(a);
            zs = q.z;
        } else {
            slot = mirror_of(a);
        }
    }
    const T *row = src + (long long)slot * g.plane + ((long long)zs * g.ny + ys) * g.sx;
    T *dst = buf + a * seg_len<T>();
    const int lo = q.x0 == 0 ? 0 : q.x0 - H;
    const int hi = q.x0 + SEG == g.nx ? g.nx : q.x0 + SEG + H;
    if (q.x0 == 0) bulk_load(smem_addr(dst), row + g.nx - H, H * sizeof(T), bar);
    bulk_load(smem_addr(dst + (lo - q.x0 + H)), row + lo, (hi - lo) * sizeof(T), bar);
    if (q.x0 + SEG == g.nx) bulk_load(smem_addr(dst + SEG + H), row, H * sizeof(T), bar);
}

template <typename T>
__device__ __forceinline__ void issue_segment(const T *__restrict__ src, const Geom &g, int wall, long long s, T *buf,
                                              uint32_t bar, int lane)
{
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(stage_elems<T>() * sizeof(T)));
    __syncwarp();
    if (lane < Q) issue_population<T>(src, g, wall, seg_of(g, s), lane, buf, bar);
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

// Populations of the lane's pair from the staged segment.
template <typename T>
__device__ __forceinline__ void read_segment(const T *buf, int wall, bool wall_row, int lane, float2 (&f)[Q], int y,
                                             int ny)
{
    constexpr int H = halo<T>();
    const int i0 = H + 2 * lane;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const T *b = buf + a * seg_len<T>();
        const int ex = ex_of(a), ey = ey_of(a);
        if (ex == 0) {
            f[a] = lds2<T>(b + i0);
        } else {
            const bool bb_cross = wall_row && wall == WALL_BB && ((y == 0 && ey == 1) || (y == ny - 1 && ey == -1));
            if (bb_cross)
                f[a] = lds2<T>(b + i0);
            else
                f[a] = make_float2(lds1<T>(b + i0 - ex), lds1<T>(b + i0 + 1 - ex));
        }
    }
}

template <typename T, bool STATS>
__global__ void __launch_bounds__(TMA_WARPS * 32) k_step_tma(const T *__restrict__ src, T *__restrict__ dst, Geom g,
                                                            Phys p, float *__restrict__ tw_out,
                                                            double *__restrict__ part, int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem) + warp * TMA_STAGES;
    T *ring = reinterpret_cast<T *>(smem + 128) + (long long)warp * TMA_STAGES * stage_elems<T>();

    if (lane == 0)
        for (int st = 0; st < TMA_STAGES; ++st) mbar_init(smem_addr(bars + st), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();

    const long long nseg = (long long)(g.nx / SEG) * g.ny * g.nz;
    const long long gw = (long long)blockIdx.x * TMA_WARPS + warp;
    const long long GW = (long long)gridDim.x * TMA_WARPS;
    const long long mine = gw < nseg ? (nseg - gw + GW - 1) / GW : 0;

    for (long long i = 0; i < TMA_STAGES - 1 && i < mine; ++i)
        issue_segment<T>(src, g, p.wall, gw + i * GW, ring + (i % TMA_STAGES) * stage_elems<T>(),
                         smem_addr(bars + i % TMA_STAGES), lane);

    for (long long i = 0; i < mine; ++i) {
        const long long ahead = i + TMA_STAGES - 1;
        if (ahead < mine) {
            // the stage being refilled was read in iteration i - 1 by this warp
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            issue_segment<T>(src, g, p.wall, gw + ahead * GW, ring + (ahead % TMA_STAGES) * stage_elems<T>(),
                             smem_addr(bars + ahead % TMA_STAGES), lane);
        }
        const int st = (int)(i % TMA_STAGES);
        if (!warp_wait(smem_addr(bars + st), (uint32_t)((i / TMA_STAGES) & 1))) {
            if (lane == 0) atomicExch(err, 1);
            // drain the copies still in flight (bounded) before leaving
            const long long last = ahead < mine ? ahead : mine - 1;
            for (long long k = i; k <= last; ++k)
                warp_wait(smem_addr(bars + k % TMA_STAGES), (uint32_t)((k / TMA_STAGES) & 1));
            return;
        }
        const Seg q = seg_of(g, gw + i * GW);
        const bool wall_row = q.y == 0 || q.y == g.ny - 1;
        float2 f[Q];
        read_segment<T>(ring + st * stage_elems<T>(), p.wall, wall_row, lane, f, q.y, g.ny);
        const PairState c = collide_pair(f, p);

        const int x0 = q.x0 + 2 * lane;
        float2 twx = bc(0.f), twz = bc(0.f);
        if (wall_row) {
            float fa[Q], fb[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                fa[a] = f[a].x;
                fb[a] = f[a].y;
            }
            const CellState ca{c.rho.x, c.ux.x, c.uy.x, c.uz.x}, cb{c.rho.y, c.ux.y, c.uy.y, c.uz.y};
            wall_layer(fa, ca, p, q.y == 0, 0xffffffffu, twx.x, twz.x);
            wall_layer(fb, cb, p, q.y == 0, 0xffffffffu, twx.y, twz.y);
#pragma unroll
            for (int a = 0; a < Q; ++a) f[a] = make_float2(fa[a], fb[a]);
            float4 *t = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(tw_out) +
                                                   ((long long)((q.y == 0 ? 0 : 1) * g.nz + q.z) * g.nx + x0));
            *t = make_float4(twx.x, twz.x, twx.y, twz.y);
        }
        T *d = dst + ((long long)q.z * g.ny + q.y) * g.sx + x0;
#pragma unroll
        for (int a = 0; a < Q; ++a) st2<T>(d + a * g.plane, f[a]);

        if (STATS) {
            double v[K_PART];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const double r = h ? c.rho.y : c.rho.x, ux = h ? c.ux.y : c.ux.x, uy = h ? c.uy.y : c.uy.x,
                             uz = h ? c.uz.y : c.uz.x;
                const double tx = h ? twx.y : twx.x, tz = h ? twz.y : twz.x, m2 = tx * tx + tz * tz;
                const double add[K_PART] = {r,  ux,     uy,     uz, ux * ux, uy * uy,  uz * uz, ux * uy,
                                            r * ux, r * uy, r * uz, tx, tz,  sqrt(m2), m2};
#pragma unroll
                for (int k = 0; k < K_PART; ++k) v[k] = h ? v[k] + add[k] : add[k];
            }
#pragma unroll
            for (int k = 0; k < K_PART; ++k) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
            }
            if (lane < K_PART) {
                double mine_v = 0.0;
#pragma unroll
                for (int k = 0; k < K_PART; ++k)
                    if (lane == k) mine_v = v[k];
                const long long pi = ((long long)q.y * g.nz + q.z) * (g.nx / SEG) + q.x0 / SEG;
                part[pi * K_PART + lane] = mine_v;
            }
        }
    }
}

}  // namespace lbm
