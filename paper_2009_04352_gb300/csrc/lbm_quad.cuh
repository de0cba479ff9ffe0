// Four cells per thread for FP16 storage (nx a multiple of 4).
//
// FP16 storage halves the bytes per cell, so the per-cell instruction count,
// not DRAM, bounds the two-cell kernel. Here a thread owns the x-quad
// (x0 .. x0 + 3): every population is one aligned 8-byte load of four halves,
// an x-shifted direction costs one warp shuffle and two byte permutes for four
// cells, and every store is one 8-byte store, so the address, load, shuffle
// and store instructions per cell are half those of the two-cell form. The
// collision runs as two packed pairs (collide_pair of lbm_pair.cuh), one after
// the other, on the same raw registers.
#pragma once

#include "lbm_pair.cuh"

namespace lbm {

__device__ __forceinline__ float2 h2f(uint32_t w)
{
    __half2 h = *reinterpret_cast<__half2 *>(&w);
    return __half22float2(h);
}

__device__ __forceinline__ uint32_t f2h(float2 v)
{
    __half2 h = __floats2half2_rn(v.x, v.y);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Four halves of one source row for cells x0 .. x0 + 3 shifted by SH (cell x
// reads x - SH), as two 32-bit words (x0, x0 + 1 | x0 + 2, x0 + 3), lower
// element in the low half.
template <bool NC>
__device__ __forceinline__ uint2 ld_u2(const __half *p)
{
    return NC ? __ldg(reinterpret_cast<const uint2 *>(p)) : __ldca(reinterpret_cast<const uint2 *>(p));
}

template <bool NC>
__device__ __forceinline__ uint32_t ld_u16(const __half *p)
{
    return NC ? (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(p))
              : (uint32_t)__ldca(reinterpret_cast<const unsigned short *>(p));
}

template <int SH, bool NC = true>
__device__ __forceinline__ uint2 row_quad(const __half *row, int x0, int nx, int lane)
{
    const uint2 v = ld_u2<NC>(row + x0);
    if (SH == 0) return v;
    if (SH == 1) {   // (x0 - 1, x0 | x0 + 1, x0 + 2)
        uint32_t lw = __shfl_up_sync(0xffffffffu, v.y, 1);   // (x0 - 2, x0 - 1) of the left lane
        if (lane == 0 || x0 == 0) {
            const int xl = x0 == 0 ? nx - 1 : x0 - 1;
            lw = ld_u16<NC>(row + xl) << 16;
        }
        return make_uint2(__byte_perm(lw, v.x, 0x5432), __byte_perm(v.x, v.y, 0x5432));
    }
    // SH == -1: (x0 + 1, x0 + 2 | x0 + 3, x0 + 4)
    uint32_t rw = __shfl_down_sync(0xffffffffu, v.x, 1);     // (x0 + 4, x0 + 5) of the right lane
    if (lane == 31 || x0 + 4 >= nx) {
        const int xr = x0 + 4 >= nx ? x0 + 4 - nx : x0 + 4;
        rw = ld_u16<NC>(row + xr);
    }
    return make_uint2(__byte_perm(v.x, v.y, 0x5432), __byte_perm(v.y, rw, 0x5432));
}

// Gather of the quad (streaming with the wall reflection of src_offset); the
// layouts as in gather_pair of lbm_pair.cuh. The four-cell wall rows serve
// halfway walls only (with wall nodes the step runs its interior rows with the
// four-cell tile and the node rows with the two-cell wall tile), so the
// bounce-back map is taken for WALL_BB alone.
template <int ROW, int LAY = LAY_PULL>
__device__ __forceinline__ void gather_quad(const __half *src, const Geom &g, int wall, int x0, int y, int z, int zm,
                                            int zp, int lane, uint2 (&r)[Q])
{
    constexpr bool NC = LAY == LAY_PULL && pull_nc<__half>;   // coherent: the quad kernels launch with PDL
    if constexpr (LAY == LAY_AA_EVEN) {
        const __half *own = src + ((long long)z * g.ny + y) * g.sx + x0;
#pragma unroll
        for (int a = 0; a < Q; ++a) r[a] = ld_u2<false>(own + a * g.plane);
    } else {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int ex = ex_of(a), ey = ey_of(a), ez = ez_of(a);
            const bool crosses = (ROW == ROW_BOTTOM && ey == 1) || (ROW == ROW_TOP && ey == -1);
            const int zs = ez == 1 ? zm : (ez == -1 ? zp : z);
            const int sa = LAY == LAY_AA_ODD ? opp_of(a) : a;
            if (!crosses) {
                const __half *row = src + (long long)sa * g.plane + ((long long)zs * g.ny + (y - ey)) * g.sx;
                if (ex == 1)
                    r[a] = row_quad<1, NC>(row, x0, g.nx, lane);
                else if (ex == -1)
                    r[a] = row_quad<-1, NC>(row, x0, g.nx, lane);
                else
                    r[a] = row_quad<0, NC>(row, x0, g.nx, lane);
            } else if (wall == WALL_BB) {
                const int sb = LAY == LAY_AA_ODD ? a : opp_of(a);
                const __half *row = src + (long long)sb * g.plane + ((long long)z * g.ny + y) * g.sx;
                r[a] = row_quad<0, NC>(row, x0, g.nx, lane);
            } else {
                const int sm = LAY == LAY_AA_ODD ? opp_of(mirror_of(a)) : mirror_of(a);
                const __half *row = src + (long long)sm * g.plane + ((long long)zs * g.ny + y) * g.sx;
                if (ex == 1)
                    r[a] = row_quad<1, NC>(row, x0, g.nx, lane);
                else if (ex == -1)
                    r[a] = row_quad<-1, NC>(row, x0, g.nx, lane);
                else
                    r[a] = row_quad<0, NC>(row, x0, g.nx, lane);
            }
        }
    }
}

__device__ __forceinline__ void st_u16(__half *p, uint32_t v) { *reinterpret_cast<unsigned short *>(p) = (unsigned short)v; }
__device__ __forceinline__ void st_u32(__half *p, uint32_t v) { *reinterpret_cast<uint32_t *>(p) = v; }

// Store of the quad's four halves into one row shifted by SH (the AA push;
// push_row of lbm_pair.cuh for four cells). Interior lanes store one aligned
// 8-byte word built with a shuffle and byte permutes; at the warp and row ends
// the crossing element is stored alone. All 32 lanes must call it.
template <int SH>
__device__ __forceinline__ void push_row_quad(__half *row, int x0, int nx, int lane, bool valid, uint2 v)
{
    if (SH == 0) {
        if (valid) *reinterpret_cast<uint2 *>(row + x0) = v;
        return;
    }
    if (SH == 1) {   // cells x0 .. x0 + 3 -> x0 + 1 .. x0 + 4
        const uint32_t lw = __shfl_up_sync(0xffffffffu, v.y, 1);   // (x0 - 2, x0 - 1) of the left lane
        if (!valid) return;
        if (lane == 0 || x0 == 0) {
            st_u16(row + x0 + 1, v.x & 0xffffu);
            st_u32(row + x0 + 2, __byte_perm(v.x, v.y, 0x5432));
        } else {
            *reinterpret_cast<uint2 *>(row + x0) = make_uint2(__byte_perm(lw, v.x, 0x5432), __byte_perm(v.x, v.y, 0x5432));
        }
        if (lane == 31 || x0 + 4 >= nx) st_u16(row + (x0 + 4 >= nx ? x0 + 4 - nx : x0 + 4), v.y >> 16);
        return;
    }
    // SH == -1: cells x0 .. x0 + 3 -> x0 - 1 .. x0 + 2
    const uint32_t rw = __shfl_down_sync(0xffffffffu, v.x, 1);   // (x0 + 4, x0 + 5) of the right lane
    if (!valid) return;
    if (lane == 31 || x0 + 4 >= nx) {
        st_u32(row + x0, __byte_perm(v.x, v.y, 0x5432));
        st_u16(row + x0 + 2, v.y >> 16);
    } else {
        *reinterpret_cast<uint2 *>(row + x0) = make_uint2(__byte_perm(v.x, v.y, 0x5432), __byte_perm(v.y, rw, 0x5432));
    }
    if (lane == 0 || x0 == 0) st_u16(row + (x0 == 0 ? nx - 1 : x0 - 1), v.x & 0xffffu);
}

// AA odd step store of the quad (push_offset of lbm_device.cuh, four cells).
template <int ROW>
__device__ __forceinline__ void push_quad(__half *dst, const Geom &g, int wall, int x0, int y, int z, int zm, int zp,
                                          int lane, bool valid, const uint2 (&r)[Q])
{
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int ex = ex_of(a), ey = ey_of(a), ez = ez_of(a);
        const bool crosses = (ROW == ROW_BOTTOM && ey == -1) || (ROW == ROW_TOP && ey == 1);
        const int zt = ez == 1 ? zp : (ez == -1 ? zm : z);
        if (!crosses) {
            __half *row = dst + (long long)a * g.plane + ((long long)zt * g.ny + (y + ey)) * g.sx;
            if (ex == 1)
                push_row_quad<1>(row, x0, g.nx, lane, valid, r[a]);
            else if (ex == -1)
                push_row_quad<-1>(row, x0, g.nx, lane, valid, r[a]);
            else
                push_row_quad<0>(row, x0, g.nx, lane, valid, r[a]);
        } else if (wall == WALL_BB) {
            __half *row = dst + (long long)opp_of(a) * g.plane + ((long long)z * g.ny + y) * g.sx;
            push_row_quad<0>(row, x0, g.nx, lane, valid, r[a]);
        } else {
            __half *row = dst + (long long)mirror_of(a) * g.plane + ((long long)zt * g.ny + y) * g.sx;
            if (ex == 1)
                push_row_quad<1>(row, x0, g.nx, lane, valid, r[a]);
            else if (ex == -1)
                push_row_quad<-1>(row, x0, g.nx, lane, valid, r[a]);
            else
                push_row_quad<0>(row, x0, g.nx, lane, valid, r[a]);
        }
    }
}

// Collision (and wall layer) of one packed pair held in word H of the quad.
// The pair-sum form of collide_pair (PS, same bits) measured faster for MRT
// and for the AA even step, slower for the BGK pull and AA odd steps, whose
// register allocation it worsens (c4: 72.6 against 79.8 GLUPS pull).
template <int H, bool STATS, int COLL, int LAY>
__device__ __forceinline__ void quad_half(uint2 (&r)[Q], const Phys &p, float smag, bool wall_row, bool bottom,
                                          float4 &tw, float (&v)[K_ACC], bool valid)
{
    float2 f[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) f[a] = h2f(H ? r[a].y : r[a].x);
    const PairState c = collide_pair<COLL, false, COLL == COLL_MRT || LAY == LAY_AA_EVEN>(f, p, smag);
    float2 twx = bc(0.f), twz = bc(0.f);
    if (wall_row) {
        wall_layer_pair(f, c, p, bottom, twx, twz);
        tw = make_float4(twx.x, twz.x, twx.y, twz.y);
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        if (H)
            r[a].y = f2h(f[a]);
        else
            r[a].x = f2h(f[a]);
    }
    if (STATS && valid) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            stats_cell(v, h ? c.rho.y : c.rho.x, h ? c.ux.y : c.ux.x, h ? c.uy.y : c.uy.x, h ? c.uz.y : c.uz.x,
                       h ? twx.y : twx.x, h ? twz.y : twz.x, wall_row);
        }
    }
}

#ifndef LBM_QUAD_MIN_BLOCKS
#define LBM_QUAD_MIN_BLOCKS 5   // resident CTAs per SM the register budget must allow
#endif
#ifndef LBM_QUAD_MRT_MIN_BLOCKS
#define LBM_QUAD_MRT_MIN_BLOCKS 4   // the same for the MRT instantiations (128 registers)
#endif
#ifndef LBM_QUAD_STATS_MIN_BLOCKS
#define LBM_QUAD_STATS_MIN_BLOCKS 4   // sampled steps (16 FP32 accumulators more): 128 registers
#endif
#ifndef LBM_QUAD_AA_MIN_BLOCKS
#define LBM_QUAD_AA_MIN_BLOCKS 4    // the same for the in-place AA steps with BGK (128 registers)
#endif
#ifndef LBM_QUAD_AA_ROWS_MIN_BLOCKS
#define LBM_QUAD_AA_ROWS_MIN_BLOCKS 4   // AA steps with the wall tile called (k_step_quad_aa_rows)
#endif

// One tile: the x-quads xb * blockDim.x + threadIdx.x of row (y, z), i.e.
// cells [4 xb blockDim.x, 4 (xb + 1) blockDim.x). With STATS the block writes
// its FP64 partial sums to part_blk[0..K_PART).
// The two-lattice four-cell step serves the row sets of pair_tile (lbm_pair.cuh):
// every row, the interior rows 1 .. ny - 2 only (their instantiation carries
// no wall-layer code), or the two wall rows only.

// Collision, wall layer, store (or AA push) and statistics of the quad whose
// 19 populations the gather left in r (the part of a tile after its loads).
template <bool STATS, int COLL, int LAY, int ROWS>
__device__ __forceinline__ void quad_finish(uint2 (&r)[Q], __half *dst, const Geom &g, const Phys &p,
                                            float *__restrict__ tw_out, double *__restrict__ part_blk, int x0, int xl,
                                            bool valid, int y, int z, int zm, int zp, int lane)
{
    const bool wall_row = ROWS == ROWS_INTERIOR ? false : (ROWS == ROWS_WALL ? true : (y == 0 || y == g.ny - 1));
    float v[K_ACC];
    if (STATS) stats_zero(v);
    float4 twa = make_float4(0.f, 0.f, 0.f, 0.f), twb = twa;
    const float smag = row_smag(p, y, g.ny);
    quad_half<0, STATS, COLL, LAY>(r, p, smag, wall_row, y == 0, twa, v, valid);
    quad_half<1, STATS, COLL, LAY>(r, p, smag, wall_row, y == 0, twb, v, valid);
    if (valid && wall_row) {
        float4 *t = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(tw_out) +
                                               ((long long)((y == 0 ? 0 : 1) * g.nz + z) * g.nx + x0));
        t[0] = twa;
        t[1] = twb;
    }
    if (LAY == LAY_AA_ODD) {
        if (ROWS != ROWS_INTERIOR && y == 0)
            push_quad<ROW_BOTTOM>(dst, g, p.wall, xl, y, z, zm, zp, lane, valid, r);
        else if (ROWS != ROWS_INTERIOR && y == g.ny - 1)
            push_quad<ROW_TOP>(dst, g, p.wall, xl, y, z, zm, zp, lane, valid, r);
        else
            push_quad<ROW_INTERIOR>(dst, g, p.wall, xl, y, z, zm, zp, lane, valid, r);
    } else if (valid) {
        __half *d = dst + ((long long)z * g.ny + y) * g.sx + x0;
#pragma unroll
        for (int a = 0; a < Q; ++a)
            *reinterpret_cast<uint2 *>(d + (LAY == LAY_AA_EVEN ? opp_of(a) : a) * g.plane) = r[a];
    }
    if (STATS) stats_block_store(v, part_blk);
}

template <bool STATS, int COLL = COLL_BGK, int LAY = LAY_PULL, int ROWS = ROWS_ALL>
__device__ __forceinline__ void quad_tile(const __half *src, __half *dst, const Geom &g, const Phys &p,
                                          float *__restrict__ tw_out, double *__restrict__ part_blk, int xb, int y,
                                          int z)
{
    const int lane = threadIdx.x & 31;
    const int x0 = 4 * (xb * blockDim.x + threadIdx.x);
    const bool valid = x0 < g.nx;
    const int xl = valid ? x0 : g.nx - 4;   // lanes past the row end read in bounds and store nothing
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;

    uint2 r[Q];
    if (ROWS != ROWS_INTERIOR && y == 0)
        gather_quad<ROW_BOTTOM, LAY>(src, g, p.wall, xl, y, z, zm, zp, lane, r);
    else if (ROWS != ROWS_INTERIOR && y == g.ny - 1)
        gather_quad<ROW_TOP, LAY>(src, g, p.wall, xl, y, z, zm, zp, lane, r);
    else
        gather_quad<ROW_INTERIOR, LAY>(src, g, p.wall, xl, y, z, zm, zp, lane, r);
    quad_finish<STATS, COLL, LAY, ROWS>(r, dst, g, p, tw_out, part_blk, x0, xl, valid, y, z, zm, zp, lane);
}

// The two-lattice step over the row set ROWS: grid.y is ny (ROWS_ALL), ny - 2
// (ROWS_INTERIOR, row blockIdx.y + 1) or 2 (ROWS_WALL, rows 0 and ny - 1).
// The step runs as an interior launch and a wall-row launch, so that the wall
// layer's code does not shape the register allocation of the interior rows.
template <bool STATS, int COLL = COLL_BGK, int ROWS = ROWS_ALL>
__global__ void __launch_bounds__(128, COLL == COLL_MRT ? LBM_QUAD_MRT_MIN_BLOCKS
                                                         : (STATS ? LBM_QUAD_STATS_MIN_BLOCKS : LBM_QUAD_MIN_BLOCKS))
    k_step_quad(const __half *__restrict__ src,
                                                                         __half *__restrict__ dst, Geom g, Phys p,
                                                                         float *__restrict__ tw_out,
                                                                         double *__restrict__ part)
{
    pdl_begin();
    const int y = ROWS == ROWS_INTERIOR ? (int)blockIdx.y + 1
                                        : (ROWS == ROWS_WALL ? (blockIdx.y == 0 ? 0 : g.ny - 1) : (int)blockIdx.y);
    const int z = blockIdx.z;
    const long long blk = ((long long)y * g.nz + z) * gridDim.x + blockIdx.x;
    quad_tile<STATS, COLL, LAY_PULL, ROWS>(src, dst, g, p, tw_out, STATS ? part + blk * K_PART : nullptr,
                                           blockIdx.x, y, z);
}

// The wall-row tile of the two-lattice four-cell step as a separate function:
// called from k_step_quad_rows, it is compiled apart from the interior tile,
// so the wall layer's code does not shape the interior's register allocation.
template <bool STATS, int COLL>
__device__ __noinline__ void quad_wall_tile(const __half *src, __half *dst, const Geom &g, const Phys &p,
                                            float *tw_out, double *part_blk, int xb, int y, int z)
{
    quad_tile<STATS, COLL, LAY_PULL, ROWS_WALL>(src, dst, g, p, tw_out, part_blk, xb, y, z);
}

// The two-lattice four-cell step over every row in one launch: rows 1 .. ny - 2
// run the interior tile inline, rows 0 and ny - 1 call quad_wall_tile. Unlike a
// separate wall-row launch, the wall rows' CTAs (Newton iterations of the wall
// law) overlap with the interior ones instead of running after them.
template <bool STATS, int COLL>
__global__ void __launch_bounds__(128, COLL == COLL_MRT ? LBM_QUAD_MRT_MIN_BLOCKS
                                                         : (STATS ? LBM_QUAD_STATS_MIN_BLOCKS : LBM_QUAD_MIN_BLOCKS))
    k_step_quad_rows(const __half *__restrict__ src, __half *__restrict__ dst, Geom g, Phys p,
                     float *__restrict__ tw_out, double *__restrict__ part)
{
    pdl_begin();
    const int y = blockIdx.y, z = blockIdx.z;
    const long long blk = ((long long)y * g.nz + z) * gridDim.x + blockIdx.x;
    double *pb = STATS ? part + blk * K_PART : nullptr;
    if (y == 0 || y == g.ny - 1)
        quad_wall_tile<STATS, COLL>(src, dst, g, p, tw_out, pb, blockIdx.x, y, z);
    else
        quad_tile<STATS, COLL, LAY_PULL, ROWS_INTERIOR>(src, dst, g, p, tw_out, pb, blockIdx.x, y, z);
}

// The four-cell step on the single AA array (LAY_AA_EVEN or LAY_AA_ODD) over
// the row set ROWS (grid.y ny, or ny - 2 for the interior rows, row
// blockIdx.y + 1).
template <bool STATS, int COLL, int LAY, int ROWS = ROWS_ALL>
__global__ void __launch_bounds__(128, COLL == COLL_MRT ? LBM_QUAD_MRT_MIN_BLOCKS
                                                         : (STATS ? LBM_QUAD_STATS_MIN_BLOCKS : LBM_QUAD_AA_MIN_BLOCKS))
    k_step_quad_aa(__half *f, Geom g, Phys p,
                                                                            float *__restrict__ tw_out,
                                                                            double *__restrict__ part)
{
    pdl_begin();
    const int y = ROWS == ROWS_INTERIOR ? (int)blockIdx.y + 1 : (int)blockIdx.y, z = blockIdx.z;
    const long long blk = ((long long)y * g.nz + z) * gridDim.x + blockIdx.x;
    quad_tile<STATS, COLL, LAY, ROWS>(f, f, g, p, tw_out, STATS ? part + blk * K_PART : nullptr, blockIdx.x, y, z);
}

// The wall-row tile of the four-cell AA step, compiled apart from the
// interior tile (see quad_wall_tile).
template <bool STATS, int COLL, int LAY>
__device__ __noinline__ void quad_aa_wall_tile(__half *f, const Geom &g, const Phys &p, float *tw_out,
                                               double *part_blk, int xb, int y, int z)
{
    quad_tile<STATS, COLL, LAY, ROWS_WALL>(f, f, g, p, tw_out, part_blk, xb, y, z);
}

// The four-cell AA step over every row in one launch, the wall rows' CTAs
// calling quad_aa_wall_tile, the interior rows running the interior tile
// inline (its registers are not shaped by the wall layer's code).
template <bool STATS, int COLL, int LAY>
__global__ void __launch_bounds__(128, LBM_QUAD_AA_ROWS_MIN_BLOCKS)
    k_step_quad_aa_rows(__half *f, Geom g, Phys p, float *__restrict__ tw_out, double *__restrict__ part)
{
    pdl_begin();
    const int y = blockIdx.y, z = blockIdx.z;
    const long long blk = ((long long)y * g.nz + z) * gridDim.x + blockIdx.x;
    double *pb = STATS ? part + blk * K_PART : nullptr;
    if (y == 0 || y == g.ny - 1)
        quad_aa_wall_tile<STATS, COLL, LAY>(f, g, p, tw_out, pb, blockIdx.x, y, z);
    else
        quad_tile<STATS, COLL, LAY, ROWS_INTERIOR>(f, f, g, p, tw_out, pb, blockIdx.x, y, z);
}

}  // namespace lbm
