// Two cells per thread: the fast form of the fused step for even nx.
//
// A thread owns the x-pair (x0, x0 + 1), x0 even. Every population is fetched
// with one aligned 2-wide load (float2 for FP32 storage, __half2 for FP16) of
// the source row; the x-shifted directions take the missing neighbour from
// the adjacent lane with a warp shuffle (lane 0 and the last lane of a row
// fetch it directly, with the periodic wrap). The collision runs on both
// cells at once with Blackwell's packed FP32 instructions (fma.rn.f32x2),
// so the instruction count per cell is about half that of the one-cell form.
// Arithmetic is the same as collide() in lbm_kernels.cuh, lane by lane.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <typename T> __device__ __forceinline__ float2 ld2(const T *p);
template <> __device__ __forceinline__ float2 ld2<float>(const float *p)
{
    return __ldg(reinterpret_cast<const float2 *>(p));
}
template <> __device__ __forceinline__ float2 ld2<__half>(const __half *p)
{
    return __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
}

template <typename T> __device__ __forceinline__ void st2(T *p, float2 v);
template <> __device__ __forceinline__ void st2<float>(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
template <> __device__ __forceinline__ void st2<__half>(__half *p, float2 v)
{
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x, v.y);
}

// Values of one source row for the pair (x0, x0 + 1) shifted by SH: the cells
// read x0 - SH and x0 + 1 - SH. `row` points at the start of the source row.
template <typename T, int SH>
__device__ __forceinline__ float2 row_pair(const T *__restrict__ row, int x0, int nx, int lane)
{
    const float2 v = ld2<T>(row + x0);
    if (SH == 0) return v;
    if (SH == 1) {
        float l = __shfl_up_sync(0xffffffffu, v.y, 1);
        if (lane == 0 || x0 == 0) l = ld<T>(row + (x0 == 0 ? nx - 1 : x0 - 1));
        return make_float2(l, v.x);
    }
    float r = __shfl_down_sync(0xffffffffu, v.x, 1);
    if (lane == 31 || x0 + 2 >= nx) r = ld<T>(row + (x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2));
    return make_float2(v.y, r);
}

// Gather of the 19 populations of the pair (streaming with the wall
// reflection of lbm_device.cuh's src_offset, two cells at a time).
template <typename T, int ROW>
__device__ __forceinline__ void gather_pair(const T *__restrict__ src, const Geom &g, int wall, int x0, int y, int z,
                                            int zm, int zp, int lane, float2 (&f)[Q])
{
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int ex = ex_of(a), ey = ey_of(a), ez = ez_of(a);
        const bool crosses = (ROW == ROW_BOTTOM && ey == 1) || (ROW == ROW_TOP && ey == -1);
        const int zs = ez == 1 ? zm : (ez == -1 ? zp : z);
        if (!crosses) {
            const T *row = src + (long long)a * g.plane + ((long long)zs * g.ny + (y - ey)) * g.sx;
            if (ex == 1)
                f[a] = row_pair<T, 1>(row, x0, g.nx, lane);
            else if (ex == -1)
                f[a] = row_pair<T, -1>(row, x0, g.nx, lane);
            else
                f[a] = row_pair<T, 0>(row, x0, g.nx, lane);
        } else if (wall == WALL_BB) {
            const T *row = src + (long long)opp_of(a) * g.plane + ((long long)z * g.ny + y) * g.sx;
            f[a] = row_pair<T, 0>(row, x0, g.nx, lane);
        } else {
            const T *row = src + (long long)mirror_of(a) * g.plane + ((long long)zs * g.ny + y) * g.sx;
            if (ex == 1)
                f[a] = row_pair<T, 1>(row, x0, g.nx, lane);
            else if (ex == -1)
                f[a] = row_pair<T, -1>(row, x0, g.nx, lane);
            else
                f[a] = row_pair<T, 0>(row, x0, g.nx, lane);
        }
    }
}

struct PairState {
    float2 rho, ux, uy, uz;
};

// collide() of lbm_kernels.cuh for two cells (in place: f becomes f*).
__device__ __forceinline__ PairState collide_pair(float2 (&f)[Q], const Phys &p)
{
    PairState c;
    const float2 drho = add2(add2(add2(add2(f[0], f[1]), add2(f[2], f[3])), add2(add2(f[4], f[5]), add2(f[6], f[7]))),
                             add2(add2(add2(f[8], f[9]), add2(f[10], f[11])),
                                  add2(add2(add2(f[12], f[13]), add2(f[14], f[15])),
                                       add2(add2(f[16], f[17]), f[18]))));
    const float2 jx = add2(add2(sub2(f[1], f[2]), sub2(f[7], f[8])),
                           add2(add2(sub2(f[9], f[10]), sub2(f[13], f[14])), sub2(f[15], f[16])));
    const float2 jy = add2(add2(sub2(f[3], f[4]), sub2(f[7], f[8])),
                           add2(add2(sub2(f[11], f[12]), sub2(f[14], f[13])), sub2(f[17], f[18])));
    const float2 jz = add2(add2(sub2(f[5], f[6]), sub2(f[9], f[10])),
                           add2(add2(sub2(f[11], f[12]), sub2(f[16], f[15])), sub2(f[18], f[17])));
    c.rho = add2(bc(1.f), drho);
    const float2 idev = make_float2(-drho.x / c.rho.x, -drho.y / c.rho.y);   // 1/rho - 1
    const float2 jfx = fma2(bc(0.5f), bc(p.Fx), jx), jfy = fma2(bc(0.5f), bc(p.Fy), jy),
                 jfz = fma2(bc(0.5f), bc(p.Fz), jz);
    c.ux = fma2(jfx, idev, jfx);
    c.uy = fma2(jfy, idev, jfy);
    c.uz = fma2(jfz, idev, jfz);
    const float2 rho = c.rho, ux = c.ux, uy = c.uy, uz = c.uz;

    float2 pxx = add2(add2(add2(f[1], f[2]), add2(f[7], f[8])),
                      add2(add2(add2(f[9], f[10]), add2(f[13], f[14])), add2(f[15], f[16])));
    float2 pyy = add2(add2(add2(f[3], f[4]), add2(f[7], f[8])),
                      add2(add2(add2(f[11], f[12]), add2(f[13], f[14])), add2(f[17], f[18])));
    float2 pzz = add2(add2(add2(f[5], f[6]), add2(f[9], f[10])),
                      add2(add2(add2(f[11], f[12]), add2(f[15], f[16])), add2(f[17], f[18])));
    float2 pxy = sub2(add2(f[7], f[8]), add2(f[13], f[14]));
    float2 pxz = sub2(add2(f[9], f[10]), add2(f[15], f[16]));
    float2 pyz = sub2(add2(f[11], f[12]), add2(f[17], f[18]));
    const float2 cd = mul2(drho, bc(1.f / 3.f));
    const float2 rux = mul2(rho, ux), ruy = mul2(rho, uy), ruz = mul2(rho, uz);
    pxx = sub2(pxx, fma2(rux, ux, cd));
    pyy = sub2(pyy, fma2(ruy, uy, cd));
    pzz = sub2(pzz, fma2(ruz, uz, cd));
    pxy = sub2(pxy, mul2(rux, uy));
    pxz = sub2(pxz, mul2(rux, uz));
    pyz = sub2(pyz, mul2(ruy, uz));
    const float2 q2 = fma2(bc(2.f), fma2(pxy, pxy, fma2(pxz, pxz, mul2(pyz, pyz))),
                           fma2(pxx, pxx, fma2(pyy, pyy, mul2(pzz, pzz))));
    float2 omega;
    {
        const float t02 = p.tau0 * p.tau0;
        const float cqx = p.smag * sqrtf(q2.x) / rho.x, cqy = p.smag * sqrtf(q2.y) / rho.y;
        const float tx = p.tau0 + cqx / (2.f * (sqrtf(t02 + cqx) + p.tau0));
        const float ty = p.tau0 + cqy / (2.f * (sqrtf(t02 + cqy) + p.tau0));
        omega = make_float2(1.f / tx, 1.f / ty);
    }
    const float2 gk = fma2(bc(-0.5f), omega, bc(1.f));
    const float2 usq = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
    const float2 uF = fma2(ux, bc(p.Fx), fma2(uy, bc(p.Fy), mul2(uz, bc(p.Fz))));
    const float2 S0 = fma2(bc(-1.5f), mul2(rho, usq), drho);
    const float2 r45 = mul2(bc(4.5f), rho), r3 = mul2(bc(3.f), rho);
    const float2 g9 = mul2(bc(9.f), gk), g3 = mul2(bc(3.f), gk);
    const float2 ng3uF = mul2(bc(-1.f), mul2(g3, uF));

    float2 mass = bc(0.f), mx = bc(0.f), my = bc(0.f), mz = bc(0.f);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int a = 2 * k + 1;
        const float2 w = bc((float)w_of(a));
        float2 eu = bc(0.f);
        if (ex_of(a)) eu = ex_of(a) > 0 ? add2(eu, ux) : sub2(eu, ux);
        if (ey_of(a)) eu = ey_of(a) > 0 ? add2(eu, uy) : sub2(eu, uy);
        if (ez_of(a)) eu = ez_of(a) > 0 ? add2(eu, uz) : sub2(eu, uz);
        const float eFs = ex_of(a) * p.Fx + ey_of(a) * p.Fy + ez_of(a) * p.Fz;
        const float2 eF = bc(eFs);
        const float2 fe = mul2(bc(0.5f), add2(f[a], f[a + 1]));
        const float2 fo = mul2(bc(0.5f), sub2(f[a], f[a + 1]));
        // de = omega (w (S0 + 4.5 rho eu^2) - fe) + w (9 gk eu eF - 3 gk uF)
        const float2 eqe = mul2(w, fma2(mul2(r45, eu), eu, S0));
        const float2 fre = mul2(w, fma2(mul2(g9, eu), eF, ng3uF));
        const float2 de = fma2(omega, sub2(eqe, fe), fre);
        // dd = omega (3 w rho eu - fo) + 3 w gk eF
        const float2 eqo = mul2(w, mul2(r3, eu));
        const float2 dd = fma2(omega, sub2(eqo, fo), mul2(w, mul2(g3, eF)));
        mass = add2(mass, de);
        if (ex_of(a)) mx = ex_of(a) > 0 ? add2(mx, dd) : sub2(mx, dd);
        if (ey_of(a)) my = ey_of(a) > 0 ? add2(my, dd) : sub2(my, dd);
        if (ez_of(a)) mz = ez_of(a) > 0 ? add2(mz, dd) : sub2(mz, dd);
        f[a] = add2(f[a], add2(de, dd));
        f[a + 1] = add2(f[a + 1], sub2(de, dd));
    }
    // exact momentum F and mass 0 of the update (see collide())
    const float2 cx = sub2(bc(0.5f * p.Fx), mx), cy = sub2(bc(0.5f * p.Fy), my), cz = sub2(bc(0.5f * p.Fz), mz);
    f[1] = add2(f[1], cx);
    f[2] = sub2(f[2], cx);
    f[3] = add2(f[3], cy);
    f[4] = sub2(f[4], cy);
    f[5] = add2(f[5], cz);
    f[6] = sub2(f[6], cz);
    f[0] = fma2(bc(-2.f), mass, f[0]);
    return c;
}

template <typename T, bool STATS>
__global__ void __launch_bounds__(128) k_step_pair(const T *__restrict__ src, T *__restrict__ dst, Geom g, Phys p,
                                                   float *__restrict__ tw_out, double *__restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y, z = blockIdx.z;
    const bool valid = x0 < g.nx;
    const int xl = valid ? x0 : g.nx - 2;   // lanes past the row end read in bounds and store nothing
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;

    float2 f[Q];
    if (y == 0)
        gather_pair<T, ROW_BOTTOM>(src, g, p.wall, xl, y, z, zm, zp, lane, f);
    else if (y == g.ny - 1)
        gather_pair<T, ROW_TOP>(src, g, p.wall, xl, y, z, zm, zp, lane, f);
    else
        gather_pair<T, ROW_INTERIOR>(src, g, p.wall, xl, y, z, zm, zp, lane, f);

    const PairState c = collide_pair(f, p);

    float2 twx = bc(0.f), twz = bc(0.f);
    if (y == 0 || y == g.ny - 1) {
        // the wall layer of both cells, lane by lane (all 32 lanes are present)
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
        if (valid) {
            float4 *t = reinterpret_cast<float4 *>(
                reinterpret_cast<float2 *>(tw_out) + ((long long)((y == 0 ? 0 : 1) * g.nz + z) * g.nx + x0));
            *t = make_float4(twx.x, twz.x, twx.y, twz.y);
        }
    }
    if (valid) {
        T *d = dst + ((long long)z * g.ny + y) * g.sx + x0;
#pragma unroll
        for (int a = 0; a < Q; ++a) st2<T>(d + a * g.plane, f[a]);
    }
    if (STATS) {
        double v[K_PART];
#pragma unroll
        for (int k = 0; k < K_PART; ++k) v[k] = 0.0;
        if (valid) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const double r = h ? c.rho.y : c.rho.x, ux = h ? c.ux.y : c.ux.x, uy = h ? c.uy.y : c.uy.x,
                             uz = h ? c.uz.y : c.uz.x;
                const double tx = h ? twx.y : twx.x, tz = h ? twz.y : twz.x, m2 = tx * tx + tz * tz;
                v[0] += r;
                v[1] += ux;
                v[2] += uy;
                v[3] += uz;
                v[4] += ux * ux;
                v[5] += uy * uy;
                v[6] += uz * uz;
                v[7] += ux * uy;
                v[8] += r * ux;
                v[9] += r * uy;
                v[10] += r * uz;
                v[11] += tx;
                v[12] += tz;
                v[13] += sqrt(m2);
                v[14] += m2;
            }
        }
        const long long blk = ((long long)y * g.nz + z) * gridDim.x + blockIdx.x;
        block_reduce_store<K_PART>(v, part + blk * K_PART);
    }
}

}  // namespace lbm
