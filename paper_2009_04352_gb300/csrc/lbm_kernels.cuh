// Kernels of the fused LBM-LES channel step (see lbm_device.cuh for the
// storage scheme). One thread updates one cell; a block covers a run of x
// cells of one (y, z) row, so the wall-layer branch is uniform per block.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Post-collision populations of one cell: BGK with the Smagorinsky relaxation
// time and the Guo forcing (Eq. 1), on deviations fb_a = f_a - w_a:
//   rho = 1 + drho, u = (j + F/2) / rho (Eq. 2 with the Guo half-force shift)
//   Pi_neq = sum e e (f - f^eq) = sum e e fb - c_s^2 drho I - rho u u
//   tau_eff = (tau0 + sqrt(tau0^2 + 18 sqrt(2) C_s^2 |Pi_neq| / rho)) / 2
//   fb*_a = fb_a + omega (f^eq_a - w_a - fb_a) + F_a,  omega = 1 / tau_eff
//   f^eq_a - w_a = w_a [drho + rho (3 e.u + 9/2 (e.u)^2 - 3/2 u.u)]
//   F_a = (1 - omega / 2) w_a [3 (e_a - u) . F + 9 (e_a . u)(e_a . F)]
// The update is formed per opposite pair from its even and odd parts. In
// exact arithmetic sum delta = 0 and sum e delta = F. FP32 roundings that
// repeat the same way in every cell add up over the channel to a momentum
// error of the order of a percent of the channels' body force (~1e-8 of
// rho u per step against F ~ 4e-8): the rounded weights 1/18 and 1/36 break
// the lattice sums, and the small half force added to j rounds to whole ulps
// of j alike everywhere. Here the weights are scaled by 36 (36 w = 12, 2, 1:
// exact) with 1/36 folded into the rate, the non-equilibrium difference is
// formed before the rate multiplies it, and the odd (momentum) part uses
// rho (e.u) = e.(j + F/2) directly. The axis pairs then take the small
// momentum residual, so sum e delta = F exactly up to the final store, and
// the rest population its own update (mass change zero up to unbiased
// roundings). The FP16-storage form of the packed kernels (lbm_pair.cuh)
// keeps rounded weights with the rate folded in and corrects mass and
// momentum on the rest population and the axis pairs.
struct CellState {
    float rho, ux, uy, uz;
};

// u = (j + F/2) / rho evaluated as j + (j (1/rho - 1) + (F/2) / rho) with
// 1/rho - 1 = -drho / rho: no rounded 1/rho near 1, and the half force, a few
// ulps of j in the channels, is added to a value that varies from cell to
// cell rather than straight to j, whose rounding would move it to whole ulps
// of j the same way everywhere.
__device__ __forceinline__ CellState velocity(const Moments &m, const Phys &p)
{
    CellState c;
    c.rho = 1.f + m.drho;
    const float idev = -m.drho / c.rho;
    c.ux = m.jx + fmaf(m.jx, idev, fmaf(p.hF[0], idev, p.hF[0]));
    c.uy = m.jy + fmaf(m.jy, idev, fmaf(p.hF[1], idev, p.hF[1]));
    c.uz = m.jz + fmaf(m.jz, idev, fmaf(p.hF[2], idev, p.hF[2]));
    return c;
}

template <int COLL = COLL_BGK>
__device__ __forceinline__ CellState collide(const float (&f)[Q], float (&fs)[Q], const Phys &p, float smag)
{
    const Moments m = moments_of(f);
    const CellState c = velocity(m, p);
    const float ux = c.ux, uy = c.uy, uz = c.uz, rho = c.rho;

    // second moments of the deviations
    float pxx = ((f[1] + f[2]) + (f[7] + f[8])) + ((f[9] + f[10]) + (f[13] + f[14])) + (f[15] + f[16]);
    float pyy = ((f[3] + f[4]) + (f[7] + f[8])) + ((f[11] + f[12]) + (f[13] + f[14])) + (f[17] + f[18]);
    float pzz = ((f[5] + f[6]) + (f[9] + f[10])) + ((f[11] + f[12]) + (f[15] + f[16])) + (f[17] + f[18]);
    float pxy = (f[7] + f[8]) - (f[13] + f[14]);
    float pxz = (f[9] + f[10]) - (f[15] + f[16]);
    float pyz = (f[11] + f[12]) - (f[17] + f[18]);
    const float cd = m.drho * (1.f / 3.f);
    pxx -= cd + rho * ux * ux;
    pyy -= cd + rho * uy * uy;
    pzz -= cd + rho * uz * uz;
    pxy -= rho * ux * uy;
    pxz -= rho * ux * uz;
    pyz -= rho * uy * uz;
    const float q2 = (pxx * pxx + pyy * pyy + pzz * pzz) + 2.f * (pxy * pxy + pxz * pxz + pyz * pyz);
    // positive root of tau^2 - tau0 tau - smag Q / (4 rho) = 0, written as
    // tau0 + (root - tau0) so that a small eddy viscosity is not lost to
    // cancellation against tau0
    const float cq = smag * sqrtf(q2) / rho;
    const float tau = p.tau0 + cq / (2.f * (sqrtf(p.tau0 * p.tau0 + cq) + p.tau0));
    const float omega = 1.f / tau;
    const float gk = 1.f - 0.5f * omega;

    const float usq = ux * ux + uy * uy + uz * uz;
    const float uF = fmaf(ux, p.Fx, fmaf(uy, p.Fy, uz * p.Fz));
    // MRT (d'Humieres et al. 2002): BGK plus the corrections of the ghost
    // groups e, eps, q, m whose rates differ from omega (mrt_ghost_pair in
    // lbm_pair.cuh states the brackets); the pair k of the loop below then
    // changes by ge[k] in its half sum and go[k] in its half difference
    float ge_ax = 0.f, ge_dg = 0.f, ge_rest = 0.f, go[9];
    if constexpr (COLL == COLL_MRT) {
        float hs[9], hd[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            hs[k] = 0.5f * (f[2 * k + 1] + f[2 * k + 2]);
            hd[k] = 0.5f * (f[2 * k + 1] - f[2 * k + 2]);
        }
        const float A = hs[0] + hs[1] + hs[2];
        const float D = ((hs[3] + hs[4]) + (hs[5] + hs[6])) + (hs[7] + hs[8]);
        const float du = rho * usq - uF;
        const float ce = fmaf(omega, p.mrt_a[MRT_E], p.mrt_b[MRT_E]) * ((2.f * D - f[0]) - du);
        const float cp = fmaf(omega, p.mrt_a[MRT_EPS], p.mrt_b[MRT_EPS]) *
                         fmaf(9.f, f[0], fmaf(-14.f, A, fmaf(-4.f, D, 5.5f * du)));
        ge_ax = fmaf(-11.f, ce, -4.f * cp);
        ge_dg = fmaf(8.f, ce, cp);
        ge_rest = fmaf(-30.f, ce, 12.f * cp);
        const float kq = fmaf(omega, p.mrt_a[MRT_Q], p.mrt_b[MRT_Q]);
        const float km = fmaf(omega, p.mrt_a[MRT_M], p.mrt_b[MRT_M]);
        const float sxa = hd[3] + hd[6], sxb = hd[4] + hd[7];
        const float sya = hd[5] + hd[8], syb = hd[3] - hd[6];
        const float sza = hd[4] - hd[7], szb = hd[5] - hd[8];
        const float qx = kq * fmaf(-2.f, hd[0], sxa + sxb);
        const float qy = kq * fmaf(-2.f, hd[1], sya + syb);
        const float qz = kq * fmaf(-2.f, hd[2], sza + szb);
        const float mx = km * (sxa - sxb), my = km * (sya - syb), mz = km * (sza - szb);
        const float t36a = qx + mx, t36b = qy - my, t47a = qx - mx, t47b = qz + mz, t58a = qy + my,
                    t58b = qz - mz;
        go[0] = -4.f * qx;
        go[1] = -4.f * qy;
        go[2] = -4.f * qz;
        go[3] = t36a + t36b;
        go[4] = t47a + t47b;
        go[5] = t58a + t58b;
        go[6] = t36a - t36b;
        go[7] = t47a - t47b;
        go[8] = t58a - t58b;
    }
    // BGK (see the comment above the struct): weights scaled by 36, o36 = omega / 36
    const float S0 = fmaf(-1.5f, rho * usq, m.drho);   // isotropic part of (f^eq - w) / w
    const float o36 = omega * (1.f / 36.f);
    const float r45 = 4.5f * rho;
    const float g9 = 0.25f * gk, g3 = (1.f / 12.f) * gk;   // 9 gk / 36, 3 gk / 36
    const float mgu = (-1.f / 12.f) * gk * uF;              // -3 gk u.F / 36
    float d0 = fmaf(o36, fmaf(-36.f, f[0], 12.f * S0), 12.f * mgu);
    if constexpr (COLL == COLL_MRT) d0 += ge_rest;
    fs[0] = f[0] + d0;
    float de[9], dd[9];
    float mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int a = 2 * k + 1;
        const float W = k < 3 ? 2.f : 1.f;   // 36 w
        const float eu = ex_of(a) * ux + ey_of(a) * uy + ez_of(a) * uz;
        const float ej = ex_of(a) * m.jx + ey_of(a) * m.jy + ez_of(a) * m.jz;
        const float WeF = p.WeF[k];
        const float fe = 0.5f * (f[a] + f[a + 1]);
        const float fo = 0.5f * (f[a] - f[a + 1]);
        // 36 (f^eq - f) of the pair's even and odd parts, rho (e.u) = e.(j + F/2)
        const float ne = fmaf(W * r45 * eu, eu, fmaf(-36.f, fe, W * S0));
        const float nd = fmaf(3.f * W, ej, fmaf(-36.f, fo, 1.5f * WeF));
        de[k] = fmaf(o36, ne, fmaf(g9 * WeF, eu, W * mgu));
        dd[k] = fmaf(o36, nd, g3 * WeF);
        if constexpr (COLL == COLL_MRT) {
            de[k] += k < 3 ? ge_ax : ge_dg;
            dd[k] += go[k];
        }
        if (ex_of(a)) mx += ex_of(a) * dd[k];
        if (ey_of(a)) my += ey_of(a) * dd[k];
        if (ez_of(a)) mz += ez_of(a) * dd[k];
    }
    // pairs 0, 1, 2 are the axis directions 1, 3, 5: they take the momentum
    // residual, so that sum e delta = F exactly up to the final store
    dd[0] += 0.5f * p.Fx - mx;
    dd[1] += 0.5f * p.Fy - my;
    dd[2] += 0.5f * p.Fz - mz;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int a = 2 * k + 1;
        fs[a] = f[a] + (de[k] + dd[k]);
        fs[a + 1] = f[a + 1] + (de[k] - dd[k]);
    }
    return c;
}

// Wall layer after collision: the wall stress and, for WFB, the Eq. 14a,b
// correction folded into the wall-bound slots. A population b leaving toward
// the wall returns through the specular partner of b, displaced by b's
// tangential velocity, and must carry +(1/2) tau_w . e_b (dt = dy = 1): at the
// bottom wall 13 -> 7 (+x), 8 -> 14 (-x), 18 -> 11 (+z), 12 -> 17 (-z); at the
// top wall 7 -> 13, 14 -> 8, 11 -> 18, 17 -> 12. The stress itself is
// tau_w = rho u_tau^2 with u_tau = |u_t| / u+ from Spalding's law, directed
// against the tangential velocity (Eq. 15). For bounce-back the reported stress
// is the tangential momentum the reflection returns, -2 sum e_b,t f*_b.
// Wall shear stress of the wall function from the state c of the cell that
// feeds it (Eqs. 15-17): |tau_w| = rho (|u_t| / u+)^2 against u_t. The lanes
// in `lanes` iterate the wall law together. Roundings are explicit here and in
// the wall laws, so every kernel form computes the same tau_w.
__device__ __forceinline__ void wfb_stress(const CellState &c, const Phys &p, unsigned lanes, float &twx, float &twz)
{
    twx = 0.f;
    twz = 0.f;
    const float ut = sqrtf(__fmaf_rn(c.uz, c.uz, __fmul_rn(c.ux, c.ux)));
    const float R = fmaxf(p.y1_over_nu * ut, 1e-30f);
    const float up = wall_uplus(R, p, lanes);
    const float utau = ut / up;
    const float tw = c.rho * utau * utau;
    if (ut > 0.f) {
        twx = -c.ux / ut * tw;
        twz = -c.uz / ut * tw;
    }
}

// Full-way WFB at a wall node (layer 0 or ny - 1, WALL_NODE): f holds the
// node's gathered populations and ca the state of the first fluid node. fs
// receives what the node sends out: for each population b entering the fluid
// the specular partner of the one that arrived from it plus (tau_w . e_b) / 2
// (Eqs. 13, 14a,b; the axis one unchanged), every other population reversed
// (full-way bounce-back; those never reach the fluid).
__device__ __forceinline__ void wall_node(const float (&f)[Q], float (&fs)[Q], const CellState &ca, const Phys &p,
                                          bool bottom, unsigned lanes, float &twx, float &twz)
{
    wfb_stress(ca, p, lanes, twx, twz);
    const float hx = 0.5f * twx, hz = 0.5f * twz;
#pragma unroll
    for (int a = 0; a < Q; ++a) fs[a] = f[opp_of(a)];
    if (bottom) {
        fs[7] = f[13] + hx;
        fs[14] = f[8] - hx;
        fs[11] = f[18] + hz;
        fs[17] = f[12] - hz;
    } else {
        fs[13] = f[7] + hx;
        fs[8] = f[14] - hx;
        fs[18] = f[11] + hz;
        fs[12] = f[17] - hz;
    }
}

__device__ __forceinline__ void wall_layer(float (&fs)[Q], const CellState &c, const Phys &p, bool bottom,
                                           unsigned lanes, float &twx, float &twz)
{
    twx = 0.f;
    twz = 0.f;
    if (p.wall == WALL_WFB) {
        wfb_stress(c, p, lanes, twx, twz);
        const float hx = 0.5f * twx, hz = 0.5f * twz;
        if (bottom) {
            fs[13] += hx;
            fs[8] -= hx;
            fs[18] += hz;
            fs[12] -= hz;
        } else {
            fs[7] += hx;
            fs[14] -= hx;
            fs[11] += hz;
            fs[17] -= hz;
        }
    } else if (p.wall == WALL_BB) {
        if (bottom) {
            twx = -2.f * (fs[13] - fs[8]);
            twz = -2.f * (fs[18] - fs[12]);
        } else {
            twx = -2.f * (fs[7] - fs[14]);
            twz = -2.f * (fs[11] - fs[17]);
        }
    }
}

// Fused plane statistics of a sampled step. FP64 arithmetic runs at 1/64 of
// the FP32 rate on this GPU, so a per-cell FP64 accumulation made a sampled
// step several times slower than a plain one. The per-cell values are FP32
// anyway; a thread adds its cells in FP32, the warp sums them in FP32 (a
// tree of depth 5), and only the warp sums are converted: the block, plane and
// time sums are FP64. K_ACC = the K_PART sums (rho kept as rho - 1, which is
// exact, so that adding values near 1 loses nothing) and the cell count.
constexpr int K_ACC = K_PART + 1;

__device__ __forceinline__ void stats_zero(float (&v)[K_ACC])
{
#pragma unroll
    for (int k = 0; k < K_ACC; ++k) v[k] = 0.f;
}

// Add one cell (K_STATS plane sums, then the wall sums tau_x, tau_z, |tau|,
// |tau|^2 for a cell of a wall layer). Every rounding is explicit, so the sums
// do not depend on how the compiler contracts them in a given kernel.
__device__ __forceinline__ void stats_cell(float (&v)[K_ACC], float rho, float ux, float uy, float uz, float tx,
                                           float tz, bool wall)
{
    const float dr = __fsub_rn(rho, 1.f);
    v[0] = __fadd_rn(v[0], dr);
    v[1] = __fadd_rn(v[1], ux);
    v[2] = __fadd_rn(v[2], uy);
    v[3] = __fadd_rn(v[3], uz);
    v[4] = __fmaf_rn(ux, ux, v[4]);
    v[5] = __fmaf_rn(uy, uy, v[5]);
    v[6] = __fmaf_rn(uz, uz, v[6]);
    v[7] = __fmaf_rn(ux, uy, v[7]);
    v[8] = __fadd_rn(v[8], __fmul_rn(rho, ux));
    v[9] = __fadd_rn(v[9], __fmul_rn(rho, uy));
    v[10] = __fadd_rn(v[10], __fmul_rn(rho, uz));
    if (wall) {
        const float m2 = __fmaf_rn(tz, tz, __fmul_rn(tx, tx));
        v[11] = __fadd_rn(v[11], tx);
        v[12] = __fadd_rn(v[12], tz);
        v[13] = __fadd_rn(v[13], __fsqrt_rn(m2));
        v[14] = __fadd_rn(v[14], m2);
    }
    v[15] = __fadd_rn(v[15], 1.f);
}

// Sum the 16 accumulators over the warp by reduce-scatter: at the steps with
// lane offsets 16, 8, 4 and 2 each lane keeps the half of its sums selected by
// that bit of its lane index (8, 4, 2, 1 sums) and adds its partner's copy of
// them; a last step adds the pair (lane, lane ^ 1). Lane L then holds the
// warp's sum number L / 2 (16 shuffles and 16 adds per lane instead of 80).
__device__ __forceinline__ float warp_stats_reduce(float (&v)[K_ACC])
{
    static_assert(K_ACC == 16, "the reduce-scatter splits 16 sums over 32 lanes");
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
        }
    }
    return __fadd_rn(v[0], __shfl_xor_sync(0xffffffffu, v[0], 1));
}

// Warp sums of the block's threads (FP32, warp_stats_reduce), added over the
// warps in FP64 in a fixed order; writes the K_PART block sums to out
// (rho as count + sum of rho - 1). All threads of the block must call it.
__device__ __forceinline__ void stats_block_store(float (&v)[K_ACC], double *__restrict__ out)
{
    __shared__ double red[32][K_ACC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float w = warp_stats_reduce(v);
    if (!(lane & 1)) red[warp][lane >> 1] = (double)w;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (threadIdx.x < K_PART) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += red[i][threadIdx.x];
        if (threadIdx.x == 0)
            for (int i = 0; i < nw; ++i) s += red[i][K_PART];
        out[threadIdx.x] = s;
    }
    __syncthreads();   // red[] may be reused by the next call in the same block
}

template <int N>
__device__ __forceinline__ void block_reduce_store(double (&v)[N], double *__restrict__ out)
{
    __shared__ double red[32][N];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) red[warp][k] = v[k];
    }
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (threadIdx.x < N) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();   // red[] may be reused by the next call in the same block
}

// One time step, two lattices: gather from src (streaming + wall reflection),
// collide, wall treatment, store into the own cell of dst. With STATS the
// block also writes its FP64 partial plane sums (K_PART values) to part.
//
// LAY selects the storage scheme: LAY_PULL reads src through the pull map and
// writes the own cell of dst; the AA kinds (src == dst, one array) read
// through the phase map and write the opposite own slot (even) or push to the
// cell the population streams to (odd).
template <typename T, bool STATS, int COLL, int LAY>
__device__ __forceinline__ void cell_step(const T *src, T *dst, const Geom &g, const Phys &p, float *tw_out,
                                          double *part)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const bool valid = x < g.nx;
    if (!STATS && !valid) return;
    const int xc = valid ? x : 0;

    float f[Q], fs[Q];
    if (LAY == LAY_PULL)
        gather<T, MAP_PULL, true>(src, g, p.wall, xc, y, z, f);
    else if (LAY == LAY_AA_EVEN)
        gather<T, MAP_AA0, false>(src, g, p.wall, xc, y, z, f);
    else
        gather<T, MAP_AA1, false>(src, g, p.wall, xc, y, z, f);

    float twx = 0.f, twz = 0.f;
    const bool wall_row = (y == 0) || (y == g.ny - 1);
    // lanes of this warp still running: all of them with STATS (no early
    // exit), otherwise those with x < nx
    unsigned lanes = 0xffffffffu;
    if (!STATS) {
        const int first = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
        const int nv = g.nx - first;
        lanes = nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u);
    }
    CellState c;
    const bool node_row = LAY == LAY_PULL && wall_row && p.wall == WALL_NODE;
    if (node_row) {
        // wall node of the full-way WFB: no collision; tau_w from the first
        // fluid node (the two-lattice source is not written during the step)
        float fa[Q];
        gather<T, MAP_PULL, true>(src, g, p.wall, xc, y == 0 ? 1 : g.ny - 2, z, fa);
        const CellState ca = velocity(moments_of(fa), p);
        c = velocity(moments_of(f), p);
        wall_node(f, fs, ca, p, y == 0, lanes, twx, twz);
        if (valid) {
            float2 *t = reinterpret_cast<float2 *>(tw_out) + ((long long)((y == 0 ? 0 : 1) * g.nz + z) * g.nx + x);
            *t = make_float2(twx, twz);
        }
    } else {
        c = collide<COLL>(f, fs, p, row_smag(p, y, g.ny));
    }
    if (wall_row && !node_row) {
        wall_layer(fs, c, p, y == 0, lanes, twx, twz);
        if (valid) {
            float2 *t = reinterpret_cast<float2 *>(tw_out) + ((long long)((y == 0 ? 0 : 1) * g.nz + z) * g.nx + x);
            *t = make_float2(twx, twz);
        }
    }
    if (valid) {
        if (LAY == LAY_AA_ODD) {
            const Nbr n = neighbours(g, x, z);
            if (y == 0) {
#pragma unroll
                for (int a = 0; a < Q; ++a)
                    st<T>(dst + push_offset<ROW_BOTTOM>(g, p.wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp), fs[a]);
            } else if (y == g.ny - 1) {
#pragma unroll
                for (int a = 0; a < Q; ++a)
                    st<T>(dst + push_offset<ROW_TOP>(g, p.wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp), fs[a]);
            } else {
#pragma unroll
                for (int a = 0; a < Q; ++a)
                    st<T>(dst + push_offset<ROW_INTERIOR>(g, p.wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp), fs[a]);
            }
        } else {
            T *d = dst + ((long long)z * g.ny + y) * g.sx + x;
#pragma unroll
            for (int a = 0; a < Q; ++a) st<T>(d + (LAY == LAY_AA_EVEN ? opp_of(a) : a) * g.plane, fs[a]);
        }
    }
    if (STATS) {
        float v[K_ACC];
        stats_zero(v);
        if (valid) stats_cell(v, c.rho, c.ux, c.uy, c.uz, twx, twz, y == 0 || y == g.ny - 1);
        const long long blk = ((long long)y * g.nz + z) * gridDim.x + blockIdx.x;
        stats_block_store(v, part + blk * K_PART);
    }
}

template <typename T, bool STATS, int COLL = COLL_BGK>
__global__ void __launch_bounds__(128) k_step(const T *__restrict__ src, T *__restrict__ dst, Geom g, Phys p,
                                              float *__restrict__ tw_out, double *__restrict__ part)
{
    cell_step<T, STATS, COLL, LAY_PULL>(src, dst, g, p, tw_out, part);
}

// The one-cell step on the single AA array (LAY_AA_EVEN or LAY_AA_ODD).
template <typename T, bool STATS, int COLL, int LAY>
__global__ void __launch_bounds__(128) k_step_aa(T *f, Geom g, Phys p, float *__restrict__ tw_out,
                                                 double *__restrict__ part)
{
    cell_step<T, STATS, COLL, LAY>(f, f, g, p, tw_out, part);
}

// Sum the block partials of each plane (one block per plane, fixed order, so
// the result is deterministic) into the FP64 accumulators.
static __global__ void k_reduce_planes(const double *__restrict__ part, long long per_plane, int ny,
                                double *__restrict__ acc, double *__restrict__ wacc)
{
    const int y = blockIdx.x;
    double v[K_PART];
#pragma unroll
    for (int k = 0; k < K_PART; ++k) v[k] = 0.0;
    for (long long i = threadIdx.x; i < per_plane; i += blockDim.x) {
        const double *q = part + ((long long)y * per_plane + i) * K_PART;
#pragma unroll
        for (int k = 0; k < K_PART; ++k) v[k] += q[k];
    }
    __shared__ double tot[K_PART];
    block_reduce_store<K_PART>(v, tot);
    __syncthreads();
    if (threadIdx.x < K_STATS) acc[y * K_STATS + threadIdx.x] += tot[threadIdx.x];
    if (threadIdx.x < K_WALL) {
        if (y == 0) wacc[threadIdx.x] += tot[K_STATS + threadIdx.x];
        if (y == ny - 1) wacc[K_WALL + threadIdx.x] += tot[K_STATS + threadIdx.x];
    }
}

// Exports of the current populations f(t) (gathered exactly as the step does):
// moments (FP32), unshifted populations (FP64) and FP64 block partials of
// (sum f - 1, sum e f) for the conservation check.
template <typename T>
__global__ void __launch_bounds__(256) k_export(const T *__restrict__ src, Geom g, Phys p, int map,
                                                float *__restrict__ rho_out, float *__restrict__ u_out,
                                                double *__restrict__ pop_out, double *__restrict__ part)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const bool valid = x < g.nx;
    const int xc = valid ? x : 0;
    float f[Q];
    gather_any<T>(src, g, p.wall, map, xc, y, z, f);
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long cell = ((long long)z * g.ny + y) * g.nx + x;
    if (valid) {
        if (rho_out || u_out) {
            const CellState c = velocity(moments_of(f), p);
            if (rho_out) rho_out[cell] = c.rho;
            if (u_out) {
                u_out[cell] = c.ux;
                u_out[n + cell] = c.uy;
                u_out[2 * n + cell] = c.uz;
            }
        }
        if (pop_out) {
#pragma unroll
            for (int a = 0; a < Q; ++a) pop_out[a * n + cell] = (double)f[a] + w_of(a);
        }
    }
    if (part) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (valid) {
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const double fa = f[a];
                v[0] += fa;
                v[1] += ex_of(a) * fa;
                v[2] += ey_of(a) * fa;
                v[3] += ez_of(a) * fa;
            }
        }
        const long long blk = ((long long)z * g.ny + y) * gridDim.x + blockIdx.x;
        block_reduce_store<4>(v, part + blk * 4);
    }
}

static __global__ void k_reduce_all(const double *__restrict__ part, long long nblk, double *__restrict__ out)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long i = threadIdx.x; i < nblk; i += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += part[i * 4 + k];
    }
    block_reduce_store<4>(v, out);
}

template <typename T> __device__ __forceinline__ void st_d(T *p, double v);
template <> __device__ __forceinline__ void st_d<float>(float *p, double v) { *p = __double2float_rn(v); }
template <> __device__ __forceinline__ void st_d<__half>(__half *p, double v) { *p = __double2half(v); }

// Write f_a(x) (FP64, unshifted, dense) into the slot that the gather of
// (x, a) reads under storage map `map`, so that the next gather returns
// exactly these populations.
template <typename T>
__global__ void k_scatter(const double *__restrict__ in, T *__restrict__ dst, Geom g, int wall, int map)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const Nbr n = neighbours(g, x, z);
    const long long ncell = (long long)g.nx * g.ny * g.nz;
    const long long cell = ((long long)z * g.ny + y) * g.nx + x;
#pragma unroll
    for (int a = 0; a < Q; ++a) st_d<T>(dst + state_offset(g, wall, map, a, x, y, z, n), in[a * ncell + cell] - w_of(a));
}

// SplitMix64 (Steele, Lea & Flood 2014): first output for state s.
__device__ __forceinline__ uint64_t splitmix64(uint64_t s)
{
    uint64_t z = s + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Seeded channel field f = f^eq(1, u0), u0 = mean profile + uniform noise, in
// FP64 without contraction, then rounded once to the storage precision and
// written to the slots the next gather reads.
template <typename T>
__global__ void k_init_channel(T *__restrict__ dst, Geom g, int wall, int map, const double *__restrict__ umean,
                               double amp, uint64_t seed)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const unsigned long long cell = ((unsigned long long)z * g.ny + y) * g.nx + x;
    double u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double r = (double)(splitmix64(seed ^ (cell * 3ULL + (unsigned long long)c)) >> 11) *
                         (1.0 / 9007199254740992.0);
        const double noise = __dmul_rn(__dsub_rn(__dmul_rn(2.0, r), 1.0), amp);
        u[c] = __dadd_rn(c == 0 ? umean[y] : 0.0, noise);
    }
    const double uu = __dadd_rn(__dadd_rn(__dmul_rn(u[0], u[0]), __dmul_rn(u[1], u[1])), __dmul_rn(u[2], u[2]));
    const Nbr n = neighbours(g, x, z);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const double eu = __dadd_rn(__dadd_rn(__dmul_rn((double)ex_of(a), u[0]), __dmul_rn((double)ey_of(a), u[1])),
                                    __dmul_rn((double)ez_of(a), u[2]));
        const double poly = __dsub_rn(__dadd_rn(__dadd_rn(1.0, __dmul_rn(3.0, eu)), __dmul_rn(__dmul_rn(4.5, eu), eu)),
                                      __dmul_rn(1.5, uu));
        const double feq = __dmul_rn(__dmul_rn(w_of(a), 1.0), poly);
        st_d<T>(dst + state_offset(g, wall, map, a, x, y, z, n), __dsub_rn(feq, w_of(a)));
    }
}

}  // namespace lbm
