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

// coherent 2-wide loads (see pull_nc in lbm_device.cuh)
template <typename T> __device__ __forceinline__ float2 ldc2(const T *p);
template <> __device__ __forceinline__ float2 ldc2<float>(const float *p)
{
    return __ldca(reinterpret_cast<const float2 *>(p));
}
template <> __device__ __forceinline__ float2 ldc2<__half>(const __half *p)
{
    return __half22float2(__ldca(reinterpret_cast<const __half2 *>(p)));
}

template <typename T> __device__ __forceinline__ void st2(T *p, float2 v);
template <> __device__ __forceinline__ void st2<float>(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
template <> __device__ __forceinline__ void st2<__half>(__half *p, float2 v)
{
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x, v.y);
}

// Values of one source row for the pair (x0, x0 + 1) shifted by SH: the cells
// read x0 - SH and x0 + 1 - SH. `row` points at the start of the source row.
template <typename T, int SH, bool NC = true>
__device__ __forceinline__ float2 row_pair(const T *row, int x0, int nx, int lane)
{
    const float2 v = NC ? ld2<T>(row + x0) : ldc2<T>(row + x0);
    if (SH == 0) return v;
    if (SH == 1) {
        float l = __shfl_up_sync(0xffffffffu, v.y, 1);
        if (lane == 0 || x0 == 0) l = ldx<T, NC>(row + (x0 == 0 ? nx - 1 : x0 - 1));
        return make_float2(l, v.x);
    }
    float r = __shfl_down_sync(0xffffffffu, v.x, 1);
    if (lane == 31 || x0 + 2 >= nx) r = ldx<T, NC>(row + (x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2));
    return make_float2(v.y, r);
}

// Gather of the 19 populations of the pair (streaming with the wall
// reflection of lbm_device.cuh's src_offset, two cells at a time). LAY_PULL
// reads the pull map through the read-only path; LAY_AA_ODD reads the same
// positions in the opposite slots (map MAP_AA1); LAY_AA_EVEN reads the own
// slots (map MAP_AA0).
template <typename T, int ROW, int LAY = LAY_PULL>
__device__ __forceinline__ void gather_pair(const T *src, const Geom &g, int wall, int x0, int y, int z, int zm,
                                            int zp, int lane, float2 (&f)[Q])
{
    constexpr bool NC = LAY == LAY_PULL && pull_nc<T>;
    if constexpr (LAY == LAY_AA_EVEN) {
        const T *own = src + ((long long)z * g.ny + y) * g.sx + x0;
#pragma unroll
        for (int a = 0; a < Q; ++a) f[a] = ldc2<T>(own + a * g.plane);
    } else {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int ex = ex_of(a), ey = ey_of(a), ez = ez_of(a);
            const bool crosses = (ROW == ROW_BOTTOM && ey == 1) || (ROW == ROW_TOP && ey == -1);
            const int zs = ez == 1 ? zm : (ez == -1 ? zp : z);
            const int sa = LAY == LAY_AA_ODD ? opp_of(a) : a;
            if (!crosses) {
                const T *row = src + (long long)sa * g.plane + ((long long)zs * g.ny + (y - ey)) * g.sx;
                if (ex == 1)
                    f[a] = row_pair<T, 1, NC>(row, x0, g.nx, lane);
                else if (ex == -1)
                    f[a] = row_pair<T, -1, NC>(row, x0, g.nx, lane);
                else
                    f[a] = row_pair<T, 0, NC>(row, x0, g.nx, lane);
            } else if (bb_map(wall)) {
                const int sb = LAY == LAY_AA_ODD ? a : opp_of(a);
                const T *row = src + (long long)sb * g.plane + ((long long)z * g.ny + y) * g.sx;
                f[a] = row_pair<T, 0, NC>(row, x0, g.nx, lane);
            } else {
                const int sm = LAY == LAY_AA_ODD ? opp_of(mirror_of(a)) : mirror_of(a);
                const T *row = src + (long long)sm * g.plane + ((long long)zs * g.ny + y) * g.sx;
                if (ex == 1)
                    f[a] = row_pair<T, 1, NC>(row, x0, g.nx, lane);
                else if (ex == -1)
                    f[a] = row_pair<T, -1, NC>(row, x0, g.nx, lane);
                else
                    f[a] = row_pair<T, 0, NC>(row, x0, g.nx, lane);
            }
        }
    }
}

// Store of the pair's values into one row shifted by SH (cell x goes to
// x + SH, periodic): the counterpart of row_pair for the AA push. Interior
// lanes store one aligned pair built with a warp shuffle; the first and last
// lane of the warp (and the row ends) store the element that crosses into the
// neighbouring warp's pair alone, so every element is written exactly once.
// All 32 lanes must call it (the shuffle); lanes past the row end store nothing.
template <typename T, int SH>
__device__ __forceinline__ void push_row(T *row, int x0, int nx, int lane, bool valid, float2 v)
{
    if (SH == 0) {
        if (valid) st2<T>(row + x0, v);
        return;
    }
    if (SH == 1) {   // cells x0, x0 + 1 -> x0 + 1, x0 + 2
        const float l = __shfl_up_sync(0xffffffffu, v.y, 1);
        if (!valid) return;
        if (lane == 0 || x0 == 0)
            st<T>(row + x0 + 1, v.x);
        else
            st2<T>(row + x0, make_float2(l, v.x));
        if (lane == 31 || x0 + 2 >= nx) st<T>(row + (x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2), v.y);
        return;
    }
    // SH == -1: cells x0, x0 + 1 -> x0 - 1, x0
    const float r = __shfl_down_sync(0xffffffffu, v.x, 1);
    if (!valid) return;
    if (lane == 31 || x0 + 2 >= nx)
        st<T>(row + x0, v.y);
    else
        st2<T>(row + x0, make_float2(v.y, r));
    if (lane == 0 || x0 == 0) st<T>(row + (x0 == 0 ? nx - 1 : x0 - 1), v.x);
}

// AA odd step store of the pair: f*_a to the slot and cell of push_offset
// (lbm_device.cuh), two cells at a time.
template <typename T, int ROW>
__device__ __forceinline__ void push_pair(T *dst, const Geom &g, int wall, int x0, int y, int z, int zm, int zp,
                                          int lane, bool valid, const float2 (&f)[Q])
{
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int ex = ex_of(a), ey = ey_of(a), ez = ez_of(a);
        const bool crosses = (ROW == ROW_BOTTOM && ey == -1) || (ROW == ROW_TOP && ey == 1);
        const int zt = ez == 1 ? zp : (ez == -1 ? zm : z);
        if (!crosses) {
            T *row = dst + (long long)a * g.plane + ((long long)zt * g.ny + (y + ey)) * g.sx;
            if (ex == 1)
                push_row<T, 1>(row, x0, g.nx, lane, valid, f[a]);
            else if (ex == -1)
                push_row<T, -1>(row, x0, g.nx, lane, valid, f[a]);
            else
                push_row<T, 0>(row, x0, g.nx, lane, valid, f[a]);
        } else if (bb_map(wall)) {
            T *row = dst + (long long)opp_of(a) * g.plane + ((long long)z * g.ny + y) * g.sx;
            push_row<T, 0>(row, x0, g.nx, lane, valid, f[a]);
        } else {
            T *row = dst + (long long)mirror_of(a) * g.plane + ((long long)zt * g.ny + y) * g.sx;
            if (ex == 1)
                push_row<T, 1>(row, x0, g.nx, lane, valid, f[a]);
            else if (ex == -1)
                push_row<T, -1>(row, x0, g.nx, lane, valid, f[a]);
            else
                push_row<T, 0>(row, x0, g.nx, lane, valid, f[a]);
        }
    }
}

struct PairState {
    float2 rho, ux, uy, uz;
};

// wall_layer() of lbm_kernels.cuh for a packed pair of first-layer cells:
// the wall stress lane by lane, the correction of the four wall-bound
// populations with packed adds (the same single roundings as the scalar form).
__device__ __forceinline__ void wall_layer_pair(float2 (&f)[Q], const PairState &c, const Phys &p, bool bottom,
                                                float2 &twx, float2 &twz)
{
    twx = make_float2(0.f, 0.f);
    twz = make_float2(0.f, 0.f);
    if (p.wall == WALL_WFB) {
        const CellState ca{c.rho.x, c.ux.x, c.uy.x, c.uz.x}, cb{c.rho.y, c.ux.y, c.uy.y, c.uz.y};
        wfb_stress(ca, p, 0xffffffffu, twx.x, twz.x);
        wfb_stress(cb, p, 0xffffffffu, twx.y, twz.y);
        const float2 hx = make_float2(0.5f * twx.x, 0.5f * twx.y), hz = make_float2(0.5f * twz.x, 0.5f * twz.y);
        const float2 mhx = make_float2(-hx.x, -hx.y), mhz = make_float2(-hz.x, -hz.y);
        if (bottom) {
            f[13] = __fadd2_rn(f[13], hx);
            f[8] = __fadd2_rn(f[8], mhx);
            f[18] = __fadd2_rn(f[18], hz);
            f[12] = __fadd2_rn(f[12], mhz);
        } else {
            f[7] = __fadd2_rn(f[7], hx);
            f[14] = __fadd2_rn(f[14], mhx);
            f[11] = __fadd2_rn(f[11], hz);
            f[17] = __fadd2_rn(f[17], mhz);
        }
    } else if (p.wall == WALL_BB) {
        const int a = bottom ? 13 : 7, b = bottom ? 8 : 14, cz = bottom ? 18 : 11, dz = bottom ? 12 : 17;
        twx = make_float2(-2.f * (f[a].x - f[b].x), -2.f * (f[a].y - f[b].y));
        twz = make_float2(-2.f * (f[cz].x - f[dz].x), -2.f * (f[cz].y - f[dz].y));
    }
}

// MRT of d'Humieres et al. (2002), written as the BGK update plus the
// corrections of the ghost moments whose rates differ from omega = 1/tau_eff:
// the energy e (s_e), its square eps (s_eps), the energy fluxes q (s_q) and
// the third-order moments m (s_m); the stress and fourth-order pi moments
// relax with omega as in BGK. With the orthogonal basis rows phi_i, moving
// moment i from the BGK change -omega m_i^neq + (1 - omega/2) g_i to the MRT
// change -s_i m_i^neq + (1 - s_i/2) g_i (g_i the moment of the Guo force term)
// adds C_i phi_i to the populations, C_i = (omega - s_i)(m_i^neq + g_i/2)/|phi_i|^2.
// On the pair half sums hs_k and half differences hd_k of the deviations,
// with A and D the sums of hs over the axis and the diagonal pairs and Guo's
// rho u = j + F/2, the brackets m_i^neq + g_i/2 are
//   e:    19 (2 D - f_0 - rho u.u + u.F)
//   eps:  9 f_0 - 14 A - 4 D + 11/2 (rho u.u - u.F)
//   q_x:  10/3 (sum of hd over the four diagonal pairs with e_x != 0, signed
//         by e_x of the pair's first member, - 2 hd_x)  (the equilibrium and
//         force parts cancel; q_y, q_z alike)
//   m_x:  2 (hd_(1,1,0) - hd_(1,0,1) + hd_(1,-1,0) - hd_(1,0,-1))  (m_y, m_z alike)
// and the change of a pair's half sum is phi_e C_e + phi_eps C_eps of its
// class (axis -11, -4; diagonal 8, 1; rest -30, 12), of its half difference
// the sum of phi_i C_i over q and m for its first member.
struct MrtPair {
    float2 ea, ed, er;     // half-sum change of an axis / diagonal pair, change of the rest population
    float2 cq[3];          // C of q_x, q_y, q_z (axis pairs: half difference -4 C_q)
    float2 od[6];          // half-difference change of the diagonal pairs 3 .. 8
};

// s, d: the half sums and differences hs, hd of the pairs, or with PS their
// doubles (the pair sums and differences): the factors 2 then go exactly into
// the constants, and the bits are those of the half-sum form.
template <bool PS>
__device__ __forceinline__ MrtPair mrt_ghost_pair(const float2 (&s)[9], const float2 (&d)[9], float2 f0,
                                                  float2 rusq, float2 uF, float2 omega, const Phys &p)
{
    MrtPair m;
    const float2 A = add2(add2(s[0], s[1]), s[2]);                                        // A (PS: 2 A)
    const float2 D = add2(add2(add2(s[3], s[4]), add2(s[5], s[6])), add2(s[7], s[8]));   // D (PS: 2 D)
    const float2 D2 = PS ? D : add2(D, D);
    const float2 ke = fma2(omega, bc(p.mrt_a[MRT_E]), bc(p.mrt_b[MRT_E]));
    const float2 kp = fma2(omega, bc(p.mrt_a[MRT_EPS]), bc(p.mrt_b[MRT_EPS]));
    // with PS, C_q and C_m take half of their brackets' doubled partial sums
    const float hq = PS ? 0.5f : 1.f;
    const float2 kq = fma2(omega, bc(hq * p.mrt_a[MRT_Q]), bc(hq * p.mrt_b[MRT_Q]));
    const float2 km = fma2(omega, bc(hq * p.mrt_a[MRT_M]), bc(hq * p.mrt_b[MRT_M]));
    const float2 du = sub2(rusq, uF);
    const float2 ce = mul2(ke, sub2(sub2(D2, f0), du));
    const float2 cp = mul2(kp, fma2(bc(9.f), f0, fma2(bc(PS ? -7.f : -14.f), A,
                                                      fma2(bc(PS ? -2.f : -4.f), D, mul2(bc(5.5f), du)))));
    m.ea = fma2(bc(-11.f), ce, mul2(bc(-4.f), cp));
    m.ed = fma2(bc(8.f), ce, cp);
    m.er = fma2(bc(-30.f), ce, mul2(bc(12.f), cp));
    // pairs 3..8: first members (1,1,0), (1,0,1), (0,1,1), (1,-1,0), (1,0,-1),
    // (0,1,-1); the q and m brackets share their partial sums
    const float2 sxa = add2(d[3], d[6]), sxb = add2(d[4], d[7]);   // q_x = sxa + sxb - 2 hd_x, m_x = sxa - sxb
    const float2 sya = add2(d[5], d[8]), syb = sub2(d[3], d[6]);   // q_y = sya + syb - 2 hd_y, m_y = sya - syb
    const float2 sza = sub2(d[4], d[7]), szb = sub2(d[5], d[8]);   // q_z = sza + szb - 2 hd_z, m_z = sza - szb
    m.cq[0] = mul2(kq, fma2(bc(-2.f), d[0], add2(sxa, sxb)));
    m.cq[1] = mul2(kq, fma2(bc(-2.f), d[1], add2(sya, syb)));
    m.cq[2] = mul2(kq, fma2(bc(-2.f), d[2], add2(sza, szb)));
    const float2 cmx = mul2(km, sub2(sxa, sxb)), cmy = mul2(km, sub2(sya, syb)), cmz = mul2(km, sub2(sza, szb));
    // pair 3 / 6: (Cq_x + Cm_x) +/- (Cq_y - Cm_y); 4 / 7: (Cq_x - Cm_x) +/- (Cq_z + Cm_z);
    // 5 / 8: (Cq_y + Cm_y) +/- (Cq_z - Cm_z)
    const float2 t36a = add2(m.cq[0], cmx), t36b = sub2(m.cq[1], cmy);
    const float2 t47a = sub2(m.cq[0], cmx), t47b = add2(m.cq[2], cmz);
    const float2 t58a = add2(m.cq[1], cmy), t58b = sub2(m.cq[2], cmz);
    m.od[0] = add2(t36a, t36b);
    m.od[3] = sub2(t36a, t36b);
    m.od[1] = add2(t47a, t47b);
    m.od[4] = sub2(t47a, t47b);
    m.od[2] = add2(t58a, t58b);
    m.od[5] = sub2(t58a, t58b);
    return m;
}

// dd + the half-difference change of pair k from the q and m corrections.
__device__ __forceinline__ float2 mrt_odd_add(const MrtPair &m, int k, float2 dd)
{
    return k < 3 ? fma2(bc(-4.f), m.cq[k], dd) : add2(dd, m.od[k - 3]);
}

// collide() of lbm_kernels.cuh for two cells (in place: f becomes f*),
// organised around the opposite pairs k = 0..8 (directions 2k+1, 2k+2):
// s_k = f_a + f_b and d_k = f_a - f_b carry all moments the update needs,
//   drho = f_0 + sum s,  j = sum e_k d_k,  Pi_ab = sum e_k,a e_k,b s_k,
// and the update of the pair is  delta_a = de + dd,  delta_b = de - dd  with
//   de = omega (w (S0 + 9/2 rho (e.u)^2) - s / 2) - 3 w gk u.F + 9 w gk (e.u)(e.F)
//   dd = omega (3 w rho (e.u) - d / 2) + 3 w gk (e.F),
// evaluated with the weights scaled by 36 as collide() states.
// Only the half sums and differences s/2, d/2 are kept through the collision
// (the new populations are their sum and difference), which keeps 18 fewer
// values live.
//
// PS selects how the pairs enter: the half sums and differences hs = s/2,
// hd = d/2 (PS false), or s and d themselves (PS true), every later use taking
// the 1/2 into a power-of-two constant or a doubling it would otherwise need.
// Halving commutes with rounding, so both forms compute the same bits; PS
// saves 28 packed operations per pair, and each kernel takes the form that
// measured faster with its register budget: PS_DEFAULT for the two-lattice
// steps (FP32 BGK: +1.7% on c4; FP16 MRT: +2.1% on c3; FP32 MRT -0.3%, FP16
// BGK two-cell not timed faster), the half sums in the in-place AA pair steps
// (FP32 c3: 42.3 against 41.2 GLUPS), and per step kind in the four-cell
// kernels (quad_half). The update stores the new half values hs' = hs + de,
// hd' = hd + dd in s and d.
template <int COLL, bool EXACT_W>
constexpr bool PS_DEFAULT = EXACT_W != (COLL == COLL_MRT);

template <int COLL = COLL_BGK, bool EXACT_W = false, bool PS = PS_DEFAULT<COLL, EXACT_W>>
__device__ __forceinline__ PairState collide_pair(float2 (&f)[Q], const Phys &p, float smag)
{
    PairState c;
    float2 s[9], d[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        s[k] = add2(f[2 * k + 1], f[2 * k + 2]);
        d[k] = sub2(f[2 * k + 1], f[2 * k + 2]);
        if constexpr (!PS) {
            s[k] = mul2(bc(0.5f), s[k]);
            d[k] = mul2(bc(0.5f), d[k]);
        }
    }
    // without PS, doubling by addition (exact) keeps constants out of the packed ops
    const float2 ss = add2(add2(add2(s[0], s[1]), add2(s[2], s[3])),
                           add2(add2(s[4], s[5]), add2(add2(s[6], s[7]), s[8])));
    const float2 drho = add2(PS ? ss : add2(ss, ss), f[0]);
    float2 jx = add2(add2(d[0], d[3]), add2(add2(d[4], d[6]), d[7]));
    float2 jy = add2(add2(d[1], d[3]), add2(sub2(d[5], d[6]), d[8]));
    float2 jz = sub2(add2(add2(d[2], d[4]), d[5]), add2(d[7], d[8]));
    float2 pxx = add2(add2(s[0], s[3]), add2(add2(s[4], s[6]), s[7]));
    float2 pyy = add2(add2(s[1], s[3]), add2(add2(s[5], s[6]), s[8]));
    float2 pzz = add2(add2(s[2], s[4]), add2(add2(s[5], s[7]), s[8]));
    float2 pxy = sub2(s[3], s[6]);
    float2 pxz = sub2(s[4], s[7]);
    float2 pyz = sub2(s[5], s[8]);
    if constexpr (!PS) {
        jx = add2(jx, jx);
        jy = add2(jy, jy);
        jz = add2(jz, jz);
        pxx = add2(pxx, pxx);
        pyy = add2(pyy, pyy);
        pzz = add2(pzz, pzz);
        pxy = add2(pxy, pxy);
        pxz = add2(pxz, pxz);
        pyz = add2(pyz, pyz);
    }

    c.rho = add2(bc(1.f), drho);
    const float2 idev = make_float2(-drho.x / c.rho.x, -drho.y / c.rho.y);   // 1/rho - 1
    if constexpr (EXACT_W) {
        // u = j + (j (1/rho - 1) + F/2 / rho), as velocity() in lbm_kernels.cuh
        c.ux = add2(jx, fma2(jx, idev, fma2(bc(p.hF[0]), idev, bc(p.hF[0]))));
        c.uy = add2(jy, fma2(jy, idev, fma2(bc(p.hF[1]), idev, bc(p.hF[1]))));
        c.uz = add2(jz, fma2(jz, idev, fma2(bc(p.hF[2]), idev, bc(p.hF[2]))));
    } else {
        // u = (j + F/2)(1 + (1/rho - 1)); the momentum projection of the
        // update below makes its momentum exact whatever the rounding of u
        const float2 jfx = add2(jx, bc(p.hF[0])), jfy = add2(jy, bc(p.hF[1])), jfz = add2(jz, bc(p.hF[2]));
        c.ux = fma2(jfx, idev, jfx);
        c.uy = fma2(jfy, idev, jfy);
        c.uz = fma2(jfz, idev, jfz);
    }
    const float2 rho = c.rho, ux = c.ux, uy = c.uy, uz = c.uz;

    const float2 cd = mul2(drho, bc(1.f / 3.f));
    const float2 rux = mul2(rho, ux), ruy = mul2(rho, uy), ruz = mul2(rho, uz);
    pxx = sub2(pxx, fma2(rux, ux, cd));
    pyy = sub2(pyy, fma2(ruy, uy, cd));
    pzz = sub2(pzz, fma2(ruz, uz, cd));
    pxy = sub2(pxy, mul2(rux, uy));
    pxz = sub2(pxz, mul2(rux, uz));
    pyz = sub2(pyz, mul2(ruy, uz));
    const float2 qo = fma2(pxy, pxy, fma2(pxz, pxz, mul2(pyz, pyz)));
    const float2 q2 = add2(add2(qo, qo), fma2(pxx, pxx, fma2(pyy, pyy, mul2(pzz, pzz))));
    // omega = 1 / tau_eff = 2 / (tau0 + sqrt(tau0^2 + smag |Pi_neq| / rho)),
    // 1/rho = 1 + idev (a sum of positive terms: no cancellation); explicit
    // roundings, so every kernel that inlines this computes the same bits
    float2 omega;
    {
        const float t02 = p.t02;
        const float cqx = __fmul_rn(__fmul_rn(smag, sqrtf(q2.x)), __fadd_rn(1.f, idev.x));
        const float cqy = __fmul_rn(__fmul_rn(smag, sqrtf(q2.y)), __fadd_rn(1.f, idev.y));
        omega = make_float2(2.f / __fadd_rn(p.tau0, sqrtf(__fadd_rn(t02, cqx))),
                            2.f / __fadd_rn(p.tau0, sqrtf(__fadd_rn(t02, cqy))));
    }
    const float2 usq = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
    const float2 uF = fma2(ux, bc(p.Fx), fma2(uy, bc(p.Fy), mul2(uz, bc(p.Fz))));
    // MRT: corrections of the ghost groups (zero cost for BGK)
    MrtPair mg;
    if constexpr (COLL == COLL_MRT) mg = mrt_ghost_pair<PS>(s, d, f[0], mul2(rho, usq), uF, omega, p);
    if constexpr (EXACT_W) {
    // BGK with the weights scaled by 36 (36 w = 12 rest, 2 axis, 1 diagonal:
    // exact) and 1/36 folded into the rate, o36 = omega / 36. Per pair, with
    // W = 36 w, the non-equilibrium difference is formed before the rate
    // multiplies it, and the odd part uses rho (e.u) = e.(j + F/2) directly:
    //   ne = 36 (feq_even - hs) = W (S0 + 9/2 rho (e.u)^2) - 36 hs   (36 hs = 18 s)
    //   nd = 36 (feq_odd - hd)  = 3 W (e.j) + 3 W (e.F) / 2 - 36 hd   (36 hd = 18 d)
    //   de = o36 ne + W gk (9 (e.u)(e.F) - 3 u.F) / 36,  dd = o36 nd + W gk 3 (e.F) / 36
    // and the rest population its own update 36 (feq_0 - f_0) = 12 S0 - 36 f_0.
    // The axis pairs take the momentum residual F/2 - sum e dd (zero in exact
    // arithmetic): it now holds only the roundings of small non-equilibrium
    // terms, not the rounding of the weights or of the rate times the
    // equilibrium, which halves the update's FP32 error against an FP64
    // reference while momentum stays exact up to the final store; the mass
    // change is zero up to unbiased roundings.
    const float2 gk = fma2(bc(-0.5f), omega, bc(1.f));
    const float2 o36 = mul2(omega, bc(1.f / 36.f));
    const float2 S0 = fma2(bc(-1.5f), mul2(rho, usq), drho);
    const float2 r45 = mul2(bc(4.5f), rho);
    const float2 r45a = add2(r45, r45), S0a = add2(S0, S0);               // W = 2 (exact doublings)
    const float2 g9 = mul2(bc(0.25f), gk);                                 // 9 gk / 36
    const float2 g3 = mul2(bc(1.f / 12.f), gk);                            // 3 gk / 36
    const float2 mgu = mul2(mul2(bc(-1.f / 12.f), gk), uF);                // -3 gk u.F / 36
    const float2 mgua = add2(mgu, mgu);

    // e.u and e.j of the odd member of each pair (directions 1, 3, ..., 17)
    const float2 eus[9] = {ux, uy, uz, add2(ux, uy), add2(ux, uz), add2(uy, uz),
                           sub2(ux, uy), sub2(ux, uz), sub2(uy, uz)};
    const float2 ejs[9] = {jx, jy, jz, add2(jx, jy), add2(jx, jz), add2(jy, jz),
                           sub2(jx, jy), sub2(jx, jz), sub2(jy, jz)};
    float2 d0 = fma2(o36, fma2(bc(-36.f), f[0], mul2(bc(12.f), S0)), mul2(bc(12.f), mgu));
    if constexpr (COLL == COLL_MRT) d0 = add2(d0, mg.er);
    f[0] = add2(f[0], d0);
    float2 mx, my, mz;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int a = 2 * k + 1;
        const bool axis = k < 3;
        const float W3 = axis ? 6.f : 3.f;    // 3 W
        const float2 eu = eus[k];
        const float2 WeF = bc(p.WeF[k]);      // 36 w (e.F)
        const float2 ne = fma2(mul2(axis ? r45a : r45, eu), eu, fma2(bc(PS ? -18.f : -36.f), s[k], axis ? S0a : S0));
        const float2 nd = fma2(bc(W3), ejs[k], fma2(bc(PS ? -18.f : -36.f), d[k], mul2(bc(1.5f), WeF)));
        float2 de = fma2(o36, ne, fma2(mul2(g9, WeF), eu, axis ? mgua : mgu));
        float2 dd = fma2(o36, nd, mul2(g3, WeF));
        if constexpr (COLL == COLL_MRT) {
            de = add2(de, axis ? mg.ea : mg.ed);
            dd = mrt_odd_add(mg, k, dd);
        }
        if (k == 0) mx = dd;
        else if (ex_of(a)) mx = ex_of(a) > 0 ? add2(mx, dd) : sub2(mx, dd);
        if (k == 1) my = dd;
        else if (k > 1 && ey_of(a)) my = ey_of(a) > 0 ? add2(my, dd) : sub2(my, dd);
        if (k == 2) mz = dd;
        else if (k > 2 && ez_of(a)) mz = ez_of(a) > 0 ? add2(mz, dd) : sub2(mz, dd);
        s[k] = PS ? fma2(bc(0.5f), s[k], de) : add2(s[k], de);
        d[k] = PS ? fma2(bc(0.5f), d[k], dd) : add2(d[k], dd);
    }
    d[0] = add2(d[0], sub2(bc(p.hF[0]), mx));
    d[1] = add2(d[1], sub2(bc(p.hF[1]), my));
    d[2] = add2(d[2], sub2(bc(p.hF[2]), mz));
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        f[2 * k + 1] = add2(s[k], d[k]);
        f[2 * k + 2] = sub2(s[k], d[k]);
    }
    return c;
    } else {
    // BGK with rounded weights folded into the rate; the momentum and mass
    // of the update are then corrected on the axis pairs and the rest
    // population (the storage form of FP16, whose rounding dominates)
    const float2 gk = fma2(bc(-0.5f), omega, bc(1.f));
    const float2 nw = mul2(bc(PS ? -0.5f : -1.f), omega);                  // -omega (PS: -omega / 2)
    const float2 S0 = fma2(bc(-1.5f), mul2(rho, usq), drho);
    const float2 oS = sub2(mul2(omega, S0), mul2(mul2(bc(3.f), gk), uF));  // omega S0 - 3 gk u.F
    const float2 oR45 = mul2(omega, mul2(bc(4.5f), rho));                // 4.5 omega rho
    const float2 oR3 = mul2(omega, mul2(bc(3.f), rho));                  // 3 omega rho
    const float2 g9 = mul2(bc(9.f), gk), g3 = mul2(bc(3.f), gk);
    // class constants (w = 1/18 axis, 1/36 diagonal)
    const float2 Ca = mul2(bc(1.f / 18.f), oS), Cd = mul2(bc(1.f / 36.f), oS);
    const float2 Aa = mul2(bc(1.f / 18.f), oR45), Ad = mul2(bc(1.f / 36.f), oR45);
    const float2 Da = mul2(bc(1.f / 18.f), oR3), Dd = mul2(bc(1.f / 36.f), oR3);

    // e.u of the odd member of each pair (directions 1, 3, 5, 7, 9, 11, 13, 15, 17)
    const float2 eus[9] = {ux, uy, uz, add2(ux, uy), add2(ux, uz), add2(uy, uz),
                           sub2(ux, uy), sub2(ux, uz), sub2(uy, uz)};
    float2 mass, mx, my, mz;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int a = 2 * k + 1;
        const bool axis = k < 3;
        const float2 eu = eus[k];
        const float2 eF = bc(p.weF[k]);   // w e.F
        const float2 Gk = mul2(g9, eF), Hk = mul2(g3, eF);
        // -omega hs (= (-omega / 2) s exactly)
        float2 de = fma2(nw, s[k], fma2(fma2(axis ? Aa : Ad, eu, Gk), eu, axis ? Ca : Cd));
        float2 dd = fma2(nw, d[k], fma2(axis ? Da : Dd, eu, Hk));
        if constexpr (COLL == COLL_MRT) {
            de = add2(de, axis ? mg.ea : mg.ed);
            dd = mrt_odd_add(mg, k, dd);
        }
        // accumulate sum de and sum e dd (first terms: pairs 0, 1, 2 are the axes)
        mass = k == 0 ? de : add2(mass, de);
        if (k == 0) mx = dd;
        else if (ex_of(a)) mx = ex_of(a) > 0 ? add2(mx, dd) : sub2(mx, dd);
        if (k == 1) my = dd;
        else if (k > 1 && ey_of(a)) my = ey_of(a) > 0 ? add2(my, dd) : sub2(my, dd);
        if (k == 2) mz = dd;
        else if (k > 2 && ez_of(a)) mz = ez_of(a) > 0 ? add2(mz, dd) : sub2(mz, dd);
        // the pair's new half sum and half difference (delta_a = de + dd, delta_b = de - dd)
        s[k] = PS ? fma2(bc(0.5f), s[k], de) : add2(s[k], de);
        d[k] = PS ? fma2(bc(0.5f), d[k], dd) : add2(d[k], dd);
    }
    // exact momentum F and mass 0 of the update (see collide()): the axis pairs
    // take the momentum residual, the rest population the mass residual
    d[0] = add2(d[0], sub2(bc(p.hF[0]), mx));
    d[1] = add2(d[1], sub2(bc(p.hF[1]), my));
    d[2] = add2(d[2], sub2(bc(p.hF[2]), mz));
    f[0] = sub2(f[0], add2(mass, mass));
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        f[2 * k + 1] = add2(s[k], d[k]);
        f[2 * k + 2] = sub2(s[k], d[k]);
    }
    return c;
    }
}

// One tile: the x-pairs xb * blockDim.x + threadIdx.x of row (y, z), i.e.
// cells [2 xb blockDim.x, 2 (xb + 1) blockDim.x). With STATS the block writes
// its FP64 partial sums to part_blk[0..K_PART).
//
// LAY selects the storage scheme (LAY_PULL: src and dst are the two lattices;
// LAY_AA_EVEN / LAY_AA_ODD: src == dst, the single AA array).
// Row sets a tile instantiation serves: any row, the interior rows only (no
// wall-layer code in the instantiation), or the two wall rows only.
enum { ROWS_ALL = 0, ROWS_INTERIOR = 1, ROWS_WALL = 2 };

template <typename T, bool STATS, int COLL = COLL_BGK, int LAY = LAY_PULL, int ROWS = ROWS_ALL>
__device__ __forceinline__ void pair_tile(const T *src, T *dst, const Geom &g, const Phys &p,
                                          float *__restrict__ tw_out, double *__restrict__ part_blk, int xb, int y,
                                          int z)
{
    const int lane = threadIdx.x & 31;
    const int x0 = 2 * (xb * blockDim.x + threadIdx.x);
    const bool valid = x0 < g.nx;
    const int xl = valid ? x0 : g.nx - 2;   // lanes past the row end read in bounds and store nothing
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;

    // wall node of the full-way WFB (two-lattice layout only): no collision;
    // tau_w from the first fluid node, whose state is gathered first so that
    // its populations are dead before the node's own are loaded
    const bool node_row =
        ROWS != ROWS_INTERIOR && LAY == LAY_PULL && p.wall == WALL_NODE && (y == 0 || y == g.ny - 1);
    CellState ca0{}, ca1{};
    if (node_row) {
        float2 fa[Q];
        gather_pair<T, ROW_INTERIOR, LAY>(src, g, p.wall, xl, y == 0 ? 1 : g.ny - 2, z, zm, zp, lane, fa);
        float a0[Q], a1[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            a0[a] = fa[a].x;
            a1[a] = fa[a].y;
        }
        ca0 = velocity(moments_of(a0), p);
        ca1 = velocity(moments_of(a1), p);
    }

    float2 f[Q];
    if (ROWS != ROWS_INTERIOR && y == 0)
        gather_pair<T, ROW_BOTTOM, LAY>(src, g, p.wall, xl, y, z, zm, zp, lane, f);
    else if (ROWS != ROWS_INTERIOR && y == g.ny - 1)
        gather_pair<T, ROW_TOP, LAY>(src, g, p.wall, xl, y, z, zm, zp, lane, f);
    else
        gather_pair<T, ROW_INTERIOR, LAY>(src, g, p.wall, xl, y, z, zm, zp, lane, f);

    float2 twx = bc(0.f), twz = bc(0.f);
    PairState c;
    if (node_row) {
        float fa[Q], fb[Q], oa[Q], ob[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            fa[a] = f[a].x;
            fb[a] = f[a].y;
        }
        const CellState sa = velocity(moments_of(fa), p), sb = velocity(moments_of(fb), p);
        c.rho = make_float2(sa.rho, sb.rho);
        c.ux = make_float2(sa.ux, sb.ux);
        c.uy = make_float2(sa.uy, sb.uy);
        c.uz = make_float2(sa.uz, sb.uz);
        wall_node(fa, oa, ca0, p, y == 0, 0xffffffffu, twx.x, twz.x);
        wall_node(fb, ob, ca1, p, y == 0, 0xffffffffu, twx.y, twz.y);
#pragma unroll
        for (int a = 0; a < Q; ++a) f[a] = make_float2(oa[a], ob[a]);
        if (valid) {
            float4 *t = reinterpret_cast<float4 *>(
                reinterpret_cast<float2 *>(tw_out) + ((long long)((y == 0 ? 0 : 1) * g.nz + z) * g.nx + x0));
            *t = make_float4(twx.x, twz.x, twx.y, twz.y);
        }
    } else {
        c = collide_pair<COLL, sizeof(T) == 4, LAY == LAY_PULL && PS_DEFAULT<COLL, sizeof(T) == 4>>(
            f, p, row_smag(p, y, g.ny));
    }

    if (ROWS != ROWS_INTERIOR && !node_row && (y == 0 || y == g.ny - 1)) {
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
    if (LAY == LAY_AA_ODD) {
        if (y == 0)
            push_pair<T, ROW_BOTTOM>(dst, g, p.wall, xl, y, z, zm, zp, lane, valid, f);
        else if (y == g.ny - 1)
            push_pair<T, ROW_TOP>(dst, g, p.wall, xl, y, z, zm, zp, lane, valid, f);
        else
            push_pair<T, ROW_INTERIOR>(dst, g, p.wall, xl, y, z, zm, zp, lane, valid, f);
    } else if (valid) {
        T *d = dst + ((long long)z * g.ny + y) * g.sx + x0;
#pragma unroll
        for (int a = 0; a < Q; ++a) st2<T>(d + (LAY == LAY_AA_EVEN ? opp_of(a) : a) * g.plane, f[a]);
    }
    if (STATS) {
        float v[K_ACC];
        stats_zero(v);
        if (valid) {
            const bool wall = ROWS != ROWS_INTERIOR && (y == 0 || y == g.ny - 1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                stats_cell(v, h ? c.rho.y : c.rho.x, h ? c.ux.y : c.ux.x, h ? c.uy.y : c.uy.x, h ? c.uz.y : c.uz.x,
                           h ? twx.y : twx.x, h ? twz.y : twz.x, wall);
            }
        }
        stats_block_store(v, part_blk);
    }
}

// Programmatic dependent launch: let the next step's grid start launching once
// every CTA of this one is running, and wait for the previous grid (whose
// output this step reads and whose input it overwrites) to complete before
// touching global memory. Both are no-ops for ordinary launches. The wait
// orders coherent loads only: read-only loads may be scheduled above it, so a
// kernel launched this way reads the previous step's output with coherent
// loads (pull_nc in lbm_device.cuh).
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

#ifndef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_MIN_BLOCKS 6   // resident CTAs per SM the register budget must allow (80 registers)
#endif
#ifndef LBM_PAIR_MRT_MIN_BLOCKS
#define LBM_PAIR_MRT_MIN_BLOCKS 5   // the same for the MRT instantiations (96 registers)
#endif

template <typename T, bool STATS, int COLL = COLL_BGK>
__global__ void __launch_bounds__(128, COLL == COLL_MRT ? LBM_PAIR_MRT_MIN_BLOCKS : LBM_PAIR_MIN_BLOCKS) k_step_pair(const T *__restrict__ src, T *__restrict__ dst, Geom g, Phys p,
                                                   float *__restrict__ tw_out, double *__restrict__ part)
{
    pdl_begin();
    const int y = blockIdx.y, z = blockIdx.z;
    const long long blk = ((long long)y * g.nz + z) * gridDim.x + blockIdx.x;
    pair_tile<T, STATS, COLL>(src, dst, g, p, tw_out, STATS ? part + blk * K_PART : nullptr, blockIdx.x, y, z);
}

// The two wall rows of the four-cell (FP16) step, run with the two-cell tile:
// a CTA of twice the four-cell launch's threads covers the same cells as one
// four-cell CTA (so the partial sums keep the four-cell layout) and each
// thread carries half the serial work (wall law, collision) of a four-cell
// thread, which shortens this one-wave, latency-bound launch. The two tile
// forms compute the same bits. grid (four-cell tiles per row, 2, nz); LAY as
// in pair_tile (for the AA kinds src == dst).
template <typename T, bool STATS, int COLL, int LAY = LAY_PULL>
__global__ void __launch_bounds__(256) k_step_pair_wall(const T *src, T *dst, Geom g, Phys p,
                                                        float *__restrict__ tw_out, double *__restrict__ part)
{
    pdl_begin();
    const int y = blockIdx.y == 0 ? 0 : g.ny - 1, z = blockIdx.z;
    const long long blk = ((long long)y * g.nz + z) * gridDim.x + blockIdx.x;
    pair_tile<T, STATS, COLL, LAY, ROWS_WALL>(src, dst, g, p, tw_out, STATS ? part + blk * K_PART : nullptr,
                                              blockIdx.x, y, z);
}

// The two-cell step on the single AA array (LAY_AA_EVEN or LAY_AA_ODD).
template <typename T, bool STATS, int COLL, int LAY>
__global__ void __launch_bounds__(128, COLL == COLL_MRT ? LBM_PAIR_MRT_MIN_BLOCKS : LBM_PAIR_MIN_BLOCKS) k_step_pair_aa(T *f, Geom g, Phys p,
                                                                            float *__restrict__ tw_out,
                                                                            double *__restrict__ part)
{
    pdl_begin();
    const int y = blockIdx.y, z = blockIdx.z;
    const long long blk = ((long long)y * g.nz + z) * gridDim.x + blockIdx.x;
    pair_tile<T, STATS, COLL, LAY>(f, f, g, p, tw_out, STATS ? part + blk * K_PART : nullptr, blockIdx.x, y, z);
}

}  // namespace lbm
