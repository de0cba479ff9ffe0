// Device-side building blocks of the fused D3Q19 LBM-LES update with the
// wall-function bounce (WFB) boundary (Han, Ooka & Kikumoto, arXiv 2009.04352).
//
// Storage: populations are kept as deviations fb_a = f_a - w_a from the rest
// state, in FP32 or FP16, structure-of-arrays [19][nz][ny][sx] with x fastest
// (sx = row pitch >= nx). The two-lattice pull scheme keeps post-collision
// values: streaming is a gather from the neighbours at the start of the next
// step. At a wall layer the populations that left toward the wall in the
// previous step are taken from the specular (WFB, free-slip) or opposite
// (bounce-back) slot, so the WFB correction of Eq. 14a,b is added when the
// wall-bound population is stored.
//
// The single-lattice AA layout keeps one array and alternates two step kinds.
// Where the state is "natural" (phase 0) f_a(x) sits in slot a of x; the even
// step reads the own slots, collides and writes f*_a into slot opp(a) of the
// same cell. The state is then in phase 1: f_a(x) is the post-collision value
// the pull gather would read, kept in the opposite slot (map MAP_AA1 below).
// The odd step gathers through that map, collides, and pushes f*_a to the slot
// and cell whose next gather it feeds (push_offset), which restores phase 0.
// Each thread reads and then rewrites the same set of slots in both kinds
// (also at the walls, where the specular push of one cell lands in the slots
// its own gather read), so the update is in place without races.
#pragma once

#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int Q = 19;

// D3Q19 velocities, numbered as in Table A-1.
__host__ __device__ constexpr int ex_of(int a)
{
    constexpr int v[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0};
    return v[a];
}
__host__ __device__ constexpr int ey_of(int a)
{
    constexpr int v[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 1, -1};
    return v[a];
}
__host__ __device__ constexpr int ez_of(int a)
{
    constexpr int v[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 1, -1, 1};
    return v[a];
}
// Opposite direction: the pairs (1,2), (3,4), ... of Table A-1.
__host__ __device__ constexpr int opp_of(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
// y-mirror (specular partner in a y = const wall): 3<->4, 7<->13, 8<->14,
// 11<->18, 12<->17, the rest unchanged (Eq. 14a,b partners).
__host__ __device__ constexpr int mirror_of(int a)
{
    constexpr int v[Q] = {0, 1, 2, 4, 3, 5, 6, 13, 14, 9, 10, 18, 17, 7, 8, 15, 16, 12, 11};
    return v[a];
}
// Weights 1/3, 1/18, 1/36 (the DdQq scheme the paper cites as ref. [27]).
__host__ __device__ constexpr double w_of(int a) { return a == 0 ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

enum { WALL_BB = 0, WALL_WFB = 1, WALL_FREESLIP = 2, WALL_NODE = 3 };
// Walls whose out-of-channel populations return to the own cell's opposite
// slot: halfway bounce-back, and the wall nodes of the full-way WFB (their
// outward populations never reach the fluid).
__host__ __device__ constexpr bool bb_map(int wall) { return wall == WALL_BB || wall == WALL_NODE; }
enum { ROW_INTERIOR = 0, ROW_BOTTOM = 1, ROW_TOP = 2 };
// Step kinds: two-lattice pull, AA even step (phase 0 -> 1), AA odd step (1 -> 0).
enum { LAY_PULL = 0, LAY_AA_EVEN = 1, LAY_AA_ODD = 2 };
// Where f_a(x) of the current state is stored: after a pull step, in AA
// phase 0 (own slot), in AA phase 1 (opposite slot of the pull source).
enum { MAP_PULL = 0, MAP_AA0 = 1, MAP_AA1 = 2 };

// Statistics layout of one block partial: 11 plane sums then 4 wall sums.
constexpr int K_STATS = 11;
constexpr int K_WALL = 4;
constexpr int K_PART = K_STATS + K_WALL;

struct Geom {
    int nx, ny, nz;
    int sx;              // row pitch in elements
    long long plane;     // elements per population = sx * ny * nz
};

struct Phys {
    float tau0;
    float smag;          // 18 sqrt(2) C_s^2 (Smagorinsky closure coefficient)
    float Fx, Fy, Fz;
    int wall;            // WALL_*
    float kappa, B;
    float ekb;           // exp(-kappa B)
    float y1_over_nu;    // y1 / nu of the wall law
    int newton_iters;
    int law;             // LAW_*: wall function that gives tau_w
    float ikappa;        // 1 / kappa
    float law_r2;        // R = (y+)^2 where the viscous branch of the log or power law ends
    float pw_a;          // power law: 8.3^(7/8), u+ = pw_a R^(1/8)
    // derived on the host once, so kernels do not recompute them per tile
    float hF[3];         // F / 2
    float weF[9];        // w_k (e_k . F) for the opposite pairs k = 0..8 (directions 2k+1, 2k+2)
    float WeF[9];        // 36 w_k (e_k . F), the same with the weights scaled by 36
    float t02;           // tau0^2
    // LES model
    int collision;       // COLL_BGK or COLL_MRT
    float vd_scale;      // van Driest: u_tau / (nu A+); 0 = no damping
    // MRT: ghost groups e, eps, q, m (rates s_g different from 1/tau_eff);
    // the correction factor of group g is omega a_g + b_g = (omega - s_g) c_g
    // (c_g from the basis norms, mrt_ghost_pair in lbm_pair.cuh)
    float mrt_a[4];
    float mrt_b[4];
};

enum { COLL_BGK = 0, COLL_MRT = 1 };
enum { LAW_SPALDING = 0, LAW_LOG = 1, LAW_POWER = 2 };

// Row i, direction a of the D3Q19 MRT moment basis of d'Humieres et al. (2002)
// (rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww,
// p_xy, p_yz, p_xz, m_x, m_y, m_z), evaluated at compile time.
__host__ __device__ constexpr int mrt_coef(int i, int a)
{
    const int x = ex_of(a), y = ey_of(a), z = ez_of(a);
    const int e2 = x * x + y * y + z * z;
    switch (i) {
    case 0: return 1;
    case 1: return 19 * e2 - 30;
    case 2: return (21 * e2 * e2 - 53 * e2 + 24) / 2;
    case 3: return x;
    case 4: return (5 * e2 - 9) * x;
    case 5: return y;
    case 6: return (5 * e2 - 9) * y;
    case 7: return z;
    case 8: return (5 * e2 - 9) * z;
    case 9: return 3 * x * x - e2;
    case 10: return (3 * e2 - 5) * (3 * x * x - e2);
    case 11: return y * y - z * z;
    case 12: return (3 * e2 - 5) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
    }
}

// Squared norm of basis row i (the rows are orthogonal: M^-1 = M^T / norm).
__host__ __device__ constexpr int mrt_norm(int i)
{
    int n = 0;
    for (int a = 0; a < Q; ++a) n += mrt_coef(i, a) * mrt_coef(i, a);
    return n;
}

// Ghost groups of the basis whose rates differ from 1/tau_eff: the energy e
// (row 1), its square eps (row 2), the energy fluxes q (rows 4, 6, 8) and the
// third-order m (rows 16-18). The five stress moments (rows 9, 11, 13-15) and
// the two fourth-order pi moments (rows 10, 12) relax with 1/tau_eff, as in
// BGK: with the published pi rate of 1.4 the scheme is linearly unstable for
// tau0 below about 0.502, where the channel runs operate (the q rates are
// raised to 1.99 for the same reason).
enum { MRT_E = 0, MRT_EPS = 1, MRT_Q = 2, MRT_M = 3 };

// Smagorinsky coefficient of layer y with the van Driest factor
// D = 1 - exp(-y+/A+) of the layer centre (j + 1/2 from the nearer wall).
__device__ __forceinline__ float row_smag(const Phys &p, int y, int ny)
{
    if (p.vd_scale <= 0.f) return p.smag;
    // distance to the nearer wall: layer centre j + 1/2 (halfway walls) or j
    // (wall nodes at layers 0 and ny - 1)
    const float d = p.wall == WALL_NODE ? (float)min(y, ny - 1 - y) : fminf(y + 0.5f, ny - y - 0.5f);
    const float D = 1.f - expf(-d * p.vd_scale);
    return p.smag * D * D;
}

// Loads of the source lattice. The read-only path (ld, __ldg) is valid only
// for data that no grid writes while the reading grid lives, and the compiler
// may schedule its loads before griddepcontrol.wait (measured: a four-cell
// step that read the previous step's output that way, launched while that step
// drained, read stale populations). So the two-lattice FP32 kernels, whose
// read-only loads measure faster, launch without programmatic dependent
// launch, and every other step kernel, launched with it, reads through
// explicitly coherent loads (ldc, ld.global.ca), which the compiler neither
// turns into read-only loads nor moves above the wait.
template <typename T> constexpr bool pull_nc = std::is_same<T, float>::value;

template <typename T> __device__ __forceinline__ float ld(const T *p);
template <> __device__ __forceinline__ float ld<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<__half>(const __half *p) { return __half2float(__ldg(p)); }

template <typename T> __device__ __forceinline__ float ldc(const T *p);
template <> __device__ __forceinline__ float ldc<float>(const float *p) { return __ldca(p); }
template <> __device__ __forceinline__ float ldc<__half>(const __half *p) { return __half2float(__ldca(p)); }

template <typename T, bool NC> __device__ __forceinline__ float ldx(const T *p) { return NC ? ld<T>(p) : ldc<T>(p); }

template <typename T> __device__ __forceinline__ void st(T *p, float v);
template <> __device__ __forceinline__ void st<float>(float *p, float v) { *p = v; }
template <> __device__ __forceinline__ void st<__half>(__half *p, float v) { *p = __float2half_rn(v); }

// Element offset that the gather of population a at cell (x, y, z) reads.
// Periodic wrap in x and z; at the wall layers the population that would come
// from outside the channel is the one that left toward the wall in the
// previous step: the own cell's opposite slot (bounce-back) or the mirrored
// slot of the cell displaced by the tangential part of e_a (specular, WFB).
template <int ROW>
__device__ __forceinline__ long long src_position(const Geom &g, int wall, int a, int x, int y, int z, int xm,
                                                  int xp, int zm, int zp, int &slot)
{
    const int ex = ex_of(a), ey = ey_of(a), ez = ez_of(a);
    int xs = ex == 1 ? xm : (ex == -1 ? xp : x);
    int zs = ez == 1 ? zm : (ez == -1 ? zp : z);
    int ys = y - ey;
    slot = a;
    const bool crosses = (ROW == ROW_BOTTOM && ey == 1) || (ROW == ROW_TOP && ey == -1);
    if (crosses) {
        ys = y;
        if (bb_map(wall)) {
            xs = x;
            zs = z;
            slot = opp_of(a);
        } else {
            slot = mirror_of(a);
        }
    }
    return ((long long)zs * g.ny + ys) * g.sx + xs;
}

template <int ROW>
__device__ __forceinline__ long long src_offset(const Geom &g, int wall, int a, int x, int y, int z,
                                                int xm, int xp, int zm, int zp)
{
    int slot;
    const long long pos = src_position<ROW>(g, wall, a, x, y, z, xm, xp, zm, zp, slot);
    return (long long)slot * g.plane + pos;
}

// Element offset of f_a(x, y, z) of the current state under storage map MAP.
template <int ROW, int MAP>
__device__ __forceinline__ long long map_offset(const Geom &g, int wall, int a, int x, int y, int z, int xm, int xp,
                                                int zm, int zp)
{
    if (MAP == MAP_AA0) return (long long)a * g.plane + ((long long)z * g.ny + y) * g.sx + x;
    int slot;
    const long long pos = src_position<ROW>(g, wall, a, x, y, z, xm, xp, zm, zp, slot);
    return (long long)(MAP == MAP_AA1 ? opp_of(slot) : slot) * g.plane + pos;
}

// AA odd step: where f*_a of cell (x, y, z) goes so that the following even
// step finds it as f_b of the cell it streams to (the inverse of the pull
// gather): slot a of x + e_a; a wall-bound population goes to the opposite
// slot of the own cell (bounce-back) or to the mirrored slot of the cell
// displaced by its tangential velocity (WFB, free slip).
template <int ROW>
__device__ __forceinline__ long long push_offset(const Geom &g, int wall, int a, int x, int y, int z, int xm, int xp,
                                                 int zm, int zp)
{
    const int ex = ex_of(a), ey = ey_of(a), ez = ez_of(a);
    int xt = ex == 1 ? xp : (ex == -1 ? xm : x);
    int zt = ez == 1 ? zp : (ez == -1 ? zm : z);
    int yt = y + ey;
    int slot = a;
    const bool crosses = (ROW == ROW_BOTTOM && ey == -1) || (ROW == ROW_TOP && ey == 1);
    if (crosses) {
        yt = y;
        if (bb_map(wall)) {
            xt = x;
            zt = z;
            slot = opp_of(a);
        } else {
            slot = mirror_of(a);
        }
    }
    return (long long)slot * g.plane + ((long long)zt * g.ny + yt) * g.sx + xt;
}

struct Nbr {
    int xm, xp, zm, zp;
};

__device__ __forceinline__ Nbr neighbours(const Geom &g, int x, int z)
{
    Nbr n;
    n.xm = x == 0 ? g.nx - 1 : x - 1;
    n.xp = x == g.nx - 1 ? 0 : x + 1;
    n.zm = z == 0 ? g.nz - 1 : z - 1;
    n.zp = z == g.nz - 1 ? 0 : z + 1;
    return n;
}

template <typename T, int ROW, int MAP, bool NC>
__device__ __forceinline__ void gather_row(const T *src, const Geom &g, int wall, int x, int y, int z, const Nbr &n,
                                           float (&fb)[Q])
{
#pragma unroll
    for (int a = 0; a < Q; ++a)
        fb[a] = ldx<T, NC>(src + map_offset<ROW, MAP>(g, wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp));
}

// f(t) of one cell under storage map MAP (NC: the array is not written
// during the launch, so the read-only path may serve it).
template <typename T, int MAP = MAP_PULL, bool NC = true>
__device__ __forceinline__ void gather(const T *src, const Geom &g, int wall, int x, int y, int z, float (&fb)[Q])
{
    const Nbr n = neighbours(g, x, z);
    if (y == 0)
        gather_row<T, ROW_BOTTOM, MAP, NC>(src, g, wall, x, y, z, n, fb);
    else if (y == g.ny - 1)
        gather_row<T, ROW_TOP, MAP, NC>(src, g, wall, x, y, z, n, fb);
    else
        gather_row<T, ROW_INTERIOR, MAP, NC>(src, g, wall, x, y, z, n, fb);
}

// gather() with the map chosen at run time (exports, off the hot path).
template <typename T>
__device__ __forceinline__ void gather_any(const T *src, const Geom &g, int wall, int map, int x, int y, int z,
                                           float (&fb)[Q])
{
    if (map == MAP_AA0)
        gather<T, MAP_AA0>(src, g, wall, x, y, z, fb);
    else if (map == MAP_AA1)
        gather<T, MAP_AA1>(src, g, wall, x, y, z, fb);
    else
        gather<T, MAP_PULL>(src, g, wall, x, y, z, fb);
}

// Element offset of f_a(x, y, z) under the run-time map (for writers of the state).
__device__ __forceinline__ long long state_offset(const Geom &g, int wall, int map, int a, int x, int y, int z,
                                                  const Nbr &n)
{
    if (map == MAP_AA0) return map_offset<ROW_INTERIOR, MAP_AA0>(g, wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp);
    if (y == 0)
        return map == MAP_AA1 ? map_offset<ROW_BOTTOM, MAP_AA1>(g, wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp)
                              : map_offset<ROW_BOTTOM, MAP_PULL>(g, wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp);
    if (y == g.ny - 1)
        return map == MAP_AA1 ? map_offset<ROW_TOP, MAP_AA1>(g, wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp)
                              : map_offset<ROW_TOP, MAP_PULL>(g, wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp);
    return map == MAP_AA1 ? map_offset<ROW_INTERIOR, MAP_AA1>(g, wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp)
                          : map_offset<ROW_INTERIOR, MAP_PULL>(g, wall, a, x, y, z, n.xm, n.xp, n.zm, n.zp);
}

// Moments of the deviations: drho = sum fb (rho - 1) and j = sum e fb
// (sum e w = 0, so j is the full momentum).
struct Moments {
    float drho, jx, jy, jz;
};

__device__ __forceinline__ Moments moments_of(const float (&f)[Q])
{
    Moments m;
    m.drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + ((f[8] + f[9]) + (f[10] + f[11])) +
             ((f[12] + f[13]) + (f[14] + f[15])) + ((f[16] + f[17]) + f[18]);
    m.jx = ((f[1] - f[2]) + (f[7] - f[8])) + ((f[9] - f[10]) + (f[13] - f[14])) + (f[15] - f[16]);
    m.jy = ((f[3] - f[4]) + (f[7] - f[8])) + ((f[11] - f[12]) + (f[14] - f[13])) + (f[17] - f[18]);
    m.jz = ((f[5] - f[6]) + (f[9] - f[10])) + ((f[11] - f[12]) + (f[16] - f[15])) + (f[18] - f[17]);
    return m;
}

// Spalding's law (Eq. 16) inverted for u+ by Newton's method (Sec. 2.3) on
// h(u+) = u+ y+(u+) - R, R = y1 |u_t| / nu (Eq. 17 gives y+ = R / u+). h is
// increasing and convex, so any start at or above the root descends
// monotonically. The start is the laminar guess sqrt(R), lowered for R > 100
// to the log-law bound ln(R)/kappa + B, which also lies above the root and
// saves the slow exponential-regime steps. Each lane keeps its value once its
// own relative step is below 1e-7, so a cell's result does not depend on which
// cells share its warp (every kernel form gives the same bits); the warp
// leaves the loop when all its lanes have stopped.
__device__ __forceinline__ float spalding_uplus(float R, const Phys &p, unsigned mask)
{
    float up = sqrtf(R);
    if (R > 100.f) up = fminf(up, __fadd_rn(logf(R) / p.kappa, p.B));
    bool done = false;
    for (int it = 0; it < p.newton_iters; ++it) {
        const float k = p.kappa * up;
        const float ek = expf(k);
        const float k2 = __fmul_rn(k, k);
        const float t2 = __fsub_rn(__fsub_rn(__fsub_rn(ek, 1.f), k), __fmul_rn(0.5f, k2));   // e^k - 1 - k - k^2/2
        const float t3 = __fsub_rn(t2, __fmul_rn(__fmul_rn(k2, k), 1.f / 6.f));            // ... - k^3/6
        const float S = __fmaf_rn(p.ekb, t3, up);                                           // y+(u+)
        const float dS = __fmaf_rn(__fmul_rn(p.ekb, p.kappa), t2, 1.f);                     // dy+/du+
        const float step = done ? 0.f : __fmaf_rn(up, S, -R) / __fmaf_rn(up, dS, S);
        up -= step;
        done = done || fabsf(step) <= 1e-7f * up;
        if (__all_sync(mask, done)) break;
    }
    return up;
}

// Two-layer log law: u+ = sqrt(R) (u+ = y+) while R <= y_c^2, else the root of
// u+ + (ln u+ - ln R) / kappa - B = 0. That function is concave and increasing,
// so Newton from the left of the root climbs to it monotonically; the start,
// one fixed-point step from the log law at y+ = R, lies left of the root for
// every R above the crossing. Same per-lane stop as spalding_uplus.
__device__ __forceinline__ float loglaw_uplus(float R, const Phys &p, unsigned mask)
{
    const bool visc = R <= p.law_r2;
    const float lr = logf(fmaxf(R, p.law_r2));
    const float u0 = __fmaf_rn(lr, p.ikappa, p.B);
    float up = __fmaf_rn(-logf(u0), p.ikappa, u0);
    bool done = visc;
    for (int it = 0; it < p.newton_iters; ++it) {
        const float h = __fsub_rn(__fmaf_rn(__fsub_rn(logf(up), lr), p.ikappa, up), p.B);
        const float step = done ? 0.f : h / __fadd_rn(1.f, p.ikappa / up);
        up -= step;
        done = done || fabsf(step) <= 1e-7f * up;
        if (__all_sync(mask, done)) break;
    }
    return visc ? sqrtf(R) : up;
}

// Werner-Wengle power law: u+ = sqrt(R) while R <= 8.3^(7/3), else
// u+ = (8.3 R^(1/7))^(7/8) = 8.3^(7/8) R^(1/8), three square roots.
__device__ __forceinline__ float powerlaw_uplus(float R, const Phys &p)
{
    const float r2 = sqrtf(R);
    return R <= p.law_r2 ? r2 : p.pw_a * sqrtf(sqrtf(r2));
}

// u+ of the selected wall function (p.law is uniform over the launch).
__device__ __forceinline__ float wall_uplus(float R, const Phys &p, unsigned mask)
{
    if (p.law == LAW_LOG) return loglaw_uplus(R, p, mask);
    if (p.law == LAW_POWER) return powerlaw_uplus(R, p);
    return spalding_uplus(R, p, mask);
}

}  // namespace lbm
