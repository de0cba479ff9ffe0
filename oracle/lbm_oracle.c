/*
 * FP64 CPU oracle of the LBM-LES channel update with the wall-function bounce
 * (WFB) boundary of Han, Ooka & Kikumoto (arXiv 2009.04352).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference that the
 * CUDA path is checked against. Only the tests, the package smoke check and
 * the CPU-baseline leg of the benchmark may build, load or call it. It shares
 * no code, header, table or helper with the CUDA library.
 *
 * Everything is IEEE double, written as the definitions read, one cell and one
 * direction at a time, two population arrays (push: collide, wall fix, stream).
 * Build with -ffp-contract=off so results do not depend on FMA contraction.
 *
 * Lattice units: dx = dt = 1, c_s^2 = 1/3. Grid nx*ny*nz, x periodic
 * (streamwise), y wall-normal, z periodic (spanwise). All ny layers are fluid;
 * the walls sit half a link outside them, at y = -1/2 and y = ny - 1/2.
 * Population arrays are [19][nz][ny][nx], x fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* D3Q19 velocities in the numbering of Table A-1 (odd a: upper sign of the
 * pair, even a: lower sign). */
static const int E[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},   {-1, 0, 0},
    {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0},
    {1, 0, 1},   {-1, 0, -1},
    {0, 1, 1},   {0, -1, -1},
    {1, -1, 0},  {-1, 1, 0},
    {1, 0, -1},  {-1, 0, 1},
    {0, 1, -1},  {0, -1, 1},
};

/* Textbook D3Q19 weights (the paper cites the DdQq scheme, ref. [27], and
 * does not print them): 1/3 rest, 1/18 axis, 1/36 diagonal. */
static double weight(int a)
{
    if (a == 0) return 1.0 / 3.0;
    if (a <= 6) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* The direction with the opposite velocity (bounce-back partner). */
static int opposite(int a)
{
    for (int b = 0; b < Q; ++b)
        if (E[b][0] == -E[a][0] && E[b][1] == -E[a][1] && E[b][2] == -E[a][2]) return b;
    return -1;
}

/* The direction mirrored in a y = const wall: y component reversed, x and z
 * kept (free-slip / specular partner, Sec. 2.1 Eq. 4 and Sec. 2.2 Eq. 14). */
static int mirror_y(int a)
{
    for (int b = 0; b < Q; ++b)
        if (E[b][0] == E[a][0] && E[b][1] == -E[a][1] && E[b][2] == E[a][2]) return b;
    return -1;
}

/* ---------------------------------------------------------------- tables -- */

void or_table(int *e_out, double *w_out, int *opp_out, int *mirror_out)
{
    for (int a = 0; a < Q; ++a) {
        for (int c = 0; c < 3; ++c) e_out[3 * a + c] = E[a][c];
        w_out[a] = weight(a);
        opp_out[a] = opposite(a);
        mirror_out[a] = mirror_y(a);
    }
}

/* ------------------------------------------------------- cell arithmetic -- */

/* Second-order equilibrium f_a^eq = w_a rho [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u]. */
void or_feq(double rho, const double *u, double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int a = 0; a < Q; ++a) {
        double eu = E[a][0] * u[0] + E[a][1] * u[1] + E[a][2] * u[2];
        feq[a] = weight(a) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Zeroth and first moments (Eq. 2), with the half-force velocity shift of the
 * Guo forcing: rho = sum f, u = (sum e f + F/2) / rho. */
void or_moments_cell(const double *f, const double *F, double *rho, double *u)
{
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < Q; ++a) {
        r += f[a];
        for (int c = 0; c < 3; ++c) m[c] += E[a][c] * f[a];
    }
    *rho = r;
    for (int c = 0; c < 3; ++c) u[c] = (m[c] + 0.5 * F[c]) / r;
}

/* Non-equilibrium momentum flux Pi_ab = sum_a e_a,alpha e_a,beta (f_a - f_a^eq),
 * as a row-major 3x3 matrix. */
void or_pi_neq(const double *f, const double *feq, double *pi)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int a = 0; a < Q; ++a) s += E[a][i] * E[a][j] * (f[a] - feq[a]);
            pi[3 * i + j] = s;
        }
}

/* Standard Smagorinsky closure (Sec. 3.1, C_s = 0.1): the eddy viscosity
 * nu_t = C_s^2 |S| with the strain rate taken from the non-equilibrium flux,
 * |S| = Q / (sqrt(2) rho c_s^2 tau_eff), Q = sqrt(Pi:Pi). Writing
 * c_s^2 (tau_eff - 1/2) = c_s^2 (tau0 - 1/2) + nu_t gives a quadratic in
 * tau_eff whose positive root is returned. Filter width = 1 lattice spacing. */
double or_tau_eff(double tau0, double cs, double rho, const double *pi)
{
    double qq = 0.0;
    for (int k = 0; k < 9; ++k) qq += pi[k] * pi[k];
    double qn = sqrt(qq);
    double cs2 = 1.0 / 3.0;
    /* tau^2 - tau0 tau - C_s^2 Q / (sqrt(2) rho c_s^4) = 0 */
    double c = cs * cs * qn / (sqrt(2.0) * rho * cs2 * cs2);
    return 0.5 * (tau0 + sqrt(tau0 * tau0 + 4.0 * c));
}

/* Guo et al. (2002) forcing term of Eq. 1 for relaxation time tau:
 * F_a = (1 - 1/(2 tau)) w_a [3 (e_a - u) + 9 (e_a . u) e_a] . F. */
void or_guo(double tau, const double *u, const double *F, double *Fa)
{
    for (int a = 0; a < Q; ++a) {
        double eu = E[a][0] * u[0] + E[a][1] * u[1] + E[a][2] * u[2];
        double s = 0.0;
        for (int c = 0; c < 3; ++c) s += (3.0 * (E[a][c] - u[c]) + 9.0 * eu * E[a][c]) * F[c];
        Fa[a] = (1.0 - 1.0 / (2.0 * tau)) * weight(a) * s;
    }
}

/* One BGK collision of a cell (Eq. 1 with Omega_a = -(f_a - f_a^eq)/tau_eff):
 * f*_a = f_a - (f_a - f_a^eq)/tau_eff + F_a. Returns rho, u, tau_eff too. */
void or_collide(const double *f, double tau0, double cs, const double *F,
                double *fstar, double *rho_out, double *u_out, double *tau_out)
{
    double rho, u[3], feq[Q], pi[9], Fa[Q];
    or_moments_cell(f, F, &rho, u);
    or_feq(rho, u, feq);
    or_pi_neq(f, feq, pi);
    double tau = or_tau_eff(tau0, cs, rho, pi);
    or_guo(tau, u, F, Fa);
    for (int a = 0; a < Q; ++a) fstar[a] = f[a] - (f[a] - feq[a]) / tau + Fa[a];
    if (rho_out) *rho_out = rho;
    if (u_out) for (int c = 0; c < 3; ++c) u_out[c] = u[c];
    if (tau_out) *tau_out = tau;
}

/* ------------------------------------------------------- MRT collision -- */

/* Moment basis of the D3Q19 multiple-relaxation-time model of d'Humieres et
 * al. (2002), the MRT of ref. [40] used in Sec. 3.1. Row i, direction a, with
 * e = e_a and |e|^2 = e.e:
 *   0 rho 1                     1 e   19|e|^2 - 30        2 eps (21|e|^4 - 53|e|^2 + 24)/2
 *   3 j_x e_x                   4 q_x (5|e|^2 - 9) e_x    5 j_y, 6 q_y, 7 j_z, 8 q_z alike
 *   9 3p_xx 3e_x^2 - |e|^2     10 3pi_xx (3|e|^2 - 5)(3e_x^2 - |e|^2)
 *  11 p_ww e_y^2 - e_z^2       12 pi_ww (3|e|^2 - 5)(e_y^2 - e_z^2)
 *  13 p_xy e_x e_y             14 p_yz e_y e_z             15 p_xz e_x e_z
 *  16 m_x (e_y^2 - e_z^2) e_x  17 m_y (e_z^2 - e_x^2) e_y  18 m_z (e_x^2 - e_y^2) e_z */
void or_mrt_matrix(double *M)
{
    for (int a = 0; a < Q; ++a) {
        const double x = E[a][0], y = E[a][1], z = E[a][2];
        const double e2 = x * x + y * y + z * z;
        double r[Q];
        r[0] = 1.0;
        r[1] = 19.0 * e2 - 30.0;
        r[2] = (21.0 * e2 * e2 - 53.0 * e2 + 24.0) / 2.0;
        r[3] = x;
        r[4] = (5.0 * e2 - 9.0) * x;
        r[5] = y;
        r[6] = (5.0 * e2 - 9.0) * y;
        r[7] = z;
        r[8] = (5.0 * e2 - 9.0) * z;
        r[9] = 3.0 * x * x - e2;
        r[10] = (3.0 * e2 - 5.0) * (3.0 * x * x - e2);
        r[11] = y * y - z * z;
        r[12] = (3.0 * e2 - 5.0) * (y * y - z * z);
        r[13] = x * y;
        r[14] = y * z;
        r[15] = x * z;
        r[16] = (y * y - z * z) * x;
        r[17] = (z * z - x * x) * y;
        r[18] = (x * x - y * y) * z;
        for (int i = 0; i < Q; ++i) M[i * Q + a] = r[i];
    }
}

/* Relaxation rates of the D3Q19 MRT model after d'Humieres et al. (2002):
 * s_e = 1.19, s_eps = 1.4, s_m = 1.98; the five stress moments
 * (9, 11, 13, 14, 15) and the two pi moments (10, 12) relax with 1/tau_eff,
 * and the energy fluxes q with 1.99 (the published s_pi = 1.4 and s_q = 1.2
 * are replaced, see below); the conserved moments (0, 3, 5, 7) take 1 (their
 * value does not enter the result). */
void or_mrt_rates(double tau, double *s)
{
    for (int i = 0; i < Q; ++i) s[i] = 1.0;
    s[1] = 1.19;
    s[2] = 1.4;
    s[16] = s[17] = s[18] = 1.98;
    s[9] = s[11] = s[13] = s[14] = s[15] = 1.0 / tau;
    /* The channel runs of Sec. 3.1 operate at tau0 ~ 0.5002, where the
     * published rates make the scheme linearly unstable: a normal-stress mode
     * grows at rest unless the fourth-order pi moments relax with the shear
     * rate, and with a mean flow of a few percent of the lattice speed unless
     * the energy fluxes q relax near 2 as well. */
    s[10] = s[12] = 1.0 / tau;
    s[4] = s[6] = s[8] = 1.99;
}

/* One MRT collision with the same moments, equilibrium, Smagorinsky closure
 * and Guo forcing as or_collide: with m = M f,
 *   m* = m - S (m - M f^eq) + (I - S/2) M G,  G_a = w_a [3 (e_a - u) + 9 (e_a.u) e_a].F
 *   f* = M^-1 m*  (M has orthogonal rows: M^-1 = M^T diag(1 / |row|^2)).
 * `damp` multiplies C_s (van Driest factor, 1 = none). With every rate 1/tau
 * the update is exactly BGK. */
void or_collide_mrt_rates(const double *f, double tau0, double cs, const double *F, double damp,
                          const double *rates, double *fstar, double *rho_out, double *u_out,
                          double *tau_out);

void or_collide_mrt(const double *f, double tau0, double cs, const double *F, double damp,
                    double *fstar, double *rho_out, double *u_out, double *tau_out)
{
    or_collide_mrt_rates(f, tau0, cs, F, damp, NULL, fstar, rho_out, u_out, tau_out);
}

/* As or_collide_mrt with the 19 rates given explicitly (rates != NULL). */
void or_collide_mrt_rates(const double *f, double tau0, double cs, const double *F, double damp,
                          const double *rates, double *fstar, double *rho_out, double *u_out,
                          double *tau_out)
{
    static double M[Q * Q];
    static int built = 0;
    if (!built) {
        or_mrt_matrix(M);
        built = 1;
    }
    double rho, u[3], feq[Q], pi[9], G[Q], s[Q];
    or_moments_cell(f, F, &rho, u);
    or_feq(rho, u, feq);
    or_pi_neq(f, feq, pi);
    const double tau = or_tau_eff(tau0, cs * damp, rho, pi);
    or_mrt_rates(tau, s);
    if (rates)
        for (int i = 0; i < Q; ++i) s[i] = rates[i];
    for (int a = 0; a < Q; ++a) {
        double eu = E[a][0] * u[0] + E[a][1] * u[1] + E[a][2] * u[2];
        double t = 0.0;
        for (int c = 0; c < 3; ++c) t += (3.0 * (E[a][c] - u[c]) + 9.0 * eu * E[a][c]) * F[c];
        G[a] = weight(a) * t;
    }
    double dm[Q];
    for (int i = 0; i < Q; ++i) {
        double m = 0.0, meq = 0.0, mg = 0.0;
        for (int a = 0; a < Q; ++a) {
            m += M[i * Q + a] * f[a];
            meq += M[i * Q + a] * feq[a];
            mg += M[i * Q + a] * G[a];
        }
        dm[i] = -s[i] * (m - meq) + (1.0 - 0.5 * s[i]) * mg;
    }
    for (int a = 0; a < Q; ++a) {
        double df = 0.0;
        for (int i = 0; i < Q; ++i) {
            double n2 = 0.0;
            for (int b = 0; b < Q; ++b) n2 += M[i * Q + b] * M[i * Q + b];
            df += M[i * Q + a] * dm[i] / n2;
        }
        fstar[a] = f[a] + df;
    }
    if (rho_out) *rho_out = rho;
    if (u_out) for (int c = 0; c < 3; ++c) u_out[c] = u[c];
    if (tau_out) *tau_out = tau;
}

/* van Driest damping factor 1 - exp(-y+ / A+) of the Smagorinsky length for
 * layer j of ny (halfway walls: the layer centre lies j + 1/2 from the bottom
 * wall), with y+ = y u_tau / nu from a reference friction velocity. */
double or_van_driest(int j, int ny, double u_tau, double nu, double a_plus)
{
    double d = j + 0.5;
    if (ny - j - 0.5 < d) d = ny - j - 0.5;
    return 1.0 - exp(-d * u_tau / nu / a_plus);
}

/* --------------------------------------------------- Spalding wall law -- */

/* Eq. 16: y+ as an explicit function of u+. */
double or_spalding_yplus(double up, double kappa, double B)
{
    double k = kappa * up;
    return up + exp(-kappa * B) * (exp(k) - 1.0 - k - k * k / 2.0 - k * k * k / 6.0);
}

static double spalding_dyplus(double up, double kappa, double B)
{
    double k = kappa * up;
    return 1.0 + exp(-kappa * B) * kappa * (exp(k) - 1.0 - k - k * k / 2.0);
}

/* Newton's method for u+ given R = y1 |u_t| / nu (Sec. 2.3). With y+ = R / u+
 * (Eq. 17), Eq. 16 becomes h(u+) = u+ y+(u+) - R = 0. The first guess is the
 * laminar one, u_tau = sqrt(nu |u_t| / y1), i.e. u+ = sqrt(R). Iterates until
 * the step is below tol * u+ or max_iter steps. Far in the log layer the
 * laminar guess is large and the first steps shrink u+ by about 1/kappa each,
 * so the cap must be generous (the wall stress uses 1000). Where the laminar
 * guess would overflow exp(kappa u+) (kappa sqrt(R) > 700, R above about 3e6)
 * the first guess is the log law at y+ = R instead, ln(R) / kappa + B, which
 * lies above the root (y+ = R / u+ < R) so Newton on the convex h still
 * descends monotonically. Returns the number of steps taken; iterates[0..n]
 * (optional) receives the sequence of u+. */
int or_spalding_newton(double R, double kappa, double B, int max_iter, double tol,
                       double *up_out, double *iterates)
{
    double up = sqrt(R);
    if (kappa * up > 700.0) up = log(R) / kappa + B;
    int n = 0;
    if (iterates) iterates[0] = up;
    while (n < max_iter) {
        double S = or_spalding_yplus(up, kappa, B);
        double h = up * S - R;
        double dh = S + up * spalding_dyplus(up, kappa, B);
        double step = h / dh;
        up -= step;
        ++n;
        if (iterates) iterates[n] = up;
        if (fabs(step) <= tol * fabs(up)) break;
    }
    *up_out = up;
    return n;
}

/* Other wall functions of the WFB frame (Sec. 2.3: any law that gives tau_w):
 *  law 1, two-layer log law: u+ = y+ below the crossing y_c of the two
 *    branches, u+ = ln(y+)/kappa + B above it;
 *  law 2, power law of Werner & Wengle: u+ = y+ below y+ = A^(1/(1-b)),
 *    u+ = A (y+)^b above it, A = 8.3, b = 1/7 (point-wise form).
 * Each returns u+ for R = y1 |u_t| / nu (y+ = R / u+). */
double or_loglaw_crossing(double kappa, double B)
{
    double y = 11.0;   /* y = ln(y)/kappa + B, by Newton from above the root */
    for (int i = 0; i < 100; ++i) y -= (y - log(y) / kappa - B) / (1.0 - 1.0 / (kappa * y));
    return y;
}

double or_loglaw_uplus(double R, double kappa, double B)
{
    const double yc = or_loglaw_crossing(kappa, B);
    if (sqrt(R) <= yc) return sqrt(R);   /* viscous branch: u+ = y+ = R/u+ */
    double up = yc;                       /* log branch: u+ = ln(R/u+)/kappa + B */
    for (int i = 0; i < 200; ++i) {
        const double h = up - log(R / up) / kappa - B;
        const double step = h / (1.0 + 1.0 / (kappa * up));
        up -= step;
        if (fabs(step) <= 1e-15 * up) break;
    }
    return up;
}

double or_powerlaw_uplus(double R)
{
    const double A = 8.3, b = 1.0 / 7.0;
    const double ym = pow(A, 1.0 / (1.0 - b));   /* where the two branches meet */
    if (sqrt(R) <= ym) return sqrt(R);
    /* u+ = A (R/u+)^b  ->  u+ = (A R^b)^(1/(1+b)) */
    return pow(A * pow(R, b), 1.0 / (1.0 + b));
}

/* u+ of wall function `law` (0 Spalding, 1 log law, 2 power law). */
double or_wall_uplus(int law, double R, double kappa, double B)
{
    if (law == 1) return or_loglaw_uplus(R, kappa, B);
    if (law == 2) return or_powerlaw_uplus(R);
    double up;
    or_spalding_newton(R, kappa, B, 1000, 1e-14, &up, NULL);
    return up;
}

/* Wall shear stress vector from the first-layer cell (Eqs. 15-17): magnitude
 * tau_w = rho u_tau^2, direction opposite to the tangential velocity. Zero when
 * the tangential velocity vanishes. tw[0] = tau_w,x, tw[1] = tau_w,z. */
void or_wfb_stress_law(int law, double rho, const double *u, double kappa, double B, double y1,
                       double nu, double *tw)
{
    double ut = sqrt(u[0] * u[0] + u[2] * u[2]);
    tw[0] = 0.0;
    tw[1] = 0.0;
    if (ut == 0.0) return;
    const double up = or_wall_uplus(law, y1 * ut / nu, kappa, B);
    double utau = ut / up;
    double taw = rho * utau * utau;
    tw[0] = -u[0] / ut * taw;
    tw[1] = -u[2] / ut * taw;
}

void or_wfb_stress(double rho, const double *u, double kappa, double B, double y1,
                   double nu, double *tw)
{
    or_wfb_stress_law(0, rho, u, kappa, B, y1, nu, tw);
}

/* ------------------------------------------------- seeded initial field -- */

/* SplitMix64 (Steele, Lea & Flood 2014): first output of the generator whose
 * state is s: s += 0x9e3779b97f4a7c15, then the two xor-shift-multiply rounds. */
uint64_t or_splitmix64(uint64_t s)
{
    uint64_t z = s + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Uniform [0,1) variate for (seed, counter): top 53 bits times 2^-53. */
double or_uniform(uint64_t seed, uint64_t counter)
{
    return (double)(or_splitmix64(seed ^ counter) >> 11) * (1.0 / 9007199254740992.0);
}

/* --------------------------------------------------------- the lattice -- */

typedef struct {
    int nx, ny, nz;
    long long n;                /* cells */
    double tau0, cs, F[3];
    int wall;                   /* 0 bounce-back, 1 WFB, 2 free-slip, 3 wall-node WFB */
    double kappa, B, y1, nu;
    int collision;              /* 0 BGK, 1 MRT */
    double vd_utau, vd_aplus;   /* van Driest reference u_tau and A+ (A+ <= 0: off) */
    int law;                    /* wall function: 0 Spalding, 1 log law, 2 power law */
    int threads;                /* > 1: the all-cores timing mode of or_step */
    double *f, *g;              /* current and next populations [19][n] */
    double *tw;                 /* wall stress of the last step [2][nz][nx][2] */
    double *dfw;                /* Eq. B-1 per wall of the last step [2] */
    long long step;
    int stats_every;
    double *stats;              /* [ny][11] */
    double wstats[8];           /* [2 walls][4] */
    long long nsamples;
} or_lattice;

enum { K_STATS = 11 };

static long long cidx(const or_lattice *L, int x, int y, int z)
{
    return ((long long)z * L->ny + y) * L->nx + x;
}

static int wrap(int i, int n)
{
    return ((i % n) + n) % n;
}

or_lattice *or_create(int nx, int ny, int nz, double tau0, double cs, const double *F,
                      int wall, double kappa, double B, double y1, double nu, int stats_every)
{
    if (nx < 1 || ny < 2 || nz < 1 || tau0 <= 0.5 || wall < 0 || wall > 3) return NULL;
    if (wall == 3 && ny < 3) return NULL;   /* two wall nodes and at least one fluid layer */
    or_lattice *L = (or_lattice *)calloc(1, sizeof(or_lattice));
    L->nx = nx; L->ny = ny; L->nz = nz;
    L->n = (long long)nx * ny * nz;
    L->tau0 = tau0; L->cs = cs;
    for (int c = 0; c < 3; ++c) L->F[c] = F[c];
    L->wall = wall; L->kappa = kappa; L->B = B; L->y1 = y1;
    L->nu = nu > 0 ? nu : (tau0 - 0.5) / 3.0;
    L->f = (double *)calloc((size_t)Q * L->n, sizeof(double));
    L->g = (double *)calloc((size_t)Q * L->n, sizeof(double));
    L->tw = (double *)calloc((size_t)4 * nx * nz, sizeof(double));
    L->dfw = (double *)calloc(2, sizeof(double));
    L->stats = (double *)calloc((size_t)ny * K_STATS, sizeof(double));
    L->stats_every = stats_every;
    if (!L->f || !L->g || !L->tw || !L->stats) return NULL;
    /* fluid at rest: f = w */
    for (int a = 0; a < Q; ++a)
        for (long long i = 0; i < L->n; ++i) L->f[a * L->n + i] = weight(a);
    return L;
}

void or_destroy(or_lattice *L)
{
    if (!L) return;
    free(L->f); free(L->g); free(L->tw); free(L->dfw); free(L->stats);
    free(L);
}

/* f = f^eq(rho = 1, u0) with u0 = (u_mean_x[j] + a (2U0 - 1), a (2U1 - 1),
 * a (2U2 - 1)); U_c = uniform(seed, 3 * cell + c) and cell the linear index. */
void or_init_channel(or_lattice *L, const double *u_mean_x, double amp, uint64_t seed)
{
    for (int z = 0; z < L->nz; ++z)
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                long long i = cidx(L, x, y, z);
                double u[3], feq[Q];
                for (int c = 0; c < 3; ++c) {
                    double r = or_uniform(seed, (uint64_t)i * 3u + (uint64_t)c);
                    double noise = (2.0 * r - 1.0) * amp;
                    u[c] = (c == 0 ? u_mean_x[y] : 0.0) + noise;
                }
                or_feq(1.0, u, feq);
                for (int a = 0; a < Q; ++a) L->f[a * L->n + i] = feq[a];
            }
    L->step = 0;
}

void or_set_populations(or_lattice *L, const double *f)
{
    memcpy(L->f, f, sizeof(double) * Q * L->n);
}

void or_get_populations(const or_lattice *L, double *f)
{
    memcpy(f, L->f, sizeof(double) * Q * L->n);
}

/* rho [n] and u [3][n] of the current populations (u with the F/2 shift). */
void or_moments(const or_lattice *L, double *rho, double *u)
{
    for (long long i = 0; i < L->n; ++i) {
        double f[Q], r, uu[3];
        for (int a = 0; a < Q; ++a) f[a] = L->f[a * L->n + i];
        or_moments_cell(f, L->F, &r, uu);
        if (rho) rho[i] = r;
        if (u) for (int c = 0; c < 3; ++c) u[c * L->n + i] = uu[c];
    }
}

/* Mass and raw momentum sum_cells sum_a (1, e_a) f_a; out[4]. */
void or_conservation(const or_lattice *L, double *out)
{
    for (int k = 0; k < 4; ++k) out[k] = 0.0;
    for (int a = 0; a < Q; ++a)
        for (long long i = 0; i < L->n; ++i) {
            double v = L->f[a * L->n + i];
            out[0] += v;
            for (int c = 0; c < 3; ++c) out[1 + c] += E[a][c] * v;
        }
}

void or_wall_stress(const or_lattice *L, double *tw)
{
    memcpy(tw, L->tw, sizeof(double) * 4 * L->nx * L->nz);
}

void or_wall_delta_f(const or_lattice *L, double *out)
{
    out[0] = L->dfw[0];
    out[1] = L->dfw[1];
}

/* Plane statistics: per layer y the sums over samples and over the layer of
 * rho, u_x, u_y, u_z, u_x^2, u_y^2, u_z^2, u_x u_y, rho u_x, rho u_y, rho u_z;
 * wall sums [2][4] of tau_w,x, tau_w,z, |tau_w|, |tau_w|^2. */
void or_plane_stats(or_lattice *L, double *out, double *wall_out, long long *nsamples,
                    int reset)
{
    if (out) memcpy(out, L->stats, sizeof(double) * L->ny * K_STATS);
    if (wall_out) memcpy(wall_out, L->wstats, sizeof(double) * 8);
    if (nsamples) *nsamples = L->nsamples;
    if (reset) {
        memset(L->stats, 0, sizeof(double) * L->ny * K_STATS);
        memset(L->wstats, 0, sizeof(L->wstats));
        L->nsamples = 0;
    }
}

long long or_get_step(const or_lattice *L)
{
    return L->step;
}

/* Collision operator (0 BGK, 1 MRT) and van Driest damping of the
 * Smagorinsky length (a_plus <= 0 turns it off). */
/* Wall function of the WFB layer (0 Spalding Eq. 16, 1 log law, 2 power law). */
int or_set_wall_law(or_lattice *L, int law)
{
    if (law < 0 || law > 2) return -1;
    L->law = law;
    return 0;
}

void or_set_les(or_lattice *L, int collision, double u_tau, double a_plus)
{
    L->collision = collision;
    L->vd_utau = u_tau;
    L->vd_aplus = a_plus;
}

/* Full-way (wall-node) WFB at the wall node (x, y, z), y = 0 or ny - 1: the
 * literal geometry of Eq. 14 and Table 1, with wall nodes and the first fluid
 * node one lattice spacing from the wall. tau_w is the wall law applied to the
 * first fluid node's velocity (Eqs. 15-17 with y+ = y1 u_tau / nu, y1 = 1 for
 * this geometry). The node sends back into the fluid the specular partners of
 * the populations that arrived from it, plus (dt / 2 dy) (tau_w . e)
 * (Eqs. 13, 14a,b), and reverses every other population (full-way
 * bounce-back: axis f3 <- f4 and the in-plane and outward ones, which never
 * reach the fluid). rho and u receive the node's own moments. */
static void or_wall_node(const or_lattice *L, int x, int y, int z, const double *f, double *fs, double *tw,
                         double *rho, double *u)
{
    const long long n = L->n;
    const int ya = (y == 0) ? 1 : L->ny - 2;   /* the first fluid node */
    const int into = (y == 0) ? 1 : -1;        /* e_y of the populations entering the fluid */
    double fa[Q], rho_a, ua[3];
    const long long ia = cidx(L, x, ya, z);
    for (int a = 0; a < Q; ++a) fa[a] = L->f[a * n + ia];
    or_moments_cell(fa, L->F, &rho_a, ua);
    or_wfb_stress_law(L->law, rho_a, ua, L->kappa, L->B, L->y1, L->nu, tw);
    for (int a = 0; a < Q; ++a) fs[a] = f[opposite(a)];
    for (int b = 0; b < Q; ++b)
        if (E[b][1] == into) fs[b] = f[mirror_y(b)] + 0.5 * (tw[0] * E[b][0] + tw[1] * E[b][2]);
    or_moments_cell(f, L->F, rho, u);
}

/* One cell of one step: collide, wall treatment, stream into L->g; adds the
 * cell's Eq. B-1 difference to dfsum[wall] and, on sampled steps, its moments
 * to the plane statistics. */
static void or_cell(or_lattice *L, int x, int y, int z, int sample, double *dfsum)
{
    const int nx = L->nx, ny = L->ny, nz = L->nz;
    const long long n = L->n;
    long long i = cidx(L, x, y, z);
    double f[Q], fs[Q], rho, u[3], tau;
    for (int a = 0; a < Q; ++a) f[a] = L->f[a * n + i];
    int wall_id = (y == 0) ? 0 : ((y == ny - 1) ? 1 : -1);
    const int node = L->wall == 3 && wall_id >= 0;
    double tw[2] = {0.0, 0.0};
    if (node) {
        or_wall_node(L, x, y, z, f, fs, tw, &rho, u);
    } else {
        double damp = 1.0;
        if (L->vd_aplus > 0.0) {
            if (L->wall == 3) {   /* distance to the nearer wall node */
                const double d = (y < ny - 1 - y) ? y : ny - 1 - y;
                damp = 1.0 - exp(-d * L->vd_utau / L->nu / L->vd_aplus);
            } else {
                damp = or_van_driest(y, ny, L->vd_utau, L->nu, L->vd_aplus);
            }
        }
        if (L->collision == 1)
            or_collide_mrt(f, L->tau0, L->cs, L->F, damp, fs, &rho, u, &tau);
        else
            or_collide(f, L->tau0, L->cs * damp, L->F, fs, &rho, u, &tau);
    }

    if (wall_id >= 0 && L->wall == 1)
        or_wfb_stress_law(L->law, rho, u, L->kappa, L->B, L->y1, L->nu, tw);
    if (wall_id >= 0 && L->wall == 0) {
        /* momentum the bounce-back returns to the fluid */
        int dir = (wall_id == 0) ? -1 : 1;
        for (int a = 0; a < Q; ++a)
            if (E[a][1] == dir) {
                tw[0] += -2.0 * E[a][0] * fs[a];
                tw[1] += -2.0 * E[a][2] * fs[a];
            }
    }
    if (wall_id >= 0) {
        double *t = L->tw + ((size_t)(wall_id * nz + z) * nx + x) * 2;
        t[0] = tw[0];
        t[1] = tw[1];
    }

    if (sample) {
        double *st = L->stats + (size_t)y * K_STATS;
        st[0] += rho;
        st[1] += u[0]; st[2] += u[1]; st[3] += u[2];
        st[4] += u[0] * u[0]; st[5] += u[1] * u[1]; st[6] += u[2] * u[2];
        st[7] += u[0] * u[1];
        st[8] += rho * u[0]; st[9] += rho * u[1]; st[10] += rho * u[2];
        if (wall_id >= 0) {
            double m2 = tw[0] * tw[0] + tw[1] * tw[1];
            double *ws = L->wstats + 4 * wall_id;
            ws[0] += tw[0]; ws[1] += tw[1]; ws[2] += sqrt(m2); ws[3] += m2;
        }
    }

    /* stream */
    double out_sum = 0.0, back_sum = 0.0;
    if (node) {   /* Eq. B-1 at a wall node: what it sends back vs what arrived */
        const int into = (wall_id == 0) ? 1 : -1;
        for (int a = 0; a < Q; ++a) {
            if (E[a][1] == into) back_sum += fs[a];
            if (E[a][1] == -into) out_sum += f[a];
        }
    }
    for (int a = 0; a < Q; ++a) {
        int ty = y + E[a][1];
        if (ty >= 0 && ty < ny) {
            int tx = wrap(x + E[a][0], nx), tz = wrap(z + E[a][2], nz);
            L->g[a * n + cidx(L, tx, ty, tz)] = fs[a];
        } else if (L->wall == 0 || L->wall == 3) {
            L->g[opposite(a) * n + i] = fs[a];
        } else {
            int tx = wrap(x + E[a][0], nx), tz = wrap(z + E[a][2], nz);
            double corr = 0.0;
            if (L->wall == 1) corr = 0.5 * (tw[0] * E[a][0] + tw[1] * E[a][2]);
            double v = fs[a] + corr;
            L->g[mirror_y(a) * n + cidx(L, tx, y, tz)] = v;
            out_sum += fs[a];
            back_sum += v;
        }
    }
    if (wall_id >= 0) dfsum[wall_id] += back_sum - out_sum;
}

/* One time step t -> t+1: for every cell collide (Eq. 1), find the wall
 * stress of wall-layer cells, then stream each post-collision population to
 * x + e_a. A population that would cross a wall is
 *   bounce-back: returned to the same cell in the opposite direction;
 *   WFB:         reflected specularly to x + (e_x, 0, e_z) in the mirrored
 *                direction, plus (dt / 2 dy) (tau_w . e_a) (Eqs. 14a,b, 15);
 *   free-slip:   as WFB with tau_w = 0.
 * The wall stress reported for bounce-back is the tangential momentum the
 * reflection adds, -2 sum over wall-bound a of e_a,t f*_a. */
void or_step(or_lattice *L, int nsteps)
{
    const int nx = L->nx, ny = L->ny, nz = L->nz;
    for (int s = 0; s < nsteps; ++s) {
        int sample = L->stats_every > 0 && (L->step % L->stats_every) == 0;
        double dfsum[2] = {0.0, 0.0};
        if (L->threads > 1 && !sample) {
            /* all-cores timing mode: planes z in parallel (each target slot is
             * written by exactly one source cell), the Eq. B-1 sums per plane
             * added up in plane order afterwards */
            double *dfz = (double *)calloc((size_t)2 * nz, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(L->threads)
#endif
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x) or_cell(L, x, y, z, 0, dfz + 2 * z);
            for (int z = 0; z < nz; ++z) {
                dfsum[0] += dfz[2 * z];
                dfsum[1] += dfz[2 * z + 1];
            }
            free(dfz);
        } else {
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x) or_cell(L, x, y, z, sample, dfsum);
        }
        L->dfw[0] = dfsum[0] / ((double)nx * nz);
        L->dfw[1] = dfsum[1] / ((double)nx * nz);
        if (sample) L->nsamples += 1;
        double *tmp = L->f;
        L->f = L->g;
        L->g = tmp;
        L->step += 1;
    }
}

/* Threads of the all-cores mode (1, the default, is the plain serial oracle;
 * without OpenMP support at build time the loop runs serially anyway).
 * Returns the number that will be used. */
int or_set_threads(or_lattice *L, int threads)
{
#ifdef _OPENMP
    L->threads = threads > 1 ? threads : 1;
#else
    (void)threads;
    L->threads = 1;
#endif
    return L->threads;
}
