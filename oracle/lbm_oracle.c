/*
 * FP64 CPU oracle for the kinetic-closure LES lattice-Boltzmann update
 * (Marson & Malaspinas, "Kinetic closure of turbulence: collision-side
 * modeling beyond the filtered Boltzmann equation", arXiv 2605.19796).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of the paper's lattice algorithm that the CUDA library is
 * checked against.  It shares no code, header, table or constant with the
 * CUDA path; only tests, the package's smoke check and the benchmark's CPU
 * baseline may load it.
 *
 * Every function cites the passage it follows.  Arithmetic is IEEE double,
 * compiled with -ffp-contract=off; every sum runs over the populations in the
 * lattice's canonical order (index i below), cells in x-fastest order.
 *
 * Canonical lattice order (an interface shared with the CUDA library through
 * the public header's documentation, implemented here independently):
 *   D3Q27: i = 9*(cz+1) + 3*(cy+1) + (cx+1) for c in {-1,0,1}^3
 *   D3Q19: the same enumeration with the 8 corner velocities (|c|^2 = 3) left out.
 * Population arrays are structure-of-arrays [box][q][z][y][x], x fastest.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - D3Q19 uses the standard second-order Hermite equilibrium (the paper
 *     defines D3Q27 only, App. F "Velocity space discretization").
 *   - k_sgs divides by rho_0 = 1, as in Eq. (omega_sgs_operational).
 *   - The clip selects the molecular rate itself when nu_t <= nu, so the
 *     resolved-BGK limit uses the identical omega_hat value.
 *   - H:m is the full double sum over alpha, beta.
 *   - Bounce-back walls (channel) use halfway bounce-back; at the first and
 *     last fluid layers the gradient uses the one-sided formulas of
 *     Eqs. (fd_boundary_lower/upper).
 *   - Body force (channel only): Guo forcing with the molecular omega_hat in
 *     the source prefactor; u = (sum f xi + F/2)/rho.
 *
 * Parity pins live in tests/test_oracle_*.py (lattice quadrature identities,
 * equilibrium moments and the D1Q3 closed form, brute-force moments,
 * finite-difference exactness on quadratics, carrier moment identities,
 * conservation, resolved-BGK limit, shear-wave and 2D Taylor-Green decay).
 * KC-RR (App. F.4) pins: the recombination at omega_s = omega (BGK of the
 * full D3Q27 representation) and conservation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_THETA (1.0 / 3.0) /* theta_R = c_l^2 = 1/3, App. F */

enum { ORC_BGK = 0, ORC_KCMP = 1, ORC_KCRB_HERMITE = 2, ORC_KCRB_RAW = 3, ORC_KCRR = 4 };

/* ------------------------------------------------------------------ */
/* Lattice (App. F, "Velocity space discretization"; Eq. discrete_equilibrium
 * for the D1Q3 weights 2/3 and 1/6).                                  */
/* ------------------------------------------------------------------ */
typedef struct {
    int q;
    int c[27][3];
    double w[27];
    int opp[27];
} orc_lattice;

static double orc_w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

int orc_lattice_init(int q, orc_lattice* L)
{
    if (q != 19 && q != 27) return -1;
    L->q = q;
    int n = 0;
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int s = abs(cx) + abs(cy) + abs(cz);
                if (q == 19 && s == 3) continue;
                L->c[n][0] = cx;
                L->c[n][1] = cy;
                L->c[n][2] = cz;
                if (q == 27)
                    L->w[n] = orc_w1d(cx) * orc_w1d(cy) * orc_w1d(cz);
                else
                    L->w[n] = (s == 0) ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                ++n;
            }
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
    return 0;
}

/* exported copy of the tables, for the quadrature pins */
int orc_lattice_tables(int q, int* c_out /*[q*3]*/, double* w_out /*[q]*/, int* opp_out /*[q]*/)
{
    orc_lattice L;
    if (orc_lattice_init(q, &L)) return -1;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) c_out[3 * i + a] = L.c[i][a];
        w_out[i] = L.w[i];
        opp_out[i] = L.opp[i];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Equilibrium, Eq. (discrete_equilibrium) for D3Q27:
 *   f0_i = w_i rho prod_a (1 + c_ia u_a/theta + (c_ia^2 - theta) u_a^2/(2 theta^2)).
 * D3Q19 (reading): w_i rho (1 + c.u/theta + (c.u)^2/(2 theta^2) - u.u/(2 theta)). */
/* ------------------------------------------------------------------ */
void orc_equilibrium_L(const orc_lattice* L, double rho, const double* u, double* feq)
{
    const double th = ORC_THETA;
    for (int i = 0; i < L->q; ++i) {
        if (L->q == 27) {
            double p = 1.0;
            for (int a = 0; a < 3; ++a) {
                double ca = (double)L->c[i][a];
                p = p * (1.0 + ca * u[a] / th + (ca * ca - th) * u[a] * u[a] / (2.0 * th * th));
            }
            feq[i] = L->w[i] * rho * p;
        } else {
            double cu = 0.0, uu = 0.0;
            for (int a = 0; a < 3; ++a) {
                cu = cu + (double)L->c[i][a] * u[a];
                uu = uu + u[a] * u[a];
            }
            feq[i] = L->w[i] * rho * (1.0 + cu / th + cu * cu / (2.0 * th * th) - uu / (2.0 * th));
        }
    }
}

int orc_equilibrium(int q, double rho, const double* u, double* feq)
{
    orc_lattice L;
    if (orc_lattice_init(q, &L)) return -1;
    orc_equilibrium_L(&L, rho, u, feq);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Macroscopic fields, App. F.1 step 1: rho = sum f_i, rho u = sum f_i c_i.
 * With a body force F (reading, channel only): rho u = sum f_i c_i + F/2. */
/* ------------------------------------------------------------------ */
static void orc_moments_L(const orc_lattice* L, const double* f, const double* F, double* rho, double* u)
{
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->q; ++i) {
        r = r + f[i];
        for (int a = 0; a < 3; ++a) m[a] = m[a] + f[i] * (double)L->c[i][a];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * F[a]) / r;
}

/* ------------------------------------------------------------------ */
/* Turbulent rate, Eq. (omega_sgs_operational):
 *   k = |tr m_sgs| / (2 rho_0), rho_0 = 1
 *   nu_eff = max(nu, C_nu Delta sqrt(k))
 *   omega_s = (nu_eff/theta + 1/2)^-1 = min(omega, (C_nu Delta sqrt k/theta + 1/2)^-1)  */
/* ------------------------------------------------------------------ */
double orc_omega_sgs(double tr_msgs, double nu, double omega, double c_nu, double delta)
{
    const double rho0 = 1.0;
    double k = fabs(tr_msgs) / (2.0 * rho0);
    double nu_t = c_nu * delta * sqrt(k);
    if (nu_t > nu) return 1.0 / (nu_t / ORC_THETA + 0.5);
    return omega;
}

/* H_{i ab} = c_ia c_ib - theta delta_ab, Eq. (discrete_second_order_hermite) */
static double orc_H(const orc_lattice* L, int i, int a, int b)
{
    return (double)L->c[i][a] * (double)L->c[i][b] - (a == b ? ORC_THETA : 0.0);
}

/* ------------------------------------------------------------------ */
/* KC-RR pieces, App. F.4.  The 17 high-order components of B_high, each a
 * triple of directional degrees (nx, ny, nz) in {0,1,2}.  The directional
 * Hermite factors are H_a^0 = 1, H_a^1 = c_a, H_a^2 = c_a^2 - theta.       */
/* ------------------------------------------------------------------ */
static const int orc_rr_modes[17][3] = {
    /* third order: xxy, xxz, yyz, xyy, xzz, yzz, xyz */
    {2, 1, 0}, {2, 0, 1}, {0, 2, 1}, {1, 2, 0}, {1, 0, 2}, {0, 1, 2}, {1, 1, 1},
    /* fourth order: xxyy, xxzz, yyzz, xxyz, xyyz, xyzz */
    {2, 2, 0}, {2, 0, 2}, {0, 2, 2}, {2, 1, 1}, {1, 2, 1}, {1, 1, 2},
    /* fifth order: xxyyz, xxyzz, xyyzz */
    {2, 2, 1}, {2, 1, 2}, {1, 2, 2},
    /* sixth order: xxyyzz */
    {2, 2, 2}};

static double orc_hdir(int c, int deg)
{
    if (deg == 0) return 1.0;
    if (deg == 1) return (double)c;
    return (double)(c * c) - ORC_THETA;
}

/* Recursive-regularised coefficient a^rr for a mode given as a multiset of
 * axes, Eq. (kcrr_rr):
 *   a^rr_{a1..an} = u_{an} a^rr_{a1..a(n-1)} + (1/rho) sum_{i=1}^{n-1} a0_{a1..a(n-1) without ai} a^rr_{ai an}
 * with a0 the equilibrium Hermite coefficients in the isothermal case,
 * a0_{a1..am} = rho u_a1 ... u_am (App. E with theta~ = theta_R), and the
 * second-order seed a^rr_{ab} = m^CE_{ab}.                                  */
static double orc_rr_coef(const int* ax, int n, double rho, const double* u, const double mce[3][3])
{
    if (n == 2) return mce[ax[0]][ax[1]];
    int an = ax[n - 1];
    double r = u[an] * orc_rr_coef(ax, n - 1, rho, u, mce);
    for (int i = 0; i < n - 1; ++i) {
        /* a0 over the n-2 indices {a1..a(n-1)} \ {ai}: rho * prod u */
        double a0 = rho;
        for (int j = 0; j < n - 1; ++j)
            if (j != i) a0 = a0 * u[ax[j]];
        r = r + (1.0 / rho) * a0 * mce[ax[i]][an];
    }
    return r;
}

/* ------------------------------------------------------------------ */
/* One-cell collision, App. F.1 steps 2, 4, 5, 6 (the strain S comes from
 * step 3, done by the caller with the neighbour velocities).
 *   BGK:  f_post = f - omega (f - f0)                                          (Sec. 7 "BGK")
 *   KC-RB: Eqs. (kcrb_operational_fone/raw_fone, kcrb_operational_fsgs,
 *          kcrb_operational_msgstrace, kcrb_operational_collision)
 *   KC-MP: App. F.3, Eq. (kcmp_operational_collision)
 *   KC-RR: App. F.4, Eqs. (kcrr_operational_second_order_collision ...
 *          kcrr_operational_post_population)
 * Guo forcing (channel reading) adds (1 - omega/2) w_i [(c_i - u)/theta + (c_i.u) c_i/theta^2].F */
/* ------------------------------------------------------------------ */
static void orc_collide_L(const orc_lattice* L, int closure, const double* f, double rho, const double* u,
                          const double S[3][3], const double* F, double nu, double omega, double c_nu,
                          double delta, double* fpost, double* omega_s_out, double* parts)
{
    const double th = ORC_THETA;
    const double tau_hat = 1.0 / omega; /* tau_hat = nu/theta + 1/2 */
    const int q = L->q;
    double feq[27], f1[27], fsgs[27];
    orc_equilibrium_L(L, rho, u, feq); /* step 2 */
    double omega_s = omega;

    if (closure == ORC_BGK) {
        for (int i = 0; i < q; ++i) fpost[i] = f[i] - omega * (f[i] - feq[i]);
    } else if (closure == ORC_KCRB_HERMITE || closure == ORC_KCRB_RAW) {
        /* step 4: f1 = -w rho tau_hat/theta H:S (or c c : S, raw form) */
        for (int i = 0; i < q; ++i) {
            double hs = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double h = (closure == ORC_KCRB_HERMITE) ? orc_H(L, i, a, b)
                                                              : (double)L->c[i][a] * (double)L->c[i][b];
                    hs = hs + h * S[a][b];
                }
            f1[i] = -L->w[i] * rho * tau_hat / th * hs;
            fsgs[i] = f[i] - feq[i] - f1[i];
        }
        double tr = 0.0;
        for (int i = 0; i < q; ++i) {
            double c2 = 0.0;
            for (int a = 0; a < 3; ++a) c2 = c2 + (double)(L->c[i][a] * L->c[i][a]);
            tr = tr + fsgs[i] * c2;
        }
        omega_s = orc_omega_sgs(tr, nu, omega, c_nu, delta); /* step 5 */
        for (int i = 0; i < q; ++i) fpost[i] = f[i] - omega * f1[i] - omega_s * fsgs[i];
    } else if (closure == ORC_KCMP || closure == ORC_KCRR) {
        double mce[3][3], mneq[3][3], msgs[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                mce[a][b] = -2.0 * rho * th * tau_hat * S[a][b];
                double s = 0.0;
                for (int i = 0; i < q; ++i)
                    s = s + (f[i] - feq[i]) * (double)L->c[i][a] * (double)L->c[i][b];
                mneq[a][b] = s;
                msgs[a][b] = mneq[a][b] - mce[a][b];
            }
        double tr = msgs[0][0] + msgs[1][1] + msgs[2][2];
        omega_s = orc_omega_sgs(tr, nu, omega, c_nu, delta);
        if (closure == ORC_KCMP) {
            for (int i = 0; i < q; ++i) {
                double hm = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) hm = hm + orc_H(L, i, a, b) * msgs[a][b];
                fsgs[i] = L->w[i] / (2.0 * th * th) * hm;
                f1[i] = (f[i] - feq[i]) - fsgs[i];
                fpost[i] = f[i] - omega * f1[i] - omega_s * fsgs[i];
            }
        } else {
            /* KC-RR, D3Q27 only: relax second-order and 17 high-order coefficients */
            double a2post[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    a2post[a][b] = (1.0 - omega) * mce[a][b] + (1.0 - omega_s) * msgs[a][b];
            double ahpost[17];
            for (int m = 0; m < 17; ++m) {
                const int* dg = orc_rr_modes[m];
                double aneq = 0.0;
                for (int i = 0; i < q; ++i)
                    aneq = aneq + (f[i] - feq[i]) * orc_hdir(L->c[i][0], dg[0]) * orc_hdir(L->c[i][1], dg[1]) *
                                      orc_hdir(L->c[i][2], dg[2]);
                int ax[6], n = 0;
                for (int a = 0; a < 3; ++a)
                    for (int k = 0; k < dg[a]; ++k) ax[n++] = a;
                double arr = orc_rr_coef(ax, n, rho, u, mce);
                double asgs = aneq - arr;
                ahpost[m] = (1.0 - omega) * arr + (1.0 - omega_s) * asgs;
            }
            for (int i = 0; i < q; ++i) {
                /* T2: 1/(2 th^2) sum_a Haa a_aa + 1/th^2 sum_{a<b} Ha Hb a_ab */
                double t2 = 0.0;
                for (int a = 0; a < 3; ++a) t2 = t2 + orc_hdir(L->c[i][a], 2) * a2post[a][a] / (2.0 * th * th);
                for (int a = 0; a < 3; ++a)
                    for (int b = a + 1; b < 3; ++b)
                        t2 = t2 + orc_hdir(L->c[i][a], 1) * orc_hdir(L->c[i][b], 1) * a2post[a][b] / (th * th);
                /* T3..T6: each mode enters with 1/(prod_a deg_a!) / theta^n */
                double th_ = 0.0;
                for (int m = 0; m < 17; ++m) {
                    const int* dg = orc_rr_modes[m];
                    int n = dg[0] + dg[1] + dg[2];
                    double fact = 1.0;
                    for (int a = 0; a < 3; ++a)
                        if (dg[a] == 2) fact = fact * 2.0;
                    double h = orc_hdir(L->c[i][0], dg[0]) * orc_hdir(L->c[i][1], dg[1]) * orc_hdir(L->c[i][2], dg[2]);
                    th_ = th_ + h * ahpost[m] / (fact * pow(th, (double)n));
                }
                fpost[i] = feq[i] + L->w[i] * (t2 + th_);
            }
        }
    }
    if (parts) {
        /* parts = [f0 | f1 | f_sgs], each q long (BGK: f1 = f - f0, f_sgs = 0;
         * KC-RR: the KC-MP second-order split, which it shares) */
        for (int i = 0; i < q; ++i) {
            parts[i] = feq[i];
            if (closure == ORC_BGK) {
                parts[q + i] = f[i] - feq[i];
                parts[2 * q + i] = 0.0;
            } else if (closure == ORC_KCRR) {
                double hm = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        double s = 0.0;
                        for (int j = 0; j < q; ++j)
                            s = s + (f[j] - feq[j]) * (double)L->c[j][a] * (double)L->c[j][b];
                        hm = hm + orc_H(L, i, a, b) * (s - (-2.0 * rho * th * tau_hat * S[a][b]));
                    }
                parts[2 * q + i] = L->w[i] / (2.0 * th * th) * hm;
                parts[q + i] = (f[i] - feq[i]) - parts[2 * q + i];
            } else {
                parts[q + i] = f1[i];
                parts[2 * q + i] = fsgs[i];
            }
        }
    }
    if (F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0) {
        for (int i = 0; i < q; ++i) {
            double cu = 0.0;
            for (int a = 0; a < 3; ++a) cu = cu + (double)L->c[i][a] * u[a];
            double s = 0.0;
            for (int a = 0; a < 3; ++a)
                s = s + (((double)L->c[i][a] - u[a]) / th + cu * (double)L->c[i][a] / (th * th)) * F[a];
            fpost[i] = fpost[i] + (1.0 - 0.5 * omega) * L->w[i] * s;
        }
    }
    if (omega_s_out) *omega_s_out = omega_s;
}

/* exported single-cell collision (for the identity pins) */
int orc_collide_cell(int q, int closure, const double* f, const double* S9, const double* F, double nu,
                     double c_nu, double delta, double* fpost, double* omega_s_out)
{
    orc_lattice L;
    if (orc_lattice_init(q, &L)) return -1;
    if (closure == ORC_KCRR && q != 27) return -6;
    double S[3][3], rho, u[3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[a][b] = S9[3 * a + b];
    orc_moments_L(&L, f, F, &rho, u);
    double omega = 1.0 / (nu / ORC_THETA + 0.5);
    orc_collide_L(&L, closure, f, rho, u, S, F, nu, omega, c_nu, delta, fpost, omega_s_out, NULL);
    return 0;
}

/* exported: the closure's intermediate populations of one cell,
 * parts = [f0 | f1 | f_sgs] (3q values), and omega_s */
int orc_closure_parts(int q, int closure, const double* f, const double* S9, double nu, double c_nu, double delta,
                      double* parts, double* omega_s_out)
{
    orc_lattice L;
    if (orc_lattice_init(q, &L)) return -1;
    if (closure == ORC_KCRR && q != 27) return -6;
    double S[3][3], rho, u[3], fpost[27];
    const double F[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[a][b] = S9[3 * a + b];
    orc_moments_L(&L, f, F, &rho, u);
    double omega = 1.0 / (nu / ORC_THETA + 0.5);
    orc_collide_L(&L, closure, f, rho, u, S, F, nu, omega, c_nu, delta, fpost, omega_s_out, parts);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Grid helpers                                                        */
/* ------------------------------------------------------------------ */
typedef struct {
    int q, nx, ny, nz;
    int closure;
    int bc[3]; /* 0 periodic, 1 halfway bounce-back walls on both faces */
    double nu, c_nu, delta;
    double F[3];
} orc_params;

static size_t orc_cell(const orc_params* P, int x, int y, int z)
{
    return ((size_t)z * (size_t)P->ny + (size_t)y) * (size_t)P->nx + (size_t)x;
}

static int orc_wrap(int a, int n) { return ((a % n) + n) % n; }

/* ------------------------------------------------------------------ */
/* Strain rate, App. F.1 step 3, Eqs. (fd), (strain_rate_discrete),
 * (fd_boundary_lower), (fd_boundary_upper).  u is [3][N].             */
/* ------------------------------------------------------------------ */
static double orc_u_at(const orc_params* P, const double* u, int comp, int x, int y, int z)
{
    size_t N = (size_t)P->nx * P->ny * P->nz;
    return u[(size_t)comp * N + orc_cell(P, x, y, z)];
}

static void orc_strain_at(const orc_params* P, const double* u, int x, int y, int z, double S[3][3])
{
    int n[3] = {P->nx, P->ny, P->nz};
    int p[3] = {x, y, z};
    double du[3][3]; /* du[a][b] = d_a u_b */
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
            int pp[3] = {p[0], p[1], p[2]};
            if (P->bc[a] == 0 || (p[a] > 0 && p[a] < n[a] - 1)) {
                /* central, Eq. (fd) */
                int q1[3] = {pp[0], pp[1], pp[2]}, q2[3] = {pp[0], pp[1], pp[2]};
                q1[a] = orc_wrap(p[a] + 1, n[a]);
                q2[a] = orc_wrap(p[a] - 1, n[a]);
                du[a][b] = (orc_u_at(P, u, b, q1[0], q1[1], q1[2]) - orc_u_at(P, u, b, q2[0], q2[1], q2[2])) / 2.0;
            } else if (p[a] == 0) {
                /* lower boundary, Eq. (fd_boundary_lower) */
                int q1[3] = {pp[0], pp[1], pp[2]}, q2[3] = {pp[0], pp[1], pp[2]};
                q1[a] = 1;
                q2[a] = 2;
                du[a][b] = (-3.0 * orc_u_at(P, u, b, pp[0], pp[1], pp[2]) + 4.0 * orc_u_at(P, u, b, q1[0], q1[1], q1[2]) -
                            orc_u_at(P, u, b, q2[0], q2[1], q2[2])) /
                           2.0;
            } else {
                /* upper boundary, Eq. (fd_boundary_upper) */
                int q1[3] = {pp[0], pp[1], pp[2]}, q2[3] = {pp[0], pp[1], pp[2]};
                q1[a] = n[a] - 2;
                q2[a] = n[a] - 3;
                du[a][b] = (3.0 * orc_u_at(P, u, b, pp[0], pp[1], pp[2]) - 4.0 * orc_u_at(P, u, b, q1[0], q1[1], q1[2]) +
                            orc_u_at(P, u, b, q2[0], q2[1], q2[2])) /
                           2.0;
            }
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[a][b] = 0.5 * (du[b][a] + du[a][b]); /* Eq. (strain_rate_discrete) */
}

/* exported: strain field of a velocity field u[3][N] -> S[9][N] */
int orc_strain_field(int nx, int ny, int nz, const int* bc, const double* u, double* S_out)
{
    orc_params P;
    memset(&P, 0, sizeof(P));
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    for (int a = 0; a < 3; ++a) P.bc[a] = bc[a];
    size_t N = (size_t)nx * ny * nz;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double S[3][3];
                orc_strain_at(&P, u, x, y, z, S);
                for (int k = 0; k < 9; ++k) S_out[(size_t)k * N + orc_cell(&P, x, y, z)] = S[k / 3][k % 3];
            }
    return 0;
}

/* ------------------------------------------------------------------ */
/* One full time step, App. F.1 steps 1-7 (collide-then-stream written in
 * pull form: the array holds post-collision populations; the step first
 * streams them, Eq. (streaming), then collides at every node).
 * Pass 1: pull-stream into fpre and compute rho, u at every node.
 * Pass 2: strain from the stored u, then equilibrium, closure, collision. */
/* ------------------------------------------------------------------ */
/* pass 1 of a step: pull-stream fin into fpre (Eq. streaming; halfway
 * bounce-back on wall axes) and compute rho, u at every node (step 1) */
static void orc_stream_moments(const orc_params* P, const orc_lattice* L, const double* fin, double* fpre, double* rho,
                               double* u)
{
    const int q = L->q, nx = P->nx, ny = P->ny, nz = P->nz;
    const size_t N = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t cidx = orc_cell(P, x, y, z);
                double f[27];
                for (int i = 0; i < q; ++i) {
                    int s[3] = {x - L->c[i][0], y - L->c[i][1], z - L->c[i][2]};
                    int n3[3] = {nx, ny, nz};
                    int solid = 0;
                    for (int a = 0; a < 3; ++a) {
                        if (P->bc[a] == 1) {
                            if (s[a] < 0 || s[a] >= n3[a]) solid = 1;
                        } else {
                            s[a] = orc_wrap(s[a], n3[a]);
                        }
                    }
                    if (solid) /* halfway bounce-back: the population leaving x towards the wall returns */
                        f[i] = fin[(size_t)L->opp[i] * N + cidx];
                    else
                        f[i] = fin[(size_t)i * N + orc_cell(P, s[0], s[1], s[2])];
                    fpre[(size_t)i * N + cidx] = f[i];
                }
                double r, uu[3];
                orc_moments_L(L, f, P->F, &r, uu);
                rho[cidx] = r;
                for (int a = 0; a < 3; ++a) u[(size_t)a * N + cidx] = uu[a];
            }
    }
}

static void orc_step_once(const orc_params* P, const orc_lattice* L, const double* fin, double* fout, double* fpre,
                          double* rho, double* u)
{
    const int q = L->q, nx = P->nx, ny = P->ny, nz = P->nz;
    const size_t N = (size_t)nx * ny * nz;
    const double omega = 1.0 / (P->nu / ORC_THETA + 0.5); /* Eq. (omega_t_discrete) */

    /* pass 1: stream + moments */
    orc_stream_moments(P, L, fin, fpre, rho, u);
    /* pass 2: gradient + closure + collision */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t cidx = orc_cell(P, x, y, z);
                double f[27], fp[27], S[3][3], uu[3];
                for (int i = 0; i < q; ++i) f[i] = fpre[(size_t)i * N + cidx];
                for (int a = 0; a < 3; ++a) uu[a] = u[(size_t)a * N + cidx];
                orc_strain_at(P, u, x, y, z, S);
                orc_collide_L(L, P->closure, f, rho[cidx], uu, S, P->F, P->nu, omega, P->c_nu, P->delta, fp, NULL, NULL);
                for (int i = 0; i < q; ++i) fout[(size_t)i * N + cidx] = fp[i];
            }
    }
}

static int orc_fill_params(orc_params* P, int q, int nx, int ny, int nz, int closure, const int* bc, double nu,
                           double c_nu, double delta, const double* F)
{
    memset(P, 0, sizeof(*P));
    if ((q != 19 && q != 27) || nx < 1 || ny < 1 || nz < 1) return -1;
    if (closure < 0 || closure > 4) return -1;
    if (closure == ORC_KCRR && q != 27) return -6;
    P->q = q;
    P->nx = nx;
    P->ny = ny;
    P->nz = nz;
    P->closure = closure;
    for (int a = 0; a < 3; ++a) {
        P->bc[a] = bc ? bc[a] : 0;
        P->F[a] = F ? F[a] : 0.0;
        int n = a == 0 ? nx : (a == 1 ? ny : nz);
        if (P->bc[a] == 1 && n < 3) return -1; /* one-sided stencils need 3 layers */
    }
    P->nu = nu;
    P->c_nu = c_nu;
    P->delta = delta;
    return 0;
}

/* Advance f (in place, [q][N]) by nsteps.  Returns 0 on success. */
int orc_run(int q, int nx, int ny, int nz, int closure, const int* bc, double nu, double c_nu, double delta,
            const double* F, double* f, int nsteps)
{
    orc_params P;
    int rc = orc_fill_params(&P, q, nx, ny, nz, closure, bc, nu, c_nu, delta, F);
    if (rc) return rc;
    orc_lattice L;
    orc_lattice_init(q, &L);
    size_t N = (size_t)nx * ny * nz;
    double* fout = (double*)malloc(sizeof(double) * q * N);
    double* fpre = (double*)malloc(sizeof(double) * q * N);
    double* rho = (double*)malloc(sizeof(double) * N);
    double* u = (double*)malloc(sizeof(double) * 3 * N);
    if (!fout || !fpre || !rho || !u) {
        free(fout);
        free(fpre);
        free(rho);
        free(u);
        return -2;
    }
    for (int s = 0; s < nsteps; ++s) {
        orc_step_once(&P, &L, f, fout, fpre, rho, u);
        memcpy(f, fout, sizeof(double) * q * N);
    }
    free(fout);
    free(fpre);
    free(rho);
    free(u);
    return 0;
}

/* Post-collision populations of ONE cell (x,y,z) after one step, computed
 * from a local block of the pre-step array.  blk holds populations
 * [q][5][5][5] for cells (x+dx, y+dy, z+dz), dx,dy,dz in -2..2, already
 * wrapped periodically by the caller (periodic axes only).  This is the
 * same algorithm as orc_step_once restricted to one output cell; it lets
 * tests check sampled cells of lattices too large for the full oracle. */
int orc_step_cell(int q, int closure, double nu, double c_nu, double delta, const double* blk, double* fpost_out)
{
    orc_lattice L;
    if (orc_lattice_init(q, &L)) return -1;
    if (closure == ORC_KCRR && q != 27) return -6;
    const double omega = 1.0 / (nu / ORC_THETA + 0.5);
    const double F[3] = {0.0, 0.0, 0.0};
    /* streamed populations, rho and u at the 3x3x3 cells around the centre */
    double fc[27], rho_c = 0.0, u3[3][3][3][3];
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                double f[27];
                for (int i = 0; i < q; ++i) {
                    int sx = dx - L.c[i][0] + 2, sy = dy - L.c[i][1] + 2, sz = dz - L.c[i][2] + 2;
                    f[i] = blk[(size_t)i * 125 + (size_t)(sz * 25 + sy * 5 + sx)];
                }
                double r, uu[3];
                orc_moments_L(&L, f, F, &r, uu);
                for (int a = 0; a < 3; ++a) u3[dz + 1][dy + 1][dx + 1][a] = uu[a];
                if (dx == 0 && dy == 0 && dz == 0) {
                    for (int i = 0; i < q; ++i) fc[i] = f[i];
                    rho_c = r;
                }
            }
    double du[3][3];
    for (int b = 0; b < 3; ++b) {
        du[0][b] = (u3[1][1][2][b] - u3[1][1][0][b]) / 2.0;
        du[1][b] = (u3[1][2][1][b] - u3[1][0][1][b]) / 2.0;
        du[2][b] = (u3[2][1][1][b] - u3[0][1][1][b]) / 2.0;
    }
    double S[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[a][b] = 0.5 * (du[b][a] + du[a][b]);
    orc_collide_L(&L, closure, fc, rho_c, u3[1][1][1], S, F, nu, omega, c_nu, delta, fpost_out, NULL, NULL);
    return 0;
}

/* Equilibrium initialisation f_i = f0_i(rho, u) at every node (Eq. discrete_equilibrium).
 * rho may be NULL (rho = 1).  u is [3][N]. */
int orc_init_equilibrium(int q, int nx, int ny, int nz, const double* rho, const double* u, double* f)
{
    orc_lattice L;
    if (orc_lattice_init(q, &L)) return -1;
    size_t N = (size_t)nx * ny * nz;
    for (size_t c = 0; c < N; ++c) {
        double uu[3] = {u[c], u[N + c], u[2 * N + c]}, feq[27];
        orc_equilibrium_L(&L, rho ? rho[c] : 1.0, uu, feq);
        for (int i = 0; i < q; ++i) f[(size_t)i * N + c] = feq[i];
    }
    return 0;
}

/* Macroscopic fields of a stored (post-collision) population array, App. F.1
 * step 1.  With Guo forcing the collision adds the full impulse F to sum f c,
 * so the velocity of time n is (sum f c - F/2)/rho: the moments are taken
 * with the force -F. */
int orc_fields(int q, int nx, int ny, int nz, const double* F, const double* f, double* rho, double* u)
{
    orc_lattice L;
    if (orc_lattice_init(q, &L)) return -1;
    double mF[3] = {0.0, 0.0, 0.0};
    if (F)
        for (int a = 0; a < 3; ++a) mF[a] = -F[a];
    size_t N = (size_t)nx * ny * nz;
    for (size_t c = 0; c < N; ++c) {
        double fc[27], r, uu[3];
        for (int i = 0; i < q; ++i) fc[i] = f[(size_t)i * N + c];
        orc_moments_L(&L, fc, mF, &r, uu);
        rho[c] = r;
        for (int a = 0; a < 3; ++a) u[(size_t)a * N + c] = uu[a];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Diagnostics, Sec. 7.1, Eq. (tgv_energy_enstrophy): arithmetic averages of
 * (1/2) rho |u|^2 and (1/2)|curl u|^2 over the nodes; the curl uses the
 * sixth-order centred stencil on periodic axes (on wall axes the
 * second-order stencils of App. F.1 step 3).
 * out: [0] mass sum, [1..3] momentum sums, [4] E_k, [5] enstrophy,
 *      [6] number of non-finite rho/u values                           */
/* ------------------------------------------------------------------ */
static double orc_d1(const orc_params* P, const double* u, int comp, int axis, int x, int y, int z)
{
    int n[3] = {P->nx, P->ny, P->nz}, p[3] = {x, y, z};
    if (P->bc[axis] == 0) {
        static const double c6[3] = {45.0 / 60.0, -9.0 / 60.0, 1.0 / 60.0};
        double s = 0.0;
        for (int k = 1; k <= 3; ++k) {
            int a1[3] = {x, y, z}, a2[3] = {x, y, z};
            a1[axis] = orc_wrap(p[axis] + k, n[axis]);
            a2[axis] = orc_wrap(p[axis] - k, n[axis]);
            s = s + c6[k - 1] * (orc_u_at(P, u, comp, a1[0], a1[1], a1[2]) - orc_u_at(P, u, comp, a2[0], a2[1], a2[2]));
        }
        return s;
    }
    int a1[3] = {x, y, z}, a2[3] = {x, y, z}, a0[3] = {x, y, z};
    if (p[axis] > 0 && p[axis] < n[axis] - 1) {
        a1[axis] = p[axis] + 1;
        a2[axis] = p[axis] - 1;
        return (orc_u_at(P, u, comp, a1[0], a1[1], a1[2]) - orc_u_at(P, u, comp, a2[0], a2[1], a2[2])) / 2.0;
    } else if (p[axis] == 0) {
        a1[axis] = 1;
        a2[axis] = 2;
        return (-3.0 * orc_u_at(P, u, comp, a0[0], a0[1], a0[2]) + 4.0 * orc_u_at(P, u, comp, a1[0], a1[1], a1[2]) -
                orc_u_at(P, u, comp, a2[0], a2[1], a2[2])) /
               2.0;
    }
    a1[axis] = n[axis] - 2;
    a2[axis] = n[axis] - 3;
    return (3.0 * orc_u_at(P, u, comp, a0[0], a0[1], a0[2]) - 4.0 * orc_u_at(P, u, comp, a1[0], a1[1], a1[2]) +
            orc_u_at(P, u, comp, a2[0], a2[1], a2[2])) /
           2.0;
}

int orc_diagnostics(int q, int nx, int ny, int nz, const int* bc, const double* F, const double* f, double* out)
{
    orc_params P;
    int rc = orc_fill_params(&P, q, nx, ny, nz, 0, bc, 0.0, 0.0, 1.0, F);
    if (rc) return rc;
    size_t N = (size_t)nx * ny * nz;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* u = (double*)malloc(sizeof(double) * 3 * N);
    if (!rho || !u) {
        free(rho);
        free(u);
        return -2;
    }
    orc_fields(q, nx, ny, nz, F, f, rho, u);
    double mass = 0.0, mom[3] = {0.0, 0.0, 0.0}, ek = 0.0, zz = 0.0, bad = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t c = orc_cell(&P, x, y, z);
                double r = rho[c], ux = u[c], uy = u[N + c], uz = u[2 * N + c];
                if (!isfinite(r) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz)) bad = bad + 1.0;
                mass = mass + r;
                mom[0] = mom[0] + r * ux;
                mom[1] = mom[1] + r * uy;
                mom[2] = mom[2] + r * uz;
                ek = ek + 0.5 * r * (ux * ux + uy * uy + uz * uz);
                double wx = orc_d1(&P, u, 2, 1, x, y, z) - orc_d1(&P, u, 1, 2, x, y, z);
                double wy = orc_d1(&P, u, 0, 2, x, y, z) - orc_d1(&P, u, 2, 0, x, y, z);
                double wz = orc_d1(&P, u, 1, 0, x, y, z) - orc_d1(&P, u, 0, 1, x, y, z);
                zz = zz + 0.5 * (wx * wx + wy * wy + wz * wz);
            }
    out[0] = mass;
    out[1] = mom[0];
    out[2] = mom[1];
    out[3] = mom[2];
    out[4] = ek / (double)N;
    out[5] = zz / (double)N;
    out[6] = bad;
    out[7] = 0.0;
    free(rho);
    free(u);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Dissipation rates of a pre-collision state (a reading: the paper reports
 * E_k and enstrophy, Sec. 7.1, and is silent on the dissipation).  At every
 * node, with rho, u (step 1), S (step 3, Eqs. fd, fd_boundary_lower/upper,
 * strain_rate_discrete) and the closure's clipped rate omega_s (step 5, Eq.
 * omega_sgs_operational; omega for BGK), the effective viscosity is
 * nu_eff = theta (1/omega_s - 1/2), the viscosity the two-rate relaxation
 * applies to the SGS part; then
 *   out[0] = < 2 rho nu_eff S:S >,   out[1] = < 2 rho nu S:S >
 * (arithmetic averages over the nodes, S:S = sum_ab S_ab^2).              */
/* ------------------------------------------------------------------ */
static void orc_dissipation_core(const orc_params* P, const orc_lattice* L, const double* fpre, const double* rho,
                                 const double* u, double* out)
{
    const int q = L->q, nx = P->nx, ny = P->ny, nz = P->nz;
    const size_t N = (size_t)nx * ny * nz;
    const double omega = 1.0 / (P->nu / ORC_THETA + 0.5);
    double e_eff = 0.0, e_mol = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t cidx = orc_cell(P, x, y, z);
                double f[27], fp[27], S[3][3], uu[3], omega_s;
                for (int i = 0; i < q; ++i) f[i] = fpre[(size_t)i * N + cidx];
                for (int a = 0; a < 3; ++a) uu[a] = u[(size_t)a * N + cidx];
                orc_strain_at(P, u, x, y, z, S);
                orc_collide_L(L, P->closure, f, rho[cidx], uu, S, P->F, P->nu, omega, P->c_nu, P->delta, fp, &omega_s,
                              NULL);
                double ss = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) ss = ss + S[a][b] * S[a][b];
                double nu_eff = ORC_THETA * (1.0 / omega_s - 0.5);
                e_eff = e_eff + 2.0 * rho[cidx] * nu_eff * ss;
                e_mol = e_mol + 2.0 * rho[cidx] * P->nu * ss;
            }
    out[0] = e_eff / (double)N;
    out[1] = e_mol / (double)N;
}

/* exported: dissipation rates of the pre-collision state fpre [q][N] */
int orc_dissipation_pre(int q, int nx, int ny, int nz, int closure, const int* bc, double nu, double c_nu,
                        double delta, const double* F, const double* fpre, double* out)
{
    orc_params P;
    int rc = orc_fill_params(&P, q, nx, ny, nz, closure, bc, nu, c_nu, delta, F);
    if (rc) return rc;
    orc_lattice L;
    orc_lattice_init(q, &L);
    size_t N = (size_t)nx * ny * nz;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* u = (double*)malloc(sizeof(double) * 3 * N);
    if (!rho || !u) {
        free(rho);
        free(u);
        return -2;
    }
    for (size_t c = 0; c < N; ++c) {
        double f[27], r, uu[3];
        for (int i = 0; i < q; ++i) f[i] = fpre[(size_t)i * N + c];
        orc_moments_L(&L, f, P.F, &r, uu);
        rho[c] = r;
        for (int a = 0; a < 3; ++a) u[(size_t)a * N + c] = uu[a];
    }
    orc_dissipation_core(&P, &L, fpre, rho, u, out);
    free(rho);
    free(u);
    return 0;
}

/* exported: dissipation rates of the state the next step collides, i.e. of
 * the stored post-collision populations f [q][N] after pull streaming */
int orc_dissipation(int q, int nx, int ny, int nz, int closure, const int* bc, double nu, double c_nu, double delta,
                    const double* F, const double* f, double* out)
{
    orc_params P;
    int rc = orc_fill_params(&P, q, nx, ny, nz, closure, bc, nu, c_nu, delta, F);
    if (rc) return rc;
    orc_lattice L;
    orc_lattice_init(q, &L);
    size_t N = (size_t)nx * ny * nz;
    double* fpre = (double*)malloc(sizeof(double) * q * N);
    double* rho = (double*)malloc(sizeof(double) * N);
    double* u = (double*)malloc(sizeof(double) * 3 * N);
    if (!fpre || !rho || !u) {
        free(fpre);
        free(rho);
        free(u);
        return -2;
    }
    orc_stream_moments(&P, &L, f, fpre, rho, u);
    orc_dissipation_core(&P, &L, fpre, rho, u, out);
    free(fpre);
    free(rho);
    free(u);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
