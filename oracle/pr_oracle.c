/*
 * Plain FP64 CPU oracle for the real-fluid property evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline / reference arm load this library.  The CUDA library
 * shares no code, header, table or constant with it: every constant below is
 * written here on its own, and the species data arrive as arguments.
 *
 * What it computes, per cell (T, p, Y_1..Y_N), following the paper's Sec. 2
 * (Eq. 1 and the text after it) and the published methods that the paper
 * delegates to Cantera:
 *   1. mole fractions X_k and mean molar mass;
 *   2. Peng-Robinson pure-species a_c, b (Eq. 1 constants, taken at their exact
 *      critical-point values; the printed 0.45724 / 0.07780 are their roundings)
 *      and the PR-1976 alpha(T, omega);
 *   3. van der Waals one-fluid mixing a_m = sum_i sum_j X_i X_j (1-k_ij)
 *      sqrt(a_i a_j), b_m = sum X_i b_i, with first and second T-derivatives,
 *      as the plain double sum;
 *   4. all real roots of the PR cubic in Z by bracketing + bisection, the
 *      physical root being the one with Z > B and least residual Gibbs energy;
 *   5. density, departure enthalpy and heat capacity on NASA-7 ideal-gas terms;
 *   6. Chung et al. (1988) dense-fluid viscosity and conductivity with Chung's
 *      mixture corresponding-states rules (the paper's "modified Chung's
 *      transport model", Sec. 2);
 *   7. the inversion T(h, p, Y) by a safeguarded Newton iteration.
 * Nothing is blocked, fused or factorised beyond these definitions.
 *
 * Parity pins (tests, CPU only): Z_c of a pure species at its critical point,
 * the low-pressure (ideal-gas) limit, cp against the finite-difference dh/dT,
 * all cubic roots against high-precision polynomial roots and brute-force sign
 * scans, T(h(T)) = T, mixing invariances, the dilute limit of the Chung
 * correlations, and the paper's Table 1 kinematic viscosity of LOX.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of one batch call: nthreads when positive, else the OpenMP default.
 * Given per loop (num_threads clause), so a one-thread call leaves the
 * default of later calls unchanged. */
static int orc_threads(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

#define ORC_R 8.314462618 /* J/(mol K) */

/* Step markers for the operation-counting build (opcount.cpp includes this
 * file with ORC_STEP defined); nothing in the oracle's own build.  Steps:
 * 1 composition, 2 species EOS terms, 3 mixing, 4 cubic roots, 5 root
 * selection, 6 ideal gas, 7 departures, 8 Chung mixture rules, 9 Chung
 * dense correlation, 10 output assembly, 0 diagnostics (not the method). */
#ifndef ORC_STEP
#define ORC_STEP(s) ((void)0)
#endif

/* Species data, all arrays of length N (nasa_*: N x 7, kij: N x N or NULL). */
typedef struct {
    int32_t N;
    int32_t transport_rule;     /* 0: Chung mixture rules; 1: mole-fraction average of pure-species Chung viscosity */
    int32_t printed_constants;  /* 1: use the printed 0.45724 / 0.07780 instead of the exact values */
    int32_t pad;
    const double *W;            /* g/mol */
    const double *Tc, *pc, *omega, *Vc; /* K, Pa, -, cm^3/mol */
    const double *dipole, *kappa;       /* debye, - */
    const double *nasa_lo, *nasa_hi;    /* N x 7 */
    const double *T_mid;                /* K */
    const double *kij;                  /* N x N or NULL (zero) */
} orc_species;

/* Per-cell diagnostics for the tests. */
typedef struct {
    double Wbar;                 /* kg/mol */
    double am, dam, d2am, bm;    /* mixture a, da/dT, d2a/dT2 (J m^3/mol^2), b (m^3/mol) */
    double A, B;                 /* dimensionless cubic parameters */
    double roots[3];             /* all real roots, ascending */
    int32_t n_roots;             /* number of real roots */
    int32_t n_phys;              /* roots with Z > B */
    double Z;                    /* selected root */
    double gres_gap;             /* |g1 - g2| between the two best physical roots (or +inf) */
    double cond;                 /* root condition number */
    double h_ig, cp_ig, cv_ig_molar; /* J/kg, J/(kg K), J/(mol K) */
    double h_dep, cp_dep;        /* J/mol, J/(mol K) */
    double dpdT, dpdV;           /* (dp/dT)_V, (dp/dV)_T */
    double mu_dilute, lambda_dilute; /* Pa s, W/(m K): the y -> 0 limit of the dense forms */
    /* cancellation ratios sum|t_i| / |sum t_i| of the sums in Chung's dense
     * viscosity (G2's numerator and denominator, 1/G2 + E6 y, the two eta*
     * terms) and conductivity (the same of H2, 1/H2 + B6 y, the two lambda
     * terms): the factor by which rounding errors of the terms grow in them */
    double cancel_mu, cancel_lam;
} orc_diag;

enum { ORC_OK = 0, ORC_NEWTON_MAXIT = 1, ORC_H_OUT_OF_RANGE = 2, ORC_NO_ROOT = 3,
       ORC_BAD_INPUT = 4, ORC_AMBIGUOUS = 5 };

/* ---------------------------------------------------------------------- */
/* PR constants from the critical-point condition.  At T = Tc, p = pc the
 * cubic in Z has a triple root Z_c; matching (Z - Z_c)^3 term by term gives
 * Z_c = (1 - B_c)/3, A_c = 3 Z_c^2 + 3 B_c^2 + 2 B_c and, for B_c = Omega_b,
 * 64 x^3 + 6 x^2 + 12 x - 1 = 0.  The root is found by bisection here. */
static void orc_pr_omegas(int printed, double *Oa, double *Ob)
{
    if (printed) { *Oa = 0.45724; *Ob = 0.07780; return; }
    double lo = 0.0, hi = 0.5;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double f = ((64.0 * mid + 6.0) * mid + 12.0) * mid - 1.0;
        if (f > 0) hi = mid; else lo = mid;
    }
    double b = 0.5 * (lo + hi);
    double zc = (1.0 - b) / 3.0;
    *Ob = b;
    *Oa = 3.0 * zc * zc + 3.0 * b * b + 2.0 * b;
}

void orc_pr_constants(int printed, double *Oa, double *Ob) { orc_pr_omegas(printed, Oa, Ob); }

/* ---------------------------------------------------------------------- */
/* Cubic Z^3 + c2 Z^2 + c1 Z + c0 (Eq. 1 written in Z = pV/RT). */
static double cubic_eval(double c2, double c1, double c0, double z)
{
    return ((z + c2) * z + c1) * z + c0;
}

static double bisect_root(double c2, double c1, double c0, double lo, double hi)
{
    double flo = cubic_eval(c2, c1, c0, lo);
    if (flo == 0.0) return lo;
    double fhi = cubic_eval(c2, c1, c0, hi);
    if (fhi == 0.0) return hi;
    for (int it = 0; it < 2000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double fm = cubic_eval(c2, c1, c0, mid);
        if (fm == 0.0) return mid;
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; fhi = fm; }
    }
    double z = 0.5 * (lo + hi);
    /* two Newton polish steps, kept only if they reduce |P| */
    for (int k = 0; k < 2; ++k) {
        double f = cubic_eval(c2, c1, c0, z);
        double d = (3.0 * z + 2.0 * c2) * z + c1;
        if (d == 0.0) break;
        double zn = z - f / d;
        if (fabs(cubic_eval(c2, c1, c0, zn)) < fabs(f)) z = zn;
    }
    return z;
}

/* All real roots of Z^3 + c2 Z^2 + c1 Z + c0, ascending.  Returns their count.
 * The real line is cut at the critical points of the cubic (roots of its
 * derivative) into monotone pieces; each piece with a sign change holds one
 * root, found by bisection.  A critical point where the cubic vanishes to
 * within rounding is a double root and is reported once. */
int orc_cubic_real_roots(double c2, double c1, double c0, double roots[3])
{
    double M = 1.0 + fmax(fabs(c2), fmax(fabs(c1), fabs(c0)));  /* Cauchy bound */
    double pts[4];
    int np = 0;
    pts[np++] = -M;
    double disc = c2 * c2 - 3.0 * c1;           /* derivative 3z^2 + 2 c2 z + c1 */
    double crit[2]; int nc = 0;
    if (disc > 0) {
        double s = sqrt(disc);
        crit[0] = (-c2 - s) / 3.0;
        crit[1] = (-c2 + s) / 3.0;
        nc = 2;
        pts[np++] = crit[0];
        pts[np++] = crit[1];
    }
    pts[np++] = M;
    int n = 0;
    for (int k = 0; k + 1 < np; ++k) {
        double a = pts[k], b = pts[k + 1];
        double fa = cubic_eval(c2, c1, c0, a), fb = cubic_eval(c2, c1, c0, b);
        if ((fa < 0 && fb > 0) || (fa > 0 && fb < 0)) {
            roots[n++] = bisect_root(c2, c1, c0, a, b);
        }
    }
    /* touching roots at the critical points */
    for (int k = 0; k < nc; ++k) {
        double z = crit[k];
        double f = cubic_eval(c2, c1, c0, z);
        double scale = fabs(z * z * z) + fabs(c2 * z * z) + fabs(c1 * z) + fabs(c0);
        if (fabs(f) <= 8.0 * 2.220446049250313e-16 * scale) {
            int dup = 0;
            for (int j = 0; j < n; ++j) if (fabs(roots[j] - z) <= 1e-7 * (1.0 + fabs(z))) dup = 1;
            if (!dup && n < 3) roots[n++] = z;
        }
    }
    /* ascending */
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (roots[j] < roots[i]) { double t = roots[i]; roots[i] = roots[j]; roots[j] = t; }
    return n;
}

/* Residual Gibbs energy g = G_res/(RT) of the PR fluid at root Z. */
static double pr_gres(double Z, double A, double B)
{
    const double s2 = sqrt(2.0);
    return Z - 1.0 - log(Z - B) - A / (2.0 * s2 * B) * log((Z + (1.0 + s2) * B) / (Z + (1.0 - s2) * B));
}

double orc_pr_gres(double Z, double A, double B) { return pr_gres(Z, A, B); }

/* ---------------------------------------------------------------------- */
/* NASA-7 ideal-gas cp/R and h/(RT) of one species (two T ranges; the low set
 * below T_mid, the high set at and above it; evaluated outside [T_low,
 * T_high] by extrapolation). */
static void nasa7(const double *lo, const double *hi, double Tmid, double T, double *cpR, double *hRT, double *dcpR)
{
    const double *a = (T < Tmid) ? lo : hi;
    *cpR = a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T + a[4] * T * T * T * T;
    *hRT = a[0] + a[1] * T / 2.0 + a[2] * T * T / 3.0 + a[3] * T * T * T / 4.0 + a[4] * T * T * T * T / 5.0 + a[5] / T;
    if (dcpR) *dcpR = a[1] + 2.0 * a[2] * T + 3.0 * a[3] * T * T + 4.0 * a[4] * T * T * T;
}

/* ---------------------------------------------------------------------- */
/* Chung et al. (1988) coefficient tables: E_i = a + b*omega + c*mu_r^4 + d*kappa
 * for the viscosity (i = 1..10) and B_i for the conductivity (i = 1..7),
 * as tabulated in Poling, Prausnitz & O'Connell, Tables 9-6 and 10-3. */
static const double CHUNG_VISC[10][4] = {
    {6.324, 50.412, -51.680, 1189.0},
    {1.210e-3, -1.154e-3, -6.257e-3, 0.03728},
    {5.283, 254.209, -168.48, 3898.0},
    {6.623, 38.096, -8.464, 31.42},
    {19.745, 7.630, -14.354, 31.53},
    {-1.900, -12.537, 4.985, -18.15},
    {24.275, 3.450, -11.291, 69.35},
    {0.7972, 1.117, 0.01235, -4.117},
    {-0.2382, 0.06770, -0.8163, 4.025},
    {0.06863, 0.3479, 0.5926, -0.727},
};
static const double CHUNG_COND[7][4] = {
    {2.4166, 0.74824, -0.91858, 121.72},
    {-0.50924, -1.5094, -49.991, 69.983},
    {6.6107, 5.6207, 64.760, 27.039},
    {14.543, -8.9139, -5.6379, 74.344},
    {0.79274, 0.82019, -0.69369, 6.3173},
    {-5.8634, 12.801, 9.5893, 65.529},
    {91.089, 128.11, -54.217, 523.81},
};

/* Neufeld et al. (1972) reduced collision integral for viscosity, as used by Chung. */
static double neufeld_omega_v(double Ts)
{
    return 1.16145 * pow(Ts, -0.14874) + 0.52487 * exp(-0.77320 * Ts) + 2.16178 * exp(-2.43787 * Ts);
}

/* Corresponding-states inputs of one Chung evaluation. */
typedef struct {
    double Tc, Vc, omega, M, mur4, kappa; /* K, cm^3/mol, -, g/mol, -, - */
} chung_cs;

/* Chung dense-fluid viscosity [Pa s] and conductivity [W/(m K)] of a fluid
 * with corresponding-states parameters cs at temperature T, molar density
 * rho_mol [mol/m^3] and ideal-gas molar cv (for the conductivity). */
/* sum|t_i| / |sum t_i| of a three-term sum (1 without cancellation) */
static double cancel3(double a, double b, double c)
{
    return (fabs(a) + fabs(b) + fabs(c)) / fabs(a + b + c);
}

static void chung_dense(const chung_cs *cs, double T, double rho_mol, double cv_molar,
                        double *mu, double *lam, double *mu0, double *lam0, double *cmu, double *clam)
{
    double Ts = 1.2593 * T / cs->Tc;
    double Fc = 1.0 - 0.2756 * cs->omega + 0.059035 * cs->mur4 + cs->kappa;
    double Ov = neufeld_omega_v(Ts);
    double y = rho_mol * 1e-6 * cs->Vc / 6.0;       /* rho in mol/cm^3 */
    double G1 = (1.0 - 0.5 * y) / ((1.0 - y) * (1.0 - y) * (1.0 - y));
    double E[10];
    for (int i = 0; i < 10; ++i)
        E[i] = CHUNG_VISC[i][0] + CHUNG_VISC[i][1] * cs->omega + CHUNG_VISC[i][2] * cs->mur4 + CHUNG_VISC[i][3] * cs->kappa;
    /* (1 - exp(-E4 y))/y, with its limit E4 as y -> 0 */
    double fy4 = (y > 0) ? -expm1(-E[3] * y) / y : E[3];
    double G2 = (E[0] * fy4 + E[1] * G1 * exp(E[4] * y) + E[2] * G1) / (E[0] * E[3] + E[1] + E[2]);
    double etass = E[6] * y * y * G2 * exp(E[7] + E[8] / Ts + E[9] / (Ts * Ts));
    double etas = sqrt(Ts) / Ov * Fc * (1.0 / G2 + E[5] * y) + etass;
    double Vc23 = pow(cs->Vc, 2.0 / 3.0);
    double eta_uP = etas * 36.344 * sqrt(cs->M * cs->Tc) / Vc23;
    *mu = eta_uP * 1e-7;
    /* dilute gas viscosity (the y -> 0 limit of the dense form) */
    double eta0_uP = 40.785 * Fc * sqrt(cs->M * T) / (Vc23 * Ov);
    double eta0 = eta0_uP * 1e-7;
    *mu0 = eta0;
    /* conductivity */
    double Bc[7];
    for (int i = 0; i < 7; ++i)
        Bc[i] = CHUNG_COND[i][0] + CHUNG_COND[i][1] * cs->omega + CHUNG_COND[i][2] * cs->mur4 + CHUNG_COND[i][3] * cs->kappa;
    double fyb4 = (y > 0) ? -expm1(-Bc[3] * y) / y : Bc[3];
    double H2 = (Bc[0] * fyb4 + Bc[1] * G1 * exp(Bc[4] * y) + Bc[2] * G1) / (Bc[0] * Bc[3] + Bc[1] + Bc[2]);
    double Tr = T / cs->Tc;
    double alpha = cv_molar / ORC_R - 1.5;
    double beta = 0.7862 - 0.7109 * cs->omega + 1.3168 * cs->omega * cs->omega;
    double Zp = 2.0 + 10.5 * Tr * Tr;
    double Psi = 1.0 + alpha * ((0.215 + 0.28288 * alpha - 1.061 * beta + 0.26665 * Zp) /
                                (0.6366 + beta * Zp + 1.061 * alpha * beta));
    double Mkg = cs->M * 1e-3;
    double q = 3.586e-3 * sqrt(cs->Tc / Mkg) / Vc23;
    *lam = 31.2 * eta0 * Psi / Mkg * (1.0 / H2 + Bc[5] * y) + q * Bc[6] * y * y * sqrt(Tr) * H2;
    ORC_STEP(0);
    *lam0 = 31.2 * eta0 * Psi / Mkg;
    if (cmu) {
        double c = cancel3(E[0] * fy4, E[1] * G1 * exp(E[4] * y), E[2] * G1);
        c = fmax(c, cancel3(E[0] * E[3], E[1], E[2]));
        c = fmax(c, cancel3(1.0 / G2, E[5] * y, 0.0));
        c = fmax(c, cancel3(sqrt(Ts) / Ov * Fc * (1.0 / G2 + E[5] * y), etass, 0.0));
        *cmu = c;
    }
    if (clam) {
        double c = cancel3(Bc[0] * fyb4, Bc[1] * G1 * exp(Bc[4] * y), Bc[2] * G1);
        c = fmax(c, cancel3(Bc[0] * Bc[3], Bc[1], Bc[2]));
        c = fmax(c, cancel3(1.0 / H2, Bc[5] * y, 0.0));
        c = fmax(c, cancel3(31.2 * eta0 * Psi / Mkg * (1.0 / H2 + Bc[5] * y), q * Bc[6] * y * y * sqrt(Tr) * H2, 0.0));
        *clam = c;
    }
}

/* Chung's dense-fluid viscosity and conductivity of one pure fluid at a given
 * temperature and molar density (a test aid: the correlation alone, on the
 * state a worked example or a measurement states).  Units as the species
 * table: Tc [K], Vc [cm^3/mol], M [g/mol], dipole [debye]; rho_mol
 * [mol/m^3], cv_molar [J/(mol K)].  out = {mu, lambda, mu_dilute,
 * lambda_dilute} [Pa s, W/(m K)]. */
void orc_chung_pure(double Tc, double Vc, double omega, double M, double dipole, double kappa, double T,
                    double rho_mol, double cv_molar, double out[4])
{
    chung_cs cs;
    cs.Tc = Tc; cs.Vc = Vc; cs.omega = omega; cs.M = M; cs.kappa = kappa;
    const double mur = 131.3 * dipole / sqrt(Vc * Tc);
    cs.mur4 = mur * mur * mur * mur;
    chung_dense(&cs, T, rho_mol, cv_molar, &out[0], &out[1], &out[2], &out[3], NULL, NULL);
}

/* ---------------------------------------------------------------------- */
/* Thermodynamic part of one cell: everything up to h and cp.  Returns the
 * status (0, 3, 4 or 5).  Output arrays may be NULL except d. */
static int cell_thermo(const orc_species *sp, double T, double p, const double *Y, ptrdiff_t ystride,
                       double *X, orc_diag *d, const double *Z_given)
{
    const int N = sp->N;
    memset(d, 0, sizeof(*d));
    if (!(T > 0) || !(p > 0) || !isfinite(T) || !isfinite(p)) return ORC_BAD_INPUT;
    double ysum = 0.0, s = 0.0;
    for (int k = 0; k < N; ++k) {
        double y = Y[k * ystride];
        if (!(y >= 0.0) || !isfinite(y)) return ORC_BAD_INPUT;
        ysum += y;
        s += y / (sp->W[k] * 1e-3);
    }
    if (fabs(ysum - 1.0) > 1e-6) return ORC_BAD_INPUT;
    /* 1. mole fractions */
    ORC_STEP(1);
    for (int k = 0; k < N; ++k) X[k] = (Y[k * ystride] / (sp->W[k] * 1e-3)) / s;
    double Wbar = 0.0;
    for (int k = 0; k < N; ++k) Wbar += X[k] * sp->W[k] * 1e-3;
    d->Wbar = Wbar;

    /* 2. pure-species PR parameters and alpha(T, omega) (PR 1976) */
    ORC_STEP(2);
    double Oa, Ob;
    orc_pr_omegas(sp->printed_constants, &Oa, &Ob);
    double a[64], r[64], dr[64], d2r[64], b[64];
    for (int k = 0; k < N; ++k) {
        double Tc = sp->Tc[k], pc = sp->pc[k], w = sp->omega[k];
        double ac = Oa * ORC_R * ORC_R * Tc * Tc / pc;
        b[k] = Ob * ORC_R * Tc / pc;
        double kap = 0.37464 + 1.54226 * w - 0.26992 * w * w;
        double u = 1.0 + kap * (1.0 - sqrt(T / Tc));
        a[k] = ac * u * u;                             /* a_k(T) */
        double sg = (u >= 0.0) ? 1.0 : -1.0;           /* one-sided at u = 0 */
        r[k] = sqrt(ac) * fabs(u);                     /* sqrt(a_k) */
        dr[k] = -sg * sqrt(ac) * kap / (2.0 * sqrt(T * Tc));
        d2r[k] = sg * sqrt(ac) * kap / (4.0 * sqrt(Tc)) * pow(T, -1.5);
    }
    /* 3. van der Waals mixing: plain double sums */
    ORC_STEP(3);
    double am = 0, dam = 0, d2am = 0, bm = 0;
    for (int i = 0; i < N; ++i) {
        bm += X[i] * b[i];
        for (int j = 0; j < N; ++j) {
            double kk = sp->kij ? (1.0 - sp->kij[i * N + j]) : 1.0;
            double w2 = X[i] * X[j] * kk;
            am += w2 * sqrt(a[i] * a[j]);
            dam += w2 * (dr[i] * r[j] + r[i] * dr[j]);
            d2am += w2 * (d2r[i] * r[j] + 2.0 * dr[i] * dr[j] + r[i] * d2r[j]);
        }
    }
    d->am = am; d->dam = dam; d->d2am = d2am; d->bm = bm;

    /* 4. cubic and root selection */
    ORC_STEP(4);
    double RT = ORC_R * T;
    double A = am * p / (RT * RT), B = bm * p / RT;
    d->A = A; d->B = B;
    double c2 = -(1.0 - B), c1 = A - 3.0 * B * B - 2.0 * B, c0 = -(A * B - B * B - B * B * B);
    d->n_roots = orc_cubic_real_roots(c2, c1, c0, d->roots);
    ORC_STEP(5);
    double best = NAN, gbest = INFINITY, gsecond = INFINITY;
    int nphys = 0;
    for (int k = 0; k < d->n_roots; ++k)
        if (d->roots[k] > B) { if (nphys == 0) best = d->roots[k]; ++nphys; }
    /* one physical root: it is the root; several: the least residual Gibbs energy */
    if (nphys > 1) {
        int seen = 0;
        for (int k = 0; k < d->n_roots; ++k) {
            double z = d->roots[k];
            if (!(z > B)) continue;
            double g = pr_gres(z, A, B);
            if (++seen == 1) { best = z; gbest = g; continue; }
            double gap = fabs(g - gbest);
            if (g < gbest - 1e-12 || (gap <= 1e-12 && z > best)) {
                gsecond = gbest; gbest = g; best = z;
            } else if (g < gsecond) {
                gsecond = g;
            }
        }
    }
    ORC_STEP(0);
    d->n_phys = nphys;
    d->gres_gap = (nphys > 1) ? fabs(gsecond - gbest) : INFINITY;
    if (nphys == 0) return ORC_NO_ROOT;
    double Z = best;
    /* a caller-given Z in place of the selected root: the derived outputs as
     * functions of Z (their sensitivity to the root, for the tests) */
    if (Z_given) Z = *Z_given;
    d->Z = Z;
    {
        double dP = (3.0 * Z + 2.0 * c2) * Z + c1;
        double num = fabs(Z * Z * Z) + fabs(c2) * Z * Z + fabs(c1) * fabs(Z) + fabs(c0);
        d->cond = num / (fabs(Z) * fabs(dP));
    }

    /* 5. ideal-gas part (NASA-7) */
    ORC_STEP(6);
    double h_ig = 0, cp_ig = 0;
    for (int k = 0; k < N; ++k) {
        double cpR, hRT;
        nasa7(sp->nasa_lo + 7 * k, sp->nasa_hi + 7 * k, sp->T_mid[k], T, &cpR, &hRT, NULL);
        double Wk = sp->W[k] * 1e-3;
        h_ig += Y[k * ystride] * hRT * ORC_R * T / Wk;
        cp_ig += Y[k * ystride] * cpR * ORC_R / Wk;
    }
    d->h_ig = h_ig; d->cp_ig = cp_ig;
    d->cv_ig_molar = cp_ig * Wbar - ORC_R;

    /* 6. departures from the PR residual Helmholtz energy */
    ORC_STEP(7);
    const double s2 = sqrt(2.0);
    double V = Z * RT / p;
    double L = log((Z + (1.0 + s2) * B) / (Z + (1.0 - s2) * B));
    double h_dep = RT * (Z - 1.0) + (T * dam - am) / (2.0 * s2 * bm) * L;
    double cv_dep = T * d2am / (2.0 * s2 * bm) * L;
    double den = V * V + 2.0 * bm * V - bm * bm;
    double dpdT = ORC_R / (V - bm) - dam / den;
    double dpdV = -RT / ((V - bm) * (V - bm)) + 2.0 * am * (V + bm) / (den * den);
    double cp_dep = cv_dep - T * dpdT * dpdT / dpdV - ORC_R;
    d->h_dep = h_dep; d->cp_dep = cp_dep; d->dpdT = dpdT; d->dpdV = dpdV;
    ORC_STEP(0);
    if (nphys > 1 && d->gres_gap < 1e-9) return ORC_AMBIGUOUS;
    return ORC_OK;
}

/* Chung transport for a thermodynamic state already evaluated. */
static void cell_transport(const orc_species *sp, double T, double p, const double *X, const orc_diag *d,
                           double *mu, double *lam, double *mu0, double *lam0, double *cmu, double *clam)
{
    if (cmu) *cmu = 1.0;
    if (clam) *clam = 1.0;
    const int N = sp->N;
    double rho_mol = p / (d->Z * ORC_R * T);            /* mol/m^3 */
    if (sp->transport_rule == 1) {
        /* mole-fraction-averaged pure-species Chung properties */
        double m = 0, l = 0, m0 = 0, l0 = 0;
        for (int k = 0; k < N; ++k) {
            chung_cs cs;
            cs.Tc = sp->Tc[k]; cs.Vc = sp->Vc[k]; cs.omega = sp->omega[k]; cs.M = sp->W[k];
            double mur = 131.3 * sp->dipole[k] / sqrt(sp->Vc[k] * sp->Tc[k]);
            cs.mur4 = mur * mur * mur * mur; cs.kappa = sp->kappa[k];
            double mk, lk, m0k, l0k;
            double cmk, clk;
            chung_dense(&cs, T, rho_mol, d->cv_ig_molar, &mk, &lk, &m0k, &l0k, &cmk, &clk);
            m += X[k] * mk; l += X[k] * lk; m0 += X[k] * m0k; l0 += X[k] * l0k;
            if (cmu) *cmu = fmax(*cmu, cmk);
            if (clam) *clam = fmax(*clam, clk);
        }
        *mu = m; *lam = l; *mu0 = m0; *lam0 = l0;
        return;
    }
    ORC_STEP(8);
    /* Chung mixing rules: sigma_i = 0.809 Vc^(1/3) [A], eps_i/k = Tc/1.2593,
     * pair values by geometric/arithmetic/harmonic combining, then
     * sigma_m^3, (eps/k)_m, M_m, omega_m, mu_m^4, kappa_m as double sums. */
    double s3 = 0, e_s3 = 0, e_s2_M = 0, w_s3 = 0, mu4_sum = 0, kap = 0;
    for (int i = 0; i < N; ++i) {
        double si = 0.809 * cbrt(sp->Vc[i]), ei = sp->Tc[i] / 1.2593;
        for (int j = 0; j < N; ++j) {
            double sj = 0.809 * cbrt(sp->Vc[j]), ej = sp->Tc[j] / 1.2593;
            double sij = sqrt(si * sj), eij = sqrt(ei * ej);
            double wij = 0.5 * (sp->omega[i] + sp->omega[j]);
            double Mij = 2.0 * sp->W[i] * sp->W[j] / (sp->W[i] + sp->W[j]);
            double kij = sqrt(sp->kappa[i] * sp->kappa[j]);
            double xx = X[i] * X[j];
            double sij3 = sij * sij * sij;
            s3 += xx * sij3;
            e_s3 += xx * eij * sij3;
            e_s2_M += xx * eij * sij * sij * sqrt(Mij);
            w_s3 += xx * wij * sij3;
            mu4_sum += xx * sp->dipole[i] * sp->dipole[i] * sp->dipole[j] * sp->dipole[j] / sij3;
            kap += xx * kij;
        }
    }
    double sm = cbrt(s3);
    double em = e_s3 / s3;
    double Mm_root = e_s2_M / (em * sm * sm);
    chung_cs cs;
    cs.M = Mm_root * Mm_root;
    cs.omega = w_s3 / s3;
    double mum4 = s3 * mu4_sum;                          /* debye^4 */
    cs.kappa = kap;
    cs.Vc = pow(sm / 0.809, 3.0);
    cs.Tc = 1.2593 * em;
    double mum = sqrt(sqrt(mum4));
    double mur = 131.3 * mum / sqrt(cs.Vc * cs.Tc);
    cs.mur4 = mur * mur * mur * mur;
    ORC_STEP(9);
    chung_dense(&cs, T, rho_mol, d->cv_ig_molar, mu, lam, mu0, lam0, cmu, clam);
}

/* One cell, all outputs.  out = {rho, Z, h, cp, mu, lambda}.  Z_given (NULL
 * for the method itself) replaces the selected root. */
static int orc_cell_z(const orc_species *sp, double T, double p, const double *Y, ptrdiff_t ystride,
                      double out[6], orc_diag *diag, const double *Z_given)
{
    double X[64];
    orc_diag dl;
    orc_diag *d = diag ? diag : &dl;
    int st = cell_thermo(sp, T, p, Y, ystride, X, d, Z_given);
    if (st != ORC_OK && st != ORC_AMBIGUOUS) {
        for (int q = 0; q < 6; ++q) out[q] = NAN;
        return st;
    }
    double Z = d->Z;
    ORC_STEP(10);
    out[0] = p * d->Wbar / (Z * ORC_R * T);
    out[1] = Z;
    out[2] = d->h_ig + d->h_dep / d->Wbar;
    out[3] = d->cp_ig + d->cp_dep / d->Wbar;
    double mu0, lam0;
    cell_transport(sp, T, p, X, d, &out[4], &out[5], &mu0, &lam0, &d->cancel_mu, &d->cancel_lam);
    d->mu_dilute = mu0; d->lambda_dilute = lam0;
    return st;
}

int orc_cell(const orc_species *sp, double T, double p, const double *Y, ptrdiff_t ystride,
             double out[6], orc_diag *diag)
{
    return orc_cell_z(sp, T, p, Y, ystride, out, diag, NULL);
}

/* The outputs of n cells with the root Z[i] substituted for the selected one
 * (out[6*n] as orc_props; status as orc_props').  A test aid: how the derived
 * outputs move with the root, at the oracle's own root and near it. */
void orc_props_at_Z(const orc_species *sp, int64_t n, const double *T, const double *p, const double *Y,
                    const double *Z, double *out, int32_t *status)
{
    for (int64_t i = 0; i < n; ++i) {
        double o[6];
        orc_diag d;
        int st = orc_cell_z(sp, T[i], p[i], Y + i, (ptrdiff_t)n, o, &d, &Z[i]);
        for (int q = 0; q < 6; ++q) out[q * n + i] = o[q];
        if (status) status[i] = st;
    }
}

/* Batch over n cells, SoA: T[n], p[n], Y[N*n] species-major; out[6*n] as
 * rho, Z, h, cp, mu, lambda blocks of n; status[n] may be NULL.  nthreads <= 0
 * uses the OpenMP default. */
void orc_props(const orc_species *sp, int64_t n, const double *T, const double *p, const double *Y,
               double *out, int32_t *status, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(orc_threads(nthreads))
#endif
    for (int64_t i = 0; i < n; ++i) {
        double o[6];
        int st = orc_cell(sp, T[i], p[i], Y + i, (ptrdiff_t)n, o, NULL);
        for (int q = 0; q < 6; ++q) out[q * n + i] = o[q];
        if (status) status[i] = st;
    }
    (void)nthreads;
}

/* Batch with the two further outputs of the paper's networks (Sec. 4.1):
 * out[8*n] as rho, Z, h, cp, mu, lambda, psi, alpha blocks of n, where
 *   psi   = (d rho / d p) at constant h [s^2/m^2], written out as the chain
 *           (d rho/d p)_T + (d rho/d T)_p (d T/d p)_h with
 *           (d T/d p)_h = -(d h/d p)_T / cp and (d h/d p)_T = V - T (d V/d T)_p,
 *           every partial from the PR equation's (dp/dT)_V and (dp/dV)_T;
 *   alpha = lambda / cp [kg/(m s)], the thermal diffusivity of the enthalpy
 *           equation in the form an OpenFOAM-derived solver carries it. */
void orc_props_ext(const orc_species *sp, int64_t n, const double *T, const double *p, const double *Y,
                   double *out, int32_t *status, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(orc_threads(nthreads))
#endif
    for (int64_t i = 0; i < n; ++i) {
        double o[6];
        orc_diag d;
        int st = orc_cell(sp, T[i], p[i], Y + i, (ptrdiff_t)n, o, &d);
        for (int q = 0; q < 6; ++q) out[q * n + i] = o[q];
        double psi = NAN, alpha = NAN;
        if (st == ORC_OK || st == ORC_AMBIGUOUS) {
            const double W = d.Wbar;                          /* kg/mol */
            const double V = d.Z * ORC_R * T[i] / p[i];       /* m^3/mol */
            const double cp_molar = o[3] * W;                 /* J/(mol K) */
            const double drho_dp_T = -W / (V * V * d.dpdV);
            const double dV_dT_p = -d.dpdT / d.dpdV;
            const double drho_dT_p = -W / (V * V) * dV_dT_p;
            const double dh_dp_T = V - T[i] * dV_dT_p;        /* J/(mol Pa) */
            const double dT_dp_h = -dh_dp_T / cp_molar;
            psi = drho_dp_T + drho_dT_p * dT_dp_h;
            alpha = o[5] / o[3];
        }
        out[6 * n + i] = psi;
        out[7 * n + i] = alpha;
        if (status) status[i] = st;
    }
    (void)nthreads;
}

/* Mass-specific ideal-gas enthalpy h_ig = sum_k Y_k h_k(T) / W_k [J/kg] of n
 * cells (NASA-7, the ideal-gas part of the enthalpy, Sec. 2), SoA as
 * orc_props. */
void orc_h_ideal(const orc_species *sp, int64_t n, const double *T, const double *Y, double *h)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = 0; k < sp->N; ++k) {
            double cpR, hRT;
            nasa7(sp->nasa_lo + 7 * k, sp->nasa_hi + 7 * k, sp->T_mid[k], T[i], &cpR, &hRT, NULL);
            s += Y[(int64_t)k * n + i] * hRT * ORC_R * T[i] / (sp->W[k] * 1e-3);
        }
        h[i] = s;
    }
}

/* ---------------------------------------------------------------------- */
/* Per-species outputs of the paper's networks (Sec. 4.1, the list of seven
 * networks; Sec. 2 for the diffusion model).
 *
 * hk_RT[k]: the nondimensional standard-state enthalpy h_k^0(T) / (R T) of the
 *   NASA-7 fit of species k.
 * Dk[k]: the mixture-averaged diffusion coefficient of species k [m^2/s],
 *   D_km = (1 - Y_k) / sum_{j != k} X_j / D_kj, with 1 - Y_k taken as the
 *   other species' share of the mass, sum_{j != k} Y_j / sum_j Y_j (the same
 *   number when the Y sum to 1, and without the cancellation of 1 - Y_k as
 *   Y_k -> 1), from the binary coefficients
 *   of the Chapman-Enskog theory (Poling, Prausnitz & O'Connell, Eq. 11-3.2):
 *     D_kj [cm^2/s] = 0.00266 T^(3/2) / (p[bar] M_kj^(1/2) sigma_kj^2 Omega_D),
 *     M_kj = 2 / (1/M_k + 1/M_j) [g/mol], sigma_kj = (sigma_k + sigma_j)/2 [A],
 *     eps_kj = sqrt(eps_k eps_j), Omega_D(T* = T / eps_kj) by Neufeld et
 *     al. (1972), with the Lennard-Jones parameters of Chung's corresponding
 *     states, sigma = 0.809 Vc^(1/3), eps/k = Tc / 1.2593.
 *   A species with no partner in the cell (sum empty) gets its
 *   self-diffusion coefficient D_kk.
 *   The high-pressure correction the paper takes from Takahashi multiplies
 *   every D_kj p by f(T_r, p_r); here f is a caller table (bilinear in T_r
 *   and p_r, clamped to its edges; none means f = 1) evaluated at the
 *   mixture's pseudo-reduced state by Kay's rule, T_r = T / sum X_i Tc_i,
 *   p_r = p / sum X_i pc_i.
 */
typedef struct {
    int32_t n_Tr, n_pr;
    const double *Tr, *pr;      /* ascending axes */
    const double *f;            /* n_Tr x n_pr, row-major (T_r rows) */
} orc_corr;

/* Neufeld et al. (1972) reduced collision integral for diffusion. */
static double neufeld_omega_d(double Ts)
{
    return 1.06036 / pow(Ts, 0.15610) + 0.19300 / exp(0.47635 * Ts) + 1.03587 / exp(1.52996 * Ts)
           + 1.76474 / exp(3.89411 * Ts);
}

double orc_neufeld_omega_d(double Ts) { return neufeld_omega_d(Ts); }

/* Binary diffusion coefficient [m^2/s] of species i and j at T, p. */
static double binary_d(const orc_species *sp, int i, int j, double T, double p)
{
    const double sig_i = 0.809 * cbrt(sp->Vc[i]), sig_j = 0.809 * cbrt(sp->Vc[j]);
    const double eps_i = sp->Tc[i] / 1.2593, eps_j = sp->Tc[j] / 1.2593;
    const double sig = 0.5 * (sig_i + sig_j);
    const double eps = sqrt(eps_i * eps_j);
    const double Mij = 2.0 / (1.0 / sp->W[i] + 1.0 / sp->W[j]);
    const double om = neufeld_omega_d(T / eps);
    const double d_cgs = 0.00266 * pow(T, 1.5) / ((p / 1e5) * sqrt(Mij) * sig * sig * om);
    return d_cgs * 1e-4;
}

/* Bilinear interpolation of the correction table at (x, y), clamped. */
static double corr_eval(const orc_corr *c, double x, double y)
{
    if (!c) return 1.0;
    if (x < c->Tr[0]) x = c->Tr[0];
    if (x > c->Tr[c->n_Tr - 1]) x = c->Tr[c->n_Tr - 1];
    if (y < c->pr[0]) y = c->pr[0];
    if (y > c->pr[c->n_pr - 1]) y = c->pr[c->n_pr - 1];
    int i = 0, j = 0;
    while (i < c->n_Tr - 2 && x > c->Tr[i + 1]) ++i;
    while (j < c->n_pr - 2 && y > c->pr[j + 1]) ++j;
    const double tx = (x - c->Tr[i]) / (c->Tr[i + 1] - c->Tr[i]);
    const double ty = (y - c->pr[j]) / (c->pr[j + 1] - c->pr[j]);
    const double f00 = c->f[i * c->n_pr + j], f01 = c->f[i * c->n_pr + j + 1];
    const double f10 = c->f[(i + 1) * c->n_pr + j], f11 = c->f[(i + 1) * c->n_pr + j + 1];
    return (1.0 - tx) * ((1.0 - ty) * f00 + ty * f01) + tx * ((1.0 - ty) * f10 + ty * f11);
}

void orc_species_props(const orc_species *sp, const orc_corr *corr, int64_t n, const double *T, const double *p,
                       const double *Y, double *hk_RT, double *Dk, int32_t *status, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(orc_threads(nthreads))
#endif
    for (int64_t i = 0; i < n; ++i) {
        const int N = sp->N;
        double X[64];
        double ysum = 0.0, msum = 0.0;
        int ok = isfinite(T[i]) && isfinite(p[i]) && T[i] > 0.0 && p[i] > 0.0;
        for (int k = 0; k < N; ++k) {
            const double y = Y[(int64_t)k * n + i];
            if (!(y >= 0.0) || !isfinite(y)) ok = 0;
            ysum += y;
            X[k] = y / sp->W[k];
            msum += X[k];
        }
        if (!(fabs(ysum - 1.0) <= 1e-6) || !(msum > 0.0)) ok = 0;
        if (!ok) {
            for (int k = 0; k < N; ++k) {
                if (hk_RT) hk_RT[(int64_t)k * n + i] = NAN;
                if (Dk) Dk[(int64_t)k * n + i] = NAN;
            }
            if (status) status[i] = ORC_BAD_INPUT;
            continue;
        }
        for (int k = 0; k < N; ++k) X[k] /= msum;
        for (int k = 0; k < N; ++k) {
            double cpR, hRT;
            nasa7(sp->nasa_lo + 7 * k, sp->nasa_hi + 7 * k, sp->T_mid[k], T[i], &cpR, &hRT, NULL);
            if (hk_RT) hk_RT[(int64_t)k * n + i] = hRT;
        }
        if (Dk) {
            double Tpc = 0.0, ppc = 0.0;
            for (int k = 0; k < N; ++k) {
                Tpc += X[k] * sp->Tc[k];
                ppc += X[k] * sp->pc[k];
            }
            const double f = corr_eval(corr, T[i] / Tpc, p[i] / ppc);
            for (int k = 0; k < N; ++k) {
                double s = 0.0;
                for (int j = 0; j < N; ++j)
                    if (j != k) s += X[j] / binary_d(sp, k, j, T[i], p[i]);
                double others = 0.0;
                for (int j = 0; j < N; ++j)
                    if (j != k) others += Y[(int64_t)j * n + i];
                const double d0 = (s > 0.0) ? (others / ysum) / s : binary_d(sp, k, k, T[i], p[i]);
                Dk[(int64_t)k * n + i] = f * d0;
            }
        }
        if (status) status[i] = ORC_OK;
    }
    (void)nthreads;
}

/* ---------------------------------------------------------------------- */
/* Bilger's mixture fraction (the networks' composition input, Sec. 4.1):
 * element mass fractions Z_e = sum_k a_ek W_e Y_k / W_k of carbon, hydrogen and
 * oxygen (a_ek atoms of element e in species k, atomic masses W_e), Bilger's
 * coupling function beta = 2 Z_C / W_C + Z_H / (2 W_H) - Z_O / W_O, and
 * Z = (beta - beta_ox) / (beta_fuel - beta_ox) between the oxidiser and fuel
 * streams.  atoms: N x 3 (C, H, O); W: species molar masses [g/mol]. */
static double bilger_beta(int N, const int32_t *atoms, const double *W, const double *Y, ptrdiff_t ys)
{
    const double WC = 12.011, WH = 1.008, WO = 15.999;
    double ZC = 0.0, ZH = 0.0, ZO = 0.0;
    for (int k = 0; k < N; ++k) {
        const double y = Y[(ptrdiff_t)k * ys];
        ZC += atoms[3 * k + 0] * WC * y / W[k];
        ZH += atoms[3 * k + 1] * WH * y / W[k];
        ZO += atoms[3 * k + 2] * WO * y / W[k];
    }
    return 2.0 * ZC / WC + ZH / (2.0 * WH) - ZO / WO;
}

void orc_bilger_z(int N, const int32_t *atoms, const double *W, const double *Y_fuel, const double *Y_ox,
                  int64_t n, const double *Y, double *Z)
{
    const double bf = bilger_beta(N, atoms, W, Y_fuel, 1);
    const double bo = bilger_beta(N, atoms, W, Y_ox, 1);
    for (int64_t i = 0; i < n; ++i)
        Z[i] = (bilger_beta(N, atoms, W, Y + i, (ptrdiff_t)n) - bo) / (bf - bo);
}

/* Diagnostics for n cells (serial). */
void orc_diagnose(const orc_species *sp, int64_t n, const double *T, const double *p, const double *Y,
                  double *out, int32_t *status, orc_diag *diag)
{
    for (int64_t i = 0; i < n; ++i) {
        double o[6];
        int st = orc_cell(sp, T[i], p[i], Y + i, (ptrdiff_t)n, o, &diag[i]);
        for (int q = 0; q < 6; ++q) out[q * n + i] = o[q];
        if (status) status[i] = st;
    }
}

/* ---------------------------------------------------------------------- */
/* Inversion T(h*, p, Y): safeguarded Newton on f(T) = h(T) - h*, f' = cp.
 * Bracket [60, 5000] K.  A Newton step that leaves the current bracket, or
 * that follows a step which failed to halve |f|, is replaced by bisection.
 * Stops when |dT| <= 1e-13 T or |f| <= 1e-13 max(|h*|, cp T).  Status 1 after
 * max_iter iterations; status 2 when h* lies outside [h(60 K), h(5000 K)]
 * (T clamped to the bracket end) or when the bracket collapses onto a jump of
 * h(T) (a switch of the physical root) that h* falls inside. */
static int cell_h(const orc_species *sp, double T, double p, const double *Y, ptrdiff_t ys, double *h, double *cp)
{
    double X[64];
    orc_diag d;
    int st = cell_thermo(sp, T, p, Y, ys, X, &d, NULL);
    if (st != ORC_OK && st != ORC_AMBIGUOUS) return st;
    *h = d.h_ig + d.h_dep / d.Wbar;
    *cp = d.cp_ig + d.cp_dep / d.Wbar;
    return ORC_OK;
}

int orc_T_from_h_cell(const orc_species *sp, double hstar, double p, const double *Y, ptrdiff_t ys,
                      double Tguess, int max_iter, double rtol, double *Tout, int *iters)
{
    const double Tlo0 = 60.0, Thi0 = 5000.0;
    double hlo, cplo, hhi, cphi;
    *iters = 0;
    if (!isfinite(hstar) || !isfinite(Tguess)) { *Tout = NAN; return ORC_BAD_INPUT; }
    int st = cell_h(sp, Tlo0, p, Y, ys, &hlo, &cplo);
    if (st) { *Tout = NAN; return st; }
    st = cell_h(sp, Thi0, p, Y, ys, &hhi, &cphi);
    if (st) { *Tout = NAN; return st; }
    if (hstar < hlo) { *Tout = Tlo0; return ORC_H_OUT_OF_RANGE; }
    if (hstar > hhi) { *Tout = Thi0; return ORC_H_OUT_OF_RANGE; }
    double a = Tlo0, b = Thi0;
    double T = fmin(fmax(Tguess, a), b);
    double fprev = INFINITY;
    for (int it = 1; it <= max_iter; ++it) {
        double h, cp;
        st = cell_h(sp, T, p, Y, ys, &h, &cp);
        *iters = it;
        if (st) { *Tout = T; return st; }
        double f = h - hstar;
        double ftol = rtol * fmax(fabs(hstar), fabs(cp) * T);
        if (fabs(f) <= ftol) { *Tout = T; return ORC_OK; }
        if (f < 0) a = T; else b = T;
        double Tn = T - f / cp;
        int newton_ok = (cp > 0) && (Tn > a) && (Tn < b) && (fabs(f) <= 0.5 * fabs(fprev));
        if (!newton_ok) Tn = 0.5 * (a + b);
        fprev = f;
        if (fabs(Tn - T) <= rtol * T) {
            *Tout = Tn;
            /* converged in T: accept only if h(T) meets h* (no jump inside) */
            double h2, cp2;
            if (cell_h(sp, Tn, p, Y, ys, &h2, &cp2)) return ORC_NO_ROOT;
            if (fabs(h2 - hstar) <= 1e-6 * fmax(fabs(hstar), fabs(cp2) * Tn)) return ORC_OK;
            return ORC_H_OUT_OF_RANGE;
        }
        T = Tn;
    }
    *Tout = T;
    return ORC_NEWTON_MAXIT;
}

void orc_T_from_h(const orc_species *sp, int64_t n, const double *hstar, const double *p, const double *Y,
                  const double *Tguess, double *Tout, int32_t *status, int32_t *iters,
                  int max_iter, double rtol, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(orc_threads(nthreads))
#endif
    for (int64_t i = 0; i < n; ++i) {
        int it = 0;
        int st = orc_T_from_h_cell(sp, hstar[i], p[i], Y + i, (ptrdiff_t)n, Tguess[i], max_iter, rtol, &Tout[i], &it);
        if (status) status[i] = st;
        if (iters) iters[i] = it;
    }
    (void)nthreads;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
