/*
 * Operation counter of the oracle -- TEST AND MEASUREMENT INFRASTRUCTURE ONLY
 * (only tests/ and the counting script beside this file load it).
 *
 * A debug build of pr_oracle.c: this file includes it with `double` replaced
 * by a counting number type, so that every floating-point operation the
 * oracle performs on one cell is counted, per step of the method (the
 * ORC_STEP markers of pr_oracle.c) and per kind: additions and subtractions,
 * multiplications, divisions, square roots, cube roots, exp, expm1, log,
 * log1p, pow, trigonometric calls, and comparisons (not arithmetic; reported
 * apart).
 *
 * What is counted is the per-cell work of the method:
 *  - operations whose operands all come from the species table or are
 *    literals (a_c, b, kappa, sigma_i ...) are table set-up, not per-cell
 *    work: each value carries a flag "depends on the cell's state (T, p, Y)"
 *    and only operations on such values count;
 *  - an operation repeated on the same operands within one cell (the same
 *    sqrt(T) for every species, X_i X_j and X_j X_i) counts once: a memo of
 *    (operation, operand bits) per cell.
 *  - a division by a table constant or a literal counts as a multiplication.
 * The per-step counts are exactly the oracle's; the counting script replaces
 * five steps by exact short forms (the mixing sums and Chung's mixture rules
 * factorised, as the identities for k_ij = 0 allow; the cubic's roots in
 * closed form instead of bracketing; the species terms with the
 * temperature-only factors taken once; the ideal-gas sums over mole-weighted
 * NASA-7 coefficients), each counted here by running that form on the cell's
 * own values under the same counter and checked against the oracle's result.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <unordered_set>
#include <vector>

namespace oc {

enum Cat { ADD = 0, MUL, DIV, SQRT, CBRT, EXP, EXPM1, LOG, LOG1P, POW, TRIG, CMP, NCAT };
constexpr int NSTEP = 16;

struct Counts {
    double c[NSTEP][NCAT];
};

thread_local Counts *g_counts = nullptr;
thread_local int g_step = 0;
thread_local std::unordered_set<uint64_t> *g_memo = nullptr;

inline uint64_t bits(double x)
{
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
}

// count one operation of kind c on operands (a, b), once per cell
inline void tick(int c, double a, double b)
{
    if (!g_counts) return;
    if (c == ADD || c == MUL) {   // commutative: canonical operand order
        if (bits(a) > bits(b)) { double t = a; a = b; b = t; }
    }
    uint64_t h = bits(a) * 0x9E3779B97F4A7C15ull ^ (bits(b) + 0x632BE59BD9B4E019ull + (bits(a) << 6)) ^
                 ((uint64_t)c << 58);
    if (g_memo && !g_memo->insert(h).second) return;
    g_counts->c[g_step][c] += 1.0;
}

struct Real {
    double v;
    bool dep;   // depends on the cell's state
    Real() : v(0.0), dep(false) {}
    Real(double x) : v(x), dep(false) {}
    Real(double x, bool d) : v(x), dep(d) {}
    explicit operator double() const { return v; }
    explicit operator int() const { return (int)v; }
    explicit operator float() const { return (float)v; }
    Real &operator+=(Real b);
    Real &operator-=(Real b);
    Real &operator*=(Real b);
    Real &operator/=(Real b);
};

inline Real bin(int c, double r, Real a, Real b)
{
    const bool d = a.dep || b.dep;
    if (d) tick(c, a.v, b.v);
    return Real(r, d);
}
inline Real operator+(Real a, Real b) { return bin(ADD, a.v + b.v, a, b); }
inline Real operator-(Real a, Real b) { return bin(ADD, a.v - b.v, a, Real(-b.v, b.dep)); }
inline Real operator*(Real a, Real b) { return bin(MUL, a.v * b.v, a, b); }
// a division by a table constant or a literal is a multiplication by its
// reciprocal (table set-up); only a state-dependent divisor costs a division
inline Real operator/(Real a, Real b) { return bin(b.dep ? DIV : MUL, a.v / b.v, a, b); }
inline Real operator-(Real a) { return Real(-a.v, a.dep); }
inline Real operator+(Real a) { return a; }
inline Real &Real::operator+=(Real b) { *this = *this + b; return *this; }
inline Real &Real::operator-=(Real b) { *this = *this - b; return *this; }
inline Real &Real::operator*=(Real b) { *this = *this * b; return *this; }
inline Real &Real::operator/=(Real b) { *this = *this / b; return *this; }

inline bool cmp(Real a, Real b, bool r)
{
    if (a.dep || b.dep) tick(CMP, a.v, b.v);
    return r;
}
inline bool operator<(Real a, Real b) { return cmp(a, b, a.v < b.v); }
inline bool operator>(Real a, Real b) { return cmp(a, b, a.v > b.v); }
inline bool operator<=(Real a, Real b) { return cmp(a, b, a.v <= b.v); }
inline bool operator>=(Real a, Real b) { return cmp(a, b, a.v >= b.v); }
inline bool operator==(Real a, Real b) { return cmp(a, b, a.v == b.v); }
inline bool operator!=(Real a, Real b) { return cmp(a, b, a.v != b.v); }

inline Real un(int c, double r, Real a)
{
    if (a.dep) tick(c, a.v, 0.0);
    return Real(r, a.dep);
}
inline Real sqrt(Real a) { return un(SQRT, std::sqrt(a.v), a); }
inline Real cbrt(Real a) { return un(CBRT, std::cbrt(a.v), a); }
inline Real exp(Real a) { return un(EXP, std::exp(a.v), a); }
inline Real expm1(Real a) { return un(EXPM1, std::expm1(a.v), a); }
inline Real log(Real a) { return un(LOG, std::log(a.v), a); }
inline Real log1p(Real a) { return un(LOG1P, std::log1p(a.v), a); }
inline Real pow(Real a, Real b) { return bin(POW, std::pow(a.v, b.v), a, b); }
inline Real fabs(Real a) { return Real(std::fabs(a.v), a.dep); }   // a sign-bit operation
inline Real fmax(Real a, Real b) { return bin(CMP, std::fmax(a.v, b.v), a, b); }
inline Real fmin(Real a, Real b) { return bin(CMP, std::fmin(a.v, b.v), a, b); }
inline bool isfinite(Real a) { return std::isfinite(a.v); }
inline bool isnan(Real a) { return std::isnan(a.v); }

}  // namespace oc

#define double oc::Real
#define ORC_STEP(s) (oc::g_step = (s))
#include "pr_oracle.c"
#undef double

namespace {

using oc::Real;

// Exact short forms counted in place of three steps of the oracle.

// Step 3 with k_ij = 0: a_m = S0^2, da_m/dT = 2 S0 S1, d2a_m/dT2 = 2 (S0 S2 + S1^2)
// with S_n = sum_k x_k (d^n sqrt(a_k)/dT^n), and b_m = sum_k x_k b_k.
void mixing_factorised(int N, const Real *X, const Real *r, const Real *dr, const Real *d2r, const Real *b,
                       Real *am, Real *dam, Real *d2am, Real *bm)
{
    Real S0 = 0.0, S1 = 0.0, S2 = 0.0, B = 0.0;
    for (int k = 0; k < N; ++k) {
        S0 += X[k] * r[k];
        S1 += X[k] * dr[k];
        S2 += X[k] * d2r[k];
        B += X[k] * b[k];
    }
    *am = S0 * S0;
    *dam = 2.0 * S0 * S1;
    *d2am = 2.0 * (S0 * S2 + S1 * S1);
    *bm = B;
}

// Step 2 with the temperature-only factors taken once: sqrt(T), 1/sqrt(T)
// and T^(-3/2) per cell; per species u_k = (1 + kappa_k) - kappa_k/sqrt(Tc_k)
// sqrt(T), sqrt(a_k) = sqrt(a_c,k) |u_k|, its T-derivatives
// -sgn(u_k) sqrt(a_c,k) kappa_k/(2 sqrt(Tc_k)) T^(-1/2) and
// sgn(u_k) sqrt(a_c,k) kappa_k/(4 sqrt(Tc_k)) T^(-3/2) (table constants
// hoisted).
void species_terms_short(int N, Real T, const double *Tc, const double *pc, const double *omega, double Oa, Real *r,
                         Real *dr, Real *d2r)
{
    const Real sT = sqrt(T);
    const Real isT = 1.0 / sT;
    const Real iT32 = isT / T;
    for (int k = 0; k < N; ++k) {
        const double kp = 0.37464 + 1.54226 * omega[k] - 0.26992 * omega[k] * omega[k];
        const double sac = std::sqrt(Oa * ORC_R * ORC_R * Tc[k] * Tc[k] / pc[k]);
        const double q = kp / std::sqrt(Tc[k]);
        const Real u = (1.0 + kp) - q * sT;
        const double sg = (u.v >= 0.0) ? 1.0 : -1.0;
        r[k] = (sg * sac) * u;
        dr[k] = (-0.5 * sg * sac * q) * isT;
        d2r[k] = (0.25 * sg * sac * q) * iT32;
    }
}

// Step 6 (ideal gas) as sums over mole-weighted coefficients of one NASA-7
// range (every species switches at the same T_mid here):
// cp = sum_j A_j T^j, h = sum_j A_j T^(j+1)/(j+1) + A_5, A_j = sum_k x_k R a_j,k,
// then per unit mass with 1 / W (W = sum_k x_k W_k).
void ideal_gas_short(int N, Real T, const Real *X, const double *lo, const double *hi, double Tmid, Real *h, Real *cp)
{
    const double *set = (T.v < Tmid) ? lo : hi;
    Real A[6];
    for (int j = 0; j < 6; ++j) A[j] = 0.0;
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < 6; ++j) A[j] += X[k] * (ORC_R * set[7 * k + j]);
    *cp = A[0] + T * (A[1] + T * (A[2] + T * (A[3] + T * A[4])));
    *h = T * (A[0] + T * (A[1] * 0.5 + T * (A[2] * (1.0 / 3.0) + T * (A[3] * 0.25 + T * (A[4] * 0.2))))) + A[5];
}

// Step 8 with the combining rules of Chung's mixture rules: every double sum
// but the molar-mass one is a product of single sums (sigma_ij^3 =
// (sigma_i sigma_j)^(3/2), eps_ij sigma_ij^3 = sqrt(eps_i eps_j) (sigma_i
// sigma_j)^(3/2), ...); the molar-mass sum is taken over pairs i <= j.  The
// per-species and per-pair constants are table set-up.
void chung_rules_factorised(const orc_species *sp, const Real *X, Real *s3, Real *e_s3, Real *e_s2_M, Real *w_s3,
                            Real *mu4_sum, Real *kap)
{
    const int N = sp->N;
    Real P1 = 0.0, P2 = 0.0, P3 = 0.0, P4 = 0.0, P5 = 0.0, Q = 0.0;
    for (int i = 0; i < N; ++i) {
        const Real si = 0.809 * cbrt(sp->Vc[i]), ei = sp->Tc[i] / 1.2593;
        const Real s15 = si * sqrt(si);
        P1 += X[i] * s15;
        P2 += X[i] * (sqrt(ei) * s15);
        P3 += X[i] * (sp->omega[i] * s15);
        P4 += X[i] * (sp->dipole[i] * sp->dipole[i] / s15);
        P5 += X[i] * sqrt(sp->kappa[i]);
        for (int j = i; j < N; ++j) {
            const Real sj = 0.809 * cbrt(sp->Vc[j]), ej = sp->Tc[j] / 1.2593;
            const Real Mij = 2.0 * sp->W[i] * sp->W[j] / (sp->W[i] + sp->W[j]);
            const Real c = sqrt(ei * ej) * si * sj * sqrt(Mij) * (i == j ? 1.0 : 2.0);
            Q += X[i] * (X[j] * c);
        }
    }
    *s3 = P1 * P1;
    *e_s3 = P2 * P2;
    *e_s2_M = Q;
    *w_s3 = P3 * P1;
    *mu4_sum = P4 * P4;
    *kap = P5 * P5;
}

// Step 4 in closed form: the real roots of z^3 + c2 z^2 + c1 z + c0 by the
// depressed cubic t^3 + P t + Q (z = t - c2/3): one root by Cardano's formula
// when the discriminant is positive, else three by the trigonometric form.
inline Real acos_(Real a) { if (a.dep) oc::tick(oc::TRIG, a.v, 1.0); return Real(std::acos(a.v), a.dep); }
inline Real cos_(Real a) { if (a.dep) oc::tick(oc::TRIG, a.v, 2.0); return Real(std::cos(a.v), a.dep); }

int cubic_closed_form(Real c2, Real c1, Real c0, Real z[3])
{
    const Real c23 = c2 / 3.0;
    const Real P = c1 - c2 * c23;
    const Real Q = c0 + c23 * (2.0 * c23 * c23 - c1);
    const Real hq = 0.5 * Q, tp = P / 3.0;
    const Real disc = hq * hq + tp * tp * tp;
    if (disc > 0.0) {
        const Real s = sqrt(disc);
        const Real u = cbrt(-hq + (hq > 0.0 ? -s : s));
        z[0] = u - tp / u - c23;
        return 1;
    }
    const Real m = 2.0 * sqrt(-tp);
    Real arg = 3.0 * Q / (P * m);
    arg = fmin(1.0, fmax(-1.0, arg));
    const Real th = acos_(arg) / 3.0;
    z[0] = m * cos_(th + 2.0943951023931957) - c23;
    z[1] = m * cos_(th + 4.1887902047863905) - c23;
    z[2] = m * cos_(th) - c23;
    return 3;
}

inline double relerr(Real a, Real b) { return std::fabs(a.v - b.v) / std::fmax(std::fabs(b.v), 1e-300); }

}  // namespace

extern "C" {

/* Per-cell operation counts of the oracle on n cells (SoA inputs as
 * orc_props): counts[s][c] summed over the cells for step s (ORC_STEP) and
 * kind c (ADD, MUL, DIV, SQRT, CBRT, EXP, EXPM1, LOG, LOG1P, POW, TRIG, CMP);
 * short[r][c] the same for the five replacement forms (r = 0 mixing, 1
 * Chung mixture rules, 2 cubic roots, 3 species EOS terms, 4 ideal gas).
 * check[5]: the largest relative difference of each replacement from the
 * oracle's own result over the cells.  Returns the number of cells evaluated
 * (status 0). */
int64_t orc_count_ops(const double *W, const double *Tc, const double *pc, const double *omega, const double *Vc,
                      const double *dipole, const double *kappa, const double *nasa_lo, const double *nasa_hi,
                      const double *T_mid, int N, int64_t n, const double *T, const double *p, const double *Y,
                      double *counts, double *short_counts, double *check)
{
    // the table as counting numbers (constants: not state-dependent)
    std::vector<Real> tW(W, W + N), tTc(Tc, Tc + N), tpc(pc, pc + N), tom(omega, omega + N), tVc(Vc, Vc + N),
        tdip(dipole, dipole + N), tkap(kappa, kappa + N), tlo(nasa_lo, nasa_lo + 7 * N), thi(nasa_hi, nasa_hi + 7 * N),
        tmid(T_mid, T_mid + N);
    orc_species sp;
    memset(&sp, 0, sizeof(sp));
    sp.N = N;
    sp.W = tW.data(); sp.Tc = tTc.data(); sp.pc = tpc.data(); sp.omega = tom.data(); sp.Vc = tVc.data();
    sp.dipole = tdip.data(); sp.kappa = tkap.data(); sp.nasa_lo = tlo.data(); sp.nasa_hi = thi.data();
    sp.T_mid = tmid.data(); sp.kij = nullptr;
    oc::Counts total, shortc, cell;   // shortc rows: 0 mixing, 1 Chung rules, 2 roots, 3 species terms, 4 ideal gas
    memset(&total, 0, sizeof(total));
    memset(&shortc, 0, sizeof(shortc));
    for (int k = 0; k < 5; ++k) check[k] = 0.0;
    std::unordered_set<uint64_t> memo;
    int64_t good = 0;
    std::vector<Real> Yc(N);
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < N; ++k) Yc[k] = Real(Y[(int64_t)k * n + i], true);
        const Real Ti(T[i], true), pi(p[i], true);
        memset(&cell, 0, sizeof(cell));
        memo.clear();
        oc::g_counts = &cell;
        oc::g_memo = &memo;
        oc::g_step = 0;
        Real out[6];
        orc_diag d;
        const int st = orc_cell(&sp, Ti, pi, Yc.data(), 1, out, &d);
        oc::g_counts = nullptr;
        if (st != ORC_OK) continue;
        ++good;
        for (int s = 0; s < oc::NSTEP; ++s)
            for (int c = 0; c < oc::NCAT; ++c) total.c[s][c] += cell.c[s][c];

        // the replacement forms on this cell's values, counted the same way:
        // their inputs (mole fractions, sqrt(a_k) and its T-derivatives, b_k,
        // the cubic's coefficients) come from steps 1-2 and 4 of the oracle and
        // are set up here uncounted, marked as state-dependent
        Real X[64], r[64], dr[64], d2r[64], b[64];
        {
            double s = 0.0, Ys = 0.0;
            for (int k = 0; k < N; ++k) s += Y[(int64_t)k * n + i] / (W[k] * 1e-3);
            double Oa, Ob;
            {
                Real oa, ob;
                orc_pr_omegas(0, &oa, &ob);
                Oa = oa.v; Ob = ob.v;
            }
            (void)Ys;
            for (int k = 0; k < N; ++k) {
                const double x = (Y[(int64_t)k * n + i] / (W[k] * 1e-3)) / s;
                const double ac = Oa * ORC_R * ORC_R * Tc[k] * Tc[k] / pc[k];
                const double kp = 0.37464 + 1.54226 * omega[k] - 0.26992 * omega[k] * omega[k];
                const double u = 1.0 + kp * (1.0 - std::sqrt(T[i] / Tc[k]));
                const double sg = (u >= 0.0) ? 1.0 : -1.0;
                X[k] = Real(x, true);
                r[k] = Real(std::sqrt(ac) * std::fabs(u), true);
                dr[k] = Real(-sg * std::sqrt(ac) * kp / (2.0 * std::sqrt(T[i] * Tc[k])), true);
                d2r[k] = Real(sg * std::sqrt(ac) * kp / (4.0 * std::sqrt(Tc[k])) * std::pow(T[i], -1.5), true);
                b[k] = Real(Ob * ORC_R * Tc[k] / pc[k], false);
            }
        }
        memo.clear();
        memset(&cell, 0, sizeof(cell));
        oc::g_counts = &cell;
        oc::g_step = 0;
        {
            Real rs[64], drs[64], d2rs[64];
            double Oa;
            {
                oc::Counts *keep = oc::g_counts;
                oc::g_counts = nullptr;
                Real oa, ob;
                orc_pr_omegas(0, &oa, &ob);
                Oa = oa.v;
                oc::g_counts = keep;
            }
            species_terms_short(N, Ti, Tc, pc, omega, Oa, rs, drs, d2rs);
            for (int k = 0; k < N; ++k)
                check[3] = std::fmax(check[3], std::fmax(relerr(rs[k], r[k]), relerr(drs[k], dr[k])));
            for (int c = 0; c < oc::NCAT; ++c) shortc.c[3][c] += cell.c[0][c];
            memo.clear();
            memset(&cell, 0, sizeof(cell));
            Real hs, cps;
            ideal_gas_short(N, Ti, X, nasa_lo, nasa_hi, T_mid[0], &hs, &cps);
            // per unit mass: the oracle's h_ig, cp_ig are J/kg; W = 1 / sum(Y/W) from step 1
            const double Wbar = d.Wbar.v;
            check[4] = std::fmax(check[4], std::fmax(relerr(Real(hs.v / Wbar), d.h_ig), relerr(Real(cps.v / Wbar), d.cp_ig)));
            for (int c = 0; c < oc::NCAT; ++c) shortc.c[4][c] += cell.c[0][c];
            shortc.c[4][oc::MUL] += 2.0;   // the two divisions by W are multiplications by 1/W (taken in step 10)
            memo.clear();
            memset(&cell, 0, sizeof(cell));
        }
        Real am, dam, d2am, bm;
        mixing_factorised(N, X, r, dr, d2r, b, &am, &dam, &d2am, &bm);
        check[0] = std::fmax(check[0], std::fmax(relerr(am, d.am), relerr(bm, d.bm)));
        for (int c = 0; c < oc::NCAT; ++c) shortc.c[0][c] += cell.c[0][c];
        memo.clear();
        memset(&cell, 0, sizeof(cell));
        Real s3, e_s3, e_s2_M, w_s3, mu4, kp;
        chung_rules_factorised(&sp, X, &s3, &e_s3, &e_s2_M, &w_s3, &mu4, &kp);
        {
            // the plain double sum of sigma_m^3 (uncounted) as the check
            oc::g_counts = nullptr;
            double ref = 0.0;
            for (int a = 0; a < N; ++a)
                for (int c2 = 0; c2 < N; ++c2) {
                    const double sa = 0.809 * std::cbrt(Vc[a]), sb = 0.809 * std::cbrt(Vc[c2]);
                    const double sab = std::sqrt(sa * sb);
                    ref += X[a].v * X[c2].v * sab * sab * sab;
                }
            check[1] = std::fmax(check[1], relerr(s3, Real(ref)));
            oc::g_counts = &cell;
        }
        for (int c = 0; c < oc::NCAT; ++c) shortc.c[1][c] += cell.c[0][c];
        memo.clear();
        memset(&cell, 0, sizeof(cell));
        const Real A(d.A.v, true), B(d.B.v, true);
        const Real c2 = -(1.0 - B), c1 = A - 3.0 * B * B - 2.0 * B, c0 = -(A * B - B * B - B * B * B);
        memset(&cell, 0, sizeof(cell));   // the coefficients are counted in the oracle's step 4
        memo.clear();
        Real zc[3];
        const int nz = cubic_closed_form(c2, c1, c0, zc);
        for (int c = 0; c < oc::NCAT; ++c) shortc.c[2][c] += cell.c[0][c];
        oc::g_counts = nullptr;
        double best = 1e300;
        for (int k = 0; k < nz; ++k) best = std::fmin(best, std::fabs(zc[k].v - d.Z.v) / d.Z.v);
        check[2] = std::fmax(check[2], best);
    }
    for (int s = 0; s < oc::NSTEP; ++s)
        for (int c = 0; c < oc::NCAT; ++c) counts[s * oc::NCAT + c] = total.c[s][c];
    for (int s = 0; s < 5; ++s)
        for (int c = 0; c < oc::NCAT; ++c) short_counts[s * oc::NCAT + c] = shortc.c[s][c];
    return good;
}

}  // extern "C"
