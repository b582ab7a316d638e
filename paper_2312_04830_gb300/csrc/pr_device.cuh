// Device-side arithmetic of the real-fluid property evaluation.
//
// One thread evaluates one cell.  Everything a cell needs from the species
// data sits in shared memory (staged once per CTA); per-cell state lives in
// registers.  `Real` is the type of the mixing, ideal-gas and transport
// arithmetic, `RZ` the type of the cubic solve (FP64/FP64, FP32/FP32 or the
// mixed FP32/FP64 path).
//
// Sources of each step (arxiv 2312.04830 and the published methods it
// delegates to Cantera):
//   * Peng-Robinson EOS, Eq. 1, with a = Omega_a R^2 Tc^2/pc, b = Omega_b R Tc/pc
//     (Sec. 2).  Omega_a, Omega_b are taken at their exact critical-point
//     values (the printed 0.45724 and 0.07780 are their 5-digit roundings).
//   * alpha(T, omega) = [1 + kappa (1 - sqrt(T/Tc))]^2 with the PR-1976 kappa.
//   * van der Waals one-fluid mixing (Sec. 2).  With k_ij = 0 the double sum
//     sum_i sum_j X_i X_j sqrt(a_i a_j) equals (sum_i X_i sqrt(a_i))^2 exactly;
//     sqrt(a_i) = sqrt(a_c,i) |u_i| keeps the cross terms non-negative past the
//     temperature where u_i = 1 + kappa_i (1 - sqrt(T/Tc,i)) changes sign.
//   * Residual properties from the PR residual Helmholtz energy.
//   * NASA-7 two-range ideal-gas polynomials.
//   * Chung et al. (1988) dense-fluid viscosity and conductivity with Chung's
//     mixture corresponding-states rules (Sec. 2, "modified Chung's
//     transport model"), evaluated in factorised form.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "prgb300.h"

#include "pr_math64.cuh"

namespace prk {

constexpr double kR = 8.314462618;                     // J/(mol K)
constexpr double kOmegaA = 0.45723552892138219;        // Eq. 1, exact critical-point value
constexpr double kOmegaB = 0.07779607390388846;
constexpr double kOmegaAPrinted = 0.45724;
constexpr double kOmegaBPrinted = 0.07780;
constexpr double kSqrt2 = 1.4142135623730950488;
constexpr double kTLo = 60.0, kTHi = 5000.0;           // inversion bracket [K]

enum CellStatus : int32_t { kOk = 0, kMaxIt = 1, kHRange = 2, kNoRoot = 3, kBadInput = 4, kAmbiguous = 5 };

// Per-species record, derived on the device by the setup kernel.
template <typename Real>
struct SpeciesRec {
    Real inv_W;              // 1/W [mol/kg]
    Real sqrt_ac;            // sqrt(Omega_a) R Tc / sqrt(pc)
    Real b;                  // Omega_b R Tc / pc [m^3/mol]
    Real kappa;              // PR-1976 slope of sqrt(alpha)
    Real kq;                 // kappa / sqrt(Tc)
    Real T_mid;              // NASA-7 range switch [K]
    Real cp_lo[5], cp_hi[5]; // R a1..a5  -> molar cp [J/(mol K)]
    Real h_lo[6], h_hi[6];   // R (a1, a2/2, a3/3, a4/4, a5/5, a6) -> molar h [J/mol]
    // Chung mixture rules in factorised form (sigma in Angstrom, eps/k in K)
    Real s15;                // sigma^(3/2)
    Real e05s15;             // sqrt(eps/k) sigma^(3/2)
    Real ws15;               // omega sigma^(3/2)
    Real mu2s15;             // dipole^2 / sigma^(3/2)
    Real sqkap;              // sqrt(kappa_assoc)
    // pure-species Chung inputs (mole-fraction-averaged transport rule)
    Real Tc, Vc, omega, M, mur4, kap;
};

// ------------------------------------------------------------------ math
template <typename T> struct M;
template <> struct M<double> {
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
    static __device__ __forceinline__ double cbrt(double x) { return ::cbrt(x); }
    // table-driven forms with fewer FP64-pipe operations (pr_math64.cuh)
    static __device__ __forceinline__ double log(double x) { return m64::log(x); }
    static __device__ __forceinline__ double log1p(double x) { return m64::log1p(x); }
    static __device__ __forceinline__ double exp(double x) { return m64::exp(x); }
    static __device__ __forceinline__ double expm1(double x) { return m64::expm1(x); }
    static __device__ __forceinline__ double fabs(double x) { return ::fabs(x); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
    static __device__ __forceinline__ bool finite(double x) { return isfinite(x); }
    static __device__ __forceinline__ double nan() { return __longlong_as_double(0x7ff8000000000000ULL); }
    static constexpr double eps = 2.220446049250313e-16;
};
template <> struct M<float> {
    static __device__ __forceinline__ float sqrt(float x) { return ::sqrtf(x); }
    static __device__ __forceinline__ float rsqrt(float x) { return ::rsqrtf(x); }
    static __device__ __forceinline__ float cbrt(float x) { return ::cbrtf(x); }
    static __device__ __forceinline__ float log(float x) { return ::logf(x); }
    static __device__ __forceinline__ float log1p(float x) { return ::log1pf(x); }
    static __device__ __forceinline__ float exp(float x) { return ::expf(x); }
    static __device__ __forceinline__ float expm1(float x) { return ::expm1f(x); }
    static __device__ __forceinline__ float fabs(float x) { return ::fabsf(x); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return ::fmaf(a, b, c); }
    static __device__ __forceinline__ bool finite(float x) { return isfinite(x); }
    static __device__ __forceinline__ float nan() { return __int_as_float(0x7fc00000); }
    static constexpr float eps = 1.1920929e-07f;
};

// -------------------------------------------------------- composition
// T-independent part of a cell: mole fractions, mean molar mass, b_m.
// Per-species branch decisions of the FP64 path on the integer pipe (an FP64
// compare takes an FP64-pipe slot, the scarce resource of these kernels).
// For a positive finite a and a non-NaN b, a < b exactly when a's bit pattern
// is below b's as a signed integer: positive numbers order like their
// patterns, and every negative b (-0 included) has a negative pattern.
template <typename Real>
__device__ __forceinline__ bool lt_pos(Real a, Real b)
{
    if constexpr (sizeof(Real) == 8)
        return __double_as_longlong(a) < __double_as_longlong(b);
    else
        return a < b;
}

// y >= 0 and finite (-0 included): on the bit pattern for FP64.
template <typename Real>
__device__ __forceinline__ bool nonneg_finite(Real y)
{
    if constexpr (sizeof(Real) == 8) {
        const long long b = __double_as_longlong(y);
        return (b >= 0 && b < 0x7FF0000000000000LL) || b == (long long)0x8000000000000000ULL;
    } else {
        return (y >= Real(0)) && M<Real>::finite(y);
    }
}

// u >= 0 for a non-NaN u (-0 counts as 0): sign bit clear, or magnitude 0.
template <typename Real>
__device__ __forceinline__ bool nonneg(Real u)
{
    if constexpr (sizeof(Real) == 8) {
        const long long b = __double_as_longlong(u);
        return b >= 0 || (b << 1) == 0;
    } else {
        return u >= Real(0);
    }
}

template <typename Real, int NS>
struct Comp {
    Real x[NS];     // mole fractions
    Real Wbar;      // kg/mol
    Real bm;        // m^3/mol
};

template <typename Real, int NS>
__device__ __forceinline__ bool load_comp(Comp<Real, NS> &c, const Real *__restrict__ Y, int64_t ldY, int64_t i,
                                          int N, const SpeciesRec<Real> *sp)
{
    Real ysum = 0, s = 0;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        Real y = (k < N) ? __ldg(Y + (int64_t)k * ldY + i) : Real(0);
        ok = ok && nonneg_finite(y);
        ysum += y;
        c.x[k] = y * sp[k].inv_W;            // moles per kg, normalised below
        s += c.x[k];
    }
    ok = ok && (M<Real>::fabs(ysum - Real(1)) <= Real(1e-6)) && (s > Real(0));
    Real inv_s = Real(1) / s;
    Real bm = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        c.x[k] *= inv_s;
        bm = M<Real>::fma(c.x[k], sp[k].b, bm);
    }
    c.Wbar = inv_s;
    c.bm = bm;
    return ok;
}

// ------------------------------------------------------- a_m(T) and derivatives
// (D2 = false: the second derivative is not needed and left at 0)
template <typename Real, int NS, bool KIJ, bool D2 = true>
__device__ __forceinline__ void mix_a(const Comp<Real, NS> &c, Real T, const SpeciesRec<Real> *sp,
                                      const Real *kij1m, Real &am, Real &dam, Real &d2am)
{
    const Real sqT = M<Real>::sqrt(T);
    const Real isqT = Real(1) / sqT;
    const Real h1 = Real(-0.5) * isqT;          // d sqrt(T)/dT factor (with sign)
    const Real h2 = Real(0.25) * isqT / T;
    if (!KIJ) {
        Real S0 = 0, S1 = 0, S2 = 0;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const Real u = M<Real>::fma(-sp[k].kq, sqT, Real(1) + sp[k].kappa);
            const Real g = nonneg(u) ? sp[k].sqrt_ac : -sp[k].sqrt_ac;  // sqrt(ac) sgn(u)
            const Real xg = c.x[k] * g;
            S0 = M<Real>::fma(xg, u, S0);              // x sqrt(ac) |u|
            const Real xgq = xg * sp[k].kq;
            S1 = M<Real>::fma(xgq, h1, S1);
            if constexpr (D2) S2 = M<Real>::fma(xgq, h2, S2);
        }
        am = S0 * S0;
        dam = Real(2) * S0 * S1;
        d2am = D2 ? Real(2) * M<Real>::fma(S0, S2, S1 * S1) : Real(0);
    } else {
        // O(N^2) with (1 - k_ij) weights; per-species terms recomputed in the
        // inner loop instead of being held in N-long register arrays
        Real a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 1
        for (int i = 0; i < NS; ++i) {
            Real xi = 0;   // x_i by selects (no dynamic index into the registers)
#pragma unroll
            for (int j = 0; j < NS; ++j) xi = (j == i) ? c.x[j] : xi;
            const Real ui = M<Real>::fma(-sp[i].kq, sqT, Real(1) + sp[i].kappa);
            const Real gi = xi * (nonneg(ui) ? sp[i].sqrt_ac : -sp[i].sqrt_ac);
            const Real ri = gi * ui, dri = gi * sp[i].kq * h1, d2ri = gi * sp[i].kq * h2;
            Real t0 = 0, t1 = 0;
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                const Real uj = M<Real>::fma(-sp[j].kq, sqT, Real(1) + sp[j].kappa);
                const Real gj = c.x[j] * kij1m[i * NS + j] * (nonneg(uj) ? sp[j].sqrt_ac : -sp[j].sqrt_ac);
                t0 = M<Real>::fma(gj, uj, t0);
                t1 = M<Real>::fma(gj * sp[j].kq, h1, t1);
            }
            a0 = M<Real>::fma(ri, t0, a0);
            a1 = M<Real>::fma(Real(2) * dri, t0, a1);
            if constexpr (D2) a2 = M<Real>::fma(Real(2), M<Real>::fma(d2ri, t0, dri * t1), a2);
        }
        am = a0;
        dam = a1;
        d2am = a2;
    }
}

// ------------------------------------------------------------------ cubic
// Real roots of Z^3 + c2 Z^2 + c1 Z + c0 that exceed B, each seeded by the
// closed form (Cardano / trigonometric, in FP32) and refined by Newton
// iterations in RZ.  Returns the number of such roots in z[] (ascending).
template <typename RZ>
__device__ __forceinline__ RZ cubic_polish(RZ z, RZ c2, RZ c1, RZ c0)
{
#pragma unroll 1
    for (int it = 0; it < 12; ++it) {
        const RZ f = M<RZ>::fma(M<RZ>::fma(z + c2, z, c1), z, c0);
        const RZ d = M<RZ>::fma(M<RZ>::fma(RZ(3), z, RZ(2) * c2), z, c1);
        if (d == RZ(0)) break;
        const RZ dz = f / d;
        z -= dz;
        if (M<RZ>::fabs(dz) <= RZ(2) * M<RZ>::eps * M<RZ>::fabs(z)) break;
    }
    return z;
}

// *clear (optional): the count of physical roots is settled by margins its
// rounding cannot close: the cubic is away from the one-/three-real-root
// boundary, |disc| > 1e-4 (hq^2 + |tp^3|), and at most one root lies above
// 0.999 B (the others, if any, below it by more than FP32 rounding moves them).
template <typename RZ>
__device__ __forceinline__ int cubic_phys_roots(RZ c2, RZ c1, RZ c0, RZ B, RZ z[3], bool *clear = nullptr)
{
    const RZ c23 = c2 * RZ(1.0 / 3.0);
    const RZ P = M<RZ>::fma(-c2, c23, c1);                         // c1 - c2^2/3
    const RZ Q = M<RZ>::fma(c23, M<RZ>::fma(RZ(2) * c23, c23, -c1), c0);
    const RZ hq = RZ(0.5) * Q, tp = P * RZ(1.0 / 3.0);
    const RZ disc = M<RZ>::fma(hq, hq, tp * tp * tp);
    const bool far = M<RZ>::fabs(disc) > RZ(1e-4) * (hq * hq + M<RZ>::fabs(tp * tp * tp));
    // seeds: one real root (Cardano), or three (trigonometric form, ascending)
    float seed0, seed1 = 0.f, seed2 = 0.f;
    bool three = false;
    if (disc > RZ(0)) {
        const float sq = sqrtf((float)disc);
        const float hqf = (float)hq;
        const float u = cbrtf(-hqf - copysignf(sq, hqf));
        seed0 = ((u != 0.f) ? (u - (float)P / (3.f * u)) : 0.f) - (float)c23;
    } else {
        const float m = 2.f * sqrtf(fmaxf(-(float)tp, 0.f));
        float arg = (m > 0.f) ? (3.f * (float)Q) / ((float)P * m) : 0.f;
        arg = fminf(1.f, fmaxf(-1.f, arg));
        const float th = acosf(arg) * (1.f / 3.f);
        const float c23f = (float)c23;
        seed0 = m * cosf(th + 2.09439510239320f) - c23f;   // smallest
        seed1 = m * cosf(th + 4.18879020478639f) - c23f;   // middle
        seed2 = m * cosf(th) - c23f;                      // largest
        three = true;
    }
    // polish the seeds above B; every array below is indexed by constants
    // only, so it stays in registers
    const float Bcut = (float)B * (1.f - 1e-3f);
    RZ r[3] = {RZ(0), RZ(0), RZ(0)};
    bool v[3];
    v[0] = seed0 > Bcut;
    v[1] = three && seed1 > Bcut;
    v[2] = three && seed2 > Bcut;
    if (clear) *clear = far && ((int)v[0] + (int)v[1] + (int)v[2]) <= 1;
    if (v[0]) r[0] = cubic_polish<RZ>((RZ)seed0, c2, c1, c0);
    if (v[1]) r[1] = cubic_polish<RZ>((RZ)seed1, c2, c1, c0);
    if (v[2]) r[2] = cubic_polish<RZ>((RZ)seed2, c2, c1, c0);
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = v[k] && r[k] > B;
    // drop duplicates produced by converging seeds (against the roots kept)
    const RZ dtol = RZ(64) * M<RZ>::eps;
    if (v[1] && v[0] && M<RZ>::fabs(r[1] - r[0]) <= dtol * M<RZ>::fabs(r[1])) v[1] = false;
    if (v[2] && ((v[0] && M<RZ>::fabs(r[2] - r[0]) <= dtol * M<RZ>::fabs(r[2])) ||
                 (v[1] && M<RZ>::fabs(r[2] - r[1]) <= dtol * M<RZ>::fabs(r[2]))))
        v[2] = false;
    // ascending, the dropped ones last
    const RZ big = RZ(3e38);
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = v[k] ? r[k] : big;
    RZ t;
    if (r[1] < r[0]) { t = r[0]; r[0] = r[1]; r[1] = t; }
    if (r[2] < r[1]) { t = r[1]; r[1] = r[2]; r[2] = t; }
    if (r[1] < r[0]) { t = r[0]; r[0] = r[1]; r[1] = t; }
#pragma unroll
    for (int k = 0; k < 3; ++k) z[k] = r[k];
    return (int)v[0] + (int)v[1] + (int)v[2];
}

// Residual Gibbs energy G_res/(RT) of the PR fluid at root Z.
template <typename RZ>
__device__ __forceinline__ RZ pr_gres(RZ Z, RZ A, RZ B)
{
    const RZ dp = RZ(1.0 + kSqrt2), dm = RZ(1.0 - kSqrt2);
    return Z - RZ(1) - M<RZ>::log(Z - B) - A / (RZ(2.0 * kSqrt2) * B) * M<RZ>::log((Z + dp * B) / (Z + dm * B));
}

// Select the physical root: the one of least residual Gibbs energy; ties
// (|dg| <= 1e-12) go to the larger Z; |dg| < 1e-9 flags the cell ambiguous.
template <typename RZ>
__device__ __forceinline__ int select_root(const RZ *z, int n, RZ A, RZ B, RZ &Z)
{
    if (n == 0) return kNoRoot;
    Z = z[0];
    if (n == 1) return kOk;
    RZ gbest = pr_gres<RZ>(z[0], A, B), gsecond = RZ(3e38);
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        if (k >= n) break;
        const RZ g = pr_gres<RZ>(z[k], A, B);
        const RZ gap = M<RZ>::fabs(g - gbest);
        if (g < gbest - RZ(1e-12) || (gap <= RZ(1e-12) && z[k] > Z)) {
            gsecond = gbest; gbest = g; Z = z[k];
        } else if (g < gsecond) {
            gsecond = g;
        }
    }
    return (M<RZ>::fabs(gsecond - gbest) < RZ(1e-9)) ? kAmbiguous : kOk;
}

// ------------------------------------------------------ thermodynamics
template <typename Real>
struct Thermo {
    Real Z, rho_mol;      // compressibility, molar density [mol/m^3]
    Real h, cp;           // J/kg, J/(kg K)
    Real cv_ig_molar;     // ideal-gas molar cv [J/(mol K)]
    Real dpdT, dpdV;      // (dp/dT)_V [Pa/K], (dp/dV)_T [Pa mol/m^3], V molar
    int status;
    int nroots;           // physical roots (Z > B) of the cubic at this state
};

// Mole-weighted NASA-7 coefficient sums of one range: A_j = sum_k x_k R a_j,k
// (j = 0..4, the cp coefficients) and A5 = sum_k x_k R a_6,k.
template <typename Real, int NS, bool LO>
__device__ __forceinline__ void nasa_sums(const Comp<Real, NS> &c, const SpeciesRec<Real> *sp, Real (&A)[5], Real &A5)
{
#pragma unroll
    for (int j = 0; j < 5; ++j) A[j] = Real(0);
    A5 = Real(0);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const Real *a = LO ? sp[k].cp_lo : sp[k].cp_hi;
#pragma unroll
        for (int j = 0; j < 5; ++j) A[j] = M<Real>::fma(c.x[k], a[j], A[j]);
        A5 = M<Real>::fma(c.x[k], LO ? sp[k].h_lo[5] : sp[k].h_hi[5], A5);
    }
}

// tmid_u > 0: every species switches NASA-7 range at tmid_u, so the ideal-gas
// sums are taken over mole-weighted coefficients (one range test per cell,
// one polynomial each for cp and h); otherwise species by species.
// CP = false: Z, h and the ideal-gas cv only (cp, the density and the
// pressure derivatives are left at 0).
template <typename Real, typename RZ, int NS, bool KIJ, bool CP = true>
__device__ __forceinline__ void thermo(const Comp<Real, NS> &c, Real T, Real p, const SpeciesRec<Real> *sp,
                                       const Real *kij1m, Thermo<Real> &o, Real tmid_u = Real(0))
{
    Real am, dam, d2am;
    mix_a<Real, NS, KIJ, CP>(c, T, sp, kij1m, am, dam, d2am);
    const Real bm = c.bm;
    const Real RT = Real(kR) * T;
    RZ Zz;
    RZ larg;   // 2 sqrt 2 B / (Z + (1 - sqrt 2) B), the departure logarithm's argument
    bool need_rz = true;
    if constexpr (!std::is_same<Real, RZ>::value) {
        // Mixed precision: the FP32 cubic decides where FP64 is needed.  A
        // single physical root, with the root count settled by margins FP32
        // rounding cannot close (see cubic_phys_roots), is taken as it is: its
        // coefficients are FP32 numbers, so an FP64 polish would not make it
        // more accurate.  Several physical roots (the Gibbs selection between
        // them) or a near-degenerate cubic go through the FP64 solve.
        const Real iRTf = Real(1) / RT;
        const Real Bf = bm * p * iRTf;
        const Real Af = am * p * iRTf * iRTf;
        const Real c2f = Bf - Real(1);
        const Real c1f = Af - Bf * M<Real>::fma(Real(3), Bf, Real(2));
        const Real c0f = Bf * (Bf + M<Real>::fma(Bf, Bf, -Af));
        Real zf[3];
        bool clear = false;
        const int nf = cubic_phys_roots<Real>(c2f, c1f, c0f, Bf, zf, &clear);
        if (nf == 1 && clear) {
            o.status = kOk;
            o.nroots = 1;
            Zz = (RZ)zf[0];
            larg = (RZ)(Real(2.0 * kSqrt2) * Bf / (zf[0] + Real(1.0 - kSqrt2) * Bf));
            need_rz = false;
        }
    }
    if (need_rz) {
        // pairs of quotients below share one reciprocal (an FP64 division is
        // several FP64-pipe instructions)
        const RZ iRT = RZ(1) / (RZ)RT;
        const RZ pRT = (RZ)p * iRT;
        const RZ B = (RZ)bm * pRT;
        const RZ A = (RZ)am * pRT * iRT;
        const RZ c2 = B - RZ(1);
        const RZ c1 = A - B * M<RZ>::fma(RZ(3), B, RZ(2));
        const RZ c0 = B * (B + M<RZ>::fma(B, B, -A));
        RZ zr[3];
        const int nr = cubic_phys_roots<RZ>(c2, c1, c0, B, zr);
        o.nroots = nr;
        o.status = select_root<RZ>(zr, nr, A, B, Zz);
        if (o.status == kNoRoot) return;
        larg = RZ(2.0 * kSqrt2) * B / (Zz + RZ(1.0 - kSqrt2) * B);
    }

    // ideal-gas part (NASA-7), molar
    Real cp_ig = 0, h_ig = 0;
    if (tmid_u > Real(0)) {
        Real A[5], A5;
        if (lt_pos(T, tmid_u)) nasa_sums<Real, NS, true>(c, sp, A, A5);   // T > 0 here
        else nasa_sums<Real, NS, false>(c, sp, A, A5);
        cp_ig = M<Real>::fma(M<Real>::fma(M<Real>::fma(M<Real>::fma(A[4], T, A[3]), T, A[2]), T, A[1]), T, A[0]);
        // h = sum_j A_j T^(j+1) / (j+1) + A5
        const Real hp = M<Real>::fma(M<Real>::fma(M<Real>::fma(M<Real>::fma(A[4] * Real(0.2), T, A[3] * Real(0.25)), T,
                                                                A[2] * Real(1.0 / 3.0)), T, A[1] * Real(0.5)), T, A[0]);
        h_ig = M<Real>::fma(hp, T, A5);
    } else {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const bool lo = lt_pos(T, sp[k].T_mid);   // T > 0 here
            const Real *a = lo ? sp[k].cp_lo : sp[k].cp_hi;
            const Real *e = lo ? sp[k].h_lo : sp[k].h_hi;
            const Real cpk = M<Real>::fma(M<Real>::fma(M<Real>::fma(M<Real>::fma(a[4], T, a[3]), T, a[2]), T, a[1]), T, a[0]);
            const Real hk = M<Real>::fma(M<Real>::fma(M<Real>::fma(M<Real>::fma(M<Real>::fma(e[4], T, e[3]), T, e[2]), T, e[1]), T, e[0]), T, e[5]);
            cp_ig = M<Real>::fma(c.x[k], cpk, cp_ig);
            h_ig = M<Real>::fma(c.x[k], hk, h_ig);
        }
    }
    const Real rWb = Real(1) / (c.Wbar * bm);
    const Real iW = bm * rWb;                                         // 1 / Wbar
    const Real inv2s2b = Real(1.0 / (2.0 * kSqrt2)) * c.Wbar * rWb;   // 1 / (2 sqrt 2 bm)

    // departures (in RZ where the root enters, then Real)
    // ln[(Z + (1 + sqrt 2) B)/(Z + (1 - sqrt 2) B)] = log1p(2 sqrt 2 B / (Z + (1 - sqrt 2) B)):
    // the argument (larg, above) from the root's precision; the logarithm at
    // the outputs'
    const Real Z = (Real)Zz;
    const Real Lr = M<Real>::log1p((Real)larg);
    const Real h_dep = M<Real>::fma(RT, (Real)(Zz - RZ(1)), M<Real>::fma(T, dam, -am) * inv2s2b * Lr);
    if constexpr (!CP) {
        o.Z = Z;
        o.rho_mol = 0;
        o.h = (h_ig + h_dep) * iW;
        o.cp = 0;
        o.cv_ig_molar = cp_ig - Real(kR);
        o.dpdT = 0;
        o.dpdV = 0;
        return;
    }
    const Real cv_dep = T * d2am * inv2s2b * Lr;
    const Real ZRT = Z * RT;
    const Real rzp = Real(1) / (ZRT * p);
    const Real V = ZRT * ZRT * rzp;                                   // Z R T / p
    const Real rho_mol = p * p * rzp;                                 // p / (Z R T)
    const Real Vmb = V - bm;
    const Real den = M<Real>::fma(V, V + Real(2) * bm, -bm * bm);
    const Real rvd = Real(1) / (Vmb * den);
    const Real iVmb = den * rvd, iden = Vmb * rvd;
    const Real dpdT = Real(kR) * iVmb - dam * iden;
    const Real dpdV = -RT * iVmb * iVmb + Real(2) * am * (V + bm) * iden * iden;
    const Real cp_dep = cv_dep - T * dpdT * dpdT / dpdV - Real(kR);
    o.Z = Z;
    o.rho_mol = rho_mol;
    o.h = (h_ig + h_dep) * iW;
    o.cp = (cp_ig + cp_dep) * iW;
    o.cv_ig_molar = cp_ig - Real(kR);
    o.dpdT = dpdT;
    o.dpdV = dpdV;
}

// ------------------------------------------------------------ transport
// Chung et al. (1988) coefficient tables (Poling, Prausnitz & O'Connell,
// Tables 9-6 and 10-3): E_i = a + b omega + c mu_r^4 + d kappa.
__constant__ float kChungVisc[10][4] = {
    {6.324f, 50.412f, -51.680f, 1189.0f},
    {1.210e-3f, -1.154e-3f, -6.257e-3f, 0.03728f},
    {5.283f, 254.209f, -168.48f, 3898.0f},
    {6.623f, 38.096f, -8.464f, 31.42f},
    {19.745f, 7.630f, -14.354f, 31.53f},
    {-1.900f, -12.537f, 4.985f, -18.15f},
    {24.275f, 3.450f, -11.291f, 69.35f},
    {0.7972f, 1.117f, 0.01235f, -4.117f},
    {-0.2382f, 0.06770f, -0.8163f, 4.025f},
    {0.06863f, 0.3479f, 0.5926f, -0.727f},
};
__constant__ double kChungViscD[10][4] = {
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
__constant__ float kChungCond[7][4] = {
    {2.4166f, 0.74824f, -0.91858f, 121.72f},
    {-0.50924f, -1.5094f, -49.991f, 69.983f},
    {6.6107f, 5.6207f, 64.760f, 27.039f},
    {14.543f, -8.9139f, -5.6379f, 74.344f},
    {0.79274f, 0.82019f, -0.69369f, 6.3173f},
    {-5.8634f, 12.801f, 9.5893f, 65.529f},
    {91.089f, 128.11f, -54.217f, 523.81f},
};
__constant__ double kChungCondD[7][4] = {
    {2.4166, 0.74824, -0.91858, 121.72},
    {-0.50924, -1.5094, -49.991, 69.983},
    {6.6107, 5.6207, 64.760, 27.039},
    {14.543, -8.9139, -5.6379, 74.344},
    {0.79274, 0.82019, -0.69369, 6.3173},
    {-5.8634, 12.801, 9.5893, 65.529},
    {91.089, 128.11, -54.217, 523.81},
};

template <typename Real> __device__ __forceinline__ Real chung_visc(int i, int j);
template <> __device__ __forceinline__ double chung_visc<double>(int i, int j) { return kChungViscD[i][j]; }
template <> __device__ __forceinline__ float chung_visc<float>(int i, int j) { return kChungVisc[i][j]; }
template <typename Real> __device__ __forceinline__ Real chung_cond(int i, int j);
template <> __device__ __forceinline__ double chung_cond<double>(int i, int j) { return kChungCondD[i][j]; }
template <> __device__ __forceinline__ float chung_cond<float>(int i, int j) { return kChungCond[i][j]; }

// Chung dense-fluid mu [Pa s] and lambda [W/(m K)] for corresponding-states
// parameters (Tc [K], Vc [cm^3/mol] and its cube root cVc, omega, M [g/mol],
// mu_r^4, kappa).  The square roots of T*, M T and Tc / M all follow from
// sqrt(T / Tc) and sqrt(M Tc).
template <typename Real>
__device__ __forceinline__ void chung_dense(Real Tc, Real Vc, Real cVc, Real omega, Real Mg, Real mur4, Real kap,
                                            Real T, Real rho_mol, Real cv_molar, Real &mu, Real &lam)
{
    // pairs of quotients share one reciprocal (FP64 divisions are costly)
    const Real rTM = Real(1) / (Tc * Mg);
    const Real Tr = T * Mg * rTM;                  // T / Tc
    const Real iMg = Tc * rTM;                     // 1 / M
    const Real sTr = M<Real>::sqrt(Tr);
    const Real sMTc = M<Real>::sqrt(Mg * Tc);
    const Real Ts = Real(1.2593) * Tr;
    const Real Fc = Real(1) - Real(0.2756) * omega + Real(0.059035) * mur4 + kap;
    const Real lnTs = M<Real>::log(Ts);
    const Real Ov = Real(1.16145) * M<Real>::exp(Real(-0.14874) * lnTs) + Real(0.52487) * M<Real>::exp(Real(-0.77320) * Ts)
                    + Real(2.16178) * M<Real>::exp(Real(-2.43787) * Ts);
    const Real y = rho_mol * Real(1e-6) * Vc * Real(1.0 / 6.0);
    const Real omy = Real(1) - y;
    const Real omy3 = omy * omy * omy;
    const Real yp = (y > Real(0)) ? y : Real(1);   // y = 0 only for p = 0, kept finite
    const Real ryo = Real(1) / (omy3 * yp);
    const Real G1 = (Real(1) - Real(0.5) * y) * yp * ryo;   // (1 - y/2) / (1 - y)^3
    Real E[10];
#pragma unroll
    for (int i = 0; i < 10; ++i)
        E[i] = chung_visc<Real>(i, 0) + chung_visc<Real>(i, 1) * omega + chung_visc<Real>(i, 2) * mur4 + chung_visc<Real>(i, 3) * kap;
    const Real iy = omy3 * ryo;                    // 1 / y
    const Real fy4 = (y > Real(0)) ? -M<Real>::expm1(-E[3] * y) * iy : E[3];
    const Real nG = E[0] * fy4 + E[1] * G1 * M<Real>::exp(E[4] * y) + E[2] * G1;
    const Real dG = E[0] * E[3] + E[1] + E[2];
    const Real rG = Real(1) / (nG * dG);
    const Real G2 = nG * nG * rG, iG2 = dG * dG * rG;
    const Real rTO = Real(1) / (Ts * Ov);
    const Real iTs = Ov * rTO, iOv = Ts * rTO;
    const Real etass = E[6] * y * y * G2 * M<Real>::exp(E[7] + iTs * (E[8] + E[9] * iTs));
    const Real sqTs = Real(1.1221853679316978) * sTr;   // sqrt(1.2593) sqrt(Tr)
    const Real etas = sqTs * iOv * Fc * (iG2 + E[5] * y) + etass;
    const Real cVc2 = cVc * cVc;
    const Real al = cv_molar * Real(1.0 / kR) - Real(1.5);
    const Real be = Real(0.7862) - Real(0.7109) * omega + Real(1.3168) * omega * omega;
    const Real Zp = Real(2.0) + Real(10.5) * Tr * Tr;
    const Real dPsi = Real(0.6366) + be * Zp + Real(1.061) * al * be;
    const Real rPV = Real(1) / (dPsi * cVc2);
    const Real iVc23 = dPsi * rPV;                 // Vc^(-2/3)
    mu = etas * Real(36.344e-7) * sMTc * iVc23;
    const Real eta0 = Real(40.785e-7) * Fc * (sMTc * sTr) * iVc23 * iOv;   // sqrt(M T)
    Real Bc[7];
#pragma unroll
    for (int i = 0; i < 7; ++i)
        Bc[i] = chung_cond<Real>(i, 0) + chung_cond<Real>(i, 1) * omega + chung_cond<Real>(i, 2) * mur4 + chung_cond<Real>(i, 3) * kap;
    const Real fyb4 = (y > Real(0)) ? -M<Real>::expm1(-Bc[3] * y) * iy : Bc[3];
    const Real nH = Bc[0] * fyb4 + Bc[1] * G1 * M<Real>::exp(Bc[4] * y) + Bc[2] * G1;
    const Real dH = Bc[0] * Bc[3] + Bc[1] + Bc[2];
    const Real rH = Real(1) / (nH * dH);
    const Real H2 = nH * nH * rH, iH2 = dH * dH * rH;
    const Real Psi = Real(1) + al * (Real(0.215) + Real(0.28288) * al - Real(1.061) * be + Real(0.26665) * Zp) *
                                   cVc2 * rPV;
    const Real iMkg = Real(1e3) * iMg;
    const Real q = Real(3.586e-3) * (Real(31.622776601683793) * sMTc * iMg) * iVc23;   // sqrt(Tc / M[kg/mol])
    lam = Real(31.2) * eta0 * Psi * iMkg * (iH2 + Bc[5] * y) + q * Bc[6] * y * y * sTr * H2;
}

// Chung's mixture rules.  With the combining rules sigma_ij = sqrt(sigma_i
// sigma_j), eps_ij = sqrt(eps_i eps_j), omega_ij = (omega_i + omega_j)/2 and
// kappa_ij = sqrt(kappa_i kappa_j), every double sum but the molar-mass one
// is a product of single sums; the molar-mass sum (M_ij harmonic) uses the
// pair table C_ij = sqrt(eps_i eps_j) sigma_i sigma_j sqrt(M_ij).
template <typename Real, int NS>
__device__ __forceinline__ void transport(const Comp<Real, NS> &c, Real T, const Thermo<Real> &th,
                                          const SpeciesRec<Real> *sp, const Real *pair, int flags,
                                          Real &mu, Real &lam)
{
    if (flags & PR_FLAG_TRANSPORT_XAVG) {
        Real m = 0, l = 0;
#pragma unroll 1
        for (int k = 0; k < NS; ++k) {
            // x_k by selects over constant indices: a dynamic index would put
            // the mole fractions of every cell in local memory
            Real xk = 0;
#pragma unroll
            for (int j = 0; j < NS; ++j) xk = (j == k) ? c.x[j] : xk;
            if (xk == Real(0)) continue;
            Real mk, lk;
            chung_dense<Real>(sp[k].Tc, sp[k].Vc, M<Real>::cbrt(sp[k].Vc), sp[k].omega, sp[k].M, sp[k].mur4,
                              sp[k].kap, T, th.rho_mol, th.cv_ig_molar, mk, lk);
            m = M<Real>::fma(xk, mk, m);
            l = M<Real>::fma(xk, lk, l);
        }
        mu = m;
        lam = l;
        return;
    }
    Real P1 = 0, P2 = 0, P3 = 0, P4 = 0, P5 = 0, Q = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        P1 = M<Real>::fma(c.x[i], sp[i].s15, P1);
        P2 = M<Real>::fma(c.x[i], sp[i].e05s15, P2);
        P3 = M<Real>::fma(c.x[i], sp[i].ws15, P3);
        P4 = M<Real>::fma(c.x[i], sp[i].mu2s15, P4);
        P5 = M<Real>::fma(c.x[i], sp[i].sqkap, P5);
        Real t = Real(0.5) * pair[i * NS + i] * c.x[i];
#pragma unroll
        for (int j = i + 1; j < NS; ++j) t = M<Real>::fma(pair[i * NS + j], c.x[j], t);
        Q = M<Real>::fma(Real(2) * c.x[i], t, Q);
    }
    const Real s3 = P1 * P1;                      // sigma_m^3
    const Real iP1 = Real(1) / P1;
    const Real em = P2 * P2 * iP1 * iP1;          // (eps/k)_m
    const Real wm = P3 * iP1;                     // omega_m
    const Real mu4 = s3 * P4 * P4;                // mu_m^4 [debye^4]
    const Real km = P5 * P5;                      // kappa_m
    const Real sm = M<Real>::cbrt(s3);
    const Real sqM = Q / (em * sm * sm);
    const Real Mm = sqM * sqM;
    const Real Vcm = s3 * Real(1.0 / (0.809 * 0.809 * 0.809));
    const Real Tcm = Real(1.2593) * em;
    const Real murd = Real(131.3 * 131.3) / (Vcm * Tcm);   // mu_r^2 / mu^2
    const Real mur4 = mu4 * murd * murd;
    chung_dense<Real>(Tcm, Vcm, sm * Real(1.0 / 0.809), wm, Mm, mur4, km, T, th.rho_mol, th.cv_ig_molar, mu, lam);
}

// FP64 properties of cell i from FP32 inputs, written as FP32 to
// out[q * ldo + i] (q = rho, Z, h, cp, mu, lambda): the Peng-Robinson step
// that replaces the surrogate on a flagged cell.  Inputs are validated as
// load_comp does (positive finite T and p, non-negative finite Y, |sum Y - 1|
// <= 1e-6); a bad input or a cubic without a root Z > B gives NaN outputs.
// sp, pair and kij are the shared-memory copies of the context's tables;
// tmid_u its common NASA-7 switch temperature (or 0), as pr_props uses it, so
// that the cell's values are those of the FP64 property path.
template <int NS, bool KIJ>
__device__ __forceinline__ void fallback_cell_fp64(int64_t i, const float *__restrict__ T,
                                                   const float *__restrict__ p, const float *__restrict__ Y,
                                                   int64_t ldY, float *out, int64_t ldo, const SpeciesRec<double> *sp,
                                                   const double *pair, const double *kij, int N, int flags,
                                                   double tmid_u)
{
    const double Tv = (double)__ldg(T + i), pv = (double)__ldg(p + i);
    Comp<double, NS> c;
    double ysum = 0, s = 0;
    bool ok = (Tv > 0) && (pv > 0) && isfinite(Tv) && isfinite(pv);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const double y = (k < N) ? (double)__ldg(Y + (int64_t)k * ldY + i) : 0.0;
        ok = ok && (y >= 0) && isfinite(y);
        ysum += y;
        c.x[k] = y * sp[k].inv_W;
        s += c.x[k];
    }
    ok = ok && fabs(ysum - 1.0) <= 1e-6 && s > 0;
    const double is = 1.0 / s;
    double bm = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        c.x[k] *= is;
        bm = fma(c.x[k], sp[k].b, bm);
    }
    c.Wbar = is;
    c.bm = bm;
    float o[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) o[q] = __int_as_float(0x7fc00000);
    if (ok) {
        Thermo<double> th;
        thermo<double, double, NS, KIJ>(c, Tv, pv, sp, kij, th, tmid_u);
        if (th.status != kNoRoot) {
            double mu, lam;
            transport<double, NS>(c, Tv, th, sp, pair, flags, mu, lam);
            o[0] = (float)(pv * c.Wbar / (th.Z * kR * Tv));
            o[1] = (float)th.Z;
            o[2] = (float)th.h;
            o[3] = (float)th.cp;
            o[4] = (float)mu;
            o[5] = (float)lam;
        }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) out[(int64_t)q * ldo + i] = o[q];
}

}  // namespace prk
