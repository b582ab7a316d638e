// Per-cell arithmetic of the per-species outputs (Sec. 4.1's species
// networks: standard-state enthalpies and mixture-averaged diffusion with a
// high-pressure correction, Sec. 2), shared by pr_species_props and the
// surrogate's FP64 fallback for its per-species outputs.
//
//   D_km = (sum_{j != k} Y_j / sum_j Y_j) / sum_{j != k} X_j / D_kj, the
//   Chapman-Enskog D_kj = c_kj T^(3/2) / (p Omega_D(T / eps_kj)) from the pair
//   table (1/eps, eps^B, 1/c), times the correction f(T_r, p_r) at the mixture's
//   Kay's-rule state; a species alone in its cell gets D_kk.
#pragma once

#include "pr_device.cuh"

namespace prs {

using prk::M;

// Neufeld et al. (1972) fit of the Lennard-Jones Omega^(1,1)*.
constexpr double kNA = 1.06036, kNB = 0.15610, kNC = 0.19300, kND = 0.47635;
constexpr double kNE = 1.03587, kNF = 1.52996, kNG = 1.76474, kNH = 3.89411;

// Flat per-context table: tc[NS], pc[NS], ie[NS*NS], epsB[NS*NS], ic[NS*NS].
inline size_t dtab_len(int NS) { return 2 * (size_t)NS + 3 * (size_t)NS * NS; }

// Omega_D at T* = Ts, with pw = T*^-B given.
template <typename Real>
__device__ __forceinline__ Real omega_d(Real Ts, Real pw)
{
    Real om = Real(kNA) * pw;
    if (Ts < Real(40.0 / kND)) om = M<Real>::fma(Real(kNC), M<Real>::exp(Real(-kND) * Ts), om);
    if (Ts < Real(40.0 / kNF)) om = M<Real>::fma(Real(kNE), M<Real>::exp(Real(-kNF) * Ts), om);
    if (Ts < Real(40.0 / kNH)) om = M<Real>::fma(Real(kNG), M<Real>::exp(Real(-kNH) * Ts), om);
    return om;
}

// Bilinear, clamped to the table's edges.
template <typename Real>
__device__ __forceinline__ Real corr_factor(const Real *__restrict__ c, int cT, int cP, Real x, Real y)
{
    const Real *Tr = c, *pr = c + cT, *f = c + cT + cP;
    x = fmin(fmax(x, Tr[0]), Tr[cT - 1]);
    y = fmin(fmax(y, pr[0]), pr[cP - 1]);
    int i = 0, j = 0;
    while (i < cT - 2 && x > Tr[i + 1]) ++i;
    while (j < cP - 2 && y > pr[j + 1]) ++j;
    const Real tx = (x - Tr[i]) / (Tr[i + 1] - Tr[i]);
    const Real ty = (y - pr[j]) / (pr[j + 1] - pr[j]);
    const Real *r0 = f + i * cP + j, *r1 = r0 + cP;
    const Real g0 = M<Real>::fma(ty, r0[1] - r0[0], r0[0]);
    const Real g1 = M<Real>::fma(ty, r1[1] - r1[0], r1[0]);
    return M<Real>::fma(tx, g1 - g0, g0);
}

// Mixture-averaged D_k [m^2/s] of one valid cell: y its mass fractions
// (ysum their sum), x its mole fractions (normalised), tab the flat pair table,
// corr the correction table (cT = 0: none).
template <typename Real, int NS>
__device__ __forceinline__ void diffusion_cell(const Real (&y)[NS], const Real (&x)[NS], Real ysum, Real T, Real p,
                                               int N, const Real *tab, const Real *corr, int cT, int cP, Real (&D)[NS])
{
    const Real *tc = tab, *pc = tab + NS, *ie = tab + 2 * NS, *epsB = ie + NS * NS, *ic = epsB + NS * NS;
    Real Tpc = 0, ppc = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        Tpc = M<Real>::fma(x[k], tc[k], Tpc);
        ppc = M<Real>::fma(x[k], pc[k], ppc);
    }
    const Real f = (cT > 0) ? corr_factor<Real>(corr, cT, cP, T / Tpc, p / ppc) : Real(1);
    const Real TmB = M<Real>::exp(Real(-kNB) * M<Real>::log(T));   // T^-B
    Real acc[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) acc[k] = 0;
#pragma unroll
    for (int k = 0; k < NS - 1; ++k) {
        if (k >= N - 1) break;
#pragma unroll
        for (int j = k + 1; j < NS; ++j) {
            if (j >= N) break;
            const int q = k * NS + j;
            const Real om = omega_d<Real>(T * ie[q], TmB * epsB[q]);
            const Real w = om * ic[q];
            acc[k] = M<Real>::fma(x[j], w, acc[k]);
            acc[j] = M<Real>::fma(x[k], w, acc[j]);
        }
    }
    const Real scale = f * T * M<Real>::sqrt(T) / p;   // f T^(3/2) / p
    // sum_{j != k} y_j from prefix and suffix sums
    Real others[NS];
    Real run = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        others[k] = run;
        run += y[k];
    }
    run = 0;
#pragma unroll
    for (int k = NS - 1; k >= 0; --k) {
        others[k] += run;
        run += y[k];
    }
    const Real iys = Real(1) / ysum;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        if (k >= N) break;
        if (acc[k] > Real(0)) {
            D[k] = others[k] * iys * scale / acc[k];
        } else {   // alone in the cell: self-diffusion
            const int q = k * NS + k;
            D[k] = scale / (omega_d<Real>(T * ie[q], TmB * epsB[q]) * ic[q]);
        }
    }
}

// h_k^0 / (R T) of one species from its NASA-7 enthalpy record e (molar h =
// ((((e4 T + e3) T + e2) T + e1) T + e0) T + e5) and iRT = 1 / (R T).
template <typename Real>
__device__ __forceinline__ Real h_over_RT(const Real *e, Real T, Real iRT)
{
    const Real h = M<Real>::fma(
        M<Real>::fma(M<Real>::fma(M<Real>::fma(M<Real>::fma(e[4], T, e[3]), T, e[2]), T, e[1]), T, e[0]), T, e[5]);
    return h * iRT;
}

}  // namespace prs
