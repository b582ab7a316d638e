// Kernel templates of the forward-property and inversion paths, and their
// launchers.  Instantiated per precision in pr_inst_{fp64,fp32,mixed}.cu so
// that the three precisions compile in parallel.
//
// Kernel layout: persistent grid-stride CTAs of 128 threads, one cell per
// thread per iteration.  Each CTA stages the species records, the Chung pair
// table and (if any) the (1 - k_ij) matrix into shared memory once, then walks
// the cells.  Cell arrays are read and written coalesced (SoA, consecutive
// threads on consecutive cells).
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "pr_device.cuh"

namespace prk {

constexpr int kBlock = 128;

// --------------------------------------------------------- shared staging
template <typename Real, int NS, bool KIJ>
struct Smem {
    SpeciesRec<Real> sp[NS];
    Real pair[NS * NS];
    Real kij[KIJ ? NS * NS : 1];
};

template <typename Real, int NS, bool KIJ>
__device__ __forceinline__ void stage(Smem<Real, NS, KIJ> &s, const SpeciesRec<Real> *sp, const Real *pair,
                                      const Real *kij)
{
    const Real *src = reinterpret_cast<const Real *>(sp);
    Real *dst = reinterpret_cast<Real *>(s.sp);
    constexpr int nw = NS * sizeof(SpeciesRec<Real>) / sizeof(Real);
    for (int j = threadIdx.x; j < nw; j += blockDim.x) dst[j] = src[j];
    for (int j = threadIdx.x; j < NS * NS; j += blockDim.x) s.pair[j] = pair[j];
    if (KIJ)
        for (int j = threadIdx.x; j < NS * NS; j += blockDim.x) s.kij[j] = kij[j];
    __syncthreads();
}

// ------------------------------------------------ tables in parameter space
// The property kernels of up to 9 species take the species records and pair
// tables by value, in the kernel's parameter space (a constant bank): with
// the species loops unrolled, every table entry becomes a constant operand of
// the instruction that uses it, with no load instruction (the shared-memory
// staging above costs one load per entry and use).  Larger tables (the
// 32-species kernels) stay in shared memory.
template <typename Real, int NS, bool KIJ>
struct ParamTab {
    SpeciesRec<Real> sp[NS];
    Real pair[NS * NS];
    Real kij[KIJ ? NS * NS : 1];
};
struct NoTab {
    int unused;
};
template <typename Real, int NS, bool KIJ>
using TabArg = typename std::conditional<NS == 9, ParamTab<Real, 9, KIJ>, NoTab>::type;

// Host image of a 9-species context's tables (pair and (1 - k_ij) [9][9]).
template <typename Real>
struct HostTab9 {
    SpeciesRec<Real> sp[9];
    Real pair[81];
    Real kij[81];
};

template <typename Real, int NS, bool KIJ>
inline TabArg<Real, NS, KIJ> make_tab(const void *host)
{
    TabArg<Real, NS, KIJ> t;
    memset(&t, 0, sizeof(t));
    if constexpr (NS == 9) {
        const HostTab9<Real> *h = static_cast<const HostTab9<Real> *>(host);
        memcpy(t.sp, h->sp, sizeof(t.sp));
        memcpy(t.pair, h->pair, sizeof(t.pair));
        if (KIJ) memcpy(t.kij, h->kij, sizeof(t.kij));
    }
    return t;
}

// ----------------------------------------------------------- props kernel
template <typename Real>
struct PropsArgs {
    int64_t n, ldY;
    const Real *T, *p, *Y;
    Real *rho, *Z, *h, *cp, *mu, *lam;
    int32_t *status;
    const SpeciesRec<Real> *sp;
    const Real *pair, *kij;
    int N, flags;
    Real *psi, *alpha;   // (d rho/d p)_h [s^2/m^2], lambda/cp [kg/(m s)]; NULL to skip
    Real tmid_u;         // common NASA-7 switch temperature of every species, or 0
};

// psi = (d rho / d p) at constant h (Sec. 4.1) from the EOS partials of the
// cell: (d rho/d p)_T + (d rho/d T)_p (d T/d p)_h, (d T/d p)_h =
// -(d h/d p)_T / cp, (d h/d p)_T = V - T (d V/d T)_p, (d V/d T)_p = -(dp/dT)_V
// / (dp/dV)_T; molar V, cp, mean molar mass W.
template <typename Real>
__device__ __forceinline__ Real psi_h(const Thermo<Real> &th, Real T, Real W)
{
    const Real V = Real(1) / th.rho_mol;
    const Real iV2 = th.rho_mol * th.rho_mol;
    const Real dV_dT = -th.dpdT / th.dpdV;
    const Real drho_dp_T = -W * iV2 / th.dpdV;
    const Real drho_dT_p = -W * iV2 * dV_dT;
    const Real dh_dp_T = V - T * dV_dT;
    return drho_dp_T - drho_dT_p * dh_dp_T / (th.cp * W);
}

// resident CTAs per SM the property kernels ask the compiler to allow for
// (a register cap; 0 leaves the choice to the compiler)
#ifndef PRK_FP32_MINB
#define PRK_FP32_MINB 0
#endif
#ifndef PRK_FP64_MINB
#define PRK_FP64_MINB 0
#endif
template <typename Real>
constexpr int props_min_blocks() { return sizeof(Real) == 4 ? PRK_FP32_MINB : PRK_FP64_MINB; }

template <typename Real, typename RZ, int NS, bool KIJ>
__global__ void __launch_bounds__(kBlock, props_min_blocks<Real>()) props_kernel(const __grid_constant__ PropsArgs<Real> a,
                                                       const __grid_constant__ TabArg<Real, NS, KIJ> t)
{
    constexpr bool kParam = NS == 9;
    __shared__ typename std::conditional<kParam, char, Smem<Real, NS, KIJ>>::type s_[1];
    const SpeciesRec<Real> *sp;
    const Real *pair, *kij;
    if constexpr (kParam) {
        sp = t.sp;
        pair = t.pair;
        kij = t.kij;
    } else {
        stage<Real, NS, KIJ>(s_[0], a.sp, a.pair, a.kij);
        sp = s_[0].sp;
        pair = s_[0].pair;
        kij = s_[0].kij;
    }
    const bool want_tr = (a.mu != nullptr) || (a.lam != nullptr) || (a.alpha != nullptr);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const Real T = __ldg(a.T + i), p = __ldg(a.p + i);
        Comp<Real, NS> c;
        bool ok = load_comp<Real, NS>(c, a.Y, a.ldY, i, a.N, sp);
        ok = ok && (T > Real(0)) && (p > Real(0)) && M<Real>::finite(T) && M<Real>::finite(p);
        Thermo<Real> th;
        th.status = kBadInput;
        Real mu = M<Real>::nan(), lam = M<Real>::nan();
        if (ok) {
            thermo<Real, RZ, NS, KIJ>(c, T, p, sp, kij, th, a.tmid_u);
            if (th.status != kNoRoot && want_tr) transport<Real, NS>(c, T, th, sp, pair, a.flags, mu, lam);
        }
        const bool good = ok && th.status != kNoRoot;
        const Real nanv = M<Real>::nan();
        if (a.rho) a.rho[i] = good ? p * c.Wbar / (th.Z * Real(kR) * T) : nanv;
        if (a.Z) a.Z[i] = good ? th.Z : nanv;
        if (a.h) a.h[i] = good ? th.h : nanv;
        if (a.cp) a.cp[i] = good ? th.cp : nanv;
        if (a.mu) a.mu[i] = good ? mu : nanv;
        if (a.lam) a.lam[i] = good ? lam : nanv;
        if (a.psi) a.psi[i] = good ? psi_h<Real>(th, T, c.Wbar) : nanv;
        if (a.alpha) a.alpha[i] = good ? lam / th.cp : nanv;
        if (a.status) a.status[i] = th.status;
    }
}

// ---------------------------------------------------------- Newton kernel
template <typename Real>
struct NewtonArgs {
    int64_t n, ldY;
    const Real *hstar, *p, *Y, *Tg;
    Real *Tout;
    int32_t *status, *iters;
    const SpeciesRec<Real> *sp;
    const Real *pair, *kij;
    int N, flags, max_iter;
    double rtol;
    // FP32 tables for the warm start of the FP64 inversion (FP64 kernel only)
    const SpeciesRec<float> *sp32;
    const float *pair32, *kij32;
    // FP64 tables for the FP64 re-solve of the mixed inversion (mixed kernel only)
    const SpeciesRec<double> *sp64;
    const double *pair64, *kij64;
    double tmid_u;   // common NASA-7 switch temperature of every species, or 0
};

// h(T) and cp(T) of a cell at fixed p and composition; status 0 or an error.
template <typename Real, typename RZ, int NS, bool KIJ>
__device__ __noinline__ int eval_h(const Comp<Real, NS> &c, double T, Real p, const SpeciesRec<Real> *sp,
                                      const Real *kij, Real tmid_u, double &h, double &cp)
{
    Thermo<Real> th;
    thermo<Real, RZ, NS, KIJ>(c, (Real)T, p, sp, kij, th, tmid_u);
    if (th.status == kNoRoot) return kNoRoot;
    h = (double)th.h;
    cp = (double)th.cp;
    return kOk;
}

// The first FP64 evaluation of the inversion after the FP32 warm start: h,
// and what the one-step acceptance below needs, the root count and the
// ideal-gas molar cv.  cp is not evaluated in FP64 here: the step and the
// acceptance take the FP32 cp at the same T (the warm start's), whose
// relative error (~1e-6) moves a step of at most 1e-6 T by ~1e-12 T.
struct FirstEval {
    int status;        // the thermodynamics' status (kOk, kAmbiguous or kNoRoot)
    int nroots;        // physical roots of the cubic
    double h, cp;      // J/kg; J/(kg K), set by the caller
    float cv_ig;       // ideal-gas molar cv [J/(mol K)]
};

template <typename Real, typename RZ, int NS, bool KIJ>
__device__ __noinline__ FirstEval eval_h_first(const Comp<Real, NS> &c, double T, Real p, const SpeciesRec<Real> *sp,
                                               const Real *kij, Real tmid_u)
{
    Thermo<Real> th;
    thermo<Real, RZ, NS, KIJ, false>(c, (Real)T, p, sp, kij, th, tmid_u);
    FirstEval f;
    f.status = th.status;
    f.nroots = th.status == kNoRoot ? 0 : th.nroots;
    f.h = (double)th.h;
    f.cp = 0.0;
    f.cv_ig = (float)th.cv_ig_molar;
    return f;
}

// One-step acceptance of the FP64 inversion.  After the FP32 warm start, a
// Newton step dT from T on a smooth branch of h(T) leaves an error
// |e| <= (kappa / 2) (dT / T)^2 T, kappa = T |dcp/dT| / cp (Newton's
// quadratic convergence), plus |dT| times the relative error of the cp it
// divides by (the FP32 cp: ~1e-6).  The step T + dT is taken without a second
// FP64 evaluation when |dT| <= kAcceptStep T (e <= kappa 5e-13 T + 1e-12 T), the cubic has
// a single physical root (no phase branch nearby), cp is below the
// pseudo-boiling band (cp <= kPseudoCriticalCp x the ideal-gas cp, where
// kappa stays O(10)), and no kink of h(T) -- a species' NASA-7 range switch
// or the zero of its alpha factor 1 + kappa_k (1 - sqrt(T / Tc_k)) -- lies
// within 10 |dT| + 1e-5 T of T (checked in FP32 from the FP32 tables).  Other
// cells continue the safeguarded iteration from this evaluation.
constexpr double kAcceptStep = 1e-6;

template <int NS>
__device__ __forceinline__ bool one_step_ok(const FirstEval &f, double T, double dT, double Wbar,
                                            const SpeciesRec<float> *sp32, float tmid_u)
{
    constexpr double kPseudoCp = 3.0;   // as kPseudoCriticalCp below
    if (f.status != kOk || f.nroots != 1 || !(f.cp > 0.0)) return false;
    if (!(fabs(dT) <= kAcceptStep * T)) return false;
    const double T1 = T + dT;
    if (!(T1 > kTLo && T1 < kTHi)) return false;
    if (!((float)f.cp * (float)Wbar <= (float)kPseudoCp * (f.cv_ig + (float)kR))) return false;
    const float Tf = (float)T, margin = 10.f * fabsf((float)dT) + 1e-5f * Tf;
    bool clear = true;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const float tm = tmid_u > 0.f ? tmid_u : sp32[k].T_mid;
        clear = clear && fabsf(Tf - tm) > margin;
        const float kq = sp32[k].kq;
        if (kq > 0.f) {
            const float r = (1.f + sp32[k].kappa) / kq;   // sqrt of the alpha factor's zero
            clear = clear && fabsf(Tf - r * r) > margin;
        }
    }
    return clear;
}

// h(T) and cp(T) in FP32 with FP32 arguments (the warm start's evaluations).
template <int NS, bool KIJ>
__device__ __noinline__ int eval_h_f32(const Comp<float, NS> &c, float T, float p, const SpeciesRec<float> *sp,
                                       const float *kij, float tmid_u, float &h, float &cp)
{
    Thermo<float> th;
    thermo<float, float, NS, KIJ>(c, T, p, sp, kij, th, tmid_u);
    if (th.status == kNoRoot) return kNoRoot;
    h = th.h;
    cp = th.cp;
    return kOk;
}

// Warm start of the FP64 inversion: plain Newton on the FP32 thermodynamics
// from T0 until a step is below 1e-5 T (at most 8 steps).  Returns the FP32
// root, or T0 when a step fails, leaves [kTLo, kTHi] or does not settle (the
// FP64 iteration then starts from T0 as it would without a warm start).  The
// update runs in FP32 as well (h* rounded to FP32 moves the root by less than
// the FP32 enthalpy's own error), so the FP64 pipe only does the final
// conversion.  cp_end: the FP32 cp at the returned root (0 if that
// evaluation fails), for the first FP64 step.
template <int NS, bool KIJ>
__device__ __noinline__ double warm_start_fp32(const Comp<double, NS> &c64, double T0, double hs, double p,
                                               const SpeciesRec<float> *sp, const float *kij, float tmid_u, bool &ok,
                                               float &cp_end)
{
    ok = false;
    cp_end = 0.f;
    Comp<float, NS> c;
#pragma unroll
    for (int k = 0; k < NS; ++k) c.x[k] = (float)c64.x[k];
    c.Wbar = (float)c64.Wbar;
    c.bm = (float)c64.bm;
    const float hsf = (float)hs, pf = (float)p;
    float T = (float)T0;
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        float h, cp;
        if (eval_h_f32<NS, KIJ>(c, T, pf, sp, kij, tmid_u, h, cp) || !(cp > 0.f)) return T0;
        const float Tn = T - (h - hsf) / cp;
        if (!(Tn > (float)kTLo && Tn < (float)kTHi)) return T0;
        const bool done = fabsf(Tn - T) <= 1e-5f * Tn;
        T = Tn;
        if (done) {
            ok = true;
            float he, cpe;
            if (!eval_h_f32<NS, KIJ>(c, T, pf, sp, kij, tmid_u, he, cpe) && cpe > 0.f) cp_end = cpe;
            return (double)T;
        }
    }
    return T0;
}

// Safeguarded Newton on f(T) = h(T) - h* from T inside [kTLo, kTHi]: a step
// that leaves the bracket, or follows one that did not halve |f|, becomes a
// bisection; before leaning on a bracket end whose h is unknown, h* is checked
// to lie inside the range.  Converged when |f| <= rtol max(|h*|, cp T), or
// when |dT| <= rtol T and h at the new T is within jump_tol (else h* sits in a
// jump of h(T)).  Returns the status; Tres, iters and the last cp out.
template <typename Real, typename RZ, int NS, bool KIJ>
__device__ __forceinline__ int newton_solve(const Comp<Real, NS> &c, double hs, Real p, double T,
                                            const SpeciesRec<Real> *sp, const Real *kij, Real tmid_u, int max_iter,
                                            double rtol, double jump_tol, double &Tres, int &iters, double &cp_last,
                                            bool first_given = false, double h0 = 0.0, double cp0 = 0.0)
{
    double lo = kTLo, hi = kTHi;
    bool lo_done = false, hi_done = false;   // endpoint h evaluated (range checked)
    double fprev = INFINITY;
    int st = kMaxIt, it;
    Tres = T;
    cp_last = 0.0;
#pragma unroll 1
    for (it = 1; it <= max_iter; ++it) {
        double h = h0, cp = cp0;   // the first evaluation, when the caller made it
        if (it > 1 || !first_given) {
            int e = eval_h<Real, RZ, NS, KIJ>(c, T, p, sp, kij, tmid_u, h, cp);
            if (e) { st = e; Tres = T; break; }
        }
        cp_last = cp;
        const double f = h - hs;
        if (fabs(f) <= rtol * fmax(fabs(hs), fabs(cp) * T)) { st = kOk; Tres = T; break; }
        if (f < 0) lo = T; else hi = T;
        double Tn = T - f / cp;
        const bool newton_ok = (cp > 0) && (Tn > lo) && (Tn < hi) && (fabs(f) <= 0.5 * fabs(fprev));
        if (!newton_ok) Tn = 0.5 * (lo + hi);
        if (!newton_ok && ((lo == kTLo && !lo_done) || (hi == kTHi && !hi_done))) {
            const bool use_lo = (lo == kTLo && !lo_done);
            const double Te = use_lo ? kTLo : kTHi;
            double he, cpe;
            int e2 = eval_h<Real, RZ, NS, KIJ>(c, Te, p, sp, kij, tmid_u, he, cpe);
            if (e2) { st = e2; Tres = T; break; }
            if (use_lo) lo_done = true; else hi_done = true;
            if ((use_lo && hs < he) || (!use_lo && hs > he)) { st = kHRange; Tres = Te; break; }
        }
        fprev = f;
        if (fabs(Tn - T) <= rtol * T) {
            Tres = Tn;
            double h2, cp2;
            if (eval_h<Real, RZ, NS, KIJ>(c, Tn, p, sp, kij, tmid_u, h2, cp2)) { st = kNoRoot; break; }
            cp_last = cp2;
            st = (fabs(h2 - hs) <= jump_tol * fmax(fabs(hs), fabs(cp2) * Tn)) ? kOk : kHRange;
            break;
        }
        T = Tn;
        Tres = T;
    }
    iters = it > max_iter ? max_iter : it;
    return st;
}

// Mass-specific ideal-gas cp of a cell [J/(kg K)] (NASA-7).
template <typename Real, int NS>
__device__ __forceinline__ double cp_ideal_mass(const Comp<Real, NS> &c, Real T, const SpeciesRec<Real> *sp)
{
    Real s = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const Real *a = (T < sp[k].T_mid) ? sp[k].cp_lo : sp[k].cp_hi;
        const Real cpk = M<Real>::fma(M<Real>::fma(M<Real>::fma(M<Real>::fma(a[4], T, a[3]), T, a[2]), T, a[1]), T, a[0]);
        s = M<Real>::fma(c.x[k], cpk, s);
    }
    return (double)s / (double)c.Wbar;
}

// Composition in FP64 from FP32 mass fractions (the FP64 re-solve of the
// mixed inversion works on exactly the caller's FP32 inputs).
template <int NS>
__device__ __forceinline__ bool comp_fp64_of_fp32(Comp<double, NS> &c, const float *__restrict__ Y, int64_t ldY,
                                                  int64_t i, int N, const SpeciesRec<double> *sp)
{
    double ysum = 0, s = 0;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const double y = (k < N) ? (double)__ldg(Y + (int64_t)k * ldY + i) : 0.0;
        ok = ok && (y >= 0.0) && isfinite(y);
        ysum += y;
        c.x[k] = y * sp[k].inv_W;
        s += c.x[k];
    }
    ok = ok && (fabs(ysum - 1.0) <= 1e-6) && (s > 0.0);
    const double inv_s = 1.0 / s;
    double bm = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        c.x[k] *= inv_s;
        bm = fma(c.x[k], sp[k].b, bm);
    }
    c.Wbar = inv_s;
    c.bm = bm;
    return ok;
}

// cp above this multiple of the ideal-gas cp marks the pseudo-boiling band
// (and the near-critical region), where the mixed inversion re-solves in FP64.
constexpr double kPseudoCriticalCp = 3.0;

// The FP64 inversion with the FP32 warm start: every cell first tries the
// one-step acceptance (one FP64 evaluation); the others -- and cells whose
// warm start failed -- go into a block-wide queue with that evaluation, and
// whenever the queue holds a block's worth, all threads of the block finish
// those cells by the safeguarded iteration together, so its longer iterations
// run in full warps instead of holding back warps whose other cells are done.
template <int NS, bool KIJ>
__device__ __forceinline__ void newton_fp64_queued(const NewtonArgs<double> &a, const Smem<double, NS, KIJ> &s,
                                                   const Smem<float, NS, KIJ> &s32, int64_t stride, double rtol,
                                                   double jump_tol)
{
    __shared__ int q_n;
    __shared__ int64_t q_i[2 * kBlock];
    __shared__ double q_T[2 * kBlock], q_h[2 * kBlock], q_cp[2 * kBlock];
    __shared__ unsigned char q_first[2 * kBlock];
    if (threadIdx.x == 0) q_n = 0;
    __syncthreads();
    // a queued cell through the safeguarded iteration (from its first
    // evaluation when it has one)
    auto finish = [&](int e) {
        const int64_t i = q_i[e];
        Comp<double, NS> c;
        load_comp<double, NS>(c, a.Y, a.ldY, i, a.N, s.sp);
        double Tres, cp_last;
        int it;
        const int st = newton_solve<double, double, NS, KIJ>(c, (double)__ldg(a.hstar + i), __ldg(a.p + i), q_T[e],
                                                             s.sp, s.kij, a.tmid_u, a.max_iter, rtol, jump_tol, Tres,
                                                             it, cp_last, q_first[e] != 0, q_h[e], q_cp[e]);
        a.Tout[i] = Tres;
        a.status[i] = st;
        if (a.iters) a.iters[i] = it;
    };
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += stride) {
        const int64_t i = base + threadIdx.x;
        if (i < a.n) {
            const double hs = __ldg(a.hstar + i);
            const double p = __ldg(a.p + i);
            const double Tg = __ldg(a.Tg + i);
            Comp<double, NS> c;
            bool ok = load_comp<double, NS>(c, a.Y, a.ldY, i, a.N, s.sp);
            ok = ok && isfinite(hs) && isfinite(Tg) && (p > 0.0) && isfinite(p);
            if (!ok) {
                a.Tout[i] = nan("");
                a.status[i] = kBadInput;
                if (a.iters) a.iters[i] = 0;
            } else {
                bool wok;
                float cp32;
                const double T = warm_start_fp32<NS, KIJ>(c, fmin(fmax(Tg, kTLo), kTHi), hs, p, s32.sp, s32.kij,
                                                          (float)a.tmid_u, wok, cp32);
                bool accepted = false, first = false;
                double h0 = 0.0, cp0 = 0.0;
                if (wok && cp32 > 0.f) {
                    FirstEval f = eval_h_first<double, double, NS, KIJ>(c, T, p, s.sp, s.kij, a.tmid_u);
                    f.cp = (double)cp32;
                    if (f.status != kNoRoot) {
                        const double dT = (f.cp > 0.0) ? -(f.h - hs) / f.cp : 0.0;
                        if (one_step_ok<NS>(f, T, dT, c.Wbar, s32.sp, (float)a.tmid_u)) {
                            a.Tout[i] = T + dT;
                            a.status[i] = kOk;
                            if (a.iters) a.iters[i] = 1;
                            accepted = true;
                        } else {
                            first = true;
                            h0 = f.h;
                            cp0 = f.cp;
                        }
                    }
                }
                if (!accepted) {   // the safeguarded iteration, in a full batch of the block
                    const int e = atomicAdd(&q_n, 1);
                    q_i[e] = i;
                    q_T[e] = T;
                    q_h[e] = h0;
                    q_cp[e] = cp0;
                    q_first[e] = first ? 1 : 0;
                }
            }
        }
        __syncthreads();
        while (q_n >= (int)blockDim.x) {
            finish(q_n - (int)blockDim.x + (int)threadIdx.x);
            __syncthreads();
            if (threadIdx.x == 0) q_n -= (int)blockDim.x;
            __syncthreads();
        }
    }
    if ((int)threadIdx.x < q_n) finish((int)threadIdx.x);
}

template <typename Real, typename RZ, int NS, bool KIJ>
__global__ void __launch_bounds__(kBlock) newton_kernel(const NewtonArgs<Real> a)
{
    __shared__ Smem<Real, NS, KIJ> s;
    stage<Real, NS, KIJ>(s, a.sp, a.pair, a.kij);
    // FP64 inversion: FP32 tables for the warm start
    constexpr bool kFp64 = sizeof(Real) == 8;
    __shared__ Smem<float, NS, KIJ> s32[1];
    const bool warm = kFp64 && !(a.flags & PR_FLAG_NEWTON_FP64_ONLY);
    if (warm) stage<float, NS, KIJ>(s32[0], a.sp32, a.pair32, a.kij32);
    // mixed inversion (FP32 with the FP64 cubic): FP64 tables for the re-solve
    constexpr bool kMixed = sizeof(Real) == 4 && sizeof(RZ) == 8;
    __shared__ typename std::conditional<kMixed, Smem<double, NS, KIJ>, char>::type s64[1];
    if constexpr (kMixed) stage<double, NS, KIJ>(s64[0], a.sp64, a.pair64, a.kij64);
    // FP32 thermodynamics resolve h to ~1e-7 of its scale: floor the tolerance
    const double rtol = (sizeof(Real) == 4) ? fmax(a.rtol, 2e-6) : a.rtol;
    const double jump_tol = (sizeof(Real) == 4) ? 2e-5 : 1e-6;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if constexpr (kFp64) {
        if (warm) {
            newton_fp64_queued<NS, KIJ>(a, s, s32[0], stride, rtol, jump_tol);
            return;
        }
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const double hs = (double)__ldg(a.hstar + i);
        const Real p = __ldg(a.p + i);
        const double Tg = (double)__ldg(a.Tg + i);
        Comp<Real, NS> c;
        bool ok = load_comp<Real, NS>(c, a.Y, a.ldY, i, a.N, s.sp);
        ok = ok && isfinite(hs) && isfinite(Tg) && (p > Real(0)) && M<Real>::finite(p);
        int st = kBadInput, it = 0;
        double Tres = nan("");
        if (ok) {
            double T = fmin(fmax(Tg, kTLo), kTHi);
            double cp_last;
            st = newton_solve<Real, RZ, NS, KIJ>(c, hs, p, T, s.sp, s.kij, (Real)a.tmid_u, a.max_iter, rtol, jump_tol,
                                                 Tres, it, cp_last);
            if constexpr (kMixed) {
                // FP64 where FP32 is least reliable: failed cells, and cells in
                // the pseudo-boiling band, from the FP32 root (or the guess)
                const bool band = st == kOk && cp_last > kPseudoCriticalCp * cp_ideal_mass<Real, NS>(c, (Real)Tres, s.sp);
                if (st != kOk || band) {
                    Comp<double, NS> c64;
                    if (comp_fp64_of_fp32<NS>(c64, a.Y, a.ldY, i, a.N, s64[0].sp)) {
                        const double T0 = (st == kOk) ? Tres : fmin(fmax(Tg, kTLo), kTHi);
                        double T64, cp64;
                        int it64;
                        st = newton_solve<double, double, NS, KIJ>(c64, hs, (double)p, T0, s64[0].sp, s64[0].kij,
                                                                   a.tmid_u, a.max_iter, a.rtol, 1e-6, T64, it64, cp64);
                        Tres = T64;
                        it += it64;
                    }
                }
            }
        }
        a.Tout[i] = (Real)Tres;
        a.status[i] = st;
        if (a.iters) a.iters[i] = it;
    }
}


// ------------------------------------------------------------- launchers
inline int grid_for(int64_t n, int occ, int sms)
{
    int64_t need = (n + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)occ * sms;
    return (int)(need < cap ? need : cap);
}

// htab: the context's HostTab9<Real> (used when NS == 9)
template <typename Real, typename RZ, int NS>
void launch_props(const PropsArgs<Real> &a, const void *htab, bool kij, int occ, int sms, cudaStream_t st)
{
    const int g = grid_for(a.n, occ, sms);
    if (kij) props_kernel<Real, RZ, NS, true><<<g, kBlock, 0, st>>>(a, make_tab<Real, NS, true>(htab));
    else props_kernel<Real, RZ, NS, false><<<g, kBlock, 0, st>>>(a, make_tab<Real, NS, false>(htab));
}

template <typename Real, typename RZ, int NS>
void launch_newton(const NewtonArgs<Real> &a, bool kij, int occ, int sms, cudaStream_t st)
{
    const int g = grid_for(a.n, occ, sms);
    if (kij) newton_kernel<Real, RZ, NS, true><<<g, kBlock, 0, st>>>(a);
    else newton_kernel<Real, RZ, NS, false><<<g, kBlock, 0, st>>>(a);
}

// resident CTAs per SM of the property kernels (occ[0..1]: kij off/on) and of
// the inversion kernels of one (Real, RZ, NS)
template <typename Real, typename RZ, int NS>
void occupancy_props(int occ[2])
{
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], props_kernel<Real, RZ, NS, false>, kBlock, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], props_kernel<Real, RZ, NS, true>, kBlock, 0);
    for (int k = 0; k < 2; ++k) occ[k] = occ[k] > 0 ? occ[k] : 1;
}

template <typename Real, typename RZ, int NS>
void occupancy_newton(int occ[2])
{
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], newton_kernel<Real, RZ, NS, false>, kBlock, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], newton_kernel<Real, RZ, NS, true>, kBlock, 0);
    for (int k = 0; k < 2; ++k) occ[k] = occ[k] > 0 ? occ[k] : 1;
}

// Explicit instantiations, one translation unit per (precision, kernel kind) so
// that each can take its own compiler flags.
#define PRK_DECLARE_PROPS(Real, RZ, NS, EXT)                                                              \
    EXT template void launch_props<Real, RZ, NS>(const PropsArgs<Real> &, const void *, bool, int, int, cudaStream_t); \
    EXT template void occupancy_props<Real, RZ, NS>(int *);
#define PRK_DECLARE_NEWTON(Real, RZ, NS, EXT)                                                             \
    EXT template void launch_newton<Real, RZ, NS>(const NewtonArgs<Real> &, bool, int, int, cudaStream_t); \
    EXT template void occupancy_newton<Real, RZ, NS>(int *);
#define PRK_DECLARE(Real, RZ, NS, EXT) PRK_DECLARE_PROPS(Real, RZ, NS, EXT) PRK_DECLARE_NEWTON(Real, RZ, NS, EXT)

}  // namespace prk
