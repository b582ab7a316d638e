// C ABI of the property library: context creation (species setup kernel),
// argument validation and dispatch of pr_props / pr_T_from_h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <new>

#include "pr_internal.h"
#include "pr_kernels.cuh"

using namespace prk;

namespace prk {
PRK_DECLARE(double, double, 9, extern)
PRK_DECLARE(double, double, 32, extern)
PRK_DECLARE(float, float, 9, extern)
PRK_DECLARE(float, float, 32, extern)
PRK_DECLARE(float, double, 9, extern)
PRK_DECLARE(float, double, 32, extern)
}  // namespace prk

namespace prgb {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

const char *last_error() { return g_err; }

}  // namespace prgb

namespace {

// ----------------------------------------------------------------- setup
struct HostTable {
    double W[PR_MAX_SPECIES], Tc[PR_MAX_SPECIES], pc[PR_MAX_SPECIES], omega[PR_MAX_SPECIES];
    double Vc[PR_MAX_SPECIES], dipole[PR_MAX_SPECIES], kappa[PR_MAX_SPECIES], T_mid[PR_MAX_SPECIES];
    double nasa_lo[PR_MAX_SPECIES][7], nasa_hi[PR_MAX_SPECIES][7];
    double kij[PR_MAX_SPECIES][PR_MAX_SPECIES];
};

// Derive the per-species records from the raw table (one thread per
// species, plus the pair tables).  Entries k >= N are zero records.
__global__ void setup_species_kernel(const HostTable *__restrict__ t, int N, int NS, int flags,
                                     SpeciesRec<double> *sp64, SpeciesRec<float> *sp32,
                                     double *pair64, float *pair32, double *kij64, float *kij32)
{
    const int k = threadIdx.x;
    if (k < NS) {
        SpeciesRec<double> r;
        memset(&r, 0, sizeof(r));
        r.T_mid = 1e30;
        if (k < N) {
            const double Oa = (flags & PR_FLAG_PRINTED_CONSTANTS) ? kOmegaAPrinted : kOmegaA;
            const double Ob = (flags & PR_FLAG_PRINTED_CONSTANTS) ? kOmegaBPrinted : kOmegaB;
            const double Wkg = t->W[k] * 1e-3, Tc = t->Tc[k], pc = t->pc[k], w = t->omega[k];
            r.inv_W = 1.0 / Wkg;
            r.sqrt_ac = sqrt(Oa) * kR * Tc / sqrt(pc);
            r.b = Ob * kR * Tc / pc;
            r.kappa = 0.37464 + 1.54226 * w - 0.26992 * w * w;
            r.kq = r.kappa / sqrt(Tc);
            r.T_mid = t->T_mid[k];
            for (int j = 0; j < 5; ++j) {
                r.cp_lo[j] = kR * t->nasa_lo[k][j];
                r.cp_hi[j] = kR * t->nasa_hi[k][j];
                r.h_lo[j] = kR * t->nasa_lo[k][j] / (j + 1);
                r.h_hi[j] = kR * t->nasa_hi[k][j] / (j + 1);
            }
            r.h_lo[5] = kR * t->nasa_lo[k][5];
            r.h_hi[5] = kR * t->nasa_hi[k][5];
            const double sig = 0.809 * cbrt(t->Vc[k]);
            const double eps = Tc / 1.2593;
            r.s15 = sig * sqrt(sig);
            r.e05s15 = sqrt(eps) * r.s15;
            r.ws15 = w * r.s15;
            r.mu2s15 = t->dipole[k] * t->dipole[k] / r.s15;
            r.sqkap = sqrt(t->kappa[k]);
            r.Tc = Tc;
            r.Vc = t->Vc[k];
            r.omega = w;
            r.M = t->W[k];
            const double mur = 131.3 * t->dipole[k] / sqrt(t->Vc[k] * Tc);
            r.mur4 = mur * mur * mur * mur;
            r.kap = t->kappa[k];
        }
        sp64[k] = r;
        SpeciesRec<float> f;
        const double *src = reinterpret_cast<const double *>(&r);
        float *dst = reinterpret_cast<float *>(&f);
        for (size_t j = 0; j < sizeof(r) / sizeof(double); ++j) dst[j] = (float)src[j];
        sp32[k] = f;
    }
    for (int idx = threadIdx.x; idx < NS * NS; idx += blockDim.x) {
        const int i = idx / NS, j = idx % NS;
        double c = 0.0, w1 = 0.0;
        if (i < N && j < N) {
            const double si = 0.809 * cbrt(t->Vc[i]), sj = 0.809 * cbrt(t->Vc[j]);
            const double ei = t->Tc[i] / 1.2593, ej = t->Tc[j] / 1.2593;
            const double Mij = 2.0 * t->W[i] * t->W[j] / (t->W[i] + t->W[j]);
            c = sqrt(ei * ej) * si * sj * sqrt(Mij);
            w1 = 1.0 - t->kij[i][j];
        }
        pair64[idx] = c;
        pair32[idx] = (float)c;
        kij64[idx] = w1;
        kij32[idx] = (float)w1;
    }
}


template <typename Real, typename RZ>
void fill_occ(int NS, int occ_p[2], int occ_n[2])
{
    if (NS == 9) {
        occupancy_props<Real, RZ, 9>(occ_p);
        occupancy_newton<Real, RZ, 9>(occ_n);
    } else {
        occupancy_props<Real, RZ, 32>(occ_p);
        occupancy_newton<Real, RZ, 32>(occ_n);
    }
}

bool bad_double(double v) { return !std::isfinite(v); }

}  // namespace

// ===================================================================== ABI
extern "C" {

const char *pr_last_error(void) { return prgb::last_error(); }

const char *pr_version(void) { return "prgb300 0.1 (sm_103a)"; }

pr_status pr_create(const pr_species_table *tbl, pr_ctx **out)
{
    PR_CHECK_ARG(tbl != nullptr && out != nullptr, "pr_create: null argument");
    *out = nullptr;
    const int N = tbl->n_species;
    PR_CHECK_ARG(N >= 1 && N <= PR_MAX_SPECIES, "pr_create: n_species=%d outside 1..%d", N, PR_MAX_SPECIES);
    PR_CHECK_ARG(tbl->W && tbl->Tc && tbl->pc && tbl->omega && tbl->Vc && tbl->dipole && tbl->kappa &&
                     tbl->nasa_lo && tbl->nasa_hi && tbl->T_mid,
                 "pr_create: null species array");
    PR_CHECK_ARG((tbl->flags & ~(PR_FLAG_PRINTED_CONSTANTS | PR_FLAG_TRANSPORT_XAVG | PR_FLAG_NEWTON_FP64_ONLY)) == 0,
                 "pr_create: unknown flags 0x%x", tbl->flags);
    HostTable *h = new (std::nothrow) HostTable();
    if (!h) { prgb::set_error("pr_create: host allocation failed"); return PR_ENOMEM; }
    bool has_kij = false;
    for (int k = 0; k < N; ++k) {
        h->W[k] = tbl->W[k]; h->Tc[k] = tbl->Tc[k]; h->pc[k] = tbl->pc[k]; h->omega[k] = tbl->omega[k];
        h->Vc[k] = tbl->Vc[k]; h->dipole[k] = tbl->dipole[k]; h->kappa[k] = tbl->kappa[k]; h->T_mid[k] = tbl->T_mid[k];
        bool bad = !(h->W[k] > 0) || !(h->Tc[k] > 0) || !(h->pc[k] > 0) || !(h->Vc[k] > 0) || !(h->kappa[k] >= 0) ||
                   bad_double(h->omega[k]) || bad_double(h->dipole[k]) || bad_double(h->T_mid[k]) ||
                   bad_double(h->W[k]) || bad_double(h->Tc[k]) || bad_double(h->pc[k]) || bad_double(h->Vc[k]);
        for (int j = 0; j < 7; ++j) {
            h->nasa_lo[k][j] = tbl->nasa_lo[7 * k + j];
            h->nasa_hi[k][j] = tbl->nasa_hi[7 * k + j];
            bad = bad || bad_double(h->nasa_lo[k][j]) || bad_double(h->nasa_hi[k][j]);
        }
        if (bad) { delete h; prgb::set_error("pr_create: invalid data for species %d", k); return PR_EINVAL; }
        for (int j = 0; j < N; ++j) {
            const double v = tbl->kij ? tbl->kij[k * N + j] : 0.0;
            if (bad_double(v)) { delete h; prgb::set_error("pr_create: kij not finite"); return PR_EINVAL; }
            h->kij[k][j] = v;
            has_kij = has_kij || (v != 0.0);
        }
    }
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
            if (h->kij[k][j] != h->kij[j][k]) {
                delete h;
                prgb::set_error("pr_create: kij must be symmetric");
                return PR_EINVAL;
            }

    pr_ctx *c = new (std::nothrow) pr_ctx();
    if (!c) { delete h; prgb::set_error("pr_create: host allocation failed"); return PR_ENOMEM; }
    c->n_species = N;
    c->ns_pad = (N <= 9) ? 9 : 32;
    c->flags = tbl->flags;
    c->has_kij = has_kij;
    const int NS = c->ns_pad;
    HostTable *d_tab = nullptr;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_sp64, NS * sizeof(SpeciesRec<double>));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_sp32, NS * sizeof(SpeciesRec<float>));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_pair64, NS * NS * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_pair32, NS * NS * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_kij64, NS * NS * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_kij32, NS * NS * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_tab, sizeof(HostTable));
    if (e == cudaSuccess) e = cudaMemcpy(d_tab, h, sizeof(HostTable), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        setup_species_kernel<<<1, 64>>>(d_tab, N, NS, c->flags, (SpeciesRec<double> *)c->d_sp64,
                                        (SpeciesRec<float> *)c->d_sp32, c->d_pair64, c->d_pair32, c->d_kij64,
                                        c->d_kij32);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && NS == 9) {
        HostTab9<double> *t64 = new (std::nothrow) HostTab9<double>();
        HostTab9<float> *t32 = new (std::nothrow) HostTab9<float>();
        c->h_tab64 = t64;
        c->h_tab32 = t32;
        if (!t64 || !t32) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaMemcpy(t64->sp, c->d_sp64, sizeof(t64->sp), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(t64->pair, c->d_pair64, sizeof(t64->pair), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(t64->kij, c->d_kij64, sizeof(t64->kij), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(t32->sp, c->d_sp32, sizeof(t32->sp), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(t32->pair, c->d_pair32, sizeof(t32->pair), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(t32->kij, c->d_kij32, sizeof(t32->kij), cudaMemcpyDeviceToHost);
    }
    // one NASA-7 switch temperature for every species: the ideal-gas sums then
    // take one range test per cell
    c->tmid_u = h->T_mid[0] > 0 ? h->T_mid[0] : 0.0;
    for (int k = 1; k < N; ++k)
        if (h->T_mid[k] != h->T_mid[0]) c->tmid_u = 0.0;
    if (d_tab) cudaFree(d_tab);
    delete h;
    if (e != cudaSuccess) {
        prgb::set_error("pr_create: %s", cudaGetErrorString(e));
        pr_destroy(c);
        return (e == cudaErrorMemoryAllocation) ? PR_ENOMEM : PR_ECUDA;
    }
    if (pr_status ss = prgb::species_tables_init(c, tbl)) {
        pr_destroy(c);
        return ss;
    }
    fill_occ<double, double>(NS, c->occ_props[PR_FP64], c->occ_newton[PR_FP64]);
    fill_occ<float, float>(NS, c->occ_props[PR_FP32], c->occ_newton[PR_FP32]);
    fill_occ<float, double>(NS, c->occ_props[PR_MIXED], c->occ_newton[PR_MIXED]);
    // with the context's device current; a failed lookup only disables
    // pr_fallback_props_noalloc (which then reports it)
    if (prgb::noalloc_scratch_address(&c->noalloc_scratch) != PR_OK) {
        c->noalloc_scratch = nullptr;
        prgb::set_error("");
    }
    *out = c;
    return PR_OK;
}

void pr_destroy(pr_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    cudaFree(c->d_sp64);
    cudaFree(c->d_sp32);
    cudaFree(c->d_pair64);
    cudaFree(c->d_pair32);
    cudaFree(c->d_kij64);
    cudaFree(c->d_kij32);
    prgb::species_tables_free(c);
    delete static_cast<HostTab9<double> *>(c->h_tab64);
    delete static_cast<HostTab9<float> *>(c->h_tab32);
    delete c;
}

static pr_status check_arrays(int64_t n, size_t esz, std::initializer_list<const void *> req,
                              std::initializer_list<const void *> opt, const char *fn)
{
    for (const void *p : req) {
        PR_CHECK_ARG(p != nullptr, "%s: required array is NULL", fn);
        PR_CHECK_ARG(prgb::aligned(p, esz), "%s: array not aligned to %zu bytes", fn, esz);
    }
    for (const void *p : opt) PR_CHECK_ARG(prgb::aligned(p, esz), "%s: array not aligned to %zu bytes", fn, esz);
    (void)n;
    return PR_OK;
}

static pr_status props_impl(pr_ctx *ctx, pr_precision prec, int64_t n, const void *T, const void *p, const void *Y,
                            int64_t ldY, void *rho, void *Z, void *h, void *cp, void *mu, void *lambda, void *psi,
                            void *alpha, int32_t *cell_status, void *stream)
{
    PR_CHECK_ARG(ctx != nullptr, "pr_props: null context");
    PR_CHECK_ARG(prec == PR_FP64 || prec == PR_FP32 || prec == PR_MIXED, "pr_props: bad precision %d", (int)prec);
    PR_CHECK_ARG(n >= 0, "pr_props: n < 0");
    if (n == 0) return PR_OK;
    PR_CHECK_ARG(ldY >= n, "pr_props: ldY (%lld) < n (%lld)", (long long)ldY, (long long)n);
    const size_t esz = (prec == PR_FP64) ? 8 : 4;
    pr_status s = check_arrays(n, esz, {T, p, Y}, {rho, Z, h, cp, mu, lambda, psi, alpha}, "pr_props");
    if (s) return s;
    PR_CHECK_ARG(prgb::aligned(cell_status, 4), "pr_props: cell_status misaligned");
    cudaStream_t st = (cudaStream_t)stream;
    const bool kij = ctx->has_kij;
    const int occ = ctx->occ_props[prec][kij ? 1 : 0];
    if (prec == PR_FP64) {
        PropsArgs<double> a{n, ldY, (const double *)T, (const double *)p, (const double *)Y, (double *)rho,
                            (double *)Z, (double *)h, (double *)cp, (double *)mu, (double *)lambda, cell_status,
                            (const SpeciesRec<double> *)ctx->d_sp64, ctx->d_pair64, ctx->d_kij64,
                            ctx->n_species, ctx->flags, (double *)psi, (double *)alpha, ctx->tmid_u};
        if (ctx->ns_pad == 9) launch_props<double, double, 9>(a, ctx->h_tab64, kij, occ, ctx->num_sms, st);
        else launch_props<double, double, 32>(a, nullptr, kij, occ, ctx->num_sms, st);
    } else {
        PropsArgs<float> a{n, ldY, (const float *)T, (const float *)p, (const float *)Y, (float *)rho,
                           (float *)Z, (float *)h, (float *)cp, (float *)mu, (float *)lambda, cell_status,
                           (const SpeciesRec<float> *)ctx->d_sp32, ctx->d_pair32, ctx->d_kij32,
                           ctx->n_species, ctx->flags, (float *)psi, (float *)alpha, (float)ctx->tmid_u};
        if (prec == PR_FP32) {
            if (ctx->ns_pad == 9) launch_props<float, float, 9>(a, ctx->h_tab32, kij, occ, ctx->num_sms, st);
            else launch_props<float, float, 32>(a, nullptr, kij, occ, ctx->num_sms, st);
        } else {
            if (ctx->ns_pad == 9) launch_props<float, double, 9>(a, ctx->h_tab32, kij, occ, ctx->num_sms, st);
            else launch_props<float, double, 32>(a, nullptr, kij, occ, ctx->num_sms, st);
        }
    }
    PR_CUDA_TRY(cudaGetLastError());
    return PR_OK;
}

pr_status pr_props(pr_ctx *ctx, pr_precision prec, int64_t n, const void *T, const void *p, const void *Y,
                   int64_t ldY, void *rho, void *Z, void *h, void *cp, void *mu, void *lambda,
                   int32_t *cell_status, void *stream)
{
    return props_impl(ctx, prec, n, T, p, Y, ldY, rho, Z, h, cp, mu, lambda, nullptr, nullptr, cell_status, stream);
}

pr_status pr_props_ext(pr_ctx *ctx, pr_precision prec, int64_t n, const void *T, const void *p, const void *Y,
                       int64_t ldY, void *rho, void *Z, void *h, void *cp, void *mu, void *lambda, void *psi,
                       void *alpha, int32_t *cell_status, void *stream)
{
    return props_impl(ctx, prec, n, T, p, Y, ldY, rho, Z, h, cp, mu, lambda, psi, alpha, cell_status, stream);
}

pr_status pr_T_from_h(pr_ctx *ctx, pr_precision prec, int64_t n, const void *hstar, const void *p, const void *Y,
                      int64_t ldY, const void *T_guess, void *T_out, int32_t *cell_status, int32_t *iters,
                      int max_iter, double rtol, void *stream)
{
    PR_CHECK_ARG(ctx != nullptr, "pr_T_from_h: null context");
    PR_CHECK_ARG(prec == PR_FP64 || prec == PR_FP32 || prec == PR_MIXED, "pr_T_from_h: bad precision %d", (int)prec);
    PR_CHECK_ARG(n >= 0, "pr_T_from_h: n < 0");
    PR_CHECK_ARG(max_iter >= 1 && max_iter <= 1000, "pr_T_from_h: max_iter %d outside 1..1000", max_iter);
    PR_CHECK_ARG(rtol >= 1e-15 && rtol <= 1e-2, "pr_T_from_h: rtol %g outside [1e-15, 1e-2]", rtol);
    if (n == 0) return PR_OK;
    PR_CHECK_ARG(ldY >= n, "pr_T_from_h: ldY < n");
    const size_t esz = (prec == PR_FP64) ? 8 : 4;
    pr_status s = check_arrays(n, esz, {hstar, p, Y, T_guess, T_out}, {}, "pr_T_from_h");
    if (s) return s;
    PR_CHECK_ARG(cell_status != nullptr && prgb::aligned(cell_status, 4), "pr_T_from_h: cell_status required");
    PR_CHECK_ARG(prgb::aligned(iters, 4), "pr_T_from_h: iters misaligned");
    cudaStream_t st = (cudaStream_t)stream;
    const bool kij = ctx->has_kij;
    const int occ = ctx->occ_newton[prec][kij ? 1 : 0];
    if (prec == PR_FP64) {
        NewtonArgs<double> a{n, ldY, (const double *)hstar, (const double *)p, (const double *)Y,
                             (const double *)T_guess, (double *)T_out, cell_status, iters,
                             (const SpeciesRec<double> *)ctx->d_sp64, ctx->d_pair64, ctx->d_kij64,
                             ctx->n_species, ctx->flags, max_iter, rtol,
                             (const SpeciesRec<float> *)ctx->d_sp32, ctx->d_pair32, ctx->d_kij32,
                             nullptr, nullptr, nullptr, ctx->tmid_u};
        if (ctx->ns_pad == 9) launch_newton<double, double, 9>(a, kij, occ, ctx->num_sms, st);
        else launch_newton<double, double, 32>(a, kij, occ, ctx->num_sms, st);
    } else {
        NewtonArgs<float> a{n, ldY, (const float *)hstar, (const float *)p, (const float *)Y, (const float *)T_guess,
                            (float *)T_out, cell_status, iters, (const SpeciesRec<float> *)ctx->d_sp32,
                            ctx->d_pair32, ctx->d_kij32, ctx->n_species, ctx->flags, max_iter, rtol,
                            nullptr, nullptr, nullptr,
                            (const SpeciesRec<double> *)ctx->d_sp64, ctx->d_pair64, ctx->d_kij64, ctx->tmid_u};
        if (prec == PR_FP32) {
            if (ctx->ns_pad == 9) launch_newton<float, float, 9>(a, kij, occ, ctx->num_sms, st);
            else launch_newton<float, float, 32>(a, kij, occ, ctx->num_sms, st);
        } else {
            if (ctx->ns_pad == 9) launch_newton<float, double, 9>(a, kij, occ, ctx->num_sms, st);
            else launch_newton<float, double, 32>(a, kij, occ, ctx->num_sms, st);
        }
    }
    PR_CUDA_TRY(cudaGetLastError());
    return PR_OK;
}

}  // extern "C"
