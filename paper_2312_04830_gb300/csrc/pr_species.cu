// Per-species outputs of the property networks (Sec. 4.1 lists, among the
// seven networks, the nondimensional standard-state enthalpies and the
// mixture-averaged diffusion coefficients of every species; Sec. 2 names the
// binary diffusion model with Takahashi's high-pressure correction):
//
//   h_k^0 / (R T)   NASA-7 fit of species k;
//   D_km            = (1 - Y_k) / sum_{j != k} X_j / D_kj  (mass-fraction form
//                     of the mixture average), 1 - Y_k evaluated as
//                     sum_{j != k} Y_j / sum_j Y_j (no cancellation as Y_k -> 1,
//                     which FP32 inputs reach), a species alone in its cell
//                     taking its self-diffusion coefficient D_kk;
//   D_kj            Chapman-Enskog, D_kj = c_kj T^(3/2) / (p Omega_D(T / eps_kj)),
//                     c_kj = 0.0266 / (M_kj^(1/2) sigma_kj^2) [m^2 Pa/(s K^1.5)]
//                     (0.00266 cm^2 bar units), Neufeld's Omega_D,
//                     sigma = 0.809 Vc^(1/3) [A], eps/k = Tc / 1.2593 (Chung's
//                     corresponding states), sigma_kj arithmetic, eps_kj
//                     geometric, M_kj = 2 / (1/W_k + 1/W_j) [g/mol];
//   f(T_r, p_r)     optional caller table multiplying every D_kj p, bilinear
//                     and edge-clamped, at the mixture's Kay's-rule state.
//
// One thread per cell.  The pair terms are symmetric, so each unordered pair
// evaluates its collision integral once and feeds both species' sums.  In
// Neufeld's Omega_D = A T*^-B + C e^(-D T*) + E e^(-F T*) + G e^(-H T*) the
// power term factors as A T^-B eps_kj^B (one power per cell, a constant per
// pair), and an exponential term whose argument exceeds 40 is dropped: it is
// below 8e-18 while Omega_D >= 0.4, under half an FP64 ulp of the sum.  Pair
// constants (1/eps, eps^B, 1/c) are derived on the host when the context is
// created and staged in shared memory per CTA.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "pr_device.cuh"
#include "pr_internal.h"
#include "pr_species.cuh"

namespace {

using prk::M;
using prk::SpeciesRec;
using prs::corr_factor;
using prs::dtab_len;
using prs::omega_d;

constexpr int kSpBlock = 128;
constexpr int kCorrMax = 64;
constexpr int kCorrFloats = 2 * kCorrMax + kCorrMax * kCorrMax;

template <typename Real>
struct SpArgs {
    int64_t n, ldY, ldo;
    const Real *T, *p, *Y;
    Real *hk, *Dk;
    int32_t *status;
    const SpeciesRec<Real> *sp;
    const Real *dtab;
    const Real *corr;     // Tr[cT], pr[cP], f[cT][cP]; cT = 0: no correction
    int N, cT, cP;
};

template <typename Real, int NS>
__global__ void __launch_bounds__(kSpBlock) species_kernel(const SpArgs<Real> a)
{
    __shared__ Real s_h[2][NS][6];
    __shared__ Real s_tmid[NS], s_iW[NS];
    __shared__ Real s_tab[2 * NS + 3 * NS * NS];
    for (int e = threadIdx.x; e < NS * 6; e += blockDim.x) {
        const int k = e / 6, j = e % 6;
        s_h[0][k][j] = a.sp[k].h_lo[j];
        s_h[1][k][j] = a.sp[k].h_hi[j];
    }
    for (int k = threadIdx.x; k < NS; k += blockDim.x) {
        s_tmid[k] = a.sp[k].T_mid;
        s_iW[k] = a.sp[k].inv_W;
    }
    for (int e = threadIdx.x; e < 2 * NS + 3 * NS * NS; e += blockDim.x) s_tab[e] = a.dtab[e];
    __syncthreads();

    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const Real T = __ldg(a.T + i), p = __ldg(a.p + i);
        Real y[NS], x[NS];
        Real ysum = 0, s = 0;
        bool ok = (T > Real(0)) && (p > Real(0)) && M<Real>::finite(T) && M<Real>::finite(p);
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            y[k] = (k < a.N) ? __ldg(a.Y + (int64_t)k * a.ldY + i) : Real(0);
            ok = ok && (y[k] >= Real(0)) && M<Real>::finite(y[k]);
            ysum += y[k];
            x[k] = y[k] * s_iW[k];
            s += x[k];
        }
        ok = ok && (M<Real>::fabs(ysum - Real(1)) <= Real(1e-6)) && (s > Real(0));
        if (a.status) a.status[i] = ok ? prk::kOk : prk::kBadInput;
        if (!ok) {
            const Real nanv = M<Real>::nan();
            for (int k = 0; k < a.N; ++k) {
                if (a.hk) a.hk[(int64_t)k * a.ldo + i] = nanv;
                if (a.Dk) a.Dk[(int64_t)k * a.ldo + i] = nanv;
            }
            continue;
        }
        if (a.hk) {
            const Real iRT = Real(1) / (Real(prk::kR) * T);
#pragma unroll
            for (int k = 0; k < NS; ++k) {
                if (k >= a.N) break;
                a.hk[(int64_t)k * a.ldo + i] = prs::h_over_RT<Real>(s_h[T < s_tmid[k] ? 0 : 1][k], T, iRT);
            }
        }
        if (a.Dk) {
            const Real inv_s = Real(1) / s;
#pragma unroll
            for (int k = 0; k < NS; ++k) x[k] *= inv_s;
            Real D[NS];
            prs::diffusion_cell<Real, NS>(y, x, ysum, T, p, a.N, s_tab, a.corr, a.cT, a.cP, D);
#pragma unroll
            for (int k = 0; k < NS; ++k) {
                if (k >= a.N) break;
                a.Dk[(int64_t)k * a.ldo + i] = D[k];
            }
        }
    }
}

// Bilger's mixture fraction per cell: Z = (sum_k b_k Y_k - beta_ox) / (beta_fuel - beta_ox).
template <typename Real>
__global__ void __launch_bounds__(kSpBlock) bilger_kernel(int64_t n, const Real *__restrict__ Y, int64_t ldY,
                                                          int N, const Real *__restrict__ coef, Real *Z)
{
    const Real bo = coef[N], ir = coef[N + 1];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        Real beta = 0;
        for (int k = 0; k < N; ++k) beta = M<Real>::fma(__ldg(coef + k), __ldg(Y + (int64_t)k * ldY + i), beta);
        Z[i] = (beta - bo) * ir;
    }
}

template <typename Real, int NS>
void launch_species(const SpArgs<Real> &a, int occ, int sms, cudaStream_t st)
{
    int64_t need = (a.n + kSpBlock - 1) / kSpBlock;
    const int64_t cap = (int64_t)occ * sms;
    const int g = (int)(need < cap ? need : cap);
    species_kernel<Real, NS><<<g, kSpBlock, 0, st>>>(a);
}

template <typename Real, int NS>
int occ_of()
{
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, species_kernel<Real, NS>, kSpBlock, 0);
    return o > 0 ? o : 1;
}

}  // namespace

namespace prgb {

// Pair constants from the validated species table (entries of species >= N
// are zero and never read).
pr_status species_tables_init(pr_ctx *c, const pr_species_table *tbl)
{
    const int N = tbl->n_species, NS = c->ns_pad;
    std::vector<double> t(dtab_len(NS), 0.0);
    double *tc = t.data(), *pc = tc + NS, *ie = pc + NS, *epsB = ie + NS * NS, *ic = epsB + NS * NS;
    for (int k = 0; k < N; ++k) {
        tc[k] = tbl->Tc[k];
        pc[k] = tbl->pc[k];
    }
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j) {
            const double sk = 0.809 * std::cbrt(tbl->Vc[k]), sj = 0.809 * std::cbrt(tbl->Vc[j]);
            const double sig = 0.5 * (sk + sj);
            const double eps = std::sqrt((tbl->Tc[k] / 1.2593) * (tbl->Tc[j] / 1.2593));
            const double Mkj = 2.0 / (1.0 / tbl->W[k] + 1.0 / tbl->W[j]);
            const double ckj = 0.0266 / (std::sqrt(Mkj) * sig * sig);
            ie[k * NS + j] = 1.0 / eps;
            epsB[k * NS + j] = std::pow(eps, prs::kNB);
            ic[k * NS + j] = 1.0 / ckj;
        }
    std::vector<float> t32(t.size());
    for (size_t e = 0; e < t.size(); ++e) t32[e] = (float)t[e];
    PR_CUDA_TRY(cudaMalloc(&c->d_dtab64, t.size() * sizeof(double)));
    PR_CUDA_TRY(cudaMalloc(&c->d_dtab32, t.size() * sizeof(float)));
    PR_CUDA_TRY(cudaMalloc(&c->d_corr64, kCorrFloats * sizeof(double)));
    PR_CUDA_TRY(cudaMalloc(&c->d_corr32, kCorrFloats * sizeof(float)));
    PR_CUDA_TRY(cudaMalloc(&c->d_bilger64, (N + 2) * sizeof(double)));
    PR_CUDA_TRY(cudaMalloc(&c->d_bilger32, (N + 2) * sizeof(float)));
    c->has_bilger = 0;
    PR_CUDA_TRY(cudaMemcpy(c->d_dtab64, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
    PR_CUDA_TRY(cudaMemcpy(c->d_dtab32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice));
    c->corr_nT = c->corr_nP = 0;
    c->occ_species[0] = (NS == 9) ? occ_of<double, 9>() : occ_of<double, 32>();
    c->occ_species[1] = (NS == 9) ? occ_of<float, 9>() : occ_of<float, 32>();
    return PR_OK;
}

void species_tables_free(pr_ctx *c)
{
    cudaFree(c->d_dtab64);
    cudaFree(c->d_dtab32);
    cudaFree(c->d_corr64);
    cudaFree(c->d_corr32);
    cudaFree(c->d_bilger64);
    cudaFree(c->d_bilger32);
}

}  // namespace prgb

extern "C" {

pr_status pr_set_diffusion_correction(pr_ctx *ctx, const pr_diffusion_correction *corr)
{
    PR_CHECK_ARG(ctx != nullptr, "pr_set_diffusion_correction: null context");
    if (corr == nullptr) {
        PR_CUDA_TRY(cudaDeviceSynchronize());
        ctx->corr_nT = ctx->corr_nP = 0;
        return PR_OK;
    }
    const int nT = corr->n_Tr, nP = corr->n_pr;
    PR_CHECK_ARG(nT >= 2 && nT <= kCorrMax && nP >= 2 && nP <= kCorrMax,
                 "pr_set_diffusion_correction: table %d x %d outside 2..%d", nT, nP, kCorrMax);
    PR_CHECK_ARG(corr->Tr && corr->pr && corr->f, "pr_set_diffusion_correction: null array");
    for (int i = 0; i < nT; ++i)
        PR_CHECK_ARG(std::isfinite(corr->Tr[i]) && (i == 0 || corr->Tr[i] > corr->Tr[i - 1]),
                     "pr_set_diffusion_correction: Tr must be finite and strictly increasing");
    for (int j = 0; j < nP; ++j)
        PR_CHECK_ARG(std::isfinite(corr->pr[j]) && (j == 0 || corr->pr[j] > corr->pr[j - 1]),
                     "pr_set_diffusion_correction: pr must be finite and strictly increasing");
    for (int e = 0; e < nT * nP; ++e)
        PR_CHECK_ARG(std::isfinite(corr->f[e]) && corr->f[e] >= 0.0,
                     "pr_set_diffusion_correction: factors must be finite and >= 0");
    std::vector<double> t(nT + nP + nT * nP);
    std::memcpy(t.data(), corr->Tr, nT * sizeof(double));
    std::memcpy(t.data() + nT, corr->pr, nP * sizeof(double));
    std::memcpy(t.data() + nT + nP, corr->f, (size_t)nT * nP * sizeof(double));
    std::vector<float> t32(t.size());
    for (size_t e = 0; e < t.size(); ++e) t32[e] = (float)t[e];
    PR_CUDA_TRY(cudaDeviceSynchronize());
    PR_CUDA_TRY(cudaMemcpy(ctx->d_corr64, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
    PR_CUDA_TRY(cudaMemcpy(ctx->d_corr32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice));
    ctx->corr_nT = nT;
    ctx->corr_nP = nP;
    return PR_OK;
}

pr_status pr_set_bilger(pr_ctx *ctx, const int32_t *atoms, const double *Y_fuel, const double *Y_ox)
{
    PR_CHECK_ARG(ctx != nullptr && atoms != nullptr && Y_fuel != nullptr && Y_ox != nullptr,
                 "pr_set_bilger: null argument");
    const int N = ctx->n_species;
    // species molar masses back from the device records (1 / inv_W, kg -> g)
    std::vector<prk::SpeciesRec<double>> sp(ctx->ns_pad);
    PR_CUDA_TRY(cudaMemcpy(sp.data(), ctx->d_sp64, sp.size() * sizeof(sp[0]), cudaMemcpyDeviceToHost));
    // [N] coefficients b_k, then beta_ox and 1 / (beta_fuel - beta_ox)
    std::vector<double> packed(N + 2, 0.0);
    double bf = 0.0, bo = 0.0;
    for (int k = 0; k < N; ++k) {
        PR_CHECK_ARG(atoms[3 * k] >= 0 && atoms[3 * k + 1] >= 0 && atoms[3 * k + 2] >= 0,
                     "pr_set_bilger: negative atom count for species %d", k);
        PR_CHECK_ARG(std::isfinite(Y_fuel[k]) && std::isfinite(Y_ox[k]), "pr_set_bilger: stream not finite");
        const double Wg = 1e3 / sp[k].inv_W;
        // beta = 2 n_C + n_H / 2 - n_O, n_e = sum_k a_ek Y_k / W_k (moles of element per gram)
        packed[k] = (2.0 * atoms[3 * k] + 0.5 * atoms[3 * k + 1] - 1.0 * atoms[3 * k + 2]) / Wg;
        bf += packed[k] * Y_fuel[k];
        bo += packed[k] * Y_ox[k];
    }
    PR_CHECK_ARG(bf != bo, "pr_set_bilger: fuel and oxidiser streams have the same coupling function");
    packed[N] = bo;
    packed[N + 1] = 1.0 / (bf - bo);
    std::vector<float> p32(packed.begin(), packed.end());
    PR_CUDA_TRY(cudaDeviceSynchronize());
    PR_CUDA_TRY(cudaMemcpy(ctx->d_bilger64, packed.data(), packed.size() * sizeof(double), cudaMemcpyHostToDevice));
    PR_CUDA_TRY(cudaMemcpy(ctx->d_bilger32, p32.data(), p32.size() * sizeof(float), cudaMemcpyHostToDevice));
    ctx->has_bilger = 1;
    return PR_OK;
}

pr_status pr_bilger_z(pr_ctx *ctx, pr_precision prec, int64_t n, const void *Y, int64_t ldY, void *Z, void *stream)
{
    PR_CHECK_ARG(ctx != nullptr, "pr_bilger_z: null context");
    PR_CHECK_ARG(ctx->has_bilger, "pr_bilger_z: no element table set (pr_set_bilger)");
    PR_CHECK_ARG(prec == PR_FP64 || prec == PR_FP32 || prec == PR_MIXED, "pr_bilger_z: bad precision %d", (int)prec);
    PR_CHECK_ARG(n >= 0, "pr_bilger_z: n < 0");
    if (n == 0) return PR_OK;
    PR_CHECK_ARG(ldY >= n, "pr_bilger_z: ldY < n");
    const size_t esz = (prec == PR_FP64) ? 8 : 4;
    PR_CHECK_ARG(Y != nullptr && Z != nullptr, "pr_bilger_z: null array");
    PR_CHECK_ARG(prgb::aligned(Y, esz) && prgb::aligned(Z, esz), "pr_bilger_z: array not aligned to %zu bytes", esz);
    int64_t need = (n + kSpBlock - 1) / kSpBlock;
    const int64_t cap = (int64_t)ctx->num_sms * 16;
    const int g = (int)(need < cap ? need : cap);
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == PR_FP64)
        bilger_kernel<double><<<g, kSpBlock, 0, st>>>(n, (const double *)Y, ldY, ctx->n_species, ctx->d_bilger64,
                                                      (double *)Z);
    else
        bilger_kernel<float><<<g, kSpBlock, 0, st>>>(n, (const float *)Y, ldY, ctx->n_species, ctx->d_bilger32,
                                                     (float *)Z);
    PR_CUDA_TRY(cudaGetLastError());
    return PR_OK;
}

pr_status pr_species_props(pr_ctx *ctx, pr_precision prec, int64_t n, const void *T, const void *p, const void *Y,
                           int64_t ldY, void *hk_RT, void *Dk, int64_t ldo, int32_t *cell_status, void *stream)
{
    PR_CHECK_ARG(ctx != nullptr, "pr_species_props: null context");
    PR_CHECK_ARG(prec == PR_FP64 || prec == PR_FP32 || prec == PR_MIXED, "pr_species_props: bad precision %d",
                 (int)prec);
    PR_CHECK_ARG(n >= 0, "pr_species_props: n < 0");
    if (n == 0) return PR_OK;
    PR_CHECK_ARG(ldY >= n, "pr_species_props: ldY (%lld) < n (%lld)", (long long)ldY, (long long)n);
    PR_CHECK_ARG((hk_RT == nullptr && Dk == nullptr) || ldo >= n, "pr_species_props: ldo (%lld) < n (%lld)",
                 (long long)ldo, (long long)n);
    const size_t esz = (prec == PR_FP64) ? 8 : 4;
    for (const void *q : {T, p, Y}) {
        PR_CHECK_ARG(q != nullptr, "pr_species_props: required array is NULL");
        PR_CHECK_ARG(prgb::aligned(q, esz), "pr_species_props: array not aligned to %zu bytes", esz);
    }
    for (const void *q : {hk_RT, Dk})
        PR_CHECK_ARG(prgb::aligned(q, esz), "pr_species_props: array not aligned to %zu bytes", esz);
    PR_CHECK_ARG(prgb::aligned(cell_status, 4), "pr_species_props: cell_status misaligned");
    cudaStream_t st = (cudaStream_t)stream;
    const bool nine = ctx->ns_pad == 9;
    if (prec == PR_FP64) {
        SpArgs<double> a{n, ldY, ldo, (const double *)T, (const double *)p, (const double *)Y, (double *)hk_RT,
                         (double *)Dk, cell_status, (const SpeciesRec<double> *)ctx->d_sp64, ctx->d_dtab64,
                         ctx->d_corr64, ctx->n_species, ctx->corr_nT, ctx->corr_nP};
        if (nine) launch_species<double, 9>(a, ctx->occ_species[0], ctx->num_sms, st);
        else launch_species<double, 32>(a, ctx->occ_species[0], ctx->num_sms, st);
    } else {
        SpArgs<float> a{n, ldY, ldo, (const float *)T, (const float *)p, (const float *)Y, (float *)hk_RT,
                        (float *)Dk, cell_status, (const SpeciesRec<float> *)ctx->d_sp32, ctx->d_dtab32,
                        ctx->d_corr32, ctx->n_species, ctx->corr_nT, ctx->corr_nP};
        if (nine) launch_species<float, 9>(a, ctx->occ_species[1], ctx->num_sms, st);
        else launch_species<float, 32>(a, ctx->occ_species[1], ctx->num_sms, st);
    }
    PR_CUDA_TRY(cudaGetLastError());
    return PR_OK;
}

}  // extern "C"
