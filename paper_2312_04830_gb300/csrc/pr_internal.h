// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "prgb300.h"

namespace prgb {

// Thread-local error message, returned by pr_last_error().
void set_error(const char *fmt, ...);
const char *last_error();

#define PR_CUDA_TRY(call)                                                                 \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ::prgb::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return PR_ECUDA;                                                              \
        }                                                                                 \
    } while (0)

#define PR_CHECK_ARG(cond, ...)                 \
    do {                                        \
        if (!(cond)) {                          \
            ::prgb::set_error(__VA_ARGS__);     \
            return PR_EINVAL;                   \
        }                                       \
    } while (0)

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace prgb

// The context: species data on the device in FP64 and FP32, launch limits.
struct pr_ctx {
    int device;
    int n_species;
    int ns_pad;          // compiled species bound used for this table (9 or 32)
    int flags;
    bool has_kij;
    int num_sms;
    void *d_sp64;        // SpeciesRec<double>[ns_pad]
    void *d_sp32;        // SpeciesRec<float>[ns_pad]
    double *d_pair64;    // [ns_pad][ns_pad] Chung pair weights
    float *d_pair32;
    double *d_kij64;     // [ns_pad][ns_pad] (1 - k_ij), zero padded
    float *d_kij32;
    int occ_props[3][2]; // resident blocks per SM: [precision][kij]
    int occ_newton[3][2];
    // per-species outputs (pr_species.cu): Kay's-rule and diffusion pair
    // constants, the optional high-pressure correction table
    double *d_dtab64;
    float *d_dtab32;
    double *d_corr64;
    float *d_corr32;
    int corr_nT, corr_nP;
    int occ_species[2];  // [FP64, FP32]
    // Bilger's mixture fraction: per-species coefficients b_k of the coupling
    // function, then beta_ox and 1 / (beta_fuel - beta_ox) ([n_species + 2])
    double *d_bilger64;
    float *d_bilger32;
    int has_bilger;
    // host images of the 9-species tables (HostTab9<double> / <float>), which
    // the property kernels take by value; NULL for the 32-species kernels
    void *h_tab64;
    void *h_tab32;
    double tmid_u;       // common NASA-7 switch temperature of every species, or 0
    // device address of the allocation-free entry point's scratch array on
    // this context's device (noalloc.cu), or NULL if the lookup failed
    void *noalloc_scratch;
};

namespace prgb {
// Build / release the per-species tables of a context (pr_species.cu).
pr_status species_tables_init(pr_ctx *c, const pr_species_table *tbl);
void species_tables_free(pr_ctx *c);
// Device address of the allocation-free scratch array on the current device (noalloc.cu).
pr_status noalloc_scratch_address(void **ptr);
}  // namespace prgb

// SG_MODE_FORWARD, SG_MODE_INVERSE or SG_MODE_BILGER of a surrogate (surrogate.cu).
int sg_mode_of(const sg_model *m);
