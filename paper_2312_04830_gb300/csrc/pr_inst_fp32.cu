// Instantiation of the property kernels for float arithmetic with a float
// cubic solve, compiled with the fast single-precision forms (build.py
// UNIT_FLAGS); the FP32 inversion is instantiated in pr_inst_fp32_newton.cu.
#include "pr_kernels.cuh"

namespace prk {
PRK_DECLARE_PROPS(float, float, 9, )
PRK_DECLARE_PROPS(float, float, 32, )
}  // namespace prk
