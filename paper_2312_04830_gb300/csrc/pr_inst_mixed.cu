// Instantiation of the property kernels for float arithmetic with a double cubic solve (compiled with
// the fast single-precision forms: see build.py UNIT_FLAGS).
#include "pr_kernels.cuh"

namespace prk {
PRK_DECLARE(float, double, 9, )
PRK_DECLARE(float, double, 32, )
}  // namespace prk
