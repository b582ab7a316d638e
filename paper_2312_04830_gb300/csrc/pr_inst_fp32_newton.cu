// Instantiation of the inversion kernels for float arithmetic with a float
// cubic solve, with IEEE single-precision division, square root and math
// functions: the fast forms cost the iteration more steps than they save.
#include "pr_kernels.cuh"

namespace prk {
PRK_DECLARE_NEWTON(float, float, 9, )
PRK_DECLARE_NEWTON(float, float, 32, )
}  // namespace prk
