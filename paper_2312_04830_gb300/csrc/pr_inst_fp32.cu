// Instantiation of the property kernels for float arithmetic with a float cubic solve.
#include "pr_kernels.cuh"

namespace prk {
PRK_DECLARE(float, float, 9, )
PRK_DECLARE(float, float, 32, )
}  // namespace prk
