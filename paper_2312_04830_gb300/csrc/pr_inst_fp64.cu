// Instantiation of the property kernels for double arithmetic with a double cubic solve.
#include "pr_kernels.cuh"

namespace prk {
PRK_DECLARE(double, double, 9, )
PRK_DECLARE(double, double, 32, )
}  // namespace prk
