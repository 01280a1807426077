// Search kernel for one-word int_ne problems of at most 32 variables, with each node's
// domains held in registers (a translation unit of its own so that it compiles in parallel).
#include "search.cuh"

namespace cubics {
CUBICS_DEFINE_REG
}  // namespace cubics
