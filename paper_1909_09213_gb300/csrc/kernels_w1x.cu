// Search kernels with the learned brancher and subtree logging for domains of 1 uint32
// word(s) (a translation unit of their own so that they compile in parallel).
#include "search.cuh"

namespace cubics {
CUBICS_DEFINE_WIDTH_EXT(1)
}  // namespace cubics
