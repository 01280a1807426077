// Search kernels with the learned brancher and subtree logging for domains of 2 uint32
// word(s) (a translation unit of their own so that they compile in parallel).
#include "search.cuh"

namespace cubics {
CUBICS_DEFINE_WIDTH_EXT(2)
}  // namespace cubics
