// Search and propagate kernels for domains of 1 uint32 word(s) (one translation unit per
// width so the widths compile in parallel).
#include "search.cuh"

namespace cubics {
CUBICS_DEFINE_WIDTH(1)
}  // namespace cubics
