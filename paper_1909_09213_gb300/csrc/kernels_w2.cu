// Search and propagate kernels for domains of 2 uint32 word(s) (one translation unit per
// width so the widths compile in parallel).
#include "search.cuh"

namespace cubics {
CUBICS_DEFINE_WIDTH(2)
}  // namespace cubics
