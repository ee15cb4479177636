// tile_matrix.cu -- the fused tile kernel over a precomputed binary matrix
// (Sect. 9): the cross-recurrence line machinery with the recurrence words
// read from the caller's bits instead of computed from distances.
#include "rqa_kernels.h"
#include "rqa_tile.cuh"

namespace rqa {

TileFn tile_kernel_matrix(int cols, bool bands) {
  if (cols != 4) return nullptr;
  return bands ? (TileFn)tile_kernel<1, 0, 4, false, true, true, true>
               : (TileFn)tile_kernel<1, 0, 4, false, true, true>;
}

}  // namespace rqa
