// tile_dispatch.cu -- selects the tile kernel instantiation for a series.
#include "rqa_kernels.h"
#include "rqa_tile.cuh"

namespace rqa {

TileFn tile_kernel_for(int m, int norm, int cols, bool f64, bool cross, bool bands) {
  switch (norm) {
    case 0: return cross ? tile_kernel_cross_norm0(m, cols, f64, bands) : tile_kernel_norm0(m, cols, f64, bands);
    case 1: return cross ? tile_kernel_cross_norm1(m, cols, f64, bands) : tile_kernel_norm1(m, cols, f64, bands);
    case 2: return cross ? tile_kernel_cross_norm2(m, cols, f64, bands) : tile_kernel_norm2(m, cols, f64, bands);
    default: return nullptr;
  }
}

size_t tile_smem_for(int m, int norm, bool f64, int warps, int cols) {
  const int row_elems = f64 ? m : (norm == 1 ? ((2 * m + 3) / 4) * 4 : ((m + 3) / 4) * 4);
  return tile_smem_bytes(warps, row_elems, f64 ? 8 : 4, cols);
}

}  // namespace rqa
