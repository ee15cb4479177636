// tile_dispatch.cu -- selects the tile kernel instantiation for a series.
#include "../../include/rqa.h"
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

// Load every tile kernel instantiation now: with lazy module loading a
// kernel is otherwise loaded at its first launch, which can stall the whole
// context in the middle of other work.  Querying a function's attributes
// loads it.
int preload_tile_kernels() {
  int loaded = 0;
  cudaFuncAttributes a;
  for (int bands = 0; bands < 2; ++bands) {
    for (int cross = 0; cross < 2; ++cross)
      for (int f64 = 0; f64 < 2; ++f64)
        for (int norm = 0; norm < 3; ++norm)
          for (int m = 1; m <= RQA_MAX_M; ++m)
            for (int cols = 2; cols <= 4; cols += 2) {
              TileFn fn = tile_kernel_for(m, norm, cols, f64 != 0, cross != 0, bands != 0);
              if (!fn) continue;
              if (cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(fn)) != cudaSuccess)
                return -1;
              ++loaded;
            }
    if (TileFn fn = tile_kernel_matrix(4, bands != 0)) {
      if (cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(fn)) != cudaSuccess) return -1;
      ++loaded;
    }
  }
  return loaded;
}

size_t tile_smem_for(int m, int norm, bool f64, int warps, int cols) {
  const int row_elems = f64 ? m : ((2 * m + 3) / 4) * 4;  // each coordinate twice
  (void)norm;
  return tile_smem_bytes(warps, row_elems, f64 ? 8 : 4, cols);
}

}  // namespace rqa
