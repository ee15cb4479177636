// tile_norm1.cu -- instantiations of the fused tile kernel for norm 1
// (0 = L-infinity, 1 = L2, 2 = L1), m = 1..10, FP32 + recheck and FP64, with and
// without row bands; four columns per lane, and two for FP32.
#include "rqa_kernels.h"
#include "rqa_tile.cuh"

namespace rqa {

template <int M>
static TileFn pick(int cols, bool f64, bool bands) {
  if (cols == 2) {  // two columns per lane: FP32 only (narrower strips, fewer registers)
    if (f64) return nullptr;
    return bands ? (TileFn)tile_kernel<M, 1, 2, false, false, false, true>
                 : (TileFn)tile_kernel<M, 1, 2, false, false>;
  }
  if (cols != 4) return nullptr;
  if (bands)
    return f64 ? (TileFn)tile_kernel<M, 1, 4, true, false, false, true>
               : (TileFn)tile_kernel<M, 1, 4, false, false, false, true>;
  return f64 ? (TileFn)tile_kernel<M, 1, 4, true, false>
             : (TileFn)tile_kernel<M, 1, 4, false, false>;
}

TileFn tile_kernel_norm1(int m, int cols, bool f64, bool bands) {
  switch (m) {
    case 1: return pick<1>(cols, f64, bands);
    case 2: return pick<2>(cols, f64, bands);
    case 3: return pick<3>(cols, f64, bands);
    case 4: return pick<4>(cols, f64, bands);
    case 5: return pick<5>(cols, f64, bands);
    case 6: return pick<6>(cols, f64, bands);
    case 7: return pick<7>(cols, f64, bands);
    case 8: return pick<8>(cols, f64, bands);
    case 9: return pick<9>(cols, f64, bands);
    case 10: return pick<10>(cols, f64, bands);
    default: return nullptr;
  }
}

TileFn tile_kernel_wait_test() {
  return (TileFn)tile_kernel<3, 1, 4, false, false, false, false, true>;
}

}  // namespace rqa
