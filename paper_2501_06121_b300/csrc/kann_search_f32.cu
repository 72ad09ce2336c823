// kann_search_f32.cu -- the FP32 dense search kernels (general and exact-tiling
// forms, L2 and inner product).  Each storage format's kernels are compiled in
// a translation unit of their own so that the library builds in parallel.
#include "kann_search_impl.cuh"

namespace kann {

SearchKernelFn pick_search_f32(int cplt, bool lean, int metric, int lpr_exact) {
  return pick_dense_t<KANN_F32>(cplt, lean, metric, lpr_exact);
}

}  // namespace kann
