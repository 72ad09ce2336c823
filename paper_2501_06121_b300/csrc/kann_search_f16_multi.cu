// kann_search_f16_multi.cu -- the FP16 dense search kernels with the
// multi-expansion layer-0 step (kann_search_opts.expand > 1), compiled apart
// from the one-expansion kernels so that the library builds in parallel.
#include "kann_search_impl.cuh"

namespace kann {

SearchKernelFn pick_search_f16_multi(int cplt, int metric, int lpr_exact) {
  return pick_dense_multi_t<KANN_F16>(cplt, metric, lpr_exact);
}

}  // namespace kann
