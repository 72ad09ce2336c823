// kann_search_bf16_team.cu -- the BF16 dense search kernels run by a team of
// warps per query (kann_search_opts.team = 2 or 4), compiled apart from the
// one-warp kernels so that the library builds in parallel.
#include "kann_search_impl.cuh"

namespace kann {

SearchKernelFn pick_search_bf16_team(int cplt, int metric, int lpr_exact, int team) {
  return pick_dense_team_t<KANN_BF16>(cplt, metric, lpr_exact, team);
}

}  // namespace kann
