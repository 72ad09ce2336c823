// kann_search_e4m3_team.cu -- the E4M3 dense search kernels run by a team of
// warps per query (kann_search_opts.team = 2 or 4), compiled apart from the
// one-warp kernels so that the library builds in parallel.
#include "kann_search_impl.cuh"

namespace kann {

SearchKernelFn pick_search_e4m3_team(int cplt, int metric, int lpr_exact, int team) {
  return pick_dense_team_t<KANN_E4M3>(cplt, metric, lpr_exact, team);
}

}  // namespace kann
