// Stage-kernel specialisation for any M (see qb_stage.cuh).
#include "qb_stage.cuh"

namespace qb {
int stage_launch_any(const Tables& t, const DfArgs& a, int final_stage, int B, bool cplx, cudaStream_t st,
                   int* grid) {
  return stage_launch_t<0>(t, a, final_stage, B, cplx, st, grid);
}
}  // namespace qb
