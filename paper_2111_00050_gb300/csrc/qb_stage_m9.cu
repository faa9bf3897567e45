// Stage-kernel specialisation for M = 9 modes (see qb_stage.cuh).
#include "qb_stage.cuh"

namespace qb {
int stage_launch_m9(const Tables& t, const DfArgs& a, int final_stage, int B, bool cplx, cudaStream_t st,
                   int* grid) {
  return stage_launch_t<9>(t, a, final_stage, B, cplx, st, grid);
}
}  // namespace qb
