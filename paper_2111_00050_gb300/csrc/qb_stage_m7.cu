// Stage-kernel specialisation for M = 7 modes (see qb_stage.cuh).
#include "qb_stage.cuh"

namespace qb {
int stage_launch_m7(const Tables& t, const DfArgs& a, int final_stage, int B, bool cplx, cudaStream_t st,
                   int* grid) {
  return stage_launch_t<7>(t, a, final_stage, B, cplx, st, grid);
}
}  // namespace qb
