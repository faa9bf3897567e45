// Stage-kernel specialisation for M = 11 modes (see qb_stage.cuh).
#include "qb_stage.cuh"

namespace qb {
int stage_launch_m11(const Tables& t, const DfArgs& a, int mode, int B, bool cplx, bool bil, int shape, cudaStream_t st,
                   int* grid) {
  return stage_launch_t<11>(t, a, mode, B, cplx, bil, shape, st, grid);
}
int resident_launch_m11(const Tables& t, const ResArgs& r, bool cplx, cudaStream_t st) {
  return resident_launch_t<11>(t, r, cplx, st);
}
}  // namespace qb
