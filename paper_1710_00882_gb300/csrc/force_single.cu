// Tersoff force kernels instantiated for single mode (float32 throughout, Sec. 4).
#include "force_kernels.cuh"

namespace tsf {

cudaError_t launch_force_single(int part, cudaStream_t st, int fast_slots, const FastTab &ft, int gen_slots, int eflag,
                                int vflag, int N, int ld, const dbl4 *x, const int4 *q, const int *nbr, const int *cnt,
                                const SysTab *sys, const void *pairs, const void *trips, int nt, void *contrib,
                                void *selfF, unsigned long long *mask, int *work, int *nwork, double *partial,
                                RunState *rs, double *eatom, const ForceRoutes *routes, int stats, int *rows)
{
  return launch_force_m<MathS>(part, st, fast_slots, ft, gen_slots, eflag, vflag, N, ld, x, q, nbr, cnt, sys, pairs,
                               trips, nt, contrib, selfF, mask, work, nwork, partial, rs, eatom, routes, stats, rows);
}

}  // namespace tsf
