// Host-side dispatch of the Tersoff force evaluation (kernels in force_kernels.cuh,
// one translation unit per precision) and the reduction of its energy/virial
// partial sums.
#include "internal.cuh"

namespace tsf {

// Sum n partial rows of (E, W[6]) in a fixed order into rs->epot / rs->virial:
// thread k adds rows k, k + 1024, ...; then a fixed tree over the threads.
__global__ void __launch_bounds__(1024) k_reduce_partials(const double *__restrict__ partial, int n, RunState *rs)
{
  __shared__ double sh[32][7];
  griddep_wait();
  if (rs->status != 0) return;
  double a[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int k = threadIdx.x; k < n; k += 1024)
    for (int c = 0; c < 7; ++c) a[c] += partial[(size_t)k * 8 + c];
  for (int c = 0; c < 7; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[c] += __shfl_xor_sync(0xffffffffu, a[c], o);
  }
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 7; ++c) sh[threadIdx.x >> 5][c] = a[c];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int c = 0; c < 7; ++c) {
      double v = sh[threadIdx.x][c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      a[c] = v;
    }
    if (threadIdx.x == 0) {
      rs->epot += a[0];
      for (int c = 0; c < 6; ++c) rs->virial[c] += a[1 + c];
    }
  }
}

#define TSF_FORCE_DECL(NAME)                                                                                        \
  cudaError_t NAME(int part, cudaStream_t st, int fast_slots, const FastTab &ft, int gen_slots, int eflag,       \
                   int vflag,                                                                                      \
                   int N, int ld, const dbl4 *x, const int4 *q, const int *nbr, const int *cnt,                   \
                   const SysTab *sys,                                                                              \
                   const void *pairs, const void *trips, int nt, void *contrib, void *selfF,                       \
                   unsigned long long *mask, int *work, int *nwork, double *partial, RunState *rs, double *eatom,  \
                   const ForceRoutes *routes, int stats, int *rows);
TSF_FORCE_DECL(launch_force_fp64)
TSF_FORCE_DECL(launch_force_mixed)
TSF_FORCE_DECL(launch_force_single)
#undef TSF_FORCE_DECL

int force_slots_for(int need)
{
  if (need <= 8) return 8;
  if (need <= 16) return 16;
  if (need <= 32) return 32;
  return 64;
}

// Rows of 8 doubles the partial-sum buffer needs for N atoms (any launch shape).
int force_partial_rows(int N) { return (N + 31) / 32 + 2 + GEN_BLOCKS; }

// Overflow-queue blocks for N atoms split into up to two register-kernel launches.
int force_queue_blocks(int N) { return (N + FAST_THREADS - 1) / FAST_THREADS + 2; }

// One force evaluation in precision prec (PREC_FP64, PREC_MIXED or PREC_SINGLE).
// fast_slots 4 or 8 runs the register kernel plus the warp kernel over its overflow
// queue; fast_slots 0 runs the general kernel (gen_slots wide) over all atoms.
// ld: the list stride (slot s of atom i at s * ld + i of nbr and contrib, ld >= N).
// routes (may be null: every atom in index order with fast_slots) splits the
// register kernel into launches over atom subsets, each with its own slot count.
// Buffers: partial force_partial_rows(N) x 8 doubles; work force_queue_blocks(N) x
// 128 ints; nwork force_queue_blocks(N) ints.  With eflag/vflag the energy and
// virial are added to rs->epot / rs->virial.  part: 1 launches the register
// kernel(s) only, 2 the rest (overflow or general kernel and the reduction), 3 both.
// stats: record the largest in-cutoff counts (rs->maxnc, rs->maxnc_t).
cudaError_t launch_force_part(int part, cudaStream_t st, int prec, int fast_slots, const FastTab &ft, int gen_slots,
                              int eflag, int vflag, int N, int ld, const dbl4 *x, const int4 *q, const int *nbr,
                              const int *cnt, const SysTab *sys, const void *pairs, const void *trips, int nt,
                              void *contrib, void *selfF, unsigned long long *mask, int *work, int *nwork,
                              double *partial, RunState *rs, double *eatom, const ForceRoutes *routes, int stats)
{
  auto f = prec == PREC_FP64 ? launch_force_fp64 : prec == PREC_MIXED ? launch_force_mixed : launch_force_single;
  int rows = 0;
  cudaError_t e = f(part, st, fast_slots, ft, gen_slots, eflag, vflag, N, ld, x, q, nbr, cnt, sys, pairs, trips, nt,
                    contrib, selfF, mask, work, nwork, partial, rs, eatom, routes, stats, &rows);
  if (e != cudaSuccess) return e;
  if ((eflag || vflag) && rows > 0 && (part & 2)) {
    e = launch_dep(k_reduce_partials, 1, 1024, 0, st, (const double *)partial, rows, rs);
  }
  return e;
}

cudaError_t launch_force(cudaStream_t st, int prec, int fast_slots, const FastTab &ft, int gen_slots, int eflag,
                         int vflag, int N, const dbl4 *x, const int4 *q, const int *nbr, const int *cnt,
                         const SysTab *sys, const void *pairs, const void *trips, int nt, void *contrib, void *selfF,
                         unsigned long long *mask, int *work, int *nwork, double *partial, RunState *rs,
                         double *eatom)
{
  return launch_force_part(3, st, prec, fast_slots, ft, gen_slots, eflag, vflag, N, N, x, q, nbr, cnt, sys, pairs,
                           trips, nt, contrib, selfF, mask, work, nwork, partial, rs, eatom, nullptr, 1);
}

}  // namespace tsf
