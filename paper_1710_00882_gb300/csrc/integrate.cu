// Ingest, reverse force gather, float64 velocity Verlet and step bookkeeping.
//
// Force gather: the force kernel leaves, for each atom i, the sum of the force
// contributions of i's terms on each in-cutoff neighbour in slot s of i's list
// (contrib[s][i]), the force on i itself (selfF[i]) and the set of in-cutoff
// slots (mask[i]).  The force on atom m is selfF[m] plus, for each in-cutoff slot
// s of m's list, the contribution of its neighbour j's terms on m, stored at the
// slot of m in j's list: flat index rev[s][m] (written by the list build).
// In-cutoff is symmetric (the minimum-image r^2 is bitwise symmetric and
// r_C(i,j) = r_C(j,i)), so exactly the slots the force kernel wrote are read.
// The sum runs in list order: deterministic.
#include "internal.cuh"

namespace tsf {

// Knuth's TwoSum: s + e == a + b exactly (float32 round-to-nearest; explicit
// intrinsics so that no step is contracted or reassociated).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Exact float -> double widening on the integer pipe.  This GPU's FP64 pipe, which
// runs at 1/65 of the FP32 rate and bounds the integrator, also executes the F2F
// conversion; the bit construction below costs a few integer operations instead.  A
// normal float's exponent moves from 8 to 11 bits (bias 127 -> 1023: + 896 << 20 in the
// high word) and its 23-bit mantissa splits into the high word's top 20 bits and the
// low word's top 3.  Zero and subnormal floats give +-0 (a force contribution is
// either exactly 0 or far above 1e-38); Inf and NaN stay Inf and NaN.
__device__ __forceinline__ double widen(float f)
{
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7fffffffu;
  unsigned hi = a >= 0x7f800000u ? ((a >> 3) | 0x7ff00000u) : ((a >> 3) + 0x38000000u);
  unsigned lo = u << 29;
  if (a < 0x00800000u) hi = lo = 0u;
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)lo);
}

// Force accumulators of the gather, one per precision; V is the contribution type.

// mixed mode: float32 contributions summed with TwoSum, a head and tail float per
// component; the force is head + tail rounded once to float64.  Its error is that of
// a float64 sum of the same float32 terms, on the float32 pipe.
struct AccMixed {
  using V = float4;
  float h[3], l[3];
  __device__ __forceinline__ void init(const float4 &c)
  {
    h[0] = c.x; h[1] = c.y; h[2] = c.z;
    l[0] = l[1] = l[2] = 0.0f;
  }
  __device__ __forceinline__ void add(const float4 &c)
  {
    float e;
    two_sum(h[0], c.x, h[0], e); l[0] = __fadd_rn(l[0], e);
    two_sum(h[1], c.y, h[1], e); l[1] = __fadd_rn(l[1], e);
    two_sum(h[2], c.z, h[2], e); l[2] = __fadd_rn(l[2], e);
  }
  __device__ __forceinline__ void out(double &fx, double &fy, double &fz) const
  {
    fx = widen(h[0]) + widen(l[0]);
    fy = widen(h[1]) + widen(l[1]);
    fz = widen(h[2]) + widen(l[2]);
  }
};

// mixed mode, float64 sum: each float32 contribution widened and added in float64
// (the literal reading of float64 force accumulation; on this GPU each add runs on
// the FP64 pipe at 1/65 of the FP32 rate)
struct AccMixed64 {
  using V = float4;
  double f[3];
  __device__ __forceinline__ void init(const float4 &c) { f[0] = widen(c.x); f[1] = widen(c.y); f[2] = widen(c.z); }
  __device__ __forceinline__ void add(const float4 &c)
  {
    f[0] += widen(c.x);
    f[1] += widen(c.y);
    f[2] += widen(c.z);
  }
  __device__ __forceinline__ void out(double &fx, double &fy, double &fz) const { fx = f[0]; fy = f[1]; fz = f[2]; }
};

// single mode: a plain float32 sum (the paper's all-float32 accumulation)
struct AccSingle {
  using V = float4;
  float f[3];
  __device__ __forceinline__ void init(const float4 &c) { f[0] = c.x; f[1] = c.y; f[2] = c.z; }
  __device__ __forceinline__ void add(const float4 &c)
  {
    f[0] = __fadd_rn(f[0], c.x);
    f[1] = __fadd_rn(f[1], c.y);
    f[2] = __fadd_rn(f[2], c.z);
  }
  __device__ __forceinline__ void out(double &fx, double &fy, double &fz) const
  {
    fx = widen(f[0]); fy = widen(f[1]); fz = widen(f[2]);
  }
};

struct AccFP64 {
  using V = dbl4;
  double f[3];
  __device__ __forceinline__ void init(const dbl4 &c) { f[0] = c.x; f[1] = c.y; f[2] = c.z; }
  __device__ __forceinline__ void add(const dbl4 &c) { f[0] += c.x; f[1] += c.y; f[2] += c.z; }
  __device__ __forceinline__ void out(double &fx, double &fy, double &fz) const { fx = f[0]; fy = f[1]; fz = f[2]; }
};

template <class A>
__device__ __forceinline__ void gather_force(int m, int ld, const typename A::V *__restrict__ contrib,
                                             const typename A::V *__restrict__ selfF,
                                             const unsigned long long *__restrict__ mask, const int *__restrict__ rev,
                                             double &fx, double &fy, double &fz)
{
  using V = typename A::V;
  constexpr int U = 4;   // slots whose loads are issued together
  A acc;
  // The reverse indices of the first U list slots are loaded together with the mask
  // (every list holds at least U slots), so when all in-cutoff slots are among them
  // (diamond-like solids: the whole list is the four nearest neighbours) the gather
  // is two dependent loads deep instead of three.
  unsigned g0[U];
#pragma unroll
  for (int u = 0; u < U; ++u) g0[u] = (unsigned)rev[(size_t)u * ld + m];
  const V self = selfF[m];
  unsigned long long mb = mask[m];
  acc.init(self);
  if ((mb >> U) == 0ull) {
    V c[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if ((mb >> u) & 1ull) c[u] = contrib[g0[u]];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if ((mb >> u) & 1ull) acc.add(c[u]);
  } else {
    while (mb) {
      int sl[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        sl[u] = mb ? __ffsll((long long)mb) - 1 : -1;
        mb &= mb - 1;
      }
      unsigned g[U];
#pragma unroll
      for (int u = 0; u < U; ++u) g[u] = sl[u] >= 0 ? (unsigned)rev[(size_t)sl[u] * ld + m] : 0u;
      V c[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (sl[u] >= 0) c[u] = contrib[g[u]];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (sl[u] >= 0) acc.add(c[u]);
    }
  }
  acc.out(fx, fy, fz);
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// AoS float64 input -> dbl4 positions (type in w's bits) + fixed-point int4
// (type in w).  Positions are kept as given (not wrapped): every distance is a
// minimum image, and an MD state copied out and back in reproduces the same
// float64 values.  The fixed-point copy wraps by construction (mod 2^32).
__global__ void k_ingest(int N, const double *__restrict__ pos, const int *__restrict__ types, int nt, int sid,
                         const SysTab *__restrict__ sys, dbl4 *__restrict__ x, int4 *__restrict__ q, RunState *rs)
{
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const Geom &geo = sys[sid].geo;
  int t = types[i];
  if (t < 0 || t >= nt) {
    atomicOr(&rs->status, ST_BAD_TYPE);
    t = 0;
  }
  double p[3];
  int qq[3];
  for (int a = 0; a < 3; ++a) {
    double v = pos[3 * (size_t)i + a];
    if (!isfinite(v) || fabs(v * geo.invL[a]) > 1e5) {
      atomicOr(&rs->status, ST_NONFINITE);
      v = 0.0;
    }
    p[a] = v;
    qq[a] = fixed_q(v, geo.to_q[a]);
  }
  const int w = make_w(t, sid);
  x[i] = make_dbl4(p[0], p[1], p[2], __longlong_as_double((long long)w));
  q[i] = make_int4(qq[0], qq[1], qq[2], w);
}

// AoS float64 velocities -> dbl4
__global__ void k_ingest_vel(int N, const double *__restrict__ vel, dbl4 *__restrict__ v)
{
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  v[i] = make_dbl4(vel[3 * (size_t)i], vel[3 * (size_t)i + 1], vel[3 * (size_t)i + 2], 0.0);
}

// reverse gather into AoS float64 forces; flags non-finite values
// (perm non-null: atom i's row of out is perm[i], the caller's order of a permuted state)
template <class A>
__global__ void k_gather_out(int N, const typename A::V *__restrict__ contrib, const typename A::V *__restrict__ selfF,
                             const unsigned long long *__restrict__ mask, const int *__restrict__ rev,
                             double *__restrict__ out, const int *__restrict__ perm, RunState *rs)
{
  if (rs->status != 0) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double fx, fy, fz;
  gather_force<A>(i, N, contrib, selfF, mask, rev, fx, fy, fz);
  if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(&rs->status, ST_NONFINITE);
  const size_t o = perm ? (size_t)perm[i] : (size_t)i;
  out[3 * o] = fx;
  out[3 * o + 1] = fy;
  out[3 * o + 2] = fz;
}

enum { VV_FINISH = 1, VV_START = 2 };
constexpr int VV_THREADS = 128;   // integrator block size (more resident blocks per SM than 256)

// Velocity Verlet around the force evaluation, float64.
//   FINISH: v += dt/2 F/m          (second half kick of the previous step)
//   START:  v += dt/2 F/m; x += dt v; refresh fixed-point q; flag a rebuild when
//           some atom moved more than skin/2 since the last build
// KE: accumulate sum m v^2 of the full-step velocity (after FINISH, before START).
template <class A, bool KE>
__global__ void __launch_bounds__(VV_THREADS, sizeof(typename A::V) == 16 ? 12 : 1) k_vv(int N, int ld, int mode, dbl4 *__restrict__ x, dbl4 *__restrict__ v, int4 *__restrict__ q,
                     const int4 *__restrict__ qref, const typename A::V *__restrict__ contrib,
                     const typename A::V *__restrict__ selfF, const unsigned long long *__restrict__ mask,
                     const int *__restrict__ rev, const SysTab *__restrict__ sys, SysCtl *__restrict__ ctl,
                     const double *__restrict__ mass, float disp2_lim, double *__restrict__ kepart, RunState *rs)
{
  __shared__ double sw[8];
  if (rs->status != 0) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool active = i < N;
  double ke = 0.0;
  bool moved = false;
  if (active) {
    // the atom's word (type, system) from the w field of its float64 position (the
    // drift reads the rest of that line later); the fixed-point copy is only written
    const int w = (int)__double_as_longlong(reinterpret_cast<const double *>(x + i)[3]);
    const int t = type_of(w);
    const int sid = sys_of(w);
    const SysTab &T = sys[sid];
    const Geom &geo = T.geo;
    const double c = T.kick[t];
    const double dt = T.dt;
    int mode_i = mode;
    if (mode_i < 0) {
      // per-system step control: running, closing (last half kick pending) or done
      const SysCtl C = ctl[sid];
      mode_i = C.steps_left > 0 ? (C.open ? (VV_FINISH | VV_START) : VV_START) : (C.open ? VV_FINISH : 0);
    }
    // a system that neither kicks nor drifts in this step (finished, or a freed range
    // of a packed layout) needs no forces
    double fx = 0.0, fy = 0.0, fz = 0.0;
    if (mode_i != 0) gather_force<A>(i, ld, contrib, selfF, mask, rev, fx, fy, fz);
    dbl4 vi = (mode_i != 0 || KE) ? v[i] : make_dbl4(0.0, 0.0, 0.0, 0.0);
    if (mode_i & VV_FINISH) {
      vi.x = fma(c, fx, vi.x);
      vi.y = fma(c, fy, vi.y);
      vi.z = fma(c, fz, vi.z);
    }
    if (KE) ke = mass[t] * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z);
    if (mode_i & VV_START) {
      vi.x = fma(c, fx, vi.x);
      vi.y = fma(c, fy, vi.y);
      vi.z = fma(c, fz, vi.z);
      dbl4 xi = x[i];
      xi.x = fma(dt, vi.x, xi.x);
      xi.y = fma(dt, vi.y, xi.y);
      xi.z = fma(dt, vi.z, xi.z);
      x[i] = xi;
      const int4 qi = make_int4(fixed_q(xi.x, geo.to_q[0]), fixed_q(xi.y, geo.to_q[1]), fixed_q(xi.z, geo.to_q[2]), w);
      q[i] = qi;
      const int4 qr = qref[i];
      const float dx = (float)qdiff(qi.x, qr.x) * geo.q_to_f[0];
      const float dy = (float)qdiff(qi.y, qr.y) * geo.q_to_f[1];
      const float dz = (float)qdiff(qi.z, qr.z) * geo.q_to_f[2];
      moved = dx * dx + dy * dy + dz * dz > disp2_lim;
      if (moved && ctl[sid].rebuild == 0) atomicOr(&ctl[sid].rebuild, 1);
    }
    if (mode_i != 0) v[i] = vi;
  }
  if (__any_sync(0xffffffffu, moved) && (threadIdx.x & 31) == 0) atomicOr(&rs->rebuild, 1);
  if (KE) {
    // per-block partial in a fixed order; k_ke_reduce adds the blocks in order
    double s = warp_sum_d(ke);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sw[w];
      kepart[blockIdx.x] = a;
    }
  }
}

__global__ void k_ke_reduce(const double *__restrict__ kepart, int n, RunState *rs)
{
  __shared__ double sh[256];
  if (rs->status != 0) return;
  double a = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) a += kepart[k];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) rs->ekin2 += sh[0];
}

// AoS copies out of the device state (perm non-null: atom i goes to row perm[i])
__global__ void k_extract(int N, const dbl4 *__restrict__ x, const dbl4 *__restrict__ v, double *__restrict__ pos,
                          double *__restrict__ vel, const int *__restrict__ perm)
{
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const size_t o = perm ? (size_t)perm[i] : (size_t)i;
  if (pos) {
    dbl4 a = x[i];
    pos[3 * o] = a.x;
    pos[3 * o + 1] = a.y;
    pos[3 * o + 2] = a.z;
  }
  if (vel) {
    dbl4 b = v[i];
    vel[3 * o] = b.x;
    vel[3 * o + 1] = b.y;
    vel[3 * o + 2] = b.z;
  }
}

// Atom k of the permuted state is atom perm[k] of the source (all three records).
__global__ void k_permute_atoms(int N, const int *__restrict__ perm, const dbl4 *__restrict__ sx,
                                const dbl4 *__restrict__ sv, const int4 *__restrict__ sq, dbl4 *__restrict__ dx,
                                dbl4 *__restrict__ dv, int4 *__restrict__ dq)
{
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int i = perm[k];
  dx[k] = sx[i];
  dv[k] = sv[i];
  dq[k] = sq[i];
}

// End of an MD step: record (PE_k, KE_{k-1}) in the trace (row k = rs->trace_k),
// roll the accumulators, count the step; inside a graph, decide whether the step
// loop goes on.  One block: thread 0 rolls the run state, all threads update the
// per-system step control.
__global__ void k_step_end(RunState *rs, SysCtl *ctl, int nsys, cudaGraphConditionalHandle loop, int use_cond)
{
  griddep_wait();
  if (rs->status != 0) {
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(loop, 0);
    return;
  }
  // per system: a running system counts its step; a closing one is now done
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
    SysCtl &C = ctl[s];
    if (C.steps_left > 0) {
      C.steps_left -= 1;
      C.open = 1;
    } else if (C.open) {
      C.open = 0;
    }
    C.rebuild = 0;
  }
  if (threadIdx.x != 0) return;
  const long long k = rs->trace_k;
  double *trace = rs->trace;
  if (trace) {
    if (k == 1) trace[0] = rs->epot_last;
    trace[2 * k] = rs->epot;
    trace[2 * k - 1] = 0.5 * rs->ekin2 / ACCEL;
  }
  rs->epot_last = rs->epot;
  rs->epot = 0.0;
  rs->ekin2 = 0.0;
  for (int c = 0; c < 6; ++c) rs->virial[c] = 0.0;
  rs->step += 1;
  rs->over_total = 0;
  rs->trace_k = k + 1;
  rs->steps_left -= 1;
  if (use_cond) cudaGraphSetConditional(loop, rs->steps_left > 0 ? 1u : 0u);
}

// First node of a step-loop graph: the launch's controls (as k_set_control, system
// 0 when ctl is non-null) and the loop's first condition.  The host sets its
// parameters before each launch.
__global__ void k_loop_start(RunState *rs, SysCtl *ctl, long long steps, double *trace, long long trace_k, int open,
                             cudaGraphConditionalHandle loop)
{
  if (rs->status != 0) {
    rs->steps_left += steps;
    if (ctl) ctl[0].steps_left += steps;
    cudaGraphSetConditional(loop, 0u);
    return;
  }
  rs->steps_left = steps;
  if (ctl) {
    ctl[0].steps_left = steps;
    ctl[0].open = open;
  }
  rs->trace = trace;
  rs->trace_k = trace_k;
  cudaGraphSetConditional(loop, steps > 0 ? 1u : 0u);
}

// after the integrator of a step: rebuild the list in this step?
__global__ void k_decide(RunState *rs, cudaGraphConditionalHandle build)
{
  griddep_wait();
  cudaGraphSetConditional(build, (rs->status == 0 && rs->rebuild != 0) ? 1u : 0u);
}

// Host-chosen controls of the next launch of a single system (system 0).  After a
// failure the launched steps do not run; their count is added to the steps left
// so that recovery resumes them all.
__global__ void k_set_control(RunState *rs, SysCtl *ctl, long long steps, double *trace, long long trace_k, int open)
{
  if (rs->status != 0) {
    rs->steps_left += steps;
    ctl[0].steps_left += steps;
    return;
  }
  rs->steps_left = steps;
  ctl[0].steps_left = steps;
  ctl[0].open = open;
  rs->trace = trace;
  rs->trace_k = trace_k;
}

// after the closing half kick of a single system: KE of the last step (row trace_k - 1)
__global__ void k_final(RunState *rs, SysCtl *ctl)
{
  if (rs->status != 0) return;
  if (rs->trace) rs->trace[2 * (rs->trace_k - 1) + 1] = 0.5 * rs->ekin2 / ACCEL;
  rs->ekin2 = 0.0;
  ctl[0].open = 0;
}

// after a standalone force evaluation: keep its energy as the current PE
__global__ void k_force_done(RunState *rs)
{
  if (rs->status != 0) return;
  rs->epot_last = rs->epot;
  rs->epot = 0.0;
  rs->over_total = 0;
  for (int c = 0; c < 6; ++c) rs->virial[c] = 0.0;
}

template <class A>
static void launch_vv_a(cudaStream_t st, bool ke, int B, int N, int ld, int mode, dbl4 *x, dbl4 *v, int4 *q, const int4 *qref,
                        const void *contrib, const void *selfF, const unsigned long long *mask, const int *rev,
                        const SysTab *sys, SysCtl *ctl, const double *mass, float disp2_lim, double *kepart,
                        RunState *rs)
{
  using V = const typename A::V *;
  if (ke)
    k_vv<A, true><<<B, VV_THREADS, 0, st>>>(N, ld, mode, x, v, q, qref, (V)contrib, (V)selfF, mask, rev, sys, ctl, mass,
                                            disp2_lim, kepart, rs);
  else
    k_vv<A, false><<<B, VV_THREADS, 0, st>>>(N, ld, mode, x, v, q, qref, (V)contrib, (V)selfF, mask, rev, sys, ctl, mass,
                                             disp2_lim, kepart, rs);
}

cudaError_t launch_vv(cudaStream_t st, int prec, bool ke, int N, int ld, int mode, dbl4 *x, dbl4 *v, int4 *q,
                      const int4 *qref, const void *contrib, const void *selfF, const unsigned long long *mask,
                      const int *rev, const SysTab *sys, SysCtl *ctl, const double *mass, float disp2_lim,
                      double *kepart, RunState *rs)
{
  if (N == 0) return cudaSuccess;
  const int B = (N + VV_THREADS - 1) / VV_THREADS;
  auto f = prec == PREC_FP64          ? launch_vv_a<AccFP64>
           : prec == PREC_MIXED        ? launch_vv_a<AccMixed>
           : prec == PREC_MIXED_ACC64  ? launch_vv_a<AccMixed64>
                                       : launch_vv_a<AccSingle>;
  f(st, ke, B, N, ld, mode, x, v, q, qref, contrib, selfF, mask, rev, sys, ctl, mass, disp2_lim, kepart, rs);
  if (ke) k_ke_reduce<<<1, 256, 0, st>>>(kepart, B, rs);
  return cudaGetLastError();
}

int vv_blocks(int N) { return (N + VV_THREADS - 1) / VV_THREADS; }

cudaError_t launch_gather_out(cudaStream_t st, int prec, int N, const void *contrib, const void *selfF,
                              const unsigned long long *mask, const int *rev, double *out, RunState *rs,
                              const int *perm)
{
  if (N == 0) return cudaSuccess;
  const int T = 256, B = (N + T - 1) / T;
  if (prec == PREC_FP64)
    k_gather_out<AccFP64><<<B, T, 0, st>>>(N, (const dbl4 *)contrib, (const dbl4 *)selfF, mask, rev, out, perm, rs);
  else if (prec == PREC_MIXED)
    k_gather_out<AccMixed><<<B, T, 0, st>>>(N, (const float4 *)contrib, (const float4 *)selfF, mask, rev, out, perm,
                                            rs);
  else if (prec == PREC_MIXED_ACC64)
    k_gather_out<AccMixed64><<<B, T, 0, st>>>(N, (const float4 *)contrib, (const float4 *)selfF, mask, rev, out,
                                              perm, rs);
  else
    k_gather_out<AccSingle><<<B, T, 0, st>>>(N, (const float4 *)contrib, (const float4 *)selfF, mask, rev, out, perm,
                                             rs);
  return cudaGetLastError();
}

}  // namespace tsf

namespace tsf {

cudaError_t launch_ingest(cudaStream_t st, int N, const double *pos, const int *types, int nt, int sid,
                          const SysTab *sys, dbl4 *x, int4 *q, RunState *rs)
{
  if (N == 0) return cudaSuccess;
  k_ingest<<<(N + 255) / 256, 256, 0, st>>>(N, pos, types, nt, sid, sys, x, q, rs);
  return cudaGetLastError();
}

cudaError_t launch_ingest_vel(cudaStream_t st, int N, const double *vel, dbl4 *v)
{
  if (N == 0) return cudaSuccess;
  k_ingest_vel<<<(N + 255) / 256, 256, 0, st>>>(N, vel, v);
  return cudaGetLastError();
}

cudaError_t launch_extract(cudaStream_t st, int N, const dbl4 *x, const dbl4 *v, double *pos, double *vel,
                           const int *perm)
{
  if (N == 0) return cudaSuccess;
  k_extract<<<(N + 255) / 256, 256, 0, st>>>(N, x, v, pos, vel, perm);
  return cudaGetLastError();
}

cudaError_t launch_permute_atoms(cudaStream_t st, int N, const int *perm, const dbl4 *sx, const dbl4 *sv,
                                 const int4 *sq, dbl4 *dx, dbl4 *dv, int4 *dq)
{
  if (N == 0) return cudaSuccess;
  k_permute_atoms<<<(N + 255) / 256, 256, 0, st>>>(N, perm, sx, sv, sq, dx, dv, dq);
  return cudaGetLastError();
}

cudaError_t launch_step_end(cudaStream_t st, RunState *rs, SysCtl *ctl, int nsys, cudaGraphConditionalHandle loop,
                            int use_cond)
{
  return launch_dep(k_step_end, 1, nsys > 1 ? 256 : 32, 0, st, rs, ctl, nsys, loop, use_cond);
}

cudaError_t launch_loop_start(cudaStream_t st, RunState *rs, SysCtl *ctl, long long steps, double *trace,
                              long long trace_k, int open, cudaGraphConditionalHandle loop)
{
  k_loop_start<<<1, 1, 0, st>>>(rs, ctl, steps, trace, trace_k, open, loop);
  return cudaGetLastError();
}

// New parameters of a captured k_loop_start node in an instantiated graph.
cudaError_t set_loop_start(cudaGraphExec_t exec, cudaGraphNode_t node, RunState *rs, SysCtl *ctl, long long steps,
                           double *trace, long long trace_k, int open, cudaGraphConditionalHandle loop)
{
  void *args[] = {&rs, &ctl, &steps, &trace, &trace_k, &open, &loop};
  cudaKernelNodeParams p = {};
  p.func = (void *)k_loop_start;
  p.gridDim = dim3(1, 1, 1);
  p.blockDim = dim3(1, 1, 1);
  p.sharedMemBytes = 0;
  p.kernelParams = args;
  p.extra = nullptr;
  return cudaGraphExecKernelNodeSetParams(exec, node, &p);
}

cudaError_t launch_decide(cudaStream_t st, RunState *rs, cudaGraphConditionalHandle build)
{
  return launch_dep(k_decide, 1, 1, 0, st, rs, build);
}

// New parameters of a captured k_set_control node in an instantiated graph.
cudaError_t set_control_node(cudaGraphExec_t exec, cudaGraphNode_t node, RunState *rs, SysCtl *ctl, long long steps,
                             double *trace, long long trace_k, int open)
{
  void *args[] = {&rs, &ctl, &steps, &trace, &trace_k, &open};
  cudaKernelNodeParams p = {};
  p.func = (void *)k_set_control;
  p.gridDim = dim3(1, 1, 1);
  p.blockDim = dim3(1, 1, 1);
  p.sharedMemBytes = 0;
  p.kernelParams = args;
  p.extra = nullptr;
  return cudaGraphExecKernelNodeSetParams(exec, node, &p);
}

cudaError_t launch_set_control(cudaStream_t st, RunState *rs, SysCtl *ctl, long long steps, double *trace,
                               long long trace_k, int open)
{
  k_set_control<<<1, 1, 0, st>>>(rs, ctl, steps, trace, trace_k, open);
  return cudaGetLastError();
}

cudaError_t launch_final(cudaStream_t st, RunState *rs, SysCtl *ctl)
{
  k_final<<<1, 1, 0, st>>>(rs, ctl);
  return cudaGetLastError();
}

cudaError_t launch_force_done(cudaStream_t st, RunState *rs)
{
  k_force_done<<<1, 1, 0, st>>>(rs);
  return cudaGetLastError();
}

}  // namespace tsf
