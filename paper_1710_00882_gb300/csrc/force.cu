// Tersoff energy/force kernel: Algorithm 1 of the paper, one thread per atom i.
//
// Per atom the thread
//   1. walks i's Verlet list and packs the in-cutoff neighbours (Sec. 3: skin
//      atoms are tested once and never enter the K loops) into per-thread
//      shared-memory slots: unit vector, r, 1/r, f_C(r), f_C'(r), type;
//   2. first K loop (pass A): zeta_ij for every packed j (Eq. 3), then the pair
//      term V(i,j,zeta_ij) (Eqs. 1-2), its r-derivative and dV/dzeta;
//   3. second K loop (pass B): dzeta(i,j,k)/dx_j and /dx_k scaled by dV/dzeta
//      (the restructuring of Sec. 2: zeta is complete before any derivative is
//      scaled, so each derivative is formed once).
// All force contributions that i's terms make to neighbour j are summed per j in
// the thread and written once, to slot s of i's list (contrib[s][i]); the
// force on i itself follows from translation invariance (minus their sum).  No
// atomics: a reverse gather (gather.cu / integrate.cu) adds, for each atom m,
// the contributions written in m's slot of each neighbour's list, in list order,
// so the result is bitwise reproducible.  This replaces the serialised
// conflicting updates of the paper's "I" vectorisation (Sec. 3).
//
// Precision: R = double (FP64 mode) or float (mixed mode).  In mixed mode the
// relative vector d_ij is the exact int32 difference of 32-bit fixed-point
// coordinates, converted once to float.
#include "internal.cuh"

namespace tsf {

template <class R> struct V4t;
template <> struct V4t<float> { using type = float4; };
template <> struct V4t<double> { using type = dbl4; };

__device__ __forceinline__ float t_exp(float x) { return expf(x); }
__device__ __forceinline__ double t_exp(double x) { return exp(x); }
__device__ __forceinline__ float t_exp2(float x) { return exp2f(x); }
__device__ __forceinline__ double t_exp2(double x) { return exp2(x); }
__device__ __forceinline__ float t_log2(float x) { return log2f(x); }
__device__ __forceinline__ double t_log2(double x) { return log2(x); }
__device__ __forceinline__ float t_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double t_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float t_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double t_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ void t_sincospi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void t_sincospi(double x, double *s, double *c) { sincospi(x, s, c); }

// f_C and f_C' for r < R + D
template <class R>
__device__ __forceinline__ void cutoff_fn(R r, const PairP<R> &P, R &fc, R &dfc)
{
  if (r <= P.r_in) {
    fc = R(1);
    dfc = R(0);
  } else {
    R s, c;
    t_sincospi((r - P.Rc) * P.inv2D, &s, &c);
    fc = R(0.5) - R(0.5) * s;
    dfc = P.dfc_scale * c;
  }
}

constexpr int NRF = 11;   // real fields per slot
enum { S_UX = 0, S_UY, S_UZ, S_R, S_IR, S_FC, S_DFC, S_DZ, S_FX, S_FY, S_FZ };

template <class R, int MAXNC>
struct ForceCfg {
  static constexpr int slot_bytes = NRF * (int)sizeof(R) + 4;
  static constexpr int raw = 98304 / (MAXNC * slot_bytes);
  static constexpr int threads = raw >= 128 ? 128 : raw >= 64 ? 64 : 32;
  static constexpr size_t smem_slots = (size_t)threads * MAXNC * slot_bytes;
};

template <class R> __device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class R, int MAXNC, bool EFLAG, bool VFLAG>
__global__ void __launch_bounds__(ForceCfg<R, MAXNC>::threads)
k_force(int N, const dbl4 *__restrict__ x, const int4 *__restrict__ q, const int *__restrict__ nbr,
        const int *__restrict__ cnt, Geom geo, const PairP<R> *__restrict__ gpairs,
        const TripP<R> *__restrict__ gtrips, int nt, typename V4t<R>::type *__restrict__ contrib,
        typename V4t<R>::type *__restrict__ selfF, unsigned long long *__restrict__ mask, RunState *rs)
{
  using V4 = typename V4t<R>::type;
  constexpr int T = ForceCfg<R, MAXNC>::threads;
  constexpr bool MIXED = sizeof(R) == 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PairP<R> *pairs = reinterpret_cast<PairP<R> *>(smem_raw);
  TripP<R> *trips = reinterpret_cast<TripP<R> *>(smem_raw + sizeof(PairP<R>) * MAX_TYPES * MAX_TYPES);
  R *sr = reinterpret_cast<R *>(smem_raw + sizeof(PairP<R>) * MAX_TYPES * MAX_TYPES +
                                sizeof(TripP<R>) * MAX_TYPES * MAX_TYPES * MAX_TYPES);
  int *smeta = reinterpret_cast<int *>(sr + (size_t)NRF * MAXNC * T);

  if (rs->status != 0) return;   // uniform across the grid
  for (int k = threadIdx.x; k < nt * nt; k += T) pairs[k] = gpairs[k];
  for (int k = threadIdx.x; k < nt * nt * nt; k += T) trips[k] = gtrips[k];
  __syncthreads();

  const int t = threadIdx.x;
  const int i = blockIdx.x * T + t;
  const bool active = i < N;
#define SLOT(f, s) sr[((f) * MAXNC + (s)) * T + t]
#define META(s) smeta[(s) * T + t]

  int ti = 0, nc = 0;
  unsigned long long mbits = 0ull;
  bool overflow = false;
  int4 qi = make_int4(0, 0, 0, 0);
  dbl4 xi = make_dbl4(0, 0, 0, 0);
  if (active) {
    if (MIXED) {
      qi = q[i];
      ti = qi.w;
    } else {
      xi = x[i];
      ti = (int)__double_as_longlong(xi.w);
    }
    const int n = cnt[i];
    for (int s = 0; s < n; ++s) {
      const int j = nbr[(size_t)s * N + i];
      R dx, dy, dz;
      int tj;
      if (MIXED) {
        int4 qj = q[j];
        tj = qj.w;
        dx = (R)(float)qdiff(qj.x, qi.x) * (R)geo.q_to_f[0];
        dy = (R)(float)qdiff(qj.y, qi.y) * (R)geo.q_to_f[1];
        dz = (R)(float)qdiff(qj.z, qi.z) * (R)geo.q_to_f[2];
      } else {
        dbl4 xj = x[j];
        tj = (int)__double_as_longlong(xj.w);
        double ddx = xj.x - xi.x, ddy = xj.y - xi.y, ddz = xj.z - xi.z;
        ddx -= geo.L[0] * rint(ddx * geo.invL[0]);
        ddy -= geo.L[1] * rint(ddy * geo.invL[1]);
        ddz -= geo.L[2] * rint(ddz * geo.invL[2]);
        dx = (R)ddx; dy = (R)ddy; dz = (R)ddz;
      }
      const R r2 = dx * dx + dy * dy + dz * dz;
      const PairP<R> &P = pairs[ti * nt + tj];
      if (r2 < P.rc2) {
        if (nc < MAXNC) {
          const R ir = t_rsqrt(r2);
          const R r = r2 * ir;
          R fc, dfc;
          cutoff_fn(r, P, fc, dfc);
          SLOT(S_UX, nc) = dx * ir;
          SLOT(S_UY, nc) = dy * ir;
          SLOT(S_UZ, nc) = dz * ir;
          SLOT(S_R, nc) = r;
          SLOT(S_IR, nc) = ir;
          SLOT(S_FC, nc) = fc;
          SLOT(S_DFC, nc) = dfc;
          META(nc) = s | (tj << 8);
        } else {
          overflow = true;
        }
        ++nc;
        mbits |= 1ull << s;
      }
    }
    if (overflow) {
      atomicOr(&rs->status, ST_NC_OVERFLOW);
      atomicMax(&rs->maxnc, nc);
      nc = 0;
    }
  }

  // ---- pass A: zeta_ij, pair term, dV/dzeta --------------------------------
  R e_i = R(0);
  for (int a = 0; a < nc; ++a) {
    const int tj = META(a) >> 8;
    const R uax = SLOT(S_UX, a), uay = SLOT(S_UY, a), uaz = SLOT(S_UZ, a), ra = SLOT(S_R, a);
    const TripP<R> *Tj = trips + (ti * nt + tj) * nt;
    R zeta = R(0);
    for (int b = 0; b < nc; ++b) {
      if (b == a) continue;
      const TripP<R> &Tp = Tj[META(b) >> 8];
      const R cost = uax * SLOT(S_UX, b) + uay * SLOT(S_UY, b) + uaz * SLOT(S_UZ, b);
      const R u = Tp.h - cost;
      const R u2 = u * u;
      const R g = Tp.gamma + Tp.K * u2 * t_rcp(Tp.d2 + u2);
      R ex = R(1);
      if (Tp.lam3 != R(0)) {
        R arg = Tp.lam3 * (ra - SLOT(S_R, b));
        if (Tp.m3 != R(0)) arg = arg * arg * arg;
        ex = t_exp(arg);
      }
      zeta += SLOT(S_FC, b) * g * ex;
    }
    const PairP<R> &P = pairs[ti * nt + tj];
    const R fc = SLOT(S_FC, a), dfc = SLOT(S_DFC, a);
    const R fR = P.A * t_exp(-P.lam1 * ra);
    const R fA = -P.B * t_exp(-P.lam2 * ra);
    R bij = R(1), dbij = R(0);
    if (zeta > R(0)) {
      const R xb = t_exp2(P.n * t_log2(P.beta * zeta));
      bij = t_exp2(P.neg_inv2n * t_log2(R(1) + xb));
      dbij = R(-0.5) * bij * xb * t_rcp((R(1) + xb) * zeta);
    }
    const R pr = fR + bij * fA;
    e_i += R(0.5) * fc * pr;
    const R dvdr = R(0.5) * (dfc * pr + fc * (-P.lam1 * fR - bij * P.lam2 * fA));
    SLOT(S_DZ, a) = R(0.5) * fc * fA * dbij;
    SLOT(S_FX, a) = -dvdr * uax;
    SLOT(S_FY, a) = -dvdr * uay;
    SLOT(S_FZ, a) = -dvdr * uaz;
  }

  // ---- pass B: zeta derivatives scaled by dV/dzeta ------------------------
  for (int a = 0; a < nc; ++a) {
    const R dzv = SLOT(S_DZ, a);
    if (dzv == R(0)) continue;
    const int tj = META(a) >> 8;
    const R uax = SLOT(S_UX, a), uay = SLOT(S_UY, a), uaz = SLOT(S_UZ, a), ra = SLOT(S_R, a), ira = SLOT(S_IR, a);
    const TripP<R> *Tj = trips + (ti * nt + tj) * nt;
    R fjx = R(0), fjy = R(0), fjz = R(0);
    for (int b = 0; b < nc; ++b) {
      if (b == a) continue;
      const TripP<R> &Tp = Tj[META(b) >> 8];
      const R ubx = SLOT(S_UX, b), uby = SLOT(S_UY, b), ubz = SLOT(S_UZ, b), irb = SLOT(S_IR, b);
      const R cost = uax * ubx + uay * uby + uaz * ubz;
      const R u = Tp.h - cost;
      const R u2 = u * u;
      const R inv = t_rcp(Tp.d2 + u2);
      const R g = Tp.gamma + Tp.K * u2 * inv;
      const R dg = -Tp.G2 * u * inv * inv;
      R ex = R(1), darg = R(0);
      if (Tp.lam3 != R(0)) {
        R tt = Tp.lam3 * (ra - SLOT(S_R, b));
        R arg = tt;
        darg = Tp.lam3;
        if (Tp.m3 != R(0)) {
          arg = tt * tt * tt;
          darg = R(3) * Tp.lam3 * tt * tt;
        }
        ex = t_exp(arg);
      }
      const R fcb = SLOT(S_FC, b), dfcb = SLOT(S_DFC, b);
      const R a1 = fcb * ex * dg;          // coefficient of dcos/dx
      const R a2 = fcb * ex * g * darg;    // coefficient of dr_ij/dx_j and -dr_ik/dx_k
      const R a3 = dfcb * g * ex;          // coefficient of dr_ik/dx_k from f_C(r_ik)
      // dzeta/dx_j = a1 (u_b - cos u_a)/r_a + a2 u_a
      const R cj = a1 * ira;
      const R dzjx = cj * (ubx - cost * uax) + a2 * uax;
      const R dzjy = cj * (uby - cost * uay) + a2 * uay;
      const R dzjz = cj * (ubz - cost * uaz) + a2 * uaz;
      // dzeta/dx_k = a3 u_b + a1 (u_a - cos u_b)/r_b - a2 u_b
      const R ck = a1 * irb;
      const R dzkx = (a3 - a2) * ubx + ck * (uax - cost * ubx);
      const R dzky = (a3 - a2) * uby + ck * (uay - cost * uby);
      const R dzkz = (a3 - a2) * ubz + ck * (uaz - cost * ubz);
      fjx -= dzv * dzjx;
      fjy -= dzv * dzjy;
      fjz -= dzv * dzjz;
      SLOT(S_FX, b) -= dzv * dzkx;
      SLOT(S_FY, b) -= dzv * dzky;
      SLOT(S_FZ, b) -= dzv * dzkz;
    }
    SLOT(S_FX, a) += fjx;
    SLOT(S_FY, a) += fjy;
    SLOT(S_FZ, a) += fjz;
  }

  // ---- outputs --------------------------------------------------------------
  R fix = R(0), fiy = R(0), fiz = R(0);
  R w0 = R(0), w1 = R(0), w2 = R(0), w3 = R(0), w4 = R(0), w5 = R(0);
  for (int a = 0; a < nc; ++a) {
    const R fx = SLOT(S_FX, a), fy = SLOT(S_FY, a), fz = SLOT(S_FZ, a);
    fix -= fx;
    fiy -= fy;
    fiz -= fz;
    V4 c;
    c.x = fx; c.y = fy; c.z = fz; c.w = R(0);
    contrib[(size_t)(META(a) & 0xff) * N + i] = c;
    if (VFLAG) {
      const R r = SLOT(S_R, a);
      const R dx = r * SLOT(S_UX, a), dy = r * SLOT(S_UY, a), dz = r * SLOT(S_UZ, a);
      w0 += dx * fx; w1 += dy * fy; w2 += dz * fz;
      w3 += dx * fy; w4 += dx * fz; w5 += dy * fz;
    }
  }
  if (active) {
    V4 c;
    c.x = fix; c.y = fiy; c.z = fiz; c.w = R(0);
    selfF[i] = c;
    mask[i] = mbits;
  }
  if (EFLAG) {
    // float32 sums over the 32 atoms of a warp, then float64 across warps
    R e = warp_sum(e_i);
    if ((t & 31) == 0) atomicAdd(&rs->epot, (double)e);
  }
  if (VFLAG) {
    R w[6] = {w0, w1, w2, w3, w4, w5};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      R v = warp_sum(w[c]);
      if ((t & 31) == 0) atomicAdd(&rs->virial[c], (double)v);
    }
  }
  {
    int m = nc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((t & 31) == 0) atomicMax(&rs->maxnc, m);
  }
#undef SLOT
#undef META
}

// ---- host-side launch ------------------------------------------------------
template <class R, int MAXNC, bool EFLAG, bool VFLAG>
static cudaError_t launch_force_t(cudaStream_t st, int N, const dbl4 *x, const int4 *q, const int *nbr,
                                  const int *cnt, const Geom &geo, const void *pairs, const void *trips, int nt,
                                  void *contrib, void *selfF, unsigned long long *mask, RunState *rs)
{
  using C = ForceCfg<R, MAXNC>;
  const size_t smem = sizeof(PairP<R>) * MAX_TYPES * MAX_TYPES + sizeof(TripP<R>) * MAX_TYPES * MAX_TYPES * MAX_TYPES +
                      C::smem_slots;
  auto kern = k_force<R, MAXNC, EFLAG, VFLAG>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (N == 0) return cudaSuccess;
  const int blocks = (N + C::threads - 1) / C::threads;
  kern<<<blocks, C::threads, smem, st>>>(N, x, q, nbr, cnt, geo, (const PairP<R> *)pairs, (const TripP<R> *)trips,
                                         nt, (typename V4t<R>::type *)contrib, (typename V4t<R>::type *)selfF, mask,
                                         rs);
  return cudaGetLastError();
}

template <class R, int MAXNC>
static cudaError_t launch_force_nc(cudaStream_t st, int eflag, int vflag, int N, const dbl4 *x, const int4 *q,
                                   const int *nbr, const int *cnt, const Geom &geo, const void *pairs,
                                   const void *trips, int nt, void *contrib, void *selfF, unsigned long long *mask,
                                   RunState *rs)
{
  if (vflag)
    return launch_force_t<R, MAXNC, true, true>(st, N, x, q, nbr, cnt, geo, pairs, trips, nt, contrib, selfF, mask, rs);
  if (eflag)
    return launch_force_t<R, MAXNC, true, false>(st, N, x, q, nbr, cnt, geo, pairs, trips, nt, contrib, selfF, mask, rs);
  return launch_force_t<R, MAXNC, false, false>(st, N, x, q, nbr, cnt, geo, pairs, trips, nt, contrib, selfF, mask, rs);
}

// Smallest compiled slot count >= need (8, 16, 32 or 64).
int force_slots_for(int need)
{
  if (need <= 8) return 8;
  if (need <= 16) return 16;
  if (need <= 32) return 32;
  return 64;
}

cudaError_t launch_force(cudaStream_t st, bool mixed, int maxnc, int eflag, int vflag, int N, const dbl4 *x,
                         const int4 *q, const int *nbr, const int *cnt, const Geom &geo, const void *pairs,
                         const void *trips, int nt, void *contrib, void *selfF, unsigned long long *mask,
                         RunState *rs)
{
#define TSF_CASE(NC)                                                                                          \
  case NC:                                                                                                    \
    return mixed ? launch_force_nc<float, NC>(st, eflag, vflag, N, x, q, nbr, cnt, geo, pairs, trips, nt, contrib, \
                                              selfF, mask, rs)                                                \
                 : launch_force_nc<double, NC>(st, eflag, vflag, N, x, q, nbr, cnt, geo, pairs, trips, nt,     \
                                               contrib, selfF, mask, rs);
  switch (force_slots_for(maxnc)) {
    TSF_CASE(8)
    TSF_CASE(16)
    TSF_CASE(32)
    TSF_CASE(64)
  }
#undef TSF_CASE
  return cudaErrorInvalidValue;
}

}  // namespace tsf
