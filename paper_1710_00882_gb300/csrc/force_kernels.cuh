// Tersoff energy/force kernels: Algorithm 1 of the paper, one thread (or, for
// atoms with many neighbours, one warp) per atom i.
//
// Per atom i the thread
//   0. walks i's Verlet list once and marks the in-cutoff entries (Sec. 3: skin
//      atoms are tested once and never enter the K loops);
//   1. packs the in-cutoff neighbours into slots: unit vector, r, 1/r, f_C(r),
//      f_C'(r), type, list slot;
//   2. first K loop: zeta_ij for every slot j (Eq. 3); then the pair term
//      V(i,j,zeta_ij) (Eqs. 1-2), its r-derivative and dV/dzeta;
//   3. second K loop: the derivatives of zeta(i,j,k) scaled by dV/dzeta (the
//      restructuring of Sec. 2: zeta is complete before any derivative is formed).
//
// Fast kernel (k_force_reg): slots live in registers (compile-time slot count 4
// or 8, loops fully unrolled; the 8-slot kernel keeps four slot fields in shared
// memory and sorts its block's atoms by in-cutoff count before the K loops, so that
// each warp's lanes share their trip counts).  Both K loops run over unordered neighbour pairs
// {j,k}: cos(theta), g and g' are shared by zeta(i,j,k) and zeta(i,k,j) whenever
// the angular constants of rows (i,j,k) and (i,k,j) agree (Tersoff's tables take
// them from atom i), so each is evaluated once per pair instead of twice.  Atoms
// with more in-cutoff neighbours than slots are queued, per block and in order,
// for the warp kernel.
//
// Warp kernel (k_force_warp): one warp per queued atom, up to 64 in-cutoff
// neighbours in shared-memory slots, ordered (j,k) terms spread over the lanes.
//
// General kernel (k_force_gen): one thread per atom, slots in per-thread shared
// memory (8..64), loops over ordered (j,k) as in Algorithm 1; runs every atom for
// tables whose rows (i,j,k) and (i,k,j) differ in their angular constants.
//
// Scatter: all force contributions of i's terms on neighbour j are summed per j in
// the thread and written once, to slot s of i's list (contrib[s][i]); the force of
// i's terms on i itself is minus their sum (translation invariance).  No atomics:
// the gather (integrate.cu) reads, for each atom m and in-cutoff slot s of its list,
// the contribution at the flat index rev[s][m] (m's slot in its neighbour's list)
// and adds them in list order, so forces are bitwise reproducible.  Energy and
// virial go to per-block partial sums that a single block reduces in a fixed order.
//
// Precision: the math policy M (MathD: FP64 mode; MathF: mixed mode; MathS:
// single mode) fixes the real type R and how distances and exponentials are formed.
// Mixed and single modes both form the relative vector d_ij from the exact int32
// difference of 32-bit fixed-point coordinates.  Mixed mode rounds it once to float
// for pairs with 0.7 R <= r <= R - D and splits it into head and tail (d_ij within
// ~1 ulp, r = rh + rl) for pairs in the f_C taper or shorter (pair_geom_mixed), and
// exp(-lambda r) forms lambda r with an FMA-exact product from lambda as head + tail,
// because the pair term's r-derivative is a difference of two terms ~10x larger than
// itself and a rounded lambda would bias every pair alike.  Single mode (the paper's
// all-float32 variant, Sec. 4) rounds the difference once to float, takes r from
// rsqrt and exp from one ex2, and sums everything in float32.
//
// This header holds the kernels and their template launchers; each precision is
// instantiated in a translation unit of its own (force_fp64.cu, force_mixed.cu,
// force_single.cu) so that the three compile in parallel.
#pragma once
#include <type_traits>

#include "internal.cuh"

namespace tsf {

template <class R> struct V4t;
template <> struct V4t<float> { using type = float4; };
template <> struct V4t<double> { using type = dbl4; };

constexpr float L2E_F = 1.44269502f;                   // log2(e) rounded to float
constexpr float L2E_F_LO = 1.925963033500011e-08f;     // log2(e) - L2E_F

// ---- math of the two precisions ------------------------------------------

struct MathF {
  using R = float;
  static constexpr bool fine = true;   // head+tail exponents; head+tail distances where pair_geom_mixed asks
  static __device__ __forceinline__ float rcp(float x)
  {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float rsqrt(float x)
  {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float lg2(float x)
  {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float ex2(float x)
  {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  // e^{-x} for x = xh + xl (|xl| << |xh|): e^{-x} = 2^{-x log2 e}; the product
  // xh * log2(e) is split exactly with an FMA and the small remainder applied to
  // first order, so the result carries the error of one ex2 only.
  static __device__ __forceinline__ float expneg2(float xh, float xl)
  {
    // explicit round-to-nearest operations: a contracted product would break the split
    const float yh = __fmul_rn(xh, L2E_F);
    const float yl = __fadd_rn(__fmaf_rn(xh, L2E_F, -yh), __fmaf_rn(xh, L2E_F_LO, __fmul_rn(xl, L2E_F)));
    return __fmul_rn(ex2(-yh), __fmaf_rn(-yl, 0.69314718f, 1.0f));
  }
  // e^{-(lh + ll)(rh + rl)}: lambda and r both given as float head + tail
  static __device__ __forceinline__ float expneg(float lh, float ll, float rh, float rl)
  {
    const float p = __fmul_rn(lh, rh);
    const float pe = __fadd_rn(__fmaf_rn(lh, rh, -p), __fmaf_rn(ll, rh, __fmul_rn(lh, rl)));
    return expneg2(p, pe);
  }
  static __device__ __forceinline__ float expv(float x) { return expneg2(-x, 0.0f); }
  static __device__ __forceinline__ void sincospi(float t, float *s, float *c) { sincospif(t, s, c); }
};

struct MathD {
  using R = double;
  static constexpr bool fine = false;
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
  static __device__ __forceinline__ double lg2(double x) { return ::log2(x); }
  static __device__ __forceinline__ double ex2(double x) { return ::exp2(x); }
  static __device__ __forceinline__ double expneg(double lh, double, double r, double) { return ::exp(-lh * r); }
  static __device__ __forceinline__ double expv(double x) { return ::exp(x); }
  static __device__ __forceinline__ void sincospi(double t, double *s, double *c) { ::sincospi(t, s, c); }
};

// Single mode: the float32 operations of MathF without the compensation: e^{-x}
// from one ex2 of the rounded product, so lambda r carries the rounding of r and of
// the product (a relative error of a few 1e-7 in f_R and f_A).
struct MathS {
  using R = float;
  static constexpr bool fine = false;
  static __device__ __forceinline__ float rcp(float x) { return MathF::rcp(x); }
  static __device__ __forceinline__ float rsqrt(float x) { return MathF::rsqrt(x); }
  static __device__ __forceinline__ float lg2(float x) { return MathF::lg2(x); }
  static __device__ __forceinline__ float ex2(float x) { return MathF::ex2(x); }
  static __device__ __forceinline__ float expneg(float lh, float, float rh, float)
  {
    return MathF::ex2(-(lh * rh) * L2E_F);
  }
  static __device__ __forceinline__ float expv(float x) { return MathF::ex2(x * L2E_F); }
  static __device__ __forceinline__ void sincospi(float t, float *s, float *c) { sincospif(t, s, c); }
};

// f_C and f_C' for r = rh + rl < R + D.  In the taper
//   f_C = 1/2 - 1/2 sin(pi (r - R)/(2D)) = sin^2(pi w),  w = (R + D - r)/(4D),
//   f_C' = -pi/(4D) cos(pi (r - R)/(2D)) = -pi/(4D) sin(2 pi w),
// identities that avoid the cancellation of 1/2 - 1/2 sin near the outer cutoff,
// where f_C is small and zeta, hence dV/dzeta, is most sensitive to it.  R + D - r
// is formed from head+tail values so it keeps its relative accuracy there.
template <class M, class R>
__device__ __forceinline__ void cutoff_fn(R rh, R rl, const PairP<R> &P, R &fc, R &dfc)
{
  if (rh <= P.r_in) {
    fc = R(1);
    dfc = R(0);
  } else {
    const R w = ((P.r_out - rh) + (P.r_out_lo - rl)) * P.inv4D;
    R s, c;
    M::sincospi(w, &s, &c);
    fc = s * s;
    dfc = P.dfc_scale * R(2) * s * c;
  }
}

// bond order b(zeta) (Eq. 2) and db/dzeta
template <class M, class R>
__device__ __forceinline__ void bond_order(R zeta, const PairP<R> &P, R &b, R &db)
{
  b = R(1);
  db = R(0);
  if (zeta > R(0)) {
    const R xb = M::ex2(P.n * M::lg2(P.beta * zeta));
    b = M::ex2(P.neg_inv2n * M::lg2(R(1) + xb));
    db = R(-0.5) * b * xb * M::rcp((R(1) + xb) * zeta);
  }
}

// minimum-image relative vector of a fixed-point pair, accurate to ~1 ulp:
// the int32 difference is split into a 24-bit head and an 8-bit tail (both exact in
// float) and the scale into float head + tail.
// (Error-free transformations: every operation is an explicit round-to-nearest
// intrinsic, which the compiler never contracts or reassociates.)
__device__ __forceinline__ void qd_fine(int dq, float sh, float sl, float &dh, float &dl)
{
  const float h = (float)(dq & ~0xff);
  const float l = (float)(dq & 0xff);
  const float p = __fmul_rn(h, sh);
  const float t = __fmaf_rn(h, sl, __fmaf_rn(l, sh, __fmaf_rn(h, sh, -p)));
  dh = __fadd_rn(p, t);
  dl = __fsub_rn(t, __fsub_rn(dh, p));   // |p| >= |t|: exact tail
}

// r = |d| as head + tail from d given as head + tail per component: squares split
// exactly with FMAs, summed with TwoSum, square root refined by one Newton step.
// Returns rh (the rounded distance), rl (its tail) and 1/rh.
__device__ __forceinline__ void norm_fine(const float (&dh)[3], const float (&dl)[3], float &rh, float &rl,
                                          float &irh)
{
  float sq[3], er[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    sq[a] = __fmul_rn(dh[a], dh[a]);
    er[a] = __fmaf_rn(__fmul_rn(2.0f, dh[a]), dl[a], __fmaf_rn(dh[a], dh[a], -sq[a]));
  }
  const float s1 = __fadd_rn(sq[0], sq[1]);
  const float bb1 = __fsub_rn(s1, sq[0]);
  const float e1 = __fadd_rn(__fsub_rn(sq[0], __fsub_rn(s1, bb1)), __fsub_rn(sq[1], bb1));
  const float s2 = __fadd_rn(s1, sq[2]);
  const float bb2 = __fsub_rn(s2, s1);
  const float e2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, bb2)), __fsub_rn(sq[2], bb2));
  const float r2l = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(er[0], __fadd_rn(er[1], er[2])));
  irh = MathF::rsqrt(s2);
  rh = __fmul_rn(s2, irh);
  rl = __fmul_rn(__fmul_rn(__fadd_rn(__fmaf_rn(-rh, rh, s2), r2l), 0.5f), irh);
}

// Mixed-mode geometry of the pair (i, j): relative vector d, r = rh + rl and 1/rh.
// A pair with 0.7 R <= r <= R - D (r from the rounded float32 difference) keeps that
// float32 geometry, rl = 0: the bulk of the pairs of solids (f_C = 1), whose energy
// and forces are insensitive to r's last bits (a relative error of ~1e-7; the
// exponents keep lambda as head + tail).  A pair in the f_C taper, where R + D - r
// must keep its relative accuracy, or a short, strongly repulsive pair (large forces)
// takes head + tail geometry.  Every kernel forms a pair's geometry with this one
// function, so it does not depend on the kernel that evaluates the pair.
__device__ __forceinline__ void pair_geom_mixed(const int4 &qj, const int4 &qi, const Geom *gp, float r_short,
                                                float r_in, float &dx, float &dy, float &dz, float &r, float &rl,
                                                float &inv)
{
  const int ex = qdiff(qj.x, qi.x), ey = qdiff(qj.y, qi.y), ez = qdiff(qj.z, qi.z);
  const float fx = q_scaled(ex, gp->q_to_f[0]), fy = q_scaled(ey, gp->q_to_f[1]), fz = q_scaled(ez, gp->q_to_f[2]);
  const float r2 = r2_decide(fx, fy, fz);
  const float is = MathF::rsqrt(r2);
  const float rs = __fmul_rn(r2, is);
  if (rs <= r_in && rs >= r_short) {
    dx = fx; dy = fy; dz = fz;
    r = rs; rl = 0.0f; inv = is;
  } else {
    float dh[3], dl[3];
    qd_fine(ex, gp->q_to_f[0], gp->q_to_f_lo[0], dh[0], dl[0]);
    qd_fine(ey, gp->q_to_f[1], gp->q_to_f_lo[1], dh[1], dl[1]);
    qd_fine(ez, gp->q_to_f[2], gp->q_to_f_lo[2], dh[2], dl[2]);
    norm_fine(dh, dl, r, rl, inv);
    dx = dh[0]; dy = dh[1]; dz = dh[2];
  }
}

template <class R> __device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-block partial of (E, W[6]) in a fixed order: float/double per-thread values,
// warp sums in R, warps combined in warp order in float64 (in float32 when F32SUM:
// single mode's all-float32 accumulation).
template <class R, int T, bool F32SUM = false>
__device__ __forceinline__ void block_partial(const R (&v)[7], bool eflag, bool vflag, double *out)
{
  __shared__ double sw[T / 32][7];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = 0; c < 7; ++c) {
    if ((c == 0 && !eflag) || (c > 0 && !vflag)) continue;
    R s = warp_sum(v[c]);
    if (lane == 0) sw[w][c] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 7; ++c) {
      const bool skip = (c == 0 && !eflag) || (c > 0 && !vflag);
      if (F32SUM) {
        float a = 0.0f;
        for (int k = 0; k < T / 32; ++k) a += skip ? 0.0f : (float)sw[k][c];
        out[c] = (double)a;
      } else {
        double a = 0.0;
        for (int k = 0; k < T / 32; ++k) a += skip ? 0.0 : sw[k][c];
        out[c] = a;
      }
    }
    out[7] = 0.0;
  }
}

// ============================================================================
// fast kernel: register slots, unordered neighbour pairs

// A e^{-lambda r} in float32 (mixed mode) for r = rh + rl: y = mu r with mu =
// lambda log2(e) given as float head muh + tail mul; muh rh is split exactly with an
// FMA, so y = yh + yl with |yl| ~ 1e-6, and 2^{-y} = 2^{-yh} (1 - yl ln 2) to first
// order in the tail, with A folded into the tail factor (Aln2 = A ln 2).
__device__ __forceinline__ float aexp_mixed(float A, float Aln2, float muh, float mul, float rh, float rl)
{
  const float yh = __fmul_rn(muh, rh);
  const float yl = __fadd_rn(__fmaf_rn(muh, rh, -yh), __fmaf_rn(mul, rh, __fmul_rn(muh, rl)));
  return __fmul_rn(MathF::ex2(-yh), __fmaf_rn(-Aln2, yl, A));
}

// KIND: how the table is read (FastTab): 0 from the device table through shared
// memory, with the lambda3 factor of Eq. 3 evaluated per term; 1 (one type) and 2
// (two types) from the kernel argument kp (constant bank), lambda3 = 0 compiled out.
template <class M, int MAXNC, int KIND, bool EFLAG, bool VFLAG>
__global__ void __launch_bounds__(FAST_THREADS, sizeof(typename M::R) == 4 ? (MAXNC == 4 ? 7 : 5) : 1)
k_force_reg(int ld, const dbl4 *__restrict__ x, const int4 *__restrict__ q, const int *__restrict__ nbr,
            const int *__restrict__ cnt, const SysTab *__restrict__ sys,
            const PairP<typename M::R> *__restrict__ gpairs,
            const TripP<typename M::R> *__restrict__ gtrips, int nt,
            const __grid_constant__ KParams<typename M::R> kp,
            typename V4t<typename M::R>::type *__restrict__ contrib,
            typename V4t<typename M::R>::type *__restrict__ selfF, unsigned long long *__restrict__ mask,
            int *__restrict__ work, int *__restrict__ nwork, double *__restrict__ partial, RunState *rs,
            double *__restrict__ eatom, const int *__restrict__ order, int begin, int count, int block_base,
            int stats, int pf)
{
  using R = typename M::R;
  using V4 = typename V4t<R>::type;
  constexpr bool MIXED = sizeof(R) == 4;   // float32 arithmetic on fixed-point positions (mixed or single)
  constexpr bool L3 = KIND == 0;           // the lambda3 factor is evaluated
  constexpr bool ONE = KIND == 1;
  constexpr int T = FAST_THREADS;
  __shared__ PairP<R> spairs[KIND == 0 ? MAX_TYPES * MAX_TYPES : 1];
  __shared__ TripP<R> strips[KIND == 0 ? MAX_TYPES * MAX_TYPES * MAX_TYPES : 1];
  __shared__ int warp_over[T / 32];

  griddep_wait();
  if (rs->status != 0) return;   // uniform across the grid
  if constexpr (KIND == 0) {
    if (threadIdx.x < nt * nt) spairs[threadIdx.x] = gpairs[threadIdx.x];
    if (threadIdx.x < nt * nt * nt) strips[threadIdx.x] = gtrips[threadIdx.x];
    __syncthreads();
  }
  // table rows: (ti,tj,tj) for the pair terms, (ti,tj,tk) for the angular terms.
  // Returned by value: fields of kp at fixed offsets then enter the arithmetic as
  // constant-bank operands (a reference would be a generic pointer into the
  // parameter space, read with loads).
  auto pairp = [&](int ti_, int tj_) -> PairP<R> {
    if constexpr (KIND == 0) return spairs[ti_ * nt + tj_];
    else if constexpr (KIND == 1) return kp.p[0];
    else return kp.p[ti_ * 2 + tj_];
  };
  auto tripp = [&](int ti_, int tj_, int tk_) -> TripP<R> {
    if constexpr (KIND == 0) return strips[(ti_ * nt + tj_) * nt + tk_];
    else if constexpr (KIND == 1) return kp.t[0];
    else return kp.t[(ti_ * 2 + tj_) * 2 + tk_];
  };

  const int t = threadIdx.x;
  const int tg = blockIdx.x * T + t;
  // (both reassigned by the count sort of the 8-slot kernels, below)
  bool active = tg < count;
  int i = active ? (order ? order[begin + tg] : begin + tg) : 0;
  if (i < 0) {
    // padding entry of a route order (segments that start a warp): nothing here
    active = false;
    i = 0;
  }
  const int fb = block_base + (int)blockIdx.x;   // this block's queue and partial-sum row
  // pf atoms ahead (one resident wave of blocks): the counts and list rows the next
  // wave reads, from DRAM after a cold start, are requested into L2 now
  if (pf > 0 && !order && tg + pf < count) {
    const int ip = begin + tg + pf;
    prefetch_l2(cnt + ip);
#pragma unroll
    for (int s = 0; s < MAXNC; ++s) prefetch_l2(nbr + (size_t)s * ld + ip);
  }

  int ti = 0;
  int4 qi = make_int4(0, 0, 0, 0);
  dbl4 xi = make_dbl4(0, 0, 0, 0);
  unsigned long long mb = 0ull;
  int n = 0;
  const Geom *gp = &sys[0].geo;   // geometry of atom i's system (all its neighbours share it)
  if (active) {
    int w;
    if (MIXED) {
      qi = q[i];
      w = qi.w;
    } else {
      xi = x[i];
      w = (int)__double_as_longlong(xi.w);
    }
    ti = type_of(w);
    gp = &sys[sys_of(w)].geo;
    n = cnt[i];
  }
  // Direct path: the whole list fits the slots, so slot s is list entry s (entries
  // outside the cutoff get f_C = f_C' = 0 and contribute nothing) and every load is
  // issued in one unrolled burst.  Otherwise the list is packed: a first pass marks
  // in-cutoff entries, the second loads them into consecutive slots.
  // (8-slot kernels always pack: their atoms change threads before the slots are filled)
  constexpr bool SORT = MAXNC == 8;
  const bool direct = !SORT && active && n <= MAXNC;

  // Slot fields.  The 8-slot kernels keep the four that the K loops read least (the
  // distance tail, 1/r, f_C' and the slot's list entry and type) in shared memory,
  // one column per thread, so that more blocks fit an SM; the others stay in registers.
  constexpr bool SMEM = MAXNC == 8;
  __shared__ R s_rl[SMEM ? MAXNC : 1][T], s_ir[SMEM ? MAXNC : 1][T], s_dfc[SMEM ? MAXNC : 1][T];
  __shared__ int s_meta[SMEM ? MAXNC : 1][T];
  R ux[MAXNC], uy[MAXNC], uz[MAXNC], rr[MAXNC], fc[MAXNC];
  R rl_r[SMEM ? 1 : MAXNC], ir_r[SMEM ? 1 : MAXNC], dfc_r[SMEM ? 1 : MAXNC];
  int meta_r[SMEM ? 1 : MAXNC];
  auto rl = [&](int s) -> R & { if constexpr (SMEM) return s_rl[s][t]; else return rl_r[s]; };
  auto ir = [&](int s) -> R & { if constexpr (SMEM) return s_ir[s][t]; else return ir_r[s]; };
  auto dfc = [&](int s) -> R & { if constexpr (SMEM) return s_dfc[s][t]; else return dfc_r[s]; };
  auto meta = [&](int s) -> int & { if constexpr (SMEM) return s_meta[s][t]; else return meta_r[s]; };
#pragma unroll
  for (int s = 0; s < MAXNC; ++s) {
    ux[s] = uy[s] = uz[s] = R(0);
    rr[s] = R(1);
    ir(s) = R(1);
    rl(s) = fc[s] = dfc(s) = R(0);
    meta(s) = 0;
  }

  // 8-slot mixed kernels: the first pass over the list stages each in-cutoff
  // neighbour's fixed-point record, list entry and type in shared memory, in the
  // column of the thread that tested it; after the count sort the evaluating thread
  // fills its slots from that column instead of gathering the neighbours again.
  constexpr bool STAGE = SORT && MIXED;
  __shared__ int4 s_qn[STAGE ? MAXNC : 1][STAGE ? T : 1];
  __shared__ int s_en[STAGE ? MAXNC : 1][STAGE ? T : 1];
  __shared__ int4 s_qi[STAGE ? T : 1];
  __shared__ int s_src[STAGE ? T : 1];

  // geometry of slot s from list entry e (neighbour j): unit vector, r, 1/r, f_C, f_C'
  auto fill_slot = [&](int s, int e, int j, const int4 &qj, const dbl4 &xj, int tj) {
    R dx, dy, dz, r, rlo, inv;
    const PairP<R> Pp = pairp(ti, tj);
    if (MIXED && M::fine) {
      // the kernels share pair_geom_mixed, so an atom's forces do not depend on which
      // of them evaluates it
      float gx, gy, gz, gr, grl, gi;
      pair_geom_mixed(qj, qi, gp, (float)Pp.r_short, (float)Pp.r_in, gx, gy, gz, gr, grl, gi);
      dx = (R)gx; dy = (R)gy; dz = (R)gz;
      r = (R)gr; rlo = (R)grl; inv = (R)gi;
    } else if (MIXED) {
      dx = (R)q_scaled(qdiff(qj.x, qi.x), gp->q_to_f[0]);
      dy = (R)q_scaled(qdiff(qj.y, qi.y), gp->q_to_f[1]);
      dz = (R)q_scaled(qdiff(qj.z, qi.z), gp->q_to_f[2]);
      const R r2 = r2_decide(dx, dy, dz);
      inv = M::rsqrt(r2);
      r = r2 * inv;
      rlo = R(0);
    } else {
      dx = (R)min_image(__dsub_rn(xj.x, xi.x), gp->L[0], gp->invL[0]);
      dy = (R)min_image(__dsub_rn(xj.y, xi.y), gp->L[1], gp->invL[1]);
      dz = (R)min_image(__dsub_rn(xj.z, xi.z), gp->L[2], gp->invL[2]);
      const R r2 = r2_decide(dx, dy, dz);
      inv = M::rsqrt(r2);
      r = r2 * inv;
      rlo = R(0);
    }
    ux[s] = dx * inv;
    uy[s] = dy * inv;
    uz[s] = dz * inv;
    rr[s] = r;
    rl(s) = rlo;
    ir(s) = inv;
    cutoff_fn<M>(r, rlo, Pp, fc[s], dfc(s));
    meta(s) = e | (tj << 8);
  };

  // cheap in-cutoff test of entry (i, j)
  auto in_cutoff = [&](const int4 &qj, const dbl4 &xj, int tj) -> bool {
    R r2;
    if (MIXED) {
      r2 = r2_decide(q_scaled(qdiff(qj.x, qi.x), gp->q_to_f[0]), q_scaled(qdiff(qj.y, qi.y), gp->q_to_f[1]),
                     q_scaled(qdiff(qj.z, qi.z), gp->q_to_f[2]));
    } else {
      r2 = r2_decide(min_image(__dsub_rn(xj.x, xi.x), gp->L[0], gp->invL[0]),
                     min_image(__dsub_rn(xj.y, xi.y), gp->L[1], gp->invL[1]),
                     min_image(__dsub_rn(xj.z, xi.z), gp->L[2], gp->invL[2]));
    }
    return r2 < pairp(ti, tj).rc2;
  };

  int nc_all = 0;
  if (direct) {
    int jj[MAXNC];
#pragma unroll
    for (int s = 0; s < MAXNC; ++s) jj[s] = s < n ? nbr[(size_t)s * ld + i] : i;
    int4 qq[MAXNC];
    dbl4 xx[MAXNC];
#pragma unroll
    for (int s = 0; s < MAXNC; ++s) {
      if (MIXED) qq[s] = q[jj[s]];
      else xx[s] = x[jj[s]];
    }
#pragma unroll
    for (int s = 0; s < MAXNC; ++s) {
      if (s < n) {
        const int tj = type_of(MIXED ? qq[s].w : (int)__double_as_longlong(xx[s].w));
        if (in_cutoff(qq[s], xx[s], tj)) {
          mb |= 1ull << s;
          fill_slot(s, s, jj[s], qq[s], xx[s], tj);
        } else {
          meta(s) = s | (tj << 8);
        }
      }
    }
    nc_all = __popcll(mb);
  } else if (active) {
    // PU list entries per round: their loads are issued together
    constexpr int PU = MIXED ? 4 : 2;
    int staged = 0;
    for (int s0 = 0; s0 < n; s0 += PU) {
      int jj[PU];
#pragma unroll
      for (int k = 0; k < PU; ++k) jj[k] = s0 + k < n ? nbr[(size_t)(s0 + k) * ld + i] : i;
      int4 qq[PU];
      dbl4 xx[PU];
#pragma unroll
      for (int k = 0; k < PU; ++k) {
        if (MIXED) qq[k] = q[jj[k]];
        else xx[k] = x[jj[k]];
      }
#pragma unroll
      for (int k = 0; k < PU; ++k) {
        const int tj = type_of(MIXED ? qq[k].w : (int)__double_as_longlong(xx[k].w));
        if (s0 + k < n && in_cutoff(qq[k], xx[k], tj)) {
          mb |= 1ull << (s0 + k);
          if constexpr (STAGE) {
            if (staged < MAXNC) {
              s_qn[staged][t] = qq[k];
              s_en[staged][t] = (s0 + k) | (tj << 8);
            }
            ++staged;
          }
        }
      }
    }
    nc_all = __popcll(mb);
  }
  bool over = !direct && nc_all > MAXNC;
  // queue atoms with too many neighbours, per block and in thread order
  {
    const unsigned bal = __ballot_sync(0xffffffffu, over);
    if ((t & 31) == 0) warp_over[t >> 5] = __popc(bal);
    __syncthreads();
    if (over) {
      int base = 0;
      for (int w = 0; w < (t >> 5); ++w) base += warp_over[w];
      const int k = base + __popc(bal & ((1u << (t & 31)) - 1u));
      work[(size_t)fb * T + k] = i;
    }
    if (t == 0) {
      int s = 0;
      for (int w = 0; w < T / 32; ++w) s += warp_over[w];
      nwork[fb] = s;
      if (s > 0) atomicAdd(&rs->over_total, s);
    }
  }
  if (stats) {
    // largest in-cutoff counts, overall and per type (they choose the slot counts of
    // later launches): warp maxima, then one atomic per block and statistic
    __shared__ unsigned smax[T / 32][MAX_TYPES + 1];
    const unsigned m = __reduce_max_sync(0xffffffffu, (unsigned)nc_all);
    if ((t & 31) == 0) smax[t >> 5][MAX_TYPES] = m;
    for (int ty = 0; ty < (ONE ? 1 : nt); ++ty) {
      const unsigned mt = __reduce_max_sync(0xffffffffu, (unsigned)((active && (ONE || ti == ty)) ? nc_all : 0));
      if ((t & 31) == 0) smax[t >> 5][ty] = mt;
    }
    __syncthreads();
    if (t <= MAX_TYPES && (t == MAX_TYPES || t < (ONE ? 1 : nt))) {
      unsigned bm = 0;
      for (int w = 0; w < T / 32; ++w) bm = max(bm, smax[w][t]);
      if (bm > 0) atomicMax(t == MAX_TYPES ? &rs->maxnc : &rs->maxnc_t[t], (int)bm);
    }
  }
  if (SORT) {
    // Count sort of the block's atoms (8-slot kernels): the unrolled pair loops below
    // run, per warp, up to the largest in-cutoff count of its lanes, and counts of 4..8
    // mixed in one warp make every warp run all 28 pairs.  The atoms this block
    // evaluates are reassigned to threads in order of their count (stable: ties keep
    // thread order), so each warp holds similar counts.  An atom's result does not
    // depend on the thread that evaluates it.
    constexpr int NK = MAXNC + 2;   // keys 0..MAXNC; MAXNC + 1: not evaluated here
    __shared__ int s_cnt[T / 32][NK];
    __shared__ int s_atom[T];
    __shared__ unsigned long long s_mb[T];
    const int lane = t & 31, w = t >> 5;
    const int key = (active && !over) ? nc_all : MAXNC + 1;
    int r = 0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      const unsigned b = __ballot_sync(0xffffffffu, key == k);
      if (lane == 0) s_cnt[w][k] = __popc(b);
      if (key == k) r = __popc(b & ((1u << lane) - 1u));
    }
    __syncthreads();
    for (int k = 0; k < key; ++k)
      for (int v = 0; v < T / 32; ++v) r += s_cnt[v][k];
    for (int v = 0; v < w; ++v) r += s_cnt[v][key];
    s_atom[r] = key <= MAXNC ? i : -1;
    s_mb[r] = mb;
    if constexpr (STAGE) {
      s_src[r] = t;
      s_qi[r] = qi;
    }
    __syncthreads();
    const int inew = s_atom[t];
    active = inew >= 0;
    over = false;
    i = active ? inew : 0;
    mb = active ? s_mb[t] : 0ull;
    nc_all = __popcll(mb);
    if (active) {
      int wn;
      if constexpr (STAGE) {
        qi = s_qi[t];
        wn = qi.w;
      } else if (MIXED) {
        qi = q[i];
        wn = qi.w;
      } else {
        xi = x[i];
        wn = (int)__double_as_longlong(xi.w);
      }
      ti = type_of(wn);
      gp = &sys[sys_of(wn)].geo;
    }
  }
  // slots in use: the whole list on the direct path, the packed in-cutoff entries else
  const int nc = direct ? n : (over ? 0 : nc_all);
  if (STAGE && active) {
    const int src = s_src[t];
#pragma unroll
    for (int s = 0; s < MAXNC; ++s) {
      if (s < nc) {
        const int en = s_en[s][src];
        fill_slot(s, en & 0xff, 0, s_qn[s][src], make_dbl4(0, 0, 0, 0), en >> 8);
      }
    }
  } else if (!direct && !over && active) {
    unsigned long long rem = mb;
#pragma unroll
    for (int s = 0; s < MAXNC; ++s) {
      if (s < nc) {
        const int e = __ffsll((long long)rem) - 1;
        rem &= rem - 1;
        const int j = nbr[(size_t)e * ld + i];
        int4 qj = make_int4(0, 0, 0, 0);
        dbl4 xj = make_dbl4(0, 0, 0, 0);
        int tj;
        if (MIXED) { qj = q[j]; tj = type_of(qj.w); }
        else { xj = x[j]; tj = type_of((int)__double_as_longlong(xj.w)); }
        fill_slot(s, e, j, qj, xj, tj);
      }
    }
  }

  // ---- K loops and pair terms ------------------------------------------------
  // Evaluated in one of two forms: FULL, when every lane of the warp has all MAXNC
  // slots within the cutoff and inside R - D (f_C = 1, f_C' = 0; the usual case of
  // diamond-like solids), with no bounds test per slot pair and the f_C factors
  // compiled out; else the general form.  Both compute the same terms; the sums into
  // Ab and e_i are explicit fma, so the terms the general form adds on top are exact
  // zeros when f_C = 1 and f_C' = 0.  Callers that need an atom's result independent
  // of the other atoms in its warp give each independent set of atoms its own warps.
  R zeta[MAXNC], dz[MAXNC], Ab[MAXNC], Fx[MAXNC], Fy[MAXNC], Fz[MAXNC];
  R e_i = R(0);
  auto evaluate = [&](auto full_c) {
    constexpr bool FULL = decltype(full_c)::value;
    const int ncx = FULL ? MAXNC : nc;
    auto FC = [&](int s) -> R { if constexpr (FULL) return R(1); else return fc[s]; };
    auto DFC = [&](int s) -> R { if constexpr (FULL) return R(0); else return dfc(s); };
    // ---- first K loop: zeta over unordered pairs --------------------------------
    // The 4-slot kernels with a kernel-argument table keep cos, g and g' of their 6
    // unordered pairs in registers for the second K loop (the 8-slot kernel's 28 would
    // not fit): computed once, not twice.
    constexpr bool CACHE = MAXNC == 4 && KIND != 0;
    constexpr int CN = CACHE ? MAXNC : 1;
    [[maybe_unused]] R c_cos[CN][CN], c_g[CN][CN], c_dg[CN][CN];
#pragma unroll
    for (int s = 0; s < MAXNC; ++s) zeta[s] = R(0);
#pragma unroll
    for (int a = 0; a < MAXNC; ++a) {
#pragma unroll
      for (int b = a + 1; b < MAXNC; ++b) {
        if (b < ncx) {
          const TripP<R> Tp = tripp(ti, meta(a) >> 8, meta(b) >> 8);
          const R cost = ux[a] * ux[b] + uy[a] * uy[b] + uz[a] * uz[b];
          const R u = Tp.h - cost;
          const R inv = M::rcp(Tp.d2 + u * u);
          const R w = u * inv;
          const R g = Tp.gamma + Tp.K * u * w;   // gamma + K u^2/(d2 + u^2)
          if constexpr (CACHE) {
            c_cos[a][b] = cost;
            c_g[a][b] = g;
            c_dg[a][b] = -Tp.G2 * w * inv;       // dg/dcos = -G2 u/(d2 + u^2)^2
          }
          if constexpr (L3) {
            R eab = R(1), eba = R(1);
            if (Tp.lam3 != R(0)) {
              R arg = Tp.lam3 * (rr[a] - rr[b]);
              if (Tp.m3 != R(0)) arg = arg * arg * arg;
              eab = M::expv(arg);
              eba = M::expv(-arg);
            }
            zeta[a] += FC(b) * g * eab;
            zeta[b] += FC(a) * g * eba;
          } else {
            zeta[a] += FC(b) * g;
            zeta[b] += FC(a) * g;
          }
        }
      }
    }

    // ---- pair terms ---------------------------------------------------------------
    // The force of i's terms on neighbour a is -(Ab[a] u_a + C_a): Ab collects every
    // term along the bond i-a (the pair term's dV/dr first), C_a = (Fx, Fy, Fz) the
    // terms along the other bonds, so that each term along a's own bond costs one
    // scalar update instead of a vector one.
#pragma unroll
    for (int a = 0; a < MAXNC; ++a) {
      dz[a] = Ab[a] = Fx[a] = Fy[a] = Fz[a] = R(0);
      if (a < ncx) {
        const PairP<R> P = pairp(ti, meta(a) >> 8);
        R fR, fA;
        if constexpr (MIXED && M::fine) {
          fR = (R)aexp_mixed(P.A, P.Aln2, P.mu1h, P.mu1l, rr[a], rl(a));
          fA = (R)aexp_mixed(-P.B, -P.Bln2, P.mu2h, P.mu2l, rr[a], rl(a));
        } else {
          fR = P.A * M::expneg(P.lam1, P.lam1_lo, rr[a], rl(a));
          fA = -P.B * M::expneg(P.lam2, P.lam2_lo, rr[a], rl(a));
        }
        R bij, dbij;
        bond_order<M>(zeta[a], P, bij, dbij);
        const R bfA = bij * fA;
        const R pr = fR + bfA;
        e_i = fma(R(0.5) * FC(a), pr, e_i);
        // dV/dr of V = fc (fR + b fA)/2 at fixed zeta: fc' pr/2 - fc (lambda1 fR + lambda2 b fA)/2
        const R lam = fma(P.hlam1, fR, P.hlam2 * bfA);
        if constexpr (FULL) Ab[a] = -lam;
        else Ab[a] = fma(R(0.5) * DFC(a), pr, -(FC(a) * lam));
        dz[a] = R(0.5) * FC(a) * fA * dbij;
      }
    }

    // ---- second K loop: zeta derivatives over unordered pairs -------------------
    // With P = dV/dzeta_ij fc_k e_jk, Q = dV/dzeta_ik fc_j e_kj, S = (P + Q) g'
    // (e_jk the lambda3 factor, arg' its exponent's derivative):
    //   F_j -= S/r_j u_k + (dV/dzeta_ik fc'_j g e_kj - S/r_j cos + (P - Q) g arg') u_j
    //   F_k -= S/r_k u_j + (dV/dzeta_ij fc'_k g e_jk - S/r_k cos - (P - Q) g arg') u_k
    // (the u_j and u_k coefficients go to Ab[j], Ab[k]).
#pragma unroll
    for (int a = 0; a < MAXNC; ++a) {
#pragma unroll
      for (int b = a + 1; b < MAXNC; ++b) {
        if (b < ncx) {
          const TripP<R> Tp = tripp(ti, meta(a) >> 8, meta(b) >> 8);
          R cost, g, dg;
          if constexpr (CACHE) {
            cost = c_cos[a][b];
            g = c_g[a][b];
            dg = c_dg[a][b];
          } else {
            cost = ux[a] * ux[b] + uy[a] * uy[b] + uz[a] * uz[b];
            const R u = Tp.h - cost;
            const R inv = M::rcp(Tp.d2 + u * u);
            const R w = u * inv;
            g = Tp.gamma + Tp.K * u * w;
            dg = -Tp.G2 * w * inv;
          }
          R cj, ck;
          if constexpr (L3) {
            R eab = R(1), eba = R(1), darg = R(0);
            if (Tp.lam3 != R(0)) {
              const R tt = Tp.lam3 * (rr[a] - rr[b]);
              R arg = tt;
              darg = Tp.lam3;
              if (Tp.m3 != R(0)) {
                arg = tt * tt * tt;
                darg = R(3) * Tp.lam3 * tt * tt;
              }
              eab = M::expv(arg);
              eba = M::expv(-arg);
            }
            const R Pv = dz[a] * FC(b) * eab;
            const R Qv = dz[b] * FC(a) * eba;
            const R S = (Pv + Qv) * dg;
            const R PQd = (Pv - Qv) * g * darg;
            cj = S * ir(a);
            ck = S * ir(b);
            Ab[a] += dz[b] * DFC(a) * g * eba - cj * cost + PQd;
            Ab[b] += dz[a] * DFC(b) * g * eab - ck * cost - PQd;
          } else {
            const R S = (dz[a] * FC(b) + dz[b] * FC(a)) * dg;
            cj = S * ir(a);
            ck = S * ir(b);
            Ab[a] = fma(-cj, cost, Ab[a]);
            Ab[b] = fma(-ck, cost, Ab[b]);
            if constexpr (!FULL) {
              Ab[a] = fma(dz[b] * DFC(a), g, Ab[a]);
              Ab[b] = fma(dz[a] * DFC(b), g, Ab[b]);
            }
          }
          Fx[a] -= cj * ux[b];
          Fy[a] -= cj * uy[b];
          Fz[a] -= cj * uz[b];
          Fx[b] -= ck * ux[a];
          Fy[b] -= ck * uy[a];
          Fz[b] -= ck * uz[a];
        }
      }
    }
  };
  constexpr bool HAS_FULL = MAXNC == 4 && KIND != 0;
  if constexpr (HAS_FULL) {
    bool full = active && !over && nc == MAXNC && nc_all == MAXNC;
#pragma unroll
    // f_C' = 0 too: near R - D the taper's f_C can round to 1 while its slope does not
    for (int s = 0; s < MAXNC; ++s) full = full && fc[s] == R(1) && dfc(s) == R(0);
    if (__all_sync(0xffffffffu, full)) evaluate(std::true_type{});
    else evaluate(std::false_type{});
  } else {
    evaluate(std::false_type{});
  }

  // ---- outputs ------------------------------------------------------------------
  R red[7] = {e_i, R(0), R(0), R(0), R(0), R(0), R(0)};
  if (active && !over) {
    R fix = R(0), fiy = R(0), fiz = R(0);
#pragma unroll
    for (int a = 0; a < MAXNC; ++a) {
      if (a < nc && ((mb >> (meta(a) & 0xff)) & 1ull)) {
        Fx[a] -= Ab[a] * ux[a];
        Fy[a] -= Ab[a] * uy[a];
        Fz[a] -= Ab[a] * uz[a];
        fix -= Fx[a];
        fiy -= Fy[a];
        fiz -= Fz[a];
        V4 c;
        c.x = Fx[a]; c.y = Fy[a]; c.z = Fz[a]; c.w = R(0);
        contrib[(size_t)(meta(a) & 0xff) * ld + i] = c;
        if (VFLAG) {
          const R dx = rr[a] * ux[a], dy = rr[a] * uy[a], dzz = rr[a] * uz[a];
          red[1] += dx * Fx[a]; red[2] += dy * Fy[a]; red[3] += dzz * Fz[a];
          red[4] += dx * Fy[a]; red[5] += dx * Fz[a]; red[6] += dy * Fz[a];
        }
      }
    }
    V4 c;
    c.x = fix; c.y = fiy; c.z = fiz; c.w = R(0);
    selfF[i] = c;
    mask[i] = mb;
    if (eatom) eatom[i] = (double)e_i;
  }
  if (EFLAG || VFLAG) block_partial<R, T, MIXED && !M::fine>(red, EFLAG, VFLAG, partial + (size_t)fb * 8);
}

// ============================================================================
// off[k] = sum of in[0..k) for k <= n (n <= GEN_SUB), computed by the T threads of a
// block: each thread sums a run of entries, then the runs are offset in order.
constexpr int GEN_SUB = 256;
template <int T>
__device__ __forceinline__ void block_exclusive_offsets(const int *__restrict__ in, int n, int *off)
{
  constexpr int PER = (GEN_SUB + T - 1) / T;
  __shared__ int runs[T + 1];
  const int t = threadIdx.x;
  int v[PER], sum = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = t * PER + k;
    v[k] = idx < n ? in[idx] : 0;
    sum += v[k];
  }
  runs[t] = sum;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int k = 0; k < T; ++k) {
      const int x = runs[k];
      runs[k] = acc;
      acc += x;
    }
    runs[T] = acc;
  }
  __syncthreads();
  int acc = runs[t];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = t * PER + k;
    if (idx < n) off[idx] = acc;
    acc += v[k];
  }
  if (t == 0) off[n] = runs[T];
  __syncthreads();
}

// general kernel: per-thread shared-memory slots, ordered (j,k) loops

constexpr int NRF = 12;   // real fields per slot
enum { S_UX = 0, S_UY, S_UZ, S_R, S_IR, S_FC, S_DFC, S_DZ, S_FX, S_FY, S_FZ, S_RL };

template <class R, int MAXNC>
struct GenCfg {
  static constexpr int slot_bytes = NRF * (int)sizeof(R) + 4;
  static constexpr int raw = 98304 / (MAXNC * slot_bytes);
  static constexpr int threads = raw >= 128 ? 128 : raw >= 64 ? 64 : 32;
  static constexpr size_t smem_slots = (size_t)threads * MAXNC * slot_bytes;
};

// Evaluates every atom (one thread per atom) with ordered (j,k) loops as in
// Algorithm 1: the path for tables whose angular constants differ between rows
// (i,j,k) and (i,k,j), and the reference the register kernel is tested against.
template <class M, int MAXNC, bool EFLAG, bool VFLAG>
__global__ void __launch_bounds__(GenCfg<typename M::R, MAXNC>::threads)
k_force_gen(int N, int ld, const dbl4 *__restrict__ x, const int4 *__restrict__ q, const int *__restrict__ nbr,
            const int *__restrict__ cnt, const SysTab *__restrict__ sys,
            const PairP<typename M::R> *__restrict__ gpairs, const TripP<typename M::R> *__restrict__ gtrips, int nt,
            typename V4t<typename M::R>::type *__restrict__ contrib,
            typename V4t<typename M::R>::type *__restrict__ selfF, unsigned long long *__restrict__ mask,
            double *__restrict__ partial, RunState *rs, double *__restrict__ eatom)
{
  using R = typename M::R;
  using V4 = typename V4t<R>::type;
  constexpr int T = GenCfg<R, MAXNC>::threads;
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
#define SLOT(f, s) sr[((f) * MAXNC + (s)) * T + t]
#define META(s) smeta[(s) * T + t]
  R red[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
  bool overflow = false;
  int maxnc = 0;

  // one atom: in-cutoff slots, first K loop and pair terms, second K loop, outputs
  auto process = [&](const int i) {
    int ti, w;
    int4 qi = make_int4(0, 0, 0, 0);
    dbl4 xi = make_dbl4(0, 0, 0, 0);
    if (MIXED) {
      qi = q[i];
      w = qi.w;
    } else {
      xi = x[i];
      w = (int)__double_as_longlong(xi.w);
    }
    ti = type_of(w);
    // atoms of a freed range of a packed layout belong to a system without atoms
    if (sys[sys_of(w)].natoms == 0) return;
    const Geom *gp = &sys[sys_of(w)].geo;
    int nc = 0;
    unsigned long long mbits = 0ull;
    const int n = cnt[i];
    // GU list entries per round: their index and position loads are issued together
    constexpr int GU = 4;
    for (int s0 = 0; s0 < n; s0 += GU) {
      int jj[GU];
#pragma unroll
      for (int k = 0; k < GU; ++k) jj[k] = s0 + k < n ? nbr[(size_t)(s0 + k) * ld + i] : i;
      int4 qq[GU];
      dbl4 xx[GU];
#pragma unroll
      for (int k = 0; k < GU; ++k) {
        if (MIXED) qq[k] = q[jj[k]];
        else xx[k] = x[jj[k]];
      }
#pragma unroll
      for (int k = 0; k < GU; ++k) {
        const int s = s0 + k;
        if (s >= n) continue;
        R dx, dy, dz;
        int tj;
        if (MIXED) {
          tj = type_of(qq[k].w);
          dx = (R)q_scaled(qdiff(qq[k].x, qi.x), gp->q_to_f[0]);
          dy = (R)q_scaled(qdiff(qq[k].y, qi.y), gp->q_to_f[1]);
          dz = (R)q_scaled(qdiff(qq[k].z, qi.z), gp->q_to_f[2]);
        } else {
          tj = type_of((int)__double_as_longlong(xx[k].w));
          dx = (R)min_image(__dsub_rn(xx[k].x, xi.x), gp->L[0], gp->invL[0]);
          dy = (R)min_image(__dsub_rn(xx[k].y, xi.y), gp->L[1], gp->invL[1]);
          dz = (R)min_image(__dsub_rn(xx[k].z, xi.z), gp->L[2], gp->invL[2]);
        }
        const R r2 = r2_decide(dx, dy, dz);
        const PairP<R> &P = pairs[ti * nt + tj];
        if (r2 < P.rc2) {
          if (nc < MAXNC) {
            R r, rlo, inv;
            if (MIXED && M::fine) {
              float gx, gy, gz, gr, grl, gi;
              pair_geom_mixed(qq[k], qi, gp, (float)P.r_short, (float)P.r_in, gx, gy, gz, gr, grl, gi);
              dx = (R)gx; dy = (R)gy; dz = (R)gz;
              r = (R)gr; rlo = (R)grl; inv = (R)gi;
            } else {
              const R rf2 = r2_decide(dx, dy, dz);
              inv = M::rsqrt(rf2);
              r = rf2 * inv;
              rlo = R(0);
            }
            R fcv, dfcv;
            cutoff_fn<M>(r, rlo, P, fcv, dfcv);
            SLOT(S_UX, nc) = dx * inv;
            SLOT(S_UY, nc) = dy * inv;
            SLOT(S_UZ, nc) = dz * inv;
            SLOT(S_R, nc) = r;
            SLOT(S_RL, nc) = rlo;
            SLOT(S_IR, nc) = inv;
            SLOT(S_FC, nc) = fcv;
            SLOT(S_DFC, nc) = dfcv;
            META(nc) = s | (tj << 8);
          }
          ++nc;
          mbits |= 1ull << s;
        }
      }
    }
    maxnc = max(maxnc, nc);
    if (nc > MAXNC) {
      overflow = true;
      return;
    }

    // first K loop and pair terms
    R e_atom = R(0);
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
        const R g = Tp.gamma + Tp.K * u2 * M::rcp(Tp.d2 + u2);
        R ex = R(1);
        if (Tp.lam3 != R(0)) {
          R arg = Tp.lam3 * (ra - SLOT(S_R, b));
          if (Tp.m3 != R(0)) arg = arg * arg * arg;
          ex = M::expv(arg);
        }
        zeta += SLOT(S_FC, b) * g * ex;
      }
      const PairP<R> &P = pairs[ti * nt + tj];
      const R fcv = SLOT(S_FC, a), dfcv = SLOT(S_DFC, a);
      const R fR = P.A * M::expneg(P.lam1, P.lam1_lo, ra, SLOT(S_RL, a));
      const R fA = -P.B * M::expneg(P.lam2, P.lam2_lo, ra, SLOT(S_RL, a));
      R bij, dbij;
      bond_order<M>(zeta, P, bij, dbij);
      const R pr = fR + bij * fA;
      red[0] += R(0.5) * fcv * pr;
      e_atom += R(0.5) * fcv * pr;
      const R dvdr = R(0.5) * (dfcv * pr + fcv * (-P.lam1 * fR - bij * P.lam2 * fA));
      SLOT(S_DZ, a) = R(0.5) * fcv * fA * dbij;
      SLOT(S_FX, a) = -dvdr * uax;
      SLOT(S_FY, a) = -dvdr * uay;
      SLOT(S_FZ, a) = -dvdr * uaz;
    }

    // second K loop
    for (int a = 0; a < nc; ++a) {
      const R dzv = SLOT(S_DZ, a);
      if (dzv == R(0)) continue;
      const int tj = META(a) >> 8;
      const R uax = SLOT(S_UX, a), uay = SLOT(S_UY, a), uaz = SLOT(S_UZ, a), ra = SLOT(S_R, a),
              ira = SLOT(S_IR, a);
      const TripP<R> *Tj = trips + (ti * nt + tj) * nt;
      R fjx = R(0), fjy = R(0), fjz = R(0);
      for (int b = 0; b < nc; ++b) {
        if (b == a) continue;
        const TripP<R> &Tp = Tj[META(b) >> 8];
        const R ubx = SLOT(S_UX, b), uby = SLOT(S_UY, b), ubz = SLOT(S_UZ, b), irb = SLOT(S_IR, b);
        const R cost = uax * ubx + uay * uby + uaz * ubz;
        const R u = Tp.h - cost;
        const R u2 = u * u;
        const R inv = M::rcp(Tp.d2 + u2);
        const R g = Tp.gamma + Tp.K * u2 * inv;
        const R dg = -Tp.G2 * u * inv * inv;
        R ex = R(1), darg = R(0);
        if (Tp.lam3 != R(0)) {
          const R tt = Tp.lam3 * (ra - SLOT(S_R, b));
          R arg = tt;
          darg = Tp.lam3;
          if (Tp.m3 != R(0)) {
            arg = tt * tt * tt;
            darg = R(3) * Tp.lam3 * tt * tt;
          }
          ex = M::expv(arg);
        }
        const R fcb = SLOT(S_FC, b), dfcb = SLOT(S_DFC, b);
        const R a1 = fcb * ex * dg;
        const R a2 = fcb * ex * g * darg;
        const R a3 = dfcb * g * ex;
        const R cj = a1 * ira;
        const R dzjx = cj * (ubx - cost * uax) + a2 * uax;
        const R dzjy = cj * (uby - cost * uay) + a2 * uay;
        const R dzjz = cj * (ubz - cost * uaz) + a2 * uaz;
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

    R fix = R(0), fiy = R(0), fiz = R(0);
    for (int a = 0; a < nc; ++a) {
      const R fx = SLOT(S_FX, a), fy = SLOT(S_FY, a), fz = SLOT(S_FZ, a);
      fix -= fx;
      fiy -= fy;
      fiz -= fz;
      V4 c;
      c.x = fx; c.y = fy; c.z = fz; c.w = R(0);
      contrib[(size_t)(META(a) & 0xff) * ld + i] = c;
      if (VFLAG) {
        const R r = SLOT(S_R, a);
        const R dx = r * SLOT(S_UX, a), dy = r * SLOT(S_UY, a), dz = r * SLOT(S_UZ, a);
        red[1] += dx * fx; red[2] += dy * fy; red[3] += dz * fz;
        red[4] += dx * fy; red[5] += dx * fz; red[6] += dy * fz;
      }
    }
    V4 c;
    c.x = fix; c.y = fiy; c.z = fiz; c.w = R(0);
    selfF[i] = c;
    mask[i] = mbits;
    if (eatom) eatom[i] = (double)e_atom;
  };

  {
    const int i = (int)blockIdx.x * T + t;
    if (i < N) process(i);
  }
  if (overflow) atomicOr(&rs->status, ST_NC_OVERFLOW);
  if (maxnc > 0) atomicMax(&rs->maxnc, maxnc);
  if (EFLAG || VFLAG) block_partial<R, T, MIXED && !M::fine>(red, EFLAG, VFLAG, partial + (size_t)blockIdx.x * 8);
#undef SLOT
#undef META
}

// ============================================================================
// warp kernel: one warp per atom of the register kernel's overflow queues

constexpr int WARP_BLOCK = 128;   // 4 warps per block
constexpr int WSLOTS = MAX_CAP;   // slots per warp: a list holds at most MAX_CAP entries

// The atoms the register kernel queued (more in-cutoff neighbours than its slots)
// are evaluated one per warp, with ordered (j,k) terms as in Algorithm 1:
//   - the lanes test list entries lane, lane + 32, ...; a ballot packs the in-cutoff
//     ones into the warp's shared-memory slots in list order;
//   - lane a computes zeta for slot a (Eq. 3) and its pair term (Eqs. 1-2);
//   - lane c sums the whole force on neighbour c: its pair term, the derivatives of
//     zeta(i,c,p) with respect to x_c and those of zeta(i,p,c), over p in slot order.
// Every sum runs in a fixed order, so results are deterministic.  Block b takes the
// contiguous run of register-kernel blocks [b G, (b + 1) G), G = ceil(nfast /
// gridDim.x), as one flat queue in order; its warps take entries w, w + 4, ...
template <class M, bool EFLAG, bool VFLAG>
__global__ void __launch_bounds__(WARP_BLOCK)
k_force_warp(int ld, const dbl4 *__restrict__ x, const int4 *__restrict__ q, const int *__restrict__ nbr,
             const int *__restrict__ cnt, const SysTab *__restrict__ sys,
             const PairP<typename M::R> *__restrict__ gpairs, const TripP<typename M::R> *__restrict__ gtrips,
             int nt, typename V4t<typename M::R>::type *__restrict__ contrib,
             typename V4t<typename M::R>::type *__restrict__ selfF, unsigned long long *__restrict__ mask,
             const int *__restrict__ work, const int *__restrict__ nwork, int nfast, double *__restrict__ partial,
             RunState *rs, double *__restrict__ eatom)
{
  using R = typename M::R;
  using V4 = typename V4t<R>::type;
  constexpr int T = WARP_BLOCK, NW = T / 32;
  constexpr bool MIXED = sizeof(R) == 4;
  __shared__ PairP<R> pairs[MAX_TYPES * MAX_TYPES];
  __shared__ TripP<R> trips[MAX_TYPES * MAX_TYPES * MAX_TYPES];
  __shared__ R sl[NW][NRF][WSLOTS];
  __shared__ int smeta[NW][WSLOTS];
  __shared__ int qoff[GEN_SUB + 1];

  griddep_wait();
  if (rs->status != 0) return;   // uniform across the grid
  if (rs->over_total == 0) {
    // no atom was queued: leave zero partial sums and stop
    if ((EFLAG || VFLAG) && threadIdx.x < 8) partial[(size_t)blockIdx.x * 8 + threadIdx.x] = 0.0;
    return;
  }
  for (int k = threadIdx.x; k < nt * nt; k += T) pairs[k] = gpairs[k];
  for (int k = threadIdx.x; k < nt * nt * nt; k += T) trips[k] = gtrips[k];
  __syncthreads();

  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  R(&S)[NRF][WSLOTS] = sl[w];
  int *meta = smeta[w];
  R red[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
  int maxnc = 0;

  // atom i, by all 32 lanes of the warp
  auto process = [&](const int i) {
    int w_i;
    int4 qi = make_int4(0, 0, 0, 0);
    dbl4 xi = make_dbl4(0, 0, 0, 0);
    if (MIXED) {
      qi = q[i];
      w_i = qi.w;
    } else {
      xi = x[i];
      w_i = (int)__double_as_longlong(xi.w);
    }
    const int ti = type_of(w_i);
    const Geom *gp = &sys[sys_of(w_i)].geo;
    const int n = cnt[i];
    unsigned long long mbits = 0ull;
    int nc = 0;
    for (int s0 = 0; s0 < n; s0 += 32) {
      const int s = s0 + lane;
      bool inc = false;
      int tj = 0;
      int4 qj = make_int4(0, 0, 0, 0);
      dbl4 xj = make_dbl4(0, 0, 0, 0);
      R dx = R(0), dy = R(0), dz = R(0);
      if (s < n) {
        const int j = nbr[(size_t)s * ld + i];
        if (MIXED) {
          qj = q[j];
          tj = type_of(qj.w);
          dx = (R)q_scaled(qdiff(qj.x, qi.x), gp->q_to_f[0]);
          dy = (R)q_scaled(qdiff(qj.y, qi.y), gp->q_to_f[1]);
          dz = (R)q_scaled(qdiff(qj.z, qi.z), gp->q_to_f[2]);
        } else {
          xj = x[j];
          tj = type_of((int)__double_as_longlong(xj.w));
          dx = (R)min_image(__dsub_rn(xj.x, xi.x), gp->L[0], gp->invL[0]);
          dy = (R)min_image(__dsub_rn(xj.y, xi.y), gp->L[1], gp->invL[1]);
          dz = (R)min_image(__dsub_rn(xj.z, xi.z), gp->L[2], gp->invL[2]);
        }
        inc = r2_decide(dx, dy, dz) < pairs[ti * nt + tj].rc2;
      }
      const unsigned b = __ballot_sync(0xffffffffu, inc);
      if (inc) {
        const int slot = nc + __popc(b & ((1u << lane) - 1u));
        const PairP<R> &P = pairs[ti * nt + tj];
        R r, rlo, inv;
        if (MIXED && M::fine) {
          float gx, gy, gz, gr, grl, gi;
          pair_geom_mixed(qj, qi, gp, (float)P.r_short, (float)P.r_in, gx, gy, gz, gr, grl, gi);
          dx = (R)gx; dy = (R)gy; dz = (R)gz;
          r = (R)gr; rlo = (R)grl; inv = (R)gi;
        } else {
          const R rf2 = r2_decide(dx, dy, dz);
          inv = M::rsqrt(rf2);
          r = rf2 * inv;
          rlo = R(0);
        }
        R fcv, dfcv;
        cutoff_fn<M>(r, rlo, P, fcv, dfcv);
        S[S_UX][slot] = dx * inv;
        S[S_UY][slot] = dy * inv;
        S[S_UZ][slot] = dz * inv;
        S[S_R][slot] = r;
        S[S_RL][slot] = rlo;
        S[S_IR][slot] = inv;
        S[S_FC][slot] = fcv;
        S[S_DFC][slot] = dfcv;
        meta[slot] = s | (tj << 8);
      }
      mbits |= (unsigned long long)b << s0;
      nc += __popc(b);
    }
    maxnc = max(maxnc, nc);
    __syncwarp();

    // zeta and the pair term of slot a
    R e_lane = R(0);
    for (int a = lane; a < nc; a += 32) {
      const int ta = meta[a] >> 8;
      const R uax = S[S_UX][a], uay = S[S_UY][a], uaz = S[S_UZ][a], ra = S[S_R][a];
      const TripP<R> *Ta = trips + (ti * nt + ta) * nt;
      R zeta = R(0);
      for (int p = 0; p < nc; ++p) {
        if (p == a) continue;
        const TripP<R> &Tp = Ta[meta[p] >> 8];
        const R cost = uax * S[S_UX][p] + uay * S[S_UY][p] + uaz * S[S_UZ][p];
        const R u = Tp.h - cost;
        const R u2 = u * u;
        const R g = Tp.gamma + Tp.K * u2 * M::rcp(Tp.d2 + u2);
        R ex = R(1);
        if (Tp.lam3 != R(0)) {
          R arg = Tp.lam3 * (ra - S[S_R][p]);
          if (Tp.m3 != R(0)) arg = arg * arg * arg;
          ex = M::expv(arg);
        }
        zeta += S[S_FC][p] * g * ex;
      }
      const PairP<R> &P = pairs[ti * nt + ta];
      const R fcv = S[S_FC][a], dfcv = S[S_DFC][a];
      const R fR = P.A * M::expneg(P.lam1, P.lam1_lo, ra, S[S_RL][a]);
      const R fA = -P.B * M::expneg(P.lam2, P.lam2_lo, ra, S[S_RL][a]);
      R bij, dbij;
      bond_order<M>(zeta, P, bij, dbij);
      const R pr = fR + bij * fA;
      e_lane += R(0.5) * fcv * pr;
      const R dvdr = R(0.5) * (dfcv * pr + fcv * (-P.lam1 * fR - bij * P.lam2 * fA));
      S[S_DZ][a] = R(0.5) * fcv * fA * dbij;
      S[S_FX][a] = -dvdr * uax;
      S[S_FY][a] = -dvdr * uay;
      S[S_FZ][a] = -dvdr * uaz;
    }
    __syncwarp();

    // the force on neighbour c
    R sx = R(0), sy = R(0), sz = R(0);
    for (int c = lane; c < nc; c += 32) {
      const int tc = meta[c] >> 8;
      const R ucx = S[S_UX][c], ucy = S[S_UY][c], ucz = S[S_UZ][c], rc = S[S_R][c], irc = S[S_IR][c];
      const R fcc = S[S_FC][c], dfcc = S[S_DFC][c], dzc = S[S_DZ][c];
      R fx = S[S_FX][c], fy = S[S_FY][c], fz = S[S_FZ][c];
      for (int p = 0; p < nc; ++p) {
        if (p == c) continue;
        const int tp = meta[p] >> 8;
        const R upx = S[S_UX][p], upy = S[S_UY][p], upz = S[S_UZ][p], rp = S[S_R][p];
        const R cost = ucx * upx + ucy * upy + ucz * upz;
        if (dzc != R(0)) {
          // zeta(i,c,p) with respect to x_c (c as j): row (ti, tc, tp)
          const TripP<R> &Tp = trips[(ti * nt + tc) * nt + tp];
          const R u = Tp.h - cost;
          const R u2 = u * u;
          const R inv = M::rcp(Tp.d2 + u2);
          const R g = Tp.gamma + Tp.K * u2 * inv;
          const R dg = -Tp.G2 * u * inv * inv;
          R ex = R(1), darg = R(0);
          if (Tp.lam3 != R(0)) {
            const R tt = Tp.lam3 * (rc - rp);
            R arg = tt;
            darg = Tp.lam3;
            if (Tp.m3 != R(0)) {
              arg = tt * tt * tt;
              darg = R(3) * Tp.lam3 * tt * tt;
            }
            ex = M::expv(arg);
          }
          const R fcp = S[S_FC][p];
          const R a1 = fcp * ex * dg;
          const R a2 = fcp * ex * g * darg;
          const R cj = a1 * irc;
          fx -= dzc * (cj * (upx - cost * ucx) + a2 * ucx);
          fy -= dzc * (cj * (upy - cost * ucy) + a2 * ucy);
          fz -= dzc * (cj * (upz - cost * ucz) + a2 * ucz);
        }
        const R dzp = S[S_DZ][p];
        if (dzp != R(0)) {
          // zeta(i,p,c) with respect to x_c (c as k): row (ti, tp, tc)
          const TripP<R> &Tp = trips[(ti * nt + tp) * nt + tc];
          const R u = Tp.h - cost;
          const R u2 = u * u;
          const R inv = M::rcp(Tp.d2 + u2);
          const R g = Tp.gamma + Tp.K * u2 * inv;
          const R dg = -Tp.G2 * u * inv * inv;
          R ex = R(1), darg = R(0);
          if (Tp.lam3 != R(0)) {
            const R tt = Tp.lam3 * (rp - rc);
            R arg = tt;
            darg = Tp.lam3;
            if (Tp.m3 != R(0)) {
              arg = tt * tt * tt;
              darg = R(3) * Tp.lam3 * tt * tt;
            }
            ex = M::expv(arg);
          }
          const R a1 = fcc * ex * dg;
          const R a2 = fcc * ex * g * darg;
          const R a3 = dfcc * g * ex;
          const R ck = a1 * irc;
          fx -= dzp * ((a3 - a2) * ucx + ck * (upx - cost * ucx));
          fy -= dzp * ((a3 - a2) * ucy + ck * (upy - cost * ucy));
          fz -= dzp * ((a3 - a2) * ucz + ck * (upz - cost * ucz));
        }
      }
      V4 o;
      o.x = fx; o.y = fy; o.z = fz; o.w = R(0);
      contrib[(size_t)(meta[c] & 0xff) * ld + i] = o;
      sx -= fx;
      sy -= fy;
      sz -= fz;
      if (VFLAG) {
        const R dx = rc * ucx, dy = rc * ucy, dzz = rc * ucz;
        red[1] += dx * fx; red[2] += dy * fy; red[3] += dzz * fz;
        red[4] += dx * fy; red[5] += dx * fz; red[6] += dy * fz;
      }
    }
    red[0] += e_lane;
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    sz = warp_sum(sz);
    const R e_atom = warp_sum(e_lane);
    if (lane == 0) {
      V4 o;
      o.x = sx; o.y = sy; o.z = sz; o.w = R(0);
      selfF[i] = o;
      mask[i] = mbits;
      if (eatom) eatom[i] = (double)e_atom;
    }
    __syncwarp();   // the slots are reused by the warp's next atom
  };

  const int G = (nfast + (int)gridDim.x - 1) / (int)gridDim.x;
  const int fb0 = (int)blockIdx.x * G, fb1 = min(fb0 + G, nfast);
  for (int sb = fb0; sb < fb1; sb += GEN_SUB) {
    const int ns = min(GEN_SUB, fb1 - sb);
    block_exclusive_offsets<T>(nwork + sb, ns, qoff);
    const int total = qoff[ns];
    for (int pidx = w; pidx < total; pidx += NW) {
      int lo = 0, hi = ns - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (qoff[mid] <= pidx) lo = mid; else hi = mid - 1;
      }
      process(work[(size_t)(sb + lo) * FAST_THREADS + (pidx - qoff[lo])]);
    }
    __syncthreads();
  }
  if (lane == 0 && maxnc > 0) atomicMax(&rs->maxnc, maxnc);
  if (EFLAG || VFLAG) block_partial<R, T, MIXED && !M::fine>(red, EFLAG, VFLAG, partial + (size_t)blockIdx.x * 8);
}


// ---- host-side launch ------------------------------------------------------

template <class M, int MAXNC, bool EFLAG, bool VFLAG>
static cudaError_t launch_gen_t(cudaStream_t st, int N, int ld, const dbl4 *x, const int4 *q, const int *nbr, const int *cnt,
                                const SysTab *sys, const void *pairs, const void *trips, int nt, void *contrib,
                                void *selfF, unsigned long long *mask, double *partial, RunState *rs, double *eatom)
{
  using R = typename M::R;
  using C = GenCfg<R, MAXNC>;
  const size_t smem = sizeof(PairP<R>) * MAX_TYPES * MAX_TYPES + sizeof(TripP<R>) * MAX_TYPES * MAX_TYPES * MAX_TYPES +
                      C::smem_slots;
  auto kern = k_force_gen<M, MAXNC, EFLAG, VFLAG>;
  if (N == 0) return cudaSuccess;
  // set on every launch: the attribute is per device, and launches come from the
  // caller's threads and the server's worker alike
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (N + C::threads - 1) / C::threads;
  kern<<<blocks, C::threads, smem, st>>>(N, ld, x, q, nbr, cnt, sys, (const PairP<R> *)pairs, (const TripP<R> *)trips,
                                         nt, (typename V4t<R>::type *)contrib, (typename V4t<R>::type *)selfF, mask,
                                         partial, rs, eatom);
  return cudaGetLastError();
}

template <class M, int MAXNC>
static cudaError_t launch_gen(cudaStream_t st, int eflag, int vflag, int N, int ld, const dbl4 *x, const int4 *q,
                              const int *nbr, const int *cnt, const SysTab *sys, const void *pairs, const void *trips,
                              int nt, void *contrib, void *selfF, unsigned long long *mask, double *partial,
                              RunState *rs, double *eatom)
{
  if (vflag)
    return launch_gen_t<M, MAXNC, true, true>(st, N, ld, x, q, nbr, cnt, sys, pairs, trips, nt, contrib, selfF, mask,
                                              partial, rs, eatom);
  if (eflag)
    return launch_gen_t<M, MAXNC, true, false>(st, N, ld, x, q, nbr, cnt, sys, pairs, trips, nt, contrib, selfF, mask,
                                               partial, rs, eatom);
  return launch_gen_t<M, MAXNC, false, false>(st, N, ld, x, q, nbr, cnt, sys, pairs, trips, nt, contrib, selfF, mask,
                                              partial, rs, eatom);
}

template <class R>
static int gen_threads(int slots)
{
  switch (slots) {
    case 8: return GenCfg<R, 8>::threads;
    case 16: return GenCfg<R, 16>::threads;
    case 32: return GenCfg<R, 32>::threads;
    default: return GenCfg<R, 64>::threads;
  }
}

template <class M>
static cudaError_t launch_gen_any(cudaStream_t st, int slots, int eflag, int vflag, int N, int ld, const dbl4 *x,
                                  const int4 *q, const int *nbr, const int *cnt, const SysTab *sys, const void *pairs,
                                  const void *trips, int nt, void *contrib, void *selfF, unsigned long long *mask,
                                  double *partial, RunState *rs, double *eatom)
{
#define TSF_GEN(NC)                                                                                                \
  case NC:                                                                                                         \
    return launch_gen<M, NC>(st, eflag, vflag, N, ld, x, q, nbr, cnt, sys, pairs, trips, nt, contrib, selfF, mask,     \
                             partial, rs, eatom);
  switch (slots) {
    TSF_GEN(8)
    TSF_GEN(16)
    TSF_GEN(32)
    TSF_GEN(64)
  }
#undef TSF_GEN
  return cudaErrorInvalidValue;
}

// the warp kernel over the register kernel's overflow queues (GEN_BLOCKS blocks)
template <class M>
static cudaError_t launch_warp(cudaStream_t st, int eflag, int vflag, int ld, const dbl4 *x, const int4 *q,
                               const int *nbr, const int *cnt, const SysTab *sys, const void *pairs, const void *trips,
                               int nt, void *contrib, void *selfF, unsigned long long *mask, const int *work,
                               const int *nwork, int nfast, double *partial, RunState *rs, double *eatom)
{
  using R = typename M::R;
  using P = const PairP<R> *;
  using Tt = const TripP<R> *;
  using V = typename V4t<R>::type *;
  auto k = vflag ? k_force_warp<M, true, true> : eflag ? k_force_warp<M, true, false> : k_force_warp<M, false, false>;
  return launch_dep(k, GEN_BLOCKS, WARP_BLOCK, 0, st, ld, x, q, nbr, cnt, sys, (P)pairs, (Tt)trips, nt, (V)contrib,
                    (V)selfF, mask, work, nwork, nfast, partial, rs, eatom);
}

// the kernel-argument table of the precision R
template <class R>
inline const KParams<R> &kparams_of(const FastTab &ft)
{
  if constexpr (std::is_same<R, float>::value) return ft.f;
  else return ft.d;
}

template <class M, int MAXNC, int KIND>
static cudaError_t launch_reg(cudaStream_t st, int eflag, int vflag, int ld, const dbl4 *x, const int4 *q,
                              const int *nbr, const int *cnt, const SysTab *sys, const void *pairs, const void *trips,
                              int nt, const FastTab &ft, void *contrib, void *selfF, unsigned long long *mask,
                              int *work, int *nwork, double *partial, RunState *rs, double *eatom,
                              const ForceRoute &rt, int stats)
{
  const int blocks = (rt.count + FAST_THREADS - 1) / FAST_THREADS;
  if (blocks == 0) return cudaSuccess;
  using R = typename M::R;
  using P = const PairP<R> *;
  using Tt = const TripP<R> *;
  using V = typename V4t<R>::type *;
  const KParams<R> &kp = kparams_of<R>(ft);
  // one resident wave of blocks (SMs x resident blocks x threads) of the launched form
  auto wave = [](auto kern) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, FAST_THREADS, 0);
    return sms * per * FAST_THREADS;
  };
  static const int pf_v = wave(k_force_reg<M, MAXNC, KIND, true, true>);
  static const int pf_e = wave(k_force_reg<M, MAXNC, KIND, true, false>);
  static const int pf_0 = wave(k_force_reg<M, MAXNC, KIND, false, false>);
  auto k = vflag ? k_force_reg<M, MAXNC, KIND, true, true>
                 : eflag ? k_force_reg<M, MAXNC, KIND, true, false> : k_force_reg<M, MAXNC, KIND, false, false>;
  return launch_dep(k, blocks, FAST_THREADS, 0, st, ld, x, q, nbr, cnt, sys, (P)pairs, (Tt)trips, nt, kp, (V)contrib,
                    (V)selfF, mask, work, nwork, partial, rs, eatom, rt.order, rt.begin, rt.count, rt.block_base, stats,
                    vflag ? pf_v : eflag ? pf_e : pf_0);
}

// The force kernels of one evaluation in the precision of M (launch_force_part in
// force.cu, which adds the partial-sum reduction, documents the arguments).  *rows:
// the partial-sum rows the launched kernels write (0: none launched).
template <class M>
cudaError_t launch_force_m(int part, cudaStream_t st, int fast_slots, const FastTab &ft, int gen_slots, int eflag,
                           int vflag, int N, int ld, const dbl4 *x, const int4 *q, const int *nbr, const int *cnt,
                           const SysTab *sys, const void *pairs, const void *trips, int nt, void *contrib,
                           void *selfF, unsigned long long *mask, int *work, int *nwork, double *partial, RunState *rs,
                           double *eatom, const ForceRoutes *routes, int stats, int *rows)
{
  using R = typename M::R;
  *rows = 0;
  if (N == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (fast_slots > 0) {
    ForceRoutes one{1, {{nullptr, 0, N, fast_slots, 0}, {nullptr, 0, 0, 0, 0}}};
    const ForceRoutes &RT = routes ? *routes : one;
    int nfast = 0;
    for (int k = 0; k < RT.n; ++k) {
      ForceRoute rt = RT.r[k];
      rt.block_base = nfast;
      nfast += (rt.count + FAST_THREADS - 1) / FAST_THREADS;
      if (!(part & 1)) continue;
#define TSF_REG_K(NC, K)                                                                                          \
  launch_reg<M, NC, K>(st, eflag, vflag, ld, x, q, nbr, cnt, sys, pairs, trips, nt, ft, contrib, selfF, mask, work, \
                       nwork, partial, rs, eatom, rt, stats)
#define TSF_REG(NC) \
  e = ft.kind == 1 ? TSF_REG_K(NC, 1) : ft.kind == 2 ? TSF_REG_K(NC, 2) : TSF_REG_K(NC, 0);
      if (rt.slots <= 4) { TSF_REG(4) } else { TSF_REG(8) }
#undef TSF_REG
#undef TSF_REG_K
      if (e != cudaSuccess) return e;
    }
    if (!(part & 2)) return cudaSuccess;
    double *gp = partial + (size_t)nfast * 8;
    e = launch_warp<M>(st, eflag, vflag, ld, x, q, nbr, cnt, sys, pairs, trips, nt, contrib, selfF, mask, work, nwork,
                       nfast, gp, rs, eatom);
    if (e == cudaSuccess) *rows = nfast + GEN_BLOCKS;
  } else {
    if (!(part & 2)) return cudaSuccess;
    e = launch_gen_any<M>(st, gen_slots, eflag, vflag, N, ld, x, q, nbr, cnt, sys, pairs, trips, nt, contrib, selfF, mask,
                          partial, rs, eatom);
    const int T = gen_threads<R>(gen_slots);
    if (e == cudaSuccess) *rows = (N + T - 1) / T;
  }
  return e;
}

}  // namespace tsf
