// Internal device-side definitions shared by the kernels and the host runtime
// of libtersoff.so.  Nothing here is part of the C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tsf {

// 32-byte aligned float64 quadruple (one 256-bit access)
using dbl4 = double4_32a;
__host__ __device__ __forceinline__ dbl4 make_dbl4(double x, double y, double z, double w)
{
  return make_double4_32a(x, y, z, w);
}

constexpr int MAX_TYPES = 4;
constexpr int FAST_THREADS = 128;   // block size of the register force kernel

// arithmetic precision of a run (the values of tersoff_precision); the gather and the
// integrator also take PREC_MIXED_ACC64: mixed-mode contributions summed in float64
// (the literal float64 accumulation, measured beside the compensated float32 sum)
enum Prec : int { PREC_FP64 = 0, PREC_MIXED = 1, PREC_SINGLE = 2, PREC_MIXED_ACC64 = 3 };
constexpr int MAX_CAP = 64;       // neighbour-list capacity limit per atom (64-bit in-cutoff mask)
constexpr int NFIELDS = 14;       // {m, gamma, lambda3, c, d, h, n, beta, lambda2, B, R, D, lambda1, A}
enum Field { F_M = 0, F_GAMMA, F_LAM3, F_C, F_D, F_H, F_N, F_BETA, F_LAM2, F_B, F_R, F_DD, F_LAM1, F_A };

// sticky device status bits
enum : int {
  ST_NLIST_OVERFLOW = 1,   // an atom has more list entries than the list capacity
  ST_NC_OVERFLOW = 2,      // an atom has more in-cutoff neighbours than the force kernel's slot count
  ST_REV_MISSING = 4,      // reverse slot of a list entry not found (list not symmetric)
  ST_NONFINITE = 8,
  ST_ALLPAIRS_TOO_BIG = 16,
};

// Pair part of the table (row (ti,tj,tj)), derived constants in the kernel's precision.
template <class R>
struct PairP {
  R A, lam1, B, lam2;     // f_R = A e^{-lam1 r}, f_A = -B e^{-lam2 r}
  R lam1_lo, lam2_lo;     // float32 tables: lam - (float)lam, so that lam r is formed to ~1 ulp
  R beta, n, neg_inv2n;   // b = (1 + (beta zeta)^n)^(-1/(2n))
  R Rc, Dc;               // cutoff centre and half width
  R r_in, r_out, rc2;     // R - D, R + D, (R + D)^2
  R r_short;              // 0.7 R: mixed mode forms shorter pairs' geometry as head + tail
  R r_out_lo;             // float32 tables: (R + D) - (float)(R + D)
  R inv4D, dfc_scale;     // 1/(4D), -pi/(4D)
  R mu1h, mu1l, mu2h, mu2l;   // float32 tables: lambda1,2 * log2(e) as float head + tail
  R Aln2, Bln2;               // A ln 2, B ln 2 (the first-order tail factor of 2^-y)
  R hlam1, hlam2;             // lambda1 / 2, lambda2 / 2
};

// Angular part of the table (row (ti,tj,tk)).
template <class R>
struct TripP {
  R gamma, lam3, K, G2, d2, h;   // g = gamma + K u^2/(d2 + u^2), dg/dcos = -G2 u/(d2 + u^2)^2, u = h - cos
  R m3;                          // 1 when the lambda3 exponent is cubed (m = 3), else 0
  R pad;
};

// Constants of the register force kernel passed by value as a kernel argument (they
// then live in the constant bank and enter arithmetic as operands): kind 1 holds one
// type's row in p[0], t[0]; kind 2 holds two types, p[ti*2 + tj], t[(ti*2 + tj)*2 + tk].
template <class R>
struct KParams {
  PairP<R> p[4];
  TripP<R> t[8];
};

// How the register force kernel reads the table.  kind 0: the device table, staged
// in shared memory (any table with symmetric angular rows); kind 1 (one type) and
// kind 2 (two types): the kernel-argument copies below, for tables whose rows all
// have lambda3 = 0 (the lambda3 factor of Eq. 3 is then compiled out).
struct FastTab {
  int kind = 0;
  KParams<float> f{};
  KParams<double> d{};
};

// Box geometry.  Positions are also kept as 32-bit fixed point per axis:
// q = round(x / L * 2^32) mod 2^32, so q_j - q_i taken as int32 is the minimum
// image of x_j - x_i in units of L / 2^32, exact in integer arithmetic.
struct Geom {
  double L[3], invL[3];
  double to_q[3];     // 2^32 / L
  double q_to_d[3];   // L / 2^32
  float q_to_f[3];    // L / 2^32 rounded to float
  float q_to_f_lo[3]; // L / 2^32 - q_to_f (the rounding error of q_to_f)
};

// Device-resident run bookkeeping (one per MD state / computation).
struct RunState {
  int status;            // sticky ST_* bits
  int rebuild;           // nonzero: rebuild the list in this step
  int maxcount;          // max list length seen at the last build
  int maxnc;             // max in-cutoff count seen by the force kernel
  long long step;        // MD steps completed
  long long nrebuild;    // list builds done
  double epot;           // potential energy accumulator (force kernel)
  double ekin2;          // sum m v^2 accumulator (integrator), amu A^2/ps^2
  double virial[6];
  double epot_last;      // potential energy of the last completed step
  int nfast_blocks;      // blocks of the last force launch (partials to reduce)
  int ngen_blocks;       // blocks of the overflow kernel
  int nvv_blocks;        // blocks of the last integrator launch with kinetic energy
  double *trace;         // device trace [..][2] or null
  long long trace_k;     // trace row of the step in progress (1-based within a call)
  long long steps_left;  // steps still to run in the current graph launch
  int over_total;        // atoms the register force kernel queued for the general kernel
  int maxnc_t[MAX_TYPES];  // max in-cutoff count seen by the register force kernel, per atom type
};

// Atoms of a register-force-kernel launch: order[begin .. begin + count) (or atoms
// begin .. begin + count - 1 when order is null), slots per atom; block indices of
// the overflow queues and partial sums start at block_base.
struct ForceRoute {
  const int *order;
  int begin, count, slots, block_base;
};
struct ForceRoutes {
  int n;                 // 1 or 2 launches
  ForceRoute r[2];
};

// Ask L2 for the line holding p (no register result, no wait).
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Programmatic dependent launch.  A kernel launched with launch_dep while pdl_scope
// is active and its stream is being captured right behind a single kernel node may be
// scheduled before that kernel has drained; its first statement, griddep_wait(), holds
// it until that kernel has completed and its writes are visible (in a kernel launched
// the ordinary way it returns at once).  Every kernel launched with launch_dep calls
// griddep_wait() ahead of any global memory access.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

struct PdlFlag {
  static bool &on()
  {
    static thread_local bool f = false;
    return f;
  }
};
// Active for its lifetime on this host thread (graph captures of the step loop).
struct pdl_scope {
  bool prev;
  pdl_scope() : prev(PdlFlag::on()) { PdlFlag::on() = true; }
  ~pdl_scope() { PdlFlag::on() = prev; }
};

template <typename... K, typename... A>
inline cudaError_t launch_dep(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... args)
{
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 0;
  if (PdlFlag::on()) {
    // only behind exactly one kernel node of the graph being captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaGraphNodeType ty = cudaGraphNodeTypeEmpty;
    if (cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess &&
        cs == cudaStreamCaptureStatusActive && nd == 1 && cudaGraphNodeGetType(deps[0], &ty) == cudaSuccess &&
        ty == cudaGraphNodeTypeKernel)
      cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// minimum-image difference of two fixed-point coordinates, in units of L / 2^32
__host__ __device__ __forceinline__ int qdiff(int qj, int qi)
{
  return (int)((unsigned)qj - (unsigned)qi);
}

// Squared length used for every neighbour / cutoff decision.  Written with explicit
// round-to-nearest operations so that the compiler cannot contract or reassociate
// it differently in different places: the decision for (i, j) and (j, i) must be
// bitwise the same wherever it is taken.
__device__ __forceinline__ float r2_decide(float dx, float dy, float dz)
{
  return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
}
__device__ __forceinline__ double r2_decide(double dx, double dy, double dz)
{
  return __fma_rn(dx, dx, __fma_rn(dy, dy, __dmul_rn(dz, dz)));
}
// minimum image in float64, one rounding per operation in a fixed order
__device__ __forceinline__ double min_image(double d, double L, double invL)
{
  return __fma_rn(-L, rint(__dmul_rn(d, invL)), d);
}
// round(x * to_q) mod 2^32 with one rounding: adding 1.5 * 2^52 inside the FMA puts
// the nearest integer in the low mantissa bits (valid for |x * to_q| < 2^51).
__device__ __forceinline__ int fixed_q(double x, double to_q)
{
  return __double2loint(fma(x, to_q, 6755399441055744.0));
}

// fixed-point difference scaled to Angstrom, one rounding
__device__ __forceinline__ float q_scaled(int dq, float s) { return __fmul_rn((float)dq, s); }

// blocks of the general force kernel over the register kernel's overflow queues:
// four per SM of a GB300 (its shared-memory slots fit four blocks per SM)
constexpr int GEN_BLOCKS = 4 * 152;

constexpr int ST_BAD_TYPE = 32;
constexpr double ACCEL = 1.602176634e-19 / 1.66053906660e-27 * 1e-4;   // (eV/A)/amu in A/ps^2

// Atom record word w (fixed-point q.w; bits of the float64 position's w): the
// type in the low 3 bits, the system index above them (packed multi-system layouts).
constexpr int TYPE_BITS = 3;
__host__ __device__ __forceinline__ int type_of(int w) { return w & ((1 << TYPE_BITS) - 1); }
__host__ __device__ __forceinline__ int sys_of(int w) { return (int)((unsigned)w >> TYPE_BITS); }
__host__ __device__ __forceinline__ int make_w(int type, int sys) { return type | (sys << TYPE_BITS); }

// Constant description of one system of a (possibly packed) layout.
struct SysTab {
  Geom geo;                 // its box
  int nc[3];                // its cell grid
  int cell_off;             // its first cell in the global cell numbering
  int atom_off;             // its first atom
  int natoms;
  double dt;                // ps
  double kick[MAX_TYPES];   // dt/2 * ACCEL / m per type
};

// Run control of one system (device-updated every step).
struct SysCtl {
  long long steps_left;     // steps this system still runs
  int open;                 // velocities at the half step: a closing kick is pending
  int rebuild;              // some atom of this system moved skin/2 since its last list build
};

// Squared neighbour-list radius per type pair, (r_C(a,b) + skin)^2 with a small
// safety margin, float32 and symmetric (rl2[a][b] == rl2[b][a]), so that the pairs
// (i,j) and (j,i) are decided identically.
struct PairRadii {
  float rl2[MAX_TYPES * MAX_TYPES];
};

// Atom record of the cell-ordered copy used by the list build: fixed-point x, y, z
// and, in w, the atom index in the low CELL_IDX_BITS bits with its type above them.
constexpr int CELL_IDX_BITS = 30;
constexpr int CELL_IDX_MASK = (1 << CELL_IDX_BITS) - 1;
constexpr int64_t MAX_LIST_ATOMS = CELL_IDX_MASK;   // atoms per neighbour list

struct CellGrid {
  int nc[3];
  int ncell;
  PairRadii radii;   // list radius per type pair
};

}  // namespace tsf
