/*
 * tersoff.h -- C ABI of libtersoff.so: the Tersoff many-body potential on one
 * GB300 (sm_103a).
 *
 * The operations follow Sec. 2 of Hoehnerbach, Ismail & Bientinesi, "The
 * Tersoff many-body potential: sustainable performance through vectorization":
 *
 *   E       = 1/2 sum_i sum_{j: r_ij < r_C} f_C(r_ij) [f_R(r_ij) + b_ij f_A(r_ij)]   (Eq. 1)
 *   b_ij    = (1 + beta^n zeta_ij^n)^(-1/(2n))                                       (Eq. 2)
 *   zeta_ij = sum_{k != i,j: r_ik < r_C} f_C(r_ik) g(theta_ijk) exp(lambda3 (r_ij - r_ik))   (Eq. 3)
 *
 * and the forces of Algorithm 1 (per i and in-cutoff neighbour j: accumulate
 * zeta_ij over neighbours k, apply V(i,j,zeta_ij) and its r-derivative, then
 * scatter dV/dzeta * dzeta(i,j,k)/dx to i, j and k).  The 1/2 of Eq. 1 is
 * Tersoff's convention (the paper prints Eq. 1 without it).  f_C, f_R, f_A and
 * g, which the paper omits as "trivial definitions", are Tersoff's forms:
 *   f_C(r) = 1 (r < R-D), 1/2 - 1/2 sin(pi (r-R)/(2D)) (|r-R| <= D), 0 (r > R+D)
 *   f_R(r) = A exp(-lambda1 r),  f_A(r) = -B exp(-lambda2 r)
 *   g      = gamma (1 + c^2/d^2 - c^2/(d^2 + (h - cos theta)^2))
 * The cutoff test of Sec. 3 (pack in-cutoff neighbours, skip skin atoms) runs
 * inside the force kernel on every evaluation.
 *
 * Units: Angstrom, eV, amu, ps (forces eV/A, velocities A/ps).  Boxes are
 * orthorhombic and periodic in x, y and z (minimum image); every side must be
 * at least 2 * (cutoff + skin), else TERSOFF_ERR_BOX_TOO_SMALL.
 *
 * Conventions for every call:
 *  - The caller owns every array it passes; the library copies inputs and
 *    writes results into caller buffers.  Opaque handles are freed only by
 *    their *_destroy call.
 *  - Array pointers are host pointers unless the call takes `flags` and
 *    TERSOFF_DEVICE_PTRS is set, in which case they are device pointers on the
 *    context's device (e.g. from torch.cuda), used in place.
 *  - Calls are synchronous with respect to the host unless stated otherwise:
 *    they return after their results are in the caller's buffers.
 *  - No exception crosses the ABI.  A negative return is an error; outputs are
 *    then unspecified and tersoff_last_error(ctx) holds a message.
 *  - Positions may lie outside the box (|x| < 1e6 box lengths); every distance
 *    is a minimum image.  They are stored as given, not wrapped.
 *  - Arrays of atoms are AoS: pos[N][3], forces[N][3], vel[N][3] (float64),
 *    types[N] (int32, in [0, ntypes)).
 */
#ifndef TERSOFF_H
#define TERSOFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define TERSOFF_OK 0
#define TERSOFF_ERR_ARG (-1)              /* bad argument (null pointer, N < 0, type out of range, ...) */
#define TERSOFF_ERR_NOMEM (-2)            /* device or host allocation failed / budget exceeded */
#define TERSOFF_ERR_CUDA (-3)             /* a CUDA runtime call failed */
#define TERSOFF_ERR_NLIST_OVERFLOW (-4)   /* neighbour list longer than its capacity */
#define TERSOFF_ERR_NONFINITE (-5)        /* NaN or Inf in energy or forces */
#define TERSOFF_ERR_TIMEOUT (-6)          /* a bounded wait ran out */
#define TERSOFF_ERR_BOX_TOO_SMALL (-7)    /* a box side < 2 * (cutoff + skin) */
#define TERSOFF_ERR_BUSY (-8)             /* server: no slot free and queue full */
#define TERSOFF_ERR_NOT_FOUND (-9)        /* server: unknown job id */

/* precision of the force evaluation (Sec. 4 of the paper compares single, double
 * and mixed modes; it does not define "mixed").  Integration is float64 in all
 * three.
 * TERSOFF_FP64: all arithmetic in float64.
 * TERSOFF_MIXED: relative vectors formed exactly from 32-bit fixed-point
 *   positions and converted to float32, as head + tail (r to ~1 ulp) for pairs in
 *   the cutoff taper or shorter than 0.7 R, rounded once for the others; lambda*r
 *   with lambda as head + tail; f_C, g, exp, pow and all per-term arithmetic in
 *   float32; the float32
 *   force contributions on each atom summed with compensation (TwoSum), so the sum
 *   has float64 accuracy; energy and virial summed over atoms in float64.
 * TERSOFF_SINGLE: the paper's single mode: float32 throughout the evaluation:
 *   relative vectors rounded once to float32, r from a float32 rsqrt, exp from one
 *   float32 exp2, float32 force sums per atom and float32 energy/virial sums per
 *   block of 128 atoms (only the sum over blocks is float64).  Cheapest, and
 *   the least accurate: see the tolerances the tests state. */
typedef enum { TERSOFF_FP64 = 0, TERSOFF_MIXED = 1, TERSOFF_SINGLE = 2 } tersoff_precision;

/* flags */
#define TERSOFF_HOST_PTRS 0
#define TERSOFF_DEVICE_PTRS 1     /* array arguments are device pointers */
/* There is no determinism flag: every force scatter is a reverse accumulation in
 * list order (no atomics), so results are run-to-run bitwise identical always. */

typedef struct tersoff_ctx tersoff_ctx;
typedef struct tersoff_params tersoff_params;
typedef struct tersoff_nlist tersoff_nlist;
typedef struct tersoff_md tersoff_md;
typedef struct tersoff_server tersoff_server;

/* ---- context ---------------------------------------------------------------
 * A context binds a CUDA device and a stream (NULL: the library creates its
 * own non-blocking stream).  `stream` is a cudaStream_t passed as void*; it
 * must outlive the context.  Not thread safe: one host thread per context. */
int tersoff_ctx_create(int device, void *stream, tersoff_ctx **out);
void tersoff_ctx_destroy(tersoff_ctx *ctx);
/* last error message of this context ("" if none); valid until the next call */
const char *tersoff_last_error(const tersoff_ctx *ctx);
/* library version string */
const char *tersoff_version(void);

/* ---- parameters ------------------------------------------------------------
 * entries: ntypes^3 rows of 14 float64 in the order
 *   {m, gamma, lambda3, c, d, h, n, beta, lambda2, B, R, D, lambda1, A}
 * row (ti,tj,tk) at index (ti*ntypes + tj)*ntypes + tk.  Two-body terms of the
 * pair (i,j) read row (ti,tj,tj); zeta(i,j,k) (Eq. 3) reads row (ti,tj,tk) for
 * gamma, lambda3, m, c, d, h and the cutoff R, D of f_C(r_ik), which must equal
 * those of row (ti,tk,tk) (true of Tersoff's combination rules; otherwise
 * TERSOFF_ERR_ARG).  m is 1 (Eq. 3 as printed) or 3 (exp((lambda3 dr)^3)).
 * masses_amu: ntypes masses (used by the MD calls).  1 <= ntypes <= 4.
 * The table is copied; the caller may free its buffers on return. */
int tersoff_params_create(tersoff_ctx *ctx, int ntypes, const double *entries, const double *masses_amu,
                          tersoff_params **out);
void tersoff_params_destroy(tersoff_params *p);
/* largest r_C = R + D in the table */
double tersoff_params_cutoff(const tersoff_params *p);

/* ---- neighbour list (Sec. 3: Verlet list with skin) ------------------------
 * Builds, on the GPU, for every atom i the list of j != i with minimum-image
 * distance < cutoff + skin (cell list with 27-cell stencil; all pairs when a
 * box side holds fewer than 3 cells).  Each list is sorted by j.  *inout is
 * created when NULL, else reused (its capacity grows as needed).  `cutoff` is
 * normally tersoff_params_cutoff(); `skin` >= 0. */
int tersoff_neighbor_build(tersoff_ctx *ctx, const double *pos, int64_t N, const double box[3], double cutoff,
                           double skin, int flags, tersoff_nlist **inout);
/* The same list with one radius per type pair: j is listed for i when the
 * minimum-image distance is < r_C(t_i, t_j) + skin, r_C = R + D of the table's
 * row (t_i, t_j, t_j) (the larger of the rows (a,b,b) and (b,a,a), so that the lists
 * stay symmetric).  This is the list tersoff_compute, the MD driver and the
 * server build internally.  Its pairs within r_C are those of the one-radius
 * list with cutoff = tersoff_params_cutoff(); pairs of types with a shorter r_C
 * carry a shorter skin shell (in 3C-SiC the C-C second shell, 3.08 A, drops out of
 * the C lists).  The list is valid for `params` (or tables whose r_C are no
 * larger).  types: [N] in [0, ntypes). */
int tersoff_neighbor_build_typed(tersoff_ctx *ctx, const double *pos, const int32_t *types, int64_t N,
                                 const double box[3], const tersoff_params *params, double skin, int flags,
                                 tersoff_nlist **inout);
void tersoff_nlist_destroy(tersoff_nlist *nl);
/* copy a built list to host arrays: counts[N] and idx[N * (*stride)] (row i
 * at idx + i*stride, first counts[i] entries valid).  Call with idx == NULL to
 * read N and the stride only. */
int tersoff_nlist_get(tersoff_ctx *ctx, const tersoff_nlist *nl, int64_t *N, int32_t *stride, int32_t *counts,
                      int32_t *idx);

/* ---- one energy + force evaluation (Algorithm 1) ---------------------------
 * nl: a list built for these positions (or positions within skin/2 of them);
 * NULL builds one internally with skin 0.  energy: eV (may be NULL).
 * forces: [N][3] eV/A, overwritten (may be NULL).  virial: 6 float64
 * (xx, yy, zz, xy, xz, yz) = sum over terms of d_a F_b with d relative to atom
 * i, in eV (may be NULL).  Returns TERSOFF_ERR_NONFINITE if E or F is not
 * finite. */
int tersoff_compute(tersoff_ctx *ctx, const double *pos, const int32_t *types, int64_t N, const double box[3],
                    const tersoff_params *params, const tersoff_nlist *nl, tersoff_precision prec, int flags,
                    double *energy, double *forces, double *virial);

/* ---- velocity-Verlet NVE molecular dynamics --------------------------------
 * One step: v += dt/2 F/m; x += dt v; (rebuild the list on the GPU when some
 * atom moved more than skin/2 since the last build); F = F(x); v += dt/2 F/m.
 * Integration is float64 in both precisions.
 *
 * tersoff_md_create uploads the state, builds the list and evaluates F(x0).
 * tersoff_md_step advances nsteps steps; energy_trace (nullable, host,
 * [nsteps+1][2]) receives (potential, kinetic) energy in eV after each step,
 * row 0 = the state before the call.  tersoff_md_step_async only enqueues the
 * steps on the context's stream (no trace, no error check; follow with
 * tersoff_md_sync).  tersoff_md_get copies positions/velocities (and the forces of
 * the last evaluation) out (host or, with TERSOFF_DEVICE_PTRS, device buffers), in
 * the caller's atom order: a state with several atom types stores its atoms
 * grouped by type, in an order fixed by the types alone, so a state read out and
 * created again continues bitwise as the original would have. */
int tersoff_md_create(tersoff_ctx *ctx, const double *pos, const double *vel, const int32_t *types, int64_t N,
                      const double box[3], const tersoff_params *params, double dt_ps, double skin,
                      tersoff_precision prec, int flags, tersoff_md **out);
int tersoff_md_step(tersoff_md *md, int64_t nsteps, double *energy_trace);
int tersoff_md_step_async(tersoff_md *md, int64_t nsteps);
int tersoff_md_sync(tersoff_md *md);
int tersoff_md_get(tersoff_md *md, double *pos, double *vel, double *forces, int flags);
/* counters: steps done, list rebuilds, current list stride */
int tersoff_md_stats(tersoff_md *md, int64_t *steps, int64_t *rebuilds, int32_t *stride);
/* Per-phase device time.  With profiling on, every step enqueued afterwards is
 * bracketed phase by phase with CUDA events on the context's stream.
 * tersoff_md_profile(md, 1) starts (and resets) recording, (md, 0) stops it.
 * tersoff_md_profile_read waits for the stream and returns, summed over the
 * recorded steps, ms[5] = {integrator (force gather, kicks, drift), neighbour-
 * list build (launched every step, skipped on the device when no atom moved
 * skin/2), register force kernel, overflow force kernel and energy/virial
 * reduction, step bookkeeping} and launches[5] = kernel launches of each phase. */
int tersoff_md_profile(tersoff_md *md, int enable);
int tersoff_md_profile_read(tersoff_md *md, double ms[5], int64_t launches[5]);
void tersoff_md_destroy(tersoff_md *md);

/* one call: create, step nsteps, copy pos/vel back in place, destroy */
int tersoff_md_run(tersoff_ctx *ctx, double *pos, double *vel, const int32_t *types, int64_t N,
                   const double box[3], const tersoff_params *params, double dt_ps, int64_t nsteps, double skin,
                   tersoff_precision prec, int flags, double *energy_trace);

/* ---- evaluation without device allocation --------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that must
 * not allocate device memory while they run: a program whose framework allocator
 * has already reserved the device's memory (a cudaMalloc would fail or make it
 * give memory back), or a latency-critical loop where cudaMalloc/cudaFree would
 * synchronize the device.  It computes the same energy, forces and virial as
 * tersoff_compute with no list given (list built internally with skin 0) and calls
 * no cudaMalloc, cudaFree or other allocating routine: every working buffer lives
 * in one fixed device array of
 * TERSOFF_NOALLOC_SCRATCH_BYTES (about 22 MB) compiled into the library, which
 * every device that loads it holds until the process exits.
 *
 * Limits: N <= TERSOFF_NOALLOC_MAX_ATOMS, at most TERSOFF_NOALLOC_MAX_NEIGHBORS
 * atoms within the cutoff of any atom, cell grids coarsened to at most
 * TERSOFF_NOALLOC_MAX_CELLS cells.  A larger N returns TERSOFF_ERR_NOMEM before
 * any GPU work; a longer neighbour list returns TERSOFF_ERR_NLIST_OVERFLOW.
 *
 * params: created beforehand (tersoff_params_create allocates; do it at set-up)
 * on the device that is current at this call.  pos [N][3] float64 and types [N]
 * int32: DEVICE pointers.  box: host, 3 sides (A), each >= 2 * cutoff.
 * stream: cudaStream_t of the call (NULL: the default stream).
 * energy_virial: DEVICE [7] float64 (E in eV, then virial xx, yy, zz, xy, xz, yz
 * as in tersoff_compute) or NULL.  forces: DEVICE [N][3] float64 eV/A or NULL.
 * errbuf/errlen: optional host buffer for a message on failure.
 * The call returns after the stream has finished its work (it reads the device
 * status word).
 *
 * The first call on a device looks up the array's device address with that
 * device current and keeps it; make that first call before any stream capture.
 * The kept address belongs to the device's primary context: calls made after
 * that context was torn down (cudaDeviceReset) are not supported.
 * All calls on a device share the array and find the last call's contents in it;
 * each call clears what must start at zero.  Calls whose GPU work may overlap
 * (several host threads, or streams not ordered with each other) race on the
 * array: serialize them. */
#define TERSOFF_NOALLOC_MAX_ATOMS 16384
#define TERSOFF_NOALLOC_MAX_NEIGHBORS 32
#define TERSOFF_NOALLOC_MAX_CELLS 32768
#define TERSOFF_NOALLOC_SCRATCH_BYTES 23540480
int tersoff_compute_noalloc(const tersoff_params *params, const double *pos, const int32_t *types, int64_t N,
                            const double box[3], tersoff_precision prec, void *stream, double *energy_virial,
                            double *forces, char *errbuf, size_t errlen);

/* ---- serving: continuous batching of MD jobs ---------------------------------
 * A server runs many independent NVE jobs (periodic boxes of any size, each with
 * its own dt and step count) on one GPU.  Admitted jobs live in one packed
 * device layout (atoms, neighbour lists and cells of all jobs in contiguous
 * per-job ranges); every kernel of a step covers all of them in one launch, and
 * chunks of steps run as one CUDA graph launch.  A scheduler thread owned by the
 * server retires finished jobs and admits queued ones at chunk boundaries, as
 * slots and the device-memory budget allow (continuous batching): requests that
 * arrive while others run join the next chunk.  A job keeps its atom range for
 * its whole run: a new job goes into a free range and only its own list and
 * forces are computed on admission; the layout is compacted (resident jobs moved,
 * every list rebuilt) only when no free range holds a new job or freed atoms pass
 * 30% of the occupied range (environment TERSOFF_COMPACT_FREED=f sets that share).
 * A job with several atom types is stored grouped by type and each type is routed
 * to the register kernel its own first force evaluation calls for; results come
 * back in the caller's atom order.  A job's trajectory does not depend on the other
 * jobs in the batch or on where it sits (same arithmetic, same order, its own warps):
 * its result is bitwise the same alone and in any mix.
 *
 * params: shared by all jobs (job types index into it).  prec: precision of all
 * jobs.  skin: Verlet skin (A).  device_mem_budget: bytes the packed layout may
 * use; it fixes the largest number of resident atoms.  max_slots: largest number
 * of resident jobs (1..4096).  chunk_steps: steps between scheduling points.
 * The server uses the context's device with its own stream and thread and holds a
 * reference to the context.  The paper evaluates one system per process; the
 * packed layout applies the same per-atom work (Algorithm 1, Eqs. 1-3) to many
 * systems at once. */
typedef struct {
  int64_t n_atoms;
  const double *pos;     /* [n][3] A (host) */
  const double *vel;     /* [n][3] A/ps (host) */
  const int32_t *types;  /* [n] (host) */
  double box[3];         /* A */
  double dt_ps;
  int64_t nsteps;
} tersoff_job;

typedef struct {
  int64_t submitted, admitted, completed, failed, queued, running;
  int64_t atom_steps;    /* atom-steps of completed work */
  int64_t chunks, repacks;   /* chunks of steps run; admissions that placed new jobs */
  double busy_s;         /* wall time with jobs resident */
  int64_t capacity_atoms;
  /* scheduler wall time by activity (s): retiring finished jobs, admitting new
   * jobs (placement, their lists and first forces, compactions), capturing graphs,
   * running chunks of steps.  Handing results to retired jobs and staging the
   * next queued jobs run on the host while a chunk runs and count in run_s. */
  double retire_s, repack_s, graph_s, run_s;
  int64_t compactions;   /* admissions that moved resident jobs (layout compacted) */
  double layout_fill;    /* resident atoms / atoms the step kernels cover (freed ranges included), over chunks */
} tersoff_server_stats;

int tersoff_server_create(tersoff_ctx *ctx, const tersoff_params *params, tersoff_precision prec, double skin,
                          size_t device_mem_budget, int max_slots, int chunk_steps, tersoff_server **out);
/* Copies the job's inputs and queues it.  TERSOFF_ERR_NOMEM: the job can never
 * fit the budget; TERSOFF_ERR_ARG: bad job; TERSOFF_ERR_BOX_TOO_SMALL. */
int tersoff_server_submit(tersoff_server *s, const tersoff_job *job, uint64_t *job_id);
/* *done = 1 when the job finished (or failed). */
int tersoff_server_poll(tersoff_server *s, uint64_t job_id, int *done);
/* Blocks until the job finished; TERSOFF_ERR_TIMEOUT after timeout_s seconds. */
int tersoff_server_wait(tersoff_server *s, uint64_t job_id, double timeout_s);
/* Results of a finished job (any pointer may be NULL): final positions and
 * velocities [n][3], energy[2] = (potential, kinetic) eV, times[3] = seconds from
 * submission to admission, from admission to completion, and in total.  Releases
 * the job. */
int tersoff_server_result(tersoff_server *s, uint64_t job_id, double *pos, double *vel, double energy[2],
                          double times[3]);
int tersoff_server_get_stats(tersoff_server *s, tersoff_server_stats *out);
/* Why the last rejected submission or the last failed batch failed (valid until
 * the next call on this server). */
const char *tersoff_server_last_error(tersoff_server *s);
/* Stops the scheduler after the chunk of steps in flight; unfinished and queued
 * jobs are dropped. */
void tersoff_server_destroy(tersoff_server *s);

#ifdef __cplusplus
}
#endif
#endif /* TERSOFF_H */
