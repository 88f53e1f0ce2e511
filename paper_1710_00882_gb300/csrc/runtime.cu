// Host runtime and C ABI of libtersoff.so (declared in include/tersoff.h):
// contexts, parameter tables, neighbour lists, single evaluations and the
// velocity-Verlet MD driver.  Every step of the computation runs in the kernels
// of neighbor.cu, force.cu and integrate.cu; this file validates arguments,
// owns device buffers, enqueues launches and reads back status words.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tersoff.h"
#include "internal.cuh"
#include "runtime.h"

namespace tsf {

// ---------------------------------------------------------------------------
// device buffers

// ---------------------------------------------------------------------------
// geometry

Geom make_geom(const double box[3])
{
  Geom g;
  for (int a = 0; a < 3; ++a) {
    g.L[a] = box[a];
    g.invL[a] = 1.0 / box[a];
    g.to_q[a] = 4294967296.0 / box[a];
    g.q_to_d[a] = box[a] / 4294967296.0;
    g.q_to_f[a] = (float)(box[a] / 4294967296.0);
    g.q_to_f_lo[a] = (float)(box[a] / 4294967296.0 - (double)g.q_to_f[a]);
  }
  return g;
}

int make_grid(const double box[3], double rl, CellGrid *g)
{
  long long ncell = 1;
  for (int a = 0; a < 3; ++a) {
    int n = (int)std::floor(box[a] / (rl * (1.0 + 1e-6)));
    if (n < 1) n = 1;
    if (n > 1024) n = 1024;
    g->nc[a] = n;
    ncell *= n;
  }
  if (ncell > (1LL << 30)) return TERSOFF_ERR_ARG;
  g->ncell = (int)ncell;
  g->radii = uniform_radii(rl);
  return TERSOFF_OK;
}

// Squared list radius with the build's relative safety margin, rounded to float32.
static float list_rl2(double rl) { return (float)(rl * rl * (1.0 + 1e-5)); }

PairRadii uniform_radii(double rl)
{
  PairRadii r;
  for (int k = 0; k < MAX_TYPES * MAX_TYPES; ++k) r.rl2[k] = list_rl2(rl);
  return r;
}

// List radius per type pair: r_C(a,b) + skin, r_C = R + D of row (a,b,b) (the larger
// of rows (a,b,b) and (b,a,a), so that the table is symmetric whatever the rows
// hold).  A pair outside its radius at a build cannot come within r_C(a,b) before
// one of its atoms has moved skin/2, the rebuild criterion, as with one radius.
// Types the table does not have get the largest radius.
PairRadii pair_radii(const tersoff_params *P, double skin)
{
  PairRadii r = uniform_radii(P->rcmax + skin);
  const int nt = P->nt;
  auto rc = [&](int a, int b) {
    const double *row = &P->entries[(size_t)((a * nt + b) * nt + b) * NFIELDS];
    return row[F_R] + row[F_DD];
  };
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) r.rl2[a * MAX_TYPES + b] = list_rl2(std::max(rc(a, b), rc(b, a)) + skin);
  return r;
}

// one-entry system table: allocate device storage
bool sys_alloc(SysDev &S, int cap)
{
  if (S.tab && S.cap >= cap) return true;
  if (S.tab) cudaFree(S.tab);
  if (S.ctl) cudaFree(S.ctl);
  S.tab = nullptr;
  S.ctl = nullptr;
  S.cap = 0;
  if (cudaMalloc((void **)&S.tab, sizeof(SysTab) * cap) != cudaSuccess ||
      cudaMalloc((void **)&S.ctl, sizeof(SysCtl) * cap) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaMemset(S.ctl, 0, sizeof(SysCtl) * cap);
  S.cap = cap;
  return true;
}

void sys_free(SysDev &S)
{
  if (S.tab) cudaFree(S.tab);
  if (S.ctl) cudaFree(S.ctl);
  S = SysDev();
}

}  // namespace tsf

using namespace tsf;

// ---------------------------------------------------------------------------
// context

struct tersoff_nlist {
  tersoff_ctx *ctx = nullptr;
  SysDev sys;
  AtomState atoms;    // positions the list was built from
  ListState list;
  RunState *rs = nullptr;
};

struct MdGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t start = nullptr;       // k_loop_start node (parameters set per launch)
  cudaGraphConditionalHandle hloop = 0;
  bool valid = false;
};

// profiled phases: integrator, list build, register force kernel, overflow force
// kernel + reductions, step bookkeeping
constexpr int TSF_PHASES = 5;

struct tersoff_md {
  tersoff_ctx *ctx = nullptr;
  cudaStream_t cap_stream = nullptr;   // stream used only to capture the step graphs
  MdGraph graph[3];                    // step loop without / with energy trace; one step without trace
  bool use_graphs = true;
  bool pending = false;                // async steps launched and not yet checked
  const tersoff_params *params = nullptr;
  AtomState atoms;
  ListState list;
  SysDev sys;
  RunState *rs = nullptr;
  double *d_trace = nullptr;
  size_t trace_cap = 0;
  double dt = 0, skin = 0;
  int prec = TERSOFF_FP64;
  int gprec = TERSOFF_FP64;   // accumulation of the force gather (PREC_MIXED_ACC64: float64 sums)
  bool f32 = false;     // float32 force arithmetic (mixed or single precision)
  bool fused_lists = true;   // list builds sort and find reverse indices in one kernel (lists <= 16 slots)
  bool open = false;            // velocities are at the half step (a closing kick is pending)
  bool pe_valid = false;        // rs->epot_last holds the potential energy of the current positions
  long long steps_done = 0;     // host count of completed steps
  long long steps_target = 0;   // host count of enqueued steps
  int fast_slots = 8;   // register force kernel slots (4 or 8; 0 = general kernel only)
  int gen_slots = 8;    // general force kernel slots
  bool routed = false;  // register kernel split by atom type into a 4-slot and an 8-slot launch
  ForceRoutes routes{};
  int *d_order = nullptr;
  int *perm = nullptr;   // [N] caller index of each atom (atoms grouped by type), or null: caller order
  // phase profiling: event pairs per phase, reused across reads
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, std::pair<size_t, size_t>>> ev_marks;  // (phase, (start idx, end idx))
  long long launches[TSF_PHASES] = {0, 0, 0, 0, 0};
};

namespace tsf {

int set_err(tersoff_ctx *ctx, int code, const char *fmt, ...)
{
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int cuda_err(tersoff_ctx *ctx, cudaError_t e, const char *what)
{
  return set_err(ctx, TERSOFF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                        \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call);             \
  } while (0)

#define CKR(call)                                                       \
  do {                                                                  \
    int r_ = (call);                                                    \
    if (r_ != TERSOFF_OK) return r_;                                    \
  } while (0)

int status_to_code(tersoff_ctx *ctx, int st, const RunState &h)
{
  if (st & ST_BAD_TYPE) return set_err(ctx, TERSOFF_ERR_ARG, "atom type out of range");
  if (st & ST_NONFINITE) return set_err(ctx, TERSOFF_ERR_NONFINITE, "non-finite force or energy");
  if (st & ST_REV_MISSING) return set_err(ctx, TERSOFF_ERR_NLIST_OVERFLOW, "neighbour list not symmetric");
  if (st & ST_NLIST_OVERFLOW)
    return set_err(ctx, TERSOFF_ERR_NLIST_OVERFLOW, "neighbour list overflow (%d entries)", h.maxcount);
  if (st & ST_NC_OVERFLOW)
    return set_err(ctx, TERSOFF_ERR_NLIST_OVERFLOW, "too many in-cutoff neighbours (%d)", h.maxnc);
  return set_err(ctx, TERSOFF_ERR_CUDA, "device status %d", st);
}

int read_rs(tersoff_ctx *ctx, RunState *rs, RunState *h)
{
  CK(cudaMemcpyAsync(h, rs, sizeof(RunState), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return TERSOFF_OK;
}

int new_rs(tersoff_ctx *ctx, RunState **rs)
{
  void *p = nullptr;
  if (cudaMalloc(&p, sizeof(RunState)) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, TERSOFF_ERR_NOMEM, "cannot allocate run state");
  }
  CK(cudaMemsetAsync(p, 0, sizeof(RunState), ctx->stream));
  *rs = (RunState *)p;
  return TERSOFF_OK;
}

void free_atoms(AtomState &A)
{
  dfree(A.x); dfree(A.v); dfree(A.q);
  dfree(A.contrib); dfree(A.selfF); dfree(A.mask);
  dfree(A.work); dfree(A.nwork); dfree(A.partial); dfree(A.kepart);
  A = AtomState();
}

void free_list(ListState &L)
{
  dfree(L.nbr); dfree(L.rev); dfree(L.cnt); dfree(L.qref);
  dfree(L.cell_count); dfree(L.cell_start); dfree(L.tile_sums);
  dfree(L.cell_atoms); dfree(L.cell_of); dfree(L.rank);
  L = ListState();
}

int ensure_atoms(tersoff_ctx *ctx, AtomState &A, int64_t N, bool need_v)
{
  size_t n = (size_t)std::max<int64_t>(N, 1);
  if (!dreserve(A.x, A.x_b, n * sizeof(dbl4)) || !dreserve(A.q, A.q_b, n * sizeof(int4)) ||
      (need_v && !dreserve(A.v, A.v_b, n * sizeof(dbl4))))
    return set_err(ctx, TERSOFF_ERR_NOMEM, "cannot allocate atom arrays for N=%lld", (long long)N);
  A.N = N;
  return TERSOFF_OK;
}

int ensure_scatter(tersoff_ctx *ctx, AtomState &A, int64_t N, int cap, bool f32)
{
  size_t v4 = f32 ? sizeof(float4) : sizeof(dbl4);
  size_t n = (size_t)std::max<int64_t>(N, 1);
  const size_t nfast = (size_t)force_queue_blocks((int)n);
  if (!dreserve(A.contrib, A.contrib_b, n * (size_t)cap * v4) || !dreserve(A.selfF, A.selfF_b, n * v4) ||
      !dreserve(A.mask, A.mask_b, n * sizeof(unsigned long long)) ||
      !dreserve(A.work, A.work_b, nfast * 128 * sizeof(int)) || !dreserve(A.nwork, A.nwork_b, nfast * sizeof(int)) ||
      !dreserve(A.partial, A.partial_b, (size_t)force_partial_rows((int)n) * 8 * sizeof(double)) ||
      !dreserve(A.kepart, A.kepart_b, (size_t)vv_blocks((int)n) * sizeof(double)))
    return set_err(ctx, TERSOFF_ERR_NOMEM, "cannot allocate force scatter buffers (N=%lld, cap=%d)", (long long)N,
                   cap);
  return TERSOFF_OK;
}

int ensure_list(tersoff_ctx *ctx, ListState &L, int64_t N, int cap, int ncell)
{
  size_t n = (size_t)std::max<int64_t>(N, 1);
  if (N > MAX_LIST_ATOMS)
    return set_err(ctx, TERSOFF_ERR_NOMEM, "N=%lld exceeds %lld atoms per neighbour list", (long long)N,
                   (long long)MAX_LIST_ATOMS);
  // list slots are addressed by 32-bit flat indices (slot * N + atom)
  if (n * (size_t)cap > 0xffffffffull)
    return set_err(ctx, TERSOFF_ERR_NOMEM, "N=%lld x %d list slots exceeds 2^32 entries", (long long)N, cap);
  bool ok = dreserve(L.nbr, L.nbr_b, n * cap * sizeof(int)) &&
            dreserve(L.rev, L.rev_b, n * cap * sizeof(int)) &&
            dreserve(L.cnt, L.cnt_b, n * sizeof(int)) &&
            dreserve(L.qref, L.qref_b, n * sizeof(int4)) &&
            dreserve(L.cell_atoms, L.cell_atoms_b, n * sizeof(int4)) &&
            dreserve(L.cell_of, L.cell_of_b, n * sizeof(int)) &&
            dreserve(L.rank, L.rank_b, n * sizeof(int)) &&
            dreserve(L.cell_start, L.cell_start_b, ((size_t)ncell + 1) * sizeof(int)) &&
            dreserve(L.tile_sums, L.tile_sums_b, (size_t)scan_tiles_for(ncell) * sizeof(int) + 16);
  if (ok && (size_t)ncell * sizeof(int) > L.cell_count_b) {
    ok = dreserve(L.cell_count, L.cell_count_b, (size_t)ncell * sizeof(int));
    if (ok) CK(cudaMemsetAsync(L.cell_count, 0, L.cell_count_b, ctx->stream));
  }
  if (!ok) return set_err(ctx, TERSOFF_ERR_NOMEM, "cannot allocate neighbour list (N=%lld, cap=%d)", (long long)N, cap);
  L.N = N;
  L.cap = cap;
  return TERSOFF_OK;
}

int check_box(tersoff_ctx *ctx, const double box[3], double rl)
{
  for (int a = 0; a < 3; ++a) {
    if (!(box[a] > 0) || !std::isfinite(box[a])) return set_err(ctx, TERSOFF_ERR_ARG, "box side %d not positive", a);
    if (box[a] < 2.0 * rl)
      return set_err(ctx, TERSOFF_ERR_BOX_TOO_SMALL, "box side %d = %g < 2*(cutoff+skin) = %g", a, box[a], 2 * rl);
  }
  return TERSOFF_OK;
}

// Host-visible list build from A.q: the first capacity from the mean density, grown
// on overflow to the longest list plus headroom.
int build_list_sync(tersoff_ctx *ctx, const AtomState &A, ListState &L, RunState *rs, const double box[3],
                    double cutoff, double skin, SysDev &S, const tersoff_params *P)
{
  const double rl = cutoff + skin;
  CKR(check_box(ctx, box, rl));
  CellGrid g;
  if (make_grid(box, rl, &g) != TERSOFF_OK) return set_err(ctx, TERSOFF_ERR_ARG, "cell grid too large");
  if (P) g.radii = pair_radii(P, skin);
  L.grid = g;
  L.geo = make_geom(box);
  L.cutoff = cutoff;
  L.skin = skin;
  // system 0 of the table: geometry and cell grid
  S.host.geo = L.geo;
  for (int a = 0; a < 3; ++a) S.host.nc[a] = g.nc[a];
  S.host.cell_off = 0;
  S.host.atom_off = 0;
  S.host.natoms = (int)A.N;
  CK(cudaMemcpyAsync(S.tab, &S.host, sizeof(SysTab), cudaMemcpyHostToDevice, ctx->stream));
  int cap = L.cap;
  if (cap <= 0) {
    // first build: room for the mean number of atoms within the list radius plus 4 (at
    // least 8, a multiple of 4); a list that overflows it makes the next attempt size
    // the capacity from the longest list found
    const double nexp = (double)A.N / (box[0] * box[1] * box[2]) * (4.0 / 3.0) * M_PI * rl * rl * rl;
    cap = (int)std::min<double>(MAX_CAP, std::ceil(nexp + 4.0));
    cap = std::min(MAX_CAP, std::max(8, (cap + 3) & ~3));
  }
  for (int attempt = 0; attempt < 3; ++attempt) {
    CKR(ensure_list(ctx, L, A.N, cap, g.ncell));
    CK(cudaMemsetAsync(&rs->maxcount, 0, sizeof(int), ctx->stream));
    CK(launch_build(ctx->stream, (int)A.N, (int)A.N, A.q, S.tab, nullptr, g.ncell, g.radii, L.cell_count, L.cell_start, L.tile_sums,
                    L.cell_atoms, L.cell_of, L.rank, L.nbr, L.rev, L.cnt, cap, L.qref, rs, 0));
    RunState h;
    CKR(read_rs(ctx, rs, &h));
    L.maxcount = h.maxcount;
    if (h.status == 0) {
      // shrink an oversized first allocation (contrib buffers scale with the capacity)
      int want = std::min(MAX_CAP, h.maxcount + std::max(4, h.maxcount / 4));
      want = (want + 3) & ~3;
      if (want < cap && cap == MAX_CAP && attempt == 0) {
        cap = want;
        free_list(L);
        L.grid = g; L.geo = make_geom(box); L.cutoff = cutoff; L.skin = skin;
        continue;
      }
      return TERSOFF_OK;
    }
    if (h.status != ST_NLIST_OVERFLOW) return status_to_code(ctx, h.status, h);
    if (h.maxcount > MAX_CAP)
      return set_err(ctx, TERSOFF_ERR_NLIST_OVERFLOW, "%d neighbours within cutoff+skin exceed the limit %d",
                     h.maxcount, MAX_CAP);
    cap = std::min(MAX_CAP, ((h.maxcount + std::max(4, h.maxcount / 4)) + 3) & ~3);
    CK(cudaMemsetAsync(&rs->status, 0, sizeof(int), ctx->stream));
  }
  return set_err(ctx, TERSOFF_ERR_NLIST_OVERFLOW, "neighbour list build did not converge");
}

// Copy AoS positions (+ types) into the device state; host or device pointers.
int ingest(tersoff_ctx *ctx, AtomState &A, const double *pos, const int32_t *types, int64_t N, int nt,
           const double box[3], bool dev, RunState *rs, SysDev &S)
{
  A.geo = make_geom(box);
  if (!sys_alloc(S, 1)) return set_err(ctx, TERSOFF_ERR_NOMEM, "system table");
  S.host.geo = A.geo;
  S.host.atom_off = 0;
  S.host.natoms = (int)N;
  CK(cudaMemcpyAsync(S.tab, &S.host, sizeof(SysTab), cudaMemcpyHostToDevice, ctx->stream));
  if (N == 0) return TERSOFF_OK;
  const double *dpos = pos;
  const int *dtyp = types;
  if (!dev) {
    size_t need = (size_t)N * (3 * sizeof(double) + sizeof(int));
    if (!dreserve(ctx->stage, ctx->stage_bytes, need)) return set_err(ctx, TERSOFF_ERR_NOMEM, "staging buffer");
    double *sp = (double *)ctx->stage;
    int *st = (int *)(sp + 3 * N);
    CK(cudaMemcpyAsync(sp, pos, (size_t)N * 3 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(st, types, (size_t)N * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    dpos = sp;
    dtyp = st;
  }
  CK(launch_ingest(ctx->stream, (int)N, dpos, dtyp, nt, 0, S.tab, A.x, A.q, rs));
  return TERSOFF_OK;
}

int check_common(tersoff_ctx *ctx, const double *pos, int64_t N, const double box[3])
{
  if (!ctx) return TERSOFF_ERR_ARG;
  if (N < 0 || N > (int64_t)INT32_MAX / 16) return set_err(ctx, TERSOFF_ERR_ARG, "N=%lld out of range", (long long)N);
  if (N > 0 && !pos) return set_err(ctx, TERSOFF_ERR_ARG, "null positions");
  if (!box) return set_err(ctx, TERSOFF_ERR_ARG, "null box");
  return TERSOFF_OK;
}

static void ctx_free(tersoff_ctx *ctx)
{
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_atoms(ctx->cstate);
  sys_free(ctx->csys);
  free_list(ctx->clist);
  dfree(ctx->crs);
  dfree(ctx->stage);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

// Lists and MD states keep their context alive: destroying handles in any order is safe.
void ctx_release(tersoff_ctx *ctx)
{
  if (ctx && --ctx->refs == 0) ctx_free(ctx);
}

}  // namespace tsf

// ===========================================================================
// C ABI

extern "C" {

const char *tersoff_version(void) { return "tersoff-gb300 0.1 (sm_103a)"; }

int tersoff_ctx_create(int device, void *stream, tersoff_ctx **out)
{
  if (!out) return TERSOFF_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return TERSOFF_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return TERSOFF_ERR_CUDA;
  tersoff_ctx *ctx = new (std::nothrow) tersoff_ctx();
  if (!ctx) return TERSOFF_ERR_NOMEM;
  ctx->device = device;
  {
    const char *fk = getenv("TERSOFF_FORCE_KERNEL");
    ctx->general_only = fk && strcmp(fk, "general") == 0;
  }
  if (stream) {
    ctx->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return TERSOFF_ERR_CUDA;
    }
    ctx->own_stream = true;
  }
  if (new_rs(ctx, &ctx->crs) != TERSOFF_OK) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return TERSOFF_ERR_NOMEM;
  }
  *out = ctx;
  return TERSOFF_OK;
}

void tersoff_ctx_destroy(tersoff_ctx *ctx)
{
  if (!ctx || ctx->destroyed) return;
  ctx->destroyed = true;
  ctx_release(ctx);
}

const char *tersoff_last_error(const tersoff_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// ---------------------------------------------------------------------------

int tersoff_params_create(tersoff_ctx *ctx, int ntypes, const double *entries, const double *masses_amu,
                          tersoff_params **out)
{
  if (!ctx || !out) return TERSOFF_ERR_ARG;
  *out = nullptr;
  if (ntypes < 1 || ntypes > MAX_TYPES) return set_err(ctx, TERSOFF_ERR_ARG, "ntypes=%d not in [1,%d]", ntypes, MAX_TYPES);
  if (!entries || !masses_amu) return set_err(ctx, TERSOFF_ERR_ARG, "null parameter table or masses");
  const int nt = ntypes, nrow = nt * nt * nt;
  auto row = [&](int a, int b, int c) { return entries + (size_t)((a * nt + b) * nt + c) * NFIELDS; };
  for (int r = 0; r < nrow; ++r)
    for (int f = 0; f < NFIELDS; ++f)
      if (!std::isfinite(entries[(size_t)r * NFIELDS + f])) return set_err(ctx, TERSOFF_ERR_ARG, "non-finite table entry");
  for (int a = 0; a < nt; ++a) {
    if (!(masses_amu[a] > 0)) return set_err(ctx, TERSOFF_ERR_ARG, "mass of type %d not positive", a);
    for (int b = 0; b < nt; ++b) {
      const double *p = row(a, b, b);
      if (!(p[F_DD] > 0) || !(p[F_R] > p[F_DD]))
        return set_err(ctx, TERSOFF_ERR_ARG, "row (%d,%d,%d): need R > D > 0", a, b, b);
      if (!(p[F_N] > 0) || !(p[F_BETA] >= 0))
        return set_err(ctx, TERSOFF_ERR_ARG, "row (%d,%d,%d): need n > 0, beta >= 0", a, b, b);
      const double *q = row(b, a, a);
      if (p[F_R] != q[F_R] || p[F_DD] != q[F_DD])
        return set_err(ctx, TERSOFF_ERR_ARG, "cutoff of pair (%d,%d) differs from (%d,%d)", a, b, b, a);
      for (int c = 0; c < nt; ++c) {
        const double *t = row(a, b, c), *u = row(a, c, c);
        if (t[F_R] != u[F_R] || t[F_DD] != u[F_DD])
          return set_err(ctx, TERSOFF_ERR_ARG, "row (%d,%d,%d): cutoff must equal that of row (%d,%d,%d)", a, b, c, a,
                         c, c);
        if (t[F_M] != 1.0 && t[F_M] != 3.0) return set_err(ctx, TERSOFF_ERR_ARG, "row (%d,%d,%d): m must be 1 or 3", a, b, c);
        if (!(t[F_D] != 0)) return set_err(ctx, TERSOFF_ERR_ARG, "row (%d,%d,%d): d must be nonzero", a, b, c);
      }
    }
  }
  tersoff_params *P = new (std::nothrow) tersoff_params();
  if (!P) return TERSOFF_ERR_NOMEM;
  P->nt = nt;
  P->entries.assign(entries, entries + (size_t)nrow * NFIELDS);
  // the register force kernel evaluates g(theta) once per unordered neighbour pair:
  // allowed when rows (i,j,k) and (i,k,j) carry the same angular constants
  P->sym_angular = true;
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b)
      for (int c = 0; c < nt; ++c) {
        const double *t1 = row(a, b, c), *t2 = row(a, c, b);
        for (int f : {F_M, F_GAMMA, F_LAM3, F_C, F_D, F_H})
          if (t1[f] != t2[f]) P->sym_angular = false;
      }
  for (int a = 0; a < nt; ++a) P->masses[a] = masses_amu[a];
  std::vector<PairP<float>> pf(nt * nt);
  std::vector<PairP<double>> pd(nt * nt);
  std::vector<TripP<float>> tf(nrow);
  std::vector<TripP<double>> td(nrow);
  const double PI = 3.14159265358979323846;
  const double LOG2E = 1.4426950408889634074;   // log2(e)
  const double LN2 = 0.69314718055994530942;    // ln(2)
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      const double *p = row(a, b, b);
      PairP<double> d;
      d.A = p[F_A]; d.lam1 = p[F_LAM1]; d.B = p[F_B]; d.lam2 = p[F_LAM2];
      d.lam1_lo = 0.0; d.lam2_lo = 0.0;
      d.beta = p[F_BETA]; d.n = p[F_N]; d.neg_inv2n = -1.0 / (2.0 * p[F_N]);
      d.Rc = p[F_R]; d.Dc = p[F_DD];
      d.r_in = p[F_R] - p[F_DD]; d.r_out = p[F_R] + p[F_DD]; d.rc2 = d.r_out * d.r_out;
      d.r_short = 0.7 * p[F_R];
      d.inv4D = 1.0 / (4.0 * p[F_DD]); d.dfc_scale = -PI / (4.0 * p[F_DD]); d.r_out_lo = 0.0;
      d.mu1h = d.lam1 * LOG2E; d.mu1l = 0.0; d.mu2h = d.lam2 * LOG2E; d.mu2l = 0.0;
      d.Aln2 = d.A * LN2; d.Bln2 = d.B * LN2;
      d.hlam1 = 0.5 * d.lam1; d.hlam2 = 0.5 * d.lam2;
      P->rcmax = std::max(P->rcmax, d.r_out);
      pd[a * nt + b] = d;
      PairP<float> f;
      f.A = (float)d.A; f.lam1 = (float)d.lam1; f.B = (float)d.B; f.lam2 = (float)d.lam2;
      f.lam1_lo = (float)(d.lam1 - (double)f.lam1);
      f.lam2_lo = (float)(d.lam2 - (double)f.lam2);
      f.beta = (float)d.beta; f.n = (float)d.n; f.neg_inv2n = (float)d.neg_inv2n;
      f.Rc = (float)d.Rc; f.Dc = (float)d.Dc; f.r_in = (float)d.r_in; f.r_out = (float)d.r_out;
      f.r_short = (float)d.r_short;
      // float cutoff test must not admit a pair the float64 test rejects: use the float below r_out^2
      f.rc2 = (float)d.rc2;
      if ((double)f.rc2 > d.rc2) f.rc2 = std::nextafter(f.rc2, 0.0f);
      f.inv4D = (float)d.inv4D; f.dfc_scale = (float)d.dfc_scale;
      f.r_out_lo = (float)(d.r_out - (double)f.r_out);
      // lambda log2(e) as float head + tail: the product is formed in float64, so the
      // pair lambda r log2(e) carries the rounding of r only
      f.mu1h = (float)d.mu1h; f.mu1l = (float)(d.mu1h - (double)f.mu1h);
      f.mu2h = (float)d.mu2h; f.mu2l = (float)(d.mu2h - (double)f.mu2h);
      f.Aln2 = (float)d.Aln2; f.Bln2 = (float)d.Bln2;
      f.hlam1 = (float)d.hlam1; f.hlam2 = (float)d.hlam2;
      pf[a * nt + b] = f;
      for (int c = 0; c < nt; ++c) {
        const double *t = row(a, b, c);
        TripP<double> e;
        e.gamma = t[F_GAMMA]; e.lam3 = t[F_LAM3];
        const double c2 = t[F_C] * t[F_C], d2 = t[F_D] * t[F_D];
        e.K = t[F_GAMMA] * c2 / d2; e.G2 = 2.0 * t[F_GAMMA] * c2; e.d2 = d2; e.h = t[F_H];
        e.m3 = t[F_M] == 3.0 ? 1.0 : 0.0; e.pad = 0;
        td[(a * nt + b) * nt + c] = e;
        TripP<float> g;
        g.gamma = (float)e.gamma; g.lam3 = (float)e.lam3; g.K = (float)e.K; g.G2 = (float)e.G2;
        g.d2 = (float)e.d2; g.h = (float)e.h; g.m3 = (float)e.m3; g.pad = 0;
        tf[(a * nt + b) * nt + c] = g;
      }
    }
  // the register kernel's kernel-argument table: one or two types whose rows all
  // have lambda3 = 0 (else the kernel reads the device table, kind 0)
  {
    bool lam3_zero = true;
    for (int r = 0; r < nrow; ++r) lam3_zero = lam3_zero && entries[(size_t)r * NFIELDS + F_LAM3] == 0.0;
    P->fast.kind = (lam3_zero && P->sym_angular && nt <= 2) ? nt : 0;
    // TERSOFF_FORCE_TABLE=generic: the register kernel reads the shared-memory table
    // for every table (the same terms; a measurement switch for the specialised kinds)
    const char *ft = getenv("TERSOFF_FORCE_TABLE");
    if (ft && strcmp(ft, "generic") == 0) P->fast.kind = 0;
    if (P->fast.kind > 0) {
      for (int k = 0; k < nt * nt; ++k) {
        P->fast.f.p[k] = pf[k];
        P->fast.d.p[k] = pd[k];
      }
      for (int k = 0; k < nrow; ++k) {
        P->fast.f.t[k] = tf[k];
        P->fast.d.t[k] = td[k];
      }
    }
  }
  bool ok = cudaMalloc(&P->pair_f, pf.size() * sizeof(pf[0])) == cudaSuccess &&
            cudaMalloc(&P->pair_d, pd.size() * sizeof(pd[0])) == cudaSuccess &&
            cudaMalloc(&P->trip_f, tf.size() * sizeof(tf[0])) == cudaSuccess &&
            cudaMalloc(&P->trip_d, td.size() * sizeof(td[0])) == cudaSuccess &&
            cudaMalloc((void **)&P->d_mass, MAX_TYPES * sizeof(double)) == cudaSuccess;
  if (ok)
    ok = cudaMemcpy(P->pair_f, pf.data(), pf.size() * sizeof(pf[0]), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(P->pair_d, pd.data(), pd.size() * sizeof(pd[0]), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(P->trip_f, tf.data(), tf.size() * sizeof(tf[0]), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(P->trip_d, td.data(), td.size() * sizeof(td[0]), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(P->d_mass, P->masses, MAX_TYPES * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    tersoff_params_destroy(P);
    return set_err(ctx, TERSOFF_ERR_NOMEM, "cannot upload parameter table");
  }
  *out = P;
  return TERSOFF_OK;
}

void tersoff_params_destroy(tersoff_params *P)
{
  if (!P) return;
  dfree(P->pair_f); dfree(P->pair_d); dfree(P->trip_f); dfree(P->trip_d); dfree(P->d_mass);
  delete P;
}

double tersoff_params_cutoff(const tersoff_params *P) { return P ? P->rcmax : 0.0; }

// ---------------------------------------------------------------------------

// Shared body of the two list builders: P null builds every pair within
// cutoff + skin (types ignored); P non-null builds per type pair within
// r_C(ti,tj) + skin of P's table (types required).
static int nlist_build(tersoff_ctx *ctx, const double *pos, const int32_t *types_in, int64_t N, const double box[3],
                       double cutoff, double skin, const tersoff_params *P, int flags, tersoff_nlist **inout)
{
  CKR(check_common(ctx, pos, N, box));
  if (!inout) return set_err(ctx, TERSOFF_ERR_ARG, "null list handle");
  if (!(cutoff > 0) || !(skin >= 0)) return set_err(ctx, TERSOFF_ERR_ARG, "need cutoff > 0, skin >= 0");
  cudaSetDevice(ctx->device);
  tersoff_nlist *nl = *inout;
  bool created = false;
  if (!nl) {
    nl = new (std::nothrow) tersoff_nlist();
    if (!nl) return TERSOFF_ERR_NOMEM;
    nl->ctx = ctx;
    ctx->refs += 1;
    if (new_rs(ctx, &nl->rs) != TERSOFF_OK) {
      tersoff_nlist_destroy(nl);
      return TERSOFF_ERR_NOMEM;
    }
    created = true;
  }
  int rc = TERSOFF_OK;
  CK(cudaMemsetAsync(nl->rs, 0, sizeof(RunState), ctx->stream));
  rc = ensure_atoms(ctx, nl->atoms, N, false);
  if (rc == TERSOFF_OK) rc = check_box(ctx, box, cutoff + skin);
  if (rc == TERSOFF_OK) {
    // without a table the types are irrelevant to the list: pass zeros through the ingest path
    std::vector<int32_t> zeros;
    const int32_t *types = types_in;
    void *dz = nullptr;
    if (!P && (flags & TERSOFF_DEVICE_PTRS)) {
      if (N > 0 && cudaMalloc(&dz, (size_t)N * sizeof(int)) != cudaSuccess) rc = set_err(ctx, TERSOFF_ERR_NOMEM, "types");
      else if (N > 0) cudaMemsetAsync(dz, 0, (size_t)N * sizeof(int), ctx->stream);
      types = (const int32_t *)dz;
    } else if (!P) {
      zeros.assign((size_t)N, 0);
      types = zeros.data();
    }
    if (rc == TERSOFF_OK)
      rc = ingest(ctx, nl->atoms, pos, types, N, P ? P->nt : 1, box, flags & TERSOFF_DEVICE_PTRS, nl->rs, nl->sys);
    if (rc == TERSOFF_OK) rc = build_list_sync(ctx, nl->atoms, nl->list, nl->rs, box, cutoff, skin, nl->sys, P);
    if (dz) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(dz);
    }
  }
  if (rc != TERSOFF_OK) {
    if (created) tersoff_nlist_destroy(nl);
    return rc;
  }
  *inout = nl;
  return TERSOFF_OK;
}

int tersoff_neighbor_build(tersoff_ctx *ctx, const double *pos, int64_t N, const double box[3], double cutoff,
                           double skin, int flags, tersoff_nlist **inout)
{
  return nlist_build(ctx, pos, nullptr, N, box, cutoff, skin, nullptr, flags, inout);
}

int tersoff_neighbor_build_typed(tersoff_ctx *ctx, const double *pos, const int32_t *types, int64_t N,
                                 const double box[3], const tersoff_params *params, double skin, int flags,
                                 tersoff_nlist **inout)
{
  if (!ctx) return TERSOFF_ERR_ARG;
  if (!params) return set_err(ctx, TERSOFF_ERR_ARG, "null parameters");
  if (N > 0 && !types) return set_err(ctx, TERSOFF_ERR_ARG, "null types");
  return nlist_build(ctx, pos, types, N, box, params->rcmax, skin, params, flags, inout);
}

void tersoff_nlist_destroy(tersoff_nlist *nl)
{
  if (!nl) return;
  if (nl->ctx) cudaStreamSynchronize(nl->ctx->stream);
  free_atoms(nl->atoms);
  sys_free(nl->sys);
  free_list(nl->list);
  dfree(nl->rs);
  ctx_release(nl->ctx);
  delete nl;
}

int tersoff_nlist_get(tersoff_ctx *ctx, const tersoff_nlist *nl, int64_t *N, int32_t *stride, int32_t *counts,
                      int32_t *idx)
{
  if (!ctx || !nl) return TERSOFF_ERR_ARG;
  const ListState &L = nl->list;
  if (N) *N = L.N;
  if (stride) *stride = L.cap;
  if (!idx && !counts) return TERSOFF_OK;
  std::vector<int> tmp((size_t)L.N * L.cap);
  std::vector<int> cnt((size_t)L.N);
  if (L.N > 0) {
    CK(cudaMemcpyAsync(cnt.data(), L.cnt, (size_t)L.N * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(tmp.data(), L.nbr, (size_t)L.N * L.cap * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  for (int64_t i = 0; i < L.N; ++i) {
    if (counts) counts[i] = cnt[i];
    if (idx)
      for (int s = 0; s < L.cap; ++s) idx[i * L.cap + s] = s < cnt[i] ? tmp[(size_t)s * L.N + i] : -1;
  }
  return TERSOFF_OK;
}

// ---------------------------------------------------------------------------

int tersoff_compute(tersoff_ctx *ctx, const double *pos, const int32_t *types, int64_t N, const double box[3],
                    const tersoff_params *P, const tersoff_nlist *nl, tersoff_precision prec, int flags,
                    double *energy, double *forces, double *virial)
{
  CKR(check_common(ctx, pos, N, box));
  if (!P) return set_err(ctx, TERSOFF_ERR_ARG, "null parameters");
  if (N > 0 && !types) return set_err(ctx, TERSOFF_ERR_ARG, "null types");
  if (prec != TERSOFF_FP64 && prec != TERSOFF_MIXED && prec != TERSOFF_SINGLE)
    return set_err(ctx, TERSOFF_ERR_ARG, "bad precision");
  if (nl && nl->list.N != N) return set_err(ctx, TERSOFF_ERR_ARG, "list built for %lld atoms, not %lld", (long long)nl->list.N, (long long)N);
  if (nl && nl->list.cutoff < P->rcmax) return set_err(ctx, TERSOFF_ERR_ARG, "list cutoff below the table's cutoff");
  cudaSetDevice(ctx->device);
  const bool f32 = prec != TERSOFF_FP64;
  const bool dev = flags & TERSOFF_DEVICE_PTRS;
  AtomState &A = ctx->cstate;
  RunState *rs = ctx->crs;
  CK(cudaMemsetAsync(rs, 0, sizeof(RunState), ctx->stream));
  CKR(ensure_atoms(ctx, A, N, false));
  CKR(check_box(ctx, box, P->rcmax));
  CKR(ingest(ctx, A, pos, types, N, P->nt, box, dev, rs, ctx->csys));
  const ListState *L = nl ? &nl->list : nullptr;
  if (!L) {
    CKR(build_list_sync(ctx, A, ctx->clist, rs, box, P->rcmax, 0.0, ctx->csys, P));
    L = &ctx->clist;
  } else {
    for (int a = 0; a < 3; ++a)
      if (nl->list.geo.L[a] != box[a]) return set_err(ctx, TERSOFF_ERR_ARG, "list built for another box");
  }
  CKR(ensure_scatter(ctx, A, N, L->cap, f32));
  const int gen_slots = force_slots_for(std::max(1, L->maxcount));
  const int fast_slots = (P->sym_angular && !ctx->general_only) ? (L->maxcount <= 4 ? 4 : 8) : 0;
  CK(launch_force(ctx->stream, prec, fast_slots, P->fast, gen_slots, 1, virial != nullptr, (int)N, A.x, A.q,
                  L->nbr, L->cnt, ctx->csys.tab, f32 ? P->pair_f : P->pair_d, f32 ? P->trip_f : P->trip_d, P->nt,
                  A.contrib, A.selfF, A.mask, A.work, A.nwork, A.partial, rs, nullptr));
  double *dF = nullptr;
  if (forces) {
    if (dev) {
      dF = forces;
    } else {
      size_t need = (size_t)std::max<int64_t>(N, 1) * 3 * sizeof(double);
      if (!dreserve(ctx->stage, ctx->stage_bytes, std::max(need, (size_t)N * (3 * sizeof(double) + sizeof(int)))))
        return set_err(ctx, TERSOFF_ERR_NOMEM, "staging buffer");
      dF = (double *)ctx->stage;
    }
    CK(launch_gather_out(ctx->stream, prec, (int)N, A.contrib, A.selfF, A.mask, L->rev, dF, rs));
  }
  RunState h;
  CKR(read_rs(ctx, rs, &h));
  if (h.status != 0) return status_to_code(ctx, h.status, h);
  if (!std::isfinite(h.epot)) return set_err(ctx, TERSOFF_ERR_NONFINITE, "non-finite energy");
  if (energy) *energy = h.epot;
  if (virial)
    for (int c = 0; c < 6; ++c) virial[c] = h.virial[c];
  if (forces && !dev && N > 0) {
    CK(cudaMemcpyAsync(forces, dF, (size_t)N * 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return TERSOFF_OK;
}

// ---------------------------------------------------------------------------
// MD

static cudaEvent_t md_event(tersoff_md *md)
{
  if (md->ev_used == md->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    md->ev_pool.push_back(e);
  }
  return md->ev_pool[md->ev_used++];
}

// Profiling only: a bounded busy wait of ~50 us on the device before a phase's start
// event, so that the host has enqueued the phase's launches before the device reaches
// the event; otherwise the host's launch latency would be counted as device time.
__global__ void k_profile_spin(long long cycles)
{
  const long long t0 = clock64();
  while (clock64() - t0 < cycles) {
  }
}

// bracket one phase with events when profiling; returns the start index
static size_t md_mark_begin(tersoff_md *md)
{
  if (!md->prof) return 0;
  k_profile_spin<<<1, 32, 0, md->ctx->stream>>>(100000);
  size_t i = md->ev_used;
  cudaEvent_t e = md_event(md);
  if (e) cudaEventRecord(e, md->ctx->stream);
  return i;
}

static void md_mark_end(tersoff_md *md, int phase, size_t begin, int nlaunch)
{
  md->launches[phase] += nlaunch;
  if (!md->prof) return;
  size_t i = md->ev_used;
  cudaEvent_t e = md_event(md);
  if (e) {
    cudaEventRecord(e, md->ctx->stream);
    md->ev_marks.push_back({phase, {begin, i}});
  }
}

// stats: record the largest in-cutoff counts (set-up and recovery; off in steps)
static int md_force(tersoff_md *md, cudaStream_t st, int eflag, int part = 3, int stats = 0)
{
  tersoff_ctx *ctx = md->ctx;
  const tersoff_params *P = md->params;
  CK(launch_force_part(part, st, md->prec, md->fast_slots, P->fast, md->gen_slots, eflag, 0, (int)md->atoms.N,
                       (int)md->atoms.N, md->atoms.x,
                  md->atoms.q, md->list.nbr, md->list.cnt, md->sys.tab, md->f32 ? P->pair_f : P->pair_d,
                  md->f32 ? P->trip_f : P->trip_d, P->nt, md->atoms.contrib, md->atoms.selfF, md->atoms.mask,
                  md->atoms.work, md->atoms.nwork, md->atoms.partial, md->rs, nullptr, md->routed ? &md->routes : nullptr, stats));
  return TERSOFF_OK;
}

// mode: VV_FINISH (1), VV_START (2), both (3), 0 (kinetic energy only) or -1 (from rs->open)
static int md_vv(tersoff_md *md, cudaStream_t st, int mode, bool ke)
{
  tersoff_ctx *ctx = md->ctx;
  const float lim = (float)(0.25 * md->skin * md->skin);
  CK(launch_vv(st, md->gprec, ke, (int)md->atoms.N, (int)md->atoms.N, mode, md->atoms.x, md->atoms.v, md->atoms.q, md->list.qref,
               md->atoms.contrib, md->atoms.selfF, md->atoms.mask, md->list.rev, md->sys.tab,
               md->sys.ctl, md->params->d_mass, lim, md->atoms.kepart, md->rs));
  return TERSOFF_OK;
}

// gated: skipped on the device unless some atom moved skin/2; full: every atom gets
// a new list (recovery), else only systems whose rebuild flag is set
static int md_build(tersoff_md *md, cudaStream_t st, int gated, bool full = false)
{
  tersoff_ctx *ctx = md->ctx;
  ListState &L = md->list;
  // Raw-list scratch: the force scatter buffers, which hold nothing between the
  // integrator's gather and the force evaluation that follows every build of an MD
  // state (one system: every atom gets a new list).
  const size_t n = (size_t)md->atoms.N;
  const bool scratch = md->fused_lists && md->atoms.contrib_b >= n * (size_t)L.cap * sizeof(int) &&
                       md->atoms.selfF_b >= n * sizeof(int);
  int *raw = scratch ? (int *)md->atoms.contrib : nullptr;
  int *rawcnt = scratch ? (int *)md->atoms.selfF : nullptr;
  CK(launch_build(st, (int)md->atoms.N, (int)md->atoms.N, md->atoms.q, md->sys.tab, full ? nullptr : md->sys.ctl, L.grid.ncell,
                  L.grid.radii, L.cell_count, L.cell_start, L.tile_sums, L.cell_atoms, L.cell_of, L.rank, L.nbr, L.rev,
                  L.cnt, L.cap, L.qref, md->rs, gated, raw, rawcnt));
  return TERSOFF_OK;
}

static void md_graphs_free(tersoff_md *md)
{
  for (auto &G : md->graph) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.g) cudaGraphDestroy(G.g);
    G = MdGraph();
  }
}

// Graph of the step loop (which = 1: with energy trace):
//   loop_start -> WHILE(steps_left > 0) { vv -> decide -> IF(rebuild) { list build } -> force -> step_end }
// loop_start takes the launch controls (steps, trace rows, open half kick), set per
// launch in the instantiated graph, and sets the first loop condition.
// step_end decrements steps_left and sets the loop condition, so one launch runs any
// number of steps, and a step without a rebuild launches no build kernel.
// which = 2: one step without trace, with no loop node (a conditional node costs
// microseconds of device-side scheduling per launch):
//   set_control -> vv -> list build (gated on the device) -> force -> step_end
// or, above kGatedBuildAtoms atoms,
//   set_control -> vv -> decide -> IF(rebuild) { list build } -> force -> step_end
static int md_graph_build(tersoff_md *md, int which)
{
  tersoff_ctx *ctx = md->ctx;
  const bool tr = which == 1;
  MdGraph &G = md->graph[which];
  cudaStream_t st = md->cap_stream;
  // kernels captured right behind another kernel become programmatic dependents
  pdl_scope pdl;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  G.g = g;
  if (which == 2) {
    // Up to kGatedBuildAtoms atoms the list-build kernels follow the integrator
    // unconditionally and exit at once on the device when no atom moved skin/2: eight
    // empty launches over grids of that size cost less than an IF node in a graph
    // launched for one step (Si 512k: 83.5 against 89.5 us per flushed step); over the
    // larger grids of a 3C-SiC 950k state they cost more (328 against 324 us).  In the
    // step loop the IF node is the cheaper of the two at both sizes.
    constexpr int64_t kGatedBuildAtoms = 750000;
    if (md->atoms.N <= kGatedBuildAtoms) {
      CK(cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, mode));
      CK(launch_set_control(st, md->rs, md->sys.ctl, 1, nullptr, 0, 0));
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t *deps = nullptr;
      size_t nd = 0;
      CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd));
      if (nd != 1) return set_err(ctx, TERSOFF_ERR_CUDA, "unexpected graph capture state");
      G.start = deps[0];
      CKR(md_vv(md, st, -1, false));
      CKR(md_build(md, st, 1));
      CKR(md_force(md, st, 0));
      CK(launch_step_end(st, md->rs, md->sys.ctl, 1, 0, 0));
      cudaGraph_t gc = g;
      CK(cudaStreamEndCapture(st, &gc));
      CK(cudaGraphInstantiate(&G.exec, g, 0));
      G.valid = true;
      return TERSOFF_OK;
    }
    cudaGraphConditionalHandle hbuild;
    CK(cudaGraphConditionalHandleCreate(&hbuild, g, 0, cudaGraphCondAssignDefault));
    CK(cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, mode));
    CK(launch_set_control(st, md->rs, md->sys.ctl, 1, nullptr, 0, 0));
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, &edges, &nd));
    if (nd != 1) return set_err(ctx, TERSOFF_ERR_CUDA, "unexpected graph capture state");
    G.start = deps[0];
    CKR(md_vv(md, st, -1, false));
    CK(launch_decide(st, md->rs, hbuild));
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, &edges, &nd));
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hbuild;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    CK(cudaGraphAddNode(&inode, g, deps, edges, nd, &ip));
    CK(cudaStreamUpdateCaptureDependencies(st, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
    CKR(md_force(md, st, 0));
    CK(launch_step_end(st, md->rs, md->sys.ctl, 1, 0, 0));
    cudaGraph_t gc = g;
    CK(cudaStreamEndCapture(st, &gc));
    cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(st, ifbody, nullptr, nullptr, 0, mode));
    CKR(md_build(md, st, 0));
    cudaGraph_t ifc = ifbody;
    CK(cudaStreamEndCapture(st, &ifc));
    CK(cudaGraphInstantiate(&G.exec, g, 0));
    G.valid = true;
    return TERSOFF_OK;
  }
  cudaGraphConditionalHandle hloop, hbuild;
  CK(cudaGraphConditionalHandleCreate(&hloop, g, 0, cudaGraphCondAssignDefault));
  CK(cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, mode));
  CK(launch_loop_start(st, md->rs, md->sys.ctl, 0, nullptr, 1, 0, hloop));
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *edges = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, &edges, &nd));
  if (nd != 1) return set_err(ctx, TERSOFF_ERR_CUDA, "unexpected graph capture state");
  G.start = deps[0];
  G.hloop = hloop;
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hloop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  CK(cudaGraphAddNode(&wnode, g, deps, edges, nd, &wp));
  CK(cudaStreamUpdateCaptureDependencies(st, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  CK(cudaStreamEndCapture(st, &g));
  cudaGraph_t body = wp.conditional.phGraph_out[0];

  CK(cudaGraphConditionalHandleCreate(&hbuild, body, 0, cudaGraphCondAssignDefault));
  CK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, mode));
  CKR(md_vv(md, st, -1, tr));
  CK(launch_decide(st, md->rs, hbuild));
  CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, &edges, &nd));
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hbuild;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t inode;
  CK(cudaGraphAddNode(&inode, body, deps, edges, nd, &ip));
  CK(cudaStreamUpdateCaptureDependencies(st, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
  CKR(md_force(md, st, tr ? 1 : 0));
  CK(launch_step_end(st, md->rs, md->sys.ctl, 1, hloop, 1));
  cudaGraph_t bodyc = body;
  CK(cudaStreamEndCapture(st, &bodyc));

  cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(st, ifbody, nullptr, nullptr, 0, mode));
  CKR(md_build(md, st, 0));
  cudaGraph_t ifc = ifbody;
  CK(cudaStreamEndCapture(st, &ifc));

  CK(cudaGraphInstantiate(&G.exec, g, 0));
  G.valid = true;
  return TERSOFF_OK;
}

// Enqueue n steps on the context stream: one graph launch, or, when profiling,
// kernel by kernel with events around each phase.  trace rows start at k0.
static int md_launch_steps(tersoff_md *md, long long n, double *d_trace, long long k0)
{
  tersoff_ctx *ctx = md->ctx;
  cudaStream_t st = ctx->stream;
  if (n <= 0) return TERSOFF_OK;
  const bool tr = d_trace != nullptr;
  if (!md->prof && md->use_graphs) {
    const int which = tr ? 1 : (n == 1 ? 2 : 0);
    MdGraph &G = md->graph[which];
    if (!G.valid) {
      int rc = md_graph_build(md, which);
      if (rc != TERSOFF_OK) {
        // fall back to kernel-by-kernel launches for this state
        cudaGetLastError();
        md_graphs_free(md);
        md->use_graphs = false;
      }
    }
    if (md->use_graphs) {
      // the launch's controls go into the graph's first node
      if (which == 2)
        CK(set_control_node(G.exec, G.start, md->rs, md->sys.ctl, 1, nullptr, k0, md->open ? 1 : 0));
      else
        CK(set_loop_start(G.exec, G.start, md->rs, md->sys.ctl, n, d_trace, k0, md->open ? 1 : 0, G.hloop));
      CK(cudaGraphLaunch(G.exec, st));
      md->launches[0] += n;
      md->open = true;
      return TERSOFF_OK;
    }
  }
  CK(launch_set_control(st, md->rs, md->sys.ctl, n, d_trace, k0, md->open ? 1 : 0));
  for (long long k = 0; k < n; ++k) {
    size_t b = md_mark_begin(md);
    CKR(md_vv(md, st, -1, tr));
    md_mark_end(md, 0, b, 1);
    b = md_mark_begin(md);
    CKR(md_build(md, st, 1));
    md_mark_end(md, 1, b, 8);
    b = md_mark_begin(md);
    CKR(md_force(md, st, tr ? 1 : 0, 1));
    md_mark_end(md, 2, b, md->fast_slots > 0 ? (md->routed ? md->routes.n : 1) : 0);
    b = md_mark_begin(md);
    CKR(md_force(md, st, tr ? 1 : 0, 2));
    md_mark_end(md, 3, b, 1 + (tr ? 1 : 0));
    b = md_mark_begin(md);
    CK(launch_step_end(st, md->rs, md->sys.ctl, 1, 0, 0));
    md_mark_end(md, 4, b, 1);
  }
  md->open = true;
  return TERSOFF_OK;
}

// Recover from a device status raised inside launched steps.  The failing step
// stopped after its drift (list overflow: in the build; slot overflow: in the force
// kernel): fix the cause, finish that step, then launch the rest.
static int md_recover(tersoff_md *md, const RunState &h, double *d_trace)
{
  tersoff_ctx *ctx = md->ctx;
  cudaStream_t st = ctx->stream;
  if (h.status & ST_NLIST_OVERFLOW) {
    if (h.maxcount > MAX_CAP)
      return set_err(ctx, TERSOFF_ERR_NLIST_OVERFLOW, "%d neighbours within cutoff+skin exceed the limit %d",
                     h.maxcount, MAX_CAP);
    int cap = std::min(MAX_CAP, ((h.maxcount + std::max(4, h.maxcount / 4)) + 3) & ~3);
    md_graphs_free(md);
    CKR(ensure_list(ctx, md->list, md->atoms.N, cap, md->list.grid.ncell));
    CKR(ensure_scatter(ctx, md->atoms, md->atoms.N, cap, md->f32));
    CK(cudaMemsetAsync(&md->rs->status, 0, sizeof(int), st));
    CKR(md_build(md, st, 0, true));
  } else if (h.status & ST_NC_OVERFLOW) {
    md_graphs_free(md);
    md->gen_slots = force_slots_for(h.maxnc);
    CK(cudaMemsetAsync(&md->rs->status, 0, sizeof(int), st));
  } else {
    return status_to_code(ctx, h.status, h);
  }
  CK(cudaMemsetAsync(&md->rs->epot, 0, sizeof(double), st));
  CKR(md_force(md, st, d_trace ? 1 : 0, 3, 1));
  CK(launch_step_end(st, md->rs, md->sys.ctl, 1, 0, 0));
  const long long rest = h.steps_left - 1;
  if (rest > 0) CKR(md_launch_steps(md, rest, d_trace, h.trace_k + 1));
  return TERSOFF_OK;
}

// Close the pending half kick (optional), wait, check status and recover if needed.
static int md_finish(tersoff_md *md, double *d_trace, bool close)
{
  tersoff_ctx *ctx = md->ctx;
  for (int attempt = 0; attempt < 8; ++attempt) {
    if (close && md->open) {
      CKR(md_vv(md, ctx->stream, 1, d_trace != nullptr));
      CK(launch_final(ctx->stream, md->rs, md->sys.ctl));
    }
    RunState h;
    CKR(read_rs(ctx, md->rs, &h));
    if (h.status == 0) {
      if (close) md->open = false;
      md->steps_done = h.step;
      md->steps_target = h.step;
      return TERSOFF_OK;
    }
    CKR(md_recover(md, h, d_trace));
  }
  return set_err(ctx, TERSOFF_ERR_NLIST_OVERFLOW, "MD recovery did not converge");
}

int tersoff_md_create(tersoff_ctx *ctx, const double *pos, const double *vel, const int32_t *types, int64_t N,
                      const double box[3], const tersoff_params *P, double dt_ps, double skin, tersoff_precision prec,
                      int flags, tersoff_md **out)
{
  CKR(check_common(ctx, pos, N, box));
  if (!out || !P || (N > 0 && (!vel || !types))) return set_err(ctx, TERSOFF_ERR_ARG, "null argument");
  if (!(dt_ps > 0) || !(skin >= 0)) return set_err(ctx, TERSOFF_ERR_ARG, "need dt > 0 and skin >= 0");
  if (prec != TERSOFF_FP64 && prec != TERSOFF_MIXED && prec != TERSOFF_SINGLE)
    return set_err(ctx, TERSOFF_ERR_ARG, "bad precision");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  tersoff_md *md = new (std::nothrow) tersoff_md();
  if (!md) return TERSOFF_ERR_NOMEM;
  md->ctx = ctx;
  ctx->refs += 1;
  md->params = P;
  md->dt = dt_ps;
  md->skin = skin;
  md->prec = prec;
  md->f32 = prec != TERSOFF_FP64;
  // TERSOFF_MIXED_ACCUMULATE=fp64: mixed-mode force contributions summed in float64
  // instead of the compensated float32 sum (the same forces to ~1e-16 relative; a
  // measurement switch for the accumulation reading)
  md->gprec = prec;
  {
    const char *acc = getenv("TERSOFF_MIXED_ACCUMULATE");
    if (prec == TERSOFF_MIXED && acc && strcmp(acc, "fp64") == 0) md->gprec = PREC_MIXED_ACC64;
    // TERSOFF_LIST_FUSED=0: the step's list builds sort the lists and search the
    // reverse indices in two kernels (the same lists and indices; a comparison switch)
    const char *fl = getenv("TERSOFF_LIST_FUSED");
    md->fused_lists = !(fl && strcmp(fl, "0") == 0);
  }
  auto fail = [&](int rc) {
    tersoff_md_destroy(md);
    return rc;
  };
  int rc = new_rs(ctx, &md->rs);
  if (rc != TERSOFF_OK) return fail(rc);
  if ((rc = ensure_atoms(ctx, md->atoms, N, true)) != TERSOFF_OK) return fail(rc);
  if ((rc = check_box(ctx, box, P->rcmax + skin)) != TERSOFF_OK) return fail(rc);
  if ((rc = ingest(ctx, md->atoms, pos, types, N, P->nt, box, flags & TERSOFF_DEVICE_PTRS, md->rs, md->sys)) !=
      TERSOFF_OK)
    return fail(rc);
  if (N > 0) {
    const double *dvel = vel;
    void *tmp = nullptr;
    if (!(flags & TERSOFF_DEVICE_PTRS)) {
      if (cudaMalloc(&tmp, (size_t)N * 3 * sizeof(double)) != cudaSuccess) return fail(set_err(ctx, TERSOFF_ERR_NOMEM, "vel"));
      cudaMemcpyAsync(tmp, vel, (size_t)N * 3 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
      dvel = (const double *)tmp;
    }
    cudaError_t e = launch_ingest_vel(ctx->stream, (int)N, dvel, md->atoms.v);
    cudaStreamSynchronize(ctx->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return fail(cuda_err(ctx, e, "ingest velocities"));
  }
  // Atoms grouped by type (stable; an order fixed by the types alone, so a state
  // copied out and created again gets the same one): the per-type register-kernel
  // launches then read whole rows of the per-atom arrays.  md_get scatters back to
  // the caller's order.
  if (N > 0 && P->nt > 1) {
    std::vector<int4> hq((size_t)N);
    if (cudaMemcpy(hq.data(), md->atoms.q, sizeof(int4) * N, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(set_err(ctx, TERSOFF_ERR_CUDA, "types for grouping"));
    std::vector<int> perm;
    perm.reserve((size_t)N);
    for (int t = 0; t < P->nt; ++t)
      for (int64_t i = 0; i < N; ++i)
        if (type_of(hq[i].w) == t) perm.push_back((int)i);
    bool identity = true;
    for (int64_t k = 0; k < N && identity; ++k) identity = perm[k] == (int)k;
    if (!identity) {
      void *tmp = nullptr;
      const size_t nb = (size_t)N * (2 * sizeof(dbl4) + sizeof(int4));
      if (cudaMalloc((void **)&md->perm, sizeof(int) * N) != cudaSuccess || cudaMalloc(&tmp, nb) != cudaSuccess) {
        if (tmp) cudaFree(tmp);
        cudaGetLastError();
        return fail(set_err(ctx, TERSOFF_ERR_NOMEM, "atom grouping"));
      }
      dbl4 *tx = (dbl4 *)tmp, *tv = tx + N;
      int4 *tq = (int4 *)(tv + N);
      cudaError_t e = cudaMemcpyAsync(md->perm, perm.data(), sizeof(int) * N, cudaMemcpyHostToDevice, ctx->stream);
      if (e == cudaSuccess)
        e = launch_permute_atoms(ctx->stream, (int)N, md->perm, md->atoms.x, md->atoms.v, md->atoms.q, tx, tv, tq);
      if (e == cudaSuccess) e = cudaMemcpyAsync(md->atoms.x, tx, sizeof(dbl4) * N, cudaMemcpyDeviceToDevice, ctx->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(md->atoms.v, tv, sizeof(dbl4) * N, cudaMemcpyDeviceToDevice, ctx->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(md->atoms.q, tq, sizeof(int4) * N, cudaMemcpyDeviceToDevice, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      cudaFree(tmp);
      if (e != cudaSuccess) return fail(cuda_err(ctx, e, "atom grouping"));
    }
  }
  md->sys.host.dt = dt_ps;
  for (int a = 0; a < MAX_TYPES; ++a) md->sys.host.kick[a] = a < P->nt ? 0.5 * dt_ps * ACCEL / P->masses[a] : 0.0;
  if ((rc = build_list_sync(ctx, md->atoms, md->list, md->rs, box, P->rcmax, skin, md->sys, P)) != TERSOFF_OK)
    return fail(rc);
  if ((rc = ensure_scatter(ctx, md->atoms, N, md->list.cap, md->f32)) != TERSOFF_OK) return fail(rc);
  md->gen_slots = force_slots_for(std::max(1, md->list.maxcount));
  md->fast_slots = (P->sym_angular && !ctx->general_only) ? 8 : 0;
  if ((rc = md_force(md, ctx->stream, 1, 3, 1)) != TERSOFF_OK) return fail(rc);
  if (launch_force_done(ctx->stream, md->rs) != cudaSuccess) return fail(set_err(ctx, TERSOFF_ERR_CUDA, "force_done"));
  RunState h;
  if ((rc = read_rs(ctx, md->rs, &h)) != TERSOFF_OK) return fail(rc);
  if (h.status != 0) return fail(status_to_code(ctx, h.status, h));
  // register kernel with 4 slots when no atom has more than 4 in-cutoff neighbours
  // (diamond-like solids), else 8; atoms beyond that go to the warp kernel
  if (md->fast_slots > 0 && h.maxnc <= 4) md->fast_slots = 4;
  // several types with different neighbour counts (C atoms in SiC have 4, Si atoms up
  // to 8): one register-kernel launch per slot count over the atoms of those types, so
  // that the atoms of a warp share their loop trip counts
  if (md->fast_slots > 0 && P->nt > 1) {
    int slots_t[MAX_TYPES];
    bool differ = false;
    for (int t = 0; t < P->nt; ++t) {
      slots_t[t] = h.maxnc_t[t] <= 4 ? 4 : 8;
      differ = differ || slots_t[t] != slots_t[0];
    }
    if (differ) {
      std::vector<int4> hq((size_t)N);
      if (cudaMemcpy(hq.data(), md->atoms.q, sizeof(int4) * N, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(set_err(ctx, TERSOFF_ERR_CUDA, "types for routing"));
      std::vector<int> order;
      order.reserve((size_t)N);
      for (int pass = 4; pass <= 8; pass += 4)
        for (int64_t i = 0; i < N; ++i)
          if (slots_t[type_of(hq[i].w)] == pass) order.push_back((int)i);
      const int n4 = (int)std::count_if(hq.begin(), hq.end(), [&](const int4 &a) { return slots_t[type_of(a.w)] == 4; });
      // each launch over a contiguous range of atoms (atoms grouped by type) needs no
      // order array
      auto contiguous = [&](int b, int n) {
        for (int k = 1; k < n; ++k)
          if (order[b + k] != order[b] + k) return false;
        return true;
      };
      if (contiguous(0, n4) && contiguous(n4, (int)N - n4)) {
        md->routes.n = 2;
        md->routes.r[0] = ForceRoute{nullptr, n4 > 0 ? order[0] : 0, n4, 4, 0};
        md->routes.r[1] = ForceRoute{nullptr, n4 < N ? order[n4] : 0, (int)N - n4, 8, 0};
      } else {
        if (cudaMalloc((void **)&md->d_order, sizeof(int) * N) != cudaSuccess ||
            cudaMemcpy(md->d_order, order.data(), sizeof(int) * N, cudaMemcpyHostToDevice) != cudaSuccess)
          return fail(set_err(ctx, TERSOFF_ERR_NOMEM, "routing order"));
        md->routes.n = 2;
        md->routes.r[0] = ForceRoute{md->d_order, 0, n4, 4, 0};
        md->routes.r[1] = ForceRoute{md->d_order, n4, (int)N - n4, 8, 0};
      }
      md->routed = true;
    }
  }
  // the general kernel (the path without the register kernel) needs slots for
  // in-cutoff neighbours only (not the whole list): size it from the largest count
  // seen plus headroom; a later overflow widens it (recovery in md_finish)
  md->gen_slots = force_slots_for(std::max(8, h.maxnc + 2));
  md->steps_done = md->steps_target = 0;
  md->pe_valid = true;
  {
    const char *g = getenv("TERSOFF_GRAPHS");
    md->use_graphs = !(g && strcmp(g, "0") == 0);
  }
  if (cudaStreamCreateWithFlags(&md->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(set_err(ctx, TERSOFF_ERR_CUDA, "capture stream"));
  CK(cudaMemsetAsync(&md->rs->step, 0, sizeof(long long), ctx->stream));
  *out = md;
  return TERSOFF_OK;
}

int tersoff_md_step_async(tersoff_md *md, int64_t nsteps)
{
  if (!md || nsteps < 0) return TERSOFF_ERR_ARG;
  tersoff_ctx *ctx = md->ctx;
  cudaSetDevice(ctx->device);
  if (nsteps == 0) return TERSOFF_OK;
  CKR(md_launch_steps(md, nsteps, nullptr, 1));
  md->steps_target += nsteps;
  md->pending = true;
  md->pe_valid = false;
  return TERSOFF_OK;
}

int tersoff_md_sync(tersoff_md *md)
{
  if (!md) return TERSOFF_ERR_ARG;
  cudaSetDevice(md->ctx->device);
  md->pending = false;
  return md_finish(md, nullptr, true);
}

int tersoff_md_step(tersoff_md *md, int64_t nsteps, double *trace)
{
  if (!md || nsteps < 0) return TERSOFF_ERR_ARG;
  tersoff_ctx *ctx = md->ctx;
  cudaSetDevice(ctx->device);
  CKR(tersoff_md_sync(md));
  double *d_trace = nullptr;
  if (trace) {
    size_t need = (size_t)(nsteps + 1) * 2 * sizeof(double);
    if (!dreserve(md->d_trace, md->trace_cap, need)) return set_err(ctx, TERSOFF_ERR_NOMEM, "trace");
    d_trace = md->d_trace;
  }
  if (trace && !md->pe_valid) {
    // steps run without energy accumulation left no potential energy for the
    // current positions: evaluate it (the forces come out bitwise the same)
    CK(cudaMemsetAsync(&md->rs->epot, 0, sizeof(double), ctx->stream));
    CKR(md_force(md, ctx->stream, 1));
    CK(launch_force_done(ctx->stream, md->rs));
    md->pe_valid = true;
  }
  if (nsteps == 0) {
    if (!trace) return TERSOFF_OK;
    // no step: report the current state
    RunState h;
    CKR(md_vv(md, ctx->stream, 0, true));
    CKR(read_rs(ctx, md->rs, &h));
    trace[0] = h.epot_last;
    trace[1] = 0.5 * h.ekin2 / ACCEL;
    CK(cudaMemsetAsync(&md->rs->ekin2, 0, sizeof(double), ctx->stream));
    return TERSOFF_OK;
  }
  CKR(md_launch_steps(md, nsteps, d_trace, 1));
  md->steps_target += nsteps;
  CKR(md_finish(md, d_trace, true));
  md->pe_valid = trace != nullptr;
  if (trace) {
    CK(cudaMemcpyAsync(trace, d_trace, (size_t)(nsteps + 1) * 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return TERSOFF_OK;
}

int tersoff_md_get(tersoff_md *md, double *pos, double *vel, double *forces, int flags)
{
  if (!md) return TERSOFF_ERR_ARG;
  tersoff_ctx *ctx = md->ctx;
  cudaSetDevice(ctx->device);
  CKR(tersoff_md_sync(md));
  const int64_t N = md->atoms.N;
  if (N == 0) return TERSOFF_OK;
  const bool dev = flags & TERSOFF_DEVICE_PTRS;
  const size_t bytes = (size_t)N * 3 * sizeof(double);
  double *dp = nullptr, *dv = nullptr, *df = nullptr;
  void *tmp = nullptr;
  if (dev) {
    dp = pos; dv = vel; df = forces;
  } else {
    if (cudaMalloc(&tmp, 3 * bytes) != cudaSuccess) return set_err(ctx, TERSOFF_ERR_NOMEM, "staging");
    dp = pos ? (double *)tmp : nullptr;
    dv = vel ? (double *)tmp + 3 * N : nullptr;
    df = forces ? (double *)tmp + 6 * N : nullptr;
  }
  int rc = TERSOFF_OK;
  if (launch_extract(ctx->stream, (int)N, md->atoms.x, md->atoms.v, dp, dv, md->perm) != cudaSuccess)
    rc = TERSOFF_ERR_CUDA;
  if (rc == TERSOFF_OK && df &&
      launch_gather_out(ctx->stream, md->gprec, (int)N, md->atoms.contrib, md->atoms.selfF, md->atoms.mask,
                        md->list.rev, df, md->rs, md->perm) != cudaSuccess)
    rc = TERSOFF_ERR_CUDA;
  if (rc == TERSOFF_OK && !dev) {
    if (pos) cudaMemcpyAsync(pos, dp, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (vel) cudaMemcpyAsync(vel, dv, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (forces) cudaMemcpyAsync(forces, df, bytes, cudaMemcpyDeviceToHost, ctx->stream);
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = set_err(ctx, TERSOFF_ERR_CUDA, "md_get sync");
  if (tmp) cudaFree(tmp);
  return rc;
}

int tersoff_md_stats(tersoff_md *md, int64_t *steps, int64_t *rebuilds, int32_t *stride)
{
  if (!md) return TERSOFF_ERR_ARG;
  RunState h;
  CKR(read_rs(md->ctx, md->rs, &h));
  if (steps) *steps = h.step;
  if (rebuilds) *rebuilds = h.nrebuild;
  if (stride) *stride = md->list.cap;
  return TERSOFF_OK;
}

int tersoff_md_profile(tersoff_md *md, int enable)
{
  if (!md) return TERSOFF_ERR_ARG;
  tersoff_ctx *ctx = md->ctx;
  CK(cudaStreamSynchronize(ctx->stream));
  md->prof = enable != 0;
  md->ev_used = 0;
  md->ev_marks.clear();
  for (int p = 0; p < TSF_PHASES; ++p) md->launches[p] = 0;
  return TERSOFF_OK;
}

int tersoff_md_profile_read(tersoff_md *md, double ms[5], int64_t launches[5])
{
  if (!md) return TERSOFF_ERR_ARG;
  tersoff_ctx *ctx = md->ctx;
  CK(cudaStreamSynchronize(ctx->stream));
  double acc[TSF_PHASES] = {0, 0, 0, 0, 0};
  for (auto &m : md->ev_marks) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, md->ev_pool[m.second.first], md->ev_pool[m.second.second]));
    acc[m.first] += t;
  }
  for (int p = 0; p < TSF_PHASES; ++p) {
    if (ms) ms[p] = acc[p];
    if (launches) launches[p] = md->launches[p];
  }
  return TERSOFF_OK;
}

void tersoff_md_destroy(tersoff_md *md)
{
  if (!md) return;
  if (md->ctx) cudaStreamSynchronize(md->ctx->stream);
  md_graphs_free(md);
  if (md->cap_stream) cudaStreamDestroy(md->cap_stream);
  for (auto e : md->ev_pool) cudaEventDestroy(e);
  free_atoms(md->atoms);
  sys_free(md->sys);
  free_list(md->list);
  dfree(md->rs);
  dfree(md->d_trace);
  dfree(md->d_order);
  dfree(md->perm);
  ctx_release(md->ctx);
  delete md;
}

int tersoff_md_run(tersoff_ctx *ctx, double *pos, double *vel, const int32_t *types, int64_t N, const double box[3],
                   const tersoff_params *P, double dt_ps, int64_t nsteps, double skin, tersoff_precision prec,
                   int flags, double *energy_trace)
{
  tersoff_md *md = nullptr;
  CKR(tersoff_md_create(ctx, pos, vel, types, N, box, P, dt_ps, skin, prec, flags, &md));
  int rc = tersoff_md_step(md, nsteps, energy_trace);
  if (rc == TERSOFF_OK) rc = tersoff_md_get(md, pos, vel, nullptr, flags);
  tersoff_md_destroy(md);
  return rc;
}

}  // extern "C"
