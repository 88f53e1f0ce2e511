// Continuous-batching MD server (tersoff_server_* in include/tersoff.h).
//
// All admitted jobs live in one packed layout: atom arrays with a contiguous range
// per job, one cell numbering over all jobs' grids, one neighbour list over all
// atoms.  Every atom record carries its job's system index, and the kernels of a
// step (integrator, list build, force, bookkeeping) read that system's geometry,
// cell grid, time step and step control from per-system tables, so one launch per
// kernel covers the whole batch.  A chunk of steps is one CUDA graph launch:
//   WHILE(chunk steps left) { vv -> decide -> IF(rebuild) { build } -> force -> step_end }
// Jobs whose steps run out take their closing half kick in the next step and then
// stay frozen until the chunk ends.  Between chunks the scheduler thread retires
// finished jobs (results copied out), admits queued jobs that fit the slots and the
// atom capacity implied by the device-memory budget, and repacks the layout.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "runtime.h"

namespace tsf {

// index k of the range containing t among n ranges starting at off[0..n) (off ascending)
__device__ __forceinline__ int range_of(const int *__restrict__ off, int n, int t)
{
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Register-kernel routes of a layout: atom d of system k goes to position
// route_off[k] + (d - dst_off[k]) of the route order.
__global__ void k_route_order(int n, const int *__restrict__ dst_off, const int *__restrict__ route_off, int nsys,
                              int *__restrict__ order)
{
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const int k = range_of(dst_off, nsys, d);
  order[route_off[k] + (d - dst_off[k])] = d;
}

// Survivors of a repack: atom d of the new layout (systems 0..nsurv-1 come first)
// is atom src_off[k] + (d - atom_off[k]) of the old layout; its word gets the new
// system index.
__global__ void k_move(int n, const dbl4 *__restrict__ sx, const dbl4 *__restrict__ sv, const int4 *__restrict__ sq,
                       dbl4 *__restrict__ dx, dbl4 *__restrict__ dv, int4 *__restrict__ dq,
                       const int *__restrict__ dst_off, const int *__restrict__ src_off, int nsurv)
{
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const int k = range_of(dst_off, nsurv, d);
  const int src = src_off[k] + (d - dst_off[k]);
  dbl4 x = sx[src];
  int4 q = sq[src];
  const int w = make_w(type_of(q.w), k);
  q.w = w;
  x.w = __longlong_as_double((long long)w);
  dx[d] = x;
  dq[d] = q;
  dv[d] = sv[src];
}

// New jobs of a repack, staged back to back (pos [n][3], vel [n][3], types [n]):
// staged atom t belongs to new job k (staging offsets st_off), system sys0 + k.
__global__ void k_ingest_batch(int n, const double *__restrict__ pos, const double *__restrict__ vel,
                               const int *__restrict__ types, const int *__restrict__ st_off, int nnew, int sys0,
                               const SysTab *__restrict__ sys, int nt, dbl4 *__restrict__ x, dbl4 *__restrict__ v,
                               int4 *__restrict__ q, RunState *rs)
{
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int k = range_of(st_off, nnew, t);
  const int sid = sys0 + k;
  const SysTab &T = sys[sid];
  const int d = T.atom_off + (t - st_off[k]);
  int ty = types[t];
  if (ty < 0 || ty >= nt) {
    atomicOr(&rs->status, ST_BAD_TYPE);
    ty = 0;
  }
  double p[3];
  int qq[3];
  for (int a = 0; a < 3; ++a) {
    double c = pos[3 * (size_t)t + a];
    if (!isfinite(c) || fabs(c * T.geo.invL[a]) > 1e5) {
      atomicOr(&rs->status, ST_NONFINITE);
      c = 0.0;
    }
    p[a] = c;
    qq[a] = fixed_q(c, T.geo.to_q[a]);
  }
  const int w = make_w(ty, sid);
  x[d] = make_dbl4(p[0], p[1], p[2], __longlong_as_double((long long)w));
  q[d] = make_int4(qq[0], qq[1], qq[2], w);
  v[d] = make_dbl4(vel[3 * (size_t)t], vel[3 * (size_t)t + 1], vel[3 * (size_t)t + 2], 0.0);
}

// Finished jobs: staged atom t belongs to retiring job k (offsets r_off), system
// r_sys[k]; positions and velocities go out back to back as AoS float64.
__global__ void k_extract_batch(int n, const dbl4 *__restrict__ x, const dbl4 *__restrict__ v,
                                const int *__restrict__ r_off, const int *__restrict__ r_sys, int nret,
                                const SysTab *__restrict__ sys, double *__restrict__ pos, double *__restrict__ vel)
{
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int k = range_of(r_off, nret, t);
  const int d = sys[r_sys[k]].atom_off + (t - r_off[k]);
  const dbl4 a = x[d], b = v[d];
  pos[3 * (size_t)t] = a.x;
  pos[3 * (size_t)t + 1] = a.y;
  pos[3 * (size_t)t + 2] = a.z;
  vel[3 * (size_t)t] = b.x;
  vel[3 * (size_t)t + 1] = b.y;
  vel[3 * (size_t)t + 2] = b.z;
}

// Per-system potential and kinetic energy: one block per system, fixed-order sums.
__global__ void k_sys_energy(const double *__restrict__ eatom, const dbl4 *__restrict__ v, const int4 *__restrict__ q,
                             const double *__restrict__ mass, const SysTab *__restrict__ sys, double *__restrict__ out)
{
  __shared__ double sp[256], sk[256];
  const SysTab &T = sys[blockIdx.x];
  double pe = 0.0, ke = 0.0;
  for (int k = threadIdx.x; k < T.natoms; k += 256) {
    const int i = T.atom_off + k;
    pe += eatom[i];
    const dbl4 vi = v[i];
    ke += mass[type_of(q[i].w)] * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z);
  }
  sp[threadIdx.x] = pe;
  sk[threadIdx.x] = ke;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sp[threadIdx.x] += sp[threadIdx.x + w];
      sk[threadIdx.x] += sk[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = sp[0];
    out[2 * blockIdx.x + 1] = 0.5 * sk[0] / ACCEL;
  }
}

// Steps of the next chunk; after a failure the count is added to what is left.
__global__ void k_set_loop(RunState *rs, long long n)
{
  if (rs->status != 0) {
    rs->steps_left += n;
    return;
  }
  rs->steps_left = n;
  rs->trace = nullptr;
  rs->trace_k = 1;
}

}  // namespace tsf

using namespace tsf;

namespace {

double now_s()
{
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
  uint64_t id = 0;
  int64_t n = 0;
  std::vector<double> pos, vel;
  std::vector<int32_t> types;
  double box[3] = {0, 0, 0};
  double dt = 0;
  int64_t nsteps = 0;
  int state = 0;   // 0 queued, 1 running, 2 done, 3 failed
  int err = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  SysCtl ctl{};    // device step control at the last chunk boundary
  double epot = 0, ekin = 0;
  std::vector<double> rpos, rvel;
};

}  // namespace

struct tersoff_server {
  tersoff_ctx *ctx = nullptr;   // the caller's context (device, reference held)
  tersoff_ctx priv;             // private context on the scheduler's stream: helpers and errors of the worker
  const tersoff_params *P = nullptr;
  int prec = TERSOFF_FP64;
  bool f32 = false;             // float32 force arithmetic (mixed or single precision)
  double skin = 0, rl = 0;
  PairRadii radii{};            // list radius per type pair of the shared table
  int max_slots = 0, chunk = 0, listcap = 32;
  int64_t cap_atoms = 0;
  cudaStream_t st = nullptr, cap_st = nullptr;
  AtomState A[2];          // packed positions/velocities (x, v, q); repacks copy between the two
  int cur = 0;
  AtomState SC;            // force scatter buffers of the packed layout
  ListState L;
  SysDev S;
  RunState *rs = nullptr;
  double *eatom = nullptr, *sysE = nullptr;
  double *stage = nullptr;      // device staging (new jobs in, finished jobs out)
  size_t stage_b = 0;
  char *hstage = nullptr;       // pinned host staging
  size_t hstage_b = 0;
  int *dtabs = nullptr;         // device index tables of a repack / retire (4 x (max_slots + 1) ints)
  // register-kernel routes: atoms of one-species jobs (at most 4 in-cutoff
  // neighbours in the solids served) through the 4-slot kernel, the others through
  // the 8-slot kernel.  A job's route follows from its own atoms only, so its
  // arithmetic does not depend on the batch.
  ForceRoutes routes{};
  bool routed = false;
  int *d_order = nullptr;       // [capacity] atom order of the two routes
  std::vector<SysTab> tab;
  std::vector<Job *> batch;      // resident jobs in layout order (owned by `jobs`; touched by the worker only)
  int64_t natoms = 0;
  int ncell = 0;
  int fast_slots = 8, gen_slots = 32;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;
  cudaGraphNode_t start_node = nullptr;   // k_loop_start node (steps set per launch)
  cudaGraphConditionalHandle hloop = 0;
  bool use_graphs = true;   // TERSOFF_GRAPHS=0: chunks kernel by kernel (profiling)
  bool broken = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  tersoff_server_stats stats{};   // published under mu
  // worker-side counters, published into stats under mu once per loop
  int64_t w_chunks = 0, w_repacks = 0;
  double w_retire = 0, w_repack = 0, w_graph = 0, w_run = 0;
  std::string msg;              // last error reported to the caller (under mu)
};

namespace {

#define SK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return srv_err(s, TERSOFF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define SKR(call)                        \
  do {                                   \
    int r_ = (call);                     \
    if (r_ != TERSOFF_OK) return r_;     \
  } while (0)

int srv_err(tersoff_server *s, int code, const char *fmt, ...)
{
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  s->priv.err = buf;
  return code;
}

size_t bytes_per_atom(bool f32, int listcap)
{
  const size_t v4 = f32 ? 16 : 32;
  return 2 * (32 + 32 + 16)                        // two copies of x, v, q
         + (size_t)listcap * (v4 + 8)              // contrib + nbr/rev
         + v4 + 8 + 8 + 4 + 16 + 12 + 8 + 4 + 16;  // selfF, mask, work, cnt, qref, cells, eatom, route order, slack
}

// pinned host staging of at least `bytes` (contents not kept)
bool host_reserve(tersoff_server *s, size_t bytes)
{
  if (bytes <= s->hstage_b && s->hstage) return true;
  if (s->hstage) cudaFreeHost(s->hstage);
  s->hstage = nullptr;
  s->hstage_b = 0;
  bytes = std::max<size_t>(bytes + bytes / 4, 1 << 20);
  if (cudaHostAlloc((void **)&s->hstage, bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  s->hstage_b = bytes;
  return true;
}

int read_state(tersoff_server *s, RunState *h)
{
  SK(cudaMemcpyAsync(h, s->rs, sizeof(RunState), cudaMemcpyDeviceToHost, s->st));
  SK(cudaStreamSynchronize(s->st));
  return TERSOFF_OK;
}

AtomState &cur_atoms(tersoff_server *s) { return s->A[s->cur]; }

int srv_force(tersoff_server *s, cudaStream_t st)
{
  const tersoff_params *P = s->P;
  AtomState &X = cur_atoms(s);
  SK(launch_force_part(3, st, s->prec, s->fast_slots, P->fast, s->gen_slots, 0, 0, (int)s->natoms, X.x, X.q,
                       s->L.nbr, s->L.cnt, s->S.tab, s->f32 ? P->pair_f : P->pair_d,
                       s->f32 ? P->trip_f : P->trip_d, P->nt, s->SC.contrib, s->SC.selfF, s->SC.mask, s->SC.work,
                       s->SC.nwork, s->SC.partial, s->rs, s->eatom, s->routed ? &s->routes : nullptr, 0));
  return TERSOFF_OK;
}

int srv_vv(tersoff_server *s, cudaStream_t st)
{
  AtomState &X = cur_atoms(s);
  const float lim = (float)(0.25 * s->skin * s->skin);
  SK(launch_vv(st, s->prec, false, (int)s->natoms, -1, X.x, X.v, X.q, s->L.qref, s->SC.contrib, s->SC.selfF,
               s->SC.mask, s->L.rev, s->S.tab, s->S.ctl, s->P->d_mass, lim, s->SC.kepart, s->rs));
  return TERSOFF_OK;
}

// full: every atom gets a new list; else only systems whose rebuild flag is set
int srv_build(tersoff_server *s, cudaStream_t st, bool full)
{
  AtomState &X = cur_atoms(s);
  ListState &L = s->L;
  SK(launch_build(st, (int)s->natoms, X.q, s->S.tab, full ? nullptr : s->S.ctl, s->ncell, s->radii, L.cell_count, L.cell_start, L.tile_sums, L.cell_atoms,
                  L.cell_of, L.rank, L.nbr, L.rev, L.cnt, L.cap, L.qref, s->rs, 0));
  return TERSOFF_OK;
}

void graph_free(tersoff_server *s)
{
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->g) cudaGraphDestroy(s->g);
  s->exec = nullptr;
  s->g = nullptr;
  s->graph_ok = false;
}

// loop_start (launch controls, first condition) -> WHILE { vv -> decide -> IF(rebuild) { build } -> force -> step_end }
int graph_build(tersoff_server *s)
{
  graph_free(s);
  cudaStream_t st = s->cap_st;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  cudaGraph_t g = nullptr;
  SK(cudaGraphCreate(&g, 0));
  s->g = g;
  cudaGraphConditionalHandle hloop, hbuild;
  SK(cudaGraphConditionalHandleCreate(&hloop, g, 0, cudaGraphCondAssignDefault));
  SK(cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, mode));
  SK(launch_loop_start(st, s->rs, nullptr, 0, nullptr, 1, 0, hloop));
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *edges = nullptr;
  size_t nd = 0;
  SK(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, &edges, &nd));
  if (nd != 1) return srv_err(s, TERSOFF_ERR_CUDA, "unexpected graph capture state");
  s->start_node = deps[0];
  s->hloop = hloop;
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hloop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  SK(cudaGraphAddNode(&wnode, g, deps, edges, nd, &wp));
  SK(cudaStreamUpdateCaptureDependencies(st, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  SK(cudaStreamEndCapture(st, &g));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  SK(cudaGraphConditionalHandleCreate(&hbuild, body, 0, cudaGraphCondAssignDefault));
  SK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, mode));
  SKR(srv_vv(s, st));
  SK(launch_decide(st, s->rs, hbuild));
  SK(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, &edges, &nd));
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hbuild;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t inode;
  SK(cudaGraphAddNode(&inode, body, deps, edges, nd, &ip));
  SK(cudaStreamUpdateCaptureDependencies(st, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
  SKR(srv_force(s, st));
  SK(launch_step_end(st, s->rs, s->S.ctl, (int)s->batch.size(), hloop, 1));
  cudaGraph_t bodyc = body;
  SK(cudaStreamEndCapture(st, &bodyc));
  cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
  SK(cudaStreamBeginCaptureToGraph(st, ifbody, nullptr, nullptr, 0, mode));
  SKR(srv_build(s, st, false));
  cudaGraph_t ifc = ifbody;
  SK(cudaStreamEndCapture(st, &ifc));
  SK(cudaGraphInstantiate(&s->exec, g, 0));
  s->graph_ok = true;
  return TERSOFF_OK;
}

// Full list build and force evaluation of the current layout, growing the list
// capacity on overflow.
int build_and_force(tersoff_server *s)
{
  for (int attempt = 0; attempt < 3; ++attempt) {
    SK(cudaMemsetAsync(&s->rs->maxcount, 0, sizeof(int), s->st));
    SKR(srv_build(s, s->st, true));
    SKR(srv_force(s, s->st));
    RunState h;
    SKR(read_state(s, &h));
    if (h.status == 0) return TERSOFF_OK;
    if (h.status != ST_NLIST_OVERFLOW || h.maxcount > MAX_CAP)
      return srv_err(s, TERSOFF_ERR_NLIST_OVERFLOW, "list build or force failed (status %d, %d entries)", h.status,
                     h.maxcount);
    const int cap = std::min(MAX_CAP, ((h.maxcount + std::max(4, h.maxcount / 4)) + 3) & ~3);
    graph_free(s);
    if (ensure_list(&s->priv, s->L, s->cap_atoms, cap, std::max(1, s->ncell)) != TERSOFF_OK ||
        ensure_scatter(&s->priv, s->SC, s->cap_atoms, cap, s->f32) != TERSOFF_OK)
      return srv_err(s, TERSOFF_ERR_NOMEM, "cannot grow neighbour lists to %d entries", cap);
    s->listcap = cap;
    SK(cudaMemsetAsync(&s->rs->status, 0, sizeof(int), s->st));
  }
  return srv_err(s, TERSOFF_ERR_NLIST_OVERFLOW, "list build did not converge");
}

// Rebuild the packed layout from the jobs in `order` (survivors first, then new):
// survivors move with one kernel, new jobs are staged back to back and ingested
// with one copy and one kernel.
int repack(tersoff_server *s, const std::vector<Job *> &order, const std::vector<bool> &is_new)
{
  const tersoff_params *P = s->P;
  const int S = (int)order.size();
  std::vector<SysTab> tab(S);
  std::vector<SysCtl> ctl(S);
  std::map<const Job *, int> prev;
  for (size_t k = 0; k < s->batch.size(); ++k) prev[s->batch[k]] = s->tab[k].atom_off;
  // index tables: [0, S) new atom offsets, [S+1, ...) survivor source offsets, then
  // staging offsets of the new jobs
  std::vector<int> itab(4 * (size_t)(S + 1), 0);
  int *dst_off = itab.data(), *src_off = itab.data() + (S + 1), *st_off = itab.data() + 2 * (S + 1),
      *route_off = itab.data() + 3 * (S + 1);
  int64_t off = 0, staged = 0;
  int coff = 0, nsurv = 0, nnew = 0;
  for (int k = 0; k < S; ++k) {
    Job &J = *order[k];
    SysTab &T = tab[k];
    T.geo = make_geom(J.box);
    CellGrid gr;
    if (make_grid(J.box, s->rl, &gr) != TERSOFF_OK) return srv_err(s, TERSOFF_ERR_ARG, "cell grid too large");
    for (int a = 0; a < 3; ++a) T.nc[a] = gr.nc[a];
    T.cell_off = coff;
    T.atom_off = (int)off;
    T.natoms = (int)J.n;
    T.dt = J.dt;
    for (int a = 0; a < MAX_TYPES; ++a) T.kick[a] = a < P->nt ? 0.5 * J.dt * ACCEL / P->masses[a] : 0.0;
    ctl[k] = is_new[k] ? SysCtl{J.nsteps, 0, 0} : J.ctl;
    J.ctl = ctl[k];
    dst_off[k] = (int)off;
    if (!is_new[k]) {
      if (nnew > 0) return srv_err(s, TERSOFF_ERR_ARG, "survivors must precede new jobs");
      src_off[k] = prev[order[k]];
      ++nsurv;
    } else {
      st_off[nnew++] = (int)staged;
      staged += J.n;
    }
    off += J.n;
    coff += gr.ncell;
  }
  const int64_t surv_atoms = nsurv < S ? dst_off[nsurv] : off;
  // routes: one-species jobs first (4 slots), then the others (8 slots)
  int64_t n4 = 0;
  std::vector<char> one_species(S, 0);
  for (int k = 0; k < S; ++k) {
    const Job &J = *order[k];
    one_species[k] = std::all_of(J.types.begin(), J.types.end(), [&](int32_t t) { return t == J.types[0]; });
    if (one_species[k]) n4 += J.n;
  }
  {
    int64_t r4 = 0, r8 = n4;
    for (int k = 0; k < S; ++k) {
      route_off[k] = (int)(one_species[k] ? r4 : r8);
      (one_species[k] ? r4 : r8) += order[k]->n;
    }
  }
  s->routed = s->fast_slots > 0 && n4 > 0;
  if (s->routed) {
    s->routes.n = n4 < off ? 2 : 1;
    s->routes.r[0] = ForceRoute{n4 < off ? s->d_order : nullptr, 0, (int)n4, 4, 0};
    s->routes.r[1] = ForceRoute{s->d_order, (int)n4, (int)(off - n4), 8, 0};
  }
  s->natoms = off;
  s->ncell = coff;
  if (!sys_alloc(s->S, std::max(1, S))) return srv_err(s, TERSOFF_ERR_NOMEM, "system tables");
  if (ensure_list(&s->priv, s->L, s->cap_atoms, s->listcap, std::max(1, coff)) != TERSOFF_OK)
    return srv_err(s, TERSOFF_ERR_NOMEM, "cell arrays for %d cells", coff);
  // pinned staging: tables, then the new jobs' positions, velocities and types
  const size_t tbytes = sizeof(SysTab) * S + sizeof(SysCtl) * S + sizeof(int) * itab.size();
  const size_t tpad = (tbytes + 255) / 256 * 256;
  const size_t nbytes = (size_t)staged * (6 * sizeof(double) + sizeof(int32_t));
  if (!host_reserve(s, tpad + nbytes)) return srv_err(s, TERSOFF_ERR_NOMEM, "pinned staging");
  if (nbytes && !dreserve(s->stage, s->stage_b, nbytes)) return srv_err(s, TERSOFF_ERR_NOMEM, "staging");
  char *h = s->hstage;
  memcpy(h, tab.data(), sizeof(SysTab) * S);
  memcpy(h + sizeof(SysTab) * S, ctl.data(), sizeof(SysCtl) * S);
  memcpy(h + sizeof(SysTab) * S + sizeof(SysCtl) * S, itab.data(), sizeof(int) * itab.size());
  double *hpos = (double *)(h + tpad);
  double *hvel = hpos + 3 * staged;
  int32_t *hty = (int32_t *)(hvel + 3 * staged);
  for (int k = nsurv, m = 0; k < S; ++k, ++m) {
    const Job &J = *order[k];
    memcpy(hpos + 3 * (size_t)st_off[m], J.pos.data(), sizeof(double) * 3 * J.n);
    memcpy(hvel + 3 * (size_t)st_off[m], J.vel.data(), sizeof(double) * 3 * J.n);
    memcpy(hty + st_off[m], J.types.data(), sizeof(int32_t) * J.n);
  }
  SK(cudaMemcpyAsync(s->S.tab, h, sizeof(SysTab) * S, cudaMemcpyHostToDevice, s->st));
  SK(cudaMemcpyAsync(s->S.ctl, h + sizeof(SysTab) * S, sizeof(SysCtl) * S, cudaMemcpyHostToDevice, s->st));
  SK(cudaMemcpyAsync(s->dtabs, h + sizeof(SysTab) * S + sizeof(SysCtl) * S, sizeof(int) * itab.size(),
                     cudaMemcpyHostToDevice, s->st));
  AtomState &src = s->A[s->cur];
  AtomState &dst = s->A[1 - s->cur];
  const int *d_dst = s->dtabs, *d_src = s->dtabs + (S + 1), *d_st = s->dtabs + 2 * (S + 1);
  if (surv_atoms > 0) {
    k_move<<<(int)((surv_atoms + 255) / 256), 256, 0, s->st>>>((int)surv_atoms, src.x, src.v, src.q, dst.x, dst.v,
                                                                dst.q, d_dst, d_src, nsurv);
    SK(cudaGetLastError());
  }
  if (staged > 0) {
    double *dpos = s->stage, *dvel = dpos + 3 * staged;
    int *dty = (int *)(dvel + 3 * staged);
    SK(cudaMemcpyAsync(dpos, hpos, nbytes, cudaMemcpyHostToDevice, s->st));
    k_ingest_batch<<<(int)((staged + 255) / 256), 256, 0, s->st>>>((int)staged, dpos, dvel, dty, d_st, nnew, nsurv,
                                                                   s->S.tab, P->nt, dst.x, dst.v, dst.q, s->rs);
    SK(cudaGetLastError());
  }
  if (s->routed && s->routes.n == 2) {
    k_route_order<<<(int)((off + 255) / 256), 256, 0, s->st>>>((int)off, d_dst, s->dtabs + 3 * (S + 1), S,
                                                               s->d_order);
    SK(cudaGetLastError());
  }
  s->cur = 1 - s->cur;
  s->tab = tab;
  s->batch = order;
  graph_free(s);
  SKR(build_and_force(s));
  s->w_repacks += 1;
  return TERSOFF_OK;
}

// n steps: one graph launch, or kernel by kernel without graphs
int launch_steps(tersoff_server *s, long long n)
{
  if (s->use_graphs) {
    if (!s->graph_ok) {
      const double t0 = now_s();
      SKR(graph_build(s));
      s->w_graph += now_s() - t0;
    }
    SK(set_loop_start(s->exec, s->start_node, s->rs, nullptr, n, nullptr, 1, 0, s->hloop));
    SK(cudaGraphLaunch(s->exec, s->st));
    return TERSOFF_OK;
  }
  k_set_loop<<<1, 1, 0, s->st>>>(s->rs, n);
  SK(cudaGetLastError());
  for (long long k = 0; k < n; ++k) {
    SKR(srv_vv(s, s->st));
    AtomState &X = cur_atoms(s);
    ListState &L = s->L;
    SK(launch_build(s->st, (int)s->natoms, X.q, s->S.tab, s->S.ctl, s->ncell, s->radii, L.cell_count, L.cell_start, L.tile_sums, L.cell_atoms, L.cell_of, L.rank, L.nbr, L.rev, L.cnt,
                    L.cap, L.qref, s->rs, 1));
    SKR(srv_force(s, s->st));
    SK(launch_step_end(s->st, s->rs, s->S.ctl, (int)s->batch.size(), 0, 0));
  }
  return TERSOFF_OK;
}

// One chunk of steps for the whole batch (recovering from list or slot overflow).
int run_chunk(tersoff_server *s)
{
  SKR(launch_steps(s, s->chunk));
  for (int attempt = 0; attempt < 8; ++attempt) {
    RunState h;
    SKR(read_state(s, &h));
    if (h.status == 0) break;
    // finish the failed step (its integrator part ran), then the rest of the chunk
    if (h.status & ST_NLIST_OVERFLOW) {
      SK(cudaMemsetAsync(&s->rs->status, 0, sizeof(int), s->st));
      SKR(build_and_force(s));
    } else if (h.status & ST_NC_OVERFLOW) {
      if (h.maxnc > MAX_CAP) return srv_err(s, TERSOFF_ERR_NLIST_OVERFLOW, "%d in-cutoff neighbours", h.maxnc);
      s->gen_slots = force_slots_for(h.maxnc);
      graph_free(s);
      SK(cudaMemsetAsync(&s->rs->status, 0, sizeof(int), s->st));
      SKR(srv_force(s, s->st));
    } else {
      return srv_err(s, h.status & ST_NONFINITE ? TERSOFF_ERR_NONFINITE : TERSOFF_ERR_CUDA, "device status %d",
                     h.status);
    }
    SK(launch_step_end(s->st, s->rs, s->S.ctl, (int)s->batch.size(), 0, 0));
    const long long rest = h.steps_left - 1;
    if (rest > 0) SKR(launch_steps(s, rest));
  }
  s->w_chunks += 1;
  return TERSOFF_OK;
}

// Copy results of jobs whose run is over (steps done, closing kick applied): one
// energy kernel, one extraction kernel and one copy for all of them.
int retire(tersoff_server *s, std::vector<Job *> &done)
{
  const int S = (int)s->batch.size();
  if (!S) return TERSOFF_OK;
  std::vector<SysCtl> ctl(S);
  SK(cudaMemcpyAsync(ctl.data(), s->S.ctl, sizeof(SysCtl) * S, cudaMemcpyDeviceToHost, s->st));
  SK(cudaStreamSynchronize(s->st));
  std::vector<int> rtab;   // [nret + 1] staging offsets, then [nret] systems
  std::vector<int> rsys;
  int64_t staged = 0;
  for (int k = 0; k < S; ++k) {
    Job &J = *s->batch[k];
    J.ctl = ctl[k];
    if (ctl[k].steps_left == 0 && ctl[k].open == 0) {
      rtab.push_back((int)staged);
      rsys.push_back(k);
      staged += J.n;
    }
  }
  const int nret = (int)rsys.size();
  if (!nret) return TERSOFF_OK;
  rtab.push_back((int)staged);
  rtab.insert(rtab.end(), rsys.begin(), rsys.end());
  const size_t ebytes = sizeof(double) * 2 * S;
  const size_t tbytes = (sizeof(int) * rtab.size() + 255) / 256 * 256;
  const size_t nbytes = (size_t)staged * 6 * sizeof(double);
  if (!host_reserve(s, ebytes + tbytes + nbytes) || !dreserve(s->stage, s->stage_b, nbytes))
    return srv_err(s, TERSOFF_ERR_NOMEM, "staging");
  char *h = s->hstage;
  double *hE = (double *)h;
  int *ht = (int *)(h + ebytes);
  double *hpos = (double *)(h + ebytes + tbytes);
  memcpy(ht, rtab.data(), sizeof(int) * rtab.size());
  AtomState &X = cur_atoms(s);
  k_sys_energy<<<S, 256, 0, s->st>>>(s->eatom, X.v, X.q, s->P->d_mass, s->S.tab, s->sysE);
  SK(cudaGetLastError());
  SK(cudaMemcpyAsync(s->dtabs, ht, sizeof(int) * rtab.size(), cudaMemcpyHostToDevice, s->st));
  double *dpos = s->stage, *dvel = dpos + 3 * staged;
  k_extract_batch<<<(int)((staged + 255) / 256), 256, 0, s->st>>>((int)staged, X.x, X.v, s->dtabs,
                                                                   s->dtabs + nret + 1, nret, s->S.tab, dpos, dvel);
  SK(cudaGetLastError());
  SK(cudaMemcpyAsync(hE, s->sysE, ebytes, cudaMemcpyDeviceToHost, s->st));
  SK(cudaMemcpyAsync(hpos, dpos, nbytes, cudaMemcpyDeviceToHost, s->st));
  SK(cudaStreamSynchronize(s->st));
  const double *hvel = hpos + 3 * staged;
  for (int m = 0; m < nret; ++m) {
    Job &J = *s->batch[rsys[m]];
    J.rpos.assign(hpos + 3 * (size_t)rtab[m], hpos + 3 * (size_t)rtab[m] + 3 * J.n);
    J.rvel.assign(hvel + 3 * (size_t)rtab[m], hvel + 3 * (size_t)rtab[m] + 3 * J.n);
    J.epot = hE[2 * rsys[m]];
    J.ekin = hE[2 * rsys[m] + 1];
    done.push_back(&J);
  }
  return TERSOFF_OK;
}

void fail_all(tersoff_server *s, int code)
{
  std::lock_guard<std::mutex> lk(s->mu);
  s->msg = s->priv.err;
  for (Job *jp : s->batch) {
    Job &J = *jp;
    J.state = 3;
    J.err = code;
    J.t_done = now_s();
    s->stats.failed += 1;
    s->stats.running -= 1;
  }
  s->batch.clear();
  s->tab.clear();
  s->natoms = 0;
  s->broken = true;
  s->cv_done.notify_all();
}

void worker_loop(tersoff_server *s)
{
  cudaSetDevice(s->ctx->device);
  double busy_since = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty() || !s->batch.empty(); });
      if (s->stop) break;
    }
    if (s->broken) {
      // a device error ended the batch: fail what is queued as well
      std::lock_guard<std::mutex> lk(s->mu);
      while (!s->queue.empty()) {
        Job &J = *s->jobs.at(s->queue.front());
        s->queue.pop_front();
        J.state = 3;
        J.err = TERSOFF_ERR_CUDA;
        J.t_done = now_s();
        s->stats.failed += 1;
        s->stats.queued -= 1;
      }
      s->cv_done.notify_all();
      continue;
    }
    // retire finished jobs
    std::vector<Job *> done;
    double t0 = now_s();
    int rc = retire(s, done);
    s->w_retire += now_s() - t0;
    if (rc != TERSOFF_OK) {
      fail_all(s, rc);
      continue;
    }
    std::vector<Job *> order;
    std::vector<bool> is_new;
    bool changed = !done.empty();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const double t = now_s();
      s->stats.chunks = s->w_chunks;
      s->stats.repacks = s->w_repacks;
      s->stats.retire_s = s->w_retire;
      s->stats.repack_s = s->w_repack;
      s->stats.graph_s = s->w_graph;
      s->stats.run_s = s->w_run;
      for (Job *jp : done) {
        jp->state = 2;
        jp->t_done = t;
        s->stats.completed += 1;
        s->stats.running -= 1;
        s->stats.atom_steps += jp->n * jp->nsteps;
      }
      int64_t atoms = 0;
      for (Job *jp : s->batch) {
        if (std::find(done.begin(), done.end(), jp) != done.end()) continue;
        order.push_back(jp);
        is_new.push_back(false);
        atoms += jp->n;
      }
      // admit queued jobs in arrival order while slots and atom capacity allow
      while (!s->queue.empty()) {
        Job &J = *s->jobs.at(s->queue.front());
        if ((int)order.size() >= s->max_slots || atoms + J.n > s->cap_atoms) break;
        s->queue.pop_front();
        J.state = 1;
        J.t_admit = t;
        order.push_back(&J);
        is_new.push_back(true);
        atoms += J.n;
        s->stats.admitted += 1;
        s->stats.queued -= 1;
        s->stats.running += 1;
        changed = true;
      }
      if (!done.empty()) s->cv_done.notify_all();
    }
    if (changed) {
      if (order.empty()) {
        s->batch.clear();
        s->tab.clear();
        s->natoms = 0;
        graph_free(s);
      } else {
        t0 = now_s();
        rc = repack(s, order, is_new);
        s->w_repack += now_s() - t0;
        if (rc != TERSOFF_OK) {
          s->batch = order;
          fail_all(s, rc);
          continue;
        }
      }
    }
    // nothing left to integrate (all resident jobs finished): retire without stepping
    bool active = false;
    for (size_t k = 0; k < s->batch.size(); ++k) {
      const SysCtl &c = s->batch[k]->ctl;
      if (c.steps_left > 0 || c.open) active = true;
    }
    if (s->batch.empty()) {
      if (busy_since > 0) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.busy_s += now_s() - busy_since;
        busy_since = 0;
      }
      continue;
    }
    if (busy_since == 0) busy_since = now_s();
    if (active) {
      t0 = now_s();
      const double g0 = s->w_graph;
      rc = run_chunk(s);
      s->w_run += now_s() - t0 - (s->w_graph - g0);
      if (rc != TERSOFF_OK) fail_all(s, rc);
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (busy_since > 0) s->stats.busy_s += now_s() - busy_since;
}

}  // namespace

extern "C" {

int tersoff_server_create(tersoff_ctx *ctx, const tersoff_params *P, tersoff_precision prec, double skin,
                          size_t budget, int max_slots, int chunk_steps, tersoff_server **out)
{
  if (!ctx || !P || !out) return TERSOFF_ERR_ARG;
  *out = nullptr;
  if (!(skin >= 0) || max_slots < 1 || max_slots > 4096 || chunk_steps < 1 ||
      (prec != TERSOFF_FP64 && prec != TERSOFF_MIXED && prec != TERSOFF_SINGLE))
    return set_err(ctx, TERSOFF_ERR_ARG, "bad server arguments");
  cudaSetDevice(ctx->device);
  tersoff_server *s = new (std::nothrow) tersoff_server();
  if (!s) return TERSOFF_ERR_NOMEM;
  s->ctx = ctx;
  ctx->refs += 1;
  s->P = P;
  s->prec = prec;
  s->f32 = prec != TERSOFF_FP64;
  s->skin = skin;
  s->rl = P->rcmax + skin;
  s->radii = pair_radii(P, skin);
  s->max_slots = max_slots;
  s->chunk = chunk_steps;
  s->listcap = 32;
  s->fast_slots = (P->sym_angular && !ctx->general_only) ? 8 : 0;
  s->gen_slots = 16;
  s->use_graphs = !(getenv("TERSOFF_GRAPHS") && strcmp(getenv("TERSOFF_GRAPHS"), "0") == 0);
  s->cap_atoms = std::min<int64_t>((int64_t)(budget / bytes_per_atom(s->f32, s->listcap)), MAX_LIST_ATOMS);
  auto fail = [&](int rc) {
    tersoff_server_destroy(s);
    return rc;
  };
  if (s->cap_atoms < 1) return fail(set_err(ctx, TERSOFF_ERR_NOMEM, "budget below one atom"));
  if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking) != cudaSuccess)
    return fail(set_err(ctx, TERSOFF_ERR_CUDA, "streams"));
  s->priv.device = ctx->device;
  s->priv.stream = s->st;
  s->priv.refs = 0;
  tersoff_ctx *pc = &s->priv;
  if (new_rs(pc, &s->rs) != TERSOFF_OK) return fail(TERSOFF_ERR_NOMEM);
  const int64_t cap = s->cap_atoms;
  if (ensure_atoms(pc, s->A[0], cap, true) != TERSOFF_OK || ensure_atoms(pc, s->A[1], cap, true) != TERSOFF_OK ||
      ensure_scatter(pc, s->SC, cap, s->listcap, s->f32) != TERSOFF_OK ||
      ensure_list(pc, s->L, cap, s->listcap, 1) != TERSOFF_OK || !sys_alloc(s->S, max_slots) ||
      cudaMalloc((void **)&s->eatom, sizeof(double) * cap) != cudaSuccess ||
      cudaMalloc((void **)&s->sysE, sizeof(double) * 2 * max_slots) != cudaSuccess ||
      cudaMalloc((void **)&s->dtabs, sizeof(int) * 4 * (size_t)(max_slots + 1)) != cudaSuccess ||
      cudaMalloc((void **)&s->d_order, sizeof(int) * (size_t)std::max<int64_t>(cap, 1)) != cudaSuccess) {
    cudaGetLastError();
    return fail(set_err(ctx, TERSOFF_ERR_NOMEM, "cannot allocate the packed layout for %lld atoms", (long long)cap));
  }
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return fail(set_err(ctx, TERSOFF_ERR_CUDA, "server set-up"));
  s->stats.capacity_atoms = cap;
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return TERSOFF_OK;
}

int tersoff_server_submit(tersoff_server *s, const tersoff_job *job, uint64_t *job_id)
{
  if (!s || !job || !job_id) return TERSOFF_ERR_ARG;
  auto reject = [&](int code, const char *why) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->msg = why;
    return code;
  };
  if (job->n_atoms < 1 || !job->pos || !job->vel || !job->types || !(job->dt_ps > 0) || job->nsteps < 0)
    return reject(TERSOFF_ERR_ARG, "bad job (null pointer, n_atoms < 1, dt <= 0 or nsteps < 0)");
  if (job->n_atoms > s->cap_atoms) return reject(TERSOFF_ERR_NOMEM, "job larger than the server's atom capacity");
  for (int a = 0; a < 3; ++a) {
    if (!(job->box[a] > 0) || !std::isfinite(job->box[a])) return reject(TERSOFF_ERR_ARG, "box side not positive");
    if (job->box[a] < 2.0 * s->rl) return reject(TERSOFF_ERR_BOX_TOO_SMALL, "box side below 2*(cutoff+skin)");
  }
  std::unique_ptr<Job> J(new (std::nothrow) Job());
  if (!J) return TERSOFF_ERR_NOMEM;
  const int64_t n = job->n_atoms;
  J->n = n;
  J->pos.assign(job->pos, job->pos + 3 * n);
  J->vel.assign(job->vel, job->vel + 3 * n);
  J->types.assign(job->types, job->types + n);
  for (int64_t i = 0; i < n; ++i)
    if (J->types[i] < 0 || J->types[i] >= s->P->nt) return reject(TERSOFF_ERR_ARG, "atom type out of range");
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(J->pos[i]) || !std::isfinite(J->vel[i])) return reject(TERSOFF_ERR_ARG, "non-finite input");
  for (int a = 0; a < 3; ++a) J->box[a] = job->box[a];
  J->dt = job->dt_ps;
  J->nsteps = job->nsteps;
  J->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->broken) {
      s->msg = "server stopped after a device error: " + s->msg;
      return TERSOFF_ERR_CUDA;
    }
    J->id = s->next_id++;
    *job_id = J->id;
    s->queue.push_back(J->id);
    s->jobs[J->id] = std::move(J);
    s->stats.submitted += 1;
    s->stats.queued += 1;
  }
  s->cv_work.notify_one();
  return TERSOFF_OK;
}

int tersoff_server_poll(tersoff_server *s, uint64_t id, int *done)
{
  if (!s || !done) return TERSOFF_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return TERSOFF_ERR_NOT_FOUND;
  *done = it->second->state >= 2;
  return TERSOFF_OK;
}

int tersoff_server_wait(tersoff_server *s, uint64_t id, double timeout_s)
{
  if (!s) return TERSOFF_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return TERSOFF_ERR_NOT_FOUND;
  Job *J = it->second.get();
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(std::max(0.0, timeout_s));
  if (!s->cv_done.wait_until(lk, until, [&] { return J->state >= 2; })) return TERSOFF_ERR_TIMEOUT;
  return J->state == 2 ? TERSOFF_OK : J->err;
}

int tersoff_server_result(tersoff_server *s, uint64_t id, double *pos, double *vel, double energy[2], double times[3])
{
  if (!s) return TERSOFF_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return TERSOFF_ERR_NOT_FOUND;
  Job &J = *it->second;
  if (J.state < 2) return TERSOFF_ERR_BUSY;
  const int rc = J.state == 2 ? TERSOFF_OK : J.err;
  if (J.state == 2) {
    if (pos) memcpy(pos, J.rpos.data(), sizeof(double) * 3 * J.n);
    if (vel) memcpy(vel, J.rvel.data(), sizeof(double) * 3 * J.n);
    if (energy) {
      energy[0] = J.epot;
      energy[1] = J.ekin;
    }
  }
  if (times) {
    times[0] = J.t_admit - J.t_submit;
    times[1] = J.t_done - J.t_admit;
    times[2] = J.t_done - J.t_submit;
  }
  s->jobs.erase(it);
  return rc;
}

int tersoff_server_get_stats(tersoff_server *s, tersoff_server_stats *out)
{
  if (!s || !out) return TERSOFF_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return TERSOFF_OK;
}

const char *tersoff_server_last_error(tersoff_server *s)
{
  if (!s) return "null server";
  std::lock_guard<std::mutex> lk(s->mu);
  return s->msg.c_str();
}

void tersoff_server_destroy(tersoff_server *s)
{
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
  }
  if (s->st) cudaStreamSynchronize(s->st);
  graph_free(s);
  free_atoms(s->A[0]);
  free_atoms(s->A[1]);
  free_atoms(s->SC);
  free_list(s->L);
  sys_free(s->S);
  dfree(s->rs);
  dfree(s->eatom);
  dfree(s->sysE);
  dfree(s->stage);
  dfree(s->dtabs);
  dfree(s->d_order);
  if (s->hstage) cudaFreeHost(s->hstage);
  if (s->st) cudaStreamDestroy(s->st);
  if (s->cap_st) cudaStreamDestroy(s->cap_st);
  tersoff_ctx *ctx = s->ctx;
  delete s;
  if (ctx) ctx_release(ctx);
}

}  // extern "C"
