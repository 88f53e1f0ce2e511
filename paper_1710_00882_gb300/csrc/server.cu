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
// finished jobs (results copied out, their atoms freed) and admits queued jobs that
// fit the slots and the atom capacity implied by the device-memory budget: each new
// job gets a free system slot and a free atom range, and only the new jobs' lists
// and forces are computed (the layout section below).
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

// Register-kernel route order of nseg segments of atoms: segment k starts at
// position route_off[k] (ascending) and holds atoms atom_off[k] .. atom_off[k] +
// len[k] - 1; the positions between segments hold -1 (nothing to evaluate).
__global__ void k_route_order(int n, const int *__restrict__ route_off, const int *__restrict__ atom_off,
                              const int *__restrict__ len, int nseg, int *__restrict__ order)
{
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int k = range_of(route_off, nseg, t);
  const int u = t - route_off[k];
  order[t] = u < len[k] ? atom_off[k] + u : -1;
}

// Largest in-cutoff count (bits of the in-cutoff mask) per system and atom type of
// the atoms order[0, n).
__global__ void k_type_ncmax(int n, const int *__restrict__ order, const int4 *__restrict__ q,
                             const unsigned long long *__restrict__ mask, int *__restrict__ ncmax)
{
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = order[t];
  if (i < 0) return;
  const int w = q[i].w;
  atomicMax(&ncmax[sys_of(w) * MAX_TYPES + type_of(w)], __popcll(mask[i]));
}

// Survivors of a compaction: atom d of the new layout (survivors come first, dst_off
// ascending) is atom src_off[k] + (d - dst_off[k]) of the old one.  System indices
// are slots and do not change, so the atom words are copied as they are.
__global__ void k_move(int n, const dbl4 *__restrict__ sx, const dbl4 *__restrict__ sv, const int4 *__restrict__ sq,
                       dbl4 *__restrict__ dx, dbl4 *__restrict__ dv, int4 *__restrict__ dq,
                       const int *__restrict__ dst_off, const int *__restrict__ src_off, int nsurv)
{
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const int k = range_of(dst_off, nsurv, d);
  const int src = src_off[k] + (d - dst_off[k]);
  dx[d] = sx[src];
  dq[d] = sq[src];
  dv[d] = sv[src];
}

// New jobs, one staging block each at stage + boff[k] doubles (pos [n_k][3], vel
// [n_k][3], types [n_k] int32): atom t0 of the admission belongs to new job k (atom
// offsets st_off, st_off[nnew] = n), system slot[k].
__global__ void k_ingest_batch(int n, const double *__restrict__ stage, const int *__restrict__ boff,
                               const int *__restrict__ st_off, int nnew, const int *__restrict__ slot,
                               const SysTab *__restrict__ sys, int nt, dbl4 *__restrict__ x, dbl4 *__restrict__ v,
                               int4 *__restrict__ q, RunState *rs)
{
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 >= n) return;
  const int k = range_of(st_off, nnew, t0);
  const int t = t0 - st_off[k], nk = st_off[k + 1] - st_off[k];
  const double *pos = stage + boff[k], *vel = pos + 3 * (size_t)nk;
  const int *types = reinterpret_cast<const int *>(vel + 3 * (size_t)nk);
  const int sid = slot[k];
  const SysTab &T = sys[sid];
  const int d = T.atom_off + t;
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
// r_sys[k]; positions and velocities go out back to back as AoS float64.  The atoms
// then get the word dead_w (the system without atoms): every kernel of the layout
// leaves them alone until a new job is placed over them.
__global__ void k_extract_batch(int n, dbl4 *__restrict__ x, const dbl4 *__restrict__ v, int4 *__restrict__ q,
                                const int *__restrict__ r_off, const int *__restrict__ r_sys, int nret,
                                const SysTab *__restrict__ sys, int dead_w, double *__restrict__ pos,
                                double *__restrict__ vel)
{
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int k = range_of(r_off, nret, t);
  const int d = sys[r_sys[k]].atom_off + (t - r_off[k]);
  const dbl4 a = x[d], b = v[d];
  reinterpret_cast<double *>(x + d)[3] = __longlong_as_double((long long)dead_w);
  reinterpret_cast<int *>(q + d)[3] = dead_w;
  pos[3 * (size_t)t] = a.x;
  pos[3 * (size_t)t + 1] = a.y;
  pos[3 * (size_t)t + 2] = a.z;
  vel[3 * (size_t)t] = b.x;
  vel[3 * (size_t)t + 1] = b.y;
  vel[3 * (size_t)t + 2] = b.z;
}

// Potential and kinetic energy of the systems sys_ids[0..gridDim.x): one block per
// system, fixed-order sums.
__global__ void k_sys_energy(const double *__restrict__ eatom, const dbl4 *__restrict__ v, const int4 *__restrict__ q,
                             const double *__restrict__ mass, const SysTab *__restrict__ sys,
                             const int *__restrict__ sys_ids, double *__restrict__ out)
{
  __shared__ double sp[256], sk[256];
  const SysTab &T = sys[sys_ids[blockIdx.x]];
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
  bool one_species = false;   // every atom of one type: the 4-slot register route
  std::vector<int> perm;      // caller index of each stored atom (atoms grouped by type), or empty
  int tcount[MAX_TYPES] = {0, 0, 0, 0};   // atoms of each type (stored in type order)
  int cls[MAX_TYPES] = {8, 8, 8, 8};      // register-kernel slots of each type's atoms (multi-species jobs)
  double box[3] = {0, 0, 0};
  double dt = 0;
  int64_t nsteps = 0;
  int state = 0;   // 0 queued, 1 running, 2 done, 3 failed
  int err = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int slot = -1;        // system index while resident
  int64_t off = 0;      // first atom while resident
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
  int64_t cap_atoms = 0;        // atom capacity; also the stride of every [slot][atom] list array
  cudaStream_t st = nullptr, cap_st = nullptr;
  AtomState A[2];          // packed positions/velocities (x, v, q); compactions copy between the two
  int cur = 0;
  AtomState SC;            // force scatter buffers of the packed layout
  ListState L;
  SysDev S;                // [max_slots + 1] system tables; system index = slot, slot max_slots: freed atoms
  RunState *rs = nullptr;
  double *eatom = nullptr, *sysE = nullptr;
  double *stage = nullptr;      // device staging (new jobs in, finished jobs out)
  size_t stage_b = 0;
  char *hstage = nullptr;       // pinned host staging
  size_t hstage_b = 0;
  // results of the jobs retired last: copied to pinned memory on the stream, then
  // handed to the jobs while the next chunk runs
  char *hres = nullptr;
  size_t hres_b = 0;
  double *rstage = nullptr;     // their device staging
  size_t rstage_b = 0;
  cudaEvent_t ev_res = nullptr; // recorded after their copy to hres
  std::vector<Job *> pending;   // retired jobs whose results are in flight
  std::vector<int64_t> pend_off;   // their atom offsets in hres, size pending + 1
  // staging blocks of the first queued jobs, written while a chunk runs
  char *hpre = nullptr;
  size_t hpre_b = 0;
  std::vector<Job *> pre_jobs;  // those jobs, in queue order (a prefix of the queue)
  std::vector<size_t> pre_off;  // their block offsets in hpre (bytes), size pre_jobs + 1
  int *dtabs = nullptr;         // device index tables of an admission / retirement (TAB_INTS ints)
  // register-kernel routes: atoms of one-species jobs (at most 4 in-cutoff
  // neighbours in the solids served) through the 4-slot kernel, the others through
  // the 8-slot kernel.  A job's route follows from its own atoms only, so its
  // arithmetic does not depend on the batch.
  ForceRoutes routes{};         // every resident atom (the step graph)
  ForceRoutes new_routes{};     // the atoms of the jobs admitted last (their first force evaluation)
  int *d_order = nullptr;       // [capacity + padding] route order of every resident atom
  int *d_order_new = nullptr;   // [capacity + padding] route order of the newly admitted atoms
  int *d_ncmax = nullptr;       // [max_slots + 1][MAX_TYPES] largest in-cutoff count per system and type
  int *h_ncmax = nullptr;       // its pinned host copy
  std::vector<SysTab> tab;      // host copy of the system tables [max_slots + 1]
  std::vector<Job *> slot_job;  // resident job of each slot (owned by `jobs`; touched by the worker only)
  int64_t hw = 0;               // atoms [0, hw) hold every resident job (the rest of the range is freed atoms)
  int64_t live = 0;             // resident atoms
  int nres = 0;                 // resident jobs
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
  int64_t w_chunks = 0, w_repacks = 0, w_compactions = 0;
  double w_retire = 0, w_repack = 0, w_graph = 0, w_run = 0;
  double w_hw = 0, w_live = 0;  // sums over chunks of the layout's atoms [0, hw) and of the resident atoms
  double compact_frac = 0.3;    // compaction threshold: share of freed atoms below hw ...
  int64_t compact_min = 1 << 16;   // ... and their least number
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
         + v4 + 8 + 8 + 4 + 16 + 12 + 8 + 8 + 16;  // selfF, mask, work, cnt, qref, cells, eatom, route orders, slack
}

// pinned host staging of at least `bytes` (contents not kept)
bool pinned_reserve(char *&p, size_t &have, size_t bytes)
{
  if (bytes <= have && p) return true;
  if (p) cudaFreeHost(p);
  p = nullptr;
  have = 0;
  bytes = std::max<size_t>(bytes + bytes / 4, 1 << 20);
  if (cudaHostAlloc((void **)&p, bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  have = bytes;
  return true;
}

bool host_reserve(tersoff_server *s, size_t bytes) { return pinned_reserve(s->hstage, s->hstage_b, bytes); }

// Staging block of a job of n atoms: positions [n][3] and velocities [n][3] as
// float64, then types [n] as int32, padded to whole doubles.
size_t block_doubles(int64_t n) { return 6 * (size_t)n + ((size_t)n + 1) / 2; }

void write_block(char *dst, const Job &J)
{
  double *d = reinterpret_cast<double *>(dst);
  memcpy(d, J.pos.data(), sizeof(double) * 3 * J.n);
  memcpy(d + 3 * J.n, J.vel.data(), sizeof(double) * 3 * J.n);
  memcpy(d + 6 * J.n, J.types.data(), sizeof(int32_t) * J.n);
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
  SK(launch_force_part(3, st, s->prec, s->fast_slots, P->fast, s->gen_slots, 0, 0, (int)s->hw, (int)s->cap_atoms,
                       X.x, X.q, s->L.nbr, s->L.cnt, s->S.tab, s->f32 ? P->pair_f : P->pair_d,
                       s->f32 ? P->trip_f : P->trip_d, P->nt, s->SC.contrib, s->SC.selfF, s->SC.mask, s->SC.work,
                       s->SC.nwork, s->SC.partial, s->rs, s->eatom, s->fast_slots > 0 ? &s->routes : nullptr, 0));
  return TERSOFF_OK;
}

// First force evaluation of the jobs admitted last (the others keep theirs): their
// own route order with the register kernels, or every atom with the general kernel.
int srv_force_new(tersoff_server *s)
{
  if (s->fast_slots == 0) return srv_force(s, s->st);
  const tersoff_params *P = s->P;
  AtomState &X = cur_atoms(s);
  SK(launch_force_part(3, s->st, s->prec, s->fast_slots, P->fast, s->gen_slots, 0, 0, (int)s->hw,
                       (int)s->cap_atoms, X.x, X.q, s->L.nbr, s->L.cnt, s->S.tab, s->f32 ? P->pair_f : P->pair_d,
                       s->f32 ? P->trip_f : P->trip_d, P->nt, s->SC.contrib, s->SC.selfF, s->SC.mask, s->SC.work,
                       s->SC.nwork, s->SC.partial, s->rs, s->eatom, &s->new_routes, 0));
  return TERSOFF_OK;
}

int srv_vv(tersoff_server *s, cudaStream_t st)
{
  AtomState &X = cur_atoms(s);
  const float lim = (float)(0.25 * s->skin * s->skin);
  SK(launch_vv(st, s->prec, false, (int)s->hw, (int)s->cap_atoms, -1, X.x, X.v, X.q, s->L.qref, s->SC.contrib, s->SC.selfF,
               s->SC.mask, s->L.rev, s->S.tab, s->S.ctl, s->P->d_mass, lim, s->SC.kepart, s->rs));
  return TERSOFF_OK;
}

// full: every resident atom gets a new list; else only systems whose rebuild flag is set
int srv_build(tersoff_server *s, cudaStream_t st, bool full)
{
  AtomState &X = cur_atoms(s);
  ListState &L = s->L;
  SK(launch_build(st, (int)s->hw, (int)s->cap_atoms, X.q, s->S.tab, full ? nullptr : s->S.ctl, s->ncell, s->radii, L.cell_count, L.cell_start, L.tile_sums, L.cell_atoms,
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
  // kernels captured right behind another kernel become programmatic dependents
  pdl_scope pdl;
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
  SK(launch_step_end(st, s->rs, s->S.ctl, s->max_slots + 1, hloop, 1));
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

// ---- layout: system slots, atom ranges, tables ------------------------------
//
// A resident job keeps its system slot and its atom range [off, off + n) for its
// whole run: admissions place new jobs into free ranges (first fit, lowest address)
// and build lists and forces for the new jobs only; retirements turn a job's atoms
// into freed atoms (system max_slots, no atoms), which every kernel leaves alone.
// The list arrays are strided by the capacity, so no resident job's list, reverse
// indices or force contributions move.  When a job fits no free range, or freed
// atoms below the high-water mark pass a share of it, the layout is compacted:
// survivors move down in address order, and every list and force is rebuilt.

int TAB_INTS(const tersoff_server *s) { return 32 * (s->max_slots + 2); }   // ints of dtabs

// most padding a route order holds: a warp's worth before each segment (a job, or one
// type of a multi-species job) and before the 8-slot group
int64_t route_pad(const tersoff_server *s) { return 32 * ((int64_t)s->max_slots * MAX_TYPES + 2); }

constexpr double FREED_COMPACT_FRAC = 0.3;     // compact above this share of freed atoms below hw ...
constexpr int64_t FREED_COMPACT_MIN = 1 << 16; // ... when they are at least this many

int dead_word(const tersoff_server *s) { return make_w(0, s->max_slots); }

// System tables (cell numbering in slot order), high-water mark and counts of the
// resident jobs; entry max_slots (freed atoms) has no atoms and no cells.
int layout_tables(tersoff_server *s)
{
  const tersoff_params *P = s->P;
  int coff = 0, nres = 0;
  int64_t hw = 0, live = 0;
  for (int k = 0; k <= s->max_slots; ++k) {
    SysTab &T = s->tab[k];
    T = SysTab{};
    const Job *J = k < s->max_slots ? s->slot_job[k] : nullptr;
    if (!J) continue;
    CellGrid gr;
    if (make_grid(J->box, s->rl, &gr) != TERSOFF_OK) return srv_err(s, TERSOFF_ERR_ARG, "cell grid too large");
    T.geo = make_geom(J->box);
    for (int a = 0; a < 3; ++a) T.nc[a] = gr.nc[a];
    T.cell_off = coff;
    T.atom_off = (int)J->off;
    T.natoms = (int)J->n;
    T.dt = J->dt;
    for (int a = 0; a < MAX_TYPES; ++a) T.kick[a] = a < P->nt ? 0.5 * J->dt * ACCEL / P->masses[a] : 0.0;
    coff += gr.ncell;
    hw = std::max<int64_t>(hw, J->off + J->n);
    live += J->n;
    ++nres;
  }
  s->ncell = coff;
  s->hw = hw;
  s->live = live;
  s->nres = nres;
  if (ensure_list(&s->priv, s->L, s->cap_atoms, s->listcap, std::max(1, coff)) != TERSOFF_OK)
    return srv_err(s, TERSOFF_ERR_NOMEM, "cell arrays for %d cells", coff);
  return TERSOFF_OK;
}

// Route table of the jobs js appended to the host int table `it`: segments of atoms
// (a one-species job, or the atoms of one type of a multi-species job, stored grouped
// by type), those for 4 slots first, then those for 8, each group in job order; R
// gets the launches over order[0, total).  A type of a multi-species job takes 4
// slots when the job's first force evaluation saw at most 4 in-cutoff neighbours on
// every atom of that type (classify), else 8 (8 until then).  Every segment starts a
// warp (the positions between segments hold -1), so the atoms a warp evaluates
// together, and the choice of route, depend on the job alone: its results do not
// depend on the batch.
void route_table(const std::vector<Job *> &js, int *order, std::vector<int> &it, size_t *at, int *nsys,
                 int64_t *total, ForceRoutes &R)
{
  std::vector<std::pair<int64_t, int64_t>> s4, s8;   // (first atom, atoms)
  for (const Job *J : js) {
    if (J->one_species) {
      s4.push_back({J->off, J->n});
      continue;
    }
    int64_t o = J->off;
    for (int t = 0; t < MAX_TYPES; ++t) {
      if (!J->tcount[t]) continue;
      (J->cls[t] == 4 ? s4 : s8).push_back({o, J->tcount[t]});
      o += J->tcount[t];
    }
  }
  const size_t n4s = s4.size();
  s4.insert(s4.end(), s8.begin(), s8.end());
  const int n = (int)s4.size();
  *at = it.size();
  it.resize(it.size() + 3 * (size_t)n + 1);
  int *ro = it.data() + *at, *ao = ro + n + 1, *ln = ao + n;
  auto warp_up = [](int64_t p) { return (p + 31) & ~(int64_t)31; };
  int64_t pos = 0, end4 = 0;
  for (int k = 0; k < n; ++k) {
    pos = warp_up(pos);
    ro[k] = (int)pos;
    ao[k] = (int)s4[k].first;
    ln[k] = (int)s4[k].second;
    pos += s4[k].second;
    if ((size_t)k + 1 == n4s) end4 = pos;
  }
  ro[n] = (int)pos;
  *nsys = n;
  *total = pos;
  R = ForceRoutes{};
  if (n4s > 0 && n4s < (size_t)n) {
    const int64_t b8 = warp_up(end4);
    R.n = 2;
    R.r[0] = ForceRoute{order, 0, (int)end4, 4, 0};
    R.r[1] = ForceRoute{order, (int)b8, (int)(pos - b8), 8, 0};
  } else {
    R.n = 1;
    R.r[0] = ForceRoute{order, 0, (int)pos, n4s > 0 ? 4 : 8, 0};
  }
}

std::vector<Job *> resident(const tersoff_server *s)
{
  std::vector<Job *> r;
  for (Job *J : s->slot_job)
    if (J) r.push_back(J);
  return r;
}

// First-fit placement of a job of n atoms among the resident ranges (sorted by
// offset, updated in place); -1 when no free range holds it.
int64_t place(std::vector<std::pair<int64_t, int64_t>> &ranges, int64_t n, int64_t cap)
{
  int64_t prev = 0;
  for (size_t k = 0; k <= ranges.size(); ++k) {
    const int64_t next = k < ranges.size() ? ranges[k].first : cap;
    if (next - prev >= n) {
      ranges.insert(ranges.begin() + k, {prev, n});
      return prev;
    }
    if (k < ranges.size()) prev = ranges[k].first + ranges[k].second;
  }
  return -1;
}

// Status of an admission's list build and force evaluation: a list overflow grows
// the lists and rebuilds every job (build_and_force); a neighbour count above the
// general kernel's slots widens it.
int check_admission(tersoff_server *s, bool *recovered)
{
  *recovered = false;
  for (int attempt = 0; attempt < 4; ++attempt) {
    RunState h;
    SKR(read_state(s, &h));
    if (h.status == 0) return TERSOFF_OK;
    *recovered = true;
    SK(cudaMemsetAsync(&s->rs->status, 0, sizeof(int), s->st));
    if (h.status & ST_NLIST_OVERFLOW) {
      SKR(build_and_force(s));
    } else if (h.status & ST_NC_OVERFLOW) {
      if (h.maxnc > MAX_CAP) return srv_err(s, TERSOFF_ERR_NLIST_OVERFLOW, "%d in-cutoff neighbours", h.maxnc);
      s->gen_slots = force_slots_for(h.maxnc);
      SKR(srv_force(s, s->st));
    } else {
      return srv_err(s, h.status & ST_NONFINITE ? TERSOFF_ERR_NONFINITE : TERSOFF_ERR_CUDA, "device status %d",
                     h.status);
    }
  }
  return srv_err(s, TERSOFF_ERR_NLIST_OVERFLOW, "admission did not converge");
}

bool any_multi(const std::vector<Job *> &fresh)
{
  for (const Job *J : fresh)
    if (!J->one_species) return true;
  return false;
}

// Largest in-cutoff count per system and type of the new atoms (bits of their
// in-cutoff masks, after their first force evaluation), copied to h_ncmax; the copy
// is complete after the stream's next synchronisation.
int count_enqueue(tersoff_server *s, int64_t tot_new)
{
  const size_t nb = sizeof(int) * (size_t)(s->max_slots + 1) * MAX_TYPES;
  SK(cudaMemsetAsync(s->d_ncmax, 0, nb, s->st));
  AtomState &X = cur_atoms(s);
  k_type_ncmax<<<(int)((tot_new + 255) / 256), 256, 0, s->st>>>((int)tot_new, s->d_order_new, X.q, s->SC.mask,
                                                                 s->d_ncmax);
  SK(cudaGetLastError());
  SK(cudaMemcpyAsync(s->h_ncmax, s->d_ncmax, nb, cudaMemcpyDeviceToHost, s->st));
  return TERSOFF_OK;
}

// Register-kernel slots of the types of the new multi-species jobs from h_ncmax (at
// most 4 in-cutoff neighbours on every atom of a type: 4 slots, else 8), then the
// route order of every resident atom again when a type moved to the 4-slot kernel.
int classify(tersoff_server *s, const std::vector<Job *> &fresh)
{
  bool changed = false;
  for (Job *J : fresh) {
    if (J->one_species) continue;
    for (int t = 0; t < MAX_TYPES; ++t) {
      const int c = J->tcount[t] && s->h_ncmax[(size_t)J->slot * MAX_TYPES + t] <= 4 ? 4 : 8;
      changed = changed || c != J->cls[t];
      J->cls[t] = c;
    }
  }
  if (!changed) return TERSOFF_OK;
  std::vector<int> it;
  size_t at = 0;
  int ns = 0;
  int64_t tot = 0;
  route_table(resident(s), s->d_order, it, &at, &ns, &tot, s->routes);
  SK(cudaMemcpy(s->dtabs, it.data(), sizeof(int) * it.size(), cudaMemcpyHostToDevice));
  if (tot > 0) {
    k_route_order<<<(int)((tot + 255) / 256), 256, 0, s->st>>>((int)tot, s->dtabs, s->dtabs + ns + 1,
                                                               s->dtabs + 2 * ns + 1, ns, s->d_order);
    SK(cudaGetLastError());
  }
  graph_free(s);
  return TERSOFF_OK;
}

// Make the resident set of slot_job current on the device.  fresh: the jobs placed
// since the last layout (slot, offset and step control set).  compacted: survivors
// moved to the offsets they now hold, from old_off (same order as surv).
int apply_layout(tersoff_server *s, const std::vector<Job *> &fresh, const std::vector<Job *> &surv,
                 const std::vector<int64_t> &old_off, bool compacted)
{
  const tersoff_params *P = s->P;
  SKR(layout_tables(s));
  const int NS = s->max_slots + 1;
  const int nnew = (int)fresh.size();
  const int nsurv = compacted ? (int)surv.size() : 0;
  // int tables: new jobs' atom offsets [nnew + 1], slots [nnew] and staging block
  // offsets [nnew] (doubles); survivors' destination and source offsets [nsurv]
  // each; the two route tables
  std::vector<int> it(3 * (size_t)nnew + 1 + 2 * (size_t)nsurv, 0);
  int *st_off = it.data(), *nslot = st_off + nnew + 1, *boff = nslot + nnew, *dst_off = boff + nnew,
      *src_off = dst_off + nsurv;
  // the first new jobs may be staged already (prestage, while the last chunk ran)
  size_t npre = 0;
  while (npre < s->pre_jobs.size() && npre < (size_t)nnew && s->pre_jobs[npre] == fresh[npre]) ++npre;
  const size_t pre_bytes = npre ? s->pre_off[npre] - s->pre_off[0] : 0;
  int64_t staged = 0, moved = 0;
  size_t rest_doubles = 0;
  for (int k = 0; k < nnew; ++k) {
    st_off[k] = (int)staged;
    nslot[k] = fresh[k]->slot;
    if ((size_t)k < npre) {
      boff[k] = (int)((s->pre_off[k] - s->pre_off[0]) / sizeof(double));
    } else {
      boff[k] = (int)(pre_bytes / sizeof(double) + rest_doubles);
      rest_doubles += block_doubles(fresh[k]->n);
    }
    staged += fresh[k]->n;
  }
  st_off[nnew] = (int)staged;
  for (int k = 0; k < nsurv; ++k) {
    dst_off[k] = (int)surv[k]->off;
    src_off[k] = (int)old_off[k];
    moved = std::max<int64_t>(moved, surv[k]->off + surv[k]->n);
  }
  size_t at_all = 0, at_new = 0;
  int ns_all = 0, ns_new = 0;
  int64_t tot_all = 0, tot_new = 0;
  route_table(resident(s), s->d_order, it, &at_all, &ns_all, &tot_all, s->routes);
  route_table(fresh, s->d_order_new, it, &at_new, &ns_new, &tot_new, s->new_routes);
  // the route tables grew the vector: take its pointers again
  st_off = it.data();
  nslot = st_off + nnew + 1;
  boff = nslot + nnew;
  dst_off = boff + nnew;
  src_off = dst_off + nsurv;
  if (it.size() > (size_t)TAB_INTS(s)) return srv_err(s, TERSOFF_ERR_ARG, "index tables exceed their buffer");
  // step control: resident jobs as the last chunk left them, new jobs from the start;
  // copy A flags the new jobs for their first list build, copy B clears the flags
  std::vector<SysCtl> ctlA(NS, SysCtl{0, 0, 0}), ctlB;
  for (Job *J : resident(s)) ctlA[J->slot] = SysCtl{J->ctl.steps_left, J->ctl.open, 0};
  ctlB = ctlA;
  for (Job *J : fresh) ctlA[J->slot].rebuild = 1;
  // pinned staging: tables, then the blocks of the new jobs not staged already
  const size_t b_tab = sizeof(SysTab) * NS, b_ctl = sizeof(SysCtl) * NS, b_int = sizeof(int) * it.size();
  const size_t tbytes = b_tab + 2 * b_ctl + b_int;
  const size_t tpad = (tbytes + 255) / 256 * 256;
  const size_t rest_bytes = rest_doubles * sizeof(double);
  if (!host_reserve(s, tpad + rest_bytes)) return srv_err(s, TERSOFF_ERR_NOMEM, "pinned staging");
  if (pre_bytes + rest_bytes && !dreserve(s->stage, s->stage_b, pre_bytes + rest_bytes))
    return srv_err(s, TERSOFF_ERR_NOMEM, "staging");
  char *h = s->hstage;
  memcpy(h, s->tab.data(), b_tab);
  memcpy(h + b_tab, ctlA.data(), b_ctl);
  memcpy(h + b_tab + b_ctl, ctlB.data(), b_ctl);
  memcpy(h + b_tab + 2 * b_ctl, it.data(), b_int);
  for (int k = (int)npre; k < nnew; ++k)
    write_block(h + tpad + ((size_t)boff[k] * sizeof(double) - pre_bytes), *fresh[k]);
  SK(cudaMemcpyAsync(s->S.tab, h, b_tab, cudaMemcpyHostToDevice, s->st));
  SK(cudaMemcpyAsync(s->S.ctl, h + b_tab + (compacted ? b_ctl : 0), b_ctl, cudaMemcpyHostToDevice, s->st));
  SK(cudaMemcpyAsync(s->dtabs, h + b_tab + 2 * b_ctl, b_int, cudaMemcpyHostToDevice, s->st));
  const int *d_st = s->dtabs, *d_slot = d_st + nnew + 1, *d_boff = d_slot + nnew, *d_dst = d_boff + nnew,
            *d_src = d_dst + nsurv;
  AtomState &src = s->A[s->cur];
  AtomState &dst = s->A[compacted ? 1 - s->cur : s->cur];
  if (nsurv > 0 && moved > 0) {
    k_move<<<(int)((moved + 255) / 256), 256, 0, s->st>>>((int)moved, src.x, src.v, src.q, dst.x, dst.v, dst.q, d_dst,
                                                          d_src, nsurv);
    SK(cudaGetLastError());
  }
  if (staged > 0) {
    if (pre_bytes)
      SK(cudaMemcpyAsync(s->stage, s->hpre + s->pre_off[0], pre_bytes, cudaMemcpyHostToDevice, s->st));
    if (rest_bytes)
      SK(cudaMemcpyAsync((char *)s->stage + pre_bytes, h + tpad, rest_bytes, cudaMemcpyHostToDevice, s->st));
    k_ingest_batch<<<(int)((staged + 255) / 256), 256, 0, s->st>>>((int)staged, s->stage, d_boff, d_st, nnew, d_slot,
                                                                   s->S.tab, P->nt, dst.x, dst.v, dst.q, s->rs);
    SK(cudaGetLastError());
  }
  // the prestaged blocks used here stay valid until this admission's copies are
  // done (the synchronisation below); the entries go now
  s->pre_jobs.erase(s->pre_jobs.begin(), s->pre_jobs.begin() + npre);
  s->pre_off.erase(s->pre_off.begin(), s->pre_off.begin() + npre);
  if (tot_all > 0) {
    const int *t = s->dtabs + at_all;
    k_route_order<<<(int)((tot_all + 255) / 256), 256, 0, s->st>>>((int)tot_all, t, t + ns_all + 1,
                                                                   t + 2 * ns_all + 1, ns_all, s->d_order);
    SK(cudaGetLastError());
  }
  if (tot_new > 0) {
    const int *t = s->dtabs + at_new;
    k_route_order<<<(int)((tot_new + 255) / 256), 256, 0, s->st>>>((int)tot_new, t, t + ns_new + 1,
                                                                   t + 2 * ns_new + 1, ns_new, s->d_order_new);
    SK(cudaGetLastError());
  }
  if (compacted) s->cur = 1 - s->cur;
  graph_free(s);
  // the new multi-species jobs' in-cutoff counts per type decide their routes
  const bool counts = nnew > 0 && s->fast_slots > 0 && tot_new > 0 && any_multi(fresh);
  if (compacted) {
    SKR(build_and_force(s));
    s->w_compactions += 1;
    if (counts) {
      SKR(count_enqueue(s, tot_new));
      SK(cudaStreamSynchronize(s->st));
    }
  } else if (nnew > 0) {
    // lists of the new jobs only (their rebuild flags), then their first forces and
    // in-cutoff counts, read at one synchronisation
    SK(cudaMemsetAsync(&s->rs->maxcount, 0, sizeof(int), s->st));
    SKR(srv_build(s, s->st, false));
    SK(cudaMemcpyAsync(s->S.ctl, h + b_tab + b_ctl, b_ctl, cudaMemcpyHostToDevice, s->st));
    SKR(srv_force_new(s));
    if (counts) SKR(count_enqueue(s, tot_new));
    bool recovered = false;
    SKR(check_admission(s, &recovered));
    if (counts && recovered) {
      SKR(count_enqueue(s, tot_new));
      SK(cudaStreamSynchronize(s->st));
    }
  }
  if (counts) SKR(classify(s, fresh));
  if (nnew > 0) s->w_repacks += 1;
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
    SK(launch_build(s->st, (int)s->hw, (int)s->cap_atoms, X.q, s->S.tab, s->S.ctl, s->ncell, s->radii, L.cell_count,
                    L.cell_start, L.tile_sums, L.cell_atoms, L.cell_of, L.rank, L.nbr, L.rev, L.cnt, L.cap, L.qref,
                    s->rs, 1));
    SKR(srv_force(s, s->st));
    SK(launch_step_end(s->st, s->rs, s->S.ctl, s->max_slots + 1, 0, 0));
  }
  return TERSOFF_OK;
}

// One chunk of steps for the whole batch: launched, then waited for.
int chunk_launch(tersoff_server *s) { return launch_steps(s, s->chunk); }

// Wait for the chunk (recovering from list or slot overflow).
int chunk_wait(tersoff_server *s)
{
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
    SK(launch_step_end(s->st, s->rs, s->S.ctl, s->max_slots + 1, 0, 0));
    const long long rest = h.steps_left - 1;
    if (rest > 0) SKR(launch_steps(s, rest));
  }
  s->w_chunks += 1;
  return TERSOFF_OK;
}

// Jobs whose run is over (steps done, closing kick applied): one energy kernel, one
// extraction kernel and one copy to pinned memory for all of them, enqueued on the
// stream (the event ev_res follows the copy).  Their slots are freed at once and
// their atoms become freed atoms; finish_retire hands the results to the jobs.
int retire(tersoff_server *s)
{
  if (s->nres == 0) return TERSOFF_OK;
  const int NS = s->max_slots + 1;
  std::vector<SysCtl> ctl(NS);
  SK(cudaMemcpyAsync(ctl.data(), s->S.ctl, sizeof(SysCtl) * NS, cudaMemcpyDeviceToHost, s->st));
  SK(cudaStreamSynchronize(s->st));
  std::vector<int> rtab;   // [nret + 1] staging offsets, then [nret] systems
  std::vector<int> rsys;
  int64_t staged = 0;
  for (int k = 0; k < s->max_slots; ++k) {
    Job *J = s->slot_job[k];
    if (!J) continue;
    J->ctl = ctl[k];
    if (ctl[k].steps_left == 0 && ctl[k].open == 0) {
      rtab.push_back((int)staged);
      rsys.push_back(k);
      staged += J->n;
    }
  }
  const int nret = (int)rsys.size();
  if (!nret) return TERSOFF_OK;
  rtab.push_back((int)staged);
  rtab.insert(rtab.end(), rsys.begin(), rsys.end());
  const size_t ebytes = sizeof(double) * 2 * nret;
  const size_t epad = (ebytes + 255) / 256 * 256;
  const size_t tbytes = sizeof(int) * rtab.size();
  const size_t nbytes = (size_t)staged * 6 * sizeof(double);
  if (!pinned_reserve(s->hres, s->hres_b, epad + nbytes + tbytes) || !dreserve(s->rstage, s->rstage_b, nbytes))
    return srv_err(s, TERSOFF_ERR_NOMEM, "result staging");
  char *h = s->hres;
  int *ht = (int *)(h + epad + nbytes);
  memcpy(ht, rtab.data(), tbytes);
  AtomState &X = cur_atoms(s);
  SK(cudaMemcpyAsync(s->dtabs, ht, tbytes, cudaMemcpyHostToDevice, s->st));
  k_sys_energy<<<nret, 256, 0, s->st>>>(s->eatom, X.v, X.q, s->P->d_mass, s->S.tab, s->dtabs + nret + 1, s->sysE);
  SK(cudaGetLastError());
  double *dpos = s->rstage, *dvel = dpos + 3 * staged;
  k_extract_batch<<<(int)((staged + 255) / 256), 256, 0, s->st>>>((int)staged, X.x, X.v, X.q, s->dtabs,
                                                                   s->dtabs + nret + 1, nret, s->S.tab,
                                                                   dead_word(s), dpos, dvel);
  SK(cudaGetLastError());
  SK(cudaMemcpyAsync(h, s->sysE, ebytes, cudaMemcpyDeviceToHost, s->st));
  SK(cudaMemcpyAsync(h + epad, dpos, nbytes, cudaMemcpyDeviceToHost, s->st));
  SK(cudaEventRecord(s->ev_res, s->st));
  s->pend_off.assign(rtab.begin(), rtab.begin() + nret + 1);
  for (int m = 0; m < nret; ++m) {
    Job &J = *s->slot_job[rsys[m]];
    s->slot_job[J.slot] = nullptr;
    J.slot = -1;
    s->pending.push_back(&J);
  }
  return TERSOFF_OK;
}

// Hand the results of the jobs retired last to them (after their copy, ev_res) and
// report the jobs done; runs while the next chunk is on the device.
int finish_retire(tersoff_server *s)
{
  if (s->pending.empty()) return TERSOFF_OK;
  SK(cudaEventSynchronize(s->ev_res));
  const int nret = (int)s->pending.size();
  const int64_t staged = s->pend_off[nret];
  const size_t epad = (sizeof(double) * 2 * nret + 255) / 256 * 256;
  const double *hE = (const double *)s->hres;
  const double *hpos = (const double *)(s->hres + epad), *hvel = hpos + 3 * staged;
  for (int m = 0; m < nret; ++m) {
    Job &J = *s->pending[m];
    const size_t o = 3 * (size_t)s->pend_off[m];
    if (J.perm.empty()) {
      J.rpos.assign(hpos + o, hpos + o + 3 * J.n);
      J.rvel.assign(hvel + o, hvel + o + 3 * J.n);
    } else {
      J.rpos.resize(3 * J.n);
      J.rvel.resize(3 * J.n);
      for (int64_t k = 0; k < J.n; ++k) {
        const size_t c = 3 * (size_t)J.perm[k];
        for (int a = 0; a < 3; ++a) {
          J.rpos[c + a] = hpos[o + 3 * k + a];
          J.rvel[c + a] = hvel[o + 3 * k + a];
        }
      }
    }
    J.epot = hE[2 * m];
    J.ekin = hE[2 * m + 1];
  }
  std::lock_guard<std::mutex> lk(s->mu);
  const double t = now_s();
  for (Job *jp : s->pending) {
    jp->state = 2;
    jp->t_done = t;
    s->stats.completed += 1;
    s->stats.running -= 1;
    s->stats.atom_steps += jp->n * jp->nsteps;
  }
  s->pending.clear();
  s->cv_done.notify_all();
  return TERSOFF_OK;
}

// Stage the first queued jobs into hpre while a chunk runs, so that their admission
// copies them to the device without a host copy of its own.  The blocks of jobs
// still queued from last time move to the front first (their copies, if any, are
// done: every admission that staged jobs waited for its copies).
void prestage(tersoff_server *s)
{
  if (!s->hpre) return;
  if (!s->pre_off.empty() && s->pre_off[0] > 0) {
    const size_t base = s->pre_off[0];
    memmove(s->hpre, s->hpre + base, s->pre_off.back() - base);
    for (size_t &o : s->pre_off) o -= base;
  }
  if (s->pre_off.empty()) s->pre_off.push_back(0);
  std::vector<Job *> add;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    size_t end = s->pre_off.back();
    int64_t atoms = 0;
    for (const Job *J : s->pre_jobs) atoms += J->n;
    for (size_t k = s->pre_jobs.size(); k < s->queue.size() && k < (size_t)s->max_slots; ++k) {
      Job *J = s->jobs.at(s->queue[k]).get();
      const size_t b = block_doubles(J->n) * sizeof(double);
      if (end + b > s->hpre_b || atoms + J->n > s->cap_atoms) break;
      add.push_back(J);
      end += b;
      atoms += J->n;
    }
  }
  for (Job *J : add) {
    const size_t o = s->pre_off.back();
    write_block(s->hpre + o, *J);
    s->pre_jobs.push_back(J);
    s->pre_off.push_back(o + block_doubles(J->n) * sizeof(double));
  }
}

void fail_all(tersoff_server *s, int code)
{
  std::lock_guard<std::mutex> lk(s->mu);
  s->msg = s->priv.err;
  for (Job *&jp : s->slot_job) {
    if (!jp) continue;
    Job &J = *jp;
    J.state = 3;
    J.err = code;
    J.t_done = now_s();
    J.slot = -1;
    s->stats.failed += 1;
    s->stats.running -= 1;
    jp = nullptr;
  }
  for (Job *jp : s->pending) {
    jp->state = 3;
    jp->err = code;
    jp->t_done = now_s();
    s->stats.failed += 1;
    s->stats.running -= 1;
  }
  s->pending.clear();
  s->pre_jobs.clear();
  s->pre_off.clear();
  s->nres = 0;
  s->live = 0;
  s->hw = 0;
  s->broken = true;
  s->cv_done.notify_all();
}

// Places the admitted jobs `fresh` (slots, offsets, step control) and applies the
// layout: in place when every job fits a free range and freed atoms stay below
// the compaction threshold, else compacted.
int admit(tersoff_server *s, const std::vector<Job *> &fresh)
{
  std::vector<std::pair<int64_t, int64_t>> ranges;
  for (Job *J : resident(s)) ranges.push_back({J->off, J->n});
  std::sort(ranges.begin(), ranges.end());
  bool compacted = false;
  int64_t live = 0, hw = 0;
  for (auto &r : ranges) live += r.second;
  for (Job *J : fresh) {
    const int64_t off = place(ranges, J->n, s->cap_atoms);
    if (off < 0) {
      compacted = true;
      break;
    }
    J->off = off;
    live += J->n;
  }
  if (!compacted) {
    for (auto &r : ranges) hw = std::max(hw, r.first + r.second);
    compacted = !fresh.empty() && hw - live >= s->compact_min && (double)(hw - live) > s->compact_frac * hw;
  }
  std::vector<Job *> surv;
  std::vector<int64_t> old_off;
  if (compacted) {
    surv = resident(s);
    std::sort(surv.begin(), surv.end(), [](const Job *a, const Job *b) { return a->off < b->off; });
    int64_t off = 0;
    for (Job *J : surv) {
      old_off.push_back(J->off);
      J->off = off;
      off += J->n;
    }
    for (Job *J : fresh) {
      J->off = off;
      off += J->n;
    }
  }
  int k = 0;
  for (Job *J : fresh) {
    while (s->slot_job[k]) ++k;
    s->slot_job[k] = J;
    J->slot = k;
    J->ctl = SysCtl{J->nsteps, 0, 0};
  }
  return apply_layout(s, fresh, surv, old_off, compacted);
}

void worker_loop(tersoff_server *s)
{
  cudaSetDevice(s->ctx->device);
  double busy_since = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty() || s->nres > 0; });
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
    // retire finished jobs (their results reach them while the next chunk runs)
    double t0 = now_s();
    int rc = retire(s);
    s->w_retire += now_s() - t0;
    if (rc != TERSOFF_OK) {
      fail_all(s, rc);
      continue;
    }
    std::vector<Job *> fresh;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const double t = now_s();
      s->stats.chunks = s->w_chunks;
      s->stats.repacks = s->w_repacks;
      s->stats.compactions = s->w_compactions;
      s->stats.layout_fill = s->w_hw > 0 ? s->w_live / s->w_hw : 1.0;
      s->stats.retire_s = s->w_retire;
      s->stats.repack_s = s->w_repack;
      s->stats.graph_s = s->w_graph;
      s->stats.run_s = s->w_run;
      int nres = 0;
      int64_t atoms = 0;
      for (const Job *J : s->slot_job)
        if (J) {
          ++nres;
          atoms += J->n;
        }
      // admit queued jobs in arrival order while slots and atom capacity allow
      while (!s->queue.empty()) {
        Job &J = *s->jobs.at(s->queue.front());
        if (nres + (int)fresh.size() >= s->max_slots || atoms + J.n > s->cap_atoms) break;
        s->queue.pop_front();
        J.state = 1;
        J.t_admit = t;
        fresh.push_back(&J);
        atoms += J.n;
        s->stats.admitted += 1;
        s->stats.queued -= 1;
        s->stats.running += 1;
      }
    }
    if (!s->pending.empty() || !fresh.empty()) {
      t0 = now_s();
      rc = admit(s, fresh);
      s->w_repack += now_s() - t0;
      if (rc != TERSOFF_OK) {
        fail_all(s, rc);
        continue;
      }
    }
    // nothing left to integrate (all resident jobs finished): retire without stepping
    bool active = false;
    for (const Job *J : s->slot_job)
      if (J && (J->ctl.steps_left > 0 || J->ctl.open)) active = true;
    double g0 = s->w_graph;
    t0 = now_s();
    if (active) {
      s->w_hw += (double)s->hw;
      s->w_live += (double)s->live;
      rc = chunk_launch(s);
      if (rc != TERSOFF_OK) {
        fail_all(s, rc);
        continue;
      }
    }
    // on the host while the chunk runs: results of the retired jobs, staging of the
    // next queued jobs
    const double tf = now_s();
    rc = finish_retire(s);
    if (rc != TERSOFF_OK) {
      fail_all(s, rc);
      continue;
    }
    prestage(s);
    if (!active) s->w_retire += now_s() - tf;
    if (s->nres == 0) {
      if (busy_since > 0) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.busy_s += now_s() - busy_since;
        busy_since = 0;
      }
      continue;
    }
    if (busy_since == 0) busy_since = t0;
    if (active) {
      rc = chunk_wait(s);
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
  s->compact_frac = FREED_COMPACT_FRAC;
  s->compact_min = FREED_COMPACT_MIN;
  if (const char *c = getenv("TERSOFF_COMPACT_FREED")) {
    // compact whenever freed atoms below the high-water mark pass this share of it
    s->compact_frac = std::max(0.0, atof(c));
    s->compact_min = 1;
  }
  s->cap_atoms = std::min<int64_t>((int64_t)(budget / bytes_per_atom(s->f32, s->listcap)), MAX_LIST_ATOMS);
  auto fail = [&](int rc) {
    tersoff_server_destroy(s);
    return rc;
  };
  if (s->cap_atoms < 1) return fail(set_err(ctx, TERSOFF_ERR_NOMEM, "budget below one atom"));
  s->tab.assign((size_t)max_slots + 1, SysTab{});
  s->slot_job.assign((size_t)max_slots, nullptr);
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
      ensure_list(pc, s->L, cap, s->listcap, 1) != TERSOFF_OK || !sys_alloc(s->S, max_slots + 1) ||
      cudaMalloc((void **)&s->eatom, sizeof(double) * cap) != cudaSuccess ||
      cudaMalloc((void **)&s->sysE, sizeof(double) * 2 * max_slots) != cudaSuccess ||
      cudaMalloc((void **)&s->dtabs, sizeof(int) * (size_t)TAB_INTS(s)) != cudaSuccess ||
      cudaMalloc((void **)&s->d_order, sizeof(int) * (size_t)(cap + route_pad(s))) != cudaSuccess ||
      cudaMalloc((void **)&s->d_order_new, sizeof(int) * (size_t)(cap + route_pad(s))) != cudaSuccess ||
      // the register-kernel queues cover the padded route orders
      !dreserve(s->SC.work, s->SC.work_b,
                (size_t)force_queue_blocks((int)(cap + route_pad(s))) * FAST_THREADS * sizeof(int)) ||
      !dreserve(s->SC.nwork, s->SC.nwork_b, (size_t)force_queue_blocks((int)(cap + route_pad(s))) * sizeof(int)) ||
      cudaMalloc((void **)&s->d_ncmax, sizeof(int) * (size_t)(max_slots + 1) * MAX_TYPES) != cudaSuccess) {
    cudaGetLastError();
    return fail(set_err(ctx, TERSOFF_ERR_NOMEM, "cannot allocate the packed layout for %lld atoms", (long long)cap));
  }
  if (cudaEventCreateWithFlags(&s->ev_res, cudaEventDisableTiming) != cudaSuccess)
    return fail(set_err(ctx, TERSOFF_ERR_CUDA, "event"));
  // staging of queued jobs while chunks run: about 30 MB of pinned memory (without
  // it, admissions stage every job themselves)
  pinned_reserve(s->hpre, s->hpre_b, (size_t)24 << 20);
  if (cudaHostAlloc((void **)&s->h_ncmax, sizeof(int) * (size_t)(max_slots + 1) * MAX_TYPES, cudaHostAllocDefault) !=
      cudaSuccess)
    return fail(set_err(ctx, TERSOFF_ERR_NOMEM, "pinned counts"));
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
  J->one_species = std::all_of(J->types.begin(), J->types.end(), [&](int32_t t) { return t == J->types[0]; });
  for (int64_t i = 0; i < n; ++i) J->tcount[J->types[i]] += 1;
  if (!J->one_species) {
    // atoms grouped by type (stable): the register kernel reads whole rows of the
    // per-atom arrays; results go back to the caller's order
    std::vector<int> perm;
    perm.reserve((size_t)n);
    for (int t = 0; t < s->P->nt; ++t)
      for (int64_t i = 0; i < n; ++i)
        if (J->types[i] == t) perm.push_back((int)i);
    std::vector<double> p(3 * n), v(3 * n);
    std::vector<int32_t> ty(n);
    for (int64_t k = 0; k < n; ++k) {
      const int64_t i = perm[k];
      for (int a = 0; a < 3; ++a) {
        p[3 * k + a] = J->pos[3 * i + a];
        v[3 * k + a] = J->vel[3 * i + a];
      }
      ty[k] = J->types[i];
    }
    J->pos.swap(p);
    J->vel.swap(v);
    J->types.swap(ty);
    J->perm.swap(perm);
  }
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
  dfree(s->d_order_new);
  dfree(s->d_ncmax);
  dfree(s->rstage);
  if (s->hstage) cudaFreeHost(s->hstage);
  if (s->hres) cudaFreeHost(s->hres);
  if (s->hpre) cudaFreeHost(s->hpre);
  if (s->h_ncmax) cudaFreeHost(s->h_ncmax);
  if (s->ev_res) cudaEventDestroy(s->ev_res);
  if (s->st) cudaStreamDestroy(s->st);
  if (s->cap_st) cudaStreamDestroy(s->cap_st);
  tersoff_ctx *ctx = s->ctx;
  delete s;
  if (ctx) ctx_release(ctx);
}

}  // extern "C"
