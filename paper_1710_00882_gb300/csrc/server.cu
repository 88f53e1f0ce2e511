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

// Rewrite the system index in every atom word from the table's atom ranges.
__global__ void k_resid(int N, int4 *__restrict__ q, dbl4 *__restrict__ x, const SysTab *__restrict__ sys, int nsys)
{
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sys[mid].atom_off <= i) lo = mid; else hi = mid - 1;
  }
  const int w = make_w(type_of(q[i].w), lo);
  q[i].w = w;
  x[i].w = __longlong_as_double((long long)w);
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
  bool mixed = false;
  double skin = 0, rl = 0;
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
  double *stage = nullptr;
  size_t stage_b = 0;
  std::vector<SysTab> tab;
  std::vector<Job *> batch;      // resident jobs in layout order (owned by `jobs`; touched by the worker only)
  int64_t natoms = 0;
  int ncell = 0;
  int fast_slots = 8, gen_slots = 32;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;
  bool broken = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  tersoff_server_stats stats{};
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

size_t bytes_per_atom(bool mixed, int listcap)
{
  const size_t v4 = mixed ? 16 : 32;
  return 2 * (32 + 32 + 16)                        // two copies of x, v, q
         + (size_t)listcap * (v4 + 8)              // contrib + nbr/rev
         + v4 + 8 + 8 + 4 + 16 + 12 + 8 + 16;      // selfF, mask, work, cnt, qref, cells, eatom, slack
}

// staging bytes of one new job (positions, velocities, types), 256-byte aligned
size_t stage_bytes(int64_t n) { return ((size_t)n * (6 * sizeof(double) + sizeof(int32_t)) + 255) / 256 * 256; }

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
  SK(launch_force(st, s->mixed, s->fast_slots, P->nt == 1, s->gen_slots, 0, 0, (int)s->natoms, X.x, X.q, s->L.nbr,
                  s->L.cnt, s->S.tab, s->mixed ? P->pair_f : P->pair_d, s->mixed ? P->trip_f : P->trip_d, P->nt,
                  s->SC.contrib, s->SC.selfF, s->SC.mask, s->SC.work, s->SC.nwork, s->SC.partial, s->rs, s->eatom));
  return TERSOFF_OK;
}

int srv_vv(tersoff_server *s, cudaStream_t st)
{
  AtomState &X = cur_atoms(s);
  const float lim = (float)(0.25 * s->skin * s->skin);
  SK(launch_vv(st, s->mixed, false, (int)s->natoms, -1, X.x, X.v, X.q, s->L.qref, s->SC.contrib, s->SC.selfF,
               s->SC.mask, s->L.rev, s->S.tab, s->S.ctl, s->P->d_mass, lim, s->SC.kepart, s->rs));
  return TERSOFF_OK;
}

int srv_build(tersoff_server *s, cudaStream_t st, int gated)
{
  AtomState &X = cur_atoms(s);
  ListState &L = s->L;
  SK(launch_build(st, (int)s->natoms, X.q, s->S.tab, s->ncell, (float)(s->rl * s->rl * (1.0 + 1e-5)), L.cell_count,
                  L.cell_start, L.tile_sums, L.cell_atoms, L.cell_of, L.rank, L.nbr, L.rev, L.cnt, L.cap, L.qref,
                  s->rs, gated));
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

// loop_begin -> WHILE { vv -> decide -> IF(rebuild) { build } -> force -> step_end }
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
  SK(launch_loop_begin(st, s->rs, hloop));
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *edges = nullptr;
  size_t nd = 0;
  SK(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, &edges, &nd));
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
  SKR(srv_build(s, st, 0));
  cudaGraph_t ifc = ifbody;
  SK(cudaStreamEndCapture(st, &ifc));
  SK(cudaGraphInstantiate(&s->exec, g, 0));
  s->graph_ok = true;
  return TERSOFF_OK;
}

// Full list build of the current layout, growing the list capacity within the
// budget on overflow.
int build_sync(tersoff_server *s)
{
  for (int attempt = 0; attempt < 3; ++attempt) {
    SK(cudaMemsetAsync(&s->rs->maxcount, 0, sizeof(int), s->st));
    SKR(srv_build(s, s->st, 0));
    RunState h;
    SKR(read_state(s, &h));
    if (h.status == 0) return TERSOFF_OK;
    if (h.status != ST_NLIST_OVERFLOW || h.maxcount > MAX_CAP)
      return srv_err(s, TERSOFF_ERR_NLIST_OVERFLOW, "list build failed (status %d, %d entries)", h.status, h.maxcount);
    const int cap = std::min(MAX_CAP, ((h.maxcount + std::max(4, h.maxcount / 4)) + 3) & ~3);
    graph_free(s);
    if (ensure_list(&s->priv, s->L, s->cap_atoms, cap, std::max(1, s->ncell)) != TERSOFF_OK ||
        ensure_scatter(&s->priv, s->SC, s->cap_atoms, cap, s->mixed) != TERSOFF_OK)
      return srv_err(s, TERSOFF_ERR_NOMEM, "cannot grow neighbour lists to %d entries", cap);
    s->listcap = cap;
    SK(cudaMemsetAsync(&s->rs->status, 0, sizeof(int), s->st));
  }
  return srv_err(s, TERSOFF_ERR_NLIST_OVERFLOW, "list build did not converge");
}

// Rebuild the packed layout from the jobs in `order` (survivors first, then new).
int repack(tersoff_server *s, const std::vector<Job *> &order, const std::vector<bool> &is_new)
{
  const tersoff_params *P = s->P;
  std::vector<SysTab> tab(order.size());
  std::vector<SysCtl> ctl(order.size());
  std::vector<int64_t> old_off(order.size(), -1);
  std::map<const Job *, int64_t> prev;
  for (size_t k = 0; k < s->batch.size(); ++k) prev[s->batch[k]] = s->tab[k].atom_off;
  int64_t off = 0;
  int coff = 0;
  for (size_t k = 0; k < order.size(); ++k) {
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
    if (!is_new[k]) old_off[k] = prev[order[k]];
    off += J.n;
    coff += gr.ncell;
  }
  s->natoms = off;
  s->ncell = coff;
  if (!sys_alloc(s->S, std::max(1, (int)order.size()))) return srv_err(s, TERSOFF_ERR_NOMEM, "system tables");
  if (ensure_list(&s->priv, s->L, s->cap_atoms, s->listcap, std::max(1, coff)) != TERSOFF_OK)
    return srv_err(s, TERSOFF_ERR_NOMEM, "cell arrays for %d cells", coff);
  SK(cudaMemcpyAsync(s->S.tab, tab.data(), sizeof(SysTab) * tab.size(), cudaMemcpyHostToDevice, s->st));
  SK(cudaMemcpyAsync(s->S.ctl, ctl.data(), sizeof(SysCtl) * ctl.size(), cudaMemcpyHostToDevice, s->st));
  AtomState &src = s->A[s->cur];
  AtomState &dst = s->A[1 - s->cur];
  // survivors: copy their ranges; new jobs: stage and ingest
  size_t need = 0;
  for (size_t k = 0; k < order.size(); ++k)
    if (is_new[k]) need += stage_bytes(order[k]->n);
  if (need && !dreserve(s->stage, s->stage_b, need)) return srv_err(s, TERSOFF_ERR_NOMEM, "staging");
  char *sp = (char *)s->stage;
  for (size_t k = 0; k < order.size(); ++k) {
    Job &J = *order[k];
    const int64_t o = tab[k].atom_off;
    if (!is_new[k]) {
      const int64_t p = old_off[k];
      SK(cudaMemcpyAsync(dst.x + o, src.x + p, sizeof(dbl4) * J.n, cudaMemcpyDeviceToDevice, s->st));
      SK(cudaMemcpyAsync(dst.v + o, src.v + p, sizeof(dbl4) * J.n, cudaMemcpyDeviceToDevice, s->st));
      SK(cudaMemcpyAsync(dst.q + o, src.q + p, sizeof(int4) * J.n, cudaMemcpyDeviceToDevice, s->st));
    } else {
      double *dpos = (double *)sp;
      double *dvel = dpos + 3 * J.n;
      int32_t *dty = (int32_t *)(dvel + 3 * J.n);
      sp += stage_bytes(J.n);
      SK(cudaMemcpyAsync(dpos, J.pos.data(), sizeof(double) * 3 * J.n, cudaMemcpyHostToDevice, s->st));
      SK(cudaMemcpyAsync(dvel, J.vel.data(), sizeof(double) * 3 * J.n, cudaMemcpyHostToDevice, s->st));
      SK(cudaMemcpyAsync(dty, J.types.data(), sizeof(int32_t) * J.n, cudaMemcpyHostToDevice, s->st));
      SK(launch_ingest(s->st, (int)J.n, dpos, dty, P->nt, (int)k, s->S.tab, dst.x + o, dst.q + o, s->rs));
      SK(launch_ingest_vel(s->st, (int)J.n, dvel, dst.v + o));
    }
  }
  if (s->natoms > 0) {
    k_resid<<<(int)((s->natoms + 255) / 256), 256, 0, s->st>>>((int)s->natoms, dst.q, dst.x, s->S.tab,
                                                              (int)order.size());
    SK(cudaGetLastError());
  }
  s->cur = 1 - s->cur;
  s->tab = tab;
  s->batch = order;
  graph_free(s);
  SKR(build_sync(s));
  SKR(srv_force(s, s->st));
  RunState h;
  SKR(read_state(s, &h));
  if (h.status != 0) return srv_err(s, TERSOFF_ERR_CUDA, "force after repack: status %d", h.status);
  s->stats.repacks += 1;
  return TERSOFF_OK;
}

// One chunk of steps for the whole batch (recovering from list or slot overflow).
int run_chunk(tersoff_server *s)
{
  if (!s->graph_ok) SKR(graph_build(s));
  k_set_loop<<<1, 1, 0, s->st>>>(s->rs, s->chunk);
  SK(cudaGetLastError());
  SK(cudaGraphLaunch(s->exec, s->st));
  for (int attempt = 0; attempt < 8; ++attempt) {
    RunState h;
    SKR(read_state(s, &h));
    if (h.status == 0) break;
    if (h.status & ST_NLIST_OVERFLOW) {
      SK(cudaMemsetAsync(&s->rs->status, 0, sizeof(int), s->st));
      SKR(build_sync(s));
    } else if (h.status & ST_NC_OVERFLOW) {
      if (h.maxnc > MAX_CAP) return srv_err(s, TERSOFF_ERR_NLIST_OVERFLOW, "%d in-cutoff neighbours", h.maxnc);
      s->gen_slots = force_slots_for(h.maxnc);
      graph_free(s);
      SK(cudaMemsetAsync(&s->rs->status, 0, sizeof(int), s->st));
    } else {
      return srv_err(s, h.status & ST_NONFINITE ? TERSOFF_ERR_NONFINITE : TERSOFF_ERR_CUDA, "device status %d",
                     h.status);
    }
    // finish the failed step (its integrator part ran), then the rest of the chunk
    SK(cudaMemsetAsync(&s->rs->epot, 0, sizeof(double), s->st));
    SKR(srv_force(s, s->st));
    SK(launch_step_end(s->st, s->rs, s->S.ctl, (int)s->batch.size(), 0, 0));
    const long long rest = h.steps_left - 1;
    if (rest > 0) {
      if (!s->graph_ok) SKR(graph_build(s));
      k_set_loop<<<1, 1, 0, s->st>>>(s->rs, rest);
      SK(cudaGetLastError());
      SK(cudaGraphLaunch(s->exec, s->st));
    }
  }
  s->stats.chunks += 1;
  return TERSOFF_OK;
}

// Copy results of jobs whose run is over (steps done, closing kick applied).
int retire(tersoff_server *s, std::vector<Job *> &done)
{
  const size_t S = s->batch.size();
  if (!S) return TERSOFF_OK;
  std::vector<SysCtl> ctl(S);
  SK(cudaMemcpyAsync(ctl.data(), s->S.ctl, sizeof(SysCtl) * S, cudaMemcpyDeviceToHost, s->st));
  SK(cudaStreamSynchronize(s->st));
  bool any = false;
  for (size_t k = 0; k < S; ++k) {
    Job &J = *s->batch[k];
    J.ctl = ctl[k];
    if (ctl[k].steps_left == 0 && ctl[k].open == 0) any = true;
  }
  if (!any) return TERSOFF_OK;
  AtomState &X = cur_atoms(s);
  k_sys_energy<<<(int)S, 256, 0, s->st>>>(s->eatom, X.v, X.q, s->P->d_mass, s->S.tab, s->sysE);
  SK(cudaGetLastError());
  std::vector<double> E(2 * S);
  SK(cudaMemcpyAsync(E.data(), s->sysE, sizeof(double) * 2 * S, cudaMemcpyDeviceToHost, s->st));
  for (size_t k = 0; k < S; ++k) {
    Job &J = *s->batch[k];
    if (!(J.ctl.steps_left == 0 && J.ctl.open == 0)) continue;
    const int64_t o = s->tab[k].atom_off;
    if (!dreserve(s->stage, s->stage_b, sizeof(double) * 6 * (size_t)J.n + 64))
      return srv_err(s, TERSOFF_ERR_NOMEM, "staging");
    double *dp = (double *)s->stage;
    double *dv = dp + 3 * J.n;
    SK(launch_extract(s->st, (int)J.n, X.x + o, X.v + o, dp, dv));
    J.rpos.resize(3 * J.n);
    J.rvel.resize(3 * J.n);
    SK(cudaMemcpyAsync(J.rpos.data(), dp, sizeof(double) * 3 * J.n, cudaMemcpyDeviceToHost, s->st));
    SK(cudaMemcpyAsync(J.rvel.data(), dv, sizeof(double) * 3 * J.n, cudaMemcpyDeviceToHost, s->st));
    SK(cudaStreamSynchronize(s->st));
    J.epot = E[2 * k];
    J.ekin = E[2 * k + 1];
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
    int rc = retire(s, done);
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
      } else if ((rc = repack(s, order, is_new)) != TERSOFF_OK) {
        s->batch = order;
        fail_all(s, rc);
        continue;
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
        s->stats.busy_s += now_s() - busy_since;
        busy_since = 0;
      }
      continue;
    }
    if (busy_since == 0) busy_since = now_s();
    if (active && (rc = run_chunk(s)) != TERSOFF_OK) fail_all(s, rc);
  }
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
      (prec != TERSOFF_FP64 && prec != TERSOFF_MIXED))
    return set_err(ctx, TERSOFF_ERR_ARG, "bad server arguments");
  cudaSetDevice(ctx->device);
  tersoff_server *s = new (std::nothrow) tersoff_server();
  if (!s) return TERSOFF_ERR_NOMEM;
  s->ctx = ctx;
  ctx->refs += 1;
  s->P = P;
  s->mixed = prec == TERSOFF_MIXED;
  s->skin = skin;
  s->rl = P->rcmax + skin;
  s->max_slots = max_slots;
  s->chunk = chunk_steps;
  s->listcap = 32;
  s->fast_slots = (P->sym_angular && !ctx->general_only) ? 8 : 0;
  s->gen_slots = 32;
  s->cap_atoms = (int64_t)(budget / bytes_per_atom(s->mixed, s->listcap));
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
      ensure_scatter(pc, s->SC, cap, s->listcap, s->mixed) != TERSOFF_OK ||
      ensure_list(pc, s->L, cap, s->listcap, 1) != TERSOFF_OK || !sys_alloc(s->S, max_slots) ||
      cudaMalloc((void **)&s->eatom, sizeof(double) * cap) != cudaSuccess ||
      cudaMalloc((void **)&s->sysE, sizeof(double) * 2 * max_slots) != cudaSuccess) {
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
  if (s->st) cudaStreamDestroy(s->st);
  if (s->cap_st) cudaStreamDestroy(s->cap_st);
  tersoff_ctx *ctx = s->ctx;
  delete s;
  if (ctx) ctx_release(ctx);
}

}  // extern "C"
