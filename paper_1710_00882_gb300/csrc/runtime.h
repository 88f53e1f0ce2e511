// Host-side state structs of the runtime (not part of the C ABI).
#pragma once
#include <cstddef>
#include <cstdint>

#include <string>
#include <vector>

#include "tersoff.h"
#include "internal.cuh"

namespace tsf {

// Device arrays of one set of atoms.
struct AtomState {
  int64_t N = 0;
  Geom geo{};
  dbl4 *x = nullptr;             // float64 positions, type in w (bits)
  dbl4 *v = nullptr;             // float64 velocities
  int4 *q = nullptr;                // 32-bit fixed-point positions, type in w
  void *contrib = nullptr;          // [cap][N] float4/dbl4 force contributions (force kernel -> gather)
  void *selfF = nullptr;            // [N] force of each atom's own terms on itself
  unsigned long long *mask = nullptr;  // [N] in-cutoff list slots
  int *work = nullptr;              // [ceil(N/128)*128] overflow atoms of the register force kernel
  int *nwork = nullptr;             // [ceil(N/128)] overflow count per block
  double *partial = nullptr;        // per-block (E, W[6]) partial sums
  double *kepart = nullptr;         // per-block kinetic-energy partial sums
  size_t x_b = 0, v_b = 0, q_b = 0, contrib_b = 0, selfF_b = 0, mask_b = 0, work_b = 0, nwork_b = 0, partial_b = 0,
         kepart_b = 0;
};

// Device arrays of one neighbour list and its cell grid.
struct ListState {
  int64_t N = 0;
  int cap = 0;        // slots per atom
  int maxcount = 0;   // longest list at the last host-visible build
  CellGrid grid{};
  Geom geo{};
  double cutoff = 0, skin = 0;
  int *nbr = nullptr, *rev = nullptr, *cnt = nullptr;
  int4 *qref = nullptr;
  int *cell_count = nullptr, *cell_start = nullptr, *tile_sums = nullptr, *cell_of = nullptr, *rank = nullptr;
  int4 *cell_atoms = nullptr;   // atoms in cell order: fixed-point position and index
  size_t nbr_b = 0, rev_b = 0, cnt_b = 0, qref_b = 0, cell_count_b = 0, cell_start_b = 0, tile_sums_b = 0,
         cell_atoms_b = 0, cell_of_b = 0, rank_b = 0;
};

// One system's device-side table and run control (the single-system paths use
// system 0 of a one-entry table; packed layouts use many).
struct SysDev {
  SysTab host{};            // host copy of the table entries
  SysTab *tab = nullptr;    // device [cap]
  SysCtl *ctl = nullptr;    // device [cap]
  int cap = 0;
};

}  // namespace tsf

namespace tsf {

// launchers defined in the kernel translation units
cudaError_t launch_build(cudaStream_t, int, int, const int4 *, const SysTab *, const SysCtl *, int, const PairRadii &, int *, int *,
                         int *, int4 *, int *, int *, int *, int *, int *, int, int4 *, RunState *, int, int *raw = nullptr,
                         int *rawcnt = nullptr);
int scan_tiles_for(int ncell);
int force_slots_for(int need);
int force_partial_rows(int N);
int vv_blocks(int N);
cudaError_t launch_force(cudaStream_t, int, int, const FastTab &, int, int, int, int, const dbl4 *, const int4 *, const int *,
                         const int *, const SysTab *, const void *, const void *, int, void *, void *,
                         unsigned long long *, int *, int *, double *, RunState *, double *);
cudaError_t launch_force_part(int, cudaStream_t, int, int, const FastTab &, int, int, int, int, int, const dbl4 *,
                              const int4 *,
                              const int *, const int *, const SysTab *, const void *, const void *, int, void *, void *,
                              unsigned long long *, int *, int *, double *, RunState *, double *,
                              const ForceRoutes *routes = nullptr, int stats = 1);
int force_queue_blocks(int N);
cudaError_t launch_vv(cudaStream_t, int, bool, int, int, int, dbl4 *, dbl4 *, int4 *, const int4 *, const void *,
                      const void *, const unsigned long long *, const int *, const SysTab *, SysCtl *,
                      const double *, float, double *, RunState *);
cudaError_t launch_permute_atoms(cudaStream_t, int, const int *, const dbl4 *, const dbl4 *, const int4 *, dbl4 *,
                                 dbl4 *, int4 *);
cudaError_t launch_gather_out(cudaStream_t, int, int, const void *, const void *, const unsigned long long *,
                              const int *, double *, RunState *, const int *perm = nullptr);
cudaError_t launch_ingest(cudaStream_t, int, const double *, const int *, int, int, const SysTab *, dbl4 *, int4 *,
                          RunState *);
cudaError_t launch_ingest_vel(cudaStream_t, int, const double *, dbl4 *);
cudaError_t launch_extract(cudaStream_t, int, const dbl4 *, const dbl4 *, double *, double *,
                           const int *perm = nullptr);
cudaError_t launch_step_end(cudaStream_t, RunState *, SysCtl *, int, cudaGraphConditionalHandle, int);
cudaError_t launch_loop_start(cudaStream_t, RunState *, SysCtl *, long long, double *, long long, int,
                              cudaGraphConditionalHandle);
cudaError_t set_loop_start(cudaGraphExec_t, cudaGraphNode_t, RunState *, SysCtl *, long long, double *, long long, int,
                           cudaGraphConditionalHandle);
cudaError_t launch_decide(cudaStream_t, RunState *, cudaGraphConditionalHandle);
cudaError_t launch_set_control(cudaStream_t, RunState *, SysCtl *, long long, double *, long long, int);
cudaError_t set_control_node(cudaGraphExec_t, cudaGraphNode_t, RunState *, SysCtl *, long long, double *, long long,
                             int);
cudaError_t launch_final(cudaStream_t, RunState *, SysCtl *);
cudaError_t launch_force_done(cudaStream_t, RunState *);


template <class T>
inline void dfree(T *&p)
{
  if (p) cudaFree((void *)p);
  p = nullptr;
}

// (re)allocate p to hold at least `bytes`; contents are not kept
template <class T>
inline bool dreserve(T *&p, size_t &have, size_t bytes)
{
  if (bytes <= have && p) return true;
  dfree(p);
  have = 0;
  if (bytes == 0) bytes = 16;
  void *q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  p = (T *)q;
  have = bytes;
  return true;
}


Geom make_geom(const double box[3]);
int make_grid(const double box[3], double rl, CellGrid *g);
PairRadii uniform_radii(double rl);
bool sys_alloc(SysDev &S, int cap);
void sys_free(SysDev &S);
void free_atoms(AtomState &A);
void free_list(ListState &L);

}  // namespace tsf

using tsf::AtomState;
using tsf::ListState;
using tsf::SysDev;

struct tersoff_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  tsf::AtomState cstate;        // scratch state of tersoff_compute
  tsf::SysDev csys;             // its system table
  tsf::ListState clist;         // internal list of tersoff_compute when none is given
  tsf::RunState *crs = nullptr; // run state of tersoff_compute
  void *stage = nullptr;   // host-pointer staging (AoS positions/forces, types)
  size_t stage_bytes = 0;
  bool general_only = false;  // TERSOFF_FORCE_KERNEL=general: skip the register force kernel
  int refs = 1;               // the caller's handle plus one per live list / MD state
  bool destroyed = false;     // tersoff_ctx_destroy called; freed when refs reaches 0
};

struct tersoff_params {
  int nt = 0;
  std::vector<double> entries;
  double masses[tsf::MAX_TYPES] = {0, 0, 0, 0};
  double rcmax = 0;
  void *pair_f = nullptr, *trip_f = nullptr, *pair_d = nullptr, *trip_d = nullptr;
  double *d_mass = nullptr;
  bool sym_angular = false;   // rows (i,j,k) and (i,k,j) share their angular constants
  tsf::FastTab fast;          // the register force kernel's table kind and kernel-argument copies
};


namespace tsf {
int set_err(tersoff_ctx *ctx, int code, const char *fmt, ...);
int cuda_err(tersoff_ctx *ctx, cudaError_t e, const char *what);
int status_to_code(tersoff_ctx *ctx, int st, const RunState &h);
int new_rs(tersoff_ctx *ctx, RunState **rs);
int ensure_atoms(tersoff_ctx *ctx, AtomState &A, int64_t N, bool need_v);
int ensure_scatter(tersoff_ctx *ctx, AtomState &A, int64_t N, int cap, bool f32);
int ensure_list(tersoff_ctx *ctx, ListState &L, int64_t N, int cap, int ncell);
int check_box(tersoff_ctx *ctx, const double box[3], double rl);
PairRadii pair_radii(const tersoff_params *P, double skin);
void ctx_release(tersoff_ctx *ctx);   // drops one reference; frees the context at zero
}  // namespace tsf
