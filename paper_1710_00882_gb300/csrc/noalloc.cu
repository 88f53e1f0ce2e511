// tersoff_compute_noalloc: one energy + force + virial evaluation whose working
// buffers all live in a fixed device array compiled into the library, so the call
// allocates no device memory.
//
// Who needs it: host code that may not call cudaMalloc/cudaFree at the point where
// it evaluates forces.  Typical cases are a program that embeds this library next to
// a framework whose caching allocator already reserved the device's memory (a raw
// cudaMalloc there fails, or forces the framework to release its pool), and a
// latency-critical loop where cudaMalloc/cudaFree would synchronize the device.
// Such callers still create the parameter table once, at set-up time, and own every
// input and output buffer.
//
// The array `g_scratch` holds, for at most TERSOFF_NOALLOC_MAX_ATOMS atoms, the run
// status word, one system table, the fixed-point positions, the cell arrays (at most
// TERSOFF_NOALLOC_MAX_CELLS cells), a neighbour list of TERSOFF_NOALLOC_MAX_NEIGHBORS
// entries per atom and the force kernel's per-slot contributions.  Host code cannot
// use the symbol as a device address: the first call on each device looks the
// address up with cudaGetSymbolAddress, with that device current, and keeps it.
// All calls on a device share the array and find the previous call's contents in it;
// every call clears the parts that must start at zero (status word, cell counts).
// Calls whose GPU work may overlap (several host threads, or unordered streams) race
// on the array and must be serialized by the caller.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "runtime.h"

namespace {

using namespace tsf;

constexpr int64_t kMaxAtoms = TERSOFF_NOALLOC_MAX_ATOMS;
constexpr int kCap = TERSOFF_NOALLOC_MAX_NEIGHBORS;
constexpr int kMaxCells = TERSOFF_NOALLOC_MAX_CELLS;
constexpr size_t kTileBytes = 4096;   // scan tile sums: >= 4 * tiles of kMaxCells cells + 16

constexpr size_t up256(size_t b) { return (b + 255) / 256 * 256; }

// Byte offsets of the regions of the scratch array (contributions sized for float64).
struct Layout {
  static constexpr size_t rs = 0;
  static constexpr size_t sys = rs + up256(sizeof(RunState));
  static constexpr size_t x = sys + up256(sizeof(SysTab));
  static constexpr size_t q = x + up256(kMaxAtoms * sizeof(dbl4));
  static constexpr size_t qref = q + up256(kMaxAtoms * sizeof(int4));
  static constexpr size_t nbr = qref + up256(kMaxAtoms * sizeof(int4));
  static constexpr size_t rev = nbr + up256(kMaxAtoms * kCap * sizeof(int));
  static constexpr size_t cnt = rev + up256(kMaxAtoms * kCap * sizeof(int));
  static constexpr size_t cell_atoms = cnt + up256(kMaxAtoms * sizeof(int));
  static constexpr size_t cell_of = cell_atoms + up256(kMaxAtoms * sizeof(int4));
  static constexpr size_t rank = cell_of + up256(kMaxAtoms * sizeof(int));
  static constexpr size_t cell_count = rank + up256(kMaxAtoms * sizeof(int));
  static constexpr size_t cell_start = cell_count + up256(kMaxCells * sizeof(int));
  static constexpr size_t tile_sums = cell_start + up256((kMaxCells + 1) * sizeof(int));
  static constexpr size_t contrib = tile_sums + kTileBytes;
  static constexpr size_t selfF = contrib + up256(kMaxAtoms * kCap * sizeof(dbl4));
  static constexpr size_t mask = selfF + up256(kMaxAtoms * sizeof(dbl4));
  static constexpr size_t work = mask + up256(kMaxAtoms * sizeof(unsigned long long));
  // overflow queues: force_queue_blocks(N) = ceil(N / 128) + 2 blocks of 128 entries
  static constexpr size_t queue_blocks = (kMaxAtoms + 127) / 128 + 2;
  static constexpr size_t nwork = work + up256(queue_blocks * 128 * sizeof(int));
  static constexpr size_t partial = nwork + up256(queue_blocks * sizeof(int));
  // force_partial_rows(N) = ceil(N / 32) + 2 + GEN_BLOCKS rows of 8 float64
  static constexpr size_t partial_rows = (kMaxAtoms + 31) / 32 + 2 + GEN_BLOCKS;
  static constexpr size_t total = partial + up256(partial_rows * 8 * sizeof(double));
};

static_assert(Layout::total == TERSOFF_NOALLOC_SCRATCH_BYTES, "scratch size stated in tersoff.h is out of date");

// The fixed scratch array: every device that loads this module holds it until the
// process exits.
static __device__ __align__(256) unsigned char g_scratch[Layout::total];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

int fail(char *errbuf, size_t errlen, int code, const char *fmt, ...)
{
  if (errbuf && errlen) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(errbuf, errlen, fmt, ap);
    va_end(ap);
  }
  return code;
}

// Device address of g_scratch on the current device (looked up on first use).
int scratch_address(int dev, unsigned char **out, char *errbuf, size_t errlen)
{
  if (dev < 0 || dev >= kMaxDevices) return fail(errbuf, errlen, TERSOFF_ERR_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return fail(errbuf, errlen, TERSOFF_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_addr[dev] = (unsigned char *)p;
  }
  *out = g_addr[dev];
  return TERSOFF_OK;
}

}  // namespace

#define NK(call)                                                                                        \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return fail(errbuf, errlen, TERSOFF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" int tersoff_compute_noalloc(const tersoff_params *P, const double *pos, const int32_t *types, int64_t N,
                                       const double box[3], tersoff_precision prec, void *stream,
                                       double *energy_virial, double *forces, char *errbuf, size_t errlen)
{
  if (errbuf && errlen) errbuf[0] = '\0';
  if (!P || !box || N < 0 || (N > 0 && (!pos || !types)))
    return fail(errbuf, errlen, TERSOFF_ERR_ARG, "null argument or N < 0");
  if (prec != TERSOFF_FP64 && prec != TERSOFF_MIXED && prec != TERSOFF_SINGLE)
    return fail(errbuf, errlen, TERSOFF_ERR_ARG, "bad precision");
  if (N > kMaxAtoms)
    return fail(errbuf, errlen, TERSOFF_ERR_NOMEM,
                "N = %lld atoms exceeds the fixed scratch limit of %d atoms of tersoff_compute_noalloc",
                (long long)N, (int)kMaxAtoms);
  for (int a = 0; a < 3; ++a) {
    if (!(box[a] > 0) || !std::isfinite(box[a])) return fail(errbuf, errlen, TERSOFF_ERR_ARG, "box side %d not positive", a);
    if (box[a] < 2.0 * P->rcmax)
      return fail(errbuf, errlen, TERSOFF_ERR_BOX_TOO_SMALL, "box side %d = %g < 2*cutoff = %g", a, box[a],
                  2.0 * P->rcmax);
  }
  // cell grid with cells at least the cutoff wide, coarsened to fit the fixed cell arrays
  CellGrid g;
  make_grid(box, P->rcmax, &g);   // a grid over the cell limit is coarsened below
  g.radii = pair_radii(P, 0.0);
  while ((long long)g.nc[0] * g.nc[1] * g.nc[2] > kMaxCells) {
    int a = 0;
    for (int b = 1; b < 3; ++b)
      if (g.nc[b] > g.nc[a]) a = b;
    g.nc[a] = (g.nc[a] + 1) / 2;
  }
  g.ncell = g.nc[0] * g.nc[1] * g.nc[2];
  if ((size_t)scan_tiles_for(g.ncell) * sizeof(int) + 16 > kTileBytes ||
      (size_t)force_partial_rows((int)N) > Layout::partial_rows)
    return fail(errbuf, errlen, TERSOFF_ERR_NOMEM, "cell scan or partial sums do not fit the fixed scratch");

  int dev = 0;
  NK(cudaGetDevice(&dev));
  unsigned char *base = nullptr;
  int rc = scratch_address(dev, &base, errbuf, errlen);
  if (rc != TERSOFF_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = prec != TERSOFF_FP64;
  RunState *rs = (RunState *)(base + Layout::rs);
  SysTab *sys = (SysTab *)(base + Layout::sys);
  dbl4 *x = (dbl4 *)(base + Layout::x);
  int4 *q = (int4 *)(base + Layout::q);
  int4 *qref = (int4 *)(base + Layout::qref);
  int *nbr = (int *)(base + Layout::nbr), *rev = (int *)(base + Layout::rev), *cnt = (int *)(base + Layout::cnt);
  int4 *cell_atoms = (int4 *)(base + Layout::cell_atoms);
  int *cell_of = (int *)(base + Layout::cell_of);
  int *rank = (int *)(base + Layout::rank), *cell_count = (int *)(base + Layout::cell_count);
  int *cell_start = (int *)(base + Layout::cell_start), *tile_sums = (int *)(base + Layout::tile_sums);
  void *contrib = base + Layout::contrib, *selfF = base + Layout::selfF;
  unsigned long long *mask = (unsigned long long *)(base + Layout::mask);
  int *work = (int *)(base + Layout::work), *nwork = (int *)(base + Layout::nwork);
  double *partial = (double *)(base + Layout::partial);

  // what must start at zero: the status word / accumulators and the cell counts
  NK(cudaMemsetAsync(rs, 0, sizeof(RunState), st));
  NK(cudaMemsetAsync(cell_count, 0, (size_t)g.ncell * sizeof(int), st));
  if (N == 0) {
    if (energy_virial) NK(cudaMemsetAsync(energy_virial, 0, 7 * sizeof(double), st));
    NK(cudaStreamSynchronize(st));
    return TERSOFF_OK;
  }
  SysTab T{};
  T.geo = make_geom(box);
  for (int a = 0; a < 3; ++a) T.nc[a] = g.nc[a];
  T.cell_off = 0;
  T.atom_off = 0;
  T.natoms = (int)N;
  NK(cudaMemcpyAsync(sys, &T, sizeof(SysTab), cudaMemcpyHostToDevice, st));
  NK(launch_ingest(st, (int)N, pos, types, P->nt, 0, sys, x, q, rs));
  NK(launch_build(st, (int)N, (int)N, q, sys, nullptr, g.ncell, g.radii, cell_count, cell_start, tile_sums, cell_atoms, cell_of, rank,
                  nbr, rev, cnt, kCap, qref, rs, 0));
  const int fast_slots = P->sym_angular ? 8 : 0;
  NK(launch_force(st, prec, fast_slots, P->fast, force_slots_for(kCap), 1, 1, (int)N, x, q, nbr, cnt, sys,
                  f32 ? P->pair_f : P->pair_d, f32 ? P->trip_f : P->trip_d, P->nt, contrib, selfF, mask, work,
                  nwork, partial, rs, nullptr));
  if (forces) NK(launch_gather_out(st, prec, (int)N, contrib, selfF, mask, rev, forces, rs));
  if (energy_virial) {
    NK(cudaMemcpyAsync(energy_virial, &rs->epot, sizeof(double), cudaMemcpyDeviceToDevice, st));
    NK(cudaMemcpyAsync(energy_virial + 1, rs->virial, 6 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  RunState h;
  NK(cudaMemcpyAsync(&h, rs, sizeof(RunState), cudaMemcpyDeviceToHost, st));
  NK(cudaStreamSynchronize(st));
  if (h.status & ST_BAD_TYPE) return fail(errbuf, errlen, TERSOFF_ERR_ARG, "atom type out of range");
  if (h.status & ST_NLIST_OVERFLOW)
    return fail(errbuf, errlen, TERSOFF_ERR_NLIST_OVERFLOW,
                "%d neighbours within the cutoff exceed the fixed limit of %d per atom", h.maxcount, kCap);
  if (h.status & ST_NONFINITE) return fail(errbuf, errlen, TERSOFF_ERR_NONFINITE, "non-finite position, force or energy");
  if (h.status != 0) return fail(errbuf, errlen, TERSOFF_ERR_CUDA, "device status %d", h.status);
  if (!std::isfinite(h.epot)) return fail(errbuf, errlen, TERSOFF_ERR_NONFINITE, "non-finite energy");
  return TERSOFF_OK;
}
