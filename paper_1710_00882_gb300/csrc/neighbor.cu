// Cell-list / Verlet neighbour build with skin (the list the paper's Sec. 3
// packing works on).  Everything here runs on 32-bit fixed-point positions:
// the minimum image is the int32 difference of two fixed-point coordinates, so
// the list is exactly symmetric (j in list(i) <=> i in list(j)) and needs no
// float64 arithmetic.
//
// Build sequence (all launches are skipped on the device unless rs->rebuild is
// set, so an MD step can enqueue them unconditionally):
//   k_cell_count  -> cell of each atom of a system that gets new lists, rank inside
//                    its cell (atomic)
//   k_scan_*      -> exclusive scan of the cell counts (three-phase block scan)
//   k_cell_fill   -> atoms in cell order
//   k_build       -> per atom: half stencil, each pair within its type pair's list
//                    radius r_C(ti,tj) + skin appended to both lists
//   k_sort_lists  -> each list sorted by j; overflow check
//   k_reverse     -> for each entry (i,s) the flat index of i's slot in j's list
//   (k_sort_reverse does both in one kernel when the caller gives scratch for the
//   raw lists and the lists hold at most 16 slots)
#include "internal.cuh"

namespace tsf {

__device__ __forceinline__ bool skip_build(const RunState *rs, int gated)
{
  return rs->status != 0 || (gated && rs->rebuild == 0);
}

__device__ __forceinline__ int cell_coord(uint32_t qa, int nc)
{
  return (int)(((unsigned long long)qa * (unsigned long long)nc) >> 32);
}

// Each atom's cell in its own system's grid, numbered globally (system cell offset
// + local cell), and its rank inside the cell.
__global__ void k_cell_count(int N, const int4 *__restrict__ q, const SysTab *__restrict__ sys,
                             const SysCtl *__restrict__ ctl, int *__restrict__ cell_of, int *__restrict__ rank,
                             int *__restrict__ cell_count, int *__restrict__ cnt, const RunState *rs, int gated)
{
  if (skip_build(rs, gated)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int4 p = q[i];
  const SysTab &T = sys[sys_of(p.w)];
  // only the systems that get new lists take cells (atoms of a freed range of a
  // packed layout, a system without atoms, never do); their list counts start at
  // zero (pairs are appended)
  if (T.natoms == 0 || (ctl && ctl[sys_of(p.w)].rebuild == 0)) {
    cell_of[i] = -1;
    return;
  }
  cnt[i] = 0;
  int cx = cell_coord((uint32_t)p.x, T.nc[0]);
  int cy = cell_coord((uint32_t)p.y, T.nc[1]);
  int cz = cell_coord((uint32_t)p.z, T.nc[2]);
  int c = T.cell_off + (cz * T.nc[1] + cy) * T.nc[0] + cx;
  cell_of[i] = c;
  rank[i] = atomicAdd(&cell_count[c], 1);
}

// ---- exclusive scan over n ints: SCAN_ITEMS per thread, SCAN_THREADS per block
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int block_exclusive_scan(int v, int *total)
{
  __shared__ int warp_sums[SCAN_THREADS / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < SCAN_THREADS / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  int prefix = (w > 0 ? warp_sums[w - 1] : 0) + x - v;
  *total = warp_sums[SCAN_THREADS / 32 - 1];
  __syncthreads();
  return prefix;
}

// phase 1: scan each tile, write tile totals
__global__ void k_scan_tiles(int n, const int *__restrict__ in, int *__restrict__ out, int *__restrict__ tile_sums,
                             const RunState *rs, int gated)
{
  griddep_wait();
  if (skip_build(rs, gated)) return;
  int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS], s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  int total;
  int pre = block_exclusive_scan(s, &total);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// phase 2: one block scans the tile totals (sequentially over chunks of SCAN_TILE)
__global__ void k_scan_sums(int ntiles, int *__restrict__ tile_sums, int *__restrict__ grand_total,
                            const RunState *rs, int gated)
{
  griddep_wait();
  if (skip_build(rs, gated)) return;
  int carry = 0;
  for (int base = 0; base < ntiles; base += SCAN_TILE) {
    int b = base + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      v[k] = b + k < ntiles ? tile_sums[b + k] : 0;
      s += v[k];
    }
    int total;
    int pre = block_exclusive_scan(s, &total) + carry;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      if (b + k < ntiles) tile_sums[b + k] = pre;
      pre += v[k];
    }
    carry += total;
  }
  if (threadIdx.x == 0) *grand_total = carry;
}

// phase 3: add tile offsets; zero the counts for the next build
__global__ void k_scan_add(int n, int *__restrict__ out, const int *__restrict__ tile_sums, int *__restrict__ counts,
                           const RunState *rs, int gated)
{
  griddep_wait();
  if (skip_build(rs, gated)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] += tile_sums[i / SCAN_TILE];
  counts[i] = 0;
}

// atoms in cell order, each with its fixed-point position and its type: the stencil
// scan of k_build then reads candidates as contiguous runs
__global__ void k_cell_fill(int N, const int4 *__restrict__ q, const int *__restrict__ cell_of,
                            const int *__restrict__ rank, const int *__restrict__ cell_start,
                            int4 *__restrict__ cell_atoms, const RunState *rs, int gated)
{
  griddep_wait();
  if (skip_build(rs, gated)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int c = cell_of[i];
  if (c < 0) return;
  const int4 p = q[i];
  cell_atoms[cell_start[c] + rank[i]] = make_int4(p.x, p.y, p.z, i | (type_of(p.w) << CELL_IDX_BITS));
}

// Stencil range along one axis: 3 neighbouring cells, or every cell when the axis
// has fewer than 3 (then -1, 0, +1 would visit a cell twice).
__device__ __forceinline__ void axis_range(int c, int nc, int *lo, int *n)
{
  if (nc >= 3) { *lo = c - 1; *n = 3; }
  else { *lo = 0; *n = nc; }
}

// One stage pair (K, J) of a bitonic sorting network over v[W], then the next;
// all indices are compile-time so v[] stays in registers.
template <int W, int K, int J>
__device__ __forceinline__ void bitonic(int (&v)[W])
{
#pragma unroll
  for (int a = 0; a < W; ++a) {
    const int b = a ^ J;
    if (b > a) {
      const int x = v[a], y = v[b];
      const int lo = min(x, y), hi = max(x, y);
      const bool up = (a & K) == 0;
      v[a] = up ? lo : hi;
      v[b] = up ? hi : lo;
    }
  }
  if constexpr (J > 1) bitonic<W, K, J / 2>(v);
  else if constexpr (K < W) bitonic<W, 2 * K, K>(v);
}

// List counts during a build: the low 16 bits count the entries an atom found itself
// ("forward", written from slot 0 up by its own thread), the high 16 bits the entries
// other atoms appended to it ("backward", written from slot cap - 1 down, slot from
// an atomic count).  The two ranges meet only when the list overflows.
constexpr int BACK = 1 << 16;

// Append the pair (i, j) found by i: j goes to i's forward range (no atomic), i to
// j's backward range.
__device__ __forceinline__ void add_pair(int i, int j, int ld, int cap, int *__restrict__ nbr, int *__restrict__ cnt,
                                         int &nf)
{
  if (nf < cap) nbr[(size_t)nf * ld + i] = j;
  ++nf;
  const int b = atomicAdd(&cnt[j], BACK) >> 16;
  if (b < cap) nbr[(size_t)(cap - 1 - b) * ld + j] = i;
}

// One thread per atom, atoms taken in cell order (threads of a warp share most of
// their stencil cells, so candidate loads hit L1).  Each pair within its type pair's
// list radius is found once and appended to both lists: atom i scans its own cell (j > i) and the 13
// "forward" neighbour cells (dz = +1; dz = 0, dy = +1; dz = dy = 0, dx = +1), which
// with every axis >= 3 cells hold each neighbouring cell pair exactly once.  A
// system with an axis of fewer than 3 cells scans its whole (deduplicated) stencil
// and keeps j > i.  Candidates of one stencil row are one run of cell_atoms (two
// where the row wraps).
template <bool TYPED>
__global__ void __launch_bounds__(128, 12) k_build(int ld, int ncell, const int4 *__restrict__ q, const SysTab *__restrict__ sys,
                                               const SysCtl *__restrict__ ctl,
                                               const __grid_constant__ PairRadii radii,
                                               const int *__restrict__ cell_start,
                                               const int4 *__restrict__ cell_atoms, int *__restrict__ nbr,
                                               int *__restrict__ cnt, int cap, int4 *__restrict__ qref, RunState *rs,
                                               int gated)
{
  griddep_wait();
  if (skip_build(rs, gated)) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cell_start[ncell]) return;   // atoms with a cell (systems that get new lists)
  const int i = cell_atoms[t].w & CELL_IDX_MASK;
  const int4 pi = q[i];
  // Most candidates fail the largest radius of i's row; only the others decode j's
  // type and read their pair's radius (from the constant bank).
  const float *lrow = radii.rl2 + type_of(pi.w) * MAX_TYPES;
  const float lmax = fmaxf(fmaxf(lrow[0], lrow[1]), fmaxf(lrow[2], lrow[3]));
  auto limit = [&](int tj) { return lrow[tj]; };
  // per-system builds: a system none of whose atoms moved skin/2 keeps its lists
  if (ctl && ctl[sys_of(pi.w)].rebuild == 0) return;
  qref[i] = pi;
  const SysTab &T = sys[sys_of(pi.w)];
  const float s0 = T.geo.q_to_f[0], s1 = T.geo.q_to_f[1], s2 = T.geo.q_to_f[2];
  const int nc0 = T.nc[0], nc1 = T.nc[1], nc2 = T.nc[2];
  const int coff = T.cell_off;
  const int cx = cell_coord((uint32_t)pi.x, nc0), cy = cell_coord((uint32_t)pi.y, nc1),
            cz = cell_coord((uint32_t)pi.z, nc2);
  const bool half = nc0 >= 3 && nc1 >= 3 && nc2 >= 3;
  int nf = 0;   // entries this thread found for i

  // scan candidates [b, e) of cell_atoms (four per round: their loads go together)
  auto scan = [&](int b, int e) {
    for (int u = b; u < e; u += 4) {
      int4 pj[4];
#pragma unroll
      // padding record: index 0, never > i
      for (int k = 0; k < 4; ++k) pj[k] = u + k < e ? cell_atoms[u + k] : make_int4(0, 0, 0, 0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = pj[k].w & CELL_IDX_MASK;
        const float dx = q_scaled(qdiff(pj[k].x, pi.x), s0);
        const float dy = q_scaled(qdiff(pj[k].y, pi.y), s1);
        const float dz = q_scaled(qdiff(pj[k].z, pi.z), s2);
        const float r2 = r2_decide(dx, dy, dz);
        if (j > i && r2 < lmax && (!TYPED || r2 < limit((int)((unsigned)pj[k].w >> CELL_IDX_BITS))))
          add_pair(i, j, ld, cap, nbr, cnt, nf);
      }
    }
  };
  // cells x0 .. x0 + nx - 1 (mod nc0) of row (y, z): one or two runs
  auto scan_row = [&](int y, int z, int x0, int nx) {
    y += (y < 0) ? nc1 : 0;
    y -= (y >= nc1) ? nc1 : 0;
    z += (z < 0) ? nc2 : 0;
    z -= (z >= nc2) ? nc2 : 0;
    x0 += (x0 < 0) ? nc0 : 0;
    x0 -= (x0 >= nc0) ? nc0 : 0;
    const int row = coff + (z * nc1 + y) * nc0;
    const int xe = x0 + nx;
    scan(cell_start[row + x0], cell_start[row + min(xe, nc0)]);
    if (xe > nc0) scan(cell_start[row], cell_start[row + xe - nc0]);
  };

  if (half) {
    // own cell and its +x neighbour; keep j > i only in the own cell
    const int row = coff + (cz * nc1 + cy) * nc0;
    {
      const int b = cell_start[row + cx], e = cell_start[row + cx + 1];
      scan(b, e);
    }
    // forward cells: j may be smaller or larger than i, so test j != i by cell instead
    auto scan_any = [&](int b, int e) {
      for (int u = b; u < e; u += 4) {
        int4 pj[4];
#pragma unroll
        // padding record: word -1, which no atom has (indices stay below 2^30 - 1)
        for (int k = 0; k < 4; ++k) pj[k] = u + k < e ? cell_atoms[u + k] : make_int4(0, 0, 0, -1);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float dx = q_scaled(qdiff(pj[k].x, pi.x), s0);
          const float dy = q_scaled(qdiff(pj[k].y, pi.y), s1);
          const float dz = q_scaled(qdiff(pj[k].z, pi.z), s2);
          const float r2 = r2_decide(dx, dy, dz);
          if (pj[k].w != -1 && r2 < lmax && (!TYPED || r2 < limit((int)((unsigned)pj[k].w >> CELL_IDX_BITS))))
            add_pair(i, pj[k].w & CELL_IDX_MASK, ld, cap, nbr, cnt, nf);
        }
      }
    };
    auto row_any = [&](int y, int z, int x0, int nx) {
      y += (y < 0) ? nc1 : 0;
      y -= (y >= nc1) ? nc1 : 0;
      z += (z < 0) ? nc2 : 0;
      z -= (z >= nc2) ? nc2 : 0;
      x0 += (x0 < 0) ? nc0 : 0;
      x0 -= (x0 >= nc0) ? nc0 : 0;
      const int r = coff + (z * nc1 + y) * nc0;
      const int xe = x0 + nx;
      scan_any(cell_start[r + x0], cell_start[r + min(xe, nc0)]);
      if (xe > nc0) scan_any(cell_start[r], cell_start[r + xe - nc0]);
    };
    row_any(cy, cz, cx + 1, 1);
    row_any(cy + 1, cz, cx - 1, 3);
    row_any(cy - 1, cz + 1, cx - 1, 3);
    row_any(cy, cz + 1, cx - 1, 3);
    row_any(cy + 1, cz + 1, cx - 1, 3);
  } else {
    // whole stencil, every cell once
    const int ny = nc1 >= 3 ? 3 : nc1, nz = nc2 >= 3 ? 3 : nc2, nx = nc0 >= 3 ? 3 : nc0;
    const int y0 = nc1 >= 3 ? cy - 1 : 0, z0 = nc2 >= 3 ? cz - 1 : 0, x0 = nc0 >= 3 ? cx - 1 : 0;
    for (int oz = 0; oz < nz; ++oz)
      for (int oy = 0; oy < ny; ++oy) scan_row(y0 + oy, z0 + oz, x0, nx);
  }
  atomicAdd(&cnt[i], min(nf, BACK - 1));
}

// Sort each rebuilt list by neighbour index, so that the list order depends only on
// the set of neighbours; flag lists longer than the capacity.
__global__ void __launch_bounds__(128) k_sort_lists(int N, int ld, const int4 *__restrict__ q,
                                                    const SysCtl *__restrict__ ctl, const int *__restrict__ cell_of,
                                                    int *__restrict__ nbr, int *__restrict__ cnt, int cap,
                                                    RunState *rs, int gated)
{
  __shared__ int sbuf[32][128];
  griddep_wait();
  if (skip_build(rs, gated)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || cell_of[i] < 0) return;
  if (ctl && ctl[sys_of(q[i].w)].rebuild == 0) return;
  const int c = cnt[i];
  const int nf = c & (BACK - 1), nb = c >> 16, n = nf + nb;
  atomicMax(&rs->maxcount, n);
  if (n > cap) {
    atomicOr(&rs->status, ST_NLIST_OVERFLOW);
    return;
  }
  cnt[i] = n;
  // entry s of the list: forward entries first, then the backward ones
  auto entry = [&](int s) -> size_t { return (size_t)(s < nf ? s : cap - nb + (s - nf)) * ld + i; };
  if (n <= 16) {
    int v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = s < n ? nbr[entry(s)] : 0x7fffffff;
    if (n <= 8) {
      int w[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) w[s] = v[s];
      bitonic<8, 2, 1>(w);
#pragma unroll
      for (int s = 0; s < 8; ++s)
        if (s < n) nbr[(size_t)s * ld + i] = w[s];
    } else {
      bitonic<16, 2, 1>(v);
#pragma unroll
      for (int s = 0; s < 16; ++s)
        if (s < n) nbr[(size_t)s * ld + i] = v[s];
    }
  } else if (n <= 32) {
    // insertion sort in this thread's shared-memory column (stride 128: no bank conflicts)
    for (int s1 = 0; s1 < n; ++s1) {
      const int v = nbr[entry(s1)];
      int k = s1 - 1;
      while (k >= 0 && sbuf[k][threadIdx.x] > v) {
        sbuf[k + 1][threadIdx.x] = sbuf[k][threadIdx.x];
        --k;
      }
      sbuf[k + 1][threadIdx.x] = v;
    }
    for (int s1 = 0; s1 < n; ++s1) nbr[(size_t)s1 * ld + i] = sbuf[s1][threadIdx.x];
  } else {
    // move the backward entries down behind the forward ones (cap - nb >= nf), then
    // insertion sort in place
    for (int k = 0; k < nb; ++k) nbr[(size_t)(nf + k) * ld + i] = nbr[(size_t)(cap - nb + k) * ld + i];
    for (int s1 = 1; s1 < n; ++s1) {
      const int v = nbr[(size_t)s1 * ld + i];
      int k = s1 - 1;
      while (k >= 0) {
        const int w = nbr[(size_t)k * ld + i];
        if (w <= v) break;
        nbr[(size_t)(k + 1) * ld + i] = w;
        --k;
      }
      nbr[(size_t)(k + 1) * ld + i] = v;
    }
  }
}

// rev[s][i] = where the force gather finds the contribution of the terms of i's
// neighbour j = nbr[s][i] on i: the flat index s2 * ld + j of i's slot s2 in j's
// (sorted) list, found by binary search (a 32-bit unsigned value: cap * ld < 2^32).
// Lists are symmetric, so one search serves both entries of a pair: atom i takes the
// entries with j > i (the tail of its sorted list), finds s2, and writes rev[s][i]
// and rev[s2][j]; every entry has exactly one writer.  One thread per atom; the
// searches of up to RS slots run interleaved, level by level, so their loads are in
// flight together.
constexpr int RS = 8;
__global__ void k_reverse(int N, int ld, const int4 *__restrict__ q, const SysCtl *__restrict__ ctl,
                          const int *__restrict__ cell_of, const int *__restrict__ nbr, const int *__restrict__ cnt,
                          int *__restrict__ rev, RunState *rs, int gated)
{
  griddep_wait();
  if (skip_build(rs, gated)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || cell_of[i] < 0) return;
  if (ctl && ctl[sys_of(q[i].w)].rebuild == 0) return;
  const int n = cnt[i];
  // the entries with j > i start at the first index above i (lists are sorted); their
  // searches then fill whole rounds
  int first = 0;
  {
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (nbr[(size_t)mid * ld + i] > i) hi = mid; else lo = mid + 1;
    }
    first = lo;
  }
  bool missing = false;
  for (int s0 = first; s0 < n; s0 += RS) {
    int j[RS], lo[RS], hi[RS], found[RS];
#pragma unroll
    for (int k = 0; k < RS; ++k) j[k] = s0 + k < n ? nbr[(size_t)(s0 + k) * ld + i] : -1;
#pragma unroll
    for (int k = 0; k < RS; ++k) {
      lo[k] = 0;
      hi[k] = j[k] >= 0 ? cnt[j[k]] - 1 : -1;
      found[k] = -1;
    }
    bool more = true;
    while (more) {
      more = false;
#pragma unroll
      for (int k = 0; k < RS; ++k) {
        if (found[k] < 0 && lo[k] <= hi[k]) {
          const int mid = (lo[k] + hi[k]) >> 1;
          const int v = nbr[(size_t)mid * ld + j[k]];
          if (v == i) found[k] = mid;
          else if (v < i) lo[k] = mid + 1;
          else hi[k] = mid - 1;
          more = true;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < RS; ++k) {
      if (j[k] < 0) continue;
      if (found[k] < 0) {
        missing = true;
        rev[(size_t)(s0 + k) * ld + i] = (int)(unsigned)j[k];
        continue;
      }
      rev[(size_t)(s0 + k) * ld + i] = (int)((unsigned)found[k] * (unsigned)ld + (unsigned)j[k]);
      rev[(size_t)found[k] * ld + j[k]] = (int)((unsigned)(s0 + k) * (unsigned)ld + (unsigned)i);
    }
  }
  if (missing) atomicOr(&rs->status, ST_REV_MISSING);
}

// Sorted lists and reverse indices in one pass, for lists of up to 16 slots.  k_build
// then wrote its raw lists to raw/rawcnt (forward entries from slot 0, backward ones
// from slot cap - 1 down, packed counts), which no thread writes here.  Thread i sorts
// its own raw list in registers and writes it to nbr.  The slot of i in the sorted list
// of a neighbour j is the number of entries of j's raw list below i, so no search in a
// sorted list is needed: for each neighbour j > i (the tail of i's sorted list) thread
// i counts them and writes both reverse entries of the pair, as k_reverse does, so
// every entry has one writer.  The lists, counts and reverse indices equal those of
// k_sort_lists + k_reverse.  (Longer lists keep those two kernels: for the 3C-SiC lists
// of ~16 entries a shared-memory sort and ~100 neighbour-list loads per atom were
// slower than the binary searches.)
__global__ void __launch_bounds__(128, 8) k_sort_reverse(int N, int ld, const int4 *__restrict__ q,
                                                      const SysCtl *__restrict__ ctl, const int *__restrict__ cell_of,
                                                      const int *__restrict__ raw, const int *__restrict__ rawcnt,
                                                      int *__restrict__ nbr, int *__restrict__ cnt,
                                                      int *__restrict__ rev, int cap, RunState *rs, int gated)
{
  griddep_wait();
  if (skip_build(rs, gated)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || cell_of[i] < 0) return;
  if (ctl && ctl[sys_of(q[i].w)].rebuild == 0) return;
  const int c = rawcnt[i];
  const int nf = c & (BACK - 1), nb = c >> 16, n = nf + nb;
  atomicMax(&rs->maxcount, n);
  if (n > cap) {
    atomicOr(&rs->status, ST_NLIST_OVERFLOW);
    return;
  }
  cnt[i] = n;
  auto slot = [&](int s, int f, int b) { return s < f ? s : cap - b + (s - f); };
  int v[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) v[s] = s < n ? raw[(size_t)slot(s, nf, nb) * ld + i] : 0x7fffffff;
  if (n <= 8) {
    int w[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) w[s] = v[s];
    bitonic<8, 2, 1>(w);
#pragma unroll
    for (int s = 0; s < 8; ++s) v[s] = w[s];
  } else {
    bitonic<16, 2, 1>(v);
  }
#pragma unroll
  for (int s = 0; s < 16; ++s)
    if (s < n) nbr[(size_t)s * ld + i] = v[s];
  bool missing = false;
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    if (s < n && v[s] > i) {
      const int j = v[s];
      const int cj = rawcnt[j];
      // a neighbour whose list overflowed (it flags that itself) is not read: its
      // ranges may overlap or start below slot 0
      const int fj = cj & (BACK - 1), bj = cj >> 16, nj = fj + bj <= cap ? fj + bj : 0;
      int below = 0;
      bool found = false;
      for (int t0 = 0; t0 < nj; t0 += 4) {
        int e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] = t0 + k < nj ? raw[(size_t)slot(t0 + k, fj, bj) * ld + j] : 0x7fffffff;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          below += e[k] < i;
          found = found || e[k] == i;
        }
      }
      if (found) {
        rev[(size_t)s * ld + i] = (int)((unsigned)below * (unsigned)ld + (unsigned)j);
        rev[(size_t)below * ld + j] = (int)((unsigned)s * (unsigned)ld + (unsigned)i);
      } else {
        missing = true;
        rev[(size_t)s * ld + i] = (int)(unsigned)j;
      }
    }
  }
  if (missing) atomicOr(&rs->status, ST_REV_MISSING);
}

// close a build: count it, clear the request
__global__ void k_build_done(RunState *rs, int gated)
{
  griddep_wait();
  if (skip_build(rs, gated)) return;
  rs->nrebuild += 1;
  rs->rebuild = 0;
}

}  // namespace tsf

namespace tsf {

// Enqueue one list build on st (ctl non-null: only the systems whose rebuild flag is
// set get new lists; null: every atom).  N <= MAX_LIST_ATOMS atoms; atoms of a
// system without atoms (freed ranges of a packed layout) are left out.  ld >= N:
// the list stride.  radii: list radius per type pair.  Buffers: cell_count[ncell]
// (zero on entry, zero on exit), cell_start[ncell+1], tile_sums[ceil(ncell/SCAN_TILE)],
// cell_atoms[N] (int4), cell_of[N], rank[N]; list nbr/rev [cap][ld], cnt[N]; qref[N].
// raw [cap][ld] and rawcnt[N] (optional): scratch for the raw lists, every column of
// an atom that gets a new list free to overwrite (the build's atoms only).
cudaError_t launch_build(cudaStream_t st, int N, int ld, const int4 *q, const SysTab *sys, const SysCtl *ctl, int ncell,
                         const PairRadii &radii,
                         int *cell_count, int *cell_start, int *tile_sums, int4 *cell_atoms, int *cell_of, int *rank,
                         int *nbr, int *rev, int *cnt, int cap, int4 *qref, RunState *rs, int gated, int *raw,
                         int *rawcnt)
{
  if (N == 0) return cudaSuccess;
  // lists of up to 16 slots with raw scratch: k_build appends there and one kernel
  // sorts and finds the reverse indices; else k_build appends in place, then
  // k_sort_lists and k_reverse
  const bool fused = raw && rawcnt && cap <= 16;
  int *bnbr = fused ? raw : nbr, *bcnt = fused ? rawcnt : cnt;
  const int T = 256;
  const int BN = (N + T - 1) / T;
  const int ntiles = (ncell + SCAN_TILE - 1) / SCAN_TILE;
  k_cell_count<<<BN, T, 0, st>>>(N, q, sys, ctl, cell_of, rank, cell_count, bcnt, rs, gated);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_dep(k_scan_tiles, ntiles, SCAN_THREADS, 0, st, ncell, (const int *)cell_count, cell_start, tile_sums,
                      (const RunState *)rs, gated)) != cudaSuccess)
    return e;
  if ((e = launch_dep(k_scan_sums, 1, SCAN_THREADS, 0, st, ntiles, tile_sums, cell_start + ncell,
                      (const RunState *)rs, gated)) != cudaSuccess)
    return e;
  if ((e = launch_dep(k_scan_add, (ncell + T - 1) / T, T, 0, st, ncell, cell_start, (const int *)tile_sums, cell_count,
                      (const RunState *)rs, gated)) != cudaSuccess)
    return e;
  if ((e = launch_dep(k_cell_fill, BN, T, 0, st, N, q, (const int *)cell_of, (const int *)rank,
                      (const int *)cell_start, cell_atoms, (const RunState *)rs, gated)) != cudaSuccess)
    return e;
  const int BN128 = (N + 127) / 128;
  // one radius for every type pair (one-type tables, or lists built with one cutoff):
  // the row's largest radius decides alone
  bool typed = false;
  for (int k = 1; k < MAX_TYPES * MAX_TYPES; ++k) typed = typed || radii.rl2[k] != radii.rl2[0];
  if ((e = launch_dep(typed ? k_build<true> : k_build<false>, BN128, 128, 0, st, ld, ncell, q, sys, ctl, radii,
                      (const int *)cell_start, (const int4 *)cell_atoms, bnbr, bcnt, cap, qref, rs, gated)) != cudaSuccess)
    return e;
  if (fused) {
    if ((e = launch_dep(k_sort_reverse, BN128, 128, 0, st, N, ld, q, ctl, (const int *)cell_of, (const int *)raw,
                        (const int *)rawcnt, nbr, cnt, rev, cap, rs, gated)) != cudaSuccess)
      return e;
    return launch_dep(k_build_done, 1, 1, 0, st, rs, gated);
  }
  if ((e = launch_dep(k_sort_lists, BN128, 128, 0, st, N, ld, q, ctl, (const int *)cell_of, nbr, cnt, cap, rs,
                      gated)) != cudaSuccess)
    return e;
  if ((e = launch_dep(k_reverse, BN128, 128, 0, st, N, ld, q, ctl, (const int *)cell_of, (const int *)nbr,
                      (const int *)cnt, rev, rs, gated)) != cudaSuccess)
    return e;
  return launch_dep(k_build_done, 1, 1, 0, st, rs, gated);
}

int scan_tiles_for(int ncell) { return (ncell + SCAN_TILE - 1) / SCAN_TILE; }

}  // namespace tsf
