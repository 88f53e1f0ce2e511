// Host-side state structs of the runtime (not part of the C ABI).
#pragma once
#include <cstddef>
#include <cstdint>

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
  int *cell_count = nullptr, *cell_start = nullptr, *tile_sums = nullptr, *cell_atoms = nullptr, *cell_of = nullptr,
      *rank = nullptr;
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
