// layout.hpp -- device data layout shared by the host builder and the kernels.
//
// Each level is a sparse set of 32 x 8 cell tiles.  A cell slot is
// tile * 256 + ly * 32 + lx; populations are stored structure-of-arrays per
// direction, f[d * n_slots + slot], shifted by the lattice weight (f - w_q), in one
// lattice updated in place (even steps keep a cell's populations in its own slots,
// odd steps move them to the neighbours' slots).
#pragma once

#include <cstdint>

#define LBM_TX 32
#define LBM_TY 8
#define LBM_TILE (LBM_TX * LBM_TY)
#define LBM_MAXL 16

// cell kinds
#define KIND_ABSENT 0u
#define KIND_ACTIVE 1u
#define KIND_COVERED 2u
#define KIND_GHOST 3u

// per-cell flag word
#define FL_KIND_MASK 0x3u
#define FL_SOLID (1u << 2)
#define FL_BAND (1u << 3)      // active cell with ghost children on the next level
#define FL_BNODE (1u << 4)     // boundary node B (has cut links)
#define FL_COAL_SHIFT 5        // bits 5..12: coalesced pulled directions 1..8
#define FL_CUT_SHIFT 13        // bits 13..20: cut pulled directions 1..8 (boundary nodes, finest level)
#define FL_KEEP_SHIFT 13       // ghost cells, bits 13..20: the cell upstream along direction 1..8 is
                               // not an active or ghost fluid cell (the ghost keeps its own value)
#define FL_SCH_SHIFT 13        // band cells, bits 13..16: child b * 2 + a is solid or has no tile
#define FL_INLET (1u << 21)    // level 0, i == 0
#define FL_OUTLET (1u << 22)   // level 0, i == nx0 - 1
#define FL_BOTTOM (1u << 23)   // level 0, j == 0
#define FL_TOP (1u << 24)      // level 0, j == ny0 - 1
#define FL_OUTLET2 (1u << 25)  // level 0, i == nx0 - 2 (feeds the outlet's extrapolation)

// D2Q9 directions (paper index = q + 1), eq 2
#define LBM_CX_INIT {0, 1, -1, 0, 0, 1, -1, 1, -1}
#define LBM_CY_INIT {0, 0, 0, 1, -1, 1, -1, -1, 1}
