// grid.hpp -- host-side builder of the sparse tiled multilevel grid (Sec 2.1
// pre-processor: 2:1 distance-band refinement, cell-centred solid painting,
// inter-level connectivity; Sec 2.3 preprocessing: cut links, wall records).
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "layout.hpp"

namespace lbmgrid {

// allocator whose value-less construct leaves elements uninitialised: the large per-cell
// tables are sized first and then filled in parallel, so that their pages are first
// touched by the threads that fill them instead of being zeroed by one thread
template <class T>
struct NoInit : std::allocator<T> {
    template <class U> struct rebind { using other = NoInit<U>; };
    NoInit() = default;
    template <class U> NoInit(const NoInit<U> &) noexcept {}
    template <class U> void construct(U *p) noexcept { ::new ((void *)p) U; }
    template <class U, class... A> void construct(U *p, A &&...a) { ::new ((void *)p) U(std::forward<A>(a)...); }
};
template <class T> using cellvec = std::vector<T, NoInit<T>>;

struct Spec {
    int levels, nx0, ny0, layers;
    double x0, y0, h0;
    double d_wr, d_wv;
    int periodic, solid_walls, wall_model;
};

struct IPt { long long x, y; };

struct Level {
    int l = 0;
    long long scale = 1;            // finest cells per cell edge: 2^(L-1-l)
    // dense build-time box (global level indices)
    int bi0 = 0, bj0 = 0, bnx = 0, bny = 0;
    cellvec<uint8_t> kind;          // KIND_* over the box
    cellvec<uint8_t> solid, band, bnode;
    cellvec<uint16_t> coal, cut;
    cellvec<double> dist;           // wall distance, level lattice units
    cellvec<int> rec;               // wall record of a B node
    // present-cell box
    int pi0 = 0, pj0 = 0, pnx = 0, pny = 0;
    // tiles
    int tx0 = 0, ty0 = 0, ntx = 0, nty = 0;
    std::vector<int> tile_of;       // ntx * nty -> tile index or -1
    std::vector<int> tile_x, tile_y;
    std::vector<int> nbr;           // 9 per tile (D2Q9 order), -1 absent
    std::vector<int> child;         // 4 per tile: level l+1 tiles (b * 2 + a)
    std::vector<int> parent;        // level l-1 tile holding the parents of this tile's cells, or -1
    std::vector<int> band_tiles;    // tiles holding at least one band cell (explosion / prolongation)
    std::vector<int> work_tiles;    // tiles holding at least one active or ghost fluid cell
    int ntiles = 0;
    int n_wall_tiles = 0;           // tiles holding boundary nodes come first in the tile order

    long idx(long long i, long long j) const {
        if (i < bi0 || j < bj0 || i >= bi0 + bnx || j >= bj0 + bny) return -1;
        return (long)(j - bj0) * bnx + (long)(i - bi0);
    }
    // device slot of a cell (tile * 256 + ly * 32 + lx), or -1
    long slot(long long i, long long j) const;
};

struct Record {
    int i, j, seg, loop;
    double iw[2], n[2], dwb, r[2];
    int ns;
    int si[16], sj[16];
    double q[9];
};

struct Grid {
    Spec spec;
    int L = 0;
    std::vector<IPt> v;
    std::vector<int> sa, sb, sloop, loop_ccw;
    std::vector<Level> lv;
    std::vector<Record> recs;
    std::vector<int> seg_b1, seg_b2;
    std::vector<double> seg_w1, seg_w2;
    long long n_cut = 0;
};

// Returns 0 on success, otherwise an LBM status code with msg filled in.
int build(const Spec &spec, const double *xy, const int *loop_off, int n_loops, Grid &g, std::string &msg);

}  // namespace lbmgrid
