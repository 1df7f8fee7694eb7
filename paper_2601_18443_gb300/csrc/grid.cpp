// grid.cpp -- host builder of the sparse tiled 2:1 multilevel grid.
//
// Reading of the paper's pre-processor (Sec 2.1; its octree/ADT/advancing-front
// generator is not specified): level l >= 1 holds the children of level l-1
// cells whose centre lies within R_l of a wall, R_{L-1} = layers h_{L-1},
// R_l = R_{l+1} + layers h_l.  Active cells with a covered D2Q9 neighbour form the
// band whose children are ghost cells of the next level (Rohde transfers).  A cell
// is solid iff its centre lies inside or on a wall loop.  All yes/no decisions use
// exact integer arithmetic on vertices snapped to 1/4096 of the finest cell, so
// that the tables are bit-exact and reproducible.
//
// Algorithms: per-segment candidate boxes for the refinement bands, a row scanline
// with exact rational crossings for the solid painting, a bounding-volume tree over
// the wall segments for distances, feet of perpendiculars and link crossings.
#include "grid.hpp"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <limits>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace lbmgrid {

typedef __int128 i128;
static const int CX[9] = LBM_CX_INIT;
static const int CY[9] = LBM_CY_INIT;
static const long long FIXU = 4096;   // fixed-point units per finest cell
static const double DCAP = 1.0e12;

static inline long long fdiv(i128 a, i128 b)
{   // floor(a / b), b > 0
    i128 q = a / b;
    if ((a % b) != 0 && (a < 0)) q -= 1;
    return (long long)q;
}
static inline long long cdiv(i128 a, i128 b) { return -fdiv(-a, b); }

long Level::slot(long long i, long long j) const
{
    long long tx = fdiv(i, LBM_TX), ty = fdiv(j, LBM_TY);
    if (tx < tx0 || ty < ty0 || tx >= tx0 + ntx || ty >= ty0 + nty) return -1;
    int t = tile_of[(size_t)(ty - ty0) * ntx + (tx - tx0)];
    if (t < 0) return -1;
    return (long)t * LBM_TILE + (long)(j - ty * LBM_TY) * LBM_TX + (long)(i - tx * LBM_TX);
}

// ---------------------------------------------------------------- exact tests
static bool within_r(IPt a, IPt b, IPt p, long long R)
{
    i128 ex = b.x - a.x, ey = b.y - a.y, px = p.x - a.x, py = p.y - a.y;
    i128 l2 = ex * ex + ey * ey, dot = px * ex + py * ey, R2 = (i128)R * R;
    if (l2 == 0 || dot <= 0) return px * px + py * py <= R2;
    if (dot >= l2) {
        i128 qx = p.x - b.x, qy = p.y - b.y;
        return qx * qx + qy * qy <= R2;
    }
    i128 c = ex * py - ey * px;
    return c * c <= R2 * l2;
}

static bool on_seg(IPt a, IPt b, IPt p)
{
    i128 ex = b.x - a.x, ey = b.y - a.y, px = p.x - a.x, py = p.y - a.y;
    if (ex * py - ey * px != 0) return false;
    i128 dot = px * ex + py * ey;
    return dot >= 0 && dot <= ex * ex + ey * ey;
}

// exact test whether segments ab and cd cross properly (each strictly separates the other's
// ends); touching, a shared end and collinear overlap are not crossings
static int orient(IPt a, IPt b, IPt c)
{
    const i128 v = (i128)(b.x - a.x) * (c.y - a.y) - (i128)(b.y - a.y) * (c.x - a.x);
    return v > 0 ? 1 : (v < 0 ? -1 : 0);
}

static bool segs_cross(IPt a, IPt b, IPt c, IPt d)
{
    return orient(a, b, c) * orient(a, b, d) < 0 && orient(c, d, a) * orient(c, d, b) < 0;
}

// ---------------------------------------------------------------- segment tree
struct SegTree {
    // node: bounding box, and a capsule (the chord from the range's first to its last vertex,
    // with a radius covering every endpoint) of the segments [lo, hi)
    struct Node { double x0, y0, x1, y1, c0x, c0y, c1x, c1y, rad, ux, uy, il2; int lo, hi, left, right, up; };
    std::vector<Node> nodes;
    std::vector<double> ax, ay, bx, by;   // finest lattice units
    std::vector<int> leaf_of;             // leaf node holding each segment
    int root = -1;

    // nodes of the subtree over n segments (a range splits in halves while it holds more
    // than 8); the tree is stored in pre-order, so a node's right child follows its left
    // subtree and every subtree can be built independently
    static int tree_count(int n) { return n <= 8 ? 1 : 1 + tree_count(n / 2) + tree_count(n - n / 2); }

    void make(int id, int lo, int hi, int up)
    {
        Node nd;
        nd.lo = lo; nd.hi = hi; nd.left = nd.right = -1; nd.up = up;
        nd.x0 = nd.y0 = std::numeric_limits<double>::infinity();
        nd.x1 = nd.y1 = -std::numeric_limits<double>::infinity();
        for (int k = lo; k < hi; k++) {
            nd.x0 = std::min(nd.x0, std::min(ax[k], bx[k])); nd.x1 = std::max(nd.x1, std::max(ax[k], bx[k]));
            nd.y0 = std::min(nd.y0, std::min(ay[k], by[k])); nd.y1 = std::max(nd.y1, std::max(ay[k], by[k]));
        }
        nd.c0x = ax[lo]; nd.c0y = ay[lo]; nd.c1x = bx[hi - 1]; nd.c1y = by[hi - 1];
        double r2 = 0.0;
        for (int k = lo; k < hi; k++) {
            r2 = std::max(r2, pt_seg2(nd.c0x, nd.c0y, nd.c1x, nd.c1y, ax[k], ay[k]));
            r2 = std::max(r2, pt_seg2(nd.c0x, nd.c0y, nd.c1x, nd.c1y, bx[k], by[k]));
        }
        // every segment lies inside the capsule (it is convex and holds both endpoints); the
        // margin keeps the bound below the true distance whatever the rounding
        const double span = std::fabs(nd.x1 - nd.x0) + std::fabs(nd.y1 - nd.y0);
        nd.rad = std::sqrt(r2) * (1.0 + 1e-9) + 1e-9 * (span + 1.0);
        nd.ux = nd.c1x - nd.c0x; nd.uy = nd.c1y - nd.c0y;
        const double l2 = nd.ux * nd.ux + nd.uy * nd.uy;
        nd.il2 = l2 > 0 ? 1.0 / l2 : 0.0;
        if (hi - lo > 8) {
            const int mid = (lo + hi) / 2;
            nd.left = id + 1;
            nd.right = id + 1 + tree_count(mid - lo);
            nodes[id] = nd;
            if (hi - lo > 8192) {
#pragma omp task
                make(nd.left, lo, mid, id);
#pragma omp task
                make(nd.right, mid, hi, id);
#pragma omp taskwait
            } else {
                make(nd.left, lo, mid, id);
                make(nd.right, mid, hi, id);
            }
        } else {
            nodes[id] = nd;
            for (int k = lo; k < hi; k++) leaf_of[k] = id;
        }
    }
    static double pt_seg2(double ax_, double ay_, double bx_, double by_, double px, double py)
    {
        const double dx = bx_ - ax_, dy = by_ - ay_;
        const double len2 = dx * dx + dy * dy;
        double t = len2 > 0 ? ((px - ax_) * dx + (py - ay_) * dy) / len2 : 0.0;
        if (t < 0) t = 0;
        if (t > 1) t = 1;
        const double qx = ax_ + t * dx - px, qy = ay_ + t * dy - py;
        return qx * qx + qy * qy;
    }
    // lower bound of the squared distance from p to the node's segments: the larger of the
    // box distance and the capsule distance (distance to the chord minus the radius).  The
    // chord distance is measured to the computed projection of p (the chord's reciprocal
    // squared length precomputed); rounding can only move that point off the nearest chord
    // point and so overstate the distance, by far less than the radius margin
    static double node_lb2(const Node &nd, double px, double py)
    {
        const double dx = std::max(0.0, std::max(nd.x0 - px, px - nd.x1));
        const double dy = std::max(0.0, std::max(nd.y0 - py, py - nd.y1));
        const double box2 = dx * dx + dy * dy;
        double t = ((px - nd.c0x) * nd.ux + (py - nd.c0y) * nd.uy) * nd.il2;
        t = t < 0 ? 0 : (t > 1 ? 1 : t);
        const double qx = nd.c0x + t * nd.ux - px, qy = nd.c0y + t * nd.uy - py;
        const double cap = std::sqrt(qx * qx + qy * qy) - nd.rad;
        return cap > 0.0 ? std::max(box2, cap * cap) : box2;
    }
    void init(const Grid &g)
    {
        size_t n = g.sa.size();
        ax.resize(n); ay.resize(n); bx.resize(n); by.resize(n);
        for (size_t k = 0; k < n; k++) {
            ax[k] = (double)g.v[g.sa[k]].x / FIXU; ay[k] = (double)g.v[g.sa[k]].y / FIXU;
            bx[k] = (double)g.v[g.sb[k]].x / FIXU; by[k] = (double)g.v[g.sb[k]].y / FIXU;
        }
        leaf_of.assign(n, -1);
        nodes.assign(n ? tree_count((int)n) : 0, Node());
        root = n ? 0 : -1;
        if (n) {
#pragma omp parallel
#pragma omp single
            make(0, 0, (int)n, -1);
        }
    }
    // distance from p to segment k and the foot of the perpendicular
    double seg_dist(int k, double px, double py, double &qx, double &qy) const
    {
        double dx = bx[k] - ax[k], dy = by[k] - ay[k];
        double len2 = dx * dx + dy * dy;
        double t = len2 > 0 ? ((px - ax[k]) * dx + (py - ay[k]) * dy) / len2 : 0.0;
        if (t < 0) t = 0;
        if (t > 1) t = 1;
        qx = ax[k] + t * dx; qy = ay[k] + t * dy;
        return std::sqrt((px - qx) * (px - qx) + (py - qy) * (py - qy));
    }
    static double box_dist(const Node &nd, double px, double py)
    {
        double dx = std::max(0.0, std::max(nd.x0 - px, px - nd.x1));
        double dy = std::max(0.0, std::max(nd.y0 - py, py - nd.y1));
        return std::sqrt(dx * dx + dy * dy);
    }
    // nearest segment; ties go to the lowest segment index
    double nearest(double px, double py, int &kbest, double &cx, double &cy) const
    {
        double best = std::numeric_limits<double>::infinity();
        kbest = -1; cx = cy = 0;
        if (root < 0) return best;
        int stack[128];
        int sp = 0;
        stack[sp++] = root;
        while (sp) {
            const Node &nd = nodes[stack[--sp]];
            if (box_dist(nd, px, py) > best) continue;
            if (nd.left < 0) {
                for (int k = nd.lo; k < nd.hi; k++) {
                    double qx, qy, d = seg_dist(k, px, py, qx, qy);
                    if (d < best || (d == best && k < kbest)) { best = d; kbest = k; cx = qx; cy = qy; }
                }
            } else {
                double dl = box_dist(nodes[nd.left], px, py), dr = box_dist(nodes[nd.right], px, py);
                if (dl <= dr) { stack[sp++] = nd.right; stack[sp++] = nd.left; }
                else { stack[sp++] = nd.left; stack[sp++] = nd.right; }
            }
        }
        return best;
    }
    // distance from p to the nearest segment, searching only within `bound` (an upper bound
    // of that distance, or infinity); squared distances throughout, so that the result
    // equals the sqrt of the smallest squared distance nearest() evaluates: bit for bit
    // the distance nearest() returns.  Infinity if no segment lies within bound.
    double nearest_dist(double px, double py, double bound, int &kfound) const
    {
        double best2 = bound * bound;
        bool found = false;
        kfound = -1;
        if (root < 0) return std::numeric_limits<double>::infinity();
        // each stacked node carries its lower bound, evaluated once when it is pushed and
        // tested again when it is popped, against the best distance found by then
        int stack[128];
        double slb2[128];
        int sp = 0;
        stack[sp] = root; slb2[sp++] = 0.0;
        while (sp) {
            --sp;
            if (slb2[sp] > best2) continue;
            const Node &nd = nodes[stack[sp]];
            if (nd.left < 0) {
                for (int k = nd.lo; k < nd.hi; k++) {
                    const double d2 = seg_dist2(k, px, py);
                    if (d2 <= best2) { best2 = d2; found = true; kfound = k; }
                }
            } else {
                const double dl = node_lb2(nodes[nd.left], px, py), dr = node_lb2(nodes[nd.right], px, py);
                // the nearer child is popped first
                const int first = dl <= dr ? nd.left : nd.right, second = dl <= dr ? nd.right : nd.left;
                const double lf = std::min(dl, dr), ls = std::max(dl, dr);
                if (ls <= best2) { stack[sp] = second; slb2[sp++] = ls; }
                if (lf <= best2) { stack[sp] = first; slb2[sp++] = lf; }
            }
        }
        return found ? std::sqrt(best2) : std::numeric_limits<double>::infinity();
    }
    // distance from p to the nearest segment, searched outwards from the leaf of segment
    // `kstart` (the nearest segment of a neighbouring point): that leaf first, then the
    // sibling of each of its ancestors, each subtree pruned by the best distance found so
    // far.  Every segment is either evaluated or pruned by a valid lower bound, so the
    // result is the smallest squared distance over all segments, as in nearest_dist.
    double nearest_dist_from(double px, double py, int kstart, int &kfound) const
    {
        double best2 = std::numeric_limits<double>::infinity();
        int node = leaf_of[kstart];
        for (int k = nodes[node].lo; k < nodes[node].hi; k++) {
            const double d2 = seg_dist2(k, px, py);
            if (d2 <= best2) { best2 = d2; kfound = k; }
        }
        int stack[128];
        double slb2[128];
        while (nodes[node].up >= 0) {
            const Node &pa = nodes[nodes[node].up];
            const int sib = pa.left == node ? pa.right : pa.left;
            node = nodes[node].up;
            int sp = 0;
            stack[sp] = sib; slb2[sp++] = node_lb2(nodes[sib], px, py);
            while (sp) {
                --sp;
                if (slb2[sp] > best2) continue;
                const Node &nd = nodes[stack[sp]];
                if (nd.left < 0) {
                    for (int k = nd.lo; k < nd.hi; k++) {
                        const double d2 = seg_dist2(k, px, py);
                        if (d2 <= best2) { best2 = d2; kfound = k; }
                    }
                } else {
                    const double dl = node_lb2(nodes[nd.left], px, py), dr = node_lb2(nodes[nd.right], px, py);
                    const int first = dl <= dr ? nd.left : nd.right, second = dl <= dr ? nd.right : nd.left;
                    const double lf = std::min(dl, dr), ls = std::max(dl, dr);
                    if (ls <= best2) { stack[sp] = second; slb2[sp++] = ls; }
                    if (lf <= best2) { stack[sp] = first; slb2[sp++] = lf; }
                }
            }
        }
        return std::sqrt(best2);
    }
    double seg_dist2(int k, double px, double py) const
    {
        double dx = bx[k] - ax[k], dy = by[k] - ay[k];
        double len2 = dx * dx + dy * dy;
        double t = len2 > 0 ? ((px - ax[k]) * dx + (py - ay[k]) * dy) / len2 : 0.0;
        if (t < 0) t = 0;
        if (t > 1) t = 1;
        const double qx = ax[k] + t * dx, qy = ay[k] + t * dy;
        return (px - qx) * (px - qx) + (py - qy) * (py - qy);
    }
    void overlapping(double x0, double y0, double x1, double y1, std::vector<int> &out) const
    {
        out.clear();
        if (root < 0) return;
        int stack[128];
        int sp = 0;
        stack[sp++] = root;
        while (sp) {
            const Node &nd = nodes[stack[--sp]];
            if (nd.x1 < x0 || nd.x0 > x1 || nd.y1 < y0 || nd.y0 > y1) continue;
            if (nd.left < 0) {
                for (int k = nd.lo; k < nd.hi; k++) out.push_back(k);
            } else {
                stack[sp++] = nd.left; stack[sp++] = nd.right;
            }
        }
        std::sort(out.begin(), out.end());
    }
};

// first wall crossing along the link p -> p + d (fraction in (0, 1]), exact tests
static double link_q(const Grid &g, const SegTree &T, IPt p, IPt d)
{
    std::vector<int> cand;
    double x0 = (double)std::min(p.x, p.x + d.x) / FIXU - 1e-9, x1 = (double)std::max(p.x, p.x + d.x) / FIXU + 1e-9;
    double y0 = (double)std::min(p.y, p.y + d.y) / FIXU - 1e-9, y1 = (double)std::max(p.y, p.y + d.y) / FIXU + 1e-9;
    T.overlapping(x0, y0, x1, y1, cand);
    double best = 2.0;
    for (int k : cand) {
        IPt a = g.v[g.sa[k]], b = g.v[g.sb[k]];
        i128 ex = b.x - a.x, ey = b.y - a.y;
        i128 den = (i128)d.x * ey - (i128)d.y * ex;
        i128 rx = a.x - p.x, ry = a.y - p.y;
        i128 tn = rx * ey - ry * ex;          // parameter along the link (x den)
        i128 un = rx * d.y - ry * d.x;        // parameter along the segment (x den)
        if (den != 0) {
            if (den < 0) { den = -den; tn = -tn; un = -un; }
            if (tn >= 0 && tn <= den && un >= 0 && un <= den) best = std::min(best, (double)tn / (double)den);
        } else if (tn == 0) {
            double dd = (double)((i128)d.x * d.x + (i128)d.y * d.y);
            double ta = (double)(rx * d.x + ry * d.y) / dd;
            double tb = (double)((i128)(b.x - p.x) * d.x + (i128)(b.y - p.y) * d.y) / dd;
            double lo = std::min(ta, tb), hi = std::max(ta, tb);
            if (hi >= 0 && lo <= 1) best = std::min(best, std::max(lo, 0.0));
        }
    }
    return best;
}

// ---------------------------------------------------------------- build
static int failmsg(std::string &msg, const char *m)
{
    msg = m;
    return -5;
}

static void alloc_level(Level &Lv, int i0, int j0, int nx, int ny)
{
    Lv.bi0 = i0; Lv.bj0 = j0; Lv.bnx = nx; Lv.bny = ny;
    const long n = (long)nx * ny;
    Lv.kind.resize(n); Lv.solid.resize(n); Lv.band.resize(n); Lv.bnode.resize(n);
    Lv.coal.resize(n); Lv.cut.resize(n); Lv.dist.resize(n); Lv.rec.resize(n);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; c++) {
        Lv.kind[c] = KIND_ABSENT; Lv.solid[c] = 0; Lv.band[c] = 0; Lv.bnode[c] = 0;
        Lv.coal[c] = 0; Lv.cut[c] = 0; Lv.dist[c] = 0.0; Lv.rec[c] = -1;
    }
}

// centre of level cell (i, j) in fixed units
static inline IPt centre(const Level &Lv, long long i, long long j)
{
    long long hh = Lv.scale * FIXU / 2;
    return IPt{(2 * i + 1) * hh, (2 * j + 1) * hh};
}

// solid painting of one level by exact row scanlines
static void paint_solid(const Grid &g, Level &Lv)
{
    const long long hh = Lv.scale * FIXU / 2;     // half cell
    const size_t nseg = g.sa.size();
    // rows crossed by each segment (half-open rule ymin <= Y < ymax), as lists per row
    // (counted, then filled; the order inside a row does not matter, the parity is a XOR)
    auto row_span = [&](long k, long long &jl, long long &jh) {
        IPt a = g.v[g.sa[k]], b = g.v[g.sb[k]];
        jl = jh = 0;
        if (a.y == b.y) return;
        long long ymin = std::min(a.y, b.y), ymax = std::max(a.y, b.y);
        jl = cdiv((i128)ymin - hh, 2 * (i128)hh); jh = cdiv((i128)ymax - hh, 2 * (i128)hh);
        jl = std::max<long long>(jl, Lv.bj0);
        jh = std::min<long long>(jh, (long long)Lv.bj0 + Lv.bny);
    };
    std::vector<long> row_off(Lv.bny + 1, 0);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < (long)nseg; k++) {
        long long jl, jh;
        row_span(k, jl, jh);
        for (long long j = jl; j < jh; j++) {
#pragma omp atomic
            row_off[j - Lv.bj0 + 1]++;
        }
    }
    for (int r = 0; r < Lv.bny; r++) row_off[r + 1] += row_off[r];
    std::vector<int> row_seg(row_off[Lv.bny]);
    std::vector<long> fill(row_off.begin(), row_off.end() - 1);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < (long)nseg; k++) {
        long long jl, jh;
        row_span(k, jl, jh);
        for (long long j = jl; j < jh; j++) {
            long at;
#pragma omp atomic capture
            at = fill[j - Lv.bj0]++;
            row_seg[at] = (int)k;
        }
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int r = 0; r < Lv.bny; r++) {
        long long j = Lv.bj0 + r;
        long long Y = (2 * j + 1) * hh;
        std::vector<uint8_t> diff(Lv.bnx + 1, 0);
        for (long m = row_off[r]; m < row_off[r + 1]; m++) {
            const int k = row_seg[m];
            IPt a = g.v[g.sa[k]], b = g.v[g.sb[k]];
            if (a.y > b.y) std::swap(a, b);
            i128 den = (i128)(b.y - a.y);
            i128 num = (i128)a.x * den + (i128)(Y - a.y) * (b.x - a.x);   // crossing x = num / den
            i128 M = (i128)hh * den;
            long long imax = fdiv((i128)cdiv(num, M) - 2, 2);             // last centre strictly left
            long long hi = std::min<long long>(imax, (long long)Lv.bi0 + Lv.bnx - 1);
            if (hi < Lv.bi0) continue;
            diff[0] ^= 1;
            diff[hi - Lv.bi0 + 1] ^= 1;
        }
        uint8_t par = 0;
        for (int c = 0; c < Lv.bnx; c++) {
            par ^= diff[c];
            Lv.solid[(size_t)r * Lv.bnx + c] = par;
        }
    }
    // centres lying exactly on a segment are solid
#pragma omp parallel for schedule(static)
    for (long k = 0; k < (long)nseg; k++) {
        IPt a = g.v[g.sa[k]], b = g.v[g.sb[k]];
        long long il = cdiv((i128)std::min(a.x, b.x) - hh, 2 * (i128)hh), ih = fdiv((i128)std::max(a.x, b.x) - hh, 2 * (i128)hh);
        long long jl = cdiv((i128)std::min(a.y, b.y) - hh, 2 * (i128)hh), jh = fdiv((i128)std::max(a.y, b.y) - hh, 2 * (i128)hh);
        for (long long j = jl; j <= jh; j++)
            for (long long i = il; i <= ih; i++) {
                long c = Lv.idx(i, j);
                if (c >= 0 && on_seg(a, b, centre(Lv, i, j))) {
#pragma omp atomic write
                    Lv.solid[c] = 1;
                }
            }
    }
#pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)Lv.solid.size(); c++)
        if (Lv.kind[c] == KIND_ABSENT) Lv.solid[c] = 0;
}

int build(const Spec &sp, const double *xy, const int *loop_off, int n_loops, Grid &g, std::string &msg)
{
    g = Grid();
    g.spec = sp;
    const int L = sp.levels;
    g.L = L;
    const double hf = sp.h0 / (double)(1LL << (L - 1));
    int nv = n_loops > 0 ? loop_off[n_loops] : 0;
    g.v.resize(nv);
    for (int k = 0; k < nv; k++) {
        g.v[k].x = llround((xy[2 * k] - sp.x0) / hf * (double)FIXU);
        g.v[k].y = llround((xy[2 * k + 1] - sp.y0) / hf * (double)FIXU);
    }
    g.loop_ccw.assign(std::max(n_loops, 1), 1);
    for (int lp = 0; lp < n_loops; lp++) {
        int a = loop_off[lp], b = loop_off[lp + 1];
        if (b - a < 3) return failmsg(msg, "loop with fewer than 3 vertices");
        i128 area2 = 0;
        int nl = 0;
        for (int k = a; k < b; k++) {
            int k2 = (k + 1 < b) ? k + 1 : a;
            // vertices that coincide after snapping are merged: no zero-length segments
            if (g.v[k].x == g.v[k2].x && g.v[k].y == g.v[k2].y) continue;
            g.sa.push_back(k); g.sb.push_back(k2); g.sloop.push_back(lp); nl++;
            area2 += (i128)g.v[k].x * g.v[k2].y - (i128)g.v[k2].x * g.v[k].y;
            if (std::llabs(g.v[k2].x - g.v[k].x) > (1LL << 30) || std::llabs(g.v[k2].y - g.v[k].y) > (1LL << 30))
                return failmsg(msg, "wall segment longer than 2^18 finest cells");
        }
        if (area2 == 0 || nl < 3) return failmsg(msg, "degenerate loop");
        g.loop_ccw[lp] = area2 > 0;
    }
    if (!sp.solid_walls) g.loop_ccw.assign(std::max(n_loops, 1), 1);
    SegTree T;
    T.init(g);
    // no two wall segments may cross: a loop that crosses itself or another loop has no
    // consistent inside.  Contacts without crossing (the zero-width tip a closed trailing
    // edge can leave after snapping, loops sharing an edge) are accepted.
    if (sp.solid_walls) {
        const long nseg = (long)g.sa.size();
        int bad = 0;
#pragma omp parallel
        {
        std::vector<int> cand;
#pragma omp for schedule(dynamic, 256)
        for (long k = 0; k < nseg; k++) {
            int flag;
#pragma omp atomic read
            flag = bad;
            if (flag) continue;
            const IPt a = g.v[g.sa[k]], b = g.v[g.sb[k]];
            T.overlapping((double)std::min(a.x, b.x) / FIXU - 1e-9, (double)std::min(a.y, b.y) / FIXU - 1e-9,
                          (double)std::max(a.x, b.x) / FIXU + 1e-9, (double)std::max(a.y, b.y) / FIXU + 1e-9, cand);
            for (int m : cand)
                if (m > k && segs_cross(a, b, g.v[g.sa[m]], g.v[g.sb[m]])) {
#pragma omp atomic write
                    bad = 1;
                }
        }
        }
        if (bad) return failmsg(msg, "wall loops cross themselves or each other");
    }

    g.lv.resize(L);
    for (int l = 0; l < L; l++) { g.lv[l].l = l; g.lv[l].scale = 1LL << (L - 1 - l); }
    alloc_level(g.lv[0], 0, 0, sp.nx0, sp.ny0);
    std::fill(g.lv[0].kind.begin(), g.lv[0].kind.end(), (uint8_t)KIND_ACTIVE);

    std::vector<long long> R(L, 0);
    R[L - 1] = (long long)sp.layers * FIXU;
    for (int l = L - 2; l >= 1; l--) R[l] = R[l + 1] + (long long)sp.layers * g.lv[l].scale * FIXU;

    // runs of consecutive segments whose joint bounding box stays within the smallest band
    // radius, and each run's bounding box
    std::vector<int> run_start;
    std::vector<long long> run_box;     // x0, x1, y0, y1 per run
    {
        const long long lim = R[L - 1];
        long long x0 = 0, x1 = 0, y0 = 0, y1 = 0;
        for (int k = 0; k < (int)g.sa.size(); k++) {
            IPt a = g.v[g.sa[k]], b = g.v[g.sb[k]];
            const long long ax = std::min(a.x, b.x), bx = std::max(a.x, b.x);
            const long long ay = std::min(a.y, b.y), by = std::max(a.y, b.y);
            if (run_start.empty() || std::max(bx, x1) - std::min(ax, x0) > lim || std::max(by, y1) - std::min(ay, y0) > lim ||
                k - run_start.back() >= 64) {
                if (!run_start.empty()) run_box.insert(run_box.end(), {x0, x1, y0, y1});
                run_start.push_back(k);
                x0 = ax; x1 = bx; y0 = ay; y1 = by;
            } else {
                x0 = std::min(x0, ax); x1 = std::max(x1, bx); y0 = std::min(y0, ay); y1 = std::max(y1, by);
            }
        }
        if (!run_start.empty()) run_box.insert(run_box.end(), {x0, x1, y0, y1});
        run_start.push_back((int)g.sa.size());
    }
    const long nruns = (long)run_start.size() - 1;
    // each run's capsule, in fixed units: the chord from its first to its last vertex and a
    // radius holding every vertex (plus a margin far above the rounding of these doubles);
    // every segment of the run lies in the capsule.  A run whose segments join end to end
    // also comes within `rad` of every chord point (the chain runs from one chord end to
    // the other), so a centre within R - rad of the chord is within R of a segment.
    std::vector<double> run_cap(6 * std::max(nruns, 0L));
    std::vector<uint8_t> run_chain(std::max(nruns, 0L));
    for (long ru = 0; ru < nruns; ru++) {
        const int k0 = run_start[ru], k1 = run_start[ru + 1];
        const IPt a = g.v[g.sa[k0]], b = g.v[g.sb[k1 - 1]];
        double *cp = &run_cap[6 * ru];
        cp[0] = (double)a.x; cp[1] = (double)a.y;
        cp[2] = (double)(b.x - a.x); cp[3] = (double)(b.y - a.y);
        const double l2 = cp[2] * cp[2] + cp[3] * cp[3];
        cp[4] = l2 > 0 ? 1.0 / l2 : 0.0;
        double r2 = 0.0;
        bool chain = true;
        for (int k = k0; k < k1; k++) {
            const IPt e0 = g.v[g.sa[k]], e1 = g.v[g.sb[k]];
            for (const IPt &e : {e0, e1}) {
                double t = (((double)e.x - cp[0]) * cp[2] + ((double)e.y - cp[1]) * cp[3]) * cp[4];
                t = t < 0 ? 0 : (t > 1 ? 1 : t);
                const double qx = cp[0] + t * cp[2] - (double)e.x, qy = cp[1] + t * cp[3] - (double)e.y;
                r2 = std::max(r2, qx * qx + qy * qy);
            }
            if (k + 1 < k1) {
                const IPt n0 = g.v[g.sa[k + 1]];
                chain = chain && n0.x == e1.x && n0.y == e1.y;
            }
        }
        cp[5] = std::sqrt(r2) + 1.0;
        run_chain[ru] = chain;
    }

    for (int l = 1; l < L; l++) {
        Level &P = g.lv[l - 1];
        const long long hh = P.scale * FIXU / 2;
        // refinement: a cell is covered iff its centre lies within R_l of a segment (exact
        // test).  Consecutive runs are grouped while the group's bounding box stays within
        // R_l / 2 (and at most 1/128 of the runs, to leave work for every thread), so that a
        // group's candidate cells (its box grown by R_l) are enumerated once; each candidate
        // is tested against the runs of the group whose box lies within R_l.  Groups run in
        // parallel; marks only go 0 -> 1.
        std::vector<long> group_start;
        {
            const long long glim = std::max(R[l] / 2, R[L - 1]);
            const long gmax = std::max(1L, nruns / 128);
            long long x0 = 0, x1 = 0, y0 = 0, y1 = 0;
            for (long ru = 0; ru < nruns; ru++) {
                const long long *b = &run_box[4 * ru];
                if (group_start.empty() || std::max(b[1], x1) - std::min(b[0], x0) > glim ||
                    std::max(b[3], y1) - std::min(b[2], y0) > glim || ru - group_start.back() >= gmax) {
                    group_start.push_back(ru);
                    x0 = b[0]; x1 = b[1]; y0 = b[2]; y1 = b[3];
                } else {
                    x0 = std::min(x0, b[0]); x1 = std::max(x1, b[1]); y0 = std::min(y0, b[2]); y1 = std::max(y1, b[3]);
                }
            }
            group_start.push_back(nruns);
        }
        const long ngroups = (long)group_start.size() - 1;
        std::vector<uint8_t> near(P.kind.size(), 0);
#pragma omp parallel for schedule(dynamic, 1)
        for (long gr = 0; gr < ngroups; gr++) {
            const long r0 = group_start[gr], r1 = group_start[gr + 1];
            long long x0 = LLONG_MAX, x1 = LLONG_MIN, y0 = LLONG_MAX, y1 = LLONG_MIN;
            for (long ru = r0; ru < r1; ru++) {
                const long long *b = &run_box[4 * ru];
                x0 = std::min(x0, b[0]); x1 = std::max(x1, b[1]); y0 = std::min(y0, b[2]); y1 = std::max(y1, b[3]);
            }
            long long il = cdiv((i128)x0 - R[l] - hh, 2 * (i128)hh);
            long long ih = fdiv((i128)x1 + R[l] - hh, 2 * (i128)hh);
            long long jl = cdiv((i128)y0 - R[l] - hh, 2 * (i128)hh);
            long long jh = fdiv((i128)y1 + R[l] - hh, 2 * (i128)hh);
            il = std::max<long long>(il, P.bi0); jl = std::max<long long>(jl, P.bj0);
            ih = std::min<long long>(ih, (long long)P.bi0 + P.bnx - 1);
            jh = std::min<long long>(jh, (long long)P.bj0 + P.bny - 1);
            for (long long j = jl; j <= jh; j++)
                for (long long i = il; i <= ih; i++) {
                    long c = P.idx(i, j);
                    uint8_t seen;
#pragma omp atomic read
                    seen = near[c];
                    if (seen || P.kind[c] != KIND_ACTIVE) continue;
                    const IPt pc = centre(P, i, j);
                    const double Rd = (double)R[l];
                    bool hit = false;
                    for (long ru = r0; ru < r1 && !hit; ru++) {
                        // every segment of a run lies in its bounding box: a centre farther
                        // than R from the box is farther than R from all of them
                        const long long *b = &run_box[4 * ru];
                        const i128 dx = pc.x < b[0] ? (i128)b[0] - pc.x : (pc.x > b[1] ? (i128)pc.x - b[1] : 0);
                        const i128 dy = pc.y < b[2] ? (i128)b[2] - pc.y : (pc.y > b[3] ? (i128)pc.y - b[3] : 0);
                        if (dx * dx + dy * dy > (i128)R[l] * R[l]) continue;
                        // the capsule settles the run unless the centre lies within its
                        // radius (plus a margin) of the distance R; the exact test does the rest
                        const double *cp = &run_cap[6 * ru];
                        double t = (((double)pc.x - cp[0]) * cp[2] + ((double)pc.y - cp[1]) * cp[3]) * cp[4];
                        t = t < 0 ? 0 : (t > 1 ? 1 : t);
                        const double qx = cp[0] + t * cp[2] - (double)pc.x, qy = cp[1] + t * cp[3] - (double)pc.y;
                        const double dc = std::sqrt(qx * qx + qy * qy);
                        if (dc - cp[5] > Rd + 1.0) continue;
                        if (run_chain[ru] && dc + cp[5] < Rd - 1.0) { hit = true; break; }
                        for (int k = run_start[ru]; k < run_start[ru + 1] && !hit; k++)
                            hit = within_r(g.v[g.sa[k]], g.v[g.sb[k]], pc, R[l]);
                    }
                    if (!hit) continue;
#pragma omp atomic write
                    near[c] = 1;
                }
        }
#pragma omp parallel for schedule(static)
        for (long c = 0; c < (long)near.size(); c++)
            if (near[c]) P.kind[c] = KIND_COVERED;
        // nesting checks, band, child box.  Rows run in parallel; each notes its first
        // violation, and the first row with one names the error (as a row-major scan would)
        long long ci0 = (1LL << 40), cj0 = (1LL << 40), ci1 = -(1LL << 40), cj1 = -(1LL << 40);
        std::vector<uint8_t> row_err(P.bny, 0);
#pragma omp parallel for schedule(dynamic, 8) reduction(min : ci0, cj0) reduction(max : ci1, cj1)
        for (int r = 0; r < P.bny; r++)
            for (int q = 0; q < P.bnx && !row_err[r]; q++) {
                if (P.kind[(size_t)r * P.bnx + q] != KIND_COVERED) continue;
                long long i = P.bi0 + q, j = P.bj0 + r;
                if (l == 1 && (i < 2 || j < 2 || i >= sp.nx0 - 2 || j >= sp.ny0 - 2)) { row_err[r] = 1; break; }
                for (int d = 1; d < 9; d++) {
                    long c = P.idx(i + CX[d], j + CY[d]);
                    if (c < 0 || (P.kind[c] != KIND_ACTIVE && P.kind[c] != KIND_COVERED)) { row_err[r] = 2; break; }
                    if (P.kind[c] == KIND_ACTIVE) {
#pragma omp atomic write
                        P.band[c] = 1;
                    }
                }
                ci0 = std::min(ci0, i - 1); cj0 = std::min(cj0, j - 1);
                ci1 = std::max(ci1, i + 1); cj1 = std::max(cj1, j + 1);
            }
        for (int r = 0; r < P.bny; r++) {
            if (row_err[r] == 1) return failmsg(msg, "refinement reaches the level-0 box edge");
            if (row_err[r] == 2) return failmsg(msg, "refinement band violates 2:1 nesting (increase layers)");
        }
        if (ci1 < ci0) return failmsg(msg, "level has no cells (wall far from the box?)");
        Level &F = g.lv[l];
        alloc_level(F, (int)(2 * ci0 - 1), (int)(2 * cj0 - 1), (int)(2 * (ci1 - ci0 + 1) + 2), (int)(2 * (cj1 - cj0 + 1) + 2));
#pragma omp parallel for schedule(static)
        for (long long j = cj0; j <= cj1; j++)
            for (long long i = ci0; i <= ci1; i++) {
                long c = P.idx(i, j);
                uint8_t kd = P.kind[c] == KIND_COVERED ? KIND_ACTIVE : (P.band[c] ? KIND_GHOST : KIND_ABSENT);
                if (kd == KIND_ABSENT) continue;
                for (int b = 0; b < 2; b++)
                    for (int a = 0; a < 2; a++) F.kind[F.idx(2 * i + a, 2 * j + b)] = kd;
            }
    }
    // coalescence: pulled direction d of band cell c comes from the fine ghosts iff
    // c - c_d, c - (c_dx, 0) or c - (0, c_dy) is covered
    for (int l = 0; l < L - 1; l++) {
        Level &P = g.lv[l];
#pragma omp parallel for schedule(static)
        for (int r = 0; r < P.bny; r++)
            for (int q = 0; q < P.bnx; q++) {
                size_t c = (size_t)r * P.bnx + q;
                if (!P.band[c]) continue;
                long long i = P.bi0 + q, j = P.bj0 + r;
                uint16_t m = 0;
                for (int d = 1; d < 9; d++) {
                    long n3[3] = {P.idx(i - CX[d], j - CY[d]), P.idx(i - CX[d], j), P.idx(i, j - CY[d])};
                    for (long cc : n3)
                        if (cc >= 0 && P.kind[cc] == KIND_COVERED) { m |= (uint16_t)(1u << d); break; }
                }
                P.coal[c] = m;
            }
    }
    // solid painting
    if (sp.solid_walls && !g.sa.empty())
        for (int l = 0; l < L; l++) paint_solid(g, g.lv[l]);
    // cut links; walls may only touch active cells of the finest level
    for (int l = 0; l < L; l++) {
        Level &P = g.lv[l];
        int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
        for (int r = 0; r < P.bny; r++)
            for (int q = 0; q < P.bnx; q++) {
                size_t c = (size_t)r * P.bnx + q;
                if (P.kind[c] == KIND_ABSENT || P.kind[c] == KIND_COVERED || P.solid[c]) continue;
                long long i = P.bi0 + q, j = P.bj0 + r;
                uint16_t m = 0;
                for (int d = 1; d < 9; d++) {
                    long long si = i - CX[d], sj = j - CY[d];
                    if (l == 0 && sp.periodic) { si = (si + sp.nx0) % sp.nx0; sj = (sj + sp.ny0) % sp.ny0; }
                    long cc = P.idx(si, sj);
                    if (cc >= 0 && P.kind[cc] != KIND_ABSENT && P.solid[cc]) m |= (uint16_t)(1u << d);
                }
                if (!m) continue;
                if (l != L - 1 || P.kind[c] != KIND_ACTIVE) { bad = 1; continue; }
                P.cut[c] = m;
                P.bnode[c] = 1;
            }
        if (bad) return failmsg(msg, "wall reaches a cell that is not on the finest active level");
    }
    // wall distance of active fluid cells
    for (int l = 0; l < L; l++) {
        Level &P = g.lv[l];
#pragma omp parallel for schedule(dynamic, 4)
        for (int r = 0; r < P.bny; r++) {
            // the search for a cell starts from the nearest segment of the previous cell in
            // the row, whose leaf usually holds or neighbours the new nearest segment
            int kprev = -1;
            for (int q = 0; q < P.bnx; q++) {
                size_t c = (size_t)r * P.bnx + q;
                if (P.kind[c] != KIND_ACTIVE || P.solid[c]) continue;
                double dd = DCAP;
                if (sp.solid_walls && !g.sa.empty()) {
                    double px = (P.bi0 + q + 0.5) * (double)P.scale, py = (P.bj0 + r + 0.5) * (double)P.scale;
                    int kb = -1;
                    const double d = kprev >= 0 ? T.nearest_dist_from(px, py, kprev, kb)
                                                : T.nearest_dist(px, py, std::numeric_limits<double>::infinity(), kb);
                    kprev = kb;
                    dd = d / (double)P.scale;
                    if (dd > DCAP) dd = DCAP;
                }
                P.dist[c] = dd;
            }
        }
    }
    // wall records in (j, i) order at the finest level: the boundary nodes are listed row by
    // row, then each record is built independently; an error is reported for the first
    // record, in that order, that has one (the same one a sequential build meets first)
    Level &Fn = g.lv[L - 1];
    std::vector<long> bcell;
    {
        std::vector<std::vector<long>> per_row(Fn.bny);
#pragma omp parallel for schedule(dynamic, 16)
        for (int r = 0; r < Fn.bny; r++)
            for (int q = 0; q < Fn.bnx; q++)
                if (Fn.bnode[(size_t)r * Fn.bnx + q]) per_row[r].push_back((long)r * Fn.bnx + q);
        for (auto &v : per_row) bcell.insert(bcell.end(), v.begin(), v.end());
    }
    const long nrec = (long)bcell.size();
    g.recs.resize(nrec);
    std::vector<int> rec_err(nrec, 0);
    long long n_cut = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : n_cut)
    for (long k = 0; k < nrec; k++) {
        const long c = bcell[k];
        const int r = (int)(c / Fn.bnx), q = (int)(c % Fn.bnx);
        Record &rc = g.recs[k];
        std::memset(&rc, 0, sizeof rc);
        rc.i = Fn.bi0 + q; rc.j = Fn.bj0 + r;
        double bx = rc.i + 0.5, by = rc.j + 0.5, cx, cy;
        int kb;
        double dwb = T.nearest(bx, by, kb, cx, cy);
        rc.seg = kb; rc.loop = g.sloop[kb];
        rc.iw[0] = cx; rc.iw[1] = cy; rc.dwb = dwb;
        rc.n[0] = (bx - cx) / dwb; rc.n[1] = (by - cy) / dwb;
        rc.r[0] = cx + sp.d_wr * rc.n[0]; rc.r[1] = cy + sp.d_wr * rc.n[1];
        IPt pb = centre(Fn, rc.i, rc.j);
        int err = 0;
        for (int d = 1; d < 9 && !err; d++) {
            if (!(Fn.cut[c] >> d & 1)) continue;
            double t = link_q(g, T, pb, IPt{-CX[d] * FIXU, -CY[d] * FIXU});
            if (t > 1.0) { err = 1; break; }
            rc.q[d] = t;
            n_cut++;
        }
        int ic = (int)std::floor(rc.r[0] - 0.5), jc = (int)std::floor(rc.r[1] - 0.5);
        rc.ns = 0;
        for (int b = -1; b <= 2 && !err; b++)
            for (int a = -1; a <= 2; a++) {
                long cc = Fn.idx(ic + a, jc + b);
                bool act = cc >= 0 && Fn.kind[cc] == KIND_ACTIVE;
                if (sp.wall_model <= 1 && !act) { err = 2; break; }
                if (!act || Fn.solid[cc] || Fn.bnode[cc]) continue;
                rc.si[rc.ns] = ic + a; rc.sj[rc.ns] = jc + b; rc.ns++;
            }
        if (!err && sp.wall_model <= 1 && rc.ns == 0) err = 3;
        rec_err[k] = err;
        Fn.rec[c] = (int)k;
    }
    for (long k = 0; k < nrec; k++) {
        if (rec_err[k] == 1) return failmsg(msg, "cut link without a wall crossing");
        if (rec_err[k] == 2) return failmsg(msg, "reference point stencil leaves the finest active level");
        if (rec_err[k] == 3) return failmsg(msg, "empty reference stencil");
    }
    g.n_cut = n_cut;
    // surface element centroid -> two nearest boundary nodes (ties: lower record index)
    size_t nseg = g.sa.size();
    g.seg_b1.assign(nseg, -1); g.seg_b2.assign(nseg, -1); g.seg_w1.assign(nseg, 0); g.seg_w2.assign(nseg, 0);
    if (!g.recs.empty()) {
        const int BK = 4;
        int mi = 1 << 30, mj = 1 << 30, Mi = -(1 << 30), Mj = -(1 << 30);
        for (auto &rc : g.recs) { mi = std::min(mi, rc.i); mj = std::min(mj, rc.j); Mi = std::max(Mi, rc.i); Mj = std::max(Mj, rc.j); }
        int gbx0 = (int)fdiv(mi, BK), gby0 = (int)fdiv(mj, BK);
        int gnx = (int)fdiv(Mi, BK) - gbx0 + 1, gny = (int)fdiv(Mj, BK) - gby0 + 1;
        std::vector<std::vector<int>> bucket((size_t)gnx * gny);
        for (size_t k = 0; k < g.recs.size(); k++)
            bucket[(size_t)(fdiv(g.recs[k].j, BK) - gby0) * gnx + (fdiv(g.recs[k].i, BK) - gbx0)].push_back((int)k);
#pragma omp parallel for schedule(dynamic, 16)
        for (long k = 0; k < (long)nseg; k++) {
            double mx = 0.5 * (double)(g.v[g.sa[k]].x + g.v[g.sb[k]].x) / FIXU;
            double my = 0.5 * (double)(g.v[g.sa[k]].y + g.v[g.sb[k]].y) / FIXU;
            int cbx = (int)std::floor(mx / BK) - gbx0, cby = (int)std::floor(my / BK) - gby0;
            double d1 = INFINITY, d2 = INFINITY;
            int b1 = -1, b2 = -1;
            for (int ring = 0;; ring++) {
                for (int by = cby - ring; by <= cby + ring; by++)
                    for (int bx = cbx - ring; bx <= cbx + ring; bx++) {
                        if (std::max(std::abs(bx - cbx), std::abs(by - cby)) != ring) continue;
                        if (bx < 0 || by < 0 || bx >= gnx || by >= gny) continue;
                        for (int rr : bucket[(size_t)by * gnx + bx]) {
                            double dx = g.recs[rr].i + 0.5 - mx, dy = g.recs[rr].j + 0.5 - my;
                            double dd = dx * dx + dy * dy;
                            if (dd < d1 || (dd == d1 && rr < b1)) { d2 = d1; b2 = b1; d1 = dd; b1 = rr; }
                            else if (dd < d2 || (dd == d2 && rr < b2)) { d2 = dd; b2 = rr; }
                        }
                    }
                double reach = (double)ring * BK;
                bool all_out = (cbx - ring <= 0 && cby - ring <= 0 && cbx + ring >= gnx - 1 && cby + ring >= gny - 1);
                if ((b2 >= 0 && d2 <= reach * reach) || all_out) break;
            }
            g.seg_b1[k] = b1; g.seg_b2[k] = b2;
            g.seg_w1[k] = b1 >= 0 ? 1.0 / (d1 > 1e-300 ? d1 : 1e-300) : 0.0;
            g.seg_w2[k] = b2 >= 0 ? 1.0 / (d2 > 1e-300 ? d2 : 1e-300) : 0.0;
        }
    }
    // tiles
    for (int l = 0; l < L; l++) {
        Level &P = g.lv[l];
        int a0 = 1 << 30, b0 = 1 << 30, a1 = -(1 << 30), b1 = -(1 << 30);
#pragma omp parallel for schedule(static) reduction(min : a0, b0) reduction(max : a1, b1)
        for (int r = 0; r < P.bny; r++)
            for (int q = 0; q < P.bnx; q++)
                if (P.kind[(size_t)r * P.bnx + q] != KIND_ABSENT) {
                    a0 = std::min(a0, P.bi0 + q); a1 = std::max(a1, P.bi0 + q);
                    b0 = std::min(b0, P.bj0 + r); b1 = std::max(b1, P.bj0 + r);
                }
        P.pi0 = a0; P.pj0 = b0; P.pnx = a1 - a0 + 1; P.pny = b1 - b0 + 1;
        P.tx0 = (int)fdiv(a0, LBM_TX); P.ty0 = (int)fdiv(b0, LBM_TY);
        P.ntx = (int)fdiv(a1, LBM_TX) - P.tx0 + 1; P.nty = (int)fdiv(b1, LBM_TY) - P.ty0 + 1;
        P.tile_of.assign((size_t)P.ntx * P.nty, -1);
        P.tile_x.clear(); P.tile_y.clear();
        // Level 0 keeps every tile of its box in row-major order (the box-edge conditions
        // address it arithmetically).  Finer levels keep tiles with at least one non-solid
        // present cell -- solid cells carry no state: no population is ever pulled from
        // them and no stencil reads them -- and list tiles with boundary nodes first, so
        // that their wall-function work starts in the first wave of every launch.
        // tile classes of each tile row (0 wall tiles, 1 the others, 2 none), then the two
        // lists in row-major order
        std::vector<uint8_t> tcls((size_t)P.ntx * P.nty, 2);
#pragma omp parallel for schedule(dynamic, 4)
        for (int ty = 0; ty < P.nty; ty++)
            for (int tx = 0; tx < P.ntx; tx++) {
                bool any = false, wall = false;
                int gx = (P.tx0 + tx) * LBM_TX, gy = (P.ty0 + ty) * LBM_TY;
                for (int y = 0; y < LBM_TY; y++)
                    for (int x = 0; x < LBM_TX; x++) {
                        long c = P.idx(gx + x, gy + y);
                        if (c < 0 || P.kind[c] == KIND_ABSENT) continue;
                        if (l == 0 || !P.solid[c]) any = true;
                        if (P.bnode[c]) wall = true;
                    }
                if (any) tcls[(size_t)ty * P.ntx + tx] = (l > 0 && wall) ? 0 : 1;
            }
        for (int cls = 0; cls < 2; cls++) {
            for (int ty = 0; ty < P.nty; ty++)
                for (int tx = 0; tx < P.ntx; tx++) {
                    if (tcls[(size_t)ty * P.ntx + tx] != cls) continue;
                    P.tile_of[(size_t)ty * P.ntx + tx] = (int)P.tile_x.size();
                    P.tile_x.push_back(P.tx0 + tx); P.tile_y.push_back(P.ty0 + ty);
                }
            if (cls == 0) P.n_wall_tiles = (int)P.tile_x.size();
        }
        P.ntiles = (int)P.tile_x.size();
        // tiles with a non-solid band cell (explosion, prolongation) and tiles with a
        // non-solid active or ghost cell (the level kernel's work list)
        std::vector<uint8_t> tband(P.ntiles, 0), twork(P.ntiles, 0);
#pragma omp parallel for schedule(dynamic, 64)
        for (int t = 0; t < P.ntiles; t++) {
            bool band = false, work = false;
            for (int y = 0; y < LBM_TY; y++)
                for (int x = 0; x < LBM_TX; x++) {
                    long c = P.idx(P.tile_x[t] * LBM_TX + x, P.tile_y[t] * LBM_TY + y);
                    if (c < 0 || P.solid[c]) continue;
                    band = band || P.band[c];
                    work = work || P.kind[c] == KIND_ACTIVE || P.kind[c] == KIND_GHOST;
                }
            tband[t] = band; twork[t] = work;
        }
        P.band_tiles.clear();
        P.work_tiles.clear();
        for (int t = 0; t < P.ntiles; t++) {
            if (tband[t]) P.band_tiles.push_back(t);
            if (twork[t]) P.work_tiles.push_back(t);
        }
        P.nbr.assign((size_t)P.ntiles * 9, -1);
        const bool wrap = (l == 0 && sp.periodic);
        const int wtx = sp.nx0 / LBM_TX, wty = sp.ny0 / LBM_TY;
        for (int t = 0; t < P.ntiles; t++)
            for (int d = 0; d < 9; d++) {
                int tx = P.tile_x[t] + CX[d], ty = P.tile_y[t] + CY[d];
                if (wrap) { tx = (tx % wtx + wtx) % wtx; ty = (ty % wty + wty) % wty; }
                if (tx < P.tx0 || ty < P.ty0 || tx >= P.tx0 + P.ntx || ty >= P.ty0 + P.nty) continue;
                P.nbr[(size_t)t * 9 + d] = P.tile_of[(size_t)(ty - P.ty0) * P.ntx + (tx - P.tx0)];
            }
    }
    for (int l = 0; l < L; l++) {
        Level &P = g.lv[l];
        P.parent.assign((size_t)P.ntiles, -1);
        if (l == 0) continue;
        const Level &C = g.lv[l - 1];
        for (int t = 0; t < P.ntiles; t++) {
            int tx = P.tile_x[t] >> 1, ty = P.tile_y[t] >> 1;
            if (tx < C.tx0 || ty < C.ty0 || tx >= C.tx0 + C.ntx || ty >= C.ty0 + C.nty) continue;
            P.parent[t] = C.tile_of[(size_t)(ty - C.ty0) * C.ntx + (tx - C.tx0)];
        }
    }
    for (int l = 0; l < L; l++) {
        Level &P = g.lv[l];
        P.child.assign((size_t)P.ntiles * 4, -1);
        if (l == L - 1) continue;
        Level &F = g.lv[l + 1];
        for (int t = 0; t < P.ntiles; t++)
            for (int b = 0; b < 2; b++)
                for (int a = 0; a < 2; a++) {
                    int tx = 2 * P.tile_x[t] + a, ty = 2 * P.tile_y[t] + b;
                    if (tx < F.tx0 || ty < F.ty0 || tx >= F.tx0 + F.ntx || ty >= F.ty0 + F.nty) continue;
                    P.child[(size_t)t * 4 + b * 2 + a] = F.tile_of[(size_t)(ty - F.ty0) * F.ntx + (tx - F.tx0)];
                }
    }
    return 0;
}

}  // namespace lbmgrid
