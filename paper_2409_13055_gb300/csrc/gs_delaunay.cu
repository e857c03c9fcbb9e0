// gs_delaunay.cu -- Delaunay triangulation of tracked pixels (paper Sec.
// III-A: the image is divided into triangles with the tracked pixels as
// vertices, and points in flat regions take the mean depth of their
// triangle's vertices).  Host code: the triangulation is built on the CPU
// while the GPU selects the pixels and interpolates (gs_pointcloud.cu).
//
// Bowyer-Watson insertion with exact predicates on integer coordinates
// (orientation in 64-bit, in-circle in 128-bit integers) and "ghost"
// triangles for the outside: every hull edge (a, b) carries a triangle
// (a, b, inf) whose "circumcircle" is the open half-plane beyond the edge
// plus the open edge itself, so no finite super-triangle can perturb the
// hull.  Points are inserted along a Z-order curve and located by walking
// from the previous insertion, so each insertion touches O(1) triangles on
// average.  On co-circular points the in-circle test is strict, so the
// result is one of the valid Delaunay triangulations.
#include <algorithm>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "gs.h"

namespace {

struct Tri {
    int v[3];   // counter-clockwise; -1 = the vertex at infinity (always v[2])
    int nb[3];  // neighbour across the edge opposite v[i]
    bool alive;
};

using i64 = long long;
using i128 = __int128;

struct Del {
    const int32_t* xy;
    std::vector<Tri> t;
    std::vector<int> mark;  // insertion stamp of the cavity search
    int stamp = 0;

    i64 X(int i) const { return xy[2 * i]; }
    i64 Y(int i) const { return xy[2 * i + 1]; }

    i64 orient(int a, int b, int c) const {
        return (X(b) - X(a)) * (Y(c) - Y(a)) - (Y(b) - Y(a)) * (X(c) - X(a));
    }

    // > 0: d strictly inside the circle through the CCW triangle a, b, c
    bool incircle(int a, int b, int c, int d) const {
        const i64 adx = X(a) - X(d), ady = Y(a) - Y(d);
        const i64 bdx = X(b) - X(d), bdy = Y(b) - Y(d);
        const i64 cdx = X(c) - X(d), cdy = Y(c) - Y(d);
        const i128 al = (i128)adx * adx + (i128)ady * ady;
        const i128 bl = (i128)bdx * bdx + (i128)bdy * bdy;
        const i128 cl = (i128)cdx * cdx + (i128)cdy * cdy;
        const i128 det = (i128)adx * ((i128)bdy * cl - (i128)cdy * bl) -
                         (i128)ady * ((i128)bdx * cl - (i128)cdx * bl) +
                         al * ((i128)bdx * cdy - (i128)cdx * bdy);
        return det > 0;
    }

    // p in the circumcircle of triangle k (the half-plane test for ghosts)
    bool in_circum(int k, int p) const {
        const Tri& T = t[k];
        if (T.v[2] >= 0) return incircle(T.v[0], T.v[1], T.v[2], p);
        const int a = T.v[0], b = T.v[1];
        const i64 o = orient(a, b, p);
        if (o != 0) return o > 0;
        // on the hull line: inside iff strictly between a and b
        const i64 d = (X(p) - X(a)) * (X(b) - X(a)) + (Y(p) - Y(a)) * (Y(b) - Y(a));
        const i64 l = (X(b) - X(a)) * (X(b) - X(a)) + (Y(b) - Y(a)) * (Y(b) - Y(a));
        return d > 0 && d < l;
    }

    // A triangle (real or ghost) whose circumcircle contains p, found by a
    // visibility walk from triangle `start`.
    int locate(int start, int p) const {
        int k = start;
        for (long long steps = 0; steps < (long long)4 * (long long)t.size() + 16; ++steps) {
            const Tri& T = t[k];
            if (T.v[2] < 0) return k;  // a ghost: p is beyond the hull edge (or on it)
            int next = -1;
            for (int i = 0; i < 3 && next < 0; ++i) {
                const int a = T.v[(i + 1) % 3], b = T.v[(i + 2) % 3];
                if (orient(a, b, p) < 0) next = T.nb[i];
            }
            if (next < 0) return k;  // p inside or on the boundary of T
            k = next;
        }
        return -1;  // cannot happen for a valid triangulation; reported as an error
    }

    int add(int a, int b, int c) {
        Tri T;
        T.v[0] = a; T.v[1] = b; T.v[2] = c;
        T.nb[0] = T.nb[1] = T.nb[2] = -1;
        T.alive = true;
        t.push_back(T);
        mark.push_back(0);
        return (int)t.size() - 1;
    }

    // edge (a -> b) of triangle k: index of the opposite vertex
    static int edge_index(const Tri& T, int a, int b) {
        for (int i = 0; i < 3; ++i)
            if (T.v[(i + 1) % 3] == a && T.v[(i + 2) % 3] == b) return i;
        return -1;
    }

    // Inserts p; returns a new triangle containing p, or -1 on failure.
    int insert(int start, int p) {
        const int k0 = locate(start, p);
        if (k0 < 0 || !in_circum(k0, p)) return -1;
        ++stamp;
        std::vector<int> bad{k0}, stack{k0};
        mark[k0] = stamp;
        while (!stack.empty()) {
            const int k = stack.back();
            stack.pop_back();
            for (int i = 0; i < 3; ++i) {
                const int q = t[k].nb[i];
                if (q < 0 || mark[q] == stamp) continue;
                if (in_circum(q, p)) {
                    mark[q] = stamp;
                    bad.push_back(q);
                    stack.push_back(q);
                }
            }
        }
        // the cavity's boundary edges, each turned into a triangle with p
        struct Edge { int a, b, outside; };
        std::vector<Edge> edges;
        for (int k : bad)
            for (int i = 0; i < 3; ++i) {
                const int q = t[k].nb[i];
                if (q >= 0 && mark[q] == stamp) continue;
                edges.push_back({t[k].v[(i + 1) % 3], t[k].v[(i + 2) % 3], q});
            }
        for (int k : bad) t[k].alive = false;
        std::unordered_map<long long, int> by_edge;  // directed edge (u -> v) -> new triangle
        auto key = [](int u, int v) { return ((long long)(u + 1) << 32) ^ (unsigned)(v + 1); };
        int last = -1;
        for (const Edge& e : edges) {
            // triangle (a, b, p), with the infinite vertex rotated last
            int k;
            if (e.a < 0) k = add(e.b, p, -1);
            else if (e.b < 0) k = add(p, e.a, -1);
            else k = add(e.a, e.b, p);
            Tri& T = t[k];
            // the outside neighbour across edge (a, b)
            const int io = edge_index(T, e.a, e.b);
            T.nb[io] = e.outside;
            if (e.outside >= 0) {
                const int j = edge_index(t[e.outside], e.b, e.a);
                if (j >= 0) t[e.outside].nb[j] = k;
            }
            for (int i = 0; i < 3; ++i) by_edge[key(T.v[(i + 1) % 3], T.v[(i + 2) % 3])] = k;
            if (T.v[2] >= 0) last = k;
        }
        // link the fan: each new edge (u -> v) meets its reverse (v -> u)
        for (size_t s = t.size() - edges.size(); s < t.size(); ++s) {
            Tri& T = t[s];
            for (int i = 0; i < 3; ++i) {
                if (T.nb[i] >= 0) continue;
                const int u = T.v[(i + 1) % 3], v = T.v[(i + 2) % 3];
                auto it = by_edge.find(key(v, u));
                if (it != by_edge.end()) T.nb[i] = it->second;
            }
        }
        return last >= 0 ? last : (int)t.size() - 1;
    }
};

long long morton(int32_t x, int32_t y) {
    long long m = 0;
    for (int b = 0; b < 21; ++b)
        m |= ((long long)((x >> b) & 1) << (2 * b)) | ((long long)((y >> b) & 1) << (2 * b + 1));
    return m;
}

}  // namespace

extern "C" gs_status gs_delaunay(const int32_t* xy_host, int32_t n, int32_t* tri_host,
                                 int32_t tri_capacity, int32_t* n_tri) {
    if (!xy_host || !n_tri || n < 0 || tri_capacity < 0 || (tri_capacity > 0 && !tri_host))
        return GS_ERR_INVALID;
    *n_tri = 0;
    for (int i = 0; i < n; ++i)
        if (xy_host[2 * i] < 0 || xy_host[2 * i] >= (1 << 20) || xy_host[2 * i + 1] < 0 ||
            xy_host[2 * i + 1] >= (1 << 20))
            return GS_ERR_INVALID;
    if (n < 3) return GS_OK;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return morton(xy_host[2 * a], xy_host[2 * a + 1]) < morton(xy_host[2 * b], xy_host[2 * b + 1]);
    });
    for (int i = 1; i < n; ++i)
        if (xy_host[2 * order[i]] == xy_host[2 * order[i - 1]] &&
            xy_host[2 * order[i] + 1] == xy_host[2 * order[i - 1] + 1])
            return GS_ERR_INVALID;  // duplicate points
    Del d;
    d.xy = xy_host;
    d.t.reserve((size_t)6 * n + 16);
    // first triangle: the first point, the next one, and the first point off
    // their line (points before it are collinear and inserted afterwards)
    const int a = order[0], b = order[1];
    int c_pos = -1;
    for (int i = 2; i < n && c_pos < 0; ++i)
        if (d.orient(a, b, order[i]) != 0) c_pos = i;
    if (c_pos < 0) return GS_OK;  // all collinear: no triangle
    int c = order[c_pos];
    int A = a, Bv = b, C = c;
    if (d.orient(A, Bv, C) < 0) std::swap(Bv, C);
    const int t0 = d.add(A, Bv, C);
    // ghosts on the three hull edges, each (u, v, inf) with the outside left of u -> v
    const int g0 = d.add(Bv, A, -1), g1 = d.add(C, Bv, -1), g2 = d.add(A, C, -1);
    // neighbours of t0: across edge opposite A = (Bv, C) -> ghost (C, Bv)
    d.t[t0].nb[0] = g1;
    d.t[t0].nb[1] = g2;
    d.t[t0].nb[2] = g0;
    auto link_ghost = [&](int g, int prev, int next) {
        // ghost (u, v, inf): nb[2] across (u, v) is t0; nb[0] across (v, inf),
        // nb[1] across (inf, u)
        d.t[g].nb[2] = t0;
        d.t[g].nb[0] = next;
        d.t[g].nb[1] = prev;
    };
    // hull (clockwise as seen from outside): g0 = (Bv, A), g2 = (A, C), g1 = (C, Bv)
    link_ghost(g0, g1, g2);
    link_ghost(g2, g0, g1);
    link_ghost(g1, g2, g0);
    int last = t0;
    for (int i = 2; i < n; ++i) {
        if (i == c_pos) continue;
        const int r = d.insert(last, order[i]);
        if (r < 0) return GS_ERR_INVALID;
        last = r;
    }
    int cnt = 0;
    for (const Tri& T : d.t) {
        if (!T.alive || T.v[2] < 0) continue;
        if (cnt < tri_capacity) {
            tri_host[3 * cnt] = T.v[0];
            tri_host[3 * cnt + 1] = T.v[1];
            tri_host[3 * cnt + 2] = T.v[2];
        }
        ++cnt;
    }
    *n_tri = cnt;
    return cnt > tri_capacity ? GS_ERR_CAPACITY : GS_OK;
}
