// quad_tables.h -- host-side tables of a mesh of the paper's 9-node
// quadrilaterals (Sec. III): element frames (corners unwrapped across
// periodic boundaries), neighbours across the four edges with their frame
// shifts, tie-break ranks (larger computational area first, then lower
// original id), node fans, owner elements (Sec. IV), the wall condition's
// gradient elements (reading R8), wall normals and probe points B located
// by Newton's method on the bilinear map (Sec. IV.A), Morton renumbering.
// The generic fields of HostTables (sizes, node order, coordinates, map
// factors) are filled as for the triangles, so that the code shared by
// both element kinds reads them unchanged.
#pragma once
#include "quad.cuh"
#include "tables.h"

namespace alelb {

struct QuadTables {
    std::vector<double2> ev;       // [4E] corners in each element's frame
    std::vector<int> nbr;          // [4E] neighbour across edge k, -1 on a boundary
    std::vector<uint32_t> einfo;   // [E] byte k: kind(2) | nbr edge(2) | dsx+1(2) | dsy+1(2)
    std::vector<int> rank, conn, orig, fan_ptr, wall_idx, probe_e;
    std::vector<int2> fan, owner, bcel, wedges;
    std::vector<uint8_t> bkind;
    std::vector<double2> probe_xi, wall_nrm;
    // the certified FP32 decisions of the deviation forms
    std::vector<float4> Xf;  // [N] node coordinates split hi + lo in FP32
    std::vector<float4> evf; // [4E] corners split hi + lo in FP32
    std::vector<float> bdist; // [N] lower bound of the distance to the nearest boundary edge
    // the FP32 derivative passes: J^{-1} of the owner element's bilinear map
    // at the node, (d xi/dX, d xi/dY, d eta/dX, d eta/dY)
    std::vector<float4> ownJf; // [N]
};

// Local coordinates of p in the quadrilateral with corners w (x, y pairs),
// by the Newton iteration the kernels use (centre start, QUAD_NEWTON_ITERS
// steps); false when it has not converged.
inline bool host_quad_local(const double w[8], double px, double py, double &xi, double &eta)
{
    double c[8];
    for (int k = 0; k < 4; ++k) {
        c[2 * k] = w[2 * k] - px;
        c[2 * k + 1] = w[2 * k + 1] - py;
    }
    return quad_newton(c, xi, eta);
}

inline alelb_status build_quad_tables(const alelb_mesh_desc *d, HostTables &T, QuadTables &Q, std::string &err)
{
    if (!d || d->n_nodes <= 0 || d->n_elems <= 0 || !d->X || !d->conn || !d->edge_kind) {
        err = "null pointer or empty mesh";
        return ALELB_ERR_ARG;
    }
    const int N = d->n_nodes, E = d->n_elems;
    if (E > CACHE_ELEM) {
        err = "more than 2^25 - 1 elements";
        return ALELB_ERR_ARG;
    }
    T.N = N;
    T.E = E;
    T.Lx = d->period[0] > 0 ? d->period[0] : 0.0;
    T.Ly = d->period[1] > 0 ? d->period[1] : 0.0;
    T.mkind = d->motion_kind;
    std::memcpy(T.mp, d->motion, sizeof(T.mp));
    if (T.mkind < 0 || T.mkind > MK_BLENDED) { err = "unknown motion kind"; return ALELB_ERR_ARG; }
    const double *X = d->X;
    const int *C = d->conn;
    for (long k = 0; k < 9L * E; ++k)
        if (C[k] < 0 || C[k] >= N) { err = "connectivity out of range"; return ALELB_ERR_MESH; }
    // element frames (original order), doubled areas, shape checks
    std::vector<double2> fr((size_t)4 * E);
    std::vector<double> area2(E);
    for (int e = 0; e < E; ++e) {
        const int *c = C + 9 * e;
        const double x0 = X[2 * c[0]], y0 = X[2 * c[0] + 1];
        double w[18];
        for (int l = 0; l < 9; ++l) {
            w[2 * l] = x0 + unwrap1(X[2 * c[l]] - x0, T.Lx);
            w[2 * l + 1] = y0 + unwrap1(X[2 * c[l] + 1] - y0, T.Ly);
        }
        for (int k = 0; k < 4; ++k) {
            const int k1 = (k + 1) % 4, k2 = (k + 2) % 4;
            if (w[8 + 2 * k] != 0.5 * (w[2 * k] + w[2 * k1]) || w[9 + 2 * k] != 0.5 * (w[2 * k + 1] + w[2 * k1 + 1]))
                { err = "a midside node is not its edge's exact midpoint"; return ALELB_ERR_MESH; }
            const double cr = (w[2 * k1] - w[2 * k]) * (w[2 * k2 + 1] - w[2 * k1 + 1]) -
                              (w[2 * k1 + 1] - w[2 * k + 1]) * (w[2 * k2] - w[2 * k1]);
            if (!(cr > 0)) { err = "a quadrilateral is not strictly convex (or is inverted)"; return ALELB_ERR_MESH; }
            fr[4 * e + k] = make_double2(w[2 * k], w[2 * k + 1]);
        }
        if (w[16] != 0.25 * (((w[0] + w[2]) + w[4]) + w[6]) || w[17] != 0.25 * (((w[1] + w[3]) + w[5]) + w[7]))
            { err = "a centre node is not the mean of its cell's corners"; return ALELB_ERR_MESH; }
        area2[e] = (w[4] - w[0]) * (w[7] - w[3]) - (w[6] - w[2]) * (w[5] - w[1]);
    }
    std::vector<int> order(E);
    for (int e = 0; e < E; ++e) order[e] = e;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        if (area2[a] != area2[b]) return area2[a] > area2[b];
        return a < b;
    });
    std::vector<int> rank_o(E);
    for (int r = 0; r < E; ++r) rank_o[order[r]] = r;
    // renumbering: Morton order of nodes and cell centres
    T.node_old2new.resize(N);
    T.node_new2old.resize(N);
    T.elem_old2new.resize(E);
    T.elem_new2old.resize(E);
    for (int a = 0; a < N; ++a) T.node_new2old[a] = a;
    for (int e = 0; e < E; ++e) T.elem_new2old[e] = e;
    if (d->renumber == ALELB_RENUMBER_MORTON) {
        double x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
        for (int a = 0; a < N; ++a) {
            x0 = std::min(x0, X[2 * a]);
            x1 = std::max(x1, X[2 * a]);
            y0 = std::min(y0, X[2 * a + 1]);
            y1 = std::max(y1, X[2 * a + 1]);
        }
        const double sx = 65535.0 / std::max(x1 - x0, 1e-300), sy = 65535.0 / std::max(y1 - y0, 1e-300);
        auto code = [&](double x, double y) {
            double u = std::min(std::max((x - x0) * sx, 0.0), 65535.0);
            double v = std::min(std::max((y - y0) * sy, 0.0), 65535.0);
            return morton2((uint32_t)u, (uint32_t)v);
        };
        std::vector<uint32_t> kn(N), ke(E);
        for (int a = 0; a < N; ++a) kn[a] = code(X[2 * a], X[2 * a + 1]);
        for (int e = 0; e < E; ++e) {
            double cx = 0.25 * (fr[4 * e].x + fr[4 * e + 1].x + fr[4 * e + 2].x + fr[4 * e + 3].x);
            double cy = 0.25 * (fr[4 * e].y + fr[4 * e + 1].y + fr[4 * e + 2].y + fr[4 * e + 3].y);
            if (T.Lx > 0) cx = std::fmod(std::fmod(cx, T.Lx) + T.Lx, T.Lx);
            if (T.Ly > 0) cy = std::fmod(std::fmod(cy, T.Ly) + T.Ly, T.Ly);
            ke[e] = code(cx, cy);
        }
        std::stable_sort(T.node_new2old.begin(), T.node_new2old.end(), [&](int a, int b) { return kn[a] < kn[b]; });
        std::stable_sort(T.elem_new2old.begin(), T.elem_new2old.end(), [&](int a, int b) { return ke[a] < ke[b]; });
    }
    for (int a = 0; a < N; ++a) T.node_old2new[T.node_new2old[a]] = a;
    for (int e = 0; e < E; ++e) T.elem_old2new[T.elem_new2old[e]] = e;
    const std::vector<int> &n2o = T.node_new2old, &o2n = T.node_old2new;
    const std::vector<int> &e2o = T.elem_new2old, &eo2n = T.elem_old2new;
    // neighbours across edges (original ids)
    std::unordered_map<uint64_t, std::vector<int>> edges;
    edges.reserve((size_t)4 * E);
    for (int e = 0; e < E; ++e)
        for (int k = 0; k < 4; ++k) {
            uint64_t a = (uint64_t)C[9 * e + k], b = (uint64_t)C[9 * e + (k + 1) % 4];
            edges[std::min(a, b) * (uint64_t)N + std::max(a, b)].push_back(4 * e + k);
        }
    std::vector<int> nbr_o((size_t)4 * E, -1), nedge_o((size_t)4 * E, 0), dsx_o((size_t)4 * E, 0),
        dsy_o((size_t)4 * E, 0);
    for (auto &kv : edges) {
        auto &v = kv.second;
        const int ek0 = v[0];
        const uint8_t kind0 = d->edge_kind[ek0];
        if (v.size() == 1) {
            if (kind0 == ALELB_EDGE_INTERIOR)
                { err = "an edge with one element is not marked as boundary"; return ALELB_ERR_MESH; }
            continue;
        }
        if (v.size() != 2) { err = "an edge is shared by more than two elements"; return ALELB_ERR_MESH; }
        const int ek1 = v[1];
        if (kind0 != ALELB_EDGE_INTERIOR || d->edge_kind[ek1] != ALELB_EDGE_INTERIOR)
            { err = "a shared edge is marked as boundary"; return ALELB_ERR_MESH; }
        for (int s = 0; s < 2; ++s) {
            const int a = s ? ek1 : ek0, b = s ? ek0 : ek1;
            const int ea = a / 4, ka = a % 4, eb = b / 4, kb = b % 4;
            nbr_o[a] = eb;
            nedge_o[a] = kb;
            // corner k of ea is corner kb + 1 of eb
            const double2 pa = fr[4 * ea + ka], pb = fr[4 * eb + (kb + 1) % 4];
            dsx_o[a] = T.Lx > 0 ? (int)std::lround((pa.x - pb.x) / T.Lx) : 0;
            dsy_o[a] = T.Ly > 0 ? (int)std::lround((pa.y - pb.y) / T.Ly) : 0;
            if (dsx_o[a] < -1 || dsx_o[a] > 1 || dsy_o[a] < -1 || dsy_o[a] > 1)
                { err = "element larger than half the period"; return ALELB_ERR_MESH; }
        }
    }
    // internal-order element tables
    Q.ev.assign((size_t)4 * E, make_double2(0, 0));
    Q.nbr.assign((size_t)4 * E, -1);
    Q.conn.assign((size_t)9 * E, 0);
    Q.rank.assign(E, 0);
    Q.orig.assign(E, 0);
    Q.einfo.assign(E, 0u);
    for (int en = 0; en < E; ++en) {
        const int eo = e2o[en];
        Q.orig[en] = eo;
        Q.rank[en] = rank_o[eo];
        uint32_t info = 0;
        for (int k = 0; k < 4; ++k) {
            Q.ev[4 * en + k] = fr[4 * eo + k];
            const int nb = nbr_o[4 * eo + k];
            Q.nbr[4 * en + k] = nb >= 0 ? eo2n[nb] : -1;
            const uint32_t kind = d->edge_kind[4 * eo + k] & 3u;
            info |= (kind | ((uint32_t)nedge_o[4 * eo + k] << 2) | ((uint32_t)(dsx_o[4 * eo + k] + 1) << 4) |
                     ((uint32_t)(dsy_o[4 * eo + k] + 1) << 6)) << (8 * k);
        }
        Q.einfo[en] = info;
        for (int l = 0; l < 9; ++l) Q.conn[9 * en + l] = o2n[C[9 * eo + l]];
    }
    // node coordinates, fans (the element's frame shift of each node), owners
    T.X.resize(N);
    for (int a = 0; a < N; ++a) T.X[a] = make_double2(X[2 * n2o[a]], X[2 * n2o[a] + 1]);
    std::vector<int> cnt(N + 1, 0);
    for (int en = 0; en < E; ++en)
        for (int l = 0; l < 9; ++l) cnt[Q.conn[9 * en + l] + 1]++;
    for (int a = 0; a < N; ++a) cnt[a + 1] += cnt[a];
    Q.fan_ptr = cnt;
    Q.fan.assign(cnt[N], make_int2(0, 0));
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    Q.owner.assign(N, make_int2(-1, 0));
    for (int en = 0; en < E; ++en) {
        const int eo = e2o[en];
        for (int l = 0; l < 9; ++l) {
            const int a = Q.conn[9 * en + l];
            const double xi = quad_ix(l) - 1.0, eta = quad_iy(l) - 1.0;
            double w[8];
            for (int k = 0; k < 4; ++k) {
                w[2 * k] = Q.ev[4 * en + k].x;
                w[2 * k + 1] = Q.ev[4 * en + k].y;
            }
            double px, py, J[4];
            quad_bilinear(w, xi, eta, px, py, J);
            const int sx = T.Lx > 0 ? (int)std::lround((T.X[a].x - px) / T.Lx) : 0;
            const int sy = T.Ly > 0 ? (int)std::lround((T.X[a].y - py) / T.Ly) : 0;
            if (sx < -1 || sx > 1 || sy < -1 || sy > 1) { err = "node far outside its element frame"; return ALELB_ERR_MESH; }
            Q.fan[fill[a]++] = make_int2(en, l | ((sx + 1) << 4) | ((sy + 1) << 6));
            const int cur = Q.owner[a].x;
            if (cur < 0 || area2[eo] > area2[e2o[cur]] || (area2[eo] == area2[e2o[cur]] && eo < e2o[cur]))
                Q.owner[a] = make_int2(en, l);
        }
    }
    // boundary kinds, wall nodes and their normals into the fluid
    Q.bkind.assign(N, 0);
    std::vector<double2> wn(N, make_double2(0, 0));
    std::vector<uint8_t> is_wall(N, 0);
    Q.wedges.clear();
    for (int en = 0; en < E; ++en)
        for (int k = 0; k < 4; ++k) {
            const uint32_t kind = (Q.einfo[en] >> (8 * k)) & 3u;
            if (!kind) continue;
            const int k1 = (k + 1) % 4;
            const int nodes[3] = {Q.conn[9 * en + k], Q.conn[9 * en + 4 + k], Q.conn[9 * en + k1]};
            for (int j = 0; j < 3; ++j) Q.bkind[nodes[j]] = (uint8_t)kind;
            if (kind == ALELB_EDGE_WALL) {
                Q.wedges.push_back(make_int2(en, k));
                const double tx = Q.ev[4 * en + k1].x - Q.ev[4 * en + k].x, ty = Q.ev[4 * en + k1].y - Q.ev[4 * en + k].y;
                const double L = std::sqrt(tx * tx + ty * ty);
                for (int j = 0; j < 3; ++j) {
                    is_wall[nodes[j]] = 1;
                    wn[nodes[j]].x += -ty / L;
                    wn[nodes[j]].y += tx / L;
                }
            }
        }
    // wall-condition gradient element (reading R8): among the incident
    // elements with a corner on a wall edge the one of larger area, then
    // lower original id; the owner when none touches a wall.  (elem, local)
    Q.bcel.assign(N, make_int2(-1, 0));
    for (int a = 0; a < N; ++a) {
        int best = -1, bl = 0;
        for (int k = Q.fan_ptr[a]; k < Q.fan_ptr[a + 1]; ++k) {
            const int en = Q.fan[k].x;
            bool touch = false;
            for (int c = 0; c < 4; ++c) touch = touch || is_wall[Q.conn[9 * en + c]];
            if (!touch) continue;
            const int eo = e2o[en];
            if (best < 0 || area2[eo] > area2[e2o[best]] || (area2[eo] == area2[e2o[best]] && eo < e2o[best])) {
                best = en;
                bl = Q.fan[k].y & 15;
            }
        }
        Q.bcel[a] = best >= 0 ? make_int2(best, bl) : Q.owner[a];
    }
    // wall probes B = A + n dt: breadth-first search over the adjacency from
    // the node's fan for the containing element of best rank (closed, exact
    // signs), then its local coordinates by Newton's method
    Q.wall_idx.assign(N, -1);
    Q.probe_e.clear();
    Q.probe_xi.clear();
    Q.wall_nrm.clear();
    {
        std::vector<int> seen(E, -1);
        for (int a = 0; a < N; ++a) {
            if (!is_wall[a]) continue;
            double nx = wn[a].x, ny = wn[a].y;
            const double L = std::sqrt(nx * nx + ny * ny);
            nx /= L;
            ny /= L;
            const double Bx = T.X[a].x + nx * 1.0, By = T.X[a].y + ny * 1.0;
            struct Qe { int e, sx, sy, depth; };
            std::vector<Qe> q;
            for (int k = Q.fan_ptr[a]; k < Q.fan_ptr[a + 1]; ++k) {
                const int e = Q.fan[k].x;
                if (seen[e] == a) continue;
                seen[e] = a;
                q.push_back({e, ((Q.fan[k].y >> 4) & 3) - 1, ((Q.fan[k].y >> 6) & 3) - 1, 0});
            }
            int best = -1, bsx = 0, bsy = 0;
            for (size_t h = 0; h < q.size(); ++h) {
                const Qe cur = q[h];
                const double ox = cur.sx * T.Lx, oy = cur.sy * T.Ly;
                bool in = true;
                for (int k = 0; k < 4 && in; ++k) {
                    const int k1 = (k + 1) % 4;
                    in = host_orient(Q.ev[4 * cur.e + k].x + ox, Q.ev[4 * cur.e + k].y + oy, Q.ev[4 * cur.e + k1].x + ox,
                                     Q.ev[4 * cur.e + k1].y + oy, Bx, By) >= 0;
                }
                if (in && (best < 0 || Q.rank[cur.e] < Q.rank[best])) {
                    best = cur.e;
                    bsx = cur.sx;
                    bsy = cur.sy;
                }
                if (cur.depth >= 12) continue;
                for (int k = 0; k < 4; ++k) {
                    const int nb = Q.nbr[4 * cur.e + k];
                    if (nb < 0 || seen[nb] == a) continue;
                    seen[nb] = a;
                    const uint32_t inf = (Q.einfo[cur.e] >> (8 * k)) & 255u;
                    q.push_back({nb, cur.sx + (int)((inf >> 4) & 3) - 1, cur.sy + (int)((inf >> 6) & 3) - 1,
                                 cur.depth + 1});
                }
            }
            if (best < 0) { err = "wall probe point B lies outside the mesh"; return ALELB_ERR_MESH; }
            double w[8];
            for (int k = 0; k < 4; ++k) {
                w[2 * k] = Q.ev[4 * best + k].x + bsx * T.Lx;
                w[2 * k + 1] = Q.ev[4 * best + k].y + bsy * T.Ly;
            }
            double xi, eta;
            if (!host_quad_local(w, Bx, By, xi, eta))
                { err = "wall probe point: Newton's method did not converge"; return ALELB_ERR_MESH; }
            Q.wall_idx[a] = (int)Q.probe_e.size();
            Q.wall_nrm.push_back(make_double2(nx, ny));
            Q.probe_e.push_back(best);
            Q.probe_xi.push_back(make_double2(xi, eta));
        }
    }
    // FP32 hi + lo splits (hi = fl32(x), lo = fl32(x - hi)) of the node
    // coordinates and the corners
    auto split = [](double2 v) {
        const float xh = (float)v.x, yh = (float)v.y;
        return make_float4(xh, yh, (float)(v.x - (double)xh), (float)(v.y - (double)yh));
    };
    Q.Xf.resize(N);
    for (int a = 0; a < N; ++a) Q.Xf[a] = split(T.X[a]);
    Q.evf.resize((size_t)4 * E);
    for (size_t k = 0; k < (size_t)4 * E; ++k) Q.evf[k] = split(Q.ev[k]);
    Q.ownJf.resize(N);
    for (int a = 0; a < N; ++a) {
        const int e = Q.owner[a].x, l = Q.owner[a].y;
        double w[8], x, y, J[4];
        for (int k = 0; k < 4; ++k) {
            w[2 * k] = Q.ev[4 * e + k].x;
            w[2 * k + 1] = Q.ev[4 * e + k].y;
        }
        quad_bilinear(w, quad_ix(l) - 1.0, quad_iy(l) - 1.0, x, y, J);
        const double det = J[0] * J[3] - J[2] * J[1];
        Q.ownJf[a] = make_float4((float)(J[3] / det), (float)(-J[1] / det), (float)(-J[2] / det), (float)(J[0] / det));
    }
    // lower bound of every node's distance to the nearest boundary edge,
    // capped at DCAP (zero on periodic meshes with boundaries: those always
    // walk): a departure segment shorter than it cannot leave the mesh
    {
        const double DCAP = 16.0;
        Q.bdist.assign(N, (float)DCAP);
        std::vector<std::pair<double2, double2>> be;
        for (int en = 0; en < E; ++en)
            for (int k = 0; k < 4; ++k)
                if ((Q.einfo[en] >> (8 * k)) & 3u) be.push_back({Q.ev[4 * en + k], Q.ev[4 * en + (k + 1) % 4]});
        if (!be.empty() && (T.Lx > 0 || T.Ly > 0)) {
            Q.bdist.assign(N, 0.0f);
        } else if (!be.empty()) {
            std::unordered_map<uint64_t, std::vector<int>> grid;
            auto key = [](long ix, long iy) { return ((uint64_t)(uint32_t)ix << 32) | (uint32_t)iy; };
            for (size_t b = 0; b < be.size(); ++b) {
                const double x0 = std::min(be[b].first.x, be[b].second.x) - DCAP;
                const double x1 = std::max(be[b].first.x, be[b].second.x) + DCAP;
                const double y0 = std::min(be[b].first.y, be[b].second.y) - DCAP;
                const double y1 = std::max(be[b].first.y, be[b].second.y) + DCAP;
                for (long ix = (long)std::floor(x0 / DCAP); ix <= (long)std::floor(x1 / DCAP); ++ix)
                    for (long iy = (long)std::floor(y0 / DCAP); iy <= (long)std::floor(y1 / DCAP); ++iy)
                        grid[key(ix, iy)].push_back((int)b);
            }
            for (int a = 0; a < N; ++a) {
                const double px = T.X[a].x, py = T.X[a].y;
                auto it = grid.find(key((long)std::floor(px / DCAP), (long)std::floor(py / DCAP)));
                if (it == grid.end()) continue;
                double dmin = DCAP;
                for (int b : it->second) {
                    const double ax = be[b].first.x, ay = be[b].first.y, dx = be[b].second.x - ax,
                                 dy = be[b].second.y - ay, L2 = dx * dx + dy * dy;
                    double t = L2 > 0 ? ((px - ax) * dx + (py - ay) * dy) / L2 : 0.0;
                    t = std::min(1.0, std::max(0.0, t));
                    const double qx = ax + t * dx - px, qy = ay + t * dy - py;
                    dmin = std::min(dmin, std::sqrt(qx * qx + qy * qy));
                }
                Q.bdist[a] = (float)(dmin * (1.0 - 1e-6));
            }
        }
    }
    T.ms = static_map_factors(T.mkind, T.mp, T.X);
    T.msf.resize(T.ms.size());
    for (size_t k = 0; k < T.ms.size(); ++k) T.msf[k] = (float)T.ms[k];
    T.n_wall_nodes = (int)Q.probe_e.size();
    T.wedges = Q.wedges;
    return ALELB_OK;
}

} // namespace alelb
