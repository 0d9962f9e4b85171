// tables.h -- host-side construction of the static mesh tables used by the
// kernels: element frames (vertex coordinates with periodic unwrapping),
// neighbours across edges with their frame shifts, tie-break ranks (larger
// computational area first, then lower original id), node fans, owner
// elements (Sec. IV: a node on element edges belongs to the incident element
// of larger area), wall normals and probe points B (Sec. IV.A), Morton
// renumbering and the static per-node map factors.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "alelb.h"
#include "geom.cuh"

namespace alelb {

inline int host_orient(double ax, double ay, double bx, double by, double cx, double cy)
{
    return orient(ax, ay, bx, by, cx, cy);
}

inline double unwrap1(double d, double L)
{
    if (L > 0) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

inline uint32_t morton2(uint32_t x, uint32_t y)
{
    auto spread = [](uint32_t v) {
        v &= 0xffff;
        v = (v | (v << 8)) & 0x00ff00ff;
        v = (v | (v << 4)) & 0x0f0f0f0f;
        v = (v | (v << 2)) & 0x33333333;
        v = (v | (v << 1)) & 0x55555555;
        return v;
    };
    return spread(x) | (spread(y) << 1);
}

struct HostTables {
    int N = 0, E = 0;
    double Lx = 0, Ly = 0;
    int mkind = 0;
    double mp[16] = {0};
    std::vector<int> node_old2new, node_new2old, elem_old2new, elem_new2old;
    std::vector<double2> X, ev, probe_xi, wall_nrm;
    std::vector<int> nbr, conn, rank, orig, fan_ptr, wall_idx, probe_e, bcel, ring_ptr, ring;
    std::vector<float2> nscale;
    std::vector<uint32_t> einfo;
    std::vector<int2> fan, owner, wedges;
    std::vector<int4> ostn; // [2N] owner stencils (MeshDev::ostn)
    std::vector<uint8_t> bkind, vzero, conek;
    std::vector<float4> cone;
    std::vector<double> ms;
    std::vector<float4> ejf, Xf, v0f, evf;
    std::vector<float> bdist, msf;
    std::vector<int> nb_ptr;
    std::vector<float4> nb;
    std::vector<uint8_t> nbf;
    int n_wall_nodes = 0;

    // a MeshDev whose pointers address these host vectors (host-side walk)
    MeshDev host_view() const
    {
        MeshDev D{};
        D.N = N;
        D.E = E;
        D.Lx = Lx;
        D.Ly = Ly;
        D.X = X.data();
        D.ev = ev.data();
        D.nbr = nbr.data();
        D.einfo = einfo.data();
        D.rank = rank.data();
        D.conn = conn.data();
        D.fan_ptr = fan_ptr.data();
        D.fan = fan.data();
        D.owner = owner.data();
        D.ostn = ostn.data();
        D.bcel = bcel.data();
        D.bkind = bkind.data();
        D.vzero = vzero.data();
        D.cone = cone.data();
        D.conek = conek.data();
        D.wall_idx = wall_idx.data();
        D.probe_e = probe_e.data();
        D.probe_xi = probe_xi.data();
        D.wall_nrm = wall_nrm.data();
        D.orig_elem = orig.data();
        D.ejf = ejf.data();
        D.bdist = bdist.data();
        D.Xf = Xf.data();
        D.v0f = v0f.data();
        D.evf = evf.data();
        D.ring_ptr = ring_ptr.data();
        D.ring = ring.data();
        D.nscale = nscale.data();
        D.nb_ptr = nb_ptr.data();
        D.nb = nb.data();
        D.nbf = nbf.data();
        return D;
    }
    MapStatic host_map() const
    {
        MapStatic S{};
        S.kind = mkind;
        S.Xc = mp[3];
        S.Yc = mp[4];
        S.N = N;
        S.ms = ms.empty() ? nullptr : ms.data();
        S.msf = msf.empty() ? nullptr : msf.data();
        return S;
    }
};

inline MapScalars map_scalars(int kind, const double *p, double t)
{
    MapScalars S;
    std::memset(&S, 0, sizeof(S));
    if (kind == MK_SINE) {
        double Tp = p[2];
        S.s = std::sin(2.0 * M_PI * t / Tp);
        S.sd = (2.0 * M_PI / Tp) * std::cos(2.0 * M_PI * t / Tp);
    } else if (kind == MK_PLUNGE) {
        double h = p[0], om = p[1];
        S.yoff = -h * std::sin(om * t);
        S.vy = -(h * om) * std::cos(om * t);
    } else if (kind >= MK_PITCH) {
        double th = p[0] + p[1] * std::sin(p[2] * t);
        S.c = std::cos(th);
        S.sn = std::sin(th);
        S.thd = (p[1] * p[2]) * std::cos(p[2] * t);
        S.cm = -2.0 * std::sin(0.5 * th) * std::sin(0.5 * th);
        if (kind == MK_PITCH_PLUNGE) {
            double h = p[5], omh = p[6];
            S.yoff = -h * std::sin(omh * t);
            S.vy = -(h * omh) * std::cos(omh * t);
        }
    }
    return S;
}

// Validates the description and fills T.  Returns ALELB_OK or an error
// with a message in err.
// Neighbour ring of each node for the learned departure-element proposal:
// the node's own elements sorted by the angle of their centroid about the
// node, then the elements across their edges (not already listed) sorted
// the same way, at most RING_MAX, in the cache code of an unshifted
// element (elements reached through a periodic shift are left out: the
// verified fast test accepts unshifted elements only).  nscale[a] = (h, n):
// h the square root of the mean area of the node's elements, n their count.
constexpr int RING_MAX = 32;
inline void build_rings(HostTables &T, const std::vector<double> &area2)
{
    const int N = T.N;
    T.ring_ptr.assign(N + 1, 0);
    T.ring.clear();
    T.nscale.assign(N, make_float2(1.0f, 0.0f));
    std::vector<std::pair<double, int>> g1, g2;
    std::vector<int> seen(T.E, -1);
    for (int a = 0; a < N; ++a) {
        g1.clear();
        g2.clear();
        const double ax = T.X[a].x, ay = T.X[a].y;
        double asum = 0;
        int nf = 0;
        auto angle = [&](int e) {
            const double cx = (T.ev[3 * e].x + T.ev[3 * e + 1].x + T.ev[3 * e + 2].x) / 3.0;
            const double cy = (T.ev[3 * e].y + T.ev[3 * e + 1].y + T.ev[3 * e + 2].y) / 3.0;
            return std::atan2(cy - ay, cx - ax);
        };
        for (int k = T.fan_ptr[a]; k < T.fan_ptr[a + 1]; ++k) {
            const int e = T.fan[k].x, code = T.fan[k].y;
            asum += 0.5 * area2[T.orig[e]];
            ++nf;
            seen[e] = a;
            if (((code >> 4) & 3) != 1 || ((code >> 6) & 3) != 1) continue; // shifted
            g1.push_back({angle(e), e});
        }
        for (int k = T.fan_ptr[a]; k < T.fan_ptr[a + 1]; ++k) {
            const int e = T.fan[k].x, code = T.fan[k].y;
            if (((code >> 4) & 3) != 1 || ((code >> 6) & 3) != 1) continue;
            for (int j = 0; j < 3; ++j) {
                const int nb = T.nbr[3 * e + j];
                if (nb < 0 || seen[nb] == a) continue;
                seen[nb] = a;
                const uint32_t inf = (T.einfo[e] >> (8 * j)) & 255u;
                if (((inf >> 4) & 3) != 1 || ((inf >> 6) & 3) != 1) continue; // across a periodic edge
                g2.push_back({angle(nb), nb});
            }
        }
        std::sort(g1.begin(), g1.end());
        std::sort(g2.begin(), g2.end());
        int n = 0;
        for (auto &p : g1)
            if (n < RING_MAX) { T.ring.push_back(p.second | (1 << 28) | (1 << 30)); ++n; }
        for (auto &p : g2)
            if (n < RING_MAX) { T.ring.push_back(p.second | (1 << 28) | (1 << 30)); ++n; }
        T.ring_ptr[a + 1] = T.ring_ptr[a] + n;
        T.nscale[a] = make_float2((float)std::sqrt(asum / std::max(nf, 1)), (float)nf);
    }
}

// Static per-node factors of the map (host libm, the same expressions for
// every element kind): SINE {A sin(w Y), A sin(w X), ...} (6 per node),
// BLENDED {b, db/dX, db/dY} (3 per node), none for the rigid maps.  X in the
// library's node order.
inline std::vector<double> static_map_factors(int mkind, const double *mp, const std::vector<double2> &X)
{
    const int N = (int)X.size();
    std::vector<double> ms;
    if (mkind == MK_SINE) {
        ms.assign((size_t)6 * N, 0.0);
        double A = mp[0], L = mp[1];
        double w = 2.0 * M_PI / L;
        for (int a = 0; a < N; ++a) {
            double Xx = X[a].x, Yy = X[a].y;
            double f[6];
            if (mp[3] == 0.0) {
                f[0] = A * std::sin(w * Yy);
                f[1] = A * std::sin(w * Xx);
                f[2] = 0.0;
                f[3] = (A * w) * std::cos(w * Yy);
                f[4] = (A * w) * std::cos(w * Xx);
                f[5] = 0.0;
            } else {
                double S = std::sin(w * Xx) * std::sin(w * Yy);
                f[0] = A * S;
                f[1] = A * S;
                f[2] = (A * w) * (std::cos(w * Xx) * std::sin(w * Yy));
                f[3] = (A * w) * (std::sin(w * Xx) * std::cos(w * Yy));
                f[4] = f[2];
                f[5] = f[3];
            }
            for (int k = 0; k < 6; ++k) ms[(size_t)k * N + a] = f[k];
        }
    } else if (mkind == MK_BLENDED) {
        ms.assign((size_t)3 * N, 0.0);
        double Xc = mp[3], Yc = mp[4], r1 = mp[5], r2 = mp[6];
        for (int a = 0; a < N; ++a) {
            double dx = X[a].x - Xc, dy = X[a].y - Yc;
            double r = std::sqrt(dx * dx + dy * dy);
            double b = 1.0, bX = 0.0, bY = 0.0;
            if (r >= r2) {
                b = 0.0;
            } else if (r > r1) {
                double s = (r - r1) / (r2 - r1);
                b = 1.0 - s * s * (3.0 - 2.0 * s);
                double dbdr = -(6.0 * s * (1.0 - s)) / (r2 - r1);
                bX = dbdr * (dx / r);
                bY = dbdr * (dy / r);
            }
            ms[a] = b;
            ms[(size_t)N + a] = bX;
            ms[(size_t)2 * N + a] = bY;
        }
    }
    return ms;
}

inline alelb_status build_tables(const alelb_mesh_desc *d, HostTables &T, std::string &err)
{
    if (!d || d->n_nodes <= 0 || d->n_elems <= 0 || !d->X || !d->conn || !d->edge_kind) {
        err = "null pointer or empty mesh";
        return ALELB_ERR_ARG;
    }
    const int N = d->n_nodes, E = d->n_elems;
    if (E > CACHE_ELEM) { // the element cache codes hold 25 bits of element
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
    for (long k = 0; k < 6L * E; ++k)
        if (C[k] < 0 || C[k] >= N) { err = "connectivity out of range"; return ALELB_ERR_MESH; }
    // element frames (original order) and doubled areas
    std::vector<double2> fr((size_t)3 * E);
    std::vector<double> area2(E);
    for (int e = 0; e < E; ++e) {
        const int *c = C + 6 * e;
        double x0 = X[2 * c[0]], y0 = X[2 * c[0] + 1];
        double w[12];
        for (int l = 0; l < 6; ++l) {
            w[2 * l] = x0 + unwrap1(X[2 * c[l]] - x0, T.Lx);
            w[2 * l + 1] = y0 + unwrap1(X[2 * c[l] + 1] - y0, T.Ly);
        }
        for (int k = 0; k < 3; ++k) {
            int k1 = (k + 1) % 3;
            if (w[6 + 2 * k] != 0.5 * (w[2 * k] + w[2 * k1]) ||
                w[7 + 2 * k] != 0.5 * (w[2 * k + 1] + w[2 * k1 + 1]))
                { err = "a midside node is not its edge's exact midpoint"; return ALELB_ERR_MESH; }
            fr[3 * e + k] = make_double2(w[2 * k], w[2 * k + 1]);
        }
        double a2 = (w[2] - w[0]) * (w[5] - w[1]) - (w[4] - w[0]) * (w[3] - w[1]);
        if (!(a2 > 0)) { err = "inverted or degenerate element"; return ALELB_ERR_MESH; }
        area2[e] = a2;
    }
    // tie-break rank: larger area first, then lower original id
    std::vector<int> order(E);
    for (int e = 0; e < E; ++e) order[e] = e;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        if (area2[a] != area2[b]) return area2[a] > area2[b];
        return a < b;
    });
    std::vector<int> rank_o(E);
    for (int r = 0; r < E; ++r) rank_o[order[r]] = r;
    // renumbering: Morton order of nodes and element centroids
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
        double sx = 65535.0 / std::max(x1 - x0, 1e-300), sy = 65535.0 / std::max(y1 - y0, 1e-300);
        auto code = [&](double x, double y) {
            double u = std::min(std::max((x - x0) * sx, 0.0), 65535.0);
            double v = std::min(std::max((y - y0) * sy, 0.0), 65535.0);
            return morton2((uint32_t)u, (uint32_t)v);
        };
        std::vector<uint32_t> kn(N), ke(E);
        for (int a = 0; a < N; ++a) kn[a] = code(X[2 * a], X[2 * a + 1]);
        for (int e = 0; e < E; ++e) {
            double cx = (fr[3 * e].x + fr[3 * e + 1].x + fr[3 * e + 2].x) / 3.0;
            double cy = (fr[3 * e].y + fr[3 * e + 1].y + fr[3 * e + 2].y) / 3.0;
            if (T.Lx > 0) cx = std::fmod(std::fmod(cx, T.Lx) + T.Lx, T.Lx);
            if (T.Ly > 0) cy = std::fmod(std::fmod(cy, T.Ly) + T.Ly, T.Ly);
            ke[e] = code(cx, cy);
        }
        std::stable_sort(T.node_new2old.begin(), T.node_new2old.end(),
                         [&](int a, int b) { return kn[a] < kn[b]; });
        std::stable_sort(T.elem_new2old.begin(), T.elem_new2old.end(),
                         [&](int a, int b) { return ke[a] < ke[b]; });
    }
    for (int a = 0; a < N; ++a) T.node_old2new[T.node_new2old[a]] = a;
    for (int e = 0; e < E; ++e) T.elem_old2new[T.elem_new2old[e]] = e;
    const std::vector<int> &n2o = T.node_new2old, &o2n = T.node_old2new;
    const std::vector<int> &e2o = T.elem_new2old, &eo2n = T.elem_old2new;
    // neighbours across edges (original ids)
    std::unordered_map<uint64_t, std::vector<int>> edges;
    edges.reserve((size_t)3 * E);
    for (int e = 0; e < E; ++e)
        for (int k = 0; k < 3; ++k) {
            uint64_t a = (uint64_t)C[6 * e + k], b = (uint64_t)C[6 * e + (k + 1) % 3];
            uint64_t key = std::min(a, b) * (uint64_t)N + std::max(a, b);
            edges[key].push_back(3 * e + k);
        }
    std::vector<int> nbr_o((size_t)3 * E, -1), nedge_o((size_t)3 * E, 0);
    std::vector<int> dsx_o((size_t)3 * E, 0), dsy_o((size_t)3 * E, 0);
    for (auto &kv : edges) {
        auto &v = kv.second;
        int ek0 = v[0];
        uint8_t kind0 = d->edge_kind[ek0];
        if (v.size() == 1) {
            if (kind0 == ALELB_EDGE_INTERIOR)
                { err = "an edge with one element is not marked as boundary"; return ALELB_ERR_MESH; }
            continue;
        }
        if (v.size() != 2) { err = "an edge is shared by more than two elements"; return ALELB_ERR_MESH; }
        int ek1 = v[1];
        if (kind0 != ALELB_EDGE_INTERIOR || d->edge_kind[ek1] != ALELB_EDGE_INTERIOR)
            { err = "a shared edge is marked as boundary"; return ALELB_ERR_MESH; }
        for (int s = 0; s < 2; ++s) {
            int a = s ? ek1 : ek0, b = s ? ek0 : ek1;
            int ea = a / 3, ka = a % 3, eb = b / 3, kb = b % 3;
            nbr_o[a] = eb;
            nedge_o[a] = kb;
            // vertex v_ka of ea is vertex v_(kb+1) of eb
            double2 pa = fr[3 * ea + ka], pb = fr[3 * eb + (kb + 1) % 3];
            dsx_o[a] = T.Lx > 0 ? (int)std::lround((pa.x - pb.x) / T.Lx) : 0;
            dsy_o[a] = T.Ly > 0 ? (int)std::lround((pa.y - pb.y) / T.Ly) : 0;
            if (dsx_o[a] < -1 || dsx_o[a] > 1 || dsy_o[a] < -1 || dsy_o[a] > 1)
                { err = "element larger than half the period"; return ALELB_ERR_MESH; }
        }
    }
    // internal-order element tables
    auto &ev = T.ev; auto &nbr = T.nbr; auto &conn = T.conn; auto &rank = T.rank; auto &orig = T.orig;
    auto &einfo = T.einfo;
    ev.assign((size_t)3 * E, make_double2(0, 0));
    nbr.assign((size_t)3 * E, -1);
    conn.assign((size_t)6 * E, 0);
    rank.assign(E, 0);
    orig.assign(E, 0);
    einfo.assign(E, 0u);
    for (int en = 0; en < E; ++en) {
        int eo = e2o[en];
        orig[en] = eo;
        rank[en] = rank_o[eo];
        uint32_t info = 0;
        for (int k = 0; k < 3; ++k) {
            ev[3 * en + k] = fr[3 * eo + k];
            int nb = nbr_o[3 * eo + k];
            nbr[3 * en + k] = nb >= 0 ? eo2n[nb] : -1;
            uint32_t kind = d->edge_kind[3 * eo + k] & 3u;
            uint32_t byte = kind | ((uint32_t)nedge_o[3 * eo + k] << 2) |
                            ((uint32_t)(dsx_o[3 * eo + k] + 1) << 4) |
                            ((uint32_t)(dsy_o[3 * eo + k] + 1) << 6);
            info |= byte << (8 * k);
        }
        einfo[en] = info;
        for (int l = 0; l < 6; ++l) conn[6 * en + l] = o2n[C[6 * eo + l]];
    }
    // node coordinates, fans, owners, boundary kinds
    T.X.resize(N);
    for (int a = 0; a < N; ++a) T.X[a] = make_double2(X[2 * n2o[a]], X[2 * n2o[a] + 1]);
    std::vector<int> cnt(N + 1, 0);
    for (int en = 0; en < E; ++en)
        for (int l = 0; l < 6; ++l) cnt[conn[6 * en + l] + 1]++;
    for (int a = 0; a < N; ++a) cnt[a + 1] += cnt[a];
    auto &fan_ptr = T.fan_ptr; auto &fan = T.fan;
    fan_ptr = cnt;
    fan.assign(cnt[N], make_int2(0, 0));
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    auto &owner = T.owner;
    owner.assign(N, make_int2(-1, 0));

    for (int en = 0; en < E; ++en) {
        int eo = e2o[en];
        for (int l = 0; l < 6; ++l) {
            int a = conn[6 * en + l];
            double px, py;
            if (l < 3) {
                px = ev[3 * en + l].x;
                py = ev[3 * en + l].y;
            } else {
                int k = l - 3, k1 = (k + 1) % 3;
                px = 0.5 * (ev[3 * en + k].x + ev[3 * en + k1].x);
                py = 0.5 * (ev[3 * en + k].y + ev[3 * en + k1].y);
            }
            int sx = T.Lx > 0 ? (int)std::lround((T.X[a].x - px) / T.Lx) : 0;
            int sy = T.Ly > 0 ? (int)std::lround((T.X[a].y - py) / T.Ly) : 0;
            if (sx < -1 || sx > 1 || sy < -1 || sy > 1)
                { err = "node far outside its element frame"; return ALELB_ERR_MESH; }
            fan[fill[a]++] = make_int2(en, l | ((sx + 1) << 4) | ((sy + 1) << 6));
            int cur = owner[a].x;
            if (cur < 0 || area2[eo] > area2[e2o[cur]] ||
                (area2[eo] == area2[e2o[cur]] && eo < e2o[cur]))
                owner[a] = make_int2(en, l);
        }
    }
    auto &bkind = T.bkind;
    bkind.assign(N, 0);
    std::vector<double2> wn(N, make_double2(0, 0));
    std::vector<uint8_t> is_wall(N, 0);
    for (int en = 0; en < E; ++en)
        for (int k = 0; k < 3; ++k) {
            uint32_t kind = (einfo[en] >> (8 * k)) & 3u;
            if (!kind) continue;
            int k1 = (k + 1) % 3;
            int nodes[3] = {conn[6 * en + k], conn[6 * en + 3 + k], conn[6 * en + k1]};
            for (int j = 0; j < 3; ++j) bkind[nodes[j]] = (uint8_t)kind;
            if (kind == ALELB_EDGE_WALL) {
                T.wedges.push_back(make_int2(en, k));
                double tx = ev[3 * en + k1].x - ev[3 * en + k].x;
                double ty = ev[3 * en + k1].y - ev[3 * en + k].y;
                double L = std::sqrt(tx * tx + ty * ty);
                for (int j = 0; j < 3; ++j) {
                    is_wall[nodes[j]] = 1;
                    wn[nodes[j]].x += -ty / L;
                    wn[nodes[j]].y += tx / L;
                }
            }
        }
    // exterior cone of each boundary node: its outgoing and incoming boundary
    // edges (the domain on their left) when it has exactly one of each, of
    // one kind; a departure direction strictly right of both leaves the mesh
    // at once (the population is missing)
    {
        std::vector<int> nout(N, 0), nin(N, 0), kk(N, 0);
        T.cone.assign(N, make_float4(0, 0, 0, 0));
        T.conek.assign(N, 0);
        for (int en = 0; en < E; ++en)
            for (int k = 0; k < 3; ++k) {
                const int kind = (int)((einfo[en] >> (8 * k)) & 3u);
                if (!kind) continue;
                const int k1 = (k + 1) % 3;
                const double ex = ev[3 * en + k1].x - ev[3 * en + k].x, ey = ev[3 * en + k1].y - ev[3 * en + k].y;
                const int va = conn[6 * en + k], vb = conn[6 * en + k1], mid = conn[6 * en + 3 + k];
                auto add = [&](int node, bool out, double x, double y) {
                    if (kk[node] && kk[node] != kind) kk[node] = -1;
                    else if (!kk[node]) kk[node] = kind;
                    if (out) { nout[node]++; T.cone[node].x = (float)x; T.cone[node].y = (float)y; }
                    else { nin[node]++; T.cone[node].z = (float)x; T.cone[node].w = (float)y; }
                };
                add(va, true, ex, ey);
                add(vb, false, ex, ey);
                add(mid, true, 0.5 * ex, 0.5 * ey);
                add(mid, false, 0.5 * ex, 0.5 * ey);
            }
        // bit 2: a convex corner of the domain (the boundary turns left by a
        // clear margin), where the domain near the node is the intersection
        // of the two left half-planes, so leaving across either edge line
        // leaves the mesh; bit 3: a reflex corner (turns right by a clear
        // margin), where the domain near the node is their union
        for (int a = 0; a < N; ++a)
            if (nout[a] == 1 && nin[a] == 1 && kk[a] > 0) {
                const double ox = T.cone[a].x, oy = T.cone[a].y, ix = T.cone[a].z, iy = T.cone[a].w;
                const double cr = ix * oy - iy * ox;
                const double tol = 1e-6 * std::sqrt((ix * ix + iy * iy) * (ox * ox + oy * oy));
                T.conek[a] = (uint8_t)(kk[a] | (cr > tol ? 4 : 0) | (cr < -tol ? 8 : 0));
            }
    }
    // element of each node's wall-condition gradients: among the incident
    // elements with a vertex on a wall edge the one of larger computational
    // area, then lower original id; the owner element when none touches a
    // wall
    auto &bcel = T.bcel;
    bcel.assign(N, -1);
    for (int a = 0; a < N; ++a) {
        int best = -1;
        for (int k = fan_ptr[a]; k < fan_ptr[a + 1]; ++k) {
            const int en = fan[k].x;
            if (!is_wall[conn[6 * en]] && !is_wall[conn[6 * en + 1]] && !is_wall[conn[6 * en + 2]]) continue;
            const int eo = e2o[en];
            if (best < 0 || area2[eo] > area2[e2o[best]] || (area2[eo] == area2[e2o[best]] && eo < e2o[best]))
                best = en;
        }
        bcel[a] = best >= 0 ? best : owner[a].x;
    }
    // wall probes B = A + n dt, located by breadth-first search over the
    // adjacency from the node's fan (tie rule as everywhere else)
    auto &wall_idx = T.wall_idx; auto &probe_e = T.probe_e; auto &probe_xi = T.probe_xi;
    wall_idx.assign(N, -1);
    probe_e.clear();
    probe_xi.clear();
    T.wall_nrm.clear();
    {
        std::vector<int> seen(E, -1);
        for (int a = 0; a < N; ++a) {
            if (!is_wall[a]) continue;
            double nx = wn[a].x, ny = wn[a].y, L = std::sqrt(nx * nx + ny * ny);
            nx /= L;
            ny /= L;
            double Bx = T.X[a].x + nx * 1.0, By = T.X[a].y + ny * 1.0;
            struct Q { int e, sx, sy, depth; };
            std::vector<Q> q;
            for (int k = fan_ptr[a]; k < fan_ptr[a + 1]; ++k) {
                int e = fan[k].x;
                if (seen[e] == a) continue;
                seen[e] = a;
                q.push_back({e, ((fan[k].y >> 4) & 3) - 1, ((fan[k].y >> 6) & 3) - 1, 0});
            }
            int best = -1, bsx = 0, bsy = 0;
            for (size_t h = 0; h < q.size(); ++h) {
                Q cur = q[h];
                double ox = cur.sx * T.Lx, oy = cur.sy * T.Ly;
                double2 w0 = ev[3 * cur.e], w1 = ev[3 * cur.e + 1], w2 = ev[3 * cur.e + 2];
                double w[6] = {w0.x + ox, w0.y + oy, w1.x + ox, w1.y + oy, w2.x + ox, w2.y + oy};
                bool in = true;
                for (int k = 0; k < 3 && in; ++k) {
                    int k1 = (k + 1) % 3;
                    in = host_orient(w[2 * k], w[2 * k + 1], w[2 * k1], w[2 * k1 + 1], Bx, By) >= 0;
                }
                if (in && (best < 0 || rank[cur.e] < rank[best])) {
                    best = cur.e;
                    bsx = cur.sx;
                    bsy = cur.sy;
                }
                if (cur.depth >= 12) continue;
                for (int k = 0; k < 3; ++k) {
                    int nb = nbr[3 * cur.e + k];
                    if (nb < 0 || seen[nb] == a) continue;
                    seen[nb] = a;
                    uint32_t inf = (einfo[cur.e] >> (8 * k)) & 255u;
                    q.push_back({nb, cur.sx + (int)((inf >> 4) & 3) - 1,
                                 cur.sy + (int)((inf >> 6) & 3) - 1, cur.depth + 1});
                }
            }
            if (best < 0) { err = "wall probe point B lies outside the mesh"; return ALELB_ERR_MESH; }
            double2 v0 = ev[3 * best], v1 = ev[3 * best + 1], v2 = ev[3 * best + 2];
            double x0 = v0.x + bsx * T.Lx, y0 = v0.y + bsy * T.Ly;
            double x_xi = v1.x - v0.x, x_eta = v2.x - v0.x, y_xi = v1.y - v0.y, y_eta = v2.y - v0.y;
            double detJ = x_xi * y_eta - y_xi * x_eta;
            wall_idx[a] = (int)probe_e.size();
            T.wall_nrm.push_back(make_double2(nx, ny));
            probe_e.push_back(best);
            probe_xi.push_back(make_double2((y_eta * (Bx - x0) - x_eta * (By - y0)) / detJ,
                                            (-y_xi * (Bx - x0) + x_xi * (By - y0)) / detJ));
        }
    }
    // static per-node map factors (host libm, same expressions everywhere)
    T.ms = static_map_factors(T.mkind, T.mp, T.X);
    T.n_wall_nodes = (int)T.probe_e.size();
    // FP32 edge vectors and inverse Jacobians (interpolation weights and the
    // certified FP32 containment filter)
    T.ejf.assign((size_t)2 * E, make_float4(0, 0, 0, 0));
    for (int en = 0; en < E; ++en) {
        double2 v0 = ev[3 * en], v1 = ev[3 * en + 1], v2 = ev[3 * en + 2];
        double e1x = v1.x - v0.x, e1y = v1.y - v0.y, e2x = v2.x - v0.x, e2y = v2.y - v0.y;
        double det = e1x * e2y - e2x * e1y;
        T.ejf[2 * en] = make_float4((float)e1x, (float)e1y, (float)e2x, (float)e2y);
        T.ejf[2 * en + 1] = make_float4((float)(e2y / det), (float)(-e2x / det), (float)(-e1y / det),
                                        (float)(e1x / det));
    }
    // coordinates split into FP32 hi + lo parts: hi = fl32(x), lo = fl32(x - hi)
    auto split = [](double2 v) {
        float xh = (float)v.x, yh = (float)v.y;
        return make_float4(xh, yh, (float)(v.x - (double)xh), (float)(v.y - (double)yh));
    };
    T.Xf.resize(N);
    for (int a = 0; a < N; ++a) T.Xf[a] = split(T.X[a]);
    T.v0f.resize(E);
    for (int en = 0; en < E; ++en) T.v0f[en] = split(ev[3 * en]);
    T.evf.resize((size_t)3 * E);
    for (size_t k = 0; k < (size_t)3 * E; ++k) T.evf[k] = split(ev[k]);
    T.msf.resize(T.ms.size());
    for (size_t k = 0; k < T.ms.size(); ++k) T.msf[k] = (float)T.ms[k];
    // nodes whose mesh velocity is exactly zero at every time: no motion, or
    // a blended map whose blending factor is exactly zero there (then the
    // rest population's c^ is exactly zero and it keeps the node's value)
    T.vzero.assign(N, 0);
    for (int a = 0; a < N; ++a)
        T.vzero[a] = (uint8_t)(T.mkind == MK_NONE || (T.mkind == MK_BLENDED && T.ms[a] == 0.0));
    // lower bound of every node's distance to the nearest boundary edge
    // (capped at DCAP): a departure segment shorter than this cannot leave
    // the mesh
    // The same pass lists, for non-periodic meshes, every wall or far-field
    // edge within NEAR_R of each node, relative to the node (the departure
    // segment certificates of the fast path).
    const double DCAP = 16.0;
    T.bdist.assign(N, (float)DCAP);
    T.nb_ptr.assign(N + 1, 0);
    T.nb.clear();
    T.nbf.clear();
    {
        std::vector<std::pair<double2, double2>> be;
        std::vector<int> bkd, bn0, bn1, bn2;
        for (int en = 0; en < E; ++en)
            for (int k = 0; k < 3; ++k)
                if ((einfo[en] >> (8 * k)) & 3u) {
                    const int k1 = (k + 1) % 3;
                    be.push_back({ev[3 * en + k], ev[3 * en + k1]});
                    bkd.push_back((int)((einfo[en] >> (8 * k)) & 3u));
                    bn0.push_back(conn[6 * en + k]);
                    bn1.push_back(conn[6 * en + k1]);
                    bn2.push_back(conn[6 * en + 3 + k]);
                }
        if (!be.empty() && (T.Lx > 0 || T.Ly > 0)) {
            T.bdist.assign(N, 0.0f); // periodic meshes with boundaries: always walk
        } else if (!be.empty()) {
            const double cs = DCAP;
            std::unordered_map<uint64_t, std::vector<int>> grid;
            auto key = [](long ix, long iy) { return ((uint64_t)(uint32_t)ix << 32) | (uint32_t)iy; };
            for (size_t b = 0; b < be.size(); ++b) {
                double x0 = std::min(be[b].first.x, be[b].second.x) - DCAP, x1 = std::max(be[b].first.x, be[b].second.x) + DCAP;
                double y0 = std::min(be[b].first.y, be[b].second.y) - DCAP, y1 = std::max(be[b].first.y, be[b].second.y) + DCAP;
                for (long ix = (long)std::floor(x0 / cs); ix <= (long)std::floor(x1 / cs); ++ix)
                    for (long iy = (long)std::floor(y0 / cs); iy <= (long)std::floor(y1 / cs); ++iy)
                        grid[key(ix, iy)].push_back((int)b);
            }
            const double RN = (double)NEAR_R * (1.0 + 1e-6) + 1e-6;
            for (int a = 0; a < N; ++a) {
                T.nb_ptr[a + 1] = T.nb_ptr[a];
                double px = T.X[a].x, py = T.X[a].y;
                auto it = grid.find(key((long)std::floor(px / cs), (long)std::floor(py / cs)));
                if (it == grid.end()) continue;
                double dmin = DCAP;
                for (int b : it->second) {
                    double ax = be[b].first.x, ay = be[b].first.y, bx = be[b].second.x, by = be[b].second.y;
                    double dx = bx - ax, dy = by - ay, L2 = dx * dx + dy * dy;
                    double t = L2 > 0 ? ((px - ax) * dx + (py - ay) * dy) / L2 : 0.0;
                    t = std::min(1.0, std::max(0.0, t));
                    double qx = ax + t * dx - px, qy = ay + t * dy - py;
                    const double d = std::sqrt(qx * qx + qy * qy);
                    dmin = std::min(dmin, d);
                    if (d < RN) {
                        const bool on = bn0[b] == a || bn1[b] == a || bn2[b] == a;
                        T.nb.push_back(make_float4((float)(ax - px), (float)(ay - py), (float)(bx - px),
                                                   (float)(by - py)));
                        T.nbf.push_back((uint8_t)(bkd[b] | (on ? 4 : 0)));
                        T.nb_ptr[a + 1]++;
                    }
                }
                T.bdist[a] = (float)(dmin * (1.0 - 1e-6));
            }
        }
    }
    build_rings(T, area2);
    return ALELB_OK;
}

} // namespace alelb
