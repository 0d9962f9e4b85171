// alelb.cu -- host side of the C-ABI declared in include/alelb.h: mesh
// tables, solver state, launches.  All arithmetic of the time step runs in
// the kernels of kernels.cuh; the host prepares static tables (element
// frames, adjacency, fans, owner elements, wall probes, static map factors)
// and per-step map scalars.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "alelb.h"
#include "kernels.cuh"

using namespace alelb;

namespace {

// ----------------------------------------------------------------------------
// exact orientation on the host (wall probe location at set-up)
// ----------------------------------------------------------------------------
int host_orient(double ax, double ay, double bx, double by, double cx, double cy)
{
    double pa[6] = {ax, -ax, -cx, -ay, ay, cy};
    double pb[6] = {by, cy, by, bx, cx, bx};
    double e[16];
    int m = 0;
    for (int k = 0; k < 12; ++k) {
        double hi = pa[k >> 1] * pb[k >> 1];
        double q = (k & 1) ? std::fma(pa[k >> 1], pb[k >> 1], -hi) : hi;
        int mm = 0;
        for (int j = 0; j < m; ++j) {
            double s = q + e[j];
            double bv = s - q;
            double av = s - bv;
            double err = (q - av) + (e[j] - bv);
            if (err != 0.0) e[mm++] = err;
            q = s;
        }
        if (q != 0.0) e[mm++] = q;
        m = mm;
    }
    if (m == 0) return 0;
    return e[m - 1] > 0.0 ? 1 : -1;
}

double unwrap1(double d, double L)
{
    if (L > 0) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

uint32_t morton2(uint32_t x, uint32_t y)
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

struct DevBuf {
    std::vector<void *> ptrs;
    template <class T> T *put(const std::vector<T> &h, cudaError_t &st)
    {
        if (h.empty()) return nullptr;
        void *p = nullptr;
        if (st == cudaSuccess) st = cudaMalloc(&p, h.size() * sizeof(T));
        if (st == cudaSuccess) {
            ptrs.push_back(p);
            st = cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
        }
        return (T *)p;
    }
    template <class T> T *alloc(size_t n, cudaError_t &st)
    {
        void *p = nullptr;
        if (st == cudaSuccess) st = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
        if (st == cudaSuccess) ptrs.push_back(p);
        return (T *)p;
    }
    void release()
    {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

} // namespace

struct alelb_mesh {
    std::string err;
    int N = 0, E = 0;
    double Lx = 0, Ly = 0;
    int mkind = 0;
    double mp[16] = {0};
    std::vector<int> node_old2new, node_new2old, elem_old2new, elem_new2old;
    std::vector<double2> X;
    std::vector<int2> wedges;
    int n_wall_nodes = 0;
    MeshDev dev{};
    MapStatic mst{};
    int2 *d_wedges = nullptr;
    int nw = 0;
    DevBuf buf;
    int n_solvers = 0;
};

namespace {

template <class T> void put_state(DevBuf &b, StateDev<T> &s, int N, cudaError_t &st)
{
    s.post = b.alloc<T>((size_t)18 * N, st);
    s.str = b.alloc<T>((size_t)18 * N, st);
    s.rho = b.alloc<T>(N, st);
    s.ux = b.alloc<T>(N, st);
    s.uy = b.alloc<T>(N, st);
    s.T = b.alloc<T>(N, st);
    s.Qx = b.alloc<T>(N, st);
    s.Qy = b.alloc<T>(N, st);
    s.mrt = b.alloc<T>(N, st);
    s.Dx = b.alloc<T>(N, st);
    s.Dy = b.alloc<T>(N, st);
}

MapScalars map_scalars(int kind, const double *p, double t)
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

} // namespace

// ============================================================================
// mesh
// ============================================================================
extern "C" alelb_status alelb_mesh_create(const alelb_mesh_desc *d, alelb_mesh **out)
{
    if (!d || !out || d->n_nodes <= 0 || d->n_elems <= 0 || !d->X || !d->conn || !d->edge_kind)
        return ALELB_ERR_ARG;
    *out = nullptr;
    alelb_mesh *m = new (std::nothrow) alelb_mesh();
    if (!m) return ALELB_ERR_OOM;
    auto fail = [&](alelb_status s, const char *msg) {
        m->err = msg;
        *out = m; // returned so that alelb_mesh_last_error can be read
        return s;
    };
    const int N = d->n_nodes, E = d->n_elems;
    m->N = N;
    m->E = E;
    m->Lx = d->period[0] > 0 ? d->period[0] : 0.0;
    m->Ly = d->period[1] > 0 ? d->period[1] : 0.0;
    m->mkind = d->motion_kind;
    std::memcpy(m->mp, d->motion, sizeof(m->mp));
    if (m->mkind < 0 || m->mkind > MK_BLENDED) return fail(ALELB_ERR_ARG, "unknown motion kind");
    const double *X = d->X;
    const int *C = d->conn;
    for (long k = 0; k < 6L * E; ++k)
        if (C[k] < 0 || C[k] >= N) return fail(ALELB_ERR_MESH, "connectivity out of range");
    // element frames (original order) and doubled areas
    std::vector<double2> fr((size_t)3 * E);
    std::vector<double> area2(E);
    for (int e = 0; e < E; ++e) {
        const int *c = C + 6 * e;
        double x0 = X[2 * c[0]], y0 = X[2 * c[0] + 1];
        double w[12];
        for (int l = 0; l < 6; ++l) {
            w[2 * l] = x0 + unwrap1(X[2 * c[l]] - x0, m->Lx);
            w[2 * l + 1] = y0 + unwrap1(X[2 * c[l] + 1] - y0, m->Ly);
        }
        for (int k = 0; k < 3; ++k) {
            int k1 = (k + 1) % 3;
            if (w[6 + 2 * k] != 0.5 * (w[2 * k] + w[2 * k1]) ||
                w[7 + 2 * k] != 0.5 * (w[2 * k + 1] + w[2 * k1 + 1]))
                return fail(ALELB_ERR_MESH, "a midside node is not its edge's exact midpoint");
            fr[3 * e + k] = make_double2(w[2 * k], w[2 * k + 1]);
        }
        double a2 = (w[2] - w[0]) * (w[5] - w[1]) - (w[4] - w[0]) * (w[3] - w[1]);
        if (!(a2 > 0)) return fail(ALELB_ERR_MESH, "inverted or degenerate element");
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
    m->node_old2new.resize(N);
    m->node_new2old.resize(N);
    m->elem_old2new.resize(E);
    m->elem_new2old.resize(E);
    for (int a = 0; a < N; ++a) m->node_new2old[a] = a;
    for (int e = 0; e < E; ++e) m->elem_new2old[e] = e;
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
            if (m->Lx > 0) cx = std::fmod(std::fmod(cx, m->Lx) + m->Lx, m->Lx);
            if (m->Ly > 0) cy = std::fmod(std::fmod(cy, m->Ly) + m->Ly, m->Ly);
            ke[e] = code(cx, cy);
        }
        std::stable_sort(m->node_new2old.begin(), m->node_new2old.end(),
                         [&](int a, int b) { return kn[a] < kn[b]; });
        std::stable_sort(m->elem_new2old.begin(), m->elem_new2old.end(),
                         [&](int a, int b) { return ke[a] < ke[b]; });
    }
    for (int a = 0; a < N; ++a) m->node_old2new[m->node_new2old[a]] = a;
    for (int e = 0; e < E; ++e) m->elem_old2new[m->elem_new2old[e]] = e;
    const std::vector<int> &n2o = m->node_new2old, &o2n = m->node_old2new;
    const std::vector<int> &e2o = m->elem_new2old, &eo2n = m->elem_old2new;
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
                return fail(ALELB_ERR_MESH, "an edge with one element is not marked as boundary");
            continue;
        }
        if (v.size() != 2) return fail(ALELB_ERR_MESH, "an edge is shared by more than two elements");
        int ek1 = v[1];
        if (kind0 != ALELB_EDGE_INTERIOR || d->edge_kind[ek1] != ALELB_EDGE_INTERIOR)
            return fail(ALELB_ERR_MESH, "a shared edge is marked as boundary");
        for (int s = 0; s < 2; ++s) {
            int a = s ? ek1 : ek0, b = s ? ek0 : ek1;
            int ea = a / 3, ka = a % 3, eb = b / 3, kb = b % 3;
            nbr_o[a] = eb;
            nedge_o[a] = kb;
            // vertex v_ka of ea is vertex v_(kb+1) of eb
            double2 pa = fr[3 * ea + ka], pb = fr[3 * eb + (kb + 1) % 3];
            dsx_o[a] = m->Lx > 0 ? (int)std::lround((pa.x - pb.x) / m->Lx) : 0;
            dsy_o[a] = m->Ly > 0 ? (int)std::lround((pa.y - pb.y) / m->Ly) : 0;
            if (dsx_o[a] < -1 || dsx_o[a] > 1 || dsy_o[a] < -1 || dsy_o[a] > 1)
                return fail(ALELB_ERR_MESH, "element larger than half the period");
        }
    }
    // internal-order element tables
    std::vector<double2> ev((size_t)3 * E);
    std::vector<int> nbr((size_t)3 * E), conn((size_t)6 * E), rank(E), orig(E);
    std::vector<uint32_t> einfo(E);
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
    m->X.resize(N);
    for (int a = 0; a < N; ++a) m->X[a] = make_double2(X[2 * n2o[a]], X[2 * n2o[a] + 1]);
    std::vector<int> cnt(N + 1, 0);
    for (int en = 0; en < E; ++en)
        for (int l = 0; l < 6; ++l) cnt[conn[6 * en + l] + 1]++;
    for (int a = 0; a < N; ++a) cnt[a + 1] += cnt[a];
    std::vector<int> fan_ptr(cnt);
    std::vector<int2> fan(cnt[N]);
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    std::vector<int2> owner(N, make_int2(-1, 0));
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
            int sx = m->Lx > 0 ? (int)std::lround((m->X[a].x - px) / m->Lx) : 0;
            int sy = m->Ly > 0 ? (int)std::lround((m->X[a].y - py) / m->Ly) : 0;
            if (sx < -1 || sx > 1 || sy < -1 || sy > 1)
                return fail(ALELB_ERR_MESH, "node far outside its element frame");
            fan[fill[a]++] = make_int2(en, l | ((sx + 1) << 4) | ((sy + 1) << 6));
            int cur = owner[a].x;
            if (cur < 0 || area2[eo] > area2[e2o[cur]] ||
                (area2[eo] == area2[e2o[cur]] && eo < e2o[cur]))
                owner[a] = make_int2(en, l);
        }
    }
    std::vector<uint8_t> bkind(N, 0);
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
                m->wedges.push_back(make_int2(en, k));
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
    // wall probes B = A + n dt, located by breadth-first search over the
    // adjacency from the node's fan (tie rule as everywhere else)
    std::vector<int> wall_idx(N, -1), probe_e;
    std::vector<double2> probe_xi;
    {
        std::vector<int> seen(E, -1);
        for (int a = 0; a < N; ++a) {
            if (!is_wall[a]) continue;
            double nx = wn[a].x, ny = wn[a].y, L = std::sqrt(nx * nx + ny * ny);
            nx /= L;
            ny /= L;
            double Bx = m->X[a].x + nx * 1.0, By = m->X[a].y + ny * 1.0;
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
                double ox = cur.sx * m->Lx, oy = cur.sy * m->Ly;
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
            if (best < 0) return fail(ALELB_ERR_MESH, "wall probe point B lies outside the mesh");
            double2 v0 = ev[3 * best], v1 = ev[3 * best + 1], v2 = ev[3 * best + 2];
            double x0 = v0.x + bsx * m->Lx, y0 = v0.y + bsy * m->Ly;
            double x_xi = v1.x - v0.x, x_eta = v2.x - v0.x, y_xi = v1.y - v0.y, y_eta = v2.y - v0.y;
            double detJ = x_xi * y_eta - y_xi * x_eta;
            wall_idx[a] = (int)probe_e.size();
            probe_e.push_back(best);
            probe_xi.push_back(make_double2((y_eta * (Bx - x0) - x_eta * (By - y0)) / detJ,
                                            (-y_xi * (Bx - x0) + x_xi * (By - y0)) / detJ));
        }
    }
    m->n_wall_nodes = (int)probe_e.size();
    // static per-node map factors (host libm, same expressions everywhere)
    int nms = 0;
    std::vector<double> ms;
    if (m->mkind == MK_SINE) {
        nms = 6;
        ms.assign((size_t)6 * N, 0.0);
        double A = m->mp[0], L = m->mp[1];
        double w = 2.0 * M_PI / L;
        for (int a = 0; a < N; ++a) {
            double Xx = m->X[a].x, Yy = m->X[a].y;
            double f[6];
            if (m->mp[3] == 0.0) {
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
    } else if (m->mkind == MK_BLENDED) {
        nms = 3;
        ms.assign((size_t)3 * N, 0.0);
        double Xc = m->mp[3], Yc = m->mp[4], r1 = m->mp[5], r2 = m->mp[6];
        for (int a = 0; a < N; ++a) {
            double dx = m->X[a].x - Xc, dy = m->X[a].y - Yc;
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
    (void)nms;
    // upload
    cudaError_t st = cudaSuccess;
    DevBuf &B = m->buf;
    MeshDev &D = m->dev;
    D.N = N;
    D.E = E;
    D.Lx = m->Lx;
    D.Ly = m->Ly;
    D.X = B.put(m->X, st);
    D.ev = B.put(ev, st);
    D.nbr = B.put(nbr, st);
    D.einfo = B.put(einfo, st);
    D.rank = B.put(rank, st);
    D.conn = B.put(conn, st);
    D.fan_ptr = B.put(fan_ptr, st);
    D.fan = B.put(fan, st);
    D.owner = B.put(owner, st);
    D.bkind = B.put(bkind, st);
    D.wall_idx = B.put(wall_idx, st);
    D.probe_e = B.put(probe_e, st);
    D.probe_xi = B.put(probe_xi, st);
    D.orig_elem = B.put(orig, st);
    m->d_wedges = B.put(m->wedges, st);
    m->nw = (int)m->wedges.size();
    m->mst.kind = m->mkind;
    m->mst.Xc = m->mp[3];
    m->mst.Yc = m->mp[4];
    m->mst.N = N;
    m->mst.ms = B.put(ms, st);
    // P2 derivative tables at the six node positions
    static const double LXI[6][2] = {{0, 0}, {1, 0}, {0, 1}, {0.5, 0}, {0.5, 0.5}, {0, 0.5}};
    double dxi[6][6], deta[6][6];
    for (int l = 0; l < 6; ++l) {
        double xi = LXI[l][0], eta = LXI[l][1], l0 = 1.0 - xi - eta;
        double nx[6] = {-(4 * l0 - 1), 4 * xi - 1, 0, 4 * (l0 - xi), 4 * eta, -4 * eta};
        double ne[6] = {-(4 * l0 - 1), 0, 4 * eta - 1, -4 * xi, 4 * xi, 4 * (l0 - eta)};
        for (int s = 0; s < 6; ++s) {
            dxi[l][s] = nx[s];
            deta[l][s] = ne[s];
        }
    }
    if (st == cudaSuccess) st = cudaMemcpyToSymbol(c_dNxi, dxi, sizeof(dxi));
    if (st == cudaSuccess) st = cudaMemcpyToSymbol(c_dNeta, deta, sizeof(deta));
    if (st != cudaSuccess) {
        m->buf.release();
        return fail(st == cudaErrorMemoryAllocation ? ALELB_ERR_OOM : ALELB_ERR_CUDA,
                    cudaGetErrorString(st));
    }
    *out = m;
    return ALELB_OK;
}

extern "C" void alelb_mesh_destroy(alelb_mesh *m)
{
    if (!m) return;
    m->buf.release();
    delete m;
}

extern "C" const char *alelb_mesh_last_error(alelb_mesh *m) { return m ? m->err.c_str() : "null mesh"; }

extern "C" alelb_status alelb_mesh_move(alelb_mesh *m, double t)
{
    if (!m) return ALELB_ERR_ARG;
    MapScalars S = map_scalars(m->mkind, m->mp, t);
    int *d_bad = nullptr, bad = 0;
    cudaError_t st = cudaMalloc(&d_bad, sizeof(int));
    if (st == cudaSuccess) st = cudaMemset(d_bad, 0, sizeof(int));
    if (st == cudaSuccess) {
        k_check_map<<<(m->N + 255) / 256, 256>>>(m->mst, S, m->dev.X, m->N, d_bad);
        st = cudaGetLastError();
    }
    if (st == cudaSuccess) st = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (d_bad) cudaFree(d_bad);
    if (st != cudaSuccess) {
        m->err = cudaGetErrorString(st);
        return ALELB_ERR_CUDA;
    }
    if (bad) {
        m->err = "det g <= 0 at " + std::to_string(bad) + " nodes";
        return ALELB_ERR_MAP;
    }
    return ALELB_OK;
}

// ============================================================================
// solver
// ============================================================================
namespace {

enum { KT_STREAM = 0, KT_DERIV1 = 1, KT_COLLIDE = 2, KT_N = 3 };
const char *KT_NAMES[KT_N] = {"k_stream", "k_deriv1", "k_collide"};

// Reference and far-field populations computed on the device with the
// same kernel code that the step uses.
__global__ void k_kin_consts(KinParams<double> K, double rho_inf, double uxi, double uyi,
                             double T_inf, int dev_mode, double *out)
{
    double f[NQ], g[NQ], M0, qx, qy, Rxx, Rxy, Ryy, pr, px, py;
    // reference state (rest at rho_inf, T_inf)
    feq9(rho_inf, 0.0, 0.0, T_inf, f);
    double E0 = K.Cv * T_inf;
    gmoments(rho_inf, 0.0, 0.0, T_inf, E0, M0, qx, qy, Rxx, Rxy, Ryy);
    psi_terms(rho_inf, 0.0, 0.0, T_inf, E0, pr, px, py);
    gform9(T_inf, M0, qx, qy, Rxx, Rxy, Ryy, pr, px, py, g);
    for (int i = 0; i < NQ; ++i) {
        out[i] = dev_mode ? f[i] : 0.0;
        out[NQ + i] = dev_mode ? g[i] : 0.0;
    }
    // far field
    feq9(rho_inf, uxi, uyi, T_inf, f);
    double E = K.Cv * T_inf + 0.5 * (uxi * uxi + uyi * uyi);
    gmoments(rho_inf, uxi, uyi, T_inf, E, M0, qx, qy, Rxx, Rxy, Ryy);
    psi_terms(rho_inf, uxi, uyi, T_inf, E, pr, px, py);
    gform9(T_inf, M0, qx, qy, Rxx, Rxy, Ryy, pr, px, py, g);
    for (int i = 0; i < NQ; ++i) {
        out[2 * NQ + i] = f[i];
        out[3 * NQ + i] = g[i];
    }
}

// Free-stream state (deviations) and fields.
template <class S>
__global__ void k_fill_uniform(StateDev<S> st, int N, const double *consts, double rho,
                               double ux, double uy, double T)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    for (int i = 0; i < NQ; ++i) {
        st.post[i * N + a] = (S)(consts[2 * NQ + i] - consts[i]);
        st.post[(NQ + i) * N + a] = (S)(consts[3 * NQ + i] - consts[NQ + i]);
    }
    st.rho[a] = (S)rho;
    st.ux[a] = (S)ux;
    st.uy[a] = (S)uy;
    st.T[a] = (S)T;
}

// Full FP64 populations <-> stored deviations (internal order).
template <class S>
__global__ void k_import(StateDev<S> st, int N, const double *consts, const double *full,
                         const double *fields, int have_fields, double Cv)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    double r = 0, jx = 0, jy = 0, e2 = 0;
    for (int i = 0; i < NQ; ++i) {
        double f = full[i * N + a], g = full[(NQ + i) * N + a];
        st.post[i * N + a] = (S)(f - consts[i]);
        st.post[(NQ + i) * N + a] = (S)(g - consts[NQ + i]);
        r += f;
        jx += c_cx[i] * f;
        jy += c_cy[i] * f;
        e2 += g;
    }
    if (have_fields) {
        st.rho[a] = (S)fields[a];
        st.ux[a] = (S)fields[N + a];
        st.uy[a] = (S)fields[2 * N + a];
        st.T[a] = (S)fields[3 * N + a];
    } else {
        double ux = jx / r, uy = jy / r, E = e2 / (2 * r);
        st.rho[a] = (S)r;
        st.ux[a] = (S)ux;
        st.uy[a] = (S)uy;
        st.T[a] = (S)((E - 0.5 * (ux * ux + uy * uy)) / Cv);
    }
}

template <class S>
__global__ void k_export(StateDev<S> st, int N, const double *consts, double *full, double *fields)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    if (full)
        for (int i = 0; i < NQ; ++i) {
            full[i * N + a] = (double)st.post[i * N + a] + consts[i];
            full[(NQ + i) * N + a] = (double)st.post[(NQ + i) * N + a] + consts[NQ + i];
        }
    if (fields) {
        fields[a] = (double)st.rho[a];
        fields[N + a] = (double)st.ux[a];
        fields[2 * N + a] = (double)st.uy[a];
        fields[3 * N + a] = (double)st.T[a];
    }
}

} // namespace

struct alelb_solver {
    alelb_mesh *mesh = nullptr;
    std::string err;
    int prec = 0, flags = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double gamma = 1.4, Pr = 0.71, mu = 0, rho_inf = 1, T_inf = 0.3, uinf[2] = {0, 0}, chord = 1;
    double Cv = 2.5, Cp = 3.5;
    double t = 0;
    int64_t nstep = 0;
    StateDev<double> sd{};
    StateDev<float> sf{};
    KinParams<double> kd{};
    KinParams<float> kf{};
    double consts[4 * NQ] = {0};
    double *d_consts = nullptr;
    double *d_scratch = nullptr; // 22 N doubles: import/export staging
    int *d_err = nullptr;
    double *d_out = nullptr;
    DevBuf buf;
    int sticky = 0;
    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { int k; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    double ms_acc[KT_N] = {0, 0, 0};
    int64_t n_acc[KT_N] = {0, 0, 0};
};

namespace {

alelb_status cuda_fail(alelb_solver *s, cudaError_t st)
{
    s->err = cudaGetErrorString(st);
    return st == cudaErrorMemoryAllocation ? ALELB_ERR_OOM : ALELB_ERR_CUDA;
}

void flush_prof(alelb_solver *s)
{
    for (auto &r : s->pending) {
        float ms = 0;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            s->ms_acc[r.k] += ms;
            s->n_acc[r.k] += 1;
        }
        s->ev_pool.push_back(r.a);
        s->ev_pool.push_back(r.b);
    }
    s->pending.clear();
}

cudaEvent_t get_event(alelb_solver *s)
{
    if (s->ev_pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
}

template <class S, class A>
cudaError_t launch_step(alelb_solver *s, StateDev<S> &st, KinParams<A> &K, const MapScalars &sc)
{
    alelb_mesh *m = s->mesh;
    const int N = m->N;
    const bool phi = !(s->flags & (ALELB_FLAG_PHI_OFF | ALELB_FLAG_COLLIDE_OFF));
    for (int k = 0; k < KT_N; ++k) {
        if (k == KT_DERIV1 && !phi) continue;
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (s->prof) {
            ea = get_event(s);
            eb = get_event(s);
            cudaEventRecord(ea, s->stream);
        }
        if (k == KT_STREAM)
            k_stream<S, A><<<(N + 127) / 128, 128, 0, s->stream>>>(m->dev, m->mst, sc, K, st, s->d_err);
        else if (k == KT_DERIV1)
            k_deriv1<S, A><<<(N + 255) / 256, 256, 0, s->stream>>>(m->dev, m->mst, sc, st);
        else
            k_collide<S, A><<<(N + 127) / 128, 128, 0, s->stream>>>(m->dev, m->mst, sc, K, st, s->d_err);
        if (s->prof) {
            cudaEventRecord(eb, s->stream);
            s->pending.push_back({k, ea, eb});
        }
    }
    return cudaGetLastError();
}

template <class A> void fill_kin(alelb_solver *s, KinParams<A> &K)
{
    K.Cv = (A)s->Cv;
    K.Cp = (A)s->Cp;
    K.mu = (A)s->mu;
    K.Pr = (A)s->Pr;
    double rref = 0, e2 = 0;
    for (int i = 0; i < NQ; ++i) {
        K.fref[i] = (A)s->consts[i];
        K.gref[i] = (A)s->consts[NQ + i];
        K.finf[i] = (A)(s->consts[2 * NQ + i] - s->consts[i]);
        K.ginf[i] = (A)(s->consts[3 * NQ + i] - s->consts[NQ + i]);
        rref += s->consts[i];
        e2 += s->consts[NQ + i];
    }
    K.rho_ref = (A)rref;
    K.E2_ref = (A)e2;
    K.T_ref = (A)(s->prec == ALELB_PREC_FP64 ? 0.0 : s->T_inf);
    K.flags = s->flags;
}

alelb_status check_sticky(alelb_solver *s)
{
    if (s->sticky & ERR_LOCATE) {
        s->err = "element walk exceeded its step limit";
        return ALELB_ERR_LOCATE;
    }
    if (s->sticky & ERR_NONFINITE) {
        s->err = "non-finite or non-positive density or temperature";
        return ALELB_ERR_NONFINITE;
    }
    return ALELB_OK;
}

} // namespace

extern "C" alelb_status alelb_lb_init(alelb_mesh *m, const alelb_params *p, alelb_solver **out)
{
    if (!m || !p || !out) return ALELB_ERR_ARG;
    if (!(p->gamma > 1.0) || !(p->Pr > 0) || !(p->mu > 0) || !(p->rho_inf > 0) || !(p->T_inf > 0) ||
        (p->precision != ALELB_PREC_FP64 && p->precision != ALELB_PREC_FP32_DEV))
        return ALELB_ERR_ARG;
    alelb_solver *s = new (std::nothrow) alelb_solver();
    if (!s) return ALELB_ERR_OOM;
    *out = s;
    s->mesh = m;
    s->prec = p->precision;
    s->flags = p->flags;
    s->gamma = p->gamma;
    s->Pr = p->Pr;
    s->mu = p->mu;
    s->rho_inf = p->rho_inf;
    s->T_inf = p->T_inf;
    s->uinf[0] = p->u_inf[0];
    s->uinf[1] = p->u_inf[1];
    s->chord = p->chord;
    s->Cv = 1.0 / (p->gamma - 1.0);
    s->Cp = s->Cv + 1.0;
    cudaError_t st = cudaSuccess;
    if (p->stream) {
        s->stream = (cudaStream_t)p->stream;
    } else {
        st = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        s->own_stream = true;
    }
    const int N = m->N;
    if (s->prec == ALELB_PREC_FP64) put_state(s->buf, s->sd, N, st);
    else put_state(s->buf, s->sf, N, st);
    s->d_consts = s->buf.alloc<double>(4 * NQ, st);
    s->d_scratch = s->buf.alloc<double>((size_t)22 * N, st);
    s->d_err = s->buf.alloc<int>(1, st);
    s->d_out = s->buf.alloc<double>(8, st);
    if (st != cudaSuccess) return cuda_fail(s, st);
    KinParams<double> K0{};
    K0.Cv = s->Cv;
    k_kin_consts<<<1, 1, 0, s->stream>>>(K0, s->rho_inf, s->uinf[0], s->uinf[1], s->T_inf,
                                         s->prec == ALELB_PREC_FP32_DEV, s->d_consts);
    st = cudaGetLastError();
    if (st == cudaSuccess)
        st = cudaMemcpyAsync(s->consts, s->d_consts, sizeof(s->consts), cudaMemcpyDeviceToHost, s->stream);
    if (st == cudaSuccess) st = cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream);
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    fill_kin(s, s->kd);
    fill_kin(s, s->kf);
    if (s->prec == ALELB_PREC_FP64)
        k_fill_uniform<double><<<(N + 255) / 256, 256, 0, s->stream>>>(
            s->sd, N, s->d_consts, s->rho_inf, s->uinf[0], s->uinf[1], s->T_inf);
    else
        k_fill_uniform<float><<<(N + 255) / 256, 256, 0, s->stream>>>(
            s->sf, N, s->d_consts, s->rho_inf, s->uinf[0], s->uinf[1], s->T_inf);
    st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    m->n_solvers++;
    return ALELB_OK;
}

extern "C" void alelb_solver_destroy(alelb_solver *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    flush_prof(s);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    s->buf.release();
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    if (s->mesh) s->mesh->n_solvers--;
    delete s;
}

extern "C" alelb_status alelb_lb_step(alelb_solver *s, int32_t n)
{
    if (!s || n < 0) return ALELB_ERR_ARG;
    if (!s->mesh) return ALELB_ERR_STATE;
    for (int k = 0; k < n; ++k) {
        double t1 = s->t + 1.0;
        MapScalars sc = map_scalars(s->mesh->mkind, s->mesh->mp, t1);
        cudaError_t st = s->prec == ALELB_PREC_FP64 ? launch_step(s, s->sd, s->kd, sc)
                                                     : launch_step(s, s->sf, s->kf, sc);
        if (st != cudaSuccess) return cuda_fail(s, st);
        s->t = t1;
        s->nstep++;
    }
    return ALELB_OK;
}

extern "C" alelb_status alelb_sync(alelb_solver *s)
{
    if (!s) return ALELB_ERR_ARG;
    int e = 0;
    cudaError_t st = cudaMemcpyAsync(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    s->sticky |= e;
    if (s->prof) flush_prof(s);
    return check_sticky(s);
}

extern "C" alelb_status alelb_time(alelb_solver *s, double *t, int64_t *step)
{
    if (!s) return ALELB_ERR_ARG;
    if (t) *t = s->t;
    if (step) *step = s->nstep;
    return ALELB_OK;
}

namespace {
alelb_status export_state(alelb_solver *s, bool pops, std::vector<double> &full,
                          std::vector<double> &fields)
{
    alelb_mesh *m = s->mesh;
    const int N = m->N;
    double *dfull = pops ? s->d_scratch : nullptr;
    double *dfields = s->d_scratch + (size_t)18 * N;
    if (s->prec == ALELB_PREC_FP64)
        k_export<double><<<(N + 255) / 256, 256, 0, s->stream>>>(s->sd, N, s->d_consts, dfull, dfields);
    else
        k_export<float><<<(N + 255) / 256, 256, 0, s->stream>>>(s->sf, N, s->d_consts, dfull, dfields);
    cudaError_t st = cudaGetLastError();
    fields.resize((size_t)4 * N);
    if (pops) full.resize((size_t)18 * N);
    if (st == cudaSuccess && pops)
        st = cudaMemcpyAsync(full.data(), dfull, (size_t)18 * N * sizeof(double),
                             cudaMemcpyDeviceToHost, s->stream);
    if (st == cudaSuccess)
        st = cudaMemcpyAsync(fields.data(), dfields, (size_t)4 * N * sizeof(double),
                             cudaMemcpyDeviceToHost, s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    return alelb_sync(s);
}
} // namespace

extern "C" alelb_status alelb_moments(alelb_solver *s, double *rho, double *ux, double *uy, double *T)
{
    if (!s) return ALELB_ERR_ARG;
    std::vector<double> full, fields;
    alelb_status r = export_state(s, false, full, fields);
    if (r != ALELB_OK) return r;
    const int N = s->mesh->N;
    double *outs[4] = {rho, ux, uy, T};
    for (int c = 0; c < 4; ++c)
        if (outs[c])
            for (int a = 0; a < N; ++a) outs[c][s->mesh->node_new2old[a]] = fields[(size_t)c * N + a];
    return ALELB_OK;
}

extern "C" alelb_status alelb_get_pops(alelb_solver *s, double *f, double *g)
{
    if (!s) return ALELB_ERR_ARG;
    std::vector<double> full, fields;
    alelb_status r = export_state(s, true, full, fields);
    if (r != ALELB_OK) return r;
    const int N = s->mesh->N;
    for (int i = 0; i < NQ; ++i)
        for (int a = 0; a < N; ++a) {
            int o = s->mesh->node_new2old[a];
            if (f) f[(size_t)i * N + o] = full[(size_t)i * N + a];
            if (g) g[(size_t)i * N + o] = full[(size_t)(NQ + i) * N + a];
        }
    return ALELB_OK;
}

extern "C" alelb_status alelb_set_pops(alelb_solver *s, const double *f, const double *g,
                                       const double *rho, const double *ux, const double *uy,
                                       const double *T, double t)
{
    if (!s || !f || !g) return ALELB_ERR_ARG;
    const int N = s->mesh->N;
    std::vector<double> full((size_t)18 * N), fields((size_t)4 * N, 0.0);
    bool have = rho && ux && uy && T;
    for (int a = 0; a < N; ++a) {
        int o = s->mesh->node_new2old[a];
        for (int i = 0; i < NQ; ++i) {
            full[(size_t)i * N + a] = f[(size_t)i * N + o];
            full[(size_t)(NQ + i) * N + a] = g[(size_t)i * N + o];
        }
        if (have) {
            fields[a] = rho[o];
            fields[(size_t)N + a] = ux[o];
            fields[(size_t)2 * N + a] = uy[o];
            fields[(size_t)3 * N + a] = T[o];
        }
    }
    cudaError_t st = cudaMemcpyAsync(s->d_scratch, full.data(), full.size() * sizeof(double),
                                     cudaMemcpyHostToDevice, s->stream);
    if (st == cudaSuccess)
        st = cudaMemcpyAsync(s->d_scratch + (size_t)18 * N, fields.data(), fields.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    if (s->prec == ALELB_PREC_FP64)
        k_import<double><<<(N + 255) / 256, 256, 0, s->stream>>>(
            s->sd, N, s->d_consts, s->d_scratch, s->d_scratch + (size_t)18 * N, have, s->Cv);
    else
        k_import<float><<<(N + 255) / 256, 256, 0, s->stream>>>(
            s->sf, N, s->d_consts, s->d_scratch, s->d_scratch + (size_t)18 * N, have, s->Cv);
    st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    s->t = t;
    return ALELB_OK;
}

extern "C" alelb_status alelb_forces(alelb_solver *s, double out[6])
{
    if (!s || !out) return ALELB_ERR_ARG;
    alelb_mesh *m = s->mesh;
    MapScalars sc = map_scalars(m->mkind, m->mp, s->t);
    if (m->nw > 0) {
        if (s->prec == ALELB_PREC_FP64)
            k_forces<double><<<1, 256, 0, s->stream>>>(m->dev, m->mst, sc, s->sd, m->d_wedges, m->nw,
                                                       s->mu, s->Cv, s->d_out);
        else
            k_forces<float><<<1, 256, 0, s->stream>>>(m->dev, m->mst, sc, s->sf, m->d_wedges, m->nw,
                                                      s->mu, s->Cv, s->d_out);
    } else {
        cudaMemsetAsync(s->d_out, 0, 4 * sizeof(double), s->stream);
    }
    double F[4];
    cudaError_t st = cudaGetLastError();
    if (st == cudaSuccess)
        st = cudaMemcpyAsync(F, s->d_out, sizeof(F), cudaMemcpyDeviceToHost, s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    alelb_status r = alelb_sync(s);
    if (r != ALELB_OK) return r;
    double U2 = s->uinf[0] * s->uinf[0] + s->uinf[1] * s->uinf[1], U = std::sqrt(U2);
    double ex = U > 0 ? s->uinf[0] / U : 1.0, ey = U > 0 ? s->uinf[1] / U : 0.0;
    double q = 0.5 * s->rho_inf * U2 * s->chord;
    double Fx = F[0] + F[2], Fy = F[1] + F[3];
    for (int k = 0; k < 4; ++k) out[k] = F[k];
    out[4] = q > 0 ? (Fx * ex + Fy * ey) / q : 0.0;
    out[5] = q > 0 ? (-Fx * ey + Fy * ex) / q : 0.0;
    return ALELB_OK;
}

extern "C" alelb_status alelb_locate(alelb_solver *s, double t, int32_t *elem, int8_t *kind)
{
    if (!s || !elem || !kind) return ALELB_ERR_ARG;
    alelb_mesh *m = s->mesh;
    const int N = m->N;
    MapScalars sc = map_scalars(m->mkind, m->mp, t);
    int *de = (int *)s->d_scratch;
    int8_t *dk = (int8_t *)(s->d_scratch + (size_t)9 * N);
    k_locate<<<(N + 127) / 128, 128, 0, s->stream>>>(m->dev, m->mst, sc, s->flags, de, dk, s->d_err);
    std::vector<int> he((size_t)9 * N);
    std::vector<int8_t> hk((size_t)9 * N);
    cudaError_t st = cudaGetLastError();
    if (st == cudaSuccess)
        st = cudaMemcpyAsync(he.data(), de, he.size() * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (st == cudaSuccess)
        st = cudaMemcpyAsync(hk.data(), dk, hk.size(), cudaMemcpyDeviceToHost, s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    alelb_status r = alelb_sync(s);
    if (r != ALELB_OK) return r;
    for (int i = 0; i < NQ; ++i)
        for (int a = 0; a < N; ++a) {
            int o = m->node_new2old[a];
            elem[(size_t)i * N + o] = he[(size_t)i * N + a];
            kind[(size_t)i * N + o] = hk[(size_t)i * N + a];
        }
    return ALELB_OK;
}

extern "C" alelb_status alelb_profile(alelb_solver *s, int32_t enable)
{
    if (!s) return ALELB_ERR_ARG;
    if (s->prof) {
        cudaStreamSynchronize(s->stream);
        flush_prof(s);
    }
    s->prof = enable != 0;
    for (int k = 0; k < KT_N; ++k) {
        s->ms_acc[k] = 0;
        s->n_acc[k] = 0;
    }
    return ALELB_OK;
}

extern "C" alelb_status alelb_kernel_times(alelb_solver *s, const char **names, double *ms,
                                           int64_t *launches, int32_t *n)
{
    if (!s || !n) return ALELB_ERR_ARG;
    cudaStreamSynchronize(s->stream);
    flush_prof(s);
    int cap = *n;
    for (int k = 0; k < KT_N && k < cap; ++k) {
        if (names) names[k] = KT_NAMES[k];
        if (ms) ms[k] = s->ms_acc[k];
        if (launches) launches[k] = s->n_acc[k];
    }
    *n = KT_N;
    return ALELB_OK;
}

extern "C" alelb_status alelb_info(alelb_solver *s, double out[8])
{
    if (!s || !out) return ALELB_ERR_ARG;
    alelb_mesh *m = s->mesh;
    double sz = s->prec == ALELB_PREC_FP64 ? 8.0 : 4.0;
    out[0] = m->N;
    out[1] = m->E;
    out[2] = sz;
    out[3] = 0;
    out[4] = m->n_wall_nodes;
    out[5] = s->prec;
    out[6] = m->nw;
    out[7] = 0;
    return ALELB_OK;
}

extern "C" const char *alelb_last_error(alelb_solver *s) { return s ? s->err.c_str() : "null solver"; }
