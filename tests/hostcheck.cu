// hostcheck.cu -- the library's device element walk compiled for the host,
// for CPU tests of the walk against the oracle (test tooling; not on the
// product path).  Builds the same tables as alelb_mesh_create and runs the same
// per-node location routine that k_locate runs.
#include <cstring>
#include <string>

#include "quad_tables.h"
#include "tables.h"

using namespace alelb;

static QuadDev quad_host_view(const HostTables &T, const QuadTables &Q)
{
    QuadDev M{};
    M.N = T.N;
    M.E = T.E;
    M.Lx = T.Lx;
    M.Ly = T.Ly;
    M.X = T.X.data();
    M.ev = Q.ev.data();
    M.nbr = Q.nbr.data();
    M.einfo = Q.einfo.data();
    M.rank = Q.rank.data();
    M.conn = Q.conn.data();
    M.fan_ptr = Q.fan_ptr.data();
    M.fan = Q.fan.data();
    M.owner = Q.owner.data();
    M.bcel = Q.bcel.data();
    M.bkind = Q.bkind.data();
    M.orig_elem = Q.orig.data();
    M.Xf = Q.Xf.data();
    M.evf = Q.evf.data();
    M.bdist = Q.bdist.data();
    M.ownJf = Q.ownJf.data();
    return M;
}

// The quadrilateral walk (quad_walk, the routine kq_locate runs) on the
// host, for meshes of 9-node quadrilaterals.
extern "C" int alelb_hostcheck_locate_q2(const alelb_mesh_desc *d, double t, int literal, int32_t *elem,
                                         int8_t *kind, char *errbuf, int errlen)
{
    HostTables T;
    QuadTables Q;
    std::string err;
    alelb_status st = build_quad_tables(d, T, Q, err);
    if (st != ALELB_OK) {
        if (errbuf && errlen > 0) std::strncpy(errbuf, err.c_str(), errlen - 1);
        return st;
    }
    const QuadDev M = quad_host_view(T, Q);
    MapStatic MS = T.host_map();
    MapScalars sc = map_scalars(T.mkind, T.mp, t);
    int e = 0;
    const int N = T.N;
    for (int a = 0; a < N; ++a) {
        const double2 Xa = M.X[a];
        double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22, wx, wy;
        map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
        metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
        mesh_velocity_term(a11, a12, a21, a22, ds(Vx, sc.Ux), ds(Vy, sc.Uy), literal != 0, wx, wy);
        const int o = T.node_new2old[a];
        for (int i = 0; i < NQ; ++i) {
            double chx, chy, px, py;
            departure(a11, a12, a21, a22, wx, wy, (double)lat_cx(i), (double)lat_cy(i), Xa.x, Xa.y, chx, chy, px,
                      py);
            int el = -2, k = 0;
            if (!(chx == 0.0 && chy == 0.0)) {
                const Loc L = quad_walk(M, a, Xa.x, Xa.y, px, py, &e);
                if (L.e >= 0) {
                    el = M.orig_elem[L.vnode >= 0 ? quad_fan_best(M, L.vnode) : L.e];
                } else if (L.e == -1) {
                    el = -1;
                    k = L.kind;
                }
            }
            elem[(size_t)i * N + o] = el;
            kind[(size_t)i * N + o] = (int8_t)k;
        }
    }
    return e ? ALELB_ERR_LOCATE : ALELB_OK;
}

extern "C" int alelb_hostcheck_locate(const alelb_mesh_desc *d, double t, int literal,
                                      int32_t *elem, int8_t *kind, char *errbuf, int errlen)
{
    HostTables T;
    std::string err;
    alelb_status st = build_tables(d, T, err);
    if (st != ALELB_OK) {
        if (errbuf && errlen > 0) std::strncpy(errbuf, err.c_str(), errlen - 1);
        return st;
    }
    MeshDev M = T.host_view();
    MapStatic MS = T.host_map();
    MapScalars sc = map_scalars(T.mkind, T.mp, t);
    int e = 0;
    const int N = T.N;
    for (int a = 0; a < N; ++a) {
        int e9[NQ];
        int8_t k9[NQ];
        locate_node(M, MS, sc, literal, a, e9, k9, &e);
        int o = T.node_new2old[a];
        for (int i = 0; i < NQ; ++i) {
            elem[(size_t)i * N + o] = e9[i];
            kind[(size_t)i * N + o] = k9[i];
        }
    }
    return e ? ALELB_ERR_LOCATE : ALELB_OK;
}

// The certified FP32 strict-containment filter of the fast propagation path,
// on the host: out[k] = 1 when the filter accepts point k in element elem[k]
// (internal numbering of the Morton-renumbered mesh; frame shift 0).
extern "C" int alelb_hostcheck_inside(const alelb_mesh_desc *d, int n, const int32_t *elem_orig,
                                      const double *px, const double *py, int8_t *out)
{
    HostTables T;
    std::string err;
    alelb_status st = build_tables(d, T, err);
    if (st != ALELB_OK) return st;
    MeshDev M = T.host_view();
    for (int k = 0; k < n; ++k) {
        float qx, qy;
        int e = T.elem_old2new[elem_orig[k]];
        out[k] = strictly_inside_f32(M, e, 0, 0, px[k], py[k], qx, qy) ? 1 : 0;
    }
    return ALELB_OK;
}


// The FP32-deviation propagation's element decisions on the host: the cache
// is what an exact walk at t_prev leaves (each population's element), then
// every population at t takes the fast decision where it applies and the
// walk elsewhere.  fast[] marks the populations the fast path settled.
extern "C" int alelb_hostcheck_fast(const alelb_mesh_desc *d, double t_prev, double t, int32_t *elem,
                                    int8_t *kind, int8_t *fast)
{
    HostTables T;
    std::string err;
    alelb_status st = build_tables(d, T, err);
    if (st != ALELB_OK) return st;
    MeshDev M = T.host_view();
    MapStatic MS = T.host_map();
    const int N = T.N;
    std::vector<int> cache((size_t)9 * N, -1);
    int e = 0;
    {
        MapScalars sc = map_scalars(T.mkind, T.mp, t_prev);
        for (int a = 0; a < N; ++a) {
            const double2 Xa = M.X[a];
            double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22, wx, wy;
            map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
            metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
            mesh_velocity_term(a11, a12, a21, a22, ds(Vx, sc.Ux), ds(Vy, sc.Uy), false, wx, wy);
            const int CXh[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
            const int CYh[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
            for (int i = 0; i < NQ; ++i) {
                double chx, chy, px, py;
                departure(a11, a12, a21, a22, wx, wy, CXh[i], CYh[i], Xa.x, Xa.y, chx, chy, px, py);
                if (chx == 0.0 && chy == 0.0) continue;
                Loc L = walk(M, a, Xa.x, Xa.y, px, py, &e);
                if (L.e >= 0 && L.vnode < 0) cache[(size_t)i * N + a] = L.e | ((L.sx + 1) << 28) | ((L.sy + 1) << 30);
            }
        }
    }
    MapScalars sc = map_scalars(T.mkind, T.mp, t);
    MapScalarsF sf{};
    sf.s = (float)sc.s;
    sf.sd = (float)sc.sd;
    sf.vy = (float)sc.vy;
    sf.c = (float)sc.c;
    sf.sn = (float)sc.sn;
    sf.thd = (float)sc.thd;
    sf.cm = (float)sc.cm;
    sf.Xc = (float)T.mp[3];
    sf.Yc = (float)T.mp[4];
    sf.er0 = 2.0f;
    for (int a = 0; a < N; ++a) {
        int e9[NQ];
        int8_t k9[NQ], f9[NQ];
        mixed_locate_node(M, MS, sc, sf, cache.data(), a, e9, k9, f9, &e);
        const int o = T.node_new2old[a];
        for (int i = 0; i < NQ; ++i) {
            elem[(size_t)i * N + o] = e9[i];
            kind[(size_t)i * N + o] = k9[i];
            fast[(size_t)i * N + o] = f9[i];
        }
    }
    return e ? ALELB_ERR_LOCATE : ALELB_OK;
}

// The library's exact orientation predicate on the host: out[k] = sign of
// orient(a, b, c) for the k-th six doubles (ax, ay, bx, by, cx, cy); stage[k]
// = the integer stage's answer alone (2 where it does not apply).
extern "C" void alelb_hostcheck_orient(const double *p, int n, int32_t *out, int32_t *stage)
{
    for (int k = 0; k < n; ++k) {
        const double *q = p + 6 * k;
        out[k] = orient(q[0], q[1], q[2], q[3], q[4], q[5]);
        stage[k] = orient_int(q[0], q[1], q[2], q[3], q[4], q[5]);
    }
}

// The deviation forms' decisions on quadrilaterals at map time t with the
// element cache an exact walk at t_prev leaves (quad_fast_decide, then the
// walk), on the host: elem/kind as alelb_locate, fast = 1 where the
// certified FP32 check settled the population.
extern "C" int alelb_hostcheck_fast_q2(const alelb_mesh_desc *d, double t_prev, double t, int32_t *elem,
                                       int8_t *kind, int8_t *fast)
{
    HostTables T;
    QuadTables Q;
    std::string err;
    alelb_status st = build_quad_tables(d, T, Q, err);
    if (st != ALELB_OK) return st;
    const QuadDev M = quad_host_view(T, Q);
    MapStatic MS = T.host_map();
    const int N = T.N;
    std::vector<int> cache((size_t)9 * N, -1);
    int e = 0;
    auto depart = [&](const MapScalars &sc, int a, int i, double &chx, double &chy, double &px, double &py) {
        const double2 Xa = M.X[a];
        double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22, wx, wy;
        map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
        metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
        mesh_velocity_term(a11, a12, a21, a22, ds(Vx, sc.Ux), ds(Vy, sc.Uy), false, wx, wy);
        departure(a11, a12, a21, a22, wx, wy, (double)lat_cx(i), (double)lat_cy(i), Xa.x, Xa.y, chx, chy, px, py);
    };
    {
        const MapScalars sc = map_scalars(T.mkind, T.mp, t_prev);
        for (int a = 0; a < N; ++a)
            for (int i = 0; i < NQ; ++i) {
                double chx, chy, px, py;
                depart(sc, a, i, chx, chy, px, py);
                if (chx == 0.0 && chy == 0.0) continue;
                const Loc L = quad_walk(M, a, M.X[a].x, M.X[a].y, px, py, &e);
                if (L.e >= 0) cache[(size_t)i * N + a] = L.e | ((L.sx + 1) << 28) | ((L.sy + 1) << 30);
            }
    }
    const MapScalars sc = map_scalars(T.mkind, T.mp, t);
    MapScalarsF sf{};
    sf.s = (float)sc.s;
    sf.sd = (float)sc.sd;
    sf.vy = (float)sc.vy;
    sf.c = (float)sc.c;
    sf.sn = (float)sc.sn;
    sf.thd = (float)sc.thd;
    sf.cm = (float)sc.cm;
    sf.Xc = (float)T.mp[3];
    sf.Yc = (float)T.mp[4];
    sf.er0 = 2.0f;
    for (int a = 0; a < N; ++a) {
        const FastMap F = fast_map(MS, sf, a, M.Xf[a]);
        const int o = T.node_new2old[a];
        for (int i = 0; i < NQ; ++i) {
            int el = -2, k = 0, f = 0, ef;
            float cw[8];
            if (quad_fast_decide(M, F, M.Xf[a], a, i, cache[(size_t)i * N + a], ef, cw)) {
                el = M.orig_elem[ef];
                f = 1;
            } else {
                double chx, chy, px, py;
                depart(sc, a, i, chx, chy, px, py);
                if (!(chx == 0.0 && chy == 0.0)) {
                    const Loc L = quad_walk(M, a, M.X[a].x, M.X[a].y, px, py, &e);
                    if (L.e >= 0) el = M.orig_elem[L.vnode >= 0 ? quad_fan_best(M, L.vnode) : L.e];
                    else if (L.e == -1) {
                        el = -1;
                        k = L.kind;
                    }
                }
            }
            elem[(size_t)i * N + o] = el;
            kind[(size_t)i * N + o] = (int8_t)k;
            fast[(size_t)i * N + o] = (int8_t)f;
        }
    }
    return e ? ALELB_ERR_LOCATE : ALELB_OK;
}
