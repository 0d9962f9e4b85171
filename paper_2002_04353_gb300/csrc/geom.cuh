// geom.cuh -- device geometry of the ALE propagation (Sec. II, Sec. III):
// the mesh map and its metrics, the transformed discrete velocities, the
// departure points, an exact orientation predicate and the straight-line
// element walk that locates each departure point.
//
// Bitwise agreement of element choices with an independent FP64 reference
// requires that the departure point be computed with one fixed sequence of
// correctly rounded FP64 operations.  Every FP64 operation on that path is
// therefore written with __dadd_rn/__dsub_rn/__dmul_rn/__ddiv_rn, which the
// compiler never contracts into FMAs; the sequence is:
//   det g = x_X y_Y - y_X x_Y,  inv = 1/det g,
//   A = g^{-1,T} = [[y_Y inv, -(x_Y inv)], [-(y_X inv), x_X inv]],
//   w = A V_G,  c^_i = (A c_i) - w,  X_dp = X - c^_i     (dt = 1)
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

namespace alelb {

constexpr int NQ = 9;
__constant__ int c_cx[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int c_cy[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};


enum : int { MK_NONE = 0, MK_SINE = 1, MK_PLUNGE = 2, MK_PITCH = 3, MK_PITCH_PLUNGE = 4,
             MK_BLENDED = 5 };
enum : int { ERR_LOCATE = 1, ERR_NONFINITE = 2, ERR_TIMEOUT = 4 };

// Per-step scalars of the map (host libm, once per step).
struct MapScalars {
    double s, sd;      // sine map: s(t), s'(t)
    double vy, yoff;   // plunge velocity and offset
    double c, sn, thd; // rotation: cos, sin, angular rate
    double cm;         // cos - 1
    double Ux, Uy;     // lattice shift U: the velocities are c_i + U (zero when unshifted)
};

struct MapStatic {
    int kind;
    double Xc, Yc;
    const double *ms; // per-node static factors, SoA [k * N + a]
    const float *msf; // the same rounded to FP32
    int N;
};

// The geometry is compiled for the device and, for the CPU check of the
// walk, for the host; host code is built without FP contraction, so the
// plain operators round exactly like the intrinsics.
#define ALELB_HD __host__ __device__

// The same lattice velocities for a run-time direction index, formed from
// comparisons so that they stay in registers.
ALELB_HD __forceinline__ int lat_cx(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
ALELB_HD __forceinline__ int lat_cy(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
ALELB_HD __forceinline__ double dm(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
ALELB_HD __forceinline__ double da(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
ALELB_HD __forceinline__ double ds(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}
ALELB_HD __forceinline__ double ddiv(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __ddiv_rn(a, b);
#else
    return a / b;
#endif
}
ALELB_HD __forceinline__ double dfma(double a, double b, double c)
{
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}
ALELB_HD __forceinline__ void set_err(int *err, int bit)
{
#ifdef __CUDA_ARCH__
    atomicOr(err, bit);
#else
    *err |= bit;
#endif
}

// Metrics x_X, x_Y, y_X, y_Y and mesh velocity V_G at a node.
ALELB_HD __forceinline__ void map_node(const MapStatic &M, const MapScalars &S, int a,
                                         double X, double Y, double &xX, double &xY,
                                         double &yX, double &yY, double &Vx, double &Vy)
{
    switch (M.kind) {
    case MK_SINE: {
        const double *m = M.ms;
        const int N = M.N;
        xX = da(1.0, dm(m[2 * N + a], S.s));
        xY = dm(m[3 * N + a], S.s);
        yX = dm(m[4 * N + a], S.s);
        yY = da(1.0, dm(m[5 * N + a], S.s));
        Vx = dm(m[a], S.sd);
        Vy = dm(m[N + a], S.sd);
        break;
    }
    case MK_PLUNGE:
        xX = 1.0;
        xY = 0.0;
        yX = 0.0;
        yY = 1.0;
        Vx = 0.0;
        Vy = S.vy;
        break;
    case MK_PITCH:
    case MK_PITCH_PLUNGE: {
        double dx = ds(X, M.Xc), dy = ds(Y, M.Yc);
        xX = S.c;
        xY = -S.sn;
        yX = S.sn;
        yY = S.c;
        Vx = dm(S.thd, ds(dm(-S.sn, dx), dm(S.c, dy)));
        Vy = da(dm(S.thd, ds(dm(S.c, dx), dm(S.sn, dy))), S.vy);
        break;
    }
    case MK_BLENDED: {
        const int N = M.N;
        double dx = ds(X, M.Xc), dy = ds(Y, M.Yc);
        double b = M.ms[a], bX = M.ms[N + a], bY = M.ms[2 * N + a];
        double qx = ds(dm(S.cm, dx), dm(S.sn, dy));
        double qy = da(dm(S.sn, dx), dm(S.cm, dy));
        double one_bcm = da(1.0, dm(b, S.cm));
        xX = da(one_bcm, dm(qx, bX));
        xY = da(-dm(b, S.sn), dm(qx, bY));
        yX = da(dm(b, S.sn), dm(qy, bX));
        yY = da(one_bcm, dm(qy, bY));
        double bt = dm(b, S.thd);
        Vx = dm(bt, ds(dm(-S.sn, dx), dm(S.c, dy)));
        Vy = dm(bt, ds(dm(S.c, dx), dm(S.sn, dy)));
        break;
    }
    default:
        xX = 1.0;
        xY = 0.0;
        yX = 0.0;
        yY = 1.0;
        Vx = 0.0;
        Vy = 0.0;
    }
}

// Physical position G(X, t) (forces only; not on the bitwise path).
__device__ __forceinline__ void map_position(const MapStatic &M, const MapScalars &S, int a,
                                             double X, double Y, double &x, double &y)
{
    const int N = M.N;
    switch (M.kind) {
    case MK_SINE:
        x = X + M.ms[a] * S.s;
        y = Y + M.ms[N + a] * S.s;
        break;
    case MK_PLUNGE:
        x = X;
        y = Y + S.yoff;
        break;
    case MK_PITCH:
    case MK_PITCH_PLUNGE: {
        double dx = X - M.Xc, dy = Y - M.Yc;
        x = M.Xc + (dx * S.c - dy * S.sn);
        y = M.Yc + (dx * S.sn + dy * S.c) + S.yoff;
        break;
    }
    case MK_BLENDED: {
        double dx = X - M.Xc, dy = Y - M.Yc, b = M.ms[a];
        x = X + b * (S.cm * dx - S.sn * dy);
        y = Y + b * (S.sn * dx + S.cm * dy);
        break;
    }
    default:
        x = X;
        y = Y;
    }
}

// The map's metrics and V_G in FP32 (no FP64 operation): an approximation
// whose error the fast propagation path bounds and absorbs; never used to
// decide anything on its own.
struct MapScalarsF {
    float s, sd, vy, c, sn, thd, cm;
    float Xc, Yc;
    float Ux, Uy; // lattice shift (FP32-exact)
    float Us;     // |Ux| + |Uy|
    float er0;    // 2 + 2 Us: the offset's reach in the canonical point's rounding bound
};

ALELB_HD __forceinline__ void map_node_f32(const MapStatic &M, const MapScalarsF &S, int a,
                                             float4 Xf, float &xX, float &xY, float &yX,
                                             float &yY, float &Vx, float &Vy)
{
    const int N = M.N;
    switch (M.kind) {
    case MK_SINE:
        xX = 1.0f + M.msf[2 * N + a] * S.s;
        xY = M.msf[3 * N + a] * S.s;
        yX = M.msf[4 * N + a] * S.s;
        yY = 1.0f + M.msf[5 * N + a] * S.s;
        Vx = M.msf[a] * S.sd;
        Vy = M.msf[N + a] * S.sd;
        break;
    case MK_PLUNGE:
        xX = 1.0f;
        xY = 0.0f;
        yX = 0.0f;
        yY = 1.0f;
        Vx = 0.0f;
        Vy = S.vy;
        break;
    case MK_PITCH:
    case MK_PITCH_PLUNGE: {
        float dx = (Xf.x - S.Xc) + Xf.z, dy = (Xf.y - S.Yc) + Xf.w;
        xX = S.c;
        xY = -S.sn;
        yX = S.sn;
        yY = S.c;
        Vx = S.thd * (-S.sn * dx - S.c * dy);
        Vy = S.thd * (S.c * dx - S.sn * dy) + S.vy;
        break;
    }
    case MK_BLENDED: {
        float dx = (Xf.x - S.Xc) + Xf.z, dy = (Xf.y - S.Yc) + Xf.w;
        float b = M.msf[a], bX = M.msf[N + a], bY = M.msf[2 * N + a];
        float qx = S.cm * dx - S.sn * dy;
        float qy = S.sn * dx + S.cm * dy;
        xX = 1.0f + b * S.cm + qx * bX;
        xY = -b * S.sn + qx * bY;
        yX = b * S.sn + qy * bX;
        yY = 1.0f + b * S.cm + qy * bY;
        float bt = b * S.thd;
        Vx = bt * (-S.sn * dx - S.c * dy);
        Vy = bt * (S.c * dx - S.sn * dy);
        break;
    }
    default:
        xX = 1.0f;
        xY = 0.0f;
        yX = 0.0f;
        yY = 1.0f;
        Vx = 0.0f;
        Vy = 0.0f;
    }
}

// A = g^{-1,T} = (1/det g) [[y_Y, -x_Y], [-y_X, x_X]]; returns det g.
ALELB_HD __forceinline__ double metric_inverse_T(double xX, double xY, double yX, double yY,
                                                   double &a11, double &a12, double &a21,
                                                   double &a22)
{
    double det = ds(dm(xX, yY), dm(yX, xY));
    double inv = ddiv(1.0, det);
    a11 = dm(yY, inv);
    a12 = -dm(xY, inv);
    a21 = -dm(yX, inv);
    a22 = dm(xX, inv);
    return det;
}

// w = A V_G (or V_G itself for the printed form of Eq. 7).
ALELB_HD __forceinline__ void mesh_velocity_term(double a11, double a12, double a21, double a22,
                                                 double Vx, double Vy, bool literal, double &wx,
                                                 double &wy)
{
    if (literal) {
        wx = Vx;
        wy = Vy;
    } else {
        wx = da(dm(a11, Vx), dm(a12, Vy));
        wy = da(dm(a21, Vx), dm(a22, Vy));
    }
}

// c^_i = (A c_i) - w and the departure point X_dp = X - c^_i dt (dt = 1).
ALELB_HD __forceinline__ void departure(double a11, double a12, double a21, double a22,
                                        double wx, double wy, double cx, double cy, double X,
                                        double Y, double &chx, double &chy, double &px, double &py)
{
    chx = ds(da(dm(a11, cx), dm(a12, cy)), wx);
    chy = ds(da(dm(a21, cx), dm(a22, cy)), wy);
    px = ds(X, chx);
    py = ds(Y, chy);
}

// Departure point on the exact characteristic of a rigid map (no map,
// plunge, pitch, pitch with plunge; the characteristic of Sec. III with
// the motions of Sec. V): the arrival point x = G(X, t), the point
// x - c_i one time unit earlier, and its reference position
// G^-1(x - c_i, t - 1).  S1, S0: the map at t and at t - 1.  The rotation
// is applied about the centre, with no detour through absolute positions.
ALELB_HD __forceinline__ void exact_departure(const MapStatic &M, const MapScalars &S1,
                                              const MapScalars &S0, double cx, double cy,
                                              double X, double Y, double &chx, double &chy,
                                              double &px, double &py)
{
    cx = da(cx, S1.Ux); // the lattice velocity c_i + U
    cy = da(cy, S1.Uy);
    switch (M.kind) {
    case MK_PLUNGE:
        px = ds(X, cx);
        py = ds(ds(da(Y, S1.yoff), cy), S0.yoff);
        break;
    case MK_PITCH:
    case MK_PITCH_PLUNGE: {
        const double dx = ds(X, M.Xc), dy = ds(Y, M.Yc);
        // x - c_i - (centre at t - 1), relative to the reference centre
        const double rx = ds(ds(dm(dx, S1.c), dm(dy, S1.sn)), cx);
        const double ry = ds(da(da(dm(dx, S1.sn), dm(dy, S1.c)), ds(S1.yoff, S0.yoff)), cy);
        px = da(M.Xc, da(dm(rx, S0.c), dm(ry, S0.sn)));
        py = da(M.Yc, ds(dm(ry, S0.c), dm(rx, S0.sn)));
        break;
    }
    default:
        px = ds(X, cx);
        py = ds(Y, cy);
    }
    chx = ds(X, px);
    chy = ds(Y, py);
}

// ---------------------------------------------------------------------------
// Exact orientation sign of (a, b, c): sign of (a-c) x (b-c).
// Stage 1: the FP64 determinant with the certified error bound of Shewchuk
// (1997), errbound = (3 + 16 eps) eps (|l| + |r|), eps = 2^-53.
// Stage 2: exact integer evaluation (orient_int below) when the operands
// of each coordinate difference have nearby exponents.
// Stage 3 (otherwise): the determinant expanded into six products, each
// split exactly into two doubles with an FMA, and the twelve terms summed
// exactly as a non-overlapping expansion (Two-Sum / Grow-Expansion).
// ---------------------------------------------------------------------------
static ALELB_HD __noinline__ int orient_exact(double ax, double ay, double bx, double by, double cx,
                                         double cy)
{
    double pa[6] = {ax, -ax, -cx, -ay, ay, cy};
    double pb[6] = {by, cy, by, bx, cx, bx};
    double e[16];
    int m = 0;
    for (int k = 0; k < 12; ++k) {
        double hi = dm(pa[k >> 1], pb[k >> 1]);
        double q = (k & 1) ? dfma(pa[k >> 1], pb[k >> 1], -hi) : hi;
        int mm = 0;
        for (int j = 0; j < m; ++j) {
            double s = da(q, e[j]);
            double bv = ds(s, q);
            double av = ds(s, bv);
            double err = da(ds(q, av), ds(e[j], bv));
            if (err != 0.0) e[mm++] = err;
            q = s;
        }
        if (q != 0.0) e[mm++] = q;
        m = mm;
    }
    if (m == 0) return 0;
    return e[m - 1] > 0.0 ? 1 : -1;
}

// ---------------------------------------------------------------------------
// Stage 2 of the exact orientation, in integers: the exact sign from the
// binary representations.  A
// finite double is m 2^k with |m| < 2^53.  When the two operands of each
// difference have exponents at most 9 apart, the difference is D 2^K with
// |D| < 2^63 exactly; each product is then an exact 128-bit integer times a
// power of two, and the two products are compared exactly (a term whose
// leading bit lies above the other's after alignment decides alone).
// Returns 2 when the exponents are too far apart (stage 3 decides).  Only
// integer arithmetic: FP64 throughput on this GPU is a small fraction of
// its integer throughput.
// ---------------------------------------------------------------------------
ALELB_HD __forceinline__ void dsplit(double x, long long &m, int &k)
{
#ifdef __CUDA_ARCH__
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    std::memcpy(&b, &x, sizeof b);
#endif
    const int ex = (int)((b >> 52) & 0x7ffu);
    unsigned long long f = b & ((1ull << 52) - 1ull);
    if (ex) {
        f |= 1ull << 52;
        k = ex - 1075;
    } else {
        k = -1074;
    }
    m = (b >> 63) ? -(long long)f : (long long)f;
}

ALELB_HD __forceinline__ bool ddiff_int(double a, double c, long long &D, int &K)
{
    long long ma, mc;
    int ka, kc;
    dsplit(a, ma, ka);
    dsplit(c, mc, kc);
    if (ma == 0) {
        D = -mc;
        K = kc;
        return true;
    }
    if (mc == 0) {
        D = ma;
        K = ka;
        return true;
    }
    const int km = ka < kc ? ka : kc;
    if (ka - km > 9 || kc - km > 9) return false;
    D = ma * (1ll << (ka - km)) - mc * (1ll << (kc - km));
    K = km;
    return true;
}

ALELB_HD __forceinline__ int bitlen128(__int128 v)
{
    const unsigned __int128 u = v < 0 ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
#ifdef __CUDA_ARCH__
    return hi ? 128 - __clzll((long long)hi) : (lo ? 64 - __clzll((long long)lo) : 0);
#else
    return hi ? 128 - __builtin_clzll(hi) : (lo ? 64 - __builtin_clzll(lo) : 0);
#endif
}

static ALELB_HD __noinline__ int orient_int(double ax, double ay, double bx, double by, double cx,
                                            double cy)
{
    long long d1, d2, d3, d4;
    int k1, k2, k3, k4;
    if (!ddiff_int(ax, cx, d1, k1) || !ddiff_int(by, cy, d2, k2) || !ddiff_int(ay, cy, d3, k3) ||
        !ddiff_int(bx, cx, d4, k4))
        return 2;
    __int128 P = (__int128)d1 * d2, R = (__int128)d3 * d4; // det = P 2^KP - R 2^KR
    const int KP = k1 + k2, KR = k3 + k4;
    if (P == 0) return R > 0 ? -1 : (R < 0 ? 1 : 0);
    if (R == 0) return P > 0 ? 1 : -1;
    const int bp = bitlen128(P), br = bitlen128(R);
    if (KP >= KR) {
        const int sh = KP - KR;
        if (bp + sh - 1 >= br) return P > 0 ? 1 : -1;
        P *= (__int128)1 << sh;
    } else {
        const int sh = KR - KP;
        if (br + sh - 1 >= bp) return R > 0 ? -1 : 1;
        R *= (__int128)1 << sh;
    }
    return P > R ? 1 : (P < R ? -1 : 0);
}

ALELB_HD __forceinline__ int orient(double ax, double ay, double bx, double by, double cx,
                                    double cy)
{
    const double acx = ds(ax, cx), bcy = ds(by, cy), acy = ds(ay, cy), bcx = ds(bx, cx);
    double l = dm(acx, bcy);
    double r = dm(acy, bcx);
    double det = ds(l, r);
    double bound = 3.3306690738754716e-16 * (fabs(l) + fabs(r));
    if (det > bound) return 1;
    if (-det > bound) return -1;
    // fl(a - b) is zero only when a == b: a zero difference is exact, so
    // when each product has a zero factor the determinant is exactly 0
    if ((acx == 0.0 || bcy == 0.0) && (acy == 0.0 || bcx == 0.0)) return 0;
    const int si = orient_int(ax, ay, bx, by, cx, cy);
    if (si != 2) return si;
    return orient_exact(ax, ay, bx, by, cx, cy);
}

// ---------------------------------------------------------------------------
// Mesh topology for the walk
// ---------------------------------------------------------------------------
struct MeshDev {
    int N, E;
    double Lx, Ly;
    const double2 *X;      // [N] node coordinates
    const double2 *ev;     // [3E] vertex coordinates in each element's frame
    const int *nbr;        // [3E] neighbour across edge k (-1 on a boundary)
    const uint32_t *einfo; // [E] per edge k, byte k: kind(2) | nbr edge(2) | dsx+1(2) | dsy+1(2)
    const int *rank;       // [E] tie-break rank: larger area first, then lower original id
    const int *conn;       // [6E]
    const int *fan_ptr;    // [N+1]
    const int2 *fan;       // (elem, loc | (sx+1)<<4 | (sy+1)<<6)
    const int2 *owner;     // (elem, local index) of each node
    const int4 *ostn;      // [2N] owner element's six node numbers, then (elem, local index):
                           // {n0, n1, n2, n3}, {n4, n5, elem, local} (the derivative passes)
    const int *bcel;       // element of each node's wall-condition gradients
    const int *ring_ptr;   // [N + 1] neighbour ring of each node (learned proposal)
    const int *ring;       // ring elements, cache code of an unshifted element
    const float2 *nscale;  // (length scale, number of own elements) per node
    const uint8_t *bkind;  // [N] boundary kind of the node (0 interior)
    const uint8_t *vzero;  // [N] 1: mesh velocity exactly zero at all times
    const float4 *cone;    // [N] boundary node: outgoing, incoming boundary edge (domain on the left)
    const uint8_t *conek;  // [N] kind of those edges (0 when the node has no such pair), | 4 at a
                           // convex corner of the domain, | 8 at a reflex one
    const int *wall_idx;   // [N] index into the wall tables or -1
    const int *probe_e;    // [NW]
    const double2 *probe_xi; // [NW]
    const double2 *wall_nrm; // [NW] unit wall normal into the fluid, computational frame
    const int *orig_elem;  // [E] original element id
    const float4 *ejf;     // [2E] FP32 edge vectors (v1-v0, v2-v0) and inverse Jacobian rows
    const float *bdist;    // [N] lower bound of the node's distance to the nearest boundary edge
    const float4 *Xf;      // [N] node coordinates split hi + lo in FP32 (xh, yh, xl, yl)
    const float4 *v0f;     // [E] first frame vertex split hi + lo in FP32
    const float4 *evf;     // [3E] all frame vertices split hi + lo in FP32
    const int *nb_ptr;     // [N + 1] wall and far-field edges within NEAR_R of each node
    const float4 *nb;      // (P - X_a, Q - X_a) in FP32, the domain on the left of P -> Q
    const uint8_t *nbf;    // kind | 4 when the node lies on the edge
};

// Element cache code of a population: element (bits 0-24) | node's local
// index in it + 1 (bits 25-27; 7: not one of the node's elements; 0: not
// recorded) | (sx + 1) << 28 | (sy + 1) << 30 (frame shift), or -1.
constexpr int CACHE_ELEM = 0x01ffffff;
ALELB_HD __forceinline__ int cache_code(const MeshDev &M, int e, int sx, int sy, int a)
{
    int lb = 7;
    if (sx == 0 && sy == 0)
        for (int k = 0; k < 6; ++k)
            if (M.conn[6 * e + k] == a) lb = k + 1;
    return e | (lb << 25) | ((sx + 1) << 28) | ((sy + 1) << 30);
}

// Radius of the per-node lists of nearby boundary edges (lattice units).
// Every departure segment shorter than it lies in the disk that the list
// covers.
constexpr float NEAR_R = 2.5f;

struct Loc {
    int e;      // element (>= 0), or -1 missing, -2 the node itself
    int sx, sy; // frame shift of e (periods)
    int kind;   // boundary kind when missing
    int vnode;  // >= 0: the departure point coincides with this vertex node
};

ALELB_HD __forceinline__ void load_frame(const MeshDev &M, int e, int sx, int sy, double w[6])
{
    double ox = sx ? sx * M.Lx : 0.0, oy = sy ? sy * M.Ly : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double2 v = M.ev[3 * e + k];
        w[2 * k] = (sx ? da(v.x, ox) : v.x);
        w[2 * k + 1] = (sy ? da(v.y, oy) : v.y);
    }
}

// Best-ranked element of the fan of node v (the choice for a departure
// point that coincides with vertex v).
ALELB_HD __forceinline__ int fan_best(const MeshDev &M, int v)
{
    int best = -1;
    for (int k = M.fan_ptr[v]; k < M.fan_ptr[v + 1]; ++k) {
        int e = M.fan[k].x;
        if (best < 0 || M.rank[e] < M.rank[best]) best = e;
    }
    return best;
}

constexpr int WALK_LIMIT = 256;

// Orientation provider of the walk: exact FP64 predicates on the FP64
// departure point p and the element frames.
// Frame vertices of element e shifted by (sx, sy) periods, from the table
// itself (the predicate providers keep table pointers, never the address of
// a kernel parameter, so that they stay in registers).
ALELB_HD __forceinline__ void load_frame_t(const double2 *ev, double Lx, double Ly, int e, int sx,
                                           int sy, double w[6])
{
    double ox = sx ? sx * Lx : 0.0, oy = sy ? sy * Ly : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double2 v = ev[3 * e + k];
        w[2 * k] = (sx ? da(v.x, ox) : v.x);
        w[2 * k + 1] = (sy ? da(v.y, oy) : v.y);
    }
}

struct Pred64 {
    const double2 *ev;
    double Lx, Ly;
    double Xa, Ya, px, py;
    double w[6];
    ALELB_HD void load(int e, int sx, int sy) { load_frame_t(ev, Lx, Ly, e, sx, sy, w); }
    // orient(w_k1, w_k2, p) of the loaded element
    ALELB_HD int vvp(int k1, int k2)
    {
        return orient(w[2 * k1], w[2 * k1 + 1], w[2 * k2], w[2 * k2 + 1], px, py);
    }
    // orient(X_a, p, w_k) of the loaded element
    ALELB_HD int avp(int k) { return orient(Xa, Ya, px, py, w[2 * k], w[2 * k + 1]); }
    // p, known to lie on the line through w_l and w_k, lies on the ray from
    // w_l through w_k (the two terms of a dot product of collinear vectors
    // share one sign, so its sign is exact)
    ALELB_HD bool fwd(int l, int k)
    {
        return (px - w[2 * l]) * (w[2 * k] - w[2 * l]) + (py - w[2 * l + 1]) * (w[2 * k + 1] - w[2 * l + 1]) > 0.0;
    }
    ALELB_HD bool p_is_node() const { return px == Xa && py == Ya; }
};

// Straight-line walk from node a along the segment X_a -> p through the
// element adjacency (reading of Sec. III's departure-point search: the
// paper does not name a search).  A population is missing when the walk
// leaves the mesh through a boundary edge, or when no element of the node's
// fan holds the first piece of the segment.  A line through a vertex is
// treated as passing to the vertex's right.  Ties (p on an edge or vertex)
// go to the containing element of larger computational area, then lower
// original id.  P supplies the orientation signs, always exact.
// The location of a departure point in the closed element e (frame shift
// sx, sy), given its orientations against the three edges: strictly inside
// e; on one edge, then the element of lower rank (larger area, then lower
// original id) of the two that share it; on a vertex, which is then named.
ALELB_HD __forceinline__ Loc finish_loc(const MeshDev &M, int e, int sx, int sy, int o0, int o1, int o2)
{
    Loc r;
    r.kind = 0;
    r.vnode = -1;
    int nz = (o0 == 0) + (o1 == 0) + (o2 == 0);
    if (nz == 1) {
        int kz = o0 == 0 ? 0 : (o1 == 0 ? 1 : 2);
        uint32_t inf = (M.einfo[e] >> (8 * kz)) & 255u;
        if ((inf & 3) == 0) {
            int e2 = M.nbr[3 * e + kz];
            if (M.rank[e2] < M.rank[e]) {
                e = e2;
                sx += (int)((inf >> 4) & 3) - 1;
                sy += (int)((inf >> 6) & 3) - 1;
            }
        }
    } else if (nz >= 2) {
        // p is the vertex shared by the two zero edges
        int vl = (o0 == 0 && o1 == 0) ? 1 : ((o1 == 0 && o2 == 0) ? 2 : 0);
        r.vnode = M.conn[6 * e + vl];
    }
    r.e = e;
    r.sx = sx;
    r.sy = sy;
    return r;
}

template <class P> ALELB_HD __forceinline__ Loc walk_t(const MeshDev &M, P &pr, int a, int *err)
{
    Loc r;
    r.kind = 0;
    r.vnode = -1;
    r.sx = r.sy = 0;
    if (pr.p_is_node()) {
        // a nonzero but negligible c^ that rounds away: the departure point
        // is the node itself, held by every element of its fan
        r.e = fan_best(M, a);
        r.vnode = a;
        return r;
    }
    int beg = M.fan_ptr[a], end = M.fan_ptr[a + 1];
    int e = -1, loc = 0, sx = 0, sy = 0;
    for (int k = beg; k < end; ++k) {
        int2 fe = M.fan[k];
        int ll = fe.y & 15, ssx = ((fe.y >> 4) & 3) - 1, ssy = ((fe.y >> 6) & 3) - 1;
        pr.load(fe.x, ssx, ssy);
        bool hit;
        if (ll < 3) {
            int k1 = (ll + 1) % 3, k2 = (ll + 2) % 3;
            hit = pr.vvp(ll, k1) >= 0;
            if (hit) {
                // the sector ends before the ray ll -> k2, which the next fan
                // element holds; when edge (k2, ll) is a boundary edge no
                // element does, and a segment along it stays in the closed mesh
                const int s2 = pr.vvp(ll, k2);
                hit = s2 < 0 || (s2 == 0 && ((M.einfo[fe.x] >> (8 * k2)) & 3u) && pr.fwd(ll, k2));
            }
        } else {
            int k0 = ll - 3, k1 = (k0 + 1) % 3;
            hit = pr.vvp(k0, k1) >= 0;
        }
        if (hit) {
            e = fe.x;
            loc = ll;
            sx = ssx;
            sy = ssy;
            break;
        }
    }
    if (e < 0) {
        if (!M.bkind[a]) { // an interior node's sectors cover every direction
            set_err(err, ERR_LOCATE);
            r.e = -2;
            return r;
        }
        r.e = -1;
        r.kind = M.bkind[a];
        return r;
    }
    int o0, o1, o2; // orientation of p against edges 0, 1, 2 of e
    int kout;
    pr.load(e, sx, sy);
    o0 = pr.vvp(0, 1);
    o1 = pr.vvp(1, 2);
    o2 = pr.vvp(2, 0);
    bool found = o0 >= 0 && o1 >= 0 && o2 >= 0;
    if (!found) {
        if (loc < 3) {
            kout = (loc + 1) % 3;
        } else {
            int k0 = loc - 3, k2 = (k0 + 2) % 3;
            kout = pr.avp(k2) >= 0 ? (k0 + 1) % 3 : k2;
        }
        int step = 0;
        for (; step < WALK_LIMIT; ++step) {
            uint32_t inf = (M.einfo[e] >> (8 * kout)) & 255u;
            int kind = inf & 3;
            if (kind) {
                r.e = -1;
                r.kind = kind;
                return r;
            }
            int kin = (inf >> 2) & 3;
            sx += (int)((inf >> 4) & 3) - 1;
            sy += (int)((inf >> 6) & 3) - 1;
            e = M.nbr[3 * e + kout];
            pr.load(e, sx, sy);
            int k1 = (kin + 1) % 3, k2 = (kin + 2) % 3;
            int s1 = pr.vvp(k1, k2);
            int s2 = pr.vvp(k2, kin);
            if (s1 >= 0 && s2 >= 0) {
                // edge kin was crossed from outside: p lies strictly inside it
                o0 = kin == 0 ? 1 : (k1 == 0 ? s1 : s2);
                o1 = kin == 1 ? 1 : (k1 == 1 ? s1 : s2);
                o2 = kin == 2 ? 1 : (k1 == 2 ? s1 : s2);
                found = true;
                break;
            }
            kout = pr.avp(k2) >= 0 ? k1 : k2;
        }
        if (!found) {
            set_err(err, ERR_LOCATE);
            r.e = -2; // fall back to the node's own value
            return r;
        }
    }
    return finish_loc(M, e, sx, sy, o0, o1, o2);
}

static ALELB_HD __noinline__ Loc walk(const MeshDev M, int a, double Xa, double Ya, double px, double py,
                               int *err)
{
    Pred64 pr;
    pr.ev = M.ev;
    pr.Lx = M.Lx;
    pr.Ly = M.Ly;
    pr.Xa = Xa;
    pr.Ya = Ya;
    pr.px = px;
    pr.py = py;
    return walk_t(M, pr, a, err);
}

// Local coordinates (xi, eta) of p in element e (frame shift sx, sy).
ALELB_HD __forceinline__ void local_coords(const MeshDev &M, int e, int sx, int sy, double px,
                                             double py, double &xi, double &eta)
{
    double2 v0 = M.ev[3 * e], v1 = M.ev[3 * e + 1], v2 = M.ev[3 * e + 2];
    double x0 = v0.x + (sx ? sx * M.Lx : 0.0), y0 = v0.y + (sy ? sy * M.Ly : 0.0);
    double x_xi = v1.x - v0.x, x_eta = v2.x - v0.x;
    double y_xi = v1.y - v0.y, y_eta = v2.y - v0.y;
    double detJ = x_xi * y_eta - y_xi * x_eta;
    double dx = px - x0, dy = py - y0;
    xi = (y_eta * dx - x_eta * dy) / detJ;
    eta = (-y_xi * dx + x_xi * dy) / detJ;
}

// Element choices of the nine populations of node a (parity report):
// original element id, -2 (node itself) or -1 with kind.
ALELB_HD inline void locate_node(const MeshDev &M, const MapStatic &MS, const MapScalars &sc,
                                 int flags_literal, int a, int *elem9, int8_t *kind9, int *err)
{
    const double2 Xa = M.X[a];
    double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22, wx, wy;
    map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
    metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
    mesh_velocity_term(a11, a12, a21, a22, ds(Vx, sc.Ux), ds(Vy, sc.Uy), flags_literal != 0, wx, wy);
    for (int i = 0; i < NQ; ++i) {
        double chx, chy, px, py;
        departure(a11, a12, a21, a22, wx, wy, (double)lat_cx(i), (double)lat_cy(i), Xa.x, Xa.y, chx,
                  chy, px, py);
        int e = -2, k = 0;
        if (!(chx == 0.0 && chy == 0.0)) {
            Loc L = walk(M, a, Xa.x, Xa.y, px, py, err);
            if (L.e >= 0) {
                int ee = L.vnode >= 0 ? fan_best(M, L.vnode) : L.e;
                e = M.orig_elem[ee];
            } else if (L.e == -1) {
                e = -1;
                k = L.kind;
            }
        }
        elem9[i] = e;
        kind9[i] = (int8_t)k;
    }
}

// Certified FP32 test that p lies strictly inside element e (frame shift
// sx, sy).  Relative coordinates q = p - v0 are formed in FP64 and rounded
// once; the three orientations e1 x q, (e1 - q) x (e2 - q), e2 x q ... are
// evaluated in FP32 and accepted only when each clears the error bound
// 2^-17 M^2 (M the largest |coordinate| involved), which covers the input
// roundings and the FP32 operations.  A false return decides nothing: the
// caller then runs the exact walk.  On success q holds the FP32 offset
// from v0 for the interpolation weights.
ALELB_HD __forceinline__ bool strictly_inside_f32(const MeshDev &M, int e, int sx, int sy,
                                                  double px, double py, float &qx, float &qy)
{
    double2 v0 = M.ev[3 * e];
    double x0 = sx ? da(v0.x, sx * M.Lx) : v0.x;
    double y0 = sy ? da(v0.y, sy * M.Ly) : v0.y;
    qx = (float)ds(px, x0);
    qy = (float)ds(py, y0);
    float4 ed = M.ejf[2 * e];
    float e1x = ed.x, e1y = ed.y, e2x = ed.z, e2y = ed.w;
    float m = fmaxf(fmaxf(fmaxf(fabsf(e1x), fabsf(e1y)), fmaxf(fabsf(e2x), fabsf(e2y))),
                    fmaxf(fabsf(qx), fabsf(qy)));
    float bound = 7.62939453125e-06f * m * m; // 2^-17 M^2
    float o0 = e1x * qy - e1y * qx;                 // orient(v0, v1, p)
    float o1 = (e1x - qx) * (e2y - qy) - (e1y - qy) * (e2x - qx); // orient(v1, v2, p)
    float o2 = e2y * qx - e2x * qy;                 // orient(v2, v0, p)
    return o0 > bound && o1 > bound && o2 > bound;
}

// Certified FP32 sign of orient(A, B, C) = (A - C) x (B - C) from
// approximations of A, B, C with per-coordinate error bounds ea, eb, ec:
// +1 or -1 when certain, 0 when the exact predicate must decide.
ALELB_HD __forceinline__ int orient3_f32(float ax, float ay, float ea, float bx, float by, float eb,
                                         float cx, float cy, float ec)
{
    const float u = 5.9604644775390625e-08f;
    const float d1x = ax - cx, d1y = ay - cy, d2x = bx - cx, d2y = by - cy;
    const float D1 = fmaxf(fabsf(d1x), fabsf(d1y)), D2 = fmaxf(fabsf(d2x), fabsf(d2y));
    const float e1 = ea + ec + u * D1, e2 = eb + ec + u * D2;
    const float o = d1x * d2y - d1y * d2x;
    const float bound = 4.0f * (D1 * e2 + D2 * e1 + e1 * e2) + 8.0f * u * D1 * D2;
    if (o > bound) return 1;
    if (o < -bound) return -1;
    return 0;
}

// Error bound of a listed boundary-edge endpoint (relative to the node): the
// FP32 rounding of the FP64 difference, plus 2^-25 for that difference's own
// rounding.
ALELB_HD __forceinline__ float nb_err(float x, float y)
{
    return 5.9604644775390625e-08f * fmaxf(fabsf(x), fabsf(y)) + 2.98023223876953125e-08f;
}

// One pass over node a's nearby boundary edges for the segment from the
// node to its departure point a + (bx, by) (error eb per component; the
// caller ensures length + eb < NEAR_R, so the segment lies in the disk the
// list covers).  Up to 8 entries are loaded at once.
//   clear: certified to meet no listed edge, except at the node itself on
//     the edges through the node, from where it enters the domain: strictly
//     left of every such edge's line, or, at a reflex corner of the domain
//     (the union of the two left half-planes), of one of them (a straight
//     segment meets the line of an edge through its start only there).
//     Another edge is passed when both ends of the segment lie strictly on
//     one side of its line, or both ends of the edge strictly on one side
//     of the segment's line.
//   cross: the boundary kind when the segment certainly crosses a listed
//     edge not through the node (strictly opposite sides both ways: some of
//     its points lie outside the mesh, so the population is missing) and
//     every listed edge has that kind (the first boundary it meets is then
//     of that kind); 0 otherwise.
struct NbTest {
    bool clear;
    int cross;
};
ALELB_HD __forceinline__ NbTest nb_test(const MeshDev &M, int a, float bx, float by, float eb)
{
    constexpr int PRE = 8;
    const int beg = M.nb_ptr[a], end = M.nb_ptr[a + 1];
    int inc = 0, left = 0, kind = 0;
    bool mixed = false, crossed = false, clear = true;
    for (int base = beg; base < end; base += PRE) {
        float4 E[PRE];
        int fl[PRE];
#pragma unroll
        for (int j = 0; j < PRE; ++j) {
            E[j] = base + j < end ? M.nb[base + j] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            fl[j] = base + j < end ? (int)M.nbf[base + j] : 0;
        }
#pragma unroll
        for (int j = 0; j < PRE; ++j) {
            if (base + j >= end) break;
            const int f = fl[j];
            if (kind && (f & 3) != kind) mixed = true;
            kind = f & 3;
            const float eP = nb_err(E[j].x, E[j].y), eQ = nb_err(E[j].z, E[j].w);
            const int sB = orient3_f32(E[j].x, E[j].y, eP, E[j].z, E[j].w, eQ, bx, by, eb);
            if (f & 4) { // the node lies on this edge
                ++inc;
                left += sB > 0;
                continue;
            }
            const int sA = orient3_f32(E[j].x, E[j].y, eP, E[j].z, E[j].w, eQ, 0.0f, 0.0f, 0.0f);
            if (sA != 0 && sA == sB) continue; // the segment stays on one side of the line
            const int sP = orient3_f32(0.0f, 0.0f, 0.0f, bx, by, eb, E[j].x, E[j].y, eP);
            const int sQ = orient3_f32(0.0f, 0.0f, 0.0f, bx, by, eb, E[j].z, E[j].w, eQ);
            if (sP != 0 && sP == sQ) continue; // the edge stays on one side of the segment
            clear = false;
            if (sA * sB < 0 && sP * sQ < 0) crossed = true;
        }
    }
    NbTest r;
    r.clear = clear && (left == inc || (left > 0 && inc == 2 && (M.conek[a] & 8)));
    r.cross = crossed && !mixed ? kind : 0;
    return r;
}

// Bound of the FP32 transformed velocities c^_i against the FP64 canonical
// ones, from the FP32 metrics themselves (u = 2^-24):
//   entries of g:   eps_g   = 8u (1 + G) (blended map; 4u (1 + G) sine, 2u
//                   rigid pitch, 0 identity and plunge),  G = max |g_ij|
//   det g:          eps_det = 4 G eps_g + 3u (|x_X y_Y| + |y_X x_Y|)
//   A = g^{-1,T}:   eps_A   = (eps_g + G eps_det / det) / det + 2u max|A|
//   V_G:            eps_V   = 8u Vmag (Vmag: sum of the magnitudes entering V)
//   c^ = A c - A V: eps_c   = 2 [eps_A (2 + 2|V|) + 2 max|A| eps_V + 6u max|A| (2 + 2|V|)]
//   c^_0 = -A V:    eps_0   = 2 [eps_A 2|V| + 2 max|A| eps_V + 6u max|A| 2|V|]
//                   (c_0 = 0: the rest population's bound scales with the mesh
//                   velocity, which is small wherever the mesh barely moves)
// and er, the FP64 rounding of the canonical departure point X - c^ (at
// most 2^-53 (max|X| + 2) per component, taken twice).
struct FastMap {
    float A11, A12, A21, A22, W1, W2, eps_c, Vx, Vy, eps0, er;
    bool ok;
    // bound of c^_i, and of the departure offset -c^_i against the
    // canonical FP64 departure point relative to the node
    ALELB_HD float eps(int i) const { return i ? eps_c : eps0; }
    ALELB_HD float eq(int i) const { return (i ? eps_c : eps0) + er; }
};

ALELB_HD __forceinline__ FastMap fast_map(const MapStatic &MS, const MapScalarsF &sf, int a,
                                            float4 Xf)
{
    const float u = 5.9604644775390625e-08f;
    float xX, xY, yX, yY, Vx, Vy;
    map_node_f32(MS, sf, a, Xf, xX, xY, yX, yY, Vx, Vy);
    FastMap F;
    float det = xX * yY - yX * xY;
    float G = fmaxf(fmaxf(fabsf(xX), fabsf(xY)), fmaxf(fabsf(yX), fabsf(yY)));
    float inv = 1.0f / det;
    F.A11 = yY * inv;
    F.A12 = -xY * inv;
    F.A21 = -yX * inv;
    F.A22 = xX * inv;
    // the departure sees V_G - U (U the lattice shift, exact in FP32); the
    // wall condition keeps V_G
    const float Wx = Vx - sf.Ux, Wy = Vy - sf.Uy;
    F.W1 = F.A11 * Wx + F.A12 * Wy;
    F.W2 = F.A21 * Wx + F.A22 * Wy;
    F.Vx = Vx;
    F.Vy = Vy;
    float Amax = fmaxf(fmaxf(fabsf(F.A11), fabsf(F.A12)), fmaxf(fabsf(F.A21), fabsf(F.A22)));
    float Vmax = fmaxf(fabsf(Wx), fabsf(Wy));
    float Vmag = fabsf(Vx) + fabsf(Vy) + sf.Us; // (the subtraction's rounding: u |V - U|)
    if (MS.kind == MK_PITCH || MS.kind == MK_PITCH_PLUNGE || MS.kind == MK_BLENDED) {
        float dx = fabsf((Xf.x - sf.Xc) + Xf.z), dy = fabsf((Xf.y - sf.Yc) + Xf.w);
        Vmag += fabsf(sf.thd) * (dx + dy) + fabsf(sf.vy);
    }
    // error of the FP32 metric entries against the FP64 canonical ones, by
    // map kind: exact (identity, plunge), rounded cos/sin (rigid pitch),
    // a rounded product plus one (sine), a handful of terms (blended)
    float eps_g = 8.0f * u * (1.0f + G);
    if (MS.kind == MK_NONE || MS.kind == MK_PLUNGE) eps_g = 0.0f;
    else if (MS.kind == MK_PITCH || MS.kind == MK_PITCH_PLUNGE) eps_g = 2.0f * u;
    else if (MS.kind == MK_SINE) eps_g = 4.0f * u * (1.0f + G);
    float eps_det = 4.0f * G * eps_g + 3.0f * u * (fabsf(xX * yY) + fabsf(yX * xY));
    // (the bound's own roundings, a few u relative, vanish against its factor 2)
    float eps_A = (eps_g + G * eps_det * inv) * inv + 2.0f * u * Amax;
    float eps_V = 8.0f * u * Vmag;
    float cv = 2.0f + 2.0f * Vmax;
    F.eps_c = 2.0f * (eps_A * cv + 2.0f * Amax * eps_V + 6.0f * u * Amax * cv);
    const float cv0 = 2.0f * Vmax;
    F.eps0 = 2.0f * (eps_A * cv0 + 2.0f * Amax * eps_V + 6.0f * u * Amax * cv0);
    F.er = 2.3e-16f * (fmaxf(fabsf(Xf.x), fabsf(Xf.y)) + sf.er0);
    F.ok = det > 16.0f * eps_det && isfinite(F.eps_c);
    return F;
}

// fast_map for the translations (no map, plunge): the identity metric and
// V_G = (0, vy), with every term of the general bound that is fixed by them
// written as its value (det = G = Amax = 1, eps_g = 0, eps_det = 3u,
// eps_A = 5u, all exact); saves the general map's instructions in the
// propagation kernel, which is bound by instruction issue.
ALELB_HD __forceinline__ FastMap fast_map_translation(const MapScalarsF &sf, float4 Xf)
{
    const float u = 5.9604644775390625e-08f;
    FastMap F;
    F.A11 = 1.0f;
    F.A12 = -0.0f;
    F.A21 = -0.0f;
    F.A22 = 1.0f;
    const float Vy = sf.vy; // zero without a map
    const float Wx = 0.0f - sf.Ux, Wy = Vy - sf.Uy;
    F.W1 = Wx;
    F.W2 = Wy;
    F.Vx = 0.0f;
    F.Vy = Vy;
    const float Vmax = fmaxf(fabsf(Wx), fabsf(Wy));
    const float Vmag = fabsf(Vy) + sf.Us;
    const float eps_A = 5.0f * u;
    const float eps_V = 8.0f * u * Vmag;
    const float cv = 2.0f + 2.0f * Vmax;
    F.eps_c = 2.0f * (eps_A * cv + 2.0f * eps_V + 6.0f * u * cv);
    const float cv0 = 2.0f * Vmax;
    F.eps0 = 2.0f * (eps_A * cv0 + 2.0f * eps_V + 6.0f * u * cv0);
    F.er = 2.3e-16f * (fmaxf(fabsf(Xf.x), fabsf(Xf.y)) + sf.er0);
    F.ok = isfinite(F.eps_c); // det = 1 > 16 eps_det
    return F;
}

// The fast path's decision for population i of a node: true (element e,
// FP32 offset q from its first vertex) when the cached element c provably
// holds the FP64 departure point strictly inside and the departure segment
// cannot reach a boundary.
// The segment node -> departure point cannot leave the mesh when it is
// shorter than the node's distance to any boundary, or when the element is
// one of the node's own (a triangle is convex and holds both ends).  The
// departure point is strictly inside the element when its three
// barycentric coordinates (xi, eta, 1 - xi - eta) -- normalised
// orientations -- exceed their certified error margins:
//   |q - (p - v0)| <= eq per component, J the FP32-rounded inverse
//   Jacobian (relative error <= 2u), S_k = |J_k1| + |J_k2|:
//   |xi - xi_exact|  <= S_1 eq + 2u S_1 Q + 3u (|J_11 q_x| + |J_12 q_y|)
//   |eta - eta_exact| likewise, |lambda_0 error| <= both + 2u (1 + |xi| + |eta|)
// (each taken twice).  On success (xi, eta) are the interpolation's local
// coordinates.
ALELB_HD __forceinline__ bool fast_decide(const MeshDev &M, const FastMap &F, float4 Xf,
                                          float bdist, int a, int i, int c, int &e, float &xi,
                                          float &eta)
{
    const float u = 5.9604644775390625e-08f;
    const float cx = (float)lat_cx(i), cy = (float)lat_cy(i);
    const float chx = F.A11 * cx + F.A12 * cy - F.W1;
    const float chy = F.A21 * cx + F.A22 * cy - F.W2;
    // lengths compared squared (the margins have ample slack for the
    // rounding of the squares; bdist carries a 1e-6 relative reserve)
    const float len2 = chx * chx + chy * chy;
    const float q4 = 4.0f * F.eq(i);
    if (!(c >= 0 && (c >> 28) == 5 && len2 > q4 * q4)) return false;
    e = c & CACHE_ELEM;
    const int lb = (c >> 25) & 7; // node's local index + 1, 7 not own, 0 unknown
    int l = lb == 7 ? -1 : lb - 1;
    if (lb == 0) {
        const int *cn = M.conn + 6 * e;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (cn[k] == a) l = k;
    }
    // near a boundary the exact path decides (with the segment certificate
    // against the node's nearby boundary edges)
    const float room = bdist - F.eq(i);
    if (l < 0 && !(room > 0.0f && len2 < room * room)) return false;
    const float4 J = M.ejf[2 * e + 1];
    if (l >= 0) {
        // the node is node l of element e: its local coordinates are exact
        // (0, 1/2 or 1), so only the small offset -c^ is taken through the
        // FP32 inverse Jacobian; errors: F.eq(i) on c^ (eps of the direction plus the
        // FP64 rounding of the canonical departure point), u/2 on each J
        // entry, the products, the sums and the additions to the node's
        // coordinates
        // local coordinates of node l, twice over, as 2-bit fields of one
        // word ({0, 2, 0, 1, 1, 0} and {0, 0, 2, 0, 1, 1}): a run-time index
        // into a constant array would put the array in local memory
        const float xl = 0.5f * (float)((0x148u >> (2 * l)) & 3u);
        const float el = 0.5f * (float)((0x520u >> (2 * l)) & 3u);
        const float rx = -chx, ry = -chy;
        const float t11 = J.x * rx, t12 = J.y * ry, t21 = J.z * rx, t22 = J.w * ry;
        const float T1 = t11 + t12, T2 = t21 + t22;
        xi = xl + T1;
        eta = el + T2;
        // the third coordinate from its exact value at the node minus the
        // offsets (1 - xi - eta would cancel at nodes where it is zero)
        const float l0 = (1.0f - xl - el) - (T1 + T2);
        const float eq = F.eq(i);
        const float S1 = fabsf(J.x) + fabsf(J.y), S2 = fabsf(J.z) + fabsf(J.w);
        const float d1 = 2.0f * (S1 * eq + 3.0f * u * (fabsf(t11) + fabsf(t12)));
        const float d2 = 2.0f * (S2 * eq + 3.0f * u * (fabsf(t21) + fabsf(t22)));
        const float m1 = d1 + 2.0f * u * fabsf(xi);
        const float m2 = d2 + 2.0f * u * fabsf(eta);
        const float m0 = d1 + d2 + 2.0f * u * (fabsf(T1) + fabsf(T2) + fabsf(l0));
        return xi > m1 && eta > m2 && l0 > m0;
    }
    const float4 ed = M.ejf[2 * e];
    // node position relative to v0 (the node is not one of e's: l < 0 here)
    const float4 v0 = M.v0f[e];
    const float dx = (Xf.x - v0.x) + (Xf.z - v0.z);
    const float dy = (Xf.y - v0.y) + (Xf.w - v0.w);
    const float qx = dx - chx, qy = dy - chy;
    const float E = fmaxf(fmaxf(fabsf(ed.x), fabsf(ed.y)), fmaxf(fabsf(ed.z), fabsf(ed.w)));
    const float Q = fmaxf(fabsf(qx), fabsf(qy));
    const float eq = F.eq(i) + 2.0f * u * fmaxf(fmaxf(fabsf(dx), fabsf(dy)), E) + u * Q;
    const float t11 = J.x * qx, t12 = J.y * qy, t21 = J.z * qx, t22 = J.w * qy;
    xi = t11 + t12;
    eta = t21 + t22;
    const float l0 = 1.0f - xi - eta;
    const float S1 = fabsf(J.x) + fabsf(J.y), S2 = fabsf(J.z) + fabsf(J.w);
    const float m1 = 2.0f * (S1 * (eq + 2.0f * u * Q) + 3.0f * u * (fabsf(t11) + fabsf(t12)));
    const float m2 = 2.0f * (S2 * (eq + 2.0f * u * Q) + 3.0f * u * (fabsf(t21) + fabsf(t22)));
    const float m0 = m1 + m2 + 4.0f * u * (1.0f + fabsf(xi) + fabsf(eta));
    return xi > m1 && eta > m2 && l0 > m0;
}

// Certified FP32 test that population i of boundary node a is missing
// because its departure direction -c^ points strictly into the exterior at
// the node: strictly to the right of both boundary edges through the node
// (the domain lies on their left), or, at a convex corner of the domain,
// strictly to the right of either.  The points of the segment next to the
// node then lie outside the closed mesh.  Returns the boundary kind, or 0
// when not certain.  Errors: F.eq(i) per component of -c^, the FP32
// rounding of the edge vectors and of the cross products.
ALELB_HD __forceinline__ int cone_missing(const MeshDev &M, const FastMap &F, int a, int i)
{
    const int ck = M.conek[a];
    if (!ck) return 0;
    const int k = ck & 3;
    const float u = 5.9604644775390625e-08f;
    const float cx = (float)lat_cx(i), cy = (float)lat_cy(i);
    const float dx = -(F.A11 * cx + F.A12 * cy - F.W1);
    const float dy = -(F.A21 * cx + F.A22 * cy - F.W2);
    if (!(sqrtf(dx * dx + dy * dy) > 4.0f * F.eq(i))) return 0;
    const float4 c = M.cone[a];
    const float eq = F.eq(i);
    const float s1 = c.x * dy - c.y * dx, s2 = c.z * dy - c.w * dx;
    const float b1 = 2.0f * (3.0f * u * (fabsf(c.x * dy) + fabsf(c.y * dx)) + (fabsf(c.x) + fabsf(c.y)) * eq);
    const float b2 = 2.0f * (3.0f * u * (fabsf(c.z * dy) + fabsf(c.w * dx)) + (fabsf(c.z) + fabsf(c.w)) * eq);
    if (ck & 4) return (s1 < -b1 || s2 < -b2) ? k : 0; // convex corner: either edge
    return (s1 < -b1 && s2 < -b2) ? k : 0;
}

// A population certified missing without the walk: the exterior cone at a
// boundary node, else a certified crossing of one of the node's nearby
// boundary edges.  Returns the boundary kind, or 0 when not certain; clear
// (when given) receives the segment test of the same pass over the nearby
// edges (1 clear, 0 not, -1 not evaluated).
ALELB_HD __forceinline__ int certified_missing(const MeshDev &M, const FastMap &F, int a, int i,
                                               int *clear = nullptr)
{
    if (clear) *clear = -1;
    const int ck = cone_missing(M, F, a, i);
    if (ck || M.nb_ptr[a] == M.nb_ptr[a + 1]) return ck;
    const float cx = (float)lat_cx(i), cy = (float)lat_cy(i);
    const float chx = F.A11 * cx + F.A12 * cy - F.W1;
    const float chy = F.A21 * cx + F.A22 * cy - F.W2;
    const float len = sqrtf(chx * chx + chy * chy);
    const float eb = F.eq(i);
    if (!(len > 4.0f * F.eq(i)) || !(len + eb < NEAR_R)) return 0;
    const NbTest t = nb_test(M, a, -chx, -chy, eb);
    if (clear) *clear = t.clear ? 1 : 0;
    return t.cross;
}


// Orientation provider of the walk in FP32: every point relative to the
// node, the departure point from the FP32 c^ (bound F.eq(i)), element
// vertices from their hi/lo splits.  Uncertain signs fall back to the exact
// FP64 predicate on the FP64 canonical departure point, computed lazily.
struct Pred32 {
    const float4 *evf;
    const double2 *ev;
    double Lx, Ly;
    MapStatic MS;
    MapScalars sc;
    int a, i, literal;
    float4 Xf;
    float rpx, rpy, ep;
    int e, sx, sy;
    // the element's vertices relative to the node and their error bounds
    // (scalars with selectors rather than arrays: run-time indices would
    // put arrays in local memory)
    float rx0, rx1, rx2, ry0, ry1, ry2, er0, er1, er2;
    bool have64, wload;
    double Xa, Ya, px, py;
    double w0, w1, w2, w3, w4, w5;

    ALELB_HD float RX(int k) const { return k == 0 ? rx0 : (k == 1 ? rx1 : rx2); }
    ALELB_HD float RY(int k) const { return k == 0 ? ry0 : (k == 1 ? ry1 : ry2); }
    ALELB_HD float ER(int k) const { return k == 0 ? er0 : (k == 1 ? er1 : er2); }
    ALELB_HD double WX(int k) const { return k == 0 ? w0 : (k == 1 ? w2 : w4); }
    ALELB_HD double WY(int k) const { return k == 0 ? w1 : (k == 1 ? w3 : w5); }

    ALELB_HD void load(int e_, int sx_, int sy_)
    {
        const float u = 5.9604644775390625e-08f;
        e = e_;
        sx = sx_;
        sy = sy_;
        wload = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 v = evf[3 * e + k];
            const float hx = v.x - Xf.x, hy = v.y - Xf.y;
            float x = hx + (v.z - Xf.z), y = hy + (v.w - Xf.w);
            float sh = 0.0f;
            if (sx) {
                x += (float)sx * (float)Lx;
                sh = fabsf((float)Lx);
            }
            if (sy) {
                y += (float)sy * (float)Ly;
                sh = fmaxf(sh, fabsf((float)Ly));
            }
            const float ek = 4.0f * u * (fmaxf(fabsf(x), fabsf(y)) + fmaxf(fabsf(hx), fabsf(hy)) + sh) +
                             9.313225746154785e-10f;
            if (k == 0) {
                rx0 = x;
                ry0 = y;
                er0 = ek;
            } else if (k == 1) {
                rx1 = x;
                ry1 = y;
                er1 = ek;
            } else {
                rx2 = x;
                ry2 = y;
                er2 = ek;
            }
        }
    }
    ALELB_HD void ensure64()
    {
        if (!have64) {
            double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22, wx, wy, chx, chy;
            map_node(MS, sc, a, Xa, Ya, xX, xY, yX, yY, Vx, Vy);
            metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
            mesh_velocity_term(a11, a12, a21, a22, ds(Vx, sc.Ux), ds(Vy, sc.Uy), literal != 0, wx, wy);
            departure(a11, a12, a21, a22, wx, wy, lat_cx(i), lat_cy(i), Xa, Ya, chx, chy, px, py);
            have64 = true;
        }
        if (!wload) {
            double w[6];
            load_frame_t(ev, Lx, Ly, e, sx, sy, w);
            w0 = w[0];
            w1 = w[1];
            w2 = w[2];
            w3 = w[3];
            w4 = w[4];
            w5 = w[5];
            wload = true;
        }
    }
    ALELB_HD int vvp(int k1, int k2)
    {
        const int s = orient3_f32(RX(k1), RY(k1), ER(k1), RX(k2), RY(k2), ER(k2), rpx, rpy, ep);
        if (s) return s;
        ensure64();
        return orient(WX(k1), WY(k1), WX(k2), WY(k2), px, py);
    }
    ALELB_HD int avp(int k)
    {
        const int s = orient3_f32(0.0f, 0.0f, 0.0f, rpx, rpy, ep, RX(k), RY(k), ER(k));
        if (s) return s;
        ensure64();
        return orient(Xa, Ya, px, py, WX(k), WY(k));
    }
    // as Pred64::fwd, on the FP64 departure point (asked only after an
    // exactly zero sign, which came from the FP64 stage)
    ALELB_HD bool fwd(int l, int k)
    {
        ensure64();
        return (px - WX(l)) * (WX(k) - WX(l)) + (py - WY(l)) * (WY(k) - WY(l)) > 0.0;
    }
    // the caller ensures |c^| > 4 F.eq(i): then the FP64 departure point is
    // not the node
    ALELB_HD bool p_is_node() const { return false; }
};

// The exact element decision of population i of node a in the
// FP32-deviation form, when the verified previous-step element did not
// settle it: the walk on certified FP32 predicates (exact fallback) when
// the FP32 map is usable and c^ is clearly nonzero, else on FP64 ones.
// Returns the walk's Loc; for an interior element, q = p - v0 in FP32.
// src >= 0: the population takes node src's value as is.
// hint: the population's element cache entry.  When it names an unshifted
// element and the segment provably stays in the mesh (the element is one
// of the node's own, or the segment is shorter than the boundary distance,
// or it passes the nearby boundary edges), the three exact orientations
// against that element decide: a departure point in the closed element is
// located there by the walk too, with the same rule for edges and vertices
// (a departure point near an element edge, where the FP32 margins fail, no
// longer needs the scan of the node's fan).
// s1 (not null): the departure point on the exact characteristic, s1 the
// map at the arrival time and sc at the departure time (F is then not ok).
ALELB_HD __forceinline__ Loc slow_decide(const MeshDev &M, const MapStatic &MS,
                                         const MapScalars &sc, const FastMap &F, float4 Xf, int a,
                                         int i, int literal, float &qx, float &qy, int &src,
                                         int *err, int hint = -1, int clear = -1,
                                         const MapScalars *s1 = nullptr, bool *hint_taken = nullptr)
{
    const double2 Xa = M.X[a];
    src = -1;
    Loc L;
    bool done = false;
    if (F.ok && !literal) {
        const float cx = (float)lat_cx(i), cy = (float)lat_cy(i);
        const float chx = F.A11 * cx + F.A12 * cy - F.W1;
        const float chy = F.A21 * cx + F.A22 * cy - F.W2;
        if (sqrtf(chx * chx + chy * chy) > 4.0f * F.eq(i)) {
            Pred32 pr;
            pr.evf = M.evf;
            pr.ev = M.ev;
            pr.Lx = M.Lx;
            pr.Ly = M.Ly;
            pr.MS = MS;
            pr.sc = sc;
            pr.a = a;
            pr.i = i;
            pr.literal = literal;
            pr.Xf = Xf;
            pr.rpx = -chx;
            pr.rpy = -chy;
            pr.ep = F.eq(i);
            pr.have64 = false;
            pr.wload = false;
            pr.Xa = Xa.x;
            pr.Ya = Xa.y;
            bool have = false;
            if (hint >= 0 && (hint >> 28) == 5) {
                const int ce = hint & CACHE_ELEM;
                const int lb = (hint >> 25) & 7;
                bool own = lb != 0 && lb != 7;
                if (lb == 0)
#pragma unroll
                    for (int k = 0; k < 6; ++k) own |= M.conn[6 * ce + k] == a;
                const float len = sqrtf(chx * chx + chy * chy);
                const float eb = F.eq(i);
                if (own || len + eb < M.bdist[a] ||
                    (clear >= 0 ? clear == 1 : (len + eb < NEAR_R && nb_test(M, a, -chx, -chy, eb).clear))) {
                    pr.load(ce, 0, 0);
                    const int o0 = pr.vvp(0, 1);
                    if (o0 >= 0) {
                        const int o1 = pr.vvp(1, 2);
                        if (o1 >= 0) {
                            const int o2 = pr.vvp(2, 0);
                            if (o2 >= 0) {
                                L = finish_loc(M, ce, 0, 0, o0, o1, o2);
                                have = true;
                                if (hint_taken) *hint_taken = true;
                            }
                        }
                    }
                }
            }
            if (!have) L = walk_t(M, pr, a, err);
            if (L.e >= 0 && L.vnode < 0) {
                const float4 v = M.evf[3 * L.e];
                float x0 = (v.x - Xf.x) + (v.z - Xf.z), y0 = (v.y - Xf.y) + (v.w - Xf.w);
                if (L.sx) x0 += (float)L.sx * (float)M.Lx;
                if (L.sy) y0 += (float)L.sy * (float)M.Ly;
                qx = -chx - x0;
                qy = -chy - y0;
            }
            done = true;
        }
    }
    if (!done) {
        double chx, chy, px, py;
        if (s1) { // the exact characteristic: s1 the arrival map, sc the departure map
            exact_departure(MS, *s1, sc, lat_cx(i), lat_cy(i), Xa.x, Xa.y, chx, chy, px, py);
        } else {
            double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22, wx, wy;
            map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
            metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
            mesh_velocity_term(a11, a12, a21, a22, ds(Vx, sc.Ux), ds(Vy, sc.Uy), literal != 0, wx, wy);
            departure(a11, a12, a21, a22, wx, wy, lat_cx(i), lat_cy(i), Xa.x, Xa.y, chx, chy, px, py);
        }
        if (chx == 0.0 && chy == 0.0) {
            L.e = -2;
            L.vnode = -1;
            L.kind = 0;
            L.sx = L.sy = 0;
            src = a;
            return L;
        }
        L = walk(M, a, Xa.x, Xa.y, px, py, err);
        if (L.e >= 0 && L.vnode < 0) {
            const double2 v0 = M.ev[3 * L.e];
            qx = (float)(px - (L.sx ? v0.x + L.sx * M.Lx : v0.x));
            qy = (float)(py - (L.sy ? v0.y + L.sy * M.Ly : v0.y));
        }
    }
    if (L.e == -2) src = a;
    else if (L.e >= 0 && L.vnode >= 0) src = L.vnode;
    return L;
}

// Element decisions of the FP32-deviation propagation for the nine
// populations of node a, given the element cache (parity report and host
// emulation): the fast decision where it applies, slow_decide elsewhere.
ALELB_HD inline void mixed_locate_node(const MeshDev &M, const MapStatic &MS,
                                       const MapScalars &sc, const MapScalarsF &sf,
                                       const int *cache, int a, int *elem9, int8_t *kind9,
                                       int8_t *fast9, int *err)
{
    const float4 Xf = M.Xf[a];
    const FastMap F = fast_map(MS, sf, a, Xf);
    for (int i = 0; i < NQ; ++i) {
        int e;
        float qx, qy;
        if (i == 0 && M.vzero[a] && sf.Ux == 0.0f && sf.Uy == 0.0f) { // c^_0 exactly zero: the node's own value
            if (fast9) fast9[i] = 1;
            elem9[i] = -2;
            kind9[i] = 0;
            continue;
        }
        const bool f = F.ok && fast_decide(M, F, Xf, M.bdist[a], a, i, cache[(size_t)i * M.N + a], e, qx, qy);
        if (fast9) fast9[i] = f ? 1 : 0;
        if (f) {
            elem9[i] = M.orig_elem[e];
            kind9[i] = 0;
            continue;
        }
        const int ck = F.ok ? cone_missing(M, F, a, i) : 0;
        if (ck) { // certified missing at the node itself
            if (fast9) fast9[i] = 1;
            elem9[i] = -1;
            kind9[i] = (int8_t)ck;
            continue;
        }
        // the exact path: a certified crossing of a nearby boundary edge,
        // else the decision of slow_decide
        const int cx = F.ok ? certified_missing(M, F, a, i) : 0;
        if (cx) {
            elem9[i] = -1;
            kind9[i] = (int8_t)cx;
            continue;
        }
        int src;
        const Loc L = slow_decide(M, MS, sc, F, Xf, a, i, 0, qx, qy, src, err, cache[(size_t)i * M.N + a]);
        if (L.e == -2 && src == a && L.vnode < 0) {
            elem9[i] = -2;
            kind9[i] = 0;
        } else if (L.e >= 0) {
            elem9[i] = M.orig_elem[L.vnode >= 0 ? fan_best(M, L.vnode) : L.e];
            kind9[i] = 0;
        } else {
            elem9[i] = -1;
            kind9[i] = (int8_t)L.kind;
        }
    }
}

} // namespace alelb
