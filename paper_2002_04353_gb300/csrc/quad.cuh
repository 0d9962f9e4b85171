// quad.cuh -- the paper's 9-node quadrilateral element (Sec. III): the
// bilinear geometry of Eq. NonLinear_Eq, the local coordinates of a
// departure point by Newton's method, the nine second-order Lagrange shape
// functions of Eq. Propagation (s = 1..9), the straight-line element walk
// over quadrilaterals and the element gradients (the kernels of a time step
// on such a mesh are in quad.cu).
//
// Node order of an element: corners v0 (-1,-1), v1 (1,-1), v2 (1,1),
// v3 (-1,1) counter-clockwise, the midside nodes of edges (v0,v1), (v1,v2),
// (v2,v3), (v3,v0), then the centre (0,0).  Edge k runs from v_k to v_k+1.
//
// The exact path: the FP64 departure point, exact orientation signs for the
// walk and the tie rules, Newton in the interpolation's arithmetic; the
// populations are stored and interpolated in the solver's precision.  The
// deviation forms settle most populations before it with a certified FP32
// test of the previous-step element (quad_fast_decide).
#pragma once
#include "geom.cuh"

namespace alelb {

// Index (0, 1, 2 for -1, 0, 1) of local node l's xi and eta.
ALELB_HD __forceinline__ int quad_ix(int l) { return (int)((0x11928u >> (2 * l)) & 3u); }
ALELB_HD __forceinline__ int quad_iy(int l) { return (int)((0x164a0u >> (2 * l)) & 3u); }

// Bilinear map of the corners w (x, y pairs) at (xi, eta), Eq. NonLinear_Eq:
// x = sum_k n_k w_k with n = (1 -+ xi)(1 -+ eta)/4, and its Jacobian
// J = {x_xi, x_eta, y_xi, y_eta}.
ALELB_HD __forceinline__ void quad_bilinear(const double w[8], double xi, double eta, double &x, double &y,
                                            double J[4])
{
    const double n0 = 0.25 * (1.0 - xi) * (1.0 - eta), n1 = 0.25 * (1.0 + xi) * (1.0 - eta);
    const double n2 = 0.25 * (1.0 + xi) * (1.0 + eta), n3 = 0.25 * (1.0 - xi) * (1.0 + eta);
    const double a0 = -0.25 * (1.0 - eta), a1 = 0.25 * (1.0 - eta), a2 = 0.25 * (1.0 + eta), a3 = -0.25 * (1.0 + eta);
    const double b0 = -0.25 * (1.0 - xi), b1 = -0.25 * (1.0 + xi), b2 = 0.25 * (1.0 + xi), b3 = 0.25 * (1.0 - xi);
    x = n0 * w[0] + n1 * w[2] + n2 * w[4] + n3 * w[6];
    y = n0 * w[1] + n1 * w[3] + n2 * w[5] + n3 * w[7];
    J[0] = a0 * w[0] + a1 * w[2] + a2 * w[4] + a3 * w[6];
    J[1] = b0 * w[0] + b1 * w[2] + b2 * w[4] + b3 * w[6];
    J[2] = a0 * w[1] + a1 * w[3] + a2 * w[5] + a3 * w[7];
    J[3] = b0 * w[1] + b1 * w[3] + b2 * w[5] + b3 * w[7];
}

// Newton's method on Eq. NonLinear_Eq for corners c taken relative to the
// point (so the root is x(xi, eta) = 0), in the arithmetic A of the values
// it serves: start at the centre, at most QUAD_NEWTON_ITERS steps, stopping
// once a step is below `done` (quadratic convergence: the next one would be
// below the rounding); converged when the last step is below `tol`.  The
// element choice never depends on it (exact signs decide), only the
// interpolation weights.
constexpr int QUAD_NEWTON_ITERS = 8;
template <class A>
ALELB_HD __forceinline__ bool quad_newton_t(const A c[8], A done, A tol, A &xi, A &eta)
{
    A a = A(0), b = A(0), da = A(0), db = A(0);
#pragma unroll 1
    for (int it = 0; it < QUAD_NEWTON_ITERS; ++it) {
        const A n0 = A(0.25) * (A(1) - a) * (A(1) - b), n1 = A(0.25) * (A(1) + a) * (A(1) - b);
        const A n2 = A(0.25) * (A(1) + a) * (A(1) + b), n3 = A(0.25) * (A(1) - a) * (A(1) + b);
        const A a0 = A(-0.25) * (A(1) - b), a1 = A(0.25) * (A(1) - b), a2 = A(0.25) * (A(1) + b), a3 = -a2;
        const A b0 = A(-0.25) * (A(1) - a), b1 = A(-0.25) * (A(1) + a), b2 = -b1, b3 = -b0;
        const A rx = n0 * c[0] + n1 * c[2] + n2 * c[4] + n3 * c[6];
        const A ry = n0 * c[1] + n1 * c[3] + n2 * c[5] + n3 * c[7];
        const A J0 = a0 * c[0] + a1 * c[2] + a2 * c[4] + a3 * c[6];
        const A J1 = b0 * c[0] + b1 * c[2] + b2 * c[4] + b3 * c[6];
        const A J2 = a0 * c[1] + a1 * c[3] + a2 * c[5] + a3 * c[7];
        const A J3 = b0 * c[1] + b1 * c[3] + b2 * c[5] + b3 * c[7];
        const A inv = A(1) / (J0 * J3 - J1 * J2);
        da = (J3 * rx - J1 * ry) * inv;
        db = (-J2 * rx + J0 * ry) * inv;
        a -= da;
        b -= db;
        if (fabs(da) + fabs(db) < done) break;
    }
    xi = a;
    eta = b;
    return fabs(da) <= tol && fabs(db) <= tol;
}
ALELB_HD __forceinline__ bool quad_newton(const double c[8], double &xi, double &eta)
{
    return quad_newton_t<double>(c, 1e-12, 1e-9, xi, eta);
}

// One-dimensional quadratic Lagrange polynomials through -1, 0, 1 and
// their derivatives.
template <class A> ALELB_HD __forceinline__ void lagrange3(A s, A L[3], A dL[3])
{
    L[0] = A(0.5) * s * (s - A(1));
    L[1] = (A(1) - s) * (A(1) + s);
    L[2] = A(0.5) * s * (s + A(1));
    dL[0] = s - A(0.5);
    dL[1] = A(-2) * s;
    dL[2] = s + A(0.5);
}

// N_s(xi, eta) = L_i(xi) L_j(eta) for the nine nodes (Eq. Propagation).
template <class A> ALELB_HD __forceinline__ void shape9(A xi, A eta, A N[9])
{
    A Lx[3], Ly[3], dx[3], dy[3];
    lagrange3(xi, Lx, dx);
    lagrange3(eta, Ly, dy);
#pragma unroll
    for (int s = 0; s < 9; ++s) N[s] = Lx[quad_ix(s)] * Ly[quad_iy(s)];
}

struct QuadDev {
    int N, E;
    double Lx, Ly;
    const double2 *X;      // [N]
    const double2 *ev;     // [4E] corners in each element's frame
    const int *nbr;        // [4E]
    const uint32_t *einfo; // [E] byte k: kind(2) | nbr edge(2) | dsx+1(2) | dsy+1(2)
    const int *rank;       // [E]
    const int *conn;       // [9E]
    const int *fan_ptr;    // [N + 1]
    const int2 *fan;       // (elem, local | (sx+1)<<4 | (sy+1)<<6)
    const int2 *owner;     // (elem, local)
    const int2 *bcel;      // (elem, local): wall-condition gradient element
    const uint8_t *bkind;  // [N]
    const int *wall_idx;   // [N]
    const int *probe_e;    // [NW]
    const double2 *probe_xi; // [NW]
    const double2 *wall_nrm; // [NW]
    const int *orig_elem;  // [E]
    const float4 *Xf;      // [N] node coordinates, FP32 hi + lo
    const float4 *evf;     // [4E] corners, FP32 hi + lo
    const float *bdist;    // [N] lower bound of the distance to the nearest boundary edge
    const float4 *ownJf;   // [N] owner element's J^{-1} at the node, FP32
};

// The four corners of element e shifted by (sx, sy) periods.
ALELB_HD __forceinline__ void quad_frame(const QuadDev &M, int e, int sx, int sy, double w[8])
{
    const double ox = sx ? sx * M.Lx : 0.0, oy = sy ? sy * M.Ly : 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double2 v = M.ev[4 * e + k];
        w[2 * k] = sx ? v.x + ox : v.x;
        w[2 * k + 1] = sy ? v.y + oy : v.y;
    }
}

ALELB_HD __forceinline__ int quad_fan_best(const QuadDev &M, int v)
{
    int best = -1;
    for (int k = M.fan_ptr[v]; k < M.fan_ptr[v + 1]; ++k) {
        const int e = M.fan[k].x;
        if (best < 0 || M.rank[e] < M.rank[best]) best = e;
    }
    return best;
}

// Location of p in the closed element e, given its signs against the four
// edges: strictly inside; on one edge, then the better-ranked of the two
// elements sharing it (larger area, then lower original id); on a corner,
// which is named.
ALELB_HD __forceinline__ Loc quad_finish(const QuadDev &M, int e, int sx, int sy, const int o[4])
{
    Loc r;
    r.kind = 0;
    r.vnode = -1;
    const int nz = (o[0] == 0) + (o[1] == 0) + (o[2] == 0) + (o[3] == 0);
    if (nz == 1) {
        const int kz = o[0] == 0 ? 0 : o[1] == 0 ? 1 : o[2] == 0 ? 2 : 3;
        const uint32_t inf = (M.einfo[e] >> (8 * kz)) & 255u;
        if ((inf & 3) == 0) {
            const int e2 = M.nbr[4 * e + kz];
            if (M.rank[e2] < M.rank[e]) {
                e = e2;
                sx += (int)((inf >> 4) & 3) - 1;
                sy += (int)((inf >> 6) & 3) - 1;
            }
        }
    } else if (nz >= 2) {
        // the corner shared by two zero edges k, k + 1 is corner k + 1
        int vl = 0;
        for (int k = 0; k < 4; ++k)
            if (o[k] == 0 && o[(k + 1) & 3] == 0) vl = (k + 1) & 3;
        r.vnode = M.conn[9 * e + vl];
    }
    r.e = e;
    r.sx = sx;
    r.sy = sy;
    return r;
}

// Straight-line walk from node a along the segment X_a -> p over the
// quadrilaterals, with exact orientation signs (the same reading of the
// departure search as on triangles: a line through a vertex passes to the
// vertex's right; a population is missing when the walk leaves the mesh
// through a boundary edge or no element of the node's fan holds the first
// piece of the segment; a segment along a boundary edge stays inside the
// closed mesh).  Exit edges follow from the side of the segment line that
// each corner lies on: the walk leaves a convex cell where the corners
// change from the right of the line to its left, counter-clockwise.
ALELB_HD inline Loc quad_walk(const QuadDev &M, int a, double Xa, double Ya, double px, double py, int *err)
{
    Loc r;
    r.kind = 0;
    r.vnode = -1;
    r.sx = r.sy = 0;
    if (px == Xa && py == Ya) {
        r.e = quad_fan_best(M, a);
        r.vnode = a;
        return r;
    }
    double w[8];
    int e = -1, loc = 0, sx = 0, sy = 0;
    for (int k = M.fan_ptr[a]; k < M.fan_ptr[a + 1]; ++k) {
        const int2 fe = M.fan[k];
        const int ll = fe.y & 15, ssx = ((fe.y >> 4) & 3) - 1, ssy = ((fe.y >> 6) & 3) - 1;
        quad_frame(M, fe.x, ssx, ssy, w);
        bool hit;
        if (ll < 4) { // corner: the sector between rays ll -> ll+1 and ll -> ll+3
            const int k1 = (ll + 1) & 3, k3 = (ll + 3) & 3;
            const int s1 = orient(w[2 * ll], w[2 * ll + 1], w[2 * k1], w[2 * k1 + 1], px, py);
            const int s3 = orient(w[2 * ll], w[2 * ll + 1], w[2 * k3], w[2 * k3 + 1], px, py);
            hit = s1 >= 0 && s3 < 0;
            if (s1 >= 0 && s3 == 0 && ((M.einfo[fe.x] >> (8 * k3)) & 3u)) {
                // along the incoming boundary edge: no other element holds that ray
                const double dx = px - w[2 * ll], dy = py - w[2 * ll + 1];
                hit = dx * (w[2 * k3] - w[2 * ll]) + dy * (w[2 * k3 + 1] - w[2 * ll + 1]) > 0.0;
            }
        } else if (ll < 8) { // midside node of edge ll - 4: the element's half-plane
            const int k0 = ll - 4, k1 = (k0 + 1) & 3;
            hit = orient(w[2 * k0], w[2 * k0 + 1], w[2 * k1], w[2 * k1 + 1], px, py) >= 0;
        } else { // the centre: strictly inside
            hit = true;
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
        if (!M.bkind[a]) {
            set_err(err, ERR_LOCATE);
            r.e = -2;
            return r;
        }
        r.e = -1;
        r.kind = M.bkind[a];
        return r;
    }
    quad_frame(M, e, sx, sy, w);
    int o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int k1 = (k + 1) & 3;
        o[k] = orient(w[2 * k], w[2 * k + 1], w[2 * k1], w[2 * k1 + 1], px, py);
    }
    if (o[0] >= 0 && o[1] >= 0 && o[2] >= 0 && o[3] >= 0) return quad_finish(M, e, sx, sy, o);
    // side of the segment line of corner k: >= 0 left (or on it), < 0 right
    auto side = [&](int k) { return orient(Xa, Ya, px, py, w[2 * k], w[2 * k + 1]); };
    int kout;
    if (loc < 4) {
        kout = side((loc + 2) & 3) >= 0 ? (loc + 1) & 3 : (loc + 2) & 3;
    } else if (loc < 8) {
        const int k0 = loc - 4;
        kout = side((k0 + 2) & 3) >= 0 ? (k0 + 1) & 3 : side((k0 + 3) & 3) >= 0 ? (k0 + 2) & 3 : (k0 + 3) & 3;
    } else {
        int sd[4];
        for (int k = 0; k < 4; ++k) sd[k] = side(k);
        kout = 0;
        for (int k = 0; k < 4; ++k)
            if (sd[k] < 0 && sd[(k + 1) & 3] >= 0) kout = k;
    }
#pragma unroll 1
    for (int step = 0; step < WALK_LIMIT; ++step) {
        const uint32_t inf = (M.einfo[e] >> (8 * kout)) & 255u;
        const int kind = inf & 3;
        if (kind) {
            r.e = -1;
            r.kind = kind;
            return r;
        }
        const int kin = (inf >> 2) & 3;
        sx += (int)((inf >> 4) & 3) - 1;
        sy += (int)((inf >> 6) & 3) - 1;
        e = M.nbr[4 * e + kout];
        quad_frame(M, e, sx, sy, w);
        bool in = true;
        o[kin] = 1; // crossed from outside: p lies strictly on the inner side of kin
        for (int j = 1; j < 4; ++j) {
            const int k = (kin + j) & 3, k1 = (k + 1) & 3;
            o[k] = orient(w[2 * k], w[2 * k + 1], w[2 * k1], w[2 * k1 + 1], px, py);
            in = in && o[k] >= 0;
        }
        if (in) return quad_finish(M, e, sx, sy, o);
        kout = side((kin + 2) & 3) >= 0 ? (kin + 1) & 3 : side((kin + 3) & 3) >= 0 ? (kin + 2) & 3 : (kin + 3) & 3;
    }
    set_err(err, ERR_LOCATE);
    r.e = -2;
    return r;
}

// The certified FP32 decision of the deviation forms for population i of
// node a: its previous-step element (cache code c, unshifted) holds the FP64
// departure point strictly inside -- four orientation signs certified in
// FP32 against their error bounds (the departure offset -c^ carries F.eq(i)
// per component, the node-relative corners their hi/lo rounding) -- and the
// segment from the node cannot leave the mesh: the cell is one of the
// node's own (convex, it holds both ends) or the segment is shorter than
// the node's distance to any boundary.  The oracle's exhaustive search
// then picks the same cell: a point strictly inside one cell lies in no
// other.  On success cw holds the corners relative to the departure point
// (FP32) for Newton.
ALELB_HD __forceinline__ bool quad_fast_decide(const QuadDev &M, const FastMap &F, float4 Xf, int a, int i, int c,
                                               int &e, float cw[8])
{
    if (!F.ok || c < 0 || (c >> 28) != 5) return false;
    const float u = 5.9604644775390625e-08f;
    const float cx = (float)lat_cx(i), cy = (float)lat_cy(i);
    const float chx = F.A11 * cx + F.A12 * cy - F.W1;
    const float chy = F.A21 * cx + F.A22 * cy - F.W2;
    const float eq = F.eq(i);
    const float len2 = chx * chx + chy * chy;
    const float q4 = 4.0f * eq;
    if (!(len2 > q4 * q4)) return false;
    e = c & CACHE_ELEM;
    bool own = false;
#pragma unroll
    for (int k = 0; k < 9; ++k) own = own || M.conn[9 * e + k] == a;
    if (!own) {
        const float room = M.bdist[a] - eq;
        if (!(room > 0.0f && len2 < room * room)) return false;
    }
    const float px = -chx, py = -chy;
    float rx[4], ry[4], er[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 v = M.evf[4 * e + k];
        const float hx = v.x - Xf.x, hy = v.y - Xf.y;
        rx[k] = hx + (v.z - Xf.z);
        ry[k] = hy + (v.w - Xf.w);
        er[k] = 4.0f * u * (fmaxf(fabsf(rx[k]), fabsf(ry[k])) + fmaxf(fabsf(hx), fabsf(hy))) + 9.313225746154785e-10f;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int k1 = (k + 1) & 3;
        if (orient3_f32(rx[k], ry[k], er[k], rx[k1], ry[k1], er[k1], px, py, eq) <= 0) return false;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cw[2 * k] = rx[k] - px;
        cw[2 * k + 1] = ry[k] - py;
    }
    return true;
}

// Local coordinates of p in element e (frame shift sx, sy) by Newton, in
// the arithmetic A of the interpolation (the corners relative to p are
// formed in FP64, then rounded to A).
template <class A>
ALELB_HD __forceinline__ bool quad_local(const QuadDev &M, int e, int sx, int sy, double px, double py, A &xi,
                                         A &eta)
{
    double w[8];
    quad_frame(M, e, sx, sy, w);
    A c[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c[2 * k] = (A)(w[2 * k] - px);
        c[2 * k + 1] = (A)(w[2 * k + 1] - py);
    }
    if (sizeof(A) == 8) return quad_newton_t<A>(c, A(1e-12), A(1e-9), xi, eta);
    return quad_newton_t<A>(c, A(1e-5), A(1e-4), xi, eta); // FP32: converged near 1e-7
}

// d K / d X at node a in element el = (elem, local): the nine-node
// derivative (full = true; Eq. FE_Derivative in the owner element) or the
// derivative of the bilinear interpolant of the corner values alone (full =
// false; the first-order gradient of the wall condition), with J^{-1} of
// the bilinear map at the node's local position.
template <class S>
__device__ __forceinline__ void quad_grad(const QuadDev &M, int2 el, const S *K, bool full, double &KX, double &KY)
{
    const int e = el.x, l = el.y;
    const double xi = quad_ix(l) - 1.0, eta = quad_iy(l) - 1.0;
    double w[8], x, y, J[4];
    quad_frame(M, e, 0, 0, w);
    quad_bilinear(w, xi, eta, x, y, J);
    double sxi = 0.0, seta = 0.0;
    if (full) {
        double Lx[3], Ly[3], dx[3], dy[3];
        lagrange3(xi, Lx, dx);
        lagrange3(eta, Ly, dy);
#pragma unroll
        for (int s = 0; s < 9; ++s) {
            const double Ks = (double)K[M.conn[9 * e + s]];
            sxi += Ks * (dx[quad_ix(s)] * Ly[quad_iy(s)]);
            seta += Ks * (Lx[quad_ix(s)] * dy[quad_iy(s)]);
        }
    } else {
        const double a[4] = {-0.25 * (1.0 - eta), 0.25 * (1.0 - eta), 0.25 * (1.0 + eta), -0.25 * (1.0 + eta)};
        const double b[4] = {-0.25 * (1.0 - xi), -0.25 * (1.0 + xi), 0.25 * (1.0 + xi), 0.25 * (1.0 - xi)};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double Kk = (double)K[M.conn[9 * e + k]];
            sxi += a[k] * Kk;
            seta += b[k] * Kk;
        }
    }
    const double det = J[0] * J[3] - J[2] * J[1];
    KX = (J[3] * sxi - J[2] * seta) / det;
    KY = (-J[1] * sxi + J[0] * seta) / det;
}

} // namespace alelb

namespace alelb {

// Local node at grid position (i, j) of the 3 x 3 node lattice of an
// element (i along xi, j along eta; 0, 1, 2 for -1, 0, 1): 4-bit fields of
// one word, row j = 0 first (a run-time index into a constant array would
// put the array in local memory).
ALELB_HD __forceinline__ int quad_node_at(int i, int j)
{
    return (int)((0x263587140ull >> (4 * (3 * j + i))) & 15ull);
}

// FP32 d K / d X at node a in its owner element (Eq. FE_Derivative): at a
// node the nine shape functions' xi derivatives vanish off the node's eta
// row and their eta derivatives off its xi column, so each derivative is a
// three-term sum; dL_m at the node's coordinate t in {-1, 0, 1} is t - 1/2,
// -2 t, t + 1/2 (exact in FP32).
template <class S>
__device__ __forceinline__ void quad_grad_f32(const QuadDev &M, int a, const S *K, float &KX, float &KY)
{
    const int2 ow = M.owner[a];
    const int e = ow.x, l = ow.y;
    const int li = quad_ix(l), lj = quad_iy(l);
    const float tx = (float)(li - 1), ty = (float)(lj - 1);
    const int *cn = M.conn + 9 * e;
    const float sxi = (tx - 0.5f) * (float)K[cn[quad_node_at(0, lj)]] + (-2.0f * tx) * (float)K[cn[quad_node_at(1, lj)]] +
                      (tx + 0.5f) * (float)K[cn[quad_node_at(2, lj)]];
    const float seta = (ty - 0.5f) * (float)K[cn[quad_node_at(li, 0)]] + (-2.0f * ty) * (float)K[cn[quad_node_at(li, 1)]] +
                       (ty + 0.5f) * (float)K[cn[quad_node_at(li, 2)]];
    const float4 J = M.ownJf[a];
    KX = sxi * J.x + seta * J.z;
    KY = sxi * J.y + seta * J.w;
}

} // namespace alelb
