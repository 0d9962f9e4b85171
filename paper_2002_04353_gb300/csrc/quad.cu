// quad.cu -- one time step on a mesh of the paper's 9-node quadrilaterals
// (Sec. III), the element-choice report and the wall forces, plus the upload
// of the mesh tables.  The kinetic model (equilibria, collision, Grad-type
// missing populations) is the one the triangles use (kinetic.cuh); only the
// geometry differs: the walk over quadrilaterals, Newton's method for the
// local coordinates of Eq. NonLinear_Eq, the nine shape functions of
// Eq. Propagation and the element gradients (quad.cuh).  The deviation
// forms first try the previous-step element under a certified FP32 test
// (quad_fast_decide); every other population, and every population of the
// FP64 form, takes the exact FP64 path.
#include <cuda_runtime.h>

#include <string>
#include <type_traits>

#include "internal.h"

namespace alelb {
namespace {

// Population i of node a by the certified FP32 decision of the deviation
// forms: its previous-step element, accepted by quad_fast_decide, Newton in
// FP32, the nine-node interpolation.  False: left to the exact path.
template <class S, class A>
__device__ __forceinline__ bool quad_fast_pop(const QuadDev &M, const FastMap &F, float4 Xf, const StateDev<S> &st,
                                              int a, int i)
{
    const int N = M.N;
    const int c = st.cache[i * N + a];
    int e;
    float cw[8];
    float xi, eta;
    if (!(quad_fast_decide(M, F, Xf, a, i, c, e, cw) && quad_newton_t<float>(cw, 1e-5f, 1e-4f, xi, eta)))
        return false;
    A Nw[9];
    shape9<A>((A)xi, (A)eta, Nw);
    A fi = 0, gi = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int b = M.conn[9 * e + k];
        A fb, gb;
        fg_get(st.post, i, b, N, fb, gb);
        fi += Nw[k] * fb;
        gi += Nw[k] * gb;
    }
    fg_put(st.str, i, a, N, fi, gi);
    return true;
}

// Propagation of population pairs i0 .. i0 + G - 1 of node a (Eq.
// Propagation over the nine nodes of the departure element) and, for those
// that are missing, the condition of Sec. IV.A.  TRY: first the certified
// FP32 decision (deviation forms).  The moments, Q'_aaa and mu/(rho T)
// follow in k_moments, as on triangles.
// Returns the number of element walks taken.
template <int G, bool TRY, class S, class A>
__device__ __forceinline__ unsigned quad_stream_pops(const QuadDev &M, const MapStatic &MS, const MapScalars &sc,
                                                     const MapScalars &scd, const MapScalarsF &sfd,
                                                     const KinParams<A> &K, const StateDev<S> &st, int *err, int a,
                                                     int i0)
{
    constexpr bool FAST = !std::is_same<S, double>::value; // the deviation forms keep the element cache
    const int N = M.N;
    const double2 Xa = M.X[a];
    bool have64 = false;
    double a11 = 0, a12 = 0, a21 = 0, a22 = 0, wx = 0, wy = 0, Vx = 0, Vy = 0;
    int miss = 0, far = 0;
    unsigned walks = 0;
    float4 Xf = make_float4(0.f, 0.f, 0.f, 0.f);
    FastMap F;
    F.ok = false;
    if (FAST && TRY) {
        Xf = M.Xf[a];
        F = fast_map(MS, sfd, a, Xf);
        if (K.flags & (FLAG_LITERAL_VG | FLAG_EXACT_CHAR)) F.ok = false;
    }
#pragma unroll 1
    for (int i = i0; i < i0 + G; ++i) {
        A fi = 0, gi = 0;
        int src = -1;
        if (FAST && TRY && F.ok && quad_fast_pop<S, A>(M, F, Xf, st, a, i)) continue;
        if (!have64 && !(K.flags & FLAG_EXACT_CHAR)) {
            double xX, xY, yX, yY;
            map_node(MS, scd, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
            metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
            mesh_velocity_term(a11, a12, a21, a22, ds(Vx, scd.Ux), ds(Vy, scd.Uy), (K.flags & FLAG_LITERAL_VG) != 0,
                               wx, wy);
            have64 = true;
        }
        double chx, chy, px, py;
        if (K.flags & FLAG_EXACT_CHAR)
            exact_departure(MS, sc, scd, (double)c_cx[i], (double)c_cy[i], Xa.x, Xa.y, chx, chy, px, py);
        else
            departure(a11, a12, a21, a22, wx, wy, (double)c_cx[i], (double)c_cy[i], Xa.x, Xa.y, chx, chy, px, py);
        if (chx == 0.0 && chy == 0.0) {
            src = a;
        } else {
            ++walks;
            const Loc L = quad_walk(M, a, Xa.x, Xa.y, px, py, err);
            if (FAST) // the element for the next step's certified check
                st.cache[i * N + a] = L.e >= 0 ? (L.e | ((L.sx + 1) << 28) | ((L.sy + 1) << 30)) : -1;
            if (L.e == -2) {
                src = a;
            } else if (L.e == -1) {
                miss |= 1 << i;
                if (L.kind == 2) far |= 1 << i;
                continue;
            } else if (L.vnode >= 0) {
                src = L.vnode;
            } else {
                A xi, eta;
                if (!quad_local<A>(M, L.e, L.sx, L.sy, px, py, xi, eta)) set_err(err, ERR_LOCATE);
                A Nw[9];
                shape9<A>(xi, eta, Nw);
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const int b = M.conn[9 * L.e + k];
                    A fb, gb;
                    fg_get(st.post, i, b, N, fb, gb);
                    fi += Nw[k] * fb;
                    gi += Nw[k] * gb;
                }
            }
        }
        if (src >= 0) fg_get(st.post, i, src, N, fi, gi);
        fg_put(st.str, i, a, N, fi, gi);
    }

    if (miss) {
        if (!have64 || (K.flags & FLAG_MIDPOINT)) { // the wall condition's map: arrival time
            double xX, xY, yX, yY;
            map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
            metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
        }
        A fm[NQ], gm[NQ];
        if (miss & ~far) {
            A rt, uxt, uyt, Tt;
            const int wi = M.wall_idx[a];
            if (wi >= 0) { // wall node: u = V_G, rho and T at the probe B
                const int pe = M.probe_e[wi];
                const double2 pxi = M.probe_xi[wi];
                A Nw[9];
                shape9<A>((A)pxi.x, (A)pxi.y, Nw);
                A r = 0, t = 0, ub = 0, vb = 0;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const int b = M.conn[9 * pe + k];
                    r += Nw[k] * (A)st.rho[b];
                    t += Nw[k] * (A)st.T[b];
                    if (K.flags & FLAG_SLIP) {
                        ub += Nw[k] * (A)st.ux[b];
                        vb += Nw[k] * (A)st.uy[b];
                    }
                }
                rt = r;
                Tt = t;
                uxt = (A)Vx;
                uyt = (A)Vy;
                if (K.flags & FLAG_SLIP) {
                    const double2 nw = M.wall_nrm[wi];
                    slip_target<A>((A)a11, (A)a12, (A)a21, (A)a22, (A)nw.x, (A)nw.y, ub, vb, (A)Vx, (A)Vy, uxt, uyt);
                }
            } else { // off-wall node: its previous-step fields (mesh velocity under R8c)
                const bool vg = (K.flags & FLAG_OFFWALL_VG) != 0;
                rt = (A)st.rho[a];
                uxt = vg ? (A)Vx : (A)st.ux[a];
                uyt = vg ? (A)Vy : (A)st.uy[a];
                Tt = (A)st.T[a];
            }
            A du[4] = {0, 0, 0, 0}, dT[2] = {0, 0};
            if (!(K.flags & FLAG_BC_EQ) && !((K.flags & FLAG_SLIP) && wi >= 0)) {
                const int2 bc = M.bcel[a];
                double KX, KY;
                quad_grad(M, bc, st.ux, false, KX, KY);
                du[0] = (A)(a11 * KX + a21 * KY);
                du[1] = (A)(a12 * KX + a22 * KY);
                quad_grad(M, bc, st.uy, false, KX, KY);
                du[2] = (A)(a11 * KX + a21 * KY);
                du[3] = (A)(a12 * KX + a22 * KY);
                quad_grad(M, bc, st.T, false, KX, KY);
                dT[0] = (A)(a11 * KX + a21 * KY);
                dT[1] = (A)(a12 * KX + a22 * KY);
            }
            grad_missing(K, rt, uxt, uyt, Tt, du, dT, fm, gm);
        }
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            if (!(miss >> i & 1)) continue;
            const A fi = (far >> i & 1) ? K.finf[i] : fm[i];
            const A gi = (far >> i & 1) ? K.ginf[i] : gm[i];
            fg_put(st.str, i, a, N, fi, gi);
        }
    }
    return walks;
}

// Grid (node blocks, 9 / G direction groups): G directions per thread.
template <class S, class A, int G>
__global__ void __launch_bounds__(128) kq_stream(QuadDev M, MapStatic MS, MapScalars sc, MapScalars scd,
                                                 MapScalarsF sfd, KinParams<A> K, StateDev<S> st, int *err,
                                                 unsigned long long *stats)
{
    wait_prior_grid();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned walks = 0;
    if (a < M.N) walks = quad_stream_pops<G, true>(M, MS, sc, scd, sfd, K, st, err, a, G * blockIdx.y);
    // one atomic per warp (all lanes here: blocks of whole warps)
    const unsigned wsum = __reduce_add_sync(0xffffffffu, walks);
    if (stats && (threadIdx.x & 31u) == 0u && wsum) atomicAdd(stats, (unsigned long long)wsum);
}

// The deviation forms in two passes, as on triangles: kq_fast settles the
// populations whose previous-step element passes the certified FP32 test
// (one thread per population, grid y = direction) and lists the others;
// kq_slow runs the exact path over the list, spread over all blocks, so
// that the walks do not hold up the warps of settled populations.
template <class S, class A>
__global__ void __launch_bounds__(128) kq_fast(QuadDev M, MapStatic MS, MapScalarsF sfd, KinParams<A> K,
                                               StateDev<S> st)
{
    wait_prior_grid();
    const int a = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    int code = 0;
    if (a < M.N) {
        const float4 Xf = M.Xf[a];
        FastMap F = fast_map(MS, sfd, a, Xf);
        if (K.flags & (FLAG_LITERAL_VG | FLAG_EXACT_CHAR)) F.ok = false;
        code = F.ok && quad_fast_pop<S, A>(M, F, Xf, st, a, i) ? 0 : 1;
    }
    if (__any_sync(0xffffffffu, code != 0)) append_pop(st, a, M.N, i, code);
}

template <class S, class A>
__global__ void __launch_bounds__(128) kq_slow(QuadDev M, MapStatic MS, MapScalars sc, MapScalars scd,
                                               MapScalarsF sfd, KinParams<A> K, StateDev<S> st, int *err,
                                               unsigned long long *stats)
{
    wait_prior_grid();
    __shared__ unsigned pre[NQ + 1];
    if (threadIdx.x == 0) work_prefix(st.wcount, pre);
    __syncthreads();
    const unsigned n = pre[NQ];
    if (stats && blockIdx.x == 0 && threadIdx.x == 0 && n) atomicAdd(stats, (unsigned long long)n);
    for (unsigned w = spread_first(); w < n; w += spread_stride()) {
        const int code = work_at(st.work, M.N, pre, w);
        quad_stream_pops<1, false>(M, MS, sc, scd, sfd, K, st, err, code / NQ, code % NQ);
    }
}

// Directions per thread of kq_stream (the FP64 form): one per population,
// the most threads to hide the walks' dependent loads (3.90 ms per launch
// at 150k nodes, against 4.00 at three and 4.12 at nine).
#ifndef ALELB_QUAD_G
#define ALELB_QUAD_G 1
#endif
static_assert(NQ % ALELB_QUAD_G == 0, "directions per thread");

// D_a = (mu / rho T) d_a Q'_aaa in the owner element (Eq. Xa); FP32 in the
// deviation forms (the FP32 map and the node's FP32 owner-element J^{-1}),
// FP64 otherwise.
template <class S, class A>
__global__ void __launch_bounds__(256) kq_deriv1(QuadDev M, MapStatic MS, MapScalars sc, MapScalarsF sf,
                                                 StateDev<S> st)
{
    wait_prior_grid();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= M.N) return;
    if (!std::is_same<S, double>::value) {
        const FastMap F = fast_map(MS, sf, a, M.Xf[a]);
        float KX, KY;
        quad_grad_f32(M, a, st.Qx, KX, KY);
        const float dQx = F.A11 * KX + F.A21 * KY; // d_x Q'_xxx
        quad_grad_f32(M, a, st.Qy, KX, KY);
        const float dQy = F.A12 * KX + F.A22 * KY; // d_y Q'_yyy
        const float m = (float)st.mrt[a];
        st.Dx[a] = (fld_t<S>)(m * dQx);
        st.Dy[a] = (fld_t<S>)(m * dQy);
        return;
    }
    const double2 Xa = M.X[a];
    double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22;
    map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
    metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
    double KX, KY;
    quad_grad(M, M.owner[a], st.Qx, true, KX, KY);
    const double dQx = a11 * KX + a21 * KY;
    quad_grad(M, M.owner[a], st.Qy, true, KX, KY);
    const double dQy = a12 * KX + a22 * KY;
    const double m = (double)st.mrt[a];
    st.Dx[a] = (fld_t<S>)(m * dQx);
    st.Dy[a] = (fld_t<S>)(m * dQy);
}

// X_a = -d_a D_a in the owner element, then the collision (Eqs. feqn, geqn).
template <class S, class A>
__global__ void __launch_bounds__(128) kq_collide(QuadDev M, MapStatic MS, MapScalars sc, MapScalarsF sf,
                                                  KinParams<A> K, StateDev<S> st, int *err)
{
    wait_prior_grid();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= M.N) return;
    const int N = M.N;
    A Xx = 0, Xy = 0;
    if (!std::is_same<S, double>::value && !(K.flags & FLAG_PHI_OFF)) {
        const FastMap F = fast_map(MS, sf, a, M.Xf[a]);
        float KX, KY;
        quad_grad_f32(M, a, st.Dx, KX, KY);
        Xx = (A)(-(F.A11 * KX + F.A21 * KY));
        quad_grad_f32(M, a, st.Dy, KX, KY);
        Xy = (A)(-(F.A12 * KX + F.A22 * KY));
    } else if (!(K.flags & FLAG_PHI_OFF)) {
        const double2 Xa = M.X[a];
        double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22;
        map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
        metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
        double KX, KY;
        quad_grad(M, M.owner[a], st.Dx, true, KX, KY);
        Xx = (A)(-(a11 * KX + a21 * KY));
        quad_grad(M, M.owner[a], st.Dy, true, KX, KY);
        Xy = (A)(-(a12 * KX + a22 * KY));
    }
    A f[NQ], g[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) fg_get(st.str, i, a, N, f[i], g[i]);
    A rho, ux, uy, T;
    if (!collide_node(K, f, g, Xx, Xy, rho, ux, uy, T)) atomicOr(err, ERR_NONFINITE);
#pragma unroll
    for (int i = 0; i < NQ; ++i) fg_put(st.post, i, a, N, f[i], g[i]);
    st.rho[a] = (fld_t<S>)rho;
    st.ux[a] = (fld_t<S>)ux;
    st.uy[a] = (fld_t<S>)uy;
    st.T[a] = (fld_t<S>)T;
}

// Element choice of every population (parity report): original element id,
// -2 (the node itself) or -1 with the boundary kind.
static __global__ void kq_locate(QuadDev M, MapStatic MS, MapScalars sc, int literal, int *elem, int8_t *kind,
                                 int *err)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = M.N;
    if (a >= N) return;
    const double2 Xa = M.X[a];
    double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22, wx, wy;
    map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
    metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
    mesh_velocity_term(a11, a12, a21, a22, ds(Vx, sc.Ux), ds(Vy, sc.Uy), literal != 0, wx, wy);
    for (int i = 0; i < NQ; ++i) {
        double chx, chy, px, py;
        departure(a11, a12, a21, a22, wx, wy, (double)lat_cx(i), (double)lat_cy(i), Xa.x, Xa.y, chx, chy, px, py);
        int e = -2, k = 0;
        if (!(chx == 0.0 && chy == 0.0)) {
            const Loc L = quad_walk(M, a, Xa.x, Xa.y, px, py, err);
            if (L.e >= 0) {
                e = M.orig_elem[L.vnode >= 0 ? quad_fan_best(M, L.vnode) : L.e];
            } else if (L.e == -1) {
                e = -1;
                k = L.kind;
            }
        }
        elem[i * N + a] = e;
        kind[i * N + a] = (int8_t)k;
    }
}

// Wall forces (reading R9): Simpson's rule on each straight 3-node wall edge
// of the mapped geometry, owner-element gradients; one block, fixed-order
// FP64 reduction.  out = {Fx_p, Fy_p, Fx_v, Fy_v}.
template <class S>
__global__ void __launch_bounds__(256) kq_forces(QuadDev M, MapStatic MS, MapScalars sc, StateDev<S> st,
                                                 const int2 *wedges, int nw, double mu, double Cv, double *out)
{
    __shared__ double red[4][256];
    double acc[4] = {0, 0, 0, 0};
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        const int e = wedges[w].x, k = wedges[w].y, k1 = (k + 1) & 3;
        const int nodes[3] = {M.conn[9 * e + k], M.conn[9 * e + 4 + k], M.conn[9 * e + k1]};
        const double2 A0 = M.X[nodes[0]], B0 = M.X[nodes[2]];
        double xa, ya, xb, yb;
        map_position(MS, sc, nodes[0], A0.x, A0.y, xa, ya);
        map_position(MS, sc, nodes[2], B0.x, B0.y, xb, yb);
        const double tx = xb - xa, ty = yb - ya, L = sqrt(tx * tx + ty * ty);
        const double nx = -ty / L, ny = tx / L; // out of the body, into the fluid
        const double wgt[3] = {L / 6.0, 4.0 * L / 6.0, L / 6.0};
        for (int j = 0; j < 3; ++j) {
            const int a = nodes[j];
            const double2 Xa = M.X[a];
            double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22;
            map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
            metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
            double KX, KY, d[4];
            quad_grad(M, M.owner[a], st.ux, true, KX, KY);
            d[0] = a11 * KX + a21 * KY;
            d[1] = a12 * KX + a22 * KY;
            quad_grad(M, M.owner[a], st.uy, true, KX, KY);
            d[2] = a11 * KX + a21 * KY;
            d[3] = a12 * KX + a22 * KY;
            const double div = d[0] + d[3];
            const double p = (double)st.rho[a] * (double)st.T[a];
            const double txx = mu * (2.0 * d[0] - div / Cv);
            const double tyy = mu * (2.0 * d[3] - div / Cv);
            const double txy = mu * (d[1] + d[2]);
            acc[0] += wgt[j] * (-p * nx);
            acc[1] += wgt[j] * (-p * ny);
            acc[2] += wgt[j] * (txx * nx + txy * ny);
            acc[3] += wgt[j] * (txy * nx + tyy * ny);
        }
    }
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = red[threadIdx.x][0];
}

} // namespace

alelb_status quad_mesh_upload(alelb_mesh *m)
{
    const QuadTables &Q = m->QT;
    const HostTables &T = m->T;
    cudaError_t st = cudaSuccess;
    DevBuf &B = m->buf;
    QuadDev &D = m->qdev;
    D.N = T.N;
    D.E = T.E;
    D.Lx = T.Lx;
    D.Ly = T.Ly;
    D.X = B.put(T.X, st);
    D.ev = B.put(Q.ev, st);
    D.nbr = B.put(Q.nbr, st);
    D.einfo = B.put(Q.einfo, st);
    D.rank = B.put(Q.rank, st);
    D.conn = B.put(Q.conn, st);
    D.fan_ptr = B.put(Q.fan_ptr, st);
    D.fan = B.put(Q.fan, st);
    D.owner = B.put(Q.owner, st);
    D.bcel = B.put(Q.bcel, st);
    D.bkind = B.put(Q.bkind, st);
    D.wall_idx = B.put(Q.wall_idx, st);
    D.probe_e = B.put(Q.probe_e, st);
    D.probe_xi = B.put(Q.probe_xi, st);
    D.wall_nrm = B.put(Q.wall_nrm, st);
    D.orig_elem = B.put(Q.orig, st);
    D.Xf = B.put(Q.Xf, st);
    D.evf = B.put(Q.evf, st);
    D.bdist = B.put(Q.bdist, st);
    D.ownJf = B.put(Q.ownJf, st);
    m->d_wedges = B.put(Q.wedges, st);
    m->d_n2o = B.put(T.node_new2old, st);
    m->nw = (int)Q.wedges.size();
    m->mst = T.host_map();
    m->mst.ms = B.put(T.ms, st);
    m->mst.msf = B.put(T.msf, st);
    if (st == cudaSuccess) st = cudaDeviceSynchronize();
    if (st != cudaSuccess) {
        m->buf.release();
        m->err = cudaGetErrorString(st);
        return st == cudaErrorMemoryAllocation ? ALELB_ERR_OOM : ALELB_ERR_CUDA;
    }
    return ALELB_OK;
}

cudaError_t quad_launch(alelb_solver *s, int kernel, const MapScalars &sc, const MapScalars &scd)
{
    alelb_mesh *m = s->mesh;
    const int N = m->T.N;
    with_state(s, [&](auto &st, auto &K) {
        using S = typename std::remove_reference<decltype(st)>::type::Tag;
        using A = typename std::remove_reference<decltype(K)>::type::Arith;
        switch (kernel) {
        case KT_STREAM: {
            constexpr int G = ALELB_QUAD_G;
            launch_pdl(kq_stream<S, A, G>, dim3((N + 127) / 128, NQ / G), dim3(128), s->stream, m->qdev, m->mst, sc,
                       scd, to_f32(scd, m->T), K, st, s->d_err, s->d_stats);
            break;
        }
        case KT_FAST:
            launch_pdl(kq_fast<S, A>, dim3((N + 127) / 128, NQ), dim3(128), s->stream, m->qdev, m->mst,
                       to_f32(scd, m->T), K, st);
            break;
        case KT_SLOW: {
            // every block resident at once (the list spread over all of them)
            static const int per_sm = [] {
                int v = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kq_slow<S, A>, 128, 0);
                return v > 0 ? v : 1;
            }();
            launch_pdl(kq_slow<S, A>, dim3(per_sm * s->n_sm), dim3(128), s->stream, m->qdev, m->mst, sc, scd,
                       to_f32(scd, m->T), K, st, s->d_err, s->d_stats);
            break;
        }
        case KT_MOMENTS:
            launch_pdl(k_moments<S, A>, dim3((N + 255) / 256), dim3(256), s->stream, K, st, N, s->d_err);
            break;
        case KT_DERIV1:
            launch_pdl(kq_deriv1<S, A>, dim3((N + 255) / 256), dim3(256), s->stream, m->qdev, m->mst, sc,
                       to_f32(sc, m->T), st);
            break;
        default:
            launch_pdl(kq_collide<S, A>, dim3((N + 127) / 128), dim3(128), s->stream, m->qdev, m->mst, sc,
                       to_f32(sc, m->T), K, st, s->d_err);
        }
    });
    return cudaGetLastError();
}

cudaError_t quad_locate(alelb_solver *s, const MapScalars &sc, int *elem, int8_t *kind)
{
    alelb_mesh *m = s->mesh;
    kq_locate<<<(m->T.N + 127) / 128, 128, 0, s->stream>>>(m->qdev, m->mst, sc, (s->flags & ALELB_FLAG_LITERAL_VG) != 0,
                                                           elem, kind, s->d_err);
    return cudaGetLastError();
}

cudaError_t quad_forces(alelb_solver *s, const MapScalars &sc)
{
    alelb_mesh *m = s->mesh;
    with_state(s, [&](auto &st, auto &) {
        using S = typename std::remove_reference<decltype(st)>::type::Tag;
        kq_forces<S><<<1, 256, 0, s->stream>>>(m->qdev, m->mst, sc, st, m->d_wedges, m->nw, s->mu, s->Cv, s->d_out);
    });
    return cudaGetLastError();
}

} // namespace alelb
