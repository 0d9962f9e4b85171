// kernels.cuh -- the kernels of one time step plus the element-choice
// report and the force reduction.  The plain FP64 form:
//
//   k_stream   propagation (Eq. Propagation): transformed velocities,
//              departure points, element walk, P2 interpolation of the
//              post-collision populations, Grad-type missing populations
//              (Sec. IV.A); then moments, Q'_aaa (Eq. DeviationTerms) and
//              mu/(rho T)
//   k_deriv1   D_a = (mu/rho T) d_a Q'_aaa in the owner element (Eq. Xa,
//              Eqs. Ph_Derivative / FE_Derivative)
//   k_collide  X_a = -d_a D_a, then the collision of Eqs. feqn/geqn
//
// and the deviation forms' propagation (k_stream_fast, k_stream_slow,
// k_moments, below), which share k_deriv1 and k_collide.  One thread per
// node unless noted.  Populations are stored by direction: FP64 buffers
// as pop[q * N + node] with q = 0..8 for f and 9..17 for g, the deviation
// forms as (f_i, g_i) pairs, pop[2 (i N + node) + {0, 1}] (fg_get).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "geom.cuh"
#include "kinetic.cuh"

namespace alelb {

// Storage of a state: populations (deviations from the reference state) in
// pop_t<S>, node fields in fld_t<S>.  S = double or float stores both in S.
// The two 16-bit forms store the populations in 2 bytes and everything else,
// the arithmetic included, in FP32:
//   Bf16Dev  bfloat16 (8 significant bits, round to nearest even);
//   Fp16Dev  IEEE binary16 of the deviation times 2^10 (11 significant bits;
//            the power-of-two scale is exact and moves deviations down to
//            about 6e-8 out of the subnormal range; |deviation| < 64).
struct Bf16Dev {};
struct Fp16Dev {};
template <class S> struct Store { using pop = S; using fld = S; };
template <> struct Store<Bf16Dev> { using pop = __nv_bfloat16; using fld = float; };
template <> struct Store<Fp16Dev> { using pop = __half; using fld = float; };
template <class S> using pop_t = typename Store<S>::pop;
template <class S> using fld_t = typename Store<S>::fld;

constexpr float FP16_DEV_SCALE = 1024.f, FP16_DEV_UNSCALE = 1.f / 1024.f;

// The pair (f_i, g_i) of node x in a population buffer.  FP64 buffers keep
// f and g in separate planes, pop[q N + x] with q = i for f and 9 + i for
// g.  The deviation forms keep the two side by side, pop[2 (i N + x)] and
// pop[2 (i N + x) + 1], so that one 8-byte (FP32) or 4-byte (16-bit) access
// moves both: the interpolation gathers them at the same six nodes.
template <class A> __device__ __forceinline__ void fg_get(const double *p, int i, int x, int N, A &f, A &g)
{
    f = (A)p[i * N + x];
    g = (A)p[(NQ + i) * N + x];
}
template <class A> __device__ __forceinline__ void fg_get(const float *p, int i, int x, int N, A &f, A &g)
{
    const float2 v = reinterpret_cast<const float2 *>(p)[i * N + x];
    f = (A)v.x;
    g = (A)v.y;
}
template <class A>
__device__ __forceinline__ void fg_get(const __nv_bfloat16 *p, int i, int x, int N, A &f, A &g)
{
    const __nv_bfloat162 v = reinterpret_cast<const __nv_bfloat162 *>(p)[i * N + x];
    f = (A)__low2float(v);
    g = (A)__high2float(v);
}
template <class A> __device__ __forceinline__ void fg_get(const __half *p, int i, int x, int N, A &f, A &g)
{
    const __half2 v = reinterpret_cast<const __half2 *>(p)[i * N + x];
    f = (A)(__low2float(v) * FP16_DEV_UNSCALE);
    g = (A)(__high2float(v) * FP16_DEV_UNSCALE);
}
template <class A> __device__ __forceinline__ void fg_put(double *p, int i, int x, int N, A f, A g)
{
    p[i * N + x] = (double)f;
    p[(NQ + i) * N + x] = (double)g;
}
template <class A> __device__ __forceinline__ void fg_put(float *p, int i, int x, int N, A f, A g)
{
    reinterpret_cast<float2 *>(p)[i * N + x] = make_float2((float)f, (float)g);
}
template <class A> __device__ __forceinline__ void fg_put(__nv_bfloat16 *p, int i, int x, int N, A f, A g)
{
    reinterpret_cast<__nv_bfloat162 *>(p)[i * N + x] = __floats2bfloat162_rn((float)f, (float)g);
}
template <class A> __device__ __forceinline__ void fg_put(__half *p, int i, int x, int N, A f, A g)
{
    reinterpret_cast<__half2 *>(p)[i * N + x] =
        __floats2half2_rn((float)f * FP16_DEV_SCALE, (float)g * FP16_DEV_SCALE);
}
// One half of the pair: part 0 writes f_i, part 1 writes g_i (rounded as
// fg_put rounds it).
__device__ __forceinline__ void pop_put1(double *p, int i, int x, int N, int part, double v)
{
    p[(part * NQ + i) * N + x] = v;
}
__device__ __forceinline__ void pop_put1(float *p, int i, int x, int N, int part, double v)
{
    p[2 * (i * N + x) + part] = (float)v;
}
__device__ __forceinline__ void pop_put1(__nv_bfloat16 *p, int i, int x, int N, int part, double v)
{
    p[2 * (i * N + x) + part] = __float2bfloat16_rn((float)v);
}
__device__ __forceinline__ void pop_put1(__half *p, int i, int x, int N, int part, double v)
{
    p[2 * (i * N + x) + part] = __float2half_rn((float)v * FP16_DEV_SCALE);
}
template <class P> __device__ __forceinline__ void fg_copy(P *dst, const P *src, int i, int x, int N)
{
    if (sizeof(P) == 8) { // FP64 planes
        dst[i * N + x] = src[i * N + x];
        dst[(NQ + i) * N + x] = src[(NQ + i) * N + x];
    } else {
        dst[2 * (i * N + x)] = src[2 * (i * N + x)];
        dst[2 * (i * N + x) + 1] = src[2 * (i * N + x) + 1];
    }
}

// Requests the line holding p into L1 (no result; a later load hits there).
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// Waits until the grids this one depends on have completed and their
// stores are visible.  The step's kernels are launched with programmatic
// stream serialization: a kernel's blocks may start while the previous
// kernel drains, and each waits here before touching memory.  A kernel
// launched the ordinary way returns at once.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class S> struct StateDev {
    using Tag = S; // the storage form
    using P = pop_t<S>;
    using F = fld_t<S>;
    P *post;  // [18 N] post-collision populations (deviations), layout of fg_get
    P *str;   // [18 N] streamed populations
    F *rho, *ux, *uy, *T; // fields of the latest step
    F *Qx, *Qy, *mrt;     // Q'_xxx, Q'_yyy, mu/(rho T)
    F *Dx, *Dy;           // first-pass results
    int *cache;           // [9 N] element of each population's previous departure point
                          // (elem | (sx+1)<<28 | (sy+1)<<30), -1 when empty
    int *work;            // [11 N] populations (9 node + direction) left to the exact path,
                          // direction i's at work[i N + k], k < wcount[i]; then the nodes
                          // with populations certified missing at a wall, at work[9 N + k],
                          // k < wcount[9], their directions in wmask; then the nodes whose
                          // moments the fused batched propagation left to the moments
                          // kernel, at work[10 N + k], k < wcount[10]
    unsigned *wcount;     // [11] entries of each segment
    unsigned *wmask;      // [N] directions certified missing at a wall (bits 0-8); set by the
                          // propagation kernel, read by the exact path, cleared by the
                          // moments kernel
};
constexpr unsigned WMASK_DIRS = (1u << NQ) - 1u;
constexpr int SEG_PENDING = NQ + 1; // the pending-moments segment of the work list

// The exact-path kernels number the work list direction by direction
// (populations of one direction at neighbouring nodes take similar paths,
// so the lanes of a warp stay together): pre[i] = entries before direction
// i; the listed wall nodes follow the nine directions.
__device__ __forceinline__ void work_prefix(const unsigned *wcount, unsigned pre[NQ + 1])
{
    pre[0] = 0u;
#pragma unroll
    for (int i = 0; i < NQ; ++i) pre[i + 1] = pre[i] + wcount[i];
}
__device__ __forceinline__ int work_at(const int *work, int N, const unsigned *pre, unsigned w)
{
    int i = 0;
    while (i < NQ - 1 && w >= pre[i + 1]) ++i;
    return work[(size_t)i * N + (w - pre[i])];
}

// d N_s / d xi and d N_s / d eta of the P2 triangle at the six node
// positions (0,0), (1,0), (0,1), (1/2,0), (1/2,1/2), (0,1/2).
__constant__ double c_dNxi[6][6];
__constant__ double c_dNeta[6][6];

template <class A> __device__ __forceinline__ void shape6(A xi, A eta, A N[6])
{
    A l0 = A(1) - xi - eta;
    N[0] = l0 * (A(2) * l0 - A(1));
    N[1] = xi * (A(2) * xi - A(1));
    N[2] = eta * (A(2) * eta - A(1));
    N[3] = A(4) * l0 * xi;
    N[4] = A(4) * xi * eta;
    N[5] = A(4) * eta * l0;
}

// Slip wall (inviscid variant): the target velocity keeps the wall's
// velocity V_G plus the tangential part of the previous-step velocity
// u_B - V_G at the probe point B.  The tangent is the physical one: the
// computational normal n maps to g^{-1,T} n (normals transform like
// gradients), and t is that vector turned by +90 degrees, normalised.
template <class A>
__device__ __forceinline__ void slip_target(A a11, A a12, A a21, A a22, A nX, A nY, A uB, A vB,
                                            A Vx, A Vy, A &ux, A &uy)
{
    const A nx = a11 * nX + a21 * nY, ny = a12 * nX + a22 * nY;
    const A L = sqrt(nx * nx + ny * ny);
    const A tx = -ny / L, ty = nx / L;
    const A ut = (uB - Vx) * tx + (vB - Vy) * ty;
    ux = Vx + ut * tx;
    uy = Vy + ut * ty;
}

// d K / d X at node a in its owner element (full P2 derivative).
template <class S>
__device__ __forceinline__ void owner_grad(const MeshDev &M, int a, const S *K, double &KX,
                                           double &KY)
{
    int2 ow = M.owner[a];
    int e = ow.x, l = ow.y;
    double2 v0 = M.ev[3 * e], v1 = M.ev[3 * e + 1], v2 = M.ev[3 * e + 2];
    double x_xi = v1.x - v0.x, x_eta = v2.x - v0.x;
    double y_xi = v1.y - v0.y, y_eta = v2.y - v0.y;
    double detJ = x_xi * y_eta - y_xi * x_eta;
    double sxi = 0, seta = 0;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        double Ks = (double)K[M.conn[6 * e + s]];
        sxi += Ks * c_dNxi[l][s];
        seta += Ks * c_dNeta[l][s];
    }
    KX = (y_eta * sxi - y_xi * seta) / detJ;
    KY = (-x_eta * sxi + x_xi * seta) / detJ;
}

// First-order d K / d X for the wall condition: gradient of the linear
// interpolant through the vertices of the node's smallest incident element
// (the wall-side element of a body-fitted mesh).
template <class S>
__device__ __forceinline__ void owner_grad_linear(const MeshDev &M, int a, const S *K,
                                                  double &KX, double &KY)
{
    int e = M.bcel[a];
    double2 v0 = M.ev[3 * e], v1 = M.ev[3 * e + 1], v2 = M.ev[3 * e + 2];
    double x_xi = v1.x - v0.x, x_eta = v2.x - v0.x;
    double y_xi = v1.y - v0.y, y_eta = v2.y - v0.y;
    double detJ = x_xi * y_eta - y_xi * x_eta;
    double K0 = (double)K[M.conn[6 * e]];
    double sxi = (double)K[M.conn[6 * e + 1]] - K0;
    double seta = (double)K[M.conn[6 * e + 2]] - K0;
    KX = (y_eta * sxi - y_xi * seta) / detJ;
    KY = (-x_eta * sxi + x_xi * seta) / detJ;
}

// The plain FP64 propagation: every population through the FP64 departure
// point and the exact walk, one thread per node.
// scd: map scalars of the transformed velocities (sc, or those of the
// midpoint time under FLAG_MIDPOINT); the wall condition keeps sc.
template <class S, class A>
__device__ __forceinline__ void stream_plain_node(const MeshDev &M, const MapStatic &MS,
                                                  const MapScalars &sc, const MapScalars &scd,
                                                  const KinParams<A> &K, const StateDev<S> &st,
                                                  int *err, unsigned long long *stats, int a)
{
    const int N = M.N;
    const double2 Xa = M.X[a];
    bool have64 = false;
    double a11 = 0, a12 = 0, a21 = 0, a22 = 0, wx = 0, wy = 0, Vx = 0, Vy = 0;
    int miss = 0, far = 0;
    unsigned walks = 0;
    // running moments of the streamed populations (deviations)
    A sfm = 0, jx = 0, jy = 0, sg = 0;
#pragma unroll 1
    for (int i = 0; i < NQ; ++i) {
        A fi = 0, gi = 0;
        int src = -1; // node whose value is taken as is
        {
            if (!have64 && !(K.flags & FLAG_EXACT_CHAR)) {
                double xX, xY, yX, yY;
                map_node(MS, scd, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
                metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
                mesh_velocity_term(a11, a12, a21, a22, ds(Vx, scd.Ux), ds(Vy, scd.Uy),
                                   (K.flags & FLAG_LITERAL_VG) != 0, wx, wy);
                have64 = true;
            }
            double chx, chy, px, py;
            if (K.flags & FLAG_EXACT_CHAR)
                exact_departure(MS, sc, scd, (double)c_cx[i], (double)c_cy[i], Xa.x, Xa.y, chx, chy, px, py);
            else
                departure(a11, a12, a21, a22, wx, wy, (double)c_cx[i], (double)c_cy[i], Xa.x, Xa.y, chx,
                          chy, px, py);
            if (chx == 0.0 && chy == 0.0) {
                src = a;
            } else {
                ++walks;
                Loc L = walk(M, a, Xa.x, Xa.y, px, py, err);
                if (L.e == -2) {
                    src = a;
                } else if (L.e == -1) {
                    miss |= 1 << i;
                    if (L.kind == 2) far |= 1 << i;
                    continue;
                } else if (L.vnode >= 0) {
                    src = L.vnode;
                } else {
                    const int e = L.e;
                    double xi, eta;
                    local_coords(M, e, L.sx, L.sy, px, py, xi, eta);
                    A Nw[6];
                    shape6<A>((A)xi, (A)eta, Nw);
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        const int b = M.conn[6 * e + k];
                        A fb, gb;
                        fg_get(st.post, i, b, N, fb, gb);
                        fi += Nw[k] * fb;
                        gi += Nw[k] * gb;
                    }
                }
            }
        }
        if (src >= 0) {
            fg_get(st.post, i, src, N, fi, gi);
        }
        fg_put(st.str, i, a, N, fi, gi);
        sfm += fi;
        jx += (A)c_cx[i] * fi;
        jy += (A)c_cy[i] * fi;
        sg += gi;
    }
    if (stats && walks) atomicAdd(stats, (unsigned long long)walks);
    if (miss) {
        if (!have64 || (K.flags & FLAG_MIDPOINT)) { // the wall condition's map: arrival time
            double xX, xY, yX, yY;
            map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
            metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
        }
        A fm[NQ], gm[NQ];
        if (miss & ~far) {
            // targets (Sec. IV.A): wall node -> u = V_G, rho and T at the
            // probe point B; other nodes -> their previous-step fields
            A rt, uxt, uyt, Tt;
            const int wi = M.wall_idx[a];
            if (wi >= 0) {
                const int pe = M.probe_e[wi];
                const double2 pxi = M.probe_xi[wi];
                A Nw[6];
                shape6<A>((A)pxi.x, (A)pxi.y, Nw);
                A r = 0, t = 0, ub = 0, vb = 0;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    int b = M.conn[6 * pe + k];
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
            } else {
                // off-wall node: its previous-step fields; the velocity is the
                // mesh velocity instead under FLAG_OFFWALL_VG
                const bool vg = (K.flags & FLAG_OFFWALL_VG) != 0;
                rt = (A)st.rho[a];
                uxt = vg ? (A)Vx : (A)st.ux[a];
                uyt = vg ? (A)Vy : (A)st.uy[a];
                Tt = (A)st.T[a];
            }
            A du[4] = {0, 0, 0, 0}, dT[2] = {0, 0};
            if (!(K.flags & FLAG_BC_EQ) && !((K.flags & FLAG_SLIP) && wi >= 0)) {
                double KX, KY;
                owner_grad_linear(M, a, st.ux, KX, KY);
                du[0] = (A)(a11 * KX + a21 * KY);
                du[1] = (A)(a12 * KX + a22 * KY);
                owner_grad_linear(M, a, st.uy, KX, KY);
                du[2] = (A)(a11 * KX + a21 * KY);
                du[3] = (A)(a12 * KX + a22 * KY);
                owner_grad_linear(M, a, st.T, KX, KY);
                dT[0] = (A)(a11 * KX + a21 * KY);
                dT[1] = (A)(a12 * KX + a22 * KY);
            }
            grad_missing(K, rt, uxt, uyt, Tt, du, dT, fm, gm);
        }
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            if (!(miss >> i & 1)) continue;
            A fi = (far >> i & 1) ? K.finf[i] : fm[i];
            A gi = (far >> i & 1) ? K.ginf[i] : gm[i];
            fg_put(st.str, i, a, N, fi, gi);
            sfm += fi;
            jx += (A)c_cx[i] * fi;
            jy += (A)c_cy[i] * fi;
            sg += gi;
        }
    }
    // moments (Sec. IV): rho, u, E, T from the streamed populations
    A rho = K.rho_ref + sfm;
    // w = u - U (relative to the lattice shift), u = w + U
    A rwx = (K.jx_ref + jx) / rho, rwy = (K.jy_ref + jy) / rho;
    A ux = rwx + K.Ux, uy = rwy + K.Uy;
    A E = (K.E2_ref + sg) / (A(2) * rho);
    A T = (E - A(0.5) * (ux * ux + uy * uy)) / K.Cv;
    if (!(rho > A(0)) || !(T > A(0)) || !isfinite(rho) || !isfinite(T)) atomicOr(err, ERR_NONFINITE);
    A k3 = A(1) - A(3) * T;
    st.Qx[a] = (fld_t<S>)(rho * rwx * k3 - rho * rwx * rwx * rwx);
    st.Qy[a] = (fld_t<S>)(rho * rwy * k3 - rho * rwy * rwy * rwy);
    st.mrt[a] = (fld_t<S>)(K.mu / (rho * T));
}

template <class S, class A>
__global__ void __launch_bounds__(128) k_stream(MeshDev M, MapStatic MS, MapScalars sc, MapScalars scd,
                                                KinParams<A> K, StateDev<S> st, int *err,
                                                unsigned long long *stats)
{
    wait_prior_grid();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < M.N) stream_plain_node(M, MS, sc, scd, K, st, err, stats, a);
}

// ---------------------------------------------------------------------------
// The deviation-form propagation, split by path so that the rare exact
// work does not stall the warps of the common case:
//   k_stream_fast  per population: FP32 map; a population whose
//                  previous-step element is verified (fast_decide) is
//                  interpolated and stored, one certified missing by the
//                  exterior cone takes the far-field equilibria or marks
//                  the node's wall mask; the others are appended to a work
//                  list by direction
//   k_stream_slow  per listed entry: the nearby-edge certificates, the
//                  exact check of the cached element, else the walk on
//                  certified FP32 predicates with exact fallback; then the
//                  interpolation or the missing-population condition
//                  (Sec. IV.A); refreshes the element cache.  A listed wall
//                  node runs the wall condition once for its masked
//                  directions
//   k_moments      per node: moments, Q'_aaa and mu/(rho T) of the streamed
//                  populations; resets the work list
// ---------------------------------------------------------------------------
// Missing populations at walls (Sec. IV.A) of node a, the directions in
// mask: the targets (wall node: u = V_G, rho and T at the probe B; other
// nodes: their previous-step fields) and first-order gradients are formed
// once, then every direction of the mask is written.
template <class S, class A>
__device__ __forceinline__ void stream_bc_node(const MeshDev &M, const MapStatic &MS,
                                               const MapScalars &sc, const MapScalarsF &sf,
                                               const KinParams<A> &K, const StateDev<S> &st, int a,
                                               const FastMap &F, unsigned mask)
{
    const int N = M.N;
    float a11, a12, a21, a22, Vx, Vy;
    if (F.ok) {
        a11 = F.A11;
        a12 = F.A12;
        a21 = F.A21;
        a22 = F.A22;
        Vx = F.Vx;
        Vy = F.Vy;
    } else {
        const double2 Xa = M.X[a];
        double xX, xY, yX, yY, vx, vy, b11, b12, b21, b22;
        map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, vx, vy);
        metric_inverse_T(xX, xY, yX, yY, b11, b12, b21, b22);
        a11 = (float)b11;
        a12 = (float)b12;
        a21 = (float)b21;
        a22 = (float)b22;
        Vx = (float)vx;
        Vy = (float)vy;
    }
    A rt, uxt, uyt, Tt;
    const int wi = M.wall_idx[a];
    if (wi >= 0) {
        const int pe = M.probe_e[wi];
        const double2 pxi = M.probe_xi[wi];
        A Nw[6];
        shape6<A>((A)pxi.x, (A)pxi.y, Nw);
        A r = 0, t = 0, ub = 0, vb = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int b = M.conn[6 * pe + k];
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
    } else {
        const bool vg = (K.flags & FLAG_OFFWALL_VG) != 0; // mesh velocity as the target
        rt = (A)st.rho[a];
        uxt = vg ? (A)Vx : (A)st.ux[a];
        uyt = vg ? (A)Vy : (A)st.uy[a];
        Tt = (A)st.T[a];
    }
    A du[4] = {0, 0, 0, 0}, dT[2] = {0, 0};
    if (!(K.flags & FLAG_BC_EQ) && !((K.flags & FLAG_SLIP) && wi >= 0)) {
        float KX, KY;
        owner_grad_linear_f32(M, a, st.ux, KX, KY);
        du[0] = (A)(a11 * KX + a21 * KY);
        du[1] = (A)(a12 * KX + a22 * KY);
        owner_grad_linear_f32(M, a, st.uy, KX, KY);
        du[2] = (A)(a11 * KX + a21 * KY);
        du[3] = (A)(a12 * KX + a22 * KY);
        owner_grad_linear_f32(M, a, st.T, KX, KY);
        dT[0] = (A)(a11 * KX + a21 * KY);
        dT[1] = (A)(a12 * KX + a22 * KY);
    }
    A fm[NQ], gm[NQ];
    grad_missing(K, rt, uxt, uyt, Tt, du, dT, fm, gm);
#pragma unroll
    for (int i = 0; i < NQ; ++i)
        if (mask >> i & 1u) {
            fg_put(st.str, i, a, N, fm[i], gm[i]);
        }
}

// Population i of node a (one thread each): interpolated when its
// previous-step element is verified, the node's own value when c^_0 is
// exactly zero, free-stream equilibria when certified missing at the far
// field.  Returns 0 when settled, 1 when left to the exact path, 2 when
// certified missing at a wall (the wall condition then runs once per node
// in the exact-path kernel).
// fo, go: the settled pair as stored (the moments of the fused batched
// kernel read them; unused elsewhere).
template <class S, class A>
__device__ __forceinline__ int stream_fast_pop(const MeshDev &M, const KinParams<A> &K,
                                               const StateDev<S> &st, int a, int i,
                                               const FastMap &F, float4 Xf, float bd, int c, A &fo, A &go)
{
    const int N = M.N;
    if (i == 0 && M.vzero[a] && !(K.flags & FLAG_SHIFT)) { // c^_0 exactly zero: the node's own value
        fg_copy(st.str, st.post, 0, a, N);
        fg_get(st.post, 0, a, N, fo, go);
        return 0;
    }
    if (!F.ok) return 1;
    int e;
    float xi, eta;
    if (fast_decide(M, F, Xf, bd, a, i, c, e, xi, eta)) {
        A Nw[6];
        shape6<A>((A)xi, (A)eta, Nw);
        // the element's six nodes in three 8-byte loads (conn is 8-byte
        // aligned at every element: 24 bytes per element)
        int nb[6];
        const int2 *cp = reinterpret_cast<const int2 *>(M.conn + 6 * e);
#pragma unroll
        for (int h = 0; h < 3; ++h) {
            const int2 v = cp[h];
            nb[2 * h] = v.x;
            nb[2 * h + 1] = v.y;
        }
        A fi = 0, gi = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int b = nb[k];
            A fb, gb;
            fg_get(st.post, i, b, N, fb, gb);
            fi += Nw[k] * fb;
            gi += Nw[k] * gb;
        }
        fg_put(st.str, i, a, N, fi, gi);
        fo = fi;
        go = gi;
        return 0;
    }
    const int ck = cone_missing(M, F, a, i);
    if (ck == 2) { // far field: free-stream equilibria
        fg_put(st.str, i, a, N, K.finf[i], K.ginf[i]);
        fo = K.finf[i];
        go = K.ginf[i];
        return 0;
    }
    return ck == 1 ? 2 : 1;
}
template <class S, class A>
__device__ __forceinline__ int stream_fast_pop(const MeshDev &M, const KinParams<A> &K,
                                               const StateDev<S> &st, int a, int i,
                                               const FastMap &F, float4 Xf, float bd, int c)
{
    A fo, go;
    return stream_fast_pop(M, K, st, a, i, F, Xf, bd, c, fo, go);
}

// Work-list entries of the lanes of a warp (all lanes take part; direction
// i is the same for the whole warp): code 1 appends population (a, i) to
// direction i's segment, code 2 sets bit i of the node's wall mask, and the
// lane that set the first bit appends the node to the wall-node segment.
// The moments kernel clears the masks once the exact path has used them.
template <class S>
__device__ __forceinline__ void append_pop(const StateDev<S> &st, int a, int N, int i, int code)
{
    const unsigned lane = threadIdx.x & 31u;
    bool first = false;
    if (code == 2) first = atomicOr(st.wmask + a, 1u << i) == 0u;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const bool mine = r == 0 ? code == 1 : first;
        const unsigned m = __ballot_sync(0xffffffffu, mine);
        if (!m) continue;
        const int seg = r == 0 ? i : NQ;
        const int leader = __ffs(m) - 1;
        unsigned base = 0;
        if ((int)lane == leader) base = atomicAdd(st.wcount + seg, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (mine) st.work[(size_t)seg * N + base + __popc(m & ((1u << lane) - 1u))] = r == 0 ? a * NQ + i : a;
    }
}

// Directions per thread of the propagation kernels: the grid's y extent is
// 9 / G; a thread evaluates the node's FP32 map once for its G populations.
// One per thread hides the gathers' latency best on small meshes; nine
// (one thread per node) evaluates each node's map once and wins on large
// meshes with a rotating or deforming map (single case: FAST_G below
// FAST_G_NODES nodes or for translations, else 9; the batch takes
// BATCH_FAST_G).
#ifndef ALELB_FAST_G
#define ALELB_FAST_G 1
#endif
#ifndef ALELB_BATCH_FAST_G
#define ALELB_BATCH_FAST_G 9
#endif
constexpr int FAST_G = ALELB_FAST_G, BATCH_FAST_G = ALELB_BATCH_FAST_G, FAST_G_NODES = 300000;
static_assert(NQ % FAST_G == 0 && NQ % BATCH_FAST_G == 0, "directions per thread");

// Populations G y .. G y + G - 1 of node a (y = blockIdx.y): settled, or
// entered in the work list.
template <int G, class S, class A, bool TR = false>
__device__ __forceinline__ void stream_fast_group(const MeshDev &M, const MapStatic &MS,
                                                  const MapScalarsF &sf, const KinParams<A> &K,
                                                  const StateDev<S> &st, int a)
{
    const int i0 = G * blockIdx.y;
    int code[G];
#pragma unroll
    for (int j = 0; j < G; ++j) code[j] = 0;
    if (a < M.N) {
        // the loads of the thread's cache entries go out together (the
        // stores of the populations would otherwise order them one by one)
        int c[G];
#pragma unroll
        for (int j = 0; j < G; ++j) c[j] = st.cache[(i0 + j) * M.N + a];
        const float bd = M.bdist[a];
        const float4 Xf = M.Xf[a];
        // TR: the map is a translation (no map, plunge)
        FastMap F = TR ? fast_map_translation(sf, Xf) : fast_map(MS, sf, a, Xf);
        if (K.flags & (FLAG_LITERAL_VG | FLAG_EXACT_CHAR)) F.ok = false;
#pragma unroll
        for (int j = 0; j < G; ++j) code[j] = stream_fast_pop(M, K, st, a, i0 + j, F, Xf, bd, c[j]);
    }
    // most warps list nothing: one vote spares them the appends' ballots
    int any = 0;
#pragma unroll
    for (int j = 0; j < G; ++j) any |= code[j];
    if (__any_sync(0xffffffffu, any != 0)) {
#pragma unroll
        for (int j = 0; j < G; ++j) append_pop(st, a, M.N, i0 + j, code[j]);
    }
}

// Threads per block of the single-case propagation kernel.
#ifndef ALELB_FAST_BS
#define ALELB_FAST_BS 128
#endif
constexpr int FAST_BS = ALELB_FAST_BS;

// Grid (node blocks, 9 / G direction groups).  TR: the map is a
// translation (no map, plunge).
template <class S, class A, int G, bool TR>
__global__ void __launch_bounds__(FAST_BS) k_stream_fast(MeshDev M, MapStatic MS, MapScalarsF sf,
                                                     KinParams<A> K, StateDev<S> st)
{
    wait_prior_grid();
    stream_fast_group<G, S, A, TR>(M, MS, sf, K, st, blockIdx.x * blockDim.x + threadIdx.x);
}

// One listed population (code = 9 node + direction): exact decision, then
// interpolation, far-field equilibrium or the missing-population condition.
// pc: a proposed element (cache code) or -1; it is taken only when the
// certified test that accepts previous-step elements accepts it, with the
// interpolation offset formed as the FP32 walk forms it, so the result is
// the walk's bit for bit.  hits (may be null) counts the accepted ones.
// sc, sf: the map at the arrival time (wall condition); scd, sfd: the map
// of the transformed velocities (the same, or the midpoint time under
// FLAG_MIDPOINT).
template <class S, class A>
__device__ __forceinline__ void stream_slow_item(const MeshDev &M, const MapStatic &MS,
                                                 const MapScalars &sc, const MapScalarsF &sf,
                                                 const MapScalars &scd, const MapScalarsF &sfd,
                                                 const KinParams<A> &K, const StateDev<S> &st,
                                                 int *err, int code, int pc = -1,
                                                 unsigned long long *hits = nullptr)
{
    const int N = M.N;
    {
        const int a = code / NQ, i = code % NQ;
        // the entry's chain of dependent loads is its latency: the node's
        // and the cached element's records are requested into L1 up front
        prefetch_l1(M.X + a);
        prefetch_l1(M.bdist + a);
        prefetch_l1(M.nb_ptr + a);
        prefetch_l1(M.fan_ptr + a);
        prefetch_l1(M.conek + a);
        const int hint = st.cache[i * N + a];
        if (hint >= 0) {
            const int e = hint & CACHE_ELEM;
            prefetch_l1(M.conn + 6 * e);
            prefetch_l1(M.evf + 3 * e);
            prefetch_l1(M.evf + 3 * e + 2);
            prefetch_l1(M.ejf + 2 * e + 1);
        }
        const float4 Xf = M.Xf[a];
        FastMap F = fast_map(MS, sfd, a, Xf);
        const FastMap Fb = (K.flags & (FLAG_MIDPOINT | FLAG_EXACT_CHAR)) ? fast_map(MS, sf, a, Xf) : F; // wall condition
        const bool exact_char = (K.flags & FLAG_EXACT_CHAR) != 0;
        if (exact_char) F.ok = false; // the FP32 certificates bound the c^ departure only
        const int literal = (K.flags & FLAG_LITERAL_VG) != 0;
        float qx = 0.f, qy = 0.f;
        int src;
        int clear = -1; // the segment test of the nearby-edge pass, for slow_decide
        const int ck = F.ok && !literal ? certified_missing(M, F, a, i, &clear) : 0;
        if (ck == 1) { // certified to meet a wall first
            stream_bc_node<S, A>(M, MS, sc, sf, K, st, a, Fb, 1u << i);
            return;
        }
        if (ck == 2) { // certified to leave through the far field
            fg_put(st.str, i, a, N, K.finf[i], K.ginf[i]);
            return;
        }
        Loc L;
        int pe;
        float pxi, peta;
        if (pc >= 0 && F.ok && !literal && fast_decide(M, F, Xf, M.bdist[a], a, i, pc, pe, pxi, peta)) {
            // strictly inside element pe: the walk finds pe with no shift and
            // forms the offset from the element's first vertex as below
            const float cx = (float)c_cx[i], cy = (float)c_cy[i];
            const float chx = F.A11 * cx + F.A12 * cy - F.W1;
            const float chy = F.A21 * cx + F.A22 * cy - F.W2;
            const float4 v = M.evf[3 * pe];
            const float x0 = (v.x - Xf.x) + (v.z - Xf.z), y0 = (v.y - Xf.y) + (v.w - Xf.w);
            qx = -chx - x0;
            qy = -chy - y0;
            L.e = pe;
            L.sx = L.sy = 0;
            L.kind = 0;
            L.vnode = -1;
            src = -1;
            if (hits) atomicAdd(hits, 1ull);
        } else {
            // the exact check runs on the previous-step element, or, when
            // there is none (a cold cache), on the proposal: the element it
            // accepts is the one the walk would reach
            bool taken = false;
            const bool use_prop = hint < 0 && pc >= 0;
            L = slow_decide(M, MS, scd, F, Xf, a, i, literal, qx, qy, src, err, use_prop ? pc : hint, clear,
                            exact_char ? &sc : nullptr, use_prop ? &taken : nullptr);
            if (taken && hits) atomicAdd(hits, 1ull);
        }
        A fi = 0, gi = 0;
        if (src >= 0) {
            fg_get(st.post, i, src, N, fi, gi);
        } else if (L.e >= 0) {
            const int e = L.e;
            st.cache[i * N + a] = cache_code(M, e, L.sx, L.sy, a);
            const float4 J = M.ejf[2 * e + 1];
            A Nw[6];
            shape6<A>((A)(J.x * qx + J.y * qy), (A)(J.z * qx + J.w * qy), Nw);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int b = M.conn[6 * e + k];
                A fb, gb;
                fg_get(st.post, i, b, N, fb, gb);
                fi += Nw[k] * fb;
                gi += Nw[k] * gb;
            }
        } else if (L.kind == 2) {
            fi = K.finf[i];
            gi = K.ginf[i];
        } else {
            stream_bc_node<S, A>(M, MS, sc, sf, K, st, a, Fb, 1u << i);
            return;
        }
        fg_put(st.str, i, a, N, fi, gi);
    }
}

// First entry of the exact-path list taken by this thread, and the stride:
// 32 consecutive entries per warp (one direction, coherent), warps dealt
// out across the blocks first, so that a short list spreads over all SMs
// rather than filling the first few (its walks are latency chains that
// would otherwise queue on those SMs' few FP64 units).
__device__ __forceinline__ unsigned spread_first()
{
    return (blockIdx.x + (threadIdx.x >> 5) * gridDim.x) * 32u + (threadIdx.x & 31u);
}
__device__ __forceinline__ unsigned spread_stride() { return gridDim.x * blockDim.x; }

// Entry w of the exact path's numbering (work_prefix over the 10 segments):
// a population (9 node + direction), or a listed wall node, whose wall
// condition is computed once for all its certified directions.
template <class S, class A>
__device__ __forceinline__ void slow_entry(const MeshDev &M, const MapStatic &MS,
                                           const MapScalars &sc, const MapScalarsF &sf,
                                           const MapScalars &scd, const MapScalarsF &sfd,
                                           const KinParams<A> &K, const StateDev<S> &st, int *err,
                                           const unsigned *pre, unsigned w, const int *prop,
                                           unsigned long long *stats)
{
    if (w < pre[NQ]) {
        stream_slow_item(M, MS, sc, sf, scd, sfd, K, st, err, work_at(st.work, M.N, pre, w),
                         prop ? prop[w] : -1, prop && stats ? stats + 1 : nullptr);
    } else {
        const int a = st.work[(size_t)NQ * M.N + (w - pre[NQ])];
        const unsigned mask = st.wmask[a] & WMASK_DIRS;
        if (stats) atomicAdd(stats, (unsigned long long)__popc(mask));
        stream_bc_node<S, A>(M, MS, sc, sf, K, st, a, fast_map(MS, sf, a, M.Xf[a]), mask);
    }
}

template <class S, class A>
__global__ void __launch_bounds__(128) k_stream_slow(MeshDev M, MapStatic MS, MapScalars sc,
                                                     MapScalarsF sf, MapScalars scd, MapScalarsF sfd,
                                                     KinParams<A> K, StateDev<S> st, int *err,
                                                     unsigned long long *stats, const int *prop)
{
    wait_prior_grid();
    __shared__ unsigned pre[NQ + 1];
    if (threadIdx.x == 0) work_prefix(st.wcount, pre);
    __syncthreads();
    const unsigned n = pre[NQ];
    const unsigned total = n + st.wcount[NQ];
    if (stats && blockIdx.x == 0 && threadIdx.x == 0 && n) atomicAdd(stats, (unsigned long long)n);
    for (unsigned w = spread_first(); w < total; w += spread_stride())
        slow_entry(M, MS, sc, sf, scd, sfd, K, st, err, pre, w, prop, stats);
}


// rho, u, E, T of the streamed pairs f, g of node a, then Q'_aaa and
// mu / (rho T) (the fused batched propagation kernel shares this).
template <class S, class A>
__device__ __forceinline__ void moments_store(const KinParams<A> &K, const StateDev<S> &st, int *err, int a,
                                              const A f[NQ], const A g[NQ])
{
    const A sf = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    const A jx = K.jx_ref + ((f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]));
    const A jy = K.jy_ref + ((f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]));
    const A sg = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
    const A rho = K.rho_ref + sf;
    const A wx = jx / rho, wy = jy / rho; // u - U
    const A ux = wx + K.Ux, uy = wy + K.Uy;
    const A E = (K.E2_ref + sg) / (A(2) * rho);
    const A T = (E - A(0.5) * (ux * ux + uy * uy)) / K.Cv;
    if (!(rho > A(0)) || !(T > A(0)) || !isfinite(rho) || !isfinite(T)) atomicOr(err, ERR_NONFINITE);
    const A k3 = A(1) - A(3) * T;
    st.Qx[a] = (fld_t<S>)(rho * wx * k3 - rho * wx * wx * wx);
    st.Qy[a] = (fld_t<S>)(rho * wy * k3 - rho * wy * wy * wy);
    st.mrt[a] = (fld_t<S>)(K.mu / (rho * T));
}

template <class S, class A>
__device__ __forceinline__ void moments_node(const KinParams<A> &K, const StateDev<S> &st, int N,
                                             int *err, int a)
{
    st.wmask[a] = 0u; // used by the exact path of this step
    A f[NQ], g[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        fg_get(st.str, i, a, N, f[i], g[i]);
    }
    moments_store(K, st, err, a, f, g);
}

template <class S, class A>
__global__ void __launch_bounds__(256) k_moments(KinParams<A> K, StateDev<S> st, int N, int *err)
{
    wait_prior_grid();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a <= NQ) st.wcount[a] = 0u; // the work list has been consumed
    if (a < N) moments_node(K, st, N, err, a);
}

// FP32 owner-element derivative d K / d X (rows of the FP32 inverse
// Jacobian: grad xi = (j11, j12), grad eta = (j21, j22)).
__constant__ float c_dNxif[6][6];
__constant__ float c_dNetaf[6][6];

// Fills this module's derivative tables: d N_s / d xi and d N_s / d eta of
// the P2 shape functions at the six node positions.  Internal linkage, so
// every translation unit that launches the kernels uploads its own copy.
static inline cudaError_t upload_fe_tables()
{
    static const double LXI[6][2] = {{0, 0}, {1, 0}, {0, 1}, {0.5, 0}, {0.5, 0.5}, {0, 0.5}};
    double dxi[6][6], deta[6][6];
    float dxif[6][6], detaf[6][6];
    for (int l = 0; l < 6; ++l) {
        const double xi = LXI[l][0], eta = LXI[l][1], l0 = 1.0 - xi - eta;
        const double nx[6] = {-(4 * l0 - 1), 4 * xi - 1, 0, 4 * (l0 - xi), 4 * eta, -4 * eta};
        const double ne[6] = {-(4 * l0 - 1), 0, 4 * eta - 1, -4 * xi, 4 * xi, 4 * (l0 - eta)};
        for (int s = 0; s < 6; ++s) {
            dxi[l][s] = nx[s];
            deta[l][s] = ne[s];
            dxif[l][s] = (float)nx[s];
            detaf[l][s] = (float)ne[s];
        }
    }
    cudaError_t st = cudaMemcpyToSymbol(c_dNxi, dxi, sizeof(dxi));
    if (st == cudaSuccess) st = cudaMemcpyToSymbol(c_dNeta, deta, sizeof(deta));
    if (st == cudaSuccess) st = cudaMemcpyToSymbol(c_dNxif, dxif, sizeof(dxif));
    if (st == cudaSuccess) st = cudaMemcpyToSymbol(c_dNetaf, detaf, sizeof(detaf));
    return st;
}

// d N_s / d xi and d N_s / d eta of the P2 shape functions at local node l,
// from its local coordinates (0, 1/2 or 1, as 2-bit fields of one word):
// the values of the c_dNxif / c_dNetaf tables, exact in FP32, without a
// per-thread index into constant memory (which serialises when the lanes'
// l differ).
__device__ __forceinline__ void p2_dN_at_node(int l, float nx[6], float ne[6])
{
    const float xi = 0.5f * (float)((0x148u >> (2 * l)) & 3u);
    const float eta = 0.5f * (float)((0x520u >> (2 * l)) & 3u);
    const float l0 = (1.0f - xi) - eta;
    nx[0] = -(4.0f * l0 - 1.0f);
    nx[1] = 4.0f * xi - 1.0f;
    nx[2] = 0.0f;
    nx[3] = 4.0f * (l0 - xi);
    nx[4] = 4.0f * eta;
    nx[5] = -4.0f * eta;
    ne[0] = -(4.0f * l0 - 1.0f);
    ne[1] = 0.0f;
    ne[2] = 4.0f * eta - 1.0f;
    ne[3] = -4.0f * xi;
    ne[4] = 4.0f * xi;
    ne[5] = 4.0f * (l0 - eta);
}

// The FP32 derivative passes read each node's owner stencil from one
// per-node record (MeshDev::ostn), so the node values they gather wait on
// one load, not on the owner record and then the element's node numbers.
template <class S>
__device__ __forceinline__ void owner_grad_f32(const MeshDev &M, int a, const S *K, float &KX,
                                               float &KY)
{
    const int4 p = M.ostn[2 * a], q = M.ostn[2 * a + 1];
    const int e = q.z, l = q.w;
    const float4 J = M.ejf[2 * e + 1];
    const int nb[6] = {p.x, p.y, p.z, p.w, q.x, q.y};
    float nx[6], ne[6];
    p2_dN_at_node(l, nx, ne);
    float sxi = 0.f, seta = 0.f;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const float Ks = (float)K[nb[s]];
        sxi += Ks * nx[s];
        seta += Ks * ne[s];
    }
    KX = sxi * J.x + seta * J.z;
    KY = sxi * J.y + seta * J.w;
}

// First-order FP32 d K / d X for the wall condition, through the vertices
// of the node's smallest incident element.
template <class S>
__device__ __forceinline__ void owner_grad_linear_f32(const MeshDev &M, int a, const S *K,
                                                      float &KX, float &KY)
{
    const int e = M.bcel[a];
    const float4 J = M.ejf[2 * e + 1];
    const float K0 = (float)K[M.conn[6 * e]];
    const float sxi = (float)K[M.conn[6 * e + 1]] - K0;
    const float seta = (float)K[M.conn[6 * e + 2]] - K0;
    KX = sxi * J.x + seta * J.z;
    KY = sxi * J.y + seta * J.w;
}

template <class S, class A, bool FAST>
__device__ __forceinline__ void deriv1_node(const MeshDev &M, const MapStatic &MS,
                                            const MapScalars &sc, const MapScalarsF &sf,
                                            const StateDev<S> &st, int a)
{
    if (FAST) {
        const FastMap F = fast_map(MS, sf, a, M.Xf[a]);
        float KX, KY;
        owner_grad_f32(M, a, st.Qx, KX, KY);
        const float dQx = F.A11 * KX + F.A21 * KY; // d_x Q'_xxx
        owner_grad_f32(M, a, st.Qy, KX, KY);
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
    owner_grad(M, a, st.Qx, KX, KY);
    double dQx = a11 * KX + a21 * KY; // d_x Q'_xxx
    owner_grad(M, a, st.Qy, KX, KY);
    double dQy = a12 * KX + a22 * KY; // d_y Q'_yyy
    double m = (double)st.mrt[a];
    st.Dx[a] = (fld_t<S>)(m * dQx);
    st.Dy[a] = (fld_t<S>)(m * dQy);
}

template <class S, class A, bool FAST>
__global__ void __launch_bounds__(256) k_deriv1(MeshDev M, MapStatic MS, MapScalars sc,
                                                MapScalarsF sf, StateDev<S> st)
{
    wait_prior_grid();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < M.N) deriv1_node<S, A, FAST>(M, MS, sc, sf, st, a);
}

template <class S, class A, bool FAST>
__device__ __forceinline__ void collide_at(const MeshDev &M, const MapStatic &MS,
                                           const MapScalars &sc, const MapScalarsF &sf,
                                           const KinParams<A> &K, const StateDev<S> &st, int *err,
                                           int a)
{
    const int N = M.N;
    A Xx = 0, Xy = 0;
    if (FAST && !(K.flags & FLAG_PHI_OFF)) {
        const FastMap F = fast_map(MS, sf, a, M.Xf[a]);
        float KX, KY;
        owner_grad_f32(M, a, st.Dx, KX, KY);
        Xx = (A)(-(F.A11 * KX + F.A21 * KY));
        owner_grad_f32(M, a, st.Dy, KX, KY);
        Xy = (A)(-(F.A12 * KX + F.A22 * KY));
    } else if (!(K.flags & FLAG_PHI_OFF)) {
        const double2 Xa = M.X[a];
        double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22;
        map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
        metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
        double KX, KY;
        owner_grad(M, a, st.Dx, KX, KY);
        Xx = (A)(-(a11 * KX + a21 * KY));
        owner_grad(M, a, st.Dy, KX, KY);
        Xy = (A)(-(a12 * KX + a22 * KY));
    }
    A f[NQ], g[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        fg_get(st.str, i, a, N, f[i], g[i]);
    }
    A rho, ux, uy, T;
    if (!collide_node(K, f, g, Xx, Xy, rho, ux, uy, T)) atomicOr(err, ERR_NONFINITE);
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        fg_put(st.post, i, a, N, f[i], g[i]);
    }
    st.rho[a] = (fld_t<S>)rho;
    st.ux[a] = (fld_t<S>)ux;
    st.uy[a] = (fld_t<S>)uy;
    st.T[a] = (fld_t<S>)T;
}

template <class S, class A, bool FAST>
__global__ void __launch_bounds__(128) k_collide(MeshDev M, MapStatic MS, MapScalars sc,
                                                 MapScalarsF sf, KinParams<A> K, StateDev<S> st,
                                                 int *err)
{
    wait_prior_grid();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < M.N) collide_at<S, A, FAST>(M, MS, sc, sf, K, st, err, a);
}

// Element choice of every population at map time t (parity report).  With
// cache != nullptr each population first takes the propagation kernel's
// fast decision (verified previous-step element), as k_stream would.
static __global__ void k_locate(MeshDev M, MapStatic MS, MapScalars sc, MapScalarsF sf, int flags,
                         const int *cache, int *elem, int8_t *kind, int *err)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = M.N;
    if (a >= N) return;
    int e9[NQ];
    int8_t k9[NQ];
    if (cache && !(flags & FLAG_LITERAL_VG)) {
        mixed_locate_node(M, MS, sc, sf, cache, a, e9, k9, nullptr, err);
    } else {
        locate_node(M, MS, sc, flags & FLAG_LITERAL_VG, a, e9, k9, err);
    }
    for (int i = 0; i < NQ; ++i) {
        elem[i * N + a] = e9[i];
        kind[i * N + a] = k9[i];
    }
}

// Wall forces: one block, fixed-order FP64 reduction.
// out = {Fx_p, Fy_p, Fx_v, Fy_v}.
template <class S>
__global__ void __launch_bounds__(256) k_forces(MeshDev M, MapStatic MS, MapScalars sc,
                                                StateDev<S> st, const int2 *wedges, int nw,
                                                double mu, double Cv, double *out)
{
    __shared__ double red[4][256];
    double acc[4] = {0, 0, 0, 0};
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        int e = wedges[w].x, k = wedges[w].y, k1 = (k + 1) % 3;
        int nodes[3] = {M.conn[6 * e + k], M.conn[6 * e + 3 + k], M.conn[6 * e + k1]};
        double2 A0 = M.X[nodes[0]], B0 = M.X[nodes[2]];
        double xa, ya, xb, yb;
        map_position(MS, sc, nodes[0], A0.x, A0.y, xa, ya);
        map_position(MS, sc, nodes[2], B0.x, B0.y, xb, yb);
        double tx = xb - xa, ty = yb - ya, L = sqrt(tx * tx + ty * ty);
        double nx = -ty / L, ny = tx / L; // out of the body, into the fluid
        double wgt[3] = {L / 6.0, 4.0 * L / 6.0, L / 6.0};
        for (int j = 0; j < 3; ++j) {
            int a = nodes[j];
            double2 Xa = M.X[a];
            double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22;
            map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
            metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
            double KX, KY, d[4];
            owner_grad(M, a, st.ux, KX, KY);
            d[0] = a11 * KX + a21 * KY;
            d[1] = a12 * KX + a22 * KY;
            owner_grad(M, a, st.uy, KX, KY);
            d[2] = a11 * KX + a21 * KY;
            d[3] = a12 * KX + a22 * KY;
            double div = d[0] + d[3];
            double p = (double)st.rho[a] * (double)st.T[a];
            double txx = mu * (2.0 * d[0] - div / Cv);
            double tyy = mu * (2.0 * d[3] - div / Cv);
            double txy = mu * (d[1] + d[2]);
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

// det g > 0 check at every node (alelb_mesh_move).
static __global__ void k_check_map(MapStatic MS, MapScalars sc, const double2 *X, int N, int *bad)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22;
    map_node(MS, sc, a, X[a].x, X[a].y, xX, xY, yX, yY, Vx, Vy);
    double det = metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
    if (!(det > 0.0)) atomicAdd(bad, 1);
}

} // namespace alelb
