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

#include "internal.h"

using namespace alelb;

namespace {
void forget_noalloc_scratch(int dev);
}

namespace alelb {

const char *const KT_NAMES[KT_N] = {"k_stream", "k_stream_fast", "k_stream_slow", "k_moments", "k_deriv1",
                                    "k_collide", "k_propose"};

// A lattice shift the library accepts: finite, |U_d| <= 1, and exact in
// FP32, so that the FP32 and FP64 paths see the same velocities c_i + U.
static bool shift_ok(const double U[2])
{
    for (int d = 0; d < 2; ++d)
        if (!std::isfinite(U[d]) || std::fabs(U[d]) > 1.0 || (double)(float)U[d] != U[d]) return false;
    return true;
}

MapScalarsF to_f32(const MapScalars &S, const HostTables &T)
{
    MapScalarsF F;
    F.s = (float)S.s;
    F.sd = (float)S.sd;
    F.vy = (float)S.vy;
    F.c = (float)S.c;
    F.sn = (float)S.sn;
    F.thd = (float)S.thd;
    F.cm = (float)S.cm;
    F.Xc = (float)T.mp[3];
    F.Yc = (float)T.mp[4];
    F.Ux = (float)S.Ux;
    F.Uy = (float)S.Uy;
    F.Us = std::fabs(F.Ux) + std::fabs(F.Uy);
    F.er0 = 2.0f + 2.0f * F.Us;
    return F;
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
    if (s->sticky & ERR_TIMEOUT) {
        s->err = "a grid-wide wait of the persistent batched step ran out of time";
        return ALELB_ERR_TIMEOUT;
    }
    return ALELB_OK;
}

} // namespace alelb

namespace {

template <class S> void put_state(DevBuf &b, StateDev<S> &s, int N, cudaError_t &st)
{
    using P = pop_t<S>;
    using F = fld_t<S>;
    s.post = b.alloc<P>((size_t)18 * N, st);
    s.str = b.alloc<P>((size_t)18 * N, st);
    s.rho = b.alloc<F>(N, st);
    s.ux = b.alloc<F>(N, st);
    s.uy = b.alloc<F>(N, st);
    s.T = b.alloc<F>(N, st);
    s.Qx = b.alloc<F>(N, st);
    s.Qy = b.alloc<F>(N, st);
    s.mrt = b.alloc<F>(N, st);
    s.Dx = b.alloc<F>(N, st);
    s.Dy = b.alloc<F>(N, st);
    s.cache = b.alloc<int>((size_t)9 * N, st);
    if (st == cudaSuccess) st = cudaMemset(s.cache, 0xff, (size_t)9 * N * sizeof(int)); // -1: empty
    s.work = b.alloc<int>((size_t)(SEG_PENDING + 1) * N, st);
    s.wcount = b.alloc<unsigned>(SEG_PENDING + 1, st);
    if (st == cudaSuccess) st = cudaMemset(s.wcount, 0, (SEG_PENDING + 1) * sizeof(unsigned));
    s.wmask = b.alloc<unsigned>(N, st);
    if (st == cudaSuccess) st = cudaMemset(s.wmask, 0, (size_t)N * sizeof(unsigned));
}


} // namespace

// ============================================================================
// mesh
// ============================================================================
extern "C" alelb_status alelb_mesh_create(const alelb_mesh_desc *d, alelb_mesh **out)
{
    if (!d || !out) return ALELB_ERR_ARG;
    *out = nullptr;
    alelb_mesh *m = new (std::nothrow) alelb_mesh();
    if (!m) return ALELB_ERR_OOM;
    HostTables &T = m->T;
    if (d->elem_type != ALELB_ELEM_P2TRI && d->elem_type != ALELB_ELEM_Q2QUAD) {
        *out = m;
        m->err = "unknown element type";
        return ALELB_ERR_ARG;
    }
    m->etype = d->elem_type;
    alelb_status bs = m->etype == ALELB_ELEM_Q2QUAD ? build_quad_tables(d, T, m->QT, m->err)
                                                    : build_tables(d, T, m->err);
    if (bs != ALELB_OK) {
        *out = m; // returned so that alelb_mesh_last_error can be read
        return bs;
    }
    {
        uint64_t h = 1469598103934665603ull;
        auto mix = [&h](const void *p, size_t n) {
            const unsigned char *b = (const unsigned char *)p;
            for (size_t k = 0; k < n; ++k) {
                h ^= b[k];
                h *= 1099511628211ull;
            }
        };
        const bool q = m->etype == ALELB_ELEM_Q2QUAD;
        const std::vector<int> &cn = q ? m->QT.conn : T.conn;
        const std::vector<uint32_t> &ei = q ? m->QT.einfo : T.einfo;
        mix(&m->etype, sizeof(int));
        mix(T.X.data(), T.X.size() * sizeof(double2));
        mix(cn.data(), cn.size() * sizeof(int));
        mix(ei.data(), ei.size() * sizeof(uint32_t));
        mix(&T.Lx, sizeof(double));
        mix(&T.Ly, sizeof(double));
        mix(&T.mkind, sizeof(int));
        mix(T.mp, sizeof(T.mp));
        m->fingerprint = h;
    }
    // upload
    cudaError_t st = cudaGetDevice(&m->device);
    if (st == cudaSuccess) forget_noalloc_scratch(m->device);
    if (st == cudaSuccess && m->etype == ALELB_ELEM_Q2QUAD) {
        *out = m;
        return quad_mesh_upload(m);
    }
    DevBuf &B = m->buf;
    MeshDev &D = m->dev;
    D.N = T.N;
    D.E = T.E;
    D.Lx = T.Lx;
    D.Ly = T.Ly;
    D.X = B.put(T.X, st);
    D.ev = B.put(T.ev, st);
    D.nbr = B.put(T.nbr, st);
    D.einfo = B.put(T.einfo, st);
    D.rank = B.put(T.rank, st);
    D.conn = B.put(T.conn, st);
    D.fan_ptr = B.put(T.fan_ptr, st);
    D.fan = B.put(T.fan, st);
    D.owner = B.put(T.owner, st);
    T.ostn.resize((size_t)2 * T.N);
    for (int a = 0; a < T.N; ++a) {
        const int e = T.owner[a].x;
        const int *c = T.conn.data() + (size_t)6 * e;
        T.ostn[2 * a] = make_int4(c[0], c[1], c[2], c[3]);
        T.ostn[2 * a + 1] = make_int4(c[4], c[5], e, T.owner[a].y);
    }
    D.ostn = B.put(T.ostn, st);
    D.bcel = B.put(T.bcel, st);
    D.ring_ptr = B.put(T.ring_ptr, st);
    D.ring = B.put(T.ring, st);
    D.nscale = B.put(T.nscale, st);
    D.bkind = B.put(T.bkind, st);
    D.vzero = B.put(T.vzero, st);
    D.cone = B.put(T.cone, st);
    D.conek = B.put(T.conek, st);
    D.wall_idx = B.put(T.wall_idx, st);
    D.probe_e = B.put(T.probe_e, st);
    D.probe_xi = B.put(T.probe_xi, st);
    D.wall_nrm = B.put(T.wall_nrm, st);
    D.orig_elem = B.put(T.orig, st);
    D.ejf = B.put(T.ejf, st);
    D.bdist = B.put(T.bdist, st);
    D.Xf = B.put(T.Xf, st);
    D.v0f = B.put(T.v0f, st);
    D.evf = B.put(T.evf, st);
    D.nb_ptr = B.put(T.nb_ptr, st);
    D.nb = B.put(T.nb, st);
    D.nbf = B.put(T.nbf, st);
    m->d_wedges = B.put(T.wedges, st);
    m->d_n2o = B.put(T.node_new2old, st);
    m->nw = (int)T.wedges.size();
    m->mst = T.host_map();
    m->mst.ms = B.put(T.ms, st);
    m->mst.msf = B.put(T.msf, st);
    if (st == cudaSuccess) st = upload_fe_tables();
    if (st == cudaSuccess) st = batch_fe_tables();
    // the uploads above run on the legacy default stream, which solvers on
    // non-blocking streams do not wait for
    if (st == cudaSuccess) st = cudaDeviceSynchronize();
    *out = m;
    if (st != cudaSuccess) {
        m->buf.release();
        m->err = cudaGetErrorString(st);
        return st == cudaErrorMemoryAllocation ? ALELB_ERR_OOM : ALELB_ERR_CUDA;
    }
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
    MapScalars S = map_scalars(m->T.mkind, m->T.mp, t);
    int *d_bad = nullptr, bad = 0;
    cudaError_t st = cudaMalloc(&d_bad, sizeof(int));
    if (st == cudaSuccess) st = cudaMemset(d_bad, 0, sizeof(int));
    if (st == cudaSuccess) {
        k_check_map<<<(m->T.N + 255) / 256, 256>>>(m->mst, S, m->dev.X, m->T.N, d_bad);
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


// Reference and far-field populations computed on the device with the
// same kernel code that the step uses.  Reference: none (ref_mode 0, the
// FP64 form stores full populations), the equilibria at rest at rho_inf,
// T_inf (1, FP32 deviations), or the far-field equilibria (2, the 16-bit
// forms: far from the body the stored deviations are then close to zero,
// where the 16-bit formats have their finest absolute spacing).
__global__ void k_kin_consts(KinParams<double> K, double rho_inf, double uxi, double uyi,
                             double T_inf, int ref_mode, double *out)
{
    double f[NQ], g[NQ];
    const double urx = ref_mode == 2 ? uxi : 0.0, ury = ref_mode == 2 ? uyi : 0.0;
    equilibria(K, rho_inf, urx, ury, T_inf, f, g);
    for (int i = 0; i < NQ; ++i) {
        out[i] = ref_mode ? f[i] : 0.0;
        out[NQ + i] = ref_mode ? g[i] : 0.0;
    }
    // far field
    equilibria(K, rho_inf, uxi, uyi, T_inf, f, g);
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
        fg_put(st.post, i, a, N, consts[2 * NQ + i] - consts[i], consts[3 * NQ + i] - consts[NQ + i]);
    }
    st.rho[a] = (fld_t<S>)rho;
    st.ux[a] = (fld_t<S>)ux;
    st.uy[a] = (fld_t<S>)uy;
    st.T[a] = (fld_t<S>)T;
}

// Full FP64 populations <-> stored deviations (internal order), one
// population set per launch so that each half's kernel overlaps the other
// half's host copy.  plane ([9 N]) and fields are in the caller's node
// order: internal node a is caller node n2o[a].
// part 0: the f plane; without fields, rho and u = sum (c_i + U) f_i / rho
// go to tmp ([3 N], internal order, FP64).  part 1: the g plane, then the
// fields (given, or T from sum g_i and tmp).
template <class S>
__global__ void k_import(StateDev<S> st, int N, const double *consts, const double *plane,
                         const double *fields, int have_fields, double Cv, double Ux, double Uy,
                         const int *n2o, double *tmp, int part)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    const int o = n2o[a];
    double sum = 0, jx = 0, jy = 0;
    for (int i = 0; i < NQ; ++i) {
        const double v = plane[i * N + o];
        pop_put1(st.post, i, a, N, part, v - consts[part * NQ + i]);
        sum += v;
        if (part == 0) {
            jx += c_cx[i] * v;
            jy += c_cy[i] * v;
        }
    }
    if (part == 0) {
        if (!have_fields) {
            tmp[a] = sum;
            tmp[N + a] = jx / sum + Ux; // lattice c_i + U
            tmp[2 * N + a] = jy / sum + Uy;
        }
    } else if (have_fields) {
        st.rho[a] = (fld_t<S>)fields[o];
        st.ux[a] = (fld_t<S>)fields[N + o];
        st.uy[a] = (fld_t<S>)fields[2 * N + o];
        st.T[a] = (fld_t<S>)fields[3 * N + o];
    } else {
        const double r = tmp[a], ux = tmp[N + a], uy = tmp[2 * N + a], E = sum / (2 * r);
        st.rho[a] = (fld_t<S>)r;
        st.ux[a] = (fld_t<S>)ux;
        st.uy[a] = (fld_t<S>)uy;
        st.T[a] = (fld_t<S>)((E - 0.5 * (ux * ux + uy * uy)) / Cv);
    }
}

// The FP32-deviation form's stored pairs <-> the caller's [9][N] FP32
// planes of the same deviations, without conversion (the exchange is exact
// both ways).  Import, part 0: the f plane, and rho and u into tmp from the
// full FP64 populations d + ref, as k_import computes them; part 1: the g
// plane and the fields.
__global__ void k_import_stored(StateDev<float> st, int N, const double *consts, const float *plane, double Cv,
                               double Ux, double Uy, const int *n2o, double *tmp, int part)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    const int o = n2o[a];
    double sum = 0, jx = 0, jy = 0;
    for (int i = 0; i < NQ; ++i) {
        const float d = plane[i * N + o];
        pop_put1(st.post, i, a, N, part, (double)d);
        const double v = (double)d + consts[part * NQ + i];
        sum += v;
        if (part == 0) {
            jx += c_cx[i] * v;
            jy += c_cy[i] * v;
        }
    }
    if (part == 0) {
        tmp[a] = sum;
        tmp[N + a] = jx / sum + Ux;
        tmp[2 * N + a] = jy / sum + Uy;
    } else {
        const double r = tmp[a], ux = tmp[N + a], uy = tmp[2 * N + a], E = sum / (2 * r);
        st.rho[a] = (float)r;
        st.ux[a] = (float)ux;
        st.uy[a] = (float)uy;
        st.T[a] = (float)((E - 0.5 * (ux * ux + uy * uy)) / Cv);
    }
}

// Export: part 0 the f deviations, part 1 the g deviations.
__global__ void k_export_stored(StateDev<float> st, int N, float *plane, const int *n2o, int part)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    const int o = n2o[a];
    for (int i = 0; i < NQ; ++i) {
        float f, g;
        fg_get(st.post, i, a, N, f, g);
        plane[i * N + o] = part == 0 ? f : g;
    }
}

// part 0: the f plane into plane; part 1: the g plane (plane may be
// null) and the fields (may be null).
template <class S>
__global__ void k_export(StateDev<S> st, int N, const double *consts, double *plane, double *fields,
                         const int *n2o, int part)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    const int o = n2o[a];
    if (plane)
        for (int i = 0; i < NQ; ++i) {
            double f, g;
            fg_get(st.post, i, a, N, f, g);
            plane[i * N + o] = (part == 0 ? f : g) + consts[part * NQ + i];
        }
    if (part == 0) return;
    if (fields) {
        fields[o] = (double)st.rho[a];
        fields[N + o] = (double)st.ux[a];
        fields[2 * N + o] = (double)st.uy[a];
        fields[3 * N + o] = (double)st.T[a];
    }
}

} // namespace


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
cudaError_t launch_step(alelb_solver *s, StateDev<S> &st, KinParams<A> &K, const MapScalars &sc_in)
{
    alelb_mesh *m = s->mesh;
    const MapScalars sc = solver_map(s, sc_in);
    const int N = m->T.N;
    const bool phi = !(s->flags & (ALELB_FLAG_PHI_OFF | ALELB_FLAG_COLLIDE_OFF));
    const bool fast = s->prec != ALELB_PREC_FP64;
    const MapScalarsF sf = to_f32(sc, m->T);
    // the transformed velocities' map: arrival time, or t_{n+1/2} (flag)
    // (the departure time under ALELB_FLAG_EXACT_CHAR)
    const MapScalars scd = (s->flags & ALELB_FLAG_EXACT_CHAR) ? solver_map(s, map_scalars(m->T.mkind, m->T.mp, s->t))
                           : (s->flags & ALELB_FLAG_MIDPOINT) ? solver_map(s, map_scalars(m->T.mkind, m->T.mp, s->t + 0.5))
                                                              : sc;
    const MapScalarsF sfd = to_f32(scd, m->T);
    if (m->etype == ALELB_ELEM_Q2QUAD) { // quad.cu: propagation, moments, the two derivative passes
        const int qseq64[4] = {KT_STREAM, KT_MOMENTS, KT_DERIV1, KT_COLLIDE};
        const int qseq32[5] = {KT_FAST, KT_SLOW, KT_MOMENTS, KT_DERIV1, KT_COLLIDE};
        const int *qseq = fast ? qseq32 : qseq64;
        const int nq = fast ? 5 : 4;
        for (int q = 0; q < nq; ++q) {
            if (qseq[q] == KT_DERIV1 && !phi) continue;
            cudaEvent_t ea = nullptr, eb = nullptr;
            if (s->prof) {
                ea = get_event(s);
                eb = get_event(s);
                cudaEventRecord(ea, s->stream);
            }
            const cudaError_t qs = quad_launch(s, qseq[q], sc, scd);
            if (qs != cudaSuccess) return qs;
            if (s->prof) {
                cudaEventRecord(eb, s->stream);
                s->pending.push_back({qseq[q], ea, eb});
            }
        }
        return cudaGetLastError();
    }
    int seq[KT_N], ns = 0;
    if (fast) {
        seq[ns++] = KT_FAST;
        if (s->mlp) seq[ns++] = KT_PROPOSE;
        seq[ns++] = KT_SLOW;
        seq[ns++] = KT_MOMENTS;
    } else {
        seq[ns++] = KT_STREAM;
    }
    if (phi) seq[ns++] = KT_DERIV1;
    seq[ns++] = KT_COLLIDE;
    for (int q = 0; q < ns; ++q) {
        const int k = seq[q];
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (s->prof) {
            ea = get_event(s);
            eb = get_event(s);
            cudaEventRecord(ea, s->stream);
        }
        switch (k) {
        case KT_STREAM:
            launch_pdl(k_stream<S, A>, dim3((N + 127) / 128), dim3(128), s->stream, m->dev, m->mst, sc, scd, K, st,
                       s->d_err, s->d_stats);
            break;
        case KT_FAST:
            // one thread per node saves the nine map evaluations of a node,
            // which count on large meshes unless the map is a translation
            if (m->T.mkind == MK_NONE || m->T.mkind == MK_PLUNGE)
                launch_pdl(k_stream_fast<S, A, FAST_G, true>, dim3((N + FAST_BS - 1) / FAST_BS, NQ / FAST_G),
                           dim3(FAST_BS), s->stream, m->dev, m->mst, sfd, K, st);
            else if (N < FAST_G_NODES)
                launch_pdl(k_stream_fast<S, A, FAST_G, false>, dim3((N + FAST_BS - 1) / FAST_BS, NQ / FAST_G),
                           dim3(FAST_BS), s->stream, m->dev, m->mst, sfd, K, st);
            else
                launch_pdl(k_stream_fast<S, A, NQ, false>, dim3((N + FAST_BS - 1) / FAST_BS, 1), dim3(FAST_BS),
                           s->stream, m->dev, m->mst, sfd, K, st);
            break;
        case KT_SLOW: {
            // every block resident at once: the list is spread over all
            // blocks, and a second wave would wait for the first one's walks
            static const int per_sm = [] {
                int v = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_stream_slow<S, A>, 128, 0);
                return v > 0 ? v : 1;
            }();
            launch_pdl(k_stream_slow<S, A>, dim3(per_sm * s->n_sm), dim3(128), s->stream, m->dev, m->mst, sc, sf,
                       scd, sfd, K, st, s->d_err, s->d_stats, (const int *)(s->mlp ? s->d_prop : nullptr));
            break;
        }
        case KT_PROPOSE:
            mlp_propose(s, sfd);
            break;
        case KT_MOMENTS:
            launch_pdl(k_moments<S, A>, dim3((N + 255) / 256), dim3(256), s->stream, K, st, N, s->d_err);
            break;
        case KT_DERIV1:
            if (fast)
                launch_pdl(k_deriv1<S, A, true>, dim3((N + 255) / 256), dim3(256), s->stream, m->dev, m->mst, sc,
                           sf, st);
            else
                launch_pdl(k_deriv1<S, A, false>, dim3((N + 255) / 256), dim3(256), s->stream, m->dev, m->mst, sc,
                           sf, st);
            break;
        default:
            if (fast)
                launch_pdl(k_collide<S, A, true>, dim3((N + 127) / 128), dim3(128), s->stream, m->dev, m->mst, sc,
                           sf, K, st, s->d_err);
            else
                launch_pdl(k_collide<S, A, false>, dim3((N + 127) / 128), dim3(128), s->stream, m->dev, m->mst,
                           sc, sf, K, st, s->d_err);
        }
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
    double r = 0, jx = 0, jy = 0, pxx = 0, pxy = 0, pyy = 0, e2 = 0;
    for (int i = 0; i < NQ; ++i) {
        const double fr = s->consts[i];
        K.fref[i] = (A)fr;
        K.gref[i] = (A)s->consts[NQ + i];
        K.finf[i] = (A)(s->consts[2 * NQ + i] - fr);
        K.ginf[i] = (A)(s->consts[3 * NQ + i] - s->consts[NQ + i]);
        r += fr;
        jx += lat_cx(i) * fr;
        jy += lat_cy(i) * fr;
        pxx += lat_cx(i) * lat_cx(i) * fr;
        pxy += lat_cx(i) * lat_cy(i) * fr;
        pyy += lat_cy(i) * lat_cy(i) * fr;
        e2 += s->consts[NQ + i];
    }
    K.rho_ref = (A)r;
    K.jx_ref = (A)jx;
    K.jy_ref = (A)jy;
    K.Pxx_ref = (A)pxx;
    K.Pxy_ref = (A)pxy;
    K.Pyy_ref = (A)pyy;
    K.E2_ref = (A)e2;
    K.Ux = (A)s->U[0];
    K.Uy = (A)s->U[1];
    K.flags = (s->flags & ~FLAG_SHIFT) | shift_flag(s->U);
}


} // namespace

extern "C" alelb_status alelb_lb_init(alelb_mesh *m, const alelb_params *p, alelb_solver **out)
{
    if (!m || !p || !out) return ALELB_ERR_ARG;
    if (!(p->gamma > 1.0) || !(p->Pr > 0) || !(p->mu > 0) || !(p->rho_inf > 0) || !(p->T_inf > 0) ||
        p->precision < ALELB_PREC_FP64 || p->precision > ALELB_PREC_FP16_DEV)
        return ALELB_ERR_ARG;
    if ((p->flags & ALELB_FLAG_EXACT_CHAR) && (m->T.mkind == MK_SINE || m->T.mkind == MK_BLENDED)) {
        m->err = "lb_init: the exact characteristic needs a rigid map (none, plunge, pitch, pitch with plunge)";
        return ALELB_ERR_ARG;
    }
    if (!shift_ok(p->shift)) {
        m->err = "lb_init: the lattice shift must be finite, at most 1 per component, and exact in FP32";
        return ALELB_ERR_ARG;
    }
    alelb_solver *s = new (std::nothrow) alelb_solver();
    if (!s) return ALELB_ERR_OOM;
    *out = s;
    s->mesh = m;
    s->prec = p->precision;
    s->flags = p->flags & ~FLAG_SHIFT;
    s->U[0] = p->shift[0];
    s->U[1] = p->shift[1];
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
    // host exchange: a second stream for copies, ordered by two events
    if (st == cudaSuccess) st = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && st == cudaSuccess; ++k)
        st = cudaEventCreateWithFlags(&s->ev_copy[k], cudaEventDisableTiming);
    const int N = m->T.N;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            s->n_sm = nsm;
    }
    with_state(s, [&](auto &sx, auto &) { put_state(s->buf, sx, N, st); });
    s->d_consts = s->buf.alloc<double>(4 * NQ, st);
    s->d_scratch = s->buf.alloc<double>((size_t)22 * N, st);
    s->d_err = s->buf.alloc<int>(1, st);
    s->d_stats = s->buf.alloc<unsigned long long>(4, st);
    if (st == cudaSuccess) st = cudaMemset(s->d_stats, 0, 4 * sizeof(unsigned long long));
    s->d_out = s->buf.alloc<double>(8, st);
    if (st == cudaSuccess) st = cudaDeviceSynchronize(); // the memsets above (legacy default stream)
    if (st != cudaSuccess) return cuda_fail(s, st);
    KinParams<double> K0{};
    K0.Cv = s->Cv;
    K0.Ux = s->U[0];
    K0.Uy = s->U[1];
    K0.flags = shift_flag(s->U);
    const int ref_mode = s->prec == ALELB_PREC_FP64 ? 0 : s->prec == ALELB_PREC_FP32_DEV ? 1 : 2;
    k_kin_consts<<<1, 1, 0, s->stream>>>(K0, s->rho_inf, s->uinf[0], s->uinf[1], s->T_inf, ref_mode,
                                         s->d_consts);
    st = cudaGetLastError();
    if (st == cudaSuccess)
        st = cudaMemcpyAsync(s->consts, s->d_consts, sizeof(s->consts), cudaMemcpyDeviceToHost, s->stream);
    if (st == cudaSuccess) st = cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream);
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    fill_kin(s, s->kd);
    fill_kin(s, s->kf);
    with_state(s, [&](auto &sx, auto &) {
        k_fill_uniform<<<(N + 255) / 256, 256, 0, s->stream>>>(sx, N, s->d_consts, s->rho_inf, s->uinf[0],
                                                                s->uinf[1], s->T_inf);
    });
    st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    return ALELB_OK;
}

extern "C" void alelb_solver_destroy(alelb_solver *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    flush_prof(s);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    s->buf.release();
    if (s->copy_stream) {
        cudaStreamSynchronize(s->copy_stream);
        cudaStreamDestroy(s->copy_stream);
    }
    for (cudaEvent_t e : s->ev_copy)
        if (e) cudaEventDestroy(e);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s; // never touches the mesh: it may already be gone

}

extern "C" alelb_status alelb_lb_step(alelb_solver *s, int32_t n)
{
    if (!s || n < 0) return ALELB_ERR_ARG;
    if (!s->mesh) return ALELB_ERR_STATE;
    for (int k = 0; k < n; ++k) {
        double t1 = s->t + 1.0;
        MapScalars sc = map_scalars(s->mesh->T.mkind, s->mesh->T.mp, t1);
        cudaError_t st = with_state(s, [&](auto &sx, auto &K) { return launch_step(s, sx, K, sc); });
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
// Device state -> the caller's host arrays, in the caller's node order (the
// permutation runs on the device; each array is one copy).  Null pointers
// are skipped.
alelb_status export_to_host(alelb_solver *s, double *f, double *g, double *const fld[4])
{
    const cudaError_t st = export_enqueue(s, f, g, fld);
    if (st != cudaSuccess) return cuda_fail(s, st);
    return alelb_sync(s);
}
} // namespace

// The exchange's device side, queued without waiting (the batched exchange
// queues every case before it waits once per case).
cudaError_t alelb::export_enqueue(alelb_solver *s, double *f, double *g, double *const fld[4])
{
    alelb_mesh *m = s->mesh;
    const int N = m->T.N;
    double *dfields = s->d_scratch + (size_t)18 * N;
    const size_t plane = (size_t)9 * N * sizeof(double);
    const dim3 grid((N + 255) / 256), block(256);
    cudaError_t st = cudaSuccess;
    // the f plane first; its copy on the copy stream overlaps the g half's
    // kernel on the solver's stream (every kernel stays on that stream)
    if (f) {
        with_state(s, [&](auto &sx, auto &) {
            k_export<<<grid, block, 0, s->stream>>>(sx, N, s->d_consts, s->d_scratch, nullptr, m->d_n2o, 0);
        });
        st = cudaGetLastError();
        if (st == cudaSuccess) st = cudaEventRecord(s->ev_copy[0], s->stream);
        if (st == cudaSuccess) st = cudaStreamWaitEvent(s->copy_stream, s->ev_copy[0], 0);
        if (st == cudaSuccess) st = cudaMemcpyAsync(f, s->d_scratch, plane, cudaMemcpyDeviceToHost, s->copy_stream);
        if (st == cudaSuccess) st = cudaEventRecord(s->ev_copy[1], s->copy_stream);
    }
    if (st == cudaSuccess && (g || fld)) {
        with_state(s, [&](auto &sx, auto &) {
            k_export<<<grid, block, 0, s->stream>>>(sx, N, s->d_consts, g ? s->d_scratch + (size_t)9 * N : nullptr,
                                                    fld ? dfields : nullptr, m->d_n2o, 1);
        });
        st = cudaGetLastError();
    }
    if (st == cudaSuccess && g)
        st = cudaMemcpyAsync(g, s->d_scratch + (size_t)9 * N, plane, cudaMemcpyDeviceToHost, s->stream);
    for (int c = 0; c < 4 && st == cudaSuccess; ++c)
        if (fld && fld[c])
            st = cudaMemcpyAsync(fld[c], dfields + (size_t)c * N, (size_t)N * sizeof(double),
                                 cudaMemcpyDeviceToHost, s->stream);
    if (st == cudaSuccess && f) st = cudaStreamWaitEvent(s->stream, s->ev_copy[1], 0); // the f copy too
    return st;
}

extern "C" alelb_status alelb_moments(alelb_solver *s, double *rho, double *ux, double *uy, double *T)
{
    if (!s) return ALELB_ERR_ARG;
    double *const fld[4] = {rho, ux, uy, T};
    return export_to_host(s, nullptr, nullptr, fld);
}

extern "C" alelb_status alelb_get_pops(alelb_solver *s, double *f, double *g)
{
    if (!s) return ALELB_ERR_ARG;
    return export_to_host(s, f, g, nullptr);
}

extern "C" alelb_status alelb_set_pops(alelb_solver *s, const double *f, const double *g,
                                       const double *rho, const double *ux, const double *uy,
                                       const double *T, double t)
{
    if (!s || !f || !g) return ALELB_ERR_ARG;
    cudaError_t st = import_enqueue(s, f, g, rho, ux, uy, T);
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream); // the caller's arrays are free again
    if (st != cudaSuccess) return cuda_fail(s, st);
    s->t = t;
    return ALELB_OK;
}

cudaError_t alelb::import_enqueue(alelb_solver *s, const double *f, const double *g, const double *rho,
                                  const double *ux, const double *uy, const double *T)
{
    const int N = s->mesh->T.N;
    const bool have = rho && ux && uy && T;
    const size_t plane = (size_t)9 * N * sizeof(double);
    double *dfields = s->d_scratch + (size_t)18 * N; // the fields, or the f half's rho and u
    // f on the solver's stream; g (and the fields) on the copy stream once f
    // is in, so that the f half's kernel overlaps the g copy
    cudaError_t st = cudaMemcpyAsync(s->d_scratch, f, plane, cudaMemcpyHostToDevice, s->stream);
    if (st == cudaSuccess) st = cudaEventRecord(s->ev_copy[0], s->stream);
    if (st == cudaSuccess) st = cudaStreamWaitEvent(s->copy_stream, s->ev_copy[0], 0);
    if (st == cudaSuccess)
        st = cudaMemcpyAsync(s->d_scratch + (size_t)9 * N, g, plane, cudaMemcpyHostToDevice, s->copy_stream);
    const double *fl[4] = {rho, ux, uy, T};
    for (int c = 0; c < 4 && have && st == cudaSuccess; ++c)
        st = cudaMemcpyAsync(dfields + (size_t)c * N, fl[c], (size_t)N * sizeof(double), cudaMemcpyHostToDevice,
                             s->copy_stream);
    if (st == cudaSuccess) st = cudaEventRecord(s->ev_copy[1], s->copy_stream);
    if (st != cudaSuccess) return st;
    const dim3 grid((N + 255) / 256), block(256);
    with_state(s, [&](auto &sx, auto &) {
        k_import<<<grid, block, 0, s->stream>>>(sx, N, s->d_consts, s->d_scratch, dfields, have, s->Cv, s->U[0],
                                                s->U[1], s->mesh->d_n2o, dfields, 0);
    });
    st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaStreamWaitEvent(s->stream, s->ev_copy[1], 0);
    if (st == cudaSuccess)
        with_state(s, [&](auto &sx, auto &) {
            k_import<<<grid, block, 0, s->stream>>>(sx, N, s->d_consts, s->d_scratch + (size_t)9 * N, dfields,
                                                    have, s->Cv, s->U[0], s->U[1], s->mesh->d_n2o, dfields, 1);
        });
    if (st == cudaSuccess) st = cudaGetLastError();
    return st;
}

// The FP32-deviation form's exchange in its stored form: half the bytes of
// the FP64 exchange, and exact.  The planes sit in the FP64 scratch as
// floats ([0, 9N) f, [9N, 18N) g), clear of the fields area at 18N doubles.
cudaError_t alelb::export_stored_enqueue(alelb_solver *s, float *f, float *g)
{
    alelb_mesh *m = s->mesh;
    const int N = m->T.N;
    float *pf = reinterpret_cast<float *>(s->d_scratch), *pg = pf + (size_t)9 * N;
    const size_t plane = (size_t)9 * N * sizeof(float);
    const dim3 grid((N + 255) / 256), block(256);
    // the f copy on the copy stream overlaps the g kernel (as export_enqueue)
    k_export_stored<<<grid, block, 0, s->stream>>>(s->sf, N, pf, m->d_n2o, 0);
    cudaError_t st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaEventRecord(s->ev_copy[0], s->stream);
    if (st == cudaSuccess) st = cudaStreamWaitEvent(s->copy_stream, s->ev_copy[0], 0);
    if (st == cudaSuccess) st = cudaMemcpyAsync(f, pf, plane, cudaMemcpyDeviceToHost, s->copy_stream);
    if (st == cudaSuccess) st = cudaEventRecord(s->ev_copy[1], s->copy_stream);
    if (st == cudaSuccess) {
        k_export_stored<<<grid, block, 0, s->stream>>>(s->sf, N, pg, m->d_n2o, 1);
        st = cudaGetLastError();
    }
    if (st == cudaSuccess) st = cudaMemcpyAsync(g, pg, plane, cudaMemcpyDeviceToHost, s->stream);
    if (st == cudaSuccess) st = cudaStreamWaitEvent(s->stream, s->ev_copy[1], 0);
    return st;
}

cudaError_t alelb::import_stored_enqueue(alelb_solver *s, const float *f, const float *g)
{
    const int N = s->mesh->T.N;
    float *pf = reinterpret_cast<float *>(s->d_scratch), *pg = pf + (size_t)9 * N;
    double *tmp = s->d_scratch + (size_t)18 * N;
    const size_t plane = (size_t)9 * N * sizeof(float);
    cudaError_t st = cudaMemcpyAsync(pf, f, plane, cudaMemcpyHostToDevice, s->stream);
    if (st == cudaSuccess) st = cudaEventRecord(s->ev_copy[0], s->stream);
    if (st == cudaSuccess) st = cudaStreamWaitEvent(s->copy_stream, s->ev_copy[0], 0);
    if (st == cudaSuccess) st = cudaMemcpyAsync(pg, g, plane, cudaMemcpyHostToDevice, s->copy_stream);
    if (st == cudaSuccess) st = cudaEventRecord(s->ev_copy[1], s->copy_stream);
    if (st != cudaSuccess) return st;
    const dim3 grid((N + 255) / 256), block(256);
    k_import_stored<<<grid, block, 0, s->stream>>>(s->sf, N, s->d_consts, pf, s->Cv, s->U[0], s->U[1],
                                                  s->mesh->d_n2o, tmp, 0);
    st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaStreamWaitEvent(s->stream, s->ev_copy[1], 0);
    if (st == cudaSuccess) {
        k_import_stored<<<grid, block, 0, s->stream>>>(s->sf, N, s->d_consts, pg, s->Cv, s->U[0], s->U[1],
                                                      s->mesh->d_n2o, tmp, 1);
        st = cudaGetLastError();
    }
    return st;
}

extern "C" alelb_status alelb_get_pops_stored(alelb_solver *s, float *f, float *g)
{
    if (!s || !f || !g) return ALELB_ERR_ARG;
    if (s->prec != ALELB_PREC_FP32_DEV) {
        s->err = "get_pops_stored: the solver is not of the FP32-deviation form";
        return ALELB_ERR_ARG;
    }
    const cudaError_t st = export_stored_enqueue(s, f, g);
    if (st != cudaSuccess) return cuda_fail(s, st);
    return alelb_sync(s);
}

extern "C" alelb_status alelb_set_pops_stored(alelb_solver *s, const float *f, const float *g, double t)
{
    if (!s || !f || !g) return ALELB_ERR_ARG;
    if (s->prec != ALELB_PREC_FP32_DEV) {
        s->err = "set_pops_stored: the solver is not of the FP32-deviation form";
        return ALELB_ERR_ARG;
    }
    cudaError_t st = import_stored_enqueue(s, f, g);
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream); // the caller's arrays are free again
    if (st != cudaSuccess) return cuda_fail(s, st);
    s->t = t;
    return ALELB_OK;
}

namespace {
// A caller's device array for the zero-copy exchange: device (or managed)
// memory of the mesh's device, else an argument error (so that no kernel
// is ever handed a host address).
bool on_mesh_device(alelb_solver *s, const void *p, const char *what)
{
    cudaPointerAttributes at{};
    const cudaError_t st = cudaPointerGetAttributes(&at, p);
    if (st != cudaSuccess) cudaGetLastError(); // clears the error of an unknown pointer
    const bool ok = st == cudaSuccess &&
                    (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
                    at.device == s->mesh->device;
    if (!ok) s->err = std::string(what) + ": not device memory of the mesh's device";
    return ok;
}
} // namespace

extern "C" alelb_status alelb_get_pops_dev(alelb_solver *s, double *f, double *g)
{
    if (!s || !f || !g) return ALELB_ERR_ARG;
    if (!on_mesh_device(s, f, "get_pops_dev") || !on_mesh_device(s, g, "get_pops_dev")) return ALELB_ERR_ARG;
    alelb_mesh *m = s->mesh;
    const int N = m->T.N;
    const dim3 grid((N + 255) / 256), block(256);
    with_state(s, [&](auto &sx, auto &) {
        k_export<<<grid, block, 0, s->stream>>>(sx, N, s->d_consts, f, nullptr, m->d_n2o, 0);
        k_export<<<grid, block, 0, s->stream>>>(sx, N, s->d_consts, g, nullptr, m->d_n2o, 1);
    });
    const cudaError_t st = cudaGetLastError();
    if (st != cudaSuccess) return cuda_fail(s, st);
    return alelb_sync(s);
}

extern "C" alelb_status alelb_set_pops_dev(alelb_solver *s, const double *f, const double *g, double t)
{
    if (!s || !f || !g) return ALELB_ERR_ARG;
    if (!on_mesh_device(s, f, "set_pops_dev") || !on_mesh_device(s, g, "set_pops_dev")) return ALELB_ERR_ARG;
    const int N = s->mesh->T.N;
    double *tmp = s->d_scratch + (size_t)18 * N;
    const dim3 grid((N + 255) / 256), block(256);
    with_state(s, [&](auto &sx, auto &) {
        k_import<<<grid, block, 0, s->stream>>>(sx, N, s->d_consts, f, nullptr, 0, s->Cv, s->U[0], s->U[1],
                                                s->mesh->d_n2o, tmp, 0);
        k_import<<<grid, block, 0, s->stream>>>(sx, N, s->d_consts, g, nullptr, 0, s->Cv, s->U[0], s->U[1],
                                                s->mesh->d_n2o, tmp, 1);
    });
    cudaError_t st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    s->t = t;
    return ALELB_OK;
}

extern "C" alelb_status alelb_moments_dev(alelb_solver *s, double *rho, double *ux, double *uy, double *T)
{
    if (!s) return ALELB_ERR_ARG;
    double *const out[4] = {rho, ux, uy, T};
    for (double *p : out)
        if (p && !on_mesh_device(s, p, "moments_dev")) return ALELB_ERR_ARG;
    alelb_mesh *m = s->mesh;
    const int N = m->T.N;
    double *dfields = s->d_scratch + (size_t)18 * N;
    with_state(s, [&](auto &sx, auto &) {
        k_export<<<(N + 255) / 256, 256, 0, s->stream>>>(sx, N, s->d_consts, nullptr, dfields, m->d_n2o, 1);
    });
    cudaError_t st = cudaGetLastError();
    for (int c = 0; c < 4 && st == cudaSuccess; ++c)
        if (out[c])
            st = cudaMemcpyAsync(out[c], dfields + (size_t)c * N, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice,
                                 s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    return alelb_sync(s);
}

extern "C" alelb_status alelb_forces(alelb_solver *s, double out[6])
{
    if (!s || !out) return ALELB_ERR_ARG;
    alelb_mesh *m = s->mesh;
    MapScalars sc = map_scalars(m->T.mkind, m->T.mp, s->t);
    if (m->nw > 0 && m->etype == ALELB_ELEM_Q2QUAD) {
        quad_forces(s, sc);
    } else if (m->nw > 0) {
        with_state(s, [&](auto &sx, auto &) {
            k_forces<<<1, 256, 0, s->stream>>>(m->dev, m->mst, sc, sx, m->d_wedges, m->nw, s->mu, s->Cv,
                                               s->d_out);
        });
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

extern "C" alelb_status alelb_locate(alelb_solver *s, double t, int32_t use_cache, int32_t *elem,
                                     int8_t *kind)
{
    if (!s || !elem || !kind) return ALELB_ERR_ARG;
    const int *cache = nullptr;
    if (use_cache) {
        if (s->prec == ALELB_PREC_FP64) {
            s->err = "locate: the cached fast decisions exist in the deviation forms only";
            return ALELB_ERR_ARG;
        }
        with_state(s, [&](auto &sx, auto &) { cache = sx.cache; });
    }
    alelb_mesh *m = s->mesh;
    const int N = m->T.N;
    const MapScalars sc = solver_map(s, map_scalars(m->T.mkind, m->T.mp, t));
    int *de = (int *)s->d_scratch;
    int8_t *dk = (int8_t *)(s->d_scratch + (size_t)9 * N);
    if (m->etype == ALELB_ELEM_Q2QUAD) // no fast path: the walk decides every population
        quad_locate(s, sc, de, dk);
    else
        k_locate<<<(N + 127) / 128, 128, 0, s->stream>>>(m->dev, m->mst, sc, to_f32(sc, m->T), s->flags, cache,
                                                         de, dk, s->d_err);
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
            int o = m->T.node_new2old[a];
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
    double sz = s->prec == ALELB_PREC_FP64 ? 8.0 : s->prec == ALELB_PREC_FP32_DEV ? 4.0 : 2.0;
    out[0] = m->T.N;
    out[1] = m->T.E;
    out[2] = sz;
    out[3] = 0;
    out[4] = m->T.n_wall_nodes;
    out[5] = s->prec;
    out[6] = m->nw;
    unsigned long long walks = 0;
    cudaError_t st = cudaMemcpyAsync(&walks, s->d_stats, sizeof(walks), cudaMemcpyDeviceToHost, s->stream);
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) return cuda_fail(s, st);
    out[7] = (double)walks;
    return ALELB_OK;
}

extern "C" const char *alelb_last_error(alelb_solver *s) { return s ? s->err.c_str() : "null solver"; }

// ============================================================================
// One FP64 step that allocates nothing (alelb_lb_step_noalloc).
//
// For callers that cannot allocate device memory once they are running: a
// host application whose device memory is entirely pre-reserved by its own
// allocator, or a coupling loop that must not call cudaMalloc/cudaFree
// (cudaFree waits for the whole device).  The caller passes the state; the
// step's scratch -- the streamed populations, Q'_xxx, Q'_yyy, mu/(rho T),
// D_x, D_y, the reference/far-field constants and the error word -- lives
// in the file-scope array below, which every GPU that loads this library
// holds until the process exits.  All calls share it: it keeps the last
// call's contents, the error word is cleared at the start of each call, and
// calls that overlap on the GPU race on it.
// ============================================================================
#define ALELB_NOALLOC_MAX_NODES 131072
namespace {
constexpr size_t NOALLOC_SCRATCH_DOUBLES = (size_t)23 * ALELB_NOALLOC_MAX_NODES + 64;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];
double *g_noalloc_ptr[64] = {nullptr}; // device address of the array, per device
// A new mesh on a device drops the cached address: after a device reset
// (which frees every table, so meshes must be created again) the next call
// asks the runtime again instead of using an address of the old context.
void forget_noalloc_scratch(int dev)
{
    if (dev >= 0 && dev < 64) g_noalloc_ptr[dev] = nullptr;
}
}

extern "C" alelb_status alelb_lb_step_noalloc(alelb_mesh *m, const alelb_params *p, double t,
                                              double *post, double *rho, double *ux, double *uy,
                                              double *T)
{
    if (!m || !p || !post || !rho || !ux || !uy || !T) return ALELB_ERR_ARG;
    if (p->precision != ALELB_PREC_FP64 || !(p->gamma > 1.0) || !(p->Pr > 0) || !(p->mu > 0) ||
        !(p->rho_inf > 0) || !(p->T_inf > 0)) {
        m->err = "lb_step_noalloc: needs FP64 precision and positive fluid parameters";
        return ALELB_ERR_ARG;
    }
    if ((p->flags & ALELB_FLAG_EXACT_CHAR) && (m->T.mkind == MK_SINE || m->T.mkind == MK_BLENDED)) {
        m->err = "lb_step_noalloc: the exact characteristic needs a rigid map (none, plunge, pitch, pitch with plunge)";
        return ALELB_ERR_ARG;
    }
    if (!shift_ok(p->shift)) {
        m->err = "lb_step_noalloc: the lattice shift must be finite, at most 1 per component, and exact in FP32";
        return ALELB_ERR_ARG;
    }
    if (m->etype != ALELB_ELEM_P2TRI) {
        m->err = "lb_step_noalloc: 6-node triangle meshes only";
        return ALELB_ERR_ARG;
    }
    const int N = m->T.N;
    if (N > ALELB_NOALLOC_MAX_NODES) {
        m->err = "lb_step_noalloc: the mesh has " + std::to_string(N) + " nodes; at most " +
                 std::to_string(ALELB_NOALLOC_MAX_NODES) + " fit the static scratch";
        return ALELB_ERR_ARG;
    }
    for (int a = 0; a < N; ++a)
        if (m->T.node_new2old[a] != a) {
            m->err = "lb_step_noalloc: the mesh must be created with ALELB_RENUMBER_NONE";
            return ALELB_ERR_ARG;
        }
    int dev = 0;
    cudaError_t st = cudaGetDevice(&dev);
    if (st != cudaSuccess || dev < 0 || dev >= 64) {
        m->err = "lb_step_noalloc: no usable current device";
        return ALELB_ERR_CUDA;
    }
    if (dev != m->device) {
        m->err = "lb_step_noalloc: the current device (" + std::to_string(dev) +
                 ") is not the one the mesh was created on (" + std::to_string(m->device) + ")";
        return ALELB_ERR_ARG;
    }
    // set-up, once per device: the host-side name of the array is not a
    // device address; ask the runtime for it with this device current
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        st = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (st != cudaSuccess || !ptr) {
            m->err = std::string("lb_step_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(st);
            return ALELB_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = (double *)ptr;
    }
    double *base = g_noalloc_ptr[dev];
    cudaStream_t stream = (cudaStream_t)p->stream;
    StateDev<double> sd{};
    sd.post = post;
    sd.rho = rho;
    sd.ux = ux;
    sd.uy = uy;
    sd.T = T;
    sd.str = base;
    sd.Qx = base + (size_t)18 * N;
    sd.Qy = sd.Qx + N;
    sd.mrt = sd.Qy + N;
    sd.Dx = sd.mrt + N;
    sd.Dy = sd.Dx + N;
    double *consts = base + (size_t)23 * ALELB_NOALLOC_MAX_NODES;     // 36 doubles
    int *err = (int *)(consts + 4 * NQ);                              // inside the last 64
    KinParams<double> K{};
    K.Cv = 1.0 / (p->gamma - 1.0);
    K.Ux = p->shift[0];
    K.Uy = p->shift[1];
    K.flags = shift_flag(p->shift);
    k_kin_consts<<<1, 1, 0, stream>>>(K, p->rho_inf, p->u_inf[0], p->u_inf[1], p->T_inf, 0, consts);
    double hc[4 * NQ];
    st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaMemsetAsync(err, 0, sizeof(int), stream);
    if (st == cudaSuccess) st = cudaMemcpyAsync(hc, consts, sizeof(hc), cudaMemcpyDeviceToHost, stream);
    if (st == cudaSuccess) st = cudaStreamSynchronize(stream);
    if (st != cudaSuccess) {
        m->err = cudaGetErrorString(st);
        return ALELB_ERR_CUDA;
    }
    K.Cp = K.Cv + 1.0;
    K.mu = p->mu;
    K.Pr = p->Pr;
    K.rho_ref = 0.0;
    K.E2_ref = 0.0;
    for (int i = 0; i < NQ; ++i) {
        K.fref[i] = 0.0;
        K.gref[i] = 0.0;
        K.finf[i] = hc[2 * NQ + i];
        K.ginf[i] = hc[3 * NQ + i];
    }
    K.flags = (p->flags & ~FLAG_SHIFT) | shift_flag(p->shift);
    MapScalars sc = with_shift(map_scalars(m->T.mkind, m->T.mp, t + 1.0), p->shift);
    const MapScalars scd =
        (p->flags & ALELB_FLAG_EXACT_CHAR) ? with_shift(map_scalars(m->T.mkind, m->T.mp, t), p->shift)
        : (p->flags & ALELB_FLAG_MIDPOINT) ? with_shift(map_scalars(m->T.mkind, m->T.mp, t + 0.5), p->shift)
                                           : sc;
    k_stream<double, double><<<(N + 127) / 128, 128, 0, stream>>>(m->dev, m->mst, sc, scd, K, sd, err, nullptr);
    if (!(p->flags & (ALELB_FLAG_PHI_OFF | ALELB_FLAG_COLLIDE_OFF)))
        k_deriv1<double, double, false><<<(N + 255) / 256, 256, 0, stream>>>(m->dev, m->mst, sc, to_f32(sc, m->T), sd);
    k_collide<double, double, false><<<(N + 127) / 128, 128, 0, stream>>>(m->dev, m->mst, sc, to_f32(sc, m->T), K,
                                                                        sd, err);
    int herr = 0;
    st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (st == cudaSuccess) st = cudaStreamSynchronize(stream);
    if (st != cudaSuccess) {
        m->err = cudaGetErrorString(st);
        return ALELB_ERR_CUDA;
    }
    if (herr & ERR_LOCATE) {
        m->err = "lb_step_noalloc: element walk exceeded its step limit";
        return ALELB_ERR_LOCATE;
    }
    if (herr & ERR_NONFINITE) {
        m->err = "lb_step_noalloc: non-finite or non-positive density or temperature";
        return ALELB_ERR_NONFINITE;
    }
    return ALELB_OK;
}
