// batch.cu -- the batched step over many independent cases (alelb_batch_*
// in include/alelb.h).
//
// Every phase of the time step is one launch over all cases.  Node-parallel
// phases number their thread blocks through a prefix sum of the cases' tile
// counts (off[c] = first tile of case c, a tile being one block of nodes);
// block b finds its case with one ballot over the B <= 32 offsets, copies
// the case's descriptor (mesh tables, map statics, kinetic constants, state
// pointers) into shared memory and runs the same per-node code as the
// single-case kernels.  The exact part of the propagation takes every
// case's work list as one numbered list dealt out over the grid.  Map scalars of each (step, case) are computed on the
// host, exactly as for a single solver, and staged per chunk of steps; a
// chunk's launches are captured once into a CUDA graph and replayed.  The
// cases may also run as two or four groups, each group's launches on a
// stream of its own (branches of the chunk's graph), so that the groups'
// kernels share the SMs.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"

using namespace alelb;

namespace alelb {
cudaError_t batch_fe_tables() { return upload_fe_tables(); }
} // namespace alelb

namespace {

constexpr int BATCH_MAX = 32;
constexpr int CHUNK_MAX = 64; // steps per captured graph
constexpr int N_BS = 3;       // block sizes 64, 128, 256
// flag of the directions-per-thread choice (FP32 form): kb_fast_fused
constexpr int FAST_FUSED = 256;
// flags of the same choice word for the case groups of a graph-mode step:
// the cases in two or four groups, each group's phase kernels on a stream
// of its own (captured as branches of the chunk's graph); PIPELINED (x 1
// or 2) also orders each group's propagation after the previous group's
// latest one, so that one group's propagation runs beside the other
// groups' later phases
constexpr int TWO_GROUPS = 512, FOUR_GROUPS = 1024, PIPELINED = 4096;
constexpr int GROUPS_MAX = 8; // 2 or 4 in graph mode; 8 for the pipelined host step

template <class S, class A> struct CaseDev {
    MeshDev M;
    MapStatic MS;
    KinParams<A> K;
    StateDev<S> st;
    int *err;
    unsigned long long *stats;
};

// Case of tile `tile`: the number of cases whose tile range ends at or
// before it.  All 32 lanes of the warp take part.
__device__ __forceinline__ int tile_case(const int *__restrict__ off, int B, int tile)
{
    const int lane = threadIdx.x & 31;
    const int v = lane < B ? __ldg(off + lane + 1) : INT_MAX;
    return __popc(__ballot_sync(0xffffffffu, tile >= v));
}

template <class T> __device__ __forceinline__ void copy_words(void *dst, const T *src)
{
    static_assert(sizeof(T) % 4 == 0, "descriptor size");
    const int *s = reinterpret_cast<const int *>(src);
    for (int w = threadIdx.x; w < (int)(sizeof(T) / 4); w += blockDim.x) ((int *)dst)[w] = __ldg(s + w);
}

// Shared-memory copies of one case's descriptor and its map scalars.
template <class S, class A> struct SharedCase {
    __align__(16) unsigned char c[sizeof(CaseDev<S, A>)];
    __align__(16) unsigned char sc[sizeof(MapScalars)];
    __align__(16) unsigned char sf[sizeof(MapScalarsF)];
    __device__ const CaseDev<S, A> &C() const { return *reinterpret_cast<const CaseDev<S, A> *>(c); }
    __device__ const MapScalars &SC() const { return *reinterpret_cast<const MapScalars *>(sc); }
    __device__ const MapScalarsF &SF() const { return *reinterpret_cast<const MapScalarsF *>(sf); }
    __device__ void load(const CaseDev<S, A> *cases, const MapScalars *scs, const MapScalarsF *sfs, int k)
    {
        copy_words(c, cases + k);
        if (scs) copy_words(sc, scs + k);
        if (sfs) copy_words(sf, sfs + k);
    }
};

template <class S, class A>
__global__ void __launch_bounds__(256) kb_stream(const CaseDev<S, A> *__restrict__ cases,
                                                 const int *__restrict__ off, int B,
                                                 const MapScalars *__restrict__ sc, int count)
{
    wait_prior_grid();
    __shared__ SharedCase<S, A> sh;
    const int c = tile_case(off, B, blockIdx.x);
    sh.load(cases, sc, nullptr, c);
    __syncthreads();
    const CaseDev<S, A> &C = sh.C();
    const int a = (blockIdx.x - __ldg(off + c)) * blockDim.x + threadIdx.x;
    if (a < C.M.N) stream_plain_node(C.M, C.MS, sh.SC(), sh.SC(), C.K, C.st, C.err, count ? C.stats : nullptr, a);
}

// G directions per thread (grid y: 9 / G groups), chosen by the tuner:
// one map evaluation per thread, fewer and longer load chains as G grows.
template <class S, class A, int G>
__global__ void __launch_bounds__(256) kb_fast(const CaseDev<S, A> *__restrict__ cases,
                                               const int *__restrict__ off, int B,
                                               const MapScalarsF *__restrict__ sf)
{
    wait_prior_grid();
    __shared__ SharedCase<S, A> sh;
    const int c = tile_case(off, B, blockIdx.x);
    sh.load(cases, nullptr, sf, c);
    __syncthreads();
    const CaseDev<S, A> &C = sh.C();
    stream_fast_group<G>(C.M, C.MS, sh.SF(), C.K, C.st, (blockIdx.x - __ldg(off + c)) * blockDim.x + threadIdx.x);
}

// The exact path over the work lists of all cases as one list, numbered
// case by case and, within a case, direction by direction and then the
// listed wall nodes: block-local prefix sums of the B x 10 segment counts, one population per thread, its
// segment by binary search; the case descriptor is read from global memory
// (the populations of a warp mostly share one case and one direction).
template <class S, class A>
__global__ void __launch_bounds__(256) kb_slow(const CaseDev<S, A> *__restrict__ cases, int B,
                                               const MapScalars *__restrict__ sc,
                                               const MapScalarsF *__restrict__ sf, int count)
{
    wait_prior_grid();
    constexpr int NS = NQ + 1; // segments per case: nine directions, then wall nodes
    __shared__ unsigned pre[BATCH_MAX * NS + 1];
    const int nseg = B * NS;
    if (threadIdx.x < 32) {
        // lane l sums the segments of case l, then a warp scan
        const int lane = threadIdx.x;
        unsigned loc[NS];
        unsigned s = 0, npop = 0;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            loc[i] = lane < B ? cases[lane].st.wcount[i] : 0u;
            s += loc[i];
            if (i < NQ) npop += loc[i];
        }
        unsigned incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < B) {
            unsigned run = incl - s;
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                pre[lane * NS + i] = run;
                run += loc[i];
            }
            if (lane == B - 1) pre[nseg] = run;
            if (count && npop && blockIdx.x == 0 && cases[lane].stats)
                atomicAdd(cases[lane].stats, (unsigned long long)npop);
        }
    }
    __syncthreads();
    const unsigned total = pre[nseg];
    for (unsigned w = spread_first(); w < total; w += spread_stride()) {
        int lo = 0, hi = nseg - 1; // last segment with pre <= w
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const int c = lo / NS, i = lo % NS;
        const CaseDev<S, A> &C = cases[c];
        const int entry = C.st.work[(size_t)i * C.M.N + (w - pre[lo])];
        if (i < NQ) {
            stream_slow_item(C.M, C.MS, sc[c], sf[c], sc[c], sf[c], C.K, C.st, C.err, entry);
        } else {
            const unsigned mask = C.st.wmask[entry] & WMASK_DIRS;
            if (count && C.stats) atomicAdd(C.stats, (unsigned long long)__popc(mask));
            stream_bc_node<S, A>(C.M, C.MS, sc[c], sf[c], C.K, C.st, entry,
                                 fast_map(C.MS, sf[c], entry, C.M.Xf[entry]), mask);
        }
    }
}

template <class S, class A>
__global__ void __launch_bounds__(256) kb_moments(const CaseDev<S, A> *__restrict__ cases,
                                                  const int *__restrict__ off, int B)
{
    wait_prior_grid();
    __shared__ SharedCase<S, A> sh;
    const int c = tile_case(off, B, blockIdx.x);
    sh.load(cases, nullptr, nullptr, c);
    __syncthreads();
    const CaseDev<S, A> &C = sh.C();
    const int a = (blockIdx.x - __ldg(off + c)) * blockDim.x + threadIdx.x;
    if (a <= NQ) C.st.wcount[a] = 0u; // the case's work list has been consumed
    if (a < C.M.N) moments_node(C.K, C.st, C.M.N, C.err, a);
}

// After the fused propagation (kb_fast_fused): the moments of the nodes it
// listed as pending.  All cases' lists form one numbering (a warp scan of
// the B counts into shared memory, the case of an entry by binary search),
// dealt out over the whole grid; the case descriptors are read from global
// memory.  The pending list itself is emptied by the collision kernel, once
// every reader is done.
template <class S, class A>
__global__ void __launch_bounds__(256) kb_moments_pending(const CaseDev<S, A> *__restrict__ cases, int B)
{
    wait_prior_grid();
    __shared__ unsigned pre[BATCH_MAX + 1];
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned v = lane < B ? cases[lane].st.wcount[SEG_PENDING] : 0u;
        unsigned incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane < B) pre[lane + 1] = incl;
        if (lane == 0) pre[0] = 0u;
    }
    __syncthreads();
    const unsigned total = pre[B];
    const unsigned stride = gridDim.x * blockDim.x, first = blockIdx.x * blockDim.x + threadIdx.x;
    for (unsigned w = first; w < total; w += stride) {
        int lo = 0, hi = B - 1; // last case with pre <= w
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const CaseDev<S, A> &C = cases[lo];
        const int N = C.M.N;
        moments_node(C.K, C.st, N, C.err, C.st.work[(size_t)SEG_PENDING * N + (w - pre[lo])]);
    }
    if (first < (unsigned)(B * (NQ + 1))) // every case's exact-path list has been consumed
        cases[first / (NQ + 1)].st.wcount[first % (NQ + 1)] = 0u;
}

// The propagation of the FP32 form fused with the moments: a block holds
// the NQ / G direction groups of a tile of T nodes (group-uniform warps),
// each thread settles its G populations as kb_fast does and leaves the
// settled pairs in shared memory; then (after a block barrier when G < 9)
// one thread per node computes the node's moments from them, exactly as the
// moments kernel would, unless a population of the node went to the exact
// path or its wall condition: then the node goes to the pending list, which
// kb_moments_pending works through.  The nodes the exact path never touches
// are read once per step instead of twice.
template <int G, int T>
__global__ void __launch_bounds__(T *NQ / G) kb_fast_fused(const CaseDev<float, float> *__restrict__ cases,
                                                           const int *__restrict__ off, int B,
                                                           const MapScalarsF *__restrict__ sf)
{
    static_assert(NQ % G == 0 && T % 32 == 0, "group-uniform warps");
    constexpr int NG = NQ / G;
    wait_prior_grid();
    __shared__ SharedCase<float, float> sh;
    __shared__ float fs[NQ][T], gs[NQ][T];
    __shared__ int pend[NG][T];
    const int c = tile_case(off, B, blockIdx.x);
    sh.load(cases, nullptr, sf, c);
    __syncthreads();
    const CaseDev<float, float> &C = sh.C();
    const MeshDev &M = C.M;
    const StateDev<float> &st = C.st;
    const int tx = threadIdx.x % T, grp = threadIdx.x / T, i0 = G * grp;
    const int a = (blockIdx.x - __ldg(off + c)) * T + tx;
    int code[G];
#pragma unroll
    for (int j = 0; j < G; ++j) code[j] = 0;
    if (a < M.N) {
        int cc[G];
#pragma unroll
        for (int j = 0; j < G; ++j) cc[j] = st.cache[(i0 + j) * M.N + a];
        const float bd = M.bdist[a];
        const float4 Xf = M.Xf[a];
        FastMap F = fast_map(C.MS, sh.SF(), a, Xf);
        if (C.K.flags & (FLAG_LITERAL_VG | FLAG_EXACT_CHAR)) F.ok = false;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            float fo = 0.f, go = 0.f;
            code[j] = stream_fast_pop(M, C.K, st, a, i0 + j, F, Xf, bd, cc[j], fo, go);
            fs[i0 + j][tx] = fo;
            gs[i0 + j][tx] = go;
        }
    }
    int any = 0;
#pragma unroll
    for (int j = 0; j < G; ++j) any |= code[j];
    if (__any_sync(0xffffffffu, any != 0)) {
#pragma unroll
        for (int j = 0; j < G; ++j) append_pop(st, a, M.N, i0 + j, code[j]);
    }
    pend[grp][tx] = any;
    // every group's pairs and wall bits of the tile are in; with one thread
    // per node (G = 9) a thread reads back only what it wrote itself
    if (NG > 1) __syncthreads();
    int p = 0;
    if (grp == 0 && a < M.N) {
#pragma unroll
        for (int q = 0; q < NG; ++q) p |= pend[q][tx];
    }
    // pending nodes to the moments kernel's list, one atomic per warp
    const unsigned pm = __ballot_sync(0xffffffffu, p != 0);
    if (pm) {
        const unsigned lane = threadIdx.x & 31u;
        const int leader = __ffs(pm) - 1;
        unsigned base = 0;
        if ((int)lane == leader) base = atomicAdd(st.wcount + SEG_PENDING, (unsigned)__popc(pm));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (p) st.work[(size_t)SEG_PENDING * M.N + base + __popc(pm & ((1u << lane) - 1u))] = a;
    }
    if (grp == 0 && a < M.N) {
        if (!p) {
            float f[NQ], g[NQ];
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                f[i] = fs[i][tx];
                g[i] = gs[i][tx];
            }
            moments_store(C.K, st, C.err, a, f, g);
        }
    }
}

template <class S, class A, bool FAST>
__global__ void __launch_bounds__(256) kb_deriv1(const CaseDev<S, A> *__restrict__ cases,
                                                 const int *__restrict__ off, int B,
                                                 const MapScalars *__restrict__ sc,
                                                 const MapScalarsF *__restrict__ sf)
{
    wait_prior_grid();
    __shared__ SharedCase<S, A> sh;
    const int c = tile_case(off, B, blockIdx.x);
    sh.load(cases, sc, sf, c);
    __syncthreads();
    const CaseDev<S, A> &C = sh.C();
    const int a = (blockIdx.x - __ldg(off + c)) * blockDim.x + threadIdx.x;
    if (a < C.M.N) deriv1_node<S, A, FAST>(C.M, C.MS, sh.SC(), sh.SF(), C.st, a);
}

template <class S, class A, bool FAST>
__global__ void __launch_bounds__(256) kb_collide(const CaseDev<S, A> *__restrict__ cases,
                                                  const int *__restrict__ off, int B,
                                                  const MapScalars *__restrict__ sc,
                                                  const MapScalarsF *__restrict__ sf)
{
    wait_prior_grid();
    __shared__ SharedCase<S, A> sh;
    const int c = tile_case(off, B, blockIdx.x);
    sh.load(cases, sc, sf, c);
    __syncthreads();
    const CaseDev<S, A> &C = sh.C();
    const int a = (blockIdx.x - __ldg(off + c)) * blockDim.x + threadIdx.x;
    if (a < C.M.N) collide_at<S, A, FAST>(C.M, C.MS, sh.SC(), sh.SF(), C.K, C.st, C.err, a);
}

// ---------------------------------------------------------------------------
// Shared-memory staging of a tile's neighbour stencil (a tuner candidate for
// the FP32 derivative passes): the block copies the two node fields it
// differentiates over the index window [first node - STAGE_HALO, last node +
// STAGE_HALO] into shared memory (Morton numbering keeps most of a tile's
// owner-element nodes in it) and reads its gradient stencils there, from
// global memory outside it.  Same values as the unstaged kernels.
// ---------------------------------------------------------------------------
constexpr int STAGE_HALO = 256, STAGE_MAX = 256 + 2 * STAGE_HALO;

struct StagedPair {
    float *s0, *s1; // shared windows
    int lo, n;      // window [lo, lo + n)
    const float *g0, *g1;
    __device__ __forceinline__ float v0(int b) const { return (unsigned)(b - lo) < (unsigned)n ? s0[b - lo] : g0[b]; }
    __device__ __forceinline__ float v1(int b) const { return (unsigned)(b - lo) < (unsigned)n ? s1[b - lo] : g1[b]; }
};

__device__ __forceinline__ StagedPair stage_pair(float *s0, float *s1, const float *g0, const float *g1, int first,
                                                 int N, int stage)
{
    StagedPair P;
    P.lo = max(0, first - STAGE_HALO);
    P.n = stage ? min(N, first + (int)blockDim.x + STAGE_HALO) - P.lo : 0; // 0: every read from global
    P.s0 = s0;
    P.s1 = s1;
    P.g0 = g0;
    P.g1 = g1;
    for (int j = threadIdx.x; j < P.n; j += blockDim.x) {
        s0[j] = g0[P.lo + j];
        s1[j] = g1[P.lo + j];
    }
    return P;
}

// FP32 owner-element derivatives d/dX of both staged fields at node a.
__device__ __forceinline__ void owner_grad2_staged(const MeshDev &M, int a, const StagedPair &P, float &K0X,
                                                   float &K0Y, float &K1X, float &K1Y)
{
    const int4 p = M.ostn[2 * a], q = M.ostn[2 * a + 1];
    const int e = q.z, l = q.w;
    const float4 J = M.ejf[2 * e + 1];
    const int nb[6] = {p.x, p.y, p.z, p.w, q.x, q.y};
    float nx[6], ne[6];
    p2_dN_at_node(l, nx, ne);
    float s0x = 0.f, s0e = 0.f, s1x = 0.f, s1e = 0.f;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const int b = nb[s];
        const float v0 = P.v0(b), v1 = P.v1(b);
        s0x += v0 * nx[s];
        s0e += v0 * ne[s];
        s1x += v1 * nx[s];
        s1e += v1 * ne[s];
    }
    K0X = s0x * J.x + s0e * J.z;
    K0Y = s0x * J.y + s0e * J.w;
    K1X = s1x * J.x + s1e * J.z;
    K1Y = s1x * J.y + s1e * J.w;
}

// kb_deriv1 / kb_collide of the FP32-deviation form, with (stage != 0) or
// without staged stencils: one kernel either way, so that the choice cannot
// change a single bit of the result.
__global__ void __launch_bounds__(256) kb_deriv1_staged(const CaseDev<float, float> *__restrict__ cases,
                                                        const int *__restrict__ off, int B,
                                                        const MapScalarsF *__restrict__ sf, int stage)
{
    wait_prior_grid();
    __shared__ SharedCase<float, float> sh;
    __shared__ float w0[STAGE_MAX], w1[STAGE_MAX];
    const int c = tile_case(off, B, blockIdx.x);
    sh.load(cases, nullptr, sf, c);
    __syncthreads();
    const CaseDev<float, float> &C = sh.C();
    const int first = (blockIdx.x - __ldg(off + c)) * blockDim.x;
    const StagedPair P = stage_pair(w0, w1, C.st.Qx, C.st.Qy, first, C.M.N, stage);
    __syncthreads();
    const int a = first + threadIdx.x;
    if (a >= C.M.N) return;
    const FastMap F = fast_map(C.MS, sh.SF(), a, C.M.Xf[a]);
    float QxX, QxY, QyX, QyY;
    owner_grad2_staged(C.M, a, P, QxX, QxY, QyX, QyY);
    const float dQx = F.A11 * QxX + F.A21 * QxY; // d_x Q'_xxx
    const float dQy = F.A12 * QyX + F.A22 * QyY; // d_y Q'_yyy
    const float m = C.st.mrt[a];
    C.st.Dx[a] = m * dQx;
    C.st.Dy[a] = m * dQy;
}

__global__ void __launch_bounds__(256, 4) kb_collide_staged(const CaseDev<float, float> *__restrict__ cases,
                                                         const int *__restrict__ off, int B,
                                                         const MapScalarsF *__restrict__ sf, int stage)
{
    wait_prior_grid();
    __shared__ SharedCase<float, float> sh;
    __shared__ float w0[STAGE_MAX], w1[STAGE_MAX];
    const int c = tile_case(off, B, blockIdx.x);
    sh.load(cases, nullptr, sf, c);
    __syncthreads();
    const CaseDev<float, float> &C = sh.C();
    const int first = (blockIdx.x - __ldg(off + c)) * blockDim.x;
    // the pending-moments list has been read (kb_moments_pending ran before)
    if (first == 0 && threadIdx.x == 0) C.st.wcount[SEG_PENDING] = 0u;
    const StagedPair P = stage_pair(w0, w1, C.st.Dx, C.st.Dy, first, C.M.N, stage);
    __syncthreads();
    const int a = first + threadIdx.x;
    if (a >= C.M.N) return;
    const int N = C.M.N;
    const KinParams<float> &K = C.K;
    float Xx = 0.f, Xy = 0.f;
    if (!(K.flags & FLAG_PHI_OFF)) {
        const FastMap F = fast_map(C.MS, sh.SF(), a, C.M.Xf[a]);
        float DxX, DxY, DyX, DyY;
        owner_grad2_staged(C.M, a, P, DxX, DxY, DyX, DyY);
        Xx = -(F.A11 * DxX + F.A21 * DxY);
        Xy = -(F.A12 * DyX + F.A22 * DyY);
    }
    float f[NQ], g[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) fg_get(C.st.str, i, a, N, f[i], g[i]);
    float rho, ux, uy, T;
    if (!collide_node(K, f, g, Xx, Xy, rho, ux, uy, T)) atomicOr(C.err, ERR_NONFINITE);
#pragma unroll
    for (int i = 0; i < NQ; ++i) fg_put(C.st.post, i, a, N, f[i], g[i]);
    C.st.rho[a] = rho;
    C.st.ux[a] = ux;
    C.st.uy[a] = uy;
    C.st.T[a] = T;
}

// Empties every case's work list and the wall masks and pending marks of
// its nodes (before a repeated launch of kb_fast while tuning): one block
// per case.
template <class S, class A>
__global__ void kb_clear_work(const CaseDev<S, A> *__restrict__ cases, int B)
{
    const int c = blockIdx.x;
    if (c >= B) return;
    const StateDev<S> &st = cases[c].st;
    const int N = cases[c].M.N;
    for (int i = 0; i <= SEG_PENDING; ++i) {
        const unsigned n = st.wcount[i];
        for (unsigned k = threadIdx.x; k < n; k += blockDim.x) {
            const int e = st.work[(size_t)i * N + k];
            st.wmask[i < NQ ? e / NQ : e] = 0u;
        }
    }
    __syncthreads();
    if (threadIdx.x <= SEG_PENDING) st.wcount[threadIdx.x] = 0u;
}

// ---------------------------------------------------------------------------
// The persistent form: one cooperative launch runs a chunk of steps, every
// phase of every step over all cases, with a grid-wide barrier between
// phases (each phase reads what the previous one wrote anywhere in the
// mesh).  Each wait at a barrier is bounded: past the limit the block sets
// ERR_TIMEOUT in every case's error word and an abort flag that releases
// every other wait, and the kernel returns.
// ---------------------------------------------------------------------------
struct GridSync {
    unsigned *count;   // arrivals at the barrier being formed
    unsigned *gen;     // barriers completed so far
    int *abort;        // set once a wait has run out: every later wait returns at once
    unsigned expected; // arrivals that complete a barrier (the grid, plus a test's missing ones)
    unsigned long long limit_ns;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Returns false when the kernel must stop (a wait ran out here or elsewhere).
template <class S, class A>
__device__ bool grid_barrier(const GridSync &g, const CaseDev<S, A> *cases, int B)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence(); // this block's writes of the phase, before it arrives
        const unsigned my_gen = *(volatile unsigned *)g.gen;
        if (atomicAdd(g.count, 1u) + 1u == g.expected) {
            *(volatile unsigned *)g.count = 0u;
            __threadfence();
            atomicAdd(g.gen, 1u); // opens the barrier
        } else {
            const unsigned long long t0 = global_ns();
            while (*(volatile unsigned *)g.gen == my_gen) {
                if (*(volatile int *)g.abort) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > g.limit_ns) {
                    for (int c = 0; c < B; ++c) atomicOr(cases[c].err, ERR_TIMEOUT);
                    atomicExch(g.abort, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence(); // the other blocks' writes, before this block reads them
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Steps 0..K-1 of a chunk (map scalars sc[k B + c], sf[k B + c]), one block
// per SM-resident slot, node tiles of blockDim.x nodes (offsets off) dealt
// out over the grid in every node-parallel phase.
template <class S, class A>
__global__ void __launch_bounds__(128) kb_persistent(const CaseDev<S, A> *__restrict__ cases,
                                                     const int *__restrict__ off, int B,
                                                     const MapScalars *__restrict__ scs,
                                                     const MapScalarsF *__restrict__ sfs, int K, GridSync g)
{
    constexpr int NS = NQ + 1;
    constexpr bool FAST = !std::is_same<S, double>::value;
    __shared__ SharedCase<S, A> sh;
    __shared__ unsigned pre[BATCH_MAX * NS + 1];
    const int tiles = __ldg(off + B);
    // node-parallel phase: body(C, sc, sf, node) for every node of every case
    auto tiles_loop = [&](int k, auto &&body) {
        for (int vt = blockIdx.x; vt < tiles; vt += gridDim.x) {
            const int c = tile_case(off, B, vt);
            __syncthreads(); // the previous tile's users of sh are done
            sh.load(cases, scs + (size_t)k * B, sfs + (size_t)k * B, c);
            __syncthreads();
            body(sh.C(), sh.SC(), sh.SF(), (vt - __ldg(off + c)) * blockDim.x + threadIdx.x);
        }
    };
    for (int k = 0; k < K; ++k) {
        const MapScalars *sc = scs + (size_t)k * B;
        const MapScalarsF *sf = sfs + (size_t)k * B;
        if (FAST) {
            tiles_loop(k, [&](const CaseDev<S, A> &C, const MapScalars &, const MapScalarsF &SF, int a) {
                stream_fast_group<BATCH_FAST_G>(C.M, C.MS, SF, C.K, C.st, a);
            });
            if (!grid_barrier(g, cases, B)) return;
            // the exact path over every case's work list (kb_slow's numbering)
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                unsigned loc[NS];
                unsigned s = 0, npop = 0;
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    loc[i] = lane < B ? *(volatile unsigned *)(cases[lane].st.wcount + i) : 0u;
                    s += loc[i];
                    if (i < NQ) npop += loc[i];
                }
                unsigned incl = s;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                if (lane < B) {
                    unsigned run = incl - s;
#pragma unroll
                    for (int i = 0; i < NS; ++i) {
                        pre[lane * NS + i] = run;
                        run += loc[i];
                    }
                    if (lane == B - 1) pre[B * NS] = run;
                    if (npop && blockIdx.x == 0 && cases[lane].stats)
                        atomicAdd(cases[lane].stats, (unsigned long long)npop);
                }
            }
            __syncthreads();
            const unsigned total = pre[B * NS];
            for (unsigned w = spread_first(); w < total; w += spread_stride()) {
                int lo = 0, hi = B * NS - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (pre[mid] <= w) lo = mid;
                    else hi = mid - 1;
                }
                const int c = lo / NS, i = lo % NS;
                const CaseDev<S, A> &C = cases[c];
                const int entry = C.st.work[(size_t)i * C.M.N + (w - pre[lo])];
                if (i < NQ) {
                    stream_slow_item(C.M, C.MS, sc[c], sf[c], sc[c], sf[c], C.K, C.st, C.err, entry);
                } else {
                    const unsigned mask = C.st.wmask[entry] & WMASK_DIRS;
                    if (C.stats) atomicAdd(C.stats, (unsigned long long)__popc(mask));
                    stream_bc_node<S, A>(C.M, C.MS, sc[c], sf[c], C.K, C.st, entry,
                                         fast_map(C.MS, sf[c], entry, C.M.Xf[entry]), mask);
                }
            }
            if (!grid_barrier(g, cases, B)) return;
            tiles_loop(k, [&](const CaseDev<S, A> &C, const MapScalars &, const MapScalarsF &, int a) {
                if (a <= NQ) C.st.wcount[a] = 0u; // the case's work list has been consumed
                if (a < C.M.N) moments_node(C.K, C.st, C.M.N, C.err, a);
            });
        } else {
            tiles_loop(k, [&](const CaseDev<S, A> &C, const MapScalars &SC, const MapScalarsF &, int a) {
                if (a < C.M.N) stream_plain_node(C.M, C.MS, SC, SC, C.K, C.st, C.err, C.stats, a);
            });
        }
        if (!grid_barrier(g, cases, B)) return;
        tiles_loop(k, [&](const CaseDev<S, A> &C, const MapScalars &SC, const MapScalarsF &SF, int a) {
            if (a < C.M.N) deriv1_node<S, A, FAST>(C.M, C.MS, SC, SF, C.st, a);
        });
        if (!grid_barrier(g, cases, B)) return;
        tiles_loop(k, [&](const CaseDev<S, A> &C, const MapScalars &SC, const MapScalarsF &SF, int a) {
            if (a < C.M.N) collide_at<S, A, FAST>(C.M, C.MS, SC, SF, C.K, C.st, C.err, a);
        });
        if (!grid_barrier(g, cases, B)) return;
    }
}

int bs_index(int bs) { return bs == 64 ? 0 : bs == 128 ? 1 : 2; }

// Blocks of the exact-path kernel resident per SM at block size bs.
template <class S, class A> int slow_resident_t(int bs)
{
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kb_slow<S, A>, bs, 0);
    return v > 0 ? v : 1;
}

} // namespace

struct alelb_batch {
    std::string err;
    std::vector<alelb_solver *> cs;
    int B = 0, prec = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevBuf buf;
    void *d_cases = nullptr;
    int *d_off[N_BS] = {nullptr, nullptr, nullptr};
    std::vector<int> h_off[N_BS];
    MapScalars *d_sc = nullptr;
    MapScalarsF *d_sf = nullptr;
    MapScalars *h_sc[2] = {nullptr, nullptr};
    MapScalarsF *h_sf[2] = {nullptr, nullptr};
    cudaEvent_t h_ev[2] = {nullptr, nullptr};
    int slot = 0;
    std::vector<cudaEvent_t> ev_in;
    cudaEvent_t ev_done = nullptr;
    int *h_err = nullptr; // pinned: every case's error word, read in one wait
    // launch shapes (threads per block per kernel; blocks of k_stream_slow)
    int bs[KT_N] = {128, 128, 128, 256, 256, 128, 128};
    int slow_grid = 0;
    int fast_g = BATCH_FAST_G; // directions per thread of k_stream_fast
    bool stage[KT_N] = {};     // shared-memory staging of the derivative stencils (FP32 form)
    int n_sm = 152;
    std::map<int, cudaGraphExec_t> graphs;
    // case groups (graph mode): the descriptor array, tile tables and staged
    // scalars hold the cases in the order ord (positions of b->cs), which
    // splits into four contiguous runs of balanced node counts; two groups
    // join runs 0-1 and 2-3; groups = 1 runs all cases as one
    std::vector<int> ord;
    int groups = 1;
    int pipe = 0; // 0: groups run free; 1, 2: alternating propagations (enqueue_groups)
    struct Run {
        int c0 = 0, n = 0;       // first descriptor, number of cases
        int *d_off[N_BS] = {};   // tile tables of the run (device)
        std::vector<int> h_off[N_BS];
    };
    Run run2[2], run4[4], run8[8];
    bool has2 = false, has4 = false, has8 = false; // every group of the split holds a case
    cudaStream_t gstream[GROUPS_MAX] = {}; // [0] unused: group 0 runs on the batch's stream
    cudaEvent_t gev_fork = nullptr, gev_join[GROUPS_MAX] = {}, gev_fast[GROUPS_MAX] = {};
    cudaEvent_t gev_up[GROUPS_MAX] = {}; // alelb_batch_step_host: group g's uploads are in
    // the persistent form (mode ALELB_BATCH_PERSISTENT): threads per block,
    // blocks (all resident), barrier words {count, gen, abort}, wait limit
    int mode = ALELB_BATCH_GRAPHS;
    int pers_bs = 128, pers_grid = 0;
    unsigned *d_sync = nullptr;
    double wait_limit_s = 1.0;
    int missing = 0;
    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { int k; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    double ms_acc[KT_N] = {};
    int64_t n_acc[KT_N] = {};
};

namespace {
int slow_resident(const alelb_batch *b, int bs)
{
    return b->prec == ALELB_PREC_FP32_DEV ? slow_resident_t<float, float>(bs) : slow_resident_t<double, double>(bs);
}
} // namespace

namespace {

alelb_status bfail(alelb_batch *b, cudaError_t st, const char *what)
{
    b->err = std::string(what) + ": " + cudaGetErrorString(st);
    return st == cudaErrorMemoryAllocation ? ALELB_ERR_OOM : ALELB_ERR_CUDA;
}

cudaEvent_t bget_event(alelb_batch *b)
{
    if (b->ev_pool.empty()) {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t e = b->ev_pool.back();
    b->ev_pool.pop_back();
    return e;
}

void bflush_prof(alelb_batch *b)
{
    for (auto &r : b->pending) {
        float ms = 0;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            b->ms_acc[r.k] += ms;
            b->n_acc[r.k] += 1;
        }
        b->ev_pool.push_back(r.a);
        b->ev_pool.push_back(r.b);
    }
    b->pending.clear();
}

void drop_graphs(alelb_batch *b)
{
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
}

// Phase kernels of one step, in order.
int step_sequence(const alelb_batch *b, int seq[KT_N])
{
    int n = 0;
    if (b->prec == ALELB_PREC_FP32_DEV) {
        seq[n++] = KT_FAST;
        seq[n++] = KT_SLOW;
        seq[n++] = KT_MOMENTS;
    } else {
        seq[n++] = KT_STREAM;
    }
    seq[n++] = KT_DERIV1;
    seq[n++] = KT_COLLIDE;
    return n;
}

// The cases one launch covers: all of them, or one group.
struct Part {
    cudaStream_t stream;
    int c0, B;            // first descriptor, number of cases
    const int *off[N_BS]; // their tile tables (device), per block size
    int tiles[N_BS];
    bool pdl;             // programmatic serialization after the stream's previous kernel
};

Part whole(const alelb_batch *b)
{
    Part P{b->stream, 0, b->B, {}, {}, true};
    for (int q = 0; q < N_BS; ++q) {
        P.off[q] = b->d_off[q];
        P.tiles[q] = b->h_off[q][b->B];
    }
    return P;
}

// Group g of the split into `groups` (2, 4 or 8) groups.
Part group(const alelb_batch *b, int groups, int g, bool pdl)
{
    const alelb_batch::Run &R = groups == 8 ? b->run8[g] : groups == 4 ? b->run4[g] : b->run2[g];
    Part P{g ? b->gstream[g] : b->stream, R.c0, R.n, {}, {}, pdl};
    for (int q = 0; q < N_BS; ++q) {
        P.off[q] = R.d_off[q];
        P.tiles[q] = R.h_off[q][R.n];
    }
    return P;
}

// A phase kernel on a part's stream: with programmatic serialization, or
// (right after a wait on another stream's event) as a plain launch, whose
// wait_prior_grid returns at once.
template <class... KArgs, class... Args>
void launch_after(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t stream, Args... args)
{
    if (pdl) launch_pdl(kern, grid, block, stream, args...);
    else kern<<<grid, block, 0, stream>>>(static_cast<KArgs>(args)...);
}

// One phase kernel over the part's cases with the scalars of chunk step k.
// bs: threads per block; grid: blocks (k_stream_slow only).
template <class S, class A>
void launch_phase(alelb_batch *b, const Part &P, int kt, int bs, int grid, int k, int count, int fast_g, bool stage)
{
    const auto *cases = reinterpret_cast<const CaseDev<S, A> *>(b->d_cases) + P.c0;
    const int q = bs_index(bs);
    const int *off = P.off[q];
    const int tiles = P.tiles[q];
    const MapScalars *sc = b->d_sc + (size_t)k * b->B + P.c0;
    const MapScalarsF *sf = b->d_sf + (size_t)k * b->B + P.c0;
    const int B = P.B;
    const bool fast = b->prec == ALELB_PREC_FP32_DEV;
    switch (kt) {
    case KT_STREAM:
        launch_after(P.pdl, kb_stream<S, A>, dim3(tiles), dim3(bs), P.stream, cases, off, B, sc, count);
        break;
    case KT_FAST:
        // fast_g: directions per thread, plus FAST_FUSED for the propagation
        // fused with the moments
        if (fast_g & FAST_FUSED) {
            if constexpr (std::is_same<S, float>::value) {
                const auto *cf = reinterpret_cast<const CaseDev<float, float> *>(cases);
                const int G = fast_g & 15;
                if (G == 3 && bs == 64)
                    launch_after(P.pdl, kb_fast_fused<3, 64>, dim3(tiles), dim3(64 * 3), P.stream, cf, off, B, sf);
                else if (G == 3 && bs == 128)
                    launch_after(P.pdl, kb_fast_fused<3, 128>, dim3(tiles), dim3(128 * 3), P.stream, cf, off, B, sf);
                else if (G == 3)
                    launch_after(P.pdl, kb_fast_fused<3, 256>, dim3(tiles), dim3(256 * 3), P.stream, cf, off, B, sf);
                else if (bs == 64)
                    launch_after(P.pdl, kb_fast_fused<9, 64>, dim3(tiles), dim3(64), P.stream, cf, off, B, sf);
                else if (bs == 128)
                    launch_after(P.pdl, kb_fast_fused<9, 128>, dim3(tiles), dim3(128), P.stream, cf, off, B, sf);
                else
                    launch_after(P.pdl, kb_fast_fused<9, 256>, dim3(tiles), dim3(256), P.stream, cf, off, B, sf);
            }
        } else if (fast_g == 1)
            launch_after(P.pdl, kb_fast<S, A, 1>, dim3(tiles, NQ), dim3(bs), P.stream, cases, off, B, sf);
        else if (fast_g == 3)
            launch_after(P.pdl, kb_fast<S, A, 3>, dim3(tiles, NQ / 3), dim3(bs), P.stream, cases, off, B, sf);
        else
            launch_after(P.pdl, kb_fast<S, A, 9>, dim3(tiles, 1), dim3(bs), P.stream, cases, off, B, sf);
        break;
    case KT_SLOW:
        launch_after(P.pdl, kb_slow<S, A>, dim3(grid), dim3(bs), P.stream, cases, B, sc, sf, count);
        break;
    case KT_MOMENTS:
        if (fast_g & FAST_FUSED) // the pending nodes only, over one wave of blocks
            launch_after(P.pdl, kb_moments_pending<S, A>, dim3(b->n_sm * (2048 / bs)), dim3(bs), P.stream, cases, B);
        else
            launch_after(P.pdl, kb_moments<S, A>, dim3(tiles), dim3(bs), P.stream, cases, off, B);
        break;
    case KT_DERIV1:
        if (fast)
            launch_after(P.pdl, kb_deriv1_staged, dim3(tiles), dim3(bs), P.stream,
                       reinterpret_cast<const CaseDev<float, float> *>(cases), off, B, sf, (int)stage);
        else launch_after(P.pdl, kb_deriv1<S, A, false>, dim3(tiles), dim3(bs), P.stream, cases, off, B, sc, sf);
        break;
    default:
        if (fast)
            launch_after(P.pdl, kb_collide_staged, dim3(tiles), dim3(bs), P.stream,
                       reinterpret_cast<const CaseDev<float, float> *>(cases), off, B, sf, (int)stage);
        else launch_after(P.pdl, kb_collide<S, A, false>, dim3(tiles), dim3(bs), P.stream, cases, off, B, sc, sf);
    }
}

void launch_kernel(alelb_batch *b, const Part &P, int kt, int bs, int grid, int k, int count, int fast_g, bool stage)
{
    if (b->prec == ALELB_PREC_FP32_DEV) launch_phase<float, float>(b, P, kt, bs, grid, k, count, fast_g, stage);
    else launch_phase<double, double>(b, P, kt, bs, grid, k, count, fast_g, stage);
}
void launch_kernel(alelb_batch *b, int kt, int bs, int grid, int k, int count, int fast_g, bool stage)
{
    launch_kernel(b, whole(b), kt, bs, grid, k, count, fast_g, stage);
}

// One cooperative launch of the persistent kernel for chunk steps 0..K-1.
template <class S, class A> cudaError_t launch_persistent_t(alelb_batch *b, int K)
{
    const auto *cases = reinterpret_cast<const CaseDev<S, A> *>(b->d_cases);
    GridSync g;
    g.count = b->d_sync;
    g.gen = b->d_sync + 1;
    g.abort = reinterpret_cast<int *>(b->d_sync + 2);
    g.expected = (unsigned)b->pers_grid + (unsigned)b->missing;
    g.limit_ns = (unsigned long long)(b->wait_limit_s * 1e9);
    // a barrier left half formed by an earlier wait that ran out starts afresh
    cudaError_t st = cudaMemsetAsync(b->d_sync, 0, sizeof(unsigned), b->stream);
    if (st == cudaSuccess) st = cudaMemsetAsync(b->d_sync + 2, 0, sizeof(unsigned), b->stream);
    if (st != cudaSuccess) return st;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->pers_grid);
    cfg.blockDim = dim3(b->pers_bs);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative; // every block resident at once
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kb_persistent<S, A>, cases, (const int *)b->d_off[bs_index(b->pers_bs)], b->B,
                              (const MapScalars *)b->d_sc, (const MapScalarsF *)b->d_sf, K, g);
}

cudaError_t launch_persistent(alelb_batch *b, int K)
{
    return b->prec == ALELB_PREC_FP32_DEV ? launch_persistent_t<float, float>(b, K)
                                          : launch_persistent_t<double, double>(b, K);
}

// Blocks of the persistent kernel that fit on the device at once.
template <class S, class A> int persistent_grid_t(int bs, int n_sm)
{
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kb_persistent<S, A>, bs, 0);
    return std::max(v, 1) * n_sm;
}

void enqueue_step(alelb_batch *b, int k)
{
    int seq[KT_N];
    const int ns = step_sequence(b, seq);
    for (int q = 0; q < ns; ++q) {
        const int kt = seq[q];
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (b->prof) {
            ea = bget_event(b);
            eb = bget_event(b);
            cudaEventRecord(ea, b->stream);
        }
        launch_kernel(b, kt, b->bs[kt], b->slow_grid, k, 1, b->fast_g, b->stage[kt]);
        if (b->prof) {
            cudaEventRecord(eb, b->stream);
            b->pending.push_back({kt, ea, eb});
        }
    }
}

// Step k of every case group, inside a capture: group g >= 1 on its own
// stream (forked from the batch's stream at the chunk's start).  With
// pipe = p > 0 the first p phase kernels of each group's step (the
// propagation, and with p = 2 its exact part) follow those of the previous
// group (of the previous step for group 0); a kernel after such a wait, or
// first on its stream, is launched plainly.
cudaError_t enqueue_groups(alelb_batch *b, int k)
{
    int seq[KT_N];
    const int ns = step_sequence(b, seq);
    const int lead = std::min(b->pipe ? (b->pipe == 2 ? 2 : 1) : 0, ns);
    cudaError_t st = cudaSuccess;
    for (int g = 0; g < b->groups && st == cudaSuccess; ++g) {
        cudaStream_t sg = g ? b->gstream[g] : b->stream;
        bool pdl = !(k == 0 && g > 0);
        if (lead && (k > 0 || g > 0)) {
            st = cudaStreamWaitEvent(sg, b->gev_fast[g > 0 ? g - 1 : b->groups - 1], 0);
            pdl = false;
        }
        for (int q = 0; q < ns && st == cudaSuccess; ++q) {
            const int kt = seq[q];
            launch_kernel(b, group(b, b->groups, g, pdl), kt, b->bs[kt], b->slow_grid, k, 1, b->fast_g, b->stage[kt]);
            pdl = true;
            if (q + 1 == lead) st = cudaEventRecord(b->gev_fast[g], sg);
        }
    }
    return st;
}

cudaError_t get_graph(alelb_batch *b, int K, cudaGraphExec_t &exec)
{
    auto it = b->graphs.find(K);
    if (it != b->graphs.end()) {
        exec = it->second;
        return cudaSuccess;
    }
    cudaGraph_t g = nullptr;
    cudaError_t st = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (st != cudaSuccess) return st;
    cudaError_t st_q = cudaSuccess;
    if (b->groups > 1) {
        st_q = cudaEventRecord(b->gev_fork, b->stream);
        for (int h = 1; h < b->groups && st_q == cudaSuccess; ++h) st_q = cudaStreamWaitEvent(b->gstream[h], b->gev_fork, 0);
        for (int k = 0; k < K && st_q == cudaSuccess; ++k) st_q = enqueue_groups(b, k);
        // every branch joins the batch's stream (also after a failure, so
        // that the capture can end)
        for (int h = 1; h < b->groups; ++h) {
            cudaError_t sj = cudaEventRecord(b->gev_join[h], b->gstream[h]);
            if (sj == cudaSuccess) sj = cudaStreamWaitEvent(b->stream, b->gev_join[h], 0);
            if (st_q == cudaSuccess) st_q = sj;
        }
    } else {
        for (int k = 0; k < K; ++k) enqueue_step(b, k);
    }
    cudaError_t st_launch = cudaGetLastError();
    if (st_launch == cudaSuccess) st_launch = st_q;
    st = cudaStreamEndCapture(b->stream, &g);
    if (st == cudaSuccess) st = st_launch;
    if (st == cudaSuccess) st = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st == cudaSuccess) b->graphs[K] = exec;
    return st;
}

// Stages the map scalars of chunk steps 0..K-1 (case times t_c + done + k + 1)
// and copies them to the device table.
cudaError_t stage_scalars(alelb_batch *b, int done, int K)
{
    const int sl = b->slot;
    cudaError_t st = cudaEventSynchronize(b->h_ev[sl]); // earlier copy out of this slot finished
    if (st != cudaSuccess) return st;
    for (int k = 0; k < K; ++k)
        for (int c = 0; c < b->B; ++c) {
            const alelb_solver *s = b->cs[b->ord[c]];
            const HostTables &T = s->mesh->T;
            const MapScalars sc = solver_map(s, map_scalars(T.mkind, T.mp, s->t + (double)(done + k + 1)));
            b->h_sc[sl][(size_t)k * b->B + c] = sc;
            b->h_sf[sl][(size_t)k * b->B + c] = to_f32(sc, T);
        }
    st = cudaMemcpyAsync(b->d_sc, b->h_sc[sl], sizeof(MapScalars) * K * b->B, cudaMemcpyHostToDevice, b->stream);
    if (st == cudaSuccess)
        st = cudaMemcpyAsync(b->d_sf, b->h_sf[sl], sizeof(MapScalarsF) * K * b->B, cudaMemcpyHostToDevice,
                             b->stream);
    if (st == cudaSuccess) st = cudaEventRecord(b->h_ev[sl], b->stream);
    b->slot ^= 1;
    return st;
}

// Orders the batch's stream after each case's earlier work.
cudaError_t join_cases(alelb_batch *b)
{
    cudaError_t st = cudaSuccess;
    for (int c = 0; c < b->B && st == cudaSuccess; ++c) {
        cudaStream_t cs = b->cs[c]->stream;
        if (cs == b->stream) continue;
        st = cudaEventRecord(b->ev_in[c], cs);
        if (st == cudaSuccess) st = cudaStreamWaitEvent(b->stream, b->ev_in[c], 0);
    }
    return st;
}

// Orders each case's stream after the batch's last launch.
cudaError_t release_cases(alelb_batch *b)
{
    cudaError_t st = cudaEventRecord(b->ev_done, b->stream);
    for (int c = 0; c < b->B && st == cudaSuccess; ++c) {
        cudaStream_t cs = b->cs[c]->stream;
        if (cs != b->stream) st = cudaStreamWaitEvent(cs, b->ev_done, 0);
    }
    return st;
}

template <class S, class A> CaseDev<S, A> case_desc(alelb_solver *s);
template <> CaseDev<float, float> case_desc<float, float>(alelb_solver *s)
{
    return CaseDev<float, float>{s->mesh->dev, s->mesh->mst, s->kf, s->sf, s->d_err, s->d_stats};
}
template <> CaseDev<double, double> case_desc<double, double>(alelb_solver *s)
{
    return CaseDev<double, double>{s->mesh->dev, s->mesh->mst, s->kd, s->sd, s->d_err, s->d_stats};
}

template <class S, class A> cudaError_t upload_cases(alelb_batch *b)
{
    std::vector<CaseDev<S, A>> h(b->B);
    for (int c = 0; c < b->B; ++c) h[c] = case_desc<S, A>(b->cs[b->ord[c]]);
    cudaError_t st = cudaSuccess;
    auto *d = b->buf.alloc<CaseDev<S, A>>(b->B, st);
    b->d_cases = d;
    if (st == cudaSuccess) st = cudaMemcpy(d, h.data(), sizeof(CaseDev<S, A>) * b->B, cudaMemcpyHostToDevice);
    return st;
}

} // namespace

extern "C" alelb_status alelb_batch_create(alelb_solver *const *cases, int32_t B, void *stream,
                                           alelb_batch **out)
{
    if (!out) return ALELB_ERR_ARG;
    *out = nullptr;
    if (!cases || B < 1 || B > BATCH_MAX) return ALELB_ERR_ARG;
    for (int c = 0; c < B; ++c) {
        if (!cases[c] || !cases[c]->mesh) return ALELB_ERR_ARG;
        if (cases[c]->prec != cases[0]->prec) return ALELB_ERR_ARG;
        // the batched kernels are built for the FP64 and FP32-deviation forms
        // and the arrival-time transformed velocities
        if (cases[c]->prec != ALELB_PREC_FP64 && cases[c]->prec != ALELB_PREC_FP32_DEV) return ALELB_ERR_ARG;
        if (cases[c]->flags & (ALELB_FLAG_MIDPOINT | ALELB_FLAG_EXACT_CHAR)) return ALELB_ERR_ARG;
        if (cases[c]->mesh->etype != ALELB_ELEM_P2TRI) return ALELB_ERR_ARG; // 6-node triangles only
        for (int d = 0; d < c; ++d)
            if (cases[d] == cases[c]) return ALELB_ERR_ARG;
    }
    alelb_batch *b = new (std::nothrow) alelb_batch();
    if (!b) return ALELB_ERR_OOM;
    *out = b;
    b->cs.assign(cases, cases + B);
    b->B = B;
    b->prec = cases[0]->prec;
    b->n_sm = cases[0]->n_sm;
    b->slow_grid = slow_resident(b, 128) * b->n_sm;
    cudaError_t st = cudaSuccess;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        st = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = st == cudaSuccess;
    }
    if (st != cudaSuccess) return bfail(b, st, "stream");
    // descriptor order: the cases dealt, largest first, to the half (runs
    // 0-1 or 2-3) with fewer nodes so far, within it to the run with fewer
    // nodes, each run's cases then in the callers' order; two groups are the
    // halves, four the runs, eight each run split where its nodes are
    // closest to halved (the pipelined host step)
    int first4[5] = {}, first8[9] = {};
    {
        std::vector<int> idx(B);
        for (int c = 0; c < B; ++c) idx[c] = c;
        std::stable_sort(idx.begin(), idx.end(),
                         [b](int x, int y) { return b->cs[x]->mesh->T.N > b->cs[y]->mesh->T.N; });
        std::vector<int> rof(B, 0);
        long long load[4] = {};
        for (int c : idx) {
            const int h = load[2] + load[3] < load[0] + load[1] ? 2 : 0;
            const int r = load[h + 1] < load[h] ? h + 1 : h;
            rof[c] = r;
            load[r] += b->cs[c]->mesh->T.N;
        }
        for (int r = 0; r < 4; ++r) {
            for (int c = 0; c < B; ++c)
                if (rof[c] == r) b->ord.push_back(c);
            first4[r + 1] = (int)b->ord.size();
        }
        for (int r = 0; r < 4; ++r) {
            // the split point of run r: at least one case each side when it
            // holds two, the two sides' node counts as close as possible
            const int c0 = first4[r], c1 = first4[r + 1];
            long long tot = 0, left = 0, best = -1;
            for (int j = c0; j < c1; ++j) tot += b->cs[b->ord[j]]->mesh->T.N;
            int cut = c1 - c0 >= 2 ? c0 + 1 : c1;
            for (int j = c0; j + 1 < c1; ++j) {
                left += b->cs[b->ord[j]]->mesh->T.N;
                const long long d = left * 2 > tot ? left * 2 - tot : tot - left * 2;
                if (best < 0 || d < best) {
                    best = d;
                    cut = j + 1;
                }
            }
            first8[2 * r] = c0;
            first8[2 * r + 1] = cut;
        }
        first8[8] = B;
    }
    // tile offsets per block size, of all cases and of each run
    const auto tiles_of = [b](int j, int bs) { return (b->cs[b->ord[j]]->mesh->T.N + bs - 1) / bs; };
    const auto set_run = [&](alelb_batch::Run &R, int c0, int c1) {
        R.c0 = c0;
        R.n = c1 - c0;
        for (int q = 0; q < N_BS; ++q) {
            auto &o = R.h_off[q];
            o.assign(R.n + 1, 0);
            for (int c = 0; c < R.n; ++c) o[c + 1] = o[c] + tiles_of(c0 + c, 64 << q);
            R.d_off[q] = b->buf.put(o, st);
        }
    };
    for (int q = 0; q < N_BS; ++q) {
        const int bs = 64 << q;
        auto &o = b->h_off[q];
        o.assign(B + 1, 0);
        for (int c = 0; c < B; ++c) o[c + 1] = o[c] + tiles_of(c, bs);
        b->d_off[q] = b->buf.put(o, st);
    }
    for (int r = 0; r < 8; ++r) set_run(b->run8[r], first8[r], first8[r + 1]);
    for (int q = 0; q < 4; ++q) set_run(b->run4[q], first4[q], first4[q + 1]);
    for (int h = 0; h < 2; ++h) set_run(b->run2[h], first4[2 * h], first4[2 * h + 2]);
    const auto all_held = [](const alelb_batch::Run *R, int n) {
        for (int k = 0; k < n; ++k)
            if (R[k].n == 0) return false;
        return true;
    };
    b->has2 = all_held(b->run2, 2);
    b->has4 = all_held(b->run4, 4);
    b->has8 = all_held(b->run8, 8);
    for (int g = 1; g < GROUPS_MAX && st == cudaSuccess; ++g)
        st = cudaStreamCreateWithFlags(&b->gstream[g], cudaStreamNonBlocking);
    if (st == cudaSuccess) st = cudaEventCreateWithFlags(&b->gev_fork, cudaEventDisableTiming);
    for (int g = 0; g < GROUPS_MAX && st == cudaSuccess; ++g) {
        st = cudaEventCreateWithFlags(&b->gev_join[g], cudaEventDisableTiming);
        if (st == cudaSuccess) st = cudaEventCreateWithFlags(&b->gev_fast[g], cudaEventDisableTiming);
        if (st == cudaSuccess) st = cudaEventCreateWithFlags(&b->gev_up[g], cudaEventDisableTiming);
    }
    if (st == cudaSuccess)
        st = b->prec == ALELB_PREC_FP32_DEV ? upload_cases<float, float>(b) : upload_cases<double, double>(b);
    b->d_sync = b->buf.alloc<unsigned>(4, st);
    if (st == cudaSuccess) st = cudaMemset(b->d_sync, 0, 4 * sizeof(unsigned));
    b->pers_grid = b->prec == ALELB_PREC_FP32_DEV ? persistent_grid_t<float, float>(b->pers_bs, b->n_sm)
                                                  : persistent_grid_t<double, double>(b->pers_bs, b->n_sm);
    b->d_sc = b->buf.alloc<MapScalars>((size_t)CHUNK_MAX * B, st);
    b->d_sf = b->buf.alloc<MapScalarsF>((size_t)CHUNK_MAX * B, st);
    for (int sl = 0; sl < 2; ++sl) {
        if (st == cudaSuccess) st = cudaHostAlloc((void **)&b->h_sc[sl], sizeof(MapScalars) * CHUNK_MAX * B, 0);
        if (st == cudaSuccess) st = cudaHostAlloc((void **)&b->h_sf[sl], sizeof(MapScalarsF) * CHUNK_MAX * B, 0);
        if (st == cudaSuccess) st = cudaEventCreateWithFlags(&b->h_ev[sl], cudaEventDisableTiming);
    }
    b->ev_in.assign(B, nullptr);
    for (int c = 0; c < B && st == cudaSuccess; ++c)
        st = cudaEventCreateWithFlags(&b->ev_in[c], cudaEventDisableTiming);
    if (st == cudaSuccess) st = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming);
    if (st == cudaSuccess) st = cudaHostAlloc((void **)&b->h_err, sizeof(int) * B, 0);
    // the table uploads above run on the legacy default stream, which the
    // batch's non-blocking stream does not wait for
    if (st == cudaSuccess) st = cudaDeviceSynchronize();
    if (st != cudaSuccess) return bfail(b, st, "batch_create");
    return ALELB_OK;
}

extern "C" void alelb_batch_destroy(alelb_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    bflush_prof(b);
    drop_graphs(b);
    for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_in)
        if (e) cudaEventDestroy(e);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    if (b->gev_fork) cudaEventDestroy(b->gev_fork);
    for (int g = 0; g < GROUPS_MAX; ++g) {
        if (b->gev_join[g]) cudaEventDestroy(b->gev_join[g]);
        if (b->gev_fast[g]) cudaEventDestroy(b->gev_fast[g]);
        if (b->gev_up[g]) cudaEventDestroy(b->gev_up[g]);
        if (b->gstream[g]) cudaStreamDestroy(b->gstream[g]);
    }
    if (b->h_err) cudaFreeHost(b->h_err);
    for (int sl = 0; sl < 2; ++sl) {
        if (b->h_ev[sl]) cudaEventDestroy(b->h_ev[sl]);
        if (b->h_sc[sl]) cudaFreeHost(b->h_sc[sl]);
        if (b->h_sf[sl]) cudaFreeHost(b->h_sf[sl]);
    }
    b->buf.release();
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

extern "C" const char *alelb_batch_last_error(alelb_batch *b) { return b ? b->err.c_str() : "null batch"; }

namespace {
// Steps t .. t + n of every case on the batch's stream (chunks of at most
// CHUNK_MAX steps), without advancing the solvers' clocks.
cudaError_t run_steps(alelb_batch *b, int n)
{
    cudaError_t st = cudaSuccess;
    for (int done = 0; done < n && st == cudaSuccess;) {
        const int K = std::min(CHUNK_MAX, n - done);
        st = stage_scalars(b, done, K);
        if (st != cudaSuccess) break;
        if (b->prof) {
            for (int k = 0; k < K; ++k) enqueue_step(b, k);
            st = cudaGetLastError();
        } else if (b->mode == ALELB_BATCH_PERSISTENT) {
            st = launch_persistent(b, K);
        } else {
            cudaGraphExec_t g = nullptr;
            st = get_graph(b, K, g);
            if (st == cudaSuccess) st = cudaGraphLaunch(g, b->stream);
        }
        done += K;
    }
    return st;
}

// A copy of what a step reads of every case's FP32 state (the stored
// post-collision populations, the latest fields, the element cache, the
// walk counters and the error word; the rest is rebuilt inside a step),
// taken and put back on the batch's stream.
struct Snapshot {
    DevBuf buf;
    std::vector<std::array<void *, 7>> part;
    std::vector<std::array<size_t, 7>> len;
    cudaError_t take(alelb_batch *b)
    {
        cudaError_t st = cudaSuccess;
        for (alelb_solver *s : b->cs) {
            const size_t N = (size_t)s->mesh->T.N;
            const StateDev<float> &x = s->sf;
            const std::array<void *, 7> src = {x.post, x.rho, x.ux, x.uy, x.T, x.cache, s->d_stats};
            const std::array<size_t, 7> l = {18 * N * sizeof(float), N * sizeof(float), N * sizeof(float),
                                             N * sizeof(float), N * sizeof(float), 9 * N * sizeof(int),
                                             4 * sizeof(unsigned long long)};
            std::array<void *, 7> dst{};
            for (int k = 0; k < 7 && st == cudaSuccess; ++k) {
                dst[k] = buf.alloc<unsigned char>(l[k], st);
                if (st == cudaSuccess) st = cudaMemcpyAsync(dst[k], src[k], l[k], cudaMemcpyDeviceToDevice, b->stream);
            }
            part.push_back(dst);
            len.push_back(l);
        }
        return st;
    }
    cudaError_t put(alelb_batch *b)
    {
        cudaError_t st = cudaSuccess;
        for (size_t c = 0; c < b->cs.size() && st == cudaSuccess; ++c) {
            alelb_solver *s = b->cs[c];
            const StateDev<float> &x = s->sf;
            void *const dst[7] = {x.post, x.rho, x.ux, x.uy, x.T, x.cache, s->d_stats};
            for (int k = 0; k < 7 && st == cudaSuccess; ++k)
                st = cudaMemcpyAsync(dst[k], part[c][k], len[c][k], cudaMemcpyDeviceToDevice, b->stream);
            if (st == cudaSuccess) st = cudaMemsetAsync(s->d_err, 0, sizeof(int), b->stream);
        }
        return st;
    }
};

// Whole-step refinement (FP32, graph mode): the per-kernel timing of
// alelb_batch_tune does not see how a launch form fares inside a replayed
// step (its moments pass, its overlap with its neighbours, the other case
// group's kernels beside it), so each candidate (apply(j), j = 0 .. n - 1,
// candidate 0 the current form) runs REFINE_STEPS steps twice from the
// same saved state, the second run timed; the fastest is applied and the
// state put back, so no case advances.  A batch in which a case has
// already failed keeps its form.
constexpr int REFINE_STEPS = 8;
template <class Apply> cudaError_t refine_whole_steps(alelb_batch *b, int n, Apply apply)
{
    int err0 = 0;
    for (alelb_solver *s : b->cs) {
        int e = 0;
        cudaError_t st = cudaMemcpy(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (st != cudaSuccess) return st;
        err0 |= e;
    }
    if (err0) return cudaSuccess;
    Snapshot snap;
    cudaError_t st = snap.take(b);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == cudaSuccess) st = cudaEventCreate(&e0);
    if (st == cudaSuccess) st = cudaEventCreate(&e1);
    float best = 1e30f;
    int pick = 0;
    for (int j = 0; j < n && st == cudaSuccess; ++j) {
        apply(j);
        drop_graphs(b);
        float ms = 0.f;
        for (int r = 0; r < 2 && st == cudaSuccess; ++r) {
            st = cudaEventRecord(e0, b->stream);
            if (st == cudaSuccess) st = run_steps(b, REFINE_STEPS);
            if (st == cudaSuccess) st = cudaEventRecord(e1, b->stream);
            if (st == cudaSuccess) st = snap.put(b);
            if (st == cudaSuccess) st = cudaEventSynchronize(e1);
            if (st == cudaSuccess) st = cudaEventElapsedTime(&ms, e0, e1);
        }
        if (st == cudaSuccess && ms < best) {
            best = ms;
            pick = j;
        }
    }
    apply(pick);
    drop_graphs(b);
    if (st == cudaSuccess) st = cudaStreamSynchronize(b->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    snap.buf.release();
    return st;
}

// The propagation's form: G = 3 and 9, plain and fused with the moments,
// at 128 and 256 threads, and the per-kernel pick.
cudaError_t refine_fast_form(alelb_batch *b)
{
    struct Form { int g, bs; };
    std::vector<Form> forms = {{b->fast_g, b->bs[KT_FAST]}};
    for (int g : {3, 9, 3 | FAST_FUSED, 9 | FAST_FUSED})
        for (int bs : {128, 256})
            if (!(g == b->fast_g && bs == b->bs[KT_FAST])) forms.push_back({g, bs});
    return refine_whole_steps(b, (int)forms.size(), [&](int j) {
        b->fast_g = forms[j].g;
        b->bs[KT_FAST] = forms[j].bs;
    });
}

// The case groups: all cases as one, two or four groups running free, or
// with their propagations in turn (pipe 1 and 2).
cudaError_t refine_groups(alelb_batch *b)
{
    if (!b->has2) return cudaSuccess;
    const int cand[7][2] = {{1, 0}, {2, 0}, {2, 1}, {2, 2}, {4, 0}, {4, 1}, {4, 2}};
    return refine_whole_steps(b, b->has4 ? 7 : 4, [&](int j) {
        b->groups = cand[j][0];
        b->pipe = cand[j][1];
    });
}
} // namespace

extern "C" alelb_status alelb_batch_step(alelb_batch *b, int32_t n)
{
    if (!b || n < 0) return ALELB_ERR_ARG;
    if (n == 0) return ALELB_OK;
    cudaError_t st = join_cases(b);
    if (st != cudaSuccess) return bfail(b, st, "batch_step");
    st = run_steps(b, n);
    if (st != cudaSuccess) return bfail(b, st, "batch_step: launch");
    for (alelb_solver *s : b->cs) {
        s->t += (double)n;
        s->nstep += n;
    }
    st = release_cases(b);
    if (st != cudaSuccess) return bfail(b, st, "batch_step");
    return ALELB_OK;
}

extern "C" alelb_status alelb_batch_sync(alelb_batch *b)
{
    if (!b) return ALELB_ERR_ARG;
    cudaError_t st = cudaStreamSynchronize(b->stream);
    if (st != cudaSuccess) return bfail(b, st, "batch_sync");
    if (b->prof) bflush_prof(b);
    for (int c = 0; c < b->B; ++c) {
        alelb_solver *s = b->cs[c];
        int e = 0;
        st = cudaMemcpy(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (st != cudaSuccess) return bfail(b, st, "batch_sync");
        s->sticky |= e;
        const alelb_status r = check_sticky(s);
        if (r != ALELB_OK) {
            b->err = "case " + std::to_string(c) + ": " + s->err;
            return r;
        }
    }
    return ALELB_OK;
}

extern "C" alelb_status alelb_batch_tune(alelb_batch *b, int32_t reps, int32_t choice[8])
{
    if (!b || reps < 1 || reps > 16) return ALELB_ERR_ARG;
    cudaError_t st = join_cases(b);
    if (st == cudaSuccess) st = stage_scalars(b, 0, 1);
    if (st != cudaSuccess) return bfail(b, st, "batch_tune");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    st = cudaEventCreate(&e0);
    if (st == cudaSuccess) st = cudaEventCreate(&e1);
    if (st != cudaSuccess) return bfail(b, st, "batch_tune");
    int seq[KT_N];
    const int ns = step_sequence(b, seq);
    const auto clear = [b]() {
        if (b->prec == ALELB_PREC_FP32_DEV)
            kb_clear_work<float, float>
                <<<b->B, 256, 0, b->stream>>>(reinterpret_cast<const CaseDev<float, float> *>(b->d_cases), b->B);
        else
            kb_clear_work<double, double>
                <<<b->B, 256, 0, b->stream>>>(reinterpret_cast<const CaseDev<double, double> *>(b->d_cases), b->B);
    };
    for (int q = 0; q < ns && st == cudaSuccess; ++q) {
        const int kt = seq[q];
        struct Cand { int bs, grid, g; bool stage; };
        std::vector<Cand> cands;
        const bool stageable = (kt == KT_DERIV1 || kt == KT_COLLIDE) && b->prec == ALELB_PREC_FP32_DEV;
        for (int bsq = 0; bsq < N_BS; ++bsq) {
            const int bs = 64 << bsq;
            if (kt == KT_SLOW) {
                for (int gm = 1; gm <= 16; gm *= 2) cands.push_back({bs, gm * b->n_sm, b->fast_g, false});
                cands.push_back({bs, slow_resident(b, bs) * b->n_sm, b->fast_g, false}); // one wave
            } else if (kt == KT_FAST) {
                for (int g : {1, 3, 9}) cands.push_back({bs, 0, g, false});
                if (b->prec == ALELB_PREC_FP32_DEV)
                    for (int g : {3 | FAST_FUSED, 9 | FAST_FUSED}) cands.push_back({bs, 0, g, false});
            } else {
                cands.push_back({bs, 0, b->fast_g, false});
                if (stageable) cands.push_back({bs, 0, b->fast_g, true});
            }
        }
        float best = 1e30f;
        Cand pick = {b->bs[kt], b->slow_grid, b->fast_g, b->stage[kt]};
        for (const Cand &cd : cands) {
            float tmin = 1e30f;
            for (int r = 0; r < reps && st == cudaSuccess; ++r) {
                if (kt == KT_FAST) clear();
                st = cudaEventRecord(e0, b->stream);
                launch_kernel(b, kt, cd.bs, cd.grid, 0, 0, cd.g, cd.stage);
                // a propagation candidate is timed with the moments launch it
                // implies (the fused form leaves kb_moments only the nodes it
                // marked pending)
                if (kt == KT_FAST && b->prec == ALELB_PREC_FP32_DEV)
                    launch_kernel(b, KT_MOMENTS, b->bs[KT_MOMENTS], 0, 0, 0, cd.g, false);
                if (st == cudaSuccess) st = cudaGetLastError();
                if (st == cudaSuccess) st = cudaEventRecord(e1, b->stream);
                if (st == cudaSuccess) st = cudaEventSynchronize(e1);
                float ms = 0;
                if (st == cudaSuccess) st = cudaEventElapsedTime(&ms, e0, e1);
                tmin = std::min(tmin, ms);
            }
            if (tmin < best) {
                best = tmin;
                pick = cd;
            }
        }
        if (st != cudaSuccess) break;
        b->bs[kt] = pick.bs;
        if (kt == KT_SLOW) b->slow_grid = pick.grid;
        if (kt == KT_FAST) b->fast_g = pick.g;
        b->stage[kt] = pick.stage;
        // the launch that counts (walk statistics) with the chosen shape
        if (kt == KT_FAST) clear();
        launch_kernel(b, kt, pick.bs, pick.grid, 0, 1, b->fast_g, b->stage[kt]);
        st = cudaGetLastError();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == cudaSuccess) st = cudaStreamSynchronize(b->stream);
    if (st != cudaSuccess) return bfail(b, st, "batch_tune");
    for (alelb_solver *s : b->cs) {
        s->t += 1.0;
        s->nstep += 1;
    }
    drop_graphs(b);
    if (b->prec == ALELB_PREC_FP32_DEV && b->mode == ALELB_BATCH_GRAPHS && !b->prof) {
        st = refine_fast_form(b);
        if (st == cudaSuccess) st = refine_groups(b);
        if (st != cudaSuccess) return bfail(b, st, "batch_tune: refinement");
    }
    st = release_cases(b);
    if (st != cudaSuccess) return bfail(b, st, "batch_tune");
    if (choice) {
        for (int k = 0; k < 6; ++k) choice[k] = b->bs[k];
        choice[6] = b->slow_grid;
        choice[7] = b->fast_g | (b->stage[KT_DERIV1] ? 16 : 0) | (b->stage[KT_COLLIDE] ? 32 : 0) |
                    (b->groups == 2 ? TWO_GROUPS : b->groups == 4 ? FOUR_GROUPS : 0) |
                    b->pipe * PIPELINED; // FAST_FUSED = 256
    }
    return ALELB_OK;
}

extern "C" alelb_status alelb_batch_profile(alelb_batch *b, int32_t enable)
{
    if (!b) return ALELB_ERR_ARG;
    cudaStreamSynchronize(b->stream);
    bflush_prof(b);
    b->prof = enable != 0;
    for (int k = 0; k < KT_N; ++k) {
        b->ms_acc[k] = 0;
        b->n_acc[k] = 0;
    }
    return ALELB_OK;
}

extern "C" alelb_status alelb_batch_kernel_times(alelb_batch *b, const char **names, double *ms,
                                                 int64_t *launches, int32_t *n)
{
    if (!b || !n) return ALELB_ERR_ARG;
    cudaError_t st = cudaStreamSynchronize(b->stream);
    if (st != cudaSuccess) return bfail(b, st, "batch_kernel_times");
    bflush_prof(b);
    const int m = std::min<int>(*n, KT_N);
    for (int k = 0; k < m; ++k) {
        if (names) names[k] = KT_NAMES[k];
        if (ms) ms[k] = b->ms_acc[k];
        if (launches) launches[k] = b->n_acc[k];
    }
    *n = m;
    return ALELB_OK;
}

namespace {
// The batched host exchange: every case's copies and kernels are queued
// first (on its own streams, so that the copies of different cases
// overlap), then the batch's stream joins all of them and one wait covers
// the lot.  enqueue(c) queues case c's part.
template <class Enqueue> alelb_status batch_set(alelb_batch *b, Enqueue enqueue, const double *t, const char *what)
{
    cudaError_t st = cudaSuccess;
    for (int c = 0; c < b->B && st == cudaSuccess; ++c) st = enqueue(c);
    if (st == cudaSuccess) st = join_cases(b);
    const cudaError_t sw = cudaStreamSynchronize(b->stream);
    if (st == cudaSuccess) st = sw;
    if (st != cudaSuccess) {
        for (int c = 0; c < b->B; ++c) cudaStreamSynchronize(b->cs[c]->stream);
        return bfail(b, st, what);
    }
    if (t)
        for (int c = 0; c < b->B; ++c) b->cs[c]->t = t[c];
    return ALELB_OK;
}

// The same for reading; each case's error word comes back with its arrays.
template <class Enqueue> alelb_status batch_get(alelb_batch *b, Enqueue enqueue, const char *what)
{
    cudaError_t st = cudaSuccess;
    for (int c = 0; c < b->B && st == cudaSuccess; ++c) {
        alelb_solver *s = b->cs[c];
        st = enqueue(c);
        if (st == cudaSuccess)
            st = cudaMemcpyAsync(b->h_err + c, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    }
    if (st == cudaSuccess) st = join_cases(b);
    const cudaError_t sw = cudaStreamSynchronize(b->stream);
    if (st == cudaSuccess) st = sw;
    if (st != cudaSuccess) {
        for (int c = 0; c < b->B; ++c) cudaStreamSynchronize(b->cs[c]->stream);
        return bfail(b, st, what);
    }
    for (int c = 0; c < b->B; ++c) {
        alelb_solver *s = b->cs[c];
        s->sticky |= b->h_err[c];
        const alelb_status r = check_sticky(s);
        if (r != ALELB_OK) {
            b->err = "case " + std::to_string(c) + ": " + s->err;
            return r;
        }
    }
    return ALELB_OK;
}

template <class P> bool all_set(const alelb_batch *b, P *const *f, P *const *g)
{
    if (!f || !g) return false;
    for (int c = 0; c < b->B; ++c)
        if (!f[c] || !g[c]) return false;
    return true;
}
} // namespace

extern "C" alelb_status alelb_batch_set_pops(alelb_batch *b, const double *const *f, const double *const *g,
                                             const double *t)
{
    if (!b || !all_set(b, f, g)) return ALELB_ERR_ARG;
    return batch_set(b, [&](int c) { return import_enqueue(b->cs[c], f[c], g[c], nullptr, nullptr, nullptr, nullptr); },
                     t, "batch_set_pops");
}

extern "C" alelb_status alelb_batch_get_pops(alelb_batch *b, double *const *f, double *const *g)
{
    if (!b || !all_set(b, f, g)) return ALELB_ERR_ARG;
    return batch_get(b, [&](int c) { return export_enqueue(b->cs[c], f[c], g[c], nullptr); }, "batch_get_pops");
}

extern "C" alelb_status alelb_batch_set_pops_stored(alelb_batch *b, const float *const *f, const float *const *g,
                                                   const double *t)
{
    if (!b || !all_set(b, f, g) || b->prec != ALELB_PREC_FP32_DEV) return ALELB_ERR_ARG;
    return batch_set(b, [&](int c) { return import_stored_enqueue(b->cs[c], f[c], g[c]); }, t,
                     "batch_set_pops_stored");
}

extern "C" alelb_status alelb_batch_get_pops_stored(alelb_batch *b, float *const *f, float *const *g)
{
    if (!b || !all_set(b, f, g) || b->prec != ALELB_PREC_FP32_DEV) return ALELB_ERR_ARG;
    return batch_get(b, [&](int c) { return export_stored_enqueue(b->cs[c], f[c], g[c]); },
                     "batch_get_pops_stored");
}

// One step with the state in host memory, pipelined by case group: the
// groups' uploads run one group after another (a group's copies wait until
// the previous group's are in: the copy engine would otherwise interleave
// every case's copies, and no group would be ready before all of them);
// each group's phase kernels start on the group's stream once its own
// cases are in, and each case's read-back once its group's step is done,
// so that the uploads of later groups, the steps and the read-back of
// earlier ones overlap (the host link carries both directions at once).
// Per case the same kernels as set_pops_stored, one batch step and
// get_pops_stored.
extern "C" alelb_status alelb_batch_step_host(alelb_batch *b, const float *const *f_in, const float *const *g_in,
                                              float *const *f_out, float *const *g_out, const double *t)
{
    if (!b || !all_set(b, f_in, g_in) || !all_set(b, f_out, g_out) || b->prec != ALELB_PREC_FP32_DEV)
        return ALELB_ERR_ARG;
    if (t)
        for (int c = 0; c < b->B; ++c) b->cs[c]->t = t[c];
    const int P = b->has8 ? 8 : b->has4 ? 4 : b->has2 ? 2 : 1;
    const auto part = [&](int g) {
        Part G = P > 1 ? group(b, P, g, false) : whole(b);
        G.pdl = false; // its first kernel follows waits on other streams
        return G;
    };
    cudaError_t st = stage_scalars(b, 0, 1); // the map scalars of time t_c + 1
    if (st == cudaSuccess) st = cudaEventRecord(b->gev_fork, b->stream);
    int seq[KT_N];
    const int ns = step_sequence(b, seq);
    for (int g = 0; g < P && st == cudaSuccess; ++g) {
        Part G = part(g);
        // the group's uploads, after the previous group's
        for (int j = G.c0; j < G.c0 + G.B && st == cudaSuccess; ++j) {
            const int u = b->ord[j];
            if (g > 0) st = cudaStreamWaitEvent(b->cs[u]->stream, b->gev_up[g - 1], 0);
            if (st == cudaSuccess) st = import_stored_enqueue(b->cs[u], f_in[u], g_in[u]);
        }
        // the group's stream waits for them (and the scalars)
        if (st == cudaSuccess) st = cudaStreamWaitEvent(G.stream, b->gev_fork, 0);
        for (int j = G.c0; j < G.c0 + G.B && st == cudaSuccess; ++j) {
            const int u = b->ord[j];
            st = cudaEventRecord(b->ev_in[u], b->cs[u]->stream);
            if (st == cudaSuccess) st = cudaStreamWaitEvent(G.stream, b->ev_in[u], 0);
        }
        if (st == cudaSuccess) st = cudaEventRecord(b->gev_up[g], G.stream);
        for (int q = 0; q < ns && st == cudaSuccess; ++q) {
            const int kt = seq[q];
            launch_kernel(b, G, kt, b->bs[kt], b->slow_grid, 0, 1, b->fast_g, b->stage[kt]);
            G.pdl = true;
            st = cudaGetLastError();
        }
        if (st == cudaSuccess) st = cudaEventRecord(b->gev_fast[g], G.stream);
        for (int j = G.c0; j < G.c0 + G.B && st == cudaSuccess; ++j) {
            const int u = b->ord[j];
            alelb_solver *s = b->cs[u];
            st = cudaStreamWaitEvent(s->stream, b->gev_fast[g], 0);
            if (st == cudaSuccess) st = export_stored_enqueue(s, f_out[u], g_out[u]);
            if (st == cudaSuccess)
                st = cudaMemcpyAsync(b->h_err + u, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
        }
    }
    // the batch's stream after every case (so later batch calls follow), one wait
    if (st == cudaSuccess) st = join_cases(b);
    const cudaError_t sw = cudaStreamSynchronize(b->stream);
    if (st == cudaSuccess) st = sw;
    if (st != cudaSuccess) {
        for (int c = 0; c < b->B; ++c) cudaStreamSynchronize(b->cs[c]->stream);
        for (int g = 1; g < GROUPS_MAX; ++g)
            if (b->gstream[g]) cudaStreamSynchronize(b->gstream[g]);
        return bfail(b, st, "batch_step_host");
    }
    for (alelb_solver *s : b->cs) {
        s->t += 1.0;
        s->nstep += 1;
    }
    for (int c = 0; c < b->B; ++c) {
        alelb_solver *s = b->cs[c];
        s->sticky |= b->h_err[c];
        const alelb_status r = check_sticky(s);
        if (r != ALELB_OK) {
            b->err = "case " + std::to_string(c) + ": " + s->err;
            return r;
        }
    }
    return ALELB_OK;
}

extern "C" alelb_status alelb_batch_set_choice(alelb_batch *b, const int32_t choice[8])
{
    if (!b || !choice) return ALELB_ERR_ARG;
    for (int k = 0; k < 6; ++k)
        if (choice[k] != 64 && choice[k] != 128 && choice[k] != 256) return ALELB_ERR_ARG;
    if (choice[6] < 1 || choice[6] > 64 * b->n_sm) return ALELB_ERR_ARG;
    const int c7 = choice[7], G = c7 & 15, fl = c7 & ~15 & ~(TWO_GROUPS | FOUR_GROUPS | 3 * PIPELINED);
    const bool fp32 = b->prec == ALELB_PREC_FP32_DEV;
    if (G != 1 && G != 3 && G != 9) return ALELB_ERR_ARG;
    if (fl & ~(16 | 32 | FAST_FUSED)) return ALELB_ERR_ARG;
    if (!fp32 && fl) return ALELB_ERR_ARG;
    const int form = fl & FAST_FUSED;
    if (form && G == 1) return ALELB_ERR_ARG;
    if ((c7 & TWO_GROUPS) && (c7 & FOUR_GROUPS)) return ALELB_ERR_ARG;
    const int groups = c7 & TWO_GROUPS ? 2 : c7 & FOUR_GROUPS ? 4 : 1, pipe = (c7 / PIPELINED) & 3;
    if ((groups == 2 && !b->has2) || (groups == 4 && !b->has4) || pipe == 3 || (pipe && groups == 1))
        return ALELB_ERR_ARG;
    cudaError_t st = cudaStreamSynchronize(b->stream);
    if (st != cudaSuccess) return bfail(b, st, "batch_set_choice");
    for (int k = 0; k < 6; ++k) b->bs[k] = choice[k];
    b->slow_grid = choice[6];
    b->fast_g = G | form;
    b->stage[KT_DERIV1] = (c7 & 16) != 0;
    b->stage[KT_COLLIDE] = (c7 & 32) != 0;
    b->groups = groups;
    b->pipe = pipe;
    drop_graphs(b);
    return ALELB_OK;
}

extern "C" alelb_status alelb_batch_set_mode(alelb_batch *b, int32_t mode)
{
    if (!b || (mode != ALELB_BATCH_GRAPHS && mode != ALELB_BATCH_PERSISTENT)) return ALELB_ERR_ARG;
    cudaError_t st = cudaStreamSynchronize(b->stream);
    if (st != cudaSuccess) return bfail(b, st, "batch_set_mode");
    b->mode = mode;
    return ALELB_OK;
}

extern "C" alelb_status alelb_batch_set_wait(alelb_batch *b, double limit_seconds, int32_t missing_arrivals)
{
    if (!b || !(limit_seconds > 0.0) || limit_seconds > 60.0 || missing_arrivals < 0 || missing_arrivals > 1)
        return ALELB_ERR_ARG;
    cudaError_t st = cudaStreamSynchronize(b->stream);
    if (st != cudaSuccess) return bfail(b, st, "batch_set_wait");
    b->wait_limit_s = limit_seconds;
    b->missing = missing_arrivals;
    return ALELB_OK;
}
