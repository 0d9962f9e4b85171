// mlp.cu -- the learned departure-element proposal (alelb_mlp_*,
// alelb_samples, alelb_solver_set_mlp in include/alelb.h).
//
//   k_samples      training data from the solver itself: for every query
//                  (node, direction) its features and the slot of the exact
//                  element (FP64 departure point, exact walk) in the node's
//                  ring, with the barycentric coordinates there
//   k_mlp_fwd_bwd  forward and backward pass over a tile of 64 samples per
//                  block on the CUDA cores (FP16-rounded weights, FP32
//                  arithmetic), weight gradients summed into one FP32 vector
//   k_mlp_adam     Adam update of the FP32 master weights, FP16 copies
//   k_propose      inference for the work list of the exact path: 16 queries
//                  per warp through the three layers with FP16 tensor-core
//                  MMA (mma.sync m16n8k16, FP32 accumulation)
//   k_mlp_predict  the same inference on given features (tests)
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "mlp.cuh"

using namespace alelb;

namespace {

constexpr int TS = 64;        // samples per training block
constexpr int TRAIN_THREADS = 256;
constexpr int PRED_WARPS = 4; // warps per inference block

// ---------------------------------------------------------------------------
// training data
// ---------------------------------------------------------------------------
__global__ void k_samples(MeshDev M, MapStatic MS, MapScalars sc, MapScalarsF sf, int flags,
                          float *feat, int16_t *slot, float *bary, uint8_t *nring, int *err)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = M.N;
    if (a >= N) return;
    const double2 Xa = M.X[a];
    const FastMap F = fast_map(MS, sf, a, M.Xf[a]);
    double xX, xY, yX, yY, Vx, Vy, a11, a12, a21, a22, wx, wy;
    map_node(MS, sc, a, Xa.x, Xa.y, xX, xY, yX, yY, Vx, Vy);
    metric_inverse_T(xX, xY, yX, yY, a11, a12, a21, a22);
    const int literal = (flags & FLAG_LITERAL_VG) != 0;
    mesh_velocity_term(a11, a12, a21, a22, ds(Vx, sc.Ux), ds(Vy, sc.Uy), literal != 0, wx, wy);
    const int r0 = M.ring_ptr[a], r1 = M.ring_ptr[a + 1];
    for (int i = 0; i < NQ; ++i) {
        const size_t q = (size_t)i * N + a;
        float f[MLP_IN];
        const int nr = mlp_features(M, F, a, i, f);
        for (int k = 0; k < MLP_IN; ++k) feat[q * MLP_IN + k] = f[k];
        nring[q] = (uint8_t)nr;
        int s = -1;
        double l0 = 0, xi = 0, eta = 0;
        double chx, chy, px, py;
        departure(a11, a12, a21, a22, wx, wy, (double)c_cx[i], (double)c_cy[i], Xa.x, Xa.y, chx, chy,
                  px, py);
        if (F.ok && !literal && !(chx == 0.0 && chy == 0.0)) {
            const Loc L = walk(M, a, Xa.x, Xa.y, px, py, err);
            if (L.e >= 0 && L.vnode < 0 && L.sx == 0 && L.sy == 0) {
                const int code = L.e | (1 << 28) | (1 << 30);
                for (int j = r0; j < r1; ++j)
                    if (M.ring[j] == code) s = j - r0;
                if (s >= 0) {
                    local_coords(M, L.e, 0, 0, px, py, xi, eta);
                    l0 = 1.0 - xi - eta;
                }
            }
        }
        slot[q] = (int16_t)s;
        bary[q * 3 + 0] = (float)l0;
        bary[q * 3 + 1] = (float)xi;
        bary[q * 3 + 2] = (float)eta;
    }
}

// ---------------------------------------------------------------------------
// training
// ---------------------------------------------------------------------------
__global__ void k_mlp_to_half(const float *w, __half *h, int n)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) h[p] = __float2half_rn(w[p]);
}

// Sample of minibatch position k: (mul * (base + k) + add) mod n, a
// permutation of 0..n-1 when gcd(mul, n) = 1.
__device__ __forceinline__ int64_t sample_index(int64_t k, int64_t n, int64_t mul, int64_t add)
{
    // n < 2^31, so mul * k + add < 2^63
    return (int64_t)(((uint64_t)mul * (uint64_t)k + (uint64_t)add) % (uint64_t)n);
}

__global__ void __launch_bounds__(TRAIN_THREADS)
k_mlp_fwd_bwd(const __half *__restrict__ Wh, const float *__restrict__ feat,
              const int16_t *__restrict__ slot, const float *__restrict__ bary,
              const uint8_t *__restrict__ nring, int64_t n, int64_t base, int cnt, int64_t mul,
              int64_t add, float w_bary, float *__restrict__ grad, double *__restrict__ loss_sum)
{
    extern __shared__ float sm[];
    float *W = sm;                       // MLP_NP
    float *X = W + MLP_NP;               // TS x 6
    float *H1 = X + TS * MLP_IN;         // TS x 64
    float *H2 = H1 + TS * MLP_H;         // TS x 64, later dA1
    float *O = H2 + TS * MLP_H;          // TS x 35, later dO
    float *dA2 = O + TS * MLP_OUT;       // TS x 64
    float *B = dA2 + TS * MLP_H;         // TS x 3
    int *SL = (int *)(B + TS * 3);       // TS
    int *NR = SL + TS;                   // TS
    const int tid = threadIdx.x;
    const int t0 = blockIdx.x * TS;      // first sample of this tile within the minibatch
    const int nt = min(TS, cnt - t0);    // samples in this tile
    for (int p = tid; p < MLP_NP; p += blockDim.x) W[p] = __half2float(Wh[p]);
    for (int s = tid; s < TS; s += blockDim.x) {
        if (s < nt) {
            const int64_t q = sample_index(base + t0 + s, n, mul, add);
            for (int k = 0; k < MLP_IN; ++k) X[s * MLP_IN + k] = feat[q * MLP_IN + k];
            for (int k = 0; k < 3; ++k) B[s * 3 + k] = bary[q * 3 + k];
            SL[s] = slot[q];
            NR[s] = nring[q];
        } else {
            for (int k = 0; k < MLP_IN; ++k) X[s * MLP_IN + k] = 0.0f;
            for (int k = 0; k < 3; ++k) B[s * 3 + k] = 0.0f;
            SL[s] = 0;
            NR[s] = 1;
        }
    }
    __syncthreads();
    const float *W1 = W + MLP_OFF_W1, *b1 = W + MLP_OFF_B1, *W2 = W + MLP_OFF_W2, *b2 = W + MLP_OFF_B2;
    const float *W3 = W + MLP_OFF_W3, *b3 = W + MLP_OFF_B3;
    for (int o = tid; o < TS * MLP_H; o += blockDim.x) {
        const int s = o / MLP_H, j = o % MLP_H;
        float z = b1[j];
        for (int k = 0; k < MLP_IN; ++k) z += W1[j * MLP_IN + k] * X[s * MLP_IN + k];
        H1[o] = tanhf(z);
    }
    __syncthreads();
    for (int o = tid; o < TS * MLP_H; o += blockDim.x) {
        const int s = o / MLP_H, j = o % MLP_H;
        float z = b2[j];
        for (int k = 0; k < MLP_H; ++k) z += W2[j * MLP_H + k] * H1[s * MLP_H + k];
        H2[o] = tanhf(z);
    }
    __syncthreads();
    for (int o = tid; o < TS * MLP_OUT; o += blockDim.x) {
        const int s = o / MLP_OUT, j = o % MLP_OUT;
        float z = b3[j];
        for (int k = 0; k < MLP_H; ++k) z += W3[j * MLP_H + k] * H2[s * MLP_H + k];
        O[o] = z;
    }
    __syncthreads();
    // loss and dO per sample (in place)
    float ls = 0.0f;
    if (tid < TS) {
        const int s = tid;
        float *o = O + s * MLP_OUT;
        if (s < nt) {
            const int nr = NR[s], sl = SL[s];
            float m = -INFINITY;
            for (int j = 0; j < nr; ++j) m = fmaxf(m, o[j]);
            float Z = 0.0f;
            for (int j = 0; j < nr; ++j) Z += expf(o[j] - m);
            const float lz = logf(Z);
            const float ce = -(o[sl] - m - lz);
            float mse = 0.0f;
            for (int k = 0; k < 3; ++k) {
                const float g = o[MLP_K + k] - B[s * 3 + k];
                mse += g * g;
                o[MLP_K + k] = w_bary * 2.0f * g / (3.0f * (float)cnt);
            }
            for (int j = 0; j < MLP_K; ++j) {
                const float p = j < nr ? expf(o[j] - m - lz) : 0.0f;
                o[j] = (p - (j == sl ? 1.0f : 0.0f)) / (float)cnt;
            }
            ls = ce + w_bary * mse / 3.0f;
        } else {
            for (int j = 0; j < MLP_OUT; ++j) o[j] = 0.0f;
        }
    }
    // block sum of the sample losses
    if (tid < 64) {
        for (int off = 16; off > 0; off >>= 1) ls += __shfl_down_sync(0xffffffffu, ls, off);
        if ((tid & 31) == 0) atomicAdd(loss_sum, (double)ls);
    }
    __syncthreads();
    // layer 3 gradients and dA2
    for (int o = tid; o < MLP_OUT * MLP_H; o += blockDim.x) {
        const int j = o / MLP_H, k = o % MLP_H;
        float g = 0.0f;
        for (int s = 0; s < nt; ++s) g += O[s * MLP_OUT + j] * H2[s * MLP_H + k];
        atomicAdd(grad + MLP_OFF_W3 + o, g);
    }
    for (int j = tid; j < MLP_OUT; j += blockDim.x) {
        float g = 0.0f;
        for (int s = 0; s < nt; ++s) g += O[s * MLP_OUT + j];
        atomicAdd(grad + MLP_OFF_B3 + j, g);
    }
    for (int o = tid; o < TS * MLP_H; o += blockDim.x) {
        const int s = o / MLP_H, k = o % MLP_H;
        float g = 0.0f;
        for (int j = 0; j < MLP_OUT; ++j) g += O[s * MLP_OUT + j] * W3[j * MLP_H + k];
        const float h = H2[o];
        dA2[o] = g * (1.0f - h * h);
    }
    __syncthreads();
    // layer 2 gradients and dA1 (into H2)
    for (int o = tid; o < MLP_H * MLP_H; o += blockDim.x) {
        const int j = o / MLP_H, k = o % MLP_H;
        float g = 0.0f;
        for (int s = 0; s < nt; ++s) g += dA2[s * MLP_H + j] * H1[s * MLP_H + k];
        atomicAdd(grad + MLP_OFF_W2 + o, g);
    }
    for (int j = tid; j < MLP_H; j += blockDim.x) {
        float g = 0.0f;
        for (int s = 0; s < nt; ++s) g += dA2[s * MLP_H + j];
        atomicAdd(grad + MLP_OFF_B2 + j, g);
    }
    for (int o = tid; o < TS * MLP_H; o += blockDim.x) {
        const int s = o / MLP_H, k = o % MLP_H;
        float g = 0.0f;
        for (int j = 0; j < MLP_H; ++j) g += dA2[s * MLP_H + j] * W2[j * MLP_H + k];
        const float h = H1[o];
        H2[o] = g * (1.0f - h * h);
    }
    __syncthreads();
    // layer 1 gradients
    for (int o = tid; o < MLP_H * MLP_IN; o += blockDim.x) {
        const int j = o / MLP_IN, k = o % MLP_IN;
        float g = 0.0f;
        for (int s = 0; s < nt; ++s) g += H2[s * MLP_H + j] * X[s * MLP_IN + k];
        atomicAdd(grad + MLP_OFF_W1 + o, g);
    }
    for (int j = tid; j < MLP_H; j += blockDim.x) {
        float g = 0.0f;
        for (int s = 0; s < nt; ++s) g += H2[s * MLP_H + j];
        atomicAdd(grad + MLP_OFF_B1 + j, g);
    }
}

constexpr size_t TRAIN_SMEM =
    sizeof(float) * (MLP_NP + TS * MLP_IN + 3 * TS * MLP_H + TS * MLP_OUT + TS * 3) + sizeof(int) * 2 * TS;

__global__ void k_mlp_adam(float *w, float *m, float *v, float *g, __half *h, int n, float lr,
                           float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float gp = g[p];
    const float mp = 0.9f * m[p] + 0.1f * gp;
    const float vp = 0.999f * v[p] + 0.001f * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float wp = w[p] - lr * (mp * c1) / (sqrtf(vp * c2) + 1e-8f);
    w[p] = wp;
    h[p] = __float2half_rn(wp);
    g[p] = 0.0f;
}

// ---------------------------------------------------------------------------
// inference on the tensor cores
// ---------------------------------------------------------------------------
struct PredSmem {
    __half W1[MLP_H][16];  // input padded 6 -> 16
    __half W2[MLP_H][MLP_H];
    __half W3[40][MLP_H];  // outputs padded 35 -> 40
    float b1[MLP_H], b2[MLP_H], b3[40];
    __half Xs[PRED_WARPS][16][16];
    float Os[PRED_WARPS][16][40];
};

__device__ __forceinline__ void load_pred_weights(PredSmem &S, const __half *__restrict__ Wh)
{
    for (int p = threadIdx.x; p < MLP_H * 16; p += blockDim.x) {
        const int j = p / 16, k = p % 16;
        S.W1[j][k] = k < MLP_IN ? Wh[MLP_OFF_W1 + j * MLP_IN + k] : __float2half_rn(0.0f);
    }
    for (int p = threadIdx.x; p < MLP_H * MLP_H; p += blockDim.x) S.W2[p / MLP_H][p % MLP_H] = Wh[MLP_OFF_W2 + p];
    for (int p = threadIdx.x; p < 40 * MLP_H; p += blockDim.x) {
        const int j = p / MLP_H, k = p % MLP_H;
        S.W3[j][k] = j < MLP_OUT ? Wh[MLP_OFF_W3 + p] : __float2half_rn(0.0f);
    }
    for (int p = threadIdx.x; p < MLP_H; p += blockDim.x) {
        S.b1[p] = __half2float(Wh[MLP_OFF_B1 + p]);
        S.b2[p] = __half2float(Wh[MLP_OFF_B2 + p]);
    }
    for (int p = threadIdx.x; p < 40; p += blockDim.x) S.b3[p] = p < MLP_OUT ? __half2float(Wh[MLP_OFF_B3 + p]) : 0.0f;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t lds32(const __half *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The network on the 16 queries of this warp's tile: features in
// S.Xs[w] (FP16, rows 0..15), outputs to S.Os[w] (FP32).  All 32 lanes.
__device__ __forceinline__ void warp_forward(PredSmem &S, int w)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t A[4][4];
    float c[8][4];
    {
        uint32_t a0[4] = {lds32(&S.Xs[w][g][2 * t]), lds32(&S.Xs[w][g + 8][2 * t]),
                          lds32(&S.Xs[w][g][8 + 2 * t]), lds32(&S.Xs[w][g + 8][8 + 2 * t])};
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = nt * 8 + 2 * t;
            c[nt][0] = c[nt][2] = S.b1[col];
            c[nt][1] = c[nt][3] = S.b1[col + 1];
            mma16816(c[nt], a0, lds32(&S.W1[nt * 8 + g][2 * t]), lds32(&S.W1[nt * 8 + g][8 + 2 * t]));
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        A[q][0] = pack2(tanhf(c[2 * q][0]), tanhf(c[2 * q][1]));
        A[q][1] = pack2(tanhf(c[2 * q][2]), tanhf(c[2 * q][3]));
        A[q][2] = pack2(tanhf(c[2 * q + 1][0]), tanhf(c[2 * q + 1][1]));
        A[q][3] = pack2(tanhf(c[2 * q + 1][2]), tanhf(c[2 * q + 1][3]));
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
        c[nt][0] = c[nt][2] = S.b2[col];
        c[nt][1] = c[nt][3] = S.b2[col + 1];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            mma16816(c[nt], A[q], lds32(&S.W2[nt * 8 + g][16 * q + 2 * t]),
                     lds32(&S.W2[nt * 8 + g][16 * q + 8 + 2 * t]));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        A[q][0] = pack2(tanhf(c[2 * q][0]), tanhf(c[2 * q][1]));
        A[q][1] = pack2(tanhf(c[2 * q][2]), tanhf(c[2 * q][3]));
        A[q][2] = pack2(tanhf(c[2 * q + 1][0]), tanhf(c[2 * q + 1][1]));
        A[q][3] = pack2(tanhf(c[2 * q + 1][2]), tanhf(c[2 * q + 1][3]));
    }
#pragma unroll
    for (int nt = 0; nt < 5; ++nt) {
        const int col = nt * 8 + 2 * t;
        float d[4] = {S.b3[col], S.b3[col + 1], S.b3[col], S.b3[col + 1]};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            mma16816(d, A[q], lds32(&S.W3[nt * 8 + g][16 * q + 2 * t]),
                     lds32(&S.W3[nt * 8 + g][16 * q + 8 + 2 * t]));
        S.Os[w][g][col] = d[0];
        S.Os[w][g][col + 1] = d[1];
        S.Os[w][g + 8][col] = d[2];
        S.Os[w][g + 8][col + 1] = d[3];
    }
}

__device__ __forceinline__ int masked_argmax(const float *o, int nr)
{
    int best = 0;
    float bv = o[0];
    for (int j = 1; j < nr && j < MLP_K; ++j)
        if (o[j] > bv) {
            bv = o[j];
            best = j;
        }
    return best;
}

// Proposals for the work list of the exact path (after k_stream_fast):
// prop[w] = ring element of the largest logit, or -1 (no usable map).
template <class T>
__global__ void __launch_bounds__(PRED_WARPS * 32)
k_propose(MeshDev M, MapStatic MS, MapScalarsF sf, StateDev<T> st, const __half *__restrict__ Wh,
          int flags, int *prop, unsigned long long *made)
{
    wait_prior_grid();
    __shared__ PredSmem S;
    load_pred_weights(S, Wh);
    __syncthreads();
    __shared__ unsigned pre[NQ + 1];
    if (threadIdx.x == 0) work_prefix(st.wcount, pre);
    __syncthreads();
    const unsigned n = pre[NQ];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned nwarps = gridDim.x * PRED_WARPS;
    unsigned count = 0;
    for (unsigned base = (blockIdx.x * PRED_WARPS + w) * 16u; base < n; base += nwarps * 16u) {
        int a = -1, nr = 0;
        const unsigned q = base + (unsigned)lane;
        if (lane < 16) {
            float f[MLP_IN] = {0, 0, 0, 0, 0, 0};
            if (q < n) {
                const int code = work_at(st.work, M.N, pre, q);
                a = code / NQ;
                const int i = code % NQ;
                const FastMap F = fast_map(MS, sf, a, M.Xf[a]);
                const int r = mlp_features(M, F, a, i, f);
                nr = (F.ok && !(flags & FLAG_LITERAL_VG)) ? r : 0;
            }
            for (int k = 0; k < 16; ++k) S.Xs[w][lane][k] = __float2half_rn(k < MLP_IN ? f[k] : 0.0f);
        }
        __syncwarp();
        warp_forward(S, w);
        __syncwarp();
        if (lane < 16 && q < n) {
            int pc = -1;
            if (nr > 0) {
                pc = M.ring[M.ring_ptr[a] + masked_argmax(S.Os[w][lane], nr)];
                ++count;
            }
            prop[q] = pc;
        }
        __syncwarp();
    }
    for (int off = 16; off > 0; off >>= 1) count += __shfl_down_sync(0xffffffffu, count, off);
    if (lane == 0 && count && made) atomicAdd(made, (unsigned long long)count);
}

// Inference on given features (tests): slot of the largest logit among the
// first nring, and optionally all 35 outputs.
__global__ void __launch_bounds__(PRED_WARPS * 32)
k_mlp_predict(const __half *__restrict__ Wh, const float *__restrict__ feat,
              const uint8_t *__restrict__ nring, int64_t n, int32_t *pslot, float *out)
{
    __shared__ PredSmem S;
    load_pred_weights(S, Wh);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * PRED_WARPS;
    for (int64_t base = ((int64_t)blockIdx.x * PRED_WARPS + w) * 16; base < n; base += nwarps * 16) {
        const int64_t q = base + lane;
        if (lane < 16)
            for (int k = 0; k < 16; ++k)
                S.Xs[w][lane][k] = __float2half_rn(k < MLP_IN && q < n ? feat[q * MLP_IN + k] : 0.0f);
        __syncwarp();
        warp_forward(S, w);
        __syncwarp();
        if (lane < 16 && q < n) {
            const int nr = nring[q];
            pslot[q] = nr > 0 ? masked_argmax(S.Os[w][lane], nr) : -1;
            if (out)
                for (int j = 0; j < MLP_OUT; ++j) out[q * MLP_OUT + j] = S.Os[w][lane][j];
        }
        __syncwarp();
    }
}

uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

int64_t gcd64(int64_t a, int64_t b)
{
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

} // namespace

struct alelb_mlp {
    std::string err;
    float *d_w = nullptr, *d_m = nullptr, *d_v = nullptr, *d_g = nullptr;
    __half *d_h = nullptr;
    double *d_loss = nullptr;
    int64_t t = 0;
    cudaStream_t stream = nullptr;
    DevBuf buf;
};

namespace {

alelb_status mfail(alelb_mlp *m, cudaError_t st, const char *what)
{
    m->err = std::string(what) + ": " + cudaGetErrorString(st);
    return st == cudaErrorMemoryAllocation ? ALELB_ERR_OOM : ALELB_ERR_CUDA;
}

cudaError_t refresh_half(alelb_mlp *m)
{
    k_mlp_to_half<<<(MLP_NP + 255) / 256, 256, 0, m->stream>>>(m->d_w, m->d_h, MLP_NP);
    return cudaGetLastError();
}

cudaError_t fwd_bwd(alelb_mlp *m, const float *feat, const int16_t *slot, const float *bary,
                    const uint8_t *nring, int64_t n, int64_t base, int cnt, int64_t mul, int64_t add,
                    float w_bary)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t st = cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)TRAIN_SMEM);
        if (st != cudaSuccess) return st;
        attr = true;
    }
    const int blocks = (cnt + TS - 1) / TS;
    k_mlp_fwd_bwd<<<blocks, TRAIN_THREADS, TRAIN_SMEM, m->stream>>>(m->d_h, feat, slot, bary, nring, n, base,
                                                                     cnt, mul, add, w_bary, m->d_g,
                                                                     m->d_loss);
    return cudaGetLastError();
}

} // namespace

namespace alelb {

// Proposals for the solver's current work list (deviation-form step).
cudaError_t mlp_propose(alelb_solver *s, const MapScalarsF &sf)
{
    alelb_mesh *m = s->mesh;
    with_state(s, [&](auto &st, auto &) {
        k_propose<<<2 * s->n_sm, PRED_WARPS * 32, 0, s->stream>>>(m->dev, m->mst, sf, st, s->mlp->d_h, s->flags,
                                                                   s->d_prop, s->d_stats + 2);
    });
    return cudaGetLastError();
}

} // namespace alelb

extern "C" alelb_status alelb_mlp_create(const float *params, uint64_t seed, alelb_mlp **out)
{
    if (!out) return ALELB_ERR_ARG;
    alelb_mlp *m = new (std::nothrow) alelb_mlp();
    if (!m) return ALELB_ERR_OOM;
    *out = m;
    std::vector<float> w(MLP_NP);
    if (params) {
        for (int p = 0; p < MLP_NP; ++p) w[p] = params[p];
    } else {
        // Glorot-uniform weights, zero biases
        uint64_t x = seed;
        const int fan[3][2] = {{MLP_IN, MLP_H}, {MLP_H, MLP_H}, {MLP_H, MLP_OUT}};
        const int offw[3] = {MLP_OFF_W1, MLP_OFF_W2, MLP_OFF_W3};
        const int offb[3] = {MLP_OFF_B1, MLP_OFF_B2, MLP_OFF_B3};
        for (int l = 0; l < 3; ++l) {
            const double lim = std::sqrt(6.0 / (fan[l][0] + fan[l][1]));
            for (int p = 0; p < fan[l][0] * fan[l][1]; ++p) {
                const double u = (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0);
                w[offw[l] + p] = (float)((2.0 * u - 1.0) * lim);
            }
            for (int p = 0; p < fan[l][1]; ++p) w[offb[l] + p] = 0.0f;
        }
    }
    cudaError_t st = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
    m->d_w = m->buf.put(w, st);
    m->d_m = m->buf.alloc<float>(MLP_NP, st);
    m->d_v = m->buf.alloc<float>(MLP_NP, st);
    m->d_g = m->buf.alloc<float>(MLP_NP, st);
    m->d_h = m->buf.alloc<__half>(MLP_NP, st);
    m->d_loss = m->buf.alloc<double>(1, st);
    if (st == cudaSuccess) st = cudaMemset(m->d_m, 0, MLP_NP * sizeof(float));
    if (st == cudaSuccess) st = cudaMemset(m->d_v, 0, MLP_NP * sizeof(float));
    if (st == cudaSuccess) st = cudaMemset(m->d_g, 0, MLP_NP * sizeof(float));
    if (st == cudaSuccess) st = cudaDeviceSynchronize(); // legacy-stream uploads before m->stream work
    if (st == cudaSuccess) st = refresh_half(m);
    if (st == cudaSuccess) st = cudaStreamSynchronize(m->stream);
    if (st != cudaSuccess) return mfail(m, st, "mlp_create");
    return ALELB_OK;
}

extern "C" void alelb_mlp_destroy(alelb_mlp *m)
{
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    m->buf.release();
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

extern "C" const char *alelb_mlp_last_error(alelb_mlp *m) { return m ? m->err.c_str() : "null network"; }

extern "C" alelb_status alelb_mlp_get_params(alelb_mlp *m, int32_t rounded, float *params)
{
    if (!m || !params) return ALELB_ERR_ARG;
    cudaError_t st = cudaSuccess;
    if (rounded) {
        std::vector<__half> h(MLP_NP);
        st = cudaMemcpyAsync(h.data(), m->d_h, MLP_NP * sizeof(__half), cudaMemcpyDeviceToHost, m->stream);
        if (st == cudaSuccess) st = cudaStreamSynchronize(m->stream);
        if (st == cudaSuccess)
            for (int p = 0; p < MLP_NP; ++p) params[p] = __half2float(h[p]);
    } else {
        st = cudaMemcpyAsync(params, m->d_w, MLP_NP * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
        if (st == cudaSuccess) st = cudaStreamSynchronize(m->stream);
    }
    if (st != cudaSuccess) return mfail(m, st, "mlp_get_params");
    return ALELB_OK;
}

extern "C" alelb_status alelb_mlp_loss_grad(alelb_mlp *m, const float *feat, const int16_t *slot,
                                            const float *bary, const uint8_t *nring, int64_t n,
                                            float w_bary, double *loss, float *grad)
{
    if (!m || !feat || !slot || !bary || !nring || n < 1 || n > (1 << 30)) return ALELB_ERR_ARG;
    cudaError_t st = cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->stream);
    if (st == cudaSuccess) st = cudaMemsetAsync(m->d_g, 0, MLP_NP * sizeof(float), m->stream);
    if (st == cudaSuccess) st = fwd_bwd(m, feat, slot, bary, nring, n, 0, (int)n, 1, 0, w_bary);
    double ls = 0;
    if (st == cudaSuccess) st = cudaMemcpyAsync(&ls, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
    if (st == cudaSuccess && grad)
        st = cudaMemcpyAsync(grad, m->d_g, MLP_NP * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (st == cudaSuccess) st = cudaMemsetAsync(m->d_g, 0, MLP_NP * sizeof(float), m->stream);
    if (st == cudaSuccess) st = cudaStreamSynchronize(m->stream);
    if (st != cudaSuccess) return mfail(m, st, "mlp_loss_grad");
    if (loss) *loss = ls / (double)n;
    return ALELB_OK;
}

extern "C" alelb_status alelb_mlp_train(alelb_mlp *m, const float *feat, const int16_t *slot,
                                        const float *bary, const uint8_t *nring, int64_t n,
                                        int32_t epochs, int32_t batch, float lr, float w_bary,
                                        uint64_t seed, double *epoch_loss)
{
    if (!m || !feat || !slot || !bary || !nring || n < 1 || n > 2147483647LL || epochs < 0 || batch < 1 ||
        batch > (1 << 20) || !(lr > 0.0f))
        return ALELB_ERR_ARG;
    uint64_t x = seed;
    cudaError_t st = cudaSuccess;
    for (int ep = 0; ep < epochs && st == cudaSuccess; ++ep) {
        int64_t mul = 1 + (int64_t)(splitmix64(x) % (uint64_t)n);
        while (gcd64(mul, n) != 1) mul = mul % n + 1;
        const int64_t add = (int64_t)(splitmix64(x) % (uint64_t)n);
        st = cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->stream);
        for (int64_t base = 0; base < n && st == cudaSuccess; base += batch) {
            const int cnt = (int)std::min<int64_t>(batch, n - base);
            st = fwd_bwd(m, feat, slot, bary, nring, n, base, cnt, mul, add, w_bary);
            if (st != cudaSuccess) break;
            m->t += 1;
            const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)m->t)));
            const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)m->t)));
            k_mlp_adam<<<(MLP_NP + 255) / 256, 256, 0, m->stream>>>(m->d_w, m->d_m, m->d_v, m->d_g, m->d_h, MLP_NP,
                                                                   lr, c1, c2);
            st = cudaGetLastError();
        }
        double ls = 0;
        if (st == cudaSuccess)
            st = cudaMemcpyAsync(&ls, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
        if (st == cudaSuccess) st = cudaStreamSynchronize(m->stream);
        if (epoch_loss) epoch_loss[ep] = ls / (double)n;
    }
    if (st != cudaSuccess) return mfail(m, st, "mlp_train");
    return ALELB_OK;
}

extern "C" alelb_status alelb_mlp_predict(alelb_mlp *m, const float *feat, const uint8_t *nring, int64_t n,
                                          int32_t *slot, float *out)
{
    if (!m || !feat || !nring || !slot || n < 1) return ALELB_ERR_ARG;
    const int64_t tiles = (n + 15) / 16;
    const int blocks = (int)std::min<int64_t>((tiles + PRED_WARPS - 1) / PRED_WARPS, 4096);
    k_mlp_predict<<<blocks, PRED_WARPS * 32, 0, m->stream>>>(m->d_h, feat, nring, n, slot, out);
    cudaError_t st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaStreamSynchronize(m->stream);
    if (st != cudaSuccess) return mfail(m, st, "mlp_predict");
    return ALELB_OK;
}

extern "C" alelb_status alelb_samples(alelb_solver *s, double t, float *feat, int16_t *slot, float *bary,
                                      uint8_t *nring)
{
    if (!s || !s->mesh || !feat || !slot || !bary || !nring) return ALELB_ERR_ARG;
    alelb_mesh *m = s->mesh;
    if (m->etype != ALELB_ELEM_P2TRI) {
        s->err = "samples: the learned proposal serves 6-node triangle meshes";
        return ALELB_ERR_ARG;
    }
    const MapScalars sc = solver_map(s, map_scalars(m->T.mkind, m->T.mp, t));
    k_samples<<<(m->T.N + 127) / 128, 128, 0, s->stream>>>(m->dev, m->mst, sc, to_f32(sc, m->T), s->flags, feat,
                                                            slot, bary, nring, s->d_err);
    cudaError_t st = cudaGetLastError();
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) {
        s->err = cudaGetErrorString(st);
        return ALELB_ERR_CUDA;
    }
    return ALELB_OK;
}

extern "C" alelb_status alelb_solver_set_mlp(alelb_solver *s, alelb_mlp *m)
{
    if (!s) return ALELB_ERR_ARG;
    if (m && s->prec == ALELB_PREC_FP64) {
        s->err = "the learned proposal serves the deviation-form propagation only";
        return ALELB_ERR_ARG;
    }
    if (m && s->mesh->etype != ALELB_ELEM_P2TRI) {
        s->err = "the learned proposal serves 6-node triangle meshes";
        return ALELB_ERR_ARG;
    }
    if (m && !s->d_prop) {
        cudaError_t st = cudaSuccess;
        s->d_prop = s->buf.alloc<int>((size_t)9 * s->mesh->T.N, st);
        if (st != cudaSuccess) {
            s->err = cudaGetErrorString(st);
            return ALELB_ERR_OOM;
        }
    }
    // the network's weights are final once the solver's stream reaches this point
    if (m) cudaStreamSynchronize(m->stream);
    s->mlp = m;
    return ALELB_OK;
}

extern "C" alelb_status alelb_mlp_stats(alelb_solver *s, int64_t out[3])
{
    if (!s || !out) return ALELB_ERR_ARG;
    unsigned long long h[3] = {0, 0, 0};
    cudaError_t st = cudaMemcpyAsync(h, s->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) {
        s->err = cudaGetErrorString(st);
        return ALELB_ERR_CUDA;
    }
    out[0] = (int64_t)h[0]; // populations left to the exact path
    out[1] = (int64_t)h[2]; // proposals made
    out[2] = (int64_t)h[1]; // proposals accepted
    return ALELB_OK;
}
