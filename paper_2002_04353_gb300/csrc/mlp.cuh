// mlp.cuh -- layout and input features of the learned departure-element
// proposal (the paper has no counterpart: it locates every departure point
// by search).  A small network maps the features of a query (node a,
// direction i) to a slot of the node's neighbour ring; the proposed element
// is used only when the certified FP32 containment test accepts it, exactly
// as the previous-step element is, and the exact walk decides otherwise, so
// no element choice and no streamed value depends on the network.
#pragma once
#include "geom.cuh"

namespace alelb {

// 6 features -> 64 tanh -> 64 tanh -> 32 slot logits + 3 barycentric guesses
constexpr int MLP_IN = 6, MLP_H = 64, MLP_K = 32, MLP_OUT = 35;
// flat parameter vector: W1 [64][6], b1 [64], W2 [64][64], b2 [64], W3 [35][64], b3 [35]
constexpr int MLP_OFF_W1 = 0, MLP_OFF_B1 = 384, MLP_OFF_W2 = 448, MLP_OFF_B2 = 4544,
              MLP_OFF_W3 = 4608, MLP_OFF_B3 = 6848, MLP_NP = 6883;

// Features of query (a, i) from the FP32 map: the departure offset
// -c^_i in units of the node's length scale h (x, y, length, angle / pi),
// the node's number of own elements / 16 and its ring size / 32.  Returns
// the ring size.
ALELB_HD __forceinline__ int mlp_features(const MeshDev &M, const FastMap &F, int a, int i,
                                          float f[MLP_IN])
{
    const float cx = (float)lat_cx(i), cy = (float)lat_cy(i);
    const float chx = F.A11 * cx + F.A12 * cy - F.W1;
    const float chy = F.A21 * cx + F.A22 * cy - F.W2;
    const float2 ns = M.nscale[a];
    const float inv = 1.0f / ns.x;
    const float dx = -chx * inv, dy = -chy * inv;
    const int nring = M.ring_ptr[a + 1] - M.ring_ptr[a];
    f[0] = dx;
    f[1] = dy;
    f[2] = sqrtf(dx * dx + dy * dy);
    f[3] = atan2f(dy, dx) * 0.3183098861837907f;
    f[4] = ns.y * 0.0625f;
    f[5] = (float)nring * 0.03125f;
    return nring;
}

} // namespace alelb
