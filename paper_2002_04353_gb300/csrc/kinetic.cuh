// kinetic.cuh -- the two-population compressible kinetic model of Sec. IV
// on the D2Q9 lattice: equilibria (Eq. feq, Eq. geq_gstar with Table I),
// the BGK-type collision of Eqs. feqn/geqn with the correction phi_i, and
// the Grad-type missing populations of Sec. IV.A (Table II).
//
// Populations travel as deviations d_i = f_i - ref_i from a fixed
// reference state; with ref = 0 (FP64 mode) they are the populations
// themselves.  In FP32 mode ref_i = f^eq_i(rho_inf, 0, T_inf) and
// g^eq_i(rho_inf, 0, T_inf), which keeps the stored numbers small.
//
// Shifted lattice (Sec. V.D: velocities c_i + U; the model is deferred to
// another paper, so this is a reading): every population set carries the
// lab-frame moments it carries on the plain lattice.  f^eq is the product
// form in u - U; the general form of Eq. geq_gstar is applied to moments
// taken about U; psi restores the diagonal second central moments (the
// printed psi at U = 0); Q' is taken in u - U; phi_i = A_ia X_a stays on
// the relative velocities c_i.  Moments: rho u = sum (c_i + U) f_i.
#pragma once

namespace alelb {

template <class A> struct KinParams {
    using Arith = A; // the arithmetic type
    A Cv, Cp, mu, Pr;
    // moments of the reference populations: sum f_ref, sum c f_ref,
    // sum c c f_ref, sum g_ref
    A rho_ref, jx_ref, jy_ref, Pxx_ref, Pxy_ref, Pyy_ref, E2_ref;
    A fref[NQ], gref[NQ];           // reference populations (zero in FP64 mode)
    A finf[NQ], ginf[NQ];           // far-field populations minus the reference
    A Ux, Uy;                       // lattice shift U (zero on the plain lattice)
    int flags;
};

enum : int { FLAG_PHI_OFF = 1, FLAG_COLLIDE_OFF = 2, FLAG_LITERAL_VG = 4, FLAG_BC_EQ = 8, FLAG_SLIP = 16,
             FLAG_MIDPOINT = 32, FLAG_EXACT_CHAR = 64,
             FLAG_SHIFT = 128 /* internal: U != 0 */, FLAG_OFFWALL_VG = 256 };

// One-dimensional factors Phi_c(u, T) of Eq. feq.
template <class A> __device__ __forceinline__ void phi3(A u, A T, A &m, A &z, A &p)
{
    A u2T = u * u + T;
    m = (u2T - u) * A(0.5);
    z = A(1) - u2T;
    p = (u2T + u) * A(0.5);
}

// f^eq_i = rho Phi_cx Phi_cy.
template <class A> __device__ __forceinline__ void feq9(A rho, A ux, A uy, A T, A f[NQ])
{
    A xm, xz, xp, ym, yz, yp;
    phi3(ux, T, xm, xz, xp);
    phi3(uy, T, ym, yz, yp);
    f[0] = rho * xz * yz;
    f[1] = rho * xp * yz;
    f[2] = rho * xz * yp;
    f[3] = rho * xm * yz;
    f[4] = rho * xz * ym;
    f[5] = rho * xp * yp;
    f[6] = rho * xm * yp;
    f[7] = rho * xm * ym;
    f[8] = rho * xp * ym;
}

// General form G_i = W_i (M0 + M.c/T + (M - M0 T I):(cc - T I)/(2T^2)) + Psi_i,
// W_i = W_cx W_cy, W_0 = 1 - T, W_{+-1} = T/2.  psi_rest, psi_x, psi_y give
// Psi on the rest velocity and on the x- and y-axis velocities (zero on the
// diagonals).
template <class A>
__device__ __forceinline__ void gform9(A T, A M0, A Mx, A My, A Mxx, A Mxy, A Myy, A psi_rest,
                                       A psi_x, A psi_y, A G[NQ])
{
    A iT = A(1) / T;
    A h = A(0.5) * iT * iT;
    A Nxx = Mxx - M0 * T, Nyy = Myy - M0 * T;
    A W0 = A(1) - T, W1 = A(0.5) * T;
    // quadratic term q(cx, cy) = h (Nxx (cx^2 - T) + 2 Mxy cx cy + Nyy (cy^2 - T))
    A ax0 = -Nxx * T, ax1 = Nxx * (A(1) - T);
    A ay0 = -Nyy * T, ay1 = Nyy * (A(1) - T);
    A lx = Mx * iT, ly = My * iT;
    A Wr = W0 * W0, Wa = W0 * W1, Wd = W1 * W1;
    G[0] = Wr * (M0 + h * (ax0 + ay0)) + psi_rest;
    G[1] = Wa * (M0 + lx + h * (ax1 + ay0)) + psi_x;
    G[2] = Wa * (M0 + ly + h * (ax0 + ay1)) + psi_y;
    G[3] = Wa * (M0 - lx + h * (ax1 + ay0)) + psi_x;
    G[4] = Wa * (M0 - ly + h * (ax0 + ay1)) + psi_y;
    A c2 = A(2) * Mxy;
    G[5] = Wd * (M0 + lx + ly + h * (ax1 + ay1 + c2));
    G[6] = Wd * (M0 - lx + ly + h * (ax1 + ay1 - c2));
    G[7] = Wd * (M0 - lx - ly + h * (ax1 + ay1 + c2));
    G[8] = Wd * (M0 + lx - ly + h * (ax1 + ay1 - c2));
}

// psi_i = B_ia rho (1 - 3T)(T^2 + 2 u_a^2 T + E u_a^2)/T: B = 1 on the rest
// velocity (both a), -1/2 on the axis velocities along a, 0 on diagonals.
template <class A>
__device__ __forceinline__ void psi_terms(A rho, A ux, A uy, A T, A E, A &pr, A &px, A &py)
{
    A k = rho * (A(1) - A(3) * T) / T;
    A Yx = k * (T * T + (A(2) * T + E) * ux * ux);
    A Yy = k * (T * T + (A(2) * T + E) * uy * uy);
    pr = Yx + Yy;
    px = A(-0.5) * Yx;
    py = A(-0.5) * Yy;
}

// General form of lab-frame moments on the lattice shifted by U: the
// moments about U, M'_a = M_a - U_a M0, M'_ab = M_ab - U_a M_b - U_b M_a +
// U_a U_b M0, then Eq. geq_gstar on the relative velocities, with psi
// (when with_psi) Y_a = (M'_aa - M0 T)(1 - 3T)/(2T) on the rest (+) and
// axis (-1/2) velocities: the part of the diagonal second moments that
// the W_i-weighted form misses on the lattice (sum W_i c_a^4 = T).
template <class A>
__device__ __forceinline__ void gform_about(A Ux, A Uy, A T, A M0, A Mx, A My, A Mxx, A Mxy, A Myy,
                                            bool with_psi, A G[NQ])
{
    const A cMx = Mx - Ux * M0, cMy = My - Uy * M0;
    const A cMxx = Mxx - A(2) * Ux * Mx + Ux * Ux * M0;
    const A cMxy = Mxy - Ux * My - Uy * Mx + Ux * Uy * M0;
    const A cMyy = Myy - A(2) * Uy * My + Uy * Uy * M0;
    A pr = 0, px = 0, py = 0;
    if (with_psi) {
        const A k = (A(1) - A(3) * T) / (A(2) * T);
        const A Yx = (cMxx - M0 * T) * k, Yy = (cMyy - M0 * T) * k;
        pr = Yx + Yy;
        px = A(-0.5) * Yx;
        py = A(-0.5) * Yy;
    }
    gform9(T, M0, cMx, cMy, cMxx, cMxy, cMyy, pr, px, py, G);
}

// g^eq (Table I, first row) or g* (second row, with q*_a = q^eq_a +
// 2 u_b (P_ab - P^eq_ab)) for the given macroscopic state.
template <class A>
__device__ __forceinline__ void gmoments(A rho, A ux, A uy, A T, A E, A &M0, A &qx, A &qy,
                                         A &Rxx, A &Rxy, A &Ryy)
{
    M0 = A(2) * rho * E;
    A ET = E + T;
    qx = A(2) * rho * ux * ET;
    qy = A(2) * rho * uy * ET;
    A a = A(2) * rho * E, b = A(2) * rho * T;
    Rxx = a * (T + ux * ux) + b * (T + A(2) * ux * ux);
    Rxy = a * (ux * uy) + b * (A(2) * ux * uy);
    Ryy = a * (T + uy * uy) + b * (T + A(2) * uy * uy);
}

// f^eq and g^eq (Table I, first row) of the solver's lattice at (rho, u, T).
template <class A>
__device__ __forceinline__ void equilibria(const KinParams<A> &K, A rho, A ux, A uy, A T, A f[NQ], A g[NQ])
{
    feq9(rho, ux - K.Ux, uy - K.Uy, T, f);
    const A E = K.Cv * T + A(0.5) * (ux * ux + uy * uy);
    A M0, qx, qy, Rxx, Rxy, Ryy, pr, px, py;
    gmoments(rho, ux, uy, T, E, M0, qx, qy, Rxx, Rxy, Ryy);
    if (K.flags & FLAG_SHIFT) {
        gform_about(K.Ux, K.Uy, T, M0, qx, qy, Rxx, Rxy, Ryy, true, g);
    } else {
        psi_terms(rho, ux, uy, T, E, pr, px, py);
        gform9(T, M0, qx, qy, Rxx, Rxy, Ryy, pr, px, py, g);
    }
}

// Collision of one node on deviations: f, g in (streamed, deviations),
// out (post-collision deviations).  Returns false on a non-physical state.
template <class A>
__device__ __forceinline__ bool collide_node(const KinParams<A> &K, A f[NQ], A g[NQ], A Xx, A Xy,
                                             A &rho_o, A &ux_o, A &uy_o, A &T_o)
{
    A sf = 0, jx = 0, jy = 0, dxx = 0, dxy = 0, dyy = 0, sg = 0;
#pragma unroll
    for (int i = 0; i < NQ; ++i) sg += g[i];
    sf = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    jx = K.jx_ref + ((f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]));
    jy = K.jy_ref + ((f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]));
    dxx = f[1] + f[3] + f[5] + f[6] + f[7] + f[8];
    dyy = f[2] + f[4] + f[5] + f[6] + f[7] + f[8];
    dxy = (f[5] + f[7]) - (f[6] + f[8]);
    A rho = K.rho_ref + sf;
    // relative velocity w = sum c_i f_i / rho; lab velocity u = w + U
    const A wx = jx / rho, wy = jy / rho;
    A ux = wx + K.Ux, uy = wy + K.Uy;
    A E = (K.E2_ref + sg) / (A(2) * rho);
    A T = (E - A(0.5) * (ux * ux + uy * uy)) / K.Cv;
    rho_o = rho;
    ux_o = ux;
    uy_o = uy;
    T_o = T;
    if (!(rho > A(0)) || !(T > A(0))) return false;
    if (K.flags & FLAG_COLLIDE_OFF) return true;
    // P_ab - P^eq_ab from deviations plus the reference's own P_ab (about
    // U on the shifted lattice: the difference is the same in every frame)
    A Pxx = K.Pxx_ref + dxx, Pyy = K.Pyy_ref + dyy, Pxy = K.Pxy_ref + dxy;
    A dPxx = Pxx - (rho * wx * wx + rho * T);
    A dPxy = Pxy - rho * wx * wy;
    A dPyy = Pyy - (rho * wy * wy + rho * T);
    A omega = A(1) / (K.mu / (rho * T) + A(0.5));
    A omega1 = A(1) / ((A(1) / omega - A(0.5)) / K.Pr + A(0.5));
    A fe[NQ], ge[NQ], gs[NQ];
    feq9(rho, wx, wy, T, fe);
    A M0, qx, qy, Rxx, Rxy, Ryy, pr, px, py;
    gmoments(rho, ux, uy, T, E, M0, qx, qy, Rxx, Rxy, Ryy);
    A qsx = qx + A(2) * (ux * dPxx + uy * dPxy);
    A qsy = qy + A(2) * (ux * dPxy + uy * dPyy);
    if (K.flags & FLAG_SHIFT) {
        gform_about(K.Ux, K.Uy, T, M0, qx, qy, Rxx, Rxy, Ryy, true, ge);
        gform_about(K.Ux, K.Uy, T, M0, qsx, qsy, Rxx, Rxy, Ryy, true, gs);
    } else {
        psi_terms(rho, ux, uy, T, E, pr, px, py);
        gform9(T, M0, qx, qy, Rxx, Rxy, Ryy, pr, px, py, ge);
        gform9(T, M0, qsx, qsy, Rxx, Rxy, Ryy, pr, px, py, gs);
    }
    A hx = A(0.5) * Xx, hy = A(0.5) * Xy; // phi_i = A_ia X_a: +-X/2 on the axis velocities
    A om1 = omega1 - omega;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        A deq = fe[i] - K.fref[i];
        f[i] = f[i] + omega * (deq - f[i]);
        A dge = ge[i] - K.gref[i], dgs = gs[i] - K.gref[i];
        g[i] = g[i] + omega * (dge - g[i]) + om1 * (dgs - g[i]);
    }
    f[1] += hx;
    f[3] -= hx;
    f[2] += hy;
    f[4] -= hy;
    return true;
}

// Missing populations f^eq(tgt) + f^(1), g^eq(tgt) + g^(1) (Sec. IV.A,
// Table II), as deviations.  du = {d_x ux, d_y ux, d_x uy, d_y uy},
// dT = {d_x T, d_y T}, physical.
template <class A>
__device__ __forceinline__ void grad_missing(const KinParams<A> &K, A rho, A ux, A uy, A T,
                                             const A du[4], const A dT[2], A f[NQ], A g[NQ])
{
    A omega = A(1) / (K.mu / (rho * T) + A(0.5));
    A omega1 = A(1) / ((A(1) / omega - A(0.5)) / K.Pr + A(0.5));
    A E = K.Cv * T + A(0.5) * (ux * ux + uy * uy);
    A Sxx = A(2) * du[0], Syy = A(2) * du[3], Sxy = du[2] + du[1];
    A divu = du[0] + du[3];
    A dEx = K.Cv * dT[0] + ux * du[0] + uy * du[2];
    A dEy = K.Cv * dT[1] + ux * du[1] + uy * du[3];
    A c1 = -(A(1) / omega) * rho * T;
    A P1xx = c1 * (Sxx - divu / K.Cv), P1xy = c1 * Sxy, P1yy = c1 * (Syy - divu / K.Cv);
    A c2 = -(A(2) / omega1) * rho * T;
    A q1x = c2 * K.Cp * dT[0] + A(2) * (ux * P1xx + uy * P1xy);
    A q1y = c2 * K.Cp * dT[1] + A(2) * (ux * P1xy + uy * P1yy);
    A ET2 = E + A(2) * T;
    A R1xx = c2 * (Sxx * ET2 + A(2) * ux * dEx);
    A R1xy = c2 * (Sxy * ET2 + ux * dEy + uy * dEx);
    A R1yy = c2 * (Syy * ET2 + A(2) * uy * dEy);
    A fe[NQ], ge[NQ], f1[NQ], g1[NQ];
    feq9(rho, ux - K.Ux, uy - K.Uy, T, fe);
    A M0, qx, qy, Rxx, Rxy, Ryy, pr, px, py;
    gmoments(rho, ux, uy, T, E, M0, qx, qy, Rxx, Rxy, Ryy);
    gform9(T, A(0), A(0), A(0), P1xx, P1xy, P1yy, A(0), A(0), A(0), f1);
    if (K.flags & FLAG_SHIFT) {
        gform_about(K.Ux, K.Uy, T, M0, qx, qy, Rxx, Rxy, Ryy, true, ge);
        gform_about(K.Ux, K.Uy, T, A(0), q1x, q1y, R1xx, R1xy, R1yy, false, g1);
    } else {
        psi_terms(rho, ux, uy, T, E, pr, px, py);
        gform9(T, M0, qx, qy, Rxx, Rxy, Ryy, pr, px, py, ge);
        gform9(T, A(0), q1x, q1y, R1xx, R1xy, R1yy, A(0), A(0), A(0), g1);
    }
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        f[i] = (fe[i] - K.fref[i]) + f1[i];
        g[i] = (ge[i] - K.gref[i]) + g1[i];
    }
}

} // namespace alelb
