/*
 * alelb_oracle.c -- plain FP64 CPU oracle of the ALE compressible lattice
 * Boltzmann step (Saadat & Karlin, "Arbitrary Lagrangian-Eulerian
 * formulation of lattice Boltzmann model for compressible flows on
 * unstructured moving meshes", arXiv 2002.04353).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously correct reference
 * the CUDA library is checked against.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code, table or helper with the CUDA library: the two read the
 * same mesh arrays and nothing else.
 *
 * Everything is FP64, one node at a time, in the order the paper states.
 * Where the paper is silent the reading used is stated at the spot:
 *   R1  transformed velocity  c^_i = g^{-1,T} (c_i - V_G)        (Eq. 7 + chain rule)
 *   R2  map, Jacobian and V_G evaluated at the arrival time t_{n+1}; flag
 *       MIDPOINT evaluates those of the transformed velocities at t_{n+1/2};
 *       flag EXACT_CHAR takes the departure point on the exact characteristic,
 *       X_dp = G^-1(G(X, t_{n+1}) - c_i dt, t_n), for maps with a closed-form
 *       inverse (none, plunge, rigid pitch, pitch with plunge)
 *   R3  q*_a = q^eq_a + 2 u_b (P_ab - P^eq_ab)   (Table I's q* as printed drops q^eq)
 *   R4  forcing enters as + dt*phi_i with phi from the same time level; the
 *       equilibria use the plain velocity sum(c f)/rho
 *   R5  a departure point on element edges/vertices belongs to the
 *       containing element of larger computational area, then lower id;
 *       a departure point that coincides with the node itself (c^_i = 0)
 *       takes the node's own value
 *   R6  a population is "missing" when some point of the segment from the
 *       node to its departure point lies outside the closed mesh (the
 *       departure point itself, or a stretch that passes through the body);
 *       far-field missing populations take the free-stream equilibria
 *   R7  D2Q9 order (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1)
 *   R8  wall targets: u = V_G at the wall node, rho and T interpolated at
 *       B = A + n dt from the previous step's fields; off-wall targets are
 *       the node's previous-step fields; gradients are first-order
 *       (vertex-linear) FE derivatives of the previous-step fields (Sec.
 *       IV.A) in the node's wall-side element: among its incident elements
 *       with a vertex on a wall edge the one of larger computational area
 *       (then lower id), else its owner element.  The larger-area rule of
 *       Sec. IV is stated for the correction-term derivatives; applied to a
 *       node one layer off the wall it takes a difference away from the
 *       wall, and the normal velocity next to the wall then grows without
 *       bound.
 *       Flag BC_EQUILIBRIUM drops the non-equilibrium part (a stabilising
 *       variant, not the paper's condition).  Flag SLIP_WALL (the inviscid
 *       variant; the paper has none): wall nodes take u = V_G plus the
 *       tangential part of u_B - V_G at the probe B, tangent taken in the
 *       physical frame, and no non-equilibrium part (no wall shear)
 *   R8c flag OFFWALL_VG: off-wall nodes' missing populations take the mesh
 *       velocity V_G at the node as the target velocity (the paper states
 *       targets for wall nodes only); pinned by the one-step closed form
 *       next to a receding wall (the reading itself has no passage)
 *   R9  forces: p = rho T, tau = mu (S - (1/Cv) div u I), Simpson's rule
 *       on each straight 3-node wall edge of the mapped geometry
 *   R12 elements: straight-sided 6-node triangles, or the paper's 9-node
 *       quadrilaterals (Sec. III) whose local coordinates solve the
 *       bilinear system of Eq. NonLinear_Eq by Newton's method from the
 *       cell centre with a fixed number of iterations (the paper names no
 *       method); on quadrilaterals the wall condition's first-order
 *       gradient is that of the bilinear interpolant of the vertex values
 *   R14 shifted lattice (velocities c_i + U, Sec. V.D; the model itself is
 *       deferred to another paper): every population set carries the same
 *       lab-frame moments as on the plain lattice -- f^eq in u - U, the
 *       general form on moments taken about U, psi the correction of the
 *       diagonal second central moments (the printed psi at U = 0), Q' in
 *       u - U, phi_i = A_ia X_a on the relative velocities c_i; the
 *       departure uses c_i + U and the moments sum (c_i + U) f
 * Parity status of each function is given in its comment.  The forces, the
 * probe point B, the wall condition's gradient element and the R8c target
 * are pinned by closed forms (quadratic fields on a closed body through the
 * divergence theorem; one step without collision against the Grad
 * reconstruction); the paper prints no force values for these setups.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define NQ 9
static const int CXI[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CYI[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

enum { ST_OK = 0, ST_ARG = -1, ST_OOM = -2, ST_MESH = -4, ST_MAP = -5, ST_LOCATE = -6,
       ST_NONFINITE = -7 };
enum { FLAG_PHI_OFF = 1, FLAG_COLLIDE_OFF = 2, FLAG_LITERAL_VG = 4, FLAG_BC_EQUILIBRIUM = 8,
       FLAG_SLIP_WALL = 16, FLAG_MIDPOINT = 32, FLAG_EXACT_CHAR = 64, FLAG_OFFWALL_VG = 256 };
enum { MK_NONE = 0, MK_SINE = 1, MK_PLUNGE = 2, MK_PITCH = 3, MK_PITCH_PLUNGE = 4,
       MK_BLENDED = 5 };
enum { EK_INTERIOR = 0, EK_WALL = 1, EK_FAR = 2 };

/* ======================================================================
 * Exact orientation sign.  det = (a-c) x (b-c) expanded into six products,
 * each split exactly into two doubles (product + FMA error term), and the
 * twelve terms summed exactly as a non-overlapping floating-point expansion
 * (Shewchuk 1997, "Adaptive precision floating-point arithmetic and fast
 * robust geometric predicates", Two-Sum / Two-Product / Grow-Expansion).
 * Pinned by tests against integer arithmetic on random and collinear inputs.
 * ==================================================================== */
static void two_sum(double a, double b, double *x, double *y)
{
    double s = a + b;
    double bv = s - a;
    double av = s - bv;
    *x = s;
    *y = (a - av) + (b - bv);
}

static int exact_sign_of_sum(const double *v, int n)
{
    double e[64];
    int m = 0;
    for (int k = 0; k < n; ++k) {
        double q = v[k];
        int mm = 0;
        for (int j = 0; j < m; ++j) {
            double s, err;
            two_sum(q, e[j], &s, &err);
            if (err != 0.0) e[mm++] = err;
            q = s;
        }
        if (q != 0.0) e[mm++] = q;
        m = mm;
    }
    if (m == 0) return 0;
    return e[m - 1] > 0.0 ? 1 : -1;
}

int orc_orient(double ax, double ay, double bx, double by, double cx, double cy)
{
    /* (ax-cx)(by-cy) - (ay-cy)(bx-cx)
       = ax*by - ax*cy - cx*by - ay*bx + ay*cx + cy*bx */
    double p[6][2] = {{ax, by}, {-ax, cy}, {-cx, by}, {-ay, bx}, {ay, cx}, {cy, bx}};
    double t[12];
    for (int k = 0; k < 6; ++k) {
        double hi = p[k][0] * p[k][1];
        t[2 * k] = hi;
        t[2 * k + 1] = fma(p[k][0], p[k][1], -hi);
    }
    return exact_sign_of_sum(t, 12);
}

/* ======================================================================
 * Kinetic model (Sec. IV)
 * ==================================================================== */
typedef struct {
    double gamma, Pr, mu, rho_inf, T_inf, ux_inf, uy_inf, chord;
    int flags;
    double Cv, Cp;
    double Ux, Uy; /* lattice shift U: the discrete velocities are c_i + U (Sec. V.D) */
} kin_t;

static void kin_from(const double *k, kin_t *K)
{
    K->gamma = k[0];
    K->Pr = k[1];
    K->mu = k[2];
    K->rho_inf = k[3];
    K->T_inf = k[4];
    K->ux_inf = k[5];
    K->uy_inf = k[6];
    K->chord = k[7];
    K->flags = (int)k[8];
    K->Ux = k[9];
    K->Uy = k[10];
    K->Cv = 1.0 / (K->gamma - 1.0); /* R = 1 */
    K->Cp = K->Cv + 1.0;
}

/* Phi_{c}(u, T): Eq. feq, the one-dimensional factors of f^eq. */
static double Phi(int c, double u, double T)
{
    if (c == -1) return (-u + u * u + T) / 2.0;
    if (c == 0) return 1.0 - (u * u + T);
    return (u + u * u + T) / 2.0;
}

/* f^eq_i = rho Phi_{cix} Phi_{ciy}  (Eq. feq).
   Pinned: its moments {1, c, cc} are rho, rho u, rho(uu + T delta). */
void orc_feq(double rho, double ux, double uy, double T, double *f)
{
    for (int i = 0; i < NQ; ++i) f[i] = rho * Phi(CXI[i], ux, T) * Phi(CYI[i], uy, T);
}

/* W_c(T) of Eq. Wi. */
static double Wc(int c, double T) { return c == 0 ? 1.0 - T : T / 2.0; }

/* General form G_i of Eq. geq_gstar for given moments M0, M_a, M_ab and Psi_i. */
static void gform(double T, double M0, double Mx, double My, double Mxx, double Mxy,
                  double Myy, const double *Psi, double *G)
{
    for (int i = 0; i < NQ; ++i) {
        double cx = CXI[i], cy = CYI[i];
        double W = Wc(CXI[i], T) * Wc(CYI[i], T);
        double lin = (Mx * cx + My * cy) / T;
        double quad = ((Mxx - M0 * T) * (cx * cx - T) + (Mxy) * (cx * cy) + (Mxy) * (cy * cx) +
                       (Myy - M0 * T) * (cy * cy - T)) / (2.0 * T * T);
        G[i] = W * (M0 + lin + quad) + (Psi ? Psi[i] : 0.0);
    }
}

/* psi_i = B_ia rho (1 - 3T)(T^2 + 2 u_a^2 T + E u_a^2)/T, summed over a;
   B_ia = 1 for the rest velocity, -|c_ia - c_ia c_i^2 / 2| otherwise. */
static void psi_terms(double rho, double ux, double uy, double T, double E, double *psi)
{
    double Y[2];
    double u[2] = {ux, uy};
    for (int a = 0; a < 2; ++a)
        Y[a] = rho * (1.0 - 3.0 * T) * (T * T + 2.0 * u[a] * u[a] * T + E * u[a] * u[a]) / T;
    for (int i = 0; i < NQ; ++i) {
        double c[2] = {CXI[i], CYI[i]};
        double c2 = c[0] * c[0] + c[1] * c[1];
        double s = 0.0;
        for (int a = 0; a < 2; ++a) {
            double B = (c2 == 0.0) ? 1.0 : -fabs(c[a] - 0.5 * c[a] * c2);
            s += B * Y[a];
        }
        psi[i] = s;
    }
}

/* R^eq_ab = 2 rho E (T d_ab + u_a u_b) + 2 rho T (T d_ab + 2 u_a u_b). */
static void Req(double rho, double ux, double uy, double T, double E, double *R)
{
    R[0] = 2.0 * rho * E * (T + ux * ux) + 2.0 * rho * T * (T + 2.0 * ux * ux);
    R[1] = 2.0 * rho * E * (ux * uy) + 2.0 * rho * T * (2.0 * ux * uy);
    R[2] = 2.0 * rho * E * (T + uy * uy) + 2.0 * rho * T * (T + 2.0 * uy * uy);
}

/* g^eq_i: Table I row 1 (M0 = 2 rho E, M_a = q^eq_a = 2 rho u_a (E + T),
   M_ab = R^eq_ab, Psi = psi).  Pinned: moments 2rhoE, q^eq, R^eq exact. */
void orc_geq(double rho, double ux, double uy, double T, double Cv, double *g)
{
    double E = Cv * T + 0.5 * (ux * ux + uy * uy);
    double R[3], psi[NQ];
    Req(rho, ux, uy, T, E, R);
    psi_terms(rho, ux, uy, T, E, psi);
    gform(T, 2.0 * rho * E, 2.0 * rho * ux * (E + T), 2.0 * rho * uy * (E + T), R[0], R[1], R[2],
          psi, g);
}

/* g*_i: Table I row 2 with q*_a = q^eq_a + 2 u_b (P_ab - P^eq_ab) (reading R3). */
void orc_gqe(double rho, double ux, double uy, double T, double Cv, double Pxx, double Pxy,
             double Pyy, double *g)
{
    double E = Cv * T + 0.5 * (ux * ux + uy * uy);
    double R[3], psi[NQ];
    Req(rho, ux, uy, T, E, R);
    psi_terms(rho, ux, uy, T, E, psi);
    double dPxx = Pxx - (rho * ux * ux + rho * T);
    double dPxy = Pxy - (rho * ux * uy);
    double dPyy = Pyy - (rho * uy * uy + rho * T);
    double qx = 2.0 * rho * ux * (E + T) + 2.0 * (ux * dPxx + uy * dPxy);
    double qy = 2.0 * rho * uy * (E + T) + 2.0 * (ux * dPxy + uy * dPyy);
    gform(T, 2.0 * rho * E, qx, qy, R[0], R[1], R[2], psi, g);
}

/* ----------------------------------------------------------------------
 * Shifted lattice (Sec. V.D: velocities c_i + U, U = (0.3, 0) for the
 * transonic case; the model's details are deferred to its own reference,
 * so this is reading R14).  Every population set is built to carry the
 * same lab-frame moments as on the plain lattice:
 *   f^eq: the product form in the relative velocity u - U (its moments
 *         {1, c, cc} about U are those of the Maxwellian about U, hence
 *         {1, c + U, (c + U)(c + U)} give rho, rho u, rho(uu + T I));
 *   general form: the lab moments M0, M_a, M_ab are converted to moments
 *         about U, M'_a = M_a - U_a M0, M'_ab = M_ab - U_a M_b - U_b M_a
 *         + U_a U_b M0, and Eq. geq_gstar is applied on the relative
 *         velocities c_i;
 *   psi:  on the plain lattice psi_i restores the diagonal second moments
 *         that Eq. geq_gstar misses (sum W_i c_a^4 = T, not 3 T^2):
 *         sum c_a^2 G_i = M0 T + (M_aa - M0 T)(1 - T)/(2T).  The printed
 *         psi is exactly that correction for g^eq; on the shifted lattice
 *         the same correction is taken of the central moments,
 *         Y_a = (M'_aa - M0 T)(1 - 3T)/(2T), psi_i = B_ia Y_a.
 * ------------------------------------------------------------------- */
void orc_feq_shift(double rho, double ux, double uy, double T, double Ux, double Uy, double *f)
{
    orc_feq(rho, ux - Ux, uy - Uy, T, f);
}

/* General form of lab moments on the lattice shifted by U (psi only when
   with_psi). */
static void gform_shift(double T, double Ux, double Uy, double M0, double Mx, double My,
                        double Mxx, double Mxy, double Myy, int with_psi, double *G)
{
    double cMx = Mx - Ux * M0, cMy = My - Uy * M0;
    double cMxx = Mxx - 2.0 * Ux * Mx + Ux * Ux * M0;
    double cMxy = Mxy - Ux * My - Uy * Mx + Ux * Uy * M0;
    double cMyy = Myy - 2.0 * Uy * My + Uy * Uy * M0;
    double psi[NQ];
    if (with_psi) {
        double Y[2] = {(cMxx - M0 * T) * (1.0 - 3.0 * T) / (2.0 * T),
                       (cMyy - M0 * T) * (1.0 - 3.0 * T) / (2.0 * T)};
        for (int i = 0; i < NQ; ++i) {
            double c[2] = {CXI[i], CYI[i]};
            double c2 = c[0] * c[0] + c[1] * c[1];
            double sum = 0.0;
            for (int a = 0; a < 2; ++a) sum += ((c2 == 0.0) ? 1.0 : -fabs(c[a] - 0.5 * c[a] * c2)) * Y[a];
            psi[i] = sum;
        }
    }
    gform(T, M0, cMx, cMy, cMxx, cMxy, cMyy, with_psi ? psi : NULL, G);
}

/* g^eq and g* on the shifted lattice: the lab moments of Table I. */
void orc_geq_shift(double rho, double ux, double uy, double T, double Cv, double Ux, double Uy,
                   double *g)
{
    double E = Cv * T + 0.5 * (ux * ux + uy * uy);
    double R[3];
    Req(rho, ux, uy, T, E, R);
    gform_shift(T, Ux, Uy, 2.0 * rho * E, 2.0 * rho * ux * (E + T), 2.0 * rho * uy * (E + T), R[0],
                R[1], R[2], 1, g);
}

/* Pxx, Pxy, Pyy: the lab-frame second moments sum (c + U)(c + U) f. */
void orc_gqe_shift(double rho, double ux, double uy, double T, double Cv, double Ux, double Uy,
                   double Pxx, double Pxy, double Pyy, double *g)
{
    double E = Cv * T + 0.5 * (ux * ux + uy * uy);
    double R[3];
    Req(rho, ux, uy, T, E, R);
    double dPxx = Pxx - (rho * ux * ux + rho * T);
    double dPxy = Pxy - (rho * ux * uy);
    double dPyy = Pyy - (rho * uy * uy + rho * T);
    double qx = 2.0 * rho * ux * (E + T) + 2.0 * (ux * dPxx + uy * dPxy);
    double qy = 2.0 * rho * uy * (E + T) + 2.0 * (ux * dPxy + uy * dPyy);
    gform_shift(T, Ux, Uy, 2.0 * rho * E, qx, qy, R[0], R[1], R[2], 1, g);
}

static int shifted(const kin_t *K) { return K->Ux != 0.0 || K->Uy != 0.0; }

/* Equilibria of the solver's lattice (the printed forms when unshifted). */
static void feq_K(const kin_t *K, double rho, double ux, double uy, double T, double *f)
{
    orc_feq_shift(rho, ux, uy, T, K->Ux, K->Uy, f);
}
static void geq_K(const kin_t *K, double rho, double ux, double uy, double T, double *g)
{
    if (shifted(K)) orc_geq_shift(rho, ux, uy, T, K->Cv, K->Ux, K->Uy, g);
    else orc_geq(rho, ux, uy, T, K->Cv, g);
}

/* Local collision of Eqs. feqn/geqn at one node, given the streamed
   populations f, g and the correction source X_a.  Writes the
   post-collision populations.  Pinned: sum f and sum g conserved exactly,
   momentum changes by X, uniform equilibrium is a fixed point. */
static void collide(const kin_t *K, const double *f, const double *g, double Xx, double Xy,
                    double *fo, double *go)
{
    double rho = 0, jx = 0, jy = 0, Pxx = 0, Pxy = 0, Pyy = 0, e2 = 0;
    for (int i = 0; i < NQ; ++i) {
        double vx = CXI[i] + K->Ux, vy = CYI[i] + K->Uy; /* the lattice velocity */
        rho += f[i];
        jx += vx * f[i];
        jy += vy * f[i];
        Pxx += vx * vx * f[i];
        Pxy += vx * vy * f[i];
        Pyy += vy * vy * f[i];
        e2 += g[i];
    }
    double ux = jx / rho, uy = jy / rho;
    double E = e2 / (2.0 * rho);
    double T = (E - 0.5 * (ux * ux + uy * uy)) / K->Cv;
    /* mu = (1/omega - 1/2) rho T dt;  kappa = Cp (1/omega1 - 1/2) rho T dt;
       Pr = Cp mu / kappa */
    double omega = 1.0 / (K->mu / (rho * T) + 0.5);
    double omega1 = 1.0 / ((1.0 / omega - 0.5) / K->Pr + 0.5);
    double feq[NQ], geq[NQ], gqe[NQ];
    feq_K(K, rho, ux, uy, T, feq);
    geq_K(K, rho, ux, uy, T, geq);
    if (shifted(K)) orc_gqe_shift(rho, ux, uy, T, K->Cv, K->Ux, K->Uy, Pxx, Pxy, Pyy, gqe);
    else orc_gqe(rho, ux, uy, T, K->Cv, Pxx, Pxy, Pyy, gqe);
    for (int i = 0; i < NQ; ++i) {
        /* A_ia on the relative velocities c_i (reading R14) */
        double cx = CXI[i], cy = CYI[i], c2 = cx * cx + cy * cy;
        double phi = (cx - 0.5 * cx * c2) * Xx + (cy - 0.5 * cy * c2) * Xy; /* A_ia X_a */
        fo[i] = f[i] + omega * (feq[i] - f[i]) + 1.0 * phi;
        go[i] = g[i] + omega * (geq[i] - g[i]) + (omega1 - omega) * (gqe[i] - g[i]);
    }
}

void orc_collide(const double *kin, const double *f, const double *g, double Xx, double Xy,
                 double *fo, double *go)
{
    kin_t K;
    kin_from(kin, &K);
    collide(&K, f, g, Xx, Xy, fo, go);
}

/* Grad-type missing populations of Sec. IV.A: f = f^eq(tgt) + dt f^(1),
   g = g^eq(tgt) + dt g^(1), with f^(1), g^(1) from the general form and the
   non-equilibrium moments of Table II (M0 = 0, Psi = 0).
   du = {d_x ux, d_y ux, d_x uy, d_y uy}, dT = {d_x T, d_y T} (physical).
   Pinned: zero gradients give the equilibria exactly; f^(1) has zero
   density and momentum and carries P^(1)_xy exactly. */
static void grad_bc(const kin_t *K, double rho, double ux, double uy, double T,
                    const double *du, const double *dT, double *f, double *g)
{
    double omega = 1.0 / (K->mu / (rho * T) + 0.5);
    double omega1 = 1.0 / ((1.0 / omega - 0.5) / K->Pr + 0.5);
    double E = K->Cv * T + 0.5 * (ux * ux + uy * uy);
    double dux[2] = {du[0], du[1]}, duy[2] = {du[2], du[3]};
    /* S_ab = d_a u_b + d_b u_a */
    double Sxx = 2.0 * dux[0];
    double Syy = 2.0 * duy[1];
    double Sxy = duy[0] + dux[1];
    double divu = dux[0] + duy[1];
    /* d_a E = Cv d_a T + u_b d_a u_b */
    double dEx = K->Cv * dT[0] + ux * dux[0] + uy * duy[0];
    double dEy = K->Cv * dT[1] + ux * dux[1] + uy * duy[1];
    double P1xx = -(1.0 / omega) * rho * T * (Sxx - (1.0 / K->Cv) * divu);
    double P1xy = -(1.0 / omega) * rho * T * (Sxy);
    double P1yy = -(1.0 / omega) * rho * T * (Syy - (1.0 / K->Cv) * divu);
    double q1x = -(2.0 / omega1) * rho * K->Cp * T * dT[0] + 2.0 * (ux * P1xx + uy * P1xy);
    double q1y = -(2.0 / omega1) * rho * K->Cp * T * dT[1] + 2.0 * (ux * P1xy + uy * P1yy);
    double R1xx = -(2.0 / omega1) * rho * T * (Sxx * (E + 2.0 * T) + ux * dEx + ux * dEx);
    double R1xy = -(2.0 / omega1) * rho * T * (Sxy * (E + 2.0 * T) + ux * dEy + uy * dEx);
    double R1yy = -(2.0 / omega1) * rho * T * (Syy * (E + 2.0 * T) + uy * dEy + uy * dEy);
    double feq[NQ], geq[NQ], f1[NQ], g1[NQ];
    feq_K(K, rho, ux, uy, T, feq);
    geq_K(K, rho, ux, uy, T, geq);
    if (shifted(K)) { /* the same lab moments, taken about U */
        gform_shift(T, K->Ux, K->Uy, 0.0, 0.0, 0.0, P1xx, P1xy, P1yy, 0, f1);
        gform_shift(T, K->Ux, K->Uy, 0.0, q1x, q1y, R1xx, R1xy, R1yy, 0, g1);
    } else {
        gform(T, 0.0, 0.0, 0.0, P1xx, P1xy, P1yy, NULL, f1);
        gform(T, 0.0, q1x, q1y, R1xx, R1xy, R1yy, NULL, g1);
    }
    for (int i = 0; i < NQ; ++i) {
        f[i] = feq[i] + 1.0 * f1[i];
        g[i] = geq[i] + 1.0 * g1[i];
    }
}

void orc_grad_bc(const double *kin, double rho, double ux, double uy, double T,
                 const double *du, const double *dT, double *f, double *g)
{
    kin_t K;
    kin_from(kin, &K);
    grad_bc(&K, rho, ux, uy, T, du, dT, f, g);
}

/* ======================================================================
 * P2 triangle shape functions in local coordinates (xi, eta) of the
 * straight-sided element, lambda0 = 1 - xi - eta.  Node order v0 v1 v2
 * m01 m12 m20.  (Sec. III, Eq. Propagation, for the 6-node triangle.)
 * Pinned: partition of unity, Kronecker property, quadratic reproduction.
 * ==================================================================== */
void orc_shape(double xi, double eta, double *N)
{
    double l0 = 1.0 - xi - eta, l1 = xi, l2 = eta;
    N[0] = l0 * (2.0 * l0 - 1.0);
    N[1] = l1 * (2.0 * l1 - 1.0);
    N[2] = l2 * (2.0 * l2 - 1.0);
    N[3] = 4.0 * l0 * l1;
    N[4] = 4.0 * l1 * l2;
    N[5] = 4.0 * l2 * l0;
}

static void shape_dxi(double xi, double eta, double *Nxi, double *Neta)
{
    double l0 = 1.0 - xi - eta;
    Nxi[0] = -(4.0 * l0 - 1.0);
    Neta[0] = -(4.0 * l0 - 1.0);
    Nxi[1] = 4.0 * xi - 1.0;
    Neta[1] = 0.0;
    Nxi[2] = 0.0;
    Neta[2] = 4.0 * eta - 1.0;
    Nxi[3] = 4.0 * (l0 - xi);
    Neta[3] = -4.0 * xi;
    Nxi[4] = 4.0 * eta;
    Neta[4] = 4.0 * xi;
    Nxi[5] = -4.0 * eta;
    Neta[5] = 4.0 * (l0 - eta);
}

static const double LOCAL_XI[6][2] = {{0, 0}, {1, 0}, {0, 1}, {0.5, 0}, {0.5, 0.5}, {0, 0.5}};

/* ======================================================================
 * The paper's 9-node quadrilateral (Sec. III, Eq. Propagation with
 * s = 1..9): second-order Lagrange polynomials on the nine equidistant
 * collocation nodes of the reference cell -1 <= xi, eta <= 1, i.e. the
 * products of the one-dimensional quadratics through -1, 0, 1.  Node
 * order: corners v0 (-1,-1), v1 (1,-1), v2 (1,1), v3 (-1,1)
 * (counter-clockwise), midside nodes of edges (v0,v1), (v1,v2), (v2,v3),
 * (v3,v0), then the centre.  Pinned: partition of unity, Kronecker
 * property, reproduction of every polynomial of degree <= 2 in each of
 * xi and eta.
 * ==================================================================== */
static const int Q2_I[9] = {0, 2, 2, 0, 1, 2, 1, 0, 1}; /* xi  = Q2_I - 1 */
static const int Q2_J[9] = {0, 0, 2, 2, 0, 1, 2, 1, 1}; /* eta = Q2_J - 1 */

static void lagrange3(double s, double *L, double *dL)
{
    L[0] = 0.5 * s * (s - 1.0);
    L[1] = (1.0 - s) * (1.0 + s);
    L[2] = 0.5 * s * (s + 1.0);
    if (dL) {
        dL[0] = s - 0.5;
        dL[1] = -2.0 * s;
        dL[2] = s + 0.5;
    }
}

void orc_shape_q2(double xi, double eta, double *N)
{
    double Lx[3], Ly[3];
    lagrange3(xi, Lx, NULL);
    lagrange3(eta, Ly, NULL);
    for (int s = 0; s < 9; ++s) N[s] = Lx[Q2_I[s]] * Ly[Q2_J[s]];
}

static void shape_dxi_q2(double xi, double eta, double *Nxi, double *Neta)
{
    double Lx[3], Ly[3], dLx[3], dLy[3];
    lagrange3(xi, Lx, dLx);
    lagrange3(eta, Ly, dLy);
    for (int s = 0; s < 9; ++s) {
        Nxi[s] = dLx[Q2_I[s]] * Ly[Q2_J[s]];
        Neta[s] = Lx[Q2_I[s]] * dLy[Q2_J[s]];
    }
}

/* The bilinear map of Eq. NonLinear_Eq, x(xi, eta) = sum_{s=1..4} N_s x_s
   over the corners, N_s = (1 +- xi)(1 +- eta)/4, with its Jacobian
   J = {x_xi, x_eta, y_xi, y_eta}.  w: the 4 corners (x, y). */
static void bilinear(const double *w, double xi, double eta, double *x, double *y, double *J)
{
    double n[4] = {0.25 * (1.0 - xi) * (1.0 - eta), 0.25 * (1.0 + xi) * (1.0 - eta),
                   0.25 * (1.0 + xi) * (1.0 + eta), 0.25 * (1.0 - xi) * (1.0 + eta)};
    double nxi[4] = {-0.25 * (1.0 - eta), 0.25 * (1.0 - eta), 0.25 * (1.0 + eta), -0.25 * (1.0 + eta)};
    double neta[4] = {-0.25 * (1.0 - xi), -0.25 * (1.0 + xi), 0.25 * (1.0 + xi), 0.25 * (1.0 - xi)};
    double sx = 0, sy = 0, a = 0, b = 0, c = 0, d = 0;
    for (int k = 0; k < 4; ++k) {
        sx += n[k] * w[2 * k];
        sy += n[k] * w[2 * k + 1];
        a += nxi[k] * w[2 * k];
        b += neta[k] * w[2 * k];
        c += nxi[k] * w[2 * k + 1];
        d += neta[k] * w[2 * k + 1];
    }
    if (x) *x = sx;
    if (y) *y = sy;
    if (J) {
        J[0] = a;
        J[1] = b;
        J[2] = c;
        J[3] = d;
    }
}

/* Local coordinates of the departure point in a quadrilateral: Newton's
   method on the bilinear system of Eq. NonLinear_Eq, which the paper
   solves every step without naming a method (reading Q5): start at the
   centre (0, 0), a fixed number of iterations so that every run takes the
   same steps, then the last update must be negligible.  The corners are
   taken relative to p.  Returns 0, or ST_LOCATE when it has not converged. */
#define Q2_NEWTON_ITERS 8
static int q2_local(const double *v, double sx, double sy, double px, double py, double *xi,
                    double *eta)
{
    double w[8];
    for (int k = 0; k < 4; ++k) {
        w[2 * k] = (v[2 * k] + sx) - px;
        w[2 * k + 1] = (v[2 * k + 1] + sy) - py;
    }
    double a = 0.0, b = 0.0, da = 0.0, db = 0.0;
    for (int it = 0; it < Q2_NEWTON_ITERS; ++it) {
        double rx, ry, J[4];
        bilinear(w, a, b, &rx, &ry, J);
        double det = J[0] * J[3] - J[1] * J[2];
        da = (J[3] * rx - J[1] * ry) / det;
        db = (-J[2] * rx + J[0] * ry) / det;
        a -= da;
        b -= db;
    }
    *xi = a;
    *eta = b;
    return (fabs(da) <= 1e-9 && fabs(db) <= 1e-9) ? 0 : ST_LOCATE;
}

/* ======================================================================
 * Oracle state
 * ==================================================================== */
typedef struct {
    int e;
    int8_t sx, sy;
} qent_t;

typedef struct {
    double x0, y0, x1, y1;
    int child; /* index of first of 4 children, -1 for a leaf */
    int start, count;
} qnode_t;

typedef struct {
    int elem, k, kind;
} bedge_t;

typedef struct {
    /* mesh */
    int nn, ne;
    int etype;    /* 0: 6-node triangles, 1: 9-node quadrilaterals */
    int nv, nne;  /* vertices and nodes per element (3, 6 or 4, 9) */
    double *X;
    int *conn;
    uint8_t *ekind;
    double Lx, Ly;
    double *ev;    /* EVS per element: node coords in the element frame */
    double *area2; /* twice the computational area */
    int *owner, *owner_loc;
    int *bcel; /* element of the wall condition's gradients (R8) */
    /* point search */
    qnode_t *qn;
    int nqn, cap_qn;
    qent_t *qe;
    int nqe, cap_qe;
    /* boundary */
    int nbe;
    bedge_t *be;
    int *bnear_ptr; /* CSR per node: nearby boundary edges with shift */
    int *bnear_e;
    int8_t *bnear_sx, *bnear_sy;
    double rchk;
    uint8_t *is_wall;
    double *wall_n; /* 2 per node (zero off the wall) */
    int *probe_e;
    double *probe_xi; /* 2 per node */
    /* motion */
    int mkind;
    double mp[16];
    double *ms; /* static per-node factors, 6 per node */
    /* kinetics */
    kin_t K;
    /* state */
    double *f, *g;             /* post-collision, [i*nn + a] */
    double *rho, *ux, *uy, *T; /* fields of the latest step */
    double t;
    long nstep;
    int status;
    /* scratch */
    double *fs, *gs, *m_rt, *Qx, *Qy, *Dx, *Dy, *Xx, *Xy, *gi;
} orc_t;

#define EVS 18 /* doubles of element frame: 9 nodes x (x, y) */

static void *xcalloc(size_t n, size_t s)
{
    void *p = calloc(n ? n : 1, s);
    if (!p) {
        fprintf(stderr, "oracle: out of memory\n");
        abort();
    }
    return p;
}

static double unwrap1(double d, double L)
{
    if (L > 0) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

/* ---------------------------------------------------------------------
 * Element kinds.  Both are straight-sided: the 6-node triangle, whose
 * local coordinates follow from the affine map in closed form, and the
 * paper's 9-node quadrilateral, whose local coordinates solve the bilinear
 * system of Eq. NonLinear_Eq.
 * ------------------------------------------------------------------- */
/* Local coordinates of p in element e shifted by (sx, sy).  Returns 0 or
   ST_LOCATE (Newton did not converge). */
static int elem_local(const orc_t *o, int e, double sx, double sy, double px, double py, double *xi,
                      double *eta)
{
    const double *v = &o->ev[EVS * e];
    if (o->etype == 1) return q2_local(v, sx, sy, px, py, xi, eta);
    double x0 = v[0] + sx, y0 = v[1] + sy;
    double x_xi = v[2] - v[0], x_eta = v[4] - v[0];
    double y_xi = v[3] - v[1], y_eta = v[5] - v[1];
    double detJ = x_xi * y_eta - y_xi * x_eta;
    *xi = (y_eta * (px - x0) - x_eta * (py - y0)) / detJ;
    *eta = (-y_xi * (px - x0) + x_xi * (py - y0)) / detJ;
    return 0;
}

static void elem_shape(const orc_t *o, double xi, double eta, double *N)
{
    if (o->etype == 1) orc_shape_q2(xi, eta, N);
    else orc_shape(xi, eta, N);
}

/* Local coordinates of local node l. */
static void node_local(const orc_t *o, int l, double *xi, double *eta)
{
    if (o->etype == 1) {
        *xi = Q2_I[l] - 1.0;
        *eta = Q2_J[l] - 1.0;
    } else {
        *xi = LOCAL_XI[l][0];
        *eta = LOCAL_XI[l][1];
    }
}

/* Jacobian {x_xi, x_eta, y_xi, y_eta} of element e at (xi, eta). */
static void elem_jacobian(const orc_t *o, int e, double xi, double eta, double *J)
{
    const double *v = &o->ev[EVS * e];
    if (o->etype == 1) {
        bilinear(v, xi, eta, NULL, NULL, J);
        return;
    }
    J[0] = v[2] - v[0];
    J[1] = v[4] - v[0];
    J[2] = v[3] - v[1];
    J[3] = v[5] - v[1];
}

/* Local index of node a in element e, or -1. */
static int local_index(const orc_t *o, int e, int a)
{
    for (int l = 0; l < o->nne; ++l)
        if (o->conn[o->nne * e + l] == a) return l;
    return -1;
}

/* ---------------------------------------------------------------------
 * Motion: x = G(X, t), its Jacobian g and the mesh velocity V_G = dG/dt|X
 * (Sec. II; maps of Sec. V).  Per-node static factors come from libm once;
 * per-step scalars come from libm once per step.
 * ------------------------------------------------------------------- */
typedef struct {
    double s, sd;       /* sine map */
    double vy, yoff;    /* plunge velocity and offset */
    double c, sn, thd;  /* rotation cos, sin, angular rate */
    double cm;          /* cos - 1 */
} mscal_t;

static void motion_static(orc_t *o)
{
    o->ms = xcalloc((size_t)6 * o->nn, sizeof(double));
    for (int a = 0; a < o->nn; ++a) {
        double X = o->X[2 * a], Y = o->X[2 * a + 1];
        double *m = &o->ms[6 * a];
        if (o->mkind == MK_SINE) {
            double A = o->mp[0], L = o->mp[1];
            double w = 2.0 * M_PI / L;
            if (o->mp[3] == 0.0) {
                /* x = X + A sin(2 pi Y/L) s(t),  y = Y + A sin(2 pi X/L) s(t) */
                m[0] = A * sin(w * Y);
                m[1] = A * sin(w * X);
                m[2] = 0.0;
                m[3] = (A * w) * cos(w * Y);
                m[4] = (A * w) * cos(w * X);
                m[5] = 0.0;
            } else {
                /* Sec. V.A: x = X + A sin(2piX/L) sin(2piY/L) s(t), same for y */
                double S = sin(w * X) * sin(w * Y);
                m[0] = A * S;
                m[1] = A * S;
                m[2] = (A * w) * (cos(w * X) * sin(w * Y));
                m[3] = (A * w) * (sin(w * X) * cos(w * Y));
                m[4] = m[2];
                m[5] = m[3];
            }
        } else if (o->mkind == MK_BLENDED) {
            /* b(r): 1 for r <= r1, 0 for r >= r2, cubic smoothstep between */
            double Xc = o->mp[3], Yc = o->mp[4], r1 = o->mp[5], r2 = o->mp[6];
            double dx = X - Xc, dy = Y - Yc;
            double r = sqrt(dx * dx + dy * dy);
            double b = 1.0, bX = 0.0, bY = 0.0;
            if (r >= r2) {
                b = 0.0;
            } else if (r > r1) {
                double s = (r - r1) / (r2 - r1);
                b = 1.0 - s * s * (3.0 - 2.0 * s);
                double dbdr = -(6.0 * s * (1.0 - s)) / (r2 - r1);
                bX = dbdr * (dx / r);
                bY = dbdr * (dy / r);
            }
            m[0] = b;
            m[1] = bX;
            m[2] = bY;
        }
    }
}

static void motion_scalars(const orc_t *o, double t, mscal_t *S)
{
    memset(S, 0, sizeof(*S));
    const double *p = o->mp;
    if (o->mkind == MK_SINE) {
        double Tp = p[2];
        S->s = sin(2.0 * M_PI * t / Tp);
        S->sd = (2.0 * M_PI / Tp) * cos(2.0 * M_PI * t / Tp);
    } else if (o->mkind == MK_PLUNGE) {
        double h = p[0], om = p[1];
        S->yoff = -h * sin(om * t);
        S->vy = -(h * om) * cos(om * t);
    } else if (o->mkind >= MK_PITCH) {
        double th0 = p[0], A = p[1], om = p[2];
        double th = th0 + A * sin(om * t);
        S->c = cos(th);
        S->sn = sin(th);
        S->thd = (A * om) * cos(om * t);
        S->cm = -2.0 * sin(0.5 * th) * sin(0.5 * th);
        if (o->mkind == MK_PITCH_PLUNGE) {
            double h = p[5], omh = p[6];
            S->yoff = -h * sin(omh * t);
            S->vy = -(h * omh) * cos(omh * t);
        }
    }
}

/* Metrics x_X, x_Y, y_X, y_Y and V_G at node a (the FP64 expression order
   here is the canonical one; both implementations follow it). */
static void motion_node(const orc_t *o, int a, const mscal_t *S, double *xX, double *xY,
                        double *yX, double *yY, double *Vx, double *Vy)
{
    const double *m = &o->ms[6 * a];
    double X = o->X[2 * a], Y = o->X[2 * a + 1];
    switch (o->mkind) {
    case MK_SINE:
        *xX = 1.0 + m[2] * S->s;
        *xY = m[3] * S->s;
        *yX = m[4] * S->s;
        *yY = 1.0 + m[5] * S->s;
        *Vx = m[0] * S->sd;
        *Vy = m[1] * S->sd;
        break;
    case MK_PLUNGE:
        *xX = 1.0;
        *xY = 0.0;
        *yX = 0.0;
        *yY = 1.0;
        *Vx = 0.0;
        *Vy = S->vy;
        break;
    case MK_PITCH:
    case MK_PITCH_PLUNGE: {
        double dx = X - o->mp[3], dy = Y - o->mp[4];
        *xX = S->c;
        *xY = -S->sn;
        *yX = S->sn;
        *yY = S->c;
        *Vx = S->thd * ((-S->sn) * dx - S->c * dy);
        *Vy = S->thd * (S->c * dx - S->sn * dy) + S->vy;
        break;
    }
    case MK_BLENDED: {
        double dx = X - o->mp[3], dy = Y - o->mp[4];
        double b = m[0], bX = m[1], bY = m[2];
        double qx = S->cm * dx - S->sn * dy;
        double qy = S->sn * dx + S->cm * dy;
        *xX = (1.0 + b * S->cm) + qx * bX;
        *xY = (-(b * S->sn)) + qx * bY;
        *yX = b * S->sn + qy * bX;
        *yY = (1.0 + b * S->cm) + qy * bY;
        *Vx = (b * S->thd) * ((-S->sn) * dx - S->c * dy);
        *Vy = (b * S->thd) * (S->c * dx - S->sn * dy);
        break;
    }
    default:
        *xX = 1.0;
        *xY = 0.0;
        *yX = 0.0;
        *yY = 1.0;
        *Vx = 0.0;
        *Vy = 0.0;
    }
}

/* Physical position G(X, t) of node a (used by the force integral). */
static void motion_position(const orc_t *o, int a, const mscal_t *S, double *x, double *y)
{
    const double *m = &o->ms[6 * a];
    double X = o->X[2 * a], Y = o->X[2 * a + 1];
    switch (o->mkind) {
    case MK_SINE:
        *x = X + m[0] * S->s;
        *y = Y + m[1] * S->s;
        break;
    case MK_PLUNGE:
        *x = X;
        *y = Y + S->yoff;
        break;
    case MK_PITCH:
    case MK_PITCH_PLUNGE: {
        double dx = X - o->mp[3], dy = Y - o->mp[4];
        *x = o->mp[3] + (dx * S->c - dy * S->sn);
        *y = o->mp[4] + (dx * S->sn + dy * S->c) + S->yoff;
        break;
    }
    case MK_BLENDED: {
        double dx = X - o->mp[3], dy = Y - o->mp[4];
        *x = X + m[0] * (S->cm * dx - S->sn * dy);
        *y = Y + m[0] * (S->sn * dx + S->cm * dy);
        break;
    }
    default:
        *x = X;
        *y = Y;
    }
}

/* g^{-1,T} (the ordinary inverse of the Jacobian) at node a:
   g^{-1} = (1/det g) [[y_Y, -y_X], [-x_Y, x_X]], det g = x_X y_Y - y_X x_Y.
   gi = {a11, a12, a21, a22} with g^{-1,T} = [[a11, a12], [a21, a22]]. */
static int metric_inverse(double xX, double xY, double yX, double yY, double *gi)
{
    double det = xX * yY - yX * xY;
    if (!(det > 0.0)) return ST_MAP;
    double inv = 1.0 / det;
    gi[0] = yY * inv;
    gi[1] = -(xY * inv);
    gi[2] = -(yX * inv);
    gi[3] = xX * inv;
    return ST_OK;
}

/* ---------------------------------------------------------------------
 * Mesh preparation
 * ------------------------------------------------------------------- */
static void qt_push_node(orc_t *o, qnode_t n)
{
    if (o->nqn == o->cap_qn) {
        o->cap_qn = o->cap_qn ? 2 * o->cap_qn : 1024;
        o->qn = realloc(o->qn, (size_t)o->cap_qn * sizeof(qnode_t));
        if (!o->qn) abort();
    }
    o->qn[o->nqn++] = n;
}

static void qt_push_ent(orc_t *o, qent_t e)
{
    if (o->nqe == o->cap_qe) {
        o->cap_qe = o->cap_qe ? 2 * o->cap_qe : 4096;
        o->qe = realloc(o->qe, (size_t)o->cap_qe * sizeof(qent_t));
        if (!o->qe) abort();
    }
    o->qe[o->nqe++] = e;
}

static void ent_bbox(const orc_t *o, qent_t q, double *b)
{
    const double *v = &o->ev[EVS * q.e];
    double x0 = v[0], x1 = v[0], y0 = v[1], y1 = v[1];
    for (int k = 1; k < o->nv; ++k) {
        x0 = fmin(x0, v[2 * k]);
        x1 = fmax(x1, v[2 * k]);
        y0 = fmin(y0, v[2 * k + 1]);
        y1 = fmax(y1, v[2 * k + 1]);
    }
    double sx = q.sx * o->Lx, sy = q.sy * o->Ly;
    b[0] = x0 + sx;
    b[1] = y0 + sy;
    b[2] = x1 + sx;
    b[3] = y1 + sy;
}

static void qt_build(orc_t *o, int node, qent_t *ents, int n, int depth)
{
    qnode_t nd = o->qn[node];
    if (n <= 12 || depth >= 26) {
        o->qn[node].child = -1;
        o->qn[node].start = o->nqe;
        o->qn[node].count = n;
        for (int k = 0; k < n; ++k) qt_push_ent(o, ents[k]);
        return;
    }
    double xm = 0.5 * (nd.x0 + nd.x1), ym = 0.5 * (nd.y0 + nd.y1);
    double bx[4][4] = {{nd.x0, nd.y0, xm, ym}, {xm, nd.y0, nd.x1, ym},
                       {nd.x0, ym, xm, nd.y1}, {xm, ym, nd.x1, nd.y1}};
    int first = o->nqn;
    for (int c = 0; c < 4; ++c) {
        qnode_t ch = {bx[c][0], bx[c][1], bx[c][2], bx[c][3], -1, 0, 0};
        qt_push_node(o, ch);
    }
    o->qn[node].child = first;
    qent_t *sub = xcalloc((size_t)n, sizeof(qent_t));
    for (int c = 0; c < 4; ++c) {
        qnode_t ch = o->qn[first + c];
        double mx = 1e-9 * (ch.x1 - ch.x0) + 1e-12, my = 1e-9 * (ch.y1 - ch.y0) + 1e-12;
        int m = 0;
        for (int k = 0; k < n; ++k) {
            double b[4];
            ent_bbox(o, ents[k], b);
            if (b[2] >= ch.x0 - mx && b[0] <= ch.x1 + mx && b[3] >= ch.y0 - my &&
                b[1] <= ch.y1 + my)
                sub[m++] = ents[k];
        }
        if (m == n && depth > 8) {
            /* no progress: make the child a leaf holding everything */
            o->qn[first + c].child = -1;
            o->qn[first + c].start = o->nqe;
            o->qn[first + c].count = m;
            for (int k = 0; k < m; ++k) qt_push_ent(o, sub[k]);
        } else {
            qt_build(o, first + c, sub, m, depth + 1);
        }
    }
    free(sub);
}

static int qt_leaf(const orc_t *o, double x, double y)
{
    const qnode_t *r = &o->qn[0];
    if (x < r->x0 || x > r->x1 || y < r->y0 || y > r->y1) return -1;
    int node = 0;
    while (o->qn[node].child >= 0) {
        const qnode_t *nd = &o->qn[node];
        double xm = 0.5 * (nd->x0 + nd->x1), ym = 0.5 * (nd->y0 + nd->y1);
        int c = (x >= xm ? 1 : 0) + (y >= ym ? 2 : 0);
        node = nd->child + c;
    }
    return node;
}

/* p in the closed (convex, straight-edged) element with nv vertices v,
   shifted by (sx, sy): exact signs against every edge. */
static int contains_closed(const double *v, int nv, double sx, double sy, double px, double py,
                           int *zeros)
{
    int z = 0;
    for (int k = 0; k < nv; ++k) {
        int k1 = (k + 1) % nv;
        int s = orc_orient(v[2 * k] + sx, v[2 * k + 1] + sy, v[2 * k1] + sx, v[2 * k1 + 1] + sy,
                           px, py);
        if (s < 0) return 0;
        if (s == 0) ++z;
    }
    if (zeros) *zeros = z;
    return 1;
}

/* Point location by exhaustive candidate search: every element whose
   bounding box holds p is tested exactly; among the containing (closed)
   elements the one of larger computational area, then lower id, wins
   (reading R5).  Returns the element, or -1 with no containing element. */
static int locate_point(const orc_t *o, double px, double py, double *shx, double *shy)
{
    double kx = 0, ky = 0, qx = px, qy = py;
    if (o->Lx > 0) {
        kx = floor(px / o->Lx);
        qx = px - kx * o->Lx;
        if (qx >= o->Lx) qx = nextafter(o->Lx, 0);
        if (qx < 0) qx = 0;
    }
    if (o->Ly > 0) {
        ky = floor(py / o->Ly);
        qy = py - ky * o->Ly;
        if (qy >= o->Ly) qy = nextafter(o->Ly, 0);
        if (qy < 0) qy = 0;
    }
    int leaf = qt_leaf(o, qx, qy);
    if (leaf < 0) return -1;
    int best = -1;
    double bsx = 0, bsy = 0;
    const qnode_t *nd = &o->qn[leaf];
    for (int k = 0; k < nd->count; ++k) {
        qent_t q = o->qe[nd->start + k];
        double sx = (q.sx + kx) * o->Lx, sy = (q.sy + ky) * o->Ly;
        const double *v = &o->ev[EVS * q.e];
        double x0 = v[0], x1 = v[0], y0 = v[1], y1 = v[1];
        for (int j = 1; j < o->nv; ++j) {
            x0 = fmin(x0, v[2 * j]);
            x1 = fmax(x1, v[2 * j]);
            y0 = fmin(y0, v[2 * j + 1]);
            y1 = fmax(y1, v[2 * j + 1]);
        }
        if (px < x0 + sx || px > x1 + sx || py < y0 + sy || py > y1 + sy)
            continue; /* outside the bounding box: cannot contain p */
        if (!contains_closed(v, o->nv, sx, sy, px, py, NULL)) continue;
        if (best < 0 || o->area2[q.e] > o->area2[best] ||
            (o->area2[q.e] == o->area2[best] && q.e < best)) {
            best = q.e;
            bsx = sx;
            bsy = sy;
        }
    }
    *shx = bsx;
    *shy = bsy;
    return best;
}

static double seg_point_dist(double ax, double ay, double bx, double by, double px, double py)
{
    double dx = bx - ax, dy = by - ay;
    double L2 = dx * dx + dy * dy;
    double t = L2 > 0 ? ((px - ax) * dx + (py - ay) * dy) / L2 : 0.0;
    t = fmin(1.0, fmax(0.0, t));
    double qx = ax + t * dx - px, qy = ay + t * dy - py;
    return sqrt(qx * qx + qy * qy);
}

static int prepare(orc_t *o)
{
    int nn = o->nn, ne = o->ne, nv = o->nv, nne = o->nne;
    o->ev = xcalloc((size_t)EVS * ne, sizeof(double));
    o->area2 = xcalloc((size_t)ne, sizeof(double));
    for (int e = 0; e < ne; ++e) {
        const int *c = &o->conn[nne * e];
        double x0 = o->X[2 * c[0]], y0 = o->X[2 * c[0] + 1];
        for (int l = 0; l < nne; ++l) {
            double x = o->X[2 * c[l]], y = o->X[2 * c[l] + 1];
            o->ev[EVS * e + 2 * l] = x0 + unwrap1(x - x0, o->Lx);
            o->ev[EVS * e + 2 * l + 1] = y0 + unwrap1(y - y0, o->Ly);
        }
        const double *v = &o->ev[EVS * e];
        double a2;
        if (o->etype == 1) {
            /* twice the area of the quadrilateral: half the cross product
               of its diagonals, doubled; every corner must turn left (a
               strictly convex cell, so that the bilinear map is one-to-one) */
            a2 = (v[4] - v[0]) * (v[7] - v[3]) - (v[6] - v[2]) * (v[5] - v[1]);
            for (int k = 0; k < 4; ++k) {
                int k1 = (k + 1) % 4, k2 = (k + 2) % 4;
                double cr = (v[2 * k1] - v[2 * k]) * (v[2 * k2 + 1] - v[2 * k1 + 1]) -
                            (v[2 * k1 + 1] - v[2 * k + 1]) * (v[2 * k2] - v[2 * k1]);
                if (!(cr > 0)) return ST_MESH;
            }
            /* the centre node is the bilinear map's value at (0, 0) */
            if (v[16] != 0.25 * (((v[0] + v[2]) + v[4]) + v[6]) ||
                v[17] != 0.25 * (((v[1] + v[3]) + v[5]) + v[7]))
                return ST_MESH;
        } else {
            a2 = (v[2] - v[0]) * (v[5] - v[1]) - (v[4] - v[0]) * (v[3] - v[1]);
        }
        if (!(a2 > 0)) return ST_MESH;
        o->area2[e] = a2;
        /* midside nodes must be the exact edge midpoints */
        for (int k = 0; k < nv; ++k) {
            int k1 = (k + 1) % nv;
            if (v[2 * nv + 2 * k] != 0.5 * (v[2 * k] + v[2 * k1]) ||
                v[2 * nv + 2 * k + 1] != 0.5 * (v[2 * k + 1] + v[2 * k1 + 1]))
                return ST_MESH;
        }
    }
    /* owner element of each node: the incident element of larger area,
       then lower id (Sec. IV: nodes on element edges belong to the element
       with the larger area) */
    o->owner = xcalloc((size_t)nn, sizeof(int));
    o->owner_loc = xcalloc((size_t)nn, sizeof(int));
    for (int a = 0; a < nn; ++a) o->owner[a] = -1;
    for (int e = 0; e < ne; ++e)
        for (int l = 0; l < nne; ++l) {
            int a = o->conn[nne * e + l];
            int b = o->owner[a];
            if (b < 0 || o->area2[e] > o->area2[b] || (o->area2[e] == o->area2[b] && e < b)) {
                o->owner[a] = e;
                o->owner_loc[a] = l;
            }
        }
    for (int a = 0; a < nn; ++a)
        if (o->owner[a] < 0) return ST_MESH;
    /* quadtree over element bounding boxes (with periodic images) */
    double bx0 = 1e300, by0 = 1e300, bx1 = -1e300, by1 = -1e300;
    if (o->Lx > 0) {
        bx0 = 0;
        bx1 = o->Lx;
    }
    if (o->Ly > 0) {
        by0 = 0;
        by1 = o->Ly;
    }
    for (int a = 0; a < nn; ++a) {
        if (o->Lx <= 0) {
            bx0 = fmin(bx0, o->X[2 * a]);
            bx1 = fmax(bx1, o->X[2 * a]);
        }
        if (o->Ly <= 0) {
            by0 = fmin(by0, o->X[2 * a + 1]);
            by1 = fmax(by1, o->X[2 * a + 1]);
        }
    }
    double pad = 1e-6 * fmax(bx1 - bx0, by1 - by0);
    if (o->Lx <= 0) {
        bx0 -= pad;
        bx1 += pad;
    }
    if (o->Ly <= 0) {
        by0 -= pad;
        by1 += pad;
    }
    qent_t *all = xcalloc((size_t)9 * ne, sizeof(qent_t));
    int nall = 0;
    for (int e = 0; e < ne; ++e)
        for (int sy = -1; sy <= 1; ++sy)
            for (int sx = -1; sx <= 1; ++sx) {
                if ((sx && o->Lx <= 0) || (sy && o->Ly <= 0)) continue;
                qent_t q = {e, (int8_t)sx, (int8_t)sy};
                double b[4];
                ent_bbox(o, q, b);
                if (b[2] < bx0 || b[0] > bx1 || b[3] < by0 || b[1] > by1) continue;
                all[nall++] = q;
            }
    qnode_t root = {bx0, by0, bx1, by1, -1, 0, 0};
    qt_push_node(o, root);
    qt_build(o, 0, all, nall, 0);
    free(all);
    /* boundary edges */
    o->nbe = 0;
    for (int e = 0; e < ne; ++e)
        for (int k = 0; k < nv; ++k)
            if (o->ekind[nv * e + k] != EK_INTERIOR) o->nbe++;
    o->be = xcalloc((size_t)o->nbe, sizeof(bedge_t));
    int nb = 0;
    for (int e = 0; e < ne; ++e)
        for (int k = 0; k < nv; ++k)
            if (o->ekind[nv * e + k] != EK_INTERIOR) {
                o->be[nb].elem = e;
                o->be[nb].k = k;
                o->be[nb].kind = o->ekind[nv * e + k];
                nb++;
            }
    /* per node: boundary edges (with periodic image) within rchk */
    o->rchk = 6.0;
    o->bnear_ptr = xcalloc((size_t)nn + 1, sizeof(int));
    int cap = 1024, cnt = 0;
    o->bnear_e = xcalloc((size_t)cap, sizeof(int));
    o->bnear_sx = xcalloc((size_t)cap, 1);
    o->bnear_sy = xcalloc((size_t)cap, 1);
    for (int a = 0; a < nn; ++a) {
        o->bnear_ptr[a] = cnt;
        double px = o->X[2 * a], py = o->X[2 * a + 1];
        for (int b = 0; b < o->nbe; ++b) {
            const double *v = &o->ev[EVS * o->be[b].elem];
            int k = o->be[b].k, k1 = (k + 1) % nv;
            for (int sy = -1; sy <= 1; ++sy)
                for (int sx = -1; sx <= 1; ++sx) {
                    if ((sx && o->Lx <= 0) || (sy && o->Ly <= 0)) continue;
                    double ox = sx * o->Lx, oy = sy * o->Ly;
                    double d = seg_point_dist(v[2 * k] + ox, v[2 * k + 1] + oy, v[2 * k1] + ox,
                                              v[2 * k1 + 1] + oy, px, py);
                    if (d < o->rchk) {
                        if (cnt == cap) {
                            cap *= 2;
                            o->bnear_e = realloc(o->bnear_e, (size_t)cap * sizeof(int));
                            o->bnear_sx = realloc(o->bnear_sx, (size_t)cap);
                            o->bnear_sy = realloc(o->bnear_sy, (size_t)cap);
                        }
                        o->bnear_e[cnt] = b;
                        o->bnear_sx[cnt] = (int8_t)sx;
                        o->bnear_sy[cnt] = (int8_t)sy;
                        cnt++;
                    }
                }
        }
    }
    o->bnear_ptr[nn] = cnt;
    /* wall nodes, their unit normals into the fluid and the probe point
       B = A + n dt (Sec. IV.A) */
    o->is_wall = xcalloc((size_t)nn, 1);
    o->wall_n = xcalloc((size_t)2 * nn, sizeof(double));
    o->probe_e = xcalloc((size_t)nn, sizeof(int));
    o->probe_xi = xcalloc((size_t)2 * nn, sizeof(double));
    for (int b = 0; b < o->nbe; ++b) {
        if (o->be[b].kind != EK_WALL) continue;
        int e = o->be[b].elem, k = o->be[b].k, k1 = (k + 1) % nv;
        const double *v = &o->ev[EVS * e];
        double tx = v[2 * k1] - v[2 * k], ty = v[2 * k1 + 1] - v[2 * k + 1];
        double L = sqrt(tx * tx + ty * ty);
        double nx = -ty / L, ny = tx / L; /* left of v_k -> v_k+1: into the element */
        int nodes[3] = {o->conn[nne * e + k], o->conn[nne * e + nv + k], o->conn[nne * e + k1]};
        for (int j = 0; j < 3; ++j) {
            o->is_wall[nodes[j]] = 1;
            o->wall_n[2 * nodes[j]] += nx;
            o->wall_n[2 * nodes[j] + 1] += ny;
        }
    }
    for (int a = 0; a < nn; ++a) {
        o->probe_e[a] = -1;
        if (!o->is_wall[a]) continue;
        double nx = o->wall_n[2 * a], ny = o->wall_n[2 * a + 1];
        double L = sqrt(nx * nx + ny * ny);
        nx /= L;
        ny /= L;
        o->wall_n[2 * a] = nx;
        o->wall_n[2 * a + 1] = ny;
        double Bx = o->X[2 * a] + nx * 1.0, By = o->X[2 * a + 1] + ny * 1.0;
        double sx, sy;
        int e = locate_point(o, Bx, By, &sx, &sy);
        if (e < 0) return ST_MESH;
        o->probe_e[a] = e;
        if (elem_local(o, e, sx, sy, Bx, By, &o->probe_xi[2 * a], &o->probe_xi[2 * a + 1])) return ST_MESH;
    }
    /* element of each node's wall-condition gradients (reading R8): the
       incident element of larger area, then lower id, among those with a
       vertex on a wall edge; the owner element when none touches a wall */
    o->bcel = xcalloc((size_t)nn, sizeof(int));
    for (int a = 0; a < nn; ++a) o->bcel[a] = -1;
    for (int e = 0; e < o->ne; ++e) {
        int touches = 0;
        for (int k = 0; k < nv; ++k) touches |= o->is_wall[o->conn[nne * e + k]];
        if (!touches) continue;
        for (int l = 0; l < nne; ++l) {
            int a = o->conn[nne * e + l], b = o->bcel[a];
            if (b < 0 || o->area2[e] > o->area2[b] || (o->area2[e] == o->area2[b] && e < b)) o->bcel[a] = e;
        }
    }
    for (int a = 0; a < nn; ++a)
        if (o->bcel[a] < 0) o->bcel[a] = o->owner[a];
    return ST_OK;
}

/* ---------------------------------------------------------------------
 * Creation, state access
 * ------------------------------------------------------------------- */
/* etype 0: 6-node triangles (conn [6 ne], ekind [3 ne]); 1: the paper's
   9-node quadrilaterals (conn [9 ne], ekind [4 ne]). */
void *orc_create(int nn, const double *X, int ne, const int *conn, const uint8_t *ekind, int etype,
                 double Lx, double Ly, int mkind, const double *mp, const double *kin,
                 int *status)
{
    orc_t *o = xcalloc(1, sizeof(orc_t));
    o->nn = nn;
    o->ne = ne;
    o->etype = etype == 1 ? 1 : 0;
    o->nv = o->etype ? 4 : 3;
    o->nne = o->etype ? 9 : 6;
    o->X = xcalloc((size_t)2 * nn, sizeof(double));
    memcpy(o->X, X, (size_t)2 * nn * sizeof(double));
    o->conn = xcalloc((size_t)o->nne * ne, sizeof(int));
    memcpy(o->conn, conn, (size_t)o->nne * ne * sizeof(int));
    o->ekind = xcalloc((size_t)o->nv * ne, 1);
    memcpy(o->ekind, ekind, (size_t)o->nv * ne);
    o->Lx = Lx;
    o->Ly = Ly;
    o->mkind = mkind;
    memcpy(o->mp, mp, 16 * sizeof(double));
    kin_from(kin, &o->K);
    for (int e = 0; e < o->nne * ne; ++e)
        if (conn[e] < 0 || conn[e] >= nn) {
            *status = ST_MESH;
            return o;
        }
    *status = prepare(o);
    if (*status) return o;
    motion_static(o);
    size_t n9 = (size_t)NQ * nn;
    o->f = xcalloc(n9, sizeof(double));
    o->g = xcalloc(n9, sizeof(double));
    o->fs = xcalloc(n9, sizeof(double));
    o->gs = xcalloc(n9, sizeof(double));
    o->rho = xcalloc(nn, sizeof(double));
    o->ux = xcalloc(nn, sizeof(double));
    o->uy = xcalloc(nn, sizeof(double));
    o->T = xcalloc(nn, sizeof(double));
    o->m_rt = xcalloc(nn, sizeof(double));
    o->Qx = xcalloc(nn, sizeof(double));
    o->Qy = xcalloc(nn, sizeof(double));
    o->Dx = xcalloc(nn, sizeof(double));
    o->Dy = xcalloc(nn, sizeof(double));
    o->Xx = xcalloc(nn, sizeof(double));
    o->Xy = xcalloc(nn, sizeof(double));
    o->gi = xcalloc((size_t)4 * nn, sizeof(double));
    return o;
}

void orc_destroy(void *h)
{
    orc_t *o = h;
    if (!o) return;
    void *ptrs[] = {o->X, o->conn, o->ekind, o->ev, o->area2, o->owner, o->owner_loc, o->bcel, o->qn,
                    o->qe, o->be, o->bnear_ptr, o->bnear_e, o->bnear_sx, o->bnear_sy,
                    o->is_wall, o->wall_n, o->probe_e, o->probe_xi, o->ms, o->f, o->g,
                    o->rho, o->ux, o->uy, o->T, o->fs, o->gs, o->m_rt, o->Qx, o->Qy, o->Dx,
                    o->Dy, o->Xx, o->Xy, o->gi};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    free(o);
}

/* Free-stream start: f = f^eq(rho_inf, u_inf, T_inf), g = g^eq (impulsive start). */
void orc_init(void *h)
{
    orc_t *o = h;
    double fe[NQ], ge[NQ];
    feq_K(&o->K, o->K.rho_inf, o->K.ux_inf, o->K.uy_inf, o->K.T_inf, fe);
    geq_K(&o->K, o->K.rho_inf, o->K.ux_inf, o->K.uy_inf, o->K.T_inf, ge);
    for (int a = 0; a < o->nn; ++a) {
        for (int i = 0; i < NQ; ++i) {
            o->f[(size_t)i * o->nn + a] = fe[i];
            o->g[(size_t)i * o->nn + a] = ge[i];
        }
        o->rho[a] = o->K.rho_inf;
        o->ux[a] = o->K.ux_inf;
        o->uy[a] = o->K.uy_inf;
        o->T[a] = o->K.T_inf;
    }
    o->t = 0.0;
    o->nstep = 0;
    o->status = ST_OK;
}

void orc_set_state(void *h, const double *f, const double *g, const double *rho,
                   const double *ux, const double *uy, const double *T, double t)
{
    orc_t *o = h;
    size_t n9 = (size_t)NQ * o->nn;
    memcpy(o->f, f, n9 * sizeof(double));
    memcpy(o->g, g, n9 * sizeof(double));
    memcpy(o->rho, rho, o->nn * sizeof(double));
    memcpy(o->ux, ux, o->nn * sizeof(double));
    memcpy(o->uy, uy, o->nn * sizeof(double));
    memcpy(o->T, T, o->nn * sizeof(double));
    o->t = t;
}

void orc_get_state(void *h, double *f, double *g, double *rho, double *ux, double *uy,
                   double *T, double *t)
{
    orc_t *o = h;
    size_t n9 = (size_t)NQ * o->nn;
    if (f) memcpy(f, o->f, n9 * sizeof(double));
    if (g) memcpy(g, o->g, n9 * sizeof(double));
    if (rho) memcpy(rho, o->rho, o->nn * sizeof(double));
    if (ux) memcpy(ux, o->ux, o->nn * sizeof(double));
    if (uy) memcpy(uy, o->uy, o->nn * sizeof(double));
    if (T) memcpy(T, o->T, o->nn * sizeof(double));
    if (t) *t = o->t;
}

int orc_owner(void *h, int *owner, int *loc)
{
    orc_t *o = h;
    memcpy(owner, o->owner, o->nn * sizeof(int));
    if (loc) memcpy(loc, o->owner_loc, o->nn * sizeof(int));
    return 0;
}

/* ---------------------------------------------------------------------
 * Departure points (Eq. Boltzmann_Discretized): X_dp = X - c^_i dt, with
 * c^_i = g^{-1,T} c_i - g^{-1,T} V_G (reading R1; flag LITERAL_VG uses the
 * printed c^_i = g^{-1,T} c_i - V_G).
 * ------------------------------------------------------------------- */
static void departure(const orc_t *o, int a, const double *gi, double Vx, double Vy, int i,
                      double *chx, double *chy, double *px, double *py)
{
    double cx = CXI[i] + o->K.Ux, cy = CYI[i] + o->K.Uy; /* the lattice velocity */
    double wx, wy;
    if (o->K.flags & FLAG_LITERAL_VG) {
        wx = Vx;
        wy = Vy;
    } else {
        wx = gi[0] * Vx + gi[1] * Vy;
        wy = gi[2] * Vx + gi[3] * Vy;
    }
    *chx = (gi[0] * cx + gi[1] * cy) - wx;
    *chy = (gi[2] * cx + gi[3] * cy) - wy;
    *px = o->X[2 * a] - *chx;
    *py = o->X[2 * a + 1] - *chy;
}

/* Departure point on the exact characteristic (flag EXACT_CHAR): the
   physical position G(X_a, t1) moved back by c_i dt (dt = 1), mapped back
   to the computational frame with the map of t0 = t1 - 1.  The inverses:
   plunge y -> y - yoff(t0); rigid pitch x -> X_c + R(theta(t0))^T (x - X_c
   - (0, yoff(t0))). */
static void exact_departure(const orc_t *o, int a, const mscal_t *S1, const mscal_t *S0, int i,
                            double *px, double *py)
{
    double x1, y1;
    motion_position(o, a, S1, &x1, &y1);
    double x0 = x1 - (CXI[i] + o->K.Ux), y0 = y1 - (CYI[i] + o->K.Uy);
    switch (o->mkind) {
    case MK_PLUNGE:
        *px = x0;
        *py = y0 - S0->yoff;
        break;
    case MK_PITCH:
    case MK_PITCH_PLUNGE: {
        double dx = x0 - o->mp[3], dy = (y0 - o->mp[4]) - S0->yoff;
        *px = o->mp[3] + (dx * S0->c + dy * S0->sn);
        *py = o->mp[4] + (dy * S0->c - dx * S0->sn);
        break;
    }
    default:
        *px = x0;
        *py = y0;
    }
}

/* Element choice for population i of node a (readings R5, R6).
   R6: the population is missing when some point of the segment X_a -> p
   lies outside the closed mesh.  Decided exactly enough by splitting the
   segment at every parameter where it meets a nearby boundary edge and
   locating p and one point inside each piece: between two consecutive
   meeting points the segment is wholly inside or wholly outside.
   Returns element >= 0 (with shift), -2 for "the node itself", or -1 with
   *kind = wall/far field for a missing population. */
static int choose_element(const orc_t *o, int a, double chx, double chy, double px, double py,
                          double *shx, double *shy, int *kind)
{
    *kind = 0;
    if (chx == 0.0 && chy == 0.0) return -2;
    if (sqrt(chx * chx + chy * chy) >= o->rchk - 1.0) return -3;
    double ax = o->X[2 * a], ay = o->X[2 * a + 1];
    int e = locate_point(o, px, py, shx, shy);
    int nb = o->bnear_ptr[a + 1] - o->bnear_ptr[a];
    if (nb == 0) {
        if (e < 0) return -3; /* outside with no boundary in reach */
        return e;
    }
    double tau[130];
    int tk[130];
    int nt = 0;
    int hit_kind = 0;
    double hit_tau = 2.0, near_d = 1e300;
    int near_kind = 0;
    double dx = px - ax, dy = py - ay, L2 = dx * dx + dy * dy;
    for (int k = o->bnear_ptr[a]; k < o->bnear_ptr[a + 1]; ++k) {
        const bedge_t *b = &o->be[o->bnear_e[k]];
        const double *v = &o->ev[EVS * b->elem];
        int k0 = b->k, k1 = (b->k + 1) % o->nv;
        double ox = o->bnear_sx[k] * o->Lx, oy = o->bnear_sy[k] * o->Ly;
        double ux = v[2 * k0] + ox, uy = v[2 * k0 + 1] + oy;
        double wx = v[2 * k1] + ox, wy = v[2 * k1 + 1] + oy;
        double d = seg_point_dist(ux, uy, wx, wy, ax, ay);
        if (d < near_d) {
            near_d = d;
            near_kind = b->kind;
        }
        int o1 = orc_orient(ax, ay, px, py, ux, uy);
        int o2 = orc_orient(ax, ay, px, py, wx, wy);
        int o3 = orc_orient(ux, uy, wx, wy, ax, ay);
        int o4 = orc_orient(ux, uy, wx, wy, px, py);
        double t1, t2 = -1.0;
        if (o1 == 0 && o2 == 0) {
            /* collinear: the edge's endpoints projected on the segment */
            t1 = ((ux - ax) * dx + (uy - ay) * dy) / L2;
            t2 = ((wx - ax) * dx + (wy - ay) * dy) / L2;
            if ((t1 < 0 && t2 < 0) || (t1 > 1 && t2 > 1)) continue;
        } else if (o1 * o2 <= 0 && o3 * o4 <= 0) {
            double den = dx * (wy - uy) - dy * (wx - ux);
            t1 = den != 0.0 ? ((ux - ax) * (wy - uy) - (uy - ay) * (wx - ux)) / den : 0.0;
        } else {
            continue;
        }
        double tt[2] = {t1, t2};
        for (int j = 0; j < 2; ++j) {
            if (j == 1 && t2 < 0 && !(o1 == 0 && o2 == 0)) break;
            double t = fmin(1.0, fmax(0.0, tt[j]));
            if (nt < 128) {
                tau[nt] = t;
                tk[nt] = b->kind;
                nt++;
            }
            if (t < hit_tau) {
                hit_tau = t;
                hit_kind = b->kind;
            }
        }
    }
    (void)tk;
    int outside = e < 0;
    if (!outside && nt > 0) {
        tau[nt++] = 0.0;
        tau[nt++] = 1.0;
        /* insertion sort */
        for (int i = 1; i < nt; ++i)
            for (int j = i; j > 0 && tau[j] < tau[j - 1]; --j) {
                double tmp = tau[j];
                tau[j] = tau[j - 1];
                tau[j - 1] = tmp;
            }
        for (int i = 0; i + 1 < nt && !outside; ++i) {
            if (!(tau[i + 1] > tau[i])) continue;
            double tm = 0.5 * (tau[i] + tau[i + 1]);
            double qx = ax + tm * dx, qy = ay + tm * dy, sx2, sy2;
            if (locate_point(o, qx, qy, &sx2, &sy2) < 0) outside = 1;
        }
    }
    if (!outside) return e;
    *kind = hit_kind ? hit_kind : near_kind;
    if (!*kind) return -3;
    return -1;
}

/* FE derivative d/dX of nodal field K at node a in its owner element
   (Eq. FE_Derivative with J^{-1} of the element at the node: constant on
   the straight-sided triangle, that of the bilinear map at the node's
   local position on the quadrilateral). */
static void fe_grad_X(const orc_t *o, int a, const double *K, double *KX, double *KY)
{
    int e = o->owner[a], l = o->owner_loc[a], nne = o->nne;
    double xl, yl, J[4];
    node_local(o, l, &xl, &yl);
    elem_jacobian(o, e, xl, yl, J);
    double x_xi = J[0], x_eta = J[1];
    double y_xi = J[2], y_eta = J[3];
    double detJ = x_xi * y_eta - y_xi * x_eta;
    double Nxi[9], Neta[9];
    if (o->etype == 1) shape_dxi_q2(xl, yl, Nxi, Neta);
    else shape_dxi(xl, yl, Nxi, Neta);
    double sxi = 0, seta = 0;
    for (int s = 0; s < nne; ++s) {
        double Ks = K[o->conn[nne * e + s]];
        sxi += Ks * Nxi[s];
        seta += Ks * Neta[s];
    }
    /* J^{-1} = (1/det J) [[d_eta y, -d_xi y], [-d_eta x, d_xi x]] */
    *KX = (y_eta * sxi - y_xi * seta) / detJ;
    *KY = (-x_eta * sxi + x_xi * seta) / detJ;
}

/* First-order FE derivative d/dX of a nodal field at node a: the gradient
   of the interpolant through the vertices alone of the node's
   wall-condition element (R8) -- linear on the triangle, bilinear on the
   quadrilateral, taken at the node.  Used for the non-equilibrium part of
   the wall condition, where a first-order gradient suffices (Sec. IV.A,
   last paragraph). */
static void fe_grad_X_linear(const orc_t *o, int a, const double *K, double *KX, double *KY)
{
    int e = o->bcel[a], nne = o->nne;
    if (o->etype == 1) {
        double xl, yl, J[4];
        node_local(o, local_index(o, e, a), &xl, &yl);
        elem_jacobian(o, e, xl, yl, J);
        double nxi[4] = {-0.25 * (1.0 - yl), 0.25 * (1.0 - yl), 0.25 * (1.0 + yl), -0.25 * (1.0 + yl)};
        double neta[4] = {-0.25 * (1.0 - xl), -0.25 * (1.0 + xl), 0.25 * (1.0 + xl), 0.25 * (1.0 - xl)};
        double sxi = 0, seta = 0;
        for (int k = 0; k < 4; ++k) {
            sxi += nxi[k] * K[o->conn[nne * e + k]];
            seta += neta[k] * K[o->conn[nne * e + k]];
        }
        double detJ = J[0] * J[3] - J[2] * J[1];
        *KX = (J[3] * sxi - J[2] * seta) / detJ;
        *KY = (-J[1] * sxi + J[0] * seta) / detJ;
        return;
    }
    const double *v = &o->ev[EVS * e];
    double x_xi = v[2] - v[0], x_eta = v[4] - v[0];
    double y_xi = v[3] - v[1], y_eta = v[5] - v[1];
    double detJ = x_xi * y_eta - y_xi * x_eta;
    double sxi = K[o->conn[nne * e + 1]] - K[o->conn[nne * e]];
    double seta = K[o->conn[nne * e + 2]] - K[o->conn[nne * e]];
    *KX = (y_eta * sxi - y_xi * seta) / detJ;
    *KY = (-x_eta * sxi + x_xi * seta) / detJ;
}

/* Physical derivative d_x K = g^{-1} d_X K (Eq. Ph_Derivative), with
   g^{-1} = [[a11, a21], [a12, a22]] in terms of gi = g^{-1,T}. */
static void phys_grad(const double *gi, double KX, double KY, double *Kx, double *Ky)
{
    *Kx = gi[0] * KX + gi[2] * KY;
    *Ky = gi[1] * KX + gi[3] * KY;
}

static double interp_field(const orc_t *o, int e, double sx, double sy, double px, double py,
                           const double *K)
{
    double xi, eta, N[9];
    elem_local(o, e, sx, sy, px, py, &xi, &eta);
    elem_shape(o, xi, eta, N);
    double s = 0;
    for (int k = 0; k < o->nne; ++k) s += N[k] * K[o->conn[o->nne * e + k]];
    return s;
}

/* Semi-Lagrangian FE propagation (Eq. Propagation) of all populations of
   one node; the missing ones from the Grad boundary condition. */
/* Sd: map scalars of the transformed velocities (the arrival time S, or
   t_{n+1/2} under FLAG_MIDPOINT, reading R2); the wall condition and the
   derivatives keep S. */
static int stream_node(orc_t *o, int a, const mscal_t *S, const mscal_t *Sd, const mscal_t *S0)
{
    int nn = o->nn;
    const double *gi = &o->gi[4 * a];
    double xX, xY, yX, yY, Vx, Vy;
    motion_node(o, a, S, &xX, &xY, &yX, &yY, &Vx, &Vy);
    double gd[4], Vdx = Vx, Vdy = Vy;
    const double *gdep = gi;
    if (Sd != S) {
        double dxX, dxY, dyX, dyY;
        motion_node(o, a, Sd, &dxX, &dxY, &dyX, &dyY, &Vdx, &Vdy);
        if (metric_inverse(dxX, dxY, dyX, dyY, gd)) return ST_MAP;
        gdep = gd;
    }
    int have_bc = 0;
    double tgt[4], du[4], dT[2];
    for (int i = 0; i < NQ; ++i) {
        double chx, chy, px, py, sx, sy;
        if (S0) { /* the exact characteristic */
            exact_departure(o, a, S, S0, i, &px, &py);
            chx = o->X[2 * a] - px;
            chy = o->X[2 * a + 1] - py;
        } else {
            departure(o, a, gdep, Vdx, Vdy, i, &chx, &chy, &px, &py);
        }
        int kind;
        int e = choose_element(o, a, chx, chy, px, py, &sx, &sy, &kind);
        if (e == -3) return ST_LOCATE;
        if (e == -2) {
            o->fs[(size_t)i * nn + a] = o->f[(size_t)i * nn + a];
            o->gs[(size_t)i * nn + a] = o->g[(size_t)i * nn + a];
            continue;
        }
        if (e >= 0) {
            /* local coordinates of the departure point (closed form on the
               triangle, Eq. NonLinear_Eq on the quadrilateral), then the
               interpolation of Eq. Propagation */
            double xi, eta, N[9];
            if (elem_local(o, e, sx, sy, px, py, &xi, &eta)) return ST_LOCATE;
            elem_shape(o, xi, eta, N);
            double sf = 0, sg = 0;
            for (int k = 0; k < o->nne; ++k) {
                int b = o->conn[o->nne * e + k];
                sf += N[k] * o->f[(size_t)i * nn + b];
                sg += N[k] * o->g[(size_t)i * nn + b];
            }
            o->fs[(size_t)i * nn + a] = sf;
            o->gs[(size_t)i * nn + a] = sg;
            continue;
        }
        /* missing population */
        double fm[NQ], gm[NQ];
        if (kind == EK_FAR) {
            feq_K(&o->K, o->K.rho_inf, o->K.ux_inf, o->K.uy_inf, o->K.T_inf, fm);
            geq_K(&o->K, o->K.rho_inf, o->K.ux_inf, o->K.uy_inf, o->K.T_inf, gm);
        } else {
            if (!have_bc) {
                if (o->is_wall[a]) {
                    int pe = o->probe_e[a];
                    double N[9];
                    elem_shape(o, o->probe_xi[2 * a], o->probe_xi[2 * a + 1], N);
                    double rB = 0, TB = 0, uB = 0, vB = 0;
                    for (int k = 0; k < o->nne; ++k) {
                        int b = o->conn[o->nne * pe + k];
                        rB += N[k] * o->rho[b];
                        TB += N[k] * o->T[b];
                        uB += N[k] * o->ux[b];
                        vB += N[k] * o->uy[b];
                    }
                    tgt[0] = rB;
                    tgt[1] = Vx; /* wall velocity: the mesh velocity of the wall node */
                    tgt[2] = Vy;
                    tgt[3] = TB;
                    if (o->K.flags & FLAG_SLIP_WALL) {
                        /* slip wall (reading of the inviscid variant): V_G plus the
                           tangential part of u_B - V_G; the physical normal is
                           g^{-1,T} applied to the computational one */
                        double nx, ny;
                        phys_grad(gi, o->wall_n[2 * a], o->wall_n[2 * a + 1], &nx, &ny);
                        double L = sqrt(nx * nx + ny * ny);
                        double tx = -ny / L, ty = nx / L;
                        double ut = (uB - Vx) * tx + (vB - Vy) * ty;
                        tgt[1] = Vx + ut * tx;
                        tgt[2] = Vy + ut * ty;
                    }
                } else {
                    tgt[0] = o->rho[a];
                    tgt[1] = o->ux[a];
                    tgt[2] = o->uy[a];
                    tgt[3] = o->T[a];
                    if (o->K.flags & FLAG_OFFWALL_VG) { /* reading R8c: the mesh velocity */
                        tgt[1] = Vx;
                        tgt[2] = Vy;
                    }
                }
                double KX, KY;
                fe_grad_X_linear(o, a, o->ux, &KX, &KY);
                phys_grad(gi, KX, KY, &du[0], &du[1]);
                fe_grad_X_linear(o, a, o->uy, &KX, &KY);
                phys_grad(gi, KX, KY, &du[2], &du[3]);
                fe_grad_X_linear(o, a, o->T, &KX, &KY);
                phys_grad(gi, KX, KY, &dT[0], &dT[1]);
                if ((o->K.flags & FLAG_BC_EQUILIBRIUM) || ((o->K.flags & FLAG_SLIP_WALL) && o->is_wall[a])) {
                    du[0] = du[1] = du[2] = du[3] = 0.0;
                    dT[0] = dT[1] = 0.0;
                }
                have_bc = 1;
            }
            grad_bc(&o->K, tgt[0], tgt[1], tgt[2], tgt[3], du, dT, fm, gm);
        }
        o->fs[(size_t)i * nn + a] = fm[i];
        o->gs[(size_t)i * nn + a] = gm[i];
    }
    return ST_OK;
}

/* One time step t_n -> t_{n+1} (Eqs. feqn, geqn). */
static int step_once(orc_t *o)
{
    int nn = o->nn;
    double t1 = o->t + 1.0;
    mscal_t S, Sh, Sz;
    motion_scalars(o, t1, &S);
    const mscal_t *Sd = &S, *S0 = NULL;
    if (o->K.flags & FLAG_EXACT_CHAR) { /* departure on the exact characteristic */
        if (!(o->mkind == MK_NONE || o->mkind == MK_PLUNGE || o->mkind == MK_PITCH ||
              o->mkind == MK_PITCH_PLUNGE))
            return ST_ARG;
        motion_scalars(o, o->t, &Sz);
        S0 = &Sz;
    } else if (o->K.flags & FLAG_MIDPOINT) { /* transformed velocities at t_{n+1/2} */
        motion_scalars(o, t1 - 0.5, &Sh);
        Sd = &Sh;
    }
    /* Every node below is computed on its own from shared read-only data and
       writes only its own entries, so the node loops may run on several
       threads (OpenMP) with results independent of the thread count. */
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int a = 0; a < nn; ++a) {
        double xX, xY, yX, yY, Vx, Vy;
        motion_node(o, a, &S, &xX, &xY, &yX, &yY, &Vx, &Vy);
        if (metric_inverse(xX, xY, yX, yY, &o->gi[4 * a])) bad = 1;
    }
    if (bad) return ST_MAP;
    /* propagation */
    int first_err = 0;
#pragma omp parallel for schedule(dynamic, 256)
    for (int a = 0; a < nn; ++a) {
        int st = stream_node(o, a, &S, Sd, S0);
        if (st) {
#pragma omp critical(orc_err)
            if (!first_err) first_err = st;
        }
    }
    if (first_err) return first_err;
    /* moments, Q'_aaa = rho w_a (1 - 3T) - rho w_a^3 with w = u - U (Eq. DeviationTerms),
       mu/(rho T) */
    double *R = xcalloc(nn, sizeof(double)), *UX = xcalloc(nn, sizeof(double)),
           *UY = xcalloc(nn, sizeof(double)), *TT = xcalloc(nn, sizeof(double));
    int nonfinite = 0;
#pragma omp parallel for schedule(static) reduction(| : nonfinite)
    for (int a = 0; a < nn; ++a) {
        double r = 0, jx = 0, jy = 0, e2 = 0;
        for (int i = 0; i < NQ; ++i) {
            double f = o->fs[(size_t)i * nn + a];
            r += f;
            jx += (CXI[i] + o->K.Ux) * f;
            jy += (CYI[i] + o->K.Uy) * f;
            e2 += o->gs[(size_t)i * nn + a];
        }
        double ux = jx / r, uy = jy / r, E = e2 / (2.0 * r);
        double T = (E - 0.5 * (ux * ux + uy * uy)) / o->K.Cv;
        if (!isfinite(r) || !isfinite(T) || !(r > 0) || !(T > 0)) {
            nonfinite = 1;
            continue;
        }
        R[a] = r;
        UX[a] = ux;
        UY[a] = uy;
        TT[a] = T;
        /* on the shifted lattice only sum c_a^3 f = sum c_a f about U departs
           from the Maxwellian: Q' in the relative velocity w = u - U (R14) */
        double wx = ux - o->K.Ux, wy = uy - o->K.Uy;
        o->Qx[a] = r * wx * (1.0 - 3.0 * T) - r * wx * wx * wx;
        o->Qy[a] = r * wy * (1.0 - 3.0 * T) - r * wy * wy * wy;
        o->m_rt[a] = o->K.mu / (r * T);
    }
    if (nonfinite) {
        free(R);
        free(UX);
        free(UY);
        free(TT);
        return ST_NONFINITE;
    }
    /* first derivative pass: D_a = (mu / rho T) d_a Q'_aaa (Eq. Xa) */
#pragma omp parallel for schedule(static)
    for (int a = 0; a < nn; ++a) {
        double KX, KY, dx, dy;
        fe_grad_X(o, a, o->Qx, &KX, &KY);
        phys_grad(&o->gi[4 * a], KX, KY, &dx, &dy);
        o->Dx[a] = o->m_rt[a] * dx;
        fe_grad_X(o, a, o->Qy, &KX, &KY);
        phys_grad(&o->gi[4 * a], KX, KY, &dx, &dy);
        o->Dy[a] = o->m_rt[a] * dy;
    }
    /* second pass: X_a = -d_a D_a */
#pragma omp parallel for schedule(static)
    for (int a = 0; a < nn; ++a) {
        double KX, KY, dx, dy;
        fe_grad_X(o, a, o->Dx, &KX, &KY);
        phys_grad(&o->gi[4 * a], KX, KY, &dx, &dy);
        o->Xx[a] = -dx;
        fe_grad_X(o, a, o->Dy, &KX, &KY);
        phys_grad(&o->gi[4 * a], KX, KY, &dx, &dy);
        o->Xy[a] = -dy;
        if (o->K.flags & FLAG_PHI_OFF) {
            o->Xx[a] = 0.0;
            o->Xy[a] = 0.0;
        }
    }
    /* collision */
#pragma omp parallel for schedule(static)
    for (int a = 0; a < nn; ++a) {
        double f[NQ], g[NQ], fo[NQ], go[NQ];
        for (int i = 0; i < NQ; ++i) {
            f[i] = o->fs[(size_t)i * nn + a];
            g[i] = o->gs[(size_t)i * nn + a];
        }
        if (o->K.flags & FLAG_COLLIDE_OFF) {
            memcpy(fo, f, sizeof(f));
            memcpy(go, g, sizeof(g));
        } else {
            collide(&o->K, f, g, o->Xx[a], o->Xy[a], fo, go);
        }
        for (int i = 0; i < NQ; ++i) {
            o->f[(size_t)i * nn + a] = fo[i];
            o->g[(size_t)i * nn + a] = go[i];
        }
    }
    memcpy(o->rho, R, nn * sizeof(double));
    memcpy(o->ux, UX, nn * sizeof(double));
    memcpy(o->uy, UY, nn * sizeof(double));
    memcpy(o->T, TT, nn * sizeof(double));
    free(R);
    free(UX);
    free(UY);
    free(TT);
    o->t = t1;
    o->nstep++;
    return ST_OK;
}

int orc_step(void *h, int n)
{
    orc_t *o = h;
    for (int k = 0; k < n; ++k) {
        int st = step_once(o);
        if (st) {
            o->status = st;
            return st;
        }
    }
    return ST_OK;
}

/* Element choices of all populations at map time t (for parity of the
   element location): elem[i*nn + a] = element id, -2 (node itself) or -1
   (missing; kind[] = 1 wall, 2 far field). */
int orc_locate(void *h, double t, int *elem, int8_t *kind)
{
    orc_t *o = h;
    mscal_t S;
    motion_scalars(o, t, &S);
    int bad = 0; /* 1: folded map, 2: walk limit */
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
    for (int a = 0; a < o->nn; ++a) {
        double xX, xY, yX, yY, Vx, Vy, gi[4];
        motion_node(o, a, &S, &xX, &xY, &yX, &yY, &Vx, &Vy);
        if (metric_inverse(xX, xY, yX, yY, gi)) {
            bad |= 1;
            continue;
        }
        for (int i = 0; i < NQ; ++i) {
            double chx, chy, px, py, sx, sy;
            int kd;
            departure(o, a, gi, Vx, Vy, i, &chx, &chy, &px, &py);
            int e = choose_element(o, a, chx, chy, px, py, &sx, &sy, &kd);
            if (e == -3) bad |= 2;
            elem[(size_t)i * o->nn + a] = e;
            kind[(size_t)i * o->nn + a] = (int8_t)(e == -1 ? kd : 0);
        }
    }
    return (bad & 1) ? ST_MAP : (bad & 2) ? ST_LOCATE : ST_OK;
}

/* Departure points at map time t (x and y, [i*nn + a]). */
int orc_departures(void *h, double t, double *px_out, double *py_out)
{
    orc_t *o = h;
    mscal_t S;
    motion_scalars(o, t, &S);
    for (int a = 0; a < o->nn; ++a) {
        double xX, xY, yX, yY, Vx, Vy, gi[4];
        motion_node(o, a, &S, &xX, &xY, &yX, &yY, &Vx, &Vy);
        if (metric_inverse(xX, xY, yX, yY, gi)) return ST_MAP;
        for (int i = 0; i < NQ; ++i) {
            double chx, chy;
            departure(o, a, gi, Vx, Vy, i, &chx, &chy, &px_out[(size_t)i * o->nn + a],
                      &py_out[(size_t)i * o->nn + a]);
        }
    }
    return ST_OK;
}

/* Departure points on the exact characteristic of a step arriving at t1
   (flag EXACT_CHAR's rule, whatever the flags; x and y, [i*nn + a]). */
int orc_departures_exact(void *h, double t1, double *px_out, double *py_out)
{
    orc_t *o = h;
    if (!(o->mkind == MK_NONE || o->mkind == MK_PLUNGE || o->mkind == MK_PITCH ||
          o->mkind == MK_PITCH_PLUNGE))
        return ST_ARG;
    mscal_t S1, S0;
    motion_scalars(o, t1, &S1);
    motion_scalars(o, t1 - 1.0, &S0);
    for (int a = 0; a < o->nn; ++a)
        for (int i = 0; i < NQ; ++i)
            exact_departure(o, a, &S1, &S0, i, &px_out[(size_t)i * o->nn + a], &py_out[(size_t)i * o->nn + a]);
    return ST_OK;
}

/* Map quantities at node a, time t: {x_X, x_Y, y_X, y_Y, V_x, V_y, x, y}. */
int orc_map(void *h, double t, int a, double *out)
{
    orc_t *o = h;
    mscal_t S;
    motion_scalars(o, t, &S);
    motion_node(o, a, &S, &out[0], &out[1], &out[2], &out[3], &out[4], &out[5]);
    motion_position(o, a, &S, &out[6], &out[7]);
    return ST_OK;
}

/* Physical owner-element gradient of a nodal field at map time t. */
int orc_fe_grad(void *h, double t, const double *K, double *gx, double *gy)
{
    orc_t *o = h;
    mscal_t S;
    motion_scalars(o, t, &S);
    for (int a = 0; a < o->nn; ++a) {
        double xX, xY, yX, yY, Vx, Vy, gi[4], KX, KY;
        motion_node(o, a, &S, &xX, &xY, &yX, &yY, &Vx, &Vy);
        if (metric_inverse(xX, xY, yX, yY, gi)) return ST_MAP;
        fe_grad_X(o, a, K, &KX, &KY);
        phys_grad(gi, KX, KY, &gx[a], &gy[a]);
    }
    return ST_OK;
}

/* Interpolate a nodal field at computational point p; returns the element
   (or -1). */
int orc_interp(void *h, double px, double py, const double *K, double *out)
{
    orc_t *o = h;
    double sx, sy;
    int e = locate_point(o, px, py, &sx, &sy);
    if (e >= 0) *out = interp_field(o, e, sx, sy, px, py, K);
    return e;
}

int orc_wall_info(void *h, uint8_t *is_wall, double *normal, int *probe_e, double *probe_xi)
{
    orc_t *o = h;
    if (is_wall) memcpy(is_wall, o->is_wall, o->nn);
    if (normal) memcpy(normal, o->wall_n, 2 * o->nn * sizeof(double));
    if (probe_e) memcpy(probe_e, o->probe_e, o->nn * sizeof(int));
    if (probe_xi) memcpy(probe_xi, o->probe_xi, 2 * o->nn * sizeof(double));
    return o->nbe;
}

/* Forces on the wall at the current time (reading R9):
   out = {Fx_p, Fy_p, Fx_v, Fy_v, c_D, c_L},
   c = F / (0.5 rho_inf |u_inf|^2 chord) along u_inf (drag) and +90 deg (lift). */
int orc_forces(void *h, double *out)
{
    orc_t *o = h;
    int nn = o->nn;
    mscal_t S;
    motion_scalars(o, o->t, &S);
    double Fp[2] = {0, 0}, Fv[2] = {0, 0};
    double *gi = xcalloc((size_t)4 * nn, sizeof(double));
    for (int a = 0; a < nn; ++a) {
        double xX, xY, yX, yY, Vx, Vy;
        motion_node(o, a, &S, &xX, &xY, &yX, &yY, &Vx, &Vy);
        metric_inverse(xX, xY, yX, yY, &gi[4 * a]);
    }
    for (int b = 0; b < o->nbe; ++b) {
        if (o->be[b].kind != EK_WALL) continue;
        int e = o->be[b].elem, k = o->be[b].k, k1 = (k + 1) % o->nv;
        int nodes[3] = {o->conn[o->nne * e + k], o->conn[o->nne * e + o->nv + k], o->conn[o->nne * e + k1]};
        double xa, ya, xb, yb;
        motion_position(o, nodes[0], &S, &xa, &ya);
        motion_position(o, nodes[2], &S, &xb, &yb);
        double tx = xb - xa, ty = yb - ya, L = sqrt(tx * tx + ty * ty);
        double nx = -ty / L, ny = tx / L; /* out of the body, into the fluid */
        double w[3] = {L / 6.0, 4.0 * L / 6.0, L / 6.0};
        for (int j = 0; j < 3; ++j) {
            int a = nodes[j];
            double p = o->rho[a] * o->T[a];
            double KX, KY, d[4];
            fe_grad_X(o, a, o->ux, &KX, &KY);
            phys_grad(&gi[4 * a], KX, KY, &d[0], &d[1]);
            fe_grad_X(o, a, o->uy, &KX, &KY);
            phys_grad(&gi[4 * a], KX, KY, &d[2], &d[3]);
            double div = d[0] + d[3];
            double txx = o->K.mu * (2.0 * d[0] - div / o->K.Cv);
            double tyy = o->K.mu * (2.0 * d[3] - div / o->K.Cv);
            double txy = o->K.mu * (d[1] + d[2]);
            Fp[0] += w[j] * (-p * nx);
            Fp[1] += w[j] * (-p * ny);
            Fv[0] += w[j] * (txx * nx + txy * ny);
            Fv[1] += w[j] * (txy * nx + tyy * ny);
        }
    }
    free(gi);
    double U2 = o->K.ux_inf * o->K.ux_inf + o->K.uy_inf * o->K.uy_inf;
    double U = sqrt(U2);
    double ex = U > 0 ? o->K.ux_inf / U : 1.0, ey = U > 0 ? o->K.uy_inf / U : 0.0;
    double q = 0.5 * o->K.rho_inf * U2 * o->K.chord;
    double Fx = Fp[0] + Fv[0], Fy = Fp[1] + Fv[1];
    out[0] = Fp[0];
    out[1] = Fp[1];
    out[2] = Fv[0];
    out[3] = Fv[1];
    out[4] = q > 0 ? (Fx * ex + Fy * ey) / q : 0.0;
    out[5] = q > 0 ? (-Fx * ey + Fy * ex) / q : 0.0;
    return ST_OK;
}

int orc_status(void *h) { return ((orc_t *)h)->status; }

/* Local coordinates of computational point p in element e (no periodic
   shift): out = {xi, eta}; returns 0 or ST_LOCATE. */
int orc_local(void *h, int e, double px, double py, double *out)
{
    orc_t *o = h;
    return elem_local(o, e, 0.0, 0.0, px, py, &out[0], &out[1]);
}

/* Threads of the node loops of a step: n > 0 sets the count (OpenMP),
   n <= 0 leaves it; returns the count in use (1 without OpenMP). */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
