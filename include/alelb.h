/*
 * alelb.h -- C-ABI of the GB300 library for the ALE compressible lattice
 * Boltzmann step on unstructured moving meshes (Saadat & Karlin,
 * arXiv 2002.04353).
 *
 * Conventions for every entry point
 *   - Return value: alelb_status (0 = OK, < 0 = error).  alelb_last_error()
 *     gives a message for the most recent error of a solver or mesh.
 *   - Ownership: the library owns all device memory it allocates; the caller
 *     owns every host array it passes.  Input host arrays are copied during
 *     the call and may be freed afterwards; output host arrays are filled
 *     before the call returns.
 *   - Node order: arrays exchanged with the caller are in the caller's
 *     original node numbering; the library renumbers internally.
 *   - Populations: D2Q9 direction order (0,0), (1,0), (0,1), (-1,0), (0,-1),
 *     (1,1), (-1,1), (-1,-1), (1,-1); population arrays are laid out
 *     [direction][node] (9 * n_nodes values for f, the same for g).
 *   - Units: lattice units, time step dt = 1.
 *   - Errors raised on the device (walk limit, non-finite state, wait
 *     limit) are sticky per solver and reported by the next synchronising
 *     call (alelb_sync, alelb_moments, alelb_get_pops, alelb_forces).
 */
#ifndef ALELB_H
#define ALELB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ALELB_OK = 0,
    ALELB_ERR_ARG = -1,       /* invalid argument */
    ALELB_ERR_OOM = -2,       /* device or host allocation failed */
    ALELB_ERR_CUDA = -3,      /* a CUDA runtime call failed */
    ALELB_ERR_MESH = -4,      /* inverted element, bad connectivity, bad midside node */
    ALELB_ERR_MAP = -5,       /* det g <= 0 somewhere at the requested time */
    ALELB_ERR_LOCATE = -6,    /* element walk exceeded its step limit */
    ALELB_ERR_NONFINITE = -7, /* non-finite or non-positive density/temperature */
    ALELB_ERR_TIMEOUT = -8,   /* a bounded device wait gave up */
    ALELB_ERR_STATE = -9      /* call order (e.g. stepping a destroyed solver) */
} alelb_status;

/* Motion kinds: the map x = G(X, t) of the computational domain onto the
   physical one (Sec. II).  Parameters in alelb_mesh_desc.motion[]:
   SINE        {A, L, T, variant}: variant 0: x = X + A sin(2 pi Y/L) s(t),
               y = Y + A sin(2 pi X/L) s(t); variant 1 (Sec. V.A):
               x = X + A sin(2 pi X/L) sin(2 pi Y/L) s(t), same for y;
               s(t) = sin(2 pi t/T)
   PLUNGE      {h, omega}: x = X, y = Y - h sin(omega t)   (Eq. Plunge_eq)
   PITCH       {theta0, A, omega, Xc, Yc}: rotation by theta = theta0 +
               A sin(omega t) about (Xc, Yc)                (Sec. V.C)
   PITCH_PLUNGE{theta0, A, omega, Xc, Yc, h, omega_h}: pitch plus plunge
   BLENDED_PITCH{theta0, A, omega, Xc, Yc, r1, r2}: x = X + b(r)[R(theta)
               (X - Xc) - (X - Xc)], b = 1 for r <= r1, 0 for r >= r2,
               cubic smoothstep between */
enum {
    ALELB_MOTION_NONE = 0,
    ALELB_MOTION_SINE = 1,
    ALELB_MOTION_PLUNGE = 2,
    ALELB_MOTION_PITCH = 3,
    ALELB_MOTION_PITCH_PLUNGE = 4,
    ALELB_MOTION_BLENDED_PITCH = 5
};

enum { ALELB_EDGE_INTERIOR = 0, ALELB_EDGE_WALL = 1, ALELB_EDGE_FARFIELD = 2 };
/* Element kinds (alelb_mesh_desc.elem_type): straight-sided 6-node
   triangles, or the paper's 9-node quadrilaterals (Sec. III). */
enum { ALELB_ELEM_P2TRI = 0, ALELB_ELEM_Q2QUAD = 1 };
enum { ALELB_RENUMBER_NONE = 0, ALELB_RENUMBER_MORTON = 1 };
/* Storage and arithmetic of a solver (Sec. IV's populations; the paper
   computes in FP64 and gives no reduced-precision form):
     FP64      full populations and fields in FP64, FP64 arithmetic, every
               departure point through the exact element walk;
     FP32_DEV  populations stored in FP32 as deviations from the rest
               equilibria at (rho_inf, T_inf), fields in FP32, FP32
               arithmetic with FP64 (certified) element decisions;
     BF16_DEV  as FP32_DEV, populations stored in bfloat16 as deviations
               from the far-field equilibria at (rho_inf, u_inf, T_inf);
     FP16_DEV  as BF16_DEV, populations stored in IEEE binary16 as 2^10
               times the deviation (|deviation| < 64).
   Element choices are the same in every form; values differ by the
   storage rounding. */
enum { ALELB_PREC_FP64 = 0, ALELB_PREC_FP32_DEV = 1, ALELB_PREC_BF16_DEV = 2, ALELB_PREC_FP16_DEV = 3 };

/* Solver flags (alelb_params.flags). */
enum {
    ALELB_FLAG_PHI_OFF = 1,        /* drop the correction terms phi_i (tests) */
    ALELB_FLAG_COLLIDE_OFF = 2,    /* pure propagation, no collision (tests) */
    ALELB_FLAG_LITERAL_VG = 4,     /* c^_i = g^{-1,T} c_i - V_G as printed in Eq. 7 */
    ALELB_FLAG_BC_EQUILIBRIUM = 8, /* missing populations: equilibrium part only */
    ALELB_FLAG_SLIP_WALL = 16,     /* slip (inviscid) walls: at wall nodes the target velocity is
                                      V_G plus the tangential part of u_B - V_G at the probe B,
                                      and the non-equilibrium part is dropped (no wall shear) */
    ALELB_FLAG_MIDPOINT = 32,      /* the transformed velocities c^_i of a step t_n -> t_{n+1}
                                      use g and V_G at t_{n+1/2} (Eq. 7 at the midpoint time;
                                      the wall condition and the derivatives stay at t_{n+1}).
                                      Single-case solvers only: alelb_batch_create refuses it */
    ALELB_FLAG_EXACT_CHAR = 64,    /* the departure point of population i is the reference position
                                      at t_n of the physical point G(X, t_{n+1}) - c_i, on the
                                      exact characteristic of Sec. III, in place of X - c^_i;
                                      rigid maps only (none, plunge, pitch, pitch with plunge):
                                      alelb_lb_init and alelb_lb_step_noalloc return
                                      ALELB_ERR_ARG for the others.  Every population of the
                                      deviation forms takes the exact path (its FP32
                                      certificates bound X - c^_i only).  Single-case solvers
                                      only: alelb_batch_create refuses it.  Takes precedence
                                      over ALELB_FLAG_MIDPOINT */
    /* 128 is reserved (internal). */
    ALELB_FLAG_OFFWALL_VG = 256    /* missing populations of off-wall nodes (nodes next to a moving
                                      wall whose departure segment crosses it) take the mesh
                                      velocity V_G at the node as their target velocity, in place
                                      of the node's previous-step velocity; density and
                                      temperature stay the node's.  The paper states targets for
                                      wall nodes only; with this reading the fluid layer that a
                                      receding wall leaves behind follows the wall, and the
                                      plunging airfoils stay stable over whole runs */
};

/* Mesh description (computational domain, Sec. III).
   ALELB_ELEM_P2TRI, straight-sided 6-node triangles: conn[6*e .. 6*e+5] =
   v0 v1 v2 (counter-clockwise), then the midside nodes of edges (v0,v1),
   (v1,v2), (v2,v0), which must be the exact edge midpoints;
   edge_kind[3*e + k] is the kind of edge k (v_k, v_k+1).
   ALELB_ELEM_Q2QUAD, the paper's 9-node quadrilaterals with straight edges
   (the bilinear cells of Eq. NonLinear_Eq): conn[9*e .. 9*e+8] = v0 v1 v2
   v3 (counter-clockwise, every corner turning left: strictly convex), the
   midside nodes of edges (v0,v1), (v1,v2), (v2,v3), (v3,v0) (exact edge
   midpoints), then the centre, exactly 0.25 (((v0 + v1) + v2) + v3);
   edge_kind[4*e + k].  The local coordinates of a departure point solve
   Eq. NonLinear_Eq by Newton's method from the cell centre (at most 8
   steps, stopping once converged).  The element choices are those of the
   exact FP64 departure path in every precision: the deviation forms accept
   the previous-step element only under a certified FP32 test, and send
   every other population down that path.  Quadrilateral meshes are not taken by the batched
   step, the learned proposal, alelb_samples or alelb_lb_step_noalloc
   (ALELB_ERR_ARG).
   period[d] > 0 makes direction d periodic with that period (coordinates
   in [0, period)).  All pointers are host pointers, read during
   alelb_mesh_create only. */
typedef struct {
    int32_t n_nodes;
    const double *X;          /* [2 * n_nodes], x0 y0 x1 y1 ... */
    int32_t n_elems;
    const int32_t *conn;      /* [6 * n_elems] */
    const uint8_t *edge_kind; /* [3 * n_elems] */
    double period[2];
    int32_t motion_kind;
    double motion[16];
    int32_t renumber;         /* ALELB_RENUMBER_* */
    int32_t elem_type;        /* ALELB_ELEM_* (zero: 6-node triangles) */
} alelb_mesh_desc;

/* Fluid and run parameters (Sec. IV; R = 1, Cv = 1/(gamma - 1), Cp = Cv + 1,
   mu constant, Pr = Cp mu / kappa).  stream: a cudaStream_t (NULL = the
   library's own non-blocking stream); every kernel of the solver runs on it. */
typedef struct {
    double gamma, Pr, mu, rho_inf, T_inf, u_inf[2], chord;
    int32_t precision; /* ALELB_PREC_* */
    int32_t flags;     /* ALELB_FLAG_* */
    void *stream;
    double shift[2];   /* lattice shift U (Sec. V.D): the discrete velocities are c_i + U.
                          Zero is the plain lattice.  Each component finite, |U_d| <= 1 and
                          exactly representable in FP32, else ALELB_ERR_ARG.  On the shifted
                          lattice the equilibria take the relative velocity u - U, the
                          general form of Eq. geq_gstar is applied to moments taken about U,
                          psi restores the diagonal second moments about U, Q' is taken in
                          u - U, and rho u = sum (c_i + U) f_i; the populations that
                          alelb_set_pops and alelb_get_pops exchange are those of c_i + U.
                          A batch may mix shifted and plain solvers */
} alelb_params;

typedef struct alelb_mesh alelb_mesh;
typedef struct alelb_solver alelb_solver;

/* Builds the device tables of a mesh: element frames, neighbours across
   edges (periodic shifts included), node fans, owner elements (Sec. IV:
   a node on element edges belongs to the incident element of larger
   area), wall normals and probe points B (Sec. IV.A), static per-node map
   factors.  Errors: ALELB_ERR_ARG (null/size), ALELB_ERR_MESH,
   ALELB_ERR_OOM, ALELB_ERR_CUDA.  The mesh must outlive its solvers. */
alelb_status alelb_mesh_create(const alelb_mesh_desc *desc, alelb_mesh **out);
void alelb_mesh_destroy(alelb_mesh *mesh);

/* Checks det g > 0 at every node at map time t (Sec. II, Eq. g_inv).
   Returns ALELB_ERR_MAP if the map folds; does not change any solver. */
alelb_status alelb_mesh_move(alelb_mesh *mesh, double t);

/* Creates a solver on the mesh and sets the free-stream state
   f = f^eq(rho_inf, u_inf, T_inf), g = g^eq (impulsive start) at t = 0. */
alelb_status alelb_lb_init(alelb_mesh *mesh, const alelb_params *p, alelb_solver **out);
void alelb_solver_destroy(alelb_solver *s);

/* Advances n >= 0 time steps t_k -> t_k + 1 (Eqs. feqn, geqn with the
   propagation of Eq. Propagation): per step, propagation with element
   location and the Grad-type missing populations (Sec. IV.A), moments,
   two FE-derivative passes for X_a (Eq. Xa), collision.  Asynchronous on
   the solver's stream. */
alelb_status alelb_lb_step(alelb_solver *s, int32_t n);

/* Waits for the solver's stream and reports any sticky device error. */
alelb_status alelb_sync(alelb_solver *s);

/* Macroscopic fields of the latest step (rho, u, T; host arrays of
   n_nodes doubles each, any may be NULL) and the current time. */
alelb_status alelb_moments(alelb_solver *s, double *rho, double *ux, double *uy, double *T);
alelb_status alelb_time(alelb_solver *s, double *t, int64_t *step);

/* Post-collision populations (full values, FP64), [9][n_nodes] each, host,
   in the caller's node order.  Each array is one device-to-host copy (the
   renumbering runs on the device); page-locked arrays are written by DMA.
   The f copy goes through a second stream the library owns, overlapping
   the device-side work of g; every kernel stays on the solver's stream.
   Synchronous. */
alelb_status alelb_get_pops(alelb_solver *s, double *f, double *g);
/* Sets the post-collision populations and the latest-step fields (used as
   the previous-step quantities of the wall condition) and the time t.
   Any field pointer may be NULL: then the field is recomputed from f, g.
   Each array is one host-to-device copy (g and the fields through a
   second stream the library owns, so that the device-side work of f
   overlaps them); returns when they may be reused. */
alelb_status alelb_set_pops(alelb_solver *s, const double *f, const double *g,
                            const double *rho, const double *ux, const double *uy,
                            const double *T, double t);

/* The same exchange in the stored form of ALELB_PREC_FP32_DEV (the paper
   has no counterpart): f, g are host arrays of [9][n_nodes] FP32 in the
   caller's node order, holding the deviations f_i - f_i^eq(rho_inf, 0,
   T_inf) and g_i - g_i^eq(rho_inf, 0, T_inf) (the equilibria at the free
   stream's density and temperature at rest, on the solver's lattice
   c_i + U) exactly as the solver stores them: half the bytes of the FP64
   exchange, and no rounding either way (a get, then a set, restores the
   state bit for bit).  set: the deviations become the post-collision
   state and the time becomes t; the fields are computed from the full
   populations d + f^eq in FP64, as alelb_set_pops without fields computes
   them.  Both synchronous (set returns once the arrays may be reused);
   ALELB_ERR_ARG for a NULL array or a solver of another precision. */
alelb_status alelb_get_pops_stored(alelb_solver *s, float *f, float *g);
alelb_status alelb_set_pops_stored(alelb_solver *s, const float *f, const float *g, double t);

/* Zero-copy forms of alelb_get_pops, alelb_set_pops (without fields) and
   alelb_moments (the paper has no counterpart): the arrays are DEVICE
   memory of the mesh's device (for example CUDA tensors), the same layouts
   and values as the host forms, in the caller's node order, and nothing
   crosses the host link.  The caller's arrays must hold their data (set)
   or be free to write (get, moments) when the call is made: the calls run
   on the solver's stream and wait for it before returning.  Any moments
   pointer may be NULL.  ALELB_ERR_ARG for a NULL population array or for
   an address that is not device (or managed) memory of the mesh's device;
   errors as the host forms otherwise. */
alelb_status alelb_get_pops_dev(alelb_solver *s, double *f, double *g);
alelb_status alelb_set_pops_dev(alelb_solver *s, const double *f, const double *g, double t);
alelb_status alelb_moments_dev(alelb_solver *s, double *rho, double *ux, double *uy, double *T);

/* Wall forces at the current time: {Fx_p, Fy_p, Fx_v, Fy_v, c_D, c_L} with
   p = rho T, tau = mu (S - (1/Cv) div u I), Simpson's rule per straight
   wall edge of the mapped geometry, c = F / (rho_inf |u_inf|^2 chord / 2)
   along u_inf (drag) and +90 degrees (lift) (Sec. V.B).  FP64, fixed
   summation order; synchronous. */
alelb_status alelb_forces(alelb_solver *s, double out[6]);

/* Element choice of every population for a propagation at map time t,
   [9][n_nodes] in original numbering: elem = original element id, -2 (the
   departure point is the node itself) or -1 (missing; kind = 1 wall,
   2 far field).  use_cache = 0: the element walk decides every population;
   use_cache = 1 (deviation-form solvers): the decision the propagation
   kernel would take now -- the previous-step element where the certified
   FP32 test accepts it, the walk elsewhere.  Synchronous; changes nothing. */
alelb_status alelb_locate(alelb_solver *s, double t, int32_t use_cache, int32_t *elem, int8_t *kind);

/* Per-kernel device time accumulated with CUDA events on the solver's
   stream since the last reset: names[k] (static strings), ms[k], launches[k]
   for k < *n (in: capacity, out: count).  enable != 0 starts timing (adds
   two events per launch); enable == 0 stops it. */
alelb_status alelb_profile(alelb_solver *s, int32_t enable);
alelb_status alelb_kernel_times(alelb_solver *s, const char **names, double *ms,
                                int64_t *launches, int32_t *n);

/* Sizes and counters: out = {n_nodes, n_elems, bytes per stored population
   value, 0, n_wall_nodes, precision, n_wall_edges, element walks run by the
   propagation kernel since lb_init (populations not settled by the verified
   previous-step element)}.  Synchronous. */
alelb_status alelb_info(alelb_solver *s, double out[8]);

/* One FP64 time step t -> t + 1 that allocates nothing (the paper has no
   counterpart: this entry point exists for callers that cannot allocate
   device memory once running -- an application whose device memory is
   pre-reserved by its own allocator, or a loop that must not call
   cudaMalloc/cudaFree, which can wait for the whole device).
   The current device must be the one that was current at
   alelb_mesh_create (else ALELB_ERR_ARG).
   The caller owns and passes the state, all device pointers on the current
   device: post [9][n_nodes] f then [9][n_nodes] g (full FP64 post-collision
   populations at t, overwritten with those at t + 1) and the latest-step
   fields rho, ux, uy, T [n_nodes] each (read by the wall condition,
   overwritten).  The mesh must have been created with ALELB_RENUMBER_NONE
   (node order = caller order) and have at most 131072 nodes;
   p->precision must be ALELB_PREC_FP64; the kernels run on p->stream
   (NULL: the default stream).  The step's
   scratch lives in a static device array of 23 * 131072 + 64 doubles
   (about 24 MB) that every GPU loading the library holds until exit.  The
   first call on a device, and the first call after each alelb_mesh_create
   on that device (a device reset frees every mesh, so this also follows a
   reset), looks up that array's device address: make that call before any
   stream capture.  Calls share the array, so calls
   that overlap on the GPU race.  Synchronous; returns ALELB_ERR_ARG for a
   larger mesh or other precision (message in alelb_mesh_last_error). */
alelb_status alelb_lb_step_noalloc(alelb_mesh *mesh, const alelb_params *p, double t,
                                   double *post, double *rho, double *ux, double *uy, double *T);

/* Checkpoints (the paper has no counterpart: it describes no restart).
   alelb_save writes the solver's state to the file `path`: the stored
   post-collision populations, the latest-step fields (the wall condition's
   previous-step values), the deviation forms' element cache, the time, the
   step count and the walk counters, with the fluid parameters, the mesh's
   fingerprint and FNV-1a checksums of header and data.  It first waits for
   the solver's stream (returning any sticky device error instead of
   saving), writes `path`.tmp and renames it to `path`.  alelb_load reads
   such a file into a solver created with alelb_lb_init on the same mesh
   (same node coordinates, connectivity, edge kinds and motion), precision,
   lattice shift, gamma and free stream; the viscosity, Prandtl number,
   chord and flags may differ and take effect from the next step.  After a
   load, stepping continues exactly as the saved solver would have: the
   results are bit-identical to an uninterrupted run.  Both are
   synchronous.  Errors: ALELB_ERR_ARG for a path that cannot be opened or
   written and for a file that is not a complete, intact checkpoint
   (truncated, bad magic or version, checksum mismatch, trailing bytes);
   ALELB_ERR_STATE for an intact checkpoint of a different mesh, precision,
   shift or free stream (the solver is then unchanged); ALELB_ERR_CUDA. */
alelb_status alelb_save(alelb_solver *s, const char *path);
alelb_status alelb_load(alelb_solver *s, const char *path);
/* Checks a checkpoint file on the host alone (no device is touched) with
   the tests alelb_load applies to the file itself.  out (may be NULL):
   {precision, n_nodes, n_elems, step count}; t (may be NULL): its time;
   msg (may be NULL): the reason of a failure, at most msg_len bytes with
   the terminating zero.  Errors as alelb_load's file errors. */
alelb_status alelb_checkpoint_info(const char *path, int64_t out[4], double *t, char *msg, int32_t msg_len);

/* Batched step (the paper runs one case at a time and has no counterpart;
   this serves parameter sweeps of many independent cases).  A batch groups
   B = 1..32 distinct solvers of one precision, each on its own mesh, and
   advances all of them together.  Each phase of the step (Eq. Propagation,
   Sec. IV.A, moments, the two derivative passes of Eq. Xa, collision) is one
   launch over all cases: its thread blocks are numbered through a prefix sum
   of the cases' node-tile counts, so block b works on the case whose tile
   range holds b; the exact part of the propagation walks every case's work
   list.  Chunks of up to 64 steps are captured once into a CUDA graph and
   replayed.  Per case the result is that of alelb_lb_step on that solver
   alone: the same per-node code with the same per-step map scalars, so the
   same element choices, with values equal up to rounding (the compiler may
   fuse multiply-adds of the shared code in another order in the batched
   kernels).
   The solvers must outlive the batch and must not be destroyed while it
   exists; between batch calls they stay usable one by one (alelb_moments,
   alelb_forces, alelb_get_pops, alelb_set_pops, alelb_lb_step): a batch
   step waits for earlier work on every case's stream, and every case's
   stream waits for the batch's last step. */
typedef struct alelb_batch alelb_batch;

/* cases: host array of B solver handles, read during the call.  stream: the
   cudaStream_t of the batch's launches (NULL: the batch's own non-blocking
   stream).  Errors: ALELB_ERR_ARG (B out of 1..32, a null or repeated
   solver, mixed precision, a 16-bit form), ALELB_ERR_OOM, ALELB_ERR_CUDA. */
alelb_status alelb_batch_create(alelb_solver *const *cases, int32_t B, void *stream, alelb_batch **out);
void alelb_batch_destroy(alelb_batch *b);

/* Advances every case by n >= 0 steps; asynchronous on the batch's stream. */
alelb_status alelb_batch_step(alelb_batch *b, int32_t n);

/* Waits for the batch's stream and reports the first case with a sticky
   device error (alelb_batch_last_error names the case). */
alelb_status alelb_batch_sync(alelb_batch *b);

/* Autotuner: runs ONE real step (every case advances by 1) in which each
   phase kernel is launched `reps` (1..16) times with every candidate launch
   shape and timed with CUDA events; the fastest shape per kernel is kept
   for later steps.  Candidates: 64, 128 or 256 threads per block (one
   node tile per block); for the propagation's fast part also 1, 3 or 9
   directions per thread, and in the FP32 form 3 or 9 fused with the
   moments; for
   the two derivative passes of the FP32 form
   also the staging of each tile's neighbour stencil in shared memory (the
   two fields over the tile's node range widened by 256 on each side); for
   the exact part of the propagation also 1, 2, 4, 8 or 16 blocks per SM.
   Then, for the FP32 form in graph mode, the propagation's form is
   refined on whole steps: the forms with 3 and 9 directions per thread,
   plain and fused with the moments, at 128 and 256 threads, and the
   per-kernel pick each run 8 steps twice from a saved copy of every case's
   state, the second run timed; the fastest is kept and the state put back
   (the cases advance by the one real step only; a device copy of each
   case's populations, fields and element cache is held meanwhile).  The
   case groups are then refined the same way: all cases as one group, or
   two or four groups of balanced node counts (cases dealt largest
   first), each with its own stream in graph mode, captured as branches of
   every chunk's graph and running side by side, so that one group's
   kernels fill the SMs that another group's leave idle (its propagation,
   bound by load latency, beside another's collision, bound by memory
   bandwidth; one kernel's tail beside another's start); free, or with
   each group's propagation (+ 4096: its first kernel; + 8192: its exact
   part too) ordered after the previous group's latest one.  The step's values do not depend on the
   shapes, and every phase kernel gives the same values when repeated
   within a step, so tuning changes no result.  choice (may be NULL, else 8
   values out): block size of {k_stream, k_stream_fast, k_stream_slow,
   k_moments, k_deriv1, k_collide}, grid of k_stream_slow, then directions
   per thread of k_stream_fast + 16 (k_deriv1 staged) + 32 (k_collide
   staged) + 256 (k_stream_fast fused with the moments: the
   moments of the nodes whose populations all settle there are computed
   in the same launch, and k_moments takes only the others) + 512 or 1024
   (two or four case groups) + 4096 or 8192 (propagations in turn).
   Groups apply in graph mode; the persistent form and profiled steps run
   all cases as one.
   Synchronous. */
alelb_status alelb_batch_tune(alelb_batch *b, int32_t reps, int32_t choice[8]);

/* The host exchange of alelb_get_pops / alelb_set_pops for every case of
   the batch in one call (the paper has no counterpart).  f[c], g[c]: host
   arrays of case c, [9][n_nodes of case c] FP64 each, the caller's node
   order (pinned memory lets the copies run at the link's rate).  Every
   case's copies and kernels are queued before the call waits on any of
   them, so the cases' copies overlap one another and the other cases'
   kernels.  set: the populations become the cases' post-collision state,
   with the fields they imply (as alelb_set_pops without fields), and, when
   t is not NULL, case c's time becomes t[c].  Both return once the caller's
   arrays may be reused; ALELB_ERR_ARG for a NULL array; get reports a
   case's sticky error (and names the case) like alelb_batch_sync. */
alelb_status alelb_batch_set_pops(alelb_batch *b, const double *const *f, const double *const *g,
                                  const double *t);
alelb_status alelb_batch_get_pops(alelb_batch *b, double *const *f, double *const *g);
/* The batched forms of alelb_get_pops_stored / alelb_set_pops_stored (FP32
   planes of each case's stored deviations; ALELB_ERR_ARG also for a batch
   of another precision). */
alelb_status alelb_batch_set_pops_stored(alelb_batch *b, const float *const *f, const float *const *g,
                                        const double *t);
alelb_status alelb_batch_get_pops_stored(alelb_batch *b, float *const *f, float *const *g);
/* One step of every case with its state in host memory, in the stored form
   of ALELB_PREC_FP32_DEV (the paper has no counterpart): the same values as
   alelb_batch_set_pops_stored(f_in, g_in, t), alelb_batch_step(b, 1) and
   alelb_batch_get_pops_stored(f_out, g_out), bit for bit, but pipelined by
   case group: each group steps as soon as its own cases are uploaded, and
   its cases are read back while later groups still upload, so that the
   host link carries both directions at once.  f_out[c] may be f_in[c]
   (likewise g).  The step's kernels are launched directly on the groups'
   streams (not from the captured graphs, not profiled) with the batch's
   launch shapes.  t (may be NULL): the cases' times before the step; each
   case advances by one step.  Synchronous; errors as
   alelb_batch_get_pops_stored. */
alelb_status alelb_batch_step_host(alelb_batch *b, const float *const *f_in, const float *const *g_in,
                                   float *const *f_out, float *const *g_out, const double *t);

/* Sets the launch shapes that alelb_batch_tune would choose, in its
   encoding (for example a choice saved from an earlier tuning):
   block sizes 64, 128 or 256; a k_stream_slow grid of 1 .. 64 x the SM
   count; directions per thread 1, 3 or 9, optionally + 256 (fused with
   the moments; 3 or 9 only); + 16, + 32 (staging), which need the FP32
   form; + 512 (two case groups) or + 1024 (four; only when every group
   receives a case), optionally + 4096 or + 8192 (their propagations in
   turn), in either form.  Changes no result; ALELB_ERR_ARG for a value
   outside these. */
alelb_status alelb_batch_set_choice(alelb_batch *b, const int32_t choice[8]);

/* How a batch runs its steps.  ALELB_BATCH_GRAPHS (the default): one
   launch per phase over all cases, chunks of up to 64 steps captured once
   into CUDA graphs and replayed.  ALELB_BATCH_PERSISTENT: one cooperative
   launch per chunk of up to 64 steps, every block resident, a grid-wide
   barrier between phases; each wait at a barrier gives up after the limit
   of alelb_batch_set_wait (1 s by default), sets ALELB_ERR_TIMEOUT on every
   case and returns, so a wait cannot hang the device.  Both give every
   case the result of alelb_lb_step on that solver alone (the same per-node
   code, values equal up to the compiler's multiply-add fusion).  While
   profiling is on, steps are launched one kernel at a time in either mode.
   Waits for the batch's stream; ALELB_ERR_ARG for another mode. */
enum { ALELB_BATCH_GRAPHS = 0, ALELB_BATCH_PERSISTENT = 1 };
alelb_status alelb_batch_set_mode(alelb_batch *b, int32_t mode);
/* Limit of each grid-wide wait of the persistent form, in seconds
   (0 < limit <= 60).  missing_arrivals (0 or 1) makes every barrier wait
   for that many blocks more than the grid holds, so that every wait runs
   out: a test of the time-out path, which leaves the cases' state
   mid-step and ALELB_ERR_TIMEOUT sticky on them.  Waits for the batch's
   stream. */
alelb_status alelb_batch_set_wait(alelb_batch *b, double limit_seconds, int32_t missing_arrivals);

/* Per-kernel device times of the batch, as alelb_profile and
   alelb_kernel_times for a solver.  While enabled, steps are launched one
   kernel at a time (not through the graph) between two events each. */
alelb_status alelb_batch_profile(alelb_batch *b, int32_t enable);
alelb_status alelb_batch_kernel_times(alelb_batch *b, const char **names, double *ms,
                                      int64_t *launches, int32_t *n);

/* Learned departure-element proposal (the paper has no counterpart: it
   locates every departure point by search, Sec. III).  A small network
   (6 features -> 64 tanh -> 64 tanh -> 32 slot logits + 3 barycentric
   guesses, 6883 parameters, flat order W1[64][6], b1[64], W2[64][64],
   b2[64], W3[35][64], b3[35]) proposes, for a population left to the exact
   path of the FP32-deviation propagation, an element of the node's
   neighbour ring (its own elements by angle, then the elements across
   their edges by angle, at most 32).  A proposal is used only when the
   certified FP32 test that accepts previous-step elements accepts it
   (departure point strictly inside; the segment from the node cannot
   leave the mesh); the exact walk decides otherwise.  Streamed values are
   bit-identical with and without the network.
   Features of query (node a, direction i), FP32: d = -c^_i / h with h the
   square root of the mean area of a's elements: d_x, d_y, |d|,
   atan2(d_y, d_x) / pi, (number of a's elements) / 16, (ring size) / 32. */
typedef struct alelb_mlp alelb_mlp;

/* params: host array of 6883 FP32 values, or NULL for Glorot-uniform
   weights and zero biases drawn from seed (splitmix64). */
alelb_status alelb_mlp_create(const float *params, uint64_t seed, alelb_mlp **out);
void alelb_mlp_destroy(alelb_mlp *m);
/* The FP32 master parameters (rounded = 0) or the FP16 copies the network
   runs with, widened to FP32 (rounded != 0); host array of 6883. */
alelb_status alelb_mlp_get_params(alelb_mlp *m, int32_t rounded, float *params);

/* Training data from a solver's mesh and map: for every query at map time
   t (internal node order, laid out [direction][node]), with no change to
   the solver's state: its
   features feat[q][6], the slot of the exact element (FP64 departure point,
   exact walk) in the node's ring or -1 (departure on the node itself, a
   node, outside the mesh, an element outside the ring, or no certified
   FP32 map), the barycentric coordinates there bary[q][3] and the ring size
   nring[q].  DEVICE arrays of 9 * n_nodes entries, caller-owned.
   Synchronous. */
alelb_status alelb_samples(alelb_solver *s, double t, float *feat, int16_t *slot, float *bary,
                           uint8_t *nring);

/* Mean loss over n (1..2^31-1) samples -- cross-entropy of the softmax of
   the first nring logits at slot, plus w_bary times the mean squared error
   of the 3 guesses -- and its gradient (host, 6883 FP32, may be NULL),
   computed with the FP16 weights in FP32 arithmetic.  Every slot must lie
   in 0..nring-1.  DEVICE inputs.  Synchronous. */
alelb_status alelb_mlp_loss_grad(alelb_mlp *m, const float *feat, const int16_t *slot,
                                 const float *bary, const uint8_t *nring, int64_t n,
                                 float w_bary, double *loss, float *grad);
/* Adam (beta 0.9, 0.999, eps 1e-8) on that loss over `epochs` passes of
   the n samples in minibatches of `batch`, the order of each pass a seeded
   affine permutation of the samples; FP32 master weights, FP16 copies for
   the forward pass.  epoch_loss (host, may be NULL): mean loss of each
   pass.  DEVICE inputs.  Synchronous. */
alelb_status alelb_mlp_train(alelb_mlp *m, const float *feat, const int16_t *slot,
                             const float *bary, const uint8_t *nring, int64_t n, int32_t epochs,
                             int32_t batch, float lr, float w_bary, uint64_t seed,
                             double *epoch_loss);
/* Inference as the propagation runs it (FP16 tensor-core MMA, FP32
   accumulation): slot[q] = largest of the first nring logits (-1 when
   nring = 0); out[q][35] all outputs (may be NULL).  DEVICE arrays.
   Synchronous. */
alelb_status alelb_mlp_predict(alelb_mlp *m, const float *feat, const uint8_t *nring, int64_t n,
                               int32_t *slot, float *out);

/* Use network m (NULL: none) for the proposals of a deviation-form
   solver's later steps.  The network is not copied and must outlive its
   use; ALELB_ERR_ARG for an FP64 solver. */
alelb_status alelb_solver_set_mlp(alelb_solver *s, alelb_mlp *m);
/* Counters since lb_init: {populations left to the exact path, proposals
   made, proposals accepted}.  Synchronous. */
alelb_status alelb_mlp_stats(alelb_solver *s, int64_t out[3]);

const char *alelb_last_error(alelb_solver *s);
const char *alelb_mesh_last_error(alelb_mesh *m);
const char *alelb_batch_last_error(alelb_batch *b);
const char *alelb_mlp_last_error(alelb_mlp *m);

#ifdef __cplusplus
}
#endif
#endif /* ALELB_H */
