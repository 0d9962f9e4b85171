// internal.h -- host-side objects shared by the translation units of the
// library (single-case solver in alelb.cu, batched step in batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "alelb.h"
#include "kernels.cuh"
#include "quad_tables.h"
#include "tables.h"

namespace alelb {

// Device allocations released together.
struct DevBuf {
    std::vector<void *> ptrs;
    template <class T> T *put(const std::vector<T> &h, cudaError_t &st)
    {
        if (h.empty()) return nullptr;
        void *p = nullptr;
        if (st == cudaSuccess) st = cudaMalloc(&p, h.size() * sizeof(T));
        if (st == cudaSuccess) {
            ptrs.push_back(p);
            st = cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
        }
        return (T *)p;
    }
    template <class T> T *alloc(size_t n, cudaError_t &st)
    {
        void *p = nullptr;
        if (st == cudaSuccess) st = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
        if (st == cudaSuccess) ptrs.push_back(p);
        return (T *)p;
    }
    void release()
    {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

enum { KT_STREAM = 0, KT_FAST = 1, KT_SLOW = 2, KT_MOMENTS = 3, KT_DERIV1 = 4, KT_COLLIDE = 5, KT_PROPOSE = 6,
       KT_N = 7 };
extern const char *const KT_NAMES[KT_N];

// A kernel of the step, launched with programmatic stream serialization:
// its blocks may start while the previous kernel drains (each waits in
// wait_prior_grid before touching memory).
template <class... KArgs, class... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t stream, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// FP32 copies of the per-step map scalars.
MapScalarsF to_f32(const MapScalars &S, const HostTables &T);
// the host exchange's copies and kernels for one solver, queued on its
// streams without waiting (alelb_set_pops / alelb_get_pops and their
// batched forms wait afterwards)
cudaError_t import_enqueue(alelb_solver *s, const double *f, const double *g, const double *rho,
                           const double *ux, const double *uy, const double *T);
cudaError_t export_enqueue(alelb_solver *s, double *f, double *g, double *const fld[4]);
// the same for the FP32-deviation form's stored deviations (FP32 planes)
cudaError_t import_stored_enqueue(alelb_solver *s, const float *f, const float *g);
cudaError_t export_stored_enqueue(alelb_solver *s, float *f, float *g);
// Uploads the P2 derivative tables of batch.cu's module.
cudaError_t batch_fe_tables();
// Status of a solver's sticky device errors (message in s->err).
alelb_status check_sticky(alelb_solver *s);
// Learned proposals for the solver's current work list (mlp.cu).
cudaError_t mlp_propose(alelb_solver *s, const MapScalarsF &sf);
// 9-node quadrilateral meshes (quad.cu): upload of the tables built by
// build_quad_tables; one kernel of a step (KT_STREAM, KT_DERIV1 or
// KT_COLLIDE) on the solver's stream; the element-choice report; the wall
// forces into s->d_out.
alelb_status quad_mesh_upload(alelb_mesh *m);
cudaError_t quad_launch(alelb_solver *s, int kernel, const MapScalars &sc, const MapScalars &scd);
cudaError_t quad_locate(alelb_solver *s, const MapScalars &sc, int *elem, int8_t *kind);
cudaError_t quad_forces(alelb_solver *s, const MapScalars &sc);


} // namespace alelb

// The C-ABI's opaque objects (global names, as declared in alelb.h).
using namespace alelb;

struct alelb_mesh {
    std::string err;
    int etype = ALELB_ELEM_P2TRI; // element kind (alelb_mesh_desc.elem_type)
    HostTables T;   // host copies of every table (also used by the host-side walk check);
                    // for quadrilaterals only the generic fields (sizes, node order,
                    // coordinates, map factors, wall edges)
    QuadTables QT;  // quadrilateral meshes: their element tables
    QuadDev qdev{}; // quadrilateral meshes: the device tables
    MeshDev dev{};
    MapStatic mst{};
    int2 *d_wedges = nullptr;
    int *d_n2o = nullptr; // [N] caller's node number of each internal node
    int nw = 0;
    int device = 0; // the CUDA device current at alelb_mesh_create, which holds the tables
    uint64_t fingerprint = 0; // FNV-1a of the node coordinates, connectivity, edge kinds,
                              // periods and motion (checkpoints name the mesh by it)
    DevBuf buf;
};

struct alelb_solver {
    alelb_mesh *mesh = nullptr;
    std::string err;
    int prec = 0, flags = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;        // host exchange copies (set_pops, get_pops)
    cudaEvent_t ev_copy[2] = {nullptr, nullptr}; // orders them against the solver's stream
    double gamma = 1.4, Pr = 0.71, mu = 0, rho_inf = 1, T_inf = 0.3, uinf[2] = {0, 0}, chord = 1;
    double Cv = 2.5, Cp = 3.5;
    double U[2] = {0, 0}; // lattice shift: velocities c_i + U
    double t = 0;
    int64_t nstep = 0;
    StateDev<double> sd{};  // ALELB_PREC_FP64
    StateDev<float> sf{};   // ALELB_PREC_FP32_DEV
    StateDev<Bf16Dev> sb{}; // ALELB_PREC_BF16_DEV
    StateDev<Fp16Dev> sh{}; // ALELB_PREC_FP16_DEV
    KinParams<double> kd{};
    KinParams<float> kf{};
    double consts[4 * NQ] = {0};
    double *d_consts = nullptr;
    double *d_scratch = nullptr; // 22 N doubles: import/export staging (caller's node order)
    int *d_err = nullptr;
    unsigned long long *d_stats = nullptr; // [0]: element walks run by the propagation kernel
    double *d_out = nullptr;
    DevBuf buf;
    int sticky = 0;
    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { int k; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    double ms_acc[KT_N] = {};
    int64_t n_acc[KT_N] = {};
    int n_sm = 152;
    alelb_mlp *mlp = nullptr; // learned proposal (not owned), deviation-form solvers
    int *d_prop = nullptr;    // [9 N] proposal per work-list entry
};

namespace alelb {
// The internal flag bit of a shifted lattice.
inline int shift_flag(const double U[2]) { return (U[0] != 0.0 || U[1] != 0.0) ? FLAG_SHIFT : 0; }
// Map scalars carrying the lattice shift U.
inline MapScalars with_shift(MapScalars S, const double U[2])
{
    S.Ux = U[0];
    S.Uy = U[1];
    return S;
}
inline MapScalars solver_map(const alelb_solver *s, const MapScalars &S) { return with_shift(S, s->U); }

// Calls fn(state, kinetic parameters) with the solver's state of its
// precision (the deviation forms share the FP32 kinetic parameters).
template <class Fn> auto with_state(alelb_solver *s, Fn &&fn)
{
    switch (s->prec) {
    case ALELB_PREC_FP64: return fn(s->sd, s->kd);
    case ALELB_PREC_FP32_DEV: return fn(s->sf, s->kf);
    case ALELB_PREC_BF16_DEV: return fn(s->sb, s->kf);
    default: return fn(s->sh, s->kf);
    }
}
} // namespace alelb
