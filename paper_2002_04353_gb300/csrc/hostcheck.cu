// hostcheck.cu -- the device element walk compiled for the host, for CPU
// tests of the walk against the oracle (test tooling; not on the product
// path).  Builds the same tables as alelb_mesh_create and runs the same
// per-node location routine that k_locate runs.
#include <cstring>
#include <string>

#include "tables.h"

using namespace alelb;

extern "C" int alelb_hostcheck_locate(const alelb_mesh_desc *d, double t, int literal,
                                      int32_t *elem, int8_t *kind, char *errbuf, int errlen)
{
    HostTables T;
    std::string err;
    alelb_status st = build_tables(d, T, err);
    if (st != ALELB_OK) {
        if (errbuf && errlen > 0) std::strncpy(errbuf, err.c_str(), errlen - 1);
        return st;
    }
    MeshDev M = T.host_view();
    MapStatic MS = T.host_map();
    MapScalars sc = map_scalars(T.mkind, T.mp, t);
    int e = 0;
    const int N = T.N;
    for (int a = 0; a < N; ++a) {
        int e9[NQ];
        int8_t k9[NQ];
        locate_node(M, MS, sc, literal, a, e9, k9, &e);
        int o = T.node_new2old[a];
        for (int i = 0; i < NQ; ++i) {
            elem[(size_t)i * N + o] = e9[i];
            kind[(size_t)i * N + o] = k9[i];
        }
    }
    return e ? ALELB_ERR_LOCATE : ALELB_OK;
}

// The certified FP32 strict-containment filter of the fast propagation path,
// on the host: out[k] = 1 when the filter accepts point k in element elem[k]
// (internal numbering of the Morton-renumbered mesh; frame shift 0).
extern "C" int alelb_hostcheck_inside(const alelb_mesh_desc *d, int n, const int32_t *elem_orig,
                                      const double *px, const double *py, int8_t *out)
{
    HostTables T;
    std::string err;
    alelb_status st = build_tables(d, T, err);
    if (st != ALELB_OK) return st;
    MeshDev M = T.host_view();
    for (int k = 0; k < n; ++k) {
        float qx, qy;
        int e = T.elem_old2new[elem_orig[k]];
        out[k] = strictly_inside_f32(M, e, 0, 0, px[k], py[k], qx, qy) ? 1 : 0;
    }
    return ALELB_OK;
}
