// checkpoint.cu -- alelb_save / alelb_load / alelb_checkpoint_info: a
// solver's state written to a file and read back bit for bit.
//
// The state that a step reads is the post-collision population buffer, the
// latest-step fields (the wall condition's previous-step values), the
// element cache of the deviation forms (the propagation kernel's
// previous-step elements, which decide whether a population takes the fast
// or the exact path and so the last bits of its value), the time and step
// count.  Everything else a step touches (streamed populations, Q', D, the
// exact-path work list) is rebuilt inside the step, and the work list is
// empty between steps.
//
// File layout (little-endian, the byte order of every supported host):
// a 192-byte header (struct CkHeader below), then the payload: populations
// as stored (18 N values of the solver's storage type), the fields rho, ux,
// uy, T (N values each, storage type), the element cache (9 N int32,
// deviation forms only) and the four 64-bit counters.  The header carries
// FNV-1a 64-bit checksums of itself and of the payload.
#include <cuda_runtime.h>

#include <cerrno>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace {

constexpr char CK_MAGIC[8] = {'A', 'L', 'E', 'L', 'B', 'C', 'K', '1'};
constexpr uint32_t CK_VERSION = 1;

struct CkHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int32_t precision, flags, n_nodes, n_elems;
    uint64_t mesh_fingerprint;
    double t;
    int64_t nstep;
    double gamma, Pr, mu, rho_inf, T_inf, u_inf[2], chord, shift[2];
    uint64_t pop_bytes, fld_bytes, cache_bytes, stats_bytes;
    uint64_t payload_bytes;
    uint64_t payload_fnv;
    uint64_t header_fnv; // of every byte of the header before this field
};
static_assert(sizeof(CkHeader) == 192, "checkpoint header layout");

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char *b = (const unsigned char *)p;
    for (size_t k = 0; k < n; ++k) {
        h ^= b[k];
        h *= 1099511628211ull;
    }
    return h;
}

// Section sizes of a solver's payload.
struct CkSizes {
    uint64_t pop, fld, cache, stats;
    uint64_t total() const { return pop + 4 * fld + cache + stats; }
};

CkSizes sizes_of(int prec, int N)
{
    const uint64_t ps = prec == ALELB_PREC_FP64 ? 8 : prec == ALELB_PREC_FP32_DEV ? 4 : 2;
    const uint64_t fs = prec == ALELB_PREC_FP64 ? 8 : 4;
    CkSizes z;
    z.pop = 18ull * N * ps;
    z.fld = (uint64_t)N * fs;
    z.cache = prec == ALELB_PREC_FP64 ? 0 : 9ull * N * sizeof(int);
    z.stats = 4 * sizeof(unsigned long long);
    return z;
}

// Reads and checks a checkpoint file: header fields, sizes, both checksums.
alelb_status ck_read(const char *path, CkHeader &h, std::vector<unsigned char> &payload, std::string &err)
{
    if (!path) {
        err = "checkpoint: null path";
        return ALELB_ERR_ARG;
    }
    FILE *fp = std::fopen(path, "rb");
    if (!fp) {
        err = std::string("checkpoint: cannot open ") + path + ": " + std::strerror(errno);
        return ALELB_ERR_ARG;
    }
    const size_t nh = std::fread(&h, 1, sizeof(h), fp);
    if (nh != sizeof(h)) {
        std::fclose(fp);
        err = "checkpoint: file ends inside the header (" + std::to_string(nh) + " of " +
              std::to_string(sizeof(h)) + " bytes)";
        return ALELB_ERR_ARG;
    }
    if (std::memcmp(h.magic, CK_MAGIC, sizeof(CK_MAGIC)) != 0) {
        std::fclose(fp);
        err = "checkpoint: not a checkpoint file (bad magic)";
        return ALELB_ERR_ARG;
    }
    if (h.version != CK_VERSION || h.header_bytes != sizeof(CkHeader)) {
        std::fclose(fp);
        err = "checkpoint: unsupported version " + std::to_string(h.version);
        return ALELB_ERR_ARG;
    }
    if (fnv1a(&h, offsetof(CkHeader, header_fnv)) != h.header_fnv) {
        std::fclose(fp);
        err = "checkpoint: header checksum mismatch (corrupted header)";
        return ALELB_ERR_ARG;
    }
    if (h.precision < ALELB_PREC_FP64 || h.precision > ALELB_PREC_FP16_DEV || h.n_nodes <= 0 || h.n_elems <= 0) {
        std::fclose(fp);
        err = "checkpoint: invalid header values";
        return ALELB_ERR_ARG;
    }
    const CkSizes z = sizes_of(h.precision, h.n_nodes);
    if (h.pop_bytes != z.pop || h.fld_bytes != z.fld || h.cache_bytes != z.cache || h.stats_bytes != z.stats ||
        h.payload_bytes != z.total()) {
        std::fclose(fp);
        err = "checkpoint: section sizes do not match the header's precision and node count";
        return ALELB_ERR_ARG;
    }
    payload.resize(h.payload_bytes);
    const size_t np = std::fread(payload.data(), 1, payload.size(), fp);
    const bool extra = np == payload.size() && std::fgetc(fp) != EOF;
    std::fclose(fp);
    if (np != payload.size()) {
        err = "checkpoint: file ends inside the payload (" + std::to_string(np) + " of " +
              std::to_string(payload.size()) + " bytes)";
        return ALELB_ERR_ARG;
    }
    if (extra) {
        err = "checkpoint: trailing bytes after the payload";
        return ALELB_ERR_ARG;
    }
    if (fnv1a(payload.data(), payload.size()) != h.payload_fnv) {
        err = "checkpoint: payload checksum mismatch (corrupted data)";
        return ALELB_ERR_ARG;
    }
    return ALELB_OK;
}

alelb_status cuda_err(alelb_solver *s, cudaError_t st)
{
    s->err = std::string("checkpoint: ") + cudaGetErrorString(st);
    return st == cudaErrorMemoryAllocation ? ALELB_ERR_OOM : ALELB_ERR_CUDA;
}

// Device sections of a solver's state, in payload order.
template <class S> void sections(alelb_solver *s, StateDev<S> &st, void *ptr[7])
{
    ptr[0] = st.post;
    ptr[1] = st.rho;
    ptr[2] = st.ux;
    ptr[3] = st.uy;
    ptr[4] = st.T;
    ptr[5] = st.cache;
    ptr[6] = s->d_stats;
}

} // namespace

extern "C" alelb_status alelb_save(alelb_solver *s, const char *path)
{
    if (!s || !path) return ALELB_ERR_ARG;
    if (!s->mesh) return ALELB_ERR_STATE;
    alelb_status r = alelb_sync(s); // the state of the last step, and no sticky error
    if (r != ALELB_OK) return r;
    const int N = s->mesh->T.N;
    const CkSizes z = sizes_of(s->prec, N);
    std::vector<unsigned char> payload(z.total());
    void *ptr[7];
    with_state(s, [&](auto &sx, auto &) { sections(s, sx, ptr); });
    const uint64_t len[7] = {z.pop, z.fld, z.fld, z.fld, z.fld, z.cache, z.stats};
    uint64_t off = 0;
    cudaError_t st = cudaSuccess;
    for (int k = 0; k < 7 && st == cudaSuccess; ++k) {
        if (len[k]) st = cudaMemcpyAsync(payload.data() + off, ptr[k], len[k], cudaMemcpyDeviceToHost, s->stream);
        off += len[k];
    }
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream);
    if (st != cudaSuccess) return cuda_err(s, st);
    CkHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, CK_MAGIC, sizeof(CK_MAGIC));
    h.version = CK_VERSION;
    h.header_bytes = sizeof(CkHeader);
    h.precision = s->prec;
    h.flags = s->flags;
    h.n_nodes = N;
    h.n_elems = s->mesh->T.E;
    h.mesh_fingerprint = s->mesh->fingerprint;
    h.t = s->t;
    h.nstep = s->nstep;
    h.gamma = s->gamma;
    h.Pr = s->Pr;
    h.mu = s->mu;
    h.rho_inf = s->rho_inf;
    h.T_inf = s->T_inf;
    h.u_inf[0] = s->uinf[0];
    h.u_inf[1] = s->uinf[1];
    h.chord = s->chord;
    h.shift[0] = s->U[0];
    h.shift[1] = s->U[1];
    h.pop_bytes = z.pop;
    h.fld_bytes = z.fld;
    h.cache_bytes = z.cache;
    h.stats_bytes = z.stats;
    h.payload_bytes = z.total();
    h.payload_fnv = fnv1a(payload.data(), payload.size());
    h.header_fnv = fnv1a(&h, offsetof(CkHeader, header_fnv));
    // written beside the target, then renamed: a reader never sees half a file
    const std::string tmp = std::string(path) + ".tmp";
    FILE *fp = std::fopen(tmp.c_str(), "wb");
    if (!fp) {
        s->err = "save: cannot create " + tmp + ": " + std::strerror(errno);
        return ALELB_ERR_ARG;
    }
    bool ok = std::fwrite(&h, 1, sizeof(h), fp) == sizeof(h) &&
              std::fwrite(payload.data(), 1, payload.size(), fp) == payload.size();
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        s->err = std::string("save: cannot write ") + path + ": " + std::strerror(errno);
        std::remove(tmp.c_str());
        return ALELB_ERR_ARG;
    }
    return ALELB_OK;
}

extern "C" alelb_status alelb_load(alelb_solver *s, const char *path)
{
    if (!s || !path) return ALELB_ERR_ARG;
    if (!s->mesh) return ALELB_ERR_STATE;
    CkHeader h;
    std::vector<unsigned char> payload;
    alelb_status r = ck_read(path, h, payload, s->err);
    if (r != ALELB_OK) return r;
    const alelb_mesh *m = s->mesh;
    std::string why;
    if (h.precision != s->prec) why = "precision";
    else if (h.n_nodes != m->T.N || h.n_elems != m->T.E || h.mesh_fingerprint != m->fingerprint) why = "mesh";
    else if (h.shift[0] != s->U[0] || h.shift[1] != s->U[1]) why = "lattice shift";
    else if (h.gamma != s->gamma || h.rho_inf != s->rho_inf || h.T_inf != s->T_inf || h.u_inf[0] != s->uinf[0] ||
             h.u_inf[1] != s->uinf[1])
        why = "free-stream state or gamma (the stored deviations are relative to it)";
    if (!why.empty()) {
        s->err = "load: the checkpoint's " + why + " differs from this solver's";
        return ALELB_ERR_STATE;
    }
    const CkSizes z = sizes_of(s->prec, m->T.N);
    void *ptr[7];
    with_state(s, [&](auto &sx, auto &) { sections(s, sx, ptr); });
    const uint64_t len[7] = {z.pop, z.fld, z.fld, z.fld, z.fld, z.cache, z.stats};
    // every earlier step of this solver has finished before its state is replaced
    cudaError_t st = cudaStreamSynchronize(s->stream);
    uint64_t off = 0;
    for (int k = 0; k < 7 && st == cudaSuccess; ++k) {
        if (len[k]) st = cudaMemcpyAsync(ptr[k], payload.data() + off, len[k], cudaMemcpyHostToDevice, s->stream);
        off += len[k];
    }
    // the exact-path work list is empty between steps
    with_state(s, [&](auto &sx, auto &) {
        if (st == cudaSuccess) st = cudaMemsetAsync(sx.wcount, 0, (SEG_PENDING + 1) * sizeof(unsigned), s->stream);
        if (st == cudaSuccess) st = cudaMemsetAsync(sx.wmask, 0, (size_t)m->T.N * sizeof(unsigned), s->stream);
    });
    if (st == cudaSuccess) st = cudaStreamSynchronize(s->stream); // the host buffer is released below
    if (st != cudaSuccess) return cuda_err(s, st);
    s->t = h.t;
    s->nstep = h.nstep;
    return ALELB_OK;
}

extern "C" alelb_status alelb_checkpoint_info(const char *path, int64_t out[4], double *t, char *msg,
                                              int32_t msg_len)
{
    CkHeader h;
    std::vector<unsigned char> payload;
    std::string err;
    alelb_status r = ck_read(path, h, payload, err);
    if (msg && msg_len > 0) {
        std::strncpy(msg, err.c_str(), (size_t)msg_len - 1);
        msg[msg_len - 1] = '\0';
    }
    if (r != ALELB_OK) return r;
    if (out) {
        out[0] = h.precision;
        out[1] = h.n_nodes;
        out[2] = h.n_elems;
        out[3] = h.nstep;
    }
    if (t) *t = h.t;
    return ALELB_OK;
}
