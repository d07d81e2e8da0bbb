// checkpoint.cu -- state snapshot and resume of a single-plume context (no counterpart in the
// paper, whose runs are single 300-day jobs; long runs on shared machines need to stop and
// continue).
//
// A snapshot is one host buffer: a fixed header (magic, format version, dim, n, mode bits, step,
// simulated time, time step and the context's parameters), then the payload -- positions
// xq [dim][n], concentrations C [n], the Cattaneo flux Q [n] (tau > 0) and the velocity field
// v [dim][n] (vmax > 0) -- and a CRC-32 of header and payload.  Restoring checks the magic, the
// size, the checksum and that the parameters match the context's before anything is copied to
// the device, so a truncated or corrupted file changes nothing.
//
// CRC-32 here is the IEEE 802.3 / zlib checksum: reflected polynomial 0xEDB88320, initial value
// and final XOR 0xFFFFFFFF, computed with a 256-entry table built from the polynomial.
#include <string.h>

#include <mutex>

#include "ade_internal.h"

namespace {

constexpr char kMagic[8] = {'A', 'D', 'E', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kVersion = 1u;

struct Header {
    char magic[8];
    uint32_t version;
    uint32_t dim;
    uint32_t n;
    uint32_t mode;          // bit 0: velocity field, bit 1: Cattaneo flux
    long long step;
    double t;
    double dt;
    ade_params p;
    uint64_t payload_bytes;
};

uint32_t g_crc_table[256];
std::once_flag g_crc_once;

void crc_init()
{
    for (uint32_t i = 0; i < 256; ++i) {
        uint32_t c = i;
        for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
        g_crc_table[i] = c;
    }
}

uint32_t crc32(const unsigned char *p, size_t len, uint32_t crc = 0u)
{
    std::call_once(g_crc_once, crc_init);
    crc = ~crc;
    for (size_t i = 0; i < len; ++i) crc = g_crc_table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return ~crc;
}

uint32_t mode_of(const ade_ctx *c) { return (c->field ? 1u : 0u) | (c->catt ? 2u : 0u); }

size_t payload_bytes(const ade_ctx *c)
{
    size_t b = (size_t)c->dim * c->n * 4 + (size_t)c->n * 4;
    if (c->catt) b += (size_t)c->n * 4;
    if (c->field) b += (size_t)c->dim * c->n * 4;
    return b;
}

size_t total_bytes(const ade_ctx *c) { return sizeof(Header) + payload_bytes(c) + sizeof(uint32_t); }

// The physical and numerical parameters a snapshot must share with the context it resumes.
bool same_problem(const ade_params &a, const ade_params &b)
{
    if (a.dim != b.dim || a.kernel != b.kernel) return false;
    for (int i = 0; i < 3; ++i)
        if (a.box[i] != b.box[i] || a.v[i] != b.v[i]) return false;
    return a.h == b.h && a.alpha_L == b.alpha_L && a.alpha_T == b.alpha_T && a.D_m == b.D_m &&
           a.mass == b.mass && a.rho == b.rho && a.gamma == b.gamma && a.vmax == b.vmax && a.tau == b.tau;
}

#define CK(call)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return ade::report_error(ADE_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" {

int ade_checkpoint_bytes(const ade_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return ade::report_error(ADE_ERR_ARG, "NULL argument");
    *bytes = total_bytes(c);
    return ADE_OK;
}

int ade_checkpoint_save(ade_ctx *c, void *host_buf, size_t bytes, void *stream)
{
    if (!c || !host_buf) return ade::report_error(ADE_ERR_ARG, "NULL argument");
    if (bytes < total_bytes(c)) return ade::report_error(ADE_ERR_CAPACITY, "checkpoint buffer too small");
    if (c->field && !c->field_set) return ade::report_error(ADE_ERR_STATE, "no velocity field set");
    if (c->catt && !c->flux_set) return ade::report_error(ADE_ERR_STATE, "no flux set");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *out = static_cast<unsigned char *>(host_buf);
    Header h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kMagic, sizeof(kMagic));
    h.version = kVersion;
    h.dim = (uint32_t)c->dim;
    h.n = (uint32_t)c->n;
    h.mode = mode_of(c);
    h.step = c->step;
    h.t = c->t;
    h.dt = c->dt;
    h.p = c->p;
    h.payload_bytes = payload_bytes(c);
    memcpy(out, &h, sizeof(h));
    unsigned char *q = out + sizeof(h);
    const size_t n = (size_t)c->n, dim = (size_t)c->dim;
    if (n > 0) {
        CK(cudaMemcpyAsync(q, c->xq, dim * n * 4, cudaMemcpyDeviceToHost, s));
        q += dim * n * 4;
        CK(cudaMemcpyAsync(q, c->C, n * 4, cudaMemcpyDeviceToHost, s));
        q += n * 4;
        if (c->catt) {
            CK(cudaMemcpyAsync(q, c->Q, n * 4, cudaMemcpyDeviceToHost, s));
            q += n * 4;
        }
        if (c->field) {
            // the velocities are the first dim lanes of the caller-order float4 records
            for (size_t d = 0; d < dim; ++d) {
                CK(cudaMemcpy2DAsync(q, 4, reinterpret_cast<const char *>(c->fw.Vc) + 4 * d, 16, 4, n,
                                     cudaMemcpyDeviceToHost, s));
                q += n * 4;
            }
        }
        CK(cudaStreamSynchronize(s));
    }
    const uint32_t crc = crc32(out, sizeof(h) + h.payload_bytes);
    memcpy(out + sizeof(h) + h.payload_bytes, &crc, sizeof(crc));
    return ADE_OK;
}

int ade_checkpoint_load(ade_ctx *c, const void *host_buf, size_t bytes, void *stream)
{
    if (!c || !host_buf) return ade::report_error(ADE_ERR_ARG, "NULL argument");
    const unsigned char *in = static_cast<const unsigned char *>(host_buf);
    if (bytes < sizeof(Header) + sizeof(uint32_t)) return ade::report_error(ADE_ERR_ARG, "checkpoint truncated");
    Header h;
    memcpy(&h, in, sizeof(h));
    if (memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.version != kVersion)
        return ade::report_error(ADE_ERR_ARG, "not a checkpoint of this format");
    if (h.payload_bytes != payload_bytes(c) || h.dim != (uint32_t)c->dim || h.n != (uint32_t)c->n ||
        h.mode != mode_of(c))
        return ade::report_error(ADE_ERR_ARG, "checkpoint was written for a different particle count or mode");
    if (bytes < total_bytes(c)) return ade::report_error(ADE_ERR_ARG, "checkpoint truncated");
    uint32_t crc = 0u;
    memcpy(&crc, in + sizeof(h) + h.payload_bytes, sizeof(crc));
    if (crc != crc32(in, sizeof(h) + h.payload_bytes))
        return ade::report_error(ADE_ERR_ARG, "checkpoint checksum mismatch (corrupted)");
    if (!same_problem(h.p, c->p) || h.dt != c->dt)
        return ade::report_error(ADE_ERR_ARG, "checkpoint was written for different parameters");
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned char *q = in + sizeof(h);
    const size_t n = (size_t)c->n, dim = (size_t)c->dim;
    if (n > 0) {
        CK(cudaMemcpyAsync(c->xq, q, dim * n * 4, cudaMemcpyHostToDevice, s));
        q += dim * n * 4;
        CK(cudaMemcpyAsync(c->C, q, n * 4, cudaMemcpyHostToDevice, s));
        q += n * 4;
        if (c->catt) {
            CK(cudaMemcpyAsync(c->Q, q, n * 4, cudaMemcpyHostToDevice, s));
            q += n * 4;
        }
        if (c->field) {
            // stage v [dim][n] in the sorted records (rebuilt from Vc after every cell build),
            // then re-form the caller-order records and drift increments from it
            float *stage = reinterpret_cast<float *>(c->fw.V);
            CK(cudaMemcpyAsync(stage, q, dim * n * 4, cudaMemcpyHostToDevice, s));
            CK(ade::launch_field_records(c->dim, stage, c->n, c->fp, c->fw, s));
        }
        CK(cudaStreamSynchronize(s));
    }
    c->step = h.step;
    c->t = h.t;
    if (c->field) {
        c->field_set = true;
        c->field_dirty = false;
    }
    if (c->catt) c->flux_set = true;
    c->status_cleared = false;   // the status word is cleared again before the next step
    return ADE_OK;
}

}  // extern "C"
