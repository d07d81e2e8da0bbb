// noalloc.cu -- ade_build_cells_noalloc: the cell-list build for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: plug-ins that receive
// only their input and output buffers, code whose device memory is owned by another allocator
// or pool, and loops that cannot afford cudaMalloc's implicit device-wide synchronisation.  This
// entry point runs the same cell build as ade_build_cells (keys, counting sort, per-cell order,
// sorted copy), but its scratch buffers live in one static device array defined below, so it
// allocates nothing.  The array is reserved by every GPU that loads the library, until the
// process exits.
//
// Limits and sharing: at most ADE_NOALLOC_MAX_PARTICLES particles and ADE_NOALLOC_MAX_CELLS cells
// per call.  All calls share the one array; it keeps the last call's contents, and the per-cell
// counters are cleared at the start of every call.  Two calls whose work overlaps on the GPU
// (different streams, or different host threads, on the same device) race on the array: the
// caller must order them.
#include <cuda.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "ade_internal.h"

namespace {

constexpr size_t kMaxN = ADE_NOALLOC_MAX_PARTICLES;
constexpr size_t kMaxCells = ADE_NOALLOC_MAX_CELLS;
constexpr size_t kMaxScanBlocks = (kMaxCells + ade::kScanTileCells - 1) / ade::kScanTileCells;

// Word offsets of the scratch buffers inside the array (each 256-byte aligned).
constexpr size_t kAlignWords = 64;
constexpr size_t round_words(size_t w) { return (w + kAlignWords - 1) / kAlignWords * kAlignWords; }
constexpr size_t kOffKeys = 0;
constexpr size_t kOffRank = kOffKeys + round_words(kMaxN);
constexpr size_t kOffPermTmp = kOffRank + round_words(kMaxN);
constexpr size_t kOffCount = kOffPermTmp + round_words(kMaxN);
constexpr size_t kOffBlockSums = kOffCount + round_words(kMaxCells);
constexpr size_t kScratchWords = kOffBlockSums + round_words(kMaxScanBlocks);

static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

// Device address of g_noalloc_scratch, looked up once per device with that device current.  A
// context reset (cudaDeviceReset, or another library destroying the primary context) reloads the
// module and may move the array, so each entry remembers the context it was taken in, by the
// driver's context ID (unique for the life of the process), and the address is looked up again
// when the current context is a different one.
constexpr int kMaxDevices = 64;
struct ScratchEntry {
    unsigned long long ctx_id;
    uint32_t *addr;
};
ScratchEntry g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mutex;

int noalloc_fail(int code, const char *msg) { return ade::report_error(code, msg); }

// The driver's ID of the calling thread's current context (0 if it cannot be read).  The driver
// entry points are fetched through the runtime, so the library does not link libcuda.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q0 == cudaDriverEntryPointSuccess && q1 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f0);
            get_id = reinterpret_cast<GetId>(f1);
        }
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

extern "C" int ade_build_cells_noalloc(int dim, int n, const uint32_t *xq_dev, const float *C_dev,
                                       const int *nc_host, uint32_t *perm_dev,
                                       uint32_t *cell_start_dev, void *sorted_dev, void *stream)
{
    if (dim != 2 && dim != 3) return noalloc_fail(ADE_ERR_ARG, "dim must be 2 or 3");
    if (!nc_host) return noalloc_fail(ADE_ERR_ARG, "nc_host is NULL");
    if (n < 0) return noalloc_fail(ADE_ERR_ARG, "n must be >= 0");
    int nc[3] = {1, 1, 1};
    size_t ncells = 1;
    for (int i = 0; i < dim; ++i) {
        if (nc_host[i] < 1 || nc_host[i] > 65535) return noalloc_fail(ADE_ERR_ARG, "nc must be in 1..65535");
        nc[i] = nc_host[i];
        ncells *= (size_t)nc[i];
    }
    if ((size_t)n > kMaxN)
        return noalloc_fail(ADE_ERR_CAPACITY, "n exceeds ADE_NOALLOC_MAX_PARTICLES (1048576)");
    if (ncells > kMaxCells)
        return noalloc_fail(ADE_ERR_CAPACITY, "cell count exceeds ADE_NOALLOC_MAX_CELLS (1048576)");
    if (!cell_start_dev || (n > 0 && (!xq_dev || !C_dev || !perm_dev || !sorted_dev)))
        return noalloc_fail(ADE_ERR_ARG, "NULL buffer");
    // the kernels store 16-byte records and 4-byte words through these pointers
    if (!aligned(sorted_dev, 16))
        return noalloc_fail(ADE_ERR_ARG, "sorted_dev must be 16-byte aligned");
    if (!aligned(perm_dev, 4) || !aligned(cell_start_dev, 4) || !aligned(xq_dev, 4) || !aligned(C_dev, 4))
        return noalloc_fail(ADE_ERR_ARG, "xq_dev, C_dev, perm_dev and cell_start_dev must be 4-byte aligned");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(ADE_ERR_CUDA, "cudaGetDevice failed or device ordinal out of range");
    uint32_t *scratch;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        ScratchEntry &ent = g_scratch[dev];
        unsigned long long id = current_context_id();
        if (!ent.addr || id == 0 || id != ent.ctx_id) {
            // set-up: the runtime binds the device's context to this thread if none is current
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return noalloc_fail(ADE_ERR_CUDA, "cudaGetSymbolAddress failed");
            ent.addr = static_cast<uint32_t *>(p);
            ent.ctx_id = id ? id : current_context_id();
        }
        scratch = ent.addr;
    }

    ade::Work w;
    memset(&w, 0, sizeof(w));
    w.keys = scratch + kOffKeys;
    w.rank = scratch + kOffRank;
    w.perm_tmp = scratch + kOffPermTmp;
    w.count = scratch + kOffCount;
    w.block_sums = scratch + kOffBlockSums;
    w.perm = perm_dev;
    w.cell_start = cell_start_dev;
    w.P0 = static_cast<uint4 *>(sorted_dev);
    cudaError_t e = ade::launch_build_cells(dim, xq_dev, C_dev, n, nc, (int)ncells, w, (cudaStream_t)stream);
    if (e != cudaSuccess) return noalloc_fail(ADE_ERR_CUDA, cudaGetErrorString(e));
    return ADE_OK;
}
