// mad_noalloc.cu -- the m-th best-match distance re-check (the FP64
// recompute behind mad_discords' dist_recheck) with its working memory in a
// fixed, statically sized device array instead of cudaMalloc'd buffers.
//
// Why a caller may be unable to allocate: cudaMalloc can fail, or make a
// caching allocator give memory back, when the process's device memory is
// held in pools (a PyTorch process, for one); cudaFree waits for the whole
// device, which stalls unrelated streams of a latency-bound caller; and some
// callers must know their memory footprint before they start. The entry
// point below allocates nothing: its scratch is linked into the library and
// its address is looked up in the calling context.
//
// The paper has no counterpart of this function; the quantity it computes is
// the m-th best-match distance (Def. "m-th best match") at one length, from a full
// FP64 distance profile (Eq. DIST, two-pass window statistics).
#include <climits>
#include <string>

#include "kernels.cuh"
#include "mad.h"

namespace mad {

void set_thread_error(const std::string &msg);   // mad_api.cu

namespace {

// Scratch layout (one copy per device):
//   cells : NOALLOC_MAX_SLOTS x 3 int32   (off, len, m) copied from the host
//   sd    : NOALLOC_MAX_SLOTS x RSLICES doubles   per-slice sorted distances
//   sj    : NOALLOC_MAX_SLOTS x RSLICES int32     their offsets
// with one slot per (cell, rank) pair: a call needs ncells * m_max slots.
constexpr int NOALLOC_RSLICES = 64;                 // slices per cell of k_recheck_slices
constexpr size_t ALIGN = 256;
constexpr size_t round_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }
constexpr size_t CELLS_BYTES = round_up((size_t)MAD_NOALLOC_MAX_SLOTS * 3 * sizeof(int32_t));
constexpr size_t SD_BYTES = round_up((size_t)MAD_NOALLOC_MAX_SLOTS * NOALLOC_RSLICES * sizeof(double));
constexpr size_t SJ_BYTES = round_up((size_t)MAD_NOALLOC_MAX_SLOTS * NOALLOC_RSLICES * sizeof(int32_t));
constexpr size_t SCRATCH_BYTES = CELLS_BYTES + SD_BYTES + SJ_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;

// Device address of the scratch in the current context. Looked up on every
// call rather than cached: after cudaDeviceReset (or in another context on
// the same device) the module is loaded again, possibly at another address,
// and a cached pointer would then point at freed memory. Once the module is
// loaded in the context the lookup allocates nothing; the first call in a
// context loads it, which is set-up work (make that first call before any
// stream capture begins).
cudaError_t scratch_address(unsigned char **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}

bool is_device_pointer(const void *p, int dev)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // a failed query stays as the last error: clear it
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

mad_status fail(mad_status s, const std::string &msg)
{
    set_thread_error(msg);
    return s;
}

}  // namespace
}  // namespace mad

using namespace mad;

MAD_API mad_status mad_mth_nn_dist_noalloc(const double *x, int64_t n, const int32_t *cells, int32_t ncells,
                                           int32_t m_max, int32_t excl_num, int32_t excl_den, double *out,
                                           void *stream)
{
    // argument checks first: none of them touches the GPU
    if (ncells < 0) return fail(MAD_EINVAL, "ncells must be >= 0");
    if (ncells == 0) return MAD_OK;
    if (!x || !cells || !out) return fail(MAD_EINVAL, "x, cells and out must not be NULL");
    if (n < 4) return fail(MAD_EINVAL, "series needs at least 4 samples");
    // offsets and partners are 32-bit in the re-check kernels
    if (n - 1 > (int64_t)INT32_MAX) return fail(MAD_EINVAL, "series longer than 2^31 samples");
    if (m_max < 1 || m_max > MAXP) return fail(MAD_EINVAL, "m_max must be in [1, 64]");
    if (excl_num < 0 || excl_den < 1) return fail(MAD_EINVAL, "exclusion fraction needs num >= 0 and den >= 1");
    if ((int64_t)ncells * m_max > MAD_NOALLOC_MAX_SLOTS)
        return fail(MAD_EINVAL, "ncells * m_max = " + std::to_string((int64_t)ncells * m_max) +
                                    " exceeds the fixed scratch of " + std::to_string(MAD_NOALLOC_MAX_SLOTS) +
                                    " (cell, rank) slots");
    for (int32_t c = 0; c < ncells; ++c) {
        const int64_t off = cells[3 * c], len = cells[3 * c + 1], m = cells[3 * c + 2];
        if (len < 2 || len > n) return fail(MAD_EINVAL, "cell " + std::to_string(c) + ": len must be in [2, n]");
        if (off < 0 || off + len > n)
            return fail(MAD_EINVAL, "cell " + std::to_string(c) + ": window [off, off+len) outside the series");
        if (m < 1 || m > m_max) return fail(MAD_EINVAL, "cell " + std::to_string(c) + ": m must be in [1, m_max]");
    }

    // the scratch was sized for the re-check kernel's slice count
    if (recheck_scratch(1, 1) != (size_t)NOALLOC_RSLICES)
        return fail(MAD_EINTERNAL, "slice count of the re-check kernel differs from the scratch layout");

    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MAD_ECUDA, std::string("cudaGetDevice(): ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(MAD_EINVAL, "device ordinal out of range");
    if (!is_device_pointer(x, dev) || !is_device_pointer(out, dev))
        return fail(MAD_EINVAL, "x and out must be device memory of the current device");
    unsigned char *base = nullptr;
    e = scratch_address(&base);
    if (e != cudaSuccess) return fail(MAD_ECUDA, std::string("cudaGetSymbolAddress(): ") + cudaGetErrorString(e));

    // No part of the scratch has to start at zero: the cells region is
    // written by the copy below, and the merge kernel reads, per cell, the
    // first m slots of each slice, which the slice kernel writes earlier in
    // the same call.
    int32_t *dcells = reinterpret_cast<int32_t *>(base);
    double *sd = reinterpret_cast<double *>(base + CELLS_BYTES);
    int32_t *sj = reinterpret_cast<int32_t *>(base + CELLS_BYTES + SD_BYTES);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(dcells, cells, (size_t)ncells * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(MAD_ECUDA, std::string("cudaMemcpyAsync(): ") + cudaGetErrorString(e));
    launch_recheck_discords(x, n, dcells, ncells, excl_num, excl_den, out, sd, sj, m_max, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MAD_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(MAD_ECUDA, std::string("cudaStreamSynchronize(): ") + cudaGetErrorString(e));
    return MAD_OK;
}
