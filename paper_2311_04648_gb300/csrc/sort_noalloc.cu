// sort_noalloc.cu -- the radix sort for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is being
// captured (an allocation there is not allowed), host code of a framework that owns the
// device memory through its own pool, or latency-critical loops in which an allocation
// could synchronise the device.  dem_util_radix_sort_u32_noalloc serves them: they pass
// device buffers for the input and the output, and the sort's temporary storage (the
// alternate key/value buffers and the digit histogram) lives in one file-scope device
// array, sized for at most DEM_NOALLOC_SORT_MAX keys, that every GPU loading this
// library keeps until the process exits.
#include <mutex>

#include "../../include/dem.h"
#include "kernels.cuh"

namespace dem {

// the pass kernels of sort.cu
__global__ void rs_hist(const uint32_t *keys, int64_t n, int shift, uint32_t *hist, int64_t tiles);
__global__ void rs_rowscan(uint32_t *a, int64_t tiles, uint32_t *totals);
__global__ void rs_digitscan(uint32_t *totals);
__global__ void rs_scatter(const uint32_t *keys, const uint32_t *vals, int64_t n, int shift, const uint32_t *offs,
                           const uint32_t *digit_base, int64_t tiles, uint32_t *keys_out, uint32_t *vals_out);

namespace {

constexpr int64_t MAXN = DEM_NOALLOC_SORT_MAX;
constexpr int64_t MAX_HIST = 256 * ((MAXN + 4095) / 4096) + 256;   // digit rows + digit totals
constexpr int64_t SCRATCH_WORDS = 2 * MAXN + MAX_HIST;

// Alternate keys [0, MAXN), alternate values [MAXN, 2 MAXN), histogram after them.
static __device__ __align__(256) uint32_t g_sort_scratch[SCRATCH_WORDS];

std::mutex g_mu;
constexpr int MAX_DEV = 64;
void *g_ptr[MAX_DEV] = {};

thread_local const char *g_msg = "";

// [a, a + len) and [b, b + len) share a byte
bool ranges_overlap(uint64_t a, uint64_t b, uint64_t len) { return a < b + len && b < a + len; }

}  // namespace
}  // namespace dem

using namespace dem;

extern "C" const char *dem_util_noalloc_error(void) { return g_msg; }

extern "C" dem_status dem_util_radix_sort_u32_noalloc(int64_t n, const uint32_t *keys, const uint32_t *vals,
                                                       int32_t bits, uint32_t *keys_out, uint32_t *vals_out,
                                                       void *stream)
{
    g_msg = "";                          // a message describes the last call only
    if (n < 0 || bits < 1 || bits > 32) { g_msg = "need n >= 0 and 1 <= bits <= 32"; return DEM_ERR_ARG; }
    if (n > MAXN) { g_msg = "n exceeds DEM_NOALLOC_SORT_MAX keys"; return DEM_ERR_CAPACITY; }
    if (n == 0) return DEM_OK;
    if (!keys || !vals || !keys_out || !vals_out) { g_msg = "null buffer"; return DEM_ERR_ARG; }
    // a pass reads its whole input while other blocks write its output: neither output
    // may share a byte with an input or with the other output
    const uint64_t bytes = 4ull * (uint64_t)n;
    const uint64_t ko = (uint64_t)(uintptr_t)keys_out, vo = (uint64_t)(uintptr_t)vals_out;
    const uint64_t ki = (uint64_t)(uintptr_t)keys, vi = (uint64_t)(uintptr_t)vals;
    if (ranges_overlap(ko, ki, bytes) || ranges_overlap(ko, vi, bytes) || ranges_overlap(vo, ki, bytes) ||
        ranges_overlap(vo, vi, bytes) || ranges_overlap(ko, vo, bytes)) {
        g_msg = "output buffers must not overlap the inputs or each other";
        return DEM_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) { g_msg = "no current CUDA device"; return DEM_ERR_CUDA; }
    void *base = nullptr;
    {
        // set-up, once per device, with that device current: the host-side name of the
        // array is not a device address, so the address is looked up and kept
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
            if (e != cudaSuccess || !p) { g_msg = "cudaGetSymbolAddress failed for the sort scratch"; return DEM_ERR_CUDA; }
            g_ptr[dev] = p;
        }
        base = g_ptr[dev];
    }
    uint32_t *alt_k = reinterpret_cast<uint32_t *>(base);
    uint32_t *alt_v = alt_k + MAXN;
    uint32_t *hist = alt_k + 2 * MAXN;
    const int64_t tiles = (radix_hist_entries(n) - 256) / 256;
    uint32_t *totals = hist + 256 * tiles;
    cudaStream_t st = (cudaStream_t)stream;
    // every histogram entry and digit total is written before it is read, so nothing in
    // the shared array has to start at zero; the passes ping-pong so that the last one
    // lands in the caller's output
    const int passes = (bits + 7) / 8;
    const uint32_t *sk = keys, *sv = vals;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t *dk = to_out ? keys_out : alt_k;
        uint32_t *dv = to_out ? vals_out : alt_v;
        const int shift = 8 * p;
        rs_hist<<<(unsigned)tiles, 256, 0, st>>>(sk, n, shift, hist, tiles);
        rs_rowscan<<<256, 1024, 0, st>>>(hist, tiles, totals);
        rs_digitscan<<<1, 256, 0, st>>>(totals);
        rs_scatter<<<(unsigned)tiles, 256, 0, st>>>(sk, sv, n, shift, hist, totals, tiles, dk, dv);
        sk = dk;
        sv = dv;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { g_msg = cudaGetErrorString(e); return DEM_ERR_CUDA; }
    return DEM_OK;
}
