// sort.cu -- stable LSD radix sort of (u32 key, u32 value) pairs for the cell binning.
//
// Each 8-bit pass runs four kernels:
//   rs_hist    : per-tile digit histogram (shared-memory atomics), stored digit-major;
//   rs_rowscan : exclusive scan of each digit's row over the tiles (block per digit);
//   rs_digitscan: exclusive scan of the 256 digit totals -> global scatter offsets;
//   rs_scatter : tile-stable ranking (warp __match_any_sync peers, per-warp digit counts
//                scanned across warps in order) and scatter.
// Only ceil(bits / 8) passes run: cell keys use ~23-27 bits.  The order of equal keys
// is the input order, so the sorted cell runs list sphere slots in ascending order.
#include <cstdio>

#include "kernels.cuh"

namespace dem {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

int64_t radix_hist_entries(int64_t n)
{
    int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    return 256 * (tiles > 0 ? tiles : 1) + 256;     // matrix + digit totals
}

__global__ void __launch_bounds__(RS_THREADS) rs_hist(const uint32_t *keys, int64_t n, int shift, uint32_t *hist,
                                                      int64_t tiles)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t idx = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of one digit's row of the (digit, tile) histogram, in place; one block
// per digit, coalesced, carrying the running total across 1024-wide chunks.  The row
// total goes to totals[digit].
__global__ void __launch_bounds__(1024) rs_rowscan(uint32_t *a, int64_t tiles, uint32_t *totals)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t *row = a + (int64_t)blockIdx.x * tiles;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < tiles; base += 1024) {
        const int64_t i = base + t;
        const uint32_t v = i < tiles ? row[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const uint32_t c = carry;
        const uint32_t excl = c + (x - v) + (warp > 0 ? wsum[warp - 1] : 0u);
        if (i < tiles) row[i] = excl;
        __syncthreads();
        if (t == 1023) carry = excl + v;
        __syncthreads();
    }
    if (t == 0) totals[blockIdx.x] = carry;
}

// Exclusive scan of the 256 digit totals (one block).
__global__ void __launch_bounds__(256) rs_digitscan(uint32_t *totals)
{
    __shared__ uint32_t s[256];
    const int t = threadIdx.x;
    s[t] = totals[t];
    __syncthreads();
    if (t == 0) {
        uint32_t run = 0;
        for (int d = 0; d < 256; ++d) {
            uint32_t v = s[d];
            s[d] = run;
            run += v;
        }
    }
    __syncthreads();
    totals[t] = s[t];
}

__global__ void __launch_bounds__(RS_THREADS) rs_scatter(const uint32_t *keys, const uint32_t *vals, int64_t n,
                                                         int shift, const uint32_t *offs, const uint32_t *digit_base,
                                                         int64_t tiles, uint32_t *keys_out, uint32_t *vals_out)
{
    __shared__ uint32_t base_d[256];             // next output position per digit
    __shared__ uint32_t wcnt[RS_WARPS][256];     // per warp, per digit counts -> warp offsets
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    base_d[t] = digit_base[t] + offs[(int64_t)t * tiles + blockIdx.x];
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) wcnt[w][t] = 0;
        __syncthreads();
        const int64_t idx = tile0 + (int64_t)r * RS_THREADS + t;
        const bool valid = idx < n;
        uint32_t key = valid ? keys[idx] : 0u;
        uint32_t val = valid ? vals[idx] : 0u;
        const uint32_t dg = valid ? ((key >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][dg] = __popc(peers);
        __syncthreads();
        // thread t scans digit t across the warps of this round
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t c = wcnt[w][t];
            wcnt[w][t] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = base_d[dg] + wcnt[warp][dg] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        base_d[t] += run;
        __syncthreads();
    }
}

void radix_sort_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, int64_t n, int bits,
                    uint32_t *hist, int64_t hist_cap, cudaStream_t st, uint32_t **keys_out, uint32_t **vals_out)
{
    uint32_t *ka = keys, *va = vals, *kb = keys_alt, *vb = vals_alt;
    if (n > 0) {
        int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
        (void)hist_cap;
        for (int shift = 0; shift < bits; shift += 8) {
            uint32_t *totals = hist + 256 * tiles;
            rs_hist<<<(unsigned)tiles, RS_THREADS, 0, st>>>(ka, n, shift, hist, tiles);
            rs_rowscan<<<256, 1024, 0, st>>>(hist, tiles, totals);
            rs_digitscan<<<1, 256, 0, st>>>(totals);
            rs_scatter<<<(unsigned)tiles, RS_THREADS, 0, st>>>(ka, va, n, shift, hist, totals, tiles, kb, vb);
            uint32_t *tk = ka; ka = kb; kb = tk;
            uint32_t *tv = va; va = vb; vb = tv;
        }
    }
    *keys_out = ka;
    *vals_out = va;
}

}  // namespace dem
