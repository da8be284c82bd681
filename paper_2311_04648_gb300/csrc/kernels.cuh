// kernels.cuh -- launch declarations shared between the host orchestration (world.cu)
// and the kernel translation units.
#pragma once
#include "common.cuh"

namespace dem {

// Buffers of one contact-detection pass.
struct DetectBuffers {
    int64_t n;                 // sphere slots
    uint32_t *keys, *vals;     // hash output (unsorted)
    uint32_t *keys_alt, *vals_alt;
    uint32_t *hist;            // radix histogram / offsets
    int64_t hist_cap;          // entries
    uint32_t *cell_start, *cell_end;
    uint32_t n_cells_total;    // sentinel key (inactive / padding slots)
    int key_bits;
    // snapshot of sphere centres in slot order and the same gathered in sorted order
    void *snap;                // double4_32a (x, y, z, R) or {uint64 vox ; float4 (off, R)}
    void *snap_aux;            // float4 part of the FP32 form (nullptr for FP64)
    void *sorted;              // gathered snapshot in cell order
    void *sorted_aux;
    uint32_t *sorted_owner;    // owner of each sorted entry
    uint32_t *n_valid;         // device counter: active entries at the front of the order
};

// Two contact lists (ELL rows) plus two history buffers; DevStatus selects which.
template <typename R>
struct ListBuffers {
    uint32_t *partner[2];
    uint8_t *mirror[2];
    uint8_t *cnt[2];
    R *hx[2], *hy[2], *hz[2];
    // compacted work of each list: slots with listed partners (single spheres) or
    // 32-slot groups containing any (clumps), and their number
    uint32_t *act[2];
    uint32_t *n_act[2];
};

// Owner-state double buffers.
template <class F>
struct StateBuffers {
    typename F::PosStore pos[2];
    typename F::R4 *vel[2], *omg[2], *quat[2];
    uint8_t *active[2];
};

// Selectors read by the kernels from DevStatus.
struct Parity {
    int state;   // owner state buffer holding the current state
    int hist;    // history buffer holding the current history
    int list;    // contact list in use
};

// ---- radix sort (sort.cu)
void radix_sort_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, int64_t n, int bits,
                    uint32_t *hist, int64_t hist_cap, cudaStream_t st, uint32_t **keys_out, uint32_t **vals_out);
int64_t radix_hist_entries(int64_t n);

}  // namespace dem
