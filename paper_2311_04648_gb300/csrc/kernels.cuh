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
    // per cell (start, stamp, end, 0): the sorted run [start, end) of the cell, valid only
    // when stamp equals the build's stamp (the table is never cleared; one 16-byte load
    // per cell)
    uint4 *cell_tab;
    uint32_t n_cells_total;    // sentinel key (inactive / padding slots)
    int key_bits;
    // snapshot of sphere centres in slot order and the same gathered in sorted order
    void *snap;                // double4_32a (x, y, z, R) or {uint64 vox ; float4 (off, R)}
    void *snap_aux;            // float4 part of the FP32 form (nullptr for FP64)
    void *sorted;              // gathered snapshot in cell order
    void *sorted_aux;
    uint32_t *sorted_owner;    // owner of each sorted entry
    uint8_t *sorted_family;    // family of each sorted entry (only where families mask contacts)
    // mesh facets (walls of type WALL_TRIANGLE): each build bins the facets, at their pose
    // at the snapshot, into the cells their reach covers, as (cell key, facet) pairs sorted
    // by key; a sphere tests the facets of its own cell
    int n_facets;
    const int *facet_wall;     // wall index of facet f
    const int64_t *facet_off;  // first pair slot of facet f (n_facets + 1 entries)
    double *tri_snap;          // facet vertices at the snapshot (9 per facet)
    uint32_t *fkeys, *fvals, *fkeys_alt, *fvals_alt, *fhist;
    int64_t n_fpairs, fhist_cap;
    const uint32_t *fkeys_sorted, *fvals_sorted;   // after the sort (one of the two buffers)
    uint32_t *n_valid;         // device counter: active entries at the front of the order
    uint32_t *rowcnt;          // per slot: entries appended to its row by the narrow phase
    // counting-sort binning: per-cell counts (a whole number of scan tiles, zero between
    // builds), each slot's rank in its cell, the scan's per-tile sums
    uint32_t *ccount, *crank, *ctile;
    int64_t ccount_len;
    int counting;              // 1: this build bins by counting sort, 0: by radix sort
    uint8_t *cell_wall;        // per cell: 1 if a (non-facet) wall may be in reach from it
};

// Two contact lists (ELL rows) plus two history buffers; DevStatus selects which.
// Tangential history of one list entry as one vector (x, y, z, unused): a scattered
// entry costs one memory sector to read or write instead of three.
template <typename R> struct HistVec;
template <> struct HistVec<float> { using T = float4; };
template <> struct HistVec<double> { using T = double4_32a; };

// A sphere's constants packed for the scattered loads of the contact kernel (one
// memory sector): FP32 form (radius, radius low word, material as int bits, 0), FP64
// form (radius, material).
template <typename R> struct SphPack;
template <> struct SphPack<float> { using T = float4; };
template <> struct SphPack<double> { using T = double2; };

template <typename R>
struct ListBuffers {
    uint32_t *partner[2];
    uint8_t *cnt[2];
    typename HistVec<R>::T *hist[2];
    // compacted work of each list: slots with listed partners (single spheres) or
    // 32-slot groups containing any (clumps), and their number
    uint4 *act[2];
    uint32_t *n_act[2];
    // single spheres: per block of 256 slots, the slots' offsets within the block in
    // order of row length (empty rows first), for the fused step kernel
    uint8_t *perm[2];
    // contact wildcards 4..7 of each entry (contact models with more than four; else null)
    typename HistVec<R>::T *wild[2];
    // single spheres: busy slots per block of 256, scanned into each block's offset in the
    // compacted work (so that the work follows slot order), the total last; one array for
    // the compaction of the new list and one for that of the list in use
    uint32_t *bcount[2];
};

// Owner-state double buffers.
template <class F>
struct StateBuffers {
    typename F::PosStore pos[2];
    // linear and angular velocity of owner o side by side, kv[2o] = (v, acc[0]) and
    // kv[2o + 1] = (w, acc[1]): one 32-byte sector per owner in the voxel form
    typename F::R4 *kv[2], *quat[2];
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
