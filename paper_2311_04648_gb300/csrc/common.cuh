// common.cuh -- shared device/host definitions of the GB300 DEM pipeline.
//
// Two position forms share every kernel through the policies FormF64 / FormF32:
//   FormF64: owner position = three doubles (the plain FP64 form);
//   FormF32: owner position = integer voxel index per axis (21 bits each, packed in a
//            u64) + FP32 offset in [0, L) inside the voxel.  The voxel IS the detection
//            cell, so binning needs no floating point, and every position difference is
//            (ci - cj) * L + (oi - oj), exact in the integer part (Sec. 2.3 motivates
//            integer-based coordinates; the FP32 offset replaces the paper's 3 x u16).
// Arithmetic that decides a discrete outcome (sphere centres, pair predicate, voxel
// carry) uses explicit round-to-nearest intrinsics so that it never contracts into
// FMA and every kernel computes bit-identical values.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#ifndef DEM_HD
#define DEM_HD __host__ __device__ __forceinline__
#endif

namespace dem {

constexpr uint32_t WALL_BIT = 0x80000000u;   // partner id with this bit set is a wall
constexpr int KMAX = 64;                      // hard upper bound of a contact-list row
constexpr int VOX_BITS = 21;
constexpr int VOX_BIAS = 1 << (VOX_BITS - 1);
constexpr uint64_t VOX_MASK = (1ull << VOX_BITS) - 1;

enum : int { WALL_PLANE = 0, WALL_CYLINDER = 1, WALL_CONE = 2, WALL_TRIANGLE = 3 };

// halt reasons written by the kernels into DevStatus::halt
enum : int { HALT_NONE = 0, HALT_DIVERGED = 1, HALT_OVERFLOW = 2, HALT_TIMEOUT = 3, HALT_FACETS = 4 };

template <typename R> struct V3 { R x, y, z; };

template <typename R> DEM_HD V3<R> mk(R x, R y, R z) { return V3<R>{x, y, z}; }
template <typename R> DEM_HD V3<R> operator+(V3<R> a, V3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename R> DEM_HD V3<R> operator-(V3<R> a, V3<R> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename R> DEM_HD V3<R> operator-(V3<R> a) { return {-a.x, -a.y, -a.z}; }
template <typename R> DEM_HD V3<R> operator*(R s, V3<R> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename R> DEM_HD R dot(V3<R> a, V3<R> b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
template <typename R> DEM_HD V3<R> cross(V3<R> a, V3<R> b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Exactly rounded (never fused) primitives, overloaded per precision.
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }

// R(q) a with the rotation matrix of the unit quaternion (w, x, y, z), every product and
// sum rounded separately in the fixed order ((R0 a0 + R1 a1) + R2 a2).
template <typename R>
__device__ __forceinline__ V3<R> rotate_exact(R qw, R qx, R qy, R qz, V3<R> a)
{
    const R one = R(1), two = R(2);
    R xx = rmul(qx, qx), yy = rmul(qy, qy), zz = rmul(qz, qz);
    R xy = rmul(qx, qy), xz = rmul(qx, qz), yz = rmul(qy, qz);
    R wx = rmul(qw, qx), wy = rmul(qw, qy), wz = rmul(qw, qz);
    R m00 = rsub(one, rmul(two, radd(yy, zz))), m01 = rmul(two, rsub(xy, wz)), m02 = rmul(two, radd(xz, wy));
    R m10 = rmul(two, radd(xy, wz)), m11 = rsub(one, rmul(two, radd(xx, zz))), m12 = rmul(two, rsub(yz, wx));
    R m20 = rmul(two, rsub(xz, wy)), m21 = rmul(two, radd(yz, wx)), m22 = rsub(one, rmul(two, radd(xx, yy)));
    V3<R> o;
    o.x = radd(radd(rmul(m00, a.x), rmul(m01, a.y)), rmul(m02, a.z));
    o.y = radd(radd(rmul(m10, a.x), rmul(m11, a.y)), rmul(m12, a.z));
    o.z = radd(radd(rmul(m20, a.x), rmul(m21, a.y)), rmul(m22, a.z));
    return o;
}

// Ordinary (contractible) rotation and its transpose, for dynamics.
template <typename R>
DEM_HD void quat_mat(R qw, R qx, R qy, R qz, R m[9])
{
    R xx = qx * qx, yy = qy * qy, zz = qz * qz, xy = qx * qy, xz = qx * qz, yz = qy * qz;
    R wx = qw * qx, wy = qw * qy, wz = qw * qz;
    m[0] = R(1) - R(2) * (yy + zz); m[1] = R(2) * (xy - wz); m[2] = R(2) * (xz + wy);
    m[3] = R(2) * (xy + wz); m[4] = R(1) - R(2) * (xx + zz); m[5] = R(2) * (yz - wx);
    m[6] = R(2) * (xz - wy); m[7] = R(2) * (yz + wx); m[8] = R(1) - R(2) * (xx + yy);
}
template <typename R> DEM_HD V3<R> mat_vec(const R m[9], V3<R> a)
{
    return {(m[0] * a.x + m[1] * a.y) + m[2] * a.z, (m[3] * a.x + m[4] * a.y) + m[5] * a.z,
            (m[6] * a.x + m[7] * a.y) + m[8] * a.z};
}
template <typename R> DEM_HD V3<R> mat_tvec(const R m[9], V3<R> a)
{
    return {(m[0] * a.x + m[3] * a.y) + m[6] * a.z, (m[1] * a.x + m[4] * a.y) + m[7] * a.z,
            (m[2] * a.x + m[5] * a.y) + m[8] * a.z};
}

// ------------------------------------------------------------------ scene-level data

struct Wall {            // analytical wall (device copy); geometry in FP64
    int type, mat;       // global material id
    double p[3], n[3];
    double r0, z0, r1, z1;
    double omega[3];
    float pf[3], nf[3];  // FP32 copies for screening tests (decide only far from the
    float r0f, r1f, z0f, z1f;   // threshold, see wall_gap_f)
    float tolf;          // screening tolerance per unit of (|centre|_1 + 1), see wall_gap_f
    // a plane normal to a coordinate axis and not moving: axis (else -1), side (+1 / -1)
    // and its position on the scene's voxel grid (voxel index, offset in [0, Lv) as a
    // float-float pair), so that the voxel form measures gaps from voxel differences in FP32
    int axis, ax_c;
    float ax_sign, ax_off, ax_off_lo;
    // a mesh facet (WALL_TRIANGLE): vertices at time 0 and at the current step (the mesh
    // turns with omega about p), two-sided
    double tri[9];
    double cur[9];
    int scene;           // the scene it belongs to
};

struct Scene {           // per-scene constants (device copy)
    double lo[3];        // origin of the cell grid
    float lof[3];        // the same rounded to FP32 (screening only)
    int nc[3];           // cells per axis
    uint32_t cell_base;  // first global cell index of this scene
    double h, g[3];
    float hf, gf[3];
    double v_err;        // <= 0: off
    float v_errf;        // largest float not above v_err: a float speed s has s <= v_errf
                         // exactly when s <= v_err
    int wall_begin, wall_count;
    int has_sink;
    double sink_p[3], sink_n[3];
    int mat_base, n_mat, pair_base;
    int nb[3];           // schedule bins per axis (BIN_CELLS smallest cells each)
    int nbc[3];          // smallest cells per axis (the bins' grid; detection cells may be larger)
    int bin_base;        // first global bin of this scene
    int has_rolling;     // a material pair of this scene has C_r > 0
    int facet_begin, facet_count;   // mesh facets: walls found by the binned facet search
};

constexpr int BIN_CELLS = 8;     // cells per schedule-bin edge
constexpr int NSTAT = 10;        // per-bin motion statistics

// Family tags (Sec. 2.2.2): every owner carries a family (0..255).  A family may have a
// prescribed linear and/or angular velocity (global frame) that replaces the one its
// forces would give; pairs of families may have their contacts left unresolved.
constexpr int N_FAMILY = 256;
struct FamilyMotion {
    int fix_v, fix_w;
    double v[3], w[3];
    float vf[3], wf[3];  // the same rounded to FP32
};
// contact mask: bit b of word (a * 8 + b / 32) set = contacts of families a and b resolved
constexpr int FAMILY_MASK_WORDS = N_FAMILY * N_FAMILY / 32;
DEM_HD bool families_meet(const uint32_t *mask, int a, int b)
{
    return (mask[(a << 3) | (b >> 5)] >> (b & 31)) & 1u;
}

struct PairParam {       // pairwise contact constants, precomputed on the host in FP64
    double Estar, Gstar, beta, mu;
};
struct PairParamF {      // the same rounded to FP32 once, for the voxel form
    float Estar, Gstar, beta, mu;
};

// Device-resident control block (one per world).  Kernels read the selectors and flags
// here, so the host can queue work (or replay a CUDA graph) without knowing in advance
// which buffers hold the current state, whether a list went stale or a step diverged.
// Per-warp maxima of a step (float bits: displacement bound of the list in use, of the
// list being built, speed) land in AUDIT_SLOTS slots of their own array, one 128-byte
// line per slot (AUDIT_STRIDE words), so the atomics spread over the L2 instead of
// sharing lines with each other or with the control block that every thread reads.
constexpr int AUDIT_SLOTS = 64;
constexpr int AUDIT_STRIDE = 32;

struct DevStatus {
    // read by every thread of the step kernels; written by single threads between kernels
    int halt;                    // HALT_*: every kernel returns immediately
    int list_stale;              // list in use no longer covers every contact: force skips
    int state_par;               // owner-state buffer holding the current state
    int hist_par;                // history buffer holding the current history
    int list_cur;                // contact list in use
    int acc_par;                 // displacement accumulator of the list in use (the other: next)
    unsigned int step_disp_bits; // max over owners of this step's displacement bound (float bits)
    unsigned int vmax_bits;      // max |v| over owners this step (float bits)
    unsigned int upload_disp_bits; // max over uploaded owners of the in-use list's bound after
                                   // their displacement by a state upload (float bits)
    double disp_cur;             // displacement bound since the snapshot of the list in use
    double disp_next;            // ... since the snapshot of the list being built
    double beta_cur, beta_next;  // margins of those lists
    float beta_next_f;           // beta_next rounded to FP32
    double vmax_last;            // max |v| after the last completed step
    double disp_slack;           // added per step: rounding of the position update
    float disp_slack_f;          // the same (a power of two, exact in FP32)
    long long steps_done;
    long long rebuilds;
    unsigned int cell_stamp;     // stamp of the cell table of the build in progress (from 1)
    unsigned long long pair_steps;   // sum over completed steps of the pairs in use
    unsigned long long busy_steps;   // sum over completed steps of the slots with partners
    long long stale_events;
    long long snap_step;         // step of the snapshot of the list being built (mesh poses)
    // updated by atomics of many threads (narrow phase, compaction, link, divergence): a
    // line of their own, away from the fields above
    alignas(128) int overflow;   // a row exceeded the list capacity in the last narrow phase
    int max_row;                 // longest row of the last narrow phase
    int diverged;                // set by the force kernel, turned into a halt by the audit
    unsigned int list_pairs[2];  // sphere-sphere pairs of each list (each pair once)
    unsigned int list_busy[2];   // slots of each list with listed partners
    unsigned int n_screen;       // spheres the screening pass of this step passed on to the
                                 // evaluation (zeroed by the audit after every step)
};

// ------------------------------------------------------------------ position forms

struct PosF64 { double x, y, z; };
struct PosF32 { int cx, cy, cz; float x, y, z; };

DEM_HD uint64_t pack_vox(int cx, int cy, int cz)
{
    return (uint64_t)((uint32_t)(cx + VOX_BIAS) & VOX_MASK) |
           ((uint64_t)((uint32_t)(cy + VOX_BIAS) & VOX_MASK) << VOX_BITS) |
           ((uint64_t)((uint32_t)(cz + VOX_BIAS) & VOX_MASK) << (2 * VOX_BITS));
}
DEM_HD void unpack_vox(uint64_t v, int &cx, int &cy, int &cz)
{
    cx = (int)(v & VOX_MASK) - VOX_BIAS;
    cy = (int)((v >> VOX_BITS) & VOX_MASK) - VOX_BIAS;
    cz = (int)((v >> (2 * VOX_BITS)) & VOX_MASK) - VOX_BIAS;
}

struct FormF64 {
    using R = double;
    using R4 = double4_32a;
    using Pos = PosF64;
    static constexpr bool voxel = false;
    // owner position storage: double4_32a (x, y, z, mass)
    struct PosStore { double4_32a *xm; };
    struct Aux {};              // nothing rides along with the position in this form

    __device__ static Pos load(const PosStore &s, int64_t o, R &mass)
    {
        double4_32a a = s.xm[o];
        mass = a.w;
        return Pos{a.x, a.y, a.z};
    }
    __device__ static Pos load(const PosStore &s, int64_t o, R &mass, Aux &) { return load(s, o, mass); }
    __device__ static void store(PosStore &s, int64_t o, Pos p, R mass, const Aux & = Aux{})
    {
        s.xm[o] = make_double4_32a(p.x, p.y, p.z, mass);
    }
    // a - b, exactly rounded component-wise
    __device__ static V3<R> diff(const Pos &a, const Pos &b, float /*L*/)
    {
        return {rsub(a.x, b.x), rsub(a.y, b.y), rsub(a.z, b.z)};
    }
    __device__ static Pos advance(Pos p, V3<R> d, float /*L*/) { return Pos{radd(p.x, d.x), radd(p.y, d.y), radd(p.z, d.z)}; }
    // cell of a position in a scene grid (unclamped)
    __device__ static void cell(const Pos &p, const Scene &sc, double invL, int /*vpc*/, int &cx, int &cy, int &cz)
    {
        cx = (int)floor(rmul(rsub(p.x, sc.lo[0]), invL));
        cy = (int)floor(rmul(rsub(p.y, sc.lo[1]), invL));
        cz = (int)floor(rmul(rsub(p.z, sc.lo[2]), invL));
    }
    __device__ static V3<double> absolute(const Pos &p, const Scene &, double) { return {p.x, p.y, p.z}; }
};

struct FormF32 {
    using R = float;
    using R4 = float4;
    using Pos = PosF32;
    static constexpr bool voxel = true;
    // owner position storage: one 32-byte record per owner (one DRAM sector): offset and
    // mass, the packed voxel index, and for a single sphere its radius as a float-float
    // pair (the sphere's constants travel with its position, so a partner's gather reads
    // one sector; for clumps the two words are unused)
    struct PosRec {
        float4 om;              // offset x, y, z, mass
        uint4 vr;               // voxel index (low, high word), radius, radius low word (bits)
    };
    struct PosStore { PosRec *rec; };
    struct Aux { float rad, rlo; };

    __device__ static Pos load(const PosStore &s, int64_t o, R &mass, Aux &aux)
    {
        const float4 a = s.rec[o].om;
        const uint4 b = s.rec[o].vr;
        Pos p;
        unpack_vox((uint64_t)b.x | ((uint64_t)b.y << 32), p.cx, p.cy, p.cz);
        p.x = a.x; p.y = a.y; p.z = a.z;
        mass = a.w;
        aux.rad = __uint_as_float(b.z);
        aux.rlo = __uint_as_float(b.w);
        return p;
    }
    __device__ static Pos load(const PosStore &s, int64_t o, R &mass)
    {
        Aux aux;
        return load(s, o, mass, aux);
    }
    // the whole record is written (no partially written sector)
    __device__ static void store(PosStore &s, int64_t o, Pos p, R mass, const Aux &aux)
    {
        const uint64_t v = pack_vox(p.cx, p.cy, p.cz);
        s.rec[o].om = make_float4(p.x, p.y, p.z, mass);
        s.rec[o].vr = make_uint4((uint32_t)v, (uint32_t)(v >> 32), __float_as_uint(aux.rad), __float_as_uint(aux.rlo));
    }
    // (ca - cb) * L + (oa - ob): the integer part is exact, then two rounded operations
    __device__ static V3<R> diff(const Pos &a, const Pos &b, float L)
    {
        V3<R> d;
        d.x = radd(rmul((float)(a.cx - b.cx), L), rsub(a.x, b.x));
        d.y = radd(rmul((float)(a.cy - b.cy), L), rsub(a.y, b.y));
        d.z = radd(rmul((float)(a.cz - b.cz), L), rsub(a.z, b.z));
        return d;
    }
    // keep the offset in [0, L): carry whole voxels into the index
    __device__ static void carry(int &c, float &o, float L)
    {
        if (o >= L || o < 0.0f) {
            float k = floorf(__fdiv_rn(o, L));
            o = rsub(o, rmul(k, L));
            c += (int)k;
            if (o >= L) { o = rsub(o, L); c += 1; }
            if (o < 0.0f) { o = radd(o, L); c -= 1; }
        }
    }
    __device__ static Pos advance(Pos p, V3<R> d, float L)
    {
        Pos q = p;
        q.x = radd(p.x, d.x); q.y = radd(p.y, d.y); q.z = radd(p.z, d.z);
        carry(q.cx, q.x, L); carry(q.cy, q.y, L); carry(q.cz, q.z, L);
        return q;
    }
    // detection cell of a voxel: floor division by the voxels per cell edge
    __device__ static int floordiv(int a, int b) { int q = a / b; return (a % b != 0 && a < 0) ? q - 1 : q; }
    __device__ static void cell(const Pos &p, const Scene &, double, int vpc, int &cx, int &cy, int &cz)
    {
        cx = floordiv(p.cx, vpc); cy = floordiv(p.cy, vpc); cz = floordiv(p.cz, vpc);
    }
    // world-frame position in FP64: (lo + c L) + o
    __device__ static V3<double> absolute(const Pos &p, const Scene &sc, double L)
    {
        return {radd(radd(sc.lo[0], rmul((double)p.cx, L)), (double)p.x),
                radd(radd(sc.lo[1], rmul((double)p.cy, L)), (double)p.y),
                radd(radd(sc.lo[2], rmul((double)p.cz, L)), (double)p.z)};
    }
};

}  // namespace dem
