// pipeline.cuh -- the per-timestep kernels of the DEM contact pipeline, templated on the
// position form (FormF64 / FormF32).  Included by engine_f64.cu and engine_f32.cu.
//
// Per step (arXiv 2311.04648 Sec. 2.1 and Sec. 4):
//   [rebuild]  k_hash -> radix sort -> k_cellstart -> k_narrow -> k_link -> k_compact -> k_commit
//   [advance]  k_contact (contact forces, per-owner sums) -> k_integrate -> k_audit
// Contact lists are ELL rows: entry k of sphere s at k*Np + s, each row holds every
// partner of s (both orientations) sorted by partner id, walls (WALL_BIT | id) last.
// Each side of a pair keeps the tangential history in its own row, in its own
// orientation; both threads evaluate the pair from their own side, every term odd in the
// orientation, so the two copies stay exact negations and the force on B is exactly the
// negated force on A: no force array, no atomic, no lookup of the partner's row.
#pragma once
#include "stage.cuh"
#include "common.cuh"
#include "contact.cuh"
#include "force_models.cuh"
#include "kernels.cuh"

namespace dem {

// One history entry: the tangential displacement (x, y, z) and, in the fourth lane, the
// time the contact has lasted (kept where a scene has rolling resistance, else zero).
template <typename H, typename R>
__device__ __forceinline__ V3<R> hist_get(const H *h, int64_t e)
{
    const H v = h[e];
    return {(R)v.x, (R)v.y, (R)v.z};
}
template <typename H, typename R>
__device__ __forceinline__ V3<R> hist_get(const H *h, int64_t e, R &age)
{
    const H v = h[e];
    age = (R)v.w;
    return {(R)v.x, (R)v.y, (R)v.z};
}
template <typename H, typename R>
__device__ __forceinline__ void hist_put(H *h, int64_t e, V3<R> u, R age = R(0))
{
    H v;
    v.x = u.x; v.y = u.y; v.z = u.z; v.w = age;
    h[e] = v;
}


enum : int { MODE_STEP = 0, MODE_EVAL = 1 };

template <class F>
struct Dev {
    using R = typename F::R;
    using R4 = typename F::R4;
    int64_t M, N, Np;               // owners, sphere slots, ELL stride (multiple of 32)
    int K;                          // list row capacity
    float L;                        // cell (= voxel) edge
    double Ld, invL;
    int gyro;                       // gyroscopic term on
    // voxel form, single spheres, every owner with I = moi_coef m R^2 (one coefficient):
    // 1/m and 1/I are derived from the mass and radius in the position record instead of
    // read from inv_mass / inv_moi
    int solid;
    float moi_coef;
    // single spheres, two-kernel step: 1 where the contact kernel wrote the owner's force
    // of the step (its entries touched something), per owner with listed partners
    uint8_t *touched;
    uint4 *screen;          // two-pass contact step: spheres with entries to evaluate (slot, first
                            // masked partner, entry mask low and high words)
    int n_scenes;
    int vpc;                        // voxels per cell edge (voxel form)
    double bin_invL;                // the smallest cells (schedule bins are made of them)
    int bin_vpc;
    StateBuffers<F> st;
    ListBuffers<R> lists;
    R4 *inv_moi;                    // (1/I1, 1/I2, 1/I3, r_ext)
    R *inv_mass;
    uint16_t *owner_scene;
    uint8_t *owner_iso;
    uint32_t *sph_owner;            // 0xffffffff: padding slot
    R *sph_rad;
    float *sph_rlo;                 // voxel form: radius minus its FP32 rounding (float-float)
    uint16_t *sph_mat;
    R4 *sph_rloc;                   // body-frame offset (x, y, z, 0); clumps only
    typename SphPack<R>::T *sph_pack;   // radius, low word, material in one vector
    uint8_t *sph_head;              // first slot of its owner
    uint8_t *sph_segend;            // lane (within the warp) one past the owner's last slot
    int64_t *owner_first;           // first sphere slot of each owner
    uint8_t *owner_nsph;            // spheres of each owner
    // Per owner, the accumulated displacement bounds since the snapshots of the two lists
    // (acc[0] and acc[1]; acc[acc_par] belongs to the list in use) ride in the unused
    // fourth lanes of the velocity (acc[0]) and angular velocity (acc[1]) vectors, so they
    // are double-buffered with the state and cost no separate memory traffic.
    float *amag;                    // per owner |F|/m of the last step (schedule features)
    R4 *fo, *to;                    // per owner contact force and torque of the step
    const Scene *scenes;
    const Wall *walls;
    const PairParam *pairs;
    const PairParamF *pairs_f;
    const double *crr;              // rolling resistance per material pair (pairs' indexing)
    const float *crr_f;             // the same rounded to FP32
    // family tags; owner_family is null while no family has prescribed motion or masked
    // contacts (the kernels then skip every family lookup)
    const uint8_t *owner_family;
    const FamilyMotion *fam_motion; // [N_FAMILY]
    const uint32_t *fam_mask;       // [FAMILY_MASK_WORDS]
    // a contact model other than the built-in one (force_models.cuh) and its parameters
    int model;
    const double *model_par;
    const float *model_par_f;
    const double *pair_nu;          // mean Poisson ratio per material pair (pairs' indexing)
    const uint16_t *mat_scene, *mat_local;
    DevStatus *status;
    unsigned int *audit;            // AUDIT_SLOTS x AUDIT_STRIDE words (per-warp maxima of a step)
};

// FP32 position of a sphere centre for screening tests (FP64 form: rounded absolute;
// voxel form: grid origin + voxel * edge + offset in FP32).
template <class F>
__device__ __forceinline__ float3 approx_pos(const typename F::Pos &p, const Scene &sc, float L)
{
    if constexpr (F::voxel) {
        return make_float3(sc.lof[0] + (float)p.cx * L + p.x, sc.lof[1] + (float)p.cy * L + p.y,
                           sc.lof[2] + (float)p.cz * L + p.z);
    } else {
        return make_float3((float)p.x, (float)p.y, (float)p.z);
    }
}

// ------------------------------------------------------------------ sphere kinematics

template <class F>
struct SphereK {
    using R = typename F::R;
    typename F::Pos p;   // sphere centre
    V3<R> rl;            // centre minus owner centre of mass, world frame
    V3<R> v, w;          // owner linear velocity and world-frame angular velocity
    R acc0, acc1;        // the fourth lanes of v and w (the audit accumulators)
    R rad, mass;
    float rlo;           // low word of the radius (voxel form)
    int mat;
    uint32_t owner;
};

// A single sphere's position record (and, in the FP64 form, its radius and material)
// without its velocities: the partner of a listed pair, whose velocities are read only
// where the pair overlaps.  The same values as load_sphere<F, false, false> otherwise.
template <class F>
__device__ __forceinline__ SphereK<F> load_sphere_pos(const Dev<F> &d, int sp, uint32_t s)
{
    using R = typename F::R;
    SphereK<F> k;
    k.owner = s;
    R mass;
    typename F::Aux aux;
    k.p = F::load(d.st.pos[sp], s, mass, aux);
    k.mass = mass;
    k.rl = {R(0), R(0), R(0)};
    k.v = {R(0), R(0), R(0)};
    k.w = {R(0), R(0), R(0)};
    k.acc0 = k.acc1 = R(0);
    if constexpr (F::voxel) {
        k.rad = aux.rad;
        k.rlo = aux.rlo;
        k.mat = -1;
    } else {
        const auto pk = d.sph_pack[s];
        k.rad = pk.x;
        k.rlo = 0.0f;
        k.mat = (int)pk.y;
    }
    return k;
}

// MAT false: the material is left at -1 where it would need a load of its own (a single
// sphere in the voxel form, whose other constants ride in its position record); the
// caller reads it only if the scene has several materials.
template <class F, bool CLUMPS, bool MAT = true>
__device__ __forceinline__ SphereK<F> load_sphere(const Dev<F> &d, int sp, uint32_t s)
{
    using R = typename F::R;
    SphereK<F> k;
    // a world of single spheres has one slot per owner, in owner order
    uint32_t o = CLUMPS ? d.sph_owner[s] : s;
    k.owner = o;
    R mass;
    typename F::Aux aux;
    typename F::Pos po = F::load(d.st.pos[sp], o, mass, aux);
    auto v4 = d.st.kv[sp][2 * o];
    auto w4 = d.st.kv[sp][2 * o + 1];
    k.v = {v4.x, v4.y, v4.z};
    k.w = {w4.x, w4.y, w4.z};
    k.acc0 = v4.w;
    k.acc1 = w4.w;
    k.mass = mass;
    if constexpr (F::voxel && !CLUMPS) {
        k.rad = aux.rad;
        k.rlo = aux.rlo;
        k.mat = MAT ? (int)d.sph_mat[s] : -1;
    } else {
        const auto pk = d.sph_pack[s];
        if constexpr (F::voxel) {
            k.rad = pk.x;
            k.rlo = pk.y;
            k.mat = __float_as_int(pk.z);
        } else {
            k.rad = pk.x;
            k.rlo = 0.0f;
            k.mat = (int)pk.y;
        }
    }
    if (CLUMPS) {
        auto q = d.st.quat[sp][o];
        auto r4 = d.sph_rloc[s];
        k.rl = rotate_exact<R>(q.x, q.y, q.z, q.w, V3<R>{r4.x, r4.y, r4.z});
        k.p = F::advance(po, k.rl, d.L);
    } else {
        k.rl = {R(0), R(0), R(0)};
        k.p = po;
    }
    return k;
}

// Velocity of the contact point as a point of a body: v + w x arm, and the arm
// rl + s * n, each product and sum rounded on its own so that the two threads of a pair
// compute bit-identical values for the same side.
template <typename R>
__device__ __forceinline__ V3<R> arm_of(V3<R> rl, R s, V3<R> n)
{
    return {radd(rl.x, rmul(s, n.x)), radd(rl.y, rmul(s, n.y)), radd(rl.z, rmul(s, n.z))};
}
template <typename R>
__device__ __forceinline__ V3<R> point_velocity(V3<R> v, V3<R> w, V3<R> r)
{
    return {radd(v.x, rsub(rmul(w.y, r.z), rmul(w.z, r.y))), radd(v.y, rsub(rmul(w.z, r.x), rmul(w.x, r.z))),
            radd(v.z, rsub(rmul(w.x, r.y), rmul(w.y, r.x)))};
}

// Sphere-sphere contact seen from A (the calling thread's sphere) against B.  Every term
// is an odd function of the orientation and IEEE round-to-nearest is symmetric under
// negation, so B's thread, calling with the roles exchanged (and its copy of the history,
// the negation of A's), obtains exactly the negated force: no canonical reordering.  False if the
// overlap is not positive.
// ANY: the geometry whatever the sign of the overlap (bonded contacts act across a gap);
// false only where the centres coincide.
// Centre difference, distance and overlap of two spheres (positions and radii only).
template <class F>
__device__ __forceinline__ void sphere_gap(const Dev<F> &d, const SphereK<F> &A, const SphereK<F> &B,
                                           V3<typename F::R> &dd, typename F::R &dist, typename F::R &delta)
{
    using R = typename F::R;
    if constexpr (F::voxel) {
        delta = overlap_ff(A.p, B.p, d.L, A.rad, A.rlo, B.rad, B.rlo, dd, dist);
    } else {
        dd = F::diff(A.p, B.p, d.L);
        R ss = radd(radd(rmul(dd.x, dd.x), rmul(dd.y, dd.y)), rmul(dd.z, dd.z));
        dist = sqrt(ss);
        delta = rsub(radd(A.rad, B.rad), dist);
    }
}

// The rest of a sphere pair's contact geometry and kinematics from its gap: normal, arms,
// contact-point velocities, effective radius and mass.
template <class F, bool PARAMS = true>
__device__ __forceinline__ void sphere_finish(const Dev<F> &d, const SphereK<F> &A, const SphereK<F> &B,
                                              V3<typename F::R> dd, typename F::R dist, typename F::R delta,
                                              ContactIn<typename F::R> &c, V3<typename F::R> &armA,
                                              V3<typename F::R> &armB)
{
    using R = typename F::R;
    R inv = R(1) / dist;
    c.n = {rmul(inv, dd.x), rmul(inv, dd.y), rmul(inv, dd.z)};
    c.delta = delta;
    const R half = rmul(R(0.5), delta);
    armA = arm_of(A.rl, -rsub(A.rad, half), c.n);
    armB = arm_of(B.rl, rsub(B.rad, half), c.n);
    c.uA = point_velocity(A.v, A.w, armA);
    c.uB = point_velocity(B.v, B.w, armB);
    c.Rbar = (A.rad * B.rad) / (A.rad + B.rad);
    c.mbar = (A.mass * B.mass) / (A.mass + B.mass);
    if constexpr (PARAMS) load_pair(d.pairs, d.pairs_f, d.mat_scene, d.mat_local, d.scenes, A.mat, B.mat, c);
}

template <class F, bool PARAMS = true, bool ANY = false>
__device__ __forceinline__ bool sphere_contact(const Dev<F> &d, const SphereK<F> &A, const SphereK<F> &B,
                                               ContactIn<typename F::R> &c, V3<typename F::R> &armA,
                                               V3<typename F::R> &armB)
{
    using R = typename F::R;
    V3<R> dd;
    R dist, delta;
    sphere_gap<F>(d, A, B, dd, dist, delta);
    if ((!ANY && !(delta > R(0))) || !(dist > R(0))) return false;
    R inv = R(1) / dist;
    c.n = {rmul(inv, dd.x), rmul(inv, dd.y), rmul(inv, dd.z)};
    c.delta = delta;
    const R half = rmul(R(0.5), delta);
    armA = arm_of(A.rl, -rsub(A.rad, half), c.n);
    armB = arm_of(B.rl, rsub(B.rad, half), c.n);
    c.uA = point_velocity(A.v, A.w, armA);
    c.uB = point_velocity(B.v, B.w, armB);
    c.Rbar = (A.rad * B.rad) / (A.rad + B.rad);
    c.mbar = (A.mass * B.mass) / (A.mass + B.mass);
    if constexpr (PARAMS) load_pair(d.pairs, d.pairs_f, d.mat_scene, d.mat_local, d.scenes, A.mat, B.mat, c);
    return true;
}

// Sphere-wall contact (B = wall of infinite radius and mass), geometry in FP64.  With
// PARAMS false the caller fills the material constants of c.
template <class F, bool PARAMS = true>
__device__ __forceinline__ bool wall_contact(const Dev<F> &d, const SphereK<F> &A, const Scene &sc, const Wall &w,
                                             ContactIn<typename F::R> &c, V3<typename F::R> &armA,
                                             V3<double> *point = nullptr)
{
    using R = typename F::R;
    if constexpr (F::voxel) {
        if (w.axis >= 0) {
            // an axis-aligned resting plane: the signed distance of the centre is
            // (voxel index - plane's) Lv (exact) plus the offset difference, kept in
            // float-float, so the overlap is exact to a few ulps without FP64
            const int a = w.axis;
            const int ci = a == 0 ? A.p.cx : (a == 1 ? A.p.cy : A.p.cz);
            const float oi = a == 0 ? A.p.x : (a == 1 ? A.p.y : A.p.z);
            float bh, bl, gh, gl;
            two_sum(oi, -w.ax_off, bh, bl);                      // exact offset difference
            two_sum(__fmul_rn((float)(ci - w.ax_c), d.L), bh, gh, gl);
            gl = __fadd_rn(gl, __fsub_rn(bl, w.ax_off_lo));
            gh = __fmul_rn(gh, w.ax_sign);
            gl = __fmul_rn(gl, w.ax_sign);
            const float delta = __fadd_rn(__fsub_rn(A.rad, gh), __fsub_rn(A.rlo, gl));
            if (!(delta > 0.0f)) return false;
            const float arm = __fsub_rn(A.rad, __fmul_rn(0.5f, delta));
            V3<float> n = {0.0f, 0.0f, 0.0f};
            if (a == 0) n.x = w.ax_sign; else if (a == 1) n.y = w.ax_sign; else n.z = w.ax_sign;
            c.n = n;
            c.delta = delta;
            armA = arm_of(A.rl, -arm, c.n);
            c.uA = point_velocity(A.v, A.w, armA);
            c.uB = {0.0f, 0.0f, 0.0f};
            c.Rbar = A.rad;
            c.mbar = A.mass;
            if constexpr (PARAMS) load_pair(d.pairs, d.pairs_f, d.mat_scene, d.mat_local, d.scenes, A.mat, w.mat, c);
            if (point) {
                // read-backs: the contact point in FP64 (the force above is the step's)
                const V3<double> pa = F::absolute(A.p, sc, d.Ld);
                const double ad = (double)arm;
                *point = {pa.x - ad * (double)n.x, pa.y - ad * (double)n.y, pa.z - ad * (double)n.z};
            }
            return true;
        }
    }
    if (w.type == WALL_PLANE) {
        const float3 pf = approx_pos<F>(A.p, sc, d.L);
        if (!plane_may_reach(w, pf, (float)A.rad, fabsf(pf.x) + fabsf(pf.y) + fabsf(pf.z) + 1.0f)) return false;
    }
    V3<double> pa = F::absolute(A.p, sc, d.Ld);
    double gap;
    V3<double> n;
    if (!wall_gap(w, pa, gap, n)) return false;
    const double Rd = (double)A.rad + (double)A.rlo;
    double delta = rsub(Rd, gap);
    if (!(delta > 0.0)) return false;
    double a = Rd - 0.5 * delta;
    V3<double> cp = {pa.x - a * n.x, pa.y - a * n.y, pa.z - a * n.z};
    V3<double> om = {w.omega[0], w.omega[1], w.omega[2]};
    V3<double> vw = cross(om, V3<double>{cp.x - w.p[0], cp.y - w.p[1], cp.z - w.p[2]});
    if (point) *point = cp;
    c.n = {(R)n.x, (R)n.y, (R)n.z};
    c.delta = (R)delta;
    armA = arm_of(A.rl, -(R)a, c.n);
    c.uA = point_velocity(A.v, A.w, armA);
    c.uB = {(R)vw.x, (R)vw.y, (R)vw.z};
    c.Rbar = A.rad;
    c.mbar = A.mass;
    if constexpr (PARAMS) load_pair(d.pairs, d.pairs_f, d.mat_scene, d.mat_local, d.scenes, A.mat, w.mat, c);
    return true;
}

// Position of `key` in a sorted ELL row (entries partner[k*Np + row], k < n); -1 if absent.
__device__ __forceinline__ int row_find(const uint32_t *partner, int64_t Np, int64_t row, int n, uint32_t key)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        uint32_t v = partner[(int64_t)mid * Np + row];
        if (v < key) lo = mid + 1;
        else hi = mid;
    }
    if (lo < n && partner[(int64_t)lo * Np + row] == key) return lo;
    return -1;
}

// ------------------------------------------------------------------ detection

// Snapshot of sphere centres and their cell keys (slot order).  Resets the displacement
// bound of the list being built: this is the snapshot time of that list.
template <class F, bool CLUMPS>
__global__ void __launch_bounds__(256) k_hash(Dev<F> d, DetectBuffers b, double beta)
{
    DevStatus *stp = d.status;
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (stp->halt) return;
    if (s == 0) {
        stp->disp_next = 0.0;
        stp->snap_step = stp->steps_done;  // mesh facets are binned at their pose of this step
        stp->cell_stamp += 1;            // a new cell table (the previous entries go stale)
        stp->beta_next = beta;
        stp->beta_next_f = (float)beta;
    }
    if (s >= d.N) return;
    const int sp = stp->state_par;
    uint32_t o = d.sph_owner[s];
    if (o != 0xffffffffu && d.sph_head[s]) {
        // the next list's bound starts at zero (the lane of the state the next step reads)
        typename F::R4 *lane = (stp->acc_par ^ 1) == 0 ? &d.st.kv[sp][2 * o] : &d.st.kv[sp][2 * o + 1];
        lane->w = typename F::R(0);
    }
    uint32_t key = b.n_cells_total;
    if (o != 0xffffffffu && d.st.active[sp][o]) {
        SphereK<F> k = load_sphere<F, CLUMPS>(d, sp, (uint32_t)s);
        const Scene &sc = d.scenes[d.owner_scene[o]];
        int cx, cy, cz;
        F::cell(k.p, sc, d.invL, d.vpc, cx, cy, cz);
        cx = min(max(cx, 0), sc.nc[0] - 1);
        cy = min(max(cy, 0), sc.nc[1] - 1);
        cz = min(max(cz, 0), sc.nc[2] - 1);
        key = sc.cell_base + (uint32_t)((cz * sc.nc[1] + cy) * sc.nc[0] + cx);
        if constexpr (F::voxel) {
            // voxel indices as floats (exact below 2^24): the listed predicate's
            // (float)(ia - ib) is then the exact difference fa - fb, with no conversions
            reinterpret_cast<float4 *>(b.snap)[s] = make_float4((float)k.p.cx, (float)k.p.cy, (float)k.p.cz, 0.0f);
            reinterpret_cast<float4 *>(b.snap_aux)[s] = make_float4(k.p.x, k.p.y, k.p.z, (float)k.rad);
        } else {
            reinterpret_cast<double4_32a *>(b.snap)[s] = make_double4_32a(k.p.x, k.p.y, k.p.z, (double)k.rad);
        }
    }
    b.keys[s] = key;
    if (!b.counting) b.vals[s] = (uint32_t)s;      // the counting sort scatters slots itself
}

// Cell table from the sorted keys (no clearing: an entry is valid only if it carries this
// build's stamp) and the snapshot gathered in cell order.
template <class F>
__global__ void __launch_bounds__(256) k_cellstart(Dev<F> d, DetectBuffers b, const uint32_t *keys,
                                                    const uint32_t *vals)
{
    if (d.status->halt) return;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.n) return;
    uint32_t k = keys[t];
    const uint32_t sent = b.n_cells_total;
    const uint32_t stamp = d.status->cell_stamp;
    if (k != sent) {
        // the first entry of a run writes (start, stamp), the last writes end: disjoint words
        if (t == 0 || keys[t - 1] != k) {
            reinterpret_cast<uint2 *>(&b.cell_tab[k])[0] = make_uint2((uint32_t)t, stamp);
            b.cell_tab[k].w = 0u;                 // no facet pairs until k_facet_cells says so
        }
        if (t == b.n - 1 || keys[t + 1] != k) b.cell_tab[k].z = (uint32_t)(t + 1);
        if (t == b.n - 1 || keys[t + 1] == sent) *b.n_valid = (uint32_t)(t + 1);
    } else if (t == 0) {
        *b.n_valid = 0;
    }
    uint32_t id = vals[t];
    if constexpr (F::voxel) {
        reinterpret_cast<int4 *>(b.sorted)[t] = reinterpret_cast<const int4 *>(b.snap)[id];
        reinterpret_cast<float4 *>(b.sorted_aux)[t] = reinterpret_cast<const float4 *>(b.snap_aux)[id];
    } else {
        reinterpret_cast<double4_32a *>(b.sorted)[t] = reinterpret_cast<const double4_32a *>(b.snap)[id];
    }
    b.sorted_owner[t] = d.sph_owner[id];
    if (d.owner_family) {
        const uint32_t o = d.sph_owner[id];
        b.sorted_family[t] = o != 0xffffffffu ? d.owner_family[o] : (uint8_t)0;
    }
}

// ---- counting sort of the snapshot by cell (the binning where cells are not much more
// numerous than spheres): each sphere takes its rank in its cell with an atomic, an
// exclusive scan of the per-cell counts gives each cell's start and writes the cell
// table, and each sphere is placed at start + rank.  The order within a cell is the
// order of the atomics; nothing downstream depends on it (the narrow phase tests each
// pair once whatever the order, and rows are sorted by partner).
constexpr int CS_THREADS = 256;
constexpr int CS_ITEMS = 16;
constexpr int CS_TILE = CS_THREADS * CS_ITEMS;

template <class F>
__global__ void __launch_bounds__(256) k_ccount(Dev<F> d, DetectBuffers b)
{
    if (d.status->halt) return;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.n) return;
    const uint32_t key = b.keys[s];
    if (key != b.n_cells_total) b.crank[s] = atomicAdd(&b.ccount[key], 1u);
}

// Sum of a block's value over the block (every thread gets it).
__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += wsum[k];
    __syncthreads();
    return t;
}

// Per tile of CS_TILE cells: the sum of the counts.
static __global__ void __launch_bounds__(CS_THREADS) k_cscan_reduce(const DevStatus *stp, const uint32_t *count,
                                                                     uint32_t *tile_sum)
{
    __shared__ uint32_t wsum[CS_THREADS / 32];
    if (stp->halt) return;
    const uint4 *c4 = reinterpret_cast<const uint4 *>(count + (int64_t)blockIdx.x * CS_TILE);
    uint32_t v = 0;
#pragma unroll
    for (int r = 0; r < CS_ITEMS / 4; ++r) {
        const uint4 q = c4[r * CS_THREADS + threadIdx.x];
        v += q.x + q.y + q.z + q.w;
    }
    v = block_sum_u32(v, wsum);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = v;
}

// Exclusive scan of the tile sums in place (one block, 1024-wide chunks with a carry);
// the total is the number of spheres in cells (the valid entries of the order).
static __global__ void __launch_bounds__(1024) k_cscan_tiles(const DevStatus *stp, uint32_t *tile_sum, int64_t n_tiles,
                                                             uint32_t *n_valid)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    if (stp->halt) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n_tiles; base += 1024) {
        const int64_t i = base + t;
        const uint32_t v = i < n_tiles ? tile_sum[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const uint32_t incl = x + (warp > 0 ? wsum[warp - 1] : 0u) + carry;
        if (i < n_tiles) tile_sum[i] = incl - v;
        __syncthreads();
        if (t == 1023) carry = incl;
        __syncthreads();
    }
    if (t == 0) *n_valid = carry;
}

// Per tile: each thread takes CS_ITEMS consecutive cells, the block scans the threads'
// sums, and every cell with spheres gets its table entry (start, stamp, end).
template <class F>
__global__ void __launch_bounds__(CS_THREADS) k_cscan_write(Dev<F> d, DetectBuffers b, const uint32_t *tile_start)
{
    __shared__ uint32_t wsum[CS_THREADS / 32];
    const DevStatus *stp = d.status;
    if (stp->halt) return;
    const uint32_t stamp = stp->cell_stamp;
    const int64_t c0 = (int64_t)blockIdx.x * CS_TILE + (int64_t)threadIdx.x * CS_ITEMS;
    const uint4 *c4 = reinterpret_cast<const uint4 *>(b.ccount + c0);
    uint32_t cnt[CS_ITEMS];
#pragma unroll
    for (int r = 0; r < CS_ITEMS / 4; ++r) {
        const uint4 q = c4[r];
        cnt[4 * r] = q.x; cnt[4 * r + 1] = q.y; cnt[4 * r + 2] = q.z; cnt[4 * r + 3] = q.w;
    }
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < CS_ITEMS; ++k) mine += cnt[k];
    // exclusive scan of the threads' sums over the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int k = 0; k < warp; ++k) before += wsum[k];
    uint32_t start = tile_start[blockIdx.x] + before + x - mine;
#pragma unroll
    for (int k = 0; k < CS_ITEMS; ++k) {
        if (cnt[k]) b.cell_tab[c0 + k] = make_uint4(start, stamp, start + cnt[k], 0u);
        start += cnt[k];
    }
}

// Each sphere of a cell to its place in the order, with its key, slot, snapshot, owner and
// family (what the radix path's sort and k_cellstart produce).
template <class F>
__global__ void __launch_bounds__(256) k_cscatter(Dev<F> d, DetectBuffers b, uint32_t *keys_out, uint32_t *vals_out)
{
    if (d.status->halt) return;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.n) return;
    const uint32_t key = b.keys[s];
    if (key == b.n_cells_total) return;
    const uint32_t pos = b.cell_tab[key].x + b.crank[s];
    keys_out[pos] = key;
    vals_out[pos] = (uint32_t)s;
    if constexpr (F::voxel) {
        reinterpret_cast<int4 *>(b.sorted)[pos] = reinterpret_cast<const int4 *>(b.snap)[s];
        reinterpret_cast<float4 *>(b.sorted_aux)[pos] = reinterpret_cast<const float4 *>(b.snap_aux)[s];
    } else {
        reinterpret_cast<double4_32a *>(b.sorted)[pos] = reinterpret_cast<const double4_32a *>(b.snap)[s];
    }
    const uint32_t o = d.sph_owner[s];
    b.sorted_owner[pos] = o;
    if (d.owner_family) b.sorted_family[pos] = o != 0xffffffffu ? d.owner_family[o] : (uint8_t)0;
}

// Listed-pair predicate on snapshot entries: squared distance below
// ((Ri + Rj) + 2 beta)^2, rounded in a fixed order (FP64 or voxel + FP32).
__device__ __forceinline__ bool listed_f64(double4_32a a, double4_32a b, double b2)
{
    double dx = rsub(a.x, b.x), dy = rsub(a.y, b.y), dz = rsub(a.z, b.z);
    double s = radd(radd(rmul(dx, dx), rmul(dy, dy)), rmul(dz, dz));
    double t = radd(radd(a.w, b.w), b2);
    return s < rmul(t, t);
}
// ca, cb: voxel indices held as floats (integers below 2^21 in magnitude, so their float
// difference is exactly the converted integer difference)
__device__ __forceinline__ bool listed_f32(float4 ca, float4 oa, float4 cb, float4 ob, float L, float b2)
{
    float dx = radd(rmul(rsub(ca.x, cb.x), L), rsub(oa.x, ob.x));
    float dy = radd(rmul(rsub(ca.y, cb.y), L), rsub(oa.y, ob.y));
    float dz = radd(rmul(rsub(ca.z, cb.z), L), rsub(oa.z, ob.z));
    float s = radd(radd(rmul(dx, dx), rmul(dy, dy)), rmul(dz, dz));
    float t = radd(radd(oa.w, ob.w), b2);
    return s < rmul(t, t);
}

__device__ __forceinline__ void row_insert(uint32_t *buf, int &n, uint32_t e)
{
    if (n < KMAX) {
        int pos = n;
        while (pos > 0 && buf[pos - 1] > e) {
            buf[pos] = buf[pos - 1];
            --pos;
        }
        buf[pos] = e;
    }
    ++n;
}

// Vertices of facet w at time t: p + R(omega t)(v - p) (Rodrigues' rotation about the unit
// axis omega / |omega| by |omega| t), every operation rounded on its own in that order.
__device__ __forceinline__ void facet_pose(const Wall &w, double t, double *v)
{
    const V3<double> om = {w.omega[0], w.omega[1], w.omega[2]};
    const double wn = __dsqrt_rn(radd(radd(rmul(om.x, om.x), rmul(om.y, om.y)), rmul(om.z, om.z)));
    if (!(wn > 0.0)) {
        for (int q = 0; q < 9; ++q) v[q] = w.tri[q];
        return;
    }
    const V3<double> k = {__ddiv_rn(om.x, wn), __ddiv_rn(om.y, wn), __ddiv_rn(om.z, wn)};
    const double th = rmul(wn, t);
    // the lanes turning by the same angle (the facets of one mesh) share one FP64
    // sine and cosine, computed by the first of them: the same values, far fewer FP64
    // instructions on a part where they are scarce
    const unsigned grp = __match_any_sync(__activemask(), (unsigned long long)__double_as_longlong(th));
    const int leader = __ffs(grp) - 1;
    double sn = 0.0, cs = 0.0;
    if ((int)(threadIdx.x & 31) == leader) sincos(th, &sn, &cs);
    sn = __shfl_sync(grp, sn, leader);
    cs = __shfl_sync(grp, cs, leader);
    const double omc = rsub(1.0, cs);
    for (int m = 0; m < 3; ++m) {
        const V3<double> r = {rsub(w.tri[3 * m], w.p[0]), rsub(w.tri[3 * m + 1], w.p[1]), rsub(w.tri[3 * m + 2], w.p[2])};
        const V3<double> kxr = {rsub(rmul(k.y, r.z), rmul(k.z, r.y)), rsub(rmul(k.z, r.x), rmul(k.x, r.z)),
                                rsub(rmul(k.x, r.y), rmul(k.y, r.x))};
        const double kr = radd(radd(rmul(k.x, r.x), rmul(k.y, r.y)), rmul(k.z, r.z));
        const double f = rmul(kr, omc);
        v[3 * m + 0] = radd(w.p[0], radd(radd(rmul(r.x, cs), rmul(kxr.x, sn)), rmul(k.x, f)));
        v[3 * m + 1] = radd(w.p[1], radd(radd(rmul(r.y, cs), rmul(kxr.y, sn)), rmul(k.y, f)));
        v[3 * m + 2] = radd(w.p[2], radd(radd(rmul(r.z, cs), rmul(kxr.z, sn)), rmul(k.z, f)));
    }
}

// Current pose of every facet (the step's time, steps_done * h); runs after each step.
template <class F>
__global__ void __launch_bounds__(128) k_facet_pose(Dev<F> d, Wall *walls, const int *facet_wall, int n_facets)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_facets) return;
    Wall &w = walls[facet_wall[f]];
    const double t = rmul((double)d.status->steps_done, d.scenes[w.scene].h);
    facet_pose(w, t, w.cur);
}

// Squared distance from p to the triangle (0, u, w) in FP32 (the region tests of the
// closest-point-on-triangle algorithm); only used to decide, with an allowance, which
// cells a facet is binned into.
__device__ __forceinline__ float tri_dist2_f(float3 p, float3 u, float3 w)
{
    auto dt = [](float3 x, float3 y) { return x.x * y.x + x.y * y.y + x.z * y.z; };
    auto sub = [](float3 x, float3 y) { return make_float3(x.x - y.x, x.y - y.y, x.z - y.z); };
    float3 q;
    const float d1 = dt(u, p), d2 = dt(w, p);
    const float3 bp = sub(p, u), cp = sub(p, w);
    const float d3 = dt(u, bp), d4 = dt(w, bp), d5 = dt(u, cp), d6 = dt(w, cp);
    const float vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
    if (d1 <= 0.0f && d2 <= 0.0f) {
        q = make_float3(0.0f, 0.0f, 0.0f);
    } else if (d3 >= 0.0f && d4 <= d3) {
        q = u;
    } else if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
        const float t = d1 / (d1 - d3);
        q = make_float3(t * u.x, t * u.y, t * u.z);
    } else if (d6 >= 0.0f && d5 <= d6) {
        q = w;
    } else if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
        const float t = d2 / (d2 - d6);
        q = make_float3(t * w.x, t * w.y, t * w.z);
    } else if (va <= 0.0f && (d4 - d3) >= 0.0f && (d5 - d6) >= 0.0f) {
        const float t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        q = make_float3(u.x + t * (w.x - u.x), u.y + t * (w.y - u.y), u.z + t * (w.z - u.z));
    } else {
        const float den = 1.0f / (va + vb + vc);
        const float v = vb * den, ww = vc * den;
        q = make_float3(v * u.x + ww * w.x, v * u.y + ww * w.y, v * u.z + ww * w.z);
    }
    const float3 e = sub(p, q);
    return dt(e, e);
}

// Bin every facet, at its pose of the snapshot step, into the cells whose centre lies
// within rr = largest radius + margin + half a cell diagonal of it (a sphere centred in
// the cell within R + margin of the facet implies that): pairs (cell key, facet) from the
// facet's first slot, the unused slots of its share keyed past every cell.  One warp per
// facet walks the facet's bounding box (grown by rr): a plane test, then the distance to
// the triangle, in FP32 relative to the facet's first vertex with an allowance.  A share
// holds every such cell (its size bounds the volume of the facet's neighbourhood, see
// setup_facets); should it not, the step halts (HALT_FACETS) rather than lose a contact.
template <class F>
__global__ void __launch_bounds__(128) k_facet_bin(Dev<F> d, DetectBuffers b, double r_max)
{
    const int f = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (f >= b.n_facets || d.status->halt) return;       // whole warps
    const Wall &w = d.walls[b.facet_wall[f]];
    const Scene &sc = d.scenes[w.scene];
    double v[9];
    facet_pose(w, rmul((double)d.status->snap_step, sc.h), v);
    if (lane < 9) b.tri_snap[9 * (int64_t)f + lane] = v[lane];
    const double cell = 1.0 / d.invL;
    const double rr = r_max + d.status->beta_next + 0.8660254037844387 * cell;
    int lo[3], n[3];
    for (int a = 0; a < 3; ++a) {
        const double mn = fmin(fmin(v[a], v[3 + a]), v[6 + a]) - rr;
        const double mx = fmax(fmax(v[a], v[3 + a]), v[6 + a]) + rr;
        int l = (int)floor((mn - sc.lo[a]) * d.invL), h = (int)floor((mx - sc.lo[a]) * d.invL);
        l = min(max(l, 0), sc.nc[a] - 1);
        h = min(max(h, 0), sc.nc[a] - 1);
        lo[a] = l;
        n[a] = h - l + 1;
    }
    const float3 u = make_float3((float)(v[3] - v[0]), (float)(v[4] - v[1]), (float)(v[5] - v[2]));
    const float3 ww = make_float3((float)(v[6] - v[0]), (float)(v[7] - v[1]), (float)(v[8] - v[2]));
    float3 nrm = make_float3(u.y * ww.z - u.z * ww.y, u.z * ww.x - u.x * ww.z, u.x * ww.y - u.y * ww.x);
    const float nl = sqrtf(nrm.x * nrm.x + nrm.y * nrm.y + nrm.z * nrm.z);
    nrm = make_float3(nrm.x / nl, nrm.y / nl, nrm.z / nl);
    const float ext = fmaxf(fmaxf(fabsf(u.x) + fabsf(u.y) + fabsf(u.z), fabsf(ww.x) + fabsf(ww.y) + fabsf(ww.z)),
                            (float)(rr + cell));
    const float lim = (float)rr + 1e-5f * ext + 1e-9f;       // rr plus the FP32 allowance
    const int64_t base = b.facet_off[f], end = b.facet_off[f + 1];
    const int64_t total = (int64_t)n[0] * n[1] * n[2];
    int64_t count = 0;                                        // the same in every lane
    for (int64_t k0 = 0; k0 < total; k0 += 32) {
        const int64_t k = k0 + lane;
        bool hit = false;
        uint32_t key = 0;
        if (k < total) {
            const int x = lo[0] + (int)(k % n[0]), y = lo[1] + (int)((k / n[0]) % n[1]),
                      z = lo[2] + (int)(k / ((int64_t)n[0] * n[1]));
            const float3 p = make_float3((float)(sc.lo[0] + (x + 0.5) * cell - v[0]),
                                         (float)(sc.lo[1] + (y + 0.5) * cell - v[1]),
                                         (float)(sc.lo[2] + (z + 0.5) * cell - v[2]));
            const float pd = p.x * nrm.x + p.y * nrm.y + p.z * nrm.z;
            if (fabsf(pd) <= lim && tri_dist2_f(p, u, ww) <= lim * lim) {
                hit = true;
                key = sc.cell_base + (uint32_t)((z * sc.nc[1] + y) * sc.nc[0] + x);
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, hit);
        const int64_t pos = base + count + __popc(ball & ((1u << lane) - 1u));
        if (hit && pos < end) {
            b.fkeys[pos] = key;
            b.fvals[pos] = (uint32_t)f;
        }
        count += __popc(ball);
    }
    if (base + count > end && lane == 0) atomicCAS(&d.status->halt, HALT_NONE, HALT_FACETS);
    for (int64_t q = base + count + lane; q < end; q += 32) {
        b.fkeys[q] = b.n_cells_total;
        b.fvals[q] = (uint32_t)f;
    }
}

// After the facet pairs are sorted by cell: the first pair of each cell's run, plus one,
// into the fourth word of the cell's table entry (the binning wrote that word zero in
// every cell holding spheres; cells without spheres are never looked up).
static __global__ void __launch_bounds__(256) k_facet_cells(const DevStatus *stp, DetectBuffers b)
{
    if (stp->halt) return;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= b.n_fpairs) return;
    const uint32_t key = b.fkeys_sorted[q];
    if (key >= b.n_cells_total) return;
    if (q == 0 || b.fkeys_sorted[q - 1] != key) b.cell_tab[key].w = (uint32_t)(q + 1);
}

// Per cell: 1 if a wall of its scene (facets excepted: they are binned) may be within
// reach_max = largest radius + largest margin of a sphere centred anywhere in the cell.
// Plane and cylinder gaps are 1-Lipschitz signed distances, so a cell whose FP64 gap at
// the centre, less half its diagonal, exceeds reach_max by a rounding allowance is out of
// every listed sphere's reach; cones and the cells on the grid's boundary (where centres
// outside the grid are clamped) are always flagged.
template <class F>
__global__ void __launch_bounds__(256) k_cell_walls(Dev<F> d, DetectBuffers b, double cell, double reach_max)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (int64_t)b.n_cells_total) return;
    int lo = 0, hi = d.n_scenes - 1;     // the scene whose cells hold c: last base <= c
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)d.scenes[mid].cell_base <= c) lo = mid;
        else hi = mid - 1;
    }
    const Scene &sc = d.scenes[lo];
    const uint32_t local = (uint32_t)(c - (int64_t)sc.cell_base);
    const int nx = sc.nc[0], ny = sc.nc[1], nz = sc.nc[2];
    const int cx = (int)(local % (uint32_t)nx), cy = (int)((local / (uint32_t)nx) % (uint32_t)ny),
              cz = (int)(local / (uint32_t)(nx * ny));
    uint8_t near = 0;
    if (cx == 0 || cy == 0 || cz == 0 || cx == nx - 1 || cy == ny - 1 || cz == nz - 1) near = 1;
    const V3<double> ctr = {sc.lo[0] + (cx + 0.5) * cell, sc.lo[1] + (cy + 0.5) * cell, sc.lo[2] + (cz + 0.5) * cell};
    const double half_diag = 0.8660254037844387 * cell * (1.0 + 1e-6);
    const double allow = 1e-9 * (fabs(ctr.x) + fabs(ctr.y) + fabs(ctr.z) + 1.0) + 1e-12;
    for (int wi = 0; wi < sc.wall_count && !near; ++wi) {
        const Wall &wl = d.walls[sc.wall_begin + wi];
        if (wl.type != WALL_PLANE && wl.type != WALL_CYLINDER) {
            near = 1;
            break;
        }
        double gap;
        V3<double> nn;
        wall_gap(wl, ctr, gap, nn);
        if (!(gap - half_diag > reach_max + allow)) near = 1;
    }
    b.cell_wall[c] = near;
}

// Narrow phase, first pass: one thread per sorted entry t tests the candidates after it
// in the sorted order within its 27 neighbour cells (the half shell: the rest of its own
// x-run of three cells, from t + 1, and the four full x-runs of cells with larger keys,
// each run contiguous in the sorted order), so each pair is tested once, by its first
// entry.  A listed pair is appended to both rows of the list that is not in use, at
// slots reserved by per-row atomic counters (b.rowcnt, zeroed before the pass); the
// thread also appends its sphere's walls and facets.  The listed predicate is symmetric
// in its two spheres, so the rows hold what each sphere's own full scan would list; the
// second pass (k_rows_finish) sorts them.
constexpr int NS_THREADS = 256;     // block of the staged narrow phase
constexpr int NS_CAP = 2048;        // snapshot entries a block stages in shared memory

// STAGED: the block of NS_THREADS sorted entries first reduces its threads' candidate runs
// to five ranges of the sorted order (one per run of the half shell: each the union of
// its threads' runs, contiguous since cells are ordered z-major) and copies them into
// shared memory, records, slots, owners and families; the candidate tests then read
// shared memory instead of L1/L2.  A block whose ranges exceed NS_CAP entries reads
// global memory as the plain kernel does.  The same tests in the same order: the same
// rows.
template <class F, bool CLUMPS, bool STAGED = false>
__global__ void __launch_bounds__(256, STAGED ? 2 : 4) k_narrow(Dev<F> d, DetectBuffers b, const uint32_t *keys,
                                                               const uint32_t *vals)
{
    DevStatus *stp = d.status;
    if (stp->halt) return;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nvalid = *b.n_valid;
    const bool live = t < nvalid;
    if (!STAGED && !live) return;
    const uint32_t stamp = stp->cell_stamp;
    const int ln = stp->list_cur ^ 1;
    const double beta = stp->beta_next;
    const float betaf = stp->beta_next_f;
    // entries past the valid ones (staged blocks only) take part in the staging alone
    const uint32_t i = live ? vals[t] : 0u;
    const uint32_t key = live ? keys[t] : 0u;
    const uint32_t oi = live ? b.sorted_owner[t] : 0u;
    const Scene &sc = d.scenes[live ? d.owner_scene[oi] : 0];
    // families: candidates of a family whose contacts with this one are masked are skipped
    const bool fam = d.owner_family != nullptr;
    const int fi = (fam && live) ? (int)b.sorted_family[t] : 0;
    const uint32_t local = key - sc.cell_base;
    const int nx = sc.nc[0], ny = sc.nc[1], nz = sc.nc[2];
    const int cx = (int)(local % (uint32_t)nx);
    const int cy = (int)((local / (uint32_t)nx) % (uint32_t)ny);
    const int cz = (int)(local / (uint32_t)(nx * ny));

    double4_32a a64 = make_double4_32a(0, 0, 0, 0);
    float4 acf = make_float4(0, 0, 0, 0);
    int4 ac = make_int4(0, 0, 0, 0);
    float4 ao = make_float4(0, 0, 0, 0);
    if (live) {
        if constexpr (F::voxel) {
            acf = reinterpret_cast<const float4 *>(b.sorted)[t];
            ac = make_int4((int)acf.x, (int)acf.y, (int)acf.z, 0);
            ao = reinterpret_cast<const float4 *>(b.sorted_aux)[t];
        } else {
            a64 = reinterpret_cast<const double4_32a *>(b.sorted)[t];
        }
    }
    const float b2f = 2.0f * betaf;
    const double b2d = 2.0 * beta;

    // append e to the row of slot r (entries beyond K are counted, not stored: the second
    // pass reports the overflow)
    const uint32_t K = (uint32_t)d.K;
    uint32_t *prow = d.lists.partner[ln];
    uint32_t *rc = b.rowcnt;
    auto put = [&](uint32_t r, uint32_t e) {
        const uint32_t pos = atomicAdd(&rc[r], 1u);
        if (pos < K) prow[(int64_t)pos * d.Np + r] = e;
    };
    const int x0 = max(cx - 1, 0), x1 = min(cx + 1, nx - 1);
    uint32_t own_facets = 0;     // the own cell's first (cell, facet) pair + 1, 0 for none
    // runs (dz, dy): (0, 0) from t + 1, then (0, +1), (+1, -1), (+1, 0), (+1, +1); an
    // empty run has rlo = rhi
    uint32_t rlo[5], rhi[5];
#pragma unroll
    for (int run = 0; run < 5; ++run) {
        rlo[run] = 0u;
        rhi[run] = 0u;
        const int dz = run < 2 ? 0 : 1;
        const int dy = run == 0 ? 0 : (run == 1 ? 1 : run - 3);
        const int z = cz + dz, y = cy + dy;
        if (!live || z >= nz || y < 0 || y >= ny) continue;
        const uint32_t rowbase = sc.cell_base + (uint32_t)((z * ny + y) * nx);
        uint32_t lo = 0xffffffffu, hi = 0;
        for (int x = x0; x <= x1; ++x) {
            const uint4 r = b.cell_tab[rowbase + (uint32_t)x];
            if (r.y == stamp) {
                if (lo == 0xffffffffu) lo = r.x;
                hi = r.z;
            }
            if (run == 0 && x == cx) own_facets = r.w;
        }
        if (lo == 0xffffffffu) continue;
        // the own run holds this entry's cell: only the entries after it
        if (run == 0) lo = (uint32_t)t + 1u;
        if (lo < hi) {
            rlo[run] = lo;
            rhi[run] = hi;
        }
    }
    // staging (STAGED): five ranges of the sorted order into shared memory
    extern __shared__ __align__(32) unsigned char ns_mem[];
    __shared__ uint32_t seg_lo[5], seg_hi[5], seg_base[5];
    __shared__ int seg_ok;
    bool staged = false;
    if constexpr (STAGED) {
        if (threadIdx.x < 5) {
            seg_lo[threadIdx.x] = 0xffffffffu;
            seg_hi[threadIdx.x] = 0u;
        }
        __syncthreads();
#pragma unroll
        for (int run = 0; run < 5; ++run)
            if (rlo[run] < rhi[run]) {
                atomicMin(&seg_lo[run], rlo[run]);
                atomicMax(&seg_hi[run], rhi[run]);
            }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int r = 0; r < 5; ++r) {
                if (seg_hi[r] <= seg_lo[r] || seg_lo[r] == 0xffffffffu) {
                    seg_lo[r] = 0u;
                    seg_hi[r] = 0u;
                }
                seg_base[r] = tot;
                tot += seg_hi[r] - seg_lo[r];
            }
            seg_ok = tot <= (uint32_t)NS_CAP ? 1 : 0;
        }
        __syncthreads();
        staged = seg_ok != 0;
        if (staged) {
            float4 *srec = reinterpret_cast<float4 *>(ns_mem);
            uint32_t *sval = reinterpret_cast<uint32_t *>(ns_mem + 32 * NS_CAP);
            uint32_t *sown = sval + NS_CAP;
            uint8_t *sfam = reinterpret_cast<uint8_t *>(sown + NS_CAP);
            for (int r = 0; r < 5; ++r) {
                const uint32_t lo = seg_lo[r], sz = seg_hi[r] - lo, base = seg_base[r];
                for (uint32_t q = threadIdx.x; q < sz; q += blockDim.x) {
                    const uint32_t src = lo + q, dst = base + q;
                    if constexpr (F::voxel) {
                        srec[2 * dst] = reinterpret_cast<const float4 *>(b.sorted)[src];
                        srec[2 * dst + 1] = reinterpret_cast<const float4 *>(b.sorted_aux)[src];
                    } else {
                        srec[2 * dst] = reinterpret_cast<const float4 *>(b.sorted)[2 * (int64_t)src];
                        srec[2 * dst + 1] = reinterpret_cast<const float4 *>(b.sorted)[2 * (int64_t)src + 1];
                    }
                    sval[dst] = vals[src];
                    if (CLUMPS) sown[dst] = b.sorted_owner[src];
                    if (fam) sfam[dst] = b.sorted_family[src];
                }
            }
        }
        __syncthreads();
    }
    if (!live) return;
    const float4 *srec = reinterpret_cast<const float4 *>(ns_mem);
    const uint32_t *sval = reinterpret_cast<const uint32_t *>(ns_mem + 32 * NS_CAP);
    const uint32_t *sown = sval + NS_CAP;
    const uint8_t *sfam = reinterpret_cast<const uint8_t *>(sown + NS_CAP);
#pragma unroll 1
    for (int run = 0; run < 5; ++run) {
        const uint32_t lo = rlo[run], hi = rhi[run];
        if (lo >= hi) continue;
        // the offset from a sorted position to its staged slot
        const int64_t off = staged ? (int64_t)seg_base[run] - (int64_t)seg_lo[run] : 0;
        for (uint32_t u = lo; u < hi; ++u) {
            const int64_t su = (int64_t)u + off;
            if (CLUMPS && (staged ? sown[su] : b.sorted_owner[u]) == oi) continue;
            if (fam && !families_meet(d.fam_mask, fi, staged ? sfam[su] : b.sorted_family[u])) continue;
            bool hit;
            if constexpr (F::voxel) {
                const float4 c0 = staged ? srec[2 * su] : reinterpret_cast<const float4 *>(b.sorted)[u];
                const float4 c1 = staged ? srec[2 * su + 1] : reinterpret_cast<const float4 *>(b.sorted_aux)[u];
                hit = listed_f32(acf, ao, c0, c1, d.L, b2f);
            } else {
                const double4_32a c = staged ? reinterpret_cast<const double4_32a *>(srec)[su]
                                             : reinterpret_cast<const double4_32a *>(b.sorted)[u];
                hit = listed_f64(a64, c, b2d);
            }
            if (hit) {
                const uint32_t j = staged ? sval[su] : vals[u];
                put(i, j);
                put(j, i);
            }
        }
    }
    // mesh facets binned into this cell: distance from the centre below R + beta (FP64, at
    // the facets' pose of the snapshot)
    if (b.n_facets > 0 && own_facets) {
        const uint32_t *fk = b.fkeys_sorted;
        const int64_t lo = (int64_t)own_facets - 1;      // k_facet_cells: the cell's first pair
        {
            V3<double> pa;
            double Rs;
            if constexpr (F::voxel) {
                pa = F::absolute(PosF32{ac.x, ac.y, ac.z, ao.x, ao.y, ao.z}, sc, d.Ld);
                Rs = (double)ao.w;
            } else {
                pa = {a64.x, a64.y, a64.z};
                Rs = a64.w;
            }
            for (int64_t q = lo; q < b.n_fpairs && fk[q] == key; ++q) {
                const uint32_t f = b.fvals_sorted[q];
                const double *v = b.tri_snap + 9 * (int64_t)f;
                const V3<double> c = closest_on_triangle(pa, V3<double>{v[0], v[1], v[2]}, V3<double>{v[3], v[4], v[5]},
                                                         V3<double>{v[6], v[7], v[8]});
                const V3<double> e = {rsub(pa.x, c.x), rsub(pa.y, c.y), rsub(pa.z, c.z)};
                const double dist = __dsqrt_rn(radd(radd(rmul(e.x, e.x), rmul(e.y, e.y)), rmul(e.z, e.z)));
                if (dist < Rs + beta) put(i, WALL_BIT | (uint32_t)b.facet_wall[f]);
            }
        }
    }
    // walls: signed gap below R + beta (FP64).  An FP32 gap decides every wall that is
    // clear of the threshold by more than its error bound; only the thin band around the
    // threshold takes the FP64 test (FP64 throughput is scarce on this part).  Cells that
    // no wall can reach from any point inside skip the loop (b.cell_wall).
    if (sc.wall_count > 0 && b.cell_wall[key]) {
        float Rf;
        double R;
        typename F::Pos pp;
        if constexpr (F::voxel) {
            pp = PosF32{ac.x, ac.y, ac.z, ao.x, ao.y, ao.z};
            Rf = ao.w;
        } else {
            pp = PosF64{a64.x, a64.y, a64.z};
            Rf = (float)a64.w;
        }
        const float3 pf = approx_pos<F>(pp, sc, d.L);
        const float reach = Rf + betaf;
        bool have64 = false;
        V3<double> pa;
        for (int wi = 0; wi < sc.wall_count; ++wi) {
            const int wg = sc.wall_begin + wi;
            const Wall &wl = d.walls[wg];
            const float gf = wall_gap_f(wl, pf);
            const float tol = wall_gap_tol(wl, pf) + 1e-6f * reach;
            if (gf > reach + tol) continue;
            if (gf < reach - tol) {
                put(i, WALL_BIT | (uint32_t)wg);
                continue;
            }
            if (!have64) {
                pa = F::absolute(pp, sc, d.Ld);
                if constexpr (F::voxel) R = (double)ao.w;
                else R = a64.w;
                have64 = true;
            }
            double gap;
            V3<double> nn;
            wall_gap(wl, pa, gap, nn);
            if (gap < R + beta) put(i, WALL_BIT | (uint32_t)wg);
        }
    }
}

// Narrow phase, second pass: one thread per slot sorts its row of the new list by
// partner (spheres by id, then walls: their ids carry the top bit) and writes its length;
// a row longer than K stops the step for a larger K, as a full scan would.  Slots that
// are inactive or padding get empty rows.
// Single spheres: the number of rows with entries in each block of 256 slots goes to
// bcount[block] (the blocks of the compaction), for the scan that orders the compacted work.
template <class F>
__global__ void __launch_bounds__(256) k_rows_finish(Dev<F> d, DetectBuffers b, uint32_t *bcount)
{
    __shared__ uint32_t wsum[8];
    DevStatus *stp = d.status;
    if (stp->halt) return;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s < d.Np;               // every thread stays for the block sum
    const int ln = stp->list_cur ^ 1;
    const int K = d.K;
    int n = live ? (int)min(b.rowcnt[s], 0x7fffffffu) : 0;
    const int mx = (int)__reduce_max_sync(0xffffffffu, (unsigned)n);
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(&stp->max_row, mx);
    if (n > K) {
        stp->overflow = 1;
        stp->halt = HALT_OVERFLOW;
        n = K;
    }
    uint32_t *prow = d.lists.partner[ln];
    if (n > 1) {
        uint32_t buf[KMAX];
        int m = 0;
        for (int k = 0; k < n; ++k) row_insert(buf, m, prow[(int64_t)k * d.Np + s]);
        for (int k = 0; k < n; ++k) prow[(int64_t)k * d.Np + s] = buf[k];
    }
    if (live) d.lists.cnt[ln][s] = (uint8_t)n;
    const uint32_t busy = block_sum_u32((live && s < d.N && n > 0) ? 1u : 0u, wsum);
    if (threadIdx.x == 0) bcount[blockIdx.x] = busy;
}

// The row counters of the list being built start at zero.
template <class F>
__global__ void __launch_bounds__(256) k_clear_rows(Dev<F> d, DetectBuffers b)
{
    DevStatus *stp = d.status;
    if (stp->halt) return;
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.Np) return;
    b.rowcnt[s] = 0u;
}

// Reset the work counter of the new list (which = 0) or of the list in use (which = 1).
// pairs_only: the compacted work of the new list was built on the detection stream (its
// count and busy slots are set); only its pair count starts again.
template <class F>
__global__ void k_act_reset(Dev<F> d, int which, int pairs_only = 0)
{
    const int l = d.status->list_cur ^ (which ? 0 : 1);
    if (!pairs_only) {
        *d.lists.n_act[l] = 0;
        d.status->list_busy[l] = 0;
    }
    if (!which) d.status->list_pairs[l] = 0;
}

// Flags any non-finite value of a[0, count).
static __global__ void __launch_bounds__(256) k_nonfinite(const double *a, int64_t count, int *bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count && !isfinite(a[i])) *bad = 1;
}

// Compact the work of a list: slots with a non-empty row (single spheres) or 32-slot
// groups with any (clumps: the segmented reduction needs whole warps).  Single spheres
// (phase 1) keep each block of 256 consecutive slots together, ordered by row length
// within the block (a shared-memory counting sort): the contact kernel's warps then take
// neighbouring spheres (shared memory sectors) with rows of equal length (no lanes idle
// through longer rows).  The order of equal lengths and of the blocks depends on
// scheduling; results do not (every slot's outputs are its own).
// Single spheres, before phase 1: the busy slots of each block of 256 (bcount[block]); a
// scan of bcount then gives each block its offset, so the compacted work lists the blocks
// in slot order (the contact kernel's concurrent threads then cover a narrow window of
// slots, whose partners' records stay in L2).  For a new list k_rows_finish counts them.
template <class F>
__global__ void __launch_bounds__(256) k_compact_count(Dev<F> d, int which, uint32_t *bcount)
{
    __shared__ uint32_t wsum[8];
    DevStatus *stp = d.status;
    if (stp->halt) return;
    const int l = stp->list_cur ^ (which ? 0 : 1);
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool busy = s < d.N && d.lists.cnt[l][s] > 0;
    const uint32_t tot = block_sum_u32(busy ? 1u : 0u, wsum);
    if (threadIdx.x == 0) bcount[blockIdx.x] = tot;
}

template <class F>
__global__ void __launch_bounds__(256) k_compact(Dev<F> d, int which, int phase, const uint32_t *bstart,
                                                 int64_t nblocks)
{
    const int warp_level = phase == 0;
    DevStatus *stp = d.status;
    if (stp->halt) return;
    const int l = stp->list_cur ^ (which ? 0 : 1);
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int nrow = s < d.N ? d.lists.cnt[l][s] : 0;
    const bool busy = nrow > 0;
    const unsigned int ball = __ballot_sync(0xffffffffu, busy);
    if (phase == 0 && lane == 0 && ball) atomicAdd(&stp->list_busy[l], (unsigned int)__popc(ball));
    if (phase == 1) {
        __shared__ unsigned int bins[KMAX + 1];
        __shared__ unsigned int all[KMAX + 1];
        __shared__ unsigned int block_base;
        for (int k = threadIdx.x; k <= KMAX; k += blockDim.x) bins[k] = all[k] = 0;
        __syncthreads();
        if (busy) atomicAdd(&bins[nrow], 1u);
        if (s < d.Np) atomicAdd(&all[nrow], 1u);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int run = 0, run_all = 0;
            for (int k = 0; k <= KMAX; ++k) {
                const unsigned int c = bins[k], ca = all[k];
                bins[k] = run;
                all[k] = run_all;
                run += c;
                run_all += ca;
            }
            // the block's offset from the scan of the per-block counts (total last)
            block_base = bstart[blockIdx.x];
            if (blockIdx.x == 0) {
                *d.lists.n_act[l] = bstart[nblocks];
                stp->list_busy[l] = bstart[nblocks];
            }
        }
        __syncthreads();
        // every slot of the block (empty rows first) by row length, for the fused step
        // (the block is 256 slots: the position fits a byte)
        if (s < d.Np) d.lists.perm[l][(s & ~(int64_t)255) + atomicAdd(&all[nrow], 1u)] = (uint8_t)(s & 255);
        if (busy) {
            // the first partner travels with the entry: the contact kernel starts on that
            // pair without waiting for the row
            const unsigned int pos = block_base + atomicAdd(&bins[nrow], 1u);
            const uint32_t j0 = d.lists.partner[l][s];
            d.lists.act[l][pos] = make_uint4((uint32_t)s, (uint32_t)nrow, j0, 0u);
        }
        return;
    }
    if (warp_level) {
        if (lane == 0 && ball) {
            unsigned int pos = atomicAdd(d.lists.n_act[l], 1u);
            d.lists.act[l][pos] = make_uint4((uint32_t)(s >> 5), 0u, 0u, 0u);
        }
        // owners never span two groups: an idle group's owners get no contact force for as
        // long as this list is in use, and the steps of the previous list are done
        if (!ball && s < d.N && d.sph_head[s]) {
            using R = typename F::R;
            const uint32_t o = d.sph_owner[s];
            if (o != 0xffffffffu) {
                d.fo[o] = typename F::R4{R(0), R(0), R(0), R(0)};
                d.to[o] = typename F::R4{R(0), R(0), R(0), R(0)};
            }
        }
    }
}

// Link the new list: every entry carries its tangential history over from the same pair
// in the list in use (zero for a pair that is new: Sec. 4.2, contact wildcards start at
// zero); each side its own copy.
// ACT (single spheres): one thread per entry of the new list's compacted work (its slots
// with entries, compacted on the detection stream), not per slot.
template <class F, bool ACT = false>
__global__ void __launch_bounds__(256) k_link(Dev<F> d)
{
    using R = typename F::R;
    DevStatus *stp = d.status;
    if (stp->halt) return;
    const int lo = stp->list_cur, ln = lo ^ 1;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t s = g;
    bool live;                               // every lane stays for the warp sum below
    int n;
    if constexpr (ACT) {
        const int64_t na = min((int64_t)*d.lists.n_act[ln], d.Np);
        live = g < na;
        const uint4 a = live ? d.lists.act[ln][g] : make_uint4(0u, 0u, 0u, 0u);
        s = a.x;
        n = live ? (int)a.y : 0;
    } else {
        live = s < d.N;
        n = live ? d.lists.cnt[ln][s] : 0;
    }
    const int hs = stp->hist_par, hd = hs ^ 1;
    const uint32_t *pn = d.lists.partner[ln];
    const uint32_t *po = d.lists.partner[lo];
    const int nold = live ? d.lists.cnt[lo][s] : 0;
    unsigned int owned = 0;                  // pairs this slot owns (partner id above its own)
    // the first LINK_REG entries of the old row in one batch of independent loads; a new
    // entry is matched against them by compares in registers (longer rows search the
    // rest), not by a chain of dependent loads
    constexpr int LINK_REG = 8;
    uint32_t oldr[LINK_REG];
#pragma unroll
    for (int q = 0; q < LINK_REG; ++q) oldr[q] = q < nold ? po[(int64_t)q * d.Np + s] : 0xffffffffu;
    for (int k = 0; k < n; ++k) {
        int64_t e = (int64_t)k * d.Np + s;
        uint32_t j = pn[e];
        if (!(j & WALL_BIT) && j > (uint32_t)s) ++owned;
        int ko = -1;
#pragma unroll
        for (int q = 0; q < LINK_REG; ++q)
            if (q < nold && oldr[q] == j) ko = q;
        if (ko < 0 && nold > LINK_REG && j > oldr[LINK_REG - 1]) {
            const int kr = row_find(po + (int64_t)LINK_REG * d.Np, d.Np, s, nold - LINK_REG, j);
            if (kr >= 0) ko = kr + LINK_REG;
        }
        V3<R> u = {R(0), R(0), R(0)};
        R age = R(0);
        if (ko >= 0) u = hist_get<typename HistVec<R>::T, R>(d.lists.hist[hs], (int64_t)ko * d.Np + s, age);
        hist_put(d.lists.hist[hd], e, u, age);
        if (d.lists.wild[0]) {
            // a contact model's further wildcards travel with the pair too
            typename HistVec<R>::T wv;
            wv.x = R(0); wv.y = R(0); wv.z = R(0); wv.w = R(0);
            if (ko >= 0) wv = d.lists.wild[hs][(int64_t)ko * d.Np + s];
            d.lists.wild[hd][e] = wv;
        }
    }
    const unsigned int tot = __reduce_add_sync(0xffffffffu, owned);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&stp->list_pairs[ln], tot);
}

// Switch to the new list (single thread, after k_link).
static __global__ void k_commit(DevStatus *stp)
{
    if (stp->halt) return;
    stp->list_cur ^= 1;
    stp->hist_par ^= 1;
    stp->acc_par ^= 1;
    stp->disp_cur = stp->disp_next;
    stp->beta_cur = stp->beta_next;
    stp->list_stale = stp->disp_cur > stp->beta_cur ? 1 : 0;
    stp->rebuilds += 1;
}

// ------------------------------------------------------------------ force + integration

// Quaternion increment for a rotation vector th (angle |th|): (cos(|th|/2), sin(|th|/2) th/|th|).
// Integration arithmetic with every product and sum rounded on its own (no fused
// multiply-add): the same update compiled into different kernels (plain and staged
// loads) gives the same bits, and the order is that of the written formulas.
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
template <typename R> __device__ __forceinline__ V3<R> vadd_rn(V3<R> a, V3<R> b)
{
    return {radd(a.x, b.x), radd(a.y, b.y), radd(a.z, b.z)};
}
template <typename R> __device__ __forceinline__ V3<R> vscale_rn(R k, V3<R> a)
{
    return {rmul(k, a.x), rmul(k, a.y), rmul(k, a.z)};
}
template <typename R> __device__ __forceinline__ R dot_rn(V3<R> a, V3<R> b)
{
    return radd(radd(rmul(a.x, b.x), rmul(a.y, b.y)), rmul(a.z, b.z));
}
template <typename R> __device__ __forceinline__ V3<R> cross_rn(V3<R> a, V3<R> b)
{
    return {rsub(rmul(a.y, b.z), rmul(a.z, b.y)), rsub(rmul(a.z, b.x), rmul(a.x, b.z)),
            rsub(rmul(a.x, b.y), rmul(a.y, b.x))};
}
template <typename R> __device__ __forceinline__ void quat_mat_rn(R qw, R qx, R qy, R qz, R m[9])
{
    const R one = R(1), two = R(2);
    R xx = rmul(qx, qx), yy = rmul(qy, qy), zz = rmul(qz, qz);
    R xy = rmul(qx, qy), xz = rmul(qx, qz), yz = rmul(qy, qz);
    R wx = rmul(qw, qx), wy = rmul(qw, qy), wz = rmul(qw, qz);
    m[0] = rsub(one, rmul(two, radd(yy, zz))); m[1] = rmul(two, rsub(xy, wz)); m[2] = rmul(two, radd(xz, wy));
    m[3] = rmul(two, radd(xy, wz)); m[4] = rsub(one, rmul(two, radd(xx, zz))); m[5] = rmul(two, rsub(yz, wx));
    m[6] = rmul(two, rsub(xz, wy)); m[7] = rmul(two, radd(yz, wx)); m[8] = rsub(one, rmul(two, radd(xx, yy)));
}
template <typename R> __device__ __forceinline__ V3<R> mat_vec_rn(const R m[9], V3<R> a)
{
    return {radd(radd(rmul(m[0], a.x), rmul(m[1], a.y)), rmul(m[2], a.z)),
            radd(radd(rmul(m[3], a.x), rmul(m[4], a.y)), rmul(m[5], a.z)),
            radd(radd(rmul(m[6], a.x), rmul(m[7], a.y)), rmul(m[8], a.z))};
}
template <typename R> __device__ __forceinline__ V3<R> mat_tvec_rn(const R m[9], V3<R> a)
{
    return {radd(radd(rmul(m[0], a.x), rmul(m[3], a.y)), rmul(m[6], a.z)),
            radd(radd(rmul(m[1], a.x), rmul(m[4], a.y)), rmul(m[7], a.z)),
            radd(radd(rmul(m[2], a.x), rmul(m[5], a.y)), rmul(m[8], a.z))};
}

// Rotation increment [cos(h|w|/2), sin(h|w|/2) w/|w|] of angular velocity w over h.
template <typename R>
__device__ __forceinline__ void quat_increment(V3<R> w, R h, R &dw, R &dx, R &dy, R &dz)
{
    R wn = sqrt(dot_rn(w, w));
    if (wn >= R(1e-30)) {
        R half = rmul(rmul(R(0.5), h), wn);
        R sn = rdiv(sin(half), wn);
        dw = cos(half);
        dx = rmul(sn, w.x);
        dy = rmul(sn, w.y);
        dz = rmul(sn, w.z);
    } else {
        dw = R(1); dx = R(0); dy = R(0); dz = R(0);
    }
}

template <typename R>
__device__ __forceinline__ void quat_mul(R aw, R ax, R ay, R az, R bw, R bx, R by, R bz, R &w, R &x, R &y, R &z)
{
    w = rsub(rsub(rsub(rmul(aw, bw), rmul(ax, bx)), rmul(ay, by)), rmul(az, bz));
    x = rsub(radd(radd(rmul(aw, bx), rmul(ax, bw)), rmul(ay, bz)), rmul(az, by));
    y = radd(radd(rsub(rmul(aw, by), rmul(ax, bz)), rmul(ay, bw)), rmul(az, bx));
    z = radd(rsub(radd(rmul(aw, bz), rmul(ax, by)), rmul(ay, bx)), rmul(az, bw));
}

// Contact forces of every listed pair of slot s and the per-owner sums (segmented warp
// reduction over the owner's consecutive slots).  MODE_STEP writes the owner's contact
// force and torque (fo, to) for k_integrate and the updated tangential history; a single
// sphere without listed partners leaves at once.  MODE_EVAL writes the per-owner force
// (gravity included) and torque in FP64 and changes nothing.
constexpr int CONTACT_BLOCK_MAX = 128;   // launch shapes are tuned at run time up to these
constexpr int INTEGRATE_BLOCK_MAX = 512;

// Pairwise material constants of the form's precision.
template <class F>
__device__ __forceinline__ const PairParamF *pair_table(const Dev<F> &d, float)
{
    return d.pairs_f;
}
template <class F>
__device__ __forceinline__ const PairParam *pair_table(const Dev<F> &d, double)
{
    return d.pairs;
}

// The fourth lane of a history vector counts a contact's duration: in the FP64 form its
// age in seconds, accumulated as age + h every step (the wildcard of Sec. 4.2.1); in the
// voxel form the number of steps it has lasted, an integer held exactly in FP32 up to
// 2^24 steps, whose age count * h has one rounding instead of one per step.
template <class F>
__device__ __forceinline__ typename F::R advance_age(typename F::R lane, typename F::R h)
{
    if constexpr (F::voxel) return radd(lane, typename F::R(1));
    else return radd(lane, h);
}
template <class F>
__device__ __forceinline__ typename F::R age_seconds(typename F::R lane, typename F::R h)
{
    if constexpr (F::voxel) return rmul(lane, h);
    else return lane;
}

template <class F>
__device__ __forceinline__ const float *crr_table(const Dev<F> &d, float)
{
    return d.crr_f;
}
template <class F>
__device__ __forceinline__ const double *crr_table(const Dev<F> &d, double)
{
    return d.crr;
}

// The n listed entries of sphere s (first partner j_first) evaluated from s's side: the
// sums of the contact forces on s and of their torques about its owner's centre, and
// (MODE_STEP) each entry's updated history written to the other history buffer.  Every
// load of an entry (history, partner state, the partner's flag) is issued before any is
// used, so an entry costs one memory round trip; the material constants come from the
// sphere's own scene (both bodies of a contact belong to it), without a lookup of the
// partner's material where the scene has only one.
// ROLL compiles in rolling resistance (worlds where a material pair has C_r > 0): each
// entry's age is kept in its history vector, and past the collision time the rolling
// force's torque is added after the contact force's.
// LAZY (single spheres): me comes without its velocities, which are read at the first
// entry that needs them (a wall, or a sphere pair that overlaps).  Returns whether any
// entry made contact (Fs and Ts are exactly zero otherwise).
// MASKED (the evaluation pass of the two-pass step): only the entries whose bit is set in
// mask are evaluated (the screening pass wrote the others' zero history), in row order;
// j_first is the first masked entry's partner, the others' ids are read from the row.
// A masked sphere entry is known to overlap (the screening pass took the same test on
// the same values), so its velocities and history are loaded with its position record.
template <class F, bool CLUMPS, int MODE, bool ROLL = false, bool LAZY = false, bool MASKED = false>
__device__ __forceinline__ bool pair_sums(const Dev<F> &d, const SphereK<F> &me_in, const Scene &sc, int64_t s, int n,
                                          uint32_t j_first, int sp, int hp, int lc, V3<typename F::R> &Fs,
                                          V3<typename F::R> &Ts, uint64_t mask = ~0ull)
{
    static_assert(!LAZY || !CLUMPS, "only single spheres read their velocities late");
    using R = typename F::R;
    SphereK<F> me = me_in;
    bool have_v = !LAZY, any = false;
    auto need_v = [&]() {
        if (LAZY && !have_v) {
            const auto v4 = d.st.kv[sp][2 * (int64_t)me.owner];
            const auto w4 = d.st.kv[sp][2 * (int64_t)me.owner + 1];
            me.v = {v4.x, v4.y, v4.z};
            me.w = {w4.x, w4.y, w4.z};
            have_v = true;
        }
    };
    const R h = F::voxel ? (R)sc.hf : (R)sc.h;
    const uint32_t *prow = d.lists.partner[lc];
    using H = typename HistVec<R>::T;
    const H *hin = d.lists.hist[hp];
    H *hout = d.lists.hist[hp ^ 1];
    const V3<R> zero = {R(0), R(0), R(0)};
    const auto *tab = pair_table(d, R(0));
    const bool one = sc.n_mat == 1;
    const int row = sc.pair_base + (me.mat - sc.mat_base) * sc.n_mat - sc.mat_base;
    uint32_t j_next = j_first;
    bool first = true;
    for (int k = 0; k < n; ++k) {
        if constexpr (MASKED) {
            if (!((mask >> k) & 1ull)) continue;
        }
        const int64_t e = (int64_t)k * d.Np + s;
        uint32_t j;
        if constexpr (MASKED) {
            j = first ? j_first : prow[e];
            first = false;
        } else {
            j = j_next;
            if (k + 1 < n) j_next = prow[e + d.Np];  // next partner's id in flight early
        }
        R age = R(0);
        V3<R> ut = zero;
        ContactIn<R> c;
        V3<R> armA, armB;
        V3<R> wB = zero;                 // the partner's angular velocity (ROLL only)
        bool on;
        int mb = 0;
        if (j & WALL_BIT) {
            need_v();
            ut = ROLL ? hist_get<H, R>(hin, e, age) : hist_get<H, R>(hin, e);
            const Wall &w = d.walls[j & ~WALL_BIT];
            mb = w.mat;
            on = wall_contact<F, false>(d, me, sc, w, c, armA);
        } else if constexpr (!CLUMPS) {
            // single spheres: the partner's position record first; its velocities, its
            // activity and this entry's history only where the two overlap (most listed
            // pairs do not touch).  The pair is evaluated in this thread's own orientation
            // with this side's copy of the history (the partner's is its exact negation)
            SphereK<F> other = load_sphere_pos<F>(d, sp, j);
            typename F::R4 v4{}, w4{};
            if constexpr (MASKED) {
                v4 = d.st.kv[sp][2 * j];
                w4 = d.st.kv[sp][2 * j + 1];
                ut = ROLL ? hist_get<H, R>(hin, e, age) : hist_get<H, R>(hin, e);
            }
            V3<R> dd;
            R dist, delta;
            sphere_gap<F>(d, me, other, dd, dist, delta);
            on = delta > R(0) && dist > R(0) && d.st.active[sp][j];
            if (on) {
                need_v();
                if constexpr (!MASKED) {
                    v4 = d.st.kv[sp][2 * j];
                    w4 = d.st.kv[sp][2 * j + 1];
                    ut = ROLL ? hist_get<H, R>(hin, e, age) : hist_get<H, R>(hin, e);
                }
                other.v = {v4.x, v4.y, v4.z};
                other.w = {w4.x, w4.y, w4.z};
                mb = other.mat >= 0 || one ? other.mat : (int)d.sph_mat[j];
                sphere_finish<F, false>(d, me, other, dd, dist, delta, c, armA, armB);
                if constexpr (ROLL) wB = other.w;
            }
        } else {
            ut = ROLL ? hist_get<H, R>(hin, e, age) : hist_get<H, R>(hin, e);
            SphereK<F> other = load_sphere<F, CLUMPS, false>(d, sp, j);
            if (!d.st.active[sp][other.owner]) {
                if (MODE == MODE_STEP) hist_put(hout, e, zero);
                continue;
            }
            // the pair is evaluated in this thread's own orientation with this side's
            // copy of the history (the partner's copy is its exact negation)
            mb = other.mat >= 0 || one ? other.mat : (int)d.sph_mat[j];
            on = sphere_contact<F, false>(d, me, other, c, armA, armB);
            if constexpr (ROLL) wB = other.w;
        }
        if (on) {
            const int pk = one ? sc.pair_base : row + mb;
            const auto p = tab[pk];
            c.Estar = p.Estar;
            c.Gstar = p.Gstar;
            c.beta = p.beta;
            c.mu = p.mu;
            V3<R> Fc;
            if constexpr (ROLL) {
                R fn_abs;
                hertz_mindlin<R>(c, h, ut, Fc, &fn_abs);
                age = advance_age<F>(age, h);
                Fs = Fs + Fc;
                Ts = Ts + cross(armA, Fc);
                const R crr = crr_table(d, R(0))[pk];
                if (crr > R(0) && !within_collision_time<R>(c, age_seconds<F>(age, h))) {
                    // rolling parts of the contact-point velocities; a wall moves by
                    // rotation only, so its part is its whole surface velocity
                    const V3<R> rotA = cross_rn(me.w, armA);
                    const V3<R> rotB = (j & WALL_BIT) ? c.uB : cross_rn(wB, armB);
                    const V3<R> vr = {rsub(rotB.x, rotA.x), rsub(rotB.y, rotA.y), rsub(rotB.z, rotA.z)};
                    Ts = Ts + cross(armA, rolling_force<R>(crr, fn_abs, vr));
                }
            } else {
                hertz_mindlin<R>(c, h, ut, Fc);
                Fs = Fs + Fc;
                Ts = Ts + cross(armA, Fc);
            }
        }
        any = any || on;
        if (MODE == MODE_STEP) hist_put(hout, e, on ? ut : zero, on ? age : R(0));
    }
    return any;
}

template <class F>
__device__ __forceinline__ const float *model_params(const Dev<F> &d, float)
{
    return d.model_par_f;
}
template <class F>
__device__ __forceinline__ const double *model_params(const Dev<F> &d, double)
{
    return d.model_par;
}

// One listed entry (partner j) of sphere s through a contact model of force_models.cuh,
// with the entry's wildcards wc[8] (updated).  A sphere pair is evaluated with A the
// lower slot on both of its sides: the upper side swaps the roles, brings its copy of
// the odd wildcards into A's orientation and back, and takes the negated forces, so each
// side obtains exactly the other's reaction whatever the model computes.  Walls take the
// default model (they belong to no bond).  Returns whether the pair interacts; F and Fr
// (torque-only) act on s's owner at arm (contact point minus its centre of mass).
template <class F, bool CLUMPS, class Model>
__device__ __forceinline__ bool model_entry(const Dev<F> &d, const SphereK<F> &me, const Scene &sc, int64_t s,
                                            uint32_t j, int sp, typename F::R *wc, V3<typename F::R> &Fo,
                                            V3<typename F::R> &Fr, V3<typename F::R> &arm, typename F::R &overlap)
{
    using R = typename F::R;
    const R h = F::voxel ? (R)sc.hf : (R)sc.h;
    const R *par = model_params(d, R(0));
    const auto *tab = pair_table(d, R(0));
    const R *crr_tab = crr_table(d, R(0));
    const V3<R> zero = {R(0), R(0), R(0)};
    Fo = zero; Fr = zero; arm = zero; overlap = R(0);
    if (j & WALL_BIT) {
        const Wall &w = d.walls[j & ~WALL_BIT];
        ContactIn<R> ci;
        V3<R> armA;
        if (!wall_contact<F, false>(d, me, sc, w, ci, armA)) return false;
        const int pk = sc.pair_base + (me.mat - sc.mat_base) * sc.n_mat + (w.mat - sc.mat_base);
        const auto p = tab[pk];
        ci.Estar = p.Estar; ci.Gstar = p.Gstar; ci.beta = p.beta; ci.mu = p.mu;
        V3<R> ut = {wc[0], wc[1], wc[2]};
        R fn_abs;
        hertz_mindlin<R>(ci, h, ut, Fo, &fn_abs);
        wc[0] = ut.x; wc[1] = ut.y; wc[2] = ut.z;
        wc[3] = radd(wc[3], h);
        const R crr = crr_tab[pk];
        if (crr > R(0) && !within_collision_time<R>(ci, wc[3])) {
            const V3<R> rotA = cross_rn(me.w, armA);
            Fr = rolling_force<R>(crr, fn_abs, V3<R>{rsub(ci.uB.x, rotA.x), rsub(ci.uB.y, rotA.y),
                                                      rsub(ci.uB.z, rotA.z)});
        }
        arm = armA;
        overlap = ci.delta;
        return true;
    }
    SphereK<F> other = load_sphere<F, CLUMPS>(d, sp, j);
    if (!d.st.active[sp][other.owner]) return false;
    const bool swap = j < (uint32_t)s;
    const SphereK<F> &A = swap ? other : me;
    const SphereK<F> &B = swap ? me : other;
    ContactIn<R> ci;
    V3<R> armA, armB;
    if (!sphere_contact<F, false, true>(d, A, B, ci, armA, armB)) return false;
    if (swap) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if ((Model::odd >> q) & 1u) wc[q] = -wc[q];
    }
    const int pk = sc.pair_base + (A.mat - sc.mat_base) * sc.n_mat + (B.mat - sc.mat_base);
    const auto p = tab[pk];
    Referables<R> c;
    c.B2A = ci.n;
    c.overlapDepth = ci.delta;
    c.ts = h;
    c.locCPA = armA; c.locCPB = armB;
    c.ALinVel = A.v; c.BLinVel = B.v;
    c.ARotVel = A.w; c.BRotVel = B.w;
    c.velB2A = ci.uA - ci.uB;
    c.AOwnerMass = A.mass; c.BOwnerMass = B.mass;
    c.ARadius = A.rad; c.BRadius = B.rad;
    c.Rbar = ci.Rbar; c.mbar = ci.mbar;
    c.AMat = A.mat; c.BMat = B.mat;
    c.AFamily = d.owner_family ? (int)d.owner_family[A.owner] : 0;
    c.BFamily = d.owner_family ? (int)d.owner_family[B.owner] : 0;
    c.AGeo = swap ? j : (uint32_t)s;
    c.BGeo = swap ? (uint32_t)s : j;
    c.Estar = p.Estar; c.Gstar = p.Gstar; c.beta = p.beta; c.mu = p.mu;
    c.crr = crr_tab[pk];
    c.nu = (R)d.pair_nu[pk];
    const bool on = Model::engaged(c, wc, par);
    if (on) Model::eval(c, wc, par, Fo, Fr);
    if (swap) {
        Fo = -Fo;
        Fr = -Fr;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if ((Model::odd >> q) & 1u) wc[q] = -wc[q];
    }
    arm = swap ? armB : armA;
    overlap = ci.delta;
    return on;
}

// The listed entries of sphere s through a contact model (model_entry): sums of the
// forces and torques on s's owner, and (MODE_STEP) the entries' wildcards, zero where
// a pair does not interact (the contact has vanished).
template <class F, bool CLUMPS, int MODE, class Model>
__device__ __forceinline__ void pair_sums_model(const Dev<F> &d, const SphereK<F> &me, const Scene &sc, int64_t s,
                                                int n, int sp, int hp, int lc, V3<typename F::R> &Fs,
                                                V3<typename F::R> &Ts)
{
    using R = typename F::R;
    using H = typename HistVec<R>::T;
    const uint32_t *prow = d.lists.partner[lc];
    const H *hin = d.lists.hist[hp];
    H *hout = d.lists.hist[hp ^ 1];
    constexpr bool WILD = Model::n_wildcards > 4;
    const H *win = WILD ? d.lists.wild[hp] : nullptr;
    H *wout = WILD ? d.lists.wild[hp ^ 1] : nullptr;
    for (int k = 0; k < n; ++k) {
        const int64_t e = (int64_t)k * d.Np + s;
        const uint32_t j = prow[e];
        R wc[8];
        {
            const H a = hin[e];
            wc[0] = (R)a.x; wc[1] = (R)a.y; wc[2] = (R)a.z; wc[3] = (R)a.w;
            if constexpr (WILD) {
                const H b = win[e];
                wc[4] = (R)b.x; wc[5] = (R)b.y; wc[6] = (R)b.z; wc[7] = (R)b.w;
            } else {
                wc[4] = wc[5] = wc[6] = wc[7] = R(0);
            }
        }
        V3<R> Fc, Fr, arm;
        R ov;
        const bool on = model_entry<F, CLUMPS, Model>(d, me, sc, s, j, sp, wc, Fc, Fr, arm, ov);
        if (on) {
            Fs = Fs + Fc;
            Ts = Ts + cross(arm, Fc);
            Ts = Ts + cross(arm, Fr);
        }
        if (MODE == MODE_STEP) {
            if (!on) {
#pragma unroll
                for (int q = 0; q < 8; ++q) wc[q] = R(0);
            }
            H a;
            a.x = wc[0]; a.y = wc[1]; a.z = wc[2]; a.w = wc[3];
            hout[e] = a;
            if constexpr (WILD) {
                H b;
                b.x = wc[4]; b.y = wc[5]; b.z = wc[6]; b.w = wc[7];
                wout[e] = b;
            }
        }
    }
}

template <class F, bool CLUMPS>
__device__ __forceinline__ void integrate_core(const Dev<F> &d, DevStatus *stp, int64_t o, int sp, bool act,
                                               const typename F::Pos &po, typename F::R mass, typename F::R4 v4,
                                               typename F::R4 w4, typename F::R4 q4, typename F::R im,
                                               typename F::R4 ii, bool iso, const Scene &sc, V3<typename F::R> Fs,
                                               V3<typename F::R> Ts, const typename F::Aux &aux, float &disp,
                                               float &disp2, float &speed, const typename F::R4 *qsrc = nullptr);
__device__ __forceinline__ void audit_slots(unsigned int *audit, int64_t o, int lane, float disp, float disp2,
                                            float speed);

// 1/m and 1/I (isotropic, r_ext 0) of a single sphere from its mass and radius, where the
// world derives them (Dev::solid): every kernel that integrates rounds them the same way.
template <class F>
__device__ __forceinline__ void solid_consts(const Dev<F> &d, typename F::R mass, float rad, typename F::R &im,
                                             typename F::R4 &ii)
{
    using R = typename F::R;
    im = rdiv(R(1), mass);
    const R iI = rdiv(R(1), rmul(rmul((R)d.moi_coef, mass), rmul((R)rad, (R)rad)));
    ii = typename F::R4{iI, iI, iI, R(0)};
}

// INTEG (single spheres, MODE_STEP): the contact kernel also integrates the owner of the
// slot, from the state it has already loaded and the force it has just summed, and
// keeps the running maxima of the audit values in aud[3]; the integration kernel then
// leaves owners with listed partners alone (k_integrate<..., SKIP_LISTED>).  No
// per-owner force array is written or read, and such an owner's state is read once.
template <class F, bool CLUMPS, int MODE, bool ROLL = false, int MODEL = FORCE_MODEL_BUILTIN, bool INTEG = false>
__device__ __forceinline__ void contact_slot(const Dev<F> &d, int64_t s, int n_known, uint32_t j0_known, int sp,
                                             int hp, int lc, double *eval_F, double *eval_T, float *aud = nullptr)
{
    static_assert(!INTEG || (!CLUMPS && MODE == MODE_STEP), "the contact kernel integrates only single spheres");
    using R = typename F::R;
    using R4 = typename F::R4;
    const int lane = threadIdx.x & 31;
    bool live = s < d.N;
    // a world of single spheres has one slot per owner, in owner order
    uint32_t o = live ? (CLUMPS ? d.sph_owner[s] : (uint32_t)s) : 0xffffffffu;
    live = live && o != 0xffffffffu;
    // the row length comes with the compacted work where it is known
    const int n = !live ? 0 : (n_known >= 0 ? n_known : (int)d.lists.cnt[lc][s]);
    bool act = live && d.st.active[sp][o];
    if (!CLUMPS && MODE == MODE_STEP && (!act || n == 0)) return;

    // single spheres in the two-kernel step: the sphere's velocities are read only if an
    // entry needs them, and the force only written (with its flag) if an entry touched
    constexpr bool LAZY = !CLUMPS && MODE == MODE_STEP && !INTEG && MODEL == FORCE_MODEL_BUILTIN;
    V3<R> Fs = {R(0), R(0), R(0)}, Ts = {R(0), R(0), R(0)};
    SphereK<F> me;
    int scene = 0;
    R4 q4 = {}, ii = {};
    R im = R(0);
    if (live) {
        // a world of one scene and a scene of one material need neither index read
        scene = d.n_scenes > 1 ? d.owner_scene[o] : 0;
        if constexpr (LAZY) {
            me = load_sphere_pos<F>(d, sp, (uint32_t)s);
            if constexpr (F::voxel) {
                const Scene &sc0 = d.scenes[scene];
                me.mat = sc0.n_mat == 1 ? sc0.mat_base : (int)d.sph_mat[s];
            }
        } else {
            me = load_sphere<F, CLUMPS>(d, sp, (uint32_t)s);
        }
        if constexpr (INTEG) {
            // the rest of the owner's inputs are in flight while the pairs are summed (its
            // orientation is read by the integration only if the sphere turns)
            if (F::voxel && d.solid) {
                solid_consts<F>(d, me.mass, (float)me.rad, im, ii);
            } else {
                im = d.inv_mass[o];
                ii = d.inv_moi[o];
            }
        }
    }
    bool any = true;
    if (act) {
        if constexpr (MODEL == FORCE_MODEL_HERTZ_MINDLIN)
            pair_sums_model<F, CLUMPS, MODE, ModelHertzMindlin>(d, me, d.scenes[scene], s, n, sp, hp, lc, Fs, Ts);
        else if constexpr (MODEL == FORCE_MODEL_BONDED_BREAKAGE)
            pair_sums_model<F, CLUMPS, MODE, ModelBondedBreakage>(d, me, d.scenes[scene], s, n, sp, hp, lc, Fs, Ts);
        else
            any = pair_sums<F, CLUMPS, MODE, ROLL, LAZY>(
                d, me, d.scenes[scene], s, n, n_known >= 0 ? j0_known : (n > 0 ? d.lists.partner[lc][s] : 0u), sp,
                hp, lc, Fs, Ts);
    }
    if (CLUMPS) {
        // segmented suffix sums over the owner's consecutive lanes; the head lane ends
        // with the owner's total (fixed tree order: deterministic)
        const int end = live ? (int)d.sph_segend[s] : lane + 1;
        R v6[6] = {Fs.x, Fs.y, Fs.z, Ts.x, Ts.y, Ts.z};
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
            for (int c6 = 0; c6 < 6; ++c6) {
                R other = __shfl_down_sync(0xffffffffu, v6[c6], off);
                if (lane + off < end) v6[c6] += other;
            }
        }
        Fs = {v6[0], v6[1], v6[2]};
        Ts = {v6[3], v6[4], v6[5]};
    }
    const bool head = live && (!CLUMPS || d.sph_head[s]);
    if (!head) return;
    if (MODE == MODE_EVAL) {
        const Scene &sc = d.scenes[scene];
        const V3<R> g = F::voxel ? V3<R>{(R)sc.gf[0], (R)sc.gf[1], (R)sc.gf[2]}
                                 : V3<R>{(R)sc.g[0], (R)sc.g[1], (R)sc.g[2]};
        V3<R> Ft = act ? Fs + me.mass * g : V3<R>{R(0), R(0), R(0)};
        eval_F[3 * o + 0] = (double)Ft.x; eval_F[3 * o + 1] = (double)Ft.y; eval_F[3 * o + 2] = (double)Ft.z;
        eval_T[3 * o + 0] = (double)Ts.x; eval_T[3 * o + 1] = (double)Ts.y; eval_T[3 * o + 2] = (double)Ts.z;
    } else if constexpr (INTEG) {
        // the same update as k_integrate from the same inputs (the force it would read
        // back is the one summed here): the same bits
        typename F::Aux aux{};
        if constexpr (F::voxel) {
            aux.rad = me.rad;
            aux.rlo = me.rlo;
        }
        float disp = 0.0f, disp2 = 0.0f, speed = 0.0f;
        integrate_core<F, false>(d, d.status, o, sp, true, me.p, me.mass, R4{me.v.x, me.v.y, me.v.z, me.acc0},
                                 R4{me.w.x, me.w.y, me.w.z, me.acc1}, q4, im, ii, true, d.scenes[scene], Fs, Ts, aux,
                                 disp, disp2, speed, &d.st.quat[sp][o]);
        aud[0] = fmaxf(aud[0], disp);
        aud[1] = fmaxf(aud[1], disp2);
        aud[2] = fmaxf(aud[2], speed);
    } else {
        if constexpr (!CLUMPS) {
            // the integration reads the force of an owner with listed partners only where
            // this flag is set (an owner whose entries all missed has Fs = Ts = 0 exactly)
            d.touched[o] = any ? 1 : 0;
            if (!any) return;
        }
        d.fo[o] = R4{Fs.x, Fs.y, Fs.z, R(0)};
        d.to[o] = R4{Ts.x, Ts.y, Ts.z, R(0)};
    }
}

// MODE_STEP: persistent grid-stride loop over the compacted work of the list in use
// (every thread busy, whichever fraction of the spheres has listed partners); for clumps
// a whole warp takes a 32-slot group.  MODE_EVAL: one thread per slot over all slots.
// LEAN = 1 compiles the kernel for 5 resident blocks of CONTACT_BLOCK_MAX threads per SM
// (96 registers, some spilled to the L1-cached local memory) instead of 4: more
// warps to hide the latency of the gathers, chosen by the autotuner where it pays.
template <class F, bool CLUMPS, int MODE, int LEAN = 0, bool ROLL = false, int MODEL = FORCE_MODEL_BUILTIN,
          bool INTEG = false>
__global__ void __launch_bounds__(CONTACT_BLOCK_MAX, LEAN ? 5 : 4) k_contact(Dev<F> d, double *eval_F, double *eval_T)
{
    DevStatus *stp = d.status;
    if (MODE == MODE_STEP && (stp->halt || stp->list_stale)) return;
    const int sp = stp->state_par, hp = stp->hist_par, lc = stp->list_cur;
    if (MODE == MODE_EVAL) {
        contact_slot<F, CLUMPS, MODE, ROLL, MODEL>(d, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, -1, 0u, sp, hp,
                                                   lc, eval_F, eval_T);
        return;
    }
    // the counter never exceeds the slots (or 32-slot groups); the clamp keeps every
    // index in bounds whatever the counter holds
    const int64_t cap = CLUMPS ? (d.Np >> 5) : d.Np;
    const int64_t nw = min((int64_t)*d.lists.n_act[lc], cap);
    const uint4 *act = d.lists.act[lc];
    if (CLUMPS) {
        const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
        for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw; w += warps)
            contact_slot<F, CLUMPS, MODE, ROLL, MODEL>(d, ((int64_t)act[w].x << 5) + (threadIdx.x & 31), -1, 0u, sp,
                                                       hp, lc, eval_F, eval_T);
    } else {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        int64_t t = t0;
        uint4 a = t < nw ? act[t] : make_uint4(0u, 0u, 0u, 0u);
        float aud[3] = {0.0f, 0.0f, 0.0f};
        for (; t < nw; t += stride) {
            // the next work entry is read while this one is evaluated
            const uint4 next = t + stride < nw ? act[t + stride] : a;
            contact_slot<F, CLUMPS, MODE, ROLL, MODEL, INTEG>(d, (int64_t)a.x, (int)a.y, a.z, sp, hp, lc, eval_F,
                                                              eval_T, aud);
            a = next;
        }
        // every lane of the warp gets here (the loop's exit is the only divergence)
        if constexpr (INTEG) audit_slots(d.audit, t0, threadIdx.x & 31, aud[0], aud[1], aud[2]);
    }
}

// Two-pass contact step (single spheres, the built-in model without rolling resistance).
// Most listed pairs do not touch: in one kernel, a warp's lanes split between the whole
// Hertz-Mindlin evaluation and an early exit, and the evaluation's registers leave few
// warps to hide the gathers.  The screening pass takes each sphere of the compacted work
// with few registers, gathers its partners' position records and tests their overlap
// exactly as the evaluation does; an entry that does not touch gets its zero history
// here, a sphere none of whose entries touches its cleared flag, and a sphere with
// touching entries (or wall entries, which only the evaluation tests) is appended to
// d.screen with the mask of those entries (one atomic per warp).  The evaluation pass
// (k_contact_eval) takes the appended spheres and evaluates only the masked entries, in
// row order: the same sums, histories, forces and flags as k_contact, bit for bit.  The
// order of d.screen depends on scheduling; results do not (each sphere's outputs are
// its own).
constexpr int SCREEN_BLOCK = 256;
template <class F>
__global__ void __launch_bounds__(SCREEN_BLOCK, 5) k_contact_screen(Dev<F> d)
{
    using R = typename F::R;
    using H = typename HistVec<R>::T;
    DevStatus *stp = d.status;
    if (stp->halt || stp->list_stale) return;
    const int sp = stp->state_par, hp = stp->hist_par, lc = stp->list_cur;
    // the counter never exceeds the slots; the clamp keeps every index in bounds
    const int64_t nw = min((int64_t)*d.lists.n_act[lc], d.Np);
    const uint4 *act = d.lists.act[lc];
    const uint32_t *prow = d.lists.partner[lc];
    H *hout = d.lists.hist[hp ^ 1];
    const V3<R> zero = {R(0), R(0), R(0)};
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps iterate together: the append below is warp-wide
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nw; base += stride) {
        const int64_t t = base + lane;
        bool cand = false;
        uint4 item = make_uint4(0u, 0u, 0u, 0u);
        if (t < nw) {
            const uint4 a = act[t];
            const uint32_t s = a.x;
            const int n = (int)a.y;
            // the sphere's flag and record, its first partner's record and the second
            // partner's id are independent loads, issued together
            const bool live = n > 0 && d.st.active[sp][s];
            const SphereK<F> me = load_sphere_pos<F>(d, sp, s);
            uint32_t j = a.z;
            SphereK<F> other = (j & WALL_BIT) ? me : load_sphere_pos<F>(d, sp, j);
            uint32_t j_next = n > 1 ? prow[(int64_t)d.Np + s] : WALL_BIT;
            if (live) {
                uint64_t mask = 0;
                uint32_t j_first = 0;
                for (int k = 0; k < n; ++k) {
                    const int64_t e = (int64_t)k * d.Np + s;
                    // the next partner's record and the id after it are in flight while
                    // this entry is tested
                    SphereK<F> nxt = other;
                    if (k + 1 < n && !(j_next & WALL_BIT)) nxt = load_sphere_pos<F>(d, sp, j_next);
                    const uint32_t j_after = k + 2 < n ? prow[e + 2 * (int64_t)d.Np] : WALL_BIT;
                    bool c = true;
                    if (!(j & WALL_BIT)) {
                        V3<R> dd;
                        R dist, delta;
                        sphere_gap<F>(d, me, other, dd, dist, delta);
                        c = delta > R(0) && dist > R(0) && d.st.active[sp][j];
                    }
                    if (c) {
                        if (!mask) j_first = j;
                        mask |= 1ull << k;
                    } else {
                        hist_put(hout, e, zero, R(0));
                    }
                    j = j_next;
                    other = nxt;
                    j_next = j_after;
                }
                if (mask) {
                    cand = true;
                    item = make_uint4(s, j_first, (uint32_t)mask, (uint32_t)(mask >> 32));
                } else {
                    d.touched[s] = 0;
                }
            }
        }
        const unsigned int ball = __ballot_sync(0xffffffffu, cand);
        if (ball) {
            const int leader = __ffs(ball) - 1;
            unsigned int at = 0;
            if (lane == leader) at = atomicAdd(&stp->n_screen, (unsigned int)__popc(ball));
            at = __shfl_sync(0xffffffffu, at, leader);
            if (cand) d.screen[at + __popc(ball & ((1u << lane) - 1u))] = item;
        }
    }
}

// The evaluation pass of the two-pass step: a persistent grid over the spheres the
// screening pass appended, each evaluating its masked entries (pair_sums<..., MASKED>)
// and writing its force and flag as k_contact does.
template <class F>
__global__ void __launch_bounds__(CONTACT_BLOCK_MAX, 4) k_contact_eval(Dev<F> d)
{
    using R = typename F::R;
    using R4 = typename F::R4;
    DevStatus *stp = d.status;
    if (stp->halt || stp->list_stale) return;
    const int sp = stp->state_par, hp = stp->hist_par, lc = stp->list_cur;
    const int64_t nw = min((int64_t)stp->n_screen, d.Np);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nw; t += stride) {
        const uint4 a = d.screen[t];
        const uint32_t s = a.x;
        const uint64_t mask = (uint64_t)a.z | ((uint64_t)a.w << 32);
        const int n = 64 - __clzll((long long)mask);       // past the last masked entry
        const int scene = d.n_scenes > 1 ? d.owner_scene[s] : 0;
        const Scene &sc = d.scenes[scene];
        // nearly every sphere here has a touching entry: its velocities are read at once
        SphereK<F> me = load_sphere<F, false, false>(d, sp, s);
        if constexpr (F::voxel) me.mat = sc.n_mat == 1 ? sc.mat_base : (int)d.sph_mat[s];
        V3<R> Fs = {R(0), R(0), R(0)}, Ts = {R(0), R(0), R(0)};
        const bool any = pair_sums<F, false, MODE_STEP, false, false, true>(d, me, sc, s, n, a.y, sp, hp, lc, Fs,
                                                                             Ts, mask);
        d.touched[s] = any ? 1 : 0;
        if (any) {
            d.fo[s] = R4{Fs.x, Fs.y, Fs.z, R(0)};
            d.to[s] = R4{Ts.x, Ts.y, Ts.z, R(0)};
        }
    }
}

// Warp max of the displacement bounds and the speed (non-negative floats order like
// their bit patterns), one atomic per warp and value into one of AUDIT_SLOTS slots: no
// block barrier, little contention; k_audit reduces the slots.
__device__ __forceinline__ void audit_slots(unsigned int *audit, int64_t o, int lane, float disp, float disp2,
                                            float speed)
{
    unsigned int db = __reduce_max_sync(0xffffffffu, __float_as_uint(disp));
    unsigned int db2 = __reduce_max_sync(0xffffffffu, __float_as_uint(disp2));
    unsigned int vb = __reduce_max_sync(0xffffffffu, __float_as_uint(speed));
    if (lane == 0) {
        unsigned int *slot = audit + ((o >> 5) & (AUDIT_SLOTS - 1)) * AUDIT_STRIDE;
        if (db) atomicMax(&slot[0], db);
        if (db2) atomicMax(&slot[1], db2);
        if (vb) atomicMax(&slot[2], vb);
    }
}

// Where the per-owner inputs of the integration are read: the state arrays in global
// memory (index = owner) or a tile of them staged in shared memory (index = position in
// the tile).  Both paths run the same arithmetic (integrate_owner).
template <class F>
struct OwnerSrc {
    typename F::PosStore pos;
    const typename F::R4 *kv, *quat, *inv_moi;      // kv: v and w of owner i at 2i, 2i + 1
    const typename F::R *inv_mass;
    const uint8_t *active, *cnt, *iso;
    const uint16_t *scene;
};

// Semi-implicit Euler update of one owner from its loaded state and the contact force
// and torque on it: v with the contact force plus gravity, then the body-frame angular
// velocity (Euler's equations, gyroscopic term switchable), then x with the new v, then
// the quaternion with the new angular velocity; removal by the sink; the per-owner
// displacement bounds of the audit.  Outputs go to the other state buffer.
template <class F, bool CLUMPS>
__device__ __forceinline__ void integrate_core(const Dev<F> &d, DevStatus *stp, int64_t o, int sp, bool act,
                                               const typename F::Pos &po, typename F::R mass, typename F::R4 v4,
                                               typename F::R4 w4, typename F::R4 q4, typename F::R im,
                                               typename F::R4 ii, bool iso, const Scene &sc, V3<typename F::R> Fs,
                                               V3<typename F::R> Ts, const typename F::Aux &aux, float &disp,
                                               float &disp2, float &speed, const typename F::R4 *qsrc)
{
    using R = typename F::R;
    using R4 = typename F::R4;
    const int ap = stp->acc_par;
    const float acc0 = (float)v4.w, acc1 = (float)w4.w;      // acc[0], acc[1]
    const float acc_a = ap == 0 ? acc0 : acc1, acc_b = ap == 0 ? acc1 : acc0;
    float a0 = acc_a, a1 = acc_b;
    const int so = sp ^ 1;
    V3<R> vn = {v4.x, v4.y, v4.z}, wn = {w4.x, w4.y, w4.z};
    // single spheres: a sphere that does not turn in a step keeps its orientation as it is
    // (no rotation, no renormalisation).  While a sphere's stored angular velocity is zero
    // both orientation buffers hold the same quaternion (uploads and restores write both;
    // a step that ends with zero angular velocity writes both), so such a step reads and
    // writes no quaternion.  With qsrc set, q4 was not read and is fetched from there if
    // the sphere turns.
    const bool w_zero0 = w4.x == R(0) && w4.y == R(0) && w4.z == R(0);
    bool q_valid = qsrc == nullptr;
    bool rot = true;
    R qw = q4.x, qx = q4.y, qy = q4.z, qz = q4.w;
    auto fetch_q = [&]() {
        if (!q_valid) {
            const R4 qq = *qsrc;
            qw = qq.x; qx = qq.y; qy = qq.z; qz = qq.w;
            q_valid = true;
        }
    };
    uint8_t active_out = act ? 1 : 0;
    typename F::Pos pn = po;
    if (act) {
        const R h = F::voxel ? (R)sc.hf : (R)sc.h;
        const V3<R> g = F::voxel ? V3<R>{(R)sc.gf[0], (R)sc.gf[1], (R)sc.gf[2]}
                                 : V3<R>{(R)sc.g[0], (R)sc.g[1], (R)sc.g[2]};
        const V3<R> Ft = vadd_rn(Fs, vscale_rn(mass, g));
        vn = vadd_rn(vn, vscale_rn(h, vscale_rn(im, Ft)));
        // prescribed motion of the owner's family replaces what the forces give
        const FamilyMotion *pm = d.owner_family ? &d.fam_motion[d.owner_family[o]] : nullptr;
        if (pm && pm->fix_v) {
            if constexpr (F::voxel) vn = {pm->vf[0], pm->vf[1], pm->vf[2]};
            else vn = {(R)pm->v[0], (R)pm->v[1], (R)pm->v[2]};
        }
        R nw = qw, nx = qx, ny = qy, nz = qz;
        if (pm && pm->fix_w) {
            // turn by the prescribed (global-frame) angular velocity: q <- dq(h w) q
            if constexpr (F::voxel) wn = {pm->wf[0], pm->wf[1], pm->wf[2]};
            else wn = {(R)pm->w[0], (R)pm->w[1], (R)pm->w[2]};
            rot = CLUMPS || !(wn.x == R(0) && wn.y == R(0) && wn.z == R(0));
            if (rot) {
                fetch_q();
                R dw, dx, dy, dz;
                quat_increment<R>(wn, h, dw, dx, dy, dz);
                quat_mul<R>(dw, dx, dy, dz, qw, qx, qy, qz, nw, nx, ny, nz);
            }
        } else if (iso) {
            // isotropic inertia: the body-frame update equals a world-frame one
            wn = vadd_rn(wn, vscale_rn(h, vscale_rn(ii.x, Ts)));
            rot = CLUMPS || !(wn.x == R(0) && wn.y == R(0) && wn.z == R(0));
            if (rot) {
                fetch_q();
                R dw, dx, dy, dz;
                quat_increment<R>(wn, h, dw, dx, dy, dz);
                quat_mul<R>(dw, dx, dy, dz, qw, qx, qy, qz, nw, nx, ny, nz);
            }
        } else {
            fetch_q();
            R m[9];
            quat_mat_rn<R>(qw, qx, qy, qz, m);
            V3<R> wb = mat_tvec_rn<R>(m, wn);
            V3<R> Tb = mat_tvec_rn<R>(m, Ts);
            V3<R> gyro = {R(0), R(0), R(0)};
            if (d.gyro) {
                V3<R> Iw = {rdiv(wb.x, ii.x), rdiv(wb.y, ii.y), rdiv(wb.z, ii.z)};
                gyro = cross_rn(wb, Iw);
            }
            V3<R> dwb = {rmul(ii.x, rsub(Tb.x, gyro.x)), rmul(ii.y, rsub(Tb.y, gyro.y)),
                         rmul(ii.z, rsub(Tb.z, gyro.z))};
            wb = vadd_rn(wb, vscale_rn(h, dwb));
            R dw, dx, dy, dz;
            quat_increment<R>(wb, h, dw, dx, dy, dz);
            quat_mul<R>(qw, qx, qy, qz, dw, dx, dy, dz, nw, nx, ny, nz);
            R qn = sqrt(radd(radd(radd(rmul(nw, nw), rmul(nx, nx)), rmul(ny, ny)), rmul(nz, nz)));
            R m2[9];
            quat_mat_rn<R>(rdiv(nw, qn), rdiv(nx, qn), rdiv(ny, qn), rdiv(nz, qn), m2);
            wn = mat_vec_rn<R>(m2, wb);
        }
        if (rot) {
            R qn = sqrt(radd(radd(radd(rmul(nw, nw), rmul(nx, nx)), rmul(ny, ny)), rmul(nz, nz)));
            qw = rdiv(nw, qn); qx = rdiv(nx, qn); qy = rdiv(ny, qn); qz = rdiv(nz, qn);
        }
        pn = F::advance(po, vscale_rn(h, vn), d.L);
        if (sc.has_sink) {
            V3<double> pa = F::absolute(pn, sc, d.Ld);
            double side = radd(radd(rmul(rsub(pa.x, sc.sink_p[0]), sc.sink_n[0]),
                                    rmul(rsub(pa.y, sc.sink_p[1]), sc.sink_n[1])),
                               rmul(rsub(pa.z, sc.sink_p[2]), sc.sink_n[2]));
            if (side < 0.0) {
                active_out = 0;
                vn = {R(0), R(0), R(0)};
                wn = {R(0), R(0), R(0)};
            }
        }
        R sv = sqrt(dot_rn(vn, vn));
        R sw = sqrt(dot_rn(wn, wn));
        speed = (float)sv;
        // displacement bound of this step (centre moves h|v|, a component centre at
        // most h|w| r_ext more) plus the rounding slack of the position update,
        // accumulated per owner since each list's snapshot
        const float step_d = radd(rmul((float)rmul(h, radd(sv, rmul(sw, ii.w))), 1.0000005f), stp->disp_slack_f);
        a0 = acc_a + step_d;
        a1 = acc_b + step_d;
        disp = a0;
        disp2 = a1;
        if (d.amag) d.amag[o] = (float)rmul(sqrt(dot_rn(Ft, Ft)), im);
        if constexpr (F::voxel) {
            if (sc.v_errf > 0.0f && !(sv <= sc.v_errf)) atomicOr(&stp->diverged, 1);
        } else {
            if (sc.v_err > 0.0 && !((double)sv <= sc.v_err)) atomicOr(&stp->diverged, 1);
        }
        if (!(sv == sv) || !(sw == sw)) atomicOr(&stp->diverged, 1);
    } else {
        vn = {R(0), R(0), R(0)};
        wn = {R(0), R(0), R(0)};
    }
    typename F::PosStore pos_out = d.st.pos[so];
    F::store(pos_out, o, pn, mass, aux);
    d.st.kv[so][2 * o] = R4{vn.x, vn.y, vn.z, (R)(ap == 0 ? a0 : a1)};
    d.st.kv[so][2 * o + 1] = R4{wn.x, wn.y, wn.z, (R)(ap == 0 ? a1 : a0)};
    if constexpr (CLUMPS) {
        d.st.quat[so][o] = R4{qw, qx, qy, qz};
    } else {
        const bool w_zero1 = wn.x == R(0) && wn.y == R(0) && wn.z == R(0);
        // !act: the orientation is kept, as in a step without rotation
        const bool turned = act && rot;
        if (turned || !w_zero0) {
            fetch_q();      // turned: already current; otherwise the stored orientation
            d.st.quat[so][o] = R4{qw, qx, qy, qz};
            // a turned sphere that ends at rest: both buffers hold its new orientation
            if (turned && w_zero1) d.st.quat[sp][o] = R4{qw, qx, qy, qz};
        }
    }
    d.st.active[so][o] = active_out;
}

// integrate_core with the inputs read from src (global state arrays or a staged tile)
// and the contact force and torque from the per-owner arrays written by k_contact.
// FREE (single spheres whose owners with listed partners the contact kernel integrates):
// every owner here has zero contact force and torque, so neither the force array nor the
// inverse inertia is read; a single sphere's r_ext is 0 and the torque term adds exactly
// zero whatever its inverse inertia, so the results are the same bits.
template <class F, bool CLUMPS, bool FREE = false>
__device__ __forceinline__ void integrate_owner(const Dev<F> &d, DevStatus *stp, int64_t o, const OwnerSrc<F> &src,
                                                int64_t i, int sp, float &disp, float &disp2, float &speed)
{
    static_assert(!FREE || !CLUMPS, "FREE is for single spheres");
    using R = typename F::R;
    using R4 = typename F::R4;
    // every load of this owner is issued before the first one is used: the thread waits
    // for one memory round trip, not a chain of them
    const bool act = src.active[i];
    // the flag is read beside the row length, not after it (both are always valid)
    const uint8_t touched = (FREE || CLUMPS) ? (uint8_t)1 : d.touched[o];
    const bool has = FREE ? false : (CLUMPS ? true : (src.cnt[i] > 0) & (touched != 0));
    R mass;
    typename F::Aux aux;
    const typename F::Pos po = F::load(src.pos, i, mass, aux);
    const R4 v4 = src.kv[2 * i], w4 = src.kv[2 * i + 1];
    // clumps read their orientation at once; a single sphere's is read only if it turns
    const R4 q4 = CLUMPS ? src.quat[i] : R4{};
    R im;
    R4 ii;
    if (!CLUMPS && F::voxel && d.solid) {
        float rad = 0.0f;
        if constexpr (F::voxel) rad = aux.rad;
        solid_consts<F>(d, mass, rad, im, ii);
        if (FREE) ii = R4{R(0), R(0), R(0), R(0)};
    } else {
        im = src.inv_mass[i];
        ii = FREE ? R4{R(0), R(0), R(0), R(0)} : src.inv_moi[i];
    }
    const bool iso = CLUMPS ? (bool)src.iso[i] : true;     // a single sphere is isotropic
    const Scene &sc = d.scenes[d.n_scenes > 1 ? src.scene[i] : 0];
    V3<R> Fs = {R(0), R(0), R(0)}, Ts = {R(0), R(0), R(0)};
    if (act && has) {
        const R4 f4 = d.fo[o], t4 = d.to[o];
        Fs = {f4.x, f4.y, f4.z};
        Ts = {t4.x, t4.y, t4.z};
    }
    integrate_core<F, CLUMPS>(d, stp, o, sp, act, po, mass, v4, w4, q4, im, ii, iso, sc, Fs, Ts, aux, disp, disp2,
                              speed, CLUMPS ? nullptr : &src.quat[i]);
}

// One thread per owner, reading its inputs straight from the state arrays.
// SKIP_LISTED (single spheres): owners that are active with listed partners are left to
// the contact kernel, which integrates them (k_contact<..., INTEG>).
template <class F, bool CLUMPS, bool SKIP_LISTED = false>
__global__ void __launch_bounds__(INTEGRATE_BLOCK_MAX) k_integrate(Dev<F> d)
{
    static_assert(!SKIP_LISTED || !CLUMPS, "only single spheres are integrated by the contact kernel");
    DevStatus *stp = d.status;
    if (stp->halt || stp->list_stale) return;
    const int sp = stp->state_par, lc = stp->list_cur;
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    float disp = 0.0f, disp2 = 0.0f, speed = 0.0f;
    if (o < d.M && !(SKIP_LISTED && d.st.active[sp][o] && d.lists.cnt[lc][o] > 0)) {
        OwnerSrc<F> src{d.st.pos[sp], d.st.kv[sp], d.st.quat[sp], d.inv_moi, d.inv_mass,
                        d.st.active[sp], d.lists.cnt[lc], d.owner_iso, d.owner_scene};
        integrate_owner<F, CLUMPS, SKIP_LISTED>(d, stp, o, src, o, sp, disp, disp2, speed);
    }
    audit_slots(d.audit, o, lane, disp, disp2, speed);
}

// ------------------------------------------------------------------ fused step

// One step of a world of single spheres in one kernel: a thread takes one sphere, sums
// the contact forces of its listed entries in registers (pair_sums, as k_contact) and
// integrates its owner at once (integrate_core, as k_integrate) into the other state
// buffer.  The owner state is read once and no per-owner force array is written or
// read.  Each block of 256 slots is taken in the order of the list's row-length
// permutation of that block (written by k_compact), so the lanes of a warp loop over
// rows of equal length.  Bit-identical to k_contact followed by k_integrate: the same
// arithmetic in the same order for every sphere.
constexpr int FUSED_BLOCK_MAX = 256;

template <class F>
__global__ void __launch_bounds__(FUSED_BLOCK_MAX, 2) k_step_fused(Dev<F> d)
{
    using R = typename F::R;
    using R4 = typename F::R4;
    DevStatus *stp = d.status;
    if (stp->halt || stp->list_stale) return;
    const int sp = stp->state_par, hp = stp->hist_par, lc = stp->list_cur;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    float disp = 0.0f, disp2 = 0.0f, speed = 0.0f;
    // perm holds positions within the slot's own 256-block: s stays below Np
    const int64_t s = g < d.Np ? (g & ~(int64_t)255) + d.lists.perm[lc][g] : d.M;
    if (s < d.M) {
        const int n = d.lists.cnt[lc][s];
        const uint32_t j0 = d.lists.partner[lc][s];      // entry 0 of the row (unused when n = 0)
        const bool act = d.st.active[sp][s];
        SphereK<F> me;
        typename F::Aux aux;
        const typename F::Pos po = F::load(d.st.pos[sp], s, me.mass, aux);
        const R4 v4 = d.st.kv[sp][2 * s], w4 = d.st.kv[sp][2 * s + 1];
        const Scene &sc = d.scenes[d.n_scenes > 1 ? d.owner_scene[s] : 0];
        me.p = po;
        me.rl = {R(0), R(0), R(0)};
        me.v = {v4.x, v4.y, v4.z};
        me.w = {w4.x, w4.y, w4.z};
        if constexpr (F::voxel) {
            // the radius rides in the position record; the material is needed only
            // where the scene has several
            me.rad = aux.rad;
            me.rlo = aux.rlo;
            me.mat = sc.n_mat == 1 ? sc.mat_base : (int)d.sph_mat[s];
        } else {
            const auto pk = d.sph_pack[s];
            me.rad = pk.x;
            me.rlo = 0.0f;
            me.mat = (int)pk.y;
        }
        me.owner = (uint32_t)s;
        V3<R> Fs = {R(0), R(0), R(0)}, Ts = {R(0), R(0), R(0)};
        if (act && n > 0) pair_sums<F, false, MODE_STEP>(d, me, sc, s, n, j0, sp, hp, lc, Fs, Ts);
        R im;
        R4 ii;
        if (F::voxel && d.solid) {
            solid_consts<F>(d, me.mass, (float)me.rad, im, ii);
        } else {
            im = d.inv_mass[s];
            ii = d.inv_moi[s];
        }
        integrate_core<F, false>(d, stp, s, sp, act, po, me.mass, v4, w4, R4{}, im, ii, true, sc, Fs, Ts, aux, disp,
                                 disp2, speed, &d.st.quat[sp][s]);
    }
    audit_slots(d.audit, g, lane, disp, disp2, speed);
}

// ------------------------------------------------------------------ staged integration
// The same update with the inputs streamed through shared memory: a persistent block
// walks tiles of ITILE owners; one thread issues bulk asynchronous copies (TMA) of a
// whole tile of every input array, completed on an mbarrier, two tiles ahead, so all of
// a tile's bytes are in flight at once while the previous tile is computed.  Voxel form
// only (its arrays are 16-byte vectors or packed scalars; owner arrays are allocated in
// whole tiles so every copy is a full, 16-byte-aligned tile).
constexpr int ITILE = 256;
struct StageLayout {                                        // byte offsets within a stage
    static constexpr int rec = 0;                           // 32-byte position records
    static constexpr int kv = rec + 32 * ITILE;             // float4 (v, acc[0]), (w, acc[1])
    static constexpr int quat = kv + 32 * ITILE;            // float4 q
    static constexpr int moi = quat + 16 * ITILE;           // float4 1/I, r_ext
    static constexpr int imass = moi + 16 * ITILE;          // float 1/m
    static constexpr int active = imass + 4 * ITILE;        // u8
    static constexpr int flags = active + ITILE;            // u8 row length (spheres) / isotropy (clumps)
    static constexpr int scene = flags + ITILE;             // u16 scene (several scenes only)
    static constexpr int bytes = scene + 2 * ITILE;
};
constexpr int STAGES = 2;
constexpr uint64_t STAGE_WAIT_NS = 1000000000ull;           // a copy later than this is a fault

template <bool CLUMPS>
__global__ void __launch_bounds__(ITILE) k_integrate_staged(Dev<FormF32> d)
{
    using F = FormF32;
    extern __shared__ __align__(128) unsigned char stage_mem[];
    __shared__ uint64_t bar[STAGES];
    __shared__ int skip;
    DevStatus *stp = d.status;
    // one reading of the flags for the whole block: its threads leave together or not at all
    if (threadIdx.x == 0) skip = (stp->halt || stp->list_stale) ? 1 : 0;
    __syncthreads();
    if (skip) return;
    const int sp = stp->state_par, lc = stp->list_cur;
    const int64_t ntiles = (d.M + ITILE - 1) / ITILE;
    const bool scenes = d.n_scenes > 1;
    // derived constants (Dev::solid): the 1/I and 1/m arrays are not copied
    const bool solid = !CLUMPS && d.solid;
    const uint32_t tile_bytes =
        (uint32_t)(StageLayout::scene + (scenes ? 2 * ITILE : 0) - (solid ? (16 + 4) * ITILE : 0));
    const int lane = threadIdx.x & 31;
    const uint64_t deadline = global_ns() + STAGE_WAIT_NS;

    auto issue = [&](int64_t tile, int st) {
        unsigned char *b = stage_mem + st * StageLayout::bytes;
        const int64_t o0 = tile * ITILE;
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(&bar[st], tile_bytes);
        bulk_g2s(b + StageLayout::rec, d.st.pos[sp].rec + o0, 32 * ITILE, &bar[st]);
        bulk_g2s(b + StageLayout::kv, d.st.kv[sp] + 2 * o0, 32 * ITILE, &bar[st]);
        bulk_g2s(b + StageLayout::quat, d.st.quat[sp] + o0, 16 * ITILE, &bar[st]);
        if (!solid) {
            bulk_g2s(b + StageLayout::moi, d.inv_moi + o0, 16 * ITILE, &bar[st]);
            bulk_g2s(b + StageLayout::imass, d.inv_mass + o0, 4 * ITILE, &bar[st]);
        }
        bulk_g2s(b + StageLayout::active, d.st.active[sp] + o0, ITILE, &bar[st]);
        bulk_g2s(b + StageLayout::flags, CLUMPS ? (const void *)(d.owner_iso + o0) : (const void *)(d.lists.cnt[lc] + o0),
                 ITILE, &bar[st]);
        if (scenes) bulk_g2s(b + StageLayout::scene, d.owner_scene + o0, 2 * ITILE, &bar[st]);
    };

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) mbar_init(&bar[st], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st)
            if (blockIdx.x + (int64_t)st * gridDim.x < ntiles) issue(blockIdx.x + (int64_t)st * gridDim.x, st);
    }
    int k = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int st = k % STAGES;
        const bool ok = mbar_wait(&bar[st], (uint32_t)((k / STAGES) & 1), deadline);
        if (__syncthreads_or(!ok)) {
            // a tile did not arrive in time: report it, let the copies still in flight
            // land (bounded again) so that none writes into a finished block, and leave
            if (threadIdx.x == 0) {
                atomicCAS(&stp->halt, HALT_NONE, HALT_TIMEOUT);
                const uint64_t late = global_ns() + STAGE_WAIT_NS;
                for (int q = 0; q < STAGES; ++q) {
                    const int64_t t = tile + (int64_t)q * gridDim.x;
                    if (t < ntiles) mbar_wait(&bar[(k + q) % STAGES], (uint32_t)(((k + q) / STAGES) & 1), late);
                }
            }
            __syncthreads();
            return;
        }
        unsigned char *b = stage_mem + st * StageLayout::bytes;
        const int64_t o = tile * ITILE + threadIdx.x;
        float disp = 0.0f, disp2 = 0.0f, speed = 0.0f;
        if (o < d.M) {
            const uint8_t *flags = b + StageLayout::flags;
            OwnerSrc<F> src{F::PosStore{reinterpret_cast<F::PosRec *>(b + StageLayout::rec)},
                            reinterpret_cast<const float4 *>(b + StageLayout::kv),
                            reinterpret_cast<const float4 *>(b + StageLayout::quat),
                            reinterpret_cast<const float4 *>(b + StageLayout::moi),
                            reinterpret_cast<const float *>(b + StageLayout::imass),
                            b + StageLayout::active, flags, flags,
                            reinterpret_cast<const uint16_t *>(b + StageLayout::scene)};
            integrate_owner<F, CLUMPS>(d, stp, o, src, threadIdx.x, sp, disp, disp2, speed);
        }
        audit_slots(d.audit, o, lane, disp, disp2, speed);
        __syncthreads();                          // every thread has read this stage
        const int64_t next = tile + (int64_t)STAGES * gridDim.x;
        if (threadIdx.x == 0 && next < ntiles) issue(next, st);
    }
}

// Completes a step (single thread): flips the state and history buffers, takes the largest
// per-owner displacement bound of the list in use and of the list being built, and flags
// the list stale when its bound exceeds the margin (Sec. 2.1: the margin must cover the
// motion between list updates); turns a divergence into a halt, leaving the last good
// state.  A pair touching now was, at the snapshot, at most R_i + R_j + acc_i + acc_j
// apart, so every touching pair is listed while the largest acc stays below the margin.
static __global__ void k_audit(DevStatus *stp, unsigned int *audit)
{
    // one warp: each lane reads and clears AUDIT_SLOTS / 32 slots, a warp max combines them
    // (the screening pass's counter restarts after every step, whatever happened in it)
    if (threadIdx.x == 0) stp->n_screen = 0;
    if (stp->halt || stp->list_stale) return;
    const int lane = threadIdx.x & 31;
    unsigned int md = 0, md2 = 0, mv = 0;
    for (int k = lane; k < AUDIT_SLOTS; k += 32) {
        unsigned int *slot = audit + k * AUDIT_STRIDE;
        md = max(md, slot[0]);
        md2 = max(md2, slot[1]);
        mv = max(mv, slot[2]);
        slot[0] = 0;
        slot[1] = 0;
        slot[2] = 0;
    }
    md = __reduce_max_sync(0xffffffffu, md);
    md2 = __reduce_max_sync(0xffffffffu, md2);
    mv = __reduce_max_sync(0xffffffffu, mv);
    if (lane != 0) return;
    float sd = __uint_as_float(md);
    float sd2 = __uint_as_float(md2);
    float vm = __uint_as_float(mv);
    if (stp->diverged || !(sd == sd) || !(vm == vm)) {
        stp->halt = HALT_DIVERGED;
        return;
    }
    stp->steps_done += 1;
    stp->pair_steps += stp->list_pairs[stp->list_cur];
    stp->busy_steps += stp->list_busy[stp->list_cur];
    stp->state_par ^= 1;
    stp->hist_par ^= 1;
    // largest per-owner accumulated bound of each list (owners accumulate on their own)
    stp->disp_cur = (double)sd;
    stp->disp_next = (double)sd2;
    stp->vmax_last = (double)vm;
    if (stp->disp_cur > stp->beta_cur) {
        stp->list_stale = 1;
        stp->stale_events += 1;
    }
}

// ------------------------------------------------------------------ learned schedule

// Bin of an owner: its centre of mass's cell of the smallest size divided by BIN_CELLS
// per axis (independent of the detection cell size).
template <class F>
__device__ __forceinline__ int owner_bin(const Dev<F> &d, int sp, int64_t o, const Scene &sc)
{
    typename F::R mass;
    typename F::Pos p = F::load(d.st.pos[sp], o, mass);
    int cx, cy, cz;
    F::cell(p, sc, d.bin_invL, d.bin_vpc, cx, cy, cz);
    cx = min(max(cx, 0), sc.nbc[0] - 1) / BIN_CELLS;
    cy = min(max(cy, 0), sc.nbc[1] - 1) / BIN_CELLS;
    cz = min(max(cz, 0), sc.nbc[2] - 1) / BIN_CELLS;
    return sc.bin_base + (cz * sc.nb[1] + cy) * sc.nb[0] + cx;
}

// Per-bin motion statistics of the active owners: count, sum |v|, sum |v|^2, max |v|,
// sum |a|, max |a|, sum |w| r_ext, max |w| r_ext, sum of list rows, max list row.  Also
// records each owner's bin (for labels).  Neighbouring owners mostly share a bin, so each
// warp first reduces runs of consecutive lanes in the same bin (segmented shuffles) and
// only the first lane of a run updates the bin: about one set of atomics per run instead
// of one per owner.  Float atomics: order-dependent last bits only affect the schedule's
// choice, never the trajectory (lists are audited).
template <class F>
__global__ void __launch_bounds__(256) k_bin_stats(Dev<F> d, float *stats, int *obin)
{
    const int sp = d.status->state_par, lc = d.status->list_cur;
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int b = -1;                                   // -1: no contribution (past the end, inactive)
    float x[NSTAT] = {};
    if (o < d.M) {
        const Scene &sc = d.scenes[d.owner_scene[o]];
        const int bo = owner_bin(d, sp, o, sc);
        obin[o] = bo;
        if (d.st.active[sp][o]) {
            b = bo;
            auto v4 = d.st.kv[sp][2 * o];
            auto w4 = d.st.kv[sp][2 * o + 1];
            float v = sqrtf((float)(v4.x * v4.x + v4.y * v4.y + v4.z * v4.z));
            float wr = sqrtf((float)(w4.x * w4.x + w4.y * w4.y + w4.z * w4.z)) * (float)d.inv_moi[o].w;
            float a = d.amag ? d.amag[o] : 0.0f;
            float rows = 0.0f, rmax = 0.0f;
            const int64_t first = d.owner_first[o];
            for (int c = 0; c < (int)d.owner_nsph[o]; ++c) {     // list rows of the owner's spheres
                float r = (float)d.lists.cnt[lc][first + c];
                rows += r;
                rmax = fmaxf(rmax, r);
            }
            x[0] = 1.0f; x[1] = v; x[2] = v * v; x[3] = v; x[4] = a; x[5] = a; x[6] = wr; x[7] = wr;
            x[8] = rows; x[9] = rmax;
        }
    }
    // runs of equal bins within the warp: a lane heads a run when its bin differs from the
    // previous lane's; each lane reduces towards the head over the lanes of its run
    const int prev = __shfl_up_sync(0xffffffffu, b, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != b);
    const unsigned above = heads & ~((2u << lane) - 1u);
    const int end = above ? __ffs(above) - 1 : 32;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int k = 0; k < NSTAT; ++k) {
            const float y = __shfl_down_sync(0xffffffffu, x[k], off);
            if (lane + off < end) x[k] = (k == 3 || k == 5 || k == 7 || k == 9) ? fmaxf(x[k], y) : x[k] + y;
        }
    }
    if (b < 0 || !((heads >> lane) & 1u)) return;
    float *st = stats + (int64_t)b * NSTAT;
    atomicAdd(&st[0], x[0]);
    atomicAdd(&st[1], x[1]);
    atomicAdd(&st[2], x[2]);
    atomicMax(reinterpret_cast<unsigned int *>(&st[3]), __float_as_uint(x[3]));
    atomicAdd(&st[4], x[4]);
    atomicMax(reinterpret_cast<unsigned int *>(&st[5]), __float_as_uint(x[5]));
    atomicAdd(&st[6], x[6]);
    atomicMax(reinterpret_cast<unsigned int *>(&st[7]), __float_as_uint(x[7]));
    atomicAdd(&st[8], x[8]);
    atomicMax(reinterpret_cast<unsigned int *>(&st[9]), __float_as_uint(x[9]));
}

// The 16 features of each bin, made dimensionless with the step h and the margin beta
// (displacements per step over beta); X[bin][16], valid[bin] = owners present.
static __global__ void k_bin_features(const float *stats, int nbins, const int *bin_scene, const Scene *scenes, float beta,
                               float r_max, float *X, int *valid)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const float *st = stats + (int64_t)b * NSTAT;
    const Scene &sc = scenes[bin_scene[b]];
    const float n = st[0];
    float *x = X + (int64_t)b * 16;
    valid[b] = n > 0.0f ? 1 : 0;
    const float inv = n > 0.0f ? 1.0f / n : 0.0f;
    const float q = sc.hf / fmaxf(beta, 1e-30f);
    const float mv = st[1] * inv;
    const float sv = sqrtf(fmaxf(st[2] * inv - mv * mv, 0.0f));
    const float g = sqrtf(sc.gf[0] * sc.gf[0] + sc.gf[1] * sc.gf[1] + sc.gf[2] * sc.gf[2]);
    x[0] = log2f(1.0f + n) / 8.0f;
    x[1] = st[3] * q;
    x[2] = mv * q;
    x[3] = sv * q;
    x[4] = st[5] * sc.hf * q;
    x[5] = st[4] * inv * sc.hf * q;
    x[6] = st[7] * q;
    x[7] = st[6] * inv * q;
    x[8] = st[8] * inv / 16.0f;
    x[9] = st[9] / 16.0f;
    x[10] = g * sc.hf * q;
    x[11] = log2f(1.0f + 1.0f / (x[1] + x[6] + 1e-6f)) / 16.0f;
    x[12] = sqrtf(x[4]);
    x[13] = x[1] + x[6];
    x[14] = beta / fmaxf(r_max, 1e-30f);
    x[15] = 1.0f;
}

// Labels: after each step of a collection window, owners accumulate their displacement
// bound; the first step at which an owner of a bin passes beta / 2 and beta is recorded
// per bin (atomicMin over owners: order-independent).
template <class F>
__global__ void __launch_bounds__(256) k_collect_step(Dev<F> d, float *acc_lab, const int *obin, int *cross,
                                                      long long window_start, float beta)
{
    const DevStatus *stp = d.status;
    int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= d.M) return;
    const int sp = stp->state_par;
    if (!d.st.active[sp][o]) return;
    const Scene &sc = d.scenes[d.owner_scene[o]];
    auto v4 = d.st.kv[sp][2 * o];
    auto w4 = d.st.kv[sp][2 * o + 1];
    float v = sqrtf((float)(v4.x * v4.x + v4.y * v4.y + v4.z * v4.z));
    float w = sqrtf((float)(w4.x * w4.x + w4.y * w4.y + w4.z * w4.z));
    float a0 = acc_lab[o];
    float a1 = a0 + sc.hf * (v + w * (float)d.inv_moi[o].w);
    acc_lab[o] = a1;
    const int k = (int)(stp->steps_done - window_start);
    const int b = obin[o];
    if (a0 <= 0.5f * beta && a1 > 0.5f * beta) atomicMin(&cross[2 * b + 1], k);
    if (a0 <= beta && a1 > beta) atomicMin(&cross[2 * b + 0], k);
}

// Smallest predicted log2(steps) over the occupied bins (one block, fixed order).  The
// network predicts the residual over the kinematic estimate log2(beta / (h (|v| + |w| r)
// max)) = -log2(feature 13), added back here.
static __global__ void __launch_bounds__(256) k_min_pred(const float *out, const float *X, const int *valid, int nbins,
                                                         float *res)
{
    __shared__ float red[256];
    float m = 1e30f;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (valid[b]) m = fminf(m, out[2 * b] - log2f(fmaxf(X[(int64_t)b * 16 + 13], 1e-6f)));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fminf(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *res = red[0];
}

// ------------------------------------------------------------------ read-back helpers

// Evaluate every owned entry (canonical sphere pairs and wall entries) at the current
// state: overlap (<= 0 if not in contact), force on A, contact point and updated history.
template <class F, bool CLUMPS>
__global__ void __launch_bounds__(128) k_contacts(Dev<F> d, double *ov, double *fo, double *pt, double *hi,
                                                  double *ag, double *rf)
{
    using R = typename F::R;
    DevStatus *stp = d.status;
    const int sp = stp->state_par, hp = stp->hist_par, lc = stp->list_cur;
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.N) return;
    uint32_t o = d.sph_owner[s];
    if (o == 0xffffffffu) return;
    SphereK<F> me = load_sphere<F, CLUMPS>(d, sp, (uint32_t)s);
    const Scene &sc = d.scenes[d.owner_scene[o]];
    const R h = F::voxel ? (R)sc.hf : (R)sc.h;
    const bool act = d.st.active[sp][o];
    const int n = d.lists.cnt[lc][s];
    for (int k = 0; k < n; ++k) {
        int64_t e = (int64_t)k * d.Np + s;
        uint32_t j = d.lists.partner[lc][e];
        ov[e] = -1.0;
        if (!act) continue;
        ContactIn<R> c;
        V3<R> armA, armB;
        R age;
        V3<R> ut = hist_get<typename HistVec<R>::T, R>(d.lists.hist[hp], e, age);
        V3<R> Fc;
        V3<double> cp;
        V3<R> wB = {R(0), R(0), R(0)};
        int mb;
        if (j & WALL_BIT) {
            const Wall &wl = d.walls[j & ~WALL_BIT];
            if (!wall_contact<F>(d, me, sc, wl, c, armA, &cp)) continue;
            mb = wl.mat;
        } else {
            if (j < (uint32_t)s) continue;
            SphereK<F> B = load_sphere<F, CLUMPS>(d, sp, j);
            if (!d.st.active[sp][B.owner]) continue;
            if (!sphere_contact<F>(d, me, B, c, armA, armB)) continue;
            V3<double> pa = F::absolute(me.p, sc, d.Ld);
            double a = ((double)me.rad + (double)me.rlo) - 0.5 * (double)c.delta;
            cp = {pa.x - a * (double)c.n.x, pa.y - a * (double)c.n.y, pa.z - a * (double)c.n.z};
            wB = B.w;
            mb = B.mat;
        }
        R fn_abs;
        hertz_mindlin<R>(c, h, ut, Fc, &fn_abs);
        V3<R> Fr = {R(0), R(0), R(0)};
        if (sc.has_rolling) {
            age = advance_age<F>(age, h);
            const int pk = sc.pair_base + (me.mat - sc.mat_base) * sc.n_mat + (mb - sc.mat_base);
            const R crr = crr_table(d, R(0))[pk];
            if (crr > R(0) && !within_collision_time<R>(c, age_seconds<F>(age, h))) {
                const V3<R> rotA = cross_rn(me.w, armA);
                const V3<R> rotB = (j & WALL_BIT) ? c.uB : cross_rn(wB, armB);
                Fr = rolling_force<R>(crr, fn_abs, V3<R>{rsub(rotB.x, rotA.x), rsub(rotB.y, rotA.y),
                                                          rsub(rotB.z, rotA.z)});
            }
            age = age_seconds<F>(age, h);
        } else {
            age = R(0);
        }
        ov[e] = (double)c.delta;
        fo[3 * e + 0] = (double)Fc.x; fo[3 * e + 1] = (double)Fc.y; fo[3 * e + 2] = (double)Fc.z;
        pt[3 * e + 0] = cp.x; pt[3 * e + 1] = cp.y; pt[3 * e + 2] = cp.z;
        hi[3 * e + 0] = (double)ut.x; hi[3 * e + 1] = (double)ut.y; hi[3 * e + 2] = (double)ut.z;
        ag[e] = (double)age;
        rf[3 * e + 0] = (double)Fr.x; rf[3 * e + 1] = (double)Fr.y; rf[3 * e + 2] = (double)Fr.z;
    }
}

// Read-back through a contact model: every owned entry (canonical sphere pairs and wall
// entries) at the current state with the model's engagement (en: 1 / 0), overlap, force
// on the lower sphere, contact point, wildcards after the update (wc: 8 per entry) and
// torque-only force.
template <class F, bool CLUMPS, class Model>
__global__ void __launch_bounds__(128) k_contacts_model(Dev<F> d, double *ov, double *fo, double *pt, double *wco,
                                                        double *rf, double *en)
{
    using R = typename F::R;
    using H = typename HistVec<R>::T;
    DevStatus *stp = d.status;
    const int sp = stp->state_par, hp = stp->hist_par, lc = stp->list_cur;
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.N) return;
    uint32_t o = d.sph_owner[s];
    if (o == 0xffffffffu) return;
    SphereK<F> me = load_sphere<F, CLUMPS>(d, sp, (uint32_t)s);
    const Scene &sc = d.scenes[d.owner_scene[o]];
    const bool act = d.st.active[sp][o];
    const int n = d.lists.cnt[lc][s];
    for (int k = 0; k < n; ++k) {
        int64_t e = (int64_t)k * d.Np + s;
        uint32_t j = d.lists.partner[lc][e];
        en[e] = 0.0;
        if (!act || (!(j & WALL_BIT) && j < (uint32_t)s)) continue;
        R wc[8];
        const H a = d.lists.hist[hp][e];
        wc[0] = (R)a.x; wc[1] = (R)a.y; wc[2] = (R)a.z; wc[3] = (R)a.w;
        if (d.lists.wild[0]) {
            const H b = d.lists.wild[hp][e];
            wc[4] = (R)b.x; wc[5] = (R)b.y; wc[6] = (R)b.z; wc[7] = (R)b.w;
        } else {
            wc[4] = wc[5] = wc[6] = wc[7] = R(0);
        }
        V3<R> Fc, Fr, arm;
        R overlap;
        if (!model_entry<F, CLUMPS, Model>(d, me, sc, s, j, sp, wc, Fc, Fr, arm, overlap)) continue;
        en[e] = 1.0;
        ov[e] = (double)overlap;
        const V3<double> pa = F::absolute(me.p, sc, d.Ld);
        for (int q = 0; q < 3; ++q) {
            const double rl = q == 0 ? (double)me.rl.x : (q == 1 ? (double)me.rl.y : (double)me.rl.z);
            const double am = q == 0 ? (double)arm.x : (q == 1 ? (double)arm.y : (double)arm.z);
            const double pq = q == 0 ? pa.x : (q == 1 ? pa.y : pa.z);
            pt[3 * e + q] = (pq - rl) + am;
        }
        fo[3 * e + 0] = (double)Fc.x; fo[3 * e + 1] = (double)Fc.y; fo[3 * e + 2] = (double)Fc.z;
        rf[3 * e + 0] = (double)Fr.x; rf[3 * e + 1] = (double)Fr.y; rf[3 * e + 2] = (double)Fr.z;
        for (int q = 0; q < 8; ++q) wco[8 * e + q] = (double)wc[q];
    }
}

// Counts of the list in use: sphere pairs (each once), wall entries, and entries in
// contact (overlap > 0) at the current state.  Integer atomics: order-independent.
template <class F, bool CLUMPS>
__global__ void __launch_bounds__(256) k_count(Dev<F> d, unsigned long long *out)
{
    using R = typename F::R;
    const int sp = d.status->state_par, lc = d.status->list_cur;
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long np = 0, nw = 0, nc = 0, ne = 0;
    if (s < d.N) {
        uint32_t o = d.sph_owner[s];
        if (o != 0xffffffffu) {
            const int n = d.lists.cnt[lc][s];
            ne = n > 0 ? 1 : 0;
            const bool act = d.st.active[sp][o];
            SphereK<F> me;
            if (act) me = load_sphere<F, CLUMPS>(d, sp, (uint32_t)s);
            const Scene &sc = d.scenes[d.owner_scene[o]];
            for (int k = 0; k < n; ++k) {
                uint32_t j = d.lists.partner[lc][(int64_t)k * d.Np + s];
                ContactIn<R> c;
                V3<R> a, b;
                if (j & WALL_BIT) {
                    ++nw;
                    if (act && wall_contact<F>(d, me, sc, d.walls[j & ~WALL_BIT], c, a)) ++nc;
                } else if (j > (uint32_t)s) {
                    ++np;
                    if (act) {
                        SphereK<F> B = load_sphere<F, CLUMPS>(d, sp, j);
                        if (d.st.active[sp][B.owner] && sphere_contact<F>(d, me, B, c, a, b)) ++nc;
                    }
                }
            }
        }
    }
    np = __reduce_add_sync(0xffffffffu, (unsigned)np);
    nw = __reduce_add_sync(0xffffffffu, (unsigned)nw);
    nc = __reduce_add_sync(0xffffffffu, (unsigned)nc);
    ne = __reduce_add_sync(0xffffffffu, (unsigned)ne);
    if ((threadIdx.x & 31) == 0) {
        if (np) atomicAdd(&out[0], np);
        if (nw) atomicAdd(&out[1], nw);
        if (nc) atomicAdd(&out[2], nc);
        if (ne) atomicAdd(&out[3], ne);
    }
}

// Owner state to FP64 host layout (quaternion (w,x,y,z); angular velocity to body frame).
// Active box (Sec. 6.4): owners [first, first + n) whose centre lies inside [lo, hi]
// take family fin, the others fout.
template <class F>
__global__ void __launch_bounds__(256) k_active_box(Dev<F> d, int64_t first, int64_t n, double3 lo, double3 hi,
                                                    int fin, int fout, uint8_t *family)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = first + k;
    const int sp = d.status->state_par;
    typename F::R mass;
    const typename F::Pos p = F::load(d.st.pos[sp], o, mass);
    const V3<double> x = F::absolute(p, d.scenes[d.owner_scene[o]], d.Ld);
    const bool in = x.x >= lo.x && x.x <= hi.x && x.y >= lo.y && x.y <= hi.y && x.z >= lo.z && x.z <= hi.z;
    family[o] = (uint8_t)(in ? fin : fout);
}

// Owner state in the FP64 host layout (position, orientation, velocity, body-frame
// angular velocity; 3, 4, 3 and 3 doubles per owner), each output optional (null: not
// written).  A block of 256 owners stages its values in shared memory and writes each
// array as one contiguous run of whole warps' 8-byte stores, so that the outputs may be
// mapped host memory written across the host link without partial lines.
constexpr int DOWNLOAD_BLOCK = 256;
template <class F>
__global__ void __launch_bounds__(DOWNLOAD_BLOCK) k_owner_download(Dev<F> d, int64_t first, int64_t n, double *x,
                                                                   double *q, double *v, double *w)
{
    using R = typename F::R;
    __shared__ double sx[3 * DOWNLOAD_BLOCK], sq[4 * DOWNLOAD_BLOCK], sv[3 * DOWNLOAD_BLOCK],
        sw[3 * DOWNLOAD_BLOCK];
    const int t = threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.x * DOWNLOAD_BLOCK;
    const int64_t k = k0 + t;
    if (k < n) {
        const int64_t o = first + k;
        const int sp = d.status->state_par;
        R mass;
        typename F::Pos p = F::load(d.st.pos[sp], o, mass);
        const Scene &sc = d.scenes[d.owner_scene[o]];
        const V3<double> pa = F::absolute(p, sc, d.Ld);
        sx[3 * t] = pa.x; sx[3 * t + 1] = pa.y; sx[3 * t + 2] = pa.z;
        const auto q4 = d.st.quat[sp][o];
        sq[4 * t] = q4.x; sq[4 * t + 1] = q4.y; sq[4 * t + 2] = q4.z; sq[4 * t + 3] = q4.w;
        const auto v4 = d.st.kv[sp][2 * o];
        sv[3 * t] = v4.x; sv[3 * t + 1] = v4.y; sv[3 * t + 2] = v4.z;
        const auto w4 = d.st.kv[sp][2 * o + 1];
        R m[9];
        quat_mat<R>(q4.x, q4.y, q4.z, q4.w, m);
        const V3<R> wb = mat_tvec<R>(m, V3<R>{w4.x, w4.y, w4.z});
        sw[3 * t] = wb.x; sw[3 * t + 1] = wb.y; sw[3 * t + 2] = wb.z;
    }
    __syncthreads();
    const int nb = (int)min((int64_t)DOWNLOAD_BLOCK, n - k0);
    if (x) for (int i = t; i < 3 * nb; i += DOWNLOAD_BLOCK) x[3 * k0 + i] = sx[i];
    if (q) for (int i = t; i < 4 * nb; i += DOWNLOAD_BLOCK) q[4 * k0 + i] = sq[i];
    if (v) for (int i = t; i < 3 * nb; i += DOWNLOAD_BLOCK) v[3 * k0 + i] = sv[i];
    if (w) for (int i = t; i < 3 * nb; i += DOWNLOAD_BLOCK) w[3 * k0 + i] = sw[i];
}

// FP64 host layout to owner state (both buffers' current one); world-frame angular
// velocity stored.  In the voxel form the position is split into voxel index and
// offset: c = floor((x - lo) / L), o = (float)((x - lo) - c L), then carried into [0, L).
// bounds: 0 restarts the audit accumulators (the upload at initialisation); 1 (a state
// upload between steps) adds each owner's displacement by the upload, rounded up, to
// both of them, and the largest accumulator of the list in use goes to
// upload_disp_bits, so that the host keeps the list where no owner moved past its
// margin; 2 leaves them as they are.  inv_ld: the reciprocal of the voxel edge where
// that edge is a power of two (the quotient by it is then a product), else 0.
template <class F>
__device__ __forceinline__ unsigned int owner_upload_one(const Dev<F> &d, int64_t first, int64_t k, const double *x,
                                                         const double *q, const double *v, const double *w,
                                                         const uint8_t *act, int bounds, double inv_ld)
{
    using R = typename F::R;
    using R4 = typename F::R4;
    unsigned int bits = 0;
    const int64_t o = first + k;
    const int sp = d.status->state_par;
    R mass;
    typename F::Aux aux;
    typename F::Pos p = F::load(d.st.pos[sp], o, mass, aux);
    const Scene &sc = d.scenes[d.owner_scene[o]];
    float moved_f = 0.0f;
    const typename F::Pos p0 = p;
    if (x) {
        if constexpr (F::voxel) {
            PosF32 &pv = p;
            double rx = rsub(x[3 * k], sc.lo[0]), ry = rsub(x[3 * k + 1], sc.lo[1]), rz = rsub(x[3 * k + 2], sc.lo[2]);
            // the voxel edge is a power of two: scaling by its reciprocal is the quotient
            // exactly, without a division per coordinate (slow in FP64)
            double fx, fy, fz;
            if (inv_ld > 0.0) {
                fx = floor(rx * inv_ld); fy = floor(ry * inv_ld); fz = floor(rz * inv_ld);
            } else {
                fx = floor(__ddiv_rn(rx, d.Ld)); fy = floor(__ddiv_rn(ry, d.Ld)); fz = floor(__ddiv_rn(rz, d.Ld));
            }
            pv.cx = (int)fx; pv.cy = (int)fy; pv.cz = (int)fz;
            pv.x = (float)rsub(rx, rmul(fx, d.Ld));
            pv.y = (float)rsub(ry, rmul(fy, d.Ld));
            pv.z = (float)rsub(rz, rmul(fz, d.Ld));
            FormF32::carry(pv.cx, pv.x, d.L);
            FormF32::carry(pv.cy, pv.y, d.L);
            FormF32::carry(pv.cz, pv.z, d.L);
        } else {
            p.x = x[3 * k]; p.y = x[3 * k + 1]; p.z = x[3 * k + 2];
        }
        typename F::PosStore pos_out = d.st.pos[sp];
        F::store(pos_out, o, p, mass, aux);
        // the displacement from the two encodings: in the voxel form the voxel difference
        // times the power-of-two edge (exact) plus the offsets' difference, each component
        // within two roundings of its own size; then an upper bound in FP32 with every
        // operation rounded up (the bound is kept in FP32 in the voxel form anyway)
        V3<double> dm;
        if constexpr (F::voxel) {
            const PosF32 &a = p, &b = p0;
            dm = {(double)(a.cx - b.cx) * d.Ld + ((double)a.x - (double)b.x),
                  (double)(a.cy - b.cy) * d.Ld + ((double)a.y - (double)b.y),
                  (double)(a.cz - b.cz) * d.Ld + ((double)a.z - (double)b.z)};
        } else {
            dm = {p.x - p0.x, p.y - p0.y, p.z - p0.z};
        }
        const float ax = __double2float_ru(fabs(dm.x) * (1.0 + 1e-15));
        const float ay = __double2float_ru(fabs(dm.y) * (1.0 + 1e-15));
        const float az = __double2float_ru(fabs(dm.z) * (1.0 + 1e-15));
        moved_f = __fsqrt_ru(__fadd_ru(__fadd_ru(__fmul_ru(ax, ax), __fmul_ru(ay, ay)), __fmul_ru(az, az)));
    }
    R4 q4 = d.st.quat[sp][o];
    if (q) {
        q4 = R4{(R)q[4 * k], (R)q[4 * k + 1], (R)q[4 * k + 2], (R)q[4 * k + 3]};
        d.st.quat[sp][o] = q4;
    }
    R4 kv0 = d.st.kv[sp][2 * o], kv1 = d.st.kv[sp][2 * o + 1];
    if (bounds == 1) {
        // the bounds grow by the displacement (rounded up in the voxel form's FP32)
        if constexpr (F::voxel) {
            kv0.w = __fadd_ru(kv0.w, moved_f);
            kv1.w = __fadd_ru(kv1.w, moved_f);
        } else {
            kv0.w = __dadd_ru(kv0.w, (double)moved_f);
            kv1.w = __dadd_ru(kv1.w, (double)moved_f);
        }
        const R in_use = d.status->acc_par == 0 ? kv0.w : kv1.w;
        bits = __float_as_uint(__double2float_ru((double)in_use));
    } else if (bounds == 0) {
        kv0.w = R(0);
        kv1.w = R(0);
    }
    if (v) kv0 = R4{(R)v[3 * k], (R)v[3 * k + 1], (R)v[3 * k + 2], kv0.w};
    if (w) {
        if constexpr (F::voxel) {
            // the voxel form keeps the angular velocity in FP32 and reads it back with an
            // FP32 rotation: the upload rotates in FP32 too (GB300's FP64 rate is low)
            float m[9];
            quat_mat<float>(q4.x, q4.y, q4.z, q4.w, m);
            const V3<float> wg =
                mat_vec<float>(m, V3<float>{(float)w[3 * k], (float)w[3 * k + 1], (float)w[3 * k + 2]});
            kv1 = R4{wg.x, wg.y, wg.z, kv1.w};
        } else {
            double m[9];
            quat_mat<double>((double)q4.x, (double)q4.y, (double)q4.z, (double)q4.w, m);
            V3<double> wg = mat_vec<double>(m, V3<double>{w[3 * k], w[3 * k + 1], w[3 * k + 2]});
            kv1 = R4{(R)wg.x, (R)wg.y, (R)wg.z, kv1.w};
        }
    }
    if (v || bounds == 1) d.st.kv[sp][2 * o] = kv0;
    if (w || bounds == 1) d.st.kv[sp][2 * o + 1] = kv1;
    if (act) d.st.active[sp][o] = act[k];
    return bits;
}

// One thread per uploaded owner (blocks of whole warps).  bounds 1: the largest in-use
// bound of the upload goes to status->upload_disp_bits (a non-negative float's bits
// order as the float), one atomic per warp.
template <class F>
__global__ void __launch_bounds__(256) k_owner_upload(Dev<F> d, int64_t first, int64_t n, const double *x,
                                                      const double *q, const double *v, const double *w,
                                                      const uint8_t *act, int bounds, double inv_ld)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int bits = 0;
    if (k < n) bits = owner_upload_one<F>(d, first, k, x, q, v, w, act, bounds, inv_ld);
    if (bounds == 1) {
        bits = __reduce_max_sync(0xffffffffu, bits);
        if ((threadIdx.x & 31) == 0 && bits != 0) atomicMax(&d.status->upload_disp_bits, bits);
    }
}

// Both orientation buffers get the current orientation (single spheres: a sphere at rest
// reads and writes none in a step, so both must hold it; see integrate_core).
template <class F>
__global__ void __launch_bounds__(256) k_mirror_quat(Dev<F> d, int64_t first, int64_t n)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int sp = d.status->state_par;
    d.st.quat[sp ^ 1][first + k] = d.st.quat[sp][first + k];
}

// Sphere centres (FP64 world frame), radii, and the raw voxel encoding.
template <class F, bool CLUMPS>
__global__ void k_sphere_download(Dev<F> d, const int64_t *slots, int64_t n, double *xyz, double *rad, int *cell,
                                  float *off)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int sp = d.status->state_par;
    uint32_t s = (uint32_t)slots[k];
    SphereK<F> me = load_sphere<F, CLUMPS>(d, sp, s);
    const Scene &sc = d.scenes[d.owner_scene[me.owner]];
    V3<double> pa = F::absolute(me.p, sc, d.Ld);
    if (xyz) { xyz[3 * k] = pa.x; xyz[3 * k + 1] = pa.y; xyz[3 * k + 2] = pa.z; }
    if (rad) rad[k] = (double)me.rad + (double)me.rlo;
    if constexpr (F::voxel) {
        if (cell) {
            cell[3 * k] = me.p.cx; cell[3 * k + 1] = me.p.cy; cell[3 * k + 2] = me.p.cz;
            off[3 * k] = me.p.x; off[3 * k + 1] = me.p.y; off[3 * k + 2] = me.p.z;
        }
    }
}

// FP64 diagnostics: per-block partial sums in a fixed order (per owner: kinetic,
// potential, momentum, angular momentum; per owned contact: Hertz elastic energy).
template <class F, bool CLUMPS>
__global__ void __launch_bounds__(256) k_diag(Dev<F> d, double *partials)
{
    using R = typename F::R;
    const int sp = d.status->state_par, lc = d.status->list_cur;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // ke, pe, el, P[3], L[3]
    if (t < d.M) {
        int64_t o = t;
        R mass;
        typename F::Pos p = F::load(d.st.pos[sp], o, mass);
        const Scene &sc = d.scenes[d.owner_scene[o]];
        V3<double> x = F::absolute(p, sc, d.Ld);
        auto v4 = d.st.kv[sp][2 * o];
        auto w4 = d.st.kv[sp][2 * o + 1];
        auto q4 = d.st.quat[sp][o];
        auto ii = d.inv_moi[o];
        double m = (double)mass;
        V3<double> v = {(double)v4.x, (double)v4.y, (double)v4.z};
        double Q[9];
        quat_mat<double>((double)q4.x, (double)q4.y, (double)q4.z, (double)q4.w, Q);
        V3<double> wb = mat_tvec<double>(Q, V3<double>{(double)w4.x, (double)w4.y, (double)w4.z});
        V3<double> I = {1.0 / (double)ii.x, 1.0 / (double)ii.y, 1.0 / (double)ii.z};
        acc[0] = 0.5 * m * dot(v, v) + 0.5 * ((I.x * wb.x * wb.x + I.y * wb.y * wb.y) + I.z * wb.z * wb.z);
        acc[1] = -m * ((sc.g[0] * x.x + sc.g[1] * x.y) + sc.g[2] * x.z);
        V3<double> mv = m * v;
        acc[3] = mv.x; acc[4] = mv.y; acc[5] = mv.z;
        V3<double> orb = cross(x, mv);
        V3<double> spin = mat_vec<double>(Q, V3<double>{I.x * wb.x, I.y * wb.y, I.z * wb.z});
        acc[6] = orb.x + spin.x; acc[7] = orb.y + spin.y; acc[8] = orb.z + spin.z;
    }
    if (t < d.N) {
        uint32_t o = d.sph_owner[t];
        if (o != 0xffffffffu && d.st.active[sp][o]) {
            SphereK<F> me = load_sphere<F, CLUMPS>(d, sp, (uint32_t)t);
            const Scene &sc = d.scenes[d.owner_scene[o]];
            const int n = d.lists.cnt[lc][t];
            for (int k = 0; k < n; ++k) {
                uint32_t j = d.lists.partner[lc][(int64_t)k * d.Np + t];
                ContactIn<R> c;
                V3<R> armA, armB;
                bool on;
                if (j & WALL_BIT) {
                    on = wall_contact<F>(d, me, sc, d.walls[j & ~WALL_BIT], c, armA);
                } else {
                    if (j < (uint32_t)t) continue;
                    SphereK<F> B = load_sphere<F, CLUMPS>(d, sp, j);
                    if (!d.st.active[sp][B.owner]) continue;
                    on = sphere_contact<F>(d, me, B, c, armA, armB);
                }
                if (on) {
                    double dl = (double)c.delta;
                    acc[2] += (8.0 / 15.0) * (double)c.Estar * sqrt((double)c.Rbar) * dl * dl * sqrt(dl);
                }
            }
        }
    }
    __shared__ double red[9][256];
    for (int c = 0; c < 9; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int c = 0; c < 9; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 9; ++c) partials[(int64_t)blockIdx.x * 9 + c] = red[c][0];
}

}  // namespace dem
