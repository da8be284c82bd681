/*
 * dem_oracle.h -- plain FP64 CPU oracle of the per-timestep DEM contact pipeline.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py may load this library.  It shares no code, header, table or constant
 * with the CUDA library under paper_2311_04648_gb300/csrc and includes nothing from it.
 *
 * What it computes (arXiv 2311.04648, "Chrono DEM-Engine"):
 *   - contacts by brute force over all sphere pairs i<j of different owners and all
 *     sphere-wall pairs; a contact exists iff the overlap delta > 0 (Sec. 4.1, Eq. 1);
 *   - the history-based Hertz-Mindlin force with Coulomb capping as the default model
 *     of Sec. 4.2.1 computes it (normal force, history update of Eq. 3, tangential force,
 *     capping with the damping term included and the history back-solved);
 *   - tangential history that is created at zero when a contact appears and dropped when
 *     it disappears (Sec. 4.2, contact wildcards);
 *   - rolling resistance (the F_r, tau_r equations of Sec. 4.1 as the default model of
 *     Sec. 4.2.1): after a contact has lasted longer than a collision time, a force of
 *     magnitude C_r |F_n| along the rolling part of the relative velocity of the contact
 *     point, applied as an action-reaction pair that changes only the torques;
 *   - per-owner force/torque sums (Eqs. 5a-5b);
 *   - family tags (Sec. 2.2.2): prescribed linear / angular velocities per family and
 *     contact masks between families;
 *   - a second contact model, the bonded breakable contact of Sec. 6.3 (the paper's
 *     worked custom model), see orc_world.model;
 *   - a semi-implicit Euler step of velocity, body-frame angular velocity (with the
 *     gyroscopic term, switchable), position and quaternion.  The paper does not state
 *     the integrator; this is the reading adopted for the whole project.
 * Everything is double precision, evaluated in the written order (build with
 * -ffp-contract=off so no multiply-add is fused).
 *
 * Every function returns 0 on success or a negative error code; nothing is allocated
 * for the caller except the opaque history object, freed by orc_history_free.
 */
#ifndef DEM_ORACLE_H
#define DEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_WALL_PLANE = 0, ORC_WALL_CYLINDER = 1, ORC_WALL_CONE = 2, ORC_WALL_TRIANGLE = 3 };
/* contact force models (Sec. 4.2: the default model; Sec. 6.3: a bonded, breakable
 * contact for brittle solids, the paper's worked example of a custom model) */
enum { ORC_MODEL_HERTZ_MINDLIN = 0, ORC_MODEL_BONDED_BREAKAGE = 1 };
/* parameters of ORC_MODEL_BONDED_BREAKAGE (model_params[k]) */
enum { ORC_BRK_TENSION = 0, ORC_BRK_COHESION = 1, ORC_BRK_ETA = 2, ORC_BRK_DAMPING = 3, ORC_BRK_NPARAM = 4 };
enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_CAPACITY = -2, ORC_ERR_DIVERGED = -3, ORC_ERR_NOMEM = -4 };

/* One analytical wall.  All walls move rigidly with angular velocity `omega` about the
 * point `p`; their geometry is invariant under that motion (planes spin about their
 * normal, cylinders and cones about their axis), so only the surface velocity matters.
 *   plane   : point p, unit normal n pointing into the granular domain
 *   cylinder: axis point p, unit axis n, inner surface radius r0 (spheres live inside)
 *   cone    : axis point p, unit axis n, generator segment (r0,z0)-(r1,z1) in the
 *             (radius, axial coordinate) half plane; spheres live on the axis side
 *   triangle: one facet of a rigid mesh (Sec. 2.4, geometry hierarchy; Sec. 5, the
 *             mixer), vertices tri[9] at time 0, turning with omega about p, so at time
 *             t its vertices are p + R(omega t)(v - p); two-sided: the gap is the distance
 *             from the centre to the closest point of the facet                         */
typedef struct {
    int32_t type;
    int32_t mat;
    double p[3];
    double n[3];
    double r0, z0, r1, z1;
    double omega[3];
    double tri[9];
} orc_wall;

/* Prescribed motion of a family (Sec. 2.2.2, family tags): where fix_v (fix_w) is set,
 * every owner of the family moves with linear velocity v (angular velocity w, global
 * frame) instead of the one its forces would give; fix_v = fix_w = 1 with zero
 * velocities holds the family fixed. */
typedef struct {
    int32_t fix_v, fix_w;
    double v[3], w[3];
} orc_family_motion;

typedef struct {
    int64_t n_owner, n_sphere;
    int32_t n_mat, n_wall;
    /* materials: E, nu per material; restitution and friction per ordered pair, row-major */
    const double *E, *nu, *cor, *mu;
    const orc_wall *walls;
    /* owner state, mutated by orc_step: x[3M], v[3M], wb[3M] (body frame), q[4M] (w,x,y,z) */
    double *x, *v, *wb, *q;
    const double *mass, *moi;       /* mass[M], principal moments moi[3M] (body frame)   */
    int32_t *active;                /* active[M]: 1 = simulated, 0 = removed by the sink  */
    /* spheres: owner[N], body-frame offset from the owner's centre of mass rloc[3N],
     * radius rad[N], material mat[N] */
    const int64_t *owner;
    const double *rloc, *rad;
    const int32_t *mat;
    /* parameters */
    double h;
    double g[3];
    int32_t gyroscopic;
    int32_t has_sink;
    double sink_p[3], sink_n[3];    /* owners with (x - sink_p).sink_n < 0 are removed    */
    double v_err;                   /* |v| above this (or NaN) is divergence; <= 0: off  */
    void *hist;                     /* opaque history object (orc_history_new)            */
    int32_t cell_list;              /* 1: enumerate candidates from a uniform grid instead
                                       of all j > i; the same contacts in the same order,
                                       so results are bit-identical (a faster variant)   */
    int32_t n_threads;              /* > 1: find contacts and integrate owners on that
                                       many OpenMP threads; the reduction onto owners stays
                                       serial in (i, partner) order, so results are
                                       bit-identical to one thread                        */
    const double *crr;              /* rolling resistance coefficient per ordered material
                                       pair, row-major; NULL: zero for every pair         */
    /* family tags (Sec. 2.2.2): family[M] (NULL: every owner in family 0); contact_mask
     * [256 * 256], 0 where contacts between two families are not resolved (NULL: all
     * resolved; walls belong to no family and meet every sphere); motion[256] (NULL: no
     * prescribed motion) */
    const uint8_t *family;
    const uint8_t *contact_mask;
    const orc_family_motion *motion;
    /* contact force model (ORC_MODEL_*) and its parameters (NULL for the default) */
    int32_t model;
    const double *model_params;
    int64_t step;                   /* steps taken (time = step * h: the pose of meshes)  */
} orc_world;

/* One resolved contact.  j >= 0 is a sphere, j < 0 is wall (-1 - j).  force acts on
 * sphere i (the equal and opposite force acts on j); n points from j to i. */
typedef struct {
    int64_t i, j;
    double force[3];
    double point[3];
    double normal[3];
    double overlap;
    double ut[3];                   /* tangential history after this step's update       */
    double age;                     /* time in contact after this step's update (the
                                       delta_time wildcard of Sec. 4.2.1)                 */
    double torque_force[3];         /* rolling resistance: a force on i (-it on j) that
                                       acts through the contact torque only (Sec. 4.1) */
    double wc[4];                   /* the model's further contact wildcards after this
                                       step (bonded breakage: bond state, bond length)    */
} orc_contact;

void *orc_history_new(void);
void  orc_history_free(void *h);
int64_t orc_history_size(const void *h);
/* Replace the history by n entries (i, j, ut[3n], age[n]); j < 0 denotes wall -1-j;
 * age NULL: zero.  Entries need not be sorted.  get: age may be NULL. */
int orc_history_set(void *h, int64_t n, const int64_t *i, const int64_t *j, const double *ut, const double *age);
int orc_history_get(const void *h, int64_t cap, int64_t *n, int64_t *i, int64_t *j, double *ut, double *age);
/* The further wildcards wc[4n] of the entries (i, j) (model wildcards; entries that are
 * not in the history are added with zero ut and age).  get: wc[4 * count]. */
int orc_history_set_wildcards(void *h, int64_t n, const int64_t *i, const int64_t *j, const double *wc);
int orc_history_get_wildcards(const void *h, int64_t cap, int64_t *n, double *wc);

/* Sphere centres in the global frame: p_s = x_o + R(q_o) rloc_s. */
int orc_sphere_positions(const orc_world *w, double *p);

/* The listed (margin-enlarged) sphere-sphere set: i<j, different active owners, and
 * ((dx*dx + dy*dy) + dz*dz) < t*t with t = (R_i + R_j) + 2*beta, all in FP64 and in
 * that order.  Output sorted lexicographically. */
int orc_listed_pairs_f64(int64_t n, const double *p, const double *rad, const int64_t *owner,
                         const uint8_t *sphere_active, double beta, int64_t cap,
                         int64_t *count, int64_t *pi, int64_t *pj);

/* The same set for the voxel + FP32 offset position encoding: p = cell*L + off with an
 * integer cell per axis and an FP32 offset; the difference is formed as
 * (float)(ci - cj) * L + (oi - oj) with every operation in IEEE single precision, the
 * squared distance as ((dx*dx + dy*dy) + dz*dz) and the threshold t = (Ri + Rj) + 2*beta
 * in single precision, compared as s < t*t. */
int orc_listed_pairs_voxel_f32(int64_t n, const int32_t *cell, const float *off, float L,
                               const float *rad, const int64_t *owner,
                               const uint8_t *sphere_active, float beta, int64_t cap,
                               int64_t *count, int64_t *pi, int64_t *pj);

/* The listed sphere-wall set: signed gap from the sphere centre to the wall surface
 * (positive on the domain side) below R + beta.  Output sorted by (sphere, wall). */
int orc_listed_wall_pairs(const orc_world *w, const double *p, double beta, int64_t cap,
                          int64_t *count, int64_t *si, int64_t *wi);

/* Contact forces at the current state without advancing it.  F[3M], T[3M] receive the
 * per-owner sums (gravity included in F, torques global); the contact list (nullable)
 * receives every contact with delta > 0.  The history in w->hist is NOT modified; the
 * updated history of each contact is reported in contacts[k].ut. */
int orc_eval(const orc_world *w, double *F, double *T, int64_t cap, int64_t *count,
             orc_contact *contacts);

/* Advance nsteps: contacts, forces, history, reduction, integration, sink.  Returns
 * ORC_ERR_DIVERGED (state left after the offending step) if a speed exceeds v_err. */
int orc_step(orc_world *w, int64_t nsteps);

/* Diagnostics in FP64: kinetic (translational + rotational), gravitational potential
 * -sum m g.x, Hertz elastic energy sum (8/15) E* sqrt(Rbar) delta^(5/2) over contacts,
 * linear momentum, angular momentum about the origin (orbital + spin).  Every sum is
 * compensated (Neumaier's variant of Kahan summation), so it is accurate to a few ulps
 * of the sum of the magnitudes of its terms whatever their number. */
int orc_diagnostics(const orc_world *w, double *ke, double *pe, double *elastic,
                    double *mom, double *angmom);

/* Threads OpenMP would use (1 when built without OpenMP). */
int orc_max_threads(void);

/* Material combination used for E* and G* (readings of the unstated formula). */
void orc_effective_moduli(double E_a, double nu_a, double E_b, double nu_b,
                          double *E_star, double *G_star);

#ifdef __cplusplus
}
#endif
#endif
