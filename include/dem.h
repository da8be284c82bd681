/*
 * dem.h -- C ABI of the GB300-native DEM contact pipeline (libdem_gb300.so).
 *
 * The library advances granular systems of spheres and rigid sphere clumps with the
 * method of arXiv 2311.04648 (Chrono DEM-Engine): per time step, contact detection on
 * margin-enlarged spheres (Sec. 2.1), a contact list carrying tangential history
 * (Sec. 4.2, contact wildcards), the history-based Hertz-Mindlin force with Coulomb
 * capping (Sec. 4.1 Eqs. 1-4 as computed by the default model of Sec. 4.2.1), per-clump
 * force and torque sums (Sec. 4.1 Eqs. 5a-5b) and rigid-body integration.  All compute
 * runs in hand-written CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Conventions (every entry point):
 *   - Returns dem_status; DEM_OK == 0.  dem_last_error(w) describes the last failure of
 *     calls made on w (a static, thread-local string for calls that have no world).
 *   - Handles are opaque.  The library owns all device memory it allocates (cudaMalloc
 *     unless dem_world_desc.alloc is given).  The caller owns every host buffer it passes;
 *     inputs are copied in before the call returns, outputs are written before it returns.
 *   - Units are SI.  Quaternions are (w, x, y, z), unit norm, body-to-world.  Angular
 *     velocities passed in and out are in the owner's body (principal) frame, as the
 *     paper's user-referable variables define them (Sec. 4.2, table of referables).
 *   - Arrays of vectors are row-major: xyz[3*k + a].
 *   - Owner ("clump") ids and sphere ids are dense and assigned in insertion order.
 *   - One world must not be used from two host threads at the same time.
 *   - No C++ exception crosses this interface.
 */
#ifndef DEM_GB300_H
#define DEM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DEM_OK = 0,
    DEM_ERR_ARG = 1,        /* invalid argument (null pointer, bad id, non-finite value) */
    DEM_ERR_STATE = 2,      /* call not allowed in the current state (e.g. after init) */
    DEM_ERR_CUDA = 3,       /* a CUDA runtime call failed; see dem_last_error */
    DEM_ERR_CAPACITY = 4,   /* caller buffer too small; *count holds the size needed */
    DEM_ERR_DIVERGED = 5,   /* a speed exceeded the error-out velocity or became NaN */
    DEM_ERR_TIMEOUT = 6,    /* a bounded wait on the device or host ran out */
    DEM_ERR_OVERFLOW = 7,   /* contact list capacity exceeded and could not be grown */
    DEM_ERR_NOMEM = 8,      /* device or host allocation failed */
    DEM_ERR_UNSUPPORTED = 9 /* feature not available in this build / configuration */
} dem_status;

/* Position encoding and arithmetic of the whole pipeline (Sec. 2.3 discusses the
 * paper's own compressed encoding).
 *   DEM_PRECISION_FP64_PLAIN : FP64 positions, velocities, forces and history.
 *   DEM_PRECISION_VOXEL_FP32 : position = integer voxel index + FP32 offset inside the
 *     voxel; velocities, forces, reductions and history in FP32 with a fixed reduction
 *     order.  FP64 is used on the GPU only for wall distances and global diagnostics. */
typedef enum { DEM_PRECISION_FP64_PLAIN = 0, DEM_PRECISION_VOXEL_FP32 = 1 } dem_precision;

/* When the contact list is rebuilt (Sec. 2.1: delayed active-contact-set update).
 *   EVERY_STEP     : detect before every step (margin 0 unless dem_set_margin).
 *   VELOCITY_BOUND : detection on a second CUDA stream from a position snapshot, the
 *                    margin-enlarged list reused for a number of steps chosen from the
 *                    maximum speed; every step is audited against the margin.
 *   LEARNED        : as VELOCITY_BOUND but the reuse length comes from a small MLP fed
 *                    with per-bin motion statistics (dem_load_schedule_model); audited. */
typedef enum { DEM_SCHEDULE_EVERY_STEP = 0, DEM_SCHEDULE_VELOCITY_BOUND = 1, DEM_SCHEDULE_LEARNED = 2 } dem_schedule;

typedef enum { DEM_PROP_COR = 0, DEM_PROP_MU = 1, DEM_PROP_CRR = 2 } dem_prop;

typedef struct dem_world dem_world;
typedef struct dem_batch dem_batch;

typedef struct {
    double box_lo[3], box_hi[3];   /* simulation domain; the cell grid covers it           */
    int32_t precision;             /* dem_precision                                        */
    int32_t schedule;              /* dem_schedule                                         */
    int32_t device;                /* CUDA device ordinal                                  */
    int32_t gyroscopic;            /* 1: include w x (I w) in the body-frame update        */
    int64_t max_spheres;           /* optional capacity hint (0: exact)                    */
    double margin_max;             /* largest contact margin ever used (sizes the cells);
                                      0 selects 5% of the largest sphere radius            */
    void *stream;                  /* cudaStream_t for force/integration; NULL: own stream */
    void *detect_stream;           /* cudaStream_t for detection; NULL: own stream         */
    /* optional device allocator (e.g. a framework's caching allocator); both or neither */
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *alloc_ctx;
} dem_world_desc;

typedef struct {
    int64_t steps;                 /* steps completed since initialize                     */
    int64_t rebuilds;              /* contact-list builds                                  */
    int64_t audit_fallbacks;       /* builds forced because the audit found the list stale */
    int64_t overflow_regrows;      /* contact-list capacity increases                     */
    int64_t listed_pairs;          /* sphere-sphere pairs in the list in use (each once)   */
    int64_t wall_pairs;            /* sphere-wall entries in the list in use               */
    int64_t active_contacts;       /* pairs with overlap > 0 at the last evaluated step    */
    int32_t list_capacity;         /* entries per sphere row of the contact list           */
    int32_t list_max_row;          /* longest row at the last build                        */
    double margin;                 /* margin of the list in use                            */
    double displacement_bound;     /* audited displacement bound since the list snapshot   */
    double max_speed;              /* max |v| over owners at the last audit                */
    double mean_steps_per_build;   /* steps / rebuilds                                     */
    double cell_size;              /* detection cell edge                                  */
    int64_t n_cells;               /* cells of all scenes                                  */
    double ms_detect, ms_force;    /* profiled GPU time: detection (sort, cells, narrow) /
                                      contact-force kernel (dem_set_profiling)             */
    double ms_hash, ms_link;       /* profiled GPU time: snapshot + keys / list link       */
    int64_t n_detect, n_force;     /* profiled launches of each                            */
    double ms_total;               /* wall GPU time of all dem_step calls                  */
    int64_t last_cycle;            /* steps per list chosen by the delayed schedules       */
    int64_t schedule_samples;      /* (features, label) rows collected for the schedule    */
    double ms_integrate;           /* profiled GPU time of the integration kernel          */
    int64_t n_integrate;           /* profiled launches of it                              */
    int64_t spheres_with_entries;  /* spheres whose row of the list in use is not empty    */
    int64_t pair_steps;            /* sum over completed steps of the listed sphere-sphere
                                      pairs in use (each pair once): per-step averages     */
    int64_t busy_steps;            /* sum over completed steps of the spheres with listed
                                      partners                                              */
    int32_t derived_constants;     /* 1: the voxel-form kernels derive 1/m and 1/I from
                                      each sphere's mass and radius (single spheres whose
                                      inertia is c m R^2 for one c) instead of reading them */
    int32_t counting_sort;         /* 1: detection orders spheres by cell with the counting
                                      sort, 0: with the radix sort                         */
    double ms_contact_eval;        /* two-pass contact step: profiled GPU time of its
                                      evaluation pass (within ms_force, which spans both
                                      passes)                                              */
    int64_t n_contact_eval;        /* profiled launches of it                              */
} dem_stats;

typedef struct {
    double kinetic;                /* sum 1/2 m v^2 + 1/2 w_b . I w_b                       */
    double potential;              /* - sum m g . x                                        */
    double elastic;                /* sum over contacts (8/15) E* sqrt(Rbar) delta^(5/2)   */
    double momentum[3];            /* sum m v                                              */
    double angular_momentum[3];    /* sum x x m v + R(q) I w_b, about the origin           */
} dem_diagnostics;

/* ---------------------------------------------------------------- world lifecycle */

/* Create an empty world (Sec. 3.1: DEMSolver + InstructBoxDomainDimension).
 * d: descriptor (copied); *out receives the handle.  Errors: ARG, CUDA, NOMEM. */
dem_status dem_world_create(const dem_world_desc *d, dem_world **out);
/* Free the world and all its device memory.  Accepts NULL. */
dem_status dem_world_destroy(dem_world *w);
/* Human-readable description of the last error on w (w may be NULL). Never NULL. */
const char *dem_last_error(const dem_world *w);

/* ---------------------------------------------------------------- set-up (before init) */

/* Register a material (Sec. 3.1: LoadMaterial with E, nu, CoR, mu, Crr).  E > 0,
 * 0 <= nu < 0.5, 0 <= CoR <= 1, mu >= 0, Crr >= 0 (the rolling resistance coefficient
 * of Sec. 4.1: after a contact has outlasted its collision time, a force of Crr |F_n|
 * along the rolling part of the contact point's relative velocity, applied as an
 * action-reaction pair that changes only the torques).  *mat_id receives the dense id.
 * A pair of materials takes the CoR, mu and Crr set for it with dem_set_material_pair; a
 * pair left unset takes its two materials' common value where they agree, and
 * dem_initialize returns DEM_ERR_STATE where they differ (the paper sets pairwise
 * properties explicitly and gives no rule for combining two materials). */
dem_status dem_add_material(dem_world *w, double E, double nu, double CoR, double mu, double Crr,
                            int32_t *mat_id);
/* Override a pairwise property for materials (a, b), symmetric (Sec. 3.1:
 * SetMaterialPropertyPair).  prop is dem_prop: CoR in [0, 1], mu >= 0, Crr >= 0. */
dem_status dem_set_material_pair(dem_world *w, int32_t prop, int32_t a, int32_t b, double value);

/* Six planes on the faces of the domain box, normals pointing inwards
 * (Sec. 3.1: InstructBoxDomainBoundingBC("all")).  Wall ids are returned in order
 * -x, +x, -y, +y, -z, +z starting at *first_id (nullable). */
dem_status dem_add_box_walls(dem_world *w, int32_t mat, int32_t *first_id);
/* Plane through p with unit normal n pointing into the granular domain. */
dem_status dem_add_plane(dem_world *w, const double p[3], const double n[3], int32_t mat, int32_t *id);
/* Inner surface of an infinite cylinder (Sec. 3.1: AddCylinder): axis through c along
 * the unit vector axis, radius r; spheres live inside.  omega: prescribed spin (rad/s)
 * about the axis (the drum); the geometry is invariant, only its surface moves. */
dem_status dem_add_cylinder(dem_world *w, const double c[3], const double axis[3], double radius,
                            int32_t mat, double omega, int32_t *id);
/* Surface of revolution of the segment (r0, z0)-(r1, z1) about the axis through p along
 * the unit vector axis (z measured along the axis from p); spheres live on the axis
 * side (the conical hopper wall). */
dem_status dem_add_cone_segment(dem_world *w, const double p[3], const double axis[3], double r0,
                                double z0, double r1, double z1, int32_t mat, int32_t *id);
/* A rigid triangle mesh (Sec. 2.4: meshes in the geometry hierarchy; Sec. 5: the bladed
 * mixer): n_facets two-sided facets, vertices[9 n] (three xyz points per facet, global
 * frame, SI units, at time 0), one material, turning with the prescribed angular
 * velocity omega[3] (world frame; zero: static) about axis_point[3], so that at time t a
 * vertex v sits at axis_point + R(omega t)(v - axis_point).  Each facet is a wall
 * (ids first_id .. first_id + n_facets - 1; contacts report j = -1 - id); a sphere's
 * gap to it is its centre's distance to the facet's closest point, and the facet's
 * surface velocity omega x (c - axis_point) enters the contact.  Facets are found by
 * binning them into the detection cells at every list build (not by the per-sphere wall
 * loop), and their motion is added to the audited displacement bound.  Add a scene's
 * meshes after its other walls (DEM_ERR_STATE otherwise).  Degenerate facets:
 * DEM_ERR_ARG. */
dem_status dem_add_mesh(dem_world *w, int64_t n_facets, const double *vertices, int32_t mat,
                        const double axis_point[3], const double omega[3], int32_t *first_id);
/* Prescribed rigid spin of wall `id` about its own point p with angular velocity
 * omega[3] (world frame); only walls whose geometry is invariant under the spin are
 * accepted (planes about their normal, cylinders and cones about their axis). */
dem_status dem_set_wall_spin(dem_world *w, int32_t id, const double omega[3]);

/* Register a clump template (Sec. 3.1: LoadClumpType): n component spheres with centres
 * rel_xyz[3n] in the principal frame about the centre of mass, radii[n] > 0, materials
 * mats[n]; total mass and principal moments moi[3].  Components may overlap. */
dem_status dem_add_clump_template(dem_world *w, int32_t n, const double *rel_xyz, const double *radii,
                                  const int32_t *mats, double mass, const double moi[3], int32_t *tid);
/* Instantiate n clumps of template tid (Sec. 3.1: AddClumps).  xyz[3n] centres of mass;
 * quat[4n], vel[3n], omega[3n] (body frame) nullable (identity / zero); scale[n]
 * nullable: per-instance geometric scale s (offsets and radii times s, mass times s^3,
 * moments times s^5).  *first_id receives the id of the first new owner (nullable). */
dem_status dem_add_clumps(dem_world *w, int32_t tid, int64_t n, const double *xyz, const double *quat,
                          const double *vel, const double *omega, const double *scale, int64_t *first_id);

/* As dem_add_clumps with a template id per instance, tids[n] (Sec. 3.1: AddClumps also
 * takes one template per position); instance order is preserved. */
dem_status dem_add_clumps_mixed(dem_world *w, int64_t n, const int32_t *tids, const double *xyz, const double *quat,
                                const double *vel, const double *omega, const double *scale, int64_t *first_id);

/* Time step h > 0 (Sec. 3.1: SetInitTimeStep). */
dem_status dem_set_timestep(dem_world *w, double h);
/* Gravitational acceleration (Sec. 3.1: SetGravitationalAcceleration). */
dem_status dem_set_gravity(dem_world *w, const double g[3]);
/* Error-out speed (Sec. 3.1: SetErrorOutVelocity); 0 disables.  Exceeding it (or NaN)
 * stops dem_step with DEM_ERR_DIVERGED, the world left at the last good step. */
dem_status dem_set_error_velocity(dem_world *w, double v);
/* Contact margin beta >= 0 added to every sphere for detection (Sec. 2.1: artificial
 * margin); must not exceed desc.margin_max.  EVERY_STEP defaults to 0, the delayed
 * schedules to margin_max.  A floor of 16 ulps of the largest centre distance in the
 * form's precision is always applied, so that the listed predicate never drops a
 * touching pair to rounding. */
dem_status dem_set_margin(dem_world *w, double beta);
/* Owners whose centre of mass x satisfies (x - p).n < 0 after a step are removed from
 * the simulation (frozen, no contacts): the hopper outlet. */
dem_status dem_set_sink(dem_world *w, const double p[3], const double n[3]);
/* Weights of the learned schedule (format written by dem_schedule_export). */
dem_status dem_load_schedule_model(dem_world *w, const void *weights, size_t bytes);

/* Upload, allocate and build the first contact list (Sec. 3.1: Initialize).  After
 * this, calls that change topology return DEM_ERR_STATE. */
dem_status dem_initialize(dem_world *w);

/* ---------------------------------------------------------------- stepping */

/* Advance nsteps (Sec. 3.1: DoDynamics).  Synchronous: returns when the GPU is done.
 * DEM_ERR_DIVERGED / DEM_ERR_TIMEOUT / DEM_ERR_OVERFLOW leave the world at the last
 * good step (stats.steps tells which). */
dem_status dem_step(dem_world *w, int64_t nsteps);
/* Wait for all work queued by w. */
dem_status dem_sync(dem_world *w);
/* Launch shapes, detection cell size and placement of the detection work, chosen by
 * dem_autotune or set directly.  Results do not depend on them (every choice gives
 * bit-identical states).  For a batch, a scene handle's tuning applies to all scenes. */
typedef struct {
    int32_t contact_block;         /* threads per block of the contact kernel: 32, 64, 128  */
    int32_t integrate_block;       /* threads per block of the integration kernel: 128..512 */
    int32_t narrow_block;          /* threads per block of the narrow phase: 64..256        */
    int32_t detect_inline;         /* delayed schedules: 0 = detection on the second stream
                                      beside the steps, 1 = on the force stream at the
                                      cycle boundary                                        */
    double step_ms;                /* dem_autotune: measured time per step of the choice   */
    double cell_factor;            /* detection cell edge over the smallest usable one
                                      (2 r_max + 2 margin_max, rounded up to whole voxels
                                      in the voxel form), 1 <= f <= 4: larger cells mean
                                      fewer cells and more candidates per sphere.  The
                                      voxel edge stays that of f = 1, so positions and
                                      contact lists are the same for every f.  0 reads
                                      as 1.                                                 */
    int32_t integrate_staged;      /* voxel form: 1 = integration streams whole tiles of
                                      owners through shared memory with bulk asynchronous
                                      copies (TMA), 0 = one thread per owner reading global
                                      memory directly; ignored by the FP64 form             */
    int32_t contact_lean;          /* 1 = the contact kernel compiled for more resident
                                      warps (fewer registers, some spilled), 0 = fewer warps
                                      with every value in registers                         */
    int32_t fused_block;           /* worlds of single spheres: 0 (the default) = contact
                                      forces and integration as two kernels (with a
                                      per-owner force array between them); 64, 128 or 256
                                      = one fused kernel of that block size (a thread sums
                                      its sphere's contact forces in registers and
                                      integrates it); always 0 for clumps                   */
    double margin;                 /* delayed schedules: the detection margin beta in m,
                                      0 < beta <= the world's margin_max (0 = keep the
                                      current one).  A smaller margin lists fewer pairs
                                      that do not touch and rebuilds more often.  Every
                                      touching pair is listed either way, so results are
                                      the same bits.  dem_get_tuning reports the margin in
                                      use.  Ignored by the every-step schedule.            */
    int32_t contact_integrates;    /* worlds of single spheres with the two-kernel step
                                      (fused_block 0), no rolling resistance and the
                                      built-in contact model: 1 = the contact kernel also
                                      integrates the owners with listed partners (no
                                      per-owner force array), the integration kernel the
                                      others; 0 = the integration kernel integrates every
                                      owner.  The same bits either way; ignored elsewhere  */
    int32_t binning;               /* how detection orders the spheres by cell: 0 = automatic
                                      (counting sort where the cells number at most 8 per
                                      sphere slot, else radix sort), 1 = radix sort of the
                                      cell keys, 2 = counting sort (per-cell counts, a scan,
                                      a scatter).  The same contact lists either way       */
    int32_t narrow_staged;         /* 1 = the narrow phase stages each block's candidate
                                      ranges of the sorted snapshot in shared memory (256
                                      threads per block, narrow_block ignored), 0 = its
                                      threads read them from L1/L2.  The same lists        */
    int32_t contact_screen;        /* worlds of single spheres with the two-kernel step, no
                                      rolling resistance, the built-in contact model and
                                      contact_integrates 0: 1 = two contact passes, a
                                      screening kernel that tests every listed entry's
                                      overlap and an evaluation kernel for the spheres
                                      with touching entries; 0 = one contact kernel.  The
                                      same bits either way; ignored elsewhere              */
} dem_tuning;

dem_status dem_set_tuning(dem_world *w, const dem_tuning *t);
dem_status dem_get_tuning(dem_world *w, dem_tuning *t);
/* Time `steps` steps (at least 2 cycles) for each candidate configuration from a
 * checkpoint of the current state, restore the state, and keep the fastest.  With
 * cache_path (nullable) the choice is read from / appended to that file, keyed by the
 * world's size, form, schedule and GPU name; a cached choice skips the trials. */
dem_status dem_autotune(dem_world *w, int32_t steps, const char *cache_path, dem_tuning *chosen);
/* Replay the per-step (every-step schedule) or per-cycle (delayed schedules) work from
 * captured CUDA graphs (on = 1, the default) or launch kernels one by one (on = 0). */
dem_status dem_set_graphs(dem_world *w, int32_t on);

/* Bracket every force launch and every detection phase with CUDA events on the stream
 * that runs it and accumulate their durations into dem_stats (on = 1); off by default. */
dem_status dem_set_profiling(dem_world *w, int32_t on);
/* The CUDA stream (cudaStream_t) on which force/integration kernels run. */
dem_status dem_get_stream(dem_world *w, void **stream);

/* ---------------------------------------------------------------- read back / set state */

/* Owner state for ids [first, first + n); any output may be NULL.  xyz[3n], quat[4n],
 * vel[3n], omega[3n] (body frame).  Tracker Pos / Vel / AngVel in the paper.  Outputs in
 * pinned (page-locked, mapped) host memory are written by the device directly across the
 * host link; any other memory through device scratch and a copy.  Returns when the
 * outputs hold the values (the world's streams are synchronised). */
dem_status dem_get_owner_state(dem_world *w, int64_t first, int64_t n, double *xyz, double *quat,
                               double *vel, double *omega);
/* Overwrite owner state (tracker SetPos etc.); NULL inputs keep the current value.
 * Inputs are FP64 in the layouts of dem_get_owner_state (omega in the body frame).  A
 * non-finite position, velocity or angular velocity rejects the whole call with
 * DEM_ERR_ARG before anything is applied.  Worlds of single spheres on a delayed schedule keep the contact
 * list in use: each owner's displacement by the call is added to its audit bounds, and
 * the next step rebuilds the list (history carried over) only if the largest bound then
 * exceeds the margin.  Clump worlds and the every-step schedule rebuild the list before
 * the next step after any change of positions or orientations.  Inputs are read before
 * the call returns. */
dem_status dem_set_owner_state(dem_world *w, int64_t first, int64_t n, const double *xyz,
                               const double *quat, const double *vel, const double *omega);
/* Sphere centres (world frame) and radii for sphere ids [first, first + n). */
dem_status dem_get_sphere_positions(dem_world *w, int64_t first, int64_t n, double *xyz, double *radius);
/* The voxel encoding of sphere centres (DEM_PRECISION_VOXEL_FP32 only): integer voxel
 * index cell[3n] and FP32 offset offset[3n] in [0, edge) per axis, centre = (scene
 * box_lo + cell * edge) + offset; *edge (nullable) receives the voxel edge, a power of
 * two at most 1/16 of the detection cell.  DEM_ERR_STATE in the FP64 form. */
dem_status dem_get_sphere_voxels(dem_world *w, int64_t first, int64_t n, int32_t *cell, float *offset, double *edge);
/* Every contact with overlap > 0 at the current state, ordered by (i, partner) with
 * spheres before walls.  i < j for sphere pairs; j = -1 - wall_id for walls.  force[3]
 * acts on sphere i (global frame); point[3] is the contact point; overlap > 0; history
 * is the tangential displacement that the next step starts from.  Outputs nullable.
 * DEM_ERR_CAPACITY if cap < count (count is always written). */
dem_status dem_get_contacts(dem_world *w, int64_t cap, int64_t *count, int64_t *i, int64_t *j,
                            double *force, double *point, double *overlap, double *history);
/* The listed (margin-enlarged) sphere-sphere pairs of the list in use, i < j, sorted. */
dem_status dem_get_listed_pairs(dem_world *w, int64_t cap, int64_t *count, int64_t *i, int64_t *j);
/* The listed sphere-wall entries (sphere id, wall id), sorted. */
dem_status dem_get_listed_wall_pairs(dem_world *w, int64_t cap, int64_t *count, int64_t *sphere,
                                     int64_t *wall);
/* Per-owner force (contacts plus gravity) and contact torque about the centre of mass
 * (global frame) evaluated at the current state without advancing it, ids
 * [first, first + n).  The history is not modified. */
dem_status dem_get_owner_forces(dem_world *w, int64_t first, int64_t n, double *force, double *torque);
/* Set the tangential history of the listed contacts (i, j, ut[3k]); unlisted entries
 * are ignored and all other history is zeroed.  For exact replays in tests. */
dem_status dem_set_history(dem_world *w, int64_t k, const int64_t *i, const int64_t *j, const double *ut);
/* The same with each contact's age age[k] (time in contact, seconds; NULL: zero), the
 * history the rolling-resistance gate of Sec. 4.2.1 reads. */
dem_status dem_set_history_age(dem_world *w, int64_t k, const int64_t *i, const int64_t *j, const double *ut,
                               const double *age);
/* ---------------------------------------------------------------- contact force models */

/* Contact force models (Sec. 4.2: a custom model replaces the default one; Sec. 6.3 its
 * worked example).  Each model is a device functor compiled into its own build of the
 * contact kernel (no just-in-time compilation): it reads the per-contact referable
 * variables (normal, overlap, contact arms, velocities, masses, radii, material pair
 * constants, families, time step), keeps up to 8 contact wildcards (zero when a contact
 * appears, dropped when it vanishes) and gives the force on A and a torque-only force.
 * Every sphere pair is evaluated with A the lower sphere id, so a model need not be
 * symmetric in A and B.  Walls always take the default model.
 *   DEM_MODEL_DEFAULT          the built-in default model (the fastest path)
 *   DEM_MODEL_HERTZ_MINDLIN    the same default model through the functor interface
 *                              (no parameters; gives the built-in results)
 *   DEM_MODEL_BONDED_BREAKAGE  the bonded, breakable contact of Sec. 6.3, 4 parameters:
 *                              tensile strength sigma_t (Pa, negative), cohesion c (Pa),
 *                              bending coefficient eta, normal damping factor (0.01 in
 *                              the paper); wildcards 4 and 5 are the bond state (> 0
 *                              bonded, -1 broken) and the bond's unloaded overlap.  A bond
 *                              acts across a gap while its pair stays listed: give the
 *                              margin room for the separation at which it fails. */
typedef enum { DEM_MODEL_DEFAULT = 0, DEM_MODEL_HERTZ_MINDLIN = 1, DEM_MODEL_BONDED_BREAKAGE = 2 } dem_model;
/* Before dem_initialize.  params[n_params] as listed above. */
dem_status dem_set_force_model(dem_world *w, int32_t model, const double *params, int32_t n_params);
/* Contact wildcards 4..7 of the listed sphere pairs (i, j), wc[4k], in the orientation
 * of the lower sphere id (e.g. bonding pairs at the start of a run).  Pairs not in the
 * list in use are ignored.  DEM_ERR_STATE where the model has no such wildcards. */
dem_status dem_set_contact_wildcards(dem_world *w, int64_t k, const int64_t *i, const int64_t *j, const double *wc);
/* The model's 8 wildcards of each contact after this step's update, wc[8 count], in the
 * order and count of dem_get_contacts (which, in a model world, reports every pair the
 * model engages: a bond across a gap has a negative overlap). */
dem_status dem_get_contact_wildcards(dem_world *w, int64_t cap, int64_t *count, double *wc);

/* ---------------------------------------------------------------- family tags */

/* Family tags (Sec. 2.2.2): every owner carries a family in [0, 255] (0 by default).
 * Owners [first, first + n) of this scene (insertion order) take family[n].  Before
 * dem_initialize for owners added so far; after it, the contact list is rebuilt before
 * the next step.  The first use of any family call turns on family lookups in the step
 * kernels (a few bytes per owner and per detection candidate). */
dem_status dem_set_family(dem_world *w, int64_t first, int64_t n, const uint8_t *family);
/* Prescribed motion of a family (Sec. 2.2.2, SetFamilyPrescribedLinVel / AngVel): where
 * v (omega) is non-NULL, every owner of the family moves with that linear (angular,
 * global-frame) velocity instead of the one its forces give; it still exerts contact
 * forces on others.  v = omega = {0, 0, 0} holds the family fixed; both NULL frees it.
 * Valid before and after dem_initialize; applies to every scene of a batch. */
dem_status dem_set_family_motion(dem_world *w, int32_t family, const double *v, const double *omega);
/* Resolve (on = 1, the default) or ignore (on = 0) contacts between owners of families
 * fa and fb (fa == fb: within one family).  Walls meet every family. */
dem_status dem_set_family_contacts(dem_world *w, int32_t fa, int32_t fb, int32_t on);
/* Active box (Sec. 6.4): every owner of this scene whose centre lies inside the
 * axis-aligned box [lo, hi] takes family_inside, every other family_outside (typically
 * a family held fixed with its contacts to itself off: dormant, it costs next to
 * nothing).  After dem_initialize; call it again as the region of interest moves. */
dem_status dem_set_active_box(dem_world *w, const double lo[3], const double hi[3], int32_t family_inside,
                              int32_t family_outside);

/* Per contact, in the order and count of dem_get_contacts: age[count] (time in contact
 * after this step's update; kept only in worlds where some material pair has Crr > 0,
 * else 0) and torque_force[3 count] (the rolling-resistance force on sphere i, global
 * frame; -it acts on j; it changes only the torques, Sec. 4.1 F_r / tau_r).  Outputs
 * nullable; DEM_ERR_CAPACITY if cap < count (count is always written). */
dem_status dem_get_contact_rolling(dem_world *w, int64_t cap, int64_t *count, double *age, double *torque_force);
dem_status dem_get_stats(dem_world *w, dem_stats *s);
/* FP64 diagnostics computed on the GPU with a fixed-order reduction. */
dem_status dem_get_diagnostics(dem_world *w, dem_diagnostics *d);

/* ---------------------------------------------------------------- checkpoint */

/* Serialise owner state, contact list with history and schedule state into buf.
 * *used receives the size; DEM_ERR_CAPACITY (with *used set) if cap is too small. */
dem_status dem_save_state(dem_world *w, void *buf, size_t cap, size_t *used);
/* Restore a blob written by dem_save_state of a world with identical set-up.  Tuning
 * choices, the detection margin among them, stay as they are; a contact list saved
 * under another margin is rebuilt before the next step. */
dem_status dem_load_state(dem_world *w, const void *buf, size_t bytes);

/* ---------------------------------------------------------------- batched scenes */

/* A batch of independent scenes stepped together by the same kernels (one launch per
 * stage over all scenes).  descs[k] describes scene k; precision and schedule of
 * descs[0] apply to all.  Scenes are set up through dem_batch_world handles, which
 * accept every set-up call above; then dem_batch_initialize.  Scene handles stay valid
 * until dem_batch_destroy and give per-scene read-back; owner ids are per scene. */
dem_status dem_batch_create(int32_t nscenes, const dem_world_desc *descs, dem_batch **out);
dem_status dem_batch_world(dem_batch *b, int32_t k, dem_world **scene);
dem_status dem_batch_initialize(dem_batch *b);
/* Advance every scene by nsteps; the per-step work is replayed from a CUDA graph. */
dem_status dem_batch_step(dem_batch *b, int64_t nsteps);
dem_status dem_batch_destroy(dem_batch *b);

/* ---------------------------------------------------------------- learned schedule */

/* Record per-bin features and labels during dem_step (on = 1) or stop (on = 0).  Bins
 * are 8 x 8 x 8 detection cells; every 256 steps each occupied bin yields one sample:
 * 16 motion features at the window start (speeds, accelerations, spins in units of the
 * margin per step, list density, gravity) and, as labels, log2 of the steps until the
 * largest per-owner displacement bound in the bin passed the margin and half of it,
 * stored relative to the kinematic estimate (margin over the largest displacement per
 * step in the bin) so that the network learns the correction to it. */
dem_status dem_schedule_collect(dem_world *w, int32_t on);
/* Train the schedule MLP (16 -> 64 -> 64 -> 2, BF16 tensor-core products, FP32 Adam)
 * on the recorded samples with the GPU kernels; *final_loss (nullable) receives the mean
 * loss of the last epoch. */
dem_status dem_schedule_train(dem_world *w, int32_t epochs, float lr, uint64_t seed, float *final_loss);
/* Export the current weights (format accepted by dem_load_schedule_model). */
dem_status dem_schedule_export(dem_world *w, void *buf, size_t cap, size_t *used);

/* ---------------------------------------------------------------- kernels as utilities */

/* The schedule network's forward pass and loss gradient on the GPU for given parameters
 * (flat FP32, 5378 values: W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]),
 * host buffers X[rows][16], Y[rows][2], out[rows][2], grad[5378].  The loss is the mean
 * over rows and outputs of w (y_hat - y)^2 with w = 4 where y_hat > y, else 1. */
dem_status dem_util_mlp_forward(const float *params, int32_t rows, const float *X, float *out);
dem_status dem_util_mlp_loss_grad(const float *params, int32_t rows, const float *X, const float *Y, float *loss,
                                  float *grad);

/* Stable LSD radix sort of (key, value) pairs of 32-bit unsigned integers on the GPU,
 * sorting on the low `bits` bits of the keys (1..32).  Host buffers; n >= 0. */
dem_status dem_util_radix_sort_u32(int64_t n, const uint32_t *keys, const uint32_t *vals, int32_t bits,
                                   uint32_t *keys_out, uint32_t *vals_out);

/* ---------------------------------------------------------------- no-allocation variant */

/* The paper has no counterpart of this entry point: it serves callers that cannot call
 * cudaMalloc (code running while a CUDA graph is captured, frameworks that own device
 * memory through their own pools, loops where an allocation could synchronise the
 * device).  Same stable LSD radix sort as dem_util_radix_sort_u32, but on DEVICE
 * buffers owned by the caller: keys[n], vals[n] in, keys_out[n], vals_out[n] out (an
 * output that shares any byte with an input or with the other output is rejected with
 * DEM_ERR_ARG), queued on `stream` (a cudaStream_t;
 * NULL = legacy default stream) and returning once queued.  It allocates nothing: its
 * temporary storage is one array of device memory inside the library, sized for
 * DEM_NOALLOC_SORT_MAX keys (about 8.7 MB), which every GPU that loads the library keeps
 * until the process exits.  n above the maximum returns DEM_ERR_CAPACITY before any work.
 * The first call on each device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture.  The
 * address is kept for the life of the process, so a device reset (cudaDeviceReset, or
 * anything else that destroys the primary context) while the library is loaded is not
 * supported: later calls would use the stale address.  Every
 * call shares the array, so calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller; nothing in it needs clearing
 * between calls.  Errors are described by dem_util_noalloc_error(), which describes the
 * calling thread's last call ("" after a call that succeeded). */
#define DEM_NOALLOC_SORT_MAX (1 << 20)
dem_status dem_util_radix_sort_u32_noalloc(int64_t n, const uint32_t *keys, const uint32_t *vals, int32_t bits,
                                           uint32_t *keys_out, uint32_t *vals_out, void *stream);
const char *dem_util_noalloc_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DEM_GB300_H */
