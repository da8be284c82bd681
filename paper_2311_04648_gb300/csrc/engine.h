// engine.h -- host-side flattened world and the engine interface between the C ABI
// (api.cu) and the per-form engines (engine_f64.cu, engine_f32.cu).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dem.h"
#include "common.cuh"

namespace dem {

// A world (all scenes of a batch) flattened to the arrays the engines upload.
struct HostModel {
    int precision = DEM_PRECISION_FP64_PLAIN;
    int schedule = DEM_SCHEDULE_EVERY_STEP;
    int gyroscopic = 1;
    int device = 0;
    double L = 0.0;                 // cell edge
    double Lv = 0.0;                // voxel edge (voxel form: a power of two, L = vpc * Lv)
    int vpc = 1;                    // voxels per cell edge
    double L_min = 0.0;             // smallest usable cell edge (cell factor 1)
    int vpc_min = 1;                // voxels per edge of that cell
    double cell_factor = 1.0;       // L over L_min
    std::vector<double> scene_ext;  // box extent per scene and axis (3 per scene)
    double margin = 0.0;            // margin of the lists (EVERY_STEP) / upper bound (delayed)
    double margin_max = 0.0;
    double r_max = 0.0;
    std::vector<Scene> scenes;
    std::vector<Wall> walls;
    std::vector<PairParam> pairs;
    std::vector<double> pair_crr;   // rolling resistance per material pair (pairs' indexing)
    bool rolling = false;           // some pair has C_r > 0
    // family tags: per-owner family (empty: all 0), prescribed motion per family, contact
    // mask; families_used once any of them departs from the default
    std::vector<uint8_t> owner_family;
    std::vector<FamilyMotion> fam_motion;       // N_FAMILY entries
    std::vector<uint32_t> fam_mask;             // FAMILY_MASK_WORDS words
    bool families_used = false;
    // contact model (force_models.cuh: FORCE_MODEL_*), its parameters, and the mean
    // Poisson ratio per material pair (pairs' indexing) that models may read
    int model = 0;
    std::vector<double> model_params;
    std::vector<double> pair_nu;
    std::vector<uint16_t> mat_scene, mat_local;
    // owners, M
    std::vector<double> x, q, v, wb, mass, moi, r_ext;
    std::vector<uint16_t> owner_scene;
    std::vector<uint8_t> owner_iso;
    std::vector<int64_t> owner_first_slot;
    std::vector<int32_t> owner_nsph;
    // sphere slots, N (padding slots included)
    std::vector<uint32_t> sph_owner;
    std::vector<double> sph_rloc, sph_rad;
    std::vector<uint16_t> sph_mat;
    std::vector<uint8_t> sph_head, sph_segend;
    std::vector<int64_t> slot_of_sphere, sphere_of_slot;
    bool clumps = false;
    uint32_t n_cells_total = 0;
    int n_bins = 0;                 // schedule bins of all scenes
    // per scene: first owner id and first user sphere id in the flattened order
    std::vector<int64_t> scene_owner_base, scene_sphere_base, scene_wall_base;
    void *stream = nullptr, *detect_stream = nullptr;
    void *(*alloc)(size_t, void *) = nullptr;
    void (*free)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    // learned schedule weights (may be empty)
    std::vector<uint8_t> schedule_model;
};

struct ContactOut {
    int64_t i, j;                   // user sphere ids; j = -1 - wall for walls
    double force[3], point[3], overlap, hist[3];
    double age, trf[3];             // time in contact; rolling-resistance force on i (torque only)
    double wc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // contact model wildcards (model worlds)
};

// Detection cells of edge f * L_min (whole voxels in the voxel form) for every scene:
// cells per axis, global cell bases and the total.  Schedule bins keep the f = 1 grid.
dem_status layout_cells(HostModel &m, double factor, std::string &err);

class EngineBase {
public:
    virtual ~EngineBase() {}
    virtual dem_status init(HostModel &m, std::string &err) = 0;
    virtual dem_status step(int64_t n, std::string &err) = 0;
    virtual dem_status sync(std::string &err) = 0;
    virtual void *stream() = 0;
    virtual dem_status owner_state(int64_t first, int64_t n, double *x, double *q, double *v, double *w,
                                   std::string &err) = 0;
    virtual dem_status set_owner_state(int64_t first, int64_t n, const double *x, const double *q, const double *v,
                                       const double *w, std::string &err) = 0;
    virtual dem_status sphere_positions(int64_t first, int64_t n, double *xyz, double *r, int32_t *cell, float *off,
                                        std::string &err) = 0;
    virtual dem_status contacts(std::vector<ContactOut> &out, std::string &err) = 0;
    virtual dem_status listed(std::vector<int64_t> &i, std::vector<int64_t> &j, std::vector<int64_t> &si,
                              std::vector<int64_t> &wi, std::string &err) = 0;
    virtual dem_status owner_forces(std::vector<double> &F, std::vector<double> &T, std::string &err) = 0;
    virtual dem_status set_history(int64_t k, const int64_t *i, const int64_t *j, const double *ut,
                                   const double *age, std::string &err) = 0;
    virtual dem_status set_wildcards(int64_t k, const int64_t *i, const int64_t *j, const double *wc,
                                     std::string &err) = 0;
    virtual dem_status stats(dem_stats *s, std::string &err) = 0;
    virtual dem_status diagnostics(dem_diagnostics *d, std::string &err) = 0;
    virtual dem_status save(std::vector<uint8_t> &blob, std::string &err) = 0;
    virtual dem_status load(const uint8_t *blob, size_t n, std::string &err) = 0;
    virtual dem_status set_margin(double beta, std::string &err) = 0;
    virtual void set_profiling(bool on) = 0;
    // launch shapes and detection placement; autotune times candidates on a checkpoint
    virtual dem_status set_tuning(const dem_tuning *t, std::string &err) = 0;
    virtual dem_status get_tuning(dem_tuning *t, std::string &err) = 0;
    virtual dem_status autotune(int steps, const char *cache_path, dem_tuning *chosen, std::string &err) = 0;
    virtual void set_graphs(bool on) = 0;
    virtual dem_status schedule_collect(int on, std::string &err) = 0;
    virtual dem_status schedule_train(int epochs, float lr, uint64_t seed, float *loss, std::string &err) = 0;
    virtual dem_status schedule_export(std::vector<uint8_t> &w, std::string &err) = 0;
    virtual dem_status schedule_load(const uint8_t *w, size_t n, std::string &err) = 0;
    // family tags after initialisation (owner ids global)
    virtual dem_status set_family(int64_t first, int64_t n, const uint8_t *fam, std::string &err) = 0;
    virtual dem_status set_family_motion(int f, const double *v, const double *w, std::string &err) = 0;
    virtual dem_status set_family_contacts(int fa, int fb, int on, std::string &err) = 0;
    virtual dem_status set_active_box(int64_t first, int64_t n, const double lo[3], const double hi[3], int fin,
                                      int fout, std::string &err) = 0;
};

// Host-side family tables in their default state: no prescribed motion, all contacts.
void family_defaults(std::vector<FamilyMotion> &motion, std::vector<uint32_t> &mask);
void family_set_motion(FamilyMotion &m, const double *v, const double *w);
void family_set_contacts(std::vector<uint32_t> &mask, int fa, int fb, int on);

EngineBase *make_engine_f64();
EngineBase *make_engine_f32();

}  // namespace dem
