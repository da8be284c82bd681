// api.cu -- the C ABI (include/dem.h): set-up validation, flattening of the scenes into
// the host model, dispatch to the engine of the chosen position form, batches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "engine.h"
#include "force_models.cuh"
#include "kernels.cuh"
#include "mlp.h"

using namespace dem;

namespace {

thread_local std::string g_err;

struct WallSetup {
    int type, mat;
    double p[3], n[3], r0, z0, r1, z1, omega[3];
    double tri[9];
};

struct TemplateSetup {
    std::vector<double> rel, rad;
    std::vector<int32_t> mats;
    double mass, moi[3];
};

struct SceneSetup {
    dem_world_desc desc{};
    std::vector<double> E, nu, cor, mu, crr;
    std::map<std::pair<int, int>, double> cor_pair, mu_pair, crr_pair;
    std::vector<WallSetup> walls;
    std::vector<TemplateSetup> templates;
    std::vector<int32_t> inst_tid;
    std::vector<double> inst_x, inst_q, inst_v, inst_w, inst_s;
    double h = 1e-6;
    double g[3] = {0.0, 0.0, 0.0};
    double v_err = 0.0;
    double margin = -1.0;          // unset
    bool has_sink = false;
    double sink_p[3] = {0, 0, 0}, sink_n[3] = {0, 0, 1};
    std::vector<uint8_t> inst_family;   // family tag per owner (shorter: the rest are 0)
};

struct WorldImpl {
    std::vector<SceneSetup> scenes;
    dem_world_desc desc{};         // of scene 0: precision, schedule, device, streams, allocator
    bool initialized = false;
    std::unique_ptr<EngineBase> engine;
    HostModel model;
    std::string err;
    std::vector<uint8_t> schedule_model;
    // contact force model of the world and its parameters
    int force_model = 0;
    std::vector<double> force_params;
    // family tags of the world (all its scenes): prescribed motion and contact mask
    std::vector<FamilyMotion> fam_motion;
    std::vector<uint32_t> fam_mask;
    bool families_used = false;
};

}  // namespace

struct dem_world {
    WorldImpl *impl;
    int scene;
    bool proxy;
};

struct dem_batch {
    WorldImpl *impl;
    std::vector<dem_world *> handles;
};

namespace dem {

dem_status layout_cells(HostModel &m, double factor, std::string &err)
{
    if (!(factor >= 1.0 && factor <= 4.0)) {
        err = "cell_factor must be in [1, 4]";
        return DEM_ERR_ARG;
    }
    if (m.precision == DEM_PRECISION_VOXEL_FP32) {
        m.vpc = (int)std::ceil(factor * m.vpc_min - 1e-9);
        m.L = m.vpc * m.Lv;
    } else {
        m.vpc = 1;
        m.L = factor * m.L_min;
    }
    uint64_t cell_base = 0;
    for (size_t si = 0; si < m.scenes.size(); ++si) {
        Scene &g = m.scenes[si];
        for (int a = 0; a < 3; ++a) {
            double n = std::ceil(m.scene_ext[3 * si + a] / m.L);
            if (n < 1) n = 1;
            if (n > (double)(1 << 19)) {
                err = "too many cells along an axis";
                return DEM_ERR_ARG;
            }
            g.nc[a] = (int)n;
        }
        uint64_t nc = (uint64_t)g.nc[0] * (uint64_t)g.nc[1] * (uint64_t)g.nc[2];
        if (nc >= (1ull << 31)) {
            err = "scene cell grid too large";
            return DEM_ERR_ARG;
        }
        g.cell_base = (uint32_t)cell_base;
        cell_base += nc;
        if (cell_base >= 0xffffffffull) {
            err = "total cell count exceeds 2^32 - 1";
            return DEM_ERR_ARG;
        }
    }
    m.n_cells_total = (uint32_t)cell_base;
    m.cell_factor = factor;
    return DEM_OK;
}

void family_defaults(std::vector<FamilyMotion> &motion, std::vector<uint32_t> &mask)
{
    motion.assign(N_FAMILY, FamilyMotion{});
    mask.assign(FAMILY_MASK_WORDS, 0xffffffffu);
}

void family_set_motion(FamilyMotion &m, const double *v, const double *w)
{
    m.fix_v = v ? 1 : 0;
    m.fix_w = w ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        m.v[a] = v ? v[a] : 0.0;
        m.w[a] = w ? w[a] : 0.0;
        m.vf[a] = (float)m.v[a];
        m.wf[a] = (float)m.w[a];
    }
}

void family_set_contacts(std::vector<uint32_t> &mask, int fa, int fb, int on)
{
    for (int k = 0; k < 2; ++k) {
        const int a = k ? fb : fa, b = k ? fa : fb;
        uint32_t &word = mask[(a << 3) | (b >> 5)];
        const uint32_t bit = 1u << (b & 31);
        word = on ? (word | bit) : (word & ~bit);
    }
}

}  // namespace dem

namespace {

dem_status fail(dem_world *w, dem_status s, const std::string &msg)
{
    if (w) w->impl->err = msg;
    else g_err = msg;
    return s;
}

bool finite3(const double *a) { return std::isfinite(a[0]) && std::isfinite(a[1]) && std::isfinite(a[2]); }

#define CHECK_W(w)                                                          \
    do {                                                                    \
        if (!(w)) return fail(nullptr, DEM_ERR_ARG, "null world handle");   \
    } while (0)
#define CHECK_SETUP(w)                                                                      \
    do {                                                                                    \
        CHECK_W(w);                                                                         \
        if ((w)->impl->initialized) return fail(w, DEM_ERR_STATE, "world already initialized"); \
    } while (0)
#define CHECK_INIT(w)                                                                   \
    do {                                                                                \
        CHECK_W(w);                                                                     \
        if (!(w)->impl->initialized) return fail(w, DEM_ERR_STATE, "world not initialized"); \
    } while (0)

SceneSetup &S(dem_world *w) { return w->impl->scenes[w->scene]; }

dem_status check_desc(const dem_world_desc *d)
{
    if (!d) return fail(nullptr, DEM_ERR_ARG, "null descriptor");
    if (!finite3(d->box_lo) || !finite3(d->box_hi)) return fail(nullptr, DEM_ERR_ARG, "non-finite box");
    for (int a = 0; a < 3; ++a)
        if (!(d->box_hi[a] > d->box_lo[a])) return fail(nullptr, DEM_ERR_ARG, "box_hi must exceed box_lo");
    if (d->precision != DEM_PRECISION_FP64_PLAIN && d->precision != DEM_PRECISION_VOXEL_FP32)
        return fail(nullptr, DEM_ERR_ARG, "unknown precision");
    if (d->schedule < DEM_SCHEDULE_EVERY_STEP || d->schedule > DEM_SCHEDULE_LEARNED)
        return fail(nullptr, DEM_ERR_ARG, "unknown schedule");
    if (d->margin_max < 0 || !std::isfinite(d->margin_max)) return fail(nullptr, DEM_ERR_ARG, "bad margin_max");
    if ((d->alloc == nullptr) != (d->free == nullptr))
        return fail(nullptr, DEM_ERR_ARG, "alloc and free callbacks go together");
    return DEM_OK;
}

// E*, G* (standard Hertz-Mindlin combination) and the damping ratio of Sec. 4.2.1.
PairParam pair_param(double Ea, double nua, double Eb, double nub, double cor, double mu)
{
    PairParam p;
    double ia = (1.0 - nua * nua) / Ea, ib = (1.0 - nub * nub) / Eb;
    p.Estar = 1.0 / (ia + ib);
    double ga = 2.0 * (2.0 - nua) * (1.0 + nua) / Ea, gb = 2.0 * (2.0 - nub) * (1.0 + nub) / Eb;
    p.Gstar = 1.0 / (ga + gb);
    double e = cor < 1e-12 ? 1e-12 : cor;
    double le = std::log(e);
    const double pi = 3.14159265358979323846;
    p.beta = le / std::sqrt(le * le + pi * pi);
    p.mu = mu;
    return p;
}

// Flatten every scene of the world into the host model.
dem_status build_model(WorldImpl &W, HostModel &m, std::string &err)
{
    const dem_world_desc &d0 = W.desc;
    m = HostModel();
    m.precision = d0.precision;
    m.schedule = d0.schedule;
    m.gyroscopic = d0.gyroscopic;
    m.device = d0.device;
    m.stream = d0.stream;
    m.detect_stream = d0.detect_stream;
    m.alloc = d0.alloc;
    m.free = d0.free;
    m.alloc_ctx = d0.alloc_ctx;
    m.schedule_model = W.schedule_model;
    m.model = W.force_model;
    m.model_params = W.force_params;
    if (W.families_used) {
        m.fam_motion = W.fam_motion;
        m.fam_mask = W.fam_mask;
        m.families_used = true;
    }

    // largest radius over all instances
    double rmax = 0.0;
    bool clumps = false;
    for (auto &sc : W.scenes) {
        for (size_t k = 0; k < sc.inst_tid.size(); ++k) {
            const TemplateSetup &t = sc.templates[sc.inst_tid[k]];
            double s = sc.inst_s[k];
            for (size_t c = 0; c < t.rad.size(); ++c) rmax = std::max(rmax, t.rad[c] * s);
        }
        for (auto &t : sc.templates) {
            if (t.rad.size() > 1) clumps = true;
            for (double r : t.rel) if (r != 0.0) clumps = true;
        }
    }
    if (rmax <= 0.0) rmax = 1e-3;
    m.r_max = rmax;
    double mmax = d0.margin_max > 0 ? d0.margin_max : 0.05 * rmax;
    double margin = -1.0;
    for (auto &sc : W.scenes) margin = std::max(margin, sc.margin);
    if (margin < 0) margin = (d0.schedule == DEM_SCHEDULE_EVERY_STEP) ? 0.0 : mmax;
    if (margin > mmax) {
        err = "margin exceeds margin_max";
        return DEM_ERR_ARG;
    }
    // The listed predicate is evaluated in the form's own precision while contacts are
    // decided from an (almost) exact overlap: a floor of a few ulps of the largest
    // centre distance keeps every touching pair listed even at margin 0.
    const bool vox = d0.precision == DEM_PRECISION_VOXEL_FP32;
    const double floor_margin = vox ? 16.0 * std::ldexp(1.0, std::ilogb(2.0 * (rmax + mmax)) - 23)
                                    : 16.0 * std::ldexp(1.0, std::ilogb(2.0 * (rmax + mmax)) - 52);
    if (margin < floor_margin) margin = floor_margin;
    if (mmax < margin) mmax = margin;
    m.margin = margin;
    m.margin_max = mmax;
    const double Lmin = 1.001 * 2.0 * (rmax + mmax);
    if (vox) {
        // voxels: a power of two at most 1/16 of the smallest cell, so that integer voxel
        // differences times the voxel edge are exact in FP32 and the FP32 offset inside
        // a voxel resolves ~2^-24 of it; a cell is a whole number of voxels
        m.Lv = std::ldexp(1.0, (int)std::floor(std::log2(Lmin / 16.0)));
        m.vpc_min = (int)std::ceil(Lmin / m.Lv);
        m.L_min = m.vpc_min * m.Lv;
    } else {
        m.L_min = Lmin;
        m.Lv = Lmin;
        m.vpc_min = 1;
    }
    m.clumps = clumps;
    m.scene_ext.clear();
    for (auto &sc : W.scenes)
        for (int a = 0; a < 3; ++a) m.scene_ext.push_back(sc.desc.box_hi[a] - sc.desc.box_lo[a]);

    int mat_base = 0, pair_base = 0;
    for (size_t si = 0; si < W.scenes.size(); ++si) {
        SceneSetup &sc = W.scenes[si];
        Scene g{};
        for (int a = 0; a < 3; ++a) {
            g.lo[a] = sc.desc.box_lo[a];
            double n = std::ceil(m.scene_ext[3 * si + a] / m.L_min);
            if (n < 1) n = 1;
            if (n > (double)(1 << 19)) {
                err = "too many cells along an axis";
                return DEM_ERR_ARG;
            }
            g.nbc[a] = (int)n;
            g.lof[a] = (float)g.lo[a];
            g.g[a] = sc.g[a];
            g.gf[a] = (float)sc.g[a];
        }
        g.h = sc.h;
        g.hf = (float)sc.h;
        g.v_err = sc.v_err;
        g.v_errf = (float)sc.v_err;
        if ((double)g.v_errf > sc.v_err) g.v_errf = std::nextafter(g.v_errf, -INFINITY);
        g.wall_begin = (int)m.walls.size();
        // mesh facets come after the scene's other walls: the narrow phase's wall loop
        // covers the others, the facets are found through their cell bins
        g.wall_count = 0;
        for (auto &ws : sc.walls) g.wall_count += ws.type != WALL_TRIANGLE ? 1 : 0;
        g.facet_begin = g.wall_begin + g.wall_count;
        g.facet_count = (int)sc.walls.size() - g.wall_count;
        g.has_sink = sc.has_sink ? 1 : 0;
        for (int a = 0; a < 3; ++a) { g.sink_p[a] = sc.sink_p[a]; g.sink_n[a] = sc.sink_n[a]; }
        const int nm = (int)sc.E.size();
        if (nm == 0) {
            err = "scene has no material";
            return DEM_ERR_ARG;
        }
        g.mat_base = mat_base;
        g.n_mat = nm;
        g.pair_base = pair_base;
        for (int a = 0; a < 3; ++a) g.nb[a] = (g.nbc[a] + BIN_CELLS - 1) / BIN_CELLS;
        g.bin_base = m.n_bins;
        m.n_bins += g.nb[0] * g.nb[1] * g.nb[2];
        for (int a = 0; a < nm; ++a) {
            m.mat_scene.push_back((uint16_t)si);
            m.mat_local.push_back((uint16_t)a);
        }
        // Pairwise restitution and friction (Sec. 3.1 sets them per pair and states no
        // rule for combining two materials): a pair takes the value set for it, or the
        // common value of its two materials where they agree; two materials that differ
        // and have no value set for the pair are an error.
        g.has_rolling = 0;
        for (int a = 0; a < nm; ++a)
            for (int b = 0; b < nm; ++b) {
                auto key = std::make_pair(std::min(a, b), std::max(a, b));
                if ((!sc.cor_pair.count(key) && sc.cor[a] != sc.cor[b]) ||
                    (!sc.mu_pair.count(key) && sc.mu[a] != sc.mu[b]) ||
                    (!sc.crr_pair.count(key) && sc.crr[a] != sc.crr[b])) {
                    err = "materials " + std::to_string(key.first) + " and " + std::to_string(key.second) +
                          " differ in CoR, mu or Crr: set the pair's value with dem_set_material_pair";
                    return DEM_ERR_STATE;
                }
                double cor = sc.cor_pair.count(key) ? sc.cor_pair[key] : sc.cor[a];
                double mu = sc.mu_pair.count(key) ? sc.mu_pair[key] : sc.mu[a];
                double crr = sc.crr_pair.count(key) ? sc.crr_pair[key] : sc.crr[a];
                m.pairs.push_back(pair_param(sc.E[a], sc.nu[a], sc.E[b], sc.nu[b], cor, mu));
                m.pair_crr.push_back(crr);
                m.pair_nu.push_back(0.5 * (sc.nu[a] + sc.nu[b]));
                if (crr > 0.0) {
                    g.has_rolling = 1;
                    m.rolling = true;
                }
            }
        mat_base += nm;
        pair_base += nm * nm;
        m.scene_wall_base.push_back((int64_t)m.walls.size());
        for (auto &ws : sc.walls) {
            Wall w{};
            w.type = ws.type;
            w.mat = g.mat_base + ws.mat;
            for (int a = 0; a < 3; ++a) { w.p[a] = ws.p[a]; w.n[a] = ws.n[a]; w.omega[a] = ws.omega[a]; }
            w.r0 = ws.r0; w.z0 = ws.z0; w.r1 = ws.r1; w.z1 = ws.z1;
            w.scene = (int)si;
            for (int q = 0; q < 9; ++q) { w.tri[q] = ws.tri[q]; w.cur[q] = ws.tri[q]; }
            for (int a = 0; a < 3; ++a) { w.pf[a] = (float)ws.p[a]; w.nf[a] = (float)ws.n[a]; }
            w.r0f = (float)ws.r0; w.r1f = (float)ws.r1; w.z0f = (float)ws.z0; w.z1f = (float)ws.z1;
            {
                // An FP32 evaluation of the gap (about ten rounded operations on values no
                // larger than |centre| + this scale) errs by well under 1e-6 of that sum; the
                // screen allows 2e-5 of it.  A cone's closest-point parameter divides by the
                // segment's squared length, which amplifies errors by scale / length.
                double scale = std::fabs(ws.p[0]) + std::fabs(ws.p[1]) + std::fabs(ws.p[2]) + std::fabs(ws.r0) +
                               std::fabs(ws.r1) + std::fabs(ws.z0) + std::fabs(ws.z1) + 1.0;
                double cond = 1.0;
                if (ws.type == WALL_CONE) {
                    double len = std::sqrt((ws.r1 - ws.r0) * (ws.r1 - ws.r0) + (ws.z1 - ws.z0) * (ws.z1 - ws.z0));
                    cond += scale / std::max(len, 1e-30);
                }
                w.tolf = (float)(2e-5 * scale * cond);
            }
            w.axis = -1;
            if (ws.type == WALL_PLANE && ws.omega[0] == 0.0 && ws.omega[1] == 0.0 && ws.omega[2] == 0.0) {
                for (int a = 0; a < 3; ++a) {
                    const int b = (a + 1) % 3, c = (a + 2) % 3;
                    if ((ws.n[a] == 1.0 || ws.n[a] == -1.0) && ws.n[b] == 0.0 && ws.n[c] == 0.0) {
                        const double rel = ws.p[a] - g.lo[a];
                        const double k = std::floor(rel / m.Lv);
                        if (std::fabs(k) < 1e6 * (double)(1 << 20)) {
                            w.axis = a;
                            w.ax_c = (int)k;
                            const double off = rel - k * m.Lv;
                            w.ax_off = (float)off;
                            w.ax_off_lo = (float)(off - (double)w.ax_off);
                            w.ax_sign = (float)ws.n[a];
                        }
                    }
                }
            }
            m.walls.push_back(w);
        }
        m.scenes.push_back(g);
    }
    {
        dem_status ls = layout_cells(m, 1.0, err);
        if (ls) return ls;
    }

    // owners and sphere slots
    m.scene_owner_base.clear();
    m.scene_sphere_base.clear();
    int64_t slot = 0;
    for (size_t si = 0; si < W.scenes.size(); ++si) {
        SceneSetup &sc = W.scenes[si];
        m.scene_owner_base.push_back((int64_t)m.mass.size());
        m.scene_sphere_base.push_back((int64_t)m.slot_of_sphere.size());
        const int mb = m.scenes[si].mat_base;
        for (size_t k = 0; k < sc.inst_tid.size(); ++k) {
            const TemplateSetup &t = sc.templates[sc.inst_tid[k]];
            const double s = sc.inst_s[k];
            const int64_t o = (int64_t)m.mass.size();
            const int nsph = (int)t.rad.size();
            for (int a = 0; a < 3; ++a) m.x.push_back(sc.inst_x[3 * k + a]);
            double q[4] = {sc.inst_q[4 * k], sc.inst_q[4 * k + 1], sc.inst_q[4 * k + 2], sc.inst_q[4 * k + 3]};
            double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
            if (std::fabs(qn - 1.0) < 1e-14) qn = 1.0;          // unit input is kept bit for bit
            for (int a = 0; a < 4; ++a) m.q.push_back(q[a] / qn);
            for (int a = 0; a < 3; ++a) { m.v.push_back(sc.inst_v[3 * k + a]); m.wb.push_back(sc.inst_w[3 * k + a]); }
            m.mass.push_back(t.mass * s * s * s);
            double s5 = s * s * s * s * s;
            for (int a = 0; a < 3; ++a) m.moi.push_back(t.moi[a] * s5);
            m.owner_scene.push_back((uint16_t)si);
            m.owner_iso.push_back((t.moi[0] == t.moi[1] && t.moi[1] == t.moi[2]) ? 1 : 0);
            m.owner_family.push_back(k < sc.inst_family.size() ? sc.inst_family[k] : (uint8_t)0);
            // keep an owner's slots inside one warp (segmented reduction)
            if (clumps && (slot % 32) + nsph > 32) {
                while (slot % 32 != 0) {
                    m.sph_owner.push_back(0xffffffffu);
                    for (int a = 0; a < 3; ++a) m.sph_rloc.push_back(0.0);
                    m.sph_rad.push_back(0.0);
                    m.sph_mat.push_back(0);
                    m.sph_head.push_back(0);
                    m.sph_segend.push_back((uint8_t)(slot % 32 + 1));
                    m.sphere_of_slot.push_back(-1);
                    ++slot;
                }
            }
            m.owner_first_slot.push_back(slot);
            m.owner_nsph.push_back(nsph);
            double rext = 0.0;
            const int lane0 = (int)(slot % 32);
            for (int c = 0; c < nsph; ++c) {
                m.sph_owner.push_back((uint32_t)o);
                double r2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double rl = t.rel[3 * c + a] * s;
                    m.sph_rloc.push_back(rl);
                    r2 += rl * rl;
                }
                rext = std::max(rext, std::sqrt(r2));
                m.sph_rad.push_back(t.rad[c] * s);
                m.sph_mat.push_back((uint16_t)(mb + t.mats[c]));
                m.sph_head.push_back(c == 0 ? 1 : 0);
                m.sph_segend.push_back((uint8_t)(lane0 + nsph));
                m.slot_of_sphere.push_back(slot);
                m.sphere_of_slot.push_back((int64_t)m.slot_of_sphere.size() - 1);
                ++slot;
            }
            m.r_ext.push_back(rext);
        }
    }
    if ((int64_t)m.sph_owner.size() >= (int64_t)0x7fffffff) {
        err = "too many spheres";
        return DEM_ERR_ARG;
    }
    return DEM_OK;
}

dem_status do_initialize(WorldImpl &W, dem_world *w)
{
    std::string err;
    dem_status s = build_model(W, W.model, err);
    if (s) return fail(w, s, err);
    EngineBase *e = W.desc.precision == DEM_PRECISION_VOXEL_FP32 ? make_engine_f32() : make_engine_f64();
    W.engine.reset(e);
    s = e->init(W.model, err);
    if (s) {
        W.engine.reset();
        return fail(w, s, err);
    }
    W.initialized = true;
    return DEM_OK;
}

int64_t owner_base(dem_world *w) { return w->impl->model.scene_owner_base[w->scene]; }
int64_t sphere_base(dem_world *w) { return w->impl->model.scene_sphere_base[w->scene]; }
int64_t scene_owners(dem_world *w)
{
    auto &m = w->impl->model;
    int64_t e = (size_t)w->scene + 1 < m.scene_owner_base.size() ? m.scene_owner_base[w->scene + 1] : (int64_t)m.mass.size();
    return e - owner_base(w);
}
int64_t scene_spheres(dem_world *w)
{
    auto &m = w->impl->model;
    int64_t e = (size_t)w->scene + 1 < m.scene_sphere_base.size() ? m.scene_sphere_base[w->scene + 1]
                                                                    : (int64_t)m.slot_of_sphere.size();
    return e - sphere_base(w);
}

dem_world *new_handle(WorldImpl *impl, int scene, bool proxy)
{
    dem_world *w = new dem_world;
    w->impl = impl;
    w->scene = scene;
    w->proxy = proxy;
    return w;
}

}  // namespace

extern "C" {

const char *dem_last_error(const dem_world *w)
{
    if (w) return w->impl->err.c_str();
    return g_err.c_str();
}

dem_status dem_world_create(const dem_world_desc *d, dem_world **out)
{
    if (!out) return fail(nullptr, DEM_ERR_ARG, "null output handle");
    *out = nullptr;
    dem_status s = check_desc(d);
    if (s) return s;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(nullptr, DEM_ERR_CUDA, "no CUDA device available");
    if (d->device < 0 || d->device >= ndev) return fail(nullptr, DEM_ERR_ARG, "bad device ordinal");
    WorldImpl *W = new WorldImpl;
    W->desc = *d;
    W->scenes.resize(1);
    W->scenes[0].desc = *d;
    *out = new_handle(W, 0, false);
    return DEM_OK;
}

dem_status dem_world_destroy(dem_world *w)
{
    if (!w) return DEM_OK;
    if (w->proxy) return fail(w, DEM_ERR_ARG, "scene handles are destroyed with their batch");
    delete w->impl;
    delete w;
    return DEM_OK;
}

dem_status dem_add_material(dem_world *w, double E, double nu, double CoR, double mu, double Crr, int32_t *mat_id)
{
    CHECK_SETUP(w);
    if (!(E > 0) || !(nu >= 0 && nu < 0.5) || !(CoR >= 0 && CoR <= 1) || !(mu >= 0) || !std::isfinite(E) ||
        !std::isfinite(mu) || !(Crr >= 0) || !std::isfinite(Crr))
        return fail(w, DEM_ERR_ARG, "material needs E > 0, 0 <= nu < 0.5, 0 <= CoR <= 1, mu >= 0, Crr >= 0");
    SceneSetup &sc = S(w);
    if (sc.E.size() >= 256) return fail(w, DEM_ERR_ARG, "at most 256 materials per scene");
    sc.E.push_back(E);
    sc.nu.push_back(nu);
    sc.cor.push_back(CoR);
    sc.mu.push_back(mu);
    sc.crr.push_back(Crr);
    if (mat_id) *mat_id = (int32_t)sc.E.size() - 1;
    return DEM_OK;
}

dem_status dem_set_material_pair(dem_world *w, int32_t prop, int32_t a, int32_t b, double value)
{
    CHECK_SETUP(w);
    SceneSetup &sc = S(w);
    if (a < 0 || b < 0 || a >= (int)sc.E.size() || b >= (int)sc.E.size()) return fail(w, DEM_ERR_ARG, "bad material id");
    auto key = std::make_pair(std::min(a, b), std::max(a, b));
    if (prop == DEM_PROP_COR) {
        if (!(value >= 0 && value <= 1)) return fail(w, DEM_ERR_ARG, "CoR must be in [0, 1]");
        sc.cor_pair[key] = value;
    } else if (prop == DEM_PROP_MU) {
        if (!(value >= 0) || !std::isfinite(value)) return fail(w, DEM_ERR_ARG, "mu must be >= 0");
        sc.mu_pair[key] = value;
    } else if (prop == DEM_PROP_CRR) {
        if (!(value >= 0) || !std::isfinite(value)) return fail(w, DEM_ERR_ARG, "Crr must be >= 0");
        sc.crr_pair[key] = value;
    } else {
        return fail(w, DEM_ERR_ARG, "unknown property");
    }
    return DEM_OK;
}

static dem_status add_wall(dem_world *w, const WallSetup &ws, int32_t *id)
{
    SceneSetup &sc = S(w);
    if (ws.mat < 0 || ws.mat >= (int)sc.E.size()) return fail(w, DEM_ERR_ARG, "bad material id");
    if (ws.type != WALL_TRIANGLE && !sc.walls.empty() && sc.walls.back().type == WALL_TRIANGLE)
        return fail(w, DEM_ERR_STATE, "add a scene's meshes after its other walls");
    sc.walls.push_back(ws);
    if (id) *id = (int32_t)sc.walls.size() - 1;
    return DEM_OK;
}

static bool unit(const double *n, double out[3])
{
    if (!n || !finite3(n)) return false;
    double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(l > 0)) return false;
    for (int a = 0; a < 3; ++a) out[a] = n[a] / l;
    return true;
}

dem_status dem_add_box_walls(dem_world *w, int32_t mat, int32_t *first_id)
{
    CHECK_SETUP(w);
    const dem_world_desc &d = S(w).desc;
    int32_t first = -1;
    for (int a = 0; a < 3; ++a)
        for (int side = 0; side < 2; ++side) {
            WallSetup ws{};
            ws.type = WALL_PLANE;
            ws.mat = mat;
            for (int b = 0; b < 3; ++b) ws.p[b] = side ? d.box_hi[b] : d.box_lo[b];
            ws.n[a] = side ? -1.0 : 1.0;
            int32_t id;
            dem_status s = add_wall(w, ws, &id);
            if (s) return s;
            if (first < 0) first = id;
        }
    if (first_id) *first_id = first;
    return DEM_OK;
}

dem_status dem_add_plane(dem_world *w, const double p[3], const double n[3], int32_t mat, int32_t *id)
{
    CHECK_SETUP(w);
    WallSetup ws{};
    ws.type = WALL_PLANE;
    ws.mat = mat;
    if (!p || !finite3(p) || !unit(n, ws.n)) return fail(w, DEM_ERR_ARG, "bad plane");
    for (int a = 0; a < 3; ++a) ws.p[a] = p[a];
    return add_wall(w, ws, id);
}

dem_status dem_add_cylinder(dem_world *w, const double c[3], const double axis[3], double radius, int32_t mat,
                            double omega, int32_t *id)
{
    CHECK_SETUP(w);
    WallSetup ws{};
    ws.type = WALL_CYLINDER;
    ws.mat = mat;
    if (!c || !finite3(c) || !unit(axis, ws.n) || !(radius > 0) || !std::isfinite(omega))
        return fail(w, DEM_ERR_ARG, "bad cylinder");
    for (int a = 0; a < 3; ++a) { ws.p[a] = c[a]; ws.omega[a] = omega * ws.n[a]; }
    ws.r0 = radius;
    return add_wall(w, ws, id);
}

dem_status dem_add_cone_segment(dem_world *w, const double p[3], const double axis[3], double r0, double z0, double r1,
                                double z1, int32_t mat, int32_t *id)
{
    CHECK_SETUP(w);
    WallSetup ws{};
    ws.type = WALL_CONE;
    ws.mat = mat;
    if (!p || !finite3(p) || !unit(axis, ws.n) || !(r0 >= 0) || !(r1 >= 0) || !std::isfinite(z0) ||
        !std::isfinite(z1) || ((r1 - r0) * (r1 - r0) + (z1 - z0) * (z1 - z0)) <= 0)
        return fail(w, DEM_ERR_ARG, "bad cone segment");
    for (int a = 0; a < 3; ++a) ws.p[a] = p[a];
    ws.r0 = r0; ws.z0 = z0; ws.r1 = r1; ws.z1 = z1;
    return add_wall(w, ws, id);
}

dem_status dem_set_wall_spin(dem_world *w, int32_t id, const double omega[3])
{
    CHECK_SETUP(w);
    SceneSetup &sc = S(w);
    if (id < 0 || id >= (int)sc.walls.size() || !omega || !finite3(omega)) return fail(w, DEM_ERR_ARG, "bad wall spin");
    WallSetup &ws = sc.walls[id];
    // the spin must leave the geometry invariant: parallel to the normal / axis
    double c[3] = {omega[1] * ws.n[2] - omega[2] * ws.n[1], omega[2] * ws.n[0] - omega[0] * ws.n[2],
                   omega[0] * ws.n[1] - omega[1] * ws.n[0]};
    double on = std::sqrt(omega[0] * omega[0] + omega[1] * omega[1] + omega[2] * omega[2]);
    if (std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]) > 1e-12 * (on + 1e-300))
        return fail(w, DEM_ERR_ARG, "wall spin must be parallel to the wall normal or axis");
    for (int a = 0; a < 3; ++a) ws.omega[a] = omega[a];
    return DEM_OK;
}

dem_status dem_add_clump_template(dem_world *w, int32_t n, const double *rel_xyz, const double *radii,
                                  const int32_t *mats, double mass, const double moi[3], int32_t *tid)
{
    CHECK_SETUP(w);
    SceneSetup &sc = S(w);
    if (n < 1 || n > 32 || !rel_xyz || !radii || !mats || !moi) return fail(w, DEM_ERR_ARG, "bad template (1..32 spheres)");
    if (!(mass > 0) || !(moi[0] > 0) || !(moi[1] > 0) || !(moi[2] > 0) || !std::isfinite(mass))
        return fail(w, DEM_ERR_ARG, "template mass and moments must be positive");
    TemplateSetup t;
    for (int k = 0; k < n; ++k) {
        if (!(radii[k] > 0) || !finite3(rel_xyz + 3 * k)) return fail(w, DEM_ERR_ARG, "bad template sphere");
        if (mats[k] < 0 || mats[k] >= (int)sc.E.size()) return fail(w, DEM_ERR_ARG, "bad material id");
        t.rel.insert(t.rel.end(), rel_xyz + 3 * k, rel_xyz + 3 * k + 3);
        t.rad.push_back(radii[k]);
        t.mats.push_back(mats[k]);
    }
    t.mass = mass;
    for (int a = 0; a < 3; ++a) t.moi[a] = moi[a];
    sc.templates.push_back(t);
    if (tid) *tid = (int32_t)sc.templates.size() - 1;
    return DEM_OK;
}

dem_status dem_add_clumps(dem_world *w, int32_t tid, int64_t n, const double *xyz, const double *quat,
                          const double *vel, const double *omega, const double *scale, int64_t *first_id)
{
    CHECK_SETUP(w);
    SceneSetup &sc = S(w);
    if (tid < 0 || tid >= (int)sc.templates.size()) return fail(w, DEM_ERR_ARG, "bad template id");
    if (n < 0 || (n > 0 && !xyz)) return fail(w, DEM_ERR_ARG, "bad clump count or positions");
    int64_t first = (int64_t)sc.inst_tid.size();
    for (int64_t k = 0; k < n; ++k) {
        if (!finite3(xyz + 3 * k)) return fail(w, DEM_ERR_ARG, "non-finite position");
        if (vel && !finite3(vel + 3 * k)) return fail(w, DEM_ERR_ARG, "non-finite velocity");
        if (omega && !finite3(omega + 3 * k)) return fail(w, DEM_ERR_ARG, "non-finite angular velocity");
        if (scale && !(scale[k] > 0 && std::isfinite(scale[k]))) return fail(w, DEM_ERR_ARG, "bad scale");
        if (quat) {
            const double *q = quat + 4 * k;
            double qn = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
            if (!(qn > 0) || !std::isfinite(qn)) return fail(w, DEM_ERR_ARG, "bad quaternion");
        }
    }
    sc.inst_tid.insert(sc.inst_tid.end(), (size_t)n, tid);
    sc.inst_x.insert(sc.inst_x.end(), xyz, xyz + 3 * n);
    for (int64_t k = 0; k < n; ++k) {
        if (quat) sc.inst_q.insert(sc.inst_q.end(), quat + 4 * k, quat + 4 * k + 4);
        else { sc.inst_q.push_back(1.0); sc.inst_q.push_back(0.0); sc.inst_q.push_back(0.0); sc.inst_q.push_back(0.0); }
        for (int a = 0; a < 3; ++a) {
            sc.inst_v.push_back(vel ? vel[3 * k + a] : 0.0);
            sc.inst_w.push_back(omega ? omega[3 * k + a] : 0.0);
        }
        sc.inst_s.push_back(scale ? scale[k] : 1.0);
    }
    if (first_id) *first_id = first;
    return DEM_OK;
}

dem_status dem_add_clumps_mixed(dem_world *w, int64_t n, const int32_t *tids, const double *xyz, const double *quat,
                                const double *vel, const double *omega, const double *scale, int64_t *first_id)
{
    CHECK_SETUP(w);
    SceneSetup &sc = S(w);
    if (n < 0 || (n > 0 && (!xyz || !tids))) return fail(w, DEM_ERR_ARG, "bad clump count, ids or positions");
    for (int64_t k = 0; k < n; ++k)
        if (tids[k] < 0 || tids[k] >= (int)sc.templates.size()) return fail(w, DEM_ERR_ARG, "bad template id");
    const size_t before = sc.inst_tid.size();
    int64_t first = (int64_t)before;
    // validate and append through the single-template path, then patch the template ids
    dem_status s = dem_add_clumps(w, 0, n, xyz, quat, vel, omega, scale, nullptr);
    if (s) return s;
    for (int64_t k = 0; k < n; ++k) sc.inst_tid[before + k] = tids[k];
    if (first_id) *first_id = first;
    return DEM_OK;
}

dem_status dem_set_timestep(dem_world *w, double h)
{
    CHECK_SETUP(w);
    if (!(h > 0) || !std::isfinite(h)) return fail(w, DEM_ERR_ARG, "time step must be positive");
    S(w).h = h;
    return DEM_OK;
}

dem_status dem_set_gravity(dem_world *w, const double g[3])
{
    CHECK_SETUP(w);
    if (!g || !finite3(g)) return fail(w, DEM_ERR_ARG, "bad gravity");
    for (int a = 0; a < 3; ++a) S(w).g[a] = g[a];
    return DEM_OK;
}

dem_status dem_set_error_velocity(dem_world *w, double v)
{
    CHECK_SETUP(w);
    if (!(v >= 0) || !std::isfinite(v)) return fail(w, DEM_ERR_ARG, "error-out velocity must be >= 0");
    S(w).v_err = v;
    return DEM_OK;
}

dem_status dem_set_margin(dem_world *w, double beta)
{
    CHECK_W(w);
    if (!(beta >= 0) || !std::isfinite(beta)) return fail(w, DEM_ERR_ARG, "margin must be >= 0");
    if (w->impl->initialized) {
        if (beta > w->impl->model.margin_max) return fail(w, DEM_ERR_ARG, "margin exceeds margin_max");
        std::string err;
        dem_status s = w->impl->engine->set_margin(beta, err);
        return s ? fail(w, s, err) : DEM_OK;
    }
    S(w).margin = beta;
    return DEM_OK;
}

dem_status dem_set_sink(dem_world *w, const double p[3], const double n[3])
{
    CHECK_SETUP(w);
    SceneSetup &sc = S(w);
    if (!p || !finite3(p) || !unit(n, sc.sink_n)) return fail(w, DEM_ERR_ARG, "bad sink plane");
    for (int a = 0; a < 3; ++a) sc.sink_p[a] = p[a];
    sc.has_sink = true;
    return DEM_OK;
}

dem_status dem_load_schedule_model(dem_world *w, const void *weights, size_t bytes)
{
    CHECK_W(w);
    if (!weights && bytes) return fail(w, DEM_ERR_ARG, "null weights");
    const uint8_t *p = (const uint8_t *)weights;
    w->impl->schedule_model.assign(p, p + bytes);
    if (w->impl->initialized) {
        std::string err;
        dem_status s = w->impl->engine->schedule_load(p, bytes, err);
        return s ? fail(w, s, err) : DEM_OK;
    }
    return DEM_OK;
}

dem_status dem_initialize(dem_world *w)
{
    CHECK_SETUP(w);
    if (w->proxy) return fail(w, DEM_ERR_STATE, "initialize a batch with dem_batch_initialize");
    return do_initialize(*w->impl, w);
}

dem_status dem_step(dem_world *w, int64_t nsteps)
{
    CHECK_INIT(w);
    if (w->proxy) return fail(w, DEM_ERR_STATE, "step a batch with dem_batch_step");
    std::string err;
    dem_status s = w->impl->engine->step(nsteps, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_sync(dem_world *w)
{
    CHECK_INIT(w);
    std::string err;
    dem_status s = w->impl->engine->sync(err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_set_profiling(dem_world *w, int32_t on)
{
    CHECK_INIT(w);
    w->impl->engine->set_profiling(on != 0);
    return DEM_OK;
}

dem_status dem_set_tuning(dem_world *w, const dem_tuning *t)
{
    CHECK_INIT(w);
    if (!t) return fail(w, DEM_ERR_ARG, "null tuning");
    std::string err;
    dem_status s = w->impl->engine->set_tuning(t, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_get_tuning(dem_world *w, dem_tuning *t)
{
    CHECK_INIT(w);
    if (!t) return fail(w, DEM_ERR_ARG, "null tuning");
    std::string err;
    dem_status s = w->impl->engine->get_tuning(t, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_autotune(dem_world *w, int32_t steps, const char *cache_path, dem_tuning *chosen)
{
    CHECK_INIT(w);
    if (steps < 1) return fail(w, DEM_ERR_ARG, "steps must be >= 1");
    std::string err;
    dem_status s = w->impl->engine->autotune(steps, cache_path, chosen, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_set_graphs(dem_world *w, int32_t on)
{
    CHECK_INIT(w);
    w->impl->engine->set_graphs(on != 0);
    return DEM_OK;
}

dem_status dem_get_stream(dem_world *w, void **stream)
{
    CHECK_INIT(w);
    if (!stream) return fail(w, DEM_ERR_ARG, "null output");
    *stream = w->impl->engine->stream();
    return DEM_OK;
}

dem_status dem_get_owner_state(dem_world *w, int64_t first, int64_t n, double *xyz, double *quat, double *vel,
                               double *omega)
{
    CHECK_INIT(w);
    if (first < 0 || n < 0 || first + n > scene_owners(w)) return fail(w, DEM_ERR_ARG, "owner range out of bounds");
    std::string err;
    dem_status s = w->impl->engine->owner_state(owner_base(w) + first, n, xyz, quat, vel, omega, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_set_owner_state(dem_world *w, int64_t first, int64_t n, const double *xyz, const double *quat,
                               const double *vel, const double *omega)
{
    CHECK_INIT(w);
    if (first < 0 || n < 0 || first + n > scene_owners(w)) return fail(w, DEM_ERR_ARG, "owner range out of bounds");
    // non-finite positions and velocities are rejected on the device before any is applied
    std::string err;
    dem_status s = w->impl->engine->set_owner_state(owner_base(w) + first, n, xyz, quat, vel, omega, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_get_sphere_positions(dem_world *w, int64_t first, int64_t n, double *xyz, double *radius)
{
    CHECK_INIT(w);
    if (first < 0 || n < 0 || first + n > scene_spheres(w)) return fail(w, DEM_ERR_ARG, "sphere range out of bounds");
    std::string err;
    dem_status s = w->impl->engine->sphere_positions(sphere_base(w) + first, n, xyz, radius, nullptr, nullptr, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_get_sphere_voxels(dem_world *w, int64_t first, int64_t n, int32_t *cell, float *offset, double *edge)
{
    CHECK_INIT(w);
    if (first < 0 || n < 0 || first + n > scene_spheres(w)) return fail(w, DEM_ERR_ARG, "sphere range out of bounds");
    if (w->impl->desc.precision != DEM_PRECISION_VOXEL_FP32)
        return fail(w, DEM_ERR_STATE, "voxel encoding exists only in the VOXEL_FP32 form");
    if (edge) *edge = w->impl->model.Lv;
    if (n == 0) return DEM_OK;
    if (!cell || !offset) return fail(w, DEM_ERR_ARG, "null output");
    std::string err;
    dem_status s = w->impl->engine->sphere_positions(sphere_base(w) + first, n, nullptr, nullptr, cell, offset, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_get_contacts(dem_world *w, int64_t cap, int64_t *count, int64_t *i, int64_t *j, double *force,
                            double *point, double *overlap, double *history)
{
    CHECK_INIT(w);
    if (!count) return fail(w, DEM_ERR_ARG, "null count");
    std::vector<ContactOut> cs;
    std::string err;
    dem_status s = w->impl->engine->contacts(cs, err);
    if (s) return fail(w, s, err);
    const int64_t b = sphere_base(w), e = b + scene_spheres(w);
    int64_t c = 0;
    for (auto &x : cs) {
        if (x.i < b || x.i >= e) continue;
        if (c < cap) {
            if (i) i[c] = x.i - b;
            if (j) j[c] = x.j >= 0 ? x.j - b : x.j;
            for (int a = 0; a < 3; ++a) {
                if (force) force[3 * c + a] = x.force[a];
                if (point) point[3 * c + a] = x.point[a];
                if (history) history[3 * c + a] = x.hist[a];
            }
            if (overlap) overlap[c] = x.overlap;
        }
        ++c;
    }
    *count = c;
    return c > cap ? fail(w, DEM_ERR_CAPACITY, "contact buffer too small") : DEM_OK;
}

dem_status dem_get_listed_pairs(dem_world *w, int64_t cap, int64_t *count, int64_t *i, int64_t *j)
{
    CHECK_INIT(w);
    if (!count) return fail(w, DEM_ERR_ARG, "null count");
    std::vector<int64_t> pi, pj, si, wi;
    std::string err;
    dem_status s = w->impl->engine->listed(pi, pj, si, wi, err);
    if (s) return fail(w, s, err);
    const int64_t b = sphere_base(w), e = b + scene_spheres(w);
    int64_t c = 0;
    for (size_t k = 0; k < pi.size(); ++k) {
        if (pi[k] < b || pi[k] >= e) continue;
        if (c < cap) {
            if (i) i[c] = pi[k] - b;
            if (j) j[c] = pj[k] - b;
        }
        ++c;
    }
    *count = c;
    return c > cap ? fail(w, DEM_ERR_CAPACITY, "pair buffer too small") : DEM_OK;
}

dem_status dem_get_listed_wall_pairs(dem_world *w, int64_t cap, int64_t *count, int64_t *sphere, int64_t *wall)
{
    CHECK_INIT(w);
    if (!count) return fail(w, DEM_ERR_ARG, "null count");
    std::vector<int64_t> pi, pj, si, wi;
    std::string err;
    dem_status s = w->impl->engine->listed(pi, pj, si, wi, err);
    if (s) return fail(w, s, err);
    const int64_t b = sphere_base(w), e = b + scene_spheres(w);
    int64_t c = 0;
    for (size_t k = 0; k < si.size(); ++k) {
        if (si[k] < b || si[k] >= e) continue;
        if (c < cap) {
            if (sphere) sphere[c] = si[k] - b;
            if (wall) wall[c] = wi[k];
        }
        ++c;
    }
    *count = c;
    return c > cap ? fail(w, DEM_ERR_CAPACITY, "pair buffer too small") : DEM_OK;
}

dem_status dem_get_owner_forces(dem_world *w, int64_t first, int64_t n, double *force, double *torque)
{
    CHECK_INIT(w);
    if (first < 0 || n < 0 || first + n > scene_owners(w)) return fail(w, DEM_ERR_ARG, "owner range out of bounds");
    std::vector<double> F, T;
    std::string err;
    dem_status s = w->impl->engine->owner_forces(F, T, err);
    if (s) return fail(w, s, err);
    const int64_t b = owner_base(w) + first;
    if (force) std::memcpy(force, F.data() + 3 * b, 3 * n * sizeof(double));
    if (torque) std::memcpy(torque, T.data() + 3 * b, 3 * n * sizeof(double));
    return DEM_OK;
}

// ---------------------------------------------------------------- meshes (Sec. 2.4)

dem_status dem_add_mesh(dem_world *w, int64_t n_facets, const double *vertices, int32_t mat, const double axis_point[3],
                        const double omega[3], int32_t *first_id)
{
    CHECK_SETUP(w);
    if (n_facets <= 0 || !vertices || !axis_point || !omega) return fail(w, DEM_ERR_ARG, "bad mesh arrays");
    if (!finite3(axis_point) || !finite3(omega)) return fail(w, DEM_ERR_ARG, "non-finite axis point or omega");
    SceneSetup &sc = S(w);
    if (mat < 0 || mat >= (int)sc.E.size()) return fail(w, DEM_ERR_ARG, "bad material id");
    for (int64_t f = 0; f < n_facets; ++f) {
        const double *v = vertices + 9 * f;
        for (int q = 0; q < 9; ++q)
            if (!std::isfinite(v[q])) return fail(w, DEM_ERR_ARG, "non-finite facet vertex");
        const double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
        const double e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
        const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        if (!((c[0] * c[0] + c[1] * c[1] + c[2] * c[2]) > 0.0)) return fail(w, DEM_ERR_ARG, "degenerate facet");
    }
    if (first_id) *first_id = (int32_t)sc.walls.size();
    for (int64_t f = 0; f < n_facets; ++f) {
        WallSetup ws{};
        ws.type = WALL_TRIANGLE;
        ws.mat = mat;
        for (int a = 0; a < 3; ++a) { ws.p[a] = axis_point[a]; ws.omega[a] = omega[a]; }
        for (int q = 0; q < 9; ++q) ws.tri[q] = vertices[9 * f + q];
        sc.walls.push_back(ws);
    }
    return DEM_OK;
}

// ---------------------------------------------------------------- contact force models (Sec. 4.2)

dem_status dem_set_force_model(dem_world *w, int32_t model, const double *params, int32_t n_params)
{
    CHECK_SETUP(w);
    int need;
    switch (model) {
    case DEM_MODEL_DEFAULT: need = 0; break;
    case DEM_MODEL_HERTZ_MINDLIN: need = ModelHertzMindlin::n_params; break;
    case DEM_MODEL_BONDED_BREAKAGE: need = ModelBondedBreakage::n_params; break;
    default: return fail(w, DEM_ERR_ARG, "unknown contact model");
    }
    if (n_params != need || (need > 0 && !params)) return fail(w, DEM_ERR_ARG, "wrong number of model parameters");
    for (int k = 0; k < n_params; ++k)
        if (!std::isfinite(params[k])) return fail(w, DEM_ERR_ARG, "non-finite model parameter");
    WorldImpl &W = *w->impl;
    W.force_model = model == DEM_MODEL_DEFAULT ? FORCE_MODEL_BUILTIN
                                               : (model == DEM_MODEL_HERTZ_MINDLIN ? FORCE_MODEL_HERTZ_MINDLIN
                                                                                    : FORCE_MODEL_BONDED_BREAKAGE);
    W.force_params.assign(params, params + n_params);
    return DEM_OK;
}

dem_status dem_set_contact_wildcards(dem_world *w, int64_t k, const int64_t *i, const int64_t *j, const double *wc)
{
    CHECK_INIT(w);
    if (k < 0 || (k > 0 && (!i || !j || !wc))) return fail(w, DEM_ERR_ARG, "bad wildcard arrays");
    const int64_t b = sphere_base(w);
    std::vector<int64_t> gi(k), gj(k);
    for (int64_t q = 0; q < k; ++q) {
        if (i[q] < 0 || j[q] < 0) return fail(w, DEM_ERR_ARG, "wildcards are for sphere pairs");
        gi[q] = std::min(i[q], j[q]) + b;
        gj[q] = std::max(i[q], j[q]) + b;
    }
    std::string err;
    dem_status s = w->impl->engine->set_wildcards(k, gi.data(), gj.data(), wc, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_get_contact_wildcards(dem_world *w, int64_t cap, int64_t *count, double *wc)
{
    CHECK_INIT(w);
    if (!count) return fail(w, DEM_ERR_ARG, "null count");
    std::vector<ContactOut> cs;
    std::string err;
    dem_status s = w->impl->engine->contacts(cs, err);
    if (s) return fail(w, s, err);
    const int64_t b = sphere_base(w), e = b + scene_spheres(w);
    int64_t c = 0;
    for (auto &x : cs) {
        if (x.i < b || x.i >= e) continue;
        if (c < cap && wc)
            for (int q = 0; q < 8; ++q) wc[8 * c + q] = x.wc[q];
        ++c;
    }
    *count = c;
    return c > cap ? fail(w, DEM_ERR_CAPACITY, "wildcard buffer too small") : DEM_OK;
}

// ---------------------------------------------------------------- family tags (Sec. 2.2.2)

static void families_on(WorldImpl &W)
{
    if (!W.families_used) {
        family_defaults(W.fam_motion, W.fam_mask);
        W.families_used = true;
    }
}

dem_status dem_set_family(dem_world *w, int64_t first, int64_t n, const uint8_t *family)
{
    CHECK_W(w);
    if (n < 0 || first < 0 || (n > 0 && !family)) return fail(w, DEM_ERR_ARG, "bad family range");
    WorldImpl &W = *w->impl;
    if (W.initialized) {
        if (first + n > scene_owners(w)) return fail(w, DEM_ERR_ARG, "owner range out of bounds");
        std::string err;
        dem_status s = W.engine->set_family(owner_base(w) + first, n, family, err);
        return s ? fail(w, s, err) : DEM_OK;
    }
    SceneSetup &sc = S(w);
    if (first + n > (int64_t)sc.inst_tid.size()) return fail(w, DEM_ERR_ARG, "owner range out of bounds");
    if ((int64_t)sc.inst_family.size() < first + n) sc.inst_family.resize((size_t)(first + n), 0);
    std::copy(family, family + n, sc.inst_family.begin() + first);
    families_on(W);
    return DEM_OK;
}

dem_status dem_set_family_motion(dem_world *w, int32_t family, const double *v, const double *omega)
{
    CHECK_W(w);
    if (family < 0 || family >= N_FAMILY) return fail(w, DEM_ERR_ARG, "family must be in [0, 255]");
    if ((v && !finite3(v)) || (omega && !finite3(omega))) return fail(w, DEM_ERR_ARG, "non-finite velocity");
    WorldImpl &W = *w->impl;
    families_on(W);
    family_set_motion(W.fam_motion[family], v, omega);
    if (W.initialized) {
        std::string err;
        dem_status s = W.engine->set_family_motion(family, v, omega, err);
        return s ? fail(w, s, err) : DEM_OK;
    }
    return DEM_OK;
}

dem_status dem_set_family_contacts(dem_world *w, int32_t fa, int32_t fb, int32_t on)
{
    CHECK_W(w);
    if (fa < 0 || fa >= N_FAMILY || fb < 0 || fb >= N_FAMILY) return fail(w, DEM_ERR_ARG, "family must be in [0, 255]");
    WorldImpl &W = *w->impl;
    families_on(W);
    family_set_contacts(W.fam_mask, fa, fb, on);
    if (W.initialized) {
        std::string err;
        dem_status s = W.engine->set_family_contacts(fa, fb, on, err);
        return s ? fail(w, s, err) : DEM_OK;
    }
    return DEM_OK;
}

dem_status dem_set_active_box(dem_world *w, const double lo[3], const double hi[3], int32_t family_inside,
                              int32_t family_outside)
{
    CHECK_INIT(w);
    if (!lo || !hi || !finite3(lo) || !finite3(hi)) return fail(w, DEM_ERR_ARG, "bad box");
    if (family_inside < 0 || family_inside >= N_FAMILY || family_outside < 0 || family_outside >= N_FAMILY)
        return fail(w, DEM_ERR_ARG, "family must be in [0, 255]");
    std::string err;
    dem_status s = w->impl->engine->set_active_box(owner_base(w), scene_owners(w), lo, hi, family_inside,
                                                   family_outside, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_get_contact_rolling(dem_world *w, int64_t cap, int64_t *count, double *age, double *torque_force)
{
    CHECK_INIT(w);
    if (!count) return fail(w, DEM_ERR_ARG, "null count");
    std::vector<ContactOut> cs;
    std::string err;
    dem_status s = w->impl->engine->contacts(cs, err);
    if (s) return fail(w, s, err);
    const int64_t b = sphere_base(w), e = b + scene_spheres(w);
    int64_t c = 0;
    for (auto &x : cs) {
        if (x.i < b || x.i >= e) continue;
        if (c < cap) {
            if (age) age[c] = x.age;
            for (int a = 0; a < 3; ++a)
                if (torque_force) torque_force[3 * c + a] = x.trf[a];
        }
        ++c;
    }
    *count = c;
    return c > cap ? fail(w, DEM_ERR_CAPACITY, "contact buffer too small") : DEM_OK;
}

dem_status dem_set_history(dem_world *w, int64_t k, const int64_t *i, const int64_t *j, const double *ut)
{
    return dem_set_history_age(w, k, i, j, ut, nullptr);
}

dem_status dem_set_history_age(dem_world *w, int64_t k, const int64_t *i, const int64_t *j, const double *ut,
                               const double *age)
{
    CHECK_INIT(w);
    if (k < 0 || (k > 0 && (!i || !j || !ut))) return fail(w, DEM_ERR_ARG, "bad history arrays");
    const int64_t b = sphere_base(w);
    std::vector<int64_t> gi(k), gj(k);
    for (int64_t q = 0; q < k; ++q) {
        gi[q] = i[q] + b;
        gj[q] = j[q] >= 0 ? j[q] + b : j[q];
    }
    std::string err;
    dem_status s = w->impl->engine->set_history(k, gi.data(), gj.data(), ut, age, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_get_stats(dem_world *w, dem_stats *st)
{
    CHECK_INIT(w);
    if (!st) return fail(w, DEM_ERR_ARG, "null output");
    std::string err;
    dem_status s = w->impl->engine->stats(st, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_get_diagnostics(dem_world *w, dem_diagnostics *d)
{
    CHECK_INIT(w);
    if (!d) return fail(w, DEM_ERR_ARG, "null output");
    std::string err;
    dem_status s = w->impl->engine->diagnostics(d, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_save_state(dem_world *w, void *buf, size_t cap, size_t *used)
{
    CHECK_INIT(w);
    if (!used) return fail(w, DEM_ERR_ARG, "null size output");
    std::vector<uint8_t> blob;
    std::string err;
    dem_status s = w->impl->engine->save(blob, err);
    if (s) return fail(w, s, err);
    *used = blob.size();
    if (blob.size() > cap || !buf) return fail(w, DEM_ERR_CAPACITY, "state buffer too small");
    std::memcpy(buf, blob.data(), blob.size());
    return DEM_OK;
}

dem_status dem_load_state(dem_world *w, const void *buf, size_t bytes)
{
    CHECK_INIT(w);
    if (!buf) return fail(w, DEM_ERR_ARG, "null buffer");
    std::string err;
    dem_status s = w->impl->engine->load((const uint8_t *)buf, bytes, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_batch_create(int32_t nscenes, const dem_world_desc *descs, dem_batch **out)
{
    if (!out) return fail(nullptr, DEM_ERR_ARG, "null output handle");
    *out = nullptr;
    if (nscenes < 1 || nscenes > 65535 || !descs) return fail(nullptr, DEM_ERR_ARG, "bad scene count");
    for (int k = 0; k < nscenes; ++k) {
        dem_status s = check_desc(&descs[k]);
        if (s) return s;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(nullptr, DEM_ERR_CUDA, "no CUDA device available");
    WorldImpl *W = new WorldImpl;
    W->desc = descs[0];
    W->scenes.resize(nscenes);
    dem_batch *b = new dem_batch;
    b->impl = W;
    for (int k = 0; k < nscenes; ++k) {
        W->scenes[k].desc = descs[k];
        b->handles.push_back(new_handle(W, k, true));
    }
    *out = b;
    return DEM_OK;
}

dem_status dem_batch_world(dem_batch *b, int32_t k, dem_world **scene)
{
    if (!b || !scene || k < 0 || k >= (int)b->handles.size()) return fail(nullptr, DEM_ERR_ARG, "bad batch scene");
    *scene = b->handles[k];
    return DEM_OK;
}

dem_status dem_batch_initialize(dem_batch *b)
{
    if (!b) return fail(nullptr, DEM_ERR_ARG, "null batch");
    if (b->impl->initialized) return fail(b->handles[0], DEM_ERR_STATE, "batch already initialized");
    dem_status s = do_initialize(*b->impl, b->handles[0]);
    if (s) g_err = b->impl->err;
    return s;
}

dem_status dem_batch_step(dem_batch *b, int64_t nsteps)
{
    if (!b) return fail(nullptr, DEM_ERR_ARG, "null batch");
    if (!b->impl->initialized) return fail(b->handles[0], DEM_ERR_STATE, "batch not initialized");
    std::string err;
    dem_status s = b->impl->engine->step(nsteps, err);
    if (s) {
        b->impl->err = err;
        g_err = err;
    }
    return s;
}

dem_status dem_batch_destroy(dem_batch *b)
{
    if (!b) return DEM_OK;
    for (auto *h : b->handles) delete h;
    delete b->impl;
    delete b;
    return DEM_OK;
}

dem_status dem_schedule_collect(dem_world *w, int32_t on)
{
    CHECK_INIT(w);
    std::string err;
    dem_status s = w->impl->engine->schedule_collect(on, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_schedule_train(dem_world *w, int32_t epochs, float lr, uint64_t seed, float *final_loss)
{
    CHECK_INIT(w);
    std::string err;
    dem_status s = w->impl->engine->schedule_train(epochs, lr, seed, final_loss, err);
    return s ? fail(w, s, err) : DEM_OK;
}

dem_status dem_schedule_export(dem_world *w, void *buf, size_t cap, size_t *used)
{
    CHECK_INIT(w);
    if (!used) return fail(w, DEM_ERR_ARG, "null size output");
    std::vector<uint8_t> blob;
    std::string err;
    dem_status s = w->impl->engine->schedule_export(blob, err);
    if (s) return fail(w, s, err);
    *used = blob.size();
    if (blob.size() > cap || !buf) return fail(w, DEM_ERR_CAPACITY, "weight buffer too small");
    std::memcpy(buf, blob.data(), blob.size());
    return DEM_OK;
}

static dem_status mlp_util(const float *params, int32_t rows, const float *X, const float *Y, float *out, float *loss,
                           float *grad)
{
    if (!params || rows < 1 || !X) return fail(nullptr, DEM_ERR_ARG, "bad MLP arguments");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(nullptr, DEM_ERR_CUDA, "no CUDA device available");
    Mlp net;
    float *dx = nullptr, *dy = nullptr, *dout = nullptr;
    cudaError_t e = net.set_params(params, 0);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dx, (size_t)rows * MLP_IN * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dx, X, (size_t)rows * MLP_IN * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && out) {
        e = cudaMalloc((void **)&dout, (size_t)rows * MLP_OUT * sizeof(float));
        if (e == cudaSuccess) e = net.forward(dx, rows, dout, 0);
        if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)rows * MLP_OUT * sizeof(float), cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess && Y) {
        e = cudaMalloc((void **)&dy, (size_t)rows * MLP_OUT * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpy(dy, Y, (size_t)rows * MLP_OUT * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = net.loss_grad(dx, dy, rows, loss, grad, 0);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (dx) cudaFree(dx);
    if (dy) cudaFree(dy);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) return fail(nullptr, DEM_ERR_CUDA, cudaGetErrorString(e));
    return DEM_OK;
}

dem_status dem_util_mlp_forward(const float *params, int32_t rows, const float *X, float *out)
{
    if (!out) return fail(nullptr, DEM_ERR_ARG, "null output");
    return mlp_util(params, rows, X, nullptr, out, nullptr, nullptr);
}

dem_status dem_util_mlp_loss_grad(const float *params, int32_t rows, const float *X, const float *Y, float *loss,
                                  float *grad)
{
    if (!Y || !grad) return fail(nullptr, DEM_ERR_ARG, "null labels or gradient");
    return mlp_util(params, rows, X, Y, nullptr, loss, grad);
}

dem_status dem_util_radix_sort_u32(int64_t n, const uint32_t *keys, const uint32_t *vals, int32_t bits,
                                   uint32_t *keys_out, uint32_t *vals_out)
{
    if (n < 0 || bits < 1 || bits > 32 || (n > 0 && (!keys || !vals || !keys_out || !vals_out)))
        return fail(nullptr, DEM_ERR_ARG, "bad sort arguments");
    if (n == 0) return DEM_OK;
    if (n > 0x7fffffff) return fail(nullptr, DEM_ERR_ARG, "too many keys");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(nullptr, DEM_ERR_CUDA, "no CUDA device available");
    uint32_t *buf = nullptr;
    int64_t hc = radix_hist_entries(n);
    size_t bytes = (size_t)(4 * n + hc) * sizeof(uint32_t);
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return fail(nullptr, DEM_ERR_NOMEM, "cudaMalloc failed");
    uint32_t *k0 = buf, *v0 = buf + n, *k1 = buf + 2 * n, *v1 = buf + 3 * n, *h = buf + 4 * n;
    cudaMemcpy(k0, keys, n * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(v0, vals, n * 4, cudaMemcpyHostToDevice);
    uint32_t *ko, *vo;
    radix_sort_u32(k0, v0, k1, v1, n, bits, h, hc, 0, &ko, &vo);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(keys_out, ko, n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(vals_out, vo, n * 4, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(nullptr, DEM_ERR_CUDA, cudaGetErrorString(e));
    return DEM_OK;
}

}  // extern "C"
