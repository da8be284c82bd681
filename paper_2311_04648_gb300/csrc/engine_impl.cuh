// engine_impl.cuh -- host orchestration of the pipeline for one position form.
//
// Streams: the force stream runs the per-step work (force + integration + audit) and the
// list switch; the detection stream runs the sort, cell tables and narrow phase of the
// next list from a snapshot, concurrently (Sec. 2.1: contact detection and dynamics as
// two concurrent workers, here two CUDA streams on one GPU instead of two GPUs).
// All control state lives on the device (DevStatus): kernels pick the buffers and skip
// themselves when the list in use went stale or the run halted, so queued work never
// needs host decisions; the host reads the status at cycle ends and recovers
// (audit fallback rebuild, list capacity regrow, divergence report).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "engine.h"
#include "mlp.h"
#include "pipeline.cuh"

namespace dem {

#define DEM_CU(call)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return DEM_ERR_CUDA;                                                      \
        }                                                                             \
    } while (0)

template <class F>
class Engine : public EngineBase {
    using R = typename F::R;
    using R4 = typename F::R4;

public:
    ~Engine() override { release(); }

    dem_status init(HostModel &m, std::string &err) override
    {
        m_ = m;
        DEM_CU(cudaSetDevice(m_.device));
        // the force stream gets the highest priority: the detection of the next list fills
        // the SMs only where the step in progress leaves room
        int prio_lo = 0, prio_hi = 0;
        DEM_CU(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        if (m_.stream) {
            sf_ = (cudaStream_t)m_.stream;
        } else {
            DEM_CU(cudaStreamCreateWithPriority(&sf_, cudaStreamNonBlocking, prio_hi));
            own_sf_ = true;
        }
        if (m_.detect_stream) {
            sd_ = (cudaStream_t)m_.detect_stream;
        } else {
            DEM_CU(cudaStreamCreateWithPriority(&sd_, cudaStreamNonBlocking, prio_lo));
            own_sd_ = true;
        }
        DEM_CU(cudaEventCreateWithFlags(&ev_snap_, cudaEventDisableTiming));
        DEM_CU(cudaEventCreateWithFlags(&ev_det_, cudaEventDisableTiming));
        DEM_CU(cudaEventCreate(&ev_a_));
        DEM_CU(cudaEventCreate(&ev_b_));
        DEM_CU(cudaEventCreate(&ev_c_));
        // host uploads are copied on a stream of their own, so that the force stream can
        // check each piece while the next one is copied
        DEM_CU(cudaStreamCreateWithFlags(&sc_, cudaStreamNonBlocking));
        DEM_CU(cudaEventCreateWithFlags(&ev_up_, cudaEventDisableTiming));

        const int64_t M = (int64_t)m_.mass.size();
        const int64_t N = (int64_t)m_.sph_owner.size();
        d_.M = M;
        d_.N = N;
        d_.Np = std::max<int64_t>(32, (N + 31) / 32 * 32);
        d_.K = 16;
        // position unit: the voxel edge in the voxel form, the cell edge in the FP64 form
        d_.L = (float)(F::voxel ? m_.Lv : m_.L);
        d_.Ld = F::voxel ? m_.Lv : m_.L;
        d_.invL = 1.0 / m_.L;
        d_.vpc = m_.vpc;
        d_.bin_invL = 1.0 / m_.L_min;
        d_.bin_vpc = m_.vpc_min;
        d_.gyro = m_.gyroscopic;
        d_.n_scenes = (int)m_.scenes.size();
        beta_ = m_.margin;
        {
            int sms = 0;
            DEM_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m_.device));
            n_sm_ = std::max(1, sms);
        }
        const int64_t Np = d_.Np;
        // owner arrays that the staged integration copies tile by tile hold whole tiles
        const int64_t Mp = (M + ITILE - 1) / ITILE * ITILE;
        Mp_ = Mp;

        dem_status s;
        // owner state, double-buffered
        for (int b = 0; b < 2; ++b) {
            if constexpr (F::voxel) {
                if ((s = alloc(d_.st.pos[b].rec, Mp, err))) return s;
            } else {
                if ((s = alloc(d_.st.pos[b].xm, M, err))) return s;
            }
            if ((s = alloc(d_.st.kv[b], 2 * Mp, err))) return s;
            if ((s = alloc(d_.st.quat[b], Mp, err))) return s;
            if ((s = alloc(d_.st.active[b], Mp, err))) return s;
        }
        if ((s = alloc(d_.inv_moi, Mp, err))) return s;
        if ((s = alloc(d_.inv_mass, Mp, err))) return s;
        if ((s = alloc(d_.owner_scene, Mp, err))) return s;
        if ((s = alloc(d_.owner_iso, Mp, err))) return s;
        if ((s = alloc(d_.touched, std::max(Mp, d_.Np), err))) return s;
        if (!m_.clumps)
            if ((s = alloc(d_.screen, std::max<int64_t>(d_.Np, 1), err))) return s;
        if ((s = alloc(d_.fo, M, err))) return s;
        if ((s = alloc(d_.to, M, err))) return s;
        if ((s = alloc(d_.owner_first, M, err))) return s;
        if ((s = alloc(d_.owner_nsph, M, err))) return s;
        d_.amag = nullptr;
        if ((s = alloc(d_.sph_owner, N, err))) return s;
        if ((s = alloc(d_.sph_rad, N, err))) return s;
        if ((s = alloc(d_.sph_rlo, N, err))) return s;
        if ((s = alloc(d_.sph_mat, N, err))) return s;
        if ((s = alloc(d_.sph_rloc, N, err))) return s;
        if ((s = alloc(d_.sph_pack, N, err))) return s;
        if ((s = alloc(d_.sph_head, N, err))) return s;
        if ((s = alloc(d_.sph_segend, N, err))) return s;
        Scene *scenes;
        Wall *walls;
        PairParam *pairs;
        PairParamF *pairs_f;
        uint16_t *ms, *ml;
        if ((s = alloc(scenes, m_.scenes.size(), err))) return s;
        if ((s = alloc(walls, std::max<size_t>(1, m_.walls.size()), err))) return s;
        if ((s = alloc(pairs, m_.pairs.size(), err))) return s;
        if ((s = alloc(pairs_f, m_.pairs.size(), err))) return s;
        if ((s = alloc(ms, m_.mat_scene.size(), err))) return s;
        if ((s = alloc(ml, m_.mat_local.size(), err))) return s;
        d_.scenes = scenes; d_.walls = walls; d_.pairs = pairs; d_.pairs_f = pairs_f;
        walls_dev_ = walls;
        d_.mat_scene = ms; d_.mat_local = ml;
        {
            double *crr;
            float *crr_f;
            if ((s = alloc(crr, m_.pairs.size(), err))) return s;
            if ((s = alloc(crr_f, m_.pairs.size(), err))) return s;
            std::vector<double> cd(m_.pairs.size(), 0.0);
            for (size_t k = 0; k < cd.size() && k < m_.pair_crr.size(); ++k) cd[k] = m_.pair_crr[k];
            std::vector<float> cf(cd.begin(), cd.end());
            if ((s = up(crr, cd.data(), (int64_t)cd.size(), err))) return s;
            if ((s = up(crr_f, cf.data(), (int64_t)cf.size(), err))) return s;
            d_.crr = crr;
            d_.crr_f = crr_f;
            double *nu;
            if ((s = alloc(nu, m_.pairs.size(), err))) return s;
            std::vector<double> nv(m_.pairs.size(), 0.0);
            for (size_t k = 0; k < nv.size() && k < m_.pair_nu.size(); ++k) nv[k] = m_.pair_nu[k];
            if ((s = up(nu, nv.data(), (int64_t)nv.size(), err))) return s;
            d_.pair_nu = nu;
            double *mp;
            float *mpf;
            if ((s = alloc(mp, MODEL_MAX_PARAMS, err))) return s;
            if ((s = alloc(mpf, MODEL_MAX_PARAMS, err))) return s;
            std::vector<double> pd(MODEL_MAX_PARAMS, 0.0);
            for (size_t k = 0; k < pd.size() && k < m_.model_params.size(); ++k) pd[k] = m_.model_params[k];
            std::vector<float> pf(pd.begin(), pd.end());
            if ((s = up(mp, pd.data(), MODEL_MAX_PARAMS, err))) return s;
            if ((s = up(mpf, pf.data(), MODEL_MAX_PARAMS, err))) return s;
            d_.model = m_.model;
            d_.model_par = mp;
            d_.model_par_f = mpf;
        }
        if ((s = alloc(st_, 1, err))) return s;
        if ((s = alloc(d_.audit, AUDIT_SLOTS * AUDIT_STRIDE, err))) return s;
        DEM_CU(cudaMallocHost((void **)&sth_, sizeof(DevStatus)));
        if ((s = alloc_lists(d_.K, err))) return s;

        // detection buffers
        db_.n = N;
        db_.n_cells_total = m_.n_cells_total;
        db_.key_bits = 1;
        while (db_.key_bits < 32 && ((uint64_t)1 << db_.key_bits) <= (uint64_t)m_.n_cells_total) ++db_.key_bits;
        const int64_t Nk = std::max<int64_t>(N, 1);
        if ((s = alloc(db_.keys, Nk, err))) return s;
        if ((s = alloc(db_.vals, Nk, err))) return s;
        if ((s = alloc(db_.keys_alt, Nk, err))) return s;
        if ((s = alloc(db_.vals_alt, Nk, err))) return s;
        db_.hist_cap = radix_hist_entries(Nk);
        if ((s = alloc(db_.hist, db_.hist_cap, err))) return s;
        if ((s = alloc(db_.cell_tab, (int64_t)m_.n_cells_total + 1, err))) return s;
        if (F::voxel) {
            int4 *a; float4 *b2; int4 *c; float4 *e;
            if ((s = alloc(a, Nk, err))) return s;
            if ((s = alloc(b2, Nk, err))) return s;
            if ((s = alloc(c, Nk, err))) return s;
            if ((s = alloc(e, Nk, err))) return s;
            db_.snap = a; db_.snap_aux = b2; db_.sorted = c; db_.sorted_aux = e;
        } else {
            double4_32a *a, *c;
            if ((s = alloc(a, Nk, err))) return s;
            if ((s = alloc(c, Nk, err))) return s;
            db_.snap = a; db_.sorted = c; db_.snap_aux = nullptr; db_.sorted_aux = nullptr;
        }
        if ((s = alloc(db_.sorted_owner, Nk, err))) return s;
        if ((s = alloc(db_.n_valid, 1, err))) return s;
        if ((s = alloc(db_.rowcnt, Np, err))) return s;
        if ((s = alloc(db_.crank, Nk, err))) return s;
        if ((s = alloc_cell_counts(m_.n_cells_total, err))) return s;
        choose_binning();
        if ((s = setup_facets(err))) return s;

        // constants
        std::vector<R4> inv_moi(M);
        std::vector<R> inv_mass(M);
        for (int64_t o = 0; o < M; ++o) {
            inv_moi[o] = R4{(R)(1.0 / m_.moi[3 * o]), (R)(1.0 / m_.moi[3 * o + 1]), (R)(1.0 / m_.moi[3 * o + 2]),
                            (R)m_.r_ext[o]};
            inv_mass[o] = (R)(1.0 / m_.mass[o]);
        }
        std::vector<R> rad(N);
        std::vector<float> rlo(N, 0.0f);
        std::vector<R4> rloc(N);
        for (int64_t k = 0; k < N; ++k) {
            rad[k] = (R)m_.sph_rad[k];
            if (F::voxel) rlo[k] = (float)(m_.sph_rad[k] - (double)rad[k]);
            rloc[k] = R4{(R)m_.sph_rloc[3 * k], (R)m_.sph_rloc[3 * k + 1], (R)m_.sph_rloc[3 * k + 2], R(0)};
        }
        if ((s = up(d_.inv_moi, inv_moi.data(), M, err))) return s;
        if ((s = up(d_.inv_mass, inv_mass.data(), M, err))) return s;
        // voxel form, single spheres: if every owner is isotropic with I = c m R^2 for one
        // c, the kernels derive 1/m and 1/I from the position record (20 bytes less per
        // owner and step)
        d_.solid = 0;
        if (F::voxel && !m_.clumps && M > 0) {
            bool ok = true;
            double c0 = 0.0;
            for (int64_t o = 0; o < M && ok; ++o) {
                const double r = m_.sph_rad[m_.owner_first_slot[o]], mass = m_.mass[o];
                const double *I = &m_.moi[3 * o];
                const double c = I[0] / (mass * r * r);
                if (o == 0) c0 = c;
                ok = I[1] == I[0] && I[2] == I[0] && m_.r_ext[o] == 0.0 && std::isfinite(c) && c > 0.0 &&
                     std::fabs(c - c0) <= 1e-12 * c0;
            }
            if (ok) {
                d_.solid = 1;
                d_.moi_coef = (float)c0;
            }
        }
        if ((s = up(d_.owner_scene, m_.owner_scene.data(), M, err))) return s;
        if ((s = up(d_.owner_iso, m_.owner_iso.data(), M, err))) return s;
        if ((s = up(d_.owner_first, m_.owner_first_slot.data(), M, err))) return s;
        {
            std::vector<uint8_t> ns(M);
            for (int64_t o = 0; o < M; ++o) ns[o] = (uint8_t)m_.owner_nsph[o];
            if ((s = up(d_.owner_nsph, ns.data(), M, err))) return s;
        }
        if ((s = up(d_.sph_owner, m_.sph_owner.data(), N, err))) return s;
        if ((s = up(d_.sph_rad, rad.data(), N, err))) return s;
        if ((s = up(d_.sph_rlo, rlo.data(), N, err))) return s;
        if ((s = up(d_.sph_mat, m_.sph_mat.data(), N, err))) return s;
        if ((s = up(d_.sph_rloc, rloc.data(), N, err))) return s;
        {
            using P = typename SphPack<R>::T;
            std::vector<P> pk(N);
            for (int64_t k = 0; k < N; ++k) {
                if constexpr (F::voxel) {
                    int mi = (int)m_.sph_mat[k];
                    float mf;
                    std::memcpy(&mf, &mi, sizeof(mf));
                    pk[k] = make_float4((float)rad[k], rlo[k], mf, 0.0f);
                } else {
                    pk[k] = make_double2((double)rad[k], (double)m_.sph_mat[k]);
                }
            }
            if ((s = up(d_.sph_pack, pk.data(), N, err))) return s;
        }
        if ((s = up(d_.sph_head, m_.sph_head.data(), N, err))) return s;
        if ((s = up(d_.sph_segend, m_.sph_segend.data(), N, err))) return s;
        if ((s = up(scenes, m_.scenes.data(), m_.scenes.size(), err))) return s;
        if (!m_.walls.empty() && (s = up(walls, m_.walls.data(), m_.walls.size(), err))) return s;
        if ((s = up(pairs, m_.pairs.data(), m_.pairs.size(), err))) return s;
        {
            std::vector<PairParamF> pf(m_.pairs.size());
            for (size_t k = 0; k < pf.size(); ++k)
                pf[k] = PairParamF{(float)m_.pairs[k].Estar, (float)m_.pairs[k].Gstar, (float)m_.pairs[k].beta,
                                   (float)m_.pairs[k].mu};
            if ((s = up(pairs_f, pf.data(), pf.size(), err))) return s;
        }
        if ((s = up(ms, m_.mat_scene.data(), m_.mat_scene.size(), err))) return s;
        if ((s = up(ml, m_.mat_local.data(), m_.mat_local.size(), err))) return s;

        if (m_.families_used) {
            if ((s = alloc_families(err))) return s;
        }

        // mass into the position store of buffer 0, then the state through the upload kernel;
        // in the voxel form a single sphere's radius (float-float) rides in both buffers'
        // records from here on
        if constexpr (F::voxel) {
            using PR = typename F::PosRec;
            std::vector<PR> rec(M);
            for (int64_t o = 0; o < M; ++o) {
                uint32_t rb = 0, lb = 0;
                if (!m_.clumps) {
                    const float r = (float)rad[o], l = rlo[o];
                    std::memcpy(&rb, &r, 4);
                    std::memcpy(&lb, &l, 4);
                }
                rec[o].om = make_float4(0.f, 0.f, 0.f, (float)m_.mass[o]);
                rec[o].vr = make_uint4(0u, 0u, rb, lb);
            }
            if ((s = up(d_.st.pos[0].rec, rec.data(), M, err))) return s;
            if ((s = up(d_.st.pos[1].rec, rec.data(), M, err))) return s;
        } else {
            std::vector<double4_32a> xm(M);
            for (int64_t o = 0; o < M; ++o) xm[o] = make_double4_32a(0.0, 0.0, 0.0, m_.mass[o]);
            if ((s = up(d_.st.pos[0].xm, xm.data(), M, err))) return s;
        }
        DevStatus h{};
        h.disp_slack = F::voxel ? 4.0 * std::ldexp(1.0, std::ilogb(m_.Lv) - 23) : 0.0;
        // a turning mesh moves the facets between a list's snapshot and its use: its
        // largest surface displacement per step counts against the margin like the
        // owners' own
        h.disp_slack += mesh_slack_;
        h.disp_slack_f = (float)h.disp_slack;
        if ((double)h.disp_slack_f < h.disp_slack) h.disp_slack_f = std::nextafter(h.disp_slack_f, INFINITY);
        h.beta_cur = h.beta_next = beta_;
        for (int64_t o = 0; o < M; ++o) {   // initial speed bound for the first cycle length
            double v2 = m_.v[3 * o] * m_.v[3 * o] + m_.v[3 * o + 1] * m_.v[3 * o + 1] + m_.v[3 * o + 2] * m_.v[3 * o + 2];
            double w2 = m_.wb[3 * o] * m_.wb[3 * o] + m_.wb[3 * o + 1] * m_.wb[3 * o + 1] + m_.wb[3 * o + 2] * m_.wb[3 * o + 2];
            h.vmax_last = std::max(h.vmax_last, std::sqrt(v2) + std::sqrt(w2) * m_.r_ext[o]);
        }
        if ((s = up(st_, &h, 1, err))) return s;
        d_.status = st_;
        {
            std::vector<uint8_t> act(M, 1);
            if ((s = upload_state(0, M, m_.x.data(), m_.q.data(), m_.v.data(), m_.wb.data(), act.data(), err)))
                return s;
        }
        pose_facets(sf_);
        flag_wall_cells(sf_);
        if (N > 0) {
            rebuild_inline(sf_);
            if ((s = settle(err))) return s;
        }
        return DEM_OK;
    }

    // Which cells a wall may reach (walls keep their shape: computed per cell layout).
    void flag_wall_cells(cudaStream_t st)
    {
        if (m_.n_cells_total == 0) return;
        k_cell_walls<F><<<grid((int64_t)m_.n_cells_total, 256), 256, 0, st>>>(d_, db_, m_.L,
                                                                             m_.r_max + m_.margin_max);
    }

    // Mesh facets: their wall indices, a share of (cell, facet) pair slots each (enough
    // for any pose: the facet's extent at most twice its largest vertex distance from its
    // centroid, grown by the reach on both sides, in cells of the smallest edge), the
    // snapshot vertices and the sort buffers; the largest surface displacement per step.
    dem_status setup_facets(std::string &err)
    {
        std::vector<int> fw;
        for (size_t k = 0; k < m_.walls.size(); ++k)
            if (m_.walls[k].type == WALL_TRIANGLE) fw.push_back((int)k);
        db_.n_facets = (int)fw.size();
        mesh_slack_ = 0.0;
        if (fw.empty()) return DEM_OK;
        // A facet is binned into the cells whose centre lies within rr = r_max + margin +
        // half a cell diagonal of it (k_facet_bin; its FP32 allowance is below 1e-5 of
        // the facet's extent).  Those cells lie inside the facet's neighbourhood of radius
        // r2 = rr + half a diagonal, whose volume (Steiner's formula for a flat convex
        // piece of area A and perimeter P: 2 A r + (pi / 2) P r^2 + (4 / 3) pi r^3) over
        // the cell volume bounds their number.  The bound falls as cells grow, so the
        // smallest cell gives each facet's share, at any pose and cell size.
        const double cell = m_.L_min;
        std::vector<int64_t> off(fw.size() + 1, 0);
        for (size_t f = 0; f < fw.size(); ++f) {
            const Wall &w = m_.walls[fw[f]];
            double rp = 0.0, e[3];
            for (int v = 0; v < 3; ++v) {
                double dp = 0.0, de = 0.0;
                const int v2 = (v + 1) % 3;
                for (int a = 0; a < 3; ++a) {
                    dp += (w.tri[3 * v + a] - w.p[a]) * (w.tri[3 * v + a] - w.p[a]);
                    de += (w.tri[3 * v2 + a] - w.tri[3 * v + a]) * (w.tri[3 * v2 + a] - w.tri[3 * v + a]);
                }
                rp = std::max(rp, std::sqrt(dp));
                e[v] = std::sqrt(de);
            }
            const double perim = e[0] + e[1] + e[2];
            double cr[3];
            const double u[3] = {w.tri[3] - w.tri[0], w.tri[4] - w.tri[1], w.tri[5] - w.tri[2]};
            const double q[3] = {w.tri[6] - w.tri[0], w.tri[7] - w.tri[1], w.tri[8] - w.tri[2]};
            cr[0] = u[1] * q[2] - u[2] * q[1];
            cr[1] = u[2] * q[0] - u[0] * q[2];
            cr[2] = u[0] * q[1] - u[1] * q[0];
            const double area = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            const double ext = std::max(std::max(e[0], e[1]), e[2]) * 2.0 + 8.0 * cell;
            const double r2 = m_.r_max + m_.margin_max + std::sqrt(3.0) * cell + 2e-5 * ext + 1e-9;
            const double vol = 2.0 * area * r2 + 0.5 * M_PI * perim * r2 * r2 + 4.0 / 3.0 * M_PI * r2 * r2 * r2;
            const int64_t per = (int64_t)std::ceil(1.02 * vol / (cell * cell * cell)) + 8;
            off[f + 1] = off[f] + per;
            const double wn = std::sqrt(w.omega[0] * w.omega[0] + w.omega[1] * w.omega[1] + w.omega[2] * w.omega[2]);
            mesh_slack_ = std::max(mesh_slack_, 1.000001 * wn * rp * m_.scenes[w.scene].h);
        }
        const int64_t P = off.back();
        dem_status s;
        int *fwd;
        int64_t *offd;
        if ((s = alloc(fwd, (int64_t)fw.size(), err))) return s;
        if ((s = alloc(offd, (int64_t)off.size(), err))) return s;
        if ((s = up(fwd, fw.data(), (int64_t)fw.size(), err))) return s;
        if ((s = up(offd, off.data(), (int64_t)off.size(), err))) return s;
        db_.facet_wall = fwd;
        db_.facet_off = offd;
        if ((s = alloc(db_.tri_snap, 9 * (int64_t)fw.size(), err))) return s;
        if ((s = alloc(db_.fkeys, P, err))) return s;
        if ((s = alloc(db_.fvals, P, err))) return s;
        if ((s = alloc(db_.fkeys_alt, P, err))) return s;
        if ((s = alloc(db_.fvals_alt, P, err))) return s;
        db_.fhist_cap = radix_hist_entries(P);
        if ((s = alloc(db_.fhist, db_.fhist_cap, err))) return s;
        db_.n_fpairs = P;
        db_.fkeys_sorted = db_.fkeys;
        db_.fvals_sorted = db_.fvals;
        return DEM_OK;
    }

    // Current pose of the mesh facets (the state's step).
    void pose_facets(cudaStream_t st)
    {
        if (db_.n_facets > 0)
            k_facet_pose<F><<<grid(db_.n_facets, 128), 128, 0, st>>>(d_, walls_dev_, db_.facet_wall, db_.n_facets);
    }

    dem_status step(int64_t n, std::string &err) override
    {
        if (n < 0) { err = "negative step count"; return DEM_ERR_ARG; }
        dem_status s;
        if ((s = pull(err))) return s;
        const long long target = sth_->steps_done + n;
        if (dirty_) {
            rebuild_inline(sf_);
            if ((s = settle(err))) return s;
            dirty_ = false;
        }
        DEM_CU(cudaEventRecord(ev_a_, sf_));
        while (true) {
            if ((s = pull(err))) return s;
            long long left = target - sth_->steps_done;
            if (left <= 0) break;
            if (sth_->list_stale) {          // audit fallback: rebuild from the current state
                fallbacks_ += 1;
                cycle_scale_ = std::max(0.05, cycle_scale_ * 0.6);
                learned_left_ = 0;           // a fresh prediction from the current state
                rebuild_inline(sf_);
                if ((s = settle(err))) return s;
                continue;
            }
            const bool use_graphs = graphs_on_ && !prof_ && !collect_ && d_.N > 0;
            if (m_.schedule == DEM_SCHEDULE_EVERY_STEP || d_.N == 0) {
                long long chunk = std::min<long long>(left, 256);
                cudaGraphExec_t gx = use_graphs ? graph_for(0) : nullptr;
                for (long long k = 0; k < chunk; ++k) {
                    if (gx) {
                        DEM_CU(cudaGraphLaunch(gx, sf_));
                        continue;
                    }
                    if (d_.N > 0) rebuild_inline(sf_);
                    force_step();
                }
            } else {
                const long long cl = cycle_length();
                if (left < cl) {
                    // fewer steps than a cycle (a caller stepping a little at a time): step
                    // on with the list in use, no detection; the audit after each step flags
                    // it stale once its margin is used up, the steps launched after that do
                    // nothing, and the next pass rebuilds
                    for (long long k = 0; k < left; ++k) force_step();
                } else {
                    long long c = quantize_cycle(std::min<long long>(left, cl));
                    cudaGraphExec_t gx = use_graphs ? graph_for(c) : nullptr;
                    if (gx) {
                        DEM_CU(cudaGraphLaunch(gx, sf_));
                    } else {
                        enqueue_cycle(c);
                    }
                }
            }
            if ((s = settle(err))) return s;
            if ((s = collect_roll(err))) return s;
        }
        DEM_CU(cudaEventRecord(ev_b_, sf_));
        DEM_CU(cudaEventSynchronize(ev_b_));
        float ms = 0;
        cudaEventElapsedTime(&ms, ev_a_, ev_b_);
        ms_total_ += ms;
        return DEM_OK;
    }

    dem_status sync(std::string &err) override
    {
        DEM_CU(cudaStreamSynchronize(sf_));
        DEM_CU(cudaStreamSynchronize(sd_));
        return DEM_OK;
    }

    void *stream() override { return (void *)sf_; }

    dem_status owner_state(int64_t first, int64_t n, double *x, double *q, double *v, double *w,
                           std::string &err) override
    {
        if (n <= 0) return DEM_OK;
        // pinned (mapped) caller buffers are written by the kernel itself across the host
        // link; any other buffer goes through device scratch and a copy
        double *out[4] = {x, q, v, w};
        bool direct = true;
        for (double *&p : out) {
            if (!p) continue;
            cudaPointerAttributes a{};
            if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
                (void)cudaGetLastError();
                direct = false;
            } else if (a.type == cudaMemoryTypeHost && a.devicePointer) {
                p = static_cast<double *>(a.devicePointer);
            } else {
                direct = false;
            }
        }
        if (direct) {
            k_owner_download<F><<<grid(n, DOWNLOAD_BLOCK), DOWNLOAD_BLOCK, 0, sf_>>>(d_, first, n, out[0], out[1],
                                                                                    out[2], out[3]);
            DEM_CU(cudaGetLastError());
            DEM_CU(cudaStreamSynchronize(sf_));
            return DEM_OK;
        }
        double *buf;
        dem_status s;
        if ((s = scratch(buf, 13 * n, err))) return s;
        k_owner_download<F><<<grid(n, DOWNLOAD_BLOCK), DOWNLOAD_BLOCK, 0, sf_>>>(
            d_, first, n, x ? buf : nullptr, q ? buf + 3 * n : nullptr, v ? buf + 7 * n : nullptr,
            w ? buf + 10 * n : nullptr);
        DEM_CU(cudaGetLastError());
        if (x) DEM_CU(cudaMemcpyAsync(x, buf, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, sf_));
        if (q) DEM_CU(cudaMemcpyAsync(q, buf + 3 * n, 4 * n * sizeof(double), cudaMemcpyDeviceToHost, sf_));
        if (v) DEM_CU(cudaMemcpyAsync(v, buf + 7 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, sf_));
        if (w) DEM_CU(cudaMemcpyAsync(w, buf + 10 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        return DEM_OK;
    }

    dem_status set_owner_state(int64_t first, int64_t n, const double *x, const double *q, const double *v,
                               const double *w, std::string &err) override
    {
        dem_status s;
        // single spheres, delayed schedules: the list in use stays where no owner moved past
        // its margin (the audit's rule), with the upload's displacements in the bounds; a
        // clump's orientation moves its spheres, so that rebuilds
        const bool keep = !m_.clumps && m_.schedule != DEM_SCHEDULE_EVERY_STEP && !dirty_ && !sth_->list_stale;
        double bound = 0.0;
        if ((s = upload_state(first, n, x, q, v, w, nullptr, err, keep, &bound))) return s;
        if (keep) {
            if (x && std::max(bound, sth_->disp_cur) > sth_->beta_cur) dirty_ = true;
            // the next upload before a step compares against this one's bounds too
            sth_->disp_cur = std::max(sth_->disp_cur, bound);
        } else if (x || q) {
            dirty_ = true;
        }
        return DEM_OK;
    }

    dem_status sphere_positions(int64_t first, int64_t n, double *xyz, double *r, int32_t *cell, float *off,
                                std::string &err) override
    {
        if (n <= 0) return DEM_OK;
        dem_status s;
        int64_t *slots;
        double *buf;
        int *cb;
        float *ob;
        if ((s = scratch(buf, 4 * n + 3 * n + 2 * n, err))) return s;   // xyz, r, cell (as int), off
        slots = reinterpret_cast<int64_t *>(buf + 4 * n);
        cb = reinterpret_cast<int *>(buf + 5 * n);
        ob = reinterpret_cast<float *>(buf + 7 * n);
        DEM_CU(cudaMemcpyAsync(slots, m_.slot_of_sphere.data() + first, n * sizeof(int64_t), cudaMemcpyHostToDevice, sf_));
        if (m_.clumps)
            k_sphere_download<F, true><<<grid(n, 256), 256, 0, sf_>>>(d_, slots, n, buf, buf + 3 * n, cb, ob);
        else
            k_sphere_download<F, false><<<grid(n, 256), 256, 0, sf_>>>(d_, slots, n, buf, buf + 3 * n, cb, ob);
        DEM_CU(cudaGetLastError());
        std::vector<double> h(4 * n);
        DEM_CU(cudaMemcpyAsync(h.data(), buf, 4 * n * sizeof(double), cudaMemcpyDeviceToHost, sf_));
        std::vector<int> hc(3 * n);
        std::vector<float> ho(3 * n);
        if (F::voxel) {
            DEM_CU(cudaMemcpyAsync(hc.data(), cb, 3 * n * sizeof(int), cudaMemcpyDeviceToHost, sf_));
            DEM_CU(cudaMemcpyAsync(ho.data(), ob, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, sf_));
        }
        DEM_CU(cudaStreamSynchronize(sf_));
        if (xyz) std::memcpy(xyz, h.data(), 3 * n * sizeof(double));
        if (r) std::memcpy(r, h.data() + 3 * n, n * sizeof(double));
        if (cell) {
            if (!F::voxel) { err = "voxel encoding exists only in the VOXEL_FP32 form"; return DEM_ERR_STATE; }
            std::memcpy(cell, hc.data(), 3 * n * sizeof(int));
            if (off) std::memcpy(off, ho.data(), 3 * n * sizeof(float));
        }
        return DEM_OK;
    }

    dem_status contacts(std::vector<ContactOut> &out, std::string &err) override
    {
        out.clear();
        dem_status s;
        if ((s = fresh(err))) return s;
        const int64_t N = d_.N, K = d_.K, Np = d_.Np;
        if (N == 0) return DEM_OK;
        double *buf;
        const int64_t ne = K * Np;
        if (m_.model != FORCE_MODEL_BUILTIN) return contacts_model(out, err);
        if ((s = scratch(buf, 14 * ne, err))) return s;
        if (m_.clumps)
            k_contacts<F, true><<<grid(N, 128), 128, 0, sf_>>>(d_, buf, buf + ne, buf + 4 * ne, buf + 7 * ne,
                                                               buf + 10 * ne, buf + 11 * ne);
        else
            k_contacts<F, false><<<grid(N, 128), 128, 0, sf_>>>(d_, buf, buf + ne, buf + 4 * ne, buf + 7 * ne,
                                                                buf + 10 * ne, buf + 11 * ne);
        DEM_CU(cudaGetLastError());
        std::vector<double> h(14 * ne);
        DEM_CU(cudaMemcpyAsync(h.data(), buf, 14 * ne * sizeof(double), cudaMemcpyDeviceToHost, sf_));
        std::vector<uint32_t> partner;
        std::vector<uint8_t> cnt;
        if ((s = fetch_list(sth_->list_cur, partner, cnt, err))) return s;
        for (int64_t sl = 0; sl < N; ++sl) {
            int64_t ui = m_.sphere_of_slot[sl];
            if (ui < 0) continue;
            for (int k = 0; k < cnt[sl]; ++k) {
                int64_t e = (int64_t)k * Np + sl;
                uint32_t j = partner[e];
                if (!(j & WALL_BIT) && j < (uint32_t)sl) continue;
                if (!(h[e] > 0.0)) continue;
                ContactOut c;
                c.i = ui;
                c.j = (j & WALL_BIT) ? -1 - wall_local(j & ~WALL_BIT) : m_.sphere_of_slot[j];
                for (int a = 0; a < 3; ++a) {
                    c.force[a] = h[ne + 3 * e + a];
                    c.point[a] = h[4 * ne + 3 * e + a];
                    c.hist[a] = h[7 * ne + 3 * e + a];
                    c.trf[a] = h[11 * ne + 3 * e + a];
                }
                c.overlap = h[e];
                c.age = h[10 * ne + e];
                out.push_back(c);
            }
        }
        return DEM_OK;
    }

    // Read-back through the world's contact model: every pair it engages (a bond across a
    // gap included) with its force, point, wildcards and torque-only force.
    dem_status contacts_model(std::vector<ContactOut> &out, std::string &err)
    {
        dem_status s;
        const int64_t N = d_.N, Np = d_.Np, ne = (int64_t)d_.K * Np;
        double *buf;
        if ((s = scratch(buf, 19 * ne, err))) return s;
        double *ov = buf, *fo = buf + ne, *pt = buf + 4 * ne, *wc = buf + 7 * ne, *rf = buf + 15 * ne,
               *en = buf + 18 * ne;
        if (m_.model == FORCE_MODEL_BONDED_BREAKAGE) {
            if (m_.clumps) k_contacts_model<F, true, ModelBondedBreakage><<<grid(N, 128), 128, 0, sf_>>>(d_, ov, fo, pt, wc, rf, en);
            else k_contacts_model<F, false, ModelBondedBreakage><<<grid(N, 128), 128, 0, sf_>>>(d_, ov, fo, pt, wc, rf, en);
        } else {
            if (m_.clumps) k_contacts_model<F, true, ModelHertzMindlin><<<grid(N, 128), 128, 0, sf_>>>(d_, ov, fo, pt, wc, rf, en);
            else k_contacts_model<F, false, ModelHertzMindlin><<<grid(N, 128), 128, 0, sf_>>>(d_, ov, fo, pt, wc, rf, en);
        }
        DEM_CU(cudaGetLastError());
        std::vector<double> h(19 * ne);
        DEM_CU(cudaMemcpyAsync(h.data(), buf, 19 * ne * sizeof(double), cudaMemcpyDeviceToHost, sf_));
        std::vector<uint32_t> partner;
        std::vector<uint8_t> cnt;
        if ((s = fetch_list(sth_->list_cur, partner, cnt, err))) return s;
        for (int64_t sl = 0; sl < N; ++sl) {
            int64_t ui = m_.sphere_of_slot[sl];
            if (ui < 0) continue;
            for (int k = 0; k < cnt[sl]; ++k) {
                int64_t e = (int64_t)k * Np + sl;
                uint32_t j = partner[e];
                if (!(j & WALL_BIT) && j < (uint32_t)sl) continue;
                if (!(h[18 * ne + e] > 0.0)) continue;
                ContactOut c;
                c.i = ui;
                c.j = (j & WALL_BIT) ? -1 - wall_local(j & ~WALL_BIT) : m_.sphere_of_slot[j];
                for (int a = 0; a < 3; ++a) {
                    c.force[a] = h[ne + 3 * e + a];
                    c.point[a] = h[4 * ne + 3 * e + a];
                    c.hist[a] = h[7 * ne + 8 * e + a];
                    c.trf[a] = h[15 * ne + 3 * e + a];
                }
                for (int q = 0; q < 8; ++q) c.wc[q] = h[7 * ne + 8 * e + q];
                c.age = h[7 * ne + 8 * e + 3];
                c.overlap = h[e];
                out.push_back(c);
            }
        }
        return DEM_OK;
    }

    // Wildcards 4..7 of the contact model for listed pairs (i, j), wc[4k] (host values in
    // the lower sphere's orientation; the upper side's copy takes the odd ones negated).
    dem_status set_wildcards(int64_t nk, const int64_t *ii, const int64_t *jj, const double *wcv,
                             std::string &err) override
    {
        dem_status s;
        if ((s = pull(err))) return s;
        if (!d_.lists.wild[0]) {
            err = "the world's contact model has no wildcards beyond the history";
            return DEM_ERR_STATE;
        }
        std::vector<uint32_t> partner;
        std::vector<uint8_t> cnt;
        if ((s = fetch_list(sth_->list_cur, partner, cnt, err))) return s;
        const int64_t ne = (int64_t)d_.K * d_.Np;
        using H = typename HistVec<R>::T;
        const int hp = sth_->hist_par;
        std::vector<H> wv(ne);
        DEM_CU(cudaMemcpyAsync(wv.data(), d_.lists.wild[hp], ne * sizeof(H), cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        const unsigned odd = model_odd();
        for (int64_t q = 0; q < nk; ++q) {
            if (ii[q] < 0 || ii[q] >= (int64_t)m_.slot_of_sphere.size() || jj[q] < 0 ||
                jj[q] >= (int64_t)m_.slot_of_sphere.size())
                continue;
            const int64_t si = m_.slot_of_sphere[ii[q]], sj = m_.slot_of_sphere[jj[q]];
            for (int side = 0; side < 2; ++side) {
                const int64_t me = side ? sj : si, other = side ? si : sj;
                const bool upper = me > other;
                for (int k = 0; k < cnt[me]; ++k) {
                    const int64_t e = (int64_t)k * d_.Np + me;
                    if (partner[e] != (uint32_t)other) continue;
                    R v[4];
                    for (int a = 0; a < 4; ++a) v[a] = (R)((upper && ((odd >> (4 + a)) & 1u)) ? -wcv[4 * q + a] : wcv[4 * q + a]);
                    wv[e].x = v[0]; wv[e].y = v[1]; wv[e].z = v[2]; wv[e].w = v[3];
                }
            }
        }
        DEM_CU(cudaMemcpyAsync(d_.lists.wild[hp], wv.data(), ne * sizeof(H), cudaMemcpyHostToDevice, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        return DEM_OK;
    }

    dem_status listed(std::vector<int64_t> &pi, std::vector<int64_t> &pj, std::vector<int64_t> &si,
                      std::vector<int64_t> &wi, std::string &err) override
    {
        dem_status s;
        if ((s = pull(err))) return s;
        std::vector<uint32_t> partner;
        std::vector<uint8_t> cnt;
        if ((s = fetch_list(sth_->list_cur, partner, cnt, err))) return s;
        pi.clear(); pj.clear(); si.clear(); wi.clear();
        for (int64_t sl = 0; sl < d_.N; ++sl) {
            int64_t ui = m_.sphere_of_slot[sl];
            if (ui < 0) continue;
            for (int k = 0; k < cnt[sl]; ++k) {
                uint32_t j = partner[(int64_t)k * d_.Np + sl];
                if (j & WALL_BIT) {
                    si.push_back(ui);
                    wi.push_back(wall_local(j & ~WALL_BIT));
                } else if (j > (uint32_t)sl) {
                    pi.push_back(ui);
                    pj.push_back(m_.sphere_of_slot[j]);
                }
            }
        }
        return DEM_OK;
    }

    dem_status owner_forces(std::vector<double> &Fo, std::vector<double> &To, std::string &err) override
    {
        const int64_t M = d_.M;
        Fo.assign(3 * M, 0.0);
        To.assign(3 * M, 0.0);
        if (M == 0) return DEM_OK;
        double *buf;
        dem_status s;
        if ((s = fresh(err))) return s;
        if ((s = scratch(buf, 6 * M, err))) return s;
        launch_force<MODE_EVAL>(buf, buf + 3 * M);
        DEM_CU(cudaGetLastError());
        DEM_CU(cudaMemcpyAsync(Fo.data(), buf, 3 * M * sizeof(double), cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaMemcpyAsync(To.data(), buf + 3 * M, 3 * M * sizeof(double), cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        return DEM_OK;
    }

    dem_status set_history(int64_t nk, const int64_t *ii, const int64_t *jj, const double *ut, const double *age,
                           std::string &err) override
    {
        dem_status s;
        if ((s = pull(err))) return s;
        std::vector<uint32_t> partner;
        std::vector<uint8_t> cnt;
        if ((s = fetch_list(sth_->list_cur, partner, cnt, err))) return s;
        const int64_t ne = (int64_t)d_.K * d_.Np;
        using H = typename HistVec<R>::T;
        std::vector<H> hv(ne);
        for (auto &v : hv) { v.x = R(0); v.y = R(0); v.z = R(0); v.w = R(0); }
        for (int64_t q = 0; q < nk; ++q) {
            if (ii[q] < 0 || ii[q] >= (int64_t)m_.slot_of_sphere.size()) continue;
            int64_t sl = m_.slot_of_sphere[ii[q]];
            // the age lane: seconds (FP64 form) or whole steps (voxel form)
            R lane = R(0);
            if (age) {
                const double hs = m_.scenes[m_.owner_scene[m_.sph_owner[sl]]].h;
                lane = F::voxel ? (R)std::nearbyint(age[q] / hs) : (R)age[q];
            }
            uint32_t key;
            if (jj[q] >= 0) {
                if (jj[q] >= (int64_t)m_.slot_of_sphere.size()) continue;
                int64_t sj = m_.slot_of_sphere[jj[q]];
                if (sj < sl) continue;
                key = (uint32_t)sj;
                // the partner's copy, in its own orientation
                for (int k = 0; k < cnt[sj]; ++k) {
                    int64_t e = (int64_t)k * d_.Np + sj;
                    if (partner[e] == (uint32_t)sl) {
                        hv[e].x = -(R)ut[3 * q]; hv[e].y = -(R)ut[3 * q + 1]; hv[e].z = -(R)ut[3 * q + 2];
                        hv[e].w = lane;
                    }
                }
            } else {
                int scene = m_.owner_scene[m_.sph_owner[sl]];
                key = WALL_BIT | (uint32_t)(m_.scene_wall_base[scene] + (-1 - jj[q]));
            }
            for (int k = 0; k < cnt[sl]; ++k) {
                int64_t e = (int64_t)k * d_.Np + sl;
                if (partner[e] == key) {
                    hv[e].x = (R)ut[3 * q]; hv[e].y = (R)ut[3 * q + 1]; hv[e].z = (R)ut[3 * q + 2];
                    hv[e].w = lane;
                }
            }
        }
        const int hp = sth_->hist_par;
        DEM_CU(cudaMemcpyAsync(d_.lists.hist[hp], hv.data(), ne * sizeof(H), cudaMemcpyHostToDevice, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        return DEM_OK;
    }

    // ---- family tags (Sec. 2.2.2)

    // Device family arrays, made when families are first used; from then on the kernels
    // look the family up for every owner (and the narrow phase for every candidate).
    dem_status alloc_families(std::string &err)
    {
        dem_status s;
        if (!d_.owner_family) {
            uint8_t *of, *sf;
            FamilyMotion *fm;
            uint32_t *mk;
            if ((s = alloc(of, Mp_, err))) return s;
            if ((s = alloc(fm, N_FAMILY, err))) return s;
            if ((s = alloc(mk, FAMILY_MASK_WORDS, err))) return s;
            if ((s = alloc(sf, std::max<int64_t>(d_.N, 1), err))) return s;
            if (m_.owner_family.size() != (size_t)d_.M) m_.owner_family.assign((size_t)d_.M, 0);
            if (m_.fam_motion.size() != (size_t)N_FAMILY || m_.fam_mask.size() != (size_t)FAMILY_MASK_WORDS)
                family_defaults(m_.fam_motion, m_.fam_mask);
            if ((s = up(of, m_.owner_family.data(), d_.M, err))) return s;
            d_.owner_family = of;
            d_.fam_motion = fm;
            d_.fam_mask = mk;
            db_.sorted_family = sf;
            m_.families_used = true;
            drop_graphs();                // captured launches hold the old parameters
        }
        if ((s = up(const_cast<FamilyMotion *>(d_.fam_motion), m_.fam_motion.data(), N_FAMILY, err))) return s;
        if ((s = up(const_cast<uint32_t *>(d_.fam_mask), m_.fam_mask.data(), FAMILY_MASK_WORDS, err))) return s;
        return DEM_OK;
    }

    dem_status set_family(int64_t first, int64_t n, const uint8_t *fam, std::string &err) override
    {
        dem_status s;
        if ((s = pull(err))) return s;
        if ((s = alloc_families(err))) return s;
        std::copy(fam, fam + n, m_.owner_family.begin() + first);
        if ((s = up(const_cast<uint8_t *>(d_.owner_family) + first, fam, n, err))) return s;
        dirty_ = true;                    // masked contacts may change: rebuild before the next step
        return DEM_OK;
    }

    dem_status set_family_motion(int f, const double *v, const double *w, std::string &err) override
    {
        dem_status s;
        if ((s = pull(err))) return s;
        if ((s = alloc_families(err))) return s;
        family_set_motion(m_.fam_motion[f], v, w);
        return alloc_families(err);
    }

    dem_status set_family_contacts(int fa, int fb, int on, std::string &err) override
    {
        dem_status s;
        if ((s = pull(err))) return s;
        if ((s = alloc_families(err))) return s;
        family_set_contacts(m_.fam_mask, fa, fb, on);
        if ((s = alloc_families(err))) return s;
        dirty_ = true;
        return DEM_OK;
    }

    dem_status set_active_box(int64_t first, int64_t n, const double lo[3], const double hi[3], int fin, int fout,
                              std::string &err) override
    {
        dem_status s;
        if ((s = pull(err))) return s;
        if ((s = alloc_families(err))) return s;
        if (n > 0) {
            uint8_t *fam = const_cast<uint8_t *>(d_.owner_family);
            k_active_box<F><<<grid(n, 256), 256, 0, sf_>>>(d_, first, n, make_double3(lo[0], lo[1], lo[2]),
                                                           make_double3(hi[0], hi[1], hi[2]), fin, fout, fam);
            DEM_CU(cudaGetLastError());
            DEM_CU(cudaMemcpyAsync(m_.owner_family.data() + first, fam + first, n, cudaMemcpyDeviceToHost, sf_));
            DEM_CU(cudaStreamSynchronize(sf_));
        }
        dirty_ = true;
        return DEM_OK;
    }

    dem_status stats(dem_stats *o, std::string &err) override
    {
        dem_status s;
        if ((s = fresh(err))) return s;
        std::memset(o, 0, sizeof(*o));
        o->steps = sth_->steps_done;
        o->rebuilds = sth_->rebuilds;
        o->audit_fallbacks = fallbacks_;
        o->overflow_regrows = regrows_;
        o->list_capacity = d_.K;
        o->list_max_row = sth_->max_row;
        o->margin = sth_->beta_cur;
        o->displacement_bound = sth_->disp_cur;
        o->max_speed = sth_->vmax_last;
        o->mean_steps_per_build = sth_->rebuilds > 0 ? (double)sth_->steps_done / (double)sth_->rebuilds : 0.0;
        o->cell_size = m_.L;
        o->n_cells = m_.n_cells_total;
        o->derived_constants = d_.solid;
        o->counting_sort = db_.counting;
        o->ms_force = prof_ms_[P_FORCE];
        o->ms_detect = prof_ms_[P_DETECT];
        o->ms_hash = prof_ms_[P_HASH];
        o->ms_link = prof_ms_[P_LINK];
        o->n_force = prof_n_[P_FORCE];
        o->n_detect = prof_n_[P_DETECT];
        o->ms_integrate = prof_ms_[P_INTEG];
        o->n_integrate = prof_n_[P_INTEG];
        o->ms_contact_eval = prof_ms_[P_EVAL];
        o->n_contact_eval = prof_n_[P_EVAL];
        o->ms_total = ms_total_;
        o->last_cycle = last_cycle_;
        o->schedule_samples = (int64_t)(ds_y_.size() / MLP_OUT);
        o->pair_steps = (int64_t)sth_->pair_steps;
        o->busy_steps = (int64_t)sth_->busy_steps;
        if (d_.N > 0) {
            double *buf;
            if ((s = scratch(buf, 4, err))) return s;
            unsigned long long *cnt = reinterpret_cast<unsigned long long *>(buf);
            DEM_CU(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), sf_));
            if (m_.clumps) k_count<F, true><<<grid(d_.N, 256), 256, 0, sf_>>>(d_, cnt);
            else k_count<F, false><<<grid(d_.N, 256), 256, 0, sf_>>>(d_, cnt);
            DEM_CU(cudaGetLastError());
            unsigned long long h[4];
            DEM_CU(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, sf_));
            DEM_CU(cudaStreamSynchronize(sf_));
            o->listed_pairs = (int64_t)h[0];
            o->wall_pairs = (int64_t)h[1];
            o->active_contacts = (int64_t)h[2];
            o->spheres_with_entries = (int64_t)h[3];
        }
        return DEM_OK;
    }

    dem_status diagnostics(dem_diagnostics *o, std::string &err) override
    {
        const int64_t n = std::max<int64_t>(std::max<int64_t>(d_.M, d_.N), 1);
        const int64_t blocks = (n + 255) / 256;
        double *buf;
        dem_status s;
        if ((s = fresh(err))) return s;
        if ((s = scratch(buf, 9 * blocks, err))) return s;
        if (m_.clumps) k_diag<F, true><<<(unsigned)blocks, 256, 0, sf_>>>(d_, buf);
        else k_diag<F, false><<<(unsigned)blocks, 256, 0, sf_>>>(d_, buf);
        DEM_CU(cudaGetLastError());
        std::vector<double> h(9 * blocks);
        DEM_CU(cudaMemcpyAsync(h.data(), buf, h.size() * sizeof(double), cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        double a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t b = 0; b < blocks; ++b)
            for (int c = 0; c < 9; ++c) a[c] += h[9 * b + c];
        o->kinetic = a[0];
        o->potential = a[1];
        o->elastic = a[2];
        for (int c = 0; c < 3; ++c) {
            o->momentum[c] = a[3 + c];
            o->angular_momentum[c] = a[6 + c];
        }
        return DEM_OK;
    }

    dem_status save(std::vector<uint8_t> &blob, std::string &err) override
    {
        dem_status s;
        if ((s = pull(err))) return s;
        blob.clear();
        const int64_t M = d_.M, ne = (int64_t)d_.K * d_.Np;
        const int sp = sth_->state_par, hp = sth_->hist_par, lc = sth_->list_cur;
        auto put = [&](const void *p, size_t n) {
            size_t o = blob.size();
            blob.resize(o + n);
            std::memcpy(blob.data() + o, p, n);
        };
        uint64_t magic = 0x44454d4742333033ull;   // "DEMGB303": 32-byte position records, status lines split
        put(&magic, 8);
        int64_t hdr[6] = {M, d_.N, d_.Np, d_.K, (int64_t)F::voxel, (int64_t)sizeof(R)};
        put(hdr, sizeof(hdr));
        put(sth_, sizeof(DevStatus));
        auto dput = [&](const void *dp, size_t n) -> dem_status {
            size_t o = blob.size();
            blob.resize(o + n);
            return copy_sync(blob.data() + o, dp, n, cudaMemcpyDeviceToHost, err);
        };
        if constexpr (F::voxel) {
            if ((s = dput(d_.st.pos[sp].rec, M * 32))) return s;
        } else {
            if ((s = dput(d_.st.pos[sp].xm, M * 32))) return s;
        }
        if ((s = dput(d_.st.kv[sp], 2 * M * sizeof(R4)))) return s;
        if ((s = dput(d_.st.quat[sp], M * sizeof(R4)))) return s;
        if ((s = dput(d_.st.active[sp], M))) return s;
        if ((s = dput(d_.lists.partner[lc], ne * 4))) return s;
        if ((s = dput(d_.lists.cnt[lc], d_.Np))) return s;
        if ((s = dput(d_.lists.hist[hp], ne * sizeof(typename HistVec<R>::T)))) return s;
        if (d_.lists.wild[hp] && (s = dput(d_.lists.wild[hp], ne * sizeof(typename HistVec<R>::T)))) return s;
        double extra[2] = {beta_, (double)fallbacks_};
        put(extra, sizeof(extra));
        return DEM_OK;
    }

    dem_status load(const uint8_t *blob, size_t nb, std::string &err) override
    {
        learned_left_ = 0;                   // the next cycle asks the network again
        size_t off = 0;
        auto get = [&](void *p, size_t n) -> bool {
            if (off + n > nb) return false;
            std::memcpy(p, blob + off, n);
            off += n;
            return true;
        };
        uint64_t magic;
        int64_t hdr[6];
        DevStatus h;
        if (!get(&magic, 8) || magic != 0x44454d4742333033ull || !get(hdr, sizeof(hdr)) || !get(&h, sizeof(h))) {
            err = "not a state blob";
            return DEM_ERR_ARG;
        }
        if (hdr[0] != d_.M || hdr[1] != d_.N || hdr[2] != d_.Np || hdr[4] != (int64_t)F::voxel ||
            hdr[5] != (int64_t)sizeof(R)) {
            err = "state blob of a different world";
            return DEM_ERR_ARG;
        }
        dem_status s;
        if (hdr[3] != d_.K) {
            if ((s = realloc_lists((int)hdr[3], false, err))) return s;
        }
        DEM_CU(cudaStreamSynchronize(sf_));
        DEM_CU(cudaStreamSynchronize(sd_));
        const int64_t M = d_.M, ne = (int64_t)d_.K * d_.Np;
        const int sp = h.state_par, hp = h.hist_par, lc = h.list_cur;
        auto dget = [&](void *dp, size_t n) -> dem_status {
            if (off + n > nb) { err = "truncated state blob"; return DEM_ERR_ARG; }
            const size_t o = off;
            off += n;
            return copy_sync(dp, blob + o, n, cudaMemcpyHostToDevice, err);
        };
        if constexpr (F::voxel) {
            if ((s = dget(d_.st.pos[sp].rec, M * 32))) return s;
        } else {
            if ((s = dget(d_.st.pos[sp].xm, M * 32))) return s;
        }
        if ((s = dget(d_.st.kv[sp], 2 * M * sizeof(R4)))) return s;
        if ((s = dget(d_.st.quat[sp], M * sizeof(R4)))) return s;
        if (!m_.clumps && M > 0)     // both orientation buffers hold the restored orientation
            if ((s = copy_sync(d_.st.quat[sp ^ 1], d_.st.quat[sp], M * sizeof(R4), cudaMemcpyDeviceToDevice, err)))
                return s;
        if ((s = dget(d_.st.active[sp], M))) return s;
        if ((s = dget(d_.lists.partner[lc], ne * 4))) return s;
        if ((s = dget(d_.lists.cnt[lc], d_.Np))) return s;
        if ((s = dget(d_.lists.hist[hp], ne * sizeof(typename HistVec<R>::T)))) return s;
        if (d_.lists.wild[hp] && (s = dget(d_.lists.wild[hp], ne * sizeof(typename HistVec<R>::T)))) return s;
        double extra[2];
        if (!get(extra, sizeof(extra))) { err = "truncated state blob"; return DEM_ERR_ARG; }
        // the margin is a tuning choice (results are the same bits for every margin) and
        // stays as it is; a list built for another margin is rebuilt before the next step
        const double beta_blob = extra[0];
        fallbacks_ = (int64_t)extra[1];
        h.halt = 0;
        h.step_disp_bits = 0;
        h.vmax_bits = 0;
        h.diverged = 0;
        {
            // the cell table still holds entries stamped by builds after the checkpoint:
            // the stamp only moves forward
            unsigned int cur = 0;
            if ((s = copy_sync(&cur, &st_->cell_stamp, sizeof(cur), cudaMemcpyDeviceToHost, err))) return s;
            h.cell_stamp = std::max(h.cell_stamp, cur);
        }
        if ((s = copy_sync(st_, &h, sizeof(h), cudaMemcpyHostToDevice, err))) return s;
        DEM_CU(cudaMemsetAsync(d_.audit, 0, AUDIT_SLOTS * AUDIT_STRIDE * sizeof(unsigned int), sf_));   // no maxima of an unfinished step
        recompact_current();
        pose_facets(sf_);                    // the facets at the restored step
        DEM_CU(cudaStreamSynchronize(sf_));
        dirty_ = beta_blob != beta_;
        return DEM_OK;
    }

    void set_profiling(bool on) override
    {
        prof_ = on;
        drop_graphs();
    }

    dem_status set_margin(double beta, std::string &err) override
    {
        (void)err;
        beta_ = beta;
        dirty_ = true;
        drop_graphs();
        return DEM_OK;
    }

    dem_status schedule_collect(int on, std::string &err) override
    {
        dem_status s;
        if ((s = sched_buffers(err))) return s;
        if ((s = pull(err))) return s;
        if (on && !collect_) {
            collect_ = true;
            if ((s = window_start(err))) return s;
        } else if (!on && collect_) {
            if ((s = window_finish(err))) return s;
            collect_ = false;
        }
        return DEM_OK;
    }

    dem_status schedule_train(int epochs, float lr, uint64_t seed, float *loss, std::string &err) override
    {
        dem_status s;
        if ((s = sched_buffers(err))) return s;
        if (collect_) {
            if ((s = pull(err))) return s;
            if ((s = window_finish(err))) return s;
            if ((s = window_start(err))) return s;
        }
        if (ds_y_.empty()) { err = "no schedule samples collected (dem_schedule_collect)"; return DEM_ERR_STATE; }
        if (epochs < 1 || !(lr > 0.0f)) { err = "need epochs >= 1 and lr > 0"; return DEM_ERR_ARG; }
        DEM_CU(mlp_->train(ds_x_, ds_y_, epochs, lr, seed, loss, sf_));
        return DEM_OK;
    }

    dem_status schedule_export(std::vector<uint8_t> &w, std::string &err) override
    {
        if (!mlp_ || !mlp_->ready()) { err = "the schedule model has no weights yet"; return DEM_ERR_STATE; }
        std::vector<float> p(MLP_NPARAM);
        DEM_CU(mlp_->get_params(p.data(), sf_));
        w.resize(12 + MLP_NPARAM * sizeof(float));
        std::memcpy(w.data(), "DEMSCHD1", 8);
        uint32_t np = MLP_NPARAM;
        std::memcpy(w.data() + 8, &np, 4);
        std::memcpy(w.data() + 12, p.data(), MLP_NPARAM * sizeof(float));
        return DEM_OK;
    }

    dem_status schedule_load(const uint8_t *w, size_t n, std::string &err) override
    {
        learned_left_ = 0;                   // the next cycle asks the network again
        uint32_t np = 0;
        if (n < 12 || std::memcmp(w, "DEMSCHD1", 8) != 0 || (std::memcpy(&np, w + 8, 4), np != (uint32_t)MLP_NPARAM) ||
            n != 12 + MLP_NPARAM * sizeof(float)) {
            err = "not a schedule weight blob";
            return DEM_ERR_ARG;
        }
        dem_status s;
        if ((s = sched_buffers(err))) return s;
        std::vector<float> p(MLP_NPARAM);
        std::memcpy(p.data(), w + 12, MLP_NPARAM * sizeof(float));
        DEM_CU(mlp_->set_params(p.data(), sf_));
        return DEM_OK;
    }

    int64_t schedule_samples() const { return (int64_t)(ds_y_.size() / MLP_OUT); }

private:
    static unsigned grid(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

    int64_t wall_local(uint32_t wg) const
    {
        for (size_t sc = m_.scene_wall_base.size(); sc-- > 0;)
            if ((int64_t)wg >= m_.scene_wall_base[sc]) return (int64_t)wg - m_.scene_wall_base[sc];
        return (int64_t)wg;
    }

    template <class T>
    dem_status alloc(T *&p, int64_t count, std::string &err)
    {
        size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
        void *ptr = nullptr;
        if (m_.alloc) {
            ptr = m_.alloc(bytes, m_.alloc_ctx);
            if (!ptr) { err = "allocator callback failed"; return DEM_ERR_NOMEM; }
        } else {
            cudaError_t e = cudaMalloc(&ptr, bytes);
            if (e != cudaSuccess) { err = std::string("cudaMalloc: ") + cudaGetErrorString(e); return DEM_ERR_NOMEM; }
        }
        // zeroed on the force stream and waited for: the library's streams do not
        // synchronise with the legacy default stream, so a plain cudaMemset could still be
        // clearing the buffer when the next kernel on the force stream writes it
        cudaError_t e = cudaMemsetAsync(ptr, 0, bytes, sf_);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sf_);
        if (e != cudaSuccess) { err = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e); return DEM_ERR_CUDA; }
        allocs_.push_back(ptr);
        p = reinterpret_cast<T *>(ptr);
        return DEM_OK;
    }

    void dfree(void *p)
    {
        if (!p) return;
        auto it = std::find(allocs_.begin(), allocs_.end(), p);
        if (it != allocs_.end()) allocs_.erase(it);
        if (m_.free) m_.free(p, m_.alloc_ctx);
        else cudaFree(p);
    }

    template <class T>
    dem_status up(T *dst, const T *src, int64_t count, std::string &err)
    {
        if (count <= 0) return DEM_OK;
        return copy_sync(dst, src, (size_t)count * sizeof(T), cudaMemcpyHostToDevice, err);
    }

    // A copy outside the step, on the force stream and waited for (ordered after the work
    // queued there, complete before anything queued later on either stream).
    dem_status copy_sync(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, std::string &err)
    {
        if (bytes == 0) return DEM_OK;
        DEM_CU(cudaMemcpyAsync(dst, src, bytes, kind, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        return DEM_OK;
    }

    // grow-only scratch buffer for read-back kernels
    dem_status scratch(double *&p, int64_t count, std::string &err)
    {
        if (count > scratch_n_) {
            if (scratch_) dfree(scratch_);
            scratch_ = nullptr;
            scratch_n_ = 0;
            dem_status s = alloc(scratch_, count, err);
            if (s) return s;
            scratch_n_ = count;
        }
        p = scratch_;
        return DEM_OK;
    }

    dem_status alloc_lists(int K, std::string &err)
    {
        const int64_t ne = (int64_t)K * d_.Np;
        dem_status s;
        for (int b = 0; b < 2; ++b) {
            if ((s = alloc(d_.lists.partner[b], ne, err))) return s;
            if ((s = alloc(d_.lists.cnt[b], std::max(d_.Np, Mp_), err))) return s;
            if ((s = alloc(d_.lists.hist[b], ne, err))) return s;
            d_.lists.wild[b] = nullptr;
            if (model_wildcards() > 4 && (s = alloc(d_.lists.wild[b], ne, err))) return s;
            if (!act_alloc_) {
                if ((s = alloc(d_.lists.act[b], d_.Np, err))) return s;
                if ((s = alloc(d_.lists.n_act[b], 1, err))) return s;
                if ((s = alloc(d_.lists.perm[b], d_.Np, err))) return s;
                if ((s = alloc(d_.lists.bcount[b], (d_.Np + 255) / 256 + 1, err))) return s;
            }
        }
        act_alloc_ = true;
        d_.K = K;
        return DEM_OK;
    }

    // Grow the row capacity to K, keeping the list in use and the current history.
    dem_status realloc_lists(int K, bool keep, std::string &err)
    {
        drop_graphs();
        DEM_CU(cudaStreamSynchronize(sf_));
        DEM_CU(cudaStreamSynchronize(sd_));
        ListBuffers<R> old = d_.lists;
        const int Kold = d_.K;
        const int lc = sth_->list_cur, hp = sth_->hist_par;
        dem_status s;
        if ((s = alloc_lists(K, err))) return s;
        if (keep) {
            const int64_t ne = (int64_t)std::min(Kold, K) * d_.Np;
            if ((s = copy_sync(d_.lists.partner[lc], old.partner[lc], ne * 4, cudaMemcpyDeviceToDevice, err))) return s;
            if ((s = copy_sync(d_.lists.cnt[lc], old.cnt[lc], d_.Np, cudaMemcpyDeviceToDevice, err))) return s;
            if ((s = copy_sync(d_.lists.hist[hp], old.hist[hp], ne * sizeof(typename HistVec<R>::T),
                               cudaMemcpyDeviceToDevice, err)))
                return s;
            if (old.wild[hp] &&
                (s = copy_sync(d_.lists.wild[hp], old.wild[hp], ne * sizeof(typename HistVec<R>::T),
                               cudaMemcpyDeviceToDevice, err)))
                return s;
        }
        for (int b = 0; b < 2; ++b) {
            dfree(old.partner[b]); dfree(old.cnt[b]);
            dfree(old.hist[b]);
            dfree(old.wild[b]);
        }
        if (keep) recompact_current();
        if (tune_.integrate_staged) {               // new row-length arrays: check them again
            staged_per_sm_ = 0;
            tune_.integrate_staged = prepare_staged() ? 1 : 0;
        }
        return DEM_OK;
    }

    // keep_bounds (an upload between steps): the audit accumulators grow by each owner's
    // displacement instead of restarting; *max_bound (nullable) receives the largest one of
    // the list in use among the uploaded owners.
    dem_status upload_state(int64_t first, int64_t n, const double *x, const double *q, const double *v,
                            const double *w, const uint8_t *act, std::string &err, bool keep_bounds = false,
                            double *max_bound = nullptr)
    {
        learned_left_ = 0;
        if (n <= 0) return DEM_OK;
        double *buf;
        dem_status s;
        if ((s = scratch(buf, 13 * n + (n + 7) / 8 + 1, err))) return s;
        double *dx = x ? buf : nullptr, *dq = q ? buf + 3 * n : nullptr, *dv = v ? buf + 7 * n : nullptr,
               *dw = w ? buf + 10 * n : nullptr;
        uint8_t *da = act ? reinterpret_cast<uint8_t *>(buf + 13 * n) : nullptr;
        int *bad = reinterpret_cast<int *>(buf + 13 * n + (n + 7) / 8);
        // the arrays are copied in pieces on the copy stream (after the force stream's
        // earlier work, which may still read the scratch); the force stream checks each
        // piece for non-finite positions and velocities as soon as it has landed, while
        // the next piece is copied, and nothing is applied before every piece has passed
        DEM_CU(cudaEventRecord(ev_up_, sf_));
        DEM_CU(cudaStreamWaitEvent(sc_, ev_up_, 0));
        if (x || v || w) DEM_CU(cudaMemsetAsync(bad, 0, sizeof(int), sf_));
        struct Piece {
            const double *h;   // caller's array
            double *dev;       // its scratch copy
            int c;             // doubles per owner
            bool check;        // rejected if not finite
        };
        const Piece arrs[4] = {{x, dx, 3, true}, {q, dq, 4, false}, {v, dv, 3, true}, {w, dw, 3, true}};
        const int64_t chunk = n >= (int64_t)1 << 20 ? (n + 3) / 4 : n;
        for (int64_t c0 = 0; c0 < n; c0 += chunk) {
            const int64_t cn = std::min(chunk, n - c0);
            for (const Piece &a : arrs)
                if (a.h)
                    DEM_CU(cudaMemcpyAsync(a.dev + a.c * c0, a.h + a.c * c0, a.c * cn * sizeof(double),
                                           cudaMemcpyHostToDevice, sc_));
            DEM_CU(cudaEventRecord(ev_up_, sc_));
            DEM_CU(cudaStreamWaitEvent(sf_, ev_up_, 0));
            for (const Piece &a : arrs)
                if (a.h && a.check)
                    k_nonfinite<<<grid(a.c * cn, 256), 256, 0, sf_>>>(a.dev + a.c * c0, a.c * cn, bad);
        }
        if (act) {
            DEM_CU(cudaMemcpyAsync(da, act, n, cudaMemcpyHostToDevice, sc_));
            DEM_CU(cudaEventRecord(ev_up_, sc_));
            DEM_CU(cudaStreamWaitEvent(sf_, ev_up_, 0));
        }
        DEM_CU(cudaGetLastError());
        if (x || v || w) {
            int hbad = 0;
            DEM_CU(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, sf_));
            DEM_CU(cudaStreamSynchronize(sf_));
            if (hbad) {
                err = "non-finite state";
                return DEM_ERR_ARG;
            }
        }
        const int bounds = keep_bounds ? 1 : 0;
        if (keep_bounds)
            DEM_CU(cudaMemsetAsync(&st_->upload_disp_bits, 0, sizeof(unsigned int), sf_));
        // one pass: a thread converts its angular velocity with the orientation it has just
        // stored
        int ex = 0;
        const double inv_ld = (F::voxel && std::frexp(d_.Ld, &ex) == 0.5) ? 1.0 / d_.Ld : 0.0;
        k_owner_upload<F><<<grid(n, 256), 256, 0, sf_>>>(d_, first, n, dx, dq, dv, dw, da, bounds, inv_ld);
        if (!m_.clumps) k_mirror_quat<F><<<grid(n, 256), 256, 0, sf_>>>(d_, first, n);
        DEM_CU(cudaGetLastError());
        unsigned int bits = 0;
        if (keep_bounds) DEM_CU(cudaMemcpyAsync(&bits, &st_->upload_disp_bits, sizeof(bits), cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        if (max_bound) {
            float f;
            std::memcpy(&f, &bits, sizeof(f));
            *max_bound = (double)f;
        }
        return DEM_OK;
    }

    dem_status fetch_list(int lc, std::vector<uint32_t> &partner, std::vector<uint8_t> &cnt, std::string &err)
    {
        const int64_t ne = (int64_t)d_.K * d_.Np;
        partner.resize(ne);
        cnt.resize(d_.Np);
        DEM_CU(cudaMemcpyAsync(partner.data(), d_.lists.partner[lc], ne * 4, cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaMemcpyAsync(cnt.data(), d_.lists.cnt[lc], d_.Np, cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        return DEM_OK;
    }

    // Copy the device status into the pinned mirror (synchronous).
    dem_status pull(std::string &err)
    {
        DEM_CU(cudaStreamSynchronize(sd_));
        DEM_CU(cudaMemcpyAsync(sth_, st_, sizeof(DevStatus), cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        if (!marks_.empty()) harvest();
        return DEM_OK;
    }

    // ---- cycles, graphs, tuning
    // One cycle of a delayed schedule: snapshot, detection of the next list (beside the
    // steps on the detection stream, or before them on the force stream), c steps with
    // the list in use, switch.
    void enqueue_cycle(long long c)
    {
        if (tune_.detect_inline) {
            Mark m1, m2;
            mark_begin(P_HASH, sf_, m1);
            launch_hash(sf_);
            mark_end(sf_, m1);
            mark_begin(P_DETECT, sf_, m2);
            launch_detect(sf_);
            mark_end(sf_, m2);
            for (long long k = 0; k < c; ++k) force_step();
            Mark m3;
            mark_begin(P_LINK, sf_, m3);
            launch_link(sf_);
            mark_end(sf_, m3);
        } else {
            start_detect();
            for (long long k = 0; k < c; ++k) force_step();
            finish_detect();
        }
    }

    // Cycle lengths are rounded down to {1, 2, 3} and {4, 5, 6, 7} x 2^j so that a few
    // captured graphs serve every cycle (the schedule only affects timing, not results).
    static long long quantize_cycle(long long c)
    {
        if (c <= 3) return std::max<long long>(c, 1);
        long long p = 4;
        while (p * 2 <= c) p *= 2;
        long long step = p / 4;
        return p + ((c - p) / step) * step;
    }

    // Captured graph of one every-step step (c = 0) or one delayed cycle of length c.
    cudaGraphExec_t graph_for(long long c)
    {
        for (auto &g : graphs_)
            if (g.c == c) return g.exec;
        if (graphs_.size() >= 24) drop_graphs();
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cudaStreamBeginCapture(sf_, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (c == 0) {
            rebuild_inline(sf_);
            force_step();
        } else {
            enqueue_cycle(c);
        }
        if (cudaStreamEndCapture(sf_, &graph) != cudaSuccess || !graph) {
            cudaGetLastError();
            graphs_on_ = false;                      // fall back to direct launches
            return nullptr;
        }
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(graph);
            graphs_on_ = false;
            return nullptr;
        }
        cudaGraphDestroy(graph);
        graphs_.push_back({c, exec});
        return exec;
    }

    void drop_graphs()
    {
        for (auto &g : graphs_) cudaGraphExecDestroy(g.exec);
        graphs_.clear();
    }

    dem_status set_tuning(const dem_tuning *t, std::string &err) override
    {
        if (t->contact_block < 32 || t->contact_block > CONTACT_BLOCK_MAX || t->contact_block % 32 ||
            t->integrate_block < 32 || t->integrate_block > INTEGRATE_BLOCK_MAX || t->integrate_block % 32 ||
            t->narrow_block < 32 || t->narrow_block > 256 || t->narrow_block % 32) {
            err = "block sizes must be multiples of 32 within the kernels' limits";
            return DEM_ERR_ARG;
        }
        if (t->fused_block != 0 && t->fused_block != 64 && t->fused_block != 128 && t->fused_block != 256) {
            err = "fused_block must be 0, 64, 128 or 256";
            return DEM_ERR_ARG;
        }
        if (t->binning < 0 || t->binning > 2) {
            err = "binning must be 0 (automatic), 1 (radix sort) or 2 (counting sort)";
            return DEM_ERR_ARG;
        }
        const double f = t->cell_factor == 0.0 ? 1.0 : t->cell_factor;
        if (!(f >= 1.0 && f <= 4.0)) {
            err = "cell_factor must be in [1, 4]";
            return DEM_ERR_ARG;
        }
        if (!(t->margin >= 0.0) || t->margin > m_.margin_max) {
            err = "margin must be in [0, margin_max]";
            return DEM_ERR_ARG;
        }
        dem_status s;
        if ((s = sync(err))) return s;
        drop_graphs();
        if (f != m_.cell_factor) {
            if ((s = relayout_cells(f, err))) return s;
        }
        tune_ = *t;
        tune_.cell_factor = m_.cell_factor;
        tune_.integrate_staged = (t->integrate_staged && prepare_staged()) ? 1 : 0;
        tune_.contact_lean = t->contact_lean ? 1 : 0;
        tune_.fused_block = m_.clumps ? 0 : t->fused_block;
        tune_.contact_integrates = (!m_.clumps && t->contact_integrates) ? 1 : 0;
        tune_.narrow_staged = (t->narrow_staged && prepare_narrow_staged()) ? 1 : 0;
        tune_.contact_screen = (!m_.clumps && t->contact_screen) ? 1 : 0;
        choose_binning();
        tune_.margin = 0.0;
        apply_margin(t->margin);
        return DEM_OK;
    }

    // A new detection margin for the delayed schedules (0: keep the current one).  The
    // list in use was built for the old margin, so the next step rebuilds it first.
    void apply_margin(double beta)
    {
        if (beta > 0.0 && m_.schedule != DEM_SCHEDULE_EVERY_STEP && beta != beta_) {
            beta_ = beta;
            dirty_ = true;
            drop_graphs();
        }
    }

    // The staged integration needs its shared-memory size allowed once (outside any
    // stream capture) and 16-byte aligned owner arrays (a user allocator might not give
    // them); false where it cannot run.
    bool prepare_staged()
    {
        if constexpr (!F::voxel) {
            return false;
        } else {
            if (staged_per_sm_ > 0) return true;
            const void *ptrs[] = {d_.st.pos[0].rec, d_.st.pos[1].rec, d_.st.kv[0], d_.st.kv[1], d_.st.quat[0],
                                  d_.st.quat[1], d_.st.active[0], d_.st.active[1], d_.inv_moi, d_.inv_mass,
                                  d_.owner_scene, d_.owner_iso, d_.lists.cnt[0], d_.lists.cnt[1]};
            for (const void *p : ptrs)
                if ((uintptr_t)p % 16 != 0) return false;
            const int smem = STAGES * StageLayout::bytes;
            if (cudaFuncSetAttribute(k_integrate_staged<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
                    cudaSuccess ||
                cudaFuncSetAttribute(k_integrate_staged<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
                    cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            int per_sm = 0;
            cudaError_t e = m_.clumps
                                ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate_staged<true>, ITILE, smem)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate_staged<false>, ITILE, smem);
            if (e != cudaSuccess || per_sm < 1) {
                cudaGetLastError();
                return false;
            }
            staged_per_sm_ = per_sm;
            return true;
        }
    }

    // Per-cell counts of the counting-sort binning (zeroed; a whole number of scan tiles)
    // and the scan's per-tile sums.
    dem_status alloc_cell_counts(int64_t n_cells, std::string &err)
    {
        const int64_t len = std::max<int64_t>((n_cells + CS_TILE - 1) / CS_TILE, 1) * CS_TILE;
        uint32_t *cc = nullptr, *ct = nullptr;
        uint8_t *cw = nullptr;
        dem_status s;
        if ((s = alloc(cc, len, err))) return s;
        if ((s = alloc(ct, len / CS_TILE, err)) || (s = alloc(cw, std::max<int64_t>(n_cells, 1), err))) {
            dfree(cc);
            dfree(ct);
            return s;
        }
        if (db_.ccount) dfree(db_.ccount);
        if (db_.ctile) dfree(db_.ctile);
        if (db_.cell_wall) dfree(db_.cell_wall);
        db_.ccount = cc;
        db_.ctile = ct;
        db_.cell_wall = cw;
        db_.ccount_len = len;
        return DEM_OK;
    }

    // Shared memory of the staged narrow phase: records, slots, owners, families.
    static size_t narrow_smem() { return (size_t)NS_CAP * (32 + 4 + 4 + 1); }

    // The staged narrow phase needs its shared-memory size allowed once.
    bool prepare_narrow_staged()
    {
        const int smem = (int)narrow_smem();
        if (cudaFuncSetAttribute(k_narrow<F, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_narrow<F, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
                cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    }

    // Counting sort where the cells are not much more numerous than the sphere slots
    // (its scan reads every cell), else the radix sort; the tuning may force either.
    void choose_binning()
    {
        const int b = tune_.binning;
        db_.counting = b == 2 || (b == 0 && (int64_t)m_.n_cells_total <= 8 * std::max<int64_t>(d_.N, 1)) ? 1 : 0;
    }

    // New detection cells (nothing in flight: called after sync).  The list in use and
    // the history do not depend on the cells; the next build uses the new ones.
    dem_status relayout_cells(double f, std::string &err)
    {
        HostModel trial = m_;
        dem_status s;
        if ((s = layout_cells(trial, f, err))) return s;
        uint4 *ct = nullptr;
        if ((s = alloc(ct, (int64_t)trial.n_cells_total + 1, err))) return s;
        if ((s = alloc_cell_counts(trial.n_cells_total, err))) {
            dfree(ct);
            return s;
        }
        dfree(db_.cell_tab);
        db_.cell_tab = ct;
        m_.L = trial.L;
        m_.vpc = trial.vpc;
        m_.cell_factor = trial.cell_factor;
        m_.n_cells_total = trial.n_cells_total;
        m_.scenes = trial.scenes;
        if (!F::voxel) {
            d_.L = (float)m_.L;
            d_.Ld = m_.L;
        }
        d_.invL = 1.0 / m_.L;
        d_.vpc = m_.vpc;
        db_.n_cells_total = m_.n_cells_total;
        db_.key_bits = 1;
        while (db_.key_bits < 32 && ((uint64_t)1 << db_.key_bits) <= (uint64_t)m_.n_cells_total) ++db_.key_bits;
        choose_binning();
        if ((s = copy_sync(const_cast<Scene *>(d_.scenes), m_.scenes.data(), m_.scenes.size() * sizeof(Scene),
                           cudaMemcpyHostToDevice, err)))
            return s;
        flag_wall_cells(sf_);
        return DEM_OK;
    }

    dem_status get_tuning(dem_tuning *t, std::string &err) override
    {
        (void)err;
        *t = tune_;
        t->margin = beta_;
        return DEM_OK;
    }

    void set_graphs(bool on) override
    {
        graphs_on_ = on;
        if (!on) drop_graphs();
    }

    std::string tune_key()
    {
        cudaDeviceProp prop;
        std::string gpu = "gpu";
        if (cudaGetDeviceProperties(&prop, m_.device) == cudaSuccess) gpu = prop.name;
        for (auto &ch : gpu)
            if (ch == ' ' || ch == '"') ch = '_';
        return std::string(F::voxel ? "voxel_fp32" : "fp64") + "|" + std::to_string(m_.schedule) + "|" +
               std::to_string(d_.N) + "|" + std::to_string(d_.M) + "|" + std::to_string((int)m_.clumps) + "|" + gpu;
    }

    dem_status autotune(int steps, const char *cache_path, dem_tuning *chosen, std::string &err) override
    {
        dem_status s;
        const std::string key = tune_key();
        if (cache_path) {
            FILE *f = std::fopen(cache_path, "r");
            if (f) {
                char line[512];
                dem_tuning best{};
                bool found = false;
                while (std::fgets(line, sizeof line, f)) {
                    char k[300];
                    dem_tuning t{};
                    if (std::sscanf(line, "{\"key\": \"%299[^\"]\", \"contact_block\": %d, \"integrate_block\": %d, "
                                          "\"narrow_block\": %d, \"detect_inline\": %d, \"cell_factor\": %lf, "
                                          "\"integrate_staged\": %d, \"contact_lean\": %d, \"fused_block\": %d, "
                                          "\"contact_integrates\": %d, \"binning\": %d, \"narrow_staged\": %d, "
                                          "\"contact_screen\": %d, \"margin\": %lf, \"step_ms\": %lf}",
                                    k, &t.contact_block, &t.integrate_block, &t.narrow_block, &t.detect_inline,
                                    &t.cell_factor, &t.integrate_staged, &t.contact_lean, &t.fused_block,
                                    &t.contact_integrates, &t.binning, &t.narrow_staged, &t.contact_screen,
                                    &t.margin, &t.step_ms) == 15 &&
                        key == k) {
                        best = t;
                        found = true;
                    }
                }
                std::fclose(f);
                if (found) {
                    if ((s = set_tuning(&best, err))) return s;
                    if (chosen) *chosen = best;
                    return DEM_OK;
                }
            }
        }
        std::vector<uint8_t> blob;
        if ((s = save(blob, err))) return s;
        const bool delayed = m_.schedule != DEM_SCHEDULE_EVERY_STEP;
        const double beta0 = beta_;                   // the margin of candidates that leave it
        dem_tuning best = tune_;
        best.margin = 0.0;
        double best_ms = 1e300;
        auto trial = [&](const dem_tuning &t0) -> dem_status {
            dem_status st;
            dem_tuning t = t0;
            if (t.margin <= 0.0) t.margin = beta0;
            if ((st = set_tuning(&t, err))) return st;
            if ((st = load(blob.data(), blob.size(), err))) return st;
            if ((st = step(std::max(2, steps / 4), err))) return st;     // warm-up, graph capture
            DEM_CU(cudaEventRecord(ev_c_, sf_));
            if ((st = step(steps, err))) return st;
            DEM_CU(cudaEventRecord(ev_b_, sf_));
            DEM_CU(cudaEventSynchronize(ev_b_));
            float ms = 0.0f;
            DEM_CU(cudaEventElapsedTime(&ms, ev_c_, ev_b_));
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
            return DEM_OK;
        };
        // phase 1: contact block and detection placement; phase 2: the other two shapes;
        // phase 3: the detection cell size
        const double f0 = m_.cell_factor;
        for (int cb : {32, 64, 128})
            for (int di = 0; di <= (delayed ? 1 : 0); ++di)
                if ((s = trial(dem_tuning{cb, 256, 128, di, 0.0, f0, 0, 0, 0}))) return s;
        const dem_tuning b1 = best;
        for (int ib : {256, 512})
            for (int nb : {128, 256})
                if (ib != b1.integrate_block || nb != b1.narrow_block)
                    if ((s = trial(dem_tuning{b1.contact_block, ib, nb, b1.detect_inline, 0.0, f0, 0, 0, 0})))
                        return s;
        if (F::voxel)
            if ((s = trial(dem_tuning{b1.contact_block, 256, best.narrow_block, b1.detect_inline, 0.0, f0, 1, 0, 0})))
                return s;
        {
            dem_tuning t = best;
            t.contact_lean = 1;
            t.step_ms = 0.0;
            if ((s = trial(t))) return s;
        }
        // single spheres: the two-pass contact step (built-in model, no rolling resistance),
        // the contact kernel integrating the owners with partners (each contact build),
        // then forces and integration in one kernel, each block size
        if (!m_.clumps && !m_.rolling && m_.model == FORCE_MODEL_BUILTIN) {
            dem_tuning t = best;
            t.contact_screen = 1;
            t.contact_lean = 0;
            t.step_ms = 0.0;
            if ((s = trial(t))) return s;
        }
        if (!m_.clumps) {
            const dem_tuning b3 = best;
            for (int lean = 0; lean <= 1; ++lean) {
                dem_tuning t = b3;
                t.contact_integrates = 1;
                t.contact_screen = 0;
                t.contact_lean = lean;
                t.step_ms = 0.0;
                if ((s = trial(t))) return s;
            }
            for (int fb : {64, 128, 256}) {
                dem_tuning t = b3;
                t.fused_block = fb;
                t.contact_integrates = 0;
                t.contact_screen = 0;
                t.step_ms = 0.0;
                if ((s = trial(t))) return s;
            }
        }
        const dem_tuning b2 = best;
        for (double f : {1.0, 1.5, 2.0})
            if (f != b2.cell_factor)
                if ((s = trial(dem_tuning{b2.contact_block, b2.integrate_block, b2.narrow_block, b2.detect_inline,
                                          0.0, f, b2.integrate_staged, b2.contact_lean, b2.fused_block, 0.0,
                                          b2.contact_integrates, b2.binning, b2.narrow_staged,
                                          b2.contact_screen})))
                    return s;
        // the binning: radix sort against counting sort (the automatic choice is one of
        // them), then the narrow phase staged in shared memory
        {
            const dem_tuning b5 = best;
            for (int bn : {1, 2}) {
                dem_tuning t = b5;
                t.binning = bn;
                t.step_ms = 0.0;
                if ((s = trial(t))) return s;
            }
            dem_tuning t = best;
            t.narrow_staged = 1;
            t.step_ms = 0.0;
            if ((s = trial(t))) return s;
        }
        // phase 4 (delayed schedules): smaller detection margins list fewer pairs that do
        // not touch, at the price of more rebuilds; the results are the same bits
        if (delayed) {
            const dem_tuning b4 = best;
            for (double fm : {0.75, 0.5, 0.35, 0.25, 0.18}) {
                dem_tuning t = b4;
                t.margin = fm * m_.margin_max;
                t.step_ms = 0.0;
                if ((s = trial(t))) return s;
            }
        }
        best.step_ms = best_ms / steps;
        if (best.margin <= 0.0) best.margin = beta0;
        if ((s = set_tuning(&best, err))) return s;
        if ((s = load(blob.data(), blob.size(), err))) return s;
        best.margin = beta_;
        if (chosen) *chosen = best;
        if (cache_path) {
            FILE *f = std::fopen(cache_path, "a");
            if (f) {
                std::fprintf(f,
                             "{\"key\": \"%s\", \"contact_block\": %d, \"integrate_block\": %d, \"narrow_block\": "
                             "%d, \"detect_inline\": %d, \"cell_factor\": %.3f, \"integrate_staged\": %d, "
                             "\"contact_lean\": %d, \"fused_block\": %d, \"contact_integrates\": %d, "
                             "\"binning\": %d, \"narrow_staged\": %d, \"contact_screen\": %d, \"margin\": %.17g, "
                             "\"step_ms\": %.6f}\n",
                             key.c_str(), best.contact_block, best.integrate_block, best.narrow_block,
                             best.detect_inline, best.cell_factor, best.integrate_staged, best.contact_lean,
                             best.fused_block, best.contact_integrates, best.binning, best.narrow_staged,
                             best.contact_screen, best.margin, best.step_ms);
                std::fclose(f);
            }
        }
        return DEM_OK;
    }

    // ---- learned schedule
    dem_status sched_buffers(std::string &err)
    {
        if (!mlp_) mlp_.reset(new Mlp());
        if (bin_stats_) return DEM_OK;
        const int nb = std::max(1, m_.n_bins);
        dem_status s;
        if ((s = alloc(bin_stats_, (int64_t)nb * NSTAT, err))) return s;
        if ((s = alloc(obin_, d_.M, err))) return s;
        if ((s = alloc(X_, (int64_t)nb * 16, err))) return s;
        if ((s = alloc(valid_, nb, err))) return s;
        if ((s = alloc(pred_, (int64_t)nb * MLP_OUT, err))) return s;
        if ((s = alloc(predmin_, 1, err))) return s;
        if ((s = alloc(bin_scene_, nb, err))) return s;
        if ((s = alloc(acc_lab_, d_.M, err))) return s;
        if ((s = alloc(cross_, 2 * (int64_t)nb, err))) return s;
        if ((s = alloc(d_.amag, d_.M, err))) return s;
        drop_graphs();                                   // captured launches hold the old view
        std::vector<int> bs(nb, 0);
        for (size_t sc = 0; sc < m_.scenes.size(); ++sc) {
            const Scene &g = m_.scenes[sc];
            for (int b = 0; b < g.nb[0] * g.nb[1] * g.nb[2]; ++b) bs[g.bin_base + b] = (int)sc;
        }
        if ((s = up(bin_scene_, bs.data(), nb, err))) return s;
        if (!m_.schedule_model.empty() && !mlp_->ready()) {
            if ((s = schedule_load(m_.schedule_model.data(), m_.schedule_model.size(), err))) return s;
        }
        return DEM_OK;
    }

    // Per-bin features of the current state into X_ / valid_ (force stream).
    dem_status features(std::string &err)
    {
        const int nb = std::max(1, m_.n_bins);
        DEM_CU(cudaMemsetAsync(bin_stats_, 0, (size_t)nb * NSTAT * sizeof(float), sf_));
        if (d_.M > 0) k_bin_stats<F><<<grid(d_.M, 256), 256, 0, sf_>>>(d_, bin_stats_, obin_);
        k_bin_features<<<grid(nb, 256), 256, 0, sf_>>>(bin_stats_, nb, bin_scene_, d_.scenes, (float)beta_,
                                                        (float)m_.r_max, X_, valid_);
        DEM_CU(cudaGetLastError());
        return DEM_OK;
    }

    dem_status window_start(std::string &err)
    {
        dem_status s;
        if ((s = features(err))) return s;
        const int nb = std::max(1, m_.n_bins);
        win_x_.resize((size_t)nb * 16);
        win_valid_.resize(nb);
        DEM_CU(cudaMemcpyAsync(win_x_.data(), X_, win_x_.size() * sizeof(float), cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaMemcpyAsync(win_valid_.data(), valid_, nb * sizeof(int), cudaMemcpyDeviceToHost, sf_));
        std::vector<int> init(2 * (size_t)nb, win_len_);
        DEM_CU(cudaMemcpyAsync(cross_, init.data(), init.size() * sizeof(int), cudaMemcpyHostToDevice, sf_));
        DEM_CU(cudaMemsetAsync(acc_lab_, 0, (size_t)std::max<int64_t>(d_.M, 1) * sizeof(float), sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        win_start_ = sth_->steps_done;
        return DEM_OK;
    }

    // Close the window: label every occupied bin with log2 of the steps its largest
    // displacement bound took to pass beta and beta/2 (censored at the window length).
    dem_status window_finish(std::string &err)
    {
        const long long len = sth_->steps_done - win_start_;
        if (win_start_ < 0 || len < 8) return DEM_OK;      // too short to label anything
        const int nb = std::max(1, m_.n_bins);
        std::vector<int> cr(2 * (size_t)nb);
        DEM_CU(cudaMemcpyAsync(cr.data(), cross_, cr.size() * sizeof(int), cudaMemcpyDeviceToHost, sf_));
        DEM_CU(cudaStreamSynchronize(sf_));
        const int cap = (int)std::min<long long>(len, win_len_);
        for (int b = 0; b < nb; ++b) {
            if (!win_valid_[b]) continue;
            for (int k = 0; k < 16; ++k) ds_x_.push_back(win_x_[(size_t)b * 16 + k]);
            // target: residual over the kinematic estimate log2(1 / feature 13)
            const float lin = std::log2(std::max(win_x_[(size_t)b * 16 + 13], 1e-6f));
            for (int j = 0; j < 2; ++j)
                ds_y_.push_back(std::log2((float)std::max(1, std::min(cr[2 * b + j], cap))) + lin);
        }
        return DEM_OK;
    }

    // After a synchronisation: roll the collection window when it is long enough.
    dem_status collect_roll(std::string &err)
    {
        if (!collect_ || sth_->steps_done - win_start_ < win_len_) return DEM_OK;
        dem_status s;
        if ((s = window_finish(err))) return s;
        return window_start(err);
    }

    // Learned cycle length: the smallest predicted log2(steps until a bin passes beta) over
    // the occupied bins; a list is used from c to 2c steps after its snapshot, so c is
    // half of it, with a 20% allowance.
    // The network runs at every LEARNED_REUSE-th cycle boundary (and after any audit
    // fallback); the cycles between reuse its last answer: the features move little over a
    // few cycles, and each evaluation (a pass over all owners, the network, a read-back)
    // sits on the critical path at the boundary.  Any answer is audited.
    static constexpr int LEARNED_REUSE = 4;
    long long learned_c_ = 0;
    int learned_left_ = 0;
    long long learned_cycle(std::string &err)
    {
        if (learned_left_ > 0 && learned_c_ > 0) {
            --learned_left_;
            return learned_c_;
        }
        learned_c_ = learned_eval(err);
        learned_left_ = LEARNED_REUSE - 1;
        return learned_c_;
    }
    long long learned_eval(std::string &err)
    {
        if (sched_buffers(err) || !mlp_->ready()) return 0;
        const int nb = std::max(1, m_.n_bins);
        if (features(err)) return 0;
        if (mlp_->forward(X_, nb, pred_, sf_) != cudaSuccess) return 0;
        k_min_pred<<<1, 256, 0, sf_>>>(pred_, X_, valid_, nb, predmin_);
        float p = 0.0f;
        if (cudaMemcpyAsync(&p, predmin_, sizeof(float), cudaMemcpyDeviceToHost, sf_) != cudaSuccess) return 0;
        if (cudaStreamSynchronize(sf_) != cudaSuccess) return 0;
        if (!(p == p) || p > 30.0f) p = 30.0f;
        double n = std::exp2((double)p);
        return std::max<long long>(1, (long long)std::floor(0.4 * n));
    }

    // Read-backs that depend on the current contacts need a list that covers them: after
    // a step the list in use may be stale (every-step lists are built before the step).
    dem_status fresh(std::string &err)
    {
        dem_status s;
        if ((s = pull(err))) return s;
        if (sth_->halt == HALT_NONE && (sth_->list_stale || dirty_) && d_.N > 0) {
            rebuild_inline(sf_);
            if ((s = settle(err))) return s;
            dirty_ = false;
        }
        return DEM_OK;
    }

    // After queued work: surface launch errors, recover from overflow, report divergence.
    dem_status settle(std::string &err)
    {
        DEM_CU(cudaGetLastError());
        dem_status s;
        if ((s = pull(err))) return s;
        if (sth_->halt == HALT_OVERFLOW) {
            int need = sth_->max_row;
            if (need > KMAX) {
                err = "a contact-list row needs " + std::to_string(need) + " entries (limit " + std::to_string(KMAX) + ")";
                return DEM_ERR_OVERFLOW;
            }
            int K = std::min(KMAX, std::max(need + 4, d_.K + d_.K / 2));
            K = (K + 3) / 4 * 4;
            if (K > KMAX) K = KMAX;
            if ((s = realloc_lists(K, true, err))) return s;
            regrows_ += 1;
            DevStatus h = *sth_;
            h.halt = HALT_NONE;
            h.overflow = 0;
            h.max_row = 0;
            h.step_disp_bits = 0;
            h.vmax_bits = 0;
            if ((s = copy_sync(st_, &h, sizeof(h), cudaMemcpyHostToDevice, err))) return s;
            DEM_CU(cudaMemsetAsync(d_.audit, 0, AUDIT_SLOTS * AUDIT_STRIDE * sizeof(unsigned int), sf_));   // no maxima of an unfinished step
            rebuild_inline(sf_);
            return settle(err);
        }
        if (sth_->halt == HALT_DIVERGED) {
            err = "a speed exceeded the error-out velocity or became non-finite after step " +
                  std::to_string(sth_->steps_done);
            return DEM_ERR_DIVERGED;
        }
        if (sth_->halt == HALT_FACETS) {
            err = "a mesh facet's cell bins overflowed their share";
            return DEM_ERR_OVERFLOW;
        }
        if (sth_->halt != HALT_NONE) {
            err = "halted (code " + std::to_string(sth_->halt) + ")";
            return DEM_ERR_TIMEOUT;
        }
        return DEM_OK;
    }

    void launch_hash(cudaStream_t st)
    {
        if (m_.clumps) k_hash<F, true><<<grid(d_.N, 256), 256, 0, st>>>(d_, db_, beta_);
        else k_hash<F, false><<<grid(d_.N, 256), 256, 0, st>>>(d_, db_, beta_);
    }

    void launch_detect(cudaStream_t st)
    {
        uint32_t *ks, *vs;
        if (db_.counting) {
            const unsigned nt = (unsigned)(db_.ccount_len / CS_TILE);
            k_ccount<F><<<grid(d_.N, 256), 256, 0, st>>>(d_, db_);
            k_cscan_reduce<<<nt, CS_THREADS, 0, st>>>(st_, db_.ccount, db_.ctile);
            k_cscan_tiles<<<1, 1024, 0, st>>>(st_, db_.ctile, (int64_t)nt, db_.n_valid);
            k_cscan_write<F><<<nt, CS_THREADS, 0, st>>>(d_, db_, db_.ctile);
            k_clear_rows<F><<<grid(d_.Np, 256), 256, 0, st>>>(d_, db_);
            k_cscatter<F><<<grid(d_.N, 256), 256, 0, st>>>(d_, db_, db_.keys_alt, db_.vals_alt);
            // the counts start at zero for the next build, whether or not this one halted
            cudaMemsetAsync(db_.ccount, 0, (size_t)db_.ccount_len * sizeof(uint32_t), st);
            ks = db_.keys_alt;
            vs = db_.vals_alt;
        } else {
            radix_sort_u32(db_.keys, db_.vals, db_.keys_alt, db_.vals_alt, d_.N, db_.key_bits, db_.hist,
                           db_.hist_cap, st, &ks, &vs);
            k_clear_rows<F><<<grid(d_.Np, 256), 256, 0, st>>>(d_, db_);
            k_cellstart<F><<<grid(d_.N, 256), 256, 0, st>>>(d_, db_, ks, vs);
        }
        if (db_.n_facets > 0) {
            // bin the facets at their pose of the snapshot and sort the pairs by cell
            k_facet_bin<F><<<grid((int64_t)db_.n_facets * 32, 128), 128, 0, st>>>(d_, db_, m_.r_max);
            uint32_t *fk, *fv;
            radix_sort_u32(db_.fkeys, db_.fvals, db_.fkeys_alt, db_.fvals_alt, db_.n_fpairs, db_.key_bits, db_.fhist,
                           db_.fhist_cap, st, &fk, &fv);
            db_.fkeys_sorted = fk;
            db_.fvals_sorted = fv;
            k_facet_cells<<<grid(db_.n_fpairs, 256), 256, 0, st>>>(st_, db_);
        }
        if (tune_.narrow_staged) {
            const size_t smem = narrow_smem();
            if (m_.clumps) k_narrow<F, true, true><<<grid(d_.N, NS_THREADS), NS_THREADS, smem, st>>>(d_, db_, ks, vs);
            else k_narrow<F, false, true><<<grid(d_.N, NS_THREADS), NS_THREADS, smem, st>>>(d_, db_, ks, vs);
        } else if (m_.clumps) {
            k_narrow<F, true><<<grid(d_.N, tune_.narrow_block), tune_.narrow_block, 0, st>>>(d_, db_, ks, vs);
        } else {
            k_narrow<F, false><<<grid(d_.N, tune_.narrow_block), tune_.narrow_block, 0, st>>>(d_, db_, ks, vs);
        }
        const unsigned nb = grid(d_.Np, 256);
        k_rows_finish<F><<<nb, 256, 0, st>>>(d_, db_, d_.lists.bcount[0]);
        // single spheres: the new list's compacted work (scan of the busy slots per block,
        // then the entries), ahead of the switch: it writes only the new list's arrays
        if (!m_.clumps) {
            k_cscan_tiles<<<1, 1024, 0, st>>>(st_, d_.lists.bcount[0], (int64_t)nb, d_.lists.bcount[0] + nb);
            k_compact<F><<<nb, 256, 0, st>>>(d_, 0, 1, d_.lists.bcount[0], (int64_t)nb);
        }
    }

    void launch_link(cudaStream_t st)
    {
        if (m_.clumps) {
            k_act_reset<F><<<1, 1, 0, st>>>(d_, 0);
            k_link<F><<<grid(d_.N, 256), 256, 0, st>>>(d_);
            launch_compact(st, 0);
        } else {
            // the new list's work was compacted with its detection: link its busy slots only
            k_act_reset<F><<<1, 1, 0, st>>>(d_, 0, 1);
            k_link<F, true><<<grid(d_.Np, 256), 256, 0, st>>>(d_);
        }
        k_commit<<<1, 1, 0, st>>>(st_);
    }

    // compacted work: clump groups, or single spheres ordered by row length per block
    void launch_compact(cudaStream_t st, int which)
    {
        if (m_.clumps) {
            k_compact<F><<<grid(d_.Np, 256), 256, 0, st>>>(d_, which, 0, nullptr, 0);
        } else {
            // per-block counts and their scan (total last; for a new list both ran on the
            // detection stream after its rows), then each block writes its entries at its
            // offset: the work follows slot order
            const unsigned nb = grid(d_.Np, 256);
            uint32_t *bc = d_.lists.bcount[which];
            if (which) {
                k_compact_count<F><<<nb, 256, 0, st>>>(d_, which, bc);
                k_cscan_tiles<<<1, 1024, 0, st>>>(st_, bc, (int64_t)nb, bc + nb);
            }
            k_compact<F><<<nb, 256, 0, st>>>(d_, which, 1, bc, (int64_t)nb);
        }
    }

    // rebuild the compacted work of the list in use (after a restore or a regrow)
    void recompact_current()
    {
        k_act_reset<F><<<1, 1, 0, sf_>>>(d_, 1);
        launch_compact(sf_, 1);
    }

    void rebuild_inline(cudaStream_t st)
    {
        Mark m1, m2, m3;
        mark_begin(P_HASH, st, m1);
        launch_hash(st);
        mark_end(st, m1);
        mark_begin(P_DETECT, st, m2);
        launch_detect(st);
        mark_end(st, m2);
        mark_begin(P_LINK, st, m3);
        launch_link(st);
        mark_end(st, m3);
    }

    // snapshot on the force stream, detection of the next list on the detection stream
    void start_detect()
    {
        Mark m1, m2;
        mark_begin(P_HASH, sf_, m1);
        launch_hash(sf_);
        mark_end(sf_, m1);
        cudaEventRecord(ev_snap_, sf_);
        cudaStreamWaitEvent(sd_, ev_snap_, 0);
        mark_begin(P_DETECT, sd_, m2);
        launch_detect(sd_);
        mark_end(sd_, m2);
        cudaEventRecord(ev_det_, sd_);
    }

    void finish_detect()
    {
        cudaStreamWaitEvent(sf_, ev_det_, 0);
        Mark m;
        mark_begin(P_LINK, sf_, m);
        launch_link(sf_);
        mark_end(sf_, m);
    }

    // The time step runs k_contact persistently over the compacted work of the list: as
    // many blocks as the SMs hold at once, never more than the slots need.
    template <int MODE>
    void launch_force(double *eF, double *eT)
    {
        const int b = tune_.contact_block;
        unsigned g = grid(d_.N, b);
        if (MODE == MODE_STEP) {
            const unsigned cap = (unsigned)contact_per_sm(b) * (unsigned)n_sm_;
            g = std::min(g, std::max(1u, cap));
        }
        const bool lean = MODE == MODE_STEP && tune_.contact_lean;
        if (m_.model == FORCE_MODEL_HERTZ_MINDLIN) {
            if (m_.clumps) k_contact<F, true, MODE, 0, false, FORCE_MODEL_HERTZ_MINDLIN><<<g, b, 0, sf_>>>(d_, eF, eT);
            else k_contact<F, false, MODE, 0, false, FORCE_MODEL_HERTZ_MINDLIN><<<g, b, 0, sf_>>>(d_, eF, eT);
            return;
        }
        if (m_.model == FORCE_MODEL_BONDED_BREAKAGE) {
            if (m_.clumps) k_contact<F, true, MODE, 0, false, FORCE_MODEL_BONDED_BREAKAGE><<<g, b, 0, sf_>>>(d_, eF, eT);
            else k_contact<F, false, MODE, 0, false, FORCE_MODEL_BONDED_BREAKAGE><<<g, b, 0, sf_>>>(d_, eF, eT);
            return;
        }
        if (m_.rolling) {
            // rolling resistance: its own build of the kernel (the others carry none of it)
            if (m_.clumps) k_contact<F, true, MODE, 0, true><<<g, b, 0, sf_>>>(d_, eF, eT);
            else k_contact<F, false, MODE, 0, true><<<g, b, 0, sf_>>>(d_, eF, eT);
            return;
        }
        if (m_.clumps) {
            if (lean) k_contact<F, true, MODE_STEP, 1><<<g, b, 0, sf_>>>(d_, eF, eT);
            else k_contact<F, true, MODE><<<g, b, 0, sf_>>>(d_, eF, eT);
        } else if (MODE == MODE_STEP && integ()) {
            if (lean) k_contact<F, false, MODE_STEP, 1, false, FORCE_MODEL_BUILTIN, true><<<g, b, 0, sf_>>>(d_, eF, eT);
            else k_contact<F, false, MODE_STEP, 0, false, FORCE_MODEL_BUILTIN, true><<<g, b, 0, sf_>>>(d_, eF, eT);
        } else if (MODE == MODE_STEP && screen()) {
            k_contact_screen<F><<<(unsigned)screen_per_sm() * (unsigned)n_sm_, SCREEN_BLOCK, 0, sf_>>>(d_);
            Mark me;                         // the evaluation pass, within the contact phase's mark
            mark_begin(P_EVAL, sf_, me);
            k_contact_eval<F><<<(unsigned)eval_per_sm(b) * (unsigned)n_sm_, b, 0, sf_>>>(d_);
            mark_end(sf_, me);
        } else {
            if (lean) k_contact<F, false, MODE_STEP, 1><<<g, b, 0, sf_>>>(d_, eF, eT);
            else k_contact<F, false, MODE><<<g, b, 0, sf_>>>(d_, eF, eT);
        }
    }

    // resident blocks per SM of the two passes of the two-pass contact step
    int screen_per_sm()
    {
        if (screen_occ_ > 0) return screen_occ_;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_contact_screen<F>, SCREEN_BLOCK, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        return screen_occ_ = per_sm;
    }
    int eval_per_sm(int b)
    {
        if (b == eval_occ_block_) return eval_occ_;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_contact_eval<F>, b, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        eval_occ_block_ = b;
        return eval_occ_ = per_sm;
    }

    int contact_per_sm(int b)
    {
        const int key = b * 4 + (tune_.contact_lean ? 1 : 0) + (integ() ? 2 : 0);
        if (key == occ_block_) return occ_per_sm_;
        int per_sm = 0;
        cudaError_t e;
        if (integ())
            e = tune_.contact_lean
                    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          &per_sm, k_contact<F, false, MODE_STEP, 1, false, FORCE_MODEL_BUILTIN, true>, b, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          &per_sm, k_contact<F, false, MODE_STEP, 0, false, FORCE_MODEL_BUILTIN, true>, b, 0);
        else if (m_.model == FORCE_MODEL_HERTZ_MINDLIN)
            e = m_.clumps ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                &per_sm, k_contact<F, true, MODE_STEP, 0, false, FORCE_MODEL_HERTZ_MINDLIN>, b, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                &per_sm, k_contact<F, false, MODE_STEP, 0, false, FORCE_MODEL_HERTZ_MINDLIN>, b, 0);
        else if (m_.model == FORCE_MODEL_BONDED_BREAKAGE)
            e = m_.clumps ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                &per_sm, k_contact<F, true, MODE_STEP, 0, false, FORCE_MODEL_BONDED_BREAKAGE>, b, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                &per_sm, k_contact<F, false, MODE_STEP, 0, false, FORCE_MODEL_BONDED_BREAKAGE>, b, 0);
        else if (m_.rolling)
            e = m_.clumps
                    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_contact<F, true, MODE_STEP, 0, true>, b, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_contact<F, false, MODE_STEP, 0, true>, b, 0);
        else if (tune_.contact_lean)
            e = m_.clumps ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_contact<F, true, MODE_STEP, 1>, b, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_contact<F, false, MODE_STEP, 1>, b, 0);
        else
            e = m_.clumps ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_contact<F, true, MODE_STEP>, b, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_contact<F, false, MODE_STEP>, b, 0);
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        occ_block_ = key;
        occ_per_sm_ = per_sm;
        return per_sm;
    }

    // Plain: one thread per owner.  Staged (voxel form): a persistent grid of as many
    // blocks as the SMs hold streams tiles of owners through shared memory.
    void launch_integrate()
    {
        const int ib = tune_.integrate_block;
        if (integ()) {
            // owners with listed partners were integrated by the contact kernel
            k_integrate<F, false, true><<<grid(d_.M, ib), ib, 0, sf_>>>(d_);
            return;
        }
        if constexpr (F::voxel) {
            if (tune_.integrate_staged && d_.M > 0 && staged_per_sm_ > 0) {
                const int smem = STAGES * StageLayout::bytes;
                const int64_t ntiles = (d_.M + ITILE - 1) / ITILE;
                const unsigned g = (unsigned)std::min<int64_t>(ntiles, (int64_t)staged_per_sm_ * n_sm_);
                if (m_.clumps) k_integrate_staged<true><<<g, ITILE, smem, sf_>>>(d_);
                else k_integrate_staged<false><<<g, ITILE, smem, sf_>>>(d_);
                return;
            }
        }
        if (m_.clumps) k_integrate<F, true><<<grid(d_.M, ib), ib, 0, sf_>>>(d_);
        else k_integrate<F, false><<<grid(d_.M, ib), ib, 0, sf_>>>(d_);
    }

    // Single spheres with the fused step chosen: one kernel for forces and integration.
    bool fused() const { return !m_.clumps && !m_.rolling && m_.model == FORCE_MODEL_BUILTIN && tune_.fused_block > 0; }
    // Single spheres, two-kernel step: contacts in two passes (screening, evaluation).
    bool screen() const
    {
        return !m_.clumps && !m_.rolling && m_.model == FORCE_MODEL_BUILTIN && tune_.fused_block == 0 &&
               !tune_.contact_integrates && tune_.contact_screen;
    }
    // Single spheres, two-kernel step: the contact kernel integrates the owners it holds.
    bool integ() const
    {
        return !m_.clumps && !m_.rolling && m_.model == FORCE_MODEL_BUILTIN && tune_.fused_block == 0 &&
               tune_.contact_integrates;
    }

    // Contact wildcards of the world's contact model (4: those of the history vector).
    int model_wildcards() const
    {
        return m_.model == FORCE_MODEL_BONDED_BREAKAGE ? ModelBondedBreakage::n_wildcards : 4;
    }
    unsigned model_odd() const
    {
        return m_.model == FORCE_MODEL_BONDED_BREAKAGE ? ModelBondedBreakage::odd : ModelHertzMindlin::odd;
    }

    void force_step()
    {
        if (fused()) {
            Mark m;
            mark_begin(P_FORCE, sf_, m);
            const int b = tune_.fused_block;
            k_step_fused<F><<<grid(d_.Np, b), b, 0, sf_>>>(d_);
            mark_end(sf_, m);
        } else {
            Mark m, m2;
            mark_begin(P_FORCE, sf_, m);
            launch_force<MODE_STEP>(nullptr, nullptr);
            mark_end(sf_, m);
            mark_begin(P_INTEG, sf_, m2);
            launch_integrate();
            mark_end(sf_, m2);
        }
        k_audit<<<1, 32, 0, sf_>>>(st_, d_.audit);
        pose_facets(sf_);
        if (collect_ && d_.M > 0)
            k_collect_step<F><<<grid(d_.M, 256), 256, 0, sf_>>>(d_, acc_lab_, obin_, cross_, win_start_, (float)beta_);
    }

    // Steps per list for the delayed schedules.  A list built from a snapshot at step s is
    // used from s + c to s + 2c, so its margin must cover 2c steps of motion; the
    // velocity bound uses the largest speed seen (with a 50% allowance for acceleration).
    long long cycle_length()
    {
        const double h = m_.scenes.empty() ? 1e-6 : m_.scenes[0].h;
        double v = std::max(sth_->vmax_last, 1e-3) * 1.5;
        // the audit also counts a fixed slack per step (the position rounding of the voxel
        // form and the largest facet displacement of a turning mesh): a cycle longer than
        // the margin allows for that alone would always end in a fallback
        const double slack = sth_->disp_slack;
        long long c = (long long)std::floor(beta_ / (2.0 * (h * v + slack)));
        if (m_.schedule == DEM_SCHEDULE_LEARNED) {
            std::string err;
            long long lc = learned_cycle(err);
            if (lc > 0) c = slack > 0.0 ? std::min<long long>(lc, (long long)std::floor(beta_ / (2.0 * slack))) : lc;
        }
        // a cycle cut short by the audit shrinks the next ones (x0.6); cycles that run to
        // their end let the factor recover (x1.1 up to 1): fewer inline fallback rebuilds
        // where the motion outgrows the bound, no change where it does not
        c = (long long)std::floor((double)c * cycle_scale_);
        cycle_scale_ = std::min(1.0, cycle_scale_ * 1.1);
        // at most 512 steps a cycle: a captured cycle graph stays a few thousand nodes
        last_cycle_ = std::max<long long>(1, std::min<long long>(c, 512));
        return last_cycle_;
    }
    long long last_cycle_ = 0;
    double cycle_scale_ = 1.0;

    void release()
    {
        drop_graphs();
        if (sf_) cudaStreamSynchronize(sf_);
        if (sd_) cudaStreamSynchronize(sd_);
        std::vector<void *> a = allocs_;
        for (void *p : a) dfree(p);
        allocs_.clear();
        if (sth_) cudaFreeHost(sth_);
        sth_ = nullptr;
        for (auto &m : marks_) pool_.push_back(m);
        marks_.clear();
        for (auto &m : pool_) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
        pool_.clear();
        if (ev_snap_) cudaEventDestroy(ev_snap_);
        if (ev_det_) cudaEventDestroy(ev_det_);
        if (ev_a_) cudaEventDestroy(ev_a_);
        if (ev_b_) cudaEventDestroy(ev_b_);
        if (ev_c_) cudaEventDestroy(ev_c_);
        if (ev_up_) cudaEventDestroy(ev_up_);
        ev_snap_ = ev_det_ = ev_a_ = ev_b_ = ev_c_ = ev_up_ = nullptr;
        if (sc_) cudaStreamDestroy(sc_);
        sc_ = nullptr;
        if (own_sf_ && sf_) cudaStreamDestroy(sf_);
        if (own_sd_ && sd_) cudaStreamDestroy(sd_);
        sf_ = sd_ = nullptr;
    }

    HostModel m_;
    Dev<F> d_{};
    Wall *walls_dev_ = nullptr;     // the walls (mesh facets' current pose written each step)
    double mesh_slack_ = 0.0;       // largest facet displacement per step
    DetectBuffers db_{};
    DevStatus *st_ = nullptr;
    DevStatus *sth_ = nullptr;
    cudaStream_t sf_ = nullptr, sd_ = nullptr, sc_ = nullptr;
    bool own_sf_ = false, own_sd_ = false;
    cudaEvent_t ev_snap_ = nullptr, ev_det_ = nullptr, ev_a_ = nullptr, ev_b_ = nullptr, ev_c_ = nullptr,
                ev_up_ = nullptr;
    std::vector<void *> allocs_;
    double *scratch_ = nullptr;
    int64_t scratch_n_ = 0;
    double beta_ = 0.0;
    bool dirty_ = false;
    int64_t fallbacks_ = 0, regrows_ = 0;
    double ms_total_ = 0.0;
    dem_tuning tune_{64, 256, 128, 0, 0.0, 1.0, 0, 0, 0};   // fused_block last: the two-kernel step
    int n_sm_ = 1, occ_block_ = 0, occ_per_sm_ = 1;
    int screen_occ_ = 0, eval_occ_block_ = 0, eval_occ_ = 1;
    int64_t Mp_ = 0;                // owners rounded up to whole staging tiles
    int staged_per_sm_ = 0;
    bool act_alloc_ = false;
    bool graphs_on_ = true;
    struct GraphEntry { long long c; cudaGraphExec_t exec; };
    std::vector<GraphEntry> graphs_;
    // learned schedule
    std::unique_ptr<Mlp> mlp_;
    float *bin_stats_ = nullptr, *X_ = nullptr, *pred_ = nullptr, *predmin_ = nullptr, *acc_lab_ = nullptr;
    int *obin_ = nullptr, *valid_ = nullptr, *bin_scene_ = nullptr, *cross_ = nullptr;
    bool collect_ = false;
    long long win_start_ = -1;
    int win_len_ = 256;
    std::vector<float> win_x_;
    std::vector<int> win_valid_;
    std::vector<float> ds_x_, ds_y_;
    // profiling: event pairs recorded on the stream of the bracketed work
    enum { P_FORCE = 0, P_DETECT = 1, P_HASH = 2, P_LINK = 3, P_INTEG = 4, P_EVAL = 5, P_KINDS = 6 };
    bool prof_ = false;
    struct Mark { cudaEvent_t a, b; int kind; };
    std::vector<Mark> marks_, pool_;
    double prof_ms_[P_KINDS] = {};
    int64_t prof_n_[P_KINDS] = {};

    Mark take()
    {
        if (pool_.empty()) {
            Mark m{};
            cudaEventCreate(&m.a);
            cudaEventCreate(&m.b);
            return m;
        }
        Mark m = pool_.back();
        pool_.pop_back();
        return m;
    }
    void mark_begin(int kind, cudaStream_t st, Mark &m)
    {
        if (!prof_) return;
        m = take();
        m.kind = kind;
        cudaEventRecord(m.a, st);
    }
    void mark_end(cudaStream_t st, Mark &m)
    {
        if (!prof_) return;
        cudaEventRecord(m.b, st);
        marks_.push_back(m);
    }
    // called after a synchronisation: every recorded event has completed
    void harvest()
    {
        for (auto &m : marks_) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
                prof_ms_[m.kind] += ms;
                prof_n_[m.kind] += 1;
            }
            pool_.push_back(m);
        }
        marks_.clear();
        cudaGetLastError();
    }
};

}  // namespace dem
