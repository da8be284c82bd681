// force_models.cuh -- contact force models as compile-time device functors.
//
// The paper lets users replace the default contact model with their own (Sec. 4.2,
// "Providing a custom contact force model"): a model reads a fixed set of per-contact
// variables (the user-referable variables of Sec. 4.2's table), keeps its own per-contact
// state in "contact wildcards" (zero when a contact appears, dropped when it vanishes),
// and writes the force on body A and a torque-only force.  The paper compiles such a
// model just in time; here a model is a struct compiled into its own build of the
// contact kernel (the model's type is a template argument), so the step carries no
// branching or indirection for it.
//
// A model provides:
//   static constexpr int n_params;        // length of its parameter array
//   static constexpr unsigned odd;        // wildcards that change sign with the side (bit k)
//   static bool engaged(const Referables<R> &c, const R wc[8], const R *par)
//                                         // does the pair interact this step?
//   static void eval(const Referables<R> &c, R wc[8], const R *par, V3<R> &F, V3<R> &Fr)
//                                         // force on A, torque-only force on A, wildcards
// Wildcards 0..3 live in the entry's history vector, 4..7 in the world's second
// wildcard array (allocated when a model has more than four).  Every pair is evaluated
// with A the lower sphere id on both of its sides (the kernel swaps roles and negates
// the odd wildcards on the upper side), so a model need not be symmetric in A and B.
#pragma once
#include "common.cuh"
#include "contact.cuh"

namespace dem {

// The user-referable variables of one contact (Sec. 4.2's table), global frame.
template <typename R>
struct Referables {
    V3<R> B2A;              // unit vector from B to A
    R overlapDepth;         // R_A + R_B - |x_A - x_B| (negative across a gap)
    R ts;                   // time step
    V3<R> locCPA, locCPB;   // contact point relative to each owner's centre of mass
    V3<R> ALinVel, BLinVel; // owners' linear velocities
    V3<R> ARotVel, BRotVel; // owners' angular velocities
    V3<R> velB2A;           // velocity of the contact point on A relative to on B
    R AOwnerMass, BOwnerMass;
    R ARadius, BRadius;
    R Rbar, mbar;           // effective radius and mass
    int AMat, BMat;         // global material ids
    int AFamily, BFamily;   // family tags (0 without families)
    uint32_t AGeo, BGeo;    // sphere slots
    // pairwise material constants (host-combined: Hertz-Mindlin E*, G*, damping ratio of
    // the pair's restitution, friction, rolling resistance, mean Poisson ratio)
    R Estar, Gstar, beta, mu, crr, nu;
};

// The default model (Sec. 4.2.1: history-based Hertz-Mindlin with Coulomb capping and
// rolling resistance) through the functor interface.  Wildcards: the tangential
// displacement (0..2, odd) and the contact's age (3).  It computes exactly what the
// built-in kernel computes, so a world can be checked bit for bit against it.
struct ModelHertzMindlin {
    static constexpr int n_params = 0;
    static constexpr int n_wildcards = 4;
    static constexpr unsigned odd = 0x7u;
    template <typename R>
    __device__ static bool engaged(const Referables<R> &c, const R *, const R *)
    {
        return c.overlapDepth > R(0);
    }
    template <typename R>
    __device__ static void eval(const Referables<R> &c, R *wc, const R *, V3<R> &F, V3<R> &Fr)
    {
        ContactIn<R> ci;
        ci.n = c.B2A;
        ci.delta = c.overlapDepth;
        ci.uA = c.velB2A;
        ci.uB = V3<R>{R(0), R(0), R(0)};
        ci.Rbar = c.Rbar;
        ci.mbar = c.mbar;
        ci.Estar = c.Estar; ci.Gstar = c.Gstar; ci.beta = c.beta; ci.mu = c.mu;
        V3<R> ut = {wc[0], wc[1], wc[2]};
        R fn_abs;
        hertz_mindlin<R>(ci, c.ts, ut, F, &fn_abs);
        wc[0] = ut.x; wc[1] = ut.y; wc[2] = ut.z;
        wc[3] = radd(wc[3], c.ts);
        Fr = V3<R>{R(0), R(0), R(0)};
        if (c.crr > R(0) && !within_collision_time<R>(ci, wc[3])) {
            const V3<R> rotA = {rsub(rmul(c.ARotVel.y, c.locCPA.z), rmul(c.ARotVel.z, c.locCPA.y)),
                                rsub(rmul(c.ARotVel.z, c.locCPA.x), rmul(c.ARotVel.x, c.locCPA.z)),
                                rsub(rmul(c.ARotVel.x, c.locCPA.y), rmul(c.ARotVel.y, c.locCPA.x))};
            const V3<R> rotB = {rsub(rmul(c.BRotVel.y, c.locCPB.z), rmul(c.BRotVel.z, c.locCPB.y)),
                                rsub(rmul(c.BRotVel.z, c.locCPB.x), rmul(c.BRotVel.x, c.locCPB.z)),
                                rsub(rmul(c.BRotVel.x, c.locCPB.y), rmul(c.BRotVel.y, c.locCPB.x))};
            Fr = rolling_force<R>(c.crr, fn_abs,
                                  V3<R>{rsub(rotB.x, rotA.x), rsub(rotB.y, rotA.y), rsub(rotB.z, rotA.z)});
        }
    }
};

// The bonded, breakable contact of Sec. 6.3 (the paper's worked custom model for brittle
// solids).  Parameters: par[0] tensile strength sigma_t (Pa, negative: tension),
// par[1] cohesion c (Pa), par[2] bending coefficient eta, par[3] normal damping factor.
// Wildcards: tangential displacement (0..2, odd), age (3), bond state (4: > 1e-12
// bonded, -1 broken), bond length (5: the overlap at which the bond carries no load).
// A bonded pair interacts whatever the sign of its overlap; once broken, it is a
// Hertz-Mindlin contact while the spheres overlap.  With D = overlap - bond length,
// k_n = E* Rbar, area A = pi max(R_A, R_B)^2, D_y = sigma_t A / k_n, D_u = 3 D_y:
//   normal  k_n D above D_y, softening linearly to zero at D_u (slope -k_n / 2),
//           damped by par[3] sqrt(mbar k_n) times the normal relative velocity; the
//           bond breaks once D < D_u;
//   shear   k_t = nu k_n, F_t = -k_t ut - g_t v_t with g_t = -2 sqrt(5/6) beta
//           sqrt(mbar k_t) (the default model's history and damping); the bond breaks
//           once |F_t| > mu |F| + c A (c A only while D > D_y);
//   bending a torque-only force of magnitude min(h R_A R_B k_t / R_A, eta |F|) along the
//           rolling part of B's contact-point velocity relative to A's.
struct ModelBondedBreakage {
    static constexpr int n_params = 4;
    static constexpr int n_wildcards = 6;
    static constexpr unsigned odd = 0x7u;
    template <typename R>
    __device__ static bool engaged(const Referables<R> &c, const R *wc, const R *)
    {
        return wc[4] > R(1e-12) || c.overlapDepth > R(0);
    }
    template <typename R>
    __device__ static void eval(const Referables<R> &c, R *wc, const R *par, V3<R> &F, V3<R> &Fr)
    {
        if (!(wc[4] > R(1e-12))) {
            ModelHertzMindlin::eval<R>(c, wc, nullptr, F, Fr);
            return;
        }
        const R c56 = R(0.91287092917527690);   // sqrt(5/6)
        const V3<R> n = c.B2A;
        const V3<R> u = c.velB2A;
        const R proj = dot(u, n);
        const V3<R> vt = u - proj * n;
        V3<R> ut = {wc[0], wc[1], wc[2]};
        ut = ut + c.ts * vt;
        const R up = dot(ut, n);
        ut = ut - up * n;
        wc[0] = ut.x; wc[1] = ut.y; wc[2] = ut.z;
        wc[3] = radd(wc[3], c.ts);

        const R D = c.overlapDepth - wc[5];
        const R kn = c.Estar * c.Rbar;
        const R Rm = c.ARadius > c.BRadius ? c.ARadius : c.BRadius;
        const R area = R(3.14159265358979323846) * (Rm * Rm);
        const R Dy = (par[0] * area) / kn;
        const R Du = R(3) * Dy;
        const R fn = D > Dy ? kn * D : R(0.5) * kn * (Du - D);
        const R gn = par[3] * sqrt(c.mbar * kn);
        F = (fn - gn * proj) * n;
        if (D < Du) wc[4] = R(-1);

        const R kt = c.nu * kn;
        const R gt = R(-2) * c56 * c.beta * sqrt(c.mbar * kt);
        const R fs_max = sqrt(dot(F, F)) * c.mu + (D > Dy ? par[1] * area : R(0));
        const V3<R> Ft = (-kt) * ut - gt * vt;
        if (sqrt(dot(Ft, Ft)) > fs_max) wc[4] = R(-1);
        F = F + Ft;

        Fr = V3<R>{R(0), R(0), R(0)};
        const V3<R> rotA = cross(c.ARotVel, c.locCPA), rotB = cross(c.BRotVel, c.locCPB);
        const V3<R> vr = rotB - rotA;
        const R vm = sqrt(dot(vr, vr));
        if (vm > R(1e-12)) {
            const R kr = (c.ARadius * c.BRadius) * kt;
            const R m1 = (c.ts * kr) / c.ARadius, m2 = par[2] * sqrt(dot(F, F));
            Fr = ((m1 < m2 ? m1 : m2) / vm) * vr;
        }
    }
};

enum : int { FORCE_MODEL_BUILTIN = 0, FORCE_MODEL_HERTZ_MINDLIN = 1, FORCE_MODEL_BONDED_BREAKAGE = 2 };
constexpr int MODEL_MAX_PARAMS = 8;

}  // namespace dem
