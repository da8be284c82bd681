// contact.cuh -- per-contact physics of the default DEM-Engine force model.
//
// The history-based Hertz-Mindlin model of arXiv 2311.04648 Sec. 4.1 (Eqs. 1-4) in the
// form the default model of Sec. 4.2.1 evaluates it:
//   Sn = 2 E* sqrt(Rbar delta), k_n = 2/3 Sn, gamma_n = 2 sqrt(5/6) beta sqrt(Sn mbar),
//   u = relative contact-point velocity of A w.r.t. B, v_t = u - (u.n) n,
//   history: ut <- ut + h v_t, then ut <- ut - (ut.n) n   (update precedes the force),
//   F = (k_n delta + gamma_n u.n) n,
//   k_t = 8 G* sqrt(Rbar delta), g_t = -2 sqrt(5/6) beta sqrt(mbar k_t),
//   F_t = -k_t ut - g_t v_t; if |F_t| > mu |F| (and |F_t| > 1e-12): F_t scaled to mu |F|
//   and ut back-solved as (F_t + g_t v_t) / (-k_t); |F_t| <= 1e-12 gives F_t = 0.
// beta = ln e / sqrt(ln^2 e + pi^2) (e clamped at 1e-12) is precomputed on the host per
// material pair.  Rolling resistance (rolling_force) follows the same listing: once a
// contact has lasted longer than a collision time, a force of C_r |F_n| along the
// rolling part of the contact point's relative velocity, acting only through torques.
#pragma once
#include "common.cuh"

namespace dem {

template <typename R>
struct ContactIn {
    V3<R> n;          // unit normal from B to A
    R delta;          // overlap > 0
    V3<R> uA, uB;     // velocities of the contact point as a point of A and of B
    R Rbar, mbar;
    R Estar, Gstar, beta, mu;
};

template <typename R>
__device__ __forceinline__ void hertz_mindlin(const ContactIn<R> &c, R h, V3<R> &ut, V3<R> &F, R *fn_abs = nullptr)
{
    const R c56 = R(0.91287092917527690);   // sqrt(5/6)
    V3<R> u = c.uA - c.uB;
    R proj = dot(u, c.n);
    V3<R> vt = u - proj * c.n;
    ut = ut + h * vt;
    R up = dot(ut, c.n);
    ut = ut - up * c.n;

    R sqrtRd = sqrt(c.delta * c.Rbar);
    R Sn = R(2) * c.Estar * sqrtRd;
    R kn = (R(2) / R(3)) * Sn;
    R gn = R(2) * c56 * c.beta * sqrt(Sn * c.mbar);
    R fn = kn * c.delta + gn * proj;
    F = fn * c.n;
    if (fn_abs) *fn_abs = sqrt(radd(radd(rmul(F.x, F.x), rmul(F.y, F.y)), rmul(F.z, F.z)));
    if (c.mu > R(0)) {
        R kt = R(8) * c.Gstar * sqrtRd;
        R gt = R(-2) * c56 * c.beta * sqrt(c.mbar * kt);
        V3<R> Ft = (-kt) * ut - gt * vt;
        R ft = sqrt(dot(Ft, Ft));
        if (ft > R(1e-12)) {
            R ftmax = sqrt(dot(F, F)) * c.mu;
            if (ft > ftmax) {
                Ft = (ftmax / ft) * Ft;
                ut = (R(1) / (-kt)) * (Ft + gt * vt);
            }
        } else {
            Ft = mk(R(0), R(0), R(0));
        }
        F = F + Ft;
    }
}

// Whether a contact that has lasted `age` is still inside its first collision.  The
// default model of Sec. 4.2.1 forms a damped linear oscillator from E*, the damping
// ratio beta, mbar and Rbar in a simplified way and applies rolling resistance only
// after its collision time: with s = sqrt(Rbar), k = (4/3) E* sqrt(s) and
// g = -2 sqrt((5/3) mbar E*) beta s^(1/4), the damping ratio is z = g / (2 sqrt(k mbar))
// and, where z < 1 and 1 - z^2 > 0, the collision time is pi sqrt(mbar / (k (1 - z^2))).
// Every operation is rounded on its own in this order (the FP64 form decides exactly as
// an FP64 evaluation without fused multiply-adds), and the inputs are symmetric in the
// two bodies, so both sides of a pair decide alike.
template <typename R>
__device__ __forceinline__ bool within_collision_time(const ContactIn<R> &c, R age)
{
    const R s = sqrt(c.Rbar);
    const R k = rmul(rmul(R(4.0 / 3.0), c.Estar), sqrt(s));
    const R g = rmul(rmul(R(-2.0) * sqrt(rmul(rmul(R(5.0 / 3.0), c.mbar), c.Estar)), c.beta), sqrt(sqrt(s)));
    const R z = g / rmul(R(2), sqrt(rmul(k, c.mbar)));
    if (!(z < R(1))) return false;
    const R dz = rsub(R(1), rmul(z, z));
    if (!(dz > R(0))) return false;
    const R tc = rmul(R(3.14159265358979323846), sqrt(c.mbar / rmul(k, dz)));
    return age <= tc;
}

// Rolling-resistance force on A (Sec. 4.1, F_r and tau_r; Sec. 4.2.1): C_r |F_n| along
// vr = (rolling part of B's contact-point velocity) - (A's), i.e. w_B x r_B - w_A x r_A,
// where |vr| > 1e-12; zero otherwise.  It enters only A's torque (r_A x F_r); B's side,
// evaluated with the roles exchanged, obtains exactly -F_r.
template <typename R>
__device__ __forceinline__ V3<R> rolling_force(R crr, R fn_abs, V3<R> vr)
{
    const R vm = sqrt(radd(radd(rmul(vr.x, vr.x), rmul(vr.y, vr.y)), rmul(vr.z, vr.z)));
    if (!(vm > R(1e-12))) return V3<R>{R(0), R(0), R(0)};
    const R sc = rmul(crr, fn_abs) / vm;
    return V3<R>{rmul(sc, vr.x), rmul(sc, vr.y), rmul(sc, vr.z)};
}

// Error-free transformations in FP32 (Knuth's TwoSum; the product error from an FMA).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Overlap (Ra + Rb) - |pa - pb| of two voxel-form centres, evaluated in float-float so
// that it keeps ~2^-44 of the centre distance (the paper keeps the penetration in a
// wider type than the rest of the force arithmetic, Sec. 2.3); FP32 pipes only.  Also
// returns the rounded difference vector and distance for the rest of the contact.
__device__ __forceinline__ float overlap_ff(const PosF32 &a, const PosF32 &b, float Lv, float ra_hi, float ra_lo,
                                            float rb_hi, float rb_lo, V3<float> &dv, float &dist)
{
    const int ca[3] = {a.cx, a.cy, a.cz}, cb[3] = {b.cx, b.cy, b.cz};
    const float oa[3] = {a.x, a.y, a.z}, ob[3] = {b.x, b.y, b.z};
    float xs[3];
    float sh = 0.0f, sl = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float ax = __fmul_rn((float)(ca[k] - cb[k]), Lv);       // exact: small integer times 2^e
        float bh, bl;
        two_sum(oa[k], -ob[k], bh, bl);                          // exact offset difference
        float xh, xl;
        two_sum(ax, bh, xh, xl);
        xl = __fadd_rn(xl, bl);
        xs[k] = xh;
        float p = __fmul_rn(xh, xh);
        float pe = __fmaf_rn(xh, xh, -p);
        float t, te;
        two_sum(sh, p, t, te);
        sh = t;
        sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(te, pe), __fmul_rn(2.0f * xh, xl)));
    }
    float s2, e2;
    two_sum(sh, sl, s2, e2);
    float dh = __fsqrt_rn(s2);
    float res = __fadd_rn(__fmaf_rn(-dh, dh, s2), e2);           // s - dh^2, exact residual + low part
    float dl = __fdiv_rn(res, 2.0f * dh);
    float rh, rl;
    two_sum(ra_hi, rb_hi, rh, rl);
    rl = __fadd_rn(rl, __fadd_rn(ra_lo, rb_lo));
    dv = {xs[0], xs[1], xs[2]};
    dist = dh;
    return __fadd_rn(__fsub_rn(rh, dh), __fsub_rn(rl, dl));
}

__device__ __forceinline__ void load_pair(const PairParam *pairs, const PairParamF *, const uint16_t *mat_scene,
                                          const uint16_t *mat_local, const Scene *scenes, int ga, int gb,
                                          ContactIn<double> &c)
{
    const Scene &sc = scenes[mat_scene[ga]];
    const PairParam p = pairs[sc.pair_base + (int)mat_local[ga] * sc.n_mat + (int)mat_local[gb]];
    c.Estar = p.Estar;
    c.Gstar = p.Gstar;
    c.beta = p.beta;
    c.mu = p.mu;
}
__device__ __forceinline__ void load_pair(const PairParam *, const PairParamF *pairs, const uint16_t *mat_scene,
                                          const uint16_t *mat_local, const Scene *scenes, int ga, int gb,
                                          ContactIn<float> &c)
{
    const Scene &sc = scenes[mat_scene[ga]];
    const PairParamF p = pairs[sc.pair_base + (int)mat_local[ga] * sc.n_mat + (int)mat_local[gb]];
    c.Estar = p.Estar;
    c.Gstar = p.Gstar;
    c.beta = p.beta;
    c.mu = p.mu;
}

// FP32 screen of a plane: true if the centre may be within `reach` of the plane.  The
// allowance covers the rounding of the FP32 evaluation for coordinates of size `scale`.
__device__ __forceinline__ bool plane_may_reach(const Wall &w, float3 p, float reach, float scale)
{
    float g = (p.x - w.pf[0]) * w.nf[0] + (p.y - w.pf[1]) * w.nf[1] + (p.z - w.pf[2]) * w.nf[2];
    return g <= reach + 1e-5f * scale + 1e-9f;
}

// The signed gap of wall_gap evaluated in FP32 from an FP32 centre, for screening: it
// differs from the FP64 gap by less than wall_gap_tol, so a comparison with a threshold
// that clears the threshold by more than that is decided the same way as in FP64.
__device__ __forceinline__ float wall_gap_f(const Wall &w, float3 c)
{
    const float dx = c.x - w.pf[0], dy = c.y - w.pf[1], dz = c.z - w.pf[2];
    const float z = dx * w.nf[0] + dy * w.nf[1] + dz * w.nf[2];
    if (w.type == WALL_PLANE) return z;
    const float rx = dx - z * w.nf[0], ry = dy - z * w.nf[1], rz = dz - z * w.nf[2];
    const float rho = sqrtf(rx * rx + ry * ry + rz * rz);
    if (w.type == WALL_CYLINDER) return w.r0f - rho;
    const float dr = w.r1f - w.r0f, dzz = w.z1f - w.z0f;
    const float len2 = dr * dr + dzz * dzz;
    float t = ((rho - w.r0f) * dr + (z - w.z0f) * dzz) / len2;
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    const float Dr = rho - (w.r0f + t * dr), Dz = z - (w.z0f + t * dzz);
    const float dist = sqrtf(Dr * Dr + Dz * Dz);
    float inr = -dzz, inz = dr;            // inward normal of the generator, unnormalised
    if (inr > 0.0f) { inr = -inr; inz = -inz; }
    return (Dr * inr + Dz * inz) >= 0.0f ? dist : -dist;
}

__device__ __forceinline__ float wall_gap_tol(const Wall &w, float3 c)
{
    return w.tolf * (fabsf(c.x) + fabsf(c.y) + fabsf(c.z) + 1.0f) + 1e-9f;
}

// Point of the triangle (a, b, c) closest to p: the region tests of the published
// closest-point-on-triangle algorithm (vertex, edge and face regions by the signs of
// barycentric-coordinate numerators), every product and sum rounded on its own in the
// written order.
__device__ __forceinline__ V3<double> closest_on_triangle(V3<double> p, V3<double> a, V3<double> b, V3<double> c)
{
    auto sub = [](V3<double> u, V3<double> v) { return V3<double>{rsub(u.x, v.x), rsub(u.y, v.y), rsub(u.z, v.z)}; };
    auto dt = [](V3<double> u, V3<double> v) { return radd(radd(rmul(u.x, v.x), rmul(u.y, v.y)), rmul(u.z, v.z)); };
    auto axpy = [](V3<double> u, double s, V3<double> v) {
        return V3<double>{radd(u.x, rmul(s, v.x)), radd(u.y, rmul(s, v.y)), radd(u.z, rmul(s, v.z))};
    };
    const V3<double> ab = sub(b, a), ac = sub(c, a), ap = sub(p, a), bp = sub(p, b), cp = sub(p, c);
    const double d1 = dt(ab, ap), d2 = dt(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) return a;
    const double d3 = dt(ab, bp), d4 = dt(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) return b;
    const double vc = rsub(rmul(d1, d4), rmul(d3, d2));
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) return axpy(a, __ddiv_rn(d1, rsub(d1, d3)), ab);
    const double d5 = dt(ab, cp), d6 = dt(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) return c;
    const double vb = rsub(rmul(d5, d2), rmul(d1, d6));
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) return axpy(a, __ddiv_rn(d2, rsub(d2, d6)), ac);
    const double va = rsub(rmul(d3, d6), rmul(d5, d4));
    const double e43 = rsub(d4, d3), e56 = rsub(d5, d6);
    if (va <= 0.0 && e43 >= 0.0 && e56 >= 0.0) return axpy(b, __ddiv_rn(e43, radd(e43, e56)), sub(c, b));
    const double den = __ddiv_rn(1.0, radd(radd(va, vb), vc));
    const double v = rmul(vb, den), w = rmul(vc, den);
    return V3<double>{radd(radd(a.x, rmul(ab.x, v)), rmul(ac.x, w)), radd(radd(a.y, rmul(ab.y, v)), rmul(ac.y, w)),
                      radd(radd(a.z, rmul(ab.z, v)), rmul(ac.z, w))};
}

// Signed gap of a sphere centre to a wall (positive on the domain side) and the unit
// normal from the wall to the centre; FP64, every product and sum rounded in a fixed
// order.  Returns false where the normal is undefined (centre on an axis).
__device__ __forceinline__ bool wall_gap(const Wall &w, V3<double> c, double &gap, V3<double> &n)
{
    if (w.type == WALL_TRIANGLE) {
        // a two-sided facet at its current pose: distance to its closest point
        const V3<double> q = closest_on_triangle(c, V3<double>{w.cur[0], w.cur[1], w.cur[2]},
                                                 V3<double>{w.cur[3], w.cur[4], w.cur[5]},
                                                 V3<double>{w.cur[6], w.cur[7], w.cur[8]});
        const V3<double> e = {rsub(c.x, q.x), rsub(c.y, q.y), rsub(c.z, q.z)};
        const double dist = __dsqrt_rn(radd(radd(rmul(e.x, e.x), rmul(e.y, e.y)), rmul(e.z, e.z)));
        gap = dist;
        if (!(dist > 0.0)) return false;
        n = {__ddiv_rn(e.x, dist), __ddiv_rn(e.y, dist), __ddiv_rn(e.z, dist)};
        return true;
    }
    V3<double> d = {rsub(c.x, w.p[0]), rsub(c.y, w.p[1]), rsub(c.z, w.p[2])};
    double z = radd(radd(rmul(d.x, w.n[0]), rmul(d.y, w.n[1])), rmul(d.z, w.n[2]));
    if (w.type == WALL_PLANE) {
        gap = z;
        n = {w.n[0], w.n[1], w.n[2]};
        return true;
    }
    V3<double> rp = {rsub(d.x, rmul(z, w.n[0])), rsub(d.y, rmul(z, w.n[1])), rsub(d.z, rmul(z, w.n[2]))};
    double rho = __dsqrt_rn(radd(radd(rmul(rp.x, rp.x), rmul(rp.y, rp.y)), rmul(rp.z, rp.z)));
    if (w.type == WALL_CYLINDER) {
        gap = rsub(w.r0, rho);
        if (!(rho > 0.0)) return false;
        n = {-__ddiv_rn(rp.x, rho), -__ddiv_rn(rp.y, rho), -__ddiv_rn(rp.z, rho)};
        return true;
    }
    // cone segment in the (rho, z) half plane
    double dr = rsub(w.r1, w.r0), dz = rsub(w.z1, w.z0);
    double len2 = radd(rmul(dr, dr), rmul(dz, dz));
    double t = __ddiv_rn(radd(rmul(rsub(rho, w.r0), dr), rmul(rsub(z, w.z0), dz)), len2);
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    double cr = radd(w.r0, rmul(t, dr)), cz = radd(w.z0, rmul(t, dz));
    double Dr = rsub(rho, cr), Dz = rsub(z, cz);
    double dist = __dsqrt_rn(radd(rmul(Dr, Dr), rmul(Dz, Dz)));
    double len = __dsqrt_rn(len2);
    double inr = -__ddiv_rn(dz, len), inz = __ddiv_rn(dr, len);
    if (inr > 0.0) { inr = -inr; inz = -inz; }
    double side = radd(rmul(Dr, inr), rmul(Dz, inz));
    double sg = side >= 0.0 ? 1.0 : -1.0;
    gap = sg * dist;
    if (!(rho > 0.0) || !(dist > 0.0)) return false;
    double n2r = __ddiv_rn(sg * Dr, dist), n2z = __ddiv_rn(sg * Dz, dist);
    V3<double> er = {__ddiv_rn(rp.x, rho), __ddiv_rn(rp.y, rho), __ddiv_rn(rp.z, rho)};
    n = {radd(rmul(n2r, er.x), rmul(n2z, w.n[0])), radd(rmul(n2r, er.y), rmul(n2z, w.n[1])),
         radd(rmul(n2r, er.z), rmul(n2z, w.n[2]))};
    return true;
}

}  // namespace dem
