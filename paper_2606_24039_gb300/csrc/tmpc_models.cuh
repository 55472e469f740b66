// Model functions of the OCP family, evaluated by one thread per stage:
// dynamics residual f_t(z_t, z_{t+1}) with the Jacobian blocks A^-_t, A^+_t of
// Appendix B ("Equality constraints"), inequality functions g_t(z_t) with
// G_t = dg_t/dz_t ("Inequality constraints"), and the explicit / Newton
// rollout step used for the initial guess of Algorithm 1.
//
// Implicit dynamics follow Remark A1 / Remark 2 of the paper: the racing
// model keeps A^+_t != [-I 0] (implicit midpoint rule), which preserves the
// block-bidiagonal C and the block-tridiagonal S.
#pragma once
#include <math.h>
#include <stdint.h>

namespace tmpc {

enum { MODEL_DI = 0, MODEL_LINEAR = 1, MODEL_BICYCLE = 2, MODEL_QUAD = 3, MODEL_BICYCLE_TRAP = 4,
       MODEL_BICYCLE_NEWTON = 5, MODEL_SRB = 6, MODEL_COUNT = 7 };

// the kinematic bicycle under its three time discretisations (Remark A1): implicit
// midpoint, trapezoidal, and the explicit map defined by Newton steps on the midpoint rule
__host__ __device__ inline bool is_bicycle(int m) {
    return m == MODEL_BICYCLE || m == MODEL_BICYCLE_TRAP || m == MODEL_BICYCLE_NEWTON;
}
constexpr int kNewtonMapSteps = 3;   // Newton steps that define the explicit map of MODEL_BICYCLE_NEWTON

struct ModelDims {
    int nx, nu, ng;
};

__host__ __device__ inline ModelDims model_dims(int model, int lnx, int lnu, int lng) {
    switch (model) {
        case MODEL_DI: return {4, 2, 4};
        case MODEL_BICYCLE:
        case MODEL_BICYCLE_TRAP:
        case MODEL_BICYCLE_NEWTON: return {6, 2, 5};
        case MODEL_QUAD: return {6, 2, 2};
        case MODEL_SRB: return {12, 6, 6};
        default: return {lnx, lnu, lng};
    }
}

// Am / Ap / G blocks identical for every stage -> stored once (stage stride 0)
__host__ __device__ inline bool model_const_Am(int m) { return m == MODEL_DI || m == MODEL_LINEAR; }
__host__ __device__ inline bool model_const_Ap(int m) { return m != MODEL_BICYCLE && m != MODEL_BICYCLE_TRAP; }
__host__ __device__ inline bool model_const_G(int m) { return !is_bicycle(m); }
__host__ __device__ inline bool model_linear_dyn(int m) { return m == MODEL_DI || m == MODEL_LINEAR; }

// ---------------------------------------------------------------------------
// racing centreline: periodic table (x_c, y_c, psi_c, kappa) every ds metres,
// cubic Hermite interpolation with knot derivatives (cos psi, sin psi, kappa)
// ---------------------------------------------------------------------------
// math of either precision (the FP32 forward and the FP64 Jacobians of the direct backward)
__device__ __forceinline__ void msincos(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void msincos(double a, double* s, double* c) { sincos(a, s, c); }
__device__ __forceinline__ float mfloor(float a) { return floorf(a); }
__device__ __forceinline__ double mfloor(double a) { return floor(a); }
__device__ __forceinline__ float mtan(float a) { return tanf(a); }
__device__ __forceinline__ double mtan(double a) { return tan(a); }
__device__ __forceinline__ float mcos(float a) { return cosf(a); }
__device__ __forceinline__ double mcos(double a) { return cos(a); }

template <class R>
struct TrackPtR {
    R xc, yc, psic, dxc, dyc, dpsic;
};
using TrackPt = TrackPtR<float>;

template <class R>
__device__ __forceinline__ TrackPtR<R> track_eval(const float* tab, int nt, R ds, R s) {
    const R L = nt * ds;
    R sm = s - L * mfloor(s / L);
    int k = (int)mfloor(sm / ds);
    k = k < 0 ? 0 : (k > nt - 1 ? nt - 1 : k);
    const R tau = (sm - k * ds) / ds;
    const float* a = tab + 4 * k;
    const float* b = a + 4;
    const R t2 = tau * tau, t3 = t2 * tau;
    const R h00 = R(2) * t3 - R(3) * t2 + R(1), h10 = t3 - R(2) * t2 + tau;
    const R h01 = R(-2) * t3 + R(3) * t2, h11 = t3 - t2;
    const R d00 = R(6) * t2 - R(6) * tau, d10 = R(3) * t2 - R(4) * tau + R(1);
    const R d01 = R(-6) * t2 + R(6) * tau, d11 = R(3) * t2 - R(2) * tau;
    R sa, ca, sb, cb;
    msincos((R)a[2], &sa, &ca);
    msincos((R)b[2], &sb, &cb);
    TrackPtR<R> p;
    p.xc = h00 * a[0] + h10 * ds * ca + h01 * b[0] + h11 * ds * cb;
    p.yc = h00 * a[1] + h10 * ds * sa + h01 * b[1] + h11 * ds * sb;
    p.psic = h00 * a[2] + h10 * ds * a[3] + h01 * b[2] + h11 * ds * b[3];
    p.dxc = (d00 * a[0] + d10 * ds * ca + d01 * b[0] + d11 * ds * cb) / ds;
    p.dyc = (d00 * a[1] + d10 * ds * sa + d01 * b[1] + d11 * ds * sb) / ds;
    p.dpsic = (d00 * a[2] + d10 * ds * a[3] + d01 * b[2] + d11 * ds * b[3]) / ds;
    return p;
}

// kinematic bicycle: state (px, py, psi, v, delta, s), control (a, steer rate);
// ds/dt = v cos(psi - psi_c(s)).  Jx [6][6], Ju [6][2] row-major (nullable).
template <class R>
__device__ __forceinline__ void bicycle_fc(const R* x, const R* u, float Lf, const float* tab, int nt, float ds,
                                           R* f, R* Jx, R* Ju) {
    const R L = (R)Lf;
    const R psi = x[2], v = x[3], dl = x[4], s = x[5];
    TrackPtR<R> tp = track_eval<R>(tab, nt, (R)ds, s);
    R sp, cp;
    msincos(psi, &sp, &cp);
    const R tn = mtan(dl);
    R sd, cd;
    msincos(psi - tp.psic, &sd, &cd);
    f[0] = v * cp;
    f[1] = v * sp;
    f[2] = v * tn / L;
    f[3] = u[0];
    f[4] = u[1];
    f[5] = v * cd;
    if (Jx) {
        for (int i = 0; i < 36; ++i) Jx[i] = R(0);
        const R cdl = mcos(dl);
        Jx[0 * 6 + 2] = -v * sp;
        Jx[0 * 6 + 3] = cp;
        Jx[1 * 6 + 2] = v * cp;
        Jx[1 * 6 + 3] = sp;
        Jx[2 * 6 + 3] = tn / L;
        Jx[2 * 6 + 4] = v / (L * cdl * cdl);
        Jx[5 * 6 + 2] = -v * sd;
        Jx[5 * 6 + 3] = cd;
        Jx[5 * 6 + 5] = v * sd * tp.dpsic;
    }
    if (Ju) {
        for (int i = 0; i < 12; ++i) Ju[i] = R(0);
        Ju[3 * 2 + 0] = R(1);
        Ju[4 * 2 + 1] = R(1);
    }
}

// planar quadrotor: state (px, pz, theta, vx, vz, omega), control (T1, T2)
template <class R>
__device__ __forceinline__ void quad_fc(const R* x, const R* u, const float* dyn, R* f, R* Jx, R* Ju) {
    const R m = dyn[1], I = dyn[2], arm = dyn[3], g = dyn[4];
    R s, c;
    msincos(x[2], &s, &c);
    const R T = u[0] + u[1];
    f[0] = x[3];
    f[1] = x[4];
    f[2] = x[5];
    f[3] = -T * s / m;
    f[4] = T * c / m - g;
    f[5] = (u[1] - u[0]) * arm / I;
    if (Jx) {
        for (int i = 0; i < 36; ++i) Jx[i] = R(0);
        Jx[0 * 6 + 3] = R(1);
        Jx[1 * 6 + 4] = R(1);
        Jx[2 * 6 + 5] = R(1);
        Jx[3 * 6 + 2] = -T * c / m;
        Jx[4 * 6 + 2] = -T * s / m;
    }
    if (Ju) {
        Ju[0] = Ju[1] = Ju[2] = Ju[3] = Ju[4] = Ju[5] = R(0);
        Ju[6] = Ju[7] = -s / m;
        Ju[8] = Ju[9] = c / m;
        Ju[10] = -arm / I;
        Ju[11] = arm / I;
    }
}

// RK4 step of the quadrotor; with Jacobians by the chain rule through the stages.
template <class R>
__device__ inline void quad_rk4(const R* x, const R* u, const float* dyn, R* phi, R* dPx /*36 or null*/,
                                R* dPu /*12 or null*/) {
    const R dt = dyn[0];
    R k[4][6], xs[6];
    R dkx[6 * 6], dku[6 * 2], J[36], Ju[12], accx[36], accu[12], tx[36], tu[12];
    const R cst[4] = {R(0), R(0.5), R(0.5), R(1)};
    const R wgt[4] = {R(1), R(2), R(2), R(1)};
    const bool jac = dPx != nullptr;
    if (jac) {
        for (int i = 0; i < 36; ++i) accx[i] = R(0);
        for (int i = 0; i < 12; ++i) accu[i] = R(0);
    }
    for (int st = 0; st < 4; ++st) {
        for (int i = 0; i < 6; ++i) xs[i] = x[i] + (st ? cst[st] * dt * k[st - 1][i] : R(0));
        quad_fc<R>(xs, u, dyn, k[st], jac ? J : nullptr, jac ? Ju : nullptr);
        if (jac) {
            // d xs / dx = I + c dt dk_{prev}/dx,  d xs / du = c dt dk_{prev}/du
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    R a = R(0);
                    for (int l = 0; l < 6; ++l) {
                        R dxs = (l == j ? R(1) : R(0)) + (st ? cst[st] * dt * dkx[l * 6 + j] : R(0));
                        a += J[i * 6 + l] * dxs;
                    }
                    tx[i * 6 + j] = a;
                }
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 2; ++j) {
                    R a = Ju[i * 2 + j];
                    if (st)
                        for (int l = 0; l < 6; ++l) a += J[i * 6 + l] * cst[st] * dt * dku[l * 2 + j];
                    tu[i * 2 + j] = a;
                }
            for (int i = 0; i < 36; ++i) { dkx[i] = tx[i]; accx[i] += wgt[st] * tx[i]; }
            for (int i = 0; i < 12; ++i) { dku[i] = tu[i]; accu[i] += wgt[st] * tu[i]; }
        }
    }
    for (int i = 0; i < 6; ++i)
        phi[i] = x[i] + dt / R(6) * (k[0][i] + R(2) * k[1][i] + R(2) * k[2][i] + k[3][i]);
    if (jac) {
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) dPx[i * 6 + j] = (i == j ? R(1) : R(0)) + dt / R(6) * accx[i * 6 + j];
        for (int i = 0; i < 12; ++i) dPu[i] = dt / R(6) * accu[i];
    }
}

// ---------------------------------------------------------------------------
// single-rigid-body humanoid (App. humanoid SRB dynamics): state (p, Theta =
// ZYX (roll, pitch, yaw), v, omega body rates), control (f_L, f_R) in the world
// frame; dyn = [dt, m, Ixx, Iyy, Izz, r_L (3), r_R (3), gravity]:
//   p_dot = v, Theta_dot = T(Theta) omega, v_dot = (f_L + f_R) / m + g,
//   omega_dot = I^-1 (r_L x f_L + r_R x f_R - omega x (I omega)).
// ---------------------------------------------------------------------------
template <class R>
struct SrbTrig {
    R sp, cp, tt, sc;   // sin / cos of roll, tan and 1 / cos of pitch
};
template <class R>
__device__ __forceinline__ SrbTrig<R> srb_trig(const R* x) {
    SrbTrig<R> q;
    msincos(x[3], &q.sp, &q.cp);
    q.tt = mtan(x[4]);
    q.sc = R(1) / mcos(x[4]);
    return q;
}

template <class R>
__device__ __forceinline__ void srb_fc(const R* x, const R* u, const float* dyn, const SrbTrig<R>& q, R* f) {
    const R m = dyn[1], Ix = dyn[2], Iy = dyn[3], Iz = dyn[4], g = dyn[11];
    const float* rl = dyn + 5;
    const float* rr = dyn + 8;
    const R wx = x[9], wy = x[10], wz = x[11];
    f[0] = x[6];
    f[1] = x[7];
    f[2] = x[8];
    f[3] = wx + q.sp * q.tt * wy + q.cp * q.tt * wz;
    f[4] = q.cp * wy - q.sp * wz;
    f[5] = q.sp * q.sc * wy + q.cp * q.sc * wz;
    f[6] = (u[0] + u[3]) / m;
    f[7] = (u[1] + u[4]) / m;
    f[8] = (u[2] + u[5]) / m - g;
    // torque r_L x f_L + r_R x f_R - omega x (I omega)
    const R hx = Ix * wx, hy = Iy * wy, hz = Iz * wz;
    const R tx = (R)rl[1] * u[2] - (R)rl[2] * u[1] + (R)rr[1] * u[5] - (R)rr[2] * u[4] - (wy * hz - wz * hy);
    const R ty = (R)rl[2] * u[0] - (R)rl[0] * u[2] + (R)rr[2] * u[3] - (R)rr[0] * u[5] - (wz * hx - wx * hz);
    const R tz = (R)rl[0] * u[1] - (R)rl[1] * u[0] + (R)rr[0] * u[4] - (R)rr[1] * u[3] - (wx * hy - wy * hx);
    f[9] = tx / Ix;
    f[10] = ty / Iy;
    f[11] = tz / Iz;
}

// directional derivative df = (df_c/dx) dx + (df_c/du) du at (x, u)
template <class R>
__device__ __forceinline__ void srb_jvp(const R* x, const float* dyn, const SrbTrig<R>& q, const R* dx, const R* du,
                                        R* df) {
    const R m = dyn[1], Ix = dyn[2], Iy = dyn[3], Iz = dyn[4];
    const float* rl = dyn + 5;
    const float* rr = dyn + 8;
    const R wx = x[9], wy = x[10], wz = x[11];
    const R dwx = dx[9], dwy = dx[10], dwz = dx[11], dph = dx[3], dth = dx[4];
    const R sec2 = q.sc * q.sc;
    df[0] = dx[6];
    df[1] = dx[7];
    df[2] = dx[8];
    df[3] = dwx + q.sp * q.tt * dwy + q.cp * q.tt * dwz + dph * (q.cp * q.tt * wy - q.sp * q.tt * wz) +
            dth * (q.sp * sec2 * wy + q.cp * sec2 * wz);
    df[4] = q.cp * dwy - q.sp * dwz - dph * (q.sp * wy + q.cp * wz);
    df[5] = q.sp * q.sc * dwy + q.cp * q.sc * dwz + dph * (q.cp * q.sc * wy - q.sp * q.sc * wz) +
            dth * q.tt * q.sc * (q.sp * wy + q.cp * wz);
    df[6] = (du[0] + du[3]) / m;
    df[7] = (du[1] + du[4]) / m;
    df[8] = (du[2] + du[5]) / m;
    // d(omega x I omega) = d omega x I omega + omega x I d omega
    const R hx = Ix * wx, hy = Iy * wy, hz = Iz * wz, dhx = Ix * dwx, dhy = Iy * dwy, dhz = Iz * dwz;
    const R gx = (dwy * hz - dwz * hy) + (wy * dhz - wz * dhy);
    const R gy = (dwz * hx - dwx * hz) + (wz * dhx - wx * dhz);
    const R gz = (dwx * hy - dwy * hx) + (wx * dhy - wy * dhx);
    df[9] = ((R)rl[1] * du[2] - (R)rl[2] * du[1] + (R)rr[1] * du[5] - (R)rr[2] * du[4] - gx) / Ix;
    df[10] = ((R)rl[2] * du[0] - (R)rl[0] * du[2] + (R)rr[2] * du[3] - (R)rr[0] * du[5] - gy) / Iy;
    df[11] = ((R)rl[0] * du[1] - (R)rl[1] * du[0] + (R)rr[0] * du[4] - (R)rr[1] * du[3] - gz) / Iz;
}

// RK4 step x+ = Phi(x, u) (dt = dyn[0]); with Am != nullptr also dPhi/d(x, u) (12 x 18,
// row k at Am + k ld), column by column: each unit direction is carried through the
// four stages by directional derivatives (forward mode).
template <class R>
__device__ inline void srb_rk4(const R* x, const R* u, const float* dyn, R* phi, R* Am, int ld) {
    const R dt = dyn[0];
    R xs[4][12], k[4][12];
    SrbTrig<R> q[4];
    const R cst[4] = {R(0), R(0.5), R(0.5), R(1)};
    for (int st = 0; st < 4; ++st) {
        for (int i = 0; i < 12; ++i) xs[st][i] = x[i] + (st ? cst[st] * dt * k[st - 1][i] : R(0));
        q[st] = srb_trig<R>(xs[st]);
        srb_fc<R>(xs[st], u, dyn, q[st], k[st]);
    }
    for (int i = 0; i < 12; ++i) phi[i] = x[i] + dt / R(6) * (k[0][i] + R(2) * k[1][i] + R(2) * k[2][i] + k[3][i]);
    if (!Am) return;
    for (int j = 0; j < 18; ++j) {
        R d0[12], du[6], dxs[12], dk[12], acc[12];
        for (int i = 0; i < 12; ++i) d0[i] = (i == j) ? R(1) : R(0);
        for (int i = 0; i < 6; ++i) du[i] = (i + 12 == j) ? R(1) : R(0);
        for (int i = 0; i < 12; ++i) acc[i] = R(0);
        for (int st = 0; st < 4; ++st) {
            for (int i = 0; i < 12; ++i) dxs[i] = d0[i] + (st ? cst[st] * dt * dk[i] : R(0));
            srb_jvp<R>(xs[st], dyn, q[st], dxs, du, dk);
            const R wgt = (st == 1 || st == 2) ? R(2) : R(1);
            for (int i = 0; i < 12; ++i) acc[i] += wgt * dk[i];
        }
        for (int i = 0; i < 12; ++i) Am[i * ld + j] = d0[i] + dt / R(6) * acc[i];
    }
}

}  // namespace tmpc
