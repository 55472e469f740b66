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

enum { MODEL_DI = 0, MODEL_LINEAR = 1, MODEL_BICYCLE = 2, MODEL_QUAD = 3 };

struct ModelDims {
    int nx, nu, ng;
};

__host__ __device__ inline ModelDims model_dims(int model, int lnx, int lnu, int lng) {
    switch (model) {
        case MODEL_DI: return {4, 2, 4};
        case MODEL_BICYCLE: return {6, 2, 5};
        case MODEL_QUAD: return {6, 2, 2};
        default: return {lnx, lnu, lng};
    }
}

// Am / Ap / G blocks identical for every stage -> stored once (stage stride 0)
__host__ __device__ inline bool model_const_Am(int m) { return m == MODEL_DI || m == MODEL_LINEAR; }
__host__ __device__ inline bool model_const_Ap(int m) { return m != MODEL_BICYCLE; }
__host__ __device__ inline bool model_const_G(int m) { return m != MODEL_BICYCLE; }
__host__ __device__ inline bool model_linear_dyn(int m) { return m == MODEL_DI || m == MODEL_LINEAR; }

// ---------------------------------------------------------------------------
// racing centreline: periodic table (x_c, y_c, psi_c, kappa) every ds metres,
// cubic Hermite interpolation with knot derivatives (cos psi, sin psi, kappa)
// ---------------------------------------------------------------------------
struct TrackPt {
    float xc, yc, psic, dxc, dyc, dpsic;
};

__device__ __forceinline__ TrackPt track_eval(const float* tab, int nt, float ds, float s) {
    const float L = nt * ds;
    float sm = s - L * floorf(s / L);
    int k = (int)floorf(sm / ds);
    k = k < 0 ? 0 : (k > nt - 1 ? nt - 1 : k);
    const float tau = (sm - k * ds) / ds;
    const float* a = tab + 4 * k;
    const float* b = a + 4;
    const float t2 = tau * tau, t3 = t2 * tau;
    const float h00 = 2.f * t3 - 3.f * t2 + 1.f, h10 = t3 - 2.f * t2 + tau;
    const float h01 = -2.f * t3 + 3.f * t2, h11 = t3 - t2;
    const float d00 = 6.f * t2 - 6.f * tau, d10 = 3.f * t2 - 4.f * tau + 1.f;
    const float d01 = -6.f * t2 + 6.f * tau, d11 = 3.f * t2 - 2.f * tau;
    float sa, ca, sb, cb;
    sincosf(a[2], &sa, &ca);
    sincosf(b[2], &sb, &cb);
    TrackPt p;
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
__device__ __forceinline__ void bicycle_fc(const float* x, const float* u, float L,
                                           const float* tab, int nt, float ds,
                                           float* f, float* Jx, float* Ju) {
    const float psi = x[2], v = x[3], dl = x[4], s = x[5];
    TrackPt tp = track_eval(tab, nt, ds, s);
    float sp, cp;
    sincosf(psi, &sp, &cp);
    const float tn = tanf(dl);
    float sd, cd;
    sincosf(psi - tp.psic, &sd, &cd);
    f[0] = v * cp;
    f[1] = v * sp;
    f[2] = v * tn / L;
    f[3] = u[0];
    f[4] = u[1];
    f[5] = v * cd;
    if (Jx) {
        for (int i = 0; i < 36; ++i) Jx[i] = 0.f;
        const float cdl = cosf(dl);
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
        for (int i = 0; i < 12; ++i) Ju[i] = 0.f;
        Ju[3 * 2 + 0] = 1.f;
        Ju[4 * 2 + 1] = 1.f;
    }
}

// planar quadrotor: state (px, pz, theta, vx, vz, omega), control (T1, T2)
__device__ __forceinline__ void quad_fc(const float* x, const float* u, const float* dyn,
                                        float* f, float* Jx, float* Ju) {
    const float m = dyn[1], I = dyn[2], arm = dyn[3], g = dyn[4];
    float s, c;
    sincosf(x[2], &s, &c);
    const float T = u[0] + u[1];
    f[0] = x[3];
    f[1] = x[4];
    f[2] = x[5];
    f[3] = -T * s / m;
    f[4] = T * c / m - g;
    f[5] = (u[1] - u[0]) * arm / I;
    if (Jx) {
        for (int i = 0; i < 36; ++i) Jx[i] = 0.f;
        Jx[0 * 6 + 3] = 1.f;
        Jx[1 * 6 + 4] = 1.f;
        Jx[2 * 6 + 5] = 1.f;
        Jx[3 * 6 + 2] = -T * c / m;
        Jx[4 * 6 + 2] = -T * s / m;
    }
    if (Ju) {
        Ju[0] = Ju[1] = Ju[2] = Ju[3] = Ju[4] = Ju[5] = 0.f;
        Ju[6] = Ju[7] = -s / m;
        Ju[8] = Ju[9] = c / m;
        Ju[10] = -arm / I;
        Ju[11] = arm / I;
    }
}

// RK4 step of the quadrotor; with Jacobians by the chain rule through the stages.
__device__ inline void quad_rk4(const float* x, const float* u, const float* dyn, float* phi,
                                float* dPx /*36 or null*/, float* dPu /*12 or null*/) {
    const float dt = dyn[0];
    float k[4][6], xs[6];
    float dkx[6 * 6], dku[6 * 2], J[36], Ju[12], accx[36], accu[12], tx[36], tu[12];
    const float cst[4] = {0.f, 0.5f, 0.5f, 1.f};
    const float wgt[4] = {1.f, 2.f, 2.f, 1.f};
    const bool jac = dPx != nullptr;
    if (jac) {
        for (int i = 0; i < 36; ++i) accx[i] = 0.f;
        for (int i = 0; i < 12; ++i) accu[i] = 0.f;
    }
    for (int st = 0; st < 4; ++st) {
        for (int i = 0; i < 6; ++i) xs[i] = x[i] + (st ? cst[st] * dt * k[st - 1][i] : 0.f);
        quad_fc(xs, u, dyn, k[st], jac ? J : nullptr, jac ? Ju : nullptr);
        if (jac) {
            // d xs / dx = I + c dt dk_{prev}/dx,  d xs / du = c dt dk_{prev}/du
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    float a = 0.f;
                    for (int l = 0; l < 6; ++l) {
                        float dxs = (l == j ? 1.f : 0.f) + (st ? cst[st] * dt * dkx[l * 6 + j] : 0.f);
                        a += J[i * 6 + l] * dxs;
                    }
                    tx[i * 6 + j] = a;
                }
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 2; ++j) {
                    float a = Ju[i * 2 + j];
                    if (st)
                        for (int l = 0; l < 6; ++l) a += J[i * 6 + l] * cst[st] * dt * dku[l * 2 + j];
                    tu[i * 2 + j] = a;
                }
            for (int i = 0; i < 36; ++i) { dkx[i] = tx[i]; accx[i] += wgt[st] * tx[i]; }
            for (int i = 0; i < 12; ++i) { dku[i] = tu[i]; accu[i] += wgt[st] * tu[i]; }
        }
    }
    for (int i = 0; i < 6; ++i)
        phi[i] = x[i] + dt / 6.f * (k[0][i] + 2.f * k[1][i] + 2.f * k[2][i] + k[3][i]);
    if (jac) {
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) dPx[i * 6 + j] = (i == j ? 1.f : 0.f) + dt / 6.f * accx[i * 6 + j];
        for (int i = 0; i < 12; ++i) dPu[i] = dt / 6.f * accu[i];
    }
}

}  // namespace tmpc
