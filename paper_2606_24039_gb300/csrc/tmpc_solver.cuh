// Device side of the batched SQP / ADMM OCP solver: one CTA per instance,
// CTA-cooperative stage operations, everything resident in the handle's
// workspace (global memory, L1/L2-cached) with the n x n factorisation
// scratch in shared memory.
//
// Paper map:
//   linearize()      QP approximation at the SQP iterate (Section III-A, App. B)
//   factor()         S = P + sigma I + rho_f C'C + G' W G and its block LDL'
//                    factorisation (Theta_t, Phi_t of App. C), once per SQP
//                    step and per accepted rho (Section III-E: factor reuse)
//   admm_iter()      one iteration of Algorithm 3 (eta, S solve, relaxation,
//                    projection / smoothed projection, dual update)
//   residuals()      Eq. (admm:residuals) and the normalisers of
//                    Eq. (admm:termination:slack); rho rule of Eq. (rho:update)
//   linesearch()     Appendix D (merit, Armijo, candidates in parallel)
//   kkt()            Eq. (sqp_stop)
#pragma once
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "tmpc_models.cuh"

namespace tmpc {

struct KOpts {
    float sigma, rho0, rho_min, rho_max, alpha;
    float eps_abs, eps_rel, eps_c, eps_g, ls_eta;
    int k_rho_iter;
    float k_rho_ratio;
    int max_sqp, max_admm, n_ls, newton_steps, early_exit, check_every;
    float bwd_rho, bwd_sigma;
    int bwd_iters;
    int force_fail;   // instance index + 1 whose NOT_PD flag starts set (0: none)
    int wait_polls;   // polls of a bounded wait on an asynchronous copy (0: kMbarSpin)
    int force_timeout;   // nonzero: every bounded wait gives up at once (test hook)
    int bwd_solver;      // backward: 0 hybrid (refinement, direct where it does not converge), 1 refinement, 2 direct
    int exact_hessian;   // 1: the direct backward adds the constraint curvature of the Lagrangian
    float bwd_gamma;     // bwd_solver 3: penalty weight of the hard active rows (reduced adjoint QP)
};

struct KLayout {
    int B, Nmax, nx, nu, ng, n, n_dyn, n_track;
    int vs;   // generic kernel: 1 if the ADMM vectors live in shared memory (see carve_smem)
};

struct KParams {
    const int* N;
    const int* model;
    const float* x0;
    const float *Qd, *Rd, *Wd, *ref, *lin, *lo, *hi, *g2, *g1, *dyn, *track;
    const float* scale;   // [B][n] magnitudes of the normalised variables (shared-memory kernels), or nullptr
};

struct KSol {
    float *z, *xi, *yf, *yg;
    int* status;
    float* stats;
};

// offsets (in floats) of the per-instance workspace arrays; slot = stride floats
struct WsOff {
    long long stride;
    int Am, Ap, cv, fv, Gm, gv, glo, ghi, qv, Dinv, Om, x, xt, eta, zg, yg, xi, yf, zb, xib, yfb, ygb, gw, czb, gzb, pf, pg;
};

#define kInf __int_as_float(0x7f800000)
constexpr int kMaxLs = 16;

// 4-bit code of a line-search step: k for alpha = 2^-k (k >= 14 coded 14), 15 for alpha = 0
__device__ inline int ls_code(float a) {
    if (!(a > 0.f)) return 15;
    int k = 0;
    while (k < 14 && a < 0.75f) {
        a *= 2.f;
        ++k;
    }
    return k;
}

// shared-memory scratch of one CTA
struct Smem {
    float* A;      // n*n
    float* Bm;     // n*n
    float* Cm;     // n*n
    float* red;    // 32*8 floats
    float* red8;   // 8*96 floats (ldl_solve partial sums)
    double* redd;  // 32*2 doubles
    double* lsacc; // 2*kMaxLs doubles
    int* flags;    // 4 ints
    unsigned long long* mbar;  // 2 mbarriers of the bulk-copy pipeline (ldl_solve)
    float* vs;     // ADMM vectors of the current instance (nullptr: in the global workspace)
};

struct Ctx {
    int N, T, nx, nu, n, ng, model, nt;
    int lnx, lnu, ln, lng;
    const float *x0, *Qd, *Rd, *Wd, *ref, *lin, *lo, *hi, *g2, *g1, *dyn, *track;
    const float* bv;   // linear model: affine term b of x+ = A x + B u + b (nullptr: b = 0)
    float *Am, *Ap, *cv, *fv, *Gm, *gv, *glo, *ghi, *qv, *Dinv, *Om, *x, *xt, *eta, *zg, *yg, *xi, *yf;
    float *zb, *xib, *yfb, *ygb, *gw, *czb, *gzb, *pf, *pg;
    int amS, apS, gS;

    __device__ __forceinline__ const float* Amt(int t) const { return Am + t * amS; }
    __device__ __forceinline__ const float* Apt(int t) const { return Ap + t * apS; }
    __device__ __forceinline__ const float* Gt(int t) const { return Gm + t * gS; }
    __device__ __forceinline__ float Q(int t, int i) const { return Qd[t * lnx + i]; }
    __device__ __forceinline__ float R(int t, int j) const { return Rd[t * lnu + j]; }
    __device__ __forceinline__ float W(int j) const { return Wd ? Wd[j] : 0.f; }
    __device__ __forceinline__ float refv(int t, int k) const { return ref ? ref[t * ln + k] : 0.f; }
    __device__ __forceinline__ float linv(int t, int k) const { return lin ? lin[t * ln + k] : 0.f; }
    __device__ __forceinline__ float lob(int t, int r) const { return lo[t * lng + r]; }
    __device__ __forceinline__ float hib(int t, int r) const { return hi[t * lng + r]; }
    __device__ __forceinline__ float gam2(int r) const { return g2 ? g2[r] : kInf; }
    __device__ __forceinline__ float gam1(int r) const { return g1 ? g1[r] : 0.f; }
    // diagonal of the cost Hessian block D_t (App. B: D_t = H^+_{t-1} + H^-_t)
    __device__ __forceinline__ float Pdiag(int t, int j) const {
        if (j < nx) return Q(t, j);
        const int k = j - nx;
        float v = R(t, k);
        if (t < N) v += W(k);
        if (t > 0) v += W(k);
        return v;
    }
    // cost weight of the (x-x_ref)/(u-u_ref) term (no rate term)
    __device__ __forceinline__ float Cw(int t, int j) const { return j < nx ? Q(t, j) : R(t, j - nx); }
};

// ---------------------------------------------------------------------------
// CTA reductions (all threads get the result)
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void cta_max_k(float (&v)[K], float* red) {
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] = fmaxf(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * 32 + w] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float r = red[k * 32];
        for (int i = 1; i < nw; ++i) r = fmaxf(r, red[k * 32 + i]);
        v[k] = r;
    }
    __syncthreads();
}

__device__ __forceinline__ double cta_sum_d(double v, double* redd) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0) redd[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < nw; ++i) r += redd[i];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float fin(float v) { return (v == v) ? fabsf(v) : kInf; }

// small dense solve (Gaussian elimination, partial pivoting), M is m x m row-major, in place
__device__ inline void small_solve(float* M, float* b, int m) {
    for (int k = 0; k < m; ++k) {
        int p = k;
        float best = fabsf(M[k * m + k]);
        for (int i = k + 1; i < m; ++i)
            if (fabsf(M[i * m + k]) > best) { best = fabsf(M[i * m + k]); p = i; }
        if (p != k) {
            for (int j = 0; j < m; ++j) { float tmp = M[k * m + j]; M[k * m + j] = M[p * m + j]; M[p * m + j] = tmp; }
            float tmp = b[k]; b[k] = b[p]; b[p] = tmp;
        }
        const float d = M[k * m + k];
        for (int i = k + 1; i < m; ++i) {
            const float l = M[i * m + k] / d;
            for (int j = k; j < m; ++j) M[i * m + j] -= l * M[k * m + j];
            b[i] -= l * b[k];
        }
    }
    for (int i = m - 1; i >= 0; --i) {
        float a = b[i];
        for (int j = i + 1; j < m; ++j) a -= M[i * m + j] * b[j];
        b[i] = a / M[i * m + i];
    }
}

// ---------------------------------------------------------------------------
// model evaluation per stage (one thread)
// ---------------------------------------------------------------------------
// f_t at (zt, zn) and optionally the Jacobian blocks Am, Ap (row-major nx x n).
__device__ inline void stage_dyn(const Ctx& c, int t, const float* zt, const float* zn, float* f,
                          float* Am, float* Ap) {
    const int nx = c.nx, n = c.n;
    switch (c.model) {
        case MODEL_DI: {
            const float dt = c.dyn[0];
            f[0] = zt[0] + dt * zt[2] + 0.5f * dt * dt * zt[4] - zn[0];
            f[1] = zt[1] + dt * zt[3] + 0.5f * dt * dt * zt[5] - zn[1];
            f[2] = zt[2] + dt * zt[4] - zn[2];
            f[3] = zt[3] + dt * zt[5] - zn[3];
            break;
        }
        case MODEL_LINEAR: {
            const float* A = c.dyn;
            const float* B = c.dyn + nx * nx;
            for (int k = 0; k < nx; ++k) {
                float a = (c.bv ? c.bv[k] : 0.f) - zn[k];
                for (int j = 0; j < nx; ++j) a += A[k * nx + j] * zt[j];
                for (int j = 0; j < c.nu; ++j) a += B[k * c.nu + j] * zt[nx + j];
                f[k] = a;
            }
            break;
        }
        case MODEL_QUAD: {
            float phi[6], dPx[36], dPu[12];
            quad_rk4(zt, zt + 6, c.dyn, phi, Am ? dPx : nullptr, Am ? dPu : nullptr);
            for (int k = 0; k < 6; ++k) f[k] = phi[k] - zn[k];
            if (Am) {
                for (int k = 0; k < 6; ++k) {
                    for (int j = 0; j < 6; ++j) Am[k * n + j] = dPx[k * 6 + j];
                    for (int j = 0; j < 2; ++j) Am[k * n + 6 + j] = dPu[k * 2 + j];
                }
            }
            break;
        }
        case MODEL_SRB: {
            float phi[12];
            srb_rk4<float>(zt, zt + 12, c.dyn, phi, Am, n);
            for (int k = 0; k < 12; ++k) f[k] = phi[k] - zn[k];
            break;
        }
        case MODEL_BICYCLE_TRAP: {
            // f_t = x_t + dt/2 (f_c(z_t) + f_c(z_{t+1})) - x_{t+1}  (Remark A1)
            const float dt = c.dyn[0];
            float fa[6], fb[6], Jxa[36], Jua[12], Jxb[36], Jub[12];
            const bool jac = Am != nullptr;
            bicycle_fc<float>(zt, zt + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fa, jac ? Jxa : nullptr, jac ? Jua : nullptr);
            bicycle_fc<float>(zn, zn + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fb, jac ? Jxb : nullptr, jac ? Jub : nullptr);
            for (int k = 0; k < 6; ++k) f[k] = zt[k] + 0.5f * dt * (fa[k] + fb[k]) - zn[k];
            if (jac) {
                for (int k = 0; k < 6; ++k) {
                    for (int j = 0; j < 6; ++j) {
                        Am[k * n + j] = (k == j ? 1.f : 0.f) + 0.5f * dt * Jxa[k * 6 + j];
                        Ap[k * n + j] = (k == j ? -1.f : 0.f) + 0.5f * dt * Jxb[k * 6 + j];
                    }
                    for (int j = 0; j < 2; ++j) {
                        Am[k * n + 6 + j] = 0.5f * dt * Jua[k * 2 + j];
                        Ap[k * n + 6 + j] = 0.5f * dt * Jub[k * 2 + j];
                    }
                }
            }
            break;
        }
        case MODEL_BICYCLE_NEWTON: {
            // x_{t+1} = Phi(x_t, u_t): kNewtonMapSteps Newton steps on the midpoint residual
            // r(p) = x + dt f_c((x + p)/2, u) - p from the explicit Euler step; Jacobians by
            // the implicit function theorem at the returned p (A^+ = [-I 0], constant)
            const float dt = c.dyn[0];
            float p[6], mid[6], fc[6], Jx[36], Ju[12], Mp[36], r[6];
            bicycle_fc<float>(zt, zt + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fc, nullptr, nullptr);
            for (int k = 0; k < 6; ++k) p[k] = zt[k] + dt * fc[k];
            for (int it = 0; it < kNewtonMapSteps; ++it) {
                for (int k = 0; k < 6; ++k) mid[k] = 0.5f * (zt[k] + p[k]);
                bicycle_fc<float>(mid, zt + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fc, Jx, nullptr);
                for (int k = 0; k < 6; ++k) {
                    r[k] = zt[k] + dt * fc[k] - p[k];
                    for (int j = 0; j < 6; ++j) Mp[k * 6 + j] = (k == j ? -1.f : 0.f) + 0.5f * dt * Jx[k * 6 + j];
                }
                small_solve(Mp, r, 6);
                for (int k = 0; k < 6; ++k) p[k] -= r[k];
            }
            for (int k = 0; k < 6; ++k) f[k] = p[k] - zn[k];
            if (Ap)
                for (int k = 0; k < 6; ++k)
                    for (int j = 0; j < n; ++j) Ap[k * n + j] = (k == j) ? -1.f : 0.f;
            if (Am) {
                for (int k = 0; k < 6; ++k) mid[k] = 0.5f * (zt[k] + p[k]);
                bicycle_fc<float>(mid, zt + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fc, Jx, Ju);
                // column j of dPhi/dz = -(dr/dp)^-1 (dr/dz)_j, dr/dx = I + dt/2 J_x, dr/du = dt J_u
                for (int j = 0; j < 8; ++j) {
                    float col[6], M[36];
                    for (int k = 0; k < 6; ++k) {
                        col[k] = -(j < 6 ? (k == j ? 1.f : 0.f) + 0.5f * dt * Jx[k * 6 + j] : dt * Ju[k * 2 + j - 6]);
                        for (int l = 0; l < 6; ++l) M[k * 6 + l] = (k == l ? -1.f : 0.f) + 0.5f * dt * Jx[k * 6 + l];
                    }
                    small_solve(M, col, 6);
                    for (int k = 0; k < 6; ++k) Am[k * n + j] = col[k];
                }
            }
            break;
        }
        case MODEL_BICYCLE: {
            const float dt = c.dyn[0];
            float mid[6], fc[6], Jx[36], Ju[12];
            for (int k = 0; k < 6; ++k) mid[k] = 0.5f * (zt[k] + zn[k]);
            const bool jac = Am != nullptr;
            bicycle_fc(mid, zt + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fc, jac ? Jx : nullptr,
                       jac ? Ju : nullptr);
            for (int k = 0; k < 6; ++k) f[k] = zt[k] + dt * fc[k] - zn[k];
            if (jac) {
                for (int k = 0; k < 6; ++k) {
                    for (int j = 0; j < 6; ++j) {
                        const float h = 0.5f * dt * Jx[k * 6 + j];
                        Am[k * n + j] = (k == j ? 1.f : 0.f) + h;
                        Ap[k * n + j] = (k == j ? -1.f : 0.f) + h;
                    }
                    for (int j = 0; j < 2; ++j) {
                        Am[k * n + 6 + j] = dt * Ju[k * 2 + j];
                        Ap[k * n + 6 + j] = 0.f;
                    }
                }
            }
            break;
        }
    }
}

// g_t(z) and optionally G_t (row-major ng x n)
__device__ inline void stage_con(const Ctx& c, const float* z, float* g, float* G) {
    const int n = c.n, ng = c.ng, nx = c.nx;
    if (G)
        for (int i = 0; i < ng * n; ++i) G[i] = 0.f;
    switch (c.model) {
        case MODEL_DI:
            g[0] = z[4]; g[1] = z[5]; g[2] = z[2]; g[3] = z[3];
            if (G) { G[0 * n + 4] = 1.f; G[1 * n + 5] = 1.f; G[2 * n + 2] = 1.f; G[3 * n + 3] = 1.f; }
            break;
        case MODEL_LINEAR:
            for (int r = 0; r < ng; ++r) {
                g[r] = z[nx + r];
                if (G) G[r * n + nx + r] = 1.f;
            }
            break;
        case MODEL_QUAD:
            g[0] = z[6]; g[1] = z[7];
            if (G) { G[0 * n + 6] = 1.f; G[1 * n + 7] = 1.f; }
            break;
        case MODEL_SRB:   // the friction cone as a box on the six foot-force components
            for (int r = 0; r < 6; ++r) {
                g[r] = z[12 + r];
                if (G) G[r * n + 12 + r] = 1.f;
            }
            break;
        case MODEL_BICYCLE:
        case MODEL_BICYCLE_TRAP:
        case MODEL_BICYCLE_NEWTON: {  // accel, steer rate, speed, steering angle, lateral error
            TrackPt tp = track_eval(c.track, c.nt, c.dyn[2], z[5]);
            float sp, cp;
            sincosf(tp.psic, &sp, &cp);
            const float dx = z[0] - tp.xc, dy = z[1] - tp.yc;
            g[0] = z[6]; g[1] = z[7]; g[2] = z[3]; g[3] = z[4];
            g[4] = -dx * sp + dy * cp;
            if (G) {
                G[0 * n + 6] = 1.f; G[1 * n + 7] = 1.f; G[2 * n + 3] = 1.f; G[3 * n + 4] = 1.f;
                G[4 * n + 0] = -sp;
                G[4 * n + 1] = cp;
                G[4 * n + 5] = tp.dxc * sp - tp.dyc * cp - tp.dpsic * (dx * cp + dy * sp);
            }
            break;
        }
    }
}


// y = P x  (cost Hessian, block-tridiagonal with diagonal blocks), stage t, entry j
__device__ __forceinline__ float Px_entry(const Ctx& c, const float* x, int t, int j) {
    float v = c.Pdiag(t, j) * x[t * c.n + j];
    if (j >= c.nx) {
        const float w = c.W(j - c.nx);
        if (t > 0) v -= w * x[(t - 1) * c.n + j];
        if (t < c.N) v -= w * x[(t + 1) * c.n + j];
    }
    return v;
}

// (C' v)_t entry j with v_r given by a functor of (row r, k)
template <class V>
__device__ __forceinline__ float Ct_entry(const Ctx& c, int t, int j, V v) {
    float s = 0.f;
    if (t == 0 && j < c.nx) s += v(0, j);
    if (t < c.N) {
        const float* Am = c.Amt(t);
        float s1 = 0.f;
#pragma unroll 8
        for (int k = 0; k < c.nx; ++k) s1 += Am[k * c.n + j] * v(t + 1, k);
        s += s1;
    }
    if (t > 0) {
        const float* Ap = c.Apt(t - 1);
        float s2 = 0.f;
#pragma unroll 8
        for (int k = 0; k < c.nx; ++k) s2 += Ap[k * c.n + j] * v(t, k);
        s += s2;
    }
    return s;
}

// (C x)_r entry k
__device__ __forceinline__ float Cx_entry(const Ctx& c, const float* x, int r, int k) {
    if (r == 0) return x[k];
    const int t = r - 1;
    const float* Am = c.Amt(t);
    const float* Ap = c.Apt(t);
    const float* a = x + t * c.n;
    const float* b = x + (t + 1) * c.n;
    float s = 0.f, s2 = 0.f;
#pragma unroll 8
    for (int j = 0; j < c.n; ++j) {
        s += Am[k * c.n + j] * a[j];
        s2 += Ap[k * c.n + j] * b[j];
    }
    return s + s2;
}

// Selector structure of G: for the double integrator, linear and quadrotor
// models every inequality row selects one stage variable (the bicycle has a
// dense row).  g_col(c, r): the column row r selects; g_row(c, j): the row
// that selects column j, -1 if none.  The hot loops use them instead of
// multiplying through the zeros of G (same values: the other terms are 0).
__device__ __forceinline__ bool g_is_selector(const Ctx& c) { return !is_bicycle(c.model); }
__device__ __forceinline__ int g_col(const Ctx& c, int r) {
    switch (c.model) {
        case MODEL_LINEAR: return c.nx + r;
        case MODEL_DI: return r == 0 ? 4 : r == 1 ? 5 : r == 2 ? 2 : 3;
        case MODEL_QUAD: return r == 0 ? 6 : 7;
        case MODEL_SRB: return 12 + r;
    }
    return -1;
}
__device__ __forceinline__ int g_row(const Ctx& c, int j) {
    switch (c.model) {
        case MODEL_LINEAR: return (j >= c.nx && j - c.nx < c.ng) ? j - c.nx : -1;
        case MODEL_DI: return j == 4 ? 0 : j == 5 ? 1 : j == 2 ? 2 : j == 3 ? 3 : -1;
        case MODEL_QUAD: return j == 6 ? 0 : j == 7 ? 1 : -1;
        case MODEL_SRB: return j >= 12 && j < 18 ? j - 12 : -1;
    }
    return -1;
}

__device__ __forceinline__ float Gx_entry(const Ctx& c, const float* x, int t, int r) {
    if (g_is_selector(c)) return x[t * c.n + g_col(c, r)];
    const float* G = c.Gt(t) + r * c.n;
    const float* a = x + t * c.n;
    float s = 0.f;
#pragma unroll 8
    for (int j = 0; j < c.n; ++j) s += G[j] * a[j];
    return s;
}

// ---------------------------------------------------------------------------
// initial guess: x_0 = x_init, u_t = u_ref_t, x_{t+1} from f_t = 0 (Newton for
// the implicit model, the explicit map otherwise)
// ---------------------------------------------------------------------------
__device__ inline void rollout(const Ctx& c, const KOpts& o) {
    const int n = c.n, nx = c.nx, T = c.T;
    for (int i = threadIdx.x; i < T * n; i += blockDim.x) {
        const int t = i / n, j = i % n;
        c.zb[i] = (j >= nx) ? c.refv(t, j) : (t == 0 ? c.x0[j] : 0.f);
    }
    __syncthreads();
    if (c.model == MODEL_LINEAR) {
        const float* A = c.dyn;
        const float* B = c.dyn + nx * nx;
        for (int t = 0; t < c.N; ++t) {
            const float* z = c.zb + t * n;
            for (int k = threadIdx.x; k < nx; k += blockDim.x) {
                float a = c.bv ? c.bv[k] : 0.f;
                for (int j = 0; j < nx; ++j) a += A[k * nx + j] * z[j];
                for (int j = 0; j < c.nu; ++j) a += B[k * c.nu + j] * z[nx + j];
                c.zb[(t + 1) * n + k] = a;
            }
            __syncthreads();
        }
        return;
    }
    if (c.model == MODEL_SRB) {   // explicit RK4 map, one stage after the other
        if (threadIdx.x == 0)
            for (int t = 0; t < c.N; ++t) {
                float xn[12];
                srb_rk4<float>(c.zb + t * n, c.zb + t * n + 12, c.dyn, xn, nullptr, 0);
                for (int k = 0; k < 12; ++k) c.zb[(t + 1) * n + k] = xn[k];
            }
        __syncthreads();
        return;
    }
    if (threadIdx.x == 0) {
        float f[6], Am[6 * 8], Ap[6 * 8], M[36], xn[6], zn[8];
        for (int t = 0; t < c.N; ++t) {
            const float* z = c.zb + t * n;
            if (c.model == MODEL_QUAD) {
                quad_rk4<float>(z, z + 6, c.dyn, xn, nullptr, nullptr);
            } else if (c.model == MODEL_DI) {
                const float dt = c.dyn[0];
                xn[0] = z[0] + dt * z[2] + 0.5f * dt * dt * z[4];
                xn[1] = z[1] + dt * z[3] + 0.5f * dt * dt * z[5];
                xn[2] = z[2] + dt * z[4];
                xn[3] = z[3] + dt * z[5];
            } else {  // bicycle: explicit Euler predictor + Newton on f_t(z_t, x_{t+1}) = 0
                float fc[6];
                bicycle_fc<float>(z, z + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fc, nullptr, nullptr);
                for (int k = 0; k < 6; ++k) xn[k] = z[k] + c.dyn[0] * fc[k];
                for (int it = 0; it < o.newton_steps; ++it) {
                    for (int k = 0; k < 6; ++k) zn[k] = xn[k];
                    zn[6] = c.zb[(t + 1) * n + 6];
                    zn[7] = c.zb[(t + 1) * n + 7];
                    stage_dyn(c, t, z, zn, f, Am, Ap);
                    for (int k = 0; k < 6; ++k)
                        for (int j = 0; j < 6; ++j) M[k * 6 + j] = Ap[k * n + j];
                    small_solve(M, f, 6);
                    for (int k = 0; k < 6; ++k) xn[k] -= f[k];
                }
            }
            for (int k = 0; k < nx; ++k) c.zb[(t + 1) * n + k] = xn[k];
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// QP approximation at the SQP iterate zb (App. B), written in the coordinates
// d = x - zb of the step (an affine change of variables that leaves every
// ADMM iterate, residual and multiplier unchanged):
//   Am, Ap, G                  Jacobian blocks at zb
//   cv  = c - C zb             (x_init - zb_0; -f_t(zb))
//   qv  = q + P zb             (the cost gradient at zb)
//   glo, ghi = lo - g(zb), hi - g(zb)
// and, for the absolute-coordinate normalisers of the termination test and
// the rho rule, czb = C zb, gzb = G zb; fv = f(zb) and gv = g(zb) for the
// merit / KKT evaluations.
// ---------------------------------------------------------------------------
__device__ inline void linearize(const Ctx& c) {
    const int n = c.n, nx = c.nx, ng = c.ng, N = c.N, T = c.T;
    const bool cA = model_const_Am(c.model), cP = model_const_Ap(c.model), cG = model_const_G(c.model);
    // constant blocks
    if (cA) {
        if (c.model == MODEL_LINEAR) {
            const float* A = c.dyn;
            const float* B = c.dyn + nx * nx;
            for (int i = threadIdx.x; i < nx * n; i += blockDim.x) {
                const int k = i / n, j = i % n;
                c.Am[i] = j < nx ? A[k * nx + j] : B[k * c.nu + (j - nx)];
            }
        } else if (threadIdx.x == 0) {  // double integrator, ZOH
            const float dt = c.dyn[0];
            for (int i = 0; i < nx * n; ++i) c.Am[i] = 0.f;
            for (int k = 0; k < 4; ++k) c.Am[k * n + k] = 1.f;
            c.Am[0 * n + 2] = dt; c.Am[1 * n + 3] = dt;
            c.Am[0 * n + 4] = 0.5f * dt * dt; c.Am[1 * n + 5] = 0.5f * dt * dt;
            c.Am[2 * n + 4] = dt; c.Am[3 * n + 5] = dt;
        }
    }
    if (cP)
        for (int i = threadIdx.x; i < nx * n; i += blockDim.x) {
            const int k = i / n, j = i % n;
            c.Ap[i] = (k == j) ? -1.f : 0.f;
        }
    if (cG && threadIdx.x == 0) {
        float g[64];
        stage_con(c, c.zb, g, c.Gm);
    }
    __syncthreads();  // constant A^-, A^+, G visible to every thread
    // dynamics residual at zb (and the per-stage Jacobians of nonlinear models)
    if (model_linear_dyn(c.model)) {
        for (int i = threadIdx.x; i < N * nx; i += blockDim.x) {
            const int t = i / nx, k = i % nx;
            const float* zt = c.zb + t * n;
            float a = -c.zb[(t + 1) * n + k];
            if (c.model == MODEL_LINEAR) {
                const float* A = c.dyn;
                const float* B = c.dyn + nx * nx;
                if (c.bv) a += c.bv[k];
                for (int j = 0; j < nx; ++j) a += A[k * nx + j] * zt[j];
                for (int j = 0; j < c.nu; ++j) a += B[k * c.nu + j] * zt[nx + j];
            } else {
                const float dt = c.dyn[0];
                const float v[4] = {zt[0] + dt * zt[2] + 0.5f * dt * dt * zt[4], zt[1] + dt * zt[3] + 0.5f * dt * dt * zt[5],
                                    zt[2] + dt * zt[4], zt[3] + dt * zt[5]};
                a += v[k];
            }
            c.fv[(t + 1) * nx + k] = a;
        }
    } else {
        for (int t = threadIdx.x; t < N; t += blockDim.x) {
            float Apq[6 * 8];
            float f[12];
            stage_dyn(c, t, c.zb + t * n, c.zb + (t + 1) * n, f, c.Am + t * c.amS,
                      cP ? Apq : c.Ap + t * c.apS);
            for (int k = 0; k < nx; ++k) c.fv[(t + 1) * nx + k] = f[k];
        }
    }
    for (int k = threadIdx.x; k < nx; k += blockDim.x) c.fv[k] = c.zb[k] - c.x0[k];
    // constraints at zb
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        float g[64];
        stage_con(c, c.zb + t * n, g, cG ? nullptr : c.Gm + t * c.gS);
        for (int r = 0; r < ng; ++r) {
            c.gv[t * ng + r] = g[r];
            c.glo[t * ng + r] = c.lob(t, r) - g[r];
            c.ghi[t * ng + r] = c.hib(t, r) - g[r];
        }
    }
    // cost gradient at zb
    for (int e = threadIdx.x; e < T * n; e += blockDim.x) {
        const int t = e / n, j = e % n;
        float gr = c.Cw(t, j) * (c.zb[e] - c.refv(t, j)) + c.linv(t, j);
        if (j >= nx) {
            const float w = c.W(j - nx);
            if (t < N) gr += w * (c.zb[e] - c.zb[e + n]);
            if (t > 0) gr -= w * (c.zb[e - n] - c.zb[e]);
        }
        c.qv[e] = gr;
    }
    __syncthreads();  // per-stage Jacobians and f visible
    for (int e = threadIdx.x; e < T * nx; e += blockDim.x) {
        c.czb[e] = Cx_entry(c, c.zb, e / nx, e % nx);
        c.cv[e] = -c.fv[e];
    }
    for (int e = threadIdx.x; e < T * ng; e += blockDim.x) c.gzb[e] = Gx_entry(c, c.zb, e / ng, e % ng);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Dense n x n block products for n a multiple of 4: register tiles of 4 x 4
// entries per thread with 128-bit loads (shared or global memory).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 ldv4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void stv4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
// acc[a][b] += sum_k X[k][i0 + a] Y[k][j0 + b]   (X, Y: K rows of length ld)
__device__ __forceinline__ void tile_xty(float (&acc)[4][4], const float* X, const float* Y, int K, int ld,
                                         int i0, int j0) {
    for (int k = 0; k < K; ++k) {
        const float4 x = ldv4(X + k * ld + i0), y = ldv4(Y + k * ld + j0);
        const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xs[a], ys[b], acc[a][b]);
    }
}
// acc[a][b] += sum_k X[i0 + a][k] Y[j0 + b][k]   (rows of length ld, K % 4 == 0)
__device__ __forceinline__ void tile_xyt(float (&acc)[4][4], const float* X, const float* Y, int K, int ld,
                                         int i0, int j0) {
    for (int k = 0; k < K; k += 4) {
        float4 xr[4], yr[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) xr[a] = ldv4(X + (i0 + a) * ld + k);
#pragma unroll
        for (int b = 0; b < 4; ++b) yr[b] = ldv4(Y + (j0 + b) * ld + k);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float s = acc[a][b];
                s = fmaf(xr[a].x, yr[b].x, s);
                s = fmaf(xr[a].y, yr[b].y, s);
                s = fmaf(xr[a].z, yr[b].z, s);
                s = fmaf(xr[a].w, yr[b].w, s);
                acc[a][b] = s;
            }
    }
}

// 4 x 4 inverse of a symmetric positive definite block in registers by
// Gauss-Jordan sweeps (no pivoting; see gj_inverse); bad is set if a pivot is
// not positive (it is then taken as 1).
__device__ __forceinline__ void inv4_spd(float (&M)[4][4], bool& bad) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float p = M[k][k];
        if (!(p > 0.f)) {
            bad = true;
            p = 1.f;
        }
        const float ip = 1.f / p;
        float c[4], r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            c[q] = M[q][k];
            r[q] = M[k][q];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (i == k) M[i][j] = (j == k) ? ip : r[j] * ip;
                else if (j == k) M[i][j] = -c[i] * ip;
                else M[i][j] = fmaf(-c[i] * ip, r[j], M[i][j]);
            }
    }
}

// In-place inverse of the symmetric positive definite n x n matrix A (n % 4 == 0,
// row-major) by block Gauss-Jordan sweeps over the 4 x 4 pivot blocks
// K = 4s .. 4s+3 (no pivoting: the pivot blocks are Schur complements of an SPD
// matrix).  With P = A_KK, column block C = A_:K and row block R = A_K: before
// the sweep:
//   A_KK <- P^-1,  A_Kj <- P^-1 R_j,  A_iK <- -C_i P^-1,  A_ij <- A_ij - C_i P^-1 R_j.
// Each sweep: the pivot inverse and P^-1 R into snap (8n + 16 floats), a
// barrier, the update of every float4 group, a barrier.  A pivot that is not
// positive sets *flag.
__device__ inline void gj_inverse(float* A, int n, float* snap, int* flag) {
    const int nq = n >> 2, tid = threadIdx.x;
    float* Cs = snap;            // n x 4: column block of the sweep
    float* Rp = snap + 4 * n;    // 4 x n: P^-1 R
    float* Pi = snap + 8 * n;    // 4 x 4: P^-1
    // the thread's float4 groups g = tid + m nth, walked as (row i, group jq) without divisions
    const int i_first = tid / nq, q_first = tid % nq;
    const int di = blockDim.x / nq, dq = blockDim.x % nq;
    for (int s = 0; s < nq; ++s) {
        const int k0 = s << 2;
        if (tid < n) {
            const float4 cb = ldv4(A + tid * n + k0);
            stv4(Cs + 4 * tid, cb.x, cb.y, cb.z, cb.w);
            const int a = tid / nq, jq = tid % nq;   // tid < n = 4 nq: row a of P^-1 R, group jq
            float P[4][4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float4 r = ldv4(A + (k0 + b) * n + k0);
                P[b][0] = r.x; P[b][1] = r.y; P[b][2] = r.z; P[b][3] = r.w;
            }
            bool bad = false;
            inv4_spd(P, bad);
            if (bad && tid == 0) *flag = 1;
            float pa[4];   // row a of P^-1, selected without dynamic register indexing
#pragma unroll
            for (int b = 0; b < 4; ++b) pa[b] = a == 0 ? P[0][b] : a == 1 ? P[1][b] : a == 2 ? P[2][b] : P[3][b];
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float4 r = ldv4(A + (k0 + b) * n + 4 * jq);
                const float w = pa[b];
                acc.x = fmaf(w, r.x, acc.x);
                acc.y = fmaf(w, r.y, acc.y);
                acc.z = fmaf(w, r.z, acc.z);
                acc.w = fmaf(w, r.w, acc.w);
            }
            stv4(Rp + a * n + 4 * jq, acc.x, acc.y, acc.z, acc.w);
            if (tid == 0)
#pragma unroll
                for (int b = 0; b < 4; ++b) stv4(Pi + 4 * b, P[b][0], P[b][1], P[b][2], P[b][3]);
        }
        __syncthreads();
        int i = i_first, jq = q_first;
        for (; i < n; i += di, jq += dq) {
            if (jq >= nq) { jq -= nq; ++i; if (i >= n) break; }
            const int j0 = jq << 2, ik = i - k0;
            const bool inK = ik >= 0 && ik < 4;
            float4 v;
            if (jq == s) {
                if (inK) {
                    v = ldv4(Pi + 4 * ik);
                } else {
                    const float4 ci = ldv4(Cs + 4 * i);
                    const float4 p0 = ldv4(Pi), p1 = ldv4(Pi + 4), p2 = ldv4(Pi + 8), p3 = ldv4(Pi + 12);
                    v.x = -(ci.x * p0.x + ci.y * p1.x + ci.z * p2.x + ci.w * p3.x);
                    v.y = -(ci.x * p0.y + ci.y * p1.y + ci.z * p2.y + ci.w * p3.y);
                    v.z = -(ci.x * p0.z + ci.y * p1.z + ci.z * p2.z + ci.w * p3.z);
                    v.w = -(ci.x * p0.w + ci.y * p1.w + ci.z * p2.w + ci.w * p3.w);
                }
            } else if (inK) {
                v = ldv4(Rp + ik * n + j0);
            } else {
                v = ldv4(A + i * n + j0);
                const float4 ci = ldv4(Cs + 4 * i);
                const float c4[4] = {ci.x, ci.y, ci.z, ci.w};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float4 r = ldv4(Rp + a * n + j0);
                    v.x = fmaf(-c4[a], r.x, v.x);
                    v.y = fmaf(-c4[a], r.y, v.y);
                    v.z = fmaf(-c4[a], r.z, v.z);
                    v.w = fmaf(-c4[a], r.w, v.w);
                }
            }
            stv4(A + i * n + j0, v.x, v.y, v.z, v.w);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// S = P + sigma I + rho_f C'C + G' diag(w) G (Theta_t, Phi_t of App. C) and its
// block LDL' factorisation, sequential over stages:
//   Delta_0 = Theta_0,  Om_t = Phi_t Delta_t^{-1},  Delta_{t+1} = Theta_{t+1} - Om_t Phi_t'
// stored as Dinv_t = Delta_t^{-1} (n x n) and Om_t (n x n), row-major.
// w = per-row weights gw (T x ng) if use_gw, else rho_g on every row.
// Returns false if a pivot block was not positive definite (the factors are then
// not usable; the failing pivot is replaced by 1 so that no inf/NaN is produced).
// ---------------------------------------------------------------------------
__device__ inline bool factor_rows(const Ctx& c, const Smem& sm, float sigma, float rho_f, float rho_g,
                            bool use_gw) {
    if (threadIdx.x == 0) sm.flags[1] = 0;
    const int n = c.n, nx = c.nx, ng = c.ng, N = c.N, nn = n * n;
    float* A = sm.A;   // Delta_t -> Cholesky factor L -> Dinv
    float* Li = sm.Bm; // L^{-1}
    float* Ph = sm.Cm; // Phi_t
    for (int t = 0; t <= N; ++t) {
        const float* Amt = c.Amt(t);
        const float* Apm = t > 0 ? c.Apt(t - 1) : nullptr;
        const float* G = c.Gt(t);
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int i = e / n, j = e % n;
            float s = 0.f;
            if (t < N)
                for (int k = 0; k < nx; ++k) s += Amt[k * n + i] * Amt[k * n + j];
            if (t > 0)
                for (int k = 0; k < nx; ++k) s += Apm[k * n + i] * Apm[k * n + j];
            if (t == 0 && i == j && i < nx) s += 1.f;  // A_init' A_init
            float v = rho_f * s;
            for (int r = 0; r < ng; ++r) {
                const float wr = use_gw ? c.gw[t * ng + r] : rho_g;
                v += wr * G[r * n + i] * G[r * n + j];
            }
            if (i == j) v += c.Pdiag(t, i) + sigma;
            if (t > 0) {  // - Om_{t-1} Phi_{t-1}'
                const float* Om = c.Om + (t - 1) * nn;
                float d = 0.f;
                for (int k = 0; k < n; ++k) d += Om[i * n + k] * Ph[j * n + k];
                v -= d;
            }
            A[e] = v;
        }
        __syncthreads();
        // Cholesky (right-looking), lower triangle of A
        for (int k = 0; k < n; ++k) {
            if (threadIdx.x == 0) {
                float d = A[k * n + k];
                if (!(d > 0.f)) { sm.flags[1] = 1; d = 1.f; }
                A[k * n + k] = sqrtf(d);
            }
            __syncthreads();
            const float lkk = A[k * n + k];
            for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * n + k] /= lkk;
            __syncthreads();
            const int m = n - k - 1;
            for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
                const int i = k + 1 + e / m, j = k + 1 + e % m;
                if (j <= i) A[i * n + j] -= A[i * n + k] * A[j * n + k];
            }
            __syncthreads();
        }
        // L^{-1} column by column (thread per column, forward substitution)
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            for (int i = 0; i < j; ++i) Li[i * n + j] = 0.f;
            Li[j * n + j] = 1.f / A[j * n + j];
            for (int i = j + 1; i < n; ++i) {
                float s = 0.f;
                for (int k = j; k < i; ++k) s += A[i * n + k] * Li[k * n + j];
                Li[i * n + j] = -s / A[i * n + i];
            }
        }
        __syncthreads();
        // Dinv = L^{-T} L^{-1}
        float* Dinv = c.Dinv + t * nn;
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int i = e / n, j = e % n;
            const int k0 = i > j ? i : j;
            float s = 0.f;
            for (int k = k0; k < n; ++k) s += Li[k * n + i] * Li[k * n + j];
            A[e] = s;
            Dinv[e] = s;
        }
        __syncthreads();
        if (t < N) {
            // Phi_t = E_t + rho_f A^+_t' A^-_t   ((t+1, t) block of S)
            const float* Apt = c.Apt(t);
            for (int e = threadIdx.x; e < nn; e += blockDim.x) {
                const int i = e / n, j = e % n;
                float s = 0.f;
                for (int k = 0; k < nx; ++k) s += Apt[k * n + i] * Amt[k * n + j];
                float v = rho_f * s;
                if (i == j && i >= nx) v -= c.W(i - nx);
                Ph[e] = v;
            }
            __syncthreads();
            float* Om = c.Om + t * nn;
            for (int e = threadIdx.x; e < nn; e += blockDim.x) {
                const int i = e / n, j = e % n;
                float s = 0.f;
                for (int k = 0; k < n; ++k) s += Ph[i * n + k] * A[k * n + j];
                Om[e] = s;
            }
            __syncthreads();
        }
    }
    const bool ok = sm.flags[1] == 0;
    __syncthreads();
    return ok;
}

// The same factorisation for n a multiple of 4 (n >= 16): Theta_t - Om_{t-1} Phi_{t-1}',
// Phi_t and Om_t = Phi_t Dinv_t (Dinv_t symmetric) as register tiles, the pivot block
// inverted in place by gj_inverse.  Om_{t-1} and Phi_{t-1} stay in shared memory
// for the next stage; Phi_t is formed once when A- and A+ are constant.
__device__ inline bool factor_tiled(const Ctx& c, const Smem& sm, float sigma, float rho_f, float rho_g,
                                    bool use_gw) {
    if (threadIdx.x == 0) sm.flags[1] = 0;
    const int n = c.n, nx = c.nx, ng = c.ng, N = c.N, nn = n * n, nb = n >> 2, ntile = nb * nb;
    float* A = sm.A;     // Delta_t, inverted in place
    float* Om = sm.Bm;   // Om_{t-1}
    float* Ph = sm.Cm;   // Phi_{t-1}
    const bool sel = g_is_selector(c), const_phi = c.amS == 0 && c.apS == 0;
    for (int t = 0; t <= N; ++t) {
        const float* Amt = c.Amt(t);
        const float* Apm = t > 0 ? c.Apt(t - 1) : nullptr;
        const float* G = c.Gt(t);
        // Delta_t = Theta_t - Om_{t-1} Phi_{t-1}'
        for (int w = threadIdx.x; w < ntile; w += blockDim.x) {
            const int i0 = (w / nb) << 2, j0 = (w % nb) << 2;
            float acc[4][4], sch[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = sch[a][b] = 0.f;
            if (t < N) tile_xty(acc, Amt, Amt, nx, n, i0, j0);
            if (t > 0) {
                tile_xty(acc, Apm, Apm, nx, n, i0, j0);
                tile_xyt(sch, Om, Ph, n, n, i0, j0);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                float v[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int i = i0 + a, j = j0 + b;
                    float s = acc[a][b];
                    if (t == 0 && i == j && i < nx) s += 1.f;  // A_init' A_init
                    float u = rho_f * s;
                    if (sel) {
                        if (i == j) {
                            const int r = g_row(c, i);
                            if (r >= 0) u += use_gw ? c.gw[t * ng + r] : rho_g;
                        }
                    } else {
                        for (int r = 0; r < ng; ++r)
                            u += (use_gw ? c.gw[t * ng + r] : rho_g) * G[r * n + i] * G[r * n + j];
                    }
                    if (i == j) u += c.Pdiag(t, i) + sigma;
                    v[b] = u - sch[a][b];
                }
                stv4(A + (i0 + a) * n + j0, v[0], v[1], v[2], v[3]);
            }
        }
        __syncthreads();
        gj_inverse(A, n, sm.red8, sm.flags + 1);
        float* Dinv = c.Dinv + t * nn;
        for (int e = threadIdx.x << 2; e < nn; e += blockDim.x << 2) {
            const float4 d = ldv4(A + e);
            stv4(Dinv + e, d.x, d.y, d.z, d.w);
        }
        if (t < N) {
            if (t == 0 || !const_phi) {   // Phi_t = E_t + rho_f A+_t' A-_t
                const float* Apt = c.Apt(t);
                for (int w = threadIdx.x; w < ntile; w += blockDim.x) {
                    const int i0 = (w / nb) << 2, j0 = (w % nb) << 2;
                    float acc[4][4];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
                    tile_xty(acc, Apt, Amt, nx, n, i0, j0);
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        float v[4];
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const int i = i0 + a, j = j0 + b;
                            v[b] = rho_f * acc[a][b];
                            if (i == j && i >= nx) v[b] -= c.W(i - nx);
                        }
                        stv4(Ph + (i0 + a) * n + j0, v[0], v[1], v[2], v[3]);
                    }
                }
                __syncthreads();
            }
            // Om_t = Phi_t Dinv_t = Phi_t Dinv_t'  (shared copy for stage t + 1, and the workspace)
            float* Omg = c.Om + t * nn;
            for (int w = threadIdx.x; w < ntile; w += blockDim.x) {
                const int i0 = (w / nb) << 2, j0 = (w % nb) << 2;
                float acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
                tile_xyt(acc, Ph, A, n, n, i0, j0);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    stv4(Om + (i0 + a) * n + j0, acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
                    stv4(Omg + (i0 + a) * n + j0, acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
                }
            }
            __syncthreads();
        }
    }
    const bool ok = sm.flags[1] == 0;
    __syncthreads();
    return ok;
}

__device__ inline bool factor(const Ctx& c, const Smem& sm, float sigma, float rho_f, float rho_g,
                       bool use_gw) {
    if (c.n % 4 == 0 && c.n >= 16) return factor_tiled(c, sm, sigma, rho_f, rho_g, use_gw);
    return factor_rows(c, sm, sigma, rho_f, rho_g, use_gw);
}

// Solve S x = b with the block LDL' factors; b (T x n) is overwritten by the
// forward sweep, the result goes to xo (T x n).
//   forward   b_{t+1} -= Om_t b_t
//   diagonal  x_t = Dinv_t b_t
//   backward  x_t -= Om_t' x_{t+1}
// For n >= 32 (the factors stream from global memory) every block is read
// row-contiguously by whole warps: forward and diagonal rows are dotted by one
// warp each (lanes over the columns, shuffle sum); the backward sweep lets warp
// w accumulate the rows k = w (mod warps) of Om_t' x over its lanes' columns and
// sums the per-warp partials through `red` (warps x 96 floats of shared memory).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies global -> shared (cp.async.bulk, the TMA unit) with
// completion counted on an mbarrier.  Addresses 16-byte aligned, size a
// multiple of 16 bytes.  Waits are bounded: after kMbarSpin polls the wait
// gives up and the caller falls back to reading global memory.
// ---------------------------------------------------------------------------
constexpr unsigned kMbarSpin = 1u << 24;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// thread issuing the copy: expect `bytes` on `bar`, then start the copy
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// wait for phase `parity` of `bar` to complete; false if it did not within kMbarSpin
// polls, or as soon as *abort (shared, may be NULL) is set by a thread that gave up
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          const volatile int* abort = nullptr, unsigned polls = kMbarSpin) {
    for (unsigned k = 0; k < polls; ++k) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
        if (abort && *abort) return false;
    }
    return false;
}

// once per CTA, before the first stream: both mbarriers and the stream state
// (state[3]: polls of a bounded wait, the wait_polls option or kMbarSpin; 0 when
// the caller forces every wait to give up at once)
__device__ inline void block_stream_init(unsigned long long* mbar, int* state, int polls = 0, int force = 0) {
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        mbar_init(mbar + 1, 1);
        fence_mbar_init();
        state[0] = state[1] = state[2] = 0;
        state[3] = force ? 0 : (polls > 0 ? polls : (int)kMbarSpin);
    }
    __syncthreads();
}

// Stream of equally sized blocks (one per step) into two shared buffers: the
// block of step k + 1 is in flight while step k is consumed.  Every thread
// calls get(k) in step order and sync() after using it.
struct BlockStream {
    float* buf[2];
    unsigned long long* bar;
    unsigned phase[2];
    unsigned inflight;   // thread 0: buffers with a copy issued and not yet waited for
    unsigned polls;
    bool ok;
    int* state;   // shared: [0], [1] phase bits of the two mbarriers, [2] set if a wait gave up, [3] polls
    __device__ BlockStream(float* b0, float* b1, unsigned long long* bars, int* st)
        : bar(bars), inflight(0u), state(st) {
        buf[0] = b0;
        buf[1] = b1;
        phase[0] = (unsigned)st[0];
        phase[1] = (unsigned)st[1];
        polls = (unsigned)st[3];
        ok = st[2] == 0;   // after a wait gave up, the rest of the instance reads global memory
    }
    // after the last get / sync of a solve: store the phase bits for the next solve.
    // If a wait gave up, copies may still be in flight into the two buffers, which
    // the factorisation reuses as scratch: thread 0 waits (bounded) for each of them
    // to land before the buffers are released; state[2] = 2 records a copy that
    // did not land (the buffers are then not safe for the rest of the launch, and
    // every later wait of the CTA gives up at once).
    __device__ void finish() {
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int b = 0; b < 2; ++b) {
                if (!(inflight & (1u << b))) continue;
                if (mbar_wait(bar + b, phase[b], nullptr, (unsigned)kMbarSpin)) phase[b] ^= 1u;
                else state[2] = 2;
            }
            inflight = 0u;
            state[0] = (int)phase[0];
            state[1] = (int)phase[1];
            if (!ok && state[2] == 0) state[2] = 1;
        }
        __syncthreads();
    }
    // thread 0: start the copy of `src` into the buffer of step k
    __device__ void issue(int k, const float* src, unsigned bytes) {
        if (threadIdx.x == 0 && ok) {
            fence_proxy_async();
            bulk_load(buf[k & 1], src, bytes, bar + (k & 1));
            inflight |= 1u << (k & 1);
        }
    }
    // every thread: wait for the block of step k; returns the shared copy, or
    // `fallback` (global memory, the same values) once a wait gave up.  Each thread
    // waits on the mbarrier itself; a thread that gives up sets state[2], which ends
    // the other threads' waits, so every thread reads global memory from then on
    // (thread 0 issues no further copies).
    __device__ const float* get(int k, const float* fallback) {
        if (!ok) return fallback;
        const volatile int* gave_up = state + 2;
        if (*gave_up || polls == 0 || !mbar_wait(bar + (k & 1), phase[k & 1], gave_up, polls)) {
            ok = false;
            if (*gave_up == 0) state[2] = 1;
            return fallback;
        }
        phase[k & 1] ^= 1u;
        inflight &= ~(1u << (k & 1));
        return buf[k & 1];
    }
};

// sbuf0/sbuf1 (n^2 floats each), mbar (2 mbarriers) and mstate (4 ints) enable
// the shared-memory block stream; without them the blocks are read from global memory.
__device__ inline void ldl_solve(const Ctx& c, float* b, float* xo, float* red, float* sbuf0 = nullptr,
                                 float* sbuf1 = nullptr, unsigned long long* mbar = nullptr, int* mstate = nullptr) {
    const int n = c.n, N = c.N, nn = n * n;
    if (n >= 32 && red) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const bool k1 = lane + 32 < n, k2 = lane + 64 < n;   // n <= 72 < 96
        // blocks of n^2 floats stream through two shared buffers (n even: whole 16-byte units)
        const bool stream = sbuf0 && mstate && (n % 2 == 0);
        const unsigned bytes = (unsigned)(nn * sizeof(float));
        BlockStream bs(sbuf0, sbuf1, mbar, mstate);
        int k = 0;   // step counter of the stream
        if (stream) bs.issue(k, c.Om, bytes);
        if (n % 4 == 0 && 2 * n <= (int)blockDim.x) {
            // n a multiple of 4: 128-bit loads of the block rows.  Forward and diagonal:
            // two threads per row (float4 groups q = h, h + 2, ...) and one shuffle;
            // backward: thread (column quad cq, part p) sums the rows i = p (mod 8),
            // combined by three shuffle levels.  Shuffles run on whole warps.
            const int nq = n >> 2, tid = threadIdx.x;
            const int ri = tid >> 1, rh = tid & 1;                 // row, half
            const int cq = tid >> 3, cp = tid & 7;                 // column quad, part
            const bool rrow = ri < n, rcol = cq < nq;
            auto rowdot4 = [&](const float* M, const float* v) {  // (M v)_ri over the groups of half rh
                float s0 = 0.f, s1 = 0.f;
                if (rrow) {
                    const float* mr = M + ri * n;
                    for (int q = rh; q < nq; q += 2) {
                        const float4 a = ldv4(mr + 4 * q), x = ldv4(v + 4 * q);
                        s0 = fmaf(a.x, x.x, s0);
                        s1 = fmaf(a.y, x.y, s1);
                        s0 = fmaf(a.z, x.z, s0);
                        s1 = fmaf(a.w, x.w, s1);
                    }
                }
                float sum = s0 + s1;
                sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 1);
                return sum;
            };
            for (int t = 0; t < N; ++t, ++k) {
                if (stream) bs.issue(k + 1, t + 1 < N ? c.Om + (t + 1) * nn : c.Dinv, bytes);
                const float* Om = stream ? bs.get(k, c.Om + t * nn) : c.Om + t * nn;
                const float s = rowdot4(Om, b + t * n);
                if (rrow && rh == 0) b[(t + 1) * n + ri] -= s;
                __syncthreads();
            }
            for (int t = 0; t < c.T; ++t, ++k) {
                if (stream) bs.issue(k + 1, t + 1 < c.T ? c.Dinv + (t + 1) * nn : c.Om + (N - 1) * nn, bytes);
                const float* D = stream ? bs.get(k, c.Dinv + t * nn) : c.Dinv + t * nn;
                const float s = rowdot4(D, b + t * n);
                if (rrow && rh == 0) xo[t * n + ri] = s;
                __syncthreads();
            }
            for (int t = N - 1; t >= 0; --t, ++k) {
                if (stream && t > 0) bs.issue(k + 1, c.Om + (t - 1) * nn, bytes);
                const float* Om = stream ? bs.get(k, c.Om + t * nn) : c.Om + t * nn;
                const float* xn = xo + (t + 1) * n;
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                if (rcol)
                    for (int i = cp; i < n; i += 8) {
                        const float4 a = ldv4(Om + i * n + 4 * cq);
                        const float xi = xn[i];
                        acc.x = fmaf(a.x, xi, acc.x);
                        acc.y = fmaf(a.y, xi, acc.y);
                        acc.z = fmaf(a.z, xi, acc.z);
                        acc.w = fmaf(a.w, xi, acc.w);
                    }
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    acc.x += __shfl_xor_sync(0xFFFFFFFFu, acc.x, o);
                    acc.y += __shfl_xor_sync(0xFFFFFFFFu, acc.y, o);
                    acc.z += __shfl_xor_sync(0xFFFFFFFFu, acc.z, o);
                    acc.w += __shfl_xor_sync(0xFFFFFFFFu, acc.w, o);
                }
                if (rcol && cp == 0) {
                    float* xt = xo + t * n + 4 * cq;
                    xt[0] -= acc.x;
                    xt[1] -= acc.y;
                    xt[2] -= acc.z;
                    xt[3] -= acc.w;
                }
                __syncthreads();
            }
            if (stream) bs.finish();
            return;
        }
        for (int t = 0; t < N; ++t, ++k) {
            if (stream) bs.issue(k + 1, t + 1 < N ? c.Om + (t + 1) * nn : c.Dinv, bytes);
            const float* Om = stream ? bs.get(k, c.Om + t * nn) : c.Om + t * nn;
            const float* w = b + t * n;
            const float w0 = w[lane], w1 = k1 ? w[lane + 32] : 0.f, w2 = k2 ? w[lane + 64] : 0.f;
#pragma unroll 3
            for (int i = warp; i < n; i += nw) {
                const float* row = Om + i * n;
                float s = row[lane] * w0;
                if (k1) s += row[lane + 32] * w1;
                if (k2) s += row[lane + 64] * w2;
                s = warp_sum(s);
                if (lane == 0) b[(t + 1) * n + i] -= s;
            }
            __syncthreads();
        }
        // diagonal: x_t = Dinv_t b_t (the block of step k is Dinv_t)
        for (int t = 0; t < c.T; ++t, ++k) {
            if (stream) bs.issue(k + 1, t + 1 < c.T ? c.Dinv + (t + 1) * nn : c.Om + (N - 1) * nn, bytes);
            const float* D = stream ? bs.get(k, c.Dinv + t * nn) : c.Dinv + t * nn;
            const float* w = b + t * n;
            const float w0 = w[lane], w1 = k1 ? w[lane + 32] : 0.f, w2 = k2 ? w[lane + 64] : 0.f;
#pragma unroll 3
            for (int i = warp; i < n; i += nw) {
                const float* row = D + i * n;
                float s = row[lane] * w0;
                if (k1) s += row[lane + 32] * w1;
                if (k2) s += row[lane + 64] * w2;
                s = warp_sum(s);
                if (lane == 0) xo[t * n + i] = s;
            }
            __syncthreads();
        }
        for (int t = N - 1; t >= 0; --t, ++k) {
            if (stream && t > 0) bs.issue(k + 1, c.Om + (t - 1) * nn, bytes);
            const float* Om = stream ? bs.get(k, c.Om + t * nn) : c.Om + t * nn;
            const float* xn = xo + (t + 1) * n;
            float p0 = 0.f, p1 = 0.f, p2 = 0.f;
#pragma unroll 3
            for (int q = warp; q < n; q += nw) {
                const float* row = Om + q * n;
                const float xq = xn[q];
                p0 += row[lane] * xq;
                if (k1) p1 += row[lane + 32] * xq;
                if (k2) p2 += row[lane + 64] * xq;
            }
            float* rw = red + warp * 96;
            rw[lane] = p0;
            rw[lane + 32] = p1;
            rw[lane + 64] = p2;
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                float s = 0.f;
                for (int q = 0; q < nw; ++q) s += red[q * 96 + i];
                xo[t * n + i] -= s;
            }
            __syncthreads();
        }
        if (stream) bs.finish();
        return;
    }
    for (int t = 0; t < N; ++t) {
        const float* Om = c.Om + t * nn;
        const float* w = b + t * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            float s = 0.f;
            for (int k = 0; k < n; ++k) s += Om[i * n + k] * w[k];
            b[(t + 1) * n + i] -= s;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < c.T * n; e += blockDim.x) {
        const int t = e / n, i = e % n;
        const float* D = c.Dinv + t * nn;
        const float* w = b + t * n;
        float s = 0.f;
        for (int k = 0; k < n; ++k) s += D[i * n + k] * w[k];
        xo[e] = s;
    }
    __syncthreads();
    for (int t = N - 1; t >= 0; --t) {
        const float* Om = c.Om + t * nn;
        const float* xn = xo + (t + 1) * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            float s = 0.f;
            for (int k = 0; k < n; ++k) s += Om[k * n + i] * xn[k];
            xo[t * n + i] -= s;
        }
        __syncthreads();
    }
}

// projection onto [lo, hi] (hard row) or the L1+L2 smoothed projection (soft row)
__device__ __forceinline__ void project(float v, float lo, float hi, float rho_g, float g2,
                                        float g1, float& z, float& xi) {
    if (!(g2 < kInf)) {
        z = fminf(fmaxf(v, lo), hi);
        xi = 0.f;
        return;
    }
    if (v > hi) {
        const float s = fmaxf(0.f, (rho_g * (v - hi) - g1) / (rho_g + g2));
        z = hi + s;
        xi = -s;
    } else if (v < lo) {
        const float s = fmaxf(0.f, (rho_g * (lo - v) - g1) / (rho_g + g2));
        z = lo - s;
        xi = s;
    } else {
        z = v;
        xi = 0.f;
    }
}

// ---------------------------------------------------------------------------
// The linear model's C: A- = [A B], the same block at every stage, and
// A+ = [-I 0].  With n and nx multiples of 4 the C' and C products of all
// stages run as register tiles (4 stages x 4 entries per thread, 128-bit
// loads of A- rows and of the stage vectors) instead of one serial dot
// product per entry.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool tiled_linear(const Ctx& c) {
    return c.model == MODEL_LINEAR && (c.n & 3) == 0 && (c.nx & 3) == 0 && c.amS == 0;
}
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// acc[b][a] += sum over the 4 columns of rows a of `ar` dotted with v[b]
__device__ __forceinline__ void tile_fma(float (&acc)[4][4], const float4 (&ar)[4], const float4 (&v)[4]) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float s = acc[b][a];
            s = fmaf(ar[a].x, v[b].x, s);
            s = fmaf(ar[a].y, v[b].y, s);
            s = fmaf(ar[a].z, v[b].z, s);
            s = fmaf(ar[a].w, v[b].w, s);
            acc[b][a] = s;
        }
}

// (C'W)_{t,j} for every stage t and entry j, W: T rows of nx; f(t, j, value).
// Tile (t0, j0): stages t0..t0+3, entries j0..j0+3;
// (C'W)_{t,j} = [t < N] (A-' W_{t+1})_j + [j < nx] ([t = 0] W_{0,j} - [t > 0] W_{t,j}).
template <class F>
__device__ __forceinline__ void ct_tiled(const Ctx& c, const float* W, F f) {
    const int n = c.n, nx = c.nx, T = c.T, N = c.N;
    const int nj = n >> 2, ntile = nj * ((T + 3) >> 2);
    const float* Am = c.Amt(0);
    for (int w = threadIdx.x; w < ntile; w += blockDim.x) {
        const int j0 = (w % nj) << 2, t0 = (w / nj) << 2;
        float acc[4][4];
        const float* wr[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            wr[b] = W + min(t0 + b + 1, N) * nx;   // stages t >= N take no A- term (zeroed below)
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[b][a] = 0.f;
        }
        for (int k = 0; k < nx; k += 4) {
            float4 ar[4], v[4];   // ar[a] = column j0 + a of A- over rows k..k+3
            const float4 r0 = ldg4(Am + (k + 0) * n + j0), r1 = ldg4(Am + (k + 1) * n + j0);
            const float4 r2 = ldg4(Am + (k + 2) * n + j0), r3 = ldg4(Am + (k + 3) * n + j0);
            ar[0] = make_float4(r0.x, r1.x, r2.x, r3.x);
            ar[1] = make_float4(r0.y, r1.y, r2.y, r3.y);
            ar[2] = make_float4(r0.z, r1.z, r2.z, r3.z);
            ar[3] = make_float4(r0.w, r1.w, r2.w, r3.w);
#pragma unroll
            for (int b = 0; b < 4; ++b) v[b] = ld4(wr[b] + k);
            tile_fma(acc, ar, v);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int t = t0 + b;
            if (t >= T) break;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int j = j0 + a;
                float s = t < N ? acc[b][a] : 0.f;
                if (j < nx) s += (t == 0) ? W[j] : -W[t * nx + j];
                f(t, j, s);
            }
        }
    }
}

// (C X)_{r,k} for rows r = 0..N, k < nx, X: T rows of n; f(e = r nx + k, value).
// Row 0 is X_0; row t + 1 is A- X_t - X_{t+1}.  Tile (t0, k0): stages t0..t0+3
// (rows t0+1..t0+4), rows k0..k0+3 of A-.
template <class F>
__device__ __forceinline__ void c_tiled(const Ctx& c, const float* X, F f) {
    const int n = c.n, nx = c.nx, N = c.N;
    const int nk = nx >> 2, ntile = nk * ((N + 3) >> 2);
    const float* Am = c.Amt(0);
    for (int w = threadIdx.x; w < ntile; w += blockDim.x) {
        const int k0 = (w % nk) << 2, t0 = (w / nk) << 2;
        float acc[4][4];
        const float* xr[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            xr[b] = X + min(t0 + b, N - 1) * n;
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[b][a] = 0.f;
        }
        for (int j = 0; j < n; j += 4) {
            float4 ar[4], v[4];   // ar[a] = row k0 + a of A- over columns j..j+3
#pragma unroll
            for (int a = 0; a < 4; ++a) ar[a] = ldg4(Am + (k0 + a) * n + j);
#pragma unroll
            for (int b = 0; b < 4; ++b) v[b] = ld4(xr[b] + j);
            tile_fma(acc, ar, v);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int t = t0 + b;
            if (t >= N) break;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int k = k0 + a;
                f((t + 1) * nx + k, acc[b][a] - X[(t + 1) * n + k]);
            }
        }
    }
    for (int k = threadIdx.x; k < nx; k += blockDim.x) f(k, X[k]);
}

// one ADMM iteration (Algorithm 3) in increment form.  With p_f = C x - c
// (tracked, never recomputed from absolute values) and p_g = G x - z_g, the
// primal system S xt = eta is solved for the increment dx = xt - x:
//     S dx = eta - S x = -(P x + q) - C'(y_f + rho_f p_f) - G'(y_g + rho_g p_g),
// then z~_f - c = p_f + C dx, z~_g = G x + G dx, and the relaxation, projection
// and dual updates of Algorithm 3 follow.  In exact arithmetic this is the
// paper's iteration; in FP32 the rho_f-scaled terms only ever multiply small,
// accurately formed differences.
__device__ inline void admm_iter(const Ctx& c, const KOpts& o, float rho_bar, const Smem& sm) {
    const int n = c.n, nx = c.nx, ng = c.ng, T = c.T;
    const float rho_f = 1e3f * rho_bar, rho_g = rho_bar, alpha = o.alpha;
    const bool tiled = tiled_linear(c);
    for (int e = threadIdx.x; e < T * ng; e += blockDim.x) c.pg[e] = Gx_entry(c, c.x, e / ng, e % ng) - c.zg[e];
    if (tiled)   // w = y_f + rho_f p_f into xt (free until the solve writes it)
        for (int e = threadIdx.x; e < T * nx; e += blockDim.x) c.xt[e] = c.yf[e] + rho_f * c.pf[e];
    __syncthreads();
    if (tiled) {
        ct_tiled(c, c.xt, [&](int t, int j, float ctw) {
            float e = -(Px_entry(c, c.x, t, j) + c.qv[t * n + j]) - ctw;
            const int r = g_row(c, j);   // the linear model's G selects controls
            if (r >= 0) e -= c.yg[t * ng + r] + rho_g * c.pg[t * ng + r];
            c.eta[t * n + j] = e;
        });
    } else for (int e = threadIdx.x; e < T * n; e += blockDim.x) {
        const int t = e / n, j = e % n;
        float s = -(Px_entry(c, c.x, t, j) + c.qv[e]);
        s -= Ct_entry(c, t, j, [&](int r, int k) { return c.yf[r * nx + k] + rho_f * c.pf[r * nx + k]; });
        if (g_is_selector(c)) {
            const int r = g_row(c, j);
            if (r >= 0) s -= c.yg[t * ng + r] + rho_g * c.pg[t * ng + r];
        } else {
            const float* G = c.Gt(t);
            for (int r = 0; r < ng; ++r) s -= G[r * n + j] * (c.yg[t * ng + r] + rho_g * c.pg[t * ng + r]);
        }
        c.eta[e] = s;
    }
    __syncthreads();
    ldl_solve(c, c.eta, c.xt, sm.red8, sm.A, sm.Bm, sm.mbar, sm.flags + 12);
    if (tiled) {
        c_tiled(c, c.xt, [&](int e, float cd) {
            c.yf[e] += rho_f * alpha * (c.pf[e] + cd);
            c.pf[e] += alpha * cd;
        });
    } else for (int e = threadIdx.x; e < T * nx; e += blockDim.x) {
        const float cd = Cx_entry(c, c.xt, e / nx, e % nx);
        c.yf[e] += rho_f * alpha * (c.pf[e] + cd);
        c.pf[e] += alpha * cd;
    }
    for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
        const int t = e / ng, r = e % ng;
        const float zh = c.zg[e] + alpha * (c.pg[e] + Gx_entry(c, c.xt, t, r));
        const float v = zh + c.yg[e] / rho_g;
        float zn, xn;
        project(v, c.glo[e], c.ghi[e], rho_g, c.gam2(r), c.gam1(r), zn, xn);
        c.yg[e] += rho_g * (zh - zn);
        c.zg[e] = zn;
        c.xi[e] = xn;
    }
    for (int e = threadIdx.x; e < T * n; e += blockDim.x) c.x[e] += alpha * c.xt[e];
    __syncthreads();
}

// slack-row dual residual (second block of r_dual)
__device__ __forceinline__ float slack_res(float xi, float y, float g2, float g1) {
    if (xi != 0.f) return g2 * xi + (xi > 0.f ? g1 : -g1) + y;
    return fmaxf(0.f, fabsf(y) - g1);
}

struct Res {
    float r_prim, r_dual, pn, dn;
};

// residuals of Eq. (admm:residuals) and the normalisers of
// Eq. (admm:termination:slack), the latter in absolute coordinates
// (x_abs = zb + x, z_abs = z_g + G zb, c_abs = c + C zb, q_abs = q - P zb).
__device__ inline Res residuals(const Ctx& c, const Smem& sm) {
    const int n = c.n, nx = c.nx, ng = c.ng, T = c.T;
    float v[4] = {0.f, 0.f, 0.f, 0.f};  // r_prim, r_dual, primal norm, dual norm
    for (int e = threadIdx.x; e < T * nx; e += blockDim.x) {
        const float cabs = c.cv[e] + c.czb[e];
        v[0] = fmaxf(v[0], fin(c.pf[e]));
        v[2] = fmaxf(v[2], fmaxf(fin(c.pf[e] + cabs), fin(cabs)));
    }
    for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
        const int t = e / ng, r = e % ng;
        const float gx = Gx_entry(c, c.x, t, r);
        v[0] = fmaxf(v[0], fin(gx - c.zg[e]));
        v[2] = fmaxf(v[2], fmaxf(fin(gx + c.gzb[e]), fin(c.zg[e] + c.gzb[e])));
        const float g2 = c.gam2(r);
        if (g2 < kInf) {
            v[1] = fmaxf(v[1], fin(slack_res(c.xi[e], c.yg[e], g2, c.gam1(r))));
            v[3] = fmaxf(v[3], fmaxf(fin(g2 * c.xi[e]), fin(c.yg[e])));
        }
    }
    for (int e = threadIdx.x; e < T * n; e += blockDim.x) {
        const int t = e / n, j = e % n;
        const float px = Px_entry(c, c.x, t, j);
        const float pzb = Px_entry(c, c.zb, t, j);
        // C'y_f + G'y_g accumulated in FP64: with up to 2 nx + ng terms, an FP32 sum
        // would put a rounding floor near the termination tolerance under the residual
        double atyd = 0.0;
        if (t == 0 && j < nx) atyd += (double)c.yf[j];
        if (t < c.N) {
            const float* Am = c.Amt(t);
            for (int k = 0; k < nx; ++k) atyd += (double)Am[k * n + j] * (double)c.yf[(t + 1) * nx + k];
        }
        if (t > 0) {
            const float* Ap = c.Apt(t - 1);
            for (int k = 0; k < nx; ++k) atyd += (double)Ap[k * n + j] * (double)c.yf[t * nx + k];
        }
        if (g_is_selector(c)) {
            const int r = g_row(c, j);
            if (r >= 0) atyd += (double)c.yg[t * ng + r];
        } else {
            const float* G = c.Gt(t);
            for (int r = 0; r < ng; ++r) atyd += (double)G[r * n + j] * (double)c.yg[t * ng + r];
        }
        const float aty = (float)atyd;
        v[1] = fmaxf(v[1], fin((float)((double)px + (double)c.qv[e] + atyd)));
        v[3] = fmaxf(v[3], fmaxf(fmaxf(fin(px + pzb), fin(aty)), fin(c.qv[e] - pzb)));
    }
    cta_max_k<4>(v, sm.red);
    return {v[0], v[1], v[2], v[3]};
}

// ---------------------------------------------------------------------------
// merit contributions of stage t at the point za = zb + a dz, xia = xib + a dxi
// (Appendix D): cost (incl. slack penalty) and constraint violation V.
// ---------------------------------------------------------------------------
__device__ inline void stage_merit(const Ctx& c, int t, float a, double& cost, double& viol, double& scale) {
    const int n = c.n, nx = c.nx, ng = c.ng;
    float z[72], zn[72], f[64], g[64];
    for (int j = 0; j < n; ++j) z[j] = c.zb[t * n + j] + a * c.x[t * n + j];
    double cs = 0.0, vs = 0.0;
    for (int j = 0; j < n; ++j) {
        const float d = z[j] - c.refv(t, j);
        cs += 0.5 * (double)c.Cw(t, j) * d * d + (double)c.linv(t, j) * z[j];
        scale += 0.5 * (double)c.Cw(t, j) * d * d + fabs((double)c.linv(t, j) * z[j]) + 2.0 * fabs((double)z[j]);
    }
    if (t < c.N) {
        for (int j = 0; j < n; ++j) zn[j] = c.zb[(t + 1) * n + j] + a * c.x[(t + 1) * n + j];
        for (int k = 0; k < c.nu; ++k) {
            const float d = z[nx + k] - zn[nx + k];
            cs += 0.5 * (double)c.W(k) * d * d;
        }
        stage_dyn(c, t, z, zn, f, nullptr, nullptr);
        for (int k = 0; k < nx; ++k) vs += fabs((double)f[k]);
    }
    if (t == 0)
        for (int k = 0; k < nx; ++k) vs += fabs((double)z[k] - (double)c.x0[k]);
    stage_con(c, z, g, nullptr);
    for (int r = 0; r < ng; ++r) {
        const float xi = c.xib[t * ng + r] + a * (c.xi[t * ng + r] - c.xib[t * ng + r]);
        const float g2 = c.gam2(r);
        if (g2 < kInf) cs += 0.5 * (double)g2 * xi * xi + (double)c.gam1(r) * fabs((double)xi);
        const double gx = (double)g[r] + xi;
        vs += fmax(gx - (double)c.hib(t, r), 0.0) + fmax((double)c.lob(t, r) - gx, 0.0);
    }
    cost += cs;
    viol += vs;
    scale += fabs(cs);
}

// returns the chosen step (Appendix D)
__device__ inline float linesearch(const Ctx& c, const KOpts& o, const Smem& sm, float ystar_inf) {
    const int n = c.n, nx = c.nx, ng = c.ng, T = c.T;
    const int K = o.n_ls < 1 ? 1 : (o.n_ls > kMaxLs ? kMaxLs : o.n_ls);
    if (K == 1) return 1.f;
    // directional derivative of the cost at zb along the step d = x (qv is the gradient at zb)
    double gd = 0.0;
    for (int e = threadIdx.x; e < T * n; e += blockDim.x) gd += (double)c.qv[e] * (double)c.x[e];
    for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
        const int r = e % ng;
        const float g2 = c.gam2(r);
        if (g2 < kInf) {
            const float x0 = c.xib[e], dx = c.xi[e] - c.xib[e];
            gd += (double)g2 * x0 * dx + (double)c.gam1(r) * (x0 != 0.f ? (x0 > 0.f ? dx : -dx) : fabsf(dx));
        }
    }
    gd = cta_sum_d(gd, sm.redd);
    // merit parts at a = 0 and at every candidate: thread-strided over (k, t)
    for (int e = threadIdx.x; e < 2 * (K + 1) + 1; e += blockDim.x) sm.lsacc[e] = 0.0;
    __syncthreads();
    for (int e = threadIdx.x; e < (K + 1) * T; e += blockDim.x) {
        const int k = e / T, t = e % T;
        const float a = k == 0 ? 0.f : ldexpf(1.f, -(k - 1));
        double cs = 0.0, vs = 0.0, sc = 0.0;
        stage_merit(c, t, a, cs, vs, sc);
        if (k == 0) atomicAdd(&sm.lsacc[2 * (K + 1)], sc);
        atomicAdd(&sm.lsacc[2 * k], cs);
        atomicAdd(&sm.lsacc[2 * k + 1], vs);
    }
    __syncthreads();
    const double l0 = sm.lsacc[0], V0 = sm.lsacc[1];
    const double mu = fmax(gd / (0.5 * fmax(V0, (double)o.eps_c)), (double)ystar_inf + 1e-4);
    const double phi0 = l0 + mu * V0;
    const double D = gd - mu * V0;
    // FP32 evaluation error of the merit: differences below it are ties, and a
    // tie satisfies the Armijo test (4 units of FP32 rounding on the magnitude
    // of every term that enters phi)
    const double tau = 4.0 * 5.9604644775390625e-08 * sm.lsacc[2 * (K + 1)] * fmax(1.0, mu);
    float chosen = -1.f, best = 0.f;
    double best_phi = INFINITY;
    for (int k = 1; k <= K; ++k) {
        const float a = ldexpf(1.f, -(k - 1));
        const double ph = sm.lsacc[2 * k] + mu * sm.lsacc[2 * k + 1];
        if (isfinite(ph) && ph <= phi0 + (double)o.ls_eta * a * D + tau) { chosen = a; break; }
    }
    if (chosen < 0.f) {
        for (int k = 1; k <= K; ++k) {
            const float a = ldexpf(1.f, -(k - 1));
            const double ph = sm.lsacc[2 * k] + mu * sm.lsacc[2 * k + 1];
            if (isfinite(ph) && ph < best_phi) { best_phi = ph; best = a; }
        }
        chosen = best;
    }
    __syncthreads();
    return chosen;
}

// KKT residual of Eq. (sqp_stop) at (zb, xib, yfb, ygb) using the current
// linearisation (Am, Ap, G, fv, gv at zb)
__device__ inline float kkt(const Ctx& c, const Smem& sm) {
    const int n = c.n, nx = c.nx, ng = c.ng, T = c.T;
    float v[1] = {0.f};
    for (int e = threadIdx.x; e < T * n; e += blockDim.x) {
        const int t = e / n, j = e % n;
        float gr = c.Cw(t, j) * (c.zb[e] - c.refv(t, j)) + c.linv(t, j);
        if (j >= nx) {
            const float w = c.W(j - nx);
            if (t < c.N) gr += w * (c.zb[e] - c.zb[e + n]);
            if (t > 0) gr -= w * (c.zb[e - n] - c.zb[e]);
        }
        gr += Ct_entry(c, t, j, [&](int r, int k) { return c.yfb[r * nx + k]; });
        const float* G = c.Gt(t);
        for (int r = 0; r < ng; ++r) gr += G[r * n + j] * c.ygb[t * ng + r];
        v[0] = fmaxf(v[0], fin(gr));
    }
    for (int e = threadIdx.x; e < T * nx; e += blockDim.x) v[0] = fmaxf(v[0], fin(c.fv[e]));
    for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
        const int t = e / ng, r = e % ng;
        const float g2 = c.gam2(r);
        if (g2 < kInf) v[0] = fmaxf(v[0], fin(slack_res(c.xib[e], c.ygb[e], g2, c.gam1(r))));
        const float gx = c.gv[e] + c.xib[e];
        v[0] = fmaxf(v[0], fmaxf(gx - c.hib(t, r), c.lob(t, r) - gx));
    }
    cta_max_k<1>(v, sm.red);
    return v[0];
}

// initial primal-dual point from a solution in the padded layout
__device__ inline void read_warm(const Ctx& c, const KLayout& L, const KSol& out, int i) {
    const long long Ts = L.Nmax + 1;
    const float* z = out.z + i * Ts * L.n;
    const float* xi = out.xi + i * Ts * L.ng;
    const float* yf = out.yf + i * Ts * L.nx;
    const float* yg = out.yg + i * Ts * L.ng;
    for (int e = threadIdx.x; e < c.T * c.n; e += blockDim.x) c.zb[e] = z[(e / c.n) * L.n + e % c.n];
    for (int e = threadIdx.x; e < c.T * c.ng; e += blockDim.x) {
        c.xib[e] = xi[(e / c.ng) * L.ng + e % c.ng];
        c.ygb[e] = yg[(e / c.ng) * L.ng + e % c.ng];
    }
    for (int e = threadIdx.x; e < c.T * c.nx; e += blockDim.x) c.yfb[e] = yf[(e / c.nx) * L.nx + e % c.nx];
    __syncthreads();
}

}  // namespace tmpc
