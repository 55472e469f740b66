// Direct adjoint solve of the backward pass (Algorithm 2, Section III-D,
// Appendix E) for the small models, in FP64.
//
// The active-set KKT system of Eq. (bwd:slack_reduced_system),
//     [ H_s  C'  G_h' ] [eta_x]   [b]
//     [ C    0   0    ] [eta_f] = [0]
//     [ G_h  0   0    ] [eta_h]   [0]
// (H_s = H + G_s' diag(gamma2) G_s with the slack-active rows eliminated,
// b = dL/dz - G_s' dL/dxi, G_h the hard-active rows), is ordered stage by
// stage with the multipliers interleaved: block t = [lambda_t (the nx rows of
// C that start at stage t: x_0 = x_init for t = 0, f_{t-1} = 0 otherwise),
// eta_x,t (n), eta_h,t (ng rows; an inactive row is an identity row)].  In this
// order the matrix is block tridiagonal: the diagonal block D_t holds H_s,tt,
// A^+_{t-1} (A_init at t = 0) and G_h,t; the coupling of block t to block t-1
// is P_t = [A^-_{t-1}; H_{t,t-1}] on the eta_x,t-1 columns.  It is symmetric
// and indefinite, and is factored by block LDL' without pivoting across blocks:
//     S_0 = D_0,   S_t = D_t - P_t (S_{t-1}^-1)_xx P_t',
// each S_t inverted by Gauss-Jordan elimination with partial pivoting inside
// the block (one warp, lane r holding row r).  The forward sweep also carries
// y_t = r_t - P_t (S_{t-1}^-1 y_{t-1})_x; the backward sweep returns
// x_t = S_t^-1 (y_t - P_{t+1}' x_{t+1}).  One factorisation, no refinement.
//
// FP64 because the active-set KKT of a constrained OCP can be ill-conditioned
// (condition numbers near 1e10 on the racing model where bound rows nearly
// repeat the dynamics rows), beyond what an FP32 factorisation resolves.  If a
// pivot block is numerically singular (the active rows are linearly dependent),
// the solve is repeated with -1e-10 on the multiplier diagonal.
#pragma once
#include "tmpc_fast.cuh"

namespace tmpc {
namespace fast {

// doubles of the FP64 workspace per stage: S_t^-1 (MB^2), y_t (MB), then the FP64
// Jacobian A^-_t (NX x N) and the dense row of G_t (N), then (exact Hessian) the
// constraint-curvature blocks of the Lagrangian: Ccur_tt from f_t and the track row,
// C'_tt from f_{t-1}, C_{t,t-1} from f_{t-1} (N x N each);
// MB <= kDirectMB, NX N <= 48, N <= 8
constexpr int kDirectMB = 19;
constexpr long long kDirectJac = (long long)kDirectMB * kDirectMB + kDirectMB;
constexpr long long kDirectCurv = kDirectJac + 48 + 8;
constexpr long long kDirectStage = kDirectCurv + 3 * 64;
constexpr double kCurvStep = 1e-6;   // central-difference step of the constraint curvature
// shared scratch of the sweep (X, pivot row, y / v, w): N^2 + 2 MB + MB + N doubles
constexpr int kDirectScratch = 64 + 3 * kDirectMB + 8;

template <int M>
struct Kkt {
    static constexpr int NX = Traits<M>::NX, N = NX + Traits<M>::NU, NG = Traits<M>::NG;
    static constexpr int MB = NX + N + NG;   // block size
    static constexpr int XZ = NX;            // first eta_x row of a block
    static constexpr int XH = NX + N;        // first eta_h row
    static_assert(MB <= kDirectMB, "block of the direct adjoint solve");
};

// Entry (j, b) of P_t restricted to the eta_x rows: H_{t,t-1}, the (t, t-1) block
// of the cost Hessian (-W on the control diagonal, from the rate cost).
template <int M>
__device__ __forceinline__ double Hsub(const Inst<M>& c, int j, int b) {
    return (j == b && j >= Inst<M>::NX) ? -(double)c.W(j - Inst<M>::NX) : 0.0;
}

// Diagonal of the cost Hessian block D_t (App. B: D_t = H^+_{t-1} + H^-_t), in FP64
template <int M>
__device__ __forceinline__ double Hdiag(const Inst<M>& c, int t, int j) {
    double d = (double)c.Cw(t, j);
    if (j >= Inst<M>::NX) {
        const double w = (double)c.W(j - Inst<M>::NX);
        if (t < c.Nh) d += w;
        if (t > 0) d += w;
    }
    return d;
}

// FP64 Jacobian A^-_t = d f_t / d z_t (NX x N) at the FP32 point (zt, zn) and the
// dense row of G_t, evaluated by the model functions in double precision, so that
// the KKT system is the one at the returned point up to FP64 rounding.
template <int M>
__device__ __forceinline__ void jac_at(const Inst<M>& c, const double* zt, const double* zn, double* Ad) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX;
    {
        if constexpr (M == MODEL_DI) {
            const double dt = (double)c.dyn[0];
#pragma unroll
            for (int i = 0; i < NX * N; ++i) Ad[i] = 0.0;
            for (int k = 0; k < 4; ++k) Ad[k * N + k] = 1.0;
            Ad[0 * N + 2] = dt; Ad[1 * N + 3] = dt;
            Ad[0 * N + 4] = 0.5 * dt * dt; Ad[1 * N + 5] = 0.5 * dt * dt;
            Ad[2 * N + 4] = dt; Ad[3 * N + 5] = dt;
        } else if constexpr (M == MODEL_QUAD) {
            double phi[6], dPx[36], dPu[12];
            quad_rk4<double>(zt, zt + 6, c.dyn, phi, dPx, dPu);
            for (int k = 0; k < 6; ++k) {
                for (int j = 0; j < 6; ++j) Ad[k * N + j] = dPx[k * 6 + j];
                Ad[k * N + 6] = dPu[k * 2];
                Ad[k * N + 7] = dPu[k * 2 + 1];
            }
        } else {   // bicycle, implicit midpoint
            const double dt = (double)c.dyn[0];
            double mid[6], fc[6], Jx[36], Ju[12];
            for (int k = 0; k < 6; ++k) mid[k] = 0.5 * (zt[k] + zn[k]);
            bicycle_fc<double>(mid, zt + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fc, Jx, Ju);
            for (int k = 0; k < 6; ++k) {
                for (int j = 0; j < 6; ++j) Ad[k * N + j] = (k == j ? 1.0 : 0.0) + 0.5 * dt * Jx[k * 6 + j];
                Ad[k * N + 6] = dt * Ju[k * 2];
                Ad[k * N + 7] = dt * Ju[k * 2 + 1];
            }
        }
    }
}

// dense row of G_t (the bicycle's lateral track error) at z, FP64
template <int M>
__device__ __forceinline__ void gtrack_at(const Inst<M>& c, const double* z, double* Gd) {
    constexpr int N = Inst<M>::N;
    TrackPtR<double> tp = track_eval<double>(c.track, c.nt, (double)c.dyn[2], z[5]);
    double sp, cp;
    msincos(tp.psic, &sp, &cp);
    const double dx = z[0] - tp.xc, dy = z[1] - tp.yc;
#pragma unroll
    for (int j = 0; j < N; ++j) Gd[j] = 0.0;
    Gd[0] = -sp;
    Gd[1] = cp;
    Gd[5] = tp.dxc * sp - tp.dyc * cp - tp.dpsic * (dx * cp + dy * sp);
}

template <int M>
__device__ __forceinline__ void jacobians_fp64(const Inst<M>& c, int t, double* Ad, double* Gd) {
    constexpr int N = Inst<M>::N;
    double zt[N], zn[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        zt[j] = (double)c.zb[t * N + j];
        zn[j] = t < c.Nh ? (double)c.zb[(t + 1) * N + j] : 0.0;
    }
    if (t < c.Nh) jac_at<M>(c, zt, zn, Ad);
    if constexpr (Traits<M>::DENSE_ROW >= 0) gtrack_at<M>(c, zt, Gd);
}

// Constraint curvature of the Lagrangian (the exact-Hessian backward; App. E:
// H = Hessian of l + y_f' f + y_A' g_A), by FP64 central differences (step
// kCurvStep) of the FP64 analytic Jacobians:
//   f_t with multiplier y = y_f[t+1]: psi(z_t, z_{t+1}) = [A^-' y; A^+' y] over the 2N
//   coordinates -> blocks (t,t) into Ct[t], (t+1,t+1) into Cn[t+1], (t+1,t) into Cl[t+1];
//   the active track row with multiplier y_g: Hessian of g into Ct[t].
// Stage t's thread writes Ct[t] and the Cn, Cl slots of stage t+1 (no other writer).
template <int M>
__device__ __forceinline__ void curvature_fp64(const Inst<M>& c, const float* code, int t, double* dws) {
    using Tr = Traits<M>;
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    double* Ct = dws + (long long)t * kDirectStage + kDirectCurv;
    double* Cn = dws + (long long)(t + 1) * kDirectStage + kDirectCurv + 64;
    double* Cl = Cn + 64;
    double z0[2 * N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        z0[j] = (double)c.zb[t * N + j];
        z0[N + j] = t < c.Nh ? (double)c.zb[(t + 1) * N + j] : 0.0;
    }
    for (int i = 0; i < N * N; ++i) Ct[i] = 0.0;
    if (t == 0) {
        double* C0 = dws + kDirectCurv + 64;
        for (int i = 0; i < 2 * N * N; ++i) C0[i] = 0.0;
    }
    if (t < c.Nh && M != MODEL_DI) {
        double y[NX];
#pragma unroll
        for (int k = 0; k < NX; ++k) y[k] = (double)c.yfb[(t + 1) * NX + k];
        // psi(v) = [A^-' y; A^+' y], A^+ = A^-_x - 2I (implicit midpoint) or [-I 0] (explicit)
        auto psi = [&](const double* v, double* g) {
            double Ad[NX * N];
            jac_at<M>(c, v, v + N, Ad);
            for (int j = 0; j < N; ++j) {
                double a = 0.0, b = 0.0;
                for (int k = 0; k < NX; ++k) {
                    a += Ad[k * N + j] * y[k];
                    if (j < NX) b += (Tr::IMPLICIT ? Ad[k * N + j] - (k == j ? 2.0 : 0.0) : (k == j ? -1.0 : 0.0)) * y[k];
                }
                g[j] = a;
                g[N + j] = b;
            }
        };
        double Hc[2 * N][2 * N];
        for (int q = 0; q < 2 * N; ++q) {
            double vp[2 * N], vm[2 * N], gp[2 * N], gm[2 * N];
            for (int j = 0; j < 2 * N; ++j) { vp[j] = z0[j]; vm[j] = z0[j]; }
            vp[q] += kCurvStep;
            vm[q] -= kCurvStep;
            psi(vp, gp);
            psi(vm, gm);
            for (int j = 0; j < 2 * N; ++j) Hc[j][q] = (gp[j] - gm[j]) / (2.0 * kCurvStep);
        }
        for (int i = 0; i < 2 * N; ++i)
            for (int j = 0; j < i; ++j) {
                const double m = 0.5 * (Hc[i][j] + Hc[j][i]);
                Hc[i][j] = m;
                Hc[j][i] = m;
            }
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                Ct[i * N + j] = Hc[i][j];
                Cn[i * N + j] = Hc[N + i][N + j];
                Cl[i * N + j] = Hc[N + i][j];
            }
    } else if (t < c.Nh) {
        for (int i = 0; i < 2 * N * N; ++i) Cn[i] = 0.0;
    }
    if constexpr (Tr::DENSE_ROW >= 0) {
        const int q = Tr::DENSE_ROW;
        if (code[t * NG + q] != 0.f) {   // active (hard or slack): multiplier y_g of the row
            const double yg = (double)c.ygb[t * NG + q];
            for (int k = 0; k < N; ++k) {
                double vp[N], vm[N], gp[N], gm[N];
                for (int j = 0; j < N; ++j) { vp[j] = z0[j]; vm[j] = z0[j]; }
                vp[k] += kCurvStep;
                vm[k] -= kCurvStep;
                gtrack_at<M>(c, vp, gp);
                gtrack_at<M>(c, vm, gm);
                for (int j = 0; j < N; ++j) Ct[j * N + k] += yg * (gp[j] - gm[j]) / (2.0 * kCurvStep);
            }
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < i; ++j) {
                    const double m = 0.5 * (Ct[i * N + j] + Ct[j * N + i]);
                    Ct[i * N + j] = m;
                    Ct[j * N + i] = m;
                }
        }
    }
}

// Solve by warp 0 of the team.  code: active-set codes (0 inactive, +-1 hard,
// +-2 slack-active) per row; bx: the right-hand side b per stage entry; outputs
// eta_x -> ex, eta_f -> lam (per stage, nx), eta_h -> mu (hard-active rows, 0
// elsewhere).  dws: the instance's FP64 workspace (T kDirectStage doubles);
// sh: shared scratch of at least (N^2 + 3 MB + N) doubles, 8-byte aligned.
// Returns (to every thread of the team) true if the regularised solve was needed.
template <int M>
__device__ bool direct_adjoint(const Inst<M>& c, const float* code, const float* bx, float* ex, float* lam,
                               float* mu, double* dws, double* sh, int* flag, bool exact) {
    using K = Kkt<M>;
    constexpr int NX = K::NX, N = K::N, NG = K::NG, MB = K::MB, XZ = K::XZ, XH = K::XH;
    const int T = c.T;
    double* X = sh;                 // (S_{t-1}^-1)_xx, N x N
    double* prow = X + N * N;       // pivot row broadcast: [a | e], 2 MB
    double* yv = prow + 2 * MB;     // y_t / v_t broadcast, MB
    double* wv = yv + MB;           // w_{t-1} = (S_{t-1}^-1 y_{t-1})_x, N
    const bool warp0 = c.tid < 32;
    const int lane = c.tid & 31;
    const bool row = warp0 && lane < MB;
    for (int t = c.tid; t < T; t += c.nth) {
        double* st = dws + (long long)t * kDirectStage + kDirectJac;
        jacobians_fp64<M>(c, t, st, st + 48);
        if (exact) curvature_fp64<M>(c, code, t, dws);
    }
    if (c.tid == 0) *flag = 0;
    c.sync();
    // FP64 blocks: A^-_t, A^+_t (implicit: A^-_x - 2I; explicit: -I on the states), G_t
    auto Amd = [&](int t) -> const double* { return dws + (long long)t * kDirectStage + kDirectJac; };
    auto Apd = [&](int t, int k, int j) -> double {
        if (j >= NX) return 0.0;
        if (Traits<M>::IMPLICIT) return Amd(t)[k * N + j] - (k == j ? 2.0 : 0.0);
        return k == j ? -1.0 : 0.0;
    };
    // cost Hessian blocks plus, with the exact Hessian, the constraint curvature
    auto Htt = [&](int t, int j, int jj) -> double {
        double h = j == jj ? Hdiag<M>(c, t, j) : 0.0;
        if (exact) {
            const double* cv = dws + (long long)t * kDirectStage + kDirectCurv;
            h += cv[j * N + jj] + (t > 0 ? cv[64 + j * N + jj] : 0.0);
        }
        return h;
    };
    auto Hlow = [&](int t, int j, int b) -> double {   // (t, t-1) block, t >= 1
        double h = Hsub<M>(c, j, b);
        if (exact) h += (dws + (long long)t * kDirectStage + kDirectCurv + 128)[j * N + b];
        return h;
    };
    auto Gd = [&](int t, int q, int j) -> double {
        const int s = Traits<M>::sel(q);
        if (s >= 0) return j == s ? 1.0 : 0.0;
        return (dws + (long long)t * kDirectStage + kDirectJac + 48)[j];
    };
    for (int pass = 0; pass < 2; ++pass) {
        const double delta = pass == 0 ? 0.0 : 1e-10;
        if (warp0) {
            int singular = 0;
            for (int t = 0; t < T; ++t) {
                // ---- row `lane` of D_t ----
                double a[MB], e[MB];
#pragma unroll
                for (int q = 0; q < MB; ++q) { a[q] = 0.0; e[q] = (q == lane) ? 1.0 : 0.0; }
                if (row) {
                    if (lane < XZ) {                         // lambda_t row k
                        const int k = lane;
#pragma unroll
                        for (int j = 0; j < N; ++j)
                            a[XZ + j] = t == 0 ? (j == k ? 1.0 : 0.0) : Apd(t - 1, k, j);
                        a[k] = -delta;
                    } else if (lane < XH) {                  // eta_x,t row j
                        const int j = lane - XZ;
#pragma unroll
                        for (int k = 0; k < NX; ++k)
                            a[k] = t == 0 ? (j == k ? 1.0 : 0.0) : Apd(t - 1, k, j);
#pragma unroll
                        for (int jj = 0; jj < N; ++jj) a[XZ + jj] = Htt(t, j, jj);
#pragma unroll
                        for (int q = 0; q < NG; ++q) {
                            const float cd = code[t * NG + q];
                            const double g = Gd(t, q, j);
                            if (fabsf(cd) > 1.5f) {          // slack-active: gamma2 G_q' G_q
#pragma unroll
                                for (int jj = 0; jj < N; ++jj)
                                    a[XZ + jj] += (double)c.gam2(q) * g * Gd(t, q, jj);
                            } else if (cd != 0.f) {
                                a[XH + q] = g;
                            }
                        }
                    } else {                                 // eta_h,t row q
                        const int q = lane - XH;
                        const float cd = code[t * NG + q];
                        if (cd != 0.f && fabsf(cd) < 1.5f) {
#pragma unroll
                            for (int j = 0; j < N; ++j) a[XZ + j] = Gd(t, q, j);
                            a[lane] = -delta;
                        } else {
                            a[lane] = 1.0;
                        }
                    }
                    // ---- Schur complement: - P_t X P_t' on the lambda / eta_x rows and columns ----
                    if (t > 0 && lane < XH) {
                        double pr[N];   // row `lane` of P_t
#pragma unroll
                        for (int b = 0; b < N; ++b)
                            pr[b] = lane < XZ ? Amd(t - 1)[lane * N + b] : Hlow(t, lane - XZ, b);
                        double u[N];
#pragma unroll
                        for (int b = 0; b < N; ++b) {
                            double s = 0.0;
#pragma unroll
                            for (int q = 0; q < N; ++q) s += pr[q] * X[q * N + b];
                            u[b] = s;
                        }
#pragma unroll
                        for (int col = 0; col < XH; ++col) {
                            double s = 0.0;
#pragma unroll
                            for (int b = 0; b < N; ++b)
                                s += u[b] * (col < XZ ? Amd(t - 1)[col * N + b] : Hlow(t, col - XZ, b));
                            a[col] -= s;
                        }
                    }
                }
                // ---- Gauss-Jordan with partial pivoting: [S_t | I] -> rows of S_t^-1 ----
                double amax = 0.0;
#pragma unroll
                for (int q = 0; q < MB; ++q) amax = fmax(amax, fabs(a[q]));
                for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
                const double tiny = 1e-13 * (amax > 0.0 ? amax : 1.0);
                bool used = !row;
                int mypiv = -1;
#pragma unroll
                for (int p = 0; p < MB; ++p) {
                    double cand = used ? -1.0 : fabs(a[p]);
                    int who = lane;
                    for (int o = 16; o > 0; o >>= 1) {
                        const double oc = __shfl_xor_sync(0xffffffffu, cand, o);
                        const int ow = __shfl_xor_sync(0xffffffffu, who, o);
                        if (oc > cand || (oc == cand && ow < who)) { cand = oc; who = ow; }
                    }
                    if (!(cand > tiny)) singular = 1;
                    if (lane == who) {
                        used = true;
                        mypiv = p;
                        const double inv = (a[p] != 0.0) ? 1.0 / a[p] : 0.0;
#pragma unroll
                        for (int q = 0; q < MB; ++q) {
                            a[q] *= inv;
                            e[q] *= inv;
                            prow[q] = a[q];
                            prow[MB + q] = e[q];
                        }
                    }
                    __syncwarp();
                    if (row && lane != who) {
                        const double f = a[p];
#pragma unroll
                        for (int q = 0; q < MB; ++q) {
                            a[q] -= f * prow[q];
                            e[q] -= f * prow[MB + q];
                        }
                    }
                    __syncwarp();
                }
                // lane with pivot column p holds row p of S_t^-1
                double* Sinv = dws + (long long)t * kDirectStage;
                if (row) {
#pragma unroll
                    for (int q = 0; q < MB; ++q) Sinv[mypiv * MB + q] = e[q];
                }
                // ---- forward substitution: y_t = r_t - P_t w_{t-1} ----
                if (row) {
                    double y = 0.0;
                    if (lane >= XZ && lane < XH) y = (double)bx[t * N + lane - XZ];
                    if (t > 0 && lane < XH) {
#pragma unroll
                        for (int b = 0; b < N; ++b)
                            y -= (lane < XZ ? Amd(t - 1)[lane * N + b] : Hlow(t, lane - XZ, b)) * wv[b];
                    }
                    yv[lane] = y;
                    Sinv[MB * MB + lane] = y;
                }
                __syncwarp();
                // w_t = (S_t^-1 y_t)_x and X_t = (S_t^-1)_xx (rows XZ..XH-1, columns XZ..XH-1)
                if (row && mypiv >= XZ && mypiv < XH) {
                    double s = 0.0;
#pragma unroll
                    for (int q = 0; q < MB; ++q) s += e[q] * yv[q];
                    wv[mypiv - XZ] = s;
#pragma unroll
                    for (int j = 0; j < N; ++j) X[(mypiv - XZ) * N + j] = e[XZ + j];
                }
                __syncwarp();
            }
            // ---- backward sweep: x_t = S_t^-1 (y_t - P_{t+1}' x_{t+1}) ----
            double* xnext = wv;   // eta_x,t+1 and lambda_{t+1} of the step before, in yv / wv
            for (int t = T - 1; t >= 0; --t) {
                const double* Sinv = dws + (long long)t * kDirectStage;
                if (row) {
                    double v = Sinv[MB * MB + lane];
                    if (t < T - 1 && lane >= XZ && lane < XH) {
                        const int b = lane - XZ;
                        double s = 0.0;
#pragma unroll
                        for (int k = 0; k < NX; ++k) s += Amd(t)[k * N + b] * yv[k];
#pragma unroll
                        for (int j = 0; j < N; ++j) s += Hlow(t + 1, j, b) * xnext[j];
                        v -= s;
                    }
                    prow[lane] = v;
                }
                __syncwarp();
                double x = 0.0;
                if (row) {
#pragma unroll
                    for (int q = 0; q < MB; ++q) x += Sinv[lane * MB + q] * prow[q];
                }
                __syncwarp();
                if (row) {
                    if (lane < XZ) { lam[t * NX + lane] = (float)x; yv[lane] = x; }
                    else if (lane < XH) { ex[t * N + lane - XZ] = (float)x; xnext[lane - XZ] = x; }
                    else {
                        const float cd = code[t * NG + lane - XH];
                        mu[t * NG + lane - XH] = (cd != 0.f && fabsf(cd) < 1.5f) ? (float)x : 0.f;
                    }
                }
                __syncwarp();
            }
            if (lane == 0) *flag = singular;
        }
        c.sync();
        const bool sing = *flag != 0;
        c.sync();
        if (!sing) return pass > 0;
    }
    return true;
}

}  // namespace fast
}  // namespace tmpc
