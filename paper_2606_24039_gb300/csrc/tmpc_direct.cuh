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
// Jacobian A^-_t (NX x N) and the dense row of G_t (N); MB <= kDirectMB, NX N <= 48, N <= 8
constexpr int kDirectMB = 19;
constexpr long long kDirectJac = (long long)kDirectMB * kDirectMB + kDirectMB;
constexpr long long kDirectStage = kDirectJac + 48 + 8;

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
__device__ __forceinline__ void jacobians_fp64(const Inst<M>& c, int t, double* Ad, double* Gd) {
    using Tr = Traits<M>;
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX;
    double zt[N];
#pragma unroll
    for (int j = 0; j < N; ++j) zt[j] = (double)c.zb[t * N + j];
    if (t < c.Nh) {
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
            for (int k = 0; k < 6; ++k) mid[k] = 0.5 * (zt[k] + (double)c.zb[(t + 1) * N + k]);
            bicycle_fc<double>(mid, zt + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fc, Jx, Ju);
            for (int k = 0; k < 6; ++k) {
                for (int j = 0; j < 6; ++j) Ad[k * N + j] = (k == j ? 1.0 : 0.0) + 0.5 * dt * Jx[k * 6 + j];
                Ad[k * N + 6] = dt * Ju[k * 2];
                Ad[k * N + 7] = dt * Ju[k * 2 + 1];
            }
        }
    }
    if constexpr (Tr::DENSE_ROW >= 0) {   // lateral track error of the bicycle
        TrackPtR<double> tp = track_eval<double>(c.track, c.nt, (double)c.dyn[2], zt[5]);
        double sp, cp;
        msincos(tp.psic, &sp, &cp);
        const double dx = zt[0] - tp.xc, dy = zt[1] - tp.yc;
#pragma unroll
        for (int j = 0; j < N; ++j) Gd[j] = 0.0;
        Gd[0] = -sp;
        Gd[1] = cp;
        Gd[5] = tp.dxc * sp - tp.dyc * cp - tp.dpsic * (dx * cp + dy * sp);
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
                               float* mu, double* dws, double* sh, int* flag) {
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
                        a[XZ + j] = Hdiag<M>(c, t, j);
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
                            pr[b] = lane < XZ ? Amd(t - 1)[lane * N + b] : Hsub<M>(c, lane - XZ, b);
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
                                s += u[b] * (col < XZ ? Amd(t - 1)[col * N + b] : Hsub<M>(c, col - XZ, b));
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
                            y -= (lane < XZ ? Amd(t - 1)[lane * N + b] : Hsub<M>(c, lane - XZ, b)) * wv[b];
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
                        for (int j = 0; j < N; ++j) s += Hsub<M>(c, j, b) * xnext[j];
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
