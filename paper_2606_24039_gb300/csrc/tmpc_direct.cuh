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
// eta_x,t (n), eta_h,t (the hard-active rows of stage t)].  In this order the
// matrix is block tridiagonal: the diagonal block D_t holds H_s,tt, A^+_{t-1}
// (A_init at t = 0) and G_h,t; the coupling of block t to block t-1 is
// P_t = [A^-_{t-1}; H_{t,t-1}] on the eta_x,t-1 columns.  It is symmetric and
// indefinite, and is factored by block LDL' without pivoting across blocks:
//     S_0 = D_0,   S_t = D_t - P_t (S_{t-1}^-1)_xx P_t',
// each S_t inverted in place by Gauss-Jordan elimination with partial pivoting
// inside the block.  The forward sweep also carries y_t = r_t - P_t w_{t-1},
// w_t = (S_t^-1 y_t)_x; the backward sweep returns x_t = S_t^-1 (y_t - P_{t+1}' x_{t+1}).
// One factorisation, no refinement.
//
// FP64 because the active-set KKT of a constrained OCP can be ill-conditioned
// (condition numbers near 1e10 on the racing model where bound rows nearly
// repeat the dynamics rows), beyond what an FP32 factorisation resolves.  If a
// pivot block is numerically singular (the active rows are linearly dependent),
// the solve is repeated with -1e-10 on the multiplier diagonal.
//
// Work split: the instance's team evaluates everything that is parallel over
// the stages (FP64 Jacobians at the returned point, the constraint curvature of
// the exact Hessian, the active codes, the right-hand side and the cost
// diagonal) into a per-stage FP64 record; the sweeps, sequential over the
// stages, are one warp's (lane r holds row r of the block).  GB300 executes FP64
// at a small fraction of its FP32 rate, so the sweeps are bound by the FP64 pipe
// of the SM sub-partition the warp runs on: the CTA kernels hand the sweeps to
// a kernel of independent warps (one instance each, all four sub-partitions of
// every SM busy) and finish the gradients in a third pass; a cluster team runs
// them on its first warp.  To keep the FP64 instruction count low, the block
// drops the inactive bound rows (size nx + n + active rows, a template
// parameter), the inversion is in place (one row of the block per lane, half
// the work of inverting [S | I]), and the Schur complement is spread over all
// 32 lanes.
#pragma once
#include "tmpc_fast.cuh"

namespace tmpc {
namespace fast {

constexpr double kCurvStep = 1e-6;   // central-difference step of the constraint curvature

// Per-stage FP64 record of one instance (doubles), and the compile-time sizes
//   MB  = nx + n + ng: largest block (every bound row hard-active)
//   XH  = nx + n: the lambda and eta_x rows, always present
template <int M>
struct DRec {
    static constexpr int NX = Traits<M>::NX, NU = Traits<M>::NU, N = NX + NU, NG = Traits<M>::NG;
    static constexpr int MB = NX + N + NG, XZ = NX, XH = NX + N;
    static constexpr int Inv = 0;                 // S_t^-1, MB x MB (active-row order)
    static constexpr int Y = Inv + MB * MB;       // y_t, MB
    static constexpr int Am = Y + MB;             // A^-_t, NX x N
    static constexpr int G = Am + NX * N;         // dense row of G_t, N
    static constexpr int Ct = G + N;              // exact Hessian: curvature of stage t's terms, N x N
    static constexpr int Cn = Ct + N * N;         //   of f_{t-1} on z_t (t >= 1), N x N
    static constexpr int Cl = Cn + N * N;         //   of f_{t-1}, block (t, t-1), N x N
    static constexpr int Code = Cl + N * N;       // active codes, NG
    static constexpr int B = Code + NG;           // right-hand side b, N
    static constexpr int Hd = B + N;              // diagonal of the cost Hessian block, N
    static constexpr int X = Hd + N;              // solution [lambda_t, eta_x,t, eta_h,t] (all NG rows), MB
    static constexpr int Par = X + MB;            // stage 0 only: W (NU), gamma2 (NG)
    static constexpr int Stage = (Par + NU + NG + 1) & ~1;
    // per-warp shared scratch of the sweeps: X_{t-1} (N^2), P_t and U = P_t X_{t-1}
    // (XH N each), U P_t' (XH^2), pivot row (MB), y_t (MB), w_{t-1} (N), x_{t+1} (XH)
    static constexpr int Scratch = N * N + 2 * XH * N + XH * XH + 2 * MB + N + XH;
    static_assert(MB <= 32, "one lane per row of the block");
    static_assert((N * N + 2 * XH * N + XH * XH) % 2 == 0, "pivot row on a 16-byte boundary");
};

// Largest per-warp scratch over the small models (the bicycle's)
constexpr int kDirectScratch = 544;

// Instances handed from the backward kernel to the sweep kernel: flag[i] = 1 for
// instance i (global index); the sweep kernel and the finishing pass walk the
// group's instance order (longest first) and take the flagged ones
struct DirectQueue {
    int* flag;
};
constexpr int kDirectWarps = 8;   // warps per CTA of the sweep kernel

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
//   coordinates -> blocks (t,t) into Ct of stage t, (t+1,t+1) into Cn and (t+1,t)
//   into Cl of stage t+1;
//   the active track row with multiplier y_g: Hessian of g into Ct of stage t.
// Stage t's thread writes Ct of stage t and Cn, Cl of stage t+1 (no other writer).
template <int M>
__device__ __forceinline__ void curvature_fp64(const Inst<M>& c, const float* code, int t, double* dws) {
    using Tr = Traits<M>;
    using R = DRec<M>;
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    double* Ct = dws + (long long)t * R::Stage + R::Ct;
    double* Cn = dws + (long long)(t + 1) * R::Stage + R::Cn;
    double* Cl = dws + (long long)(t + 1) * R::Stage + R::Cl;
    double z0[2 * N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        z0[j] = (double)c.zb[t * N + j];
        z0[N + j] = t < c.Nh ? (double)c.zb[(t + 1) * N + j] : 0.0;
    }
    for (int i = 0; i < N * N; ++i) Ct[i] = 0.0;
    if (t == 0)
        for (int i = 0; i < N * N; ++i) {
            dws[R::Cn + i] = 0.0;
            dws[R::Cl + i] = 0.0;
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
        for (int i = 0; i < N * N; ++i) {
            Cn[i] = 0.0;
            Cl[i] = 0.0;
        }
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

// The team's part before the sweeps: per stage the FP64 Jacobians (and, with
// the exact Hessian, the constraint curvature), the active codes, the
// right-hand side b and the diagonal of the cost Hessian; W and gamma2 in
// stage 0's record.  code: 0 inactive, +-1 hard-active, +-2 slack-active.
template <int M>
__device__ void direct_store(const Inst<M>& c, const float* code, const float* bx, double* dws, bool exact) {
    using R = DRec<M>;
    constexpr int N = R::N, NG = R::NG, NU = R::NU;
    for (int t = c.tid; t < c.T; t += c.nth) {
        double* r = dws + (long long)t * R::Stage;
        jacobians_fp64<M>(c, t, r + R::Am, r + R::G);
        if (exact) curvature_fp64<M>(c, code, t, dws);
#pragma unroll
        for (int q = 0; q < NG; ++q) r[R::Code + q] = (double)code[t * NG + q];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            r[R::B + j] = (double)bx[t * N + j];
            r[R::Hd + j] = Hdiag<M>(c, t, j);
        }
        if (t == 0) {
#pragma unroll
            for (int k = 0; k < NU; ++k) r[R::Par + k] = (double)c.W(k);
#pragma unroll
            for (int q = 0; q < NG; ++q) r[R::Par + NU + q] = (double)c.gam2(q);
        }
    }
}

// The team's part after the sweeps: eta_x -> ex, eta_f -> lam, eta_h -> mu
// (hard-active rows; 0 elsewhere), rounded to FP32.
template <int M>
__device__ void direct_load(const Inst<M>& c, const double* dws, float* ex, float* lam, float* mu) {
    using R = DRec<M>;
    constexpr int NX = R::NX, N = R::N, NG = R::NG;
    for (int e = c.tid; e < c.T * R::MB; e += c.nth) {
        const int t = e / R::MB, r = e % R::MB;
        const double* rt = dws + (long long)t * R::Stage;
        const double x = rt[R::X + r];
        if (r < NX) lam[t * NX + r] = (float)x;
        else if (r < R::XH) ex[t * N + r - NX] = (float)x;
        else mu[t * NG + r - R::XH] = (float)x;
    }
}

// FP64 reciprocal by Newton-Raphson iteration y <- y (2 - x y) from the FP32
// estimate (two steps: the relative error squares from ~2^-23 to below FP64
// rounding).  For |x| well inside the FP32 normal range; the caller divides
// outside it.
__device__ __forceinline__ double recip_nr(double x) {
    double y = (double)(1.0f / (float)x);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// In-place Gauss-Jordan inversion of the K x K block held one row per lane
// (lanes K..31 idle), partial pivoting on the rows not yet pivoted (the pivot is
// the largest magnitude rounded to 18 bits, ties to the lower lane: one integer
// warp reduction).  Step p: the pivot row is broadcast unscaled with its entry p
// replaced by 1, and every lane applies one FMA per column, v -= g prow, with
// g = v_p / pivot on the other rows (entry p first set to 0) and g = 1 - 1/pivot
// on the pivot row (entry p first set to 1), which leaves it scaled by 1/pivot:
// the in-place form.  On return the lane that pivoted at step p holds row p of
// S^-1 with its entries in the order of the pivot steps: v[j] = (S^-1)(p, pw[j]),
// pw[j] the lane (row) that pivoted at step j.  Returns 1 if a pivot fell below
// 1e-13 of the block's largest entry (numerically singular).
template <int MB, int K>
__device__ __forceinline__ int gj_inplace(double (&v)[MB], int (&pw)[MB], int& mypiv, double* prow, int lane) {
    static_assert(K <= MB && K <= 32, "block size");
    double amax = 0.0;
#pragma unroll
    for (int q = 0; q < K; ++q) amax = fmax(amax, fabs(v[q]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const double tiny = 1e-13 * (amax > 0.0 ? amax : 1.0);
    bool used = lane >= K;
    int singular = 0;
    mypiv = -1;
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const unsigned key = used ? 0u : ((__float_as_uint((float)fabs(v[p])) & ~31u) | (unsigned)(31 - lane));
        const int who = 31 - (int)(__reduce_max_sync(0xffffffffu, key) & 31u);
        pw[p] = who;
        const double piv = __shfl_sync(0xffffffffu, v[p], who);
        const double ap = fabs(piv);
        if (!(ap > tiny)) singular = 1;
        const double inv = (ap > 1e-30 && ap < 1e30) ? recip_nr(piv) : (piv != 0.0 ? 1.0 / piv : 0.0);
        const bool me = lane == who;
        if (me) {
            used = true;
            mypiv = p;
#pragma unroll
            for (int q = 0; q < K; ++q) prow[q] = q == p ? 1.0 : v[q];
        }
        __syncwarp();
        const double g = me ? 1.0 - inv : v[p] * inv;
        v[p] = me ? 1.0 : 0.0;
#pragma unroll
        for (int q = 0; q + 1 < K; q += 2) {
            const double2 pr = *reinterpret_cast<const double2*>(prow + q);
            v[q] = fma(-g, pr.x, v[q]);
            v[q + 1] = fma(-g, pr.y, v[q + 1]);
        }
        if constexpr (K % 2 == 1) v[K - 1] = fma(-g, prow[K - 1], v[K - 1]);
        __syncwarp();
    }
    return singular;
}

// One stage of the forward sweep after D_t - P_t X_{t-1} P_t' is in v (row `lane`):
// invert in place, store S_t^-1 (active-row order), w_t = (S_t^-1 y_t)_x into wv and
// X_t = (S_t^-1)_xx into X.  yv holds y_t.
template <int M, int K>
__device__ __forceinline__ int sweep_block(double (&v)[DRec<M>::MB], double* rt, double* X, double* prow,
                                           const double* yv, double* wv, int lane) {
    using R = DRec<M>;
    constexpr int MB = R::MB, XZ = R::XZ, XH = R::XH, N = R::N;
    int pw[MB];
    int mypiv;
    const int sing = gj_inplace<MB, K>(v, pw, mypiv, prow, lane);
    if (mypiv >= 0) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            rt[R::Inv + mypiv * MB + pw[j]] = v[j];
            s += v[j] * yv[pw[j]];
        }
        if (mypiv >= XZ && mypiv < XH) {
            wv[mypiv - XZ] = s;
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (pw[j] >= XZ && pw[j] < XH) X[(mypiv - XZ) * N + pw[j] - XZ] = v[j];
        }
    }
    __syncwarp();
    return sing;
}

template <int M, int E>
__device__ __forceinline__ int sweep_block_k(int K, double (&v)[DRec<M>::MB], double* rt, double* X, double* prow,
                                             const double* yv, double* wv, int lane) {
    using R = DRec<M>;
    if constexpr (E >= R::NG) {
        return sweep_block<M, R::XH + R::NG>(v, rt, X, prow, yv, wv, lane);
    } else {
        if (K == R::XH + E) return sweep_block<M, R::XH + E>(v, rt, X, prow, yv, wv, lane);
        return sweep_block_k<M, E + 1>(K, v, rt, X, prow, yv, wv, lane);
    }
}

// The sweeps of one instance (T stages, records at dws), by one warp; sh: the
// warp's DRec<M>::Scratch doubles of shared memory.  Leaves the solution in the
// records (DRec::X).  Returns (warp-uniform) 1 if the regularised solve was needed.
template <int M>
__device__ int direct_sweep(int T, double* dws, double* sh, bool exact) {
    using R = DRec<M>;
    using Tr = Traits<M>;
    constexpr int NX = R::NX, N = R::N, NG = R::NG, NU = R::NU, MB = R::MB, XZ = R::XZ, XH = R::XH;
    static_assert(R::Scratch <= kDirectScratch, "per-warp scratch of the sweeps");
    const int lane = threadIdx.x & 31;
    double* X = sh;              // X_{t-1} = (S_{t-1}^-1)_xx, N x N
    double* Pm = X + N * N;      // P_t, XH x N
    double* U = Pm + XH * N;     // P_t X_{t-1}, XH x N  (Schur product U P_t' re-uses Pm)
    double* Sc = U + XH * N;     // U P_t', XH x XH
    double* prow = Sc + XH * XH; // pivot row / right-hand side broadcast, MB
    double* yv = prow + MB;      // y_t, MB
    double* wv = yv + MB;        // w_{t-1}, N
    double* xn = wv + N;         // [lambda, eta_x] of stage t+1 in the backward sweep, XH
    const double* par = dws + R::Par;
    auto rec = [&](int t) -> double* { return dws + (long long)t * R::Stage; };
    // P_t entry (r, b), r < XH: rows of A^-_{t-1}, then H_{t,t-1} (-W on the control
    // diagonal from the rate cost, plus the curvature block of f_{t-1})
    auto Pent = [&](int t, int r, int b) -> double {
        if (r < XZ) return rec(t - 1)[R::Am + r * N + b];
        const int j = r - XZ;
        double h = (j == b && j >= NX) ? -par[j - NX] : 0.0;
        if (exact) h += rec(t)[R::Cl + j * N + b];
        return h;
    };
    auto Apd = [&](int t, int k, int j) -> double {   // A^+_t (k, j)
        if (j >= NX) return 0.0;
        if (Tr::IMPLICIT) return rec(t)[R::Am + k * N + j] - (k == j ? 2.0 : 0.0);
        return k == j ? -1.0 : 0.0;
    };
    auto Gd = [&](const double* rt, int q, int j) -> double {
        const int s = Tr::sel(q);
        if (s >= 0) return j == s ? 1.0 : 0.0;
        return rt[R::G + j];
    };
    // active-row positions of stage t's hard-active rows (pos[q] = -1 if not hard-active)
    auto active = [&](const double* rt, int (&pos)[NG], int& myq) -> int {
        int nact = 0;
        myq = -1;
#pragma unroll
        for (int q = 0; q < NG; ++q) {
            const double cd = rt[R::Code + q];
            const bool hard = cd != 0.0 && fabs(cd) < 1.5;
            pos[q] = hard ? nact : -1;
            if (hard && lane == XH + nact) myq = q;
            nact += hard ? 1 : 0;
        }
        return XH + nact;
    };
    int regularised = 0;
    for (int pass = 0; pass < 2; ++pass) {
        const double delta = pass == 0 ? 0.0 : 1e-10;
        int singular = 0;
        for (int t = 0; t < T; ++t) {
            double* rt = rec(t);
            int pos[NG], myq;
            const int K = active(rt, pos, myq);
            if (t > 0) {   // P_t, then U = P_t X_{t-1}, then Sc = U P_t' over all lanes
                for (int e = lane; e < XH * N; e += 32) Pm[e] = Pent(t, e / N, e % N);
                __syncwarp();
                for (int e = lane; e < XH * N; e += 32) {
                    const int r = e / N, b = e % N;
                    double s = 0.0;
#pragma unroll
                    for (int q = 0; q < N; ++q) s += Pm[r * N + q] * X[q * N + b];
                    U[e] = s;
                }
                __syncwarp();
                for (int e = lane; e < XH * XH; e += 32) {
                    const int r = e / XH, cc = e % XH;
                    double s = 0.0;
#pragma unroll
                    for (int b = 0; b < N; ++b) s += U[r * N + b] * Pm[cc * N + b];
                    Sc[e] = s;
                }
            }
            // y_t = r_t - P_t w_{t-1} (row `lane`; r_t = b on the eta_x rows)
            if (lane < K) {
                double y = 0.0;
                if (lane >= XZ && lane < XH) y = rt[R::B + lane - XZ];
                if (t > 0 && lane < XH) {
#pragma unroll
                    for (int b = 0; b < N; ++b) y -= Pm[lane * N + b] * wv[b];
                }
                yv[lane] = y;
                rt[R::Y + lane] = y;
            }
            __syncwarp();
            // row `lane` of S_t = D_t - Sc (active-row order)
            double v[MB];
#pragma unroll
            for (int q = 0; q < MB; ++q) v[q] = 0.0;
            if (lane < XZ) {                        // lambda_t row k: [-delta e_k | A^+_{t-1}(k, :) | 0]
#pragma unroll
                for (int j = 0; j < N; ++j) v[XZ + j] = t == 0 ? (j == lane ? 1.0 : 0.0) : Apd(t - 1, lane, j);
#pragma unroll
                for (int q = 0; q < XZ; ++q)
                    if (q == lane) v[q] = -delta;
            } else if (lane < XH) {                 // eta_x,t row j
                const int j = lane - XZ;
#pragma unroll
                for (int k = 0; k < NX; ++k) v[k] = t == 0 ? (j == k ? 1.0 : 0.0) : Apd(t - 1, k, j);
#pragma unroll
                for (int jj = 0; jj < N; ++jj) {
                    double h = jj == j ? rt[R::Hd + j] : 0.0;
                    if (exact) h += rt[R::Ct + j * N + jj] + (t > 0 ? rt[R::Cn + j * N + jj] : 0.0);
                    v[XZ + jj] = h;
                }
#pragma unroll
                for (int q = 0; q < NG; ++q) {
                    const double cd = rt[R::Code + q];
                    const double g = Gd(rt, q, j);
                    if (fabs(cd) > 1.5) {           // slack-active: gamma2 G_q' G_q
#pragma unroll
                        for (int jj = 0; jj < N; ++jj) v[XZ + jj] += par[NU + q] * g * Gd(rt, q, jj);
                    }
#pragma unroll
                    for (int m = 0; m < NG; ++m)
                        if (pos[q] == m) v[XH + m] = g;
                }
            } else if (myq >= 0) {                  // eta_h row of hard-active row myq
#pragma unroll
                for (int j = 0; j < N; ++j) v[XZ + j] = Gd(rt, myq, j);
#pragma unroll
                for (int q = XH; q < MB; ++q)
                    if (q == lane) v[q] = -delta;
            }
            if (t > 0 && lane < XH) {
#pragma unroll
                for (int cc = 0; cc < XH; ++cc) v[cc] -= Sc[lane * XH + cc];
            }
            singular |= sweep_block_k<M, 0>(K, v, rt, X, prow, yv, wv, lane);
            if (pass == 0 && singular) break;   // warp-uniform: redo with the regularisation
        }
        if (pass == 0 && singular) {
            regularised = 1;
            continue;
        }
        // backward sweep: x_t = S_t^-1 (y_t - P_{t+1}' x_{t+1})
        for (int t = T - 1; t >= 0; --t) {
            double* rt = rec(t);
            int pos[NG], myq;
            const int K = active(rt, pos, myq);
            if (lane < K) {
                double v = rt[R::Y + lane];
                if (t < T - 1 && lane >= XZ && lane < XH) {
                    const int b = lane - XZ;
                    double s = 0.0;
#pragma unroll
                    for (int r = 0; r < XH; ++r) s += Pent(t + 1, r, b) * xn[r];
                    v -= s;
                }
                prow[lane] = v;
            }
            __syncwarp();
            double x = 0.0;
            if (lane < K) {
                const double* Si = rt + R::Inv + lane * MB;
#pragma unroll
                for (int q = 0; q < MB; ++q)
                    if (q < K) x += Si[q] * prow[q];
            }
            __syncwarp();
            if (lane < XH) {
                xn[lane] = x;
                rt[R::X + lane] = x;
            } else if (myq >= 0) {
                rt[R::X + XH + myq] = x;
            }
            if (lane < NG && lane >= 0) {
                // inactive and slack-active rows carry no multiplier in this system
                const double cd = rt[R::Code + lane];
                if (!(cd != 0.0 && fabs(cd) < 1.5)) rt[R::X + XH + lane] = 0.0;
            }
            __syncwarp();
        }
        break;
    }
    return regularised;
}

// The sweeps as a kernel of independent warps: each warp takes the next entry of
// the group's instance order (longest first) from an atomic cursor and sweeps it
// if the backward pass flagged it.  blockDim = kDirectWarps * 32.
template <int M>
__global__ void __launch_bounds__(kDirectWarps * 32, 1) direct_kernel(const int* N, const int* order, int count,
                                                                      const int* flag, int* cursor, double* dws,
                                                                      long long dstride, int exact) {
    __shared__ __align__(16) double sh[kDirectWarps][kDirectScratch];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        int k = 0;
        if (lane == 0) {
            do {
                k = atomicAdd(cursor, 1);
            } while (k < count && !flag[order[k]]);
        }
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= count) break;
        const int i = order[k];
        direct_sweep<M>(N[i] + 1, dws + (long long)i * dstride, sh[w], exact != 0);
    }
}

}  // namespace fast
}  // namespace tmpc
