// Direct FP64 adjoint solve of the backward pass (Algorithm 2) on the generic
// kernel, for layouts whose interleaved KKT block [lambda_t, eta_x,t, eta_h,t]
// has at most kGenDirectMB rows (every model but the wide linear ones): the same
// block LDL' as tmpc_direct.cuh (see there for the ordering and the recurrences),
// with run-time sizes, the working rows of each Gauss-Jordan inversion in shared
// memory, and the Jacobian blocks the generic kernel keeps (FP32) taken to FP64.
#pragma once
#include "tmpc_solver.cuh"

namespace tmpc {

constexpr int kGenDirectMB = 32;
constexpr int kGenDirectLD = kGenDirectMB + 1;
// shared scratch: rows of [S_t | I] (2 MB x LD), X (n x n, n < MB), pivot row (2 MB), y (MB), w (MB)
constexpr int kGenDirectScratch = 2 * kGenDirectMB * kGenDirectLD + kGenDirectMB * kGenDirectMB + 4 * kGenDirectMB;

__host__ __device__ inline int gen_direct_mb(int nx, int n, int ng) { return nx + n + ng; }
__host__ __device__ inline long long gen_direct_stage(int mb) { return (long long)mb * mb + mb; }

// code: active-set codes per row (0, +-1 hard, +-2 slack-active); bx: right-hand side per
// stage entry; outputs eta_x -> ex, eta_f -> lam, eta_h -> mu (hard-active rows, else 0).
// dws: the instance's FP64 workspace (T gen_direct_stage(MB) doubles).  The sweeps run on
// warp 0; every thread of the CTA calls it.
__device__ inline void direct_adjoint_ctx(const Ctx& c, const float* code, const float* bx, float* ex, float* lam,
                                          float* mu, double* dws, double* sh, int* flag) {
    const int NX = c.nx, N = c.n, NG = c.ng, T = c.T;
    const int MB = NX + N + NG, XZ = NX, XH = NX + N, LD = kGenDirectLD;
    const long long ST = gen_direct_stage(MB);
    double* Arow = sh;                      // MB x LD
    double* Erow = Arow + kGenDirectMB * LD;
    double* X = Erow + kGenDirectMB * LD;   // N x N
    double* prow = X + kGenDirectMB * kGenDirectMB;   // 2 MB
    double* yv = prow + 2 * kGenDirectMB;   // MB
    double* wv = yv + kGenDirectMB;         // N
    const bool warp0 = threadIdx.x < 32;
    const int lane = threadIdx.x & 31;
    const bool row = warp0 && lane < MB;
    // entries of the blocks
    auto Am = [&](int t, int k, int j) -> double { return (double)c.Amt(t)[k * N + j]; };
    auto Ap = [&](int t, int k, int j) -> double { return (double)c.Apt(t)[k * N + j]; };
    auto Gv = [&](int t, int q, int j) -> double { return (double)c.Gt(t)[q * N + j]; };
    auto Hsub = [&](int j, int b) -> double { return (j == b && j >= NX) ? -(double)c.W(j - NX) : 0.0; };
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        const double delta = pass == 0 ? 0.0 : 1e-10;
        if (warp0) {
            int singular = 0;
            for (int t = 0; t < T; ++t) {
                double* a = Arow + lane * LD;
                double* e = Erow + lane * LD;
                if (row) {
                    for (int q = 0; q < MB; ++q) { a[q] = 0.0; e[q] = (q == lane) ? 1.0 : 0.0; }
                    if (lane < XZ) {                         // lambda_t row k
                        const int k = lane;
                        for (int j = 0; j < N; ++j) a[XZ + j] = t == 0 ? (j == k ? 1.0 : 0.0) : Ap(t - 1, k, j);
                        a[k] = -delta;
                    } else if (lane < XH) {                  // eta_x,t row j
                        const int j = lane - XZ;
                        for (int k = 0; k < NX; ++k) a[k] = t == 0 ? (j == k ? 1.0 : 0.0) : Ap(t - 1, k, j);
                        a[XZ + j] = (double)c.Pdiag(t, j);
                        for (int q = 0; q < NG; ++q) {
                            const float cd = code[t * NG + q];
                            const double g = Gv(t, q, j);
                            if (fabsf(cd) > 1.5f) {
                                for (int jj = 0; jj < N; ++jj) a[XZ + jj] += (double)c.gam2(q) * g * Gv(t, q, jj);
                            } else if (cd != 0.f) {
                                a[XH + q] = g;
                            }
                        }
                    } else {                                 // eta_h,t row q
                        const int q = lane - XH;
                        const float cd = code[t * NG + q];
                        if (cd != 0.f && fabsf(cd) < 1.5f) {
                            for (int j = 0; j < N; ++j) a[XZ + j] = Gv(t, q, j);
                            a[lane] = -delta;
                        } else {
                            a[lane] = 1.0;
                        }
                    }
                    // Schur complement - P_t X P_t' on the lambda / eta_x rows and columns
                    if (t > 0 && lane < XH) {
                        double u[kGenDirectMB];   // row `lane` of P_t X
                        for (int b = 0; b < N; ++b) {
                            double s = 0.0;
                            for (int q = 0; q < N; ++q)
                                s += (lane < XZ ? Am(t - 1, lane, q) : Hsub(lane - XZ, q)) * X[q * N + b];
                            u[b] = s;
                        }
                        for (int col = 0; col < XH; ++col) {
                            double s = 0.0;
                            for (int b = 0; b < N; ++b) s += u[b] * (col < XZ ? Am(t - 1, col, b) : Hsub(col - XZ, b));
                            a[col] -= s;
                        }
                    }
                }
                __syncwarp();
                // Gauss-Jordan with partial pivoting on the rows in shared memory
                double amax = 0.0;
                if (row)
                    for (int q = 0; q < MB; ++q) amax = fmax(amax, fabs(a[q]));
                for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
                const double tiny = 1e-13 * (amax > 0.0 ? amax : 1.0);
                bool used = !row;
                int mypiv = -1;
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
                        for (int q = 0; q < MB; ++q) {
                            a[q] -= f * prow[q];
                            e[q] -= f * prow[MB + q];
                        }
                    }
                    __syncwarp();
                }
                double* Sinv = dws + (long long)t * ST;
                if (row)
                    for (int q = 0; q < MB; ++q) Sinv[mypiv * MB + q] = e[q];
                if (row) {   // y_t = r_t - P_t w_{t-1}
                    double y = 0.0;
                    if (lane >= XZ && lane < XH) y = (double)bx[t * N + lane - XZ];
                    if (t > 0 && lane < XH)
                        for (int b = 0; b < N; ++b) y -= (lane < XZ ? Am(t - 1, lane, b) : Hsub(lane - XZ, b)) * wv[b];
                    yv[lane] = y;
                    Sinv[MB * MB + lane] = y;
                }
                __syncwarp();
                if (row && mypiv >= XZ && mypiv < XH) {
                    double s = 0.0;
                    for (int q = 0; q < MB; ++q) s += e[q] * yv[q];
                    wv[mypiv - XZ] = s;
                    for (int j = 0; j < N; ++j) X[(mypiv - XZ) * N + j] = e[XZ + j];
                }
                __syncwarp();
            }
            // backward sweep: x_t = S_t^-1 (y_t - P_{t+1}' x_{t+1}); lambda_{t+1} in yv, eta_x,t+1 in wv
            for (int t = T - 1; t >= 0; --t) {
                const double* Sinv = dws + (long long)t * ST;
                if (row) {
                    double v = Sinv[MB * MB + lane];
                    if (t < T - 1 && lane >= XZ && lane < XH) {
                        const int b = lane - XZ;
                        double s = 0.0;
                        for (int k = 0; k < NX; ++k) s += Am(t, k, b) * yv[k];
                        for (int j = 0; j < N; ++j) s += Hsub(j, b) * wv[j];
                        v -= s;
                    }
                    prow[lane] = v;
                }
                __syncwarp();
                double x = 0.0;
                if (row)
                    for (int q = 0; q < MB; ++q) x += Sinv[lane * MB + q] * prow[q];
                __syncwarp();
                if (row) {
                    if (lane < XZ) { lam[t * NX + lane] = (float)x; yv[lane] = x; }
                    else if (lane < XH) { ex[t * N + lane - XZ] = (float)x; wv[lane - XZ] = x; }
                    else {
                        const float cd = code[t * NG + lane - XH];
                        mu[t * NG + lane - XH] = (cd != 0.f && fabsf(cd) < 1.5f) ? (float)x : 0.f;
                    }
                }
                __syncwarp();
            }
            if (lane == 0) *flag = singular;
        }
        __syncthreads();
        const bool sing = *flag != 0;
        __syncthreads();
        if (!sing) return;
    }
}

}  // namespace tmpc
