// Device code of the shared-memory SQP / ADMM path for the small models (see
// tmpc_fast.cuh): S factorisation by block cyclic reduction or a warp-swept
// block LDL', the ADMM iteration, residuals, line search, Algorithm 1 and
// Algorithm 2 per instance, and the persistent / cluster / per-phase kernels.
// Each model's kernels are instantiated in a translation unit of their own
// (tmpc_fast_di.cu, tmpc_fast_bicycle.cu, tmpc_fast_quad.cu).
#pragma once
#include <cuda_runtime.h>

#include "../../include/tmpc.h"
#include "tmpc_backward.cuh"
#include "tmpc_direct.cuh"
#include "tmpc_fast.cuh"
#include "tmpc_fast_api.h"

namespace tmpc {
namespace fast {

// ---------------------------------------------------------------------------
// S blocks and their block cyclic reduction.  Block (stage) e of Dm / Um / Fa
// starts at e * BS; entry (i, j) of a block is at bx(i, j).
// ---------------------------------------------------------------------------
// Entry (i, j) of Theta_t (diagonal block t of S) and of U_t = S[t][t+1] = Phi_t'
// with Phi_t = E_t + rho_f A^+_t' A^-_t  (E_t = -W on the u block; U_t = 0 for t = N)
template <int M>
__device__ __forceinline__ void S_entries(const Inst<M>& c, int t, int i, int j, float sigma, float rho_f, float rho_g,
                                          float& theta, float& u, const float* gw = nullptr) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    float s = 0.f;
    if (t < c.Nh) {
        const float* A = c.Amt(t);
#pragma unroll
        for (int k = 0; k < NX; ++k) s += A[k * N + i] * A[k * N + j];
    }
    if (t > 0 && i < NX && j < NX) {
#pragma unroll
        for (int k = 0; k < NX; ++k) s += c.Ap(t - 1, k, i) * c.Ap(t - 1, k, j);
    }
    if (t == 0 && i == j && i < NX) s += 1.f;
    float v = rho_f * s;
#pragma unroll
    for (int r = 0; r < NG; ++r) v += (gw ? gw[t * NG + r] : rho_g) * c.Gval(t, r, i) * c.Gval(t, r, j);
    if (i == j) v += c.Pd[t * N + i] + sigma;
    theta = v;
    u = 0.f;
    if (t < c.Nh) {
        const float* A = c.Amt(t);
        float a = 0.f;
        if (j < NX) {
#pragma unroll
            for (int k = 0; k < NX; ++k) a += A[k * N + i] * c.Ap(t, k, j);
        }
        u = rho_f * a;
        if (i == j && i >= NX) u -= c.W(i - NX);
    }
}

// Theta_t into Dm, U_t into Um, every stage
template <int M>
__device__ __forceinline__ void form_S(const Inst<M>& c, float sigma, float rho_f, float rho_g,
                                       const float* gw = nullptr) {
    constexpr int N = Inst<M>::N, NN = N * N, BS = Inst<M>::BS;
    const int T = c.T;
    for (int e = c.tid; e < T * NN; e += c.nth) {
        const int t = e / NN, ij = e % NN, i = ij / N, j = ij % N;
        float th, u;
        S_entries<M>(c, t, i, j, sigma, rho_f, rho_g, th, u, gw);
        c.Dm[t * BS + Inst<M>::bx(i, j)] = th;
        c.Um[t * BS + Inst<M>::bx(i, j)] = u;
    }
    c.sync();
}

// In-place inverse of the SPD N x N block at A (N <= 8) by a group of 8
// consecutive lanes: lane i < N keeps row i of [A | I] (lanes N..7 carry zero
// rows and write nothing); Gauss-Jordan elimination without pivoting (the
// pivots of an SPD matrix are positive), pivot rows broadcast by shuffles of
// width 8 inside the group.  Returns false in every lane if a pivot is <= 0.
template <int N>
__device__ __forceinline__ bool group_spd_inverse(float* A, int i, unsigned gmask) {
    static_assert(N <= 8, "lane groups of 8");
    float a[N], e[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        a[j] = (i < N) ? A[blk<N>(i, j)] : 0.f;
        e[j] = (i == j) ? 1.f : 0.f;
    }
    bool ok = true;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        float pa[N], pe[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            pa[j] = __shfl_sync(gmask, a[j], k, 8);
            pe[j] = __shfl_sync(gmask, e[j], k, 8);
        }
        float p = pa[k];
        if (!(p > 0.f)) { ok = false; p = 1.f; }
        const float ip = 1.f / p;
        if (i == k) {
#pragma unroll
            for (int j = 0; j < N; ++j) { a[j] = pa[j] * ip; e[j] = pe[j] * ip; }
        } else {
            const float f = a[k] * ip;
#pragma unroll
            for (int j = 0; j < N; ++j) { a[j] -= f * pa[j]; e[j] -= f * pe[j]; }
        }
    }
    if (i < N)
#pragma unroll
        for (int j = 0; j < N; ++j) A[blk<N>(i, j)] = e[j];
    return __all_sync(gmask, ok);
}

// Block cyclic reduction factorisation of S, in place:
//   Dm[e] <- Dinv_e,  Fa[e] <- Fa_e = U_a Dinv_e,  Fb[e] <- Fb_e = U_e' Dinv_e
// for every stage e eliminated at level s (U_a = S[e-s][e], U_e = S[e][e+s]);
// the surviving diagonal blocks and couplings are updated in Dm / Um.  Work is
// split in row tasks (one row of one block per thread).
// Returns false if a pivot block was not positive definite.
template <int M>
__device__ __forceinline__ bool cr_factor(const Inst<M>& c, int* flag) {
    constexpr int N = Inst<M>::N, BS = Inst<M>::BS;
    const int T = c.T;
    auto bx = [](int i, int j) { return Inst<M>::bx(i, j); };
    if (c.tid == 0) *flag = 0;
    c.sync();
    const int lane_in_group = c.tid % 8, group = c.tid / 8, ngroups = c.nth / 8;
    const unsigned gmask = 0xFFu << ((c.tid % 32) / 8 * 8);
    for (int s = 1; s < T; s <<= 1) {
        const int s2 = s << 1;
        const int ne = (T - s + s2 - 1) / s2;   // eliminated: e = s + q s2 < T
        const int nsv = (T + s2 - 1) / s2;      // surviving:  i = q s2 < T
        for (int q = group; q < ne; q += ngroups)
                if (!group_spd_inverse<N>(c.Dm + (s + q * s2) * BS, lane_in_group, gmask) && lane_in_group == 0)
                    *flag = 1;
        c.sync();
        // row i of Fa_e = U_{e-s} Dinv_e and of Fb_e = U_e' Dinv_e (U_e = S[e][e+s], 0 if e is last)
        for (int w = c.tid; w < ne * N; w += c.nth) {
            const int e = s + (w / N) * s2, i = w % N;
            const float* Ua = c.Um + (e - s) * BS;
            const float* Ue = c.Um + e * BS;
            const float* D = c.Dm + e * BS;
            const bool hasb = e + s < T;
            float ra[N], rb[N];
#pragma unroll
            for (int j = 0; j < N; ++j) { ra[j] = 0.f; rb[j] = 0.f; }
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const float ua = Ua[bx(i, k)], ub = hasb ? Ue[bx(k, i)] : 0.f;
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const float d = D[bx(k, j)];
                    ra[j] += ua * d;
                    rb[j] += ub * d;
                }
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {
                c.Fa[e * BS + bx(i, j)] = ra[j];
                c.Fb[e * BS + bx(i, j)] = rb[j];
            }
        }
        c.sync();
        // row i of D_i0 -= Fa_{i0+s} U_i0' + Fb_{i0-s} U_{i0-s}
        for (int w = c.tid; w < nsv * N; w += c.nth) {
            const int i0 = (w / N) * s2, i = w % N;
            float row[N];
#pragma unroll
            for (int j = 0; j < N; ++j) row[j] = 0.f;
            if (i0 + s < T) {
                const float* F = c.Fa + (i0 + s) * BS;
                const float* U = c.Um + i0 * BS;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float f = F[bx(i, k)];
#pragma unroll
                    for (int j = 0; j < N; ++j) row[j] += f * U[bx(j, k)];
                }
            }
            if (i0 >= s) {
                const float* F = c.Fb + (i0 - s) * BS;
                const float* U = c.Um + (i0 - s) * BS;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float f = F[bx(i, k)];
#pragma unroll
                    for (int j = 0; j < N; ++j) row[j] += f * U[bx(k, j)];
                }
            }
#pragma unroll
            for (int j = 0; j < N; ++j) c.Dm[i0 * BS + bx(i, j)] -= row[j];
        }
        c.sync();
        // row i of the coupling of surviving i0 to i0 + 2s:  U_i0 = -Fa_{i0+s} U_{i0+s}
        for (int w = c.tid; w < nsv * N; w += c.nth) {
            const int i0 = (w / N) * s2, i = w % N;
            float row[N];
#pragma unroll
            for (int j = 0; j < N; ++j) row[j] = 0.f;
            if (i0 + s2 < T) {
                const float* F = c.Fa + (i0 + s) * BS;
                const float* U = c.Um + (i0 + s) * BS;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float f = F[bx(i, k)];
#pragma unroll
                    for (int j = 0; j < N; ++j) row[j] -= f * U[bx(k, j)];
                }
            }
#pragma unroll
            for (int j = 0; j < N; ++j) c.Um[i0 * BS + bx(i, j)] = row[j];
        }
        c.sync();
    }
    if (c.tid < 8 && !group_spd_inverse<N>(c.Dm, c.tid, 0xFFu) && c.tid == 0) *flag = 1;
    c.sync();
    const bool ok = *flag == 0;
    c.sync();
    return ok;
}

// row i of a factor block dotted with an N-vector v (32-byte aligned rows for N = 8)
template <int N>
__device__ __forceinline__ float rowdot(const float* blk_, int i, const float* v) {
    if constexpr (N == 8) {
        const float4 a0 = reinterpret_cast<const float4*>(blk_ + i * 8)[0];
        const float4 a1 = reinterpret_cast<const float4*>(blk_ + i * 8)[1];
        float4 v0 = reinterpret_cast<const float4*>(v)[0], v1 = reinterpret_cast<const float4*>(v)[1];
        if (i & 4) { const float4 t = v0; v0 = v1; v1 = t; }  // swapped halves of rows 4..7
        return (a0.x * v0.x + a0.y * v0.y) + (a0.z * v0.z + a0.w * v0.w) +
               ((a1.x * v1.x + a1.y * v1.y) + (a1.z * v1.z + a1.w * v1.w));
    } else {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k) s += blk_[blk<N>(i, k)] * v[k];
        return s;
    }
}
// column i of a factor block dotted with v
template <int N>
__device__ __forceinline__ float coldot(const float* blk_, int i, const float* v) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) s += blk_[blk<N>(k, i)] * v[k];
    return s;
}

// Inverse of the reduced system left after L = top_level(T, B) levels of the
// cyclic reduction (survivors b = q 2^L, q < top_blocks(T, B), B = c.topb): the
// remaining levels of the factorisation are applied to the m = top_blocks N unit
// vectors.  Column col of Xt holds (M_R^-1) e_col with row q N + i for
// survivor q, row i.  One task per (block, column) works in place.
template <int M>
__device__ __forceinline__ void top_inverse(const Inst<M>& c) {
    constexpr int N = Inst<M>::N, BS = Inst<M>::BS;
    const int T = c.T, L = top_level(T, c.topb), S0 = 1 << L, TD = c.TD;
    const int m = top_blocks(T, c.topb) * N;
    float* X = c.Xt;
    for (int e = c.tid; e < m * TD; e += c.nth) {
        const int col = e / TD, row = e % TD;
        X[e] = (row == col) ? 1.f : 0.f;
    }
    c.sync();
    int top = 1;
    while (top < T) top <<= 1;
    for (int s = S0; s < T; s <<= 1) {
        const int s2 = s << 1, nsv = (T + s2 - 1) / s2;
        for (int w = c.tid; w < nsv * m; w += c.nth) {
            const int col = w / nsv, i0 = (w % nsv) * s2;
            float* x = X + col * TD;
            float acc[N];
#pragma unroll
            for (int i = 0; i < N; ++i) acc[i] = 0.f;
            if (i0 + s < T) {
                const float* F = c.Fa + (i0 + s) * BS;
                const float* v = x + ((i0 + s) >> L) * N;
#pragma unroll
                for (int i = 0; i < N; ++i)
#pragma unroll
                    for (int k = 0; k < N; ++k) acc[i] += F[Inst<M>::bx(i, k)] * v[k];
            }
            if (i0 >= s) {
                const float* F = c.Fb + (i0 - s) * BS;
                const float* v = x + ((i0 - s) >> L) * N;
#pragma unroll
                for (int i = 0; i < N; ++i)
#pragma unroll
                    for (int k = 0; k < N; ++k) acc[i] += F[Inst<M>::bx(i, k)] * v[k];
            }
            float* r0 = x + (i0 >> L) * N;
#pragma unroll
            for (int i = 0; i < N; ++i) r0[i] -= acc[i];
        }
        c.sync();
    }
    for (int col = c.tid; col < m; col += c.nth) {
        float* x = X + col * TD;
        float v[N];
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = x[k];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            float a = 0.f;
#pragma unroll
            for (int k = 0; k < N; ++k) a += c.Dm[Inst<M>::bx(i, k)] * v[k];
            x[i] = a;
        }
    }
    c.sync();
    for (int s = top >> 1; s >= S0; s >>= 1) {
        if (s >= T) continue;
        const int s2 = s << 1, ne = (T - s + s2 - 1) / s2;
        for (int w = c.tid; w < ne * m; w += c.nth) {
            const int col = w / ne, e = s + (w % ne) * s2;
            float* x = X + col * TD;
            const float* D = c.Dm + e * BS;
            const float* Fa = c.Fa + e * BS;
            const float* Fb = c.Fb + e * BS;
            const float* xa = x + ((e - s) >> L) * N;
            const float* xb = x + ((e + s) >> L) * N;
            const bool hasb = e + s < T;
            float* re = x + (e >> L) * N;
            float v[N], o[N];
#pragma unroll
            for (int k = 0; k < N; ++k) v[k] = re[k];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    a += D[Inst<M>::bx(i, k)] * v[k] - Fa[Inst<M>::bx(k, i)] * xa[k];
                    if (hasb) a -= Fb[Inst<M>::bx(k, i)] * xb[k];
                }
                o[i] = a;
            }
#pragma unroll
            for (int i = 0; i < N; ++i) re[i] = o[i];
        }
        c.sync();
    }
}

// Solve S x = r with the cyclic-reduction factors; r is consumed, x -> xo.
// Levels below top_level(T, c.topb): one barrier per level on the way down
// (r_i -= Fa_{i+s} r_{i+s} + Fb_{i-s} r_{i-s}) and one on the way up
// (x_e = Dinv_e r_e - Fa_e' x_{e-s} - Fb_e' x_{e+s}); the survivors in between
// are solved by the dense inverse of the reduced system (one barrier).
template <int M>
__device__ __forceinline__ void cr_solve(const Inst<M>& c, float* r, float* xo) {
    constexpr int N = Inst<M>::N, BS = Inst<M>::BS;
    const int T = c.T, L = top_level(T, c.topb), TD = c.TD;
    const int m = top_blocks(T, c.topb) * N;
    for (int l = 0; l < L; ++l) {
        const int s = 1 << l;
        const int nsv = (T + 2 * s - 1) >> (l + 1);     // survivors i0 = q 2s < T
        // two tasks per thread and step, every load before the stores (a thread writes
        // only its own survivor rows, which no other task of the level reads)
        auto down = [&](int w) {
            const int i0 = (w / N) << (l + 1), i = w % N;
            float a = 0.f;
            if (i0 + s < T) a += rowdot<N>(c.Fa + (i0 + s) * BS, i, r + (i0 + s) * N);
            if (i0 >= s) a += rowdot<N>(c.Fb + (i0 - s) * BS, i, r + (i0 - s) * N);
            return r[i0 * N + i] - a;
        };
        const int nt = nsv * N;
        if (c.cl > 1) {   // cluster teams: several passes over global memory
            for (int w = c.tid; w < nt; w += 2 * c.nth) {
                const int w1 = w + c.nth;
                const float v0 = down(w);
                const float v1 = w1 < nt ? down(w1) : 0.f;
                r[((w / N) << (l + 1)) * N + w % N] = v0;
                if (w1 < nt) r[((w1 / N) << (l + 1)) * N + w1 % N] = v1;
            }
        } else {
            for (int w = c.tid; w < nt; w += c.nth) r[((w / N) << (l + 1)) * N + w % N] = down(w);
        }
        c.sync();
    }
    // survivors: x_R = M_R^-1 r_R (column col of Xt is M_R^-1 e_col); four lanes per
    // row, lane part p summing the columns q N + k with k = p (mod 4), reduced by shuffles
    {
        const int nR = m / N, ntask = 4 * m, nround = (ntask + 31) & ~31;
        for (int w = c.tid; w < nround; w += c.nth) {   // whole warps together
            const int row = w >> 2, part = w & 3;
            float a = 0.f;
            if (w < ntask) {
                const float* Xr = c.Xt + row;
                for (int q = 0; q < nR; ++q) {
                    const float* rq = r + (q << L) * N;
                    const float* Xq = Xr + q * N * TD;
#pragma unroll
                    for (int k = 0; k < N; k += 4)
                        if (k + part < N) a += Xq[(k + part) * TD] * rq[k + part];
                }
            }
            a += __shfl_xor_sync(0xFFFFFFFFu, a, 1);
            a += __shfl_xor_sync(0xFFFFFFFFu, a, 2);
            if (w < ntask && part == 0) xo[((row / N) << L) * N + row % N] = a;
        }
    }
    c.sync();
    for (int l = L - 1; l >= 0; --l) {
        const int s = 1 << l;
        const int ne = (T + s - 1) >> (l + 1);          // eliminated e = s + q 2s < T
        auto up = [&](int w) {
            const int e = s + ((w / N) << (l + 1)), i = w % N;
            float a = rowdot<N>(c.Dm + e * BS, i, r + e * N) - coldot<N>(c.Fa + e * BS, i, xo + (e - s) * N);
            if (e + s < T) a -= coldot<N>(c.Fb + e * BS, i, xo + (e + s) * N);
            return a;
        };
        const int nt = ne * N;
        if (c.cl > 1) {
            for (int w = c.tid; w < nt; w += 2 * c.nth) {
                const int w1 = w + c.nth;
                const float v0 = up(w);
                const float v1 = w1 < nt ? up(w1) : 0.f;
                xo[(s + ((w / N) << (l + 1))) * N + w % N] = v0;
                if (w1 < nt) xo[(s + ((w1 / N) << (l + 1))) * N + w1 % N] = v1;
            }
        } else {
            for (int w = c.tid; w < nt; w += c.nth) xo[(s + ((w / N) << (l + 1))) * N + w % N] = up(w);
        }
        c.sync();
    }
}

// ---------------------------------------------------------------------------
// kLDL: sequential block LDL' of S by warp 0.  Lane l holds entries
// (i, j0), (i, j0 + 1) of an N x N block, i = l / 4, j0 = 2 (l % 4).
//   D_0 = Theta_0;  L_t = U_{t-1}' D_{t-1}^-1,  D_t = Theta_t - L_t U_{t-1}
// Dm[t] <- D_t^-1, Um[t] <- L_t (t >= 1); Theta_t and U_t are formed per step
// (U_t kept in the two scratch blocks Wk for the next step).
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ bool ldl_factor_warp(const Inst<M>& c, float sigma, float rho_f, float rho_g, int* flag) {
    constexpr int N = Inst<M>::N, BS = Inst<M>::BS;
    const int T = c.T;
    if (c.tid == 0) *flag = 0;
    c.sync();
    if (c.tid < 32) {
        const int lane = c.tid, i = lane >> 2, j0 = (lane & 3) * 2, j1 = j0 + 1;
        const bool v0 = i < N && j0 < N, v1 = i < N && j1 < N;
        bool ok = true;
        for (int t = 0; t < T; ++t) {
            float th0 = 0.f, th1 = 0.f, u0 = 0.f, u1 = 0.f;
            if (v0) S_entries<M>(c, t, i, j0, sigma, rho_f, rho_g, th0, u0);
            if (v1) S_entries<M>(c, t, i, j1, sigma, rho_f, rho_g, th1, u1);
            float* Un = c.Wk + (t & 1) * BS;           // U_t for the next step
            if (t > 0) {
                const float* Up = c.Wk + ((t - 1) & 1) * BS;   // U_{t-1}
                const float* Dp = c.Dm + (t - 1) * BS;         // D_{t-1}^-1
                float* Lt = c.Um + t * BS;
                float l0 = 0.f, l1 = 0.f;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float uki = (i < N) ? Up[Inst<M>::bx(k, i)] : 0.f;
                    if (v0) l0 += uki * Dp[Inst<M>::bx(k, j0)];
                    if (v1) l1 += uki * Dp[Inst<M>::bx(k, j1)];
                }
                if (v0) Lt[Inst<M>::bx(i, j0)] = l0;
                if (v1) Lt[Inst<M>::bx(i, j1)] = l1;
                __syncwarp();
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float lik = (i < N) ? Lt[Inst<M>::bx(i, k)] : 0.f;
                    if (v0) th0 -= lik * Up[Inst<M>::bx(k, j0)];
                    if (v1) th1 -= lik * Up[Inst<M>::bx(k, j1)];
                }
            }
            float* Dt = c.Dm + t * BS;
            if (v0) { Dt[Inst<M>::bx(i, j0)] = th0; Un[Inst<M>::bx(i, j0)] = u0; }
            if (v1) { Dt[Inst<M>::bx(i, j1)] = th1; Un[Inst<M>::bx(i, j1)] = u1; }
            __syncwarp();
            if (lane < 8) ok = group_spd_inverse<N>(Dt, lane, 0xFFu) && ok;
            __syncwarp();
        }
        if (lane == 0 && !ok) *flag = 1;
    }
    c.sync();
    const bool res = *flag == 0;
    c.sync();
    return res;
}

// Solve S x = r in place with the kLDL factors (warp 0):
//   y_0 = r_0, y_t = r_t - L_t y_{t-1};   x_{T-1} = D^-1 y,  x_t = D_t^-1 y_t - L_{t+1}' x_{t+1}
// A lane holds y (or x) entries j0, j0 + 1 of the previous stage; row sums over
// the 4 lanes of a row by xor-shuffles, redistributed from the row's lane 0.
template <int M>
__device__ __forceinline__ void ldl_solve_warp(const Inst<M>& c, float* r) {
    constexpr int N = Inst<M>::N, BS = Inst<M>::BS;
    const int T = c.T;
    if (c.tid < 32) {
        const unsigned full = 0xFFFFFFFFu;
        const int lane = c.tid, i = lane >> 2, h = lane & 3, j0 = 2 * h, j1 = j0 + 1;
        const bool vi = i < N, v0 = j0 < N, v1 = j1 < N;
        float y0 = v0 ? r[j0] : 0.f, y1 = v1 ? r[j1] : 0.f;
        for (int t = 1; t < T; ++t) {
            const float* Lb = c.Um + t * BS;
            const float rt = (vi && h == 0) ? r[t * N + i] : 0.f;
            float p = 0.f;
            if (vi && v0) p += Lb[Inst<M>::bx(i, j0)] * y0;
            if (vi && v1) p += Lb[Inst<M>::bx(i, j1)] * y1;
            p += __shfl_xor_sync(full, p, 1);
            p += __shfl_xor_sync(full, p, 2);
            const float yi = rt - p;
            if (vi && h == 0) r[t * N + i] = yi;
            y0 = __shfl_sync(full, yi, 4 * j0);
            y1 = __shfl_sync(full, yi, 4 * j1);
        }
        float x0 = 0.f, x1 = 0.f;
        for (int t = T - 1; t >= 0; --t) {
            const float* D = c.Dm + t * BS;
            const float* yt = r + t * N;
            float p = 0.f;
            if (vi && v0) p += D[Inst<M>::bx(i, j0)] * yt[j0];
            if (vi && v1) p += D[Inst<M>::bx(i, j1)] * yt[j1];
            if (t + 1 < T) {
                const float* Ln = c.Um + (t + 1) * BS;
                if (vi && v0) p -= Ln[Inst<M>::bx(j0, i)] * x0;
                if (vi && v1) p -= Ln[Inst<M>::bx(j1, i)] * x1;
            }
            p += __shfl_xor_sync(full, p, 1);
            p += __shfl_xor_sync(full, p, 2);
            __syncwarp();
            if (vi && h == 0) r[t * N + i] = p;
            x0 = __shfl_sync(full, p, 4 * j0);
            x1 = __shfl_sync(full, p, 4 * j1);
        }
    }
    c.sync();
}

// ---------------------------------------------------------------------------
// model evaluation (one thread per stage)
// ---------------------------------------------------------------------------
// f_t(z_t, z_{t+1}) and optionally the dense A^-_t (NX x N, row-major)
template <int M>
__device__ __forceinline__ void dyn_eval(const Inst<M>& c, const float* zt, const float* zn, float* f, float* Am) {
    constexpr int N = Inst<M>::N;
    if constexpr (M == MODEL_DI) {
        const float dt = c.dyn[0];
        f[0] = zt[0] + dt * zt[2] + 0.5f * dt * dt * zt[4] - zn[0];
        f[1] = zt[1] + dt * zt[3] + 0.5f * dt * dt * zt[5] - zn[1];
        f[2] = zt[2] + dt * zt[4] - zn[2];
        f[3] = zt[3] + dt * zt[5] - zn[3];
    } else if constexpr (M == MODEL_QUAD) {
        float phi[6], dPx[36], dPu[12];
        quad_rk4(zt, zt + 6, c.dyn, phi, Am ? dPx : nullptr, Am ? dPu : nullptr);
#pragma unroll
        for (int k = 0; k < 6; ++k) f[k] = phi[k] - zn[k];
        if (Am) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
#pragma unroll
                for (int j = 0; j < 6; ++j) Am[k * N + j] = dPx[k * 6 + j];
                Am[k * N + 6] = dPu[k * 2];
                Am[k * N + 7] = dPu[k * 2 + 1];
            }
        }
    } else {  // bicycle, implicit midpoint
        const float dt = c.dyn[0];
        float mid[6], fc[6], Jx[36], Ju[12];
#pragma unroll
        for (int k = 0; k < 6; ++k) mid[k] = 0.5f * (zt[k] + zn[k]);
        bicycle_fc(mid, zt + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fc, Am ? Jx : nullptr, Am ? Ju : nullptr);
#pragma unroll
        for (int k = 0; k < 6; ++k) f[k] = zt[k] + dt * fc[k] - zn[k];
        if (Am) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
#pragma unroll
                for (int j = 0; j < 6; ++j) Am[k * N + j] = (k == j ? 1.f : 0.f) + 0.5f * dt * Jx[k * 6 + j];
                Am[k * N + 6] = dt * Ju[k * 2];
                Am[k * N + 7] = dt * Ju[k * 2 + 1];
            }
        }
    }
}

// g_t(z) and the dense row of G_t (if the model has one)
template <int M>
__device__ __forceinline__ void con_eval(const Inst<M>& c, const float* z, float* g, float* grow) {
    using Tr = Traits<M>;
#pragma unroll
    for (int r = 0; r < Tr::NG; ++r)
        if (Tr::sel(r) >= 0) g[r] = z[Tr::sel(r)];
    if constexpr (Tr::DENSE_ROW >= 0) {  // lateral track error of the bicycle
        TrackPt tp = track_eval(c.track, c.nt, c.dyn[2], z[5]);
        float sp, cp;
        sincosf(tp.psic, &sp, &cp);
        const float dx = z[0] - tp.xc, dy = z[1] - tp.yc;
        g[Tr::DENSE_ROW] = -dx * sp + dy * cp;
        if (grow) {
#pragma unroll
            for (int j = 0; j < 8; ++j) grow[j] = 0.f;
            grow[0] = -sp;
            grow[1] = cp;
            grow[5] = tp.dxc * sp - tp.dyc * cp - tp.dpsic * (dx * cp + dy * sp);
        }
    }
}

// ---------------------------------------------------------------------------
// initial guess (same as tmpc_solver.cuh rollout)
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void rollout(const Inst<M>& c, int newton_steps) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX;
    for (int e = c.tid; e < c.T * N; e += c.nth) {
        const int t = e / N, j = e % N;
        c.zb[e] = (j >= NX) ? c.refv(t, j) : (t == 0 ? c.x0[j] : 0.f);
    }
    c.sync();
    if (c.tid == 0) {
        for (int t = 0; t < c.Nh; ++t) {
            const float* z = c.zb + t * N;
            float xn[NX];
            if constexpr (M == MODEL_QUAD) {
                quad_rk4<float>(z, z + 6, c.dyn, xn, nullptr, nullptr);
            } else if constexpr (M == MODEL_DI) {
                const float dt = c.dyn[0];
                xn[0] = z[0] + dt * z[2] + 0.5f * dt * dt * z[4];
                xn[1] = z[1] + dt * z[3] + 0.5f * dt * dt * z[5];
                xn[2] = z[2] + dt * z[4];
                xn[3] = z[3] + dt * z[5];
            } else {
                float fc[6], zn[8], f[6], Am[6 * 8], Mx[36];
                bicycle_fc<float>(z, z + 6, c.dyn[1], c.track, c.nt, c.dyn[2], fc, nullptr, nullptr);
#pragma unroll
                for (int k = 0; k < 6; ++k) xn[k] = z[k] + c.dyn[0] * fc[k];
                for (int it = 0; it < newton_steps; ++it) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) zn[k] = xn[k];
                    zn[6] = c.zb[(t + 1) * N + 6];
                    zn[7] = c.zb[(t + 1) * N + 7];
                    dyn_eval<M>(c, z, zn, f, Am);
                    // d f / d x_{t+1} = A^+_x = A^-_x - 2 I
#pragma unroll
                    for (int k = 0; k < 6; ++k)
#pragma unroll
                        for (int j = 0; j < 6; ++j) Mx[k * 6 + j] = Am[k * N + j] - (k == j ? 2.f : 0.f);
                    small_solve(Mx, f, 6);
#pragma unroll
                    for (int k = 0; k < 6; ++k) xn[k] -= f[k];
                }
            }
#pragma unroll
            for (int k = 0; k < NX; ++k) c.zb[(t + 1) * N + k] = xn[k];
        }
    }
    c.sync();
}

// QP approximation at zb in step coordinates (see tmpc_solver.cuh linearize)
template <int M>
__device__ __forceinline__ void linearize(const Inst<M>& c) {
    using Tr = Traits<M>;
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    const int T = c.T;
    if constexpr (Tr::LTI) {  // double integrator, ZOH
        if (c.tid == 0) {
            const float dt = c.dyn[0];
            for (int i = 0; i < NX * N; ++i) c.Am[i] = 0.f;
            for (int k = 0; k < 4; ++k) c.Am[k * N + k] = 1.f;
            c.Am[0 * N + 2] = dt; c.Am[1 * N + 3] = dt;
            c.Am[0 * N + 4] = 0.5f * dt * dt; c.Am[1 * N + 5] = 0.5f * dt * dt;
            c.Am[2 * N + 4] = dt; c.Am[3 * N + 5] = dt;
        }
    }
    for (int t = c.tid; t < T; t += c.nth) {
        const float* z = c.zb + t * N;
        if (t < c.Nh) {
            float f[NX];
            dyn_eval<M>(c, z, z + N, f, Tr::LTI ? nullptr : c.Am + t * Inst<M>::AMS);
#pragma unroll
            for (int k = 0; k < NX; ++k) c.cv[(t + 1) * NX + k] = -f[k];
        }
        if (t == 0)
#pragma unroll
            for (int k = 0; k < NX; ++k) c.cv[k] = c.x0[k] - z[k];
        float g[NG];
        con_eval<M>(c, z, g, Tr::DENSE_ROW >= 0 ? c.Grow + t * N : nullptr);
#pragma unroll
        for (int r = 0; r < NG; ++r) {
            c.glo[t * NG + r] = c.lob(t, r) - g[r];
            c.ghi[t * NG + r] = c.hib(t, r) - g[r];
        }
    }
    for (int e = c.tid; e < T * N; e += c.nth) {
        const int t = e / N, j = e % N;
        float gr = c.Cw(t, j) * (c.zb[e] - c.refv(t, j)) + c.linv(t, j);
        float pd = c.Cw(t, j);
        if (j >= NX) {
            const float w = c.W(j - NX);
            if (t < c.Nh) { gr += w * (c.zb[e] - c.zb[e + N]); pd += w; }
            if (t > 0) { gr -= w * (c.zb[e - N] - c.zb[e]); pd += w; }
        }
        c.qv[e] = gr;
        c.Pd[e] = pd;
    }
    c.sync();
}

// ---------------------------------------------------------------------------
// Problem rescaling (Remark 4): the ADMM of an instance with scales runs on the
// QP in normalised variables z = D zh, D = diag(d) on every stage, d_j a power
// of two.  The dynamics rows are divided by the scale of the state they define
// (E_f = D_x^-1, so that A^+ keeps its [-I 0] / [A^-_x - 2I, 0] form), a bound
// row of one variable by that variable's scale (it stays a unit selector), the
// dense row is left as it is (e = 1).  In scaled units:
//   A^- -> D_x^-1 A^- D,  G row -> e G D,  P -> D P D (Pd and the rate weight W),
//   q -> D q,  c -> E_f c,  bounds -> e lo, e hi,  gamma2 -> gamma2 / e^2,
//   gamma1 -> gamma1 / e,  z -> D^-1 z,  xi -> e xi,  y_f -> E_f^-1 y_f,
//   y_g -> y_g / e,  z_g -> e z_g.
// back = false maps the linearisation, the SQP iterate and its multipliers into
// scaled units before the factorisation; back = true maps everything, the ADMM
// result included, back to physical units before the line search.  Every factor
// is a power of two, so both directions are exact.
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void rescale(const Inst<M>& c, bool back) {
    using Tr = Traits<M>;
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NU = Inst<M>::NU, NG = Inst<M>::NG, AMS = Inst<M>::AMS;
    const int T = c.T;
    const float* d = c.par + kParScale;
    // u_j: the factor of a quantity that scales like d_j (q, a column of C or G)
    auto u = [&](int j) { return back ? 1.f / d[j] : d[j]; };
    const int nam = (Tr::LTI ? 1 : c.Nh) * NX * N;
    for (int e = c.tid; e < nam; e += c.nth) {
        const int kj = e % (NX * N), k = kj / N, j = kj % N;
        c.Am[(e / (NX * N)) * AMS + kj] *= u(j) / u(k);
    }
    for (int e = c.tid; e < T * N; e += c.nth) {
        const float f = u(e % N);
        c.Pd[e] *= f * f;
        c.qv[e] *= f;
        c.zb[e] /= f;
        c.x[e] /= f;
        if (Tr::DENSE_ROW >= 0) c.Grow[e] *= f;
    }
    for (int e = c.tid; e < T * NX; e += c.nth) {
        const float f = u(e % NX);
        c.cv[e] /= f;
        c.yfb[e] *= f;
        c.yf[e] *= f;
    }
    for (int e = c.tid; e < T * NG; e += c.nth) {
        const int s = Tr::sel(e % NG);
        if (s >= 0) {
            const float f = u(s);   // 1 / e of the row
            c.glo[e] /= f;
            c.ghi[e] /= f;
            c.xib[e] /= f;
            c.xi[e] /= f;
            c.zg[e] /= f;
            c.ygb[e] *= f;
            c.yg[e] *= f;
        }
    }
    if (c.tid == 0) {   // the loops above read only the scales of par, not these weights
        float* par = c.par;
        for (int k = 0; k < NU; ++k) par[k] *= u(NX + k) * u(NX + k);
        for (int r = 0; r < NG; ++r) {
            const int s = Tr::sel(r);
            if (s >= 0) {
                par[NU + r] *= u(s) * u(s);   // gamma2 (infinite on a hard row: stays infinite)
                par[NU + NG + r] *= u(s);     // gamma1
            }
        }
    }
    c.sync();
}

// ---------------------------------------------------------------------------
// one ADMM iteration in increment form (see tmpc_solver.cuh admm_iter)
// ---------------------------------------------------------------------------
// Row vectors of the right-hand side, w_f = y_f + rho_f p_f and
// w_g = y_g + rho_g p_g, from the tracked defects p_f = C x - c and
// p_g = G x - z_g (at the start of the ADMM loop and after a change of rho;
// otherwise the fused update of admm_iter produces them).
template <int M>
__device__ __forceinline__ void admm_rowvec(const Inst<M>& c, float rho_bar) {
    constexpr int NX = Inst<M>::NX, NG = Inst<M>::NG;
    const int T = c.T;
    const float rho_f = 1e3f * rho_bar, rho_g = rho_bar;
    for (int e = c.tid; e < T * NX; e += c.nth) c.wf[e] = c.yf[e] + rho_f * c.pf[e];
    for (int e = c.tid; e < T * NG; e += c.nth) c.wg[e] = c.yg[e] + rho_g * c.pg[e];
    c.sync();
}

// r = -(P x + q) - C' w_f - G' w_g;  S dx = r;  then one fused pass over the
// stage entries (t, j): x += alpha dx, equality row (t, j < NX) and
// inequality row (t, j < NG) relaxed, projected and dual-updated, and the
// next iteration's w_f, w_g.  G x is tracked through p_g like C x through p_f.
template <int M, int P>
__device__ __forceinline__ void admm_iter(const Inst<M>& c, float rho_bar, float alpha, float sigma) {
    using Tr = Traits<M>;
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    const int T = c.T;
    const float rho_f = 1e3f * rho_bar, rho_g = rho_bar, inv_rho_g = 1.f / rho_bar;
    auto rhs = [&](int e) {
        const int t = e / N, j = e % N;
        float s = -(c.Pv(c.x, t, j) + c.qv[e]);
        s -= c.Ctv(t, j, [&](int row, int k) { return c.wf[row * NX + k]; });
        const float* wg = c.wg + t * NG;
#pragma unroll
        for (int r = 0; r < NG; ++r) {
            if (Tr::sel(r) >= 0) { if (Tr::sel(r) == j) s -= wg[r]; }
            else s -= c.Grow[t * N + j] * wg[r];
        }
        return s;
    };
    if (c.cl > 1) {   // cluster teams: two entries per step, loads before stores
        for (int e = c.tid; e < T * N; e += 2 * c.nth) {
            const int e1 = e + c.nth;
            const float s0 = rhs(e);
            const float s1 = e1 < T * N ? rhs(e1) : 0.f;
            c.r[e] = s0;
            if (e1 < T * N) c.r[e1] = s1;
        }
    } else {
        for (int e = c.tid; e < T * N; e += c.nth) c.r[e] = rhs(e);
    }
    c.sync();
    if (P == kCR) {
        if (c.cl > 1) {
            // cluster teams (horizons of thousands of stages): one step of iterative
            // refinement, dx += S^-1 (r - S dx) with S dx formed matrix-free, so that
            // the FP32 solve through the many reduction levels stays accurate enough
            // for ADMM (without it one long racing instance diverged in FP32)
            for (int e = c.tid; e < T * N; e += c.nth) c.rs[e] = c.r[e];
            c.sync();
            cr_solve<M>(c, c.r, c.dx);
            for (int e = c.tid; e < T * NX; e += c.nth) c.rcx[e] = c.Cx(c.dx, e / NX, e % NX);
            for (int e = c.tid; e < T * NG; e += c.nth) c.rgx[e] = c.Gx(c.dx, e / NG, e % NG);
            c.sync();
            for (int e = c.tid; e < T * N; e += c.nth) {
                const int t = e / N, j = e % N;
                float sv = c.Pv(c.dx, t, j) + sigma * c.dx[e];
                sv += rho_f * c.Ctv(t, j, [&](int row, int k) { return c.rcx[row * NX + k]; });
                sv += rho_g * c.Gtw(t, j, [&](int r) { return c.rgx[t * NG + r]; });
                c.rs[e] -= sv;
            }
            c.sync();
            cr_solve<M>(c, c.rs, c.rd);
            for (int e = c.tid; e < T * N; e += c.nth) c.dx[e] += c.rd[e];
            c.sync();
        } else {
            cr_solve<M>(c, c.r, c.dx);
        }
    } else {
        ldl_solve_warp<M>(c, c.r);   // dx shares r
    }
    for (int e = c.tid; e < T * N; e += c.nth) {
        const int t = e / N, j = e % N;
        c.x[e] += alpha * c.dx[e];
        if (j < NX) {
            const int f = t * NX + j;
            const float cd = c.Cx(c.dx, t, j);
            const float yf = c.yf[f] + rho_f * alpha * (c.pf[f] + cd);
            const float pf = c.pf[f] + alpha * cd;
            c.yf[f] = yf;
            c.pf[f] = pf;
            c.wf[f] = yf + rho_f * pf;
        }
        if (j < NG) {
            const int g = t * NG + j;
            const float gd = c.Gx(c.dx, t, j);
            const float zg = c.zg[g], pg = c.pg[g], yg0 = c.yg[g];
            const float zh = zg + alpha * (pg + gd);
            float zn, xn;
            project(zh + yg0 * inv_rho_g, c.glo[g], c.ghi[g], rho_g, c.gam2(j), c.gam1(j), zn, xn);
            const float yg = yg0 + rho_g * (zh - zn);
            const float pgn = (pg + zg + alpha * gd) - zn;   // G x_new - z_g,new
            c.yg[g] = yg;
            c.zg[g] = zn;
            c.xi[g] = xn;
            c.pg[g] = pgn;
            c.wg[g] = yg + rho_g * pgn;
        }
    }
    c.sync();
}

// ---------------------------------------------------------------------------
// team reductions: the CTA reduction, then (cluster teams) one partial per CTA
// through the global exchange area, the team barrier and a sum / max over CTAs
// ---------------------------------------------------------------------------
template <int M, int K>
__device__ __forceinline__ void team_max_k(const Inst<M>& c, float (&v)[K], float* red) {
    static_assert(K <= kXchDoubles, "exchange area");
    cta_max_k<K>(v, red);
    if (c.cl > 1) {
        if (threadIdx.x == 0)
            for (int k = 0; k < K; ++k) c.xch[c.rank * kXchDoubles + k] = (double)v[k];
        c.sync();
        for (int k = 0; k < K; ++k) {
            float m = v[k];
            for (int q = 0; q < c.cl; ++q) m = fmaxf(m, (float)c.xch[q * kXchDoubles + k]);
            v[k] = m;
        }
        c.sync();
    }
}

template <int M>
__device__ __forceinline__ double team_sum_d(const Inst<M>& c, double v, double* redd) {
    v = cta_sum_d(v, redd);
    if (c.cl > 1) {
        if (threadIdx.x == 0) c.xch[c.rank * kXchDoubles] = v;
        c.sync();
        double s = 0.0;
        for (int q = 0; q < c.cl; ++q) s += c.xch[q * kXchDoubles];
        v = s;
        c.sync();
    }
    return v;
}

// residuals and normalisers (see tmpc_solver.cuh residuals)
template <int M>
__device__ __forceinline__ Res residuals(const Inst<M>& c, float* red) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    const int T = c.T;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    for (int e = c.tid; e < T * NX; e += c.nth) {
        const float cabs = c.cv[e] + c.Cx(c.zb, e / NX, e % NX);
        v[0] = fmaxf(v[0], fin(c.pf[e]));
        v[2] = fmaxf(v[2], fmaxf(fin(c.pf[e] + cabs), fin(cabs)));
    }
    for (int e = c.tid; e < T * NG; e += c.nth) {
        const int t = e / NG, r = e % NG;
        const float gx = c.Gx(c.x, t, r), gzb = c.Gx(c.zb, t, r);
        v[0] = fmaxf(v[0], fin(gx - c.zg[e]));
        v[2] = fmaxf(v[2], fmaxf(fin(gx + gzb), fin(c.zg[e] + gzb)));
        const float g2 = c.gam2(r);
        if (g2 < kInf) {
            v[1] = fmaxf(v[1], fin(slack_res(c.xi[e], c.yg[e], g2, c.gam1(r))));
            v[3] = fmaxf(v[3], fmaxf(fin(g2 * c.xi[e]), fin(c.yg[e])));
        }
    }
    for (int e = c.tid; e < T * N; e += c.nth) {
        const int t = e / N, j = e % N;
        const float px = c.Pv(c.x, t, j), pzb = c.Pv(c.zb, t, j);
        const float aty = c.Ctv(t, j, [&](int row, int k) { return c.yf[row * NX + k]; }) +
                          c.Gtw(t, j, [&](int r) { return c.yg[t * NG + r]; });
        v[1] = fmaxf(v[1], fin(px + c.qv[e] + aty));
        v[3] = fmaxf(v[3], fmaxf(fmaxf(fin(px + pzb), fin(aty)), fin(c.qv[e] - pzb)));
    }
    team_max_k<M, 4>(c, v, red);
    return {v[0], v[1], v[2], v[3]};
}

// merit contributions of stage t at zb + a x (Appendix D), in FP32: cost
// (incl. slack penalty), constraint violation V, and the magnitude of the
// numbers entering both (for the FP32 tie allowance of the Armijo test)
template <int M>
__device__ __forceinline__ void stage_merit(const Inst<M>& c, int t, float a, float& cost, float& viol, float& scale) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NU = Inst<M>::NU, NG = Inst<M>::NG;
    float z[N], zn[N], f[NX], g[NG];
#pragma unroll
    for (int j = 0; j < N; ++j) z[j] = c.zb[t * N + j] + a * c.x[t * N + j];
    float cs = 0.f, vs = 0.f, sc = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const float d = z[j] - c.refv(t, j);
        const float q = 0.5f * c.Cw(t, j) * d * d, l = c.linv(t, j) * z[j];
        cs += q + l;
        sc += q + fabsf(l) + 2.f * fabsf(z[j]);
    }
    if (t < c.Nh) {
#pragma unroll
        for (int j = 0; j < N; ++j) zn[j] = c.zb[(t + 1) * N + j] + a * c.x[(t + 1) * N + j];
#pragma unroll
        for (int k = 0; k < NU; ++k) {
            const float d = z[NX + k] - zn[NX + k];
            cs += 0.5f * c.W(k) * d * d;
        }
        dyn_eval<M>(c, z, zn, f, nullptr);
#pragma unroll
        for (int k = 0; k < NX; ++k) vs += fabsf(f[k]);
    }
    if (t == 0)
#pragma unroll
        for (int k = 0; k < NX; ++k) vs += fabsf(z[k] - c.x0[k]);
    con_eval<M>(c, z, g, nullptr);
#pragma unroll
    for (int r = 0; r < NG; ++r) {
        const float xi = c.xib[t * NG + r] + a * (c.xi[t * NG + r] - c.xib[t * NG + r]);
        const float g2 = c.gam2(r);
        if (g2 < kInf) cs += 0.5f * g2 * xi * xi + c.gam1(r) * fabsf(xi);
        const float gx = g[r] + xi;
        vs += fmaxf(gx - c.hib(t, r), 0.f) + fmaxf(c.lob(t, r) - gx, 0.f);
    }
    cost = cs;
    viol = vs;
    scale = sc + fabsf(cs);
}

struct Red {
    float* red;
    double* redd;
    double* lsacc;
    int* flags;
};

// Appendix D line search.  Stage values of every candidate are written in
// FP32 to scratch (the factor arena is idle here: the next SQP step refactors),
// then one thread per (candidate, quantity) sums its stages in FP64.
template <int M, int P>
__device__ __forceinline__ float linesearch(const Inst<M>& c, const KOpts& o, const Red& rs, float ystar_inf) {
    constexpr int N = Inst<M>::N, NG = Inst<M>::NG;
    const int T = c.T;
    const int K = o.n_ls < 1 ? 1 : (o.n_ls > kMaxLs ? kMaxLs : o.n_ls);
    if (K == 1) return 1.f;
    // scratch [(2k + q) T + t], q = 0 cost, 1 violation; scale at 2(K+1)T (factors are dead here)
    float* val = P == kCR ? c.Fa : c.Dm;
    double gd = 0.0;
    for (int e = c.tid; e < T * N; e += c.nth) gd += (double)(c.qv[e] * c.x[e]);
    for (int e = c.tid; e < T * NG; e += c.nth) {
        const int r = e % NG;
        const float g2 = c.gam2(r);
        if (g2 < kInf) {
            const float x0 = c.xib[e], dx = c.xi[e] - c.xib[e];
            gd += (double)(g2 * x0 * dx + c.gam1(r) * (x0 != 0.f ? (x0 > 0.f ? dx : -dx) : fabsf(dx)));
        }
    }
    gd = team_sum_d<M>(c, gd, rs.redd);
    for (int e = c.tid; e < (K + 1) * T; e += c.nth) {
        const int k = e / T, t = e % T;
        const float a = k == 0 ? 0.f : ldexpf(1.f, -(k - 1));
        float cs, vs, sc;
        stage_merit<M>(c, t, a, cs, vs, sc);
        val[(2 * k) * T + t] = cs;
        val[(2 * k + 1) * T + t] = vs;
        if (k == 0) val[2 * (K + 1) * T + t] = sc;
    }
    c.sync();
    // per-candidate sums over the stages, split over the team four at a time
    // (team reductions; a cluster team keeps them in its exchange area)
    const int nq = 2 * (K + 1) + 1;
    double* acc = c.cl > 1 ? c.xch + kTeamMax * kXchDoubles : rs.lsacc;
    if (c.cl == 1) {   // short horizons in one CTA: one thread per sum
        for (int q = c.tid; q < nq; q += c.nth) {
            double sum = 0.0;
            for (int t = 0; t < T; ++t) sum += (double)val[q * T + t];
            acc[q] = sum;
        }
    } else for (int q0 = 0; q0 < nq; q0 += 4) {
        double part[4] = {0.0, 0.0, 0.0, 0.0};
        for (int t = c.tid; t < T; t += c.nth)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (q0 + u < nq) part[u] += (double)val[(q0 + u) * T + t];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double tot = team_sum_d<M>(c, part[u], rs.redd);
            if (q0 + u < nq && c.tid == 0) acc[q0 + u] = tot;
        }
    }
    c.sync();
    const double l0 = acc[0], V0 = acc[1];
    const double mu = fmax(gd / (0.5 * fmax(V0, (double)o.eps_c)), (double)ystar_inf + 1e-4);
    const double phi0 = l0 + mu * V0;
    const double D = gd - mu * V0;
    // FP32 evaluation error of the merit: differences below it are ties, and a
    // tie satisfies the Armijo test (4 units of FP32 rounding on the magnitude
    // of every term that enters phi)
    const double tau = 4.0 * 5.9604644775390625e-08 * acc[2 * (K + 1)] * fmax(1.0, mu);
    float chosen = -1.f, best = 0.f;
    double best_phi = INFINITY;
    for (int k = 1; k <= K; ++k) {
        const float a = ldexpf(1.f, -(k - 1));
        const double ph = acc[2 * k] + mu * acc[2 * k + 1];
        if (isfinite(ph) && ph <= phi0 + (double)o.ls_eta * a * D + tau) { chosen = a; break; }
    }
    if (chosen < 0.f) {
        for (int k = 1; k <= K; ++k) {
            const float a = ldexpf(1.f, -(k - 1));
            const double ph = acc[2 * k] + mu * acc[2 * k + 1];
            if (isfinite(ph) && ph < best_phi) { best_phi = ph; best = a; }
        }
        chosen = best;
    }
    c.sync();
    return chosen;
}

// KKT residual of Eq. (sqp_stop) at (zb, xib, yfb, ygb) with the current linearisation
template <int M>
__device__ __forceinline__ float kkt(const Inst<M>& c, float* red) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    const int T = c.T;
    float v[1] = {0.f};
    for (int e = c.tid; e < T * N; e += c.nth) {
        const int t = e / N, j = e % N;
        const float gr = c.qv[e] + c.Ctv(t, j, [&](int row, int k) { return c.yfb[row * NX + k]; }) +
                         c.Gtw(t, j, [&](int r) { return c.ygb[t * NG + r]; });
        v[0] = fmaxf(v[0], fin(gr));
    }
    for (int e = c.tid; e < T * NX; e += c.nth) v[0] = fmaxf(v[0], fin(c.cv[e]));
    for (int e = c.tid; e < T * NG; e += c.nth) {
        const int r = e % NG;
        const float g2 = c.gam2(r);
        if (g2 < kInf) v[0] = fmaxf(v[0], fin(slack_res(c.xib[e], c.ygb[e], g2, c.gam1(r))));
        // bound violation of g + xi:  g + xi - hi = xi - ghi,  lo - g - xi = glo - xi
        v[0] = fmaxf(v[0], fmaxf(c.xib[e] - c.ghi[e], c.glo[e] - c.xib[e]));
    }
    team_max_k<M, 1>(c, v, red);
    return v[0];
}

template <int M, int P>
__device__ __forceinline__ bool factor(const Inst<M>& c, const KOpts& o, float rho, int* flag) {
    if (P == kLDL) return ldl_factor_warp<M>(c, o.sigma, 1e3f * rho, rho, flag);
    form_S<M>(c, o.sigma, 1e3f * rho, rho);
    const bool ok = cr_factor<M>(c, flag);
    top_inverse<M>(c);
    return ok;
}

// A factorisation of S failed (uniform over the team): classify it by the data S
// is formed from.  A NaN in the stage Jacobians A^-_t, the dense G row or the
// cost Hessian diagonal is a NaN event (bit 2 of the instance flag); otherwise a
// pivot block of a finite S was not positive definite (bit 1).
template <int M>
__device__ __forceinline__ void note_factor_failure(const Inst<M>& c, float* red) {
    using Tr = Traits<M>;
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, AMS = Inst<M>::AMS;
    float v[1] = {0.f};
    const int nam = (Tr::LTI ? 1 : c.Nh) * NX * N;   // A^-_t is written for t < N only
    for (int e = c.tid; e < nam; e += c.nth) {
        const float a = c.Am[(e / (NX * N)) * AMS + e % (NX * N)];
        if (a != a) v[0] = 1.f;
    }
    for (int e = c.tid; e < c.T * N; e += c.nth) {
        const float g = Tr::DENSE_ROW >= 0 ? c.Grow[e] : 0.f;
        if (c.Pd[e] != c.Pd[e] || g != g) v[0] = 1.f;
    }
    team_max_k<M, 1>(c, v, red);
    if (c.tid == 0) c.tflags[0] |= v[0] > 0.f ? 2 : 1;
    c.sync();
}

// per-instance status from the instance flag (bit 1: a pivot block was not
// positive definite, bit 2: NaN met by a factorisation), the final point and
// its KKT residual: the root cause first
__device__ __forceinline__ int instance_status(int flags, bool finite, float kkt, float eps_c) {
    if (flags & 2) return TMPC_INST_NAN;
    if (flags & 1) return TMPC_INST_NOT_PD;
    if (!finite || !(kkt < kInf)) return TMPC_INST_NAN;
    return kkt <= eps_c ? TMPC_INST_OK : TMPC_INST_MAX_ITER;
}

// ---------------------------------------------------------------------------
// Algorithm 1 for one instance
// ---------------------------------------------------------------------------
template <int M, int P>
__device__ __forceinline__ void solve_instance(Inst<M>& c, const KOpts& o, const Red& rs, const KLayout& L, const KSol& out,
                               int inst, int warm) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    const int T = c.T;
    if (c.tid == 0) c.tflags[0] = o.force_fail == inst + 1;   // NOT_PD flag (forced by the caller for one instance)
    c.cache_params();
    const long long Ts = L.Nmax + 1;
    if (warm) {
        const float* z = out.z + inst * Ts * L.n;
        const float* xi = out.xi + inst * Ts * L.ng;
        const float* yf = out.yf + inst * Ts * L.nx;
        const float* yg = out.yg + inst * Ts * L.ng;
        for (int e = c.tid; e < T * N; e += c.nth) c.zb[e] = z[(e / N) * L.n + e % N];
        for (int e = c.tid; e < T * NG; e += c.nth) {
            c.xib[e] = xi[(e / NG) * L.ng + e % NG];
            c.ygb[e] = yg[(e / NG) * L.ng + e % NG];
        }
        for (int e = c.tid; e < T * NX; e += c.nth) c.yfb[e] = yf[(e / NX) * L.nx + e % NX];
        c.sync();
    } else {
        rollout<M>(c, o.newton_steps);
        for (int e = c.tid; e < T * NG; e += c.nth) { c.xib[e] = 0.f; c.ygb[e] = 0.f; }
        for (int e = c.tid; e < T * NX; e += c.nth) c.yfb[e] = 0.f;
        c.sync();
    }
    float rho = o.rho0, rp = 0.f, rd = 0.f, alpha_last = 1.f;
    int ls_hist[2] = {0, 0};   // line-search step codes, 4 bits per SQP iteration
    int admm_total = 0, nfact = 0, sqp_done = 0;
    for (int it = 0; it < o.max_sqp; ++it) {
        linearize<M>(c);
        if (it > 0 && o.early_exit) {
            if (kkt<M>(c, rs.red) <= o.eps_c) break;
        }
        if (c.scl) rescale<M>(c, false);
        ++nfact;
        if (!factor<M, P>(c, o, rho, c.tflags + 1)) note_factor_failure<M>(c, rs.red);
        for (int e = c.tid; e < T * N; e += c.nth) c.x[e] = 0.f;
        for (int e = c.tid; e < T * NX; e += c.nth) { c.yf[e] = c.yfb[e]; c.pf[e] = -c.cv[e]; }
        for (int e = c.tid; e < T * NG; e += c.nth) {
            c.yg[e] = c.ygb[e];
            c.zg[e] = 0.f;
            c.xi[e] = 0.f;
            c.pg[e] = 0.f;   // G x - z_g at x = 0, z_g = 0
        }
        c.sync();
        admm_rowvec<M>(c, rho);
        int k = 0;
        for (k = 1; k <= o.max_admm; ++k) {
            admm_iter<M, P>(c, rho, o.alpha, o.sigma);
            const bool cc = o.early_exit && (k % o.check_every == 0);
            const bool cr = (k % o.k_rho_iter == 0) && k < o.max_admm;
            if (cc || cr || k == o.max_admm) {
                const Res r = residuals<M>(c, rs.red);
                rp = r.r_prim;
                rd = r.r_dual;
                const bool conv = rp <= o.eps_abs + o.eps_rel * r.pn && rd <= o.eps_abs + o.eps_rel * r.dn;
                if (cc && conv) break;
                if (cr && rd > 0.f && !conv) {
                    const float ratio = (rp / fmaxf(r.pn, 1e-30f)) / fmaxf(rd / fmaxf(r.dn, 1e-30f), 1e-30f);
                    const float cand = fminf(fmaxf(rho * sqrtf(ratio), o.rho_min), o.rho_max);
                    if (fmaxf(cand / rho, rho / cand) > o.k_rho_ratio) {
                        ++nfact;
                        if (factor<M, P>(c, o, cand, c.tflags + 1)) {
                            rho = cand;
                            admm_rowvec<M>(c, rho);
                        } else {
                            ++nfact;
                            if (!factor<M, P>(c, o, rho, c.tflags + 1)) note_factor_failure<M>(c, rs.red);
                        }
                    }
                }
            }
        }
        admm_total += (k > o.max_admm) ? o.max_admm : k;
        if (c.scl) rescale<M>(c, true);
        float ys[1] = {0.f};
        for (int e = c.tid; e < T * NX; e += c.nth) ys[0] = fmaxf(ys[0], fin(c.yf[e]));
        for (int e = c.tid; e < T * NG; e += c.nth) ys[0] = fmaxf(ys[0], fin(c.yg[e]));
        team_max_k<M, 1>(c, ys, rs.red);
        const float a = linesearch<M, P>(c, o, rs, ys[0]);
        alpha_last = a;
        if (it < 12) ls_hist[it / 6] |= ls_code(a) << (4 * (it % 6));
        for (int e = c.tid; e < T * N; e += c.nth) c.zb[e] += a * c.x[e];
        for (int e = c.tid; e < T * NG; e += c.nth) {
            c.xib[e] += a * (c.xi[e] - c.xib[e]);
            c.ygb[e] += a * (c.yg[e] - c.ygb[e]);
        }
        for (int e = c.tid; e < T * NX; e += c.nth) c.yfb[e] += a * (c.yf[e] - c.yfb[e]);
        c.sync();
        ++sqp_done;
    }
    linearize<M>(c);
    const float kk = kkt<M>(c, rs.red);
    float bad[1] = {0.f};
    for (int e = c.tid; e < T * N; e += c.nth) bad[0] = fmaxf(bad[0], fin(c.zb[e]));
    team_max_k<M, 1>(c, bad, rs.red);
    // write the solution (padded layout, zeros beyond the horizon / model dims)
    float* z = out.z + inst * Ts * L.n;
    float* xo = out.xi + inst * Ts * L.ng;
    float* yfo = out.yf + inst * Ts * L.nx;
    float* ygo = out.yg + inst * Ts * L.ng;
    for (int e = c.tid; e < Ts * L.n; e += c.nth) {
        const int t = e / L.n, j = e % L.n;
        z[e] = (t < T && j < N) ? c.zb[t * N + j] : 0.f;
    }
    for (int e = c.tid; e < Ts * L.ng; e += c.nth) {
        const int t = e / L.ng, r = e % L.ng;
        const bool ok = t < T && r < NG;
        xo[e] = ok ? c.xib[t * NG + r] : 0.f;
        ygo[e] = ok ? c.ygb[t * NG + r] : 0.f;
    }
    for (int e = c.tid; e < Ts * L.nx; e += c.nth) {
        const int t = e / L.nx, k = e % L.nx;
        yfo[e] = (t < T && k < NX) ? c.yfb[t * NX + k] : 0.f;
    }
    if (c.tid == 0) {
        const int st = instance_status(c.tflags[0], bad[0] < kInf, kk, o.eps_c);
        if (out.status) out.status[inst] = st;
        if (out.stats) {
            float* s = out.stats + (long long)inst * TMPC_STATS;
            s[0] = (float)sqp_done; s[1] = (float)admm_total; s[2] = rp; s[3] = rd;
            s[4] = rho; s[5] = (float)nfact; s[6] = kk; s[7] = alpha_last;
            s[8] = (float)ls_hist[0]; s[9] = (float)ls_hist[1];
        }
    }
    c.sync();
}

// ---------------------------------------------------------------------------
// Algorithm 2 for one instance (same method as tmpc_backward.cuh, here on the
// team and arena of the shared-memory kernels; S_b is factored by the cyclic
// reduction of the forward).  Arena reuse: code -> zg, w -> wg, rhs -> qv,
// eta_x -> x, eta_f -> yf, eta_H -> yg, G eta_x -> xi, r2 -> pf, r3 -> pg.
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void backward_instance_team(Inst<M>& c, const KOpts& o, const Red& rs, const KLayout& L,
                                                       const KSol& sol, int inst, const float* dLdz_all,
                                                       const float* dLdxi_all, const KGrads& g, double* dws,
                                                       double* dsh, const DirectQueue& dq, bool finish) {
    using Tr = Traits<M>;
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NU = Inst<M>::NU, NG = Inst<M>::NG;
    const int T = c.T;
    const long long Ts = L.Nmax + 1;
    const float* dLdz = dLdz_all + inst * Ts * L.n;
    const float* dLdxi = dLdxi_all ? dLdxi_all + inst * Ts * L.ng : nullptr;
    float rb = o.bwd_rho;
    if (c.tid == 0) c.tflags[0] = o.force_fail == inst + 1;
    c.cache_params();
    // the solution is the point of the linearisation
    {
        const float* z = sol.z + inst * Ts * L.n;
        const float* xi = sol.xi + inst * Ts * L.ng;
        const float* yf = sol.yf + inst * Ts * L.nx;
        const float* yg = sol.yg + inst * Ts * L.ng;
        for (int e = c.tid; e < T * N; e += c.nth) c.zb[e] = z[(e / N) * L.n + e % N];
        for (int e = c.tid; e < T * NG; e += c.nth) {
            c.xib[e] = xi[(e / NG) * L.ng + e % NG];
            c.ygb[e] = yg[(e / NG) * L.ng + e % NG];
        }
        for (int e = c.tid; e < T * NX; e += c.nth) c.yfb[e] = yf[(e / NX) * L.nx + e % NX];
        c.sync();
    }
    linearize<M>(c);
    float* code = c.zg;
    float* gw = c.wg;
    float* bx = c.qv;
    float* ex = c.x;
    float* lam = c.yf;
    float* mu = c.yg;
    float* gz = c.xi;
    float* r2 = c.pf;
    float* r3 = c.pg;
    for (int e = c.tid; e < T * NG; e += c.nth) {
        const int t = e / NG, r = e % NG;
        // g + xi - lo = xi - glo and hi - g - xi = ghi - xi in the shifted bounds of the linearisation
        const float lo = c.lob(t, r), hi = c.hib(t, r), y = c.ygb[e], xv = c.xib[e], eg = o.eps_g;
        const float dlo = xv - c.glo[e], dhi = c.ghi[e] - xv;
        const bool lower = (lo > -kInf) && ((y < -eg) || (fabsf(y) < eg && dlo <= eg * fmaxf(1.f, fabsf(lo))));
        const bool upper = !lower && (hi < kInf) && ((y > eg) || (fabsf(y) < eg && dhi <= eg * fmaxf(1.f, fabsf(hi))));
        float cd = 0.f;
        if (lower || upper) {
            const float side = upper ? 1.f : -1.f;
            cd = (c.gam2(r) < kInf && fabsf(xv) > eg) ? 2.f * side : side;
            if (o.bwd_solver == 3 && fabsf(cd) < 1.5f) cd = 3.f * side;   // hard row absorbed as a penalty
        }
        code[e] = cd;
        gw[e] = (cd == 0.f) ? 0.f : (fabsf(cd) > 2.5f ? o.bwd_gamma : (fabsf(cd) > 1.5f ? c.gam2(r) : rb));
        mu[e] = 0.f;
    }
    for (int e = c.tid; e < T * NX; e += c.nth) lam[e] = 0.f;
    c.sync();
    for (int e = c.tid; e < T * N; e += c.nth) {
        const int t = e / N, j = e % N;
        float b = dLdz[t * L.n + j];
        if (dLdxi)
#pragma unroll
            for (int r = 0; r < NG; ++r) {
                const float cd = fabsf(code[t * NG + r]);
                if (cd > 1.5f && cd < 2.5f) b -= c.Gval(t, r, j) * dLdxi[t * L.ng + r];
            }
        bx[e] = b;
        ex[e] = 0.f;
    }
    c.sync();
    // backward solver: 0 hybrid (refinement, then the direct solve where it did not
    // converge), 1 refinement only, 2 direct only, 3 the reduced adjoint QP (hard active
    // rows as penalties, code +-3; refinement only); the exact Hessian needs the direct solve
    const bool direct_ok = dws != nullptr && (dq.flag != nullptr || dsh != nullptr);
    const bool direct_only = direct_ok && (o.bwd_solver == 2 || o.exact_hessian);
    if (finish) {
        // the sweeps of the direct solve ran in the warp kernel: read the adjoint
        direct_load<M>(c, dws, ex, lam, mu);
        c.sync();
    } else {
        bool need_direct = direct_only;
        if (!direct_only) {
            // S_b = H + sigma_b I + rho_b C'C + G' diag(w) G; FP32 safeguard: lower rho_b up to three times
            form_S<M>(c, o.bwd_sigma, rb, rb, gw);
            bool ok = cr_factor<M>(c, c.tflags + 1);
            for (int tries = 0; !ok && tries < 3; ++tries) {
                rb *= 0.1f;
                for (int e = c.tid; e < T * NG; e += c.nth)
                    if (code[e] != 0.f && fabsf(code[e]) < 1.5f) gw[e] = rb;
                c.sync();
                form_S<M>(c, o.bwd_sigma, rb, rb, gw);
                ok = cr_factor<M>(c, c.tflags + 1);
            }
            if (!ok && c.tid == 0) c.tflags[0] = 1;
            top_inverse<M>(c);
            // divergence guard (see tmpc_backward.cuh): growing steps lower rho_b and restart
            float d0 = 0.f, dprev = kInf, dprev2 = kInf;
            int restarts = 0;
            for (int it = 0; it < o.bwd_iters; ++it) {
                for (int e = c.tid; e < T * NG; e += c.nth) gz[e] = c.Gx(ex, e / NG, e % NG);
                c.sync();
                for (int e = c.tid; e < T * N; e += c.nth) {
                    const int t = e / N, j = e % N;
                    float sv = bx[e] - c.Pv(ex, t, j);
                    sv -= c.Ctv(t, j, [&](int row, int k) { return lam[row * NX + k]; });
#pragma unroll
                    for (int r = 0; r < NG; ++r) {
                        const float cd = code[t * NG + r];
                        if (fabsf(cd) > 1.5f) sv -= gw[t * NG + r] * c.Gval(t, r, j) * gz[t * NG + r];
                        else if (cd != 0.f) sv -= c.Gval(t, r, j) * mu[t * NG + r];
                    }
                    c.r[e] = sv;
                }
                for (int e = c.tid; e < T * NX; e += c.nth) r2[e] = -c.Cx(ex, e / NX, e % NX);
                for (int e = c.tid; e < T * NG; e += c.nth) {
                    const float cd = code[e];
                    r3[e] = (cd != 0.f && fabsf(cd) < 1.5f) ? -gz[e] : 0.f;
                }
                c.sync();
                for (int e = c.tid; e < T * N; e += c.nth) {
                    const int t = e / N, j = e % N;
                    float sv = c.Ctv(t, j, [&](int row, int k) { return r2[row * NX + k]; });
                    sv += c.Gtw(t, j, [&](int r) { return r3[t * NG + r]; });
                    c.r[e] += rb * sv;
                }
                c.sync();
                cr_solve<M>(c, c.r, c.dx);
                for (int e = c.tid; e < T * NX; e += c.nth) lam[e] += rb * (c.Cx(c.dx, e / NX, e % NX) - r2[e]);
                for (int e = c.tid; e < T * NG; e += c.nth) {
                    const float cd = code[e];
                    if (cd != 0.f && fabsf(cd) < 1.5f) mu[e] += rb * (c.Gx(c.dx, e / NG, e % NG) - r3[e]);
                }
                c.sync();
                float dm[1] = {0.f};
                for (int e = c.tid; e < T * N; e += c.nth) {
                    ex[e] += c.dx[e];
                    dm[0] = fmaxf(dm[0], fin(c.dx[e]));
                }
                team_max_k<M, 1>(c, dm, rs.red);
                if (it == 0) d0 = dm[0];
                const bool diverging = !(dm[0] < kInf) || (it >= 2 && dm[0] > 2.f * dprev && dm[0] > 1e-4f * d0);
                if (diverging && restarts < 3) {
                    ++restarts;
                    rb *= 0.1f;
                    for (int e = c.tid; e < T * NG; e += c.nth) {
                        if (code[e] != 0.f && fabsf(code[e]) < 1.5f) gw[e] = rb;
                        mu[e] = 0.f;
                    }
                    for (int e = c.tid; e < T * NX; e += c.nth) lam[e] = 0.f;
                    for (int e = c.tid; e < T * N; e += c.nth) ex[e] = 0.f;
                    c.sync();
                    form_S<M>(c, o.bwd_sigma, rb, rb, gw);
                    if (!cr_factor<M>(c, c.tflags + 1) && c.tid == 0) c.tflags[0] = 1;
                    top_inverse<M>(c);
                    d0 = 0.f;
                    dprev = kInf;
                    it = -1;
                    continue;
                }
                dprev2 = dprev;
                dprev = dm[0];
                c.sync();
            }
            // convergence of the refinement: the last step at the FP32 floor of the solution, or a
            // contraction whose geometric tail (last step q / (1 - q)) is below 1e-6 of it (the
            // multipliers converge more slowly than eta_x, so the bound is kept tight)
            float xm[1] = {0.f};
            for (int e = c.tid; e < T * N; e += c.nth) xm[0] = fmaxf(xm[0], fin(ex[e]));
            team_max_k<M, 1>(c, xm, rs.red);
            const float q = dprev / fmaxf(dprev2, 1e-30f);
            bool refined_ok = dprev <= 1e-6f * xm[0] || (q < 0.9f && dprev * q / (1.f - q) <= 1e-6f * xm[0]);
            refined_ok = refined_ok && restarts == 0 && xm[0] < kInf;
            need_direct = !refined_ok && direct_ok && o.bwd_solver == 0;
        }
        if (need_direct) {
            // direct FP64 block LDL' of the interleaved active-set KKT system (tmpc_direct.cuh):
            // the team fills the per-stage records, one warp runs the sweeps
            direct_store<M>(c, code, bx, dws, o.exact_hessian != 0);
            c.sync();
            if (dq.flag) {   // sweeps in the warp kernel, gradients in the finishing pass
                if (c.tid == 0) dq.flag[inst] = 1;
                return;
            }
            if (c.tid < 32) direct_sweep<M>(T, dws, dsh, o.exact_hessian != 0);
            c.sync();
            direct_load<M>(c, dws, ex, lam, mu);
            c.sync();
        }
    }
    for (int e = c.tid; e < T * NG; e += c.nth) gz[e] = c.Gx(ex, e / NG, e % NG);
    c.sync();
    // ---- vector-Jacobian product (Eq. loss_gradient) ----
    const long long b = inst;
    if (g.x0)
        for (int k = c.tid; k < L.nx; k += c.nth) g.x0[b * L.nx + k] = k < NX ? lam[k] : 0.f;
    for (int e = c.tid; e < Ts * L.n; e += c.nth) {
        const int t = e / L.n, j = e % L.n;
        const bool okk = t < T && j < N;
        const float et = okk ? ex[t * N + j] : 0.f;
        if (g.ref) g.ref[b * Ts * L.n + e] = okk ? c.Cw(t, j) * et : 0.f;
        if (g.lin) g.lin[b * Ts * L.n + e] = -et;
    }
    for (int e = c.tid; e < Ts * L.nx; e += c.nth) {
        const int t = e / L.nx, i = e % L.nx;
        const bool okk = t < T && i < NX;
        if (g.Qd) g.Qd[b * Ts * L.nx + e] = okk ? -ex[t * N + i] * (c.zb[t * N + i] - c.refv(t, i)) : 0.f;
    }
    for (int e = c.tid; e < Ts * L.nu; e += c.nth) {
        const int t = e / L.nu, k = e % L.nu;
        const bool okk = t < T && k < NU;
        const int j = NX + k;
        if (g.Rd) g.Rd[b * Ts * L.nu + e] = okk ? -ex[t * N + j] * (c.zb[t * N + j] - c.refv(t, j)) : 0.f;
    }
    for (int e = c.tid; e < Ts * L.ng; e += c.nth) {
        const int t = e / L.ng, r = e % L.ng;
        float glo = 0.f, ghi = 0.f;
        if (t < T && r < NG) {
            const int q = t * NG + r;
            const float cd = code[q];
            float eA = 0.f;
            if (fabsf(cd) > 2.5f) eA = gw[q] * gz[q];   // penalty row of the reduced adjoint QP
            else if (fabsf(cd) > 1.5f) eA = (dLdxi ? dLdxi[t * L.ng + r] : 0.f) + c.gam2(r) * gz[q];
            else if (cd != 0.f) eA = mu[q];
            if (cd > 0.f) ghi = eA;
            if (cd < 0.f) glo = eA;
        }
        if (g.lo) g.lo[b * Ts * L.ng + e] = glo;
        if (g.hi) g.hi[b * Ts * L.ng + e] = ghi;
    }
    if (g.Wd)
        for (int k = 0; k < L.nu; ++k) {
            double sw = 0.0;
            if (k < NU)
                for (int t = c.tid; t < c.Nh; t += c.nth) {
                    const int j = NX + k;
                    sw += (double)(ex[t * N + j] - ex[(t + 1) * N + j]) * (c.zb[t * N + j] - c.zb[(t + 1) * N + j]);
                }
            sw = team_sum_d<M>(c, sw, rs.redd);
            if (c.tid == 0) g.Wd[b * L.nu + k] = (float)(-sw);
        }
    if (g.g2 || g.g1)
        for (int r = 0; r < L.ng; ++r) {
            double s2 = 0.0, s1 = 0.0;
            if (r < NG)
                for (int t = c.tid; t < T; t += c.nth) {
                    const int q = t * NG + r;
                    if (fabsf(code[q]) > 1.5f && fabsf(code[q]) < 2.5f) {
                        const float exi = -gz[q];
                        const float xv = c.xib[q];
                        s2 += (double)xv * exi;
                        s1 += (double)(xv > 0.f ? 1.f : (xv < 0.f ? -1.f : 0.f)) * exi;
                    }
                }
            s2 = team_sum_d<M>(c, s2, rs.redd);
            s1 = team_sum_d<M>(c, s1, rs.redd);
            if (c.tid == 0) {
                if (g.g2) g.g2[b * L.ng + r] = (float)(-s2);
                if (g.g1) g.g1[b * L.ng + r] = (float)(-s1);
            }
        }
    if (c.tid == 0 && sol.status && c.tflags[0]) sol.status[inst] = TMPC_INST_NOT_PD;
    c.sync();
}

// instance i's parameter pointers and sizes
template <int M>
__device__ __forceinline__ void bind_instance(Inst<M>& c, const KLayout& L, const KParams& p, const float* x0, int i) {
    c.Nh = p.N[i];
    c.T = c.Nh + 1;
    c.lnx = L.nx; c.lnu = L.nu; c.ln = L.n; c.lng = L.ng;
    const long long Ts = L.Nmax + 1;
    c.x0 = x0 + (long long)i * L.nx;
    c.Qd = p.Qd + i * Ts * L.nx;
    c.Rd = p.Rd + i * Ts * L.nu;
    c.Wd = p.Wd ? p.Wd + (long long)i * L.nu : nullptr;
    c.ref = p.ref ? p.ref + i * Ts * L.n : nullptr;
    c.lin = p.lin ? p.lin + i * Ts * L.n : nullptr;
    c.lo = p.lo + i * Ts * L.ng;
    c.hi = p.hi + i * Ts * L.ng;
    c.g2 = p.g2 ? p.g2 + (long long)i * L.ng : nullptr;
    c.g1 = p.g1 ? p.g1 + (long long)i * L.ng : nullptr;
    c.dyn = p.dyn + (long long)i * L.n_dyn;
    c.track = p.track ? p.track + (long long)i * (L.n_track + 1) * 4 : nullptr;
    c.scl = p.scale ? p.scale + (long long)i * L.n : nullptr;
    c.nt = 0;
    if (M == MODEL_BICYCLE) {
        const float ntf = c.dyn[3];
        int nt = (ntf == ntf) ? (int)fminf(fmaxf(ntf + 0.5f, 1.f), (float)L.n_track) : 1;
        c.nt = nt < 1 ? 1 : nt;
    }
}

// Persistent kernel over the instances listed in `order` (all of model M); an
// instance whose arena does not fit `smem_floats` uses its global slot.  The
// team of an instance is the CTA.  Compiled for four resident CTAs of 256
// threads per SM (64 registers a thread): with global arenas the residency is
// register-bound, and four CTAs ran the uneven batch 14 % faster than two (three:
// 10 %); shared-memory arenas stay limited by their size.
template <int M, int P>
__global__ void __launch_bounds__(256, 4) solve_kernel(KLayout L, KOpts o, KParams p, KSol out, float* gws,
                                                    long long gstride, const int* order, int count,
                                                    int* queue, const float* x0, int warm,
                                                    long long smem_floats) {
    extern __shared__ __align__(16) float arena[];
    __shared__ float red[32 * 8];
    __shared__ double redd[64];
    __shared__ double lsacc[2 * (kMaxLs + 1) + 2];
    __shared__ int flags[4];
    __shared__ int s_item;
    const Red rs{red, redd, lsacc, flags};
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_item;
        __syncthreads();
        if (q >= count) break;
        const int i = order[q];
        Inst<M> c;
        bind_instance<M>(c, L, p, x0, i);
        c.tid = threadIdx.x;
        c.nth = blockDim.x;
        c.cl = 1;
        c.rank = 0;
        c.tflags = flags;
        const long long need = arena_floats<M>(c.T, P);
        c.carve(need <= smem_floats ? arena : gws + (long long)i * gstride, P);
        solve_instance<M, P>(c, o, rs, L, out, i, warm);
    }
}

// Cluster variant for long horizons on few instances: the team of an instance
// is a thread-block cluster of `cl` CTAs (launched with that cluster size),
// working on the instance's global-memory arena; cluster k takes the
// instances order[k], order[k + clusters], ... so that every CTA of a cluster
// follows the same control flow.  Team flags live in the instance's slot.
template <int M, int P>
__global__ void __launch_bounds__(256, 2) solve_kernel_cluster(KLayout L, KOpts o, KParams p, KSol out, float* gws,
                                                            long long gstride, const int* order, int count,
                                                            const float* x0, int warm, int* gflags) {
    __shared__ float red[32 * 8];
    __shared__ double redd[64];
    __shared__ double lsacc[2 * (kMaxLs + 1) + 2];
    __shared__ int flags[4];
    const Red rs{red, redd, lsacc, flags};
    unsigned rank, ncta, cid, ncl;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(ncl));
    for (int q = (int)cid; q < count; q += (int)ncl) {
        const int i = order[q];
        Inst<M> c;
        bind_instance<M>(c, L, p, x0, i);
        c.tid = (int)rank * blockDim.x + threadIdx.x;
        c.nth = (int)ncta * blockDim.x;
        c.cl = (int)ncta;
        c.rank = (int)rank;
        c.tflags = gflags + 4LL * i;
        c.carve(gws + (long long)i * gstride, P, 1);
        solve_instance<M, P>(c, o, rs, L, out, i, warm);
        c.sync();   // the next instance reuses nothing of this one, but keep the CTAs in step
    }
}

// Backward kernels (Algorithm 2) of the shared-memory path: persistent CTA
// teams over a work queue, and one thread-block cluster per instance.
// finish = 0: every instance of `order`; the ones that need the direct solve are
// flagged in dq.flag after their records are filled (dq.flag may be null: no
// direct solve).  finish = 1: the flagged instances, whose adjoint the sweep
// kernel left in the records, take their gradients.
template <int M>
__global__ void __launch_bounds__(256, 2) backward_kernel(KLayout L, KOpts o, KParams p, KSol sol, float* gws,
                                                       long long gstride, const int* order, int count,
                                                       int* queue, const float* x0, long long smem_floats,
                                                       const float* dLdz, const float* dLdxi, KGrads g,
                                                       double* dws, long long dstride, DirectQueue dq, int finish) {
    extern __shared__ __align__(16) float arena[];
    __shared__ float red[32 * 8];
    __shared__ double redd[64];
    __shared__ double lsacc[2 * (kMaxLs + 1) + 2];
    __shared__ int flags[4];
    __shared__ int s_item;
    const Red rs{red, redd, lsacc, flags};
    for (;;) {
        if (threadIdx.x == 0) {
            int k;
            do {
                k = atomicAdd(queue, 1);
            } while (finish && k < count && !dq.flag[order[k]]);
            s_item = k;
        }
        __syncthreads();
        const int q = s_item;
        __syncthreads();
        if (q >= count) break;
        const int i = order[q];
        Inst<M> c;
        bind_instance<M>(c, L, p, x0, i);
        c.tid = threadIdx.x;
        c.nth = blockDim.x;
        c.cl = 1;
        c.rank = 0;
        c.tflags = flags;
        const long long need = arena_floats<M>(c.T, kCR);
        c.carve(need <= smem_floats ? arena : gws + (long long)i * gstride, kCR);
        backward_instance_team<M>(c, o, rs, L, sol, i, dLdz, dLdxi, g, dws ? dws + (long long)i * dstride : nullptr,
                                  nullptr, dq, finish != 0);
    }
}

template <int M>
__global__ void __launch_bounds__(256, 2) backward_kernel_cluster(KLayout L, KOpts o, KParams p, KSol sol, float* gws,
                                                               long long gstride, const int* order, int count,
                                                               const float* x0, int* gflags, const float* dLdz,
                                                               const float* dLdxi, KGrads g, double* dws,
                                                               long long dstride) {
    __shared__ __align__(16) double dsh[kDirectScratch];
    __shared__ float red[32 * 8];
    __shared__ double redd[64];
    __shared__ double lsacc[2 * (kMaxLs + 1) + 2];
    __shared__ int flags[4];
    const Red rs{red, redd, lsacc, flags};
    unsigned rank, ncta, cid, ncl;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(ncl));
    for (int q = (int)cid; q < count; q += (int)ncl) {
        const int i = order[q];
        Inst<M> c;
        bind_instance<M>(c, L, p, x0, i);
        c.tid = (int)rank * blockDim.x + threadIdx.x;
        c.nth = (int)ncta * blockDim.x;
        c.cl = (int)ncta;
        c.rank = (int)rank;
        c.tflags = gflags + 4LL * i;
        c.carve(gws + (long long)i * gstride, kCR, 1);
        backward_instance_team<M>(c, o, rs, L, sol, i, dLdz, dLdxi, g, dws ? dws + (long long)i * dstride : nullptr,
                                  dsh, DirectQueue{nullptr}, false);
        c.sync();
    }
}

// ---------------------------------------------------------------------------
// Plain per-phase form (a measurement baseline, solver 7): the same device
// code as solve_instance, cut into one launch per phase (initial guess, SQP
// step start, each ADMM iteration, SQP step end, final) with one CTA per
// instance, the state in the instance's global arena and PlainState, and the
// loop on the host.  Fixed iteration counts (early exit is not supported).
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ bool plain_bind(Inst<M>& c, const KLayout& L, const KParams& p, float* gws, long long gstride,
                                           const int* order, int count, const float* x0, PlainState* ps, int& i) {
    if ((int)blockIdx.x >= count) return false;
    i = order[blockIdx.x];
    bind_instance<M>(c, L, p, x0, i);
    c.tid = threadIdx.x;
    c.nth = blockDim.x;
    c.cl = 1;
    c.rank = 0;
    c.tflags = ps[i].flags;
    c.carve(gws + (long long)i * gstride, kCR);
    return true;
}

template <int M>
__global__ void __launch_bounds__(256, 2) plain_init(KLayout L, KOpts o, KParams p, KSol out, float* gws, long long gstride,
                                                  const int* order, int count, const float* x0, int warm, PlainState* ps) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    Inst<M> c;
    int i;
    if (!plain_bind<M>(c, L, p, gws, gstride, order, count, x0, ps, i)) return;
    const int T = c.T;
    if (c.tid == 0) {
        c.tflags[0] = o.force_fail == i + 1;
        PlainState& st = ps[i];
        st.rho = o.rho0; st.rp = 0.f; st.rd = 0.f; st.alpha_last = 1.f;
        st.admm_total = 0; st.nfact = 0; st.sqp_done = 0; st.ls_hist[0] = 0; st.ls_hist[1] = 0;
    }
    c.cache_params();
    const long long Ts = L.Nmax + 1;
    if (warm) {
        const float* z = out.z + i * Ts * L.n;
        const float* xi = out.xi + i * Ts * L.ng;
        const float* yf = out.yf + i * Ts * L.nx;
        const float* yg = out.yg + i * Ts * L.ng;
        for (int e = c.tid; e < T * N; e += c.nth) c.zb[e] = z[(e / N) * L.n + e % N];
        for (int e = c.tid; e < T * NG; e += c.nth) {
            c.xib[e] = xi[(e / NG) * L.ng + e % NG];
            c.ygb[e] = yg[(e / NG) * L.ng + e % NG];
        }
        for (int e = c.tid; e < T * NX; e += c.nth) c.yfb[e] = yf[(e / NX) * L.nx + e % NX];
        c.sync();
    } else {
        rollout<M>(c, o.newton_steps);
        for (int e = c.tid; e < T * NG; e += c.nth) { c.xib[e] = 0.f; c.ygb[e] = 0.f; }
        for (int e = c.tid; e < T * NX; e += c.nth) c.yfb[e] = 0.f;
        c.sync();
    }
}

template <int M>
__global__ void __launch_bounds__(256, 2) plain_sqp_begin(KLayout L, KOpts o, KParams p, float* gws, long long gstride,
                                                       const int* order, int count, const float* x0, PlainState* ps) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    Inst<M> c;
    int i;
    if (!plain_bind<M>(c, L, p, gws, gstride, order, count, x0, ps, i)) return;
    __shared__ float red[32 * 8];
    const int T = c.T;
    const float rho = ps[i].rho;
    linearize<M>(c);
    if (c.scl) rescale<M>(c, false);
    if (!factor<M, kCR>(c, o, rho, c.tflags + 1)) note_factor_failure<M>(c, red);
    for (int e = c.tid; e < T * N; e += c.nth) c.x[e] = 0.f;
    for (int e = c.tid; e < T * NX; e += c.nth) { c.yf[e] = c.yfb[e]; c.pf[e] = -c.cv[e]; }
    for (int e = c.tid; e < T * NG; e += c.nth) {
        c.yg[e] = c.ygb[e];
        c.zg[e] = 0.f;
        c.xi[e] = 0.f;
        c.pg[e] = 0.f;
    }
    c.sync();
    admm_rowvec<M>(c, rho);
    if (c.tid == 0) ps[i].nfact += 1;
}

template <int M>
__global__ void __launch_bounds__(256, 2) plain_admm(KLayout L, KOpts o, KParams p, float* gws, long long gstride,
                                                  const int* order, int count, const float* x0, PlainState* ps, int k) {
    Inst<M> c;
    int i;
    if (!plain_bind<M>(c, L, p, gws, gstride, order, count, x0, ps, i)) return;
    __shared__ float red[32 * 8];
    float rho = ps[i].rho;
    int nf = 0;
    admm_iter<M, kCR>(c, rho, o.alpha, o.sigma);
    const bool cr = (k % o.k_rho_iter == 0) && k < o.max_admm;
    if (cr || k == o.max_admm) {
        const Res r = residuals<M>(c, red);
        const float rp = r.r_prim, rd = r.r_dual;
        const bool conv = rp <= o.eps_abs + o.eps_rel * r.pn && rd <= o.eps_abs + o.eps_rel * r.dn;
        if (cr && rd > 0.f && !conv) {
            const float ratio = (rp / fmaxf(r.pn, 1e-30f)) / fmaxf(rd / fmaxf(r.dn, 1e-30f), 1e-30f);
            const float cand = fminf(fmaxf(rho * sqrtf(ratio), o.rho_min), o.rho_max);
            if (fmaxf(cand / rho, rho / cand) > o.k_rho_ratio) {
                ++nf;
                if (factor<M, kCR>(c, o, cand, c.tflags + 1)) {
                    rho = cand;
                    admm_rowvec<M>(c, rho);
                } else {
                    ++nf;
                    if (!factor<M, kCR>(c, o, rho, c.tflags + 1)) note_factor_failure<M>(c, red);
                }
            }
        }
        if (c.tid == 0) {
            ps[i].rp = rp;
            ps[i].rd = rd;
        }
    }
    if (c.tid == 0) {
        ps[i].rho = rho;
        ps[i].nfact += nf;
    }
}

template <int M>
__global__ void __launch_bounds__(256, 2) plain_sqp_end(KLayout L, KOpts o, KParams p, float* gws, long long gstride,
                                                     const int* order, int count, const float* x0, PlainState* ps, int it) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    Inst<M> c;
    int i;
    if (!plain_bind<M>(c, L, p, gws, gstride, order, count, x0, ps, i)) return;
    __shared__ float red[32 * 8];
    __shared__ double redd[64];
    __shared__ double lsacc[2 * (kMaxLs + 1) + 2];
    const Red rs{red, redd, lsacc, nullptr};
    const int T = c.T;
    if (c.scl) rescale<M>(c, true);
    float ys[1] = {0.f};
    for (int e = c.tid; e < T * NX; e += c.nth) ys[0] = fmaxf(ys[0], fin(c.yf[e]));
    for (int e = c.tid; e < T * NG; e += c.nth) ys[0] = fmaxf(ys[0], fin(c.yg[e]));
    team_max_k<M, 1>(c, ys, rs.red);
    const float a = linesearch<M, kCR>(c, o, rs, ys[0]);
    for (int e = c.tid; e < T * N; e += c.nth) c.zb[e] += a * c.x[e];
    for (int e = c.tid; e < T * NG; e += c.nth) {
        c.xib[e] += a * (c.xi[e] - c.xib[e]);
        c.ygb[e] += a * (c.yg[e] - c.ygb[e]);
    }
    for (int e = c.tid; e < T * NX; e += c.nth) c.yfb[e] += a * (c.yf[e] - c.yfb[e]);
    c.sync();
    if (c.tid == 0) {
        PlainState& st = ps[i];
        st.admm_total += o.max_admm;
        st.alpha_last = a;
        if (it < 12) st.ls_hist[it / 6] |= ls_code(a) << (4 * (it % 6));
        st.sqp_done += 1;
    }
}

template <int M>
__global__ void __launch_bounds__(256, 2) plain_final(KLayout L, KOpts o, KParams p, KSol out, float* gws,
                                                   long long gstride, const int* order, int count, const float* x0,
                                                   PlainState* ps) {
    constexpr int N = Inst<M>::N, NX = Inst<M>::NX, NG = Inst<M>::NG;
    Inst<M> c;
    int i;
    if (!plain_bind<M>(c, L, p, gws, gstride, order, count, x0, ps, i)) return;
    __shared__ float red[32 * 8];
    const int T = c.T;
    linearize<M>(c);
    const float kk = kkt<M>(c, red);
    float bad[1] = {0.f};
    for (int e = c.tid; e < T * N; e += c.nth) bad[0] = fmaxf(bad[0], fin(c.zb[e]));
    team_max_k<M, 1>(c, bad, red);
    const long long Ts = L.Nmax + 1;
    float* z = out.z + i * Ts * L.n;
    float* xo = out.xi + i * Ts * L.ng;
    float* yfo = out.yf + i * Ts * L.nx;
    float* ygo = out.yg + i * Ts * L.ng;
    for (int e = c.tid; e < Ts * L.n; e += c.nth) {
        const int t = e / L.n, j = e % L.n;
        z[e] = (t < T && j < N) ? c.zb[t * N + j] : 0.f;
    }
    for (int e = c.tid; e < Ts * L.ng; e += c.nth) {
        const int t = e / L.ng, r = e % L.ng;
        const bool ok = t < T && r < NG;
        xo[e] = ok ? c.xib[t * NG + r] : 0.f;
        ygo[e] = ok ? c.ygb[t * NG + r] : 0.f;
    }
    for (int e = c.tid; e < Ts * L.nx; e += c.nth) {
        const int t = e / L.nx, k = e % L.nx;
        yfo[e] = (t < T && k < NX) ? c.yfb[t * NX + k] : 0.f;
    }
    if (c.tid == 0) {
        const PlainState& st = ps[i];
        const int sts = instance_status(c.tflags[0], bad[0] < kInf, kk, o.eps_c);
        if (out.status) out.status[i] = sts;
        if (out.stats) {
            float* s = out.stats + (long long)i * TMPC_STATS;
            s[0] = (float)st.sqp_done; s[1] = (float)st.admm_total; s[2] = st.rp; s[3] = st.rd;
            s[4] = st.rho; s[5] = (float)st.nfact; s[6] = kk; s[7] = st.alpha_last;
            s[8] = (float)st.ls_hist[0]; s[9] = (float)st.ls_hist[1];
        }
    }
}

}  // namespace fast
}  // namespace tmpc
