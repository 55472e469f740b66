// Shared-memory-resident SQP / ADMM path for the small models (double
// integrator, kinematic bicycle, planar quadrotor): compile-time stage sizes,
// one CTA per instance, every per-instance array in shared memory (or in the
// handle's global workspace when an instance is too long to fit), and the
// block-tridiagonal S = P + sigma I + rho_f C'C + rho_g G'G factored and solved
// by block cyclic reduction.
//
// Block cyclic reduction = block LDL' of S after the odd-even permutation of
// its stages: at level l the active stages are the multiples of s = 2^l; the
// odd ones (e) are eliminated against their active neighbours a = e - s and
// b = e + s,
//     Dinv_e = D_e^{-1},  Fa_e = S_ae Dinv_e,  Fb_e = S_be Dinv_e,
//     D_a -= Fa_e S_ea,   D_b -= Fb_e S_eb,    S_ab = -Fa_e S_eb,
// and the solve is r_a -= Fa_e r_e, r_b -= Fb_e r_e on the way down,
// x_e = Dinv_e r_e - Fa_e' x_a - Fb_e' x_b on the way up.  Its depth is
// log2(N+1) levels instead of the 2(N+1) dependent stage steps of the
// sequential factorisation, and it is the same factorisation (Cholesky of a
// permuted SPD matrix), so it is as stable.
//
// The arithmetic of every phase is the one of tmpc_solver.cuh (same
// step-coordinate ADMM with the tracked equality defect, same line search,
// same KKT test); only the data placement and the S factorisation differ.
#pragma once
#include "tmpc_solver.cuh"

namespace tmpc {
namespace fast {

// 128-bit shared/global load of 4 consecutive floats (16-byte aligned address)
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// ---------------------------------------------------------------------------
// model traits: compile-time sizes; inequality rows are either a selection of
// one stage variable (sel[r] >= 0) or a dense row (sel[r] = -1, at most one)
// ---------------------------------------------------------------------------
template <int M> struct Traits;
template <> struct Traits<MODEL_DI> {
    static constexpr int NX = 4, NU = 2, NG = 4, IMPLICIT = 0, LTI = 1, DENSE_ROW = -1;
    __device__ static constexpr int sel(int r) { return r == 0 ? 4 : r == 1 ? 5 : r == 2 ? 2 : 3; }
};
template <> struct Traits<MODEL_BICYCLE> {
    static constexpr int NX = 6, NU = 2, NG = 5, IMPLICIT = 1, LTI = 0, DENSE_ROW = 4;
    __device__ static constexpr int sel(int r) { return r == 0 ? 6 : r == 1 ? 7 : r == 2 ? 3 : r == 3 ? 4 : -1; }
};
template <> struct Traits<MODEL_QUAD> {
    static constexpr int NX = 6, NU = 2, NG = 2, IMPLICIT = 0, LTI = 0, DENSE_ROW = -1;
    __device__ static constexpr int sel(int r) { return r == 0 ? 6 : 7; }
};

// The cyclic reduction of S stops after top_level(T, B) levels, when at most
// B blocks survive; the reduced system on those blocks (dimension top_dim =
// survivors x N) is inverted once per factorisation and applied as a dense
// matrix in every solve.  B = kTopBlocks for a CTA team (the inverse sits in
// shared memory), kTopBlocksCluster for a cluster team (global memory; a
// larger top saves cluster-wide barrier phases).
constexpr int kTopBlocks = 8, kTopBlocksCluster = 64;
__host__ __device__ constexpr int top_level(int T, int B) {
    int L = 0;
    while (((T + (1 << L) - 1) >> L) > B) ++L;
    return L;
}
__host__ __device__ constexpr int top_blocks(int T, int B) {
    return (T + (1 << top_level(T, B)) - 1) >> top_level(T, B);
}

// Factorisation policies of S:
//   kCR  block cyclic reduction by the whole CTA (depth 2 log2 T, all stages in
//        parallel), top levels by the dense inverse of the reduced system
//   kLDL sequential block LDL' (Riccati-like sweep over the stages) by one warp;
//        half the factor storage, so more instances fit on an SM
constexpr int kCR = 0, kLDL = 1;
// largest team (CTAs of a cluster) and doubles exchanged per CTA in a team reduction
constexpr int kTeamMax = 16, kXchDoubles = 40;
// first entry of the per-variable scales d_j in the cached-weights area par (N <= 8 entries)
constexpr int kParScale = 16;

// Per-instance arena: one list (name, floats) drives both the layout (carve)
// and its size (arena_floats), so the two cannot disagree.
//   factors of S:       Dm, Um                    T x BS each (padded N x N blocks)
//                       kCR:  Dm = Dinv_e, Um = couplings, Fa, Fb (T x BS each),
//                             Xt = inverse of the reduced system, top_dim^2
//                             (top_dim = top_blocks(T, B) N, rounded to 4)
//                       kLDL: Dm = Dinv_t, Um = L_t, Wk = 2 scratch blocks
//   stage vectors:      x, r, dx, qv, zb, Pd      T x N   (kLDL: dx shares r)
//   inequality rows:    zg, yg, xi, glo, ghi, xib, ygb, pg   T x NG
//   equality rows:      yf, pf, cv, yfb, wf       T x NX  (wg: T x NG)
//   refinement (cluster teams): rs, rd T x N, rcx T x NX, rgx T x NG
//   cached weights:     par                       32 (W, gamma2, gamma1; from kParScale on the
//                                                 power-of-two scales of a rescaled instance)
//   Jacobians:          Am (A^- per stage, padded stride AMS; one block if LTI), Grow (dense G row)
// Every array up to rd has a multiple of 4 floats (N = 8), so rows of Am, Grow
// and the stage vectors (the solves' right-hand sides and results among them)
// start on 16-byte boundaries (128-bit loads).
#define TMPC_FAST_ARENA(X)                                                       \
    X(Dm, (long long)T * BS) X(Um, (long long)T * BS)                            \
    X(Fa, P == kCR ? (long long)T * BS : 0LL)                                     \
    X(Fb, P == kCR ? (long long)T * BS : 0LL)                                     \
    X(Xt, P == kCR ? (long long)TD * TD : 0LL)                                    \
    X(Wk, P == kLDL ? 2LL * BS : 0LL)                                             \
    X(Xc, CL ? 2LL * (kTeamMax * kXchDoubles + 64) : 0LL)                       \
    X(Am, (Traits<M>::LTI ? (long long)AMS : (long long)T * AMS))                \
    X(Grow, (Traits<M>::DENSE_ROW >= 0 ? (long long)T * N : 0LL))                \
    X(x, T * N) X(r, T * N) X(dx, P == kCR ? T * N : 0) X(qv, T * N)             \
    X(zb, T * N) X(Pd, T * N)                                                    \
    X(rs, CL ? T * N : 0) X(rd, CL ? T * N : 0)                                  \
    X(zg, T * NG) X(yg, T * NG) X(xi, T * NG) X(glo, T * NG) X(ghi, T * NG)      \
    X(xib, T * NG) X(ygb, T * NG) X(pg, T * NG)                                  \
    X(yf, T * NX) X(pf, T * NX) X(cv, T * NX) X(yfb, T * NX)                     \
    X(wf, T * NX) X(wg, T * NG)                                                  \
    X(rcx, CL ? T * NX : 0) X(rgx, CL ? T * NG : 0)                              \
    X(par, 32)

// CL: the arena of a cluster team (with the exchange area of its reductions)
template <int M>
__host__ __device__ constexpr long long arena_floats(int T, int P, int CL = 0) {
    constexpr int NX = Traits<M>::NX, N = Traits<M>::NX + Traits<M>::NU, NG = Traits<M>::NG;
    constexpr int BS = N * N + 4, AMS = NX * N + 8;
    const int TD = (top_blocks(T, CL ? kTopBlocksCluster : kTopBlocks) * N + 3) & ~3;
    long long total = 0;
#define TMPC_SIZE(name, cnt) total += (cnt);
    TMPC_FAST_ARENA(TMPC_SIZE)
#undef TMPC_SIZE
    return total;
}

template <int M>
struct Inst {
    using Tr = Traits<M>;
    static constexpr int NX = Tr::NX, NU = Tr::NU, N = NX + NU, NG = Tr::NG, NN = N * N;
    static constexpr int AMS = NX * N + 8;
    // factor blocks: stride NN + 4 floats (spreads the banks of neighbouring blocks) and,
    // for N = 8, the two 4-float halves of rows 4..7 swapped (conflict-free 128-bit row loads)
    static constexpr int BS = NN + 4;
    __device__ static constexpr int bx(int i, int j) { return i * N + (N == 8 ? (j ^ (i & 4)) : j); }
    int Nh, T, nt;
    int lnx, lnu, ln, lng;
    // the team of threads that works on the instance: one CTA (cl = 1) or the
    // cl CTAs of a thread-block cluster; tid / nth index the whole team
    int tid, nth, cl, rank;
    int* tflags;    // team-visible flags (shared memory for one CTA, global for a cluster)
    double* xch;    // exchange area of the team reductions (global, cluster teams only)
    const float *x0, *Qd, *Rd, *Wd, *ref, *lin, *lo, *hi, *g2, *g1, *dyn, *track;
    const float* scl;   // magnitudes of the instance's variables for the rescaled ADMM, or nullptr
    float *Dm, *Um, *Fa, *Fb, *Xt, *Wk, *Xc;
    int TD;     // leading dimension of Xt
    int topb;   // most blocks of the reduced top system (kTopBlocks or kTopBlocksCluster)
    float *x, *r, *dx, *qv, *zb, *Pd;
    float *zg, *yg, *xi, *glo, *ghi, *xib, *ygb, *pg;
    float *yf, *pf, *cv, *yfb;
    float *wf, *wg;  // right-hand-side row vectors y_f + rho_f p_f, y_g + rho_g p_g
    float *rs, *rd, *rcx, *rgx;   // one step of iterative refinement of each solve (cluster teams)
    float *Am, *Grow, *par;  // par: W[NU], gamma2[NG], gamma1[NG] cached in the arena

    // barrier of the team: the CTA barrier, or the cluster barrier with release /
    // acquire ordering of the global-memory arena
    __device__ __forceinline__ void sync() const {
        if (cl > 1) {
            asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        } else {
            __syncthreads();
        }
    }
    __device__ __forceinline__ void carve(float* p, int P, int CL = 0) {
        const int T = this->T;
        topb = CL ? kTopBlocksCluster : kTopBlocks;
        TD = (top_blocks(T, topb) * N + 3) & ~3;
#define TMPC_CARVE(name, cnt) name = p; p += (cnt);
        TMPC_FAST_ARENA(TMPC_CARVE)
#undef TMPC_CARVE
        if (P == kLDL) dx = r;   // the sweep solves in place
        xch = CL ? reinterpret_cast<double*>(Xc) : nullptr;
    }
    // copy the per-instance weights used in the inner loop into the arena, and the
    // scales of a rescaled instance: d_j = the largest power of two not above the
    // caller's magnitude (s = m 2^e, m in [0.5, 1): d = 2^(e-1)); 1 for an entry
    // that is not positive and finite
    __device__ void cache_params() {
        for (int k = tid; k < NU + 2 * NG; k += nth) {
            float v;
            if (k < NU) v = Wd ? Wd[k] : 0.f;
            else if (k < NU + NG) v = g2 ? g2[k - NU] : kInf;
            else v = g1 ? g1[k - NU - NG] : 0.f;
            par[k] = v;
        }
        if (scl)
            for (int j = tid; j < N; j += nth) {
                const float v = scl[j];
                int e = 0;
                frexpf(v, &e);
                par[kParScale + j] = (v > 0.f && v < kInf) ? ldexpf(1.f, e - 1) : 1.f;
            }
    }
    __device__ __forceinline__ const float* Amt(int t) const { return Tr::LTI ? Am : Am + t * AMS; }
    __device__ __forceinline__ float W(int k) const { return par[k]; }
    __device__ __forceinline__ float refv(int t, int j) const { return ref ? ref[t * ln + j] : 0.f; }
    __device__ __forceinline__ float linv(int t, int j) const { return lin ? lin[t * ln + j] : 0.f; }
    __device__ __forceinline__ float Cw(int t, int j) const { return j < NX ? Qd[t * lnx + j] : Rd[t * lnu + j - NX]; }
    __device__ __forceinline__ float gam2(int r) const { return par[NU + r]; }
    __device__ __forceinline__ float gam1(int r) const { return par[NU + NG + r]; }
    __device__ __forceinline__ float lob(int t, int r) const { return lo[t * lng + r]; }
    __device__ __forceinline__ float hib(int t, int r) const { return hi[t * lng + r]; }

    // A^+_t entry (k, j): implicit midpoint A^+ = [A^-_x - 2I, 0], explicit A^+ = [-I, 0]
    __device__ __forceinline__ float Ap(int t, int k, int j) const {
        if (j >= NX) return 0.f;
        if (Tr::IMPLICIT) return Amt(t)[k * N + j] - (k == j ? 2.f : 0.f);
        return k == j ? -1.f : 0.f;
    }
    // (G_t)_{r, j}
    __device__ __forceinline__ float Gval(int t, int r, int j) const {
        const int s = Tr::sel(r);
        if (s >= 0) return j == s ? 1.f : 0.f;
        return Grow[t * N + j];
    }
    // (G x)_t row r
    __device__ __forceinline__ float Gx(const float* v, int t, int r) const {
        const int s = Tr::sel(r);
        if (s >= 0) return v[t * N + s];
        const float* g = Grow + t * N;
        if constexpr (N == 8) {
            const float4 g0 = ld4(g), g1 = ld4(g + 4), v0 = ld4(v + t * N), v1 = ld4(v + t * N + 4);
            return (g0.x * v0.x + g0.y * v0.y) + (g0.z * v0.z + g0.w * v0.w) +
                   ((g1.x * v1.x + g1.y * v1.y) + (g1.z * v1.z + g1.w * v1.w));
        } else {
            float a = 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) a += g[j] * v[t * N + j];
            return a;
        }
    }
    // (G' w)_t entry j, w(r) functor
    template <class F>
    __device__ __forceinline__ float Gtw(int t, int j, F w) const {
        float a = 0.f;
#pragma unroll
        for (int r = 0; r < NG; ++r) {
            const int s = Tr::sel(r);
            if (s >= 0) { if (s == j) a += w(r); }
            else a += Grow[t * N + j] * w(r);
        }
        return a;
    }
    // (C v)_row entry k
    __device__ __forceinline__ float Cx(const float* v, int row, int k) const {
        if (row == 0) return v[k];
        const int t = row - 1;
        const float* A = Amt(t) + k * N;
        const float* a = v + t * N;
        const float* b = v + (t + 1) * N;
        if constexpr (N == 8) {
            const float4 A0 = ld4(A), A1 = ld4(A + 4), a0 = ld4(a), a1 = ld4(a + 4);
            float s = (A0.x * a0.x + A0.y * a0.y) + (A0.z * a0.z + A0.w * a0.w) +
                      ((A1.x * a1.x + A1.y * a1.y) + (A1.z * a1.z + A1.w * a1.w));
            if (Tr::IMPLICIT) {
                static_assert(!Tr::IMPLICIT || NX == 6, "implicit model with NX = 6");
                const float4 b0 = ld4(b), b1 = ld4(b + 4);
                s += (A0.x * b0.x + A0.y * b0.y) + (A0.z * b0.z + A0.w * b0.w) + (A1.x * b1.x + A1.y * b1.y);
                s -= 2.f * b[k];
            } else {
                s -= b[k];
            }
            return s;
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) s += A[j] * a[j];
        if (Tr::IMPLICIT) {
#pragma unroll
            for (int j = 0; j < NX; ++j) s += A[j] * b[j];
            s -= 2.f * b[k];
        } else {
            s -= b[k];
        }
        return s;
    }
    // (C' v)_t entry j, v(row, k) functor
    template <class F>
    __device__ __forceinline__ float Ctv(int t, int j, F v) const {
        float s = 0.f;
        if (t == 0 && j < NX) s += v(0, j);
        if (t < Nh) {
            const float* A = Amt(t);
#pragma unroll
            for (int k = 0; k < NX; ++k) s += A[k * N + j] * v(t + 1, k);
        }
        if (t > 0 && j < NX) {
            if (Tr::IMPLICIT) {
                const float* A = Amt(t - 1);
#pragma unroll
                for (int k = 0; k < NX; ++k) s += A[k * N + j] * v(t, k);
                s -= 2.f * v(t, j);
            } else {
                s -= v(t, j);
            }
        }
        return s;
    }
    // (P v)_t entry j (cost Hessian: diagonal blocks Pd and the -W rate coupling)
    __device__ __forceinline__ float Pv(const float* v, int t, int j) const {
        float a = Pd[t * N + j] * v[t * N + j];
        if (j >= NX) {
            const float w = W(j - NX);
            if (t > 0) a -= w * v[(t - 1) * N + j];
            if (t < Nh) a -= w * v[(t + 1) * N + j];
        }
        return a;
    }
};

// ---------------------------------------------------------------------------
// entry (i, j) of a factor block (same swizzle as Inst::bx)
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ constexpr int blk(int i, int j) { return i * N + (N == 8 ? (j ^ (i & 4)) : j); }

}  // namespace fast
}  // namespace tmpc
