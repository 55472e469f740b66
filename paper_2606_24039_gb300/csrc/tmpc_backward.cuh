// Backward pass (Algorithm 2, Section III-D, Appendix E of the paper) for one
// instance per CTA.
//
//  1. active set from the dual sign and bound proximity (Appendix E); an
//     active softened row with |xi| > eps_g keeps its slack, an active row
//     held at xi = 0 is treated as hard;
//  2. the reduced active-set KKT system of Eq. (bwd:slack_reduced_system)
//        [H + gamma2 G_S'G_S   C'   G_H'] [eta_x]   [dL/dz - G_S' dL/dxi]
//        [C                    0    0   ] [eta_f] = [0                  ]
//        [G_H                  0    0   ] [eta_H]   [0                  ]
//     (C: initial-state and dynamics Jacobian rows, G_H hard active rows, G_S
//     soft active rows) is solved by iterative refinement preconditioned with
//     the regularised system [H_r + sigma_b I, B'; B, -I/rho_b], B = [C; G_H],
//     whose Schur complement
//        S_b = H + sigma_b I + rho_b C'C + G' diag(w) G,
//        w = rho_b (hard active), gamma2 (soft active), 0 (inactive),
//     is block tridiagonal and is factored by the same block LDL' routine as
//     the forward S.  Residuals use the unregularised operators, so the
//     iteration converges to the exact adjoint of the KKT system;
//  3. eta_xi = -G_S eta_x, eta_S = dL/dxi + gamma2 G_S eta_x (Eq. bwd:slack:eta_xi_yg);
//  4. vector-Jacobian product of Eq. (loss_gradient) into the gradient arrays.
// H is the cost Hessian (the Hessian approximation the paper's code supports).
#pragma once
#include "tmpc_direct_generic.cuh"
#include "tmpc_solver.cuh"

namespace tmpc {

struct KGrads {
    float *x0, *Qd, *Rd, *Wd, *ref, *lin, *lo, *hi, *g2, *g1;
};

// codes stored per inequality row: 0 inactive, 1/-1 hard active upper/lower,
// 2/-2 soft active upper/lower, 3/-3 hard active rows that bwd_solver 3 (the
// reduced adjoint QP of Appendix E) absorbs into the Hessian as penalties of
// weight bwd_gamma: they enter S_b and the residual like soft rows (weight in
// gw), carry no multiplier iteration, and report bwd_gamma G_A eta_x as eta_A
__device__ __forceinline__ float active_code(float y, float val, float lo, float hi, float xi,
                                             bool soft, float eg) {
    const bool lower = (lo > -kInf) && ((y < -eg) || (fabsf(y) < eg && val - lo <= eg * fmaxf(1.f, fabsf(lo))));
    const bool upper = !lower && (hi < kInf) &&
                       ((y > eg) || (fabsf(y) < eg && hi - val <= eg * fmaxf(1.f, fabsf(hi))));
    if (!lower && !upper) return 0.f;
    const float side = upper ? 1.f : -1.f;
    return (soft && fabsf(xi) > eg) ? 2.f * side : side;
}

__device__ inline void backward_instance(const Ctx& c, const KOpts& o, const Smem& sm, const KLayout& L,
                                  const KSol& sol, int inst, const float* dLdz_all,
                                  const float* dLdxi_all, const KGrads& g, double* dws, double* dsh) {
    const int n = c.n, nx = c.nx, ng = c.ng, T = c.T, N = c.N;
    const long long Ts = L.Nmax + 1;
    const float* dLdz = dLdz_all + inst * Ts * L.n;
    const float* dLdxi = dLdxi_all ? dLdxi_all + inst * Ts * L.ng : nullptr;
    float rb = o.bwd_rho;
    if (threadIdx.x == 0) { sm.flags[0] = o.force_fail == inst + 1; if (sm.flags[14] != 2) sm.flags[14] = 0; }
    read_warm(c, L, sol, inst);  // zb, xib, yfb, ygb <- solution
    linearize(c);                // Jacobians and g at the solution
    float* code = c.zg;   // active codes
    float* bx = c.qv;     // right-hand side of the reduced system
    float* ex = c.x;      // eta_x
    float* lam = c.yf;    // eta_f (multipliers of C)
    float* mu = c.yg;     // eta_H (hard active rows)
    float* gz = c.xi;     // G eta_x
    float* r2 = c.fv;     // -C eta_x
    float* r3 = c.glo;    // -G_H eta_x
    for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
        const int t = e / ng, r = e % ng;
        float cd = active_code(c.ygb[e], c.gv[e] + c.xib[e], c.lob(t, r), c.hib(t, r), c.xib[e],
                               c.gam2(r) < kInf, o.eps_g);
        if (o.bwd_solver == 3 && cd != 0.f && fabsf(cd) < 1.5f) cd *= 3.f;   // hard row absorbed as a penalty
        code[e] = cd;
        c.gw[e] = (cd == 0.f) ? 0.f : (fabsf(cd) > 2.5f ? o.bwd_gamma : (fabsf(cd) > 1.5f ? c.gam2(r) : rb));
        mu[e] = 0.f;
    }
    for (int e = threadIdx.x; e < T * nx; e += blockDim.x) lam[e] = 0.f;
    __syncthreads();
    for (int e = threadIdx.x; e < T * n; e += blockDim.x) {
        const int t = e / n, j = e % n;
        float b = dLdz[t * L.n + j];
        if (dLdxi) {
            const float* G = c.Gt(t);
            for (int r = 0; r < ng; ++r) {
                const float cd = fabsf(code[t * ng + r]);
                if (cd > 1.5f && cd < 2.5f) b -= G[r * n + j] * dLdxi[t * L.ng + r];
            }
        }
        bx[e] = b;
        ex[e] = 0.f;
    }
    __syncthreads();
    // backward solver: 0 hybrid (refinement, then the direct FP64 solve where it did not
    // converge), 1 refinement only, 2 direct only (where the interleaved block fits)
    const bool direct_ok = dws != nullptr && gen_direct_mb(nx, n, ng) <= kGenDirectMB;
    const bool direct_only = direct_ok && o.bwd_solver == 2;
    bool refined_ok = true;
    if (direct_only) {
        // one direct FP64 block LDL' of the interleaved active-set KKT system
        direct_adjoint_ctx(c, code, bx, ex, lam, mu, dws, dsh, sm.flags + 3);
    } else {
        // FP32 safeguard: if S_b cannot be factored, lower rho_b (at most three times)
        bool ok = factor(c, sm, o.bwd_sigma, rb, rb, true);
        for (int tries = 0; !ok && tries < 3; ++tries) {
            rb *= 0.1f;
            for (int e = threadIdx.x; e < T * ng; e += blockDim.x)
                if (code[e] != 0.f && fabsf(code[e]) < 1.5f) c.gw[e] = rb;
            __syncthreads();
            ok = factor(c, sm, o.bwd_sigma, rb, rb, true);
        }
        if (!ok && threadIdx.x == 0) sm.flags[0] = 1;
        // divergence guard: the refinement contracts in exact arithmetic; if the
        // steps grow (an FP32 factor of S_b too inaccurate for this rho_b), lower
        // rho_b tenfold, refactor and restart (at most three times)
        float d0 = 0.f, dprev = kInf, dprev2 = kInf;
        int restarts = 0;
        const bool tiled = tiled_linear(c);
        for (int it = 0; it < o.bwd_iters; ++it) {
            for (int e = threadIdx.x; e < T * ng; e += blockDim.x) gz[e] = Gx_entry(c, ex, e / ng, e % ng);
            if (tiled) {
                // the same sweep with the C and C' products as register tiles:
                // r2 = -C eta_x; eta = b - H_r eta_x - C'(lam - rho_b r2) - G_H' mu + rho_b G_H' r3
                c_tiled(c, ex, [&](int e, float v) { r2[e] = -v; });
                __syncthreads();
                for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
                    const float cd = code[e];
                    r3[e] = (cd != 0.f && fabsf(cd) < 1.5f) ? -gz[e] : 0.f;
                }
                for (int e = threadIdx.x; e < T * nx; e += blockDim.x) c.xt[e] = lam[e] - rb * r2[e];
                __syncthreads();
                ct_tiled(c, c.xt, [&](int t, int j, float ctw) {
                    float s = bx[t * n + j] - Px_entry(c, ex, t, j) - ctw;
                    const int r = g_row(c, j);   // selector rows of the linear model
                    if (r >= 0) {
                        const float cd = code[t * ng + r];
                        if (fabsf(cd) > 1.5f) s -= c.gw[t * ng + r] * gz[t * ng + r];
                        else if (cd != 0.f) s -= mu[t * ng + r];
                        s += rb * r3[t * ng + r];
                    }
                    c.eta[t * n + j] = s;
                });
                __syncthreads();
                ldl_solve(c, c.eta, c.xt, sm.red8, sm.A, sm.Bm, sm.mbar, sm.flags + 12);  // dx
                c_tiled(c, c.xt, [&](int e, float v) { lam[e] += rb * (v - r2[e]); });
                for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
                    const float cd = code[e];
                    if (cd != 0.f && fabsf(cd) < 1.5f) mu[e] += rb * (Gx_entry(c, c.xt, e / ng, e % ng) - r3[e]);
                }
                __syncthreads();
            } else {
            __syncthreads();
            // r1 = b - H_r eta_x - C' lam - G_H' mu   (into eta), r2 = -C eta_x, r3 = -G_H eta_x
            for (int e = threadIdx.x; e < T * n; e += blockDim.x) {
                const int t = e / n, j = e % n;
                float s = bx[e] - Px_entry(c, ex, t, j);
                s -= Ct_entry(c, t, j, [&](int r, int k) { return lam[r * nx + k]; });
                if (g_is_selector(c)) {
                    const int r = g_row(c, j);
                    const float cd = r >= 0 ? code[t * ng + r] : 0.f;
                    if (fabsf(cd) > 1.5f) s -= c.gw[t * ng + r] * gz[t * ng + r];
                    else if (cd != 0.f) s -= mu[t * ng + r];
                } else {
                    const float* G = c.Gt(t);
                    for (int r = 0; r < ng; ++r) {
                        const float cd = code[t * ng + r];
                        if (fabsf(cd) > 1.5f) s -= c.gw[t * ng + r] * G[r * n + j] * gz[t * ng + r];
                        else if (cd != 0.f) s -= G[r * n + j] * mu[t * ng + r];
                    }
                }
                c.eta[e] = s;
            }
            for (int e = threadIdx.x; e < T * nx; e += blockDim.x) r2[e] = -Cx_entry(c, ex, e / nx, e % nx);
            for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
                const float cd = code[e];
                r3[e] = (cd != 0.f && fabsf(cd) < 1.5f) ? -gz[e] : 0.f;
            }
            __syncthreads();
            // rhs of the Schur system: r1 + rho_b (C' r2 + G_H' r3)
            for (int e = threadIdx.x; e < T * n; e += blockDim.x) {
                const int t = e / n, j = e % n;
                float s = Ct_entry(c, t, j, [&](int r, int k) { return r2[r * nx + k]; });
                if (g_is_selector(c)) {
                    const int r = g_row(c, j);
                    if (r >= 0) s += r3[t * ng + r];
                } else {
                    const float* G = c.Gt(t);
                    for (int r = 0; r < ng; ++r) s += G[r * n + j] * r3[t * ng + r];
                }
                c.eta[e] += rb * s;
            }
            __syncthreads();
            ldl_solve(c, c.eta, c.xt, sm.red8, sm.A, sm.Bm, sm.mbar, sm.flags + 12);  // dx
            for (int e = threadIdx.x; e < T * nx; e += blockDim.x)
                lam[e] += rb * (Cx_entry(c, c.xt, e / nx, e % nx) - r2[e]);
            for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
                const float cd = code[e];
                if (cd != 0.f && fabsf(cd) < 1.5f) mu[e] += rb * (Gx_entry(c, c.xt, e / ng, e % ng) - r3[e]);
            }
            __syncthreads();
            }
            float dm[1] = {0.f};
            for (int e = threadIdx.x; e < T * n; e += blockDim.x) {
                ex[e] += c.xt[e];
                dm[0] = fmaxf(dm[0], fin(c.xt[e]));
            }
            cta_max_k<1>(dm, sm.red);
            if (it == 0) d0 = dm[0];
            const bool diverging = !(dm[0] < kInf) || (it >= 2 && dm[0] > 2.f * dprev && dm[0] > 1e-4f * d0);
            if (diverging && restarts < 3) {
                ++restarts;
                rb *= 0.1f;
                for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
                    if (code[e] != 0.f && fabsf(code[e]) < 1.5f) c.gw[e] = rb;
                    mu[e] = 0.f;
                }
                for (int e = threadIdx.x; e < T * nx; e += blockDim.x) lam[e] = 0.f;
                for (int e = threadIdx.x; e < T * n; e += blockDim.x) ex[e] = 0.f;
                __syncthreads();
                if (!factor(c, sm, o.bwd_sigma, rb, rb, true) && threadIdx.x == 0) sm.flags[0] = 1;
                d0 = 0.f;
                dprev = kInf;
                it = -1;
                continue;
            }
            dprev2 = dprev;
            dprev = dm[0];
            __syncthreads();
        }
        // convergence of the refinement (as on the small models' kernels)
        float xm[1] = {0.f};
        for (int e = threadIdx.x; e < T * n; e += blockDim.x) xm[0] = fmaxf(xm[0], fin(ex[e]));
        cta_max_k<1>(xm, sm.red);
        const float q = dprev / fmaxf(dprev2, 1e-30f);
        refined_ok = dprev <= 1e-6f * xm[0] || (q < 0.9f && dprev * q / (1.f - q) <= 1e-6f * xm[0]);
        refined_ok = refined_ok && restarts == 0 && xm[0] < kInf;
    }
    if (!direct_only && !refined_ok && direct_ok && o.bwd_solver == 0) {
        for (int e = threadIdx.x; e < T * ng; e += blockDim.x) mu[e] = 0.f;
        __syncthreads();
        direct_adjoint_ctx(c, code, bx, ex, lam, mu, dws, dsh, sm.flags + 3);
    }
    for (int e = threadIdx.x; e < T * ng; e += blockDim.x) gz[e] = Gx_entry(c, ex, e / ng, e % ng);
    __syncthreads();
    // ---- vector-Jacobian product ----
    const long long b = inst;
    if (g.x0)
        for (int k = threadIdx.x; k < L.nx; k += blockDim.x) g.x0[b * L.nx + k] = k < nx ? lam[k] : 0.f;
    for (int e = threadIdx.x; e < Ts * L.n; e += blockDim.x) {
        const int t = e / L.n, j = e % L.n;
        const bool ok = t < T && j < n;
        const float et = ok ? ex[t * n + j] : 0.f;
        const float d = ok ? c.zb[t * n + j] - c.refv(t, j) : 0.f;
        if (g.ref) g.ref[b * Ts * L.n + e] = ok ? c.Cw(t, j) * et : 0.f;
        if (g.lin) g.lin[b * Ts * L.n + e] = -et;
    }
    for (int e = threadIdx.x; e < Ts * L.nx; e += blockDim.x) {
        const int t = e / L.nx, i = e % L.nx;
        const bool ok = t < T && i < nx;
        if (g.Qd) g.Qd[b * Ts * L.nx + e] = ok ? -ex[t * n + i] * (c.zb[t * n + i] - c.refv(t, i)) : 0.f;
    }
    for (int e = threadIdx.x; e < Ts * L.nu; e += blockDim.x) {
        const int t = e / L.nu, k = e % L.nu;
        const bool ok = t < T && k < c.nu;
        const int j = nx + k;
        if (g.Rd) g.Rd[b * Ts * L.nu + e] = ok ? -ex[t * n + j] * (c.zb[t * n + j] - c.refv(t, j)) : 0.f;
    }
    for (int e = threadIdx.x; e < Ts * L.ng; e += blockDim.x) {
        const int t = e / L.ng, r = e % L.ng;
        float glo = 0.f, ghi = 0.f;
        if (t < T && r < ng) {
            const int q = t * ng + r;
            const float cd = code[q];
            float eA = 0.f;
            if (fabsf(cd) > 2.5f) eA = c.gw[q] * gz[q];   // penalty row of the reduced adjoint QP
            else if (fabsf(cd) > 1.5f) eA = (dLdxi ? dLdxi[t * L.ng + r] : 0.f) + c.gam2(r) * gz[q];
            else if (cd != 0.f) eA = mu[q];
            if (cd > 0.f) ghi = eA;
            if (cd < 0.f) glo = eA;
        }
        if (g.lo) g.lo[b * Ts * L.ng + e] = glo;
        if (g.hi) g.hi[b * Ts * L.ng + e] = ghi;
    }
    // per-instance sums: control-rate weights and slack weights
    if (g.Wd)
        for (int k = 0; k < L.nu; ++k) {
            double s = 0.0;
            if (k < c.nu)
                for (int t = threadIdx.x; t < N; t += blockDim.x) {
                    const int j = nx + k;
                    s += (double)(ex[t * n + j] - ex[(t + 1) * n + j]) * (c.zb[t * n + j] - c.zb[(t + 1) * n + j]);
                }
            s = cta_sum_d(s, sm.redd);
            if (threadIdx.x == 0) g.Wd[b * L.nu + k] = (float)(-s);
        }
    if (g.g2 || g.g1)
        for (int r = 0; r < L.ng; ++r) {
            double s2 = 0.0, s1 = 0.0;
            if (r < ng)
                for (int t = threadIdx.x; t < T; t += blockDim.x) {
                    const int q = t * ng + r;
                    if (fabsf(code[q]) > 1.5f && fabsf(code[q]) < 2.5f) {
                        const float exi = -gz[q];
                        const float xv = c.xib[q];
                        s2 += (double)xv * exi;
                        s1 += (double)(xv > 0.f ? 1.f : (xv < 0.f ? -1.f : 0.f)) * exi;
                    }
                }
            s2 = cta_sum_d(s2, sm.redd);
            s1 = cta_sum_d(s1, sm.redd);
            if (threadIdx.x == 0) {
                if (g.g2) g.g2[b * L.ng + r] = (float)(-s2);
                if (g.g1) g.g1[b * L.ng + r] = (float)(-s1);
            }
        }
    if (threadIdx.x == 0 && sol.status && sm.flags[0]) sol.status[inst] = 2;  // not positive definite
    if (threadIdx.x == 0 && sol.status && sm.flags[14]) sol.status[inst] = TMPC_INST_TIMEOUT;
    __syncthreads();
}

}  // namespace tmpc
