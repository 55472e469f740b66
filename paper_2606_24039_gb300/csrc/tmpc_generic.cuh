// Generic SQP / ADMM kernels (any model, any stage size up to 72): shared
// memory layout, per-instance context and Algorithm 1 for one instance.  The
// two persistent kernels are defined in their own translation units
// (tmpc_generic_fwd.cu, tmpc_generic_bwd.cu) and launched by tmpc_api.cu.
#pragma once
#include <cuda_runtime.h>

#include "../../include/tmpc.h"
#include "tmpc_backward.cuh"
#include "tmpc_solver.cuh"

namespace tmpc {

// Shared memory of the generic kernels:
//   reduction scratch, mbarriers, flags
//   A, Bm       n^2 each: factorisation scratch (Delta / L^-1) and the two buffers
//               of the block stream of ldl_solve
//   red         8 x 96 floats: per-warp partial sums of ldl_solve
//   with L.vs:  the ADMM vectors (vs_floats), eta and xt first and together at
//               least n^2 floats, which the factorisation borrows as its third
//               scratch Cm (eta and xt are dead whenever S is factored)
//   else:       Cm, n^2 floats
__host__ __device__ inline long long vs_floats(const KLayout& L) {
    const long long T = L.Nmax + 1, n = L.n;
    const long long et = T * n > n * n - T * n ? T * n : n * n - T * n;
    return T * n + et + 2 * T * n + 2 * T * L.nx + 6 * T * L.ng;
}

__device__ __forceinline__ Smem carve_smem(void* raw, const KLayout& L) {
    const int n = L.n;
    Smem s;
    char* p = reinterpret_cast<char*>(raw);
    s.redd = reinterpret_cast<double*>(p);            p += 32 * 2 * sizeof(double);
    s.lsacc = reinterpret_cast<double*>(p);           p += (2 * (kMaxLs + 1) + 2) * sizeof(double);
    s.mbar = reinterpret_cast<unsigned long long*>(p); p += 2 * sizeof(unsigned long long);
    s.red = reinterpret_cast<float*>(p);              p += 32 * 8 * sizeof(float);
    s.flags = reinterpret_cast<int*>(p);              p += 16 * sizeof(int);
    s.A = reinterpret_cast<float*>(p);                p += n * n * sizeof(float);
    s.Bm = reinterpret_cast<float*>(p);               p += n * n * sizeof(float);
    s.red8 = reinterpret_cast<float*>(p);             p += 8 * 96 * sizeof(float);
    if (L.vs) {
        s.vs = reinterpret_cast<float*>(p);
        s.Cm = s.vs;
    } else {
        s.vs = nullptr;
        s.Cm = reinterpret_cast<float*>(p);
    }
    return s;
}

inline size_t smem_bytes(const KLayout& L) {
    const size_t n = L.n;
    const size_t fixed = 32 * 2 * sizeof(double) + (2 * (kMaxLs + 1) + 2) * sizeof(double) +
                         2 * sizeof(unsigned long long) + 32 * 8 * sizeof(float) + 16 * sizeof(int) +
                         2 * n * n * sizeof(float) + 8 * 96 * sizeof(float);
    return fixed + (L.vs ? (size_t)vs_floats(L) * sizeof(float) : n * n * sizeof(float));
}

__device__ inline Ctx make_ctx(const KLayout& L, const KParams& p, float* ws, const WsOff& off, int i,
                        const float* x0, float* vs) {
    Ctx c;
    c.model = p.model[i];
    const ModelDims md = model_dims(c.model, L.nx, L.nu, L.ng);
    c.nx = md.nx; c.nu = md.nu; c.ng = md.ng; c.n = md.nx + md.nu;
    c.N = p.N[i];
    c.T = c.N + 1;
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
    c.bv = (c.model == MODEL_LINEAR && L.n_dyn >= L.nx * L.nx + L.nx * L.nu + L.nx)
               ? c.dyn + L.nx * L.nx + L.nx * L.nu : nullptr;
    if (is_bicycle(c.model)) {  // table intervals, clamped to the layout's table size
        const float ntf = c.dyn[3];
        int nt = (ntf == ntf) ? (int)fminf(fmaxf(ntf + 0.5f, 1.f), (float)L.n_track) : 1;
        c.nt = nt < 1 ? 1 : nt;
    } else {
        c.nt = 0;
    }
    float* b = ws + (long long)i * off.stride;
    c.Am = b + off.Am; c.Ap = b + off.Ap; c.cv = b + off.cv; c.fv = b + off.fv; c.Gm = b + off.Gm;
    c.gv = b + off.gv; c.glo = b + off.glo; c.ghi = b + off.ghi; c.qv = b + off.qv;
    c.Dinv = b + off.Dinv; c.Om = b + off.Om; c.x = b + off.x; c.xt = b + off.xt; c.eta = b + off.eta;
    c.zg = b + off.zg; c.yg = b + off.yg; c.xi = b + off.xi; c.yf = b + off.yf; c.zb = b + off.zb;
    c.xib = b + off.xib; c.yfb = b + off.yfb; c.ygb = b + off.ygb; c.gw = b + off.gw;
    c.czb = b + off.czb; c.gzb = b + off.gzb; c.pf = b + off.pf; c.pg = b + off.pg;
    if (vs) {   // the ADMM vectors in shared memory (layout of vs_floats)
        const long long T = L.Nmax + 1, n = L.n;
        const long long et = T * n > n * n - T * n ? T * n : n * n - T * n;
        float* q = vs;
        c.eta = q; q += T * n;
        c.xt = q;  q += et;
        c.x = q;   q += T * n;
        c.qv = q;  q += T * n;
        c.yf = q;  q += T * L.nx;
        c.pf = q;  q += T * L.nx;
        c.zg = q;  q += T * L.ng;
        c.yg = q;  q += T * L.ng;
        c.xi = q;  q += T * L.ng;
        c.glo = q; q += T * L.ng;
        c.ghi = q; q += T * L.ng;
        c.pg = q;
    }
    c.amS = model_const_Am(c.model) ? 0 : c.nx * c.n;
    c.apS = model_const_Ap(c.model) ? 0 : c.nx * c.n;
    c.gS = model_const_G(c.model) ? 0 : c.ng * c.n;
    return c;
}

__device__ inline void write_solution(const Ctx& c, const KLayout& L, const KSol& out, int i) {
    const long long Ts = L.Nmax + 1;
    float* z = out.z + i * Ts * L.n;
    float* xi = out.xi + i * Ts * L.ng;
    float* yf = out.yf + i * Ts * L.nx;
    float* yg = out.yg + i * Ts * L.ng;
    for (int e = threadIdx.x; e < Ts * L.n; e += blockDim.x) {
        const int t = e / L.n, j = e % L.n;
        z[e] = (t < c.T && j < c.n) ? c.zb[t * c.n + j] : 0.f;
    }
    for (int e = threadIdx.x; e < Ts * L.ng; e += blockDim.x) {
        const int t = e / L.ng, r = e % L.ng;
        const bool ok = t < c.T && r < c.ng;
        xi[e] = ok ? c.xib[t * c.ng + r] : 0.f;
        yg[e] = ok ? c.ygb[t * c.ng + r] : 0.f;
    }
    for (int e = threadIdx.x; e < Ts * L.nx; e += blockDim.x) {
        const int t = e / L.nx, k = e % L.nx;
        yf[e] = (t < c.T && k < c.nx) ? c.yfb[t * c.nx + k] : 0.f;
    }
}

// A factorisation of S failed (uniform over the CTA): classify it by the data S
// is formed from.  A NaN in the stage Jacobians A^-_t, A^+_t, G_t or in the cost
// weights is a NaN event (bit 2 of sm.flags[0]); otherwise a pivot block of a
// finite S was not positive definite (bit 1).
__device__ inline void note_factor_failure(const Ctx& c, const Smem& sm) {
    float v[1] = {0.f};
    const int jac = c.nx * c.n;
    const int na = (c.amS ? c.N : 1) * jac, np = (c.apS ? c.N : 1) * jac, ngm = (c.gS ? c.T : 1) * c.ng * c.n;
    for (int e = threadIdx.x; e < na; e += blockDim.x) if (c.Am[e] != c.Am[e]) v[0] = 1.f;
    for (int e = threadIdx.x; e < np; e += blockDim.x) if (c.Ap[e] != c.Ap[e]) v[0] = 1.f;
    for (int e = threadIdx.x; e < ngm; e += blockDim.x) if (c.Gm[e] != c.Gm[e]) v[0] = 1.f;
    for (int e = threadIdx.x; e < c.T * c.n; e += blockDim.x) {
        const int t = e / c.n, j = e % c.n;
        const float w = j < c.nx ? c.Q(t, j) : c.R(t, j - c.nx);
        if (w != w) v[0] = 1.f;
    }
    cta_max_k<1>(v, sm.red);
    if (threadIdx.x == 0) sm.flags[0] |= v[0] > 0.f ? 2 : 1;
    __syncthreads();
}

__device__ inline void solve_instance(const Ctx& c, const KOpts& o, const Smem& sm, const KLayout& L,
                               const KSol& out, int inst, int warm) {
    const int n = c.n, nx = c.nx, ng = c.ng, T = c.T;
    // NOT_PD flag (set by a failed factorisation, or from the start for the instance a
    // caller forces to fail); a wait whose copy never landed (2) stays for the launch
    if (threadIdx.x == 0) { sm.flags[0] = o.force_fail == inst + 1; if (sm.flags[14] != 2) sm.flags[14] = 0; }
    if (warm) {
        read_warm(c, L, out, inst);
    } else {
        rollout(c, o);
        for (int e = threadIdx.x; e < T * ng; e += blockDim.x) { c.xib[e] = 0.f; c.ygb[e] = 0.f; }
        for (int e = threadIdx.x; e < T * nx; e += blockDim.x) c.yfb[e] = 0.f;
        __syncthreads();
    }
    float rho = o.rho0, rp = 0.f, rd = 0.f, alpha_last = 1.f;
    int ls_hist[2] = {0, 0};   // line-search step codes, 4 bits per SQP iteration
    int admm_total = 0, nfact = 0, sqp_done = 0;
    for (int it = 0; it < o.max_sqp; ++it) {
        linearize(c);
        if (it > 0 && o.early_exit) {
            const float kk = kkt(c, sm);
            if (kk <= o.eps_c) break;
        }
        ++nfact;
        if (!factor(c, sm, o.sigma, 1e3f * rho, rho, false)) note_factor_failure(c, sm);
        // warm start of the QP from the current primal-dual point (x = zb, z_g = G zb),
        // i.e. zero step, with the equality defect p_f = C x - c = -cv
        for (int e = threadIdx.x; e < T * n; e += blockDim.x) c.x[e] = 0.f;
        for (int e = threadIdx.x; e < T * nx; e += blockDim.x) {
            c.yf[e] = c.yfb[e];
            c.pf[e] = -c.cv[e];
        }
        for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
            c.yg[e] = c.ygb[e];
            c.zg[e] = 0.f;
            c.xi[e] = 0.f;
        }
        __syncthreads();
        int k = 0;
        for (k = 1; k <= o.max_admm; ++k) {
            admm_iter(c, o, rho, sm);
            const bool cc = o.early_exit && (k % o.check_every == 0);
            const bool cr = (k % o.k_rho_iter == 0) && k < o.max_admm;
            if (cc || cr || k == o.max_admm) {
                const Res r = residuals(c, sm);
                rp = r.r_prim;
                rd = r.r_dual;
                const bool conv = rp <= o.eps_abs + o.eps_rel * r.pn && rd <= o.eps_abs + o.eps_rel * r.dn;
                if (cc && conv) break;
                if (cr && rd > 0.f && !conv) {
                    const float ratio = (rp / fmaxf(r.pn, 1e-30f)) / fmaxf(rd / fmaxf(r.dn, 1e-30f), 1e-30f);
                    const float cand = fminf(fmaxf(rho * sqrtf(ratio), o.rho_min), o.rho_max);
                    if (fmaxf(cand / rho, rho / cand) > o.k_rho_ratio) {
                        // FP32 safeguard: a rho whose S cannot be factored is rejected
                        ++nfact;
                        if (factor(c, sm, o.sigma, 1e3f * cand, cand, false)) {
                            rho = cand;
                        } else {
                            ++nfact;
                            if (!factor(c, sm, o.sigma, 1e3f * rho, rho, false)) note_factor_failure(c, sm);
                        }
                    }
                }
            }
        }
        admm_total += (k > o.max_admm) ? o.max_admm : k;
        // line search on the direction (x* - zb, xi* - xib)
        float ys[1] = {0.f};
        for (int e = threadIdx.x; e < T * nx; e += blockDim.x) ys[0] = fmaxf(ys[0], fin(c.yf[e]));
        for (int e = threadIdx.x; e < T * ng; e += blockDim.x) ys[0] = fmaxf(ys[0], fin(c.yg[e]));
        cta_max_k<1>(ys, sm.red);
        const float a = linesearch(c, o, sm, ys[0]);
        alpha_last = a;
        if (it < 12) ls_hist[it / 6] |= ls_code(a) << (4 * (it % 6));
        for (int e = threadIdx.x; e < T * n; e += blockDim.x) c.zb[e] += a * c.x[e];
        for (int e = threadIdx.x; e < T * ng; e += blockDim.x) {
            c.xib[e] += a * (c.xi[e] - c.xib[e]);
            c.ygb[e] += a * (c.yg[e] - c.ygb[e]);
        }
        for (int e = threadIdx.x; e < T * nx; e += blockDim.x) c.yfb[e] += a * (c.yf[e] - c.yfb[e]);
        __syncthreads();
        ++sqp_done;
    }
    linearize(c);
    const float kk = kkt(c, sm);
    float bad[1] = {0.f};
    for (int e = threadIdx.x; e < T * n; e += blockDim.x) bad[0] = fmaxf(bad[0], fin(c.zb[e]));
    cta_max_k<1>(bad, sm.red);
    write_solution(c, L, out, inst);
    if (threadIdx.x == 0) {
        int st = TMPC_INST_OK;
        // root cause first: a wait that gave up, NaN met by a factorisation, a pivot block
        // that was not positive definite, then NaN in the result
        if (sm.flags[14]) st = TMPC_INST_TIMEOUT;
        else if (sm.flags[0] & 2) st = TMPC_INST_NAN;
        else if (sm.flags[0] & 1) st = TMPC_INST_NOT_PD;
        else if (!(bad[0] < kInf) || !(kk < kInf)) st = TMPC_INST_NAN;
        else if (!(kk <= o.eps_c)) st = TMPC_INST_MAX_ITER;
        if (out.status) out.status[inst] = st;
        if (out.stats) {
            float* s = out.stats + (long long)inst * TMPC_STATS;
            s[0] = (float)sqp_done; s[1] = (float)admm_total; s[2] = rp; s[3] = rd;
            s[4] = rho; s[5] = (float)nfact; s[6] = kk; s[7] = alpha_last;
            s[8] = (float)ls_hist[0]; s[9] = (float)ls_hist[1];
        }
    }
    __syncthreads();
}

// Forward (Algorithm 1) and backward (Algorithm 2) persistent kernels over a work queue.
__global__ void __launch_bounds__(256, 2) solve_kernel(KLayout L, KOpts o, KParams p, KSol out, float* ws, WsOff off,
                             const int* order, int count, int* queue, const float* x0, int warm);
__global__ void __launch_bounds__(256, 2) backward_kernel(KLayout L, KOpts o, KParams p, KSol sol, float* ws, WsOff off,
                                const int* order, int count, int* queue, const float* x0, const float* dLdz,
                                const float* dLdxi, KGrads g, double* dws, long long dstride);

}  // namespace tmpc
