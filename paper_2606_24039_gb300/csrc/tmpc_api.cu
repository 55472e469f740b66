// C-ABI implementation (include/tmpc.h): handle, workspace, validation and the
// launches of the persistent kernels (generic: tmpc_generic_*.cu; small models:
// tmpc_fast*.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/tmpc.h"
#include "tmpc_fast_api.h"
#include "tmpc_generic.cuh"

using namespace tmpc;

namespace {

thread_local char g_last_error[256] = "";

void set_err(const char* what, cudaError_t e) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
}

#define TMPC_CUDA(call)                                  \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) {                         \
            set_err(#call, _e);                          \
            return TMPC_ERR_CUDA;                        \
        }                                                \
    } while (0)

KOpts to_kopts(const tmpc_options& o) {
    KOpts k;
    k.sigma = o.sigma; k.rho0 = o.rho0; k.rho_min = o.rho_min; k.rho_max = o.rho_max; k.alpha = o.alpha;
    k.eps_abs = o.eps_abs; k.eps_rel = o.eps_rel; k.eps_c = o.eps_c; k.eps_g = o.eps_g; k.ls_eta = o.ls_eta;
    k.k_rho_iter = o.k_rho_iter; k.k_rho_ratio = o.k_rho_ratio; k.max_sqp = o.max_sqp; k.max_admm = o.max_admm;
    k.n_ls = o.n_ls; k.newton_steps = o.newton_steps; k.early_exit = o.early_exit;
    k.check_every = o.check_every < 1 ? 1 : o.check_every;
    k.bwd_rho = o.bwd_rho; k.bwd_sigma = o.bwd_sigma; k.bwd_iters = o.bwd_iters;
    k.force_fail = o.force_pivot_failure;
    k.wait_polls = o.wait_polls;
    k.force_timeout = o.force_wait_timeout;
    k.bwd_solver = o.bwd_solver;
    k.exact_hessian = o.exact_hessian;
    k.bwd_gamma = o.bwd_gamma;
    if (k.k_rho_iter < 1) k.k_rho_iter = 1 << 30;
    return k;
}

KParams to_kparams(const tmpc_params& p) {
    KParams k;
    k.N = p.N; k.model = p.model; k.x0 = nullptr; k.Qd = p.Qd; k.Rd = p.Rd; k.Wd = p.Wd; k.ref = p.ref;
    k.lin = p.lin; k.lo = p.lo; k.hi = p.hi; k.g2 = p.gamma2; k.g1 = p.gamma1; k.dyn = p.dyn;
    k.track = p.track;
    k.scale = p.scale;
    return k;
}

long long align4(long long v) { return (v + 3) & ~3LL; }

// Per-instance workspace offsets (floats) of the generic kernels for a layout:
// the same list of arrays for the handle's workspace and the static scratch.
// Offsets are computed in 64-bit and returned false when one of them, or the
// stride, does not fit the int offsets of WsOff (the layout is then rejected).
bool ws_layout(const tmpc_dims& d, WsOff& off) {
    const long long n = (long long)d.nx + d.nu;
    const long long T = (long long)d.N_max + 1, Nm = std::max<long long>(d.N_max, 1);
    const long long nxn = (long long)d.nx * n, nn = n * n;
    long long cur = 0;
    bool fits = true;
    auto take = [&](long long cnt) {
        const long long at = align4(cur);
        cur = at + cnt;
        if (at > INT_MAX || cur > INT_MAX) fits = false;
        return fits ? (int)at : 0;
    };
    off.Am = take(Nm * nxn);
    off.Ap = take(Nm * nxn);
    off.cv = take(T * d.nx);
    off.fv = take(T * d.nx);
    off.Gm = take(T * d.ng * n);
    off.gv = take(T * d.ng);
    off.glo = take(T * d.ng);
    off.ghi = take(T * d.ng);
    off.qv = take(T * n);
    off.Dinv = take(T * nn);
    off.Om = take(Nm * nn);
    off.x = take(T * n);
    off.xt = take(T * n);
    off.eta = take(T * n);
    off.zg = take(T * d.ng);
    off.yg = take(T * d.ng);
    off.xi = take(T * d.ng);
    off.yf = take(T * d.nx);
    off.zb = take(T * n);
    off.xib = take(T * d.ng);
    off.yfb = take(T * d.nx);
    off.ygb = take(T * d.ng);
    off.gw = take(T * d.ng);
    off.czb = take(T * d.nx);
    off.gzb = take(T * d.ng);
    off.pf = take(T * d.nx);
    off.pg = take(T * d.ng);
    off.stride = align4(cur);
    return fits && off.stride <= INT_MAX;
}

// The generic kernels may be launched with any dynamic shared-memory size up to
// the device's opt-in maximum less their static shared memory; the attribute is a
// limit, not a reservation, so it is raised to that maximum and never lowered by a
// later, smaller launch.  A failed attribute call is cleared from the runtime's
// last error so that it cannot be reported by a later launch check.
cudaError_t allow_max_smem(int max_optin) {
    const void* kernels[2] = {(const void*)solve_kernel, (const void*)backward_kernel};
    for (const void* k : kernels) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     max_optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
    }
    return cudaSuccess;
}

}  // namespace

struct tmpc_handle {
    tmpc_dims d;
    tmpc_options o;
    tmpc_params p;
    KLayout L;
    WsOff off;
    float* ws = nullptr;
    int* order = nullptr;
    int* queue = nullptr;
    // work groups of the forward pass: g < 3 the shared-memory kernels of the
    // double integrator / bicycle / quadrotor, g = 3 the generic kernel
    struct Group {
        int model = -1, offset = 0, count = 0, grid = 0, threads = 0, policy = 0;
        int cluster = 0;   // > 0: CTAs per thread-block cluster (one cluster per instance)
        int bgrid = 0;     // > 0: the group's backward runs on the shared-memory path with this grid
        int plain = 0;     // 1: plain per-phase form (one launch per phase, solver 7)
        int form = 0;      // launch form, as the solver option codes 2..7 (0: generic kernel)
        int Tmax = 0;      // longest horizon + 1 in the group
        size_t smem = 0;
    } groups[4];
    std::vector<int> ord_host;          // forward instance order (groups back to back)
    std::vector<long long> work_host;   // (N+1) n^2 per instance, the longest-first key
    int max_optin = 0;
    int bwd_generic = 0;       // instances whose backward runs on the generic kernel
    int* gflags = nullptr;     // team flags of cluster-launched instances (4 per instance)
    fast::PlainState* pstate = nullptr;   // per-instance state of the plain per-phase form
    // several model groups run concurrently on internal streams (fork / join on the caller's stream)
    cudaStream_t gs[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[4] = {nullptr, nullptr, nullptr, nullptr};
    // device timing of the last launches, per forward group (slots 0..3) and the generic
    // backward (slot 4): [slot][0..1] forward start / stop, [slot][2..3] backward start / stop
    cudaEvent_t tev[5][4] = {};
    bool timed[5][2] = {};
    int n_groups = 0;
    float* fws = nullptr;      // global arenas of the shared-memory path (instances that do not fit)
    long long fstride = 0;
    double* dws = nullptr;     // FP64 workspace of the direct backward of the small models
    long long dstride = 0;
    int* dq = nullptr;         // direct-solve queues: 4 counters per group (20), then a flag per instance
    int nsm = 0;
    int threads = 128;
    size_t smem = 0;
    int grid_solve = 1, grid_bwd = 1;
    // staging for tmpc_solve_host
    void* stage = nullptr;
    size_t stage_bytes = 0;
    tmpc_params sp{};
    float* s_x0 = nullptr;
    tmpc_solution ss{};
};

// 1 if the generic kernels keep two CTAs per SM with the ADMM vectors in shared memory
int choose_vs(KLayout L, int threads, int max_optin) {
    L.vs = 1;
    const size_t bytes = smem_bytes(L);
    if ((long long)bytes > max_optin) return 0;
    if (allow_max_smem(max_optin) != cudaSuccess) return 0;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_kernel, threads, bytes) != cudaSuccess) return 0;
    return per >= 2 ? 1 : 0;
}

extern "C" {

void tmpc_default_options(tmpc_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->sigma = 1e-6f; o->rho0 = 0.1f; o->rho_min = 1e-6f; o->rho_max = 1e6f; o->alpha = 1.6f;
    o->eps_abs = 1e-5f; o->eps_rel = 1e-5f; o->eps_c = 1e-5f; o->eps_g = 1e-4f; o->ls_eta = 0.4f;
    o->k_rho_iter = 25; o->k_rho_ratio = 5.f; o->max_sqp = 1; o->max_admm = 200; o->n_ls = 8;
    o->newton_steps = 3; o->early_exit = 0; o->check_every = 25;
    o->bwd_rho = 1e4f; o->bwd_sigma = 1e-6f; o->bwd_iters = 30;
    o->bwd_solver = 2;
    o->bwd_gamma = 1e4f;
    o->threads = 0; o->solver = 0;
}

const char* tmpc_status_string(tmpc_status s) {
    switch (s) {
        case TMPC_OK: return "ok";
        case TMPC_ERR_INVALID_ARG: return "invalid argument";
        case TMPC_ERR_CUDA: return "CUDA error";
        case TMPC_ERR_OOM: return "out of device memory";
        case TMPC_ERR_NOT_SETUP: return "not set up";
        case TMPC_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* tmpc_last_error(void) { return g_last_error; }

static tmpc_status check_options(const tmpc_options* o) {
    if (!(o->sigma > 0.f) || !(o->rho0 > 0.f) || !(o->alpha > 0.f && o->alpha < 2.f)) return TMPC_ERR_INVALID_ARG;
    if (o->max_sqp < 0 || o->max_admm < 1 || o->n_ls < 1 || o->n_ls > kMaxLs) return TMPC_ERR_INVALID_ARG;
    if (o->newton_steps < 0 || o->bwd_iters < 1 || !(o->bwd_rho > 0.f)) return TMPC_ERR_INVALID_ARG;
    if (o->threads < 0 || o->threads > 256 || (o->threads % 32) != 0) return TMPC_ERR_INVALID_ARG;
    if (o->solver < 0 || o->solver > 7) return TMPC_ERR_INVALID_ARG;
    if (o->force_pivot_failure < 0 || o->wait_polls < 0) return TMPC_ERR_INVALID_ARG;
    if (o->bwd_solver < 0 || o->bwd_solver > 3) return TMPC_ERR_INVALID_ARG;
    if (o->bwd_solver == 3 && (o->exact_hessian || !(o->bwd_gamma > 0.f) || !(o->bwd_gamma < 1e30f)))
        return TMPC_ERR_INVALID_ARG;
    return TMPC_OK;
}

static bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

static tmpc_status check_params(const tmpc_dims& d, const tmpc_params* p) {
    if (!p || !p->N || !p->model || !p->Qd || !p->Rd || !p->lo || !p->hi || !p->dyn) return TMPC_ERR_INVALID_ARG;
    const void* ptrs[] = {p->N, p->model, p->Qd, p->Rd, p->Wd, p->ref, p->lin, p->lo, p->hi,
                          p->gamma2, p->gamma1, p->dyn, p->track, p->scale};
    for (const void* q : ptrs)
        if (q && !aligned4(q)) return TMPC_ERR_INVALID_ARG;
    if (d.n_track > 0 && !p->track) return TMPC_ERR_INVALID_ARG;
    return TMPC_OK;
}

// ---------------------------------------------------------------------------
// Launch forms of the model groups of the shared-memory kernels (the solver
// option codes): 2 cyclic reduction with the arena in shared memory where it
// fits, 3 the same with every arena in global memory, 4 / 5 the one-warp block
// LDL' in shared / global memory, 6 one thread-block cluster per instance,
// 7 the plain per-phase form.
// ---------------------------------------------------------------------------
namespace {

long long shared_cap(const tmpc_handle* h) {
    return std::max(48LL * 1024, (long long)h->max_optin / 2 - 8 * 1024);
}

long long arena_bytes(const tmpc_handle::Group& G, int policy) {
    return (long long)sizeof(float) * fast::arena_floats_host(G.model, G.Tmax, policy);
}

// the longest instance's cyclic-reduction arena fits with two CTAs per SM
bool shared_fits(const tmpc_handle* h, const tmpc_handle::Group& G) {
    return arena_bytes(G, fast::kPolicyCR) <= shared_cap(h);
}

// Sets the group's policy, CTA size, shared arena and grid for a form.
// cudaErrorNotSupported: no cluster size can be launched (form 6).
cudaError_t configure_group(tmpc_handle* h, tmpc_handle::Group& G, int form, int threads) {
    G.plain = 0;
    G.cluster = 0;
    G.bgrid = 0;
    G.form = form;
    G.policy = (form == 4 || form == 5) ? fast::kPolicyLDL : fast::kPolicyCR;
    G.threads = threads > 0 ? threads : (G.policy == fast::kPolicyLDL ? 128 : 256);
    // shared arena: the longest instance if it fits with 2 CTAs per SM, else a
    // third of the opt-in limit (longer instances use their global arena)
    const long long need = arena_bytes(G, G.policy), cap = shared_cap(h);
    G.smem = (size_t)std::min(need, need <= cap ? need : (long long)h->max_optin / 3);
    if (form == 3 || form == 5 || form == 7) G.smem = 0;
    if (form == 7) {   // one CTA per instance, one launch per phase
        G.plain = 1;
        G.grid = G.count;
        return cudaSuccess;
    }
    if (form == 6) {
        for (int cl = 16; cl >= 2 && G.cluster == 0; cl >>= 1) {
            int mc = 0;
            if (fast::prepare_cluster(G.model, G.policy, cl, G.threads, &mc) == cudaSuccess && mc >= 1) {
                G.cluster = cl;
                G.grid = std::min(G.count, mc);   // clusters
            }
        }
        cudaGetLastError();   // clear a refused cluster size
        return G.cluster > 0 ? cudaSuccess : cudaErrorNotSupported;
    }
    int per = 0;
    const cudaError_t e = fast::prepare(G.model, G.policy, G.smem, G.threads, &per);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    G.grid = std::max(1, std::min(G.count, per * h->nsm));
    return cudaSuccess;
}

// Global arenas (instances whose arena is not in shared memory), plain-form
// state and cluster team flags for the groups' current forms; grows, never shrinks.
tmpc_status ensure_buffers(tmpc_handle* h) {
    long long fmax = 0;
    bool any_plain = false, any_cluster = false;
    for (int g = 0; g < h->n_groups; ++g) {
        const tmpc_handle::Group& G = h->groups[g];
        if (G.model < 0) continue;
        fmax = std::max(fmax, fast::arena_floats_host(G.model, G.Tmax, G.policy));
        if (G.cluster > 0) fmax = std::max(fmax, fast::arena_floats_host(G.model, G.Tmax, G.policy, 1));
        any_plain = any_plain || G.plain;
        any_cluster = any_cluster || G.cluster > 0;
    }
    const long long B = h->d.batch;
    cudaError_t e;
    if (any_plain && !h->pstate) {
        e = cudaMalloc(&h->pstate, sizeof(fast::PlainState) * (size_t)B);
        if (e != cudaSuccess) { set_err("cudaMalloc(plain state)", e); return TMPC_ERR_OOM; }
    }
    if (any_cluster && !h->gflags) {
        e = cudaMalloc(&h->gflags, sizeof(int) * 4 * (size_t)B);
        if (e != cudaSuccess) { set_err("cudaMalloc(team flags)", e); return TMPC_ERR_OOM; }
    }
    // FP64 workspace of the direct backward: the small models' kernels and, where the
    // layout's interleaved KKT block fits, the generic kernel (every instance's slot)
    long long dneed = 0;
    for (int g = 0; g < h->n_groups; ++g)
        if (h->groups[g].model >= 0)
            dneed = std::max(dneed, fast::direct_ws_doubles(h->groups[g].model, h->groups[g].Tmax));
    if (dneed > 0 && !h->dq) {
        e = cudaMalloc(&h->dq, sizeof(int) * (20 + (size_t)B));
        if (e != cudaSuccess) { set_err("cudaMalloc(direct-solve queues)", e); return TMPC_ERR_OOM; }
    }
    const int mbg = gen_direct_mb(h->L.nx, h->L.n, h->L.ng);
    if (mbg <= kGenDirectMB) dneed = std::max(dneed, (long long)(h->L.Nmax + 1) * gen_direct_stage(mbg));
    if (dneed > 0 && dneed > h->dstride) {
        if (h->dws) cudaFree(h->dws);
        h->dws = nullptr;
        h->dstride = 0;
        e = cudaMalloc(&h->dws, sizeof(double) * dneed * B);
        if (e != cudaSuccess) { set_err("cudaMalloc(direct backward workspace)", e); return TMPC_ERR_OOM; }
        h->dstride = dneed;
    }
    const long long stride = (fmax + 31) & ~31LL;
    if (fmax > 0 && stride > h->fstride) {
        if (h->fws) cudaFree(h->fws);
        h->fws = nullptr;
        h->fstride = 0;
        e = cudaMalloc(&h->fws, sizeof(float) * stride * B);
        if (e != cudaSuccess) { set_err("cudaMalloc(fast arenas)", e); return TMPC_ERR_OOM; }
        h->fstride = stride;
    }
    return TMPC_OK;
}

// Backward plan: groups on the cyclic-reduction policy run the shared-memory
// backward over their forward order; every other instance (generic group,
// warp-LDL groups) the generic backward, longest first.  Writes the device
// order array (forward order, then the generic backward's).
tmpc_status plan_backward(tmpc_handle* h) {
    const int B = h->d.batch;
    std::vector<char> fastb(B, 0);
    for (int g = 0; g < h->n_groups; ++g) {
        tmpc_handle::Group& G = h->groups[g];
        G.bgrid = 0;
        if (G.model < 0 || G.policy != fast::kPolicyCR || h->o.solver == 1) continue;
        int per = 0;
        const cudaError_t e = fast::prepare_backward(G.model, G.cluster, G.smem, G.threads, &per);
        if (e != cudaSuccess || per < 1) { cudaGetLastError(); continue; }
        G.bgrid = G.cluster > 0 ? G.grid : std::max(1, std::min(G.count, per * h->nsm));
        for (int q = 0; q < G.count; ++q) fastb[h->ord_host[G.offset + q]] = 1;
    }
    std::vector<int> bord;
    for (int i = 0; i < B; ++i)
        if (!fastb[i]) bord.push_back(i);
    std::stable_sort(bord.begin(), bord.end(),
                     [&](int a, int b) { return h->work_host[a] > h->work_host[b]; });
    h->bwd_generic = (int)bord.size();
    bord.resize(B, 0);
    std::vector<int> ord(h->ord_host);
    ord.insert(ord.end(), bord.begin(), bord.end());
    const cudaError_t e = cudaMemcpy(h->order, ord.data(), sizeof(int) * ord.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { set_err("cudaMemcpy(order)", e); return TMPC_ERR_CUDA; }
    return TMPC_OK;
}

}  // namespace

tmpc_status tmpc_setup(tmpc_handle** hp, const tmpc_dims* d, const tmpc_options* o, const tmpc_params* p) {
    if (!hp) return TMPC_ERR_INVALID_ARG;
    *hp = nullptr;
    if (!d || !o || !p) return TMPC_ERR_INVALID_ARG;
    if (d->batch < 1 || d->N_max < 1 || d->nx < 1 || d->nu < 1 || d->ng < 1 || d->n_dyn < 1 ||
        d->n_track < 0)
        return TMPC_ERR_INVALID_ARG;
    const int n = d->nx + d->nu;
    if (n > 72 || d->nx > 64 || d->ng > 64) return TMPC_ERR_UNSUPPORTED;
    if (check_options(o) != TMPC_OK || check_params(*d, p) != TMPC_OK) return TMPC_ERR_INVALID_ARG;

    std::vector<int> Nh(d->batch), Mh(d->batch);
    TMPC_CUDA(cudaMemcpy(Nh.data(), p->N, sizeof(int) * d->batch, cudaMemcpyDeviceToHost));
    TMPC_CUDA(cudaMemcpy(Mh.data(), p->model, sizeof(int) * d->batch, cudaMemcpyDeviceToHost));
    for (int i = 0; i < d->batch; ++i) {
        if (Nh[i] < 1 || Nh[i] > d->N_max) return TMPC_ERR_INVALID_ARG;
        if (Mh[i] < 0 || Mh[i] >= MODEL_COUNT) return TMPC_ERR_INVALID_ARG;
        const ModelDims md = model_dims(Mh[i], d->nx, d->nu, d->ng);
        if (md.nx > d->nx || md.nu > d->nu || md.ng > d->ng) return TMPC_ERR_INVALID_ARG;
        if (Mh[i] == MODEL_LINEAR && (d->n_dyn < d->nx * d->nx + d->nx * d->nu || d->ng > d->nu))
            return TMPC_ERR_INVALID_ARG;
        if (is_bicycle(Mh[i]) && (d->n_track < 1 || d->n_dyn < 4)) return TMPC_ERR_INVALID_ARG;
        if (Mh[i] == MODEL_QUAD && d->n_dyn < 5) return TMPC_ERR_INVALID_ARG;
        if (Mh[i] == MODEL_SRB && d->n_dyn < 12) return TMPC_ERR_INVALID_ARG;
    }

    tmpc_handle* h = new (std::nothrow) tmpc_handle();
    if (!h) return TMPC_ERR_OOM;
    h->d = *d;
    h->o = *o;
    h->p = *p;
    KLayout& L = h->L;
    L.B = d->batch; L.Nmax = d->N_max; L.nx = d->nx; L.nu = d->nu; L.ng = d->ng; L.n = n;
    L.n_dyn = d->n_dyn; L.n_track = d->n_track;
    const long long T = d->N_max + 1;
    WsOff& off = h->off;
    if (!ws_layout(*d, off)) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "tmpc_setup: the per-instance workspace of N_max = %d exceeds 2^31 floats", d->N_max);
        delete h;
        return TMPC_ERR_INVALID_ARG;
    }
    if ((unsigned long long)off.stride > (unsigned long long)LLONG_MAX / sizeof(float) / (unsigned long long)d->batch) {
        delete h;
        return TMPC_ERR_INVALID_ARG;
    }

    cudaError_t e = cudaMalloc(&h->ws, sizeof(float) * off.stride * d->batch);
    if (e != cudaSuccess) { set_err("cudaMalloc(workspace)", e); delete h; return TMPC_ERR_OOM; }
    e = cudaMalloc(&h->order, sizeof(int) * (2 * d->batch + 8));
    if (e != cudaSuccess) { set_err("cudaMalloc(order)", e); tmpc_destroy(h); return TMPC_ERR_OOM; }
    h->queue = h->order + 2 * d->batch;   // 5 counters: 4 forward groups + backward
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&h->max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int max_optin = h->max_optin;
    // work estimate for longest-processing-time-first ordering: (N+1) n^2
    auto work = [&](int i) {
        const ModelDims m = model_dims(Mh[i], d->nx, d->nu, d->ng);
        return (long long)(Nh[i] + 1) * (m.nx + m.nu) * (m.nx + m.nu);
    };
    auto by_work = [&](int a, int b) { return work(a) > work(b); };
    // forward groups
    std::vector<int> ord;
    ord.reserve(2 * d->batch);
    for (int g = 0; g < 4; ++g) {
        std::vector<int> mem;
        for (int i = 0; i < d->batch; ++i) {
            const bool fastable = fast::supported(Mh[i]) && o->solver != 1;
            const int gi = fastable ? (Mh[i] == MODEL_DI ? 0 : Mh[i] == MODEL_BICYCLE ? 1 : 2) : 3;
            if (gi == g) mem.push_back(i);
        }
        if (mem.empty()) continue;
        std::stable_sort(mem.begin(), mem.end(), by_work);
        tmpc_handle::Group& G = h->groups[h->n_groups++];
        G.offset = (int)ord.size();
        G.count = (int)mem.size();
        ord.insert(ord.end(), mem.begin(), mem.end());
        if (g < 3) {
            G.model = Mh[mem[0]];
            for (int i : mem) G.Tmax = std::max(G.Tmax, Nh[i] + 1);
            // few instances whose arenas do not fit in shared memory: one thread-block cluster each
            const bool few_long = o->solver == 0 && !shared_fits(h, G) && (long long)G.count * 8 <= h->nsm;
            const int form = o->solver >= 2 ? o->solver : 2;
            e = cudaErrorNotSupported;
            if (few_long) e = configure_group(h, G, 6, o->threads);
            if (e != cudaSuccess) e = configure_group(h, G, form, o->threads);
            if (e == cudaErrorNotSupported && o->solver == 6) { tmpc_destroy(h); return TMPC_ERR_UNSUPPORTED; }
            if (e != cudaSuccess) { set_err("fast::prepare", e); tmpc_destroy(h); return TMPC_ERR_CUDA; }
        } else {
            G.model = -1;
        }
    }
    h->ord_host = ord;
    h->work_host.resize(d->batch);
    for (int i = 0; i < d->batch; ++i) h->work_host[i] = work(i);
    if (tmpc_status st = plan_backward(h); st != TMPC_OK) { tmpc_destroy(h); return st; }
    if (h->n_groups > 1) {
        e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        for (int g = 0; g < h->n_groups && e == cudaSuccess; ++g) {
            e = cudaStreamCreateWithFlags(&h->gs[g], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join[g], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) { set_err("group streams", e); tmpc_destroy(h); return TMPC_ERR_CUDA; }
    }
    if (tmpc_status st = ensure_buffers(h); st != TMPC_OK) { tmpc_destroy(h); return st; }
    for (int g = 0; g < 5 && e == cudaSuccess; ++g)
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&h->tev[g][k]);
    if (e != cudaSuccess) { set_err("timing events", e); tmpc_destroy(h); return TMPC_ERR_CUDA; }

    h->threads = o->threads > 0 ? o->threads : (n <= 16 ? 128 : 256);
    // ADMM vectors in shared memory when two CTAs per SM still fit
    h->L.vs = choose_vs(h->L, h->threads, max_optin);
    h->smem = smem_bytes(h->L);
    if (h->smem > 48 * 1024) {
        e = allow_max_smem(max_optin);
        if (e != cudaSuccess) { set_err("generic kernels: shared-memory limit", e); tmpc_destroy(h); return TMPC_ERR_CUDA; }
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel, h->threads, h->smem);
    h->grid_solve = std::max(1, std::min(d->batch, std::max(per_sm, 1) * h->nsm));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backward_kernel, h->threads, h->smem);
    h->grid_bwd = std::max(1, std::min(d->batch, std::max(per_sm, 1) * h->nsm));

    // staging buffers of the host-memory entry point (allocated once here)
    const long long B = d->batch;
    const size_t sz[] = {
        sizeof(int) * B, sizeof(int) * B,                                  // N, model
        sizeof(float) * B * T * d->nx, sizeof(float) * B * T * d->nu,      // Qd, Rd
        sizeof(float) * B * d->nu,                                          // Wd
        sizeof(float) * B * T * n, sizeof(float) * B * T * n,               // ref, lin
        sizeof(float) * B * T * d->ng, sizeof(float) * B * T * d->ng,       // lo, hi
        sizeof(float) * B * d->ng, sizeof(float) * B * d->ng,               // gamma2, gamma1
        sizeof(float) * B * d->n_dyn,                                       // dyn
        sizeof(float) * B * (d->n_track + 1) * 4,                           // track
        sizeof(float) * B * d->nx,                                          // x0
        sizeof(float) * B * T * n, sizeof(float) * B * T * d->ng,           // z, xi
        sizeof(float) * B * T * d->nx, sizeof(float) * B * T * d->ng,       // y_eq, y_ineq
        sizeof(int) * B, sizeof(float) * B * TMPC_STATS,                   // status, stats
        sizeof(float) * B * n};                                             // scale
    constexpr int kStaged = sizeof(sz) / sizeof(sz[0]);
    size_t tot = 0;
    size_t offs[kStaged];
    for (int k = 0; k < kStaged; ++k) { offs[k] = tot; tot += (sz[k] + 255) & ~size_t(255); }
    e = cudaMalloc(&h->stage, tot);
    if (e != cudaSuccess) { set_err("cudaMalloc(staging)", e); tmpc_destroy(h); return TMPC_ERR_OOM; }
    h->stage_bytes = tot;
    char* sb = reinterpret_cast<char*>(h->stage);
    h->sp.N = reinterpret_cast<int*>(sb + offs[0]);
    h->sp.model = reinterpret_cast<int*>(sb + offs[1]);
    h->sp.Qd = reinterpret_cast<float*>(sb + offs[2]);
    h->sp.Rd = reinterpret_cast<float*>(sb + offs[3]);
    h->sp.Wd = reinterpret_cast<float*>(sb + offs[4]);
    h->sp.ref = reinterpret_cast<float*>(sb + offs[5]);
    h->sp.lin = reinterpret_cast<float*>(sb + offs[6]);
    h->sp.lo = reinterpret_cast<float*>(sb + offs[7]);
    h->sp.hi = reinterpret_cast<float*>(sb + offs[8]);
    h->sp.gamma2 = reinterpret_cast<float*>(sb + offs[9]);
    h->sp.gamma1 = reinterpret_cast<float*>(sb + offs[10]);
    h->sp.dyn = reinterpret_cast<float*>(sb + offs[11]);
    h->sp.track = reinterpret_cast<float*>(sb + offs[12]);
    h->s_x0 = reinterpret_cast<float*>(sb + offs[13]);
    h->ss.z = reinterpret_cast<float*>(sb + offs[14]);
    h->ss.xi = reinterpret_cast<float*>(sb + offs[15]);
    h->ss.y_eq = reinterpret_cast<float*>(sb + offs[16]);
    h->ss.y_ineq = reinterpret_cast<float*>(sb + offs[17]);
    h->ss.status = reinterpret_cast<int*>(sb + offs[18]);
    h->ss.stats = reinterpret_cast<float*>(sb + offs[19]);
    h->sp.scale = reinterpret_cast<float*>(sb + offs[20]);
    *hp = h;
    return TMPC_OK;
}

tmpc_status tmpc_update_params(tmpc_handle* h, const tmpc_params* p) {
    if (!h) return TMPC_ERR_NOT_SETUP;
    if (check_params(h->d, p) != TMPC_OK) return TMPC_ERR_INVALID_ARG;
    h->p = *p;
    return TMPC_OK;
}

tmpc_status tmpc_set_options(tmpc_handle* h, const tmpc_options* o) {
    if (!h) return TMPC_ERR_NOT_SETUP;
    if (!o || check_options(o) != TMPC_OK) return TMPC_ERR_INVALID_ARG;
    if (o->threads != h->o.threads || o->solver != h->o.solver) return TMPC_ERR_INVALID_ARG;  // fixed at setup
    h->o = *o;
    return TMPC_OK;
}

// the forward launch(es) of group g on stream s
static tmpc_status launch_group(tmpc_handle* h, int g, const KOpts& ko, const KParams& kp, const KSol& ks,
                                const float* x0, int warm, cudaStream_t s) {
    const tmpc_handle::Group& G = h->groups[g];
    if (G.model >= 0 && G.plain) {
        TMPC_CUDA(fast::launch_plain(G.model, G.threads, s, h->L, ko, kp, ks, h->fws, h->fstride,
                                     h->order + G.offset, G.count, x0, warm, h->pstate));
    } else if (G.model >= 0 && G.cluster > 0) {
        TMPC_CUDA(fast::launch_cluster(G.model, G.policy, G.cluster, G.grid, G.threads, s, h->L, ko, kp, ks,
                                       h->fws, h->fstride, h->order + G.offset, G.count, x0, warm, h->gflags));
    } else if (G.model >= 0) {
        TMPC_CUDA(fast::launch(G.model, G.policy, G.grid, G.threads, G.smem, s, h->L, ko, kp, ks, h->fws, h->fstride,
                               h->order + G.offset, G.count, h->queue + g, x0, warm));
    } else {
        solve_kernel<<<std::min(h->grid_solve, G.count), h->threads, h->smem, s>>>(
            h->L, ko, kp, ks, h->ws, h->off, h->order + G.offset, G.count, h->queue + g, x0, warm);
        TMPC_CUDA(cudaGetLastError());
    }
    return TMPC_OK;
}

// launches are timed by events on their stream unless the stream is being captured
static bool timing_ok(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusNone;
}

// rescaling (params.scale) is built on the shared-memory kernels only: refuse a
// call that would send an instance to the generic kernel with a scale
static bool scale_supported(const tmpc_handle* h, const void* scale) {
    g_last_error[0] = '\0';
    if (!scale) return true;
    for (int g = 0; g < h->n_groups; ++g)
        if (h->groups[g].model < 0 && h->groups[g].count > 0) {
            snprintf(g_last_error, sizeof(g_last_error),
                     "params.scale: the rescaled ADMM runs on the shared-memory kernels (double integrator, "
                     "bicycle, quadrotor with solver 0 or 2..7); %d instance(s) of this handle use the generic kernel",
                     h->groups[g].count);
            return false;
        }
    return true;
}

static tmpc_status launch_solve(tmpc_handle* h, const tmpc_params& p, const float* x0,
                                const tmpc_solution& out, int warm, cudaStream_t s) {
    if (!scale_supported(h, p.scale)) return TMPC_ERR_INVALID_ARG;
    KSol ks{out.z, out.xi, out.y_eq, out.y_ineq, out.status, out.stats};
    TMPC_CUDA(cudaMemsetAsync(h->queue, 0, sizeof(int) * 5, s));
    const KOpts ko = to_kopts(h->o);
    const KParams kp = to_kparams(p);
    const bool fork = h->n_groups > 1 && h->ev_fork;
    const cudaStream_t s0 = s;
    if (fork) TMPC_CUDA(cudaEventRecord(h->ev_fork, s0));
    for (int g = 0; g < h->n_groups; ++g) {
        if (fork) {
            s = h->gs[g];
            TMPC_CUDA(cudaStreamWaitEvent(s, h->ev_fork, 0));
        }
        const bool t = timing_ok(s);
        if (t) TMPC_CUDA(cudaEventRecord(h->tev[g][0], s));
        if (tmpc_status st = launch_group(h, g, ko, kp, ks, x0, warm, s); st != TMPC_OK) return st;
        if (t) TMPC_CUDA(cudaEventRecord(h->tev[g][1], s));
        h->timed[g][0] = t;
        if (fork) TMPC_CUDA(cudaEventRecord(h->ev_join[g], s));
    }
    if (fork)
        for (int g = 0; g < h->n_groups; ++g) TMPC_CUDA(cudaStreamWaitEvent(s0, h->ev_join[g], 0));
    return TMPC_OK;
}

tmpc_status tmpc_solve(tmpc_handle* h, const float* x0, tmpc_solution* out, int32_t warm_start, void* stream) {
    if (!h) return TMPC_ERR_NOT_SETUP;
    if (!x0 || !out || !out->z || !out->xi || !out->y_eq || !out->y_ineq) return TMPC_ERR_INVALID_ARG;
    if (!aligned4(x0) || !aligned4(out->z) || !aligned4(out->xi) || !aligned4(out->y_eq) || !aligned4(out->y_ineq))
        return TMPC_ERR_INVALID_ARG;
    return launch_solve(h, h->p, x0, *out, warm_start ? 1 : 0, reinterpret_cast<cudaStream_t>(stream));
}

tmpc_status tmpc_autotune(tmpc_handle* h, const float* x0, const tmpc_solution* init, int32_t reps,
                          int32_t trial_sqp, tmpc_tune_result* res, void* stream) {
    if (!h) return TMPC_ERR_NOT_SETUP;
    if (!x0 || !aligned4(x0) || reps < 1 || reps > 1000 || trial_sqp < 0) return TMPC_ERR_INVALID_ARG;
    if (init && (!init->z || !init->xi || !init->y_eq || !init->y_ineq)) return TMPC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    KOpts ko = to_kopts(h->o);
    if (trial_sqp > 0) ko.max_sqp = std::min(ko.max_sqp, trial_sqp);
    const KParams kp = to_kparams(h->p);
    // trial outputs go to the staging buffers of tmpc_solve_host
    const KSol ks{h->ss.z, h->ss.xi, h->ss.y_eq, h->ss.y_ineq, h->ss.status, h->ss.stats};
    const long long B = h->d.batch, T = h->d.N_max + 1;
    const size_t bz = sizeof(float) * B * T * h->L.n, bg = sizeof(float) * B * T * h->d.ng,
                 bf = sizeof(float) * B * T * h->d.nx;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    TMPC_CUDA(cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) { cudaEventDestroy(ev[0]); return TMPC_ERR_CUDA; }
    tmpc_status st = TMPC_OK;
    // device milliseconds of one forward launch of group g in its current form,
    // from the caller's warm start when one is given (its copy is timed too)
    auto time_group = [&](int g, float* ms) -> tmpc_status {
        if (tmpc_status e = ensure_buffers(h); e != TMPC_OK) return e;
        TMPC_CUDA(cudaEventRecord(ev[0], s));
        if (init) {
            TMPC_CUDA(cudaMemcpyAsync(h->ss.z, init->z, bz, cudaMemcpyDeviceToDevice, s));
            TMPC_CUDA(cudaMemcpyAsync(h->ss.xi, init->xi, bg, cudaMemcpyDeviceToDevice, s));
            TMPC_CUDA(cudaMemcpyAsync(h->ss.y_eq, init->y_eq, bf, cudaMemcpyDeviceToDevice, s));
            TMPC_CUDA(cudaMemcpyAsync(h->ss.y_ineq, init->y_ineq, bg, cudaMemcpyDeviceToDevice, s));
        }
        TMPC_CUDA(cudaMemsetAsync(h->queue + g, 0, sizeof(int), s));
        if (tmpc_status e = launch_group(h, g, ko, kp, ks, x0, init ? 1 : 0, s); e != TMPC_OK) return e;
        TMPC_CUDA(cudaEventRecord(ev[1], s));
        TMPC_CUDA(cudaEventSynchronize(ev[1]));
        TMPC_CUDA(cudaEventElapsedTime(ms, ev[0], ev[1]));
        return TMPC_OK;
    };
    struct Cand { int form, threads; };
    for (int g = 0; g < h->n_groups && st == TMPC_OK; ++g) {
        tmpc_handle::Group& G = h->groups[g];
        tmpc_tune_result r{G.model, G.count, G.form, G.threads, G.cluster, 0, -1.f, -1.f};
        if (G.model < 0 || h->o.solver != 0) {   // generic kernel, or a form fixed by the options
            if (res) res[g] = r;
            continue;
        }
        const int def_form = G.form, def_threads = G.threads;
        const int t_full = h->o.threads > 0 ? h->o.threads : 256, t_half = h->o.threads > 0 ? h->o.threads : 128;
        std::vector<Cand> cands{{def_form, def_threads}};
        std::vector<Cand> more{{2, t_full}, {2, t_half}, {4, t_half}, {3, t_full}, {3, t_half}, {7, t_full}};
        if ((long long)G.count * 8 <= 2LL * h->nsm) more.push_back({6, t_full});   // about one wave of clusters
        for (const Cand& c : more) {
            bool seen = false;
            for (const Cand& d : cands) seen = seen || (d.form == c.form && d.threads == c.threads);
            if (!seen) cands.push_back(c);
        }
        const size_t nc = cands.size();
        std::vector<float> first(nc, -1.f), best(nc, -1.f);
        // clocks up: the setup's form until about 20 ms of device time (at most 10 launches)
        float warm_ms = 0.f;
        for (int k = 0; k < 10 && warm_ms < 20.f && st == TMPC_OK; ++k) {
            float ms = 0.f;
            if (configure_group(h, G, def_form, def_threads) != cudaSuccess) { st = TMPC_ERR_CUDA; break; }
            st = time_group(g, &ms);
            warm_ms += ms;
        }
        // one launch per form; forms four times slower than the fastest first launch are dropped
        for (size_t k = 0; k < nc && st == TMPC_OK; ++k) {
            if (configure_group(h, G, cands[k].form, cands[k].threads) != cudaSuccess) { cudaGetLastError(); continue; }
            st = time_group(g, &first[k]);
        }
        float fmin = -1.f;
        for (size_t k = 0; k < nc; ++k)
            if (first[k] >= 0.f && (fmin < 0.f || first[k] < fmin)) fmin = first[k];
        // reps interleaved passes over the remaining forms; a form's time is its fastest launch
        for (int rep = 0; rep < reps && st == TMPC_OK; ++rep)
            for (size_t k = 0; k < nc && st == TMPC_OK; ++k) {
                if (first[k] < 0.f || first[k] > 4.f * fmin) continue;
                if (configure_group(h, G, cands[k].form, cands[k].threads) != cudaSuccess) { st = TMPC_ERR_CUDA; break; }
                float ms = 0.f;
                st = time_group(g, &ms);
                if (best[k] < 0.f || ms < best[k]) best[k] = ms;
            }
        size_t kb = 0;
        for (size_t k = 0; k < nc; ++k) {
            if (best[k] < 0.f) continue;
            ++r.candidates;
            if (best[kb] < 0.f || best[k] < best[kb]) kb = k;
        }
        if (st != TMPC_OK || best[kb] < 0.f || configure_group(h, G, cands[kb].form, cands[kb].threads) != cudaSuccess) {
            cudaGetLastError();
            configure_group(h, G, def_form, def_threads);
            kb = 0;
        }
        r.solver = G.form;
        r.threads = G.threads;
        r.cluster = G.cluster;
        r.ms = best[kb];
        r.ms_default = best[0] >= 0.f ? best[0] : first[0];
        if (res) res[g] = r;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st != TMPC_OK) return st;
    if (tmpc_status e = ensure_buffers(h); e != TMPC_OK) return e;
    TMPC_CUDA(cudaStreamSynchronize(s));
    return plan_backward(h);
}

tmpc_status tmpc_backward(tmpc_handle* h, const float* x0, const tmpc_solution* sol, const float* dL_dz,
                          const float* dL_dxi, tmpc_grads* g, void* stream) {
    if (!h) return TMPC_ERR_NOT_SETUP;
    if (!x0 || !sol || !sol->z || !sol->xi || !sol->y_eq || !sol->y_ineq || !dL_dz || !g) return TMPC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    KSol ks{sol->z, sol->xi, sol->y_eq, sol->y_ineq, sol->status, sol->stats};
    KGrads kg{g->x0, g->Qd, g->Rd, g->Wd, g->ref, g->lin, g->lo, g->hi, g->gamma2, g->gamma1};
    TMPC_CUDA(cudaMemsetAsync(h->queue, 0, sizeof(int) * 5, s));
    if (h->dq) TMPC_CUDA(cudaMemsetAsync(h->dq, 0, sizeof(int) * (20 + (size_t)h->d.batch), s));
    const KOpts ko = to_kopts(h->o);
    const KParams kp = to_kparams(h->p);
    // one stream per shared-memory group plus the generic backward, forked from s when there are several
    const bool fork = h->n_groups > 1 && h->ev_fork;
    if (fork) TMPC_CUDA(cudaEventRecord(h->ev_fork, s));
    int used = 0;
    for (int gi = 0; gi < 5; ++gi) h->timed[gi][1] = false;
    for (int gi = 0; gi < h->n_groups; ++gi) {
        const tmpc_handle::Group& G = h->groups[gi];
        if (G.bgrid <= 0) continue;
        cudaStream_t sg = s;
        if (fork) {
            sg = h->gs[gi];
            TMPC_CUDA(cudaStreamWaitEvent(sg, h->ev_fork, 0));
        }
        const bool t = timing_ok(sg);
        if (t) TMPC_CUDA(cudaEventRecord(h->tev[gi][2], sg));
        TMPC_CUDA(fast::launch_backward(G.model, G.cluster, G.bgrid, G.threads, G.smem, sg, h->L, ko, kp, ks, h->fws,
                                        h->fstride, h->order + G.offset, G.count, h->queue + gi, x0, h->gflags,
                                        dL_dz, dL_dxi, kg, h->dws, h->dstride,
                                        h->dq ? h->dq + 20 : nullptr, h->dq ? h->dq + 4 * gi : nullptr,
                                        h->nsm));
        if (t) TMPC_CUDA(cudaEventRecord(h->tev[gi][3], sg));
        h->timed[gi][1] = t;
        if (fork) {
            TMPC_CUDA(cudaEventRecord(h->ev_join[gi], sg));
            used |= 1 << gi;
        }
    }
    if (h->bwd_generic > 0) {
        const bool t = timing_ok(s);
        if (t) TMPC_CUDA(cudaEventRecord(h->tev[4][2], s));
        backward_kernel<<<std::min(h->grid_bwd, h->bwd_generic), h->threads, h->smem, s>>>(
            h->L, ko, kp, ks, h->ws, h->off, h->order + h->d.batch, h->bwd_generic, h->queue + 4, x0, dL_dz, dL_dxi, kg,
            h->dws, h->dstride);
        TMPC_CUDA(cudaGetLastError());
        if (t) TMPC_CUDA(cudaEventRecord(h->tev[4][3], s));
        h->timed[4][1] = t;
    }
    for (int gi = 0; gi < h->n_groups; ++gi)
        if (used & (1 << gi)) TMPC_CUDA(cudaStreamWaitEvent(s, h->ev_join[gi], 0));
    return TMPC_OK;
}

tmpc_status tmpc_solve_host(tmpc_handle* h, const tmpc_params* hp, const float* x0, const float* z_init,
                            tmpc_solution* ho, void* stream) {
    if (!h) return TMPC_ERR_NOT_SETUP;
    if (!hp || !x0 || !ho || !ho->z || !ho->xi || !ho->y_eq || !ho->y_ineq) return TMPC_ERR_INVALID_ARG;
    if (!hp->N || !hp->model || !hp->Qd || !hp->Rd || !hp->lo || !hp->hi || !hp->dyn) return TMPC_ERR_INVALID_ARG;
    if (!scale_supported(h, hp->scale)) return TMPC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const tmpc_dims& d = h->d;
    const long long B = d.batch, T = d.N_max + 1, n = d.nx + d.nu;
    auto h2d = [&](const void* src, const void* dst, size_t bytes) -> cudaError_t {
        return cudaMemcpyAsync(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice, s);
    };
    tmpc_params dp = h->sp;
    TMPC_CUDA(h2d(hp->N, dp.N, sizeof(int) * B));
    TMPC_CUDA(h2d(hp->model, dp.model, sizeof(int) * B));
    TMPC_CUDA(h2d(hp->Qd, dp.Qd, sizeof(float) * B * T * d.nx));
    TMPC_CUDA(h2d(hp->Rd, dp.Rd, sizeof(float) * B * T * d.nu));
    if (hp->Wd) TMPC_CUDA(h2d(hp->Wd, dp.Wd, sizeof(float) * B * d.nu)); else dp.Wd = nullptr;
    if (hp->ref) TMPC_CUDA(h2d(hp->ref, dp.ref, sizeof(float) * B * T * n)); else dp.ref = nullptr;
    if (hp->lin) TMPC_CUDA(h2d(hp->lin, dp.lin, sizeof(float) * B * T * n)); else dp.lin = nullptr;
    TMPC_CUDA(h2d(hp->lo, dp.lo, sizeof(float) * B * T * d.ng));
    TMPC_CUDA(h2d(hp->hi, dp.hi, sizeof(float) * B * T * d.ng));
    if (hp->gamma2) TMPC_CUDA(h2d(hp->gamma2, dp.gamma2, sizeof(float) * B * d.ng)); else dp.gamma2 = nullptr;
    if (hp->gamma1) TMPC_CUDA(h2d(hp->gamma1, dp.gamma1, sizeof(float) * B * d.ng)); else dp.gamma1 = nullptr;
    TMPC_CUDA(h2d(hp->dyn, dp.dyn, sizeof(float) * B * d.n_dyn));
    if (hp->track && d.n_track > 0) TMPC_CUDA(h2d(hp->track, dp.track, sizeof(float) * B * (d.n_track + 1) * 4));
    else dp.track = nullptr;
    if (hp->scale) TMPC_CUDA(h2d(hp->scale, dp.scale, sizeof(float) * B * n)); else dp.scale = nullptr;
    TMPC_CUDA(h2d(x0, h->s_x0, sizeof(float) * B * d.nx));
    tmpc_solution ds = h->ss;
    if (z_init) {
        TMPC_CUDA(h2d(z_init, ds.z, sizeof(float) * B * T * n));
        TMPC_CUDA(cudaMemsetAsync(ds.xi, 0, sizeof(float) * B * T * d.ng, s));
        TMPC_CUDA(cudaMemsetAsync(ds.y_eq, 0, sizeof(float) * B * T * d.nx, s));
        TMPC_CUDA(cudaMemsetAsync(ds.y_ineq, 0, sizeof(float) * B * T * d.ng, s));
    }
    tmpc_status st = launch_solve(h, dp, h->s_x0, ds, z_init ? 1 : 0, s);
    if (st != TMPC_OK) return st;
    TMPC_CUDA(cudaMemcpyAsync(ho->z, ds.z, sizeof(float) * B * T * n, cudaMemcpyDeviceToHost, s));
    TMPC_CUDA(cudaMemcpyAsync(ho->xi, ds.xi, sizeof(float) * B * T * d.ng, cudaMemcpyDeviceToHost, s));
    TMPC_CUDA(cudaMemcpyAsync(ho->y_eq, ds.y_eq, sizeof(float) * B * T * d.nx, cudaMemcpyDeviceToHost, s));
    TMPC_CUDA(cudaMemcpyAsync(ho->y_ineq, ds.y_ineq, sizeof(float) * B * T * d.ng, cudaMemcpyDeviceToHost, s));
    if (ho->status) TMPC_CUDA(cudaMemcpyAsync(ho->status, ds.status, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
    if (ho->stats)
        TMPC_CUDA(cudaMemcpyAsync(ho->stats, ds.stats, sizeof(float) * B * TMPC_STATS, cudaMemcpyDeviceToHost, s));
    TMPC_CUDA(cudaStreamSynchronize(s));
    return TMPC_OK;
}

void tmpc_destroy(tmpc_handle* h) {
    if (!h) return;
    if (h->ws) cudaFree(h->ws);
    if (h->order) cudaFree(h->order);
    if (h->stage) cudaFree(h->stage);
    if (h->fws) cudaFree(h->fws);
    if (h->dws) cudaFree(h->dws);
    if (h->dq) cudaFree(h->dq);
    if (h->gflags) cudaFree(h->gflags);
    if (h->pstate) cudaFree(h->pstate);
    for (int g = 0; g < 4; ++g) {
        if (h->gs[g]) cudaStreamDestroy(h->gs[g]);
        if (h->ev_join[g]) cudaEventDestroy(h->ev_join[g]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    for (int g = 0; g < 5; ++g)
        for (int k = 0; k < 4; ++k)
            if (h->tev[g][k]) cudaEventDestroy(h->tev[g][k]);
    delete h;
}

tmpc_status tmpc_group_times(tmpc_handle* h, tmpc_group_time* out, int32_t* n_out) {
    if (!h) return TMPC_ERR_NOT_SETUP;
    if (!out || !n_out) return TMPC_ERR_INVALID_ARG;
    auto elapsed = [&](int slot, int k) -> float {
        if (!h->timed[slot][k / 2]) return -1.f;
        if (cudaEventSynchronize(h->tev[slot][k + 1]) != cudaSuccess) { cudaGetLastError(); return -1.f; }
        float ms = -1.f;
        if (cudaEventElapsedTime(&ms, h->tev[slot][k], h->tev[slot][k + 1]) != cudaSuccess) {
            cudaGetLastError();
            return -1.f;
        }
        return ms;
    };
    int n = 0;
    for (int g = 0; g < h->n_groups; ++g) {
        const tmpc_handle::Group& G = h->groups[g];
        tmpc_group_time& r = out[n++];
        r.model = G.model;
        r.form = G.model < 0 ? 1 : G.form;
        r.count = G.count;
        r.fwd_ms = elapsed(g, 0);
        r.bwd_ms = G.model >= 0 && G.bgrid > 0 ? elapsed(g, 2) : -1.f;
    }
    if (h->bwd_generic > 0) {   // the generic backward (generic group and the LDL forms' instances)
        tmpc_group_time& r = out[n++];
        r.model = -1;
        r.form = 1;
        r.count = h->bwd_generic;
        r.fwd_ms = -1.f;
        r.bwd_ms = elapsed(4, 2);
    }
    *n_out = n;
    return TMPC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// tmpc_solve_static: the generic solve kernel with its scratch (instance order,
// work-queue counter, per-instance workspace) in a file-scope device array
// instead of memory allocated by tmpc_setup.  Nothing here allocates.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_scratch[TMPC_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kStaticMaxDevices = 64;
void* g_static_base[kStaticMaxDevices] = {};   // scratch address per device, looked up once
std::mutex g_static_mu;

// one-time set-up per device (the device must be current): address of the scratch array
tmpc_status static_scratch_base(void** base) {
    int dev = 0;
    TMPC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kStaticMaxDevices) return TMPC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_base[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
            set_err("cudaGetSymbolAddress(static scratch)", e);
            return TMPC_ERR_CUDA;
        }
        g_static_base[dev] = ptr;
    }
    *base = g_static_base[dev];
    return TMPC_OK;
}


// One CTA: checks every instance (the checks tmpc_setup makes on the host),
// writes the valid ones to the tail of the order array and points the
// work-queue counter at the first of them; an invalid instance gets
// TMPC_INST_INVALID and zero outputs and is never solved.
__global__ void static_prologue(KLayout L, const int* N, const int* model, int* order, int* queue, KSol out) {
    __shared__ int s_valid;
    if (threadIdx.x == 0) s_valid = 0;
    __syncthreads();
    const long long T = L.Nmax + 1;
    for (int i = threadIdx.x; i < L.B; i += blockDim.x) {
        const int Ni = N[i], m = model[i];
        bool ok = Ni >= 1 && Ni <= L.Nmax && m >= 0 && m < MODEL_COUNT;
        if (ok) {
            const ModelDims md = model_dims(m, L.nx, L.nu, L.ng);
            ok = md.nx <= L.nx && md.nu <= L.nu && md.ng <= L.ng;
            if (m == MODEL_LINEAR) ok = ok && L.n_dyn >= L.nx * L.nx + L.nx * L.nu && L.ng <= L.nu;
            if (is_bicycle(m)) ok = ok && L.n_track >= 1 && L.n_dyn >= 4;
            if (m == MODEL_QUAD) ok = ok && L.n_dyn >= 5;
            if (m == MODEL_SRB) ok = ok && L.n_dyn >= 12;
        }
        if (ok) {
            const int slot = atomicAdd(&s_valid, 1);
            order[L.B - 1 - slot] = i;
        } else {
            for (long long k = 0; k < T * L.n; ++k) out.z[i * T * L.n + k] = 0.f;
            for (long long k = 0; k < T * L.ng; ++k) { out.xi[i * T * L.ng + k] = 0.f; out.yg[i * T * L.ng + k] = 0.f; }
            for (long long k = 0; k < T * L.nx; ++k) out.yf[i * T * L.nx + k] = 0.f;
            if (out.stats)
                for (int k = 0; k < TMPC_STATS; ++k) out.stats[(long long)i * TMPC_STATS + k] = 0.f;
            out.status[i] = TMPC_INST_INVALID;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *queue = L.B - s_valid;
}

}  // namespace

extern "C" {

tmpc_status tmpc_solve_static(const tmpc_dims* d, const tmpc_options* o, const tmpc_params* p, const float* x0,
                              tmpc_solution* out, int32_t warm_start, void* stream) {
    g_last_error[0] = '\0';
    if (!d || !o || !p || !x0 || !out || !out->z || !out->xi || !out->y_eq || !out->y_ineq || !out->status)
        return TMPC_ERR_INVALID_ARG;
    if (d->batch < 1 || d->N_max < 1 || d->nx < 1 || d->nu < 1 || d->ng < 1 || d->n_dyn < 1 || d->n_track < 0)
        return TMPC_ERR_INVALID_ARG;
    const int n = d->nx + d->nu;
    if (n > 72 || d->nx > 64 || d->ng > 64) return TMPC_ERR_UNSUPPORTED;
    if (check_options(o) != TMPC_OK || check_params(*d, p) != TMPC_OK) return TMPC_ERR_INVALID_ARG;
    if (o->solver != 0 && o->solver != 1) return TMPC_ERR_INVALID_ARG;
    if (p->scale) {   // the generic kernel has no rescaled ADMM
        snprintf(g_last_error, sizeof(g_last_error),
                 "tmpc_solve_static: params.scale is not supported (the generic kernel has no rescaled ADMM)");
        return TMPC_ERR_INVALID_ARG;
    }
    if (!aligned4(x0) || !aligned4(out->z) || !aligned4(out->xi) || !aligned4(out->y_eq) ||
        !aligned4(out->y_ineq) || !aligned4(out->status) || (out->stats && !aligned4(out->stats)))
        return TMPC_ERR_INVALID_ARG;

    WsOff off;
    if (!ws_layout(*d, off)) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "tmpc_solve_static: the per-instance workspace of N_max = %d exceeds 2^31 floats; "
                 "the static scratch holds %zu bytes", d->N_max, (size_t)TMPC_STATIC_SCRATCH_BYTES);
        return TMPC_ERR_INVALID_ARG;
    }
    const long long stride = off.stride;
    if ((unsigned long long)stride > (unsigned long long)TMPC_STATIC_SCRATCH_BYTES / sizeof(float) / (unsigned long long)d->batch) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "tmpc_solve_static: this batch needs more than %zu bytes of scratch (%lld per instance); "
                 "the static scratch holds %zu bytes",
                 (size_t)TMPC_STATIC_SCRATCH_BYTES, (long long)(sizeof(float) * stride), (size_t)TMPC_STATIC_SCRATCH_BYTES);
        return TMPC_ERR_INVALID_ARG;
    }
    const size_t head = ((sizeof(int) * ((size_t)d->batch + 1)) + 255) & ~size_t(255);  // order [B], counter
    const size_t need = head + sizeof(float) * (size_t)stride * (size_t)d->batch;
    if (need > (size_t)TMPC_STATIC_SCRATCH_BYTES) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "tmpc_solve_static: this batch needs %zu bytes of scratch (%lld per instance); "
                 "the static scratch holds %zu bytes",
                 need, (long long)(sizeof(float) * stride), (size_t)TMPC_STATIC_SCRATCH_BYTES);
        return TMPC_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    const tmpc_status st = static_scratch_base(&base);
    if (st != TMPC_OK) return st;
    int* order = static_cast<int*>(base);
    int* queue = order + d->batch;
    float* ws = reinterpret_cast<float*>(static_cast<char*>(base) + head);

    KLayout L;
    L.B = d->batch; L.Nmax = d->N_max; L.nx = d->nx; L.nu = d->nu; L.ng = d->ng; L.n = n;
    L.n_dyn = d->n_dyn; L.n_track = d->n_track;
    const int threads = o->threads > 0 ? o->threads : (n <= 16 ? 128 : 256);
    int max_optin = 0;
    {
        int dv = 0;
        TMPC_CUDA(cudaGetDevice(&dv));
        TMPC_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dv));
    }
    L.vs = choose_vs(L, threads, max_optin);
    const size_t smem = smem_bytes(L);
    if (smem > 48 * 1024) TMPC_CUDA(allow_max_smem(max_optin));
    int dev = 0, nsm = 1, per_sm = 1;
    TMPC_CUDA(cudaGetDevice(&dev));
    TMPC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    TMPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel, threads, smem));
    const int grid = std::max(1, std::min(d->batch, std::max(per_sm, 1) * nsm));

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const KSol ks{out->z, out->xi, out->y_eq, out->y_ineq, out->status, out->stats};
    static_prologue<<<1, 256, 0, s>>>(L, p->N, p->model, order, queue, ks);
    TMPC_CUDA(cudaGetLastError());
    solve_kernel<<<grid, threads, smem, s>>>(L, to_kopts(*o), to_kparams(*p), ks, ws, off, order, d->batch,
                                             queue, x0, warm_start ? 1 : 0);
    TMPC_CUDA(cudaGetLastError());
    return TMPC_OK;
}

}  // extern "C"
