// Host driver and C ABI of libjjacobi: handle life cycle, workspaces, the
// sweep loop (one CUDA graph per sweep), convergence test, extraction.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "jj_common.cuh"

using namespace jj;

struct jj_ctx {
    jj_params p{};
    bool cplx = false;
    int E = 1;  // doubles per element
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t m = 0, n = 0, ldw = 0;
    double tol = kDefaultTol;
    int max_sweeps = 60, inner_max_sweeps = 30;

    // ordering / blocks
    bool blocked = false;
    int bw = 0, nbl = 0, steps = 0, npairs = 0, kmax = 0;
    std::vector<int32_t> offs, sizes;
    int32_t *d_pairs = nullptr;   // blocked: [steps][npairs][4]; plain: [steps][npairs][2]
    double *Gw[2] = {nullptr, nullptr};
    double *Ablk = nullptr, *Wblk = nullptr;
    double *d_norm = nullptr;
    bool ozaki = false;                 // Gram on the tensor cores (fp16 digits)
    bool ozaki_update = false;          // update on the tensor cores too
    int32_t *d_mod = nullptr, *d_clean = nullptr, *d_flags = nullptr, *d_sweep = nullptr;
    uint8_t *d_wdig = nullptr;          // W-side digits of the digit update (per pair)
    int32_t *d_wdexp = nullptr;
    int oz_slices_gram = 8, oz_slices_update = 8;
    int32_t *d_cexp = nullptr;          // column exponents (Ozaki Gram)
    unsigned long long *d_ozacc = nullptr;  // int128 Gram accumulators

    int32_t *d_perm = nullptr;    // work column -> caller column
    int32_t *d_rank = nullptr;    // extraction with sorting: column -> rank of its lambda
    int8_t *d_Jw = nullptr;       // J in work order
    int8_t *d_Jorig = nullptr;    // J in caller order
    unsigned long long *d_cnt = nullptr, *h_cnt = nullptr;
    double *d_lam = nullptr;      // extraction temp (n)
    double *h_lam = nullptr;      // pinned (n)
    double *d_Ghost = nullptr;    // device copy for jjacobi_solve_host (lazy)
    double *d_Uhost = nullptr;

    void *G_user = nullptr;
    int64_t ldg_user = 0;
    bool solved = false;
    int launches_per_sweep = 0;

    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaEvent_t ev_legacy = nullptr;  // orders a private stream after the legacy stream
    // profiling (params.profile): events around each kernel family of each step
    std::vector<cudaEvent_t> pev;
    double prof_ms[8] = {0};
    int64_t prof_n[8] = {0};
};

namespace {

__global__ void sweep_begin_kernel(int32_t *sweep) { *sweep += 1; }

#define JJ_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            if (getenv("JJACOBI_DEBUG"))                                                \
                fprintf(stderr, "jjacobi: %s failed: %s (%s:%d)\n", #call,             \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                    \
            return JJ_CUDA_ERROR;                                                       \
        }                                                                               \
    } while (0)

int status_from_flags(unsigned long long err) {
    if (err & kErrNonfinite) return JJ_NONFINITE;
    if (err & kErrNotPosdef) return JJ_NOT_POSDEF;
    if (err & kErrTimeout) return JJ_DEVICE_TIMEOUT;
    return JJ_OK;
}

void free_ctx(jj_ctx *c) {
    if (!c) return;
    for (auto &g : c->graph)
        if (g) cudaGraphExecDestroy(g);
    cudaFree(c->d_pairs);
    cudaFree(c->Gw[0]);
    cudaFree(c->Gw[1]);
    cudaFree(c->Ablk);
    cudaFree(c->Wblk);
    cudaFree(c->d_cexp);
    cudaFree(c->d_ozacc);
    cudaFree(c->d_wdig);
    cudaFree(c->d_wdexp);
    cudaFree(c->d_mod);
    cudaFree(c->d_clean);
    cudaFree(c->d_flags);
    cudaFree(c->d_sweep);
    cudaFree(c->d_norm);
    cudaFree(c->d_perm);
    cudaFree(c->d_rank);
    cudaFree(c->d_Jw);
    cudaFree(c->d_Jorig);
    cudaFree(c->d_cnt);
    cudaFree(c->d_lam);
    cudaFree(c->d_Ghost);
    cudaFree(c->d_Uhost);
    if (c->h_cnt) cudaFreeHost(c->h_cnt);
    if (c->h_lam) cudaFreeHost(c->h_lam);
    if (c->ev_legacy) cudaEventDestroy(c->ev_legacy);
    for (auto e : c->pev) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// Profiling: event slot of (step, point) and the kernel family between points.
struct ProfMark {
    int ev;
    int family;  // family timed from this mark to the next one of the step (-1: none)
};

// Record one sweep into the stream being captured (or run it directly).
int enqueue_sweep(jj_ctx *c, int start_buf, int *launches, std::vector<ProfMark> *marks) {
    cudaStream_t st = c->stream;
    int L = 0;
    auto mark = [&](int family) -> int {
        if (!marks) return JJ_OK;
        const int idx = (int)marks->size();
        if (idx >= (int)c->pev.size()) {
            cudaEvent_t e;
            JJ_CUDA(cudaEventCreate(&e));
            c->pev.push_back(e);
        }
        JJ_CUDA(cudaEventRecord(c->pev[idx], st));
        marks->push_back({idx, family});
        return JJ_OK;
    };
    JJ_CUDA(cudaMemsetAsync(c->d_cnt, 0, kNumCounters * sizeof(unsigned long long), st));
    if (!c->blocked) {
        if (mark(4)) return JJ_CUDA_ERROR;
        JJ_CUDA(launch_column_norms(c->cplx, c->Gw[0], c->ldw, c->m, c->n, c->d_norm, st));
        ++L;
        if (mark(3)) return JJ_CUDA_ERROR;
        for (int t = 0; t < c->steps; ++t) {
            JJ_CUDA(launch_plain_step(c->cplx, c->Gw[0], c->ldw, c->m, c->n,
                                      c->d_pairs + (size_t)t * c->npairs * 2, c->npairs, c->d_Jw,
                                      c->d_norm, c->tol, c->d_cnt, st));
            ++L;
        }
        if (mark(-1)) return JJ_CUDA_ERROR;
    } else {
        sweep_begin_kernel<<<1, 1, 0, st>>>(c->d_sweep);
        JJ_CUDA(cudaGetLastError());
        ++L;
        int cur = start_buf;
        for (int t = 0; t < c->steps; ++t) {
            const int32_t *pr = c->d_pairs + (size_t)t * c->npairs * 4;
            StepCtl ctl;
            ctl.mod_step = c->d_mod;
            ctl.clean_at = c->d_clean;
            ctl.flags = c->d_flags;
            ctl.sweep = c->d_sweep;
            ctl.step = t;
            ctl.steps = c->steps;
            ctl.npairs = c->npairs;
            if (mark(0)) return JJ_CUDA_ERROR;
            if (c->ozaki) {
                JJ_CUDA(launch_colexp(c->cplx, c->Gw[cur], c->ldw, c->m, c->n, c->d_cexp, st));
                JJ_CUDA(launch_gram_ozaki(c->cplx, c->Gw[cur], c->ldw, c->m, pr, c->npairs,
                                          c->Ablk, c->kmax, c->d_cexp, c->d_ozacc,
                                          c->oz_slices_gram, c->d_cnt, st, ctl));
                L += 3;
            } else {
                JJ_CUDA(launch_gram(c->cplx, c->p.gemm, c->Gw[cur], c->ldw, c->m, pr, c->npairs,
                                    c->Ablk, c->kmax, st, ctl));
                L += 1;
            }
            if (mark(1)) return JJ_CUDA_ERROR;
            UpdDigits ud;
            if (c->ozaki_update) {
                ud.img = c->d_wdig;
                ud.wexp = c->d_wdexp;
                ud.cexp = c->d_cexp;
                ud.slices = c->oz_slices_update;
            }
            JJ_CUDA(launch_inner(c->cplx, c->Ablk, c->Wblk, c->kmax, pr, c->npairs, c->d_Jw,
                                 c->tol, c->inner_max_sweeps, c->p.inner_block_width, c->d_cnt,
                                 st, ctl, ud));
            if (mark(2)) return JJ_CUDA_ERROR;
            if (c->ozaki_update)
                JJ_CUDA(launch_update_ozaki(c->cplx, c->Gw[cur], c->Gw[cur ^ 1], c->ldw, c->m, pr,
                                            c->npairs, c->Wblk, c->kmax, c->d_cexp,
                                            c->oz_slices_update, c->d_cnt, st, ctl, ud));
            else
                JJ_CUDA(launch_update(c->cplx, c->p.gemm, c->Gw[cur], c->Gw[cur ^ 1], c->ldw, c->m,
                                      pr, c->npairs, c->Wblk, c->kmax, st, ctl));
            L += 2;
            if (mark(-1)) return JJ_CUDA_ERROR;
            cur ^= 1;
        }
    }
    JJ_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, kNumCounters * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st));
    if (launches) *launches = L;
    return JJ_OK;
}

int build_graph(jj_ctx *c, int start_buf) {
    if (c->graph[start_buf]) return JJ_OK;
    cudaGraph_t g = nullptr;
    JJ_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int L = 0;
    const int rc = enqueue_sweep(c, start_buf, &L, nullptr);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc != JJ_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return JJ_CUDA_ERROR;
    }
    e = cudaGraphInstantiate(&c->graph[start_buf], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return JJ_CUDA_ERROR;
    c->launches_per_sweep = L;
    return JJ_OK;
}

// With a private stream (the caller passed none), work the caller enqueued on
// the legacy default stream must finish before ours starts.
int order_after_legacy(jj_ctx *c) {
    if (!c->own_stream) return JJ_OK;
    JJ_CUDA(cudaEventRecord(c->ev_legacy, cudaStreamLegacy));
    JJ_CUDA(cudaStreamWaitEvent(c->stream, c->ev_legacy, 0));
    return JJ_OK;
}

int end_buffer_after_sweep(const jj_ctx *c, int start) {
    return c->blocked ? (start ^ (c->steps & 1)) : 0;
}

}  // namespace

extern "C" {

void jjacobi_default_params(jj_params *p, int64_t m, int64_t n, int32_t dtype) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->m = m;
    p->n = n;
    p->dtype = dtype;
    p->block_width = 0;
    p->inner_block_width = 0;
    p->order = JJ_ORDER_ROUND_ROBIN;
    p->gemm = JJ_GEMM_FP64;
    p->ozaki_slices = 0;
    p->tol = kDefaultTol;
    p->max_sweeps = 60;
    p->inner_max_sweeps = 30;
    p->cuda_stream = nullptr;
}

const char *jjacobi_status_string(int status) {
    switch (status) {
        case JJ_OK: return "JJ_OK";
        case JJ_INVALID_ARG: return "JJ_INVALID_ARG";
        case JJ_NOT_CONVERGED: return "JJ_NOT_CONVERGED";
        case JJ_NOT_POSDEF: return "JJ_NOT_POSDEF";
        case JJ_NONFINITE: return "JJ_NONFINITE";
        case JJ_DEVICE_TIMEOUT: return "JJ_DEVICE_TIMEOUT";
        case JJ_CUDA_ERROR: return "JJ_CUDA_ERROR";
        case JJ_NOT_SOLVED: return "JJ_NOT_SOLVED";
        default: return "JJ_UNKNOWN";
    }
}

int32_t jjacobi_version(void) { return JJACOBI_VERSION; }

int jjacobi_kernel_times(jj_handle c, double *times_ms, int64_t *launches) {
    if (!c || !times_ms) return JJ_INVALID_ARG;
    for (int i = 0; i < 8; ++i) {
        times_ms[i] = c->prof_ms[i];
        if (launches) launches[i] = c->prof_n[i];
    }
    return JJ_OK;
}

int jjacobi_create(jj_handle *h, const jj_params *p) {
    if (!h) return JJ_INVALID_ARG;
    *h = nullptr;
    if (!p || p->n < 1 || p->m < p->n || (p->dtype != JJ_F64 && p->dtype != JJ_C128) ||
        p->block_width < 0 || p->inner_block_width < 0 ||
        (p->order != JJ_ORDER_ROUND_ROBIN && p->order != JJ_ORDER_MODULUS) ||
        (p->gemm < JJ_GEMM_FP64 || p->gemm > JJ_GEMM_AUTO) ||
        p->n > (int64_t)1 << 30)
        return JJ_INVALID_ARG;
    jj_ctx *c = new jj_ctx();
    c->p = *p;
    c->cplx = p->dtype == JJ_C128;
    c->E = c->cplx ? 2 : 1;
    c->m = p->m;
    c->n = p->n;
    c->ldw = (p->m + 3) & ~int64_t(3);
    c->tol = p->tol > 0 ? p->tol : kDefaultTol;
    c->max_sweeps = p->max_sweeps > 0 ? p->max_sweeps : 60;
    c->inner_max_sweeps = p->inner_max_sweeps > 0 ? p->inner_max_sweeps : 30;
    auto fail = [&](int rc) {
        free_ctx(c);
        return rc;
    };
    if (p->cuda_stream) {
        c->stream = (cudaStream_t)p->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(JJ_CUDA_ERROR);
        c->own_stream = true;
        if (cudaEventCreateWithFlags(&c->ev_legacy, cudaEventDisableTiming) != cudaSuccess)
            return fail(JJ_CUDA_ERROR);
    }
    const int64_t n = c->n;
    std::vector<int32_t> tab;
    if (p->block_width == 0 || n < 4) {
        // plain: round-robin over single columns (n padded to even)
        c->blocked = false;
        const int npl = (int)(n + (n & 1));
        c->npairs = npl / 2;
        c->steps = npl - 1;
        if (npl >= 2) {
            tab.resize((size_t)c->steps * c->npairs * 2);
            schedule_pairs(npl, JJ_ORDER_ROUND_ROBIN, 1, tab.data());
        }
    } else {
        c->blocked = true;
        const int b = p->block_width;
        int nbl = (int)(2 * ((n + 2 * (int64_t)b - 1) / (2 * (int64_t)b)));
        if (nbl > n - (n & 1)) nbl = (int)(n - (n & 1));
        if (nbl < 2) nbl = 2;
        c->nbl = nbl;
        c->bw = b;
        const int br = (int)(n % nbl), nmin = (int)(n / nbl);
        c->sizes.resize(nbl);
        c->offs.resize(nbl + 1);
        c->offs[0] = 0;
        for (int l = 0; l < nbl; ++l) {
            c->sizes[l] = l < br ? nmin + 1 : nmin;  // uniform partition (3.3)
            c->offs[l + 1] = c->offs[l] + c->sizes[l];
        }
        c->npairs = nbl / 2;
        c->kmax = 2 * (nmin + (br ? 1 : 0));
        std::vector<int32_t> bp((size_t)2 * nbl * nbl);
        c->steps = schedule_pairs(nbl, p->order, 1, bp.data());
        tab.resize((size_t)c->steps * c->npairs * 4);
        for (int t = 0; t < c->steps; ++t)
            for (int q = 0; q < c->npairs; ++q) {
                const int i = bp[2 * (t * c->npairs + q)], j = bp[2 * (t * c->npairs + q) + 1];
                int32_t *d = &tab[4 * ((size_t)t * c->npairs + q)];
                d[0] = c->offs[i];
                d[1] = c->sizes[i];
                d[2] = c->offs[j];
                d[3] = c->sizes[j];
            }
    }
    const size_t gbytes = (size_t)c->ldw * n * c->E * sizeof(double);
    if (cudaMalloc(&c->Gw[0], gbytes) != cudaSuccess) return fail(JJ_CUDA_ERROR);
    if (c->blocked) {
        if (cudaMalloc(&c->Gw[1], gbytes) != cudaSuccess) return fail(JJ_CUDA_ERROR);
        const size_t bb = (size_t)c->npairs * c->kmax * c->kmax * c->E * sizeof(double);
        if (cudaMalloc(&c->Ablk, bb) != cudaSuccess) return fail(JJ_CUDA_ERROR);
        if (cudaMalloc(&c->Wblk, bb) != cudaSuccess) return fail(JJ_CUDA_ERROR);
        const bool oz_ok = ozaki_supported(c->cplx, c->kmax);
        if ((p->gemm == JJ_GEMM_OZAKI_FP16 || p->gemm == JJ_GEMM_OZAKI_GRAM) && !oz_ok)
            return fail(JJ_INVALID_ARG);
        c->ozaki = oz_ok && p->gemm != JJ_GEMM_FP64;
        c->ozaki_update = c->ozaki && p->gemm == JJ_GEMM_OZAKI_FP16;
        const size_t nslots = (size_t)c->steps * c->npairs;
        if (cudaMalloc(&c->d_mod, n * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&c->d_clean, nslots * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&c->d_flags, c->npairs * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&c->d_sweep, sizeof(int32_t)) != cudaSuccess)
            return fail(JJ_CUDA_ERROR);
        if (c->ozaki) {
            if (p->ozaki_slices > 0) {
                if (p->ozaki_slices > ozaki_max_update_slices(c->cplx, c->kmax))
                    return fail(JJ_INVALID_ARG);
                c->oz_slices_update = p->ozaki_slices;
            }
            if (c->ozaki_update &&
                (cudaMalloc(&c->d_wdig, (size_t)c->npairs * 16 * kUpdSliceBytes) != cudaSuccess ||
                 cudaMalloc(&c->d_wdexp, (size_t)c->npairs * 64 * sizeof(int32_t)) != cudaSuccess))
                return fail(JJ_CUDA_ERROR);
            if (cudaMalloc(&c->d_cexp, n * sizeof(int32_t)) != cudaSuccess ||
                cudaMalloc(&c->d_ozacc, ozaki_gram_workspace_bytes(c->npairs, c->kmax, c->cplx)) !=
                    cudaSuccess)
                return fail(JJ_CUDA_ERROR);
        }
    } else {
        if (cudaMalloc(&c->d_norm, n * sizeof(double)) != cudaSuccess) return fail(JJ_CUDA_ERROR);
    }
    if (!tab.empty()) {
        if (cudaMalloc(&c->d_pairs, tab.size() * sizeof(int32_t)) != cudaSuccess)
            return fail(JJ_CUDA_ERROR);
        if (cudaMemcpy(c->d_pairs, tab.data(), tab.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(JJ_CUDA_ERROR);
    }
    if (cudaMalloc(&c->d_perm, n * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_rank, n * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_Jw, n) != cudaSuccess || cudaMalloc(&c->d_Jorig, n) != cudaSuccess ||
        cudaMalloc(&c->d_cnt, kNumCounters * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_lam, n * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->h_cnt, kNumCounters * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&c->h_lam, n * sizeof(double)) != cudaSuccess)
        return fail(JJ_CUDA_ERROR);
    *h = c;
    return JJ_OK;
}

void jjacobi_destroy(jj_handle h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_ctx(h);
}

int jjacobi_solve(jj_handle c, void *G, int64_t ldg, const int8_t *J, jj_info *info) {
    const auto t0 = std::chrono::steady_clock::now();
    jj_info inf{};
    auto finish = [&](int rc) {
        inf.status = rc;
        inf.seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (info) *info = inf;
        return rc;
    };
    if (!c || !G || !J || ldg < c->m) return finish(JJ_INVALID_ARG);
    const int64_t n = c->n;
    std::vector<int32_t> perm;
    perm.reserve(n);
    for (int64_t i = 0; i < n; ++i) {
        if (J[i] != 1 && J[i] != -1) return finish(JJ_INVALID_ARG);
        if (J[i] > 0) perm.push_back((int32_t)i);
    }
    for (int64_t i = 0; i < n; ++i)
        if (J[i] < 0) perm.push_back((int32_t)i);
    std::vector<int8_t> Jw(n);
    for (int64_t i = 0; i < n; ++i) Jw[i] = J[perm[i]];
    c->solved = false;
    c->G_user = G;
    c->ldg_user = ldg;
    inf.block_width = c->blocked ? c->bw : 0;
    inf.nbl = c->nbl;
    inf.steps_per_sweep = c->steps;
    cudaStream_t st = c->stream;
    if (order_after_legacy(c) != JJ_OK) return finish(JJ_CUDA_ERROR);
    JJ_CUDA(cudaMemcpyAsync(c->d_perm, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    JJ_CUDA(cudaMemcpyAsync(c->d_Jw, Jw.data(), n, cudaMemcpyHostToDevice, st));
    JJ_CUDA(cudaMemcpyAsync(c->d_Jorig, J, n, cudaMemcpyHostToDevice, st));
    JJ_CUDA(launch_permute_columns(c->cplx, (const double *)G, ldg, c->Gw[0], c->ldw, c->m, n,
                                   c->d_perm, false, st));
    if (c->blocked) {
        JJ_CUDA(cudaMemsetAsync(c->d_mod, 0xFF, n * sizeof(int32_t), st));
        JJ_CUDA(cudaMemsetAsync(c->d_clean, 0xFF, (size_t)c->steps * c->npairs * sizeof(int32_t), st));
        JJ_CUDA(cudaMemsetAsync(c->d_flags, 0, c->npairs * sizeof(int32_t), st));
        JJ_CUDA(cudaMemsetAsync(c->d_sweep, 0, sizeof(int32_t), st));
    }
    int launches = 1;
    int cur = 0;
    int rc = JJ_NOT_CONVERGED;
    for (int sweep = 1; sweep <= c->max_sweeps; ++sweep) {
        if (c->p.profile) {
            std::vector<ProfMark> marks;
            int L = 0;
            const int r = enqueue_sweep(c, cur, &L, &marks);
            if (r != JJ_OK) return finish(r);
            JJ_CUDA(cudaStreamSynchronize(st));
            for (size_t i = 0; i + 1 < marks.size(); ++i) {
                if (marks[i].family < 0) continue;
                float ms = 0.f;
                JJ_CUDA(cudaEventElapsedTime(&ms, c->pev[marks[i].ev], c->pev[marks[i + 1].ev]));
                c->prof_ms[marks[i].family] += ms;
                c->prof_n[marks[i].family] += 1;
            }
            launches += L;
        } else {
            int r = build_graph(c, cur);
            if (r != JJ_OK) return finish(r);
            JJ_CUDA(cudaGraphLaunch(c->graph[cur], st));
            JJ_CUDA(cudaStreamSynchronize(st));
            launches += c->launches_per_sweep;
        }
        inf.sweeps = sweep;
        const unsigned long long rot = c->h_cnt[kCntRot];
        inf.rotations += (int64_t)rot;
        inf.pairs_evaluated += (int64_t)c->h_cnt[kCntPairs];
        inf.pairs_rotated += (int64_t)c->h_cnt[kCntPairsRot];
        double mo;
        std::memcpy(&mo, &c->h_cnt[kCntMaxOff], sizeof(double));
        inf.last_max_offdiag = mo;
        cur = end_buffer_after_sweep(c, cur);
        const int err = status_from_flags(c->h_cnt[kCntErr]);
        if (err != JJ_OK) {
            rc = err;
            break;
        }
        if (rot == 0) {
            rc = JJ_OK;
            break;
        }
    }
    JJ_CUDA(launch_permute_columns(c->cplx, c->Gw[cur], c->ldw, (double *)G, ldg, c->m, n,
                                   c->d_perm, true, st));
    ++launches;
    JJ_CUDA(cudaStreamSynchronize(st));
    inf.kernel_launches = launches;
    c->solved = (rc == JJ_OK || rc == JJ_NOT_CONVERGED);
    return finish(rc);
}

int jjacobi_extract(jj_handle c, double *lambda, void *U, int64_t ldu, int32_t sort) {
    if (!c) return JJ_INVALID_ARG;
    if (!c->solved) return JJ_NOT_SOLVED;
    if (!lambda || (U && ldu < c->m)) return JJ_INVALID_ARG;
    cudaStream_t st = c->stream;
    const int64_t n = c->n;
    if (order_after_legacy(c) != JJ_OK) return JJ_CUDA_ERROR;
    cudaPointerAttributes at{};
    bool lam_dev = false;
    if (cudaPointerGetAttributes(&at, lambda) == cudaSuccess)
        lam_dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    cudaGetLastError();
    const int32_t *perm = nullptr;
    if (sort) {
        JJ_CUDA(launch_extract(c->cplx, (const double *)c->G_user, c->ldg_user, c->m, n,
                               c->d_Jorig, nullptr, c->d_lam, nullptr, 0, st));
        JJ_CUDA(cudaMemcpyAsync(c->h_lam, c->d_lam, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        JJ_CUDA(cudaStreamSynchronize(st));
        std::vector<int32_t> ord(n), rank(n);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int32_t a, int32_t b) { return c->h_lam[a] < c->h_lam[b]; });
        for (int64_t k = 0; k < n; ++k) rank[ord[k]] = (int32_t)k;
        JJ_CUDA(cudaMemcpyAsync(c->d_rank, rank.data(), n * sizeof(int32_t),
                                cudaMemcpyHostToDevice, st));
        JJ_CUDA(cudaStreamSynchronize(st));
        perm = c->d_rank;
    }
    double *lam_out = lam_dev ? lambda : c->d_lam;
    JJ_CUDA(launch_extract(c->cplx, (const double *)c->G_user, c->ldg_user, c->m, n, c->d_Jorig,
                           perm, lam_out, (double *)U, ldu, st));
    if (!lam_dev)
        JJ_CUDA(cudaMemcpyAsync(lambda, c->d_lam, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    JJ_CUDA(cudaStreamSynchronize(st));
    return JJ_OK;
}

int jjacobi_solve_host(jj_handle c, const void *G_host, int64_t ldg, const int8_t *J,
                       double *lambda_host, void *U_host, int64_t ldu, jj_info *info) {
    if (!c || !G_host || !J || !lambda_host || ldg < c->m || (U_host && ldu < c->m))
        return JJ_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    const size_t esz = (size_t)c->E * sizeof(double);
    const size_t bytes = (size_t)c->ldw * c->n * esz;
    if (!c->d_Ghost) JJ_CUDA(cudaMalloc(&c->d_Ghost, bytes));
    if (U_host && !c->d_Uhost) JJ_CUDA(cudaMalloc(&c->d_Uhost, bytes));
    cudaStream_t st = c->stream;
    JJ_CUDA(cudaMemcpy2DAsync(c->d_Ghost, c->ldw * esz, G_host, ldg * esz, c->m * esz, c->n,
                              cudaMemcpyHostToDevice, st));
    jj_info inf{};
    int rc = jjacobi_solve(c, c->d_Ghost, c->ldw, J, &inf);
    if (rc == JJ_OK || rc == JJ_NOT_CONVERGED) {
        const int rx = jjacobi_extract(c, c->d_lam, U_host ? c->d_Uhost : nullptr, c->ldw, 0);
        if (rx != JJ_OK) rc = rx;
    }
    if (rc == JJ_OK || rc == JJ_NOT_CONVERGED) {
        JJ_CUDA(cudaMemcpyAsync(lambda_host, c->d_lam, c->n * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
        if (U_host)
            JJ_CUDA(cudaMemcpy2DAsync(U_host, ldu * esz, c->d_Uhost, c->ldw * esz, c->m * esz,
                                      c->n, cudaMemcpyDeviceToHost, st));
        JJ_CUDA(cudaStreamSynchronize(st));
    }
    inf.status = rc;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return rc;
}

int jjacobi_solve_batched(jj_handle h, int32_t count, void *const *G, const int64_t *m,
                          const int64_t *n, const int64_t *ldg, const int8_t *const *J,
                          double *lambda_out, jj_info *infos) {
    (void)h; (void)count; (void)G; (void)m; (void)n; (void)ldg; (void)J; (void)lambda_out;
    (void)infos;
    return JJ_INVALID_ARG;
}

// ---------------------------------------------------------------------------
// Building blocks
// ---------------------------------------------------------------------------
static bool dt_ok(int32_t dtype) { return dtype == JJ_F64 || dtype == JJ_C128; }

int jjk_column_norms(int32_t dtype, const void *G, int64_t ld, int64_t m, int64_t n, double *d,
                     void *stream) {
    if (!dt_ok(dtype) || !G || !d || ld < m || m < 1 || n < 0) return JJ_INVALID_ARG;
    JJ_CUDA(launch_column_norms(dtype == JJ_C128, (const double *)G, ld, m, n, d,
                                (cudaStream_t)stream));
    return JJ_OK;
}

int jjk_plain_step(int32_t dtype, void *G, int64_t ld, int64_t m, int64_t n,
                   const int32_t *pairs, int32_t npairs, const int8_t *J, double *d, double tol,
                   unsigned long long *counters, void *stream) {
    if (!dt_ok(dtype) || !G || !pairs || !J || !d || !counters || ld < m || m < 1 || npairs < 0)
        return JJ_INVALID_ARG;
    JJ_CUDA(launch_plain_step(dtype == JJ_C128, (double *)G, ld, m, n, pairs, npairs, J, d,
                              tol > 0 ? tol : kDefaultTol, counters, (cudaStream_t)stream));
    return JJ_OK;
}

int jjk_gram(int32_t dtype, int32_t gemm, const void *G, int64_t ld, int64_t m,
             const int32_t *pairs, int32_t npairs, double *A, int32_t kmax, void *stream) {
    if (!dt_ok(dtype) || !G || !pairs || !A || ld < m || m < 1 || kmax < 1 || npairs < 0)
        return JJ_INVALID_ARG;
    const bool cplx = dtype == JJ_C128;
    cudaStream_t st = (cudaStream_t)stream;
    if (gemm == JJ_GEMM_OZAKI_FP16) {
        if (!ozaki_supported(cplx, kmax)) return JJ_INVALID_ARG;
        // Scratch from the stream-ordered allocator: column exponents of every
        // column the pairs touch and the int128 accumulators.
        int64_t ncols = 0;
        {
            std::vector<int32_t> hp((size_t)npairs * 4);
            JJ_CUDA(cudaMemcpyAsync(hp.data(), pairs, hp.size() * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st));
            JJ_CUDA(cudaStreamSynchronize(st));
            for (int q = 0; q < npairs; ++q)
                ncols = std::max<int64_t>(ncols, std::max(hp[4 * q] + hp[4 * q + 1],
                                                          hp[4 * q + 2] + hp[4 * q + 3]));
        }
        int32_t *cexp = nullptr;
        unsigned long long *acc = nullptr;
        JJ_CUDA(cudaMallocAsync((void **)&cexp, std::max<int64_t>(ncols, 1) * sizeof(int32_t), st));
        JJ_CUDA(cudaMallocAsync((void **)&acc, ozaki_gram_workspace_bytes(npairs, kmax, cplx), st));
        cudaError_t e = launch_colexp(cplx, (const double *)G, ld, m, ncols, cexp, st);
        if (e == cudaSuccess)
            e = launch_gram_ozaki(cplx, (const double *)G, ld, m, pairs, npairs, A, kmax, cexp, acc,
                                  ozaki_default_slices(true), nullptr, st);
        cudaFreeAsync(cexp, st);
        cudaFreeAsync(acc, st);
        JJ_CUDA(e);
        return JJ_OK;
    }
    JJ_CUDA(launch_gram(cplx, gemm, (const double *)G, ld, m, pairs, npairs, A, kmax, st));
    return JJ_OK;
}

int jjk_inner(int32_t dtype, double *A, double *W, int32_t kmax, const int32_t *pairs,
              int32_t npairs, const int8_t *J, double tol, int32_t inner_max_sweeps,
              int32_t inner_block_width, unsigned long long *counters, void *stream) {
    if (!dt_ok(dtype) || !A || !W || !pairs || !J || !counters || kmax < 1 || npairs < 0)
        return JJ_INVALID_ARG;
    JJ_CUDA(launch_inner(dtype == JJ_C128, A, W, kmax, pairs, npairs, J,
                         tol > 0 ? tol : kDefaultTol, inner_max_sweeps > 0 ? inner_max_sweeps : 30,
                         inner_block_width, counters, (cudaStream_t)stream));
    return JJ_OK;
}

int jjk_update(int32_t dtype, int32_t gemm, const void *Gs, void *Gd, int64_t ld, int64_t m,
               const int32_t *pairs, int32_t npairs, const double *W, int32_t kmax,
               void *stream) {
    if (!dt_ok(dtype) || !Gs || !Gd || !pairs || !W || ld < m || m < 1 || kmax < 1 || npairs < 0)
        return JJ_INVALID_ARG;
    const bool cplx = dtype == JJ_C128;
    if (gemm == JJ_GEMM_OZAKI_FP16) {
        if (!ozaki_supported(cplx, kmax)) return JJ_INVALID_ARG;
        cudaStream_t st = (cudaStream_t)stream;
        int64_t ncols = 0;
        {
            std::vector<int32_t> hp((size_t)npairs * 4);
            JJ_CUDA(cudaMemcpyAsync(hp.data(), pairs, hp.size() * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st));
            JJ_CUDA(cudaStreamSynchronize(st));
            for (int q = 0; q < npairs; ++q)
                ncols = std::max<int64_t>(ncols, std::max(hp[4 * q] + hp[4 * q + 1],
                                                          hp[4 * q + 2] + hp[4 * q + 3]));
        }
        int32_t *cexp = nullptr;
        JJ_CUDA(cudaMallocAsync((void **)&cexp, std::max<int64_t>(ncols, 1) * sizeof(int32_t), st));
        cudaError_t e = launch_colexp(cplx, (const double *)Gs, ld, m, ncols, cexp, st);
        if (e == cudaSuccess)
            e = launch_update_ozaki(cplx, (const double *)Gs, (double *)Gd, ld, m, pairs, npairs, W,
                                    kmax, cexp, ozaki_default_slices(false), nullptr, st);
        cudaFreeAsync(cexp, st);
        JJ_CUDA(e);
        return JJ_OK;
    }
    JJ_CUDA(launch_update(cplx, gemm, (const double *)Gs, (double *)Gd, ld, m, pairs, npairs, W,
                          kmax, (cudaStream_t)stream));
    return JJ_OK;
}

int jjk_extract(int32_t dtype, const void *G, int64_t ld, int64_t m, int64_t n, const int8_t *J,
                double *lambda, void *U, int64_t ldu, void *stream) {
    if (!dt_ok(dtype) || !G || !J || !lambda || ld < m || m < 1 || (U && ldu < m))
        return JJ_INVALID_ARG;
    JJ_CUDA(launch_extract(dtype == JJ_C128, (const double *)G, ld, m, n, J, nullptr, lambda,
                           (double *)U, ldu, (cudaStream_t)stream));
    return JJ_OK;
}

}  // extern "C"
