// Host driver and C ABI of libjjacobi: handle life cycle, workspaces, the
// sweep loop of Alg. 5.2 (parallel steps of the orderings of Sec. 4, one CUDA
// graph per sweep; the three-level forms launched directly), the convergence
// test (a sweep that applies no rotation, Sec. 5.3), extraction (the end of
// Alg. 5.2), the batched solve and the building-block entry points.
#include <algorithm>
#include <chrono>
#include <map>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "jj_common.cuh"

using namespace jj;

// Blocked sweep plan: one or more independent problems side by side in one
// work matrix (a single solve is a plan of one problem). Problem p owns the
// work columns [coff_p, coff_p + n_p), rows [0, m_p), with its own uniform
// block partition (3.3) and parallel ordering (Sec. 4); step t of the sweep
// runs the pairs of step t of every problem that has one.
struct Plan {
    int count = 0;
    std::vector<int64_t> pm, pn;        // shapes the plan was built for (caller order)
    std::vector<int> order;             // packing position -> caller index
    std::vector<int64_t> coff;          // by caller index: first work column
    std::vector<int> bw, nbl, psteps;   // by caller index
    int64_t ncols = 0, ldw = 0;
    int steps = 0, maxnp = 0, kmax = 0, slots = 0;
    std::vector<int> step_np, step_slot0;
    int block_param = 0;                // block_width the plan was built with
    // special pivot factor (3.9)-(3.11): the pass over every block's own Gram
    // at the start of a sweep (one single-block "pair" per block)
    int diag_np = 0, diag_slot0 = 0;
};

// Three-level form (Sec. 5.1, 3F): per outer step, the inner blocked method
// runs on X = [R_q; W_q] of every outer pair q at once (see jj_three.cu).
struct Three {
    bool on = false;
    int ib = 0, kmax_in = 0;
    int64_t ldx = 0, xcols = 0;
    int max_np = 0, max_slots = 0;
    std::vector<std::vector<int>> np, slot0;  // [outer step][inner step]
    std::vector<int> steps;                   // inner steps per inner sweep, by outer step
    std::vector<int64_t> tab0;                // first inner slot of each outer step
    int32_t *d_tab = nullptr, *d_prob = nullptr;
    double *X = nullptr, *Ain = nullptr, *Win = nullptr;
    int8_t *d_JX = nullptr;
    int32_t *d_fail = nullptr;
    int32_t *d_mod = nullptr, *d_clean = nullptr, *d_flags = nullptr, *d_sweep = nullptr;
    unsigned long long *d_cnt = nullptr, *h_cnt = nullptr, *d_rot = nullptr;
    unsigned long long *d_touched = nullptr;
    bool ozaki = false, ozaki_update = false;
    int32_t *d_cexp = nullptr, *d_cexp2 = nullptr, *d_wdexp = nullptr;
    unsigned long long *d_ozacc = nullptr;
    uint8_t *d_wdig = nullptr;
};

struct jj_ctx {
    jj_params p{};
    bool cplx = false;
    int E = 1;  // doubles per element
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t m = 0, n = 0;
    double tol = kDefaultTol;
    int max_sweeps = 60, inner_max_sweeps = 30;

    // plain (non-blocked) form
    bool blocked = false;
    int steps = 0, npairs = 0;
    int32_t *d_ppairs = nullptr;  // [steps][npairs][2]
    double *d_norm = nullptr;
    double *Gp = nullptr;         // work copy of G for the plain form
    int64_t ldp = 0;              // its leading dimension
    int32_t *d_pperm = nullptr;   // work column -> caller column
    int8_t *d_pJw = nullptr;      // J in work order
    cudaGraphExec_t graph_plain = nullptr;
    int launches_plain = 0;

    // blocked form
    Plan P;
    Three T3;
    bool plan_batched = false;
    int32_t *d_pairs = nullptr;   // [slots][4]: (offset_i, size_i, offset_j, size_j)
    int32_t *d_rows = nullptr;    // [slots] rows of the pair's problem (batched plans)
    int32_t *d_prob = nullptr;    // [slots] problem of the pair (batched plans)
    double *Gw = nullptr;         // work matrix (updated in place)
    double *Ablk = nullptr, *Wblk = nullptr;
    bool ozaki = false;                 // Gram on the tensor cores (fp16 digits)
    bool ozaki_update = false;          // update on the tensor cores too
    int32_t *d_mod = nullptr, *d_clean = nullptr, *d_flags = nullptr, *d_sweep = nullptr;
    uint8_t *d_wdig = nullptr;          // W-side digits of the digit update (per pair)
    int32_t *d_wdexp = nullptr;
    int oz_slices_gram = 8, oz_slices_update = kUdMaxSlices;
    long long *d_udscr = nullptr;       // scratch of the digit update (per persistent block)
    int ud_nctas = 0;
    int ud_tmax = 0;                    // widest pivot (64-position tiles per side) it serves
    unsigned long long wait_ns = 2000000000ull;  // bound of device-side waits
    int32_t *d_cexp = nullptr;          // column exponents (Ozaki Gram)
    unsigned long long *d_ozacc = nullptr;  // int128 Gram accumulators
    unsigned long long *d_prob_rot = nullptr, *h_prob_rot = nullptr;  // [2 count]
    unsigned long long *d_touched = nullptr;  // [pairs of a step][2] rotated-column masks
    // batched gather/scatter tables
    double **d_bptr = nullptr;
    int64_t *d_bld = nullptr, *d_brows = nullptr, *d_blamoff = nullptr;
    int32_t *d_bcolprob = nullptr;

    int32_t *d_perm = nullptr;    // work column -> caller column (within its problem)
    int32_t *d_rank = nullptr;    // extraction with sorting: column -> rank of its lambda
    int8_t *d_Jw = nullptr;       // J in work order
    int8_t *d_Jorig = nullptr;    // J in caller order (single solve)
    unsigned long long *d_cnt = nullptr, *h_cnt = nullptr;
    double *d_lam = nullptr;      // extraction temp
    double *h_lam = nullptr;      // pinned
    int64_t lam_cap = 0;
    double *d_Ghost = nullptr;    // device copy for jjacobi_solve_host (lazy)
    double *d_Uhost = nullptr;

    void *G_user = nullptr;
    int64_t ldg_user = 0;
    bool solved = false;
    int launches_per_sweep = 0;

    cudaGraphExec_t graph = nullptr;  // one sweep of the current plan
    double three_maxoff = 0.0;
    int tuned_bw = 0;                 // block width chosen (0: not yet tuned)
    std::map<int, int> class_bw;      // batched autotuner: size class -> block width
    cudaEvent_t ev_legacy = nullptr;  // orders a private stream after the legacy stream
    // profiling (params.profile): events around each kernel family of each step
    std::vector<cudaEvent_t> pev;
    double prof_ms[8] = {0};
    int64_t prof_n[8] = {0};
};

namespace {

// NVTX range for profilers (solve, sweep, extraction); header-only NVTX is a
// no-op unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

__global__ void sweep_begin_kernel(int32_t *sweep) { *sweep += 1; }

// On a CUDA error: optional report, then `return ret` (JJ_CUDA: JJ_CUDA_ERROR;
// entry points that fill a jj_info pass their own finishing expression)
#define JJ_CUDA_RET(call, ret)                                                          \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            if (getenv("JJACOBI_DEBUG"))                                                \
                fprintf(stderr, "jjacobi: %s failed: %s (%s:%d)\n", #call,             \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                    \
            return ret;                                                                 \
        }                                                                               \
    } while (0)
#define JJ_CUDA(call) JJ_CUDA_RET(call, JJ_CUDA_ERROR)

template <typename T>
cudaError_t dmalloc(T **p, size_t count) {
    return cudaMalloc((void **)p, count ? count * sizeof(T) : 1);
}

// A wait that ran out leaves its kernel's outputs incomplete, and later kernels
// of the sweep may then meet NaN or a failed Cholesky: the timeout is the cause.
int status_from_flags(unsigned long long err) {
    if (err & kErrTimeout) return JJ_DEVICE_TIMEOUT;
    if (err & kErrNonfinite) return JJ_NONFINITE;
    if (err & kErrNotPosdef) return JJ_NOT_POSDEF;
    return JJ_OK;
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

// Scratch of the digit update: one row block per persistent block (kept while
// the plan lives; shared by the outer and inner levels, which run in turn).
cudaError_t alloc_ud_scratch(jj_ctx *c, int tmax) {
    if (c->d_udscr && c->ud_tmax >= tmax) return cudaSuccess;
    if (c->d_udscr) cudaFree(c->d_udscr);
    c->d_udscr = nullptr;
    c->ud_nctas = ud_num_ctas();
    if (c->ud_nctas < 1) return cudaErrorInvalidDevice;
    c->ud_tmax = tmax;
    return cudaMalloc((void **)&c->d_udscr, ud_scratch_bytes(c->ud_nctas, tmax));
}

void free_plan(jj_ctx *c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    dfree(c->d_pairs);
    dfree(c->d_rows);
    dfree(c->d_prob);
    dfree(c->Gw);
    dfree(c->Ablk);
    dfree(c->Wblk);
    dfree(c->d_cexp);
    dfree(c->d_ozacc);
    dfree(c->d_wdig);
    dfree(c->d_wdexp);
    dfree(c->d_udscr);
    c->ud_tmax = 0;
    dfree(c->d_mod);
    dfree(c->d_clean);
    dfree(c->d_flags);
    dfree(c->d_sweep);
    dfree(c->d_prob_rot);
    dfree(c->d_touched);
    dfree(c->d_bptr);
    dfree(c->d_bld);
    dfree(c->d_brows);
    dfree(c->d_blamoff);
    dfree(c->d_bcolprob);
    dfree(c->d_perm);
    dfree(c->d_Jw);
    if (c->h_prob_rot) cudaFreeHost(c->h_prob_rot);
    c->h_prob_rot = nullptr;
    c->P = Plan();
    Three &T = c->T3;
    dfree(T.d_tab);
    dfree(T.d_prob);
    dfree(T.X);
    dfree(T.Ain);
    dfree(T.Win);
    dfree(T.d_JX);
    dfree(T.d_fail);
    dfree(T.d_mod);
    dfree(T.d_clean);
    dfree(T.d_flags);
    dfree(T.d_sweep);
    dfree(T.d_cnt);
    dfree(T.d_rot);
    dfree(T.d_touched);
    dfree(T.d_cexp);
    dfree(T.d_cexp2);
    dfree(T.d_wdexp);
    dfree(T.d_ozacc);
    dfree(T.d_wdig);
    if (T.h_cnt) cudaFreeHost(T.h_cnt);
    T = Three();
}

void free_ctx(jj_ctx *c) {
    if (!c) return;
    free_plan(c);
    if (c->graph_plain) cudaGraphExecDestroy(c->graph_plain);
    dfree(c->d_ppairs);
    dfree(c->Gp);
    dfree(c->d_pperm);
    dfree(c->d_pJw);
    dfree(c->d_norm);
    dfree(c->d_rank);
    dfree(c->d_Jorig);
    dfree(c->d_cnt);
    dfree(c->d_lam);
    dfree(c->d_Ghost);
    dfree(c->d_Uhost);
    if (c->h_cnt) cudaFreeHost(c->h_cnt);
    if (c->h_lam) cudaFreeHost(c->h_lam);
    if (c->ev_legacy) cudaEventDestroy(c->ev_legacy);
    for (auto e : c->pev) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// Capacity of the extraction buffers (device and pinned host) in doubles.
int ensure_lam(jj_ctx *c, int64_t count) {
    if (count <= c->lam_cap) return JJ_OK;
    dfree(c->d_lam);
    if (c->h_lam) cudaFreeHost(c->h_lam);
    c->h_lam = nullptr;
    c->lam_cap = 0;
    JJ_CUDA(dmalloc(&c->d_lam, (size_t)count));
    JJ_CUDA(cudaMallocHost((void **)&c->h_lam, (size_t)count * sizeof(double)));
    c->lam_cap = count;
    return JJ_OK;
}

// Block width of one problem of a batched plan when the caller fixes none:
// the widest block the digit kernels take (complex 16, real 32 columns), or
// 32 for the FP64 form, never wider than half the problem.
int batch_block_width(const jj_ctx *c, int64_t n) {
    int b = c->p.block_width > 0 ? c->p.block_width
                                 : (c->p.gemm == JJ_GEMM_FP64 ? 32 : (c->cplx ? 16 : 32));
    if (b > (n + 1) / 2) b = (int)((n + 1) / 2);
    return b < 1 ? 1 : b;
}

// Inner tables and buffers of the three-level form for the outer pair table
// `tab` of the current plan (Alg. 3.3 on R: inner blocks of ib columns,
// uniform partition (3.3) of each pivot, the plan's ordering, inner pairs of
// all outer pairs of a step side by side).
int build_three(jj_ctx *c, const std::vector<int32_t> &tab) {
    Plan &P = c->P;
    Three &T = c->T3;
    T.on = true;
    T.ib = c->p.inner_block_width;
    T.ldx = (2 * (int64_t)P.kmax + 3) & ~int64_t(3);
    std::vector<int32_t> itab, iprob;
    for (int t = 0; t < P.steps; ++t) {
        const int np = P.step_np[t], s0 = P.step_slot0[t];
        T.tab0.push_back((int64_t)itab.size() / 4);
        std::vector<std::vector<int32_t>> offs(np), sizes(np), sched(np);
        std::vector<int> nbl(np, 0), steps(np, 0);
        int smax = 0;
        // B strategy, steps after the first: only the off-diagonal block (Alg. 5.1)
        const bool cross = c->p.block_strategy == JJ_BLOCK_ORIENTED && t > 0;
        for (int q = 0; q < np; ++q) {
            // inner blocks respect the outer boundary (Alg. 3.4's assumption):
            // nb blocks of each outer block, uniform partitions (3.3)
            const int ni = tab[4 * (s0 + q) + 1], nj = tab[4 * (s0 + q) + 3];
            int nb = std::max((ni + T.ib - 1) / T.ib, (nj + T.ib - 1) / T.ib);
            nb = std::max(1, std::min(nb, std::min(ni, nj)));
            const int nb2 = 2 * nb;
            nbl[q] = nb2;
            sizes[q].resize(nb2);
            offs[q].resize(nb2 + 1);
            offs[q][0] = 0;
            for (int h = 0; h < 2; ++h) {
                const int w = h == 0 ? ni : nj, br = w % nb, nmin = w / nb;
                for (int l = 0; l < nb; ++l) {
                    sizes[q][h * nb + l] = l < br ? nmin + 1 : nmin;
                    T.kmax_in = std::max(T.kmax_in, 2 * (nmin + (br ? 1 : 0)));
                }
            }
            for (int l = 0; l < nb2; ++l) offs[q][l + 1] = offs[q][l] + sizes[q][l];
            if (cross) {
                // round rho pairs inner block r of block i with (r + rho) mod nb of block j
                steps[q] = nb;
                sched[q].resize((size_t)2 * nb * nb);
                for (int rho = 0; rho < nb; ++rho)
                    for (int r = 0; r < nb; ++r) {
                        sched[q][2 * ((size_t)rho * nb + r)] = r;
                        sched[q][2 * ((size_t)rho * nb + r) + 1] = nb + (r + rho) % nb;
                    }
            } else {
                sched[q].resize((size_t)2 * nb2 * nb2);
                steps[q] = schedule_pairs(nb2, c->p.order, 1, sched[q].data());
                if (steps[q] < 0) return JJ_INVALID_ARG;
            }
            smax = std::max(smax, steps[q]);
        }
        T.steps.push_back(smax);
        T.np.emplace_back();
        T.slot0.emplace_back();
        int slots = 0;
        for (int ti = 0; ti < smax; ++ti) {
            T.slot0[t].push_back(slots);
            int n_in = 0;
            for (int q = 0; q < np; ++q) {
                if (ti >= steps[q]) continue;
                const int npp = nbl[q] / 2;
                for (int u = 0; u < npp; ++u) {
                    const int i = sched[q][2 * ((size_t)ti * npp + u)];
                    const int j = sched[q][2 * ((size_t)ti * npp + u) + 1];
                    itab.push_back(q * P.kmax + offs[q][i]);
                    itab.push_back(sizes[q][i]);
                    itab.push_back(q * P.kmax + offs[q][j]);
                    itab.push_back(sizes[q][j]);
                    iprob.push_back(q);
                    ++n_in;
                }
            }
            T.np[t].push_back(n_in);
            slots += n_in;
            T.max_np = std::max(T.max_np, n_in);
        }
        T.max_slots = std::max(T.max_slots, slots);
    }
    if (c->p.block_strategy == JJ_BLOCK_ORIENTED && !inner_single_pass_supported(c->cplx, T.kmax_in))
        return JJ_INVALID_ARG;
    if (T.max_np > 65535) return JJ_INVALID_ARG;
    T.ozaki = ozaki_supported(c->cplx, T.kmax_in) && c->p.gemm != JJ_GEMM_FP64;
    T.ozaki_update = T.ozaki && c->p.gemm == JJ_GEMM_OZAKI_FP16;
    const size_t np = (size_t)std::max(P.maxnp, 1), npi = (size_t)std::max(T.max_np, 1);
    const size_t xcols = np * P.kmax;
    T.xcols = (int64_t)xcols;
    JJ_CUDA(dmalloc(&T.d_tab, itab.size()));
    JJ_CUDA(dmalloc(&T.d_prob, iprob.size()));
    JJ_CUDA(cudaMemcpy(T.d_tab, itab.data(), itab.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    JJ_CUDA(cudaMemcpy(T.d_prob, iprob.data(), iprob.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    JJ_CUDA(dmalloc(&T.X, (size_t)T.ldx * xcols * c->E));
    JJ_CUDA(dmalloc(&T.Ain, npi * T.kmax_in * T.kmax_in * c->E));
    JJ_CUDA(dmalloc(&T.Win, npi * T.kmax_in * T.kmax_in * c->E));
    JJ_CUDA(dmalloc(&T.d_JX, xcols));
    JJ_CUDA(dmalloc(&T.d_fail, np));
    JJ_CUDA(dmalloc(&T.d_mod, xcols));
    JJ_CUDA(dmalloc(&T.d_clean, (size_t)std::max(T.max_slots, 1)));
    JJ_CUDA(dmalloc(&T.d_flags, npi));
    JJ_CUDA(dmalloc(&T.d_sweep, 1));
    JJ_CUDA(dmalloc(&T.d_cnt, kNumCounters));
    JJ_CUDA(dmalloc(&T.d_rot, 2 * np));
    JJ_CUDA(dmalloc(&T.d_touched, 2 * npi));
    JJ_CUDA(cudaMallocHost((void **)&T.h_cnt, kNumCounters * sizeof(unsigned long long)));
    if (T.ozaki) {
        JJ_CUDA(dmalloc(&T.d_cexp, xcols));
        JJ_CUDA(dmalloc(&T.d_cexp2, xcols));
        JJ_CUDA(cudaMalloc((void **)&T.d_ozacc, ozaki_gram_workspace_bytes((int)npi, T.kmax_in, c->cplx)));
        if (T.ozaki_update) {
            const int ti = ud_max_tiles(c->cplx, T.kmax_in);
            JJ_CUDA(dmalloc(&T.d_wdig, npi * ti * ti * kUdMaxSlices * kUpdSliceBytes));
            JJ_CUDA(dmalloc(&T.d_wdexp, npi * ti * ti * 64));
            JJ_CUDA(alloc_ud_scratch(c, ti));
        }
    }
    return JJ_OK;
}

// Build the blocked plan for `count` problems (ms, ns in caller order; bws the
// block widths) and allocate every buffer that depends on it.
int build_plan(jj_ctx *c, int count, const int64_t *ms, const int64_t *ns, const int *bws,
               bool batched) {
    free_plan(c);
    Plan &P = c->P;
    P.count = count;
    P.pm.assign(ms, ms + count);
    P.pn.assign(ns, ns + count);
    P.block_param = c->p.block_width;
    P.order.resize(count);
    std::iota(P.order.begin(), P.order.end(), 0);
    // larger problems first: their pairs lead every step
    std::stable_sort(P.order.begin(), P.order.end(),
                     [&](int a, int b) { return ns[a] > ns[b]; });
    P.coff.assign(count, 0);
    P.bw.assign(count, 0);
    P.nbl.assign(count, 0);
    P.psteps.assign(count, 0);
    int64_t mmax = 1;
    for (int k = 0; k < count; ++k) {
        const int p = P.order[k];
        P.coff[p] = P.ncols;
        P.ncols += ns[p];
        mmax = std::max(mmax, ms[p]);
    }
    P.ldw = (mmax + 3) & ~int64_t(3);
    // per-problem partitions and orderings
    std::vector<std::vector<int32_t>> offs(count), sizes(count), sched(count);
    for (int p = 0; p < count; ++p) {
        const int64_t n = ns[p];
        if (n < 2) continue;  // one column: nothing to orthogonalise
        const int b = bws[p];
        int nbl = (int)(2 * ((n + 2 * (int64_t)b - 1) / (2 * (int64_t)b)));
        if (nbl > n - (n & 1)) nbl = (int)(n - (n & 1));
        if (nbl < 2) nbl = 2;
        P.bw[p] = b;
        P.nbl[p] = nbl;
        const int br = (int)(n % nbl), nmin = (int)(n / nbl);
        sizes[p].resize(nbl);
        offs[p].resize(nbl + 1);
        offs[p][0] = 0;
        for (int l = 0; l < nbl; ++l) {
            sizes[p][l] = l < br ? nmin + 1 : nmin;  // uniform partition (3.3)
            offs[p][l + 1] = offs[p][l] + sizes[p][l];
        }
        P.kmax = std::max(P.kmax, 2 * (nmin + (br ? 1 : 0)));
        sched[p].resize((size_t)2 * nbl * nbl);
        P.psteps[p] = schedule_pairs(nbl, c->p.order, 1, sched[p].data());
        if (P.psteps[p] < 0) return JJ_INVALID_ARG;
        P.steps = std::max(P.steps, P.psteps[p]);
    }
    if (P.kmax < 2) P.kmax = 2;
    std::vector<int32_t> tab, rows, prob;
    for (int t = 0; t < P.steps; ++t) {
        P.step_slot0.push_back(P.slots);
        int np = 0;
        for (int k = 0; k < count; ++k) {
            const int p = P.order[k];
            if (t >= P.psteps[p]) continue;
            const int npp = P.nbl[p] / 2;
            for (int q = 0; q < npp; ++q) {
                const int i = sched[p][2 * ((size_t)t * npp + q)];
                const int j = sched[p][2 * ((size_t)t * npp + q) + 1];
                tab.push_back((int32_t)(P.coff[p] + offs[p][i]));
                tab.push_back(sizes[p][i]);
                tab.push_back((int32_t)(P.coff[p] + offs[p][j]));
                tab.push_back(sizes[p][j]);
                rows.push_back((int32_t)ms[p]);
                prob.push_back(p);
                ++np;
            }
        }
        P.step_np.push_back(np);
        P.slots += np;
        P.maxnp = std::max(P.maxnp, np);
    }
    if (c->p.pivot_factor == JJ_PIVOT_SPECIAL && c->p.block_width != 0) {
        if (batched || count != 1 || c->p.block_strategy != JJ_FULL_BLOCK ||
            c->p.inner_block_width > 0)
            return JJ_INVALID_ARG;
        const int p = P.order[0];
        P.diag_slot0 = P.slots;
        P.diag_np = P.nbl[p];
        for (int l = 0; l < P.nbl[p]; ++l) {
            tab.push_back((int32_t)(P.coff[p] + offs[p][l]));
            tab.push_back(sizes[p][l]);
            tab.push_back((int32_t)(P.coff[p] + offs[p][l]));  // second block: none (size 0)
            tab.push_back(0);
            rows.push_back((int32_t)ms[p]);
            prob.push_back(p);
        }
        P.slots += P.diag_np;
        P.maxnp = std::max(P.maxnp, P.diag_np);
    }
    c->plan_batched = batched;
    // the pair kernels index pairs with blockIdx.y (at most 65535 per launch)
    if (P.maxnp > 65535) return JJ_INVALID_ARG;
    // three-level: the inner method blocked with inner_block_width columns
    const int ib = c->p.inner_block_width;
    const bool three = !batched && ib > 0 && P.kmax > 2 * ib;
    // digit forms (in the three-level form the outer level uses them where the
    // outer pivot fits the digit kernels; the choice applies to the inner level)
    const bool oz_ok = ozaki_supported(c->cplx, P.kmax);
    if (!three && (c->p.gemm == JJ_GEMM_OZAKI_FP16 || c->p.gemm == JJ_GEMM_OZAKI_GRAM) && !oz_ok)
        return JJ_INVALID_ARG;
    if (c->p.block_strategy == JJ_BLOCK_ORIENTED && !three &&
        !inner_single_pass_supported(c->cplx, P.kmax))
        return JJ_INVALID_ARG;
    if (P.diag_np > 0 && !inner_single_pass_supported(c->cplx, P.kmax)) return JJ_INVALID_ARG;
    c->ozaki = oz_ok && c->p.gemm != JJ_GEMM_FP64;
    c->ozaki_update = c->ozaki && c->p.gemm == JJ_GEMM_OZAKI_FP16;
    c->oz_slices_update = ozaki_default_slices(false);
    if (c->ozaki && c->p.ozaki_slices > 0) {
        if (c->p.ozaki_slices > kUdMaxSlices) return JJ_INVALID_ARG;
        c->oz_slices_update = c->p.ozaki_slices;
    }
    // device buffers
    const size_t np = (size_t)std::max(P.maxnp, 1);
    JJ_CUDA(dmalloc(&c->Gw, (size_t)P.ldw * P.ncols * c->E));
    JJ_CUDA(dmalloc(&c->Ablk, np * P.kmax * P.kmax * c->E));
    JJ_CUDA(dmalloc(&c->Wblk, np * P.kmax * P.kmax * c->E));
    JJ_CUDA(dmalloc(&c->d_mod, (size_t)P.ncols));
    JJ_CUDA(dmalloc(&c->d_clean, (size_t)P.slots));
    JJ_CUDA(dmalloc(&c->d_flags, np));
    JJ_CUDA(dmalloc(&c->d_sweep, 1));
    JJ_CUDA(dmalloc(&c->d_perm, (size_t)P.ncols));
    JJ_CUDA(dmalloc(&c->d_Jw, (size_t)P.ncols));
    JJ_CUDA(dmalloc(&c->d_touched, 2 * np));
    if (c->ozaki) {
        if (c->ozaki_update) {
            const int tm = ud_max_tiles(c->cplx, P.kmax);
            JJ_CUDA(dmalloc(&c->d_wdig, np * tm * tm * kUdMaxSlices * kUpdSliceBytes));
            JJ_CUDA(dmalloc(&c->d_wdexp, np * tm * tm * 64));
            JJ_CUDA(alloc_ud_scratch(c, tm));
        }
        JJ_CUDA(dmalloc(&c->d_cexp, (size_t)P.ncols));
        JJ_CUDA(cudaMalloc((void **)&c->d_ozacc, ozaki_gram_workspace_bytes((int)np, P.kmax, c->cplx)));
    }
    if (!tab.empty()) {
        JJ_CUDA(dmalloc(&c->d_pairs, tab.size()));
        JJ_CUDA(cudaMemcpy(c->d_pairs, tab.data(), tab.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    if (three) {
        const int r = build_three(c, tab);
        if (r != JJ_OK) return r;
    }
    if (batched) {
        JJ_CUDA(dmalloc(&c->d_prob_rot, 2 * (size_t)count));
        JJ_CUDA(cudaMallocHost((void **)&c->h_prob_rot, 2 * (size_t)count * sizeof(unsigned long long)));
        if (!rows.empty()) {
            JJ_CUDA(dmalloc(&c->d_rows, rows.size()));
            JJ_CUDA(dmalloc(&c->d_prob, prob.size()));
            JJ_CUDA(cudaMemcpy(c->d_rows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            JJ_CUDA(cudaMemcpy(c->d_prob, prob.data(), prob.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        }
        JJ_CUDA(dmalloc(&c->d_bptr, (size_t)count));
        JJ_CUDA(dmalloc(&c->d_bld, (size_t)count));
        JJ_CUDA(dmalloc(&c->d_brows, (size_t)count));
        JJ_CUDA(dmalloc(&c->d_blamoff, (size_t)count));
        JJ_CUDA(dmalloc(&c->d_bcolprob, (size_t)P.ncols));
        std::vector<int32_t> colprob(P.ncols);
        std::vector<int64_t> lamoff(count);
        int64_t off = 0;
        for (int p = 0; p < count; ++p) {
            lamoff[p] = off;
            off += ns[p];
            for (int64_t i = 0; i < ns[p]; ++i) colprob[P.coff[p] + i] = p;
        }
        JJ_CUDA(cudaMemcpy(c->d_bcolprob, colprob.data(), colprob.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        JJ_CUDA(cudaMemcpy(c->d_brows, ms, count * sizeof(int64_t), cudaMemcpyHostToDevice));
        JJ_CUDA(cudaMemcpy(c->d_blamoff, lamoff.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice));
    }
    return JJ_OK;
}

// Profiling: event slot of (step, point) and the kernel family between points.
struct ProfMark {
    int ev;
    int family;  // family timed from this mark to the next one of the step (-1: none)
};

// Record one sweep into the stream being captured (or run it directly).
int enqueue_sweep(jj_ctx *c, bool plain, int *launches, std::vector<ProfMark> *marks) {
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
    if (plain) {
        if (mark(4)) return JJ_CUDA_ERROR;
        JJ_CUDA(launch_column_norms(c->cplx, c->Gp, c->ldp, c->m, c->n, c->d_norm, st));
        ++L;
        if (mark(3)) return JJ_CUDA_ERROR;
        for (int t = 0; t < c->steps; ++t) {
            JJ_CUDA(launch_plain_step(c->cplx, c->Gp, c->ldp, c->m, c->n,
                                      c->d_ppairs + (size_t)t * c->npairs * 2, c->npairs, c->d_pJw,
                                      c->d_norm, c->tol, c->d_cnt, st));
            ++L;
        }
        if (mark(-1)) return JJ_CUDA_ERROR;
    } else {
        const Plan &P = c->P;
        if (c->d_prob_rot)
            JJ_CUDA(cudaMemsetAsync(c->d_prob_rot, 0, 2 * (size_t)P.count * sizeof(unsigned long long), st));
        sweep_begin_kernel<<<1, 1, 0, st>>>(c->d_sweep);
        JJ_CUDA(cudaGetLastError());
        ++L;
        const int64_t mrows = c->plan_batched ? P.ldw : c->m;
        // t = -1: the pass over every block's own Gram that opens a sweep of the
        // special pivot factor (3.9)-(3.11), which needs diagonal A_ii
        for (int t = P.diag_np > 0 ? -1 : 0; t < P.steps; ++t) {
            const bool diag = t < 0;
            const int np = diag ? P.diag_np : P.step_np[t], s0 = diag ? P.diag_slot0 : P.step_slot0[t];
            if (np == 0) continue;
            const int32_t *pr = c->d_pairs + (size_t)s0 * 4;
            StepCtl ctl;
            ctl.mod_step = c->d_mod;
            ctl.clean_at = c->d_clean;
            ctl.flags = c->d_flags;
            ctl.sweep = c->d_sweep;
            ctl.step = t;
            ctl.steps = P.steps;
            ctl.npairs = np;
            ctl.slot_base = s0;
            ctl.wait_ns = c->wait_ns;
            if (c->d_rows) ctl.rows = c->d_rows + s0;
            if (c->d_prob) {
                ctl.prob = c->d_prob + s0;
                ctl.prob_rot = c->d_prob_rot;
            }
            if (!c->ozaki_update) ctl.touched = c->d_touched;
            if (mark(0)) return JJ_CUDA_ERROR;
            if (c->ozaki) {
                JJ_CUDA(launch_colexp_pairs(c->cplx, c->Gw, P.ldw, mrows, pr, np, P.kmax, c->d_cexp,
                                            st, ctl));
                JJ_CUDA(launch_gram_ozaki(c->cplx, c->Gw, P.ldw, mrows, P.ncols, pr, np, c->Ablk, P.kmax, P.kmax / 2,
                                          c->d_cexp, c->d_ozacc, c->oz_slices_gram, c->d_cnt, st,
                                          ctl));
                L += 3;
            } else {
                JJ_CUDA(launch_gram(c->cplx, c->p.gemm, c->Gw, P.ldw, mrows, pr, np, c->Ablk,
                                    P.kmax, st, ctl));
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
            // the inner solve builds the W-side digits of a narrow pivot itself;
            // those of a wide one (more than one 64-position tile) follow it
            const bool wide = c->ozaki_update && ud_max_tiles(c->cplx, P.kmax) > 1;
            UpdDigits iud = ud;
            if (wide) iud.img = nullptr;
            const int pass = c->p.block_strategy == JJ_BLOCK_ORIENTED ? (t == 0 ? 2 : 1) : 0;
            JJ_CUDA(launch_inner(c->cplx, c->Ablk, c->Wblk, P.kmax, pr, np, c->d_Jw, c->tol,
                                 c->inner_max_sweeps, c->p.inner_block_width, c->d_cnt, st, ctl,
                                 iud, pass, P.diag_np > 0 && !diag));
            if (mark(2)) return JJ_CUDA_ERROR;
            if (wide) {
                JJ_CUDA(launch_wimage(c->cplx, c->Wblk, P.kmax, pr, np, c->d_cexp, ud, st, ctl));
                ++L;
            }
            if (c->ozaki_update)
                JJ_CUDA(launch_update_digits(c->cplx, c->Gw, c->Gw, P.ldw, mrows, P.ncols, pr, np, P.kmax, P.kmax / 2,
                                             c->d_cexp, ud, c->d_udscr, c->ud_nctas, c->d_cnt, st,
                                             ctl));
            else
                JJ_CUDA(launch_update(c->cplx, c->p.gemm, c->Gw, c->Gw, P.ldw, mrows, pr, np,
                                      c->Wblk, P.kmax, st, ctl));
            L += 2;
            if (mark(-1)) return JJ_CUDA_ERROR;
        }
        if (c->d_prob_rot)
            JJ_CUDA(cudaMemcpyAsync(c->h_prob_rot, c->d_prob_rot,
                                    2 * (size_t)P.count * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, st));
    }
    JJ_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, kNumCounters * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st));
    if (launches) *launches = L;
    return JJ_OK;
}

// One sweep of the three-level form (direct launches: the inner sweeps of each
// outer step stop on the host when one applies no rotation).
int run_three_sweep(jj_ctx *c, int *launches, std::vector<ProfMark> *marks) {
    cudaStream_t st = c->stream;
    const Plan &P = c->P;
    Three &T = c->T3;
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
    sweep_begin_kernel<<<1, 1, 0, st>>>(c->d_sweep);
    JJ_CUDA(cudaGetLastError());
    ++L;
    const int64_t xcols = (int64_t)std::max(P.maxnp, 1) * P.kmax;
    for (int t = 0; t < P.steps; ++t) {
        const int np = P.step_np[t], s0 = P.step_slot0[t];
        if (np == 0) continue;
        const int32_t *pr = c->d_pairs + (size_t)s0 * 4;
        StepCtl ctl;
        ctl.mod_step = c->d_mod;
        ctl.clean_at = c->d_clean;
        ctl.flags = c->d_flags;
        ctl.sweep = c->d_sweep;
        ctl.step = t;
        ctl.steps = P.steps;
        ctl.npairs = np;
        ctl.slot_base = s0;
        ctl.wait_ns = c->wait_ns;
        if (mark(0)) return JJ_CUDA_ERROR;
        if (c->ozaki) {
            JJ_CUDA(launch_colexp_pairs(c->cplx, c->Gw, P.ldw, c->m, pr, np, P.kmax, c->d_cexp, st, ctl));
            JJ_CUDA(launch_gram_ozaki(c->cplx, c->Gw, P.ldw, c->m, P.ncols, pr, np, c->Ablk, P.kmax, P.kmax / 2, c->d_cexp,
                                      c->d_ozacc, c->oz_slices_gram, c->d_cnt, st, ctl));
            L += 3;
        } else {
            JJ_CUDA(launch_gram(c->cplx, c->p.gemm, c->Gw, P.ldw, c->m, pr, np, c->Ablk, P.kmax, st, ctl));
            L += 1;
        }
        if (mark(1)) return JJ_CUDA_ERROR;
        // inner level: Cholesky into X = [R; I], then the blocked inner method
        JJ_CUDA(launch_three_cholesky(c->cplx, c->Ablk, P.kmax, pr, np, c->d_Jw, T.X, T.ldx, T.d_JX,
                                      T.d_fail, c->d_cnt, st, ctl));
        JJ_CUDA(cudaMemsetAsync(T.d_mod, 0xFF, xcols * sizeof(int32_t), st));
        JJ_CUDA(cudaMemsetAsync(T.d_clean, 0xFF, std::max(T.max_slots, 1) * sizeof(int32_t), st));
        JJ_CUDA(cudaMemsetAsync(T.d_flags, 0, std::max(T.max_np, 1) * sizeof(int32_t), st));
        JJ_CUDA(cudaMemsetAsync(T.d_sweep, 0, sizeof(int32_t), st));
        JJ_CUDA(cudaMemsetAsync(T.d_rot, 0, 2 * (size_t)std::max(P.maxnp, 1) * sizeof(unsigned long long), st));
        L += 1;
        const int ts = T.steps[t];
        // F: inner sweeps until one applies no rotation; B: one pass (the first
        // outer step of a sweep over every inner block pair, recursively
        // block-oriented; the other steps over the cross pairs only)
        const bool bo = c->p.block_strategy == JJ_BLOCK_ORIENTED;
        const int inner_sweeps = bo ? 1 : c->inner_max_sweeps;
        for (int sw = 1; sw <= inner_sweeps; ++sw) {
            JJ_CUDA(cudaMemsetAsync(T.d_cnt, 0, kNumCounters * sizeof(unsigned long long), st));
            sweep_begin_kernel<<<1, 1, 0, st>>>(T.d_sweep);
            JJ_CUDA(cudaGetLastError());
            ++L;
            for (int ti = 0; ti < ts; ++ti) {
                const int ni = T.np[t][ti];
                if (ni == 0) continue;
                const int64_t sl = T.tab0[t] + T.slot0[t][ti];
                const int32_t *ip = T.d_tab + sl * 4;
                StepCtl ic;
                ic.mod_step = T.d_mod;
                ic.clean_at = T.d_clean;
                ic.flags = T.d_flags;
                ic.sweep = T.d_sweep;
                ic.step = ti;
                ic.steps = ts;
                ic.npairs = ni;
                ic.slot_base = T.slot0[t][ti];
                ic.prob = T.d_prob + sl;
                ic.prob_rot = T.d_rot;
                ic.wait_ns = c->wait_ns;
                if (!T.ozaki_update) ic.touched = T.d_touched;
                UpdDigits ud;
                if (T.ozaki) {
                    // Gram exponents over the R rows; update exponents over R and W rows
                    JJ_CUDA(launch_colexp_pairs(c->cplx, T.X, T.ldx, P.kmax, ip, ni, T.kmax_in, T.d_cexp, st, ic));
                    JJ_CUDA(launch_gram_ozaki(c->cplx, T.X, T.ldx, P.kmax, T.xcols, ip, ni, T.Ain, T.kmax_in, T.kmax_in / 2,
                                              T.d_cexp, T.d_ozacc, c->oz_slices_gram, T.d_cnt, st, ic));
                    L += 3;
                    if (T.ozaki_update) {
                        JJ_CUDA(launch_colexp_pairs(c->cplx, T.X, T.ldx, 2 * P.kmax, ip, ni, T.kmax_in,
                                                    T.d_cexp2, st, ic));
                        ++L;
                        ud.img = T.d_wdig;
                        ud.wexp = T.d_wdexp;
                        ud.cexp = T.d_cexp2;
                        ud.slices = c->oz_slices_update;
                    }
                } else {
                    JJ_CUDA(launch_gram(c->cplx, c->p.gemm, T.X, T.ldx, P.kmax, ip, ni, T.Ain, T.kmax_in, st, ic));
                    L += 1;
                }
                const int ipass = bo ? ((t == 0 && ti == 0) ? 2 : 1) : 0;
                JJ_CUDA(launch_inner(c->cplx, T.Ain, T.Win, T.kmax_in, ip, ni, T.d_JX, c->tol,
                                     c->inner_max_sweeps, 0, T.d_cnt, st, ic, ud, ipass));
                if (T.ozaki_update)
                    JJ_CUDA(launch_update_digits(c->cplx, T.X, T.X, T.ldx, 2 * P.kmax, T.xcols, ip, ni,
                                                 T.kmax_in, T.kmax_in / 2, T.d_cexp2, ud, c->d_udscr, c->ud_nctas,
                                                 T.d_cnt, st, ic));
                else
                    JJ_CUDA(launch_update(c->cplx, c->p.gemm, T.X, T.X, T.ldx, 2 * P.kmax, ip, ni,
                                          T.Win, T.kmax_in, st, ic));
                L += 2;
            }
            JJ_CUDA(cudaMemcpyAsync(T.h_cnt, T.d_cnt, kNumCounters * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, st));
            JJ_CUDA(cudaStreamSynchronize(st));
            double mo;
            std::memcpy(&mo, &T.h_cnt[kCntMaxOff], sizeof(double));
            if (sw == 1) c->three_maxoff = std::max(c->three_maxoff, mo);
            if (T.h_cnt[kCntErr] & kErrTimeout) return JJ_DEVICE_TIMEOUT;
            if (T.h_cnt[kCntRot] == 0) break;
        }
        JJ_CUDA(launch_three_finish(c->cplx, T.X, T.ldx, P.kmax, pr, np, c->Wblk, T.d_rot, T.d_fail,
                                    c->d_cnt, st, ctl));
        ++L;
        if (mark(2)) return JJ_CUDA_ERROR;
        if (c->ozaki_update) {
            // the outer pivots' W-side digits, then the update
            UpdDigits oud;
            oud.img = c->d_wdig;
            oud.wexp = c->d_wdexp;
            oud.cexp = c->d_cexp;
            oud.slices = c->oz_slices_update;
            JJ_CUDA(launch_wimage(c->cplx, c->Wblk, P.kmax, pr, np, c->d_cexp, oud, st, ctl));
            JJ_CUDA(launch_update_digits(c->cplx, c->Gw, c->Gw, P.ldw, c->m, P.ncols, pr, np, P.kmax, P.kmax / 2,
                                         c->d_cexp, oud, c->d_udscr, c->ud_nctas, c->d_cnt, st, ctl));
            L += 1;
        }
        else
            JJ_CUDA(launch_update(c->cplx, c->p.gemm, c->Gw, c->Gw, P.ldw, c->m, pr, np, c->Wblk,
                                  P.kmax, st, ctl));
        L += 1;
        if (mark(-1)) return JJ_CUDA_ERROR;
    }
    JJ_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, kNumCounters * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st));
    JJ_CUDA(cudaStreamSynchronize(st));
    // the outer max off-diagonal: the largest first-inner-sweep value of the step
    double mo;
    std::memcpy(&mo, &c->h_cnt[kCntMaxOff], sizeof(double));
    mo = std::max(mo, c->three_maxoff);
    std::memcpy(&c->h_cnt[kCntMaxOff], &mo, sizeof(double));
    c->three_maxoff = 0.0;
    *launches += L;
    return JJ_OK;
}

int build_graph(jj_ctx *c, bool plain) {
    cudaGraphExec_t &ge = plain ? c->graph_plain : c->graph;
    if (ge) return JJ_OK;
    cudaGraph_t g = nullptr;
    JJ_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int L = 0;
    const int rc = enqueue_sweep(c, plain, &L, nullptr);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc != JJ_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return JJ_CUDA_ERROR;
    }
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return JJ_CUDA_ERROR;
    (plain ? c->launches_plain : c->launches_per_sweep) = L;
    return JJ_OK;
}

// One sweep: graph launch (or direct launches with profiling), then wait for
// the counters.
int run_sweep(jj_ctx *c, bool plain, int *launches) {
    cudaStream_t st = c->stream;
    if (!plain && c->T3.on) {
        std::vector<ProfMark> marks;
        const int r = run_three_sweep(c, launches, c->p.profile ? &marks : nullptr);
        if (r != JJ_OK) return r;
        for (size_t i = 0; i + 1 < marks.size(); ++i) {
            if (marks[i].family < 0) continue;
            float ms = 0.f;
            JJ_CUDA(cudaEventElapsedTime(&ms, c->pev[marks[i].ev], c->pev[marks[i + 1].ev]));
            c->prof_ms[marks[i].family] += ms;
            c->prof_n[marks[i].family] += 1;
        }
        return JJ_OK;
    }
    if (c->p.profile) {
        std::vector<ProfMark> marks;
        int L = 0;
        const int r = enqueue_sweep(c, plain, &L, &marks);
        if (r != JJ_OK) return r;
        JJ_CUDA(cudaStreamSynchronize(st));
        for (size_t i = 0; i + 1 < marks.size(); ++i) {
            if (marks[i].family < 0) continue;
            float ms = 0.f;
            JJ_CUDA(cudaEventElapsedTime(&ms, c->pev[marks[i].ev], c->pev[marks[i + 1].ev]));
            c->prof_ms[marks[i].family] += ms;
            c->prof_n[marks[i].family] += 1;
        }
        *launches += L;
    } else {
        const int r = build_graph(c, plain);
        if (r != JJ_OK) return r;
        JJ_CUDA(cudaGraphLaunch(plain ? c->graph_plain : c->graph, st));
        JJ_CUDA(cudaStreamSynchronize(st));
        *launches += plain ? c->launches_plain : c->launches_per_sweep;
    }
    return JJ_OK;
}

// Blocked-state reset before a solve: no block changed, no slot clean.
int reset_skip_state(jj_ctx *c) {
    cudaStream_t st = c->stream;
    JJ_CUDA(cudaMemsetAsync(c->d_mod, 0xFF, std::max<int64_t>(c->P.ncols, 1) * sizeof(int32_t), st));
    JJ_CUDA(cudaMemsetAsync(c->d_clean, 0xFF, std::max(c->P.slots, 1) * sizeof(int32_t), st));
    JJ_CUDA(cudaMemsetAsync(c->d_flags, 0, std::max(c->P.maxnp, 1) * sizeof(int32_t), st));
    JJ_CUDA(cudaMemsetAsync(c->d_sweep, 0, sizeof(int32_t), st));
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

// J-sorting permutation of one problem: columns with J = +1 first (Sec. 2.3).
bool j_sort(const int8_t *J, int64_t n, std::vector<int32_t> &perm) {
    perm.clear();
    perm.reserve(n);
    for (int64_t i = 0; i < n; ++i) {
        if (J[i] != 1 && J[i] != -1) return false;
        if (J[i] > 0) perm.push_back((int32_t)i);
    }
    for (int64_t i = 0; i < n; ++i)
        if (J[i] < 0) perm.push_back((int32_t)i);
    return true;
}

// Block widths the autotuner tries (block_width = JJ_BLOCK_AUTO): powers of two
// from 8 up to 32 for the digit forms (the widest whose inner solve stays in
// shared memory for both element types) and 64 for FP64, and not wider than a
// quarter of n (at least two block pairs per step).
std::vector<int> autotune_candidates(const jj_ctx *c) {
    std::vector<int> out;
    if (c->p.block_width > 0) {
        out.push_back(c->p.block_width);
        return out;
    }
    const bool digits = c->p.gemm == JJ_GEMM_OZAKI_FP16 || c->p.gemm == JJ_GEMM_OZAKI_GRAM;
    const int bmax = digits ? 32 : 64;
    for (int b = 8; b <= bmax; b *= 2)
        if (4 * (int64_t)b <= c->n || b == 8) out.push_back(b);
    return out;
}

// Autotuner: one sweep of every candidate block width on a scratch copy of G
// (the caller's G, J-sorted), timed with CUDA events around the sweep's graph;
// the fastest width is kept for this and every later solve of the handle.
int autotune(jj_ctx *c, const void *G, int64_t ldg, const std::vector<int32_t> &perm,
             const std::vector<int8_t> &Jw) {
    const std::vector<int> cand = autotune_candidates(c);
    cudaStream_t st = c->stream;
    cudaEvent_t e0, e1;
    JJ_CUDA(cudaEventCreate(&e0));
    JJ_CUDA(cudaEventCreate(&e1));
    float best = 0.f;
    int best_b = cand[0];
    const int64_t m = c->m, n = c->n;
    int rc = JJ_OK;
    for (int b : cand) {
        if ((rc = build_plan(c, 1, &m, &n, &b, false)) != JJ_OK) break;
        if (cudaMemcpyAsync(c->d_perm, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(c->d_Jw, Jw.data(), n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            launch_permute_columns(c->cplx, (const double *)G, ldg, c->Gw, c->P.ldw, m, n, c->d_perm,
                                   false, st) != cudaSuccess ||
            (rc = reset_skip_state(c)) != JJ_OK) {
            rc = rc ? rc : JJ_CUDA_ERROR;
            break;
        }
        float ms = 0.f;
        if (c->T3.on) {
            int L = 0;
            cudaEventRecord(e0, st);
            if ((rc = run_three_sweep(c, &L, nullptr)) != JJ_OK) break;
            cudaEventRecord(e1, st);
        } else {
            if ((rc = build_graph(c, false)) != JJ_OK) break;
            cudaEventRecord(e0, st);
            cudaGraphLaunch(c->graph, st);
            cudaEventRecord(e1, st);
        }
        if (cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = JJ_CUDA_ERROR;
            break;
        }
        if (best == 0.f || ms < best) {
            best = ms;
            best_b = b;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != JJ_OK) return rc;
    c->tuned_bw = best_b;
    return build_plan(c, 1, &m, &n, &best_b, false);
}

// The problems of a batched plan into the work matrix: J-sorted column order
// (Sec. 2.3), J in work order, gather, fresh skip state.
int batch_load(jj_ctx *c, int count, void *const *G, const int64_t *n, const int64_t *ldg,
               const int8_t *const *J) {
    const Plan &P = c->P;
    cudaStream_t st = c->stream;
    std::vector<int32_t> srccol(P.ncols), perm;
    std::vector<int8_t> Jw(P.ncols);
    for (int p = 0; p < count; ++p) {
        if (!j_sort(J[p], n[p], perm)) return JJ_INVALID_ARG;
        for (int64_t i = 0; i < n[p]; ++i) {
            srccol[P.coff[p] + i] = perm[i];
            Jw[P.coff[p] + i] = J[p][perm[i]];
        }
    }
    JJ_CUDA(cudaMemcpyAsync(c->d_perm, srccol.data(), P.ncols * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    JJ_CUDA(cudaMemcpyAsync(c->d_Jw, Jw.data(), P.ncols, cudaMemcpyHostToDevice, st));
    JJ_CUDA(cudaMemcpyAsync(c->d_bptr, G, count * sizeof(void *), cudaMemcpyHostToDevice, st));
    JJ_CUDA(cudaMemcpyAsync(c->d_bld, ldg, count * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    JJ_CUDA(launch_batch_gather(c->cplx, c->d_bptr, c->d_bld, c->d_brows, c->d_bcolprob, c->d_perm,
                                c->Gw, P.ldw, P.ncols, st));
    JJ_CUDA(cudaStreamSynchronize(st));  // the host tables above are temporaries
    return reset_skip_state(c);
}

// Size class of a batched problem for the autotuner: floor(log2 n).
int size_class(int64_t n) {
    int b = 0;
    while ((int64_t)2 << b <= n) ++b;
    return b;
}

// Batched autotuner (block_width = JJ_BLOCK_AUTO): for every size class
// present, one sweep of the sub-batch of that class is timed (CUDA events
// around the sweep's graph, inputs gathered into the work matrix, the caller's
// G untouched) with every candidate width, and the fastest is kept for the
// class, in this and later calls of the handle.
int batch_autotune(jj_ctx *c, int count, void *const *G, const int64_t *m, const int64_t *n,
                   const int64_t *ldg, const int8_t *const *J, std::vector<int> &bws) {
    std::map<int, std::vector<int>> classes;
    for (int p = 0; p < count; ++p) classes[size_class(n[p])].push_back(p);
    cudaStream_t st = c->stream;
    cudaEvent_t e0, e1;
    JJ_CUDA(cudaEventCreate(&e0));
    JJ_CUDA(cudaEventCreate(&e1));
    int rc = JJ_OK;
    const bool digits = c->p.gemm == JJ_GEMM_OZAKI_FP16 || c->p.gemm == JJ_GEMM_OZAKI_GRAM;
    const int bmax = digits ? 32 : 64;
    for (auto &kv : classes) {
        if (c->class_bw.count(kv.first)) continue;
        const std::vector<int> &idx = kv.second;
        std::vector<void *> g;
        std::vector<int64_t> mm, nn, ll;
        std::vector<const int8_t *> jj;
        int64_t nmax = 0;
        for (int p : idx) {
            g.push_back(G[p]);
            mm.push_back(m[p]);
            nn.push_back(n[p]);
            ll.push_back(ldg[p]);
            jj.push_back(J[p]);
            nmax = std::max(nmax, n[p]);
        }
        float best = 0.f;
        int best_b = 0;
        for (int b = 8; b <= bmax; b *= 2) {
            if (b > 8 && 2 * (int64_t)b > nmax) break;  // wider than the class's problems
            std::vector<int> w(idx.size());
            for (size_t i = 0; i < idx.size(); ++i) w[i] = (int)std::min<int64_t>(b, (nn[i] + 1) / 2);
            if ((rc = build_plan(c, (int)idx.size(), mm.data(), nn.data(), w.data(), true)) != JJ_OK ||
                (rc = batch_load(c, (int)idx.size(), g.data(), nn.data(), ll.data(), jj.data())) != JJ_OK ||
                (rc = build_graph(c, false)) != JJ_OK)
                break;
            float ms = 0.f;
            cudaEventRecord(e0, st);
            cudaGraphLaunch(c->graph, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = JJ_CUDA_ERROR;
                break;
            }
            if (best_b == 0 || ms < best) {
                best = ms;
                best_b = b;
            }
        }
        if (rc != JJ_OK) break;
        c->class_bw[kv.first] = best_b;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != JJ_OK) return rc;
    for (int p = 0; p < count; ++p)
        bws[p] = (int)std::min<int64_t>(c->class_bw[size_class(n[p])], (n[p] + 1) / 2);
    return JJ_OK;
}

// Batched solve, second phase: problems whose blocked sweeps failed because a
// pivot Gram block was not positive definite in working precision (its
// columns' scaled condition squared above ~1/u; the non-blocked method never
// forms a Gram block) are finished by the plain method (Algs. 3.1/3.2, round-
// robin over each problem's columns) from their current columns: every
// transformation applied so far was J-unitary, so the pencil is unchanged.
int batch_plain_finish(jj_ctx *c, const std::vector<int> &failed, std::vector<jj_info> &inf,
                       int *launches) {
    const Plan &P = c->P;
    cudaStream_t st = c->stream;
    std::vector<std::vector<int32_t>> sched(failed.size());
    std::vector<int> steps(failed.size());
    int smax = 0;
    for (size_t f = 0; f < failed.size(); ++f) {
        const int n = (int)P.pn[failed[f]];
        const int npl = n + (n & 1);
        sched[f].resize((size_t)npl * npl);
        steps[f] = schedule_pairs(npl, JJ_ORDER_ROUND_ROBIN, 1, sched[f].data());
        smax = std::max(smax, steps[f]);
    }
    std::vector<int32_t> tab;
    std::vector<int> np_t, off_t;
    for (int t = 0; t < smax; ++t) {
        off_t.push_back((int)tab.size() / 2);
        int np = 0;
        for (size_t f = 0; f < failed.size(); ++f) {
            const int p = failed[f], n = (int)P.pn[p], npl = n + (n & 1);
            if (t >= steps[f]) continue;
            for (int q = 0; q < npl / 2; ++q) {
                const int i = sched[f][2 * ((size_t)t * (npl / 2) + q)];
                const int j = sched[f][2 * ((size_t)t * (npl / 2) + q) + 1];
                if (i >= n || j >= n) continue;  // the dummy player of an odd order
                tab.push_back((int32_t)(P.coff[p] + i));
                tab.push_back((int32_t)(P.coff[p] + j));
                ++np;
            }
        }
        np_t.push_back(np);
    }
    int32_t *d_tab = nullptr;
    double *d_norm = nullptr;
    int rc = JJ_OK;
    auto done = [&](int r) {
        dfree(d_tab);
        dfree(d_norm);
        return r;
    };
    if (dmalloc(&d_tab, std::max<size_t>(tab.size(), 2)) != cudaSuccess ||
        dmalloc(&d_norm, (size_t)P.ncols) != cudaSuccess ||
        cudaMemcpy(d_tab, tab.data(), tab.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        return done(JJ_CUDA_ERROR);
    int status = JJ_NOT_CONVERGED, sweeps = 0;
    int64_t rot_total = 0;
    for (int sweep = 1; sweep <= c->max_sweeps; ++sweep) {
        sweeps = sweep;
        if (cudaMemsetAsync(c->d_cnt, 0, kNumCounters * sizeof(unsigned long long), st) != cudaSuccess ||
            launch_column_norms(c->cplx, c->Gw, P.ldw, P.ldw, P.ncols, d_norm, st) != cudaSuccess)
            return done(JJ_CUDA_ERROR);
        ++*launches;
        for (int t = 0; t < smax; ++t) {
            if (np_t[t] == 0) continue;
            if (launch_plain_step(c->cplx, c->Gw, P.ldw, P.ldw, P.ncols, d_tab + 2 * (size_t)off_t[t],
                                  np_t[t], c->d_Jw, d_norm, c->tol, c->d_cnt, st) != cudaSuccess)
                return done(JJ_CUDA_ERROR);
            ++*launches;
        }
        if (cudaMemcpyAsync(c->h_cnt, c->d_cnt, kNumCounters * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return done(JJ_CUDA_ERROR);
        rot_total += (int64_t)c->h_cnt[kCntRot];
        const int err = status_from_flags(c->h_cnt[kCntErr]);
        if (err != JJ_OK) {
            status = err;
            break;
        }
        if (c->h_cnt[kCntRot] == 0) {
            status = JJ_OK;
            break;
        }
    }
    for (int p : failed) {
        inf[p].status = status;
        inf[p].sweeps += sweeps;
        inf[p].rotations += rot_total;  // the plain phase's total over the failed problems
        inf[p].block_width = 0;         // finished by the non-blocked form
    }
    return done(rc);
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
    p->pivot_factor = JJ_PIVOT_CHOLESKY;
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

int jjacobi_factor(int32_t dtype, const void *H, int64_t ldh, int64_t n, double rank_tol, void *G,
                   int64_t ldg, int8_t *J, int32_t *perm, int8_t *pivot_size, int64_t *rank,
                   void *stream) {
    if (rank) *rank = 0;
    if ((dtype != JJ_F64 && dtype != JJ_C128) || !H || !G || !J || n < 1 || n > 65536 || ldh < n || ldg < n)
        return JJ_INVALID_ARG;
    const double tol = rank_tol > 0.0 ? rank_tol : 16.0 * (double)n * 1.1102230246251565404e-16;
    return frontend_factor(dtype == JJ_C128, (const double *)H, ldh, (int)n, tol, (double *)G, ldg,
                           J, perm, pivot_size, rank, 2000000000ull, (cudaStream_t)stream);
}

int jjacobi_set_wait_limit(jj_handle c, int64_t ns) {
    if (!c) return JJ_INVALID_ARG;
    const unsigned long long v = ns > 0 ? (unsigned long long)ns : 2000000000ull;
    if (v != c->wait_ns) {
        c->wait_ns = v;
        // captured sweeps carry the old bound in their kernel parameters
        if (c->graph) cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return JJ_OK;
}

int jjacobi_create(jj_handle *h, const jj_params *p) {
    if (!h) return JJ_INVALID_ARG;
    *h = nullptr;
    if (!p || p->n < 1 || p->m < p->n || (p->dtype != JJ_F64 && p->dtype != JJ_C128) ||
        p->block_width < JJ_BLOCK_AUTO || p->inner_block_width < 0 ||
        (p->order != JJ_ORDER_ROUND_ROBIN && p->order != JJ_ORDER_MODULUS) ||
        (p->gemm < JJ_GEMM_FP64 || p->gemm > JJ_GEMM_AUTO) || p->ozaki_slices < 0 ||
        (p->block_strategy != JJ_FULL_BLOCK && p->block_strategy != JJ_BLOCK_ORIENTED) ||
        (p->pivot_factor != JJ_PIVOT_CHOLESKY && p->pivot_factor != JJ_PIVOT_SPECIAL) ||
        p->n > (int64_t)1 << 30)
        return JJ_INVALID_ARG;
    jj_ctx *c = new jj_ctx();
    c->p = *p;
    c->cplx = p->dtype == JJ_C128;
    c->E = c->cplx ? 2 : 1;
    c->m = p->m;
    c->n = p->n;
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
    if (cudaMalloc(&c->d_rank, n * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_Jorig, n) != cudaSuccess ||
        cudaMalloc(&c->d_cnt, kNumCounters * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&c->h_cnt, kNumCounters * sizeof(unsigned long long)) != cudaSuccess ||
        ensure_lam(c, n) != JJ_OK)
        return fail(JJ_CUDA_ERROR);
    if (p->block_width == 0 || n < 4) {
        // plain: round-robin over single columns (n padded to even)
        c->blocked = false;
        const int npl = (int)(n + (n & 1));
        c->npairs = npl / 2;
        c->steps = npl - 1;
        c->ldp = (p->m + 3) & ~int64_t(3);
        std::vector<int32_t> tab;
        if (npl >= 2) {
            tab.resize((size_t)c->steps * c->npairs * 2);
            schedule_pairs(npl, JJ_ORDER_ROUND_ROBIN, 1, tab.data());
        }
        if (dmalloc(&c->Gp, (size_t)c->ldp * n * c->E) != cudaSuccess ||
            dmalloc(&c->d_norm, (size_t)n) != cudaSuccess ||
            dmalloc(&c->d_pperm, (size_t)n) != cudaSuccess ||
            dmalloc(&c->d_pJw, (size_t)n) != cudaSuccess)
            return fail(JJ_CUDA_ERROR);
        if (!tab.empty()) {
            if (dmalloc(&c->d_ppairs, tab.size()) != cudaSuccess ||
                cudaMemcpy(c->d_ppairs, tab.data(), tab.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(JJ_CUDA_ERROR);
        }
    } else {
        c->blocked = true;
        const int64_t m = p->m;
        const std::vector<int> cand = autotune_candidates(c);
        if (cand.empty()) return fail(JJ_INVALID_ARG);
        // a fixed width builds its plan now; the autotuner builds the first
        // candidate's (so that the workspaces exist) and picks at the first solve
        const int b = cand[0];
        const int rc = build_plan(c, 1, &m, &n, &b, false);
        if (rc != JJ_OK) return fail(rc);
        c->tuned_bw = p->block_width > 0 ? p->block_width : 0;
    }
    *h = c;
    return JJ_OK;
}

void jjacobi_destroy(jj_handle h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_ctx(h);
}

int jjacobi_solve(jj_handle c, void *G, int64_t ldg, const int8_t *J, jj_info *info) {
    NvtxRange range("jjacobi_solve");
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
    if (!j_sort(J, n, perm)) return finish(JJ_INVALID_ARG);
    if (c->blocked && c->tuned_bw > 0 && (c->plan_batched || c->P.count != 1)) {
        const int64_t m = c->m;
        const int b = c->tuned_bw;
        const int r = build_plan(c, 1, &m, &n, &b, false);
        if (r != JJ_OK) return finish(r);
    }
    std::vector<int8_t> Jw(n);
    for (int64_t i = 0; i < n; ++i) Jw[i] = J[perm[i]];
    c->solved = false;
    c->G_user = G;
    c->ldg_user = ldg;
    if (c->blocked && c->tuned_bw == 0) {
        if (order_after_legacy(c) != JJ_OK) return finish(JJ_CUDA_ERROR);
        const int r = autotune(c, G, ldg, perm, Jw);
        if (r != JJ_OK) return finish(r);
    }
    inf.block_width = c->blocked ? c->P.bw[0] : 0;
    inf.nbl = c->blocked ? c->P.nbl[0] : 0;
    inf.steps_per_sweep = c->blocked ? c->P.steps : c->steps;
    cudaStream_t st = c->stream;
    const bool plain = !c->blocked;
    double *W = plain ? c->Gp : c->Gw;
    const int64_t ldw = plain ? c->ldp : c->P.ldw;
    int32_t *dperm = plain ? c->d_pperm : c->d_perm;
    if (order_after_legacy(c) != JJ_OK) return finish(JJ_CUDA_ERROR);
    JJ_CUDA_RET(cudaMemcpyAsync(dperm, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice,
                                st),
                finish(JJ_CUDA_ERROR));
    JJ_CUDA_RET(cudaMemcpyAsync(plain ? c->d_pJw : c->d_Jw, Jw.data(), n, cudaMemcpyHostToDevice,
                                st),
                finish(JJ_CUDA_ERROR));
    JJ_CUDA_RET(cudaMemcpyAsync(c->d_Jorig, J, n, cudaMemcpyHostToDevice, st),
                finish(JJ_CUDA_ERROR));
    JJ_CUDA_RET(launch_permute_columns(c->cplx, (const double *)G, ldg, W, ldw, c->m, n, dperm,
                                       false, st),
                finish(JJ_CUDA_ERROR));
    if (c->blocked && reset_skip_state(c) != JJ_OK) return finish(JJ_CUDA_ERROR);
    int launches = 1;
    int rc = JJ_NOT_CONVERGED;
    for (int sweep = 1; sweep <= c->max_sweeps; ++sweep) {
        NvtxRange sweep_range("jj sweep");
        const int r = run_sweep(c, plain, &launches);
        if (r != JJ_OK) return finish(r);
        inf.sweeps = sweep;
        const unsigned long long rot = c->h_cnt[kCntRot];
        inf.rotations += (int64_t)rot;
        inf.pairs_evaluated += (int64_t)c->h_cnt[kCntPairs];
        inf.pairs_rotated += (int64_t)c->h_cnt[kCntPairsRot];
        double mo;
        std::memcpy(&mo, &c->h_cnt[kCntMaxOff], sizeof(double));
        inf.last_max_offdiag = mo;
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
    JJ_CUDA_RET(launch_permute_columns(c->cplx, W, ldw, (double *)G, ldg, c->m, n, dperm, true, st),
                finish(JJ_CUDA_ERROR));
    ++launches;
    JJ_CUDA_RET(cudaStreamSynchronize(st), finish(JJ_CUDA_ERROR));
    inf.kernel_launches = launches;
    c->solved = (rc == JJ_OK || rc == JJ_NOT_CONVERGED);
    return finish(rc);
}

int jjacobi_extract(jj_handle c, double *lambda, void *U, int64_t ldu, int32_t sort) {
    NvtxRange range("jjacobi_extract");
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
    const auto t0 = std::chrono::steady_clock::now();
    jj_info inf{};
    auto finish = [&](int rc) {
        inf.status = rc;
        inf.seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (info) *info = inf;
        return rc;
    };
    if (!c || !G_host || !J || !lambda_host || ldg < c->m || (U_host && ldu < c->m))
        return finish(JJ_INVALID_ARG);
    const size_t esz = (size_t)c->E * sizeof(double);
    const int64_t ldh = (c->m + 3) & ~int64_t(3);
    const size_t bytes = (size_t)ldh * c->n * esz;
    if (!c->d_Ghost) JJ_CUDA_RET(cudaMalloc(&c->d_Ghost, bytes), finish(JJ_CUDA_ERROR));
    if (U_host && !c->d_Uhost)
        JJ_CUDA_RET(cudaMalloc(&c->d_Uhost, bytes), finish(JJ_CUDA_ERROR));
    cudaStream_t st = c->stream;
    JJ_CUDA_RET(cudaMemcpy2DAsync(c->d_Ghost, ldh * esz, G_host, ldg * esz, c->m * esz, c->n,
                                  cudaMemcpyHostToDevice, st),
                finish(JJ_CUDA_ERROR));
    int rc = jjacobi_solve(c, c->d_Ghost, ldh, J, &inf);
    if (rc == JJ_OK || rc == JJ_NOT_CONVERGED) {
        const int rx = jjacobi_extract(c, c->d_lam, U_host ? c->d_Uhost : nullptr, ldh, 0);
        if (rx != JJ_OK) rc = rx;
    }
    if (rc == JJ_OK || rc == JJ_NOT_CONVERGED) {
        JJ_CUDA_RET(cudaMemcpyAsync(lambda_host, c->d_lam, c->n * sizeof(double),
                                    cudaMemcpyDeviceToHost, st),
                    finish(JJ_CUDA_ERROR));
        if (U_host)
            JJ_CUDA_RET(cudaMemcpy2DAsync(U_host, ldu * esz, c->d_Uhost, ldh * esz, c->m * esz,
                                          c->n, cudaMemcpyDeviceToHost, st),
                        finish(JJ_CUDA_ERROR));
        JJ_CUDA_RET(cudaStreamSynchronize(st), finish(JJ_CUDA_ERROR));
    }
    return finish(rc);
}

int jjacobi_solve_batched(jj_handle c, int32_t count, void *const *G, const int64_t *m,
                          const int64_t *n, const int64_t *ldg, const int8_t *const *J,
                          double *lambda_out, jj_info *infos) {
    NvtxRange range("jjacobi_solve_batched");
    const auto t0 = std::chrono::steady_clock::now();
    // an error before the per-problem results exist: every problem reports it
    auto fail = [&](int r) {
        if (infos)
            for (int p = 0; p < count; ++p) {
                infos[p] = jj_info{};
                infos[p].status = r;
                infos[p].seconds =
                    std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            }
        return r;
    };
    if (!c || count < 1 || !G || !m || !n || !ldg || !J) return fail(JJ_INVALID_ARG);
    int64_t ntot = 0;
    for (int p = 0; p < count; ++p) {
        if (!G[p] || !J[p] || n[p] < 1 || m[p] < n[p] || ldg[p] < m[p] || m[p] > c->m ||
            n[p] > c->n)
            return fail(JJ_INVALID_ARG);
        ntot += n[p];
    }
    if (ntot > ((int64_t)1 << 31) - 1) return fail(JJ_INVALID_ARG);
    c->solved = false;  // jjacobi_extract refers to single solves
    // plan: reuse when the shapes repeat
    const Plan &P0 = c->P;
    const bool same = c->plan_batched && P0.count == count && P0.block_param == c->p.block_width &&
                      std::equal(m, m + count, P0.pm.begin()) &&
                      std::equal(n, n + count, P0.pn.begin());
    if (!same) {
        std::vector<int> bws(count);
        if (c->p.block_width == JJ_BLOCK_AUTO) {
            if (order_after_legacy(c) != JJ_OK) return fail(JJ_CUDA_ERROR);
            const int r = batch_autotune(c, count, G, m, n, ldg, J, bws);
            if (r != JJ_OK) {
                free_plan(c);
                return fail(r);
            }
        } else {
            for (int p = 0; p < count; ++p) bws[p] = batch_block_width(c, n[p]);
        }
        const int r = build_plan(c, count, m, n, bws.data(), true);
        if (r != JJ_OK) {
            free_plan(c);
            return fail(r);
        }
    }
    const Plan &P = c->P;
    cudaStream_t st = c->stream;
    if (order_after_legacy(c) != JJ_OK) return fail(JJ_CUDA_ERROR);
    {
        const int r = batch_load(c, count, G, n, ldg, J);
        if (r != JJ_OK) return fail(r);
    }
    std::vector<jj_info> inf(count);
    std::vector<char> done(count, 0);
    int ndone = 0;
    for (int p = 0; p < count; ++p) {
        inf[p].status = JJ_NOT_CONVERGED;
        inf[p].block_width = P.bw[p];
        inf[p].nbl = P.nbl[p];
        inf[p].steps_per_sweep = P.psteps[p];
    }
    int launches = 2;
    int rc = JJ_OK;
    int64_t pairs_eval = 0, pairs_rot = 0;
    for (int sweep = 1; sweep <= c->max_sweeps && ndone < count; ++sweep) {
        NvtxRange sweep_range("jj sweep");
        const int r = run_sweep(c, false, &launches);
        if (r != JJ_OK) return fail(r);
        pairs_eval += (int64_t)c->h_cnt[kCntPairs];
        pairs_rot += (int64_t)c->h_cnt[kCntPairsRot];
        double mo;
        std::memcpy(&mo, &c->h_cnt[kCntMaxOff], sizeof(double));
        if (c->h_cnt[kCntErr] & kErrTimeout) {
            rc = JJ_DEVICE_TIMEOUT;
            break;
        }
        for (int p = 0; p < count; ++p) {
            if (done[p]) continue;
            const unsigned long long rot = c->h_prob_rot[2 * p];
            const int err = status_from_flags(c->h_prob_rot[2 * p + 1]);
            inf[p].sweeps = sweep;
            inf[p].rotations += (int64_t)rot;
            inf[p].last_max_offdiag = mo;
            if (err != JJ_OK || rot == 0) {
                inf[p].status = err != JJ_OK ? err : JJ_OK;
                done[p] = 1;
                ++ndone;
            }
        }
    }
    if (rc == JJ_OK) {
        std::vector<int> failed;
        for (int p = 0; p < count; ++p)
            if (inf[p].status == JJ_NOT_POSDEF) failed.push_back(p);
        if (!failed.empty()) {
            const int r = batch_plain_finish(c, failed, inf, &launches);
            if (r != JJ_OK) return fail(r);
        }
    }
    // scatter back, with the eigenvalues (lambda_out host or device)
    double *lam = nullptr;
    bool lam_dev = false;
    if (lambda_out) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, lambda_out) == cudaSuccess)
            lam_dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
        cudaGetLastError();
        if (!lam_dev && ensure_lam(c, P.ncols) != JJ_OK) return fail(JJ_CUDA_ERROR);
        lam = lam_dev ? lambda_out : c->d_lam;
    }
    JJ_CUDA_RET(launch_batch_scatter(c->cplx, c->Gw, P.ldw, c->d_bptr, c->d_bld, c->d_brows,
                                     c->d_bcolprob, c->d_perm, c->d_blamoff, c->d_Jw, lam, P.ncols,
                                     st),
                fail(JJ_CUDA_ERROR));
    if (lambda_out && !lam_dev)
        JJ_CUDA_RET(cudaMemcpyAsync(lambda_out, c->d_lam, P.ncols * sizeof(double),
                                    cudaMemcpyDeviceToHost, st),
                    fail(JJ_CUDA_ERROR));
    JJ_CUDA_RET(cudaStreamSynchronize(st), fail(JJ_CUDA_ERROR));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int worst = rc;
    for (int p = 0; p < count; ++p) {
        if (rc != JJ_OK) inf[p].status = rc;
        inf[p].seconds = secs;
        inf[p].kernel_launches = launches;
        inf[p].pairs_evaluated = pairs_eval;
        inf[p].pairs_rotated = pairs_rot;
        if (worst == JJ_OK && inf[p].status != JJ_OK) worst = inf[p].status;
        if (infos) infos[p] = inf[p];
    }
    return worst;
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
    if (!dt_ok(dtype) || !G || !pairs || !J || !d || !counters || ld < m || m < 1 || n < 0 ||
        npairs < 0)
        return JJ_INVALID_ARG;
    JJ_CUDA(launch_plain_step(dtype == JJ_C128, (double *)G, ld, m, n, pairs, npairs, J, d,
                              tol > 0 ? tol : kDefaultTol, counters, (cudaStream_t)stream));
    return JJ_OK;
}

int jjk_gram(int32_t dtype, int32_t gemm, const void *G, int64_t ld, int64_t m,
             const int32_t *pairs, int32_t npairs, double *A, int32_t kmax, void *stream) {
    if (!dt_ok(dtype) || !G || !pairs || !A || ld < m || m < 1 || kmax < 1 || npairs < 0 ||
        gemm < JJ_GEMM_FP64 || gemm > JJ_GEMM_AUTO)
        return JJ_INVALID_ARG;
    const bool cplx = dtype == JJ_C128;
    cudaStream_t st = (cudaStream_t)stream;
    // the Gram's form in each solver mode: digit products unless FP64; AUTO
    // takes them where the pivot width allows, FP64 otherwise
    bool digits = gemm != JJ_GEMM_FP64;
    if (digits && !ozaki_supported(cplx, kmax)) {
        if (gemm != JJ_GEMM_AUTO) return JJ_INVALID_ARG;
        digits = false;
    }
    if (digits) {
        // Scratch from the stream-ordered allocator: column exponents of every
        // column the pairs touch and the int128 accumulators.
        int64_t ncols = 0;
        int maxblk = 0;
        {
            std::vector<int32_t> hp((size_t)npairs * 4);
            JJ_CUDA(cudaMemcpyAsync(hp.data(), pairs, hp.size() * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st));
            JJ_CUDA(cudaStreamSynchronize(st));
            for (int q = 0; q < npairs; ++q) {
                ncols = std::max<int64_t>(ncols, std::max(hp[4 * q] + hp[4 * q + 1],
                                                          hp[4 * q + 2] + hp[4 * q + 3]));
                maxblk = std::max(maxblk, std::max(hp[4 * q + 1], hp[4 * q + 3]));
            }
        }
        int32_t *cexp = nullptr;
        unsigned long long *acc = nullptr;
        JJ_CUDA(cudaMallocAsync((void **)&cexp, std::max<int64_t>(ncols, 1) * sizeof(int32_t), st));
        if (cudaMallocAsync((void **)&acc, ozaki_gram_workspace_bytes(npairs, kmax, cplx), st) !=
            cudaSuccess) {
            cudaFreeAsync(cexp, st);
            return JJ_CUDA_ERROR;
        }
        cudaError_t e = launch_colexp(cplx, (const double *)G, ld, m, ncols, cexp, st);
        if (e == cudaSuccess)
            e = launch_gram_ozaki(cplx, (const double *)G, ld, m, ncols, pairs, npairs, A, kmax, maxblk, cexp, acc,
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
    if (!dt_ok(dtype) || !A || !W || !pairs || !J || !counters || kmax < 1 || npairs < 0 ||
        inner_block_width < 0)
        return JJ_INVALID_ARG;
    JJ_CUDA(launch_inner(dtype == JJ_C128, A, W, kmax, pairs, npairs, J,
                         tol > 0 ? tol : kDefaultTol, inner_max_sweeps > 0 ? inner_max_sweeps : 30,
                         inner_block_width, counters, (cudaStream_t)stream));
    return JJ_OK;
}

int jjk_update(int32_t dtype, int32_t gemm, const void *Gs, void *Gd, int64_t ld, int64_t m,
               const int32_t *pairs, int32_t npairs, const double *W, int32_t kmax,
               void *stream) {
    if (!dt_ok(dtype) || !Gs || !Gd || !pairs || !W || ld < m || m < 1 || kmax < 1 ||
        npairs < 0 || gemm < JJ_GEMM_FP64 || gemm > JJ_GEMM_AUTO)
        return JJ_INVALID_ARG;
    const bool cplx = dtype == JJ_C128;
    // the update runs on digit products only in the all-digit form; the
    // hybrid and AUTO forms keep it in FP64, as the solver does
    if (gemm == JJ_GEMM_OZAKI_FP16) {
        if (!ozaki_supported(cplx, kmax)) return JJ_INVALID_ARG;
        cudaStream_t st = (cudaStream_t)stream;
        int64_t ncols = 0;
        int maxblk = 0;
        {
            std::vector<int32_t> hp((size_t)npairs * 4);
            JJ_CUDA(cudaMemcpyAsync(hp.data(), pairs, hp.size() * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st));
            JJ_CUDA(cudaStreamSynchronize(st));
            for (int q = 0; q < npairs; ++q) {
                ncols = std::max<int64_t>(ncols, std::max(hp[4 * q] + hp[4 * q + 1],
                                                          hp[4 * q + 2] + hp[4 * q + 3]));
                maxblk = std::max(maxblk, std::max(hp[4 * q + 1], hp[4 * q + 3]));
            }
        }
        // Scratch from the stream-ordered allocator: column exponents, the W-side
        // digits of every pair, and the update's row blocks.
        const int nctas = ud_num_ctas();
        if (nctas < 1) return JJ_CUDA_ERROR;
        const int tm = ud_max_tiles(cplx, kmax);
        UpdDigits ud;
        ud.slices = kUdMaxSlices;
        int32_t *cexp = nullptr;
        long long *scr = nullptr;
        cudaError_t e = cudaMallocAsync((void **)&cexp, std::max<int64_t>(ncols, 1) * sizeof(int32_t), st);
        if (e == cudaSuccess)
            e = cudaMallocAsync((void **)&ud.img, (size_t)std::max(npairs, 1) * tm * tm * ud.slices * kUpdSliceBytes, st);
        if (e == cudaSuccess)
            e = cudaMallocAsync((void **)&ud.wexp, (size_t)std::max(npairs, 1) * tm * tm * 64 * sizeof(int32_t), st);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&scr, ud_scratch_bytes(nctas, tm), st);
        ud.cexp = cexp;
        if (e == cudaSuccess) e = launch_colexp(cplx, (const double *)Gs, ld, m, ncols, cexp, st);
        if (e == cudaSuccess) e = launch_wimage(cplx, W, kmax, pairs, npairs, cexp, ud, st);
        if (e == cudaSuccess)
            e = launch_update_digits(cplx, (const double *)Gs, (double *)Gd, ld, m, ncols, pairs, npairs,
                                     kmax, maxblk, cexp, ud, scr, nctas, nullptr, st);
        if (cexp) cudaFreeAsync(cexp, st);
        if (ud.img) cudaFreeAsync(ud.img, st);
        if (ud.wexp) cudaFreeAsync(ud.wexp, st);
        if (scr) cudaFreeAsync(scr, st);
        JJ_CUDA(e);
        return JJ_OK;
    }
    JJ_CUDA(launch_update(cplx, gemm, (const double *)Gs, (double *)Gd, ld, m, pairs, npairs, W,
                          kmax, (cudaStream_t)stream));
    return JJ_OK;
}

int jjk_extract(int32_t dtype, const void *G, int64_t ld, int64_t m, int64_t n, const int8_t *J,
                double *lambda, void *U, int64_t ldu, void *stream) {
    if (!dt_ok(dtype) || !G || !J || !lambda || ld < m || m < 1 || n < 0 || (U && ldu < m))
        return JJ_INVALID_ARG;
    JJ_CUDA(launch_extract(dtype == JJ_C128, (const double *)G, ld, m, n, J, nullptr, lambda,
                           (double *)U, ldu, (cudaStream_t)stream));
    return JJ_OK;
}

}  // extern "C"
