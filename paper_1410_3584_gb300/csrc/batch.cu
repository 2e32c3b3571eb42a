// Batched evaluation of many FP32 plans (different grids and kernels), replayed from a
// captured CUDA graph, in one of two forms, and the spread-tile autotuner.
//
// Persistent form: one launch of a persistent kernel over all plans' stages.
// Graph form: the plans' own stage launches (the single-plan kernels, each at its own CTA
// shape and occupancy) as the nodes of one graph, the plans spread over B parallel branches
// (largest first, each to the branch with the least work so far), so that small plans run
// side by side and the launch gaps between stages go away.
//
// Persistent form in detail:
// Work is a list of tasks (plan p, stage k, block i) in stage-major order; each CTA of the
// persistent grid takes the next ticket from a global counter.  Stage k of plan p may run
// once the last non-empty earlier stage of p has completed all its blocks: the CTA's first
// thread polls that stage's completion counter (acquire) with a bounded number of tries.
// Every ticket a task can wait on is smaller than its own, so the CTAs that hold them are
// already running: progress needs no co-residency guarantee.  A poll that runs out sets the
// device error word; every CTA then drains the remaining tickets without work and the host
// reports NLP_ERR_TIMEOUT.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fft_dev.cuh"
#include "launch.h"
#include "plan.h"
#include "spread_dev.cuh"

namespace nlp {

nlp_status eval_any(nlp_plan_s *p, const void *rho, void *phi);

enum { ST_R2C = 0, ST_A1, ST_A0, ST_INTERP, ST_SPREAD, ST_WSUM, ST_COMBINE, ST_B0, ST_B1, ST_C2R, kStages };
constexpr int kRegLines = 16;          // lines (pairs) per register-engine FFT task: 16 x 16 threads
constexpr int kCombTiles = 16;         // combine tiles of G per task

struct BatchItem {
    DevPlan<float> P;
    DevPlan<float> Pr;       // as P with G = F: the inverse passes after the first read and write F
    StridedDesc a1, a0, b0, b1;
    int nb_r2c, nb_a1, nb_a0, nb_c2r;
    int ntask[kStages];
    int dep[kStages];        // stage this stage waits for (-1: none)
    int spread_warp;         // 1: one-warp-per-piece kernel (W = 8), 0: generic kernel
    int reg_fft;             // 1: FFT passes on the register radix engine (16 lines per task)
};

struct BatchArgs {
    const BatchItem *items;
    int nitems;
    const int *off;          // kStages * nitems + 1 ticket offsets (stage-major or item-major)
    int item_major;          // 0: all items' stage k before any stage k + 1; 1: item by item
    int total;
    int *ticket;             // [0] ticket counter, [1] error word
    int *done;               // nitems * kStages completion counters
    long long spin_limit;    // polls before giving up
    const float *const *rho; // per item (pointer table)
    float *const *phi;
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(256, 2) k_batch_persistent(BatchArgs A) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_task, s_ok;
    for (;;) {
        __syncthreads();   // the previous task's shared memory is no longer in use
        if (threadIdx.x == 0) s_task = atomicAdd(A.ticket, 1);
        __syncthreads();
        const int t = s_task;
        if (t >= A.total) break;
        // decode (stage, item): last offset <= t
        int lo = 0, hi = kStages * A.nitems;   // off[lo] <= t < off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (A.off[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int k = A.item_major ? lo % kStages : lo / A.nitems;
        const int p = A.item_major ? lo / kStages : lo % A.nitems, i = t - A.off[lo];
        const BatchItem &B = A.items[p];
        if (threadIdx.x == 0) {
            int ok = ld_acquire(A.ticket + 1) == 0;
            const int d = B.dep[k];
            if (ok && d >= 0) {
                const int *cnt = A.done + p * kStages + d;
                const int need = B.ntask[d];
                long long n = 0;
                while (ld_acquire(cnt) < need) {
                    if (++n > A.spin_limit || ld_acquire(A.ticket + 1) != 0) {
                        ok = 0;
                        atomicExch(A.ticket + 1, 1);
                        break;
                    }
                    __nanosleep(64);
                }
                __threadfence();   // as a grid barrier: the stage's writes are visible to this CTA
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) continue;   // drain: tickets are still taken so every CTA reaches the end
        switch (k) {
            case ST_R2C:
                // two shared buffers (the persistent kernel sizes its shared memory for every stage)
                if (B.reg_fft) fwd_r2c_reg_block<float, kRegLines, false>(A.rho[p], B.P, i, smraw);
                else fwd_r2c_block<float>(A.rho[p], B.P, B.nb_r2c, i, smraw);
                break;
            case ST_A1:
                if (B.reg_fft) fft_cols_block<float, -1, kRegLines>(B.P.F, B.a1, B.P.len[1], i, smraw);
                else fft_strided_block<float, -1>(B.P.F, B.a1, B.P.len[1], B.nb_a1, i, smraw);
                break;
            case ST_A0:
                if (B.reg_fft) fft_cols_block<float, -1, kRegLines>(B.P.F, B.a0, B.P.len[0], i, smraw);
                else fft_strided_block<float, -1>(B.P.F, B.a0, B.P.len[0], B.nb_a0, i, smraw);
                break;
            case ST_INTERP:
                interp_warp_block<8, kWarpNB>(B.P, i, smraw);
                break;
            case ST_SPREAD:
                if (B.spread_warp) spread_warp_block<8, kWarpNB>(B.P, i, smraw);
                else spread_generic_block<float>(B.P, i, smraw);
                break;
            case ST_WSUM:
                window_sum_block<float>(B.P, i, (long long *)smraw);
                break;
            case ST_COMBINE: {
                CombStage *cst = (CombStage *)smraw;
                const int64_t t1 = min((int64_t)(i + 1) * kCombTiles, B.P.cmb_nact);
                // 256 threads: a 3D tile is 2 cells per thread, a 2D tile one
                for (int64_t t = (int64_t)i * kCombTiles; t < t1; ++t) {
                    if (B.P.cmb_t[0] == 1) combine_block<float, 1>(B.P, B.P.cmb_act[t], cst);
                    else combine_block<float, 2>(B.P, B.P.cmb_act[t], cst);
                }
                break;
            }
            case ST_B0:
                if (B.reg_fft) fft_cols_block<float, +1, kRegLines>(B.P.G, B.b0, B.P.len[0], i, smraw);
                else fft_strided_block<float, +1>(B.P.G, B.b0, B.P.len[0], B.nb_a0, i, smraw);
                break;
            case ST_B1: {
                // 3D: in place on F (the first inverse pass wrote it); 2D: G -> F
                cpx<float> *src = B.ntask[ST_B0] > 0 ? B.P.F : B.P.G;
                if (B.reg_fft) fft_cols_block<float, +1, kRegLines>(src, B.b1, B.P.len[1], i, smraw);
                else fft_strided_block<float, +1>(src, B.b1, B.P.len[1], B.nb_a1, i, smraw);
                break;
            }
            case ST_C2R:
                if (B.reg_fft) inv_c2r_reg_block<float, kRegLines>(A.phi[p], B.Pr, i, smraw);
                else inv_c2r_block<float>(A.phi[p], B.Pr, B.nb_c2r, i, smraw);
                break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(A.done + p * kStages + k, 1);
        }
    }
}

// lines per block of one FFT pass, as the single-plan launchers choose it
static int lpb(int N) {
    const int budget = 160 * 1024 / (int)sizeof(cpx<float>);
    int nb = 16;
    while (nb > 1 && 2 * N * (nb + 1) + N > budget) nb >>= 1;
    return nb;
}
static size_t fft_bytes(int N, int nb) { return sizeof(cpx<float>) * ((size_t)N + 2 * (size_t)N * (nb + 1)); }

}  // namespace nlp

using namespace nlp;

struct nlp_batch_s {
    cudaStream_t stream = nullptr;
    int count = 0;
    std::vector<nlp_plan> plans;
    std::vector<void *> allocs;
    BatchItem *d_items = nullptr;
    int *d_off = nullptr, *d_ctr = nullptr;   // ctr: [ticket, err] + done counters
    const float **d_rho = nullptr;
    float **d_phi = nullptr;
    void **h_ptrs = nullptr;                  // pinned: rho[count], phi[count]
    int *h_err = nullptr;                     // pinned copy of the error word
    size_t ctr_bytes = 0;
    int total = 0, grid = 0;
    int item_major = 0;   // ticket order (see BatchArgs)
    size_t smem = 0;
    long long spin_limit = 1 << 24;
    std::vector<BatchItem> items;
    std::vector<int> off;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev = nullptr;
    bool pending = false;
    // graph form: branches, their streams and fork/join events, and the graph of the plans'
    // stage launches for the pointers it was captured with
    int mode = NLP_BATCH_PERSISTENT, branches = 1;
    std::vector<cudaStream_t> bstreams;
    std::vector<cudaEvent_t> bevents;   // [0] fork, [1 + i] join of branch i
    cudaGraph_t sgraph = nullptr;
    cudaGraphExec_t sexec = nullptr;
    std::vector<const void *> cap_ptrs;   // rho[count], phi[count] of the captured launches
};

// Ticket offsets in the batch's order: stage-major (all items' stage k, then stage k + 1: every
// stage has the whole batch's parallelism) or item-major (item p's stages in sequence, then item
// p + 1: an item's spectra stay in L2 between its stages).
static void batch_offsets(nlp_batch_s *b) {
    const int count = b->count;
    b->off.assign((size_t)kStages * count + 1, 0);
    int t = 0;
    for (int a = 0; a < (b->item_major ? count : kStages); ++a)
        for (int c = 0; c < (b->item_major ? kStages : count); ++c) {
            const int k = b->item_major ? c : a, p = b->item_major ? a : c;
            b->off[b->item_major ? (size_t)p * kStages + k : (size_t)k * count + p] = t;
            t += b->items[p].ntask[k];
        }
    b->off[(size_t)kStages * count] = t;
    b->total = t;
}

static nlp_status batch_graph(nlp_batch_s *b) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    BatchArgs A;
    A.items = b->d_items;
    A.nitems = b->count;
    A.off = b->d_off;
    A.item_major = b->item_major;
    A.total = b->total;
    A.ticket = b->d_ctr;
    A.done = b->d_ctr + 2;
    A.spin_limit = b->spin_limit;
    A.rho = b->d_rho;
    A.phi = b->d_phi;
    cudaStream_t st = b->stream;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return NLP_ERR_CUDA;
    cudaMemcpyAsync(b->d_rho, b->h_ptrs, sizeof(void *) * 2 * b->count, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(b->d_ctr, 0, b->ctr_bytes, st);
    k_batch_persistent<<<b->grid, 256, b->smem, st>>>(A);
    cudaMemcpyAsync(b->h_err, b->d_ctr + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamEndCapture(st, &b->graph) != cudaSuccess) return NLP_ERR_CUDA;
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return NLP_ERR_CUDA;
    return NLP_OK;
}

// The graph form: the plans' single-plan evaluations captured from B forked streams.  The
// launches take rho and phi as arguments, so the graph is captured again (and the
// instantiated graph updated in place) when the pointers change.
static nlp_status batch_stage_graph(nlp_batch_s *b, const void *const *rho, void *const *phi) {
    const int B = std::max(1, std::min(b->branches, b->count));
    while ((int)b->bstreams.size() < B) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return NLP_ERR_CUDA;
        b->bstreams.push_back(s);
    }
    while ((int)b->bevents.size() < B + 1) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return NLP_ERR_CUDA;
        b->bevents.push_back(e);
    }
    // plans to branches: largest fine grid first, each to the least loaded branch
    std::vector<int> order(b->count), branch(b->count);
    std::vector<double> load(B, 0.0), work(b->count);
    for (int p = 0; p < b->count; ++p) {
        const DevPlan<float> &D = b->plans[p]->pf;
        work[p] = (double)D.nf[0] * D.nf[1] * D.nf[2];
        order[p] = p;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    for (int p : order) {
        const int br = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        branch[p] = br;
        load[br] += work[p];
    }
    cudaStream_t st = b->stream;
    // relaxed capture: the launchers may set kernel attributes on their first use
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) return NLP_ERR_CUDA;
    nlp_status s = NLP_OK;
    if (cudaEventRecord(b->bevents[0], st) != cudaSuccess) s = NLP_ERR_CUDA;
    for (int br = 0; br < B && !s; ++br)
        if (cudaStreamWaitEvent(b->bstreams[br], b->bevents[0], 0) != cudaSuccess) s = NLP_ERR_CUDA;
    for (int p : order) {
        if (s) break;
        nlp_plan_s *pl = b->plans[p];
        const cudaStream_t keep = pl->stream;
        const int keep_timing = pl->timing;
        pl->stream = b->bstreams[branch[p]];
        pl->timing = 0;
        s = eval_any(pl, rho[p], phi[p]);
        pl->stream = keep;
        pl->timing = keep_timing;
    }
    for (int br = 0; br < B && !s; ++br)
        if (cudaEventRecord(b->bevents[1 + br], b->bstreams[br]) != cudaSuccess ||
            cudaStreamWaitEvent(st, b->bevents[1 + br], 0) != cudaSuccess)
            s = NLP_ERR_CUDA;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &g);
    if (s || ec != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return s ? s : NLP_ERR_CUDA;
    }
    bool updated = false;
    if (b->sexec) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(b->sexec, g, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(b->sexec);
            b->sexec = nullptr;
        }
    }
    if (!updated && cudaGraphInstantiate(&b->sexec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        b->sexec = nullptr;
        return NLP_ERR_CUDA;
    }
    if (b->sgraph) cudaGraphDestroy(b->sgraph);
    b->sgraph = g;
    b->cap_ptrs.assign(2 * (size_t)b->count, nullptr);
    for (int p = 0; p < b->count; ++p) {
        b->cap_ptrs[p] = rho[p];
        b->cap_ptrs[b->count + p] = phi[p];
    }
    return NLP_OK;
}

static void drop_stage_graph(nlp_batch_s *b) {
    if (b->sexec) cudaGraphExecDestroy(b->sexec);
    if (b->sgraph) cudaGraphDestroy(b->sgraph);
    b->sexec = nullptr;
    b->sgraph = nullptr;
    b->cap_ptrs.clear();
}

extern "C" {

void nlp_batch_destroy(nlp_batch b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_stage_graph(b);
    for (cudaStream_t s : b->bstreams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->bevents) cudaEventDestroy(e);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ev) cudaEventDestroy(b->ev);
    for (void *a : b->allocs) cudaFree(a);
    if (b->h_ptrs) cudaFreeHost(b->h_ptrs);
    if (b->h_err) cudaFreeHost(b->h_err);
    delete b;
}

nlp_status nlp_batch_create(const nlp_plan *plans, int count, void *stream, nlp_batch *out) {
    if (!out || !plans || count < 1 || count > 4096) return NLP_ERR_INVALID_ARG;
    *out = nullptr;
    for (int p = 0; p < count; ++p) {
        if (!plans[p]) return NLP_ERR_INVALID_ARG;
        if (plans[p]->prec != NLP_FP32 || plans[p]->kernel == NLP_POISSON_2D || plans[p]->opts.method != 0)
            return NLP_ERR_UNSUPPORTED;
        // register kernels other than the one-warp-per-piece kernel (FP32 tolerances below
        // 1e-6) run as their own launches only
        const DevPlan<float> &D = plans[p]->pf;
        if (D.sub_T > 0 && !(D.sub_T == 2 && D.w == 7)) return NLP_ERR_UNSUPPORTED;
    }
    nlp_batch_s *b = new (std::nothrow) nlp_batch_s();
    if (!b) return NLP_ERR_OOM;
    b->stream = (cudaStream_t)stream;
    b->count = count;
    b->plans.assign(plans, plans + count);
    b->items.resize(count);
    size_t smem = 0;
    for (int p = 0; p < count; ++p) {
        nlp_plan_s *pl = plans[p];
        const DevPlan<float> &D = pl->pf;
        BatchItem &B = b->items[p];
        memset(&B, 0, sizeof(B));
        B.P = D;
        const bool three = pl->grid.dim == 3;
        const int64_t nh = D.nh;
        B.a1.n_in = D.n[1]; B.a1.n_out = D.nf[1]; B.a1.es = nh; B.a1.ncol = (int)nh;
        B.a1.nouter = three ? D.n[0] : 1; B.a1.os = (int64_t)D.nf[1] * nh;
        B.a1.outer_map_n = three ? D.n[0] : 0; B.a1.outer_map_N = D.nf[0];
        B.b1 = B.a1; B.b1.n_in = D.nf[1]; B.b1.n_out = D.n[1];
        B.b1.out = D.F;
        if (three) {
            B.a0.n_in = D.n[0]; B.a0.n_out = D.nf[0]; B.a0.es = (int64_t)D.nf[1] * nh; B.a0.ncol = (int)nh;
            B.a0.nouter = D.nf[1]; B.a0.os = nh;
            B.b0 = B.a0; B.b0.n_in = D.nf[0]; B.b0.n_out = D.n[0];
            B.b0.out = D.F;
        }
        B.Pr = D;
        B.Pr.G = D.F;
        // register-engine FFT tasks where every axis has its factorisation and the task's shared
        // memory stays within the budget of the single-plan launchers' widest choice
        const size_t kRegBudget = 112 * 1024;
        B.reg_fft = D.len[2].nrad_reg > 0 && D.len[1].nrad_reg > 0 && (!three || D.len[0].nrad_reg > 0);
        if (B.reg_fft) {
            const size_t r2c = sizeof(cpx<float>) * (size_t)kRegLines * line_ld(D.len[2].N) * 2;
            size_t cols = cols_smem_bytes<float>(D.len[1], kRegLines);
            if (three) cols = std::max(cols, cols_smem_bytes<float>(D.len[0], kRegLines));
            if (r2c > kRegBudget || cols > kRegBudget) B.reg_fft = 0;
        }
        if (B.reg_fft) {
            B.nb_r2c = B.nb_c2r = B.nb_a1 = B.nb_a0 = kRegLines;
        } else {
            B.nb_r2c = B.nb_c2r = lpb(D.len[2].N);
            B.nb_a1 = nh >= 16 ? lpb(D.len[1].N) : (int)nh;
            B.nb_a0 = three ? (nh >= 16 ? lpb(D.len[0].N) : (int)nh) : 1;
        }
        const int64_t npairs = (int64_t)D.n[0] * D.n[1] / 2;
        B.ntask[ST_R2C] = (int)((npairs + B.nb_r2c - 1) / B.nb_r2c);
        if (B.reg_fft) {   // register engine: columns of all outer indices in blocks of kRegLines
            B.ntask[ST_A1] = (int)cols_blocks<float, kRegLines>(B.a1);
            B.ntask[ST_A0] = three ? (int)cols_blocks<float, kRegLines>(B.a0) : 0;
        } else {
            B.ntask[ST_A1] = B.a1.nouter * (int)((nh + B.nb_a1 - 1) / B.nb_a1);
            B.ntask[ST_A0] = three ? B.a0.nouter * (int)((nh + B.nb_a0 - 1) / B.nb_a0) : 0;
        }
        B.spread_warp = (D.sub_T == 2 && D.w == 7) ? 1 : 0;
        B.ntask[ST_INTERP] = (int)(B.spread_warp ? D.nrchunks : 0);
        B.ntask[ST_SPREAD] = (int)(B.spread_warp ? D.nrchunks : D.nchunks);
        B.ntask[ST_WSUM] = (int)(D.ngroups * D.grp_parts);
        B.ntask[ST_COMBINE] = (int)((D.cmb_nact + kCombTiles - 1) / kCombTiles);
        B.ntask[ST_B0] = B.ntask[ST_A0];
        B.ntask[ST_B1] = B.ntask[ST_A1];
        B.ntask[ST_C2R] = B.ntask[ST_R2C];
        // stage dependencies: each stage waits for the previous non-empty stage of its item
        // (the combine reads every window slot; the inverse passes read all of G)
        int last = -1;
        for (int k = 0; k < kStages; ++k) {
            B.dep[k] = last;
            if (B.ntask[k] > 0) last = k;
        }
        // fixed-size sums of the FFT and spreading shared memory
        if (B.reg_fft) {
            smem = std::max(smem, sizeof(cpx<float>) * (size_t)kRegLines * line_ld(D.len[2].N) * 2);
            smem = std::max(smem, cols_smem_bytes<float>(D.len[1], kRegLines));
            if (three) smem = std::max(smem, cols_smem_bytes<float>(D.len[0], kRegLines));
        } else {
            smem = std::max(smem, fft_bytes(D.len[2].N, B.nb_r2c));
            smem = std::max(smem, fft_bytes(D.len[1].N, B.nb_a1));
            if (three) smem = std::max(smem, fft_bytes(D.len[0].N, B.nb_a0));
        }
        smem = std::max(smem, B.spread_warp ? interp_spread_reg_smem<float>(D, 8) : interp_spread_smem<float>(D, 8));
        smem = std::max(smem, window_sum_smem<float>());
    }
    b->smem = smem;
    // Stages run in this order per item, so the window slots and G are never rewritten while
    // an earlier stage of the same item still reads them.
    batch_offsets(b);
    auto dalloc = [&](void **ptr, size_t bytes) -> nlp_status {
        if (cudaMalloc(ptr, bytes) != cudaSuccess) { cudaGetLastError(); return NLP_ERR_OOM; }
        b->allocs.push_back(*ptr);
        return NLP_OK;
    };
    nlp_status s;
    void *d;
    if ((s = dalloc(&d, sizeof(BatchItem) * count))) { nlp_batch_destroy(b); return s; }
    b->d_items = (BatchItem *)d;
    if ((s = dalloc(&d, sizeof(int) * b->off.size()))) { nlp_batch_destroy(b); return s; }
    b->d_off = (int *)d;
    b->ctr_bytes = sizeof(int) * (2 + (size_t)kStages * count);
    if ((s = dalloc(&d, b->ctr_bytes))) { nlp_batch_destroy(b); return s; }
    b->d_ctr = (int *)d;
    if ((s = dalloc(&d, sizeof(void *) * 2 * count))) { nlp_batch_destroy(b); return s; }
    b->d_rho = (const float **)d;
    b->d_phi = (float **)d + count;
    if (cudaMallocHost((void **)&b->h_ptrs, sizeof(void *) * 2 * count) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_err, sizeof(int)) != cudaSuccess) {
        nlp_batch_destroy(b);
        return NLP_ERR_OOM;
    }
    memset(b->h_ptrs, 0, sizeof(void *) * 2 * count);
    *b->h_err = 0;
    cudaMemcpy(b->d_items, b->items.data(), sizeof(BatchItem) * count, cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_off, b->off.data(), sizeof(int) * b->off.size(), cudaMemcpyHostToDevice);   // (item_major 0)
    if ((int)b->smem > max_dyn_smem() || allow_smem<k_batch_persistent>() != cudaSuccess) {
        nlp_batch_destroy(b);
        return NLP_ERR_UNSUPPORTED;
    }
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_persistent, 256, b->smem);
    b->grid = std::max(1, sms * std::max(1, per));
    if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess || (s = batch_graph(b))) {
        nlp_batch_destroy(b);
        return s ? s : NLP_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) { nlp_batch_destroy(b); return NLP_ERR_CUDA; }
    *out = b;
    return NLP_OK;
}

nlp_status nlp_batch_eval(nlp_batch b, const void *const *rho_dev, void *const *phi_dev) {
    if (!b || !rho_dev || !phi_dev) return NLP_ERR_INVALID_ARG;
    for (int p = 0; p < b->count; ++p)
        if (!rho_dev[p] || !phi_dev[p]) return NLP_ERR_INVALID_ARG;
    if (b->mode == NLP_BATCH_GRAPH) {
        bool same = b->sexec != nullptr;
        for (int p = 0; p < b->count && same; ++p)
            same = b->cap_ptrs[p] == rho_dev[p] && b->cap_ptrs[b->count + p] == phi_dev[p];
        if (!same) {
            // the instantiated graph is updated in place: no replay of it may be in flight
            if (b->pending && cudaEventSynchronize(b->ev) != cudaSuccess) return NLP_ERR_CUDA;
            b->pending = false;
            nlp_status s = batch_stage_graph(b, rho_dev, phi_dev);
            if (s) return s;
        }
        if (cudaGraphLaunch(b->sexec, b->stream) != cudaSuccess) return NLP_ERR_CUDA;
        if (cudaEventRecord(b->ev, b->stream) != cudaSuccess) return NLP_ERR_CUDA;
        b->pending = true;
        return NLP_OK;
    }
    if (b->pending) {   // the pinned pointer table may still be read by the previous replay
        if (cudaEventSynchronize(b->ev) != cudaSuccess) return NLP_ERR_CUDA;
        b->pending = false;
    }
    for (int p = 0; p < b->count; ++p) {
        b->h_ptrs[p] = (void *)rho_dev[p];
        b->h_ptrs[b->count + p] = phi_dev[p];
    }
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return NLP_ERR_CUDA;
    if (cudaEventRecord(b->ev, b->stream) != cudaSuccess) return NLP_ERR_CUDA;
    b->pending = true;
    return NLP_OK;
}

nlp_status nlp_batch_sync(nlp_batch b) {
    if (!b) return NLP_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return NLP_ERR_CUDA;
    b->pending = false;
    return *b->h_err ? NLP_ERR_TIMEOUT : NLP_OK;
}

nlp_status nlp_batch_get_order(nlp_batch b, int *item_major) {
    if (!b || !item_major) return NLP_ERR_INVALID_ARG;
    *item_major = b->item_major;
    return NLP_OK;
}

nlp_status nlp_batch_set_mode(nlp_batch b, int mode, int branches) {
    if (!b || (mode != NLP_BATCH_PERSISTENT && mode != NLP_BATCH_GRAPH) ||
        (mode == NLP_BATCH_GRAPH && (branches < 1 || branches > 64)))
        return NLP_ERR_INVALID_ARG;
    if (b->pending && cudaEventSynchronize(b->ev) != cudaSuccess) return NLP_ERR_CUDA;
    b->pending = false;
    if (mode == NLP_BATCH_GRAPH && (mode != b->mode || branches != b->branches)) drop_stage_graph(b);
    b->mode = mode;
    if (mode == NLP_BATCH_GRAPH) {
        b->branches = branches;
        *b->h_err = 0;   // written only by the persistent form's replays
    }
    return NLP_OK;
}

nlp_status nlp_batch_get_mode(nlp_batch b, int *mode, int *branches) {
    if (!b || !mode) return NLP_ERR_INVALID_ARG;
    *mode = b->mode;
    if (branches) *branches = b->branches;
    return NLP_OK;
}

nlp_status nlp_batch_get_info(nlp_batch b, int *tasks, int *grid, size_t *smem_bytes) {
    if (!b) return NLP_ERR_INVALID_ARG;
    if (tasks) *tasks = b->total;
    if (grid) *grid = b->grid;
    if (smem_bytes) *smem_bytes = b->smem;
    return NLP_OK;
}

nlp_status nlp_batch_autotune(nlp_batch b, const void *const *rho_dev, void *const *phi_dev, int *best_grid,
                              double *best_ms) {
    if (!b || !rho_dev || !phi_dev) return NLP_ERR_INVALID_ARG;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_persistent, 256, b->smem) != cudaSuccess)
        return NLP_ERR_CUDA;
    per = std::max(1, per);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return NLP_ERR_CUDA;
    int best = 0, best_order = 0, best_mode = NLP_BATCH_PERSISTENT, best_br = 1;
    double bms = 1e300;
    nlp_status s = NLP_OK;
    auto time_it = [&](double &tmin) {
        tmin = 1e300;
        for (int rep = 0; rep < 4 && s == NLP_OK; ++rep) {
            cudaEventRecord(e0, b->stream);
            if ((s = nlp_batch_eval(b, rho_dev, phi_dev))) break;
            cudaEventRecord(e1, b->stream);
            if ((s = nlp_batch_sync(b))) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tmin = std::min(tmin, (double)ms);   // the first replay warms up
        }
    };
    // persistent form: the ticket order, and resident CTAs per SM from one to the occupancy limit
    b->mode = NLP_BATCH_PERSISTENT;
    for (int kk = 0; kk < 2 * per && s == NLP_OK; ++kk) {
        const int order = kk / per, k = kk % per + 1;
        if (order != b->item_major) {
            b->item_major = order;
            batch_offsets(b);
            if (cudaMemcpy(b->d_off, b->off.data(), sizeof(int) * b->off.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
                s = NLP_ERR_CUDA;
                break;
            }
        }
        b->grid = sms * k;
        if ((s = batch_graph(b))) break;
        double tmin;
        time_it(tmin);
        if (s == NLP_OK && tmin < bms) {
            bms = tmin;
            best = b->grid;
            best_order = b->item_major;
        }
    }
    // graph form: 1, 2, 4, 8 branches
    for (int br = 1; br <= 8 && br <= b->count && s == NLP_OK; br *= 2) {
        if ((s = nlp_batch_set_mode(b, NLP_BATCH_GRAPH, br))) break;
        double tmin;
        time_it(tmin);
        if (s == NLP_OK && tmin < bms) {
            bms = tmin;
            best_mode = NLP_BATCH_GRAPH;
            best_br = br;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    // keep the persistent form's best settings (its graph is re-captured) and the best form
    b->mode = NLP_BATCH_PERSISTENT;
    b->grid = best ? best : b->grid;
    if (best_order != b->item_major) {
        b->item_major = best_order;
        batch_offsets(b);
        if (cudaMemcpy(b->d_off, b->off.data(), sizeof(int) * b->off.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return NLP_ERR_CUDA;
    }
    if ((s = batch_graph(b))) return s;
    if (best_mode == NLP_BATCH_GRAPH && (s = nlp_batch_set_mode(b, NLP_BATCH_GRAPH, best_br))) return s;
    if (best_grid) *best_grid = best_mode == NLP_BATCH_GRAPH ? 0 : best;
    if (best_ms) *best_ms = bms;
    return NLP_OK;
}

nlp_status nlp_batch_set_wait_limit(nlp_batch b, long long polls, int block_item, int block_stage) {
    if (!b || polls < 1 || block_item >= b->count || block_stage >= kStages) return NLP_ERR_INVALID_ARG;
    if (b->pending && cudaEventSynchronize(b->ev) != cudaSuccess) return NLP_ERR_CUDA;
    b->pending = false;
    b->spin_limit = polls;
    // fault injection for tests: one stage's completion target is made unreachable, so the
    // stages after it poll until the limit runs out and the batch reports NLP_ERR_TIMEOUT
    std::vector<BatchItem> items = b->items;
    if (block_item >= 0 && block_stage >= 0) items[block_item].ntask[block_stage] += 1;
    cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * b->count, cudaMemcpyHostToDevice);
    return batch_graph(b);
}

}  // extern "C"

// ---------------------------------------------------------------- spread-tile autotuner
static std::string tune_key(const nlp_grid *g, nlp_kernel k, nlp_precision pr, const nlp_opts &o) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%d %d %d %d %.9g %.9g %.9g %d %d %.3g %.9g %d %d %d %d", g->dim, g->n[0], g->n[1],
             g->dim == 3 ? g->n[2] : 1, g->L[0], g->L[1], g->dim == 3 ? g->L[2] : 0.0, (int)k, (int)pr, o.nufft_tol,
             o.kmax, o.n_r, o.n_theta, o.n_phi, o.spread_variant);
    return std::string(buf);
}

extern "C" nlp_status nlp_autotune_tile(const nlp_grid *grid, nlp_kernel kernel, nlp_precision prec,
                                        const nlp_opts *base, void *stream, const char *cache_path, int *best_tile,
                                        double *best_ms) {
    if (!grid || !best_tile) return NLP_ERR_INVALID_ARG;
    if (grid->dim == 1) return NLP_ERR_UNSUPPORTED;   // no spreading tiles in 1D
    nlp_opts o;
    if (base) o = *base;
    else memset(&o, 0, sizeof(o));
    const std::string key = tune_key(grid, kernel, prec, o);
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "r")) {
            char line[640];
            int found = 0;
            while (fgets(line, sizeof(line), f)) {
                const std::string l(line);
                const size_t bar = l.find('|');
                if (bar == std::string::npos) continue;
                if (l.substr(0, bar) == key) {
                    int t = 0;
                    double ms = 0;
                    if (sscanf(l.c_str() + bar + 1, "%d %lf", &t, &ms) == 2) {
                        *best_tile = t;
                        if (best_ms) *best_ms = ms;
                        found = 1;
                    }
                }
            }
            fclose(f);
            if (found) return NLP_OK;
        }
    }
    std::vector<int> cands;
    if (grid->dim == 2) cands = {8, 16, 32};
    else if (prec == NLP_FP32) cands = {4, 8, 16};
    else cands = {2, 4, 6};
    size_t N = 1;
    for (int a = 0; a < grid->dim; ++a) N *= (size_t)grid->n[a];
    const size_t rb = N * (prec == NLP_FP64 ? 8 : 4);
    void *rho = nullptr, *phi = nullptr;
    if (cudaMalloc(&rho, rb) != cudaSuccess || cudaMalloc(&phi, rb) != cudaSuccess) {
        cudaGetLastError();
        if (rho) cudaFree(rho);
        return NLP_ERR_OOM;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(rho, 0, rb, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    double bms = 1e300;
    nlp_status last = NLP_OK;
    for (int c : cands) {
        o.tile = c;
        nlp_plan p = nullptr;
        nlp_status s = nlp_plan_create(grid, kernel, prec, &o, stream, &p);
        if (s) { last = s; continue; }
        double tmin = 1e300;
        for (int rep = 0; rep < 5; ++rep) {
            cudaEventRecord(e0, st);
            s = nlp_eval_potential(p, rho, phi);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < tmin) tmin = ms;   // first evaluation is a warm-up
        }
        nlp_plan_destroy(p);
        if (s) { last = s; continue; }
        if (tmin < bms) { bms = tmin; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(rho);
    cudaFree(phi);
    if (!best) return last ? last : NLP_ERR_UNSUPPORTED;
    *best_tile = best;
    if (best_ms) *best_ms = bms;
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "a")) {
            fprintf(f, "%s|%d %.6f\n", key.c_str(), best, bms);
            fclose(f);
        }
    }
    return NLP_OK;
}
