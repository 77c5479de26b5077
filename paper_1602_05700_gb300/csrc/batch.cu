// Many independent grids advanced together (the batching workload: uneven sizes, mixed precisions).
//
// One sub-step of every grid is one batched kernel launch (stencil.cu, k_step_batch: block -> grid by a prefix
// table; compensated-float grids run the TMA-staged sweep with their tensor maps in the table, FP64 grids the
// register-staged FP64 sweep, in the same launch, so HBM-bound and FP64-bound blocks share the SMs; boundary ghosts
// are written inside the launch).  hg_batch_step(b, n) records the n sub-steps once as a CUDA graph on the batch's
// own stream and replays it with a single graph launch; the kernels read the per-grid arguments from two device
// tables (for the two time-level parities), refreshed from the grids before every replay, so the graph stays valid
// while the grids' states move on.  Results are identical to stepping each grid on its own: the per-cell arithmetic
// is the same code.
//
// Autotuning: three knobs of the launch are chosen by timing the first sub-steps of the first hg_batch_step with
// CUDA events -- every candidate computes the same result, so the timing runs are real sub-steps -- and cached per
// (device, set of grid shapes/precisions/boundaries) for the process:
//   * the tile shape of an FP64 block: rows of 128 cells (4 per lane) for every grid, or per grid whichever of
//     128- and 32-cell rows (1 per lane) leaves fewer lanes idle (a 96-cell row fills 75% of a 128-cell tile; the
//     FP64 pipe pays for idle lanes, since its rate is per warp instruction);
//   * the z extent of an FP64 block (8 .. 64 planes: the number of blocks against the share of the z warm-up);
//   * the z extent of a TMA-staged compensated-float block (8 or 16 planes);
//   * one launch per sub-step for both precisions, or two (split mode: an FP64-only launch and a float-only launch
//     per sub-step, each with its own sweep's registers and block shape, as two independent chains on two streams).
// All FP64 candidates are timed first (eight), then the split mode with the best FP64 setting, then the float
// extent of 16 planes with the better of the two.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hg_internal.cuh"

using namespace hg;

struct hg_batch {
    int n;
    std::vector<hg_grid*> grids;
    int device;
    cudaStream_t stream;  // own non-blocking stream (graphs cannot be captured on the legacy default stream)
    cudaEvent_t ev_in, ev_out;
    TmaEntry* d_tab[2];   // per-grid entries, per parity
    unsigned* d_first;
    unsigned total_blocks;
    std::vector<unsigned> first;
    int zb;    // FP64 planes per block, 0 until tuned
    int cpl;   // FP64 cells per lane: 0 = per grid, whichever tile row fits better; 4 = 128-cell rows everywhere
    int zb32;  // compensated-float (TMA-staged) planes per block
    int split; // 1: FP64 and compensated-float entries as two launches per sub-step, on two streams
    int force_split;  // -1: the autotuner chooses split; 0 or 1: pinned by hg_batch_set_split
    // split mode: the two classes' own prefix tables (FP64 entries first in the table, then the float ones)
    cudaStream_t stream2;
    cudaEvent_t ev_fork, ev_join;
    unsigned* d_first2;  // FP64 prefix (n64 + 1 entries), then float prefix (n32 + 1 entries)
    int n64, n32;
    unsigned blocks64, blocks32;
    // graph of `graph_steps` sub-steps
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int graph_steps;
};

namespace {

std::mutex g_tune_mu;
struct Tuning {
    int zb, cpl, zb32, split;
};
std::map<std::string, Tuning> g_tuned;  // autotuner cache: key -> the chosen launch

std::string tune_key(const hg_batch* b) {
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, b->device);
    std::vector<std::string> parts;
    for (hg_grid* g : b->grids) {
        char buf[96];
        snprintf(buf, sizeof buf, "%dx%dx%d/%d/%d", g->nx, g->ny, g->nz, g->prec, g->bc);
        parts.push_back(buf);
    }
    std::sort(parts.begin(), parts.end());
    std::string k = p.name;
    for (auto& s : parts) k += ";" + s;
    k += ";split=" + std::to_string(b->force_split);
    return k;
}

// device tables for the sub-step that starts from parity p (0: every grid's current level, 1: the next one)
// The table lists the FP64 grids first, largest first, then the compensated-float grids: the block scheduler hands
// out blocks in index order, so the long FP64-bound blocks start first and the short HBM-bound ones fill in around
// them and make up the tail of each launch.
std::vector<hg_grid*> launch_order(const hg_batch* b) {
    std::vector<hg_grid*> o(b->grids);
    auto cells = [](const hg_grid* g) { return (long long)g->nx * g->ny * g->nz; };
    std::stable_sort(o.begin(), o.end(), [&](const hg_grid* a, const hg_grid* c) {
        const bool a64 = a->prec == HG_PREC_F64, c64 = c->prec == HG_PREC_F64;
        if (a64 != c64) return a64;
        return cells(a) > cells(c);
    });
    return o;
}

int upload_tables(hg_batch* b) {
    std::vector<TmaEntry> tab[2];
    const std::vector<hg_grid*> order = launch_order(b);
    for (int p = 0; p < 2; ++p) {
        for (hg_grid* g : order) {
            const int cur = g->cur;
            g->cur = cur ^ p;
            TmaEntry e;
            memset(&e, 0, sizeof e);
            int rc = HG_OK;
            if (g->prec == HG_PREC_F32K) {
                rc = tma_entry(g, &e, b->zb32);
            } else {
                e.A = sweep_args(g, b->zb, b->cpl);
                e.err = g->derr;
            }
            g->cur = cur;
            if (rc) return rc;
            tab[p].push_back(e);
        }
    }
    b->first.assign(1, 0);
    for (const TmaEntry& e : tab[0]) b->first.push_back(b->first.back() + sweep_blocks(e.A));
    b->total_blocks = b->first.back();
    // the classes' own prefixes: FP64 entries are [0, n64), float entries [n64, n)
    b->n64 = 0;
    for (hg_grid* g : order) b->n64 += g->prec == HG_PREC_F64 ? 1 : 0;
    b->n32 = b->n - b->n64;
    std::vector<unsigned> first2;
    first2.push_back(0);
    for (int i = 0; i < b->n64; ++i) first2.push_back(first2.back() + sweep_blocks(tab[0][i].A));
    b->blocks64 = first2.back();
    first2.push_back(0);
    for (int i = b->n64; i < b->n; ++i) first2.push_back(first2.back() + sweep_blocks(tab[0][i].A));
    b->blocks32 = first2.back();
    HG_CUDA(cudaMemcpyAsync(b->d_first2, first2.data(), first2.size() * sizeof(unsigned), cudaMemcpyHostToDevice,
                            b->stream));
    for (int p = 0; p < 2; ++p)
        HG_CUDA(cudaMemcpyAsync(b->d_tab[p], tab[p].data(), tab[p].size() * sizeof(TmaEntry), cudaMemcpyHostToDevice,
                                b->stream));
    HG_CUDA(cudaMemcpyAsync(b->d_first, b->first.data(), b->first.size() * sizeof(unsigned), cudaMemcpyHostToDevice,
                            b->stream));
    HG_CUDA(cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
    return HG_OK;
}

// the launches of `count` sub-steps, the first of parity p0.  Split mode: the FP64 chain on the batch stream and
// the float chain on the second stream, forked from and joined back into the batch stream (the chains touch
// different grids, so they need no ordering between them).
int enqueue_substeps(hg_batch* b, int p0, int count) {
    int rc = HG_OK;
    if (!b->split) {
        for (int s = 0; s < count && rc == HG_OK; ++s)
            rc = launch_step_batch(b->stream, b->d_tab[(p0 + s) & 1], b->d_first, b->n, b->total_blocks);
        return rc;
    }
    HG_CUDA(cudaEventRecord(b->ev_fork, b->stream));
    HG_CUDA(cudaStreamWaitEvent(b->stream2, b->ev_fork, 0));
    for (int s = 0; s < count && rc == HG_OK; ++s) {
        const int p = (p0 + s) & 1;
        rc = launch_batch_class(b->stream, true, b->d_tab[p], b->d_first2, b->n64, b->blocks64);
        if (rc == HG_OK)
            rc = launch_batch_class(b->stream2, false, b->d_tab[p] + b->n64, b->d_first2 + b->n64 + 1, b->n32,
                                    b->blocks32);
    }
    // join even after an error, so that a capture in progress ends with both streams in it
    cudaError_t e1 = cudaEventRecord(b->ev_join, b->stream2);
    cudaError_t e2 = cudaStreamWaitEvent(b->stream, b->ev_join, 0);
    if (rc) return rc;
    if (e1 != cudaSuccess) return cuda_fail(e1, "cudaEventRecord");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamWaitEvent");
    return HG_OK;
}

void advance(hg_batch* b, int n) {
    for (hg_grid* g : b->grids) {
        if (n & 1) g->cur ^= 1;
        g->step += n;
    }
}

// pick the launch by timing two sub-steps per candidate (real sub-steps: every candidate gives the same result);
// returns the number of sub-steps taken in *taken
int autotune(hg_batch* b, int budget, int* taken) {
    *taken = 0;
    const std::string key = tune_key(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            b->zb = it->second.zb;
            b->cpl = it->second.cpl;
            b->zb32 = it->second.zb32;
            b->split = it->second.split;
            return upload_tables(b);
        }
    }
    bool any64 = false, any32 = false;
    for (hg_grid* g : b->grids) {
        any64 = any64 || g->prec == HG_PREC_F64;
        any32 = any32 || g->prec == HG_PREC_F32K;
    }
    std::vector<Tuning> cand;
    const int split0 = b->force_split > 0 ? 1 : 0;
    if (any64)
        for (int cpl : {0, 4})
            for (int zb : {8, 16, 32, 64}) cand.push_back({zb, cpl, 8, split0});
    else
        cand.push_back({8, 0, 8, split0});
    Tuning best = cand[0];
    float best_ms = -1.f;
    cudaEvent_t e0, e1;
    HG_CUDA(cudaEventCreate(&e0));
    HG_CUDA(cudaEventCreate(&e1));
    int rc = HG_OK;
    bool complete = true;
    auto time_one = [&](const Tuning& t) -> bool {  // false: no budget left or an error (rc)
        if (*taken + 2 > budget) {
            complete = false;
            return false;
        }
        b->zb = t.zb;
        b->cpl = t.cpl;
        b->zb32 = t.zb32;
        b->split = t.split;
        if ((rc = upload_tables(b))) return false;
        cudaEventRecord(e0, b->stream);
        if ((rc = enqueue_substeps(b, 0, 2))) return false;  // two sub-steps (both parities) per candidate
        cudaEventRecord(e1, b->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotuner timing");
            return false;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        advance(b, 2);
        *taken += 2;
        if (best_ms < 0.f || ms < best_ms) {
            best = t;
            best_ms = ms;
        }
        return true;
    };
    for (const Tuning& t : cand)
        if (!time_one(t)) break;
    if (rc == HG_OK && complete && best_ms >= 0.f && b->force_split < 0) {  // each class as a launch of its own
        Tuning t = best;
        t.split = 1;
        time_one(t);
    }
    if (rc == HG_OK && complete && any32 && best_ms >= 0.f) {
        Tuning t = best;
        t.zb32 = 16;
        time_one(t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (best_ms < 0.f) {  // no budget to tune: the default launch this time
        b->zb = 8;
        b->cpl = 0;
        b->zb32 = 8;
        b->split = split0;
        return upload_tables(b);
    }
    b->zb = best.zb;
    b->cpl = best.cpl;
    b->zb32 = best.zb32;
    b->split = best.split;
    if (complete) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[key] = best;
    }
    return upload_tables(b);
}

void destroy_graph(hg_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_steps = 0;
}

void release(hg_batch* b) {
    destroy_graph(b);
    void* ptrs[] = {b->d_tab[0], b->d_tab[1], b->d_first, b->d_first2};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    cudaEvent_t evs[] = {b->ev_in, b->ev_out, b->ev_fork, b->ev_join};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->stream2) cudaStreamDestroy(b->stream2);
}

}  // namespace

extern "C" {

int hg_batch_create(hg_grid* const* grids, int n, hg_batch** out) {
    HG_RANGE("hg_batch_create");
    if (!out) return fail(HG_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (!grids || n < 1) return fail(HG_ERR_ARG, "need at least one grid");
    for (int i = 0; i < n; ++i) {
        if (!grids[i]) return fail(HG_ERR_ARG, "grid %d is null", i);
        if (grids[i]->device != grids[0]->device) return fail(HG_ERR_ARG, "all grids of a batch must share one device");
        if (grids[i]->ziface) return fail(HG_ERR_ARG, "grid %d is a slab (z interfaces): batches hold whole grids", i);
        if (grids[i]->stream != grids[0]->stream) return fail(HG_ERR_ARG, "all grids of a batch must share one stream");
        for (int j = 0; j < i; ++j)
            if (grids[j] == grids[i]) return fail(HG_ERR_ARG, "grid %d appears twice", i);
    }
    cudaError_t e = cudaSetDevice(grids[0]->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    hg_batch* b = new hg_batch();
    b->n = n;
    b->force_split = -1;
    b->grids.assign(grids, grids + n);
    b->device = grids[0]->device;
    int rc = HG_OK;
    auto ck = [&](cudaError_t err, const char* what) {
        if (rc == HG_OK && err != cudaSuccess) rc = cuda_fail(err, what);
    };
    ck(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    ck(cudaStreamCreateWithFlags(&b->stream2, cudaStreamNonBlocking), "cudaStreamCreate");
    for (cudaEvent_t* ev : {&b->ev_in, &b->ev_out, &b->ev_fork, &b->ev_join})
        ck(cudaEventCreateWithFlags(ev, cudaEventDisableTiming), "cudaEventCreate");
    for (int p = 0; p < 2 && rc == HG_OK; ++p) ck(cudaMalloc(&b->d_tab[p], n * sizeof(TmaEntry)), "cudaMalloc(table)");
    ck(cudaMalloc(&b->d_first, (n + 1) * sizeof(unsigned)), "cudaMalloc(table)");
    ck(cudaMalloc(&b->d_first2, (n + 2) * sizeof(unsigned)), "cudaMalloc(table)");
    if (rc == HG_OK) rc = upload_tables(b);
    if (rc != HG_OK) {
        release(b);
        delete b;
        return rc;
    }
    *out = b;
    return HG_OK;
}

int hg_batch_step(hg_batch* b, int n_substeps) {
    HG_RANGE("hg_batch_step");
    if (!b) return fail(HG_ERR_ARG, "null batch");
    if (n_substeps < 0) return fail(HG_ERR_ARG, "n_substeps must be >= 0");
    if (n_substeps == 0) return HG_OK;
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t gs = b->grids[0]->stream;
    // the batch stream waits for earlier work of the grids, and the grids' stream for the batch
    HG_CUDA(cudaEventRecord(b->ev_in, gs));
    HG_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    int rc = HG_OK;
    int done = 0;
    if (b->zb == 0) {
        rc = autotune(b, n_substeps, &done);
        if (rc) return rc;
        destroy_graph(b);
    }
    const int n = n_substeps - done;
    if (n > 0) {
        if ((rc = upload_tables(b))) return rc;
        if (b->graph_steps != n) {
            destroy_graph(b);
            HG_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            rc = enqueue_substeps(b, 0, n);
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(b->stream, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            b->graph = graph;
            HG_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
            b->graph_steps = n;
        }
        HG_CUDA(cudaGraphLaunch(b->exec, b->stream));
        advance(b, n);
    }
    HG_CUDA(cudaEventRecord(b->ev_out, b->stream));
    HG_CUDA(cudaStreamWaitEvent(gs, b->ev_out, 0));
    return HG_OK;
}

int hg_batch_set_split(hg_batch* b, int mode) {
    HG_RANGE("hg_batch_set_split");
    if (!b) return fail(HG_ERR_ARG, "null batch");
    if (mode < -1 || mode > 1) return fail(HG_ERR_ARG, "mode must be -1 (autotuned), 0 or 1");
    if (mode == b->force_split) return HG_OK;
    b->force_split = mode;
    b->zb = 0;  // the next hg_batch_step tunes (or finds in the cache) the launch for this mode
    destroy_graph(b);
    return HG_OK;
}

int hg_batch_info(const hg_batch* b, int* z_planes_per_block, long long* blocks_per_substep) {
    HG_RANGE("hg_batch_info");
    if (!b) return fail(HG_ERR_ARG, "null batch");
    if (z_planes_per_block) *z_planes_per_block = b->zb;
    if (blocks_per_substep) *blocks_per_substep = b->total_blocks;
    return HG_OK;
}

int hg_batch_tuning(const hg_batch* b, int out[4]) {
    HG_RANGE("hg_batch_tuning");
    if (!b || !out) return fail(HG_ERR_ARG, "null argument");
    out[0] = b->zb;
    out[1] = b->cpl;
    out[2] = b->zb32;
    out[3] = b->split;
    return HG_OK;
}

void hg_batch_free(hg_batch* b) {
    HG_RANGE("hg_batch_free");
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    release(b);
    delete b;
}

}  // extern "C"
