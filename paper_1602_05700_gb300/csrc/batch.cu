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
// Autotuning: the z extent of an FP64 block (planes per block, which sets the number of blocks and the share of
// the z warm-up) is chosen from a few candidates by timing the first sub-steps of the first hg_batch_step with
// CUDA events -- every candidate computes the same result, so the timing runs are real sub-steps -- and cached per
// (device, set of grid shapes/precisions/boundaries) for the process.  The TMA-staged blocks of the compensated-float
// grids use 8 planes, where their stage ring hides the z warm-up.
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
    int zb;  // planes per block, 0 until tuned
    // graph of `graph_steps` sub-steps
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int graph_steps;
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tuned;  // autotuner cache: key -> planes per block

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
    return k;
}

// device tables for the sub-step that starts from parity p (0: every grid's current level, 1: the next one)
int upload_tables(hg_batch* b) {
    std::vector<TmaEntry> tab[2];
    for (int p = 0; p < 2; ++p) {
        for (hg_grid* g : b->grids) {
            const int cur = g->cur;
            g->cur = cur ^ p;
            TmaEntry e;
            memset(&e, 0, sizeof e);
            int rc = HG_OK;
            if (g->prec == HG_PREC_F32K) {
                rc = tma_entry(g, &e);  // TMA-staged blocks: a fixed 8-plane chunk
            } else {
                e.A = sweep_args(g, b->zb);
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
    for (int p = 0; p < 2; ++p)
        HG_CUDA(cudaMemcpyAsync(b->d_tab[p], tab[p].data(), tab[p].size() * sizeof(TmaEntry), cudaMemcpyHostToDevice,
                                b->stream));
    HG_CUDA(cudaMemcpyAsync(b->d_first, b->first.data(), b->first.size() * sizeof(unsigned), cudaMemcpyHostToDevice,
                            b->stream));
    HG_CUDA(cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
    return HG_OK;
}

// the launch of one sub-step of parity p
int enqueue_substep(hg_batch* b, int p) { return launch_step_batch(b->stream, b->d_tab[p], b->d_first, b->n, b->total_blocks); }

void advance(hg_batch* b, int n) {
    for (hg_grid* g : b->grids) {
        if (n & 1) g->cur ^= 1;
        g->step += n;
    }
}

// pick the planes per block by timing two sub-steps per candidate (real sub-steps: every candidate gives the same
// result); returns the number of sub-steps taken
int autotune(hg_batch* b, int budget, int* taken) {
    *taken = 0;
    const std::string key = tune_key(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            b->zb = it->second;
            return upload_tables(b);
        }
    }
    bool any64 = false;
    for (hg_grid* g : b->grids) any64 = any64 || g->prec == HG_PREC_F64;
    if (!any64) {  // nothing to tune: the TMA-staged blocks use a fixed chunk
        b->zb = 8;
        return upload_tables(b);
    }
    const int cand[] = {8, 16, 32, 64};
    int best = 0;
    float best_ms = 0.f;
    cudaEvent_t e0, e1;
    HG_CUDA(cudaEventCreate(&e0));
    HG_CUDA(cudaEventCreate(&e1));
    int rc = HG_OK;
    for (int c : cand) {
        if (*taken >= budget) break;
        if (*taken + 2 > budget) break;
        b->zb = c;
        if ((rc = upload_tables(b))) break;
        cudaEventRecord(e0, b->stream);
        if ((rc = enqueue_substep(b, 0))) break;  // two sub-steps (both parities) per candidate
        if ((rc = enqueue_substep(b, 1))) break;
        cudaEventRecord(e1, b->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotuner timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        advance(b, 2);
        *taken += 2;
        if (best == 0 || ms < best_ms) {
            best = c;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (best == 0) return HG_OK;  // no budget to tune: keep the default rule this time
    b->zb = best;
    if (*taken == 2 * (int)(sizeof cand / sizeof cand[0])) {
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
    void* ptrs[] = {b->d_tab[0], b->d_tab[1], b->d_first};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
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
    b->grids.assign(grids, grids + n);
    b->device = grids[0]->device;
    int rc = HG_OK;
    auto ck = [&](cudaError_t err, const char* what) {
        if (rc == HG_OK && err != cudaSuccess) rc = cuda_fail(err, what);
    };
    ck(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    ck(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming), "cudaEventCreate");
    ck(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming), "cudaEventCreate");
    for (int p = 0; p < 2 && rc == HG_OK; ++p) ck(cudaMalloc(&b->d_tab[p], n * sizeof(TmaEntry)), "cudaMalloc(table)");
    ck(cudaMalloc(&b->d_first, (n + 1) * sizeof(unsigned)), "cudaMalloc(table)");
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
            for (int s = 0; s < n && rc == HG_OK; ++s) rc = enqueue_substep(b, s & 1);
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

int hg_batch_info(const hg_batch* b, int* z_planes_per_block, long long* blocks_per_substep) {
    HG_RANGE("hg_batch_info");
    if (!b) return fail(HG_ERR_ARG, "null batch");
    if (z_planes_per_block) *z_planes_per_block = b->zb;
    if (blocks_per_substep) *blocks_per_substep = b->total_blocks;
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
