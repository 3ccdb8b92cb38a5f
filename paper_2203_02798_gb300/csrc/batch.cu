// batch.cu -- many independent leverage-score problems in one call.
//
// The problems are sorted by estimated cost (longest first) and assigned
// greedily to the least-loaded of S worker streams; each stream owns a
// workspace sized for the largest of its problems, so problems on different
// streams run concurrently and small problems fill the SMs that large ones
// leave idle.  The whole batch (fork from the context stream, S chains of
// per-problem pipelines, join) can be captured once into a CUDA graph and
// replayed: a repeated batch costs one graph launch.  The stream count S is
// picked by an autotuner that times the candidates on the batch itself, and
// remembers the choice per batch signature (optionally in the file named by
// LSK_AUTOTUNE_CACHE).
#include "lsk_internal.cuh"

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

struct LskBatch {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;      // capture stream (the caller's may be the legacy stream)
    std::vector<void*> ws;
    std::vector<size_t> ws_bytes;
    cudaGraphExec_t exec = nullptr;
    uint64_t exec_key = 0;
    std::map<uint64_t, int> tuned;   // batch signature -> stream count
};

namespace {

uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

double cost_of(const lsk_batch_item& it) {
    const lsk_mat& A = it.A;
    const double bytes = A.kind == LSK_DENSE ? (double)A.n * A.d * 4 : (double)A.nnz * 8 + A.n * 8.0;
    return 2.0 * bytes + 4.0 * (double)it.r * A.d + 2e5;   // two passes over A, SA, launch floor
}

int ensure_streams(lsk_ctx* ctx, int S) {
    LskBatch* b = ctx->batch;
    while ((int)b->streams.size() < S) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LSK_ERR_CUDA;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return LSK_ERR_CUDA;
        b->streams.push_back(s);
        b->done.push_back(e);
        b->ws.push_back(nullptr);
        b->ws_bytes.push_back(0);
    }
    if (!b->fork && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return LSK_ERR_CUDA;
    if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return LSK_ERR_CUDA;
    return LSK_OK;
}

// assignment of problems to S streams (longest processing time first)
std::vector<std::vector<int>> plan(const lsk_batch_item* items, int count, int S) {
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost_of(items[a]) > cost_of(items[b]); });
    std::vector<std::vector<int>> lanes(S);
    std::vector<double> load(S, 0.0);
    for (int i : order) {
        const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lanes[s].push_back(i);
        load[s] += cost_of(items[i]);
    }
    return lanes;
}

int size_workspaces(lsk_ctx* ctx, const std::vector<std::vector<int>>& lanes, const lsk_batch_item* items,
                    int32_t prec) {
    LskBatch* b = ctx->batch;
    for (size_t s = 0; s < lanes.size(); ++s) {
        size_t need = 0;
        for (int i : lanes[s])
            need = std::max(need, leverage_workspace_bytes(&items[i].A, items[i].r, items[i].k, prec, ctx->sm_count));
        if (need > b->ws_bytes[s]) {
            if (b->ws[s]) cudaFree(b->ws[s]);
            b->ws[s] = nullptr;
            b->ws_bytes[s] = 0;
            if (cudaMalloc(&b->ws[s], need + need / 8) != cudaSuccess) {
                cudaGetLastError();
                return LSK_ERR_OOM;
            }
            b->ws_bytes[s] = need + need / 8;
        }
    }
    return LSK_OK;
}

// fork -> per-stream chains -> join, all on `main`'s timeline
cudaError_t record(lsk_ctx* ctx, cudaStream_t main, const std::vector<std::vector<int>>& lanes,
                   const lsk_batch_item* items, int32_t prec) {
    LskBatch* b = ctx->batch;
    cudaError_t e = cudaEventRecord(b->fork, main);
    if (e != cudaSuccess) return e;
    for (size_t s = 0; s < lanes.size(); ++s) {
        cudaStream_t st = b->streams[s];
        if ((e = cudaStreamWaitEvent(st, b->fork, 0)) != cudaSuccess) return e;
        for (int i : lanes[s]) {
            e = leverage_pipeline(&items[i].A, items[i].r, items[i].k, items[i].seed, prec, items[i].ell, nullptr,
                                  b->ws[s], ctx->flag, ctx->sm_count, st);
            if (e != cudaSuccess) return e;
        }
        if ((e = cudaEventRecord(b->done[s], st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(main, b->done[s], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

uint64_t signature(const lsk_batch_item* items, int count, int32_t prec) {
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, &count, sizeof(count));
    h = fnv(h, &prec, sizeof(prec));
    for (int i = 0; i < count; ++i) {
        const lsk_mat& A = items[i].A;
        int64_t v[6] = {A.kind, A.n, A.d, A.nnz, items[i].r, items[i].k};
        h = fnv(h, v, sizeof(v));
    }
    return h;
}

uint64_t exact_key(const lsk_batch_item* items, int count, int32_t prec, int S) {
    uint64_t h = fnv(signature(items, count, prec), &S, sizeof(S));
    return fnv(h, items, sizeof(lsk_batch_item) * (size_t)count);
}

int cache_lookup(uint64_t sig) {
    const char* path = getenv("LSK_AUTOTUNE_CACHE");
    if (!path) return 0;
    FILE* f = fopen(path, "r");
    if (!f) return 0;
    unsigned long long k;
    int s, best = 0;
    while (fscanf(f, "%llx %d", &k, &s) == 2)
        if (k == sig) best = s;
    fclose(f);
    return best;
}

void cache_store(uint64_t sig, int S) {
    const char* path = getenv("LSK_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%llx %d\n", (unsigned long long)sig, S);
    fclose(f);
}

}  // namespace

void lsk_batch_free(lsk_ctx* ctx) {
    LskBatch* b = ctx->batch;
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (size_t s = 0; s < b->streams.size(); ++s) {
        cudaStreamSynchronize(b->streams[s]);
        if (b->ws[s]) cudaFree(b->ws[s]);
        cudaEventDestroy(b->done[s]);
        cudaStreamDestroy(b->streams[s]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    ctx->batch = nullptr;
}

extern "C" int lsk_batch_leverage_scores(lsk_ctx* ctx, int32_t count, const lsk_batch_item* items, int32_t prec,
                                         int32_t flags) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    ProfGuard pg(ctx);
    if (count < 0 || (count > 0 && !items)) {
        snprintf(ctx->err, sizeof(ctx->err), "bad batch");
        return LSK_ERR_INVALID_ARG;
    }
    if (prec == LSK_PREC_TF32) prec = LSK_PREC_FP32;
    for (int i = 0; i < count; ++i) {
        const int rc = check_leverage_args(ctx, &items[i].A, items[i].r, items[i].k, prec);
        if (rc) return rc;
        if (!items[i].ell && items[i].A.n > 0) {
            snprintf(ctx->err, sizeof(ctx->err), "item %d: ell is NULL", i);
            return LSK_ERR_INVALID_ARG;
        }
    }
    if (count == 0) return LSK_OK;
    if (!ctx->batch) ctx->batch = new LskBatch();
    LskBatch* b = ctx->batch;
    const uint64_t sig = signature(items, count, prec);

    int S = (flags & LSK_BATCH_STREAMS_MASK) ? (flags & LSK_BATCH_STREAMS_MASK) : 0;
    if (!S) {
        auto it = b->tuned.find(sig);
        if (it != b->tuned.end()) S = it->second;
        else if ((S = cache_lookup(sig)) > 0) b->tuned[sig] = S;
    }
    if (!S && (flags & LSK_BATCH_AUTOTUNE)) {
        // time each candidate on the batch itself (outside any capture)
        const int cand[] = {1, 4, 8, 16, 32};
        float best_ms = 1e30f;
        int best = 8;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int c : cand) {
            if (c > count) continue;
            int rc = ensure_streams(ctx, c);
            if (rc) return rc;
            const auto lanes = plan(items, count, c);
            if ((rc = size_workspaces(ctx, lanes, items, prec))) return rc;
            for (int rep = 0; rep < 2; ++rep) {   // first pass warms up
                cudaEventRecord(e0, ctx->stream);
                cudaError_t e = record(ctx, ctx->stream, lanes, items, prec);
                if (e != cudaSuccess) {
                    snprintf(ctx->err, sizeof(ctx->err), "batch: %s", cudaGetErrorString(e));
                    return LSK_ERR_CUDA;
                }
                cudaEventRecord(e1, ctx->stream);
            }
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        S = best;
        b->tuned[sig] = S;
        cache_store(sig, S);
    }
    if (!S) S = count < 8 ? count : 8;

    int rc = ensure_streams(ctx, S);
    if (rc) return rc;
    const auto lanes = plan(items, count, S);
    if ((rc = size_workspaces(ctx, lanes, items, prec))) return rc;

    if (!(flags & LSK_BATCH_GRAPH)) {
        cudaError_t e = record(ctx, ctx->stream, lanes, items, prec);
        if (e != cudaSuccess) {
            snprintf(ctx->err, sizeof(ctx->err), "batch: %s", cudaGetErrorString(e));
            return LSK_ERR_CUDA;
        }
        return LSK_OK;
    }
    const uint64_t key = exact_key(items, count, prec, S);
    if (!b->exec || b->exec_key != key) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        const int prof_was = ctx->prof_on;
        lsk_prof_current = nullptr;   // no event records inside the capture
        cudaGraph_t g;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t er = record(ctx, b->cap, lanes, items, prec);
            e = cudaStreamEndCapture(b->cap, &g);
            if (er != cudaSuccess) e = er;
        }
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&b->exec, g, 0);
            cudaGraphDestroy(g);
        }
        if (prof_was) lsk_prof_current = ctx->prof;
        if (e != cudaSuccess) {
            cudaGetLastError();
            snprintf(ctx->err, sizeof(ctx->err), "batch graph: %s", cudaGetErrorString(e));
            return LSK_ERR_CUDA;
        }
        b->exec_key = key;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, ctx->stream);
    if (e != cudaSuccess) {
        snprintf(ctx->err, sizeof(ctx->err), "batch graph launch: %s", cudaGetErrorString(e));
        return LSK_ERR_CUDA;
    }
    return LSK_OK;
}

extern "C" int lsk_batch_streams(lsk_ctx* ctx, int32_t count, const lsk_batch_item* items, int32_t prec) {
    if (!ctx || !ctx->batch) return 0;
    auto it = ctx->batch->tuned.find(signature(items, count, prec == LSK_PREC_TF32 ? LSK_PREC_FP32 : prec));
    return it == ctx->batch->tuned.end() ? 0 : it->second;
}
