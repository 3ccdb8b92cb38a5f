// batch.cu -- many independent leverage-score problems in one call.
//
// Problems whose Gaussian stage runs on the tensor cores (BF16) and whose R
// takes the mixed-precision path (d <= 256) are run in three phases:
//   1. CountSketch of each problem on the worker streams (memory-bound
//      passes over A, concurrent across problems), into a batch arena that
//      holds every such problem's sketch -- compacted to its non-empty
//      buckets where n < 4r, so that phase 2 draws G only for those columns;
//   2. the Gaussian stage, the whole R^-1 computation and the row norms'
//      operand built from R^-1 as grouped launches: one grid per stage over
//      all problems (qr.cu, qr_mixed.cu, gauss_tc.cu, rownorms*.cu), so the
//      latency-bound small stages of hundreds of problems run side by side
//      instead of one after another;
//   3. row norms of each problem on the worker streams.
// Other problems run their whole pipeline on the worker streams in phase 1.
// The CountSketch permutations of each wave's grouped problems (count, scan,
// place, compaction) are grouped launches too, on a stream of their own
// ahead of the gathers (phase 0).
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

// The schedule knobs of a batch (chosen by the autotuner per batch signature):
//   S      worker streams;
//   W      most waves the grouped problems are dealt into (phase 2 of a wave
//          overlaps phases 1 / 3 of its neighbours; more waves shorten the
//          head and the tail of that pipeline, fewer make larger grouped grids);
//   slice  chunks of 32 columns of r per block of the grouped Gaussian stage
//          (longer slices: fewer partials to add, fewer blocks);
//   tiles  128-row tiles per CTA, at least, of the dense row norms (more: fewer
//          CTAs per problem, so problems on other streams share the SMs).
struct BatchTune {
    int S = 8, W = 4, slice = 128, tiles = 16;
};

struct LskBatch {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    std::vector<cudaStream_t> rstreams;   // phase 3 (row norms of the grouped problems)
    std::vector<cudaEvent_t> rdone;
    cudaEvent_t fork = nullptr;
    cudaStream_t gstream = nullptr;  // grouped launches
    cudaStream_t pstream = nullptr;  // grouped CountSketch preparation of the waves
    std::vector<cudaEvent_t> ev;     // wave events: [wave][stream] sketch done, then [wave] grouped done
    cudaStream_t cap = nullptr;      // capture stream (the caller's may be the legacy stream)
    std::vector<void*> ws;
    std::vector<size_t> ws_bytes;
    cudaGraphExec_t exec = nullptr;
    uint64_t exec_key = 0;
    std::map<uint64_t, struct BatchTune> tuned;   // batch signature -> schedule
    // grouped phases
    void* arena = nullptr;           // sketches, factors and scratch of the grouped problems
    size_t arena_bytes = 0;
    unsigned char* table = nullptr;  // device copy of the grouped launches' parameter table
    size_t table_bytes = 0;
    std::vector<unsigned char> table_host;   // what `table` holds
    std::vector<char> grouped;       // per item: takes the grouped path
    std::vector<int> wave;           // per grouped item: its wave
    std::vector<float*> SA, Rinv32;  // per grouped item: its sketch and FP32 R^-1 in the arena
    std::vector<uint32_t*> cidx;     // per compacted item: the buckets of its sketch's rows, then their count
    std::vector<CsGroup> cg;         // per wave: the grouped CountSketch preparation
    std::vector<RnImageGroup> ig;    // per wave: the row norms' B images (dense) ...
    std::vector<BbtGroup> mg;        // ... and B B^T (CSR), built after the wave's R^-1
    std::vector<void*> prepared;     // per grouped item: that operand
    std::vector<int64_t> cnt_base;   // per grouped item: its counters' offset in its wave's preparation
    int waves = 0;
    std::vector<GaussGroup> gg;      // per wave
    std::vector<QrGroup> qg;
};

namespace {

uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

// A grouped problem's sketch is compacted to its non-empty buckets when more
// than ~2% of the r buckets are expected empty (e^(-n/r) > e^-4): its
// Gaussian stage then draws G only for the columns that meet a row of A.
bool compacts(const lsk_batch_item& it) { return it.A.n < 4 * it.r; }
// The row norms' operand built for a grouped problem in phase 2: the
// tensor-core image of R^-1 (dense BF16) or R^-1 R^-T (CSR); 0: none.
size_t prepared_bytes(const lsk_batch_item& it, int32_t prec) {
    const lsk_mat* A = &it.A;
    if (A->kind == LSK_DENSE)
        return (prec == LSK_PREC_BF16 && rownorms_tc_supported(A, A->d, 1)) ? rownorms_tc_workspace_bytes(A, A->d, 1)
                                                                          : 0;
    return (size_t)A->d * A->d * 4;
}
int64_t sketch_rows(const lsk_batch_item& it) { return compacts(it) ? std::min<int64_t>(it.r, it.A.n) : it.r; }

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
    while ((int)b->rstreams.size() < S) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LSK_ERR_CUDA;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return LSK_ERR_CUDA;
        b->rstreams.push_back(s);
        b->rdone.push_back(e);
    }
    if (!b->fork && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return LSK_ERR_CUDA;
    if (!b->gstream && cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking) != cudaSuccess) return LSK_ERR_CUDA;
    if (!b->pstream && cudaStreamCreateWithFlags(&b->pstream, cudaStreamNonBlocking) != cudaSuccess) return LSK_ERR_CUDA;
    const size_t nev = (size_t)std::max(b->waves, 1) * (S + 2);
    while (b->ev.size() < nev) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return LSK_ERR_CUDA;
        b->ev.push_back(e);
    }
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
        for (int i : lanes[s]) {
            const lsk_mat* A = &items[i].A;
            if (b->grouped.size() == (size_t)0 || !b->grouped[i])
                need = std::max(need, leverage_workspace_bytes(A, items[i].r, items[i].k, prec, ctx->sm_count));
            else
                need = std::max(need, std::max(cs_workspace_bytes(A->n, items[i].r),
                                               rownorms_workspace_bytes(A, A->d, 1, prec)));
        }
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

// The whole batch on `main`'s timeline.  Worker stream s runs phase 1 of every
// wave back to back (and, with wave 0, the full pipelines of ungrouped
// problems); the grouped stream runs phase 2 of wave w once every worker has
// finished its phase 1 of w; row-norm stream s runs phase 3 of each wave once
// its phase 2 is done.  So the compute-bound grouped stages of one wave
// overlap the memory-bound passes over A of the others, and no gather waits
// for a grouped stage.  (Measured on the 512-problem batch with phase-boundary
// timestamps: the gathers of all waves end by ~17 ms, the four grouped stages
// -- ~4 ms of draws and ~1.5 ms of QR each -- run back to back on the grouped
// stream from the end of wave 0's slowest gathers, and the row norms of the
// last wave end the batch: 43-45 ms, as with phase 3 queued on the worker
// streams.)
cudaError_t record(lsk_ctx* ctx, cudaStream_t main, const std::vector<std::vector<int>>& lanes,
                   const lsk_batch_item* items, int32_t prec, const BatchTune& tune) {
    LskBatch* b = ctx->batch;
    const int S = (int)lanes.size(), W = b->waves;
    auto ev_sketch = [&](int w, int s) { return b->ev[(size_t)w * (S + 2) + s]; };
    auto ev_group = [&](int w) { return b->ev[(size_t)w * (S + 2) + S]; };
    auto ev_prep = [&](int w) { return b->ev[(size_t)w * (S + 2) + S + 1]; };
    cudaError_t e = cudaEventRecord(b->fork, main);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < S; ++s)
        if ((e = cudaStreamWaitEvent(b->streams[s], b->fork, 0)) != cudaSuccess) return e;
    if (W > 0 && (e = cudaStreamWaitEvent(b->gstream, b->fork, 0)) != cudaSuccess) return e;
    // phase 0: the CountSketch permutations of every wave, grouped, ahead of the gathers
    if (W > 0) {
        if ((e = cudaStreamWaitEvent(b->pstream, b->fork, 0)) != cudaSuccess) return e;
        for (int w = 0; w < W; ++w) {
            if ((e = cs_group_launch(b->cg[w], b->table, ctx->sm_count, b->pstream)) != cudaSuccess) return e;
            if ((e = cudaEventRecord(ev_prep(w), b->pstream)) != cudaSuccess) return e;
        }
    }

    auto phase1 = [&](int s, int w) -> cudaError_t {
        cudaStream_t st = b->streams[s];
        bool prepared = false;   // this stream waits for wave w's permutations before its first gather
        for (int i : lanes[s]) {
            const lsk_batch_item& it = items[i];
            cudaError_t er = cudaSuccess;
            if (b->grouped[i]) {
                if (b->wave[i] == w) {
                    if (!prepared && (er = cudaStreamWaitEvent(st, ev_prep(w), 0)) != cudaSuccess) return er;
                    prepared = true;
                    const CsGroup& g = b->cg[w];
                    er = cs_gather_launch(&it.A, it.r, g.off + b->cnt_base[i], g.perm,
                                          b->cidx[i] ? g.cpos + b->cnt_base[i] : nullptr, b->SA[i], ctx->flag,
                                          ctx->sm_count, st);
                }
            } else if (w == 0) {
                er = leverage_pipeline(&it.A, it.r, it.k, it.seed, prec, it.ell, nullptr, b->ws[s], ctx->flag,
                                       ctx->sm_count, st);
            }
            if (er != cudaSuccess) return er;
        }
        return W > 0 ? cudaEventRecord(ev_sketch(w, s), st) : cudaSuccess;
    };
    auto phase3 = [&](int s, int w) -> cudaError_t {
        cudaStream_t st = b->rstreams[s];
        cudaError_t er = cudaStreamWaitEvent(st, ev_group(w), 0);
        for (int i : lanes[s]) {
            if (er != cudaSuccess) return er;
            if (!b->grouped[i] || b->wave[i] != w) continue;
            const lsk_batch_item& it = items[i];
            // the operand was built in phase 2: the workspace is not touched
            er = rownorms_launch(&it.A, b->Rinv32[i], it.A.d, 1.0, 0.0, 1, prec, it.ell, nullptr, ctx->flag,
                                 ctx->sm_count, st, tune.tiles, b->prepared[i]);
        }
        return er;
    };
    auto phase2 = [&](int w) -> cudaError_t {
        cudaError_t er;
        for (int s = 0; s < S; ++s)
            if ((er = cudaStreamWaitEvent(b->gstream, ev_sketch(w, s), 0)) != cudaSuccess) return er;
        if ((er = gauss_group_launch(b->gg[w], b->table, b->gstream)) != cudaSuccess) return er;
        if ((er = qr_group_launch(b->qg[w], b->table, b->gstream)) != cudaSuccess) return er;
        if ((er = rownorms_image_group_launch(b->ig[w], b->table, b->gstream)) != cudaSuccess) return er;
        if ((er = bbt_group_launch(b->mg[w], b->table, b->gstream)) != cudaSuccess) return er;
        return cudaEventRecord(ev_group(w), b->gstream);
    };

    // worker streams: the gathers of every wave back to back; the grouped
    // stream: phase 2 of each wave once its gathers are in; phase 3 on a
    // stream pool of its own (its operands are in the arena), so no gather
    // waits behind a row norm that waits for a grouped stage
    for (int s = 0; s < S; ++s)
        for (int w = 0; w < std::max(W, 1); ++w)
            if ((e = phase1(s, w)) != cudaSuccess) return e;
    for (int w = 0; w < W; ++w)
        if ((e = phase2(w)) != cudaSuccess) return e;
    for (int s = 0; s < S; ++s) {
        if (W > 0) {
            if ((e = cudaStreamWaitEvent(b->rstreams[s], b->fork, 0)) != cudaSuccess) return e;
            for (int w = 0; w < W; ++w)
                if ((e = phase3(s, w)) != cudaSuccess) return e;
            if ((e = cudaEventRecord(b->rdone[s], b->rstreams[s])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(main, b->rdone[s], 0)) != cudaSuccess) return e;
        }
        if ((e = cudaEventRecord(b->done[s], b->streams[s])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(main, b->done[s], 0)) != cudaSuccess) return e;
    }
    if (W > 0 && (e = cudaStreamWaitEvent(main, ev_group(W - 1), 0)) != cudaSuccess) return e;
    if (W > 0 && (e = cudaStreamWaitEvent(main, ev_prep(W - 1), 0)) != cudaSuccess) return e;
    return cudaSuccess;
}

constexpr int kMaxWaves = 16;          // grouped problems are split into up to 16 waves
constexpr int kMinWaveProblems = 16;   // of at least 16 problems each

bool groupable(const lsk_batch_item& it, int32_t prec) {
    return prec == LSK_PREC_BF16 && it.k > 0 && it.A.n > 0 && gauss_tc_supported(it.r, it.A.d, it.k) &&
           qr_group_supported(it.k, it.A.d);
}

// Arena layout of the grouped problems, their launch tables, and the upload
// of the tables (only when they changed; the previous batch on the context
// stream is finished first, since it may still read the old table).
int prepare_groups(lsk_ctx* ctx, const lsk_batch_item* items, int count, int32_t prec, bool allow,
                   const BatchTune& tune) {
    LskBatch* b = ctx->batch;
    b->grouped.assign(count, 0);
    b->SA.assign(count, nullptr);
    b->Rinv32.assign(count, nullptr);
    b->cidx.assign(count, nullptr);
    b->cnt_base.assign(count, 0);
    b->prepared.assign(count, nullptr);
    for (int i = 0; i < count; ++i) b->grouped[i] = (allow && groupable(items[i], prec)) ? 1 : 0;
    // waves: grouped problems by decreasing cost, dealt round-robin
    std::vector<int> order;
    for (int i = 0; i < count; ++i)
        if (b->grouped[i]) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost_of(items[x]) > cost_of(items[y]); });
    const int ng = (int)order.size();
    b->waves = ng == 0 ? 0 : std::max(1, std::min(std::min(tune.W, kMaxWaves), ng / kMinWaveProblems));
    b->wave.assign(count, 0);
    for (int q = 0; q < ng; ++q) b->wave[order[q]] = q % std::max(b->waves, 1);
    std::vector<int64_t> wrows(b->waves, 0), wcnt(b->waves, 0);
    size_t bytes = 0;
    for (int i = 0; i < count; ++i) {
        if (!b->grouped[i]) continue;
        const int64_t rs = sketch_rows(items[i]), k = items[i].k, d = items[i].A.d;
        bytes += ws_round((size_t)rs * d * 4) + ws_round((size_t)k * d * 4) +
                 gauss_group_part_bytes(rs, d, k, tune.slice) + ws_round(qr_workspace_bytes(k, d)) +
                 ws_round((size_t)d * d * 4) + (compacts(items[i]) ? ws_round((size_t)(rs + 1) * 4) : 0) +
                 ws_round(prepared_bytes(items[i], prec));
        wrows[b->wave[i]] += items[i].A.n;
        wcnt[b->wave[i]] += items[i].r + 1;
    }
    for (int w = 0; w < b->waves; ++w) bytes += cs_group_ws_bytes(wrows[w], wcnt[w]);
    if (bytes > b->arena_bytes) {
        cudaStreamSynchronize(ctx->stream);
        if (b->arena) cudaFree(b->arena);
        b->arena = nullptr;
        b->arena_bytes = 0;
        if (cudaMalloc(&b->arena, bytes) != cudaSuccess) {
            cudaGetLastError();
            snprintf(ctx->err, sizeof(ctx->err), "batch: no room for the grouped arena (%zu bytes)", bytes);
            return LSK_ERR_OOM;
        }
        b->arena_bytes = bytes;
    }
    std::vector<std::vector<GaussJob>> gj(b->waves);
    std::vector<std::vector<QrJob>> qj(b->waves);
    std::vector<std::vector<CsJob>> cj(b->waves);
    std::vector<std::vector<RnImageJob>> imj(b->waves);
    std::vector<std::vector<BbtJob>> bbj(b->waves);
    std::vector<std::vector<int>> cj_item(b->waves);
    WsCarver wc{(char*)b->arena, 0};
    for (int i = 0; i < count; ++i) {
        if (!b->grouped[i]) continue;
        const int64_t rs = sketch_rows(items[i]), k = items[i].k, d = items[i].A.d;
        float* SA = wc.take<float>((size_t)rs * d);
        float* GSA = wc.take<float>((size_t)k * d);
        float* part = (float*)wc.take<char>(gauss_group_part_bytes(rs, d, k, tune.slice));
        void* qws = wc.take<char>(qr_workspace_bytes(k, d));
        float* Ri32 = wc.take<float>((size_t)d * d);
        uint32_t* cidx = compacts(items[i]) ? wc.take<uint32_t>((size_t)rs + 1) : nullptr;
        const size_t pb = prepared_bytes(items[i], prec);
        void* prep = pb ? (void*)wc.take<char>(pb) : nullptr;
        b->prepared[i] = prep;
        if (prep && items[i].A.kind == LSK_DENSE)
            imj[b->wave[i]].push_back(RnImageJob{items[i].A, Ri32, d, 1, (uint8_t*)prep});
        else if (prep)
            bbj[b->wave[i]].push_back(BbtJob{Ri32, d, d, (float*)prep});
        b->SA[i] = SA;
        b->Rinv32[i] = Ri32;
        b->cidx[i] = cidx;
        GaussJob gjob{SA, rs, d, k, items[i].seed, GSA, part, tune.slice};
        if (cidx) {
            gjob.idx = cidx;
            gjob.rcount = cidx + rs;
        }
        gj[b->wave[i]].push_back(gjob);
        cj[b->wave[i]].push_back(CsJob{items[i].A.n, items[i].r, items[i].seed, cidx, cidx ? cidx + rs : nullptr, 0});
        cj_item[b->wave[i]].push_back(i);
        QrJob q{};
        qr_group_job(q, GSA, k, d, qws, nullptr, Ri32, ctx->flag);
        qj[b->wave[i]].push_back(q);
    }
    HostTable t;
    b->gg.assign(b->waves, GaussGroup{});
    b->qg.assign(b->waves, QrGroup{});
    b->cg.assign(b->waves, CsGroup{});
    b->ig.assign(b->waves, RnImageGroup{});
    b->mg.assign(b->waves, BbtGroup{});
    for (int w = 0; w < b->waves; ++w) {
        gauss_group_build(gj[w], t, b->gg[w]);
        qr_group_build(qj[w], t, b->qg[w]);
        void* cws = wc.take<char>(cs_group_ws_bytes(wrows[w], wcnt[w]));
        cs_group_build(cj[w], cws, t, b->cg[w]);
        for (size_t q = 0; q < cj[w].size(); ++q) b->cnt_base[cj_item[w][q]] = cj[w][q].cnt_base;
        rownorms_image_group_build(imj[w], t, b->ig[w]);
        bbt_group_build(bbj[w], t, b->mg[w]);
    }
    if (t.bytes.empty()) return LSK_OK;
    if (t.bytes != b->table_host || !b->table) {
        cudaStreamSynchronize(ctx->stream);
        if (t.bytes.size() > b->table_bytes) {
            if (b->table) cudaFree(b->table);
            b->table = nullptr;
            b->table_bytes = 0;
            if (cudaMalloc(&b->table, t.bytes.size()) != cudaSuccess) {
                cudaGetLastError();
                return LSK_ERR_OOM;
            }
            b->table_bytes = t.bytes.size();
        }
        if (cudaMemcpy(b->table, t.bytes.data(), t.bytes.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            snprintf(ctx->err, sizeof(ctx->err), "batch: table upload failed");
            return LSK_ERR_CUDA;
        }
        b->table_host.swap(t.bytes);
    }
    return LSK_OK;
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

uint64_t exact_key(const LskBatch* b, const lsk_batch_item* items, int count, int32_t prec, const BatchTune& t) {
    uint64_t h = fnv(signature(items, count, prec), &t, sizeof(t));
    const int fused = fused_sketch_on();   // ungrouped problems' sketch path is recorded in the graph
    h = fnv(h, &fused, sizeof(fused));
    h = fnv(h, &b->arena, sizeof(b->arena));
    h = fnv(h, &b->table, sizeof(b->table));
    for (size_t s = 0; s < b->ws.size(); ++s) h = fnv(h, &b->ws[s], sizeof(void*));
    return fnv(h, items, sizeof(lsk_batch_item) * (size_t)count);
}

// LSK_AUTOTUNE_CACHE: one line per tuned batch, "signature S W slice tiles"
bool cache_lookup(uint64_t sig, BatchTune& out) {
    const char* path = getenv("LSK_AUTOTUNE_CACHE");
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    unsigned long long k;
    BatchTune t;
    bool found = false;
    while (fscanf(f, "%llx %d %d %d %d", &k, &t.S, &t.W, &t.slice, &t.tiles) == 5)
        if (k == sig && t.S > 0 && t.W > 0 && t.slice > 0 && t.tiles > 0) {
            out = t;
            found = true;
        }
    fclose(f);
    return found;
}

void cache_store(uint64_t sig, const BatchTune& t) {
    const char* path = getenv("LSK_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%llx %d %d %d %d\n", (unsigned long long)sig, t.S, t.W, t.slice, t.tiles);
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
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    for (cudaStream_t st : b->rstreams) cudaStreamDestroy(st);
    for (cudaEvent_t e : b->rdone) cudaEventDestroy(e);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    if (b->pstream) cudaStreamDestroy(b->pstream);
    if (b->arena) cudaFree(b->arena);
    if (b->table) cudaFree(b->table);
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
    prec = sketch_prec(prec);   // a batch's row norms take the prepared BF16x3 images
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
    const bool allow_groups = !(flags & LSK_BATCH_PER_PROBLEM);
    const int forced_S = flags & LSK_BATCH_STREAMS_MASK;

    // the schedule: remembered for this signature, else from the cache file,
    // else tuned (LSK_BATCH_AUTOTUNE), else the defaults
    BatchTune tune;
    bool have = false;
    {
        auto it = b->tuned.find(sig);
        if (it != b->tuned.end()) {
            tune = it->second;
            have = true;
        } else if (cache_lookup(sig, tune)) {
            b->tuned[sig] = tune;
            have = true;
        }
    }
    // set up streams, arena, tables and workspaces for a schedule
    auto setup = [&](const BatchTune& t, std::vector<std::vector<int>>& lanes) -> int {
        int rc = prepare_groups(ctx, items, count, prec, allow_groups, t);
        if (rc) return rc;
        if ((rc = ensure_streams(ctx, t.S))) return rc;
        lanes = plan(items, count, t.S);
        return size_workspaces(ctx, lanes, items, prec);
    };
    if (!have && (flags & LSK_BATCH_AUTOTUNE)) {
        // coordinate descent over the knobs, each candidate timed on the
        // batch itself (outside any capture; the first of two passes warms up)
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        auto time_of = [&](const BatchTune& t, float& ms) -> int {
            std::vector<std::vector<int>> lanes;
            int rc = setup(t, lanes);
            if (rc) return rc;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(e0, ctx->stream);
                const cudaError_t e = record(ctx, ctx->stream, lanes, items, prec, t);
                if (e != cudaSuccess) {
                    snprintf(ctx->err, sizeof(ctx->err), "batch: %s", cudaGetErrorString(e));
                    return LSK_ERR_CUDA;
                }
                cudaEventRecord(e1, ctx->stream);
            }
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            return LSK_OK;
        };
        BatchTune best;
        if (forced_S) best.S = forced_S;
        best.S = std::min(best.S, count);
        float best_ms = 0.f;
        int rc = time_of(best, best_ms);
        if (rc) return rc;
        const std::vector<int> Ws = {2, 4, 8, 16}, Ss = {2, 4, 8, 16}, slices = {64, 128, 256}, tiles = {8, 16, 32};
        auto sweep = [&](const std::vector<int>& vals, int BatchTune::*knob) -> int {
            for (int v : vals) {
                if (best.*knob == v) continue;
                BatchTune t = best;
                t.*knob = v;
                if (t.S > count) continue;
                float ms = 0.f;
                const int r = time_of(t, ms);
                if (r) return r;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
            return LSK_OK;
        };
        if ((rc = sweep(Ws, &BatchTune::W))) return rc;
        if (!forced_S && (rc = sweep(Ss, &BatchTune::S))) return rc;
        if ((rc = sweep(slices, &BatchTune::slice))) return rc;
        if ((rc = sweep(tiles, &BatchTune::tiles))) return rc;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        tune = best;
        b->tuned[sig] = tune;
        cache_store(sig, tune);
    }
    if (forced_S) tune.S = forced_S;
    tune.S = std::max(1, std::min(tune.S, count));

    std::vector<std::vector<int>> lanes;
    int rc = setup(tune, lanes);
    if (rc) return rc;

    if (!(flags & LSK_BATCH_GRAPH)) {
        cudaError_t e = record(ctx, ctx->stream, lanes, items, prec, tune);
        if (e != cudaSuccess) {
            snprintf(ctx->err, sizeof(ctx->err), "batch: %s", cudaGetErrorString(e));
            return LSK_ERR_CUDA;
        }
        return LSK_OK;
    }
    const uint64_t key = exact_key(b, items, count, prec, tune);
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
            const cudaError_t er = record(ctx, b->cap, lanes, items, prec, tune);
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
    auto it = ctx->batch->tuned.find(signature(items, count, sketch_prec(prec)));
    return it == ctx->batch->tuned.end() ? 0 : it->second.S;
}

extern "C" int lsk_batch_schedule(lsk_ctx* ctx, int32_t count, const lsk_batch_item* items, int32_t prec,
                                  int32_t* out) {
    BatchTune t;
    int known = 0;
    if (ctx && ctx->batch && items) {
        auto it = ctx->batch->tuned.find(signature(items, count, sketch_prec(prec)));
        if (it != ctx->batch->tuned.end()) {
            t = it->second;
            known = 1;
        }
    }
    if (out) {
        out[0] = t.S;
        out[1] = t.W;
        out[2] = t.slice;
        out[3] = t.tiles;
    }
    return known;
}
