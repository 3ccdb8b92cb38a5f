// prof.cu -- storage and resolution of the per-kernel event timings.
#include "lsk_internal.cuh"
#include "prof.cuh"

#include <string.h>

#include <map>
#include <string>
#include <vector>

struct LskProf {
    struct Pending {
        const char* name;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<long long, double>> totals;   // name -> (launches, ms)
    std::vector<std::string> order;
    const char* open_name = nullptr;
    cudaEvent_t open_ev = nullptr;

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    void resolve() {
        for (auto& p : pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                auto it = totals.find(p.name);
                if (it == totals.end()) {
                    order.push_back(p.name);
                    totals[p.name] = {1, (double)ms};
                } else {
                    it->second.first += 1;
                    it->second.second += ms;
                }
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
    ~LskProf() {
        for (auto& p : pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

thread_local LskProf* lsk_prof_current = nullptr;

void lsk_prof_begin(const char* name, cudaStream_t st) {
    LskProf* p = lsk_prof_current;
    p->open_name = name;
    p->open_ev = p->get();
    cudaEventRecord(p->open_ev, st);
}

void lsk_prof_end(cudaStream_t st) {
    LskProf* p = lsk_prof_current;
    cudaEvent_t b = p->get();
    cudaEventRecord(b, st);
    p->pending.push_back({p->open_name, p->open_ev, b});
    p->open_ev = nullptr;
}

LskProf* lsk_prof_new() { return new LskProf(); }
void lsk_prof_delete(LskProf* p) { delete p; }

extern "C" {

int lsk_profile_enable(lsk_ctx* ctx, int on) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    if (on && !ctx->prof) ctx->prof = lsk_prof_new();
    ctx->prof_on = on ? 1 : 0;
    return LSK_OK;
}

int lsk_profile_reset(lsk_ctx* ctx) {
    if (!ctx) return LSK_ERR_INVALID_ARG;
    if (ctx->prof) {
        ctx->prof->resolve();
        ctx->prof->totals.clear();
        ctx->prof->order.clear();
    }
    return LSK_OK;
}

int lsk_profile_count(lsk_ctx* ctx) {
    if (!ctx || !ctx->prof) return 0;
    ctx->prof->resolve();
    return (int)ctx->prof->order.size();
}

int lsk_profile_get(lsk_ctx* ctx, int idx, char* name, size_t name_len, long long* launches,
                    double* total_ms) {
    if (!ctx || !ctx->prof) return LSK_ERR_INVALID_ARG;
    ctx->prof->resolve();
    if (idx < 0 || idx >= (int)ctx->prof->order.size()) return LSK_ERR_INVALID_ARG;
    const std::string& nm = ctx->prof->order[idx];
    const auto& t = ctx->prof->totals[nm];
    if (name && name_len) {
        strncpy(name, nm.c_str(), name_len - 1);
        name[name_len - 1] = 0;
    }
    if (launches) *launches = t.first;
    if (total_ms) *total_ms = t.second;
    return LSK_OK;
}

}  // extern "C"

// ---- dynamic shared memory limits (see lsk_internal.cuh) ----------------------
#include <mutex>
#include <set>
#include <utility>

cudaError_t allow_dynamic_smem(const void* fn) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({fn, dev})) return cudaSuccess;
    cudaFuncAttributes a;
    if ((e = cudaFuncGetAttributes(&a, fn)) != cudaSuccess) return e;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
    if (e == cudaSuccess) done.insert({fn, dev});
    return e;
}
