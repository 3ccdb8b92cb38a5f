// prof.cuh -- optional per-kernel CUDA-event timing.
//
// When a context has profiling on, the C-ABI layer points lsk_prof_current
// at the context's profiler for the duration of a call, and every launch site
// wrapped in LSK_PROF(...) records a start/end event pair on the launching
// stream.  Durations are resolved (after the caller synchronises) per kernel
// name: launches and total milliseconds.  Off by default; no cost when off.
#pragma once
#include <cuda_runtime.h>

struct LskProf;
extern thread_local LskProf* lsk_prof_current;

void lsk_prof_begin(const char* name, cudaStream_t st);
void lsk_prof_end(cudaStream_t st);

struct LskProfScope {
    cudaStream_t st;
    bool on;
    LskProfScope(const char* name, cudaStream_t s) : st(s), on(lsk_prof_current != nullptr) {
        if (on) lsk_prof_begin(name, st);
    }
    ~LskProfScope() {
        if (on) lsk_prof_end(st);
    }
};

#define LSK_PROF_CAT2(a, b) a##b
#define LSK_PROF_CAT(a, b) LSK_PROF_CAT2(a, b)
// LSK_PROF("name", stream) kernel<<<...>>>(...);
// Expands to "if (scope; false) {} else <statement>", so an enclosing
// if/else keeps its own else branch.
#define LSK_PROF(name, st) \
    if (LskProfScope LSK_PROF_CAT(_lsk_prof_, __LINE__){name, st}; false) { \
    } else
