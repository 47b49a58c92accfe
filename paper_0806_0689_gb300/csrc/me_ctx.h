// me_ctx.h -- host-side definition of the library context (me_ctx), shared
// by the C-ABI translation units.
#pragma once

#include "me.h"
#include "me_internal.cuh"

#include <map>
#include <string>

namespace me {

// One reusable upload slot: a device buffer [queue head | descriptor table],
// its pinned host twin and an event marking the last launch that used it.
struct Slot {
    void* dev = nullptr;
    void* host = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool used = false;
    void* queue = nullptr;  // DCDS item queue: items (16 B each) then flags (4 B each), flags zeroed
    size_t qcap = 0;        // entries
};

constexpr size_t kHeadBytes = 256;  // queue head (int) and padding before the table

}  // namespace me

struct me_ctx {
    int device = 0;
    int num_sms = 0;
    std::string err;
    std::string tune_path;
    std::map<std::string, me::Shape> tuned;
    me::Slot slots[ME_MAX_INFLIGHT];
    int next_slot = 0;
    unsigned* status = nullptr;  // device word written by kernels
    unsigned* sink = nullptr;    // microbenchmark sink
    struct me_proposal* median_ws = nullptr;  // wavefront buffers of the neighbour-median start (lazy)
};

struct me_graph {
    me_ctx* ctx = nullptr;
    void* dev = nullptr;    // [head | table]
    void* queue = nullptr;  // DCDS item queue (items, then zeroed flags)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};
