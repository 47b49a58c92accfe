// me_ctx.h -- host-side definition of the library context (me_ctx), shared
// by the C-ABI translation units.
#pragma once

#include "me.h"
#include "me_internal.cuh"

#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

namespace me {

// One reusable upload slot: a device buffer [queue head | descriptor table],
// its pinned host twin and an event marking the last launch that used it.
struct Slot {
    void* dev = nullptr;
    void* host = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool used = false;
};

constexpr size_t kHeadBytes = 256;  // the kernels' counter words and padding before the table

// Staging of me_estimate_host_batch: two sets of device buffers for a
// call's frames, FS fields and outputs (consecutive calls alternate, so one
// call's uploads can run while the previous call still searches), the two
// copy streams and the events that order them.
struct HostStage {
    void* dev = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;   // the last result copy of the call that used this set
};
struct HostPipe {
    HostStage stage[2];
    int next = 0;
    cudaStream_t in = nullptr;    // host-to-device copies
    cudaStream_t out = nullptr;   // device-to-host copies
    cudaEvent_t entry = nullptr;  // the caller's stream reached the call
    std::vector<cudaEvent_t> ev;  // per chunk: inputs uploaded, search done, results copied
};

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
    struct me_proposal* learned = nullptr;    // the context's own proposal (me_proposal_* with a NULL proposal)
    me::HostPipe pipe;                        // me_estimate_host_batch staging (lazy)
    int inject_wait_timeout = 0;              // failure-detection test hook (me_inject_wait_timeout)
    int tracing = 0;                          // me_set_tracing: NVTX ranges and CUDA events per call
    cudaEvent_t trace0 = nullptr, trace1 = nullptr;
    bool traced = false;                      // a traced call has recorded its events
};

namespace me {

// Tracing of a public call (me_set_tracing): an NVTX range around its host
// part and CUDA events around its work on its stream.  A call that ends by
// synchronising its stream closes the trace first, so that the events time
// the device work and not the wait.
struct Trace {
    me_ctx* c;
    cudaStream_t st;
    bool open = false;
    Trace(me_ctx* ctx, const char* name, cudaStream_t stream) : c(ctx), st(stream)
    {
        if (!c || !c->tracing) return;
        nvtxRangePushA(name);
        cudaEventRecord(c->trace0, st);
        open = true;
    }
    void close()
    {
        if (!open) return;
        cudaEventRecord(c->trace1, st);
        c->traced = true;
        nvtxRangePop();
        open = false;
    }
    ~Trace() { close(); }
    Trace(const Trace&) = delete;
    Trace& operator=(const Trace&) = delete;
};

}  // namespace me

struct me_graph {
    me_ctx* ctx = nullptr;
    void* dev = nullptr;    // [head | table]
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};
