// me_api.cu -- the C-ABI of libme (declared in include/me.h): argument checks,
// descriptor tables, the work-queue counters, CUDA-graph capture, the launch
// shape tuner and the byte-absdiff microbenchmark.  All arithmetic of the
// motion search runs in the kernels of dcds.cu, fs.cu and eval.cu.
#include "me.h"
#include "me_ctx.h"
#include "me_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

using me::EvalDev;
using me::FrameDev;
using me::Shape;
using me::Slot;
using me::Trace;
using me::kHeadBytes;

#ifndef ME_DCDS_STAGES
#define ME_DCDS_STAGES 1     // default tile staging of the DCDS kernel
#endif
#ifndef ME_DCDS_THREADS
#define ME_DCDS_THREADS 128  // default CTA size of the 16x16 DCDS kernel
#endif

namespace {

int fail(me_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(me_ctx* c, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, ME_ERR_CUDA, m);
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

std::string shape_key(int algo, int block, int range, int w, int h)
{
    std::ostringstream o;
    o << algo << " " << block << " " << range << " " << w << "x" << h;
    return o.str();
}

// K (candidate rows per FS thread): the fewest thread-rows of work for the
// 2R+1 rows of candidates, counting about three rows of fixed cost per task
// (its current block, its key reduction); ties go to the larger K.
int fs_pick_k(int range)
{
    const int ks[5] = {9, 11, 13, 15, 33};
    const int n = 2 * range + 1;
    int best = 9, bc = 1 << 30;
    for (int k : ks) {
        const int cost = ((n + k - 1) / k) * (k + 3);
        if (cost <= bc) { bc = cost; best = k; }
    }
    return best;
}

// FS tile width: the fewest idle threads over the tasks of a tile, with two
// CTAs per SM (shared memory <= 112 KB).
int fs_pick_tx(int block, int range, int k)
{
    const int ndx = 2 * range + 1;
    const int tpb = ndx * ((ndx + k - 1) / k);
    Shape t{};
    t.threads = 256;
    t.k = k;
    double be = -1.0;
    int bt = 0;
    for (int tx = 32; tx >= 2; tx -= (block == 8 ? 2 : 1)) {  // widest first: less halo per block on ties
        t.tx = tx;
        if (!me::fs_shape_ok(block, range, t) || me::fs_smem_bytes(block, range, t) > 112 * 1024) continue;
        const long nt = (long)tx * tpb;
        const double e = (double)nt / (double)(((nt + 255) / 256) * 256);
        if (e > be + 1e-3) { be = e; bt = tx; }
    }
    return bt > 0 ? bt : 2;
}

Shape default_shape(me_ctx* c, int algo, int block, int range)
{
    Shape s{};
    if (algo == ME_ALGO_FS) {
        s.k = fs_pick_k(range);
        s.threads = 256;
        s.ty = 1;
        s.ctas_per_sm = 0;
        s.tx = fs_pick_tx(block, range, s.k);
        return s;
    }
    // 8x8 tiles hold four times the blocks: 256 threads measured 6-14 % faster
    // than 128 on CIF (+-7, +-15), 1080p (+-16) and 2160p (+-32) batches
    s.threads = block == 8 ? 256 : ME_DCDS_THREADS;
    s.tx = me::kTile / block;
    s.ty = me::kDcdsTileH / block;
    s.k = 0;
    s.ctas_per_sm = 0;  // from the occupancy of the kernel
    s.stages = ME_DCDS_STAGES;
    (void)c;
    return s;
}

Shape pick_shape(me_ctx* c, int algo, int block, int range, int w, int h)
{
    auto it = c->tuned.find(shape_key(algo, block, range, w, h));
    if (it != c->tuned.end()) return it->second;
    return default_shape(c, algo, block, range);
}

int check_frame(me_ctx* c, const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch, int block,
                int range, const void* mv, const void* sad, const void* nsp)
{
    if (!cur || !ref) return fail(c, ME_ERR_ARG, "cur/ref must not be NULL");
    if (!aligned(cur, 16) || !aligned(ref, 16)) return fail(c, ME_ERR_ARG, "cur/ref must be 16-byte aligned");
    if (block != 8 && block != 16) return fail(c, ME_ERR_ARG, "block must be 8 or 16");
    if (w <= 0 || h <= 0) return fail(c, ME_ERR_ARG, "w and h must be positive");
    if (w % 16 || w % block || h % block) return fail(c, ME_ERR_ARG, "w must be a multiple of 16 and of block, h of block");
    if (pitch < w || pitch % 16) return fail(c, ME_ERR_ARG, "pitch must be >= w and a multiple of 16");
    if (range < 1 || range > ME_MAX_RANGE) return fail(c, ME_ERR_ARG, "range must be in 1..32");
    if (!mv || !sad) return fail(c, ME_ERR_ARG, "mv and sad must not be NULL");
    if (!aligned(mv, 4) || !aligned(sad, 4)) return fail(c, ME_ERR_ARG, "mv and sad must be 4-byte aligned");
    if (nsp && !aligned(nsp, 2)) return fail(c, ME_ERR_ARG, "nsp must be 2-byte aligned");
    return ME_OK;
}

// Take the next upload slot, wait for its previous launch, make it hold `bytes`.
int take_slot(me_ctx* c, size_t bytes, Slot** out)
{
    Slot& s = c->slots[c->next_slot];
    c->next_slot = (c->next_slot + 1) % ME_MAX_INFLIGHT;
    cudaError_t e;
    if (s.used) {
        e = cudaEventSynchronize(s.done);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
    }
    if (s.cap < bytes) {
        if (s.dev) cudaFree(s.dev);
        if (s.host) cudaFreeHost(s.host);
        s.dev = s.host = nullptr;
        s.cap = 0;
        size_t cap = std::max<size_t>(bytes, 64 * 1024);
        e = cudaMalloc(&s.dev, cap);
        if (e != cudaSuccess) return fail(c, ME_ERR_NOMEM, "cudaMalloc of a descriptor table failed");
        e = cudaMallocHost(&s.host, cap);
        if (e != cudaSuccess) return fail(c, ME_ERR_NOMEM, "cudaMallocHost of a descriptor table failed");
        s.cap = cap;
    }
    if (!s.done) {
        e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
    }
    *out = &s;
    return ME_OK;
}

// Fused evaluation of a DCDS batch: mv_fs (host array of n device pointers,
// nullable) and the device sums [n][ME_NSUMS].  d8 (FS only): the 8x8 outputs
// of the two-size full search.
struct EvalArgs {
    const int16_t* const* mv_fs = nullptr;
    uint64_t* sums = nullptr;
    const me_frame_desc* d8 = nullptr;
};

// Fill the device-side table (tiles per frame, TMA maps for DCDS) into
// `table`; returns the number of tiles, or -1 if a tensor map is rejected.
int build_table(const me_frame_desc* d, int n, int block, const Shape& s, bool fs, FrameDev* table,
                int* max_range, const EvalArgs* ev = nullptr)
{
    int tiles = 0, mr = 1;
    for (int i = 0; i < n; ++i) mr = std::max(mr, d[i].range);
    const me::FsGeom g = fs ? me::fs_geom(block, mr, s.tx, s.k) : me::FsGeom{};
    for (int i = 0; i < n; ++i) {
        FrameDev f{};
        f.cur = d[i].cur;
        f.ref = d[i].ref;
        f.mv = d[i].mv;
        f.sad = d[i].sad;
        f.nsp = d[i].nsp;
        f.w = d[i].w;
        f.h = d[i].h;
        f.pitch = d[i].pitch;
        f.range = d[i].range;
        f.nbx = d[i].w / block;
        f.nby = d[i].h / block;
        if (fs) {
            f.tiles_x = (f.nbx + s.tx - 1) / s.tx;
            f.tiles_y = f.nby;
            if (!me::encode_fs_maps(f, g.nch, me::fs_rows(block, f.range, s.k), s.tx * block, block)) return -1;
        } else {
            f.tiles_x = (f.w + me::kTile - 1) / me::kTile;
            f.tiles_y = (f.h + me::kDcdsTileH - 1) / me::kDcdsTileH;
            if (!me::encode_frame_maps(f, me::kDcdsTileH)) return -1;
        }
        if (ev && ev->sums) {
            f.sums = reinterpret_cast<unsigned long long*>(ev->sums) + (size_t)ME_NSUMS * i;
            f.mv_fs = ev->mv_fs ? ev->mv_fs[i] : nullptr;
        }
        if (ev && ev->d8) {
            f.mv8 = ev->d8[i].mv;
            f.sad8 = ev->d8[i].sad;
            f.nsp8 = ev->d8[i].nsp;
        }
        f.tile_base = tiles;
        tiles += f.tiles_x * f.tiles_y;
        table[i] = f;
    }
    me::set_uniform_tiles(table, n);
    *max_range = mr;
    return tiles;
}

int validate_batch(me_ctx* c, const me_frame_desc* d, int n, int block, int algo)
{
    if (!d || n <= 0) return fail(c, ME_ERR_ARG, "descs must not be NULL and n must be positive");
    if (algo != ME_ALGO_FS && algo != ME_ALGO_DCDS && algo != ME_ALGO_DCDS_S && algo != ME_ALGO_DCDS_LEARNED)
        return fail(c, ME_ERR_ARG, "unknown algo");
    if (algo == ME_ALGO_DCDS_LEARNED && !c->learned)
        return fail(c, ME_ERR_ARG, "learned start: no proposal weights loaded into the context (me_proposal_load)");
    for (int i = 0; i < n; ++i) {
        int rc = check_frame(c, d[i].cur, d[i].ref, d[i].w, d[i].h, d[i].pitch, block, d[i].range, d[i].mv,
                             d[i].sad, d[i].nsp);
        if (rc != ME_OK) {
            c->err = "descriptor " + std::to_string(i) + ": " + c->err;
            return rc;
        }
    }
    return ME_OK;
}

// Launch the search over a table already on the device at `dev`.
cudaError_t launch_search(me_ctx* c, void* dev, int n, int ntiles, int block, int algo, int max_range,
                          const Shape& s, cudaStream_t st, const EvalArgs* ev = nullptr)
{
    int* head = reinterpret_cast<int*>(dev);
    const FrameDev* table = reinterpret_cast<const FrameDev*>(reinterpret_cast<char*>(dev) + kHeadBytes);
    cudaError_t e = cudaMemsetAsync(head, 0, me::kCounterInts * sizeof(int), st);
    if (e != cudaSuccess) return e;
    // failure-detection test hook: a non-zero last counter word makes the DCDS
    // kernel arm its first copies for bytes that never arrive
    if (c->inject_wait_timeout && algo != ME_ALGO_FS) {
        e = cudaMemsetAsync(head + me::kCounterInts - 1, 1, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    if (ev && ev->sums) {
        // the fused evaluation runs in the tile-phase kernel; its sums accumulate from zero
        e = cudaMemsetAsync(ev->sums, 0, sizeof(uint64_t) * ME_NSUMS * (size_t)n, st);
        if (e != cudaSuccess) return e;
        Shape t = s;
        t.threads = 128;  // the fused variant uses more registers: small CTAs keep four per SM
        return me::launch_dcds(table, n, ntiles, block, max_range, algo == ME_ALGO_DCDS_S, t, head, c->status,
                               c->num_sms, st, true);
    }
    if (algo == ME_ALGO_FS)
        return me::launch_fs(table, n, ntiles, block, max_range, s, head, c->status, c->num_sms, st,
                             ev && ev->d8);
    return me::launch_dcds(table, n, ntiles, block, max_range, algo == ME_ALGO_DCDS_S, s, head, c->status,
                           c->num_sms, st);
}

int run_batch(me_ctx* c, const me_frame_desc* d, int n, int block, int algo, const Shape& s, cudaStream_t st,
              const EvalArgs* ev = nullptr)
{
    const size_t bytes = kHeadBytes + sizeof(FrameDev) * (size_t)n;
    Slot* slot = nullptr;
    int rc = take_slot(c, bytes, &slot);
    if (rc != ME_OK) return rc;
    FrameDev* table = reinterpret_cast<FrameDev*>(reinterpret_cast<char*>(slot->host) + kHeadBytes);
    int max_range = 1;
    const int ntiles = build_table(d, n, block, s, algo == ME_ALGO_FS, table, &max_range, ev);
    if (ntiles < 0) return fail(c, ME_ERR_CUDA, "cuTensorMapEncodeTiled rejected a frame description");
    cudaError_t e = cudaMemcpyAsync(slot->dev, slot->host, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "descriptor upload");
    e = launch_search(c, slot->dev, n, ntiles, block, algo, max_range, s, st, ev);
    if (e != cudaSuccess) return cuda_fail(c, e, "search launch");
    e = cudaEventRecord(slot->done, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
    slot->used = true;
    return ME_OK;
}

void load_tune_cache(me_ctx* c)
{
    if (c->tune_path.empty()) return;
    std::ifstream f(c->tune_path);
    std::string line;
    while (std::getline(f, line)) {
        // algo block range WxH tx ty threads k stages
        std::istringstream is(line);
        int algo, block, range, tx, ty, th, k, stages;
        std::string wh;
        if (is >> algo >> block >> range >> wh >> tx >> ty >> th >> k >> stages) {
            int w = 0, h = 0;
            if (sscanf(wh.c_str(), "%dx%d", &w, &h) == 2) {
                Shape s{tx, ty, th, 0, k, stages};
                c->tuned[shape_key(algo, block, range, w, h)] = s;
            }
        }
    }
}

}  // namespace

extern "C" {

int me_init(me_ctx** out, int cuda_device, const char* tune_cache_path)
{
    if (!out) return ME_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return ME_ERR_CUDA;
    if (cuda_device < 0 || cuda_device >= ndev) return ME_ERR_ARG;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, cuda_device) != cudaSuccess) return ME_ERR_CUDA;
    if (p.major != 10 || p.minor != 3) return ME_ERR_CUDA;  // the kernels are built for sm_103a only
    if (cudaSetDevice(cuda_device) != cudaSuccess) return ME_ERR_CUDA;
    me_ctx* c = new me_ctx();
    c->device = cuda_device;
    c->num_sms = p.multiProcessorCount;
    if (tune_cache_path) c->tune_path = tune_cache_path;
    if (cudaMalloc(&c->status, 256) != cudaSuccess || cudaMemset(c->status, 0, 256) != cudaSuccess) {
        delete c;
        return ME_ERR_NOMEM;
    }
    c->sink = c->status + 32;
    load_tune_cache(c);
    *out = c;
    return ME_OK;
}

void me_free(me_ctx* c)
{
    if (!c) return;
    for (auto& s : c->slots) {
        if (s.done) cudaEventDestroy(s.done);
        if (s.dev) cudaFree(s.dev);
        if (s.host) cudaFreeHost(s.host);
    }
    if (c->status) cudaFree(c->status);
    if (c->median_ws) me_proposal_free(c->median_ws);
    if (c->learned) me_proposal_free(c->learned);
    if (c->trace0) cudaEventDestroy(c->trace0);
    if (c->trace1) cudaEventDestroy(c->trace1);
    me::HostPipe& P = c->pipe;
    if (P.in) cudaStreamSynchronize(P.in);
    if (P.out) cudaStreamSynchronize(P.out);
    for (cudaEvent_t e : P.ev) cudaEventDestroy(e);
    if (P.entry) cudaEventDestroy(P.entry);
    if (P.in) cudaStreamDestroy(P.in);
    if (P.out) cudaStreamDestroy(P.out);
    for (me::HostStage& g : P.stage) {
        if (g.done) cudaEventDestroy(g.done);
        if (g.dev) cudaFree(g.dev);
    }
    delete c;
}

const char* me_last_error(const me_ctx* c) { return c ? c->err.c_str() : "null context"; }

int me_estimate(me_ctx* c, const uint8_t* cur, const uint8_t* ref, int w, int h, int block, int range, int algo,
                int16_t* mv, uint32_t* sad, uint16_t* nsp, void* stream)
{
    if (!c) return ME_ERR_ARG;
    Trace trace(c, "me_estimate", (cudaStream_t)stream);
    me_frame_desc d{cur, ref, w, h, w, range, mv, sad, nsp};
    int rc = validate_batch(c, &d, 1, block, algo);
    if (rc != ME_OK) return rc;
    if (algo == ME_ALGO_DCDS_LEARNED) return me_estimate_learned_batch(c, nullptr, &d, 1, block, nullptr, stream);
    return run_batch(c, &d, 1, block, algo, pick_shape(c, algo, block, range, w, h), (cudaStream_t)stream);
}

int me_estimate_batch(me_ctx* c, const me_frame_desc* descs, int n, int block, int algo, void* stream)
{
    if (!c) return ME_ERR_ARG;
    Trace trace(c, "me_estimate_batch", (cudaStream_t)stream);
    int rc = validate_batch(c, descs, n, block, algo);
    if (rc != ME_OK) return rc;
    if (algo == ME_ALGO_DCDS_LEARNED) return me_estimate_learned_batch(c, nullptr, descs, n, block, nullptr, stream);
    int mr = 1, mw = 0, mh = 0;
    for (int i = 0; i < n; ++i) { mr = std::max(mr, descs[i].range); mw = std::max(mw, descs[i].w); mh = std::max(mh, descs[i].h); }
    return run_batch(c, descs, n, block, algo, pick_shape(c, algo, block, mr, mw, mh), (cudaStream_t)stream);
}

}  // extern "C"

namespace {

int graph_create(me_ctx* c, const me_frame_desc* descs, int n, int block, int algo, const EvalArgs* ev,
                 me_graph** out)
{
    int rc = ME_OK;
    int mr = 1, mw = 0, mh = 0;
    for (int i = 0; i < n; ++i) { mr = std::max(mr, descs[i].range); mw = std::max(mw, descs[i].w); mh = std::max(mh, descs[i].h); }
    const Shape s = pick_shape(c, algo, block, mr, mw, mh);
    std::vector<FrameDev> table(n);
    int max_range = 1;
    const int ntiles = build_table(descs, n, block, s, algo == ME_ALGO_FS, table.data(), &max_range, ev);
    if (ntiles < 0) return fail(c, ME_ERR_CUDA, "cuTensorMapEncodeTiled rejected a frame description");
    me_graph* g = new me_graph();
    g->ctx = c;
    const size_t bytes = kHeadBytes + sizeof(FrameDev) * (size_t)n;
    cudaError_t e = cudaMalloc(&g->dev, bytes);
    if (e != cudaSuccess) { delete g; return fail(c, ME_ERR_NOMEM, "cudaMalloc of a graph table failed"); }
    e = cudaMemcpy(reinterpret_cast<char*>(g->dev) + kHeadBytes, table.data(), sizeof(FrameDev) * n,
                   cudaMemcpyHostToDevice);
    cudaStream_t cs = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = launch_search(c, g->dev, n, ntiles, block, algo, max_range, s, cs, ev);
        e = cudaStreamEndCapture(cs, &g->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        me_graph_free(g);
        return cuda_fail(c, e, "graph capture");
    }
    *out = g;
    return ME_OK;
}

int validate_eval(me_ctx* c, const me_frame_desc* descs, const int16_t* const* mv_fs, int n, int algo,
                  const uint64_t* sums)
{
    if (algo != ME_ALGO_DCDS && algo != ME_ALGO_DCDS_S)
        return fail(c, ME_ERR_UNSUPPORTED, "the fused evaluation is built for DCDS and DCDS^S");
    if (!sums || !aligned(sums, 8)) return fail(c, ME_ERR_ARG, "sums must be a non-NULL 8-byte aligned device array");
    for (int i = 0; mv_fs && i < n; ++i)
        if (mv_fs[i] && !aligned(mv_fs[i], 4)) return fail(c, ME_ERR_ARG, "mv_fs entries must be 4-byte aligned");
    (void)descs;
    return ME_OK;
}

// Copies for one stream, adjacent ones merged when both sides are contiguous.
struct CopyList {
    struct Item { char* dst; const char* src; size_t bytes; };
    std::vector<Item> v;
    void add(void* dst, const void* src, size_t bytes)
    {
        char* d = static_cast<char*>(dst);
        const char* s = static_cast<const char*>(src);
        if (!v.empty() && v.back().dst + v.back().bytes == d && v.back().src + v.back().bytes == s)
            v.back().bytes += bytes;
        else
            v.push_back({d, s, bytes});
    }
    cudaError_t issue(cudaStream_t st) const
    {
        for (const Item& it : v) {
            cudaError_t e = cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyDefault, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
};

int pipe_ready(me_ctx* c, me::HostStage& g, size_t bytes, int nchunks)
{
    me::HostPipe& P = c->pipe;
    cudaError_t e = cudaSuccess;
    if (!P.in) e = cudaStreamCreateWithFlags(&P.in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !P.out) e = cudaStreamCreateWithFlags(&P.out, cudaStreamNonBlocking);
    if (e == cudaSuccess && !P.entry) e = cudaEventCreateWithFlags(&P.entry, cudaEventDisableTiming);
    if (e == cudaSuccess && !g.done) {
        e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(g.done, P.out);
    }
    while (e == cudaSuccess && (int)P.ev.size() < 3 * nchunks) {
        cudaEvent_t x = nullptr;
        e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
        if (e == cudaSuccess) P.ev.push_back(x);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "host pipeline streams and events");
    if (g.cap < bytes) {
        // the last call that used this set has copied its results back (so its searches are done)
        e = cudaEventSynchronize(g.done);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
        if (g.dev) cudaFree(g.dev);
        g.dev = nullptr;
        g.cap = 0;
        if (cudaMalloc(&g.dev, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, ME_ERR_NOMEM, "cudaMalloc of the host-batch staging failed");
        }
        g.cap = bytes;
    }
    return ME_OK;
}

// me_estimate_host_batch: stage the batch in device memory chunk by chunk.
int host_batch(me_ctx* c, const me_frame_desc* d, const int16_t* const* mv_fs, int n, int block, int algo,
               uint64_t* sums, int chunk, cudaStream_t st)
{
    if (chunk <= 0) chunk = (n + 3) / 4;
    const int nchunks = (n + chunk - 1) / chunk;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };

    // frames, once per distinct host pointer, in the order of first use
    struct Fr { const uint8_t* h; size_t bytes, span, off; };
    std::vector<Fr> fr;
    std::unordered_map<const uint8_t*, int> index;
    std::vector<int> fc(n), frf(n);
    auto frame = [&](const uint8_t* p, const me_frame_desc& f) {
        const size_t bytes = (size_t)(f.h - 1) * f.pitch + f.w, span = (size_t)f.h * f.pitch;
        auto it = index.find(p);
        if (it != index.end()) {
            Fr& x = fr[it->second];
            x.bytes = std::max(x.bytes, bytes);
            x.span = std::max(x.span, span);
            return it->second;
        }
        index.emplace(p, (int)fr.size());
        fr.push_back({p, bytes, span, 0});
        return (int)fr.size() - 1;
    };
    for (int i = 0; i < n; ++i) { fc[i] = frame(d[i].cur, d[i]); frf[i] = frame(d[i].ref, d[i]); }
    // Device layout: frames (16-byte multiples), then mv, sad, nsp, FS fields
    // and sums.  The frames a chunk uploads first, and its FS fields, are
    // placed in host-address order, so that buffers adjacent on the host are
    // adjacent on the device and their copies merge into one.
    std::vector<std::vector<int>> up_frames(nchunks), up_fs(nchunks);
    std::vector<size_t> nb(n), o_mv(n), o_sad(n), o_nsp(n), o_fs(n, 0);
    size_t off = 0;
    {
        std::vector<char> seen(fr.size(), 0);
        for (int k = 0; k < nchunks; ++k) {
            std::vector<int>& L = up_frames[k];
            for (int i = k * chunk; i < std::min(n, (k + 1) * chunk); ++i)
                for (int f : {fc[i], frf[i]})
                    if (!seen[f]) { seen[f] = 1; L.push_back(f); }
            std::sort(L.begin(), L.end(), [&](int a, int b) { return (uintptr_t)fr[a].h < (uintptr_t)fr[b].h; });
            for (int f : L) { fr[f].off = off; off += fr[f].span; }
        }
    }
    off = up(off);
    for (int i = 0; i < n; ++i) { nb[i] = (size_t)(d[i].w / block) * (d[i].h / block); o_mv[i] = off; off += 4 * nb[i]; }
    off = up(off);
    for (int i = 0; i < n; ++i) { o_sad[i] = off; off += 4 * nb[i]; }
    off = up(off);
    for (int i = 0; i < n; ++i) { o_nsp[i] = off; off += 2 * nb[i]; }
    off = up(off);
    for (int k = 0; sums && mv_fs && k < nchunks; ++k) {
        std::vector<int>& L = up_fs[k];
        for (int i = k * chunk; i < std::min(n, (k + 1) * chunk); ++i)
            if (mv_fs[i]) L.push_back(i);
        std::sort(L.begin(), L.end(), [&](int a, int b) { return (uintptr_t)mv_fs[a] < (uintptr_t)mv_fs[b]; });
        for (int i : L) { o_fs[i] = off; off += 4 * nb[i]; }
    }
    off = up(off);
    const size_t o_sums = off;
    off += sums ? sizeof(uint64_t) * ME_NSUMS * (size_t)n : 0;
    me::HostPipe& P = c->pipe;
    me::HostStage& G = P.stage[P.next];
    int rc = pipe_ready(c, G, std::max<size_t>(off, 256), nchunks);
    if (rc != ME_OK) return rc;
    P.next ^= 1;
    char* base = static_cast<char*>(G.dev);

    int mr = 1, mw = 0, mh = 0;
    for (int i = 0; i < n; ++i) { mr = std::max(mr, d[i].range); mw = std::max(mw, d[i].w); mh = std::max(mh, d[i].h); }
    const Shape s = pick_shape(c, algo, block, mr, mw, mh);

    // Every chunk's [queue head | descriptor table] goes up in one copy ahead
    // of the frames: a small copy on the searching stream would queue behind
    // the next chunk's frames on the copy engine and hold its search back.
    const size_t per = kHeadBytes + sizeof(FrameDev) * (size_t)chunk;
    Slot* slot = nullptr;
    rc = take_slot(c, per * nchunks, &slot);
    if (rc != ME_OK) return rc;
    std::vector<me_frame_desc> dd(n);
    std::vector<const int16_t*> fsd(n);
    std::vector<int> ntiles(nchunks), mrange(nchunks);
    for (int i = 0; i < n; ++i) {
        me_frame_desc& x = dd[i];
        x = d[i];
        x.cur = reinterpret_cast<const uint8_t*>(base + fr[fc[i]].off);
        x.ref = reinterpret_cast<const uint8_t*>(base + fr[frf[i]].off);
        x.mv = reinterpret_cast<int16_t*>(base + o_mv[i]);
        x.sad = reinterpret_cast<uint32_t*>(base + o_sad[i]);
        x.nsp = d[i].nsp ? reinterpret_cast<uint16_t*>(base + o_nsp[i]) : nullptr;
        fsd[i] = (sums && mv_fs && mv_fs[i]) ? reinterpret_cast<const int16_t*>(base + o_fs[i]) : nullptr;
    }
    std::vector<EvalArgs> eas(nchunks);
    for (int k = 0; k < nchunks; ++k) {
        const int c0 = k * chunk, m = std::min(n, c0 + chunk) - c0;
        eas[k].mv_fs = fsd.data() + c0;
        eas[k].sums = sums ? reinterpret_cast<uint64_t*>(base + o_sums) + (size_t)ME_NSUMS * c0 : nullptr;
        FrameDev* table = reinterpret_cast<FrameDev*>(static_cast<char*>(slot->host) + per * k + kHeadBytes);
        ntiles[k] = build_table(dd.data() + c0, m, block, s, algo == ME_ALGO_FS, table, &mrange[k],
                                sums ? &eas[k] : nullptr);
        if (ntiles[k] < 0) return fail(c, ME_ERR_CUDA, "cuTensorMapEncodeTiled rejected a frame description");
    }

    // uploads start once the caller's stream reaches the call and the last
    // call that used this staging set has its results back
    cudaError_t e = cudaEventRecord(P.entry, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.in, P.entry, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.in, G.done, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(slot->dev, slot->host, per * nchunks, cudaMemcpyHostToDevice, P.in);
    if (e != cudaSuccess) return cuda_fail(c, e, "host pipeline ordering");
    for (int k = 0; k < nchunks; ++k) {
        const int c0 = k * chunk, c1 = std::min(n, c0 + chunk), m = c1 - c0;
        cudaEvent_t ev_in = P.ev[3 * k], ev_run = P.ev[3 * k + 1], ev_out = P.ev[3 * k + 2];
        CopyList in, out;
        for (int f : up_frames[k]) in.add(base + fr[f].off, fr[f].h, fr[f].bytes);
        for (int i : up_fs[k]) in.add(base + o_fs[i], mv_fs[i], 4 * nb[i]);
        e = in.issue(P.in);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in, P.in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_in, 0);
        if (e != cudaSuccess) return cuda_fail(c, e, "host-batch upload");
        e = launch_search(c, static_cast<char*>(slot->dev) + per * k, m, ntiles[k], block, algo, mrange[k], s, st,
                          sums ? &eas[k] : nullptr);
        if (e != cudaSuccess) return cuda_fail(c, e, "search launch");
        e = cudaEventRecord(ev_run, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P.out, ev_run, 0);
        if (e != cudaSuccess) return cuda_fail(c, e, "host pipeline ordering");
        for (int i = c0; i < c1; ++i) out.add(d[i].mv, base + o_mv[i], 4 * nb[i]);
        for (int i = c0; i < c1; ++i) out.add(d[i].sad, base + o_sad[i], 4 * nb[i]);
        for (int i = c0; i < c1; ++i)
            if (d[i].nsp) out.add(d[i].nsp, base + o_nsp[i], 2 * nb[i]);
        if (sums)
            out.add(sums + (size_t)ME_NSUMS * c0, base + o_sums + sizeof(uint64_t) * ME_NSUMS * c0,
                    sizeof(uint64_t) * ME_NSUMS * m);
        e = out.issue(P.out);
        if (e == cudaSuccess) e = cudaEventRecord(ev_out, P.out);
        if (e != cudaSuccess) return cuda_fail(c, e, "host-batch result copy");
    }
    e = cudaEventRecord(slot->done, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
    slot->used = true;
    e = cudaEventRecord(G.done, P.out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, G.done, 0);
    return e == cudaSuccess ? ME_OK : cuda_fail(c, e, "host pipeline ordering");
}

}  // namespace

extern "C" {

int me_graph_create(me_ctx* c, const me_frame_desc* descs, int n, int block, int algo, me_graph** out)
{
    if (!c || !out) return ME_ERR_ARG;
    *out = nullptr;
    int rc = validate_batch(c, descs, n, block, algo);
    if (rc == ME_OK && algo == ME_ALGO_DCDS_LEARNED)
        rc = fail(c, ME_ERR_UNSUPPORTED, "the learned start is not captured in graphs");
    if (rc != ME_OK) return rc;
    return graph_create(c, descs, n, block, algo, nullptr, out);
}

int me_graph_create_eval(me_ctx* c, const me_frame_desc* descs, const int16_t* const* mv_fs, int n, int block,
                         int algo, uint64_t* sums, me_graph** out)
{
    if (!c || !out) return ME_ERR_ARG;
    *out = nullptr;
    int rc = validate_batch(c, descs, n, block, algo);
    if (rc == ME_OK) rc = validate_eval(c, descs, mv_fs, n, algo, sums);
    if (rc != ME_OK) return rc;
    EvalArgs ev;
    ev.mv_fs = mv_fs;
    ev.sums = sums;
    return graph_create(c, descs, n, block, algo, &ev, out);
}

int me_estimate_eval_batch(me_ctx* c, const me_frame_desc* descs, const int16_t* const* mv_fs, int n, int block,
                           int algo, uint64_t* sums, void* stream)
{
    if (!c) return ME_ERR_ARG;
    Trace trace(c, "me_estimate_eval_batch", (cudaStream_t)stream);
    int rc = validate_batch(c, descs, n, block, algo);
    if (rc == ME_OK) rc = validate_eval(c, descs, mv_fs, n, algo, sums);
    if (rc != ME_OK) return rc;
    int mr = 1, mw = 0, mh = 0;
    for (int i = 0; i < n; ++i) { mr = std::max(mr, descs[i].range); mw = std::max(mw, descs[i].w); mh = std::max(mh, descs[i].h); }
    EvalArgs ev;
    ev.mv_fs = mv_fs;
    ev.sums = sums;
    return run_batch(c, descs, n, block, algo, pick_shape(c, algo, block, mr, mw, mh), (cudaStream_t)stream, &ev);
}

int me_fs_dual_batch(me_ctx* c, const me_frame_desc* d16, const me_frame_desc* d8, int n, void* stream)
{
    if (!c) return ME_ERR_ARG;
    Trace trace(c, "me_fs_dual_batch", (cudaStream_t)stream);
    int rc = validate_batch(c, d16, n, 16, ME_ALGO_FS);
    if (rc != ME_OK) return rc;
    if (!d8) return fail(c, ME_ERR_ARG, "d8 must not be NULL");
    int mr = 1, mw = 0, mh = 0;
    for (int i = 0; i < n; ++i) {
        if (!d8[i].mv || !d8[i].sad) return fail(c, ME_ERR_ARG, "8x8 mv and sad must not be NULL");
        if (!aligned(d8[i].mv, 4) || !aligned(d8[i].sad, 4) || (d8[i].nsp && !aligned(d8[i].nsp, 2)))
            return fail(c, ME_ERR_ARG, "8x8 mv/sad must be 4-byte aligned, nsp 2-byte aligned");
        mr = std::max(mr, d16[i].range); mw = std::max(mw, d16[i].w); mh = std::max(mh, d16[i].h);
    }
    // the quadrant accumulators need the short task heights (9 or 11 candidate rows)
    Shape s = pick_shape(c, ME_ALGO_FS, 16, mr, mw, mh);
    const int n1 = 2 * mr + 1;
    s.k = (((n1 + 8) / 9) * 12 <= ((n1 + 10) / 11) * 14) ? 9 : 11;
    s.tx = fs_pick_tx(16, mr, s.k);
    EvalArgs ev;
    ev.d8 = d8;
    return run_batch(c, d16, n, 16, ME_ALGO_FS, s, (cudaStream_t)stream, &ev);
}

int me_graph_launch(me_ctx* c, me_graph* g, void* stream)
{
    if (!c || !g) return ME_ERR_ARG;
    Trace trace(c, "me_graph_launch", (cudaStream_t)stream);
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? ME_OK : cuda_fail(c, e, "cudaGraphLaunch");
}

void me_graph_free(me_graph* g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->dev) cudaFree(g->dev);
    delete g;
}

int me_eval_batch(me_ctx* c, const me_eval_desc* d, int n, int block, uint64_t* sums, void* stream)
{
    if (!c) return ME_ERR_ARG;
    Trace trace(c, "me_eval_batch", (cudaStream_t)stream);
    if (!d || n <= 0 || !sums) return fail(c, ME_ERR_ARG, "descs and sums must not be NULL, n positive");
    if (!aligned(sums, 8)) return fail(c, ME_ERR_ARG, "sums must be 8-byte aligned");
    if (n > 65535) return fail(c, ME_ERR_ARG, "at most 65535 frames per evaluation batch");
    int max_blocks = 0;
    for (int i = 0; i < n; ++i) {
        int rc = check_frame(c, d[i].cur, d[i].ref, d[i].w, d[i].h, d[i].pitch, block, 1, d[i].mv, d[i].mv,
                             d[i].nsp);
        if (rc != ME_OK) return rc;
        if (d[i].mv_fs && !aligned(d[i].mv_fs, 4)) return fail(c, ME_ERR_ARG, "mv_fs must be 4-byte aligned");
        max_blocks = std::max(max_blocks, (d[i].w / block) * (d[i].h / block));
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = kHeadBytes + sizeof(EvalDev) * (size_t)n;
    Slot* slot = nullptr;
    int rc = take_slot(c, bytes, &slot);
    if (rc != ME_OK) return rc;
    EvalDev* table = reinterpret_cast<EvalDev*>(reinterpret_cast<char*>(slot->host) + kHeadBytes);
    for (int i = 0; i < n; ++i) {
        EvalDev f{};
        f.cur = d[i].cur; f.ref = d[i].ref; f.mv = d[i].mv; f.mv_fs = d[i].mv_fs; f.nsp = d[i].nsp;
        f.w = d[i].w; f.h = d[i].h; f.pitch = d[i].pitch; f.nbx = d[i].w / block; f.nby = d[i].h / block;
        table[i] = f;
    }
    cudaError_t e = cudaMemcpyAsync(slot->dev, slot->host, bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, sizeof(uint64_t) * ME_NSUMS * (size_t)n, st);
    if (e == cudaSuccess)
        e = me::launch_eval(reinterpret_cast<const EvalDev*>(reinterpret_cast<char*>(slot->dev) + kHeadBytes), n,
                            block, max_blocks, c->num_sms, reinterpret_cast<unsigned long long*>(sums), st);
    if (e == cudaSuccess) e = cudaEventRecord(slot->done, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "evaluation launch");
    slot->used = true;
    return ME_OK;
}

int me_mvp_stats(me_ctx* c, const me_frame_desc* d, int n, int range, uint64_t* out, void* stream)
{
    if (!c) return ME_ERR_ARG;
    Trace trace(c, "me_mvp_stats", (cudaStream_t)stream);
    if (!d || n <= 0 || !out) return fail(c, ME_ERR_ARG, "descs and out must not be NULL, n positive");
    if (!aligned(out, 8)) return fail(c, ME_ERR_ARG, "out must be 8-byte aligned");
    if (range < 1 || range > ME_MAX_RANGE) return fail(c, ME_ERR_ARG, "range must be in 1..32");
    long total = 0;
    for (int i = 0; i < n; ++i) {
        if (!d[i].cur || !d[i].ref || !d[i].mv) return fail(c, ME_ERR_ARG, "cur, ref and mv must not be NULL");
        if (!aligned(d[i].cur, 16) || !aligned(d[i].ref, 16) || !aligned(d[i].mv, 4))
            return fail(c, ME_ERR_ARG, "cur/ref must be 16-byte aligned, mv 4-byte aligned");
        if (d[i].w <= 0 || d[i].h <= 0 || d[i].w % 16 || d[i].h % 16 || d[i].pitch < d[i].w || d[i].pitch % 16)
            return fail(c, ME_ERR_ARG, "16x16 blocks: w and h multiples of 16, pitch >= w and a multiple of 16");
        if (d[i].range < 1 || d[i].range > range) return fail(c, ME_ERR_ARG, "every frame's range must be in 1..range");
        total += (long)(d[i].w / 16) * (d[i].h / 16);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t tbl = sizeof(EvalDev) * (size_t)n, rng = ((sizeof(int) * (size_t)n) + 7) & ~size_t(7);
    const size_t bytes = kHeadBytes + tbl + rng + sizeof(long) * (size_t)n;
    Slot* slot = nullptr;
    int rc = take_slot(c, bytes, &slot);
    if (rc != ME_OK) return rc;
    char* h = reinterpret_cast<char*>(slot->host);
    EvalDev* table = reinterpret_cast<EvalDev*>(h + kHeadBytes);
    int* ranges = reinterpret_cast<int*>(h + kHeadBytes + tbl);
    long* bases = reinterpret_cast<long*>(h + kHeadBytes + tbl + rng);
    long base = 0;
    for (int i = 0; i < n; ++i) {
        EvalDev f{};
        f.cur = d[i].cur; f.ref = d[i].ref; f.mv = d[i].mv;
        f.w = d[i].w; f.h = d[i].h; f.pitch = d[i].pitch; f.nbx = d[i].w / 16; f.nby = d[i].h / 16;
        table[i] = f;
        ranges[i] = d[i].range;
        bases[i] = base;
        base += (long)f.nbx * f.nby;
    }
    const size_t nq = (size_t)(2 * range + 1) * (2 * range + 1);
    char* dv = reinterpret_cast<char*>(slot->dev);
    cudaError_t e = cudaMemcpyAsync(slot->dev, slot->host, bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, sizeof(uint64_t) * 35 * nq, st);
    if (e == cudaSuccess)
        e = me::launch_mvp(reinterpret_cast<const EvalDev*>(dv + kHeadBytes),
                           reinterpret_cast<const int*>(dv + kHeadBytes + tbl),
                           reinterpret_cast<const long*>(dv + kHeadBytes + tbl + rng), n, total, range, c->num_sms,
                           reinterpret_cast<unsigned long long*>(out), st);
    if (e == cudaSuccess) e = cudaEventRecord(slot->done, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "motion-vector statistics launch");
    slot->used = true;
    return ME_OK;
}

int me_eval(me_ctx* c, const uint8_t* cur, const uint8_t* ref, int w, int h, int block, const int16_t* mv,
            const int16_t* mv_fs, const uint16_t* nsp, uint64_t* sums, void* stream)
{
    me_eval_desc d{cur, ref, w, h, w, mv, mv_fs, nsp};
    return me_eval_batch(c, &d, 1, block, sums, stream);
}

int me_stats_from_sums(const uint64_t* s, me_stats* out)
{
    if (!s || !out) return ME_ERR_ARG;
    const double npix = (double)s[ME_SUM_PIXELS], nb = (double)s[ME_SUM_BLOCKS];
    if (npix <= 0.0 || nb <= 0.0) return ME_ERR_ARG;
    out->mad = (double)s[ME_SUM_ABS] / npix;
    out->mse = (double)s[ME_SUM_SQ] / npix;
    out->nsp = (double)s[ME_SUM_NSP] / nb;
    out->psnr = out->mse > 0.0 ? 10.0 * std::log10(255.0 * 255.0 / out->mse) : 100.0;
    out->distance = s[ME_SUM_HAS_FS] ? (double)s[ME_SUM_DIST_Q24] / 16777216.0 / nb : 0.0;
    out->probability = s[ME_SUM_HAS_FS] ? (double)s[ME_SUM_EQUAL] / nb : 0.0;
    return ME_OK;
}

int me_tune_batch(me_ctx* c, const me_frame_desc* descs, int n, int block, int algo, int* chosen, void* stream)
{
    if (!c) return ME_ERR_ARG;
    int rc = validate_batch(c, descs, n, block, algo);
    if (rc == ME_OK && algo == ME_ALGO_DCDS_LEARNED)
        rc = fail(c, ME_ERR_UNSUPPORTED, "the learned start has no launch shapes to tune");
    if (rc != ME_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int mr = 1, mw = 0, mh = 0;
    for (int i = 0; i < n; ++i) { mr = std::max(mr, descs[i].range); mw = std::max(mw, descs[i].w); mh = std::max(mh, descs[i].h); }
    std::vector<Shape> cands;
    if (algo == ME_ALGO_FS) {
        const Shape base = default_shape(c, algo, block, mr);
        for (int k : {9, 11, 13, 15, 33}) {
            for (int tx = 4; tx <= 32; tx += (block == 8 ? 2 : 1)) {
                Shape s = base;
                s.k = k;
                s.tx = tx;
                // rows of work per thread: the picked k and its neighbours
                if (k != base.k && std::abs(k - base.k) > 2) continue;
                if (me::fs_shape_ok(block, mr, s)) cands.push_back(s);
            }
        }
    } else {
        // DCDS: CTA size and tile staging
        for (int th : {128, 256}) {
            for (int stages : {1, 2}) {
                Shape s = default_shape(c, algo, block, mr);
                s.threads = th;
                s.stages = stages;
                if (me::dcds_smem_bytes(block, mr, s) <= 220 * 1024) cands.push_back(s);
            }
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(c, ce, "cudaEventCreate");
    }
    float best = 1e30f;
    int bi = -1;
    for (size_t i = 0; i < cands.size(); ++i) {
        float tbest = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, st);
            rc = run_batch(c, descs, n, block, algo, cands[i], st);
            cudaEventRecord(e1, st);
            if (rc != ME_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tbest = std::min(tbest, ms);
        }
        if (rc != ME_OK) break;
        if (tbest < best) { best = tbest; bi = (int)i; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != ME_OK) return rc;
    if (bi < 0) return fail(c, ME_ERR_UNSUPPORTED, "no launch shape fits this configuration");
    c->tuned[shape_key(algo, block, mr, mw, mh)] = cands[bi];
    if (!c->tune_path.empty()) {
        std::ofstream f(c->tune_path, std::ios::app);
        const Shape& s = cands[bi];
        f << shape_key(algo, block, mr, mw, mh) << " " << s.tx << " " << s.ty << " " << s.threads << " " << s.k
          << " " << s.stages << "\n";
    }
    if (chosen) *chosen = bi;
    // leave the outputs computed with the chosen shape
    return run_batch(c, descs, n, block, algo, cands[bi], st);
}

int me_tune(me_ctx* c, const uint8_t* cur, const uint8_t* ref, int w, int h, int block, int range, int algo,
            int16_t* mv, uint32_t* sad, uint16_t* nsp, int* chosen, void* stream)
{
    me_frame_desc d{cur, ref, w, h, w, range, mv, sad, nsp};
    return me_tune_batch(c, &d, 1, block, algo, chosen, stream);
}

int me_absdiff_peak(me_ctx* c, int iters, double* out, int n_variants, int* used, void* stream)
{
    if (!c || !out || n_variants <= 0 || iters <= 0) return ME_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 256, blocks = c->num_sms * 8;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(c, ce, "cudaEventCreate");
    }
    for (int v = 0; v < n_variants; ++v) {
        out[v] = 0.0;
        if (v >= me::SAD_NVARIANTS) continue;
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            cudaError_t e = me::launch_absdiff_peak(v, iters, blocks, threads, c->sink, st);
            cudaEventRecord(e1, st);
            if (e != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return cuda_fail(c, e, "absdiff peak"); }
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);
        }
        out[v] = (double)blocks * threads * (double)iters * 128.0 / (best * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (used) *used = me::kSadVariant;
    return ME_OK;
}

int me_set_tracing(me_ctx* c, int on)
{
    if (!c) return ME_ERR_ARG;
    if (on) {
        cudaError_t e = cudaSuccess;
        if (!c->trace0) e = cudaEventCreate(&c->trace0);
        if (e == cudaSuccess && !c->trace1) e = cudaEventCreate(&c->trace1);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
    }
    c->tracing = on ? 1 : 0;
    return ME_OK;
}

int me_last_call_ms(me_ctx* c, float* ms)
{
    if (!c || !ms) return ME_ERR_ARG;
    if (!c->traced) return fail(c, ME_ERR_UNSUPPORTED, "no traced call yet (me_set_tracing)");
    cudaError_t e = cudaEventSynchronize(c->trace1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, c->trace0, c->trace1);
    return e == cudaSuccess ? ME_OK : cuda_fail(c, e, "me_last_call_ms");
}

int me_inject_wait_timeout(me_ctx* c, int on)
{
    if (!c) {
        // the no-allocation path has no context: a NULL context arms its hook
        me::noalloc_inject_wait_timeout(on);
        return ME_OK;
    }
    c->inject_wait_timeout = on ? 1 : 0;
    return ME_OK;
}

int me_check_status(me_ctx* c, void* stream)
{
    if (!c) return ME_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
    unsigned st = 0;
    e = cudaMemcpy(&st, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read");
    if (st) {
        cudaMemset(c->status, 0, sizeof(unsigned));
        if (st & me::STATUS_TIMEOUT) return fail(c, ME_ERR_TIMEOUT, "a bounded device-side wait gave up");
        if (st & me::STATUS_BOUNDS) return fail(c, ME_ERR_CUDA, "a bounds check failed (ME_CHECK build)");
        return fail(c, ME_ERR_ARG, "a kernel rejected its input");
    }
    return ME_OK;
}

int me_estimate_host_batch(me_ctx* c, const me_frame_desc* descs, const int16_t* const* mv_fs, int n, int block,
                           int algo, uint64_t* sums, int chunk, void* stream)
{
    if (!c) return ME_ERR_ARG;
    Trace trace(c, "me_estimate_host_batch", (cudaStream_t)stream);
    int rc = validate_batch(c, descs, n, block, algo);
    if (rc == ME_OK && algo == ME_ALGO_DCDS_LEARNED)
        rc = fail(c, ME_ERR_UNSUPPORTED, "host batches run FS, DCDS and DCDS^S");
    if (rc == ME_OK && sums) rc = validate_eval(c, descs, mv_fs, n, algo, sums);
    if (rc != ME_OK) return rc;
    if (chunk < 0) return fail(c, ME_ERR_ARG, "chunk must not be negative");
    return host_batch(c, descs, sums ? mv_fs : nullptr, n, block, algo, sums, chunk, (cudaStream_t)stream);
}

}  // extern "C"
