// noalloc.cu -- me_estimate_batch_noalloc: DCDS over a batch of frame pairs
// without any device allocation by the library.
//
// Who needs it: code that must not call cudaMalloc (or anything that may
// allocate device memory) at the point where it runs motion estimation.
// Examples: a real-time video path that cannot afford the device-wide
// synchronisation cudaMalloc/cudaFree may cause, host applications or plugin
// frameworks that own all device memory through their own pool and forbid
// libraries from allocating, and processes so close to the memory limit that
// a late allocation could fail mid-stream.  Such callers cannot create an
// me_ctx (me_init allocates), so this entry point needs no context.
//
// How: the work-queue counter and the descriptor table the DCDS kernel reads
// live in one file-scope __device__ array, g_static_scratch, of fixed size
// (room for ME_STATIC_MAX_FRAMES descriptors).  Every device that loads the
// library holds this array until the process exits.  The host never uses the
// array's name as a device address: the first call on each device, with that
// device current, asks cudaGetSymbolAddress for the address and keeps it.
// A small set-up kernel copies the descriptors (passed by value) into the
// array and clears the counters, then the regular DCDS kernel runs on it.
//
// Failures the kernel detects on the device (a bounded copy wait that gave
// up) are ORed into a status word in the same array.  It keeps accumulating
// over calls until me_noalloc_check_status reads and clears it.
#include "me.h"
#include "me_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>

namespace {

constexpr int kHeadBytes = 256;
constexpr int kStatusOffset = 128;  // bytes into the head: the status word, past the counter words
constexpr int kChunk = 16;          // descriptors per set-up launch (passed by value)
constexpr int kMaxDevices = 64;
static_assert(me::kCounterInts * sizeof(int) <= kStatusOffset, "status word overlaps the counters");

static __device__ __align__(256) unsigned char
    g_static_scratch[kHeadBytes + ME_STATIC_MAX_FRAMES * sizeof(me::FrameDev)];

struct Chunk {
    me::FrameDev f[kChunk];
};

// inject: the failure-detection test hook (me_inject_wait_timeout with a NULL
// context) -- the kernel then starves its first copy wait, see dcds.cu.
__global__ void static_setup_kernel(Chunk c, int first, int count, int inject, unsigned char* scratch)
{
    me::FrameDev* table = reinterpret_cast<me::FrameDev*>(scratch + kHeadBytes);
    // the queue head starts at zero, and so do the kernel's other counter words
    if (first == 0 && threadIdx.x < me::kCounterInts)
        reinterpret_cast<int*>(scratch)[threadIdx.x] = (threadIdx.x == me::kCounterInts - 1) ? inject : 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) table[first + i] = c.f[i];
}

struct DeviceState {
    unsigned char* scratch = nullptr;
    int num_sms = 0;
};
DeviceState g_dev[kMaxDevices];
std::once_flag g_once[kMaxDevices];
cudaError_t g_setup_err[kMaxDevices];
std::atomic<int> g_inject{0};

void setup_device(int dev)
{
    // runs once per device, with that device current
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_dev[dev].num_sms, cudaDevAttrMultiProcessorCount, dev);
    // With lazy module loading a kernel is loaded (which may allocate device
    // memory) on its first launch; load every kernel this path launches now.
    if (e == cudaSuccess) {
        cudaFuncAttributes a;
        e = cudaFuncGetAttributes(&a, static_setup_kernel);
    }
    if (e == cudaSuccess) e = me::dcds_preload();
    if (e == cudaSuccess) g_dev[dev].scratch = static_cast<unsigned char*>(p);
    g_setup_err[dev] = e;
}

// The current device's scratch array, set up on first use.
int device_scratch(unsigned char** out, int* num_sms, char* err, int err_len);

int set_err(char* err, int len, int code, const char* msg)
{
    if (err && len > 0) snprintf(err, (size_t)len, "%s", msg);
    return code;
}

int device_scratch(unsigned char** out, int* num_sms, char* err, int err_len)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_err(err, err_len, ME_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_err(err, err_len, ME_ERR_CUDA, "device index out of range");
    std::call_once(g_once[dev], setup_device, dev);
    if (g_setup_err[dev] != cudaSuccess || !g_dev[dev].scratch)
        return set_err(err, err_len, ME_ERR_CUDA, "set-up of the static scratch failed (symbol address or kernel load)");
    *out = g_dev[dev].scratch;
    if (num_sms) *num_sms = g_dev[dev].num_sms;
    return ME_OK;
}

}  // namespace

namespace me {
void noalloc_inject_wait_timeout(int on) { g_inject.store(on ? 1 : 0); }
}  // namespace me

extern "C" int me_estimate_batch_noalloc(const me_frame_desc* d, int n, int block, int algo, void* stream,
                                         char* err, int err_len)
{
    if (err && err_len > 0) err[0] = '\0';
    if (!d || n <= 0) return set_err(err, err_len, ME_ERR_ARG, "descs must not be NULL and n must be positive");
    if (n > ME_STATIC_MAX_FRAMES) {
        char m[160];
        snprintf(m, sizeof m, "%d frame pairs requested; the no-allocation path holds at most %d per call",
                 n, ME_STATIC_MAX_FRAMES);
        return set_err(err, err_len, ME_ERR_ARG, m);
    }
    if (algo != ME_ALGO_DCDS && algo != ME_ALGO_DCDS_S)
        return set_err(err, err_len, ME_ERR_UNSUPPORTED, "the no-allocation path runs DCDS and DCDS^S only");
    if (block != 8 && block != 16) return set_err(err, err_len, ME_ERR_ARG, "block must be 8 or 16");

    me::Shape s{};
    s.threads = 128;
    s.tx = me::kTile / block;
    s.ty = me::kDcdsTileH / block;
    s.k = 0;
    s.stages = 1;
    s.ctas_per_sm = 0;

    Chunk chunk;
    int tiles = 0, max_range = 1;
    me::FrameDev table[ME_STATIC_MAX_FRAMES];
    for (int i = 0; i < n; ++i) {
        const me_frame_desc& x = d[i];
        if (!x.cur || !x.ref || ((uintptr_t)x.cur % 16) || ((uintptr_t)x.ref % 16))
            return set_err(err, err_len, ME_ERR_ARG, "cur/ref must be non-NULL and 16-byte aligned");
        if (x.w <= 0 || x.h <= 0 || x.w % 16 || x.w % block || x.h % block)
            return set_err(err, err_len, ME_ERR_ARG, "w must be a multiple of 16 and of block, h of block");
        if (x.pitch < x.w || x.pitch % 16) return set_err(err, err_len, ME_ERR_ARG, "pitch must be >= w and a multiple of 16");
        if (x.range < 1 || x.range > ME_MAX_RANGE) return set_err(err, err_len, ME_ERR_ARG, "range must be in 1..32");
        if (!x.mv || !x.sad || ((uintptr_t)x.mv % 4) || ((uintptr_t)x.sad % 4) || ((uintptr_t)x.nsp % 2))
            return set_err(err, err_len, ME_ERR_ARG, "mv/sad must be non-NULL and 4-byte aligned, nsp 2-byte aligned");
        me::FrameDev f{};
        f.cur = x.cur; f.ref = x.ref; f.mv = x.mv; f.sad = x.sad; f.nsp = x.nsp;
        f.w = x.w; f.h = x.h; f.pitch = x.pitch; f.range = x.range;
        f.nbx = x.w / block; f.nby = x.h / block;
        f.tiles_x = (x.w + me::kTile - 1) / me::kTile;
        f.tiles_y = (x.h + me::kDcdsTileH - 1) / me::kDcdsTileH;
        if (!me::encode_frame_maps(f, me::kDcdsTileH))
            return set_err(err, err_len, ME_ERR_CUDA, "cuTensorMapEncodeTiled rejected a frame description");
        f.tile_base = tiles;
        tiles += f.tiles_x * f.tiles_y;
        max_range = std::max(max_range, x.range);
        table[i] = f;
    }
    me::set_uniform_tiles(table, n);

    unsigned char* scratch = nullptr;
    int num_sms = 0;
    const int rc = device_scratch(&scratch, &num_sms, err, err_len);
    if (rc != ME_OK) return rc;

    cudaStream_t st = (cudaStream_t)stream;
    const int inject = g_inject.load();
    cudaError_t e = cudaSuccess;
    for (int first = 0; first < n; first += kChunk) {
        const int cnt = std::min(kChunk, n - first);
        for (int i = 0; i < cnt; ++i) chunk.f[i] = table[first + i];
        static_setup_kernel<<<1, 32, 0, st>>>(chunk, first, cnt, inject, scratch);
        e = cudaGetLastError();
        if (e != cudaSuccess) return set_err(err, err_len, ME_ERR_CUDA, cudaGetErrorString(e));
    }
    e = me::launch_dcds(reinterpret_cast<const me::FrameDev*>(scratch + kHeadBytes), n, tiles, block, max_range,
                        algo == ME_ALGO_DCDS_S, s, reinterpret_cast<int*>(scratch),
                        reinterpret_cast<unsigned*>(scratch + kStatusOffset), num_sms, st);
    if (e != cudaSuccess) return set_err(err, err_len, ME_ERR_CUDA, cudaGetErrorString(e));
    return ME_OK;
}

extern "C" int me_noalloc_check_status(void* stream, char* err, int err_len)
{
    if (err && err_len > 0) err[0] = '\0';
    unsigned char* scratch = nullptr;
    const int rc = device_scratch(&scratch, nullptr, err, err_len);
    if (rc != ME_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned v = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, scratch + kStatusOffset, sizeof v, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && v) e = cudaMemsetAsync(scratch + kStatusOffset, 0, sizeof v, st);
    if (e == cudaSuccess && v) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_err(err, err_len, ME_ERR_CUDA, cudaGetErrorString(e));
    if (v & me::STATUS_TIMEOUT) return set_err(err, err_len, ME_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (v & me::STATUS_BOUNDS) return set_err(err, err_len, ME_ERR_CUDA, "a bounds check failed (ME_CHECK build)");
    if (v) return set_err(err, err_len, ME_ERR_ARG, "a kernel rejected its input");
    return ME_OK;
}
