// tmap.cu -- host-side encoding of the TMA tensor maps of a frame pair.
// The CUDA driver's entry point is looked up through the runtime, so libme does not
// link libcuda directly.
#include "me_internal.cuh"

#include <cudaTypedefs.h>

#include <mutex>

namespace me {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool encode_2d(CUtensorMap* m, const uint8_t* base, int w, int h, int pitch, int box_w, int box_h)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t es[2] = {1, 1};
    // out-of-bounds elements of a box are filled with zeros
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool encode_frame_maps(FrameDev& f, int tile_h)
{
    const int rx = (f.range + 15) & ~15;
    return encode_2d(&f.tm_ref, f.ref, f.w, f.h, f.pitch, kTile + 2 * rx, tile_h + 2 * f.range) &&
           encode_2d(&f.tm_cur, f.cur, f.w, f.h, f.pitch, kTile, tile_h);
}

bool encode_fs_maps(FrameDev& f, int nch, int rows, int cur_w, int block)
{
    auto fn = encode_fn();
    if (!fn || f.w % 16) return false;
    const cuuint64_t dims[3] = {16, (cuuint64_t)(f.w / 16), (cuuint64_t)f.h};
    const cuuint64_t strides[2] = {16, (cuuint64_t)f.pitch};
    const cuuint32_t box[3] = {16, (cuuint32_t)nch, (cuuint32_t)rows};
    const cuuint32_t es[3] = {1, 1, 1};
    const bool ok = fn(&f.tm_ref, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(f.ref), dims, strides, box,
                       es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    return ok && encode_2d(&f.tm_cur, f.cur, f.w, f.h, f.pitch, cur_w, block);
}

}  // namespace me
