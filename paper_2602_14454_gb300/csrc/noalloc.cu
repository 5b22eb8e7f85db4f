// Allocation-free variant of the even-odd operator application.
//
// dwf_apply performs its packing and its two hops in work fields that the
// handle allocates with cudaMalloc on first use.  Some callers cannot let a
// library allocate device memory during a call (for example an application
// that gives all device memory to its own pool, or code on a path where an
// allocation would synchronise the device), so this entry point keeps the
// four work fields in one file-scope device array instead.
//
// The array has a fixed size (kScratchBytes) and, like every file-scope
// device variable, exists on every GPU that loads the library until the
// process exits.  Its device address is looked up once per device, on the
// first call made with that device current.  All calls share it and it keeps
// whatever the last call left there; calls whose work overlaps on the GPU (on
// different streams, or on different handles of the same device) race.
#include <mutex>

#include "dwf_internal.h"

using namespace dwf;

namespace dwf_detail {
HopArgs hop_args(dwf_ctx *h, int prec, int out_par, FieldRef in, FieldRef out, int post);
cudaError_t hop(dwf_ctx *h, int prec, bool dag, const HopArgs &a, cudaStream_t st);
cudaError_t mix(dwf_ctx *h, int prec, FieldRef in, FieldRef out, int id, cudaStream_t st);
}  // namespace dwf_detail
using namespace dwf_detail;

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices];

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

extern "C" int dwf_apply_eo_noalloc(dwf_handle h, int prec, int dag, const void *in, void *out, void *stream)
{
    if (!h) return dwf_set_error(DWF_EINVAL, "NULL handle");
    if (h->slab) return dwf_set_error(DWF_EINVAL, "a slab handle applies its operator through dwf_slab_apply_eo");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    if (prec != DWF_F64 && prec != DWF_F32 && prec != DWF_F16) return dwf_set_error(DWF_EINVAL, "bad precision");
    if (!in || !out) return dwf_set_error(DWF_EINVAL, "NULL vector");
    if (((uintptr_t)in & 15u) || ((uintptr_t)out & 15u))
        return dwf_set_error(DWF_EINVAL, "vectors must be 16-byte aligned");
    const size_t fb = round256(field_bytes(prec, h->Vh, h->Ls));
    const size_t sb = round256(scale_bytes(prec, h->Vh, h->Ls));
    const size_t need = 4 * (fb + sb);
    if (need > kScratchBytes)
        return dwf_set_error(DWF_EINVAL, "lattice too large for the allocation-free path: it needs " +
                                             std::to_string(need) + " bytes of work space, the fixed array holds " +
                                             std::to_string(kScratchBytes));
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return dwf_cuda_error(e, "cudaGetSymbolAddress");
    FieldRef f[4];
    for (int k = 0; k < 4; ++k) {
        unsigned char *p = (unsigned char *)base + (size_t)k * (fb + sb);
        f[k].v = p;
        f[k].scale = sb ? (float *)(p + fb) : nullptr;
    }
    FieldRef x = f[0], xh = f[1], t = f[2], y = f[3];
    cudaStream_t st = (cudaStream_t)stream;
    if ((e = launch_pack_eo(prec, (const double *)in, x, h->Vh, h->Ls, st)) != cudaSuccess)
        return dwf_cuda_error(e, "pack");
    if ((e = mix(h, prec, x, xh, dag ? MAT_QT : MAT_P, st)) != cudaSuccess) return dwf_cuda_error(e, "mix");
    HopArgs a1 = hop_args(h, prec, 1, xh, t, dag ? MAT_MT : MAT_M);
    if ((e = hop(h, prec, dag != 0, a1, st)) != cudaSuccess) return dwf_cuda_error(e, "hop");
    HopArgs a2 = hop_args(h, prec, 0, t, y, dag ? MAT_NPT4 : MAT_NQ4);
    a2.y = x;
    a2.ymode = 1;
    if ((e = hop(h, prec, dag != 0, a2, st)) != cudaSuccess) return dwf_cuda_error(e, "hop");
    if ((e = launch_unpack_eo(prec, y, (double *)out, h->Vh, h->Ls, st)) != cudaSuccess)
        return dwf_cuda_error(e, "unpack");
    h->launches += 2;   // pack and unpack (mix and hop count their own launches)
    return DWF_OK;
}
