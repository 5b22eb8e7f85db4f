// Device helpers shared by the kernels: precision traits, field loads and
// stores in the internal layout (see dwf_internal.h), block reductions.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "dwf_internal.h"

namespace dwf {

template <int P> struct Tr;
template <> struct Tr<DWF_F64> {
    typedef double real;
    typedef double link_t;
    typedef double xs_t;
    static constexpr int G = 12;
};
template <> struct Tr<DWF_F32> {
    typedef float real;
    typedef float link_t;
    typedef float xs_t;
    static constexpr int G = 6;
};
template <> struct Tr<DWF_F16> {
    typedef float real;
    typedef __half link_t;
    typedef float xs_t;
    static constexpr int G = 3;
};

// ---------------------------------------------------------------- loads
// r[24] <- field(site, s).  RO = true uses the read-only data path.
template <int P, bool RO, typename T>
__device__ __forceinline__ void ld_field(const FieldRef &f, size_t site, int s, int Ls, T *r)
{
    if constexpr (P == DWF_F64) {
        const double2 *v = reinterpret_cast<const double2 *>(f.v) + (site * 12) * Ls + s;
#pragma unroll
        for (int g = 0; g < 12; ++g) {
            double2 q = RO ? __ldg(v + (size_t)g * Ls) : v[(size_t)g * Ls];
            r[2 * g] = (T)q.x;
            r[2 * g + 1] = (T)q.y;
        }
    } else if constexpr (P == DWF_F32) {
        const float4 *v = reinterpret_cast<const float4 *>(f.v) + (site * 6) * Ls + s;
#pragma unroll
        for (int g = 0; g < 6; ++g) {
            float4 q = RO ? __ldg(v + (size_t)g * Ls) : v[(size_t)g * Ls];
            r[4 * g] = (T)q.x;
            r[4 * g + 1] = (T)q.y;
            r[4 * g + 2] = (T)q.z;
            r[4 * g + 3] = (T)q.w;
        }
    } else {
        const uint4 *v = reinterpret_cast<const uint4 *>(f.v) + (site * 3) * Ls + s;
        const float sc = RO ? __ldg(f.scale + site * Ls + s) : f.scale[site * Ls + s];
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            uint4 q = RO ? __ldg(v + (size_t)g * Ls) : v[(size_t)g * Ls];
            const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                __half2 h2 = *reinterpret_cast<const __half2 *>(&w[k]);
                float2 f2 = __half22float2(h2);
                r[8 * g + 2 * k] = (T)(f2.x * sc);
                r[8 * g + 2 * k + 1] = (T)(f2.y * sc);
            }
        }
    }
}

// field(site, s) <- r[24]
template <int P, typename T>
__device__ __forceinline__ void st_field(const FieldRef &f, size_t site, int s, int Ls, const T *r)
{
    if constexpr (P == DWF_F64) {
        double2 *v = reinterpret_cast<double2 *>(f.v) + (site * 12) * Ls + s;
#pragma unroll
        for (int g = 0; g < 12; ++g) v[(size_t)g * Ls] = make_double2((double)r[2 * g], (double)r[2 * g + 1]);
    } else if constexpr (P == DWF_F32) {
        float4 *v = reinterpret_cast<float4 *>(f.v) + (site * 6) * Ls + s;
#pragma unroll
        for (int g = 0; g < 6; ++g)
            v[(size_t)g * Ls] = make_float4((float)r[4 * g], (float)r[4 * g + 1], (float)r[4 * g + 2], (float)r[4 * g + 3]);
    } else {
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 24; ++k) mx = fmaxf(mx, fabsf((float)r[k]));
        const float inv = mx > 0.f ? 1.0f / mx : 0.f;
        uint4 *v = reinterpret_cast<uint4 *>(f.v) + (site * 3) * Ls + s;
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            unsigned w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                __half2 h2 = __floats2half2_rn((float)r[8 * g + 2 * k] * inv, (float)r[8 * g + 2 * k + 1] * inv);
                w[k] = *reinterpret_cast<unsigned *>(&h2);
            }
            v[(size_t)g * Ls] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        f.scale[site * Ls + s] = mx;
    }
}

// ------------------------------------------------------------ reductions
// Sum of v over the block; valid in thread 0.  Handles a partial last warp.
__device__ __forceinline__ double block_sum(double v, double *wsum)
{
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    const int lane = tid & 31, w = tid >> 5;
    const int nw = (nt + 31) >> 5;
    const int wl = (w == nw - 1) ? (nt - 32 * w) : 32;
    const unsigned mask = (wl == 32) ? 0xffffffffu : ((1u << wl) - 1u);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        double o = __shfl_down_sync(mask, v, off);
        if (lane + off < wl) v += o;
    }
    if (lane == 0) wsum[w] = v;
    __syncthreads();
    double s = 0;
    if (tid == 0)
        for (int i = 0; i < nw; ++i) s += wsum[i];
    __syncthreads();
    return s;
}

__device__ __forceinline__ void finish_reduction(double total, const RedArgs &r)
{
    CgScalars *sc = r.scal;
    const bool finite = isfinite(total);
    switch (r.op) {
    case RED_STORE:
        sc->last = total;
        if (!finite) sc->flags |= 2;
        break;
    case RED_GAMMA:
        sc->gamma = total;
        sc->last = total;
        if (!finite) sc->flags |= 2;
        break;
    case RED_CG_ALPHA:
        sc->wn2 = total;
        if (!finite) {
            sc->flags |= 2;
            sc->alpha = 0.0;
        } else if (!(total > 0.0)) {
            sc->flags |= 1;
            sc->alpha = 0.0;
        } else {
            sc->alpha = sc->gamma / total;
        }
        break;
    case RED_CG_BETA:
        if (!finite) sc->flags |= 2;
        sc->beta = (sc->gamma > 0.0 && finite) ? total / sc->gamma : 0.0;
        sc->gamma = total;
        sc->last = total;
        break;
    default:
        break;
    }
}

// Deterministic grid reduction: per-block partials, the last block to finish
// adds them in index order and applies the scalar operation.
__device__ __forceinline__ void grid_reduce(double v, const RedArgs &r)
{
    __shared__ double wsum[32];
    __shared__ bool is_last;
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const unsigned nb = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    double s = block_sum(v, wsum);
    if (tid == 0) {
        r.partials[bid] = s;
        __threadfence();
        unsigned ticket = atomicAdd(r.counter, 1u);
        is_last = (ticket == nb - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double acc = 0;
        const volatile double *pp = r.partials;
        for (unsigned i = tid; i < nb; i += nt) acc += pp[i];
        double tot = block_sum(acc, wsum);
        if (tid == 0) {
            finish_reduction(tot, r);
            *r.counter = 0u;
        }
    }
}

}  // namespace dwf
