// Device helpers shared by the kernels: precision traits, spin-paired complex
// arithmetic, field loads and stores in the internal layout (dwf_internal.h),
// block reductions.
//
// Internal order of the 24 reals of one (site, s): group g = 2a + c
// (colour a, c = 0 re / 1 im) holds the four spins contiguously, so real k of
// the internal order is k = 4g + spin.  Registers hold a field as 12 pairs
// v[2g] = (spin 0, spin 1) and v[2g+1] = (spin 2, spin 3) of group g: even
// pairs are the P_+ chirality, odd pairs the P_- chirality.  Every spin
// projection, SU(3) product and fifth-direction mixing then works on pairs,
// which maps onto the packed FP32x2 instructions (FFMA2, FADD2, FMUL2).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "dwf_internal.h"

namespace dwf {

template <int P> struct Tr;
template <> struct Tr<DWF_F64> {
    typedef double real;
    typedef double2 pair;
    typedef double link_t;
    static constexpr int G = 12;
};
template <> struct Tr<DWF_F32> {
    typedef float real;
    typedef float2 pair;
    typedef float link_t;
    static constexpr int G = 6;
};
template <> struct Tr<DWF_F16> {
    typedef float real;
    typedef float2 pair;
    typedef __half link_t;
    static constexpr int G = 3;
};

template <typename T2> struct PairReal;
template <> struct PairReal<float2> { typedef float R; };
template <> struct PairReal<double2> { typedef double R; };

// ------------------------------------------------------- pair arithmetic
__device__ __forceinline__ float2 p_make(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 p_make(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 p_splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ double2 p_splat(double a) { return make_double2(a, a); }
__device__ __forceinline__ float2 p_zero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 p_zero(double2) { return make_double2(0.0, 0.0); }

// a * b + c
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 p_fma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 p_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ double2 p_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 p_mul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }

// ---------------------------------------------------------------- loads
// v[12] <- field(site, s) (FP16: scaled back to real values)
template <int P, bool RO, typename T2>
__device__ __forceinline__ void ld_pairs(const FieldRef &f, size_t site, int s, int Ls, T2 *v)
{
    typedef typename PairReal<T2>::R R;
    if constexpr (P == DWF_F64) {
        const double2 *p = reinterpret_cast<const double2 *>(f.v) + (site * 12) * Ls + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 q = RO ? __ldg(p + (size_t)k * Ls) : p[(size_t)k * Ls];
            v[k] = p_make((R)q.x, (R)q.y);
        }
    } else if constexpr (P == DWF_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(f.v) + (site * 6) * Ls + s;
#pragma unroll
        for (int g = 0; g < 6; ++g) {
            float4 q = RO ? __ldg(p + (size_t)g * Ls) : p[(size_t)g * Ls];
            v[2 * g] = p_make((R)q.x, (R)q.y);
            v[2 * g + 1] = p_make((R)q.z, (R)q.w);
        }
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(f.v) + (site * 3) * Ls + s;
        const size_t si = site * (size_t)((Ls + 3) & ~3) + s;
        const float sc = RO ? __ldg(f.scale + si) : f.scale[si];
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            uint4 q = RO ? __ldg(p + (size_t)g * Ls) : p[(size_t)g * Ls];
            const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float2 f2 = __half22float2(*reinterpret_cast<const __half2 *>(&w[k]));
                v[4 * g + k] = p_make((R)(f2.x * sc), (R)(f2.y * sc));
            }
        }
    }
}

// field(site, s) <- v[12]
template <int P, typename T2>
__device__ __forceinline__ void st_pairs(const FieldRef &f, size_t site, int s, int Ls, const T2 *v)
{
    if constexpr (P == DWF_F64) {
        double2 *p = reinterpret_cast<double2 *>(f.v) + (site * 12) * Ls + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * Ls] = make_double2((double)v[k].x, (double)v[k].y);
    } else if constexpr (P == DWF_F32) {
        float4 *p = reinterpret_cast<float4 *>(f.v) + (site * 6) * Ls + s;
#pragma unroll
        for (int g = 0; g < 6; ++g)
            p[(size_t)g * Ls] = make_float4((float)v[2 * g].x, (float)v[2 * g].y, (float)v[2 * g + 1].x,
                                            (float)v[2 * g + 1].y);
    } else {
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) mx = fmaxf(mx, fmaxf(fabsf((float)v[k].x), fabsf((float)v[k].y)));
        const float inv = mx > 0.f ? 1.0f / mx : 0.f;
        uint4 *p = reinterpret_cast<uint4 *>(f.v) + (site * 3) * Ls + s;
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            unsigned w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                __half2 h2 = __floats2half2_rn((float)v[4 * g + k].x * inv, (float)v[4 * g + k].y * inv);
                w[k] = *reinterpret_cast<unsigned *>(&h2);
            }
            p[(size_t)g * Ls] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        f.scale[site * (size_t)((Ls + 3) & ~3) + s] = mx;
    }
}

// The same with streaming stores (st.global.cs: evict first), for outputs no
// later load of the same launch reads: they then leave L2 to the data that is
// read again (the neighbour spinors of the hop).
template <int P, typename T2>
__device__ __forceinline__ void st_pairs_cs(const FieldRef &f, size_t site, int s, int Ls, const T2 *v)
{
    if constexpr (P == DWF_F64) {
        double2 *p = reinterpret_cast<double2 *>(f.v) + (site * 12) * Ls + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) __stcs(p + (size_t)k * Ls, make_double2((double)v[k].x, (double)v[k].y));
    } else if constexpr (P == DWF_F32) {
        float4 *p = reinterpret_cast<float4 *>(f.v) + (site * 6) * Ls + s;
#pragma unroll
        for (int g = 0; g < 6; ++g)
            __stcs(p + (size_t)g * Ls, make_float4((float)v[2 * g].x, (float)v[2 * g].y, (float)v[2 * g + 1].x,
                                                   (float)v[2 * g + 1].y));
    } else {
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) mx = fmaxf(mx, fmaxf(fabsf((float)v[k].x), fabsf((float)v[k].y)));
        const float inv = mx > 0.f ? 1.0f / mx : 0.f;
        uint4 *p = reinterpret_cast<uint4 *>(f.v) + (site * 3) * Ls + s;
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            unsigned w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                __half2 h2 = __floats2half2_rn((float)v[4 * g + k].x * inv, (float)v[4 * g + k].y * inv);
                w[k] = *reinterpret_cast<unsigned *>(&h2);
            }
            __stcs(p + (size_t)g * Ls, make_uint4(w[0], w[1], w[2], w[3]));
        }
        __stcs(f.scale + site * (size_t)((Ls + 3) & ~3) + s, mx);
    }
}

// v[12] <- field(site, s) with streaming loads (ld.global.cs), for inputs read once
template <int P, typename T2>
__device__ __forceinline__ void ld_pairs_cs(const FieldRef &f, size_t site, int s, int Ls, T2 *v)
{
    typedef typename PairReal<T2>::R R;
    if constexpr (P == DWF_F64) {
        const double2 *p = reinterpret_cast<const double2 *>(f.v) + (site * 12) * Ls + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 q = __ldcs(p + (size_t)k * Ls);
            v[k] = p_make((R)q.x, (R)q.y);
        }
    } else if constexpr (P == DWF_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(f.v) + (site * 6) * Ls + s;
#pragma unroll
        for (int g = 0; g < 6; ++g) {
            const float4 q = __ldcs(p + (size_t)g * Ls);
            v[2 * g] = p_make((R)q.x, (R)q.y);
            v[2 * g + 1] = p_make((R)q.z, (R)q.w);
        }
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(f.v) + (site * 3) * Ls + s;
        const float sc = __ldcs(f.scale + site * (size_t)((Ls + 3) & ~3) + s);
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            const uint4 q = __ldcs(p + (size_t)g * Ls);
            const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f2 = __half22float2(*reinterpret_cast<const __half2 *>(&w[k]));
                v[4 * g + k] = p_make((R)(f2.x * sc), (R)(f2.y * sc));
            }
        }
    }
}

// internal real index (4g + spin, g = 2a + c) <-> canonical (spin*3 + a)*2 + c
__host__ __device__ __forceinline__ int canon_of_internal(int k)
{
    const int spin = k & 3, g = k >> 2, a = g >> 1, c = g & 1;
    return (spin * 3 + a) * 2 + c;
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

// The same for FP32 per-thread values (partial sums of FP32 or FP16 fields):
// the warp level in FP32, across warps in FP64.  FP64 arithmetic is slow on
// GB300 (a warp-wide FP64 operation holds the SM's FP64 unit for about 16
// cycles), so per-element work stays in FP32 and only per-warp sums are FP64.
__device__ __forceinline__ double block_sum(float v, double *wsum)
{
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    const int lane = tid & 31, w = tid >> 5;
    const int nw = (nt + 31) >> 5;
    const int wl = (w == nw - 1) ? (nt - 32 * w) : 32;
    const unsigned mask = (wl == 32) ? 0xffffffffu : ((1u << wl) - 1u);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        float o = __shfl_down_sync(mask, v, off);
        if (lane + off < wl) v += o;
    }
    if (lane == 0) wsum[w] = (double)v;
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
// adds them in index order and applies the scalar operation.  bid / nb: this
// block's index among the nb blocks that reduce into r (a batched launch runs
// one such group of blocks per system).
// v: this thread's partial sum, FP64 or FP32 (block_sum above).
template <typename V>
__device__ __forceinline__ void grid_reduce(V v, const RedArgs &r, unsigned bid, unsigned nb)
{
    __shared__ double wsum[32];
    __shared__ bool is_last;
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y * blockDim.z;
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
        // thread t adds the contiguous run [t per, (t + 1) per) of partials (per
        // even, so the pairs are 16-byte loads; .cg loads read L2, where the other
        // blocks' stores are), several loads in flight per thread; the order of
        // the additions is fixed, so the total does not depend on which block
        // finished last
        const unsigned per = (((nb + nt - 1) / nt) + 1) & ~1u;
        const unsigned lo = min(nb, (unsigned)tid * per), hi = min(nb, lo + per);
        const double2 *p2 = reinterpret_cast<const double2 *>(r.partials);
        double acc = 0;
        unsigned i = lo;
#pragma unroll 2
        for (; i + 8 <= hi; i += 8) {
            const double2 q0 = __ldcg(p2 + i / 2), q1 = __ldcg(p2 + i / 2 + 1);
            const double2 q2 = __ldcg(p2 + i / 2 + 2), q3 = __ldcg(p2 + i / 2 + 3);
            acc += ((q0.x + q0.y) + (q1.x + q1.y)) + ((q2.x + q2.y) + (q3.x + q3.y));
        }
        for (; i < hi; ++i) acc += __ldcg(r.partials + i);
        double tot = block_sum(acc, wsum);
        if (tid == 0) {
            finish_reduction(tot, r);
            *r.counter = 0u;
        }
    }
}
template <typename V>
__device__ __forceinline__ void grid_reduce(V v, const RedArgs &r)
{
    grid_reduce(v, r, blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
}

// ------------------------------------------------- fifth-direction mixing
// Tile of one site in shared memory: Ls rows of 12 pairs.  o[n] += sum_t
// M[chi][s_n][t] tile[t], chi = pair parity; the coefficients are stored as
// mt[chi][t][x * NS + n] (x = thread's slice index, s_n = x + n Ls/NS).
__device__ __forceinline__ void ld_tile_row(const float2 *row, float2 *h)
{
    const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 v = r4[q];
        h[2 * q] = make_float2(v.x, v.y);
        h[2 * q + 1] = make_float2(v.z, v.w);
    }
}
__device__ __forceinline__ void ld_tile_row(const double2 *row, double2 *h)
{
#pragma unroll
    for (int q = 0; q < 12; ++q) h[q] = row[q];
}

// Structured mixing (see MixProg in dwf_internal.h) applied in place to the
// tiles of `nsites` sites (site stride tstride pairs, row stride 12 pairs):
// one chain = one real component of one site over all Ls rows.  The caller's
// `nthr` threads (index tid) share the chains; no barrier inside.
template <typename R, typename T2>
__device__ __forceinline__ void chain_mix(const MixProg<R> *pg, T2 *tile, int tstride, int nsites, int Ls, int tid,
                                          int nthr)
{
    R *t = reinterpret_cast<R *>(tile);
    const R kappa = pg->kappa, a0inv = pg->a0inv, mneg = pg->mneg, s0 = pg->s0, s1 = pg->s1;
    // Streaming form: each pass walks the chain in shared memory (u = 0 .. Ls-1
    // in the direction of K) with O(1) registers; the d1 / d2 scalings are
    // folded into the first read and the last write.
    for (int c = tid; c < nsites * 24; c += nthr) {
        const int jj = c / 24, k = c % 24;
        const int chi = (k >> 1) & 1;
        R *base = t + (size_t)jj * tstride * 2 + k;
        const bool up = pg->up[chi] != 0;
        const R *d1 = pg->d1[chi], *d2 = pg->d2[chi];
        const int s_last = up ? 0 : Ls - 1;   // slice of u = Ls - 1
        if (pg->inv) {
            R acc = 0;
            for (int u = 0; u < Ls; ++u) {
                const int s = up ? Ls - 1 - u : u;
                acc = kappa * acc + base[s * 24] * d1[s];
            }
            R prev = mneg * (acc * a0inv * pg->corner);
            const bool fin = !pg->shift;
            for (int u = 0; u < Ls; ++u) {
                const int s = up ? Ls - 1 - u : u;
                const R w = base[s * 24] * d1[s] * a0inv + kappa * prev;
                prev = w;
                base[s * 24] = fin ? w * d2[s] : w;
            }
            if (fin) continue;
            R prevs = mneg * base[s_last * 24];
            for (int u = 0; u < Ls; ++u) {
                const int s = up ? Ls - 1 - u : u;
                const R tt = base[s * 24];
                base[s * 24] = (s0 * tt + s1 * prevs) * d2[s];
                prevs = tt;
            }
        } else if (pg->shift) {
            R prevs = mneg * base[s_last * 24] * d1[s_last];
            for (int u = 0; u < Ls; ++u) {
                const int s = up ? Ls - 1 - u : u;
                const R tt = base[s * 24] * d1[s];
                base[s * 24] = (s0 * tt + s1 * prevs) * d2[s];
                prevs = tt;
            }
        } else {
            for (int u = 0; u < Ls; ++u) base[u * 24] *= d1[u] * d2[u];
        }
    }
}

// ------------------------------------------------- tensor-core mixing
// Per chirality the mixing of a CTA's tile is one matrix product
//   D[s][col] = sum_t M[s][t] H[t][col],   col = (site, one of 12 reals),
// [Ls x Ls] x [Ls x 12 nsites], computed with warp-level TF32 MMAs
// (m16n8k8, FP32 accumulation; rows padded to 16, contraction to 8).  TF32
// keeps FP32's exponent range, which the unscaled FP32 tile values need.
// The matrix is split as M = M_hi + M_lo (both exact TF32 values) so that its
// rounding does not enter; with NB = 2 the tile is split the same way and the
// product is M_hi H_hi + M_hi H_lo + M_lo H_hi (FP32-level accuracy, error
// ~2^-21 relative), with NB = 1 it is M_hi H + M_lo H (error ~2^-11 relative
// per element of H, the size of the FP16 storage rounding).
// Tasks are (chirality, 8-column slice); a warp reads all B fragments of its
// task before it writes the task's results, and the slices are disjoint, so
// the tile is transformed in place.  Only full warps (32 consecutive threads)
// take tasks: `nwarps` counts full warps.
__device__ __forceinline__ uint32_t f32_to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mma_tf32_1688(float *d, const uint32_t *a, const uint32_t *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// mt: the mixing matrices in shared memory as the kernels store them,
// element (chi, s, t) at mt[chi*Ls*Ls + t*Ls + (s % LsN)*NS + s / LsN].
// tile: nsites sites, site stride tstride_pairs pairs, row s at 12 s pairs.
template <int NB>
__device__ __forceinline__ void mma_mix_tile(const float *mt, float *tile, int tstride_pairs, int nsites, int Ls,
                                             int NS, int warp, int nwarps)
{
    if (warp >= nwarps) return;   // a partial last warp must not execute mma.sync
    int lane;
    asm("mov.u32 %0, %%laneid;" : "=r"(lane));
    const int g = lane >> 2, c4 = lane & 3;
    const int LsN = Ls / NS, LL = Ls * Ls;
    const int ncols = nsites * 12;
    const int ntiles = (ncols + 7) >> 3;
    const int sstride = tstride_pairs * 2;
    const int nmb = (Ls + 15) >> 4, nkb = (Ls + 7) >> 3;
    auto aval = [&](int chi, int s, int t) -> float {
        return (s < Ls && t < Ls) ? mt[chi * LL + t * Ls + (s % LsN) * NS + s / LsN] : 0.f;
    };
    // float offset in the tile of real `col` (site, q) of chirality chi, row t
    auto baddr = [&](int chi, int col, int t) -> int {
        const int jj = col / 12, q = col - jj * 12;
        return jj * sstride + t * 24 + 4 * (q >> 1) + 2 * chi + (q & 1);
    };
    for (int w = warp; w < 2 * ntiles; w += nwarps) {
        const int chi = w / ntiles, nt = w - chi * ntiles;
        const int col = nt * 8 + g;
        const bool colok = col < ncols;
        uint32_t bh[4][2], bl[4][2];
#pragma unroll
        for (int kb = 0; kb < 4; ++kb)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int t = kb * 8 + c4 + 4 * r;
                const float v = (colok && t < Ls) ? tile[baddr(chi, col, t)] : 0.f;
                bh[kb][r] = f32_to_tf32(v);
                bl[kb][r] = NB == 2 ? f32_to_tf32(v - __uint_as_float(bh[kb][r])) : 0u;
            }
        __syncwarp();
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
            if (mb >= nmb) break;
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
                if (kb >= nkb) break;
                const int s0 = mb * 16 + g, t0 = kb * 8 + c4;
                const float av[4] = {aval(chi, s0, t0), aval(chi, s0 + 8, t0), aval(chi, s0, t0 + 4),
                                     aval(chi, s0 + 8, t0 + 4)};
                uint32_t ah[4], al[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    ah[r] = f32_to_tf32(av[r]);
                    al[r] = f32_to_tf32(av[r] - __uint_as_float(ah[r]));
                }
                mma_tf32_1688(acc[mb], ah, bh[kb]);
                if (NB == 2) mma_tf32_1688(acc[mb], ah, bl[kb]);
                mma_tf32_1688(acc[mb], al, bh[kb]);
            }
        }
        // accumulator element r: row g + 8 (r >> 1) of the block, column 2 c4 + (r & 1) of the slice
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
            if (mb >= nmb) break;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int s = mb * 16 + g + (r >> 1) * 8;
                const int cc = nt * 8 + c4 * 2 + (r & 1);
                if (s < Ls && cc < ncols) tile[baddr(chi, cc, s)] = acc[mb][r];
            }
        }
    }
}

// The tile rows must be 16-byte aligned (row stride 12 pairs, site stride a
// multiple of 2 pairs).
// Cyclic tridiagonal matrix: only t = s - 1, s, s + 1 contribute to row s.
template <int NS, typename T2, typename R>
__device__ __forceinline__ void mix_pairs_band(const R *mt, const T2 *tile, int x, int Ls, T2 (*o)[12])
{
    const int LL = Ls * Ls;
    const int LsN = Ls / NS;
#pragma unroll
    for (int n = 0; n < NS; ++n) {
        const int s = x + n * LsN;
#pragma unroll
        for (int dt = -1; dt <= 1; ++dt) {
            int t = s + dt;
            t = t < 0 ? t + Ls : (t >= Ls ? t - Ls : t);
            T2 h[12];
            ld_tile_row(tile + t * 12, h);
            const T2 cu = p_splat(mt[t * Ls + x * NS + n]);
            const T2 cl = p_splat(mt[LL + t * Ls + x * NS + n]);
#pragma unroll
            for (int p = 0; p < 12; p += 2) {
                o[n][p] = p_fma(cu, h[p], o[n][p]);
                o[n][p + 1] = p_fma(cl, h[p + 1], o[n][p + 1]);
            }
        }
    }
}

template <int NS, typename T2, typename R>
__device__ __forceinline__ void mix_pairs(const R *mt, const T2 *tile, int x, int Ls, T2 (*o)[12])
{
    const int LL = Ls * Ls;
    for (int t = 0; t < Ls; ++t) {
        T2 h[12];
        ld_tile_row(tile + t * 12, h);
#pragma unroll
        for (int n = 0; n < NS; ++n) {
            const T2 cu = p_splat(mt[t * Ls + x * NS + n]);
            const T2 cl = p_splat(mt[LL + t * Ls + x * NS + n]);
#pragma unroll
            for (int p = 0; p < 12; p += 2) {
                o[n][p] = p_fma(cu, h[p], o[n][p]);
                o[n][p + 1] = p_fma(cl, h[p + 1], o[n][p + 1]);
            }
        }
    }
}

}  // namespace dwf
