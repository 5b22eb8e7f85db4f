// Learned gauge-covariant preconditioner for the even-odd normal equation
// (no counterpart in the paper, which solves with plain CG): the network
// kernels (forward, backward to the input, weight gradient), the Adam update,
// the training driver and the vector kernels of flexible CG.
//
// Network.  A field of C = Ls channels is the 5D field itself: channel c of a
// 4D site is its fifth-direction slice s = c, held in the FP32 internal layout
// (parity halves, spin pairs; fields.cuh).  A layer with complex weights
// W[p][chi][c][c'] (p = 0 self, 1 + 2 mu the hop from x + mu, 2 + 2 mu the hop
// from x - mu; chi the chirality of the output spin) computes
//     out(x, c) = sum_p sum_c' W[p][chi][c][c'] T_p(x, c'),
//     T_0 = psi(x),  T_{+mu} = (1 - gamma_mu) U_mu(x) psi(x + mu),
//     T_{-mu} = (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu),
// the spin and colour structure of the Wilson hop (with the boundary phases
// folded into the links), so the layer is gauge covariant.  The preconditioner
// M(r) puts an even-site field r on the even sites (odd sites zero), applies
// L layers and keeps the even sites.  Weights are held in FP64 (Adam master
// copy) and used by the kernels as their BF16-rounded FP32 values; activations
// and accumulation are FP32.
//
// Backward.  grad W[p][chi][c][c'] = sum_{x, alpha in chi} G(x, c)_alpha conj(T_p(x, c')_alpha)
// and the input gradient is the adjoint layer: the channel mixing with
// conj(W)^T first, then the transport of the opposite hop with the flipped
// projector (gamma5 H gamma5 structure).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cuda_bf16.h>
#include <random>
#include <vector>

#include "stencil.cuh"

namespace dwf {
namespace {

constexpr int NHOP = 9;
constexpr int NET_THREADS = 256;

// weight index of link direction d (d < 4: hop from x + d, d >= 4: from x - (d - 4))
__host__ __device__ constexpr int hop_of_dir(int d) { return d < 4 ? 1 + 2 * d : 2 + 2 * (d - 4); }

struct NetLayerArgs {
    FieldRef in[2], out[2];      // parity halves (FP32, C channels = Ls slices)
    const float2 *W = nullptr;   // [9][2][C][C] complex weights of the layer
    const float *gauge[2] = {nullptr, nullptr};   // FP32 links for output parity p: [Vh][8][18]
    const int *nbr[2] = {nullptr, nullptr};       // [Vh][8] for output parity p
    int Vh = 0, C = 0;
    int in_zero[2] = {0, 0};     // input parity q is known to be zero (its terms are skipped)
    int par0 = 0;                // output parity of blockIdx.y = 0
};

// re/im pair accumulation of w t (cmac) and conj(w) t (cmac_conj)
__device__ __forceinline__ void cmac(float2 &re, float2 &im, float2 w, float2 tr, float2 ti)
{
    re = p_fma(p_splat(w.x), tr, re);
    re = p_fma(p_splat(-w.y), ti, re);
    im = p_fma(p_splat(w.x), ti, im);
    im = p_fma(p_splat(w.y), tr, im);
}
__device__ __forceinline__ void cmac_conj(float2 &re, float2 &im, float2 w, float2 tr, float2 ti)
{
    re = p_fma(p_splat(w.x), tr, re);
    re = p_fma(p_splat(w.y), ti, re);
    im = p_fma(p_splat(w.x), ti, im);
    im = p_fma(p_splat(-w.y), tr, im);
}

// T_D(site, c) of input parity q: D = 0 self, D = 1 + d the link direction d
template <int D>
__device__ __forceinline__ void transport_in(const NetLayerArgs &a, int par, int site, int c, float2 *T)
{
    if constexpr (D == 0) {
        ld_pairs<DWF_F32, true>(a.in[par], (size_t)site, c, a.C, T);
    } else {
        constexpr int d = D - 1;
        const int nb = __ldg(a.nbr[par] + (size_t)site * 8 + d);
        float2 v[12], u[9];
        ld_pairs<DWF_F32, true>(a.in[1 - par], (size_t)nb, c, a.C, v);
        load_link<DWF_F32, true>(a.gauge[par] + ((size_t)site * 8 + d) * 18, u);
#pragma unroll
        for (int k = 0; k < 12; ++k) T[k] = make_float2(0.f, 0.f);
        hop_one<d & 3, (d < 4 ? 1 : -1)>(T, u, v);
    }
}

template <int D>
__device__ __forceinline__ void fwd_step(const NetLayerArgs &a, int par, int site, bool active, int c, int j,
                                         const float2 *Wt, float2 *Ts, float2 *acc)
{
    const int C = a.C;
    const int q = D == 0 ? par : 1 - par;
    if (a.in_zero[q]) return;   // uniform over the CTA
    if (active) {
        float2 T[12];
        transport_in<D>(a, par, site, c, T);
        float2 *dst = Ts + ((size_t)j * C + c) * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = T[k];
    }
    __syncthreads();
    if (active) {
        constexpr int p = D == 0 ? 0 : hop_of_dir(D - 1);
        const float2 *W0 = Wt + (size_t)(p * 2) * C * C, *W1 = W0 + (size_t)C * C;
        const float2 *Tj = Ts + (size_t)j * C * 12;
        for (int ci = 0; ci < C; ++ci) {
            const float2 w0 = W0[ci * C + c], w1 = W1[ci * C + c];
            const float2 *t = Tj + ci * 12;
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                cmac(acc[4 * g], acc[4 * g + 2], w0, t[4 * g], t[4 * g + 2]);
                cmac(acc[4 * g + 1], acc[4 * g + 3], w1, t[4 * g + 1], t[4 * g + 3]);
            }
        }
    }
    __syncthreads();
}

// out = layer(in); blockDim = (C, SB), grid = (tiles, parities)
__global__ void __launch_bounds__(NET_THREADS) net_fwd_kernel(const NetLayerArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = a.C, c = threadIdx.x, j = threadIdx.y, SB = blockDim.y;
    const int par = blockIdx.y + a.par0;
    const int site = blockIdx.x * SB + j;
    const bool active = site < a.Vh;
    float2 *Wt = reinterpret_cast<float2 *>(smem_raw);   // [9][2][c'][c]
    float2 *Ts = Wt + (size_t)NHOP * 2 * C * C;          // [SB][C][12]
    const int tid = j * C + c, nt = C * SB, n = NHOP * 2 * C * C;
    for (int k = tid; k < n; k += nt) {
        const int pc = k / (C * C), r = k - pc * C * C, co = r / C, ci = r - co * C;
        Wt[(size_t)pc * C * C + ci * C + co] = a.W[k];
    }
    __syncthreads();
    float2 acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = make_float2(0.f, 0.f);
    fwd_step<0>(a, par, site, active, c, j, Wt, Ts, acc);
    fwd_step<1>(a, par, site, active, c, j, Wt, Ts, acc);
    fwd_step<2>(a, par, site, active, c, j, Wt, Ts, acc);
    fwd_step<3>(a, par, site, active, c, j, Wt, Ts, acc);
    fwd_step<4>(a, par, site, active, c, j, Wt, Ts, acc);
    fwd_step<5>(a, par, site, active, c, j, Wt, Ts, acc);
    fwd_step<6>(a, par, site, active, c, j, Wt, Ts, acc);
    fwd_step<7>(a, par, site, active, c, j, Wt, Ts, acc);
    fwd_step<8>(a, par, site, active, c, j, Wt, Ts, acc);
    if (active) st_pairs<DWF_F32>(a.out[par], (size_t)site, c, C, acc);
}

// adjoint step: gT(c') = sum_c conj(W[p][chi][c][c']) G(nb, c), then the
// opposite hop's transport with the flipped projector
template <int D>
__device__ __forceinline__ void adj_step(const NetLayerArgs &a, int par, int site, bool active, int c, int j,
                                         const float2 *Ws, float2 *Gs, float2 *acc)
{
    const int C = a.C;
    const int q = D == 0 ? par : 1 - par;
    if (a.in_zero[q]) return;
    int nb = site;
    if (active) {
        if constexpr (D > 0) nb = __ldg(a.nbr[par] + (size_t)site * 8 + (D - 1));
        float2 v[12];
        ld_pairs<DWF_F32, true>(a.in[q], (size_t)nb, c, C, v);
        float2 *dst = Gs + ((size_t)j * C + c) * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = v[k];
    }
    __syncthreads();
    if (active) {
        constexpr int p = D == 0 ? 0 : hop_of_dir(((D - 1) + 4) & 7);
        const float2 *W0 = Ws + (size_t)(p * 2) * C * C, *W1 = W0 + (size_t)C * C;
        const float2 *Gj = Gs + (size_t)j * C * 12;
        float2 g[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) g[k] = make_float2(0.f, 0.f);
        for (int co = 0; co < C; ++co) {
            const float2 w0 = W0[co * C + c], w1 = W1[co * C + c];
            const float2 *t = Gj + co * 12;
#pragma unroll
            for (int gg = 0; gg < 3; ++gg) {
                cmac_conj(g[4 * gg], g[4 * gg + 2], w0, t[4 * gg], t[4 * gg + 2]);
                cmac_conj(g[4 * gg + 1], g[4 * gg + 3], w1, t[4 * gg + 1], t[4 * gg + 3]);
            }
        }
        if constexpr (D == 0) {
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = p_add(acc[k], g[k]);
        } else {
            constexpr int d = D - 1;
            float2 u[9];
            load_link<DWF_F32, true>(a.gauge[par] + ((size_t)site * 8 + d) * 18, u);
            hop_one<d & 3, (d < 4 ? -1 : 1)>(acc, u, g);
        }
    }
    __syncthreads();
}

// out = layer^dag(in): the gradient with respect to the layer input, given
// the gradient `in` of its output.
__global__ void __launch_bounds__(NET_THREADS) net_adj_kernel(const NetLayerArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = a.C, c = threadIdx.x, j = threadIdx.y, SB = blockDim.y;
    const int par = blockIdx.y + a.par0;
    const int site = blockIdx.x * SB + j;
    const bool active = site < a.Vh;
    float2 *Ws = reinterpret_cast<float2 *>(smem_raw);   // [9][2][c][c'] as given
    float2 *Gs = Ws + (size_t)NHOP * 2 * C * C;          // [SB][C][12]
    const int tid = j * C + c, nt = C * SB, n = NHOP * 2 * C * C;
    for (int k = tid; k < n; k += nt) Ws[k] = a.W[k];
    __syncthreads();
    float2 acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = make_float2(0.f, 0.f);
    adj_step<0>(a, par, site, active, c, j, Ws, Gs, acc);
    adj_step<1>(a, par, site, active, c, j, Ws, Gs, acc);
    adj_step<2>(a, par, site, active, c, j, Ws, Gs, acc);
    adj_step<3>(a, par, site, active, c, j, Ws, Gs, acc);
    adj_step<4>(a, par, site, active, c, j, Ws, Gs, acc);
    adj_step<5>(a, par, site, active, c, j, Ws, Gs, acc);
    adj_step<6>(a, par, site, active, c, j, Ws, Gs, acc);
    adj_step<7>(a, par, site, active, c, j, Ws, Gs, acc);
    adj_step<8>(a, par, site, active, c, j, Ws, Gs, acc);
    if (active) st_pairs<DWF_F32>(a.out[par], (size_t)site, c, C, acc);
}

// Weight gradient of one layer: a.in = layer input psi, a.out = gradient G of
// the layer output (read only).  Persistent CTAs over the (parity, tile)
// work items; each thread < C*C owns one (c, c') and accumulates its 18
// (hop, chirality) sums; partials[block][p][chi][c][c'].
template <int D>
__device__ __forceinline__ void wgrad_step(const NetLayerArgs &a, int par, int site, bool active, int c, int j,
                                           float2 *Ts, const float2 *Gs, float2 (*accr)[2], float2 (*acci)[2], int co,
                                           int ci, bool owner)
{
    const int C = a.C;
    const int q = D == 0 ? par : 1 - par;
    if (a.in_zero[q]) return;
    if (active) {
        float2 T[12];
        transport_in<D>(a, par, site, c, T);
        float2 *dst = Ts + ((size_t)j * C + c) * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = T[k];
    }
    __syncthreads();
    if (owner) {
        constexpr int p = D == 0 ? 0 : hop_of_dir(D - 1);
        const int SB = blockDim.y;
        for (int jj = 0; jj < SB; ++jj) {
            const float2 *G = Gs + ((size_t)jj * C + co) * 12;
            const float2 *T = Ts + ((size_t)jj * C + ci) * 12;
#pragma unroll
            for (int g = 0; g < 3; ++g)
#pragma unroll
                for (int chi = 0; chi < 2; ++chi) {
                    const float2 gr = G[4 * g + chi], gi = G[4 * g + 2 + chi];
                    const float2 tr = T[4 * g + chi], ti = T[4 * g + 2 + chi];
                    // G conj(T) = (gr tr + gi ti) + i (gi tr - gr ti), per spin of the pair
                    accr[p][chi] = p_fma(gr, tr, accr[p][chi]);
                    accr[p][chi] = p_fma(gi, ti, accr[p][chi]);
                    acci[p][chi] = p_fma(gi, tr, acci[p][chi]);
                    acci[p][chi] = p_fma(make_float2(-gr.x, -gr.y), ti, acci[p][chi]);
                }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(NET_THREADS) net_wgrad_kernel(const NetLayerArgs a, float2 *partials)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = a.C, c = threadIdx.x, j = threadIdx.y, SB = blockDim.y;
    const int tid = j * C + c;
    float2 *Ts = reinterpret_cast<float2 *>(smem_raw);   // [SB][C][12]
    float2 *Gs = Ts + (size_t)SB * C * 12;
    const bool owner = tid < C * C;
    const int co = owner ? tid / C : 0, ci = owner ? tid % C : 0;
    float2 accr[NHOP][2], acci[NHOP][2];
#pragma unroll
    for (int p = 0; p < NHOP; ++p)
#pragma unroll
        for (int chi = 0; chi < 2; ++chi) accr[p][chi] = acci[p][chi] = make_float2(0.f, 0.f);
    const int ntile = (a.Vh + SB - 1) / SB;
    for (int w = blockIdx.x; w < 2 * ntile; w += gridDim.x) {
        const int par = w / ntile, tile = w - par * ntile;
        if (a.out[par].v == nullptr) continue;   // the gradient is zero on this parity (uniform)
        const int site = tile * SB + j;
        const bool active = site < a.Vh;
        float2 g[12];
        if (active) {
            ld_pairs<DWF_F32, true>(a.out[par], (size_t)site, c, C, g);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) g[k] = make_float2(0.f, 0.f);
        }
        float2 *dst = Gs + ((size_t)j * C + c) * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = g[k];
        wgrad_step<0>(a, par, site, active, c, j, Ts, Gs, accr, acci, co, ci, owner);
        wgrad_step<1>(a, par, site, active, c, j, Ts, Gs, accr, acci, co, ci, owner);
        wgrad_step<2>(a, par, site, active, c, j, Ts, Gs, accr, acci, co, ci, owner);
        wgrad_step<3>(a, par, site, active, c, j, Ts, Gs, accr, acci, co, ci, owner);
        wgrad_step<4>(a, par, site, active, c, j, Ts, Gs, accr, acci, co, ci, owner);
        wgrad_step<5>(a, par, site, active, c, j, Ts, Gs, accr, acci, co, ci, owner);
        wgrad_step<6>(a, par, site, active, c, j, Ts, Gs, accr, acci, co, ci, owner);
        wgrad_step<7>(a, par, site, active, c, j, Ts, Gs, accr, acci, co, ci, owner);
        wgrad_step<8>(a, par, site, active, c, j, Ts, Gs, accr, acci, co, ci, owner);
        __syncthreads();   // Gs is rewritten by the next work item
    }
    if (owner) {
        float2 *out = partials + (size_t)blockIdx.x * NHOP * 2 * C * C;
#pragma unroll
        for (int p = 0; p < NHOP; ++p)
#pragma unroll
            for (int chi = 0; chi < 2; ++chi)
                out[((size_t)(p * 2 + chi) * C + co) * C + ci] =
                    make_float2(accr[p][chi].x + accr[p][chi].y, acci[p][chi].x + acci[p][chi].y);
    }
}

// gacc[k] += sum_b partials[b][k], b in index order (deterministic)
__global__ void net_reduce_kernel(const float2 *partials, int nblocks, int n, double2 *gacc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double sr = 0, si = 0;
    for (int b = 0; b < nblocks; ++b) {
        const float2 v = partials[(size_t)b * n + k];
        sr += v.x;
        si += v.y;
    }
    gacc[k] = make_double2(gacc[k].x + sr, gacc[k].y + si);
}

// Adam (Kingma and Ba 2015) on the real and imaginary parts separately; the
// FP32 compute copy holds the BF16 rounding of the updated master weights;
// the gradient accumulator is cleared.
__global__ void net_adam_kernel(double2 *W, double2 *m, double2 *v, double2 *g, float2 *Wc, int n, double lr,
                                double b1, double b2, double eps, double c1, double c2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double2 gg = g[k];
    double2 mm = m[k], vv = v[k], w = W[k];
    mm.x = b1 * mm.x + (1 - b1) * gg.x;
    mm.y = b1 * mm.y + (1 - b1) * gg.y;
    vv.x = b2 * vv.x + (1 - b2) * gg.x * gg.x;
    vv.y = b2 * vv.y + (1 - b2) * gg.y * gg.y;
    w.x -= lr * (mm.x / c1) / (sqrt(vv.x / c2) + eps);
    w.y -= lr * (mm.y / c1) / (sqrt(vv.y / c2) + eps);
    m[k] = mm;
    v[k] = vv;
    W[k] = w;
    g[k] = make_double2(0.0, 0.0);
    Wc[k] = make_float2(__bfloat162float(__float2bfloat16_rn((float)w.x)),
                        __bfloat162float(__float2bfloat16_rn((float)w.y)));
}

__global__ void net_round_kernel(const double2 *W, float2 *Wc, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    Wc[k] = make_float2(__bfloat162float(__float2bfloat16_rn((float)W[k].x)),
                        __bfloat162float(__float2bfloat16_rn((float)W[k].y)));
}

// ----------------------------------------------------------- vector kernels
// FP32 internal fields of one parity, n = Vh * Ls * 24 reals viewed as float4.
__global__ void __launch_bounds__(256) vdot_kernel(const float4 *x, const float4 *y, size_t n4, RedArgs red)
{
    double s = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const float4 a = x[i], b = y[i];
        // four products in FP32, one FP64 addition (FP64 arithmetic is slow on GB300)
        s += (double)fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
    }
    grid_reduce(s, red);
}

// y = a x + b y (y is not read when b = 0, so that it may hold anything)
__global__ void __launch_bounds__(256) vaxpby_kernel(float a, const float4 *x, float b, float4 *y, size_t n4)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const float4 u = x[i];
        float4 w = b != 0.f ? y[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        w.x = a * u.x + b * w.x;
        w.y = a * u.y + b * w.y;
        w.z = a * u.z + b * w.z;
        w.w = a * u.w + b * w.w;
        y[i] = w;
    }
}

// loss of one pair: G = s (y - x) on the even half, |y - x|^2 reduced
__global__ void __launch_bounds__(256) net_loss_kernel(const float4 *y, const float4 *x, float4 *G, float s, size_t n4,
                                                        RedArgs red)
{
    double acc = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const float4 a = y[i], b = x[i];
        const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        acc += (double)fmaf(d.w, d.w, fmaf(d.z, d.z, fmaf(d.y, d.y, d.x * d.x)));
        G[i] = make_float4(s * d.x, s * d.y, s * d.z, s * d.w);
    }
    grid_reduce(acc, red);
}

// Gaussian N(0, 1) reals for white-noise training vectors: counter-based
// (SplitMix64 of seed and index, Steele, Lea and Flood 2014), Box-Muller.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
__global__ void fill_gaussian_kernel(float *x, size_t n, unsigned long long seed)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long r = splitmix64(seed * 0x100000001b3ULL + i);
        const float u1 = ((float)(r >> 40) + 1.0f) * (1.0f / 16777217.0f);   // (0, 1]
        const float u2 = (float)((r >> 16) & 0xffffffULL) * (1.0f / 16777216.0f);
        x[i] = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    }
}

int reduce_grid(size_t n4)
{
    size_t b = (n4 + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return b < 1 ? 1 : (int)b;
}

size_t net_smem(int C, int SB) { return ((size_t)NHOP * 2 * C * C + (size_t)SB * C * 12) * sizeof(float2); }

}  // namespace

// ------------------------------------------------------------ host side
struct NetState {
    int L = 0, C = 0;
    size_t nw = 0;                 // complex weights per layer (9 * 2 * C * C)
    double2 *Wm = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;   // [L][nw]
    float2 *Wc = nullptr;          // [L][nw] BF16-rounded compute copy
    float2 *partials = nullptr;    // [nparts][nw]
    int nparts = 0;
    int t = 0;                     // Adam steps taken
    std::vector<FieldRef> pb, px;  // training pairs (FP32 even fields)
    std::vector<double> pxn2;
    std::vector<void *> pair_mem;
};

}  // namespace dwf

using namespace dwf;

namespace dwf_detail {
HopArgs hop_args(dwf_ctx *h, int prec, int out_par, FieldRef in, FieldRef out, int post);
RedArgs red(dwf_ctx *h, int op, CgScalars *scal);
}  // namespace dwf_detail
using namespace dwf_detail;

#define CK(call)                                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return dwf_cuda_error(e_, #call);      \
    } while (0)

void dwf_precond_release(dwf_ctx *h)
{
    NetState *N = h->net;
    if (!N) return;
    cudaFree(N->Wm);
    cudaFree(N->m);
    cudaFree(N->v);
    cudaFree(N->g);
    cudaFree(N->Wc);
    cudaFree(N->partials);
    for (void *p : N->pair_mem) cudaFree(p);
    delete N;
    h->net = nullptr;
}

namespace dwf {

static int net_sb(int C) { return NET_THREADS / C; }

static NetLayerArgs layer_args(dwf_ctx *h, const float2 *W)
{
    NetLayerArgs a;
    a.W = W;
    for (int p = 0; p < 2; ++p) {
        a.gauge[p] = (const float *)h->gauge_for(DWF_F32, p);
        a.nbr[p] = h->nbr_for(p);
    }
    a.Vh = h->Vh;
    a.C = h->Ls;
    return a;
}

static cudaError_t launch_net_layer(dwf_ctx *h, bool adj, NetLayerArgs a, int npar, cudaStream_t st)
{
    const int SB = net_sb(a.C);
    const size_t smem = net_smem(a.C, SB);
    static unsigned long long optin[3] = {0, 0, 0};
    {
        cudaError_t e = smem_optin(net_fwd_kernel, 200 * 1024, optin[0]);
        if (e == cudaSuccess) e = smem_optin(net_adj_kernel, 200 * 1024, optin[1]);
        if (e == cudaSuccess) e = smem_optin(net_wgrad_kernel, 200 * 1024, optin[2]);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((a.Vh + SB - 1) / SB, npar);
    h->launches += 1;
    if (adj)
        net_adj_kernel<<<grid, dim3(a.C, SB), smem, st>>>(a);
    else
        net_fwd_kernel<<<grid, dim3(a.C, SB), smem, st>>>(a);
    return cudaGetLastError();
}

// M(r): r, z even FP32 fields; work: act[l][par] activations (l = 0 .. L-2 both parities)
static cudaError_t net_forward(dwf_ctx *h, FieldRef r, FieldRef z, FieldRef (*act)[2], cudaStream_t st)
{
    NetState *N = h->net;
    FieldRef zero;
    FieldRef cur[2] = {r, zero};
    int cz[2] = {0, 1};
    for (int l = 0; l < N->L; ++l) {
        NetLayerArgs a = layer_args(h, N->Wc + (size_t)l * N->nw);
        a.in[0] = cur[0];
        a.in[1] = cur[1];
        a.in_zero[0] = cz[0];
        a.in_zero[1] = cz[1];
        const bool last = (l == N->L - 1);
        if (last) {
            a.out[0] = z;
            a.par0 = 0;
        } else {
            a.out[0] = act[l][0];
            a.out[1] = act[l][1];
        }
        cudaError_t e = launch_net_layer(h, false, a, last ? 1 : 2, st);
        if (e != cudaSuccess) return e;
        if (!last) {
            cur[0] = act[l][0];
            cur[1] = act[l][1];
            cz[0] = cz[1] = 0;
        }
    }
    return cudaSuccess;
}

// N^dag r: the adjoint layers in reverse order (r, out even FP32 fields)
static cudaError_t net_adjoint(dwf_ctx *h, FieldRef r, FieldRef out, FieldRef (*act)[2], cudaStream_t st)
{
    NetState *N = h->net;
    FieldRef zero;
    FieldRef cur[2] = {r, zero};
    int cz[2] = {0, 1};
    for (int l = N->L - 1; l >= 0; --l) {
        NetLayerArgs a = layer_args(h, N->Wc + (size_t)l * N->nw);
        a.in[0] = cur[0];
        a.in[1] = cur[1];
        a.in_zero[0] = cz[0];
        a.in_zero[1] = cz[1];
        const bool last = (l == 0);
        if (last) {
            a.out[0] = out;
            a.par0 = 0;
        } else {
            a.out[0] = act[l - 1][0];
            a.out[1] = act[l - 1][1];
        }
        cudaError_t e = launch_net_layer(h, true, a, last ? 1 : 2, st);
        if (e != cudaSuccess) return e;
        if (!last) {
            cur[0] = act[l - 1][0];
            cur[1] = act[l - 1][1];
            cz[0] = cz[1] = 0;
        }
    }
    return cudaSuccess;
}

struct NetWork {
    FieldRef act[8][2];    // activations after layers 0 .. L-2
    FieldRef grad[8][2];   // gradients of layer outputs
    FieldRef y;            // network output (even)
};

static int net_work(dwf_ctx *h, NetWork &W)
{
    cudaError_t e = cudaSuccess;
    NetState *N = h->net;
    for (int l = 0; l + 1 < N->L; ++l)
        for (int p = 0; p < 2; ++p) {
            W.act[l][p] = h->field("nn_act" + std::to_string(l) + (p ? "o" : "e"), DWF_F32, &e);
            W.grad[l][p] = h->field("nn_grad" + std::to_string(l) + (p ? "o" : "e"), DWF_F32, &e);
            if (!W.act[l][p].v || !W.grad[l][p].v) return dwf_cuda_error(e, "network workspace");
        }
    W.grad[N->L - 1][0] = h->field("nn_gradLe", DWF_F32, &e);
    W.y = h->field("nn_y", DWF_F32, &e);
    if (!W.grad[N->L - 1][0].v || !W.y.v) return dwf_cuda_error(e, "network workspace");
    return DWF_OK;
}

static cudaError_t net_wgrad(dwf_ctx *h, int l, FieldRef in0, FieldRef in1, int in_zero1, FieldRef g0, FieldRef g1,
                             cudaStream_t st)
{
    NetState *N = h->net;
    NetLayerArgs a = layer_args(h, N->Wc + (size_t)l * N->nw);
    a.in[0] = in0;
    a.in[1] = in1;
    a.in_zero[1] = in_zero1;
    a.out[0] = g0;
    a.out[1] = g1;
    const int SB = net_sb(a.C);
    const size_t smem = (size_t)2 * SB * a.C * 12 * sizeof(float2);
    net_wgrad_kernel<<<N->nparts, dim3(a.C, SB), smem, st>>>(a, N->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n = (int)N->nw;
    net_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(N->partials, N->nparts, n, N->g + (size_t)l * N->nw);
    h->launches += 2;
    return cudaGetLastError();
}

// Loss and gradient of one pair (b, x), added into N->g; |y - x|^2 -> scal->last
static int net_pair_grad(dwf_ctx *h, NetWork &W, FieldRef b, FieldRef x, double xn2, double K, CgScalars *scal,
                         cudaStream_t st)
{
    NetState *N = h->net;
    const int L = N->L;
    CK(net_forward(h, b, W.y, W.act, st));
    const size_t n4 = field_bytes(DWF_F32, h->Vh, h->Ls) / 16;
    FieldRef GL = W.grad[L - 1][0];
    net_loss_kernel<<<reduce_grid(n4), 256, 0, st>>>((const float4 *)W.y.v, (const float4 *)x.v, (float4 *)GL.v,
                                                    (float)(2.0 / (xn2 * K)), n4, red(h, RED_STORE, scal));
    CK(cudaGetLastError());
    h->launches += 1;
    FieldRef none;
    // layer l has input act[l-1] (b on even sites for l = 0) and output gradient grad[l]
    for (int l = L - 1; l >= 0; --l) {
        FieldRef in0 = l == 0 ? b : W.act[l - 1][0];
        FieldRef in1 = l == 0 ? none : W.act[l - 1][1];
        FieldRef g0 = W.grad[l][0], g1 = (l == L - 1) ? none : W.grad[l][1];
        CK(net_wgrad(h, l, in0, in1, l == 0 ? 1 : 0, g0, g1, st));
        if (l == 0) break;
        NetLayerArgs a = layer_args(h, N->Wc + (size_t)l * N->nw);
        a.in[0] = g0;
        a.in[1] = g1;
        a.in_zero[1] = (l == L - 1) ? 1 : 0;
        a.out[0] = W.grad[l - 1][0];
        a.out[1] = W.grad[l - 1][1];
        CK(launch_net_layer(h, true, a, 2, st));
    }
    return DWF_OK;
}

static int pack_even_f32(dwf_ctx *h, const void *canon, FieldRef out, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    FieldRef t64 = h->field("nn_t64", DWF_F64, &e);
    if (!t64.v) return dwf_cuda_error(e, "workspace");
    CK(launch_pack_eo(DWF_F64, (const double *)canon, t64, h->Vh, h->Ls, st));
    CK(launch_convert(DWF_F64, t64, DWF_F32, out, h->Vh, h->Ls, st));
    h->launches += 2;
    return DWF_OK;
}

static int net_alloc(dwf_ctx *h, int L)
{
    if (L < 1 || L > 8) return dwf_set_error(DWF_EINVAL, "layers must be in [1, 8]");
    if (h->Ls > 16) return dwf_set_error(DWF_EINVAL, "the learned preconditioner needs Ls <= 16 (channels = Ls)");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    if (h->net && h->net->L == L) return DWF_OK;
    dwf_precond_release(h);
    NetState *N = new NetState();
    h->net = N;
    N->L = L;
    N->C = h->Ls;
    N->nw = (size_t)NHOP * 2 * N->C * N->C;
    const size_t nall = N->nw * L;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    N->nparts = nsm * 4;
    CK(cudaMalloc(&N->Wm, nall * sizeof(double2)));
    CK(cudaMalloc(&N->m, nall * sizeof(double2)));
    CK(cudaMalloc(&N->v, nall * sizeof(double2)));
    CK(cudaMalloc(&N->g, nall * sizeof(double2)));
    CK(cudaMalloc(&N->Wc, nall * sizeof(float2)));
    CK(cudaMalloc(&N->partials, (size_t)N->nparts * N->nw * sizeof(float2)));
    CK(cudaMemset(N->m, 0, nall * sizeof(double2)));
    CK(cudaMemset(N->v, 0, nall * sizeof(double2)));
    CK(cudaMemset(N->g, 0, nall * sizeof(double2)));
    return DWF_OK;
}

static int net_upload(dwf_ctx *h, const std::vector<double> &w)
{
    NetState *N = h->net;
    const size_t nall = N->nw * N->L;
    CK(cudaMemcpy(N->Wm, w.data(), nall * sizeof(double2), cudaMemcpyHostToDevice));
    net_round_kernel<<<(int)((nall + 255) / 256), 256>>>(N->Wm, N->Wc, (int)nall);
    CK(cudaGetLastError());
    CK(cudaMemset(N->m, 0, nall * sizeof(double2)));
    CK(cudaMemset(N->v, 0, nall * sizeof(double2)));
    CK(cudaMemset(N->g, 0, nall * sizeof(double2)));
    CK(cudaDeviceSynchronize());
    N->t = 0;
    return DWF_OK;
}

// One Adam step (beta 0.9, 0.999, eps 1e-8; step count t from 1) from the
// gradient accumulated in N->g, which the step clears.
static cudaError_t net_adam(dwf_ctx *h, double lr, cudaStream_t st)
{
    NetState *N = h->net;
    const size_t nall = N->nw * N->L;
    N->t += 1;
    const double c1 = 1 - std::pow(0.9, N->t), c2 = 1 - std::pow(0.999, N->t);
    net_adam_kernel<<<(int)((nall + 255) / 256), 256, 0, st>>>(N->Wm, N->m, N->v, N->g, N->Wc, (int)nall, lr, 0.9,
                                                               0.999, 1e-8, c1, c2);
    h->launches += 1;
    return cudaGetLastError();
}

// File format of dwf_precond_save / dwf_precond_load (little-endian host
// binary): the header, then the FP64 master weights, Adam's first and second
// moments, nall complex numbers each (nall = layers * 9 * 2 * C * C).
struct NetFileHeader {
    char magic[8];              // "DWFNET\0\0"
    int32_t version;            // 1
    int32_t layers, channels;   // L, C = Ls
    int32_t adam_t;             // Adam steps taken
    int64_t nall;               // complex numbers per array
};
static const char kNetMagic[8] = {'D', 'W', 'F', 'N', 'E', 'T', 0, 0};

// which = 0: z = N r, 1: z = N^dag r, 2: z = M r = N N^dag r (FP32 even fields;
// 2 is the preconditioner of flexible CG)
int net_apply_f32(dwf_ctx *h, FieldRef r, FieldRef z, cudaStream_t st, int which)
{
    if (!h->net) return dwf_set_error(DWF_EINVAL, "no preconditioner (dwf_precond_init or dwf_precond_train first)");
    NetWork W;
    int rc = net_work(h, W);
    if (rc) return rc;
    if (which == 0) {
        CK(net_forward(h, r, z, W.act, st));
    } else if (which == 1) {
        CK(net_adjoint(h, r, z, W.act, st));
    } else {
        cudaError_t e = cudaSuccess;
        FieldRef t = h->field("nn_adj", DWF_F32, &e);
        if (!t.v) return dwf_cuda_error(e, "network workspace");
        CK(net_adjoint(h, r, t, W.act, st));
        CK(net_forward(h, t, z, W.act, st));
    }
    return DWF_OK;
}

cudaError_t launch_vdot(FieldRef x, FieldRef y, int Vh, int Ls, const RedArgs &red, cudaStream_t st)
{
    const size_t n4 = field_bytes(DWF_F32, Vh, Ls) / 16;
    vdot_kernel<<<reduce_grid(n4), 256, 0, st>>>((const float4 *)x.v, (const float4 *)y.v, n4, red);
    return cudaGetLastError();
}

cudaError_t launch_vaxpby(float a, FieldRef x, float b, FieldRef y, int Vh, int Ls, cudaStream_t st)
{
    const size_t n4 = field_bytes(DWF_F32, Vh, Ls) / 16;
    vaxpby_kernel<<<reduce_grid(n4), 256, 0, st>>>(a, (const float4 *)x.v, b, (float4 *)y.v, n4);
    return cudaGetLastError();
}

}  // namespace dwf

// ------------------------------------------------------------------- ABI
extern "C" {

void dwf_train_params_default(dwf_train_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->layers = 3;
    p->epochs = 20;
    p->batch = 16;
    p->lr = 2e-3;
    p->solve_inner_prec = DWF_F16;
    p->solve_tol = 1e-8;
    p->seed = 7;
    p->noise = 1e-3;
    p->verbose = 0;
    p->random_pairs = -1;
}

int dwf_precond_init(dwf_handle h, int layers, unsigned long long seed, double noise)
{
    if (!h) return dwf_set_error(DWF_EINVAL, "NULL handle");
    int rc = net_alloc(h, layers);
    if (rc) return rc;
    NetState *N = h->net;
    std::vector<double> w(2 * N->nw * N->L, 0.0);
    std::mt19937_64 gen(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (size_t k = 0; k < w.size(); ++k) w[k] = noise * nd(gen);
    for (int l = 0; l < N->L; ++l)
        for (int chi = 0; chi < 2; ++chi)
            for (int c = 0; c < N->C; ++c) w[2 * (l * N->nw + ((size_t)chi * N->C + c) * N->C + c)] += 1.0;
    return net_upload(h, w);
}

int dwf_precond_set_weights(dwf_handle h, int layers, const double *w)
{
    if (!h || !w) return dwf_set_error(DWF_EINVAL, "NULL argument");
    int rc = net_alloc(h, layers);
    if (rc) return rc;
    NetState *N = h->net;
    std::vector<double> v(w, w + 2 * N->nw * N->L);
    return net_upload(h, v);
}

int dwf_precond_get_weights(dwf_handle h, int layers, int compute_copy, double *w)
{
    if (!h || !w) return dwf_set_error(DWF_EINVAL, "NULL argument");
    if (!h->net || h->net->L != layers) return dwf_set_error(DWF_EINVAL, "no preconditioner with that many layers");
    NetState *N = h->net;
    const size_t nall = N->nw * N->L;
    if (compute_copy) {
        std::vector<float2> c(nall);
        CK(cudaMemcpy(c.data(), N->Wc, nall * sizeof(float2), cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < nall; ++k) w[2 * k] = c[k].x, w[2 * k + 1] = c[k].y;
    } else {
        CK(cudaMemcpy(w, N->Wm, nall * sizeof(double2), cudaMemcpyDeviceToHost));
    }
    return DWF_OK;
}

int dwf_precond_apply(dwf_handle h, int which, const void *in, void *out, void *stream)
{
    if (!h || !in || !out) return dwf_set_error(DWF_EINVAL, "NULL argument");
    if (h && h->slab) return dwf_set_error(DWF_EINVAL, "a slab handle applies its operator through dwf_slab_apply_eo");
    if (which < 0 || which > 2) return dwf_set_error(DWF_EINVAL, "which must be 0 (N), 1 (N^dag) or 2 (N N^dag)");
    if (!h->net) return dwf_set_error(DWF_EINVAL, "no preconditioner (dwf_precond_init or dwf_precond_train first)");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    FieldRef r = h->field("nn_r", DWF_F32, &e), z = h->field("nn_z", DWF_F32, &e);
    FieldRef z64 = h->field("nn_z64", DWF_F64, &e);
    if (!r.v || !z.v || !z64.v) return dwf_cuda_error(e, "workspace");
    int rc = pack_even_f32(h, in, r, st);
    if (rc) return rc;
    rc = net_apply_f32(h, r, z, st, which);
    if (rc) return rc;
    CK(launch_convert(DWF_F32, z, DWF_F64, z64, h->Vh, h->Ls, st));
    CK(launch_unpack_eo(DWF_F64, z64, (double *)out, h->Vh, h->Ls, st));
    h->launches += 2;
    return DWF_OK;
}

int dwf_precond_loss_grad(dwf_handle h, int npairs, const void *const *b, const void *const *x, double *loss,
                          double *grad, void *stream)
{
    if (!h || npairs < 1 || !b || !x) return dwf_set_error(DWF_EINVAL, "bad argument");
    if (h && h->slab) return dwf_set_error(DWF_EINVAL, "a slab handle applies its operator through dwf_slab_apply_eo");
    if (!h->net) return dwf_set_error(DWF_EINVAL, "no preconditioner");
    cudaStream_t st = (cudaStream_t)stream;
    NetState *N = h->net;
    NetWork W;
    int rc = net_work(h, W);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    FieldRef fb = h->field("nn_pb", DWF_F32, &e), fx = h->field("nn_px", DWF_F32, &e);
    if (!fb.v || !fx.v) return dwf_cuda_error(e, "workspace");
    const size_t nall = N->nw * N->L;
    CK(cudaMemsetAsync(N->g, 0, nall * sizeof(double2), st));
    CgScalars *sc = h->scal + 3;
    double L = 0;
    for (int k = 0; k < npairs; ++k) {
        if ((rc = pack_even_f32(h, b[k], fb, st))) return rc;
        if ((rc = pack_even_f32(h, x[k], fx, st))) return rc;
        CK(launch_norm2(DWF_F32, fx, h->Vh, h->Ls, red(h, RED_STORE, sc), st));
        CgScalars hs;
        CK(cudaMemcpyAsync(&hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const double xn2 = hs.last;
        if (!(xn2 > 0)) return dwf_set_error(DWF_EINVAL, "a solution of the pairs is zero");
        if ((rc = net_pair_grad(h, W, fb, fx, xn2, npairs, sc, st))) return rc;
        CK(cudaMemcpyAsync(&hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        L += hs.last / xn2 / npairs;
    }
    if (loss) *loss = L;
    if (grad) CK(cudaMemcpy(grad, N->g, nall * sizeof(double2), cudaMemcpyDeviceToHost));
    CK(cudaMemset(N->g, 0, nall * sizeof(double2)));
    return DWF_OK;
}

int dwf_precond_train(dwf_handle h, int nsrc, const void *const *b4, const dwf_train_params *tp,
                      dwf_train_stats *stats, void *stream)
{
    if (!h || nsrc < 1 || !b4) return dwf_set_error(DWF_EINVAL, "bad argument");
    if (h && h->slab) return dwf_set_error(DWF_EINVAL, "a slab handle applies its operator through dwf_slab_apply_eo");
    dwf_train_params defp;
    dwf_train_params_default(&defp);
    dwf_train_params pv = tp ? *tp : defp;
    if (pv.random_pairs < 0) pv.random_pairs = nsrc;
    const dwf_train_params *p = &pv;
    if (p->epochs < 0 || p->batch < 1 || !(p->lr > 0)) return dwf_set_error(DWF_EINVAL, "bad training parameters");
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    dwf_train_stats S;
    std::memset(&S, 0, sizeof(S));
    int rc;
    if (!h->net || h->net->L != p->layers)
        if ((rc = dwf_precond_init(h, p->layers, p->seed, p->noise))) return rc;
    NetState *N = h->net;
    // training pairs: x = the even part of the solution of D5 x5 = b5(b4), b = D x (D even-odd)
    for (void *q : N->pair_mem) cudaFree(q);
    N->pair_mem.clear();
    N->pb.clear();
    N->px.clear();
    N->pxn2.clear();
    cudaError_t e = cudaSuccess;
    const size_t b5b = (size_t)h->V * h->Ls * 24 * 8;
    void *b5 = h->ws("nn_b5", b5b, &e), *x5 = h->ws("nn_x5", b5b, &e);
    FieldRef xe64 = h->field("nn_xe64", DWF_F64, &e), xo64 = h->field("nn_xo64", DWF_F64, &e);
    if (!b5 || !x5 || !xe64.v) return dwf_cuda_error(e, "workspace");
    const size_t fb = field_bytes(DWF_F32, h->Vh, h->Ls);
    dwf_solve_params sp;
    dwf_solve_params_default(&sp);
    sp.inner_prec = p->solve_inner_prec;
    sp.tol = p->solve_tol;
    auto ts = std::chrono::steady_clock::now();
    CgScalars *sc = h->scal + 3;
    for (int k = 0; k < nsrc; ++k) {
        if ((rc = dwf_source_5d(h, b4[k], b5, stream))) return rc;
        dwf_solve_stats ss;
        rc = dwf_solve(h, b5, x5, &sp, &ss, stream);
        if (rc != DWF_OK && rc != DWF_ENOTCONV) return rc;
        void *mem = nullptr;
        CK(cudaMalloc(&mem, 2 * ((fb + 255) & ~(size_t)255)));
        N->pair_mem.push_back(mem);
        FieldRef fx, fbb;
        fx.v = mem;
        fbb.v = (char *)mem + ((fb + 255) & ~(size_t)255);
        CK(launch_pack_full(DWF_F64, (const double *)x5, xe64, xo64, h->eo2lex, h->Vh, h->V, h->Ls, st));
        CK(launch_convert(DWF_F64, xe64, DWF_F32, fx, h->Vh, h->Ls, st));
        h->launches += 2;
        if ((rc = eo_apply_f32(h, fx, fbb, st))) return rc;
        CK(launch_norm2(DWF_F32, fx, h->Vh, h->Ls, red(h, RED_STORE, sc), st));
        CgScalars hs;
        CK(cudaMemcpyAsync(&hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        N->px.push_back(fx);
        N->pb.push_back(fbb);
        N->pxn2.push_back(hs.last);
    }
    // white-noise pairs: x Gaussian, b = D x (they constrain N on the modes the
    // solutions of smooth sources hardly contain)
    for (int k = 0; k < p->random_pairs; ++k) {
        void *mem = nullptr;
        CK(cudaMalloc(&mem, 2 * ((fb + 255) & ~(size_t)255)));
        N->pair_mem.push_back(mem);
        FieldRef fx, fbb;
        fx.v = mem;
        fbb.v = (char *)mem + ((fb + 255) & ~(size_t)255);
        const size_t nreal = fb / 4;
        fill_gaussian_kernel<<<reduce_grid(nreal / 4), 256, 0, st>>>((float *)fx.v, nreal, p->seed * 7919ULL + k);
        CK(cudaGetLastError());
        h->launches += 1;
        if ((rc = eo_apply_f32(h, fx, fbb, st))) return rc;
        CK(launch_norm2(DWF_F32, fx, h->Vh, h->Ls, red(h, RED_STORE, sc), st));
        CgScalars hs;
        CK(cudaMemcpyAsync(&hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        N->px.push_back(fx);
        N->pb.push_back(fbb);
        N->pxn2.push_back(hs.last);
    }
    nsrc = (int)N->px.size();
    S.solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - ts).count();
    // least-squares scale of the output layer: N = s I minimises sum |s b - x|^2/|x|^2
    {
        double num = 0, den = 0;
        for (int k = 0; k < nsrc; ++k) {
            CgScalars hs[2];
            CK(launch_vdot(N->pb[k], N->px[k], h->Vh, h->Ls, red(h, RED_STORE, sc), st));
            CK(launch_norm2(DWF_F32, N->pb[k], h->Vh, h->Ls, red(h, RED_STORE, sc + 1), st));
            CK(cudaMemcpyAsync(hs, sc, 2 * sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            num += hs[0].last / N->pxn2[k];
            den += hs[1].last / N->pxn2[k];
        }
        if (N->t == 0 && den > 0) {
            std::vector<double> w(2 * N->nw * N->L);
            CK(cudaMemcpy(w.data(), N->Wm, w.size() * sizeof(double), cudaMemcpyDeviceToHost));
            const int l = N->L - 1;
            for (size_t k = 0; k < N->nw; ++k) {
                w[2 * (l * N->nw + k)] *= num / den;
                w[2 * (l * N->nw + k) + 1] *= num / den;
            }
            if ((rc = net_upload(h, w))) return rc;
        }
    }
    NetWork W;
    if ((rc = net_work(h, W))) return rc;
    std::mt19937_64 gen(p->seed + 1);
    std::vector<int> order(nsrc);
    for (int k = 0; k < nsrc; ++k) order[k] = k;
    S.pairs = nsrc;
    for (int ep = 0; ep < p->epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), gen);
        double Lep = 0;
        for (int b0 = 0; b0 < nsrc; b0 += p->batch) {
            const int nb = std::min(p->batch, nsrc - b0);
            double Lb = 0;
            for (int q = 0; q < nb; ++q) {
                const int k = order[b0 + q];
                if ((rc = net_pair_grad(h, W, N->pb[k], N->px[k], N->pxn2[k], nb, sc, st))) return rc;
                CgScalars hs;
                CK(cudaMemcpyAsync(&hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                Lb += hs.last / N->pxn2[k] / nb;
            }
            CK(net_adam(h, p->lr, st));
            S.steps += 1;
            Lep += Lb * nb / nsrc;
        }
        if (ep == 0) S.loss_first = Lep;
        S.loss_last = Lep;
        if (S.n_history < 64) S.loss_history[S.n_history++] = Lep;
        S.epochs = ep + 1;
        if (p->verbose) std::fprintf(stderr, "[dwf] epoch %d loss %.6e\n", ep, Lep);
    }
    CK(cudaStreamSynchronize(st));
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    S.status = DWF_OK;
    if (stats) *stats = S;
    return DWF_OK;
}

int dwf_precond_adam_step(dwf_handle h, int layers, const double *grad, double lr, void *stream)
{
    if (!h || !grad) return dwf_set_error(DWF_EINVAL, "NULL argument");
    if (!h->net || h->net->L != layers) return dwf_set_error(DWF_EINVAL, "no preconditioner with that many layers");
    if (!(lr > 0)) return dwf_set_error(DWF_EINVAL, "lr must be positive");
    NetState *N = h->net;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nall = N->nw * N->L;
    CK(cudaMemcpyAsync(N->g, grad, nall * sizeof(double2), cudaMemcpyHostToDevice, st));
    CK(net_adam(h, lr, st));
    CK(cudaStreamSynchronize(st));
    return DWF_OK;
}

int dwf_precond_save(dwf_handle h, const char *path)
{
    if (!h || !path) return dwf_set_error(DWF_EINVAL, "NULL argument");
    if (!h->net) return dwf_set_error(DWF_EINVAL, "no preconditioner to save");
    NetState *N = h->net;
    const size_t nall = N->nw * N->L;
    std::vector<double2> buf(3 * nall);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(buf.data(), N->Wm, nall * sizeof(double2), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(buf.data() + nall, N->m, nall * sizeof(double2), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(buf.data() + 2 * nall, N->v, nall * sizeof(double2), cudaMemcpyDeviceToHost));
    NetFileHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, kNetMagic, 8);
    hd.version = 1;
    hd.layers = N->L;
    hd.channels = N->C;
    hd.adam_t = N->t;
    hd.nall = (int64_t)nall;
    FILE *f = std::fopen(path, "wb");
    if (!f) return dwf_set_error(DWF_EINVAL, std::string("cannot open ") + path + " for writing");
    const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
                    std::fwrite(buf.data(), sizeof(double2), buf.size(), f) == buf.size();
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) return dwf_set_error(DWF_EINVAL, std::string("short write to ") + path);
    return DWF_OK;
}

int dwf_precond_load(dwf_handle h, const char *path)
{
    if (!h || !path) return dwf_set_error(DWF_EINVAL, "NULL argument");
    FILE *f = std::fopen(path, "rb");
    if (!f) return dwf_set_error(DWF_EINVAL, std::string("cannot open ") + path);
    NetFileHeader hd;
    if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, kNetMagic, 8) != 0) {
        std::fclose(f);
        return dwf_set_error(DWF_EINVAL, std::string(path) + " is not a preconditioner file");
    }
    if (hd.version != 1) {
        std::fclose(f);
        return dwf_set_error(DWF_EINVAL, "unsupported preconditioner file version " + std::to_string(hd.version));
    }
    if (hd.channels != h->Ls || hd.layers < 1 || hd.layers > 8 ||
        hd.nall != (int64_t)NHOP * 2 * hd.channels * hd.channels * hd.layers) {
        std::fclose(f);
        return dwf_set_error(DWF_EINVAL, "preconditioner file for " + std::to_string(hd.layers) + " layers and " +
                                             std::to_string(hd.channels) + " channels does not fit this handle (Ls " +
                                             std::to_string(h->Ls) + ")");
    }
    std::vector<double2> buf(3 * (size_t)hd.nall);
    const bool ok = std::fread(buf.data(), sizeof(double2), buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return dwf_set_error(DWF_EINVAL, std::string(path) + " is truncated");
    int rc = net_alloc(h, hd.layers);
    if (rc) return rc;
    NetState *N = h->net;
    const size_t nall = (size_t)hd.nall;
    CK(cudaMemcpy(N->Wm, buf.data(), nall * sizeof(double2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(N->m, buf.data() + nall, nall * sizeof(double2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(N->v, buf.data() + 2 * nall, nall * sizeof(double2), cudaMemcpyHostToDevice));
    CK(cudaMemset(N->g, 0, nall * sizeof(double2)));
    net_round_kernel<<<(int)((nall + 255) / 256), 256>>>(N->Wm, N->Wc, (int)nall);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    h->launches += 1;
    N->t = hd.adam_t;
    return DWF_OK;
}

}  // extern "C"
