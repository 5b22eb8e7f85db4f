// The even-odd hopping stencil of the 5D domain-wall operator with its fused
// fifth-direction mixing and epilogue (one launch = one of the two hops of
// every application of the even-odd matrix, eq. even-odd_linear_equation).
//
// H psi(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
// is the hopping sum of eq. (Wilson_matrix) (D_W = (4 - M0) - H/2); it is the
// same for every fifth-direction slice s.  A CTA handles SB sites x all Ls
// slices; each thread owns NS slices of one site (s = x + n Ls/NS), so every
// link it loads serves NS slices.  The adjoint hop is gamma5 H gamma5
// (projector signs flipped).
//
// Chiral basis: gamma_mu = [[0, e_mu], [e_mu^dag, 0]], e_k = -i sigma_k,
// e_4 = 1, so (1 - sig gamma_mu) psi = [h ; -sig e_mu^dag h] with the half
// spinor h = psi_u - sig e_mu psi_l: only h is multiplied by the link.  h is
// held as spin pairs Hx[a] = (h0.re, h1.re), Hy[a] = (h0.im, h1.im), so the
// SU(3) product is 4 packed FMAs per (a, b) for both spins at once.
//
// Variants: 0 (direct) every thread reads its 8 neighbour spinors from
// global memory; 3 the same, persistent over consecutive tiles; 4 the same
// with each CTA's sites taken as a 4D block (neighbour reuse in L1); 5 (FP16)
// variant 0 with the spin projection in FP16 arithmetic.
// After the hop each thread writes h(site, s) to the CTA's shared tile and
// forms (Post h)(site, s) = sum_t Post[s][t] h(site, t) per chirality; the
// epilogue adds a mixed second input, forms a residual, updates a solution
// accumulator, applies a final mixing and reduces |o|^2 deterministically.
#pragma once

#include <cstdint>

#include "stencil.cuh"
#include "tcgen05.cuh"

namespace dwf {
namespace {

// one (site, s) of a neighbour site copied to shared memory: the Ls x G block
// of 16-byte vectors in the global layout, followed (FP16) by its scales
template <int P, typename T2>
__device__ __forceinline__ void ld_pairs_smem(const unsigned char *slot, int s, int Ls, T2 *v)
{
    typedef typename PairReal<T2>::R R;
    if constexpr (P == DWF_F64) {
        const double2 *p = reinterpret_cast<const double2 *>(slot) + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 q = p[k * Ls];
            v[k] = p_make((R)q.x, (R)q.y);
        }
    } else if constexpr (P == DWF_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(slot) + s;
#pragma unroll
        for (int g = 0; g < 6; ++g) {
            const float4 q = p[g * Ls];
            v[2 * g] = p_make((R)q.x, (R)q.y);
            v[2 * g + 1] = p_make((R)q.z, (R)q.w);
        }
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(slot) + s;
        const float sc = reinterpret_cast<const float *>(slot + (size_t)Ls * 48)[s];
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            const uint4 q = p[g * Ls];
            const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float2 f2 = __half22float2(*reinterpret_cast<const __half2 *>(&w[k]));
                v[4 * g + k] = p_make((R)(f2.x * sc), (R)(f2.y * sc));
            }
        }
    }
}

template <typename T2>
__device__ __forceinline__ void put_tile(T2 *tile, int s, const T2 *v)
{
    T2 *dst = tile + s * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[k] = v[k];
}

// ------------------------------------------------------------ the epilogue
struct CtaBarrier {
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// Where the CTA's tile lives and which threads share the structured mixing.
template <typename T2>
struct TileCtx {
    T2 *tile0;     // tile of the CTA's first site
    int tstride;   // pairs between consecutive sites
    int nsites;    // sites in the tile
    int tid, nthr; // this thread among the threads that share the work
};

// o[n] += (mixing of this thread's rows of the tile).  MIX 0, dense: Ls x Ls
// matrix M from shared memory, per thread.  MIX 1, structured: the CTA first
// transforms the whole tile in place along its chains; MIX 2 / 3, tensor
// cores: the CTA's full warps transform the tile in place with TF32 MMAs
// (3 / 2 products, see mma_mix_tile); then every thread reads its rows back.
// The tile must hold the input and be visible to all threads on entry.
template <int MIX, int NS, typename T2, typename R, typename Bar>
__device__ __forceinline__ void mix_into(const void *prog, const R *M, const TileCtx<T2> &tc, T2 *mytile,
                                         int x, int LsN, int Ls, bool active, T2 (*o)[12], const Bar &bar,
                                         int band = 0)
{
    if constexpr (MIX >= 1) {
        if constexpr (MIX == 1)
            chain_mix<R>(reinterpret_cast<const MixProg<R> *>(prog), tc.tile0, tc.tstride, tc.nsites, Ls, tc.tid,
                         tc.nthr);
        else
            mma_mix_tile<MIX == 2 ? 2 : 1>(reinterpret_cast<const float *>(M), reinterpret_cast<float *>(tc.tile0),
                                           tc.tstride, tc.nsites, Ls, Ls / LsN, tc.tid >> 5, tc.nthr >> 5);
        bar.sync();
        if (active) {
#pragma unroll
            for (int n = 0; n < NS; ++n) {
                T2 h[12];
                ld_tile_row(mytile + (x + n * LsN) * 12, h);
#pragma unroll
                for (int k = 0; k < 12; ++k) o[n][k] = p_add(o[n][k], h[k]);
            }
        }
    } else if (active) {
        if (band)
            mix_pairs_band<NS>(M, mytile, x, Ls, o);
        else
            mix_pairs<NS>(M, mytile, x, Ls, o);
    }
}

// acc: hop result of this thread's NS slices.  Every thread taking part in
// `bar` must call it.  Returns this thread's contribution to |o|^2.
template <int P, int NS, int MIX = 0, typename T2, typename R, typename Bar>
__device__ __forceinline__ R hop_epilogue_core(const HopArgs &a, T2 (*acc)[12], const TileCtx<T2> &tc,
                                                    T2 *mytile, const R *mtx, int site, int x, int LsN, bool active,
                                                    const Bar &bar)
{
    const int Ls = a.Ls;
    const int msz = 2 * Ls * Ls;
    // tensor-core mixing: FP16 fields take the two-product form (its error is that of the FP16 storage)
    constexpr int MX = (MIX == 2 && P == DWF_F16) ? 3 : MIX;
    if (active) {
#pragma unroll
        for (int n = 0; n < NS; ++n) put_tile(mytile, x + n * LsN, acc[n]);
    }
    bar.sync();

    T2 o[NS][12];
#pragma unroll
    for (int n = 0; n < NS; ++n)
#pragma unroll
        for (int k = 0; k < 12; ++k) o[n][k] = p_splat((R)0);
    mix_into<MX, NS>(a.post_prog, mtx, tc, mytile, x, LsN, Ls, active, o, bar, a.post_band);

    if (a.ymode == 1) {
        if (active) {
#pragma unroll
            for (int n = 0; n < NS; ++n) {
                T2 y[12];
                ld_pairs<P, false>(a.y, (size_t)site, x + n * LsN, Ls, y);
#pragma unroll
                for (int k = 0; k < 12; ++k) o[n][k] = p_add(o[n][k], y[k]);
            }
        }
    } else if (a.ymode == 2) {
        bar.sync();
        if (active) {
#pragma unroll
            for (int n = 0; n < NS; ++n) {
                T2 y[12];
                ld_pairs<P, false>(a.y, (size_t)site, x + n * LsN, Ls, y);
                put_tile(mytile, x + n * LsN, y);
            }
        }
        bar.sync();
        mix_into<MX, NS>(a.y_prog, mtx + msz, tc, mytile, x, LsN, Ls, active, o, bar, a.y_band);
    }

    if (a.rin.v && active) {
        const R al = (R)(*a.ralpha);
        const T2 nal = p_splat(-al);
#pragma unroll
        for (int n = 0; n < NS; ++n) {
            T2 r[12];
            ld_pairs<P, false>(a.rin, (size_t)site, x + n * LsN, Ls, r);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[n][k] = p_fma(nal, o[n][k], r[k]);
        }
        if (a.xacc) {
            constexpr int XP = (P == DWF_F64) ? DWF_F64 : DWF_F32;
            FieldRef xf;
            xf.v = a.xacc;
            const T2 xa = p_splat((R)(*a.xalpha));
#pragma unroll
            for (int n = 0; n < NS; ++n) {
                T2 xv[12], dx[12];
                ld_pairs<XP, false>(xf, (size_t)site, x + n * LsN, Ls, xv);
                ld_pairs<P, false>(a.xdir, (size_t)site, x + n * LsN, Ls, dx);
#pragma unroll
                for (int k = 0; k < 12; ++k) xv[k] = p_fma(xa, dx[k], xv[k]);
                st_pairs<XP>(xf, (size_t)site, x + n * LsN, Ls, xv);
            }
        }
    }

    // |o|^2 of this thread in the arithmetic precision (FP32 for FP32 and FP16
    // fields); the grid reduction adds the per-warp sums in FP64
    R nrm = 0;
    if (active && a.red.op != RED_NONE) {
        T2 s2 = p_splat((R)0);
#pragma unroll
        for (int n = 0; n < NS; ++n)
#pragma unroll
            for (int k = 0; k < 12; ++k) s2 = p_fma(o[n][k], o[n][k], s2);
        nrm = s2.x + s2.y;
    }

    if (a.zmat) {
        bar.sync();
        if (active) {
#pragma unroll
            for (int n = 0; n < NS; ++n) put_tile(mytile, x + n * LsN, o[n]);
        }
        bar.sync();
        T2 z[NS][12];
#pragma unroll
        for (int n = 0; n < NS; ++n)
#pragma unroll
            for (int k = 0; k < 12; ++k) z[n][k] = p_splat((R)0);
        mix_into<MX, NS>(a.z_prog, mtx + 2 * msz, tc, mytile, x, LsN, Ls, active, z, bar, a.z_band);
        if (active) {
#pragma unroll
            for (int n = 0; n < NS; ++n) st_pairs<P>(a.out, (size_t)site, x + n * LsN, Ls, z[n]);
        }
    } else if (active) {
#pragma unroll
        for (int n = 0; n < NS; ++n) st_pairs<P>(a.out, (size_t)site, x + n * LsN, Ls, o[n]);
    }

    return nrm;
}

// Epilogue of the kernels whose whole CTA forms one tile (blockDim = (Ls/NS, SB)).
template <typename T2>
__device__ __forceinline__ TileCtx<T2> cta_tile(T2 *tile0, int Ls)
{
    TileCtx<T2> tc;
    tc.tile0 = tile0;
    tc.tstride = Ls * 12 + 2;
    tc.nsites = blockDim.y;
    tc.tid = threadIdx.y * blockDim.x + threadIdx.x;
    tc.nthr = blockDim.x * blockDim.y;
    return tc;
}

template <int P, int NS, int MIX = 0, typename T2, typename R>
__device__ __forceinline__ void hop_epilogue(const HopArgs &a, T2 (*acc)[12], T2 *tile0, int j, const R *mtx,
                                             int site, int x, int LsN, bool active)
{
    const TileCtx<T2> tc = cta_tile(tile0, a.Ls);
    const auto nrm = hop_epilogue_core<P, NS, MIX>(a, acc, tc, tile0 + j * tc.tstride, mtx, site, x, LsN, active,
                                                CtaBarrier());
    if (a.red.op != RED_NONE) grid_reduce(nrm, a.red);
}

// matrices arrive as [chi][t][s]; store them as [chi][t][x*NS + n] with s = x + n*LsN
template <int NS, typename R>
__device__ __forceinline__ void load_matrices(const HopArgs &a, R *mtx)
{
    const int Ls = a.Ls, LsN = Ls / NS, msz = 2 * Ls * Ls;
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int k = tid; k < msz; k += nt) {
        const int chi_t = k / Ls, s = k % Ls;
        const int dst = chi_t * Ls + (s % LsN) * NS + s / LsN;
        mtx[dst] = reinterpret_cast<const R *>(a.post)[k];
        if (a.ymode == 2) mtx[msz + dst] = reinterpret_cast<const R *>(a.ymat)[k];
        if (a.zmat) mtx[2 * msz + dst] = reinterpret_cast<const R *>(a.zmat)[k];
    }
}

// ------------------------------------------------------ variant 0: direct
template <int P, bool DAG, int D, int NS, typename T2>
__device__ __forceinline__ void hop_dir(T2 (*acc)[12], const FieldRef &in, int nb, int x, int LsN, int Ls,
                                        const typename Tr<P>::link_t *U)
{
    constexpr int MU = D & 3;
    constexpr int SIG = (D < 4 ? 1 : -1) * (DAG ? -1 : 1);
    T2 u[9];
    load_link<P, true>(U + D * 18, u);
#pragma unroll
    for (int n = 0; n < NS; ++n) {
        T2 v[12];
        ld_pairs<P, true>(in, (size_t)nb, x + n * LsN, Ls, v);
        hop_one<MU, SIG>(acc[n], u, v);
    }
}

// FP16 fields (variant 5): the spin projection runs in FP16 arithmetic on the
// stored half2 pairs (one rounding, at the level of the FP16 storage), only the
// six half-spinor pairs are converted to FP32, and the SU(3) product runs in
// FP32 for all NS slices of the thread at once, so that every link splat
// serves NS slices; the product is scaled by the neighbour's (site, s) scale
// and reconstructed into the FP32 accumulator.
template <bool DAG, int D, int NS>
__device__ __forceinline__ void hop_dir_h2(float2 (*acc)[12], const FieldRef &in, int nb, int x, int LsN, int Ls,
                                           const __half *U)
{
    constexpr int MU = D & 3;
    constexpr int SIG = (D < 4 ? 1 : -1) * (DAG ? -1 : 1);
    const __half2 *Uh = reinterpret_cast<const __half2 *>(U + D * 18);
    float2 u[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = __half22float2(__ldg(Uh + k));
    const uint4 *base = reinterpret_cast<const uint4 *>(in.v) + ((size_t)nb * 3) * Ls;
    const float *sbase = in.scale + (size_t)nb * ((Ls + 3) & ~3);
    float2 Hx[NS][3], Hy[NS][3];
    float sc[NS];
#pragma unroll
    for (int n = 0; n < NS; ++n) {
        const int s = x + n * LsN;
        __half2 v[12];
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            const uint4 q = __ldg(base + (size_t)g * Ls + s);
            v[4 * g] = *reinterpret_cast<const __half2 *>(&q.x);
            v[4 * g + 1] = *reinterpret_cast<const __half2 *>(&q.y);
            v[4 * g + 2] = *reinterpret_cast<const __half2 *>(&q.z);
            v[4 * g + 3] = *reinterpret_cast<const __half2 *>(&q.w);
        }
        sc[n] = __ldg(sbase + s);
        __half2 hx[3], hy[3];
        project_h2<MU, SIG>(v, hx, hy);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Hx[n][a] = __half22float2(hx[a]);
            Hy[n][a] = __half22float2(hy[a]);
        }
    }
    float2 Qx[NS][3], Qy[NS][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int n = 0; n < NS; ++n) Qx[n][a] = Qy[n][a] = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float2 ur = p_splat(u[a * 3 + b].x), ui = p_splat(u[a * 3 + b].y), nui = p_splat(-u[a * 3 + b].y);
#pragma unroll
            for (int n = 0; n < NS; ++n) {
                Qx[n][a] = p_fma(ur, Hx[n][b], Qx[n][a]);
                Qx[n][a] = p_fma(nui, Hy[n][b], Qx[n][a]);
                Qy[n][a] = p_fma(ur, Hy[n][b], Qy[n][a]);
                Qy[n][a] = p_fma(ui, Hx[n][b], Qy[n][a]);
            }
        }
    }
#pragma unroll
    for (int n = 0; n < NS; ++n) {
        const float2 scp = p_splat(sc[n]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Qx[n][a] = p_mul(Qx[n][a], scp);
            Qy[n][a] = p_mul(Qy[n][a], scp);
        }
        reconstruct<MU, SIG>(acc[n], Qx[n], Qy[n]);
    }
}

template <int P, bool DAG, int NS, bool H2>
__device__ __forceinline__ void gather8(typename Tr<P>::pair (*acc)[12], const HopArgs &a, const int *n8, int x,
                                        int LsN, int Ls, const typename Tr<P>::link_t *U)
{
    if constexpr (H2 && P == DWF_F16) {
        hop_dir_h2<DAG, 0, NS>(acc, a.in, n8[0], x, LsN, Ls, U);
        hop_dir_h2<DAG, 1, NS>(acc, a.in, n8[1], x, LsN, Ls, U);
        hop_dir_h2<DAG, 2, NS>(acc, a.in, n8[2], x, LsN, Ls, U);
        hop_dir_h2<DAG, 3, NS>(acc, a.in, n8[3], x, LsN, Ls, U);
        hop_dir_h2<DAG, 4, NS>(acc, a.in, n8[4], x, LsN, Ls, U);
        hop_dir_h2<DAG, 5, NS>(acc, a.in, n8[5], x, LsN, Ls, U);
        hop_dir_h2<DAG, 6, NS>(acc, a.in, n8[6], x, LsN, Ls, U);
        hop_dir_h2<DAG, 7, NS>(acc, a.in, n8[7], x, LsN, Ls, U);
    } else {
        hop_dir<P, DAG, 0, NS>(acc, a.in, n8[0], x, LsN, Ls, U);
        hop_dir<P, DAG, 1, NS>(acc, a.in, n8[1], x, LsN, Ls, U);
        hop_dir<P, DAG, 2, NS>(acc, a.in, n8[2], x, LsN, Ls, U);
        hop_dir<P, DAG, 3, NS>(acc, a.in, n8[3], x, LsN, Ls, U);
        hop_dir<P, DAG, 4, NS>(acc, a.in, n8[4], x, LsN, Ls, U);
        hop_dir<P, DAG, 5, NS>(acc, a.in, n8[5], x, LsN, Ls, U);
        hop_dir<P, DAG, 6, NS>(acc, a.in, n8[6], x, LsN, Ls, U);
        hop_dir<P, DAG, 7, NS>(acc, a.in, n8[7], x, LsN, Ls, U);
    }
}

// Sweep order: sweep position p -> site index.  With a.zblock = Bz (0 < Bz <
// Lz) the lattice is swept in columns of Bz z-planes, each column t-slice by
// t-slice: site = r + A (z + Lz t), A = (Lx/2) Ly sites of one parity per
// z-plane, z = column Bz + zl, p = column (Lt Bz A) + t (Bz A) + zl A + r.  A
// site's -t and +t neighbours are then read 2 Bz A positions apart instead of
// 2 Lz A, which keeps the field between the two reads within L2 once a whole
// t-slice no longer fits; only the z-planes bordering a column are read twice
// from DRAM.  Consecutive positions stay consecutive sites inside a run of Bz A.
__device__ __forceinline__ int sweep_site(const HopArgs &a, int p)
{
    const int Bz = a.zblock;
    if (Bz <= 0) return p;
    const int A = a.ext[0] * a.ext[1], plane = Bz * A, col = plane * a.ext[3];
    const int c = p / col, q = p - c * col, t = q / plane;
    return q - t * plane + A * (c * Bz + a.ext[2] * t);
}

// One tile of SB sites: blockDim = (Ls/NS, SB), site = u SB + threadIdx.y
// (in the sweep order above when a tile never straddles a run of Bz A sites).
// The norm reduction runs over the nb_red tiles that share a.red.
template <int P, bool DAG, int NS, int MIX, bool H2 = false>
__device__ __forceinline__ void hop_direct_tile(const HopArgs &a, int u, unsigned nb_red)
{
    typedef typename Tr<P>::real R;
    typedef typename Tr<P>::pair T2;
    typedef typename Tr<P>::link_t link_t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls;
    const int LsN = Ls / NS;
    const int x = threadIdx.x;
    const int j = threadIdx.y;
    const int SB = blockDim.y;
    const bool active = u * SB + j < a.Vh;
    const int site = (a.zblock > 0 && (a.zblock * a.ext[0] * a.ext[1]) % SB == 0 ? sweep_site(a, u * SB) : u * SB) + j;
    const int tstride = Ls * 12 + 2;
    T2 *tile = reinterpret_cast<T2 *>(smem_raw);
    R *mtx = reinterpret_cast<R *>(tile + SB * tstride);
    load_matrices<NS>(a, mtx);

    T2 acc[NS][12];
#pragma unroll
    for (int n = 0; n < NS; ++n)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[n][k] = p_splat((R)0);
    if (active) {
        const int *nb = a.nbr + (size_t)site * 8;
        const link_t *U = reinterpret_cast<const link_t *>(a.gauge) + (size_t)site * 8 * 18;
        int n8[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) n8[d] = __ldg(nb + d);
        gather8<P, DAG, NS, H2>(acc, a, n8, x, LsN, Ls, U);
    }
    const TileCtx<T2> tc = cta_tile(tile, Ls);
    const auto nrm = hop_epilogue_core<P, NS, MIX>(a, acc, tc, tile + j * tc.tstride, mtx, site, x, LsN, active,
                                                     CtaBarrier());
    if (a.red.op != RED_NONE) grid_reduce(nrm, a.red, u, nb_red);
}

template <int P, bool DAG, int NS, int MIX, bool H2 = false>
__global__ void __launch_bounds__(256) hop_kernel(const HopArgs a)
{
    hop_direct_tile<P, DAG, NS, MIX, H2>(a, blockIdx.x, gridDim.x);
}

// With one slice per thread the FP16 variant-5 and the FP32 direct kernels run
// faster with more resident warps (the gathers are latency bound): capped at
// 64 registers (FP16: 8 CTAs of 128 threads per SM) the hop at 16^3x32, Ls 16
// went from 96.2 us to 85.8 us, capped at 85 (FP32: 6 CTAs) from 117.8 us to
// 106.3 us.
template <int P, bool DAG, int MIX, bool H2>
__global__ void __launch_bounds__(256, P == DWF_F16 ? 4 : 3) hop_kernel_occ(const HopArgs a)
{
    hop_direct_tile<P, DAG, 1, MIX, H2>(a, blockIdx.x, gridDim.x);
}

// Batched form: one launch over nsys systems that share Ls and the CTA shape
// (each with its own fields, matrices, scalars and reduction buffers).  CTA b
// works on tile b / nsys of system b % nsys, so that consecutive CTAs read the
// same sites' links and neighbour indices, which then come from L2 for all
// systems but the first.  A system whose skip flag is set is left untouched.
template <int P, bool DAG, int NS, int MIX, bool H2>
__device__ __forceinline__ void hop_batch_body(const HopArgs *__restrict__ tab, int nsys)
{
    __shared__ __align__(16) unsigned char abuf[sizeof(HopArgs)];
    const int sys = blockIdx.x % nsys, u = blockIdx.x / nsys;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    const unsigned *src = reinterpret_cast<const unsigned *>(tab + sys);
    for (int k = tid; k < (int)(sizeof(HopArgs) / 4); k += nt) reinterpret_cast<unsigned *>(abuf)[k] = src[k];
    __syncthreads();
    const HopArgs &a = *reinterpret_cast<const HopArgs *>(abuf);
    if (a.skip && *a.skip) return;
    hop_direct_tile<P, DAG, NS, MIX, H2>(a, u, (a.Vh + blockDim.y - 1) / blockDim.y);
}

template <int P, bool DAG, int NS, int MIX, bool H2 = false>
__global__ void __launch_bounds__(256) hop_batch_kernel(const HopArgs *__restrict__ tab, int nsys)
{
    hop_batch_body<P, DAG, NS, MIX, H2>(tab, nsys);
}

// the occupancy-capped form of the batched hop (see hop_kernel_occ)
template <int P, bool DAG, int MIX, bool H2>
__global__ void __launch_bounds__(256, P == DWF_F16 ? 4 : 3) hop_batch_kernel_occ(const HopArgs *__restrict__ tab,
                                                                                 int nsys)
{
    hop_batch_body<P, DAG, 1, MIX, H2>(tab, nsys);
}

// ------------------------------------------------- variant 4: blocked tiles
// The direct kernel with each CTA's SB sites taken as a 4D block
// tb[0] x tb[1] x tb[2] x tb[3] of the half lattice (coordinates xh = x/2, y,
// z, t; the even-odd index is lexicographic in them), so that the neighbour
// sites the CTA reads overlap and are served from L1.  The block extents
// divide the half-lattice extents.
struct Tile4 {
    int tb[4];
};

template <int P, bool DAG, int NS>
__global__ void __launch_bounds__(256) hop_block_kernel(const HopArgs a, Tile4 T)
{
    typedef typename Tr<P>::real R;
    typedef typename Tr<P>::pair T2;
    typedef typename Tr<P>::link_t link_t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls;
    const int LsN = Ls / NS;
    const int x = threadIdx.x;
    const int j = threadIdx.y;
    const int SB = blockDim.y;
    // block coordinates (lexicographic over the tiled half lattice) and local offsets
    int b = blockIdx.x, l = j, c[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int nb = a.ext[d] / T.tb[d];
        const int bd = b % nb, ld = l % T.tb[d];
        b /= nb;
        l /= T.tb[d];
        c[d] = bd * T.tb[d] + ld;
    }
    const int site = c[0] + a.ext[0] * (c[1] + a.ext[1] * (c[2] + a.ext[2] * c[3]));
    const bool active = true;
    const int tstride = Ls * 12 + 2;
    T2 *tile = reinterpret_cast<T2 *>(smem_raw);
    R *mtx = reinterpret_cast<R *>(tile + SB * tstride);
    load_matrices<NS>(a, mtx);

    T2 acc[NS][12];
#pragma unroll
    for (int n = 0; n < NS; ++n)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[n][k] = p_splat((R)0);
    {
        const int *nb = a.nbr + (size_t)site * 8;
        const link_t *U = reinterpret_cast<const link_t *>(a.gauge) + (size_t)site * 8 * 18;
        int n8[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) n8[d] = __ldg(nb + d);
        hop_dir<P, DAG, 0, NS>(acc, a.in, n8[0], x, LsN, Ls, U);
        hop_dir<P, DAG, 1, NS>(acc, a.in, n8[1], x, LsN, Ls, U);
        hop_dir<P, DAG, 2, NS>(acc, a.in, n8[2], x, LsN, Ls, U);
        hop_dir<P, DAG, 3, NS>(acc, a.in, n8[3], x, LsN, Ls, U);
        hop_dir<P, DAG, 4, NS>(acc, a.in, n8[4], x, LsN, Ls, U);
        hop_dir<P, DAG, 5, NS>(acc, a.in, n8[5], x, LsN, Ls, U);
        hop_dir<P, DAG, 6, NS>(acc, a.in, n8[6], x, LsN, Ls, U);
        hop_dir<P, DAG, 7, NS>(acc, a.in, n8[7], x, LsN, Ls, U);
    }
    hop_epilogue<P, NS>(a, acc, tile, j, mtx, site, x, LsN, active);
}

// ------------------------------------------ variant 3: persistent direct sweep
// The direct kernel, persistent: CTA b handles the consecutive tiles
// [b*tpc, (b+1)*tpc).  Consecutive tiles are consecutive x-rows, so an input
// row fetched as the +y neighbour of one tile is fetched again (from L1) as
// the x neighbour and the -y neighbour of the next two tiles.
template <int P, bool DAG, int NS>
__global__ void __launch_bounds__(256) hop_sweep_kernel(const HopArgs a, int tpc)
{
    typedef typename Tr<P>::real R;
    typedef typename Tr<P>::pair T2;
    typedef typename Tr<P>::link_t link_t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls;
    const int LsN = Ls / NS;
    const int x = threadIdx.x;
    const int j = threadIdx.y;
    const int SB = blockDim.y;
    const int tstride = Ls * 12 + 2;
    T2 *tile = reinterpret_cast<T2 *>(smem_raw);
    R *mtx = reinterpret_cast<R *>(tile + SB * tstride);
    load_matrices<NS>(a, mtx);
    const int ntiles = (a.Vh + SB - 1) / SB;
    const int u0 = blockIdx.x * tpc;
    const int u1 = min(u0 + tpc, ntiles);
    double nrm = 0;
    for (int u = u0; u < u1; ++u) {
        const int site = u * SB + j;
        const bool active = site < a.Vh;
        T2 acc[NS][12];
#pragma unroll
        for (int n = 0; n < NS; ++n)
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[n][k] = p_splat((R)0);
        if (active) {
            const int *nb = a.nbr + (size_t)site * 8;
            const link_t *U = reinterpret_cast<const link_t *>(a.gauge) + (size_t)site * 8 * 18;
            int n8[8];
#pragma unroll
            for (int d = 0; d < 8; ++d) n8[d] = __ldg(nb + d);
            hop_dir<P, DAG, 0, NS>(acc, a.in, n8[0], x, LsN, Ls, U);
            hop_dir<P, DAG, 1, NS>(acc, a.in, n8[1], x, LsN, Ls, U);
            hop_dir<P, DAG, 2, NS>(acc, a.in, n8[2], x, LsN, Ls, U);
            hop_dir<P, DAG, 3, NS>(acc, a.in, n8[3], x, LsN, Ls, U);
            hop_dir<P, DAG, 4, NS>(acc, a.in, n8[4], x, LsN, Ls, U);
            hop_dir<P, DAG, 5, NS>(acc, a.in, n8[5], x, LsN, Ls, U);
            hop_dir<P, DAG, 6, NS>(acc, a.in, n8[6], x, LsN, Ls, U);
            hop_dir<P, DAG, 7, NS>(acc, a.in, n8[7], x, LsN, Ls, U);
        }
        __syncthreads();   // the previous tile's epilogue is done with `tile`
        nrm += hop_epilogue_core<P, NS>(a, acc, cta_tile(tile, Ls), tile + j * tstride, mtx, site, x, LsN, active,
                                        CtaBarrier());
    }
    if (a.red.op != RED_NONE) grid_reduce(nrm, a.red);
}

// 16-byte asynchronous copies global -> shared (per-thread commit groups)
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// --------------------------------------------- variant 7: lean on the L1 path
// The direct kernel, rebuilt around the L1/shared-memory data path, which
// bounds the FP32 hop (every byte a thread loads from L1 or shared memory
// crosses it; ncu: L1/TEX 79 % busy at 28 % of DRAM bandwidth):
//  * persistent CTAs of SB sites x Ls slices (one slice per thread in the hop)
//    walking the tiles b, b + grid, ...;
//  * the tile's links (all 8 directions of its sites, contiguous in the link
//    table) are copied into shared memory with 16-byte asynchronous copies one
//    tile ahead; each thread reads its site's link as 16-byte vectors (5 loads
//    per direction instead of 9, each serving every slice of the site);
//  * the neighbour spinors are direct 16-byte loads (the cheapest way into
//    registers);
//  * the fifth-direction mixing runs on half of the CTA's threads, each
//    forming two outputs (slices s and s + Ls/2) from one pass over the site's
//    tile rows, so that every row read serves two outputs;
//  * the tile rows (28 floats), the site stride (one extra 16 bytes) and the
//    matrix rows are padded so that the 16-byte shared accesses of a warp hit
//    distinct banks.
// Dense mixing, Ls a multiple of 4; two CTAs of 256 threads per SM worth of
// registers.
constexpr int LEAN_ROW = 14;   // float2 per tile row (24 floats used)

template <int P>
struct LeanGeom {
    static constexpr int LINK_BYTES = 8 * 18 * (P == DWF_F16 ? 2 : 4);
};

// float2 between consecutive sites of the tile; floats between matrix rows
__host__ __device__ constexpr int lean_site_stride(int Ls) { return Ls * LEAN_ROW + 2; }
__host__ __device__ constexpr int lean_mat_row(int Ls) { return ((Ls / 2) & 1) ? Ls : Ls + 2; }

template <int P>
__host__ __device__ constexpr size_t lean_smem_bytes(int Ls, int SB)
{
    return (size_t)3 * 2 * Ls * lean_mat_row(Ls) * sizeof(float)           // matrices
           + (size_t)2 * SB * LeanGeom<P>::LINK_BYTES                    // links, double buffered
           + (size_t)SB * lean_site_stride(Ls) * sizeof(float2);          // mixing tile
}

// u[9] <- link D of a site from shared memory (FP32: 72 bytes at 72 D)
template <int P, int D>
__device__ __forceinline__ void lean_link(const unsigned char *lk, float2 *u)
{
    if constexpr (P == DWF_F32) {
        const unsigned char *b = lk + D * 72;
        if constexpr ((D & 1) == 0) {   // 16-byte aligned: 4 x 16 + 8 bytes
            const float4 *q = reinterpret_cast<const float4 *>(b);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = q[k];
                u[2 * k] = make_float2(v.x, v.y);
                u[2 * k + 1] = make_float2(v.z, v.w);
            }
            u[8] = *reinterpret_cast<const float2 *>(b + 64);
        } else {                        // 8 + 4 x 16 bytes
            u[0] = *reinterpret_cast<const float2 *>(b);
            const float4 *q = reinterpret_cast<const float4 *>(b + 8);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = q[k];
                u[2 * k + 1] = make_float2(v.x, v.y);
                u[2 * k + 2] = make_float2(v.z, v.w);
            }
        }
    } else {   // FP16: 36 bytes at 36 D, 4-byte aligned
        const __half2 *q = reinterpret_cast<const __half2 *>(lk + D * 36);
#pragma unroll
        for (int k = 0; k < 9; ++k) u[k] = __half22float2(q[k]);
    }
}

template <int P, bool DAG, int D>
__device__ __forceinline__ void lean_dir(float2 *acc, const FieldRef &in, int nb, int x, int Ls,
                                         const unsigned char *lk)
{
    constexpr int MU = D & 3;
    constexpr int SIG = (D < 4 ? 1 : -1) * (DAG ? -1 : 1);
    float2 u[9];
    lean_link<P, D>(lk, u);
    if constexpr (P == DWF_F32) {
        float2 v[12];
        ld_pairs<P, true>(in, (size_t)nb, x, Ls, v);
        hop_one<MU, SIG>(acc, u, v);
    } else {
        const uint4 *base = reinterpret_cast<const uint4 *>(in.v) + ((size_t)nb * 3) * Ls + x;
        __half2 v[12];
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            const uint4 q = __ldg(base + (size_t)g * Ls);
            v[4 * g] = *reinterpret_cast<const __half2 *>(&q.x);
            v[4 * g + 1] = *reinterpret_cast<const __half2 *>(&q.y);
            v[4 * g + 2] = *reinterpret_cast<const __half2 *>(&q.z);
            v[4 * g + 3] = *reinterpret_cast<const __half2 *>(&q.w);
        }
        const float sc = __ldg(in.scale + (size_t)nb * ((Ls + 3) & ~3) + x);
        __half2 hx[3], hy[3];
        project_h2<MU, SIG>(v, hx, hy);
        float2 Hx[3], Hy[3], Qx[3], Qy[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Hx[a] = __half22float2(hx[a]);
            Hy[a] = __half22float2(hy[a]);
        }
        su3_pairs(u, Hx, Hy, Qx, Qy);
        const float2 scp = make_float2(sc, sc);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Qx[a] = p_mul(Qx[a], scp);
            Qy[a] = p_mul(Qy[a], scp);
        }
        reconstruct<MU, SIG>(acc, Qx, Qy);
    }
}

__device__ __forceinline__ float2 *lean_row(float2 *tile, int j, int s, int Ls)
{
    return tile + (size_t)j * lean_site_stride(Ls) + (size_t)s * LEAN_ROW;
}

__device__ __forceinline__ void lean_put(float2 *row, const float2 *v)
{
    float4 *r4 = reinterpret_cast<float4 *>(row);
#pragma unroll
    for (int q = 0; q < 6; ++q) r4[q] = make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
}

// o[n] += sum_t M[chi][s_n][t] tile(j, t) for the two outputs s_0 = p, s_1 = p + Ls/2;
// M: [chi][s][t] with rows of lean_mat_row(Ls) floats.  Each 16-byte chunk of a
// tile row (one colour and re/im part: the P_+ pair and the P_- pair) is used
// as soon as it is read, for both outputs.
__device__ __forceinline__ void lean_mix2(const float *M, const float2 *tile, int j, int p, int Ls, float2 (*o)[12])
{
    const int MR = lean_mat_row(Ls), half = Ls / 2;
    const float *m0u = M + (size_t)p * MR, *m1u = M + (size_t)(p + half) * MR;
    const float *m0l = M + (size_t)(Ls + p) * MR, *m1l = M + (size_t)(Ls + p + half) * MR;
    const float4 *base = reinterpret_cast<const float4 *>(tile + (size_t)j * lean_site_stride(Ls));
#pragma unroll 1
    for (int t = 0; t < Ls; t += 2) {
        const float2 a0 = *reinterpret_cast<const float2 *>(m0u + t), a1 = *reinterpret_cast<const float2 *>(m1u + t);
        const float2 b0 = *reinterpret_cast<const float2 *>(m0l + t), b1 = *reinterpret_cast<const float2 *>(m1l + t);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float2 u0 = p_splat(k ? a0.y : a0.x), u1 = p_splat(k ? a1.y : a1.x);
            const float2 l0 = p_splat(k ? b0.y : b0.x), l1 = p_splat(k ? b1.y : b1.x);
            const float4 *row = base + (size_t)(t + k) * (LEAN_ROW / 2);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float4 v = row[q];
                const float2 hp = make_float2(v.x, v.y), hm = make_float2(v.z, v.w);
                o[0][2 * q] = p_fma(u0, hp, o[0][2 * q]);
                o[0][2 * q + 1] = p_fma(l0, hm, o[0][2 * q + 1]);
                o[1][2 * q] = p_fma(u1, hp, o[1][2 * q]);
                o[1][2 * q + 1] = p_fma(l1, hm, o[1][2 * q + 1]);
            }
        }
    }
}

// The same for a cyclic tridiagonal matrix: rows t = s - 1, s, s + 1 only.
__device__ __forceinline__ void lean_mix2_band(const float *M, const float2 *tile, int j, int p, int Ls,
                                               float2 (*o)[12])
{
    const int MR = lean_mat_row(Ls), half = Ls / 2;
    const float4 *base = reinterpret_cast<const float4 *>(tile + (size_t)j * lean_site_stride(Ls));
#pragma unroll
    for (int n = 0; n < 2; ++n) {
        const int sn = p + n * half;
#pragma unroll
        for (int dt = -1; dt <= 1; ++dt) {
            int t = sn + dt;
            t = t < 0 ? t + Ls : (t >= Ls ? t - Ls : t);
            const float2 cu = p_splat(M[(size_t)sn * MR + t]), cl = p_splat(M[(size_t)(Ls + sn) * MR + t]);
            const float4 *row = base + (size_t)t * (LEAN_ROW / 2);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float4 v = row[q];
                o[n][2 * q] = p_fma(cu, make_float2(v.x, v.y), o[n][2 * q]);
                o[n][2 * q + 1] = p_fma(cl, make_float2(v.z, v.w), o[n][2 * q + 1]);
            }
        }
    }
}

// The epilogue of hop_epilogue_core (dense mixing) on the lean tile.  Every
// thread puts its hop result; threads tid < SB Ls / 2 (site j = tid / (Ls/2),
// p = tid % (Ls/2)) then own the outputs s = p and p + Ls/2 of site j.
template <int P>
__device__ __forceinline__ float lean_epilogue(const HopArgs &a, const float2 *acc, float2 *tile, const float *mats,
                                               int j0, int s0, int site0, bool active0, int u, int SB)
{
    const int Ls = a.Ls, half = Ls / 2;
    const int msz = 2 * Ls * lean_mat_row(Ls);
    if (active0) lean_put(lean_row(tile, j0, s0, Ls), acc);
    __syncthreads();
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const bool mixer = tid < SB * half;
    const int j = mixer ? tid / half : 0, p = mixer ? tid - (tid / half) * half : 0;
    const int site = u * SB + j;
    const bool active = mixer && site < a.Vh;
    const int sl[2] = {p, p + half};
    // the solution accumulator update xacc += xalpha xdir (independent of the
    // hop) first, while no output is held in registers
    if (active && a.rin.v && a.xacc) {
        FieldRef xf;
        xf.v = a.xacc;
        const float2 xa = p_splat((float)(*a.xalpha));
#pragma unroll 1
        for (int n = 0; n < 2; ++n) {
            float2 xv[12], dx[12];
            ld_pairs<DWF_F32, false>(xf, (size_t)site, sl[n], Ls, xv);
            ld_pairs<P, false>(a.xdir, (size_t)site, sl[n], Ls, dx);
#pragma unroll
            for (int k = 0; k < 12; ++k) xv[k] = p_fma(xa, dx[k], xv[k]);
            st_pairs<DWF_F32>(xf, (size_t)site, sl[n], Ls, xv);
        }
    }
    float2 o[2][12];
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int k = 0; k < 12; ++k) o[n][k] = make_float2(0.f, 0.f);
    if (active) {
        if (a.post_band) lean_mix2_band(mats, tile, j, p, Ls, o);
        else lean_mix2(mats, tile, j, p, Ls, o);
    }
    if (a.ymode == 1) {
        if (active) {
#pragma unroll
            for (int n = 0; n < 2; ++n) {
                float2 y[12];
                ld_pairs<P, false>(a.y, (size_t)site, sl[n], Ls, y);
#pragma unroll
                for (int k = 0; k < 12; ++k) o[n][k] = p_add(o[n][k], y[k]);
            }
        }
    } else if (a.ymode == 2) {
        __syncthreads();
        if (active) {
#pragma unroll 1
            for (int n = 0; n < 2; ++n) {
                float2 y[12];
                ld_pairs<P, false>(a.y, (size_t)site, sl[n], Ls, y);
                lean_put(lean_row(tile, j, sl[n], Ls), y);
            }
        }
        __syncthreads();
        if (active) {
            if (a.y_band) lean_mix2_band(mats + msz, tile, j, p, Ls, o);
            else lean_mix2(mats + msz, tile, j, p, Ls, o);
        }
    }
    // the rest output by output (each output's registers are free when it is done)
    float nrm = 0.f;
#pragma unroll
    for (int n = 0; n < 2; ++n) {
        if (active && a.rin.v) {
            const float2 nal = p_splat((float)-(*a.ralpha));
            float2 r[12];
            ld_pairs<P, false>(a.rin, (size_t)site, sl[n], Ls, r);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[n][k] = p_fma(nal, o[n][k], r[k]);
        }
        if (active && a.red.op != RED_NONE) {
            float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 12; ++k) s2 = p_fma(o[n][k], o[n][k], s2);
            nrm += s2.x + s2.y;
        }
        if (active) {
            if (a.zmat) lean_put(lean_row(tile, j, sl[n], Ls), o[n]);
            else st_pairs<P>(a.out, (size_t)site, sl[n], Ls, o[n]);
        }
    }
    if (a.zmat) {
        __syncthreads();
        float2 z[2][12];
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
            for (int k = 0; k < 12; ++k) z[n][k] = make_float2(0.f, 0.f);
        if (active) {
            if (a.z_band) lean_mix2_band(mats + 2 * msz, tile, j, p, Ls, z);
            else lean_mix2(mats + 2 * msz, tile, j, p, Ls, z);
#pragma unroll
            for (int n = 0; n < 2; ++n) st_pairs<P>(a.out, (size_t)site, sl[n], Ls, z[n]);
        }
    }
    return nrm;
}

// the CTA's share of the link copies of tile u (sites u SB .. u SB + n - 1)
template <int P>
__device__ __forceinline__ void lean_issue_links(const void *gauge, int site0, int n, unsigned char *dst)
{
    constexpr int CH = LeanGeom<P>::LINK_BYTES / 16;
    const uint4 *src = reinterpret_cast<const uint4 *>(gauge) + (size_t)site0 * CH;
    const uint32_t d = smem_addr(dst);
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int c = tid; c < n * CH; c += nt) cp_async16(d + (uint32_t)c * 16, src + c);
    cp_async_commit();
}

// blockDim = (Ls, SB); grid: persistent, CTA b takes tiles b, b + gridDim.x, ...
template <int P, bool DAG, int MINB>
__global__ void __launch_bounds__(256, MINB) hop_lean_kernel(const HopArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls, SB = blockDim.y;
    const int s = threadIdx.x, j = threadIdx.y;
    const int nt = blockDim.x * blockDim.y, tid = j * Ls + s;
    const int MR = lean_mat_row(Ls), msz = 2 * Ls * MR;
    float *mats = reinterpret_cast<float *>(smem_raw);
    unsigned char *links = smem_raw + (size_t)3 * msz * sizeof(float);
    float2 *tile = reinterpret_cast<float2 *>(links + (size_t)2 * SB * LeanGeom<P>::LINK_BYTES);
    // matrices: [chi][t][s] in, row-major [chi][s][t] (rows of MR floats) in shared memory
    {
        const float *src[3] = {reinterpret_cast<const float *>(a.post),
                               a.ymode == 2 ? reinterpret_cast<const float *>(a.ymat) : nullptr,
                               reinterpret_cast<const float *>(a.zmat)};
        for (int m = 0; m < 3; ++m) {
            if (!src[m]) continue;
            for (int k = tid; k < 2 * Ls * Ls; k += nt) {
                const int chi = k / (Ls * Ls), r = k - chi * Ls * Ls, t = r / Ls, ss = r - t * Ls;
                mats[m * msz + (chi * Ls + ss) * MR + t] = src[m][k];
            }
        }
    }
    const int ntiles = (a.Vh + SB - 1) / SB;
    int u = blockIdx.x;
    if (u < ntiles) lean_issue_links<P>(a.gauge, u * SB, min(SB, a.Vh - u * SB), links);
    float nrm = 0.f;
    for (int k = 0; u < ntiles; ++k, u += gridDim.x) {
        const int site = u * SB + j;
        const bool active = site < a.Vh;
        int n8[8];
        if (active) {
            const int4 *p = reinterpret_cast<const int4 *>(a.nbr + (size_t)site * 8);
            const int4 q0 = __ldg(p), q1 = __ldg(p + 1);
            n8[0] = q0.x; n8[1] = q0.y; n8[2] = q0.z; n8[3] = q0.w;
            n8[4] = q1.x; n8[5] = q1.y; n8[6] = q1.z; n8[7] = q1.w;
        }
        cp_async_wait<0>();
        __syncthreads();   // this tile's links are in; the previous tile's epilogue is done
        const int un = u + gridDim.x;
        if (un < ntiles)   // the next tile's links, into the other buffer
            lean_issue_links<P>(a.gauge, un * SB, min(SB, a.Vh - un * SB),
                                links + (size_t)((k + 1) & 1) * SB * LeanGeom<P>::LINK_BYTES);
        float2 acc[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) acc[q] = make_float2(0.f, 0.f);
        if (active) {
            const unsigned char *lk = links + ((size_t)(k & 1) * SB + j) * LeanGeom<P>::LINK_BYTES;
            lean_dir<P, DAG, 0>(acc, a.in, n8[0], s, Ls, lk);
            lean_dir<P, DAG, 1>(acc, a.in, n8[1], s, Ls, lk);
            lean_dir<P, DAG, 2>(acc, a.in, n8[2], s, Ls, lk);
            lean_dir<P, DAG, 3>(acc, a.in, n8[3], s, Ls, lk);
            lean_dir<P, DAG, 4>(acc, a.in, n8[4], s, Ls, lk);
            lean_dir<P, DAG, 5>(acc, a.in, n8[5], s, Ls, lk);
            lean_dir<P, DAG, 6>(acc, a.in, n8[6], s, Ls, lk);
            lean_dir<P, DAG, 7>(acc, a.in, n8[7], s, Ls, lk);
        }
        nrm += lean_epilogue<P>(a, acc, tile, mats, j, s, site, active, u, SB);
    }
    cp_async_wait<0>();
    if (a.red.op != RED_NONE) grid_reduce(nrm, a.red);
}

// ------------------------------------------ variant 9: warp-autonomous hop
// Every warp works alone on its own tiles of 32 / Ls sites (Ls dividing 32),
// persistent over its CTA's contiguous range of tiles, with no CTA barrier
// after the matrices are loaded: the warp's links (its sites' 8 directions)
// are copied into its own shared-memory buffer with 16-byte asynchronous
// copies one tile ahead (warp barrier only) and read as 16-byte vectors; the
// neighbour spinors are direct 16-byte loads; the mixing tile is the warp's
// own (rows of 28 floats, sites 16 bytes apart beyond that, so 16-byte
// accesses hit distinct banks) and the matrix rows are padded the same way,
// so a thread reads four coefficients of its row at once.  Dense mixing
// (cyclic tridiagonal matrices read three rows).
template <int P>
__host__ __device__ constexpr size_t wa_warp_bytes(int Ls)
{
    return (size_t)2 * (32 / Ls) * LeanGeom<P>::LINK_BYTES + (size_t)(32 / Ls) * (Ls * 14 + 12) * sizeof(float2);
}
__host__ __device__ constexpr int wa_mat_row(int Ls) { return ((Ls / 4) & 1) ? Ls : Ls + 4; }
// the CTA's front area: the three dense matrices, then the three structured
// programs (at most 2048 bytes, checked where they are defined)
__host__ __device__ constexpr size_t wa_front_bytes(int Ls)
{
    return (size_t)3 * 2 * Ls * wa_mat_row(Ls) * sizeof(float) + 2048;
}
template <int P>
__host__ __device__ constexpr size_t wa_cta_bytes(int Ls, int nwarps)
{
    return wa_front_bytes(Ls) + (size_t)nwarps * wa_warp_bytes<P>(Ls);
}

// o += sum_t M[chi][s][t] tile(t) over the rows of one site; M row-major with
// rows of wa_mat_row(Ls) floats
__device__ __forceinline__ void wa_mix(const float *M, const float2 *site_tile, int s, int Ls, bool band, float2 *o)
{
    const int MR = wa_mat_row(Ls);
    const float *mu = M + (size_t)s * MR, *ml = M + (size_t)(Ls + s) * MR;
    const float4 *base = reinterpret_cast<const float4 *>(site_tile);
    if (band) {
#pragma unroll
        for (int dt = -1; dt <= 1; ++dt) {
            int t = s + dt;
            t = t < 0 ? t + Ls : (t >= Ls ? t - Ls : t);
            const float2 cu = p_splat(mu[t]), cl = p_splat(ml[t]);
            const float4 *row = base + (size_t)t * (LEAN_ROW / 2);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float4 v = row[q];
                o[2 * q] = p_fma(cu, make_float2(v.x, v.y), o[2 * q]);
                o[2 * q + 1] = p_fma(cl, make_float2(v.z, v.w), o[2 * q + 1]);
            }
        }
        return;
    }
#pragma unroll 1
    for (int t0 = 0; t0 < Ls; t0 += 4) {
        const float4 a4 = *reinterpret_cast<const float4 *>(mu + t0);
        const float4 b4 = *reinterpret_cast<const float4 *>(ml + t0);
        const float ca[4] = {a4.x, a4.y, a4.z, a4.w}, cb[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 cu = p_splat(ca[k]), cl = p_splat(cb[k]);
            const float4 *row = base + (size_t)(t0 + k) * (LEAN_ROW / 2);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float4 v = row[q];
                o[2 * q] = p_fma(cu, make_float2(v.x, v.y), o[2 * q]);
                o[2 * q + 1] = p_fma(cl, make_float2(v.z, v.w), o[2 * q + 1]);
            }
        }
    }
}

// Structured fifth-direction mixing (MixProg, dwf_internal.h) by chains: one
// chain = one real component of one site over its Ls slices.  The warp's hop
// results sit in its tile (rows of 28 floats per slice); each lane takes whole
// chains (the 24 (32/Ls) chains of a warp tile, 32 at a time) into registers,
// applies x <- d1 x, A5^-1 by its recurrence x_u = w_u + kappa x_{u-1}
// (w = x / alpha0, x_{-1} = -m x_last: a backward sum for x_last, then one
// forward pass), the shift (s0 + s1 K) x (the corner -m at the chain's start)
// and x <- d2 x, and writes the chain back; u is the position along the chain
// (s, or Ls - 1 - s when K reads s + 1).  Per chain element that is one 4-byte
// shared load and one store, against Ls 16-byte broadcast reads per output for
// the dense form.  Chains c = lane + 32 r all have component k = c mod 24 of
// the same chirality, (lane >> 1) & 1, since 24 and 32 are multiples of 4.
// The sites of a warp tile lie wc_site_stride floats apart: 24 banks on, so
// the 32 chains a warp loads at once (24 components of one site, 8 of the
// next) hit distinct banks.
__host__ __device__ constexpr int wc_site_stride(int Ls) { return Ls * 14 + 12; }   // float2

// a program in shared memory with the chirality-interleaved d vectors
struct WcProg {
    int inv, shift, up[2], d1one, d2one;
    float s0, s1, a0inv, kappa, mneg, corner;
    float d1[LS_MAX][2], d2[LS_MAX][2];
};
static_assert(3 * sizeof(WcProg) <= 2048, "the programs exceed the CTA's front area");

__device__ __forceinline__ void wc_load_prog(WcProg *dst, const MixProg<float> *src, int Ls, int tid, int nt)
{
    if (tid == 0) {
        dst->inv = src->inv;
        dst->shift = src->shift;
        dst->up[0] = src->up[0];
        dst->up[1] = src->up[1];
        dst->s0 = src->s0;
        dst->s1 = src->s1;
        dst->a0inv = src->a0inv;
        dst->kappa = src->kappa;
        dst->mneg = src->mneg;
        dst->corner = src->corner;
        int o1 = 1, o2 = 1;
        for (int c = 0; c < 2; ++c)
            for (int s = 0; s < Ls; ++s) {
                o1 &= src->d1[c][s] == 1.f;
                o2 &= src->d2[c][s] == 1.f;
            }
        dst->d1one = o1;
        dst->d2one = o2;
    }
    for (int e = tid; e < 2 * Ls; e += nt) {
        const int c = e / Ls, s = e - c * Ls;
        dst->d1[s][c] = src->d1[c][s];
        dst->d2[s][c] = src->d2[c][s];
    }
}

// the program applied to every chain of the warp's tile, in place (d1 is
// applied as the chain is loaded, d2 as it is stored)
template <int LS>
__device__ __forceinline__ void wc_chains(const WcProg *pg, float *tile, int lane)
{
    constexpr int NCH = (32 / LS) * 24;
    constexpr int RS = 2 * LEAN_ROW;   // floats between slices
    const int chi = (lane >> 1) & 1;
    const bool up = pg->up[chi] != 0;
    const bool o1 = pg->d1one != 0, o2 = pg->d2one != 0;
    const float kappa = pg->kappa, a0inv = pg->a0inv, mneg = pg->mneg, s0 = pg->s0, s1 = pg->s1;
#pragma unroll 1
    for (int c = lane; c < NCH; c += 32) {
        const int jj = c / 24, k = c - jj * 24;
        float *b = tile + (size_t)jj * 2 * wc_site_stride(LS) + k;
        float v[LS];
#pragma unroll
        for (int u = 0; u < LS; ++u) {
            const int sl = up ? LS - 1 - u : u;
            v[u] = b[sl * RS];
            if (!o1) v[u] *= pg->d1[sl][chi];
        }
        if (pg->inv) {
            float acc = 0.f;
#pragma unroll
            for (int u = 0; u < LS; ++u) acc = fmaf(kappa, acc, v[u]);
            float prev = mneg * (acc * a0inv * pg->corner);
#pragma unroll
            for (int u = 0; u < LS; ++u) {
                const float w = fmaf(v[u], a0inv, kappa * prev);
                prev = w;
                v[u] = w;
            }
            if (pg->shift) {
                float prevs = mneg * v[LS - 1];
#pragma unroll
                for (int u = 0; u < LS; ++u) {
                    const float tt = v[u];
                    v[u] = fmaf(s0, tt, s1 * prevs);
                    prevs = tt;
                }
            }
        } else if (pg->shift) {
            float prevs = mneg * v[LS - 1];
#pragma unroll
            for (int u = 0; u < LS; ++u) {
                const float tt = v[u];
                v[u] = fmaf(s0, tt, s1 * prevs);
                prevs = tt;
            }
        }
#pragma unroll
        for (int u = 0; u < LS; ++u) {
            const int sl = up ? LS - 1 - u : u;
            b[sl * RS] = o2 ? v[u] : v[u] * pg->d2[sl][chi];
        }
    }
}

__device__ __forceinline__ void wc_take(const float2 *row, float2 *o)
{
    const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 v = r4[q];
        o[2 * q] = make_float2(v.x, v.y);
        o[2 * q + 1] = make_float2(v.z, v.w);
    }
}

// the epilogue of hop_epilogue_core with the structured mixings by chains
// (every lane of the warp calls it; progs: post, y, z)
template <int P, int LS>
__device__ __forceinline__ float wc_epilogue(const HopArgs &a, const float2 *acc, float2 *tile, const WcProg *progs,
                                             int j, int s, int site, bool active, int lane)
{
    float2 *row = tile + (size_t)j * wc_site_stride(LS) + (size_t)s * LEAN_ROW;
    float *tf = reinterpret_cast<float *>(tile);
    if (active && a.rin.v && a.xacc) {   // independent of the hop: first, while few registers are live
        FieldRef xf;
        xf.v = a.xacc;
        const float2 xa = p_splat((float)(*a.xalpha));
        float2 xv[12], dx[12];
        ld_pairs_cs<DWF_F32>(xf, (size_t)site, s, LS, xv);
        ld_pairs_cs<P>(a.xdir, (size_t)site, s, LS, dx);
#pragma unroll
        for (int k = 0; k < 12; ++k) xv[k] = p_fma(xa, dx[k], xv[k]);
        st_pairs_cs<DWF_F32>(xf, (size_t)site, s, LS, xv);
    }
    lean_put(row, acc);   // inactive lanes put zeros
    __syncwarp();
    float2 o[12];
    wc_chains<LS>(progs, tf, lane);
    __syncwarp();
    wc_take(row, o);
    if (a.ymode != 0) {
        float2 y[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) y[k] = make_float2(0.f, 0.f);
        if (active) ld_pairs_cs<P>(a.y, (size_t)site, s, LS, y);
        if (a.ymode == 2) {
            __syncwarp();
            lean_put(row, y);
            __syncwarp();
            wc_chains<LS>(progs + 1, tf, lane);
            __syncwarp();
            wc_take(row, y);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = p_add(o[k], y[k]);
    }
    if (active && a.rin.v) {
        const float2 nal = p_splat((float)-(*a.ralpha));
        float2 r[12];
        ld_pairs_cs<P>(a.rin, (size_t)site, s, LS, r);
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = p_fma(nal, o[k], r[k]);
    }
    float nrm = 0.f;
    if (active && a.red.op != RED_NONE) {
        float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 12; ++k) s2 = p_fma(o[k], o[k], s2);
        nrm = s2.x + s2.y;
    }
    if (a.zmat) {
        __syncwarp();
        lean_put(row, o);
        __syncwarp();
        wc_chains<LS>(progs + 2, tf, lane);
        __syncwarp();
        wc_take(row, o);
    }
    if (active) st_pairs_cs<P>(a.out, (size_t)site, s, LS, o);
    return nrm;
}

// the epilogue of hop_epilogue_core (dense mixing) on the warp's tile
template <int P>
__device__ __forceinline__ float wa_epilogue(const HopArgs &a, const float2 *acc, float2 *site_tile,
                                             const float *mats, int s, int site, bool active)
{
    const int Ls = a.Ls;
    const int msz = 2 * Ls * wa_mat_row(Ls);
    float2 *row = site_tile + (size_t)s * LEAN_ROW;
    if (active && a.rin.v && a.xacc) {   // independent of the hop: first, while few registers are live
        FieldRef xf;
        xf.v = a.xacc;
        const float2 xa = p_splat((float)(*a.xalpha));
        float2 xv[12], dx[12];
        ld_pairs_cs<DWF_F32>(xf, (size_t)site, s, Ls, xv);
        ld_pairs_cs<P>(a.xdir, (size_t)site, s, Ls, dx);
#pragma unroll
        for (int k = 0; k < 12; ++k) xv[k] = p_fma(xa, dx[k], xv[k]);
        st_pairs_cs<DWF_F32>(xf, (size_t)site, s, Ls, xv);
    }
    if (active) lean_put(row, acc);
    __syncwarp();
    float2 o[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = make_float2(0.f, 0.f);
    if (active) wa_mix(mats, site_tile, s, Ls, a.post_band != 0, o);
    if (a.ymode == 1) {
        if (active) {
            float2 y[12];
            ld_pairs_cs<P>(a.y, (size_t)site, s, Ls, y);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[k] = p_add(o[k], y[k]);
        }
    } else if (a.ymode == 2) {
        __syncwarp();
        if (active) {
            float2 y[12];
            ld_pairs_cs<P>(a.y, (size_t)site, s, Ls, y);
            lean_put(row, y);
        }
        __syncwarp();
        if (active) wa_mix(mats + msz, site_tile, s, Ls, a.y_band != 0, o);
    }
    if (active && a.rin.v) {
        const float2 nal = p_splat((float)-(*a.ralpha));
        float2 r[12];
        ld_pairs_cs<P>(a.rin, (size_t)site, s, Ls, r);
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = p_fma(nal, o[k], r[k]);
    }
    float nrm = 0.f;
    if (active && a.red.op != RED_NONE) {
        float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 12; ++k) s2 = p_fma(o[k], o[k], s2);
        nrm = s2.x + s2.y;
    }
    if (a.zmat) {
        __syncwarp();
        if (active) lean_put(row, o);
        __syncwarp();
        float2 z[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = make_float2(0.f, 0.f);
        if (active) {
            wa_mix(mats + 2 * msz, site_tile, s, Ls, a.z_band != 0, z);
            st_pairs_cs<P>(a.out, (size_t)site, s, Ls, z);
        }
    } else if (active) {
        st_pairs_cs<P>(a.out, (size_t)site, s, Ls, o);
    }
    return nrm;
}

// the lanes' share of the link copies of a warp tile (sites site0 .. site0 + n - 1)
template <int P>
__device__ __forceinline__ void wa_issue_links(const void *gauge, int site0, int n, unsigned char *dst, int lane)
{
    constexpr int CH = LeanGeom<P>::LINK_BYTES / 16;
    const uint4 *src = reinterpret_cast<const uint4 *>(gauge) + (size_t)site0 * CH;
    const uint32_t d = smem_addr(dst);
    for (int c = lane; c < n * CH; c += 32) cp_async16(d + (uint32_t)c * 16, src + c);
    cp_async_commit();
}

// Grid: warp w of CTA b (global warp g = b nwarps + w) takes the warp tiles
// g, g + G, g + 2G, ... (G = all warps of the grid), so that the tiles in work
// at any moment form one window sweeping the lattice in the sweep order of
// sweep_site: the neighbour sites a tile shares with tiles one x-row or one
// t-slice away are still in L2 when those are processed (which a contiguous
// range per CTA, spreading the tiles in work over the whole lattice, loses once
// the fields exceed L2).
template <int P, bool DAG, int MINB, int MIX>
__global__ void __launch_bounds__(128, MINB) hop_wa_kernel(const HopArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls, SPW = 32 / Ls;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int j = lane / Ls, s = lane - (lane / Ls) * Ls;
    const int MR = wa_mat_row(Ls), msz = 2 * Ls * MR;
    float *mats = reinterpret_cast<float *>(smem_raw);
    // MIX 1: the structured programs, after the matrix area
    WcProg *progs = reinterpret_cast<WcProg *>(smem_raw + (size_t)3 * msz * sizeof(float));
    if constexpr (MIX == 1) {
        const MixProg<float> *src[3] = {reinterpret_cast<const MixProg<float> *>(a.post_prog),
                                        reinterpret_cast<const MixProg<float> *>(a.y_prog),
                                        reinterpret_cast<const MixProg<float> *>(a.z_prog)};
        for (int m = 0; m < 3; ++m)
            if (src[m] && (m != 1 || a.ymode == 2) && (m != 2 || a.zmat))
                wc_load_prog(progs + m, src[m], Ls, threadIdx.x, blockDim.x);
    } else {
        const float *src[3] = {reinterpret_cast<const float *>(a.post),
                               a.ymode == 2 ? reinterpret_cast<const float *>(a.ymat) : nullptr,
                               reinterpret_cast<const float *>(a.zmat)};
        for (int m = 0; m < 3; ++m) {
            if (!src[m]) continue;
            for (int k = threadIdx.x; k < 2 * Ls * Ls; k += blockDim.x) {
                const int chi = k / (Ls * Ls), r = k - chi * Ls * Ls, t = r / Ls, ss = r - t * Ls;
                mats[m * msz + (chi * Ls + ss) * MR + t] = src[m][k];
            }
        }
    }
    unsigned char *wbase = smem_raw + wa_front_bytes(Ls) + (size_t)warp * wa_warp_bytes<P>(Ls);
    unsigned char *links = wbase;
    float2 *tile = reinterpret_cast<float2 *>(wbase + (size_t)2 * SPW * LeanGeom<P>::LINK_BYTES);
    float2 *site_tile = tile + (size_t)j * lean_site_stride(Ls);
    __syncthreads();   // the matrices (the only CTA barrier before the final reduction)

    const int ntiles = (a.Vh + SPW - 1) / SPW;
    const int G = gridDim.x * nwarps;
    float nrm = 0.f;
    int u = blockIdx.x * nwarps + warp;
    if (u < ntiles) wa_issue_links<P>(a.gauge, sweep_site(a, u * SPW), min(SPW, a.Vh - u * SPW), links, lane);
    for (int k = 0; u < ntiles; ++k, u += G) {
        const int site = sweep_site(a, u * SPW) + j;
        const bool active = u * SPW + j < a.Vh;
        int n8[8];
        if (active) {
            const int4 *p = reinterpret_cast<const int4 *>(a.nbr + (size_t)site * 8);
            const int4 q0 = __ldg(p), q1 = __ldg(p + 1);
            n8[0] = q0.x; n8[1] = q0.y; n8[2] = q0.z; n8[3] = q0.w;
            n8[4] = q1.x; n8[5] = q1.y; n8[6] = q1.z; n8[7] = q1.w;
        }
        cp_async_wait<0>();
        __syncwarp();   // this tile's links are in; every lane is done with the previous tile
        const int un = u + G;
        if (un < ntiles)   // the next tile's links, into the other buffer
            wa_issue_links<P>(a.gauge, sweep_site(a, un * SPW), min(SPW, a.Vh - un * SPW),
                              links + (size_t)((k + 1) & 1) * SPW * LeanGeom<P>::LINK_BYTES, lane);
        float2 acc[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) acc[q] = make_float2(0.f, 0.f);
        if (active) {
            const unsigned char *lk = links + ((size_t)(k & 1) * SPW + j) * LeanGeom<P>::LINK_BYTES;
            lean_dir<P, DAG, 0>(acc, a.in, n8[0], s, Ls, lk);
            lean_dir<P, DAG, 1>(acc, a.in, n8[1], s, Ls, lk);
            lean_dir<P, DAG, 2>(acc, a.in, n8[2], s, Ls, lk);
            lean_dir<P, DAG, 3>(acc, a.in, n8[3], s, Ls, lk);
            lean_dir<P, DAG, 4>(acc, a.in, n8[4], s, Ls, lk);
            lean_dir<P, DAG, 5>(acc, a.in, n8[5], s, Ls, lk);
            lean_dir<P, DAG, 6>(acc, a.in, n8[6], s, Ls, lk);
            lean_dir<P, DAG, 7>(acc, a.in, n8[7], s, Ls, lk);
        }
        if constexpr (MIX == 1) {
            if (Ls == 16) nrm += wc_epilogue<P, 16>(a, acc, tile, progs, j, s, site, active, lane);
            else nrm += wc_epilogue<P, 8>(a, acc, tile, progs, j, s, site, active, lane);   // Ls 8 (launch_pd)
        } else {
            nrm += wa_epilogue<P>(a, acc, site_tile, mats, s, site, active);
        }
    }
    cp_async_wait<0>();
    if (a.red.op != RED_NONE) grid_reduce(nrm, a.red);
}


// ---------------------------------------------------------------- variant 10
// The hop of variant 9 (warp tiles of 32/Ls sites, each warp's links staged
// in its own shared buffer one tile ahead) with the dense fifth-direction
// mixings of the epilogue on the tensor cores.  Eight warps make a CTA step of
// S = 8 (32/Ls) sites; their hop results become the A operand of a tcgen05
// product, rows r = (site, component) (24 per site, 24 S = 384 rows = three
// M = 128 blocks for Ls 16, six for Ls 8), K = slice t; B = [M_+ | M_-]
// (N = 2 Ls) holds both chiralities' matrices, so D[r][chi Ls + s] =
// sum_t M_chi[s][t] A[r][t] and each row keeps the half of its chirality.
// Operands in two TF32 terms (A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 level),
// FP32 accumulators in tensor memory.  Each warp reads its rows back
// (tcgen05.ld: TMEM lane = row) into a shared tile in the field's own order
// (site, colour-re/im group g, slice, spin; rows of one (site, g) 4 Ls + 4
// floats apart, so the 32 rows of a warp write 32 distinct banks); the
// epilogue then runs per (site, s) as in variant 9 (16-byte field loads and
// stores, the y addition, the r update, the fused norm).  A second mixing
// (zmat, after the norm) stages the result again as an A operand for a second
// product.
//
// Against variant 9 the mixing leaves the SM's load/store path (variant 9
// reads Ls rows of the site tile and of the matrix per output from shared
// memory) for 48 scalar 4-byte shared stores per thread (A hi and lo), 24 per
// row read back and six 16-byte reads.  The A stores are free of bank
// conflicts: K-groups are LBO = 16 (rows/8) 8 + 16 bytes apart (4 banks), and
// the rows of the sites of one warp are rotated within 8-row groups by
// 8/(32/Ls) per site (a permutation of the site's 24 components, undone when
// the rows are read back), so the sites of a warp store into disjoint banks.
//
// Every mbarrier wait is bounded by %globaltimer (1 s) and its outcome made
// uniform over the CTA; a CTA that gives up sets the error flag, waits
// (bounded) for its committed MMAs, frees its tensor memory and leaves.
constexpr int HT_WARPS = 8;

struct HtGeom {
    int Ls, spw, sites, rows, mblk, np, shift, dstride;
    uint32_t lbo, a_bytes, b_lbo, b_bytes, tmem_cols;
    uint32_t d_off, link_off, bar_off, smem;
};

__host__ __device__ inline HtGeom ht_geom(int Ls)
{
    HtGeom g;
    g.Ls = Ls;
    g.spw = 32 / Ls;
    g.sites = HT_WARPS * g.spw;
    g.rows = 24 * g.sites;
    g.mblk = g.rows / 128;
    g.np = 2 * Ls;
    g.shift = 8 / g.spw;
    g.dstride = 4 * Ls + 4;   // floats between the (site, g) rows of the read-back tile
    g.lbo = (uint32_t)(g.rows / 8) * 128 + 16;
    g.a_bytes = (uint32_t)(Ls / 4) * g.lbo;
    g.b_lbo = (uint32_t)(g.np / 8) * 128;
    g.b_bytes = (uint32_t)(Ls / 4) * g.b_lbo;
    uint32_t c = 32;
    while (c < (uint32_t)(g.mblk * g.np)) c *= 2;
    g.tmem_cols = c;
    g.d_off = 2 * g.a_bytes + 4 * g.b_bytes;   // A hi, A lo, B post hi / lo, B z hi / lo, read-back tile
    g.link_off = g.d_off + (uint32_t)(g.sites * 6 * g.dstride * 4);
    g.bar_off = g.link_off + (uint32_t)(HT_WARPS * 2 * g.spw * LeanGeom<DWF_F32>::LINK_BYTES);
    g.smem = g.bar_off + 16;
    return g;
}

// variant 10 applies: FP32 fields, dense mixing mode, no mixed y term, Ls 8 or 16
__host__ __device__ inline bool ht_applies(const HopArgs &a)
{
    return a.mixmode == 0 && a.ymode != 2 && (a.Ls == 8 || a.Ls == 16);
}

// the MMAs of one product: D = A B^T over every M block, committed to the mbarrier
__device__ __forceinline__ void ht_issue(const HtGeom &g, uint32_t tbase, uint32_t sA, uint32_t sB, uint64_t *bar)
{
    const uint32_t idesc = idesc_tf32(g.np);
    for (int mb = 0; mb < g.mblk; ++mb) {
        const uint32_t d = tbase + (uint32_t)(mb * g.np);
        for (int ks = 0; ks < g.Ls / 8; ++ks) {
            const uint32_t ao = (uint32_t)ks * 2 * g.lbo + (uint32_t)mb * 16 * 128;
            const uint32_t bo = (uint32_t)ks * 2 * g.b_lbo;
            const uint64_t ah = smem_desc(sA + ao, g.lbo, 128), al = smem_desc(sA + g.a_bytes + ao, g.lbo, 128);
            const uint64_t bh = smem_desc(sB + bo, g.b_lbo, 128), bl = smem_desc(sB + g.b_bytes + bo, g.b_lbo, 128);
            mma_tf32(d, ah, bh, idesc, ks > 0);
            mma_tf32(d, ah, bl, idesc, 1);
            mma_tf32(d, al, bh, idesc, 1);
        }
    }
    tc_commit(bar);
}

// every thread waits for the product; false on the whole CTA if any thread gave up
__device__ __forceinline__ bool ht_wait(uint64_t *bar, uint32_t &phase)
{
    const bool ok = mbar_wait_bounded(smem_u32addr(bar), phase, 1000000000ull);
    phase ^= 1u;
    const bool all = !__syncthreads_or(!ok);
    tc_fence_after();
    return all;
}

// A operand rows of one (site, s) thread: row (local site) 24 + rotated component, K = s
template <int LS>
__device__ __forceinline__ void ht_stage_a(const HtGeom &g, unsigned char *Ahi, int lsite, int j, int s,
                                           const float2 *v)
{
    const int rbase = lsite * 24, sh = g.shift * j;
    const uint32_t kofs = (uint32_t)(s >> 2) * g.lbo + (uint32_t)(s & 3) * 4;
    unsigned char *Alo = Ahi + g.a_bytes;
#pragma unroll
    for (int c = 0; c < 24; ++c) {
        const float x = (c & 1) ? v[c >> 1].y : v[c >> 1].x;
        const int row = rbase + ((c & ~7) | ((c + sh) & 7));
        const uint32_t off = kofs + (uint32_t)row * 16;   // 8-row groups 128 bytes apart: 16 bytes per row
        const float hi = tf32_hi(x);
        *reinterpret_cast<float *>(Ahi + off) = hi;
        *reinterpret_cast<float *>(Alo + off) = tf32_hi(x - hi);
    }
}

// this warp's rows of the product -> the read-back tile D[(site 6 + g) dstride + 4 s + spin]
template <int LS>
__device__ __forceinline__ void ht_read_back(const HtGeom &g, uint32_t tbase, float *D, int warp, int lane)
{
    for (int mb = warp >> 2; mb < g.mblk; mb += 2) {
        const int R = mb * 128 + (warp & 3) * 32 + lane;
        const int site = R / 24, cp = R - site * 24, j = site % g.spw;
        const int c = (cp & ~7) | ((cp - g.shift * j) & 7);
        const int chi = (c >> 1) & 1;
        uint32_t r[2 * LS];
        tmem_ld<2 * LS>(tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(mb * g.np), r);
        float *row = D + (size_t)(site * 6 + (c >> 2)) * g.dstride + (c & 3);
#pragma unroll
        for (int t = 0; t < LS; ++t) row[4 * t] = __uint_as_float(chi ? r[LS + t] : r[t]);
    }
}

// the (site, s) thread's 24 components from the read-back tile
template <int LS>
__device__ __forceinline__ void ht_take(const HtGeom &g, const float *D, int lsite, int s, float2 *o)
{
    const float4 *p = reinterpret_cast<const float4 *>(D + (size_t)lsite * 6 * g.dstride) + s;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 q = p[(size_t)k * (g.dstride / 4)];
        o[2 * k] = make_float2(q.x, q.y);
        o[2 * k + 1] = make_float2(q.z, q.w);
    }
}

template <bool DAG, int LS>
__global__ void __launch_bounds__(256, 2) hop_tc_kernel(const HopArgs a, const HtGeom g)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int LB = LeanGeom<DWF_F32>::LINK_BYTES;
    constexpr int SPW = 32 / LS;
    unsigned char *Ahi = smem_raw;
    unsigned char *Bm = smem_raw + 2 * g.a_bytes;   // post hi, post lo, z hi, z lo
    float *D = reinterpret_cast<float *>(smem_raw + g.d_off);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + g.bar_off);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = lane / LS, s = lane - j * LS;
    const int lsite = warp * SPW + j;
    unsigned char *links = smem_raw + g.link_off + (size_t)warp * 2 * SPW * LB;

    // B operands, B[n][t] = M_chi[n - chi Ls][t] (n = chi Ls + s), in two TF32 terms
    {
        const float *src[2] = {reinterpret_cast<const float *>(a.post), reinterpret_cast<const float *>(a.zmat)};
        for (int m = 0; m < 2; ++m) {
            if (!src[m]) continue;
            for (int e = tid; e < g.np * LS; e += blockDim.x) {
                const int n = e / LS, k = e - n * LS, chi = n / LS, so = n - chi * LS;
                const float v = src[m][(chi * LS + k) * LS + so];
                const float hi = tf32_hi(v);
                const uint32_t off = kmaj_off(n, k, g.b_lbo);
                *reinterpret_cast<float *>(Bm + (2 * m) * g.b_bytes + off) = hi;
                *reinterpret_cast<float *>(Bm + (2 * m + 1) * g.b_bytes + off) = tf32_hi(v - hi);
            }
        }
    }
    if (warp == 0) tmem_alloc(tslot, g.tmem_cols);
    if (tid == 0) mbar_init(bar, 1);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t sA = smem_u32addr(Ahi), sB = smem_u32addr(Bm);

    const int nsteps = (a.Vh + g.sites - 1) / g.sites;
    const int nwt = (a.Vh + SPW - 1) / SPW;
    float nrm = 0.f;
    uint32_t phase = 0;
    bool failed = false;
    int st = blockIdx.x;
    {
        const int wt = st * HT_WARPS + warp;
        if (st < nsteps && wt < nwt)
            wa_issue_links<DWF_F32>(a.gauge, sweep_site(a, wt * SPW), min(SPW, a.Vh - wt * SPW), links, lane);
    }
    for (int k = 0; st < nsteps; ++k, st += gridDim.x) {
        // ---- the hop of this warp's tile
        const int wt = st * HT_WARPS + warp;
        const bool active = wt * SPW + j < a.Vh;
        const int site = active ? sweep_site(a, wt * SPW) + j : 0;
        int n8[8];
        if (active) {
            const int4 *p = reinterpret_cast<const int4 *>(a.nbr + (size_t)site * 8);
            const int4 q0 = __ldg(p), q1 = __ldg(p + 1);
            n8[0] = q0.x; n8[1] = q0.y; n8[2] = q0.z; n8[3] = q0.w;
            n8[4] = q1.x; n8[5] = q1.y; n8[6] = q1.z; n8[7] = q1.w;
        }
        cp_async_wait<0>();
        __syncwarp();
        {
            const int sn = st + gridDim.x, wn = sn * HT_WARPS + warp;
            if (sn < nsteps && wn < nwt)
                wa_issue_links<DWF_F32>(a.gauge, sweep_site(a, wn * SPW), min(SPW, a.Vh - wn * SPW),
                                        links + (size_t)((k + 1) & 1) * SPW * LB, lane);
        }
        float2 acc[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) acc[q] = make_float2(0.f, 0.f);
        if (active) {
            const unsigned char *lk = links + ((size_t)(k & 1) * SPW + j) * LB;
            lean_dir<DWF_F32, DAG, 0>(acc, a.in, n8[0], s, LS, lk);
            lean_dir<DWF_F32, DAG, 1>(acc, a.in, n8[1], s, LS, lk);
            lean_dir<DWF_F32, DAG, 2>(acc, a.in, n8[2], s, LS, lk);
            lean_dir<DWF_F32, DAG, 3>(acc, a.in, n8[3], s, LS, lk);
            lean_dir<DWF_F32, DAG, 4>(acc, a.in, n8[4], s, LS, lk);
            lean_dir<DWF_F32, DAG, 5>(acc, a.in, n8[5], s, LS, lk);
            lean_dir<DWF_F32, DAG, 6>(acc, a.in, n8[6], s, LS, lk);
            lean_dir<DWF_F32, DAG, 7>(acc, a.in, n8[7], s, LS, lk);
        }
        if (active && a.rin.v && a.xacc) {   // x += xalpha xdir (independent of the hop)
            FieldRef xf;
            xf.v = a.xacc;
            const float2 xa = p_splat((float)(*a.xalpha));
            float2 xv[12], dx[12];
            ld_pairs_cs<DWF_F32>(xf, (size_t)site, s, LS, xv);
            ld_pairs_cs<DWF_F32>(a.xdir, (size_t)site, s, LS, dx);
#pragma unroll
            for (int q = 0; q < 12; ++q) xv[q] = p_fma(xa, dx[q], xv[q]);
            st_pairs_cs<DWF_F32>(xf, (size_t)site, s, LS, xv);
        }
        // ---- o = post . acc on the tensor cores (inactive lanes stage zeros)
        ht_stage_a<LS>(g, Ahi, lsite, j, s, acc);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) ht_issue(g, tbase, sA, sB, bar);
        if (!ht_wait(bar, phase)) {
            failed = true;
            break;
        }
        ht_read_back<LS>(g, tbase, D, warp, lane);
        tc_fence_before();
        __syncthreads();
        float2 o[12];
        ht_take<LS>(g, D, lsite, s, o);
        // ---- the epilogue of variant 9 without its mixings
        if (active && a.ymode == 1) {
            float2 y[12];
            ld_pairs_cs<DWF_F32>(a.y, (size_t)site, s, LS, y);
#pragma unroll
            for (int q = 0; q < 12; ++q) o[q] = p_add(o[q], y[q]);
        }
        if (active && a.rin.v) {
            const float2 nal = p_splat((float)-(*a.ralpha));
            float2 r[12];
            ld_pairs_cs<DWF_F32>(a.rin, (size_t)site, s, LS, r);
#pragma unroll
            for (int q = 0; q < 12; ++q) o[q] = p_fma(nal, o[q], r[q]);
        }
        if (active && a.red.op != RED_NONE) {
            float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 12; ++q) s2 = p_fma(o[q], o[q], s2);
            nrm += s2.x + s2.y;
        }
        if (a.zmat) {   // out = zmat . o, a second product
            if (!active)
#pragma unroll
                for (int q = 0; q < 12; ++q) o[q] = make_float2(0.f, 0.f);
            ht_stage_a<LS>(g, Ahi, lsite, j, s, o);
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) ht_issue(g, tbase, sA, sB + 2 * g.b_bytes, bar);
            if (!ht_wait(bar, phase)) {
                failed = true;
                break;
            }
            ht_read_back<LS>(g, tbase, D, warp, lane);
            tc_fence_before();
            __syncthreads();
            ht_take<LS>(g, D, lsite, s, o);
        }
        if (active) st_pairs_cs<DWF_F32>(a.out, (size_t)site, s, LS, o);
    }
    cp_async_wait<0>();
    if (failed) {
        if (tid == 0 && a.err) atomicOr(a.err, 1);
        // the last committed product may still run: let it finish before the memory is freed (bounded)
        mbar_wait_bounded(smem_u32addr(bar), phase ^ 1u, 1000000000ull);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, g.tmem_cols);
    if (a.red.op != RED_NONE) grid_reduce(nrm, a.red);
}

// ---------------------------------------------------------------- launch
template <int P>
size_t direct_smem(int Ls, int SB)
{
    typedef typename Tr<P>::real R;
    typedef typename Tr<P>::pair T2;
    return (size_t)SB * (Ls * 12 + 2) * sizeof(T2) + (size_t)3 * 2 * Ls * Ls * sizeof(R);
}

template <int P, bool DAG, int NS, int MIX = 0, bool H2 = false>
cudaError_t launch_direct(const HopArgs &a, int SB, cudaStream_t st)
{
    if constexpr (NS == 1 && MIX == 0 && ((P == DWF_F16 && H2) || (P == DWF_F32 && !H2))) {
        static unsigned long long optin_occ = 0;
        cudaError_t e = smem_optin(hop_kernel_occ<P, DAG, MIX, H2>, 200 * 1024, optin_occ);
        if (e != cudaSuccess) return e;
        hop_kernel_occ<P, DAG, MIX, H2><<<(a.Vh + SB - 1) / SB, dim3(a.Ls, SB), direct_smem<P>(a.Ls, SB), st>>>(a);
        return cudaGetLastError();
    }
    static unsigned long long optin = 0;
    {
        cudaError_t e = smem_optin(hop_kernel<P, DAG, NS, MIX, H2>, 200 * 1024, optin);
        if (e != cudaSuccess) return e;
    }
    const int LsN = a.Ls / NS;
    hop_kernel<P, DAG, NS, MIX, H2><<<(a.Vh + SB - 1) / SB, dim3(LsN, SB), direct_smem<P>(a.Ls, SB), st>>>(a);
    return cudaGetLastError();
}

template <int P, bool DAG, int NS, int MIX, bool H2 = false>
cudaError_t launch_direct_batch(const HopArgs *tab, int nsys, const HopArgs &a0, int SB, cudaStream_t st)
{
    if constexpr (NS == 1 && MIX == 0 && ((P == DWF_F16 && H2) || (P == DWF_F32 && !H2))) {
        static unsigned long long optin_occ = 0;
        cudaError_t e = smem_optin(hop_batch_kernel_occ<P, DAG, MIX, H2>, 200 * 1024, optin_occ);
        if (e != cudaSuccess) return e;
        const long long g = (long long)((a0.Vh + SB - 1) / SB) * nsys;
        if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        hop_batch_kernel_occ<P, DAG, MIX, H2><<<(unsigned)g, dim3(a0.Ls, SB), direct_smem<P>(a0.Ls, SB), st>>>(tab, nsys);
        return cudaGetLastError();
    }
    static unsigned long long optin = 0;
    {
        cudaError_t e = smem_optin(hop_batch_kernel<P, DAG, NS, MIX, H2>, 200 * 1024, optin);
        if (e != cudaSuccess) return e;
    }
    const int LsN = a0.Ls / NS;
    const long long grid = (long long)((a0.Vh + SB - 1) / SB) * nsys;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    hop_batch_kernel<P, DAG, NS, MIX, H2><<<(unsigned)grid, dim3(LsN, SB), direct_smem<P>(a0.Ls, SB), st>>>(tab, nsys);
    return cudaGetLastError();
}

template <int P, bool DAG>
cudaError_t launch_batch_pd(const HopArgs *tab, int nsys, const HopArgs &a0, int NS, int SB, cudaStream_t st)
{
    if constexpr (P == DWF_F16) {   // FP16 arithmetic (as hop variant 5) with dense mixing
        if (a0.mixmode == 0)
            return NS == 2 ? launch_direct_batch<P, DAG, 2, 0, true>(tab, nsys, a0, SB, st)
                           : launch_direct_batch<P, DAG, 1, 0, true>(tab, nsys, a0, SB, st);
    }
    if (a0.mixmode == 1)
        return NS == 2 ? launch_direct_batch<P, DAG, 2, 1>(tab, nsys, a0, SB, st)
                       : launch_direct_batch<P, DAG, 1, 1>(tab, nsys, a0, SB, st);
    if constexpr (P != DWF_F64) {
        if (a0.mixmode == 2 && (a0.Ls / NS) * SB >= 32)
            return NS == 2 ? launch_direct_batch<P, DAG, 2, 2>(tab, nsys, a0, SB, st)
                           : launch_direct_batch<P, DAG, 1, 2>(tab, nsys, a0, SB, st);
    }
    return NS == 2 ? launch_direct_batch<P, DAG, 2, 0>(tab, nsys, a0, SB, st)
                   : launch_direct_batch<P, DAG, 1, 0>(tab, nsys, a0, SB, st);
}

// The 4D block of SB sites with the smallest faces whose extents divide the
// half-lattice extents; false if SB has no such factorisation.
bool choose_tile4(const int ext[4], int SB, Tile4 &best)
{
    long bestcost = -1;
    for (int t0 = 1; t0 <= ext[0] && t0 <= SB; ++t0) {
        if (ext[0] % t0 || SB % t0) continue;
        for (int t1 = 1; t1 <= ext[1] && t0 * t1 <= SB; ++t1) {
            if (ext[1] % t1 || (SB / t0) % t1) continue;
            for (int t2 = 1; t2 <= ext[2] && t0 * t1 * t2 <= SB; ++t2) {
                if (ext[2] % t2 || (SB / (t0 * t1)) % t2) continue;
                const int t3 = SB / (t0 * t1 * t2);
                if (t3 < 1 || t3 > ext[3] || ext[3] % t3) continue;
                // halo sites fetched besides the block's own: one face per direction
                const long cost = 2L * SB / t0 + 2L * SB / t1 + 2L * SB / t2 + 2L * SB / t3;
                if (bestcost < 0 || cost < bestcost) {
                    bestcost = cost;
                    best.tb[0] = t0;
                    best.tb[1] = t1;
                    best.tb[2] = t2;
                    best.tb[3] = t3;
                }
            }
        }
    }
    return bestcost >= 0;
}

template <int P, bool DAG, int NS>
cudaError_t launch_block(const HopArgs &a, int SB, cudaStream_t st)
{
    static unsigned long long optin = 0;
    {
        cudaError_t e = smem_optin(hop_block_kernel<P, DAG, NS>, 200 * 1024, optin);
        if (e != cudaSuccess) return e;
    }
    Tile4 T;
    if (!choose_tile4(a.ext, SB, T)) return launch_direct<P, DAG, NS>(a, SB, st);
    const int LsN = a.Ls / NS;
    hop_block_kernel<P, DAG, NS><<<a.Vh / SB, dim3(LsN, SB), direct_smem<P>(a.Ls, SB), st>>>(a, T);
    return cudaGetLastError();
}

template <int P, bool DAG, int NS>
cudaError_t launch_sweep(const HopArgs &a, int SB, cudaStream_t st)
{
    static unsigned long long optin = 0;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = smem_optin(hop_sweep_kernel<P, DAG, NS>, 200 * 1024, optin)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int LsN = a.Ls / NS;
    const size_t smem = direct_smem<P>(a.Ls, SB);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hop_sweep_kernel<P, DAG, NS>, LsN * SB, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int ntiles = (a.Vh + SB - 1) / SB;
    int grid = nsm * per_sm;
    if (grid > ntiles) grid = ntiles;
    const int tpc = (ntiles + grid - 1) / grid;
    grid = (ntiles + tpc - 1) / tpc;
    hop_sweep_kernel<P, DAG, NS><<<grid, dim3(LsN, SB), smem, st>>>(a, tpc);
    return cudaGetLastError();
}

// Variant 7: persistent CTAs of SB sites, as many per SM as fit.
template <int P, bool DAG, int MINB>
cudaError_t launch_lean(const HopArgs &a, int SB, cudaStream_t st)
{
    static unsigned long long optin = 0;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = smem_optin(hop_lean_kernel<P, DAG, MINB>, 200 * 1024, optin)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (SB < 1) SB = 1;
    while (SB > 1 && a.Ls * SB > 256) --SB;
    const size_t smem = lean_smem_bytes<P>(a.Ls, SB);
    if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hop_lean_kernel<P, DAG, MINB>, a.Ls * SB, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int ntiles = (a.Vh + SB - 1) / SB;
    int grid = nsm * per_sm;
    if (grid > ntiles) grid = ntiles;
    hop_lean_kernel<P, DAG, MINB><<<grid, dim3(a.Ls, SB), smem, st>>>(a);
    return cudaGetLastError();
}

// Variant 9: persistent CTAs of `nw` warps (2, 4 or 8 resident CTAs' worth of
// registers: nw x MINB x 32 threads per SM), as many per SM as fit.
template <int P, bool DAG, int MINB, int MIX>
cudaError_t launch_wa(const HopArgs &a, int nw, cudaStream_t st)
{
    static unsigned long long optin = 0;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = smem_optin(hop_wa_kernel<P, DAG, MINB, MIX>, 200 * 1024, optin)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (nw < 1) nw = 4;
    if (nw > 4) nw = 4;
    const size_t smem = wa_cta_bytes<P>(a.Ls, nw);
    if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hop_wa_kernel<P, DAG, MINB, MIX>, 32 * nw, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int SPW = 32 / a.Ls;
    const int ntiles = (a.Vh + SPW - 1) / SPW;
    int grid = nsm * per_sm;
    if (grid > (ntiles + nw - 1) / nw) grid = (ntiles + nw - 1) / nw;
    hop_wa_kernel<P, DAG, MINB, MIX><<<grid, 32 * nw, smem, st>>>(a);
    return cudaGetLastError();
}

template <bool DAG, int LS>
cudaError_t launch_tc(const HopArgs &a, cudaStream_t st)
{
    static unsigned long long optin = 0;
    const HtGeom g = ht_geom(LS);
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = smem_optin(hop_tc_kernel<DAG, LS>, 200 * 1024, optin)) != cudaSuccess) return e;
    // two CTAs of about 100 KB per SM: ask for the largest shared-memory carveout (the
    // driver's default split admitted one)
    static bool carve = false;
    if (!carve) {
        if ((e = cudaFuncSetAttribute(hop_tc_kernel<DAG, LS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
            return e;
        carve = true;
    }
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // CTAs per SM from the shared memory and the register file (the occupancy query answered
    // one CTA where two fit); more CTAs than fit would only wait for a slot (no CTA waits on
    // another), and two take 256 of the 512 tensor-memory columns
    {
        cudaFuncAttributes fa;
        int smem_sm = 0, resv = 0, regs_sm = 0;
        if ((e = cudaFuncGetAttributes(&fa, hop_tc_kernel<DAG, LS>)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
            return e;
        if ((e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess)
            return e;
        const int by_smem = smem_sm / (int)(g.smem + fa.sharedSizeBytes + resv);
        const int by_regs = regs_sm / (fa.numRegs * 32 * HT_WARPS);
        per_sm = by_smem < by_regs ? by_smem : by_regs;
        if (per_sm > 2) per_sm = 2;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
    }
    const int nsteps = (a.Vh + g.sites - 1) / g.sites;
    int grid = nsm * per_sm;
    if (grid > nsteps) grid = nsteps;
    hop_tc_kernel<DAG, LS><<<grid, 32 * HT_WARPS, g.smem, st>>>(a, g);
    return cudaGetLastError();
}

template <int P, bool DAG>
cudaError_t launch_pd(const HopArgs &a, int var, int NS, int SB, cudaStream_t st)
{
    // variant 10: variant 9 with the dense mixings on the tensor cores (FP32 fields, Ls 8 or 16,
    // no mixed y term; else variant 9)
    if constexpr (P == DWF_F32) {
        if (var == 10 && ht_applies(a)) return a.Ls == 16 ? launch_tc<DAG, 16>(a, st) : launch_tc<DAG, 8>(a, st);
    }
    if (var == 10) {
        var = 9;
        NS = 2;
        SB = 4;
    }

    // variant 9: warp-autonomous (FP32 and FP16 fields, dense mixing, Ls dividing 32 and a
    // multiple of 4); SB = warps per CTA, NS selects the register budget (1: 5 CTAs of 4
    // warps per SM, 2: 4)
    if constexpr (P != DWF_F64) {
        if (var == 9 && a.mixmode == 0 && a.Ls <= 32 && 32 % a.Ls == 0 && a.Ls % 4 == 0)
            return NS == 2 ? launch_wa<P, DAG, 4, 0>(a, SB, st) : launch_wa<P, DAG, 5, 0>(a, SB, st);
        // structured mixing by chains in registers (Ls 8 and 16)
        if (var == 9 && a.mixmode == 1 && (a.Ls == 8 || a.Ls == 16))
            return NS == 2 ? launch_wa<P, DAG, 4, 1>(a, SB, st) : launch_wa<P, DAG, 5, 1>(a, SB, st);
    }
    if (var == 9) var = P == DWF_F16 ? 5 : 0;
    if constexpr (P != DWF_F64) {
        if (var == 7 && a.mixmode == 0 && a.Ls % 4 == 0) return launch_lean<P, DAG, 2>(a, SB, st);
    }
    if (var == 7) var = P == DWF_F16 ? 5 : 0;

    // variant 5: FP16 fields with FP16 projection and SU(3) arithmetic (dense mixing)
    if constexpr (P == DWF_F16) {
        if (var == 5 && a.mixmode == 0) {
            if (NS == 4) return launch_direct<P, DAG, 4, 0, true>(a, SB, st);
            if (NS == 2) return launch_direct<P, DAG, 2, 0, true>(a, SB, st);
            return launch_direct<P, DAG, 1, 0, true>(a, SB, st);
        }
    }
    if (var == 5) var = 0;
    if (NS == 4) NS = 2;
    // the structured and tensor-core mixings are compiled for the direct variant only
    if (a.mixmode == 1) {
        if (NS == 2) return launch_direct<P, DAG, 2, 1>(a, SB, st);
        return launch_direct<P, DAG, 1, 1>(a, SB, st);
    }
    if constexpr (P != DWF_F64) {
        if (a.mixmode == 2 && (a.Ls / NS) * SB >= 32) {
            if (NS == 2) return launch_direct<P, DAG, 2, 2>(a, SB, st);
            return launch_direct<P, DAG, 1, 2>(a, SB, st);
        }
    }
    if (var == 4) {
        if (NS == 2) return launch_block<P, DAG, 2>(a, SB, st);
        return launch_block<P, DAG, 1>(a, SB, st);
    }
    if (var == 3) {
        if (NS == 2) return launch_sweep<P, DAG, 2>(a, SB, st);
        return launch_sweep<P, DAG, 1>(a, SB, st);
    }
    if (NS == 2) return launch_direct<P, DAG, 2>(a, SB, st);
    return launch_direct<P, DAG, 1>(a, SB, st);
}

}  // namespace

// Launchers of one precision and direction, instantiated in hop_<prec>_<dir>.cu
// (one translation unit each, compiled in parallel).
template <int P, bool DAG>
cudaError_t hop_launch_pd(const HopArgs &a, int var, int NS, int SB, cudaStream_t st)
{
    return launch_pd<P, DAG>(a, var, NS, SB, st);
}
template <int P, bool DAG>
cudaError_t hop_batch_launch_pd(const HopArgs *tab, int nsys, const HopArgs &a0, int NS, int SB, cudaStream_t st)
{
    return launch_batch_pd<P, DAG>(tab, nsys, a0, NS, SB, st);
}

}  // namespace dwf
