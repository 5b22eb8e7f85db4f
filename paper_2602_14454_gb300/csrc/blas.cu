// Site-local kernels: fifth-direction mixing, CG vector updates, packing
// between the canonical complex-double layout and the internal layout,
// precision conversion, norms, index tables and link preparation.
#include "fields.cuh"

namespace dwf {
namespace {

constexpr int kThreads = 256;

inline int blocks_for(size_t n, int t = kThreads) { return (int)((n + t - 1) / t); }
inline int grid_cap(size_t n) { int b = blocks_for(n); return b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b); }

// Tiled kernels over (site, s) with one slice per thread: blockDim = (Ls, SB).
inline int tile_sb(int Ls) { int sb = 128 / Ls; return sb < 1 ? 1 : sb; }

// copy the [chi][t][s] matrix into shared memory as [chi][t][s] (NS = 1 layout)
template <typename R>
__device__ __forceinline__ void load_mat(R *dst, const void *src, int Ls)
{
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int k = tid; k < 2 * Ls * Ls; k += nt) dst[k] = reinterpret_cast<const R *>(src)[k];
}

// o = (mixing of row s of site j's tile): dense matrix or structured program
// (the structured form transforms the CTA's whole tile in place first).  The
// tile must be complete and visible; every thread of the CTA must call it.
template <int MIX, typename T2, typename R>
__device__ __forceinline__ void mix_tile_any(const void *prog, const R *mtx, T2 *tile, int tstride, int j,
                                             int s, int Ls, bool active, T2 (*o)[12], int band = 0)
{
    if constexpr (MIX == 1) {
        chain_mix<R>(reinterpret_cast<const MixProg<R> *>(prog), tile, tstride, blockDim.y, Ls,
                     threadIdx.y * blockDim.x + threadIdx.x, blockDim.x * blockDim.y);
        __syncthreads();
        if (active) {
            T2 h[12];
            ld_tile_row(tile + j * tstride + s * 12, h);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[0][k] = p_add(o[0][k], h[k]);
        }
    } else if (active) {
        if (band)
            mix_pairs_band<1>(mtx, tile + j * tstride, s, Ls, o);
        else
            mix_pairs<1>(mtx, tile + j * tstride, s, Ls, o);
    }
}

// out(site, s) = sum_t M[chi][s][t] in(site, t)
template <int P, int MIX>
__global__ void __launch_bounds__(256) mix_kernel(const MixArgs a)
{
    typedef typename Tr<P>::real R;
    typedef typename Tr<P>::pair T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls, s = threadIdx.x, j = threadIdx.y, SB = blockDim.y;
    const int site = blockIdx.x * SB + j;
    const bool active = site < a.Vh;
    const int tstride = Ls * 12 + 2;
    T2 *tile = reinterpret_cast<T2 *>(smem_raw);
    R *mtx = reinterpret_cast<R *>(tile + SB * tstride);
    load_mat<R>(mtx, a.mat, Ls);
    if (active) {
        T2 v[12];
        ld_pairs<P, true>(a.in, (size_t)site, s, Ls, v);
        T2 *dst = tile + j * tstride + s * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = v[k];
    }
    __syncthreads();
    T2 o[1][12];
#pragma unroll
    for (int k = 0; k < 12; ++k) o[0][k] = p_splat((R)0);
    mix_tile_any<MIX>(a.prog, mtx, tile, tstride, j, s, Ls, active, o, a.band);
    if (active) st_pairs<P>(a.out, (size_t)site, s, Ls, o[0]);
}

// p = r + beta p (or p = r), phat = M p, on tile u (sites u SB .. u SB + SB - 1)
template <int P, int MIX>
__device__ __forceinline__ void cg_update_tile(const CgUpdateArgs &a, int u)
{
    typedef typename Tr<P>::real R;
    typedef typename Tr<P>::pair T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls, s = threadIdx.x, j = threadIdx.y, SB = blockDim.y;
    const int site = u * SB + j;
    const bool active = site < a.Vh;
    const int tstride = Ls * 12 + 2;
    T2 *tile = reinterpret_cast<T2 *>(smem_raw);
    R *mtx = reinterpret_cast<R *>(tile + SB * tstride);
    load_mat<R>(mtx, a.mat, Ls);
    if (active) {
        T2 r[12], p[12];
        ld_pairs<P, false>(a.r, (size_t)site, s, Ls, r);
        const double xal = a.xacc ? a.scal->alpha : 0.0;
        if (!a.init || xal != 0.0) ld_pairs<P, false>(a.p, (size_t)site, s, Ls, p);
        if (xal != 0.0) {
            // x += alpha p of the previous iteration (same arithmetic as in the hop epilogue)
            constexpr int XP = (P == DWF_F64) ? DWF_F64 : DWF_F32;
            FieldRef xf;
            xf.v = a.xacc;
            T2 xv[12];
            ld_pairs<XP, false>(xf, (size_t)site, s, Ls, xv);
            const T2 xa = p_splat((R)xal);
#pragma unroll
            for (int k = 0; k < 12; ++k) xv[k] = p_fma(xa, p[k], xv[k]);
            st_pairs<XP>(xf, (size_t)site, s, Ls, xv);
        }
        if (a.init) {
#pragma unroll
            for (int k = 0; k < 12; ++k) p[k] = r[k];
        } else {
            const T2 be = p_splat((R)a.scal->beta);
#pragma unroll
            for (int k = 0; k < 12; ++k) p[k] = p_fma(be, p[k], r[k]);
        }
        st_pairs<P>(a.p, (size_t)site, s, Ls, p);
        T2 *dst = tile + j * tstride + s * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = p[k];
    }
    __syncthreads();
    T2 o[1][12];
#pragma unroll
    for (int k = 0; k < 12; ++k) o[0][k] = p_splat((R)0);
    mix_tile_any<MIX>(a.prog, mtx, tile, tstride, j, s, Ls, active, o, a.band);
    if (active) st_pairs<P>(a.phat, (size_t)site, s, Ls, o[0]);
}

template <int P, int MIX>
__global__ void __launch_bounds__(256) cg_update_kernel(const CgUpdateArgs a)
{
    cg_update_tile<P, MIX>(a, blockIdx.x);
}

// Batched form over nsys systems of equal Ls: CTA b updates tile b / nsys of
// system b % nsys; systems whose skip flag is set are left untouched.
template <int P, int MIX>
__global__ void __launch_bounds__(256) cg_update_batch_kernel(const CgUpdateArgs *__restrict__ tab, int nsys)
{
    __shared__ __align__(16) unsigned char abuf[sizeof(CgUpdateArgs)];
    const int sys = blockIdx.x % nsys, u = blockIdx.x / nsys;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    const unsigned *src = reinterpret_cast<const unsigned *>(tab + sys);
    for (int k = tid; k < (int)(sizeof(CgUpdateArgs) / 4); k += nt) reinterpret_cast<unsigned *>(abuf)[k] = src[k];
    __syncthreads();
    const CgUpdateArgs &a = *reinterpret_cast<const CgUpdateArgs *>(abuf);
    if (a.skip && *a.skip) return;
    cg_update_tile<P, MIX>(a, u);
}

template <int P>
size_t tile_smem(int Ls, int SB)
{
    typedef typename Tr<P>::real R;
    typedef typename Tr<P>::pair T2;
    return (size_t)SB * (Ls * 12 + 2) * sizeof(T2) + (size_t)2 * Ls * Ls * sizeof(R);
}

template <int P, int MIX>
cudaError_t launch_mix_m(const MixArgs &a, cudaStream_t st)
{
    static unsigned long long optin = 0;
    {
        cudaError_t e = smem_optin(mix_kernel<P, MIX>, 200 * 1024, optin);
        if (e != cudaSuccess) return e;
    }
    const int SB = tile_sb(a.Ls);
    mix_kernel<P, MIX><<<(a.Vh + SB - 1) / SB, dim3(a.Ls, SB), tile_smem<P>(a.Ls, SB), st>>>(a);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_mix_t(const MixArgs &a, cudaStream_t st)
{
    // FP32/FP16: a banded matrix takes the dense form's three-row path (faster than its program)
    return a.mixmode == 1 && (P == DWF_F64 || !a.band) ? launch_mix_m<P, 1>(a, st) : launch_mix_m<P, 0>(a, st);
}

template <int P, int MIX>
cudaError_t launch_cg_update_m(const CgUpdateArgs &a, cudaStream_t st)
{
    static unsigned long long optin = 0;
    {
        cudaError_t e = smem_optin(cg_update_kernel<P, MIX>, 200 * 1024, optin);
        if (e != cudaSuccess) return e;
    }
    const int SB = tile_sb(a.Ls);
    cg_update_kernel<P, MIX><<<(a.Vh + SB - 1) / SB, dim3(a.Ls, SB), tile_smem<P>(a.Ls, SB), st>>>(a);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_cg_update_t(const CgUpdateArgs &a, cudaStream_t st)
{
    return a.mixmode == 1 && (P == DWF_F64 || !a.band) ? launch_cg_update_m<P, 1>(a, st)
                                                       : launch_cg_update_m<P, 0>(a, st);
}

template <int P, int MIX>
cudaError_t launch_cg_update_batch_m(const CgUpdateArgs *tab, int nsys, const CgUpdateArgs &a0, cudaStream_t st)
{
    static unsigned long long optin = 0;
    {
        cudaError_t e = smem_optin(cg_update_batch_kernel<P, MIX>, 200 * 1024, optin);
        if (e != cudaSuccess) return e;
    }
    const int SB = tile_sb(a0.Ls);
    const long long grid = (long long)((a0.Vh + SB - 1) / SB) * nsys;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cg_update_batch_kernel<P, MIX><<<(unsigned)grid, dim3(a0.Ls, SB), tile_smem<P>(a0.Ls, SB), st>>>(tab, nsys);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_cg_update_batch_t(const CgUpdateArgs *tab, int nsys, const CgUpdateArgs &a0, cudaStream_t st)
{
    return a0.mixmode == 1 && (P == DWF_F64 || !a0.band) ? launch_cg_update_batch_m<P, 1>(tab, nsys, a0, st)
                                                         : launch_cg_update_batch_m<P, 0>(tab, nsys, a0, st);
}

// ------------------------------------------------------------------ packing
// canonical 24 reals (spin*3 + a)*2 + c  <->  internal pairs (4g + spin, g = 2a + c)
__device__ __forceinline__ void canon_to_pairs(const double *c, double2 *v)
{
    double r[24];
#pragma unroll
    for (int k = 0; k < 24; k += 2) {
        const double2 q = *reinterpret_cast<const double2 *>(c + k);
        r[k] = q.x;
        r[k + 1] = q.y;
    }
#pragma unroll
    for (int p = 0; p < 12; ++p)
        v[p] = make_double2(r[canon_of_internal(2 * p)], r[canon_of_internal(2 * p + 1)]);
}
__device__ __forceinline__ void pairs_to_canon(const double2 *v, double *c)
{
    double r[24];
#pragma unroll
    for (int p = 0; p < 12; ++p) {
        r[canon_of_internal(2 * p)] = v[p].x;
        r[canon_of_internal(2 * p + 1)] = v[p].y;
    }
#pragma unroll
    for (int k = 0; k < 24; k += 2) *reinterpret_cast<double2 *>(c + k) = make_double2(r[k], r[k + 1]);
}

// thread per (parity, eo site, s); canonical full field [s][lex][24 reals]
template <int P>
__global__ void pack_full_kernel(const double *canon, FieldRef even, FieldRef odd, const int *eo2lex, int Vh,
                                 int V, int Ls, int unpack)
{
    const size_t n = (size_t)2 * Vh * Ls;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(idx % Ls);
        const size_t rest = idx / Ls;
        const int site = (int)(rest % Vh);
        const int par = (int)(rest / Vh);
        const int lex = eo2lex[(size_t)par * Vh + site];
        const FieldRef &f = par ? odd : even;
        double *c = const_cast<double *>(canon) + ((size_t)s * V + lex) * 24;
        double2 v[12];
        if (!unpack) {
            canon_to_pairs(c, v);
            st_pairs<P>(f, (size_t)site, s, Ls, v);
        } else {
            ld_pairs<P, false>(f, (size_t)site, s, Ls, v);
            pairs_to_canon(v, c);
        }
    }
}

// canonical EO field [s][i][24 reals]
template <int P>
__global__ void pack_eo_kernel(const double *canon, FieldRef f, int Vh, int Ls, int unpack)
{
    const size_t n = (size_t)Vh * Ls;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(idx % Ls);
        const int site = (int)(idx / Ls);
        double *c = const_cast<double *>(canon) + ((size_t)s * Vh + site) * 24;
        double2 v[12];
        if (!unpack) {
            canon_to_pairs(c, v);
            st_pairs<P>(f, (size_t)site, s, Ls, v);
        } else {
            ld_pairs<P, false>(f, (size_t)site, s, Ls, v);
            pairs_to_canon(v, c);
        }
    }
}

template <int PI, int PO>
__global__ void convert_kernel(FieldRef in, FieldRef out, int Vh, int Ls)
{
    const size_t n = (size_t)Vh * Ls;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(idx % Ls);
        const size_t site = idx / Ls;
        double2 v[12];
        ld_pairs<PI, true>(in, site, s, Ls, v);
        st_pairs<PO>(out, site, s, Ls, v);
    }
}

// x64 += xs + alpha p, xs = 0: the accumulated x of the inner iterations with
// the last iteration's deferred update alpha p added in the accumulator's
// precision (the arithmetic of the p update kernel), then folded into FP64
template <int XP, int P>
__global__ void accum_x_kernel(double *x64, void *xs, FieldRef pf, const double *alpha, int Vh, int Ls)
{
    typedef typename Tr<XP>::real R;
    typedef typename Tr<XP>::pair T2;
    const size_t n = (size_t)Vh * Ls;
    const R al = alpha ? (R)*alpha : (R)0;
    FieldRef fx;
    fx.v = x64;
    FieldRef fs;
    fs.v = xs;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(idx % Ls);
        const size_t site = idx / Ls;
        T2 d[12];
        ld_pairs<XP, false>(fs, site, s, Ls, d);
        if (al != (R)0) {
            T2 q[12];
            ld_pairs<P, false>(pf, site, s, Ls, q);
            const T2 a2 = p_splat(al);
#pragma unroll
            for (int k = 0; k < 12; ++k) d[k] = p_fma(a2, q[k], d[k]);
        }
        double2 x[12];
        ld_pairs<DWF_F64, false>(fx, site, s, Ls, x);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            x[k] = p_add(x[k], make_double2((double)d[k].x, (double)d[k].y));
            d[k] = p_splat((R)0);
        }
        st_pairs<DWF_F64>(fx, site, s, Ls, x);
        st_pairs<XP>(fs, site, s, Ls, d);
    }
}

template <int P>
__global__ void __launch_bounds__(256) norm2_kernel(FieldRef f, int Vh, int Ls, RedArgs red)
{
    const size_t n = (size_t)Vh * Ls;
    double acc = 0;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(idx % Ls);
        const size_t site = idx / Ls;
        double2 v[12];
        ld_pairs<P, true>(f, site, s, Ls, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc += v[k].x * v[k].x + v[k].y * v[k].y;
    }
    grid_reduce(acc, red);
}

// ------------------------------------------------------------ tables, links
__device__ __forceinline__ void eo_coords(int par, int i, const int *d, int c[4])
{
    const int hx = d[0] / 2;
    int r = i / hx;
    const int xh = i % hx;
    c[1] = r % d[1];
    r /= d[1];
    c[2] = r % d[2];
    c[3] = r / d[2];
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + par) & 1);
}
__device__ __forceinline__ int lex_of(const int c[4], const int *d)
{
    return c[0] + d[0] * (c[1] + d[1] * (c[2] + d[2] * c[3]));
}
__device__ __forceinline__ int eo_of(const int c[4], const int *d)
{
    return c[0] / 2 + (d[0] / 2) * (c[1] + d[1] * (c[2] + d[2] * c[3]));
}

struct Dims {
    int d[4];
    int bc[4];
};

__global__ void tables_kernel(Dims D, int Vh, int *nbr, int *eo2lex)
{
    const int n = 2 * Vh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int par = idx / Vh, i = idx % Vh;
        int c[4];
        eo_coords(par, i, D.d, c);
        eo2lex[idx] = lex_of(c, D.d);
        for (int mu = 0; mu < 4; ++mu) {
            int f[4] = {c[0], c[1], c[2], c[3]};
            int b[4] = {c[0], c[1], c[2], c[3]};
            f[mu] = (c[mu] + 1) % D.d[mu];
            b[mu] = (c[mu] - 1 + D.d[mu]) % D.d[mu];
            nbr[(size_t)idx * 8 + mu] = eo_of(f, D.d);
            nbr[(size_t)idx * 8 + 4 + mu] = eo_of(b, D.d);
        }
    }
}

__global__ void pack_gauge_kernel(const double *U, Dims D, int Vh, int V, double *g64, float *g32, __half *g16)
{
    const size_t n = (size_t)2 * Vh * 8;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int dir = (int)(idx % 8);
        const int i = (int)((idx / 8) % Vh);
        const int par = (int)(idx / (8 * (size_t)Vh));
        int c[4];
        eo_coords(par, i, D.d, c);
        const int mu = dir & 3;
        double u[18];
        if (dir < 4) {
            const double ph = (c[mu] == D.d[mu] - 1) ? (double)D.bc[mu] : 1.0;
            const double *src = U + ((size_t)mu * V + lex_of(c, D.d)) * 18;
            for (int k = 0; k < 18; ++k) u[k] = ph * src[k];
        } else {
            int b[4] = {c[0], c[1], c[2], c[3]};
            b[mu] = (c[mu] - 1 + D.d[mu]) % D.d[mu];
            const double ph = (c[mu] == 0) ? (double)D.bc[mu] : 1.0;
            const double *src = U + ((size_t)mu * V + lex_of(b, D.d)) * 18;
            // dagger: u[a][b] = conj(U[b][a])
            for (int a = 0; a < 3; ++a)
                for (int bb = 0; bb < 3; ++bb) {
                    u[(a * 3 + bb) * 2] = ph * src[(bb * 3 + a) * 2];
                    u[(a * 3 + bb) * 2 + 1] = -ph * src[(bb * 3 + a) * 2 + 1];
                }
        }
        const size_t o = idx * 18;
        for (int k = 0; k < 18; ++k) {
            g64[o + k] = u[k];
            g32[o + k] = (float)u[k];
            g16[o + k] = __double2half(u[k]);
        }
    }
}

// x4 = P_- x5(s=1) + P_+ x5(s=Ls)
__global__ void project4d_kernel(const double *x5, double *x4, int V, int Ls)
{
    const size_t n = (size_t)V * 24;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % 24);
        const size_t site = idx / 24;
        const int spin = k / 6;
        const int s = (spin < 2) ? (Ls - 1) : 0;
        x4[idx] = x5[((size_t)s * V + site) * 24 + k];
    }
}

// v5 = P^dag (0, ..., 0, b4): v(s=1) = P_+ b4, v(s=Ls) = P_- b4, zero elsewhere
__global__ void chiral_embed_kernel(const double *b4, double *v5, int V, int Ls)
{
    const size_t n = (size_t)Ls * V * 24;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % 24);
        const size_t site = (idx / 24) % V;
        const int s = (int)(idx / (24 * (size_t)V));
        const int spin = k / 6;
        double v = 0.0;
        if (s == 0 && spin < 2) v = b4[site * 24 + k];
        if (s == Ls - 1 && spin >= 2) v = b4[site * 24 + k];
        v5[idx] = v;
    }
}

}  // namespace

size_t field_bytes(int prec, int Vh, int Ls)
{
    const size_t n = (size_t)Vh * Ls * 24;
    return prec == DWF_F64 ? n * 8 : (prec == DWF_F32 ? n * 4 : n * 2);
}
// FP16 scales: [site][Ls rounded up to 4] floats, so that one site's scales are a 16-byte multiple
size_t scale_bytes(int prec, int Vh, int Ls) { return prec == DWF_F16 ? (size_t)Vh * ((Ls + 3) & ~3) * 4 : 0; }

cudaError_t launch_mix(int prec, const MixArgs &a, cudaStream_t st)
{
    if (a.mixmode == 2 && prec != DWF_F64 && a.Ls <= 32) return launch_mix_tc(prec, a, st);
    switch (prec) {
    case DWF_F64: return launch_mix_t<DWF_F64>(a, st);
    case DWF_F32: return launch_mix_t<DWF_F32>(a, st);
    case DWF_F16: return launch_mix_t<DWF_F16>(a, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cg_update(int prec, const CgUpdateArgs &a, cudaStream_t st)
{
    switch (prec) {
    case DWF_F64: return launch_cg_update_t<DWF_F64>(a, st);
    case DWF_F32: return launch_cg_update_t<DWF_F32>(a, st);
    case DWF_F16: return launch_cg_update_t<DWF_F16>(a, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cg_update_batch(int prec, const CgUpdateArgs *tab, int nsys, const CgUpdateArgs &a0,
                                   cudaStream_t st)
{
    if (nsys < 1) return cudaSuccess;
    switch (prec) {
    case DWF_F64: return launch_cg_update_batch_t<DWF_F64>(tab, nsys, a0, st);
    case DWF_F32: return launch_cg_update_batch_t<DWF_F32>(tab, nsys, a0, st);
    case DWF_F16: return launch_cg_update_batch_t<DWF_F16>(tab, nsys, a0, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_pack_full(int prec, const double *canon, FieldRef even, FieldRef odd, const int *eo2lex, int Vh,
                             int V, int Ls, cudaStream_t st)
{
    const int g = grid_cap((size_t)2 * Vh * Ls);
    switch (prec) {
    case DWF_F64: pack_full_kernel<DWF_F64><<<g, kThreads, 0, st>>>(canon, even, odd, eo2lex, Vh, V, Ls, 0); break;
    case DWF_F32: pack_full_kernel<DWF_F32><<<g, kThreads, 0, st>>>(canon, even, odd, eo2lex, Vh, V, Ls, 0); break;
    case DWF_F16: pack_full_kernel<DWF_F16><<<g, kThreads, 0, st>>>(canon, even, odd, eo2lex, Vh, V, Ls, 0); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack_full(int prec, FieldRef even, FieldRef odd, double *canon, const int *eo2lex, int Vh,
                               int V, int Ls, cudaStream_t st)
{
    const int g = grid_cap((size_t)2 * Vh * Ls);
    switch (prec) {
    case DWF_F64: pack_full_kernel<DWF_F64><<<g, kThreads, 0, st>>>(canon, even, odd, eo2lex, Vh, V, Ls, 1); break;
    case DWF_F32: pack_full_kernel<DWF_F32><<<g, kThreads, 0, st>>>(canon, even, odd, eo2lex, Vh, V, Ls, 1); break;
    case DWF_F16: pack_full_kernel<DWF_F16><<<g, kThreads, 0, st>>>(canon, even, odd, eo2lex, Vh, V, Ls, 1); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_eo(int prec, const double *canon, FieldRef f, int Vh, int Ls, cudaStream_t st)
{
    const int g = grid_cap((size_t)Vh * Ls);
    switch (prec) {
    case DWF_F64: pack_eo_kernel<DWF_F64><<<g, kThreads, 0, st>>>(canon, f, Vh, Ls, 0); break;
    case DWF_F32: pack_eo_kernel<DWF_F32><<<g, kThreads, 0, st>>>(canon, f, Vh, Ls, 0); break;
    case DWF_F16: pack_eo_kernel<DWF_F16><<<g, kThreads, 0, st>>>(canon, f, Vh, Ls, 0); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack_eo(int prec, FieldRef f, double *canon, int Vh, int Ls, cudaStream_t st)
{
    const int g = grid_cap((size_t)Vh * Ls);
    switch (prec) {
    case DWF_F64: pack_eo_kernel<DWF_F64><<<g, kThreads, 0, st>>>(canon, f, Vh, Ls, 1); break;
    case DWF_F32: pack_eo_kernel<DWF_F32><<<g, kThreads, 0, st>>>(canon, f, Vh, Ls, 1); break;
    case DWF_F16: pack_eo_kernel<DWF_F16><<<g, kThreads, 0, st>>>(canon, f, Vh, Ls, 1); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_convert(int pi, FieldRef in, int po, FieldRef out, int Vh, int Ls, cudaStream_t st)
{
    const int g = grid_cap((size_t)Vh * Ls);
#define CONV(A, B) convert_kernel<A, B><<<g, kThreads, 0, st>>>(in, out, Vh, Ls)
    if (pi == DWF_F64 && po == DWF_F64) CONV(DWF_F64, DWF_F64);
    else if (pi == DWF_F64 && po == DWF_F32) CONV(DWF_F64, DWF_F32);
    else if (pi == DWF_F64 && po == DWF_F16) CONV(DWF_F64, DWF_F16);
    else if (pi == DWF_F32 && po == DWF_F64) CONV(DWF_F32, DWF_F64);
    else if (pi == DWF_F32 && po == DWF_F32) CONV(DWF_F32, DWF_F32);
    else if (pi == DWF_F32 && po == DWF_F16) CONV(DWF_F32, DWF_F16);
    else if (pi == DWF_F16 && po == DWF_F64) CONV(DWF_F16, DWF_F64);
    else if (pi == DWF_F16 && po == DWF_F32) CONV(DWF_F16, DWF_F32);
    else if (pi == DWF_F16 && po == DWF_F16) CONV(DWF_F16, DWF_F16);
    else return cudaErrorInvalidValue;
#undef CONV
    return cudaGetLastError();
}

cudaError_t launch_accum_x(double *x64, void *xs, int xs_prec, FieldRef p, int p_prec, const double *alpha, int Vh,
                           int Ls, cudaStream_t st)
{
    const int g = grid_cap((size_t)Vh * Ls);
    if (xs_prec == DWF_F64 && p_prec == DWF_F64)
        accum_x_kernel<DWF_F64, DWF_F64><<<g, kThreads, 0, st>>>(x64, xs, p, alpha, Vh, Ls);
    else if (xs_prec == DWF_F32 && p_prec == DWF_F32)
        accum_x_kernel<DWF_F32, DWF_F32><<<g, kThreads, 0, st>>>(x64, xs, p, alpha, Vh, Ls);
    else if (xs_prec == DWF_F32 && p_prec == DWF_F16)
        accum_x_kernel<DWF_F32, DWF_F16><<<g, kThreads, 0, st>>>(x64, xs, p, alpha, Vh, Ls);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_norm2(int prec, FieldRef f, int Vh, int Ls, const RedArgs &red, cudaStream_t st)
{
    const int g = grid_cap((size_t)Vh * Ls);
    switch (prec) {
    case DWF_F64: norm2_kernel<DWF_F64><<<g, kThreads, 0, st>>>(f, Vh, Ls, red); break;
    case DWF_F32: norm2_kernel<DWF_F32><<<g, kThreads, 0, st>>>(f, Vh, Ls, red); break;
    case DWF_F16: norm2_kernel<DWF_F16><<<g, kThreads, 0, st>>>(f, Vh, Ls, red); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_zero(int prec, FieldRef f, int Vh, int Ls, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(f.v, 0, field_bytes(prec, Vh, Ls), st);
    if (e == cudaSuccess && f.scale) e = cudaMemsetAsync(f.scale, 0, scale_bytes(prec, Vh, Ls), st);
    return e;
}

cudaError_t launch_build_tables(const int dims[4], int *nbr, int *eo2lex, cudaStream_t st)
{
    Dims D;
    for (int k = 0; k < 4; ++k) D.d[k] = dims[k], D.bc[k] = 1;
    const int V = dims[0] * dims[1] * dims[2] * dims[3];
    const int Vh = V / 2;
    tables_kernel<<<grid_cap((size_t)2 * Vh), kThreads, 0, st>>>(D, Vh, nbr, eo2lex);
    return cudaGetLastError();
}

cudaError_t launch_pack_gauge(const double *U, const int dims[4], const int bc[4], const int *eo2lex, const int *nbr,
                              void *g64, void *g32, void *g16, cudaStream_t st)
{
    (void)eo2lex;
    (void)nbr;
    Dims D;
    for (int k = 0; k < 4; ++k) D.d[k] = dims[k], D.bc[k] = bc[k];
    const int V = dims[0] * dims[1] * dims[2] * dims[3];
    const int Vh = V / 2;
    pack_gauge_kernel<<<grid_cap((size_t)2 * Vh * 8), kThreads, 0, st>>>(
        U, D, Vh, V, (double *)g64, (float *)g32, (__half *)g16);
    return cudaGetLastError();
}

cudaError_t launch_project4d(const double *x5, double *x4, int V, int Ls, cudaStream_t st)
{
    project4d_kernel<<<grid_cap((size_t)V * 24), kThreads, 0, st>>>(x5, x4, V, Ls);
    return cudaGetLastError();
}

cudaError_t launch_chiral_embed(const double *b4, double *b5, int V, int Ls, cudaStream_t st)
{
    chiral_embed_kernel<<<grid_cap((size_t)Ls * V * 24), kThreads, 0, st>>>(b4, b5, V, Ls);
    return cudaGetLastError();
}

}  // namespace dwf
