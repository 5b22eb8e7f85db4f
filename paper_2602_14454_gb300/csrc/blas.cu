// Site-local kernels: fifth-direction mixing, CG vector updates, packing
// between the canonical complex-double layout and the internal layout,
// precision conversion, norms, index tables and link preparation.
#include "fields.cuh"

namespace dwf {
namespace {

constexpr int kThreads = 256;

inline int blocks_for(size_t n, int t = kThreads) { return (int)((n + t - 1) / t); }

template <typename real>
__device__ __forceinline__ void mix_tile2(const real *M, const real *tile, int s, int Ls, real *o)
{
    for (int t = 0; t < Ls; ++t) {
        const real mu = M[t * Ls + s];
        const real ml = M[Ls * Ls + t * Ls + s];
        const real *h = tile + t * 24;
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] += mu * h[k];
#pragma unroll
        for (int k = 12; k < 24; ++k) o[k] += ml * h[k];
    }
}

inline int mix_sb(int Ls) { int sb = 128 / Ls; return sb < 1 ? 1 : sb; }

// out(site, s) = sum_t M[chi][s][t] in(site, t)
template <int P>
__global__ void __launch_bounds__(256) mix_kernel(const MixArgs a)
{
    typedef typename Tr<P>::real real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls, s = threadIdx.x, j = threadIdx.y, SB = blockDim.y;
    const int site = blockIdx.x * SB + j;
    const bool active = site < a.Vh;
    const int tstride = Ls * 24 + (sizeof(real) == 8 ? 2 : 4);
    real *tile = reinterpret_cast<real *>(smem_raw);
    real *mtx = tile + SB * tstride;
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int k = tid; k < 2 * Ls * Ls; k += nt) mtx[k] = reinterpret_cast<const real *>(a.mat)[k];
    if (active) {
        real v[24];
        ld_field<P, true>(a.in, (size_t)site, s, Ls, v);
        real *dst = tile + j * tstride + s * 24;
#pragma unroll
        for (int k = 0; k < 24; ++k) dst[k] = v[k];
    }
    __syncthreads();
    if (!active) return;
    real o[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) o[k] = 0;
    mix_tile2(mtx, tile + j * tstride, s, Ls, o);
    st_field<P>(a.out, (size_t)site, s, Ls, o);
}

// p = r + beta p (or p = r), phat = M p
template <int P>
__global__ void __launch_bounds__(256) cg_update_kernel(const CgUpdateArgs a)
{
    typedef typename Tr<P>::real real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls, s = threadIdx.x, j = threadIdx.y, SB = blockDim.y;
    const int site = blockIdx.x * SB + j;
    const bool active = site < a.Vh;
    const int tstride = Ls * 24 + (sizeof(real) == 8 ? 2 : 4);
    real *tile = reinterpret_cast<real *>(smem_raw);
    real *mtx = tile + SB * tstride;
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int k = tid; k < 2 * Ls * Ls; k += nt) mtx[k] = reinterpret_cast<const real *>(a.mat)[k];
    if (active) {
        real r[24], p[24];
        ld_field<P, false>(a.r, (size_t)site, s, Ls, r);
        if (a.init) {
#pragma unroll
            for (int k = 0; k < 24; ++k) p[k] = r[k];
        } else {
            ld_field<P, false>(a.p, (size_t)site, s, Ls, p);
            const real be = (real)a.scal->beta;
#pragma unroll
            for (int k = 0; k < 24; ++k) p[k] = r[k] + be * p[k];
        }
        st_field<P>(a.p, (size_t)site, s, Ls, p);
        real *dst = tile + j * tstride + s * 24;
#pragma unroll
        for (int k = 0; k < 24; ++k) dst[k] = p[k];
    }
    __syncthreads();
    if (!active) return;
    real o[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) o[k] = 0;
    mix_tile2(mtx, tile + j * tstride, s, Ls, o);
    st_field<P>(a.phat, (size_t)site, s, Ls, o);
}

template <int P>
size_t tile_smem(int Ls, int SB)
{
    typedef typename Tr<P>::real real;
    const int tstride = Ls * 24 + (sizeof(real) == 8 ? 2 : 4);
    return (size_t)(SB * tstride + 2 * Ls * Ls) * sizeof(real);
}

template <int P>
cudaError_t launch_mix_t(const MixArgs &a, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(mix_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int SB = mix_sb(a.Ls);
    mix_kernel<P><<<(a.Vh + SB - 1) / SB, dim3(a.Ls, SB), tile_smem<P>(a.Ls, SB), st>>>(a);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_cg_update_t(const CgUpdateArgs &a, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(cg_update_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             160 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int SB = mix_sb(a.Ls);
    cg_update_kernel<P><<<(a.Vh + SB - 1) / SB, dim3(a.Ls, SB), tile_smem<P>(a.Ls, SB), st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ packing
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
        double r[24];
        if (!unpack) {
#pragma unroll
            for (int k = 0; k < 24; k += 2) {
                double2 q = *reinterpret_cast<const double2 *>(c + k);
                r[k] = q.x;
                r[k + 1] = q.y;
            }
            st_field<P>(f, (size_t)site, s, Ls, r);
        } else {
            ld_field<P, false>(f, (size_t)site, s, Ls, r);
#pragma unroll
            for (int k = 0; k < 24; k += 2) *reinterpret_cast<double2 *>(c + k) = make_double2(r[k], r[k + 1]);
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
        double r[24];
        if (!unpack) {
#pragma unroll
            for (int k = 0; k < 24; k += 2) {
                double2 q = *reinterpret_cast<const double2 *>(c + k);
                r[k] = q.x;
                r[k + 1] = q.y;
            }
            st_field<P>(f, (size_t)site, s, Ls, r);
        } else {
            ld_field<P, false>(f, (size_t)site, s, Ls, r);
#pragma unroll
            for (int k = 0; k < 24; k += 2) *reinterpret_cast<double2 *>(c + k) = make_double2(r[k], r[k + 1]);
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
        double r[24];
        ld_field<PI, true>(in, site, s, Ls, r);
        st_field<PO>(out, site, s, Ls, r);
    }
}

template <int XP>
__global__ void accum_x_kernel(double *x64, void *xs, int Vh, int Ls)
{
    const size_t n = (size_t)Vh * Ls;
    FieldRef fx;
    fx.v = x64;
    FieldRef fs;
    fs.v = xs;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(idx % Ls);
        const size_t site = idx / Ls;
        double x[24], d[24];
        ld_field<DWF_F64, false>(fx, site, s, Ls, x);
        ld_field<XP, false>(fs, site, s, Ls, d);
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            x[k] += d[k];
            d[k] = 0.0;
        }
        st_field<DWF_F64>(fx, site, s, Ls, x);
        st_field<XP>(fs, site, s, Ls, d);
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
        double r[24];
        ld_field<P, true>(f, site, s, Ls, r);
#pragma unroll
        for (int k = 0; k < 24; ++k) acc += r[k] * r[k];
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

inline int grid_cap(size_t n) { int b = blocks_for(n); return b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b); }

}  // namespace

size_t field_bytes(int prec, int Vh, int Ls)
{
    const size_t n = (size_t)Vh * Ls * 24;
    return prec == DWF_F64 ? n * 8 : (prec == DWF_F32 ? n * 4 : n * 2);
}
size_t scale_bytes(int prec, int Vh, int Ls) { return prec == DWF_F16 ? (size_t)Vh * Ls * 4 : 0; }

cudaError_t launch_mix(int prec, const MixArgs &a, cudaStream_t st)
{
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

#define DWF_PREC_DISPATCH(prec, KER, ...)                                     \
    switch (prec) {                                                           \
    case DWF_F64: KER<DWF_F64><<<__VA_ARGS__>>>; break;                       \
    case DWF_F32: KER<DWF_F32><<<__VA_ARGS__>>>; break;                       \
    case DWF_F16: KER<DWF_F16><<<__VA_ARGS__>>>; break;                       \
    default: return cudaErrorInvalidValue;                                    \
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

cudaError_t launch_accum_x(double *x64, void *xs, int xs_prec, int Vh, int Ls, cudaStream_t st)
{
    const int g = grid_cap((size_t)Vh * Ls);
    if (xs_prec == DWF_F64) accum_x_kernel<DWF_F64><<<g, kThreads, 0, st>>>(x64, xs, Vh, Ls);
    else accum_x_kernel<DWF_F32><<<g, kThreads, 0, st>>>(x64, xs, Vh, Ls);
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
