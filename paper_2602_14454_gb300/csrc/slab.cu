// 4D domain decomposition in time: one handle per slab of nt time slices
// (global t in [t0, t0 + nt)), the hop's t-neighbours beyond the slab read
// from two ghost faces appended to the slab's fields.
//
// A field of one parity holds Vh = A3 nt local sites (A3 = Lx/2 Ly Lz sites of
// one parity per time slice; the local even-odd index has t slowest, so the
// slice t = 0 is rows [0, A3) and t = nt - 1 rows [(nt - 1) A3, nt A3)),
// followed by the ghost faces: rows [Vh, Vh + A3) hold the lower neighbour's
// last slice (global t0 - 1), rows [Vh + A3, Vh + 2 A3) the upper neighbour's
// first slice (global t0 + nt), both in the same (x, y, z) order.  Slab
// origins and lengths are even, so a site's parity is the same in local and
// global coordinates, and a face of one rank is, row for row, a ghost face of
// its neighbour: the exchange is a copy of contiguous rows (Sec. 2.3's
// operator is unchanged; the decomposition is the library's).
//
// The links of the slab's sites come from the global field, with the
// boundary phase of the global lattice: the backward t-link at the slab's
// first slice is U_t(x - t)^dag of the lower neighbour's last slice.
#include "dwf_internal.h"
#include "fields.cuh"

namespace dwf {
namespace {

constexpr int kThreads = 256;

int grid_for(size_t n)
{
    size_t g = (n + kThreads - 1) / kThreads;
    if (g > 65535u * 4u) g = 65535u * 4u;
    return (int)(g ? g : 1);
}

__device__ __forceinline__ void slab_coords(int par, int i, const int *d, int c[4])
{
    const int xh = d[0] / 2;
    c[0] = i % xh;
    int r = i / xh;
    c[1] = r % d[1];
    r /= d[1];
    c[2] = r % d[2];
    c[3] = r / d[2];
    c[0] = 2 * c[0] + ((c[1] + c[2] + c[3] + par) & 1);
}

struct SlabGeom {
    int d[4];    // local extents (Lx, Ly, Lz, nt)
    int g[4];    // global extents
    int bc[4];
    int t0, Vh, A3;
};

// neighbour table of the slab: local sites, ghost rows beyond the time faces
__global__ void slab_tables_kernel(SlabGeom G, int *nbr)
{
    const int n = 2 * G.Vh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int par = idx / G.Vh, i = idx % G.Vh;
        int c[4];
        slab_coords(par, i, G.d, c);
        const int eo3 = c[0] / 2 + (G.d[0] / 2) * (c[1] + G.d[1] * c[2]);
        for (int mu = 0; mu < 4; ++mu) {
            int f[4] = {c[0], c[1], c[2], c[3]}, b[4] = {c[0], c[1], c[2], c[3]};
            int fi, bi;
            if (mu < 3) {
                f[mu] = (c[mu] + 1) % G.d[mu];
                b[mu] = (c[mu] - 1 + G.d[mu]) % G.d[mu];
                fi = f[0] / 2 + (G.d[0] / 2) * (f[1] + G.d[1] * (f[2] + G.d[2] * f[3]));
                bi = b[0] / 2 + (G.d[0] / 2) * (b[1] + G.d[1] * (b[2] + G.d[2] * b[3]));
            } else {
                fi = c[3] + 1 < G.d[3] ? eo3 + G.A3 * (c[3] + 1) : G.Vh + G.A3 + eo3;
                bi = c[3] > 0 ? eo3 + G.A3 * (c[3] - 1) : G.Vh + eo3;
            }
            nbr[(size_t)idx * 8 + mu] = fi;
            nbr[(size_t)idx * 8 + 4 + mu] = bi;
        }
    }
}

// links of the slab's sites from the global field U[4][V_global][3][3] (lexicographic, x fastest)
__global__ void slab_pack_gauge_kernel(const double *U, SlabGeom G, double *g64, float *g32, __half *g16)
{
    const size_t n = (size_t)2 * G.Vh * 8;
    const size_t Vg = (size_t)G.g[0] * G.g[1] * G.g[2] * G.g[3];
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int dir = (int)(idx % 8);
        const int i = (int)((idx / 8) % G.Vh);
        const int par = (int)(idx / (8 * (size_t)G.Vh));
        int c[4];
        slab_coords(par, i, G.d, c);
        c[3] = (c[3] + G.t0) % G.g[3];   // global coordinates
        const int mu = dir & 3;
        double u[18];
        if (dir < 4) {
            const double ph = (c[mu] == G.g[mu] - 1) ? (double)G.bc[mu] : 1.0;
            const size_t lex = c[0] + (size_t)G.g[0] * (c[1] + (size_t)G.g[1] * (c[2] + (size_t)G.g[2] * c[3]));
            const double *src = U + ((size_t)mu * Vg + lex) * 18;
            for (int k = 0; k < 18; ++k) u[k] = ph * src[k];
        } else {
            int b[4] = {c[0], c[1], c[2], c[3]};
            b[mu] = (c[mu] - 1 + G.g[mu]) % G.g[mu];
            const double ph = (c[mu] == 0) ? (double)G.bc[mu] : 1.0;
            const size_t lex = b[0] + (size_t)G.g[0] * (b[1] + (size_t)G.g[1] * (b[2] + (size_t)G.g[2] * b[3]));
            const double *src = U + ((size_t)mu * Vg + lex) * 18;
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

SlabGeom geom_of(const dwf_ctx *h)
{
    SlabGeom G;
    for (int k = 0; k < 4; ++k) {
        G.d[k] = h->dims[k];
        G.g[k] = h->gdims[k];
        G.bc[k] = h->bc[k];
    }
    G.t0 = h->t0;
    G.Vh = h->Vh;
    G.A3 = h->Vh / h->dims[3];
    return G;
}

// FP64 complex vectors of the decomposed CG (canonical layout, n complex numbers)
constexpr int kDotBlocks = 256;

// per-block partial sums of Re sum conj(a_k) b_k, the blocks' grid-stride ranges fixed
__global__ void __launch_bounds__(kThreads) cdot_kernel(const double2 *a, const double2 *b, size_t n, double *part)
{
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double2 u = a[k], v = b[k];
        acc += u.x * v.x + u.y * v.y;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// the partials in a fixed order
__global__ void csum_kernel(const double *part, int np, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += part[i];
        *out = s;
    }
}

// y = a x + b y
__global__ void caxpby_kernel(double a, const double2 *x, double b, double2 *y, size_t n)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double2 u = x[k], v = y[k];
        y[k] = make_double2(a * u.x + b * v.x, a * u.y + b * v.y);
    }
}

}  // namespace

cudaError_t launch_cdot(const void *a, const void *b, size_t n, double *part, double *out, cudaStream_t st)
{
    cdot_kernel<<<kDotBlocks, kThreads, 0, st>>>((const double2 *)a, (const double2 *)b, n, part);
    csum_kernel<<<1, 32, 0, st>>>(part, kDotBlocks, out);
    return cudaGetLastError();
}

cudaError_t launch_caxpby(double a, const void *x, double b, void *y, size_t n, cudaStream_t st)
{
    caxpby_kernel<<<grid_for(n), kThreads, 0, st>>>(a, (const double2 *)x, b, (double2 *)y, n);
    return cudaGetLastError();
}

cudaError_t launch_slab_tables(const dwf_ctx *h, cudaStream_t st)
{
    const SlabGeom G = geom_of(h);
    slab_tables_kernel<<<grid_for((size_t)2 * G.Vh), kThreads, 0, st>>>(G, h->nbr);
    return cudaGetLastError();
}

cudaError_t launch_slab_pack_gauge(const dwf_ctx *h, const double *U, cudaStream_t st)
{
    const SlabGeom G = geom_of(h);
    slab_pack_gauge_kernel<<<grid_for((size_t)2 * G.Vh * 8), kThreads, 0, st>>>(
        U, G, (double *)h->gauge[0], (float *)h->gauge[1], (__half *)h->gauge[2]);
    return cudaGetLastError();
}

}  // namespace dwf
