// The even-odd hopping stencil of the 5D domain-wall operator with its fused
// fifth-direction mixing and epilogue (one launch = one of the two hops of
// every application of the even-odd matrix, eq. even-odd_linear_equation).
//
// H psi(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
// is the hopping sum of eq. (Wilson_matrix) (D_W = (4 - M0) - H/2); it is the
// same for every fifth-direction slice s, so one CTA handles SB sites x all
// Ls slices and every link it loads serves Ls slices.  The adjoint hop is
// gamma5 H gamma5 (signs of the projectors flipped).
//
// In the chiral basis gamma_mu = [[0, e_mu], [e_mu^dag, 0]] with
// e_k = -i sigma_k, e_4 = 1, so (1 - sig gamma_mu) psi = [h ; -sig e_mu^dag h]
// with the half spinor h = psi_u - sig e_mu psi_l: only h (6 complex) is
// multiplied by the link.
//
// After the hop, each thread owns h(site, s); the CTA writes its Ls x 24 tile
// to shared memory and each thread forms (Post h)(site, s) = sum_t Post[s][t]
// h(site, t) per chirality; the optional epilogue adds a mixed second input,
// forms a residual, updates a solution accumulator, applies a final mixing
// and reduces |o|^2 deterministically.
#include "fields.cuh"

namespace dwf {
namespace {

template <typename real, int MU, int SIG>
__device__ __forceinline__ void project(const real *p, real *h)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const real p0r = p[(0 * 3 + a) * 2], p0i = p[(0 * 3 + a) * 2 + 1];
        const real p1r = p[(1 * 3 + a) * 2], p1i = p[(1 * 3 + a) * 2 + 1];
        const real p2r = p[(2 * 3 + a) * 2], p2i = p[(2 * 3 + a) * 2 + 1];
        const real p3r = p[(3 * 3 + a) * 2], p3i = p[(3 * 3 + a) * 2 + 1];
        real h0r, h0i, h1r, h1i;
        if constexpr (MU == 0) {        // e_1 psi_l = (-i psi3, -i psi2)
            h0r = p0r - SIG * p3i; h0i = p0i + SIG * p3r;
            h1r = p1r - SIG * p2i; h1i = p1i + SIG * p2r;
        } else if constexpr (MU == 1) { // e_2 psi_l = (-psi3, psi2)
            h0r = p0r + SIG * p3r; h0i = p0i + SIG * p3i;
            h1r = p1r - SIG * p2r; h1i = p1i - SIG * p2i;
        } else if constexpr (MU == 2) { // e_3 psi_l = (-i psi2, i psi3)
            h0r = p0r - SIG * p2i; h0i = p0i + SIG * p2r;
            h1r = p1r + SIG * p3i; h1i = p1i - SIG * p3r;
        } else {                        // e_4 psi_l = (psi2, psi3)
            h0r = p0r - SIG * p2r; h0i = p0i - SIG * p2i;
            h1r = p1r - SIG * p3r; h1i = p1i - SIG * p3i;
        }
        h[(0 * 3 + a) * 2] = h0r; h[(0 * 3 + a) * 2 + 1] = h0i;
        h[(1 * 3 + a) * 2] = h1r; h[(1 * 3 + a) * 2 + 1] = h1i;
    }
}

template <typename real, int MU, int SIG>
__device__ __forceinline__ void reconstruct(real *acc, const real *q)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const real q0r = q[(0 * 3 + a) * 2], q0i = q[(0 * 3 + a) * 2 + 1];
        const real q1r = q[(1 * 3 + a) * 2], q1i = q[(1 * 3 + a) * 2 + 1];
        real *a0 = acc + (0 * 3 + a) * 2, *a1 = acc + (1 * 3 + a) * 2;
        real *a2 = acc + (2 * 3 + a) * 2, *a3 = acc + (3 * 3 + a) * 2;
        a0[0] += q0r; a0[1] += q0i;
        a1[0] += q1r; a1[1] += q1i;
        // lower = -SIG e_mu^dag q
        if constexpr (MU == 0) {        // e_1^dag q = (i q1, i q0)
            a2[0] += SIG * q1i; a2[1] -= SIG * q1r;
            a3[0] += SIG * q0i; a3[1] -= SIG * q0r;
        } else if constexpr (MU == 1) { // e_2^dag q = (q1, -q0)
            a2[0] -= SIG * q1r; a2[1] -= SIG * q1i;
            a3[0] += SIG * q0r; a3[1] += SIG * q0i;
        } else if constexpr (MU == 2) { // e_3^dag q = (i q0, -i q1)
            a2[0] += SIG * q0i; a2[1] -= SIG * q0r;
            a3[0] -= SIG * q1i; a3[1] += SIG * q1r;
        } else {                        // e_4^dag q = (q0, q1)
            a2[0] -= SIG * q0r; a2[1] -= SIG * q0i;
            a3[0] -= SIG * q1r; a3[1] -= SIG * q1i;
        }
    }
}

template <int P>
__device__ __forceinline__ void load_link(const typename Tr<P>::link_t *U, typename Tr<P>::real *u)
{
    if constexpr (P == DWF_F64) {
        const double2 *v = reinterpret_cast<const double2 *>(U);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 q = __ldg(v + k);
            u[2 * k] = q.x;
            u[2 * k + 1] = q.y;
        }
    } else if constexpr (P == DWF_F32) {
        const float2 *v = reinterpret_cast<const float2 *>(U);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float2 q = __ldg(v + k);
            u[2 * k] = q.x;
            u[2 * k + 1] = q.y;
        }
    } else {
        const __half2 *v = reinterpret_cast<const __half2 *>(U);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float2 q = __half22float2(__ldg(v + k));
            u[2 * k] = q.x;
            u[2 * k + 1] = q.y;
        }
    }
}

// q[sp][a] = sum_b U[a][b] h[sp][b]
template <typename real>
__device__ __forceinline__ void su3_mul(const real *u, const real *h, real *q)
{
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            real re = 0, im = 0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const real ur = u[(a * 3 + b) * 2], ui = u[(a * 3 + b) * 2 + 1];
                const real hr = h[(sp * 3 + b) * 2], hi = h[(sp * 3 + b) * 2 + 1];
                re += ur * hr - ui * hi;
                im += ur * hi + ui * hr;
            }
            q[(sp * 3 + a) * 2] = re;
            q[(sp * 3 + a) * 2 + 1] = im;
        }
}

template <int P, bool DAG, int D>
__device__ __forceinline__ void hop_dir(typename Tr<P>::real *acc, const FieldRef &in, int nb, int s, int Ls,
                                        const typename Tr<P>::link_t *U)
{
    typedef typename Tr<P>::real real;
    constexpr int MU = D & 3;
    constexpr int SIG = (D < 4 ? 1 : -1) * (DAG ? -1 : 1);
    real psi[24], h[12], q[12], u[18];
    ld_field<P, true>(in, (size_t)nb, s, Ls, psi);
    load_link<P>(U + D * 18, u);
    project<real, MU, SIG>(psi, h);
    su3_mul<real>(u, h, q);
    reconstruct<real, MU, SIG>(acc, q);
}

// o[k] += sum_t M[chi(k)][s][t] tile[t][k], M stored transposed [chi][t][s]
template <typename real>
__device__ __forceinline__ void mix_tile(const real *M, const real *tile, int s, int Ls, real *o)
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

template <typename real>
__device__ __forceinline__ void put_tile(real *tile, int s, const real *v)
{
    real *dst = tile + s * 24;
#pragma unroll
    for (int k = 0; k < 24; ++k) dst[k] = v[k];
}

template <int P, bool DAG>
__global__ void __launch_bounds__(256) hop_kernel(const HopArgs a)
{
    typedef typename Tr<P>::real real;
    typedef typename Tr<P>::link_t link_t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls;
    const int s = threadIdx.x;
    const int j = threadIdx.y;
    const int SB = blockDim.y;
    const int site = blockIdx.x * SB + j;
    const bool active = site < a.Vh;
    const int tstride = Ls * 24 + (sizeof(real) == 8 ? 2 : 4);
    real *tile = reinterpret_cast<real *>(smem_raw);
    real *mtx = tile + SB * tstride;
    const int msz = 2 * Ls * Ls;
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int k = tid; k < msz; k += nt) {
        mtx[k] = reinterpret_cast<const real *>(a.post)[k];
        if (a.ymode == 2) mtx[msz + k] = reinterpret_cast<const real *>(a.ymat)[k];
        if (a.zmat) mtx[2 * msz + k] = reinterpret_cast<const real *>(a.zmat)[k];
    }

    real acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0;
    if (active) {
        const int *nb = a.nbr + (size_t)site * 8;
        const link_t *U = reinterpret_cast<const link_t *>(a.gauge) + (size_t)site * 8 * 18;
        int n[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) n[d] = __ldg(nb + d);
        hop_dir<P, DAG, 0>(acc, a.in, n[0], s, Ls, U);
        hop_dir<P, DAG, 1>(acc, a.in, n[1], s, Ls, U);
        hop_dir<P, DAG, 2>(acc, a.in, n[2], s, Ls, U);
        hop_dir<P, DAG, 3>(acc, a.in, n[3], s, Ls, U);
        hop_dir<P, DAG, 4>(acc, a.in, n[4], s, Ls, U);
        hop_dir<P, DAG, 5>(acc, a.in, n[5], s, Ls, U);
        hop_dir<P, DAG, 6>(acc, a.in, n[6], s, Ls, U);
        hop_dir<P, DAG, 7>(acc, a.in, n[7], s, Ls, U);
        put_tile(tile + j * tstride, s, acc);
    }
    __syncthreads();

    real o[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) o[k] = 0;
    if (active) mix_tile(mtx, tile + j * tstride, s, Ls, o);

    if (a.ymode == 1 && active) {
        real y[24];
        ld_field<P, false>(a.y, (size_t)site, s, Ls, y);
#pragma unroll
        for (int k = 0; k < 24; ++k) o[k] += y[k];
    } else if (a.ymode == 2) {
        __syncthreads();
        if (active) {
            real y[24];
            ld_field<P, false>(a.y, (size_t)site, s, Ls, y);
            put_tile(tile + j * tstride, s, y);
        }
        __syncthreads();
        if (active) mix_tile(mtx + msz, tile + j * tstride, s, Ls, o);
    }

    if (a.rin.v && active) {
        real r[24];
        ld_field<P, false>(a.rin, (size_t)site, s, Ls, r);
        const real al = (real)(*a.ralpha);
#pragma unroll
        for (int k = 0; k < 24; ++k) o[k] = r[k] - al * o[k];
        if (a.xacc) {
            typedef typename Tr<P>::xs_t xs_t;
            constexpr int XP = (P == DWF_F64) ? DWF_F64 : DWF_F32;
            FieldRef xf;
            xf.v = a.xacc;
            real x[24], dx[24];
            ld_field<XP, false>(xf, (size_t)site, s, Ls, x);
            ld_field<P, false>(a.xdir, (size_t)site, s, Ls, dx);
            const real xa = (real)(*a.xalpha);
#pragma unroll
            for (int k = 0; k < 24; ++k) x[k] += xa * dx[k];
            st_field<XP>(xf, (size_t)site, s, Ls, x);
            (void)sizeof(xs_t);
        }
    }

    double nrm = 0;
    if (active && a.red.op != RED_NONE) {
#pragma unroll
        for (int k = 0; k < 24; ++k) nrm += (double)o[k] * (double)o[k];
    }

    if (a.zmat) {
        __syncthreads();
        if (active) put_tile(tile + j * tstride, s, o);
        __syncthreads();
        real z[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) z[k] = 0;
        if (active) mix_tile(mtx + 2 * msz, tile + j * tstride, s, Ls, z);
        if (active) st_field<P>(a.out, (size_t)site, s, Ls, z);
    } else if (active) {
        st_field<P>(a.out, (size_t)site, s, Ls, o);
    }

    if (a.red.op != RED_NONE) grid_reduce(nrm, a.red);
}

template <int P>
size_t hop_smem(int Ls, int SB)
{
    typedef typename Tr<P>::real real;
    const int tstride = Ls * 24 + (sizeof(real) == 8 ? 2 : 4);
    return (size_t)(SB * tstride + 3 * 2 * Ls * Ls) * sizeof(real);
}

template <int P, bool DAG>
cudaError_t launch_hop_t(const HopArgs &a, int SB, cudaStream_t st)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(hop_kernel<P, DAG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             160 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.Ls * SB > 256) SB = 256 / a.Ls;
    if (SB < 1) SB = 1;
    dim3 block(a.Ls, SB);
    dim3 grid((a.Vh + SB - 1) / SB);
    hop_kernel<P, DAG><<<grid, block, hop_smem<P>(a.Ls, SB), st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_hop(int prec, bool dag, const HopArgs &a, int SB, cudaStream_t st)
{
    switch (prec) {
    case DWF_F64: return dag ? launch_hop_t<DWF_F64, true>(a, SB, st) : launch_hop_t<DWF_F64, false>(a, SB, st);
    case DWF_F32: return dag ? launch_hop_t<DWF_F32, true>(a, SB, st) : launch_hop_t<DWF_F32, false>(a, SB, st);
    case DWF_F16: return dag ? launch_hop_t<DWF_F16, true>(a, SB, st) : launch_hop_t<DWF_F16, false>(a, SB, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dwf
