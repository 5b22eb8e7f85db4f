// Spin projection, SU(3) transport and reconstruction of one Wilson hop on
// spin-paired fields (layout in fields.cuh), shared by the stencil kernels.
//
// Chiral basis: gamma_mu = [[0, e_mu], [e_mu^dag, 0]], e_k = -i sigma_k,
// e_4 = 1, so (1 - sig gamma_mu) psi = [h ; -sig e_mu^dag h] with the half
// spinor h = psi_u - sig e_mu psi_l: only h is multiplied by the link.  h is
// held as spin pairs Hx[a] = (h0.re, h1.re), Hy[a] = (h0.im, h1.im), so the
// SU(3) product is 4 packed FMAs per (a, b) for both spins at once.
#pragma once

#include "fields.cuh"

namespace dwf {
namespace {

// h = P^{(mu, sig)} psi, spin-paired (see fields.cuh for the pair layout)
template <int MU, int SIG, typename T2>
__device__ __forceinline__ void project(const T2 *v, T2 *Hx, T2 *Hy)
{
    typedef typename PairReal<T2>::R R;
    constexpr R s = (R)SIG;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T2 XU = v[4 * a], XL = v[4 * a + 1], YU = v[4 * a + 2], YL = v[4 * a + 3];
        if constexpr (MU == 3) {        // h0 = p0 - s p2, h1 = p1 - s p3
            Hx[a] = p_fma(p_splat(-s), XL, XU);
            Hy[a] = p_fma(p_splat(-s), YL, YU);
        } else if constexpr (MU == 2) { // h0 = p0 + s i p2, h1 = p1 - s i p3
            Hx[a] = p_fma(p_make(-s, s), YL, XU);
            Hy[a] = p_fma(p_make(s, -s), XL, YU);
        } else if constexpr (MU == 1) { // h0 = p0 + s p3, h1 = p1 - s p2
            Hx[a] = p_make(XU.x + s * XL.y, XU.y - s * XL.x);
            Hy[a] = p_make(YU.x + s * YL.y, YU.y - s * YL.x);
        } else {                        // h0 = p0 + s i p3, h1 = p1 + s i p2
            Hx[a] = p_make(XU.x - s * YL.y, XU.y - s * YL.x);
            Hy[a] = p_make(YU.x + s * XL.y, YU.y + s * XL.x);
        }
    }
}

// acc += [q ; -sig e_mu^dag q]
template <int MU, int SIG, typename T2>
__device__ __forceinline__ void reconstruct(T2 *acc, const T2 *Qx, const T2 *Qy)
{
    typedef typename PairReal<T2>::R R;
    constexpr R s = (R)SIG;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T2 &XU = acc[4 * a], &XL = acc[4 * a + 1], &YU = acc[4 * a + 2], &YL = acc[4 * a + 3];
        XU = p_add(XU, Qx[a]);
        YU = p_add(YU, Qy[a]);
        if constexpr (MU == 3) {        // lower = -s (q0, q1)
            XL = p_fma(p_splat(-s), Qx[a], XL);
            YL = p_fma(p_splat(-s), Qy[a], YL);
        } else if constexpr (MU == 2) { // p2 += -s i q0, p3 += s i q1
            XL = p_fma(p_make(s, -s), Qy[a], XL);
            YL = p_fma(p_make(-s, s), Qx[a], YL);
        } else if constexpr (MU == 1) { // p2 += -s q1, p3 += s q0
            XL = p_make(XL.x - s * Qx[a].y, XL.y + s * Qx[a].x);
            YL = p_make(YL.x - s * Qy[a].y, YL.y + s * Qy[a].x);
        } else {                        // p2 += -s i q1, p3 += -s i q0
            XL = p_make(XL.x + s * Qy[a].y, XL.y + s * Qy[a].x);
            YL = p_make(YL.x - s * Qx[a].y, YL.y - s * Qx[a].x);
        }
    }
}

// link (row-major 3x3 complex) -> u[9] complex pairs (re, im); global (RO) or shared
template <int P, bool GLOBAL, typename T2>
__device__ __forceinline__ void load_link(const typename Tr<P>::link_t *U, T2 *u)
{
    if constexpr (P == DWF_F64) {
        const double2 *v = reinterpret_cast<const double2 *>(U);
#pragma unroll
        for (int k = 0; k < 9; ++k) u[k] = GLOBAL ? __ldg(v + k) : v[k];
    } else if constexpr (P == DWF_F32) {
        const float2 *v = reinterpret_cast<const float2 *>(U);
#pragma unroll
        for (int k = 0; k < 9; ++k) u[k] = GLOBAL ? __ldg(v + k) : v[k];
    } else {
        const __half2 *v = reinterpret_cast<const __half2 *>(U);
#pragma unroll
        for (int k = 0; k < 9; ++k) u[k] = __half22float2(GLOBAL ? __ldg(v + k) : v[k]);
    }
}

// Q = U H for both spins: Qx[a] = sum_b ur Hx[b] - ui Hy[b], Qy[a] = sum_b ur Hy[b] + ui Hx[b]
template <typename T2>
__device__ __forceinline__ void su3_pairs(const T2 *u, const T2 *Hx, const T2 *Hy, T2 *Qx, T2 *Qy)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T2 qx = p_zero(Hx[0]), qy = p_zero(Hx[0]);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T2 ur = p_splat(u[a * 3 + b].x), ui = p_splat(u[a * 3 + b].y);
            const T2 nui = p_splat(-u[a * 3 + b].y);
            qx = p_fma(ur, Hx[b], qx);
            qx = p_fma(nui, Hy[b], qx);
            qy = p_fma(ur, Hy[b], qy);
            qy = p_fma(ui, Hx[b], qy);
        }
        Qx[a] = qx;
        Qy[a] = qy;
    }
}

template <int MU, int SIG, typename T2>
__device__ __forceinline__ void hop_one(T2 *acc, const T2 *u, const T2 *v)
{
    T2 Hx[3], Hy[3], Qx[3], Qy[3];
    project<MU, SIG>(v, Hx, Hy);
    su3_pairs(u, Hx, Hy, Qx, Qy);
    reconstruct<MU, SIG>(acc, Qx, Qy);
}

// ---------------------------------------------- FP16 arithmetic (half2 pairs)
// The same projection on raw FP16 pairs (no conversion of the stored spinor):
// h = psi_u - sig e_mu psi_l in half2.  Inputs are normalised per (site, s)
// (|values| <= 1), so h stays within [-2, 2].
template <int MU, int SIG>
__device__ __forceinline__ void project_h2(const __half2 *v, __half2 *Hx, __half2 *Hy)
{
    const __half s = __float2half((float)SIG), ms = __float2half((float)-SIG);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const __half2 XU = v[4 * a], XL = v[4 * a + 1], YU = v[4 * a + 2], YL = v[4 * a + 3];
        if constexpr (MU == 3) {        // h0 = p0 - s p2, h1 = p1 - s p3
            Hx[a] = __hfma2(__halves2half2(ms, ms), XL, XU);
            Hy[a] = __hfma2(__halves2half2(ms, ms), YL, YU);
        } else if constexpr (MU == 2) { // h0 = p0 + s i p2, h1 = p1 - s i p3
            Hx[a] = __hfma2(__halves2half2(ms, s), YL, XU);
            Hy[a] = __hfma2(__halves2half2(s, ms), XL, YU);
        } else if constexpr (MU == 1) { // h0 = p0 + s p3, h1 = p1 - s p2
            Hx[a] = __hfma2(__halves2half2(s, ms), __lowhigh2highlow(XL), XU);
            Hy[a] = __hfma2(__halves2half2(s, ms), __lowhigh2highlow(YL), YU);
        } else {                        // h0 = p0 + s i p3, h1 = p1 + s i p2
            Hx[a] = __hfma2(__halves2half2(ms, ms), __lowhigh2highlow(YL), XU);
            Hy[a] = __hfma2(__halves2half2(s, s), __lowhigh2highlow(XL), YU);
        }
    }
}

}  // namespace
}  // namespace dwf
