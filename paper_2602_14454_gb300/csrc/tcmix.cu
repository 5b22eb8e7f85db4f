// Fifth-direction mixing on the 5th-generation tensor cores (tcgen05, TMEM).
//
// out(site, s) = sum_t M_chi[s][t] in(site, t), one real Ls x Ls matrix per
// chirality (the per-chirality blocks of the fifth-direction factors of
// eq. domainwall_general / domainwall_neff and of the even-odd algebra), for
// every site of an even-odd half field: a batched GEMM.  Per tile of 16 sites
// the field is the A operand, rows r = (site, colour, re/im, spin) (24 per
// site, 384 per tile = three M = 128 blocks) and K = t; the B operand holds
// both chiralities side by side, B[n][t] = M_+[n][t] for n < Lsp and
// M_-[n - Lsp][t] beyond (Lsp = Ls rounded up to 8), so that one product
// D[r][n] = sum_t A[r][t] B[n][t] serves both and each row keeps the half of
// its own chirality (spins 0, 1: P_+; spins 2, 3: P_-).
//
// Precision: TF32 operands keep 10 mantissa bits, so each operand is split
// into two TF32 terms, x = x_hi + x_lo, and D = A_hi B_hi + A_hi B_lo +
// A_lo B_hi (relative error ~2^-21, FP32 level), accumulated in FP32 in TMEM.
//
// Data path per tile (persistent CTAs of 128 threads, four per SM):
//   16-byte coalesced loads of the tile (contiguous in the field layout) ->
//   split -> shared memory in the canonical no-swizzle K-major layout (8-row x
//   16-byte core matrices, K-adjacent core matrices LBO bytes apart, 8-row
//   groups 128 bytes apart) -> one elected thread issues the 18 MMAs (3 M
//   blocks x K/8 steps x 3 products) into TMEM and commits them to an
//   mbarrier -> every warp reads its 32 TMEM lanes (tcgen05.ld) -> shared
//   memory in (site, s) order -> st_pairs (FP16: the per-(site, s) scale).
// Every wait on the mbarrier is bounded by %globaltimer (1 s); a wait that
// gives up sets the error flag, waits (bounded again) for the MMAs already
// issued, frees the TMEM and ends the CTA.
#include <cstdint>

#include "fields.cuh"
#include "tcgen05.cuh"

namespace dwf {
namespace {

constexpr int TC_SITES = 16;            // sites per tile
constexpr int TC_ROWS = TC_SITES * 24;  // A rows per tile (3 x 128)
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_A_LBO = (TC_ROWS / 8) * 128 + 16;   // padded: the K-groups start 4 banks apart

struct TcGeom {
    int Ls, Lsp, Kp, Np;     // Lsp = pad8(Ls) = K extent, Np = 2 Lsp = N
    uint32_t a_bytes;        // one A operand (hi or lo)
    uint32_t b_lbo, b_bytes; // B operand
    uint32_t tmem_cols;      // power of two >= 3 Np, >= 32
    size_t smem;             // dynamic shared memory
};

__host__ __device__ inline TcGeom tc_geom(int Ls)
{
    TcGeom g;
    g.Ls = Ls;
    g.Lsp = tc_pad8(Ls);
    g.Kp = g.Lsp;
    g.Np = 2 * g.Lsp;
    g.a_bytes = (uint32_t)(g.Kp / 4) * TC_A_LBO;
    g.b_lbo = (uint32_t)(g.Np / 8) * 128;
    g.b_bytes = (uint32_t)(g.Kp / 4) * g.b_lbo;
    uint32_t c = 32;
    while (c < (uint32_t)(3 * g.Np)) c *= 2;
    g.tmem_cols = c;
    // A hi, A lo, B hi, B lo, then 16 bytes for the mbarrier and the TMEM address
    g.smem = (size_t)2 * g.a_bytes + (size_t)2 * g.b_bytes + 16;
    return g;
}

template <int P>
__global__ void __launch_bounds__(TC_THREADS, 1) mix_tc_kernel(const MixArgs a, const TcGeom g)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *Ahi = smem_raw, *Alo = smem_raw + g.a_bytes;
    unsigned char *Bhi = Alo + g.a_bytes, *Blo = Bhi + g.b_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(Blo + g.b_bytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    float *stage = reinterpret_cast<float *>(Ahi);   // output staging, after the MMAs of a tile
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Ls = g.Ls, Lsp = g.Lsp, Kp = g.Kp, Np = g.Np;

    // zero A (padding rows and K columns stay zero) and build B = [M_+ | M_-] split in two TF32 terms
    for (uint32_t k = tid; k < 2 * g.a_bytes / 16; k += TC_THREADS)
        reinterpret_cast<uint4 *>(Ahi)[k] = make_uint4(0, 0, 0, 0);
    const float *Mt = reinterpret_cast<const float *>(a.mat);   // [chi][t][s] = M_chi[s][t]
    for (int e = tid; e < Np * Kp; e += TC_THREADS) {
        const int n = e / Kp, k = e - n * Kp;
        const int chi = n / Lsp, s = n - chi * Lsp;
        const float v = (s < Ls && k < Ls) ? Mt[(chi * Ls + k) * Ls + s] : 0.f;
        const float hi = tf32_hi(v);
        const uint32_t off = kmaj_off(n, k, g.b_lbo);
        *reinterpret_cast<float *>(Bhi + off) = hi;
        *reinterpret_cast<float *>(Blo + off) = tf32_hi(v - hi);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32addr(tslot)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32addr(bar)) : "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = *tslot;
    const uint32_t idesc = idesc_tf32(Np);
    const uint32_t sA_hi = smem_u32addr(Ahi), sA_lo = smem_u32addr(Alo);
    const uint32_t sB_hi = smem_u32addr(Bhi), sB_lo = smem_u32addr(Blo);
    const int ntiles = (a.Vh + TC_SITES - 1) / TC_SITES;
    bool failed = false;
    int issued = 0;   // tiles whose MMAs were committed

    for (int u = blockIdx.x; u < ntiles; u += gridDim.x) {
        const int site0 = u * TC_SITES;
        const int nsite = min(TC_SITES, a.Vh - site0);
        // 1. the tile, split, into A (rows of absent sites keep their zeros from the last tile: cleared below)
        if constexpr (P == DWF_F32) {
            const float4 *src = reinterpret_cast<const float4 *>(a.in.v) + (size_t)site0 * 6 * Ls;
            const int nvec = TC_SITES * 6 * Ls;
            for (int f = tid; f < nvec; f += TC_THREADS) {
                const int sl = f / (6 * Ls), r6 = f - sl * 6 * Ls, gg = r6 / Ls, s = r6 - gg * Ls;
                const float4 q = sl < nsite ? __ldg(src + f) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int sp = 0; sp < 4; ++sp) {
                    const uint32_t off = kmaj_off(sl * 24 + gg * 4 + sp, s, TC_A_LBO);
                    const float hi = tf32_hi(v[sp]);
                    *reinterpret_cast<float *>(Ahi + off) = hi;
                    *reinterpret_cast<float *>(Alo + off) = tf32_hi(v[sp] - hi);
                }
            }
        } else {
            const uint4 *src = reinterpret_cast<const uint4 *>(a.in.v) + (size_t)site0 * 3 * Ls;
            const int sst = (Ls + 3) & ~3;
            const int nvec = TC_SITES * 3 * Ls;
            for (int f = tid; f < nvec; f += TC_THREADS) {
                const int sl = f / (3 * Ls), r3 = f - sl * 3 * Ls, gg = r3 / Ls, s = r3 - gg * Ls;
                uint4 q = make_uint4(0, 0, 0, 0);
                float sc = 0.f;
                if (sl < nsite) {
                    q = __ldg(src + f);
                    sc = __ldg(a.in.scale + (size_t)(site0 + sl) * sst + s);
                }
                const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const float2 f2 = __half22float2(*reinterpret_cast<const __half2 *>(&w[h]));
                    // half2 h of vector gg: pair h of groups 2 gg (h < 2) and 2 gg + 1 (h >= 2)
                    const int grp = 2 * gg + (h >> 1), sp0 = (h & 1) * 2;
                    const float v2[2] = {f2.x * sc, f2.y * sc};
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const uint32_t off = kmaj_off(sl * 24 + grp * 4 + sp0 + e, s, TC_A_LBO);
                        const float hi = tf32_hi(v2[e]);
                        *reinterpret_cast<float *>(Ahi + off) = hi;
                        *reinterpret_cast<float *>(Alo + off) = tf32_hi(v2[e] - hi);
                    }
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // 2. the products (one thread), committed to the mbarrier
        if (tid == 0) {
            for (int mb = 0; mb < 3; ++mb) {
                const uint32_t d = tbase + (uint32_t)(mb * Np);
                int acc = 0;
                for (int ks = 0; ks < Kp / 8; ++ks) {
                    const uint32_t ao = (uint32_t)ks * 2 * TC_A_LBO + (uint32_t)mb * 16 * 128;
                    const uint32_t bo = (uint32_t)ks * 2 * g.b_lbo;
                    const uint64_t ah = smem_desc(sA_hi + ao, TC_A_LBO, 128), al = smem_desc(sA_lo + ao, TC_A_LBO, 128);
                    const uint64_t bh = smem_desc(sB_hi + bo, g.b_lbo, 128), bl = smem_desc(sB_lo + bo, g.b_lbo, 128);
                    mma_tf32(d, ah, bh, idesc, acc);
                    acc = 1;
                    mma_tf32(d, ah, bl, idesc, 1);
                    mma_tf32(d, al, bh, idesc, 1);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32addr(bar))
                         : "memory");
        }
        ++issued;
        if (!mbar_wait_bounded(smem_u32addr(bar), (uint32_t)((issued - 1) & 1), 1000000000ull)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // 3. D -> registers -> shared memory, (site, s) order: stage[((sl Ls + s) 6 + g) 4 + spin]
        for (int mb = 0; mb < 3; ++mb) {
            uint32_t r[32];
            const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(mb * Np);
            for (int c0 = 0; c0 < Np; c0 += 32) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const int row = mb * 128 + 32 * warp + lane;   // TMEM lane = A row
                const int sl = row / 24, rr = row - sl * 24, gg = rr >> 2, sp = rr & 3;
                const int chi = sp >> 1;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int n = c0 + c, s = n - chi * Lsp;
                    if (n / Lsp == chi && s < Ls) stage[((sl * Ls + s) * 6 + gg) * 4 + sp] = __uint_as_float(r[c]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        // 4. (site, s) pairs out
        for (int e = tid; e < nsite * Ls; e += TC_THREADS) {
            const int sl = e / Ls, s = e - sl * Ls;
            const float4 *q = reinterpret_cast<const float4 *>(stage) + (size_t)(sl * Ls + s) * 6;
            float2 v[12];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float4 w = q[k];
                v[2 * k] = make_float2(w.x, w.y);
                v[2 * k + 1] = make_float2(w.z, w.w);
            }
            st_pairs<P>(a.out, (size_t)(site0 + sl), s, Ls, v);
        }
        __syncthreads();   // the staging area becomes A again; every thread is done with it
        // the staging overwrote A_hi: its padding columns t = Ls .. Kp - 1 must be zero again
        // (the loads rewrite every column t < Ls of every row, absent sites with zeros)
        if (Kp != Ls)
            for (int e = tid; e < TC_ROWS * (Kp - Ls); e += TC_THREADS)
                *reinterpret_cast<float *>(Ahi + kmaj_off(e / (Kp - Ls), Ls + e % (Kp - Ls), TC_A_LBO)) = 0.f;
    }
    if (failed) {
        if (tid == 0 && a.err) atomicOr(a.err, 1);
        // let the committed MMAs finish before the TMEM is freed (bounded again)
        mbar_wait_bounded(smem_u32addr(bar), (uint32_t)((issued - 1) & 1), 1000000000ull);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(g.tmem_cols)
                     : "memory");
}

}  // namespace

// Tensor-core mixing for FP32 and FP16 fields, Ls <= 32.
cudaError_t launch_mix_tc(int prec, const MixArgs &a, cudaStream_t st)
{
    if (a.Ls < 1 || a.Ls > 32 || (prec != DWF_F32 && prec != DWF_F16)) return cudaErrorInvalidValue;
    const TcGeom g = tc_geom(a.Ls);
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // as many CTAs per SM as the tensor memory holds (512 columns)
    const int per_sm = (int)(512 / g.tmem_cols);
    const int ntiles = (a.Vh + TC_SITES - 1) / TC_SITES;
    int grid = nsm * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (prec == DWF_F32) {
        static unsigned long long optin = 0;
        if ((e = smem_optin(mix_tc_kernel<DWF_F32>, 200 * 1024, optin)) != cudaSuccess) return e;
        mix_tc_kernel<DWF_F32><<<grid, TC_THREADS, g.smem, st>>>(a, g);
    } else {
        static unsigned long long optin = 0;
        if ((e = smem_optin(mix_tc_kernel<DWF_F16>, 200 * 1024, optin)) != cudaSuccess) return e;
        mix_tc_kernel<DWF_F16><<<grid, TC_THREADS, g.smem, st>>>(a, g);
    }
    return cudaGetLastError();
}

}  // namespace dwf
