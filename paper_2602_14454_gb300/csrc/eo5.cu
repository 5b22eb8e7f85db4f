// 5D even-odd preconditioning (the alternative split of Sec. 2.3) and the
// failure-detection probe of the bounded waits.
//
// 5D split: sites
// (x, s) even when x + y + z + t + s is even.  For the standard form with
// c_s = 0 and even Ls, D_ee and D_oo are the on-site diagonal a0_s =
// b_s (4 - M0) + 1, so the Schur complement 1 - D_ee^-1 D_eo D_oo^-1 D_oe is
// two applications of the whole 5D matrix between parity masks: the part of
// D5 that maps one parity to the other is D5 itself with the on-site term
// masked away.  Fields are full 5D fields in the canonical layout
// [s][site][24 reals] (site lexicographic, x fastest), the sites of the other
// parity zero.
#include "dwf_internal.h"

namespace dwf {
namespace {

constexpr int kThreads = 256;

struct E5Dims {
    int d[4];
};

// per (s, site): keep the sites of one parity and combine
//   mode 0: out = A (even)            mode 1: out = A / a0 (odd)
//   mode 2: out = A - C / a0 (even)   mode 3: out = A / a0 (even)
//   mode 4: out = A - C (even)        mode 5: out = (A - C) / a0 (even)
//   mode 6: out = (A - C) / a0 (odd)
// the other parity's sites get zeros
__global__ void eo5_kernel(int mode, const double *A, const double *C, double *out, E5Dims D, int V, int Ls,
                           const double *inv_a0)
{
    const size_t n = (size_t)Ls * V;
    const int want = (mode == 1 || mode == 6) ? 1 : 0;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(idx / V), lex = (int)(idx % V);
        int r = lex;
        const int x = r % D.d[0];
        r /= D.d[0];
        const int y = r % D.d[1];
        r /= D.d[1];
        const int z = r % D.d[2];
        const int t = r / D.d[2];
        const int par = (x + y + z + t + s) & 1;
        const double ia = inv_a0[s];
        const double *a = A + idx * 24;
        const double *c = C ? C + idx * 24 : nullptr;
        double *o = out + idx * 24;
        if (par != want) {
            for (int k = 0; k < 24; ++k) o[k] = 0.0;
            continue;
        }
        for (int k = 0; k < 24; ++k) {
            double v;
            switch (mode) {
            case 0: v = a[k]; break;
            case 1: case 3: v = a[k] * ia; break;
            case 2: v = a[k] - c[k] * ia; break;
            case 4: v = a[k] - c[k]; break;
            default: v = (a[k] - c[k]) * ia; break;
            }
            o[k] = v;
        }
    }
}

// a single-thread wait on a flag nothing sets, bounded by %globaltimer
__global__ void wait_probe_kernel(const volatile int *flag, unsigned long long limit_ns, int *err)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (*flag == 0) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
            atomicOr(err, 1);
            return;
        }
    }
}

}  // namespace

cudaError_t launch_wait_probe(const int *flag, unsigned long long limit_ns, int *err, cudaStream_t st)
{
    wait_probe_kernel<<<1, 32, 0, st>>>(flag, limit_ns, err);
    return cudaGetLastError();
}

cudaError_t launch_eo5(int mode, const void *A, const void *C, void *out, const int dims[4], int V, int Ls,
                       const double *inv_a0, cudaStream_t st)
{
    E5Dims D;
    for (int k = 0; k < 4; ++k) D.d[k] = dims[k];
    size_t g = ((size_t)Ls * V + kThreads - 1) / kThreads;
    if (g > 65535u * 4u) g = 65535u * 4u;
    eo5_kernel<<<(unsigned)g, kThreads, 0, st>>>(mode, (const double *)A, (const double *)C, (double *)out, D, V, Ls,
                                                   inv_a0);
    return cudaGetLastError();
}

}  // namespace dwf
