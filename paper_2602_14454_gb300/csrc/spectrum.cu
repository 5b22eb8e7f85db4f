// Extremal eigenvalues of D^dag D, D the even-odd matrix of Sec. 2.3 in the
// handle's form (standard, or Neff's with its alpha).  Sec. 3.2 (condition
// number) defines the condition number as the ratio of the largest to the
// smallest eigenvalue of D^dag D and studies it against alpha; it measures
// both with the implicitly restarted Lanczos algorithm in double precision.
// Here: the Lanczos recurrence (Lanczos 1950) in FP64 on the device, without
// restarts or reorthogonalisation (loss of orthogonality only duplicates
// converged Ritz values, the extremal ones still converge), the extremal
// eigenvalues of the tridiagonal matrix by Sturm-sequence bisection on the host.
#include <cmath>
#include <vector>

#include "fields.cuh"

using namespace dwf;

namespace dwf_detail {
HopArgs hop_args(dwf_ctx *h, int prec, int out_par, FieldRef in, FieldRef out, int post);
cudaError_t hop(dwf_ctx *h, int prec, bool dag, const HopArgs &a, cudaStream_t st);
cudaError_t mix(dwf_ctx *h, int prec, FieldRef in, FieldRef out, int id, cudaStream_t st);
RedArgs red(dwf_ctx *h, int op, CgScalars *scal);
}  // namespace dwf_detail
using namespace dwf_detail;

#define CK(call)                                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return dwf_cuda_error(e_, #call);      \
    } while (0)

namespace {

constexpr int kLzThreads = 256;

int lz_grid(size_t n)
{
    size_t g = (n + kLzThreads - 1) / kLzThreads;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

// The FP64 even fields are 24 reals per (site, s); every operation below is
// the real inner product / linear combination of those reals (the real part
// of the complex inner product: D^dag D is Hermitian, so its Rayleigh quotients
// are real and the real symmetric form has the same eigenvalues).
__global__ void __launch_bounds__(kLzThreads) lz_dot_kernel(const double2 *x, const double2 *y, size_t n2, RedArgs r)
{
    double s = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = x[i], b = y[i];
        s = fma(a.x, b.x, fma(a.y, b.y, s));
    }
    grid_reduce(s, r);
}

// y = a x + b y (y not read when b = 0)
__global__ void __launch_bounds__(kLzThreads) lz_axpby_kernel(double a, const double2 *x, double b, double2 *y,
                                                             size_t n2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        const double2 u = x[i];
        const double2 w = b != 0.0 ? y[i] : make_double2(0.0, 0.0);
        y[i] = make_double2(fma(a, u.x, b * w.x), fma(a, u.y, b * w.y));
    }
}

// start vector: uniform reals in [-1, 1) from the SplitMix64 generator
// (Steele, Lea and Flood 2014) at counter seed + index
__device__ __forceinline__ double lz_uniform(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

__global__ void __launch_bounds__(kLzThreads) lz_random_kernel(double2 *x, size_t n2, unsigned long long seed)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x)
        x[i] = make_double2(lz_uniform(seed + 2 * i), lz_uniform(seed + 2 * i + 1));
}

// out = D^dag D x on FP64 even fields (the hops of one inner CG iteration)
int normal_apply_f64(dwf_ctx *h, FieldRef x, FieldRef out, cudaStream_t st)
{
    const int P = DWF_F64;
    cudaError_t e = cudaSuccess;
    FieldRef ph = h->field("lz_ph", P, &e), t = h->field("lz_t", P, &e);
    FieldRef wh = h->field("lz_wh", P, &e), u = h->field("lz_u", P, &e);
    if (!ph.v || !t.v || !wh.v || !u.v) return dwf_cuda_error(e, "workspace");
    CK(mix(h, P, x, ph, MAT_P, st));
    HopArgs a1 = hop_args(h, P, 1, ph, t, MAT_M);
    CK(hop(h, P, false, a1, st));
    HopArgs a2 = hop_args(h, P, 0, t, wh, MAT_NQ4);
    a2.y = x;
    a2.ymode = 1;
    a2.zmat = h->mat(P, MAT_QT);
    CK(hop(h, P, false, a2, st));
    HopArgs a3 = hop_args(h, P, 1, wh, u, MAT_MT);
    CK(hop(h, P, true, a3, st));
    HopArgs a4 = hop_args(h, P, 0, u, out, MAT_NPT4);
    a4.y = wh;
    a4.ymode = 2;
    a4.ymat = h->mat(P, MAT_RA5T);
    CK(hop(h, P, true, a4, st));
    return DWF_OK;
}

// out = D x, D the even-odd matrix (as dwf_apply with DWF_OP_EO_PREC), FP64
int eo_apply_f64(dwf_ctx *h, FieldRef x, FieldRef out, cudaStream_t st)
{
    const int P = DWF_F64;
    cudaError_t e = cudaSuccess;
    FieldRef ph = h->field("lz_ph", P, &e), t = h->field("lz_t", P, &e);
    if (!ph.v || !t.v) return dwf_cuda_error(e, "workspace");
    CK(mix(h, P, x, ph, MAT_P, st));
    HopArgs a1 = hop_args(h, P, 1, ph, t, MAT_M);
    CK(hop(h, P, false, a1, st));
    HopArgs a2 = hop_args(h, P, 0, t, out, MAT_NQ4);
    a2.y = x;
    a2.ymode = 1;
    CK(hop(h, P, false, a2, st));
    return DWF_OK;
}

// out = D^dag x, FP64
int eo_dag_apply_f64(dwf_ctx *h, FieldRef x, FieldRef out, cudaStream_t st)
{
    const int P = DWF_F64;
    cudaError_t e = cudaSuccess;
    FieldRef wh = h->field("lz_wh", P, &e), u = h->field("lz_u", P, &e);
    if (!wh.v || !u.v) return dwf_cuda_error(e, "workspace");
    CK(mix(h, P, x, wh, MAT_QT, st));
    HopArgs a1 = hop_args(h, P, 1, wh, u, MAT_MT);
    CK(hop(h, P, true, a1, st));
    HopArgs a2 = hop_args(h, P, 0, u, out, MAT_NPT4);
    a2.y = x;
    a2.ymode = 1;
    CK(hop(h, P, true, a2, st));
    return DWF_OK;
}

// out = D'^dag D' x for the second even-odd form of Sec. 2.3,
// eq. (another_even-odd_linear_equation): D' = 1 - D_eo D_oo^-1 D_oe D_ee^-1 =
// D_ee D D_ee^-1 with D_ee = A5 R and D_ee^-1 = Q, so that
// D'^dag D' = Q^T D^dag (A5 R)^T (A5 R) D Q (the mixings are real per chirality)
int alt_normal_apply_f64(dwf_ctx *h, FieldRef x, FieldRef out, cudaStream_t st)
{
    const int P = DWF_F64;
    cudaError_t e = cudaSuccess;
    FieldRef a = h->field("lz_a", P, &e), b = h->field("lz_b", P, &e);
    if (!a.v || !b.v) return dwf_cuda_error(e, "workspace");
    int rc;
    CK(mix(h, P, x, a, MAT_Q, st));
    if ((rc = eo_apply_f64(h, a, b, st))) return rc;
    CK(mix(h, P, b, a, MAT_A5R, st));
    CK(mix(h, P, a, b, MAT_RA5T, st));
    if ((rc = eo_dag_apply_f64(h, b, a, st))) return rc;
    CK(mix(h, P, a, out, MAT_QT, st));
    return DWF_OK;
}

// number of eigenvalues of the symmetric tridiagonal matrix (diagonal a,
// off-diagonal b[i] between rows i and i + 1) below x: the sign changes of
// the Sturm sequence, i.e. the negative pivots of the LDL^T factorisation of T - x
int sturm_count(const std::vector<double> &a, const std::vector<double> &b, double x)
{
    const size_t m = a.size();
    int cnt = 0;
    double d = 1.0;
    for (size_t i = 0; i < m; ++i) {
        const double off = i ? b[i - 1] * b[i - 1] : 0.0;
        d = (a[i] - x) - (i ? off / d : 0.0);
        if (d == 0.0) d = -1e-300;   // a zero pivot counts as negative (x is an eigenvalue)
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// k-th smallest eigenvalue (k = 1..m) by bisection on the Gershgorin interval
double tridiag_eig(const std::vector<double> &a, const std::vector<double> &b, int k)
{
    const size_t m = a.size();
    double lo = a[0], hi = a[0];
    for (size_t i = 0; i < m; ++i) {
        const double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
        lo = std::fmin(lo, a[i] - r);
        hi = std::fmax(hi, a[i] + r);
    }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(a, b, mid) >= k)
            hi = mid;
        else
            lo = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

extern "C" int dwf_spectrum_bounds(dwf_handle h, int eo_form, int max_steps, double rtol, unsigned long long seed,
                                   double *lambda_min, double *lambda_max, int *steps, void *stream)
{
    if (!h || (eo_form != 0 && eo_form != 1) || max_steps < 2 || !(rtol > 0) || !lambda_min || !lambda_max)
        return dwf_set_error(DWF_EINVAL, "bad argument");
    if (h->slab) return dwf_set_error(DWF_EINVAL, "a slab handle applies its operator through dwf_slab_apply_eo");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    FieldRef v0 = h->field("lz_v0", DWF_F64, &e), v1 = h->field("lz_v1", DWF_F64, &e);
    FieldRef w = h->field("lz_w", DWF_F64, &e);
    if (!v0.v || !v1.v || !w.v) return dwf_cuda_error(e, "workspace");
    const size_t n2 = (size_t)h->Vh * h->Ls * 12;   // double2 per field
    const int g = lz_grid(n2);
    CgScalars *sc = h->scal + 5;
    CgScalars hs;
    auto dot = [&](FieldRef x, FieldRef y, double &out) -> int {
        lz_dot_kernel<<<g, kLzThreads, 0, st>>>((const double2 *)x.v, (const double2 *)y.v, n2,
                                                red(h, RED_STORE, sc));
        CK(cudaGetLastError());
        h->launches += 1;
        CK(cudaMemcpyAsync(&hs, sc, sizeof hs, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        out = hs.last;
        if (!std::isfinite(out)) return dwf_set_error(DWF_ENONFINITE, "non-finite value in the Lanczos recurrence");
        return DWF_OK;
    };
    auto axpby = [&](double a, FieldRef x, double b, FieldRef y) -> int {
        lz_axpby_kernel<<<g, kLzThreads, 0, st>>>(a, (const double2 *)x.v, b, (double2 *)y.v, n2);
        CK(cudaGetLastError());
        h->launches += 1;
        return DWF_OK;
    };
    int rc;
    // v1 = random / |random|
    lz_random_kernel<<<g, kLzThreads, 0, st>>>((double2 *)v1.v, n2, seed * 0x100000001b3ULL);
    CK(cudaGetLastError());
    h->launches += 1;
    double nn;
    if ((rc = dot(v1, v1, nn))) return rc;
    if ((rc = axpby(1.0 / std::sqrt(nn), v1, 0.0, v1))) return rc;
    std::vector<double> al, be;   // T: diagonal alpha_j, off-diagonal beta_{j+1}
    double lmin = 0, lmax = 0, pmin = 0, pmax = 0;
    int k = 0;
    for (k = 0; k < max_steps; ++k) {
        // w = A v1 - beta_k v0 ; alpha = (w, v1) ; w -= alpha v1 ; beta = |w|
        if ((rc = eo_form ? alt_normal_apply_f64(h, v1, w, st) : normal_apply_f64(h, v1, w, st))) return rc;
        if (k > 0 && (rc = axpby(-be.back(), v0, 1.0, w))) return rc;
        double a;
        if ((rc = dot(w, v1, a))) return rc;
        if ((rc = axpby(-a, v1, 1.0, w))) return rc;
        double b2;
        if ((rc = dot(w, w, b2))) return rc;
        al.push_back(a);
        const double b = std::sqrt(b2);
        const bool last = k + 1 == max_steps || !(b > 1e-14 * std::fabs(a));
        if ((k + 1) % 10 == 0 || last) {
            lmin = tridiag_eig(al, be, 1);
            lmax = tridiag_eig(al, be, (int)al.size());
            const bool conv = k >= 19 && std::fabs(lmin - pmin) <= rtol * std::fabs(lmin) &&
                              std::fabs(lmax - pmax) <= rtol * std::fabs(lmax);
            pmin = lmin;
            pmax = lmax;
            if (conv || last) {
                ++k;
                break;
            }
        }
        be.push_back(b);
        // v0 = v1 ; v1 = w / beta  (the buffers rotate: v0 <- v1, v1 <- w, w <- old v0)
        FieldRef tmp = v0;
        v0 = v1;
        v1 = w;
        w = tmp;
        if ((rc = axpby(1.0 / b, v1, 0.0, v1))) return rc;
    }
    *lambda_min = lmin;
    *lambda_max = lmax;
    if (steps) *steps = k;
    return DWF_OK;
}
