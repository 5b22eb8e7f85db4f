// C ABI: handle life cycle, link upload, operator application, 4D <-> 5D maps.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "dwf_internal.h"

using namespace dwf;

namespace dwf {
// mixing.cpp: the fifth-direction matrices with s-dependent coefficients
bool build_fifth_matrices_s(int Ls, double M0, double mf, const double *bs, const double *cs, int form, double alpha,
                            FifthMatrices &out, std::string &err);
}  // namespace dwf

namespace {
thread_local std::string g_last_error;

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
}  // namespace

int dwf_set_error(int status, const std::string &msg)
{
    g_last_error = msg;
    return status;
}

int dwf_cuda_error(cudaError_t e, const char *where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DWF_ENOMEM : DWF_ECUDA;
}

#define CK(call)                                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return dwf_cuda_error(e_, #call);      \
    } while (0)

// ------------------------------------------------------------- dwf_ctx
const void *dwf_ctx::mat(int prec, int id) const
{
    const size_t per = (size_t)2 * Ls * Ls;
    if (prec == DWF_F64) return (const double *)mats_dev[0] + per * id;
    return (const float *)mats_dev[1] + per * id;
}

int dwf_ctx::mix_mode(int prec) const
{
    const int m = mixmode[prec];
    if (m == 1) return fm.structured ? 1 : 0;
    if (m == 2) return prec == DWF_F64 ? 0 : 2;
    // default: the structured form in FP64, where the FP64 pipe bounds the hop
    // (measured 2014 us vs 2217 us at 16^3x32, Ls 16); dense elsewhere (in FP32 the
    // structured chains of the warp-autonomous hop are 3-4 % faster for K_a and K_c
    // at 32^3x64 but slower for the banded K_d and the CG update)
    if (m < 0 && prec == DWF_F64 && fm.structured) return 1;
    return 0;
}

const void *dwf_ctx::prog(int prec, int id) const
{
    if (prec == DWF_F64) return (const MixProg<double> *)progs_dev[0] + id;
    return (const MixProg<float> *)progs_dev[1] + id;
}

// MatId of a matrix pointer handed out by mat(); -1 if it is not one
static int mat_id_of(const dwf_ctx *h, int prec, const void *p)
{
    if (!p) return -1;
    const size_t per = (size_t)2 * h->Ls * h->Ls * (prec == DWF_F64 ? 8 : 4);
    const char *base = (const char *)h->mats_dev[prec == DWF_F64 ? 0 : 1];
    const ptrdiff_t off = (const char *)p - base;
    if (off < 0 || off % (ptrdiff_t)per) return -1;
    const int id = (int)(off / (ptrdiff_t)per);
    return id < MAT_COUNT ? id : -1;
}

const void *dwf_ctx::gauge_for(int prec, int out_par) const
{
    const size_t n = (size_t)Vh * 8 * 18 * out_par;
    if (prec == DWF_F64) return (const double *)gauge[0] + n;
    if (prec == DWF_F32) return (const float *)gauge[1] + n;
    return (const __half *)gauge[2] + n;
}

void *dwf_ctx::ws(const std::string &name, size_t need, cudaError_t *err)
{
    auto it = work.find(name);
    if (it != work.end() && it->second.second >= need) return it->second.first;
    if (it != work.end()) {
        cudaFree(it->second.first);
        bytes -= it->second.second;
        work.erase(it);
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (err) *err = e;
    if (e != cudaSuccess) return nullptr;
    work[name] = {p, need};
    bytes += need;
    return p;
}

FieldRef dwf_ctx::field(const std::string &name, int prec, cudaError_t *err)
{
    FieldRef f;
    const size_t fb = field_bytes(prec, Vh + ghost, Ls);   // a slab's fields carry its ghost faces
    const size_t sb = scale_bytes(prec, Vh + ghost, Ls);
    const size_t off = (fb + 255) & ~(size_t)255;
    char *p = (char *)ws(name + "#" + std::to_string(prec), off + sb, err);
    if (!p) return f;
    f.v = p;
    f.scale = sb ? (float *)(p + off) : nullptr;
    return f;
}

// --------------------------------------------------------------- helpers
namespace dwf_detail {

// Columns of z-planes for the hop's sweep order (HopArgs::zblock): index order
// unless dwf_set_sweep chose columns.  Measured at 32^3x64, Ls 16 (FP32 variant 9):
// columns of 8 z-planes cut the hop's DRAM reads from 5.11 to 4.02 GB per launch but
// made it 2-5 % slower, since the kernel is bound by the SMs' load/store path, not by
// DRAM; the FP16 direct hop lost 4.6 %.
static int sweep_zblock(const dwf_ctx *h, int prec)
{
    return h->sweep_zb[prec] > 0 ? h->sweep_zb[prec] : 0;
}

// The automatic choice of dwf_set_sweep(h, prec, -2): the largest divisor Bz of Lz
// whose column band of Bz z-planes (input and output spinors of one parity and their
// links) stays within 16 MiB, so that the 2 Bz planes read between a site's two
// t-neighbour reads fit in L2 with room to spare; 0 (index order) while a whole
// t-slice fits.  Runs of Bz A sites are kept multiples of 32 so that no hop tile
// straddles two of them.
static int sweep_zblock_auto(const dwf_ctx *h, int prec)
{
    const long long A = (long long)(h->dims[0] / 2) * h->dims[1];
    const long long w = prec == DWF_F64 ? 8 : prec == DWF_F32 ? 4 : 2;
    const long long plane = A * ((long long)h->Ls * 24 * w * 2 + 8 * 18 * w);
    const long long budget = 16ll << 20;
    if (plane * h->dims[2] <= budget) return 0;
    for (int bz = h->dims[2] - 1; bz >= 1; --bz)
        if (h->dims[2] % bz == 0 && bz * plane <= budget && (bz * A) % 32 == 0) return bz;
    return 0;
}

HopArgs hop_args(dwf_ctx *h, int prec, int out_par, FieldRef in, FieldRef out, int post)
{
    HopArgs a;
    a.in = in;
    a.out = out;
    a.gauge = h->gauge_for(prec, out_par);
    a.nbr = h->nbr_for(out_par);
    a.Vh = h->Vh;
    a.Ls = h->Ls;
    a.post = h->mat(prec, post);
    a.err = h->errflag();
    a.ext[0] = h->dims[0] / 2;
    a.ext[1] = h->dims[1];
    a.ext[2] = h->dims[2];
    a.ext[3] = h->dims[3];
    a.zblock = sweep_zblock(h, prec);
    return a;
}

// Fills in the structured programs that match the dense matrices of `a`.
// with a given mixing mode (mode < 0: the handle's)
HopArgs with_programs_mode(dwf_ctx *h, int prec, const HopArgs &a0, int mode)
{
    HopArgs a = a0;
    {
        const int ip = mat_id_of(h, prec, a.post), iy = mat_id_of(h, prec, a.ymat), iz = mat_id_of(h, prec, a.zmat);
        a.post_band = ip >= 0 && h->fm.band[ip];
        a.y_band = iy >= 0 && h->fm.band[iy];
        a.z_band = iz >= 0 && h->fm.band[iz];
    }
    a.mixmode = mode >= 0 ? mode : h->mix_mode(prec);
    if (a.mixmode == 1) {
        const int ip = mat_id_of(h, prec, a.post), iy = mat_id_of(h, prec, a.ymat), iz = mat_id_of(h, prec, a.zmat);
        if (ip < 0 || (a.ymat && iy < 0) || (a.zmat && iz < 0)) {
            a.mixmode = 0;
        } else {
            a.post_prog = h->prog(prec, ip);
            a.y_prog = a.ymat ? h->prog(prec, iy) : nullptr;
            a.z_prog = a.zmat ? h->prog(prec, iz) : nullptr;
        }
    }
    return a;
}

HopArgs with_programs(dwf_ctx *h, int prec, const HopArgs &a0) { return with_programs_mode(h, prec, a0, -1); }

cudaError_t hop(dwf_ctx *h, int prec, bool dag, const HopArgs &a, cudaStream_t st)
{
    h->launches += 1;
    return launch_hop(prec, dag, with_programs(h, prec, a), h->hop_var[prec], h->hop_ns[prec], h->hop_sb[prec], st);
}

// The CG iteration's K_a and K_c (the hops whose only mixing is the dense M or
// M^T) in FP32 take the structured mixing by register chains when the caller
// left the mixing mode and the hop variant at their defaults (variant 9, Ls 8
// or 16): 3-4 % faster than the dense form for those two launches at 32^3x64,
// Ls 16, where the banded K_d and the two-matrix K_b are not.
cudaError_t hop_cg_plain(dwf_ctx *h, int prec, bool dag, const HopArgs &a, cudaStream_t st)
{
    const bool chains = prec == DWF_F32 && h->mixmode[prec] < 0 && h->fm.structured && (h->Ls == 8 || h->Ls == 16) &&
                        (h->hop_var[prec] < 0 || h->hop_var[prec] == 9) && !a.ymode && !a.zmat && !a.rin.v;
    if (!chains) return hop(h, prec, dag, a, st);
    h->launches += 1;
    return launch_hop(prec, dag, with_programs_mode(h, prec, a, 1), 9, h->hop_ns[prec], h->hop_sb[prec], st);
}

cudaError_t mix(dwf_ctx *h, int prec, FieldRef in, FieldRef out, int id, cudaStream_t st)
{
    MixArgs m;
    m.in = in;
    m.out = out;
    m.Vh = h->Vh;
    m.Ls = h->Ls;
    m.mat = h->mat(prec, id);
    m.mixmode = h->mix_mode(prec);
    m.prog = h->prog(prec, id);
    m.band = h->fm.band[id];
    m.err = h->errflag();
    h->launches += 1;
    return launch_mix(prec, m, st);
}

RedArgs red(dwf_ctx *h, int op, CgScalars *scal)
{
    RedArgs r;
    r.partials = h->partials;
    r.counter = h->counter;
    r.op = op;
    r.scal = scal;
    return r;
}

}  // namespace dwf_detail

using namespace dwf_detail;

void dwf_solver_release(dwf_ctx *h);

// ------------------------------------------------------------------- ABI
extern "C" {

const char *dwf_strerror(int s)
{
    switch (s) {
    case DWF_OK: return "ok";
    case DWF_EINVAL: return "invalid argument";
    case DWF_ENOMEM: return "out of device memory";
    case DWF_ECUDA: return "CUDA error";
    case DWF_ENOTCONV: return "solver did not converge";
    case DWF_ENONFINITE: return "non-finite value";
    case DWF_ETIMEOUT: return "bounded device wait timed out";
    case DWF_EBREAKDOWN: return "CG breakdown";
    case DWF_ENOGAUGE: return "gauge field not set";
    default: return "unknown status";
    }
}

const char *dwf_last_error(void) { return g_last_error.c_str(); }

static int create_impl(const int dims[4], int Ls, double M0, double mf, const double *bs, const double *cs, int form,
                       double alpha, const int bc[4], dwf_handle *out);

int dwf_create(const int dims[4], int Ls, double M0, double mf, double b, double c, int form, double alpha,
               const int bc[4], dwf_handle *out)
{
    if (Ls < 2 || Ls > LS_MAX) {
        if (out) *out = nullptr;
        return dwf_set_error(DWF_EINVAL, "Ls must be in [2, 32]");
    }
    std::vector<double> bs((size_t)Ls, b), cs((size_t)Ls, c);
    return create_impl(dims, Ls, M0, mf, bs.data(), cs.data(), form, alpha, bc, out);
}

int dwf_create_s(const int dims[4], int Ls, double M0, double mf, const double *b, const double *c, const int bc[4],
                 dwf_handle *out)
{
    if (!b || !c) {
        if (out) *out = nullptr;
        return dwf_set_error(DWF_EINVAL, "b/c is NULL");
    }
    return create_impl(dims, Ls, M0, mf, b, c, DWF_STANDARD, 1.0, bc, out);
}

static int create_impl(const int dims[4], int Ls, double M0, double mf, const double *bs, const double *cs, int form,
                       double alpha, const int bc[4], dwf_handle *out)
{
    if (!dims || !out) return dwf_set_error(DWF_EINVAL, "dims/out is NULL");
    *out = nullptr;
    long long V = 1;
    for (int k = 0; k < 4; ++k) {
        if (dims[k] < 2 || (dims[k] & 1)) return dwf_set_error(DWF_EINVAL, "every lattice extent must be even and >= 2");
        V *= dims[k];
    }
    if (V * (long long)Ls * 12 > (1LL << 40)) return dwf_set_error(DWF_EINVAL, "lattice too large");
    if (V > (1LL << 30)) return dwf_set_error(DWF_EINVAL, "lattice too large for 32-bit site indices");
    if (Ls < 2 || Ls > LS_MAX) return dwf_set_error(DWF_EINVAL, "Ls must be in [2, 32]");
    if (form != DWF_STANDARD && form != DWF_NEFF) return dwf_set_error(DWF_EINVAL, "unknown form");
    if (form == DWF_NEFF && !(alpha != 0.0 && std::isfinite(alpha)))
        return dwf_set_error(DWF_EINVAL, "alpha must be finite and nonzero");
    if (!std::isfinite(M0) || !std::isfinite(mf)) return dwf_set_error(DWF_EINVAL, "non-finite parameter");
    for (int s = 0; s < Ls; ++s)
        if (!std::isfinite(bs[s]) || !std::isfinite(cs[s])) return dwf_set_error(DWF_EINVAL, "non-finite parameter");
    int bcv[4] = {1, 1, 1, -1};
    if (bc)
        for (int k = 0; k < 4; ++k) {
            if (bc[k] != 1 && bc[k] != -1) return dwf_set_error(DWF_EINVAL, "bc entries must be +1 or -1");
            bcv[k] = bc[k];
        }
    dwf_ctx *h = new dwf_ctx();
    for (int k = 0; k < 4; ++k) h->dims[k] = dims[k], h->bc[k] = bcv[k];
    h->Ls = Ls;
    h->M0 = M0;
    h->mf = mf;
    h->b = bs[0];
    h->c = cs[0];
    h->alpha = (form == DWF_NEFF) ? alpha : 1.0;
    h->form = form;
    h->V = (int)V;
    h->Vh = (int)(V / 2);
    std::string err;
    if (!build_fifth_matrices_s(Ls, M0, mf, bs, cs, form, h->alpha, h->fm, err)) {
        delete h;
        return dwf_set_error(DWF_EINVAL, err);
    }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return dwf_cuda_error(e, "cudaGetDevice");
    }
    // matrices: [MAT_COUNT][2][Ls][Ls] transposed, FP64 and FP32
    const size_t per = (size_t)2 * Ls * Ls;
    std::vector<double> md(per * MAT_COUNT);
    std::vector<float> mf32(per * MAT_COUNT);
    for (int id = 0; id < MAT_COUNT; ++id)
        for (int chi = 0; chi < 2; ++chi)
            for (int s = 0; s < Ls; ++s)
                for (int t = 0; t < Ls; ++t) {
                    const double v = h->fm.mats[id][chi][(size_t)s * Ls + t];
                    const size_t o = per * id + (size_t)chi * Ls * Ls + (size_t)t * Ls + s;
                    md[o] = v;
                    mf32[o] = (float)v;
                }
    auto fail = [&](cudaError_t ce, const char *w) {
        int st = dwf_cuda_error(ce, w);
        dwf_destroy(h);
        return st;
    };
    if ((e = cudaMalloc(&h->mats_dev[0], md.size() * 8)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->mats_dev[1], mf32.size() * 4)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMemcpy(h->mats_dev[0], md.data(), md.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "cudaMemcpy");
    if ((e = cudaMemcpy(h->mats_dev[1], mf32.data(), mf32.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "cudaMemcpy");
    {
        // structured programs, FP64 and FP32 copies
        std::vector<MixProg<double>> pd(MAT_COUNT);
        std::vector<MixProg<float>> pf(MAT_COUNT);
        for (int id = 0; id < MAT_COUNT; ++id) {
            const FifthMatrices::Prog &s = h->fm.prog[id];
            MixProg<double> &d = pd[id];
            MixProg<float> &f = pf[id];
            std::memset(&d, 0, sizeof(d));
            std::memset(&f, 0, sizeof(f));
            d.inv = f.inv = s.inv;
            d.shift = f.shift = s.shift;
            for (int chi = 0; chi < 2; ++chi) {
                d.up[chi] = f.up[chi] = s.up[chi];
                for (int k = 0; k < LS_MAX; ++k) {
                    d.d1[chi][k] = s.d1[chi][k];
                    d.d2[chi][k] = s.d2[chi][k];
                    f.d1[chi][k] = (float)s.d1[chi][k];
                    f.d2[chi][k] = (float)s.d2[chi][k];
                }
            }
            d.s0 = s.s0, d.s1 = s.s1, d.a0inv = s.a0inv, d.kappa = s.kappa, d.mneg = s.mneg, d.corner = s.corner;
            f.s0 = (float)s.s0, f.s1 = (float)s.s1, f.a0inv = (float)s.a0inv, f.kappa = (float)s.kappa;
            f.mneg = (float)s.mneg, f.corner = (float)s.corner;
        }
        if ((e = cudaMalloc(&h->progs_dev[0], pd.size() * sizeof(pd[0]))) != cudaSuccess) return fail(e, "cudaMalloc");
        if ((e = cudaMalloc(&h->progs_dev[1], pf.size() * sizeof(pf[0]))) != cudaSuccess) return fail(e, "cudaMalloc");
        if ((e = cudaMemcpy(h->progs_dev[0], pd.data(), pd.size() * sizeof(pd[0]), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return fail(e, "cudaMemcpy");
        if ((e = cudaMemcpy(h->progs_dev[1], pf.data(), pf.size() * sizeof(pf[0]), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return fail(e, "cudaMemcpy");
    }
    if ((e = cudaMalloc(&h->nbr, (size_t)2 * h->Vh * 8 * sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->eo2lex, (size_t)2 * h->Vh * sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->partials, ((size_t)h->Vh + 8192) * sizeof(double))) != cudaSuccess)
        return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->counter, 64)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMemset(h->counter, 0, 64)) != cudaSuccess) return fail(e, "cudaMemset");
    if ((e = cudaMalloc(&h->scal, 8 * sizeof(CgScalars))) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMemset(h->scal, 0, 8 * sizeof(CgScalars))) != cudaSuccess) return fail(e, "cudaMemset");
    if ((e = cudaMalloc(&h->one, 8)) != cudaSuccess) return fail(e, "cudaMalloc");
    const double one = 1.0;
    if ((e = cudaMemcpy(h->one, &one, 8, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "cudaMemcpy");
    {   // 5D even-odd split: standard form, c_s = 0 for every s, even Ls
        bool ok = form == DWF_STANDARD && Ls % 2 == 0;
        std::vector<double> ia((size_t)Ls);
        for (int s = 0; s < Ls; ++s) {
            ok = ok && cs[s] == 0.0;
            const double a0 = bs[s] * (4.0 - M0) + 1.0;
            ok = ok && a0 != 0.0;
            ia[(size_t)s] = ok ? 1.0 / a0 : 0.0;
        }
        if (ok) {
            if ((e = cudaMalloc(&h->inv_a0, (size_t)Ls * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc");
            if ((e = cudaMemcpy(h->inv_a0, ia.data(), (size_t)Ls * sizeof(double), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
                return fail(e, "cudaMemcpy");
            h->eo5 = 1;
        }
    }
    if ((e = launch_build_tables(h->dims, h->nbr, h->eo2lex, 0)) != cudaSuccess) return fail(e, "build_tables");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "build_tables");
    h->bytes = md.size() * 8 + mf32.size() * 4 + (size_t)2 * h->Vh * 9 * sizeof(int) + ((size_t)h->Vh + 8192) * 8;
    *out = h;
    return DWF_OK;
}

int dwf_destroy(dwf_handle h)
{
    if (!h) return DWF_OK;
    dwf_solver_release(h);
    dwf_precond_release(h);
    for (auto &kv : h->work) cudaFree(kv.second.first);
    h->work.clear();
    for (int k = 0; k < 3; ++k) {
        if (h->mats_dev[k]) cudaFree(h->mats_dev[k]);
        if (h->gauge[k]) cudaFree(h->gauge[k]);
    }
    for (int k = 0; k < 2; ++k)
        if (h->progs_dev[k]) cudaFree(h->progs_dev[k]);
    if (h->nbr) cudaFree(h->nbr);
    if (h->eo2lex) cudaFree(h->eo2lex);
    if (h->partials) cudaFree(h->partials);
    if (h->counter) cudaFree(h->counter);
    if (h->scal) cudaFree(h->scal);
    if (h->one) cudaFree(h->one);
    if (h->inv_a0) cudaFree(h->inv_a0);
    delete h;
    return DWF_OK;
}

int dwf_create_slab(const int global_dims[4], int t0, int nt, int Ls, double M0, double mf, double b, double c,
                    int form, double alpha, const int bc[4], dwf_handle *out)
{
    if (!global_dims || !out) return dwf_set_error(DWF_EINVAL, "dims/out is NULL");
    *out = nullptr;
    const int Lt = global_dims[3];
    if (nt < 2 || (nt & 1) || (t0 & 1) || t0 < 0 || t0 >= Lt || nt >= Lt || Lt % 2)
        return dwf_set_error(DWF_EINVAL, "the slab needs an even origin and an even length below Lt");
    const int dims[4] = {global_dims[0], global_dims[1], global_dims[2], nt};
    dwf_handle h = nullptr;
    int rc = dwf_create(dims, Ls, M0, mf, b, c, form, alpha, bc, &h);
    if (rc) return rc;
    h->slab = 1;
    for (int k = 0; k < 4; ++k) h->gdims[k] = global_dims[k];
    h->t0 = t0;
    h->ghost = 2 * (h->Vh / nt);
    cudaError_t e = launch_slab_tables(h, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        dwf_destroy(h);
        return dwf_cuda_error(e, "slab tables");
    }
    *out = h;
    return DWF_OK;
}

int dwf_set_gauge(dwf_handle h, const void *U, void *stream)
{
    if (!h || !U) return dwf_set_error(DWF_EINVAL, "NULL handle or links");
    if (!aligned16(U)) return dwf_set_error(DWF_EINVAL, "links must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)2 * h->Vh * 8 * 18;
    const size_t sz[3] = {n * 8, n * 4, n * 2};
    for (int k = 0; k < 3; ++k)
        if (!h->gauge[k]) {
            CK(cudaMalloc(&h->gauge[k], sz[k]));
            h->bytes += sz[k];
        }
    if (h->slab)   // the global field, the slab's links with the global boundary phases
        CK(launch_slab_pack_gauge(h, (const double *)U, st));
    else
        CK(launch_pack_gauge((const double *)U, h->dims, h->bc, h->eo2lex, h->nbr, h->gauge[0], h->gauge[1],
                             h->gauge[2], st));
    h->launches += 1;
    h->has_gauge = true;
    return DWF_OK;
}

static int check_common(dwf_handle h, int prec, const void *in, const void *out)
{
    if (!h) return dwf_set_error(DWF_EINVAL, "NULL handle");
    if (h && h->slab) return dwf_set_error(DWF_EINVAL, "a slab handle applies its operator through dwf_slab_apply_eo");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    if (prec != DWF_F64 && prec != DWF_F32 && prec != DWF_F16) return dwf_set_error(DWF_EINVAL, "bad precision");
    if (!in || !out) return dwf_set_error(DWF_EINVAL, "NULL vector");
    if (!aligned16(in) || !aligned16(out)) return dwf_set_error(DWF_EINVAL, "vectors must be 16-byte aligned");
    return DWF_OK;
}

static int apply_impl(dwf_handle h, int op, int prec, const void *in, void *out, bool dag, cudaStream_t st)
{
    int rc = check_common(h, prec, in, out);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (op == DWF_OP_FULL5D) {
        FieldRef xe = h->field("ap_xe", prec, &e), xo = h->field("ap_xo", prec, &e);
        FieldRef ye = h->field("ap_ye", prec, &e), yo = h->field("ap_yo", prec, &e);
        FieldRef he = h->field("ap_he", prec, &e), ho = h->field("ap_ho", prec, &e);
        if (!xe.v || !xo.v || !ye.v || !yo.v || !he.v || !ho.v) return dwf_cuda_error(e, "workspace");
        CK(launch_pack_full(prec, (const double *)in, xe, xo, h->eo2lex, h->Vh, h->V, h->Ls, st));
        h->launches += 2;   // pack + unpack below
        if (!dag) {
            CK(mix(h, prec, xe, he, MAT_P, st));
            CK(mix(h, prec, xo, ho, MAT_P, st));
            for (int par = 0; par < 2; ++par) {
                HopArgs a = hop_args(h, prec, par, par ? he : ho, par ? yo : ye, MAT_NHALF);
                a.y = par ? xo : xe;
                a.ymode = 2;
                a.ymat = h->mat(prec, MAT_A5R);
                CK(hop(h, prec, false, a, st));
            }
        } else {
            for (int par = 0; par < 2; ++par) {
                HopArgs a = hop_args(h, prec, par, par ? xe : xo, par ? yo : ye, MAT_NHALF_RBT);
                a.y = par ? xo : xe;
                a.ymode = 2;
                a.ymat = h->mat(prec, MAT_RA5T);
                CK(hop(h, prec, true, a, st));
            }
        }
        CK(launch_unpack_full(prec, ye, yo, (double *)out, h->eo2lex, h->Vh, h->V, h->Ls, st));
        return DWF_OK;
    }
    if (op == DWF_OP_EO_PREC) {
        FieldRef x = h->field("ap_xe", prec, &e), xh = h->field("ap_he", prec, &e);
        FieldRef t = h->field("ap_ho", prec, &e), y = h->field("ap_ye", prec, &e);
        if (!x.v || !xh.v || !t.v || !y.v) return dwf_cuda_error(e, "workspace");
        CK(launch_pack_eo(prec, (const double *)in, x, h->Vh, h->Ls, st));
        h->launches += 2;   // pack + unpack below
        CK(mix(h, prec, x, xh, dag ? MAT_QT : MAT_P, st));
        HopArgs a1 = hop_args(h, prec, 1, xh, t, dag ? MAT_MT : MAT_M);
        CK(hop(h, prec, dag, a1, st));
        HopArgs a2 = hop_args(h, prec, 0, t, y, dag ? MAT_NPT4 : MAT_NQ4);
        a2.y = x;
        a2.ymode = 1;
        CK(hop(h, prec, dag, a2, st));
        CK(launch_unpack_eo(prec, y, (double *)out, h->Vh, h->Ls, st));
        return DWF_OK;
    }
    if (op == DWF_OP_EO5_PREC) {   // the 5D split's Schur complement: two whole-matrix applications
        if (!h->eo5) return dwf_set_error(DWF_EINVAL, "the 5D even-odd split needs the standard form, c = 0 and even Ls");
        const size_t by = (size_t)h->Ls * h->V * 24 * sizeof(double);
        void *A = h->ws("e5_a", by, &e), *B = h->ws("e5_b", by, &e), *C = h->ws("e5_c", by, &e);
        if (!A || !B || !C) return dwf_cuda_error(e, "workspace");
        CK(launch_eo5(0, in, nullptr, A, h->dims, h->V, h->Ls, h->inv_a0, st));   // x_e
        h->launches += 1;
        int rc2;
        if (!dag) {   // x - D_ee^-1 D_eo D_oo^-1 D_oe x
            if ((rc2 = apply_impl(h, DWF_OP_FULL5D, prec, A, B, false, st))) return rc2;
            CK(launch_eo5(1, B, nullptr, B, h->dims, h->V, h->Ls, h->inv_a0, st));
            if ((rc2 = apply_impl(h, DWF_OP_FULL5D, prec, B, C, false, st))) return rc2;
            CK(launch_eo5(2, A, C, out, h->dims, h->V, h->Ls, h->inv_a0, st));
        } else {      // x - D_oe^dag D_oo^-1 D_eo^dag D_ee^-1 x
            CK(launch_eo5(3, A, nullptr, C, h->dims, h->V, h->Ls, h->inv_a0, st));
            if ((rc2 = apply_impl(h, DWF_OP_FULL5D, prec, C, B, true, st))) return rc2;
            CK(launch_eo5(1, B, nullptr, B, h->dims, h->V, h->Ls, h->inv_a0, st));
            if ((rc2 = apply_impl(h, DWF_OP_FULL5D, prec, B, C, true, st))) return rc2;
            CK(launch_eo5(4, A, C, out, h->dims, h->V, h->Ls, h->inv_a0, st));
        }
        h->launches += 2;
        return DWF_OK;
    }
    return dwf_set_error(DWF_EINVAL, "unknown operator");
}

// the field a stage of the slab's even-odd application leaves for the exchange
static FieldRef slab_stage_field(dwf_handle h, int prec, int stage, cudaError_t *e)
{
    return h->field(stage == 0 ? "sl_xh" : "sl_t", prec, e);
}

int dwf_slab_apply_eo(dwf_handle h, int prec, int stage, int dag, const void *in, void *out, void *stream)
{
    if (!h || !h->slab) return dwf_set_error(DWF_EINVAL, "not a slab handle");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    if (prec != DWF_F64 && prec != DWF_F32) return dwf_set_error(DWF_EINVAL, "slabs run in FP64 or FP32");
    if (stage < 0 || stage > 2) return dwf_set_error(DWF_EINVAL, "stage must be 0, 1 or 2");
    if ((stage == 0 && !in) || (stage == 2 && !out)) return dwf_set_error(DWF_EINVAL, "NULL vector");
    if ((in && !aligned16(in)) || (out && !aligned16(out))) return dwf_set_error(DWF_EINVAL, "vectors must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    FieldRef x = h->field("sl_x", prec, &e), xh = h->field("sl_xh", prec, &e);
    FieldRef t = h->field("sl_t", prec, &e), y = h->field("sl_y", prec, &e);
    if (!x.v || !xh.v || !t.v || !y.v) return dwf_cuda_error(e, "workspace");
    if (stage == 0) {   // x^ = P x (Q^T x for the adjoint); its faces go to the neighbours
        CK(launch_pack_eo(prec, (const double *)in, x, h->Vh, h->Ls, st));
        h->launches += 1;
        CK(mix(h, prec, x, xh, dag ? MAT_QT : MAT_P, st));
    } else if (stage == 1) {   // t = M H_oe x^ (M^T H^dag_oe), reading x^'s ghost rows; t's faces go out
        HopArgs a1 = hop_args(h, prec, 1, xh, t, dag ? MAT_MT : MAT_M);
        CK(hop(h, prec, dag != 0, a1, st));
    } else {   // y = x - 1/4 Q H_eo t (x - 1/4 P^T H^dag_eo t), reading t's ghost rows
        HopArgs a2 = hop_args(h, prec, 0, t, y, dag ? MAT_NPT4 : MAT_NQ4);
        a2.y = x;
        a2.ymode = 1;
        CK(hop(h, prec, dag != 0, a2, st));
        CK(launch_unpack_eo(prec, y, (double *)out, h->Vh, h->Ls, st));
        h->launches += 1;
    }
    return DWF_OK;
}

int dwf_slab_faces(dwf_handle h, int prec, int stage, void **send_lo, void **send_hi, void **recv_lo,
                   void **recv_hi, size_t *bytes)
{
    if (!h || !h->slab) return dwf_set_error(DWF_EINVAL, "not a slab handle");
    if (prec != DWF_F64 && prec != DWF_F32) return dwf_set_error(DWF_EINVAL, "slabs run in FP64 or FP32");
    if (stage != 0 && stage != 1) return dwf_set_error(DWF_EINVAL, "faces exist after stages 0 and 1");
    if (!send_lo || !send_hi || !recv_lo || !recv_hi || !bytes) return dwf_set_error(DWF_EINVAL, "NULL pointer");
    cudaError_t e = cudaSuccess;
    FieldRef f = slab_stage_field(h, prec, stage, &e);
    if (!f.v) return dwf_cuda_error(e, "workspace");
    const size_t row = field_bytes(prec, 1, h->Ls);   // one site, all slices
    const size_t A3 = (size_t)h->Vh / h->dims[3];
    char *p = (char *)f.v;
    *send_lo = p;
    *send_hi = p + (size_t)(h->dims[3] - 1) * A3 * row;
    *recv_lo = p + (size_t)h->Vh * row;
    *recv_hi = p + ((size_t)h->Vh + A3) * row;
    *bytes = A3 * row;
    return DWF_OK;
}

int dwf_slab_exchange_ring(dwf_handle *hs, int n, int prec, int stage, void *stream)
{
    if (!hs || n < 2) return dwf_set_error(DWF_EINVAL, "a ring needs at least two slabs");
    for (int i = 0; i < n; ++i) {
        const dwf_handle a = hs[i], b = hs[(i + 1) % n];
        if (!a || !b || !a->slab || !b->slab) return dwf_set_error(DWF_EINVAL, "not a slab handle");
        for (int k = 0; k < 4; ++k)
            if (a->gdims[k] != b->gdims[k] || (k < 3 && a->dims[k] != b->dims[k]))
                return dwf_set_error(DWF_EINVAL, "the slabs belong to different lattices");
        if (a->Ls != b->Ls) return dwf_set_error(DWF_EINVAL, "the slabs have different Ls");
        if ((a->t0 + a->dims[3]) % a->gdims[3] != b->t0)
            return dwf_set_error(DWF_EINVAL, "the slabs are not consecutive in time");
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < n; ++i) {
        void *sl, *sh, *rl, *rh, *nsl, *nsh, *nrl, *nrh;
        size_t by = 0, nby = 0;
        int rc = dwf_slab_faces(hs[i], prec, stage, &sl, &sh, &rl, &rh, &by);
        if (rc) return rc;
        rc = dwf_slab_faces(hs[(i + 1) % n], prec, stage, &nsl, &nsh, &nrl, &nrh, &nby);
        if (rc) return rc;
        // my last slice -> the next slab's lower ghost face; its first slice -> my upper ghost face
        CK(cudaMemcpyAsync(nrl, sh, by, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(rh, nsl, by, cudaMemcpyDeviceToDevice, st));
    }
    return DWF_OK;
}

int dwf_slab_cgnr_ring(dwf_handle *hs, int n, const void *const *b, void *const *x, double tol, int max_iter,
                       int *iters, double *history, void *stream)
{
    if (!hs || n < 2 || !b || !x || !(tol > 0) || max_iter < 1) return dwf_set_error(DWF_EINVAL, "bad argument");
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || !hs[i]->slab) return dwf_set_error(DWF_EINVAL, "not a slab handle");
        if (!hs[i]->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
        if (!b[i] || !x[i] || !aligned16(b[i]) || !aligned16(x[i]))
            return dwf_set_error(DWF_EINVAL, "NULL or unaligned vector");
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    std::vector<void *> r(n), z(n), p(n), w(n);
    std::vector<size_t> nel(n);
    for (int i = 0; i < n; ++i) {
        nel[i] = (size_t)hs[i]->Vh * hs[i]->Ls * 12;   // complex numbers of one even field
        const size_t by = nel[i] * 16;
        r[i] = hs[i]->ws("dd_r", by, &e);
        z[i] = hs[i]->ws("dd_z", by, &e);
        p[i] = hs[i]->ws("dd_p", by, &e);
        w[i] = hs[i]->ws("dd_w", by, &e);
        if (!r[i] || !z[i] || !p[i] || !w[i]) return dwf_cuda_error(e, "workspace");
    }
    double *scratch = (double *)hs[0]->ws("dd_dot", (size_t)(256 + n) * sizeof(double), &e);
    if (!scratch) return dwf_cuda_error(e, "workspace");
    // D (dag = 0) or D^dag on the ring: the three stages of every slab, the faces exchanged between them
    auto apply = [&](int dag, const std::vector<void *> &in, const std::vector<void *> &out) -> int {
        int rc;
        for (int i = 0; i < n; ++i)
            if ((rc = dwf_slab_apply_eo(hs[i], DWF_F64, 0, dag, in[i], nullptr, stream))) return rc;
        if ((rc = dwf_slab_exchange_ring(hs, n, DWF_F64, 0, stream))) return rc;
        for (int i = 0; i < n; ++i)
            if ((rc = dwf_slab_apply_eo(hs[i], DWF_F64, 1, dag, nullptr, nullptr, stream))) return rc;
        if ((rc = dwf_slab_exchange_ring(hs, n, DWF_F64, 1, stream))) return rc;
        for (int i = 0; i < n; ++i)
            if ((rc = dwf_slab_apply_eo(hs[i], DWF_F64, 2, dag, nullptr, out[i], stream))) return rc;
        return DWF_OK;
    };
    // Re <a, b> over the ring: per-slab sums in a fixed order, added on the host in slab order
    std::vector<double> part(n);
    auto dot = [&](const std::vector<void *> &a, const std::vector<void *> &bb, double &res) -> int {
        for (int i = 0; i < n; ++i) CK(launch_cdot(a[i], bb[i], nel[i], scratch, scratch + 256 + i, st));
        CK(cudaMemcpyAsync(part.data(), scratch + 256, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        res = 0.0;
        for (int i = 0; i < n; ++i) res += part[i];
        return std::isfinite(res) ? DWF_OK : dwf_set_error(DWF_ENONFINITE, "non-finite inner product");
    };
    std::vector<void *> bv(n), xv(x, x + n);
    for (int i = 0; i < n; ++i) bv[i] = const_cast<void *>(b[i]);   // read only
    int rc;
    double bn2 = 0, gamma = 0, ww = 0, gnew = 0, rr = 0;
    for (int i = 0; i < n; ++i) {
        CK(cudaMemsetAsync(xv[i], 0, nel[i] * 16, st));
        CK(cudaMemcpyAsync(r[i], bv[i], nel[i] * 16, cudaMemcpyDeviceToDevice, st));
    }
    if ((rc = dot(bv, bv, bn2))) return rc;
    if (!(bn2 > 0)) return dwf_set_error(DWF_EINVAL, "zero right-hand side");
    const double bn = std::sqrt(bn2);
    if ((rc = apply(1, r, z))) return rc;
    for (int i = 0; i < n; ++i) CK(cudaMemcpyAsync(p[i], z[i], nel[i] * 16, cudaMemcpyDeviceToDevice, st));
    if ((rc = dot(z, z, gamma))) return rc;
    int it = 0;
    double res = 1.0;
    if (history) history[0] = res;
    while (res > tol && it < max_iter) {
        if ((rc = apply(0, p, w))) return rc;
        if ((rc = dot(w, w, ww))) return rc;
        if (!(ww > 0)) return dwf_set_error(DWF_EBREAKDOWN, "|D p|^2 <= 0");
        const double alpha = gamma / ww;
        for (int i = 0; i < n; ++i) {
            CK(launch_caxpby(alpha, p[i], 1.0, xv[i], nel[i], st));
            CK(launch_caxpby(-alpha, w[i], 1.0, r[i], nel[i], st));
        }
        if ((rc = apply(1, r, z))) return rc;
        if ((rc = dot(z, z, gnew))) return rc;
        for (int i = 0; i < n; ++i) CK(launch_caxpby(1.0, z[i], gnew / gamma, p[i], nel[i], st));
        gamma = gnew;
        ++it;
        if ((rc = dot(r, r, rr))) return rc;
        res = std::sqrt(rr) / bn;
        if (history) history[it] = res;
    }
    // the true residual b - D x
    if ((rc = apply(0, xv, w))) return rc;
    for (int i = 0; i < n; ++i) CK(launch_caxpby(1.0, bv[i], -1.0, w[i], nel[i], st));
    if ((rc = dot(w, w, rr))) return rc;
    if (iters) *iters = it;
    const double tres = std::sqrt(rr) / bn;
    if (history) history[it] = tres;
    return tres <= tol ? DWF_OK : dwf_set_error(DWF_ENOTCONV, "the decomposed CGNR did not reach tol");
}

int dwf_apply(dwf_handle h, int op, int prec, const void *in, void *out, void *stream)
{
    return apply_impl(h, op, prec, in, out, false, (cudaStream_t)stream);
}

int dwf_solve_eo5(dwf_handle h, const void *b5, void *x5, double tol, int max_iter, int *iters, double *history,
                  void *stream)
{
    int rc = check_common(h, DWF_F64, b5, x5);
    if (rc) return rc;
    if (!h->eo5) return dwf_set_error(DWF_EINVAL, "the 5D even-odd split needs the standard form, c = 0 and even Ls");
    if (!(tol > 0) || max_iter < 1) return dwf_set_error(DWF_EINVAL, "bad tolerance or iteration cap");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    const size_t nel = (size_t)h->Ls * h->V * 12, by = nel * 16;
    void *r = h->ws("e5_r", by, &e), *z = h->ws("e5_z", by, &e), *p = h->ws("e5_p", by, &e);
    void *w = h->ws("e5_w", by, &e), *t = h->ws("e5_t", by, &e);
    double *scr = (double *)h->ws("e5_dot", 257 * sizeof(double), &e);
    if (!r || !z || !p || !w || !t || !scr) return dwf_cuda_error(e, "workspace");
    auto dot = [&](const void *a, const void *b, double &res) -> int {
        CK(launch_cdot(a, b, nel, scr, scr + 256, st));
        CK(cudaMemcpyAsync(&res, scr + 256, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return std::isfinite(res) ? DWF_OK : dwf_set_error(DWF_ENONFINITE, "non-finite inner product");
    };
    auto D = [&](const void *in, void *out, bool dag) {
        return apply_impl(h, DWF_OP_EO5_PREC, DWF_F64, in, out, dag, st);
    };
    // b'_e = D_ee^-1 (b_e - D_eo D_oo^-1 b_o)
    CK(launch_eo5(1, b5, nullptr, t, h->dims, h->V, h->Ls, h->inv_a0, st));
    if ((rc = apply_impl(h, DWF_OP_FULL5D, DWF_F64, t, w, false, st))) return rc;
    CK(launch_eo5(5, b5, w, r, h->dims, h->V, h->Ls, h->inv_a0, st));   // r = b'_e (x_e = 0)
    CK(cudaMemcpyAsync(t, r, by, cudaMemcpyDeviceToDevice, st));        // t = b'_e, kept
    CK(cudaMemsetAsync(x5, 0, by, st));
    double bn2 = 0, gamma = 0, ww = 0, gnew = 0, rr = 0;
    if ((rc = dot(t, t, bn2))) return rc;
    if (!(bn2 > 0)) return dwf_set_error(DWF_EINVAL, "zero right-hand side");
    const double bn = std::sqrt(bn2);
    if ((rc = D(r, z, true))) return rc;
    CK(cudaMemcpyAsync(p, z, by, cudaMemcpyDeviceToDevice, st));
    if ((rc = dot(z, z, gamma))) return rc;
    int it = 0;
    double res = 1.0;
    if (history) history[0] = res;
    while (res > tol && it < max_iter) {
        if ((rc = D(p, w, false))) return rc;
        if ((rc = dot(w, w, ww))) return rc;
        if (!(ww > 0)) return dwf_set_error(DWF_EBREAKDOWN, "|D p|^2 <= 0");
        const double alpha = gamma / ww;
        CK(launch_caxpby(alpha, p, 1.0, x5, nel, st));
        CK(launch_caxpby(-alpha, w, 1.0, r, nel, st));
        if ((rc = D(r, z, true))) return rc;
        if ((rc = dot(z, z, gnew))) return rc;
        CK(launch_caxpby(1.0, z, gnew / gamma, p, nel, st));
        gamma = gnew;
        ++it;
        if ((rc = dot(r, r, rr))) return rc;
        res = std::sqrt(rr) / bn;
        if (history) history[it] = res;
    }
    h->launches += 4;
    // x_o = D_oo^-1 (b_o - D_oe x_e); x5 = x_e + x_o; the true residual of the whole system
    if ((rc = apply_impl(h, DWF_OP_FULL5D, DWF_F64, x5, w, false, st))) return rc;
    CK(launch_eo5(6, b5, w, z, h->dims, h->V, h->Ls, h->inv_a0, st));
    CK(launch_caxpby(1.0, z, 1.0, x5, nel, st));
    if ((rc = apply_impl(h, DWF_OP_FULL5D, DWF_F64, x5, w, false, st))) return rc;
    CK(launch_caxpby(1.0, b5, -1.0, w, nel, st));   // w = b5 - D x5
    double b52 = 0;
    if ((rc = dot(w, w, rr))) return rc;
    if ((rc = dot(b5, b5, b52))) return rc;
    const double tres = std::sqrt(rr / b52);
    if (iters) *iters = it;
    if (history) history[it] = tres;
    return tres <= tol ? DWF_OK : dwf_set_error(DWF_ENOTCONV, "the 5D even-odd CGNR did not reach tol");
}

int dwf_wait_probe(dwf_handle h, long long limit_ns, void *stream)
{
    if (!h || limit_ns < 0) return dwf_set_error(DWF_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    int *flag = (int *)h->ws("probe_flag", 16, &e);
    if (!flag) return dwf_cuda_error(e, "workspace");
    CK(cudaMemsetAsync(flag, 0, 16, st));
    const unsigned long long lim = limit_ns > 1000000000ll ? 1000000000ull : (unsigned long long)limit_ns;
    CK(launch_wait_probe(flag, lim, h->errflag(), st));
    h->launches += 1;
    return DWF_OK;
}

int dwf_apply_dag(dwf_handle h, int op, int prec, const void *in, void *out, void *stream)
{
    return apply_impl(h, op, prec, in, out, true, (cudaStream_t)stream);
}

int dwf_source_5d(dwf_handle h, const void *b4, void *b5, void *stream)
{
    int rc = check_common(h, DWF_F64, b4, b5);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    double *v5 = (double *)h->ws("src_v5", (size_t)h->V * h->Ls * 24 * 8, &e);
    FieldRef ve = h->field("ap_xe", DWF_F64, &e), vo = h->field("ap_xo", DWF_F64, &e);
    FieldRef oe = h->field("ap_ye", DWF_F64, &e), oo = h->field("ap_yo", DWF_F64, &e);
    if (!v5 || !ve.v || !vo.v || !oe.v || !oo.v) return dwf_cuda_error(e, "workspace");
    CK(launch_chiral_embed((const double *)b4, v5, h->V, h->Ls, st));
    h->launches += 3;   // embed, pack, unpack
    CK(launch_pack_full(DWF_F64, v5, ve, vo, h->eo2lex, h->Vh, h->V, h->Ls, st));
    for (int par = 0; par < 2; ++par) {
        HopArgs a = hop_args(h, DWF_F64, par, par ? ve : vo, par ? oo : oe, MAT_SRC_POST);
        a.y = par ? vo : ve;
        a.ymode = 2;
        a.ymat = h->mat(DWF_F64, MAT_SRC_Y);
        CK(hop(h, DWF_F64, false, a, st));
    }
    CK(launch_unpack_full(DWF_F64, oe, oo, (double *)b5, h->eo2lex, h->Vh, h->V, h->Ls, st));
    return DWF_OK;
}

int dwf_project_4d(dwf_handle h, const void *x5, void *x4, void *stream)
{
    if (!h || !x5 || !x4) return dwf_set_error(DWF_EINVAL, "NULL argument");
    if (!aligned16(x5) || !aligned16(x4)) return dwf_set_error(DWF_EINVAL, "vectors must be 16-byte aligned");
    CK(launch_project4d((const double *)x5, (double *)x4, h->V, h->Ls, (cudaStream_t)stream));
    h->launches += 1;
    return DWF_OK;
}

int dwf_fifth_matrix(dwf_handle h, int which, int chi, double *out)
{
    if (!h || !out || chi < 0 || chi > 1) return dwf_set_error(DWF_EINVAL, "bad argument");
    const std::vector<double> *m = nullptr;
    switch (which) {
    case 0: m = &h->fm.A5[chi]; break;
    case 1: m = &h->fm.A5inv[chi]; break;
    case 2: m = &h->fm.B[chi]; break;
    case 3: m = &h->fm.R[chi]; break;
    default: return dwf_set_error(DWF_EINVAL, "bad matrix id");
    }
    std::memcpy(out, m->data(), m->size() * sizeof(double));
    return DWF_OK;
}

int dwf_fifth_matrix_host(int Ls, double M0, double mf, const double *b, const double *c, int form, double alpha,
                          int which, int chi, double *out, int *banded)
{
    if (Ls < 2 || Ls > LS_MAX || (form != DWF_STANDARD && form != DWF_NEFF) || chi < 0 || chi > 1 || !out || !b ||
        !c)
        return dwf_set_error(DWF_EINVAL, "bad argument");
    if (!(which >= 0 && which <= 3) && !(which >= 16 && which < 16 + MAT_COUNT))
        return dwf_set_error(DWF_EINVAL, "bad matrix id");
    bool finite = std::isfinite(M0) && std::isfinite(mf);
    for (int s = 0; s < Ls; ++s) finite = finite && std::isfinite(b[s]) && std::isfinite(c[s]);
    if (!finite || (form == DWF_NEFF && !(alpha != 0.0 && std::isfinite(alpha))))
        return dwf_set_error(DWF_EINVAL, "non-finite parameter or alpha = 0");
    FifthMatrices fm;
    std::string err;
    if (!build_fifth_matrices_s(Ls, M0, mf, b, c, form, form == DWF_NEFF ? alpha : 1.0, fm, err))
        return dwf_set_error(DWF_EINVAL, err.c_str());
    const std::vector<double> *m = nullptr;
    switch (which) {
    case 0: m = &fm.A5[chi]; break;
    case 1: m = &fm.A5inv[chi]; break;
    case 2: m = &fm.B[chi]; break;
    case 3: m = &fm.R[chi]; break;
    default: m = &fm.mats[which - 16][chi]; break;
    }
    std::memcpy(out, m->data(), m->size() * sizeof(double));
    if (banded) *banded = which >= 16 ? (fm.band[which - 16] ? 1 : 0) : 0;
    return DWF_OK;
}

size_t dwf_device_bytes(dwf_handle h) { return h ? h->bytes : 0; }

int dwf_device_status(dwf_handle h, void *stream)
{
    if (!h) return dwf_set_error(DWF_EINVAL, "NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, h->errflag(), sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flag) {
        CK(cudaMemsetAsync(h->errflag(), 0, sizeof(int), st));
        CK(cudaStreamSynchronize(st));
        return dwf_set_error(DWF_ETIMEOUT, "a bounded wait inside a hop kernel gave up");
    }
    return DWF_OK;
}

long long dwf_launch_count(dwf_handle h) { return h ? h->launches : 0; }

int dwf_set_hop_config(dwf_handle h, int prec, int variant, int ns, int sb)
{
    if (!h || prec < 0 || prec > 2) return dwf_set_error(DWF_EINVAL, "bad handle or precision");
    if (variant < -1 || variant > 10 || variant == 1 || variant == 2 || variant == 6 || variant == 8)
        return dwf_set_error(DWF_EINVAL, "variant must be -1, 0, 3, 4, 5, 7, 9 or 10");
    if (variant == 10) {   // no tiling parameters
        if (ns != 0 || sb != 0) return dwf_set_error(DWF_EINVAL, "variant 10 takes ns 0 and sb 0");
        h->hop_var[prec] = variant;
        h->hop_ns[prec] = 0;
        h->hop_sb[prec] = 0;
        return DWF_OK;
    }
    if (variant == 9) {   // sb counts warps per CTA (1..4), ns the register budget (1, 2)
        if (ns < 0 || ns > 2) return dwf_set_error(DWF_EINVAL, "variant 9 takes ns 0, 1 or 2");
        if (sb < 0 || sb > 4) return dwf_set_error(DWF_EINVAL, "variant 9 takes sb (warps per CTA) 0..4");
        h->hop_var[prec] = variant;
        h->hop_ns[prec] = ns;
        h->hop_sb[prec] = sb;
        return DWF_OK;
    }
    if (variant == 7 && ns > 1) return dwf_set_error(DWF_EINVAL, "variant 7 takes ns 0 or 1");
    if (ns < 0 || ns > 4 || ns == 3 || (ns && h->Ls % ns) || (ns == 4 && variant != 5))
        return dwf_set_error(DWF_EINVAL, "ns must be 0, 1, 2 or (variant 5) 4, and divide Ls");
    const int nsv = ns ? ns : hop_default_ns(prec, h->Ls);
    if (sb < 0 || (sb && (h->Ls / nsv) * sb > 256)) return dwf_set_error(DWF_EINVAL, "sb out of range (CTA > 256 threads)");
    h->hop_var[prec] = variant;
    h->hop_ns[prec] = ns;
    h->hop_sb[prec] = sb;
    return DWF_OK;
}

int dwf_set_sweep(dwf_handle h, int prec, int zblock)
{
    if (!h || prec < 0 || prec > 2) return dwf_set_error(DWF_EINVAL, "bad handle or precision");
    const long long A = (long long)(h->dims[0] / 2) * h->dims[1];
    if (zblock < -2 || (zblock > 0 && (zblock >= h->dims[2] || h->dims[2] % zblock || (zblock * A) % 32)))
        return dwf_set_error(DWF_EINVAL,
                             "zblock must be -2, -1, 0 or a divisor of Lz below Lz with zblock Lx/2 Ly a multiple of 32");
    h->sweep_zb[prec] = zblock == -2 ? sweep_zblock_auto(h, prec) : zblock;
    return DWF_OK;
}

int dwf_get_sweep(dwf_handle h, int prec, int *zblock)
{
    if (!h || prec < 0 || prec > 2 || !zblock) return dwf_set_error(DWF_EINVAL, "bad argument");
    *zblock = sweep_zblock(h, prec);
    return DWF_OK;
}

int dwf_set_mix_mode(dwf_handle h, int prec, int mode)
{
    if (!h || prec < 0 || prec > 2 || mode < -1 || mode > 2) return dwf_set_error(DWF_EINVAL, "bad argument");
    if (mode == 1 && !h->fm.structured)
        return dwf_set_error(DWF_EINVAL, "the structured mixing is not available for these parameters");
    if (mode == 2 && prec == DWF_F64)
        return dwf_set_error(DWF_EINVAL, "the tensor-core mixing has no FP64 form");
    h->mixmode[prec] = mode;
    return DWF_OK;
}

int dwf_get_mix_mode(dwf_handle h, int prec, int *mode)
{
    if (!h || prec < 0 || prec > 2 || !mode) return dwf_set_error(DWF_EINVAL, "bad argument");
    *mode = h->mix_mode(prec);
    return DWF_OK;
}

int dwf_get_hop_config(dwf_handle h, int prec, int *variant, int *ns, int *sb)
{
    if (!h || prec < 0 || prec > 2 || !variant || !ns || !sb) return dwf_set_error(DWF_EINVAL, "bad argument");
    *variant = h->hop_var[prec] >= 0 ? h->hop_var[prec] : hop_default_variant(prec);
    *ns = h->hop_ns[prec] ? h->hop_ns[prec] : hop_default_ns(prec, h->Ls);
    *sb = h->hop_sb[prec] ? h->hop_sb[prec] : hop_default_sb(prec, h->Ls, *ns);
    return DWF_OK;
}

int dwf_autotune(dwf_handle h, int prec, const char *cache_path, void *stream)
{
    if (!h || prec < 0 || prec > 2) return dwf_set_error(DWF_EINVAL, "bad handle or precision");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, h->device));
    char key[256];
    std::snprintf(key, sizeof key, "%s|%dx%dx%dx%d|Ls=%d|prec=%d", prop.name, h->dims[0], h->dims[1], h->dims[2],
                  h->dims[3], h->Ls, prec);
    for (char *c = key; *c; ++c)
        if (*c == ' ') *c = '_';
    if (cache_path) {
        FILE *f = std::fopen(cache_path, "r");
        if (f) {
            char k[256];
            int var, ns, sb, mix;
            double us;
            bool hit = false;
            while (std::fscanf(f, "%255s %d %d %d %d %lf", k, &var, &ns, &sb, &mix, &us) == 6) {
                if (std::strcmp(k, key) == 0) {
                    h->hop_var[prec] = var;
                    h->hop_ns[prec] = ns;
                    h->hop_sb[prec] = sb;
                    h->mixmode[prec] = mix;
                    h->mixmode[prec] = h->mix_mode(prec);
                    hit = true;
                }
            }
            std::fclose(f);
            if (hit) return DWF_OK;
        }
    }
    double best = 1e30;
    int bvar = -1, bns = 0, bsb = 0, bmix = 0;
    for (int mix = 0; mix <= 2; ++mix)
        for (int var = 0; var <= 10; ++var)
            for (int ns = 1; ns <= 4; ns *= 2) {
                if (var == 10 && (prec != DWF_F32 || mix != 0 || (h->Ls != 8 && h->Ls != 16) || ns != 1)) continue;
                if (mix == 1 && !h->fm.structured) continue;
                if (mix == 2 && prec == DWF_F64) continue;
                if (var == 1 || var == 2 || var == 6 || var == 8) continue;   // numbers not in use
                if (mix != 0 && var != 0) continue;   // those mixings exist in the direct variant only
                if (var == 5 && prec != DWF_F16) continue;
                if ((var == 7 || var == 9) && (prec == DWF_F64 || h->Ls % 4 != 0)) continue;
                if (var == 7 && ns != 1) continue;
                if (var == 9 && (32 % h->Ls != 0 || ns > 2)) continue;
                if (ns == 4 && var != 5) continue;
                if (var != 9 && h->Ls % ns) continue;
                const int LsN = h->Ls / (var == 9 ? 1 : ns);
                for (int threads = 64; threads <= 256; threads += 64) {
                    if (var == 9 && threads > 128) continue;
                    if (var == 10 && threads != 256) continue;   // fixed CTA of 8 warps
                    const int sb = var == 10 ? 0 : var == 9 ? threads / 32 : threads / LsN;   // variant 9: warps per CTA
                    if (var != 10 && (sb < 1 || LsN * sb > 256)) continue;
                    h->mixmode[prec] = mix;
                    h->hop_var[prec] = var;
                    h->hop_ns[prec] = var == 10 ? 0 : ns;
                    h->hop_sb[prec] = sb;
                    double us = 0, by = 0;
                    int rc = dwf_time_hop(h, prec, 10, 0, &us, &by, stream);
                    if (rc) return rc;
                    if (us < best) {
                        best = us;
                        bvar = var;
                        bns = var == 10 ? 0 : ns;
                        bsb = sb;
                        bmix = mix;
                    }
                }
            }
    h->hop_var[prec] = bvar;
    h->hop_ns[prec] = bns;
    h->hop_sb[prec] = bsb;
    h->mixmode[prec] = bmix;
    if (cache_path) {
        FILE *f = std::fopen(cache_path, "a");
        if (f) {
            std::fprintf(f, "%s %d %d %d %d %.3f\n", key, bvar, bns, bsb, bmix, best);
            std::fclose(f);
        }
    }
    return DWF_OK;
}

int dwf_time_mix(dwf_handle h, int prec, int mode, int reps, int flush_l2, double *us, double *bytes, void *stream)
{
    if (!h || reps < 1 || !us || !bytes) return dwf_set_error(DWF_EINVAL, "bad argument");
    if (prec != DWF_F64 && prec != DWF_F32 && prec != DWF_F16) return dwf_set_error(DWF_EINVAL, "bad precision");
    if (mode < 0 || mode > 2 || (mode == 2 && prec == DWF_F64) || (mode == 1 && !h->fm.structured))
        return dwf_set_error(DWF_EINVAL, "mode must be 0, 1 (if available) or 2 (FP32/FP16)");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    FieldRef in = h->field("th_in", prec, &e), out = h->field("th_out", prec, &e);
    if (!in.v || !out.v) return dwf_cuda_error(e, "workspace");
    CK(cudaMemsetAsync(in.v, 0x3c, field_bytes(prec, h->Vh, h->Ls), st));
    if (in.scale) CK(cudaMemsetAsync(in.scale, 0x3f, scale_bytes(prec, h->Vh, h->Ls), st));
    const size_t flush_bytes = (size_t)512 << 20;
    void *flush = nullptr;
    if (flush_l2) {
        flush = h->ws("th_flush", flush_bytes, &e);
        if (!flush) return dwf_cuda_error(e, "workspace");
    }
    const int saved = h->mixmode[prec];
    h->mixmode[prec] = mode;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double total_ms = 0;
    for (int r = -2; r < reps && e == cudaSuccess; ++r) {
        if (flush_l2) e = cudaMemsetAsync(flush, r & 0xff, flush_bytes, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = mix(h, prec, in, out, MAT_M, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess && r >= 0) {
            cudaEventElapsedTime(&ms, e0, e1);
            total_ms += ms;
        }
    }
    h->mixmode[prec] = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return dwf_cuda_error(e, "dwf_time_mix");
    *us = 1000.0 * total_ms / reps;
    *bytes = 2.0 * (double)(field_bytes(prec, h->Vh, h->Ls) + scale_bytes(prec, h->Vh, h->Ls));
    return DWF_OK;
}

int dwf_time_hop(dwf_handle h, int prec, int reps, int flush_l2, double *us, double *bytes, void *stream)
{
    if (!h || reps < 1 || !us || !bytes) return dwf_set_error(DWF_EINVAL, "bad argument");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    if (prec != DWF_F64 && prec != DWF_F32 && prec != DWF_F16) return dwf_set_error(DWF_EINVAL, "bad precision");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    FieldRef in = h->field("th_in", prec, &e), out = h->field("th_out", prec, &e);
    if (!in.v || !out.v) return dwf_cuda_error(e, "workspace");
    CK(cudaMemsetAsync(in.v, 0x3c, field_bytes(prec, h->Vh, h->Ls), st));
    if (in.scale) CK(cudaMemsetAsync(in.scale, 0x3f, scale_bytes(prec, h->Vh, h->Ls), st));
    const size_t flush_bytes = (size_t)512 << 20;
    void *flush = nullptr;
    if (flush_l2) {
        flush = h->ws("th_flush", flush_bytes, &e);
        if (!flush) return dwf_cuda_error(e, "workspace");
    }
    HopArgs a = hop_args(h, prec, 1, in, out, MAT_M);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int w = 0; w < 3; ++w) CK(hop(h, prec, false, a, st));
    double total_ms = 0;
    if (flush_l2) {
        for (int r = 0; r < reps; ++r) {
            CK(cudaMemsetAsync(flush, r & 0xff, flush_bytes, st));
            CK(cudaEventRecord(e0, st));
            CK(hop(h, prec, false, a, st));
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            total_ms += ms;
        }
    } else {
        CK(cudaEventRecord(e0, st));
        for (int r = 0; r < reps; ++r) CK(hop(h, prec, false, a, st));
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        total_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *us = 1000.0 * total_ms / reps;
    const size_t link_sz = prec == DWF_F64 ? 8 : (prec == DWF_F32 ? 4 : 2);
    *bytes = 2.0 * (double)(field_bytes(prec, h->Vh, h->Ls) + (prec == DWF_F16 ? (size_t)h->Vh * h->Ls * 4 : 0)) +
             (double)h->Vh * 8 * 18 * link_sz;
    return DWF_OK;
}

}  // extern "C"
