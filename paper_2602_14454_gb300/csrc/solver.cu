// CG on the normal equation of the even-odd preconditioned matrix (Sec. 2.3:
// D^dag D x_e = D^dag b~_e, D = 1 - D_ee^-1 D_eo D_oo^-1 D_oe), with
//   * the inner iteration in FP64, FP32 or FP16-with-scales,
//   * FP64 reliable updates: x accumulates in FP64, and whenever the inner
//     residual has fallen by `delta` the true residual b~ - D x is recomputed
//     in FP64 and replaces the iterated one (published method: Sleijpen and
//     van der Vorst 1996; Clark et al. 2010), the search direction is kept,
//   * the final FP64 check of the full 5D residual after x_o is rebuilt.
//
// One inner iteration is five launches on the device, no host round trip:
//   K_e  x += alpha p (the previous iteration's step, deferred to the launch
//        that reads p anyway) ; p = r + beta p ;  phat = P p      (P = B R)
//   K_a  t = M H_oe phat                                  (M = B A5^-1)
//   K_b  w = p - 1/4 Q H_eo t ; what = Q^T w ; alpha = gamma / |w|^2
//   K_c  u = M^T gamma5-hop_oe what
//   K_d  r -= alpha (Q^-T what - 1/4 P^T gamma5-hop_eo u) ;
//        beta = |r|^2 / gamma ; gamma = |r|^2
// The step of the last iteration before a reliable update is added there.
// so that w = D p and D^dag w = Q^-T what - 1/4 P^T H^dag_eo M^T H^dag_oe what.
// `check_every` iterations are captured once as a CUDA graph and replayed;
// the host reads the scalars between replays.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "dwf_internal.h"

using namespace dwf;

namespace dwf_detail {
HopArgs hop_args(dwf_ctx *h, int prec, int out_par, FieldRef in, FieldRef out, int post);
HopArgs with_programs(dwf_ctx *h, int prec, const HopArgs &a0);
cudaError_t hop(dwf_ctx *h, int prec, bool dag, const HopArgs &a, cudaStream_t st);
cudaError_t hop_cg_plain(dwf_ctx *h, int prec, bool dag, const HopArgs &a, cudaStream_t st);
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

__global__ void reliable_fix_kernel(CgScalars *cg, const CgScalars *fresh, int first)
{
    const double g = fresh->last;
    if (first) {
        cg->beta = 0.0;
    } else {
        cg->beta = (cg->gamma > 0.0) ? cg->beta * (g / cg->gamma) : 0.0;
    }
    cg->gamma = g;
    cg->flags = 0;
}

struct Bufs {
    int ps;   // inner precision
    int xp;   // accumulator precision
    int form = 0;   // 0: CG on D_pc (eq. even-odd_linear_equation), 1: on D' (eq. another_even-odd_linear_equation)
    FieldRef be, bo, bt, x64, r64, t64, h64, xo64;
    FieldRef p, ph, t, wh, u, rs, xs;
    CgScalars *cg, *n64, *aux;
};

int get_bufs(dwf_ctx *h, int ps, Bufs &B)
{
    cudaError_t e = cudaSuccess;
    B.ps = ps;
    B.xp = (ps == DWF_F64) ? DWF_F64 : DWF_F32;
    B.be = h->field("sv_be", DWF_F64, &e);
    B.bo = h->field("sv_bo", DWF_F64, &e);
    B.bt = h->field("sv_bt", DWF_F64, &e);
    B.x64 = h->field("sv_x64", DWF_F64, &e);
    B.r64 = h->field("sv_r64", DWF_F64, &e);
    B.t64 = h->field("sv_t64", DWF_F64, &e);
    B.h64 = h->field("sv_h64", DWF_F64, &e);
    B.xo64 = h->field("sv_xo64", DWF_F64, &e);
    B.p = h->field("sv_p", ps, &e);
    B.ph = h->field("sv_ph", ps, &e);
    B.t = h->field("sv_t", ps, &e);
    B.wh = h->field("sv_wh", ps, &e);
    B.u = h->field("sv_u", ps, &e);
    B.rs = h->field("sv_rs", ps, &e);
    B.xs = h->field("sv_xs", B.xp, &e);
    const FieldRef *all[] = {&B.be, &B.bo, &B.bt, &B.x64, &B.r64, &B.t64, &B.h64, &B.xo64,
                             &B.p, &B.ph, &B.t, &B.wh, &B.u, &B.rs, &B.xs};
    for (auto f : all)
        if (!f->v) return dwf_cuda_error(e, "solver workspace");
    B.cg = h->scal + 0;
    B.n64 = h->scal + 1;
    B.aux = h->scal + 2;
    return DWF_OK;
}

// Arguments of the five launches of one inner iteration; ra / rb: where the
// alpha and beta reductions go.
struct IterArgs {
    CgUpdateArgs ue;
    HopArgs k[4];   // K_a, K_b (operator), K_c, K_d (adjoint)
};

// B.form = 1: the operator is D' = D_ee D_pc D_ee^-1 = 1 - 1/4 H_eo M H_oe M and
// D'^dag w = w - 1/4 M^T H^dag M^T H^dag w (the product P Q of the first form's
// outer mixings is M, and D_ee Q = 1): p^ = M p, K_b without the Q^T mixing,
// K_d with the identity in place of Q^-T and -1/4 M^T in place of -1/4 P^T.
IterArgs iteration_args(dwf_ctx *h, const Bufs &B, const RedArgs &ra, const RedArgs &rb)
{
    const int P = B.ps;
    const bool f2 = B.form == 1;
    IterArgs I;
    CgUpdateArgs &ue = I.ue;
    ue.r = B.rs;
    ue.p = B.p;
    ue.phat = B.ph;
    ue.Vh = h->Vh;
    ue.Ls = h->Ls;
    const int pre = f2 ? MAT_M : MAT_P;
    ue.mat = h->mat(P, pre);
    ue.mixmode = h->mix_mode(P);
    ue.prog = h->prog(P, pre);
    ue.band = h->fm.band[pre];
    ue.scal = B.cg;
    ue.xacc = B.xs.v;   // x += alpha p of the previous iteration

    I.k[0] = hop_args(h, P, 1, B.ph, B.t, MAT_M);

    HopArgs &kb = I.k[1];
    kb = hop_args(h, P, 0, B.t, B.wh, f2 ? MAT_NQUARTER : MAT_NQ4);
    kb.y = B.p;
    kb.ymode = 1;
    kb.zmat = f2 ? nullptr : h->mat(P, MAT_QT);
    kb.red = ra;

    I.k[2] = hop_args(h, P, 1, B.wh, B.u, MAT_MT);

    HopArgs &kd = I.k[3];
    kd = hop_args(h, P, 0, B.u, B.rs, f2 ? MAT_NMT4 : MAT_NPT4);
    kd.y = B.wh;
    kd.ymode = f2 ? 1 : 2;
    kd.ymat = f2 ? nullptr : h->mat(P, MAT_RA5T);
    kd.rin = B.rs;
    kd.ralpha = &B.cg->alpha;
    kd.red = rb;
    return I;
}

// The reliable-update threshold: the caller's delta, or by the inner precision.
// FP16 fields carry about three decimal digits, so the iterated residual is
// replaced by the FP64 true residual after every factor of 10; FP32 keeps the
// iterated residual accurate far longer, and at 32^3x64, Ls 16 a factor of 1000
// needed 4 instead of 8 FP64 recomputations for the same 352 iterations (3.19
// instead of 3.48 s).
double reliable_delta(const dwf_solve_params *p)
{
    if (p->delta > 0) return p->delta;
    return p->inner_prec == DWF_F32 ? 1e-3 : 0.1;
}

// One inner iteration (five launches).
cudaError_t inner_iteration(dwf_ctx *h, const Bufs &B, cudaStream_t st)
{
    const IterArgs I = iteration_args(h, B, red(h, RED_CG_ALPHA, B.cg), red(h, RED_CG_BETA, B.cg));
    cudaError_t e;
    h->launches += 1;
    if ((e = launch_cg_update(B.ps, I.ue, st)) != cudaSuccess) return e;
    for (int k = 0; k < 4; ++k)
        if ((e = (k == 0 || k == 2) ? hop_cg_plain(h, B.ps, k >= 2, I.k[k], st) : hop(h, B.ps, k >= 2, I.k[k], st)) !=
            cudaSuccess)
            return e;
    return cudaSuccess;
}

// r64 = b~ - D x64 in FP64; |r64|^2 -> n64->last
cudaError_t true_residual(dwf_ctx *h, const Bufs &B, cudaStream_t st)
{
    cudaError_t e;
    if ((e = mix(h, DWF_F64, B.x64, B.h64, MAT_P, st)) != cudaSuccess) return e;
    HopArgs a1 = hop_args(h, DWF_F64, 1, B.h64, B.t64, MAT_M);
    if ((e = hop(h, DWF_F64, false, a1, st)) != cudaSuccess) return e;
    HopArgs a2 = hop_args(h, DWF_F64, 0, B.t64, B.r64, MAT_NQ4);
    a2.y = B.x64;
    a2.ymode = 1;
    a2.rin = B.bt;
    a2.ralpha = h->one;
    a2.red = red(h, RED_STORE, B.n64);
    return hop(h, DWF_F64, false, a2, st);
}

// The true residual of the zero iterate: r64 = b~, whose norm the b~ hop left in
// aux; no FP64 operator application is needed.
cudaError_t zero_iterate_residual(dwf_ctx *h, const Bufs &B, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(B.r64.v, B.bt.v, field_bytes(DWF_F64, h->Vh, h->Ls), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(&B.n64->last, &B.aux->last, sizeof(double), cudaMemcpyDeviceToDevice, st);
}

// rs = D^dag r64 evaluated in the inner precision; |rs|^2 -> n64->last.
// B.form = 1: rs = D'^dag r' with r' = D_ee r64 = b' - D' y, the residual of the
// second form's equation for y = D_ee x_e.
cudaError_t normal_residual(dwf_ctx *h, const Bufs &B, cudaStream_t st)
{
    const int P = B.ps;
    cudaError_t e;
    h->launches += 1;
    if ((e = launch_convert(DWF_F64, B.r64, P, B.rs, h->Vh, h->Ls, st)) != cudaSuccess) return e;
    if ((e = mix(h, P, B.rs, B.ph, B.form == 1 ? MAT_A5R : MAT_QT, st)) != cudaSuccess) return e;
    HopArgs a1 = hop_args(h, P, 1, B.ph, B.u, MAT_MT);
    if ((e = hop(h, P, true, a1, st)) != cudaSuccess) return e;
    HopArgs a2 = hop_args(h, P, 0, B.u, B.rs, B.form == 1 ? MAT_NMT4 : MAT_NPT4);
    a2.y = B.form == 1 ? B.ph : B.rs;
    a2.ymode = 1;
    a2.red = red(h, RED_STORE, B.n64);
    return hop(h, P, true, a2, st);
}

// One FP32 cycle of flexible CG (Notay 2000) on the normal equation
//     A x = b,  A = D^dag D (D the even-odd matrix),
// preconditioned by M = N N^dag (N the handle's network, trained so that
// N D ~ 1, hence M ~ A^-1), from x = 0: r = b, z = M r, p = z; then per step
// q = A p, alpha = (r, z) / (p, q), x += alpha p, r' = r - alpha q, z' = M r',
// beta = (z', r' - r) / (r, z) (Polak-Ribiere), p = z' + beta p.  It stops when
// |r| <= eta |b| or after kmax steps; x is added into `xacc`.  With plain =
// true M is the identity (CG on D^dag D).  A non-positive (p, q) or (r, z)
// ends the cycle and sets `plain` for the rest of the solve (the caller's FP64
// defect correction continues from the iterate reached).  hist (if not null)
// receives |r_k| / |b| for k = 0, 1, ... (at most kmax + 1 values).
int fcg_cycle(dwf_ctx *h, FieldRef b, FieldRef xacc, double eta, int kmax, bool &plain, int &iters, int &napp,
              int &fallbacks, int &dapp, double *hist, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    FieldRef ra = h->field("fc_ra", DWF_F32, &e), rb = h->field("fc_rb", DWF_F32, &e);
    FieldRef z = h->field("fc_z", DWF_F32, &e), pp = h->field("fc_p", DWF_F32, &e);
    FieldRef q = h->field("fc_q", DWF_F32, &e), t1 = h->field("fc_t1", DWF_F32, &e);
    if (!ra.v || !rb.v || !z.v || !pp.v || !q.v || !t1.v) return dwf_cuda_error(e, "workspace");
    const int Vh = h->Vh, Ls = h->Ls;
    CgScalars *sc = h->scal + 4;
    CgScalars hs[2];
    int rc;
    auto dot = [&](FieldRef x, FieldRef y, double &out) -> int {
        CK(launch_vdot(x, y, Vh, Ls, red(h, RED_STORE, sc), st));
        h->launches += 1;
        CK(cudaMemcpyAsync(hs, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        out = hs[0].last;
        return DWF_OK;
    };
    auto precondition = [&](FieldRef v, FieldRef out) -> int {
        if (plain) {
            CK(launch_vaxpby(1.f, v, 0.f, out, Vh, Ls, st));
            h->launches += 1;
            return DWF_OK;
        }
        napp += 1;
        return net_apply_f32(h, v, out, st, 2);
    };
    FieldRef r = ra, rn = rb;
    CK(launch_vaxpby(1.f, b, 0.f, r, Vh, Ls, st));   // r = b - A 0
    h->launches += 1;
    double bn2;
    if ((rc = dot(b, b, bn2))) return rc;
    const double bn = std::sqrt(bn2);
    if (hist) hist[0] = 1.0;
    if (!(bn > 0) || !std::isfinite(bn)) return DWF_OK;
    if ((rc = precondition(r, z))) return rc;
    CK(launch_vaxpby(1.f, z, 0.f, pp, Vh, Ls, st));
    h->launches += 1;
    double rz;
    if ((rc = dot(r, z, rz))) return rc;
    if (!(rz > 0) || !std::isfinite(rz)) {
        if (plain) return dwf_set_error(DWF_EBREAKDOWN, "CG breakdown");
        plain = true;
        fallbacks += 1;
        return DWF_OK;
    }
    for (int k = 0; k < kmax; ++k) {
        if ((rc = eo_apply_f32(h, pp, t1, st))) return rc;     // D p
        if ((rc = eo_dag_apply_f32(h, t1, q, st))) return rc;  // q = D^dag D p
        dapp += 2;
        double pq;
        if ((rc = dot(pp, q, pq))) return rc;
        if (!(pq > 0) || !std::isfinite(pq)) {
            if (plain) return dwf_set_error(DWF_EBREAKDOWN, "CG breakdown");
            plain = true;
            fallbacks += 1;
            return DWF_OK;
        }
        const double alpha = rz / pq;
        CK(launch_vaxpby((float)alpha, pp, 1.f, xacc, Vh, Ls, st));        // x += alpha p
        CK(launch_vaxpby(1.f, r, 0.f, rn, Vh, Ls, st));                    // r' = r - alpha q
        CK(launch_vaxpby((float)-alpha, q, 1.f, rn, Vh, Ls, st));
        h->launches += 3;
        iters += 1;
        double rn2;
        if ((rc = dot(rn, rn, rn2))) return rc;
        if (!std::isfinite(rn2)) return dwf_set_error(DWF_ENONFINITE, "non-finite residual in the FCG cycle");
        if (hist) hist[k + 1] = std::sqrt(rn2) / bn;
        if (std::sqrt(rn2) <= eta * bn) break;
        if ((rc = precondition(rn, z))) return rc;                          // z' = M r'
        double zrn, zr;
        if ((rc = dot(z, rn, zrn))) return rc;
        if ((rc = dot(z, r, zr))) return rc;
        if (!(zrn > 0) || !std::isfinite(zrn)) {
            if (plain) return dwf_set_error(DWF_EBREAKDOWN, "CG breakdown");
            plain = true;
            fallbacks += 1;
            return DWF_OK;
        }
        const double beta = (zrn - zr) / rz;
        CK(launch_vaxpby(1.f, z, (float)beta, pp, Vh, Ls, st));            // p = z' + beta p
        h->launches += 1;
        rz = zrn;
        FieldRef tmp = r;
        r = rn;
        rn = tmp;
    }
    return DWF_OK;
}

int read_scalars(const Bufs &B, CgScalars *host, int n, cudaStream_t st)
{
    CK(cudaMemcpyAsync(host, B.cg, sizeof(CgScalars) * n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return DWF_OK;
}

struct GraphCache {
    std::string key;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

// Per-handle solver state that is not a device buffer.
struct SolverExtra {
    cudaStream_t cap = nullptr;
    GraphCache graph;
    CgScalars *pinned = nullptr;
};
static std::map<dwf_ctx *, SolverExtra> g_extra;
static std::mutex g_extra_mu;   // handles of different threads share the map (an entry is used by its handle only)

static SolverExtra &solver_extra(dwf_ctx *h)
{
    std::lock_guard<std::mutex> lk(g_extra_mu);
    return g_extra[h];
}

void dwf_solver_release(dwf_ctx *h)
{
    std::lock_guard<std::mutex> lk(g_extra_mu);
    auto it = g_extra.find(h);
    if (it == g_extra.end()) return;
    if (it->second.graph.exec) cudaGraphExecDestroy(it->second.graph.exec);
    if (it->second.cap) cudaStreamDestroy(it->second.cap);
    if (it->second.pinned) cudaFreeHost(it->second.pinned);
    g_extra.erase(it);
}

static int solve_impl(dwf_handle h, const void *b5, void *x5, const dwf_solve_params *p, dwf_solve_stats *stats,
                      cudaStream_t st)
{
    auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = h->launches;
    dwf_solve_stats S;
    std::memset(&S, 0, sizeof(S));
    S.status = DWF_OK;
    const int ps = p->inner_prec;
    if (ps != DWF_F64 && ps != DWF_F32 && ps != DWF_F16) return dwf_set_error(DWF_EINVAL, "bad inner precision");
    if (!(p->tol > 0) || p->max_iter < 1 || !(p->delta >= 0 && p->delta < 1) || p->check_every < 1)
        return dwf_set_error(DWF_EINVAL, "bad solver parameters");
    const double delta = reliable_delta(p);
    if (p->precond && !h->net)
        return dwf_set_error(DWF_EINVAL, "precond = 1 needs a network (dwf_precond_init or dwf_precond_train)");
    if (p->precond && ps != DWF_F32) return dwf_set_error(DWF_EINVAL, "the FCG solve runs its inner cycles in FP32");
    if (p->eo_form != 0 && p->eo_form != 1) return dwf_set_error(DWF_EINVAL, "eo_form must be 0 or 1");
    if (p->eo_form == 1 && p->precond)
        return dwf_set_error(DWF_EINVAL, "the learned preconditioner runs on the first even-odd form only");
    Bufs B;
    int rc = get_bufs(h, ps, B);
    if (rc) return rc;
    B.form = p->eo_form;
    SolverExtra &X = solver_extra(h);
    if (!X.pinned) CK(cudaMallocHost(&X.pinned, sizeof(CgScalars) * 4));
    if (!X.cap) CK(cudaStreamCreateWithFlags(&X.cap, cudaStreamNonBlocking));
    CgScalars *hs = X.pinned;

    // b5 -> (b_e, b_o); |b5|^2
    CK(launch_pack_full(DWF_F64, (const double *)b5, B.be, B.bo, h->eo2lex, h->Vh, h->V, h->Ls, st));
    CK(launch_norm2(DWF_F64, B.be, h->Vh, h->Ls, red(h, RED_STORE, B.n64), st));
    CK(launch_norm2(DWF_F64, B.bo, h->Vh, h->Ls, red(h, RED_STORE, B.aux), st));
    h->launches += 3;
    if ((rc = read_scalars(B, hs, 3, st))) return rc;
    const double b5n = std::sqrt(hs[1].last + hs[2].last);
    if (!std::isfinite(b5n)) return dwf_set_error(DWF_ENONFINITE, "source contains NaN or Inf");
    if (b5n == 0.0) {
        CK(cudaMemsetAsync(x5, 0, (size_t)h->V * h->Ls * 24 * 8, st));
        S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (stats) *stats = S;
        return DWF_OK;
    }
    // b~_e = Q b_e + 1/2 Q H_eo M b_o
    CK(mix(h, DWF_F64, B.bo, B.t64, MAT_M, st));
    {
        HopArgs a = hop_args(h, DWF_F64, 0, B.t64, B.bt, MAT_HALF_Q);
        a.y = B.be;
        a.ymode = 2;
        a.ymat = h->mat(DWF_F64, MAT_Q);
        a.red = red(h, RED_STORE, B.aux);
        CK(hop(h, DWF_F64, false, a, st));
    }
    if ((rc = read_scalars(B, hs, 3, st))) return rc;
    const double btn = std::sqrt(hs[2].last);
    // initial guess
    if (p->use_initial_guess) {
        FieldRef dummy = B.xo64;
        CK(launch_pack_full(DWF_F64, (const double *)x5, B.x64, dummy, h->eo2lex, h->Vh, h->V, h->Ls, st));
        h->launches += 1;
    } else {
        CK(launch_zero(DWF_F64, B.x64, h->Vh, h->Ls, st));
    }
    CK(launch_zero(B.xp, B.xs, h->Vh, h->Ls, st));
    CK(launch_zero(ps, B.p, h->Vh, h->Ls, st));
    CK(cudaMemsetAsync(B.cg, 0, sizeof(CgScalars), st));

    // stop when the even part of the full 5D residual is below tol |b5| / 2 (the
    // odd part vanishes after the exact reconstruction of x_o): first form,
    // r_full,e = D_ee r64, bounded by |D_ee| |r64|; second form, r_full,e = r'
    // itself, the residual of its own equation (D_ee r64)
    double target = B.form == 1 ? p->tol * b5n * 0.5 : p->tol * b5n / h->fm.dee_norm2 * 0.5;
    const int N = p->check_every;
    int iters = 0, nru = 0, dapp = 0;
    double rtrue = 0, rho = 1, rmax = 0;
    bool converged = false;
    int status = DWF_OK;

    // graph of N inner iterations
    GraphCache &G = X.graph;
    char keybuf[256];
    // the captured kernels depend on the hop configuration and mixing mode too
    std::snprintf(keybuf, sizeof keybuf, "%d/%d/%p/%p/%p/%d/%d/%d/%d/%d/%d", ps, N, B.p.v, B.rs.v, B.xs.v,
                  p->use_graph, h->hop_var[ps], h->hop_ns[ps], h->hop_sb[ps], h->mix_mode(ps), B.form);
    if (p->use_graph && G.key != keybuf) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
        cudaGraph_t g;
        const long long saved = h->launches;
        CK(cudaStreamBeginCapture(X.cap, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < N; ++k) {
            cudaError_t e = inner_iteration(h, B, X.cap);
            if (e != cudaSuccess) {
                cudaStreamEndCapture(X.cap, &g);
                return dwf_cuda_error(e, "graph capture");
            }
        }
        CK(cudaStreamEndCapture(X.cap, &g));
        h->launches = saved;
        CK(cudaGraphInstantiate(&G.exec, g, 0));
        cudaGraphDestroy(g);
        G.key = keybuf;
    }

    double q_rate = 0, rn_last = 0;   // per-iteration reduction of the inner residual, last inner residual
    // xzero: x64 is still zero (first update without an initial guess)
    auto reliable = [&](bool first, bool xzero) -> int {
        if (!first && B.form == 1) {
            // the inner CG accumulated a correction f of y = D_ee x_e: x64 += D_ee^-1 f
            CK(launch_zero(DWF_F64, B.h64, h->Vh, h->Ls, st));
            CK(launch_accum_x((double *)B.h64.v, B.xs.v, B.xp, B.p, B.ps, &B.cg->alpha, h->Vh, h->Ls, st));
            CK(mix(h, DWF_F64, B.h64, B.t64, MAT_Q, st));
            CK(launch_accum_x((double *)B.x64.v, B.t64.v, DWF_F64, B.t64, DWF_F64, nullptr, h->Vh, h->Ls, st));
            h->launches += 3;
        } else if (!first) {
            CK(launch_accum_x((double *)B.x64.v, B.xs.v, B.xp, B.p, B.ps, &B.cg->alpha, h->Vh, h->Ls, st));
            h->launches += 1;
        }
        // the deferred x update is done (or void after a restart)
        CK(cudaMemsetAsync(&B.cg->alpha, 0, sizeof(double), st));
        // always the full FP64 recomputation: r64 -= D xs in lower precision would carry
        // an error of about eps |D| |x|, i.e. eps kappa(D) |b~|, which stalls CG at light masses
        if (xzero) {
            CK(zero_iterate_residual(h, B, st));
        } else {
            CK(true_residual(h, B, st));
            dapp += 1;
        }
        if (B.form == 1) {   // |r'| = |D_ee r64|, the second form's residual
            CK(mix(h, DWF_F64, B.r64, B.t64, MAT_A5R, st));
            CK(launch_norm2(DWF_F64, B.t64, h->Vh, h->Ls, red(h, RED_STORE, B.n64), st));
            h->launches += 1;
        }
        CgScalars n64;
        CK(cudaMemcpyAsync(&hs[1], B.n64, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        n64 = hs[1];
        rtrue = std::sqrt(n64.last);
        if (!std::isfinite(rtrue)) return dwf_set_error(DWF_ENONFINITE, "non-finite residual");
        if (S.n_history < 64) S.history[S.n_history++] = rtrue / btn;
        if (rtrue <= target) {
            converged = true;
            return DWF_OK;
        }
        CK(normal_residual(h, B, st));
        reliable_fix_kernel<<<1, 1, 0, st>>>(B.cg, B.n64, first ? 1 : 0);
        CK(cudaGetLastError());
        h->launches += 1;
        dapp += 1;
        CK(cudaMemcpyAsync(hs, B.cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const double rn = std::sqrt(hs[0].gamma);
        rmax = rn;
        rn_last = rn;
        rho = (rn > 0) ? rtrue / rn : 1.0;
        nru += first ? 0 : 1;
        return DWF_OK;
    };

    int napp = 0, nfall = 0;
    bool lp_plain = false;
    cudaError_t ce = cudaSuccess;
    for (int round = 0; round < 3 && status == DWF_OK; ++round) {
        converged = false;
        const bool fresh = round == 0 && !p->use_initial_guess;
        if ((rc = reliable(fresh, fresh))) return rc;
        // learned preconditioner: FP32 cycles of flexible CG on the correction's
        // normal equation D^dag D e = D^dag r64 with M = N N^dag, each closed by an
        // FP64 defect correction (x64 += e, r64 = b~ - D x64)
        while (p->precond && !converged) {
            if (iters >= p->max_iter) {
                status = DWF_ENOTCONV;
                break;
            }
            // the right side of the correction's normal equation: D^dag r64 in FP32
            FieldRef r32 = h->field("lp_r32", DWF_F32, &ce), b32 = h->field("lp_b32", DWF_F32, &ce);
            if (!r32.v || !b32.v) return dwf_cuda_error(ce, "workspace");
            CK(launch_convert(DWF_F64, B.r64, DWF_F32, r32, h->Vh, h->Ls, st));
            h->launches += 1;
            if ((rc = eo_dag_apply_f32(h, r32, b32, st))) return rc;
            dapp += 1;
            if ((rc = fcg_cycle(h, b32, B.xs, 0.01 * (p->delta > 0 ? p->delta : 0.1), p->max_iter - iters, lp_plain, iters, napp, nfall,
                                dapp, nullptr, st)))
                return rc;
            if ((rc = reliable(false, false))) return rc;
        }
        while (!p->precond && !converged) {
            if (iters >= p->max_iter) {
                status = DWF_ENOTCONV;
                break;
            }
            // near convergence, run only the iterations the last block's residual
            // reduction rate predicts (no overshoot by up to check_every - 1)
            int nrun = N;
            if (q_rate > 0 && q_rate < 1 && rn_last > 0 && rho * rn_last > target) {
                const double k = std::ceil(std::log(target / (rho * rn_last)) / std::log(q_rate));
                if (k >= 1 && k < N) nrun = (int)k;
            }
            if (nrun == N && p->use_graph) {
                CK(cudaGraphLaunch(G.exec, st));
                h->launches += 5LL * N;
            } else {
                for (int k = 0; k < nrun; ++k) CK(inner_iteration(h, B, st));
            }
            iters += nrun;
            dapp += 2 * nrun;
            if ((rc = read_scalars(B, hs, 1, st))) return rc;
            const double rn = std::sqrt(hs[0].gamma);
            if (rn_last > 0 && rn > 0 && std::isfinite(rn)) q_rate = std::pow(rn / rn_last, 1.0 / nrun);
            rn_last = rn;
            const bool bad = (hs[0].flags != 0) || !std::isfinite(rn);
            if (p->verbose)
                std::fprintf(stderr, "[dwf] it %d |r_n| %.3e est %.3e target %.3e\n", iters, rn, rho * rn, target);
            if (bad || rn < delta * rmax || rho * rn < target || iters >= p->max_iter) {
                if (bad && hs[0].flags & 2) {
                    // non-finite inner state: restart from the FP64 iterate
                    CK(launch_zero(B.xp, B.xs, h->Vh, h->Ls, st));
                    CK(launch_zero(ps, B.p, h->Vh, h->Ls, st));
                    if ((rc = reliable(true, false))) return rc;
                    if (nru > 200) return dwf_set_error(DWF_ENONFINITE, "inner iteration keeps producing NaN");
                    ++nru;
                    continue;
                }
                if ((rc = reliable(false, false))) return rc;
                if (nru > 1000) {
                    status = DWF_ENOTCONV;
                    break;
                }
            }
        }
        // x_o = Q b_o + 1/2 Q H_oe P x_e ; full residual
        CK(mix(h, DWF_F64, B.x64, B.h64, MAT_P, st));
        {
            HopArgs a = hop_args(h, DWF_F64, 1, B.h64, B.xo64, MAT_HALF_Q);
            a.y = B.bo;
            a.ymode = 2;
            a.ymat = h->mat(DWF_F64, MAT_Q);
            CK(hop(h, DWF_F64, false, a, st));
        }
        CK(mix(h, DWF_F64, B.xo64, B.t64, MAT_P, st));
        for (int par = 0; par < 2; ++par) {
            HopArgs a = hop_args(h, DWF_F64, par, par ? B.h64 : B.t64, B.r64, MAT_NHALF);
            a.y = par ? B.xo64 : B.x64;
            a.ymode = 2;
            a.ymat = h->mat(DWF_F64, MAT_A5R);
            a.rin = par ? B.bo : B.be;
            a.ralpha = h->one;
            a.red = red(h, RED_STORE, par ? B.aux : B.n64);
            CK(hop(h, DWF_F64, false, a, st));
        }
        dapp += 2;
        if ((rc = read_scalars(B, hs, 3, st))) return rc;
        S.true_residual = std::sqrt(hs[1].last + hs[2].last) / b5n;
        S.eo_residual = rtrue / btn;
        if (S.true_residual <= p->tol || status != DWF_OK) break;
        target *= 0.1;
    }
    CK(launch_unpack_full(DWF_F64, B.x64, B.xo64, (double *)x5, h->eo2lex, h->Vh, h->V, h->Ls, st));
    h->launches += 1;
    CK(cudaStreamSynchronize(st));
    if (status == DWF_OK && S.true_residual > p->tol) status = DWF_ENOTCONV;
    S.status = status;
    S.iterations = iters;
    S.reliable_updates = nru;
    S.d_applications = dapp;
    S.kernel_launches = h->launches - launches0;
    S.waves = 1;
    S.precond_applications = napp;
    S.fallbacks = nfall;
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S;
    if (status != DWF_OK) dwf_set_error(status, "solver did not reach the tolerance");
    return status;
}

// ------------------------------------------------------------ batched solve
// Many systems on one lattice, in waves that fit in device memory.  Within a
// wave every system keeps its own CG state (FP64 solution and source, inner
// fields, scalars, reduction buffers); the FP64 temporaries of source
// preparation, reliable updates and the final check are shared, since those
// steps run one system at a time between graph replays.  The inner iteration
// runs as batched launches (one per kernel and distinct Ls) over all systems
// of the wave; systems that have converged set their skip flag.
namespace {

size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }

struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0;
    void *take(size_t nb)
    {
        const size_t o = round256(used);
        if (!base || o + nb > size) return nullptr;
        used = o + nb;
        return base + o;
    }
    FieldRef field(int prec, int Vh, int Ls)
    {
        FieldRef f;
        f.v = take(field_bytes(prec, Vh, Ls));
        if (prec == DWF_F16) f.scale = (float *)take(scale_bytes(prec, Vh, Ls));
        return f;
    }
};

size_t field_total(int prec, int Vh, int Ls) { return round256(field_bytes(prec, Vh, Ls)) + round256(scale_bytes(prec, Vh, Ls)); }

size_t system_bytes(const dwf_ctx *h, int ps)
{
    const int xp = ps == DWF_F64 ? DWF_F64 : DWF_F32;
    return 2 * field_total(DWF_F64, h->Vh, h->Ls) + 6 * field_total(ps, h->Vh, h->Ls) + field_total(xp, h->Vh, h->Ls) +
           round256(3 * sizeof(CgScalars)) + round256(((size_t)h->Vh + 8192) * 8) + 256 +
           round256(sizeof(CgUpdateArgs)) + 4 * round256(sizeof(HopArgs));
}

size_t shared_bytes(int V, int Vh, int Ls) { return 6 * field_total(DWF_F64, Vh, Ls) + round256((size_t)V * Ls * 24 * 8); }

struct SysRun {
    dwf_ctx *h = nullptr;
    int idx = 0;                 // position in the caller's arrays
    Bufs B;
    double *partials = nullptr;  // this system's reduction buffers
    unsigned *counter = nullptr;
    double b5n = 0, btn = 0, target = 0, rtrue = 0, rho = 1, rmax = 0;
    int iters = 0, nru = 0, dapp = 0, round = 0, status = DWF_OK;
    bool active = false, converged = false, done = false;
    dwf_solve_stats S;
};

// (b_e, b_o) = even / odd halves of b5 = (1 - c D_W) P^dag (0, .., b4) in the
// internal FP64 layout (the source of Sec. 2.2, as dwf_source_5d), using the
// canonical buffer v5 and the temporaries ve, vo.
cudaError_t source_eo(dwf_ctx *h, const void *b4, double *v5, FieldRef ve, FieldRef vo, FieldRef be, FieldRef bo,
                      cudaStream_t st)
{
    cudaError_t e;
    if ((e = launch_chiral_embed((const double *)b4, v5, h->V, h->Ls, st)) != cudaSuccess) return e;
    if ((e = launch_pack_full(DWF_F64, v5, ve, vo, h->eo2lex, h->Vh, h->V, h->Ls, st)) != cudaSuccess) return e;
    h->launches += 2;
    for (int par = 0; par < 2; ++par) {
        HopArgs a = hop_args(h, DWF_F64, par, par ? ve : vo, par ? bo : be, MAT_SRC_POST);
        a.y = par ? vo : ve;
        a.ymode = 2;
        a.ymat = h->mat(DWF_F64, MAT_SRC_Y);
        if ((e = hop(h, DWF_F64, false, a, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// FP64 true residual; convergence test; else the normal residual in the inner
// precision and the rescaled beta (as the reliable step of solve_impl).
int sys_reliable(SysRun &R, bool first, CgScalars *hs, cudaStream_t st, bool xzero = false)
{
    dwf_ctx *h = R.h;
    Bufs &B = R.B;
    if (!first) {
        CK(launch_accum_x((double *)B.x64.v, B.xs.v, B.xp, B.p, B.ps, &B.cg->alpha, h->Vh, h->Ls, st));
        h->launches += 1;
    }
    CK(cudaMemsetAsync(&B.cg->alpha, 0, sizeof(double), st));   // the deferred x update is done
    if (xzero) {
        CK(zero_iterate_residual(h, B, st));
    } else {
        CK(true_residual(h, B, st));
        R.dapp += 1;
    }
    CK(cudaMemcpyAsync(&hs[1], B.n64, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    R.rtrue = std::sqrt(hs[1].last);
    if (!std::isfinite(R.rtrue)) return dwf_set_error(DWF_ENONFINITE, "non-finite residual");
    if (R.S.n_history < 64) R.S.history[R.S.n_history++] = R.rtrue / R.btn;
    if (R.rtrue <= R.target) {
        R.converged = true;
        return DWF_OK;
    }
    CK(normal_residual(h, B, st));
    reliable_fix_kernel<<<1, 1, 0, st>>>(B.cg, B.n64, first ? 1 : 0);
    CK(cudaGetLastError());
    h->launches += 1;
    R.dapp += 1;
    CK(cudaMemcpyAsync(hs, B.cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double rn = std::sqrt(hs[0].gamma);
    R.rmax = rn;
    R.rho = (rn > 0) ? R.rtrue / rn : 1.0;
    R.nru += first ? 0 : 1;
    return DWF_OK;
}

// Source, b~_e and the first residual of one system.
int sys_prepare(SysRun &R, const void *b4, double *v5, const dwf_solve_params *p, CgScalars *hs, cudaStream_t st)
{
    dwf_ctx *h = R.h;
    Bufs &B = R.B;
    CK(source_eo(h, b4, v5, B.r64, B.t64, B.be, B.bo, st));
    CK(launch_norm2(DWF_F64, B.be, h->Vh, h->Ls, red(h, RED_STORE, B.n64), st));
    CK(launch_norm2(DWF_F64, B.bo, h->Vh, h->Ls, red(h, RED_STORE, B.aux), st));
    h->launches += 2;
    CK(cudaMemcpyAsync(hs, B.cg, 3 * sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    R.b5n = std::sqrt(hs[1].last + hs[2].last);
    if (!std::isfinite(R.b5n)) return dwf_set_error(DWF_ENONFINITE, "source contains NaN or Inf");
    CK(launch_zero(DWF_F64, B.x64, h->Vh, h->Ls, st));
    CK(launch_zero(B.xp, B.xs, h->Vh, h->Ls, st));
    CK(launch_zero(B.ps, B.p, h->Vh, h->Ls, st));
    CK(launch_zero(B.ps, B.rs, h->Vh, h->Ls, st));
    CK(cudaMemsetAsync(B.cg, 0, sizeof(CgScalars), st));
    if (R.b5n == 0.0) {
        R.done = true;
        return DWF_OK;
    }
    CK(mix(h, DWF_F64, B.bo, B.t64, MAT_M, st));
    {
        HopArgs a = hop_args(h, DWF_F64, 0, B.t64, B.bt, MAT_HALF_Q);
        a.y = B.be;
        a.ymode = 2;
        a.ymat = h->mat(DWF_F64, MAT_Q);
        a.red = red(h, RED_STORE, B.aux);
        CK(hop(h, DWF_F64, false, a, st));
    }
    CK(cudaMemcpyAsync(hs, B.cg, 3 * sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    R.btn = std::sqrt(hs[2].last);
    R.target = p->tol * R.b5n / h->fm.dee_norm2 * 0.5;
    R.active = true;
    int rc = sys_reliable(R, true, hs, st, true);
    if (rc) return rc;
    if (R.converged) R.active = false;
    return DWF_OK;
}

// x_o, the full 5D residual; then either the 4D solution or another round
// with a tenfold smaller target (at most three rounds, as solve_impl).
int sys_finish(SysRun &R, const void *b4, void *x4, double *v5, const dwf_solve_params *p, CgScalars *hs,
               cudaStream_t st)
{
    dwf_ctx *h = R.h;
    Bufs &B = R.B;
    CK(source_eo(h, b4, v5, B.r64, B.t64, B.be, B.bo, st));
    CK(mix(h, DWF_F64, B.x64, B.h64, MAT_P, st));
    {
        HopArgs a = hop_args(h, DWF_F64, 1, B.h64, B.xo64, MAT_HALF_Q);
        a.y = B.bo;
        a.ymode = 2;
        a.ymat = h->mat(DWF_F64, MAT_Q);
        CK(hop(h, DWF_F64, false, a, st));
    }
    CK(mix(h, DWF_F64, B.xo64, B.t64, MAT_P, st));
    for (int par = 0; par < 2; ++par) {
        HopArgs a = hop_args(h, DWF_F64, par, par ? B.h64 : B.t64, B.r64, MAT_NHALF);
        a.y = par ? B.xo64 : B.x64;
        a.ymode = 2;
        a.ymat = h->mat(DWF_F64, MAT_A5R);
        a.rin = par ? B.bo : B.be;
        a.ralpha = h->one;
        a.red = red(h, RED_STORE, par ? B.aux : B.n64);
        CK(hop(h, DWF_F64, false, a, st));
    }
    R.dapp += 2;
    CK(cudaMemcpyAsync(hs, B.cg, 3 * sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    R.S.true_residual = std::sqrt(hs[1].last + hs[2].last) / R.b5n;
    R.S.eo_residual = R.rtrue / R.btn;
    if (R.S.true_residual > p->tol && R.status == DWF_OK && R.round < 2) {
        R.round += 1;
        R.target *= 0.1;
        R.converged = false;
        R.active = true;
        int rc = sys_reliable(R, false, hs, st);
        if (rc) return rc;
        if (!R.converged) return DWF_OK;
        return sys_finish(R, b4, x4, v5, p, hs, st);
    }
    CK(launch_unpack_full(DWF_F64, B.x64, B.xo64, v5, h->eo2lex, h->Vh, h->V, h->Ls, st));
    CK(launch_project4d(v5, (double *)x4, h->V, h->Ls, st));
    h->launches += 2;
    if (R.status == DWF_OK && R.S.true_residual > p->tol) R.status = DWF_ENOTCONV;
    R.active = false;
    R.done = true;
    return DWF_OK;
}

int batch_impl(dwf_handle const *hs_in, const void *const *b4, void *const *x4, int n, const dwf_solve_params *p,
               dwf_solve_stats *stats, cudaStream_t st)
{
    auto t0 = std::chrono::steady_clock::now();
    if (n == 0) return DWF_OK;
    const int ps = p->inner_prec;
    if (ps != DWF_F64 && ps != DWF_F32 && ps != DWF_F16) return dwf_set_error(DWF_EINVAL, "bad inner precision");
    if (!(p->tol > 0) || p->max_iter < 1 || !(p->delta >= 0 && p->delta < 1) || p->check_every < 1 ||
        p->batch_wave < 0)
        return dwf_set_error(DWF_EINVAL, "bad solver parameters");
    const double delta = reliable_delta(p);
    if (p->eo_form != 0) return dwf_set_error(DWF_EINVAL, "dwf_solve_batch iterates on the first even-odd form");
    dwf_ctx *h0 = hs_in[0];
    if (!h0) return dwf_set_error(DWF_EINVAL, "NULL handle in batch");
    int Lsmax = 0;
    for (int i = 0; i < n; ++i) {
        dwf_ctx *h = hs_in[i];
        if (!h || !b4[i] || !x4[i]) return dwf_set_error(DWF_EINVAL, "NULL handle or vector in batch");
        if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
        for (int k = 0; k < 4; ++k)
            if (h->dims[k] != h0->dims[k]) return dwf_set_error(DWF_EINVAL, "batch handles differ in lattice size");
        if (h->device != h0->device) return dwf_set_error(DWF_EINVAL, "batch handles on different devices");
        if (((uintptr_t)b4[i] & 15) || ((uintptr_t)x4[i] & 15))
            return dwf_set_error(DWF_EINVAL, "vectors must be 16-byte aligned");
        Lsmax = std::max(Lsmax, h->Ls);
    }
    // order: round robin over the distinct handles, so that every wave mixes them
    std::vector<int> order;
    std::vector<dwf_ctx *> uniq_handles;
    {
        std::vector<dwf_ctx *> &uniq = uniq_handles;
        std::vector<std::vector<int>> q;
        for (int i = 0; i < n; ++i) {
            size_t u = std::find(uniq.begin(), uniq.end(), hs_in[i]) - uniq.begin();
            if (u == uniq.size()) {
                uniq.push_back(hs_in[i]);
                q.emplace_back();
            }
            q[u].push_back(i);
        }
        for (size_t r = 0; order.size() < (size_t)n; ++r)
            for (auto &v : q)
                if (r < v.size()) order.push_back(v[r]);
    }
    long long launches0 = 0;
    for (dwf_ctx *h : uniq_handles) launches0 += h->launches;
    const int V = h0->V, Vh = h0->Vh;
    const size_t shared = shared_bytes(V, Vh, Lsmax);
    size_t freeb = 0, totalb = 0;
    CK(cudaMemGetInfo(&freeb, &totalb));
    const size_t reserve = std::max((size_t)2 << 30, totalb / 20);
    const size_t budget = freeb > shared + reserve ? freeb - shared - reserve : 0;
    // waves
    std::vector<std::pair<int, int>> waves;   // [begin, end) in `order`
    for (int k = 0; k < n;) {
        size_t used = 0;
        int e = k;
        while (e < n && (p->batch_wave == 0 || e - k < p->batch_wave)) {
            const size_t need = system_bytes(hs_in[order[e]], ps);
            if (used + need > budget) break;
            used += need;
            ++e;
        }
        if (e == k) return dwf_set_error(DWF_ENOMEM, "one system of the batch does not fit in device memory");
        waves.push_back({k, e});
        k = e;
    }

    std::vector<SysRun> runs(n);
    CgScalars *hs_pinned = nullptr;
    CK(cudaMallocHost(&hs_pinned, sizeof(CgScalars) * (3 * (size_t)n + 4)));
    cudaStream_t cap = nullptr;
    int worst = DWF_OK;
    int rc = DWF_OK;
    long long launches = 0;
    const int N = p->check_every;
    Arena A;
    int *skip_host = nullptr;

    auto cleanup = [&]() {
        if (A.base) cudaFree(A.base);
        A.base = nullptr;
        if (cap) cudaStreamDestroy(cap);
        cap = nullptr;
        if (hs_pinned) cudaFreeHost(hs_pinned);
        hs_pinned = nullptr;
        if (skip_host) cudaFreeHost(skip_host);
        skip_host = nullptr;
    };
#define BCK(call)                                                             \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            cleanup();                                                        \
            return dwf_cuda_error(e_, #call);                                 \
        }                                                                     \
    } while (0)
#define BRC(call)                                                             \
    do {                                                                      \
        int r_ = (call);                                                      \
        if (r_) {                                                             \
            cleanup();                                                        \
            return r_;                                                        \
        }                                                                     \
    } while (0)

    BCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    BCK(cudaMallocHost(&skip_host, sizeof(int) * (size_t)n));
    for (auto &w : waves) {
        const int nw = w.second - w.first;
        size_t bytes = shared + 4096;
        for (int k = w.first; k < w.second; ++k) bytes += system_bytes(hs_in[order[k]], ps);
        bytes += round256(sizeof(int) * (size_t)nw);
        A.size = bytes;
        A.used = 0;
        BCK(cudaMalloc(&A.base, bytes));
        // shared FP64 temporaries
        FieldRef be = A.field(DWF_F64, Vh, Lsmax), bo = A.field(DWF_F64, Vh, Lsmax);
        FieldRef r64 = A.field(DWF_F64, Vh, Lsmax), t64 = A.field(DWF_F64, Vh, Lsmax);
        FieldRef h64 = A.field(DWF_F64, Vh, Lsmax), xo64 = A.field(DWF_F64, Vh, Lsmax);
        double *v5 = (double *)A.take((size_t)V * Lsmax * 24 * 8);
        int *skip_dev = (int *)A.take(sizeof(int) * (size_t)nw);
        if (!v5 || !skip_dev || !xo64.v) {
            cleanup();
            return dwf_set_error(DWF_ENOMEM, "batch arena");
        }
        // per-system state
        for (int k = w.first; k < w.second; ++k) {
            SysRun &R = runs[k];
            R.h = hs_in[order[k]];
            R.idx = order[k];
            std::memset(&R.S, 0, sizeof(R.S));
            dwf_ctx *h = R.h;
            Bufs &B = R.B;
            B.ps = ps;
            B.xp = ps == DWF_F64 ? DWF_F64 : DWF_F32;
            B.be = be, B.bo = bo, B.r64 = r64, B.t64 = t64, B.h64 = h64, B.xo64 = xo64;
            B.bt = A.field(DWF_F64, Vh, h->Ls);
            B.x64 = A.field(DWF_F64, Vh, h->Ls);
            B.p = A.field(ps, Vh, h->Ls);
            B.ph = A.field(ps, Vh, h->Ls);
            B.t = A.field(ps, Vh, h->Ls);
            B.wh = A.field(ps, Vh, h->Ls);
            B.u = A.field(ps, Vh, h->Ls);
            B.rs = A.field(ps, Vh, h->Ls);
            B.xs = A.field(B.xp, Vh, h->Ls);
            CgScalars *sc = (CgScalars *)A.take(3 * sizeof(CgScalars));
            R.partials = (double *)A.take(((size_t)Vh + 8192) * 8);
            R.counter = (unsigned *)A.take(256);
            if (!sc || !R.partials || !R.counter || !B.xs.v) {
                cleanup();
                return dwf_set_error(DWF_ENOMEM, "batch arena");
            }
            B.cg = sc, B.n64 = sc + 1, B.aux = sc + 2;
            BCK(cudaMemsetAsync(sc, 0, 3 * sizeof(CgScalars), st));
            BCK(cudaMemsetAsync(R.counter, 0, 256, st));
        }
        for (int k = w.first; k < w.second; ++k) {
            SysRun &R = runs[k];
            BRC(sys_prepare(R, b4[R.idx], v5, p, hs_pinned, st));
            if (R.done) {   // zero source
                BCK(cudaMemsetAsync(x4[R.idx], 0, (size_t)V * 24 * 8, st));
            } else if (R.converged) {
                BRC(sys_finish(R, b4[R.idx], x4[R.idx], v5, p, hs_pinned, st));
            }
        }
        // batched launch tables, one group per distinct Ls
        std::vector<int> lsv;
        for (int k = w.first; k < w.second; ++k)
            if (std::find(lsv.begin(), lsv.end(), runs[k].h->Ls) == lsv.end()) lsv.push_back(runs[k].h->Ls);
        struct Group {
            std::vector<int> mem;   // indices into runs
            CgUpdateArgs *ue = nullptr;
            HopArgs *k[4] = {nullptr, nullptr, nullptr, nullptr};
            CgUpdateArgs ue0;
            HopArgs k0[4];
            int ns = 0, sb = 0;
        };
        std::vector<Group> groups(lsv.size());
        for (size_t g = 0; g < lsv.size(); ++g) {
            Group &G = groups[g];
            for (int k = w.first; k < w.second; ++k)
                if (runs[k].h->Ls == lsv[g]) G.mem.push_back(k);
            const int m = (int)G.mem.size();
            std::vector<CgUpdateArgs> ue(m);
            std::vector<HopArgs> kt[4];
            for (int q = 0; q < m; ++q) {
                SysRun &R = runs[G.mem[q]];
                RedArgs ra, rb;
                ra.partials = rb.partials = R.partials;
                ra.counter = rb.counter = R.counter;
                ra.scal = rb.scal = R.B.cg;
                ra.op = RED_CG_ALPHA;
                rb.op = RED_CG_BETA;
                IterArgs I = iteration_args(R.h, R.B, ra, rb);
                I.ue.skip = skip_dev + (G.mem[q] - w.first);
                ue[q] = I.ue;
                for (int j = 0; j < 4; ++j) {
                    HopArgs a = with_programs(R.h, ps, I.k[j]);
                    a.skip = I.ue.skip;
                    kt[j].push_back(a);
                }
            }
            // one mixing mode per group (the kernels are compiled per mode); the
            // dense matrices are always present, so disagreement falls back to them
            int mixm = kt[0][0].mixmode;
            for (int j = 0; j < 4; ++j)
                for (int q = 0; q < m; ++q)
                    if (kt[j][q].mixmode != mixm) mixm = 0;
            for (int j = 0; j < 4; ++j)
                for (int q = 0; q < m; ++q) kt[j][q].mixmode = mixm;
            for (int q = 0; q < m; ++q) ue[q].mixmode = (mixm == 1) ? 1 : 0;
            G.ue0 = ue[0];
            for (int j = 0; j < 4; ++j) G.k0[j] = kt[j][0];
            dwf_ctx *hg = runs[G.mem[0]].h;
            G.ns = hg->hop_var[ps] == 0 ? hg->hop_ns[ps] : 0;
            G.sb = hg->hop_var[ps] == 0 ? hg->hop_sb[ps] : 0;
            G.ue = (CgUpdateArgs *)A.take(sizeof(CgUpdateArgs) * m);
            for (int j = 0; j < 4; ++j) G.k[j] = (HopArgs *)A.take(sizeof(HopArgs) * m);
            if (!G.ue || !G.k[3]) {
                cleanup();
                return dwf_set_error(DWF_ENOMEM, "batch arena");
            }
            BCK(cudaMemcpyAsync(G.ue, ue.data(), sizeof(CgUpdateArgs) * m, cudaMemcpyHostToDevice, st));
            for (int j = 0; j < 4; ++j)
                BCK(cudaMemcpyAsync(G.k[j], kt[j].data(), sizeof(HopArgs) * m, cudaMemcpyHostToDevice, st));
        }
        auto launch_iteration = [&](cudaStream_t s2) -> cudaError_t {
            cudaError_t e;
            for (auto &G : groups) {
                const int m = (int)G.mem.size();
                if ((e = launch_cg_update_batch(ps, G.ue, m, G.ue0, s2)) != cudaSuccess) return e;
                for (int j = 0; j < 4; ++j)
                    if ((e = launch_hop_batch(ps, j >= 2, G.k[j], m, G.k0[j], G.ns, G.sb, s2)) != cudaSuccess)
                        return e;
            }
            return cudaSuccess;
        };
        cudaGraphExec_t exec = nullptr;
        if (p->use_graph) {
            BCK(cudaStreamSynchronize(st));
            cudaGraph_t g;
            BCK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            for (int k = 0; k < N; ++k) {
                cudaError_t e = launch_iteration(cap);
                if (e != cudaSuccess) {
                    cudaStreamEndCapture(cap, &g);
                    cleanup();
                    return dwf_cuda_error(e, "graph capture");
                }
            }
            BCK(cudaStreamEndCapture(cap, &g));
            cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            BCK(e);
        }
        // lock-step iteration of the wave
        for (;;) {
            int nact = 0;
            for (int k = w.first; k < w.second; ++k) {
                skip_host[k - w.first] = runs[k].active ? 0 : 1;
                nact += runs[k].active ? 1 : 0;
            }
            if (nact == 0) break;
            BCK(cudaMemcpyAsync(skip_dev, skip_host, sizeof(int) * nw, cudaMemcpyHostToDevice, st));
            if (exec) {
                cudaError_t e = cudaGraphLaunch(exec, st);
                if (e != cudaSuccess) {
                    cudaGraphExecDestroy(exec);
                    BCK(e);
                }
            } else {
                for (int k = 0; k < N; ++k) BCK(launch_iteration(st));
            }
            launches += (long long)N * 5 * (long long)groups.size();
            for (int k = w.first; k < w.second; ++k)
                BCK(cudaMemcpyAsync(&hs_pinned[3 * (k - w.first)], runs[k].B.cg, sizeof(CgScalars),
                                    cudaMemcpyDeviceToHost, st));
            BCK(cudaStreamSynchronize(st));
            for (int k = w.first; k < w.second; ++k) {
                SysRun &R = runs[k];
                if (!R.active) continue;
                const CgScalars c = hs_pinned[3 * (k - w.first)];
                R.iters += N;
                R.dapp += 2 * N;
                const double rn = std::sqrt(c.gamma);
                const bool bad = (c.flags != 0) || !std::isfinite(rn);
                CgScalars *hsl = hs_pinned + 3 * (size_t)n;   // scratch for the single-system steps
                if (bad && (c.flags & 2)) {
                    BCK(launch_zero(R.B.xp, R.B.xs, R.h->Vh, R.h->Ls, st));
                    BCK(launch_zero(ps, R.B.p, R.h->Vh, R.h->Ls, st));
                    BRC(sys_reliable(R, true, hsl, st));
                    if (++R.nru > 200) {
                        R.status = DWF_ENONFINITE;
                        R.active = false;
                    }
                } else if (bad || rn < delta * R.rmax || R.rho * rn < R.target || R.iters >= p->max_iter) {
                    BRC(sys_reliable(R, false, hsl, st));
                    if (R.nru > 1000) R.status = DWF_ENOTCONV;
                }
                if (R.status == DWF_OK && !R.converged && R.iters >= p->max_iter) R.status = DWF_ENOTCONV;
                if (R.converged || R.status != DWF_OK) {
                    R.active = false;
                    BRC(sys_finish(R, b4[R.idx], x4[R.idx], v5, p, hsl, st));
                }
            }
        }
        if (exec) cudaGraphExecDestroy(exec);
        BCK(cudaStreamSynchronize(st));
        cudaFree(A.base);
        A.base = nullptr;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    h0->launches += launches;
    long long own = 0;
    for (dwf_ctx *h : uniq_handles) own += h->launches;
    own -= launches0;
    for (auto &R : runs) {
        R.S.status = R.status;
        R.S.iterations = R.iters;
        R.S.reliable_updates = R.nru;
        R.S.d_applications = R.dapp;
        R.S.seconds = secs;
        R.S.waves = (int)waves.size();
        if (R.status > worst) worst = R.status;
    }
    for (auto &R : runs) R.S.kernel_launches = own;
    if (stats)
        for (auto &R : runs) stats[R.idx] = R.S;
    cleanup();
#undef BCK
#undef BRC
    (void)rc;
    if (worst != DWF_OK) dwf_set_error(worst, "a system of the batch did not reach the tolerance");
    return worst;
}

}  // namespace

// out = D x on FP32 even fields (K_e..K_b of the inner iteration without the
// CG updates and the final Q^T mixing)
int dwf::eo_apply_f32(dwf_ctx *h, FieldRef x, FieldRef out, cudaStream_t st)
{
    const int P = DWF_F32;
    cudaError_t e = cudaSuccess;
    FieldRef ph = h->field("na_ph", P, &e), t = h->field("na_t", P, &e);
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

// out = D^dag w on FP32 even fields (K_c, K_d of the inner iteration on Q^T w)
int dwf::eo_dag_apply_f32(dwf_ctx *h, FieldRef w, FieldRef out, cudaStream_t st)
{
    const int P = DWF_F32;
    cudaError_t e = cudaSuccess;
    FieldRef wh = h->field("nd_wh", P, &e), u = h->field("nd_u", P, &e);
    if (!wh.v || !u.v) return dwf_cuda_error(e, "workspace");
    CK(mix(h, P, w, wh, MAT_QT, st));
    HopArgs a3 = hop_args(h, P, 1, wh, u, MAT_MT);
    CK(hop(h, P, true, a3, st));
    HopArgs a4 = hop_args(h, P, 0, u, out, MAT_NPT4);
    a4.y = wh;
    a4.ymode = 2;
    a4.ymat = h->mat(P, MAT_RA5T);
    CK(hop(h, P, true, a4, st));
    return DWF_OK;
}

// out = D^dag D x on FP32 even fields: w = D x (as K_e..K_b of the inner
// iteration, without its CG updates), then D^dag w (as K_c, K_d).
int dwf::normal_apply_f32(dwf_ctx *h, FieldRef x, FieldRef out, cudaStream_t st)
{
    const int P = DWF_F32;
    cudaError_t e = cudaSuccess;
    FieldRef ph = h->field("na_ph", P, &e), t = h->field("na_t", P, &e);
    FieldRef wh = h->field("na_wh", P, &e), u = h->field("na_u", P, &e);
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

extern "C" {

void dwf_solve_params_default(dwf_solve_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->tol = 1e-10;
    p->max_iter = 20000;
    p->inner_prec = DWF_F32;
    p->delta = 0.0;   // by the inner precision (reliable_delta)
    p->check_every = 16;
    p->use_graph = 1;
    p->precond = 0;
    p->use_initial_guess = 0;
    p->verbose = 0;
    p->batch_wave = 0;
}

int dwf_solve(dwf_handle h, const void *b5, void *x5, const dwf_solve_params *p, dwf_solve_stats *stats, void *stream)
{
    if (!h || !b5 || !x5) return dwf_set_error(DWF_EINVAL, "NULL argument");
    if (h && h->slab) return dwf_set_error(DWF_EINVAL, "a slab handle applies its operator through dwf_slab_apply_eo");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    if (((uintptr_t)b5 & 15) || ((uintptr_t)x5 & 15)) return dwf_set_error(DWF_EINVAL, "vectors must be 16-byte aligned");
    dwf_solve_params def;
    dwf_solve_params_default(&def);
    return solve_impl(h, b5, x5, p ? p : &def, stats, (cudaStream_t)stream);
}

int dwf_precond_fcg(dwf_handle h, const void *b, void *x, double tol, int max_iter, int plain, double *history,
                    int *iters, void *stream)
{
    if (!h || !b || !x) return dwf_set_error(DWF_EINVAL, "NULL argument");
    if (h && h->slab) return dwf_set_error(DWF_EINVAL, "a slab handle applies its operator through dwf_slab_apply_eo");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    if (!(tol > 0) || max_iter < 0) return dwf_set_error(DWF_EINVAL, "bad tol or max_iter");
    if (!plain && !h->net) return dwf_set_error(DWF_EINVAL, "no preconditioner (dwf_precond_init or dwf_precond_train)");
    if (((uintptr_t)b & 15u) || ((uintptr_t)x & 15u)) return dwf_set_error(DWF_EINVAL, "vectors must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    FieldRef b32 = h->field("pf_b32", DWF_F32, &e), x32 = h->field("pf_x32", DWF_F32, &e);
    FieldRef x64 = h->field("pf_x64", DWF_F64, &e);
    if (!b32.v || !x32.v || !x64.v) return dwf_cuda_error(e, "workspace");
    CK(launch_pack_eo(DWF_F32, (const double *)b, b32, h->Vh, h->Ls, st));
    CK(launch_zero(DWF_F32, x32, h->Vh, h->Ls, st));
    h->launches += 2;
    bool pl = plain != 0;
    int it = 0, napp = 0, nfall = 0, dapp = 0;
    int rc = fcg_cycle(h, b32, x32, tol, max_iter, pl, it, napp, nfall, dapp, history, st);
    if (rc) return rc;
    CK(launch_convert(DWF_F32, x32, DWF_F64, x64, h->Vh, h->Ls, st));
    CK(launch_unpack_eo(DWF_F64, x64, (double *)x, h->Vh, h->Ls, st));
    h->launches += 2;
    CK(cudaStreamSynchronize(st));
    if (iters) *iters = it;
    if (nfall) return dwf_set_error(DWF_EBREAKDOWN, "the preconditioner lost positivity");
    return DWF_OK;
}

int dwf_propagator_host(dwf_handle h, const double *b4_host, double *x4_host, const dwf_solve_params *p,
                        dwf_solve_stats *stats, void *stream)
{
    if (!h || !b4_host || !x4_host) return dwf_set_error(DWF_EINVAL, "NULL argument");
    if (h && h->slab) return dwf_set_error(DWF_EINVAL, "a slab handle applies its operator through dwf_slab_apply_eo");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    const size_t b4b = (size_t)h->V * 24 * 8, b5b = b4b * h->Ls;
    void *b4 = h->ws("pr_b4", b4b, &e);
    void *x4 = h->ws("pr_x4", b4b, &e);
    void *b5 = h->ws("pr_b5", b5b, &e);
    void *x5 = h->ws("pr_x5", b5b, &e);
    if (!b4 || !x4 || !b5 || !x5) return dwf_cuda_error(e, "workspace");
    CK(cudaMemcpyAsync(b4, b4_host, b4b, cudaMemcpyHostToDevice, st));
    int rc = dwf_source_5d(h, b4, b5, stream);
    if (rc) return rc;
    dwf_solve_params def;
    dwf_solve_params_default(&def);
    dwf_solve_params q = p ? *p : def;
    q.use_initial_guess = 0;
    rc = solve_impl(h, b5, x5, &q, stats, st);
    if (rc != DWF_OK && rc != DWF_ENOTCONV) return rc;
    int rc2 = dwf_project_4d(h, x5, x4, stream);
    if (rc2) return rc2;
    CK(cudaMemcpyAsync(x4_host, x4, b4b, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return rc;
}

int dwf_solve_batch(dwf_handle const *hs, const void *const *b4, void *const *x4, int n, const dwf_solve_params *p,
                    dwf_solve_stats *stats, void *stream)
{
    if (n < 0 || (n > 0 && (!hs || !b4 || !x4))) return dwf_set_error(DWF_EINVAL, "NULL argument");
    for (int i = 0; i < n; ++i)
        if (hs[i] && hs[i]->slab)
            return dwf_set_error(DWF_EINVAL, "a slab handle applies its operator through dwf_slab_apply_eo");
    dwf_solve_params def;
    dwf_solve_params_default(&def);
    return batch_impl(hs, b4, x4, n, p ? p : &def, stats, (cudaStream_t)stream);
}

int dwf_time_iteration(dwf_handle h, int prec, int reps, int flush_l2, double *us5, double *bytes5, void *stream)
{
    if (!h || reps < 1 || !us5 || !bytes5) return dwf_set_error(DWF_EINVAL, "bad argument");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    if (prec != DWF_F64 && prec != DWF_F32 && prec != DWF_F16) return dwf_set_error(DWF_EINVAL, "bad precision");
    cudaStream_t st = (cudaStream_t)stream;
    Bufs B;
    int rc = get_bufs(h, prec, B);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    const size_t flush_bytes = (size_t)512 << 20;
    void *flush = nullptr;
    if (flush_l2) {
        flush = h->ws("th_flush", flush_bytes, &e);
        if (!flush) return dwf_cuda_error(e, "workspace");
    }
    const FieldRef inner[] = {B.p, B.ph, B.t, B.wh, B.u, B.rs};
    const size_t fb = field_bytes(prec, h->Vh, h->Ls), sb = scale_bytes(prec, h->Vh, h->Ls);
    CgScalars c0;
    std::memset(&c0, 0, sizeof c0);
    c0.gamma = 1.0;
    c0.alpha = 0.5;   // a pending x update, as in every iteration but the first
    const IterArgs I = iteration_args(h, B, red(h, RED_CG_ALPHA, B.cg), red(h, RED_CG_BETA, B.cg));
    cudaEvent_t ev[6];
    for (auto &x : ev) CK(cudaEventCreate(&x));
    double tot[5] = {0, 0, 0, 0, 0};
    // two untimed iterations, then reps timed ones, each from the same synthetic
    // state: inner fields of bytes 0x3c, FP16 scales of bytes 0x3f, x accumulator 0
    for (int r = -2; r < reps; ++r) {
        for (const FieldRef &f : inner) {
            CK(cudaMemsetAsync(f.v, 0x3c, fb, st));
            if (f.scale) CK(cudaMemsetAsync(f.scale, 0x3f, sb, st));
        }
        CK(cudaMemsetAsync(B.xs.v, 0, field_bytes(B.xp, h->Vh, h->Ls), st));
        CK(cudaMemcpyAsync(B.cg, &c0, sizeof c0, cudaMemcpyHostToDevice, st));
        if (flush) CK(cudaMemsetAsync(flush, r & 0xff, flush_bytes, st));
        CK(cudaEventRecord(ev[0], st));
        CK(launch_cg_update(prec, I.ue, st));
        CK(cudaEventRecord(ev[1], st));
        for (int k = 0; k < 4; ++k) {
            CK((k == 0 || k == 2) ? hop_cg_plain(h, prec, k >= 2, I.k[k], st) : hop(h, prec, k >= 2, I.k[k], st));
            CK(cudaEventRecord(ev[k + 2], st));
        }
        CK(cudaEventSynchronize(ev[5]));
        if (r < 0) continue;
        for (int k = 0; k < 5; ++k) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
            tot[k] += ms;
        }
    }
    for (auto &x : ev) cudaEventDestroy(x);
    // algorithmic bytes: F an inner field (with its FP16 scales), X the x accumulator, L the links
    const double F = (double)fb + (prec == DWF_F16 ? (double)h->Vh * h->Ls * 4 : 0.0);
    const double X = (double)field_bytes(B.xp, h->Vh, h->Ls);
    const double L = (double)h->Vh * 8 * 18 * (prec == DWF_F64 ? 8 : (prec == DWF_F32 ? 4 : 2));
    const double by[5] = {4 * F + 2 * X, 2 * F + L, 3 * F + L, 2 * F + L, 4 * F + L};
    for (int k = 0; k < 5; ++k) {
        us5[k] = 1000.0 * tot[k] / reps;
        bytes5[k] = by[k];
    }
    h->launches += reps + 2;   // the p updates (hop() counts the hops)
    return DWF_OK;
}

}  // extern "C"
