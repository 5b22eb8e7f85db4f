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
//   K_e  p = r + beta p ;  phat = P p                     (P = B R)
//   K_a  t = M H_oe phat                                  (M = B A5^-1)
//   K_b  w = p - 1/4 Q H_eo t ; what = Q^T w ; alpha = gamma / |w|^2
//   K_c  u = M^T gamma5-hop_oe what
//   K_d  r -= alpha (Q^-T what - 1/4 P^T gamma5-hop_eo u) ; x += alpha p ;
//        beta = |r|^2 / gamma ; gamma = |r|^2
// so that w = D p and D^dag w = Q^-T what - 1/4 P^T H^dag_eo M^T H^dag_oe what.
// `check_every` iterations are captured once as a CUDA graph and replayed;
// the host reads the scalars between replays.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "dwf_internal.h"

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

// One inner iteration (five launches).
cudaError_t inner_iteration(dwf_ctx *h, const Bufs &B, cudaStream_t st)
{
    const int P = B.ps;
    cudaError_t e;
    CgUpdateArgs ue;
    ue.r = B.rs;
    ue.p = B.p;
    ue.phat = B.ph;
    ue.Vh = h->Vh;
    ue.Ls = h->Ls;
    ue.mat = h->mat(P, MAT_P);
    ue.mixmode = h->mix_mode(P);
    ue.prog = h->prog(P, MAT_P);
    ue.scal = B.cg;
    h->launches += 1;
    if ((e = launch_cg_update(P, ue, st)) != cudaSuccess) return e;

    HopArgs ka = hop_args(h, P, 1, B.ph, B.t, MAT_M);
    if ((e = hop(h, P, false, ka, st)) != cudaSuccess) return e;

    HopArgs kb = hop_args(h, P, 0, B.t, B.wh, MAT_NQ4);
    kb.y = B.p;
    kb.ymode = 1;
    kb.zmat = h->mat(P, MAT_QT);
    kb.red = red(h, RED_CG_ALPHA, B.cg);
    if ((e = hop(h, P, false, kb, st)) != cudaSuccess) return e;

    HopArgs kc = hop_args(h, P, 1, B.wh, B.u, MAT_MT);
    if ((e = hop(h, P, true, kc, st)) != cudaSuccess) return e;

    HopArgs kd = hop_args(h, P, 0, B.u, B.rs, MAT_NPT4);
    kd.y = B.wh;
    kd.ymode = 2;
    kd.ymat = h->mat(P, MAT_RA5T);
    kd.rin = B.rs;
    kd.ralpha = &B.cg->alpha;
    kd.xacc = B.xs.v;
    kd.xdir = B.p;
    kd.xalpha = &B.cg->alpha;
    kd.red = red(h, RED_CG_BETA, B.cg);
    return hop(h, P, true, kd, st);
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

// rs = D^dag r64 evaluated in the inner precision; |rs|^2 -> n64->last
cudaError_t normal_residual(dwf_ctx *h, const Bufs &B, cudaStream_t st)
{
    const int P = B.ps;
    cudaError_t e;
    h->launches += 1;
    if ((e = launch_convert(DWF_F64, B.r64, P, B.rs, h->Vh, h->Ls, st)) != cudaSuccess) return e;
    if ((e = mix(h, P, B.rs, B.ph, MAT_QT, st)) != cudaSuccess) return e;
    HopArgs a1 = hop_args(h, P, 1, B.ph, B.u, MAT_MT);
    if ((e = hop(h, P, true, a1, st)) != cudaSuccess) return e;
    HopArgs a2 = hop_args(h, P, 0, B.u, B.rs, MAT_NPT4);
    a2.y = B.rs;
    a2.ymode = 1;
    a2.red = red(h, RED_STORE, B.n64);
    return hop(h, P, true, a2, st);
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

void dwf_solver_release(dwf_ctx *h)
{
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
    if (!(p->tol > 0) || p->max_iter < 1 || !(p->delta > 0 && p->delta < 1) || p->check_every < 1)
        return dwf_set_error(DWF_EINVAL, "bad solver parameters");
    Bufs B;
    int rc = get_bufs(h, ps, B);
    if (rc) return rc;
    SolverExtra &X = g_extra[h];
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

    double target = p->tol * b5n / h->fm.dee_norm2 * 0.5;
    const int N = p->check_every;
    int iters = 0, nru = 0, dapp = 0;
    double rtrue = 0, rho = 1, rmax = 0;
    bool converged = false;
    int status = DWF_OK;

    // graph of N inner iterations
    GraphCache &G = X.graph;
    char keybuf[256];
    std::snprintf(keybuf, sizeof keybuf, "%d/%d/%p/%p/%p/%d", ps, N, B.p.v, B.rs.v, B.xs.v, p->use_graph);
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

    auto reliable = [&](bool first) -> int {
        if (!first) {
            CK(launch_accum_x((double *)B.x64.v, B.xs.v, B.xp, h->Vh, h->Ls, st));
            h->launches += 1;
        }
        CK(true_residual(h, B, st));
        CgScalars n64;
        CK(cudaMemcpyAsync(&hs[1], B.n64, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        n64 = hs[1];
        dapp += 1;
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
        rho = (rn > 0) ? rtrue / rn : 1.0;
        nru += first ? 0 : 1;
        return DWF_OK;
    };

    for (int round = 0; round < 3 && status == DWF_OK; ++round) {
        converged = false;
        if ((rc = reliable(round == 0 && !p->use_initial_guess))) return rc;
        while (!converged) {
            if (iters >= p->max_iter) {
                status = DWF_ENOTCONV;
                break;
            }
            if (p->use_graph) {
                CK(cudaGraphLaunch(G.exec, st));
                h->launches += 5LL * N;
            } else {
                for (int k = 0; k < N; ++k) CK(inner_iteration(h, B, st));
            }
            iters += N;
            dapp += 2 * N;
            if ((rc = read_scalars(B, hs, 1, st))) return rc;
            const double rn = std::sqrt(hs[0].gamma);
            const bool bad = (hs[0].flags != 0) || !std::isfinite(rn);
            if (p->verbose)
                std::fprintf(stderr, "[dwf] it %d |r_n| %.3e est %.3e target %.3e\n", iters, rn, rho * rn, target);
            if (bad || rn < p->delta * rmax || rho * rn < target || iters >= p->max_iter) {
                if (bad && hs[0].flags & 2) {
                    // non-finite inner state: restart from the FP64 iterate
                    CK(launch_zero(B.xp, B.xs, h->Vh, h->Ls, st));
                    CK(launch_zero(ps, B.p, h->Vh, h->Ls, st));
                    if ((rc = reliable(true))) return rc;
                    if (nru > 200) return dwf_set_error(DWF_ENONFINITE, "inner iteration keeps producing NaN");
                    ++nru;
                    continue;
                }
                if ((rc = reliable(false))) return rc;
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
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S;
    if (status != DWF_OK) dwf_set_error(status, "solver did not reach the tolerance");
    return status;
}

extern "C" {

void dwf_solve_params_default(dwf_solve_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->tol = 1e-10;
    p->max_iter = 20000;
    p->inner_prec = DWF_F32;
    p->delta = 0.1;
    p->check_every = 16;
    p->use_graph = 1;
    p->precond = 0;
    p->use_initial_guess = 0;
    p->verbose = 0;
}

int dwf_solve(dwf_handle h, const void *b5, void *x5, const dwf_solve_params *p, dwf_solve_stats *stats, void *stream)
{
    if (!h || !b5 || !x5) return dwf_set_error(DWF_EINVAL, "NULL argument");
    if (!h->has_gauge) return dwf_set_error(DWF_ENOGAUGE, "dwf_set_gauge has not been called");
    if (((uintptr_t)b5 & 15) || ((uintptr_t)x5 & 15)) return dwf_set_error(DWF_EINVAL, "vectors must be 16-byte aligned");
    dwf_solve_params def;
    dwf_solve_params_default(&def);
    return solve_impl(h, b5, x5, p ? p : &def, stats, (cudaStream_t)stream);
}

int dwf_propagator_host(dwf_handle h, const double *b4_host, double *x4_host, const dwf_solve_params *p,
                        dwf_solve_stats *stats, void *stream)
{
    if (!h || !b4_host || !x4_host) return dwf_set_error(DWF_EINVAL, "NULL argument");
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
    if (!hs || !b4 || !x4 || n < 0) return dwf_set_error(DWF_EINVAL, "NULL argument");
    int worst = DWF_OK;
    for (int i = 0; i < n; ++i) {
        dwf_handle h = hs[i];
        if (!h) return dwf_set_error(DWF_EINVAL, "NULL handle in batch");
        cudaError_t e = cudaSuccess;
        const size_t b5b = (size_t)h->V * 24 * 8 * h->Ls;
        void *b5 = h->ws("bt_b5", b5b, &e);
        void *x5 = h->ws("bt_x5", b5b, &e);
        if (!b5 || !x5) return dwf_cuda_error(e, "workspace");
        int rc = dwf_source_5d(h, b4[i], b5, stream);
        if (rc) return rc;
        rc = dwf_solve(h, b5, x5, p, stats ? stats + i : nullptr, stream);
        if (rc != DWF_OK && rc != DWF_ENOTCONV) return rc;
        if (rc > worst) worst = rc;
        rc = dwf_project_4d(h, x5, x4[i], stream);
        if (rc) return rc;
    }
    return worst;
}

}  // extern "C"
