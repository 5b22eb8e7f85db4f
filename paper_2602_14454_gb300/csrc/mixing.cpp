// Host-side construction of the fifth-direction matrices (FP64).
//
// In the chiral basis the 5D matrix of Sec. 2.2 is
//     D_DW = D_W (b + c K) + (1 - K),
// where K acts on the fifth index and the chirality only (it is the operator
// whose blocks are P_- above the diagonal, P_+ below it, and -m P_+, -m P_- in
// the corners of eq. domainwall_general).  Per chirality K is a real Ls x Ls
// matrix:
//     P_+ components: (K x)_s = x_{s-1} (s > 1),  (K x)_1  = -m x_Ls
//     P_- components: (K x)_s = x_{s+1} (s < Ls), (K x)_Ls = -m x_1
// With D_W = (4 - M0) - H/2 (eq. Wilson_matrix, H = the hopping sum):
//     site-local block  D_ee = D_oo = A5 = alpha0 + beta0 K,
//                       alpha0 = b (4 - M0) + 1, beta0 = c (4 - M0) - 1,
//     hopping blocks    D_eo = -1/2 H_eo (b + c K),  D_oe = -1/2 H_oe (b + c K).
// Neff's matrix (eq. domainwall_neff) equals D_DW R with the site-local
// R = P A P^dag = blockdiag_s(P_- + a P_+, a, ..., a, P_+ + a P_-)
// (eq. relation_to_alpha=1), i.e. per chirality
//     P_+: diag(a, ..., a, 1),   P_-: diag(1, a, ..., a).
// Every mixing the kernels apply is a product of these small matrices.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dwf_internal.h"

namespace dwf {
namespace {

using Mat = std::vector<double>;

Mat zeros(int n) { return Mat((size_t)n * n, 0.0); }
Mat eye(int n, double v = 1.0) {
    Mat m = zeros(n);
    for (int i = 0; i < n; ++i) m[(size_t)i * n + i] = v;
    return m;
}
Mat mul(const Mat &a, const Mat &b, int n) {
    Mat c = zeros(n);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            double aik = a[(size_t)i * n + k];
            if (aik == 0.0) continue;
            for (int j = 0; j < n; ++j) c[(size_t)i * n + j] += aik * b[(size_t)k * n + j];
        }
    return c;
}
Mat add(const Mat &a, double sa, const Mat &b, double sb) {
    Mat c(a.size());
    for (size_t i = 0; i < a.size(); ++i) c[i] = sa * a[i] + sb * b[i];
    return c;
}
Mat scale(const Mat &a, double s) { return add(a, s, a, 0.0); }
// row-wise coefficients: c[i][j] = sa[i] a[i][j] + sb[i] b[i][j] (the same
// arithmetic as add() when sa and sb are constant)
Mat add_rows(const Mat &a, const double *sa, const Mat &b, const double *sb, int n) {
    Mat c(a.size());
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) c[(size_t)i * n + j] = sa[i] * a[(size_t)i * n + j] + sb[i] * b[(size_t)i * n + j];
    return c;
}
Mat diag(const double *v, int n) {
    Mat d = zeros(n);
    for (int i = 0; i < n; ++i) d[(size_t)i * n + i] = v[i];
    return d;
}
Mat transpose(const Mat &a, int n) {
    Mat t = zeros(n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) t[(size_t)j * n + i] = a[(size_t)i * n + j];
    return t;
}
// Gauss-Jordan with partial pivoting; false if singular.
bool inverse(const Mat &a, int n, Mat &inv) {
    Mat w = a;
    inv = eye(n);
    double amax = 0;
    for (double v : a) amax = std::fmax(amax, std::fabs(v));
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(w[(size_t)r * n + col]) > std::fabs(w[(size_t)piv * n + col])) piv = r;
        double p = w[(size_t)piv * n + col];
        if (!(std::fabs(p) > 1e-14 * amax)) return false;
        if (piv != col)
            for (int j = 0; j < n; ++j) {
                std::swap(w[(size_t)piv * n + j], w[(size_t)col * n + j]);
                std::swap(inv[(size_t)piv * n + j], inv[(size_t)col * n + j]);
            }
        double ip = 1.0 / p;
        for (int j = 0; j < n; ++j) {
            w[(size_t)col * n + j] *= ip;
            inv[(size_t)col * n + j] *= ip;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double f = w[(size_t)r * n + col];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                w[(size_t)r * n + j] -= f * w[(size_t)col * n + j];
                inv[(size_t)r * n + j] -= f * inv[(size_t)col * n + j];
            }
        }
    }
    return true;
}
// spectral norm by power iteration on A^T A
double spectral_norm(const Mat &a, int n) {
    Mat ata = mul(transpose(a, n), a, n);
    std::vector<double> v(n, 1.0), w(n);
    double lam = 0;
    for (int it = 0; it < 500; ++it) {
        double nn = 0;
        for (int i = 0; i < n; ++i) {
            double s = 0;
            for (int j = 0; j < n; ++j) s += ata[(size_t)i * n + j] * v[j];
            w[i] = s;
            nn += s * s;
        }
        nn = std::sqrt(nn);
        if (nn == 0) return 0;
        for (int i = 0; i < n; ++i) v[i] = w[i] / nn;
        lam = nn;
    }
    return std::sqrt(lam);
}

}  // namespace

void build_programs(int L, double alpha0, double beta0, double b, double c, double mf, double M0, double a,
                    FifthMatrices &out);

bool build_fifth_matrices_s(int Ls, double M0, double mf, const double *bs, const double *cs, int form, double alpha,
                            FifthMatrices &out, std::string &err);

bool build_fifth_matrices(int Ls, double M0, double mf, double b, double c, int form, double alpha,
                          FifthMatrices &out, std::string &err)
{
    std::vector<double> bs((size_t)Ls, b), cs((size_t)Ls, c);
    return build_fifth_matrices_s(Ls, M0, mf, bs.data(), cs.data(), form, alpha, out, err);
}

// Row s of eq. (domainwall_general) holds D_+^(s) = b_s D_W + 1 and
// D_-^(s) = c_s D_W - 1, so B = diag(b) + diag(c) K and the site block
// A5 = diag(alpha0_s) + diag(beta0_s) K with alpha0_s = b_s (4 - M0) + 1,
// beta0_s = c_s (4 - M0) - 1 (both act on the chirality of their input).
bool build_fifth_matrices_s(int Ls, double M0, double mf, const double *bs, const double *cs, int form, double alpha,
                            FifthMatrices &out, std::string &err)
{
    const int n = Ls;
    out.Ls = Ls;
    bool constant = true;
    for (int s = 1; s < n; ++s) constant = constant && bs[s] == bs[0] && cs[s] == cs[0];
    if (form == DWF_NEFF && !constant) {
        err = "the Neff form takes coefficients b, c independent of s";
        return false;
    }
    std::vector<double> alpha0((size_t)n), beta0((size_t)n), src_post((size_t)n), src_y((size_t)n);
    for (int s = 0; s < n; ++s) {
        alpha0[s] = bs[s] * (4.0 - M0) + 1.0;
        beta0[s] = cs[s] * (4.0 - M0) - 1.0;
        src_post[s] = 0.5 * cs[s];
        src_y[s] = 1.0 - cs[s] * (4.0 - M0);
    }
    const double a = (form == DWF_NEFF) ? alpha : 1.0;
    double dee = 0;
    for (int chi = 0; chi < 2; ++chi) {
        Mat K = zeros(n);
        if (chi == 0) {
            for (int s = 1; s < n; ++s) K[(size_t)s * n + (s - 1)] += 1.0;
            K[(size_t)0 * n + (n - 1)] += -mf;
        } else {
            for (int s = 0; s + 1 < n; ++s) K[(size_t)s * n + (s + 1)] += 1.0;
            K[(size_t)(n - 1) * n + 0] += -mf;
        }
        Mat I = eye(n);
        Mat B = add_rows(I, bs, K, cs, n);
        Mat A5 = add_rows(I, alpha0.data(), K, beta0.data(), n);
        Mat R = eye(n, a);
        if (chi == 0) R[(size_t)(n - 1) * n + (n - 1)] = 1.0;
        else R[0] = 1.0;
        Mat Rinv = zeros(n);
        for (int i = 0; i < n; ++i) Rinv[(size_t)i * n + i] = 1.0 / R[(size_t)i * n + i];
        Mat A5inv;
        if (!inverse(A5, n, A5inv)) {
            err = "fifth-direction block A5 = alpha0 + beta0 K is singular";
            return false;
        }
        Mat P = mul(B, R, n);
        Mat Q = mul(Rinv, A5inv, n);
        Mat M = mul(B, A5inv, n);
        Mat A5R = mul(A5, R, n);
        out.A5[chi] = A5;
        out.A5inv[chi] = A5inv;
        out.B[chi] = B;
        out.R[chi] = R;
        out.Rinv[chi] = Rinv;
        out.mats[MAT_P][chi] = P;
        out.mats[MAT_PT][chi] = transpose(P, n);
        out.mats[MAT_Q][chi] = Q;
        out.mats[MAT_QT][chi] = transpose(Q, n);
        out.mats[MAT_M][chi] = M;
        out.mats[MAT_MT][chi] = transpose(M, n);
        out.mats[MAT_A5R][chi] = A5R;
        out.mats[MAT_RA5T][chi] = transpose(A5R, n);
        out.mats[MAT_NHALF][chi] = eye(n, -0.5);
        out.mats[MAT_NHALF_RBT][chi] = scale(mul(R, transpose(B, n), n), -0.5);
        out.mats[MAT_NQ4][chi] = scale(Q, -0.25);
        out.mats[MAT_NPT4][chi] = scale(transpose(P, n), -0.25);
        out.mats[MAT_ID][chi] = I;
        out.mats[MAT_HALF_Q][chi] = scale(Q, 0.5);
        out.mats[MAT_SRC_POST][chi] = diag(src_post.data(), n);
        out.mats[MAT_SRC_Y][chi] = diag(src_y.data(), n);
        out.mats[MAT_NQUARTER][chi] = eye(n, -0.25);
        out.mats[MAT_NMT4][chi] = scale(transpose(M, n), -0.25);
        dee = std::fmax(dee, spectral_norm(A5R, n));
    }
    out.dee_norm2 = dee;
    // banded matrices: nonzeros only at t = s - 1, s, s + 1 (cyclic), for both chiralities
    for (int id = 0; id < MAT_COUNT; ++id) {
        bool band = n >= 3;
        for (int chi = 0; chi < 2 && band; ++chi)
            for (int s = 0; s < n && band; ++s)
                for (int t = 0; t < n; ++t) {
                    const int d = (t - s + n) % n;
                    if (d != 0 && d != 1 && d != n - 1 && out.mats[id][chi][(size_t)s * n + t] != 0.0) {
                        band = false;
                        break;
                    }
                }
        out.band[id] = band;
    }
    // the structured programs assume coefficients independent of s
    if (constant)
        build_programs(n, alpha0[0], beta0[0], bs[0], cs[0], mf, M0, a, out);
    else
        out.structured = false;
    return true;
}

// Host copy of the device chain routine (FP64): used to check every program
// against its dense matrix before the structured path is enabled.
static void apply_prog(const FifthMatrices::Prog &p, int chi, int L, double *x)
{
    double v[LS_MAX];
    auto idx = [&](int s) { return p.up[chi] ? (L - 1 - s) : s; };
    for (int s = 0; s < L; ++s) v[s] = x[idx(s)] * p.d1[chi][idx(s)];
    if (p.inv) {
        double acc = 0;
        for (int s = 0; s < L; ++s) acc = p.kappa * acc + v[s];
        double prev = p.mneg * (acc * p.a0inv * p.corner);
        for (int s = 0; s < L; ++s) {
            v[s] = v[s] * p.a0inv + p.kappa * prev;
            prev = v[s];
        }
    }
    if (p.shift) {
        double prev = p.mneg * v[L - 1];
        for (int s = 0; s < L; ++s) {
            const double t = v[s];
            v[s] = p.s0 * t + p.s1 * prev;
            prev = t;
        }
    }
    for (int s = 0; s < L; ++s) x[idx(s)] = v[s] * p.d2[chi][idx(s)];
}

void build_programs(int L, double alpha0, double beta0, double b, double c, double mf, double M0, double a,
                    FifthMatrices &out)
{
    const double kappa = -beta0 / alpha0;
    out.structured = std::fabs(kappa) < 0.95;
    if (!out.structured) return;
    const double corner = 1.0 / (1.0 + mf * std::pow(kappa, L));
    auto R = [&](int chi, int s) { return chi == 0 ? (s == L - 1 ? 1.0 : a) : (s == 0 ? 1.0 : a); };
    enum { ONE, RD, RINV };
    struct Spec {
        int id, d1, inv, shift_kind, transposed, d2;
        double d2scale;
    };
    // shift_kind: 0 none, 1 B = b + cK, 2 A5 = alpha0 + beta0 K
    const Spec specs[] = {
        {MAT_P, RD, 0, 1, 0, ONE, 1.0},         {MAT_PT, ONE, 0, 1, 1, RD, 1.0},
        {MAT_Q, ONE, 1, 0, 0, RINV, 1.0},       {MAT_QT, RINV, 1, 0, 1, ONE, 1.0},
        {MAT_M, ONE, 1, 1, 0, ONE, 1.0},        {MAT_MT, ONE, 1, 1, 1, ONE, 1.0},
        {MAT_A5R, RD, 0, 2, 0, ONE, 1.0},       {MAT_RA5T, ONE, 0, 2, 1, RD, 1.0},
        {MAT_NHALF, ONE, 0, 0, 0, ONE, -0.5},   {MAT_NHALF_RBT, ONE, 0, 1, 1, RD, -0.5},
        {MAT_NQ4, ONE, 1, 0, 0, RINV, -0.25},   {MAT_NPT4, ONE, 0, 1, 1, RD, -0.25},
        {MAT_ID, ONE, 0, 0, 0, ONE, 1.0},       {MAT_HALF_Q, ONE, 1, 0, 0, RINV, 0.5},
        {MAT_SRC_POST, ONE, 0, 0, 0, ONE, 0.5 * c},
        {MAT_SRC_Y, ONE, 0, 0, 0, ONE, 1.0 - c * (4.0 - M0)},
        {MAT_NQUARTER, ONE, 0, 0, 0, ONE, -0.25},
        {MAT_NMT4, ONE, 1, 1, 1, ONE, -0.25},
    };
    for (const Spec &sp : specs) {
        FifthMatrices::Prog &p = out.prog[sp.id];
        std::memset(&p, 0, sizeof(p));
        p.inv = sp.inv;
        p.shift = sp.shift_kind != 0;
        p.s0 = sp.shift_kind == 1 ? b : alpha0;
        p.s1 = sp.shift_kind == 1 ? c : beta0;
        p.a0inv = 1.0 / alpha0;
        p.kappa = kappa;
        p.mneg = -mf;
        p.corner = corner;
        for (int chi = 0; chi < 2; ++chi) {
            p.up[chi] = (chi == 1) != (sp.transposed != 0);
            for (int s = 0; s < L; ++s) {
                auto val = [&](int kind) { return kind == ONE ? 1.0 : (kind == RD ? R(chi, s) : 1.0 / R(chi, s)); };
                p.d1[chi][s] = val(sp.d1);
                p.d2[chi][s] = val(sp.d2) * sp.d2scale;
            }
        }
        // the program must reproduce the dense matrix column by column
        double amax = 0, emax = 0;
        for (int chi = 0; chi < 2; ++chi)
            for (int t = 0; t < L; ++t) {
                double x[LS_MAX] = {0};
                x[t] = 1.0;
                apply_prog(p, chi, L, x);
                for (int s = 0; s < L; ++s) {
                    const double want = out.mats[sp.id][chi][(size_t)s * L + t];
                    amax = std::fmax(amax, std::fabs(want));
                    emax = std::fmax(emax, std::fabs(x[s] - want));
                }
            }
        if (!(emax <= 1e-12 * std::fmax(amax, 1e-300))) out.structured = false;
    }
}

}  // namespace dwf
