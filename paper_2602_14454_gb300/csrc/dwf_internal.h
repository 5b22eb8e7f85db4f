// Internal declarations of the GB300 domain-wall library (not part of the ABI).
//
// Data layout in device memory
// ----------------------------
// Every 5D field lives as two parity halves (Sec. 2.3: 4D even-odd split).
// One half holds Vh = V/2 four-dimensional sites; each site carries Ls slices
// of 24 reals (4 spins x 3 colours x re/im; spins 0,1 are the P_+ chirality,
// spins 2,3 the P_- chirality).  The 24 reals of a (site, s) pair are cut into
// G vectors of 16 bytes, and vector g of slice s of site i sits at
//        ((i * G + g) * Ls + s)            (16-byte units)
// so that the Ls slices of one site are adjacent: a warp that works on
// consecutive (site, s) pairs reads 16-byte vectors that are consecutive in
// memory (fully coalesced), and all Ls slices of a site share its links.
//   FP64: G = 12 (double2),  FP32: G = 6 (float4),
//   FP16: G = 3 (8 halves) plus one FP32 scale per (site, s) = max |real|,
//         stored [site][Ls rounded up to a multiple of 4].
// Links: for each output parity p, a table [Vh][8][18 reals]: directions
// 0..3 hold U_mu(x), directions 4..7 hold U_mu(x-mu)^dag, with the fermion
// boundary phase folded in; FP64, FP32 and FP16 copies.
// Neighbour table: [2][Vh][8] int32, the index (in the other parity) of x+mu
// (d < 4) and x-mu (d >= 4).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "dwf.h"

namespace dwf {

constexpr int LS_MAX = 32;

// Per-chirality Ls x Ls matrices of the fifth direction used by the kernels.
// K_+ / K_- are the chirality blocks of the fifth-direction hop, B = b + cK,
// A5 = alpha0 + beta0 K (site-local block), R = Neff factor (Sec. 2.3).
enum MatId {
    MAT_P = 0,       // B R                 (right factor of D_oe, D_eo)
    MAT_PT,          // (B R)^T
    MAT_Q,           // R^-1 A5^-1          (D_ee^-1)
    MAT_QT,          // (R^-1 A5^-1)^T
    MAT_M,           // B A5^-1             (= B R D_oo^-1)
    MAT_MT,          // (B A5^-1)^T
    MAT_A5R,         // A5 R                (D_ee)
    MAT_RA5T,        // R A5^T              (D_ee^dag)
    MAT_NHALF,       // -1/2
    MAT_NHALF_RBT,   // -1/2 R B^T
    MAT_NQ4,         // -1/4 R^-1 A5^-1
    MAT_NPT4,        // -1/4 (B R)^T
    MAT_ID,          // 1
    MAT_HALF_Q,      // +1/2 R^-1 A5^-1
    MAT_SRC_POST,    // c/2                 (hop part of 1 - c D_W, 5D source)
    MAT_SRC_Y,       // 1 - c (4 - M0)      (diagonal part of 1 - c D_W)
    MAT_NQUARTER,    // -1/4                (second even-odd form)
    MAT_NMT4,        // -1/4 (B A5^-1)^T    (its adjoint)
    MAT_COUNT
};

// CG scalars kept on the device (one set per system).
struct CgScalars {
    double gamma;   // |r|^2 of the normal-equation residual
    double alpha;   // step length
    double beta;    // direction update
    double wn2;     // |D p|^2
    double last;    // last reduction result (RED_STORE)
    int flags;      // bit 0: breakdown, bit 1: non-finite
    int pad;
};

enum RedOp { RED_NONE = 0, RED_STORE = 1, RED_CG_ALPHA = 2, RED_CG_BETA = 3, RED_GAMMA = 4 };

// A field in internal layout; scale is non-null for FP16 fields only.
struct FieldRef {
    void *v = nullptr;
    float *scale = nullptr;
};

struct RedArgs {
    double *partials = nullptr;   // one slot per block
    unsigned *counter = nullptr;  // zero between launches (the last block resets it)
    int op = RED_NONE;
    CgScalars *scal = nullptr;
};

// One launch of the even-odd hopping stencil with fused fifth-direction
// mixing and epilogue:
//   h      = H in                    (Wilson hop, eq. Wilson_matrix without the
//                                     1/2 and the diagonal; DAG: gamma5 H gamma5)
//   o      = Post h + Y y            (Post, Y per-chirality Ls x Ls; Y optional,
//                                     ymode 1 = identity, 2 = dense)
//   if rin: o = rin - (*ralpha) o    (residual form), and, if xacc, xacc += (*xalpha) xdir
//   stored = zmat ? Z o : o          (the norm is taken of o)
struct HopArgs {
    FieldRef in, out, y, rin;
    const void *gauge = nullptr;   // [Vh][8][18] for the output parity
    const int *nbr = nullptr;      // [Vh][8] for the output parity
    int Vh = 0, Ls = 0;
    const void *post = nullptr;    // [2][Ls][Ls] transposed, compute precision
    const void *ymat = nullptr;
    int ymode = 0;
    const void *zmat = nullptr;
    const double *ralpha = nullptr;
    void *xacc = nullptr;          // accumulator field (FP64 for FP64, else FP32)
    FieldRef xdir;
    const double *xalpha = nullptr;
    RedArgs red;
    int *err = nullptr;            // bit 0 set when a bounded device wait gave up
    int ext[4] = {0, 0, 0, 0};     // half-lattice extents (Lx/2, Ly, Lz, Lt): blocked hop variant
    int mixmode = 0;               // 0 dense matrices, 1 structured programs (MixProg), 2 tensor-core product
    const void *post_prog = nullptr, *y_prog = nullptr, *z_prog = nullptr;
    const int *skip = nullptr;     // batched launches: the system is left untouched while *skip != 0
    int post_band = 0, y_band = 0, z_band = 0;   // the matrix is cyclic tridiagonal (dense mode reads 3 per row)
    int zblock = 0;                // sweep the lattice in columns of zblock z-planes (0: index order)
};

struct MixArgs {
    FieldRef in, out;
    int Vh = 0, Ls = 0;
    const void *mat = nullptr;     // [2][Ls][Ls] transposed
    int mixmode = 0;
    const void *prog = nullptr;
    int band = 0;
    int *err = nullptr;            // bit 0 set when a bounded device wait gave up (tensor-core form)
};

// p = r + beta p ; phat = P p   (or with init: p = r)
struct CgUpdateArgs {
    FieldRef r, p, phat;
    int Vh = 0, Ls = 0;
    const void *mat = nullptr;
    const CgScalars *scal = nullptr;
    int init = 0;
    int mixmode = 0;
    const void *prog = nullptr;
    const int *skip = nullptr;     // batched launches: the system is left untouched while *skip != 0
    int band = 0;
    // if set, xacc += scal->alpha * p (p before its update): the x update of the
    // previous CG iteration, deferred to this launch, which reads p anyway
    // (FP64 accumulator for FP64 fields, else FP32)
    void *xacc = nullptr;
};

// Opt a kernel in to more than 48 KB of dynamic shared memory, once per device
// (`done` holds one bit per device ordinal < 64).
template <typename K>
inline cudaError_t smem_optin(K *kernel, int bytes, unsigned long long &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done |= bit;
    return e;
}

// ------------------------------------------------------------ launchers
// prec: DWF_F64 / DWF_F32 / DWF_F16 (template dispatch inside)
// var: 0 direct neighbour loads, 3 persistent sweep, 4 4D-blocked tiles, 5 FP16 projection
// arithmetic (1 and 2 select the default); ns: fifth-direction
// slices per thread (1, or 2 when Ls is even); sb: sites per CTA.
// var < 0 / ns <= 0 / sb <= 0 pick the defaults.
cudaError_t launch_hop(int prec, bool dag, const HopArgs &a, int var, int ns, int sb, cudaStream_t st);
int hop_default_variant(int prec);
int hop_default_ns(int prec, int Ls);
int hop_default_sb(int prec, int Ls, int ns);
cudaError_t launch_mix(int prec, const MixArgs &a, cudaStream_t st);
// the same on the tensor cores (tcgen05, TMEM; FP32 and FP16 fields, Ls <= 32)
cudaError_t launch_mix_tc(int prec, const MixArgs &a, cudaStream_t st);
cudaError_t launch_cg_update(int prec, const CgUpdateArgs &a, cudaStream_t st);
// Batched launches over nsys systems with equal Ls (tables in device memory;
// a0: host copy of one entry, for Ls, Vh and the mixing mode): the direct hop
// with (ns, sb) tiling, and the CG update.
cudaError_t launch_hop_batch(int prec, bool dag, const HopArgs *tab, int nsys, const HopArgs &a0, int ns, int sb,
                             cudaStream_t st);
cudaError_t launch_cg_update_batch(int prec, const CgUpdateArgs *tab, int nsys, const CgUpdateArgs &a0,
                                   cudaStream_t st);

// canonical complex-double field <-> internal halves
// full: canon [s][lex][12 cplx]; eo: canon [s][i][12 cplx] of parity `par` only
cudaError_t launch_pack_full(int prec, const double *canon, FieldRef even, FieldRef odd, const int *eo2lex,
                             int Vh, int V, int Ls, cudaStream_t st);
cudaError_t launch_unpack_full(int prec, FieldRef even, FieldRef odd, double *canon, const int *eo2lex,
                               int Vh, int V, int Ls, cudaStream_t st);
cudaError_t launch_pack_eo(int prec, const double *canon, FieldRef f, int Vh, int Ls, cudaStream_t st);
cudaError_t launch_unpack_eo(int prec, FieldRef f, double *canon, int Vh, int Ls, cudaStream_t st);

// precision conversion between internal fields of the same parity
cudaError_t launch_convert(int prec_in, FieldRef in, int prec_out, FieldRef out, int Vh, int Ls, cudaStream_t st);
// x64 += xs (xs: FP64 if xs_prec == DWF_F64 else FP32); then xs = 0
// x64 += xs + (*alpha) p (the deferred x update, in the accumulator's
// precision; alpha may be null), then xs = 0
cudaError_t launch_accum_x(double *x64, void *xs, int xs_prec, FieldRef p, int p_prec, const double *alpha, int Vh,
                           int Ls, cudaStream_t st);
// norm^2 of an internal field, reduced with op into scal (or partial sums)
cudaError_t launch_norm2(int prec, FieldRef f, int Vh, int Ls, const RedArgs &red, cudaStream_t st);
cudaError_t launch_zero(int prec, FieldRef f, int Vh, int Ls, cudaStream_t st);

// gauge and index tables
cudaError_t launch_build_tables(const int dims[4], int *nbr, int *eo2lex, cudaStream_t st);
cudaError_t launch_pack_gauge(const double *U, const int dims[4], const int bc[4], const int *eo2lex,
                              const int *nbr, void *g64, void *g32, void *g16, cudaStream_t st);

// 4D source / projection on canonical 5D fields (FP64)
cudaError_t launch_project4d(const double *x5, double *x4, int V, int Ls, cudaStream_t st);
cudaError_t launch_chiral_embed(const double *b4, double *b5, int V, int Ls, cudaStream_t st);

// bytes of one internal half field
size_t field_bytes(int prec, int Vh, int Ls);
size_t scale_bytes(int prec, int Vh, int Ls);

// ------------------------------------------------------------ host side
struct FifthMatrices {
    int Ls;
    // row-major Ls x Ls, per chirality (0: P_+, 1: P_-)
    std::vector<double> A5[2], A5inv[2], B[2], R[2], Rinv[2];
    std::vector<double> mats[MAT_COUNT][2];
    double dee_norm2 = 0;   // spectral norm of D_ee (max over chiralities)
    // nonzeros only on the cyclic tridiagonal (t = s - 1, s, s + 1): the dense
    // mixing then reads three coefficients per row (P, P^T, A5 R, diagonals)
    bool band[MAT_COUNT] = {};
    // structured form of every matrix (see MixProg); valid when `structured`
    bool structured = false;
    struct Prog {
        int inv, shift, up[2];
        double s0, s1, a0inv, kappa, mneg, corner;
        double d1[2][LS_MAX], d2[2][LS_MAX];
    } prog[MAT_COUNT];
};

// Structured fifth-direction mixing, applied along one chain x_0..x_{Ls-1}
// (one real component of one site, all slices) of chirality chi:
//   x <- d1 * x ;  if inv: x <- A5^-1 x ;  if shift: x <- (s0 + s1 K) x ;  x <- d2 * x
// where K is the chirality's fifth-direction hop and "up[chi]" tells whether
// it reads x_{s+1} (with the corner -m x_0 at s = Ls-1) or x_{s-1} (corner
// -m x_{Ls-1} at s = 0); transposed matrices flip the direction.  A5^-1 uses
// the closed form of the bidiagonal-plus-corner inverse: with
// kappa = -beta0/alpha0, x_last = (sum_t kappa^(Ls-1-t) v_t / alpha0) / (1 + m kappa^Ls),
// then the forward recurrence x_s = v_s / alpha0 + kappa x_{s-1} from
// x_{-1} = -m x_last.  Stable for |kappa| < 1.
template <typename R>
struct MixProg {
    int inv, shift, up[2];
    R s0, s1, a0inv, kappa, mneg, corner;
    R d1[2][LS_MAX], d2[2][LS_MAX];
};

struct NetState;   // learned preconditioner of a handle (precond.cu)

// Flexible-CG helpers (precond.cu, solver.cu): FP32 even fields.
cudaError_t launch_vdot(FieldRef x, FieldRef y, int Vh, int Ls, const RedArgs &red, cudaStream_t st);   // Re <x, y>
cudaError_t launch_vaxpby(float a, FieldRef x, float b, FieldRef y, int Vh, int Ls, cudaStream_t st);  // y = a x + b y

// Builds every matrix above; returns false when A5 is singular.
bool build_fifth_matrices(int Ls, double M0, double mf, double b, double c, int form, double alpha,
                          FifthMatrices &out, std::string &err);

}  // namespace dwf

// The handle.
struct dwf_ctx {
    int dims[4];
    int bc[4];
    int Ls;
    double M0, mf, b, c, alpha;
    int form;
    int V, Vh;
    int device;
    dwf::FifthMatrices fm;
    void *mats_dev[3] = {nullptr, nullptr, nullptr};   // double / float / float copies (F16 uses float)
    void *progs_dev[2] = {nullptr, nullptr};           // MixProg<double>[MAT_COUNT], MixProg<float>[MAT_COUNT]
    int mixmode[3] = {-1, -1, -1};    // fifth-direction mixing per precision: 0 dense, 1 structured, 2 tensor cores, -1 default
    int mix_mode(int prec) const;
    const void *prog(int prec, int id) const;
    int *nbr = nullptr;       // [2][Vh][8]
    int *eo2lex = nullptr;    // [2][Vh]
    void *gauge[3] = {nullptr, nullptr, nullptr};      // per precision, [2][Vh][8][18]
    bool has_gauge = false;
    double *partials = nullptr;
    unsigned *counter = nullptr;
    dwf::CgScalars *scal = nullptr;   // scratch scalars for apply/norm calls
    double *one = nullptr;            // device constant 1.0
    std::map<std::string, std::pair<void *, size_t>> work;
    size_t bytes = 0;
    long long launches = 0;           // device kernels launched through this handle
    int hop_var[3] = {-1, -1, -1};    // hop variant per precision (-1 = default), set by the autotuner
    int hop_ns[3] = {0, 0, 0};        // hop tiling per precision (0 = default)
    int hop_sb[3] = {0, 0, 0};
    int sweep_zb[3] = {-1, -1, -1};   // hop sweep columns per precision (dwf_set_sweep; -1 automatic)
    // time slab of a decomposed lattice (dwf_create_slab): global extents, first global
    // time slice, and the ghost rows appended to every field (two faces of Vh/nt sites)
    int slab = 0;
    int gdims[4] = {0, 0, 0, 0};
    int t0 = 0;
    int ghost = 0;
    // 5D even-odd split available (standard form, every c_s = 0, even Ls): 1 / a0_s on the device
    int eo5 = 0;
    double *inv_a0 = nullptr;
    dwf::NetState *net = nullptr;     // learned preconditioner (dwf_precond_*)
    int *errflag() const { return &scal[7].flags; }

    const void *mat(int prec, int id) const;
    const void *gauge_for(int prec, int out_par) const;
    const int *nbr_for(int out_par) const { return nbr + (size_t)out_par * Vh * 8; }
    // named workspace buffer (allocated on first use, grown if needed)
    void *ws(const std::string &name, size_t bytes_needed, cudaError_t *err);
    dwf::FieldRef field(const std::string &name, int prec, cudaError_t *err);
};

namespace dwf {
// the handle's network on FP32 even fields: which = 0 N, 1 N^dag, 2 M = N N^dag
int net_apply_f32(dwf_ctx *h, FieldRef r, FieldRef z, cudaStream_t st, int which = 2);
// out = D^dag D x / out = D x with D the even-odd matrix (FP32 even fields)
int normal_apply_f32(dwf_ctx *h, FieldRef x, FieldRef out, cudaStream_t st);
int eo_apply_f32(dwf_ctx *h, FieldRef x, FieldRef out, cudaStream_t st);
int eo_dag_apply_f32(dwf_ctx *h, FieldRef w, FieldRef out, cudaStream_t st);   // out = D^dag w
// time slabs (slab.cu): neighbour table with ghost rows, links from the global field
cudaError_t launch_slab_tables(const dwf_ctx *h, cudaStream_t st);
cudaError_t launch_slab_pack_gauge(const dwf_ctx *h, const double *U, cudaStream_t st);
// FP64 complex vectors (n complex numbers): *out = Re <a, b> (part: 256 doubles of scratch); y = a x + b y
cudaError_t launch_cdot(const void *a, const void *b, size_t n, double *part, double *out, cudaStream_t st);
cudaError_t launch_caxpby(double a, const void *x, double b, void *y, size_t n, cudaStream_t st);
// 5D even-odd masks and combinations on canonical full 5D fields (eo5.cu; modes there)
cudaError_t launch_eo5(int mode, const void *A, const void *C, void *out, const int dims[4], int V, int Ls,
                       const double *inv_a0, cudaStream_t st);
// a bounded wait on a flag that nothing sets (eo5.cu): sets *err bit 0 after limit_ns
cudaError_t launch_wait_probe(const int *flag, unsigned long long limit_ns, int *err, cudaStream_t st);
}  // namespace dwf
void dwf_precond_release(dwf_ctx *h);

// error reporting helpers (capi.cu)
int dwf_set_error(int status, const std::string &msg);
int dwf_cuda_error(cudaError_t e, const char *where);
