/*
 * dwf.h -- C ABI of the GB300 domain-wall fermion library.
 *
 * The library applies and inverts the 5D domain-wall fermion matrix of
 * Sec. 2.2 (eq. domainwall_general, constant b and c: Shamir, Borici, Mobius)
 * and Neff's modified matrix of Sec. 2.3 (eq. domainwall_neff), using the 4D
 * even-odd preconditioning of eq. (even-odd_linear_equation) and CG on the
 * normal equation (Sec. 2.3, last paragraphs).  The 4D Wilson kernel is
 * eq. (Wilson_matrix) with mass -M0.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice     dims = {Lx, Ly, Lz, Lt}, each even and >= 2; V = Lx*Ly*Lz*Lt.
 *             Lexicographic site index x + Lx*(y + Ly*(z + Lz*t)).
 * Gamma basis chiral: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
 *             gamma_4 = [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1),
 *             P_+ = (1+gamma_5)/2 (spins 0,1), P_- = (1-gamma_5)/2 (spins 2,3).
 * Boundaries  bc[mu] = +1 or -1 multiplies every fermion hop across the
 *             boundary in direction mu (x, y, z, t); NULL means {1, 1, 1, -1}.
 * Vectors     interleaved complex double (re, im), C order, x fastest:
 *               4D field      [t][z][y][x][spin 4][colour 3]
 *               5D field      [s][t][z][y][x][spin 4][colour 3]   (s = 1..Ls)
 *               EO 5D field   [s][i_e][spin 4][colour 3], i_e = index of the
 *                             even site among the even sites in lexicographic
 *                             order ((x+y+z+t) even is "even", Sec. 2.3)
 *               links         [mu][t][z][y][x][a][b]  (U_mu(x), 3x3 complex)
 * Memory      unless an entry point says "host", every data pointer is a
 *             device pointer that the caller owns, aligned to 16 bytes.  The
 *             library never frees caller memory.  A handle owns its internal
 *             copies (links in every precision, index tables, work vectors)
 *             and frees them in dwf_destroy.
 * Streams     stream is a cudaStream_t (NULL = legacy default stream).  All
 *             device work is ordered on it; calls that return results to the
 *             host (statistics, norms) synchronise it.  A handle must not be
 *             used from two threads at once.
 * Errors      every function returns a dwf_status; nothing aborts or exits.
 *             dwf_strerror gives a static description; dwf_last_error gives
 *             the last detailed message of the calling thread.
 */
#ifndef DWF_H
#define DWF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dwf_ctx *dwf_handle;

/* Sec. 2.2 (eq. domainwall_general) vs Sec. 2.3 (eq. domainwall_neff) */
enum dwf_form { DWF_STANDARD = 0, DWF_NEFF = 1 };

/* arithmetic of the device path: FP64; FP32; FP16 storage with one FP32
 * scale per 5D site (12 complex numbers) and FP32 arithmetic */
enum dwf_prec { DWF_F64 = 0, DWF_F32 = 1, DWF_F16 = 2 };

/* DWF_OP_FULL5D: the whole 5D matrix on full-lattice 5D fields.
 * DWF_OP_EO_PREC: D = 1 - D_ee^-1 D_eo D_oo^-1 D_oe on EO fields
 *                 (eq. even-odd_linear_equation).
 * DWF_OP_EO5_PREC: the same Schur complement for the 5D split of Sec. 2.3's
 *                 alternative (sites even when x + y + z + t + s is even), on
 *                 full-lattice 5D fields whose odd sites are ignored on input
 *                 and zero on output; needs the standard form with every
 *                 c_s = 0 and even Ls, where D_ee and D_oo are the on-site
 *                 diagonal b_s (4 - M0) + 1. */
enum dwf_op { DWF_OP_FULL5D = 0, DWF_OP_EO_PREC = 1, DWF_OP_EO5_PREC = 2 };

enum dwf_status {
    DWF_OK = 0,
    DWF_EINVAL = 1,      /* bad argument (size, pointer, alignment, enum)      */
    DWF_ENOMEM = 2,      /* device allocation failed                           */
    DWF_ECUDA = 3,       /* a CUDA call failed (message in dwf_last_error)      */
    DWF_ENOTCONV = 4,    /* max_iter reached; x holds the best iterate          */
    DWF_ENONFINITE = 5,  /* NaN or Inf met in the input or the iteration         */
    DWF_ETIMEOUT = 6,    /* a bounded device-side wait gave up                  */
    DWF_EBREAKDOWN = 7,  /* CG breakdown (p^dag A p <= 0)                        */
    DWF_ENOGAUGE = 8     /* dwf_set_gauge has not been called                    */
};

/*
 * Create a handle for one lattice and one operator.
 *   dims   {Lx, Ly, Lz, Lt}, each even, >= 2
 *   Ls     fifth-dimension extent, 2 <= Ls <= 32
 *   M0     domain-wall height (D_W = D_W(-M0), Sec. 2.2)
 *   mf     quark mass m of the corner blocks
 *   b, c   D_+ = b D_W + 1, D_- = c D_W - 1 (the same for every s)
 *   form   DWF_STANDARD or DWF_NEFF
 *   alpha  Neff parameter (ignored for DWF_STANDARD), alpha != 0
 *   bc     fermion boundary phases or NULL
 * The handle selects the current CUDA device at creation and uses it.
 * Fails with DWF_EINVAL when the 5D operator's site-local block
 * (D_ee, Sec. 2.3) is singular.
 */
int dwf_create(const int dims[4], int Ls, double M0, double mf, double b, double c,
               int form, double alpha, const int bc[4], dwf_handle *out);

/* The standard form of eq. (domainwall_general) with s-dependent coefficients
 * (Sec. 2.2: row i holds D_+^(i) = b_i D_W + 1 and D_-^(i) = c_i D_W - 1, as in
 * Chiu's optimal domain-wall fermion with b_i = c_i chosen per i): b and c are
 * host arrays of Ls values each, read during the call.  Every entry point then
 * works as for dwf_create; the source uses c_1 and c_Ls.  The FP64 mixing is
 * dense (the structured form assumes coefficients independent of i).  The
 * Neff form is defined for constant coefficients only.  Errors: as dwf_create
 * (DWF_EINVAL also for NULL b or c). */
int dwf_create_s(const int dims[4], int Ls, double M0, double mf, const double *b, const double *c,
                 const int bc[4], dwf_handle *out);
int dwf_destroy(dwf_handle h);
const char *dwf_strerror(int status);
const char *dwf_last_error(void);

/* Copy the links U_mu(x) of the 4D Wilson kernel, eq. (Wilson_matrix)
 * (device, layout above, SU(3) expected but not checked) into the handle: the
 * boundary phases are folded in and an internal copy in FP64, FP32 and FP16
 * is made for each output parity; the caller's buffer is not kept.  Must be
 * called before any operator call; calling it again replaces the links.
 * Errors: DWF_EINVAL (NULL handle or U, U not 16-byte aligned), DWF_ECUDA. */
int dwf_set_gauge(dwf_handle h, const void *U, void *stream);

/*
 * out = D in (dwf_apply) or out = D^dag in (dwf_apply_dag), D the handle's
 * form, in precision prec.  op = DWF_OP_FULL5D: in/out are 5D fields (the
 * whole matrix of Sec. 2.2 or 2.3).  op = DWF_OP_EO_PREC: in/out are EO 5D
 * fields and D is the even-odd preconditioned matrix.  in and out must not
 * overlap.  Input and output are always complex double; prec selects the
 * device arithmetic.  Errors: DWF_EINVAL (NULL handle or vector, unaligned
 * vector, bad prec or op), DWF_ENOGAUGE, DWF_ECUDA.
 */
int dwf_apply(dwf_handle h, int op, int prec, const void *in, void *out, void *stream);

/* D5 x5 = b5 through the 5D even-odd split (DWF_OP_EO5_PREC; Sec. 2.3's
 * alternative to the 4D split), FP64: b'_e = D_ee^-1 (b_e - D_eo D_oo^-1 b_o),
 * CG on the normal equation of the Schur complement from x_e = 0 until the
 * recursive residual falls below tol ||b'_e||, x_o = D_oo^-1 (b_o - D_oe x_e).
 * b5, x5: full 5D fields (device, complex double); history (host,
 * max_iter + 1 doubles, may be NULL) gets ||r||/||b'_e|| per iteration and,
 * last, the true residual ||b5 - D5 x5|| / ||b5||, which decides the status.
 * For comparing the two splits' iteration counts; the production solver is
 * dwf_solve.  Errors: DWF_EINVAL (as dwf_apply, split unavailable),
 * DWF_ENOGAUGE, DWF_ENOTCONV, DWF_ENONFINITE, DWF_EBREAKDOWN, DWF_ECUDA. */
int dwf_solve_eo5(dwf_handle h, const void *b5, void *x5, double tol, int max_iter, int *iters, double *history,
                  void *stream);

/*
 * 4D domain decomposition in time (the operator of eq. even-odd_linear_equation
 * split over ranks; Sec. 2.3 defines the operator, the split is the
 * library's).  dwf_create_slab makes a handle for the time slices
 * [t0, t0 + nt) of a lattice of extents global_dims (t0 and nt even, nt below
 * the global Lt; the other arguments as dwf_create).  Its dwf_set_gauge takes
 * the GLOBAL link field (layout above, global extents) and keeps the slab's
 * links with the global boundary phases.  Its fields are the slab's even-odd
 * fields (as DWF_OP_EO_PREC, Vh = Lx Ly Lz nt / 2 local sites, the local
 * even-odd order with t slowest, so a slab is a contiguous range of the global
 * even-odd index), and every internal field carries two ghost faces beyond its
 * Vh rows: the lower neighbour's last time slice and the upper neighbour's
 * first.  A slab handle is applied only through dwf_slab_apply_eo; the other
 * operator and solver entry points return DWF_EINVAL for it.
 *
 * dwf_slab_apply_eo runs the even-odd matrix (dag = 0) or its adjoint
 * (dag = 1) in three stages, in precision DWF_F64 or DWF_F32:
 *   stage 0: reads in (the slab's even field, complex double) and forms
 *            x^ = P x (Q^T x), whose faces are then exchanged;
 *   stage 1: t = M H_oe x^ (M^T H^dag_oe x^), reading x^'s ghost faces; t's
 *            faces are then exchanged;
 *   stage 2: out = x - 1/4 Q H_eo t (x - 1/4 P^T H^dag_eo t), reading t's
 *            ghost faces, written to out (complex double).
 * Between stages 0 and 1, and 1 and 2, each slab's last time slice goes to
 * the next slab's lower ghost face and its first slice to the previous slab's
 * upper ghost face.  dwf_slab_faces gives, after stage 0 or 1, the device
 * addresses of the slab's two boundary slices (send_lo: first slice, send_hi:
 * last) and of its two ghost faces (recv_lo, recv_hi), each `bytes` long and
 * contiguous (copy them with cudaMemcpyAsync or NCCL send/recv between
 * ranks); dwf_slab_exchange_ring does all copies of a ring of n >= 2 slabs on
 * one device, hs[i + 1] holding the slices after hs[i] and hs[0] after
 * hs[n - 1], on `stream`, ordered after the stage that made the faces.
 * Errors: DWF_EINVAL (not a slab, bad stage or precision, NULL or unaligned
 * vector, slabs of different lattices or not consecutive), DWF_ENOGAUGE,
 * DWF_ECUDA.
 */
int dwf_create_slab(const int global_dims[4], int t0, int nt, int Ls, double M0, double mf, double b, double c,
                    int form, double alpha, const int bc[4], dwf_handle *out);
int dwf_slab_apply_eo(dwf_handle h, int prec, int stage, int dag, const void *in, void *out, void *stream);
int dwf_slab_faces(dwf_handle h, int prec, int stage, void **send_lo, void **send_hi, void **recv_lo,
                   void **recv_hi, size_t *bytes);
int dwf_slab_exchange_ring(dwf_handle *hs, int n, int prec, int stage, void *stream);

/* CG on the normal equation of the even-odd matrix (Sec. 2.3, FP64) over a
 * ring of n >= 2 slabs on one device, each slab's vectors its own: b[i] the
 * slab's even right-hand side, x[i] its solution (device, complex double, the
 * slab's even-odd layout; x is overwritten from a zero start).  Every
 * application of D and D^dag runs the three stages of all slabs with the face
 * exchanges between them; the inner products are per-slab sums in a fixed
 * order added over the slabs (the all-reduce of a multi-GPU run).  Stops when
 * the recursive residual falls below tol ||b||, then recomputes b - D x:
 * history (host, max_iter + 1 doubles, may be NULL) gets ||r||/||b|| per
 * iteration and the true residual last; *iters the iteration count.
 * Errors: DWF_EINVAL, DWF_ENOGAUGE, DWF_ENOTCONV (true residual above tol),
 * DWF_ENONFINITE, DWF_EBREAKDOWN, DWF_ECUDA. */
int dwf_slab_cgnr_ring(dwf_handle *hs, int n, const void *const *b, void *const *x, double tol, int max_iter,
                       int *iters, double *history, void *stream);
int dwf_apply_dag(dwf_handle h, int op, int prec, const void *in, void *out, void *stream);

/* b5 = (-D_-) P^dag (0, ..., 0, b4)^T  (Sec. 2.3, with D_- = diag_s(c D_W - 1)):
 * b5(s=1) = (1 - c D_W) P_+ b4, b5(s=Ls) = (1 - c D_W) P_- b4, zero elsewhere.
 * b4 is a 4D field, b5 a 5D field (device, caller-owned).  FP64.
 * Errors: DWF_EINVAL (NULL or unaligned vector), DWF_ENOGAUGE, DWF_ECUDA. */
int dwf_source_5d(dwf_handle h, const void *b4, void *b5, void *stream);

/* x4 = [P^dag x5]_{s=1} = P_- x5(s=1) + P_+ x5(s=Ls)  (Sec. 2.3 and the 4D
 * quark field of Sec. 2.2).  The same formula holds for both forms.  x5 a 5D
 * field, x4 a 4D field (device, caller-owned), FP64.
 * Errors: DWF_EINVAL (NULL handle or vector, unaligned vector), DWF_ECUDA. */
int dwf_project_4d(dwf_handle h, const void *x5, void *x4, void *stream);

/* ---------------------------------------------------------------- solver */
typedef struct {
    double tol;         /* target ||b5 - D x5|| / ||b5|| of the full 5D system
                           (checked in FP64 at the end); default 1e-10          */
    int max_iter;       /* cap on inner CG iterations; default 20000            */
    int inner_prec;     /* DWF_F64 (plain FP64 CG), DWF_F32 or DWF_F16; the
                           outer residuals and corrections are always FP64     */
    double delta;       /* reliable-update trigger: recompute the FP64 residual
                           when the inner residual fell by this factor; 0 (the
                           default) takes 1e-3 for FP32 and 0.1 for FP16 and
                           FP64 inner iterations                               */
    int check_every;    /* inner iterations between host convergence checks;
                           they are captured as one CUDA graph; default 16     */
    int use_graph;      /* 1: replay the inner iterations as a CUDA graph       */
    int precond;        /* 0: CG with reliable updates; 1: flexible CG on the
                           normal equation preconditioned by M = N N^dag, N the
                           handle's learned network (FP32 cycles, FP64 defect
                           correction; dwf_precond_*); needs inner_prec =
                           DWF_F32                                             */
    int use_initial_guess; /* 1: x5 holds the initial guess on entry; 0: zero   */
    int verbose;        /* 0 quiet                                              */
    int batch_wave;     /* dwf_solve_batch: at most this many systems per wave;
                           0 (default): as many as device memory allows        */
    int eo_form;        /* the even-odd equation the inner CG iterates on:
                           0 (default) eq. (even-odd_linear_equation),
                           D x_e = b~_e with D = 1 - D_ee^-1 D_eo D_oo^-1 D_oe;
                           1 eq. (another_even-odd_linear_equation),
                           D' y_e = b'_e with D' = 1 - D_eo D_oo^-1 D_oe D_ee^-1,
                           b'_e = D_ee b~_e, x_e = D_ee^-1 y_e (Sec. 2.3: Neff's
                           factor cancels in D', so alpha does not change its
                           convergence); dwf_solve only, not with precond   */
} dwf_solve_params;

typedef struct {
    int status;               /* dwf_status of the solve                        */
    int iterations;           /* inner CG iterations                            */
    int reliable_updates;     /* FP64 residual recomputations                   */
    int d_applications;       /* applications of D or D^dag (all precisions)    */
    double true_residual;     /* ||b5 - D x5|| / ||b5||, FP64, full 5D system   */
    double eo_residual;       /* ||b~ - D_pc x_e|| / ||b~||, FP64               */
    double seconds;           /* wall time of the call (host clock)             */
    double history[64];       /* eo residual at each reliable update            */
    int n_history;
    long long kernel_launches; /* device kernels launched by the call           */
    int waves;                /* memory waves of the call (1 for dwf_solve)     */
    int precond_applications; /* applications of the learned preconditioner     */
    int fallbacks;            /* switches from the learned preconditioner to N = 1 */
} dwf_solve_stats;

void dwf_solve_params_default(dwf_solve_params *p);

/*
 * Solve D x5 = b5 for the handle's form (5D fields, device).  Route:
 * b~_e = D_ee^-1 (b_e - D_eo D_oo^-1 b_o); CG on D^dag D x_e = D^dag b~_e with
 * D the even-odd matrix (inner precision as asked, FP64 reliable updates);
 * x_o = D_oo^-1 (b_o - D_oe x_e); final FP64 residual of the full system
 * (Sec. 2.3).  x5 is the initial guess when p->use_initial_guess is set,
 * otherwise the initial guess is zero.  stats may be NULL.  b5 and x5 are
 * caller-owned device 5D fields (16-byte aligned, not overlapping).
 * Errors: DWF_EINVAL (NULL or unaligned vector, bad parameters, precond
 * without a network or with inner_prec != DWF_F32), DWF_ENOGAUGE,
 * DWF_ENONFINITE (NaN/Inf in b5 or in the iteration), DWF_EBREAKDOWN,
 * DWF_ECUDA, DWF_ENOTCONV (x5 holds the best iterate and stats are filled).
 */
int dwf_solve(dwf_handle h, const void *b5, void *x5, const dwf_solve_params *p,
              dwf_solve_stats *stats, void *stream);

/*
 * The user-level propagator call with HOST buffers: x4 = [P^dag D^-1 b5(b4)]_{s=1}
 * (Sec. 2.3: the 4D quark propagator from a 4D source).
 * b4_host and x4_host are host pointers to 4D fields (complex double); the
 * call copies b4 to the device, builds b5, solves, projects and copies x4
 * back, all on the given stream, and synchronises before returning.
 * Errors: as dwf_solve (DWF_EINVAL also for NULL host pointers); on
 * DWF_ENOTCONV x4_host holds the projection of the best iterate.
 */
int dwf_propagator_host(dwf_handle h, const double *b4_host, double *x4_host,
                        const dwf_solve_params *p, dwf_solve_stats *stats, void *stream);

/*
 * Solve n systems at once (no counterpart in the paper, which solves one
 * system at a time; the systems are independent).  hs[i] are handles of the
 * same lattice dimensions (they may differ in Ls, mf, b, c, form, alpha; a
 * handle may serve several systems); b4[i] are 4D sources and x4[i] the 4D
 * solutions x4 = P_- x5(1) + P_+ x5(Ls) (device, complex double, 16-byte
 * aligned; caller-owned).  Every handle must have its gauge field set.
 * The systems run in lock step in waves that fit in device memory (systems
 * ordered round robin over the handles, so that a wave mixes Ls and mf;
 * p->batch_wave caps the wave size).  Within a wave every kernel of the
 * inner iteration is one launch per distinct Ls over the (site tile, system)
 * work items of all its systems, the links of a tile being read once from
 * DRAM for all of them; the iterations are replayed as CUDA graphs, and
 * converged systems are skipped by their flag.  Reliable updates, the source
 * and the final FP64 check run per system between replays, as in dwf_solve.
 * The initial guess is always zero.  stats may be NULL or an array of n
 * (stats[i].waves: number of waves; seconds, kernel_launches: of the whole
 * call).  Returns the worst status of the systems; DWF_ENOMEM when one system
 * alone does not fit.
 */
int dwf_solve_batch(dwf_handle const *hs, const void *const *b4, void *const *x4, int n,
                    const dwf_solve_params *p, dwf_solve_stats *stats, void *stream);

/* ----------------------------------------------------- introspection, tests */

/* Host copy of one per-chirality fifth-direction matrix of the handle, FP64,
 * row-major Ls x Ls.  which: 0 A5 = D_ee restricted to one chirality,
 * 1 A5^-1, 2 B = b + c K, 3 R (Neff factor, identity for DWF_STANDARD).
 * chirality: 0 for P_+ components, 1 for P_-.  (Sec. 2.2-2.3; out_host holds
 * Ls*Ls doubles.)  Errors: DWF_EINVAL (NULL handle or out, bad which or
 * chirality). */
int dwf_fifth_matrix(dwf_handle h, int which, int chirality, double *out_host);

/* The same without a handle or a device (host code only): the matrices for
 * the parameters of dwf_create, with b and c host arrays of Ls values (row i of
 * the 5D matrix takes b[i], c[i], as dwf_create_s; constant for DWF_NEFF),
 * FP64 row-major Ls x Ls.  which 0..3 as above,
 * or 16 + k for the k-th per-chirality matrix the kernels apply in the fifth
 * direction (Sec. 2.3 even-odd algebra; B = b + cK, R the Neff factor):
 *   k = 0 P = B R, 1 P^T, 2 Q = R^-1 A5^-1 (D_ee^-1), 3 Q^T, 4 M = B A5^-1,
 *   5 M^T, 6 A5 R (D_ee), 7 (A5 R)^T, 8 -1/2, 9 -1/2 R B^T, 10 -1/4 Q,
 *   11 -1/4 P^T, 12 1, 13 +1/2 Q, 14 c/2 (hop part of 1 - c D_W),
 *   15 1 - c (4 - M0) (its diagonal part), 16 -1/4, 17 -1/4 M^T.
 * *banded (if non-null): 1 when every nonzero of the matrix lies on the cyclic
 * tridiagonal, which the kernels then read as three coefficients per row
 * (always 0 for which 0..3).  Errors: DWF_EINVAL (Ls outside 2..32, form,
 * which, chirality, null pointer, s-dependent coefficients with DWF_NEFF, or
 * A5 singular). */
int dwf_fifth_matrix_host(int Ls, double M0, double mf, const double *b, const double *c, int form, double alpha,
                          int which, int chirality, double *out_host, int *banded);

/* Number of device bytes the handle holds (0 for a NULL handle). */
size_t dwf_device_bytes(dwf_handle h);

/* Number of device kernels launched through the handle since its creation
 * (every entry point counts the kernels it launches, graph replays included;
 * 0 for a NULL handle). */
long long dwf_launch_count(dwf_handle h);

/* Configuration of the hop kernel in precision prec: variant 0 loads the
 * neighbour spinors directly from global memory, one CTA per tile of sb sites;
 * variant 3 is a persistent kernel sweeping consecutive tiles; variant 4 takes
 * each CTA's sites as a 4D block of the half lattice (neighbour reuse in L1);
 * variant 5 (DWF_F16 only, dense mixing; else variant 0) is variant 0 with the
 * spin projection in FP16 arithmetic on the stored FP16 values (one rounding
 * at the FP16 storage level) and the SU(3) product in FP32 shared by the
 * thread's slices; variant 7 (FP32/FP16, dense mixing, Ls a multiple of 4) is
 * a persistent kernel of sb-site tiles with the tile's links staged in shared
 * memory one tile ahead and the mixing done by half of the threads, two
 * outputs each; variant 9 (FP32/FP16, dense mixing, Ls dividing 32 and a
 * multiple of 4) is persistent and warp-autonomous: every warp walks its own
 * tiles of 32/Ls sites (a window sweeping the lattice, see dwf_set_sweep) with
 * its own shared-memory links (staged one tile ahead) and mixing tile, and no
 * CTA barrier; there sb counts warps per CTA (1..4) and ns selects the
 * register budget (1: five CTAs of sb warps per SM, 2: four); variant 10
 * (FP32, dense mixing, Ls 8 or 16, no mixed y term; else variant 9) is
 * variant 9 in CTAs of eight warps whose dense fifth-direction mixings run on
 * the tensor cores: the CTA's hop results are the A operand of tcgen05 TF32
 * products (rows = site and spinor component, K = slice; both operands split
 * in two TF32 terms, FP32 accumulators in tensor memory), the epilogue reads
 * them back row by row (ns and sb must be 0).  ns: slices per thread for the
 * other variants (1, 2 when it divides Ls, 4 for variant 5); sb: sites per
 * CTA.  -1 / 0 select the built-in defaults (FP32: variant 9 where it
 * applies, else 0; FP16: 5; FP64: 0).  Variants differ only in the order of
 * the sums, except 5 (FP16 rounding of the projection) and 10 (products of
 * the TF32 terms).  Numbers 1, 2, 6 and 8 are not used.
 * Errors: DWF_EINVAL (NULL handle or pointer, bad prec, variant not -1, 0, 3,
 * 4, 5, 7, 9 or 10, ns or sb outside the ranges above, sb making a CTA of more
 * than 256 threads). */
int dwf_set_hop_config(dwf_handle h, int prec, int variant, int ns, int sb);
int dwf_get_hop_config(dwf_handle h, int prec, int *variant, int *ns, int *sb);

/* Sweep order of the hop kernels in precision prec (variants 0, 5, 9 and 10):
 * the sites of one parity are taken in columns of zblock z-planes, each column
 * t-slice by t-slice, so that the two reads of a site as the -t and +t
 * neighbour of others lie 2 zblock (Lx/2) Ly sites apart and the field between
 * them stays in L2 on lattices whose t-slices exceed it; the z-planes at a
 * column's border are read twice.  zblock: -1 or 0 index order (the default),
 * -2 the largest divisor of Lz whose column band of input, output and links of
 * one parity stays within 16 MiB (index order when a whole t-slice does), else
 * a divisor of Lz below Lz with zblock (Lx/2) Ly a multiple of 32.  On
 * 32^3x64, Ls 16, columns of 8 planes cut the FP32 hop's DRAM reads by a fifth
 * but not its time (it is bound by the SMs' load/store path).  The order
 * changes only the order of the fused norms' partial sums.
 * Errors: DWF_EINVAL (NULL handle or pointer, bad prec or zblock). */
int dwf_set_sweep(dwf_handle h, int prec, int zblock);
int dwf_get_sweep(dwf_handle h, int prec, int *zblock);

/* Autotuner: times every hop configuration (all variants, ns in {1, 2, 4},
 * CTAs of 64 to 256 threads, every available mixing mode) on this handle's lattice with CUDA events on
 * `stream` and keeps the fastest.  cache_path (host string, may be NULL)
 * names a text file of earlier results keyed by device name, lattice, Ls and
 * precision: a hit skips the timing, a miss appends the new result.  Needs
 * the gauge field.  Errors: DWF_EINVAL, DWF_ENOGAUGE, DWF_ECUDA. */
int dwf_autotune(dwf_handle h, int prec, const char *cache_path, void *stream);

/* Fifth-direction mixing in precision prec: 0 applies the dense per-chirality
 * Ls x Ls matrices, 1 their structured form (diagonal, bidiagonal-plus-corner
 * and closed-form inverse factors, about 6 flops per element instead of
 * 2 Ls), 2 the dense matrices on the tensor cores (FP32 and FP16 only): the
 * stand-alone mixing launches run as a batched GEMM of tcgen05 MMAs, the
 * field of 16 sites as the A operand (rows = site, colour, re/im, spin;
 * K = slice), both chiralities' matrices side by side as B, operands split in
 * two TF32 terms each (FP32 accuracy), the accumulator in tensor memory;
 * inside the hop the mixing of a CTA's tile runs as warp-level TF32 MMAs (the
 * matrix split in two TF32 terms; FP32 fields also split the field, FP16
 * fields do not).  Mode 1 runs in hop variant 9 at Ls 8 and 16 (each lane
 * takes whole chains of one spinor component over the Ls slices from the
 * warp's tile into registers; in FP32/FP16 the CG update and the stand-alone
 * mixing keep the dense form's three-row path for banded matrices), else in
 * the direct variant, which it then selects; mode 2 selects the direct
 * variant (CTAs of at least 32 threads, else the dense form runs) or hop
 * variant 10; the CG update keeps the dense form in mode 2.  -1 restores the
 * default: the structured form for DWF_F64 when it is available, dense for
 * DWF_F32 and DWF_F16.  mode 1 is refused when
 * the handle's parameters make the structured form unavailable
 * (|kappa| = |beta0/alpha0| >= 0.95), mode 2 for prec = DWF_F64; both with
 * DWF_EINVAL, as a NULL handle or pointer and a bad prec or mode. */
int dwf_set_mix_mode(dwf_handle h, int prec, int mode);
int dwf_get_mix_mode(dwf_handle h, int prec, int *mode);

/*
 * Allocation-free variant of dwf_apply / dwf_apply_dag with DWF_OP_EO_PREC
 * (the paper has no counterpart: this is a service of the library).  It
 * computes the same out = D in (dag = 0) or out = D^dag in (dag != 0) on EO
 * fields, for callers that cannot let a library allocate device memory
 * during a call (an application that has handed all device memory to its own
 * pool, or a path where an allocation would synchronise the device): its
 * four work fields live in one fixed, file-scope device array of 64 MiB that
 * exists on every GPU that loads the library until the process exits.  The
 * call performs no cudaMalloc or cudaFree; the handle itself, created and
 * given its links beforehand, is reused.  Lattices whose work fields exceed
 * the array are rejected with DWF_EINVAL (4 internal half fields in
 * precision prec; FP64 on 8^4 x Ls=16 uses 25 MB).  The array's device
 * address is looked up once per device, on the first call made with that
 * device current.  Every call shares the array and it keeps the last call's
 * contents; calls whose GPU work overlaps (other streams, other handles of
 * the same device) race, so a caller that uses the array from several streams
 * must order each call after the others' work (events or a synchronisation).
 * Every call reads the handle's current state: its links (dwf_set_gauge), its
 * mixing mode and its hop configuration.  The first call on a device may also
 * make the CUDA driver load the library's device code that holds the array.
 * in/out: device EO fields as for dwf_apply.
 */
int dwf_apply_eo_noalloc(dwf_handle h, int prec, int dag, const void *in, void *out, void *stream);

/* Synchronise `stream` and report device-side failures of earlier calls on
 * the handle: DWF_ETIMEOUT if a bounded wait inside a kernel gave up (the
 * flag is cleared by this call), else DWF_OK. */
int dwf_device_status(dwf_handle h, void *stream);

/* Failure-detection probe: one device thread waits on a flag that nothing
 * sets, bounded by %globaltimer to limit_ns nanoseconds (clamped to 1 s; 0
 * checks once), then records the timeout in the handle's error flag as every
 * bounded wait of the library does, and returns; the next dwf_device_status
 * reports DWF_ETIMEOUT and the context stays usable.  Errors: DWF_EINVAL
 * (NULL handle, negative limit), DWF_ECUDA. */
int dwf_wait_probe(dwf_handle h, long long limit_ns, void *stream);

/* Timing of one hop kernel launch in the given precision: runs the EO hop
 * (the dominant kernel of every application of D) `reps` times on stream and
 * writes the mean device time per launch in microseconds, measured with CUDA
 * events on that stream, together with the kernel's algorithmic bytes per
 * launch (inputs read once, outputs written once, links read once).  With
 * flush_l2 != 0 a 512 MB buffer is written before every timed launch.
 * Errors: DWF_EINVAL (reps < 1, NULL outputs, bad prec), DWF_ENOGAUGE,
 * DWF_ECUDA. */
int dwf_time_hop(dwf_handle h, int prec, int reps, int flush_l2, double *us_per_launch,
                 double *bytes_per_launch, void *stream);

/* Timing of one stand-alone fifth-direction mixing launch (out = M in with
 * the even-odd factor M = B A5^-1 of Sec. 2.3, per chirality) on an even
 * field in precision prec with mixing mode `mode` (dwf_set_mix_mode: 0 dense
 * on the CUDA cores, 1 structured, 2 tensor cores: tcgen05 MMAs with the
 * accumulator in tensor memory, FP32/FP16 only); as dwf_time_hop otherwise
 * (*bytes: the field read once and written once).  The handle's own mixing
 * mode is restored.  Errors: DWF_EINVAL (bad argument, mode unavailable),
 * DWF_ECUDA. */
int dwf_time_mix(dwf_handle h, int prec, int mode, int reps, int flush_l2, double *us, double *bytes,
                 void *stream);

/* Profiling aid: times the five launches of one inner CG iteration of
 * dwf_solve in precision prec (DWF_F16, DWF_F32, DWF_F64) on the handle's
 * solver workspace, reset before every iteration to a synthetic state (inner
 * fields of bytes 0x3c, FP16 scales of bytes 0x3f, x accumulator 0, |r|^2 = 1,
 * alpha = 0.5).
 * k = 0: x += alpha p of the previous iteration, p = r + beta p and P p;
 * k = 1, 2: the even-odd matrix D_pc (Sec. 2.3) in its two hops (M H_oe, then
 * the Q H_eo hop with the identity term, its norm and the Q^T mixing of the
 * dagger); k = 3, 4: the dagger hops, the last one fused with
 * r -= alpha D^dag D p and |r|^2.  The launches of an
 * iteration run back to back (as in the solver); with flush_l2 != 0 a 512 MB
 * buffer is written between iterations.  Writes us5[k], the mean device time
 * in microseconds of launch k (CUDA events on `stream`, reps iterations after
 * two untimed ones), and bytes5[k], its algorithmic bytes (each field read
 * once and written once, links once; an FP16 field includes its scales).
 * Overwrites the solver's workspace (not a solve in progress: the handle is
 * used by one thread at a time). Errors: DWF_EINVAL, DWF_ENOGAUGE, DWF_ECUDA. */
int dwf_time_iteration(dwf_handle h, int prec, int reps, int flush_l2, double *us5, double *bytes5,
                       void *stream);

/* Measured arithmetic peaks of the current device (no counterpart in the
 * paper: the denominators of the hop kernels' arithmetic rooflines).
 * out (host, 4 doubles): [0] FP32 TFLOP/s with scalar FMAs, [1] FP32 TFLOP/s
 * with packed FP32x2 FMAs, [2] FP64 TFLOP/s with FMAs, [3] the device's SM
 * count.  Each rate is the best of three timed launches (CUDA events on
 * `stream`) of a kernel of 8 independent FMA chains per thread, 8 CTAs of 256
 * threads per SM, 2 flops per FMA lane.  Allocates and frees a small scratch
 * buffer; synchronises `stream`.  Errors: DWF_EINVAL (NULL out), DWF_ECUDA. */
int dwf_alu_peaks(double *out, void *stream);

/* Extremal eigenvalues of D^dag D, D the even-odd matrix D_pc of the handle's
 * form (Sec. 2.3; for Neff's form the alpha-dependent one): Sec. 3.2 takes
 * lambda_max / lambda_min as the condition number that governs CG and studies
 * it against alpha.  eo_form = 0: D = D_pc of eq. (even-odd_linear_equation),
 * the matrix dwf_solve iterates on; eo_form = 1: D = 1 - D_eo D_oo^-1 D_oe D_ee^-1
 * of eq. (another_even-odd_linear_equation), in which alpha cancels (Sec. 2.3).
 * FP64 Lanczos recurrence on the device from a
 * pseudo-random start vector (SplitMix64 at counter `seed`), no restarts;
 * every 10 steps the extremal eigenvalues of the tridiagonal matrix are taken
 * (Sturm bisection on the host) and the recurrence stops when both changed by
 * at most rtol (relative) since the previous check, after at least 20 steps,
 * at max_steps, or when the Krylov space is exhausted.  Writes lambda_min,
 * lambda_max and (if steps is non-null) the steps taken.  Uses FP64 workspace
 * of up to nine even fields.  Errors: DWF_EINVAL (eo_form not 0 or 1,
 * max_steps < 2, rtol <= 0, null outputs), DWF_ENOGAUGE, DWF_ENONFINITE,
 * DWF_ECUDA. */
int dwf_spectrum_bounds(dwf_handle h, int eo_form, int max_steps, double rtol, unsigned long long seed,
                        double *lambda_min, double *lambda_max, int *steps, void *stream);

/* ------------------------------------------------ learned preconditioner
 * No counterpart in the paper (it solves with plain CG).  A gauge-covariant
 * linear stencil network N approximates D^-1 for the even-odd matrix D, so
 * that M = N N^dag approximates (D^dag D)^-1: dwf_solve with params.precond = 1
 * runs FP32 cycles of flexible CG (Notay 2000) on D^dag D e = D^dag r
 * preconditioned by M, each closed by an FP64 defect correction (r the FP64
 * residual of the even-odd system); if M loses positivity the solve continues
 * with M = 1 (plain CG).  dwf_precond_apply with which = 2 gives M.
 * Channels are the Ls fifth-direction slices (Ls <= 16).  Layer l maps a
 * field psi of Ls channels to
 *   out(x, c) = sum_p sum_c' W[l][p][chi][c][c'] T_p(x, c'),
 *   T_0 = psi(x), T_{1+2mu} = (1 - gamma_mu) U_mu(x) psi(x+mu),
 *   T_{2+2mu} = (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)   (mu = 0..3: x, y, z, t),
 * chi = 0 for output spins 0, 1 (P_+), 1 for spins 2, 3 (P_-), with the
 * handle's boundary phases on hops across the boundary.  N(r) places an EO
 * field r on the even sites (zero on odd sites), applies the layers and keeps
 * the even sites; N^dag applies the adjoint layers in reverse order.  Weights: complex, host layout [layer][9][2][Ls][Ls]
 * interleaved (re, im); FP64 master copy (Adam), BF16-rounded copy used by
 * the FP32 kernels.
 *
 * Training: loss L = (1/K) sum_k |N(b_k) - x_k|^2 / |x_k|^2 over pairs
 * D x_k = b_k: x_k = even part of the solution of D5 x5 = b5(b4_k) (dwf_solve)
 * and, as many by default, white-noise x_k (Gaussian, counter-based), with
 * b_k = D x_k; Adam (beta 0.9, 0.999, eps 1e-8) over minibatches.  The
 * output layer starts scaled by the least-squares factor
 * s = sum Re<b,x>/|x|^2 / sum |b|^2/|x|^2.
 */
typedef struct {
    int layers;              /* network depth; default 3                          */
    int epochs;              /* passes over the pairs; default 20                 */
    int batch;               /* pairs per Adam step; default 16                   */
    double lr;               /* Adam step size; default 2e-3                      */
    int solve_inner_prec;    /* precision of the solves that make the pairs       */
    double solve_tol;        /* their tolerance; default 1e-8                     */
    unsigned long long seed; /* initial weights and pair order                    */
    double noise;            /* scale of the random part of the initial weights   */
    int verbose;
    int random_pairs;        /* white-noise pairs (x Gaussian, b = D x) added to
                                the solution pairs; -1 (default): as many        */
} dwf_train_params;

typedef struct {
    int status;
    int pairs, epochs, steps;
    double loss_first, loss_last;  /* mean loss over the first and last epoch     */
    double loss_history[64];       /* per epoch                                   */
    int n_history;
    double seconds;                /* whole call (host clock)                     */
    double solve_seconds;          /* of which: making the pairs                  */
} dwf_train_stats;

void dwf_train_params_default(dwf_train_params *p);

/* Identity network (self weights 1 on every channel and chirality) plus
 * seeded normal noise of the given scale.  Errors: DWF_EINVAL (NULL handle,
 * layers outside 1..8, Ls > 16), DWF_ENOGAUGE, DWF_ECUDA. */
int dwf_precond_init(dwf_handle h, int layers, unsigned long long seed, double noise);
/* Host weights in, FP64 (layout above); the Adam state is reset.
 * Errors: DWF_EINVAL (NULL pointer, layers outside 1..8, Ls > 16),
 * DWF_ENOGAUGE, DWF_ECUDA. */
int dwf_precond_set_weights(dwf_handle h, int layers, const double *w);
/* Host weights out: the FP64 master copy, or (compute_copy != 0) the
 * BF16-rounded values the kernels use.  Errors: DWF_EINVAL (NULL pointer, no
 * network, layers different from the network's), DWF_ECUDA. */
int dwf_precond_get_weights(dwf_handle h, int layers, int compute_copy, double *w);
/* out = N in (which = 0), N^dag in (1) or M in = N N^dag in (2) on EO fields
 * (device, complex double, layout of DWF_OP_EO_PREC); FP32 kernels.
 * Errors: DWF_EINVAL (no network, bad which, NULL or unaligned vector),
 * DWF_ENOGAUGE, DWF_ECUDA. */
int dwf_precond_apply(dwf_handle h, int which, const void *in, void *out, void *stream);
/* Loss over npairs pairs (EO fields b[k], x[k], device) and its gradient with
 * respect to the weights (host, layout above, may be NULL); FP32 kernels
 * with the BF16-rounded weights, FP64 accumulation across thread blocks.
 * Errors: DWF_EINVAL (no network, npairs < 1, NULL pointers), DWF_ENOGAUGE,
 * DWF_ECUDA. */
int dwf_precond_loss_grad(dwf_handle h, int npairs, const void *const *b, const void *const *x,
                          double *loss, double *grad, void *stream);
/* One Adam step of the training (beta 0.9, 0.999, eps 1e-8, step size lr,
 * the step count continuing from the network's), from the gradient grad
 * (host, FP64, weight layout above) instead of one computed from pairs: the
 * same update dwf_precond_train applies after each minibatch.  Errors:
 * DWF_EINVAL (NULL pointer, no network of that depth, lr <= 0), DWF_ECUDA. */
int dwf_precond_adam_step(dwf_handle h, int layers, const double *grad, double lr, void *stream);

/* Save the handle's network to a host file, and load one into a handle of the
 * same Ls: a binary header (magic "DWFNET", format version 1, layers,
 * channels = Ls, Adam step count, number of complex weights n), then the FP64
 * master weights, Adam's first moments and Adam's second moments, n complex
 * doubles each (little-endian).  Loading replaces the handle's network
 * (training continues from the saved Adam state) and recomputes the
 * BF16-rounded compute copy.  Errors: DWF_EINVAL (NULL pointer, no network to
 * save, unreadable or unwritable file, wrong magic or version, a file for
 * another Ls, a truncated file), DWF_ENOGAUGE (load before dwf_set_gauge),
 * DWF_ECUDA. */
int dwf_precond_save(dwf_handle h, const char *path);
int dwf_precond_load(dwf_handle h, const char *path);

/* One FP32 flexible-CG solve of D^dag D x = b (D the even-odd matrix; b, x
 * EO fields, device, complex double) preconditioned by M = N N^dag (plain != 0:
 * M = 1), from x = 0, as the cycles of dwf_solve with precond = 1 run it:
 * q = D^dag D p, alpha = (r, z)/(p, q), x += alpha p, r' = r - alpha q,
 * z' = M r', beta = (z', r' - r)/(r, z), p = z' + beta p, until
 * |r| <= tol |b| or max_iter steps.  history (host, max_iter + 1 doubles, may
 * be NULL) receives |r_k| / |b| from k = 0; *iters (may be NULL) the steps.
 * Errors: DWF_EINVAL (NULL or unaligned vector, tol <= 0, max_iter < 0, no
 * network without plain), DWF_ENOGAUGE, DWF_EBREAKDOWN (M not positive on a
 * residual), DWF_ENONFINITE, DWF_ECUDA. */
int dwf_precond_fcg(dwf_handle h, const void *b, void *x, double tol, int max_iter, int plain, double *history,
                    int *iters, void *stream);

/* Make the pairs from nsrc 4D sources b4[k] (device) and train (above).
 * Errors: DWF_EINVAL (nsrc < 1, NULL pointers, bad parameters, Ls > 16),
 * DWF_ENOGAUGE, DWF_ECUDA, and the solver's errors while making the pairs. */
int dwf_precond_train(dwf_handle h, int nsrc, const void *const *b4, const dwf_train_params *p,
                      dwf_train_stats *stats, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DWF_H */
