/*
 * FP64 reference of the 4D Wilson operator, eq. (Wilson_matrix) of Sec. 2.1:
 *
 *   D_W(x,y;M) = (4+M) delta_{x,y}
 *              - 1/2 sum_mu [ (1-gamma_mu) U_mu(x) delta_{x+mu,y}
 *                           + (1+gamma_mu) U_mu(x-mu)^dag delta_{x-mu,y} ]
 *
 * used with M = -M0 (domain-wall height, Sec. 2.2).  Plain site loops, full
 * 4x4 gamma matrices (no spin-projection shortcut), complex double.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the oracle: it is compiled
 * and called by the test-suite, the smoke check and the benchmark's CPU
 * baseline leg, never by the library's product path.  It shares no code with
 * the CUDA implementation.
 *
 * Layouts (complex double, x fastest, dims = {Lx, Ly, Lz, Lt}):
 *   U   [mu][t][z][y][x][a][b]
 *   psi [t][z][y][x][spin][colour]       (nf such fields back to back)
 * bc[mu] = +1 / -1 multiplies every hop that crosses the lattice boundary in
 * direction mu (boundary condition of the fermion field).
 *
 * Gamma matrices: chiral basis
 *   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1,2,3),
 *   gamma_4 = [[0, 1], [1, 0]],
 * so that gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).
 */
#include <complex.h>
#include <stddef.h>
#include <string.h>

typedef double complex cplx;

static cplx G[4][4][4]; /* G[mu][row][col] */
static int g_init = 0;

static void init_gamma(void)
{
    if (g_init) return;
    memset(G, 0, sizeof(G));
    /* gamma_1 */
    G[0][0][3] = -I; G[0][1][2] = -I; G[0][2][1] = I;  G[0][3][0] = I;
    /* gamma_2 */
    G[1][0][3] = -1; G[1][1][2] = 1;  G[1][2][1] = 1;  G[1][3][0] = -1;
    /* gamma_3 */
    G[2][0][2] = -I; G[2][1][3] = I;  G[2][2][0] = I;  G[2][3][1] = -I;
    /* gamma_4 */
    G[3][0][2] = 1;  G[3][1][3] = 1;  G[3][2][0] = 1;  G[3][3][1] = 1;
    g_init = 1;
}

/* copy of gamma_mu into a row-major 4x4 complex array (used by the tests) */
void orc_gamma(int mu, cplx *out)
{
    init_gamma();
    memcpy(out, G[mu], sizeof(G[mu]));
}

static size_t site_index(const int c[4], const int d[4])
{
    return (size_t)c[0] + (size_t)d[0] * ((size_t)c[1] + (size_t)d[1] * ((size_t)c[2] + (size_t)d[2] * (size_t)c[3]));
}

/* y[spin][a] += coef * S[spin][spin'] * (W[a][b] * v[spin'][b]) ; W = U or U^dag */
static void add_hop(cplx *y, cplx coef, const cplx S[4][4], const cplx *Um, int dagU, const cplx *v)
{
    cplx Wv[4][3];
    for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a) {
            cplx acc = 0;
            for (int b = 0; b < 3; ++b) {
                cplx w = dagU ? conj(Um[b * 3 + a]) : Um[a * 3 + b];
                acc += w * v[sp * 3 + b];
            }
            Wv[sp][a] = acc;
        }
    for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a) {
            cplx acc = 0;
            for (int tp = 0; tp < 4; ++tp) acc += S[sp][tp] * Wv[tp][a];
            y[sp * 3 + a] += coef * acc;
        }
}

/*
 * dag = 0: out = D_W(-M0) in.
 * dag = 1: out = D_W(-M0)^dag in, written out as the conjugate transpose of the
 *          matrix above (entry (x,y) of D_W^dag is the adjoint of entry (y,x)):
 *   (D_W^dag psi)(x) = (4-M0) psi(x)
 *        - 1/2 sum_mu [ (1-gamma_mu)^dag U_mu(x-mu)^dag psi(x-mu)
 *                     + (1+gamma_mu)^dag U_mu(x)        psi(x+mu) ]
 */
void orc_wilson(const cplx *U, const int dims[4], const int bc[4], double M0,
                int dag, int nf, const cplx *in, cplx *out)
{
    init_gamma();
    const size_t V = (size_t)dims[0] * dims[1] * dims[2] * dims[3];
    cplx Sm[4][4][4], Sp[4][4][4]; /* (1 - gamma_mu), (1 + gamma_mu), daggered when dag */
    for (int mu = 0; mu < 4; ++mu)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                cplx g = dag ? conj(G[mu][j][i]) : G[mu][i][j];
                cplx one = (i == j) ? 1.0 : 0.0;
                Sm[mu][i][j] = one - g;
                Sp[mu][i][j] = one + g;
            }
    for (int f = 0; f < nf; ++f) {
        const cplx *src = in + (size_t)f * V * 12;
        cplx *dst = out + (size_t)f * V * 12;
#pragma omp parallel for schedule(static)
        for (long long xi = 0; xi < (long long)V; ++xi) {
            int c[4];
            size_t r = (size_t)xi;
            for (int mu = 0; mu < 4; ++mu) { c[mu] = (int)(r % (size_t)dims[mu]); r /= (size_t)dims[mu]; }
            cplx y[12];
            for (int k = 0; k < 12; ++k) y[k] = (4.0 - M0) * src[(size_t)xi * 12 + k];
            for (int mu = 0; mu < 4; ++mu) {
                int cf[4], cb[4];
                memcpy(cf, c, sizeof(c));
                memcpy(cb, c, sizeof(c));
                cplx phf = 1.0, phb = 1.0;
                cf[mu] = c[mu] + 1;
                if (cf[mu] == dims[mu]) { cf[mu] = 0; phf = bc[mu]; }
                cb[mu] = c[mu] - 1;
                if (cb[mu] < 0) { cb[mu] = dims[mu] - 1; phb = bc[mu]; }
                size_t xf = site_index(cf, dims), xb = site_index(cb, dims);
                const cplx *U_x = U + ((size_t)mu * V + (size_t)xi) * 9;  /* U_mu(x)    */
                const cplx *U_b = U + ((size_t)mu * V + xb) * 9;          /* U_mu(x-mu) */
                if (!dag) {
                    add_hop(y, -0.5 * phf, (const cplx(*)[4])Sm[mu], U_x, 0, src + xf * 12);
                    add_hop(y, -0.5 * phb, (const cplx(*)[4])Sp[mu], U_b, 1, src + xb * 12);
                } else {
                    add_hop(y, -0.5 * conj(phb), (const cplx(*)[4])Sm[mu], U_b, 1, src + xb * 12);
                    add_hop(y, -0.5 * conj(phf), (const cplx(*)[4])Sp[mu], U_x, 0, src + xf * 12);
                }
            }
            memcpy(dst + (size_t)xi * 12, y, sizeof(y));
        }
    }
}
