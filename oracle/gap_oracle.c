/*
 * FP64 CPU oracle of the GAP hot path: SOAP descriptor, sparse-GP
 * dot-product kernel, its Cartesian derivative, the K_NM rows and the
 * regularised least-squares solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  The CUDA
 * library shares no code, header, table or constant generator with it.
 *
 * Everything is computed directly from the paper's definitions, in double
 * precision, with no blocking, tabulation or fusion:
 *   cutoff function            Eq. 18 (Sec. 3.3.1)
 *   neighbour density          Eq. 19 (Sec. 3.3.2)
 *   basis expansion            Eq. 20
 *   power spectrum             Eqs. 22-23, normalisation Eq. 24
 *   element embedding          Eq. 25 and the Z_mix/coupling keywords (Sec. 3.3.3, Appendix)
 *   dot-product kernel         Eq. 13, prefactor delta^2 (energy_scale, Appendix)
 *   local energy, total energy Eqs. 2 and 1
 *   derivative                 Eq. 3
 *   K_NM rows                  text after Eq. 4 (force entries -grad_x k . dx/dr)
 *   least squares              Eq. 4 (normal form) and Eqs. 5-9 (QR form)
 *   two-body term              Eqs. 10-11 with the cutoff factor of Sec. 3.3.1
 *
 * Readings where the paper is silent (all listed with reasons in the design
 * notes of the repository):
 *   - radial basis: Gram-Schmidt orthonormalisation, in order of increasing
 *     power, of (rc - r)^(k+2), k = 1..n_max, under the weight r^2 on [0, rc];
 *     written here through its closed form u^3 P_k^(2,6)(2u - 1), u = 1 - r/rc;
 *   - central atom: a Gaussian of weight central_weight at the origin in the
 *     channel of its own species;
 *   - power spectrum storage: channel pairs a <= a', off-diagonal pairs
 *     multiplied by sqrt(2), no l-dependent prefactor;
 *   - two-body: one term per unordered pair, half assigned to each atom;
 *     kernel f_cut(r) exp(-(r - x_m)^2 / (2 theta^2)).
 *
 * Parity unpinned: none of the functions below is unpinned; each is checked
 * by the CPU tests against closed forms, invariances, identities or finite
 * differences.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* Planted mistakes, for the tests that show the pins catch them: building
 * with -DORACLE_PLANT=k (k = 1..15, 26..31, 33) compiles mistake k, each marked
 * "planted k" where it sits.  The default, 0, compiles the oracle as written;
 * the tests, the smoke check and the benchmark's CPU legs all use that build. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif
#define PLANT(k) (ORACLE_PLANT == (k))

typedef struct {
    int n_max, l_max, n_species, mix_K;
    double rc, d, sigma, central_weight;
    const double *mix_w; /* [mix_K][n_species], used when mix_K > 0 */
    int quad_n;          /* Gauss-Legendre nodes of the radial integral (0: 160) */
} orc_soap;

typedef struct {
    int n_gp;                  /* GP s serves central atoms of species s, s < n_gp */
    const int *m_offsets;      /* [n_gp + 1] into the concatenated sparse arrays */
    const double *sparse;      /* [M_total][D] normalised sparse descriptors */
    const double *alpha;       /* [M_total] coefficients c_m of Eq. 2 */
    double delta;              /* energy_scale; kernel prefactor delta^2 */
    int zeta;                  /* integer exponent of Eq. 13 */
    int m2;                    /* two-body sparse points (0: no two-body term) */
    const double *x2, *alpha2; /* [m2] */
    double delta2, theta2, rc2, d2;
} orc_model;

/* ------------------------------------------------------------ utilities */

static double factorial(int n)
{
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    return factorial(n) / (factorial(k) * factorial(n - k));
}

static double ipow(double x, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= x;
    return r;
}

/* Gauss-Legendre nodes/weights on [a, b] by Newton iteration on P_n. */
static void gauss_legendre(int n, double a, double b, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = 0.5 * (b - a) * (-z) + 0.5 * (b + a);
        w[i] = (b - a) / ((1.0 - z * z) * dp * dp);
    }
}

/* ----------------------------------------------------- Eq. 18: cutoff */

double orc_fcut(double r, double rc, double d, double *dfdr)
{
    if (r >= rc) { if (dfdr) *dfdr = 0.0; return 0.0; }
    if (r < rc - d) { if (dfdr) *dfdr = 0.0; return 1.0; }
    double t = ORC_PI * (r - rc + d) / d;
    if (dfdr) *dfdr = (PLANT(9) ? 0.5 : -0.5) * sin(t) * ORC_PI / d; /* planted 9: sign */
    return 0.5 * (cos(t) + 1.0);
}

/* -------------------------------------------------- radial basis g_n(r)
 * Jacobi polynomial by its explicit sum (DLMF 18.5.8) with x = 2u - 1:
 *   P_k^(a,b)(2u-1) = sum_s C(k+a, k-s) C(k+b, s) (u-1)^s u^(k-s).
 * Norm: int_0^1 (1-u)^2 u^6 P_k^2 du = (k+2)!(k+6)! / ((2k+9)(k+8)! k!).   */
static double jacobi_26(int k, double u)
{
    double s = 0.0;
    for (int q = 0; q <= k; ++q)
        s += (PLANT(14) ? binom(k + 6, k - q) * binom(k + 2, q) /* planted 14: (a, b) swapped */
                        : binom(k + 2, k - q) * binom(k + 6, q)) *
             ipow(u - 1.0, q) * ipow(u, k - q);
    return s;
}

int orc_radial_basis(const orc_soap *P, double r, double *g)
{
    for (int n = 0; n < P->n_max; ++n) {
        if (r >= P->rc) { g[n] = 0.0; continue; }
        double u = 1.0 - r / P->rc;
        double nrm = factorial(n + 2) * factorial(n + 6) / ((2.0 * n + 9.0) * factorial(n + 8) * factorial(n));
        g[n] = u * u * u * jacobi_26(n, u) / sqrt(P->rc * P->rc * P->rc * nrm);
    }
    return 0;
}

/* ------------------------------- modified spherical Bessel i_l, scaled
 * Ascending series (Abramowitz & Stegun, Sec. 10.2):
 *   i_l(x) = x^l / (2l+1)!! * sum_k t_k,  t_0 = 1,
 *   t_k = t_{k-1} (x^2/2) / (k (2l + 2k + 1)).
 * Returns e^{-x} i_l(x); *deriv = e^{-x} i_l'(x) from the term-wise
 * derivative sum_k t_k (l + 2k) x^(l+2k-1) / (2l+1)!!.  All terms are
 * positive, so there is no cancellation.                                   */
double orc_bessel_scaled(int l, double x, double *deriv)
{
    double dfact = 1.0;
    for (int k = 1; k <= 2 * l + 1; k += 2) dfact *= k;
    double t = 1.0, s = 1.0, sd = (double)l;
    double h = 0.5 * x * x;
    for (int k = 1; k < 2000; ++k) {
        t *= h / (k * (2.0 * l + 2.0 * k + (PLANT(13) ? -1.0 : 1.0))); /* planted 13: off by one */
        s += t;
        sd += t * (l + 2.0 * k);
        if (t < 1e-18 * s) break;
    }
    double ex = exp(-x);
    if (deriv) {
        if (x == 0.0) *deriv = (l == 1) ? 1.0 / 3.0 : 0.0;
        else *deriv = ex * sd * ipow(x, l) / x / dfact;
    }
    return ex * s * ipow(x, l) / dfact;
}

/* -------------------------------------------- radial integral I_nl(rj)
 * Projection of one Gaussian (Eq. 19) on g_n Y_lm (Eq. 20) through the
 * plane-wave expansion e^{x cos t} = 4 pi sum_lm i_l(x) Y_lm Y_lm:
 *   I_nl(rj) = 4 pi int_0^rc r^2 g_n(r) e^{-(r^2 + rj^2)/2s^2} i_l(r rj/s^2) dr
 * and dI_nl/drj.  Gauss-Legendre quadrature on [0, rc].                    */
typedef struct {
    int q;
    double *x, *w, *g; /* nodes, weights, g_n(node) [q][N] */
} radial_quad;

static void radial_quad_init(const orc_soap *P, radial_quad *Q)
{
    Q->q = P->quad_n > 0 ? P->quad_n : 160;
    Q->x = (double *)malloc(sizeof(double) * Q->q);
    Q->w = (double *)malloc(sizeof(double) * Q->q);
    Q->g = (double *)malloc(sizeof(double) * Q->q * P->n_max);
    gauss_legendre(Q->q, 0.0, P->rc, Q->x, Q->w);
    for (int k = 0; k < Q->q; ++k) orc_radial_basis(P, Q->x[k], Q->g + (size_t)k * P->n_max);
}

static void radial_quad_free(radial_quad *Q)
{
    free(Q->x);
    free(Q->w);
    free(Q->g);
}

static void radial_integrals_q(const orc_soap *P, const radial_quad *Q, double rj, double *I, double *dI)
{
    int N = P->n_max, L = P->l_max;
    double s2 = P->sigma * P->sigma;
    memset(I, 0, sizeof(double) * N * (L + 1));
    if (dI) memset(dI, 0, sizeof(double) * N * (L + 1));
    double bes[32], dbes[32];
    for (int k = 0; k < Q->q; ++k) {
        double r = Q->x[k];
        double x = r * rj / s2;
        double gs = exp(-(r - rj) * (r - rj) / (2.0 * s2));
        for (int l = 0; l <= L; ++l) bes[l] = orc_bessel_scaled(l, x, &dbes[l]);
        for (int n = 0; n < N; ++n) {
            double wg = (PLANT(7) ? 1.0 : 4.0 * ORC_PI) /* planted 7: 4 pi dropped */ * Q->w[k] * r * r *
                        Q->g[(size_t)k * N + n] * gs;
            for (int l = 0; l <= L; ++l) {
                I[n * (L + 1) + l] += wg * bes[l];
                if (dI) dI[n * (L + 1) + l] += wg * (-(rj / s2) * bes[l] + (r / s2) * dbes[l]);
            }
        }
    }
}

int orc_radial_integrals(const orc_soap *P, double rj, double *I, double *dI)
{
    radial_quad Q;
    radial_quad_init(P, &Q);
    radial_integrals_q(P, &Q, rj, I, dI);
    radial_quad_free(&Q);
    return 0;
}

/* ------------------------------------------- real spherical harmonics
 * For a unit vector u = (x, y, z), with N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!):
 *   Y_l0    = N_l0 P_l(z)
 *   Y_l,m   = sqrt(2) N_lm P_l^(m)(z) Re (x + i y)^m     (m > 0)
 *   Y_l,-m  = sqrt(2) N_lm P_l^(m)(z) Im (x + i y)^m
 * where P_l^(m) is the m-th derivative of the Legendre polynomial, written
 * from its explicit coefficients
 *   P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k, l) z^(l-2k).
 * Index lm = l^2 + l + m.  dY (optional) is the gradient [lm][3] of this
 * polynomial in (x, y, z); its tangential part is the gradient on the sphere. */
static double legendre_deriv(int l, int m, double z)
{
    double s = 0.0;
    for (int k = 0; 2 * k <= l; ++k) {
        int e = l - 2 * k;
        if (e < m) continue;
        double a = ((k & 1) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l) / ipow(2.0, l);
        s += a * factorial(e) / factorial(e - m) * ipow(z, e - m);
    }
    return s;
}

/* Re/Im of (x + i y)^m and their x, y derivatives by the binomial theorem. */
static void xy_power(int m, double x, double y, double *re, double *im, double *dre, double *dim)
{
    *re = *im = 0.0;
    dre[0] = dre[1] = dim[0] = dim[1] = 0.0;
    for (int k = 0; k <= m; ++k) {
        double c = binom(m, k);
        double sgn = ((k / 2) & 1) ? -1.0 : 1.0;
        double v = c * sgn * ipow(x, m - k) * ipow(y, k);
        double vx = (m - k > 0) ? c * sgn * (m - k) * ipow(x, m - k - 1) * ipow(y, k) : 0.0;
        double vy = (k > 0) ? c * sgn * k * ipow(x, m - k) * ipow(y, k - 1) : 0.0;
        if ((k & 1) == 0) { *re += v; dre[0] += vx; dre[1] += vy; }
        else { *im += v; dim[0] += vx; dim[1] += vy; }
    }
}

int orc_ylm(int L, const double *u, double *Y, double *dY)
{
    double x = u[0], y = u[1], z = u[2];
    for (int l = 0; l <= L; ++l) {
        for (int m = 0; m <= l; ++m) {
            double nlm = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * factorial(l - m) / factorial(l + m));
            double pm = legendre_deriv(l, m, z), pm1 = legendre_deriv(l, m + 1, z);
            if (m == 0) {
                Y[l * l + l] = nlm * pm;
                if (dY) {
                    double *g = dY + 3 * (l * l + l);
                    g[0] = 0.0; g[1] = 0.0; g[2] = nlm * pm1;
                }
                continue;
            }
            double re, im, dre[2], dim[2];
            xy_power(m, x, y, &re, &im, dre, dim);
            double c = sqrt(2.0) * nlm;
            int ip = l * l + l + m, in = l * l + l - m;
            if (PLANT(6)) { ip = l * l + l - m; in = l * l + l + m; } /* planted 6: m and -m swapped */
            Y[ip] = c * pm * re;
            Y[in] = c * pm * im;
            if (dY) {
                double *gp = dY + 3 * ip, *gn = dY + 3 * in;
                gp[0] = c * pm * dre[0]; gp[1] = c * pm * dre[1]; gp[2] = c * pm1 * re;
                gn[0] = c * pm * dim[0]; gn[1] = c * pm * dim[1]; gn[2] = c * pm1 * im;
            }
        }
    }
    return 0;
}

/* ----------------------------------------------- channel bookkeeping
 * Channels a of group g carry the coefficients coupled in the power spectrum:
 *   mix_K = 0: one group, channels (species s, radial n), a = s*N + n, and the
 *              weight of a neighbour of species z in channel a is [s == z];
 *   mix_K > 0: K groups (embedded channels k), channels n, weight w^k_z
 *              (Eq. 25 with Z_mix=T, R_mix=F, coupling=F: element-wise in k,
 *              tensor product in n, giving p^k_nn'l).                        */
typedef struct {
    int G, Nc, N, L, LM, S, D, npair;
} layout;

static layout make_layout(const orc_soap *P)
{
    layout Y;
    Y.N = P->n_max;
    Y.L = P->l_max;
    Y.LM = (P->l_max + 1) * (P->l_max + 1);
    Y.S = P->n_species;
    if (P->mix_K > 0) { Y.G = P->mix_K; Y.Nc = P->n_max; }
    else { Y.G = 1; Y.Nc = P->n_species * P->n_max; }
    Y.npair = Y.Nc * (Y.Nc + 1) / 2;
    Y.D = Y.G * Y.npair * (Y.L + 1);
    return Y;
}

static double chan_weight(const orc_soap *P, const layout *Y, int g, int a, int z)
{
    if (P->mix_K > 0) /* planted 15: [species][K] read */
        return PLANT(15) ? P->mix_w[z * P->mix_K + g] : P->mix_w[g * P->n_species + z];
    return (a / Y->N == z) ? 1.0 : 0.0;
}

static int chan_radial(const layout *Y, int a) { return a % Y->N; }

int orc_dim(const orc_soap *P) { return make_layout(P).D; }

/* ------------------------------------------------------- neighbours
 * All (j, T) with |r_j + T - r_i| < rc, T = n1 a1 + n2 a2 + n3 a3, over every
 * atom j and every integer shift whose fractional offset can reach rc
 * (brute force; j = i allowed for T != 0).  Ordered by (j, n1, n2, n3).    */
typedef struct {
    int n;
    int *j;
    int *shift; /* [n][3] */
    double *vec; /* [n][3] r_j + T - r_i */
} nlist;

static void inv3(const double *c, double *inv)
{
    double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                 c[2] * (c[3] * c[7] - c[4] * c[6]);
    inv[0] = (c[4] * c[8] - c[5] * c[7]) / det;
    inv[1] = (c[2] * c[7] - c[1] * c[8]) / det;
    inv[2] = (c[1] * c[5] - c[2] * c[4]) / det;
    inv[3] = (c[5] * c[6] - c[3] * c[8]) / det;
    inv[4] = (c[0] * c[8] - c[2] * c[6]) / det;
    inv[5] = (c[2] * c[3] - c[0] * c[5]) / det;
    inv[6] = (c[3] * c[7] - c[4] * c[6]) / det;
    inv[7] = (c[1] * c[6] - c[0] * c[7]) / det;
    inv[8] = (c[0] * c[4] - c[1] * c[3]) / det;
}

static void neighbours_of(int n, const double *pos, const double *cell, const int *pbc, double rc, int i,
                          nlist *out)
{
    double inv[9], width[3];
    inv3(cell, inv);
    /* perpendicular width of the cell along axis k: 1 / |column k of inv| */
    for (int k = 0; k < 3; ++k)
        width[k] = 1.0 / sqrt(inv[k] * inv[k] + inv[3 + k] * inv[3 + k] + inv[6 + k] * inv[6 + k]);
    int cap = 64, cnt = 0;
    int *jj = (int *)malloc(sizeof(int) * cap);
    int *sh = (int *)malloc(sizeof(int) * cap * 3);
    double *vv = (double *)malloc(sizeof(double) * cap * 3);
    const double *ri = pos + 3 * i;
    for (int j = 0; j < n; ++j) {
        const double *rj = pos + 3 * j;
        double dv[3] = {rj[0] - ri[0], rj[1] - ri[1], rj[2] - ri[2]};
        double fd[3];
        for (int k = 0; k < 3; ++k) /* planted 26: the inverse cell read transposed */
            fd[k] = PLANT(26) ? dv[0] * inv[3 * k] + dv[1] * inv[3 * k + 1] + dv[2] * inv[3 * k + 2]
                              : dv[0] * inv[k] + dv[1] * inv[3 + k] + dv[2] * inv[6 + k];
        int lo[3], hi[3];
        for (int k = 0; k < 3; ++k) {
            if (pbc[k]) {
                lo[k] = (int)ceil(-rc / width[k] - fd[k]) - 1;
                hi[k] = (int)floor(rc / width[k] - fd[k]) + 1;
            } else lo[k] = hi[k] = 0;
        }
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c) {
                    if (j == i && (PLANT(8) || (a == 0 && b == 0 && c == 0))) continue; /* planted 8: no self images */
                    double v[3];
                    for (int k = 0; k < 3; ++k) v[k] = dv[k] + a * cell[k] + b * cell[3 + k] + c * cell[6 + k];
                    double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                    if (r2 >= rc * rc) continue;
                    if (cnt == cap) {
                        cap *= 2;
                        jj = (int *)realloc(jj, sizeof(int) * cap);
                        sh = (int *)realloc(sh, sizeof(int) * cap * 3);
                        vv = (double *)realloc(vv, sizeof(double) * cap * 3);
                    }
                    jj[cnt] = j;
                    sh[3 * cnt] = a; sh[3 * cnt + 1] = b; sh[3 * cnt + 2] = c;
                    vv[3 * cnt] = v[0]; vv[3 * cnt + 1] = v[1]; vv[3 * cnt + 2] = v[2];
                    ++cnt;
                }
    }
    out->n = cnt;
    out->j = jj;
    out->shift = sh;
    out->vec = vv;
}

static void nlist_free(nlist *L)
{
    free(L->j);
    free(L->shift);
    free(L->vec);
}

long orc_neighbours(int n, const double *pos, const double *cell, const int *pbc, double rc, int i, long cap,
                    int *j_out, int *shift_out, double *vec_out)
{
    nlist L;
    neighbours_of(n, pos, cell, pbc, rc, i, &L);
    long m = L.n;
    for (long k = 0; k < m && k < cap; ++k) {
        j_out[k] = L.j[k];
        for (int a = 0; a < 3; ++a) {
            shift_out[3 * k + a] = L.shift[3 * k + a];
            vec_out[3 * k + a] = L.vec[3 * k + a];
        }
    }
    nlist_free(&L);
    return m;
}

/* ------------------------------------------------ one atomic environment */
typedef struct {
    nlist nb;
    int np;          /* SOAP pairs (r < rc); nb may hold more for the two-body cutoff */
    int *pidx;       /* [np] index into nb of each SOAP pair */
    double *coef;    /* [G][Nc][LM] */
    double *dcoef;   /* [np][G][Nc][LM][3] derivative wrt r_ij */
    double *p, *phat;/* [D] */
    double pnorm;
    double *jac;     /* [np][D][3] d phat / d r_ij */
} env;

static void env_free(env *E)
{
    nlist_free(&E->nb);
    free(E->pidx);
    free(E->coef);
    free(E->dcoef);
    free(E->p);
    free(E->phat);
    free(E->jac);
}

/* Builds c, p, p_hat of atom i (Eqs. 19-25) and, if want_jac, dp_hat/dr_ij. */
static void env_build(const orc_soap *P, const radial_quad *Q, int n, const double *pos, const int *spec,
                      const double *cell, const int *pbc, int i, double rsearch, int want_jac, env *E)
{
    layout Y = make_layout(P);
    int N = Y.N, L = Y.L, LM = Y.LM, G = Y.G, Nc = Y.Nc, D = Y.D;
    size_t ncoef = (size_t)G * Nc * LM;
    neighbours_of(n, pos, cell, pbc, rsearch, i, &E->nb);
    E->pidx = (int *)malloc(sizeof(int) * (E->nb.n + 1));
    E->np = 0;
    for (int k = 0; k < E->nb.n; ++k) {
        const double *v = E->nb.vec + 3 * k;
        if (v[0] * v[0] + v[1] * v[1] + v[2] * v[2] < P->rc * P->rc) E->pidx[E->np++] = k;
    }
    E->coef = (double *)calloc(ncoef, sizeof(double));
    E->dcoef = want_jac ? (double *)calloc(ncoef * 3 * (E->np + 1), sizeof(double)) : NULL;
    E->p = (double *)calloc(D, sizeof(double));
    E->phat = (double *)calloc(D, sizeof(double));
    E->jac = want_jac ? (double *)calloc((size_t)D * 3 * (E->np + 1), sizeof(double)) : NULL;

    double *I = (double *)malloc(sizeof(double) * N * (L + 1));
    double *dI = (double *)malloc(sizeof(double) * N * (L + 1));
    double *Yv = (double *)malloc(sizeof(double) * LM);
    double *dY = (double *)malloc(sizeof(double) * LM * 3);

    /* central Gaussian at the origin (Eq. 19 with r_i = 0, f_cut(0) = 1) */
    if (P->central_weight != 0.0) {
        radial_integrals_q(P, Q, 0.0, I, NULL);
        double u0[3] = {0.0, 0.0, 1.0};
        orc_ylm(L, u0, Yv, NULL);
        for (int g = 0; g < G; ++g)
            for (int a = 0; a < Nc; ++a) {
                double w = (PLANT(31) ? 1.0 : chan_weight(P, &Y, g, a, spec[i])) /* planted 31: every channel */
                           * P->central_weight;
                E->coef[((size_t)g * Nc + a) * LM + 0] += w * I[chan_radial(&Y, a) * (L + 1) + 0] * Yv[0];
            }
    }
    /* neighbours: c_nlm += w f_cut(r) I_nl(r) Y_lm(u)  (Eqs. 19-20) */
    for (int q = 0; q < E->np; ++q) {
        int k = E->pidx[q];
        const double *v = E->nb.vec + 3 * k;
        int z = spec[E->nb.j[k]];
        double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double u[3] = {v[0] / r, v[1] / r, v[2] / r};
        double df, f = orc_fcut(r, P->rc, P->d, &df);
        radial_integrals_q(P, Q, r, I, dI);
        orc_ylm(L, u, Yv, dY);
        /* gradient of Y_lm(v/|v|) wrt v: tangential part of dY, divided by r */
        for (int lm = 0; lm < LM; ++lm) {
            double *gy = dY + 3 * lm;
            double ud = gy[0] * u[0] + gy[1] * u[1] + gy[2] * u[2];
            for (int a = 0; a < 3; ++a) gy[a] = (gy[a] - ud * u[a]) / r;
        }
        for (int g = 0; g < G; ++g)
            for (int a = 0; a < Nc; ++a) {
                double w = chan_weight(P, &Y, g, a, z);
                if (w == 0.0) continue;
                int nr = chan_radial(&Y, a);
                for (int l = 0; l <= L; ++l) {
                    double R = f * I[nr * (L + 1) + l];
                    double dR = df * I[nr * (L + 1) + l] + f * dI[nr * (L + 1) + l];
                    for (int m = -l; m <= l; ++m) {
                        int lm = l * l + l + m;
                        size_t ci = ((size_t)g * Nc + a) * LM + lm;
                        E->coef[ci] += w * R * Yv[lm];
                        if (want_jac) {
                            double *dc = E->dcoef + ((size_t)q * ncoef + ci) * 3;
                            for (int x = 0; x < 3; ++x) dc[x] = w * (dR * u[x] * Yv[lm] + R * dY[3 * lm + x]);
                        }
                    }
                }
            }
    }
    /* power spectrum (Eqs. 22-23, 25): p_{g,a,a',l} = s_aa' sum_m c_alm c_a'lm */
    int d = 0;
    for (int g = 0; g < G; ++g)
        for (int a = 0; a < Nc; ++a)
            for (int b = a; b < Nc; ++b) {
                double s = (a == b || PLANT(1)) ? 1.0 : sqrt(2.0); /* planted 1: no sqrt 2 */
                for (int l = 0; l <= L; ++l, ++d) {
                    double acc = 0.0;
                    for (int m = -l; m <= l; ++m) {
                        int lm = l * l + l + m;
                        acc += E->coef[((size_t)g * Nc + a) * LM + lm] * E->coef[((size_t)g * Nc + b) * LM + lm];
                    }
                    E->p[d] = s * acc;
                }
            }
    /* normalisation (Eq. 24) */
    double nn = 0.0;
    for (int k = 0; k < D; ++k) nn += E->p[k] * E->p[k];
    E->pnorm = sqrt(nn);
    for (int k = 0; k < D; ++k) E->phat[k] = E->p[k] / E->pnorm;

    if (want_jac) {
        double *dp = (double *)malloc(sizeof(double) * D * 3);
        for (int q = 0; q < E->np; ++q) {
            const double *dc = E->dcoef + (size_t)q * ncoef * 3;
            int dd = 0;
            for (int g = 0; g < G; ++g)
                for (int a = 0; a < Nc; ++a)
                    for (int b = a; b < Nc; ++b) {
                        double s = (a == b || PLANT(1)) ? 1.0 : sqrt(2.0); /* planted 1 */
                        for (int l = 0; l <= L; ++l, ++dd)
                            for (int x = 0; x < 3; ++x) {
                                double acc = 0.0;
                                for (int m = -l; m <= l; ++m) {
                                    int lm = l * l + l + m;
                                    size_t ia = ((size_t)g * Nc + a) * LM + lm, ib = ((size_t)g * Nc + b) * LM + lm;
                                    acc += dc[ia * 3 + x] * E->coef[ib] + E->coef[ia] * dc[ib * 3 + x];
                                }
                                dp[dd * 3 + x] = s * acc;
                            }
                    }
            /* d p_hat = (dp - p_hat (p_hat . dp)) / |p| */
            for (int x = 0; x < 3; ++x) {
                double pd = 0.0;
                for (int k = 0; k < D; ++k) pd += E->phat[k] * dp[k * 3 + x];
                for (int k = 0; k < D; ++k)
                    E->jac[((size_t)q * D + k) * 3 + x] =
                        (dp[k * 3 + x] - E->phat[k] * (PLANT(2) ? -pd : pd)) / E->pnorm; /* planted 2: sign */
            }
        }
        free(dp);
    }
    free(I);
    free(dI);
    free(Yv);
    free(dY);
}

/* ------------------------------------------------------- descriptors */
int orc_descriptor(const orc_soap *P, int n, const double *pos, const int *spec, const double *cell,
                   const int *pbc, int n_sel, const int *sel, double *phat, double *pnorm, double *coef)
{
    layout Y = make_layout(P);
    radial_quad Q;
    radial_quad_init(P, &Q);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < n_sel; ++t) {
        env E;
        env_build(P, &Q, n, pos, spec, cell, pbc, sel ? sel[t] : t, P->rc, 0, &E);
        memcpy(phat + (size_t)t * Y.D, E.phat, sizeof(double) * Y.D);
        if (pnorm) pnorm[t] = E.pnorm;
        if (coef) memcpy(coef + (size_t)t * Y.G * Y.Nc * Y.LM, E.coef, sizeof(double) * Y.G * Y.Nc * Y.LM);
        env_free(&E);
    }
    radial_quad_free(&Q);
    return 0;
}

/* --------------------------------------------- GP of a central atom
 * eps = delta^2 sum_m alpha_m (p_hat . x_m)^zeta          (Eqs. 2, 13)
 * grad = d eps / d p_hat = delta^2 sum_m alpha_m zeta q^(zeta-1) x_m       */
static double gp_eval(const orc_model *Mo, int D, int s, const double *phat, double *grad)
{
    if (grad) memset(grad, 0, sizeof(double) * D);
    if (s >= Mo->n_gp) return 0.0;
    double eps = 0.0, d2 = Mo->delta * Mo->delta;
    const int zeta = Mo->zeta + PLANT(3); /* planted 3: exponent zeta + 1 */
    for (int m = Mo->m_offsets[s]; m < Mo->m_offsets[s + 1]; ++m) {
        const double *x = Mo->sparse + (size_t)m * D;
        double q = 0.0;
        for (int k = 0; k < D; ++k) q += phat[k] * x[k];
        eps += d2 * Mo->alpha[m] * ipow(q, zeta);
        if (grad) {
            double c = d2 * Mo->alpha[m] * zeta * ipow(q, zeta - 1);
            for (int k = 0; k < D; ++k) grad[k] += c * x[k];
        }
    }
    return eps;
}

/* two-body energy of one pair at distance r, and de/dr (Eqs. 10-11, f_cut) */
static double pair_energy(const orc_model *Mo, double r, double *dedr)
{
    double df, f = orc_fcut(r, Mo->rc2, Mo->d2, &df);
    double e = 0.0, de = 0.0, d2 = Mo->delta2 * Mo->delta2, t2 = Mo->theta2 * Mo->theta2;
    for (int m = 0; m < Mo->m2; ++m) {
        double dx = r - Mo->x2[m];
        double k = exp(-dx * dx / (2.0 * t2));
        e += d2 * Mo->alpha2[m] * f * k;
        de += d2 * Mo->alpha2[m] * (df + (PLANT(30) ? f : -f) * dx / t2) * k; /* planted 30: sign */
    }
    if (dedr) *dedr = de;
    return e;
}

/* Local energy of atom i and d eps_i / d r_ij for every pair of its list
 * (SOAP through Eq. 3, plus half of each two-body pair term).               */
typedef struct {
    double eps;
    nlist nb;
    double *f; /* [nb.n][3] */
} local_grad;

static double search_radius(const orc_soap *P, const orc_model *Mo)
{
    double r = P->rc;
    if (Mo && Mo->m2 > 0 && Mo->rc2 > r) r = Mo->rc2;
    return r;
}

static void local_eval(const orc_soap *P, const orc_model *Mo, const radial_quad *Q, int n, const double *pos,
                       const int *spec, const double *cell, const int *pbc, int i, local_grad *out)
{
    layout Y = make_layout(P);
    int D = Y.D;
    env E;
    env_build(P, Q, n, pos, spec, cell, pbc, i, search_radius(P, Mo), 1, &E);
    double *grad = (double *)malloc(sizeof(double) * D);
    out->eps = gp_eval(Mo, D, spec[i], E.phat, grad);
    out->f = (double *)calloc((size_t)3 * (E.nb.n + 1), sizeof(double));
    for (int q = 0; q < E.np; ++q) {
        int k = E.pidx[q];
        for (int x = 0; x < 3; ++x) {
            double acc = 0.0;
            for (int dd = 0; dd < D; ++dd) acc += E.jac[((size_t)q * D + dd) * 3 + x] * grad[dd];
            out->f[3 * k + x] = acc;
        }
    }
    if (Mo->m2 > 0) {
        for (int k = 0; k < E.nb.n; ++k) {
            const double *v = E.nb.vec + 3 * k;
            double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (r >= Mo->rc2) continue;
            double de, e = pair_energy(Mo, r, &de);
            const double h = PLANT(10) ? 1.0 : 0.5; /* planted 10: whole pair term to each atom */
            out->eps += h * e;
            for (int x = 0; x < 3; ++x) out->f[3 * k + x] += h * de * v[x] / r;
        }
    }
    out->nb = E.nb;
    E.nb.j = NULL; E.nb.shift = NULL; E.nb.vec = NULL;
    env_free(&E);
    free(grad);
}

/* ------------------------------------------------------------ predict
 * energy = sum_i eps_i (Eq. 1); F_j = -dE/dr_j; virial
 * V_ab = -dE/d e_ab for the homogeneous strain r -> (I + e) r, i.e.
 * V_ab = -sum_pairs (d eps_i / d r_ij)_a (r_ij)_b.                          */
int orc_predict(const orc_soap *P, const orc_model *Mo, int n, const double *pos, const int *spec,
                const double *cell, const int *pbc, double *energy, double *local_e, double *forces,
                double *virial)
{
    radial_quad Q;
    radial_quad_init(P, &Q);
    local_grad *lg = (local_grad *)malloc(sizeof(local_grad) * n);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n; ++i) local_eval(P, Mo, &Q, n, pos, spec, cell, pbc, i, &lg[i]);
    double E = 0.0, V[9] = {0};
    if (forces) memset(forces, 0, sizeof(double) * 3 * n);
    for (int i = 0; i < n; ++i) {
        E += lg[i].eps;
        if (local_e) local_e[i] = lg[i].eps;
        for (int k = 0; k < lg[i].nb.n; ++k) {
            const double *f = lg[i].f + 3 * k, *v = lg[i].nb.vec + 3 * k;
            int j = lg[i].nb.j[k];
            const double sf = PLANT(5) ? -1.0 : 1.0; /* planted 5: F = +dE/dr */
            if (forces)
                for (int x = 0; x < 3; ++x) {
                    forces[3 * j + x] -= sf * f[x];
                    forces[3 * i + x] += sf * f[x];
                }
            const double sv = PLANT(4) ? -1.0 : 1.0; /* planted 4: virial sign */
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) V[3 * a + b] -= sv * f[a] * v[b];
        }
        nlist_free(&lg[i].nb);
        free(lg[i].f);
    }
    if (energy) *energy = E;
    if (virial) memcpy(virial, V, sizeof(V));
    free(lg);
    radial_quad_free(&Q);
    return 0;
}

/* Local energies and forces of the selected atoms only (for cells too large
 * for the full oracle): F_t needs every eps_i that depends on r_t, i.e. t
 * and its neighbours.                                                       */
int orc_predict_sampled(const orc_soap *P, const orc_model *Mo, int n, const double *pos, const int *spec,
                        const double *cell, const int *pbc, int n_sel, const int *sel, double *local_e,
                        double *forces)
{
    radial_quad Q;
    radial_quad_init(P, &Q);
    double rs = search_radius(P, Mo);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < n_sel; ++t) {
        int at = sel[t];
        nlist nb;
        neighbours_of(n, pos, cell, pbc, rs, at, &nb);
        /* distinct atoms that can depend on r_at: at itself and its neighbours */
        int *set = (int *)malloc(sizeof(int) * (nb.n + 1));
        int ns = 0;
        set[ns++] = at;
        for (int k = 0; k < nb.n; ++k) {
            int j = nb.j[k], seen = 0;
            for (int s = 0; s < ns; ++s) if (set[s] == j) { seen = 1; break; }
            if (!seen) set[ns++] = j;
        }
        double F[3] = {0, 0, 0};
        for (int s = 0; s < ns; ++s) {
            local_grad g;
            local_eval(P, Mo, &Q, n, pos, spec, cell, pbc, set[s], &g);
            if (set[s] == at && local_e) local_e[t] = g.eps;
            for (int k = 0; k < g.nb.n; ++k) {
                for (int x = 0; x < 3; ++x) {
                    if (g.nb.j[k] == at && !(PLANT(28) && set[s] != at)) /* planted 28: neighbours' terms dropped */
                        F[x] -= g.f[3 * k + x];
                    if (set[s] == at) F[x] += g.f[3 * k + x];
                }
            }
            nlist_free(&g.nb);
            free(g.f);
        }
        for (int x = 0; x < 3; ++x) forces[3 * t + x] = F[x];
        free(set);
        nlist_free(&nb);
    }
    radial_quad_free(&Q);
    return 0;
}

/* ---------------------------------------------------------- K_NM rows
 * One configuration, rows [1 + 3n][M_total] (columns: all GPs' sparse
 * points, concatenated):
 *   energy row   K[0][m]       = sum_i k(p_hat_i, x_m)
 *   force rows   K[1+3j+a][m]  = -sum_i d k(p_hat_i, x_m) / d r_ja
 * with k = delta^2 (p_hat . x_m)^zeta, nonzero only for columns of the GP
 * of atom i's species; d p_hat_i / d r_i = -sum_j d p_hat_i / d r_ij.        */
int orc_knm(const orc_soap *P, const orc_model *Mo, int n, const double *pos, const int *spec,
            const double *cell, const int *pbc, double *rows)
{
    layout Y = make_layout(P);
    int D = Y.D;
    int Mt = Mo->m_offsets[Mo->n_gp];
    radial_quad Q;
    radial_quad_init(P, &Q);
    env *E = (env *)malloc(sizeof(env) * n);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n; ++i) env_build(P, &Q, n, pos, spec, cell, pbc, i, P->rc, 1, &E[i]);
    memset(rows, 0, sizeof(double) * (size_t)(1 + 3 * n) * Mt);
    double d2 = Mo->delta * Mo->delta;
    const int zeta = Mo->zeta + PLANT(3); /* planted 3 */
    const double sk = PLANT(12) ? -1.0 : 1.0; /* planted 12: force rows +grad */
#pragma omp parallel for schedule(static)
    for (int m = 0; m < Mt; ++m) {
        int s = 0;
        while (s < Mo->n_gp && m >= Mo->m_offsets[s + 1]) ++s;
        const double *x = Mo->sparse + (size_t)m * D;
        for (int i = 0; i < n; ++i) {
            if (spec[i] != s) continue;
            double q = 0.0;
            for (int k = 0; k < D; ++k) q += E[i].phat[k] * x[k];
            rows[m] += d2 * ipow(q, zeta);
            double c = sk * d2 * zeta * ipow(q, zeta - 1);
            for (int p = 0; p < E[i].np; ++p) {
                int j = E[i].nb.j[E[i].pidx[p]];
                for (int a = 0; a < 3; ++a) {
                    double t = 0.0;
                    for (int k = 0; k < D; ++k) t += x[k] * E[i].jac[((size_t)p * D + k) * 3 + a];
                    t *= c;
                    rows[(size_t)(1 + 3 * j + a) * Mt + m] -= t;
                    rows[(size_t)(1 + 3 * i + a) * Mt + m] += t;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) env_free(&E[i]);
    free(E);
    radial_quad_free(&Q);
    return 0;
}

/* K_MM of GP s: delta^2 (x_m . x_m')^zeta (Eq. 13) */
int orc_kmm(const orc_model *Mo, int D, int s, double *out)
{
    int a = Mo->m_offsets[s], M = Mo->m_offsets[s + 1] - a;
    double d2 = Mo->delta * Mo->delta;
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) {
            double v = 0.0;
            for (int k = 0; k < D; ++k) v += Mo->sparse[(size_t)(a + p) * D + k] * Mo->sparse[(size_t)(a + q) * D + k];
            out[(size_t)p * M + q] = d2 * ipow(v, Mo->zeta + PLANT(27)); /* planted 27: exponent zeta + 1 */
        }
    return 0;
}

/* ---------------------------------------------------- regularised fit */
static int cholesky_upper(int M, double *A) /* A = U^T U in place (upper), lower zeroed */
{
    for (int j = 0; j < M; ++j) {
        double s = A[(size_t)j * M + j];
        for (int k = 0; k < j; ++k) s -= A[(size_t)k * M + j] * A[(size_t)k * M + j];
        if (s <= 0.0) return -5;
        double ujj = sqrt(s);
        A[(size_t)j * M + j] = ujj;
        for (int i = j + 1; i < M; ++i) {
            double t = A[(size_t)j * M + i];
            for (int k = 0; k < j && !PLANT(33); ++k) /* planted 33: update of the row dropped */
                t -= A[(size_t)k * M + j] * A[(size_t)k * M + i];
            A[(size_t)j * M + i] = t / ujj;
        }
        for (int i = j + 1; i < M; ++i) A[(size_t)i * M + j] = 0.0;
    }
    return 0;
}

/* Eq. 4: c = [K_MM + K^T S^-1 K]^-1 K^T S^-1 y with S = diag(sigma^2) and
 * jitter added to the diagonal of K_MM; solved by Cholesky.                 */
int orc_solve_normal(long R, int M, const double *K, const double *y, const double *sigma, const double *kmm,
                     double jitter, double *c)
{
    double *B = (double *)malloc(sizeof(double) * (size_t)M * M);
    double *rhs = (double *)calloc(M, sizeof(double));
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) B[(size_t)p * M + q] = kmm[(size_t)p * M + q] + (p == q ? jitter : 0.0);
#pragma omp parallel for schedule(static)
    for (int p = 0; p < M; ++p) {
        for (long r = 0; r < R; ++r) {
            double w = K[(size_t)r * M + p] / (PLANT(29) ? sigma[r] : sigma[r] * sigma[r]); /* planted 29: sigma not squared */
            if (w == 0.0) continue;
            for (int q = 0; q < M; ++q) B[(size_t)p * M + q] += w * K[(size_t)r * M + q];
            rhs[p] += w * y[r];
        }
    }
    int st = cholesky_upper(M, B);
    if (st == 0) {
        /* U^T z = rhs, then U c = z */
        for (int i = 0; i < M; ++i) {
            double s = rhs[i];
            for (int k = 0; k < i; ++k) s -= B[(size_t)k * M + i] * c[k];
            c[i] = s / B[(size_t)i * M + i];
        }
        for (int i = M - 1; i >= 0; --i) {
            double s = c[i];
            for (int k = i + 1; k < M; ++k) s -= B[(size_t)i * M + k] * c[k];
            c[i] = s / B[(size_t)i * M + i];
        }
    }
    free(B);
    free(rhs);
    return st;
}

/* Eqs. 5-9: A = [S^-1/2 K ; U_MM], b = [S^-1/2 y ; 0], Householder QR A = QR,
 * c = R^-1 Q^T b.                                                           */
int orc_solve_qr(long R, int M, const double *K, const double *y, const double *sigma, const double *kmm,
                 double jitter, double *c)
{
    long rows = R + M;
    double *A = (double *)malloc(sizeof(double) * (size_t)rows * M);
    double *b = (double *)malloc(sizeof(double) * rows);
    double *U = (double *)malloc(sizeof(double) * (size_t)M * M);
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) U[(size_t)p * M + q] = kmm[(size_t)p * M + q] + (p == q ? jitter : 0.0);
    int st = cholesky_upper(M, U);
    if (st) { free(A); free(b); free(U); return st; }
    for (long r = 0; r < R; ++r) {
        for (int q = 0; q < M; ++q) A[(size_t)r * M + q] = K[(size_t)r * M + q] / sigma[r];
        b[r] = PLANT(11) ? y[r] : y[r] / sigma[r]; /* planted 11: b not scaled by S^-1/2 */
    }
    for (int p = 0; p < M; ++p) {
        for (int q = 0; q < M; ++q) A[(size_t)(R + p) * M + q] = U[(size_t)p * M + q];
        b[R + p] = 0.0;
    }
    double *v = (double *)malloc(sizeof(double) * rows);
    for (int k = 0; k < M; ++k) {
        double nrm = 0.0;
        for (long r = k; r < rows; ++r) nrm += A[(size_t)r * M + k] * A[(size_t)r * M + k];
        nrm = sqrt(nrm);
        double alpha = A[(size_t)k * M + k] > 0 ? -nrm : nrm;
        double vn = 0.0;
        for (long r = k; r < rows; ++r) v[r] = A[(size_t)r * M + k];
        v[k] -= alpha;
        for (long r = k; r < rows; ++r) vn += v[r] * v[r];
        if (vn == 0.0) continue;
        /* apply H = I - 2 v v^T / (v^T v) to A[k:, k:] and b */
#pragma omp parallel for schedule(static)
        for (int q = k; q < M; ++q) {
            double s = 0.0;
            for (long r = k; r < rows; ++r) s += v[r] * A[(size_t)r * M + q];
            s = 2.0 * s / vn;
            for (long r = k; r < rows; ++r) A[(size_t)r * M + q] -= s * v[r];
        }
        double s = 0.0;
        for (long r = k; r < rows; ++r) s += v[r] * b[r];
        s = 2.0 * s / vn;
        for (long r = k; r < rows; ++r) b[r] -= s * v[r];
    }
    for (int i = M - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < M; ++k) s -= A[(size_t)i * M + k] * c[k];
        c[i] = s / A[(size_t)i * M + i];
    }
    free(v);
    free(A);
    free(b);
    free(U);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
