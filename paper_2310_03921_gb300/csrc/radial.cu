// Radial basis and radial-integral table (setup, once per descriptor).
//
// Basis: the orthonormal radial functions g_n of Eq. 20, taken as the
// Gram-Schmidt orthonormalisation (weight r^2 on [0, r_c], increasing power)
// of (r_c - r)^(k+2), k = 1..n_max.  With u = 1 - r/r_c this is
// g_n = u^3 P_n^(2,6)(2u - 1) / norm_n; here P is generated by the Jacobi
// three-term recurrence (DLMF 18.9.2) and norm_n is computed by quadrature.
//
// Table: I_nl(r) = 4 pi int_0^rc s^2 g_n(s) exp(-(s^2 + r^2)/(2 sigma^2))
// i_l(r s / sigma^2) ds (the projection of one Gaussian of Eq. 19 on
// g_n Y_lm) and dI_nl/dr at r_k = k h, k = 0..G, by Clenshaw-Curtis
// quadrature in FP64; the modified spherical Bessel functions come from
// Miller's downward recurrence normalised by e^-x i_0(x) = (1 - e^-2x)/(2x).
#include "gap_internal.h"
#include "radial.h"

#include <cmath>
#include <vector>

namespace {

constexpr int kMaxL = GAP_MAX_L + 2;

// e^-x i_l(x) and e^-x i_l'(x) for l = 0..Lp (Lp <= kMaxL - 1).
__device__ void bessel_scaled_all(int Lp, double x, double *iv, double *dv)
{
    double df = 1.0;  // (2l+1)!!
    if (x < 1e-3) {
        double ex = exp(-x), xl = 1.0, xlm1 = 0.0;  // x^l, x^(l-1)
        for (int l = 0; l <= Lp; ++l) {
            df *= (2 * l + 1);
            double c1 = 1.0 / (2.0 * (2 * l + 3)), c2 = 1.0 / (8.0 * (2 * l + 3) * (2 * l + 5));
            double x2 = x * x;
            iv[l] = ex * xl / df * (1.0 + c1 * x2 + c2 * x2 * x2);
            double di = (l * xlm1 + (l + 2) * c1 * xl * x + (l + 4) * c2 * xl * x2 * x) / df;
            dv[l] = ex * di;  // e^-x i_l'(x)
            xlm1 = xl;
            xl *= x;
        }
        return;
    }
    int ls = Lp + 24 + (int)(1.3 * x);
    double pp = 0.0, p = 1e-280;  // p_{l+1}, p_l
    double keep[kMaxL + 1];
    for (int l = 0; l <= Lp + 1; ++l) keep[l] = 0.0;
    for (int l = ls; l >= 1; --l) {
        double pm = pp + (2.0 * l + 1.0) / x * p;  // p_{l-1}
        if (l <= Lp + 1) keep[l] = p;
        pp = p;
        p = pm;
        if (fabs(p) > 1e250) {
            p *= 1e-250;
            pp *= 1e-250;
            for (int q = 0; q <= Lp + 1; ++q) keep[q] *= 1e-250;
        }
    }
    keep[0] = p;
    double i0 = -expm1(-2.0 * x) / (2.0 * x);
    double s = i0 / keep[0];
    for (int l = 0; l <= Lp + 1; ++l) keep[l] *= s;
    for (int l = 0; l <= Lp; ++l) {
        iv[l] = keep[l];
        dv[l] = keep[l + 1] + (double)l / x * keep[l];
    }
}

// One block per knot; threads stride over quadrature nodes; deterministic
// tree reduction in shared memory.
__global__ void k_radial_table(int N, int L, int G, double h, double sigma, int nq, const double *__restrict__ qx,
                               const double *__restrict__ qw, const double *__restrict__ qg, double *__restrict__ tab)
{
    extern __shared__ double red[];  // [blockDim][N*(L+1)*2]
    int k = blockIdx.x;
    int NL = N * (L + 1);
    double rj = k * h, s2 = sigma * sigma;
    double acc[2 * 12 * (GAP_MAX_L + 1)];
    for (int t = 0; t < 2 * NL; ++t) acc[t] = 0.0;
    double iv[kMaxL], dv[kMaxL];
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        double r = qx[q];
        double x = r * rj / s2;
        double gs = exp(-(r - rj) * (r - rj) / (2.0 * s2));
        bessel_scaled_all(L, x, iv, dv);
        for (int n = 0; n < N; ++n) {
            double wg = 4.0 * 3.14159265358979323846 * qw[q] * r * r * qg[q * N + n] * gs;
            for (int l = 0; l <= L; ++l) {
                acc[2 * (n * (L + 1) + l)] += wg * iv[l];
                acc[2 * (n * (L + 1) + l) + 1] += wg * (-(rj / s2) * iv[l] + (r / s2) * dv[l]);
            }
        }
    }
    for (int t = 0; t < 2 * NL; ++t) red[threadIdx.x * 2 * NL + t] = acc[t];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int t = 0; t < 2 * NL; ++t) red[threadIdx.x * 2 * NL + t] += red[(threadIdx.x + s) * 2 * NL + t];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int t = 0; t < 2 * NL; ++t) tab[(size_t)k * 2 * NL + t] = red[t];
}

// Per-interval cubic coefficients from knot values/derivatives (FP64), and
// their FP32 rounding.  knots: [G+1][NL][2]; coef: [G][NL][4].
__global__ void k_knots_to_coef(const double *__restrict__ knots, int G, int NL, double h, double *__restrict__ c64,
                                float *__restrict__ c32)
{
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)G * NL) return;
    size_t k = idx / NL, q = idx % NL;
    double f0 = knots[(k * NL + q) * 2], d0 = h * knots[(k * NL + q) * 2 + 1];
    double f1 = knots[((k + 1) * NL + q) * 2], d1 = h * knots[((k + 1) * NL + q) * 2 + 1];
    double a[4] = {f0, d0, 3.0 * (f1 - f0) - 2.0 * d0 - d1, 2.0 * (f0 - f1) + d0 + d1};
    for (int t = 0; t < 4; ++t) {
        c64[idx * 4 + t] = a[t];
        c32[idx * 4 + t] = (float)a[t];
    }
}

}  // namespace

// Clenshaw-Curtis nodes and weights on [0, rc] (n even, n+1 nodes).
static void clenshaw_curtis(int n, double rc, std::vector<double> &x, std::vector<double> &w)
{
    const double pi = 3.14159265358979323846;
    x.resize(n + 1);
    w.resize(n + 1);
    for (int j = 0; j <= n; ++j) {
        double th = j * pi / n;
        double s = 0.0;
        for (int k = 1; k <= n / 2; ++k) {
            double b = (2 * k == n) ? 1.0 : 2.0;
            s += b / (4.0 * k * k - 1.0) * std::cos(2.0 * k * th);
        }
        double c = (j == 0 || j == n) ? 1.0 : 2.0;
        w[j] = c / n * (1.0 - s) * 0.5 * rc;
        x[j] = 0.5 * rc * (1.0 - std::cos(th));
    }
}

// Jacobi P_k^(a,b)(t) for k = 0..K by the three-term recurrence.
static void jacobi_recurrence(int K, double a, double b, double t, double *P)
{
    P[0] = 1.0;
    if (K >= 1) P[1] = (a + 1.0) + (a + b + 2.0) * (t - 1.0) / 2.0;
    for (int n = 2; n <= K; ++n) {
        double c = 2.0 * n + a + b;
        double A = 2.0 * n * (n + a + b) * (c - 2.0);
        double B = (c - 1.0) * (c * (c - 2.0) * t + a * a - b * b);
        double C = 2.0 * (n + a - 1.0) * (n + b - 1.0) * c;
        P[n] = (B * P[n - 1] - C * P[n - 2]) / A;
    }
}

void gap_radial_basis_host(int N, double rc, double r, double *g_unnormalised)
{
    double P[32];
    double u = 1.0 - r / rc;
    jacobi_recurrence(N - 1, 2.0, 6.0, 2.0 * u - 1.0, P);
    for (int n = 0; n < N; ++n) g_unnormalised[n] = (r < rc) ? u * u * u * P[n] : 0.0;
}

gap_status gap_radial_table(const SoapGeom &g, double **tab64, double **coef64, float **coef32)
{
    const int nq = 512;
    std::vector<double> x, w;
    clenshaw_curtis(nq, g.rc, x, w);
    int N = g.N, L = g.L;
    std::vector<double> gq((size_t)(nq + 1) * N), norm(N, 0.0);
    for (int q = 0; q <= nq; ++q) gap_radial_basis_host(N, g.rc, x[q], &gq[(size_t)q * N]);
    for (int q = 0; q <= nq; ++q)
        for (int n = 0; n < N; ++n) norm[n] += w[q] * x[q] * x[q] * gq[(size_t)q * N + n] * gq[(size_t)q * N + n];
    for (int q = 0; q <= nq; ++q)
        for (int n = 0; n < N; ++n) gq[(size_t)q * N + n] /= std::sqrt(norm[n]);
    double *dx = nullptr, *dw = nullptr, *dg = nullptr;
    size_t nt = (size_t)(g.G + 1) * N * (L + 1) * 2;
    GAP_TRY_CUDA(cudaMalloc(&dx, sizeof(double) * (nq + 1)));
    GAP_TRY_CUDA(cudaMalloc(&dw, sizeof(double) * (nq + 1)));
    GAP_TRY_CUDA(cudaMalloc(&dg, sizeof(double) * (nq + 1) * N));
    size_t nc = (size_t)g.G * N * (L + 1) * 4;
    GAP_TRY_CUDA(cudaMalloc(tab64, sizeof(double) * nt));
    GAP_TRY_CUDA(cudaMalloc(coef64, sizeof(double) * nc));
    GAP_TRY_CUDA(cudaMalloc(coef32, sizeof(float) * nc));
    GAP_TRY_CUDA(cudaMemcpy(dx, x.data(), sizeof(double) * (nq + 1), cudaMemcpyHostToDevice));
    GAP_TRY_CUDA(cudaMemcpy(dw, w.data(), sizeof(double) * (nq + 1), cudaMemcpyHostToDevice));
    GAP_TRY_CUDA(cudaMemcpy(dg, gq.data(), sizeof(double) * (nq + 1) * N, cudaMemcpyHostToDevice));
    const int T = 64;
    size_t shm = sizeof(double) * T * 2 * N * (L + 1);
    if (shm > 48 * 1024) GAP_TRY_CUDA(cudaFuncSetAttribute(k_radial_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)shm));
    gap_count_launch();
    k_radial_table<<<g.G + 1, T, shm>>>(N, L, g.G, g.h, g.sigma, nq + 1, dx, dw, dg, *tab64);
    GAP_TRY_CUDA(cudaGetLastError());
    gap_count_launch();
    k_knots_to_coef<<<(unsigned)(((size_t)g.G * N * (L + 1) + 255) / 256), 256>>>(*tab64, g.G, N * (L + 1), g.h,
                                                                                  *coef64, *coef32);
    GAP_TRY_CUDA(cudaGetLastError());
    GAP_TRY_CUDA(cudaDeviceSynchronize());
    cudaFree(dx);
    cudaFree(dw);
    cudaFree(dg);
    return GAP_OK;
}
