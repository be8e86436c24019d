// Regularised least-squares fit of the sparse GP coefficients (Sec. 2,
// Eqs. 4-9), in FP64 on the GPU:
//   K_MM = delta^2 (X X^T)^zeta per GP (block diagonal over GPs) + jitter I
//   K_MM = U^T U (Cholesky),  A = [S^-1/2 K_NM ; U],  b = [S^-1/2 y ; 0]
//   A = Q R,                   alpha = R^-1 Q^T b
// S = diag(sigma^2) is the per-row regularisation of Eq. 4.  Two ways to the
// QR factorisation of the tall A (rows C + 3N + M, M columns):
//   gap_solve_dev     Householder (cuSOLVER geqrf/ormqr), FP64 CUDA cores;
//   gap_solve_tc_dev  shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa,
//                     Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020): the
//                     Gram matrix of the data rows formed once as an exact
//                     integer on the tensor cores (crt_gemm.cu), the Gram
//                     matrices of the later passes as exact congruences of
//                     it; M x M Cholesky factors and inverses by a recursive
//                     factorisation (modular products, FP64 blocks of <= 64).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "crt_gemm.h"
#include "gap_internal.h"
#include "solve.h"

#ifndef GAP_CHOL_BLOCK
#define GAP_CHOL_BLOCK 64
#endif

namespace {

// Kmm[p][q] (column-major, ld M) = delta^2 (x_p . x_q)^zeta within a GP block, 0 across blocks.
__global__ void k_kmm(const double *__restrict__ X, int D, const int *__restrict__ block_of, int M, double d2, int zeta,
                      double jitter, double *__restrict__ Kmm)
{
    __shared__ double As[16][65], Bs[16][65];
    int p0 = blockIdx.y * 64, q0 = blockIdx.x * 64;
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < D; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int kk = e % 16, rr = e / 16;
            As[kk][rr] = (p0 + rr < M && k0 + kk < D) ? X[(size_t)(p0 + rr) * D + k0 + kk] : 0.0;
            Bs[kk][rr] = (q0 + rr < M && k0 + kk < D) ? X[(size_t)(q0 + rr) * D + k0 + kk] : 0.0;
        }
        __syncthreads();
        for (int kk = 0; kk < 16; ++kk)
            for (int u = 0; u < 4; ++u)
                for (int v = 0; v < 4; ++v) acc[u][v] += As[kk][ty * 4 + u] * Bs[kk][tx * 4 + v];
        __syncthreads();
    }
    for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) {
            int p = p0 + ty * 4 + u, q = q0 + tx * 4 + v;
            if (p >= M || q >= M) continue;
            double val = 0.0;
            if (block_of[p] == block_of[q]) {
                double s = acc[u][v], z = 1.0;
                for (int t = 0; t < zeta; ++t) z *= s;
                val = d2 * z;
            }
            if (p == q) val += jitter;
            Kmm[(size_t)q * M + p] = val;
        }
}

// Column-major A (ld = R + M): rows 0..R-1 = K_NM / sigma, rows R.. = U (upper part of Kmm after potrf).
__global__ void k_stack(const double *__restrict__ K, const double *__restrict__ y, const double *__restrict__ sigma,
                        long R, int M, const double *__restrict__ U, double *__restrict__ A, double *__restrict__ b)
{
    long lda = R + M;
    long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long total = lda * M;
    if (idx < lda) b[idx] = idx < R ? y[idx] / sigma[idx] : 0.0;
    if (idx >= total) return;
    long col = idx / lda, row = idx - col * lda;
    double v;
    if (row < R) v = K[row * M + col] / sigma[row];
    else {
        long k = row - R;
        v = (k <= col) ? U[col * M + k] : 0.0;
    }
    A[idx] = v;
}

// Back substitution R c = z for the upper-triangular M x M leading block of A (column-major).
__global__ void k_backsub(const double *__restrict__ A, long lda, int M, const double *__restrict__ z,
                          double *__restrict__ c)
{
    // one block; columns processed right to left, threads update the remaining entries
    extern __shared__ double cs[];
    for (int k = threadIdx.x; k < M; k += blockDim.x) cs[k] = z[k];
    __syncthreads();
    for (int k = M - 1; k >= 0; --k) {
        if (threadIdx.x == 0) cs[k] /= A[(size_t)k * lda + k];
        __syncthreads();
        double ck = cs[k];
        for (int r = threadIdx.x; r < k; r += blockDim.x) cs[r] -= A[(size_t)k * lda + r] * ck;
        __syncthreads();
    }
    for (int k = threadIdx.x; k < M; k += blockDim.x) c[k] = cs[k];
}

const char *cusolver_name(cusolverStatus_t s)
{
    switch (s) {
    case CUSOLVER_STATUS_SUCCESS: return "success";
    case CUSOLVER_STATUS_NOT_INITIALIZED: return "not initialized";
    case CUSOLVER_STATUS_ALLOC_FAILED: return "alloc failed";
    case CUSOLVER_STATUS_INVALID_VALUE: return "invalid value";
    case CUSOLVER_STATUS_EXECUTION_FAILED: return "execution failed";
    case CUSOLVER_STATUS_INTERNAL_ERROR: return "internal error";
    default: return "error";
    }
}

}  // namespace

gap_status SolveWork::ensure(int slot, size_t bytes)
{
    if (slot < 0 || slot >= kSlots) {
        gap_set_error("solve workspace slot out of range");
        return GAP_EINVAL;
    }
    if (bytes == 0) bytes = 16;
    if (bytes <= cap[slot]) return GAP_OK;
    if (buf[slot]) cudaFree(buf[slot]);
    buf[slot] = nullptr;
    cap[slot] = 0;
    cudaError_t e = gap_dev_malloc(&buf[slot], bytes);
    if (e != cudaSuccess) {
        buf[slot] = nullptr;
        cudaGetLastError();
        gap_set_error("cudaMalloc of " + std::to_string(bytes) + " bytes for the solve failed");
        return GAP_ENOMEM;
    }
    cap[slot] = bytes;
    return GAP_OK;
}

gap_status SolveWork::handles(cudaStream_t st)
{
    if (!solver && cusolverDnCreate(&solver) != CUSOLVER_STATUS_SUCCESS) {
        solver = nullptr;
        gap_set_error("cusolverDnCreate failed");
        return GAP_ECUDA;
    }
    if (!blas && cublasCreate(&blas) != CUBLAS_STATUS_SUCCESS) {
        blas = nullptr;
        gap_set_error("cublasCreate failed");
        return GAP_ECUDA;
    }
    if (cusolverDnSetStream(solver, st) != CUSOLVER_STATUS_SUCCESS || cublasSetStream(blas, st) != CUBLAS_STATUS_SUCCESS) {
        gap_set_error("setting the solver stream failed");
        return GAP_ECUDA;
    }
    return GAP_OK;
}

void SolveWork::release()
{
    for (int k = 0; k < kSlots; ++k) {
        if (buf[k]) cudaFree(buf[k]);
        buf[k] = nullptr;
        cap[k] = 0;
    }
    if (solver) cusolverDnDestroy(solver);
    if (blas) cublasDestroy(blas);
    solver = nullptr;
    blas = nullptr;
    for (auto &g : chol_graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    chol_graphs.clear();
    chol_seen.clear();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
}

namespace {

enum {
    W_KMM = 0, W_A, W_B, W_TAU, W_WORK, W_INFO, W_RSIG, W_RESC, W_EC, W_OUT, W_G,
    W_R1, W_R2, W_R3, W_C, W_ERR, W_HWORK, W_CRA, W_CRB, W_CEA, W_CEB, W_COUT, W_CS, W_CT, W_RF, W_CEQ, W_KW,
    W_G1RES, W_ARES, W_HRES, W_GOUT, W_F, W_Z, W_TRMV, W_COUNT
};
static_assert(W_COUNT <= SolveWork::kSlots, "SolveWork has a slot per buffer");

gap_status solver_status(cusolverStatus_t s, const char *what)
{
    if (s == CUSOLVER_STATUS_SUCCESS) return GAP_OK;
    gap_set_error(std::string(what) + " failed: " + cusolver_name(s));
    return GAP_ECUDA;
}

gap_status blas_status(cublasStatus_t s, const char *what)
{
    if (s == CUBLAS_STATUS_SUCCESS) return GAP_OK;
    gap_set_error(std::string(what) + " failed (cuBLAS status " + std::to_string((int)s) + ")");
    return GAP_ECUDA;
}

// Kmm[p][q] = delta^2 S[p][q]^zeta within a GP block (0 across), + jitter on
// the diagonal, from the Gram matrix S = X X^T already in Kmm.
__global__ void k_kmm_power(double *__restrict__ Kmm, int M, const int *__restrict__ block_of, double d2, int zeta,
                            double jitter)
{
    long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)M * M) return;
    const int q = (int)(idx / M), p = (int)(idx - (long)q * M);
    double v = 0.0;
    if (block_of[p] == block_of[q]) {
        const double s = Kmm[idx];
        double z = 1.0;
        for (int t = 0; t < zeta; ++t) z *= s;
        v = d2 * z;
    }
    if (p == q) v += jitter;
    Kmm[idx] = v;
}

// K_MM + jitter (block-diagonal over GPs) into w[W_KMM], then its upper
// Cholesky factor U in place; GAP_ENOTPD if there is none.  tc: the sparse
// points' Gram matrix X X^T by the modular FP64 tensor-core product (else a
// CUDA-core FP64 kernel).
gap_status kmm_factor(const SolveInputs &in, SolveWork &w, cudaStream_t st, bool tc, bool factor = true)
{
    const int M = in.M;
    GAP_TRY(w.ensure(W_KMM, sizeof(double) * (size_t)M * M));
    GAP_TRY(w.ensure(W_INFO, sizeof(int)));
    if (tc && gap_crt_moduli(in.D) > 0) {
        const int T = gap_crt_moduli(in.D);
        const long kp = gap_crt_kpad(in.D), ldo = ((long)M + 255) / 256 * 256;
        GAP_TRY(w.ensure(W_CRA, 2 * (size_t)T * M * kp));
        GAP_TRY(w.ensure(W_CEA, sizeof(int) * (size_t)M));
        GAP_TRY(w.ensure(W_COUT, (size_t)T * M * ldo));
        if (!w.buf[W_ERR]) {
            GAP_TRY(w.ensure(W_ERR, sizeof(int) * 4));
            GAP_TRY_CUDA(cudaMemsetAsync(w.buf[W_ERR], 0, sizeof(int) * 4, st));
        }
        CrtVMat Xv{in.X, in.D, nullptr, M, nullptr, 0, M, in.D};
        __nv_bfloat16 *ra = w.at<__nv_bfloat16>(W_CRA);
        int *ea = w.at<int>(W_CEA);
        GAP_TRY(gap_crt_prep_rows(Xv, T, kp, ra, ea, st));
        GAP_TRY(gap_crt_gemm(ra, M, ra, M, kp, T, true, false, w.at<unsigned char>(W_COUT), ldo, w.at<int>(W_ERR),
                             st));
        GAP_TRY(gap_crt_combine(w.at<unsigned char>(W_COUT), ldo, M, M, T, ea, ea, true, w.at<double>(W_KMM), M, st));
        gap_count_launch();
        k_kmm_power<<<(unsigned)(((long)M * M + 255) / 256), 256, 0, st>>>(w.at<double>(W_KMM), M, in.block_of,
                                                                           in.delta * in.delta, in.zeta, in.jitter);
        GAP_TRY_CUDA(cudaGetLastError());
    } else {
        dim3 grid((M + 63) / 64, (M + 63) / 64);
        gap_count_launch();
        k_kmm<<<grid, 256, 0, st>>>(in.X, in.D, in.block_of, M, in.delta * in.delta, in.zeta, in.jitter,
                                    w.at<double>(W_KMM));
        GAP_TRY_CUDA(cudaGetLastError());
    }
    if (!factor) return GAP_OK;
    int lwork = 0, hinfo = 0;
    GAP_TRY(solver_status(cusolverDnDpotrf_bufferSize(w.solver, CUBLAS_FILL_MODE_UPPER, M, w.at<double>(W_KMM), M,
                                                      &lwork), "potrf_bufferSize"));
    GAP_TRY(w.ensure(W_WORK, sizeof(double) * (size_t)(lwork > 0 ? lwork : 1)));
    GAP_TRY(solver_status(cusolverDnDpotrf(w.solver, CUBLAS_FILL_MODE_UPPER, M, w.at<double>(W_KMM), M,
                                           w.at<double>(W_WORK), lwork, w.at<int>(W_INFO)), "potrf(K_MM)"));
    GAP_TRY_CUDA(cudaMemcpyAsync(&hinfo, w.buf[W_INFO], sizeof(int), cudaMemcpyDeviceToHost, st));
    GAP_TRY_CUDA(cudaStreamSynchronize(st));
    if (hinfo != 0) {
        gap_set_error("K_MM + jitter is not positive definite (potrf info " + std::to_string(hinfo) + ")");
        return GAP_ENOTPD;
    }
    return GAP_OK;
}

}  // namespace

gap_status gap_solve_dev(const SolveInputs &in, double *alpha_out, SolveWork &w, cudaStream_t st)
{
    const long R = in.rows;
    const int M = in.M;
    const long lda = R + M;
    if (M <= 0) return GAP_OK;
    if (lda > 2147483647L || lda * (long)M > (1L << 40)) {
        gap_set_error("least-squares system too large");
        return GAP_EINVAL;
    }
    GAP_TRY(w.handles(st));
    gap_prof_begin(ST_SOLVE_KMM, st);
    GAP_TRY(kmm_factor(in, w, st, false));
    gap_prof_end(ST_SOLVE_KMM, st);
    GAP_TRY(w.ensure(W_A, sizeof(double) * (size_t)lda * M));
    GAP_TRY(w.ensure(W_B, sizeof(double) * (size_t)lda));
    GAP_TRY(w.ensure(W_TAU, sizeof(double) * (size_t)M));
    double *A = w.at<double>(W_A), *b = w.at<double>(W_B), *tau = w.at<double>(W_TAU);
    int lw2 = 0, lw3 = 0;
    GAP_TRY(solver_status(cusolverDnDgeqrf_bufferSize(w.solver, (int)lda, M, A, (int)lda, &lw2), "geqrf_bufferSize"));
    GAP_TRY(solver_status(cusolverDnDormqr_bufferSize(w.solver, CUBLAS_SIDE_LEFT, CUBLAS_OP_T, (int)lda, 1, M, A,
                                                      (int)lda, tau, b, (int)lda, &lw3), "ormqr_bufferSize"));
    const int lwork = lw2 > lw3 ? lw2 : lw3;
    GAP_TRY(w.ensure(W_WORK, sizeof(double) * (size_t)(lwork > 0 ? lwork : 1)));
    gap_prof_begin(ST_SOLVE_QR, st);
    {
        long total = lda * M;
        gap_count_launch();
        k_stack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(in.K, in.y, in.sigma, R, M, w.at<double>(W_KMM), A,
                                                                 b);
        GAP_TRY_CUDA(cudaGetLastError());
    }
    GAP_TRY(solver_status(cusolverDnDgeqrf(w.solver, (int)lda, M, A, (int)lda, tau, w.at<double>(W_WORK), lwork,
                                           w.at<int>(W_INFO)), "geqrf"));
    GAP_TRY(solver_status(cusolverDnDormqr(w.solver, CUBLAS_SIDE_LEFT, CUBLAS_OP_T, (int)lda, 1, M, A, (int)lda, tau,
                                           b, (int)lda, w.at<double>(W_WORK), lwork, w.at<int>(W_INFO)), "ormqr"));
    gap_count_launch();
    k_backsub<<<1, 1024, sizeof(double) * M, st>>>(A, lda, M, b, alpha_out);
    GAP_TRY_CUDA(cudaGetLastError());
    gap_prof_end(ST_SOLVE_QR, st);
    GAP_TRY_CUDA(cudaStreamSynchronize(st));
    return GAP_OK;
}

// ------------------------------------------------- shifted CholeskyQR3 path
namespace {

__global__ void k_recip(const double *__restrict__ s, long n, double *__restrict__ r)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) r[i] = 1.0 / s[i];
}

// G += s I with s = coef trace(G) (the shift of the first CholeskyQR pass).
__global__ void k_shift_diag(double *__restrict__ G, int n, double coef)
{
    __shared__ double part[32];
    double t = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) t += G[(size_t)k * n + k];
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        double u = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if (threadIdx.x == 0) part[0] = u;
    }
    __syncthreads();
    const double s = coef * part[0];
    for (int k = threadIdx.x; k < n; k += blockDim.x) G[(size_t)k * n + k] += s;
}

// Gershgorin bound of the spectral radius of G - I (G symmetric n x n):
// max over rows of sum_j |G_ij - delta_ij|, one warp per row, the maximum
// taken on the bits of the non-negative doubles.
__global__ void k_gershgorin(const double *__restrict__ G, int n, unsigned long long *__restrict__ rho)
{
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += fabs(G[(size_t)i * n + j] - (j == i ? 1.0 : 0.0));
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicMax(rho, (unsigned long long)__double_as_longlong(s));
}

// One Richardson step for G z = c: z1 = z0 + (c - G z0), one warp per row
// (G symmetric, so row i is the contiguous column i).
__global__ void k_richardson(const double *__restrict__ G, int n, const double *__restrict__ c,
                             const double *__restrict__ z0, double *__restrict__ z1)
{
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    const double *g = G + (size_t)i * n;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;  // four independent chains
    int j = lane;
    for (; j + 96 < n; j += 128) {
        s0 = fma(g[j], z0[j], s0);
        s1 = fma(g[j + 32], z0[j + 32], s1);
        s2 = fma(g[j + 64], z0[j + 64], s2);
        s3 = fma(g[j + 96], z0[j + 96], s3);
    }
    for (; j < n; j += 32) s0 = fma(g[j], z0[j], s0);
    double s = (s0 + s1) + (s2 + s3);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) z1[i] = z0[i] + (c[i] - s);
}

// y = U x for U upper triangular n x n, column-major (ld n), in two passes
// with a fixed summation order: part[cb][i] = sum of U_ij x_j over the 128
// columns of chunk cb (blocks with cb below the row block skipped: zero),
// then y_i = sum over cb >= row block of part[cb][i].
constexpr int kTrmvTile = 128;
__global__ void __launch_bounds__(kTrmvTile) k_trmv_part(const double *__restrict__ U, int n,
                                                         const double *__restrict__ x, double *__restrict__ part)
{
    const int cb = blockIdx.x, rb = blockIdx.y;
    if (cb < rb) return;
    __shared__ double xs[kTrmvTile];
    const int j0 = cb * kTrmvTile, j1 = min(j0 + kTrmvTile, n);
    if (j0 + (int)threadIdx.x < n) xs[threadIdx.x] = x[j0 + threadIdx.x];
    __syncthreads();
    const int i = rb * kTrmvTile + threadIdx.x;
    if (i >= n) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int j = j0;
    for (; j + 3 < j1; j += 4) {
        s0 = fma(U[i + (long)j * n], xs[j - j0], s0);
        s1 = fma(U[i + (long)(j + 1) * n], xs[j + 1 - j0], s1);
        s2 = fma(U[i + (long)(j + 2) * n], xs[j + 2 - j0], s2);
        s3 = fma(U[i + (long)(j + 3) * n], xs[j + 3 - j0], s3);
    }
    for (; j < j1; ++j) s0 = fma(U[i + (long)j * n], xs[j - j0], s0);
    part[(long)cb * n + i] = (s0 + s1) + (s2 + s3);
}

__global__ void k_trmv_sum(const double *__restrict__ part, int n, int nchunk, double *__restrict__ y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int cb = i / kTrmvTile; cb < nchunk; ++cb) s += part[(long)cb * n + i];
    y[i] = s;
}

// 1 / sqrt(x) for x > 0 in FP64 without FP64 division or square root (each
// a long sequence on the narrow FP64 pipe): an FP32 estimate (x scaled by an
// even power of two into FP32 range), then Newton's iteration for x^-1/2,
// y <- y (3 - x y^2) / 2, twice (quadratic convergence: ~22 -> ~44 -> 53+
// bits; the last step is written as y + y (1 - x y^2) / 2 to keep its
// rounding below one ulp).
__device__ __forceinline__ double rsqrt_newton(double x)
{
    int e;
    const double f = frexp(x, &e);          // x = f 2^e, f in [0.5, 1)
    const int h = e >> 1;                   // floor(e / 2)
    const double xs = ldexp(f, e - 2 * h);  // x 2^-2h in [0.5, 2)
    double y = (double)rsqrtf((float)xs);
    y = y * (1.5 - 0.5 * xs * y * y);
    const double t = fma(-xs * y, y, 1.0);
    y = fma(0.5 * y, t, y);
    return ldexp(y, -h);
}

// 1 / x for x > 0 in FP64 without FP64 division, in few dependent FP64
// operations (it sits on the critical path of every elimination step):
// x = f 2^e with f in [0.5, 1); an FP32 estimate of 1 / f (f's leading 23
// bits to FP32 and the estimate back to FP64 by moving bit fields, the
// hardware's approximate reciprocal in between), then one third-order Newton
// step y <- y + y (d + d^2), d = 1 - f y, which takes the ~22-bit estimate
// to ~66 bits before the final rounding.
__device__ __forceinline__ double recip_newton(double x)
{
    int e;
    const double f = frexp(x, &e);  // x = f 2^e, f in [0.5, 1)
    const unsigned long long fb = (unsigned long long)__double_as_longlong(f);
    const float fs = __uint_as_float(0x3F000000u | (unsigned)((fb >> 29) & 0x7FFFFFu));  // f, truncated
    float rs;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(fs));  // in (1, 2]
    // FP32 -> FP64 of a positive normal number: exponent rebiased by 1023 - 127
    double y = __longlong_as_double((long long)(((unsigned long long)__float_as_uint(rs) + (896ull << 23)) << 29));
    const double d = fma(-f, y, 1.0);
    y = fma(y, fma(d, d, d), y);
    return ldexp(y, -e);
}

// The FP64 reciprocal and reciprocal square root of the factorisation
// blocks beside CUDA's own 1.0 / x and rsqrt(x), element by element (test hook).
__global__ void k_recip_check(int n, const double *__restrict__ x, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    out[4 * (size_t)i + 0] = recip_newton(v);
    out[4 * (size_t)i + 1] = rsqrt_newton(v);
    out[4 * (size_t)i + 2] = 1.0 / v;
    out[4 * (size_t)i + 3] = rsqrt(v);
}

// Upper Cholesky factor R (G = R^T R) and its inverse X of an m x m block
// (m <= kBlock) in one CTA of kBlock / 4 warps, FP64.  Elimination on M = [A | B]
// (A = G, upper triangle; B = I): step k subtracts (M_ki / M_kk) times row k
// from every row i > k, on the columns that stay live (A: j >= i; B: j <= k).
// Rows are left unscaled, so each step needs only the reciprocal pivot; at
// the end row k times M_kk^-1/2 gives row k of R (A part) and of R^-T (B
// part, the product of the elimination matrices), so X = B^T.  Each row's
// live columns are packed into 32-wide chunks (every FP64 instruction works
// on whole warps), warp w takes the rows i = k + 1 + w (mod warps), and one
// more warp forms the next pivot M_{k+1,k+1} and its reciprocal meanwhile (the
// same expression the row update would use, so that long FP64 chain runs
// beside the row updates rather than after one of them): one barrier per
// step.  G column-major (ld ldg); R and X written column-major (ld ld) with
// zero strict lower triangles.  A non-positive pivot sets *flag (the factor
// is meaningless).
constexpr int kBlock = GAP_CHOL_BLOCK;  // largest block factorised by one kernel
constexpr int kBlockWarps = kBlock / 4;  // row warps of that kernel (plus one pivot warp)
constexpr int kSplit = 32;               // granularity of the recursive split
constexpr int kBlockLd = 2 * kBlock + 1;
constexpr size_t kBlockSmem = sizeof(double) * (kBlock * kBlockLd + 2 * kBlock);

__global__ void __launch_bounds__(32 * (kBlockWarps + 1)) k_chol_inv_block(const double *__restrict__ G, long ldg, int m,
                                                                     double *__restrict__ R, double *__restrict__ X,
                                                                     long ld, int *__restrict__ flag)
{
    extern __shared__ double sm_block[];
    double(*M)[kBlockLd] = reinterpret_cast<double(*)[kBlockLd]>(sm_block);
    double *inv_s = sm_block + kBlock * kBlockLd;  // [kBlock] reciprocal pivots
    double *ri_s = inv_s + kBlock;                 // [kBlock] pivot^-1/2
    __shared__ int bad;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int idx = t; idx < m * m; idx += blockDim.x) {
        const int i = idx % m, j = idx / m;
        M[i][j] = G[i + (long)j * ldg];
        M[i][kBlock + j] = i == j ? 1.0 : 0.0;
    }
    if (t == 0) bad = 0;
    __syncthreads();
    if (t == 0) {
        const double piv = M[0][0];
        if (!(piv > 0.0)) bad = 1;
        inv_s[0] = piv > 0.0 ? recip_newton(piv) : 0.0;
    }
    __syncthreads();
    for (int k = 0; k + 1 < m; ++k) {
        const double inv = inv_s[k];
        if (w < kBlockWarps) {
            // this warp's rows and their multipliers M_ki / M_kk (lane q: row q)
            const int nr = w + k + 1 < m ? (m - (k + 1 + w) + kBlockWarps - 1) / kBlockWarps : 0;
            const int iq = k + 1 + w + kBlockWarps * lane;
            const double fl = lane < nr ? M[k][iq] * inv : 0.0;
            for (int q = 0; q < nr; ++q) {
                const int i = k + 1 + w + kBlockWarps * q;
                const double f = __shfl_sync(0xffffffffu, fl, q);
                const int na = m - i, s_i = na + k + 1;  // live A columns [i, m), B columns [0, k]
                const int cskip = i == k + 1 ? 0 : -1;  // the next pivot: the pivot warp's
                for (int c0 = 0; c0 < s_i; c0 += 32) {
                    const int c = c0 + lane;
                    if (c < s_i && c != cskip) {
                        const int col = c < na ? i + c : kBlock + (c - na);
                        M[i][col] = fma(-f, M[k][col], M[i][col]);
                    }
                }
            }
        } else if (lane == 0) {
            // the next pivot, as the row update of row k + 1 would form it
            const double f = M[k][k + 1] * inv;
            const double v = fma(-f, M[k][k + 1], M[k + 1][k + 1]);
            M[k + 1][k + 1] = v;
            if (!(v > 0.0)) bad = 1;
            inv_s[k + 1] = v > 0.0 ? recip_newton(v) : 0.0;
        }
        __syncthreads();
    }
    if (t < m) ri_s[t] = M[t][t] > 0.0 ? rsqrt_newton(M[t][t]) : 0.0;
    __syncthreads();
    if (t == 0 && bad) atomicOr(flag, 1);
    for (int idx = t; idx < m * m; idx += blockDim.x) {
        const int i = idx % m, jj = idx / m;
        R[i + (long)jj * ld] = i <= jj ? M[i][jj] * ri_s[i] : 0.0;
        X[i + (long)jj * ld] = i <= jj ? M[jj][kBlock + i] * ri_s[jj] : 0.0;
    }
}

// e_i = round(log2 sqrt(G_ii)) (0 for a non-positive diagonal), G^_ij = 2^-(e_i + e_j) G_ij.
__device__ __forceinline__ int half_exponent(double g)
{
    if (!(g > 0.0)) return 0;
    int e;
    frexp(g, &e);  // g = f 2^e, f in [0.5, 1)
    return (e - 1) >> 1;
}

// x 2^s: a multiplication by the power of two where that is a normal number
// (exact, and rounded like ldexp on underflow), else ldexp.
__device__ __forceinline__ double scale2(double x, int s)
{
    if (s >= -1022 && s <= 1023) return x * __longlong_as_double((long long)(s + 1023) << 52);
    return ldexp(x, s);
}

__global__ void k_diag_exp(const double *__restrict__ G, int n, int *__restrict__ dexp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dexp[i] = half_exponent(G[i + (long)i * n]);
}

__global__ void k_equilibrate(const double *__restrict__ G, int n, double *__restrict__ Gh,
                              const int *__restrict__ dexp)
{
    long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)n * n) return;
    const int j = (int)(idx / n), i = (int)(idx - (long)j * n);
    Gh[idx] = scale2(G[idx], -(dexp[i] + dexp[j]));
}

// R = R^ D (column j times 2^-e_j), X = D^-1 X^ (row i times 2^e_i).
__global__ void k_unscale(double *__restrict__ R, double *__restrict__ X, int n, const int *__restrict__ dexp)
{
    long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)n * n) return;
    const int j = (int)(idx / n), i = (int)(idx - (long)j * n);
    R[idx] = scale2(R[idx], dexp[j]);
    X[idx] = scale2(X[idx], -dexp[i]);
}

// Recursive Cholesky factor and inverse of an SPD n x n matrix: for
// G = [A B; B^T C] with R = [R11 R12; 0 R22] and X = R^-1 = [X11 X12; 0 X22],
//   R11, X11 from A;  R12 = X11^T B;  S = C - R12^T R12;  R22, X22 from S;
//   X12 = -X11 (R12 X22).
// The off-diagonal products per level are FP64-accurate modular GEMMs on the
// tensor cores (small ones FP64 GEMMs); blocks of 64 or fewer are factorised
// and inverted by one kernel (k_chol_inv_block).
// Products with rows x cols x K at most this go to one FP64 GEMM (GB300's
// FP64 units make larger ones slower there than a modular product); the
// crossover is measured on the device (gap_tune_small_product) and this is its
// fallback.
constexpr long kSmallProduct = 1L << 21;

__device__ __forceinline__ double op_at(const CrtVMat &V, bool cols_of, int r, int k)
{
    return cols_of ? V.Y[(long)k * V.ldy + r] : V.Y[(long)r * V.ldy + k];
}

// C[r * ldc + c] = alpha sum_k Aop[r][k] Bop[c][k] (+ Cin[r * ldcin + c]) in
// FP64 with 8 x 8 output tiles and the K range split four ways inside the CTA
// (64 threads per quarter, one output each; the four partials summed in a
// fixed order), so that a small product spreads over as many SMs as it has
// tiles and uses all four FP64 pipes of each (each SM's FP64 rate is low).
// C may alias Cin element for element.
constexpr int kSmallTile = 8;
__global__ void __launch_bounds__(256) k_gemm_f64_small(CrtVMat A, int a_cols, CrtVMat B, int b_cols, int rowsA,
                                                        int rowsB, int K, double alpha, const double *Cin, long ldcin,
                                                        double *C, long ldc)
{
    __shared__ double As[4][kSmallTile][33], Bs[4][kSmallTile][33];
    __shared__ double part[4][kSmallTile * kSmallTile];
    const int kg = threadIdx.x >> 6, tid = threadIdx.x & 63;
    const int tr = tid >> 3, tc = tid & 7;
    const int r0 = blockIdx.y * kSmallTile, c0 = blockIdx.x * kSmallTile;
    double acc = 0.0;
    // quarter kg takes the 32-wide K blocks kg, kg + 4, ... (the same trip
    // count for every thread)
    for (int k0 = 0; k0 < K; k0 += 4 * 32) {
        const int kb = k0 + 32 * kg;
        for (int e = tid; e < kSmallTile * 32; e += 64) {
            const int rr = e >> 5, kk = e & 31, gk = kb + kk;
            As[kg][rr][kk] = (r0 + rr < rowsA && gk < K) ? op_at(A, a_cols, r0 + rr, gk) : 0.0;
            Bs[kg][rr][kk] = (c0 + rr < rowsB && gk < K) ? op_at(B, b_cols, c0 + rr, gk) : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) acc = fma(As[kg][tr][kk], Bs[kg][tc][kk], acc);
        __syncthreads();
    }
    part[kg][tid] = acc;
    __syncthreads();
    if (kg == 0) {
        const int r = r0 + tr, c = c0 + tc;
        if (r < rowsA && c < rowsB) {
            double v = alpha * ((part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid]));
            if (Cin) v += Cin[(long)r * ldcin + c];
            C[(long)r * ldc + c] = v;
        }
    }
}

struct CholInv {
    SolveWork &w;
    cudaStream_t st;
    int n;
    double *R, *X;   // outputs, column-major n x n
    double *sbuf;    // stack of Schur complements
    size_t sused;
    double *tbuf;    // T = R12 X22
    bool refine = true;  // one refinement step for each R12 (FP64 backward accuracy)

    // C (rows x cols, C[r * ldc + c]) = alpha A' B'^T (+ Cin); an operand
    // given with `cols_of` = true has the columns of its view as rows.
    gap_status product(const CrtVMat &Av, bool a_cols, const CrtVMat &Bv, bool b_cols, bool sym, bool b_lower,
                       double alpha, const double *Cin, long ldcin, double *C, long ldc)
    {
        const long rowsA = a_cols ? Av.cols : Av.rows, rowsB = b_cols ? Bv.cols : Bv.rows;
        const long K = a_cols ? Av.rows : Av.cols;
        if (rowsA * rowsB * K <= (w.small_product >= 0 ? w.small_product : kSmallProduct)) {
            // small blocks: one FP64 kernel costs less than the launches of a
            // modular product
            dim3 grid((unsigned)((rowsB + kSmallTile - 1) / kSmallTile), (unsigned)((rowsA + kSmallTile - 1) / kSmallTile));
            gap_count_launch();
            k_gemm_f64_small<<<grid, 256, 0, st>>>(Av, a_cols ? 1 : 0, Bv, b_cols ? 1 : 0, (int)rowsA, (int)rowsB, (int)K,
                                                    alpha, Cin, ldcin, C, ldc);
            return gap_cuda_status(cudaGetLastError(), "k_gemm_f64_small");
        }
        const int T = gap_crt_moduli(K);
        const long kpad = gap_crt_kpad(K), ldo = (rowsB + 255) / 256 * 256;
        __nv_bfloat16 *ra = w.at<__nv_bfloat16>(W_CRA), *rb = w.at<__nv_bfloat16>(W_CRB);
        int *ea = w.at<int>(W_CEA), *eb = w.at<int>(W_CEB);
        GAP_TRY(a_cols ? gap_crt_prep_cols(Av, T, kpad, ra, ea, st) : gap_crt_prep_rows(Av, T, kpad, ra, ea, st));
        if (!sym)
            GAP_TRY(b_cols ? gap_crt_prep_cols(Bv, T, kpad, rb, eb, st) : gap_crt_prep_rows(Bv, T, kpad, rb, eb, st));
        GAP_TRY(gap_crt_gemm(ra, rowsA, sym ? ra : rb, rowsB, kpad, T, sym, b_lower, w.at<unsigned char>(W_COUT), ldo,
                             w.at<int>(W_ERR), st));
        return gap_crt_combine(w.at<unsigned char>(W_COUT), ldo, rowsA, (int)rowsB, T, ea, sym ? ea : eb, sym, C, ldc,
                               st, alpha, Cin, ldcin);
    }

    gap_status rec(const double *G, long ldg, int o, int m)
    {
        if (m <= kBlock) {
            static bool smem_set[64] = {};  // the attribute is per device
            int dev = 0;
            GAP_TRY_CUDA(cudaGetDevice(&dev));
            if (dev >= 64 || !smem_set[dev]) {
                GAP_TRY_CUDA(cudaFuncSetAttribute(k_chol_inv_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)kBlockSmem));
                if (dev < 64) smem_set[dev] = true;
            }
            gap_count_launch();
            gap_prof_begin(ST_SOLVE_BLOCK, st);
            k_chol_inv_block<<<1, 32 * (kBlockWarps + 1), kBlockSmem, st>>>(G, ldg, m, R + o + (long)o * n, X + o + (long)o * n, n,
                                                         w.at<int>(W_ERR) + 1);
            gap_prof_end(ST_SOLVE_BLOCK, st);
            return gap_cuda_status(cudaGetLastError(), "k_chol_inv_block");
        }
        const int n1 = (m / 2 + kSplit - 1) / kSplit * kSplit, n2 = m - n1;
        GAP_TRY(rec(G, ldg, o, n1));
        double *R12 = R + o + (long)(o + n1) * n;
        // R12 = R11^-T B through X11, then one step of iterative refinement
        // (Res = B - R11^T R12, R12 += X11^T Res) so that R12 solves
        // R11^T R12 = B to working accuracy, as a triangular solve would.
        // Products are formed transposed: rows j < n2, columns i < n1.
        {
            CrtVMat Bt{G + (long)n1 * ldg, ldg, nullptr, n2, nullptr, 0, n2, n1};
            CrtVMat X11t{X + o + (long)o * n, n, nullptr, n1, nullptr, 0, n1, n1};
            CrtVMat R11t{R + o + (long)o * n, n, nullptr, n1, nullptr, 0, n1, n1};
            CrtVMat R12t{R12, n, nullptr, n2, nullptr, 0, n2, n1};
            CrtVMat Rest{tbuf, n1, nullptr, n2, nullptr, 0, n2, n1};
            GAP_TRY(product(Bt, false, X11t, false, false, true, 1.0, nullptr, 0, R12, n));
            if (refine) {
                GAP_TRY(product(R12t, false, R11t, false, false, true, -1.0, G + (long)n1 * ldg, ldg, tbuf, n1));
                GAP_TRY(product(Rest, false, X11t, false, false, true, 1.0, R12, n, R12, n));
            }
        }
        // S = C - R12^T R12
        double *S = sbuf + sused;
        sused += (size_t)n2 * n2;
        {
            CrtVMat R12t{R12, n, nullptr, n2, nullptr, 0, n2, n1};
            GAP_TRY(product(R12t, false, R12t, false, true, false, -1.0, G + n1 + (long)n1 * ldg, ldg, S, n2));
        }
        GAP_TRY(rec(S, n2, o + n1, n2));
        sused -= (size_t)n2 * n2;
        // T = R12 X22 (column-major, ld n1), formed as T^T (rows j < n2, cols i < n1)
        {
            CrtVMat X22t{X + (o + n1) + (long)(o + n1) * n, n, nullptr, n2, nullptr, 0, n2, n2};
            CrtVMat R12t{R12, n, nullptr, n2, nullptr, 0, n2, n1};
            GAP_TRY(product(X22t, false, R12t, true, false, false, 1.0, nullptr, 0, tbuf, n1));
        }
        // X12 = -X11 T, formed as X12^T (rows j < n2, cols i < n1)
        {
            CrtVMat Tt{tbuf, n1, nullptr, n2, nullptr, 0, n2, n1};
            CrtVMat X11t{X + o + (long)o * n, n, nullptr, n1, nullptr, 0, n1, n1};
            GAP_TRY(product(Tt, false, X11t, true, false, false, -1.0, nullptr, 0, X + o + (long)(o + n1) * n, n));
        }
        return GAP_OK;
    }
};

}  // namespace

// Autotuner of the block-product path: times an s x s x s product with both
// the FP64 kernel and the modular tensor-core product (CUDA events, best of
// three after a warm-up) for growing s, and keeps the largest size at which
// the FP64 kernel is still faster.  Operands are whatever G holds; the
// results land in scratch.
gap_status gap_tune_small_product(SolveWork &w, int n, const double *G, cudaStream_t st)
{
    long best = 0;
    w.tune_sizes = 0;
    {
        const int T = gap_crt_moduli(n);
        const long kp = gap_crt_kpad(n), ld = ((long)n + 255) / 256 * 256;
        GAP_TRY(w.ensure(W_CRA, 2 * (size_t)T * n * kp));
        GAP_TRY(w.ensure(W_CRB, 2 * (size_t)T * n * kp));
        GAP_TRY(w.ensure(W_CEA, sizeof(int) * (size_t)n));
        GAP_TRY(w.ensure(W_CEB, sizeof(int) * (size_t)n));
        GAP_TRY(w.ensure(W_COUT, (size_t)T * n * ld));
        GAP_TRY(w.ensure(W_CT, sizeof(double) * (size_t)n * n));
        if (!w.buf[W_ERR]) {
            GAP_TRY(w.ensure(W_ERR, sizeof(int) * 4));
            GAP_TRY_CUDA(cudaMemsetAsync(w.buf[W_ERR], 0, sizeof(int) * 4, st));
        }
    }
    cudaEvent_t e0, e1;
    GAP_TRY_CUDA(cudaEventCreate(&e0));
    GAP_TRY_CUDA(cudaEventCreate(&e1));
    CholInv ci{w, st, n, nullptr, nullptr, nullptr, 0, w.at<double>(W_CT)};
    gap_status rc = GAP_OK;
    for (int sz = 32; sz <= 512 && sz <= n && rc == GAP_OK; sz *= 2) {
        const CrtVMat V{G, n, nullptr, sz, nullptr, 0, sz, sz};
        float t[2] = {1e30f, 1e30f};
        for (int path = 0; path < 2 && rc == GAP_OK; ++path) {
            w.small_product = path == 0 ? (1L << 62) : 0;  // 0: FP64 kernel, 1: modular
            for (int rep = 0; rep < 4 && rc == GAP_OK; ++rep) {
                cudaEventRecord(e0, st);
                rc = ci.product(V, false, V, true, false, false, 1.0, nullptr, 0, w.at<double>(W_CT), sz);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < t[path]) t[path] = ms;
            }
        }
        if (t[0] <= t[1]) best = (long)sz * sz * sz;
        const int idx = w.tune_sizes < 8 ? w.tune_sizes : 7;
        w.tune_ms[0][idx] = t[0];
        w.tune_ms[1][idx] = t[1];
        w.tune_sizes = idx + 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    w.small_product = rc == GAP_OK ? best : -1;
    return rc;
}


gap_status gap_chol_inv_dev(SolveWork &w, int n, const double *G, double *R, double *X, cudaStream_t st,
                            bool refine)
{
    if (n <= 0) return GAP_OK;
    GAP_TRY(w.handles(st));
    if (!w.buf[W_ERR]) {
        GAP_TRY(w.ensure(W_ERR, sizeof(int) * 4));
        GAP_TRY_CUDA(cudaMemsetAsync(w.buf[W_ERR], 0, sizeof(int) * 4, st));
    }
    const int T = gap_crt_moduli(n);
    const long kp = gap_crt_kpad(n), ld = ((long)n + 255) / 256 * 256;
    GAP_TRY(w.ensure(W_CRA, 2 * (size_t)T * n * kp));
    GAP_TRY(w.ensure(W_CRB, 2 * (size_t)T * n * kp));
    GAP_TRY(w.ensure(W_CEA, sizeof(int) * (size_t)n));
    GAP_TRY(w.ensure(W_CEB, sizeof(int) * (size_t)n));
    GAP_TRY(w.ensure(W_COUT, (size_t)T * n * ld));
    GAP_TRY(w.ensure(W_CS, sizeof(double) * (size_t)n * n));
    GAP_TRY(w.ensure(W_CT, sizeof(double) * (size_t)n * n));
    GAP_TRY(w.ensure(W_CEQ, sizeof(double) * (size_t)n * n + sizeof(int) * (size_t)n));
    double *Gh = w.at<double>(W_CEQ);
    int *dexp = reinterpret_cast<int *>(Gh + (size_t)n * n);
    if (w.small_product < 0) {
        // the crossover tuner times products on the leading blocks of the
        // equilibrated matrix (host synchronisation: before any capture)
        gap_count_launch(2);
        k_diag_exp<<<(n + 255) / 256, 256, 0, st>>>(G, n, dexp);
        k_equilibrate<<<(unsigned)(((long)n * n + 255) / 256), 256, 0, st>>>(G, n, Gh, dexp);
        GAP_TRY_CUDA(cudaGetLastError());
        GAP_TRY(gap_tune_small_product(w, n, Gh, st));
    }
    auto sequence = [&](cudaStream_t s) -> gap_status {
        GAP_TRY_CUDA(cudaMemsetAsync(w.at<int>(W_ERR) + 1, 0, sizeof(int), s));  // [0]: GEMM waits, kept
        // the recursion writes only upper triangles; the products read whole blocks
        GAP_TRY_CUDA(cudaMemsetAsync(R, 0, sizeof(double) * (size_t)n * n, s));
        GAP_TRY_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)n * n, s));
        // Equilibrate by powers of two, G^ = D G D with D_i = 2^-round(log2 sqrt(G_ii)):
        // the modular products round each operand row to 53 bits below its
        // largest entry, which is harmless only for rows of comparable scale.
        // R = R^ D, X = D^-1 X^ afterwards (exact).
        gap_count_launch();
        k_diag_exp<<<(n + 255) / 256, 256, 0, s>>>(G, n, dexp);
        GAP_TRY_CUDA(cudaGetLastError());
        gap_count_launch();
        k_equilibrate<<<(unsigned)(((long)n * n + 255) / 256), 256, 0, s>>>(G, n, Gh, dexp);
        GAP_TRY_CUDA(cudaGetLastError());
        CholInv ci{w, s, n, R, X, w.at<double>(W_CS), 0, w.at<double>(W_CT), refine};
        GAP_TRY(ci.rec(Gh, n, 0, n));
        gap_count_launch();
        k_unscale<<<(unsigned)(((long)n * n + 255) / 256), 256, 0, s>>>(R, X, n, dexp);
        GAP_TRY_CUDA(cudaGetLastError());
        return GAP_OK;
    };
    // The sequence's ~400 dependent launches are replayed from a CUDA graph
    // once a direct run with the same operands and workspace has made every
    // allocation (stage profiling, which records events inside, runs direct).
    const std::vector<const void *> key = {
        G, R, X, reinterpret_cast<const void *>((intptr_t)n), reinterpret_cast<const void *>((intptr_t)refine),
        reinterpret_cast<const void *>((intptr_t)w.small_product), w.buf[W_CRA], w.buf[W_CRB], w.buf[W_CEA],
        w.buf[W_CEB], w.buf[W_COUT], w.buf[W_CS], w.buf[W_CT], w.buf[W_CEQ], w.buf[W_ERR]};
    SolveWork::CholGraph *graph = nullptr;
    for (auto &g : w.chol_graphs)
        if (g.key == key) graph = &g;
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    GAP_TRY_CUDA(cudaStreamIsCapturing(st, &cap_status));
    if (gap_prof_enabled() || cap_status != cudaStreamCaptureStatusNone) {
        GAP_TRY(sequence(st));
    } else if (graph) {
        gap_count_launch((int)graph->kernels);
        GAP_TRY_CUDA(cudaGraphLaunch(graph->exec, st));
    } else if (std::find(w.chol_seen.begin(), w.chol_seen.end(), key) == w.chol_seen.end()) {
        GAP_TRY(sequence(st));
        if (w.chol_seen.size() >= 8) w.chol_seen.erase(w.chol_seen.begin());
        w.chol_seen.push_back(key);
    } else {
        // captured on a private stream (the caller's may be the legacy
        // default stream, which cannot be captured), replayed on st
        const long k0 = gap_launch_total();
        if (!w.cap_stream) GAP_TRY_CUDA(cudaStreamCreateWithFlags(&w.cap_stream, cudaStreamNonBlocking));
        gap_status seq = GAP_ECUDA;
        cudaGraph_t g = nullptr;
        cudaError_t end = cudaErrorUnknown;
        if (cudaStreamBeginCapture(w.cap_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
            seq = sequence(w.cap_stream);
            end = cudaStreamEndCapture(w.cap_stream, &g);
        }
        cudaGraphExec_t exec = nullptr;
        if (seq == GAP_OK && end == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
            cudaGraphDestroy(g);
            if (w.chol_graphs.size() >= 4) {  // a few operand/workspace combinations at most
                cudaGraphExecDestroy(w.chol_graphs.front().exec);
                w.chol_graphs.erase(w.chol_graphs.begin());
            }
            w.chol_graphs.push_back(SolveWork::CholGraph{key, exec, gap_launch_total() - k0});
            GAP_TRY_CUDA(cudaGraphLaunch(exec, st));
        } else {
            // not capturable here: run the sequence directly (its launches
            // counted once)
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            gap_count_launch(-(int)(gap_launch_total() - k0));
            GAP_TRY(sequence(st));
        }
    }
    int flags[2] = {0, 0};
    GAP_TRY_CUDA(cudaMemcpyAsync(flags, w.buf[W_ERR], sizeof(flags), cudaMemcpyDeviceToHost, st));
    GAP_TRY_CUDA(cudaStreamSynchronize(st));
    if (flags[0]) {
        gap_set_error("modular tensor-core GEMM wait expired (code " + std::to_string(flags[0]) + ")");
        return GAP_ETIMEOUT;
    }
    if (flags[1]) {
        gap_set_error("matrix is not positive definite");
        return GAP_ENOTPD;
    }
    return GAP_OK;
}

namespace {

struct CholQr {
    const SolveInputs &in;
    SolveWork &w;
    cudaStream_t st;
    long m;      // rows of the data block
    int n;       // columns
    int T1, T2;  // moduli of the Gram matrix (K = m) and of the congruence products
    long kpm, kp2, ldo1;

    // Pass 1: G' = V'^T V' of the fixed-point V = [S^-1/2 K | S^-1/2 y] as an
    // exact integer, plus K~ on its grid: residues modulo the T2 wide moduli
    // in W_G1RES, and the K~ block rounded to FP64 in W_G.
    gap_status exact_gram(const CrtVMat &V, const double *Kt)
    {
        __nv_bfloat16 *res = w.at<__nv_bfloat16>(W_RESC);
        int *E = w.at<int>(W_EC);
        gap_prof_begin(ST_SOLVE_PREP, st);
        GAP_TRY(gap_crt_prep_cols(V, T1, kpm, res, E, st, Kt, (long)n + 1, n));
        gap_prof_end(ST_SOLVE_PREP, st);
        gap_prof_begin(ST_SOLVE_GEMM, st);
        GAP_TRY(gap_crt_gemm(res, n + 1, res, n + 1, kpm, T1, true, false, w.at<unsigned char>(W_OUT), ldo1,
                             w.at<int>(W_ERR), st));
        gap_prof_end(ST_SOLVE_GEMM, st);
        gap_prof_begin(ST_SOLVE_CRT, st);
        GAP_TRY(gap_crt_exact_gram(w.at<unsigned char>(W_OUT), ldo1, T1, n, E, Kt, T2, kp2,
                                   w.at<__nv_bfloat16>(W_G1RES), w.at<double>(W_G), w.at<int>(W_ERR), st));
        gap_prof_end(ST_SOLVE_CRT, st);
        return GAP_OK;
    }

    // Upper Cholesky factor of W_G and its inverse `inv` (column-major, zero
    // strict lower triangle), by the recursive factorisation above.
    // refine = false: a preconditioner is enough (pass 1: the next Gram
    // matrix is formed exactly for whatever inverse factor this returns).
    gap_status factor_invert(double *inv, const char *what, bool refine = true)
    {
        gap_prof_begin(ST_SOLVE_POTRF, st);
        GAP_TRY(w.ensure(W_RF, sizeof(double) * (size_t)n * n));
        gap_status rc = gap_chol_inv_dev(w, n, w.at<double>(W_G), w.at<double>(W_RF), inv, st, refine);
        gap_prof_end(ST_SOLVE_POTRF, st);
        if (rc == GAP_ENOTPD)
            gap_set_error(std::string("CholeskyQR: Gram matrix of ") + what + " is not positive definite");
        return rc;
    }

    // Passes 2 and 3: W_G = W~^T G W~ = (V W~)^T (V W~) and W_C = W~^T V^T b,
    // exact integers rounded once, for W~ = W (upper triangular) rounded to
    // 53 bits per column (written to Wt when given).  Two products modulo each
    // wide modulus: H^T = W'^T G' and W'^T H.
    gap_status congruence(const double *Wm, double *Wt)
    {
        __nv_bfloat16 *ra = w.at<__nv_bfloat16>(W_ARES), *rh = w.at<__nv_bfloat16>(W_HRES);
        gap_prof_begin(ST_SOLVE_PREP, st);
        GAP_TRY(gap_crt_prep_congruence(Wm, n, w.at<int>(W_EC), T2, kp2, ra, w.at<int>(W_F), Wt, st));
        gap_prof_end(ST_SOLVE_PREP, st);
        gap_prof_begin(ST_SOLVE_GEMM, st);
        GAP_TRY(gap_crt_gemm(ra, n + 1, w.at<__nv_bfloat16>(W_G1RES), n + 1, kp2, T2, false, false, rh, kp2,
                             w.at<int>(W_ERR), st, true, true));
        GAP_TRY(gap_crt_gemm(ra, n + 1, rh, n + 1, kp2, T2, true, false, w.at<__nv_bfloat16>(W_GOUT), kp2,
                             w.at<int>(W_ERR), st, true, true));
        gap_prof_end(ST_SOLVE_GEMM, st);
        gap_prof_begin(ST_SOLVE_CRT, st);
        GAP_TRY(gap_crt_combine_congruence(w.at<__nv_bfloat16>(W_GOUT), kp2, n, T2, w.at<int>(W_F),
                                           w.at<double>(W_G), w.at<double>(W_C), st));
        gap_prof_end(ST_SOLVE_CRT, st);
        return GAP_OK;
    }
};

}  // namespace

gap_status gap_solve_tc_dev(const SolveInputs &in, double *alpha_out, SolveWork &w, cudaStream_t st)
{
    const long R = in.rows;
    const int n = in.M;
    if (n <= 0) return GAP_OK;
    // A = [S^-1/2 K ; U] with U^T U = K~ = K_MM + jitter I and b = [S^-1/2 y ; 0].
    // Every quantity the three passes need is a congruence of one exactly
    // known matrix: with V = [S^-1/2 K | S^-1/2 y] (the right-hand side as an
    // extra column) and G = V^T V + [K~ 0; 0 0], passes 1 and 2 factorise the
    // leading block of W^T G W for W = 1 (shifted) and W = X1; the third
    // congruence, W = X1 X2, is close to the identity and is solved by
    // iteration.  The last column of each congruence is W^T A^T b.  G is
    // formed once, exactly, from the data rows; U is never formed, and
    // neither is any m-row intermediate.
    const long m = R;
    const int n_ext = n + 1;
    const long mr = m > 0 ? m : 1;
    CholQr q{in, w, st, m, n, gap_crt_moduli(mr), gap_crt_moduli_wide(gap_crt_congruence_bits(mr, n_ext)),
             gap_crt_kpad(mr), ((long)n_ext + 255) / 256 * 256, ((long)n_ext + 255) / 256 * 256};
    if (q.T1 == 0 || q.T2 == 0 || m > 2147483647L) {
        gap_set_error("least-squares system too large for the modular tensor-core products (rows <= 2^18)");
        return GAP_EUNSUPPORTED;
    }
    GAP_TRY(w.handles(st));
    GAP_TRY(w.ensure(W_ERR, sizeof(int) * 4));
    GAP_TRY_CUDA(cudaMemsetAsync(w.buf[W_ERR], 0, sizeof(int) * 4, st));
    gap_prof_begin(ST_SOLVE_KMM, st);
    GAP_TRY(kmm_factor(in, w, st, true, false));  // K~ = K_MM + jitter I, not factorised
    gap_prof_end(ST_SOLVE_KMM, st);
    const size_t plane = (size_t)q.T2 * n_ext * q.kp2 * 2;
    GAP_TRY(w.ensure(W_RSIG, sizeof(double) * (size_t)mr));
    GAP_TRY(w.ensure(W_RESC, 2 * (size_t)q.T1 * n_ext * q.kpm));
    GAP_TRY(w.ensure(W_EC, sizeof(int) * (size_t)n_ext));
    GAP_TRY(w.ensure(W_OUT, (size_t)q.T1 * n_ext * q.ldo1));
    GAP_TRY(w.ensure(W_G1RES, plane));
    GAP_TRY(w.ensure(W_ARES, plane));
    GAP_TRY(w.ensure(W_HRES, plane));
    GAP_TRY(w.ensure(W_GOUT, plane));
    GAP_TRY(w.ensure(W_F, sizeof(int) * (size_t)n_ext));
    GAP_TRY(w.ensure(W_G, sizeof(double) * (size_t)n * n));
    GAP_TRY(w.ensure(W_R1, sizeof(double) * (size_t)n * n));
    GAP_TRY(w.ensure(W_R2, sizeof(double) * (size_t)n * n));
    GAP_TRY(w.ensure(W_R3, sizeof(double) * (size_t)n * n));
    GAP_TRY(w.ensure(W_C, sizeof(double) * (size_t)n));
    GAP_TRY(w.ensure(W_KW, sizeof(double) * (size_t)n * n));
    {
        const int T = gap_crt_moduli(n);
        const long kp = gap_crt_kpad(n), ld = ((long)n + 255) / 256 * 256;
        GAP_TRY(w.ensure(W_CRA, 2 * (size_t)T * n * kp));
        GAP_TRY(w.ensure(W_CRB, 2 * (size_t)T * n * kp));
        GAP_TRY(w.ensure(W_CEA, sizeof(int) * (size_t)n));
        GAP_TRY(w.ensure(W_CEB, sizeof(int) * (size_t)n));
        GAP_TRY(w.ensure(W_COUT, (size_t)T * n * ld));
    }
    if (R > 0) {
        gap_count_launch();
        k_recip<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(in.sigma, R, w.at<double>(W_RSIG));
        GAP_TRY_CUDA(cudaGetLastError());
    }
    double *X1 = w.at<double>(W_R1), *X2 = w.at<double>(W_R2), *X3 = w.at<double>(W_R3);
    double *W2 = w.at<double>(W_KW);
    // pass 1: shifted Cholesky QR of A
    const CrtVMat V{in.K, n, w.at<double>(W_RSIG), R, nullptr, 0, m, n_ext, in.y};
    GAP_TRY(q.exact_gram(V, w.at<double>(W_KMM)));
    const double u = std::ldexp(1.0, -53);
    gap_count_launch();
    k_shift_diag<<<1, 1024, 0, st>>>(w.at<double>(W_G), n,
                                     11.0 * ((double)(m + n) * n + (double)n * (n + 1)) * u);
    GAP_TRY_CUDA(cudaGetLastError());
    // X1 only has to precondition: G2 = X1^T G X1 is formed exactly, and an
    // inverse factor with X1^T (G + s I) X1 = I + E changes the conditioning
    // of G2 by at most (1 + |E|) / (1 - |E|); the refinement steps that
    // make a factor FP64-accurate are skipped here.
    GAP_TRY(q.factor_invert(X1, "A", false));
    // pass 2: Q1 = A X1
    GAP_TRY(q.congruence(X1, nullptr));
    GAP_TRY(q.factor_invert(X2, "A X1"));
    // pass 3: Q2 = A W2 with W2 = X1 X2 (column-major), rounded in place to
    // the matrix the congruence represents
    {
        CholInv nn{w, st, n, nullptr, nullptr, nullptr, 0, nullptr};
        const CrtVMat X2v{X2, n, nullptr, n, nullptr, 0, n, n};
        const CrtVMat X1v{X1, n, nullptr, n, nullptr, 0, n, n};
        GAP_TRY(nn.product(X2v, false, X1v, true, false, false, 1.0, nullptr, 0, W2, n));
    }
    GAP_TRY(q.congruence(W2, W2));
    // alpha = W2 G3^-1 (W2^T A^T b) with G3 = (A W2)^T (A W2).  Pass 3 of
    // CholeskyQR3 would factorise G3 = R3^T R3 to make A W2 R3^-1 orthogonal;
    // the least-squares solution needs only G3^-1 c, and G3 is known to FP64
    // accuracy and close to the identity after two passes: Richardson steps
    // z <- z + (c - G3 z) converge at the rate of the spectral radius of
    // G3 - I (bounded by Gershgorin's theorem), to the accuracy of an FP64
    // residual.  A bound of 1/2 or more factorises G3 instead.
    double *c = w.at<double>(W_C);
    // y = U x (U upper triangular, column-major); y may be x
    const int nchunk = (n + kTrmvTile - 1) / kTrmvTile;
    GAP_TRY(w.ensure(W_TRMV, sizeof(double) * ((size_t)nchunk + 1) * n));
    auto trmv = [&](const double *U, const double *x, double *y) -> gap_status {
        double *part = w.at<double>(W_TRMV), *tmp = part + (size_t)nchunk * n;
        gap_count_launch();
        k_trmv_part<<<dim3(nchunk, nchunk), kTrmvTile, 0, st>>>(U, n, x, part);
        GAP_TRY_CUDA(cudaGetLastError());
        gap_count_launch();
        k_trmv_sum<<<(n + 127) / 128, 128, 0, st>>>(part, n, nchunk, y == x ? tmp : y);
        GAP_TRY_CUDA(cudaGetLastError());
        if (y == x) GAP_TRY_CUDA(cudaMemcpyAsync(y, tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        return GAP_OK;
    };
    gap_prof_begin(ST_SOLVE_APPLY, st);
    GAP_TRY(w.ensure(W_Z, sizeof(double) * 2 * (size_t)n + 64));
    double *z0 = w.at<double>(W_Z), *z1 = z0 + n;
    unsigned long long *rho_bits = reinterpret_cast<unsigned long long *>(z0 + 2 * (size_t)n);
    GAP_TRY_CUDA(cudaMemsetAsync(rho_bits, 0, sizeof(unsigned long long), st));
    gap_count_launch();
    k_gershgorin<<<(n + 7) / 8, 256, 0, st>>>(w.at<double>(W_G), n, rho_bits);
    GAP_TRY_CUDA(cudaGetLastError());
    unsigned long long rb = 0;
    GAP_TRY_CUDA(cudaMemcpyAsync(&rb, rho_bits, sizeof(rb), cudaMemcpyDeviceToHost, st));
    GAP_TRY_CUDA(cudaStreamSynchronize(st));
    double rho;
    std::memcpy(&rho, &rb, sizeof(rho));
    gap_prof_end(ST_SOLVE_APPLY, st);
    if (rho < 0.5) {
        gap_prof_begin(ST_SOLVE_APPLY, st);
        // rho^k < 2^-60 (rho = 0 still takes one step)
        const int steps = rho > 0.0 ? (int)std::ceil(-60.0 * std::log(2.0) / std::log(rho)) : 1;
        GAP_TRY_CUDA(cudaMemcpyAsync(z0, c, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        for (int k = 0; k < steps; ++k) {
            gap_count_launch();
            k_richardson<<<(n + 7) / 8, 256, 0, st>>>(w.at<double>(W_G), n, c, z0, z1);
            GAP_TRY_CUDA(cudaGetLastError());
            std::swap(z0, z1);
        }
        GAP_TRY_CUDA(cudaMemcpyAsync(c, z0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    } else {
        GAP_TRY(q.factor_invert(X3, "A X1 X2"));
        gap_prof_begin(ST_SOLVE_APPLY, st);
        GAP_TRY(blas_status(
            cublasDtrmv(w.blas, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, n, X3, n, c, 1), "trmv"));
        GAP_TRY(trmv(X3, c, c));
    }
    GAP_TRY(trmv(W2, c, alpha_out));
    gap_prof_end(ST_SOLVE_APPLY, st);
    if (in.rinv_out) {
        // R^-1 of A^T A: A W~2 X3 has orthonormal columns for X3 the inverse
        // Cholesky factor of G3 = (A W~2)^T (A W~2), so A^T A = (W~2 X3)^-T (W~2 X3)^-1
        // and R^-1 = W~2 X3 (both factors upper triangular).
        if (rho < 0.5) GAP_TRY(q.factor_invert(X3, "A X1 X2"));
        CholInv nn{w, st, n, nullptr, nullptr, nullptr, 0, nullptr};
        const CrtVMat X3v{X3, n, nullptr, n, nullptr, 0, n, n};
        const CrtVMat W2v{W2, n, nullptr, n, nullptr, 0, n, n};
        GAP_TRY(nn.product(X3v, false, W2v, true, false, false, 1.0, nullptr, 0, in.rinv_out, n));
    }
    int err[4] = {0, 0, 0, 0};
    GAP_TRY_CUDA(cudaMemcpyAsync(err, w.buf[W_ERR], sizeof(err), cudaMemcpyDeviceToHost, st));
    GAP_TRY_CUDA(cudaStreamSynchronize(st));
    if (err[0] & 16) {
        gap_set_error("K_MM + jitter does not fit the Gram matrix's fixed-point grid (not positive semi-definite)");
        return GAP_EINVAL;
    }
    if (err[0]) {
        gap_set_error("modular tensor-core GEMM wait expired (code " + std::to_string(err[0]) + ")");
        return GAP_ETIMEOUT;
    }
    return GAP_OK;
}

extern "C" gap_status gap_test_fp64_recip(int n, const double *x, double *out)
{
    if (n < 0 || (n > 0 && (!x || !out))) {
        gap_set_error("bad arguments");
        return GAP_EINVAL;
    }
    if (n == 0) return GAP_OK;
    double *dx = nullptr, *dout = nullptr;
    gap_status st = gap_cuda_status(gap_dev_malloc((void **)&dx, sizeof(double) * (size_t)n), "cudaMalloc");
    if (st == GAP_OK) st = gap_cuda_status(gap_dev_malloc((void **)&dout, sizeof(double) * 4 * (size_t)n), "cudaMalloc");
    if (st == GAP_OK) st = gap_cuda_status(cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice), "copy");
    if (st == GAP_OK) {
        gap_count_launch();
        k_recip_check<<<(n + 255) / 256, 256>>>(n, dx, dout);
        st = gap_cuda_status(cudaGetLastError(), "k_recip_check");
    }
    if (st == GAP_OK)
        st = gap_cuda_status(cudaMemcpy(out, dout, sizeof(double) * 4 * (size_t)n, cudaMemcpyDeviceToHost), "copy");
    if (dx) cudaFree(dx);
    if (dout) cudaFree(dout);
    return st;
}

gap_status gap_f64_product(SolveWork &w, const CrtVMat &A, bool a_cols, const CrtVMat &B, bool b_cols, bool b_lower,
                           double *C, long ldc, cudaStream_t st)
{
    const long rowsA = a_cols ? A.cols : A.rows, rowsB = b_cols ? B.cols : B.rows;
    const long K = a_cols ? A.rows : A.cols;
    if (rowsA <= 0 || rowsB <= 0) return GAP_OK;
    const int T = gap_crt_moduli(K > 0 ? K : 1);
    if (T == 0) {
        gap_set_error("FP64 product: inner dimension beyond the modular products' limit");
        return GAP_EUNSUPPORTED;
    }
    const long kpad = gap_crt_kpad(K), ldo = (rowsB + 255) / 256 * 256;
    GAP_TRY(w.ensure(W_CRA, 2 * (size_t)T * rowsA * kpad));
    GAP_TRY(w.ensure(W_CRB, 2 * (size_t)T * rowsB * kpad));
    GAP_TRY(w.ensure(W_CEA, sizeof(int) * (size_t)rowsA));
    GAP_TRY(w.ensure(W_CEB, sizeof(int) * (size_t)rowsB));
    GAP_TRY(w.ensure(W_COUT, (size_t)T * rowsA * ldo));
    if (!w.buf[W_ERR]) {
        GAP_TRY(w.ensure(W_ERR, sizeof(int) * 4));
        GAP_TRY_CUDA(cudaMemsetAsync(w.buf[W_ERR], 0, sizeof(int) * 4, st));
    }
    CholInv ci{w, st, 0, nullptr, nullptr, nullptr, 0, nullptr};
    return ci.product(A, a_cols, B, b_cols, false, b_lower, 1.0, nullptr, 0, C, ldc);
}

gap_status gap_posterior_dev(const SolveInputs &in, double *kinv_out, double *rinv_out, double *alpha_scratch,
                             SolveWork &w, cudaStream_t st)
{
    const int n = in.M;
    if (n <= 0) return GAP_OK;
    SolveInputs in2 = in;
    in2.rinv_out = rinv_out;
    GAP_TRY(gap_solve_tc_dev(in2, alpha_scratch, w, st));
    // W_KMM still holds Kt = K_MM + jitter I (the solve reads it only)
    GAP_TRY(w.ensure(W_RF, sizeof(double) * (size_t)n * n));
    gap_status rc = gap_chol_inv_dev(w, n, w.at<double>(W_KMM), w.at<double>(W_RF), kinv_out, st, true);
    if (rc == GAP_ENOTPD) gap_set_error("K_MM + jitter is not positive definite");
    return rc;
}
