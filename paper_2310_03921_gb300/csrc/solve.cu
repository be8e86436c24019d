// Regularised least-squares fit of the sparse GP coefficients (Sec. 2,
// Eqs. 4-9), in FP64 on the GPU:
//   K_MM = delta^2 (X X^T)^zeta per GP (block diagonal over GPs) + jitter I
//   K_MM = U^T U (Cholesky),  A = [S^-1/2 K_NM ; U],  b = [S^-1/2 y ; 0]
//   A = Q R (Householder),     c = R^-1 Q^T b
// S = diag(sigma^2) is the per-row regularisation of Eq. 4.  The Cholesky,
// QR and Q^T b steps call cuSOLVER (library dense factorisations); the
// assembly of K_MM and of the stacked system are kernels of this file.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <string>
#include <vector>

#include "gap_internal.h"
#include "solve.h"

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

#define GAP_TRY_SOLVER(call)                                                               \
    do {                                                                                   \
        cusolverStatus_t _s = (call);                                                      \
        if (_s != CUSOLVER_STATUS_SUCCESS) {                                               \
            gap_set_error(std::string(#call) + " failed: " + cusolver_name(_s));           \
            st_out = GAP_ECUDA;                                                            \
            goto done;                                                                     \
        }                                                                                  \
    } while (0)

#define GAP_TRY_C(call)                                                                    \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess) { st_out = gap_cuda_status(_e, #call); goto done; }         \
    } while (0)

gap_status gap_solve_dev(const SolveInputs &in, double *alpha_out, cudaStream_t st)
{
    const long R = in.rows;
    const int M = in.M;
    gap_status st_out = GAP_OK;
    cusolverDnHandle_t h = nullptr;
    double *Kmm = nullptr, *A = nullptr, *b = nullptr, *tau = nullptr, *work = nullptr;
    int *info = nullptr;
    int lwork = 0, lw2 = 0, lw3 = 0, hinfo = 0;
    const long lda = R + M;
    if (M <= 0) return GAP_OK;
    if (lda > 2147483647L || lda * (long)M > (1L << 40)) {
        gap_set_error("least-squares system too large");
        return GAP_EINVAL;
    }
    GAP_TRY_C(cudaMalloc(&Kmm, sizeof(double) * (size_t)M * M));
    GAP_TRY_C(cudaMalloc(&A, sizeof(double) * (size_t)lda * M));
    GAP_TRY_C(cudaMalloc(&b, sizeof(double) * (size_t)lda));
    GAP_TRY_C(cudaMalloc(&tau, sizeof(double) * (size_t)M));
    GAP_TRY_C(cudaMalloc(&info, sizeof(int)));
    {
        dim3 grid((M + 63) / 64, (M + 63) / 64);
        gap_count_launch();
        k_kmm<<<grid, 256, 0, st>>>(in.X, in.D, in.block_of, M, in.delta * in.delta, in.zeta, in.jitter, Kmm);
        GAP_TRY_C(cudaGetLastError());
    }
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) {
        gap_set_error("cusolverDnCreate failed");
        st_out = GAP_ECUDA;
        goto done;
    }
    GAP_TRY_SOLVER(cusolverDnSetStream(h, st));
    GAP_TRY_SOLVER(cusolverDnDpotrf_bufferSize(h, CUBLAS_FILL_MODE_UPPER, M, Kmm, M, &lwork));
    GAP_TRY_SOLVER(cusolverDnDgeqrf_bufferSize(h, (int)lda, M, A, (int)lda, &lw2));
    GAP_TRY_SOLVER(cusolverDnDormqr_bufferSize(h, CUBLAS_SIDE_LEFT, CUBLAS_OP_T, (int)lda, 1, M, A, (int)lda, tau, b,
                                               (int)lda, &lw3));
    if (lw2 > lwork) lwork = lw2;
    if (lw3 > lwork) lwork = lw3;
    GAP_TRY_C(cudaMalloc(&work, sizeof(double) * (size_t)(lwork > 0 ? lwork : 1)));
    GAP_TRY_SOLVER(cusolverDnDpotrf(h, CUBLAS_FILL_MODE_UPPER, M, Kmm, M, work, lwork, info));
    GAP_TRY_C(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    GAP_TRY_C(cudaStreamSynchronize(st));
    if (hinfo != 0) {
        gap_set_error("K_MM + jitter is not positive definite (potrf info " + std::to_string(hinfo) + ")");
        st_out = GAP_ENOTPD;
        goto done;
    }
    {
        long total = lda * M;
        gap_count_launch();
        k_stack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(in.K, in.y, in.sigma, R, M, Kmm, A, b);
        GAP_TRY_C(cudaGetLastError());
    }
    GAP_TRY_SOLVER(cusolverDnDgeqrf(h, (int)lda, M, A, (int)lda, tau, work, lwork, info));
    GAP_TRY_SOLVER(cusolverDnDormqr(h, CUBLAS_SIDE_LEFT, CUBLAS_OP_T, (int)lda, 1, M, A, (int)lda, tau, b, (int)lda,
                                    work, lwork, info));
    gap_count_launch();
    k_backsub<<<1, 1024, sizeof(double) * M, st>>>(A, lda, M, b, alpha_out);
    GAP_TRY_C(cudaGetLastError());
    GAP_TRY_C(cudaStreamSynchronize(st));
done:
    if (h) cusolverDnDestroy(h);
    cudaFree(Kmm);
    cudaFree(A);
    cudaFree(b);
    cudaFree(tau);
    cudaFree(work);
    cudaFree(info);
    return st_out;
}
