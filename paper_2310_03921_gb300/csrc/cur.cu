// 'cur_points' sparse-point selection (Sec. 3.2.2: CUR decomposition based
// on the data points, Mahoney and Drineas, PNAS 106, 697 (2009)) on the
// rows of a descriptor matrix X [n][D]:
//   rank-k leverage scores  pi_i = (1/k) sum_{xi < k} U_{i xi}^2,  X = U S V^T,
// computed as pi_i = (1/k) sum_xi (x_i . v_xi)^2 / lambda_xi from the k
// largest eigenpairs of the Gram matrix G = X^T X (U_{i xi} = x_i . v_xi / s_xi);
// then the rows with the m largest scores (equal scores: lower index first),
// a row that duplicates an already chosen row within a tolerance (max norm)
// skipped, as the paper considers duplicates once.
//   G            FP64-accurate modular product on the tensor cores (exact
//                up to one rounding per entry)
//   eigenpairs   of the D x D matrix G: cuSOLVER syevd (a library call)
//   projection   Y = X B^T, B = rows v_xi / sqrt(k lambda_xi): FP64-accurate
//                modular product
//   scores, rank, selection walk: the kernels below.
#include <cmath>
#include <string>
#include <vector>

#include <cusolverDn.h>

#include "crt_gemm.h"
#include "gap_internal.h"
#include "solve.h"

namespace {

struct DevMem {
    void *p = nullptr;
    gap_status get(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        cudaError_t e = gap_dev_malloc(&p, bytes);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            gap_set_error("cudaMalloc of " + std::to_string(bytes) + " bytes for the CUR selection failed");
            return GAP_ENOMEM;
        }
        return GAP_OK;
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
    ~DevMem()
    {
        if (p) cudaFree(p);
    }
};

// Rows of B (k x D, row-major): row xi = v / sqrt(k lambda) for the xi-th
// largest eigenpair (syevd returns ascending eigenvalues, vectors as the
// columns of V, column-major).
__global__ void k_cur_basis(const double *__restrict__ V, const double *__restrict__ lam, int D, int k,
                            double *__restrict__ B)
{
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)k * D) return;
    const int xi = (int)(idx / D), d = (int)(idx - (long)xi * D);
    const int c = D - 1 - xi;
    B[idx] = V[d + (long)c * D] / sqrt((double)k * lam[c]);
}

// pi_i = sum_xi Y[i][xi]^2, one warp per row, lanes in a fixed order.
__global__ void k_cur_scores(const double *__restrict__ Y, int k, long n, double *__restrict__ pi)
{
    const long i = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double s = 0.0;
    for (int x = lane; x < k; x += 32) s = fma(Y[i * k + x], Y[i * k + x], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) pi[i] = s;
}

// order[rank_i] = i with rank_i = #{j : pi_j > pi_i or (pi_j == pi_i and
// j < i)} (a permutation: the ranks are distinct).  Scores staged in shared
// memory in tiles; one thread per i.
constexpr int kRankTile = 2048;
__global__ void __launch_bounds__(256) k_cur_rank(const double *__restrict__ pi, long n, int *__restrict__ order)
{
    __shared__ double tile[kRankTile];
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const double si = i < n ? pi[i] : 0.0;
    long rank = 0;
    for (long t0 = 0; t0 < n; t0 += kRankTile) {
        const int cnt = (int)(n - t0 < kRankTile ? n - t0 : kRankTile);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) tile[e] = pi[t0 + e];
        __syncthreads();
        if (i < n) {
            for (int e = 0; e < cnt; ++e) {
                const double sj = tile[e];
                rank += (sj > si) || (sj == si && t0 + e < i);
            }
        }
    }
    if (i < n) order[rank] = (int)i;
}

// The selection walk, one CTA: candidates in rank order; a candidate is
// taken unless max_d |x_c - x_a| <= tol for an already taken row a (the
// threads split the taken rows); stops at m taken rows or at the end.
__global__ void __launch_bounds__(1024) k_cur_walk(const double *__restrict__ X, int D, const int *__restrict__ order,
                                                    long n, int m, double tol, int *__restrict__ chosen,
                                                    int *__restrict__ n_chosen)
{
    __shared__ int taken, dup;
    if (threadIdx.x == 0) taken = 0;
    __syncthreads();
    for (long t = 0; t < n; ++t) {
        if (taken >= m) break;  // uniform: read after the barrier below
        const int c = order[t];
        if (c < 0 || c >= n) continue;  // uniform across the CTA
        if (threadIdx.x == 0) dup = 0;
        __syncthreads();
        const double *xc = X + (size_t)c * D;
        for (int a = threadIdx.x; a < taken; a += blockDim.x) {
            const double *xa = X + (size_t)chosen[a] * D;
            bool same = true;
            for (int d = 0; d < D && same; ++d) same = fabs(xc[d] - xa[d]) <= tol;
            if (same) dup = 1;
        }
        __syncthreads();
        if (threadIdx.x == 0 && !dup) {
            chosen[taken] = c;
            taken = taken + 1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_chosen = taken;
}

gap_status solver_ok(cusolverStatus_t s, const char *what)
{
    if (s == CUSOLVER_STATUS_SUCCESS) return GAP_OK;
    gap_set_error(std::string(what) + " failed (cuSOLVER status " + std::to_string((int)s) + ")");
    return GAP_ECUDA;
}

}  // namespace

extern "C" gap_status gap_cur_select(const double *x, long n, int D, int k, int m, double dup_tol, int device_ptrs,
                                     int *selected, int *n_selected, double *scores, int *k_used, void *stream)
{
    try {
        if (n < 1 || n > 2147483647L || D < 1 || m < 1 || m > n || k < 0 || k > D || !(dup_tol >= 0.0) || !x ||
            !selected || !n_selected) {
            gap_set_error("gap_cur_select: bad arguments (1 <= m <= n, 0 <= k <= D, dup_tol >= 0, non-NULL arrays)");
            return GAP_EINVAL;
        }
        cudaStream_t st = (cudaStream_t)stream;
        SolveWork w;
        struct Release {
            SolveWork &w;
            ~Release() { w.release(); }
        } rel{w};
        GAP_TRY(w.handles(st));
        DevMem dx, dG, dlam, dinfo, dwork, dB, dY, dpi, dorder, dchosen, dcount;
        const double *X = x;
        if (!device_ptrs) {
            GAP_TRY(dx.get(sizeof(double) * (size_t)n * D));
            GAP_TRY_CUDA(cudaMemcpyAsync(dx.p, x, sizeof(double) * (size_t)n * D, cudaMemcpyHostToDevice, st));
            X = dx.as<double>();
        }
        // G = X^T X (the columns of X as operand rows)
        GAP_TRY(dG.get(sizeof(double) * (size_t)D * D));
        const CrtVMat Xv{X, D, nullptr, n, nullptr, 0, n, D};
        GAP_TRY(gap_f64_product(w, Xv, true, Xv, true, false, dG.as<double>(), D, st));
        // eigenpairs (ascending)
        GAP_TRY(dlam.get(sizeof(double) * (size_t)D));
        GAP_TRY(dinfo.get(sizeof(int)));
        int lwork = 0;
        GAP_TRY(solver_ok(cusolverDnDsyevd_bufferSize(w.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, D,
                                                      dG.as<double>(), D, dlam.as<double>(), &lwork),
                          "syevd_bufferSize"));
        GAP_TRY(dwork.get(sizeof(double) * (size_t)(lwork > 0 ? lwork : 1)));
        GAP_TRY(solver_ok(cusolverDnDsyevd(w.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, D,
                                           dG.as<double>(), D, dlam.as<double>(), dwork.as<double>(), lwork,
                                           dinfo.as<int>()),
                          "syevd"));
        std::vector<double> lam(D);
        int info = 0;
        GAP_TRY_CUDA(cudaMemcpyAsync(lam.data(), dlam.p, sizeof(double) * D, cudaMemcpyDeviceToHost, st));
        GAP_TRY_CUDA(cudaMemcpyAsync(&info, dinfo.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        GAP_TRY_CUDA(cudaStreamSynchronize(st));
        if (info != 0) {
            gap_set_error("gap_cur_select: the eigensolver did not converge (info " + std::to_string(info) + ")");
            return GAP_ECUDA;
        }
        const double lmax = lam[D - 1];
        if (!(lmax > 0.0)) {
            gap_set_error("gap_cur_select: X is zero");
            return GAP_EINVAL;
        }
        // rank: singular values s >= 1e-4 s_max, i.e. lambda >= 1e-8 lambda_max
        int r = 0;
        for (int c = D - 1; c >= 0 && lam[c] >= 1e-8 * lmax; --c) ++r;
        if (k == 0) k = std::max(1, std::min(m, r));
        if (!(lam[D - k] > 0.0)) {
            gap_set_error("gap_cur_select: rank " + std::to_string(k) + " exceeds the rank of X");
            return GAP_EINVAL;
        }
        if (k_used) *k_used = k;
        GAP_TRY(dB.get(sizeof(double) * (size_t)k * D));
        gap_count_launch();
        k_cur_basis<<<(unsigned)(((long)k * D + 255) / 256), 256, 0, st>>>(dG.as<double>(), dlam.as<double>(), D, k,
                                                                          dB.as<double>());
        GAP_TRY_CUDA(cudaGetLastError());
        // Y = X B^T, pi = row norms squared
        GAP_TRY(dY.get(sizeof(double) * (size_t)n * k));
        const CrtVMat Bv{dB.as<double>(), D, nullptr, k, nullptr, 0, k, D};
        GAP_TRY(gap_f64_product(w, Xv, false, Bv, false, false, dY.as<double>(), k, st));
        double *pi = nullptr;
        GAP_TRY(dpi.get(sizeof(double) * (size_t)n));
        pi = dpi.as<double>();
        if (device_ptrs && scores) pi = scores;
        gap_count_launch();
        k_cur_scores<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(dY.as<double>(), k, n, pi);
        GAP_TRY_CUDA(cudaGetLastError());
        GAP_TRY(dorder.get(sizeof(int) * (size_t)n));
        // (a NaN score would leave slots of the permutation unwritten: zero
        // them first so that every slot holds a valid row)
        GAP_TRY_CUDA(cudaMemsetAsync(dorder.p, 0, sizeof(int) * (size_t)n, st));
        gap_count_launch();
        k_cur_rank<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pi, n, dorder.as<int>());
        GAP_TRY_CUDA(cudaGetLastError());
        int *chosen = selected;
        if (!device_ptrs) {
            GAP_TRY(dchosen.get(sizeof(int) * (size_t)m));
            chosen = dchosen.as<int>();
        }
        GAP_TRY(dcount.get(sizeof(int)));
        gap_count_launch();
        k_cur_walk<<<1, 1024, 0, st>>>(X, D, dorder.as<int>(), n, m, dup_tol, chosen, dcount.as<int>());
        GAP_TRY_CUDA(cudaGetLastError());
        GAP_TRY_CUDA(cudaMemcpyAsync(n_selected, dcount.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (!device_ptrs) {
            GAP_TRY_CUDA(cudaMemcpyAsync(selected, chosen, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, st));
            if (scores) GAP_TRY_CUDA(cudaMemcpyAsync(scores, pi, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
        }
        GAP_TRY_CUDA(cudaStreamSynchronize(st));
        return GAP_OK;
    } catch (...) {
        gap_set_error("gap_cur_select: host exception");
        return GAP_ENOMEM;
    }
}
