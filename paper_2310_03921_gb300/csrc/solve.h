// Regularised least-squares solve (internal).
#pragma once

#include <vector>

#include <cublas_v2.h>
#include <cusolverDn.h>

#include "gap_internal.h"

struct SolveInputs {
    long rows;             // rows of K_NM
    int M;                 // columns (all GPs' sparse points)
    const double *K;       // device [rows][M] row-major
    const double *y;       // device [rows]
    const double *sigma;   // device [rows]
    const double *X;       // device [M][D] sparse points (GP blocks concatenated)
    const int *block_of;   // device [M] GP index of each column
    int D;
    double delta, jitter;
    int zeta;
    // gap_solve_tc_dev only: when set, also the M x M upper-triangular
    // inverse factor R^-1 of A^T A = R^T R (column-major), A = [S^-1/2 K ; U].
    double *rinv_out = nullptr;
};

// Device buffers and library handles of the solve, kept between calls.
struct SolveWork {
    static constexpr int kSlots = 40;
    void *buf[kSlots] = {};
    size_t cap[kSlots] = {};
    cusolverDnHandle_t solver = nullptr;
    cublasHandle_t blas = nullptr;
    // Autotuned (first factorisation on the device): block products with at
    // most this many multiply-adds run on the FP64 units, larger ones as
    // modular tensor-core products.
    long small_product = -1;
    // The tuner's measurements: best times (ms) of an sz x sz x sz product,
    // sz = 32, 64, ..., on the FP64 kernel [0] and as a modular product [1].
    float tune_ms[2][8] = {};
    int tune_sizes = 0;
    // gap_chol_inv_dev's launch sequence (its kernels depend only on n, the
    // operand pointers and the workspace) captured once as a CUDA graph and
    // replayed: the keys of recent direct runs and the captured graphs.
    struct CholGraph {
        std::vector<const void *> key;
        cudaGraphExec_t exec = nullptr;
        long kernels = 0;
    };
    std::vector<std::vector<const void *>> chol_seen;
    std::vector<CholGraph> chol_graphs;
    cudaStream_t cap_stream = nullptr;  // where the sequence is captured
    gap_status ensure(int slot, size_t bytes);  // slot < kSlots (checked at compile time by the callers' enum)
    template <typename T> T *at(int slot) const { return static_cast<T *>(buf[slot]); }
    gap_status handles(cudaStream_t st);
    void release();
};

// Householder QR (cuSOLVER geqrf/ormqr) of the stacked system, all FP64.
gap_status gap_solve_dev(const SolveInputs &in, double *alpha_out, SolveWork &w, cudaStream_t st);
// Shifted CholeskyQR3 of the same system: the Gram matrix of [S^-1/2 K_NM |
// S^-1/2 y] plus K_MM + jitter I as an exact integer (modular products on the
// tensor cores, crt_gemm.h), the later passes' Gram matrices and the
// transformed right-hand side as exact congruences W^T G W of it; Cholesky
// factors and inverses of the M x M Gram matrices by gap_chol_inv_dev.
gap_status gap_solve_tc_dev(const SolveInputs &in, double *alpha_out, SolveWork &w, cudaStream_t st);
// Measures the crossover of gap_chol_inv_dev's block products on the device
// (G: a matrix of order n >= 32 on the device, its leading blocks the
// operands) into w.small_product and w.tune_ms.
gap_status gap_tune_small_product(SolveWork &w, int n, const double *G, cudaStream_t st);
// Upper Cholesky factor R (G = R^T R) and its inverse X of an SPD n x n
// matrix, all column-major (ld n): recursive halving with the off-diagonal
// products as FP64-accurate modular GEMMs on the tensor cores (small ones in
// FP64), blocks of order <= 64 factorised in FP64 by one kernel.  Synchronous.  GAP_ENOTPD for a non-positive pivot.
// refine = false skips the refinement of the off-diagonal blocks (a factor
// good as a preconditioner, not FP64-accurate).
gap_status gap_chol_inv_dev(SolveWork &w, int n, const double *G, double *R, double *X, cudaStream_t st,
                            bool refine = true);

// Posterior factors of the fitted sparse GP (predictive variances): the
// inverse Cholesky factor U^-1 of Kt = K_MM + jitter I (block diagonal over
// GPs) into kinv_out and R^-1 of A^T A into rinv_out, both M x M upper
// triangular, column-major; alpha_scratch [M] receives the coefficients of
// the same solve.  Synchronous.
gap_status gap_posterior_dev(const SolveInputs &in, double *kinv_out, double *rinv_out, double *alpha_scratch,
                             SolveWork &w, cudaStream_t st);
struct CrtVMat;
// C[r * ldc + c] = sum_k Aop[r][k] Bop[c][k], FP64-accurate (modular
// tensor-core product, or an FP64 kernel for small sizes); an operand with
// `cols_of` set contributes the columns of its view as rows; b_lower
// declares Bop[c][k] = 0 for k > c.  Uses w's product buffers.
gap_status gap_f64_product(SolveWork &w, const CrtVMat &A, bool a_cols, const CrtVMat &B, bool b_cols, bool b_lower,
                           double *C, long ldc, cudaStream_t st);
