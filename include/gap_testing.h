/*
 * Test hooks of libgap: entry points that expose one internal kernel on its
 * own so that it can be checked against an independent computation.  They
 * allocate, synchronise and are not meant for production use.
 */
#ifndef GAP_TESTING_H
#define GAP_TESTING_H

#include "gap.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C = A B^T on the tcgen05 tensor cores with the split-precision schemes of
 * GAP_BF16X3 (nsplit = 2: A, B rounded to BF16 hi + lo on the host, three
 * MMAs) and GAP_BF16X6 (nsplit = 3: hi + mid + lo, six MMAs), FP32
 * accumulation.  A is host [rows][K], B host [cols][K], C host [rows][cols],
 * all row-major FP32; K must be a positive multiple of 16.  Synchronous on the
 * legacy default stream; returns GAP_ETIMEOUT if a bounded device wait expired. */
gap_status gap_test_bf16_gemm(int nsplit, int rows, int cols, int K, const float *A, const float *B, float *C);

/* C = A B^T by the FP64-accurate integer-modular product of the
 * GAP_SOLVE_CHOLQR_TC solve (each row of A and of B rounded to 53 bits below
 * its largest element, the integer product formed exactly modulo up to 16
 * moduli on the tensor cores and rebuilt by the Chinese remainder theorem).
 * A host [rows][K], B host [cols][K], C host [rows][cols], row-major FP64;
 * b_lower != 0 declares B[j][k] = 0 for k > j (the triangular product).
 * K <= 2^18.  Synchronous. */
gap_status gap_test_f64_gemm(int rows, int cols, int K, const double *A, const double *B, int b_lower, double *C);
/* G = Y^T Y by the symmetric modular product (upper tiles only, mirrored):
 * Y host [m][n], G host [n][n], FP64; m <= 2^18.  Synchronous. */
gap_status gap_test_f64_gram(long m, int n, const double *Y, double *G);
/* Upper Cholesky factor R (G = R^T R) and inverse X = R^-1 of an SPD n x n
 * matrix by the recursive factorisation of the GAP_SOLVE_CHOLQR_TC solve
 * (off-diagonal blocks by the modular tensor-core products, blocks <= 64 in
 * FP64).  G, R, X host [n][n] column-major FP64.  Synchronous; GAP_ENOTPD for
 * a non-positive pivot. */
gap_status gap_test_chol_inv(int n, const double *G, double *R, double *X);
/* The exact congruence of the GAP_SOLVE_CHOLQR_TC solve (its passes 2 and
 * 3; the least-squares normal matrix of Sec. 2, Eq. 9, taken through a change
 * of basis W).  V = [Y | b] with Y host [m][n] row-major and b host [m]
 * (m >= 0; NULL when m = 0); G = V^T V + [Kt 0; 0 0] with V and Kt rounded
 * to V's per-column fixed-point grid (53 bits below each column's largest
 * entry), Kt host [n][n] column-major symmetric positive semi-definite or
 * NULL; W host [n][n] column-major upper triangular.  Outputs (host):
 * Wt [n][n] = W~, W rounded to 53 bits below the largest entry of each
 * column of diag(grid) W; Gout [n][n] column-major = the leading block of
 * W~^T G W~ and c [n] = W~^T Y^T b (its last column), each an exact
 * integer rounded once to FP64.  m <= 2^18.  Synchronous; GAP_EINVAL if Kt
 * does not fit the grid (far from semi-definite). */
gap_status gap_test_congruence(long m, int n, const double *Y, const double *b, const double *Kt, const double *W,
                               double *Gout, double *c, double *Wt);
/* The block-product crossover of the recursive factorisation, as its first
 * call on a device measures it: for sizes s = 32, 64, ... (up to 512 and n)
 * the best CUDA-event time of an s x s x s product on the FP64 kernel
 * (ms[k]) and as a modular tensor-core product (ms[8 + k]), k < *sizes;
 * *threshold is the multiply-add count up to which the factorisation uses
 * the FP64 kernel.  G host [n][n] (any values; its leading blocks are the
 * operands), n >= 32.  Synchronous. */
gap_status gap_test_product_crossover(int n, const double *G, float *ms, int *sizes, long *threshold);
/* Measured fused multiply-add throughput of the current GPU in TFLOP/s (two
 * flops per FMA): fp64 = 0 for FP32, 1 for FP64.  Independent FMA chains,
 * eight per thread, 8 CTAs of 256 threads per SM, best of three timed runs
 * (CUDA events) after one warm-up.  The denominator of the rooflines of the
 * ALU-bound kernels.  Synchronous. */
gap_status gap_test_fma_peak(int fp64, double *tflops);

/* The bounded-wait path of the tcgen05 GEMM: one 128 x 256 x 64 tile is
 * launched with every mbarrier wait limited to wait_ns (1 .. 1e9) and a
 * producer that issues no TMA copy, so no MMA is ever issued; each role's
 * wait runs out with nothing in flight, the CTA frees its TMEM and exits.
 * *code receives the kernel's error bits (1: producer, 2: MMA issuer,
 * 4: epilogue).  Returns GAP_ETIMEOUT when a wait expired (the expected
 * outcome), GAP_OK if none did.  The device stays usable.  Synchronous. */
gap_status gap_test_tc_timeout(unsigned long long wait_ns, int *code);
/* Makes device allocations of the library's workspaces fail: after `after`
 * more successful allocations (0: the next one), every workspace allocation
 * returns cudaErrorMemoryAllocation without calling cudaMalloc, so the entry
 * point reports GAP_ENOMEM; after < 0 restores normal allocation.  Covers
 * the per-call workspaces (descriptor, predict, K_NM, solve, neighbours);
 * object creation (gap_soap_create's tables) is not covered. */
gap_status gap_test_fail_alloc(long after);
/* The FP64 reciprocal and reciprocal square root of the factorisation's
 * block kernel (an FP32 estimate refined by Newton steps, no FP64 division
 * or square root) beside CUDA's own double-precision 1.0 / x and rsqrt(x):
 * x host [n] (positive), out host [n][4] = (recip, rsqrt, CUDA 1/x, CUDA
 * rsqrt).  Synchronous. */
gap_status gap_test_fp64_recip(int n, const double *x, double *out);
/* Forces the tensor-core contractions' tile variant (the tile autotuner's
 * candidates, in its order: 0 = 128 x 256 with two TMA stages, 1 = 128 x 128
 * with two, 2 = 128 x 128 with three, 3 = 128 x 192 with twelve epilogue
 * warps) for every later single-problem two-plane call where the variant
 * applies (the grouped launch of several GPs keeps its own tile; variant
 * 3: the K_NM force rows with K <= 256, the kernel-energy and the gradient
 * contractions); other calls keep the tuned choice.  v < 0 restores the
 * autotuner.  For parity tests of every variant; process-wide. */
gap_status gap_test_tc_force_variant(int v);

#ifdef __cplusplus
}
#endif

#endif /* GAP_TESTING_H */
