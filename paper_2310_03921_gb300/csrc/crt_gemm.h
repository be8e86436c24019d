// FP64-accurate matrix products on the BF16 tensor cores by modular integer
// arithmetic (internal; see crt_gemm.cu).
#pragma once

#include <cuda_bf16.h>

#include "gap_internal.h"

constexpr int kCrtMaxModuli = 16;      // moduli <= 256 (byte residues)
constexpr int kCrtMaxModuliWide = 40;  // the same 16, then primes 373 .. 509

// A matrix read element by element: rows [0, R) are Y[i * ldy + j] times
// rscale[i] (rscale may be NULL), rows [R, R + n_u) are the upper-triangular
// factor U (column-major, leading dimension ldu): U[(i - R) + j * ldu] for
// j >= i - R, else 0.  rows = R + n_u, cols columns.  With `ext` set, the
// last column (j = cols - 1) of the rows [0, R) is ext[i] times rscale[i]
// instead (an appended right-hand side), and 0 in the rows of U.
struct CrtVMat {
    const double *Y;
    long ldy;
    const double *rscale;
    long R;
    const double *U;
    int ldu;
    long rows;
    int cols;
    const double *ext = nullptr;
};

// Moduli needed for an inner dimension K (0 if K is beyond the 16 moduli).
int gap_crt_moduli(long K);
// Operand rows padded: the K extent of the residue planes (multiple of 64).
inline long gap_crt_kpad(long K) { return (K + 63) / 64 * 64; }

// Residues of the operand whose rows are the rows of V (inner index = column
// of V): res [T][V.rows][kpad] BF16, E [V.rows] the largest FP64 exponent
// field of each row.
gap_status gap_crt_prep_rows(const CrtVMat &V, int T, long kpad, __nv_bfloat16 *res, int *E, cudaStream_t st);
// Residues of the operand whose rows are the columns of V (inner index = row
// of V): res [T][V.cols][kpad] BF16 with kpad >= V.rows, E [V.cols].  With
// `diag` (n_diag entries, stride ld_diag), E[j] is raised for j < n_diag to
// at least the exponent field of sqrt|diag[j]|, so that a symmetric positive
// semi-definite matrix with that diagonal fits the fixed-point grid of the
// Gram matrix of V below 2^106 (gap_crt_exact_gram).
gap_status gap_crt_prep_cols(const CrtVMat &V, int T, long kpad, __nv_bfloat16 *res, int *E, cudaStream_t st,
                             const double *diag = nullptr, long ld_diag = 0, int n_diag = 0);
// Residues of C' = A' B'^T modulo each of the T moduli (of the wide set; the
// first 16 are the byte moduli): out [T][rowsA][ldo].  sym: only tiles
// touching the upper triangle (A and B are the same operand).  b_lower: row j
// of B is zero beyond column j (B^T upper triangular), so K stops at the
// tile's last column; a_lower: row i of A is zero beyond column i.  out_bf16:
// `out` holds BF16 symmetric residues (|r| <= p / 2, columns from rowsB to the
// tile's end written as 0, ldo in elements), ready as the operand of a further
// product; otherwise bytes in [0, p), T <= 16.
gap_status gap_crt_gemm(const __nv_bfloat16 *resA, long rowsA, const __nv_bfloat16 *resB, long rowsB, long kpad,
                        int T, bool sym, bool b_lower, void *out, long ldo, int *err, cudaStream_t st,
                        bool a_lower = false, bool out_bf16 = false);
// C[i * ldc + j] = alpha 2^(Ea[i] + Eb[j] - 2150) C'[i][j] (+ Cin[i * ldcin + j]
// if Cin), C' rebuilt from the residues (Chinese remainder theorem); sym reads
// the upper triangle for j < i.  C may alias Cin element for element.
gap_status gap_crt_combine(const unsigned char *out, long ldo, long rows, int cols, int T, const int *Ea,
                           const int *Eb, bool sym, double *C, long ldc, cudaStream_t st, double alpha = 1.0,
                           const double *Cin = nullptr, long ldcin = 0);

// ---------------------------------------------------------------------------
// Exact congruence products W^T G W of an exactly known Gram matrix.
//
// The Gram matrix G' = V'^T V' of the fixed-point operand of
// gap_crt_prep_cols (an integer below (rows) 2^106) plus a symmetric matrix
// Kt rounded to the same grid is kept as exact residues modulo T2 moduli of
// the wide set; for any W (FP64, upper triangular), W^T G W is then formed as
// an exact integer from one more fixed-point rounding of W and rounded once
// to FP64.  `n` is the order of Kt and W; the operand has n_ext = n + 1
// columns (the last one the appended right-hand side b), W is extended by a
// unit last column so that the last column of W^T G W is W^T V^T b.

// Wide moduli needed for signed integers below 2^bits (0 if beyond 40).
int gap_crt_moduli_wide(double bits);
// Bits of the entries of W^T G' W for an n_ext-column operand of `rows` rows.
double gap_crt_congruence_bits(long rows, int n_ext);

// From the byte residues `out` (T1 moduli, sym tiles, ldo) of the Gram matrix
// of the n_ext-column operand with column exponents E: G' + round(Kt) exactly,
// as BF16 symmetric residues res [T2][n_ext][kpad2] (columns n_ext .. kpad2
// zero), and rounded to FP64 as G (n x n, column-major; Kt's block only).
// out == NULL: no data rows (G' = 0).  Kt column-major (ld n) or NULL.
// err |= 16 if a rounded Kt entry exceeds 2^110 (not semi-definite).
gap_status gap_crt_exact_gram(const unsigned char *out, long ldo, int T1, int n, const int *E, const double *Kt,
                              int T2, long kpad2, __nv_bfloat16 *res, double *G, int *err, cudaStream_t st);
// Residues of the operand whose rows are the columns of W_ext D (D =
// diag(2^(E_k - 1075)), the Gram matrix's column scales): res
// [T2][n_ext][kpad2], row exponents F [n_ext].  Wt (may be NULL, may alias W
// element for element) receives the W actually represented (column-major,
// ld n): W rounded to 53 bits below each column's largest scaled entry.
gap_status gap_crt_prep_congruence(const double *W, int n, const int *E, int T2, long kpad2, __nv_bfloat16 *res,
                                   int *F, double *Wt, cudaStream_t st);
// C = W^T G W from the BF16 residues of its upper tiles (T2 moduli, ld ldo)
// and the row exponents F: G (n x n, column-major, both triangles) and
// c[i] = C[i][n] (i < n), the transformed right-hand side.
gap_status gap_crt_combine_congruence(const __nv_bfloat16 *out, long ldo, int n, int T2, const int *F, double *G,
                                      double *c, cudaStream_t st);
