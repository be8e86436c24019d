// FP64-accurate matrix products on the BF16 tensor cores by modular integer
// arithmetic (internal; see crt_gemm.cu).
#pragma once

#include <cuda_bf16.h>

#include "gap_internal.h"

constexpr int kCrtMaxModuli = 16;

// A matrix read element by element: rows [0, R) are Y[i * ldy + j] times
// rscale[i] (rscale may be NULL), rows [R, R + n_u) are the upper-triangular
// factor U (column-major, leading dimension ldu): U[(i - R) + j * ldu] for
// j >= i - R, else 0.  rows = R + n_u, cols columns.
struct CrtVMat {
    const double *Y;
    long ldy;
    const double *rscale;
    long R;
    const double *U;
    int ldu;
    long rows;
    int cols;
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
// of V): res [T][V.cols][kpad] BF16 with kpad >= V.rows, E [V.cols].
gap_status gap_crt_prep_cols(const CrtVMat &V, int T, long kpad, __nv_bfloat16 *res, int *E, cudaStream_t st);
// Residues of C' = A' B'^T modulo each of the T moduli: out [T][rowsA][ldo]
// bytes, ldo a multiple of 256.  sym: only tiles touching the upper triangle
// (A and B are the same operand).  b_lower: row j of B is zero beyond column
// j (B^T upper triangular), so K stops at the tile's last column.
gap_status gap_crt_gemm(const __nv_bfloat16 *resA, long rowsA, const __nv_bfloat16 *resB, long rowsB, long kpad,
                        int T, bool sym, bool b_lower, unsigned char *out, long ldo, int *err, cudaStream_t st);
// C[i * ldc + j] = alpha 2^(Ea[i] + Eb[j] - 2150) C'[i][j] (+ Cin[i * ldcin + j]
// if Cin), C' rebuilt from the residues (Chinese remainder theorem); sym reads
// the upper triangle for j < i.  C may alias Cin element for element.
gap_status gap_crt_combine(const unsigned char *out, long ldo, long rows, int cols, int T, const int *Ea,
                           const int *Eb, bool sym, double *C, long ldc, cudaStream_t st, double alpha = 1.0,
                           const double *Cin = nullptr, long ldcin = 0);
