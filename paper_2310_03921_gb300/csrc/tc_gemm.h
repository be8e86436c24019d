// Split-precision BF16 tensor-core GEMM (internal).
#pragma once

#include "gap_internal.h"

enum { EPI_STORE = 0, EPI_KERNEL = 1 };

// A: [rows][K] (leading dimension lda elements), B: [cols][K] (ldb), both BF16
// K-major, hi and lo parts.  K must be a multiple of 16; lda, ldb multiples of 8.
struct TcOperands {
    const __nv_bfloat16 *A_hi, *A_lo, *B_hi, *B_lo;
    int rows, cols, K, lda, ldb;
};

struct TcEpilogue {
    // EPI_STORE
    float *C;
    int ldc;
    // EPI_KERNEL
    const float *s_col, *alpha_col, *t_row;  // [cols padded to 256], [cols padded], [rows]
    float d2;
    int zeta;
    __nv_bfloat16 *W_hi, *W_lo;  // [rows][ldw]
    int ldw;
    float *eps_part, *wsum_part;  // [rows][n_part]
    int n_part;                   // 2 * number of column tiles
};

int gap_tc_col_tile(int epi);
// *err (device int) receives a nonzero code if a bounded wait expired.
gap_status gap_tc_gemm(const TcOperands &op, const TcEpilogue &ep, int epi, int *err, cudaStream_t st);
