// Split-precision BF16 tensor-core GEMM (internal).
#pragma once

#include "gap_internal.h"

enum { EPI_STORE = 0, EPI_KERNEL = 1, EPI_QPOW = 2, EPI_KNM = 3 };

// A: [rows][K] (leading dimension lda elements), B: [cols][K] (ldb), both BF16
// K-major, hi and lo parts.  K must be a multiple of 16; lda, ldb multiples of 8.
struct TcOperands {
    const __nv_bfloat16 *A_hi, *A_lo, *B_hi, *B_lo;
    int rows, cols, K, lda, ldb;
    int nsplit;                              // 2: hi + lo planes, 3: hi + mid + lo
    const __nv_bfloat16 *A_mid, *B_mid;      // used when nsplit == 3
};

struct TcEpilogue {
    // EPI_STORE (row_map: optional output row of each GEMM row)
    float *C;
    int ldc;
    const int *row_map;
    // EPI_KERNEL
    const float *s_col, *alpha_col, *t_row;  // [cols padded to 256], [cols padded], [rows]
    float d2;
    int zeta;
    __nv_bfloat16 *W_hi, *W_lo, *W_mid;  // [rows][ldw] (W_mid when nsplit == 3)
    int ldw;
    float *eps_part, *wsum_part;  // [rows][n_part]
    int n_part;                   // 2 * number of column tiles
    // EPI_QPOW: Wp[row_map[r]][c] = zeta d2 q^(zeta-1), kq[row_map[r]][c] = d2 q^zeta
    float *Wp, *kq;
    int ldwp;
    // EPI_KNM (also uses t_row, Wp, ldwp)
    const int *src_sign;   // [rows] +(atom+1) own row, -(atom+1) incoming row
    const int *seg;        // [rows] segment (3 * target + xyz) of each row
    const int *seg_start;  // [segments + 1]
    const int *out_row;    // [segments] row of K
    const int *dest;       // [rows] where a segment starting at this row (or a tile's first row)
                           // goes: its K row, or -1 - slot of P[tile][slot] (gap_knm_dest)
    double *K;
    int ldk, col_out0;
    float *P;              // [row tiles][2][ldp] partial sums of cut segments
    int ldp;
    // Bounded waits: limit of each mbarrier wait in ns (0: the default 2 s).
    unsigned long long wait_ns;
    // Test of the timeout path: the producer issues no copies (so no MMA is
    // ever issued either); every role's wait runs out with nothing in flight.
    int test_stall;
};

// Capacity of the energy epilogue's partial sums per row: the largest
// n_part (epilogue column groups x column tiles) any variant uses for cols.
int gap_tc_max_parts(int cols);
// The tile variant for this call's shape class, autotuned on first use (see
// tc_gemm.cu); returns its column tile and, in *groups, its epilogue column
// groups per tile.  gap_tc_gemm sets ep.n_part for EPI_KERNEL itself, to
// groups * ceil(cols / tile).
int gap_tc_plan(const TcOperands &op, const TcEpilogue &ep, int epi, int *err, cudaStream_t st,
                int *groups = nullptr);
// The tuner's record, in the order the shape classes were tuned: fields =
// (epilogue, planes, K, columns, ceil(log2 rows), column tile, stages,
// device), ms[4] = best time of each variant (256/2, 128/2, 128/3, and
// 192/2 with twelve epilogue warps for the K_NM single-chunk epilogue; -1
// where a variant is not a candidate).
int gap_tc_tuned_count();
// Test hook: every later two-plane call where variant v applies uses it (v < 0: the tuner).
void gap_tc_force_variant(int v);
bool gap_tc_tuned_entry(int k, int *fields, float *ms);
// *err (device int) receives a nonzero code if a bounded wait expired.
gap_status gap_tc_gemm(const TcOperands &op, const TcEpilogue &ep, int epi, int *err, cudaStream_t st);
// Several problems (the GEMMs of a batch's GPs: same planes, epilogue
// EPI_KERNEL or EPI_STORE) in one persistent launch per four problems, tiles
// numbered problem after problem; the default tile variant, whose column tile
// gap_tc_grouped_col_tile gives (EPI_KERNEL's n_part must be 2 ceil(cols / it)).
int gap_tc_grouped_col_tile(int nsplit);
gap_status gap_tc_gemm_grouped(const TcOperands *ops, const TcEpilogue *eps, int n, int epi, int *err, cudaStream_t st);
