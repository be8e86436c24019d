// Kernel contraction (internal).
#pragma once

#include "gap_internal.h"
#include "nbr.h"
#include "tc_gemm.h"

// Model data of one GP for the tensor-core form (all device pointers).
struct TcModelGP {
    int M, M_pad;                        // sparse points, padded to 256
    const float *mu;                     // [D16] mean sparse point (zero padded)
    const float *s_col;                  // [M_pad] x_m . mu (0 in padding)
    const float *alpha;                  // [M_pad] (0 in padding)
    const __nv_bfloat16 *B_hi, *B_lo;    // [M_pad][D16] centred sparse points
    const __nv_bfloat16 *BT_hi, *BT_lo;  // [D16][M_pad] transposed
    const __nv_bfloat16 *B_mid, *BT_mid; // middle planes of the three-plane split
};

// Per-call scratch of the tensor-core form (rows = atoms of one GP).
struct TcScratch {
    __nv_bfloat16 *A_hi, *A_lo;  // [rows][D16]
    float *t_row;                // [rows]
    __nv_bfloat16 *W_hi, *W_lo;  // [rows][M_pad]
    float *eps_part, *wsum_part; // [rows][2 * M_pad / column tile]
    float *Gs;                   // [rows][D16]
    __nv_bfloat16 *A_mid, *W_mid;  // middle planes (three-plane split)
};

template <typename T>
gap_status gap_contract_simt(const T *phat, int D, int D16, const int *rows, const int *nrows_dev, int max_rows,
                             const T *X, const T *alpha, int M, double delta, int zeta, T *W, double *eps_part,
                             T *g, double *eps, cudaStream_t st);

gap_status gap_contract_tc(const float *phat, int D, int D16, const int *rows, int nrows, const TcModelGP &gp,
                           double delta, int zeta, int nsplit, TcScratch &sc, double *eps, float *wsum, float *g,
                           int *err, cudaStream_t st);

// Column tiles of the FP64/FP32 contraction for M sparse points: the row
// stride of its per-tile partial energies (eps_part holds n_rows x tiles).
int gap_contract_simt_tiles(int M);
// The same contraction for several GPs (a batch's central species) with one
// persistent launch per GEMM stage: rows[q], nrows[q] and sc[q] per GP.
gap_status gap_contract_tc_groups(const float *phat, int D, int D16, const int *const *rows, const int *nrows,
                                  const TcModelGP *gps, int n, double delta, int zeta, int nsplit,
                                  const TcScratch *sc, double *eps, float *wsum, float *g, int *err, cudaStream_t st);
gap_status gap_contract_simt_fixed(const double *phat, int D, int ldg, const int *rows, const int *nrows_dev,
                                   int n_rows, const double *X, const double *alpha, int M, double delta, int zeta,
                                   double *W, double *eps_part, double *g, double *eps, cudaStream_t st);

// rows[] = atoms of species s in index order, *count = their number,
// gp_of_atom[atom] = s for those atoms.
gap_status gap_gp_rows(int n, const int *species, int s, int *flag, int *pos, int *scan_tmp, int *rows, int *count,
                       int *gp_of_atom, cudaStream_t st);
gap_status gap_fill_int(int *a, int n, int v, cudaStream_t st);
gap_status gap_split_rows(const float *phat, int D, int D16, const int *rows, int nrows, const float *mu,
                          __nv_bfloat16 *Ahi, __nv_bfloat16 *Alo, __nv_bfloat16 *Amid, float *t_row, cudaStream_t st);
