// K_NM assembly kernels (internal).
#pragma once

#include "gap_internal.h"

// Jacobian rows of the force-row GEMM, target-major (see knm.cu).
struct KnmRows {
    void *A;                     // [rows][D16] T (CUDA-core forms)
    __nv_bfloat16 *A_hi, *A_lo;  // [rows][D16] (tensor-core form)
    __nv_bfloat16 *A_mid;        // middle plane of the three-plane split, or NULL
    float *t_row;                // [rows] J . mu (tensor-core form)
    int *src_sign;               // [rows]
    int *seg;                    // [rows]
};

gap_status gap_knm_segments(int n, const int *offsets, const int *atom_cfg, int *seg_start, int *out_row,
                            cudaStream_t st);
template <typename T, bool SPLIT>
gap_status gap_jacobian_rows(const SoapGeom &g, const T *tab, int n, const PairList &pl, const int *species,
                             const T *coef, const T *phat, const T *pnorm, const int *gp_of_atom, const float *mu_all,
                             KnmRows &out, cudaStream_t st);
// Compressed descriptors (p~ = Q p renormalised): V = J Q^T for rows J
// [nrow][ldj] in T and Q [Dg][D] (CUDA-core forms; V [nrow][ldv], columns
// Dg .. ldv - 1 untouched) ...
template <typename T>
gap_status gap_rows_times_qt(long nrow, int D, const T *J, int ldj, int Dg, const T *Q, T *V, int ldv,
                             cudaStream_t st);
// ... and the compressed rows J~ = (|p| / |p~|) (I - p_hat~ p_hat~^T) V of each
// row's source atom, [nrow][Dg16] into out.A (T; may alias V when ldv ==
// Dg16) or, SPLIT, into out.A_hi / A_lo / A_mid with out.t_row = J~ . mu~ of
// the source atom's GP (mu_all [n_gp][Dg16]).
template <typename T, bool SPLIT>
gap_status gap_jacobian_compress(long nrow, int Dg, int Dg16, const T *V, int ldv, const int *src_sign,
                                 const int *gp_of_atom, const T *phatc, const T *pnorm, const T *pnormc,
                                 const float *mu_all, KnmRows &out, cudaStream_t st);
template <typename T>
gap_status gap_knm_qpow_simt(const T *phat, int D, const int *rows, int nrows, const T *X, int M, double delta,
                             int zeta, T *Wp, T *kq, int ld, cudaStream_t st);
template <typename T>
gap_status gap_knm_force_simt(const T *A, int D, int D16, long nrow, const int *seg, int n_seg, const int *seg_start,
                              const int *out_row, const int *src_sign, const T *X, int M, const T *Wp, int ldw,
                              double *K, int ldk, int col_out0, T *P, int ldp, cudaStream_t st);
template <typename T>
gap_status gap_knm_energy(int n_configs, const int *cfg_off, const T *kq, int ld, int M, double *K, int ldk,
                          int col_out0, cudaStream_t st);
// dest[r] for the tensor-core K_NM epilogue (128-row tiles): the K row
// out_row[seg[r]] when the segment of row r lies inside r's tile, else
// -1 - slot with slot 0 for a tile's first row and 1 otherwise (the partial
// sums of a segment cut by a tile edge).  Meaningful at segment starts and
// at tiles' first rows.
gap_status gap_knm_dest(long nrow, const int *seg, const int *seg_start, const int *out_row, int *dest,
                        cudaStream_t st);
// K rows of the segments cut by the 128-row tile edges of the tensor-core
// K_NM epilogue, from the partial sums P[tile][slot][column] it left.
gap_status gap_knm_fixup(long nrow, const int *seg, const int *seg_start, const int *out_row, const float *P, int ldp,
                         int M, double *K, int ldk, int col_out0, cudaStream_t st);
