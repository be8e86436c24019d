// Descriptor, backward and force kernels (internal).
#pragma once

#include "gap_internal.h"

struct TwoBodyDev {
    int m;
    double rc, d, theta, delta;
    const double *x, *a;  // device [m]
    // The pair energy E(r) = delta^2 f_cut(r) sum_m a_m exp(-(r - x_m)^2 / 2 theta^2)
    // as per-interval cubic coefficients (FP64): g_in intervals of width h_in
    // on [0, rc - d] (where f_cut = 1) and g_out of width h_out on [rc - d, rc],
    // so that the kinks of f_cut's derivatives fall on knots.
    const D4 *tab;
    int g_in, g_out;
    double h_in, h_out;
};

// Fills tb.tab (device [g_in + g_out]) from tb's parameters; tab must hold
// g_in + g_out entries.
gap_status gap_twobody_table(const TwoBodyDev &tb, D4 *tab, cudaStream_t st);

bool gap_shape_supported(int N, int L, int GA);

template <typename T>
gap_status gap_expand(const SoapGeom &g, const T *tab, int n, const PairList &pl, const int *species, T *coef, T *phat,
                      T *pnorm, cudaStream_t st);
template <typename T>
gap_status gap_chain(const SoapGeom &g, int n, const T *gvec, const T *wsum, const T *mu, const int *gp_of_atom,
                     const T *phat, const T *pnorm, const T *coef, T *Gam, cudaStream_t st);
template <typename T>
gap_status gap_pairforce(const SoapGeom &g, const T *tab, const PairList &pl, const int *pair_i, const int *species,
                         const T *Gam, T *fpair, cudaStream_t st);
// Two-body term in FP64: per-pair half derivatives f2[P][3], half energies per atom eps2.
gap_status gap_twobody(int n, const PairList &pl, const TwoBodyDev &tb, double *f2, double *eps2, cudaStream_t st);
// Forces and atomic virials from the per-pair derivatives fpair (and f2 if not NULL).
template <typename T>
gap_status gap_gather(int n, const PairList &pl, const T *fpair, const double *f2, double *forces, double *vir_atom,
                      cudaStream_t st);
// Per-configuration energy and virial sums; max_atoms bounds the atoms of a
// configuration, part holds 10 * n_configs * ceil(max_atoms / 2048) doubles
// (gap_config_part_doubles).
gap_status gap_config_sums(int n_configs, const int *cfg_off, int max_atoms, const double *eps, const double *eps2,
                           const double *vir_atom, double *energy, double *virial, double *part, cudaStream_t st);
inline size_t gap_config_part_doubles(int n_configs, int max_atoms)
{
    const int nchunk = max_atoms > 2048 ? (max_atoms + 2047) / 2048 : 1;
    return 10 * (size_t)n_configs * nchunk;
}
gap_status gap_local_energy(int n, const double *eps, const double *eps2, double *out, cudaStream_t st);
gap_status gap_pair_atoms(int n, const PairList &pl, int *pair_i, cudaStream_t st);
