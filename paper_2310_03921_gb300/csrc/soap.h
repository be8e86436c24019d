// Descriptor, backward and force kernels (internal).
#pragma once

#include "gap_internal.h"

struct TwoBodyDev {
    int m;
    double rc, d, theta, delta;
    const double *x, *a;  // device [m]
};

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
gap_status gap_config_sums(int n_configs, const int *cfg_off, const double *eps, const double *eps2,
                           const double *vir_atom, double *energy, double *virial, cudaStream_t st);
gap_status gap_local_energy(int n, const double *eps, const double *eps2, double *out, cudaStream_t st);
gap_status gap_pair_atoms(int n, const PairList &pl, int *pair_i, cudaStream_t st);
