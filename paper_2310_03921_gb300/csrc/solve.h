// Regularised least-squares solve (internal).
#pragma once

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
};

gap_status gap_solve_dev(const SolveInputs &in, double *alpha_out, cudaStream_t st);
