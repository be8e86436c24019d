// Radial table construction (internal).
#pragma once

#include "gap_internal.h"

// Allocates and fills the knot table [G+1][N][L+1][2] of I_nl and dI_nl/dr
// (FP64) and the per-interval cubic coefficients [G][N][L+1][4] in FP64 and FP32.
gap_status gap_radial_table(const SoapGeom &g, double **tab64, double **coef64, float **coef32);
// Unnormalised g_n (u^3 P_n^(2,6)(2u-1)) at r, n = 0..N-1 (host).
void gap_radial_basis_host(int N, double rc, double r, double *g_unnormalised);
