// Neighbour search workspace and entry points (internal).
#pragma once

#include <vector>

#include "gap_internal.h"

struct CellGeom {
    double cell[9], inv[9];
    double rc2;
    float cell32[9];
    float rc2_loose;  // squared cutoff widened past the FP32 rounding of frac32: the prefilter bound
    float rc2_tight;  // squared cutoff narrowed by the same margin: below it a pair is surely inside
    int nb[3], R[3], pbc[3];
    int bin0;
};

struct NbrWork {
    CellGeom *geo = nullptr;
    int *cfg_offsets = nullptr;
    double *frac = nullptr;
    float4 *frac32 = nullptr;  // FP32 copy of frac (prefilter of the candidate scans)
    int *atom_cfg = nullptr, *atom_bin = nullptr, *bin_atoms = nullptr, *counts = nullptr;
    int *bin_count = nullptr, *bin_fill = nullptr, *bin_start = nullptr;
    int *scan_tmp = nullptr, *total = nullptr, *err = nullptr;
    long long *keys = nullptr;
    PairList pairs{};
    // Graph mode (a captured MD step): no host synchronisation; the pair
    // arrays have a fixed capacity, cell geometry and configuration offsets
    // stay as the last ordinary build uploaded them.  A build that would
    // exceed the capacity leaves every atom without pairs and sets err bit 1.
    bool graph = false;
    int pair_cap = 0;
    size_t cap_geo = 0, cap_cfg = 0, cap_frac = 0, cap_acfg = 0, cap_abin = 0, cap_batoms = 0, cap_counts = 0,
           cap_offsets = 0, cap_bcount = 0, cap_bfill = 0, cap_bstart = 0, cap_scan = 0, cap_total = 0,
           cap_keys = 0, cap_j = 0, cap_rev = 0, cap_v64 = 0, cap_v32 = 0, cap_f32 = 0;

    gap_status reserve_atoms(int n, int n_configs, int n_bins);
    gap_status reserve_pairs(int P);
    void release();
};

gap_status gap_cell_geometry(const gap_batch *b, double rc, std::vector<CellGeom> &geo, int &n_bins);
// Builds the sorted CSR pair list of the batch on `st` (positions d_pos on the
// device).  Synchronises once to read the pair count (not in graph mode).
gap_status gap_neighbours(NbrWork &w, const gap_batch *b, const double *d_pos, double rc, cudaStream_t st);
// Reads the device error flag of the last build (synchronous): GAP_ECAPACITY
// for a graph-mode build beyond its pair capacity.
gap_status gap_neighbours_check(NbrWork &w, cudaStream_t st);
gap_status gap_scan(const int *in, int n, int *out, int *tmp, int *total, cudaStream_t st);
size_t gap_scan_tmp_ints(int n);
