/*
 * libgap: GB300 (sm_103a) implementation of the data-parallel hot path of
 * Gaussian Approximation Potentials (arXiv 2310.03921): the SOAP descriptor,
 * the sparse-GP dot-product kernel and its Cartesian derivative, and the
 * energy/force rows of the covariance matrix K_NM used by the fit.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns a gap_status; gap_last_error() gives a message for
 *    the calling thread.  No C++ exception crosses this boundary.
 *  - Structure metadata (config offsets, cells, periodicity) is always read
 *    from HOST memory.  Positions, species and every output array live on
 *    the device when gap_batch.device != 0 and on the host otherwise.
 *  - Device-pointer calls are asynchronous on `stream` (a cudaStream_t, or
 *    NULL for the legacy default stream) except for one 4-byte device-to-host
 *    read of the pair count after the neighbour search; host-pointer calls
 *    copy in, run on `stream`, copy out and synchronise before returning.
 *  - The caller owns all input and output buffers.  Handles own their
 *    device tables and workspaces; a handle must not be used by two calls at
 *    the same time.
 *  - On any error status, output arrays may have been partly written.
 *
 * Units: Angstrom, eV.  Cells are row-major [3][3] with rows = lattice
 * vectors.  Species are indices 0..n_species-1.
 *
 * Layout of a descriptor (dimension D, see gap_soap_dim): entries indexed
 * (group g, channel pair a <= b, l), l fastest, then b, then a, then g.
 *   mix_K == 0: one group, channels a = species * n_max + n (full coupling
 *               p^{alpha beta}_{nn'l} of Eq. 23 over all species);
 *   mix_K >  0: mix_K groups (embedded channels k), channels a = n
 *               (p^k_{nn'l} of Eq. 25 with element-wise coupling in k).
 * Off-diagonal pairs carry a factor sqrt(2), so that p . p' equals the full
 * double sum of Eq. 22.  Real spherical harmonics, index l*l + l + m.
 */
#ifndef GAP_H
#define GAP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GAP_OK = 0,
    GAP_EINVAL = -1,      /* invalid argument (null pointer, bad size, unsupported value) */
    GAP_ENOMEM = -2,      /* device or host allocation failed */
    GAP_ECUDA = -3,       /* a CUDA runtime/driver call failed (message has the code) */
    GAP_ETIMEOUT = -4,    /* a bounded device-side wait ran out; results are invalid */
    GAP_ENOTPD = -5,      /* Cholesky factor of K_MM + jitter does not exist */
    GAP_EUNSUPPORTED = -6,/* valid request this build does not implement */
    GAP_ECAPACITY = -7    /* a fixed-capacity buffer (see gap_reserve) was too small */
} gap_status;

typedef enum {
    GAP_FP64 = 0,   /* plain FP64 on CUDA cores for every step */
    GAP_BF16X3 = 1, /* contraction on tcgen05 tensor cores: descriptors centred on the
                       mean sparse point and split into hi+lo BF16, three MMAs per product,
                       FP32 accumulation; FP32 elsewhere, FP64 energy/virial sums */
    GAP_FP32 = 2,   /* FP32 on CUDA cores for every step (no tensor cores) */
    GAP_BF16X6 = 3  /* as GAP_BF16X3 with a three-plane split (hi + mid + lo BF16, six MMAs
                       per product): an FP32-grade contraction for diverse environments
                       and large forces, at twice the tensor-core work */
} gap_precision;

/* SOAP hyperparameters: the `soap` keywords of the paper's Appendix
 * (cutoff, cutoff_transition_width, n_max, l_max, atom_sigma, central_weight,
 * n_species) and the compression keywords Z_mix=T, R_mix=F, coupling=F, K
 * (Sec. 3.3.3, Eq. 25).  mix_w is a host array [mix_K][n_species] copied at
 * creation; the paper draws it from a normal distribution (not optimised).
 * Kernels are compiled for these (n_max, l_max, channel groups) shapes, the
 * channel groups being mix_K when mix_K > 0 and n_species otherwise:
 *   (2, 1, 1) (4, 3, 1) (4, 3, 2) (4, 3, 4) (6, 4, 1) (6, 6, 1) (8, 4, 1)
 *   (8, 4, 5) (8, 6, 1) (8, 6, 4) (8, 8, 1) (10, 8, 1)
 * - among them the paper's silicon model (6, 6, 1; Sec. 4.1) and its
 * five-element alloy model (8, 4, 5; Sec. 4.3).  gap_soap_create returns
 * GAP_EUNSUPPORTED for any other shape.  With central_weight = 0 an atom
 * without a neighbour inside the cutoff has p = 0 and so no normalised
 * descriptor (Eq. 24): its descriptor, local energy and forces come out NaN.
 * With central_weight > 0 (the paper's 1.0) every atom has one. */
typedef struct {
    int n_max;                       /* 1..12 radial functions */
    int l_max;                       /* 0..10 */
    double cutoff;                   /* r_cut of Eq. 18, Angstrom */
    double cutoff_transition_width;  /* d of Eq. 18, 0 < d <= cutoff */
    double atom_sigma;               /* sigma of Eq. 19 */
    double central_weight;           /* weight of the central atom's own Gaussian */
    int n_species;                   /* 1..8 */
    int mix_K;                       /* 0: no compression; >0: embedded channels */
    const double *mix_w;             /* host [mix_K][n_species] or NULL when mix_K == 0 */
} gap_soap_params;

/* Two-body term (distance_2b with the squared-exponential kernel, Eqs. 10-11,
 * times the cutoff function of Sec. 3.3.1): energy per unordered pair
 * delta^2 sum_m alpha_m f_cut(r) exp(-(r - x_m)^2 / (2 theta^2)).
 * Its cutoff must not exceed the SOAP cutoff. */
typedef struct {
    int n_sparse;
    double cutoff, cutoff_transition_width, theta, delta;
    const double *x;      /* host [n_sparse] sparse distances */
    const double *alpha;  /* host [n_sparse] */
} gap_2b_params;

/* A batch of configurations.  Atoms of configuration c are
 * config_offsets[c] .. config_offsets[c+1]-1. */
typedef struct {
    int n_atoms;
    int n_configs;
    const int *config_offsets;  /* host [n_configs + 1], ascending, [0] = 0 */
    const double *cell;         /* host [n_configs][3][3] */
    const int *pbc;             /* host [n_configs][3], 0/1 */
    const double *pos;          /* [n_atoms][3]; device if `device` else host */
    const int *species;         /* [n_atoms]; device if `device` else host */
    int device;
} gap_batch;

typedef struct gap_soap gap_soap;
typedef struct gap_model gap_model;

const char *gap_last_error(void);

/* ---- descriptor object: the initialise / cutoff / descriptor_sizes / calc /
 *      finalise interface of Sec. 3.1.1 ------------------------------------ */

/* Creates the descriptor on the current CUDA device: validates the
 * parameters, builds the orthonormal radial basis (Gram-Schmidt of
 * (r_c - r)^(k+2), k = 1..n_max, under the weight r^2 on [0, r_c]) and tabulates
 * the radial integral of one Gaussian against it (Eqs. 19-20), with its
 * derivative, in FP64 and FP32.  Ownership of *out passes to the caller. */
gap_status gap_soap_create(const gap_soap_params *params, gap_soap **out);
/* Releases the caller's reference.  Models built on the descriptor hold
 * their own references: its device memory is freed when the last of them is
 * destroyed, so the two may be destroyed in either order. */
gap_status gap_soap_destroy(gap_soap *soap);
/* Descriptor dimension D (Sec. 3.3.2 dimension count; layout above). */
gap_status gap_soap_dim(const gap_soap *soap, int *D);
gap_status gap_soap_cutoff(const gap_soap *soap, double *cutoff);
/* The tabulated radial integrals: *knots = G + 1 knots r_k = k * cutoff / G;
 * if out != NULL it receives [G+1][n_max][l_max+1][2] FP64 pairs
 * (I_nl(r_k), dI_nl/dr(r_k)) with
 * I_nl(r) = 4 pi int_0^rc s^2 g_n(s) exp(-(s^2 + r^2)/(2 sigma^2)) i_l(r s / sigma^2) ds,
 * the projection of one Gaussian of Eq. 19 on g_n Y_lm (Eq. 20).  Synchronous. */
gap_status gap_soap_radial_table(const gap_soap *soap, int *knots, double *out);

/* Compression of the descriptor (Sec. 3.3.3 and the soap_turbo recipes of
 * Sec. 3.3.4), applied to the fully coupled multi-species power spectrum
 * (mix_K = 0; channels a = species * n_max + n, Nc = n_species * n_max).
 * Each recipe is a linear map of the ordered power spectrum
 * P^{ab}_l = sum_m c_{a,lm} c_{b,lm}, followed by renormalisation ("the
 * descriptor is renormalized after compression"):
 *   GAP_COMPRESS_SKETCH         p~^k_l = (sum_a w^k_a c_{a,l}) . (sum_b u^k_b c_{b,l}),
 *                               K channels (R_mix = Z_mix = T, sym_mix = F); D~ = K (l_max+1)
 *   GAP_COMPRESS_DECOMPOSITION  the same with u = w (sym_mix = T)
 *   GAP_COMPRESS_NU             p^{alpha beta}_{n n' l} summed over beta (nu_S = 1) or
 *                               alpha and beta (nu_S = 0), over n' (nu_R = 1) or n and n'
 *                               (nu_R = 0); entries ordered (alpha, beta, n, n', l) with
 *                               the summed indices dropped
 *   GAP_COMPRESS_TRIVIAL        soap_turbo's "trivial" recipe: the entries P^{ab}_l with
 *                               a the first radial channel of a species (n = 0), all b, l;
 *                               ordered (species, b, l), D~ = n_species Nc (l_max+1)
 *   GAP_COMPRESS_MATRIX         p~ = P p for a user matrix P [d_out][D] acting on the
 *                               uncompressed power spectrum p = |p| p_hat (the storage of
 *                               gap_descriptor: pairs a <= a', sqrt(2) off the diagonal)
 *   GAP_COMPRESS_NONE           back to the uncompressed descriptor.
 * w, u [K][Nc] (the paper draws them at random and does not optimise them);
 * P [d_out][D]; all host, copied.  Afterwards gap_soap_dim, gap_descriptor
 * and every model made from this object use the compressed descriptor; its
 * energies, forces and virials come through the same backward kernels
 * (dE/dp = P^T dE/dp~), and the force rows of K_NM (gap_assemble_knm,
 * gap_fit) from the Jacobian rows of p_hat mapped by
 * (|p| / |p~|) (I - p_hat~ p_hat~^T) C, C [D~][D] the recipe's linear map
 * (p~ = C p).  Only while no model or step graph
 * holds the object (GAP_EINVAL otherwise). */
typedef enum {
    GAP_COMPRESS_NONE = 0, GAP_COMPRESS_MATRIX = 1, GAP_COMPRESS_SKETCH = 2, GAP_COMPRESS_DECOMPOSITION = 3,
    GAP_COMPRESS_NU = 4, GAP_COMPRESS_TRIVIAL = 5
} gap_compress_recipe;
typedef struct {
    gap_compress_recipe recipe;
    int K;              /* SKETCH, DECOMPOSITION: mixed channels */
    const double *w;    /* [K][Nc] */
    const double *u;    /* [K][Nc] (SKETCH) */
    int nu_R, nu_S;     /* NU: 0, 1 or 2 each */
    int d_out;          /* MATRIX: rows of P */
    const double *P;    /* MATRIX: [d_out][D] */
} gap_compression;
gap_status gap_soap_set_compression(gap_soap *soap, const gap_compression *comp);

/* Counts descriptors (one per atom) and directed neighbour pairs within the
 * cutoff, all periodic images included (Sec. 3.1.1 descriptor_sizes).
 * Synchronous. */
gap_status gap_descriptor_sizes(gap_soap *soap, const gap_batch *batch, long *n_descriptors, long *n_pairs,
                                void *stream);

/* Normalised power spectra p_hat (Eqs. 19-24, compression Eq. 25), one row
 * of D values per atom, row-major [n_atoms][D] FP64.  precision selects the
 * arithmetic of the expansion (GAP_BF16X3 computes in FP32). */
gap_status gap_descriptor(gap_soap *soap, const gap_batch *batch, gap_precision precision, double *p_out,
                          void *stream);

/* ---- sparse GP model (Sec. 3.1.2, Eqs. 2 and 13) ------------------------ */

/* One dot-product GP per central species s < n_gp: local energy of an atom of
 * species s is eps = delta^2 sum_m alpha_s[m] (p_hat . x_s[m])^zeta.
 * sparse[s] is a host array [M[s]][D] of normalised descriptors, alpha[s] a
 * host array [M[s]]; M[s] may be 0.  zeta must be an integer >= 1.  Data are
 * copied; the model holds a reference to `soap` (see gap_soap_destroy).
 * two_body may be NULL. */
gap_status gap_model_create(gap_soap *soap, int n_gp, const int *M, const double *const *sparse,
                            const double *const *alpha, double delta, double zeta, const gap_2b_params *two_body,
                            gap_model **out);
gap_status gap_model_destroy(gap_model *model);
/* Replaces the coefficients alpha of every GP: alpha [M_total] in column
 * order (GP 0's, then GP 1's, ...), device or host per device_ptr.  Ordered
 * on `stream` before later calls on the same stream (host arrays: synchronous). */
gap_status gap_model_set_alpha(gap_model *model, const double *alpha, int device_ptr, void *stream);
/* Total sparse points (columns of K_NM: GP 0's, then GP 1's, ...). */
gap_status gap_model_columns(const gap_model *model, int *M_total);

/* Energy (Eq. 1), local energies (Eq. 2), forces F = -dE/dr (Eq. 3) and virial
 * V_ab = -dE/de_ab for the homogeneous strain r -> (I + e) r, per
 * configuration.  energy [n_configs], local_e [n_atoms] (or NULL),
 * forces [n_atoms][3] (or NULL), virial [n_configs][3][3] (or NULL); all FP64.
 * With forces and virial both NULL the backward pass (Eq. 3) is skipped. */
gap_status gap_predict(gap_model *model, const gap_batch *batch, gap_precision precision, double *energy,
                       double *local_e, double *forces, double *virial, void *stream);

/* Captured MD step.  The paper has no counterpart: it is gap_predict (Eqs.
 * 1-3) of one fixed batch layout recorded as a CUDA graph, for a loop that
 * moves the atoms in place between steps without host round trips.
 * gap_step_graph_create runs the call twice (sizing, then without host
 * synchronisation), then captures it.  Fixed at capture: the batch's device
 * pointers (positions and species are read at every launch), its host
 * metadata (copied: configuration offsets, cells, pbc, species per atom), the
 * precision, the device outputs energy/local_e/forces/virial (each may be
 * NULL as in gap_predict) and a pair capacity of ceil(pair_capacity * pairs
 * of the sizing call), pair_capacity >= 1.  The graph holds a reference to
 * the model; coefficients replaced by gap_model_set_alpha are seen by later
 * launches.  Errors of a launch stay on the device until
 * gap_step_graph_status (synchronous on `stream`), which returns
 * GAP_ECAPACITY when the positions had more pairs than the capacity (that
 * launch's outputs are then meaningless; the graph stays usable). */
typedef struct gap_step_graph gap_step_graph;
gap_status gap_step_graph_create(gap_model *model, const gap_batch *batch, gap_precision precision,
                                 double pair_capacity, double *energy, double *local_e, double *forces,
                                 double *virial, void *stream, gap_step_graph **out);
/* Enqueues one step on `stream`; asynchronous. */
gap_status gap_step_graph_launch(gap_step_graph *graph, void *stream);
gap_status gap_step_graph_status(gap_step_graph *graph, void *stream);
/* Kernels one launch runs. */
long gap_step_graph_kernels(const gap_step_graph *graph);
gap_status gap_step_graph_destroy(gap_step_graph *graph);

/* Rows of L_hat K_NM (text after Eq. 4) for a batch: per configuration one
 * energy row sum_i k(p_hat_i, x_m) followed by 3 n_c force rows
 * -d(sum_i k(p_hat_i, x_m))/d r_ja in (atom, xyz) order; columns are all
 * sparse points of all GPs.  knm is [n_configs + 3 n_atoms][M_total] FP64. */
gap_status gap_assemble_knm(gap_model *model, const gap_batch *batch, gap_precision precision, double *knm,
                            void *stream);

/* How gap_solve factorises the stacked system A = QR:
 *   GAP_SOLVE_HOUSEHOLDER  Householder QR in FP64 on the CUDA cores (cuSOLVER);
 *   GAP_SOLVE_CHOLQR_TC    shifted CholeskyQR3 (three Cholesky QR passes, the
 *                          first with a diagonal shift 11 (m M + M (M+1)) u
 *                          ||A||_F^2, u = 2^-53).  The Gram matrix of the data
 *                          rows with the right-hand side appended, plus
 *                          K_MM + jitter I, is formed once as an exact integer
 *                          by modular products on the BF16 tensor cores; the
 *                          later passes' Gram matrices (A W)^T (A W) and
 *                          (A W)^T b are exact congruences W^T G W of it,
 *                          rounded once to FP64.  Passes 1 and 2 factorise
 *                          (M x M Cholesky factors and inverses by recursive
 *                          halving: the same products, FP64 blocks of <= 64);
 *                          pass 3, whose Gram matrix is then close to the
 *                          identity, is solved by Richardson iteration (a
 *                          factorisation if its Gershgorin bound reaches 1/2).
 *                          Needs rows <= 2^18. */
typedef enum { GAP_SOLVE_HOUSEHOLDER = 0, GAP_SOLVE_CHOLQR_TC = 1 } gap_solve_method;

/* Regularised least-squares fit of the coefficients (Sec. 2: Eq. 4 in the
 * stable form of Eqs. 5-9), on the device:
 *   K_MM = delta^2 (X X^T)^zeta within each GP (zero across GPs) + jitter I,
 *   K_MM = U^T U,  A = [S^-1/2 K ; U],  b = [S^-1/2 y ; 0],  A = QR,  alpha = R^-1 Q^T b,
 * with S = diag(sigma^2).  knm [rows][M_total] (e.g. from gap_assemble_knm),
 * y [rows] targets, sigma [rows] per-row regularisation; alpha_out [M_total].
 * device_ptrs selects device or host arrays.  Keeps its factorisation
 * workspace with the model; synchronous.  GAP_ENOTPD: Householder, if
 * K_MM + jitter has no Cholesky factor (U is formed); CholeskyQR, if one of
 * its Gram matrices has none (U is never formed: K_MM enters only through
 * A^T A = K^T S^-1 K + K_MM + jitter I, so a singular K_MM is solved when
 * the data rows make A^T A positive definite). */
gap_status gap_solve(gap_model *model, long rows, const double *knm, const double *y, const double *sigma,
                     double jitter, gap_solve_method method, double *alpha_out, int device_ptrs, void *stream);

/* The fit of Sec. 2 in one call: K_NM of the batch (the rows of
 * gap_assemble_knm) built in the model's device workspace, the regularised
 * least-squares solve of gap_solve on it, and the solution installed as the
 * model's coefficients (as gap_model_set_alpha), so that K_NM never leaves
 * the device.  y and sigma [n_configs + 3 n_atoms] follow K_NM's row order;
 * alpha_out [M_total] (may be NULL) receives the coefficients.  device_ptrs
 * selects device or host arrays for y, sigma and alpha_out (the batch's own
 * flag selects its memory).  Synchronous; the errors of gap_assemble_knm and
 * gap_solve. */
gap_status gap_fit(gap_model *model, const gap_batch *batch, gap_precision precision, const double *y,
                   const double *sigma, double jitter, gap_solve_method method, double *alpha_out, int device_ptrs,
                   void *stream);

/* Posterior of the fitted sparse GP, for predictive variances (Sec. 3.1.2:
 * gp_predict returns variances beside the local energies).  From the
 * training design of Eq. 4 (knm [rows][M_total] in the row order of
 * gap_assemble_knm, sigma [rows] the per-row regularisation, jitter) it
 * computes and keeps with the model the two M_total x M_total factors
 *   U^-1,  U^T U = Kt = K_MM + jitter I (block diagonal over the GPs), and
 *   R^-1,  R^T R = A^T A = Kt + K^T S^-1 K,  A = [S^-1/2 K ; U] (Eq. 5),
 * the second from the same shifted CholeskyQR passes as gap_solve's
 * GAP_SOLVE_CHOLQR_TC (one more factorisation of the last, near-identity
 * Gram matrix), both FP64-accurate.  rows >= 1 (GAP_EINVAL otherwise; with
 * no data the posterior is the prior, var = delta^2).  device_ptrs selects
 * device or host arrays; synchronous; replaces earlier factors.
 * GAP_ENOTPD if Kt or a Gram matrix has no Cholesky factor; on any error the
 * model has no posterior until a later call succeeds. */
gap_status gap_model_set_posterior(gap_model *model, long rows, const double *knm, const double *sigma, double jitter,
                                   int device_ptrs, void *stream);

/* Predictive variance of each atom's local energy (Sec. 3.1.2) under the
 * posterior of gap_model_set_posterior:
 *   var_i = k(x_i, x_i) - k_i^T Kt^-1 k_i + k_i^T (A^T A)^-1 k_i,
 * k_i [M_total] = delta^2 (p_hat_i . x_m)^zeta over the sparse points of
 * atom i's own GP (0 elsewhere), computed as |k_i|^2 terms of k_i U^-1 and
 * k_i R^-1.  Everything is FP64-accurate: FP64 descriptors, and the kernel
 * rows and both quadratic forms by the modular FP64 products on the tensor
 * cores (the middle term cancels most of the first near the sparse points,
 * so lower precision would not do).  var [n_atoms] (device or host per the
 * batch); atoms whose species has no GP get 0.  GAP_EINVAL if the model has
 * no posterior.  Synchronous for host outputs, else asynchronous on
 * `stream`. */
gap_status gap_predict_variance(gap_model *model, const gap_batch *batch, double *var, void *stream);

/* 'cur_points' sparse-point selection (Sec. 3.2.2: a CUR decomposition
 * based on the data points, after Mahoney and Drineas, PNAS 106, 697
 * (2009)) among the rows of a descriptor matrix x [n][dim] (e.g. the
 * normalised descriptors of gap_descriptor of the candidate atoms of one
 * species): the rank-k leverage score of each row,
 *   pi_i = (1/k) sum_{xi < k} U_{i xi}^2,   x = U S V^T,
 * then the rows with the m largest scores (equal scores: lower index first),
 * skipping a row equal within dup_tol (max norm) to a row already chosen:
 * the paper removes duplicates so that K_MM stays linearly independent.
 * k = 0 takes the numerical rank at singular values >= 1e-4 times the
 * largest, capped by m; k_used (may be NULL) receives the k used.
 * selected [m] receives the chosen rows in selection order and *n_selected
 * their number (< m only if fewer distinct rows exist); scores [n] (may be
 * NULL) the pi_i.  The Gram matrix x^T x and the projections are
 * FP64-accurate modular products on the tensor cores; the dim x dim
 * eigendecomposition is cuSOLVER's syevd.  Scores that differ only in their
 * last bits order either way, as FP64 arithmetic fixes them.  1 <= m <= n
 * <= 2^18, 0 <= k <= dim; device_ptrs selects device or host arrays for x,
 * selected and scores (n_selected and k_used are host).  Synchronous.
 * GAP_EINVAL for bad sizes, a zero x, or k beyond the rank of x. */
gap_status gap_cur_select(const double *x, long n, int dim, int k, int m, double dup_tol, int device_ptrs,
                          int *selected, int *n_selected, double *scores, int *k_used, void *stream);

/* Size in bytes of the static device scratch of gap_gp_energy_noalloc. */
#define GAP_NOALLOC_SCRATCH_BYTES (8u << 20)

/* Allocation-free local energies and descriptor gradients of one GP, for
 * callers that cannot allocate device memory while they run: an MD engine
 * whose host program owns every device buffer and forbids allocation in its
 * force callback, or a latency-critical loop that must not pay the implicit
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart; it
 * computes the same eps as gap_predict's local energies (FP64 path).
 *   p_hat  device [n_rows][D] FP64 normalised descriptors of atoms of GP `gp`
 *   eps    device [n_rows]     eps_i = delta^2 sum_m alpha_m (p_hat_i . x_m)^zeta
 *   grad   device [n_rows][D]  d eps_i / d p_hat_i
 * All arrays are the caller's; the call allocates nothing.  Its scratch (row
 * list, per-tile partial energies, the [n_rows][M] matrix of kernel
 * derivatives) is a file-scope device array of GAP_NOALLOC_SCRATCH_BYTES,
 * held by every GPU that loads the library until the process exits; a request
 * needing more (roughly n_rows * (M + M/64) * 8 bytes) returns GAP_EINVAL.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process; make that first call before any stream capture, and do not
 * use the library across a reset of the device's primary context
 * (cudaDeviceReset), after which the kept address is stale.  Every call
 * shares the array and it keeps the last call's contents: nothing in it
 * needs clearing (each element a call reads is written earlier by the same
 * call), but calls that overlap on the GPU (other streams, other threads)
 * race on it and must be serialised by the caller.  The call reads the
 * model's sparse points and coefficients on `stream`: order it after any
 * coefficient update of the same model (gap_model_set_alpha, gap_fit) that
 * was issued on another stream.  Asynchronous on `stream`. */
gap_status gap_gp_energy_noalloc(const gap_model *model, int gp, int n_rows, const double *p_hat, double *eps,
                                 double *grad, void *stream);

/* ---- instrumentation --------------------------------------------------- */

/* Stage timing: when enabled, every call records a CUDA event pair on its own
 * stream around each stage (neighbours, expansion, gp_rows, split, gemm_q,
 * gemm_g, finalize, chain, pairforce, twobody, gather, knm_rows, knm_gemm,
 * knm_reduce, the solve's stages solve_kmm ... solve_apply, and two stages
 * nested inside others: knm_jacobian, the Jacobian-row kernel inside
 * knm_rows, and solve_block, one interval per factorisation block inside
 * solve_potrf).  Enabling (or gap_profile_reset) clears the record. */
gap_status gap_profile_enable(int on);
gap_status gap_profile_reset(void);
int gap_profile_stages(void);
const char *gap_profile_stage_name(int stage);
/* Sums per stage since the last reset: ms[stage] in milliseconds and
 * count[stage] (may be NULL) intervals.  Waits for the recorded events. */
gap_status gap_profile_read(double *ms, int *count);
/* Number of kernel launches this library has issued in this process. */
long gap_launch_count(void);
/* The tile autotuner of the tensor-core contractions (the batching pattern:
 * tile shapes picked per workload).  The first call of a shape class on a
 * device (epilogue, split, K, columns, ceil(log2 rows)) outside stream
 * capture times each tile variant on its own operands - 128 x 256 with two
 * TMA stages, 128 x 128 with two, 128 x 128 with three, and for the K_NM
 * force rows (K <= 256), the kernel-energy and the gradient contractions
 * 128 x 192 with twelve epilogue warps - and keeps
 * the fastest; captured calls reuse the choice (128 x 256 with two stages
 * for a class not yet tuned).  gap_tile_tuning_count gives
 * the number of tuned classes; entry k: fields[8] = (epilogue, planes, K,
 * columns, ceil(log2 rows), chosen column tile, chosen stages, device) and
 * ms[4] = each variant's best time in that order (-1: not a candidate). */
int gap_tile_tuning_count(void);
gap_status gap_tile_tuning_entry(int k, int *fields, float *ms);

#ifdef __cplusplus
}
#endif

#endif /* GAP_H */
