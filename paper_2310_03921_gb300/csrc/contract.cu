// Kernel contraction of the sparse GP (Eqs. 2, 3 and 13): for the atoms of one
// central species and that species' M sparse points,
//   q_im = p_hat_i . x_m,   eps_i = delta^2 sum_m alpha_m q_im^zeta,
//   g_i  = d eps_i / d p_hat_i = sum_m W_im x_m,  W_im = zeta delta^2 alpha_m q_im^(zeta-1).
// Two SIMT (CUDA-core) GEMMs, templated on the arithmetic type: the plain
// FP64 path and an FP32 variant.  The tensor-core form lives in tc_gemm.cu;
// this file also holds its operand preparation (centring on the mean sparse
// point mu: a_i = p_hat_i - mu, b_m = x_m - mu, q = a.b + a.mu + x_m.mu, and the
// BF16 hi/lo split) and the per-atom finalisation of both forms.
#include <vector>

#include "contract.h"

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

// W[r][m] and per-(row, column tile) partial energies.
template <typename T>
__global__ void __launch_bounds__(256)
k_simt_qW(const T *__restrict__ phat, int D, const int *__restrict__ rows, const int *__restrict__ nrows_p,
          const T *__restrict__ X, const T *__restrict__ alpha, int M, T d2, int zeta, T *__restrict__ W, int ldw,
          double *__restrict__ eps_part, int n_tiles)
{
    __shared__ T As[TK][TM + 1], Bs[TK][TN + 1];
    const int nrows = *nrows_p;
    const int r0 = blockIdx.y * TM, m0 = blockIdx.x * TN;
    if (r0 >= nrows) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < D; k0 += TK) {
        for (int e = threadIdx.x; e < TK * TM; e += 256) {
            int kk = e % TK, rr = e / TK;
            int r = r0 + rr, k = k0 + kk;
            As[kk][rr] = (r < nrows && k < D) ? phat[(size_t)rows[r] * D + k] : T(0);
            int m = m0 + rr;
            Bs[kk][rr] = (m < M && k < D) ? X[(size_t)m * D + k] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty * 4 + u]; b[u] = Bs[kk][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
    __shared__ double red[TM][17];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int r = r0 + ty * 4 + u;
        double e = 0.0;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int m = m0 + tx * 4 + v;
            if (r < nrows && m < M) {
                T q = acc[u][v], qz = T(1);
                for (int z = 1; z < zeta; ++z) qz *= q;
                T a = d2 * alpha[m];
                e += (double)(a * qz * q);
                W[(size_t)r * ldw + m] = T(zeta) * a * qz;
            }
        }
        red[ty * 4 + u][tx] = e;
    }
    __syncthreads();
    if (threadIdx.x < TM) {
        int r = r0 + threadIdx.x;
        double e = 0.0;
        for (int t = 0; t < 16; ++t) e += red[threadIdx.x][t];
        if (r < nrows) eps_part[(size_t)r * n_tiles + blockIdx.x] = e;
    }
}

// g[rows[r]][d] = sum_m W[r][m] X[m][d]
template <typename T>
__global__ void __launch_bounds__(256)
k_simt_G(const T *__restrict__ W, int ldw, const int *__restrict__ rows, const int *__restrict__ nrows_p,
         const T *__restrict__ X, int M, int D, T *__restrict__ g, int ldg)
{
    __shared__ T As[TK][TM + 1], Bs[TK][TN + 1];
    const int nrows = *nrows_p;
    const int r0 = blockIdx.y * TM, d0 = blockIdx.x * TN;
    if (r0 >= nrows) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < M; k0 += TK) {
        for (int e = threadIdx.x; e < TK * TM; e += 256) {
            int kk = e % TK, rr = e / TK;
            int r = r0 + rr, k = k0 + kk;
            As[kk][rr] = (r < nrows && k < M) ? W[(size_t)r * ldw + k] : T(0);
            int kb = e / TN, dd = e % TN;
            int d = d0 + dd, m = k0 + kb;
            Bs[kb][dd] = (m < M && d < D) ? X[(size_t)m * D + d] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty * 4 + u]; b[u] = Bs[kk][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int r = r0 + ty * 4 + u;
        if (r >= nrows) continue;
        int atom = rows[r];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int d = d0 + tx * 4 + v;
            if (d < D) g[(size_t)atom * ldg + d] = acc[u][v];
        }
    }
}

template <typename T>
__global__ void k_eps_rows(const int *__restrict__ rows, const int *__restrict__ nrows_p,
                           const double *__restrict__ eps_part, int n_tiles, double *__restrict__ eps)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= *nrows_p) return;
    double e = 0.0;
    for (int t = 0; t < n_tiles; ++t) e += eps_part[(size_t)r * n_tiles + t];
    eps[rows[r]] = e;
}

// ---------------------------------------------------------------- rows
__global__ void k_gp_flags(int n, const int *__restrict__ species, int s, int *__restrict__ flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = species[i] == s ? 1 : 0;
}

__global__ void k_gp_compact(int n, const int *__restrict__ flag, const int *__restrict__ pos, int *__restrict__ rows,
                             int *__restrict__ gp_of_atom, int s)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) {
        rows[pos[i]] = i;
        gp_of_atom[i] = s;
    }
}

__global__ void k_fill_int(int *__restrict__ a, int n, int v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// -------------------------------------------------- tensor-core operands
// a = p_hat - mu split into BF16 hi + lo (columns D..ld-1 zero); t = a . mu.
__global__ void k_split_rows(const float *__restrict__ phat, int D, int ld, const int *__restrict__ rows, int nrows,
                             const float *__restrict__ mu, __nv_bfloat16 *__restrict__ Ahi,
                             __nv_bfloat16 *__restrict__ Alo, __nv_bfloat16 *__restrict__ Amid,
                             float *__restrict__ t_row)
{
    int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (r >= nrows) return;
    const float *p = phat + (size_t)rows[r] * D;
    float t = 0.f;
    for (int d = lane; d < ld; d += 32) {
        float a = d < D ? p[d] - mu[d] : 0.f;
        __nv_bfloat16 h = __float2bfloat16_rn(a);
        Ahi[(size_t)r * ld + d] = h;
        float rest = a - __bfloat162float(h);
        if (Amid) {
            __nv_bfloat16 m = __float2bfloat16_rn(rest);
            Amid[(size_t)r * ld + d] = m;
            rest -= __bfloat162float(m);
        }
        Alo[(size_t)r * ld + d] = __float2bfloat16_rn(rest);
        t += a * mu[d];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) t_row[r] = t;
}

// eps, wsum and g of the atoms of one GP from the tensor-core partials.
// One warp per row: the column-tile partials of eps and sum_m W summed in
// FP64 (lanes over partials, then a fixed shuffle tree), and g moved to the
// row's atom.  Four rows per block.
__global__ void __launch_bounds__(128) k_tc_finalize(const int *__restrict__ rows, int nrows,
                                                     const float *__restrict__ eps_part,
                                                     const float *__restrict__ wsum_part, int n_part,
                                                     const float *__restrict__ Gs, int D16, double *__restrict__ eps,
                                                     float *__restrict__ wsum, float *__restrict__ g)
{
    const int r = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= nrows) return;
    const int atom = rows[r];
    double e = 0.0, w = 0.0;
    for (int t = lane; t < n_part; t += 32) {
        e += eps_part[(size_t)r * n_part + t];
        w += wsum_part[(size_t)r * n_part + t];
    }
    for (int o = 16; o; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    if (lane == 0) {
        eps[atom] = e;
        wsum[atom] = (float)w;
    }
    if (g)
        for (int d = lane; d < D16; d += 32) g[(size_t)atom * D16 + d] = Gs[(size_t)r * D16 + d];
}

}  // namespace

template <typename T>
gap_status gap_contract_simt(const T *phat, int D, int D16, const int *rows, const int *nrows_dev, int max_rows,
                             const T *X, const T *alpha, int M, double delta, int zeta, T *W, double *eps_part,
                             T *g, double *eps, cudaStream_t st)
{
    if (max_rows <= 0 || M <= 0) return GAP_OK;
    int n_tiles = (M + TN - 1) / TN;
    dim3 g1(n_tiles, (max_rows + TM - 1) / TM);
    gap_prof_begin(ST_GEMM_Q, st);
    gap_count_launch();
    k_simt_qW<T><<<g1, 256, 0, st>>>(phat, D, rows, nrows_dev, X, alpha, M, (T)(delta * delta), zeta, W, M, eps_part,
                                      n_tiles);
    GAP_TRY_CUDA(cudaGetLastError());
    gap_prof_end(ST_GEMM_Q, st);
    dim3 g2((D + TN - 1) / TN, (max_rows + TM - 1) / TM);
    gap_prof_begin(ST_GEMM_G, st);
    if (g) {
        gap_count_launch();
        k_simt_G<T><<<g2, 256, 0, st>>>(W, M, rows, nrows_dev, X, M, D, g, D16);
        GAP_TRY_CUDA(cudaGetLastError());
    }
    gap_count_launch();
    k_eps_rows<T><<<(max_rows + 127) / 128, 128, 0, st>>>(rows, nrows_dev, eps_part, n_tiles, eps);
    GAP_TRY_CUDA(cudaGetLastError());
    gap_prof_end(ST_GEMM_G, st);
    return GAP_OK;
}

template gap_status gap_contract_simt<double>(const double *, int, int, const int *, const int *, int, const double *,
                                              const double *, int, double, int, double *, double *, double *, double *,
                                              cudaStream_t);
template gap_status gap_contract_simt<float>(const float *, int, int, const int *, const int *, int, const float *,
                                             const float *, int, double, int, float *, double *, float *, double *,
                                             cudaStream_t);

int gap_contract_simt_tiles(int M) { return M > 0 ? (M + TN - 1) / TN : 0; }

// The same two GEMMs as gap_contract_simt<double> on the identity row list,
// launched without stage profiling (used by the allocation-free entry point).
gap_status gap_contract_simt_fixed(const double *phat, int D, int ldg, const int *rows, const int *nrows_dev,
                                   int n_rows, const double *X, const double *alpha, int M, double delta, int zeta,
                                   double *W, double *eps_part, double *g, double *eps, cudaStream_t st)
{
    if (n_rows <= 0 || M <= 0) return GAP_OK;
    const int n_tiles = gap_contract_simt_tiles(M);
    dim3 g1(n_tiles, (n_rows + TM - 1) / TM);
    gap_count_launch();
    k_simt_qW<double><<<g1, 256, 0, st>>>(phat, D, rows, nrows_dev, X, alpha, M, delta * delta, zeta, W, M,
                                           eps_part, n_tiles);
    GAP_TRY_CUDA(cudaGetLastError());
    dim3 g2((D + TN - 1) / TN, (n_rows + TM - 1) / TM);
    gap_count_launch();
    k_simt_G<double><<<g2, 256, 0, st>>>(W, M, rows, nrows_dev, X, M, D, g, ldg);
    GAP_TRY_CUDA(cudaGetLastError());
    gap_count_launch();
    k_eps_rows<double><<<(n_rows + 127) / 128, 128, 0, st>>>(rows, nrows_dev, eps_part, n_tiles, eps);
    return gap_cuda_status(cudaGetLastError(), "k_eps_rows");
}

gap_status gap_gp_rows(int n, const int *species, int s, int *flag, int *pos, int *scan_tmp, int *rows, int *count,
                       int *gp_of_atom, cudaStream_t st)
{
    if (n == 0) {
        GAP_TRY_CUDA(cudaMemsetAsync(count, 0, sizeof(int), st));
        return GAP_OK;
    }
    gap_count_launch();
    k_gp_flags<<<(n + 255) / 256, 256, 0, st>>>(n, species, s, flag);
    GAP_TRY_CUDA(cudaGetLastError());
    GAP_TRY(gap_scan(flag, n, pos, scan_tmp, count, st));
    gap_count_launch();
    k_gp_compact<<<(n + 255) / 256, 256, 0, st>>>(n, flag, pos, rows, gp_of_atom, s);
    return gap_cuda_status(cudaGetLastError(), "k_gp_compact");
}

gap_status gap_split_rows(const float *phat, int D, int D16, const int *rows, int nrows, const float *mu,
                          __nv_bfloat16 *Ahi, __nv_bfloat16 *Alo, __nv_bfloat16 *Amid, float *t_row, cudaStream_t st)
{
    if (nrows <= 0) return GAP_OK;
    gap_count_launch();
    k_split_rows<<<(nrows + 3) / 4, 128, 0, st>>>(phat, D, D16, rows, nrows, mu, Ahi, Alo, Amid, t_row);
    return gap_cuda_status(cudaGetLastError(), "k_split_rows");
}

gap_status gap_fill_int(int *a, int n, int v, cudaStream_t st)
{
    if (n <= 0) return GAP_OK;
    gap_count_launch();
    k_fill_int<<<(n + 255) / 256, 256, 0, st>>>(a, n, v);
    return gap_cuda_status(cudaGetLastError(), "k_fill_int");
}

gap_status gap_contract_tc(const float *phat, int D, int D16, const int *rows, int nrows, const TcModelGP &gp,
                           double delta, int zeta, int nsplit, TcScratch &sc, double *eps, float *wsum, float *g,
                           int *err, cudaStream_t st)
{
    if (nrows <= 0 || gp.M <= 0) return GAP_OK;
    const bool three = nsplit == 3;
    gap_prof_begin(ST_SPLIT, st);
    gap_count_launch();
    k_split_rows<<<(nrows + 3) / 4, 128, 0, st>>>(phat, D, D16, rows, nrows, gp.mu, sc.A_hi, sc.A_lo,
                                                   three ? sc.A_mid : nullptr, sc.t_row);
    GAP_TRY_CUDA(cudaGetLastError());
    TcOperands op1{sc.A_hi, sc.A_lo, gp.B_hi, gp.B_lo, nrows, gp.M_pad, D16, D16, D16, nsplit,
                   three ? sc.A_mid : nullptr, three ? gp.B_mid : nullptr};
    TcEpilogue ep1{};
    ep1.s_col = gp.s_col;
    ep1.alpha_col = gp.alpha;
    ep1.t_row = sc.t_row;
    ep1.d2 = (float)(delta * delta);
    ep1.zeta = zeta;
    ep1.W_hi = g ? sc.W_hi : nullptr;
    ep1.W_lo = g ? sc.W_lo : nullptr;
    ep1.W_mid = g && three ? sc.W_mid : nullptr;
    ep1.ldw = gp.M_pad;
    ep1.eps_part = sc.eps_part;
    ep1.wsum_part = sc.wsum_part;
    // the energy partials per column tile of the variant the tuner picks
    int groups = 2;
    const int bn = gap_tc_plan(op1, ep1, EPI_KERNEL, err, st, &groups);
    const int n_part = groups * ((gp.M_pad + bn - 1) / bn);
    ep1.n_part = n_part;
    gap_prof_end(ST_SPLIT, st);
    gap_prof_begin(ST_GEMM_Q, st);
    GAP_TRY(gap_tc_gemm(op1, ep1, EPI_KERNEL, err, st));
    gap_prof_end(ST_GEMM_Q, st);
    TcOperands op2{sc.W_hi, sc.W_lo, gp.BT_hi, gp.BT_lo, nrows, D16, gp.M_pad, gp.M_pad, gp.M_pad, nsplit,
                   three ? sc.W_mid : nullptr, three ? gp.BT_mid : nullptr};
    TcEpilogue ep2{};
    ep2.C = sc.Gs;
    ep2.ldc = D16;
    if (g) {
        gap_prof_begin(ST_GEMM_G, st);
        GAP_TRY(gap_tc_gemm(op2, ep2, EPI_STORE, err, st));
        gap_prof_end(ST_GEMM_G, st);
    }
    gap_prof_begin(ST_FINALIZE, st);
    gap_count_launch();
    k_tc_finalize<<<(nrows + 3) / 4, 128, 0, st>>>(rows, nrows, sc.eps_part, sc.wsum_part, n_part, sc.Gs, D16, eps,
                                                     wsum, g);
    GAP_TRY_CUDA(cudaGetLastError());
    gap_prof_end(ST_FINALIZE, st);
    return GAP_OK;
}

gap_status gap_contract_tc_groups(const float *phat, int D, int D16, const int *const *rows, const int *nrows,
                                  const TcModelGP *gps, int n, double delta, int zeta, int nsplit,
                                  const TcScratch *sc, double *eps, float *wsum, float *g, int *err, cudaStream_t st)
{
    const bool three = nsplit == 3;
    const int bn = gap_tc_grouped_col_tile(nsplit);
    std::vector<TcOperands> op1(n), op2(n);
    std::vector<TcEpilogue> ep1(n), ep2(n);
    gap_prof_begin(ST_SPLIT, st);
    for (int q = 0; q < n; ++q) {
        const TcModelGP &gp = gps[q];
        op1[q] = TcOperands{};
        op2[q] = TcOperands{};
        ep1[q] = TcEpilogue{};
        ep2[q] = TcEpilogue{};
        if (nrows[q] <= 0 || gp.M <= 0) continue;
        gap_count_launch();
        k_split_rows<<<(nrows[q] + 3) / 4, 128, 0, st>>>(phat, D, D16, rows[q], nrows[q], gp.mu, sc[q].A_hi,
                                                          sc[q].A_lo, three ? sc[q].A_mid : nullptr, sc[q].t_row);
        GAP_TRY_CUDA(cudaGetLastError());
        op1[q] = TcOperands{sc[q].A_hi, sc[q].A_lo, gp.B_hi, gp.B_lo, nrows[q], gp.M_pad, D16, D16, D16, nsplit,
                            three ? sc[q].A_mid : nullptr, three ? gp.B_mid : nullptr};
        TcEpilogue &e = ep1[q];
        e.s_col = gp.s_col;
        e.alpha_col = gp.alpha;
        e.t_row = sc[q].t_row;
        e.d2 = (float)(delta * delta);
        e.zeta = zeta;
        e.W_hi = g ? sc[q].W_hi : nullptr;
        e.W_lo = g ? sc[q].W_lo : nullptr;
        e.W_mid = g && three ? sc[q].W_mid : nullptr;
        e.ldw = gp.M_pad;
        e.eps_part = sc[q].eps_part;
        e.wsum_part = sc[q].wsum_part;
        e.n_part = 2 * ((gp.M_pad + bn - 1) / bn);
        op2[q] = TcOperands{sc[q].W_hi, sc[q].W_lo, gp.BT_hi, gp.BT_lo, nrows[q], D16, gp.M_pad, gp.M_pad, gp.M_pad,
                            nsplit, three ? sc[q].W_mid : nullptr, three ? gp.BT_mid : nullptr};
        ep2[q].C = sc[q].Gs;
        ep2[q].ldc = D16;
    }
    gap_prof_end(ST_SPLIT, st);
    gap_prof_begin(ST_GEMM_Q, st);
    GAP_TRY(gap_tc_gemm_grouped(op1.data(), ep1.data(), n, EPI_KERNEL, err, st));
    gap_prof_end(ST_GEMM_Q, st);
    if (g) {
        gap_prof_begin(ST_GEMM_G, st);
        GAP_TRY(gap_tc_gemm_grouped(op2.data(), ep2.data(), n, EPI_STORE, err, st));
        gap_prof_end(ST_GEMM_G, st);
    }
    gap_prof_begin(ST_FINALIZE, st);
    for (int q = 0; q < n; ++q) {
        if (nrows[q] <= 0 || gps[q].M <= 0) continue;
        gap_count_launch();
        k_tc_finalize<<<(nrows[q] + 3) / 4, 128, 0, st>>>(rows[q], nrows[q], sc[q].eps_part, sc[q].wsum_part,
                                                          ep1[q].n_part, sc[q].Gs, D16, eps, wsum, g);
        GAP_TRY_CUDA(cudaGetLastError());
    }
    gap_prof_end(ST_FINALIZE, st);
    return GAP_OK;
}
