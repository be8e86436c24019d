// Internal declarations of libgap (device helpers shared by the .cu files).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "../../include/gap.h"

#define GAP_MAX_SPECIES 8
#define GAP_MAX_GROUPS 8
#define GAP_MAX_L 10

// ------------------------------------------------------------ error plumbing
void gap_set_error(const std::string &msg);
gap_status gap_cuda_status(cudaError_t e, const char *what);

// cudaMalloc behind a failure-injection point (gap_test_fail_alloc).
cudaError_t gap_dev_malloc(void **p, size_t bytes);

#define GAP_TRY_CUDA(call)                                        \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return gap_cuda_status(_e, #call); \
    } while (0)

// Stage profiler: CUDA events recorded on the launching stream at stage
// boundaries when enabled (gap_profile_enable); no effect otherwise.
enum GapStage {
    ST_NEIGHBOURS = 0, ST_EXPANSION, ST_GP_ROWS, ST_SPLIT, ST_GEMM_Q, ST_GEMM_G, ST_FINALIZE, ST_CHAIN,
    ST_PAIRFORCE, ST_TWOBODY, ST_GATHER, ST_KNM_ROWS, ST_KNM_GEMM, ST_KNM_REDUCE, ST_SOLVE_KMM, ST_SOLVE_QR,
    ST_SOLVE_PREP, ST_SOLVE_GEMM, ST_SOLVE_CRT, ST_SOLVE_POTRF, ST_SOLVE_TRTRI, ST_SOLVE_APPLY,
    ST_KNM_JACOBIAN, ST_SOLVE_BLOCK, ST_COUNT
};
void gap_prof_begin(int stage, cudaStream_t st);
void gap_prof_end(int stage, cudaStream_t st);
void gap_count_launch(int n = 1);
long gap_launch_total();     // kernels counted so far (gap_count_launch)
bool gap_prof_enabled();     // stage profiling on (gap_profile_enable)

#define GAP_TRY(call)                    \
    do {                                 \
        gap_status _s = (call);          \
        if (_s != GAP_OK) return _s;     \
    } while (0)

// ------------------------------------------------------- descriptor geometry
// Accumulation groups ga < GA carry c^g_{n lm} = sum_j wacc[g][Z_j] R_nl Y_lm.
//   mix_K == 0: GA = n_species, wacc = identity, coupling across all (g, n);
//   mix_K  > 0: GA = mix_K,     wacc = mix_w,    coupling within each g.
struct SoapGeom {
    int N, L, LM, S, GA;
    int mixed;          // 1: coupling within a group (Eq. 25); 0: across all channels (Eq. 23)
    int Nc;             // channels per coupling block: N (mixed) or GA*N (full)
    int nblocks;        // coupling blocks: GA (mixed) or 1 (full)
    int npair;          // channel pairs per block: Nc (Nc+1) / 2
    int D;              // nblocks * npair * (L+1)
    int D16;            // D rounded up to a multiple of 16 (row stride of padded buffers)
    double rc, d, sigma, cw;
    int G;              // table intervals; knots 0..G
    double h;           // rc / G
    float wacc32[GAP_MAX_GROUPS * GAP_MAX_SPECIES];
    double wacc64[GAP_MAX_GROUPS * GAP_MAX_SPECIES];
    // K_lm of the real spherical harmonics, index l * (GAP_MAX_L + 1) + m
    double ylmk64[(GAP_MAX_L + 1) * (GAP_MAX_L + 1)];
    float ylmk32[(GAP_MAX_L + 1) * (GAP_MAX_L + 1)];
    // Device table of the descriptor entries ordered by l (D entries):
    // {d, o1, o2, l | (a != a') << 8}, o1 and o2 the offsets of the two
    // coupled channels' (n, l, m = -l) coefficients, so that consecutive
    // entries share their m-range.
    const int4 *dtab;
};

// 32-byte aligned (dx, dy, dz, r) of a pair in FP64.
struct __align__(32) D4 {
    double x, y, z, w;
};

// Radial table: [G+1][N][L+1] of (I_nl(r_k), dI_nl/dr(r_k)); r_k = k h.
template <typename T> struct RadialTab {
    const T *v;  // interleaved value/derivative pairs
};

// ------------------------------------------------------------- pair storage
struct PairList {
    int n_pairs;      // host: pairs the arrays hold (a capacity in graph mode)
    const int *count; // device: pairs of the current build (<= n_pairs)
    int *offsets;     // [N+1]
    int *j;           // [P]
    int *rev;         // [P] index of the reverse pair (j -> i, -shift)
    D4 *vec64;        // [P] (dx, dy, dz, r)
    float4 *vec32;    // [P]
};

// --------------------------------------------------- spherical harmonics
// Real Y_lm: Y_l0 = K_l0 Q_l^0(z), Y_l,+m = K_lm Q_l^m C_m, Y_l,-m = K_lm Q_l^m S_m
// with Q_l^m the m-th derivative of P_l, C_m + i S_m = (x + i y)^m and
// K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) (times sqrt 2 for m > 0).
void gap_fill_ylm_constants(SoapGeom &g);

template <typename T> __device__ __forceinline__ T ylm_k(const SoapGeom &g, int l, int m);
template <> __device__ __forceinline__ double ylm_k<double>(const SoapGeom &g, int l, int m)
{
    return g.ylmk64[l * (GAP_MAX_L + 1) + m];
}
template <> __device__ __forceinline__ float ylm_k<float>(const SoapGeom &g, int l, int m)
{
    return g.ylmk32[l * (GAP_MAX_L + 1) + m];
}

// All Y_lm (index l*l+l+m) of unit vector (x, y, z), L known at compile time.
template <int L, typename T>
__device__ __forceinline__ void ylm_all(const SoapGeom &geo, T x, T y, T z, T *Y)
{
    T C[L + 1], S[L + 1];
    C[0] = T(1); S[0] = T(0);
#pragma unroll
    for (int m = 1; m <= L; ++m) {
        C[m] = x * C[m - 1] - y * S[m - 1];
        S[m] = x * S[m - 1] + y * C[m - 1];
    }
    T q1[L + 1], q2[L + 1];  // Q_{l-1}^m, Q_{l-2}^m
#pragma unroll
    for (int l = 0; l <= L; ++l) {
        T q[L + 1];
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            if (m > l) continue;
            if (m == l) q[m] = (l == 0) ? T(1) : T(2 * l - 1) * q1[l - 1];
            else if (m == l - 1) q[m] = T(2 * l - 1) * z * q1[m];
            else q[m] = (T(2 * l - 1) * z * q1[m] - T(l + m - 1) * q2[m]) * (T(1) / T(l - m));  // l, m unrolled: a constant
        }
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            if (m > l) continue;
            T k = ylm_k<T>(geo, l, m);
            if (m == 0) Y[l * l + l] = k * q[0];
            else {
                Y[l * l + l + m] = k * q[m] * C[m];
                Y[l * l + l - m] = k * q[m] * S[m];
            }
        }
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            if (m > l) continue;
            q2[m] = q1[m];
            q1[m] = q[m];
        }
    }
}

// ---------------------------------------------------- radial lookup (Hermite)
// R_nl(r) = f_cut(r) I_nl(r) and dR/dr from the cubic Hermite interpolant of
// the FP64 table (values and derivatives at the knots).
template <typename T>
__device__ __forceinline__ T fcut_dev(T r, T rc, T d, T *df)
{
    if (r >= rc) { *df = T(0); return T(0); }
    if (r < rc - d) { *df = T(0); return T(1); }
    const T pi = T(3.14159265358979323846);
    T t = pi * (r - rc + d) / d;
    T s, c;
    if (sizeof(T) == 8) { s = sin(t); c = cos(t); }
    else { s = sinf(float(t)); c = cosf(float(t)); }
    *df = T(-0.5) * s * pi / d;
    return T(0.5) * (c + T(1));
}

// Radial lookup.  The table holds, for every interval k of the uniform knot
// grid r_k = k h and every (n, l), the coefficients (a0, a1, a2, a3) of the
// cubic Hermite interpolant in u = r/h - k, computed in FP64 from the knot
// values and derivatives: I = a0 + u (a1 + u (a2 + u a3)),
// dI/dr = (a1 + u (2 a2 + 3 u a3)) / h.  Evaluating the polynomial instead of
// the Hermite basis avoids the (f_{k+1} - f_k)/h cancellation that would
// amplify the rounding of an FP32 table by 1/h.
template <typename T> struct Coef4;
template <> struct Coef4<float> { typedef float4 type; };
template <> struct Coef4<double> { typedef D4 type; };

template <typename T> struct RadialPos {
    int k;
    T u;
};

template <typename T>
__device__ __forceinline__ RadialPos<T> radial_pos(T r, T inv_h, int G)
{
    RadialPos<T> p;
    T t = r * inv_h;
    int kk = (int)t;
    if (kk > G - 1) kk = G - 1;
    if (kk < 0) kk = 0;
    p.k = kk;
    p.u = t - T(kk);
    return p;
}

// value and d/dr of entry q (= n (l_max+1) + l) at position p; NL entries per interval
template <typename T>
__device__ __forceinline__ void radial_eval(const T *__restrict__ tab, int NL, int q, RadialPos<T> p, T inv_h, T &v,
                                            T &dv)
{
    typename Coef4<T>::type c = reinterpret_cast<const typename Coef4<T>::type *>(tab)[(size_t)p.k * NL + q];
    T u = p.u;
    v = c.x + u * (c.y + u * (c.z + u * c.w));
    dv = (c.y + u * (T(2) * c.z + T(3) * u * c.w)) * inv_h;
}

template <typename T>
__device__ __forceinline__ T radial_value(const T *__restrict__ tab, int NL, int q, RadialPos<T> p)
{
    typename Coef4<T>::type c = reinterpret_cast<const typename Coef4<T>::type *>(tab)[(size_t)p.k * NL + q];
    T u = p.u;
    return c.x + u * (c.y + u * (c.z + u * c.w));
}
