// Rows of L_hat K_NM for fitting (text after Eq. 4): per configuration c one
// energy row  K_E[c][m] = sum_{i in c} delta^2 (p_hat_i . x_m)^zeta  and per
// atom j, direction a one force row
//   K_F[(j,a)][m] = -sum_i d k(p_hat_i, x_m) / d r_ja
//                 = sum_i W'_im x_m . (d p_hat_i / d r_ia) [i == j] - (d p_hat_i / d r_ja)
// with W'_im = zeta delta^2 (p_hat_i . x_m)^(zeta-1).  Writing J_p = d p_hat_i / d r_ij
// for pair p = (i -> j), the row of target j collects one "own" row
// S_j = sum_{p of j} J_p (scaled by +W'_j) and one "incoming" row per pair
// q = (i -> j) (scaled by -W'_i): 1 + n_j rows per (j, a), laid out
// contiguously (target-major), so every K_F entry is a segmented row sum of
// one GEMM [3 (N + P)] x D x M against the sparse points.
#include "gap_internal.h"
#include "knm.h"

namespace {

template <typename T> struct V4;
template <> struct V4<double> { typedef D4 type; };
template <> struct V4<float> { typedef float4 type; };

template <typename T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T> __device__ __forceinline__ T waccT(const SoapGeom &g, int grp, int z);
template <> __device__ __forceinline__ double waccT<double>(const SoapGeom &g, int grp, int z)
{
    return g.wacc64[grp * GAP_MAX_SPECIES + z];
}
template <> __device__ __forceinline__ float waccT<float>(const SoapGeom &g, int grp, int z)
{
    return g.wacc32[grp * GAP_MAX_SPECIES + z];
}

// Segment tables: segment sigma = 3 j + a holds rows [seg_start[sigma], seg_start[sigma+1])
// and lands in row out_row[sigma] = cfg(j) + 1 + 3 j + a of K_NM.
__global__ void k_seg_tables(int n, const int *__restrict__ offsets, const int *__restrict__ atom_cfg,
                             int *__restrict__ seg_start, int *__restrict__ out_row)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int nj = offsets[j + 1] - offsets[j];
    int base = 3 * (j + offsets[j]);
    for (int a = 0; a < 3; ++a) {
        seg_start[3 * j + a] = base + a * (1 + nj);
        out_row[3 * j + a] = atom_cfg[j] + 1 + 3 * j + a;
    }
    if (j == n - 1) seg_start[3 * n] = 3 * (n + offsets[n]);
}

// Jacobian rows: one warp per source atom i.  For each pair p = (i -> j)
// the warp builds d c / d r_ij, d p / d r_ij and J_p = (dp - p_hat (p_hat . dp)) / |p|
// and writes its three rows into target j's segments; the sum S_i of all J_p
// becomes atom i's own rows.  SPLIT: rows as BF16 hi + lo and t_row = J . mu
// (mu of atom i's GP); otherwise rows in T.
// Shared memory of k_jacobian_rows, in elements: A/B ([channels][l] quads)
// and the coefficients, rounded to whole quads; then Y_lm, its gradient,
// R_nl, dR_nl, Q_l^m and (C_m, S_m), rounded to whole quads (the rows after
// them are read as float4).
__host__ __device__ constexpr int jac_ab_words(int N, int L, int GA)
{
    return (4 * GA * N * (L + 1) + GA * N * (L + 1) * (L + 1) + 3) / 4 * 4;
}
__host__ __device__ constexpr int jac_head_words(int N, int L, int GA)
{
    return (jac_ab_words(N, L, GA) + 4 * (L + 1) * (L + 1) + 2 * N * (L + 1) + (L + 2) * (L + 2) + 2 * (L + 1) + 3) /
           4 * 4;
}

template <int N, int L, int GA, typename T, bool SPLIT>
__global__ void __launch_bounds__(32)
k_jacobian_rows(SoapGeom geo, const T *__restrict__ tab, int n_atoms, const int *__restrict__ offsets,
                const int *__restrict__ nbr_j, const int *__restrict__ rev,
                const typename V4<T>::type *__restrict__ vec, const int *__restrict__ species,
                const T *__restrict__ coef, const T *__restrict__ phat, const T *__restrict__ pnorm,
                const int *__restrict__ gp_of_atom, const float *__restrict__ mu_all, T *__restrict__ A,
                __nv_bfloat16 *__restrict__ Ahi, __nv_bfloat16 *__restrict__ Alo, __nv_bfloat16 *__restrict__ Amid,
                float *__restrict__ t_row, int *__restrict__ src_sign, int *__restrict__ seg)
{
    constexpr int LM = (L + 1) * (L + 1), NL = N * (L + 1), NC = GA * N * LM;
    typedef typename V4<T>::type V4T;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int D = geo.D, D16 = geo.D16;
    // per channel and l: A = sum_m Y_lm c_{g n lm}, B = sum_m grad Y_lm c_{g n lm}
    // (packed as (A, Bx, By, Bz)); then the coefficients c
    constexpr int NAB = GA * N * (L + 1);
    constexpr int kAB = jac_ab_words(N, L, GA);
    V4T *AB = reinterpret_cast<V4T *>(smem_raw);        // [NAB]
    T *csm = reinterpret_cast<T *>(AB + NAB);           // [NC]
    T *Ysm = reinterpret_cast<T *>(smem_raw) + kAB;     // [LM]
    T *dYsm = Ysm + LM;                          // [LM][3]
    T *Rsm = dYsm + 3 * LM;                      // [NL]
    T *dRsm = Rsm + NL;                          // [NL]
    T *Qsm = dRsm + NL;                          // [(L+2)][(L+2)]  Q_l^m
    T *CSsm = Qsm + (L + 2) * (L + 2);           // [L+1][2] (C_m, S_m)
    // rows staged direction-major, [3][D16] (entries D .. D16 - 1 zero), so
    // that a lane's eight consecutive entries are two vector loads; first
    // the row being built, then (one channel group with D > 256) the own
    // rows' sums, then p_hat
    constexpr int kHead = jac_head_words(N, L, GA);
    T *Jsm = reinterpret_cast<T *>(smem_raw) + kHead;
    // own-row accumulator: in registers (lane-owned entries d = lane + 32 k)
    // for one channel group and D <= 256, else shared memory [D][3]
    constexpr int DREG = N * (N + 1) / 2 * (L + 1);
    constexpr bool SREG = GA == 1 && DREG <= 256;
    constexpr int SK = SREG ? (DREG + 31) / 32 : 1;
    T sreg[SK][3];
    T *Ssm = Jsm + 3 * D16;                      // [3][D16] (when !SREG)
    T *psm = SREG ? Ssm : Ssm + 3 * D16;         // [D] p_hat
    const int lane = threadIdx.x;
    const int i = blockIdx.x;
    if (i >= n_atoms) return;
    for (int q = lane; q < NC; q += 32) csm[q] = coef[(size_t)i * NC + q];
    for (int d = lane; d < D; d += 32) {
        psm[d] = phat[(size_t)i * D + d];
        if (!SREG) Ssm[d] = Ssm[D16 + d] = Ssm[2 * D16 + d] = T(0);
    }
    for (int d = D + lane; d < D16; d += 32)
        for (int a = 0; a < 3; ++a) {
            Jsm[a * D16 + d] = T(0);
            if (!SREG) Ssm[a * D16 + d] = T(0);
        }
#pragma unroll
    for (int k = 0; k < SK; ++k) sreg[k][0] = sreg[k][1] = sreg[k][2] = T(0);
    const T inv_norm = T(1) / pnorm[i];
    const int gp = gp_of_atom ? gp_of_atom[i] : -1;
    const float *mu = (SPLIT && gp >= 0) ? mu_all + (size_t)gp * D16 : nullptr;
    const int p0 = offsets[i], p1 = offsets[i + 1];
    const T rc = (T)geo.rc, dw = (T)geo.d, inv_h = T(1) / (T)geo.h;
    __syncwarp();

    auto write_rows = [&](const T *Jv, int row_base, int stride, int sgn, int seg0) {
        // three rows row_base + a * stride, a = 0..2
        for (int a = 0; a < 3; ++a) {
            size_t row = (size_t)row_base + (size_t)a * stride;
            float t = 0.f;
            if constexpr (SPLIT) {
                // eight entries per lane: one 16-byte store per plane (D16 is
                // a multiple of 16, so every chunk is aligned and in the row)
                for (int d0 = 8 * lane; d0 < D16; d0 += 256) {
                    T jv[8];
                    *reinterpret_cast<float4 *>(jv) = *reinterpret_cast<const float4 *>(Jv + a * D16 + d0);
                    *reinterpret_cast<float4 *>(jv + 4) = *reinterpret_cast<const float4 *>(Jv + a * D16 + d0 + 4);
                    uint32_t hi[4], mid[4], lo[4];
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        float f2[2], r2[2], m2[2];
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const int d = d0 + u + k;
                            const float f = (float)jv[u + k];
                            const __nv_bfloat16 hb = __float2bfloat16_rn(f);
                            float rest = f - __bfloat162float(hb);
                            f2[k] = __bfloat162float(hb);
                            if (Amid) {
                                const __nv_bfloat16 mb = __float2bfloat16_rn(rest);
                                m2[k] = __bfloat162float(mb);
                                rest -= m2[k];
                            } else {
                                m2[k] = 0.f;
                            }
                            r2[k] = rest;
                            if (mu) t += f * mu[d];
                        }
                        __nv_bfloat162 h = __floats2bfloat162_rn(f2[0], f2[1]);
                        __nv_bfloat162 mm = __floats2bfloat162_rn(m2[0], m2[1]);
                        __nv_bfloat162 l2 = __floats2bfloat162_rn(r2[0], r2[1]);
                        hi[u / 2] = *reinterpret_cast<uint32_t *>(&h);
                        mid[u / 2] = *reinterpret_cast<uint32_t *>(&mm);
                        lo[u / 2] = *reinterpret_cast<uint32_t *>(&l2);
                    }
                    *reinterpret_cast<uint4 *>(Ahi + row * D16 + d0) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4 *>(Alo + row * D16 + d0) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                    if (Amid)
                        *reinterpret_cast<uint4 *>(Amid + row * D16 + d0) = make_uint4(mid[0], mid[1], mid[2], mid[3]);
                }
            } else {
                for (int d = lane; d < D16; d += 32) A[row * D16 + d] = Jv[a * D16 + d];
            }
            if (SPLIT) {
                t = warp_sum(t);
                if (lane == 0) t_row[row] = t;
            }
            if (lane == 0) {
                src_sign[row] = sgn;
                seg[row] = seg0 + a;
            }
        }
    };

    for (int p = p0; p < p1; ++p) {
        typename V4<T>::type v = vec[p];
        const T r = v.w, ir = T(1) / r;
        const T ux = v.x * ir, uy = v.y * ir, uz = v.z * ir;
        const int j = nbr_j[p], zr = species[j], z = zr >= 0 && zr < geo.S ? zr : 0;  // out of range: the call fails
        // Q_l^m columns and (x + iy)^m, one lane per m
        if (lane <= L) {
            int m = lane;
            T C = T(1), S = T(0);
            for (int k = 0; k < m; ++k) {
                T c2 = ux * C - uy * S;
                S = ux * S + uy * C;
                C = c2;
            }
            CSsm[2 * m] = C;
            CSsm[2 * m + 1] = S;
            T q2 = T(0), q1 = T(1);  // Q_m^m = (2m-1)!!
            for (int k = 1; k <= m; ++k) q1 *= T(2 * k - 1);
            for (int l = 0; l <= L + 1; ++l) Qsm[l * (L + 2) + m] = T(0);
            Qsm[m * (L + 2) + m] = q1;
            if (m + 1 <= L) {
                T qq = T(2 * m + 1) * uz * q1;
                Qsm[(m + 1) * (L + 2) + m] = qq;
                q2 = q1;
                q1 = qq;
                // over k = l - m (unrolled, so 1 / k is a constant)
#pragma unroll
                for (int k = 2; k <= L; ++k) {
                    if (k <= L - m) {
                        const int l = m + k;
                        T qn = (T(2 * l - 1) * uz * q1 - T(l + m - 1) * q2) * (T(1) / T(k));
                        Qsm[l * (L + 2) + m] = qn;
                        q2 = q1;
                        q1 = qn;
                    }
                }
            }
        }
        if (lane == L + 1)
            for (int l = 0; l <= L + 1; ++l) Qsm[l * (L + 2) + L + 1] = T(0);
        // radial functions and derivatives
        T df;
        const T f = fcut_dev<T>(r, rc, dw, &df);
        const RadialPos<T> rp = radial_pos<T>(r, inv_h, geo.G);
        for (int q = lane; q < NL; q += 32) {
            T I, dI;
            radial_eval<T>(tab, NL, q, rp, inv_h, I, dI);
            Rsm[q] = f * I;
            dRsm[q] = df * I + f * dI;
        }
        __syncwarp();
        // Y_lm and its gradient with respect to r_ij
        for (int lm = lane; lm < LM; lm += 32) {
            const int l = (int)sqrtf((float)lm + 0.5f);  // floor(sqrt(lm)), lm < 121
            int m = lm - l * l - l, am = m < 0 ? -m : m;
            T k = ylm_k<T>(geo, l, am);
            T qv = Qsm[l * (L + 2) + am], qd = Qsm[l * (L + 2) + am + 1];
            T y, gx, gy, gz;
            if (am == 0) {
                y = k * qv; gx = T(0); gy = T(0); gz = k * qd;
            } else {
                T C = CSsm[2 * am], S = CSsm[2 * am + 1], Cm = CSsm[2 * (am - 1)], Sm = CSsm[2 * (am - 1) + 1];
                if (m > 0) {
                    y = k * qv * C; gx = k * qv * T(am) * Cm; gy = -k * qv * T(am) * Sm; gz = k * qd * C;
                } else {
                    y = k * qv * S; gx = k * qv * T(am) * Sm; gy = k * qv * T(am) * Cm; gz = k * qd * S;
                }
            }
            T ud = ux * gx + uy * gy + uz * gz;
            Ysm[lm] = y;
            dYsm[3 * lm] = (gx - ud * ux) * ir;
            dYsm[3 * lm + 1] = (gy - ud * uy) * ir;
            dYsm[3 * lm + 2] = (gz - ud * uz) * ir;
        }
        __syncwarp();
        // The pair's derivative of a coefficient is separable,
        //   d c^g_{n lm} / d r_ij = w_{g z} (dR_nl u Y_lm + R_nl grad Y_lm),
        // so the m-sums of d p / d r_ij reduce to A = sum_m Y_lm c and
        // B = sum_m grad Y_lm c per channel and l.
        for (int q = lane; q < NAB; q += 32) {
            const int l = q % (L + 1), gn = q / (L + 1);
            const T *cc = csm + gn * LM + l * l;
            const T *yy = Ysm + l * l, *dy = dYsm + 3 * l * l;
            T a = T(0), bx = T(0), by = T(0), bz = T(0);
            for (int m = 0; m <= 2 * l; ++m) {
                const T c = cc[m];
                a += yy[m] * c;
                bx += dy[3 * m] * c;
                by += dy[3 * m + 1] * c;
                bz += dy[3 * m + 2] * c;
            }
            V4T v;
            v.x = a; v.y = bx; v.z = by; v.w = bz;
            AB[q] = v;
        }
        __syncwarp();
        // d p / d r_ij per entry (a, a', l):
        //   w_a (dR_a u A_a' + R_a B_a') + w_a' (dR_a' u A_a + R_a' B_a),
        // then its projection
        T pd0 = T(0), pd1 = T(0), pd2 = T(0);
        for (int k = lane; k < D; k += 32) {
            const int4 e = __ldg(geo.dtab + k);
            const int d = e.x, l = e.w & 0xff;
            const bool cross = (e.w >> 8) != 0;  // a != a': the pair counts twice
            const int gn1 = (e.y - l * l) / LM, gn2 = (e.z - l * l) / LM;
            const int n1 = gn1 % N, n2 = gn2 % N;
            const T w1 = waccT<T>(geo, gn1 / N, z), w2 = waccT<T>(geo, gn2 / N, z);
            const T f1 = w1 * dRsm[n1 * (L + 1) + l], f2 = w2 * dRsm[n2 * (L + 1) + l];
            const T h1 = w1 * Rsm[n1 * (L + 1) + l], h2 = w2 * Rsm[n2 * (L + 1) + l];
            const V4T a1 = AB[gn1 * (L + 1) + l], a2 = AB[gn2 * (L + 1) + l];
            const T cu = f1 * a2.x + f2 * a1.x;
            T s0 = cu * ux + h1 * a2.y + h2 * a1.y;
            T s1 = cu * uy + h1 * a2.z + h2 * a1.z;
            T s2 = cu * uz + h1 * a2.w + h2 * a1.w;
            T sc = cross ? T(1.41421356237309504880) : T(1);
            s0 *= sc; s1 *= sc; s2 *= sc;
            Jsm[d] = s0; Jsm[D16 + d] = s1; Jsm[2 * D16 + d] = s2;
            pd0 += psm[d] * s0; pd1 += psm[d] * s1; pd2 += psm[d] * s2;
        }
        pd0 = warp_sum(pd0); pd1 = warp_sum(pd1); pd2 = warp_sum(pd2);
        __syncwarp();  // Jsm entries were written by other lanes
        if constexpr (SREG) {
#pragma unroll
            for (int k = 0; k < SK; ++k) {
                const int d = lane + 32 * k;
                if (d < D) {
                    T pv = psm[d];
                    T j0 = (Jsm[d] - pv * pd0) * inv_norm, j1 = (Jsm[D16 + d] - pv * pd1) * inv_norm,
                      j2 = (Jsm[2 * D16 + d] - pv * pd2) * inv_norm;
                    Jsm[d] = j0; Jsm[D16 + d] = j1; Jsm[2 * D16 + d] = j2;
                    sreg[k][0] += j0; sreg[k][1] += j1; sreg[k][2] += j2;
                }
            }
        } else {
            for (int d = lane; d < D; d += 32) {
                T pv = psm[d];
                T j0 = (Jsm[d] - pv * pd0) * inv_norm, j1 = (Jsm[D16 + d] - pv * pd1) * inv_norm,
                  j2 = (Jsm[2 * D16 + d] - pv * pd2) * inv_norm;
                Jsm[d] = j0; Jsm[D16 + d] = j1; Jsm[2 * D16 + d] = j2;
                Ssm[d] += j0; Ssm[D16 + d] += j1; Ssm[2 * D16 + d] += j2;
            }
        }
        __syncwarp();
        const int nj = offsets[j + 1] - offsets[j];
        const int slot = rev[p] - offsets[j];
        write_rows(Jsm, 3 * (j + offsets[j]) + 1 + slot, 1 + nj, -(i + 1), 3 * j);
        __syncwarp();
    }
    if constexpr (SREG) {
        // the own rows from the registers: lane-owned entries into Jsm first
        __syncwarp();
#pragma unroll
        for (int k = 0; k < SK; ++k) {
            const int d = lane + 32 * k;
            if (d < D) { Jsm[d] = sreg[k][0]; Jsm[D16 + d] = sreg[k][1]; Jsm[2 * D16 + d] = sreg[k][2]; }
        }
        __syncwarp();
        write_rows(Jsm, 3 * (i + offsets[i]), 1 + (p1 - p0), i + 1, 3 * i);
    } else {
        write_rows(Ssm, 3 * (i + offsets[i]), 1 + (p1 - p0), i + 1, 3 * i);
    }
}

// ----------------------------------------------------- CUDA-core forms
constexpr int TK = 16;  // K step of the CUDA-core tiles

// Wp[atom][m] = zeta d2 q^(zeta-1), kq[atom][m] = d2 q^zeta for the atoms of one GP.
template <typename T>
__global__ void __launch_bounds__(256)
k_simt_qpow(const T *__restrict__ phat, int D, const int *__restrict__ rows, int nrows, const T *__restrict__ X,
            int M, T d2, int zeta, T *__restrict__ Wp, T *__restrict__ kq, int ld)
{
    __shared__ T As[TK][64 + 1], Bs[TK][64 + 1];
    const int r0 = blockIdx.y * 64, m0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < D; k0 += TK) {
        for (int e = threadIdx.x; e < TK * 64; e += 256) {
            int kk = e % TK, rr = e / TK;
            int r = r0 + rr, k = k0 + kk, m = m0 + rr;
            As[kk][rr] = (r < nrows && k < D) ? phat[(size_t)rows[r] * D + k] : T(0);
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
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int r = r0 + ty * 4 + u;
        if (r >= nrows) continue;
        int atom = rows[r];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int m = m0 + tx * 4 + v;
            if (m >= M) continue;
            T q = acc[u][v], qz = T(1);
            for (int z = 1; z < zeta; ++z) qz *= q;
            Wp[(size_t)atom * ld + m] = T(zeta) * d2 * qz;
            kq[(size_t)atom * ld + m] = d2 * qz * q;
        }
    }
}

// Force rows on CUDA cores: 64 x 64 tiles of T = J X^T (K-loop over D), each
// entry scaled by sign W'[src][m], then the rows of every (target, xyz)
// segment summed in shared memory; segments cut by the tile edge leave
// partial sums in P[tile][slot] for the fix-up pass (as in the tensor-core form).
template <typename T>
__global__ void __launch_bounds__(256)
k_simt_knm(const T *__restrict__ A, int D, int D16, long nrow, const int *__restrict__ seg,
           const int *__restrict__ seg_start, const int *__restrict__ out_row, const int *__restrict__ src_sign,
           const T *__restrict__ X, int M, const T *__restrict__ Wp, int ldw, double *__restrict__ K, int ldk,
           int col_out0, T *__restrict__ P, int ldp)
{
    __shared__ T As[TK][64 + 1], Bs[TK][64 + 1];
    __shared__ T red[64][64 + 1];
    __shared__ int starts[65];
    __shared__ int nstart;
    const int m0 = blockIdx.x * 64;
    const long ntiles = (nrow + 63) / 64;
    for (long tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const long r0 = tile * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int nvalid = (int)(nrow - r0 < 64 ? nrow - r0 : 64);
    T acc[4][4] = {};
    for (int k0 = 0; k0 < D; k0 += TK) {
        for (int e = threadIdx.x; e < TK * 64; e += 256) {
            int kk = e % TK, rr = e / TK;
            long row = r0 + rr;
            int m = m0 + rr, k = k0 + kk;
            As[kk][rr] = (rr < nvalid && k < D) ? A[row * D16 + k] : T(0);
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
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int rl = ty * 4 + u;
        int ss = rl < nvalid ? src_sign[r0 + rl] : 0;
        int src = (ss > 0 ? ss : -ss) - 1;
        T sg = ss > 0 ? T(1) : T(-1);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int m = m0 + tx * 4 + v;
            red[rl][tx * 4 + v] = (ss != 0 && m < M) ? sg * Wp[(size_t)src * ldw + m] * acc[u][v] : T(0);
        }
    }
    if (threadIdx.x == 0) {
        int ns = 0;
        for (int rl = 0; rl < nvalid; ++rl)
            if (rl == 0 || seg[r0 + rl] != seg[r0 + rl - 1]) starts[ns++] = rl;
        starts[ns] = nvalid;
        nstart = ns;
    }
    __syncthreads();
    for (int item = threadIdx.x; item < nstart * 64; item += 256) {
        int k = item / 64, c = item % 64, m = m0 + c;
        if (m >= M) continue;
        int s0 = starts[k], s1 = starts[k + 1];
        T sum = T(0);
        for (int rl = s0; rl < s1; ++rl) sum += red[rl][c];
        int sigma = seg[r0 + s0];
        long g0 = seg_start[sigma], g1 = seg_start[sigma + 1];
        if (g0 >= r0 && g1 <= r0 + 64) K[(size_t)out_row[sigma] * ldk + col_out0 + m] = (double)sum;
        else P[((size_t)tile * 2 + (s0 == 0 ? 0 : 1)) * ldp + m] = sum;
    }
    __syncthreads();
    }
}

// Energy rows: K[row_E(c)][col] = sum_{i in c} kq[i][m] (block per configuration).
template <typename T>
__global__ void k_knm_energy(const int *__restrict__ cfg_off, const T *__restrict__ kq, int ld, int M,
                             double *__restrict__ K, int ldk, int col_out0)
{
    int c = blockIdx.y;
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int i0 = cfg_off[c], i1 = cfg_off[c + 1];
    double s = 0.0;
    int i = i0;
    // four loads in flight; FP32 terms summed in fours before the FP64 sum
    // (GB300's FP64 adds are the scarce unit)
    for (; i + 4 <= i1; i += 4) {
        const T a = kq[(size_t)i * ld + m], b = kq[(size_t)(i + 1) * ld + m];
        const T e = kq[(size_t)(i + 2) * ld + m], f = kq[(size_t)(i + 3) * ld + m];
        s += (double)((a + b) + (e + f));
    }
    for (; i < i1; ++i) s += (double)kq[(size_t)i * ld + m];
    K[(size_t)(c + 3 * i0) * ldk + col_out0 + m] = s;
}

// Segments cut by a tile edge (tile height TH rows): sum the partials of the tiles they span.
template <typename T>
__global__ void k_knm_fixup(int n_seg, const int *__restrict__ seg_start, const int *__restrict__ out_row,
                            const T *__restrict__ P, int ldp, int M, double *__restrict__ K, int ldk, int col_out0,
                            int TH)
{
    int sigma = blockIdx.x;
    int m = blockIdx.y * blockDim.x + threadIdx.x;
    if (sigma >= n_seg || m >= M) return;
    long g0 = seg_start[sigma], g1 = seg_start[sigma + 1];
    long t0 = g0 / TH, t1 = (g1 - 1) / TH;
    if (t0 == t1) return;
    double s = (double)P[((size_t)t0 * 2 + (g0 % TH == 0 ? 0 : 1)) * ldp + m];
    for (long t = t0 + 1; t <= t1; ++t) s += (double)P[((size_t)t * 2) * ldp + m];
    K[(size_t)out_row[sigma] * ldk + col_out0 + m] = s;
}

}  // namespace

namespace {
__global__ void k_knm_dest(long nrow, const int *__restrict__ seg, const int *__restrict__ seg_start,
                           const int *__restrict__ out_row, int *__restrict__ dest)
{
    const long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (r >= nrow) return;
    const long t0 = r - r % 128;
    const int sg = seg[r];
    dest[r] = (seg_start[sg] >= t0 && seg_start[sg + 1] <= t0 + 128) ? out_row[sg] : -1 - (r == t0 ? 0 : 1);
}
}  // namespace

gap_status gap_knm_dest(long nrow, const int *seg, const int *seg_start, const int *out_row, int *dest,
                        cudaStream_t st)
{
    if (nrow <= 0) return GAP_OK;
    gap_count_launch();
    k_knm_dest<<<(unsigned)((nrow + 255) / 256), 256, 0, st>>>(nrow, seg, seg_start, out_row, dest);
    return gap_cuda_status(cudaGetLastError(), "k_knm_dest");
}

gap_status gap_knm_segments(int n, const int *offsets, const int *atom_cfg, int *seg_start, int *out_row,
                            cudaStream_t st)
{
    if (n == 0) return GAP_OK;
    gap_count_launch();
    k_seg_tables<<<(n + 127) / 128, 128, 0, st>>>(n, offsets, atom_cfg, seg_start, out_row);
    return gap_cuda_status(cudaGetLastError(), "k_seg_tables");
}

template <typename T, bool SPLIT>
struct JacLaunch {
    template <int N, int L, int GA>
    static gap_status run(const SoapGeom &g, const T *tab, int n, const PairList &pl, const int *species,
                          const T *coef, const T *phat, const T *pnorm, const int *gp_of_atom, const float *mu_all,
                          KnmRows &out, cudaStream_t st)
    {
        constexpr bool SREG = GA == 1 && N * (N + 1) / 2 * (L + 1) <= 256;  // as in the kernel
        if (SREG && g.D != N * (N + 1) / 2 * (L + 1)) {
            gap_set_error("Jacobian rows: descriptor size does not match its shape");
            return GAP_EINVAL;
        }
        constexpr int kHead = jac_head_words(N, L, GA);
        size_t shm = sizeof(T) * (kHead + (SREG ? 3 : 6) * (size_t)g.D16 + g.D);
        if (shm > 227 * 1024) {
            gap_set_error("descriptor too large for the Jacobian-row kernel's shared memory");
            return GAP_EUNSUPPORTED;
        }
        auto kern = k_jacobian_rows<N, L, GA, T, SPLIT>;
        GAP_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        const typename V4<T>::type *vec;
        if constexpr (sizeof(T) == 8) vec = pl.vec64; else vec = pl.vec32;
        gap_count_launch();
        kern<<<n, 32, shm, st>>>(g, tab, n, pl.offsets, pl.j, pl.rev, vec, species, coef, phat, pnorm, gp_of_atom,
                                 mu_all, reinterpret_cast<T *>(out.A), out.A_hi, out.A_lo, out.A_mid, out.t_row,
                                 out.src_sign, out.seg);
        return gap_cuda_status(cudaGetLastError(), "k_jacobian_rows");
    }
};

#define GAP_KNM_SHAPES(X) \
    X(2, 1, 1)            \
    X(4, 3, 1)            \
    X(4, 3, 2)            \
    X(4, 3, 4)            \
    X(6, 4, 1)            \
    X(6, 6, 1)            \
    X(8, 4, 1)            \
    X(8, 6, 1)            \
    X(8, 4, 5)            \
    X(8, 6, 4)            \
    X(8, 8, 1)            \
    X(10, 8, 1)

template <typename T, bool SPLIT>
gap_status gap_jacobian_rows(const SoapGeom &g, const T *tab, int n, const PairList &pl, const int *species,
                             const T *coef, const T *phat, const T *pnorm, const int *gp_of_atom, const float *mu_all,
                             KnmRows &out, cudaStream_t st)
{
    if (n == 0) return GAP_OK;
#define X(nn, ll, ga) \
    if (g.N == nn && g.L == ll && g.GA == ga) \
        return JacLaunch<T, SPLIT>::template run<nn, ll, ga>(g, tab, n, pl, species, coef, phat, pnorm, gp_of_atom, mu_all, out, st);
    GAP_KNM_SHAPES(X)
#undef X
    gap_set_error("unsupported (n_max, l_max, groups) for K_NM rows");
    return GAP_EUNSUPPORTED;
}

template gap_status gap_jacobian_rows<double, false>(const SoapGeom &, const double *, int, const PairList &,
                                                     const int *, const double *, const double *, const double *,
                                                     const int *, const float *, KnmRows &, cudaStream_t);
template gap_status gap_jacobian_rows<float, false>(const SoapGeom &, const float *, int, const PairList &,
                                                    const int *, const float *, const float *, const float *,
                                                    const int *, const float *, KnmRows &, cudaStream_t);
template gap_status gap_jacobian_rows<float, true>(const SoapGeom &, const float *, int, const PairList &,
                                                   const int *, const float *, const float *, const float *,
                                                   const int *, const float *, KnmRows &, cudaStream_t);

template <typename T>
gap_status gap_knm_qpow_simt(const T *phat, int D, const int *rows, int nrows, const T *X, int M, double delta,
                             int zeta, T *Wp, T *kq, int ld, cudaStream_t st)
{
    if (nrows <= 0 || M <= 0) return GAP_OK;
    dim3 grid((M + 63) / 64, (nrows + 63) / 64);
    gap_count_launch();
    k_simt_qpow<T><<<grid, 256, 0, st>>>(phat, D, rows, nrows, X, M, (T)(delta * delta), zeta, Wp, kq, ld);
    return gap_cuda_status(cudaGetLastError(), "k_simt_qpow");
}

template <typename T>
gap_status gap_knm_force_simt(const T *A, int D, int D16, long nrow, const int *seg, int n_seg, const int *seg_start,
                              const int *out_row, const int *src_sign, const T *X, int M, const T *Wp, int ldw,
                              double *K, int ldk, int col_out0, T *P, int ldp, cudaStream_t st)
{
    if (nrow <= 0 || M <= 0) return GAP_OK;
    long ntiles = (nrow + 63) / 64;
    dim3 grid((M + 63) / 64, (unsigned)(ntiles < 65535 ? ntiles : 65535));
    gap_count_launch();
    k_simt_knm<T><<<grid, 256, 0, st>>>(A, D, D16, nrow, seg, seg_start, out_row, src_sign, X, M, Wp, ldw, K, ldk,
                                         col_out0, P, ldp);
    GAP_TRY_CUDA(cudaGetLastError());
    dim3 g2(n_seg, (M + 127) / 128);
    gap_count_launch();
    k_knm_fixup<T><<<g2, 128, 0, st>>>(n_seg, seg_start, out_row, P, ldp, M, K, ldk, col_out0, 64);
    return gap_cuda_status(cudaGetLastError(), "k_knm_fixup");
}

template <typename T>
gap_status gap_knm_energy(int n_configs, const int *cfg_off, const T *kq, int ld, int M, double *K, int ldk,
                          int col_out0, cudaStream_t st)
{
    if (n_configs <= 0 || M <= 0) return GAP_OK;
    dim3 grid((M + 127) / 128, n_configs);
    gap_count_launch();
    k_knm_energy<T><<<grid, 128, 0, st>>>(cfg_off, kq, ld, M, K, ldk, col_out0);
    return gap_cuda_status(cudaGetLastError(), "k_knm_energy");
}

namespace {
// Cut segments of the 128-row tensor-core tiles: a tile originates at most
// one, its last segment when that runs past the tile's end (slot 0 of P if
// it starts at the tile's first row, else slot 1); every later tile it
// covers holds its next partial in slot 0.
// A block takes kFixTiles tiles and 128 columns: its first threads decode the
// tiles' last segments at once, then every thread sums the cut ones.
constexpr int kFixTiles = 64;
__global__ void __launch_bounds__(128) k_knm_fixup_tiles(long nrow, const int *__restrict__ seg,
                                                         const int *__restrict__ seg_start,
                                                         const int *__restrict__ out_row, const float *__restrict__ P,
                                                         int ldp, int M, double *__restrict__ K, int ldk,
                                                         int col_out0)
{
    __shared__ int cut_sg[kFixTiles];  // segment originated and cut by the tile, or -1
    __shared__ long cut_end[kFixTiles];
    __shared__ unsigned char cut_slot[kFixTiles];
    const long tiles = (nrow + 127) / 128;
    const long tb = (long)blockIdx.x * kFixTiles;
    if (threadIdx.x < kFixTiles) {
        const long t = tb + threadIdx.x;
        int sgc = -1;
        if (t < tiles) {
            const long t0 = t * 128, t1 = t0 + 128;
            const long last = (t1 < nrow ? t1 : nrow) - 1;
            const int sg = seg[last];
            const long g0 = seg_start[sg], g1 = seg_start[sg + 1];
            if (g1 > t1 && g0 >= t0) {  // runs past this tile and starts in it
                sgc = sg;
                cut_end[threadIdx.x] = g1;
                cut_slot[threadIdx.x] = g0 == t0 ? 0 : 1;
            }
        }
        cut_sg[threadIdx.x] = sgc;
    }
    __syncthreads();
    const int m = blockIdx.y * blockDim.x + threadIdx.x;
    if (m >= M) return;
    for (int k = 0; k < kFixTiles; ++k) {
        const int sg = cut_sg[k];
        if (sg < 0) continue;
        const long t = tb + k, g1 = cut_end[k];
        double s = (double)P[((size_t)t * 2 + cut_slot[k]) * ldp + m];
        for (long u = t + 1; u * 128 < g1; ++u) s += (double)P[((size_t)u * 2) * ldp + m];
        K[(size_t)out_row[sg] * ldk + col_out0 + m] = s;
    }
}
}  // namespace

gap_status gap_knm_fixup(long nrow, const int *seg, const int *seg_start, const int *out_row, const float *P, int ldp,
                         int M, double *K, int ldk, int col_out0, cudaStream_t st)
{
    if (nrow <= 0 || M <= 0) return GAP_OK;
    const long tiles = (nrow + 127) / 128;
    if (tiles > 2147483647L) {
        gap_set_error("K_NM fix-up: too many tiles");
        return GAP_EUNSUPPORTED;
    }
    dim3 grid((unsigned)((tiles + kFixTiles - 1) / kFixTiles), (M + 127) / 128);
    gap_count_launch();
    k_knm_fixup_tiles<<<grid, 128, 0, st>>>(nrow, seg, seg_start, out_row, P, ldp, M, K, ldk, col_out0);
    return gap_cuda_status(cudaGetLastError(), "k_knm_fixup_tiles");
}

#define INSTK(T)                                                                                                     \
    template gap_status gap_knm_qpow_simt<T>(const T *, int, const int *, int, const T *, int, double, int, T *, T *, \
                                             int, cudaStream_t);                                                    \
    template gap_status gap_knm_force_simt<T>(const T *, int, int, long, const int *, int, const int *, const int *,  \
                                              const int *, const T *, int, const T *, int, double *, int, int, T *,   \
                                              int, cudaStream_t);                                                    \
    template gap_status gap_knm_energy<T>(int, const int *, const T *, int, int, double *, int, int, cudaStream_t);
INSTK(double)
INSTK(float)

// ------------------------------------------------ compressed descriptors
// With p~ = Q p (Eq. 25) renormalised, d p_hat~ = (I - p_hat~ p_hat~^T) Q dp / |p~|.
// A Jacobian row J = d p_hat / d r = (I - p_hat p_hat^T) dp / |p| maps to
//   J~ = (|p| / |p~|) (I - p_hat~ p_hat~^T) Q J,
// because Q p_hat is parallel to p_hat~ and the projection removes it.  The
// rows keep their sources, segments and order, so the K_NM GEMM and its
// segment sums run unchanged on J~ against the compressed sparse points.
namespace {
// V = J Q^T on the CUDA cores: 64 x 64 output tiles, 16 x 16 threads with a
// 4 x 4 register block each, K in steps of 16 staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_rows_qt(long nrow, int D, const T *__restrict__ J, int ldj, int Dg,
                                                 const T *__restrict__ Q, T *__restrict__ V, int ldv)
{
    __shared__ T Js[16][65];
    __shared__ T Qs[16][65];
    const long r0 = (long)blockIdx.x * 64;
    const int o0 = blockIdx.y * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int k0 = 0; k0 < D; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int rr = e >> 4, kk = e & 15, k = k0 + kk;
            const long r = r0 + rr;
            const int o = o0 + rr;
            Js[kk][rr] = (r < nrow && k < D) ? J[r * ldj + k] : T(0);
            Qs[kk][rr] = (o < Dg && k < D) ? Q[(size_t)o * D + k] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = Js[kk][ty + 16 * u];
                b[u] = Qs[kk][tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const long r = r0 + ty + 16 * u;
        if (r >= nrow) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int o = o0 + tx + 16 * v;
            if (o < Dg) V[r * ldv + o] = acc[u][v];
        }
    }
}

// One warp per row: c = p_hat~ . v, J~ = s (v - c p_hat~) with s = |p| / |p~|
// of the row's source atom; entries Dg .. Dg16 - 1 written as zero.  V and
// A may be the same buffer (CUDA-core forms, ldv == Dg16): each lane reads
// its entries before the reduction and writes the same entries after it.
template <typename T, bool SPLIT>
__global__ void __launch_bounds__(256) k_jac_project(long nrow, int Dg, int Dg16, const T *V, int ldv,
                                                     const int *__restrict__ src_sign,
                                                     const int *__restrict__ gp_of_atom, const T *__restrict__ phatc,
                                                     const T *__restrict__ pnorm, const T *__restrict__ pnormc,
                                                     const float *__restrict__ mu_all, T *A,
                                                     __nv_bfloat16 *__restrict__ Ahi, __nv_bfloat16 *__restrict__ Alo,
                                                     __nv_bfloat16 *__restrict__ Amid, float *__restrict__ t_row)
{
    const long row = (long)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= nrow) return;
    const int sg = src_sign[row];
    const int i = (sg > 0 ? sg : -sg) - 1;
    const T *v = V + row * ldv;
    const T *ph = phatc + (size_t)i * Dg;
    T c = T(0);
    for (int o = lane; o < Dg; o += 32) c += v[o] * ph[o];
    c = warp_sum(c);
    const T s = pnorm[i] / pnormc[i];
    const int gp = gp_of_atom ? gp_of_atom[i] : -1;
    const float *mu = (SPLIT && gp >= 0) ? mu_all + (size_t)gp * Dg16 : nullptr;
    float t = 0.f;
    for (int o = lane; o < Dg16; o += 32) {
        const T x = o < Dg ? s * (v[o] - c * ph[o]) : T(0);
        if constexpr (SPLIT) {
            const float f = (float)x;
            const __nv_bfloat16 hb = __float2bfloat16_rn(f);
            float rest = f - __bfloat162float(hb);
            if (Amid) {
                const __nv_bfloat16 mb = __float2bfloat16_rn(rest);
                rest -= __bfloat162float(mb);
                Amid[row * Dg16 + o] = mb;
            }
            Ahi[row * Dg16 + o] = hb;
            Alo[row * Dg16 + o] = __float2bfloat16_rn(rest);
            if (mu) t += f * mu[o];
        } else {
            A[row * Dg16 + o] = x;
        }
    }
    if constexpr (SPLIT) {
        t = warp_sum(t);
        if (lane == 0) t_row[row] = t;
    }
}
}  // namespace

template <typename T>
gap_status gap_rows_times_qt(long nrow, int D, const T *J, int ldj, int Dg, const T *Q, T *V, int ldv,
                             cudaStream_t st)
{
    if (nrow <= 0 || Dg <= 0) return GAP_OK;
    const long tiles = (nrow + 63) / 64;
    if (tiles > 2147483647L) {
        gap_set_error("compressed Jacobian rows: too many tiles");
        return GAP_EUNSUPPORTED;
    }
    dim3 grid((unsigned)tiles, (Dg + 63) / 64);
    gap_count_launch();
    k_rows_qt<T><<<grid, 256, 0, st>>>(nrow, D, J, ldj, Dg, Q, V, ldv);
    return gap_cuda_status(cudaGetLastError(), "k_rows_qt");
}

template <typename T, bool SPLIT>
gap_status gap_jacobian_compress(long nrow, int Dg, int Dg16, const T *V, int ldv, const int *src_sign,
                                 const int *gp_of_atom, const T *phatc, const T *pnorm, const T *pnormc,
                                 const float *mu_all, KnmRows &out, cudaStream_t st)
{
    if (nrow <= 0) return GAP_OK;
    const long blocks = (nrow + 7) / 8;
    if (blocks > 2147483647L) {
        gap_set_error("compressed Jacobian rows: too many rows");
        return GAP_EUNSUPPORTED;
    }
    gap_count_launch();
    k_jac_project<T, SPLIT><<<(unsigned)blocks, 256, 0, st>>>(nrow, Dg, Dg16, V, ldv, src_sign, gp_of_atom, phatc,
                                                              pnorm, pnormc, mu_all, reinterpret_cast<T *>(out.A),
                                                              out.A_hi, out.A_lo, out.A_mid, out.t_row);
    return gap_cuda_status(cudaGetLastError(), "k_jac_project");
}

template gap_status gap_rows_times_qt<double>(long, int, const double *, int, int, const double *, double *, int,
                                              cudaStream_t);
template gap_status gap_rows_times_qt<float>(long, int, const float *, int, int, const float *, float *, int,
                                             cudaStream_t);
template gap_status gap_jacobian_compress<double, false>(long, int, int, const double *, int, const int *, const int *,
                                                         const double *, const double *, const double *,
                                                         const float *, KnmRows &, cudaStream_t);
template gap_status gap_jacobian_compress<float, false>(long, int, int, const float *, int, const int *, const int *,
                                                        const float *, const float *, const float *, const float *,
                                                        KnmRows &, cudaStream_t);
template gap_status gap_jacobian_compress<float, true>(long, int, int, const float *, int, const int *, const int *,
                                                       const float *, const float *, const float *, const float *,
                                                       KnmRows &, cudaStream_t);
