// SOAP expansion, power spectrum and its backward pass, per-pair forces.
//
//   expansion      c^g_{n lm} = sum_j wacc[g][Z_j] f_cut(r_ij) I_nl(r_ij) Y_lm(u_ij)
//                  + central term                                   (Eqs. 19-20, 25)
//   power spectrum p_{a a' l} = s_aa' sum_m c_{a lm} c_{a' lm}, p_hat = p / |p|
//                                                                   (Eqs. 22-24)
//   backward       h = (g - (g . p_hat) p_hat) / |p|, g = d eps / d p_hat;
//                  gamma_{a lm} = sum_a' H_{a a' l} c_{a' lm} with H = sqrt2 h off
//                  the diagonal and 2 h on it; Gamma^z_{n lm} = sum_g wacc[g][z] gamma
//   pair force     d eps_i / d r_ij = sum_lm Gamma^{Z_j}_{n lm} d(R_nl Y_lm)/d r_ij
//                  (Eq. 3 through the chain rule)
//
// Kernels are templated on (n_max, l_max, groups) and on the arithmetic type
// (double for the plain FP64 path, float for the tensor-core path).
#include "gap_internal.h"
#include "soap.h"

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

template <typename T> __device__ __forceinline__ T wacc(const SoapGeom &g, int grp, int z);
template <> __device__ __forceinline__ double wacc<double>(const SoapGeom &g, int grp, int z)
{
    return g.wacc64[grp * GAP_MAX_SPECIES + z];
}
template <> __device__ __forceinline__ float wacc<float>(const SoapGeom &g, int grp, int z)
{
    return g.wacc32[grp * GAP_MAX_SPECIES + z];
}

// channel a of coupling block b -> (group, radial n)
__device__ __forceinline__ void chan(const SoapGeom &g, int b, int a, int N, int &grp, int &n)
{
    if (g.mixed) { grp = b; n = a; }
    else { grp = a / N; n = a % N; }
}

__device__ __forceinline__ int pair_index(int Nc, int a, int ap)  // a <= ap
{
    return a * Nc - (a * (a - 1)) / 2 + (ap - a);
}

// ------------------------------------------------------------ expansion
// The accumulation c_{n lm} += w R_nl Y_lm gives each lane the m values of
// one l, in runs of at most S (the smallest S with sum_l ceil((2l+1)/S) <= 32
// runs): per pair a lane then loads its N values R_nl once for all its m.
template <int L> __host__ __device__ constexpr int expand_slots()
{
    for (int S = 1; S < 2 * L + 1; ++S) {
        int runs = 0;
        for (int l = 0; l <= L; ++l) runs += (2 * l + 1 + S - 1) / S;
        if (runs <= 32) return S;
    }
    return 2 * L + 1;
}

// Row stride of the staged Y_lm: (L+1)^2 made odd, so that the lanes' rows
// fall in distinct banks.
__host__ __device__ constexpr int expand_ylm_stride(int L) { return (L + 1) * (L + 1) | 1; }

// Neighbour pairs staged per batch of k_expand.
constexpr int kExpandBatch = 16;

// Shared memory per warp of k_expand, in elements: the pair staging area
// (Y_lm, R_nl, channel weights and the radial-table position of a batch of
// pairs) and, reusing it afterwards, the coefficients and the power spectrum
// (GA N (L+1)^2 + D).
__host__ __device__ constexpr int expand_stride(int N, int L, int GA, int D)
{
    return (kExpandBatch * (expand_ylm_stride(L) + N * (L + 1) + GA + 3) > GA * N * (L + 1) * (L + 1) + D
                ? kExpandBatch * (expand_ylm_stride(L) + N * (L + 1) + GA + 3)
                : GA * N * (L + 1) * (L + 1) + D) + 3 & ~3;
}

template <int N, int L, int GA, typename T, int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
k_expand(SoapGeom geo, const T *__restrict__ tab, int n_atoms, const int *__restrict__ offsets,
         const int *__restrict__ nbr_j, const typename V4<T>::type *__restrict__ vec, const int *__restrict__ species,
         T *__restrict__ coef, T *__restrict__ phat, T *__restrict__ pnorm)
{
    constexpr int LM = (L + 1) * (L + 1);
    constexpr int LMS = expand_ylm_stride(L);
    constexpr int NL = N * (L + 1);
    constexpr int S = expand_slots<L>();
    const int STRIDE = expand_stride(N, L, GA, geo.D);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *base = reinterpret_cast<T *>(smem_raw) + (threadIdx.x >> 5) * STRIDE;
    constexpr int BP = kExpandBatch;
    T *Ysm = base, *Rsm = base + BP * LMS, *Wsm = Rsm + BP * NL, *Psm = Wsm + BP * GA;  // Psm [3][BP]: k, u, f
    int *Ksm = reinterpret_cast<int *>(Psm);
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (i >= n_atoms) return;
    const T rc = (T)geo.rc, dw = (T)geo.d, inv_h = T(1) / (T)geo.h;
    typedef typename Coef4<T>::type C4;
    const C4 *tab4 = reinterpret_cast<const C4 *>(tab);

    // this lane's run: degree my_l, entries my_lm .. my_lm + my_cnt - 1
    int my_l = 0, my_lm = 0, my_cnt = 0;
    {
        int run = 0;
#pragma unroll
        for (int l = 0; l <= L; ++l)
#pragma unroll
            for (int m0 = 0; m0 < 2 * l + 1; m0 += S) {
                if (run == lane) {
                    my_l = l;
                    my_lm = l * l + m0;
                    my_cnt = 2 * l + 1 - m0 < S ? 2 * l + 1 - m0 : S;
                }
                ++run;
            }
    }
    T acc[S][GA][N];
#pragma unroll
    for (int o = 0; o < S; ++o)
#pragma unroll
        for (int g = 0; g < GA; ++g)
#pragma unroll
            for (int n = 0; n < N; ++n) acc[o][g][n] = T(0);

    // central Gaussian: lm = 0 only, the first slot of lane 0
    if (lane == 0 && geo.cw != 0.0) {
        const T y00 = T(0.28209479177387814347);  // 1 / (2 sqrt(pi))
        int zi = species[i];
        if (zi < 0 || zi >= geo.S) zi = 0;  // out of range: the call fails (species check)
#pragma unroll
        for (int g = 0; g < GA; ++g)
#pragma unroll
            for (int n = 0; n < N; ++n) acc[0][g][n] += wacc<T>(geo, g, zi) * (T)geo.cw * tab[4 * (n * (L + 1))] * y00;
    }

    const int p0 = offsets[i], p1 = offsets[i + 1];
    for (int base_p = p0; base_p < p1; base_p += BP) {
        const int cnt = min(BP, p1 - base_p);
        const int p = base_p + lane;
        if (lane < cnt) {
            typename V4<T>::type v = vec[p];
            T r = v.w, ir = T(1) / r;
            ylm_all<L, T>(geo, v.x * ir, v.y * ir, v.z * ir, Ysm + lane * LMS);
            T df;
            const T f = fcut_dev<T>(r, rc, dw, &df);
            const RadialPos<T> rp = radial_pos<T>(r, inv_h, geo.G);
            Ksm[lane] = rp.k;
            Psm[BP + lane] = rp.u;
            Psm[2 * BP + lane] = f;
            int z = species[nbr_j[p]];
            if (z < 0 || z >= geo.S) z = 0;  // out of range: the call fails (species check)
#pragma unroll
            for (int g = 0; g < GA; ++g) Wsm[lane * GA + g] = wacc<T>(geo, g, z);
        }
        __syncwarp();
        // f R_nl of all pairs, the warp over (pair, entry): each pair's
        // table interval is one contiguous row of NL coefficient quads; four
        // loads in flight per lane
        const int total = cnt * NL;
        for (int e0 = lane; e0 < total; e0 += 128) {
            C4 c[4];
            T u[4], f[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = e0 + 32 * k;
                if (e < total) {
                    const int t = e / NL;
                    u[k] = Psm[BP + t];
                    f[k] = Psm[2 * BP + t];
                    c[k] = tab4[(size_t)Ksm[t] * NL + (e - t * NL)];
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = e0 + 32 * k;
                if (e < total) Rsm[e] = f[k] * (c[k].x + u[k] * (c[k].y + u[k] * (c[k].z + u[k] * c[k].w)));
            }
        }
        __syncwarp();
        for (int t = 0; t < cnt; ++t) {
            const T *Rt = Rsm + t * NL + my_l;
            const T *Yt = Ysm + t * LMS + my_lm;
            T rv[N], yv[S];
#pragma unroll
            for (int n = 0; n < N; ++n) rv[n] = Rt[n * (L + 1)];
#pragma unroll
            for (int o = 0; o < S; ++o) yv[o] = o < my_cnt ? Yt[o] : T(0);
#pragma unroll
            for (int g = 0; g < GA; ++g) {
                const T wg = Wsm[t * GA + g];
#pragma unroll
                for (int o = 0; o < S; ++o) {
                    const T wy = wg * yv[o];
#pragma unroll
                    for (int n = 0; n < N; ++n) acc[o][g][n] += rv[n] * wy;
                }
            }
        }
        __syncwarp();
    }

    // coefficients to shared memory (reusing the staging area) and to global
    T *csm = base;
    T *psm = base + GA * N * LM;
#pragma unroll
    for (int o = 0; o < S; ++o) {
        const int lm = my_lm + o;
        if (o < my_cnt) {
#pragma unroll
            for (int g = 0; g < GA; ++g)
#pragma unroll
                for (int n = 0; n < N; ++n) {
                    csm[(g * N + n) * LM + lm] = acc[o][g][n];
                    coef[((size_t)i * GA * N + g * N + n) * LM + lm] = acc[o][g][n];
                }
        }
    }
    __syncwarp();
    // power spectrum
    T ss = T(0);
    const int D = geo.D;
    // entries in the l order of the descriptor table: the lanes of a warp
    // run m-loops of one length, with no index decoding
    for (int k = lane; k < D; k += 32) {
        const int4 e = __ldg(geo.dtab + k);
        const int d = e.x, l = e.w & 0xff;
        const T *c1 = csm + e.y, *c2 = csm + e.z;
        T s = T(0);
        for (int m = 0; m <= 2 * l; ++m) s += c1[m] * c2[m];
        if (e.w >> 8) s *= T(1.41421356237309504880);
        psm[d] = s;
        ss += s * s;
    }
    ss = warp_sum(ss);
    T nrm = sqrt(ss), inv = T(1) / nrm;
    __syncwarp();
    for (int d = lane; d < D; d += 32) phat[(size_t)i * D + d] = psm[d] * inv;
    if (lane == 0) pnorm[i] = nrm;
}

// ------------------------------------------------------------ backward chain
// Gam[i][z][n][lm] for every neighbour species z.
template <int N, int L, int GA, typename T>
__global__ void __launch_bounds__(32)
k_chain(SoapGeom geo, int n_atoms, const T *__restrict__ gvec, const T *__restrict__ wsum,
        const T *__restrict__ mu, const int *__restrict__ gp_of_atom, const T *__restrict__ phat,
        const T *__restrict__ pnorm, const T *__restrict__ coef, T *__restrict__ Gam)
{
    constexpr int LM = (L + 1) * (L + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int D = geo.D;
    T *hsm = reinterpret_cast<T *>(smem_raw);
    T *csm = hsm + D;
    T *gsm = csm + GA * N * LM;  // gamma [GA][N][LM]
    const int lane = threadIdx.x;
    const int i = blockIdx.x;
    if (i >= n_atoms) return;
    int s = gp_of_atom ? gp_of_atom[i] : 0;
    // g = G + wsum * mu (tensor-core path stores the centred product separately)
    T gp = T(0);
    for (int d = lane; d < D; d += 32) {
        T g = gvec[(size_t)i * geo.D16 + d];
        if (wsum && s >= 0) g += wsum[i] * mu[(size_t)s * geo.D16 + d];
        hsm[d] = g;
        gp += g * phat[(size_t)i * D + d];
    }
    gp = warp_sum(gp);
    T inv = T(1) / pnorm[i];
    __syncwarp();
    for (int d = lane; d < D; d += 32) hsm[d] = (hsm[d] - gp * phat[(size_t)i * D + d]) * inv;
    for (int q = lane; q < GA * N * LM; q += 32) csm[q] = coef[(size_t)i * GA * N * LM + q];
    __syncwarp();
    const int per = geo.npair * (L + 1);
    for (int q = lane; q < GA * N * LM; q += 32) {
        int lm = q % LM, gn = q / LM, grp = gn / N, n = gn % N;
        const int l = (int)sqrtf((float)lm + 0.5f);  // floor(sqrt(lm)), lm < 121
        int b, a;
        if (geo.mixed) { b = grp; a = n; }
        else { b = 0; a = grp * N + n; }
        T acc = T(0);
        for (int ap = 0; ap < geo.Nc; ++ap) {
            int lo = a < ap ? a : ap, hi = a < ap ? ap : a;
            T hv = hsm[b * per + pair_index(geo.Nc, lo, hi) * (L + 1) + l];
            T fac = (a == ap) ? T(2) : T(1.41421356237309504880);
            int g2, n2;
            chan(geo, b, ap, N, g2, n2);
            acc += fac * hv * csm[(g2 * N + n2) * LM + lm];
        }
        gsm[q] = acc;
    }
    __syncwarp();
    // Gam[i][z][lm][n]: the pair-force kernel reads the n values of one lm
    // as vectors
    const int S = geo.S;
    for (int q = lane; q < S * N * LM; q += 32) {
        const int z = q / (N * LM), r = q % (N * LM), lm = r / N, n = r % N, src = n * LM + lm;
        T acc = T(0);
#pragma unroll
        for (int g = 0; g < GA; ++g) acc += wacc<T>(geo, g, z) * gsm[g * N * LM + src];
        Gam[(size_t)i * S * N * LM + q] = acc;
    }
}

// The n values Gam[..][lm][0 .. N-1] as 16- or 8-byte vector loads where
// N sizeof(T) allows it (the rows start on multiples of N sizeof(T)).
template <int N, typename T>
__device__ __forceinline__ void load_n(const T *__restrict__ p, T (&out)[N])
{
    if constexpr ((N * sizeof(T)) % 16 == 0) {
#pragma unroll
        for (int k = 0; k < N * (int)sizeof(T) / 16; ++k) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + k);
            reinterpret_cast<float4 *>(out)[k] = v;
        }
    } else if constexpr ((N * sizeof(T)) % 8 == 0) {
#pragma unroll
        for (int k = 0; k < N * (int)sizeof(T) / 8; ++k) {
            const float2 v = __ldg(reinterpret_cast<const float2 *>(p) + k);
            reinterpret_cast<float2 *>(out)[k] = v;
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) out[k] = p[k];
    }
}

// ------------------------------------------------------------ pair forces
// fpair[p] = d eps_i / d r_ij for pair p = (i -> j).
template <int N, int L, typename T>
__global__ void __launch_bounds__(128, 6)
k_pairforce(SoapGeom geo, const T *__restrict__ tab, int n_pairs, const int *__restrict__ n_valid,
            const int *__restrict__ pair_i, const int *__restrict__ nbr_j,
            const typename V4<T>::type *__restrict__ vec, const int *__restrict__ species,
            const T *__restrict__ Gam, T *__restrict__ fpair)
{
    constexpr int LM = (L + 1) * (L + 1);
    constexpr int NL = N * (L + 1);
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs || p >= *n_valid) return;
    const int i = pair_i[p];
    const int zr = species[nbr_j[p]], z = zr >= 0 && zr < geo.S ? zr : 0;  // out of range: the call fails
    const T *Gm = Gam + ((size_t)i * geo.S + z) * N * LM;
    typename V4<T>::type v = vec[p];
    const T r = v.w, ir = T(1) / r;
    const T ux = v.x * ir, uy = v.y * ir, uz = v.z * ir;
    T df;
    const T f = fcut_dev<T>(r, (T)geo.rc, (T)geo.d, &df);
    const T inv_h = T(1) / (T)geo.h;
    const RadialPos<T> rp = radial_pos<T>(r, inv_h, geo.G);

    T C[L + 1], Sn[L + 1];
    C[0] = T(1); Sn[0] = T(0);
#pragma unroll
    for (int m = 1; m <= L; ++m) {
        C[m] = ux * C[m - 1] - uy * Sn[m - 1];
        Sn[m] = ux * Sn[m - 1] + uy * C[m - 1];
    }
    T q1[L + 2], q2[L + 2];
    T sU = T(0), sx = T(0), sy = T(0), sz = T(0);
#pragma unroll
    for (int l = 0; l <= L; ++l) {
        T R[N], dR[N];
#pragma unroll
        for (int n = 0; n < N; ++n) {
            T I, dI;
            radial_eval<T>(tab, NL, n * (L + 1) + l, rp, inv_h, I, dI);
            R[n] = f * I;
            dR[n] = df * I + f * dI;
        }
        T q[L + 2];
#pragma unroll
        for (int m = 0; m <= L + 1; ++m) {
            if (m > l) { q[m] = T(0); continue; }
            if (m == l) q[m] = (l == 0) ? T(1) : T(2 * l - 1) * q1[l - 1];
            else if (m == l - 1) q[m] = T(2 * l - 1) * uz * q1[m];
            else q[m] = (T(2 * l - 1) * uz * q1[m] - T(l + m - 1) * q2[m]) / T(l - m);
        }
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            if (m > l) continue;
            const T k = ylm_k<T>(geo, l, m);
            // (value, d/dx, d/dy, d/dz) of the polynomial extension, for +m and -m
            T yp, gpx, gpy, gpz, yn = T(0), gnx = T(0), gny = T(0), gnz = T(0);
            if (m == 0) {
                yp = k * q[0];
                gpx = T(0); gpy = T(0); gpz = k * q[1];
            } else {
                yp = k * q[m] * C[m];
                gpx = k * q[m] * T(m) * C[m - 1];
                gpy = -k * q[m] * T(m) * Sn[m - 1];
                gpz = k * q[m + 1] * C[m];
                yn = k * q[m] * Sn[m];
                gnx = k * q[m] * T(m) * Sn[m - 1];
                gny = k * q[m] * T(m) * C[m - 1];
                gnz = k * q[m + 1] * Sn[m];
            }
            {
                T G[N];
                load_n<N, T>(Gm + (l * l + l + m) * N, G);
                T A = T(0), B = T(0);
#pragma unroll
                for (int n = 0; n < N; ++n) { A += G[n] * R[n]; B += G[n] * dR[n]; }
                T ud = ux * gpx + uy * gpy + uz * gpz;
                sU += B * yp - A * ud * ir;
                sx += A * gpx; sy += A * gpy; sz += A * gpz;
            }
            if (m > 0) {
                T G[N];
                load_n<N, T>(Gm + (l * l + l - m) * N, G);
                T A = T(0), B = T(0);
#pragma unroll
                for (int n = 0; n < N; ++n) { A += G[n] * R[n]; B += G[n] * dR[n]; }
                T ud = ux * gnx + uy * gny + uz * gnz;
                sU += B * yn - A * ud * ir;
                sx += A * gnx; sy += A * gny; sz += A * gnz;
            }
        }
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            if (m > l) continue;
            q2[m] = q1[m];
            q1[m] = q[m];
        }
    }
    fpair[3 * (size_t)p] = sU * ux + sx * ir;
    fpair[3 * (size_t)p + 1] = sU * uy + sy * ir;
    fpair[3 * (size_t)p + 2] = sU * uz + sz * ir;
}

// ------------------------------------------------------------ two-body term
// E(r) and dE/dr of the two-body pair energy, evaluated directly (FP64).
__device__ double twobody_exact(const TwoBodyDev &tb, double r, double *dE)
{
    double df;
    const double f = fcut_dev<double>(r, tb.rc, tb.d, &df);
    const double t2 = tb.theta * tb.theta, d2 = tb.delta * tb.delta;
    double es = 0.0, des = 0.0;
    for (int m = 0; m < tb.m; ++m) {
        const double dx = r - tb.x[m];
        const double k = exp(-dx * dx / (2.0 * t2));
        es += tb.a[m] * k;
        des += tb.a[m] * (df - f * dx / t2) * k;
    }
    *dE = d2 * des;
    return d2 * f * es;
}

// Interval k of the two-body table: cubic Hermite coefficients in u = (r - r_k)/h
// from the exact values and derivatives at both knots.
__global__ void k_twobody_table(TwoBodyDev tb, D4 *__restrict__ tab)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= tb.g_in + tb.g_out) return;
    const double r0 = k < tb.g_in ? k * tb.h_in : (tb.rc - tb.d) + (k - tb.g_in) * tb.h_out;
    const double h = k < tb.g_in ? tb.h_in : tb.h_out;
    double d0, d1;
    const double e0 = twobody_exact(tb, r0, &d0), e1 = twobody_exact(tb, r0 + h, &d1);
    tab[k] = D4{e0, h * d0, 3.0 * (e1 - e0) - h * (2.0 * d0 + d1), 2.0 * (e0 - e1) + h * (d0 + d1)};
}

// Half of each pair's two-body energy goes to the pair's first atom and half
// of its derivative to f2[p], from the tabulated E(r) (FP64 in every
// precision mode: the term is large next to the 1e-4 eV/A force bound).
// One thread per atom.
__global__ void k_twobody(int n_atoms, const int *__restrict__ offsets, const D4 *__restrict__ vec, TwoBodyDev tb,
                          double *__restrict__ f2, double *__restrict__ eps2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_atoms) return;
    double e = 0.0;
    const double rt = tb.rc - tb.d, inv_in = 1.0 / tb.h_in, inv_out = 1.0 / tb.h_out;
    for (int p = offsets[i]; p < offsets[i + 1]; ++p) {
        D4 v = vec[p];
        double r = v.w, c = 0.0;
        if (r < tb.rc) {
            double s, inv;
            int k;
            if (r < rt) {
                s = r * inv_in;
                k = min((int)s, tb.g_in - 1);
                inv = inv_in;
            } else {
                s = (r - rt) * inv_out;
                k = min((int)s, tb.g_out - 1);
                inv = inv_out;
            }
            const double u = s - k;
            const D4 a = tb.tab[r < rt ? k : tb.g_in + k];
            e += 0.5 * (a.x + u * (a.y + u * (a.z + u * a.w)));
            c = 0.5 * (a.y + u * (2.0 * a.z + 3.0 * u * a.w)) * inv / r;
        }
        f2[3 * (size_t)p] = c * v.x;
        f2[3 * (size_t)p + 1] = c * v.y;
        f2[3 * (size_t)p + 2] = c * v.z;
    }
    eps2[i] = e;
}

// ------------------------------------------------------ forces and virials
// F_j = sum_{p in pairs(j)} (f[p] - f[rev p]);  W_j = -sum_{p in pairs(j)} f[p] (x) r_p.
template <typename T>
__global__ void k_gather(int n_atoms, const int *__restrict__ offsets, const int *__restrict__ rev,
                         const typename V4<T>::type *__restrict__ vec, const T *__restrict__ fpair,
                         const double *__restrict__ f2, double *__restrict__ forces, double *__restrict__ vir_atom)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_atoms) return;
    double F[3] = {0, 0, 0}, W[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = offsets[j]; p < offsets[j + 1]; ++p) {
        int q = rev[p];
        typename V4<T>::type v = vec[p];
        double fp[3] = {(double)fpair[3 * (size_t)p], (double)fpair[3 * (size_t)p + 1], (double)fpair[3 * (size_t)p + 2]};
        double vv[3] = {(double)v.x, (double)v.y, (double)v.z};
        for (int a = 0; a < 3; ++a) F[a] += fp[a] - (double)fpair[3 * (size_t)q + a];
        if (f2) {
            for (int a = 0; a < 3; ++a) {
                F[a] += f2[3 * (size_t)p + a] - f2[3 * (size_t)q + a];
                fp[a] += f2[3 * (size_t)p + a];
            }
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) W[3 * a + b] -= fp[a] * vv[b];
    }
    if (forces)
        for (int a = 0; a < 3; ++a) forces[3 * (size_t)j + a] = F[a];
    if (vir_atom)
        for (int a = 0; a < 9; ++a) vir_atom[9 * (size_t)j + a] = W[a];
}

// Per-configuration sums of local energies and atomic virials (block per config).
// Energy (eps + eps2) and virial sums of each configuration, over chunks of
// kCfgChunk atoms (block (c, k): atoms k kCfgChunk .. of configuration c) so
// that a large configuration spreads over many SMs; k_config_final adds the
// chunks in order (deterministic).
constexpr int kCfgChunk = 2048;

__global__ void k_config_part(int n_configs, int nchunk, const int *__restrict__ cfg_off,
                              const double *__restrict__ eps, const double *__restrict__ eps2,
                              const double *__restrict__ vir_atom, double *__restrict__ part)
{
    __shared__ double red[256][10];
    const int c = blockIdx.x, k = blockIdx.y;
    const int i0 = cfg_off[c] + k * kCfgChunk, i1e = cfg_off[c + 1];
    const int i1 = i0 + kCfgChunk < i1e ? i0 + kCfgChunk : i1e;
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        acc[0] += eps[i] + (eps2 ? eps2[i] : 0.0);
        if (vir_atom)
            for (int a = 0; a < 9; ++a) acc[1 + a] += vir_atom[9 * (size_t)i + a];
    }
    for (int a = 0; a < 10; ++a) red[threadIdx.x][a] = acc[a];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int a = 0; a < 10; ++a) red[threadIdx.x][a] += red[threadIdx.x + s][a];
        __syncthreads();
    }
    if (threadIdx.x < 10) part[((size_t)c * nchunk + k) * 10 + threadIdx.x] = red[0][threadIdx.x];
}

__global__ void k_config_final(int n_configs, int nchunk, const double *__restrict__ part, double *__restrict__ energy,
                               double *__restrict__ virial)
{
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= 10L * n_configs) return;
    const int c = (int)(idx / 10), a = (int)(idx % 10);
    double s = 0.0;
    for (int k = 0; k < nchunk; ++k) s += part[((size_t)c * nchunk + k) * 10 + a];
    if (a == 0) {
        if (energy) energy[c] = s;
    } else if (virial) {
        virial[9 * c + a - 1] = s;
    }
}

__global__ void k_local_energy(int n_atoms, const double *__restrict__ eps, const double *__restrict__ eps2,
                               double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_atoms) out[i] = eps[i] + (eps2 ? eps2[i] : 0.0);
}

__global__ void k_pair_atoms(int n_atoms, const int *__restrict__ offsets, int *__restrict__ pair_i)
{
    int i = blockIdx.x;
    if (i >= n_atoms) return;
    for (int p = offsets[i] + threadIdx.x; p < offsets[i + 1]; p += blockDim.x) pair_i[p] = i;
}

// ----------------------------------------------------------- dispatching
constexpr size_t kMaxSmem = 227 * 1024;  // opt-in dynamic shared memory per block

template <typename T> struct Launch {
    template <int N, int L, int GA>
    static gap_status expand(const SoapGeom &g, const T *tab, int n, const PairList &pl, const int *species, T *coef,
                             T *phat, T *pnorm, cudaStream_t st)
    {
        constexpr int WARPS = 2;
        const size_t shm = sizeof(T) * WARPS * (size_t)expand_stride(N, L, GA, g.D);
        if (shm > kMaxSmem) {
            gap_set_error("descriptor too large for the expansion kernel's shared memory");
            return GAP_EUNSUPPORTED;
        }
        auto kern = k_expand<N, L, GA, T, WARPS>;
        GAP_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        const typename V4<T>::type *vec;
        if constexpr (sizeof(T) == 8) vec = pl.vec64; else vec = pl.vec32;
        gap_count_launch();
        kern<<<(n + WARPS - 1) / WARPS, 32 * WARPS, shm, st>>>(g, tab, n, pl.offsets, pl.j, vec, species, coef, phat,
                                                              pnorm);
        return gap_cuda_status(cudaGetLastError(), "k_expand");
    }
    template <int N, int L, int GA>
    static gap_status chain(const SoapGeom &g, int n, const T *gvec, const T *wsum, const T *mu, const int *gp_of_atom,
                            const T *phat, const T *pnorm, const T *coef, T *Gam, cudaStream_t st)
    {
        constexpr int LM = (L + 1) * (L + 1);
        size_t shm = sizeof(T) * (g.D + 2 * GA * N * LM);
        if (shm > kMaxSmem) {
            gap_set_error("descriptor too large for the chain kernel's shared memory");
            return GAP_EUNSUPPORTED;
        }
        auto kern = k_chain<N, L, GA, T>;
        GAP_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        gap_count_launch();
        kern<<<n, 32, shm, st>>>(g, n, gvec, wsum, mu, gp_of_atom, phat, pnorm, coef, Gam);
        return gap_cuda_status(cudaGetLastError(), "k_chain");
    }
    template <int N, int L, int GA>
    static gap_status pairforce(const SoapGeom &g, const T *tab, const PairList &pl, const int *pair_i,
                                const int *species, const T *Gam, T *fpair, cudaStream_t st)
    {
        if (pl.n_pairs == 0) return GAP_OK;
        const typename V4<T>::type *vec;
        if constexpr (sizeof(T) == 8) vec = pl.vec64; else vec = pl.vec32;
        gap_count_launch();
        k_pairforce<N, L, T><<<(pl.n_pairs + 127) / 128, 128, 0, st>>>(g, tab, pl.n_pairs, pl.count, pair_i, pl.j,
                                                                       vec, species, Gam, fpair);
        return gap_cuda_status(cudaGetLastError(), "k_pairforce");
    }
};

// Supported (n_max, l_max, groups) instantiations.
#define GAP_SHAPES(X)  \
    X(2, 1, 1)         \
    X(4, 3, 1)         \
    X(4, 3, 2)         \
    X(4, 3, 4)         \
    X(6, 4, 1)         \
    X(6, 6, 1)         \
    X(8, 4, 1)         \
    X(8, 6, 1)         \
    X(8, 4, 5)         \
    X(8, 6, 4)         \
    X(8, 8, 1)         \
    X(10, 8, 1)

}  // namespace

bool gap_shape_supported(int N, int L, int GA)
{
#define X(n, l, ga) if (N == n && L == l && GA == ga) return true;
    GAP_SHAPES(X)
#undef X
    return false;
}

template <typename T>
gap_status gap_expand(const SoapGeom &g, const T *tab, int n, const PairList &pl, const int *species, T *coef, T *phat,
                      T *pnorm, cudaStream_t st)
{
    if (n == 0) return GAP_OK;
#define X(nn, ll, ga) \
    if (g.N == nn && g.L == ll && g.GA == ga) return Launch<T>::template expand<nn, ll, ga>(g, tab, n, pl, species, coef, phat, pnorm, st);
    GAP_SHAPES(X)
#undef X
    gap_set_error("unsupported (n_max, l_max, groups)");
    return GAP_EUNSUPPORTED;
}

template <typename T>
gap_status gap_chain(const SoapGeom &g, int n, const T *gvec, const T *wsum, const T *mu, const int *gp_of_atom,
                     const T *phat, const T *pnorm, const T *coef, T *Gam, cudaStream_t st)
{
    if (n == 0) return GAP_OK;
#define X(nn, ll, ga) \
    if (g.N == nn && g.L == ll && g.GA == ga) return Launch<T>::template chain<nn, ll, ga>(g, n, gvec, wsum, mu, gp_of_atom, phat, pnorm, coef, Gam, st);
    GAP_SHAPES(X)
#undef X
    gap_set_error("unsupported (n_max, l_max, groups)");
    return GAP_EUNSUPPORTED;
}

template <typename T>
gap_status gap_pairforce(const SoapGeom &g, const T *tab, const PairList &pl, const int *pair_i, const int *species,
                         const T *Gam, T *fpair, cudaStream_t st)
{
#define X(nn, ll, ga) \
    if (g.N == nn && g.L == ll) return Launch<T>::template pairforce<nn, ll, 1>(g, tab, pl, pair_i, species, Gam, fpair, st);
    GAP_SHAPES(X)
#undef X
    gap_set_error("unsupported (n_max, l_max)");
    return GAP_EUNSUPPORTED;
}

gap_status gap_twobody_table(const TwoBodyDev &tb, D4 *tab, cudaStream_t st)
{
    const int G = tb.g_in + tb.g_out;
    gap_count_launch();
    k_twobody_table<<<(G + 127) / 128, 128, 0, st>>>(tb, tab);
    return gap_cuda_status(cudaGetLastError(), "k_twobody_table");
}

gap_status gap_twobody(int n, const PairList &pl, const TwoBodyDev &tb, double *f2, double *eps2, cudaStream_t st)
{
    if (n == 0) return GAP_OK;
    gap_count_launch();
    k_twobody<<<(n + 127) / 128, 128, 0, st>>>(n, pl.offsets, pl.vec64, tb, f2, eps2);
    return gap_cuda_status(cudaGetLastError(), "k_twobody");
}

template <typename T>
gap_status gap_gather(int n, const PairList &pl, const T *fpair, const double *f2, double *forces, double *vir_atom,
                      cudaStream_t st)
{
    if (n == 0) return GAP_OK;
    const typename V4<T>::type *vec;
    if constexpr (sizeof(T) == 8) vec = pl.vec64; else vec = pl.vec32;
    gap_count_launch();
    k_gather<T><<<(n + 127) / 128, 128, 0, st>>>(n, pl.offsets, pl.rev, vec, fpair, f2, forces, vir_atom);
    return gap_cuda_status(cudaGetLastError(), "k_gather");
}

gap_status gap_config_sums(int n_configs, const int *cfg_off, int max_atoms, const double *eps, const double *eps2,
                           const double *vir_atom, double *energy, double *virial, double *part, cudaStream_t st)
{
    if (n_configs == 0) return GAP_OK;
    const int nchunk = max_atoms > kCfgChunk ? (max_atoms + kCfgChunk - 1) / kCfgChunk : 1;
    gap_count_launch();
    k_config_part<<<dim3(n_configs, nchunk), 256, 0, st>>>(n_configs, nchunk, cfg_off, eps, eps2, vir_atom, part);
    GAP_TRY_CUDA(cudaGetLastError());
    gap_count_launch();
    k_config_final<<<(unsigned)((10L * n_configs + 255) / 256), 256, 0, st>>>(n_configs, nchunk, part, energy, virial);
    return gap_cuda_status(cudaGetLastError(), "k_config_final");
}

gap_status gap_local_energy(int n, const double *eps, const double *eps2, double *out, cudaStream_t st)
{
    if (n == 0) return GAP_OK;
    gap_count_launch();
    k_local_energy<<<(n + 127) / 128, 128, 0, st>>>(n, eps, eps2, out);
    return gap_cuda_status(cudaGetLastError(), "k_local_energy");
}

gap_status gap_pair_atoms(int n, const PairList &pl, int *pair_i, cudaStream_t st)
{
    if (n == 0) return GAP_OK;
    gap_count_launch();
    k_pair_atoms<<<n, 64, 0, st>>>(n, pl.offsets, pair_i);
    return gap_cuda_status(cudaGetLastError(), "k_pair_atoms");
}

#define INST(T)                                                                                                      \
    template gap_status gap_expand<T>(const SoapGeom &, const T *, int, const PairList &, const int *, T *, T *, T *, \
                                      cudaStream_t);                                                                 \
    template gap_status gap_chain<T>(const SoapGeom &, int, const T *, const T *, const T *, const int *, const T *,  \
                                     const T *, const T *, T *, cudaStream_t);                                       \
    template gap_status gap_pairforce<T>(const SoapGeom &, const T *, const PairList &, const int *, const int *,     \
                                         const T *, T *, cudaStream_t);                                              \
    template gap_status gap_gather<T>(int, const PairList &, const T *, const double *, double *, double *,          \
                                      cudaStream_t);
INST(double)
INST(float)
