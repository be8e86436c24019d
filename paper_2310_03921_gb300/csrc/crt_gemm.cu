// FP64-accurate matrix products on the BF16 tensor cores by modular integer
// arithmetic (the integer-modular emulation of Ozaki, Uchino and Imamura,
// "Ozaki Scheme II"), for the least-squares solve of the fit.
//
// For C = A B^T (operands row-major with a common inner index k), every row i
// of A is scaled by a power of two and rounded to an integer
//   A'_ik = round(A_ik 2^(53 - e_i)),   max_k |A_ik| < 2^e_i,   |A'_ik| < 2^53,
// likewise every row j of B (exponent f_j), and
//   C_ij = 2^(e_i + f_j - 106) C'_ij,   C' = A' B'^T  (an exact integer).
// Rounding A and B to 53 bits below their row maxima bounds the error of C_ij
// by about K 2^-53 max_k|A_ik| max_k|B_jk|, the normwise bound of an FP64 GEMM.
// C' is formed modulo T pairwise coprime moduli p_t <= 256 whose product M
// exceeds 2 K 2^106:
//   * the residues of A' and B' (|r| <= 131) are exact BF16 values;
//   * one tcgen05 GEMM per modulus multiplies them; the products (< 2^14.1) are
//     summed exactly in FP32 tensor memory over chunks of 256 (|sum| < 2^22.1),
//     and the chunk sums are accumulated exactly in int32 registers;
//   * the Chinese remainder theorem rebuilds C' (|C'| < M / 2) from its T
//     residues in 128-bit integer arithmetic, then C is rounded to FP64.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <string>
#include <vector>

#include "crt_gemm.h"
#include "tc_prim.cuh"

namespace {

using namespace tcp;

// Pairwise coprime (256 = 2^8, 255 = 3 5 17, 253 = 11 23, 247 = 13 19,
// 217 = 7 31, the rest prime); the first 16 span 125.4 bits, all 40 span
// 336.5 bits.  The 24 primes above 256 keep symmetric residues within
// |r| <= 256, still exact BF16 values.
constexpr unsigned kModuliWide[kCrtMaxModuliWide] = {
    256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193, 509, 503, 499, 491,
    487, 479, 467, 463, 461, 457, 449, 443, 439, 433, 431, 421, 419, 409, 401, 397, 389, 383, 379, 373};
constexpr const unsigned *kModuli = kModuliWide;

struct CrtConst {
    int T;
    unsigned p[kCrtMaxModuli];
    unsigned mu[kCrtMaxModuli];   // floor(2^32 / p)
    float c14[kCrtMaxModuli][4];  // 2^(14 k) mod p, k = 0..3
    float fp[kCrtMaxModuli];      // p
    float inv_p[kCrtMaxModuli];   // 1 / p (rounded)
    unsigned y[kCrtMaxModuli];    // (M / p)^-1 mod p
    unsigned mt[kCrtMaxModuli][4];   // M / p as 32-bit limbs, least significant first
    unsigned m[4], h[4];             // M and floor(M / 2) as 32-bit limbs
    float inv_mtop;                  // (1 - 2^-20) / (M / 2^96): underestimates the quotient
};

CrtConst make_const(int T)
{
    CrtConst c{};
    c.T = T;
    unsigned __int128 M = 1;
    for (int t = 0; t < T; ++t) M *= kModuli[t];
    for (int t = 0; t < T; ++t) {
        const unsigned p = kModuli[t];
        c.p[t] = p;
        c.mu[t] = (unsigned)((1ull << 32) / p);
        for (int k = 0; k < 4; ++k) c.c14[t][k] = (float)((1ull << (14 * k)) % p);
        c.fp[t] = (float)p;
        c.inv_p[t] = (float)(1.0 / p);
        unsigned __int128 Mt = M / p;
        // inverse of Mt mod p by the extended Euclidean algorithm
        long long a = (long long)(Mt % p), b = p, x0 = 1, x1 = 0;
        while (b) {
            long long q = a / b, r = a - q * b;
            a = b;
            b = r;
            long long xn = x0 - q * x1;
            x0 = x1;
            x1 = xn;
        }
        long long inv = x0 % (long long)p;
        if (inv < 0) inv += p;
        c.y[t] = (unsigned)inv;
        for (int l = 0; l < 4; ++l) c.mt[t][l] = (unsigned)(Mt >> (32 * l));
    }
    const unsigned __int128 H = M >> 1;
    for (int l = 0; l < 4; ++l) {
        c.m[l] = (unsigned)(M >> (32 * l));
        c.h[l] = (unsigned)(H >> (32 * l));
    }
    c.inv_mtop = (float)((1.0 - std::ldexp(1.0, -20)) / (double)(M >> 96));
    return c;
}

// x mod p for x < 2^32 (Barrett: the quotient estimate is at most 2 short).
__device__ __forceinline__ unsigned mod_p(unsigned x, unsigned p, unsigned mu)
{
    unsigned r = x - __umulhi(x, mu) * p;
    if (r >= p) r -= p;
    if (r >= p) r -= p;
    return r;
}

__device__ __forceinline__ int exp_field(double x)
{
    return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// round(x 2^(53 - e)) for |x| < 2^e, e = emax - 1022 (emax the largest
// exponent field of the row), by shifting the significand; |result| < 2^53.
// Zeros and subnormals give 0.
__device__ __forceinline__ long long to_fixed(double x, int emax)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) return 0;
    const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const int d = emax - E;  // >= 0
    long long v;
    if (d == 0) v = (long long)m;
    else if (d >= 54) v = 0;
    else v = (long long)((m + (1ull << (d - 1))) >> d);
    return (b >> 63) ? -v : v;
}

// v (|v| < 2^53) as four signed 14-bit limbs held in FP32 (exact): every
// residue is then a short FP32 computation,
//   x = sum_k l_k (2^(14 k) mod p)   (|terms| < 2^22, |x| < 2^24: exact),
//   r = x - p rint(x / p),
// a representative of v mod p with |r| < 0.512 p <= 131 (the FP32 quotient
// x / p is within 0.011 of the exact one; the fused r is exact).
struct Limbs {
    float l[4];
};

__device__ __forceinline__ Limbs limbs_of(long long v)
{
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const float sg = v < 0 ? -1.f : 1.f;
    Limbs x;
#pragma unroll
    for (int k = 0; k < 4; ++k) x.l[k] = sg * (float)((unsigned)(a >> (14 * k)) & 0x3FFFu);
    return x;
}

__device__ __forceinline__ float residue(const Limbs &x, int t, const CrtConst &c)
{
    float s = x.l[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) s = fmaf(x.l[k], c.c14[t][k], s);
    return fmaf(-c.fp[t], rintf(s * c.inv_p[t]), s);
}

// BF16 of an FP32 integer of magnitude <= 256 (exact: its low 16 bits are 0).
__device__ __forceinline__ __nv_bfloat16 bf16_of_small_int(float r)
{
    return __ushort_as_bfloat16((unsigned short)(__float_as_uint(r) >> 16));
}

__device__ __forceinline__ double vat(const CrtVMat &V, long i, int j)
{
    const bool last = V.ext && j == V.cols - 1;
    if (i < V.R) {
        double v = last ? V.ext[i] : V.Y[i * V.ldy + j];
        return V.rscale ? v * V.rscale[i] : v;
    }
    long k = i - V.R;
    return (!last && j >= k) ? V.U[k + (long)j * V.ldu] : 0.0;
}

// One block per operand row (= row of V): row exponent, then residues.
__global__ void __launch_bounds__(256) k_prep_rows(CrtVMat V, long kpad, CrtConst c, __nv_bfloat16 *__restrict__ res,
                                                   int *__restrict__ E)
{
    __shared__ int smax[8];
    const long i = blockIdx.x;
    int emax = 0;
    for (int j = threadIdx.x; j < V.cols; j += blockDim.x) emax = max(emax, exp_field(vat(V, i, j)));
    emax = __reduce_max_sync(0xffffffffu, emax);
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = emax;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = smax[0];
        for (int w = 1; w < 8; ++w) m = max(m, smax[w]);
        smax[0] = m;
        E[i] = m;
    }
    __syncthreads();
    emax = smax[0];
    for (long k = threadIdx.x; k < kpad; k += blockDim.x) {
        const Limbs x = limbs_of(k < V.cols ? to_fixed(vat(V, i, (int)k), emax) : 0);
        for (int t = 0; t < c.T; ++t) res[((long)t * V.rows + i) * kpad + k] = bf16_of_small_int(residue(x, t, c));
    }
}

// Largest exponent field of each column of V over a chunk of rows (eight
// independent loads in flight per thread).
__global__ void k_col_exp(CrtVMat V, int rows_per_block, int *__restrict__ E, const double *__restrict__ diag,
                          long ld_diag, int n_diag)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= V.cols) return;
    const long i0 = (long)blockIdx.y * rows_per_block;
    long i1 = i0 + rows_per_block;
    if (i1 > V.rows) i1 = V.rows;
    int emax = 0;
    if (blockIdx.y == 0 && diag && j < n_diag) emax = exp_field(sqrt(fabs(diag[(long)j * ld_diag])));
    long i = i0;
    for (; i + 8 <= i1; i += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = vat(V, i + u, j);
#pragma unroll
        for (int u = 0; u < 8; ++u) emax = max(emax, exp_field(v[u]));
    }
    for (; i < i1; ++i) emax = max(emax, exp_field(vat(V, i, j)));
    if (emax) atomicMax(&E[j], emax);
}

// Residues of the operand whose rows are the columns of V.  Thread (j, part)
// of a 64 x 64 block takes rows i0 + 8 part .. + 7 of column j0 + j: its
// eight residues per modulus are one 16-byte chunk of the output row, stored
// directly (the eight threads of a column write 128 contiguous bytes; the
// loads of a warp touch one 32-byte sector in each of eight rows).
__global__ void __launch_bounds__(512, 3) k_prep_cols(CrtVMat V, long kpad, CrtConst c, const int *__restrict__ E,
                                                   __nv_bfloat16 *__restrict__ res)
{
    const long i0 = (long)blockIdx.y * 64;
    const int j = blockIdx.x * 64 + (threadIdx.x >> 3), part = threadIdx.x & 7;
    if (j >= V.cols) return;
    const int emax = E[j];
    const long ib = i0 + 8 * part;
    Limbs x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = limbs_of(ib + u < V.rows ? to_fixed(vat(V, ib + u, j), emax) : 0);
    for (int t = 0; t < c.T; ++t) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const unsigned lo = __bfloat16_as_ushort(bf16_of_small_int(residue(x[2 * h], t, c)));
            const unsigned hi = __bfloat16_as_ushort(bf16_of_small_int(residue(x[2 * h + 1], t, c)));
            w[h] = lo | (hi << 16);
        }
        *reinterpret_cast<uint4 *>(res + ((long)t * V.cols + j) * kpad + ib) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// ------------------------------------------------------------ modular GEMM
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4, KC = 4;
constexpr int kEpiWarps = 8, kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;

struct CrtTail {
    uint64_t full[STAGES], empty[STAGES];
    uint64_t acc_full[2], acc_empty[2];
    uint32_t tmem_base;
    int abort;
};

__constant__ unsigned c_moduli[kCrtMaxModuliWide] = {
    256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193, 509, 503, 499, 491,
    487, 479, 467, 463, 461, 457, 449, 443, 439, 433, 431, 421, 419, 409, 401, 397, 389, 383, 379, 373};

// Flags of k_crt_gemm.
enum { CG_SYM = 1, CG_B_LOWER = 2, CG_A_LOWER = 4, CG_OUT_BF16 = 8 };

// Tiles of C' mod p_t, 128 x 256 each, in a persistent grid: CTA b takes
// tiles b, b + gridDim.x, ... in the order (modulus, row tile, column tile),
// so the CTAs running at one time share operand rows in L2.  Warp 0: TMA
// producer; warp 1: TMEM allocation and MMA issue; warps 2..9: epilogue.  K
// runs in chunks of 256 into two alternating TMEM buffers (2 x 256 columns)
// that continue from tile to tile, so one tile's epilogue overlaps the next
// tile's loads and MMAs; each chunk's exact FP32 sums (|r| <= 256: at most
// 2^24) are added into int32 registers, reduced modulo p every 64 chunks.
struct CrtTile {
    int t, row0, col0, kblocks, nchunks, ncol;
    bool skip;
};

__global__ void __launch_bounds__(kThreads, 1)
k_crt_gemm(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, int rowsA, int rowsB,
           int kpad, int T, int flags, void *__restrict__ out, long ldo, int *err)
{
    // only the tiles that are computed are numbered (symmetric: those not
    // wholly below the diagonal), so the round-robin split stays even
    const int nbx = (rowsB + BN - 1) / BN, nby = (rowsA + BM - 1) / BM;
    auto first_bx = [&](int by) {  // first column tile of row tile by
        int bx = 0;
        if (flags & CG_SYM)
            while (bx < nbx && bx * BN + BN <= by * BM) ++bx;
        return bx;
    };
    int per_t = 0;
    for (int by = 0; by < nby; ++by) per_t += nbx - first_bx(by);
    const int n_tiles = T * per_t;
    auto decode = [&](int tile) {
        CrtTile c;
        c.t = tile / per_t;
        int rem = tile - c.t * per_t, by = 0;
        for (; by < nby; ++by) {
            const int cnt = nbx - first_bx(by);
            if (rem < cnt) break;
            rem -= cnt;
        }
        c.row0 = by * BM;
        c.col0 = (first_bx(by) + rem) * BN;
        c.skip = false;
        int kend = kpad;
        if ((flags & CG_B_LOWER) && c.col0 + BN < kend) kend = c.col0 + BN;  // B^T upper triangular
        if ((flags & CG_A_LOWER) && c.row0 + BM < kend) kend = c.row0 + BM;  // A lower triangular
        c.kblocks = (kend + BK - 1) / BK;
        c.nchunks = (c.kblocks + KC - 1) / KC;
        c.ncol = rowsB - c.col0 < BN ? rowsB - c.col0 : BN;
        return c;
    };

    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    CrtTail *tail = reinterpret_cast<CrtTail *>(smem + STAGES * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&tail->full[s], 1);
            mbar_init(&tail->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tail->acc_full[b], 1);
            mbar_init(&tail->acc_empty[b], kThreads - 64);
        }
        tail->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tail->tmem_base)),
                     "r"((uint32_t)(2 * BN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tail->tmem_base;
    volatile int *abort_flag = &tail->abort;

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;  // k blocks issued by this CTA
            for (int tile = blockIdx.x; tile < n_tiles && !*abort_flag; tile += gridDim.x) {
                const CrtTile c = decode(tile);
                if (c.skip) continue;
                for (int kb = 0; kb < c.kblocks; ++kb, ++g) {
                    const int s = g % STAGES, r = g / STAGES;
                    if (!mbar_wait(&tail->empty[s], (r & 1) ^ 1, abort_flag)) {
                        *abort_flag = 1;
                        atomicOr(err, 1);
                        break;
                    }
                    unsigned char *st = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&tail->full[s], STAGE_BYTES);
                    tma_load_3d(st, &mA, &tail->full[s], kb * BK, c.row0, c.t);
                    tma_load_3d(st + A_BYTES, &mB, &tail->full[s], kb * BK, c.col0, c.t);
                }
            }
            // drain: wait until the MMA has released every slot filled
            const int last = g - 1;
            for (int kb = last - STAGES + 1 < 0 ? 0 : last - STAGES + 1; kb <= last && !*abort_flag; ++kb) {
                const int s = kb % STAGES, r = kb / STAGES;
                if (!mbar_wait(&tail->empty[s], r & 1, abort_flag)) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int g = 0, gc = 0;  // k blocks and K chunks consumed by this CTA
            for (int tile = blockIdx.x; tile < n_tiles && !*abort_flag; tile += gridDim.x) {
                const CrtTile c = decode(tile);
                if (c.skip) continue;
                const uint32_t idesc = idesc_bf16((c.ncol + 15) & ~15);
                bool ok = true;
                for (int kb = 0; kb < c.kblocks; ++kb, ++g) {
                    const int q = gc + kb / KC, buf = q & 1, use = q >> 1;
                    const bool first = (kb % KC) == 0;
                    if (first && use >= 1 && !mbar_wait(&tail->acc_empty[buf], (use - 1) & 1, abort_flag)) {
                        *abort_flag = 1;
                        atomicOr(err, 8);
                        ok = false;
                        break;
                    }
                    const int s = g % STAGES, r = g / STAGES;
                    if (!mbar_wait(&tail->full[s], r & 1, abort_flag)) {
                        *abort_flag = 1;
                        atomicOr(err, 2);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tacc = tmem + (uint32_t)(buf * BN);
                    const uint32_t sa = smem_u32(smem + s * STAGE_BYTES), sb = sa + A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        umma(tacc, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), idesc,
                             (first && kk == 0) ? 0u : 1u);
                    umma_commit(&tail->empty[s]);
                    if ((kb % KC) == KC - 1 || kb == c.kblocks - 1) umma_commit(&tail->acc_full[buf]);
                }
                if (!ok) break;
                gc += c.nchunks;
            }
        }
    } else {
        const int quad = warp & 3, half = (warp - 2) >> 2;
        constexpr int HC = BN / 2;
        int gc = 0;  // K chunks consumed by this CTA
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            const CrtTile ct = decode(tile);
            if (ct.skip) continue;
            const int t = ct.t, row0 = ct.row0, col0 = ct.col0, ncol = ct.ncol;
            const int r = row0 + quad * 32 + lane;
            const int p = (int)c_moduli[t];
            int acc[HC];
#pragma unroll
            for (int k = 0; k < HC; ++k) acc[k] = 0;
            bool ok = true;
            for (int c = 0; c < ct.nchunks; ++c) {
                const int q = gc + c, buf = q & 1, use = q >> 1;
                if (!mbar_wait(&tail->acc_full[buf], use & 1, abort_flag)) {
                    *abort_flag = 1;
                    atomicOr(err, 4);
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int ch = 0; ch < HC / 32; ++ch) {
                    const int cbase = half * HC + ch * 32;
                    if (cbase < ncol) {
                        float v[32];
                        tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * BN + cbase), v);
#pragma unroll
                        for (int k = 0; k < 32; ++k) acc[ch * 32 + k] += __float2int_rn(v[k]);
                    }
                }
                tc_fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tail->acc_empty[buf]))
                             : "memory");
                if ((c & 63) == 63) {  // 64 chunks reach at most 2^30
#pragma unroll
                    for (int k = 0; k < HC; ++k) acc[k] %= p;
                }
            }
            if (!ok) break;
            gc += ct.nchunks;
            if (ok && r < rowsA && (flags & CG_OUT_BF16)) {
                // symmetric residues as BF16, 0 beyond column rowsB (the padding
                // of an operand's K extent)
                __nv_bfloat16 *orow = reinterpret_cast<__nv_bfloat16 *>(out) + ((long)t * rowsA + r) * ldo + col0;
    #pragma unroll
                for (int ch = 0; ch < HC / 32; ++ch) {
                    const int cbase = half * HC + ch * 32;
                    uint32_t w[16];
    #pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        uint32_t word = 0;
    #pragma unroll
                        for (int b = 0; b < 2; ++b) {
                            const int k = ch * 32 + q * 2 + b;
                            int m = acc[k] % p;
                            if (m < 0) m += p;
                            if (2 * m > p) m -= p;
                            if (cbase + q * 2 + b >= ncol) m = 0;
                            word |= (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)m)) << (16 * b);
                        }
                        w[q] = word;
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(orow + cbase);
                    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
                    dst[2] = make_uint4(w[8], w[9], w[10], w[11]);
                    dst[3] = make_uint4(w[12], w[13], w[14], w[15]);
                }
            } else if (ok && r < rowsA) {
    #pragma unroll
                for (int ch = 0; ch < HC / 32; ++ch) {
                    const int cbase = half * HC + ch * 32;
                    if (cbase < ncol) {
                        uint32_t w[8];
    #pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            uint32_t word = 0;
    #pragma unroll
                            for (int b = 0; b < 4; ++b) {
                                int m = acc[ch * 32 + q * 4 + b] % p;
                                if (m < 0) m += p;
                                word |= (uint32_t)m << (8 * b);
                            }
                            w[q] = word;
                        }
                        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(out) +
                                                               ((long)t * rowsA + r) * ldo + col0 + cbase);
                        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                        dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN))
                     : "memory");
    }
}

// (-1)^neg mag 2^s rounded to nearest (ties away from zero) FP64, built with
// integer operations only; results below the normal range flush to zero.
__device__ __forceinline__ double to_double(unsigned __int128 mag, bool neg, int s)
{
    const unsigned long long hi = (unsigned long long)(mag >> 64), lo = (unsigned long long)mag;
    if ((hi | lo) == 0) return 0.0;
    const int lead = hi ? 127 - __clzll(hi) : 63 - __clzll(lo);  // index of the leading bit
    unsigned long long m;                                        // 53 significant bits
    if (lead <= 52) {
        m = lo << (52 - lead);
    } else {
        const int sh = lead - 52;  // 1 .. 75
        const unsigned __int128 t = mag >> (sh - 1);
        m = (unsigned long long)(t >> 1) + ((unsigned long long)t & 1ull);
    }
    int e = lead + s + 1023;
    if (m >> 53) {  // rounding carried into a new bit
        m >>= 1;
        ++e;
    }
    if (e <= 0) return neg ? -0.0 : 0.0;
    if (e >= 2047) return neg ? -__longlong_as_double(0x7FF0000000000000ll) : __longlong_as_double(0x7FF0000000000000ll);
    const unsigned long long bits =
        ((unsigned long long)neg << 63) | ((unsigned long long)e << 52) | (m & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

// acc (5 limbs) += w * x (4 limbs), w < 2^32: one carry chain for the low
// halves of the partial products, one for the high halves.
__device__ __forceinline__ void mac4(unsigned (&acc)[5], unsigned w, const unsigned (&x)[4])
{
    asm("mad.lo.cc.u32 %0, %5, %6, %0;\n\t"
        "madc.lo.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %8, %2;\n\t"
        "madc.lo.cc.u32 %3, %5, %9, %3;\n\t"
        "addc.u32 %4, %4, 0;\n\t"
        "mad.hi.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.cc.u32 %3, %5, %8, %3;\n\t"
        "madc.hi.u32 %4, %5, %9, %4;"
        : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2]), "+r"(acc[3]), "+r"(acc[4])
        : "r"(w), "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]));
}

// acc (5 limbs) -= q * x (4 limbs); the caller guarantees no underflow.
__device__ __forceinline__ void msub4(unsigned (&acc)[5], unsigned q, const unsigned (&x)[4])
{
    unsigned long long prod = 0;
    long long borrow = 0;
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        if (l < 4) prod += (unsigned long long)q * x[l];
        long long d = (long long)acc[l] - (long long)(unsigned)prod - borrow;
        acc[l] = (unsigned)d;
        borrow = d < 0 ? 1 : 0;
        prod >>= 32;
    }
}

// a >= b over 4 limbs (a[4] == 0 assumed by the caller when it matters)
__device__ __forceinline__ bool geq4(const unsigned (&a)[5], const unsigned (&b)[4])
{
    if (a[4]) return true;
#pragma unroll
    for (int l = 3; l >= 0; --l)
        if (a[l] != b[l]) return a[l] > b[l];
    return true;
}

// Signed C' from its T byte residues (plane stride ps): C' = sum_t w_t M/p_t
// mod M with w_t = r_t (M/p_t)^-1 mod p_t (Chinese remainder theorem),
// accumulated in 32-bit limbs and reduced once with a quotient estimate;
// the representative in (-M/2, M/2] as sign and magnitude.
__device__ __forceinline__ void crt_value(const unsigned char *__restrict__ o, long ps, const CrtConst &c, bool &neg,
                                          unsigned (&mag)[4])
{
    // sum_t (r_t y_t) M/p_t without reducing r_t y_t (< 2^16): acc < 2^13 M
    unsigned acc[5] = {0, 0, 0, 0, 0};
    for (int t = 0; t < c.T; ++t) {
        const unsigned r = o[(long)t * ps];
        mac4(acc, r * c.y[t], c.mt[t]);
    }
    // subtract floor(acc / M) M (estimated from the top 64 bits, at most one short)
    const float top = fmaf((float)acc[4], 4294967296.f, (float)acc[3]);
    const unsigned q = (unsigned)(top * c.inv_mtop);
    msub4(acc, q, c.m);
    while (geq4(acc, c.m)) msub4(acc, 1u, c.m);
    // symmetric range: C' = acc - M when acc > M / 2
    neg = false;
#pragma unroll
    for (int l = 0; l < 4; ++l) mag[l] = acc[l];
    bool gt = false;
#pragma unroll
    for (int l = 3; l >= 0; --l)
        if (acc[l] != c.h[l]) {
            gt = acc[l] > c.h[l];
            break;
        }
    if (gt) {
        neg = true;
        long long borrow = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            long long d = (long long)c.m[l] - (long long)acc[l] - borrow;
            mag[l] = (unsigned)d;
            borrow = d < 0 ? 1 : 0;
        }
    }
}

__device__ __forceinline__ unsigned __int128 u128_of(const unsigned (&m)[4])
{
    return ((unsigned __int128)(((unsigned long long)m[3] << 32) | m[2]) << 64) |
           (((unsigned long long)m[1] << 32) | m[0]);
}

// C[i][j] = alpha 2^(Ea_i + Eb_j - 2150) C'[i][j] (+ Cin).
__global__ void k_crt_combine(const unsigned char *__restrict__ out, long ldo, long rows, int cols, int nb,
                              CrtConst c, const int *__restrict__ Ea, const int *__restrict__ Eb, int sym,
                              double alpha, const double *Cin, long ldcin, double *C, long ldc)
{
    const long blk = blockIdx.x;
    const long i = blk / nb;
    const int j = (int)(blk % nb) * blockDim.x + threadIdx.x;
    if (i >= rows || j >= cols) return;
    long ii = i, jj = j;
    if (sym && j < i) {
        ii = j;
        jj = i;
    }
    bool neg;
    unsigned mag[4];
    crt_value(out + ii * ldo + jj, rows * ldo, c, neg, mag);
    double v = to_double(u128_of(mag), neg, Ea[ii] + Eb[jj] - 2150);
    if (alpha != 1.0) v *= alpha;
    if (Cin) v += Cin[i * ldcin + j];
    C[i * ldc + j] = v;
}

// ------------------------------------------- exact congruence products

// Residue constants of the wide moduli for operand preparation.
struct WideRes {
    int T;
    float c14[kCrtMaxModuliWide][4];  // 2^(14 k) mod p, symmetric representative
    float fp[kCrtMaxModuliWide];
    float inv_p[kCrtMaxModuliWide];
    unsigned p[kCrtMaxModuliWide];
    unsigned mu[kCrtMaxModuliWide];      // floor(2^32 / p)
    unsigned c32[kCrtMaxModuliWide][4];  // 2^(32 k) mod p
};

WideRes make_wide_res(int T)
{
    WideRes c{};
    c.T = T;
    for (int t = 0; t < T; ++t) {
        const unsigned p = kModuliWide[t];
        c.p[t] = p;
        c.mu[t] = (unsigned)((1ull << 32) / p);
        for (int k = 0; k < 4; ++k) {
            long long r = (long long)((1ull << (14 * k)) % p);
            if (2 * r > (long long)p) r -= p;
            c.c14[t][k] = (float)r;
            unsigned long long q = 1;
            for (int e = 0; e < k; ++e) q = (q << 32) % p;
            c.c32[t][k] = (unsigned)q;
        }
        c.fp[t] = (float)p;
        c.inv_p[t] = (float)(1.0 / p);
    }
    return c;
}

// Symmetric residue of a 14-bit-limb integer (|v| < 2^53): the limb sum
// |s| < 2^14 (1 + 3 256) < 2^24 is exact in FP32, and the quotient s / p is
// within 2 / p of the exact one, so |r| <= p / 2 + 2; the last step folds the
// rare |r| > 256 back (only for p > 508).
__device__ __forceinline__ float residue_w(const Limbs &x, int t, const WideRes &c)
{
    float s = x.l[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) s = fmaf(x.l[k], c.c14[t][k], s);
    float r = fmaf(-c.fp[t], rintf(s * c.inv_p[t]), s);
    if (r > 256.f) r -= c.fp[t];
    if (r < -256.f) r += c.fp[t];
    return r;
}

// Symmetric residue of (-1)^neg mag (four 32-bit limbs) modulo p_t.
__device__ __forceinline__ int residue_mag(const unsigned (&mag)[4], bool neg, int t, const WideRes &c)
{
    const unsigned p = c.p[t], mu = c.mu[t];
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += mod_p(mag[k], p, mu) * c.c32[t][k];  // < 4 2^18
    int r = (int)mod_p(s, p, mu);
    if (neg && r) r = (int)p - r;
    if (2 * r > (int)p) r -= (int)p;
    return r;
}

// round(x 2^s) as a signed 128-bit integer; false if it is 2^110 or more (or x
// is not finite).  Subnormal x count as 0.
__device__ __forceinline__ bool fixed_of(double x, int s, __int128 &v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    v = 0;
    if (E == 0) return true;
    if (E == 0x7FF) return false;
    const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = E - 1075 + s;
    unsigned __int128 mag;
    if (sh >= 0) {
        if (sh > 110 - 53) return false;
        mag = (unsigned __int128)m << sh;
    } else if (sh < -60) {
        mag = 0;
    } else {
        mag = (m + (1ull << (-sh - 1))) >> (-sh);
    }
    v = (b >> 63) ? -(__int128)mag : (__int128)mag;
    return true;
}

// G'_ij + round(Kt_ij 2^(2150 - E_i - E_j)) for the 32 x 32 tiles on and above
// the diagonal (blockIdx.y <= blockIdx.x), the columns running on to kpad2:
// residues [t][i][j] and, through shared memory, [t][j][i]; FP64 G likewise.
__global__ void __launch_bounds__(256) k_exact_gram(const unsigned char *__restrict__ out, long ldo, CrtConst c1,
                                                    int n, const int *__restrict__ E, const double *__restrict__ Kt,
                                                    WideRes c2, long kpad2, __nv_bfloat16 *__restrict__ res,
                                                    double *__restrict__ G, int *err)
{
    const int bj = blockIdx.x, bi = blockIdx.y;
    if (bi > bj) return;
    const int n_ext = n + 1;
    __shared__ unsigned short ts[32][33];
    __shared__ double tg[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int j = bj * 32 + tx;
    unsigned mag[4][4];
    bool neg[4];
    bool bad = false;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = bi * 32 + ty + 8 * u;
        neg[u] = false;
#pragma unroll
        for (int l = 0; l < 4; ++l) mag[u][l] = 0;
        if (i >= n_ext || j >= n_ext) continue;
        __int128 v = 0;
        if (out) {
            const int ii = i < j ? i : j, jj = i < j ? j : i;
            bool ng;
            unsigned mg[4];
            crt_value(out + (long)ii * ldo + jj, (long)n_ext * ldo, c1, ng, mg);
            const __int128 a = (__int128)u128_of(mg);
            v = ng ? -a : a;
        }
        if (Kt && i < n && j < n) {
            __int128 k;
            if (!fixed_of(Kt[i + (long)j * n], 2150 - E[i] - E[j], k)) bad = true;
            else v += k;
        }
        neg[u] = v < 0;
        const unsigned __int128 a = (unsigned __int128)(v < 0 ? -v : v);
#pragma unroll
        for (int l = 0; l < 4; ++l) mag[u][l] = (unsigned)(a >> (32 * l));
    }
    if (bad) atomicOr(err, 16);
    // FP64 values (n x n block)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = bi * 32 + ty + 8 * u;
        double g = 0.0;
        if (i < n && j < n) g = to_double(u128_of(mag[u]), neg[u], E[i] + E[j] - 2150);
        if (i < n && j < n) G[j + (long)i * n] = g;
        tg[ty + 8 * u][tx] = g;
    }
    __syncthreads();
    if (bi < bj) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int jr = bj * 32 + ty + 8 * u, ic = bi * 32 + tx;
            if (jr < n && ic < n) G[ic + (long)jr * n] = tg[tx][ty + 8 * u];
        }
    }
    for (int t = 0; t < c2.T; ++t) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = bi * 32 + ty + 8 * u;
            const int r = residue_mag(mag[u], neg[u], t, c2);
            const unsigned short h = __bfloat16_as_ushort(__float2bfloat16_rn((float)r));
            if (i < n_ext && j < kpad2) res[((long)t * n_ext + i) * kpad2 + j] = __ushort_as_bfloat16(h);
            ts[ty + 8 * u][tx] = h;
        }
        __syncthreads();
        if (bi < bj) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int jr = bj * 32 + ty + 8 * u, ic = bi * 32 + tx;
                if (jr < n_ext && ic < n_ext)
                    res[((long)t * n_ext + jr) * kpad2 + ic] = __ushort_as_bfloat16(ts[tx][ty + 8 * u]);
            }
        }
    }
}

// Row i of the operand (= column i of W_ext): exponent F_i of its largest
// scaled entry W_ki 2^(E_k - 1075), then the 53-bit fixed-point entries and
// their residues.
__global__ void __launch_bounds__(256) k_prep_congruence(const double *W, int n, const int *__restrict__ E,
                                                         WideRes c, long kpad2, __nv_bfloat16 *__restrict__ res,
                                                         int *__restrict__ F, double *Wt)
{
    __shared__ int smax[8];
    const int i = blockIdx.x, n_ext = n + 1;
    auto elem = [&](int k) -> double {
        if (i < n && k < n) return W[k + (long)i * n];
        return i == k ? 1.0 : 0.0;
    };
    int emax = -(1 << 30);
    for (int k = threadIdx.x; k < n_ext; k += blockDim.x) {
        const int ex = exp_field(elem(k));
        if (ex && E[k]) emax = max(emax, ex + E[k] - 1075);
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = emax;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = smax[0];
        for (int w = 1; w < 8; ++w) m = max(m, smax[w]);
        if (m < -(1 << 29)) m = 0;  // an all-zero row
        smax[0] = m;
        F[i] = m;
    }
    __syncthreads();
    emax = smax[0];
    for (long k = threadIdx.x; k < kpad2; k += blockDim.x) {
        long long v = 0;
        if (k < n_ext) {
            const double x = elem((int)k);
            const unsigned long long b = (unsigned long long)__double_as_longlong(x);
            const int ex = (int)((b >> 52) & 0x7FF);
            if (ex && E[k]) {
                const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);
                const int d = emax - (ex + E[k] - 1075);  // >= 0
                if (d == 0) v = (long long)m;
                else if (d < 54) v = (long long)((m + (1ull << (d - 1))) >> d);
                if (b >> 63) v = -v;
            }
            if (Wt && i < n && k < n) Wt[k + (long)i * n] = v ? ldexp((double)v, emax - E[k]) : 0.0;
        }
        const Limbs x = limbs_of(v);
        for (int t = 0; t < c.T; ++t) res[((long)t * n_ext + i) * kpad2 + k] = bf16_of_small_int(residue_w(x, t, c));
    }
}

// CRT constants of the wide moduli, in L 32-bit limbs (L = limbs of M).
constexpr int kWideLimbs = 12;
struct CrtWide {
    int T, L;
    unsigned p[kCrtMaxModuliWide];
    unsigned y[kCrtMaxModuliWide];               // (M / p)^-1 mod p
    unsigned mt[kCrtMaxModuliWide][kWideLimbs];  // M / p
    unsigned m[kWideLimbs], h[kWideLimbs];       // M, floor(M / 2)
    double mtop;                                 // M / 2^(32 (L - 2)) (rounded)
};

// little-endian 32-bit limb multiplication by a small factor
void big_mul(std::vector<unsigned> &a, unsigned f)
{
    unsigned long long carry = 0;
    for (auto &x : a) {
        const unsigned long long v = (unsigned long long)x * f + carry;
        x = (unsigned)v;
        carry = v >> 32;
    }
    if (carry) a.push_back((unsigned)carry);
}

long long inv_mod(long long a, long long p)
{
    long long b = p, x0 = 1, x1 = 0;
    a %= p;
    while (b) {
        const long long q = a / b, r = a - q * b;
        a = b;
        b = r;
        const long long xn = x0 - q * x1;
        x0 = x1;
        x1 = xn;
    }
    x0 %= p;
    return x0 < 0 ? x0 + p : x0;
}

CrtWide make_wide(int T)
{
    CrtWide c{};
    c.T = T;
    std::vector<unsigned> M{1};
    for (int t = 0; t < T; ++t) big_mul(M, kModuliWide[t]);
    c.L = (int)M.size();
    for (int l = 0; l < c.L; ++l) c.m[l] = M[l];
    for (int l = 0; l < c.L; ++l) c.h[l] = (M[l] >> 1) | (l + 1 < c.L ? (M[l + 1] & 1u) << 31 : 0u);
    double top = 0.0;
    for (int l = c.L - 1; l >= 0 && l >= c.L - 3; --l) top += std::ldexp((double)M[l], 32 * (l - (c.L - 2)));
    c.mtop = top;
    for (int t = 0; t < T; ++t) {
        const unsigned p = kModuliWide[t];
        c.p[t] = p;
        std::vector<unsigned> Mt{1};
        long long rem = 1;
        for (int s = 0; s < T; ++s)
            if (s != t) {
                big_mul(Mt, kModuliWide[s]);
                rem = rem * kModuliWide[s] % p;
            }
        c.y[t] = (unsigned)inv_mod(rem, p);
        for (int l = 0; l < (int)Mt.size() && l < kWideLimbs; ++l) c.mt[t][l] = Mt[l];
    }
    return c;
}

// -1^neg mag (L limbs) 2^s as FP64: the top 128 bits decide the rounding
// (ties away from zero cannot change with the bits below them).
template <int L>
__device__ __forceinline__ double to_double_wide(const unsigned (&mag)[L + 1], bool neg, int s)
{
    int h = L - 1;
    while (h > 3 && mag[h] == 0) --h;
    const int b = h - 3;
    const unsigned m4[4] = {mag[b], mag[b + 1], mag[b + 2], mag[b + 3]};
    return to_double(u128_of(m4), neg, s + 32 * b);
}

// C = W^T G W from its residues: one thread per upper-triangle entry.
template <int L>
__global__ void __launch_bounds__(256) k_combine_congruence(const __nv_bfloat16 *__restrict__ out, long ldo, int n,
                                                            CrtWide c, const int *__restrict__ F,
                                                            double *__restrict__ G, double *__restrict__ cvec)
{
    const int n_ext = n + 1;
    const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || j < i || j >= n_ext) return;
    unsigned acc[L + 1];
#pragma unroll
    for (int l = 0; l <= L; ++l) acc[l] = 0;
    for (int t0 = 0; t0 < c.T; t0 += 8) {
        float rf[8];  // eight residue loads in flight
#pragma unroll
        for (int k = 0; k < 8; ++k)
            rf[k] = t0 + k < c.T ? __bfloat162float(out[((long)(t0 + k) * n_ext + i) * ldo + j]) : 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int t = t0 + k;
            if (t >= c.T) break;
            int r = (int)rf[k];
            if (r < 0) r += (int)c.p[t];
            const unsigned w = (unsigned)r * c.y[t];  // < 2^18
            unsigned long long carry = 0;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const unsigned long long v = (unsigned long long)w * c.mt[t][l] + acc[l] + carry;
                acc[l] = (unsigned)v;
                carry = v >> 32;
            }
            acc[L] += (unsigned)carry;
        }
    }
    // acc < T 2^18 M: subtract q M, q from the top three limbs (never above
    // the true quotient, at most two below it), then at most a few M
    {
        const double top = std::ldexp((double)acc[L], 64) + std::ldexp((double)acc[L - 1], 32) + (double)acc[L - 2];
        const unsigned q = (unsigned)floor(top / c.mtop * (1.0 - 1e-12));
        unsigned long long prod = 0;
        long long borrow = 0;
#pragma unroll
        for (int l = 0; l <= L; ++l) {
            if (l < L) prod += (unsigned long long)q * c.m[l];
            const long long d = (long long)acc[l] - (long long)(unsigned)prod - borrow;
            acc[l] = (unsigned)d;
            borrow = d < 0 ? 1 : 0;
            prod >>= 32;
        }
    }
    for (int it = 0; it < 4; ++it) {
        bool ge = acc[L] != 0;
        if (!ge) {
            ge = true;
            for (int l = L - 1; l >= 0; --l)
                if (acc[l] != c.m[l]) {
                    ge = acc[l] > c.m[l];
                    break;
                }
        }
        if (!ge) break;
        long long borrow = 0;
#pragma unroll
        for (int l = 0; l <= L; ++l) {
            const long long d = (long long)acc[l] - (long long)(l < L ? c.m[l] : 0u) - borrow;
            acc[l] = (unsigned)d;
            borrow = d < 0 ? 1 : 0;
        }
    }
    // symmetric representative
    bool gt = false;
    for (int l = L - 1; l >= 0; --l)
        if (acc[l] != c.h[l]) {
            gt = acc[l] > c.h[l];
            break;
        }
    unsigned mag[L + 1];
    if (gt) {
        long long borrow = 0;
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const long long d = (long long)c.m[l] - (long long)acc[l] - borrow;
            mag[l] = (unsigned)d;
            borrow = d < 0 ? 1 : 0;
        }
    } else {
#pragma unroll
        for (int l = 0; l < L; ++l) mag[l] = acc[l];
    }
    mag[L] = 0;
    const double v = to_double_wide<L>(mag, gt, F[i] + F[j] - 2150);
    if (j == n) {
        cvec[i] = v;
    } else {
        G[j + (long)i * n] = v;
        G[i + (long)j * n] = v;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Residue planes [T][rows][kpad] BF16 as a 3-D tensor (k, row, plane).
gap_status make_map3(CUtensorMap *m, const void *ptr, long rows, long kpad, int T, int box_rows)
{
    auto enc = encode_fn();
    if (!enc) {
        gap_set_error("cuTensorMapEncodeTiled is unavailable");
        return GAP_ECUDA;
    }
    if (reinterpret_cast<uintptr_t>(ptr) & 15) {
        gap_set_error("residue planes are not 16-byte aligned");
        return GAP_EINVAL;
    }
    cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)T};
    cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)kpad * 2 * (cuuint64_t)rows};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        gap_set_error("cuTensorMapEncodeTiled (residue planes) failed with code " + std::to_string((int)r));
        return GAP_ECUDA;
    }
    return GAP_OK;
}

}  // namespace

int gap_crt_moduli(long K)
{
    if (K < 1) K = 1;
    // need log2(M) > 107 + log2(K): |C'| <= K (2^53 - 1)^2 and M > 2 |C'|
    double need = 107.0 + std::log2((double)K) + 1e-9, have = 0.0;
    for (int t = 0; t < kCrtMaxModuli; ++t) {
        have += std::log2((double)kModuli[t]);
        if (have > need) return t + 1;
    }
    return 0;
}

gap_status gap_crt_prep_rows(const CrtVMat &V, int T, long kpad, __nv_bfloat16 *res, int *E, cudaStream_t st)
{
    if (V.rows <= 0) return GAP_OK;
    if (V.rows > 2147483647L || kpad < V.cols) {
        gap_set_error("modular GEMM operand too large");
        return GAP_EINVAL;
    }
    gap_count_launch();
    k_prep_rows<<<(unsigned)V.rows, 256, 0, st>>>(V, kpad, make_const(T), res, E);
    return gap_cuda_status(cudaGetLastError(), "k_prep_rows");
}

gap_status gap_crt_prep_cols(const CrtVMat &V, int T, long kpad, __nv_bfloat16 *res, int *E, cudaStream_t st,
                             const double *diag, long ld_diag, int n_diag)
{
    if (V.cols <= 0) return GAP_OK;
    if (kpad < V.rows || (kpad + 63) / 64 > 65535) {
        gap_set_error("modular GEMM operand too large");
        return GAP_EINVAL;
    }
    GAP_TRY_CUDA(cudaMemsetAsync(E, 0, sizeof(int) * V.cols, st));
    const int rpb = 128;
    dim3 g1((V.cols + 127) / 128, (unsigned)(V.rows > 0 ? (V.rows + rpb - 1) / rpb : 1));
    gap_count_launch();
    k_col_exp<<<g1, 128, 0, st>>>(V, rpb, E, diag, ld_diag, n_diag);
    GAP_TRY_CUDA(cudaGetLastError());
    dim3 g2((V.cols + 63) / 64, (unsigned)(kpad / 64));
    gap_count_launch();
    k_prep_cols<<<g2, 512, 0, st>>>(V, kpad, make_const(T), E, res);
    return gap_cuda_status(cudaGetLastError(), "k_prep_cols");
}

gap_status gap_crt_gemm(const __nv_bfloat16 *resA, long rowsA, const __nv_bfloat16 *resB, long rowsB, long kpad,
                        int T, bool sym, bool b_lower, void *out, long ldo, int *err, cudaStream_t st, bool a_lower,
                        bool out_bf16)
{
    if (rowsA <= 0 || rowsB <= 0) return GAP_OK;
    if (kpad % 64 || ldo % 256 || ldo < (rowsB + 255) / 256 * 256 || (rowsA + BM - 1) / BM > 65535 ||
        kpad > 2147483647L || T < 1 || T > (out_bf16 ? kCrtMaxModuliWide : kCrtMaxModuli)) {
        gap_set_error("modular GEMM: bad shape");
        return GAP_EINVAL;
    }
    CUtensorMap mA, mB;
    GAP_TRY(make_map3(&mA, resA, rowsA, kpad, T, BM));
    GAP_TRY(make_map3(&mB, resB, rowsB, kpad, T, BN));
    const size_t shm = (size_t)STAGES * STAGE_BYTES + sizeof(CrtTail) + 1024;
    GAP_TRY_CUDA(cudaFuncSetAttribute(k_crt_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    const long n_tiles = ((rowsB + BN - 1) / BN) * ((rowsA + BM - 1) / BM) * (long)T;
    if (n_tiles > 2147483647L) {
        gap_set_error("modular GEMM: too many tiles");
        return GAP_EINVAL;
    }
    int n_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm <= 0) {
        cudaGetLastError();
        n_sm = 132;
    }
    gap_count_launch();
    k_crt_gemm<<<(unsigned)(n_tiles < n_sm ? n_tiles : n_sm), kThreads, shm, st>>>(
        mA, mB, (int)rowsA, (int)rowsB, (int)kpad, T,
        (sym ? CG_SYM : 0) | (b_lower ? CG_B_LOWER : 0) | (a_lower ? CG_A_LOWER : 0) | (out_bf16 ? CG_OUT_BF16 : 0),
        out, ldo, err);
    return gap_cuda_status(cudaGetLastError(), "k_crt_gemm");
}

gap_status gap_crt_combine(const unsigned char *out, long ldo, long rows, int cols, int T, const int *Ea,
                           const int *Eb, bool sym, double *C, long ldc, cudaStream_t st, double alpha,
                           const double *Cin, long ldcin)
{
    if (rows <= 0 || cols <= 0) return GAP_OK;
    const int nb = (cols + 255) / 256;
    const long blocks = rows * nb;
    if (blocks > 2147483647L) {
        gap_set_error("modular GEMM output too large");
        return GAP_EINVAL;
    }
    gap_count_launch();
    k_crt_combine<<<(unsigned)blocks, 256, 0, st>>>(out, ldo, rows, cols, nb, make_const(T), Ea, Eb, sym ? 1 : 0,
                                                     alpha, Cin, ldcin, C, ldc);
    return gap_cuda_status(cudaGetLastError(), "k_crt_combine");
}

int gap_crt_moduli_wide(double bits)
{
    double have = 0.0;
    for (int t = 0; t < kCrtMaxModuliWide; ++t) {
        have += std::log2((double)kModuliWide[t]);
        if (have > bits + 1.0 + 1e-9) return t + 1;  // M > 2 bound
    }
    return 0;
}

double gap_crt_congruence_bits(long rows, int n_ext)
{
    // |G'| <= (rows + 2) 2^106 (V' entries below 2^53, the rounded Kt below
    // 2^106 (1 + eps)); |W'| < 2^53; |W'^T G' W'| <= n_ext^2 2^106 |G'|
    return 2.0 * std::log2((double)n_ext) + 212.0 + std::log2((double)rows + 2.0);
}

gap_status gap_crt_exact_gram(const unsigned char *out, long ldo, int T1, int n, const int *E, const double *Kt,
                              int T2, long kpad2, __nv_bfloat16 *res, double *G, int *err, cudaStream_t st)
{
    const int n_ext = n + 1;
    if (n <= 0) return GAP_OK;
    if (kpad2 % 256 || kpad2 < n_ext || T2 < 1 || T2 > kCrtMaxModuliWide || (out && (T1 < 1 || T1 > kCrtMaxModuli))) {
        gap_set_error("exact Gram matrix: bad shape");
        return GAP_EINVAL;
    }
    dim3 grid((unsigned)(kpad2 / 32), (unsigned)((n_ext + 31) / 32));
    gap_count_launch();
    k_exact_gram<<<grid, 256, 0, st>>>(out, ldo, make_const(out ? T1 : 1), n, E, Kt, make_wide_res(T2), kpad2, res,
                                       G, err);
    return gap_cuda_status(cudaGetLastError(), "k_exact_gram");
}

gap_status gap_crt_prep_congruence(const double *W, int n, const int *E, int T2, long kpad2, __nv_bfloat16 *res,
                                   int *F, double *Wt, cudaStream_t st)
{
    if (n <= 0) return GAP_OK;
    if (kpad2 % 64 || kpad2 < n + 1 || T2 < 1 || T2 > kCrtMaxModuliWide) {
        gap_set_error("congruence operand: bad shape");
        return GAP_EINVAL;
    }
    gap_count_launch();
    k_prep_congruence<<<(unsigned)(n + 1), 256, 0, st>>>(W, n, E, make_wide_res(T2), kpad2, res, F, Wt);
    return gap_cuda_status(cudaGetLastError(), "k_prep_congruence");
}

gap_status gap_crt_combine_congruence(const __nv_bfloat16 *out, long ldo, int n, int T2, const int *F, double *G,
                                      double *c, cudaStream_t st)
{
    if (n <= 0) return GAP_OK;
    if (T2 < 1 || T2 > kCrtMaxModuliWide) {
        gap_set_error("congruence combine: bad modulus count");
        return GAP_EINVAL;
    }
    const CrtWide cw = make_wide(T2);
    dim3 grid((unsigned)((n + 1 + 255) / 256), (unsigned)n);
    gap_count_launch();
    switch (cw.L) {
#define GAP_CONGRUENCE_CASE(LL)                                                             \
    case LL:                                                                                 \
        k_combine_congruence<LL><<<grid, 256, 0, st>>>(out, ldo, n, cw, F, G, c);           \
        break;
        GAP_CONGRUENCE_CASE(5)
        GAP_CONGRUENCE_CASE(6)
        GAP_CONGRUENCE_CASE(7)
        GAP_CONGRUENCE_CASE(8)
        GAP_CONGRUENCE_CASE(9)
        GAP_CONGRUENCE_CASE(10)
        GAP_CONGRUENCE_CASE(11)
#undef GAP_CONGRUENCE_CASE
    default:
        gap_set_error("congruence combine: unsupported limb count " + std::to_string(cw.L));
        return GAP_EINVAL;
    }
    return gap_cuda_status(cudaGetLastError(), "k_combine_congruence");
}
