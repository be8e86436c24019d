// Split-precision BF16 GEMM on the sm_103a tensor cores (tcgen05 + TMA + TMEM).
//
//   C[r][c] = sum_k (Ahi Bhi + Ahi Blo + Alo Bhi)[r][c][k]
//
// A and B are K-major BF16 ([rows][K] and [cols][K]); hi + lo represent an FP32
// value to ~16 significant bits, so the three products recover an FP32-grade
// dot product with FP32 accumulation in TMEM (the lo*lo term is below the
// FP32 accumulation error).  One 128 x BN output tile per CTA:
//   warp 0       TMA producer (one lane) over K blocks of 64, STAGES-deep ring
//   warp 1       TMEM allocation and MMA issue (one lane), tcgen05.commit to
//                free ring slots and to signal the accumulator
//   warps 2..9   epilogue: tcgen05.ld of TMEM lanes (two warps per lane
//                quadrant, one column half each)
// Every mbarrier wait is bounded by wall time; on expiry the CTA records an
// error code in *err, stops issuing work, and still releases its TMEM.
//
// Epilogues:
//   EPI_KERNEL   the sparse-GP kernel of Eqs. 2 and 13 on centred operands:
//                q = C + s_col + t_row, W = zeta delta^2 alpha q^(zeta-1) stored as
//                BF16 hi/lo, per-tile partial sums of delta^2 alpha q^zeta and of W
//   EPI_QPOW     per atom and sparse point, W' = zeta delta^2 q^(zeta-1) and
//                delta^2 q^zeta (FP32) for the K_NM rows
//   EPI_KNM      K_NM force rows: each Jacobian row scaled by +-W'[source atom],
//                rows summed per (target atom, direction) segment, cut segments
//                left as per-tile partials (EPI_KNM1: the form for K <= 256,
//                accumulator kept in TMEM)
//   EPI_STORE    FP32 store of C
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "gap_internal.h"
#include "tc_gemm.h"
#include "tc_prim.cuh"

namespace {

using namespace tcp;

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);

struct SharedTail {
    uint64_t full[4];
    uint64_t empty[4];
    uint64_t acc_full[2];    // MMA -> epilogue, per TMEM accumulator buffer
    uint64_t acc_empty[2];   // epilogue -> MMA (all epilogue threads arrive)
    uint32_t tmem_base;
    int abort;
    unsigned seg_mask[4][4];  // per column group of the epilogue, per lane quadrant
};

// K_NM force rows: scale row r by sign * W'[src][col], then sum the rows of
// each (target atom, xyz) segment of this 128-row tile.  Segments that are
// wholly inside the tile go to K; a segment cut by a tile edge leaves a
// partial sum in P[tile][slot] (slot 0: the tile's first segment) for the
// fix-up pass.  Runs on the 128 threads of one column half.
template <int BN>
__device__ __forceinline__ void epilogue_knm(const TcEpilogue &ep, const float (&acc)[BN / 2],
                                             unsigned char *stage_smem, SharedTail *tail, int quad, int lane,
                                             int half, int row0, int col0, int rows, int ncol, int rt)
{
    constexpr int HC = BN / 2;
    // [128 rows][32 columns] per half, column index XOR-swizzled by the row
    // so that row-wise stores and column-wise sums are both conflict-free;
    // then each row's signed source atom.
    float *buf = reinterpret_cast<float *>(stage_smem) + half * (128 * 32);
    int *rsrc = reinterpret_cast<int *>(reinterpret_cast<float *>(stage_smem) + 2 * 128 * 32) + half * 128;
    const int rl = quad * 32 + lane;  // row within tile
    const int r = row0 + rl;
    const int nvalid = rows - row0 < 128 ? rows - row0 : 128;
    int seg = -1;
    float trow = 0.f;
    rsrc[rl] = 0;
    if (rl < nvalid) {
        rsrc[rl] = ep.src_sign[r];
        seg = ep.seg[r];
        trow = ep.t_row[r];
    }
    bool start = rl < nvalid && (rl == 0 || ep.seg[r - 1] != seg);
    unsigned m = __ballot_sync(0xffffffffu, start);
    if (lane == 0) tail->seg_mask[half][quad] = m;
    named_barrier(1 + half, 128);
    unsigned masks[4] = {tail->seg_mask[half][0], tail->seg_mask[half][1], tail->seg_mask[half][2],
                         tail->seg_mask[half][3]};
    int nseg = __popc(masks[0]) + __popc(masks[1]) + __popc(masks[2]) + __popc(masks[3]);
#pragma unroll
    for (int ch = 0; ch < HC / 32; ++ch) {
        int cbase = half * HC + ch * 32;
        if (cbase < ncol) {
            int c0 = col0 + cbase;
#pragma unroll
            for (int k = 0; k < 32; ++k) buf[rl * 32 + (k ^ lane)] = acc[ch * 32 + k] + trow;
            named_barrier(1 + half, 128);
            // warp `quad` sums segments quad, quad + 4, ...; lane = column.
            // Each row is scaled by +-W'[source][column] here, where the
            // loads of W' are one coalesced 128-byte row segment per row.
            for (int sgi = quad; sgi < nseg; sgi += 4) {
                int b = sgi, q = 0;
                while (b >= __popc(masks[q])) { b -= __popc(masks[q]); ++q; }
                unsigned mm = masks[q];
                for (int t = 0; t < b; ++t) mm &= mm - 1;
                int s0 = q * 32 + __ffs(mm) - 1;
                int s1 = nvalid;
                {
                    unsigned rest = mm & (mm - 1);
                    if (rest) s1 = q * 32 + __ffs(rest) - 1;
                    else
                        for (int q2 = q + 1; q2 < 4; ++q2)
                            if (masks[q2]) { s1 = q2 * 32 + __ffs(masks[q2]) - 1; break; }
                }
                // the segment's destination, loaded ahead of the sums
                const int dest = ep.dest[row0 + s0];
                // eight rows at a time: eight W' loads in flight before the sums
                float sum = 0.f;
                int rr = s0;
                for (; rr + 8 <= s1; rr += 8) {
                    float wv[8];
                    int sv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        sv[u] = rsrc[rr + u];
                        wv[u] = __ldg(ep.Wp + (size_t)((sv[u] > 0 ? sv[u] : -sv[u]) - 1) * ep.ldwp + c0 + lane);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const float v = buf[(rr + u) * 32 + (lane ^ ((rr + u) & 31))];
                        sum = fmaf(sv[u] > 0 ? wv[u] : -wv[u], v, sum);
                    }
                }
                for (; rr < s1; ++rr) {
                    const int sv = rsrc[rr];
                    const float w = __ldg(ep.Wp + (size_t)((sv > 0 ? sv : -sv) - 1) * ep.ldwp + c0 + lane);
                    const float v = buf[rr * 32 + (lane ^ (rr & 31))];
                    sum = fmaf(sv > 0 ? w : -w, v, sum);
                }
                int col = c0 + lane;
                if (cbase + lane < ncol) {
                    if (dest >= 0) ep.K[(size_t)dest * ep.ldk + ep.col_out0 + col] = (double)sum;
                    else ep.P[((size_t)rt * 2 + (-1 - dest)) * ep.ldp + col] = sum;
                }
            }
            named_barrier(1 + half, 128);
        }
    }
}

// q^e for 0 <= e < 64 by square-and-multiply over the six bits of e: fully
// unrolled (e is the same for every thread), so the epilogue's element loops
// keep no data-dependent inner loop.
__device__ __forceinline__ float powi_small(float q, int e)
{
    float r = 1.f, b = q;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if ((e >> k) & 1) r *= b;
        b *= b;
    }
    return r;
}

// EPI_KNM with a single K chunk (K <= 256): the accumulator stays in TMEM and
// is read one 32-column slice at a time.  Each warp loads the W' slices of
// its 32 rows cooperatively (eight lanes per 128-byte row segment, the next
// slice's loads in flight during this slice's sums) into the staging rows;
// each thread then scales its row's accumulator slice by +-W' in place, so
// the segment sums read shared memory only.  Segment bounds and destinations
// are decoded once per tile.
constexpr int EPI_KNM1 = 4;
constexpr int kKnmStartBytes = 136;  // per group: up to 128 segment starts and the end
// Named barriers of the single-chunk K_NM epilogue's column groups (8 ..):
// clear of 3 and 4, which the kernel uses across all epilogue warps.
constexpr int kKnmGroupBar = 8;

// Lane L of a warp loads W' for rows 4 i + L / 8 (i < 8) of the warp's 32
// rows, columns c + 4 (L % 8) ... + 3; wsrc[i] is that row's source atom (-1:
// a row past the end of the GEMM, zeros).  c is a multiple of 32 inside the
// padded rows of W' (a multiple of 256 columns); c < 0 loads nothing.
__device__ __forceinline__ void knm_w_rows(const float *__restrict__ Wp, int ldwp, const int (&wsrc)[8], int c,
                                           int lane, float4 (&wq)[8])
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        wq[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c >= 0 && wsrc[i] >= 0)
            wq[i] = __ldg(reinterpret_cast<const float4 *>(Wp + (size_t)wsrc[i] * ldwp + c) + (lane & 7));
    }
}

template <int BN, int NG>
__device__ __forceinline__ void epilogue_knm1(const TcEpilogue &ep, uint32_t tacc, unsigned char *stage_smem,
                                              SharedTail *tail, int quad, int lane, int half, int row0, int col0,
                                              int rows, int ncol, int rt, const int (&wsrc)[8], float sgn,
                                              float4 (&wq)[8])
{
    // `half` is the warp's column group (NG groups of BN / NG columns, four
    // warps each, one per TMEM lane quadrant)
    constexpr int HC = BN / NG;
    // [128 rows][32 columns] per half; the 16-byte column group g of row R
    // sits at group g ^ (R & 7), so that 16-byte row accesses (a thread per
    // row, or eight lanes per row) and column reads (a lane per column) are
    // all free of bank conflicts.  Then per half the segments' destinations
    // and their start rows.
    float *buf = reinterpret_cast<float *>(stage_smem) + half * (128 * 32);
    int *sdest = reinterpret_cast<int *>(reinterpret_cast<float *>(stage_smem) + NG * 128 * 32);
    unsigned char *sstart = reinterpret_cast<unsigned char *>(sdest + NG * 128) + half * kKnmStartBytes;
    sdest += half * 128;
    const int rl = quad * 32 + lane;  // row within tile
    const int r = row0 + rl;
    const int nvalid = rows - row0 < 128 ? rows - row0 : 128;
    int seg = -1;
    float trow = 0.f;
    if (rl < nvalid) {
        seg = ep.seg[r];
        trow = ep.t_row[r];
    }
    const bool start = rl < nvalid && (rl == 0 || ep.seg[r - 1] != seg);
    const unsigned m = __ballot_sync(0xffffffffu, start);
    if (lane == 0) tail->seg_mask[half][quad] = m;
    named_barrier(kKnmGroupBar + half, 128);
    int before = 0, nseg = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = __popc(tail->seg_mask[half][q]);
        before += q < quad ? c : 0;
        nseg += c;
    }
    // segment k covers rows [sstart[k], sstart[k + 1]); visible to the half
    // after the first slice's barrier
    if (start) {
        const int k = before + __popc(m & ((1u << lane) - 1u));
        sstart[k] = (unsigned char)rl;
        sdest[k] = ep.dest[r];
    }
    if (rl == 0) sstart[nseg] = (unsigned char)nvalid;
    float *wrows = buf + quad * 32 * 32;  // this warp's 32 rows
    float *myrow = buf + rl * 32;
    for (int ch = 0; ch < HC / 32; ++ch) {
        const int cbase = half * HC + ch * 32;
        if (cbase >= ncol) break;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int rho = 4 * i + (lane >> 3);
            *reinterpret_cast<float4 *>(wrows + rho * 32 + 4 * ((lane & 7) ^ (rho & 7))) = wq[i];
        }
        __syncwarp();
        {
            float v[32];
            tmem_ld32(tacc + (uint32_t)cbase, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float4 *p = reinterpret_cast<float4 *>(myrow + 4 * (j ^ (lane & 7)));
                float4 w = *p;
                w.x = (sgn * w.x) * (v[4 * j] + trow);
                w.y = (sgn * w.y) * (v[4 * j + 1] + trow);
                w.z = (sgn * w.z) * (v[4 * j + 2] + trow);
                w.w = (sgn * w.w) * (v[4 * j + 3] + trow);
                *p = w;
            }
        }
        knm_w_rows(ep.Wp, ep.ldwp, wsrc, ch + 1 < HC / 32 && cbase + 32 < ncol ? col0 + cbase + 32 : -1, lane, wq);
        named_barrier(kKnmGroupBar + half, 128);
        // warp `quad` sums segments quad, quad + 4, ...; lane = column
        const int col = col0 + cbase + lane;
        const int cg = lane >> 2, cw = lane & 3;
        for (int sgi = quad; sgi < nseg; sgi += 4) {
            const int s0 = sstart[sgi], s1 = sstart[sgi + 1];
            const int dest = sdest[sgi];
            float sum = 0.f;
            int rr = s0;
            for (; rr + 8 <= s1; rr += 8) {
                float a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = buf[(rr + u) * 32 + 4 * (cg ^ ((rr + u) & 7)) + cw];
                sum += ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
            }
            for (; rr < s1; ++rr) sum += buf[rr * 32 + 4 * (cg ^ (rr & 7)) + cw];
            if (cbase + lane < ncol) {
                if (dest >= 0) ep.K[(size_t)dest * ep.ldk + ep.col_out0 + col] = (double)sum;
                else ep.P[((size_t)rt * 2 + (-1 - dest)) * ep.ldp + col] = sum;
            }
        }
        named_barrier(kKnmGroupBar + half, 128);
    }
}

// One GEMM problem of a launch: its operand maps (A hi / mid-or-lo / lo, B
// the same), sizes, first tile in the launch's tile order, and epilogue.
struct TcProblem {
    CUtensorMap mA[3], mB[3];
    int rows, cols, K, tile0;
    TcEpilogue ep;
};
// G problems in one persistent launch (the GEMMs of a batch's GPs): tiles
// are numbered problem after problem.
template <int G> struct TcProblems {
    int n, n_tiles;
    TcProblem p[G];
};

// The single-chunk K_NM instantiation (EPI_KNM1) returns to the tile loop
// before the register-accumulator path, which is unreachable there.
#pragma nv_diag_suppress 128

// NS = number of BF16 planes per operand: 2 (hi, lo: three MMAs per K step)
// or 3 (hi, mid, lo: the six products with plane-index sum <= 2, an
// FP32-grade product).
// EW = epilogue warps: 8 (two column groups), or 12 (three, the K_NM
// single-chunk epilogue on 192-column tiles).
template <int BN, int STAGES, int EPI, int NS, int G, int EW>
__global__ void __launch_bounds__(32 * (2 + EW), 1)
k_tc_gemm(const __grid_constant__ TcProblems<G> P, int *err)
{
    static_assert(BN == 128 || BN == 192 || BN == 256, "tile width");
    static_assert(NS == 2 || NS == 3, "planes");
    static_assert(EW == 8 || (EW == 12 && (EPI == EPI_KNM1 || EPI == EPI_KERNEL || EPI == EPI_STORE) && BN == 192),
                  "epilogue warps");
    constexpr int kThreads = 32 * (2 + EW);  // this instantiation's block
    constexpr int NG = EW / 4;               // epilogue column groups
    constexpr uint32_t TMEM_COLS = 2 * BN <= 256 ? 256 : 512;  // two accumulators, a power of two
    constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    constexpr uint32_t STAGE_BYTES = NS * A_BYTES + NS * B_BYTES;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    SharedTail *tail = reinterpret_cast<SharedTail *>(smem + STAGES * STAGE_BYTES);
    // epilogue scratch after the ring (the ring keeps filling for the next
    // tile while an epilogue runs): K_NM row sums, or per-column constants
    unsigned char *scratch = smem + STAGES * STAGE_BYTES + ((sizeof(SharedTail) + 127) & ~size_t(127));
    float *col_s = reinterpret_cast<float *>(scratch), *col_a = col_s + BN;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Persistent: CTA b takes tiles b, b + gridDim.x, ... (row tile major, so
    // the CTAs running at one time share A row tiles in L2).  The TMA ring
    // and the two TMEM accumulators continue across tiles, so the epilogue of
    // one tile overlaps the loads and MMAs of the next.
    const int n_tiles = P.n_tiles;
    // tile -> (problem, tile within it)
    auto locate = [&](int tile, int &gi, int &lt) {
        gi = 0;
#pragma unroll
        for (int q = 1; q < G; ++q)
            if (q < P.n && tile >= P.p[q].tile0) gi = q;
        lt = tile - P.p[gi].tile0;
    };

    // K is consumed in chunks of KC blocks; each chunk accumulates in a fresh
    // TMEM buffer (two, alternating) and the epilogue warps add the chunk
    // results into FP32 registers, so no tensor-core accumulation chain is
    // longer than KC * 4 * (3 or 6) MMAs.
    constexpr int KC = 4;
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
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tail->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tail->tmem_base;
    volatile int *abort_flag = &tail->abort;
    const unsigned long long wlim = P.p[0].ep.wait_ns ? P.p[0].ep.wait_ns : kWaitNs;
    const bool stall = P.p[0].ep.test_stall != 0;

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;  // k blocks issued by this CTA
            for (int tile = blockIdx.x; tile < n_tiles && !*abort_flag; tile += gridDim.x) {
                int gi, lt;
                locate(tile, gi, lt);
                const TcProblem &pr = P.p[gi];
                const int n_ct = (pr.cols + BN - 1) / BN, kblocks = (pr.K + BK - 1) / BK;
                const int row0 = (lt / n_ct) * BM, col0 = (lt % n_ct) * BN;
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    int s = g % STAGES, r = g / STAGES;
                    if (!mbar_wait(&tail->empty[s], (r & 1) ^ 1, abort_flag, wlim)) {
                        *abort_flag = 1;
                        atomicOr(err, 1);
                        break;
                    }
                    if (stall) continue;
                    unsigned char *st = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&tail->full[s], STAGE_BYTES);
                    tma_load_2d(st, &pr.mA[0], &tail->full[s], kb * BK, row0);
                    tma_load_2d(st + A_BYTES, &pr.mA[1], &tail->full[s], kb * BK, row0);
                    if (NS == 3) tma_load_2d(st + 2 * A_BYTES, &pr.mA[2], &tail->full[s], kb * BK, row0);
                    tma_load_2d(st + NS * A_BYTES, &pr.mB[0], &tail->full[s], kb * BK, col0);
                    tma_load_2d(st + NS * A_BYTES + B_BYTES, &pr.mB[1], &tail->full[s], kb * BK, col0);
                    if (NS == 3) tma_load_2d(st + NS * A_BYTES + 2 * B_BYTES, &pr.mB[2], &tail->full[s], kb * BK, col0);
                }
            }
            // drain: wait until the consumer has released every slot we filled
            int last = g - 1;
            for (int kb = last - STAGES + 1 < 0 ? 0 : last - STAGES + 1; kb <= last && !*abort_flag; ++kb) {
                int s = kb % STAGES, r = kb / STAGES;
                if (!mbar_wait(&tail->empty[s], r & 1, abort_flag, wlim)) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int g = 0, gc = 0;  // k blocks and K chunks consumed by this CTA
            int nchunks = 0;
            for (int tile = blockIdx.x; tile < n_tiles && !*abort_flag; tile += gridDim.x, gc += nchunks) {
                int gi, lt;
                locate(tile, gi, lt);
                const int K = P.p[gi].K, cols = P.p[gi].cols;
                const int n_ct = (cols + BN - 1) / BN, kblocks = (K + BK - 1) / BK;
                nchunks = (kblocks + KC - 1) / KC;
                int ncol = cols - (lt % n_ct) * BN;
                if (ncol > BN) ncol = BN;
                const uint32_t idesc = idesc_bf16((ncol + 15) & ~15);
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    const int q = gc + kb / KC, buf = q & 1, use = q >> 1;
                    const bool first = (kb % KC) == 0;
                    if (first && use >= 1 && !mbar_wait(&tail->acc_empty[buf], (use - 1) & 1, abort_flag, wlim)) {
                        *abort_flag = 1;
                        atomicOr(err, 8);
                        break;
                    }
                    int s = g % STAGES, r = g / STAGES;
                    if (!mbar_wait(&tail->full[s], r & 1, abort_flag, wlim)) {
                        *abort_flag = 1;
                        atomicOr(err, 2);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tacc = tmem + (uint32_t)(buf * BN);
                    uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                    uint32_t pa[3] = {sa, sa + A_BYTES, sa + 2 * A_BYTES};
                    uint32_t sb = sa + NS * A_BYTES;
                    uint32_t pb[3] = {sb, sb + B_BYTES, sb + 2 * B_BYTES};
                    int ksteps = (K - kb * BK) / 16;
                    if (ksteps > BK / 16) ksteps = BK / 16;
                    for (int kk = 0; kk < ksteps; ++kk) {
                        uint32_t off = kk * 32;
                        uint32_t acc0 = (first && kk == 0) ? 0u : 1u;
                        // plane pairs (i, j) with i + j < NS, largest products first
                        umma(tacc, sdesc_sw128(pa[0] + off), sdesc_sw128(pb[0] + off), idesc, acc0);
                        umma(tacc, sdesc_sw128(pa[0] + off), sdesc_sw128(pb[1] + off), idesc, 1u);
                        umma(tacc, sdesc_sw128(pa[1] + off), sdesc_sw128(pb[0] + off), idesc, 1u);
                        if (NS == 3) {
                            umma(tacc, sdesc_sw128(pa[1] + off), sdesc_sw128(pb[1] + off), idesc, 1u);
                            umma(tacc, sdesc_sw128(pa[0] + off), sdesc_sw128(pb[2] + off), idesc, 1u);
                            umma(tacc, sdesc_sw128(pa[2] + off), sdesc_sw128(pb[0] + off), idesc, 1u);
                        }
                    }
                    umma_commit(&tail->empty[s]);
                    if ((kb % KC) == KC - 1 || kb == kblocks - 1) umma_commit(&tail->acc_full[buf]);
                }
            }
        }
    } else {
        // epilogue warps
        const int ew = warp - 2;
        const int quad = warp & 3;        // TMEM lane quadrant this warp may access
        const int half = ew >> 2;         // column group (a half for EW = 8)
        constexpr int HC = BN / NG;         // columns per group
        int gc = 0;                         // K chunks consumed by this CTA
        int nchunks = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, gc += nchunks) {
            int gi, lt;
            locate(tile, gi, lt);
            const TcEpilogue &ep = P.p[gi].ep;
            const int rows = P.p[gi].rows, cols = P.p[gi].cols;
            const int n_ct = (cols + BN - 1) / BN;
            nchunks = ((P.p[gi].K + BK - 1) / BK + KC - 1) / KC;
            const int rt = lt / n_ct, ct = lt % n_ct;
            const int row0 = rt * BM, col0 = ct * BN;
            int ncol = cols - col0;
            if (ncol > BN) ncol = BN;
            const int r = row0 + quad * 32 + lane;
            if (EPI == EPI_KERNEL || EPI == EPI_QPOW) {
                // stage the per-column constants while the MMAs run (after every
                // epilogue thread has finished with the previous tile's)
                named_barrier(3, kThreads - 64);
                for (int c = threadIdx.x - 64; c < BN; c += kThreads - 64) {
                    // the column arrays are padded to 256; a 192-column tile
                    // can reach past them, where nothing is used
                    int cc = col0 + c;
                    col_s[c] = c < ncol ? ep.s_col[cc] : 0.f;
                    col_a[c] = c < ncol ? (EPI == EPI_KERNEL ? ep.alpha_col[cc] : 1.f) * ep.d2 : 0.f;
                }
                named_barrier(3, kThreads - 64);
            }
            if constexpr (EPI == EPI_KNM1) {
                // one K chunk: the epilogue reads the accumulator in TMEM and
                // releases the buffer when it is done
                const int buf = gc & 1, use = gc >> 1;
                // this row's sign and the source atoms of the rows whose W'
                // slices this lane loads; the first slice's loads are in
                // flight while the accumulator completes
                const int sv = r < rows ? ep.src_sign[r] : 0;
                int wsrc[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int ri = row0 + quad * 32 + 4 * i + (lane >> 3);
                    const int si = ri < rows ? ep.src_sign[ri] : 0;
                    wsrc[i] = si != 0 ? (si > 0 ? si : -si) - 1 : -1;
                }
                float4 wq[8];
                knm_w_rows(ep.Wp, ep.ldwp, wsrc, half * HC < ncol ? col0 + half * HC : -1, lane, wq);
                bool ok1 = mbar_wait(&tail->acc_full[buf], use & 1, abort_flag, wlim);
                if (!ok1) {
                    *abort_flag = 1;
                    atomicOr(err, 4);
                }
                tc_fence_after();
                ok1 = bar_and(4, kThreads - 64, ok1);
                if (!ok1) break;
                epilogue_knm1<BN, NG>(ep, tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * BN), scratch, tail,
                                  quad, lane, half, row0, col0, rows, ncol, rt, wsrc, sv > 0 ? 1.f : -1.f, wq);
                tc_fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tail->acc_empty[buf]))
                             : "memory");
                continue;
            }
            // promoted accumulation of the chunk results
            float acc[HC];
#pragma unroll
            for (int k = 0; k < HC; ++k) acc[k] = 0.f;
            bool ok = true;
            for (int c = 0; c < nchunks; ++c) {
                const int q = gc + c, buf = q & 1, use = q >> 1;
                if (!mbar_wait(&tail->acc_full[buf], use & 1, abort_flag, wlim)) {
                    *abort_flag = 1;
                    atomicOr(err, 4);
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int ch = 0; ch < HC / 32; ++ch) {
                    int cbase = half * HC + ch * 32;
                    if (cbase < ncol) {
                        float v[32];
                        tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * BN + cbase), v);
#pragma unroll
                        for (int k = 0; k < 32; ++k) acc[ch * 32 + k] += v[k];
                    }
                }
                tc_fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tail->acc_empty[buf]))
                             : "memory");
            }
            // every epilogue warp takes the same branch (the epilogues below use
            // named barriers), so a wait that expired in one warp stops them all
            ok = bar_and(4, kThreads - 64, ok);
            if (!ok) break;
            if constexpr (EPI == EPI_KNM) {
                epilogue_knm<BN>(ep, acc, scratch, tail, quad, lane, half, row0, col0, rows, ncol, rt);
            } else {
                float esum = 0.f, wsum = 0.f;
                const int zeta = ep.zeta;
#pragma unroll
                for (int ch = 0; ch < HC / 32; ++ch) {
                    int cbase = half * HC + ch * 32;   // column within tile
                    if (cbase >= ncol || r >= rows) continue;
                    const float *v = acc + ch * 32;
                    int c0 = col0 + cbase;
                    if (EPI == EPI_STORE) {
                        int orow = ep.row_map ? ep.row_map[r] : r;
                        float *out = ep.C + (size_t)orow * ep.ldc + c0;
                        if (cbase + 32 <= ncol && (ep.ldc & 3) == 0) {
#pragma unroll
                            for (int k = 0; k < 32; k += 4)
                                *reinterpret_cast<float4 *>(out + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                        } else {
#pragma unroll
                            for (int k = 0; k < 32; ++k)
                                if (cbase + k < ncol) out[k] = v[k];
                        }
                    } else if (EPI == EPI_QPOW) {
                        const float tr = ep.t_row[r];
                        int orow = ep.row_map[r];
                        float *pw = ep.Wp + (size_t)orow * ep.ldwp + c0, *pk = ep.kq + (size_t)orow * ep.ldwp + c0;
#pragma unroll
                        for (int k = 0; k < 32; k += 4) {
                            float wv[4], kv[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                float q = v[k + u] + col_s[cbase + k + u] + tr;
                                const float qz = powi_small(q, zeta - 1);
                                float a = col_a[cbase + k + u];
                                wv[u] = (float)zeta * a * qz;
                                kv[u] = a * qz * q;
                            }
                            *reinterpret_cast<float4 *>(pw + k) = make_float4(wv[0], wv[1], wv[2], wv[3]);
                            *reinterpret_cast<float4 *>(pk + k) = make_float4(kv[0], kv[1], kv[2], kv[3]);
                        }
                    } else {
                        const float tr = ep.t_row[r];
                        uint32_t hi[16], mid[16], lo[16];
#pragma unroll
                        for (int k = 0; k < 32; k += 2) {
                            float w2[2];
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                float q = v[k + u] + col_s[cbase + k + u] + tr;
                                const float qz = powi_small(q, zeta - 1);
                                float a = col_a[cbase + k + u];
                                esum += a * qz * q;
                                float w = (float)zeta * a * qz;
                                wsum += w;
                                w2[u] = w;
                            }
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(w2[0], w2[1]);
                            float2 hf = __bfloat1622float2(h2);
                            hi[k / 2] = *reinterpret_cast<uint32_t *>(&h2);
                            float r0 = w2[0] - hf.x, r1 = w2[1] - hf.y;
                            if (NS == 3) {
                                __nv_bfloat162 m2 = __floats2bfloat162_rn(r0, r1);
                                float2 mf = __bfloat1622float2(m2);
                                mid[k / 2] = *reinterpret_cast<uint32_t *>(&m2);
                                r0 -= mf.x;
                                r1 -= mf.y;
                            }
                            lo[k / 2] = pack_bf16(r0, r1);
                        }
                        if (ep.W_hi != nullptr) {  // energies only: W is not needed
                            uint4 *ph = reinterpret_cast<uint4 *>(ep.W_hi + (size_t)r * ep.ldw + c0);
                            uint4 *pl = reinterpret_cast<uint4 *>(ep.W_lo + (size_t)r * ep.ldw + c0);
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                ph[k] = make_uint4(hi[4 * k], hi[4 * k + 1], hi[4 * k + 2], hi[4 * k + 3]);
                                pl[k] = make_uint4(lo[4 * k], lo[4 * k + 1], lo[4 * k + 2], lo[4 * k + 3]);
                            }
                        }
                        if (NS == 3 && ep.W_mid != nullptr) {
                            uint4 *pm = reinterpret_cast<uint4 *>(ep.W_mid + (size_t)r * ep.ldw + c0);
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                pm[k] = make_uint4(mid[4 * k], mid[4 * k + 1], mid[4 * k + 2], mid[4 * k + 3]);
                        }
                    }
                }
                if (EPI == EPI_KERNEL && r < rows) {
                    int slot = ct * NG + half;
                    ep.eps_part[(size_t)r * ep.n_part + slot] = esum;
                    ep.wsum_part[(size_t)r * ep.n_part + slot] = wsum;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
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

int sm_count()
{
    static int n[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 132;
    if (!n[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 132;
        }
        n[dev] = v;
    }
    return n[dev];
}

gap_status make_map(CUtensorMap *m, const void *ptr, int rows, int cols, int ld, int box_rows)
{
    auto enc = encode_fn();
    if (!enc) {
        gap_set_error("cuTensorMapEncodeTiled is unavailable");
        return GAP_ECUDA;
    }
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (ld * 2) % 16) {
        gap_set_error("tensor map operand is not 16-byte aligned");
        return GAP_EINVAL;
    }
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        gap_set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
        return GAP_ECUDA;
    }
    return GAP_OK;
}

template <int BN, int STAGES, int EPI, int NS, int G, int EW = kEpiWarps>
gap_status launch_g(const TcOperands *ops, const TcEpilogue *eps, int n, int *err, cudaStream_t st)
{
    TcProblems<G> P;
    memset(&P, 0, sizeof(P));
    long tiles = 0;
    for (int q = 0; q < n; ++q) {
        const TcOperands &op = ops[q];
        if (op.rows <= 0 || op.cols <= 0) continue;
        TcProblem &pr = P.p[P.n];
        const __nv_bfloat16 *A[3] = {op.A_hi, NS == 3 ? op.A_mid : op.A_lo, op.A_lo};
        const __nv_bfloat16 *B[3] = {op.B_hi, NS == 3 ? op.B_mid : op.B_lo, op.B_lo};
        for (int pl = 0; pl < 3; ++pl) {
            GAP_TRY(make_map(&pr.mA[pl], A[pl], op.rows, op.K, op.lda, BM));
            GAP_TRY(make_map(&pr.mB[pl], B[pl], op.cols, op.K, op.ldb, BN));
        }
        pr.rows = op.rows;
        pr.cols = op.cols;
        pr.K = op.K;
        pr.tile0 = (int)tiles;
        pr.ep = eps[q];
        tiles += (long)((op.cols + BN - 1) / BN) * ((op.rows + BM - 1) / BM);
        ++P.n;
    }
    if (P.n == 0) return GAP_OK;
    if (tiles > 2147483647L) {
        gap_set_error("tensor-core GEMM: too many tiles");
        return GAP_EUNSUPPORTED;
    }
    P.n_tiles = (int)tiles;
    constexpr int NG = EW / 4;  // epilogue column groups
    const size_t scratch = EPI == EPI_KNM ? 2 * 128 * 32 * sizeof(float) + 2 * 128 * sizeof(int)
                           : EPI == EPI_KNM1
                               ? NG * (128 * 32 * sizeof(float) + 128 * sizeof(int) + kKnmStartBytes)
                               : 2 * BN * sizeof(float);
    size_t shm = (size_t)STAGES * (NS * BM * BK * 2 + NS * BN * BK * 2) + ((sizeof(SharedTail) + 127) & ~size_t(127)) +
                 scratch + 1024;
    auto kern = k_tc_gemm<BN, STAGES, EPI, NS, G, EW>;
    GAP_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    dim3 grid((unsigned)(tiles < sm_count() ? tiles : sm_count()));
    gap_count_launch();
    kern<<<grid, 32 * (2 + EW), shm, st>>>(P, err);
    return gap_cuda_status(cudaGetLastError(), "k_tc_gemm");
}

template <int BN, int STAGES, int EPI, int NS>
gap_status launch(const TcOperands &op, const TcEpilogue &ep, int *err, cudaStream_t st)
{
    return launch_g<BN, STAGES, EPI, NS, 1>(&op, &ep, 1, err, st);
}

// Up to kMaxGroups problems in one launch (the default tile variant).
constexpr int kMaxGroups = 4;
template <int NS>
gap_status launch_grouped(const TcOperands *ops, const TcEpilogue *eps, int n, int epi, int *err, cudaStream_t st)
{
    constexpr int BN = NS == 3 ? 128 : 256;
    if (epi == EPI_KERNEL) return launch_g<BN, 2, EPI_KERNEL, NS, kMaxGroups>(ops, eps, n, err, st);
    if (epi == EPI_STORE) return launch_g<BN, 2, EPI_STORE, NS, kMaxGroups>(ops, eps, n, err, st);
    gap_set_error("grouped tensor-core GEMM: energy and store epilogues only");
    return GAP_EINVAL;
}

// Tile variants of the two-plane split: (column tile, TMA stages, epilogue
// warps).  The three-plane split has one (128, 2): its 96 KB stages leave
// room for two.  The last variant (192 columns, twelve epilogue warps in
// three column groups) exists for the K_NM single-chunk epilogue only.
struct TileVariant {
    int bn, stages, ew;
};
constexpr TileVariant kVariants2[] = {{256, 2, 8}, {128, 2, 8}, {128, 3, 8}, {192, 2, 12}};
constexpr int kNumVariants2 = 4;
constexpr int kVariantKnmWide = 3;

bool variant_applies(int v, const TcOperands &op, int epi)
{
    return v < kVariantKnmWide ||
           (op.nsplit == 2 && ((epi == EPI_KNM && op.K <= 4 * BK) || epi == EPI_KERNEL || epi == EPI_STORE));
}

template <int BN, int ST, int NS>
gap_status launch_bn(const TcOperands &op, const TcEpilogue &ep, int epi, int *err, cudaStream_t st)
{
    if (epi == EPI_KERNEL) return launch<BN, ST, EPI_KERNEL, NS>(op, ep, err, st);
    if (epi == EPI_QPOW) return launch<BN, ST, EPI_QPOW, NS>(op, ep, err, st);
    if (epi == EPI_KNM)  // one K chunk of KC blocks: the TMEM-resident epilogue
        return op.K <= 4 * BK ? launch<BN, ST, EPI_KNM1, NS>(op, ep, err, st) : launch<BN, ST, EPI_KNM, NS>(op, ep, err, st);
    return launch<BN, ST, EPI_STORE, NS>(op, ep, err, st);
}

gap_status launch_variant(const TcOperands &op, const TcEpilogue &ep, int epi, int v, int *err, cudaStream_t st)
{
    if (op.nsplit == 3) return launch_bn<128, 2, 3>(op, ep, epi, err, st);
    if (v == kVariantKnmWide) {
        if (!variant_applies(v, op, epi)) {
            gap_set_error("tile variant for the K_NM and kernel-energy epilogues only");
            return GAP_EINVAL;
        }
        if (epi == EPI_KERNEL) return launch_g<192, 2, EPI_KERNEL, 2, 1, 12>(&op, &ep, 1, err, st);
        if (epi == EPI_STORE) return launch_g<192, 2, EPI_STORE, 2, 1, 12>(&op, &ep, 1, err, st);
        return launch_g<192, 2, EPI_KNM1, 2, 1, 12>(&op, &ep, 1, err, st);
    }

    switch (v) {
    case 1: return launch_bn<128, 2, 2>(op, ep, epi, err, st);
    case 2: return launch_bn<128, 3, 2>(op, ep, epi, err, st);
    default: return launch_bn<256, 2, 2>(op, ep, epi, err, st);
    }
}

// Tile autotuner.  A shape class is (device, epilogue, planes, K, columns,
// ceil(log2(rows))).  The first call of a class outside stream capture times
// every variant on that call's own operands and outputs (CUDA events on the
// call's stream: one warm-up launch, then the best of two) and keeps the
// fastest; every later call, and any call under capture, reuses the choice
// (the default variant while none is known).  All variants compute the same
// values; their outputs are rewritten by the call that follows.
struct TuneKey {
    int dev, epi, nsplit, K, cols, rlog;
    bool operator<(const TuneKey &o) const
    {
        if (dev != o.dev) return dev < o.dev;
        if (epi != o.epi) return epi < o.epi;
        if (nsplit != o.nsplit) return nsplit < o.nsplit;
        if (K != o.K) return K < o.K;
        if (cols != o.cols) return cols < o.cols;
        return rlog < o.rlog;
    }
};
struct TuneEntry {
    int variant;
    float ms[kNumVariants2];
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;
std::vector<std::pair<TuneKey, TuneEntry>> g_tune_log;  // in the order tuned

int rows_log2(int rows)
{
    int r = 0;
    while ((1 << r) < rows && r < 30) ++r;
    return r;
}

// The column tile a variant uses for this call (the energy epilogue's
// partial sums are laid out per column tile).
TcEpilogue with_parts(const TcEpilogue &ep, int epi, const TcOperands &op, const TileVariant &tv)
{
    TcEpilogue e = ep;
    if (epi == EPI_KERNEL) e.n_part = tv.ew / 4 * ((op.cols + tv.bn - 1) / tv.bn);
    return e;
}

}  // namespace

int gap_tc_max_parts(int cols)
{
    int m = 0;
    for (const TileVariant &tv : kVariants2) {
        const int p = tv.ew / 4 * ((cols + tv.bn - 1) / tv.bn);
        if (p > m) m = p;
    }
    return m;
}

namespace {
std::atomic<int> g_force_variant{-1};  // gap_tc_force_variant (test hook)

int forced_variant(const TcOperands &op, int epi)
{
    const int v = g_force_variant.load();
    return v >= 0 && v < kNumVariants2 && op.nsplit == 2 && variant_applies(v, op, epi) ? v : -1;
}
}  // namespace

void gap_tc_force_variant(int v) { g_force_variant.store(v < 0 ? -1 : v); }

int gap_tc_plan(const TcOperands &op, const TcEpilogue &ep, int epi, int *err, cudaStream_t st, int *groups)
{
    if (groups) *groups = 2;
    if (const int fv = forced_variant(op, epi); fv >= 0) {
        if (groups) *groups = kVariants2[fv].ew / 4;
        return kVariants2[fv].bn;
    }
    if (op.nsplit == 3 || op.rows <= 0 || op.cols <= 0) return 128;
    if (ep.test_stall) return kVariants2[0].bn;  // the timeout test: nothing to time
    int dev = 0;
    cudaGetDevice(&dev);
    const TuneKey key{dev, epi, op.nsplit, op.K, op.cols, rows_log2(op.rows)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            if (groups) *groups = kVariants2[it->second.variant].ew / 4;
            return kVariants2[it->second.variant].bn;
        }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return kVariants2[0].bn;
    }
    TuneEntry e{0, {}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return kVariants2[0].bn;
    }
    float best = 1e30f;
    for (int v = 0; v < kNumVariants2; ++v) {
        e.ms[v] = 1e30f;
        if (!variant_applies(v, op, epi)) {
            e.ms[v] = -1.f;  // not a candidate for this class
            continue;
        }
        const TcEpilogue ev = with_parts(ep, epi, op, kVariants2[v]);
        if (launch_variant(op, ev, epi, v, err, st) != GAP_OK) continue;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, st);
            if (launch_variant(op, ev, epi, v, err, st) != GAP_OK) break;
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < e.ms[v]) e.ms[v] = ms;
        }
        if (e.ms[v] < best) {
            best = e.ms[v];
            e.variant = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune.emplace(key, e).second) g_tune_log.emplace_back(key, e);
    if (groups) *groups = kVariants2[e.variant].ew / 4;
    return kVariants2[e.variant].bn;
}

int gap_tc_tuned_count()
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (int)g_tune_log.size();
}

bool gap_tc_tuned_entry(int k, int *fields, float *ms)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (k < 0 || k >= (int)g_tune_log.size()) return false;
    const TuneKey &key = g_tune_log[k].first;
    const TuneEntry &e = g_tune_log[k].second;
    const int f[8] = {key.epi, key.nsplit, key.K, key.cols, key.rlog, kVariants2[e.variant].bn,
                      kVariants2[e.variant].stages, key.dev};
    for (int i = 0; i < 8; ++i) fields[i] = f[i];
    for (int v = 0; v < kNumVariants2; ++v) ms[v] = e.ms[v];
    return true;
}

gap_status gap_tc_gemm(const TcOperands &op, const TcEpilogue &ep, int epi, int *err, cudaStream_t st)
{
    if (op.rows <= 0 || op.cols <= 0) return GAP_OK;
    if ((long)((op.rows + 127) / 128) * ((op.cols + 127) / 128 + 1) > 2147483647L) {
        gap_set_error("tensor-core GEMM: too many tiles");
        return GAP_EUNSUPPORTED;
    }
    if (op.K <= 0 || op.K % 16) {
        gap_set_error("tensor-core GEMM needs K to be a positive multiple of 16");
        return GAP_EINVAL;
    }
    if (op.nsplit == 3) {
        if (!op.A_mid || !op.B_mid) {
            gap_set_error("three-plane GEMM needs mid planes");
            return GAP_EINVAL;
        }
        return launch_variant(op, ep, epi, 0, err, st);
    }
    if (const int fv = forced_variant(op, epi); fv >= 0)
        return launch_variant(op, with_parts(ep, epi, op, kVariants2[fv]), epi, fv, err, st);
    const int bn = gap_tc_plan(op, ep, epi, err, st);
    int v = 0;
    for (int k = 0; k < kNumVariants2; ++k)
        if (kVariants2[k].bn == bn) { v = k; break; }
    {
        // the planned variant (the plan returns its column tile; look up the
        // full entry for the stage count)
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(TuneKey{dev, epi, op.nsplit, op.K, op.cols, rows_log2(op.rows)});
        if (it != g_tune.end()) v = it->second.variant;
    }
    return launch_variant(op, with_parts(ep, epi, op, kVariants2[v]), epi, v, err, st);
}

int gap_tc_grouped_col_tile(int nsplit) { return nsplit == 3 ? 128 : 256; }

gap_status gap_tc_gemm_grouped(const TcOperands *ops, const TcEpilogue *eps, int n, int epi, int *err, cudaStream_t st)
{
    for (int q0 = 0; q0 < n; q0 += kMaxGroups) {
        const int m = n - q0 < kMaxGroups ? n - q0 : kMaxGroups;
        for (int q = q0; q < q0 + m; ++q) {
            if (ops[q].rows <= 0 || ops[q].cols <= 0) continue;
            if (ops[q].K <= 0 || ops[q].K % 16 || ops[q].nsplit != ops[q0].nsplit ||
                (ops[q].nsplit == 3 && (!ops[q].A_mid || !ops[q].B_mid))) {
                gap_set_error("grouped tensor-core GEMM: bad problem");
                return GAP_EINVAL;
            }
        }
        GAP_TRY(ops[q0].nsplit == 3 ? launch_grouped<3>(ops + q0, eps + q0, m, epi, err, st)
                                    : launch_grouped<2>(ops + q0, eps + q0, m, epi, err, st));
    }
    return GAP_OK;
}
