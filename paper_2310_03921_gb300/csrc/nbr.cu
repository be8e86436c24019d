// Cell-list neighbour search with periodic images.
//
// Every directed pair (i, j, T) with |r_j + T - r_i| < r_c is listed, where
// T runs over all lattice translations (j = i allowed for T != 0): the
// connectivity "based on the cutoff" of Sec. 3.1.1 and the sum over all
// neighbours of Eq. 19.  Per configuration, fractional coordinates are
// wrapped into [0, 1) along periodic axes and binned on a grid whose bins are
// at least r_c wide in perpendicular width, or, for cells thinner than r_c,
// one bin per axis searched over several images.  Each atom's list is sorted
// by (j, shift), so the output does not depend on the order in which atomics
// filled the bins.
#include "gap_internal.h"
#include "nbr.h"

#include <cmath>
#include <vector>

namespace {

constexpr int kShiftBias = 128;

__device__ __forceinline__ long long pair_key(int j, int sx, int sy, int sz)
{
    return ((long long)j << 24) | ((long long)(sx + kShiftBias) << 16) | ((long long)(sy + kShiftBias) << 8) |
           (long long)(sz + kShiftBias);
}

__device__ __forceinline__ int config_of(const int *offsets, int n_configs, int i)
{
    int lo = 0, hi = n_configs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_bin(int n, const double *__restrict__ pos, const int *__restrict__ offsets, int n_configs,
                      const CellGeom *__restrict__ geo, double *__restrict__ frac, float4 *__restrict__ frac32,
                      int *__restrict__ atom_cfg, int *__restrict__ atom_bin, int *__restrict__ bin_count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = config_of(offsets, n_configs, i);
    const CellGeom &g = geo[c];
    double p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    int b[3];
    for (int k = 0; k < 3; ++k) {
        double s = p[0] * g.inv[k] + p[1] * g.inv[3 + k] + p[2] * g.inv[6 + k];
        if (g.pbc[k]) {
            s -= floor(s);
            if (s >= 1.0) s = 0.0;
        }
        int bk = (int)floor(s * g.nb[k]);
        bk = bk < 0 ? 0 : (bk >= g.nb[k] ? g.nb[k] - 1 : bk);
        frac[3 * i + k] = s;
        b[k] = bk;
    }
    int gb = g.bin0 + (b[0] * g.nb[1] + b[1]) * g.nb[2] + b[2];
    // w = 1 marks coordinates within [-4, 4] (always so along periodic
    // directions), where the FP32 copy is close enough for the prefilter
    const bool near = fabs(frac[3 * i]) <= 4.0 && fabs(frac[3 * i + 1]) <= 4.0 && fabs(frac[3 * i + 2]) <= 4.0;
    frac32[i] = make_float4((float)frac[3 * i], (float)frac[3 * i + 1], (float)frac[3 * i + 2], near ? 1.f : 0.f);
    atom_cfg[i] = c;
    atom_bin[i] = gb;
    atomicAdd(&bin_count[gb], 1);
}

__global__ void k_scatter(int n, const int *__restrict__ atom_bin, const int *__restrict__ bin_start,
                          int *__restrict__ bin_fill, int *__restrict__ bin_atoms)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int gb = atom_bin[i];
    int slot = atomicAdd(&bin_fill[gb], 1);
    bin_atoms[bin_start[gb] + slot] = i;
}

// Visits every candidate (j, shift) of atom i, one warp per atom, 32 at a
// time; f(hit, j, sx, sy, sz, v, r2) is called by every lane with uniform
// control flow (it may use warp votes), hit marking a pair within the
// cutoff.  The bins around the atom ((2R+1)^3, 32 at a time: lane b resolves
// bin b's periodic shift and atom range) are flattened into one run of
// candidates, which the lanes take 32 at a time through an FP32 prefilter:
// the cutoff widened by 5 10^-4 rc + 10^-5 of the cell's edge lengths, far
// beyond the error of the FP32 fractional coordinates (|s| <= 4: ~5 10^-7
// of the edges; atoms outside that range, beyond the box of a non-periodic
// direction, skip it).  The survivors (~15%) queue in shared memory and
// take the exact FP64 test 32 at a time, so that every FP64 instruction works
// on a full warp (GB300's FP64 pipe takes about 64 cycles per warp
// instruction, whatever the active lanes).  The pair set is the FP64 one.
// SURE (counting only): a candidate whose FP32 distance is below the cutoff
// narrowed by the same margin is inside for FP64 too; it is counted in
// sure_hits without the exact test, which then sees only the thin shell
// between the two bounds.
constexpr int kNbrQueue = 64;

template <bool SURE, typename F>
__device__ __forceinline__ void warp_candidates(int i, int lane, const double *__restrict__ frac,
                                                const float4 *__restrict__ frac32, const int *__restrict__ atom_cfg,
                                                const CellGeom *__restrict__ geo, const int *__restrict__ bin_start,
                                                const int *__restrict__ bin_atoms, int2 *__restrict__ queue, F &&f,
                                                int &sure_hits)
{
    const CellGeom &g = geo[atom_cfg[i]];
    const double si0 = frac[3 * i], si1 = frac[3 * i + 1], si2 = frac[3 * i + 2];
    const float4 s32 = frac32[i];
    int b[3];
    const double si[3] = {si0, si1, si2};
    for (int k = 0; k < 3; ++k) {
        int bk = (int)floor(si[k] * g.nb[k]);
        b[k] = bk < 0 ? 0 : (bk >= g.nb[k] ? g.nb[k] - 1 : bk);
    }
    const unsigned lt = (1u << lane) - 1u;
    int qn = 0;  // queued candidates
    // the exact test of queue[0 .. cnt) (cnt <= 32), one per lane
    auto drain = [&](int cnt) {
        bool hit = false;
        int j = -1, sx = 0, sy = 0, sz = 0;
        double v[3] = {0.0, 0.0, 0.0}, r2 = 0.0;
        if (lane < cnt) {
            const int2 e = queue[lane];
            j = e.x;
            sx = ((e.y >> 16) & 0xff) - 128;
            sy = ((e.y >> 8) & 0xff) - 128;
            sz = (e.y & 0xff) - 128;
            const double ds0 = frac[3 * j] + sx - si0, ds1 = frac[3 * j + 1] + sy - si1, ds2 = frac[3 * j + 2] + sz - si2;
            for (int a = 0; a < 3; ++a) v[a] = ds0 * g.cell[a] + ds1 * g.cell[3 + a] + ds2 * g.cell[6 + a];
            r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            hit = r2 < g.rc2;
        }
        f(hit, j, sx, sy, sz, v, r2);
    };
    const int wx = 2 * g.R[0] + 1, wy = 2 * g.R[1] + 1, wz = 2 * g.R[2] + 1, nbins = wx * wy * wz;
    for (int b0 = 0; b0 < nbins; b0 += 32) {
        int st = 0, cnt = 0, shift = 0;
        const int bb = b0 + lane;
        if (bb < nbins) {
            const int dz = bb % wz - g.R[2], dy = (bb / wz) % wy - g.R[1], dx = bb / (wz * wy) - g.R[0];
            int nx = b[0] + dx, ny = b[1] + dy, nz = b[2] + dz, sxl = 0, syl = 0, szl = 0;
            bool ok = true;
            if (g.pbc[0]) { sxl = (int)floor((double)nx / g.nb[0]); nx -= sxl * g.nb[0]; }
            else ok = ok && nx >= 0 && nx < g.nb[0];
            if (g.pbc[1]) { syl = (int)floor((double)ny / g.nb[1]); ny -= syl * g.nb[1]; }
            else ok = ok && ny >= 0 && ny < g.nb[1];
            if (g.pbc[2]) { szl = (int)floor((double)nz / g.nb[2]); nz -= szl * g.nb[2]; }
            else ok = ok && nz >= 0 && nz < g.nb[2];
            if (ok) {
                const int gb = g.bin0 + (nx * g.nb[1] + ny) * g.nb[2] + nz;
                st = bin_start[gb];
                cnt = bin_start[gb + 1] - st;
            }
            shift = ((sxl + 128) << 16) | ((syl + 128) << 8) | (szl + 128);
        }
        // exclusive prefix of the bin sizes: candidate c of this chunk lies in
        // the last bin whose prefix is <= c
        int pre = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += t;
        }
        const int total = __shfl_sync(0xffffffffu, pre, 31);
        pre -= cnt;
        for (int c0 = 0; c0 < total; c0 += 32) {
            const int c = c0 + lane;
            int lo = 0;  // binary search for the bin of c
            for (int step = 16; step; step >>= 1) {
                const int p = __shfl_sync(0xffffffffu, pre, lo + step);
                if (c >= p && lo + step < 32) lo += step;
            }
            const int bst = __shfl_sync(0xffffffffu, st, lo), bpre = __shfl_sync(0xffffffffu, pre, lo);
            const int bsh = __shfl_sync(0xffffffffu, shift, lo);
            bool pass = false, sure = false;
            int j = -1;
            if (c < total) {
                j = bin_atoms[bst + (c - bpre)];
                const int sx = ((bsh >> 16) & 0xff) - 128, sy = ((bsh >> 8) & 0xff) - 128, sz = (bsh & 0xff) - 128;
                if (!(j == i && sx == 0 && sy == 0 && sz == 0)) {
                    pass = true;
                    const float4 f32 = frac32[j];
                    if (s32.w != 0.f && f32.w != 0.f) {
                        const float d0 = (f32.x - s32.x) + (float)sx, d1 = (f32.y - s32.y) + (float)sy,
                                    d2 = (f32.z - s32.z) + (float)sz;
                        float r2f = 0.f;
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const float va = d0 * g.cell32[a] + d1 * g.cell32[3 + a] + d2 * g.cell32[6 + a];
                            r2f += va * va;
                        }
                        pass = r2f < g.rc2_loose;
                        if (SURE && r2f < g.rc2_tight) {
                            sure = true;
                            pass = false;
                        }
                    }
                }
            }
            if (SURE) sure_hits += __popc(__ballot_sync(0xffffffffu, sure));
            const unsigned pm = __ballot_sync(0xffffffffu, pass);
            if (pass) queue[qn + __popc(pm & lt)] = make_int2(j, bsh);
            qn += __popc(pm);
            __syncwarp();
            if (qn >= 32) {
                drain(32);
                __syncwarp();
                qn -= 32;
                if (lane < qn) queue[lane] = queue[32 + lane];
                __syncwarp();
            }
        }
    }
    if (qn > 0) drain(qn);
}

constexpr int kNbrWarps = 4;   // warps (atoms) per block
constexpr int kNbrSort = 128;   // pairs per atom sorted in shared memory

__global__ void __launch_bounds__(32 * kNbrWarps)
k_count_warp(int n, const double *__restrict__ frac, const float4 *__restrict__ frac32,
             const int *__restrict__ atom_cfg, const CellGeom *__restrict__ geo, const int *__restrict__ bin_start,
             const int *__restrict__ bin_atoms, int *__restrict__ counts)
{
    __shared__ int2 queue[kNbrWarps][kNbrQueue];
    const int i = blockIdx.x * kNbrWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    int c = 0, sure = 0;
    warp_candidates<true>(i, lane, frac, frac32, atom_cfg, geo, bin_start, bin_atoms, queue[threadIdx.x >> 5],
                          [&](bool hit, int, int, int, int, const double *, double) {
                              c += __popc(__ballot_sync(0xffffffffu, hit));
                          },
                          sure);
    if (lane == 0) counts[i] = c + sure;
}

// The pairs of atom i sorted by (j, shift): gathered in shared memory and
// placed by rank (keys are distinct), or, beyond kNbrSort pairs, written in
// scan order and insertion-sorted by one lane.
__global__ void __launch_bounds__(32 * kNbrWarps)
k_fill_warp(int n, const double *__restrict__ frac, const float4 *__restrict__ frac32,
            const int *__restrict__ atom_cfg, const CellGeom *__restrict__ geo, const int *__restrict__ bin_start,
            const int *__restrict__ bin_atoms, const int *__restrict__ offsets, int cap,
            long long *__restrict__ keys, int *__restrict__ nbr_j, D4 *__restrict__ vec64,
            float4 *__restrict__ vec32, int *__restrict__ err)
{
    __shared__ long long skey[kNbrWarps][kNbrSort];
    __shared__ D4 svec[kNbrWarps][kNbrSort];
    __shared__ int2 queue[kNbrWarps][kNbrQueue];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kNbrWarps + wi;
    if (i >= n) return;
    const int p0 = offsets[i], p1 = offsets[i + 1], np = p1 - p0;
    if (p1 > cap) {
        if (lane == 0) atomicOr(err, 1);
        return;
    }
    const bool local = np <= kNbrSort;
    int w = 0;  // pairs found so far
    int no_sure = 0;
    warp_candidates<false>(i, lane, frac, frac32, atom_cfg, geo, bin_start, bin_atoms, queue[wi],
                    [&](bool hit, int j, int sx, int sy, int sz, const double *v, double r2) {
                        const unsigned m = __ballot_sync(0xffffffffu, hit);
                        if (hit) {
                            const int pos = w + __popc(m & ((1u << lane) - 1u));
                            if (pos < np) {
                                const long long key = pair_key(j, sx, sy, sz);
                                const D4 d{v[0], v[1], v[2], sqrt(r2)};
                                if (local) {
                                    skey[wi][pos] = key;
                                    svec[wi][pos] = d;
                                } else {
                                    keys[p0 + pos] = key;
                                    vec64[p0 + pos] = d;
                                }
                            }
                        }
                        w += __popc(m);
                    },
                    no_sure);
    if (w != np) {
        if (lane == 0) atomicOr(err, 2);
        return;
    }
    if (local) {
        __syncwarp();
        for (int e = lane; e < np; e += 32) {
            const long long k = skey[wi][e];
            int rank = 0;
            for (int e2 = 0; e2 < np; ++e2) rank += skey[wi][e2] < k ? 1 : 0;
            const D4 d = svec[wi][e];
            keys[p0 + rank] = k;
            vec64[p0 + rank] = d;
            nbr_j[p0 + rank] = (int)(k >> 24);
            vec32[p0 + rank] = make_float4((float)d.x, (float)d.y, (float)d.z, (float)d.w);
        }
        return;
    }
    __syncwarp();
    if (lane == 0) {
        for (int a = p0 + 1; a < p1; ++a) {
            const long long k = keys[a];
            const D4 v = vec64[a];
            int bq = a - 1;
            while (bq >= p0 && keys[bq] > k) {
                keys[bq + 1] = keys[bq];
                vec64[bq + 1] = vec64[bq];
                --bq;
            }
            keys[bq + 1] = k;
            vec64[bq + 1] = v;
        }
    }
    __syncwarp();
    for (int a = p0 + lane; a < p1; a += 32) {
        nbr_j[a] = (int)(keys[a] >> 24);
        const D4 v = vec64[a];
        vec32[a] = make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
    }
}

// Graph mode: a build with more pairs than the arrays hold empties every
// neighbour list (so that no later kernel reads past the arrays) and flags it.
__global__ void k_cap_offsets(int n, int cap, const int *__restrict__ total, int *__restrict__ offsets,
                              int *__restrict__ used, int *__restrict__ err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = *total;
    if (t > cap) {
        if (i <= n) offsets[i] = 0;
        if (i == 0) {
            *used = 0;
            atomicOr(err, 1);
        }
    } else if (i == 0) {
        *used = t;
    }
}

__global__ void k_reverse(int n, const int *__restrict__ offsets, const long long *__restrict__ keys,
                          int *__restrict__ rev, int *__restrict__ err)
{
    int i = blockIdx.x;
    for (int p = offsets[i] + threadIdx.x; p < offsets[i + 1]; p += blockDim.x) {
        long long k = keys[p];
        int j = (int)(k >> 24);
        int sx = (int)((k >> 16) & 255) - kShiftBias, sy = (int)((k >> 8) & 255) - kShiftBias,
            sz = (int)(k & 255) - kShiftBias;
        long long want = pair_key(i, -sx, -sy, -sz);
        int lo = offsets[j], hi = offsets[j + 1] - 1, found = -1;
        while (lo <= hi) {
            int mid = (lo + hi) >> 1;
            long long km = keys[mid];
            if (km == want) { found = mid; break; }
            if (km < want) lo = mid + 1;
            else hi = mid - 1;
        }
        rev[p] = found;
        if (found < 0) atomicOr(err, 4);
    }
}

// ------------------------------------------------- exclusive scan of ints
__global__ void k_scan_blocks(const int *__restrict__ in, int n, int *__restrict__ out, int *__restrict__ sums)
{
    __shared__ int warp_tot[32];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int v = i < n ? in[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    int base = w > 0 ? warp_tot[w - 1] : 0;
    if (i < n) out[i] = base + x - v;
    if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = base + x;
}

__global__ void k_scan_add(int *__restrict__ out, int n, const int *__restrict__ block_off, int *__restrict__ total,
                           const int *__restrict__ in)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += block_off[blockIdx.x];
    if (i == n - 1) {
        out[n] = out[i] + in[i];
        if (total) *total = out[n];
    }
}

}  // namespace

// Exclusive scan of n ints into out[0..n] (out[n] = total); uses tmp of size
// 2 * ceil(n / 1024) + 2 ints.  Recursive over block sums.
gap_status gap_scan(const int *in, int n, int *out, int *tmp, int *total, cudaStream_t st)
{
    if (n <= 0) {
        GAP_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(int), st));
        if (total) GAP_TRY_CUDA(cudaMemsetAsync(total, 0, sizeof(int), st));
        return GAP_OK;
    }
    const int B = 1024;
    int nb = (n + B - 1) / B;
    int *sums = tmp, *offs = tmp + nb + 1;
    gap_count_launch();
    k_scan_blocks<<<nb, B, 0, st>>>(in, n, out, sums);
    GAP_TRY_CUDA(cudaGetLastError());
    if (nb > 1) {
        GAP_TRY(gap_scan(sums, nb, offs, tmp + 2 * nb + 2, nullptr, st));
    } else {
        GAP_TRY_CUDA(cudaMemsetAsync(offs, 0, sizeof(int), st));
    }
    gap_count_launch();
    k_scan_add<<<nb, B, 0, st>>>(out, n, offs, total, in);
    GAP_TRY_CUDA(cudaGetLastError());
    return GAP_OK;
}

size_t gap_scan_tmp_ints(int n)
{
    size_t t = 0;
    while (n > 1) {
        int nb = (n + 1023) / 1024;
        t += 2 * (size_t)nb + 2;
        n = nb;
    }
    return t + 4;
}

// Host-side geometry of each configuration's bin grid.
gap_status gap_cell_geometry(const gap_batch *b, double rc, std::vector<CellGeom> &geo, int &n_bins)
{
    geo.resize(b->n_configs);
    n_bins = 0;
    for (int c = 0; c < b->n_configs; ++c) {
        CellGeom &g = geo[c];
        const double *m = b->cell + 9 * c;
        double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
                     m[2] * (m[3] * m[7] - m[4] * m[6]);
        if (!(std::fabs(det) > 1e-12)) {
            gap_set_error("cell of configuration " + std::to_string(c) + " is singular");
            return GAP_EINVAL;
        }
        double inv[9] = {(m[4] * m[8] - m[5] * m[7]) / det, (m[2] * m[7] - m[1] * m[8]) / det,
                         (m[1] * m[5] - m[2] * m[4]) / det, (m[5] * m[6] - m[3] * m[8]) / det,
                         (m[0] * m[8] - m[2] * m[6]) / det, (m[2] * m[3] - m[0] * m[5]) / det,
                         (m[3] * m[7] - m[4] * m[6]) / det, (m[1] * m[6] - m[0] * m[7]) / det,
                         (m[0] * m[4] - m[1] * m[3]) / det};
        long long nbins = 1;
        for (int k = 0; k < 3; ++k) {
            double width = 1.0 / std::sqrt(inv[k] * inv[k] + inv[3 + k] * inv[3 + k] + inv[6 + k] * inv[6 + k]);
            int nb = (int)std::floor(width / rc);
            if (nb < 1) nb = 1;
            if (nb > 1024) nb = 1024;
            int R = (int)std::ceil(rc * nb / width - 1e-12);
            if (R < 1) R = 1;
            g.pbc[k] = b->pbc[3 * c + k] ? 1 : 0;
            if (g.pbc[k] && R > 60) {
                gap_set_error("cell of configuration " + std::to_string(c) + " is too thin for the cutoff");
                return GAP_EINVAL;
            }
            g.nb[k] = nb;
            g.R[k] = R;
            nbins *= nb;
        }
        for (int k = 0; k < 9; ++k) {
            g.cell[k] = m[k];
            g.inv[k] = inv[k];
            g.cell32[k] = (float)m[k];
        }
        g.rc2 = rc * rc;
        // FP32 fractional coordinates carry ~1.2e-7 of the cell per component:
        // a bound well above that error in Cartesian length
        double span = 0.0;
        for (int k = 0; k < 3; ++k) span += std::sqrt(m[3 * k] * m[3 * k] + m[3 * k + 1] * m[3 * k + 1] + m[3 * k + 2] * m[3 * k + 2]);
        const double rl = rc * (1.0 + 5e-4) + 1e-5 * span, rt = rc * (1.0 - 5e-4) - 1e-5 * span;
        g.rc2_loose = (float)(rl * rl);
        g.rc2_tight = rt > 0.0 ? (float)(rt * rt) : 0.f;
        g.bin0 = n_bins;
        if ((long long)n_bins + nbins > (1LL << 30)) {
            gap_set_error("too many neighbour bins");
            return GAP_EINVAL;
        }
        n_bins += (int)nbins;
    }
    return GAP_OK;
}

gap_status gap_neighbours(NbrWork &w, const gap_batch *b, const double *d_pos, double rc, cudaStream_t st)
{
    int n = b->n_atoms;
    std::vector<CellGeom> geo;
    int n_bins = 0;
    GAP_TRY(gap_cell_geometry(b, rc, geo, n_bins));
    GAP_TRY(w.reserve_atoms(n, b->n_configs, n_bins));
    if (!w.graph) {
        GAP_TRY_CUDA(cudaMemcpyAsync(w.geo, geo.data(), sizeof(CellGeom) * geo.size(), cudaMemcpyHostToDevice, st));
        GAP_TRY_CUDA(cudaMemcpyAsync(w.cfg_offsets, b->config_offsets, sizeof(int) * (b->n_configs + 1),
                                     cudaMemcpyHostToDevice, st));
    }
    GAP_TRY_CUDA(cudaMemsetAsync(w.bin_count, 0, sizeof(int) * (n_bins + 1), st));
    GAP_TRY_CUDA(cudaMemsetAsync(w.bin_fill, 0, sizeof(int) * (n_bins + 1), st));
    GAP_TRY_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    const int T = 128;
    int gridN = (n + T - 1) / T;
    if (n > 0) {
        gap_count_launch();
        k_bin<<<gridN, T, 0, st>>>(n, d_pos, w.cfg_offsets, b->n_configs, w.geo, w.frac, w.frac32, w.atom_cfg,
                                   w.atom_bin, w.bin_count);
        GAP_TRY_CUDA(cudaGetLastError());
    }
    GAP_TRY(gap_scan(w.bin_count, n_bins, w.bin_start, w.scan_tmp, nullptr, st));
    if (n > 0) {
        gap_count_launch();
        k_scatter<<<gridN, T, 0, st>>>(n, w.atom_bin, w.bin_start, w.bin_fill, w.bin_atoms);
        GAP_TRY_CUDA(cudaGetLastError());
        gap_count_launch();
        const int gridW = (n + kNbrWarps - 1) / kNbrWarps;
        k_count_warp<<<gridW, 32 * kNbrWarps, 0, st>>>(n, w.frac, w.frac32, w.atom_cfg, w.geo, w.bin_start,
                                                       w.bin_atoms, w.counts);
        GAP_TRY_CUDA(cudaGetLastError());
    }
    GAP_TRY(gap_scan(w.counts, n, w.pairs.offsets, w.scan_tmp, w.total, st));
    int P = 0;
    if (w.graph) {
        P = w.pair_cap;
        GAP_TRY(w.reserve_pairs(P));
        gap_count_launch();
        k_cap_offsets<<<(n + 256) / 256, 256, 0, st>>>(n, P, w.total, w.pairs.offsets, w.total + 1, w.err);
        GAP_TRY_CUDA(cudaGetLastError());
        w.pairs.count = w.total + 1;
    } else {
        GAP_TRY_CUDA(cudaMemcpyAsync(&P, w.total, sizeof(int), cudaMemcpyDeviceToHost, st));
        GAP_TRY_CUDA(cudaStreamSynchronize(st));
        GAP_TRY(w.reserve_pairs(P));
        w.pairs.count = w.total;
    }
    w.pairs.n_pairs = P;
    if (n > 0) {
        gap_count_launch();
        k_fill_warp<<<(n + kNbrWarps - 1) / kNbrWarps, 32 * kNbrWarps, 0, st>>>(
            n, w.frac, w.frac32, w.atom_cfg, w.geo, w.bin_start, w.bin_atoms, w.pairs.offsets, P, w.keys, w.pairs.j,
            w.pairs.vec64, w.pairs.vec32, w.err);
        GAP_TRY_CUDA(cudaGetLastError());
        gap_count_launch();
        k_reverse<<<n, 64, 0, st>>>(n, w.pairs.offsets, w.keys, w.pairs.rev, w.err);
        GAP_TRY_CUDA(cudaGetLastError());
    }
    return GAP_OK;
}

gap_status gap_neighbours_check(NbrWork &w, cudaStream_t st)
{
    int e = 0;
    GAP_TRY_CUDA(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GAP_TRY_CUDA(cudaStreamSynchronize(st));
    if (e & 1) {
        gap_set_error("more neighbour pairs than the pair capacity (" + std::to_string(w.pair_cap) +
                      ") of the captured step");
        return GAP_ECAPACITY;
    }
    if (e) {
        gap_set_error("neighbour list inconsistency (code " + std::to_string(e) + ")");
        return GAP_ECUDA;
    }
    return GAP_OK;
}

// ------------------------------------------------------------ workspace
static gap_status grow(void **p, size_t &cap, size_t bytes)
{
    if (bytes <= cap && *p) return GAP_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    size_t b = bytes + bytes / 4 + 256;
    cudaError_t e = gap_dev_malloc(p, b);
    if (e != cudaSuccess) {
        *p = nullptr;
        gap_set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
        return GAP_ENOMEM;
    }
    cap = b;
    return GAP_OK;
}

gap_status NbrWork::reserve_atoms(int n, int n_configs, int n_bins)
{
    GAP_TRY(grow((void **)&geo, cap_geo, sizeof(CellGeom) * (n_configs + 1)));
    GAP_TRY(grow((void **)&cfg_offsets, cap_cfg, sizeof(int) * (n_configs + 2)));
    GAP_TRY(grow((void **)&frac, cap_frac, sizeof(double) * 3 * (size_t)(n + 1)));
    GAP_TRY(grow((void **)&frac32, cap_f32, sizeof(float4) * (size_t)(n + 1)));
    GAP_TRY(grow((void **)&atom_cfg, cap_acfg, sizeof(int) * (size_t)(n + 1)));
    GAP_TRY(grow((void **)&atom_bin, cap_abin, sizeof(int) * (size_t)(n + 1)));
    GAP_TRY(grow((void **)&bin_atoms, cap_batoms, sizeof(int) * (size_t)(n + 1)));
    GAP_TRY(grow((void **)&counts, cap_counts, sizeof(int) * (size_t)(n + 1)));
    GAP_TRY(grow((void **)&pairs.offsets, cap_offsets, sizeof(int) * (size_t)(n + 2)));
    GAP_TRY(grow((void **)&bin_count, cap_bcount, sizeof(int) * (size_t)(n_bins + 2)));
    GAP_TRY(grow((void **)&bin_fill, cap_bfill, sizeof(int) * (size_t)(n_bins + 2)));
    GAP_TRY(grow((void **)&bin_start, cap_bstart, sizeof(int) * (size_t)(n_bins + 2)));
    size_t t = gap_scan_tmp_ints(n > n_bins ? n : n_bins);
    GAP_TRY(grow((void **)&scan_tmp, cap_scan, sizeof(int) * t));
    GAP_TRY(grow((void **)&total, cap_total, sizeof(int) * 4));
    err = total + 2;
    return GAP_OK;
}

gap_status NbrWork::reserve_pairs(int P)
{
    size_t p = (size_t)(P > 0 ? P : 1);
    GAP_TRY(grow((void **)&keys, cap_keys, sizeof(long long) * p));
    GAP_TRY(grow((void **)&pairs.j, cap_j, sizeof(int) * p));
    GAP_TRY(grow((void **)&pairs.rev, cap_rev, sizeof(int) * p));
    GAP_TRY(grow((void **)&pairs.vec64, cap_v64, sizeof(D4) * p));
    GAP_TRY(grow((void **)&pairs.vec32, cap_v32, sizeof(float4) * p));
    return GAP_OK;
}

void NbrWork::release()
{
    void *ps[] = {geo, cfg_offsets, frac, frac32, atom_cfg, atom_bin, bin_atoms, counts, pairs.offsets, bin_count,
                  bin_fill, bin_start, scan_tmp, total, keys, pairs.j, pairs.rev, pairs.vec64, pairs.vec32};
    for (void *p : ps)
        if (p) cudaFree(p);
    *this = NbrWork();
}
