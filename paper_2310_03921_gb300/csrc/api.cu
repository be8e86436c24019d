// Host implementation of the C ABI declared in include/gap.h.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/gap.h"
#include "../../include/gap_testing.h"
#include "contract.h"
#include "crt_gemm.h"
#include "gap_internal.h"
#include "knm.h"
#include "nbr.h"
#include "radial.h"
#include "solve.h"
#include "soap.h"
#include "tc_gemm.h"

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void gap_set_error(const std::string &msg) { g_last_error = msg; }

gap_status gap_cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return GAP_OK;
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? GAP_ENOMEM : GAP_ECUDA;
}

extern "C" const char *gap_last_error(void) { return g_last_error.c_str(); }

#define GAP_API_BEGIN try {
#define GAP_API_END                                      \
    }                                                    \
    catch (const std::bad_alloc &) {                     \
        gap_set_error("host allocation failed");         \
        return GAP_ENOMEM;                               \
    }                                                    \
    catch (...) {                                        \
        gap_set_error("unexpected host exception");      \
        return GAP_EINVAL;                               \
    }

// --------------------------------------------------- profiling, counting
static std::atomic<long> g_launches{0};
void gap_count_launch(int n) { g_launches += n; }
long gap_launch_total() { return g_launches.load(); }

static const char *kStageNames[ST_COUNT] = {"neighbours", "expansion", "gp_rows", "split", "gemm_q",
                                            "gemm_g", "finalize", "chain", "pairforce", "twobody",
                                            "gather", "knm_rows", "knm_gemm", "knm_reduce", "solve_kmm",
                                            "solve_qr", "solve_prep", "solve_gemm", "solve_crt", "solve_potrf",
                                            "solve_trtri", "solve_apply", "knm_jacobian", "solve_block"};

struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> ev;            // pool of (begin, end) pairs
    std::vector<int> stage_of;              // stage of each used pair
    int active[ST_COUNT];
    size_t used = 0;
};
static Profiler g_prof;
bool gap_prof_enabled() { return g_prof.on; }

void gap_prof_begin(int stage, cudaStream_t st)
{
    if (!g_prof.on) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (2 * (g_prof.used + 1) > g_prof.ev.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            g_prof.ev.push_back(e);
        }
        g_prof.stage_of.resize(g_prof.ev.size() / 2, -1);
    }
    size_t idx = g_prof.used++;
    g_prof.stage_of[idx] = stage;
    g_prof.active[stage] = (int)idx;
    cudaEventRecord(g_prof.ev[2 * idx], st);
}

void gap_prof_end(int stage, cudaStream_t st)
{
    if (!g_prof.on) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    int idx = g_prof.active[stage];
    if (idx >= 0) cudaEventRecord(g_prof.ev[2 * idx + 1], st);
    g_prof.active[stage] = -1;
}

extern "C" gap_status gap_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = on != 0;
    g_prof.used = 0;
    for (int s = 0; s < ST_COUNT; ++s) g_prof.active[s] = -1;
    return GAP_OK;
}

extern "C" gap_status gap_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.used = 0;
    for (int s = 0; s < ST_COUNT; ++s) g_prof.active[s] = -1;
    return GAP_OK;
}

extern "C" int gap_profile_stages(void) { return ST_COUNT; }

extern "C" const char *gap_profile_stage_name(int stage)
{
    return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : "";
}

extern "C" int gap_tile_tuning_count(void) { return gap_tc_tuned_count(); }

extern "C" gap_status gap_tile_tuning_entry(int k, int *fields, float *ms)
{
    if (!fields || !ms) { gap_set_error("NULL argument"); return GAP_EINVAL; }
    if (!gap_tc_tuned_entry(k, fields, ms)) { gap_set_error("no such tuning entry"); return GAP_EINVAL; }
    return GAP_OK;
}

extern "C" gap_status gap_profile_read(double *ms, int *count)
{
    if (!ms) { gap_set_error("ms is NULL"); return GAP_EINVAL; }
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (int s = 0; s < ST_COUNT; ++s) {
        ms[s] = 0.0;
        if (count) count[s] = 0;
    }
    for (size_t k = 0; k < g_prof.used; ++k) {
        int s = g_prof.stage_of[k];
        if (s < 0) continue;
        GAP_TRY_CUDA(cudaEventSynchronize(g_prof.ev[2 * k + 1]));
        float t = 0.f;
        GAP_TRY_CUDA(cudaEventElapsedTime(&t, g_prof.ev[2 * k], g_prof.ev[2 * k + 1]));
        ms[s] += t;
        if (count) count[s] += 1;
    }
    return GAP_OK;
}

extern "C" long gap_launch_count(void) { return g_launches.load(); }

// ------------------------------------------------------------ constants
void gap_fill_ylm_constants(SoapGeom &g)
{
    const double pi = 3.14159265358979323846;
    for (int l = 0; l <= GAP_MAX_L; ++l)
        for (int m = 0; m <= GAP_MAX_L; ++m) {
            double v = 0.0;
            if (m <= l) {
                double ratio = 1.0;  // (l-m)!/(l+m)!
                for (int k = l - m + 1; k <= l + m; ++k) ratio /= k;
                v = std::sqrt((2.0 * l + 1.0) / (4.0 * pi) * ratio);
                if (m > 0) v *= std::sqrt(2.0);
            }
            g.ylmk64[l * (GAP_MAX_L + 1) + m] = v;
            g.ylmk32[l * (GAP_MAX_L + 1) + m] = (float)v;
        }
}

// ------------------------------------------------------ device buffers
// Every device allocation of the library goes through gap_dev_malloc, which
// a test hook can make fail (gap_test_fail_alloc) to exercise GAP_ENOMEM.
static std::atomic<long> g_fail_alloc_after{-1};

cudaError_t gap_dev_malloc(void **p, size_t bytes)
{
    long left = g_fail_alloc_after.load();
    while (left >= 0) {
        if (left == 0) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) break;
    }
    return cudaMalloc(p, bytes);
}

extern "C" gap_status gap_test_fail_alloc(long after)
{
    g_fail_alloc_after.store(after < 0 ? -1 : after);
    return GAP_OK;
}

extern "C" gap_status gap_test_tc_force_variant(int v)
{
    if (v >= 4) {
        gap_set_error("tile variant must be below 4");
        return GAP_EINVAL;
    }
    gap_tc_force_variant(v);
    return GAP_OK;
}

struct DBuf {
    void *p = nullptr;
    size_t cap = 0;
    gap_status ensure(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        if (bytes <= cap) return GAP_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t b = bytes + bytes / 8 + 256;
        cudaError_t e = gap_dev_malloc(&p, b);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            gap_set_error(std::string("cudaMalloc of ") + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
            return GAP_ENOMEM;
        }
        cap = b;
        return GAP_OK;
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

template <typename T> static gap_status upload(DBuf &b, const std::vector<T> &v)
{
    GAP_TRY(b.ensure(sizeof(T) * v.size()));
    if (!v.empty()) GAP_TRY_CUDA(cudaMemcpy(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return GAP_OK;
}

struct HostPinned {
    void *p = nullptr;
    size_t cap = 0;
    gap_status ensure(size_t bytes)
    {
        if (bytes <= cap && p) return GAP_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        size_t b = bytes + 256;
        if (cudaMallocHost(&p, b) != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            gap_set_error("pinned host allocation failed");
            return GAP_ENOMEM;
        }
        cap = b;
        return GAP_OK;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

// BF16 round-to-nearest-even of an FP32 value, and back (host side).
static uint16_t bf16_rne(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40);  // NaN
    uint32_t rounding = 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)((u + rounding) >> 16);
}

static float bf16_to_float(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

struct Workspace {
    NbrWork nbr;
    DBuf pos, spec, pair_i, coef, phat, pnorm, gp_of_atom, flag, fpos, scan_tmp, rows, counts, gvec, wsum, eps, eps2,
        W, eps_part, Gam, fpair, f2, forces, vir_atom, cfgpart, energy, virial, local, err, A_hi, A_lo, t_row, W_hi, W_lo,
        epart_f, wpart_f, Gs, outbuf, kA, kAhi, kAlo, kt, ksrc, kseg, kdest, segstart, outrow, Wp, kq, P, Kbuf, A_mid, W_mid,
        kAmid, phatc, pnormc, hfull, kV;
    // Graph mode (gap_step_graph): no host synchronisation inside a call; the
    // rows of each GP are those of the last ordinary call (species are fixed).
    bool graph = false;
    std::vector<int> counts_fixed;
    void release()
    {
        nbr.release();
        DBuf *bs[] = {&pos, &spec, &pair_i, &coef, &phat, &pnorm, &gp_of_atom, &flag, &fpos, &scan_tmp, &rows,
                      &counts, &gvec, &wsum, &eps, &eps2, &W, &eps_part, &Gam, &fpair, &f2, &forces, &vir_atom, &cfgpart, &energy,
                      &virial, &local, &err, &A_hi, &A_lo, &t_row, &W_hi, &W_lo, &epart_f, &wpart_f, &Gs, &outbuf,
                      &kA, &kAhi, &kAlo, &kt, &ksrc, &kseg, &kdest, &segstart, &outrow, &Wp, &kq, &P, &Kbuf, &A_mid, &W_mid,
                      &kAmid, &phatc, &pnormc, &hfull, &kV};
        for (DBuf *b : bs) b->release();
    }
};

// Makes `dev` current for the scope of a call.  A failed switch is reported
// by the next checked call; the runtime's last-error slot is cleared so that
// it cannot surface in an unrelated later call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) cudaGetLastError();
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev && cudaSetDevice(prev) != cudaSuccess) cudaGetLastError();
    }
};

// ---------------------------------------------------------------- soap
// A descriptor is shared by the models built on it: each model holds a
// reference, so gap_soap_destroy before gap_model_destroy (as a garbage
// collector may order them) defers the release to the last model.
struct gap_soap {
    std::atomic<int> refs{1};
    int device = 0;
    SoapGeom geo{};
    double *tab64 = nullptr;   // knot values and derivatives (FP64)
    double *coef64 = nullptr;  // per-interval cubic coefficients
    float *coef32 = nullptr;
    int4 *dtab = nullptr;      // geo.dtab
    // Compression (gap_soap_set_compression): the GP sees p~ / |p~| with
    // p~ = Q p, Q [Dg][D] (FP64 and FP32 copies, and the BF16 planes
    // [Dg16][D16] of the FP32 copy for the tensor-core K_NM rows: hi, lo of
    // the two-plane split, mid and lo of the three-plane one); Dg = geo.D
    // without.
    int comp = 0;
    int Dg = 0, Dg16 = 0;
    DBuf Q64, Q32, Qhi, Qlo, Qmid, Qlo3;
    Workspace ws;
    std::mutex mu;
};

template <typename T> static const T *q_of(const gap_soap *s);
template <> const double *q_of<double>(const gap_soap *s) { return s->Q64.as<double>(); }
template <> const float *q_of<float>(const gap_soap *s) { return s->Q32.as<float>(); }

template <typename T> static const T *tab_of(const gap_soap *s);
template <> const double *tab_of<double>(const gap_soap *s) { return s->coef64; }
template <> const float *tab_of<float>(const gap_soap *s) { return s->coef32; }

static gap_status check_params(const gap_soap_params *p)
{
    if (!p) { gap_set_error("params is NULL"); return GAP_EINVAL; }
    if (p->n_max < 1 || p->n_max > 12) { gap_set_error("n_max must be in 1..12"); return GAP_EINVAL; }
    if (p->l_max < 0 || p->l_max > GAP_MAX_L) { gap_set_error("l_max must be in 0..10"); return GAP_EINVAL; }
    if (!(p->cutoff > 0.0) || !(p->cutoff_transition_width > 0.0) || p->cutoff_transition_width > p->cutoff) {
        gap_set_error("need 0 < cutoff_transition_width <= cutoff");
        return GAP_EINVAL;
    }
    if (!(p->atom_sigma > 0.0)) { gap_set_error("atom_sigma must be positive"); return GAP_EINVAL; }
    if (p->n_species < 1 || p->n_species > GAP_MAX_SPECIES) { gap_set_error("n_species must be in 1..8"); return GAP_EINVAL; }
    if (p->mix_K < 0 || p->mix_K > GAP_MAX_GROUPS) { gap_set_error("mix_K must be in 0..8"); return GAP_EINVAL; }
    if (p->mix_K > 0 && !p->mix_w) { gap_set_error("mix_w is NULL"); return GAP_EINVAL; }
    if (p->cutoff * p->cutoff / (p->atom_sigma * p->atom_sigma) > 600.0) {
        gap_set_error("cutoff / atom_sigma too large for the radial integrals");
        return GAP_EUNSUPPORTED;
    }
    int GA = p->mix_K > 0 ? p->mix_K : p->n_species;
    if (!gap_shape_supported(p->n_max, p->l_max, GA)) {
        gap_set_error("(n_max, l_max, channel groups) = (" + std::to_string(p->n_max) + ", " +
                      std::to_string(p->l_max) + ", " + std::to_string(GA) + ") has no compiled kernel");
        return GAP_EUNSUPPORTED;
    }
    return GAP_OK;
}

extern "C" gap_status gap_soap_create(const gap_soap_params *p, gap_soap **out)
{
    GAP_API_BEGIN
    if (!out) { gap_set_error("out is NULL"); return GAP_EINVAL; }
    *out = nullptr;
    GAP_TRY(check_params(p));
    gap_soap *s = new gap_soap();
    GAP_TRY_CUDA(cudaGetDevice(&s->device));
    SoapGeom &g = s->geo;
    g.N = p->n_max;
    g.L = p->l_max;
    g.LM = (p->l_max + 1) * (p->l_max + 1);
    g.S = p->n_species;
    g.mixed = p->mix_K > 0;
    g.GA = g.mixed ? p->mix_K : p->n_species;
    g.Nc = g.mixed ? g.N : g.GA * g.N;
    g.nblocks = g.mixed ? g.GA : 1;
    g.npair = g.Nc * (g.Nc + 1) / 2;
    g.D = g.nblocks * g.npair * (g.L + 1);
    g.D16 = (g.D + 15) / 16 * 16;
    s->Dg = g.D;
    s->Dg16 = g.D16;
    g.rc = p->cutoff;
    g.d = p->cutoff_transition_width;
    g.sigma = p->atom_sigma;
    g.cw = p->central_weight;
    g.G = 2048;
    g.h = g.rc / g.G;
    for (int a = 0; a < GAP_MAX_GROUPS * GAP_MAX_SPECIES; ++a) { g.wacc32[a] = 0.f; g.wacc64[a] = 0.0; }
    for (int k = 0; k < g.GA; ++k)
        for (int z = 0; z < g.S; ++z) {
            double w = g.mixed ? p->mix_w[k * g.S + z] : (k == z ? 1.0 : 0.0);
            g.wacc64[k * GAP_MAX_SPECIES + z] = w;
            g.wacc32[k * GAP_MAX_SPECIES + z] = (float)w;
        }
    gap_fill_ylm_constants(g);
    {
        // descriptor entries ordered by l (the pair enumeration of the
        // descriptor index: a-major over a <= a')
        std::vector<int4> t;
        t.reserve(g.D);
        const int per = g.npair * (g.L + 1);
        for (int l = 0; l <= g.L; ++l)
            for (int b = 0; b < g.nblocks; ++b) {
                int pi = 0;
                for (int a = 0; a < g.Nc; ++a)
                    for (int ap = a; ap < g.Nc; ++ap, ++pi) {
                        const int g1 = g.mixed ? b : a / g.N, n1 = g.mixed ? a : a % g.N;
                        const int g2 = g.mixed ? b : ap / g.N, n2 = g.mixed ? ap : ap % g.N;
                        t.push_back(make_int4(b * per + pi * (g.L + 1) + l, (g1 * g.N + n1) * g.LM + l * l,
                                              (g2 * g.N + n2) * g.LM + l * l, l | ((a != ap ? 1 : 0) << 8)));
                    }
            }
        gap_status ts = gap_cuda_status(cudaMalloc((void **)&s->dtab, sizeof(int4) * t.size()), "cudaMalloc");
        if (ts == GAP_OK)
            ts = gap_cuda_status(cudaMemcpy(s->dtab, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice),
                                 "cudaMemcpy");
        if (ts != GAP_OK) {
            if (s->dtab) cudaFree(s->dtab);
            delete s;
            return ts;
        }
        g.dtab = s->dtab;
    }
    gap_status st = gap_radial_table(g, &s->tab64, &s->coef64, &s->coef32);
    if (st != GAP_OK) {
        if (s->tab64) cudaFree(s->tab64);
        if (s->coef64) cudaFree(s->coef64);
        if (s->coef32) cudaFree(s->coef32);
        cudaFree(s->dtab);
        delete s;
        return st;
    }
    *out = s;
    return GAP_OK;
    GAP_API_END
}

static void soap_release(gap_soap *s)
{
    if (--s->refs > 0) return;
    DeviceGuard dg(s->device);
    s->ws.release();
    for (DBuf *q : {&s->Q64, &s->Q32, &s->Qhi, &s->Qlo, &s->Qmid, &s->Qlo3}) q->release();
    if (s->tab64) cudaFree(s->tab64);
    if (s->coef64) cudaFree(s->coef64);
    if (s->coef32) cudaFree(s->coef32);
    if (s->dtab) cudaFree(s->dtab);
    delete s;
}

extern "C" gap_status gap_soap_destroy(gap_soap *s)
{
    GAP_API_BEGIN
    if (!s) return GAP_OK;
    soap_release(s);
    return GAP_OK;
    GAP_API_END
}

extern "C" gap_status gap_soap_dim(const gap_soap *s, int *D)
{
    if (!s || !D) { gap_set_error("NULL argument"); return GAP_EINVAL; }
    *D = s->Dg;
    return GAP_OK;
}

extern "C" gap_status gap_soap_cutoff(const gap_soap *s, double *rc)
{
    if (!s || !rc) { gap_set_error("NULL argument"); return GAP_EINVAL; }
    *rc = s->geo.rc;
    return GAP_OK;
}

extern "C" gap_status gap_soap_radial_table(const gap_soap *s, int *knots, double *out)
{
    GAP_API_BEGIN
    if (!s || !knots) { gap_set_error("NULL argument"); return GAP_EINVAL; }
    *knots = s->geo.G + 1;
    if (out) {
        DeviceGuard dg(s->device);
        size_t n = (size_t)(s->geo.G + 1) * s->geo.N * (s->geo.L + 1) * 2;
        GAP_TRY_CUDA(cudaMemcpy(out, s->tab64, sizeof(double) * n, cudaMemcpyDeviceToHost));
    }
    return GAP_OK;
    GAP_API_END
}

// ------------------------------------------------------------ batches
static gap_status check_batch(const gap_batch *b)
{
    if (!b) { gap_set_error("batch is NULL"); return GAP_EINVAL; }
    if (b->n_atoms < 0 || b->n_configs < 0) { gap_set_error("negative sizes"); return GAP_EINVAL; }
    if (b->n_configs == 0) {
        if (b->n_atoms != 0) { gap_set_error("atoms without configurations"); return GAP_EINVAL; }
        return GAP_OK;
    }
    if (!b->config_offsets || !b->cell || !b->pbc) { gap_set_error("batch metadata is NULL"); return GAP_EINVAL; }
    if (b->n_atoms > 0 && (!b->pos || !b->species)) { gap_set_error("positions/species are NULL"); return GAP_EINVAL; }
    if (b->config_offsets[0] != 0 || b->config_offsets[b->n_configs] != b->n_atoms) {
        gap_set_error("config_offsets must start at 0 and end at n_atoms");
        return GAP_EINVAL;
    }
    for (int c = 0; c < b->n_configs; ++c)
        if (b->config_offsets[c + 1] < b->config_offsets[c]) {
            gap_set_error("config_offsets must be non-decreasing");
            return GAP_EINVAL;
        }
    if (b->n_atoms >= (1 << 28)) { gap_set_error("too many atoms"); return GAP_EINVAL; }
    return GAP_OK;
}

__global__ void k_check_species(int n, const int *__restrict__ spec, int S, int *__restrict__ err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (spec[i] < 0 || spec[i] >= S)) atomicOr(err, 1);
}

// Device copies of positions and species (staged from host if needed).
static gap_status stage_inputs(Workspace &w, const gap_batch *b, int S, const double **pos, const int **spec,
                               cudaStream_t st)
{
    int n = b->n_atoms;
    GAP_TRY(w.err.ensure(16 * sizeof(int)));
    GAP_TRY_CUDA(cudaMemsetAsync(w.err.p, 0, 16 * sizeof(int), st));
    if (b->device) {
        *pos = b->pos;
        *spec = b->species;
        if (n > 0) {
            gap_count_launch();
            k_check_species<<<(n + 255) / 256, 256, 0, st>>>(n, b->species, S, w.err.as<int>() + 1);
            GAP_TRY_CUDA(cudaGetLastError());
        }
        return GAP_OK;
    }
    for (int i = 0; i < n; ++i)
        if (b->species[i] < 0 || b->species[i] >= S) {
            gap_set_error("species index out of range at atom " + std::to_string(i));
            return GAP_EINVAL;
        }
    GAP_TRY(w.pos.ensure(sizeof(double) * 3 * (size_t)n));
    GAP_TRY(w.spec.ensure(sizeof(int) * (size_t)n));
    if (n > 0) {
        GAP_TRY_CUDA(cudaMemcpyAsync(w.pos.p, b->pos, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, st));
        GAP_TRY_CUDA(cudaMemcpyAsync(w.spec.p, b->species, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st));
    }
    *pos = w.pos.as<double>();
    *spec = w.spec.as<int>();
    return GAP_OK;
}

static gap_status check_device_errors(Workspace &w, cudaStream_t st)
{
    int e[16];
    GAP_TRY_CUDA(cudaMemcpyAsync(e, w.err.p, sizeof(e), cudaMemcpyDeviceToHost, st));
    GAP_TRY_CUDA(cudaStreamSynchronize(st));
    if (e[1]) { gap_set_error("species index out of range"); return GAP_EINVAL; }
    if (e[2]) {
        gap_set_error("tensor-core GEMM wait expired (code " + std::to_string(e[2]) + ")");
        return GAP_ETIMEOUT;
    }
    GAP_TRY(gap_neighbours_check(w.nbr, st));
    return GAP_OK;
}

extern "C" gap_status gap_soap_set_compression(gap_soap *s, const gap_compression *c)
{
    GAP_API_BEGIN
    if (!s || !c) { gap_set_error("NULL argument"); return GAP_EINVAL; }
    const SoapGeom &g = s->geo;
    if (g.mixed) {
        gap_set_error("compression acts on the fully coupled descriptor (mix_K = 0)");
        return GAP_EINVAL;
    }
    if (s->refs.load() != 1) {
        gap_set_error("the descriptor object is held by a model or step graph");
        return GAP_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    const int N = g.N, L = g.L, S = g.S, Nc = g.Nc, D = g.D, L1 = g.L + 1;
    // index of the stored entry (pair a <= a', a-major; l) and the factor
    // taking it to the ordered spectrum P^{ab}_l
    auto didx = [&](int a, int b, int l) {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        const int pi = lo * Nc - lo * (lo - 1) / 2 + (hi - lo);
        return pi * L1 + l;
    };
    const double r2 = 1.0 / std::sqrt(2.0);
    auto fac = [&](int a, int b) { return a == b ? 1.0 : r2; };
    int Dg = 0;
    std::vector<double> Q;
    switch (c->recipe) {
    case GAP_COMPRESS_NONE:
        s->comp = 0;
        s->Dg = D;
        s->Dg16 = g.D16;
        for (DBuf *q : {&s->Q64, &s->Q32, &s->Qhi, &s->Qlo, &s->Qmid, &s->Qlo3}) q->release();
        return GAP_OK;
    case GAP_COMPRESS_MATRIX:
        if (c->d_out < 1 || !c->P) { gap_set_error("MATRIX needs d_out >= 1 and P"); return GAP_EINVAL; }
        Dg = c->d_out;
        Q.assign(c->P, c->P + (size_t)Dg * D);
        break;
    case GAP_COMPRESS_SKETCH:
    case GAP_COMPRESS_DECOMPOSITION: {
        const bool sk = c->recipe == GAP_COMPRESS_SKETCH;
        if (c->K < 1 || !c->w || (sk && !c->u)) { gap_set_error("SKETCH/DECOMPOSITION need K >= 1 and weights"); return GAP_EINVAL; }
        const double *u = sk ? c->u : c->w;
        Dg = c->K * L1;
        Q.assign((size_t)Dg * D, 0.0);
        for (int k = 0; k < c->K; ++k)
            for (int l = 0; l < L1; ++l)
                for (int a = 0; a < Nc; ++a)
                    for (int b = 0; b < Nc; ++b)
                        Q[(size_t)(k * L1 + l) * D + didx(a, b, l)] += c->w[(size_t)k * Nc + a] * u[(size_t)k * Nc + b] * fac(a, b);
        break;
    }
    case GAP_COMPRESS_NU: {
        if (c->nu_S < 0 || c->nu_S > 2 || c->nu_R < 0 || c->nu_R > 2) { gap_set_error("nu_S, nu_R must be 0, 1 or 2"); return GAP_EINVAL; }
        const int sA = c->nu_S >= 1 ? S : 1, sB = c->nu_S == 2 ? S : 1, nA = c->nu_R >= 1 ? N : 1, nB = c->nu_R == 2 ? N : 1;
        Dg = sA * sB * nA * nB * L1;
        Q.assign((size_t)Dg * D, 0.0);
        for (int al = 0; al < S; ++al)
            for (int be = 0; be < S; ++be)
                for (int n = 0; n < N; ++n)
                    for (int np = 0; np < N; ++np)
                        for (int l = 0; l < L1; ++l) {
                            const int o = ((((sA > 1 ? al : 0) * sB + (sB > 1 ? be : 0)) * nA + (nA > 1 ? n : 0)) * nB +
                                           (nB > 1 ? np : 0)) * L1 + l;
                            const int a = al * N + n, b = be * N + np;
                            Q[(size_t)o * D + didx(a, b, l)] += fac(a, b);
                        }
        break;
    }
    case GAP_COMPRESS_TRIVIAL:
        Dg = S * Nc * L1;
        Q.assign((size_t)Dg * D, 0.0);
        for (int al = 0; al < S; ++al)
            for (int b = 0; b < Nc; ++b)
                for (int l = 0; l < L1; ++l) {
                    const int a = al * N;
                    Q[(size_t)((al * Nc + b) * L1 + l) * D + didx(a, b, l)] += fac(a, b);
                }
        break;
    default:
        gap_set_error("unknown compression recipe");
        return GAP_EINVAL;
    }
    DeviceGuard dg(s->device);
    std::vector<float> Q32(Q.begin(), Q.end());
    const int Dg16 = (Dg + 15) / 16 * 16;
    std::vector<uint16_t> qh((size_t)Dg16 * g.D16, 0), ql(qh.size(), 0), qm(qh.size(), 0), ql3(qh.size(), 0);
    for (int o = 0; o < Dg; ++o)
        for (int d = 0; d < D; ++d) {
            const float b = Q32[(size_t)o * D + d];
            const uint16_t h = bf16_rne(b);
            const float rest = b - bf16_to_float(h);
            const uint16_t m3 = bf16_rne(rest);
            const size_t k = (size_t)o * g.D16 + d;
            qh[k] = h;
            ql[k] = bf16_rne(rest);
            qm[k] = m3;
            ql3[k] = bf16_rne(rest - bf16_to_float(m3));
        }
    GAP_TRY(upload(s->Q64, Q));
    GAP_TRY(upload(s->Q32, Q32));
    GAP_TRY(upload(s->Qhi, qh));
    GAP_TRY(upload(s->Qlo, ql));
    GAP_TRY(upload(s->Qmid, qm));
    GAP_TRY(upload(s->Qlo3, ql3));
    s->comp = (int)c->recipe;
    s->Dg = Dg;
    s->Dg16 = Dg16;
    return GAP_OK;
    GAP_API_END
}

// p~ = Q (|p| p_hat), |p~|, p~ / |p~| per atom: one CTA of 128 threads per
// atom, p staged in shared memory, a warp per output entry.
template <typename T>
__global__ void __launch_bounds__(128) k_compress(int n, int D, int Dg, const T *__restrict__ Q,
                                                  const T *__restrict__ phat, const T *__restrict__ pnorm,
                                                  T *__restrict__ phatc, T *__restrict__ pnormc)
{
    extern __shared__ __align__(16) unsigned char cmp_smem[];
    T *ps = reinterpret_cast<T *>(cmp_smem);  // [D]
    T *vs = ps + D;                           // [Dg]
    __shared__ T red[4];
    const int i = blockIdx.x;
    if (i >= n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T sc = pnorm[i];
    for (int d = threadIdx.x; d < D; d += blockDim.x) ps[d] = phat[(size_t)i * D + d] * sc;
    __syncthreads();
    for (int o = warp; o < Dg; o += 4) {
        T acc = T(0);
        for (int d = lane; d < D; d += 32) acc += Q[(size_t)o * D + d] * ps[d];
        for (int k = 16; k; k >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, k);
        if (lane == 0) vs[o] = acc;
    }
    __syncthreads();
    T nn = T(0);
    for (int o = threadIdx.x; o < Dg; o += blockDim.x) nn += vs[o] * vs[o];
    for (int k = 16; k; k >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, k);
    if (lane == 0) red[warp] = nn;
    __syncthreads();
    const T tot = (red[0] + red[1]) + (red[2] + red[3]);
    const T nrm = sqrt(tot), inv = T(1) / nrm;
    for (int o = threadIdx.x; o < Dg; o += blockDim.x) phatc[(size_t)i * Dg + o] = vs[o] * inv;
    if (threadIdx.x == 0) pnormc[i] = nrm;
}

// dE/dp (times |p|, the input the chain kernel expects) from dE/dp_hat~:
// v = (g - (g . p_hat~) p_hat~) / |p~|, h = |p| Q^T v.  g includes wsum mu
// for the centred tensor-core form.  Since p_hat~ depends only on the
// direction of p, h . p_hat = 0 and the chain kernel's projection leaves
// h / |p| = dE/dp unchanged.
template <typename T>
__global__ void __launch_bounds__(128) k_decompress(int n, int D, int D16, int Dg, int Dg16, const T *__restrict__ Q,
                                                    const T *__restrict__ gvec, const float *__restrict__ wsum,
                                                    const float *__restrict__ mu, const int *__restrict__ gp_of_atom,
                                                    const T *__restrict__ phatc, const T *__restrict__ pnormc,
                                                    const T *__restrict__ pnorm, T *__restrict__ h)
{
    extern __shared__ __align__(16) unsigned char cmp_smem[];
    T *gs = reinterpret_cast<T *>(cmp_smem);  // [Dg]
    __shared__ T red[4];
    const int i = blockIdx.x;
    if (i >= n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = gp_of_atom ? gp_of_atom[i] : 0;
    T dot = T(0);
    for (int o = threadIdx.x; o < Dg; o += blockDim.x) {
        T gv = gvec[(size_t)i * Dg16 + o];
        if (wsum && s >= 0) gv += (T)(wsum[i] * mu[(size_t)s * Dg16 + o]);
        gs[o] = gv;
        dot += gv * phatc[(size_t)i * Dg + o];
    }
    for (int k = 16; k; k >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, k);
    if (lane == 0) red[warp] = dot;
    __syncthreads();
    const T c1 = (red[0] + red[1]) + (red[2] + red[3]);
    const T inv = T(1) / pnormc[i];
    for (int o = threadIdx.x; o < Dg; o += blockDim.x) gs[o] = (gs[o] - c1 * phatc[(size_t)i * Dg + o]) * inv;
    __syncthreads();
    const T pn = pnorm[i];
    for (int d = threadIdx.x; d < D16; d += blockDim.x) {
        T acc = T(0);
        if (d < D)
            for (int o = 0; o < Dg; ++o) acc += Q[(size_t)o * D + d] * gs[o];
        h[(size_t)i * D16 + d] = pn * acc;
    }
}

template <typename T> static gap_status shm_attr(const void *fn, size_t shm)
{
    if (shm > 48 * 1024) GAP_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    return GAP_OK;
}

// The descriptor the GP sees: p_hat (geo.D) or the compressed p_hat~ (Dg).
template <typename T> static const T *gp_phat(const gap_soap *s, const Workspace &w)
{
    return s->comp ? w.phatc.as<T>() : w.phat.as<T>();
}

// Neighbours + expansion + power spectrum for a batch, in arithmetic T.
template <typename T>
static gap_status run_descriptor(gap_soap *soap, Workspace &w, const gap_batch *b, const int **spec_out,
                                 cudaStream_t st)
{
    const SoapGeom &g = soap->geo;
    int n = b->n_atoms;
    const double *pos;
    const int *spec;
    gap_prof_begin(ST_NEIGHBOURS, st);
    GAP_TRY(stage_inputs(w, b, g.S, &pos, &spec, st));
    GAP_TRY(gap_neighbours(w.nbr, b, pos, g.rc, st));
    const PairList &pl = w.nbr.pairs;
    GAP_TRY(w.pair_i.ensure(sizeof(int) * (size_t)pl.n_pairs));
    GAP_TRY(gap_pair_atoms(n, pl, w.pair_i.as<int>(), st));
    gap_prof_end(ST_NEIGHBOURS, st);
    GAP_TRY(w.coef.ensure(sizeof(T) * (size_t)n * g.GA * g.N * g.LM));
    GAP_TRY(w.phat.ensure(sizeof(T) * (size_t)n * g.D));
    GAP_TRY(w.pnorm.ensure(sizeof(T) * (size_t)n));
    gap_prof_begin(ST_EXPANSION, st);
    GAP_TRY(gap_expand<T>(g, tab_of<T>(soap), n, pl, spec, w.coef.as<T>(), w.phat.as<T>(), w.pnorm.as<T>(), st));
    if (soap->comp && n > 0) {
        GAP_TRY(w.phatc.ensure(sizeof(T) * (size_t)n * soap->Dg));
        GAP_TRY(w.pnormc.ensure(sizeof(T) * (size_t)n));
        const size_t shm = sizeof(T) * ((size_t)g.D + soap->Dg);
        GAP_TRY(shm_attr<T>((const void *)k_compress<T>, shm));
        gap_count_launch();
        k_compress<T><<<n, 128, shm, st>>>(n, g.D, soap->Dg, q_of<T>(soap), w.phat.as<T>(), w.pnorm.as<T>(),
                                           w.phatc.as<T>(), w.pnormc.as<T>());
        GAP_TRY_CUDA(cudaGetLastError());
    }
    gap_prof_end(ST_EXPANSION, st);
    *spec_out = spec;
    return GAP_OK;
}

__global__ void k_to_double(const float *__restrict__ a, double *__restrict__ b, size_t n)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

extern "C" gap_status gap_descriptor_sizes(gap_soap *soap, const gap_batch *b, long *n_desc, long *n_pairs,
                                           void *stream)
{
    GAP_API_BEGIN
    if (!soap) { gap_set_error("soap is NULL"); return GAP_EINVAL; }
    GAP_TRY(check_batch(b));
    std::lock_guard<std::mutex> lk(soap->mu);
    DeviceGuard dg(soap->device);
    cudaStream_t st = (cudaStream_t)stream;
    Workspace &w = soap->ws;
    const double *pos;
    const int *spec;
    GAP_TRY(stage_inputs(w, b, soap->geo.S, &pos, &spec, st));
    GAP_TRY(gap_neighbours(w.nbr, b, pos, soap->geo.rc, st));
    GAP_TRY(check_device_errors(w, st));
    if (n_desc) *n_desc = b->n_atoms;
    if (n_pairs) *n_pairs = w.nbr.pairs.n_pairs;
    return GAP_OK;
    GAP_API_END
}

extern "C" gap_status gap_descriptor(gap_soap *soap, const gap_batch *b, gap_precision prec, double *p_out,
                                     void *stream)
{
    GAP_API_BEGIN
    if (!soap) { gap_set_error("soap is NULL"); return GAP_EINVAL; }
    GAP_TRY(check_batch(b));
    if (b->n_atoms > 0 && !p_out) { gap_set_error("p_out is NULL"); return GAP_EINVAL; }
    if (prec != GAP_FP64 && prec != GAP_BF16X3 && prec != GAP_BF16X6 && prec != GAP_FP32) {
        gap_set_error("bad precision");
        return GAP_EINVAL;
    }
    std::lock_guard<std::mutex> lk(soap->mu);
    DeviceGuard dg(soap->device);
    cudaStream_t st = (cudaStream_t)stream;
    Workspace &w = soap->ws;
    size_t cnt = (size_t)b->n_atoms * soap->Dg;
    const int *spec;
    double *dst = p_out;
    if (!b->device) {
        GAP_TRY(w.outbuf.ensure(sizeof(double) * cnt));
        dst = w.outbuf.as<double>();
    }
    if (prec == GAP_FP64) {
        GAP_TRY(run_descriptor<double>(soap, w, b, &spec, st));
        if (cnt)
            GAP_TRY_CUDA(cudaMemcpyAsync(dst, gp_phat<double>(soap, w), sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st));
    } else {
        GAP_TRY(run_descriptor<float>(soap, w, b, &spec, st));
        if (cnt) {
            gap_count_launch();
            k_to_double<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(gp_phat<float>(soap, w), dst, cnt);
            GAP_TRY_CUDA(cudaGetLastError());
        }
    }
    if (!b->device && cnt)
        GAP_TRY_CUDA(cudaMemcpyAsync(p_out, dst, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    GAP_TRY(check_device_errors(w, st));
    return GAP_OK;
    GAP_API_END
}

// ---------------------------------------------------------------- model
struct GPData {
    int M = 0, M_pad = 0;
    // B planes: hi; lo of the two-plane split; mid and lo of the three-plane split
    DBuf X64, a64, X32, a32, mu64, s_col, alpha_pad, Bhi, Blo, BThi, BTlo, Bmid, Blo3, BTmid, BTlo3;
};

// A model is shared with the step graphs captured from it (each holds a
// reference); its device memory is freed with the last of them.
struct gap_model {
    std::atomic<int> refs{1};
    gap_soap *soap = nullptr;
    int n_gp = 0;
    double delta = 1.0;
    int zeta = 1;
    std::vector<GPData> gp;
    DBuf mu_all;  // [n_gp][D16] float
    bool has_tb = false;
    TwoBodyDev tb{};
    DBuf tb_x, tb_a, tb_tab;
    Workspace ws;
    SolveWork solve_ws;
    DBuf solve_X, solve_blk;  // all GPs' sparse points [M_total][D] and their GP, for the solve (built once)
    DBuf fit_y, fit_s, fit_a;  // gap_fit's device copies of host targets, sigmas and coefficients
    // posterior factors for predictive variances (gap_model_set_posterior):
    // U^-1 of K_MM + jitter I and R^-1 of A^T A, [M_total][M_total] column-major
    DBuf post_kinv, post_rinv;
    bool has_post = false;
    DBuf var_P, var_Q, var_V, var_W, var_out;  // gap_predict_variance scratch
    std::mutex mu;
};


static void release_model(gap_model *m)
{
    for (auto &g : m->gp) {
        DBuf *bs[] = {&g.X64, &g.a64, &g.X32, &g.a32, &g.mu64, &g.s_col, &g.alpha_pad, &g.Bhi, &g.Blo, &g.BThi, &g.BTlo,
                      &g.Bmid, &g.Blo3, &g.BTmid, &g.BTlo3};
        for (DBuf *b : bs) b->release();
    }
    m->mu_all.release();
    m->tb_x.release();
    m->tb_a.release();
    m->tb_tab.release();
    m->ws.release();
    m->solve_ws.release();
    m->solve_X.release();
    m->solve_blk.release();
    m->fit_y.release();
    m->fit_s.release();
    m->fit_a.release();
    DBuf *pv[] = {&m->post_kinv, &m->post_rinv, &m->var_P, &m->var_Q, &m->var_V, &m->var_W, &m->var_out};
    for (DBuf *b : pv) b->release();
    m->has_post = false;
}

extern "C" gap_status gap_model_create(gap_soap *soap, int n_gp, const int *M, const double *const *sparse,
                                       const double *const *alpha, double delta, double zeta,
                                       const gap_2b_params *tb, gap_model **out)
{
    GAP_API_BEGIN
    if (!out) { gap_set_error("out is NULL"); return GAP_EINVAL; }
    *out = nullptr;
    if (!soap) { gap_set_error("soap is NULL"); return GAP_EINVAL; }
    if (n_gp < 0 || n_gp > soap->geo.S) { gap_set_error("n_gp must be in 0..n_species"); return GAP_EINVAL; }
    if (n_gp > 0 && (!M || !sparse || !alpha)) { gap_set_error("sparse data is NULL"); return GAP_EINVAL; }
    if (!(zeta >= 1.0) || zeta != std::floor(zeta) || zeta > 64) {
        gap_set_error("zeta must be an integer in 1..64");
        return GAP_EUNSUPPORTED;
    }
    if (!std::isfinite(delta)) { gap_set_error("delta must be finite"); return GAP_EINVAL; }
    if (tb) {
        if (tb->n_sparse < 0 || (tb->n_sparse > 0 && (!tb->x || !tb->alpha))) {
            gap_set_error("bad two-body sparse data");
            return GAP_EINVAL;
        }
        if (!(tb->cutoff > 0.0) || tb->cutoff > soap->geo.rc + 1e-12 || !(tb->cutoff_transition_width > 0.0) ||
            tb->cutoff_transition_width > tb->cutoff || !(tb->theta > 0.0)) {
            gap_set_error("two-body cutoff must lie in (0, SOAP cutoff], with positive width and theta");
            return GAP_EINVAL;
        }
    }
    DeviceGuard dg(soap->device);
    gap_model *m = new gap_model();
    m->soap = soap;
    m->n_gp = n_gp;
    m->delta = delta;
    m->zeta = (int)zeta;
    m->gp.resize(n_gp);
    const int D = soap->Dg, D16 = soap->Dg16;  // the descriptor the GP sees
    std::vector<float> mu_all((size_t)(n_gp > 0 ? n_gp : 1) * D16, 0.f);
    gap_status st = GAP_OK;
    for (int s = 0; s < n_gp && st == GAP_OK; ++s) {
        GPData &g = m->gp[s];
        int Ms = M[s];
        if (Ms < 0 || (Ms > 0 && (!sparse[s] || !alpha[s]))) {
            gap_set_error("bad sparse set");
            st = GAP_EINVAL;
            break;
        }
        g.M = Ms;
        g.M_pad = (Ms + 255) / 256 * 256;
        if (g.M_pad == 0) g.M_pad = 256;
        std::vector<double> X(sparse[s], sparse[s] + (size_t)Ms * D), a(alpha[s], alpha[s] + Ms);
        std::vector<float> X32(X.begin(), X.end()), a32(a.begin(), a.end());
        std::vector<double> mu(D, 0.0);
        for (int k = 0; k < Ms; ++k)
            for (int d = 0; d < D; ++d) mu[d] += X[(size_t)k * D + d];
        for (int d = 0; d < D; ++d) mu[d] = Ms > 0 ? mu[d] / Ms : 0.0;
        std::vector<float> s_col(g.M_pad, 0.f), alpha_pad(g.M_pad, 0.f);
        std::vector<uint16_t> Bhi((size_t)g.M_pad * D16, 0), Blo((size_t)g.M_pad * D16, 0),
            BThi((size_t)D16 * g.M_pad, 0), BTlo((size_t)D16 * g.M_pad, 0), Bmid((size_t)g.M_pad * D16, 0),
            Blo3((size_t)g.M_pad * D16, 0), BTmid((size_t)D16 * g.M_pad, 0), BTlo3((size_t)D16 * g.M_pad, 0);
        for (int k = 0; k < Ms; ++k) {
            double sc = 0.0;
            for (int d = 0; d < D; ++d) {
                double x = X[(size_t)k * D + d];
                sc += x * mu[d];
                float b = (float)(x - mu[d]);
                uint16_t h = bf16_rne(b), l = bf16_rne(b - bf16_to_float(h));
                float rest = b - bf16_to_float(h);
                uint16_t m3 = bf16_rne(rest), l3 = bf16_rne(rest - bf16_to_float(m3));
                Bhi[(size_t)k * D16 + d] = h;
                Blo[(size_t)k * D16 + d] = l;
                BThi[(size_t)d * g.M_pad + k] = h;
                BTlo[(size_t)d * g.M_pad + k] = l;
                Bmid[(size_t)k * D16 + d] = m3;
                Blo3[(size_t)k * D16 + d] = l3;
                BTmid[(size_t)d * g.M_pad + k] = m3;
                BTlo3[(size_t)d * g.M_pad + k] = l3;
            }
            s_col[k] = (float)sc;
            alpha_pad[k] = (float)a[k];
        }
        for (int d = 0; d < D; ++d) mu_all[(size_t)s * D16 + d] = (float)mu[d];
        if (st == GAP_OK) st = upload(g.X64, X);
        if (st == GAP_OK) st = upload(g.a64, a);
        if (st == GAP_OK) st = upload(g.X32, X32);
        if (st == GAP_OK) st = upload(g.a32, a32);
        if (st == GAP_OK) st = upload(g.mu64, mu);
        if (st == GAP_OK) st = upload(g.s_col, s_col);
        if (st == GAP_OK) st = upload(g.alpha_pad, alpha_pad);
        if (st == GAP_OK) st = upload(g.Bhi, Bhi);
        if (st == GAP_OK) st = upload(g.Blo, Blo);
        if (st == GAP_OK) st = upload(g.BThi, BThi);
        if (st == GAP_OK) st = upload(g.BTlo, BTlo);
        if (st == GAP_OK) st = upload(g.Bmid, Bmid);
        if (st == GAP_OK) st = upload(g.Blo3, Blo3);
        if (st == GAP_OK) st = upload(g.BTmid, BTmid);
        if (st == GAP_OK) st = upload(g.BTlo3, BTlo3);
    }
    if (st == GAP_OK) st = upload(m->mu_all, mu_all);
    if (st == GAP_OK && tb && tb->n_sparse > 0) {
        m->has_tb = true;
        std::vector<double> x(tb->x, tb->x + tb->n_sparse), a(tb->alpha, tb->alpha + tb->n_sparse);
        st = upload(m->tb_x, x);
        if (st == GAP_OK) st = upload(m->tb_a, a);
        m->tb = TwoBodyDev{tb->n_sparse, tb->cutoff, tb->cutoff_transition_width, tb->theta, tb->delta,
                           m->tb_x.as<double>(), m->tb_a.as<double>(), nullptr, 0, 0, 0.0, 0.0};
        // ~8192 intervals of equal width on the two pieces of [0, rc]
        const double rin = tb->cutoff - tb->cutoff_transition_width;
        m->tb.g_in = rin > 0.0 ? (int)std::ceil(8192.0 * rin / tb->cutoff) : 0;
        m->tb.g_out = (int)std::ceil(8192.0 * tb->cutoff_transition_width / tb->cutoff);
        if (m->tb.g_out < 1) m->tb.g_out = 1;
        m->tb.h_in = m->tb.g_in > 0 ? rin / m->tb.g_in : 1.0;
        m->tb.h_out = tb->cutoff_transition_width / m->tb.g_out;
        if (st == GAP_OK) st = m->tb_tab.ensure(sizeof(D4) * (size_t)(m->tb.g_in + m->tb.g_out));
        if (st == GAP_OK) {
            m->tb.tab = m->tb_tab.as<D4>();
            st = gap_twobody_table(m->tb, m->tb_tab.as<D4>(), 0);
        }
        if (st == GAP_OK) st = gap_cuda_status(cudaDeviceSynchronize(), "two-body table");
    }
    if (st != GAP_OK) {
        release_model(m);
        delete m;
        return st;
    }
    ++soap->refs;
    *out = m;
    return GAP_OK;
    GAP_API_END
}

static void model_release(gap_model *m)
{
    if (--m->refs > 0) return;
    gap_soap *soap = m->soap;
    {
        DeviceGuard dg(soap->device);
        release_model(m);
        delete m;
    }
    soap_release(soap);
}

extern "C" gap_status gap_model_destroy(gap_model *m)
{
    GAP_API_BEGIN
    if (!m) return GAP_OK;
    model_release(m);
    return GAP_OK;
    GAP_API_END
}

__global__ void k_set_alpha(const double *__restrict__ a, int M, int M_pad, double *__restrict__ a64,
                            float *__restrict__ a32, float *__restrict__ apad)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M_pad) return;
    double v = k < M ? a[k] : 0.0;
    if (k < M) {
        a64[k] = v;
        a32[k] = (float)v;
    }
    apad[k] = (float)v;
}

// The model's coefficients from a device array [M_total] (caller holds m->mu).
static gap_status set_alpha_dev(gap_model *m, const double *src, cudaStream_t st)
{
    size_t off = 0;
    for (auto &g : m->gp) {
        if (g.M) {
            gap_count_launch();
            k_set_alpha<<<(g.M_pad + 255) / 256, 256, 0, st>>>(src + off, g.M, g.M_pad, g.a64.as<double>(),
                                                                g.a32.as<float>(), g.alpha_pad.as<float>());
            GAP_TRY_CUDA(cudaGetLastError());
        }
        off += g.M;
    }
    return GAP_OK;
}

extern "C" gap_status gap_model_set_alpha(gap_model *m, const double *alpha, int device_ptr, void *stream)
{
    GAP_API_BEGIN
    if (!m) { gap_set_error("model is NULL"); return GAP_EINVAL; }
    int Mt = 0;
    for (auto &g : m->gp) Mt += g.M;
    if (Mt == 0) return GAP_OK;
    if (!alpha) { gap_set_error("alpha is NULL"); return GAP_EINVAL; }
    std::lock_guard<std::mutex> lk(m->mu);
    DeviceGuard dg(m->soap->device);
    cudaStream_t st = (cudaStream_t)stream;
    const double *src = alpha;
    DBuf tmp;
    if (!device_ptr) {
        GAP_TRY(tmp.ensure(sizeof(double) * Mt));
        GAP_TRY_CUDA(cudaMemcpyAsync(tmp.p, alpha, sizeof(double) * Mt, cudaMemcpyHostToDevice, st));
        src = tmp.as<double>();
    }
    GAP_TRY(set_alpha_dev(m, src, st));
    if (!device_ptr) GAP_TRY_CUDA(cudaStreamSynchronize(st));
    tmp.release();
    return GAP_OK;
    GAP_API_END
}

extern "C" gap_status gap_model_columns(const gap_model *m, int *M_total)
{
    if (!m || !M_total) { gap_set_error("NULL argument"); return GAP_EINVAL; }
    int t = 0;
    for (auto &g : m->gp) t += g.M;
    *M_total = t;
    return GAP_OK;
}

// -------------------------------------------------------------- predict
template <typename T> static const T *gp_X(const GPData &g);
template <> const double *gp_X<double>(const GPData &g) { return g.X64.as<double>(); }
template <> const float *gp_X<float>(const GPData &g) { return g.X32.as<float>(); }
template <typename T> static const T *gp_alpha(const GPData &g);
template <> const double *gp_alpha<double>(const GPData &g) { return g.a64.as<double>(); }
template <> const float *gp_alpha<float>(const GPData &g) { return g.a32.as<float>(); }

// Rows of every GP (atoms of species s); counts copied to host.
static gap_status gp_rows_all(gap_model *m, Workspace &w, int n, const int *spec, std::vector<int> &counts,
                              cudaStream_t st)
{
    int G = m->n_gp;
    GAP_TRY(w.gp_of_atom.ensure(sizeof(int) * (size_t)n));
    GAP_TRY(w.flag.ensure(sizeof(int) * (size_t)n));
    GAP_TRY(w.fpos.ensure(sizeof(int) * (size_t)(n + 1)));
    GAP_TRY(w.scan_tmp.ensure(sizeof(int) * gap_scan_tmp_ints(n)));
    GAP_TRY(w.rows.ensure(sizeof(int) * (size_t)(G > 0 ? G : 1) * n));
    GAP_TRY(w.counts.ensure(sizeof(int) * (size_t)(G + 1)));
    GAP_TRY(gap_fill_int(w.gp_of_atom.as<int>(), n, -1, st));
    for (int s = 0; s < G; ++s)
        GAP_TRY(gap_gp_rows(n, spec, s, w.flag.as<int>(), w.fpos.as<int>(), w.scan_tmp.as<int>(),
                            w.rows.as<int>() + (size_t)s * n, w.counts.as<int>() + s, w.gp_of_atom.as<int>(), st));
    if (w.graph) {
        counts = w.counts_fixed;
        return GAP_OK;
    }
    counts.assign(G, 0);
    if (G > 0) {
        GAP_TRY_CUDA(cudaMemcpyAsync(counts.data(), w.counts.p, sizeof(int) * G, cudaMemcpyDeviceToHost, st));
        GAP_TRY_CUDA(cudaStreamSynchronize(st));
    }
    w.counts_fixed = counts;
    return GAP_OK;
}

template <typename T>
static gap_status predict_impl(gap_model *m, Workspace &w, const gap_batch *b, gap_precision prec, double *energy,
                               double *local_e, double *forces, double *virial, cudaStream_t st)
{
    gap_soap *soap = m->soap;
    const SoapGeom &g = soap->geo;
    const int n = b->n_atoms, C = b->n_configs;
    const int *spec;
    GAP_TRY(run_descriptor<T>(soap, w, b, &spec, st));
    const PairList &pl = w.nbr.pairs;
    std::vector<int> counts;
    gap_prof_begin(ST_GP_ROWS, st);
    GAP_TRY(gp_rows_all(m, w, n, spec, counts, st));
    gap_prof_end(ST_GP_ROWS, st);

    // Forces and virial need the backward pass (Eq. 3); energies alone do not.
    const bool grad = forces != nullptr || virial != nullptr;
    const int Dg = soap->Dg, Dg16 = soap->Dg16;  // the GP's descriptor (compressed or not)
    const T *phg = gp_phat<T>(soap, w);
    GAP_TRY(w.gvec.ensure(sizeof(T) * (size_t)n * Dg16));
    GAP_TRY(w.eps.ensure(sizeof(double) * (size_t)n));
    GAP_TRY(w.wsum.ensure(sizeof(float) * (size_t)n));
    T *gvec = grad ? w.gvec.as<T>() : nullptr;
    if (n > 0) {
        if (grad) GAP_TRY_CUDA(cudaMemsetAsync(w.gvec.p, 0, sizeof(T) * (size_t)n * Dg16, st));
        GAP_TRY_CUDA(cudaMemsetAsync(w.eps.p, 0, sizeof(double) * (size_t)n, st));
        GAP_TRY_CUDA(cudaMemsetAsync(w.wsum.p, 0, sizeof(float) * (size_t)n, st));
    }
    const bool tc = prec == GAP_BF16X3 || prec == GAP_BF16X6;
    const int nsplit = prec == GAP_BF16X6 ? 3 : 2;
    int n_active = 0;
    for (int s = 0; s < m->n_gp; ++s) n_active += counts[s] > 0 && m->gp[s].M > 0;
    bool grouped = false;
    if constexpr (sizeof(T) == 4) {
        if (tc && n_active >= 2) {
            // several GPs: one persistent launch per GEMM stage over all of
            // them, each GP with its own slice of the scratch buffers
            grouped = true;
            size_t ra = 0, rw = 0, rp = 0, rr = 0;
            for (int s = 0; s < m->n_gp; ++s) {
                const size_t R = counts[s];
                ra += R * Dg16;
                rw += R * m->gp[s].M_pad;
                rp += R * gap_tc_max_parts(m->gp[s].M_pad);
                rr += R;
            }
            GAP_TRY(w.A_hi.ensure(2 * ra));
            GAP_TRY(w.A_lo.ensure(2 * ra));
            GAP_TRY(w.t_row.ensure(4 * rr));
            GAP_TRY(w.W_hi.ensure(2 * rw));
            GAP_TRY(w.W_lo.ensure(2 * rw));
            if (nsplit == 3) {
                GAP_TRY(w.A_mid.ensure(2 * ra));
                GAP_TRY(w.W_mid.ensure(2 * rw));
            }
            GAP_TRY(w.epart_f.ensure(4 * rp));
            GAP_TRY(w.wpart_f.ensure(4 * rp));
            GAP_TRY(w.Gs.ensure(4 * ra));
            std::vector<TcScratch> scs(m->n_gp);
            std::vector<TcModelGP> mgs(m->n_gp);
            std::vector<const int *> rws(m->n_gp);
            std::vector<int> nrs(m->n_gp);
            size_t oa = 0, ow = 0, op = 0, orr = 0;
            const bool three = nsplit == 3;
            for (int s = 0; s < m->n_gp; ++s) {
                const GPData &gp = m->gp[s];
                const size_t R = counts[s];
                nrs[s] = gp.M > 0 ? (int)R : 0;
                rws[s] = w.rows.as<int>() + (size_t)s * n;
                scs[s] = TcScratch{w.A_hi.as<__nv_bfloat16>() + oa, w.A_lo.as<__nv_bfloat16>() + oa,
                                   w.t_row.as<float>() + orr, w.W_hi.as<__nv_bfloat16>() + ow,
                                   w.W_lo.as<__nv_bfloat16>() + ow, w.epart_f.as<float>() + op,
                                   w.wpart_f.as<float>() + op, w.Gs.as<float>() + oa,
                                   three ? w.A_mid.as<__nv_bfloat16>() + oa : nullptr,
                                   three ? w.W_mid.as<__nv_bfloat16>() + ow : nullptr};
                mgs[s] = TcModelGP{gp.M, gp.M_pad, m->mu_all.as<float>() + (size_t)s * Dg16, gp.s_col.as<float>(),
                                   gp.alpha_pad.as<float>(), gp.Bhi.as<__nv_bfloat16>(),
                                   (three ? gp.Blo3 : gp.Blo).as<__nv_bfloat16>(), gp.BThi.as<__nv_bfloat16>(),
                                   (three ? gp.BTlo3 : gp.BTlo).as<__nv_bfloat16>(), gp.Bmid.as<__nv_bfloat16>(),
                                   gp.BTmid.as<__nv_bfloat16>()};
                oa += R * Dg16;
                ow += R * gp.M_pad;
                op += R * gap_tc_max_parts(gp.M_pad);
                orr += R;
            }
            GAP_TRY(gap_contract_tc_groups((const float *)phg, Dg, Dg16, rws.data(), nrs.data(), mgs.data(), m->n_gp,
                                           m->delta, m->zeta, nsplit, scs.data(), w.eps.as<double>(),
                                           w.wsum.as<float>(), (float *)gvec, w.err.as<int>() + 2, st));
        }
    }
    for (int s = 0; s < m->n_gp && !grouped; ++s) {
        const GPData &gp = m->gp[s];
        int R = counts[s];
        if (R == 0 || gp.M == 0) continue;
        const int *rows = w.rows.as<int>() + (size_t)s * n;
        if (!tc) {
            int nt = (gp.M + 63) / 64;
            GAP_TRY(w.W.ensure(sizeof(T) * (size_t)R * gp.M));
            GAP_TRY(w.eps_part.ensure(sizeof(double) * (size_t)R * nt));
            GAP_TRY(gap_contract_simt<T>(phg, Dg, Dg16, rows, w.counts.as<int>() + s, R, gp_X<T>(gp),
                                         gp_alpha<T>(gp), gp.M, m->delta, m->zeta, w.W.as<T>(),
                                         w.eps_part.as<double>(), gvec, w.eps.as<double>(), st));
        } else {
            if constexpr (sizeof(T) == 4) {
                int n_part = gap_tc_max_parts(gp.M_pad);
                GAP_TRY(w.A_hi.ensure(2 * (size_t)R * Dg16));
                GAP_TRY(w.A_lo.ensure(2 * (size_t)R * Dg16));
                GAP_TRY(w.t_row.ensure(4 * (size_t)R));
                GAP_TRY(w.W_hi.ensure(2 * (size_t)R * gp.M_pad));
                GAP_TRY(w.W_lo.ensure(2 * (size_t)R * gp.M_pad));
                if (nsplit == 3) {
                    GAP_TRY(w.A_mid.ensure(2 * (size_t)R * Dg16));
                    GAP_TRY(w.W_mid.ensure(2 * (size_t)R * gp.M_pad));
                }
                GAP_TRY(w.epart_f.ensure(4 * (size_t)R * n_part));
                GAP_TRY(w.wpart_f.ensure(4 * (size_t)R * n_part));
                GAP_TRY(w.Gs.ensure(4 * (size_t)R * Dg16));
                TcScratch sc{w.A_hi.as<__nv_bfloat16>(), w.A_lo.as<__nv_bfloat16>(), w.t_row.as<float>(),
                             w.W_hi.as<__nv_bfloat16>(), w.W_lo.as<__nv_bfloat16>(), w.epart_f.as<float>(),
                             w.wpart_f.as<float>(), w.Gs.as<float>(), w.A_mid.as<__nv_bfloat16>(),
                             w.W_mid.as<__nv_bfloat16>()};
                const bool three = nsplit == 3;
                TcModelGP mg{gp.M, gp.M_pad, m->mu_all.as<float>() + (size_t)s * Dg16, gp.s_col.as<float>(),
                             gp.alpha_pad.as<float>(), gp.Bhi.as<__nv_bfloat16>(),
                             (three ? gp.Blo3 : gp.Blo).as<__nv_bfloat16>(), gp.BThi.as<__nv_bfloat16>(),
                             (three ? gp.BTlo3 : gp.BTlo).as<__nv_bfloat16>(), gp.Bmid.as<__nv_bfloat16>(),
                             gp.BTmid.as<__nv_bfloat16>()};
                GAP_TRY(gap_contract_tc((const float *)phg, Dg, Dg16, rows, R, mg, m->delta, m->zeta, nsplit, sc,
                                        w.eps.as<double>(), w.wsum.as<float>(), (float *)gvec,
                                        w.err.as<int>() + 2, st));
            }
        }
    }
    // backward: d eps / d p_hat -> Gamma -> per-pair derivatives
    if (grad) {
        GAP_TRY(w.Gam.ensure(sizeof(T) * (size_t)n * g.S * g.N * g.LM));
        gap_prof_begin(ST_CHAIN, st);
        if (soap->comp) {
            // back through the compression: dE/dp = Q^T dE/dp~ (times |p|)
            GAP_TRY(w.hfull.ensure(sizeof(T) * (size_t)n * g.D16));
            if (n > 0) {
                const size_t shm = sizeof(T) * (size_t)Dg;
                GAP_TRY(shm_attr<T>((const void *)k_decompress<T>, shm));
                gap_count_launch();
                k_decompress<T><<<n, 128, shm, st>>>(n, g.D, g.D16, Dg, Dg16, q_of<T>(soap), w.gvec.as<T>(),
                                                     tc ? w.wsum.as<float>() : nullptr,
                                                     tc ? m->mu_all.as<float>() : nullptr, w.gp_of_atom.as<int>(),
                                                     w.phatc.as<T>(), w.pnormc.as<T>(), w.pnorm.as<T>(),
                                                     w.hfull.as<T>());
                GAP_TRY_CUDA(cudaGetLastError());
            }
            GAP_TRY(gap_chain<T>(g, n, w.hfull.as<T>(), nullptr, nullptr, w.gp_of_atom.as<int>(), w.phat.as<T>(),
                                 w.pnorm.as<T>(), w.coef.as<T>(), w.Gam.as<T>(), st));
        } else {
            GAP_TRY(gap_chain<T>(g, n, w.gvec.as<T>(), tc ? (const T *)w.wsum.p : nullptr,
                                 tc ? (const T *)m->mu_all.p : nullptr, w.gp_of_atom.as<int>(), w.phat.as<T>(),
                                 w.pnorm.as<T>(), w.coef.as<T>(), w.Gam.as<T>(), st));
        }
        gap_prof_end(ST_CHAIN, st);
        GAP_TRY(w.fpair.ensure(sizeof(T) * 3 * (size_t)pl.n_pairs));
        gap_prof_begin(ST_PAIRFORCE, st);
        GAP_TRY(gap_pairforce<T>(g, tab_of<T>(soap), pl, w.pair_i.as<int>(), spec, w.Gam.as<T>(), w.fpair.as<T>(), st));
        gap_prof_end(ST_PAIRFORCE, st);
    }
    double *eps2 = nullptr, *f2 = nullptr;
    if (m->has_tb) {
        GAP_TRY(w.eps2.ensure(sizeof(double) * (size_t)n));
        GAP_TRY(w.f2.ensure(sizeof(double) * 3 * (size_t)pl.n_pairs));
        eps2 = w.eps2.as<double>();
        f2 = w.f2.as<double>();
        gap_prof_begin(ST_TWOBODY, st);
        GAP_TRY(gap_twobody(n, pl, m->tb, f2, eps2, st));
        gap_prof_end(ST_TWOBODY, st);
    }
    // outputs
    double *d_forces = forces, *d_energy = energy, *d_virial = virial, *d_local = local_e;
    if (!b->device) {
        GAP_TRY(w.forces.ensure(sizeof(double) * 3 * (size_t)n));
        GAP_TRY(w.energy.ensure(sizeof(double) * (size_t)C));
        GAP_TRY(w.virial.ensure(sizeof(double) * 9 * (size_t)C));
        GAP_TRY(w.local.ensure(sizeof(double) * (size_t)n));
        d_forces = forces ? w.forces.as<double>() : nullptr;
        d_energy = energy ? w.energy.as<double>() : nullptr;
        d_virial = virial ? w.virial.as<double>() : nullptr;
        d_local = local_e ? w.local.as<double>() : nullptr;
    }
    double *vir_atom = nullptr;
    if (virial) {
        GAP_TRY(w.vir_atom.ensure(sizeof(double) * 9 * (size_t)n));
        vir_atom = w.vir_atom.as<double>();
    }
    gap_prof_begin(ST_GATHER, st);
    if (d_forces || vir_atom) GAP_TRY(gap_gather<T>(n, pl, w.fpair.as<T>(), f2, d_forces, vir_atom, st));
    if (d_energy || d_virial) {
        int max_atoms = 0;
        for (int c = 0; c < C; ++c) {
            const int na = b->config_offsets[c + 1] - b->config_offsets[c];
            if (na > max_atoms) max_atoms = na;
        }
        GAP_TRY(w.cfgpart.ensure(sizeof(double) * gap_config_part_doubles(C, max_atoms)));
        GAP_TRY(gap_config_sums(C, w.nbr.cfg_offsets, max_atoms, w.eps.as<double>(), eps2, vir_atom, d_energy,
                                d_virial, w.cfgpart.as<double>(), st));
    }
    if (d_local) GAP_TRY(gap_local_energy(n, w.eps.as<double>(), eps2, d_local, st));
    gap_prof_end(ST_GATHER, st);
    if (!b->device) {
        if (forces && n) GAP_TRY_CUDA(cudaMemcpyAsync(forces, d_forces, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
        if (energy && C) GAP_TRY_CUDA(cudaMemcpyAsync(energy, d_energy, sizeof(double) * C, cudaMemcpyDeviceToHost, st));
        if (virial && C) GAP_TRY_CUDA(cudaMemcpyAsync(virial, d_virial, sizeof(double) * 9 * C, cudaMemcpyDeviceToHost, st));
        if (local_e && n) GAP_TRY_CUDA(cudaMemcpyAsync(local_e, d_local, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    }
    if (w.graph) return GAP_OK;  // errors are read by gap_step_graph_status
    return check_device_errors(w, st);
}

extern "C" gap_status gap_predict(gap_model *m, const gap_batch *b, gap_precision prec, double *energy,
                                  double *local_e, double *forces, double *virial, void *stream)
{
    GAP_API_BEGIN
    if (!m) { gap_set_error("model is NULL"); return GAP_EINVAL; }
    GAP_TRY(check_batch(b));
    std::lock_guard<std::mutex> lk(m->mu);
    DeviceGuard dg(m->soap->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == GAP_FP64) return predict_impl<double>(m, m->ws, b, prec, energy, local_e, forces, virial, st);
    if (prec == GAP_BF16X3 || prec == GAP_BF16X6 || prec == GAP_FP32)
        return predict_impl<float>(m, m->ws, b, prec, energy, local_e, forces, virial, st);
    gap_set_error("bad precision");
    return GAP_EINVAL;
    GAP_API_END
}

// ------------------------------------------------------ captured MD step
// One gap_predict of a fixed batch layout recorded as a CUDA graph, for an MD
// loop that moves the atoms in place between steps.  The graph owns its
// workspace, so ordinary calls on the same model cannot move its buffers.
struct gap_step_graph {
    gap_model *m = nullptr;
    Workspace ws;
    gap_precision prec = GAP_BF16X3;
    gap_batch b{};
    std::vector<int> offsets, pbc;
    std::vector<double> cell;
    double *energy = nullptr, *local_e = nullptr, *forces = nullptr, *virial = nullptr;
    cudaGraphExec_t exec = nullptr;
    long n_kernels = 0;
};

template <typename T>
static gap_status step_graph_capture(gap_step_graph *G, double factor, cudaStream_t st)
{
    Workspace &w = G->ws;
    // An ordinary call sizes every buffer, uploads the cell geometry and
    // fixes the rows of each GP.
    GAP_TRY(predict_impl<T>(G->m, w, &G->b, G->prec, G->energy, G->local_e, G->forces, G->virial, st));
    const double cap = std::ceil(factor * (double)w.nbr.pairs.n_pairs);
    if (cap > (double)(1 << 30)) { gap_set_error("pair capacity too large"); return GAP_EINVAL; }
    w.graph = true;
    w.nbr.graph = true;
    w.nbr.pair_cap = (int)cap;
    // An uncaptured graph-mode call grows the pair buffers to the capacity,
    // so that nothing is allocated while capturing.
    GAP_TRY(predict_impl<T>(G->m, w, &G->b, G->prec, G->energy, G->local_e, G->forces, G->virial, st));
    GAP_TRY(check_device_errors(w, st));
    cudaStream_t cs = nullptr;
    GAP_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const bool prof = g_prof.on;
    g_prof.on = false;
    const long k0 = g_launches.load();
    gap_status rc = gap_cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaGraph_t graph = nullptr;
    if (rc == GAP_OK) {
        rc = predict_impl<T>(G->m, w, &G->b, G->prec, G->energy, G->local_e, G->forces, G->virial, cs);
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (rc == GAP_OK) rc = gap_cuda_status(e, "end capture");
    }
    G->n_kernels = g_launches.load() - k0;
    g_launches -= G->n_kernels;  // counted when the graph runs
    g_prof.on = prof;
    if (rc == GAP_OK) rc = gap_cuda_status(cudaGraphInstantiate(&G->exec, graph, 0), "cudaGraphInstantiate");
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (rc != GAP_OK) cudaGetLastError();
    return rc;
}

static void step_graph_free(gap_step_graph *G)
{
    {
        DeviceGuard dg(G->m->soap->device);
        if (G->exec) cudaGraphExecDestroy(G->exec);
        G->ws.release();
    }
    model_release(G->m);
    delete G;
}

extern "C" gap_status gap_step_graph_create(gap_model *m, const gap_batch *b, gap_precision prec,
                                            double pair_capacity, double *energy, double *local_e, double *forces,
                                            double *virial, void *stream, gap_step_graph **out)
{
    GAP_API_BEGIN
    if (!out) { gap_set_error("out is NULL"); return GAP_EINVAL; }
    *out = nullptr;
    if (!m) { gap_set_error("model is NULL"); return GAP_EINVAL; }
    GAP_TRY(check_batch(b));
    if (!b->device) { gap_set_error("a step graph needs device positions, species and outputs"); return GAP_EINVAL; }
    if (!(pair_capacity >= 1.0) || !std::isfinite(pair_capacity)) {
        gap_set_error("pair_capacity must be >= 1");
        return GAP_EINVAL;
    }
    if (prec != GAP_FP64 && prec != GAP_FP32 && prec != GAP_BF16X3 && prec != GAP_BF16X6) {
        gap_set_error("bad precision");
        return GAP_EINVAL;
    }
    DeviceGuard dg(m->soap->device);
    gap_step_graph *G = new gap_step_graph();
    ++m->refs;
    G->m = m;
    G->prec = prec;
    const int C = b->n_configs;
    G->offsets.assign(b->config_offsets, b->config_offsets + C + 1);
    G->pbc.assign(b->pbc, b->pbc + 3 * C);
    G->cell.assign(b->cell, b->cell + 9 * C);
    G->b = *b;
    G->b.config_offsets = G->offsets.data();
    G->b.pbc = G->pbc.data();
    G->b.cell = G->cell.data();
    G->energy = energy;
    G->local_e = local_e;
    G->forces = forces;
    G->virial = virial;
    cudaStream_t st = (cudaStream_t)stream;
    gap_status rc;
    {
        std::lock_guard<std::mutex> lk(m->mu);
        rc = prec == GAP_FP64 ? step_graph_capture<double>(G, pair_capacity, st)
                              : step_graph_capture<float>(G, pair_capacity, st);
    }
    if (rc != GAP_OK) {
        step_graph_free(G);
        return rc;
    }
    *out = G;
    return GAP_OK;
    GAP_API_END
}

extern "C" gap_status gap_step_graph_launch(gap_step_graph *G, void *stream)
{
    GAP_API_BEGIN
    if (!G || !G->exec) { gap_set_error("graph is NULL"); return GAP_EINVAL; }
    DeviceGuard dg(G->m->soap->device);
    GAP_TRY_CUDA(cudaGraphLaunch(G->exec, (cudaStream_t)stream));
    g_launches += G->n_kernels;
    return GAP_OK;
    GAP_API_END
}

extern "C" gap_status gap_step_graph_status(gap_step_graph *G, void *stream)
{
    GAP_API_BEGIN
    if (!G) { gap_set_error("graph is NULL"); return GAP_EINVAL; }
    DeviceGuard dg(G->m->soap->device);
    return check_device_errors(G->ws, (cudaStream_t)stream);
    GAP_API_END
}

extern "C" long gap_step_graph_kernels(const gap_step_graph *G) { return G ? G->n_kernels : 0; }

extern "C" gap_status gap_step_graph_destroy(gap_step_graph *G)
{
    GAP_API_BEGIN
    if (!G) return GAP_OK;
    step_graph_free(G);
    return GAP_OK;
    GAP_API_END
}

// knm == NULL keeps K_NM in the workspace (w.Kbuf) whatever the batch's
// memory: the fused fit reads it there.
template <typename T>
static gap_status knm_impl(gap_model *m, const gap_batch *b, gap_precision prec, double *knm, cudaStream_t st)
{
    gap_soap *soap = m->soap;
    const SoapGeom &g = soap->geo;
    // the GP's descriptor: p_hat (g.D), or the compressed p_hat~ (Dg), whose
    // Jacobian rows are those of p_hat mapped by gap_jacobian_compress
    const bool cmp = soap->comp != 0;
    const int Dg = soap->Dg, Dg16 = soap->Dg16;
    const int Dw = cmp && Dg16 > g.D16 ? Dg16 : g.D16;  // width of the row planes
    Workspace &w = m->ws;
    const int n = b->n_atoms, C = b->n_configs;
    const bool tc = prec == GAP_BF16X3 || prec == GAP_BF16X6;
    const int nsplit = prec == GAP_BF16X6 ? 3 : 2;
    const bool three = nsplit == 3;
    int Mt = 0;
    std::vector<int> col_off(m->n_gp + 1, 0);
    for (int s = 0; s < m->n_gp; ++s) col_off[s + 1] = col_off[s] + m->gp[s].M;
    Mt = col_off[m->n_gp];
    const size_t krows = (size_t)C + 3 * (size_t)n;
    double *K = knm;
    if (!b->device || !knm) {
        GAP_TRY(w.Kbuf.ensure(sizeof(double) * krows * (Mt > 0 ? Mt : 1)));
        K = w.Kbuf.as<double>();
    }
    if (krows * Mt) GAP_TRY_CUDA(cudaMemsetAsync(K, 0, sizeof(double) * krows * Mt, st));
    const int *spec;
    GAP_TRY(run_descriptor<T>(soap, w, b, &spec, st));
    const PairList &pl = w.nbr.pairs;
    std::vector<int> counts;
    GAP_TRY(gp_rows_all(m, w, n, spec, counts, st));
    const size_t nrow = 3 * ((size_t)n + pl.n_pairs);
    const int nseg = 3 * n;
    GAP_TRY(w.segstart.ensure(sizeof(int) * (nseg + 1)));
    GAP_TRY(w.outrow.ensure(sizeof(int) * (nseg + 1)));
    GAP_TRY(w.ksrc.ensure(sizeof(int) * nrow));
    GAP_TRY(w.kseg.ensure(sizeof(int) * nrow));
    gap_prof_begin(ST_KNM_ROWS, st);
    GAP_TRY(gap_knm_segments(n, pl.offsets, w.nbr.atom_cfg, w.segstart.as<int>(), w.outrow.as<int>(), st));
    KnmRows rows{};
    rows.src_sign = w.ksrc.as<int>();
    rows.seg = w.kseg.as<int>();
    if (tc) {
        if constexpr (sizeof(T) == 4) {
            GAP_TRY(w.kAhi.ensure(2 * nrow * Dw));
            GAP_TRY(w.kAlo.ensure(2 * nrow * Dw));
            GAP_TRY(w.kt.ensure(4 * nrow));
            rows.A_hi = w.kAhi.as<__nv_bfloat16>();
            rows.A_lo = w.kAlo.as<__nv_bfloat16>();
            if (three) {
                GAP_TRY(w.kAmid.ensure(2 * nrow * Dw));
                rows.A_mid = w.kAmid.as<__nv_bfloat16>();
            }
            rows.t_row = w.kt.as<float>();
            gap_prof_begin(ST_KNM_JACOBIAN, st);
            GAP_TRY((gap_jacobian_rows<float, true>(g, tab_of<float>(soap), n, pl, spec, w.coef.as<float>(),
                                                    w.phat.as<float>(), w.pnorm.as<float>(), w.gp_of_atom.as<int>(),
                                                    cmp ? nullptr : m->mu_all.as<float>(), rows, st)));
            if (cmp && nrow) {
                // V = J Q^T on the tensor cores (J's planes against Q's), then
                // J~ into the same planes (J is consumed by then), Dg16 wide
                GAP_TRY(w.kV.ensure(4 * nrow * Dg16));
                TcOperands opq{w.kAhi.as<__nv_bfloat16>(), w.kAlo.as<__nv_bfloat16>(),
                               soap->Qhi.as<__nv_bfloat16>(), (three ? soap->Qlo3 : soap->Qlo).as<__nv_bfloat16>(),
                               (int)nrow, Dg, g.D16, g.D16, g.D16, nsplit,
                               three ? w.kAmid.as<__nv_bfloat16>() : nullptr,
                               three ? soap->Qmid.as<__nv_bfloat16>() : nullptr};
                TcEpilogue eq{};
                eq.C = w.kV.as<float>();
                eq.ldc = Dg16;
                GAP_TRY(gap_tc_gemm(opq, eq, EPI_STORE, w.err.as<int>() + 2, st));
                GAP_TRY((gap_jacobian_compress<float, true>((long)nrow, Dg, Dg16, w.kV.as<float>(), Dg16,
                                                            w.ksrc.as<int>(), w.gp_of_atom.as<int>(),
                                                            w.phatc.as<float>(), w.pnorm.as<float>(),
                                                            w.pnormc.as<float>(), m->mu_all.as<float>(), rows, st)));
            }
            gap_prof_end(ST_KNM_JACOBIAN, st);
        }
    } else {
        GAP_TRY(w.kA.ensure(sizeof(T) * nrow * g.D16));
        rows.A = w.kA.p;
        gap_prof_begin(ST_KNM_JACOBIAN, st);
        GAP_TRY((gap_jacobian_rows<T, false>(g, tab_of<T>(soap), n, pl, spec, w.coef.as<T>(), w.phat.as<T>(),
                                             w.pnorm.as<T>(), w.gp_of_atom.as<int>(), m->mu_all.as<float>(), rows,
                                             st)));
        if (cmp && nrow) {
            // V = J Q^T, then J~ in place: the force GEMM reads kV [nrow][Dg16]
            GAP_TRY(w.kV.ensure(sizeof(T) * nrow * Dg16));
            GAP_TRY(gap_rows_times_qt<T>((long)nrow, g.D, w.kA.as<T>(), g.D16, Dg, q_of<T>(soap), w.kV.as<T>(), Dg16,
                                         st));
            rows.A = w.kV.p;
            GAP_TRY((gap_jacobian_compress<T, false>((long)nrow, Dg, Dg16, w.kV.as<T>(), Dg16, w.ksrc.as<int>(),
                                                     w.gp_of_atom.as<int>(), w.phatc.as<T>(), w.pnorm.as<T>(),
                                                     w.pnormc.as<T>(), nullptr, rows, st)));
        }
        gap_prof_end(ST_KNM_JACOBIAN, st);
    }
    if (tc) {  // destinations of the tensor-core epilogue's segment sums (all GPs)
        GAP_TRY(w.kdest.ensure(sizeof(int) * (nrow > 0 ? nrow : 1)));
        GAP_TRY(gap_knm_dest((long)nrow, w.kseg.as<int>(), w.segstart.as<int>(), w.outrow.as<int>(),
                             w.kdest.as<int>(), st));
    }
    gap_prof_end(ST_KNM_ROWS, st);
    for (int s = 0; s < m->n_gp; ++s) {
        const GPData &gp = m->gp[s];
        if (gp.M == 0) continue;
        const int R = counts[s];
        const int *grow = w.rows.as<int>() + (size_t)s * n;
        const int ld = tc ? gp.M_pad : gp.M;
        const __nv_bfloat16 *Blo = (three ? gp.Blo3 : gp.Blo).as<__nv_bfloat16>();
        const size_t wbytes = (tc ? sizeof(float) : sizeof(T)) * (size_t)n * ld;
        GAP_TRY(w.Wp.ensure(wbytes));
        GAP_TRY(w.kq.ensure(wbytes));
        if (n) {
            GAP_TRY_CUDA(cudaMemsetAsync(w.Wp.p, 0, wbytes, st));
            GAP_TRY_CUDA(cudaMemsetAsync(w.kq.p, 0, wbytes, st));
        }
        gap_prof_begin(ST_KNM_GEMM, st);
        if (tc) {
            if constexpr (sizeof(T) == 4) {
                if (R > 0) {
                    GAP_TRY(w.A_hi.ensure(2 * (size_t)R * Dg16));
                    GAP_TRY(w.A_lo.ensure(2 * (size_t)R * Dg16));
                    GAP_TRY(w.t_row.ensure(4 * (size_t)R));
                    if (three) GAP_TRY(w.A_mid.ensure(2 * (size_t)R * Dg16));
                    GAP_TRY(gap_split_rows(gp_phat<float>(soap, w), Dg, Dg16, grow, R,
                                           m->mu_all.as<float>() + (size_t)s * Dg16, w.A_hi.as<__nv_bfloat16>(),
                                           w.A_lo.as<__nv_bfloat16>(), three ? w.A_mid.as<__nv_bfloat16>() : nullptr,
                                           w.t_row.as<float>(), st));
                    TcOperands op1{w.A_hi.as<__nv_bfloat16>(), w.A_lo.as<__nv_bfloat16>(), gp.Bhi.as<__nv_bfloat16>(),
                                   Blo, R, gp.M, Dg16, Dg16, Dg16, nsplit,
                                   three ? w.A_mid.as<__nv_bfloat16>() : nullptr,
                                   three ? gp.Bmid.as<__nv_bfloat16>() : nullptr};
                    TcEpilogue e1{};
                    e1.s_col = gp.s_col.as<float>();
                    e1.t_row = w.t_row.as<float>();
                    e1.d2 = (float)(m->delta * m->delta);
                    e1.zeta = m->zeta;
                    e1.row_map = grow;
                    e1.Wp = w.Wp.as<float>();
                    e1.kq = w.kq.as<float>();
                    e1.ldwp = ld;
                    GAP_TRY(gap_tc_gemm(op1, e1, EPI_QPOW, w.err.as<int>() + 2, st));
                }
                const int tiles = (int)((nrow + 127) / 128);
                GAP_TRY(w.P.ensure(sizeof(float) * (size_t)tiles * 2 * ld));
                TcOperands op2{w.kAhi.as<__nv_bfloat16>(), w.kAlo.as<__nv_bfloat16>(), gp.Bhi.as<__nv_bfloat16>(),
                               Blo, (int)nrow, gp.M, Dg16, Dg16, Dg16, nsplit,
                               three ? w.kAmid.as<__nv_bfloat16>() : nullptr,
                               three ? gp.Bmid.as<__nv_bfloat16>() : nullptr};
                TcEpilogue e2{};
                e2.t_row = w.kt.as<float>();
                e2.Wp = w.Wp.as<float>();
                e2.ldwp = ld;
                e2.src_sign = w.ksrc.as<int>();
                e2.seg = w.kseg.as<int>();
                e2.seg_start = w.segstart.as<int>();
                e2.out_row = w.outrow.as<int>();
                e2.dest = w.kdest.as<int>();
                e2.K = K;
                e2.ldk = Mt;
                e2.col_out0 = col_off[s];
                e2.P = w.P.as<float>();
                e2.ldp = ld;
                GAP_TRY(gap_tc_gemm(op2, e2, EPI_KNM, w.err.as<int>() + 2, st));
                gap_prof_end(ST_KNM_GEMM, st);
                gap_prof_begin(ST_KNM_REDUCE, st);
                GAP_TRY(gap_knm_fixup((long)nrow, w.kseg.as<int>(), w.segstart.as<int>(), w.outrow.as<int>(),
                                      w.P.as<float>(), ld, gp.M, K, Mt, col_off[s], st));
                GAP_TRY(gap_knm_energy<float>(C, w.nbr.cfg_offsets, w.kq.as<float>(), ld, gp.M, K, Mt, col_off[s], st));
                gap_prof_end(ST_KNM_REDUCE, st);
            }
        } else {
            GAP_TRY(gap_knm_qpow_simt<T>(gp_phat<T>(soap, w), Dg, grow, R, gp_X<T>(gp), gp.M, m->delta, m->zeta, w.Wp.as<T>(),
                                         w.kq.as<T>(), ld, st));
            GAP_TRY(w.P.ensure(sizeof(T) * ((nrow + 63) / 64) * 2 * (size_t)ld));
            GAP_TRY(gap_knm_force_simt<T>(reinterpret_cast<const T *>(rows.A), Dg, Dg16, (long)nrow, w.kseg.as<int>(), nseg,
                                          w.segstart.as<int>(), w.outrow.as<int>(), w.ksrc.as<int>(), gp_X<T>(gp), gp.M,
                                          w.Wp.as<T>(), ld, K, Mt, col_off[s], w.P.as<T>(), ld, st));
            gap_prof_end(ST_KNM_GEMM, st);
            gap_prof_begin(ST_KNM_REDUCE, st);
            GAP_TRY(gap_knm_energy<T>(C, w.nbr.cfg_offsets, w.kq.as<T>(), ld, gp.M, K, Mt, col_off[s], st));
            gap_prof_end(ST_KNM_REDUCE, st);
        }
    }
    if (!b->device && knm && krows * Mt)
        GAP_TRY_CUDA(cudaMemcpyAsync(knm, K, sizeof(double) * krows * Mt, cudaMemcpyDeviceToHost, st));
    return check_device_errors(w, st);
}

extern "C" gap_status gap_assemble_knm(gap_model *m, const gap_batch *b, gap_precision prec, double *knm, void *stream)
{
    GAP_API_BEGIN
    if (!m) { gap_set_error("model is NULL"); return GAP_EINVAL; }
    GAP_TRY(check_batch(b));
    int Mt = 0;
    for (auto &g : m->gp) Mt += g.M;
    if (!knm && Mt > 0 && b->n_configs > 0) { gap_set_error("knm is NULL"); return GAP_EINVAL; }
    std::lock_guard<std::mutex> lk(m->mu);
    DeviceGuard dg(m->soap->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == GAP_FP64) return knm_impl<double>(m, b, prec, knm, st);
    if (prec == GAP_BF16X3 || prec == GAP_BF16X6 || prec == GAP_FP32) return knm_impl<float>(m, b, prec, knm, st);
    gap_set_error("bad precision");
    return GAP_EINVAL;
    GAP_API_END
}

// The least-squares solve on device arrays (caller holds m->mu): K [rows][Mt],
// y and sigma [rows], alpha [Mt].
// All GPs' sparse points [M_total][D] and the GP of each, for the solve
// (built once: the sparse points never change after the model is made).
static gap_status solve_points(gap_model *m, int Mt, cudaStream_t st)
{
    const int D = m->soap->Dg;
    gap_status rc = GAP_OK;
    if (!m->solve_X.p) {
        rc = m->solve_X.ensure(sizeof(double) * (size_t)Mt * D);
        if (rc == GAP_OK) rc = m->solve_blk.ensure(sizeof(int) * (size_t)Mt);
        std::vector<int> hb(Mt);
        size_t off = 0;
        for (int s = 0; s < m->n_gp && rc == GAP_OK; ++s) {
            const GPData &g = m->gp[s];
            for (int k = 0; k < g.M; ++k) hb[off + k] = s;
            if (g.M)
                rc = gap_cuda_status(cudaMemcpyAsync(m->solve_X.as<double>() + off * D, g.X64.p,
                                                     sizeof(double) * (size_t)g.M * D, cudaMemcpyDeviceToDevice, st),
                                     "copy sparse points");
            off += g.M;
        }
        if (rc == GAP_OK)
            rc = gap_cuda_status(cudaMemcpy(m->solve_blk.p, hb.data(), sizeof(int) * Mt, cudaMemcpyHostToDevice), "copy");
        if (rc != GAP_OK) {
            m->solve_X.release();
            m->solve_blk.release();
            return rc;
        }
    }
    return GAP_OK;
}

static gap_status solve_dev(gap_model *m, long rows, int Mt, const double *K, const double *Y, const double *Sg,
                            double jitter, gap_solve_method method, double *A, cudaStream_t st)
{
    const int D = m->soap->Dg;
    GAP_TRY(solve_points(m, Mt, st));
    gap_status rc = GAP_OK;
    SolveInputs in{rows, Mt, K, Y, Sg, m->solve_X.as<double>(), m->solve_blk.as<int>(), D, m->delta, jitter, m->zeta};
    rc = method == GAP_SOLVE_CHOLQR_TC ? gap_solve_tc_dev(in, A, m->solve_ws, st) : gap_solve_dev(in, A, m->solve_ws, st);
    return rc;
}

extern "C" gap_status gap_solve(gap_model *m, long rows, const double *knm, const double *y, const double *sigma,
                                double jitter, gap_solve_method method, double *alpha_out, int device_ptrs,
                                void *stream)
{
    GAP_API_BEGIN
    if (!m) { gap_set_error("model is NULL"); return GAP_EINVAL; }
    if (method != GAP_SOLVE_HOUSEHOLDER && method != GAP_SOLVE_CHOLQR_TC) {
        gap_set_error("bad solve method");
        return GAP_EINVAL;
    }
    int Mt = 0;
    for (auto &g : m->gp) Mt += g.M;
    if (rows < 0 || (Mt > 0 && (!alpha_out || (rows > 0 && (!knm || !y || !sigma))))) {
        gap_set_error("bad arguments");
        return GAP_EINVAL;
    }
    if (!(jitter >= 0.0)) { gap_set_error("jitter must be non-negative"); return GAP_EINVAL; }
    if (Mt == 0) return GAP_OK;
    std::lock_guard<std::mutex> lk(m->mu);
    DeviceGuard dg(m->soap->device);
    cudaStream_t st = (cudaStream_t)stream;
    DBuf dK, dy, ds, da;
    auto cleanup = [&]() { dK.release(); dy.release(); ds.release(); da.release(); };
    gap_status rc = GAP_OK;
    const double *K = knm, *Y = y, *Sg = sigma;
    double *A = alpha_out;
    if (!device_ptrs) {
        rc = dK.ensure(sizeof(double) * (size_t)rows * Mt);
        if (rc == GAP_OK) rc = dy.ensure(sizeof(double) * (size_t)rows);
        if (rc == GAP_OK) rc = ds.ensure(sizeof(double) * (size_t)rows);
        if (rc == GAP_OK) rc = da.ensure(sizeof(double) * (size_t)Mt);
        if (rc == GAP_OK && rows)
            rc = gap_cuda_status(cudaMemcpyAsync(dK.p, knm, sizeof(double) * (size_t)rows * Mt, cudaMemcpyHostToDevice, st), "copy K");
        if (rc == GAP_OK && rows)
            rc = gap_cuda_status(cudaMemcpyAsync(dy.p, y, sizeof(double) * (size_t)rows, cudaMemcpyHostToDevice, st), "copy y");
        if (rc == GAP_OK && rows)
            rc = gap_cuda_status(cudaMemcpyAsync(ds.p, sigma, sizeof(double) * (size_t)rows, cudaMemcpyHostToDevice, st), "copy sigma");
        K = dK.as<double>();
        Y = dy.as<double>();
        Sg = ds.as<double>();
        A = da.as<double>();
    }
    if (rc == GAP_OK) rc = solve_dev(m, rows, Mt, K, Y, Sg, jitter, method, A, st);
    if (rc == GAP_OK && !device_ptrs) {
        rc = gap_cuda_status(cudaMemcpyAsync(alpha_out, A, sizeof(double) * Mt, cudaMemcpyDeviceToHost, st), "copy alpha");
        if (rc == GAP_OK) rc = gap_cuda_status(cudaStreamSynchronize(st), "sync");
    }
    cudaStreamSynchronize(st);
    cleanup();
    return rc;
    GAP_API_END
}

extern "C" gap_status gap_fit(gap_model *m, const gap_batch *b, gap_precision prec, const double *y,
                              const double *sigma, double jitter, gap_solve_method method, double *alpha_out,
                              int device_ptrs, void *stream)
{
    GAP_API_BEGIN
    if (!m) { gap_set_error("model is NULL"); return GAP_EINVAL; }
    GAP_TRY(check_batch(b));
    if (method != GAP_SOLVE_HOUSEHOLDER && method != GAP_SOLVE_CHOLQR_TC) {
        gap_set_error("bad solve method");
        return GAP_EINVAL;
    }
    if (prec != GAP_FP64 && prec != GAP_BF16X3 && prec != GAP_BF16X6 && prec != GAP_FP32) {
        gap_set_error("bad precision");
        return GAP_EINVAL;
    }
    if (!(jitter >= 0.0)) { gap_set_error("jitter must be non-negative"); return GAP_EINVAL; }
    int Mt = 0;
    for (auto &g : m->gp) Mt += g.M;
    const long rows = (long)b->n_configs + 3L * b->n_atoms;
    if (rows > 0 && (!y || !sigma)) { gap_set_error("y or sigma is NULL"); return GAP_EINVAL; }
    if (Mt == 0) return GAP_OK;
    std::lock_guard<std::mutex> lk(m->mu);
    DeviceGuard dg(m->soap->device);
    cudaStream_t st = (cudaStream_t)stream;
    GAP_TRY(prec == GAP_FP64 ? knm_impl<double>(m, b, prec, nullptr, st) : knm_impl<float>(m, b, prec, nullptr, st));
    const double *K = m->ws.Kbuf.as<double>(), *Y = y, *Sg = sigma;
    DBuf &dy = m->fit_y, &ds = m->fit_s, &da = m->fit_a;
    gap_status rc = GAP_OK;
    if (!device_ptrs) {
        rc = dy.ensure(sizeof(double) * (size_t)(rows > 0 ? rows : 1));
        if (rc == GAP_OK) rc = ds.ensure(sizeof(double) * (size_t)(rows > 0 ? rows : 1));
        if (rc == GAP_OK && rows)
            rc = gap_cuda_status(cudaMemcpyAsync(dy.p, y, sizeof(double) * (size_t)rows, cudaMemcpyHostToDevice, st), "copy y");
        if (rc == GAP_OK && rows)
            rc = gap_cuda_status(cudaMemcpyAsync(ds.p, sigma, sizeof(double) * (size_t)rows, cudaMemcpyHostToDevice, st), "copy sigma");
        Y = dy.as<double>();
        Sg = ds.as<double>();
    }
    double *A = device_ptrs && alpha_out ? alpha_out : nullptr;
    if (rc == GAP_OK && !A) {
        rc = da.ensure(sizeof(double) * Mt);
        A = da.as<double>();
    }
    if (rc == GAP_OK) rc = solve_dev(m, rows, Mt, K, Y, Sg, jitter, method, A, st);
    if (rc == GAP_OK) rc = set_alpha_dev(m, A, st);
    if (rc == GAP_OK && alpha_out && !device_ptrs)
        rc = gap_cuda_status(cudaMemcpyAsync(alpha_out, A, sizeof(double) * Mt, cudaMemcpyDeviceToHost, st), "copy alpha");
    cudaStreamSynchronize(st);
    return rc;
    GAP_API_END
}

// ------------------------------------------------ predictive variance
__global__ void k_var_gather(const double *__restrict__ phat, int D, const int *__restrict__ rows, int nr,
                             double *__restrict__ P, double *__restrict__ pn2)
{
    // one warp per row: P[r] = phat[rows[r]], pn2[r] = |p_hat|^2
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= nr) return;
    const double *src = phat + (size_t)rows[r] * D;
    double s = 0.0;
    for (int k = lane; k < D; k += 32) {
        const double v = src[k];
        P[(size_t)r * D + k] = v;
        s = fma(v, v, s);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) pn2[r] = s;
}

__global__ void k_var_kernel(double *__restrict__ Q, long n, double d2, int zeta)
{
    // k = delta^2 q^zeta in place (Eqs. 2, 13)
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double q = Q[i];
    double z = 1.0;
    for (int t = 0; t < zeta; ++t) z *= q;
    Q[i] = d2 * z;
}

__global__ void k_var_finish(const double *__restrict__ V, int ldv, const double *__restrict__ W, int ldw, int nr,
                             const double *__restrict__ pn2, double d2, int zeta, const int *__restrict__ rows,
                             double *__restrict__ var)
{
    // var = k(x, x) - |k U^-1|^2 + |k R^-1|^2, one warp per row, fixed order
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= nr) return;
    double a = 0.0, b = 0.0;
    for (int k = lane; k < ldv; k += 32) a = fma(V[(size_t)r * ldv + k], V[(size_t)r * ldv + k], a);
    for (int k = lane; k < ldw; k += 32) b = fma(W[(size_t)r * ldw + k], W[(size_t)r * ldw + k], b);
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        double z = 1.0;
        for (int t = 0; t < zeta; ++t) z *= pn2[r];
        var[rows[r]] = d2 * z - a + b;
    }
}

extern "C" gap_status gap_model_set_posterior(gap_model *m, long rows, const double *knm, const double *sigma,
                                              double jitter, int device_ptrs, void *stream)
{
    GAP_API_BEGIN
    if (!m) { gap_set_error("model is NULL"); return GAP_EINVAL; }
    int Mt = 0;
    for (auto &g : m->gp) Mt += g.M;
    if (rows < 1 || (Mt > 0 && (!knm || !sigma))) {
        gap_set_error("gap_model_set_posterior needs rows >= 1 and non-NULL knm, sigma");
        return GAP_EINVAL;
    }
    if (!(jitter >= 0.0)) { gap_set_error("jitter must be non-negative"); return GAP_EINVAL; }
    std::lock_guard<std::mutex> lk(m->mu);
    m->has_post = false;
    if (Mt == 0) { m->has_post = true; return GAP_OK; }
    DeviceGuard dg(m->soap->device);
    cudaStream_t st = (cudaStream_t)stream;
    DBuf dK, dy, ds, da;
    auto cleanup = [&]() { dK.release(); dy.release(); ds.release(); da.release(); };
    const double *K = knm, *Sg = sigma;
    gap_status rc = dy.ensure(sizeof(double) * (size_t)(rows > 0 ? rows : 1));
    if (rc == GAP_OK && rows)
        rc = gap_cuda_status(cudaMemsetAsync(dy.p, 0, sizeof(double) * (size_t)rows, st), "cudaMemset");
    if (rc == GAP_OK && !device_ptrs && rows) {
        rc = dK.ensure(sizeof(double) * (size_t)rows * Mt);
        if (rc == GAP_OK) rc = ds.ensure(sizeof(double) * (size_t)rows);
        if (rc == GAP_OK)
            rc = gap_cuda_status(cudaMemcpyAsync(dK.p, knm, sizeof(double) * (size_t)rows * Mt, cudaMemcpyHostToDevice, st),
                                 "copy K_NM");
        if (rc == GAP_OK)
            rc = gap_cuda_status(cudaMemcpyAsync(ds.p, sigma, sizeof(double) * (size_t)rows, cudaMemcpyHostToDevice, st),
                                 "copy sigma");
        K = dK.as<double>();
        Sg = ds.as<double>();
    }
    if (rc == GAP_OK) rc = da.ensure(sizeof(double) * (size_t)Mt);
    if (rc == GAP_OK) rc = m->post_kinv.ensure(sizeof(double) * (size_t)Mt * Mt);
    if (rc == GAP_OK) rc = m->post_rinv.ensure(sizeof(double) * (size_t)Mt * Mt);
    if (rc == GAP_OK) rc = solve_points(m, Mt, st);
    if (rc == GAP_OK) {
        SolveInputs in{rows, Mt, K, dy.as<double>(), Sg, m->solve_X.as<double>(), m->solve_blk.as<int>(),
                       m->soap->Dg, m->delta, jitter, m->zeta};
        rc = gap_posterior_dev(in, m->post_kinv.as<double>(), m->post_rinv.as<double>(), da.as<double>(), m->solve_ws,
                               st);
    }
    if (rc == GAP_OK) rc = gap_cuda_status(cudaStreamSynchronize(st), "posterior");
    cleanup();
    m->has_post = rc == GAP_OK;
    return rc;
    GAP_API_END
}

extern "C" gap_status gap_predict_variance(gap_model *m, const gap_batch *b, double *var, void *stream)
{
    GAP_API_BEGIN
    if (!m) { gap_set_error("model is NULL"); return GAP_EINVAL; }
    GAP_TRY(check_batch(b));
    const int n = b->n_atoms;
    if (n > 0 && !var) { gap_set_error("var is NULL"); return GAP_EINVAL; }
    std::lock_guard<std::mutex> lk(m->mu);
    if (!m->has_post) {
        gap_set_error("no posterior factors: call gap_model_set_posterior first");
        return GAP_EINVAL;
    }
    if (n == 0) return GAP_OK;
    DeviceGuard dg(m->soap->device);
    cudaStream_t st = (cudaStream_t)stream;
    Workspace &w = m->ws;
    const int D = m->soap->Dg;
    int Mt = 0;
    for (auto &g : m->gp) Mt += g.M;
    const int *spec;
    GAP_TRY(run_descriptor<double>(m->soap, w, b, &spec, st));
    std::vector<int> counts;
    GAP_TRY(gp_rows_all(m, w, n, spec, counts, st));
    double *dvar = var;
    if (!b->device) {
        GAP_TRY(m->var_out.ensure(sizeof(double) * (size_t)n));
        dvar = m->var_out.as<double>();
    }
    // atoms of no GP (species without sparse points) have no local energy: 0
    GAP_TRY_CUDA(cudaMemsetAsync(dvar, 0, sizeof(double) * (size_t)n, st));
    const double d2 = m->delta * m->delta;
    constexpr int kChunk = 4096;
    int off = 0;
    for (int s = 0; s < m->n_gp; off += m->gp[s].M, ++s) {
        const GPData &g = m->gp[s];
        const int Ms = g.M, Rs = counts[s];
        if (Ms == 0 || Rs == 0) continue;
        const int ncolw = Mt - off;
        const int ch = Rs < kChunk ? Rs : kChunk;
        GAP_TRY(m->var_P.ensure(sizeof(double) * ((size_t)ch * D + ch)));
        GAP_TRY(m->var_Q.ensure(sizeof(double) * (size_t)ch * Ms));
        GAP_TRY(m->var_V.ensure(sizeof(double) * (size_t)ch * Ms));
        GAP_TRY(m->var_W.ensure(sizeof(double) * (size_t)ch * ncolw));
        double *P = m->var_P.as<double>(), *pn2 = P + (size_t)ch * D;
        double *Q = m->var_Q.as<double>(), *V = m->var_V.as<double>(), *Wm = m->var_W.as<double>();
        const int *grow = w.rows.as<int>() + (size_t)s * n;
        const double *kinv = m->post_kinv.as<double>() + off + (size_t)off * Mt;
        const double *rinv = m->post_rinv.as<double>() + off + (size_t)off * Mt;
        for (int c0 = 0; c0 < Rs; c0 += kChunk) {
            const int nr = Rs - c0 < kChunk ? Rs - c0 : kChunk;
            gap_count_launch();
            k_var_gather<<<(nr + 7) / 8, 256, 0, st>>>(gp_phat<double>(m->soap, w), D, grow + c0, nr, P, pn2);
            GAP_TRY_CUDA(cudaGetLastError());
            // q = P X^T, k = delta^2 q^zeta
            const CrtVMat Pv{P, D, nullptr, nr, nullptr, 0, nr, D};
            const CrtVMat Xv{g.X64.as<double>(), D, nullptr, Ms, nullptr, 0, Ms, D};
            GAP_TRY(gap_f64_product(m->solve_ws, Pv, false, Xv, false, false, Q, Ms, st));
            gap_count_launch();
            k_var_kernel<<<(unsigned)(((long)nr * Ms + 255) / 256), 256, 0, st>>>(Q, (long)nr * Ms, d2, m->zeta);
            GAP_TRY_CUDA(cudaGetLastError());
            // V = k U^-1 (this GP's block), W = k R^-1 (this GP's rows, columns >= off)
            const CrtVMat Kv{Q, Ms, nullptr, nr, nullptr, 0, nr, Ms};
            const CrtVMat Uv{kinv, Mt, nullptr, Ms, nullptr, 0, Ms, Ms};
            const CrtVMat Rv{rinv, Mt, nullptr, ncolw, nullptr, 0, ncolw, Ms};
            GAP_TRY(gap_f64_product(m->solve_ws, Kv, false, Uv, false, true, V, Ms, st));
            GAP_TRY(gap_f64_product(m->solve_ws, Kv, false, Rv, false, true, Wm, ncolw, st));
            gap_count_launch();
            k_var_finish<<<(nr + 7) / 8, 256, 0, st>>>(V, Ms, Wm, ncolw, nr, pn2, d2, m->zeta, grow + c0, dvar);
            GAP_TRY_CUDA(cudaGetLastError());
        }
    }
    if (!b->device) {
        GAP_TRY_CUDA(cudaMemcpyAsync(var, dvar, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
        GAP_TRY_CUDA(cudaStreamSynchronize(st));
    }
    return GAP_OK;
    GAP_API_END
}

// ------------------------------------------------------------ test hooks
extern "C" gap_status gap_test_bf16_gemm(int nsplit, int rows, int cols, int K, const float *A, const float *B,
                                         float *C)
{
    GAP_API_BEGIN
    if ((nsplit != 2 && nsplit != 3) || rows <= 0 || cols <= 0 || K <= 0 || K % 16 || !A || !B || !C) {
        gap_set_error("bad arguments");
        return GAP_EINVAL;
    }
    std::vector<uint16_t> ah((size_t)rows * K), am((size_t)rows * K), al((size_t)rows * K), bh((size_t)cols * K),
        bm((size_t)cols * K), bl((size_t)cols * K);
    auto split = [&](const float *x, size_t n, std::vector<uint16_t> &h, std::vector<uint16_t> &mm,
                     std::vector<uint16_t> &l) {
        for (size_t k = 0; k < n; ++k) {
            h[k] = bf16_rne(x[k]);
            float rest = x[k] - bf16_to_float(h[k]);
            if (nsplit == 3) {
                mm[k] = bf16_rne(rest);
                rest -= bf16_to_float(mm[k]);
            }
            l[k] = bf16_rne(rest);
        }
    };
    split(A, ah.size(), ah, am, al);
    split(B, bh.size(), bh, bm, bl);
    DBuf dah, dam, dal, dbh, dbm, dbl, dc, derr;
    auto cleanup = [&]() {
        dah.release(); dam.release(); dal.release(); dbh.release(); dbm.release(); dbl.release(); dc.release();
        derr.release();
    };
    gap_status st = upload(dah, ah);
    if (st == GAP_OK) st = upload(dam, am);
    if (st == GAP_OK) st = upload(dal, al);
    if (st == GAP_OK) st = upload(dbh, bh);
    if (st == GAP_OK) st = upload(dbm, bm);
    if (st == GAP_OK) st = upload(dbl, bl);
    if (st == GAP_OK) st = dc.ensure(sizeof(float) * (size_t)rows * cols);
    if (st == GAP_OK) st = derr.ensure(sizeof(int) * 4);
    if (st == GAP_OK) st = gap_cuda_status(cudaMemset(derr.p, 0, sizeof(int) * 4), "cudaMemset");
    if (st == GAP_OK) {
        TcOperands op{dah.as<__nv_bfloat16>(), dal.as<__nv_bfloat16>(), dbh.as<__nv_bfloat16>(),
                      dbl.as<__nv_bfloat16>(), rows, cols, K, K, K, nsplit, dam.as<__nv_bfloat16>(),
                      dbm.as<__nv_bfloat16>()};
        TcEpilogue ep{};
        ep.C = dc.as<float>();
        ep.ldc = cols;
        st = gap_tc_gemm(op, ep, EPI_STORE, derr.as<int>(), 0);
    }
    if (st == GAP_OK) st = gap_cuda_status(cudaDeviceSynchronize(), "tensor-core GEMM");
    int e = 0;
    if (st == GAP_OK) st = gap_cuda_status(cudaMemcpy(&e, derr.p, sizeof(int), cudaMemcpyDeviceToHost), "copy");
    if (st == GAP_OK && e) {
        gap_set_error("tensor-core GEMM wait expired (code " + std::to_string(e) + ")");
        st = GAP_ETIMEOUT;
    }
    if (st == GAP_OK)
        st = gap_cuda_status(cudaMemcpy(C, dc.p, sizeof(float) * (size_t)rows * cols, cudaMemcpyDeviceToHost), "copy");
    cleanup();
    return st;
    GAP_API_END
}

// The bounded-wait path of the tcgen05 GEMM: one 128 x 256 x 64 tile whose
// producer issues no copies (so no MMA is issued either) and whose waits
// give up after wait_ns; every role's wait runs out with nothing in flight,
// the CTA still frees its TMEM, and the call reports GAP_ETIMEOUT.
extern "C" gap_status gap_test_tc_timeout(unsigned long long wait_ns, int *code)
{
    GAP_API_BEGIN
    if (wait_ns == 0 || wait_ns > 1000000000ull || !code) {
        gap_set_error("wait_ns must be in 1..1e9 and code non-NULL");
        return GAP_EINVAL;
    }
    const int rows = 128, cols = 256, K = 64;
    DBuf da, db, dc, derr;
    auto cleanup = [&]() { da.release(); db.release(); dc.release(); derr.release(); };
    gap_status st = da.ensure(2 * (size_t)rows * K);
    if (st == GAP_OK) st = db.ensure(2 * (size_t)cols * K);
    if (st == GAP_OK) st = dc.ensure(sizeof(float) * (size_t)rows * cols);
    if (st == GAP_OK) st = derr.ensure(sizeof(int) * 4);
    if (st == GAP_OK) st = gap_cuda_status(cudaMemset(da.p, 0, 2 * (size_t)rows * K), "cudaMemset");
    if (st == GAP_OK) st = gap_cuda_status(cudaMemset(db.p, 0, 2 * (size_t)cols * K), "cudaMemset");
    if (st == GAP_OK) st = gap_cuda_status(cudaMemset(derr.p, 0, sizeof(int) * 4), "cudaMemset");
    if (st == GAP_OK) {
        TcOperands op{da.as<__nv_bfloat16>(), da.as<__nv_bfloat16>(), db.as<__nv_bfloat16>(), db.as<__nv_bfloat16>(),
                      rows, cols, K, K, K, 2, nullptr, nullptr};
        TcEpilogue ep{};
        ep.C = dc.as<float>();
        ep.ldc = cols;
        ep.wait_ns = wait_ns;
        ep.test_stall = 1;
        st = gap_tc_gemm(op, ep, EPI_STORE, derr.as<int>(), 0);
    }
    if (st == GAP_OK) st = gap_cuda_status(cudaDeviceSynchronize(), "tensor-core GEMM");
    int e = 0;
    if (st == GAP_OK) st = gap_cuda_status(cudaMemcpy(&e, derr.p, sizeof(int), cudaMemcpyDeviceToHost), "copy");
    *code = e;
    if (st == GAP_OK && e) {
        gap_set_error("tensor-core GEMM wait expired (code " + std::to_string(e) + ")");
        st = GAP_ETIMEOUT;
    }
    cleanup();
    return st;
    GAP_API_END
}

// C = A B^T through the modular FP64 tensor-core product: A [rows][K],
// B [cols][K], C [rows][cols], host row-major FP64.
extern "C" gap_status gap_test_f64_gemm(int rows, int cols, int K, const double *A, const double *B, int b_lower,
                                        double *C)
{
    GAP_API_BEGIN
    const int T = gap_crt_moduli(K);
    if (rows <= 0 || cols <= 0 || K <= 0 || !A || !B || !C || T == 0) {
        gap_set_error("bad arguments");
        return GAP_EINVAL;
    }
    const long kpad = gap_crt_kpad(K), ldo = ((long)cols + 255) / 256 * 256;
    std::vector<double> ha(A, A + (size_t)rows * K), hb(B, B + (size_t)cols * K);
    DBuf da, db, ra, rb, ea, eb, out, dc, derr;
    gap_status st = upload(da, ha);
    if (st == GAP_OK) st = upload(db, hb);
    if (st == GAP_OK) st = ra.ensure(2 * (size_t)T * rows * kpad);
    if (st == GAP_OK) st = rb.ensure(2 * (size_t)T * cols * kpad);
    if (st == GAP_OK) st = ea.ensure(sizeof(int) * rows);
    if (st == GAP_OK) st = eb.ensure(sizeof(int) * cols);
    if (st == GAP_OK) st = out.ensure((size_t)T * rows * ldo);
    if (st == GAP_OK) st = dc.ensure(sizeof(double) * (size_t)rows * cols);
    if (st == GAP_OK) st = derr.ensure(sizeof(int) * 4);
    if (st == GAP_OK) st = gap_cuda_status(cudaMemset(derr.p, 0, sizeof(int) * 4), "cudaMemset");
    CrtVMat VA{da.as<double>(), K, nullptr, rows, nullptr, 0, rows, K};
    CrtVMat VB{db.as<double>(), K, nullptr, cols, nullptr, 0, cols, K};
    if (st == GAP_OK) st = gap_crt_prep_rows(VA, T, kpad, ra.as<__nv_bfloat16>(), ea.as<int>(), 0);
    if (st == GAP_OK) st = gap_crt_prep_rows(VB, T, kpad, rb.as<__nv_bfloat16>(), eb.as<int>(), 0);
    if (st == GAP_OK)
        st = gap_crt_gemm(ra.as<__nv_bfloat16>(), rows, rb.as<__nv_bfloat16>(), cols, kpad, T, false, b_lower != 0,
                          out.as<unsigned char>(), ldo, derr.as<int>(), 0);
    if (st == GAP_OK)
        st = gap_crt_combine(out.as<unsigned char>(), ldo, rows, cols, T, ea.as<int>(), eb.as<int>(), false,
                             dc.as<double>(), cols, 0);
    if (st == GAP_OK) st = gap_cuda_status(cudaDeviceSynchronize(), "modular GEMM");
    int e = 0;
    if (st == GAP_OK) st = gap_cuda_status(cudaMemcpy(&e, derr.p, sizeof(int), cudaMemcpyDeviceToHost), "copy");
    if (st == GAP_OK && e) {
        gap_set_error("modular GEMM wait expired (code " + std::to_string(e) + ")");
        st = GAP_ETIMEOUT;
    }
    if (st == GAP_OK)
        st = gap_cuda_status(cudaMemcpy(C, dc.p, sizeof(double) * (size_t)rows * cols, cudaMemcpyDeviceToHost), "copy");
    return st;
    GAP_API_END
}

// G = Y^T Y through the symmetric modular product: Y [m][n], G [n][n], host.
extern "C" gap_status gap_test_f64_gram(long m, int n, const double *Y, double *G)
{
    GAP_API_BEGIN
    const int T = gap_crt_moduli(m);
    if (m <= 0 || n <= 0 || !Y || !G || T == 0) {
        gap_set_error("bad arguments");
        return GAP_EINVAL;
    }
    const long kpad = gap_crt_kpad(m), ldo = ((long)n + 255) / 256 * 256;
    std::vector<double> hy(Y, Y + (size_t)m * n);
    DBuf dy, res, e, out, dg, derr;
    gap_status st = upload(dy, hy);
    if (st == GAP_OK) st = res.ensure(2 * (size_t)T * n * kpad);
    if (st == GAP_OK) st = e.ensure(sizeof(int) * n);
    if (st == GAP_OK) st = out.ensure((size_t)T * n * ldo);
    if (st == GAP_OK) st = dg.ensure(sizeof(double) * (size_t)n * n);
    if (st == GAP_OK) st = derr.ensure(sizeof(int) * 4);
    if (st == GAP_OK) st = gap_cuda_status(cudaMemset(derr.p, 0, sizeof(int) * 4), "cudaMemset");
    CrtVMat V{dy.as<double>(), n, nullptr, m, nullptr, 0, m, n};
    if (st == GAP_OK) st = gap_crt_prep_cols(V, T, kpad, res.as<__nv_bfloat16>(), e.as<int>(), 0);
    if (st == GAP_OK)
        st = gap_crt_gemm(res.as<__nv_bfloat16>(), n, res.as<__nv_bfloat16>(), n, kpad, T, true, false,
                          out.as<unsigned char>(), ldo, derr.as<int>(), 0);
    if (st == GAP_OK)
        st = gap_crt_combine(out.as<unsigned char>(), ldo, n, n, T, e.as<int>(), e.as<int>(), true, dg.as<double>(), n,
                             0);
    if (st == GAP_OK) st = gap_cuda_status(cudaDeviceSynchronize(), "modular Gram");
    int ee = 0;
    if (st == GAP_OK) st = gap_cuda_status(cudaMemcpy(&ee, derr.p, sizeof(int), cudaMemcpyDeviceToHost), "copy");
    if (st == GAP_OK && ee) {
        gap_set_error("modular GEMM wait expired (code " + std::to_string(ee) + ")");
        st = GAP_ETIMEOUT;
    }
    if (st == GAP_OK)
        st = gap_cuda_status(cudaMemcpy(G, dg.p, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost), "copy");
    return st;
    GAP_API_END
}

// Exact congruence of the CholeskyQR solve (all host arrays): V = [Y | b]
// (Y row-major m x n, b m entries, m may be 0), G = V^T V + [Kt 0; 0 0] on
// V's fixed-point grid (Kt column-major n x n or NULL), W column-major upper
// triangular.  Gout = W~^T G W~ (leading n x n block, column-major),
// c = W~^T V^T b, Wt = W~ (W rounded to 53 bits per scaled column).
extern "C" gap_status gap_test_congruence(long m, int n, const double *Y, const double *b, const double *Kt,
                                          const double *W, double *Gout, double *c, double *Wt)
{
    GAP_API_BEGIN
    if (m < 0 || n <= 0 || n > 16384 || (m > 0 && (!Y || !b)) || !W || !Gout || !c || !Wt) {
        gap_set_error("bad arguments");
        return GAP_EINVAL;
    }
    const long mr = m > 0 ? m : 1;
    const int n_ext = n + 1;
    const int T1 = gap_crt_moduli(mr), T2 = gap_crt_moduli_wide(gap_crt_congruence_bits(mr, n_ext));
    if (T1 == 0 || T2 == 0) {
        gap_set_error("congruence too large for the moduli");
        return GAP_EUNSUPPORTED;
    }
    const long kpm = gap_crt_kpad(mr), kp2 = ((long)n_ext + 255) / 256 * 256;
    const size_t plane = (size_t)T2 * n_ext * kp2 * 2;
    std::vector<double> hy(Y ? Y : W, Y ? Y + (size_t)m * n : W + 1), hb(b ? b : W, b ? b + m : W + 1);
    std::vector<double> hk(Kt ? Kt : W, Kt ? Kt + (size_t)n * n : W + 1), hw(W, W + (size_t)n * n);
    DBuf dy, db, dk, dw, res1, e, out1, g1, ra, rh, go, f, dg, dc, derr;
    gap_status st = upload(dy, hy);
    if (st == GAP_OK) st = upload(db, hb);
    if (st == GAP_OK) st = upload(dk, hk);
    if (st == GAP_OK) st = upload(dw, hw);
    if (st == GAP_OK) st = res1.ensure(2 * (size_t)T1 * n_ext * kpm);
    if (st == GAP_OK) st = e.ensure(sizeof(int) * n_ext);
    if (st == GAP_OK) st = out1.ensure((size_t)T1 * n_ext * kp2);
    if (st == GAP_OK) st = g1.ensure(plane);
    if (st == GAP_OK) st = ra.ensure(plane);
    if (st == GAP_OK) st = rh.ensure(plane);
    if (st == GAP_OK) st = go.ensure(plane);
    if (st == GAP_OK) st = f.ensure(sizeof(int) * n_ext);
    if (st == GAP_OK) st = dg.ensure(sizeof(double) * (size_t)n * n);
    if (st == GAP_OK) st = dc.ensure(sizeof(double) * (size_t)n);
    if (st == GAP_OK) st = derr.ensure(sizeof(int) * 4);
    if (st == GAP_OK) st = gap_cuda_status(cudaMemset(derr.p, 0, sizeof(int) * 4), "cudaMemset");
    const double *kt = Kt ? dk.as<double>() : nullptr;
    CrtVMat V{dy.as<double>(), n, nullptr, m, nullptr, 0, m, n_ext, db.as<double>()};
    if (st == GAP_OK) st = gap_crt_prep_cols(V, T1, kpm, res1.as<__nv_bfloat16>(), e.as<int>(), 0, kt, n + 1, kt ? n : 0);
    if (st == GAP_OK)
        st = gap_crt_gemm(res1.as<__nv_bfloat16>(), n_ext, res1.as<__nv_bfloat16>(), n_ext, kpm, T1, true, false,
                          out1.p, kp2, derr.as<int>(), 0);
    if (st == GAP_OK)
        st = gap_crt_exact_gram(out1.as<unsigned char>(), kp2, T1, n, e.as<int>(), kt, T2, kp2,
                                g1.as<__nv_bfloat16>(), dg.as<double>(), derr.as<int>(), 0);
    if (st == GAP_OK)
        st = gap_crt_prep_congruence(dw.as<double>(), n, e.as<int>(), T2, kp2, ra.as<__nv_bfloat16>(), f.as<int>(),
                                     dw.as<double>(), 0);
    if (st == GAP_OK)
        st = gap_crt_gemm(ra.as<__nv_bfloat16>(), n_ext, g1.as<__nv_bfloat16>(), n_ext, kp2, T2, false, false, rh.p,
                          kp2, derr.as<int>(), 0, true, true);
    if (st == GAP_OK)
        st = gap_crt_gemm(ra.as<__nv_bfloat16>(), n_ext, rh.as<__nv_bfloat16>(), n_ext, kp2, T2, true, false, go.p,
                          kp2, derr.as<int>(), 0, true, true);
    if (st == GAP_OK)
        st = gap_crt_combine_congruence(go.as<__nv_bfloat16>(), kp2, n, T2, f.as<int>(), dg.as<double>(),
                                        dc.as<double>(), 0);
    if (st == GAP_OK) st = gap_cuda_status(cudaDeviceSynchronize(), "congruence");
    int ee = 0;
    if (st == GAP_OK) st = gap_cuda_status(cudaMemcpy(&ee, derr.p, sizeof(int), cudaMemcpyDeviceToHost), "copy");
    if (st == GAP_OK && ee) {
        gap_set_error("congruence: error flags " + std::to_string(ee));
        st = (ee & 16) ? GAP_EINVAL : GAP_ETIMEOUT;
    }
    if (st == GAP_OK)
        st = gap_cuda_status(cudaMemcpy(Gout, dg.p, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost), "copy");
    if (st == GAP_OK) st = gap_cuda_status(cudaMemcpy(c, dc.p, sizeof(double) * n, cudaMemcpyDeviceToHost), "copy");
    if (st == GAP_OK)
        st = gap_cuda_status(cudaMemcpy(Wt, dw.p, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost), "copy");
    return st;
    GAP_API_END
}

// The block-product crossover of the recursive factorisation, measured as
// gap_chol_inv_dev measures it on its first call: ms[2][8] host (times of the
// FP64 kernel, then of the modular product, for sizes 32, 64, ...), sizes the
// number of sizes timed, threshold the multiply-add count chosen.
extern "C" gap_status gap_test_product_crossover(int n, const double *G, float *ms, int *sizes, long *threshold)
{
    GAP_API_BEGIN
    if (n < 32 || n > 16384 || !G || !ms || !sizes || !threshold) {
        gap_set_error("bad arguments");
        return GAP_EINVAL;
    }
    std::vector<double> hg(G, G + (size_t)n * n);
    DBuf dg;
    SolveWork w;
    gap_status st = upload(dg, hg);
    if (st == GAP_OK) st = w.handles(0);
    if (st == GAP_OK) st = gap_tune_small_product(w, n, dg.as<double>(), 0);
    if (st == GAP_OK) st = gap_cuda_status(cudaDeviceSynchronize(), "crossover");
    if (st == GAP_OK) {
        for (int p = 0; p < 2; ++p)
            for (int k = 0; k < 8; ++k) ms[p * 8 + k] = w.tune_ms[p][k];
        *sizes = w.tune_sizes;
        *threshold = w.small_product;
    }
    cudaDeviceSynchronize();
    w.release();
    return st;
    GAP_API_END
}

// Recursive Cholesky factor and inverse of the CholeskyQR solve: G host
// [n][n] SPD (column-major = row-major), R and X host [n][n] column-major.
extern "C" gap_status gap_test_chol_inv(int n, const double *G, double *R, double *X)
{
    GAP_API_BEGIN
    if (n <= 0 || n > 16384 || !G || !R || !X) {
        gap_set_error("bad arguments");
        return GAP_EINVAL;
    }
    std::vector<double> hg(G, G + (size_t)n * n);
    DBuf dg, dr, dx;
    SolveWork w;
    gap_status st = upload(dg, hg);
    if (st == GAP_OK) st = dr.ensure(sizeof(double) * (size_t)n * n);
    if (st == GAP_OK) st = dx.ensure(sizeof(double) * (size_t)n * n);
    if (st == GAP_OK) st = gap_chol_inv_dev(w, n, dg.as<double>(), dr.as<double>(), dx.as<double>(), 0);
    if (st == GAP_OK)
        st = gap_cuda_status(cudaMemcpy(R, dr.p, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost), "copy");
    if (st == GAP_OK)
        st = gap_cuda_status(cudaMemcpy(X, dx.p, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost), "copy");
    cudaDeviceSynchronize();
    w.release();
    return st;
    GAP_API_END
}

// ------------------------------------------------- allocation-free variant
// For callers that cannot allocate device memory while they run (an MD
// engine whose host program owns every device buffer and forbids allocation
// inside its force callback, or a latency-critical loop that must not pay
// the implicit device synchronisation of cudaMalloc/cudaFree), the local
// energies and their gradients with respect to the descriptor are also
// available from an entry point whose only scratch (the matrix W and the
// per-tile partial energies of the FP64 contraction, the row list) lives in
// this file-scope device array.  Every GPU that loads the library holds it
// until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GAP_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[256];

__global__ void k_noalloc_rows(int n, int *__restrict__ rows, int *__restrict__ count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rows[i] = i;
    if (i == 0) *count = n;
}

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

extern "C" gap_status gap_gp_energy_noalloc(const gap_model *m, int gp, int n_rows, const double *p_hat, double *eps,
                                            double *grad, void *stream)
{
    GAP_API_BEGIN
    if (!m) { gap_set_error("model is NULL"); return GAP_EINVAL; }
    if (gp < 0 || gp >= m->n_gp) { gap_set_error("gp must be in 0..n_gp-1"); return GAP_EINVAL; }
    if (n_rows < 0) { gap_set_error("n_rows must be non-negative"); return GAP_EINVAL; }
    if (n_rows == 0) return GAP_OK;
    if (!p_hat || !eps || !grad) { gap_set_error("p_hat, eps and grad must be device pointers"); return GAP_EINVAL; }
    const GPData &g = m->gp[gp];
    const int D = m->soap->Dg, M = g.M;
    const size_t n_tiles = (size_t)gap_contract_simt_tiles(M);  // the kernel's own partial-energy stride
    const size_t need = align256(sizeof(int)) + align256(sizeof(int) * (size_t)n_rows) +
                        align256(sizeof(double) * (size_t)n_rows * n_tiles) +
                        align256(sizeof(double) * (size_t)n_rows * (M > 0 ? M : 1));
    if (need > GAP_NOALLOC_SCRATCH_BYTES) {
        gap_set_error("gap_gp_energy_noalloc: n_rows = " + std::to_string(n_rows) + " with M = " +
                      std::to_string(M) + " needs " + std::to_string(need) + " bytes of scratch; the static limit is " +
                      std::to_string((size_t)GAP_NOALLOC_SCRATCH_BYTES) + " bytes");
        return GAP_EINVAL;
    }
    DeviceGuard dg(m->soap->device);
    int dev = 0;
    GAP_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) { gap_set_error("device index out of range"); return GAP_EINVAL; }
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return gap_cuda_status(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            g_noalloc_ptr[dev] = p;
        }
        base = g_noalloc_ptr[dev];
    }
    unsigned char *c = static_cast<unsigned char *>(base);
    int *count = reinterpret_cast<int *>(c);
    c += align256(sizeof(int));
    int *rows = reinterpret_cast<int *>(c);
    c += align256(sizeof(int) * (size_t)n_rows);
    double *eps_part = reinterpret_cast<double *>(c);
    c += align256(sizeof(double) * (size_t)n_rows * n_tiles);
    double *W = reinterpret_cast<double *>(c);
    cudaStream_t st = (cudaStream_t)stream;
    if (M == 0) {
        GAP_TRY_CUDA(cudaMemsetAsync(eps, 0, sizeof(double) * (size_t)n_rows, st));
        GAP_TRY_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)n_rows * D, st));
        return GAP_OK;
    }
    gap_count_launch();
    k_noalloc_rows<<<(n_rows + 255) / 256, 256, 0, st>>>(n_rows, rows, count);
    GAP_TRY_CUDA(cudaGetLastError());
    return gap_contract_simt_fixed(p_hat, D, D, rows, count, n_rows, g.X64.as<double>(), g.a64.as<double>(), M,
                                   m->delta, m->zeta, W, eps_part, grad, eps, st);
    GAP_API_END
}
