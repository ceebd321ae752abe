// mad_api.cu -- the C ABI (include/mad.h) and the per-length schedule of the
// exact variable-length matrix profile (Algorithm 1 VALMOD driving Algorithms
// 3, 4 and 10, with the discord table of Algorithm 7).
//
// Schedule of one profile over [lmin, lmax] (per series):
//   lmin : window statistics; every row is recomputed: seed rows, an
//          interleaved-maxima pass for a first per-row threshold, the
//          candidate pass, selection of each row's top-p entries (repeated
//          for rows whose candidate list overflowed), flat rows, discords.
//   l > lmin : one Welford step of the statistics; extension of the stored
//          entries with the bound test; the same recompute steps for the rows
//          the bound did not certify; discords.
// Device memory is owned by the context; PyTorch (or any caller) only
// supplies the series and the stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "mad.h"
#include "kernels.cuh"

using namespace mad;

namespace {

thread_local std::string g_create_err;

// Tries of the band kernel's wavefront waits (mad_debug_wavefront_wait_limit;
// negative: the kernel's own limit).
std::atomic<int> g_wave_limit{-1};
// mad_debug_audit_error_bounds
std::atomic<int> g_audit{0};
// mad_set_graphs: capture and replay repeated profiles (default on)
std::atomic<int> g_graphs{1};
// mad_debug_tc_tma: the tensor-core path's column tiles by TMA (default off:
// measured slower inside the profile pipeline, see mad.h)
std::atomic<int> g_tc_tma{0};

// What a profile's workspace depends on: while a series is profiled again
// with the same key, its device buffers are reused as they are (no
// cudaMalloc / cudaFree) and the whole per-length launch sequence is replayed
// from a CUDA graph.
struct WsKey {
    int tsize = 0, lmin = 0, lmax = 0, p = 0, m_max = 0, k_max = 0, mode = 0, band_form = 0, keep = 0,
        observe = 0, num = 0, den = 0, audit = 0, wave_limit = 0, tc = 0, rpl = 0, limf = 0, tma = 0;
    bool operator==(const WsKey &o) const { return std::memcmp(this, &o, sizeof(WsKey)) == 0; }
};

struct Series {
    int64_t n = 0;
    double *x = nullptr;
    bool own_x = true;
    // result of the last profile
    bool profiled = false;
    int lmin = 0, lmax = 0, p = 0, m_max = 1, k_max = 10;
    int64_t n0 = 0;
    // workspace: device buffers in allocation order; while `reuse` is set,
    // allocations are handed out again from the list (sizes checked)
    std::vector<void *> allocs;
    std::vector<size_t> alloc_bytes;
    size_t cursor = 0;
    bool reuse = false;
    bool ws_valid = false;
    WsKey key{};
    // side streams and events of the per-length pipeline, kept across profiles
    cudaStream_t prep = nullptr, disc = nullptr, cap = nullptr;
    cudaEvent_t sev[10] = {};
    std::vector<cudaEvent_t> tev;           // timing events of the band kernel (pairs)
    std::vector<int> tev_li;                // length index of each pair
    std::vector<unsigned long long> host_launch;
    cudaGraphExec_t exec = nullptr;         // the captured profile, replayed while the key holds
    // read-back of the last profile
    unsigned long long *dstats = nullptr;
    int32_t *wait_err = nullptr;
    int nstat = 0;
    // scratch of the read-outs (grown, never shrunk)
    void *rscratch = nullptr;
    size_t rscratch_bytes = 0;
    // launch parameters of the next profile (chosen by the autotuner)
    int rpl = 0, limf = 0;
    bool graph_last = false;                // the last profile ran as a graph
    // pinned host buffer the error word and the counters are read back into
    unsigned long long *hbuf = nullptr;
    size_t hbuf_words = 0;
    Valmp vm{};
    DiscTable tab{};
    double *keep_nnd = nullptr;
    int obs_len = 0;                 // observation length of the last profile (0: none)
    double *obs_gap = nullptr, *obs_tlb = nullptr;
    int32_t *keep_nnj = nullptr;
    std::vector<mad_length_stats> stats;
    // TMA descriptor of the tensor-core path's column tiles (a CUtensorMap)
    alignas(64) unsigned char bmap[128] = {};
    bool bmap_ok = false;
};

}  // namespace

struct mad_ctx {
    mad_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    std::vector<Series> series;
    std::string err;
};

namespace {

struct Fail {
    mad_status st;
};

// (the batch path profiles series from several host threads)
std::mutex g_err_mu;

void set_err(mad_ctx *c, const std::string &m)
{
    if (c) {
        std::lock_guard<std::mutex> lock(g_err_mu);
        c->err = m;
    } else {
        g_create_err = m;
    }
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            set_err(ctx, std::string(#call) + ": " + cudaGetErrorString(e_));                      \
            throw Fail{e_ == cudaErrorMemoryAllocation ? MAD_ENOMEM : MAD_ECUDA};                  \
        }                                                                                          \
    } while (0)

#define REQUIRE_RET(cond, msg)                                                                     \
    do {                                                                                           \
        if (!(cond)) {                                                                             \
            set_err(ctx, msg);                                                                     \
            return MAD_EINVAL;                                                                     \
        }                                                                                          \
    } while (0)

#define REQUIRE(cond, msg)                                                                         \
    do {                                                                                           \
        if (!(cond)) {                                                                             \
            set_err(ctx, msg);                                                                     \
            throw Fail{MAD_EINVAL};                                                                \
        }                                                                                          \
    } while (0)

template <typename P>
P *dalloc(mad_ctx *ctx, Series &s, size_t count)
{
    const size_t bytes = count * sizeof(P) > 0 ? count * sizeof(P) : 1;
    if (s.reuse) {
        if (s.cursor >= s.allocs.size() || s.alloc_bytes[s.cursor] != bytes) {
            set_err(ctx, "workspace reuse out of step with its allocations");
            throw Fail{MAD_EINTERNAL};
        }
        return static_cast<P *>(s.allocs[s.cursor++]);
    }
    void *p = nullptr;
    CK(cudaMalloc(&p, bytes));
    s.allocs.push_back(p);
    s.alloc_bytes.push_back(bytes);
    return static_cast<P *>(p);
}

void free_profile(Series &s)
{
    if (s.exec) cudaGraphExecDestroy(s.exec);
    s.exec = nullptr;
    for (void *p : s.allocs) cudaFree(p);
    s.allocs.clear();
    s.alloc_bytes.clear();
    s.cursor = 0;
    s.reuse = false;
    s.ws_valid = false;
    s.dstats = nullptr;
    s.wait_err = nullptr;
    s.profiled = false;
    s.keep_nnd = nullptr;
    s.keep_nnj = nullptr;
    s.obs_len = 0;
    s.obs_gap = s.obs_tlb = nullptr;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Scratch of the read-outs: one device buffer per series, grown when a call
// needs more and kept (the read-outs then allocate nothing in steady state).
// Carve hands out 256-byte aligned pieces of it.
struct Carve {
    std::vector<size_t> sizes;
    size_t total() const
    {
        size_t t = 0;
        for (size_t b : sizes) t += (b + 255) / 256 * 256;
        return t;
    }
};
std::vector<void *> rscratch(mad_ctx *ctx, Series &s, const Carve &c, cudaStream_t st)
{
    const size_t need = c.total() > 0 ? c.total() : 256;
    if (need > s.rscratch_bytes) {
        if (s.rscratch) {
            CK(cudaStreamSynchronize(st));
            cudaFree(s.rscratch);
            s.rscratch = nullptr;
            s.rscratch_bytes = 0;
        }
        const size_t nb = need + need / 2;
        CK(cudaMalloc(&s.rscratch, nb));
        s.rscratch_bytes = nb;
    }
    std::vector<void *> out;
    size_t off = 0;
    for (size_t b : c.sizes) {
        out.push_back(static_cast<char *>(s.rscratch) + off);
        off += (b + 255) / 256 * 256;
    }
    return out;
}

mad_options defaults(const mad_options *o)
{
    mad_options r{};
    if (o) r = *o;
    if (r.excl_num == 0 && r.excl_den == 0) { r.excl_num = 1; r.excl_den = 4; }
    if (r.k_max == 0) r.k_max = 10;
    if (r.m_max == 0) r.m_max = 1;
    return r;
}

void check_options(mad_ctx *ctx, const mad_options &o)
{
    REQUIRE(o.excl_num >= 0 && o.excl_den >= 1, "exclusion zone needs excl_num >= 0 and excl_den >= 1");
    REQUIRE(o.precision == MAD_FP64 || o.precision == MAD_FP32 || o.precision == MAD_SPLIT_TC,
            "precision must be MAD_FP64, MAD_FP32 or MAD_SPLIT_TC");
    REQUIRE(o.k_max >= 1 && o.k_max <= KMAX, "k_max must be in [1, 64]");
    REQUIRE(o.m_max >= 1 && o.m_max <= MAXP, "m_max must be in [1, 64]");
    REQUIRE(o.mode >= 0 && o.mode <= 2, "mode must be 0 (exact rows), 1 (motif mode) or 2 (discord mode)");
    REQUIRE(o.mode != 1 || o.m_max == 1, "motif mode reports the motif of each length only: m_max must be 1");
    REQUIRE(o.band_form == 0 || o.band_form == 1, "band_form must be 0 or 1");
}

void init_ctx(mad_ctx *ctx, const mad_options *opt)
{
    ctx->opt = defaults(opt);
    check_options(ctx, ctx->opt);
    ctx->stream = static_cast<cudaStream_t>(ctx->opt.stream);
    CK(cudaGetDevice(&ctx->device));
    CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
}

// ------------------------------------------------------------- profile

// Error model of the band kernel's keys (see ErrModel): dq0 = u (2R + 4)
// for a chain of at most R + 1 steps (scaled per cell by the contrast
// factors), plus, on the FP64 path, the error of the FP64 seeds (a direct
// dot product at lmin, then one Welford step per length); and the distance
// tolerance that decides which reported entries are re-evaluated.
template <typename T>
struct Precision;
template <>
struct Precision<double> {
    static constexpr double u = 0x1p-53, rel_tol = 1e-9, abs_coef = 0.0;
    static double dq0(int R, int lmax) { return u * (2.0 * R + 4.0 + 4.0 * lmax + 64.0); }
};
template <>
struct Precision<float> {
    static constexpr double u = 0x1p-24, rel_tol = 0.0, abs_coef = 1e-4;
    static double dq0(int R, int) { return u * (2.0 * R + 4.0) + 0x1p-50; }
};

// Timed launches of the per-length pipeline (CUDA events recorded on the
// launching stream around each launch; in a captured profile the records are
// graph nodes of their own).
enum { TK_BAND = 0, TK_DIRECT = 1, TK_ROWS = 2 };

// Issue one profile over [lmin, lmax] on stream st: every kernel, copy and
// cross-stream dependency, and nothing that waits on the host, so that the
// same sequence can be captured into a CUDA graph. Buffers come from the
// series' workspace (reused while its key holds).
template <typename T>
void issue_profile(mad_ctx *ctx, Series &s, int lmin, int lmax, int p, cudaStream_t st, bool capture)
{
    const mad_options &o = ctx->opt;
    const int num = o.excl_num, den = o.excl_den;
    const int64_t n = s.n;
    s.lmin = lmin;
    s.lmax = lmax;
    s.p = p;
    s.m_max = o.m_max;
    s.k_max = o.k_max;
    const int64_t n0 = n - lmin + 1;
    s.n0 = n0;
    const int m_max = o.m_max, k_max = o.k_max;
    const int nL = lmax - lmin + 1;
    const int rpl = s.rpl;
    const int R = 32 * rpl * BAND_NW;
    const int nbins = band_nbins(p);
    // Seed-row spacing: the smallest power of two from one warp's rows (at
    // least 128) up to the band height whose seed rows (two copies in T and
    // the FP64 master) fit in 16 GB. Every chain of the band kernel then has
    // at most SP steps, which is what its error bound scales with; one seed
    // row per warp also removes the wavefront between the warps.
    // (The motif mode recomputes few rows per length, so there the seed
    // rows' per-length step would cost more than the tighter bound saves:
    // one seed row per band start.)
    int SP = R < 1024 ? R : 1024;
    for (int sp = 32 * rpl > 128 ? 32 * rpl : 128; o.mode != 1 && sp <= R; sp *= 2) {
        const double rows = (double)((n0 + sp - 1) / sp);
        const double bytes = rows * (double)(round_up(n0, R) + R + CH) * (2.0 * sizeof(T) + 8.0);
        if (bytes <= 16e9) {
            SP = sp;
            break;
        }
    }
    const int64_t K = (n0 + SP - 1) / SP;       // seed rows
    const int64_t KB = (n0 + R - 1) / R;        // bands
    const int64_t npad = round_up(n0, R) + R + CH;
    const int64_t spitch = round_up(n0, R) + R + CH;

    // ---- buffers
    int32_t *run = dalloc<int32_t>(ctx, s, n);
    double *mu[2] = {dalloc<double>(ctx, s, n0), dalloc<double>(ctx, s, n0)};
    double *m2[2] = {dalloc<double>(ctx, s, n0), dalloc<double>(ctx, s, n0)};
    // per-length inputs of the band kernel and the per-row kernels, double
    // buffered by length parity: length l+1's are prepared on a side stream
    // while length l's band kernel runs
    Col<T> *colb[2] = {dalloc<Col<T>>(ctx, s, npad), dalloc<Col<T>>(ctx, s, npad)};
    // Seed rows are computed for the K rows that exist; the buffers hold one
    // per SP rows of every band (the last band runs past n0), the extra rows
    // zero, so that every seeded warp's top-edge row is in bounds.
    const int64_t Kalloc = round_up(n0, R) / SP;
    T *seedb[2] = {dalloc<T>(ctx, s, Kalloc * spitch), dalloc<T>(ctx, s, Kalloc * spitch)};
    double *seedm = dalloc<double>(ctx, s, Kalloc * spitch);   // FP64 master of the seed rows
    if (!s.reuse && Kalloc > K) {
        const size_t tail = (size_t)(Kalloc - K) * spitch;
        CK(cudaMemsetAsync(seedb[0] + K * spitch, 0, tail * sizeof(T), st));
        CK(cudaMemsetAsync(seedb[1] + K * spitch, 0, tail * sizeof(T), st));
        CK(cudaMemsetAsync(seedm + K * spitch, 0, tail * sizeof(double), st));
    }
    T *thr = dalloc<T>(ctx, s, npad);
    RowState rs{dalloc<int32_t>(ctx, s, (size_t)p * n0), dalloc<double>(ctx, s, (size_t)p * n0),
                dalloc<double>(ctx, s, (size_t)p * n0), dalloc<double>(ctx, s, n0),
                dalloc<float>(ctx, s, (size_t)p * n0), dalloc<int32_t>(ctx, s, n0), dalloc<double>(ctx, s, n0),
                dalloc<int32_t>(ctx, s, n0)};
    // pruning observation at one length (options.observe_len)
    const bool observe = o.observe_len > lmin && o.observe_len <= lmax;
    s.obs_len = observe ? o.observe_len : 0;
    s.obs_gap = observe ? dalloc<double>(ctx, s, n0) : nullptr;
    s.obs_tlb = observe ? dalloc<double>(ctx, s, n0) : nullptr;
    float *kappab[2] = {dalloc<float>(ctx, s, n0), dalloc<float>(ctx, s, n0)};
    float *kmaxb[2] = {dalloc<float>(ctx, s, 1), dalloc<float>(ctx, s, 1)};
    double *m2blk = dalloc<double>(ctx, s, (n0 + 255) / 256);
    double *isdb[2] = {dalloc<double>(ctx, s, n0), dalloc<double>(ctx, s, n0)};
    float *xh = dalloc<float>(ctx, s, n), *xl = dalloc<float>(ctx, s, n);
    const int audit = g_audit.load() ? 1 : 0;
    const double dq0 = Precision<T>::dq0(SP, lmax);
    const ErrModel emb[2] = {
        {kappab[0], kmaxb[0], dq0, Precision<T>::rel_tol, Precision<T>::abs_coef, audit},
        {kappab[1], kmaxb[1], dq0, Precision<T>::rel_tol, Precision<T>::abs_coef, audit}};
    Valmp vm{dalloc<double>(ctx, s, n0), dalloc<double>(ctx, s, n0), dalloc<int32_t>(ctx, s, n0),
             dalloc<int32_t>(ctx, s, n0)};
    int *bins = dalloc<int>(ctx, s, (size_t)n0 * nbins);
    int *rowbest = dalloc<int>(ctx, s, (size_t)npad);   // band kernel: per-row threshold shared by units
    int32_t *bands = dalloc<int32_t>(ctx, s, KB);
    int32_t *counters = dalloc<int32_t>(ctx, s, 4);   // nbands, unit counter, overflow
    int32_t *krows = dalloc<int32_t>(ctx, s, K);
    // m-th best matches of the current length, double-buffered: the discord
    // tables of length l read one buffer on a side stream while length l+1
    // writes the other
    double *nndbuf[2] = {dalloc<double>(ctx, s, (size_t)m_max * n0), dalloc<double>(ctx, s, (size_t)m_max * n0)};
    int32_t *nnjbuf[2] = {dalloc<int32_t>(ctx, s, (size_t)m_max * n0), dalloc<int32_t>(ctx, s, (size_t)m_max * n0)};
    const int64_t nblk = (n0 + 255) / 256;
    double *bval = dalloc<double>(ctx, s, (size_t)m_max * nblk);
    int32_t *bidx = dalloc<int32_t>(ctx, s, (size_t)m_max * nblk);
    // per-length device counters: [0] rows left for a second pass, [1] certified,
    // [2] recomputed, [3] largest FP32-vs-FP64 correlation gap (bits),
    // [4] top-p insertions, [5] band units, [6] band cells
    // [10] motif mode: rows left undefined, [11] motif mode: full profile,
    // [12] largest observed error of a re-evaluated entry over its bound (bits)
    constexpr int NSTAT = 16;
    unsigned long long *dstats = dalloc<unsigned long long>(ctx, s, (size_t)nL * NSTAT);
    // motif mode: per-row bound of non-valid rows; per length the smallest
    // certified distance and non-valid bound (+inf until reduced)
    const bool motif_mode = o.mode == 1;
    const bool disc_mode = o.mode == 2;
    // discord mode: dkm_l, the non-valid list with its upper values, list positions
    double *dkm_d = disc_mode ? dalloc<double>(ctx, s, (size_t)k_max * m_max) : nullptr;
    int32_t *dkm_o = disc_mode ? dalloc<int32_t>(ctx, s, (size_t)k_max * m_max) : nullptr;
    int32_t *dkm_n = disc_mode ? dalloc<int32_t>(ctx, s, (size_t)k_max * m_max) : nullptr;
    double *dlub = disc_mode ? dalloc<double>(ctx, s, (size_t)n0 * m_max) : nullptr;
    int32_t *dkept = disc_mode ? dalloc<int32_t>(ctx, s, n0) : nullptr;
    int32_t *dO1 = disc_mode ? dalloc<int32_t>(ctx, s, (size_t)k_max * m_max) : nullptr;
    double *dcmin1 = disc_mode ? dalloc<double>(ctx, s, m_max) : nullptr;
    // entry / exit logs of the two passes (4 x n0) and the second pass's minima log
    int32_t *dlog = disc_mode ? dalloc<int32_t>(ctx, s, (size_t)6 * n0 + 1) : nullptr;
    double *dev_v = disc_mode ? dalloc<double>(ctx, s, n0) : nullptr;
    int32_t *hint_j = disc_mode ? dalloc<int32_t>(ctx, s, (size_t)p * n0) : nullptr;
    double *hint_c = disc_mode ? dalloc<double>(ctx, s, (size_t)p * n0) : nullptr;
    float *hint_dq = disc_mode ? dalloc<float>(ctx, s, (size_t)p * n0) : nullptr;
    RowState rs_saved{};
    if (disc_mode)
        rs_saved = RowState{dalloc<int32_t>(ctx, s, (size_t)p * n0), dalloc<double>(ctx, s, (size_t)p * n0),
                            dalloc<double>(ctx, s, (size_t)p * n0), dalloc<double>(ctx, s, n0),
                            dalloc<float>(ctx, s, (size_t)p * n0), dalloc<int32_t>(ctx, s, n0),
                            dalloc<double>(ctx, s, n0), nullptr};
    double *lbmax = motif_mode ? dalloc<double>(ctx, s, n0) : nullptr;
    double *mm = motif_mode ? dalloc<double>(ctx, s, (size_t)2 * nL) : nullptr;
    const double motif_limit = (double)n * std::log((double)p) / std::log((double)n);
    DiscTable tab{dalloc<double>(ctx, s, (size_t)k_max * m_max), dalloc<double>(ctx, s, (size_t)k_max * m_max),
                  dalloc<int32_t>(ctx, s, (size_t)k_max * m_max), dalloc<int32_t>(ctx, s, (size_t)k_max * m_max),
                  dalloc<int32_t>(ctx, s, (size_t)k_max * m_max)};
    if (o.keep_profiles) {
        s.keep_nnd = dalloc<double>(ctx, s, (size_t)nL * m_max * n0);
        s.keep_nnj = dalloc<int32_t>(ctx, s, (size_t)nL * m_max * n0);
    }
    int32_t *nbands_d = counters, *unit_ctr = counters + 1;
    int32_t *wait_err = counters + 3;
    int32_t *ndirect = dalloc<int32_t>(ctx, s, 2);   // [0] direct rows listed, [1] positions reserved

    // ---- one-off initialisation (the seed-row list is constant: written
    // when the workspace is created, outside any capture)
    if (!s.reuse) {
        std::vector<int32_t> kr(K);
        for (int64_t k = 0; k < K; ++k) kr[k] = (int32_t)k;
        CK(cudaMemcpyAsync(krows, kr.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    CK(cudaMemsetAsync(dstats, 0, (size_t)nL * NSTAT * sizeof(unsigned long long), st));
    if (motif_mode) launch_fill<double>(mm, (int64_t)2 * nL, INFINITY, st);
    if (disc_mode) {
        CK(cudaMemsetAsync(dkept, 0, n0 * sizeof(int32_t), st));
        CK(cudaMemsetAsync(dlog, 0, ((size_t)6 * n0 + 1) * sizeof(int32_t), st));
        CK(cudaMemsetAsync(hint_j, 0xff, (size_t)p * n0 * sizeof(int32_t), st));   // -1: no hint
    }
    CK(cudaMemsetAsync(counters, 0, 4 * sizeof(int32_t), st));
    CK(cudaMemsetAsync(vm.len, 0, n0 * sizeof(int32_t), st));
    CK(cudaMemsetAsync(tab.len, 0, (size_t)k_max * m_max * sizeof(int32_t), st));
    CK(cudaMemsetAsync(rs.ent_j, 0xff, (size_t)p * n0 * sizeof(int32_t), st));
    CK(cudaMemsetAsync(rs.ent_c, 0, (size_t)p * n0 * sizeof(double), st));
    CK(cudaMemsetAsync(rs.ent_dq, 0, (size_t)p * n0 * sizeof(float), st));
    launch_fill<T>(thr, npad, T(INFINITY), st);
    k_flat_runs<<<1024, 256, 0, st>>>(s.x, n, lmax, run);
    k_stats_init<<<(unsigned)((n0 + 255) / 256), 256, 0, st>>>(s.x, n0, lmin, mu[0], m2[0]);
    launch_split_x(s.x, n, xh, xl, st);
    CK(cudaGetLastError());

    const int occ_band = band_occupancy<T>(false, p, rpl);
    const int occ_bins = band_occupancy<T>(true, p, rpl);
    REQUIRE(occ_band > 0 && occ_bins > 0, "band kernel does not fit on this device");
    const int grid_band = ctx->num_sms * occ_band;
    const int grid_direct = ctx->num_sms * 4;
    const int grid_bins = ctx->num_sms * occ_bins;
    // columns per work unit: a multiple of the seed spacing, ~16 units per
    // resident CTA when possible (the dynamic unit queue then ends the launch
    // within about a sixteenth of a CTA's work)
    int64_t G = (KB * K) / (16 * (int64_t)grid_band);
    if (G < 1) G = 1;
    if (G > K) G = K;
    const int64_t group_w = G * SP;
    // column groups at lmin, the per-row slot stride rounded up to a multiple
    // of 4 (the merge reads the per-group counts four at a time; groups past
    // the last column are never written nor read as groups)
    const int ngroups_max = (int)(((n0 + group_w - 1) / group_w + 3) / 4 * 4);
    // column-side candidates per row (symmetric form): runs of adjacent
    // partners can clear a row's threshold together, so keep many
    // (allocated only for the symmetric form, the only one that touches them)
    const int ccap = p * 32 > 256 ? p * 32 : 256;
    T *ckey = nullptr;
    int32_t *cjj = nullptr, *ccnt = nullptr;
    if (o.band_form == 1) {
        ckey = dalloc<T>(ctx, s, (size_t)n0 * ccap);
        cjj = dalloc<int32_t>(ctx, s, (size_t)n0 * ccap);
        ccnt = dalloc<int32_t>(ctx, s, n0);
        CK(cudaMemsetAsync(ccnt, 0, n0 * sizeof(int32_t), st));
    }
    // direct path: row list, list positions, per (row, column block) top-p
    const int max_direct = (int)(n0 < (1 << 16) ? n0 : (1 << 16));
    const int dnblk = (int)((n0 + direct_cols_per_block() - 1) / direct_cols_per_block());
    int32_t *drows = dalloc<int32_t>(ctx, s, max_direct);
    int32_t *dindex = dalloc<int32_t>(ctx, s, n0);
    T *dkey = dalloc<T>(ctx, s, (size_t)max_direct * dnblk * p);
    int32_t *djj = dalloc<int32_t>(ctx, s, (size_t)max_direct * dnblk * p);
    int32_t *dcnt = dalloc<int32_t>(ctx, s, (size_t)max_direct * dnblk);
    float *ddq = dalloc<float>(ctx, s, (size_t)max_direct * dnblk * p);
    float *ddqmax = dalloc<float>(ctx, s, (size_t)nL);   // per length, max-reduced
    CK(cudaMemsetAsync(ddqmax, 0, (size_t)nL * sizeof(float), st));
    // tensor-core direct path: row operand images and per-row sums
    const bool tc = o.precision == MAD_SPLIT_TC;
    const int64_t max_direct_pad = (max_direct + 127) / 128 * 128;
    unsigned char *aimg = tc ? dalloc<unsigned char>(ctx, s, tc_aimg_bytes(max_direct, lmax)) : nullptr;
    float *tasum = tc ? dalloc<float>(ctx, s, (size_t)max_direct_pad) : nullptr;
    float *tsq = tc ? dalloc<float>(ctx, s, (size_t)max_direct_pad) : nullptr;
    // column tiles of the tensor-core path (p <= 16): eight shifted copies per
    // tile written per length and loaded by TMA (else built in the kernel)
    const int64_t col_tiles = tc_col_tiles(n0);
    void *tcb = (tc && p <= 16) ? dalloc<unsigned char>(ctx, s, tc_bcopy_bytes(col_tiles, lmax)) : nullptr;
    void *tcc = (tc && p <= 16) ? dalloc<unsigned char>(ctx, s, tc_gcc_bytes(col_tiles)) : nullptr;
    s.bmap_ok = tcb && g_tc_tma.load() && tc_encode_bmap(s.bmap, tcb, col_tiles, tc_copy_len(lmax));
    T *skey = dalloc<T>(ctx, s, (size_t)n0 * ngroups_max * p);
    int32_t *sj = dalloc<int32_t>(ctx, s, (size_t)n0 * ngroups_max * p);
    int32_t *scnt = dalloc<int32_t>(ctx, s, (size_t)n0 * ngroups_max);

    BandArgs<T> ba{};
    ba.spitch = spitch;
    ba.thr = thr;
    ba.bands = bands;
    ba.nbands = nbands_d;
    ba.unit_ctr = unit_ctr;
    ba.rpl = rpl;
    ba.sp = SP;
    ba.group_w = group_w;
    ba.p = p;
    ba.skey = skey;
    ba.sj = sj;
    ba.scnt = scnt;
    ba.bins = bins;
    ba.nbins = nbins;
    ba.err = wait_err;
    ba.rowbest = rowbest;
    {
        const int wl = g_wave_limit.load();
        ba.wave_limit = wl < 0 ? (1 << 20) : wl;
    }
    ba.ckey = ckey;
    ba.cj = cjj;
    ba.ccnt = ccnt;
    ba.cap = ccap;

    // the symmetric band form (upper triangle, both sides of each cell)
    const int use_sym = o.band_form == 1 ? 1 : 0;
    s.host_launch.assign(nL, 0);
    // CUDA events around the band-kernel, direct-path and per-row launches
    // (device time per kernel and length), from the series' pool
    s.tev_li.clear();
    const unsigned ev_flags = capture ? cudaEventRecordExternal : cudaEventRecordDefault;
    size_t ev_next = 0;
    auto ev_begin = [&](int li, int kind) {
        if (s.tev.size() < ev_next + 2) {
            cudaEvent_t a = nullptr, b = nullptr;
            CK(cudaEventCreate(&a));
            CK(cudaEventCreate(&b));
            s.tev.push_back(a);
            s.tev.push_back(b);
        }
        s.tev_li.push_back(li * 4 + kind);
        CK(cudaEventRecordWithFlags(s.tev[ev_next], st, ev_flags));
        ev_next += 2;
        return ev_next - 1;
    };
    auto ev_end_rec = [&](size_t e) { CK(cudaEventRecordWithFlags(s.tev[e], st, ev_flags)); };
    // launches issued for the current length, counted at each launch site
    unsigned long long nlaunch = 1 /* k_flat_runs */ + 1 /* k_stats_init */ + 1 /* k_split_x */ + 1 /* fill thr */;

    // Side streams: the seed rows of length l need only the window means, so
    // they run beside the extension, the split and the column data; the
    // discord tables of length l need only that length's m-th best matches,
    // so they run while the next length proceeds. Events order them against
    // the context's stream.
    struct SideRef {
        cudaStream_t prep, disc;
    } side{s.prep, s.disc};
    cudaEvent_t ev_nnd = s.sev[2], ev_end = s.sev[3];
    cudaEvent_t *ev_disc = s.sev + 4;   // [2], one per m-th NN buffer
    cudaEvent_t *ev_prep = s.sev + 6;   // [2], length prepared (by parity)
    cudaEvent_t *ev_ext = s.sev + 8;    // [2], extension done (by parity)
    // Preparation of length l on the side stream: window statistics (one
    // Welford step), column data and 1/sqrt(M2), contrast factors, seed rows
    // (one FP64 co-moment step from the previous length).
    // Its buffers (parity of l) held length l-2, whose last readers (band,
    // direct and merge kernels of l-2, extension of l-1 for the means) are
    // done once the extension of l-1 is.
    auto prep = [&](int l) {
        const int li = l - lmin, b = li & 1;
        const int64_t nl = n - l + 1;
        CK(cudaStreamWaitEvent(side.prep, ev_ext[b ^ 1], 0));
        if (l > lmin)
            launch_stats_step(s.x, nl, l, mu[b ^ 1], m2[b ^ 1], mu[b], m2[b], side.prep);
        launch_coldata<T>(s.x, nl, npad, l, mu[b], m2[b], run, colb[b], isdb[b], side.prep);
        launch_kappa(s.x, mu[b], m2[b], run, nl, l, SP, m2blk, kappab[b], kmaxb[b], side.prep);
        if (l == lmin) {
            // seed rows computed directly once, in FP64; every later length
            // steps them by one co-moment update
            SeedArgs<double> sa{s.x, mu[b], nl, l, SP, krows, (int)K, spitch, seedm, nullptr};
            launch_seed<double>(sa, side.prep);
            launch_seed_step<T>(s.x, mu[b], nl, l, SP, K, spitch, seedm, seedb[b], false, side.prep);
        } else {
            launch_seed_step<T>(s.x, mu[b ^ 1], nl, l - 1, SP, K, spitch, seedm, seedb[b], true, side.prep);
        }
        CK(cudaEventRecord(ev_prep[b], side.prep));
        CK(cudaGetLastError());
    };
    auto disc_args = [&](int64_t nl, int l, int64_t E, int all_valid, const LenOut &lo) {
        DiscPassArgs d{};
        d.n0 = n0;
        d.nl = nl;
        d.l = l;
        d.E = E;
        d.k = k_max;
        d.m = m_max;
        d.all_valid = all_valid;
        d.flag = rs.flag;
        if (sizeof(T) == 4) d.thr32 = reinterpret_cast<float *>(thr);
        else d.thr64 = reinterpret_cast<double *>(thr);
        d.nnd = lo.nnd;
        d.nnj = lo.nnj;
        d.D = dkm_d;
        d.O = dkm_o;
        d.N = dkm_n;
        d.lub = dlub;
        d.kept = dkept;
        d.O1 = dO1;
        d.cmin1 = dcmin1;
        d.ins1 = dlog;
        d.drop1 = dlog + n0;
        d.ins2 = dlog + 2 * n0;
        d.drop2 = dlog + 3 * n0;
        d.ev_t = dlog + 4 * n0;
        d.ev_j = dlog + 5 * n0;
        d.nev = dlog + 6 * n0;
        d.ev_v = dev_v;
        d.hint_j = hint_j;
        d.hint_c = hint_c;
        d.hint_dq = hint_dq;
        d.tab = tab;
        d.stats = lo.stats;
        d.st = rs;
        d.saved = rs_saved;
        d.p = p;
        return d;
    };
    // the row state before a length's recomputes (discord mode)
    auto save_rows = [&]() {
        CK(cudaMemcpyAsync(rs_saved.ent_j, rs.ent_j, (size_t)p * n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(rs_saved.ent_c, rs.ent_c, (size_t)p * n0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(rs_saved.ent_qb, rs.ent_qb, (size_t)p * n0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(rs_saved.ent_dq, rs.ent_dq, (size_t)p * n0 * sizeof(float), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(rs_saved.sigb, rs.sigb, (size_t)n0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(rs_saved.base, rs.base, (size_t)n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(rs_saved.bnum, rs.bnum, (size_t)n0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    };
    // length lmin: after the one-off initialisation on the context's stream
    CK(cudaEventRecord(ev_ext[1], st));
    prep(lmin);

    for (int l = lmin; l <= lmax; ++l) {
        const int li = l - lmin;
        const int64_t nl = n - l + 1;
        const int64_t E = excl_zone(l, num, den);
        double *nnd = nndbuf[li & 1];
        int32_t *nnj = nnjbuf[li & 1];
        // the discord tables of length l-2 have finished reading this buffer
        if (li >= 2) CK(cudaStreamWaitEvent(st, ev_disc[li & 1], 0));
        LenOut lo{nnd, nnj, dstats + (size_t)li * NSTAT};
        const int b = li & 1;
        const ErrModel &em = emb[b];
        CK(cudaStreamWaitEvent(st, ev_prep[b], 0));
        nlaunch += (l > lmin ? 1 : 0) + 4;   // stats step, column data, kappa (2), seeds

        if (l == lmin) {
            // every row recomputed; flat rows apart
            nlaunch += 2;
            launch_fill<int32_t>(rs.flag, n0, ROW_RECOMPUTE, st);
            k_init_flags<<<(unsigned)((n0 + 255) / 256), 256, 0, st>>>(run, n0, l, rs.flag, lo.stats);
        } else {
            ExtArgs<T> ea{};
            ea.xh = xh;
            ea.xl = xl;
            ea.isd = isdb[b];
            ea.x = s.x;
            ea.n0 = n0;
            ea.nl = nl;
            ea.l = l;
            ea.E = E;
            ea.p = p;
            ea.m_max = m_max;
            ea.mu_prev = mu[b ^ 1];
            ea.mu = mu[b];
            ea.m2 = m2[b];
            ea.run = run;
            ea.st = rs;
            ea.vm = vm;
            ea.out = lo;
            ea.thr = thr;
            ea.em = em;
            if (observe && l == o.observe_len) {
                ea.obs_gap = s.obs_gap;
                ea.obs_tlb = s.obs_tlb;
            }
            if (motif_mode) {
                ea.lbmax = lbmax;
                ea.min_dist_abs = reinterpret_cast<unsigned long long *>(mm + 2 * li);
                ea.min_lb_abs = reinterpret_cast<unsigned long long *>(mm + 2 * li + 1);
            }
            ea.ub_out = disc_mode ? 1 : 0;
            ea.hint_j = hint_j;
            ea.hint_c = hint_c;
            ea.hint_dq = hint_dq;
            {
                const size_t e = ev_begin(li, TK_ROWS);
                launch_extend<T>(ea, st);
                ev_end_rec(e);
            }
            if (disc_mode) {
                // Algorithm 10's first pass, then the rows its second pass can need
                DiscPassArgs dp = disc_args(nl, l, E, 0, lo);
                launch_discord_pass1(dp, st);
                launch_discord_mark(dp, st);
                save_rows();
                nlaunch += 2;
            }
            if (motif_mode) {
                SubmpArgs<T> sm{nl, rs.flag, thr, lbmax, ea.min_dist_abs, ea.min_lb_abs, lo.stats + 2, motif_limit,
                                nnd, nnj, lo.stats};
                launch_submp_mark<T>(sm, st);
                ++nlaunch;
            }
            ++nlaunch;
        }
        CK(cudaGetLastError());
        // the next length's preparation may start (it overlaps this length's
        // band kernel and fills the SMs its tail leaves idle)
        CK(cudaEventRecord(ev_ext[b], st));
        if (l < lmax) prep(l + 1);

        // Rows to recompute -> (bands | direct rows) -> seeds -> band kernel
        // -> direct kernel -> merge, with no host round trip: kernels read
        // their counts on the device (and do nothing when they are 0). A
        // second pass recomputes directly the rows whose lists fell short
        // (column-side list overflow in the symmetric form).
        SplitArgs sp{};
        sp.flag = rs.flag;
        sp.nl = nl;
        sp.R = R;
        // rows to recompute per band below which they go to the direct path:
        // the band kernel costs about R n_l cells at ALU speed, a direct row
        // n_l l multiply-adds (about 50x faster per lag on the tensor cores)
        {
            const int per = s.limf * R;
            sp.lim = per / l > 1 ? per / l : 1;
        }
        sp.force_direct = 0;
        sp.allow_sym = use_sym;
        sp.nflagged = lo.stats + 2;
        sp.bands = bands;
        sp.nbands = nbands_d;
        sp.drows = drows;
        sp.ndirect = ndirect;
        sp.dindex = dindex;
        sp.max_direct = max_direct;
        sp.stat_direct = lo.stats + 9;
        launch_split(sp, st);
        ++nlaunch;
        ba.col = colb[b];
        ba.seed = seedb[b];
        ba.nl = nl;
        ba.l = l;
        ba.E = E;
        ba.ngroups = ngroups_max;   // the slot layout keeps the lmin group count
        ba.stats = lo.stats;
        ba.ninsert = lo.stats + 4;
        ba.kb_total = (int)((nl + R - 1) / R);
        ba.nflagged = lo.stats + 2;
        ba.allow_sym = use_sym;
        if (l == lmin) {
            // first thresholds from interleaved maxima
            launch_fill<int32_t>(bins, (int64_t)n0 * nbins, (int32_t)0x807fffff, st);  // ord(-inf)
            CK(cudaMemsetAsync(unit_ctr, 0, sizeof(int32_t), st));
            {
                const size_t e = ev_begin(li, TK_BAND);
                launch_band<T>(ba, true, grid_bins, st);
                ev_end_rec(e);
            }
            launch_theta_bins<T>(bins, nbins, nl, p, m2[b], em, thr, st);
            launch_mask_thr<T>(rs.flag, n0, thr, st);
            nlaunch += 4;
            CK(cudaGetLastError());
        }
        DirectArgs<T> da{s.x, mu[b], colb[b], nl, l, E, p, drows, ndirect, thr, dkey, djj, dcnt, dnblk,
                         ddq, ddqmax + li};
        TcArgs ta{};
        if (tc) {
            ta.x = s.x;
            ta.xh = xh;
            ta.xl = xl;
            ta.n = n;
            ta.nl = nl;
            ta.l = l;
            ta.E = E;
            ta.p = p;
            ta.mu = mu[b];
            ta.m2 = m2[b];
            ta.isd = isdb[b];
            ta.rows = drows;
            ta.nrows = ndirect;
            ta.thr = reinterpret_cast<const float *>(thr);
            ta.nkc = tc_chunks(l);
            ta.aimg = aimg;
            ta.asum = tasum;
            ta.sqm2 = tsq;
            ta.okey = reinterpret_cast<float *>(dkey);
            ta.oj = djj;
            ta.ocnt = dcnt;
            ta.odq = ddq;
            ta.dq_max = ddqmax + li;
            ta.nblk = dnblk;
            ta.err = wait_err;
            ta.bcopy = tcb;
            ta.gcc = tcc;
            ta.ntiles = tc_col_tiles(nl);
            ta.tiles_ws = col_tiles;
            ta.lc = tc_copy_len(lmax);
            ta.bmap = s.bmap_ok ? s.bmap : nullptr;
        }
        MergeArgs<T> ma{};
        ma.x = s.x;
        ma.mu = mu[b];
        ma.n0 = n0;
        ma.nl = nl;
        ma.l = l;
        ma.E = E;
        ma.p = p;
        ma.m_max = m_max;
        ma.m2 = m2[b];
        ma.run = run;
        ma.col = colb[b];
        ma.skey = skey;
        ma.sj = sj;
        ma.scnt = scnt;
        ma.ngroups = ngroups_max;
        ma.group_w = group_w;
        ma.thr = thr;
        ma.st = rs;
        ma.vm = vm;
        ma.out = lo;
        ma.em = em;
        ma.xh = xh;
        ma.xl = xl;
        ma.isd = isdb[b];
        ma.overflow = lo.stats + 0;
        ma.nflagged = lo.stats + 2;
        ma.R = R;
        ma.ckey = ckey;
        ma.cj = cjj;
        ma.ccnt = ccnt;
        ma.cap = ccap;
        ma.dindex = dindex;
        ma.dkey = dkey;
        ma.dj = djj;
        ma.dcnt = dcnt;
        ma.ddq = ddq;
        ma.ddq_max = ddqmax + li;
        ma.dnblk = dnblk;
        for (int pass = 0; pass < 2; ++pass) {
            ma.allow_sym = pass == 0 ? use_sym : 0;
            if (pass == 0) {
                CK(cudaMemsetAsync(unit_ctr, 0, sizeof(int32_t), st));
                launch_fill<int32_t>(rowbest, npad, (int32_t)0x807fffff, st);   // ord(-inf)
                ++nlaunch;
                const size_t e = ev_begin(li, TK_BAND);
                launch_band<T>(ba, false, grid_band, st);
                ev_end_rec(e);
                nlaunch += use_sym ? 2 : 1;
            } else {
                sp.force_direct = 1;
                sp.allow_sym = 0;
                launch_split(sp, st);
                ++nlaunch;
            }
            {
                const size_t e = ev_begin(li, TK_DIRECT);
                if (tc && pass == 0) launch_direct_tc(ta, ctx->num_sms, st);
                else launch_direct<T>(da, grid_direct, st);
                ev_end_rec(e);
            }
            {
                const size_t e = ev_begin(li, TK_ROWS);
                launch_merge<T>(ma, st);
                ev_end_rec(e);
            }
            nlaunch += 2;
            CK(cudaGetLastError());
        }
        FlatArgs fa{n0, nl, l, E, p, m_max, run, rs, vm, lo, wait_err + 0 /* same error word */};
        launch_flat_rows(fa, st);
        if (disc_mode) {
            // lmin: every row exact, one pass in offset order (Algorithm 7);
            // later lengths: Algorithm 10's second pass; then Algorithm 9
            DiscPassArgs dp = disc_args(nl, l, E, l == lmin ? 1 : 0, lo);
            if (l == lmin) launch_discord_pass1(dp, st);
            launch_discord_pass2(dp, st);
            if (l > lmin) launch_discord_restore(dp, st);
            nlaunch += 2;
        }
        CK(cudaEventRecord(ev_nnd, st));
        CK(cudaStreamWaitEvent(side.disc, ev_nnd, 0));
        if (!motif_mode && !disc_mode) launch_discords_length(nnd, nnj, n0, nl, l, E, k_max, m_max, bval, bidx, tab, side.disc);
        nlaunch += 3;
        if (o.keep_profiles) {
            CK(cudaMemcpyAsync(s.keep_nnd + (size_t)li * m_max * n0, nnd, (size_t)m_max * n0 * sizeof(double),
                               cudaMemcpyDeviceToDevice, side.disc));
            CK(cudaMemcpyAsync(s.keep_nnj + (size_t)li * m_max * n0, nnj, (size_t)m_max * n0 * sizeof(int32_t),
                               cudaMemcpyDeviceToDevice, side.disc));
        }
        CK(cudaEventRecord(ev_disc[li & 1], side.disc));
        CK(cudaGetLastError());
        s.host_launch[li] = nlaunch;
        nlaunch = 0;
    }
    // the side streams' last work is done before the read-back
    CK(cudaEventRecord(ev_end, side.disc));
    CK(cudaStreamWaitEvent(st, ev_end, 0));
    CK(cudaEventRecord(ev_end, side.prep));
    CK(cudaStreamWaitEvent(st, ev_end, 0));
    s.dstats = dstats;
    s.wait_err = wait_err;
    s.nstat = NSTAT;
    s.vm = vm;
    s.tab = tab;
}

// ------------------------------------------------------------- autotuner
//
// Launch parameters with a measurable effect and no effect on the results
// (beyond FP32 rounding within the stated bounds): the band height R =
// 256 * rpl rows (smaller bands give small series more parallel work units,
// larger ones fewer per-column overheads per cell) and the number of rows to
// recompute per band below which they take the direct path (limf * R / l;
// the tensor-core direct path is much cheaper per row than the FP32 one).
// For each bucket (type, path, log2 of the windows, log2 of lmin, p, mode)
// the first profile times a short trial profile (lmin .. lmin + 3) for each
// candidate and keeps the fastest for the rest of the process.
struct TuneKey {
    int tsize, tc, nb, lb, p, mode;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(tsize, tc, nb, lb, p, mode) < std::tie(o.tsize, o.tc, o.nb, o.lb, o.p, o.mode);
    }
};
struct TuneVal { int rpl, limf; float ms; };
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
// mad_set_autotune: tune (1, default) or take the defaults (0)
std::atomic<int> g_autotune{1};

int ilog2(int64_t v)
{
    int b = 0;
    while (((int64_t)1 << (b + 1)) <= v) ++b;
    return b;
}

template <typename T>
void start_profile(mad_ctx *ctx, Series &s, int lmin, int lmax, int p, cudaStream_t st, bool graphs = true);
void finish_profile(mad_ctx *ctx, Series &s);

template <typename T>
void choose_launch(mad_ctx *ctx, Series &s, int lmin, int lmax, int p, cudaStream_t st)
{
    const mad_options &o = ctx->opt;
    const bool tc = o.precision == MAD_SPLIT_TC;
    const int max_rpl = band_rpl<T>(p);
    const int def_limf = tc ? 24 : 4;   // measured on the 262,144-point ECG-like range (16 / 24 / 40)
    s.rpl = max_rpl;
    s.limf = def_limf;
    const int64_t n0 = s.n - lmin + 1;
    // small series only: large ones always take the full band height (its
    // seed rows and units already fill the GPU)
    if (!g_autotune.load() || n0 > 32768) return;
    const TuneKey key{(int)sizeof(T), tc ? 1 : 0, ilog2(n0), ilog2(lmin), p, o.mode};
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) {
        std::vector<std::pair<int, int>> cand;
        for (int r : {4, 2, 1})
            if (r <= max_rpl)
                for (int lf : tc ? std::vector<int>{12, 24, 48} : std::vector<int>{4}) cand.push_back({r, lf});
        const int tmax = lmax < lmin + 3 ? lmax : lmin + 3;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        TuneVal best{max_rpl, def_limf, 1e30f};
        try {
            for (auto &c : cand) {
                s.rpl = c.first;
                s.limf = c.second;
                for (int rep = 0; rep < 2; ++rep) {   // the first run allocates and loads modules
                    CK(cudaEventRecord(e0, st));
                    start_profile<T>(ctx, s, lmin, tmax, p, st);
                    CK(cudaEventRecord(e1, st));
                    CK(cudaStreamSynchronize(st));
                    finish_profile(ctx, s);
                }
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best.ms) best = TuneVal{c.first, c.second, ms};
            }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        free_profile(s);
        it = g_tune.emplace(key, best).first;
    }
    s.rpl = it->second.rpl;
    s.limf = it->second.limf;
}

// Start one profile of a series on stream st: validate, reuse the workspace
// while the key holds, and issue the profile -- eagerly the first time
// (buffers allocated), into a CUDA graph the second time with the same key
// (captured, instantiated, launched), and by replaying that graph after;
// then queue the read-back of the error word and the per-length counters
// into pinned host memory. finish_profile reads them once st is done.
template <typename T>
void start_profile(mad_ctx *ctx, Series &s, int lmin, int lmax, int p, cudaStream_t st, bool graphs)
{
    const mad_options &o = ctx->opt;
    const int num = o.excl_num, den = o.excl_den;
    const int64_t n = s.n;
    REQUIRE(lmin >= 2 && lmin <= lmax, "need 2 <= lmin <= lmax");
    REQUIRE((int64_t)lmax < n, "lmax must be smaller than the series length");
    REQUIRE(p >= 1 && p <= MAXP, "p must be in [1, 64]");
    REQUIRE(o.m_max <= p, "m_max must not exceed p (the paper's p >= m)");
    const int64_t Emax = excl_zone(lmax, num, den);
    REQUIRE(n - lmax + 1 > 2 * Emax + 2, "series too short for lmax and the exclusion zone (need n-lmax+1 > 2E(lmax)+2)");
    REQUIRE(n < (int64_t)INT32_MAX - 4096, "series longer than 2^31 - 4096 samples");
    REQUIRE(s.rpl >= 1 && s.limf >= 1, "launch parameters not chosen");

    WsKey key{};
    key.tsize = (int)sizeof(T);
    key.tc = o.precision == MAD_SPLIT_TC ? 1 : 0;
    key.lmin = lmin;
    key.lmax = lmax;
    key.p = p;
    key.m_max = o.m_max;
    key.k_max = o.k_max;
    key.mode = o.mode;
    key.band_form = o.band_form;
    key.keep = o.keep_profiles ? 1 : 0;
    key.observe = o.observe_len;
    key.num = num;
    key.den = den;
    key.audit = g_audit.load();
    key.wave_limit = g_wave_limit.load();
    key.rpl = s.rpl;
    key.limf = s.limf;
    key.tma = g_tc_tma.load();
    const bool same = s.ws_valid && s.key == key;
    if (!same) {
        free_profile(s);
        s.key = key;
    }
    s.profiled = false;
    s.lmin = lmin;
    s.lmax = lmax;
    const int nL = lmax - lmin + 1;
    s.stats.assign(nL, mad_length_stats{});
    // streams and events of the pipeline, created once per series
    if (!s.prep) {
        CK(cudaStreamCreateWithFlags(&s.prep, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&s.disc, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&s.cap, cudaStreamNonBlocking));
        for (cudaEvent_t &e : s.sev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const bool replay = same && s.exec && graphs && g_graphs.load();
    if (replay) {
        CK(cudaGraphLaunch(s.exec, st));
    } else {
        s.reuse = same;
        s.cursor = 0;
        const bool capture = same && graphs && g_graphs.load();
        if (!capture) {
            issue_profile<T>(ctx, s, lmin, lmax, p, st, false);
        } else {
            // capture on the series' own stream (the caller's may be the
            // legacy default stream, which cannot be captured), then launch
            // the instantiated graph on the caller's stream
            CK(cudaStreamBeginCapture(s.cap, cudaStreamCaptureModeThreadLocal));
            cudaGraph_t g = nullptr;
            try {
                issue_profile<T>(ctx, s, lmin, lmax, p, s.cap, true);
            } catch (...) {
                cudaStreamEndCapture(s.cap, &g);
                if (g) cudaGraphDestroy(g);
                s.ws_valid = false;
                throw;
            }
            CK(cudaStreamEndCapture(s.cap, &g));
            const cudaError_t ei = cudaGraphInstantiateWithFlags(&s.exec, g, 0);
            cudaGraphDestroy(g);
            CK(ei);
            CK(cudaGraphLaunch(s.exec, st));
        }
        s.ws_valid = true;
        s.reuse = false;
    }
    s.graph_last = same && s.exec && graphs && g_graphs.load();
    const size_t words = 1 + (size_t)nL * s.nstat;
    if (words > s.hbuf_words) {
        if (s.hbuf) cudaFreeHost(s.hbuf);
        s.hbuf = nullptr;
        s.hbuf_words = 0;
        CK(cudaHostAlloc(reinterpret_cast<void **>(&s.hbuf), words * sizeof(unsigned long long), cudaHostAllocDefault));
        s.hbuf_words = words;
    }
    s.hbuf[0] = 0;
    CK(cudaMemcpyAsync(s.hbuf, s.wait_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(s.hbuf + 1, s.dstats, (size_t)nL * s.nstat * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       st));
}

// The host side of a finished profile (its stream synchronised): error word,
// per-length counters, kernel timings.
void finish_profile(mad_ctx *ctx, Series &s)
{
    const mad_options &o = ctx->opt;
    const int lmin = s.lmin, nL = s.lmax - s.lmin + 1;
    const int64_t n = s.n;
    const int NSTAT = s.nstat;
    const int32_t herr = (int32_t)(s.hbuf[0] & 0xffffffffu);
    const unsigned long long *hs = s.hbuf + 1;
    const bool motif_mode = o.mode == 1;
    const bool disc_mode = o.mode == 2;
    if (herr != 0) {
        set_err(ctx, "a bounded wait in the band kernel ran out, or a row was left without its recompute");
        throw Fail{MAD_ETIMEOUT};
    }
    for (int li = 0; li < nL; ++li) {
        mad_length_stats &q = s.stats[li];
        const unsigned long long *h = &hs[(size_t)li * NSTAT];
        q.len = lmin + li;
        q.rows = n - (lmin + li) + 1;
        q.certified = (int64_t)h[1];
        q.recomputed = (int64_t)h[2];
        q.skipped = (int64_t)h[10];
        q.full_profile = (int32_t)h[11];
        if (motif_mode && li > 0) q.recomputed = q.full_profile ? q.rows : (int64_t)(h[2] - h[10]);
        if (disc_mode && li > 0) q.recomputed = (int64_t)(h[2] - h[10]);
        q.tiles = (int64_t)h[5];
        q.passes = q.recomputed > 0 ? (h[0] > 0 ? 2 : 1) : 0;
        unsigned long long bits = h[3];
        std::memcpy(&q.fp32_dq_max, &bits, sizeof(double));
        bits = h[12];
        std::memcpy(&q.dq_ratio_max, &bits, sizeof(double));
        q.band_cells = (int64_t)h[6];
        q.inserts = (int64_t)h[4];
        q.col_appends = (int64_t)h[7];
        q.second_pass_rows = (int64_t)h[0];
        q.direct_rows = (int64_t)h[9];
        q.launches = (int64_t)s.host_launch[li];
        q.band_ms = q.direct_ms = q.rows_ms = 0.0;
        q.graph = s.graph_last ? 1 : 0;
        q.band_rows = 32 * BAND_NW * s.rpl;
    }
    for (size_t e = 0; e < s.tev_li.size(); ++e) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, s.tev[2 * e], s.tev[2 * e + 1]));
        mad_length_stats &q = s.stats[s.tev_li[e] / 4];
        switch (s.tev_li[e] % 4) {
        case TK_BAND: q.band_ms += ms; break;
        case TK_DIRECT: q.direct_ms += ms; break;
        default: q.rows_ms += ms; break;
        }
    }
    s.profiled = true;
}

template <typename T>
void profile_series(mad_ctx *ctx, Series &s, int lmin, int lmax, int p, cudaStream_t st)
{
    choose_launch<T>(ctx, s, lmin, lmax, p, st);
    start_profile<T>(ctx, s, lmin, lmax, p, st);
    CK(cudaStreamSynchronize(st));
    finish_profile(ctx, s);
}

Series &get_series(mad_ctx *ctx, int32_t idx)
{
    if (idx < 0 || idx >= (int32_t)ctx->series.size()) {
        set_err(ctx, "series index out of range");
        throw Fail{MAD_EINVAL};
    }
    return ctx->series[idx];
}

bool fp32_kernels(const mad_ctx *ctx)
{
    return ctx->opt.precision == MAD_FP32 || ctx->opt.precision == MAD_SPLIT_TC;
}

void profile_one(mad_ctx *ctx, Series &s, int lmin, int lmax, int p, cudaStream_t st)
{
    if (fp32_kernels(ctx)) profile_series<float>(ctx, s, lmin, lmax, p, st);
    else profile_series<double>(ctx, s, lmin, lmax, p, st);
}

// Batch: tune and start (no host wait) one series on stream st. Repeated
// batch profiles reuse each series' workspace but launch eagerly: with many
// series in flight on eight streams, replaying one graph per series measured
// slower than the eager launches (batch256: 19.8 s against 18.1 s per step).
void start_one(mad_ctx *ctx, Series &s, int lmin, int lmax, int p, cudaStream_t st)
{
    if (fp32_kernels(ctx)) {
        choose_launch<float>(ctx, s, lmin, lmax, p, st);
        start_profile<float>(ctx, s, lmin, lmax, p, st, false);
    } else {
        choose_launch<double>(ctx, s, lmin, lmax, p, st);
        start_profile<double>(ctx, s, lmin, lmax, p, st, false);
    }
}

template <typename F>
mad_status run_guarded(mad_ctx *ctx, F &&f)
{
    try {
        if (ctx) {
            cudaSetDevice(ctx->device);
            ctx->err.clear();
        }
        f();
        return MAD_OK;
    } catch (const Fail &e) {
        return e.st;
    } catch (const std::bad_alloc &) {
        set_err(ctx, "host allocation failed");
        return MAD_ENOMEM;
    } catch (...) {
        set_err(ctx, "internal error");
        return MAD_EINTERNAL;
    }
}

}  // namespace

// ---------------------------------------------------------------- the ABI

namespace mad {
// Error text of context-free calls, returned by mad_last_error(NULL).
void set_thread_error(const std::string &msg) { g_create_err = msg; }
}  // namespace mad

extern "C" {

MAD_API mad_status mad_create(const double *host_series, int64_t n, const mad_options *opt, mad_ctx **out)
{
    if (!out) { g_create_err = "out is NULL"; return MAD_EINVAL; }
    *out = nullptr;
    const double *const ser[1] = {host_series};
    const int64_t ns[1] = {n};
    return mad_create_batch(ser, ns, 1, opt, out);
}

MAD_API mad_status mad_create_batch(const double *const *series, const int64_t *n, int32_t count,
                                    const mad_options *opt, mad_ctx **out)
{
    if (!out) { g_create_err = "out is NULL"; return MAD_EINVAL; }
    *out = nullptr;
    mad_ctx *c = new (std::nothrow) mad_ctx;
    if (!c) { g_create_err = "host allocation failed"; return MAD_ENOMEM; }
    mad_ctx *ctx = nullptr;   // errors before success go to the thread-local message
    mad_status r = run_guarded(ctx, [&] {
        REQUIRE(series != nullptr && n != nullptr && count >= 1, "need count >= 1 series");
        for (int32_t s = 0; s < count; ++s) {
            REQUIRE(series[s] != nullptr, "series pointer is NULL");
            REQUIRE(n[s] >= 4, "series needs at least 4 samples");
        }
        {
            mad_options chk = defaults(opt);
            check_options(ctx, chk);
        }
        init_ctx(c, opt);
        cudaSetDevice(c->device);
        c->series.resize(count);
        for (int32_t s = 0; s < count; ++s) {
            Series &S = c->series[s];
            S.n = n[s];
            void *p = nullptr;
            CK(cudaMalloc(&p, n[s] * sizeof(double)));
            S.x = static_cast<double *>(p);
            S.own_x = true;
            CK(cudaMemcpyAsync(S.x, series[s], n[s] * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        }
        CK(cudaStreamSynchronize(c->stream));
    });
    if (r != MAD_OK) {
        if (!c->err.empty()) g_create_err = c->err;
        mad_destroy(c);
        return r;
    }
    *out = c;
    return MAD_OK;
}

MAD_API mad_status mad_create_device(const void *dev_series, int32_t dtype, int64_t n, const mad_options *opt,
                                     mad_ctx **out)
{
    if (!out) { g_create_err = "out is NULL"; return MAD_EINVAL; }
    *out = nullptr;
    mad_ctx *c = new (std::nothrow) mad_ctx;
    if (!c) { g_create_err = "host allocation failed"; return MAD_ENOMEM; }
    mad_ctx *ctx = nullptr;
    mad_status r = run_guarded(ctx, [&] {
        REQUIRE(dev_series != nullptr, "device series pointer is NULL");
        REQUIRE(dtype == 0 || dtype == 1, "dtype must be 0 (FP64) or 1 (FP32)");
        REQUIRE(n >= 4, "series needs at least 4 samples");
        {
            mad_options chk = defaults(opt);
            check_options(ctx, chk);
        }
        init_ctx(c, opt);
        cudaSetDevice(c->device);
        c->series.resize(1);
        Series &S = c->series[0];
        S.n = n;
        if (dtype == 0) {
            S.x = const_cast<double *>(static_cast<const double *>(dev_series));
            S.own_x = false;
        } else {
            void *p = nullptr;
            CK(cudaMalloc(&p, n * sizeof(double)));
            S.x = static_cast<double *>(p);
            S.own_x = true;
            k_widen_f32<<<256, 256, 0, c->stream>>>(static_cast<const float *>(dev_series), n, S.x);
            CK(cudaGetLastError());
        }
        CK(cudaStreamSynchronize(c->stream));
    });
    if (r != MAD_OK) {
        if (!c->err.empty()) g_create_err = c->err;
        mad_destroy(c);
        return r;
    }
    *out = c;
    return MAD_OK;
}

MAD_API void mad_debug_wavefront_wait_limit(int32_t tries) { g_wave_limit.store(tries); }

MAD_API void mad_debug_audit_error_bounds(int32_t on) { g_audit.store(on ? 1 : 0); }

MAD_API void mad_set_graphs(int32_t on) { g_graphs.store(on ? 1 : 0); }

MAD_API void mad_set_autotune(int32_t on) { g_autotune.store(on ? 1 : 0); }

MAD_API void mad_debug_tc_tma(int32_t on) { g_tc_tma.store(on ? 1 : 0); }

MAD_API mad_status mad_profile(mad_ctx *ctx, int32_t lmin, int32_t lmax, int32_t p)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    return run_guarded(ctx, [&] {
        REQUIRE(ctx->series.size() == 1, "context holds several series: use mad_profile_batch");
        profile_one(ctx, ctx->series[0], lmin, lmax, p, ctx->stream);
    });
}

MAD_API mad_status mad_profile_batch(mad_ctx *ctx, const int32_t *lmin, const int32_t *lmax, int32_t p)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    return run_guarded(ctx, [&] {
        REQUIRE(lmin != nullptr && lmax != nullptr, "lmin / lmax arrays are NULL");
        // Series are independent. Eight host threads, each with its own
        // stream, start the series' profiles without waiting on the device:
        // a series profiled before with the same shape is one graph launch
        // (its whole per-length sequence), so the series run back to back on
        // eight streams and the GPU interleaves them. Every stream first
        // waits for the context's stream (where the inputs were written);
        // each thread then waits for its stream and reads its series'
        // counters back.
        const int count = (int)ctx->series.size();
        const int nw = count < 8 ? count : 8;
        std::vector<cudaStream_t> ws(nw, nullptr);
        cudaEvent_t ready = nullptr;
        struct Guard {
            std::vector<cudaStream_t> &ws;
            cudaEvent_t &ev;
            ~Guard()
            {
                for (cudaStream_t q : ws)
                    if (q) {
                        cudaStreamSynchronize(q);
                        cudaStreamDestroy(q);
                    }
                if (ev) cudaEventDestroy(ev);
            }
        } guard{ws, ready};
        CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        CK(cudaEventRecord(ready, ctx->stream));
        for (cudaStream_t &q : ws) {
            CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
            CK(cudaStreamWaitEvent(q, ready, 0));
        }
        std::vector<mad_status> res(nw, MAD_OK);
        std::vector<std::thread> th;
        for (int t = 0; t < nw; ++t)
            th.emplace_back([&, t] {
                cudaSetDevice(ctx->device);
                try {
                    for (int k = t; k < count; k += nw) start_one(ctx, ctx->series[k], lmin[k], lmax[k], p, ws[t]);
                    CK(cudaStreamSynchronize(ws[t]));
                    for (int k = t; k < count; k += nw) finish_profile(ctx, ctx->series[k]);
                } catch (const Fail &e) {
                    res[t] = e.st;
                } catch (...) {
                    set_err(ctx, "internal error");
                    res[t] = MAD_EINTERNAL;
                }
            });
        for (std::thread &x : th) x.join();
        for (mad_status r : res)
            if (r != MAD_OK) throw Fail{r};
    });
}

MAD_API mad_status mad_motifs(mad_ctx *ctx, int32_t series, int32_t k, mad_motif *out, int32_t *n_out)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    return run_guarded(ctx, [&] {
        Series &s = get_series(ctx, series);
        REQUIRE(out != nullptr && n_out != nullptr, "output pointers are NULL");
        REQUIRE(k >= 1 && k <= 4096, "k must be in [1, 4096]");
        if (!s.profiled) {
            set_err(ctx, "mad_motifs before mad_profile");
            throw Fail{MAD_ESTATE};
        }
        cudaStream_t st = ctx->stream;
        const int64_t nblk = (s.n0 + 255) / 256;
        {
            Carve cv{{sizeof(int32_t) * 3 * k, sizeof(int32_t) * k, sizeof(double) * nblk, sizeof(int32_t) * nblk,
                      sizeof(double) * k}};
            std::vector<void *> b = rscratch(ctx, s, cv, st);
            int32_t *acc = (int32_t *)b[0];
            int32_t *picked = (int32_t *)b[1];
            double *bval = (double *)b[2];
            int32_t *bidx = (int32_t *)b[3];
            double *rd = (double *)b[4];
            for (int r = 0; r < k; ++r)
                launch_motif_round(s.vm, s.n0, ctx->opt.excl_num, ctx->opt.excl_den, acc, r, bval, bidx, picked, st);
            CK(cudaGetLastError());
            std::vector<int32_t> hp(k), ha(3 * k);
            CK(cudaMemcpyAsync(hp.data(), picked, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(ha.data(), acc, sizeof(int32_t) * 3 * k, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            int got = 0;
            while (got < k && hp[got] >= 0) ++got;
            launch_recheck_pairs(s.x, s.n, acc, got, rd, st);
            std::vector<double> hd(s.n0), hn(s.n0), hr(k);
            if (got > 0) CK(cudaMemcpyAsync(hr.data(), rd, sizeof(double) * got, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(hd.data(), s.vm.dist, sizeof(double) * s.n0, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(hn.data(), s.vm.norm, sizeof(double) * s.n0, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (int r = 0; r < got; ++r) {
                mad_motif &m = out[r];
                m.a = ha[3 * r];
                m.b = ha[3 * r + 1];
                m.len = ha[3 * r + 2];
                m.reserved = 0;
                m.dist = hd[hp[r]];
                m.norm_dist = hn[hp[r]];
                m.dist_recheck = hr[r];
            }
            *n_out = got;
        }
    });
}

MAD_API mad_status mad_motif_sets(mad_ctx *ctx, int32_t series, int32_t k, double D, int32_t cap,
                                  mad_motif_set *sets, int64_t *members, int32_t *n_out)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    // the motif pairs first (a call of its own, which validates the series
    // and its state)
    REQUIRE_RET(sets != nullptr && members != nullptr && n_out != nullptr, "output pointers are NULL");
    REQUIRE_RET(k >= 1 && k <= 64, "k must be in [1, 64]");
    REQUIRE_RET(cap >= 2 && cap <= 256, "cap must be in [2, 256]");
    REQUIRE_RET(D >= 0.0 && D <= 1e300, "D must be a finite number >= 0");
    std::vector<mad_motif> mot(k);
    int32_t got = 0;
    const mad_status ms = mad_motifs(ctx, series, k, mot.data(), &got);
    if (ms != MAD_OK) return ms;
    return run_guarded(ctx, [&] {
        Series &s = get_series(ctx, series);
        cudaStream_t st = ctx->stream;
        const int num = ctx->opt.excl_num, den = ctx->opt.excl_den;
        std::vector<void *> tmp;
        auto talloc = [&](size_t bytes) {
            void *p = nullptr;
            CK(cudaMalloc(&p, bytes > 0 ? bytes : 1));
            tmp.push_back(p);
            return p;
        };
        try {
            const int64_t capc = s.n0;
            double *ckey = (double *)talloc(sizeof(double) * capc);
            int32_t *cj = (int32_t *)talloc(sizeof(int32_t) * capc);
            int32_t *ccount = (int32_t *)talloc(sizeof(int32_t));
            int64_t *dmem = (int64_t *)talloc(sizeof(int64_t) * cap);
            int32_t *dcnt = (int32_t *)talloc(sizeof(int32_t));
            int64_t *poff = (int64_t *)talloc(sizeof(int64_t) * (size_t)k * cap);
            int64_t *pE = (int64_t *)talloc(sizeof(int64_t) * (size_t)k * cap);
            std::vector<int64_t> hoff, hE;
            for (int si = 0; si < got; ++si) {
                const mad_motif &m = mot[si];
                const int l = m.len;
                SetArgs a{};
                a.x = s.x;
                a.n = s.n;
                a.l = l;
                a.E = excl_zone(l, num, den);
                a.a = m.a;
                a.b = m.b;
                a.r = D * m.dist_recheck;
                a.nprev = (int)hoff.size();
                if (a.nprev > 0) {
                    CK(cudaMemcpyAsync(poff, hoff.data(), sizeof(int64_t) * hoff.size(), cudaMemcpyHostToDevice, st));
                    CK(cudaMemcpyAsync(pE, hE.data(), sizeof(int64_t) * hE.size(), cudaMemcpyHostToDevice, st));
                }
                a.prev_off = poff;
                a.prev_E = pE;
                a.ckey = ckey;
                a.cj = cj;
                a.ccount = ccount;
                a.capc = capc;
                CK(cudaMemsetAsync(ccount, 0, sizeof(int32_t), st));
                launch_motif_set(a, cap, dmem, dcnt, st);
                CK(cudaGetLastError());
                int32_t hc = 0;
                CK(cudaMemcpyAsync(&hc, dcnt, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                CK(cudaMemcpyAsync(members + (size_t)si * cap, dmem, sizeof(int64_t) * hc, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                mad_motif_set &o = sets[si];
                o.a = m.a;
                o.b = m.b;
                o.len = l;
                o.count = hc;
                o.radius = a.r;
                for (int t = 0; t < hc; ++t) {
                    hoff.push_back(members[(size_t)si * cap + t]);
                    hE.push_back(a.E);
                }
            }
            *n_out = got;
        } catch (...) {
            for (void *p : tmp) cudaFree(p);
            throw;
        }
        for (void *p : tmp) cudaFree(p);
    });
}

MAD_API mad_status mad_observe(mad_ctx *ctx, int32_t series, double *gap, double *tlb)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    return run_guarded(ctx, [&] {
        Series &s = get_series(ctx, series);
        if (!s.profiled || s.obs_len == 0) {
            set_err(ctx, "no observation: set options.observe_len to a length in (lmin, lmax] and profile");
            throw Fail{MAD_ESTATE};
        }
        const int64_t nl = s.n - s.obs_len + 1;
        cudaStream_t st = ctx->stream;
        if (gap) CK(cudaMemcpyAsync(gap, s.obs_gap, sizeof(double) * nl, cudaMemcpyDeviceToHost, st));
        if (tlb) CK(cudaMemcpyAsync(tlb, s.obs_tlb, sizeof(double) * nl, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    });
}

// Host side of a discord read-out: the k x m cells (rank-major, row stride
// `stride` cells) already copied to the host, each re-checked in FP64 from a
// full distance profile, written to out.
static void finish_discords(mad_ctx *ctx, Series &s, int k, int m, int stride, const std::vector<double> &nd,
                            const std::vector<double> &dd, const std::vector<int32_t> &off,
                            const std::vector<int32_t> &len, const std::vector<int32_t> &nn, mad_discord *out)
{
    cudaStream_t st = ctx->stream;
    std::vector<int32_t> req;
    std::vector<int> where;
    for (int r = 0; r < k; ++r)
        for (int c = 0; c < m; ++c) {
            const size_t cell = (size_t)r * stride + c;
            if (len[cell] > 0) {
                req.push_back(off[cell]);
                req.push_back(len[cell]);
                req.push_back(c + 1);
                where.push_back(r * m + c);
            }
        }
    std::vector<double> rec(where.size(), NAN);
    if (!where.empty()) {
        const int nc = (int)where.size();
        const size_t ns = recheck_scratch(nc, m);
        Carve cv{{req.size() * sizeof(int32_t), nc * sizeof(double), ns * sizeof(double), ns * sizeof(int32_t)}};
        std::vector<void *> b = rscratch(ctx, s, cv, st);
        CK(cudaMemcpyAsync(b[0], req.data(), req.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        launch_recheck_discords(s.x, s.n, (const int32_t *)b[0], nc, ctx->opt.excl_num, ctx->opt.excl_den,
                                (double *)b[1], (double *)b[2], (int32_t *)b[3], m, st);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(rec.data(), b[1], nc * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    size_t w = 0;
    for (int r = 0; r < k; ++r)
        for (int c = 0; c < m; ++c) {
            const size_t cell = (size_t)r * stride + c;
            mad_discord &q = out[r * m + c];
            q.rank = r + 1;
            q.m = c + 1;
            q.reserved = 0;
            if (len[cell] > 0) {
                q.off = off[cell];
                q.nn = nn[cell];
                q.len = len[cell];
                q.dist = dd[cell];
                q.norm_dist = nd[cell];
                q.dist_recheck = rec[w++];
            } else {
                q.off = -1;
                q.nn = -1;
                q.len = 0;
                q.dist = NAN;
                q.norm_dist = NAN;
                q.dist_recheck = NAN;
            }
        }
}

MAD_API mad_status mad_discords(mad_ctx *ctx, int32_t series, int32_t k, int32_t m, mad_discord *out,
                                int32_t *n_out)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    return run_guarded(ctx, [&] {
        Series &s = get_series(ctx, series);
        REQUIRE(out != nullptr && n_out != nullptr, "output pointers are NULL");
        if (!s.profiled) {
            set_err(ctx, "mad_discords before mad_profile");
            throw Fail{MAD_ESTATE};
        }
        REQUIRE(k >= 1 && k <= s.k_max, "k must be in [1, k_max]");
        REQUIRE(m >= 1 && m <= s.m_max, "m must be in [1, m_max]");
        if (ctx->opt.mode == 1) {
            set_err(ctx, "the discord table needs mode 0 (exact rows); motif mode keeps no discord table");
            throw Fail{MAD_ESTATE};
        }
        cudaStream_t st = ctx->stream;
        const size_t cells = (size_t)s.k_max * s.m_max;
        std::vector<double> nd(cells), dd(cells);
        std::vector<int32_t> off(cells), len(cells), nn(cells);
        CK(cudaMemcpyAsync(nd.data(), s.tab.norm, cells * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(dd.data(), s.tab.dist, cells * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(off.data(), s.tab.off, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(len.data(), s.tab.len, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(nn.data(), s.tab.nn, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        finish_discords(ctx, s, k, m, s.m_max, nd, dd, off, len, nn, out);
        *n_out = k * m;
    });
}

MAD_API mad_status mad_discords_global(mad_ctx *ctx, int32_t series, int32_t k, int32_t m, mad_discord *out,
                                       int32_t *n_out)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    return run_guarded(ctx, [&] {
        Series &s = get_series(ctx, series);
        REQUIRE(out != nullptr && n_out != nullptr, "output pointers are NULL");
        if (!s.profiled) {
            set_err(ctx, "mad_discords_global before mad_profile");
            throw Fail{MAD_ESTATE};
        }
        REQUIRE(k >= 1 && k <= KMAX, "k must be in [1, 64]");
        REQUIRE(m >= 1 && m <= s.m_max, "m must be in [1, m_max]");
        if (ctx->opt.mode != 0) {
            set_err(ctx, "global discords need mode 0 (exact rows)");
            throw Fail{MAD_ESTATE};
        }
        REQUIRE(s.keep_nnd != nullptr, "profile was computed without keep_profiles");
        cudaStream_t st = ctx->stream;
        GDiscArgs a{};
        a.nnd = s.keep_nnd;
        a.nnj = s.keep_nnj;
        a.n = s.n;
        a.n0 = s.n0;
        a.lmin = s.lmin;
        a.nL = s.lmax - s.lmin + 1;
        a.m_max = s.m_max;
        a.num = ctx->opt.excl_num;
        a.den = ctx->opt.excl_den;
        a.nblk = (int)((s.n0 + GDISC_TILE - 1) / GDISC_TILE);
        a.k = k;
        a.mcols = m;
        const size_t cells = (size_t)k * m, nt = (size_t)m * a.nL * a.nblk;
        // one allocation: tile table, then the k x m cells
        const size_t bytes = nt * (sizeof(double) + sizeof(int64_t)) + cells * (2 * sizeof(double) + 3 * sizeof(int32_t));
        void *buf = nullptr;
        cudaError_t e = cudaMalloc(&buf, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_err(ctx, "cudaMalloc failed for the global discord scratch");
            throw Fail{MAD_ENOMEM};
        }
        char *p = (char *)buf;
        a.tv = (double *)p;
        p += nt * sizeof(double);
        a.tk = (int64_t *)p;
        p += nt * sizeof(int64_t);
        a.out.norm = (double *)p;
        p += cells * sizeof(double);
        a.out.dist = (double *)p;
        p += cells * sizeof(double);
        a.out.off = (int32_t *)p;
        p += cells * sizeof(int32_t);
        a.out.len = (int32_t *)p;
        p += cells * sizeof(int32_t);
        a.out.nn = (int32_t *)p;
        std::vector<double> nd(cells), dd(cells);
        std::vector<int32_t> off(cells), len(cells), nn(cells);
        cudaError_t e2 = cudaMemsetAsync(a.out.len, 0, cells * sizeof(int32_t), st);
        if (e2 == cudaSuccess) {
            launch_discords_global(a, st);
            e2 = cudaGetLastError();
        }
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(nd.data(), a.out.norm, cells * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(dd.data(), a.out.dist, cells * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(off.data(), a.out.off, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(len.data(), a.out.len, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(nn.data(), a.out.nn, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        cudaError_t e3 = cudaStreamSynchronize(st);
        cudaFree(buf);
        CK(e2);
        CK(e3);
        finish_discords(ctx, s, k, m, m, nd, dd, off, len, nn, out);
        *n_out = k * m;
    });
}

MAD_API mad_status mad_discords_streamed(mad_ctx *ctx, int32_t series, int32_t k, int32_t m, mad_discord *out,
                                         int32_t *n_out)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    return run_guarded(ctx, [&] {
        Series &s = get_series(ctx, series);
        REQUIRE(out != nullptr && n_out != nullptr, "output pointers are NULL");
        if (!s.profiled) {
            set_err(ctx, "mad_discords_streamed before mad_profile");
            throw Fail{MAD_ESTATE};
        }
        REQUIRE(k >= 1 && k <= KMAX, "k must be in [1, 64]");
        REQUIRE(m >= 1 && m <= s.m_max, "m must be in [1, m_max]");
        if (ctx->opt.mode != 0) {
            set_err(ctx, "streamed discords need mode 0 (exact rows)");
            throw Fail{MAD_ESTATE};
        }
        REQUIRE(s.keep_nnd != nullptr, "profile was computed without keep_profiles");
        cudaStream_t st = ctx->stream;
        StreamArgs a{};
        a.nnd = s.keep_nnd;
        a.nnj = s.keep_nnj;
        a.n = s.n;
        a.n0 = s.n0;
        a.lmin = s.lmin;
        a.nL = s.lmax - s.lmin + 1;
        a.m_max = s.m_max;
        a.num = ctx->opt.excl_num;
        a.den = ctx->opt.excl_den;
        a.k = k;
        a.m = m;
        const size_t cells = (size_t)k * m, tab = (size_t)a.nL * cells;
        const size_t bytes = tab * (sizeof(double) + 2 * sizeof(int32_t)) + cells * (2 * sizeof(double) + 3 * sizeof(int32_t));
        void *buf = nullptr;
        cudaError_t e = cudaMalloc(&buf, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_err(ctx, "cudaMalloc failed for the streamed discord tables");
            throw Fail{MAD_ENOMEM};
        }
        char *p = (char *)buf;
        a.d = (double *)p;
        p += tab * sizeof(double);
        a.out.norm = (double *)p;
        p += cells * sizeof(double);
        a.out.dist = (double *)p;
        p += cells * sizeof(double);
        a.o = (int32_t *)p;
        p += tab * sizeof(int32_t);
        a.nn = (int32_t *)p;
        p += tab * sizeof(int32_t);
        a.out.off = (int32_t *)p;
        p += cells * sizeof(int32_t);
        a.out.len = (int32_t *)p;
        p += cells * sizeof(int32_t);
        a.out.nn = (int32_t *)p;
        std::vector<double> nd(cells), dd(cells);
        std::vector<int32_t> off(cells), len(cells), nn(cells);
        launch_discords_streamed(a, st);
        cudaError_t e2 = cudaGetLastError();
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(nd.data(), a.out.norm, cells * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(dd.data(), a.out.dist, cells * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(off.data(), a.out.off, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(len.data(), a.out.len, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(nn.data(), a.out.nn, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        cudaError_t e3 = cudaStreamSynchronize(st);
        cudaFree(buf);
        CK(e2);
        CK(e3);
        finish_discords(ctx, s, k, m, m, nd, dd, off, len, nn, out);
        *n_out = k * m;
    });
}

MAD_API mad_status mad_valmp(mad_ctx *ctx, int32_t series, double *dist, double *norm, int32_t *len, int64_t *nn)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    return run_guarded(ctx, [&] {
        Series &s = get_series(ctx, series);
        if (!s.profiled) {
            set_err(ctx, "mad_valmp before mad_profile");
            throw Fail{MAD_ESTATE};
        }
        cudaStream_t st = ctx->stream;
        std::vector<int32_t> j32(s.n0);
        if (dist) CK(cudaMemcpyAsync(dist, s.vm.dist, s.n0 * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (norm) CK(cudaMemcpyAsync(norm, s.vm.norm, s.n0 * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (len) CK(cudaMemcpyAsync(len, s.vm.len, s.n0 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        if (nn) CK(cudaMemcpyAsync(j32.data(), s.vm.nn, s.n0 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (nn)
            for (int64_t i = 0; i < s.n0; ++i) nn[i] = j32[i];
    });
}

MAD_API mad_status mad_matrix_profile(mad_ctx *ctx, int32_t series, int32_t len, double *mp, int64_t *ip,
                                      double *nnd, int64_t *nnj)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    return run_guarded(ctx, [&] {
        Series &s = get_series(ctx, series);
        if (!s.profiled) {
            set_err(ctx, "mad_matrix_profile before mad_profile");
            throw Fail{MAD_ESTATE};
        }
        REQUIRE(s.keep_nnd != nullptr, "profile was computed without keep_profiles");
        REQUIRE(len >= s.lmin && len <= s.lmax, "len outside [lmin, lmax]");
        cudaStream_t st = ctx->stream;
        const int64_t nl = s.n - len + 1, n0 = s.n0;
        const int M = s.m_max;
        std::vector<double> d((size_t)M * n0);
        std::vector<int32_t> j((size_t)M * n0);
        const size_t off = (size_t)(len - s.lmin) * M * n0;
        CK(cudaMemcpyAsync(d.data(), s.keep_nnd + off, d.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(j.data(), s.keep_nnj + off, j.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int64_t i = 0; i < nl; ++i) {
            if (mp) mp[i] = d[i];
            if (ip) ip[i] = j[i];
            for (int m = 0; m < M; ++m) {
                if (nnd) nnd[i * M + m] = d[(size_t)m * n0 + i];
                if (nnj) nnj[i * M + m] = j[(size_t)m * n0 + i];
            }
        }
    });
}

MAD_API mad_status mad_stats(mad_ctx *ctx, int32_t series, mad_length_stats *out, int32_t cap, int32_t *n_out)
{
    if (!ctx) { g_create_err = "ctx is NULL"; return MAD_EINVAL; }
    return run_guarded(ctx, [&] {
        Series &s = get_series(ctx, series);
        if (!s.profiled) {
            set_err(ctx, "mad_stats before mad_profile");
            throw Fail{MAD_ESTATE};
        }
        REQUIRE(n_out != nullptr && (out != nullptr || cap == 0), "output pointers are NULL");
        const int32_t nL = (int32_t)s.stats.size();
        for (int32_t i = 0; i < nL && i < cap; ++i) out[i] = s.stats[i];
        *n_out = nL;
    });
}

MAD_API const char *mad_last_error(const mad_ctx *ctx)
{
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

MAD_API void mad_destroy(mad_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (Series &s : ctx->series) {
        free_profile(s);
        if (s.own_x && s.x) cudaFree(s.x);
        s.x = nullptr;
        for (cudaEvent_t e : s.tev) cudaEventDestroy(e);
        for (cudaEvent_t e : s.sev)
            if (e) cudaEventDestroy(e);
        if (s.prep) cudaStreamDestroy(s.prep);
        if (s.disc) cudaStreamDestroy(s.disc);
        if (s.cap) cudaStreamDestroy(s.cap);
        if (s.rscratch) cudaFree(s.rscratch);
        if (s.hbuf) cudaFreeHost(s.hbuf);
    }
    delete ctx;
}

}  // extern "C"
