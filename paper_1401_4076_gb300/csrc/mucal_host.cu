// Host side of libmucal: the C ABI declared in include/mucal.h, device memory
// management, the acceptance-threshold build and the weight iteration of
// Sec. 2 in double precision.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mucal.h"
#include "mucal_internal.h"

using mucal::BlockWork;
using mucal::LaunchShape;
using mucal::SysParams;

namespace {

thread_local std::string g_init_error;

struct System {
    mucal_system_desc desc{};
    SysParams p{};                  // host copy holding device pointers
    std::vector<double> lnW;        // current log-weights over the window
    std::vector<uint8_t> visited;   // cumulative visited set (recursion memory)
    std::vector<double> pacc;       // accumulated pair weights (recursion memory)
    std::vector<int64_t> H;         // last summed histogram, host copy
    bool hist_on_host = false;
    int32_t t_lo = 0, t_hi = 0;     // target window (bins), -1 = default
    bool target_default = true;
    uint32_t *thr_pinned = nullptr; // staging buffer of the threshold upload
    size_t thr_count = 0;
    uint64_t last_attempts = 0;
    std::vector<double> lnW_run;    // the weights of the last iteration's thresholds
    unsigned long long *drop_acc = nullptr;  // device [3][n_bins] droplet accumulators
    int32_t *drop_last = nullptr;            // device [n_walkers] V_D of the last measurement
};

struct Context {
    int device = -1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint32_t flags = 0;
    std::vector<System> sys;
    SysParams *d_sys = nullptr;
    BlockWork *d_work = nullptr;
    int n_blocks = 0;
    int max_smem = 0;
    LaunchShape shape{};
    cudaEvent_t ev_it0 = nullptr, ev_k0 = nullptr, ev_k1 = nullptr, ev_it1 = nullptr;
    bool ran = false;
    uint64_t sweeps_last = 0;
    uint64_t launches = 0;
    int *d_drop_err = nullptr;           // droplet labelling failure flag
    uint32_t *drop_scratch = nullptr;    // global parent arrays for lattices too large for smem
    size_t drop_scratch_words = 0;
    bool measured = false;
    bool tunnel = false;                 // walker kernels with tunnelling bookkeeping
    int *d_next_item = nullptr;          // work-item counter of persistent launches
    unsigned int *d_walk_err = nullptr;  // set by a walker kernel whose bounded wait ran out
    // CUDA-graph mode: one graph per (sweeps, launch shape, flavour, grid)
    bool graph_mode = false;
    cudaGraph_t graph = nullptr;         // kept: its nodes address the executable's
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraphNode_t graph_walker = nullptr;  // the walker-update node (iteration changes)
    cudaKernelNodeParams graph_kp{};
    uint64_t graph_sweeps = 0;
    LaunchShape graph_shape{};
    bool graph_tunnel = false;
    int graph_grid = 0;
    uint32_t *d_xthr = nullptr;          // replica-exchange thresholds, [pairs][2 n_bins - 1]
    uint32_t *xthr_pinned = nullptr;     // their host staging buffer
    size_t xthr_words = 0;
    unsigned long long *d_xacc = nullptr;  // accepted exchanges per pair
    std::string err;
};

int fail(Context *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_init_error = buf;
    return code;
}

#define CUDA_TRY(ctx, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? MUCAL_ERR_OOM : MUCAL_ERR_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// ---------------------------------------------------------------------------
// Acceptance thresholds: min(1, W(E_n)/W(E_o)) of Sec. 2 as a uint32 per
// (E_o bin, dE).  Double precision, host libm exp; the device only compares.
// ---------------------------------------------------------------------------
void build_thresholds(const System &s, uint32_t *T)
{
    const int nb = s.p.n_bins;
    const int width = s.p.width;
    const int half = 2 * s.p.d;
    for (int b = 0; b < nb; ++b) {
        const double from = s.lnW[b];
        uint32_t *row = T + (size_t)b * s.p.tstride;
        for (int j = width; j < s.p.tstride; ++j) row[j] = 0u;   // row padding, never read
        for (int j = 0; j < width; ++j) {
            const int to = b + (j - half);
            if (to < 0 || to >= nb) {
                row[j] = 0u;
                continue;
            }
            const double diff = s.lnW[to] - from;
            if (diff >= 0.0) {
                row[j] = 0xFFFFFFFFu;
                continue;
            }
            const double scaled = std::floor(std::ldexp(std::exp(diff), 32));
            row[j] = scaled >= 4294967294.0 ? 0xFFFFFFFEu : (uint32_t)scaled;
        }
    }
}

int upload_thresholds(Context *c, System &s)
{
    // The pinned staging buffer may still feed an earlier asynchronous copy.
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    build_thresholds(s, s.thr_pinned);
    CUDA_TRY(c, cudaMemcpyAsync((void *)s.p.thr, s.thr_pinned, s.thr_count * sizeof(uint32_t),
                                cudaMemcpyHostToDevice, c->stream));
    return MUCAL_OK;
}

void normalise_max_zero(double *w, int n)
{
    double mx = -INFINITY;
    for (int b = 0; b < n; ++b) mx = std::max(mx, w[b]);
    for (int b = 0; b < n; ++b) w[b] -= mx;
}

// W^{i+1} = W^i / H^i where H^i > 0 (Sec. 2), in logs.
void simple_step(int nb, const int64_t *H, double *lnW, uint8_t *visited)
{
    for (int b = 0; b < nb; ++b) {
        if (H[b] > 0) {
            visited[b] = 1;
            lnW[b] -= std::log((double)H[b]);
        }
    }
    normalise_max_zero(lnW, nb);
}

// Accumulated-statistics recursion on consecutive members of the cumulative
// visited set (the recursive scheme cited in Sec. 2).
void recursive_step(int nb, const int64_t *H, double *w, uint8_t *visited, double *pacc)
{
    for (int b = 0; b < nb; ++b)
        if (H[b] > 0) visited[b] = 1;
    std::vector<int> mem;
    mem.reserve(nb);
    for (int b = 0; b < nb; ++b)
        if (visited[b]) mem.push_back(b);
    if (mem.empty()) {
        normalise_max_zero(w, nb);
        return;
    }
    const std::vector<double> old(w, w + nb);
    // rebuild from the top member downwards
    for (size_t j = mem.size() - 1; j >= 1; --j) {
        const int hi = mem[j], lo = mem[j - 1];
        double lnr = old[hi] - old[lo];
        const double hlo = (double)H[lo], hhi = (double)H[hi];
        const double g = (hlo > 0.0 && hhi > 0.0) ? hlo * hhi / (hlo + hhi) : 0.0;
        pacc[hi] += g;
        if (g > 0.0) lnr += (g / pacc[hi]) * (std::log(hlo) - std::log(hhi));
        w[lo] = w[hi] - lnr;
    }
    // bins outside the visited set ride with the nearest member above
    // (or the top member when none is above)
    int next_member = -1;
    for (int b = nb - 1; b >= 0; --b) {
        if (visited[b]) {
            next_member = b;
            continue;
        }
        const int ref = next_member >= 0 ? next_member : mem.back();
        w[b] = old[b] + (w[ref] - old[ref]);
    }
    normalise_max_zero(w, nb);
}

// Edge continuation of the weights (MUCAL_SCHEME_EXTRAPOLATE): bins below
// the lowest visited bin and above the highest take lnW continued linearly
// with the slope between that edge and the kEdgeMembers-th visited bin
// counted inwards (canonical weights at the sampled edge's microcanonical
// temperature), so that walkers keep moving into the unsampled range.
constexpr int kEdgeMembers = 8;

void extrapolate_edges(int nb, double *w, const uint8_t *visited)
{
    std::vector<int> mem;
    for (int b = 0; b < nb; ++b)
        if (visited[b]) mem.push_back(b);
    if (mem.size() >= 2) {
        const size_t k = std::min<size_t>(kEdgeMembers, mem.size() - 1);
        const int first = mem.front(), last = mem.back();
        const int in_lo = mem[k], in_hi = mem[mem.size() - 1 - k];
        const double slope_lo = (w[in_lo] - w[first]) / (double)(in_lo - first);
        const double slope_hi = (w[last] - w[in_hi]) / (double)(last - in_hi);
        for (int b = 0; b < first; ++b) w[b] = w[first] + slope_lo * (double)(b - first);
        for (int b = last + 1; b < nb; ++b) w[b] = w[last] + slope_hi * (double)(b - last);
    }
    normalise_max_zero(w, nb);
}

// One weight update: the simple or the recursive step, then (flag) the edge
// continuation.
void update_step(int scheme, int nb, const int64_t *H, double *lnW, uint8_t *visited, double *pacc)
{
    if ((scheme & 0xF) == MUCAL_SCHEME_SIMPLE)
        simple_step(nb, H, lnW, visited);
    else
        recursive_step(nb, H, lnW, visited, pacc);
    if (scheme & MUCAL_SCHEME_EXTRAPOLATE) extrapolate_edges(nb, lnW, visited);
}

bool scheme_ok(int scheme)
{
    const int base = scheme & 0xF;
    return (base == MUCAL_SCHEME_SIMPLE || base == MUCAL_SCHEME_RECURSIVE) &&
           (scheme & ~(0xF | MUCAL_SCHEME_EXTRAPOLATE)) == 0;
}

// min/max of H over the visited bins of the target window [lo, hi] (bins;
// lo < 0 selects the visited range), -1 while an end of it is unvisited.
double flatness_of(int nb, const int64_t *H, const uint8_t *visited, int t_lo, int t_hi)
{
    int first = -1, last = -1;
    for (int b = 0; b < nb; ++b)
        if (visited[b]) {
            if (first < 0) first = b;
            last = b;
        }
    if (first < 0) return -1.0;
    const int lo = t_lo < 0 ? first : t_lo;
    const int hi = t_lo < 0 ? last : t_hi;
    if (!visited[lo] || !visited[hi]) return -1.0;
    double mn = INFINITY, mx = 0.0;
    for (int b = lo; b <= hi; ++b) {
        if (!visited[b]) continue;
        const double h = (double)H[b];
        mn = std::min(mn, h);
        mx = std::max(mx, h);
    }
    return mx > 0.0 ? mn / mx : 0.0;
}

double flatness(const System &s)
{
    return flatness_of(s.p.n_bins, s.H.data(), s.visited.data(), s.target_default ? -1 : s.t_lo,
                       s.t_hi);
}

int check_desc(const mucal_system_desc &d, int i)
{
    if (d.d != 2 && d.d != 3) return fail(nullptr, MUCAL_ERR_INVALID_ARG, "system %d: d must be 2 or 3", i);
    if (d.L < 3 || d.L > 4096) return fail(nullptr, MUCAL_ERR_INVALID_ARG, "system %d: L must be in [3, 4096]", i);
    const uint64_t V = d.d == 2 ? (uint64_t)d.L * d.L : (uint64_t)d.L * d.L * d.L;
    if (V > (1u << 24) || V * (uint64_t)d.L >= (1ull << 32))
        return fail(nullptr, MUCAL_ERR_INVALID_ARG, "system %d: lattice too large", i);
    if (d.N <= 0 || (uint64_t)d.N >= V)
        return fail(nullptr, MUCAL_ERR_INVALID_ARG, "system %d: need 0 < N < L^d", i);
    if (d.n_walkers <= 0) return fail(nullptr, MUCAL_ERR_INVALID_ARG, "system %d: n_walkers must be > 0", i);
    if (!(d.e_lo == 0 && d.e_hi == 0)) {
        if (d.e_lo < -d.d * d.N || d.e_hi > 0 || d.e_lo >= d.e_hi)
            return fail(nullptr, MUCAL_ERR_INVALID_ARG,
                        "system %d: window must satisfy -dN <= e_lo < e_hi <= 0", i);
    }
    return MUCAL_OK;
}

void free_system(System &s)
{
    cudaFree(s.p.bits);
    cudaFree(s.p.S);
    cudaFree(s.p.E);
    cudaFree(s.p.hist);
    cudaFree((void *)s.p.thr);
    cudaFree(s.p.accepts);
    cudaFree(s.p.H);
    if (s.thr_pinned) cudaFreeHost(s.thr_pinned);
    cudaFree(s.drop_acc);
    cudaFree(s.drop_last);
    cudaFree(s.p.tun_state);
    cudaFree(s.p.tun_count);
    s.p = SysParams{};
    s.thr_pinned = nullptr;
    s.drop_acc = nullptr;
    s.drop_last = nullptr;
}

void destroy_context(Context *c)
{
    if (!c) return;
    if (c->device >= 0) cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &s : c->sys) free_system(s);
    cudaFree(c->d_sys);
    cudaFree(c->d_work);
    cudaFree(c->d_drop_err);
    cudaFree(c->drop_scratch);
    cudaFree(c->d_xthr);
    cudaFree(c->d_xacc);
    if (c->xthr_pinned) cudaFreeHost(c->xthr_pinned);
    cudaFree(c->d_next_item);
    cudaFree(c->d_walk_err);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->ev_it0) cudaEventDestroy(c->ev_it0);
    if (c->ev_k0) cudaEventDestroy(c->ev_k0);
    if (c->ev_k1) cudaEventDestroy(c->ev_k1);
    if (c->ev_it1) cudaEventDestroy(c->ev_it1);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// Shared memory a block of the given shape needs for system p.
size_t smem_for(const LaunchShape &sh, const SysParams &p)
{
    size_t bytes = 0;
    if (sh.thr_in_smem) bytes += mucal::thr_smem_words(p) * sizeof(uint32_t);
    if (sh.kernel == MUCAL_KERNEL_FIELD)
        bytes += (size_t)sh.walkers_per_block * mucal::field_smem_bytes(p);
    else if (sh.bits_in_smem)
        bytes += (size_t)sh.walkers_per_block * (size_t)p.words * sizeof(uint32_t);
    // the windows start on the next 16-byte boundary behind the bitsets or fields
    if (!sh.thr_in_smem && sh.thr_window && sh.kernel != MUCAL_KERNEL_THREAD)
        bytes += 16 + (size_t)sh.walkers_per_block * mucal::thr_window_bytes(p);
    return bytes;
}

// Split every system's walkers into blocks of the launch shape; order the
// blocks by decreasing cost (attempts per walker grow with N) so the longest
// blocks start first when systems of uneven size share one launch.
int build_work(Context *c, const LaunchShape &sh)
{
    std::vector<BlockWork> work;
    std::vector<int32_t> rows_of(c->sys.size(), 0);
    const bool per_walker = (c->flags & MUCAL_FLAG_PER_WALKER_HIST) != 0;
    for (int s = 0; s < (int)c->sys.size(); ++s) {
        const SysParams &p = c->sys[s].p;
        int rows = 0;
        for (int w0 = 0; w0 < p.n_walkers; w0 += sh.walkers_per_block) {
            BlockWork bw{};
            bw.sys = s;
            bw.walker0 = w0;
            bw.count = std::min(sh.walkers_per_block, p.n_walkers - w0);
            bw.hist_row = per_walker ? -1 : rows;
            ++rows;
            work.push_back(bw);
        }
        // blocks never outnumber walkers, so the per-walker allocation holds them
        rows_of[s] = per_walker ? p.n_walkers : rows;
    }
    std::stable_sort(work.begin(), work.end(), [&](const BlockWork &a, const BlockWork &b) {
        const double ca = (double)c->sys[a.sys].p.N * c->sys[a.sys].p.d;
        const double cb = (double)c->sys[b.sys].p.N * c->sys[b.sys].p.d;
        return ca > cb;
    });
    // build the new tables completely before replacing the old ones, so that
    // a failure leaves the previous launch shape usable
    BlockWork *d_work = nullptr;
    cudaError_t e = cudaMalloc(&d_work, std::max<size_t>(1, work.size()) * sizeof(BlockWork));
    if (e == cudaSuccess)
        e = cudaMemcpy(d_work, work.data(), work.size() * sizeof(BlockWork), cudaMemcpyHostToDevice);
    std::vector<SysParams> hp(c->sys.size());
    for (size_t i = 0; i < c->sys.size(); ++i) {
        hp[i] = c->sys[i].p;
        hp[i].hist_rows = rows_of[i];
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_sys, hp.data(), hp.size() * sizeof(SysParams), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_work);
        // restore the device table of the current shape
        std::vector<SysParams> cur(c->sys.size());
        for (size_t i = 0; i < c->sys.size(); ++i) cur[i] = c->sys[i].p;
        cudaMemcpy(c->d_sys, cur.data(), cur.size() * sizeof(SysParams), cudaMemcpyHostToDevice);
        return fail(c, e == cudaErrorMemoryAllocation ? MUCAL_ERR_OOM : MUCAL_ERR_CUDA,
                    "launch table upload failed: %s", cudaGetErrorString(e));
    }
    cudaFree(c->d_work);
    c->d_work = d_work;
    c->n_blocks = (int)work.size();
    for (size_t i = 0; i < c->sys.size(); ++i) c->sys[i].p.hist_rows = rows_of[i];
    return MUCAL_OK;
}

int apply_launch_config(Context *c, const mucal_launch_config &cfg)
{
    LaunchShape sh{};
    sh.kernel = cfg.kernel;
    sh.lanes = cfg.lanes_per_walker;
    sh.walkers_per_block = cfg.walkers_per_block;
    sh.bits_in_smem = cfg.bits_in_smem ? 1 : 0;
    sh.persistent = cfg.persistent ? 1 : 0;
    if (cfg.thr_window < 0 || cfg.thr_window > 2)
        return fail(c, MUCAL_ERR_INVALID_ARG, "thr_window must be 0, 1 or 2");
    sh.thr_window = cfg.kernel != MUCAL_KERNEL_THREAD ? cfg.thr_window : 0;
    if (cfg.multi_commit < 0 || cfg.multi_commit > 1)
        return fail(c, MUCAL_ERR_INVALID_ARG, "multi_commit must be 0 or 1");
    sh.multi_commit = cfg.kernel != MUCAL_KERNEL_THREAD && cfg.lanes_per_walker >= 4 ? cfg.multi_commit : 0;
    if (sh.kernel == MUCAL_KERNEL_THREAD) {
        if (sh.lanes != 1)
            return fail(c, MUCAL_ERR_INVALID_ARG, "THREAD kernel needs lanes_per_walker = 1");
        if (sh.walkers_per_block > 512)
            return fail(c, MUCAL_ERR_INVALID_ARG, "THREAD kernel blocks hold at most 512 threads");
    } else if (sh.kernel == MUCAL_KERNEL_GROUP || sh.kernel == MUCAL_KERNEL_FIELD) {
        const char *name = sh.kernel == MUCAL_KERNEL_GROUP ? "GROUP" : "FIELD";
        if (sh.lanes != 2 && sh.lanes != 4 && sh.lanes != 8 && sh.lanes != 16 && sh.lanes != 32)
            return fail(c, MUCAL_ERR_INVALID_ARG, "%s kernel needs lanes_per_walker in {2,4,8,16,32}", name);
        if ((sh.walkers_per_block * sh.lanes) % 32 != 0)
            return fail(c, MUCAL_ERR_INVALID_ARG, "%s kernel needs whole warps per block", name);
        if (sh.walkers_per_block * sh.lanes > 512)
            return fail(c, MUCAL_ERR_INVALID_ARG, "%s kernel blocks hold at most 512 threads", name);
        if (sh.kernel == MUCAL_KERNEL_FIELD && !sh.bits_in_smem)
            return fail(c, MUCAL_ERR_INVALID_ARG, "FIELD kernel keeps its counts in shared memory: "
                                                  "bits_in_smem must be 1");
    } else {
        return fail(c, MUCAL_ERR_INVALID_ARG, "unknown kernel %d", sh.kernel);
    }
    if (sh.walkers_per_block < 1 || sh.walkers_per_block * sh.lanes > 1024)
        return fail(c, MUCAL_ERR_INVALID_ARG, "walkers_per_block * lanes must be in [1, 1024]");
    // the threshold table joins the bitsets in shared memory whenever every
    // system's table fits next to its block of bitsets
    sh.thr_in_smem = 1;
    for (auto &s : c->sys)
        if (smem_for(sh, s.p) > (size_t)c->max_smem) sh.thr_in_smem = 0;
    if (cfg.thr_window == 2 && sh.thr_window) sh.thr_in_smem = 0;   // windows even if the table fits
    size_t smem = 0;
    for (auto &s : c->sys) smem = std::max(smem, smem_for(sh, s.p));
    if (smem > (size_t)c->max_smem && sh.thr_window) {
        // the threshold-row windows do not fit next to this block of walkers:
        // read the thresholds from global memory instead
        sh.thr_window = 0;
        smem = 0;
        for (auto &s : c->sys) smem = std::max(smem, smem_for(sh, s.p));
    }
    if (smem > (size_t)c->max_smem)
        return fail(c, MUCAL_ERR_INVALID_ARG, "launch needs %zu bytes of shared memory, limit %d",
                    smem, c->max_smem);
    if (!sh.thr_in_smem && sh.thr_window) sh.multi_commit = 0;   // rounds read row windows
    sh.smem_bytes = smem;
    int rc = build_work(c, sh);
    if (rc != MUCAL_OK) return rc;
    c->shape = sh;
    return MUCAL_OK;
}

Context *as_ctx(void *p) { return static_cast<Context *>(p); }

int check_sys(Context *c, int32_t s)
{
    if (!c) return MUCAL_ERR_INVALID_ARG;
    if (s < 0 || s >= (int32_t)c->sys.size())
        return fail(c, MUCAL_ERR_INVALID_ARG, "system index %d out of range", s);
    return MUCAL_OK;
}

int fetch_histogram(Context *c, System &s)
{
    if (!c->ran) return fail(c, MUCAL_ERR_NOT_READY, "no iteration has been run");
    if (!s.hist_on_host) {
        unsigned int err = 0;
        CUDA_TRY(c, cudaMemcpyAsync(s.H.data(), s.p.H, s.H.size() * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(&err, c->d_walk_err, sizeof err, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (err) {
            CUDA_TRY(c, cudaMemsetAsync(c->d_walk_err, 0, sizeof err, c->stream));
            return fail(c, MUCAL_ERR_STATE, "a walker kernel's wait for its threshold rows ran out "
                                            "(flag %u); the iteration's results are not valid", err);
        }
        s.hist_on_host = true;
    }
    return MUCAL_OK;
}

// Copy the host copies of every system's parameters to the device table,
// keeping the histogram rows of the current launch shape.
int upload_sys_table(Context *c)
{
    std::vector<SysParams> hp(c->sys.size());
    for (size_t i = 0; i < c->sys.size(); ++i) hp[i] = c->sys[i].p;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c, cudaMemcpy(c->d_sys, hp.data(), hp.size() * sizeof(SysParams), cudaMemcpyHostToDevice));
    return MUCAL_OK;
}

int reset_tunnel(Context *c, const System &s)
{
    CUDA_TRY(c, cudaMemsetAsync(s.p.tun_state, 0, (size_t)s.p.n_walkers, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(s.p.tun_count, 0, (size_t)s.p.n_walkers * 4, c->stream));
    return MUCAL_OK;
}

// The device work of one iteration, asynchronous on the context's stream:
// clear the histograms, the walker update, the histogram sums, with the
// timing events around them unless it is being captured into a graph (the
// graph launch is timed from outside instead).
int enqueue_iteration(Context *c, uint64_t sweeps, uint32_t iteration, int grid, bool events)
{
    if (events) CUDA_TRY(c, cudaEventRecord(c->ev_it0, c->stream));
    for (auto &s : c->sys) {
        CUDA_TRY(c, cudaMemsetAsync(s.p.hist, 0, (size_t)s.p.hist_rows * (size_t)s.p.n_bins * 8,
                                    c->stream));
        CUDA_TRY(c, cudaMemsetAsync(s.p.H, 0, (size_t)s.p.n_bins * 8, c->stream));
    }
    if (c->shape.persistent) CUDA_TRY(c, cudaMemsetAsync(c->d_next_item, 0, sizeof(int), c->stream));
    if (events) CUDA_TRY(c, cudaEventRecord(c->ev_k0, c->stream));
    CUDA_TRY(c, mucal::launch_walker_update(c->d_sys, c->d_work, c->n_blocks, c->shape, sweeps,
                                            iteration, c->tunnel, grid, c->d_next_item, c->stream));
    if (events) CUDA_TRY(c, cudaEventRecord(c->ev_k1, c->stream));
    std::vector<SysParams> hp(c->sys.size());
    for (size_t i = 0; i < c->sys.size(); ++i) hp[i] = c->sys[i].p;
    CUDA_TRY(c, mucal::launch_hist_reduce(hp.data(), c->d_sys, (int)hp.size(), c->stream));
    if (events) CUDA_TRY(c, cudaEventRecord(c->ev_it1, c->stream));
    return MUCAL_OK;
}

// Capture enqueue_iteration into a CUDA graph on the context's stream,
// instantiate it and remember its walker-update node.
void drop_graph(Context *c)
{
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_walker = nullptr;
}

int capture_iteration(Context *c, uint64_t sweeps, uint32_t iteration, int grid)
{
    drop_graph(c);
    CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_iteration(c, sweeps, iteration, grid, false);
    cudaGraph_t graph = nullptr;
    const cudaError_t end = cudaStreamEndCapture(c->stream, &graph);
    if (rc != MUCAL_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    CUDA_TRY(c, end);
    const void *fn = mucal::walker_update_fn(c->shape, c->tunnel);
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess) e = cudaGraphGetNodes(graph, nodes.data(), &n);
    for (size_t i = 0; e == cudaSuccess && i < n && !c->graph_walker; ++i) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[i], &t);
        if (e != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        e = cudaGraphKernelNodeGetParams(nodes[i], &kp);
        if (e == cudaSuccess && kp.func == fn) {
            c->graph_walker = nodes[i];
            c->graph_kp = kp;
        }
    }
    if (e == cudaSuccess && !c->graph_walker) e = cudaErrorInvalidValue;
    c->graph = graph;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
    if (e != cudaSuccess) {
        c->graph_exec = nullptr;
        drop_graph(c);
        return fail(c, MUCAL_ERR_CUDA, "iteration graph capture failed: %s", cudaGetErrorString(e));
    }
    c->graph_sweeps = sweeps;
    c->graph_shape = c->shape;
    c->graph_tunnel = c->tunnel;
    c->graph_grid = grid;
    return MUCAL_OK;
}

int check_droplet_error(Context *c)
{
    int flag = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&flag, c->d_drop_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (flag == 1) return fail(c, MUCAL_ERR_CUDA, "droplet labelling exceeded its iteration limit");
    if (flag == 2) return fail(c, MUCAL_ERR_CUDA, "droplet measurement met an energy outside the window");
    return MUCAL_OK;
}

}  // namespace

namespace mucal {
void set_init_error(const char *msg) { g_init_error = msg; }
}  // namespace mucal

extern "C" {

const char *mucal_version(void) { return "mucal 0.1 (sm_103a)"; }

const char *mucal_last_error(void *ctx)
{
    Context *c = as_ctx(ctx);
    return c ? c->err.c_str() : g_init_error.c_str();
}

int mucal_init_systems(void **out, const mucal_system_desc *sys, int32_t n_sys, void *cuda_stream,
                       uint32_t flags)
{
    if (!out) return fail(nullptr, MUCAL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!sys || n_sys <= 0) return fail(nullptr, MUCAL_ERR_INVALID_ARG, "need at least one system");
    for (int i = 0; i < n_sys; ++i) {
        int rc = check_desc(sys[i], i);
        if (rc != MUCAL_OK) return rc;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        return fail(nullptr, MUCAL_ERR_NO_DEVICE, "no CUDA device available");
    }
    Context *c = new (std::nothrow) Context();
    if (!c) return fail(nullptr, MUCAL_ERR_OOM, "host allocation failed");
    c->flags = flags;
    int rc = MUCAL_OK;
    auto bail = [&](int code) {
        if (c->err.size()) g_init_error = c->err;
        destroy_context(c);
        return code;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        c->device = -1;
        return bail(fail(nullptr, MUCAL_ERR_NO_DEVICE, "cudaGetDevice failed"));
    }
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(nullptr, MUCAL_ERR_CUDA, "stream creation failed"));
        c->own_stream = true;
    }
    if (mucal::walker_update_max_smem(&c->max_smem) != cudaSuccess)
        return bail(fail(nullptr, MUCAL_ERR_CUDA, "cannot query shared memory limit"));
    if (cudaEventCreate(&c->ev_it0) != cudaSuccess || cudaEventCreate(&c->ev_k0) != cudaSuccess ||
        cudaEventCreate(&c->ev_k1) != cudaSuccess || cudaEventCreate(&c->ev_it1) != cudaSuccess)
        return bail(fail(nullptr, MUCAL_ERR_CUDA, "event creation failed"));

    c->sys.resize(n_sys);
    for (int i = 0; i < n_sys; ++i) {
        System &s = c->sys[i];
        s.desc = sys[i];
        SysParams &p = s.p;
        p.d = sys[i].d;
        p.L = sys[i].L;
        p.N = sys[i].N;
        p.V = p.d == 2 ? p.L * p.L : p.L * p.L * p.L;
        p.L2 = p.L * p.L;
        if (sys[i].e_lo == 0 && sys[i].e_hi == 0) {
            p.e_lo = -p.d * p.N;
            s.desc.e_lo = p.e_lo;
            s.desc.e_hi = 0;
        } else {
            p.e_lo = sys[i].e_lo;
        }
        p.n_bins = s.desc.e_hi - p.e_lo + 1;
        p.width = 4 * p.d + 1;
        p.tstride = (p.width + 3) & ~3;
        p.words = (p.V + 31) / 32;
        p.idx16 = p.V <= 65536 ? 1 : 0;
        p.n_walkers = sys[i].n_walkers;
        p.hist_rows = p.n_walkers;
        p.magL = (uint32_t)(((1ull << 32) + (uint64_t)p.L - 1) / (uint64_t)p.L);
        p.seed_base = sys[i].seed_base;
        const size_t nw = (size_t)p.n_walkers;
        const size_t ib = p.idx16 ? 2 : 4;
        void *ptr = nullptr;
#define ALLOC(field, bytes)                                                         \
    do {                                                                            \
        cudaError_t e_ = cudaMalloc(&ptr, (bytes));                                 \
        if (e_ != cudaSuccess) {                                                    \
            cudaGetLastError();                                                     \
            return bail(fail(nullptr, MUCAL_ERR_OOM, "cudaMalloc of %zu bytes for " \
                             #field " failed", (size_t)(bytes)));                   \
        }                                                                           \
        p.field = decltype(p.field)(ptr);                                           \
    } while (0)
        ALLOC(bits, nw * p.words * sizeof(uint32_t));
        ALLOC(S, nw * (size_t)p.V * ib);
        ALLOC(E, nw * sizeof(int32_t));
        ALLOC(hist, nw * (size_t)p.n_bins * sizeof(unsigned long long));
        ALLOC(thr, (size_t)p.n_bins * p.tstride * sizeof(uint32_t));
        ALLOC(accepts, nw * sizeof(unsigned long long));
        ALLOC(H, (size_t)p.n_bins * sizeof(unsigned long long));
        ALLOC(tun_state, nw * sizeof(uint8_t));
        ALLOC(tun_count, nw * sizeof(uint32_t));
#undef ALLOC
        p.tun_lo = 0;                    // tunnelling ends: the window's ends
        p.tun_hi = p.n_bins - 1;
        s.thr_count = (size_t)p.n_bins * p.tstride;
        if (cudaMallocHost(&s.thr_pinned, s.thr_count * sizeof(uint32_t)) != cudaSuccess) {
            s.thr_pinned = nullptr;
            return bail(fail(nullptr, MUCAL_ERR_OOM, "pinned host allocation failed"));
        }
        s.lnW.assign(p.n_bins, 0.0);
        s.visited.assign(p.n_bins, 0);
        s.pacc.assign(p.n_bins, 0.0);
        s.H.assign(p.n_bins, 0);
        s.lnW_run.assign(p.n_bins, 0.0);
        if (cudaMalloc(&ptr, 3 * (size_t)p.n_bins * 8) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(nullptr, MUCAL_ERR_OOM, "cudaMalloc of droplet accumulators failed"));
        }
        s.drop_acc = static_cast<unsigned long long *>(ptr);
        if (cudaMalloc(&ptr, nw * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(nullptr, MUCAL_ERR_OOM, "cudaMalloc of droplet sizes failed"));
        }
        s.drop_last = static_cast<int32_t *>(ptr);
        if (cudaMemsetAsync(s.drop_acc, 0, 3 * (size_t)p.n_bins * 8, c->stream) != cudaSuccess ||
            cudaMemsetAsync(s.drop_last, 0, nw * sizeof(int32_t), c->stream) != cudaSuccess)
            return bail(fail(nullptr, MUCAL_ERR_CUDA, "memset failed"));
        if (cudaMemsetAsync(p.bits, 0, nw * p.words * sizeof(uint32_t), c->stream) != cudaSuccess ||
            cudaMemsetAsync(p.hist, 0, nw * (size_t)p.n_bins * 8, c->stream) != cudaSuccess ||
            cudaMemsetAsync(p.H, 0, (size_t)p.n_bins * 8, c->stream) != cudaSuccess ||
            cudaMemsetAsync(p.accepts, 0, nw * 8, c->stream) != cudaSuccess ||
            cudaMemsetAsync(p.tun_state, 0, nw, c->stream) != cudaSuccess ||
            cudaMemsetAsync(p.tun_count, 0, nw * 4, c->stream) != cudaSuccess)
            return bail(fail(nullptr, MUCAL_ERR_CUDA, "memset failed"));
    }
    if (cudaMalloc(&c->d_next_item, sizeof(int)) != cudaSuccess)
        return bail(fail(nullptr, MUCAL_ERR_OOM, "cudaMalloc of the work-item counter failed"));
    if (cudaMalloc(&c->d_walk_err, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemsetAsync(c->d_walk_err, 0, sizeof(unsigned int), c->stream) != cudaSuccess)
        return bail(fail(nullptr, MUCAL_ERR_OOM, "cudaMalloc of the walker error flag failed"));
    for (auto &s : c->sys) s.p.err = c->d_walk_err;
    if (cudaMalloc(&c->d_drop_err, sizeof(int)) != cudaSuccess ||
        cudaMemsetAsync(c->d_drop_err, 0, sizeof(int), c->stream) != cudaSuccess)
        return bail(fail(nullptr, MUCAL_ERR_OOM, "cudaMalloc of the droplet error flag failed"));
    if (cudaMalloc(&c->d_sys, n_sys * sizeof(SysParams)) != cudaSuccess)
        return bail(fail(nullptr, MUCAL_ERR_OOM, "cudaMalloc of system table failed"));
    std::vector<SysParams> hp(n_sys);
    for (int i = 0; i < n_sys; ++i) hp[i] = c->sys[i].p;
    if (cudaMemcpy(c->d_sys, hp.data(), n_sys * sizeof(SysParams), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(nullptr, MUCAL_ERR_CUDA, "copy of system table failed"));
    if (mucal::launch_fill_identity(hp.data(), c->d_sys, n_sys, c->stream) != cudaSuccess ||
        mucal::launch_init_walkers(hp.data(), c->d_sys, n_sys, c->stream) != cudaSuccess)
        return bail(fail(nullptr, MUCAL_ERR_CUDA, "initial placement launch failed"));
    for (int i = 0; i < n_sys; ++i) {
        rc = upload_thresholds(c, c->sys[i]);
        if (rc != MUCAL_OK) return bail(rc);
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
        return bail(fail(nullptr, MUCAL_ERR_CUDA, "initial placement failed: %s",
                         cudaGetErrorString(cudaGetLastError())));
    // user-given windows must contain every initial energy
    for (int i = 0; i < n_sys; ++i) {
        const System &s = c->sys[i];
        if (sys[i].e_lo == 0 && sys[i].e_hi == 0) continue;
        std::vector<int32_t> e(s.p.n_walkers);
        if (cudaMemcpy(e.data(), s.p.E, e.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return bail(fail(nullptr, MUCAL_ERR_CUDA, "energy read-back failed"));
        for (int32_t v : e)
            if (v < s.desc.e_lo || v > s.desc.e_hi)
                return bail(fail(nullptr, MUCAL_ERR_INVALID_ARG,
                                 "system %d: initial energy %d outside window [%d, %d]", i, v,
                                 s.desc.e_lo, s.desc.e_hi));
    }
    // default launch: the field kernel when every system's fields fit in
    // shared memory, else the group kernel with the bitsets in shared memory
    // when they fit, else in global memory (8 lanes, 16 walkers per block)
    mucal_launch_config def{MUCAL_KERNEL_FIELD, 8, 16, 1, 0, 1};
    for (auto &s : c->sys)
        if (smem_for(LaunchShape{MUCAL_KERNEL_FIELD, 8, 16, 1, 0, 0, 0}, s.p) > (size_t)c->max_smem)
            def.kernel = MUCAL_KERNEL_GROUP;
    if (def.kernel == MUCAL_KERNEL_GROUP)
        for (auto &s : c->sys)
            if (smem_for(LaunchShape{MUCAL_KERNEL_GROUP, 8, 16, 1, 0, 0, 0}, s.p) > (size_t)c->max_smem)
                def.bits_in_smem = 0;
    rc = apply_launch_config(c, def);
    if (rc != MUCAL_OK) return bail(rc);
    *out = c;
    return MUCAL_OK;
}

void mucal_destroy(void *ctx) { destroy_context(as_ctx(ctx)); }

int mucal_set_weights(void *ctx, int32_t sys, const double *lnW, int32_t n_bins)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    System &s = c->sys[sys];
    if (!lnW || n_bins != s.p.n_bins)
        return fail(c, MUCAL_ERR_INVALID_ARG, "lnW must hold n_bins = %d values", s.p.n_bins);
    for (int b = 0; b < n_bins; ++b)
        if (!std::isfinite(lnW[b])) return fail(c, MUCAL_ERR_INVALID_ARG, "lnW[%d] is not finite", b);
    s.lnW.assign(lnW, lnW + n_bins);
    std::fill(s.visited.begin(), s.visited.end(), 0);
    std::fill(s.pacc.begin(), s.pacc.end(), 0.0);
    CUDA_TRY(c, cudaSetDevice(c->device));
    return upload_thresholds(c, s);
}

int mucal_get_weights(void *ctx, int32_t sys, double *lnW_out, int32_t n_bins)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    const System &s = c->sys[sys];
    if (!lnW_out || n_bins != s.p.n_bins) return fail(c, MUCAL_ERR_INVALID_ARG, "bad lnW_out size");
    std::copy(s.lnW.begin(), s.lnW.end(), lnW_out);
    return MUCAL_OK;
}

int mucal_get_thresholds(void *ctx, int32_t sys, uint32_t *T, int64_t n)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    const System &s = c->sys[sys];
    if (!T || n != (int64_t)s.p.n_bins * s.p.width)
        return fail(c, MUCAL_ERR_INVALID_ARG, "bad threshold buffer size");
    CUDA_TRY(c, cudaSetDevice(c->device));
    // the device rows are padded to tstride words; the caller gets width per row
    CUDA_TRY(c, cudaMemcpy2DAsync(T, (size_t)s.p.width * 4, s.p.thr, (size_t)s.p.tstride * 4,
                                  (size_t)s.p.width * 4, (size_t)s.p.n_bins, cudaMemcpyDeviceToHost,
                                  c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return MUCAL_OK;
}

int mucal_set_launch_config(void *ctx, const mucal_launch_config *cfg)
{
    Context *c = as_ctx(ctx);
    if (!c || !cfg) return MUCAL_ERR_INVALID_ARG;
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return apply_launch_config(c, *cfg);
}

int mucal_get_launch_config(void *ctx, mucal_launch_config *cfg)
{
    Context *c = as_ctx(ctx);
    if (!c || !cfg) return MUCAL_ERR_INVALID_ARG;
    cfg->kernel = c->shape.kernel;
    cfg->lanes_per_walker = c->shape.lanes;
    cfg->walkers_per_block = c->shape.walkers_per_block;
    cfg->bits_in_smem = c->shape.bits_in_smem;
    cfg->persistent = c->shape.persistent;
    // with the whole table in shared memory the window setting has no effect
    cfg->thr_window = c->shape.thr_in_smem ? 0 : c->shape.thr_window;
    cfg->multi_commit = c->shape.multi_commit;
    return MUCAL_OK;
}

int mucal_set_graph_mode(void *ctx, int32_t enable)
{
    Context *c = as_ctx(ctx);
    if (!c) return MUCAL_ERR_INVALID_ARG;
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->graph_mode = enable != 0;
    drop_graph(c);
    return MUCAL_OK;
}

int mucal_run_iteration(void *ctx, int64_t sweeps, uint32_t iteration)
{
    Context *c = as_ctx(ctx);
    if (!c) return MUCAL_ERR_INVALID_ARG;
    if (sweeps < 1) return fail(c, MUCAL_ERR_INVALID_ARG, "sweeps must be >= 1");
    for (auto &s : c->sys)
        if ((uint64_t)sweeps * (uint64_t)s.p.N >= (1ull << 40))
            return fail(c, MUCAL_ERR_INVALID_ARG, "sweeps * N must be below 2^40");
    CUDA_TRY(c, cudaSetDevice(c->device));
    int grid = 0;
    CUDA_TRY(c, mucal::walker_update_grid(c->shape, c->tunnel, c->n_blocks, &grid));
    if (!c->graph_mode) {
        int rc = enqueue_iteration(c, (uint64_t)sweeps, iteration, grid, true);
        if (rc != MUCAL_OK) return rc;
    } else {
        const LaunchShape &a = c->shape, &b = c->graph_shape;
        const bool same = c->graph_exec && c->graph_sweeps == (uint64_t)sweeps &&
                          c->graph_tunnel == c->tunnel && c->graph_grid == grid &&
                          a.kernel == b.kernel && a.lanes == b.lanes &&
                          a.walkers_per_block == b.walkers_per_block &&
                          a.bits_in_smem == b.bits_in_smem && a.thr_in_smem == b.thr_in_smem &&
                          a.smem_bytes == b.smem_bytes && a.persistent == b.persistent &&
                          a.thr_window == b.thr_window && a.multi_commit == b.multi_commit;
        if (!same) {
            int rc = capture_iteration(c, (uint64_t)sweeps, iteration, grid);
            if (rc != MUCAL_OK) return rc;
        }
        // only the iteration number (the Philox counter word) changes
        uint64_t sw = (uint64_t)sweeps;
        int n_items = c->n_blocks;
        int *counter = c->shape.persistent ? c->d_next_item : nullptr;
        const SysParams *dsys = c->d_sys;
        const BlockWork *dwork = c->d_work;
        void *args[] = {(void *)&dsys, (void *)&dwork, (void *)&sw, (void *)&iteration,
                        (void *)&n_items, (void *)&counter};
        cudaKernelNodeParams kp = c->graph_kp;
        kp.kernelParams = args;
        kp.extra = nullptr;
        CUDA_TRY(c, cudaGraphExecKernelNodeSetParams(c->graph_exec, c->graph_walker, &kp));
        // the whole graph is timed: kernel_ms then includes the clears and sums
        CUDA_TRY(c, cudaEventRecord(c->ev_it0, c->stream));
        CUDA_TRY(c, cudaEventRecord(c->ev_k0, c->stream));
        CUDA_TRY(c, cudaGraphLaunch(c->graph_exec, c->stream));
        CUDA_TRY(c, cudaEventRecord(c->ev_k1, c->stream));
        CUDA_TRY(c, cudaEventRecord(c->ev_it1, c->stream));
    }
    for (auto &s : c->sys) {
        s.hist_on_host = false;
        s.last_attempts = (uint64_t)sweeps * (uint64_t)s.p.N * (uint64_t)s.p.n_walkers;
        s.lnW_run = s.lnW;
    }
    c->ran = true;
    c->sweeps_last = (uint64_t)sweeps;
    c->launches += 1;
    return MUCAL_OK;
}

int mucal_get_histogram(void *ctx, int32_t sys, int64_t *H, int32_t n_bins, int64_t *per_walker)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    System &s = c->sys[sys];
    if (!H || n_bins != s.p.n_bins) return fail(c, MUCAL_ERR_INVALID_ARG, "H must hold n_bins = %d", s.p.n_bins);
    if (per_walker && !(c->flags & MUCAL_FLAG_PER_WALKER_HIST))
        return fail(c, MUCAL_ERR_INVALID_ARG, "per-walker histograms need MUCAL_FLAG_PER_WALKER_HIST");
    CUDA_TRY(c, cudaSetDevice(c->device));
    rc = fetch_histogram(c, s);
    if (rc != MUCAL_OK) return rc;
    std::copy(s.H.begin(), s.H.end(), H);
    if (per_walker) {
        CUDA_TRY(c, cudaMemcpyAsync(per_walker, s.p.hist,
                                    (size_t)s.p.n_walkers * (size_t)s.p.n_bins * 8,
                                    cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    return MUCAL_OK;
}

int mucal_update_weights(void *ctx, int32_t sys, int32_t scheme, double *lnW_out, double *flatness_out)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    if (!scheme_ok(scheme)) return fail(c, MUCAL_ERR_INVALID_ARG, "unknown scheme %d", scheme);
    System &s = c->sys[sys];
    CUDA_TRY(c, cudaSetDevice(c->device));
    rc = fetch_histogram(c, s);
    if (rc != MUCAL_OK) return rc;
    update_step(scheme, s.p.n_bins, s.H.data(), s.lnW.data(), s.visited.data(), s.pacc.data());
    const double f = flatness(s);
    rc = upload_thresholds(c, s);
    if (rc != MUCAL_OK) return rc;
    if (lnW_out) std::copy(s.lnW.begin(), s.lnW.end(), lnW_out);
    if (flatness_out) *flatness_out = f;
    return MUCAL_OK;
}

int mucal_set_histogram(void *ctx, int32_t sys, const int64_t *H, int32_t n_bins)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    System &s = c->sys[sys];
    if (!H || n_bins != s.p.n_bins) return fail(c, MUCAL_ERR_INVALID_ARG, "H must hold n_bins = %d", s.p.n_bins);
    if (!c->ran) return fail(c, MUCAL_ERR_NOT_READY, "no iteration has been run");
    for (int b = 0; b < n_bins; ++b)
        if (H[b] < 0) return fail(c, MUCAL_ERR_INVALID_ARG, "H[%d] is negative", b);
    // the local histogram must not land on top of the given one later
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::copy(H, H + n_bins, s.H.begin());
    s.hist_on_host = true;
    return MUCAL_OK;
}

int mucal_get_launch_occupancy(void *ctx, int32_t *blocks_per_sm, int32_t *sm_count)
{
    Context *c = as_ctx(ctx);
    if (!c || !blocks_per_sm || !sm_count) return MUCAL_ERR_INVALID_ARG;
    CUDA_TRY(c, cudaSetDevice(c->device));
    const void *fn = mucal::walker_update_fn(c->shape, c->tunnel);
    if (!fn) return fail(c, MUCAL_ERR_INVALID_ARG, "no kernel for the current launch shape");
    int per_sm = 0, sms = 0;
    CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per_sm, fn, c->shape.walkers_per_block * c->shape.lanes, c->shape.smem_bytes));
    CUDA_TRY(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    *blocks_per_sm = per_sm;
    *sm_count = sms;
    return MUCAL_OK;
}

int mucal_weight_update(int32_t scheme, int32_t n_bins, const int64_t *H, double *lnW,
                        uint8_t *visited, double *pacc, int32_t t_lo, int32_t t_hi,
                        double *flatness_out)
{
    if (!scheme_ok(scheme)) return fail(nullptr, MUCAL_ERR_INVALID_ARG, "unknown scheme %d", scheme);
    if (n_bins < 1 || !H || !lnW || !visited || ((scheme & 0xF) == MUCAL_SCHEME_RECURSIVE && !pacc))
        return fail(nullptr, MUCAL_ERR_INVALID_ARG, "need n_bins >= 1 and H, lnW, visited (and pacc)");
    if (t_lo >= 0 && (t_hi < t_lo || t_hi >= n_bins))
        return fail(nullptr, MUCAL_ERR_INVALID_ARG, "target bins must satisfy 0 <= t_lo <= t_hi < n_bins");
    for (int b = 0; b < n_bins; ++b) {
        if (H[b] < 0) return fail(nullptr, MUCAL_ERR_INVALID_ARG, "H[%d] is negative", b);
        if (!std::isfinite(lnW[b])) return fail(nullptr, MUCAL_ERR_INVALID_ARG, "lnW[%d] is not finite", b);
    }
    update_step(scheme, n_bins, H, lnW, visited, pacc);
    if (flatness_out) *flatness_out = flatness_of(n_bins, H, visited, t_lo < 0 ? -1 : t_lo, t_hi);
    return MUCAL_OK;
}

int mucal_set_target_window(void *ctx, int32_t sys, int32_t t_lo, int32_t t_hi)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    System &s = c->sys[sys];
    if (t_lo == 0 && t_hi == 0) {
        s.target_default = true;
        return MUCAL_OK;
    }
    if (t_lo < s.desc.e_lo || t_hi > s.desc.e_hi || t_lo > t_hi)
        return fail(c, MUCAL_ERR_INVALID_ARG, "target window must lie inside [%d, %d]", s.desc.e_lo,
                    s.desc.e_hi);
    s.target_default = false;
    s.t_lo = t_lo - s.desc.e_lo;
    s.t_hi = t_hi - s.desc.e_lo;
    return MUCAL_OK;
}

int mucal_get_walker_state(void *ctx, int32_t sys, int32_t walker, uint8_t *occ, int32_t *S, int32_t *E)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    const System &s = c->sys[sys];
    const SysParams &p = s.p;
    if (walker < 0 || walker >= p.n_walkers) return fail(c, MUCAL_ERR_INVALID_ARG, "walker out of range");
    CUDA_TRY(c, cudaSetDevice(c->device));
    std::vector<uint32_t> bits(p.words);
    std::vector<uint8_t> sraw((size_t)p.V * (p.idx16 ? 2 : 4));
    int32_t e = 0;
    CUDA_TRY(c, cudaMemcpyAsync(bits.data(), p.bits + (size_t)walker * p.words, p.words * 4,
                                cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(sraw.data(), (const char *)p.S + (size_t)walker * sraw.size(),
                                sraw.size(), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(&e, p.E + walker, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (occ)
        for (int i = 0; i < p.V; ++i) occ[i] = (uint8_t)((bits[i >> 5] >> (i & 31)) & 1u);
    if (S) {
        for (int i = 0; i < p.V; ++i) {
            if (p.idx16)
                S[i] = ((const uint16_t *)sraw.data())[i];
            else
                S[i] = (int32_t)((const uint32_t *)sraw.data())[i];
        }
    }
    if (E) *E = e;
    return MUCAL_OK;
}

int mucal_get_system_info(void *ctx, int32_t sys, mucal_system_info *info)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    if (!info) return fail(c, MUCAL_ERR_INVALID_ARG, "info is NULL");
    const System &s = c->sys[sys];
    info->d = s.p.d;
    info->L = s.p.L;
    info->N = s.p.N;
    info->n_walkers = s.p.n_walkers;
    info->e_lo = s.desc.e_lo;
    info->e_hi = s.desc.e_hi;
    info->V = s.p.V;
    info->n_bins = s.p.n_bins;
    info->width = s.p.width;
    info->index_bytes = s.p.idx16 ? 2 : 4;
    info->seed_base = s.p.seed_base;
    return MUCAL_OK;
}

int mucal_get_stats(void *ctx, int32_t sys, mucal_stats *st)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    if (!st) return fail(c, MUCAL_ERR_INVALID_ARG, "stats is NULL");
    std::memset(st, 0, sizeof *st);
    st->walker_launches = c->launches;
    if (!c->ran) return MUCAL_OK;
    const System &s = c->sys[sys];
    CUDA_TRY(c, cudaSetDevice(c->device));
    std::vector<unsigned long long> acc(s.p.n_walkers);
    CUDA_TRY(c, cudaMemcpyAsync(acc.data(), s.p.accepts, acc.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (auto v : acc) st->accepts += v;
    st->attempts = s.last_attempts;
    float ms = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1));
    st->kernel_ms = ms;
    CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev_it0, c->ev_it1));
    st->iteration_ms = ms;
    return MUCAL_OK;
}

int mucal_histogram_device_ptr(void *ctx, int32_t sys, void **dptr)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    if (!dptr) return fail(c, MUCAL_ERR_INVALID_ARG, "dptr is NULL");
    *dptr = c->sys[sys].p.H;
    return MUCAL_OK;
}

int mucal_reweight_system(void *ctx, int32_t sys, const double *beta, int32_t n_beta,
                          const double *obs, int32_t n_obs, double *mean_E, double *mean_E2,
                          double *obs_out)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    System &s = c->sys[sys];
    CUDA_TRY(c, cudaSetDevice(c->device));
    rc = fetch_histogram(c, s);
    if (rc != MUCAL_OK) return rc;
    rc = mucal_reweight(s.H.data(), s.lnW_run.data(), s.p.n_bins, s.p.e_lo, beta, n_beta, obs, n_obs,
                        mean_E, mean_E2, obs_out);
    if (rc != MUCAL_OK) c->err = mucal_last_error(nullptr);
    return rc;
}

int mucal_set_tunnel_window(void *ctx, int32_t sys, int32_t e_min, int32_t e_max)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    System &s = c->sys[sys];
    if (e_min == 0 && e_max == 0) {
        e_min = s.desc.e_lo;
        e_max = s.desc.e_hi;
    }
    if (e_min < s.desc.e_lo || e_max > s.desc.e_hi || e_min >= e_max)
        return fail(c, MUCAL_ERR_INVALID_ARG, "tunnelling ends must satisfy %d <= e_min < e_max <= %d",
                    s.desc.e_lo, s.desc.e_hi);
    CUDA_TRY(c, cudaSetDevice(c->device));
    s.p.tun_lo = e_min - s.desc.e_lo;
    s.p.tun_hi = e_max - s.desc.e_lo;
    rc = upload_sys_table(c);
    if (rc != MUCAL_OK) return rc;
    c->tunnel = true;
    return reset_tunnel(c, s);
}

int mucal_get_tunnel_counts(void *ctx, int32_t sys, int64_t *total, uint32_t *per_walker,
                            uint8_t *state)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    const System &s = c->sys[sys];
    CUDA_TRY(c, cudaSetDevice(c->device));
    std::vector<uint32_t> cnt((size_t)s.p.n_walkers);
    CUDA_TRY(c, cudaMemcpyAsync(cnt.data(), s.p.tun_count, cnt.size() * 4, cudaMemcpyDeviceToHost,
                                c->stream));
    if (state)
        CUDA_TRY(c, cudaMemcpyAsync(state, s.p.tun_state, cnt.size(), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    int64_t sum = 0;
    for (uint32_t v : cnt) sum += v;
    if (total) *total = sum;
    if (per_walker) std::copy(cnt.begin(), cnt.end(), per_walker);
    return MUCAL_OK;
}

int mucal_reset_tunnel_counts(void *ctx)
{
    Context *c = as_ctx(ctx);
    if (!c) return MUCAL_ERR_INVALID_ARG;
    CUDA_TRY(c, cudaSetDevice(c->device));
    for (const System &s : c->sys) {
        const int rc = reset_tunnel(c, s);
        if (rc != MUCAL_OK) return rc;
    }
    return MUCAL_OK;
}

int mucal_replica_exchange(void *ctx, const double *beta, int32_t n_sys, uint32_t round,
                           int32_t parity, int64_t *accepted)
{
    Context *c = as_ctx(ctx);
    if (!c) return MUCAL_ERR_INVALID_ARG;
    if (!beta) return fail(c, MUCAL_ERR_INVALID_ARG, "beta is NULL");
    if (n_sys != (int32_t)c->sys.size() || n_sys < 2)
        return fail(c, MUCAL_ERR_INVALID_ARG, "n_sys must equal the context's %d systems (>= 2)",
                    (int)c->sys.size());
    if (parity != 0 && parity != 1) return fail(c, MUCAL_ERR_INVALID_ARG, "parity must be 0 or 1");
    const SysParams &p0 = c->sys[0].p;
    for (int k = 0; k < n_sys; ++k) {
        const SysParams &p = c->sys[k].p;
        if (p.d != p0.d || p.L != p0.L || p.N != p0.N || p.n_walkers != p0.n_walkers ||
            p.e_lo != p0.e_lo || p.n_bins != p0.n_bins)
            return fail(c, MUCAL_ERR_INVALID_ARG, "system %d differs from system 0: a tempering "
                        "ladder needs copies of one lattice, walker count and window", k);
        if (!std::isfinite(beta[k])) return fail(c, MUCAL_ERR_INVALID_ARG, "beta[%d] is not finite", k);
    }
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int nb = p0.n_bins;
    const int width = 2 * nb - 1;
    const int pairs = n_sys - 1;
    const size_t words = (size_t)pairs * (size_t)width;
    if (words > c->xthr_words) {
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        cudaFree(c->d_xthr);
        cudaFree(c->d_xacc);
        if (c->xthr_pinned) cudaFreeHost(c->xthr_pinned);
        c->d_xthr = nullptr;
        c->d_xacc = nullptr;
        c->xthr_pinned = nullptr;
        c->xthr_words = 0;
        CUDA_TRY(c, cudaMalloc(&c->d_xthr, words * sizeof(uint32_t)));
        CUDA_TRY(c, cudaMalloc(&c->d_xacc, (size_t)pairs * sizeof(unsigned long long)));
        CUDA_TRY(c, cudaMallocHost(&c->xthr_pinned, words * sizeof(uint32_t)));
        c->xthr_words = words;
    }
    // the staging buffer may still feed the previous exchange's upload
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < pairs; ++k) {
        const double db = beta[k] - beta[k + 1];
        uint32_t *row = c->xthr_pinned + (size_t)k * width;
        for (int j = 0; j < width; ++j) {
            const double x = db * (double)(j - (nb - 1));   // (beta_k - beta_k+1)(E_k - E_k+1)
            if (x >= 0.0) {
                row[j] = 0xFFFFFFFFu;
                continue;
            }
            const double scaled = std::floor(std::ldexp(std::exp(x), 32));
            row[j] = scaled >= 4294967294.0 ? 0xFFFFFFFEu : (uint32_t)scaled;
        }
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_xthr, c->xthr_pinned, words * sizeof(uint32_t),
                                cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->d_xacc, 0, (size_t)pairs * sizeof(unsigned long long), c->stream));
    CUDA_TRY(c, mucal::launch_exchange(c->d_sys, n_sys, p0.n_walkers, parity, round, c->d_xthr, width,
                                       c->d_xacc, c->stream));
    if (accepted) {
        CUDA_TRY(c, cudaMemcpyAsync(accepted, c->d_xacc, (size_t)pairs * 8, cudaMemcpyDeviceToHost,
                                    c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    return MUCAL_OK;
}

int mucal_measure_droplets(void *ctx)
{
    Context *c = as_ctx(ctx);
    if (!c) return MUCAL_ERR_INVALID_ARG;
    CUDA_TRY(c, cudaSetDevice(c->device));
    std::vector<mucal::DropletPlan> plans(c->sys.size());
    size_t scratch = 0;
    for (size_t i = 0; i < c->sys.size(); ++i) {
        CUDA_TRY(c, mucal::droplet_plan(c->sys[i].p, &plans[i]));
        scratch = std::max(scratch, plans[i].scratch_words);
    }
    if (scratch > c->drop_scratch_words) {
        // the previous scratch may still be read by an earlier measurement
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        cudaFree(c->drop_scratch);
        c->drop_scratch = nullptr;
        c->drop_scratch_words = 0;
        CUDA_TRY(c, cudaMalloc(&c->drop_scratch, scratch * sizeof(uint32_t)));
        c->drop_scratch_words = scratch;
    }
    for (size_t i = 0; i < c->sys.size(); ++i) {
        const System &s = c->sys[i];
        const mucal::DropletOut o{s.drop_acc, s.drop_last, c->d_drop_err};
        CUDA_TRY(c, mucal::launch_droplets(s.p, o, plans[i], c->drop_scratch, c->stream));
    }
    c->measured = true;
    return MUCAL_OK;
}

int mucal_get_droplet_stats(void *ctx, int32_t sys, int64_t *count, int64_t *sum, int64_t *sum2,
                            int32_t n_bins)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    const System &s = c->sys[sys];
    if (n_bins != s.p.n_bins) return fail(c, MUCAL_ERR_INVALID_ARG, "n_bins must be %d", s.p.n_bins);
    if (!c->measured) return fail(c, MUCAL_ERR_NOT_READY, "no droplet measurement yet");
    CUDA_TRY(c, cudaSetDevice(c->device));
    rc = check_droplet_error(c);
    if (rc != MUCAL_OK) return rc;
    int64_t *dst[3] = {count, sum, sum2};
    for (int k = 0; k < 3; ++k)
        if (dst[k])
            CUDA_TRY(c, cudaMemcpyAsync(dst[k], s.drop_acc + (size_t)k * s.p.n_bins,
                                        (size_t)s.p.n_bins * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return MUCAL_OK;
}

int mucal_get_largest_droplets(void *ctx, int32_t sys, int32_t *V_D, int32_t n_walkers)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    const System &s = c->sys[sys];
    if (!V_D || n_walkers != s.p.n_walkers)
        return fail(c, MUCAL_ERR_INVALID_ARG, "V_D must hold n_walkers = %d", s.p.n_walkers);
    if (!c->measured) return fail(c, MUCAL_ERR_NOT_READY, "no droplet measurement yet");
    CUDA_TRY(c, cudaSetDevice(c->device));
    rc = check_droplet_error(c);
    if (rc != MUCAL_OK) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(V_D, s.drop_last, (size_t)n_walkers * 4, cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return MUCAL_OK;
}

int mucal_reset_droplet_stats(void *ctx)
{
    Context *c = as_ctx(ctx);
    if (!c) return MUCAL_ERR_INVALID_ARG;
    CUDA_TRY(c, cudaSetDevice(c->device));
    for (const System &s : c->sys)
        CUDA_TRY(c, cudaMemsetAsync(s.drop_acc, 0, 3 * (size_t)s.p.n_bins * 8, c->stream));
    return MUCAL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoint / resume.  Random numbers are counter-based (seed, iteration,
// attempt), so a restored system continues bit-for-bit.
// ---------------------------------------------------------------------------
namespace {

struct CheckpointHeader {
    char magic[8];          // "MUCALCK1"
    int32_t d, L, N, n_walkers, e_lo, e_hi;
    uint64_t seed_base;
    int32_t index_bytes, words, n_bins, target_default;
    int32_t t_lo, t_hi;
};

size_t checkpoint_bytes(const System &s)
{
    const SysParams &p = s.p;
    const size_t nw = (size_t)p.n_walkers;
    return sizeof(CheckpointHeader) + nw * p.words * 4 + nw * (size_t)p.V * (p.idx16 ? 2 : 4) +
           nw * 4 + (size_t)p.n_bins * (8 + 1 + 8);
}

}  // namespace

extern "C" {

int mucal_checkpoint_size(void *ctx, int32_t sys, int64_t *bytes)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    if (!bytes) return fail(c, MUCAL_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = (int64_t)checkpoint_bytes(c->sys[sys]);
    return MUCAL_OK;
}

int mucal_checkpoint_save(void *ctx, int32_t sys, void *buf, int64_t bytes)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    const System &s = c->sys[sys];
    const SysParams &p = s.p;
    if (!buf || bytes != (int64_t)checkpoint_bytes(s))
        return fail(c, MUCAL_ERR_INVALID_ARG, "checkpoint buffer must hold %zu bytes", checkpoint_bytes(s));
    CUDA_TRY(c, cudaSetDevice(c->device));
    char *o = static_cast<char *>(buf);
    CheckpointHeader h{};
    std::memcpy(h.magic, "MUCALCK1", 8);
    h.d = p.d; h.L = p.L; h.N = p.N; h.n_walkers = p.n_walkers;
    h.e_lo = s.desc.e_lo; h.e_hi = s.desc.e_hi; h.seed_base = p.seed_base;
    h.index_bytes = p.idx16 ? 2 : 4; h.words = p.words; h.n_bins = p.n_bins;
    h.target_default = s.target_default ? 1 : 0; h.t_lo = s.t_lo; h.t_hi = s.t_hi;
    std::memcpy(o, &h, sizeof h);
    o += sizeof h;
    const size_t nw = (size_t)p.n_walkers;
    const size_t b_bits = nw * p.words * 4, b_S = nw * (size_t)p.V * (p.idx16 ? 2 : 4), b_E = nw * 4;
    CUDA_TRY(c, cudaMemcpyAsync(o, p.bits, b_bits, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(o + b_bits, p.S, b_S, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(o + b_bits + b_S, p.E, b_E, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    o += b_bits + b_S + b_E;
    std::memcpy(o, s.lnW.data(), (size_t)p.n_bins * 8);
    o += (size_t)p.n_bins * 8;
    std::memcpy(o, s.visited.data(), (size_t)p.n_bins);
    o += p.n_bins;
    std::memcpy(o, s.pacc.data(), (size_t)p.n_bins * 8);
    return MUCAL_OK;
}

int mucal_checkpoint_load(void *ctx, int32_t sys, const void *buf, int64_t bytes)
{
    Context *c = as_ctx(ctx);
    int rc = check_sys(c, sys);
    if (rc != MUCAL_OK) return rc;
    System &s = c->sys[sys];
    const SysParams &p = s.p;
    if (!buf || bytes != (int64_t)checkpoint_bytes(s))
        return fail(c, MUCAL_ERR_INVALID_ARG, "checkpoint must hold %zu bytes", checkpoint_bytes(s));
    const char *in = static_cast<const char *>(buf);
    CheckpointHeader h;
    std::memcpy(&h, in, sizeof h);
    if (std::memcmp(h.magic, "MUCALCK1", 8) != 0 || h.d != p.d || h.L != p.L || h.N != p.N ||
        h.n_walkers != p.n_walkers || h.e_lo != s.desc.e_lo || h.e_hi != s.desc.e_hi ||
        h.seed_base != p.seed_base || h.index_bytes != (p.idx16 ? 2 : 4) || h.words != p.words ||
        h.n_bins != p.n_bins)
        return fail(c, MUCAL_ERR_INVALID_ARG, "checkpoint does not belong to system %d", sys);
    const size_t nw = (size_t)p.n_walkers;
    const size_t b_bits = nw * p.words * 4, b_S = nw * (size_t)p.V * (p.idx16 ? 2 : 4), b_E = nw * 4;
    const char *bits = in + sizeof h;
    const char *S = bits + b_bits;
    const char *E = S + b_S;
    const char *w = E + b_E;
    // validate before touching the device: energies inside the window, list
    // entries on the lattice, finite weights
    for (size_t i = 0; i < nw; ++i) {
        int32_t e;
        std::memcpy(&e, E + 4 * i, 4);
        if (e < s.desc.e_lo || e > s.desc.e_hi)
            return fail(c, MUCAL_ERR_INVALID_ARG, "checkpoint energy of walker %zu outside the window", i);
    }
    for (size_t i = 0; i < nw * (size_t)p.V; ++i) {
        uint32_t v;
        if (p.idx16) {
            uint16_t x;
            std::memcpy(&x, S + 2 * i, 2);
            v = x;
        } else {
            std::memcpy(&v, S + 4 * i, 4);
        }
        if (v >= (uint32_t)p.V) return fail(c, MUCAL_ERR_INVALID_ARG, "checkpoint list entry %zu is not a site", i);
    }
    std::vector<double> lnW((size_t)p.n_bins);
    std::memcpy(lnW.data(), w, (size_t)p.n_bins * 8);
    for (double x : lnW)
        if (!std::isfinite(x)) return fail(c, MUCAL_ERR_INVALID_ARG, "checkpoint weight is not finite");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(p.bits, bits, b_bits, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(p.S, S, b_S, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(p.E, E, b_E, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    s.lnW = lnW;
    std::memcpy(s.visited.data(), w + (size_t)p.n_bins * 8, (size_t)p.n_bins);
    std::memcpy(s.pacc.data(), w + (size_t)p.n_bins * 9, (size_t)p.n_bins * 8);
    s.target_default = h.target_default != 0;
    s.t_lo = h.t_lo;
    s.t_hi = h.t_hi;
    s.hist_on_host = false;
    rc = reset_tunnel(c, s);   // tunnelling is counted afresh after a restore
    if (rc != MUCAL_OK) return rc;
    return upload_thresholds(c, s);
}

}  // extern "C"
