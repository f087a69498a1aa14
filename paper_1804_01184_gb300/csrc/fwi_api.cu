// fwi_api.cu -- host side of libfwi.so: argument checks, workspace plans, time loops.
// The C ABI is declared in include/fwi.h.  Every arithmetic step of the method runs in the
// kernels of fwi_kernels.cuh; this file only plans memory and orders launches.
#include <cuda.h>          // CUtensorMap and its enums (the encoder is looked up at run time)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/fwi.h"
#include "fwi_kernels.cuh"
#include "fwi_stream.cuh"
#include "fwi_warp.cuh"

namespace {

thread_local std::string g_err;
thread_local long long g_launches = 0;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// Optional per-launch timing: an event pair on the launching stream around every kernel,
// harvested by fwi_profile_report() after the caller has synchronised.
struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> ev;     // pairs, reused between reports
    std::vector<int> kind;           // kernel id of pair k
    size_t used = 0;                 // pairs recorded since the last report
    std::map<std::string, int> ids;
    std::vector<std::string> names;

    int id(const char *name)
    {
        auto it = ids.find(name);
        if (it != ids.end()) return it->second;
        int k = (int)names.size();
        ids.emplace(name, k);
        names.emplace_back(name);
        return k;
    }
    int every = 1;                   // time one launch in `every` of each kernel
    std::vector<long long> seen;     // launches of kernel k since profiling was enabled
    // returns the event pair for the next launch, or nullptr if profiling is off (or this
    // launch is not sampled)
    cudaEvent_t *next(const char *name)
    {
        if (!on) return nullptr;
        std::lock_guard<std::mutex> lk(mu);
        const int k = id(name);
        if ((int)seen.size() <= k) seen.resize(k + 1, 0);
        if (seen[k]++ % every) return nullptr;
        if (2 * (used + 1) > ev.size()) {
            size_t add = std::max<size_t>(1024, ev.size());
            for (size_t k = 0; k < add; ++k) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
                ev.push_back(e);
            }
        }
        kind.resize(used + 1);
        kind[used] = k;
        return &ev[2 * used++];
    }
};
Profiler g_prof;

// Phase ranges for timeline tools (NVTX), on while fwi_trace(1): each marks the host thread's
// enqueueing of one phase of an operation; fwi_trace_report() counts the ranges opened.
enum Phase { PH_MODEL_BUILD, PH_FORWARD, PH_RECOMPUTE, PH_ADJOINT, PH_REDUCE, PH_BORN, PH_ENGINE, PH_COUNT };
const char *const kPhaseName[PH_COUNT] = {"fwi:model_build", "fwi:forward", "fwi:recompute", "fwi:adjoint",
                                          "fwi:reduce", "fwi:born", "fwi:engine_iteration"};
std::atomic<bool> g_trace{false};
std::atomic<long long> g_trace_count[PH_COUNT];

struct TraceRange {
    bool on;
    explicit TraceRange(Phase p) : on(g_trace.load(std::memory_order_relaxed))
    {
        if (!on) return;
        nvtxRangePushA(kPhaseName[p]);
        g_trace_count[p].fetch_add(1, std::memory_order_relaxed);
    }
    ~TraceRange()
    {
        if (on) nvtxRangePop();
    }
};

// Launch-shape overrides set by fwi_set_tile (0: built-in defaults); read when a plan is made.
int g_tile_tz = 0;
int g_tile_variant = 0;
// Checkpoint interval forced by fwi_set_checkpoint (0: the planner chooses).
int g_ckpt_every = 0;
// Adjoint steps whose gradient products accumulate in FP32 before they are flushed into the
// FP64 running sums (fwi_set_accumulation; 0: ACC_STEPS).
constexpr int ACC_STEPS = 64;
int g_acc_every = 0;

constexpr size_t ALIGN = 256;
constexpr int RED_BLOCKS = 264;   // misfit partial sums per shot group

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Plan {
    fwi::Dims d;
    fwi::Stencil st;
    int M = 0, ns = 0, nr = 0, nt = 0;
    int B = 0;        // shots per group
    int C = 0;        // steps per snapshot segment (== nt: whole history kept)
    int nseg = 1;     // segments
    int ngroups = 0;
    int tz = 0;       // rows per warp strip
    int variant = 0;  // kernel variant (register budget) chosen by the tuner
    int acc = ACC_STEPS;   // adjoint steps per FP32 accumulation chunk
    // byte offsets into the workspace
    size_t status = 0, K = 0, bx = 0, bz = 0, ax = 0, axh = 0, az = 0, azh = 0;
    size_t sidx = 0, sw = 0, ridx = 0, rw = 0, rl = 0;
    size_t p[2] = {0, 0}, vx[2] = {0, 0}, vz[2] = {0, 0};          // ping-pong state
    size_t dK = 0, dbx = 0, dbz = 0, dp[2] = {0, 0}, dvx[2] = {0, 0}, dvz[2] = {0, 0};
    size_t ap[2] = {0, 0}, avx[2] = {0, 0}, avz[2] = {0, 0};
    size_t accK = 0, accBx = 0, accBz = 0, snap = 0, ckpt = 0;
    size_t gK = 0, hx = 0, hz = 0, traces = 0, partial = 0;   // gK, hx, hz: FP64 running sums
    size_t total = 0;
};

// The time-step kernels address a shot's field with 32-bit offsets: Px * Nz < 2^31.
bool grid_ok(const fwi_grid *g)
{
    return g && g->nx >= 2 && g->nz >= 2 && g->sponge >= 0 && (g->order == 4 || g->order == 8) &&
           (long long)(((g->nx + 2LL * g->sponge + 31) / 32) * 32) * (g->nz + 2LL * g->sponge) < (1LL << 31) &&
           g->nt >= 1 && g->dx > 0 && g->dt > 0 && g->vp_o > 0 && g->rho_o > 0 &&
           std::isfinite(g->dx) && std::isfinite(g->dt);
}

// Fills dims / stencil and lays out the workspace for (B, C).
void layout(Plan &P, const fwi_grid *g, fwi_op op, int ns, int nr, int B, int C)
{
    fwi::Dims &d = P.d;
    d.nx = g->nx; d.nz = g->nz; d.S = g->sponge;
    d.Nx = g->nx + 2 * g->sponge; d.Nz = g->nz + 2 * g->sponge;
    d.Px = (int)up((size_t)d.Nx, 32);
    d.Np = (long long)d.Px * d.Nz;
    P.M = g->order / 2;
    static const double c4[2] = {9.0 / 8.0, -1.0 / 24.0};
    static const double c8[4] = {1225.0 / 1024.0, -245.0 / 3072.0, 49.0 / 5120.0, -5.0 / 7168.0};
    for (int k = 0; k < 4; ++k) {
        double c = k < P.M ? (P.M == 2 ? c4[k] : c8[k]) : 0.0;
        P.st.c[k] = (float)(c * g->dt / g->dx);
        P.st.nc[k] = -P.st.c[k];
    }
    P.ns = ns; P.nr = nr; P.nt = g->nt;
    P.tz = g_tile_tz;   // 0: chosen per launch by strip_height()
    P.variant = g_tile_variant;
    P.acc = g_acc_every > 0 ? g_acc_every : ACC_STEPS;
    P.B = std::max(1, std::min(B, std::max(ns, 1)));
    P.C = std::max(1, std::min(C, g->nt));
    P.nseg = (g->nt + P.C - 1) / P.C;
    P.ngroups = ns > 0 ? (ns + P.B - 1) / P.B : 0;

    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = up(off + bytes, ALIGN); return o; };
    const size_t F = sizeof(float), D = sizeof(double);
    const size_t field = (size_t)d.Np * F, bfield = (size_t)P.B * field;
    P.status = take(ALIGN);
    P.K = take(field); P.bx = take(field); P.bz = take(field);
    P.ax = take(d.Px * F); P.axh = take(d.Px * F); P.az = take(d.Nz * F); P.azh = take(d.Nz * F);
    P.sidx = take(4 * (size_t)std::max(ns, 1) * sizeof(long long));
    P.sw = take(4 * (size_t)std::max(ns, 1) * F);
    P.ridx = take(4 * (size_t)std::max(nr, 1) * sizeof(long long));
    P.rw = take(4 * (size_t)std::max(nr, 1) * F);
    P.rl = take(4 * (size_t)std::max(nr, 1) * sizeof(int));
    for (int b = 0; b < 2; ++b) { P.p[b] = take(bfield); P.vx[b] = take(bfield); P.vz[b] = take(bfield); }
    if (op == FWI_OP_BORN) {
        P.dK = take(field); P.dbx = take(field); P.dbz = take(field);
        for (int b = 0; b < 2; ++b) { P.dp[b] = take(bfield); P.dvx[b] = take(bfield); P.dvz[b] = take(bfield); }
    }
    if (op == FWI_OP_ADJOINT || op == FWI_OP_GRADIENT) {
        for (int b = 0; b < 2; ++b) { P.ap[b] = take(bfield); P.avx[b] = take(bfield); P.avz[b] = take(bfield); }
        P.accK = take(bfield); P.accBx = take(bfield); P.accBz = take(bfield);
        P.snap = take((size_t)(P.C + 1) * bfield);
        if (P.nseg > 1) P.ckpt = take((size_t)P.nseg * 3 * bfield);
        P.gK = take((size_t)d.Np * D); P.hx = take((size_t)d.Np * D); P.hz = take((size_t)d.Np * D);
    }
    if (op == FWI_OP_GRADIENT) {
        P.traces = take((size_t)P.B * std::max(nr, 1) * g->nt * F);
        P.partial = take((size_t)std::max(P.ngroups, 1) * RED_BLOCKS * D);
    }
    P.total = off;
}

// Chooses (B, C) for the budget: first the whole history for as many shots as fit while a
// group still fills the GPU (>= 4M cells); then checkpoints every ~sqrt(3 nt) steps with
// recomputation, for as many shots as fit.  budget 0 -> the minimum plan.
bool make_plan(Plan &P, const fwi_grid *g, fwi_op op, int ns, int nr, size_t budget)
{
    const int nsm = std::max(ns, 1);
    const int nt = g->nt;
    if (op == FWI_OP_MODEL || op == FWI_OP_BORN) {
        layout(P, g, op, ns, nr, 1, nt);
        if (budget == 0) return true;
        if (P.total > budget) return false;
        for (int B = nsm; B >= 1; --B) {
            layout(P, g, op, ns, nr, B, nt);
            if (P.total <= budget) return true;
        }
        return false;
    }
    Plan tmp;
    layout(tmp, g, op, ns, nr, 1, nt);
    const long long Np = tmp.d.Np;
    if (g_ckpt_every > 0 && g_ckpt_every < nt) {
        // checkpoints every g_ckpt_every steps, as many shots per group as fit
        layout(P, g, op, ns, nr, 1, g_ckpt_every);
        if (budget == 0) return true;
        if (P.total > budget) return false;
        for (int B = nsm; B >= 1; --B) {
            layout(P, g, op, ns, nr, B, g_ckpt_every);
            if (P.total <= budget) return true;
        }
        return false;
    }
    const int Cs = std::max(1, (int)std::ceil(std::sqrt(3.0 * nt)));
    // minimum: one shot, whichever history scheme is smaller
    Plan a, b;
    layout(a, g, op, ns, nr, 1, nt);
    layout(b, g, op, ns, nr, 1, Cs);
    const Plan &mn = a.total <= b.total ? a : b;
    if (budget == 0) { P = mn; return true; }
    if (mn.total > budget) return false;
    const int Bpar = (int)std::min<long long>(nsm, std::max<long long>(1, (4000000 + Np - 1) / Np));
    for (int B = nsm; B >= Bpar; --B) {
        layout(P, g, op, ns, nr, B, nt);
        if (P.total <= budget) return true;
    }
    for (int B = nsm; B >= 1; --B) {
        layout(P, g, op, ns, nr, B, Cs);
        if (P.total <= budget) return true;
    }
    P = mn;
    return true;
}

template <typename T>
T *at(void *work, size_t off) { return reinterpret_cast<T *>(static_cast<char *>(work) + off); }

int check_common(const fwi_grid *g, const float *xa, const float *xb, const fwi_sources *src,
                 const fwi_receivers *rec, void *work, size_t work_bytes)
{
    if (!grid_ok(g))
        return fail(FWI_EINVAL, "invalid grid (nx, nz >= 2, fewer than 2^31 padded cells per shot, order 4 or 8, "
                                "nt >= 1, dx, dt, vp_o, rho_o > 0)");
    if (!xa || !xb) return fail(FWI_EINVAL, "null contrast pointer");
    if (!src || !rec || src->ns < 0 || rec->nr < 0) return fail(FWI_EINVAL, "invalid sources/receivers");
    if (src->ns > 0 && (!src->xy || !src->wavelet)) return fail(FWI_EINVAL, "null source arrays");
    if (rec->nr > 0 && !rec->xy) return fail(FWI_EINVAL, "null receiver array");
    if (src->ns > (1 << 20) || rec->nr > (1 << 20) || (long long)src->ns * rec->nr > (1LL << 28))
        return fail(FWI_EINVAL, "too many sources or receivers (at most 2^20 each, 2^28 traces)");
    if (!work) return fail(FWI_EINVAL, "null workspace");
    if (reinterpret_cast<uintptr_t>(work) % ALIGN) return fail(FWI_EINVAL, "workspace not 256-byte aligned");
    (void)work_bytes;
    return FWI_OK;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(FWI_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

#define LAUNCH(kernel, grid, block, smem, stream, ...)             \
    do {                                                           \
        cudaEvent_t *ev_ = g_prof.next(#kernel);                   \
        if (ev_) cudaEventRecord(ev_[0], stream);                  \
        kernel<<<grid, block, smem, stream>>>(__VA_ARGS__);        \
        if (ev_) cudaEventRecord(ev_[1], stream);                  \
        ++g_launches;                                              \
    } while (0)


// Model, sponge tables and acquisition geometry (S1, S2).
int setup(const Plan &P, const fwi_grid *g, int pz, const float *xa, const float *xb,
          const fwi_sources *src, const fwi_receivers *rec, void *work, cudaStream_t st)
{
    TraceRange tr(PH_MODEL_BUILD);
    const fwi::Dims &d = P.d;
    const double sum_c = P.M == 2 ? 9.0 / 8.0 + 1.0 / 24.0
                                  : 1225.0 / 1024.0 + 245.0 / 3072.0 + 49.0 / 5120.0 + 5.0 / 7168.0;
    const double cfl = g->dt * std::sqrt(2.0) * sum_c / g->dx;
    int *status = at<int>(work, P.status);
    CK(cudaMemsetAsync(status, 0, sizeof(int), st));
    dim3 b2(32, 8), g2((d.Px + 31) / 32, (d.Nz + 7) / 8);
    LAUNCH(fwi::k_model, g2, b2, 0, st, xa, xb, pz, g->vp_o, g->rho_o, cfl, d, at<float>(work, P.K),
           at<float>(work, P.bx), at<float>(work, P.bz), status);
    const double sv = g->sponge_v > 0 ? g->sponge_v : g->vp_o;
    const double sR = (g->sponge_R > 0 && g->sponge_R < 1) ? g->sponge_R : 1e-3;
    LAUNCH(fwi::k_sponge, (d.Px + 127) / 128, 128, 0, st, at<float>(work, P.ax), d.Px, d.nx, d.S, g->dx, g->dt, sv, sR, 0);
    LAUNCH(fwi::k_sponge, (d.Px + 127) / 128, 128, 0, st, at<float>(work, P.axh), d.Px, d.nx, d.S, g->dx, g->dt, sv, sR, 1);
    LAUNCH(fwi::k_sponge, (d.Nz + 127) / 128, 128, 0, st, at<float>(work, P.az), d.Nz, d.nz, d.S, g->dx, g->dt, sv, sR, 0);
    LAUNCH(fwi::k_sponge, (d.Nz + 127) / 128, 128, 0, st, at<float>(work, P.azh), d.Nz, d.nz, d.S, g->dx, g->dt, sv, sR, 1);
    if (src->ns > 0)
        LAUNCH(fwi::k_geometry, (src->ns + 127) / 128, 128, 0, st, src->xy, src->ns, d, g->dx,
               g->dt / (g->dx * g->dx), at<long long>(work, P.sidx), at<float>(work, P.sw), status);
    if (rec->nr > 0) {
        LAUNCH(fwi::k_geometry, (rec->nr + 127) / 128, 128, 0, st, rec->xy, rec->nr, d, g->dx, 1.0,
               at<long long>(work, P.ridx), at<float>(work, P.rw), status);
        LAUNCH(fwi::k_receiver_chain, (4 * rec->nr + 127) / 128, 128, 0, st, at<long long>(work, P.ridx), 4 * rec->nr,
               at<int>(work, P.rl));
    }
    return FWI_OK;
}

// Opts `kernel` in to `bytes` of dynamic shared memory (once per kernel and device).
void dyn_smem(const void *kernel, size_t bytes)
{
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!done.insert({kernel, dev}).second) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    // the whole unified L1/shared array as shared memory: the staging, not L1, holds the reuse
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

// Launch of a streaming kernel with `smem` bytes of dynamic shared memory.
#define SLAUNCH(kernel, grid, block, smem, stream, ...)            \
    do {                                                           \
        dyn_smem((const void *)kernel, smem);                      \
        LAUNCH(kernel, grid, block, smem, stream, __VA_ARGS__);    \
    } while (0)

// Warps of `kernel` (blocks of `threads`, `smem` bytes of dynamic shared memory) resident on
// the whole GPU at once, from the occupancy calculator; cached per kernel and device.
int resident_warps(const void *kernel, int threads, size_t smem)
{
    dyn_smem(kernel, smem);
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({kernel, dev});
    if (it != cache.end()) return it->second;
    int blocks = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        blocks = 1;
        sms = 1;
    }
    const int w = std::max(1, blocks * (threads / 32) * sms);
    cache[{kernel, dev}] = w;
    return w;
}

// Strip height of a streaming launch (the tile-shape autotuner's rule).  A warp marches
// down its strip row by row, so a launch lasts at least (tz + 4M - 1) row times, while the
// row work of the whole launch grows as tz shrinks (each strip recomputes 4M - 1 halo rows).
// Modelling the launch as max(one strip, total row work / resident warps), the best height
// makes the strips just fill the resident warps: tz = column strips x rows x shots /
// resident warps, rounded up to a multiple of 8 and kept within [8, 64].  fwi_set_tile's
// height, when set, overrides the rule.  Any height gives bitwise identical results.
long long strip_rows(const fwi::Dims &d, long long shots)
{
    return (long long)((d.Nx + fwi::WS - 1) / fwi::WS) * d.Nz * shots;
}

int strip_height_for_rows(long long rows, int resident)
{
    long long tz = (rows + resident - 1) / std::max(resident, 1);
    tz = (tz + 7) / 8 * 8;
    return (int)std::min<long long>(64, std::max<long long>(8, tz));
}

// Online strip-height tuner (the measured half of the autotuner).  For each launch shape --
// (kernel, grid, shots) for the single-job calls, (kernel, quarter-octave bucket of the total
// strip rows) for the engine's batched launches -- the first launches try candidate heights,
// each twice, timed by an event pair on the launching stream.  A single-job shape tries the
// rule's height and the heights that cut its Nz rows into c equal strips, ceil(Nz / c), for
// every c from ceil(Nz / 136) to ceil(Nz / 32) (heights with equal strip counts differ only in
// the last strip, and the even split is the one worth timing; measured on 681 rows, the best
// height moved between 60 and 124 with the kernel and the shot count); a batched shape, whose
// jobs have different heights, tries the rule's height and 32 .. 120.  The timings are
// collected without blocking as later launches of the same shape arrive; once every candidate
// has two, the shape keeps its fastest height.  Launches under stream capture are not timed
// and use the rule's height (or the shape's chosen one).
class StripTuner {
public:
    struct Slot {
        int tz = 0;
        size_t cand = 0;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        bool timed = false;
    };
    using Key = std::tuple<const void *, long long, long long, int>;

    // Height for the next launch of shape `key` on `st`; when the launch is to be timed the
    // start event is already recorded and finish(slot) must follow the launch.
    // nz > 0: the launch covers one grid of nz rows (even-split candidates)
    Slot pick(const Key &key, int rule, cudaStream_t st, int nz = 0)
    {
        Slot s;
        s.tz = rule;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            cudaGetLastError();
            return s;
        }
        std::lock_guard<std::mutex> lk(mu_);
        Shape &sh = shapes_[key];
        if (sh.cand.empty()) init(sh, rule, nz);
        poll(sh);
        if (sh.chosen) {
            s.tz = sh.chosen;
            return s;
        }
        if (cs != cudaStreamCaptureStatusNone) return s;
        size_t best = sh.cand.size();
        for (size_t k = 0; k < sh.cand.size(); ++k) {
            const size_t c = (sh.next + k) % sh.cand.size();
            if (sh.nsamp[c] + sh.inflight[c] < SAMPLES) { best = c; break; }
        }
        if (best == sh.cand.size()) return s;     // every sample is in flight
        sh.next = best + 1;
        s.tz = sh.cand[best];
        s.cand = best;
        s.e0 = event();
        s.e1 = event();
        if (!s.e0 || !s.e1 || cudaEventRecord(s.e0, st) != cudaSuccess) {
            cudaGetLastError();
            release(s);
            s.tz = rule;
            return s;
        }
        s.timed = true;
        ++sh.inflight[best];
        return s;
    }

    void finish(const Key &key, Slot &s, cudaStream_t st)
    {
        if (!s.timed) return;
        std::lock_guard<std::mutex> lk(mu_);
        Shape &sh = shapes_[key];
        if (cudaEventRecord(s.e1, st) != cudaSuccess) {
            cudaGetLastError();
            --sh.inflight[s.cand];
            release(s);
            return;
        }
        sh.pending.push_back(s);
    }

private:
    static constexpr int SAMPLES = 2;
    struct Shape {
        std::vector<int> cand, nsamp, inflight;
        std::vector<float> best;
        std::deque<Slot> pending;
        size_t next = 0;
        int chosen = 0;
    };

    void init(Shape &sh, int rule, int nz)
    {
        std::set<int> c = {rule};
        if (nz > 0) {
            for (int k = (nz + 135) / 136; k <= (nz + 31) / 32; ++k) c.insert((nz + k - 1) / k);
        } else {
            c.insert({32, 40, 48, 56, 64, 80, 96, 120});
        }
        sh.cand.assign(c.begin(), c.end());
        sh.nsamp.assign(sh.cand.size(), 0);
        sh.inflight.assign(sh.cand.size(), 0);
        sh.best.assign(sh.cand.size(), 1e30f);
    }

    void poll(Shape &sh)
    {
        while (!sh.pending.empty()) {
            Slot &s = sh.pending.front();
            const cudaError_t q = cudaEventQuery(s.e1);
            if (q == cudaErrorNotReady) break;
            float ms = 0.f;
            if (q == cudaSuccess && cudaEventElapsedTime(&ms, s.e0, s.e1) == cudaSuccess) {
                sh.best[s.cand] = std::min(sh.best[s.cand], ms);
                ++sh.nsamp[s.cand];
            } else {
                cudaGetLastError();
            }
            --sh.inflight[s.cand];
            release(s);
            sh.pending.pop_front();
        }
        if (sh.chosen) return;
        for (size_t c = 0; c < sh.cand.size(); ++c)
            if (sh.nsamp[c] < SAMPLES) return;
        size_t b = 0;
        for (size_t c = 1; c < sh.cand.size(); ++c)
            if (sh.best[c] < sh.best[b]) b = c;
        sh.chosen = sh.cand[b];
    }

    cudaEvent_t event()
    {
        if (!pool_.empty()) {
            cudaEvent_t e = pool_.back();
            pool_.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }

    void release(Slot &s)
    {
        if (s.e0) pool_.push_back(s.e0);
        if (s.e1) pool_.push_back(s.e1);
        s.e0 = s.e1 = nullptr;
    }

    std::mutex mu_;
    std::map<Key, Shape> shapes_;
    std::vector<cudaEvent_t> pool_;
};

StripTuner g_tuner;

int strip_height(int fixed, const fwi::Dims &d, long long shots, int resident)
{
    return fixed > 0 ? fixed : strip_height_for_rows(strip_rows(d, shots), resident);
}

// Strip height of a single-job launch: fixed, or tuned per (kernel, grid, shots).  Returns the
// tuner slot the caller closes with g_tuner.finish() after the launch.
StripTuner::Slot tuned_height(int fixed, const void *kernel, const fwi::Dims &d, int shots, int resident,
                              cudaStream_t st, StripTuner::Key &key)
{
    StripTuner::Slot s;
    s.tz = strip_height(fixed, d, shots, resident);
    if (fixed > 0) return s;
    key = StripTuner::Key{kernel, ((long long)d.Nx << 32) | (unsigned)d.Nz, shots, 0};
    return g_tuner.pick(key, s.tz, st, d.Nz);
}

// Warp-strip launch shape: one warp per (120-column strip, tz-row strip, shot), then
// `extra` sampling warps, wpb warps a block.
dim3 warp_grid(const Plan &P, int tz, int shots, int wpb = 2, int extra = 0)
{
    return dim3((unsigned)(((long long)fwi::strip_warps(P.d, tz, shots) + extra + wpb - 1) / wpb));
}

// Sampling of the previous step carried by a single-job launch (none: count 0).
fwi::Tail tail_of(const Plan &P, void *work, const float *field, float *traces, int bg, int col)
{
    const bool on = traces && field && P.nr > 0 && bg > 0 && col >= 0;
    return fwi::Tail{field, traces, at<long long>(work, P.ridx), at<float>(work, P.rw), P.d.Np, P.nr, P.nt, col,
                     on ? bg * P.nr : 0};
}

fwi::Model model_of(const Plan &P, void *work)
{
    return fwi::Model{at<float>(work, P.K),   at<float>(work, P.bx), at<float>(work, P.bz),
                      at<float>(work, P.ax),  at<float>(work, P.axh), at<float>(work, P.az),
                      at<float>(work, P.azh), at<int>(work, P.status)};
}

struct Fwd {
    const Plan &P;
    void *work;
    cudaStream_t st;
    const float *wav;

    // one forward step n for the group's shots [s0, s0 + bg): p^n in p0 -> p^{n+1} in p1,
    // velocities ping-pong on the parity of n
    // tl: sampling of the previous step by extra warps of this launch (count 0: none)
    void step(int n, int s0, int bg, const float *p0, float *p1, const fwi::Tail &tl = fwi::Tail{}) const
    {
        const fwi::Dims &d = P.d;
        const fwi::Source src{at<long long>(work, P.sidx) + 4LL * s0, at<float>(work, P.sw) + 4LL * s0, wav};
        const float *vx0 = at<float>(work, P.vx[n & 1]), *vz0 = at<float>(work, P.vz[n & 1]);
        float *vx1 = at<float>(work, P.vx[(n + 1) & 1]), *vz1 = at<float>(work, P.vz[(n + 1) & 1]);
        constexpr int T = 32 * fwi::FWD_WPB;
        const size_t S = P.M == 2 ? fwi::fwd_smem<2>() : fwi::fwd_smem<4>();
        constexpr int B170d = fwi::minb(170, T);
        const void *K0 = P.M == 2 ? (const void *)fwi::k_fwd_warp<2, B170d> : (const void *)fwi::k_fwd_warp<4, B170d>;
        StripTuner::Key key;
        StripTuner::Slot ts = tuned_height(P.tz, K0, d, bg, resident_warps(K0, T, S), st, key);
        const int tz = ts.tz;
        const dim3 grid = warp_grid(P, tz, bg, fwi::FWD_WPB, fwi::tail_warps(tl));
        const fwi::FwdArgs args{p0, vx0, vz0, p1, vx1, vz1, model_of(P, work), d, P.st, src, n, tz, bg};
        constexpr int B128 = fwi::minb(128, T), B170 = fwi::minb(170, T);
        // the forward kernel's default build is the 170-register one (measured: its register
        // queues otherwise take it to 184 registers and 10 resident warps, 6 % slower)
        if (P.M == 2) {
            switch (P.variant) {
            case 1: SLAUNCH((fwi::k_fwd_warp<2, B128>), grid, T, S, st, args, tl); break;
            default: SLAUNCH((fwi::k_fwd_warp<2, B170>), grid, T, S, st, args, tl);
            }
        } else {
            switch (P.variant) {
            case 1: SLAUNCH((fwi::k_fwd_warp<4, B128>), grid, T, S, st, args, tl); break;
            default: SLAUNCH((fwi::k_fwd_warp<4, B170>), grid, T, S, st, args, tl);
            }
        }
        g_tuner.finish(key, ts, st);
    }

    void sample(int n, int bg, int nr, const float *p, float *traces) const
    {
        if (nr == 0) return;
        LAUNCH(fwi::k_sample, (bg * nr + 127) / 128, 128, 0, st, p, bg, nr, P.nt, n, P.d.Np,
               at<long long>(work, P.ridx), at<float>(work, P.rw), traces);
    }
};

int finish(cudaStream_t st)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    (void)st;
    return FWI_OK;
}

int plan_for(Plan &P, const fwi_grid *g, fwi_op op, int ns, int nr, size_t work_bytes)
{
    if (!make_plan(P, g, op, ns, nr, work_bytes))
        return fail(FWI_ENOMEM, "workspace of %zu bytes is below the minimum %zu for this operation",
                    work_bytes, fwi_workspace_bytes(g, ns, nr, op, 0));
    return FWI_OK;
}

// Forward over all steps for one group, used by model, adjoint and gradient.
//   traces: [bg][nr][nt] output or null.
//   with_hist: keep the pressure history of the last segment (it is the pressure state of those
//   steps: p^n lives in snapshot slot n - last0) and checkpoints (p, vx, vz) every C steps.
int forward_group(const Plan &P, void *work, cudaStream_t st, const float *wav, int s0, int bg,
                  float *traces, bool with_hist)
{
    TraceRange tr(PH_FORWARD);
    const Fwd f{P, work, st, wav};
    const size_t bf = (size_t)bg * P.d.Np * sizeof(float);
    const size_t slot = (size_t)P.B * P.d.Np;   // floats between snapshot slots
    const int last0 = with_hist ? (P.nseg - 1) * P.C : P.nt + 1;
    float *snap = with_hist ? at<float>(work, P.snap) : nullptr;
    auto pbuf = [&](int n) -> float * {
        return n >= last0 ? snap + (size_t)(n - last0) * slot : at<float>(work, P.p[n & 1]);
    };
    CK(cudaMemsetAsync(pbuf(0), 0, bf, st));
    CK(cudaMemsetAsync(at<char>(work, P.vx[0]), 0, bf, st));
    CK(cudaMemsetAsync(at<char>(work, P.vz[0]), 0, bf, st));
    for (int n = 0; n < P.nt; ++n) {
        if (with_hist && P.nseg > 1 && n % P.C == 0) {
            float *ck = at<float>(work, P.ckpt) + (size_t)(n / P.C) * 3 * slot;
            CK(cudaMemcpyAsync(ck, pbuf(n), bf, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(ck + slot, at<float>(work, P.vx[n & 1]), bf, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(ck + 2 * slot, at<float>(work, P.vz[n & 1]), bf, cudaMemcpyDeviceToDevice, st));
        }
        // this launch's extra warps sample p^n (the previous step's output) into column n - 1
        f.step(n, s0, bg, pbuf(n), pbuf(n + 1), tail_of(P, work, pbuf(n), traces, bg, n - 1));
    }
    if (traces && P.nt > 0) f.sample(P.nt - 1, bg, P.nr, pbuf(P.nt), traces);   // the last sample
    return FWI_OK;
}

// FP32 accumulators of the group's bg slots into the FP64 running sums, slots cleared.
int flush_acc(const Plan &P, void *work, int bg, cudaStream_t st)
{
    const long long units = P.d.Np / 4;
    LAUNCH(fwi::k_acc_flush, dim3((unsigned)((units + fwi::FLUSH_X - 1) / fwi::FLUSH_X), 3),
           dim3(fwi::FLUSH_X, fwi::FLUSH_Y), 0, st, at<float>(work, P.accK), at<float>(work, P.accBx),
           at<float>(work, P.accBz), bg, P.d.Np, at<double>(work, P.gK), at<double>(work, P.hx), at<double>(work, P.hz));
    const size_t bf = (size_t)bg * P.d.Np * sizeof(float);
    for (size_t o : {P.accK, P.accBx, P.accBz}) CK(cudaMemsetAsync(at<char>(work, o), 0, bf, st));
    return FWI_OK;
}

// Adjoint step n of a group (one launch): pbar^{n+1} (after its receiver injection),
// vbar^{n+1/2} -> pbar^n, vbar^{n-1/2}, the gradient products into the FP32 accumulators.
// pn: p^n of the group's shots.  Shared by the single calls and the engine.
fwi::AdjArgs adj_args(const Plan &P, void *work, int n, int bg, const float *pn)
{
    const int i = (n + 1) & 1, o = n & 1;
    return fwi::AdjArgs{at<float>(work, P.ap[i]), at<float>(work, P.avx[i]), at<float>(work, P.avz[i]),
                        at<float>(work, P.ap[o]), at<float>(work, P.avx[o]), at<float>(work, P.avz[o]),
                        model_of(P, work), pn, at<float>(work, P.accK), at<float>(work, P.accBx),
                        at<float>(work, P.accBz), P.d, P.st, P.tz, bg};
}

// Adjoint over all segments for one group (history from forward_group), accumulating into
// the per-slot FP32 accumulators and, every P.acc steps and after step 0, into the FP64
// running sums.  res: [bg][nr][nt] residual of the group.
int adjoint_group(const Plan &P, void *work, cudaStream_t st, const float *wav, int s0, int bg,
                  const float *res)
{
    const fwi::Dims &d = P.d;
    const Fwd f{P, work, st, wav};
    const size_t bf = (size_t)bg * d.Np * sizeof(float);
    const size_t slot = (size_t)P.B * d.Np;
    const int first = P.nt & 1;   // buffers holding pbar^{nt}, vbar^{nt-1/2} = 0
    CK(cudaMemsetAsync(at<char>(work, P.ap[first]), 0, bf, st));
    CK(cudaMemsetAsync(at<char>(work, P.avx[first]), 0, bf, st));
    CK(cudaMemsetAsync(at<char>(work, P.avz[first]), 0, bf, st));
    float *snap = at<float>(work, P.snap);
    for (int k = P.nseg - 1; k >= 0; --k) {
        const int n0 = k * P.C, n1 = std::min(n0 + P.C, P.nt);
        if (k < P.nseg - 1) {   // recompute the segment from its checkpoint
            TraceRange tr(PH_RECOMPUTE);
            const float *ck = at<float>(work, P.ckpt) + (size_t)k * 3 * slot;
            CK(cudaMemcpyAsync(snap, ck, bf, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(at<float>(work, P.vx[n0 & 1]), ck + slot, bf, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(at<float>(work, P.vz[n0 & 1]), ck + 2 * slot, bf, cudaMemcpyDeviceToDevice, st));
            for (int n = n0; n < n1; ++n)
                f.step(n, s0, bg, snap + (size_t)(n - n0) * slot, snap + (size_t)(n + 1 - n0) * slot);
        }
        TraceRange tr(PH_ADJOINT);
        for (int n = n1 - 1; n >= n0; --n) {
            const float *pn = snap + (size_t)(n - n0) * slot, *pn1 = snap + (size_t)(n + 1 - n0) * slot;
            if (P.nr > 0)   // pbar^{n+1} += R^T r_n, with its K-gradient term (R^T r_n) p^{n+1}
                LAUNCH(fwi::k_adj_inject_k, (bg * 4 * P.nr + 127) / 128, 128, 0, st, at<float>(work, P.ap[(n + 1) & 1]),
                       at<float>(work, P.accK), pn1, bg, P.nr, P.nt, n, d.Np, at<long long>(work, P.ridx),
                       at<float>(work, P.rw), at<int>(work, P.rl), res);
            const size_t S = P.M == 2 ? fwi::adj_smem<2>() : fwi::adj_smem<4>();
            const void *K0 = P.M == 2 ? (const void *)fwi::k_adj_warp<2, 1> : (const void *)fwi::k_adj_warp<4, 1>;
            StripTuner::Key key;
            StripTuner::Slot ts = tuned_height(P.tz, K0, d, bg, resident_warps(K0, 32, S), st, key);
            fwi::AdjArgs args = adj_args(P, work, n, bg, pn);
            args.tz = ts.tz;
            const dim3 grid = warp_grid(P, ts.tz, bg, 1);
            constexpr int B128 = fwi::minb(128, 32), B170 = fwi::minb(170, 32);
            if (P.M == 2) {
                switch (P.variant) {
                case 1: SLAUNCH((fwi::k_adj_warp<2, B128>), grid, 32, S, st, args); break;
                case 2: SLAUNCH((fwi::k_adj_warp<2, B170>), grid, 32, S, st, args); break;
                default: SLAUNCH((fwi::k_adj_warp<2, 1>), grid, 32, S, st, args);
                }
            } else {
                switch (P.variant) {
                case 1: SLAUNCH((fwi::k_adj_warp<4, B128>), grid, 32, S, st, args); break;
                case 2: SLAUNCH((fwi::k_adj_warp<4, B170>), grid, 32, S, st, args); break;
                default: SLAUNCH((fwi::k_adj_warp<4, 1>), grid, 32, S, st, args);
                }
            }
            g_tuner.finish(key, ts, st);
            if (n % P.acc == 0) {
                const int rc = flush_acc(P, work, bg, st);
                if (rc) return rc;
            }
        }
    }
    return FWI_OK;
}

// Zeroes the FP32 slot accumulators and the FP64 running sums of a gradient plan.
int clear_acc(const Plan &P, void *work, cudaStream_t st)
{
    const size_t bf = (size_t)P.B * P.d.Np * sizeof(float), bd = (size_t)P.d.Np * sizeof(double);
    for (size_t o : {P.accK, P.accBx, P.accBz}) CK(cudaMemsetAsync(at<char>(work, o), 0, bf, st));
    for (size_t o : {P.gK, P.hx, P.hz}) CK(cudaMemsetAsync(at<char>(work, o), 0, bd, st));
    return FWI_OK;
}

int finalize_grad(const Plan &P, const fwi_grid *g, int pz, const float *xa, const float *xb, void *work,
                  double *grads, cudaStream_t st)
{
    TraceRange tr(PH_REDUCE);
    const fwi::Dims &d = P.d;
    dim3 b2(32, 8), gp((d.Nx + 31) / 32, (d.Nz + 7) / 8), gq((d.nx + 31) / 32, (d.nz + 7) / 8);
    LAUNCH(fwi::k_grad_cells, gp, b2, 0, st, at<float>(work, P.K), at<float>(work, P.bx), at<float>(work, P.bz), d,
           at<double>(work, P.gK), at<double>(work, P.hx), at<double>(work, P.hz));
    LAUNCH(fwi::k_grad_final, gq, b2, 0, st, at<double>(work, P.gK), at<double>(work, P.hx),
           at<double>(work, P.hz), xa, xb, pz, g->vp_o, g->rho_o, d, grads);
    return FWI_OK;
}

int adjoint_impl(const fwi_grid *g, int pz, const float *xa, const float *xb, const fwi_sources *src,
                 const fwi_receivers *rec, const float *residual, const float *data, double *misfit,
                 double *grads, void *work, size_t work_bytes, cudaStream_t st, const float *weights = nullptr)
{
    const fwi_op op = data ? FWI_OP_GRADIENT : FWI_OP_ADJOINT;
    Plan P;
    int rc = plan_for(P, g, op, src->ns, rec->nr, work_bytes);
    if (rc) return rc;
    if ((rc = setup(P, g, pz, xa, xb, src, rec, work, st))) return rc;
    if ((rc = clear_acc(P, work, st))) return rc;
    const long long per_shot = (long long)P.nr * P.nt;
    for (int gi = 0; gi < P.ngroups; ++gi) {
        const int s0 = gi * P.B, bg = std::min(P.B, P.ns - s0);
        const float *res;
        if (data) {
            float *tr = at<float>(work, P.traces);
            if ((rc = forward_group(P, work, st, src->wavelet, s0, bg, tr, true))) return rc;
            const long long n = bg * per_shot;
            if (n > 0)
                LAUNCH(fwi::k_residual, RED_BLOCKS, fwi::RED_THREADS, 0, st, tr, data + s0 * per_shot, n,
                       at<double>(work, P.partial) + (size_t)gi * RED_BLOCKS,
                       weights ? weights + (size_t)s0 * P.nr : nullptr, P.nt);
            else
                CK(cudaMemsetAsync(at<double>(work, P.partial) + (size_t)gi * RED_BLOCKS, 0,
                                   RED_BLOCKS * sizeof(double), st));
            res = tr;
        } else {
            if ((rc = forward_group(P, work, st, src->wavelet, s0, bg, nullptr, true))) return rc;
            res = residual + s0 * per_shot;
        }
        if ((rc = adjoint_group(P, work, st, src->wavelet, s0, bg, res))) return rc;
    }
    if (data) {
        if (P.ngroups > 0)
            LAUNCH(fwi::k_sum_final, 1, fwi::RED_THREADS, 0, st, at<double>(work, P.partial),
                   P.ngroups * RED_BLOCKS, misfit);
        else
            CK(cudaMemsetAsync(misfit, 0, sizeof(double), st));
    }
    if ((rc = finalize_grad(P, g, pz, xa, xb, work, grads, st))) return rc;
    return finish(st);
}

}  // namespace

namespace fwi_internal {
void set_error(const char *msg) { g_err = msg ? msg : ""; }
}

#include "fwi_arena.h"
#include "fwi_engine.inc"
#include "fwi_fborn.inc"

extern "C" {

size_t fwi_workspace_bytes(const fwi_grid *g, int ns, int nr, fwi_op op, size_t budget_bytes)
{
    if (!grid_ok(g) || ns < 0 || nr < 0 || op < FWI_OP_MODEL || op > FWI_OP_GRADIENT) return 0;
    Plan P;
    if (!make_plan(P, g, op, ns, nr, budget_bytes)) {
        make_plan(P, g, op, ns, nr, 0);
    }
    return P.total;
}

int fwi_model(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b, const fwi_sources *src,
              const fwi_receivers *rec, float *traces, void *work, size_t work_bytes, void *stream)
{
    g_err.clear();
    g_launches = 0;
    int rc = check_common(g, xi_a, xi_b, src, rec, work, work_bytes);
    if (rc) return rc;
    if ((int)pz < 0 || (int)pz > 4) return fail(FWI_EINVAL, "unknown parameterization %d", (int)pz);
    if (src->ns > 0 && rec->nr > 0 && !traces) return fail(FWI_EINVAL, "null traces");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan P;
    if ((rc = plan_for(P, g, FWI_OP_MODEL, src->ns, rec->nr, work_bytes))) return rc;
    if ((rc = setup(P, g, pz, xi_a, xi_b, src, rec, work, st))) return rc;
    for (int gi = 0; gi < P.ngroups; ++gi) {
        const int s0 = gi * P.B, bg = std::min(P.B, P.ns - s0);
        if ((rc = forward_group(P, work, st, src->wavelet, s0, bg, traces + (size_t)s0 * P.nr * P.nt, false))) return rc;
    }
    return finish(st);
}

int fwi_born(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b, const float *dxi_a,
             const float *dxi_b, const fwi_sources *src, const fwi_receivers *rec, float *dtraces, void *work,
             size_t work_bytes, void *stream)
{
    g_err.clear();
    g_launches = 0;
    int rc = check_common(g, xi_a, xi_b, src, rec, work, work_bytes);
    if (rc) return rc;
    if ((int)pz < 0 || (int)pz > 4) return fail(FWI_EINVAL, "unknown parameterization %d", (int)pz);
    if (!dxi_a || !dxi_b) return fail(FWI_EINVAL, "null perturbation pointer");
    if (src->ns > 0 && rec->nr > 0 && !dtraces) return fail(FWI_EINVAL, "null dtraces");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan P;
    if ((rc = plan_for(P, g, FWI_OP_BORN, src->ns, rec->nr, work_bytes))) return rc;
    if ((rc = setup(P, g, pz, xi_a, xi_b, src, rec, work, st))) return rc;
    const fwi::Dims &d = P.d;
    dim3 b2(32, 8), g2((d.Px + 31) / 32, (d.Nz + 7) / 8);
    LAUNCH(fwi::k_model_pert, g2, b2, 0, st, xi_a, xi_b, dxi_a, dxi_b, (int)pz, g->vp_o, g->rho_o, d,
           at<float>(work, P.dK), at<float>(work, P.dbx), at<float>(work, P.dbz));
    const fwi::Model mo = model_of(P, work);
    const fwi::Pert pe{at<float>(work, P.dK), at<float>(work, P.dbx), at<float>(work, P.dbz)};
    for (int gi = 0; gi < P.ngroups; ++gi) {
        TraceRange tr(PH_BORN);
        const int s0 = gi * P.B, bg = std::min(P.B, P.ns - s0);
        const size_t bf = (size_t)bg * d.Np * sizeof(float);
        for (size_t off : {P.p[0], P.vx[0], P.vz[0], P.dp[0], P.dvx[0], P.dvz[0]})
            CK(cudaMemsetAsync(at<char>(work, off), 0, bf, st));
        const fwi::Source sr{at<long long>(work, P.sidx) + 4LL * s0, at<float>(work, P.sw) + 4LL * s0, src->wavelet};
        float *out = dtraces + (size_t)s0 * P.nr * P.nt;
        for (int n = 0; n < P.nt; ++n) {
            const int i = n & 1, o = (n + 1) & 1;
            auto F = [&](const size_t *a) { return at<float>(work, a[i]); };
            auto G = [&](const size_t *a) { return at<float>(work, a[o]); };
            const size_t S = P.M == 2 ? fwi::born_smem<2>() : fwi::born_smem<4>();
            const void *K0 = P.M == 2 ? (const void *)fwi::k_born_warp<2, 1> : (const void *)fwi::k_born_warp<4, 1>;
            StripTuner::Key key;
            StripTuner::Slot ts = tuned_height(P.tz, K0, d, bg, resident_warps(K0, 32, S), st, key);
            const int tz = ts.tz;
            const fwi::Tail tl = tail_of(P, work, F(P.dp), out, bg, n - 1);   // samples q^n into column n - 1
            const dim3 grid = warp_grid(P, tz, bg, 1, fwi::tail_warps(tl));
#define BORN_ARGS fwi::BornArgs{F(P.p), F(P.vx), F(P.vz), F(P.dp), F(P.dvx), F(P.dvz), G(P.p), G(P.vx), \
                  G(P.vz), G(P.dp), G(P.dvx), G(P.dvz), mo, pe, d, P.st, sr, n, tz, bg}
            constexpr int B170 = fwi::minb(170, 32);
            if (P.M == 2) {
                if (P.variant == 2) SLAUNCH((fwi::k_born_warp<2, B170>), grid, 32, S, st, BORN_ARGS, tl);
                else SLAUNCH((fwi::k_born_warp<2, 1>), grid, 32, S, st, BORN_ARGS, tl);
            } else {
                if (P.variant == 2) SLAUNCH((fwi::k_born_warp<4, B170>), grid, 32, S, st, BORN_ARGS, tl);
                else SLAUNCH((fwi::k_born_warp<4, 1>), grid, 32, S, st, BORN_ARGS, tl);
            }
            g_tuner.finish(key, ts, st);
#undef BORN_ARGS
        }
        if (P.nr > 0 && P.nt > 0)   // the last sample: q^{nt}
            LAUNCH(fwi::k_sample, (bg * P.nr + 127) / 128, 128, 0, st, at<float>(work, P.dp[P.nt & 1]), bg, P.nr,
                   P.nt, P.nt - 1, d.Np, at<long long>(work, P.ridx), at<float>(work, P.rw), out);
    }
    return finish(st);
}

int fwi_adjoint(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b, const fwi_sources *src,
                const fwi_receivers *rec, const float *residual, double *grads, void *work, size_t work_bytes,
                void *stream)
{
    g_err.clear();
    g_launches = 0;
    int rc = check_common(g, xi_a, xi_b, src, rec, work, work_bytes);
    if (rc) return rc;
    if ((int)pz < 0 || (int)pz > 4) return fail(FWI_EINVAL, "unknown parameterization %d", (int)pz);
    if (!grads) return fail(FWI_EINVAL, "null grads");
    if (src->ns > 0 && rec->nr > 0 && !residual) return fail(FWI_EINVAL, "null residual");
    return adjoint_impl(g, pz, xi_a, xi_b, src, rec, residual, nullptr, nullptr, grads, work, work_bytes,
                        static_cast<cudaStream_t>(stream));
}

int fwi_gradient_weighted(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b,
                          const fwi_sources *src, const fwi_receivers *rec, const float *data,
                          const float *weights, double *misfit, double *grads, void *work, size_t work_bytes,
                          void *stream)
{
    g_err.clear();
    g_launches = 0;
    int rc = check_common(g, xi_a, xi_b, src, rec, work, work_bytes);
    if (rc) return rc;
    if ((int)pz < 0 || (int)pz > 4) return fail(FWI_EINVAL, "unknown parameterization %d", (int)pz);
    if (!grads || !misfit) return fail(FWI_EINVAL, "null grads or misfit");
    if (src->ns > 0 && rec->nr > 0 && !data) return fail(FWI_EINVAL, "null data");
    static const float dummy = 0.f;
    return adjoint_impl(g, pz, xi_a, xi_b, src, rec, nullptr, data ? data : &dummy, misfit, grads, work,
                        work_bytes, static_cast<cudaStream_t>(stream), weights);
}

int fwi_gradient(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b, const fwi_sources *src,
                 const fwi_receivers *rec, const float *data, double *misfit, double *grads, void *work,
                 size_t work_bytes, void *stream)
{
    return fwi_gradient_weighted(g, pz, xi_a, xi_b, src, rec, data, nullptr, misfit, grads, work, work_bytes,
                                 stream);
}

int fwi_status(void *work, void *stream)
{
    if (!work) return fail(FWI_EINVAL, "null workspace");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int h = 0;
    CK(cudaMemcpyAsync(&h, work, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemsetAsync(work, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    if (h & fwi::ST_EINVAL) return fail(FWI_EINVAL, "a contrast has 1 + xi <= 0 or a position lies outside the physical grid");
    if (h & fwi::ST_ECFL) return fail(FWI_ECFL, "dt exceeds the stability limit of the stencil for this model");
    if (h & fwi::ST_EBOUNDS)
        return fail(FWI_EINVAL, "a bounds check of the checked build caught an out-of-range access (skipped)");
    return FWI_OK;
}

const char *fwi_last_error(void) { return g_err.c_str(); }

int fwi_misfit_weighted(const float *traces, const float *data, long long ntraces, int nt, const float *weights,
                        double *misfit, void *stream)
{
    g_err.clear();
    g_launches = 0;
    if (ntraces < 0 || nt < 1 || !misfit || (ntraces > 0 && (!traces || !data)))
        return fail(FWI_EINVAL, "invalid misfit arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LAUNCH(fwi::k_misfit, 1, fwi::RED_THREADS, 0, st, traces, data, ntraces * nt, weights, nt, misfit);
    return finish(st);
}

int fwi_misfit(const float *traces, const float *data, long long count, double *misfit, void *stream)
{
    if (count < 0) return fail(FWI_EINVAL, "invalid misfit arguments");
    return fwi_misfit_weighted(traces, data, count, 1, nullptr, misfit, stream);
}


int fwi_set_checkpoint(int every)
{
    if (every < 0) return fail(FWI_EINVAL, "checkpoint interval must be >= 0");
    g_ckpt_every = every;
    return FWI_OK;
}

int fwi_trace(int enable)
{
    if (enable < 0) return fail(FWI_EINVAL, "trace switch must be 0 or 1");
    g_trace.store(enable != 0);
    return FWI_OK;
}

int fwi_trace_report(char *buf, size_t len)
{
    std::string out;
    char line[96];
    for (int p = 0; p < PH_COUNT; ++p) {
        snprintf(line, sizeof line, "%s %lld\n", kPhaseName[p], g_trace_count[p].exchange(0));
        out += line;
    }
    if (buf && len) {
        strncpy(buf, out.c_str(), len - 1);
        buf[len - 1] = 0;
    }
    return (int)out.size();
}

int fwi_set_accumulation(int steps)
{
    if (steps < 0) return fail(FWI_EINVAL, "accumulation chunk must be >= 0 steps");
    g_acc_every = steps;
    return FWI_OK;
}

int fwi_set_tile(int tz, int variant)
{
    if (tz < 0 || variant < 0 || variant > 2)
        return fail(FWI_EINVAL, "tile height must be >= 0, variant 0, 1 or 2");
    g_tile_tz = tz;
    g_tile_variant = variant;
    return FWI_OK;
}

int fwi_profile(int enable)
{
    if (enable < 0) return fail(FWI_EINVAL, "profile sampling period must be >= 0");
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = enable != 0;
    g_prof.every = enable > 1 ? enable : 1;
    if (enable) g_prof.seen.assign(g_prof.seen.size(), 0);   // disabling keeps the counts for the report
    return FWI_OK;
}

int fwi_profile_report(char *buf, size_t len)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    std::vector<double> ms(g_prof.names.size(), 0.0);
    std::vector<long long> cnt(g_prof.names.size(), 0);
    int rc = FWI_OK;
    for (size_t k = 0; k < g_prof.used; ++k) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(g_prof.ev[2 * k + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, g_prof.ev[2 * k], g_prof.ev[2 * k + 1]);
        if (e != cudaSuccess) { rc = cuda_fail(e, "profile events"); break; }
        ms[g_prof.kind[k]] += t;
        ++cnt[g_prof.kind[k]];
    }
    g_prof.used = 0;
    std::string out;
    char line[256];
    for (size_t k = 0; k < g_prof.names.size(); ++k) {
        if (!cnt[k]) continue;
        const long long seen = k < g_prof.seen.size() ? g_prof.seen[k] : cnt[k];
        snprintf(line, sizeof line, "%s %lld %lld %.6f\n", g_prof.names[k].c_str(), seen, cnt[k], ms[k]);
        out += line;
    }
    g_prof.seen.assign(g_prof.seen.size(), 0);
    if (buf && len) {
        strncpy(buf, out.c_str(), len - 1);
        buf[len - 1] = 0;
    }
    return rc ? rc : (int)out.size();
}

long long fwi_launch_count(void) { return g_launches; }

}  // extern "C"
