// Host driver of libqubo.so: device workspace, kernel sequencing, the time limit, result merging,
// batches and wide instances, and the C ABI of qubo.h (the planning is in plan.cu).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <new>
#include <random>
#include <string>
#include <thread>
#include <unordered_set>
#include <utility>
#include <vector>

#include "../../include/qubo.h"
#include "internal.h"
#include "host.h"

using namespace qubo;
using namespace qubo::host;

namespace {

constexpr unsigned long long kDefaultRecCap = 1ull << 22;  // candidate records per job (64 MiB)
constexpr unsigned long long kBatchGraphRecords = 1ull << 18;  // candidate records of a replayed batch
// Run fn(lo, hi) over [0, count) split into contiguous ranges on up to one host thread per core,
// at least min_per_thread items per thread (small counts run on the calling thread).
template <class F>
void parallel_ranges(int count, int min_per_thread, F &&fn)
{
    const int nt = std::max(1, std::min<int>(count / std::max(1, min_per_thread),
                                             (int)std::thread::hardware_concurrency()));
    if (nt <= 1) {
        fn(0, count);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&fn, count, nt, t] {
            fn((int)((int64_t)count * t / nt), (int)((int64_t)count * (t + 1) / nt));
        });
    for (auto &x : th)
        x.join();
}

// ------------------------------------------------------------------------------------------------
// Encodings shared with the device (ordered integers for atomics).
// ------------------------------------------------------------------------------------------------

uint32_t ord32h(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
uint64_t ord64h(double d)
{
    uint64_t u;
    std::memcpy(&u, &d, 8);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
double bits_to_double(int64_t b)
{
    double d;
    std::memcpy(&d, &b, 8);
    return d;
}
double ubits_to_double(unsigned long long b)
{
    double d;
    std::memcpy(&d, &b, 8);
    return d;
}

unsigned long long encode_thr(Acc acc, double t)
{
    switch (acc) {
    case ACC_I32:
    case ACC_I32F:
    case ACC_I16P:
    case ACC_I32Z: return (unsigned long long)(uint32_t)(int32_t)t;
    case ACC_I64: return (unsigned long long)(int64_t)t;
    case ACC_F32:
    case ACC_F32Z: {
        float f = (float)t;
        if ((double)f < t)
            f = std::nextafter(f, INFINITY);
        return ord32h(f);
    }
    case ACC_F64: return ord64h(t);
    }
    return 0;
}

unsigned long long encode_max(Acc acc)
{
    switch (acc) {
    case ACC_I32:
    case ACC_I32F:
    case ACC_I16P:
    case ACC_I32Z: return (unsigned long long)(uint32_t)INT32_MAX;
    case ACC_I64: return (unsigned long long)INT64_MAX;
    case ACC_F32:
    case ACC_F32Z: return ord32h(INFINITY);
    case ACC_F64: return ord64h(INFINITY);
    }
    return 0;
}

// ------------------------------------------------------------------------------------------------
// Partial results and their merge (map-reduce of Sec. 3.3).
// ------------------------------------------------------------------------------------------------

struct Part {
    bool has = false;
    bool is_float = false;
    int64_t min_i = 0;
    double min_f = 0.0;
    uint64_t n_ties = 0, n_near = 0;
    std::vector<uint64_t> ties;                    // ascending, <= cap
    std::vector<std::pair<double, uint64_t>> topf;  // float: (E, code) ascending
    std::vector<std::pair<int64_t, uint64_t>> topi; // int
    uint64_t scanned = 0, candidates = 0;
    double drift = 0.0, err = 0.0;
    bool overflow = false;
    uint64_t dbg = 0;  // QUBO_DEBUG builds: site of the first failed device check
    // energy-window mode: every state with E <= min + window, (E, code) ascending (energies as
    // double; integer energies are exact in double below 2^53)
    std::vector<std::pair<double, uint64_t>> win;
};

bool part_less_min(const Part &a, const Part &b)
{
    return a.is_float ? a.min_f < b.min_f : a.min_i < b.min_i;
}
bool part_eq_min(const Part &a, const Part &b) { return a.is_float ? a.min_f == b.min_f : a.min_i == b.min_i; }

Part merge_parts(const Part &a, const Part &b, size_t cap, int K)
{
    if (!a.has)
        return b;
    if (!b.has)
        return a;
    Part o;
    o.has = true;
    o.is_float = a.is_float;
    o.scanned = a.scanned + b.scanned;
    o.candidates = a.candidates + b.candidates;
    o.drift = std::max(a.drift, b.drift);
    o.err = std::max(a.err, b.err);
    o.overflow = a.overflow || b.overflow;
    if (part_eq_min(a, b)) {
        o.min_i = a.min_i;
        o.min_f = a.min_f;
        o.n_ties = a.n_ties + b.n_ties;
        o.n_near = a.n_near + b.n_near;
        o.ties.resize(a.ties.size() + b.ties.size());
        std::merge(a.ties.begin(), a.ties.end(), b.ties.begin(), b.ties.end(), o.ties.begin());
        if (o.ties.size() > cap)
            o.ties.resize(cap);
    } else {
        const Part &w = part_less_min(a, b) ? a : b;
        o.min_i = w.min_i;
        o.min_f = w.min_f;
        o.n_ties = w.n_ties;
        o.n_near = w.n_near;
        o.ties = w.ties;
    }
    o.topf.resize(a.topf.size() + b.topf.size());
    std::merge(a.topf.begin(), a.topf.end(), b.topf.begin(), b.topf.end(), o.topf.begin());
    if ((int)o.topf.size() > K)
        o.topf.resize(K);
    o.topi.resize(a.topi.size() + b.topi.size());
    std::merge(a.topi.begin(), a.topi.end(), b.topi.begin(), b.topi.end(), o.topi.begin());
    if ((int)o.topi.size() > K)
        o.topi.resize(K);
    return o;
}

// Window lists of disjoint parts: union, then keep E <= merged minimum + window.  Each part's list
// holds every state of the part with E <= (its minimum) + window, a superset of its states within
// the merged window because the merged minimum is not larger.
void merge_windows(const Part &a, const Part &b, double window, Part &o)
{
    o.win.resize(a.win.size() + b.win.size());
    std::merge(a.win.begin(), a.win.end(), b.win.begin(), b.win.end(), o.win.begin());
    const double lim = o.min_f + window;
    size_t k = 0;
    while (k < o.win.size() && o.win[k].first <= lim)
        ++k;
    o.win.resize(k);
}

// ------------------------------------------------------------------------------------------------
// Device workspace: grow-only buffers per device, reused between calls.
// ------------------------------------------------------------------------------------------------

std::atomic<int> g_abort_all{0};

struct Workspace {
    int dev = -1;
    int sms = 0;
    void *d_arena = nullptr;
    size_t arena_cap = 0;
    Rec *d_rec = nullptr;
    unsigned long long rec_cap = 0;
    void *h_up = nullptr;
    size_t up_cap = 0;
    void *h_down = nullptr;
    size_t down_cap = 0;
    int *h_abort = nullptr;        // host-mapped flag read by the scan kernel
    const int *d_abort = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // tables start, scan end, finalize end, scan start
    std::mutex mu;

    ~Workspace() { release(); }

    void release()
    {
        if (dev < 0)
            return;
        int cur = -1;
        cudaGetDevice(&cur);
        cudaSetDevice(dev);
        if (d_arena)
            cudaFree(d_arena);
        if (d_rec)
            cudaFree(d_rec);
        if (h_up)
            cudaFreeHost(h_up);
        if (h_down)
            cudaFreeHost(h_down);
        if (h_abort)
            cudaFreeHost(h_abort);
        for (auto &e : ev)
            if (e)
                cudaEventDestroy(e);
        if (cur >= 0)
            cudaSetDevice(cur);
        d_arena = nullptr;
        d_rec = nullptr;
        h_up = h_down = nullptr;
        h_abort = nullptr;
        dev = -1;
    }

    int init(int device)
    {
        if (dev == device)
            return QUBO_OK;
        release();
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
            return QUBO_ERR_CUDA;
        sms = prop.multiProcessorCount;
        if (cudaHostAlloc((void **)&h_abort, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
            return QUBO_ERR_NOMEM;
        *h_abort = 0;
        int *dp = nullptr;
        if (cudaHostGetDevicePointer((void **)&dp, h_abort, 0) != cudaSuccess)
            return QUBO_ERR_CUDA;
        d_abort = dp;
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess)
                return QUBO_ERR_CUDA;
        dev = device;
        return QUBO_OK;
    }

    static int grow_dev(void **p, size_t *cap, size_t need)
    {
        if (*cap >= need)
            return QUBO_OK;
        if (*p)
            cudaFree(*p);
        *p = nullptr;
        *cap = 0;
        size_t sz = std::max(need, (size_t)1 << 20);
        if (cudaMalloc(p, sz) != cudaSuccess) {
            cudaGetLastError();
            return QUBO_ERR_NOMEM;
        }
        *cap = sz;
        return QUBO_OK;
    }
    static int grow_host(void **p, size_t *cap, size_t need)
    {
        if (*cap >= need)
            return QUBO_OK;
        if (*p)
            cudaFreeHost(*p);
        *p = nullptr;
        *cap = 0;
        size_t sz = std::max(need, (size_t)1 << 20);
        if (cudaMallocHost(p, sz) != cudaSuccess) {
            cudaGetLastError();
            return QUBO_ERR_NOMEM;
        }
        *cap = sz;
        return QUBO_OK;
    }
    int ensure(size_t arena, unsigned long long recs, size_t up, size_t down)
    {
        // fault injection for tests: QUBO_FAIL_ALLOC=1 makes every workspace request fail the
        // way an exhausted device or pinned-host pool does (nothing is freed or touched)
        const char *fail = std::getenv("QUBO_FAIL_ALLOC");
        if (fail && fail[0] == '1')
            return QUBO_ERR_NOMEM;
        int st;
        if ((st = grow_dev(&d_arena, &arena_cap, arena)))
            return st;
        if (rec_cap < recs) {
            if (d_rec)
                cudaFree(d_rec);
            d_rec = nullptr;
            rec_cap = 0;
            if (cudaMalloc((void **)&d_rec, sizeof(Rec) * recs) != cudaSuccess) {
                cudaGetLastError();
                return QUBO_ERR_NOMEM;
            }
            rec_cap = recs;
        }
        if ((st = grow_host(&h_up, &up_cap, up)))
            return st;
        return grow_host(&h_down, &down_cap, down);
    }
};

std::mutex g_ws_mu;
Workspace *g_ws[64] = {};
std::vector<Workspace *> g_all_ws;

Workspace *shared_workspace(int dev)
{
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if (dev < 0 || dev >= 64)
        return nullptr;
    if (!g_ws[dev]) {
        g_ws[dev] = new (std::nothrow) Workspace();
        if (g_ws[dev])
            g_all_ws.push_back(g_ws[dev]);
    }
    return g_ws[dev];
}

void register_ws(Workspace *w)
{
    std::lock_guard<std::mutex> lk(g_ws_mu);
    g_all_ws.push_back(w);
}
void unregister_ws(Workspace *w)
{
    std::lock_guard<std::mutex> lk(g_ws_mu);
    g_all_ws.erase(std::remove(g_all_ws.begin(), g_all_ws.end(), w), g_all_ws.end());
}

// Candidate-buffer records per job; QUBO_MAX_RECORDS lowers it (exercises the overflow path).
unsigned long long record_capacity()
{
    const char *v = std::getenv("QUBO_MAX_RECORDS");
    if (v) {
        const unsigned long long x = std::strtoull(v, nullptr, 10);
        if (x >= 1 && x < kDefaultRecCap)
            return x;
    }
    return kDefaultRecCap;
}



// Plans installed by the autotuner: (device, accumulator, n) -> (variant, walk bits); n = 0 is
// the entry used by batches.  Consulted when the caller fixes neither split_k nor walk_bits and
// QUBO_SCAN_VARIANT is unset.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tuned;

bool tuned_plan(Acc acc, int n, int *variant, int *walk)
{
    if (std::getenv("QUBO_SCAN_VARIANT"))
        return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find({dev, (int)acc, n});
    if (it == g_tuned.end())
        return false;
    *variant = it->second.first;
    *walk = it->second.second;
    return true;
}

void install_plan(Acc acc, int n, int variant, int walk)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[{dev, (int)acc, n}] = {variant, walk};
}

// Timing events: recorded as event nodes of the graph while the stream is being captured,
// plainly otherwise.
cudaError_t record_event(cudaEvent_t e, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t q = cudaStreamIsCapturing(s, &cs);
    if (q != cudaSuccess)
        return q;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                               : cudaEventRecord(e, s);
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            cudaGetLastError();                                                                    \
            return QUBO_ERR_CUDA;                                                                  \
        }                                                                                          \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ------------------------------------------------------------------------------------------------
// One job: a set of instances with one accumulator type, scanned by one persistent launch.
// ------------------------------------------------------------------------------------------------

struct Job {
    std::vector<HostInst *> insts;
    Acc acc = ACC_I32;
    int K = 0;
    size_t cap = 0;      // tie codes kept per instance
    double margin = 0.0;
    double time_limit = 0.0;
    int variant = 0;
    cudaStream_t stream = nullptr;
    // layout (byte offsets into the arena)
    size_t off_inst = 0, off_state = 0, off_items = 0, up_bytes = 0;
    size_t off_res = 0, off_ties = 0, off_topk = 0, off_topke = 0, off_starts = 0, off_ctr = 0;
    size_t arena_bytes = 0, down_bytes = 0;
    std::vector<size_t> off_W, off_W64, off_U64, off_Es, off_M, off_EL, off_perm;
    int max_entries = 0;
    int blocks = 0;
    unsigned long long rec_cap = 0;
    double t_start = 0.0;
    bool aborted = false;
    // accounting
    int launches = 0;
    uint64_t h2d = 0, d2h = 0;
    double scan_seconds = 0.0;
    uint64_t total_items = 0;
    double window = -1.0;  // >= 0: energy-window mode (single instance)
};

int job_layout(Job &j)
{
    const int ni = (int)j.insts.size();
    const int eb = acc_bytes(j.acc);
    size_t o = 0;
    j.off_inst = o;
    o = align_up(o + sizeof(Inst) * ni, 256);
    j.off_state = o;
    o = align_up(o + sizeof(InstState) * ni, 256);
    j.off_items = o;
    o = align_up(o + sizeof(uint64_t) * (ni + 1), 256);
    j.off_W.resize(ni);
    j.off_W64.resize(ni);
    j.off_U64.resize(ni);
    j.off_Es.resize(ni);
    j.off_M.resize(ni);
    j.off_EL.resize(ni);
    j.off_perm.assign(ni, 0);
    for (int i = 0; i < ni; ++i) {
        const HostInst &h = *j.insts[i];
        const size_t nn = (size_t)h.n * h.n;
        if (h.is_float) {
            j.off_W[i] = o;
            o = align_up(o + (size_t)eb * nn, 256);
            j.off_W64[i] = o;
            o = align_up(o + 8 * nn, 256);
            j.off_U64[i] = o;
            o = align_up(o + 8 * nn, 256);
        } else {
            j.off_W[i] = o;
            o = align_up(o + (size_t)eb * nn, 256);
        }
        if (acc_factored(j.acc) && !h.small) {  // scan order of the variables
            j.off_perm[i] = o;
            o = align_up(o + 64, 256);
        }
    }
    j.up_bytes = o;
    j.max_entries = 1;
    for (int i = 0; i < ni; ++i) {
        const HostInst &h = *j.insts[i];
        if (h.small)
            continue;
        const size_t NB = 1ull << h.B, NL = 1ull << h.L;
        j.off_Es[i] = o;
        o = align_up(o + eb * NB, 256);
        j.off_M[i] = o;
        o = align_up(o + eb * NB * h.L, 256);
        j.off_EL[i] = o;
        o = align_up(o + eb * (NL + NL / 16 + 1), 256);  // E_L, then its group minima (FP32 lanes)
        j.max_entries = std::max(j.max_entries, (int)(NB * (h.L + 1) + NL + NL / 16));
    }
    // results
    size_t d = 0;
    j.off_res = o;
    o = align_up(o + sizeof(ResOut) * ni, 256);
    j.off_ties = o;
    o = align_up(o + 8 * j.cap * ni, 256);
    j.off_topk = o;
    o = align_up(o + 8 * (size_t)j.K * ni, 256);
    j.off_topke = o;
    o = align_up(o + 8 * (size_t)j.K * ni, 256);
    j.off_starts = o;
    o = align_up(o + 16 * (size_t)ni, 256);
    j.off_ctr = o;
    o = align_up(o + 16 * 8, 256);
    j.arena_bytes = o;
    d = sizeof(ResOut) * ni + sizeof(InstState) * ni + 8 * j.cap * ni + 16 * (size_t)j.K * ni + 16 * 8 + 4096;
    j.down_bytes = d;
    return QUBO_OK;
}

// Lay out the job, size the workspace and fill the host staging buffer (descriptors, initial
// thresholds, item bases, coupling matrices).
int job_stage(Workspace &ws, Job &j, size_t extra_arena = 0)
{
    const int ni = (int)j.insts.size();
    int st;
    if ((st = job_layout(j)))
        return st;
    if ((st = ws.ensure(j.arena_bytes + extra_arena, kDefaultRecCap, j.up_bytes, j.down_bytes)))
        return st;
    char *up = (char *)ws.h_up;
    char *dev = (char *)ws.d_arena;
    Inst *hi = (Inst *)(up + j.off_inst);
    InstState *hs = (InstState *)(up + j.off_state);
    uint64_t *items = (uint64_t *)(up + j.off_items);
    uint64_t total = 0;
    for (int i = 0; i < ni; ++i) {
        items[i] = total;
        total += j.insts[i]->items;
    }
    items[ni] = total;
    // descriptors, initial state and coupling matrices; instances write disjoint regions
    auto stage_one = [&](int i) {
        HostInst &h = *j.insts[i];
        Inst d{};
        d.n = h.n;
        d.B = h.B;
        d.L = h.L;
        d.k = h.k;
        d.small = h.small;
        d.clampC = h.clampC;
        d.el_fused = j.acc == ACC_I16P ? h.el_fused : 0;
        d.elmin = h.elmin;
        d.geps = 0.0f;
        if (j.acc == ACC_F32) {  // 16 ulp of beta: every column and E_L value is at most beta
            const float b = (float)h.beta;
            d.geps = 16.0f * (std::nextafter(b, std::numeric_limits<float>::infinity()) - b);
        }
        d.unit_begin = h.unit_begin;
        d.units = h.units;
        d.sub_base = h.sub_base;
        d.sub_count = h.sub_count;
        if (h.is_float) {
            double *W64 = (double *)(up + j.off_W64[i]);
            double *U64 = (double *)(up + j.off_U64[i]);
            // the factored scan's tables and fields follow its scan order; the rescore reads the
            // caller's order (records carry the caller's codes)
            const bool permuted = j.acc == ACC_F32Z && !h.small;
            for (int a = 0; a < h.n; ++a)
                for (int b = 0; b < h.n; ++b) {
                    const int va = permuted ? h.perm[a] : a, vb = permuted ? h.perm[b] : b;
                    const int lo = std::min(va, vb), hi2 = std::max(va, vb);
                    const double w = h.Uf[(size_t)lo * h.n + hi2];
                    W64[(size_t)a * h.n + b] = w;
                    U64[(size_t)a * h.n + b] = h.Uf[(size_t)a * h.n + b];
                    if (j.acc == ACC_F32 || j.acc == ACC_F32Z)
                        ((float *)(up + j.off_W[i]))[(size_t)a * h.n + b] = (float)w;
                    else
                        ((double *)(up + j.off_W[i]))[(size_t)a * h.n + b] = w;
                }
            d.W = dev + j.off_W[i];
            d.W64 = (const double *)(dev + j.off_W64[i]);
            d.U64 = (const double *)(dev + j.off_U64[i]);
            if (permuted)
                std::memcpy(up + j.off_perm[i], h.perm.data(), h.n);
        } else {
            if (j.acc == ACC_I32Z && !h.small) {
                // the couplings in scan order: W[a][b] couples the variables perm[a] and perm[b]
                int32_t *W = (int32_t *)(up + j.off_W[i]);
                for (int a = 0; a < h.n; ++a)
                    for (int b = 0; b < h.n; ++b) {
                        const int va = h.perm[a], vb = h.perm[b];
                        W[(size_t)a * h.n + b] = (int32_t)h.Ui[(size_t)std::min(va, vb) * h.n + std::max(va, vb)];
                    }
                std::memcpy(up + j.off_perm[i], h.perm.data(), h.n);
            } else if (j.acc == ACC_I32 || j.acc == ACC_I32F || j.acc == ACC_I16P || j.acc == ACC_I32Z) {
                int32_t *W = (int32_t *)(up + j.off_W[i]);
                for (int a = 0; a < h.n; ++a)
                    for (int b = 0; b < h.n; ++b)
                        W[(size_t)a * h.n + b] = (int32_t)h.Ui[(size_t)std::min(a, b) * h.n + std::max(a, b)];
            } else {
                int64_t *W = (int64_t *)(up + j.off_W[i]);
                for (int a = 0; a < h.n; ++a)
                    for (int b = 0; b < h.n; ++b)
                        W[(size_t)a * h.n + b] = h.Ui[(size_t)std::min(a, b) * h.n + std::max(a, b)];
            }
            d.W = dev + j.off_W[i];
            d.W64 = nullptr;
            d.U64 = nullptr;
        }
        d.Es = h.small ? nullptr : dev + j.off_Es[i];
        d.M = h.small ? nullptr : dev + j.off_M[i];
        d.EL = h.small ? nullptr : dev + j.off_EL[i];
        d.thr0 = 0;
        d.Z = h.Z;
        d.anchor = j.acc == ACC_F32 ? h.anchor_bits : 0;
        d.perm = (acc_factored(j.acc) && !h.small) ? (const uint8_t *)(dev + j.off_perm[i]) : nullptr;
        hi[i] = d;
        InstState s{};
        s.thr = encode_thr(j.acc, h.thr0);
        s.gmin = encode_max(j.acc);
        hs[i] = s;
    };
    parallel_ranges(ni, 64, [&](int lo, int hi) {
        for (int i = lo; i < hi; ++i)
            stage_one(i);
    });
    j.total_items = total;
    j.rec_cap = std::min(ws.rec_cap, record_capacity());
    int bps = scan_blocks_per_sm(j.acc, j.K <= 1, j.variant);
    if (bps < 1)
        bps = 1;
    j.blocks = ws.sms * bps;
    const uint64_t need_blocks = (total * 32 + kScanThreads - 1) / kScanThreads;
    if ((uint64_t)j.blocks > need_blocks)
        j.blocks = (int)std::max<uint64_t>(1, need_blocks);
    return QUBO_OK;
}

// Enqueue the run's inputs and the table build and scan on j.stream.  With state_init set, the
// descriptors are already on the device and the per-run state is copied from state_init
// (device to device), so the sequence can be captured and replayed as a graph.
int job_enqueue_scan(Workspace &ws, Job &j, const void *state_init = nullptr)
{
    const int ni = (int)j.insts.size();
    char *up = (char *)ws.h_up;
    char *dev = (char *)ws.d_arena;
    cudaStream_t s = j.stream;
    if (state_init) {
        CK(cudaMemcpyAsync(dev + j.off_state, state_init, sizeof(InstState) * ni, cudaMemcpyDeviceToDevice, s));
    } else {
        CK(cudaMemcpyAsync(dev, up, j.up_bytes, cudaMemcpyHostToDevice, s));
        j.h2d += j.up_bytes;
    }
    CK(cudaMemsetAsync(dev + j.off_ctr, 0, 16 * 8, s));
    CK(record_event(ws.ev[0], s));
    CK(launch_tables(j.acc, (const Inst *)(dev + j.off_inst), ni, j.max_entries, s));
    CK(record_event(ws.ev[3], s));
    ScanArgs a{};
    a.inst = (const Inst *)(dev + j.off_inst);
    a.state = (InstState *)(dev + j.off_state);
    a.item_base = (const uint64_t *)(dev + j.off_items);
    a.n_inst = ni;
    a.k1 = j.K <= 1 ? 1 : 0;
    a.total_items = j.total_items;
    a.queue = (unsigned long long *)(dev + j.off_ctr);
    a.rec = ws.d_rec;
    a.rec_cap = j.rec_cap;
    a.nrec = (unsigned long long *)(dev + j.off_ctr) + 1;
    a.abort_flag = ws.d_abort;
    a.margin = acc_float(j.acc) ? j.margin : 0.0;
    if (j.window >= 0.0)  // record everything within the window of the running minimum
        a.margin += acc_float(j.acc) ? j.window : std::floor(j.window);
    a.zero = 0;
    CK(launch_scan(j.acc, a, j.blocks, j.variant, s));
    CK(record_event(ws.ev[1], s));
    j.launches += 2;
    return QUBO_OK;
}

// Stage, upload and launch tables + scan.  Does not wait.
int job_launch(Workspace &ws, Job &j)
{
    int st;
    if ((st = job_stage(ws, j)))
        return st;
    *ws.h_abort = g_abort_all.load() ? 1 : 0;
    if ((st = job_enqueue_scan(ws, j)))
        return st;
    j.t_start = now_s();
    return QUBO_OK;
}

// Wait for `ev` (the scan's end), honouring the time limit and qubo_abort.
int job_wait(Workspace &ws, Job &j, cudaEvent_t ev)
{
    for (;;) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess)
            break;
        if (q != cudaErrorNotReady) {
            cudaGetLastError();
            return QUBO_ERR_CUDA;
        }
        const bool over = j.time_limit > 0 && now_s() - j.t_start > j.time_limit;
        if ((over || g_abort_all.load()) && !*(volatile int *)ws.h_abort) {
            *(volatile int *)ws.h_abort = 1;
            j.aborted = true;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    if (*(volatile int *)ws.h_abort)
        j.aborted = true;
    return QUBO_OK;
}

// Host-side view of the download staging buffer.
struct Down {
    ResOut *res;
    InstState *sts;
    uint64_t *ties, *tk;
    int64_t *tke;
};

Down down_view(Workspace &ws, const Job &j)
{
    const int ni = (int)j.insts.size();
    char *down = (char *)ws.h_down;
    Down d;
    size_t o = 0;
    d.res = (ResOut *)(down + o);
    o += sizeof(ResOut) * ni;
    d.sts = (InstState *)(down + o);
    o += sizeof(InstState) * ni;
    d.ties = (uint64_t *)(down + o);
    o += 8 * j.cap * ni;
    d.tk = (uint64_t *)(down + o);
    o += 8 * (size_t)j.K * ni;
    d.tke = (int64_t *)(down + o);
    return d;
}

// Enqueue rescoring (floats), the sort of the candidate records, extraction and the download
// of the results.  max_pow2 bounds the sort network; the kernels read the record count on the
// device, so a larger bound only costs empty launches (this is what a captured graph uses).
int job_enqueue_finalize(Workspace &ws, Job &j, unsigned long long max_count, unsigned long long max_pow2)
{
    const int ni = (int)j.insts.size();
    char *dev = (char *)ws.d_arena;
    cudaStream_t s = j.stream;
    const bool batched = ni > 1;
    const bool is_float = acc_float(j.acc);
    const unsigned long long *d_nrec = (const unsigned long long *)(dev + j.off_ctr) + 1;
    if (is_float) {
        CK(launch_rescore((const Inst *)(dev + j.off_inst), (InstState *)(dev + j.off_state), ws.d_rec, d_nrec,
                          j.rec_cap, batched, max_count, s));
        j.launches += 1;
    }
    CK(launch_sort(ws.d_rec, d_nrec, j.rec_cap, max_pow2, batched, is_float, s, &j.launches));
    j.launches += 2;  // bounds + extract
    CK(launch_extract((const Inst *)(dev + j.off_inst), ws.d_rec, d_nrec, j.rec_cap, ni, batched, is_float, j.K,
                      j.cap, (ResOut *)(dev + j.off_res), (uint64_t *)(dev + j.off_ties),
                      (uint64_t *)(dev + j.off_topk), (int64_t *)(dev + j.off_topke),
                      (unsigned long long *)(dev + j.off_starts), s));
    CK(record_event(ws.ev[2], s));
    const Down d = down_view(ws, j);
    CK(cudaMemcpyAsync(d.res, dev + j.off_res, sizeof(ResOut) * ni, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(d.sts, dev + j.off_state, sizeof(InstState) * ni, cudaMemcpyDeviceToHost, s));
    if (j.cap)
        CK(cudaMemcpyAsync(d.ties, dev + j.off_ties, 8 * j.cap * ni, cudaMemcpyDeviceToHost, s));
    if (j.K) {
        CK(cudaMemcpyAsync(d.tk, dev + j.off_topk, 8 * (size_t)j.K * ni, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(d.tke, dev + j.off_topke, 8 * (size_t)j.K * ni, cudaMemcpyDeviceToHost, s));
    }
    j.d2h += sizeof(ResOut) * ni + sizeof(InstState) * ni + (j.cap ? 8 * j.cap * ni : 0) + 16 * (size_t)j.K * ni;
    return QUBO_OK;
}

Part part_from(const Down &d, const Job &j, int i);

// After the stream has finished: timings and per-instance results from the staging buffer.
void job_unpack(Workspace &ws, Job &j, std::vector<Part> &parts, double *gpu_seconds)
{
    const int ni = (int)j.insts.size();
    const bool is_float = acc_float(j.acc);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ws.ev[0], ws.ev[2]) == cudaSuccess && gpu_seconds)
        *gpu_seconds = ms * 1e-3;
    if (cudaEventElapsedTime(&ms, ws.ev[3], ws.ev[1]) == cudaSuccess)
        j.scan_seconds = ms * 1e-3;
    const Down d = down_view(ws, j);
    parts.assign(ni, Part());
    for (int i = 0; i < ni; ++i)
        parts[i] = part_from(d, j, i);
}

// Per-instance result of a finished job, read from the download staging buffer.
Part part_from(const Down &d, const Job &j, int i)
{
    const bool is_float = acc_float(j.acc);
    Part p;
    {
        const ResOut &r = d.res[i];
        p.is_float = is_float;
        p.has = r.has != 0;
        p.min_i = r.min_i;
        p.min_f = is_float ? r.min_f : (double)r.min_i;
        p.n_ties = r.n_ties;
        p.n_near = r.n_near;
        p.ties.assign(d.ties + (size_t)i * j.cap, d.ties + (size_t)i * j.cap + r.n_written);
        for (int t = 0; t < r.nk; ++t) {
            const uint64_t c = d.tk[(size_t)i * j.K + t];
            const int64_t e = d.tke[(size_t)i * j.K + t];
            if (is_float)
                p.topf.emplace_back(bits_to_double(e), c);
            else
                p.topi.emplace_back(e, c);
        }
        p.scanned = d.sts[i].scanned;
        p.candidates = d.sts[i].nrec;
        p.drift = ubits_to_double(d.sts[i].drift);
        p.err = ubits_to_double(d.sts[i].err);
        p.overflow = d.sts[i].dropped > 0;
        p.dbg = d.sts[i].dbg;
    }
    return p;
}

// Wait for the scan, finalize with the exact record count, download and unpack.
int job_finish(Workspace &ws, Job &j, std::vector<Part> &parts, double *gpu_seconds)
{
    char *dev = (char *)ws.d_arena;
    int st;
    if ((st = job_wait(ws, j, ws.ev[1])))
        return st;
    unsigned long long nrec = 0;
    CK(cudaMemcpy(&nrec, dev + j.off_ctr + 8, 8, cudaMemcpyDeviceToHost));
    j.d2h += 8;
    const unsigned long long cnt = std::min(nrec, j.rec_cap);
    unsigned long long P = 1;
    while (P < cnt)
        P <<= 1;
    if ((st = job_enqueue_finalize(ws, j, cnt, P)))
        return st;
    std::vector<Rec> sorted;
    if (j.window >= 0.0 && cnt) {
        sorted.resize(cnt);
        CK(cudaMemcpyAsync(sorted.data(), ws.d_rec, sizeof(Rec) * cnt, cudaMemcpyDeviceToHost, j.stream));
        j.d2h += sizeof(Rec) * cnt;
    }
    CK(cudaStreamSynchronize(j.stream));
    job_unpack(ws, j, parts, gpu_seconds);
    for (size_t i = 0; i < parts.size(); ++i)
        if (parts[i].dbg) {
#ifdef QUBO_DEBUG
            std::fprintf(stderr, "qubo: device check %llu failed (instance %zu of the launch)\n",
                         (unsigned long long)parts[i].dbg, i);
#endif
            return QUBO_ERR_INTERNAL;
        }
    if (j.window >= 0.0 && !parts.empty() && parts[0].has) {
        Part &p = parts[0];
        const bool fl = acc_float(j.acc);
        const double lim = p.min_f + j.window;
        for (const Rec &r : sorted) {
            const double e = fl ? bits_to_double(r.e) : (double)r.e;
            if (e > lim)
                break;
            p.win.emplace_back(e, r.key);
        }
    }
    return j.aborted ? QUBO_ERR_TIMEOUT : QUBO_OK;
}

struct SolveCfg {
    double window = -1.0;
    int K = 0;
    size_t cap = 0;
    uint32_t flags = 0;
    double margin = kDefaultMargin;
    double time_limit = 0.0;
    int split_k = 0, walk_bits = 0;
    int variant = -1;  // < 0: the accumulator's default (or QUBO_SCAN_VARIANT)
};

struct SolveStats {
    double gpu_seconds = 0.0;
    double scan_seconds = 0.0;
    int passes = 0;
    int blocks = 0;
    int launches = 0;
    uint64_t h2d = 0, d2h = 0;
    void add(const Job &j, double gs)
    {
        gpu_seconds += gs;
        scan_seconds += j.scan_seconds;
        passes += 1;
        blocks = std::max(blocks, j.blocks);
        launches += j.launches;
        h2d += j.h2d;
        d2h += j.d2h;
    }
};

// Solve the sub-cube (fix_bits, fix_value) of one prepared instance.  When the candidate buffer
// overflows, the sub-cube is split in two along its next code bit and both halves are solved
// and merged, down to halves small enough to fit.
int solve_range(Workspace &ws, HostInst &h, int fix_bits, uint64_t fix_value, const SolveCfg &c,
                cudaStream_t stream, Part &out, SolveStats &stats, double t_deadline)
{
    int st = plan_run(h, fix_bits, fix_value, c.split_k, c.walk_bits, c.variant, c.flags, c.margin);
    if (st)
        return st;
    h.thr0 = threshold_bound(h, std::max(1, c.K));
    Job j;
    j.insts = {&h};
    j.acc = h.acc;
    j.K = c.K;
    j.cap = c.cap;
    j.margin = c.margin;
    j.time_limit = t_deadline > 0 ? std::max(1e-3, t_deadline - now_s()) : 0.0;
    j.variant = h.variant;
    j.stream = stream;
    j.window = c.window;
    if ((st = job_launch(ws, j)))
        return st;
    std::vector<Part> parts;
    double gs = 0.0;
    st = job_finish(ws, j, parts, &gs);
    stats.add(j, gs);
    if (st)
        return st;
    Part p = parts[0];
    if (!p.overflow) {
        out = p;
        return QUBO_OK;
    }
    if (fix_bits >= h.n)
        return QUBO_ERR_INTERNAL;  // a single state cannot overflow the buffer
    Part a, b;
    if ((st = solve_range(ws, h, fix_bits + 1, fix_value << 1, c, stream, a, stats, t_deadline)))
        return st;
    if ((st = solve_range(ws, h, fix_bits + 1, (fix_value << 1) | 1, c, stream, b, stats, t_deadline)))
        return st;
    out = merge_parts(a, b, c.cap, c.K);
    if (c.window >= 0.0)
        merge_windows(a, b, c.window, out);
    return QUBO_OK;
}

// FP32 scans: the candidate margin must cover twice the measured drift plus the rounding of the
// per-step threshold arithmetic (a few FP32 operations on values bounded by beta; the factored
// scan's E_L plus up to 14 zero-row couplings, more).  Otherwise the caller rescans with a
// shorter walk, the dense FP32 scan, or FP64.
bool float_margin_ok(const HostInst &h, const Part &p, double margin)
{
    if (h.acc != ACC_F32 && h.acc != ACC_F32Z)
        return true;
    const double slack = (h.acc == ACC_F32Z ? 32.0 : 8.0) * std::ldexp(1.0, -24) * (1.0 + h.beta);
    return 2.0 * p.drift + slack < margin;
}

void fill_outputs(const HostInst &h, const Part &p, int K, size_t cap, void *out_min, uint64_t *out_states,
                  uint64_t *out_topk, void *out_topk_E, qubo_result *info)
{
    if (out_min) {
        if (h.is_float)
            *(double *)out_min = p.min_f;
        else
            *(int64_t *)out_min = p.min_i;
    }
    const size_t nw = std::min(cap, p.ties.size());
    if (out_states)
        for (size_t t = 0; t < nw; ++t)
            out_states[t] = p.ties[t];
    const int nk = h.is_float ? (int)p.topf.size() : (int)p.topi.size();
    if (K > 0 && out_topk)
        for (int t = 0; t < nk && t < K; ++t) {
            out_topk[t] = h.is_float ? p.topf[t].second : p.topi[t].second;
            if (out_topk_E) {
                if (h.is_float)
                    ((double *)out_topk_E)[t] = p.topf[t].first;
                else
                    ((int64_t *)out_topk_E)[t] = p.topi[t].first;
            }
        }
    if (info) {
        info->min_i = h.is_float ? (int64_t)0 : p.min_i;
        info->min_f = p.min_f;
        info->n_ties = p.n_ties;
        info->n_written = nw;
        info->truncated = p.n_ties > cap ? 1 : 0;
        info->acc = (int32_t)h.acc;
        info->n_topk = std::min(nk, K);
        info->fp32_max_abs_err = h.is_float ? p.err : 0.0;
        info->fp32_max_drift = h.is_float ? p.drift : 0.0;
        info->n_near_ties = p.n_near;
        info->states_scanned = p.scanned;
        info->candidates = p.candidates;
    }
}

int resolve_device(Workspace **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QUBO_ERR_CUDA;
    }
    Workspace *w = shared_workspace(dev);
    if (!w)
        return QUBO_ERR_NOMEM;
    *out = w;
    return QUBO_OK;
}

int check_opts(const qubo_options *o, size_t states_cap, const uint64_t *out_states, const uint64_t *out_topk)
{
    if (o->topk < 0 || o->topk > QUBO_MAX_TOPK)
        return QUBO_ERR_ARG;
    if (states_cap > 0 && !out_states)
        return QUBO_ERR_ARG;
    if (o->topk > 0 && !out_topk)
        return QUBO_ERR_ARG;
    return QUBO_OK;
}

// Configuration of one solve from the caller's options: the tuned plan for this size (when the
// caller fixes neither split_k nor walk_bits) or the accumulator's default variant.
SolveCfg solve_cfg(const HostInst &h, const qubo_options &o, size_t states_cap, double window)
{
    SolveCfg c;
    c.window = window;
    c.K = o.topk;
    c.cap = states_cap;
    c.flags = o.flags;
    c.margin = o.margin > 0 ? o.margin : kDefaultMargin;
    c.time_limit = o.time_limit_s;
    c.split_k = o.split_k;
    c.walk_bits = o.walk_bits;
    c.variant = std::getenv("QUBO_SCAN_VARIANT") ? scan_variant(h.acc) : -1;
    c.flags = o.flags;
    if (o.split_k <= 0 && o.walk_bits <= 0 && acc_bytes(h.acc) == 4) {
        int tv = 0, tw = 0;
        if (tuned_plan(h.acc, h.n, &tv, &tw)) {
            c.variant = tv;
            HostInst probe = h;
            probe.variant = tv;
            if (plan(probe, o.fix_bits, o.fix_value, 0, tw) == QUBO_OK)
                c.walk_bits = tw;
        }
    }
    return c;
}

int solve_one(Workspace &ws, HostInst &h, const qubo_options &o, size_t states_cap, cudaStream_t stream, Part &p,
              SolveStats &stats, double window = -1.0)
{
    SolveCfg c = solve_cfg(h, o, states_cap, window);
    const double deadline = o.time_limit_s > 0 ? now_s() + o.time_limit_s : 0.0;
    int st = solve_range(ws, h, o.fix_bits, o.fix_value, c, stream, p, stats, deadline);
    if (st)
        return st;
    // FP32 drift above the margin's budget: shorten the re-anchoring period, and as a last resort
    // rescan in FP64.
    while (!float_margin_ok(h, p, c.margin)) {
        const int period = std::min(h.anchor_bits, h.L);
        if (h.acc == ACC_F32Z) {  // the dense FP32 scan next
            h.no_factored = true;
            h.acc = ACC_F32;
            c.walk_bits = o.walk_bits;
        } else if (h.acc == ACC_F32 && !h.small && period > variant_reg_rows(h) + 1) {
            h.anchor_bits = std::max(variant_reg_rows(h) + 1, period - 2);
        } else {
            h.acc = ACC_F64;
            c.walk_bits = o.walk_bits;
        }
        p = Part();
        st = solve_range(ws, h, o.fix_bits, o.fix_value, c, stream, p, stats, deadline);
        if (st)
            return st;
        if (h.acc == ACC_F64)
            break;
    }
    const uint64_t expect = 1ull << (h.n - o.fix_bits);
    if (p.scanned != expect || !p.has)
        return QUBO_ERR_INTERNAL;
    return QUBO_OK;
}

void fill_plan_info(const HostInst &h, const SolveStats &stats, double t0, qubo_result *info)
{
    if (!info)
        return;
    info->seconds = now_s() - t0;
    info->seconds_gpu = stats.gpu_seconds;
    info->seconds_scan = stats.scan_seconds;
    info->kernel_launches = stats.launches;
    info->h2d_bytes = stats.h2d;
    info->d2h_bytes = stats.d2h;
    info->states_per_s = info->seconds > 0 ? (double)info->states_scanned / info->seconds : 0.0;
    info->n = h.n;
    info->split_k = h.k;
    info->walk_bits = h.L;
    info->suffix_bits = h.small ? 0 : h.B;
    info->cols_per_thread = h.small ? 0 : acc_cols_per_thread(h.acc, h.variant);
    info->reg_rows = h.small ? 0 : variant_reg_rows(h);
    info->variant = h.small || acc_factored(h.acc) ? -1 : h.variant;
    info->grouped = !h.small && grouped_form(h.acc, h.variant);
    info->fp32_err_bound = 0.0;  // single-instance calls fill these in (fill_fp32_bound)
    info->fp32_rigorous_anchor_bits = -1;
    info->zero_rows = acc_factored(h.acc) ? h.Z : 0;
    info->anchor_bits = (h.acc == ACC_F32 && !h.small) ? std::min(h.anchor_bits, h.L) : 0;
    info->threads = kScanThreads;
    info->blocks = stats.blocks;
    info->passes = stats.passes;
}

// The FP32 scan's worst-case rounding bound at the run's re-anchoring period and the longest
// period at which it alone proves the candidates (single-instance results).
void fill_fp32_bound(const HostInst &h, double margin, qubo_result *info)
{
    if (!info)
        return;
    info->fp32_err_bound = 0.0;
    info->fp32_rigorous_anchor_bits = -1;
    if (h.acc != ACC_F32 || h.small)
        return;
    info->fp32_err_bound = fp32_error_bound(h, std::min(h.anchor_bits, h.L), margin);
    info->fp32_rigorous_anchor_bits = fp32_rigorous_anchor_bits(h, margin);
}

int batch_plan(std::vector<HostInst> &hs, int topk, std::vector<int> &order);

// Walk length of a batched instance in (acc, variant): the walk the batch autotuner installed
// for its size under this variant, else as long as the instance allows (at most wmax); 0 when
// the instance is too small to split.  h.acc and h.variant must be set.
int batch_walk(Acc acc, int variant, const HostInst &h, int wmax)
{
    const int B = acc_suffix_bits(acc, variant);
    const int rmin = variant_reg_rows(h) + 1;
    if (h.n - B < rmin)
        return 0;
    int walk = std::min(wmax, h.n - B);
    int tv = 0, tw = 0;
    if (tuned_plan(acc, -h.n, &tv, &tw) && tv == variant && tw >= rmin && tw <= walk)
        walk = tw;
    return walk;
}

// Fold, bound, plan and threshold every instance of a batch (in parallel on the host), one
// accumulator for all, and the launch order (longest work first, so the persistent launch's
// tail is short).
int batch_prepare(const void *Q_packed, const int *n, const size_t *offsets, int count, qubo_dtype dtype, int topk,
                  std::vector<HostInst> &hs, std::vector<int> &order)
{
    const size_t esz = dtype == QUBO_I16 ? 2 : (dtype == QUBO_I32 || dtype == QUBO_F32) ? 4 : 8;
    hs.assign(count, HostInst());
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || n[i] > kMaxBatchedN)
            return QUBO_ERR_ARG;
        if (topk > 0 && (uint64_t)topk > (1ull << n[i]))
            return QUBO_ERR_ARG;
    }
    // Host preparation (fold, bound, threshold) of the instances, in parallel.
    std::vector<int> pst(count, QUBO_OK);
    auto prep_range = [&](int lo, int hi) {
        for (int i = lo; i < hi; ++i)
            pst[i] = prepare((const char *)Q_packed + offsets[i] * esz, n[i], dtype, 0, hs[i]);
    };
    auto parallel = [&](auto &&fn) { parallel_ranges(count, 64, fn); };
    parallel(prep_range);
    for (int i = 0; i < count; ++i)
        if (pst[i])
            return pst[i];
    return batch_plan(hs, topk, order);
}

// Plan every prepared instance of a batch (in parallel on the host): one accumulator for all,
// thresholds, and the launch order (longest work first, so the persistent launch's tail is
// short).
int batch_plan(std::vector<HostInst> &hs, int topk, std::vector<int> &order)
{
    const int count = (int)hs.size();
    std::vector<int> pst(count, QUBO_OK);
    auto parallel = [&](auto &&fn) { parallel_ranges(count, 64, fn); };
    // one accumulator for the whole batch: the widest any instance needs
    Acc acc = hs[0].acc;
    for (auto &h : hs)
        if (acc_bytes(h.acc) > acc_bytes(acc))
            acc = h.acc;
    for (auto &h : hs)
        h.acc = acc;
    // The batch supplies the parallelism, so every instance walks as long as it can (fewest,
    // largest units: less per-unit set-up).
    int variant = scan_variant(acc);
    {
        int tv = 0, tw = 0;
        if (tuned_plan(acc, 0, &tv, &tw))
            variant = tv;
    }
    auto plan_range = [&](int lo, int hi) {
        for (int i = lo; i < hi; ++i) {
            HostInst &h = hs[i];
            h.variant = acc_bytes(acc) == 4 ? variant : 0;
            const int wmax = acc == ACC_F32 ? kFloatMaxWalkBits : kDefaultMaxWalkBits;
            pst[i] = plan(h, 0, 0, 0, batch_walk(acc, h.variant, h, wmax));
            // batches are many small instances: fewer descents (K = 1 thresholds also tighten on
            // the device as soon as a lower state is found)
            if (!pst[i])
                h.thr0 = threshold_bound(h, std::max(1, topk), topk > 1 ? 16 : 6);
        }
    };
    parallel(plan_range);
    for (int i = 0; i < count; ++i)
        if (pst[i])
            return pst[i];
    // One accumulator for the batch: packed 16-bit lanes, else FP32 lanes (2^14-step walks, else
    // 2^12), when every instance's plan is exact in it (instances evaluated directly need nothing).
    const std::pair<Acc, int> alts[] = {
        {ACC_I16P, kDefaultMaxWalkBits}, {ACC_I32F, kI32FMaxWalkBits}, {ACC_I32F, kDefaultMaxWalkBits}};
    for (const auto &[alt_acc, alt_walk] : alts) {
        if (acc != ACC_I32)
            break;
        if (!(alt_acc == ACC_I16P ? i16p_allowed() : i32f_allowed()))
            continue;
        // plan in place; the previous plans are kept (not the matrices) to restore on failure
        std::vector<PlanFields> saved(count);
        for (int i = 0; i < count; ++i)
            saved[i] = plan_fields(hs[i]);
        int v2 = pick_variant(alt_acc, -1);
        int tv = 0, tw = 0;
        if (tuned_plan(alt_acc, 0, &tv, &tw))
            v2 = tv;
        std::atomic<bool> all{true};
        auto alt_range = [&](int lo, int hi) {
            for (int i = lo; i < hi && all.load(std::memory_order_relaxed); ++i) {
                HostInst &h = hs[i];
                h.acc = alt_acc;
                h.variant = v2;
                const bool ok = plan(h, 0, 0, 0, batch_walk(alt_acc, v2, h, alt_walk)) == QUBO_OK &&
                                (h.small || (alt_acc == ACC_I16P ? i16p_exact(h) : i32f_exact(h, &h.clampC)));
                if (!ok)
                    all = false;
                else if (alt_acc == ACC_I16P)
                    i16p_fuse_el(h);
            }
        };
        parallel(alt_range);
        if (all && alt_acc == ACC_I16P) {
            // one kernel for the batch: the fused-only twin when every instance's E_L is fused
            bool fused = true;
            for (const HostInst &h : hs)
                fused = fused && (h.small || h.el_fused);
            const int v3 = packed_variant_for(v2, fused);
            for (HostInst &h : hs)
                h.variant = v3;
        }
        if (all)
            break;
        for (int i = 0; i < count; ++i)
            set_plan_fields(hs[i], saved[i]);
    }
    // longest work first (LPT order) so the tail of the persistent launch is short
    order.resize(count);
    for (int i = 0; i < count; ++i)
        order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hs[a].states > hs[b].states; });
    return QUBO_OK;
}

// Solve a planned batch in one persistent launch; parts[i] is instance i's result.  An instance
// that overflowed the shared candidate buffer (or whose FP32 drift used up the margin) is solved
// again alone.
int batch_parts(Workspace &ws, std::vector<HostInst> &hs, const std::vector<int> &order, int topk, size_t cap,
                cudaStream_t stream, std::vector<Part> &parts, SolveStats &stats)
{
    const int count = (int)hs.size();
    Job j;
    for (int i : order)
        j.insts.push_back(&hs[i]);
    j.acc = hs[0].acc;
    j.K = topk;
    j.cap = cap;
    j.margin = kDefaultMargin;
    j.variant = hs[0].variant;
    j.stream = stream;
    int st;
    if ((st = job_launch(ws, j)))
        return st;
    std::vector<Part> run_parts;
    double gs = 0.0;
    if ((st = job_finish(ws, j, run_parts, &gs)))
        return st;
    stats.add(j, gs);
    SolveCfg c;
    c.K = topk;
    c.cap = cap;
    c.variant = j.variant;
    parts.assign(count, Part());
    for (int r = 0; r < count; ++r) {
        const int i = order[r];
        Part &p = run_parts[r];
        HostInst &h = hs[i];
        if (p.overflow || !float_margin_ok(h, p, c.margin)) {
            // rare: this instance overflowed the shared candidate buffer; solve it alone
            if (!float_margin_ok(h, p, c.margin))
                h.acc = ACC_F64;
            p = Part();
            if ((st = solve_range(ws, h, 0, 0, c, stream, p, stats, 0.0)))
                return st;
        }
        if (p.scanned != (1ull << h.n) || !p.has)
            return QUBO_ERR_INTERNAL;
        parts[i] = std::move(p);
    }
    return QUBO_OK;
}

// Prepare an instance given directly as its folded upper-triangular matrix (a sub-problem of a
// larger instance): bound check and accumulator as in prepare().
int prepare_folded(std::vector<int64_t> *Ui, std::vector<double> *Uf, int n, uint32_t flags, HostInst &h)
{
    h = HostInst();
    h.n = n;
    h.is_float = Uf != nullptr;
    if (h.is_float) {
        h.Uf = std::move(*Uf);
        for (double v : h.Uf)
            h.beta += std::fabs(v);
        h.acc = (flags & QUBO_FLAG_PLAIN) ? ACC_F64 : ACC_F32;
        return QUBO_OK;
    }
    h.Ui = std::move(*Ui);
    int64_t beta = 0;
    for (int64_t v : h.Ui) {
        beta += v < 0 ? -v : v;
        if (beta >= (1ll << 62))
            return QUBO_ERR_OVERFLOW;
    }
    h.beta = (double)beta;
    h.acc = ((flags & QUBO_FLAG_PLAIN) || beta >= (1ll << 30)) ? ACC_I64 : ACC_I32;
    return QUBO_OK;
}

// Result over many sub-problems of a wide instance, with 128-bit state codes (lo, hi words).
struct WideAcc {
    bool has = false;
    bool is_float = false;
    int64_t min_i = 0;
    double min_f = 0.0;
    uint64_t n_ties = 0, scanned = 0, candidates = 0;
    std::vector<std::pair<uint64_t, uint64_t>> ties;  // (hi, lo), ascending
    std::vector<std::tuple<double, uint64_t, uint64_t>> topf;  // (E, hi, lo)
    std::vector<std::tuple<int64_t, uint64_t, uint64_t>> topi;
};

// Fold a sub-problem result (inner codes, energies without the constant c) into the wide result.
// Sub-problems must arrive in ascending outer value so that the tie codes stay ascending.
void wide_add(WideAcc &w, const Part &p, int n_in, uint64_t outer, int64_t ci, double cf, size_t cap, int K)
{
    auto code = [&](uint64_t inner) {
        const uint64_t lo = n_in == 64 ? inner : (inner | (outer << n_in));
        const uint64_t hi = n_in == 0 ? 0 : (n_in == 64 ? outer : (outer >> (64 - n_in)));
        return std::make_pair(hi, lo);
    };
    const bool fl = p.is_float;
    const int64_t Ei = p.min_i + ci;
    const double Ef = p.min_f + cf;
    w.is_float = fl;
    w.scanned += p.scanned;
    w.candidates += p.candidates;
    const bool lower = !w.has || (fl ? Ef < w.min_f : Ei < w.min_i);
    const bool equal = w.has && (fl ? Ef == w.min_f : Ei == w.min_i);
    if (lower) {
        w.has = true;
        w.min_i = Ei;
        w.min_f = Ef;
        w.n_ties = 0;
        w.ties.clear();
    }
    if (lower || equal) {
        w.n_ties += p.n_ties;
        for (uint64_t t : p.ties) {
            if (w.ties.size() >= cap)
                break;
            w.ties.push_back(code(t));
        }
    }
    if (K <= 0)
        return;
    if (fl) {
        std::vector<std::tuple<double, uint64_t, uint64_t>> add, out;
        for (auto &e : p.topf) {
            const auto c = code(e.second);
            add.emplace_back(e.first + cf, c.first, c.second);
        }
        std::merge(w.topf.begin(), w.topf.end(), add.begin(), add.end(), std::back_inserter(out));
        if ((int)out.size() > K)
            out.resize(K);
        w.topf.swap(out);
    } else {
        std::vector<std::tuple<int64_t, uint64_t, uint64_t>> add, out;
        for (auto &e : p.topi) {
            const auto c = code(e.second);
            add.emplace_back(e.first + ci, c.first, c.second);
        }
        std::merge(w.topi.begin(), w.topi.end(), add.begin(), add.end(), std::back_inserter(out));
        if ((int)out.size() > K)
            out.resize(K);
        w.topi.swap(out);
    }
}

}  // namespace

bool qubo::abort_requested() { return g_abort_all.load() != 0; }

// ================================================================================================
// C ABI
// ================================================================================================

struct qubo_batch {
    std::vector<HostInst> hs;
    std::vector<int> order;   // launch order (longest first) -> caller index
    Job job;
    Workspace ws;
    int count = 0;
    int topk = 0;
    size_t cap = 0;
    bool is_float = false;
    size_t off_state_init = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    bool launched = false;
    double t0 = 0.0;
    ~qubo_batch()
    {
        if (exec)
            cudaGraphExecDestroy(exec);
        if (graph)
            cudaGraphDestroy(graph);
        if (cap_stream)
            cudaStreamDestroy(cap_stream);
    }
};

struct qubo_problem {
    HostInst h;
    qubo_options opt{};
    Workspace ws;
    Job job;
    bool launched = false;
    int launch_status = QUBO_OK;
    int fix_bits = 0;
    uint64_t fix_value = 0;
    double t0 = 0.0;
    cudaStream_t stream = nullptr;
};

extern "C" {

const char *qubo_version(void) { return "qubo-gb300 0.1 (sm_103a)"; }

const char *qubo_strerror(int status)
{
    switch (status) {
    case QUBO_OK: return "ok";
    case QUBO_TRUNCATED: return "tie set truncated to states_cap (results valid, count exact)";
    case QUBO_ERR_ARG: return "bad argument";
    case QUBO_ERR_OVERFLOW: return "integer energies exceed every supported accumulator";
    case QUBO_ERR_CUDA: return "CUDA error";
    case QUBO_ERR_NOMEM: return "out of memory";
    case QUBO_ERR_TIMEOUT: return "time limit expired or aborted";
    case QUBO_ERR_INTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

void qubo_abort(void)
{
    g_abort_all.store(1);
    std::lock_guard<std::mutex> lk(g_ws_mu);
    for (Workspace *w : g_all_ws)
        if (w->h_abort)
            *(volatile int *)w->h_abort = 1;
}

void qubo_abort_clear(void) { g_abort_all.store(0); }

int qubo_device_sm_count(void)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QUBO_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return QUBO_ERR_CUDA;
    }
    return sms;
}

int qubo_solve_ex(const void *Q_host, int n, qubo_dtype dtype, const qubo_options *opt, void *out_min,
                  uint64_t *out_states, size_t states_cap, uint64_t *out_topk, void *out_topk_E, qubo_result *info,
                  void *stream)
{
    const double t0 = now_s();
    qubo_options o{};
    if (opt)
        o = *opt;
    int st = check_opts(&o, states_cap, out_states, out_topk);
    if (st)
        return st;
    if (!out_min)
        return QUBO_ERR_ARG;
    HostInst h;
    if ((st = prepare(Q_host, n, dtype, o.flags, h)))
        return st;
    if (o.fix_bits < 0 || o.fix_bits > n)
        return QUBO_ERR_ARG;
    if (o.topk > 0 && (uint64_t)o.topk > (1ull << std::min(62, n - o.fix_bits)))
        return QUBO_ERR_ARG;
    Workspace *ws = nullptr;
    if ((st = resolve_device(&ws)))
        return st;
    std::lock_guard<std::mutex> lk(ws->mu);
    int dev = -1;
    cudaGetDevice(&dev);
    if ((st = ws->init(dev)))
        return st;
    Part p;
    SolveStats stats;
    st = solve_one(*ws, h, o, states_cap, (cudaStream_t)stream, p, stats);
    if (st)
        return st;
    if (info)
        std::memset(info, 0, sizeof(*info));
    fill_outputs(h, p, o.topk, states_cap, out_min, out_states, out_topk, out_topk_E, info);
    fill_plan_info(h, stats, t0, info);
    fill_fp32_bound(h, o.margin > 0 ? o.margin : kDefaultMargin, info);
    return p.n_ties > states_cap ? QUBO_TRUNCATED : QUBO_OK;
}

int qubo_plan_query(const void *Q_host, int n, qubo_dtype dtype, const qubo_options *opt, qubo_result *info)
{
    const double t0 = now_s();
    qubo_options o{};
    if (opt)
        o = *opt;
    if (!info || o.topk < 0 || o.topk > QUBO_MAX_TOPK)
        return QUBO_ERR_ARG;
    HostInst h;
    int st = prepare(Q_host, n, dtype, o.flags, h);
    if (st)
        return st;
    if (o.fix_bits < 0 || o.fix_bits > n)
        return QUBO_ERR_ARG;
    const SolveCfg c = solve_cfg(h, o, 0, -1.0);
    if ((st = plan_run(h, o.fix_bits, o.fix_value, c.split_k, c.walk_bits, c.variant, c.flags, c.margin)))
        return st;
    std::memset(info, 0, sizeof(*info));
    info->acc = (int32_t)h.acc;
    fill_plan_info(h, SolveStats(), t0, info);
    fill_fp32_bound(h, c.margin, info);
    return QUBO_OK;
}

int qubo_solve_window(const void *Q_host, int n, qubo_dtype dtype, double window, const qubo_options *opt,
                      uint64_t *out_codes, void *out_E, size_t cap, uint64_t *out_count, qubo_result *info,
                      void *stream)
{
    const double t0 = now_s();
    qubo_options o{};
    if (opt)
        o = *opt;
    o.topk = 0;
    if (!(window >= 0.0) || !std::isfinite(window) || !out_count || (cap > 0 && (!out_codes || !out_E)))
        return QUBO_ERR_ARG;
    HostInst h;
    int st = prepare(Q_host, n, dtype, o.flags, h);
    if (st)
        return st;
    if (o.fix_bits < 0 || o.fix_bits > n)
        return QUBO_ERR_ARG;
    if (!h.is_float && window >= 1073741824.0)
        return QUBO_ERR_ARG;  // the int32 threshold arithmetic bounds the window
    if (!h.is_float && h.acc == ACC_I32 && h.beta + window >= 1073741824.0)
        h.acc = ACC_I64;
    Workspace *ws = nullptr;
    if ((st = resolve_device(&ws)))
        return st;
    std::lock_guard<std::mutex> lk(ws->mu);
    int dev = -1;
    cudaGetDevice(&dev);
    if ((st = ws->init(dev)))
        return st;
    Part p;
    SolveStats stats;
    if ((st = solve_one(*ws, h, o, 0, (cudaStream_t)stream, p, stats, window)))
        return st;
    if (info)
        std::memset(info, 0, sizeof(*info));
    fill_outputs(h, p, 0, 0, nullptr, nullptr, nullptr, nullptr, info);
    fill_plan_info(h, stats, t0, info);
    fill_fp32_bound(h, o.margin > 0 ? o.margin : kDefaultMargin, info);
    *out_count = p.win.size();
    const size_t nw = std::min(cap, p.win.size());
    for (size_t t = 0; t < nw; ++t) {
        out_codes[t] = p.win[t].second;
        if (h.is_float)
            ((double *)out_E)[t] = p.win[t].first;
        else
            ((int64_t *)out_E)[t] = (int64_t)p.win[t].first;
    }
    if (info)
        info->n_written = nw;
    return p.win.size() > cap ? QUBO_TRUNCATED : QUBO_OK;
}

int qubo_solve(const void *Q_host, int n, qubo_dtype dtype, int split_k, int topk, void *out_min,
               uint64_t *out_states, size_t states_cap, uint64_t *out_topk, void *out_topk_E, qubo_result *info,
               void *stream)
{
    qubo_options o{};
    o.split_k = split_k;
    o.topk = topk;
    return qubo_solve_ex(Q_host, n, dtype, &o, out_min, out_states, states_cap, out_topk, out_topk_E, info, stream);
}

int qubo_solve_batched(const void *Q_packed, const int *n, const size_t *offsets, int count, qubo_dtype dtype,
                       int topk, void *out_min, uint64_t *out_states, size_t states_cap_per_inst, uint64_t *out_topk,
                       void *out_topk_E, qubo_result *info, void *stream)
{
    const double t0 = now_s();
    if (!Q_packed || !n || !offsets || count < 1 || count > 65535 || !out_min || !dtype_ok(dtype))
        return QUBO_ERR_ARG;
    if (topk < 0 || topk > QUBO_MAX_TOPK || (topk > 0 && !out_topk) || (states_cap_per_inst > 0 && !out_states))
        return QUBO_ERR_ARG;
    std::vector<HostInst> hs;
    std::vector<int> order;
    int st = batch_prepare(Q_packed, n, offsets, count, dtype, topk, hs, order);
    if (st)
        return st;
    Workspace *ws = nullptr;
    if ((st = resolve_device(&ws)))
        return st;
    std::lock_guard<std::mutex> lk(ws->mu);
    int dev = -1;
    cudaGetDevice(&dev);
    if ((st = ws->init(dev)))
        return st;
    std::vector<Part> parts;
    SolveStats stats;
    if ((st = batch_parts(*ws, hs, order, topk, states_cap_per_inst, (cudaStream_t)stream, parts, stats)))
        return st;
    int worst = QUBO_OK;
    for (int i = 0; i < count; ++i) {
        Part &p = parts[i];
        HostInst &h = hs[i];
        void *om = h.is_float ? (void *)((double *)out_min + i) : (void *)((int64_t *)out_min + i);
        void *otke = nullptr;
        if (out_topk_E)
            otke = h.is_float ? (void *)((double *)out_topk_E + (size_t)i * topk)
                              : (void *)((int64_t *)out_topk_E + (size_t)i * topk);
        qubo_result *inf = info ? info + i : nullptr;
        if (inf)
            std::memset(inf, 0, sizeof(*inf));
        fill_outputs(h, p, topk, states_cap_per_inst, om,
                     out_states ? out_states + (size_t)i * states_cap_per_inst : nullptr,
                     out_topk ? out_topk + (size_t)i * topk : nullptr, otke, inf);
        fill_plan_info(h, stats, t0, inf);
        if (p.n_ties > states_cap_per_inst)
            worst = std::max(worst, (int)QUBO_TRUNCATED);
    }
    return worst;
}

int qubo_solve_wide(const void *Q_host, int n, qubo_dtype dtype, int n_inner, uint64_t outer_begin,
                    uint64_t outer_count, const qubo_options *opt, void *out_min, uint64_t *out_states,
                    size_t states_cap, uint64_t *out_n_ties, uint64_t *out_topk, void *out_topk_E, qubo_result *info,
                    void *stream)
{
    const double t0 = now_s();
    qubo_options o{};
    if (opt)
        o = *opt;
    if (!Q_host || !out_min || !dtype_ok(dtype) || n_inner < 1 || n_inner > 64 || n < n_inner ||
        n - n_inner > 64 || n > QUBO_WIDE_MAX_N || outer_count < 1 || o.fix_bits != 0)
        return QUBO_ERR_ARG;
    const int n_out = n - n_inner;
    if (n_out < 64 && (outer_begin >> n_out != 0 || outer_count > (1ull << n_out) - outer_begin))
        return QUBO_ERR_ARG;
    if (n_out == 64 && outer_begin + outer_count < outer_begin && outer_begin + outer_count != 0)
        return QUBO_ERR_ARG;
    if (o.topk < 0 || o.topk > QUBO_MAX_TOPK || (o.topk > 0 && !out_topk) || (states_cap > 0 && !out_states))
        return QUBO_ERR_ARG;
    if (n_inner < 62 && (uint64_t)o.topk > (1ull << n_inner))
        return QUBO_ERR_ARG;
    // fold the whole instance: U_ii = Q_ii, U_ij = Q_ij + Q_ji (i < j)
    const bool fl = dtype_float(dtype);
    std::vector<int64_t> Ui;
    std::vector<double> Uf;
    (fl ? Uf.assign((size_t)n * n, 0.0) : Ui.assign((size_t)n * n, 0));
    {
        int64_t beta = 0;
        for (int i = 0; i < n; ++i)
            for (int j = i; j < n; ++j) {
                const size_t a = (size_t)i * n + j, b = (size_t)j * n + i;
                if (fl) {
                    auto q = [&](size_t k) {
                        return dtype == QUBO_F32 ? (double)((const float *)Q_host)[k] : ((const double *)Q_host)[k];
                    };
                    const double v = i == j ? q(a) : q(a) + q(b);
                    if (!std::isfinite(v))
                        return QUBO_ERR_ARG;
                    Uf[a] = v;
                } else {
                    auto q = [&](size_t k) {
                        return dtype == QUBO_I16 ? (int64_t)((const int16_t *)Q_host)[k]
                                                 : (int64_t)((const int32_t *)Q_host)[k];
                    };
                    const int64_t v = i == j ? q(a) : q(a) + q(b);
                    Ui[a] = v;
                    beta += v < 0 ? -v : v;
                }
            }
        if (beta >= (1ll << 62))
            return QUBO_ERR_OVERFLOW;
    }
    Workspace *ws = nullptr;
    int st;
    if ((st = resolve_device(&ws)))
        return st;
    std::lock_guard<std::mutex> lk(ws->mu);
    int dev = -1;
    cudaGetDevice(&dev);
    if ((st = ws->init(dev)))
        return st;
    // Sub-problem of outer value v (variable n_inner + f = bit f of v): the inner variables keep
    // their couplings, each inner diagonal gains the couplings to the set outer variables, and the
    // set outer variables contribute the constant c(v) (Sec. 3.3.1; the scaling by fixed bits of
    // Sec. 4.3).
    auto reduce = [&](uint64_t v, HostInst &h, int64_t &ci, double &cf) {
        const int m = n_inner;
        std::vector<int64_t> ri;
        std::vector<double> rf;
        (fl ? rf.assign((size_t)m * m, 0.0) : ri.assign((size_t)m * m, 0));
        for (int i = 0; i < m; ++i)
            for (int j = i; j < m; ++j) {
                if (fl)
                    rf[(size_t)i * m + j] = Uf[(size_t)i * n + j];
                else
                    ri[(size_t)i * m + j] = Ui[(size_t)i * n + j];
            }
        ci = 0;
        cf = 0.0;
        for (int f = 0; f < n_out; ++f) {
            if (!((v >> f) & 1))
                continue;
            const int vf = n_inner + f;
            for (int i = 0; i < m; ++i) {
                if (fl)
                    rf[(size_t)i * m + i] += Uf[(size_t)i * n + vf];
                else
                    ri[(size_t)i * m + i] += Ui[(size_t)i * n + vf];
            }
            for (int g = f; g < n_out; ++g) {
                if (!((v >> g) & 1))
                    continue;
                if (fl)
                    cf += Uf[(size_t)vf * n + n_inner + g];
                else
                    ci += Ui[(size_t)vf * n + n_inner + g];
            }
        }
        return prepare_folded(fl ? nullptr : &ri, fl ? &rf : nullptr, m, o.flags, h);
    };
    const double deadline = o.time_limit_s > 0 ? t0 + o.time_limit_s : 0.0;
    const int K = o.topk;
    WideAcc w;
    SolveStats stats;
    HostInst last;
    const bool batched = n_inner <= kMaxBatchedN && outer_count > 1;
    const uint64_t chunk = batched ? 4096 : 1;
    for (uint64_t done = 0; done < outer_count; done += chunk) {
        if (deadline > 0 && now_s() > deadline)
            return QUBO_ERR_TIMEOUT;
        const int cnt = (int)std::min<uint64_t>(chunk, outer_count - done);
        std::vector<HostInst> hs(cnt);
        std::vector<int64_t> ci(cnt);
        std::vector<double> cf(cnt);
        for (int t = 0; t < cnt; ++t)
            if ((st = reduce(outer_begin + done + t, hs[t], ci[t], cf[t])))
                return st;
        std::vector<Part> parts;
        if (batched) {
            std::vector<int> order;
            if ((st = batch_plan(hs, K, order)))
                return st;
            if ((st = batch_parts(*ws, hs, order, K, states_cap, (cudaStream_t)stream, parts, stats)))
                return st;
        } else {
            qubo_options so = o;
            if (deadline > 0)
                so.time_limit_s = std::max(1e-3, deadline - now_s());
            parts.resize(1);
            if ((st = solve_one(*ws, hs[0], so, states_cap, (cudaStream_t)stream, parts[0], stats)))
                return st;
        }
        for (int t = 0; t < cnt; ++t)
            wide_add(w, parts[t], n_inner, outer_begin + done + t, ci[t], cf[t], states_cap, K);
        last = hs[cnt - 1];
    }
    if (fl)
        *(double *)out_min = w.min_f;
    else
        *(int64_t *)out_min = w.min_i;
    for (size_t t = 0; t < w.ties.size(); ++t) {
        out_states[2 * t] = w.ties[t].second;
        out_states[2 * t + 1] = w.ties[t].first;
    }
    if (out_n_ties)
        *out_n_ties = w.n_ties;
    const int nk = fl ? (int)w.topf.size() : (int)w.topi.size();
    for (int t = 0; t < nk; ++t) {
        out_topk[2 * t] = fl ? std::get<2>(w.topf[t]) : std::get<2>(w.topi[t]);
        out_topk[2 * t + 1] = fl ? std::get<1>(w.topf[t]) : std::get<1>(w.topi[t]);
        if (out_topk_E) {
            if (fl)
                ((double *)out_topk_E)[t] = std::get<0>(w.topf[t]);
            else
                ((int64_t *)out_topk_E)[t] = std::get<0>(w.topi[t]);
        }
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->min_i = fl ? 0 : w.min_i;
        info->min_f = fl ? w.min_f : (double)w.min_i;
        info->n_ties = w.n_ties;
        info->n_written = w.ties.size();
        info->truncated = w.n_ties > states_cap ? 1 : 0;
        info->acc = (int32_t)last.acc;
        info->n_topk = nk;
        info->states_scanned = w.scanned;
        info->candidates = w.candidates;
        fill_plan_info(last, stats, t0, info);
        info->n = n;
    }
    return w.n_ties > states_cap ? QUBO_TRUNCATED : QUBO_OK;
}

int qubo_problem_create(const void *Q_host, int n, qubo_dtype dtype, const qubo_options *opt, qubo_problem **out)
{
    if (!out)
        return QUBO_ERR_ARG;
    *out = nullptr;
    qubo_problem *p = new (std::nothrow) qubo_problem();
    if (!p)
        return QUBO_ERR_NOMEM;
    if (opt)
        p->opt = *opt;
    if (p->opt.topk < 0 || p->opt.topk > QUBO_MAX_TOPK) {
        delete p;
        return QUBO_ERR_ARG;
    }
    int st = prepare(Q_host, n, dtype, p->opt.flags, p->h);
    int dev = -1;
    if (!st && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        st = QUBO_ERR_CUDA;
    }
    if (!st)
        st = p->ws.init(dev);
    if (st) {
        delete p;
        return st;
    }
    register_ws(&p->ws);
    *out = p;
    return QUBO_OK;
}

int qubo_problem_run(qubo_problem *p, int fix_bits, uint64_t fix_value, void *stream)
{
    if (!p)
        return QUBO_ERR_ARG;
    p->t0 = now_s();
    p->fix_bits = fix_bits;
    p->fix_value = fix_value;
    p->stream = (cudaStream_t)stream;
    int st = plan_run(p->h, fix_bits, fix_value, p->opt.split_k, p->opt.walk_bits,
                      std::getenv("QUBO_SCAN_VARIANT") ? scan_variant(p->h.acc) : -1, p->opt.flags,
                      p->opt.margin > 0 ? p->opt.margin : kDefaultMargin);
    if (st)
        return st;
    p->h.thr0 = threshold_bound(p->h, std::max(1, p->opt.topk));
    p->job = Job();
    p->job.insts = {&p->h};
    p->job.acc = p->h.acc;
    p->job.K = p->opt.topk;
    p->job.cap = 1 << 16;
    p->job.margin = p->opt.margin > 0 ? p->opt.margin : kDefaultMargin;
    p->job.time_limit = p->opt.time_limit_s;
    p->job.variant = p->h.variant;
    p->job.stream = p->stream;
    st = job_launch(p->ws, p->job);
    p->launched = st == QUBO_OK;
    p->launch_status = st;
    return st;
}

int qubo_problem_fetch(qubo_problem *p, void *out_min, uint64_t *out_states, size_t states_cap, uint64_t *out_topk,
                       void *out_topk_E, qubo_result *info)
{
    if (!p || !out_min || (states_cap > 0 && !out_states) || (p->opt.topk > 0 && !out_topk))
        return QUBO_ERR_ARG;
    if (!p->launched)
        return p->launch_status ? p->launch_status : QUBO_ERR_ARG;
    p->launched = false;
    std::vector<Part> parts;
    SolveStats stats;
    double gs = 0.0;
    int st = job_finish(p->ws, p->job, parts, &gs);
    stats.add(p->job, gs);
    if (st)
        return st;
    Part part = parts[0];
    const size_t cap = std::min<size_t>(states_cap, p->job.cap);
    if (part.overflow || !float_margin_ok(p->h, part, p->job.margin) || states_cap > p->job.cap) {
        // repeat through the splitting path (exact, uses this problem's workspace)
        qubo_options o = p->opt;
        o.fix_bits = p->fix_bits;
        o.fix_value = p->fix_value;
        part = Part();
        if ((st = solve_one(p->ws, p->h, o, states_cap, p->stream, part, stats)))
            return st;
    }
    if (part.scanned != (1ull << (p->h.n - p->fix_bits)) || !part.has)
        return QUBO_ERR_INTERNAL;
    if (info)
        std::memset(info, 0, sizeof(*info));
    fill_outputs(p->h, part, p->opt.topk, states_cap, out_min, out_states, out_topk, out_topk_E, info);
    fill_plan_info(p->h, stats, p->t0, info);
    fill_fp32_bound(p->h, p->opt.margin > 0 ? p->opt.margin : kDefaultMargin, info);
    (void)cap;
    return part.n_ties > states_cap ? QUBO_TRUNCATED : QUBO_OK;
}

void qubo_problem_destroy(qubo_problem *p)
{
    if (!p)
        return;
    unregister_ws(&p->ws);
    delete p;
}

int qubo_batch_create(const void *Q_packed, const int *n, const size_t *offsets, int count, qubo_dtype dtype, int topk,
                      size_t states_cap_per_inst, qubo_batch **out)
{
    if (!out || !Q_packed || !n || !offsets || count < 1 || count > 65535 || !dtype_ok(dtype))
        return QUBO_ERR_ARG;
    if (topk < 0 || topk > QUBO_MAX_TOPK)
        return QUBO_ERR_ARG;
    *out = nullptr;
    qubo_batch *b = new (std::nothrow) qubo_batch();
    if (!b)
        return QUBO_ERR_NOMEM;
    std::unique_ptr<qubo_batch> guard(b);
    b->count = count;
    b->topk = topk;
    b->cap = states_cap_per_inst;
    b->is_float = dtype_float(dtype);
    int st = batch_prepare(Q_packed, n, offsets, count, dtype, topk, b->hs, b->order);
    if (st)
        return st;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QUBO_ERR_CUDA;
    }
    if ((st = b->ws.init(dev)))
        return st;
    Job &j = b->job;
    for (int i : b->order)
        j.insts.push_back(&b->hs[i]);
    j.acc = b->hs[0].acc;
    j.K = topk;
    j.cap = states_cap_per_inst;
    j.margin = kDefaultMargin;
    j.variant = b->hs[0].variant;
    // the initial per-instance state lives after the job's arena and is copied in at every run
    const size_t state_bytes = sizeof(InstState) * (size_t)count;
    if ((st = job_stage(b->ws, j, state_bytes + 256)))
        return st;
    // A graph sorts with a fixed network sized by the buffer; batches produce few candidates per
    // instance, so a smaller buffer keeps the replay short (an instance that overflows it is
    // solved again on its own at fetch time).
    j.rec_cap = std::min<unsigned long long>(j.rec_cap, kBatchGraphRecords);
    b->off_state_init = align_up(j.arena_bytes, 256);
    char *dev_arena = (char *)b->ws.d_arena;
    CK(cudaMemcpy(dev_arena, b->ws.h_up, j.up_bytes, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dev_arena + b->off_state_init, (char *)b->ws.h_up + j.off_state, state_bytes,
                  cudaMemcpyHostToDevice));
    j.h2d += j.up_bytes + state_bytes;
    // capture tables -> scan -> (rescore) -> sort -> extract -> download as one graph
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return QUBO_ERR_CUDA;
    }
    j.stream = b->cap_stream;
    unsigned long long P = 1;
    while (P < j.rec_cap)
        P <<= 1;
    CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    int st1 = job_enqueue_scan(b->ws, j, dev_arena + b->off_state_init);
    int st2 = st1 ? st1 : job_enqueue_finalize(b->ws, j, j.rec_cap, P);
    const cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (st1 || st2 || ce != cudaSuccess) {
        cudaGetLastError();
        return st1 ? st1 : (st2 ? st2 : QUBO_ERR_CUDA);
    }
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return QUBO_ERR_CUDA;
    }
    register_ws(&b->ws);
    *out = guard.release();
    return QUBO_OK;
}

int qubo_batch_run(qubo_batch *b, void *stream)
{
    if (!b)
        return QUBO_ERR_ARG;
    b->t0 = now_s();
    Job &j = b->job;
    j.stream = (cudaStream_t)stream;
    j.aborted = false;
    j.launches = 0;
    j.h2d = j.d2h = 0;
    *b->ws.h_abort = g_abort_all.load() ? 1 : 0;
    if (cudaGraphLaunch(b->exec, j.stream) != cudaSuccess) {
        cudaGetLastError();
        b->launched = false;
        return QUBO_ERR_CUDA;
    }
    j.t_start = now_s();
    b->launched = true;
    return QUBO_OK;
}

int qubo_batch_fetch(qubo_batch *b, void *out_min, uint64_t *out_states, uint64_t *out_topk, void *out_topk_E,
                     qubo_result *info)
{
    if (!b || !out_min || (b->cap > 0 && !out_states) || (b->topk > 0 && !out_topk))
        return QUBO_ERR_ARG;
    if (!b->launched)
        return QUBO_ERR_ARG;
    b->launched = false;
    Job &j = b->job;
    int st;
    if ((st = job_wait(b->ws, j, b->ws.ev[2])))
        return st;
    CK(cudaStreamSynchronize(j.stream));
    double gs = 0.0;
    {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b->ws.ev[0], b->ws.ev[2]) == cudaSuccess)
            gs = ms * 1e-3;
        if (cudaEventElapsedTime(&ms, b->ws.ev[3], b->ws.ev[1]) == cudaSuccess)
            j.scan_seconds = ms * 1e-3;
    }
    // the graph's launches: the same kernels a direct run makes, with every sort stage present
    {
        const bool is_float = acc_float(j.acc);
        unsigned long long P = 1;
        while (P < j.rec_cap)
            P <<= 1;
        int nl = 2 + (is_float ? 1 : 0) + 2 + (P >= 2 ? 2 : 0);
        for (unsigned long long k = 4096; k <= P; k <<= 1) {
            for (unsigned long long jj = k >> 1; jj >= 2048; jj >>= 1)
                ++nl;
            ++nl;
        }
        j.launches = nl;
    }
    j.d2h = sizeof(ResOut) * b->count + sizeof(InstState) * b->count + 8 * j.cap * b->count + 16 * (size_t)j.K * b->count;
    if (j.aborted)
        return QUBO_ERR_TIMEOUT;
    const Down d = down_view(b->ws, j);
    const bool is_float = acc_float(j.acc);
    SolveStats stats;
    stats.add(j, gs);
    int worst = QUBO_OK;
    SolveCfg c;
    c.K = b->topk;
    c.cap = b->cap;
    c.variant = j.variant;
    for (int r = 0; r < b->count; ++r) {
        const int i = b->order[r];
        HostInst &h = b->hs[i];
        const ResOut &res = d.res[r];
        const InstState &sts = d.sts[r];
        const double drift = ubits_to_double(sts.drift);
        const bool fast = res.has && sts.dropped == 0 && sts.scanned == (1ull << h.n) &&
                          (h.acc != ACC_F32 || 2.0 * drift + 8.0 * std::ldexp(1.0, -24) * (1.0 + h.beta) < c.margin);
        qubo_result *inf = info ? info + i : nullptr;
        if (fast) {
            // common case: copy straight from the staging buffer
            if (h.is_float)
                ((double *)out_min)[i] = res.min_f;
            else
                ((int64_t *)out_min)[i] = res.min_i;
            if (b->cap)
                std::memcpy(out_states + (size_t)i * b->cap, d.ties + (size_t)r * b->cap,
                            sizeof(uint64_t) * res.n_written);
            for (int t = 0; t < res.nk; ++t) {
                out_topk[(size_t)i * b->topk + t] = d.tk[(size_t)r * b->topk + t];
                if (out_topk_E) {
                    const int64_t e = d.tke[(size_t)r * b->topk + t];
                    if (h.is_float)
                        ((double *)out_topk_E)[(size_t)i * b->topk + t] = bits_to_double(e);
                    else
                        ((int64_t *)out_topk_E)[(size_t)i * b->topk + t] = e;
                }
            }
            if (inf) {
                std::memset(inf, 0, sizeof(*inf));
                inf->min_i = h.is_float ? 0 : res.min_i;
                inf->min_f = res.min_f;
                inf->n_ties = res.n_ties;
                inf->n_written = res.n_written;
                inf->truncated = res.n_ties > b->cap ? 1 : 0;
                inf->acc = (int32_t)h.acc;
                inf->n_topk = res.nk;
                inf->fp32_max_abs_err = is_float ? ubits_to_double(sts.err) : 0.0;
                inf->fp32_max_drift = is_float ? drift : 0.0;
                inf->n_near_ties = res.n_near;
                inf->states_scanned = sts.scanned;
                inf->candidates = sts.nrec;
                fill_plan_info(h, stats, b->t0, inf);
            }
            if (res.n_ties > b->cap)
                worst = std::max(worst, (int)QUBO_TRUNCATED);
            continue;
        }
        Part p = part_from(d, j, r);
        SolveStats st2 = stats;
        if (p.overflow || !float_margin_ok(h, p, c.margin)) {
            // rare: solve this instance alone on the shared workspace (the graph's is fixed)
            Workspace *sw = nullptr;
            if ((st = resolve_device(&sw)))
                return st;
            std::lock_guard<std::mutex> lk(sw->mu);
            int dev = -1;
            cudaGetDevice(&dev);
            if ((st = sw->init(dev)))
                return st;
            HostInst hc = h;
            if (!float_margin_ok(hc, p, c.margin))
                hc.acc = ACC_F64;
            p = Part();
            if ((st = solve_range(*sw, hc, 0, 0, c, j.stream, p, st2, 0.0)))
                return st;
        }
        if (p.scanned != (1ull << h.n) || !p.has)
            return QUBO_ERR_INTERNAL;
        void *om = h.is_float ? (void *)((double *)out_min + i) : (void *)((int64_t *)out_min + i);
        void *otke = nullptr;
        if (out_topk_E)
            otke = h.is_float ? (void *)((double *)out_topk_E + (size_t)i * b->topk)
                              : (void *)((int64_t *)out_topk_E + (size_t)i * b->topk);
        if (inf)
            std::memset(inf, 0, sizeof(*inf));
        fill_outputs(h, p, b->topk, b->cap, om, out_states ? out_states + (size_t)i * b->cap : nullptr,
                     out_topk ? out_topk + (size_t)i * b->topk : nullptr, otke, inf);
        fill_plan_info(h, st2, b->t0, inf);
        if (p.n_ties > b->cap)
            worst = std::max(worst, (int)QUBO_TRUNCATED);
    }
    return worst;
}

void qubo_batch_destroy(qubo_batch *b)
{
    if (!b)
        return;
    unregister_ws(&b->ws);
    delete b;
}

int qubo_autotune(const void *Q_host, int n, qubo_dtype dtype, int fix_bits, qubo_plan *best)
{
    if (!best || fix_bits < 0)
        return QUBO_ERR_ARG;
    HostInst h;
    int st = prepare(Q_host, n, dtype, 0, h);
    if (st)
        return st;
    if (fix_bits > n)
        return QUBO_ERR_ARG;
    Workspace *ws = nullptr;
    if ((st = resolve_device(&ws)))
        return st;
    std::lock_guard<std::mutex> lk(ws->mu);
    int dev = -1;
    cudaGetDevice(&dev);
    if ((st = ws->init(dev)))
        return st;
    const int nvar = acc_bytes(h.acc) == 4 ? kScanVariants : 1;
    std::memset(best, 0, sizeof(*best));
    double best_rate = -1.0;
    for (int v = 0; v < nvar; ++v) {
        HostInst base = h;
        base.variant = v;
        if (plan(base, fix_bits, 0, 0, 0))
            continue;
        if (base.small)
            break;  // nothing to tune: the sub-cube is evaluated directly
        const int L0 = base.L;
        for (int L = std::max(kRegRows + 1, L0 - 2); L <= std::min(kMaxWalkBits, L0 + 2); L += 2) {
            SolveCfg c;
            c.K = 0;
            c.cap = 0;
            c.variant = v;
            c.walk_bits = L;
            HostInst t = h;
            t.variant = v;
            if (plan(t, fix_bits, 0, 0, L) || reg_rows_of(t.acc, v) + 1 > L)
                continue;
            double rate = 0.0;
            for (int rep = 0; rep < 2; ++rep) {  // the first run warms the workspace
                Part p;
                SolveStats stats;
                HostInst r = h;
                if ((st = solve_range(*ws, r, fix_bits, (uint64_t)rep, c, nullptr, p, stats, 0.0)))
                    return st;
                if (stats.scan_seconds > 0)
                    rate = (double)p.scanned / stats.scan_seconds;
            }
            best->trials += 1;
            if (rate > best_rate) {
                best_rate = rate;
                best->variant = v;
                best->walk_bits = L;
                best->states_per_s = rate;
            }
        }
    }
    if (best_rate > 0)
        install_plan(h.acc, n, best->variant, best->walk_bits);
    return QUBO_OK;
}

int qubo_autotune_batched_ex(const void *Q_packed, const int *n, const size_t *offsets, int count, qubo_dtype dtype,
                             qubo_plan *best, qubo_plan *per_n)
{
    if (!best)
        return QUBO_ERR_ARG;
    std::memset(best, 0, sizeof(*best));
    if (per_n)
        std::memset(per_n, 0, sizeof(qubo_plan) * 65);
    // start from the untuned plans: forget the batch plans installed on this device
    {
        int d = -1;
        if (cudaGetDevice(&d) != cudaSuccess) {
            cudaGetLastError();
            return QUBO_ERR_CUDA;
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto it = g_tuned.begin(); it != g_tuned.end();)
            it = (std::get<0>(it->first) == d && std::get<2>(it->first) <= 0) ? g_tuned.erase(it) : std::next(it);
    }
    std::vector<HostInst> hs;
    std::vector<int> order;
    int st = batch_prepare(Q_packed, n, offsets, count, dtype, 0, hs, order);
    if (st)
        return st;
    const Acc acc = hs[0].acc;
    const bool lanes4 = acc_bytes(acc) == 4;
    const int nvar = lanes4 ? kScanVariants : 1;
    // the untuned walk, as in batch_plan: as long as the instance allows, at most wmax (integers
    // in FP32 lanes: 2^14 steps when exact, else 2^12)
    const int wmax = acc == ACC_F32 ? kFloatMaxWalkBits : (acc == ACC_I32F ? kI32FMaxWalkBits : kDefaultMaxWalkBits);
    Workspace *ws = nullptr;
    if ((st = resolve_device(&ws)))
        return st;
    std::lock_guard<std::mutex> lk(ws->mu);
    int dev = -1;
    cudaGetDevice(&dev);
    if ((st = ws->init(dev)))
        return st;
    uint64_t states = 0;
    for (auto &h : hs)
        states += 1ull << h.n;

    // Plan instance h under variant v with walk w (0: the untuned rule); false when the plan is
    // not admitted (too short a walk, or lanes that would not stay exact).
    auto plan_one = [&](HostInst &h, int v, int w) -> bool {
        h.acc = acc;
        h.variant = lanes4 ? v : 0;
        const int B = acc_suffix_bits(acc, h.variant);
        const int rmin = reg_rows_of(acc, h.variant) + 1;
        const int wd = h.n - B >= rmin ? std::min(wmax, h.n - B) : 0;
        if (w > 0 && (w < rmin || w > wd))
            return false;
        auto admitted = [&](int walk) {
            if (plan(h, 0, 0, 0, walk))
                return false;
            if (h.small)
                return true;
            if (acc == ACC_I16P) {
                if (!i16p_exact(h))
                    return false;
                i16p_fuse_el(h);
                // a fused-only packed kernel takes only plans whose E_L is fused
                return h.el_fused || !packed_fused_only(h.variant);
            }
            if (acc == ACC_I32F)
                return i32f_exact(h, &h.clampC);
            return true;
        };
        if (w > 0)
            return admitted(w);
        if (admitted(wd))
            return true;
        return acc == ACC_I32F && wd > kDefaultMaxWalkBits && admitted(kDefaultMaxWalkBits);
    };
    // Device time (tables, scan, reduction) of one launch over the whole batch, best of two.
    auto time_batch = [&](std::vector<HostInst> &hv, int v, double *t) -> int {
        *t = 0.0;
        for (int rep = 0; rep < 2; ++rep) {
            Job j;
            for (int i : order)
                j.insts.push_back(&hv[i]);
            j.acc = acc;
            j.variant = lanes4 ? v : 0;
            j.margin = kDefaultMargin;
            std::vector<Part> parts;
            double gs = 0.0;
            int e;
            if ((e = job_launch(*ws, j)) || (e = job_finish(*ws, j, parts, &gs)))
                return e;
            if (gs > 0 && (*t == 0.0 || gs < *t))
                *t = gs;
        }
        best->trials += 1;
        return QUBO_OK;
    };

    // Step 1: the kernel variant, every instance on the untuned walk.
    double best_t = 0.0;
    int vbest = -1;
    std::vector<HostInst> hbest;
    for (int v = 0; v < nvar; ++v) {
        std::vector<HostInst> hv = hs;
        bool ok = true;
        for (auto &h : hv)
            ok = ok && plan_one(h, v, 0);
        if (!ok)
            continue;
        double t = 0.0;
        if ((st = time_batch(hv, v, &t)))
            return st;
        if (t > 0 && (best_t == 0.0 || t < best_t)) {
            best_t = t;
            vbest = v;
            hbest = std::move(hv);
        }
    }
    if (vbest < 0)
        return QUBO_OK;  // no variant admitted: nothing installed

    // Step 2: per instance size, in order of the size's share of the work, shorter walks for
    // every instance of that size; a change is kept when the batch's device time falls by more
    // than 0.2%.
    std::map<int, uint64_t> work;
    for (auto &h : hbest)
        if (!h.small)
            work[h.n] += 1ull << h.n;
    std::vector<std::pair<uint64_t, int>> sizes;
    for (auto &kv : work)
        sizes.push_back({kv.second, kv.first});
    std::sort(sizes.rbegin(), sizes.rend());
    std::map<int, int> walk_of;  // n -> tuned walk
    std::map<int, int> trials_of;
    for (auto &sz : sizes) {
        const int nn = sz.second;
        int wcur = 0;
        for (auto &h : hbest)
            if (h.n == nn) {
                wcur = h.L;
                break;
            }
        const int w0 = wcur;
        for (int w = w0 - 1; w >= w0 - 4; --w) {
            std::vector<PlanFields> saved;
            std::vector<int> idx;
            bool ok = true;
            for (int i = 0; i < (int)hbest.size() && ok; ++i)
                if (hbest[i].n == nn) {
                    idx.push_back(i);
                    saved.push_back(plan_fields(hbest[i]));
                    ok = plan_one(hbest[i], vbest, w);
                }
            double t = 0.0;
            if (ok) {
                if ((st = time_batch(hbest, vbest, &t)))
                    return st;
                trials_of[nn] += 1;
            }
            if (ok && t > 0 && t < best_t * (1.0 - 2e-3)) {
                best_t = t;
                wcur = w;
            } else {
                for (size_t q = 0; q < idx.size(); ++q)
                    set_plan_fields(hbest[idx[q]], saved[q]);
                if (!ok)
                    break;  // shorter walks are not admitted either
            }
        }
        walk_of[nn] = wcur;
    }
    install_plan(acc, 0, vbest, 0);
    for (auto &kv : walk_of)
        install_plan(acc, -kv.first, vbest, kv.second);
    best->variant = vbest;
    best->walk_bits = 0;
    best->states_per_s = (double)states / best_t;
    if (per_n)
        for (auto &kv : walk_of) {
            per_n[kv.first].variant = vbest;
            per_n[kv.first].walk_bits = kv.second;
            per_n[kv.first].states_per_s = best->states_per_s;
            per_n[kv.first].trials = trials_of[kv.first];
        }
    return QUBO_OK;
}

int qubo_autotune_batched(const void *Q_packed, const int *n, const size_t *offsets, int count, qubo_dtype dtype,
                          qubo_plan *best)
{
    return qubo_autotune_batched_ex(Q_packed, n, offsets, count, dtype, best, nullptr);
}

void qubo_autotune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
}

namespace {
// Name and SM count of the current device: the key a saved plan is valid for.
bool device_key(int *dev, std::string *name, int *sms)
{
    cudaDeviceProp prop;
    if (cudaGetDevice(dev) != cudaSuccess || cudaGetDeviceProperties(&prop, *dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    *name = prop.name;
    std::replace(name->begin(), name->end(), '\t', ' ');
    *sms = prop.multiProcessorCount;
    return true;
}
}  // namespace

int qubo_autotune_save(const char *path)
{
    int dev = -1, sms = 0;
    std::string name;
    if (!path || !device_key(&dev, &name, &sms))
        return path ? QUBO_ERR_CUDA : QUBO_ERR_ARG;
    FILE *f = std::fopen(path, "w");
    if (!f)
        return QUBO_ERR_ARG;
    std::fprintf(f, "qubo-autotune 1\n");
    int count = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto &kv : g_tuned) {
            if (std::get<0>(kv.first) != dev)
                continue;
            std::fprintf(f, "%s\t%d\t%d\t%d\t%d\t%d\n", name.c_str(), sms, std::get<1>(kv.first),
                         std::get<2>(kv.first), kv.second.first, kv.second.second);
            ++count;
        }
    }
    const bool ok = std::fclose(f) == 0;
    return ok ? count : QUBO_ERR_ARG;
}

int qubo_autotune_load(const char *path)
{
    int dev = -1, sms = 0;
    std::string name;
    if (!path || !device_key(&dev, &name, &sms))
        return path ? QUBO_ERR_CUDA : QUBO_ERR_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f)
        return QUBO_ERR_ARG;
    char line[512];
    int count = 0, st = QUBO_OK;
    if (!std::fgets(line, sizeof line, f) || std::strncmp(line, "qubo-autotune 1", 15) != 0)
        st = QUBO_ERR_ARG;
    std::vector<std::pair<std::tuple<int, int, int>, std::pair<int, int>>> plans;
    while (st == QUBO_OK && std::fgets(line, sizeof line, f)) {
        char *tab = std::strchr(line, '\t');
        int fs = 0, acc = 0, n = 0, variant = 0, walk = 0;
        if (!tab || std::sscanf(tab + 1, "%d\t%d\t%d\t%d\t%d", &fs, &acc, &n, &variant, &walk) != 5 ||
            acc < ACC_I32 || acc > ACC_F32Z || n < -64 || n > 64 || variant < 0 || variant >= kScanVariants ||
            walk < 0 || walk > kMaxWalkBits) {
            st = QUBO_ERR_ARG;
            break;
        }
        *tab = 0;
        if (name == line && fs == sms)
            plans.push_back({{dev, acc, n}, {variant, walk}});
    }
    std::fclose(f);
    if (st)
        return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto &p : plans) {
        g_tuned[p.first] = p.second;
        ++count;
    }
    return count;
}

int qubo_merge_wide(const qubo_partial_wide *a, const qubo_partial_wide *b, size_t cap, int topk,
                    qubo_partial_wide *out)
{
    if (!a || !b || !out || topk < 0 || topk > QUBO_MAX_TOPK || a->is_float != b->is_float)
        return QUBO_ERR_ARG;
    if ((cap > 0 && !out->ties) || (topk > 0 && (!out->topk || !out->topk_E)))
        return QUBO_ERR_ARG;
    for (const qubo_partial_wide *x : {a, b})  // the inputs' arrays must hold what their counts say
        if (x->n_topk < 0 || x->n_topk > QUBO_MAX_TOPK || (x->n_topk > 0 && (!x->topk || !x->topk_E)) ||
            (x->n_written > 0 && !x->ties) || x->n_written > x->n_ties)
            return QUBO_ERR_ARG;
    const bool fl = a->is_float != 0;
    using Code = std::pair<uint64_t, uint64_t>;  // (bits 64..127, bits 0..63): ordered as the code
    auto code = [](const uint64_t *w, size_t t) { return Code(w[2 * t + 1], w[2 * t]); };
    auto energy = [&](const qubo_partial_wide *x, int t) {
        return fl ? ((const double *)x->topk_E)[t] : (double)((const int64_t *)x->topk_E)[t];
    };
    const bool ha = a->states_scanned > 0, hb = b->states_scanned > 0;
    const bool a_lower = fl ? a->min_f < b->min_f : a->min_i < b->min_i;
    const bool equal = fl ? a->min_f == b->min_f : a->min_i == b->min_i;
    std::vector<Code> ties;
    const qubo_partial_wide *lo = (!hb || (ha && a_lower)) ? a : b;
    if (ha && hb && equal) {
        std::vector<Code> ta, tb;
        for (size_t t = 0; t < a->n_written; ++t)
            ta.push_back(code(a->ties, t));
        for (size_t t = 0; t < b->n_written; ++t)
            tb.push_back(code(b->ties, t));
        std::merge(ta.begin(), ta.end(), tb.begin(), tb.end(), std::back_inserter(ties));
        out->n_ties = a->n_ties + b->n_ties;
    } else {
        for (size_t t = 0; t < lo->n_written; ++t)
            ties.push_back(code(lo->ties, t));
        out->n_ties = lo->n_ties;
    }
    out->is_float = a->is_float;
    out->min_i = lo->min_i;
    out->min_f = lo->min_f;
    out->states_scanned = a->states_scanned + b->states_scanned;
    out->n_written = std::min(cap, ties.size());
    for (size_t t = 0; t < out->n_written; ++t) {
        out->ties[2 * t] = ties[t].second;
        out->ties[2 * t + 1] = ties[t].first;
    }
    // K lowest by (E, code); integer energies stay exact as int64 in the comparison key
    std::vector<std::tuple<double, int64_t, Code>> top;
    for (const qubo_partial_wide *x : {a, b})
        for (int t = 0; t < x->n_topk; ++t)
            top.emplace_back(energy(x, t), fl ? 0 : ((const int64_t *)x->topk_E)[t], code(x->topk, t));
    std::sort(top.begin(), top.end(), [&](const auto &p, const auto &q) {
        if (fl ? std::get<0>(p) != std::get<0>(q) : std::get<1>(p) != std::get<1>(q))
            return fl ? std::get<0>(p) < std::get<0>(q) : std::get<1>(p) < std::get<1>(q);
        return std::get<2>(p) < std::get<2>(q);
    });
    const int nk = std::min<int>(topk, (int)top.size());
    out->n_topk = nk;
    for (int t = 0; t < nk; ++t) {
        out->topk[2 * t] = std::get<2>(top[t]).second;
        out->topk[2 * t + 1] = std::get<2>(top[t]).first;
        if (fl)
            ((double *)out->topk_E)[t] = std::get<0>(top[t]);
        else
            ((int64_t *)out->topk_E)[t] = std::get<1>(top[t]);
    }
    return QUBO_OK;
}

int qubo_merge(const qubo_partial *a, const qubo_partial *b, size_t cap, int topk, qubo_partial *out)
{
    if (!a || !b || !out || topk < 0 || topk > QUBO_MAX_TOPK || a->is_float != b->is_float)
        return QUBO_ERR_ARG;
    if ((cap > 0 && !out->ties) || (topk > 0 && (!out->topk || !out->topk_E)))
        return QUBO_ERR_ARG;
    for (const qubo_partial *x : {a, b})  // the inputs' arrays must hold what their counts say
        if (x->n_topk < 0 || x->n_topk > QUBO_MAX_TOPK || (x->n_topk > 0 && (!x->topk || !x->topk_E)) ||
            (x->n_written > 0 && !x->ties) || x->n_written > x->n_ties)
            return QUBO_ERR_ARG;
    auto to_part = [&](const qubo_partial *x) {
        Part p;
        p.has = x->states_scanned > 0;
        p.is_float = x->is_float != 0;
        p.min_i = x->min_i;
        p.min_f = x->min_f;
        p.n_ties = x->n_ties;
        p.scanned = x->states_scanned;
        if (x->n_written && x->ties)
            p.ties.assign(x->ties, x->ties + x->n_written);
        for (int t = 0; t < x->n_topk; ++t) {
            if (p.is_float)
                p.topf.emplace_back(((const double *)x->topk_E)[t], x->topk[t]);
            else
                p.topi.emplace_back(((const int64_t *)x->topk_E)[t], x->topk[t]);
        }
        return p;
    };
    const Part m = merge_parts(to_part(a), to_part(b), cap, topk);
    out->is_float = a->is_float;
    out->min_i = m.min_i;
    out->min_f = m.min_f;
    out->n_ties = m.n_ties;
    out->states_scanned = m.scanned;
    out->n_written = std::min(cap, m.ties.size());
    for (size_t t = 0; t < out->n_written; ++t)
        out->ties[t] = m.ties[t];
    const int nk = std::min(topk, m.is_float ? (int)m.topf.size() : (int)m.topi.size());
    out->n_topk = nk;
    for (int t = 0; t < nk; ++t) {
        if (m.is_float) {
            out->topk[t] = m.topf[t].second;
            ((double *)out->topk_E)[t] = m.topf[t].first;
        } else {
            out->topk[t] = m.topi[t].second;
            ((int64_t *)out->topk_E)[t] = m.topi[t].first;
        }
    }
    return QUBO_OK;
}

}  // extern "C"
