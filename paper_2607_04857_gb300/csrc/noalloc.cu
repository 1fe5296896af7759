// qubo_solve_noalloc: the exhaustive scan with every byte of device scratch taken from one
// file-scope __device__ array, for callers that must not allocate (see include/qubo.h).
//
// Nothing here calls cudaMalloc, cudaFree, cudaMallocHost or any other allocating routine,
// and the host side uses fixed-size stack arrays only.  The kernels are the library's own
// table-build, enumeration, sort and extraction kernels; they receive pointers into the array.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/qubo.h"
#include "internal.h"

using namespace qubo;

namespace {

constexpr size_t kScratchBytes = 2u << 20;  // QUBO_NOALLOC_SCRATCH_BYTES
constexpr unsigned long long kRecords = 1ull << 16;  // candidate records (a power of two)
constexpr int kB = suffix_bits(4, 0);        // int32 accumulator, scan variant 0: 10 suffix bits
constexpr int kMaxWalk = 12;

static_assert(QUBO_NOALLOC_SCRATCH_BYTES == kScratchBytes, "header and implementation must agree");

// Scratch of the no-allocation entry point.  Device code could name it directly; the host only
// passes its address, looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
unsigned char *g_scratch_ptr[64] = {};

int scratch_for_device(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= 64)
        return QUBO_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return QUBO_ERR_CUDA;
        }
        g_scratch_ptr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_ptr[dev];
    return QUBO_OK;
}

constexpr size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Byte offsets of the regions inside the scratch array.
struct Layout {
    size_t inst, state, items, ctr, abort, W, Es, M, EL, rec, res, starts, ties, end;
};

constexpr Layout layout(int n, int L, size_t cap)
{
    Layout l{};
    size_t o = 0;
    l.inst = o;
    o = up256(o + sizeof(Inst));
    l.state = o;
    o = up256(o + sizeof(InstState));
    l.items = o;
    o = up256(o + 2 * sizeof(uint64_t));
    l.ctr = o;
    o = up256(o + 2 * sizeof(unsigned long long));
    l.abort = o;
    o = up256(o + sizeof(int));
    l.W = o;
    o = up256(o + sizeof(int32_t) * n * n);
    l.Es = o;
    o = up256(o + sizeof(int32_t) * (1u << kB));
    l.M = o;
    o = up256(o + sizeof(int32_t) * (1u << kB) * L);
    l.EL = o;
    o = up256(o + sizeof(int32_t) * (1u << L));
    l.rec = o;
    o = up256(o + sizeof(Rec) * kRecords);
    l.res = o;
    o = up256(o + sizeof(ResOut));
    l.starts = o;
    o = up256(o + 2 * sizeof(unsigned long long));
    l.ties = o;
    o = up256(o + sizeof(uint64_t) * (cap ? cap : 1));
    l.end = o;
    return l;
}

// Walk length of the plan at n variables (the largest layout is the one at the largest n).
constexpr int walk_bits_of(int n)
{
    const int L = n - kB - 15;
    return L < kRegRows + 1 ? kRegRows + 1 : (L > kMaxWalk ? kMaxWalk : L);
}

// The header (Inst, InstState, item bases, counters, abort word, symmetric int32 matrix) is staged
// in one stack buffer of this size.
constexpr size_t kHeaderBytes = 8192;
constexpr Layout kLargest = layout(QUBO_NOALLOC_MAX_N, walk_bits_of(QUBO_NOALLOC_MAX_N), QUBO_NOALLOC_MAX_TIES);
static_assert(kLargest.end <= kScratchBytes, "the largest admitted problem must fit the scratch array");
static_assert(kLargest.W + sizeof(int32_t) * QUBO_NOALLOC_MAX_N * QUBO_NOALLOC_MAX_N <= kHeaderBytes,
              "the largest admitted header must fit its stack buffer");

// Energy of one state with the folded matrix (fixed summation order).
int64_t energy_host(const int64_t (*U)[QUBO_NOALLOC_MAX_N], int n, uint64_t x)
{
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
        if (!((x >> i) & 1))
            continue;
        acc += U[i][i];
        for (int j = i + 1; j < n; ++j)
            if ((x >> j) & 1)
                acc += U[i][j];
    }
    return acc;
}

// Lowest energy met by a few greedy one-flip descents: an upper bound on the minimum.
int64_t descent_bound(const int64_t (*U)[QUBO_NOALLOC_MAX_N], int n)
{
    int64_t best = 0;  // E(0) = 0
    uint64_t seed = 0x9e3779b97f4a7c15ull;
    for (int r = 0; r < 8; ++r) {
        seed ^= seed << 13;
        seed ^= seed >> 7;
        seed ^= seed << 17;
        uint64_t x = r == 0 ? 0 : (seed & (n >= 64 ? ~0ull : ((1ull << n) - 1)));
        int64_t E = energy_host(U, n, x);
        int64_t h[QUBO_NOALLOC_MAX_N];
        for (int j = 0; j < n; ++j) {
            int64_t a = 0;
            for (int i = 0; i < n; ++i)
                if (i != j && ((x >> i) & 1))
                    a += i < j ? U[i][j] : U[j][i];
            h[j] = a;
        }
        for (int it = 0; it < 4 * n; ++it) {
            int bv = -1;
            int64_t bd = 0;
            for (int v = 0; v < n; ++v) {
                const int64_t d = ((x >> v) & 1) ? -(U[v][v] + h[v]) : (U[v][v] + h[v]);
                if (d < bd) {
                    bd = d;
                    bv = v;
                }
            }
            if (bv < 0)
                break;
            const bool upf = !((x >> bv) & 1);
            x ^= 1ull << bv;
            E += bd;
            for (int j = 0; j < n; ++j)
                if (j != bv) {
                    const int64_t w = j < bv ? U[j][bv] : U[bv][j];
                    h[j] += upf ? w : -w;
                }
        }
        if (E < best)
            best = E;
    }
    return best;
}

}  // namespace

extern "C" int qubo_solve_noalloc(const void *Q_host, int n, qubo_dtype dtype, int64_t *out_min, uint64_t *out_states,
                                  size_t states_cap, uint64_t *out_n_ties, void *stream)
{
    if (!Q_host || !out_min || !out_n_ties || (states_cap > 0 && !out_states))
        return QUBO_ERR_ARG;
    if (n < 1 || n > QUBO_NOALLOC_MAX_N || states_cap > QUBO_NOALLOC_MAX_TIES)
        return QUBO_ERR_ARG;
    if (dtype != QUBO_I16 && dtype != QUBO_I32)
        return QUBO_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;

    // fold and bound, on the stack
    int64_t U[QUBO_NOALLOC_MAX_N][QUBO_NOALLOC_MAX_N];
    int64_t beta = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            auto q = [&](int a, int b) -> int64_t {
                const size_t o = (size_t)a * n + b;
                return dtype == QUBO_I16 ? (int64_t)((const int16_t *)Q_host)[o] : (int64_t)((const int32_t *)Q_host)[o];
            };
            U[i][j] = i == j ? q(i, i) : (i < j ? q(i, j) + q(j, i) : 0);
            if (i <= j)
                beta += U[i][j] < 0 ? -U[i][j] : U[i][j];
        }
    if (beta >= (1ll << 30))
        return QUBO_ERR_OVERFLOW;  // the fixed scratch holds int32 tables only

    // plan: small sub-cubes are evaluated directly, larger ones split as in qubo_solve
    const int small = n < kB + kRegRows + 1;
    int L = 0, k = 0;
    if (!small) {
        L = walk_bits_of(n);
        k = n - kB - L;
    }
    const Layout lo = layout(n, small ? 1 : L, states_cap);
    if (lo.end > kScratchBytes)
        return QUBO_ERR_INTERNAL;  // excluded at compile time for every admitted n and states_cap
    if (abort_requested())
        return QUBO_ERR_TIMEOUT;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QUBO_ERR_CUDA;
    }
    unsigned char *base = nullptr;
    int st = scratch_for_device(dev, &base);
    if (st)
        return st;

    // header staged in one stack buffer: Inst, InstState, item bases, symmetric int32 matrix
    alignas(16) unsigned char hdr[kHeaderBytes];
    const size_t hdr_bytes = lo.W + sizeof(int32_t) * n * n;
    if (hdr_bytes > sizeof(hdr))
        return QUBO_ERR_INTERNAL;  // excluded at compile time for every admitted n
    std::memset(hdr, 0, hdr_bytes);
    Inst d{};
    d.n = n;
    d.B = small ? 0 : kB;
    d.L = L;
    d.k = k;
    d.small = small;
    d.unit_begin = 0;
    d.units = small ? 0 : (1ull << k);
    d.sub_base = 0;
    d.sub_count = small ? (1ull << n) : 0;
    d.W = base + lo.W;
    d.W64 = nullptr;
    d.U64 = nullptr;
    d.Es = small ? nullptr : base + lo.Es;
    d.M = small ? nullptr : base + lo.M;
    d.EL = small ? nullptr : base + lo.EL;
    std::memcpy(hdr + lo.inst, &d, sizeof(d));
    InstState is{};
    is.thr = (unsigned long long)(uint32_t)(int32_t)descent_bound(U, n);
    is.gmin = (unsigned long long)(uint32_t)INT32_MAX;
    std::memcpy(hdr + lo.state, &is, sizeof(is));
    const uint64_t items[2] = {0, small ? 1ull : (1ull << k)};
    std::memcpy(hdr + lo.items, items, sizeof(items));
    int32_t *W = (int32_t *)(hdr + lo.W);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            W[a * n + b] = (int32_t)(a <= b ? U[a][b] : U[b][a]);

    // Every call reuses the array: the header is rewritten and the counters, the abort word
    // and the per-instance bounds are cleared before any kernel runs.
#define NA_CK(call)                                                                                \
    do {                                                                                           \
        if ((call) != cudaSuccess) {                                                               \
            cudaGetLastError();                                                                    \
            return QUBO_ERR_CUDA;                                                                  \
        }                                                                                          \
    } while (0)
    NA_CK(cudaMemcpyAsync(base, hdr, hdr_bytes, cudaMemcpyHostToDevice, s));
    NA_CK(cudaMemsetAsync(base + lo.ctr, 0, lo.W - lo.ctr, s));
    NA_CK(launch_tables(ACC_I32, (const Inst *)(base + lo.inst), 1, small ? 1 : (int)((1 << kB) * (L + 1) + (1 << L)),
                        s));
    ScanArgs a{};
    a.inst = (const Inst *)(base + lo.inst);
    a.state = (InstState *)(base + lo.state);
    a.item_base = (const uint64_t *)(base + lo.items);
    a.n_inst = 1;
    a.k1 = 1;
    a.total_items = items[1];
    a.queue = (unsigned long long *)(base + lo.ctr);
    a.rec = (Rec *)(base + lo.rec);
    a.rec_cap = kRecords;
    a.nrec = (unsigned long long *)(base + lo.ctr) + 1;
    a.abort_flag = (const volatile int *)(base + lo.abort);
    a.margin = 0.0;
    a.zero = 0;
    int sms = 0;
    NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int bps = scan_blocks_per_sm(ACC_I32, true, 0);
    if (bps < 1)
        bps = 1;
    uint64_t blocks = (uint64_t)sms * bps;
    const uint64_t need = (items[1] * 32 + kScanThreads - 1) / kScanThreads;
    if (blocks > need)
        blocks = need ? need : 1;
    NA_CK(launch_scan(ACC_I32, a, (int)blocks, 0, s));
    unsigned long long nrec = 0;
    NA_CK(cudaMemcpyAsync(&nrec, base + lo.ctr + sizeof(unsigned long long), sizeof(nrec), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (abort_requested())
        return QUBO_ERR_TIMEOUT;  // raised while the scan ran; its abort word is not watched
    if (nrec > kRecords)
        return QUBO_ERR_NOMEM;  // more candidates than the fixed scratch holds
    unsigned long long P = 1;
    while (P < nrec)
        P <<= 1;
    const unsigned long long *d_nrec = a.nrec;
    NA_CK(launch_sort(a.rec, d_nrec, kRecords, P, false, false, s, nullptr));
    NA_CK(launch_extract(a.inst, a.rec, d_nrec, kRecords, 1, false, false, 0, states_cap, (ResOut *)(base + lo.res),
                         (uint64_t *)(base + lo.ties), nullptr, nullptr, (unsigned long long *)(base + lo.starts), s));
    ResOut res{};
    InstState fin{};
    NA_CK(cudaMemcpyAsync(&res, base + lo.res, sizeof(res), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(&fin, base + lo.state, sizeof(fin), cudaMemcpyDeviceToHost, s));
    if (states_cap)
        NA_CK(cudaMemcpyAsync(out_states, base + lo.ties, sizeof(uint64_t) * states_cap, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
    if (!res.has || fin.scanned != (1ull << n) || fin.dropped || fin.dbg)
        return QUBO_ERR_INTERNAL;
    *out_min = res.min_i;
    *out_n_ties = res.n_ties;
    for (size_t t = res.n_written; t < states_cap; ++t)
        out_states[t] = 0;
    return res.n_ties > states_cap ? QUBO_TRUNCATED : QUBO_OK;
}
