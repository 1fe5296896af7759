// Finalize kernels: FP64 rescoring of float candidates, sorting of the candidate records by
// (instance, energy, code), and extraction of the minimum, tie set and K lowest states per
// instance (the reduce step of the map-reduce in Sec. 3.3).  Also the accumulator dispatch.
#include <cstdint>

#include "internal.h"

namespace qubo {

cudaError_t launch_tables(Acc acc, const Inst *d_inst, int n_inst, int max_entries, cudaStream_t s)
{
    switch (acc) {
    case ACC_I32: return launch_tables_t<int32_t>(d_inst, n_inst, max_entries, s);
    case ACC_I64: return launch_tables_t<int64_t>(d_inst, n_inst, max_entries, s);
    case ACC_F32: return launch_tables_t<float>(d_inst, n_inst, max_entries, s);
    case ACC_F64: return launch_tables_t<double>(d_inst, n_inst, max_entries, s);
    case ACC_I32F: return launch_tables_t<i32f>(d_inst, n_inst, max_entries, s);
    case ACC_I16P: return launch_tables_t<i16p>(d_inst, n_inst, max_entries, s);
    case ACC_I32Z: return launch_tables_t<int32_t>(d_inst, n_inst, max_entries, s);
    case ACC_F32Z: return launch_tables_t<float>(d_inst, n_inst, max_entries, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_scan(Acc acc, const ScanArgs &a, int blocks, int variant, cudaStream_t s)
{
    switch (acc) {
    case ACC_I32: return launch_scan_t<int32_t>(a, blocks, variant, s);
    case ACC_I64: return launch_scan_t<int64_t>(a, blocks, variant, s);
    case ACC_F32: return launch_scan_t<float>(a, blocks, variant, s);
    case ACC_F64: return launch_scan_t<double>(a, blocks, variant, s);
    case ACC_I32F: return launch_scan_t<i32f>(a, blocks, variant, s);
    case ACC_I16P: return launch_scan_t<i16p>(a, blocks, variant, s);
    case ACC_I32Z: return launch_zscan(a, blocks, variant, false, s);
    case ACC_F32Z: return launch_zscan(a, blocks, variant, true, s);
    }
    return cudaErrorInvalidValue;
}

int scan_blocks_per_sm(Acc acc, bool k1, int variant)
{
    switch (acc) {
    case ACC_I32: return scan_blocks_per_sm_t<int32_t>(k1, variant);
    case ACC_I64: return scan_blocks_per_sm_t<int64_t>(k1, variant);
    case ACC_F32: return scan_blocks_per_sm_t<float>(k1, variant);
    case ACC_F64: return scan_blocks_per_sm_t<double>(k1, variant);
    case ACC_I32F: return scan_blocks_per_sm_t<i32f>(k1, variant);
    case ACC_I16P: return scan_blocks_per_sm_t<i16p>(k1, variant);
    case ACC_I32Z: return zscan_blocks_per_sm(k1, variant, false);
    case ACC_F32Z: return zscan_blocks_per_sm(k1, variant, true);
    }
    return -1;
}

namespace {

constexpr unsigned kFullMask = 0xffffffffu;

__device__ __forceinline__ unsigned long long rec_count(const unsigned long long *d_nrec, unsigned long long cap)
{
    const unsigned long long c = *d_nrec;
    return c < cap ? c : cap;
}

__device__ __forceinline__ unsigned long long pow2_ceil(unsigned long long v)
{
    unsigned long long p = 1;
    while (p < v)
        p <<= 1;
    return p;
}

__device__ __forceinline__ uint64_t rec_inst(uint64_t key, bool batched) { return batched ? key >> kInstShift : 0; }
__device__ __forceinline__ uint64_t rec_code(uint64_t key, bool batched)
{
    return batched ? key & ((1ull << kInstShift) - 1) : key;
}

template <bool FL>
__device__ __forceinline__ bool rec_less(const Rec &a, const Rec &b, bool batched)
{
    const uint64_t ia = rec_inst(a.key, batched), ib = rec_inst(b.key, batched);
    if (ia != ib)
        return ia < ib;
    if (FL) {
        const double ea = __longlong_as_double(a.e), eb = __longlong_as_double(b.e);
        if (ea != eb)
            return ea < eb;
    } else if (a.e != b.e) {
        return a.e < b.e;
    }
    return a.key < b.key;
}

// FP64 energy in the fixed order i ascending, then j ascending (adds only, so no contraction).
__device__ double energy_fp64(const double *U, int n, uint64_t x)
{
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!((x >> i) & 1ull))
            continue;
        acc += U[i * n + i];
        for (int j = i + 1; j < n; ++j)
            if ((x >> j) & 1ull)
                acc += U[i * n + j];
    }
    return acc;
}

__global__ void rescore_kernel(const Inst *insts, InstState *state, Rec *rec, const unsigned long long *d_nrec,
                               unsigned long long cap, bool batched)
{
    const unsigned long long cnt = rec_count(d_nrec, cap);
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        Rec r = rec[i];
        const uint64_t inst = rec_inst(r.key, batched);
        const Inst &d = insts[inst];
        const double e64 = energy_fp64(d.U64, d.n, rec_code(r.key, batched));
        const double err = fabs(__longlong_as_double(r.e) - e64);
        atomicMax(&state[inst].err, (unsigned long long)__double_as_longlong(err));
        r.e = __double_as_longlong(e64);
        rec[i] = r;
    }
}

// Pad [count, pow2_ceil(count)) with records that sort after every real one.
__global__ void pad_kernel(Rec *rec, const unsigned long long *d_nrec, unsigned long long cap, bool is_float)
{
    const unsigned long long cnt = rec_count(d_nrec, cap);
    const unsigned long long P = pow2_ceil(cnt);
    for (unsigned long long i = cnt + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < P;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        Rec r;
        r.key = ~0ull;
        r.e = is_float ? __double_as_longlong(__longlong_as_double(0x7ff0000000000000ll)) : 0x7fffffffffffffffll;
        rec[i] = r;
    }
}

constexpr int kChunk = 2048;  // elements sorted in shared memory by one block (1024 threads)

// Bitonic network on the padded power-of-two prefix [0, P).  Stages with k > P are skipped,
// which sorts the prefix on its own.
template <bool FL>
__global__ void __launch_bounds__(1024) sort_local_kernel(Rec *rec, const unsigned long long *d_nrec,
                                                          unsigned long long cap, bool batched,
                                                          unsigned long long k_merge)
{
    __shared__ Rec sh[kChunk];
    const unsigned long long P = pow2_ceil(rec_count(d_nrec, cap));
    const unsigned long long base = (unsigned long long)blockIdx.x * kChunk;
    if (P < 2 || base >= P || (k_merge && k_merge > P))
        return;
    const unsigned long long len = P - base < kChunk ? P - base : kChunk;
    for (unsigned long long t = threadIdx.x; t < len; t += blockDim.x)
        sh[t] = rec[base + t];
    __syncthreads();
    const unsigned long long kmax = len < kChunk ? len : kChunk;
    // k_merge == 0: full local sort (k = 2 .. kmax); otherwise only the j < kChunk steps of stage k_merge.
    const unsigned long long k_lo = k_merge ? k_merge : 2, k_hi = k_merge ? k_merge : kmax;
    for (unsigned long long k = k_lo; k <= k_hi; k <<= 1) {
        unsigned long long j0 = k >> 1;
        if (j0 >= kChunk)
            j0 = kChunk >> 1;
        for (unsigned long long j = j0; j > 0; j >>= 1) {
            for (unsigned long long t = threadIdx.x; t < len; t += blockDim.x) {
                const unsigned long long l = t ^ j;
                if (l > t && l < len) {
                    const unsigned long long gi = base + t;
                    const bool up = (gi & k) == 0;
                    const Rec a = sh[t], b = sh[l];
                    const bool swap = up ? rec_less<FL>(b, a, batched) : rec_less<FL>(a, b, batched);
                    if (swap) {
                        sh[t] = b;
                        sh[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (unsigned long long t = threadIdx.x; t < len; t += blockDim.x)
        rec[base + t] = sh[t];
}

template <bool FL>
__global__ void sort_global_kernel(Rec *rec, const unsigned long long *d_nrec, unsigned long long cap, bool batched,
                                   unsigned long long k, unsigned long long j)
{
    const unsigned long long P = pow2_ceil(rec_count(d_nrec, cap));
    if (k > P)
        return;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < P;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long l = i ^ j;
        if (l <= i)
            continue;
        const bool up = (i & k) == 0;
        const Rec a = rec[i], b = rec[l];
        const bool swap = up ? rec_less<FL>(b, a, batched) : rec_less<FL>(a, b, batched);
        if (swap) {
            rec[i] = b;
            rec[l] = a;
        }
    }
}

// Per instance: first and one-past-last record index in sorted order.
__global__ void bounds_kernel(const Rec *rec, const unsigned long long *d_nrec, unsigned long long cap, bool batched,
                              unsigned long long *starts, int n_inst)
{
    const unsigned long long cnt = rec_count(d_nrec, cap);
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint64_t a = rec_inst(rec[i].key, batched);
        if (a >= (uint64_t)n_inst)
            continue;
        if (i == 0 || rec_inst(rec[i - 1].key, batched) != a)
            starts[2 * a] = i;
        if (i + 1 == cnt || rec_inst(rec[i + 1].key, batched) != a)
            starts[2 * a + 1] = i + 1;
    }
}

// One warp per instance: minimum, exact tie run, first states_cap tie codes, K lowest.
template <bool FL>
__global__ void extract_kernel(const Rec *rec, bool batched, int n_inst, int topk, unsigned long long states_cap,
                               const unsigned long long *starts, ResOut *res, uint64_t *ties, uint64_t *topk_codes,
                               int64_t *topk_e)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_inst)
        return;
    const unsigned long long s = starts[2 * warp], e = starts[2 * warp + 1];
    ResOut out{};
    if (e <= s) {
        if (lane == 0)
            res[warp] = out;
        return;
    }
    const int64_t emin = rec[s].e;
    const double fmin = __longlong_as_double(emin);
    const double near_lim = fmin + 1e-9 * fmax(1.0, fabs(fmin));
    // the ties and the near-ties are prefixes of [s, e)
    unsigned long long nt = 0, nn = 0;
    bool done_t = false, done_n = !FL;
    for (unsigned long long b = s; b < e && !(done_t && done_n); b += 32) {
        const unsigned long long i = b + lane;
        const bool valid = i < e;
        const int64_t ei = valid ? rec[i].e : 0;
        if (!done_t) {
            const unsigned m = __ballot_sync(kFullMask, valid && ei == emin);
            const int c = __ffs(~m) - 1;  // first lane that is not a tie (-1: all 32 are)
            if (c < 0) {
                nt += 32;
            } else {
                nt += c;
                done_t = true;
            }
        }
        if (!done_n) {
            const unsigned m = __ballot_sync(kFullMask, valid && __longlong_as_double(ei) <= near_lim);
            const int c = __ffs(~m) - 1;
            if (c < 0) {
                nn += 32;
            } else {
                nn += c;
                done_n = true;
            }
        }
    }
    const unsigned long long nw = nt < states_cap ? nt : states_cap;
    for (unsigned long long t = lane; t < nw; t += 32)
        ties[(unsigned long long)warp * states_cap + t] = rec_code(rec[s + t].key, batched);
    const unsigned long long avail = e - s;
    const int nk = (int)(avail < (unsigned long long)topk ? avail : (unsigned long long)topk);
    for (int t = lane; t < nk; t += 32) {
        topk_codes[(size_t)warp * topk + t] = rec_code(rec[s + t].key, batched);
        topk_e[(size_t)warp * topk + t] = rec[s + t].e;
    }
    if (lane == 0) {
        out.min_i = emin;
        out.min_f = FL ? fmin : (double)emin;
        out.n_ties = nt;
        out.n_written = nw;
        out.n_near = FL ? nn : nt;
        out.nk = nk;
        out.has = 1;
        res[warp] = out;
    }
}

}  // namespace

cudaError_t launch_rescore(const Inst *d_inst, InstState *d_state, Rec *rec, const unsigned long long *d_nrec,
                           unsigned long long cap, bool batched, unsigned long long max_count, cudaStream_t s)
{
    unsigned long long blocks = (max_count + 255) / 256;
    if (blocks < 1)
        blocks = 1;
    if (blocks > 8192)
        blocks = 8192;
    rescore_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_inst, d_state, rec, d_nrec, cap, batched);
    return cudaGetLastError();
}

cudaError_t launch_sort(Rec *rec, const unsigned long long *d_nrec, unsigned long long cap, unsigned long long max_pow2,
                        bool batched, bool is_float, cudaStream_t s, int *launches)
{
    if (max_pow2 < 2)
        return cudaSuccess;
    int nl = 0;
    {
        unsigned long long blocks = (max_pow2 + 255) / 256;
        if (blocks > 8192)
            blocks = 8192;
        pad_kernel<<<(unsigned)blocks, 256, 0, s>>>(rec, d_nrec, cap, is_float);
        ++nl;
    }
    const unsigned long long chunks = (max_pow2 + kChunk - 1) / kChunk;
    auto local = [&](unsigned long long k_merge) {
        ++nl;
        if (is_float)
            sort_local_kernel<true><<<(unsigned)chunks, 1024, 0, s>>>(rec, d_nrec, cap, batched, k_merge);
        else
            sort_local_kernel<false><<<(unsigned)chunks, 1024, 0, s>>>(rec, d_nrec, cap, batched, k_merge);
    };
    local(0);
    for (unsigned long long k = 2 * kChunk; k <= max_pow2; k <<= 1) {
        for (unsigned long long j = k >> 1; j >= (unsigned long long)kChunk; j >>= 1) {
            unsigned long long blocks = (max_pow2 + 255) / 256;
            if (blocks > 2048)
                blocks = 2048;  // grid-stride; keeps stages that the device count skips cheap
            ++nl;
            if (is_float)
                sort_global_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(rec, d_nrec, cap, batched, k, j);
            else
                sort_global_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(rec, d_nrec, cap, batched, k, j);
        }
        local(k);
    }
    if (launches)
        *launches += nl;
    return cudaGetLastError();
}

cudaError_t launch_extract(const Inst *d_inst, const Rec *rec, const unsigned long long *d_nrec, unsigned long long cap,
                           int n_inst, bool batched, bool is_float, int topk, unsigned long long states_cap,
                           ResOut *res, uint64_t *ties, uint64_t *topk_codes, int64_t *topk_e,
                           unsigned long long *d_starts, cudaStream_t s)
{
    (void)d_inst;
    cudaError_t e = cudaMemsetAsync(d_starts, 0, sizeof(unsigned long long) * 2 * (size_t)n_inst, s);
    if (e != cudaSuccess)
        return e;
    bounds_kernel<<<1024, 256, 0, s>>>(rec, d_nrec, cap, batched, d_starts, n_inst);
    const int threads = 256;
    const int blocks = (n_inst * 32 + threads - 1) / threads;
    if (is_float)
        extract_kernel<true><<<blocks, threads, 0, s>>>(rec, batched, n_inst, topk, states_cap, d_starts, res, ties,
                                                       topk_codes, topk_e);
    else
        extract_kernel<false><<<blocks, threads, 0, s>>>(rec, batched, n_inst, topk, states_cap, d_starts, res, ties,
                                                        topk_codes, topk_e);
    return cudaGetLastError();
}

}  // namespace qubo
