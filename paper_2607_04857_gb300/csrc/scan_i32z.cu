// Factored scan of sparse integer instances (int32 energies).
//
// The host reorders the variables (Sec. 2.4 permutation invariance) so that the first Z walked
// rows have no coupling to any suffix variable.  Their table rows M_r are then zero: flipping
// them never changes a column energy.  Within a unit, the Gray walk over the L walked bits
// visits the 2^Z patterns of those rows in consecutive blocks while the other L - Z walked bits
// stay fixed (a property of the reflected Gray code), so for block k
//   E(k, i, j) = [c(x_f) + P_k] + e(i) + col_k(j),  e(i) = E_L(g(i)) + sum_{r < Z, g_r(i) = 1} w_r,
// with w_r the coupling of zero row r to the set fixed variables (Sec. 3.3.1).  The minimum
// over the block separates into min_i e(i) + min_j col_k(j): the columns are updated once per
// block (2^(L-Z) times per unit instead of 2^L), each block costs one table lookup and one
// compare, and a block whose separated minimum reaches the threshold is enumerated state by
// state, so minimum, tie set and K lowest stay exact.  Records carry codes in the caller's
// variable order.
#include "scan_impl.cuh"

namespace qubo {

namespace {

// Code of the scan order -> code of the caller's order (scan bit p is variable perm[p]).
__device__ __forceinline__ uint64_t unpermute(uint64_t c, const uint8_t *perm)
{
    uint64_t o = 0;
    while (c) {
        const int p = __ffsll((long long)c) - 1;
        c &= c - 1;
        o |= 1ull << perm[p];
    }
    return o;
}

constexpr int kZWarpScratch = (1 << kZMaxRows) + (1 << kZMaxBlocksLog2);

template <int S, bool K1>
__device__ void zscan_unit(const ScanArgs &a, const Inst &d, int inst, uint64_t unit, int32_t &Treg, int lane,
                           int32_t *wsm, int32_t *scratch, int32_t *stage)
{
    using T = int32_t;
    constexpr int V = 4, G = S / V, LOGG = ilog2c(G);
    constexpr int B = 2 + 5 + LOGG;
    constexpr int NB = 1 << B;
    const int n = d.n, L = d.L, k = d.k, BL = B + L, Z = d.Z;
    const int nz = 1 << Z, nblk = 1 << (L - Z);
    int32_t *wz = scratch;                        // 2^Z sums of zero-row couplings w_r
    int32_t *mel = scratch + (1 << kZMaxRows);    // per block: min_i e(i)
    InstState *st = a.state + inst;
    const int32_t *W = (const int32_t *)d.W;

    int32_t f0, cx;
    unit_fields<T>(W, n, k, BL, unit, lane, f0, cx);
    __syncwarp();
    if (lane >= B && lane < BL)
        wsm[lane - B] = f0;
    __syncwarp();
    int32_t lin_t, lin_e[V], lin_g[G];
    column_fields<int32_t, V, G>(f0, lane, lin_t, lin_e, lin_g);
    const int32_t *Es = (const int32_t *)d.Es;
    int32_t E[S];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        int32_t ev[V];
        vload<int32_t>(Es + (g * 32 + lane) * V, ev);
#pragma unroll
        for (int e = 0; e < V; ++e)
            E[g * V + e] = ev[e] + lin_e[e] + lin_t + lin_g[g];
    }

    // Per-unit tables: w sums of the zero rows, then the minimum of e(i) over every block.
    for (int m = lane; m < nz; m += 32) {
        int32_t s = 0;
        for (int r = 0; r < Z; ++r)
            if ((m >> r) & 1)
                s += wsm[r];
        wz[m] = s;
    }
    __syncwarp();
    // Lanes take consecutive walk steps (coalesced E_L reads).  The zero-row sum a step needs
    // depends only on its offset in the block and, through the top Gray bit, on the block's
    // parity, so each lane keeps the few it needs in registers.  A block's minimum is reduced
    // over the lanes that hold it (butterfly over aligned groups of min(2^Z, 32) lanes).
    const int32_t *EL = (const int32_t *)d.EL;
    if (Z >= 5) {
        constexpr int kPer = 1 << (kZMaxRows - 5);  // warp iterations per block, at most
        const int per = 1 << (Z - 5);
        int32_t wze[kPer], wzo[kPer];
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            const int ie = (t << 5) + lane, io = ie | (1 << Z);
            wze[t] = t < per ? wz[(ie ^ (ie >> 1)) & (nz - 1)] : 0;
            wzo[t] = t < per ? wz[(io ^ (io >> 1)) & (nz - 1)] : 0;
        }
#pragma unroll 4
        for (int kb = 0; kb < nblk; ++kb) {
            const int32_t *e = EL + (kb << Z) + lane;
            const bool odd = kb & 1;
            int32_t acc = INT32_MAX;
#pragma unroll
            for (int t = 0; t < kPer; ++t)
                if (t < per)
                    acc = min(acc, __ldg(e + (t << 5)) + (odd ? wzo[t] : wze[t]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                acc = min(acc, __shfl_xor_sync(kFull, acc, o));
            if (lane == (kb & 31))
                mel[kb] = acc;
        }
    } else {
        // blocks shorter than a warp: a lane's step offset, and so its zero-row sum, is fixed
        const int32_t wl = wz[(lane ^ (lane >> 1)) & (nz - 1)];
        const int total = 1 << L, iters = (total + 31) >> 5;
        for (int t = 0; t < iters; ++t) {
            const int i = (t << 5) + lane;
            int32_t acc = i < total ? __ldg(EL + i) + wl : INT32_MAX;
            for (int o = 1; o < nz; o <<= 1)
                acc = min(acc, __shfl_xor_sync(kFull, acc, o));
            if (i < total && (lane & (nz - 1)) == 0)
                mel[i >> Z] = acc;
        }
    }
    __syncwarp();

    {
        const int32_t tg = Tr<T>::thr_load(st);
        Treg = K1 ? min(Treg, tg) : tg;
    }
    const int32_t mu = (int32_t)a.margin;
    int32_t P = cx;  // c(x_f) + couplings of the set walked rows >= Z to the fixed variables
    const int32_t *Mt = (const int32_t *)d.M;
    const uint64_t cbase = unit << BL;

    for (int kb = 0; kb < nblk; ++kb) {
        if (kb > 0) {  // walked row Z + kk flips (Gray step over the blocks)
            const int kk = __ffs(kb) - 1;
            const int r = Z + kk;
            const bool neg = (kb >> (kk + 1)) & 1;
            const int32_t *row = Mt + (size_t)r * NB;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                int32_t mv[V];
                vload<int32_t>(row + (g * 32 + lane) * V, mv);
#pragma unroll
                for (int e = 0; e < V; ++e)
                    E[g * V + e] = neg ? E[g * V + e] - mv[e] : E[g * V + e] + mv[e];
            }
            P = neg ? P - wsm[r] : P + wsm[r];
        }
        const int32_t cm = tree_min<int32_t, 3, S>(E);
        if (cm + mel[kb] <= Treg + mu - P) {
            // rare: every state of the block, 2^Z zero-row patterns x the thread's columns
#pragma unroll
            for (int q = 0; q < S; ++q)
                stage[q * 32 + lane] = E[q];
            for (int i = kb << Z; i < (kb + 1) << Z; ++i) {
                const int g = i ^ (i >> 1);
                const int32_t el = EL[i] + wz[g & (nz - 1)];
                int32_t tp = Treg + mu - P - el;
                if (cm > tp)
                    continue;
                const uint64_t cb = cbase | ((uint64_t)g << B);
                for (int q = 0; q < S; ++q) {
                    const int32_t ev = stage[q * 32 + lane];
                    if (ev <= tp) {
                        const int32_t Et = ev + el + P;
                        const uint32_t j = (uint32_t)(((q / V) * 32 + lane) * V + (q % V));
                        record<T>(a, inst, Et, unpermute(cb | j, d.perm));
                        if (K1 && Et < Treg) {
                            Treg = Et;
                            tp = Treg + mu - P - el;
                            Tr<T>::thr_min(st, Et);
                        }
                    }
                }
            }
        }
    }
    if (lane == 0)
        atomicAdd(&st->scanned, 1ull << BL);
}

template <int S, bool K1>
__global__ void __launch_bounds__(kScanThreads, 3) zscan_kernel(const ScanArgs a)
{
    __shared__ int32_t stage_all[kScanThreads / 32][S * 32];
    __shared__ int32_t wsm_all[kScanThreads / 32][kMaxWalkBits];
    __shared__ int32_t scratch_all[kScanThreads / 32][kZWarpScratch];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cur = -1;
    int32_t Treg = 0;
    for (;;) {
        unsigned long long item = 0;
        int stop = 0;
        if (lane == 0) {
            stop = *a.abort_flag != 0;
            if (!stop)
                item = atomicAdd(a.queue, 1ull);
        }
        stop = __shfl_sync(kFull, stop, 0);
        item = __shfl_sync(kFull, item, 0);
        if (stop || item >= a.total_items)
            break;
        int inst = 0;
        if (a.n_inst > 1) {
            int lo = 0, hi = a.n_inst;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (a.item_base[mid] <= item)
                    lo = mid;
                else
                    hi = mid;
            }
            inst = lo;
        }
        if (inst != cur) {
            cur = inst;
            Treg = Tr<int32_t>::thr_load(a.state + inst);
        }
        const Inst d = a.inst[inst];
        const uint64_t off = item - a.item_base[inst];
        if (d.small)
            small_unit<int32_t>(a, d, inst, lane);
        else
            zscan_unit<S, K1>(a, d, inst, d.unit_begin + off, Treg, lane, wsm_all[warp], scratch_all[warp],
                              stage_all[warp]);
    }
}

template <bool K1>
auto zpick(int variant)
{
    return variant == 2 ? zscan_kernel<kZCols[2], K1>
           : variant == 1 ? zscan_kernel<kZCols[1], K1> : zscan_kernel<kZCols[0], K1>;
}

}  // namespace

cudaError_t launch_zscan(const ScanArgs &a, int blocks, int variant, cudaStream_t s)
{
    auto k = a.k1 ? zpick<true>(variant) : zpick<false>(variant);
    k<<<blocks, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

int zscan_blocks_per_sm(bool k1, int variant)
{
    int nb = 0;
    auto k = k1 ? zpick<true>(variant) : zpick<false>(variant);
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kScanThreads, 0);
    return e == cudaSuccess ? nb : -1;
}

}  // namespace qubo
