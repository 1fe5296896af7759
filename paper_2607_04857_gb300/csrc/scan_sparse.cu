// Factored scan of sparse instances (int32 energies, or FP32 energies with FP64 rescoring).
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

template <class X>
__device__ __forceinline__ X zbig();
template <>
__device__ __forceinline__ int32_t zbig<int32_t>() { return INT32_MAX; }
template <>
__device__ __forceinline__ float zbig<float>() { return __int_as_float(0x7f800000); }
__device__ __forceinline__ int32_t emax(int32_t a, int32_t b) { return max(a, b); }
__device__ __forceinline__ float emax(float a, float b) { return fmaxf(a, b); }

// Per-warp scratch: the (parity, t) table of zero-row sums (at most 2^(16-4) entries would be
// needed for 16 zero rows; the host keeps Z <= kZMaxRows) and the block minima.
constexpr int kZTableEntries = 1 << (kZMaxRows - 4);
constexpr int kZWarpScratch = 1 << kZMaxBlocksLog2;

// Sum of the couplings w_r of the zero rows r set in the pattern m (slow path only).
template <class X>
__device__ __forceinline__ X zero_row_sum(int m, const X *wsm, int Z)
{
    X s = 0;
    for (int r = 0; r < Z; ++r)
        if ((m >> r) & 1)
            s += wsm[r];
    return s;
}

template <class T, int S, bool K1>
__device__ void zscan_unit(const ScanArgs &a, const Inst &d, int inst, uint64_t unit, typename Tr<T>::TP &Treg,
                           int lane, typename Tr<T>::TC *wsm, typename Tr<T>::TC *scratch, typename Tr<T>::TC *stage)
{
    using X = typename Tr<T>::TC;
    constexpr int V = 4, G = S / V, LOGG = ilog2c(G);
    constexpr int B = 2 + 5 + LOGG;
    constexpr int NB = 1 << B;
    const int n = d.n, L = d.L, k = d.k, BL = B + L, Z = d.Z;
    const int nz = 1 << Z, nblk = 1 << (L - Z);
    InstState *st = a.state + inst;
    const X *W = unit_matrix<T>(d);

    X f0, cx;
    unit_fields<T>(W, n, k, BL, unit, lane, f0, cx);
    __syncwarp();
    if (lane >= B && lane < BL)
        wsm[lane - B] = f0;
    __syncwarp();
    X lin_t, lin_e[V], lin_g[G];
    column_fields<X, V, G>(f0, lane, lin_t, lin_e, lin_g);
    const X *Es = (const X *)d.Es;
    X E[S];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        X ev[V];
        vload<X>(Es + (g * 32 + lane) * V, ev);
#pragma unroll
        for (int e = 0; e < V; ++e)
            E[g * V + e] = ev[e] + lin_e[e] + lin_t + lin_g[g];
    }

    // Per-unit minimum of e(i) over every block (lanes take consecutive walk steps: coalesced
    // E_L reads).  The zero-row sum of step i is linear in the bits of g(i) = i ^ (i >> 1):
    // bits 0-3 of g come from the lane, bit 4 from the lane and the warp iteration t, bits
    // 5..Z-1 from t and, at the top, the block's parity.  So a lane adds its own part after its
    // running minimum, and the t part comes from a small per-warp table (a broadcast read).
    // A block's minimum is then reduced over the lanes that hold it.
    const X *EL = (const X *)d.EL;
    X *wt = stage;                         // Z >= 5: 2^(Z-4) entries (parity, t); the slow
                                                 // path's staging reuses it after the table
    X *mel = scratch;                      // per block: min_i e(i)
    if (Z >= 7) {
        // Lanes take 4 consecutive steps each (one 16-byte E_L read), a warp iteration t covers
        // 128 steps: step bits 0-1 are the element k, bits 2-6 the lane, bits 7..Z-1 t, bit Z
        // the block's parity.  Gray bits g_0..g_5 follow from (k, lane), g_6 from the lane's top
        // bit and bit 7 of the step, g_7..g_{Z-1} from (parity, t) through a per-warp table.
        const int zt = Z - 7;
        X *gs = mel;
        if (lane == 0)
            gs[0] = 0;
        __syncwarp();
        for (int b = 0; b < zt; ++b) {
            const X wb = wsm[7 + b];
            for (int m = lane; m < (1 << b); m += 32)
                gs[m + (1 << b)] = gs[m] + wb;
            __syncwarp();
        }
        for (int e = lane; e < (2 << zt); e += 32)
            wt[e] = gs[(e ^ (e >> 1)) & ((1 << zt) - 1)];
        X a = 0;  // g_2..g_5 from the lane bits
        for (int r = 0; r < 4; ++r)
            if (((lane >> r) ^ (lane >> (r + 1))) & 1)
                a += wsm[2 + r];
        const bool l0 = lane & 1, l4 = (lane >> 4) & 1;
        X ae[4], ao[4];  // per element k, for bit 7 of the step = 0 (ae) and 1 (ao)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool g0 = (k ^ (k >> 1)) & 1, g1 = ((k >> 1) & 1) ^ l0;
            const X base = a + (g0 ? wsm[0] : 0) + (g1 ? wsm[1] : 0);
            ae[k] = base + (l4 ? wsm[6] : 0);
            ao[k] = base + (l4 ? 0 : wsm[6]);
        }
        __syncwarp();
        const int nt = 1 << zt;
        for (int kb = 0; kb < nblk; ++kb) {
            const X *e = EL + (kb << Z) + 4 * lane;
            const X *w = wt + ((kb & 1) << zt);
            X acc;
            if (nt == 1) {  // Z == 7: bit 7 of the step index is the block's parity
                X v[4], ak[4];
                vload<X>(e, v);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    ak[k] = (kb & 1) ? ao[k] : ae[k];
                acc = emin(emin3(v[0] + ak[0], v[1] + ak[1], v[2] + ak[2]), v[3] + ak[3]);
            } else {
                X me = zbig<X>(), mo = zbig<X>();
#pragma unroll 2
                for (int t = 0; t < nt; t += 2) {
                    X v[4], u[4];
                    vload<X>(e + (t << 7), v);
                    vload<X>(e + ((t + 1) << 7), u);
                    const X mv = emin(emin3(v[0] + ae[0], v[1] + ae[1], v[2] + ae[2]), v[3] + ae[3]);
                    const X mu2 = emin(emin3(u[0] + ao[0], u[1] + ao[1], u[2] + ao[2]), u[3] + ao[3]);
                    me = emin(me, mv + w[t]);
                    mo = emin(mo, mu2 + w[t + 1]);
                }
                acc = emin(me, mo);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                acc = emin(acc, __shfl_xor_sync(kFull, acc, o));
            if (lane == (kb & 31))
                mel[kb] = acc;
        }
    } else if (Z >= 5) {
        const int zt = Z - 5;
        // subset sums of w_5..w_{Z-1} by doubling (mel is free until the block minima), then
        // wt[e] for e = (parity << zt) | t, the bits 5..Z of the step index: the Gray bits
        // g_5..g_{Z-1} of the step are the Gray code of e cut to zt bits.
        X *gs = mel;
        if (lane == 0)
            gs[0] = 0;
        __syncwarp();
        for (int b = 0; b < zt; ++b) {
            const X wb = wsm[5 + b];
            for (int m = lane; m < (1 << b); m += 32)
                gs[m + (1 << b)] = gs[m] + wb;
            __syncwarp();
        }
        for (int e = lane; e < (2 << zt); e += 32)
            wt[e] = gs[(e ^ (e >> 1)) & ((1 << zt) - 1)];
        X a = 0;
        for (int r = 0; r < 4; ++r)
            if (((lane >> r) ^ (lane >> (r + 1))) & 1)
                a += wsm[r];
        const bool l4 = (lane >> 4) & 1;
        const X a0 = a + (l4 ? wsm[4] : 0);  // even t: bit 5 of the step index is 0
        const X a1 = a + (l4 ? 0 : wsm[4]);  // odd t
        __syncwarp();
        const int nt = 1 << zt;
#pragma unroll 2
        for (int kb = 0; kb < nblk; ++kb) {
            const X *e = EL + (kb << Z) + lane;
            const X *w = wt + ((kb & 1) << zt);
            X acc;
            if (nt == 1) {  // Z == 5: bit 5 of the step index is the block's parity
                acc = __ldg(e) + ((kb & 1) ? a1 : a0);
            } else {
                X ae = zbig<X>(), ao = zbig<X>();
#pragma unroll 4
                for (int t = 0; t < nt; t += 2) {
                    ae = emin(ae, __ldg(e + (t << 5)) + w[t]);
                    ao = emin(ao, __ldg(e + ((t + 1) << 5)) + w[t + 1]);
                }
                acc = emin(ae + a0, ao + a1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                acc = emin(acc, __shfl_xor_sync(kFull, acc, o));
            if (lane == (kb & 31))
                mel[kb] = acc;
        }
    } else {
        // blocks shorter than a warp: the whole zero-row sum of a step follows from its lane
        X wl = 0;
        for (int r = 0; r < Z; ++r)
            if (((lane >> r) ^ (lane >> (r + 1))) & 1)
                wl += wsm[r];
        const int total = 1 << L, iters = (total + 31) >> 5;
        for (int t = 0; t < iters; ++t) {
            const int i = (t << 5) + lane;
            X acc = i < total ? __ldg(EL + i) + wl : zbig<X>();
            for (int o = 1; o < nz; o <<= 1)
                acc = emin(acc, __shfl_xor_sync(kFull, acc, o));
            if (i < total && (lane & (nz - 1)) == 0)
                mel[i >> Z] = acc;
        }
    }
    __syncwarp();

    {
        const X tg = Tr<T>::thr_load(st);
        Treg = K1 ? emin(Treg, tg) : tg;
    }
    const X mu = (X)a.margin;
    X P = cx;  // c(x_f) + couplings of the set walked rows >= Z to the fixed variables
    const X *Mt = (const X *)d.M;
    const uint64_t cbase = unit << BL;

    // Enumeration of block kb whose columns are staged in `stage` (prefix Pb, lane minimum cmb):
    // the warp enumerates the block together.  Lanes take consecutive walk steps (coalesced E_L
    // reads); a step whose e(i) plus the smallest column of any lane reaches the largest
    // threshold of any lane is broadcast, and every lane checks its own columns at that step.
    auto enumerate_block = [&](int kb, X Pb, X cmb) {
        X cmin = cmb, tmax = Treg;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cmin = emin(cmin, __shfl_xor_sync(kFull, cmin, o));
            tmax = emax(tmax, __shfl_xor_sync(kFull, tmax, o));
        }
        const X umax = tmax + mu - Pb;
        const int i0 = kb << Z;
        int ii = i0 + lane;
        int gi = ii ^ (ii >> 1);
        X zs = zero_row_sum(gi & (nz - 1), wsm, Z);
        for (int off = 0; off < nz; off += 32) {
            if (off > 0) {  // ii advances by 32: refresh the zero-row bits that changed
                ii += 32;
                const int gn = ii ^ (ii >> 1);
                int diff = (gi ^ gn) & (nz - 1);
                while (diff) {
                    const int r = __ffs(diff) - 1;
                    diff &= diff - 1;
                    zs = ((gn >> r) & 1) ? zs + wsm[r] : zs - wsm[r];
                }
                gi = gn;
            }
            const bool valid = off + lane < nz;
            const X el = valid ? __ldg(EL + ii) + zs : 0;
            unsigned m = __ballot_sync(kFull, valid && cmin + el <= umax);
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const X els = __shfl_sync(kFull, el, src);
                const int is = i0 + off + src;
                X tp = Treg + mu - Pb - els;
                if (cmb > tp)
                    continue;
                const uint64_t cb = cbase | ((uint64_t)(is ^ (is >> 1)) << B);
                for (int q = 0; q < S; ++q) {
                    const X ev = stage[q * 32 + lane];
                    if (ev <= tp) {
                        const X Et = ev + els + Pb;
                        const uint32_t j = (uint32_t)(((q / V) * 32 + lane) * V + (q % V));
                        record<T>(a, inst, Et, unpermute(cb | j, d.perm));
                        if (K1 && Et < Treg) {
                            Treg = Et;
                            tp = Treg + mu - Pb - els;
                            Tr<T>::thr_min(st, Et);
                        }
                    }
                }
            }
        }
        __syncwarp();
    };
    // Flip of walked row Z + kk before block kb (Gray step over the blocks), row from L1.
    auto flip_from_memory = [&](int kb) {
        const int kk = __ffs(kb) - 1;
        const int r = Z + kk;
        const X sg = ((kb >> (kk + 1)) & 1) ? (X)-1 : (X)1;  // one multiply-add per column
        const X *row = Mt + (size_t)r * NB;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            X mv[V];
            vload<X>(row + (g * 32 + lane) * V, mv);
#pragma unroll
            for (int e = 0; e < V; ++e)
                E[g * V + e] = E[g * V + e] + sg * mv[e];
        }
        P = P + sg * wsm[r];
    };

    // With 16 columns per thread, walked rows Z and Z+1 stay in registers and bodies of 8 blocks
    // are unrolled, so their flips have compile-time rows and signs; row Z+2 flips at a body's
    // middle and the rows above at body starts, from L1.  Per block one tree min and the block
    // minimum cm + mel + P go into a running minimum, compared once per body.
    constexpr int RB = S == 16 ? 2 : 0;
    constexpr int NBODY = 2 << RB;
    bool walked = false;
    if constexpr (RB > 0) {
        if (nblk >= NBODY) {
            walked = true;
            X Mr[RB][S], wr[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const X *row = Mt + (size_t)(Z + r) * NB;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    X mv[V];
                    vload<X>(row + (g * 32 + lane) * V, mv);
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        Mr[r][g * V + e] = mv[e];
                }
                wr[r] = wsm[Z + r];
            }
            const X *rowMid = Mt + (size_t)(Z + RB) * NB;
            for (int kb0 = 0; kb0 < nblk; kb0 += NBODY) {
                if (kb0 > 0)
                    flip_from_memory(kb0);
                const X sgMid = ((kb0 >> (RB + 1)) & 1) ? (X)-1 : (X)1;
                X acc;
                static_for<NBODY>([&](auto pc) {
                    constexpr int p = decltype(pc)::value;
                    if constexpr (p > 0) {
                        constexpr int kk = ctzc(p);
                        if constexpr (kk < RB) {
                            constexpr bool neg = (p >> (kk + 1)) & 1;
#pragma unroll
                            for (int q = 0; q < S; ++q)
                                E[q] = neg ? E[q] - Mr[kk][q] : E[q] + Mr[kk][q];
                            P = neg ? P - wr[kk] : P + wr[kk];
                        } else {
#pragma unroll
                            for (int g = 0; g < G; ++g) {
                                X mv[V];
                                vload<X>(rowMid + (g * 32 + lane) * V, mv);
#pragma unroll
                                for (int e = 0; e < V; ++e)
                                    E[g * V + e] = E[g * V + e] + sgMid * mv[e];
                            }
                            P = P + sgMid * wsm[Z + RB];
                        }
                    }
                    const X m = tree_min<X, 3, S>(E) + (mel[kb0 + p] + P);
                    if constexpr (p == 0)
                        acc = m;
                    else
                        acc = emin(acc, m);
                });
                if (__any_sync(kFull, acc <= Treg + mu)) {
                    // rare: rebuild each block of the body from the body-end registers (the rows
                    // whose Gray bits differ) and enumerate the blocks that reach the threshold
                    const int kend = kb0 + NBODY - 1;
                    const int gend = kend ^ (kend >> 1);
#pragma unroll 1
                    for (int p = 0; p < NBODY; ++p) {
                        const int kb = kb0 + p;
                        const int gp = kb ^ (kb >> 1);
                        X sr[RB + 1];
#pragma unroll
                        for (int r = 0; r <= RB; ++r)
                            sr[r] = (X)(((gp >> r) & 1) - ((gend >> r) & 1));
                        X Pb = P;
#pragma unroll
                        for (int r = 0; r < RB; ++r)
                            Pb = Pb + sr[r] * wr[r];
                        Pb = Pb + sr[RB] * wsm[Z + RB];
                        X cmb = zbig<X>();
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            X mv[V];
                            vload<X>(rowMid + (g * 32 + lane) * V, mv);
#pragma unroll
                            for (int e = 0; e < V; ++e) {
                                const int q = g * V + e;
                                X ev = E[q];
#pragma unroll
                                for (int r = 0; r < RB; ++r)
                                    ev = ev + sr[r] * Mr[r][q];
                                ev = ev + sr[RB] * mv[e];
                                stage[q * 32 + lane] = ev;
                                cmb = emin(cmb, ev);
                            }
                        }
                        if (__any_sync(kFull, cmb + (mel[kb] + Pb) <= Treg + mu))
                            enumerate_block(kb, Pb, cmb);
                        __syncwarp();
                    }
                }
            }
        }
    }
    if (!walked) {
        for (int kb = 0; kb < nblk; ++kb) {
            if (kb > 0)
                flip_from_memory(kb);
            const X cm = tree_min<X, 3, S>(E);
            if (__any_sync(kFull, cm + mel[kb] <= Treg + mu - P)) {
#pragma unroll
                for (int q = 0; q < S; ++q)
                    stage[q * 32 + lane] = E[q];
                enumerate_block(kb, P, cm);
            }
        }
    }

    if constexpr (Tr<T>::kFloat) {
        // FP32 drift: the columns and P after 2^(L-Z) - 1 block updates against fresh values at
        // the walk's end, where only walked row L - 1 (the top one) is set
        X f0r, cxr, lt, le[V], lg[G];
        unit_fields<T>(W, n, k, BL, unit, lane, f0r, cxr);
        column_fields<X, V, G>(f0r, lane, lt, le, lg);
        const X *rowT = Mt + (size_t)(L - 1) * NB;
        double dmax = 0.0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            X ev[V], mv[V];
            vload<X>(Es + (g * 32 + lane) * V, ev);
            vload<X>(rowT + (g * 32 + lane) * V, mv);
#pragma unroll
            for (int e = 0; e < V; ++e)
                dmax = fmax(dmax, fabs((double)E[g * V + e] - (double)(ev[e] + le[e] + lt + lg[g] + mv[e])));
        }
        const X wtop = __shfl_sync(kFull, f0r, B + L - 1);
        dmax = fmax(dmax, fabs((double)P - (double)(cxr + wtop)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            dmax = fmax(dmax, __shfl_xor_sync(kFull, dmax, o));
        if (lane == 0)
            atomicMax(&st->drift, (unsigned long long)__double_as_longlong(dmax));
    }
}

template <class T, int S, bool K1>
__global__ void __launch_bounds__(kScanThreads, S == 16 ? 4 : 3) zscan_kernel(const ScanArgs a)
{
    using X = typename Tr<T>::TC;
    __shared__ X stage_all[kScanThreads / 32][S * 32 > kZTableEntries ? S * 32 : kZTableEntries];
    __shared__ X wsm_all[kScanThreads / 32][kMaxWalkBits];
    __shared__ X scratch_all[kScanThreads / 32][kZWarpScratch];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    typename Tr<T>::TP Treg = 0;
    persistent_units<T, 8>(a, lane, Treg, [&](const Inst &d, int inst, uint64_t unit) {
        zscan_unit<T, S, K1>(a, d, inst, unit, Treg, lane, wsm_all[warp], scratch_all[warp], stage_all[warp]);
    });
}

// ---- one block per unit: every walked row factored out (Z = L >= 7) --------------------------
// The columns are used once (their minimum, and in a hit unit each column again), so they are
// not kept in registers: the kernel runs at more warps per SM to hide the E_L reads' latency.
// A warp takes the units it claims two at a time: both units' minima of e are formed in one pass
// over E_L, which halves the L1 traffic of that pass (it ran near the L1 load bandwidth).

// Minima over the 2^Z walk steps of U units of e_u(i) = E_L(g(i)) + the sum of unit u's
// zero-row couplings of the set bits of g(i) (Z >= 7; the same decomposition as zscan_unit's
// block minima, parity 0), one read of E_L for all U units.  out[u] is the warp's minimum.
template <class X, int U>
__device__ __forceinline__ void walk_min_units(const X *EL, int Z, int lane, X *const (&wsm)[U], X *const (&wt)[U],
                                               X *gs, X (&out)[U])
{
    const int zt = Z - 7;
#pragma unroll
    for (int u = 0; u < U; ++u) {  // the high-bit table of unit u, built by doubling in gs
        if (lane == 0)
            gs[0] = 0;
        __syncwarp();
        for (int b = 0; b < zt; ++b) {
            const X wb = wsm[u][7 + b];
            for (int m = lane; m < (1 << b); m += 32)
                gs[m + (1 << b)] = gs[m] + wb;
            __syncwarp();
        }
        for (int e = lane; e < (1 << zt); e += 32)  // parity 0: only the lower half of the table
            wt[u][e] = gs[(e ^ (e >> 1)) & ((1 << zt) - 1)];
        __syncwarp();  // gs is rebuilt for the next unit
    }
    const bool l0 = lane & 1, l4 = (lane >> 4) & 1;
    X ae[U][4], ao[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        X a = 0;
        for (int r = 0; r < 4; ++r)
            if (((lane >> r) ^ (lane >> (r + 1))) & 1)
                a += wsm[u][2 + r];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool g0 = (k ^ (k >> 1)) & 1, g1 = ((k >> 1) & 1) ^ l0;
            const X base = a + (g0 ? wsm[u][0] : 0) + (g1 ? wsm[u][1] : 0);
            ae[u][k] = base + (l4 ? wsm[u][6] : 0);
            ao[u][k] = base + (l4 ? 0 : wsm[u][6]);
        }
    }
    const X *e = EL + 4 * lane;
    if (zt == 0) {
        X v[4];
        vload<X>(e, v);
#pragma unroll
        for (int u = 0; u < U; ++u)
            out[u] = emin(emin3(v[0] + ae[u][0], v[1] + ae[u][1], v[2] + ae[u][2]), v[3] + ae[u][3]);
    } else {
        X me[U], mo[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            me[u] = mo[u] = zbig<X>();
        const int nt = 1 << zt;
#pragma unroll 4
        for (int t = 0; t < nt; t += 2) {
            X v[4], w[4];
            vload<X>(e + (t << 7), v);
            vload<X>(e + ((t + 1) << 7), w);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const X mv = emin(emin3(v[0] + ae[u][0], v[1] + ae[u][1], v[2] + ae[u][2]), v[3] + ae[u][3]);
                const X mw = emin(emin3(w[0] + ao[u][0], w[1] + ao[u][1], w[2] + ao[u][2]), w[3] + ao[u][3]);
                me[u] = emin(me[u], mv + wt[u][t]);
                mo[u] = emin(mo[u], mw + wt[u][t + 1]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            out[u] = emin(me[u], mo[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            out[u] = emin(out[u], __shfl_xor_sync(kFull, out[u], o));
}

// Set-up of one unit x_f: the fields of its set fixed bits (f0, one variable per lane), c(x_f),
// the zero-row couplings w_r into wsm, and the lane's minimum over its columns
// E_s(j) + lin(j), j = (g * 32 + lane) * 4 + e.
template <class T, int S>
__device__ __forceinline__ void unit_one_setup(const Inst &d, uint64_t unit, int lane, typename Tr<T>::TC *wsm,
                                               typename Tr<T>::TC &f0, typename Tr<T>::TC &cx, typename Tr<T>::TC &cm)
{
    using X = typename Tr<T>::TC;
    constexpr int V = 4, G = S / V, LOGG = ilog2c(G);
    constexpr int B = 2 + 5 + LOGG;
    const int BL = B + d.L;
    unit_fields<T>(unit_matrix<T>(d), d.n, d.k, BL, unit, lane, f0, cx);
    __syncwarp();
    if (lane >= B && lane < BL)
        wsm[lane - B] = f0;
    __syncwarp();
    X lin_t, lin_e[V], lin_g[G];
    column_fields<X, V, G>(f0, lane, lin_t, lin_e, lin_g);
    const X *Es = (const X *)d.Es;
    cm = zbig<X>();
#pragma unroll
    for (int g = 0; g < G; ++g) {
        X ev[V];
        vload<X>(Es + (g * 32 + lane) * V, ev);
        const X l = lin_t + lin_g[g];
        cm = emin(cm, emin3(ev[0] + lin_e[0] + l, ev[1] + lin_e[1] + l,
                            emin(ev[2] + lin_e[2] + l, ev[3] + lin_e[3] + l)));
    }
}

// Threshold test of a unit whose walk minimum of e is mel; a unit that reaches the threshold is
// enumerated by the whole warp, as in zscan_unit: lanes take consecutive steps, each lane
// recomputes its columns at a broadcast step.
template <class T, int S, bool K1>
__device__ void unit_one_finish(const ScanArgs &a, const Inst &d, int inst, uint64_t unit, typename Tr<T>::TP &Treg,
                                int lane, const typename Tr<T>::TC *wsm, typename Tr<T>::TC *lin_sm,
                                typename Tr<T>::TC f0, typename Tr<T>::TC cx, typename Tr<T>::TC cm,
                                typename Tr<T>::TC mel)
{
    using X = typename Tr<T>::TC;
    constexpr int V = 4, G = S / V, LOGG = ilog2c(G);
    constexpr int B = 2 + 5 + LOGG;
    const int Z = d.L, BL = B + Z, nz = 1 << Z;
    InstState *st = a.state + inst;
    {
        const X tg = Tr<T>::thr_load(st);
        Treg = K1 ? emin(Treg, tg) : tg;
    }
    const X mu = (X)a.margin;
    const X P = cx;
    if (!__any_sync(kFull, cm + mel <= Treg + mu - P))
        return;
    X lin_t, lin_e[V], lin_g[G];
    column_fields<X, V, G>(f0, lane, lin_t, lin_e, lin_g);
    const X *Es = (const X *)d.Es;
    const X *EL = (const X *)d.EL;
    const uint64_t cbase = unit << BL;
    X cmin = cm, tmax = Treg;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cmin = emin(cmin, __shfl_xor_sync(kFull, cmin, o));
        tmax = emax(tmax, __shfl_xor_sync(kFull, tmax, o));
    }
    const X umax = tmax + mu - P;
#pragma unroll
    for (int g = 0; g < G; ++g)  // the enumeration indexes the column groups at run time
        lin_sm[g * 32 + lane] = lin_g[g];
    int ii = lane;
    int gi = ii ^ (ii >> 1);
    X zs = zero_row_sum(gi & (nz - 1), wsm, Z);
    for (int off = 0; off < nz; off += 32) {
        if (off > 0) {
            ii += 32;
            const int gn = ii ^ (ii >> 1);
            int diff = (gi ^ gn) & (nz - 1);
            while (diff) {
                const int r = __ffs(diff) - 1;
                diff &= diff - 1;
                zs = ((gn >> r) & 1) ? zs + wsm[r] : zs - wsm[r];
            }
            gi = gn;
        }
        const X el = __ldg(EL + ii) + zs;
        unsigned m = __ballot_sync(kFull, cmin + el <= umax);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const X els = __shfl_sync(kFull, el, src);
            const int is = off + src;
            X tp = Treg + mu - P - els;
            if (cm > tp)
                continue;
            const uint64_t cb = cbase | ((uint64_t)(is ^ (is >> 1)) << B);
            for (int g = 0; g < G; ++g) {
                X ev[V];
                vload<X>(Es + (g * 32 + lane) * V, ev);
                const X lg = lin_sm[g * 32 + lane];
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const X c = ev[e] + lin_e[e] + lin_t + lg;
                    if (c <= tp) {
                        const X Et = c + els + P;
                        const uint32_t j = (uint32_t)((g * 32 + lane) * V + e);
                        record<T>(a, inst, Et, unpermute(cb | j, d.perm));
                        if (K1 && Et < Treg) {
                            Treg = Et;
                            tp = Treg + mu - P - els;
                            Tr<T>::thr_min(st, Et);
                        }
                    }
                }
            }
        }
    }
    __syncwarp();
}

// Per-warp shared memory of the one-block kernel: two units' zero-row couplings and high-bit
// tables, the doubling scratch, and the column groups' fields of a hit unit.
template <class X, int S>
struct OneSmem {
    X wsm[2][kMaxWalkBits];
    X wt[2][1 << (kZMaxRows - 7)];
    X gs[1 << (kZMaxRows - 7)];
    X lin[S / 4 * 32];
};

template <class T, int S, bool K1>
__global__ void __launch_bounds__(kScanThreads, 6) zscan_one_kernel(const ScanArgs a)
{
    using X = typename Tr<T>::TC;
    __shared__ OneSmem<X, S> sm_all[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    OneSmem<X, S> &sm = sm_all[warp];
    typename Tr<T>::TP Treg = 0;
    // the persistent loop of persistent_units, taking the units of a claim two at a time
    constexpr unsigned long long kChunk = 8;
    int cur = -1;
    unsigned long long done = 0;
    unsigned long long next = lane == 0 ? atomicAdd(a.queue, kChunk) : 0ull;
    for (;;) {
        unsigned long long base = 0;
        int stop = 0;
        if (lane == 0) {
            stop = *a.abort_flag != 0;
            base = next;
            if (!stop && base < a.total_items)
                next = atomicAdd(a.queue, kChunk);
        }
        stop = __shfl_sync(kFull, stop, 0);
        base = __shfl_sync(kFull, base, 0);
        if (stop || base >= a.total_items)
            break;
        const unsigned long long end = base + kChunk < a.total_items ? base + kChunk : (unsigned long long)a.total_items;
        for (unsigned long long item = base; item < end;) {
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
                if (lane == 0 && done)
                    atomicAdd(&a.state[cur].scanned, done);
                done = 0;
                cur = inst;
                Treg = Tr<T>::thr_load(a.state + inst);
            }
            const Inst d = a.inst[inst];
            if (d.small) {
                small_unit<T>(a, d, inst, lane);  // counts its own states
                ++item;
                continue;
            }
            const uint64_t unit = d.unit_begin + (item - a.item_base[inst]);
            const bool pair = item + 1 < end && a.item_base[inst + 1] > item + 1;
            X f0a, cxa, cma, f0b = 0, cxb = 0, cmb = 0;
            unit_one_setup<T, S>(d, unit, lane, sm.wsm[0], f0a, cxa, cma);
            if (pair) {
                unit_one_setup<T, S>(d, unit + 1, lane, sm.wsm[1], f0b, cxb, cmb);
                X *const w[2] = {sm.wsm[0], sm.wsm[1]};
                X *const t[2] = {sm.wt[0], sm.wt[1]};
                X mel[2];
                walk_min_units<X, 2>((const X *)d.EL, d.L, lane, w, t, sm.gs, mel);
                unit_one_finish<T, S, K1>(a, d, inst, unit, Treg, lane, sm.wsm[0], sm.lin, f0a, cxa, cma, mel[0]);
                unit_one_finish<T, S, K1>(a, d, inst, unit + 1, Treg, lane, sm.wsm[1], sm.lin, f0b, cxb, cmb, mel[1]);
                done += 2ull << (d.B + d.L);
                item += 2;
            } else {
                X *const w[1] = {sm.wsm[0]};
                X *const t[1] = {sm.wt[0]};
                X mel[1];
                walk_min_units<X, 1>((const X *)d.EL, d.L, lane, w, t, sm.gs, mel);
                unit_one_finish<T, S, K1>(a, d, inst, unit, Treg, lane, sm.wsm[0], sm.lin, f0a, cxa, cma, mel[0]);
                done += 1ull << (d.B + d.L);
                item += 1;
            }
        }
    }
    if (lane == 0 && done)
        atomicAdd(&a.state[cur].scanned, done);
}

template <class T, bool K1>
auto zpick(int variant)
{
    return variant == 3   ? zscan_one_kernel<T, kZCols[3], K1>
           : variant == 2 ? zscan_kernel<T, kZCols[2], K1>
           : variant == 1 ? zscan_kernel<T, kZCols[1], K1>
                          : zscan_kernel<T, kZCols[0], K1>;
}

template <class T>
cudaError_t launch_z(const ScanArgs &a, int blocks, int variant, cudaStream_t s)
{
    auto k = a.k1 ? zpick<T, true>(variant) : zpick<T, false>(variant);
    k<<<blocks, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class T>
int z_blocks_per_sm(bool k1, int variant)
{
    int nb = 0;
    auto k = k1 ? zpick<T, true>(variant) : zpick<T, false>(variant);
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kScanThreads, 0);
    return e == cudaSuccess ? nb : -1;
}

}  // namespace

cudaError_t launch_zscan(const ScanArgs &a, int blocks, int variant, bool is_float, cudaStream_t s)
{
    return is_float ? launch_z<float>(a, blocks, variant, s) : launch_z<int32_t>(a, blocks, variant, s);
}

int zscan_blocks_per_sm(bool k1, int variant, bool is_float)
{
    return is_float ? z_blocks_per_sm<float>(k1, variant) : z_blocks_per_sm<int32_t>(k1, variant);
}

}  // namespace qubo
