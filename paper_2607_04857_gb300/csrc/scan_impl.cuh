// Exhaustive-scan kernels (table build and the persistent Gray-walk enumeration).
//
// Decomposition (Sec. 2, eq. 3-4; Sec. 3.3): a state code is split, low bits first, into
//   j   : B suffix bits, the columns (Sec. 3.3.2 column-wise split; 32 * S columns per unit),
//   g   : L prefix bits walked in reflected Gray order inside a unit (Sec. 3.2),
//   x_f : k = n - B - L fixed bits, one work unit per value (Sec. 3.3.1 straightforward split).
// For a unit, E(x_f, g, j) = c(x_f) + lin(x_f, g) + E_L(g) + E_sd(g, j) with
//   E_sd(0, j) = E_s(j) + sum_b j_b v_b(x_f)            (Q' = Q_rr + diag(x_f Q_fr))
//   E_sd(g', j) = E_sd(g, j) +/- M_k[j]                  (eq. incremental update)
// so each state costs one add, then one min over the thread's S columns and one compare of
// that min with a per-step threshold (the argmin / strict-less update of Alg. 2, extended to
// keep every state at or below the running K-th best).
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include "internal.h"

namespace qubo {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t ord32(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord32(uint32_t o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}
__device__ __forceinline__ unsigned long long ord64(double d)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord64(unsigned long long o)
{
    return __longlong_as_double((long long)((o & 0x8000000000000000ull) ? (o & 0x7fffffffffffffffull) : ~o));
}

// ---- accumulator traits ----------------------------------------------------------------------
// TC: type of the column energies and table rows; TP: type of the prefix energy, thresholds and
// recorded energies; F: table-build precision; FU: per-unit field precision.
template <class T>
struct Tr;

// Integer instances whose partial sums stay below 2^24 in magnitude: columns and tables are FP32
// holding exact integers (FP32 adds use both halves of the fused multiply-add pipe), while the
// prefix energy and thresholds stay int32.
struct i32f {};
struct i16p {};

template <>
struct Tr<int32_t> {
    // No grouped step form: integer adds are associative, so the compiler folds a skipped group's
    // 15 column updates into one, and the scan would no longer form every state's energy.
    static constexpr bool kGrouped = false;
    using TC = int32_t;
    using TP = int32_t;
    static constexpr bool kIntInFloat = false;
    static constexpr int kPack = 1;
    using F = int32_t;   // precision of the tables
    using FU = int32_t;  // precision of the per-unit fields
    using Vec = int4;
    static constexpr int V = 4;
    static constexpr bool kFloat = false;
    __device__ static int32_t thr_load(const InstState *s) { return *(const volatile int32_t *)&s->thr; }
    __device__ static void thr_min(InstState *s, int32_t v) { atomicMin((int *)&s->thr, v); }
    __device__ static void gmin_min(InstState *s, int32_t v) { atomicMin((int *)&s->gmin, v); }
    __device__ static int64_t bits(int32_t v) { return v; }
    __device__ static int32_t tmin(int32_t a, int32_t b) { return min(a, b); }
    __device__ static int32_t tmin3(int32_t a, int32_t b, int32_t c) { return __vimin3_s32(a, b, c); }
};

template <>
struct Tr<int64_t> {
    static constexpr bool kGrouped = false;
    using TC = int64_t;
    using TP = int64_t;
    static constexpr bool kIntInFloat = false;
    static constexpr int kPack = 1;
    using F = int64_t;
    using FU = int64_t;
    using Vec = longlong2;
    static constexpr int V = 2;
    static constexpr bool kFloat = false;
    __device__ static int64_t thr_load(const InstState *s) { return *(const volatile long long *)&s->thr; }
    __device__ static void thr_min(InstState *s, int64_t v) { atomicMin((long long *)&s->thr, (long long)v); }
    __device__ static void gmin_min(InstState *s, int64_t v) { atomicMin((long long *)&s->gmin, (long long)v); }
    __device__ static int64_t bits(int64_t v) { return v; }
    __device__ static int64_t tmin(int64_t a, int64_t b) { return min(a, b); }
    __device__ static int64_t tmin3(int64_t a, int64_t b, int64_t c) { return min(min(a, b), c); }
};

template <>
struct Tr<float> {
    static constexpr bool kGrouped = true;
    using TC = float;
    using TP = float;
    static constexpr bool kIntInFloat = false;
    static constexpr int kPack = 1;
    using F = double;
    using FU = float;
    using Vec = float4;
    static constexpr int V = 4;
    static constexpr bool kFloat = true;
    __device__ static float thr_load(const InstState *s) { return unord32(*(const volatile uint32_t *)&s->thr); }
    __device__ static void thr_min(InstState *s, float v) { atomicMin((unsigned *)&s->thr, ord32(v)); }
    __device__ static void gmin_min(InstState *s, float v) { atomicMin((unsigned *)&s->gmin, ord32(v)); }
    __device__ static int64_t bits(float v) { return __double_as_longlong((double)v); }
    __device__ static float tmin(float a, float b) { return fminf(a, b); }
    __device__ static float tmin3(float a, float b, float c)
    {
        float d;
        asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
        return d;
    }
};

template <>
struct Tr<double> {
    static constexpr bool kGrouped = false;
    using TC = double;
    using TP = double;
    static constexpr bool kIntInFloat = false;
    static constexpr int kPack = 1;
    using F = double;
    using FU = double;
    using Vec = double2;
    static constexpr int V = 2;
    static constexpr bool kFloat = true;
    __device__ static double thr_load(const InstState *s)
    {
        return unord64(*(const volatile unsigned long long *)&s->thr);
    }
    __device__ static void thr_min(InstState *s, double v) { atomicMin(&s->thr, ord64(v)); }
    __device__ static void gmin_min(InstState *s, double v) { atomicMin(&s->gmin, ord64(v)); }
    __device__ static int64_t bits(double v) { return __double_as_longlong(v); }
    __device__ static double tmin(double a, double b) { return fmin(a, b); }
    __device__ static double tmin3(double a, double b, double c) { return fmin(fmin(a, b), c); }
};

// Symmetric coupling matrix in the table precision (tables) and in the unit-field precision.
template <>
struct Tr<i32f> {
    static constexpr bool kGrouped = true;  // compiles the grouped step form (variants 20-23)
    using TC = float;
    using TP = int32_t;
    static constexpr bool kIntInFloat = true;
    static constexpr int kPack = 1;
    using F = int32_t;
    using FU = int32_t;
    using Vec = float4;
    static constexpr int V = 4;
    static constexpr bool kFloat = false;
    __device__ static int32_t thr_load(const InstState *s) { return *(const volatile int32_t *)&s->thr; }
    __device__ static void thr_min(InstState *s, int32_t v) { atomicMin((int *)&s->thr, v); }
    __device__ static void gmin_min(InstState *s, int32_t v) { atomicMin((int *)&s->gmin, v); }
    __device__ static int64_t bits(int32_t v) { return v; }
    __device__ static int32_t tmin(int32_t a, int32_t b) { return min(a, b); }
};

// Small integer instances (every column energy within +-32767): two columns per 32-bit word,
// each a 16-bit lane biased by 2^15, so one 32-bit add updates both columns exactly (no lane
// ever leaves [0, 65535], so no carry crosses) and packed unsigned mins reduce two per
// instruction.  The table rows are stored as packed deltas lo + 65536 * hi.
template <>
struct Tr<i16p> {
    static constexpr bool kGrouped = false;
    using TC = uint32_t;
    using TP = int32_t;
    static constexpr bool kIntInFloat = false;
    static constexpr int kPack = 2;
    using F = int32_t;
    using FU = int32_t;
    using Vec = uint4;
    static constexpr int V = 4;
    static constexpr bool kFloat = false;
    __device__ static int32_t thr_load(const InstState *s) { return *(const volatile int32_t *)&s->thr; }
    __device__ static void thr_min(InstState *s, int32_t v) { atomicMin((int *)&s->thr, v); }
    __device__ static void gmin_min(InstState *s, int32_t v) { atomicMin((int *)&s->gmin, v); }
    __device__ static int64_t bits(int32_t v) { return v; }
    __device__ static int32_t tmin(int32_t a, int32_t b) { return min(a, b); }
};
constexpr int32_t kLaneBias = 32768;

// Column value of a prefix-type threshold.  For FP32 columns holding integers the threshold is
// clamped to +-C first: beyond C every column (|column| <= C - 1 - max|E_L|) is decided the same
// way, and within it the value is exact in FP32.
template <class T>
__device__ __forceinline__ typename Tr<T>::TC to_col(typename Tr<T>::TP v, int32_t clampC)
{
    if constexpr (Tr<T>::kIntInFloat)
        return (float)max(-clampC, min(clampC, v));
    else
        return v;
}

template <class T>
__device__ __forceinline__ const typename Tr<T>::F *field_matrix(const Inst &d)
{
    if constexpr (Tr<T>::kFloat)
        return d.W64;
    else
        return (const typename Tr<T>::F *)d.W;
}
template <class T>
__device__ __forceinline__ const typename Tr<T>::FU *unit_matrix(const Inst &d)
{
    return (const typename Tr<T>::FU *)d.W;
}


__device__ __forceinline__ void vsplit(const int4 &v, int32_t (&o)[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
__device__ __forceinline__ void vsplit(const float4 &v, float (&o)[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
__device__ __forceinline__ void vsplit(const longlong2 &v, int64_t (&o)[2]) { o[0] = v.x; o[1] = v.y; }
__device__ __forceinline__ void vsplit(const uint4 &v, uint32_t (&o)[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
__device__ __forceinline__ void vsplit(const double2 &v, double (&o)[2]) { o[0] = v.x; o[1] = v.y; }

// 16-byte read-only load of consecutive table entries (4 x 4 bytes or 2 x 8 bytes).
template <class E>
struct VecOf;
template <>
struct VecOf<int32_t> { using type = int4; static constexpr int V = 4; };
template <>
struct VecOf<float> { using type = float4; static constexpr int V = 4; };
template <>
struct VecOf<int64_t> { using type = longlong2; static constexpr int V = 2; };
template <>
struct VecOf<uint32_t> { using type = uint4; static constexpr int V = 4; };
template <>
struct VecOf<double> { using type = double2; static constexpr int V = 2; };

template <class E>
__device__ __forceinline__ void vload(const E *p, E (&o)[VecOf<E>::V])
{
    vsplit(__ldg((const typename VecOf<E>::type *)p), o);
}
__device__ __forceinline__ float4 vjoin(const float *v) { return make_float4(v[0], v[1], v[2], v[3]); }
__device__ __forceinline__ double2 vjoin(const double *v) { return make_double2(v[0], v[1]); }

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }
__host__ __device__ constexpr int ctzc(int v) { return (v & 1) ? 0 : 1 + ctzc(v >> 1); }

template <int N, class Fn>
__device__ __forceinline__ void static_for(Fn &&fn)
{
    [&]<int... I>(std::integer_sequence<int, I...>) { (fn(std::integral_constant<int, I>{}), ...); }(
        std::make_integer_sequence<int, N>{});
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int32_t emin(int32_t a, int32_t b) { return min(a, b); }
__device__ __forceinline__ int64_t emin(int64_t a, int64_t b) { return min(a, b); }
__device__ __forceinline__ float emin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double emin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ int32_t emin3(int32_t a, int32_t b, int32_t c) { return __vimin3_s32(a, b, c); }
__device__ __forceinline__ int64_t emin3(int64_t a, int64_t b, int64_t c) { return min(min(a, b), c); }
__device__ __forceinline__ float emin3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ double emin3(double a, double b, double c) { return fmin(fmin(a, b), c); }
// uint32 columns are pairs of biased 16-bit lanes: lane-wise unsigned mins.
__device__ __forceinline__ uint32_t emin(uint32_t a, uint32_t b) { return __vminu2(a, b); }
__device__ __forceinline__ uint32_t emin3(uint32_t a, uint32_t b, uint32_t c) { return __vimin3_u16x2(a, b, c); }

// Paired FP32 arithmetic (one instruction updates two columns): x += a, y += b; x -= a, y -= b;
// x += a * s, y += b * s.  Each lane is rounded exactly as the scalar operation would be.
__device__ __forceinline__ void add_f32x2(float &x, float &y, float a, float b)
{
    asm("{\n\t.reg .b64 p, q;\n\tmov.b64 p, {%0, %1};\n\tmov.b64 q, {%2, %3};\n\t"
        "add.rn.f32x2 p, p, q;\n\tmov.b64 {%0, %1}, p;\n\t}"
        : "+f"(x), "+f"(y) : "f"(a), "f"(b));
}
__device__ __forceinline__ void sub_f32x2(float &x, float &y, float a, float b)
{
    asm("{\n\t.reg .b64 p, q;\n\tmov.b64 p, {%0, %1};\n\tmov.b64 q, {%2, %3};\n\t"
        "sub.rn.f32x2 p, p, q;\n\tmov.b64 {%0, %1}, p;\n\t}"
        : "+f"(x), "+f"(y) : "f"(a), "f"(b));
}
__device__ __forceinline__ void fma_f32x2(float &x, float &y, float a, float b, float s)
{
    asm("{\n\t.reg .b64 p, q, r;\n\tmov.b64 p, {%0, %1};\n\tmov.b64 q, {%2, %3};\n\tmov.b64 r, {%4, %4};\n\t"
        "fma.rn.f32x2 p, q, r, p;\n\tmov.b64 {%0, %1}, p;\n\t}"
        : "+f"(x), "+f"(y) : "f"(a), "f"(b), "f"(s));
}

// min over N register values: a tree of 2-input (MINM == 2) or 3-input (MINM == 3) mins.
template <class T, int MINM, int N>
__device__ __forceinline__ T tree_min(const T (&E)[N])
{
    if constexpr (N == 1) {
        return E[0];
    } else if constexpr (MINM == 3 && N >= 3) {
        constexpr int M = N / 3 + (N % 3);
        T m[M];
#pragma unroll
        for (int q = 0; q < N / 3; ++q)
            m[q] = emin3(E[3 * q], E[3 * q + 1], E[3 * q + 2]);
#pragma unroll
        for (int q = 0; q < N % 3; ++q)
            m[N / 3 + q] = E[3 * (N / 3) + q];
        return tree_min<T, MINM, M>(m);
    } else {
        constexpr int M = N / 2 + (N % 2);
        T m[M];
#pragma unroll
        for (int q = 0; q < N / 2; ++q)
            m[q] = emin(E[2 * q], E[2 * q + 1]);
        if constexpr (N % 2)
            m[M - 1] = E[N - 1];
        return tree_min<T, MINM, M>(m);
    }
}

// Offer one state to the candidate buffer.
template <class T>
__device__ __forceinline__ void record(const ScanArgs &a, int inst, typename Tr<T>::TP E, uint64_t code)
{
    InstState *st = a.state + inst;
    atomicAdd(&st->nrec, 1ull);
    const unsigned long long idx = atomicAdd(a.nrec, 1ull);
    if (idx < a.rec_cap) {
        Rec r;
        r.key = a.n_inst > 1 ? (((uint64_t)inst << kInstShift) | code) : code;
        r.e = Tr<T>::bits(E);
        a.rec[idx] = r;
    } else {
        atomicAdd(&st->dropped, 1ull);
    }
    Tr<T>::gmin_min(st, E);
}

// ---- table build (preprocessing of Alg. 1-2: E(U_B), M_int = Q_ps U_B^T, E(U_A)) ------------------
// One thread per table entry; entries are subset sums of the symmetric coupling matrix W.
template <class T>
__global__ void tables_kernel(const Inst *insts)
{
    using F = typename Tr<T>::F;
    using TC = typename Tr<T>::TC;
    using TP = typename Tr<T>::TP;
    constexpr bool kPacked = Tr<T>::kPack == 2;
    const Inst &d = insts[blockIdx.y];
    if (d.small)
        return;
    const int n = d.n, B = d.B, L = d.L;
    const long NB = 1l << B, NL = 1l << L;
    const long NM = kPacked ? NB / 2 : NB;  // words per interaction row
    // the grouped scans (integers in FP32 lanes, FP32): after E_L, the minimum of E_L over each
    // group of 16 walk steps, as stored
    const long NLG = Tr<T>::kGrouped ? NL / 16 : 0;
    const long total = NB + NM * L + NL + NLG;
    const F *W = field_matrix<T>(d);
    // M_int row r at column j: coupling of walked variable r to the suffix pattern j
    auto m_entry = [&](long r, long j) {
        const int vr = B + (int)r;
        F acc = 0;
        for (int b = 0; b < B; ++b)
            if ((j >> b) & 1)
                acc += W[vr * n + b];
        return acc;
    };
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        if (idx < NB) {  // E_s(j): energy of the suffix pattern j alone
            const long j = idx;
            F acc = 0;
            for (int b = 0; b < B; ++b) {
                if (!((j >> b) & 1))
                    continue;
                acc += W[b * n + b];
                for (int b2 = b + 1; b2 < B; ++b2)
                    if ((j >> b2) & 1)
                        acc += W[b * n + b2];
            }
            if constexpr (kPacked)
                ((TP *)d.Es)[j] = (TP)acc;
            else
                ((TC *)d.Es)[j] = (TC)acc;
        } else if (idx < NB + NM * L) {
            const long r = (idx - NB) / NM, w = (idx - NB) % NM;
            if constexpr (kPacked)  // packed delta: column w in the low lane, w + NB/2 in the high
                ((TC *)d.M)[r * NM + w] = (uint32_t)m_entry(r, w) + ((uint32_t)m_entry(r, w + NB / 2) << 16);
            else
                ((TC *)d.M)[r * NM + w] = (TC)m_entry(r, w);
        } else {  // E_L(g(i)): energy of the i-th walked pattern, stored in walk order
            const long i = idx - NB - NM * L;
            auto el_of = [&](long ii) {
                const long g = ii ^ (ii >> 1);
                F e = 0;
                for (int r = 0; r < L; ++r) {
                    if (!((g >> r) & 1))
                        continue;
                    e += W[(B + r) * n + (B + r)];
                    for (int r2 = r + 1; r2 < L; ++r2)
                        if ((g >> r2) & 1)
                            e += W[(B + r) * n + (B + r2)];
                }
                return e;
            };
            if (i >= NL) {  // group minimum (grouped scans; rounding to TC is monotonic)
                const long g0 = 16 * (i - NL);
                F m = el_of(g0);
                for (int t = 1; t < 16; ++t)
                    m = min(m, el_of(g0 + t));
                ((TC *)d.EL)[i] = (TC)m;
                continue;
            }
            const F acc = el_of(i);
            if constexpr (kPacked) {
                if (d.el_fused)  // E_L - elmin in both halves, added to the packed minima of a step
                    ((uint32_t *)d.EL)[i] = (uint32_t)((TP)acc - d.elmin) * 0x10001u;
                else  // stored minus the lane bias: threshold - E_L is then a lane value
                    ((TP *)d.EL)[i] = (TP)acc - kLaneBias;
            } else {
                ((TC *)d.EL)[i] = (TC)acc;
            }
        }
    }
}

// ---- direct evaluation for sub-cubes too small to split ---------------------------------------
template <class T>
__device__ void small_unit(const ScanArgs &a, const Inst &d, int inst, int lane)
{
    using F = typename Tr<T>::F;
    const int n = d.n;
    const F *W = field_matrix<T>(d);
    // states above the run's threshold (plus margin) cannot be in the answer
    const double lim = (double)Tr<T>::thr_load(a.state + inst) + a.margin;
    for (uint64_t s = lane; s < d.sub_count; s += 32) {
        const uint64_t x = d.sub_base + s;
        F acc = 0;
        for (int i = 0; i < n; ++i) {
            if (!((x >> i) & 1))
                continue;
            acc += W[i * n + i];
            for (int j = i + 1; j < n; ++j)
                if ((x >> j) & 1)
                    acc += W[i * n + j];
        }
        if ((double)acc <= lim + (Tr<T>::kFloat ? 1e-6 * (1.0 + fabs(lim)) : 0.0))
            record<T>(a, inst, (typename Tr<T>::TP)acc, x);
    }
    if (lane == 0)
        atomicAdd(&a.state[inst].scanned, (unsigned long long)d.sub_count);
}

// Fields of the set fixed bits of unit x_f: lane l returns in f0 the coupling of variable l
// (l < B + L) to the set fixed variables, and every lane returns c(x_f), the energy of the fixed
// variables alone (Sec. 3.3.1: Q' = Q_rr + diag(x_f Q_fr), c(x_f) = x_f Q_ff x_f^T).
template <class T, class F = typename Tr<T>::FU>
__device__ __forceinline__ void unit_fields(const F *W, int n, int k, int BL, uint64_t unit, int lane, F &f0, F &cx)
{
    F a0 = 0, up0 = 0, up1 = 0;
    for (int f = 0; f < k; ++f) {
        if (!((unit >> f) & 1ull))
            continue;
        const int vf = BL + f;
        const F *row = W + (size_t)vf * n;
        if (lane < n && lane != vf) {
            const F w = row[lane];
            a0 += w;
            if (vf > lane)
                up0 += w;
        }
        if (lane + 32 < n && lane + 32 != vf && vf > lane + 32)
            up1 += row[lane + 32];
    }
    F cpart = 0;
    if (lane >= BL && lane < n && ((unit >> (lane - BL)) & 1ull))
        cpart += W[lane * n + lane] + up0;
    if (lane + 32 >= BL && lane + 32 < n && ((unit >> (lane + 32 - BL)) & 1ull))
        cpart += W[(lane + 32) * n + lane + 32] + up1;
    f0 = a0;
    cx = warp_sum(cpart);
}

// Subset sums of the suffix fields over the bits of this thread's columns
// j = (g * 32 + lane) * V + e: lin(j) = lin_e[e] + lin_t + lin_g[g].
template <class F, int V, int G>
__device__ __forceinline__ void column_fields(F f0, int lane, F &lin_t, F (&lin_e)[V], F (&lin_g)[G])
{
    constexpr int LOGV = ilog2c(V), LOGG = ilog2c(G);
    lin_t = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const F vb = __shfl_sync(kFull, f0, LOGV + i);
        if ((lane >> i) & 1)
            lin_t += vb;
    }
    lin_e[0] = 0;
#pragma unroll
    for (int i = 0; i < LOGV; ++i) {
        const F vb = __shfl_sync(kFull, f0, i);
#pragma unroll
        for (int e = 0; e < (1 << i); ++e)
            lin_e[e + (1 << i)] = lin_e[e] + vb;
    }
    lin_g[0] = 0;
#pragma unroll
    for (int i = 0; i < LOGG; ++i) {
        const F vb = __shfl_sync(kFull, f0, LOGV + 5 + i);
#pragma unroll
        for (int g = 0; g < (1 << i); ++g)
            lin_g[g + (1 << i)] = lin_g[g] + vb;
    }
}

// One register-row Gray step of S columns, adds only: E[q] +- M[q], pairs of FP32 columns as one
// f32x2 instruction where the add mode says so (4: all pairs, 5: every 2nd, 6: every 4th, 7: 3 of 4).
template <class TC, int S, int ADDM, bool NEG>
__device__ __forceinline__ void add_row(TC (&E)[S], const TC (&M)[S])
{
    if constexpr (ADDM >= 4 && std::is_same_v<TC, float>) {
#pragma unroll
        for (int q = 0; q < S; q += 2) {
            const int pr = q / 2;
            if (ADDM == 4 || (ADDM == 5 && pr % 2 == 0) || (ADDM == 6 && pr % 4 == 0) || (ADDM == 7 && pr % 4 != 0)) {
                if constexpr (NEG)
                    sub_f32x2(E[q], E[q + 1], M[q], M[q + 1]);
                else
                    add_f32x2(E[q], E[q + 1], M[q], M[q + 1]);
            } else {
                E[q] = NEG ? E[q] - M[q] : E[q] + M[q];
                E[q + 1] = NEG ? E[q + 1] - M[q + 1] : E[q + 1] + M[q + 1];
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < S; ++q)
            E[q] = NEG ? E[q] - M[q] : E[q] + M[q];
    }
}

// One register-row Gray step of S columns fused with the min over them, in an interleaved order:
// each triple of columns is reduced by a 3-input min as soon as its adds are issued, so the FMA
// pipe (adds) and the ALU pipe (mins) receive alternating work from one warp.  Pair q of columns
// is one f32x2 instruction where the add mode says so (as in scan_unit).  Returns the minimum.
template <bool PAIRED, bool NEG, class TC>
__device__ __forceinline__ void add_pair(TC &x, TC &y, TC a, TC b)
{
    if constexpr (PAIRED && std::is_same_v<TC, float>) {
        if constexpr (NEG)
            sub_f32x2(x, y, a, b);
        else
            add_f32x2(x, y, a, b);
    } else {
        x = NEG ? x - a : x + a;
        y = NEG ? y - b : y + b;
    }
}

// Integer column update as a 3-input add with a run-time zero, which issues to the ALU pipe
// rather than the FMA-heavy pipe that takes the plain integer adds (shares the adds between the
// two pipes; the value is the plain sum).
template <bool NEG, class TC>
__device__ __forceinline__ void add_alu(TC &x, TC a, TC z)
{
    x = NEG ? (x - a) + z : (x + a) + z;
}

// ADDM 2 / 3 (integer columns): one column in four / in eight updated on the ALU pipe.
template <class TC, int S, int ADDM, bool NEG>
__device__ __forceinline__ TC add_min_interleaved(TC (&E)[S], const TC (&M)[S], TC z = TC(0))
{
    constexpr int NT = S / 3, NL = NT + S % 3;
    TC l1[NL];
    static_for<S / 2>([&](auto pc) {
        constexpr int pr = decltype(pc)::value, q = 2 * pr;
        constexpr bool paired = ADDM == 4 || (ADDM == 5 && pr % 2 == 0) || (ADDM == 6 && pr % 4 == 0) ||
                                (ADDM == 7 && pr % 4 != 0);
        constexpr bool alu = !std::is_same_v<TC, float> && ((ADDM == 2 && q % 4 == 0) || (ADDM == 3 && q % 8 == 0));
        if constexpr (alu) {
            add_alu<NEG>(E[q], M[q], z);
            E[q + 1] = NEG ? E[q + 1] - M[q + 1] : E[q + 1] + M[q + 1];
        } else {
            add_pair<paired, NEG>(E[q], E[q + 1], M[q], M[q + 1]);
        }
        // triples completed by this pair: (3t, 3t+1, 3t+2) with 3t+2 in {q, q+1}
        static_for<2>([&](auto cc) {
            constexpr int c = q + decltype(cc)::value;
            if constexpr (c % 3 == 2 && c / 3 < NT)
                l1[c / 3] = emin3(E[c - 2], E[c - 1], E[c]);
        });
    });
    static_for<S % 3>([&](auto rc) {
        constexpr int c = 3 * NT + decltype(rc)::value;
        l1[NT + decltype(rc)::value] = E[c];
    });
    return tree_min<TC, 3, NL>(l1);
}

// ---- one work unit: all 2^(B+L) states with fixed bits x_f = unit --------------------------------
// ADDM >= 4 issues some or all FP32 column adds as paired f32x2 operations (two columns per
// instruction; 4: all pairs, 5: every second, 6: every fourth, 7: three in four); other modes
// leave the adds to the compiler.  MINM selects 2- or 3-input mins.
template <class T, int S, int RC, bool K1, int ADDM, int MINM, int ILV = 0>
__device__ __forceinline__ void scan_unit(const ScanArgs &a, const Inst &d, int inst, uint64_t unit,
                                          typename Tr<T>::TP &Treg, int lane, typename Tr<T>::TC *stage,
                                          typename Tr<T>::TP *wsm, typename Tr<T>::TC *anc)
{
    using F = typename Tr<T>::FU;
    using TC = typename Tr<T>::TC;
    using TP = typename Tr<T>::TP;
    constexpr int V = VecOf<TC>::V;
    constexpr int G = S / V;
    constexpr int LOGV = ilog2c(V);
    constexpr int LOGG = ilog2c(G);
    constexpr int B = LOGV + 5 + LOGG;
    constexpr int NB = 1 << B;
    constexpr int BODY = 1 << (RC + 1);
    const int n = d.n, L = d.L, k = d.k, BL = B + L;
    InstState *st = a.state + inst;
    // Fields of the set fixed bits on every other variable and c(x_f) (Sec. 3.3.1).  FP32 scans
    // sum them in FP64 and round each once (their rounding bound then carries one rounding per
    // field and per c(x_f), not one per term).
    F f0, cx;
    if constexpr (std::is_same_v<F, float>) {
        double f0d, cxd;
        unit_fields<T, double>(d.W64, n, k, BL, unit, lane, f0d, cxd);
        f0 = (float)f0d;
        cx = (float)cxd;
    } else {
        unit_fields<T, F>(unit_matrix<T>(d), n, k, BL, unit, lane, f0, cx);
    }
    // Walked-row couplings w_r, read at every flip of a row >= RC.
    __syncwarp();
    if (lane >= B && lane < BL)
        wsm[lane - B] = (TP)f0;
    __syncwarp();

    // Column fields: lin(j) = sum_b j_b v_b; bits of j are [e | lane | g] (LOGV, 5, LOGG bits).
    F lin_t, lin_e[V], lin_g[G];
    column_fields<F, V, G>(f0, lane, lin_t, lin_e, lin_g);

    // Initial suffix-dependent energies (walked bits all zero): E_s(j) + lin(j).
    const TC *Es = (const TC *)d.Es;
    TC E[S];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        TC ev[V];
        vload<TC>(Es + (g * 32 + lane) * V, ev);
#pragma unroll
        for (int e = 0; e < V; ++e)
            E[g * V + e] = (TC)((F)ev[e] + (lin_e[e] + lin_t + lin_g[g]));
    }
    if constexpr (Tr<T>::kFloat) {
        // float scans: these columns (walked bits all zero) are the base of every re-anchoring
#pragma unroll
        for (int g = 0; g < G; ++g)
            *(typename VecOf<TC>::type *)(anc + (g * 32 + lane) * V) = vjoin(E + g * V);
    }

    // Register rows r < RC: M_r[j] + w_r, the walked-fixed coupling of row r folded in.
    const TC *Mt = (const TC *)d.M;
    TC Mr[RC][S];
#pragma unroll
    for (int r = 0; r < RC; ++r) {
        const F wr = __shfl_sync(kFull, f0, B + r);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            TC mv[V];
            vload<TC>(Mt + (size_t)r * NB + (g * 32 + lane) * V, mv);
#pragma unroll
            for (int e = 0; e < V; ++e)
                Mr[r][g * V + e] = (TC)((F)mv[e] + wr);
        }
    }

    // Step form 2 (integers in FP32 lanes): the walk runs in groups of 16 states, and a group
    // skips the min tree when no column of it can reach the threshold.  At a group's first state
    // the exact column minimum m of each thread is taken; a register-row step adds +-M_r[q] to
    // column q, so over the group's next 15 steps (rows 0-3, the same pattern in every group but
    // for the sign of row 3, which alternates) the minimum never falls below m + D, D the
    // smallest running sum of the steps' smallest column moves (min_q M_r[q] on an add,
    // -max_q M_r[q] on a subtract), computed once per unit in int32 and rounded down.  With
    // min E_L over the group's states (a table), m + D > uc - min E_L in every lane proves that
    // the group holds no candidate, and it runs its adds alone.  m + D is summed rounding down;
    // with integers in FP32 lanes uc - min E_L is exact (|uc|, |E_L| and their difference stay
    // below 2^24).  FP32 columns take 16 ulp of beta (geps) off the left side, more than the
    // rounding of the group's 15 adds and of the E_L add the interleaved form compares, and round
    // uc - min E_L up, so a group is skipped only when the interleaved form records nothing in it.
    constexpr bool BOUND = ILV == 2 && Tr<T>::kGrouped;
    static_assert(!BOUND || (RC >= 4 && MINM == 3), "the grouped form needs register rows 0-3 and 3-input mins");
    // D per parity of the group index, rounded down to FP32 (summed exactly in int64 for integer
    // columns, in FP64 for FP32 columns, whose table rows are FP32 values)
    using DD = std::conditional_t<Tr<T>::kFloat, double, int64_t>;
    float Dgrp[2] = {0, 0};
    if constexpr (BOUND) {
        DD dpos[4], dneg[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            TC lo = Mr[r][0], hi = Mr[r][0];
#pragma unroll
            for (int q = 1; q < S; ++q) {
                lo = emin(lo, Mr[r][q]);
                hi = hi > Mr[r][q] ? hi : Mr[r][q];
            }
            dpos[r] = (DD)lo;
            dneg[r] = -(DD)hi;
        }
        static_for<2>([&](auto pc) {
            constexpr int par = decltype(pc)::value;
            DD cum = 0, lo = 0;
            static_for<15>([&](auto tc) {
                constexpr int t = decltype(tc)::value + 1, kk = ctzc(t);
                constexpr bool neg = kk == 3 ? par != 0 : ((t >> (kk + 1)) & 1) != 0;
                cum += neg ? dneg[kk] : dpos[kk];
                lo = min(lo, cum);
            });
            if constexpr (Tr<T>::kFloat)
                Dgrp[par] = __double2float_rd(lo);
            else
                Dgrp[par] = __ll2float_rd(lo);
        });
    }

    // Threshold: a state is recorded when its energy is <= Treg (+ margin).
    {
        const TP tg = Tr<T>::thr_load(st);
        Treg = K1 ? min(Treg, tg) : tg;
    }
    const TP mu = (TP)a.margin;
    const int32_t clampC = d.clampC;
    TP P = (TP)cx;  // c(x_f) + coupling of the walked rows >= RC that are set
    TP u = Treg + mu - P;
    TC uc = to_col<T>(u, clampC);

    // Flip of a walked row kk >= RC (row from memory, runtime sign).
    auto high_flip = [&](int kk, int sgn) {
        if (!QUBO_DCHECK(kk >= RC && kk < L, st, 1))
            kk = RC;
        const TC *row = Mt + (size_t)kk * NB;
        const TC sg = (TC)sgn;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            TC mv[V];
            vload<TC>(row + (g * 32 + lane) * V, mv);
            if constexpr (ADDM >= 4 && std::is_same_v<TC, float>) {
#pragma unroll
                for (int e = 0; e < V; e += 2)
                    fma_f32x2(E[g * V + e], E[g * V + e + 1], mv[e], mv[e + 1], sg);
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                    E[g * V + e] = E[g * V + e] + sg * mv[e];
            }
        }
        P = P + (TP)sgn * wsm[kk];
        u = Treg + mu - P;
        uc = to_col<T>(u, clampC);
    };

    // Float scans re-anchor (Sec. 6.2, periodic correction): at walk step i (a multiple of 2^(RC+1),
    // so the register rows are clear) the columns are rebuilt as the base columns plus the rows of
    // the set walked bits, and P as c(x_f) plus their couplings; the largest difference to the
    // incrementally updated values is the drift the host checks against the candidate margin.
    // Mid-walk anchors every 2^anchor steps; one at the walk's end in any case.
    TC dl = 0;
    auto reanchor = [&](int i) {
        const int gi = i ^ (i >> 1);
        TP Pf = (TP)cx;
        TC fr[S];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            TC bv[V];
            vsplit(*(const typename VecOf<TC>::type *)(anc + (g * 32 + lane) * V), bv);
#pragma unroll
            for (int e = 0; e < V; ++e)
                fr[g * V + e] = bv[e];
        }
        for (unsigned bits = (unsigned)gi >> RC; bits; bits &= bits - 1) {
            int r = RC + __ffs(bits) - 1;
            if (!QUBO_DCHECK(r < L, st, 2))
                r = RC;
            Pf = Pf + wsm[r];
            const TC *row = Mt + (size_t)r * NB;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                TC mv[V];
                vload<TC>(row + (g * 32 + lane) * V, mv);
#pragma unroll
                for (int e = 0; e < V; ++e)
                    fr[g * V + e] = fr[g * V + e] + mv[e];
            }
        }
#pragma unroll
        for (int q = 0; q < S; ++q) {
            const TC dd = E[q] - fr[q];  // exact for close values
            const TC ad = dd < 0 ? -dd : dd;
            dl = dl > ad ? dl : ad;
            E[q] = fr[q];
        }
        const TC dp = (TC)(P < Pf ? Pf - P : P - Pf);
        dl = dl > dp ? dl : dp;
        P = Pf;
        u = Treg + mu - P;
        uc = to_col<T>(u, clampC);
    };
    // anchor period in bodies minus one; -1 (never) without mid-walk anchors
    const int amask = (Tr<T>::kFloat && d.anchor > RC && d.anchor < L) ? (1 << (d.anchor - RC - 1)) - 1 : -1;

    const TC *ELp = (const TC *)d.EL;
    const int nblk = 1 << (L - RC - 1);
    const uint64_t cbase = unit << BL;

    if (!QUBO_DCHECK(L >= RC + 1 && L <= kMaxWalkBits && nblk * BODY == (1 << L), st, 3))
        return;
    const TC *ELg = ELp + (1 << L);  // step form 2: min E_L over each group of 16 states
    for (int blk = 0; blk < nblk; ++blk) {
        const int i0 = blk * BODY;
        if constexpr (Tr<T>::kFloat) {
            if (blk != 0 && (blk & amask) == 0)
                reanchor(i0);
        }
        TC elv[V];
        bool hit = false;
        TP Pmid = P;
        // Running minima over the steps of each half body (the row-RC flip between the halves
        // moves the threshold) of (minimum over the columns + E_L of the step); a column can be
        // at or below the threshold exactly when its half's minimum is at or below uc.
        TC acc_lo, acc_hi, mprev;
        if constexpr (BOUND) {
            constexpr int NG = BODY / 16;
            TC elg[NG];
#pragma unroll
            for (int g = 0; g < NG; ++g)
                elg[g] = ELg[(i0 >> 4) + g];
            static_for<NG>([&](auto gc) {
                constexpr int g = decltype(gc)::value, p0 = 16 * g;
                if constexpr (g > 0) {  // the step into the group's first state
                    constexpr int kk = ctzc(p0);
                    if constexpr (kk < RC) {
                        add_row<TC, S, ADDM, ((p0 >> (kk + 1)) & 1) != 0>(E, Mr[kk]);
                    } else {
                        Pmid = P;
                        high_flip(RC, (blk & 1) ? -1 : 1);
                    }
                }
                const TC m0 = tree_min<TC, MINM, S>(E);
                bool clear;
                if constexpr (Tr<T>::kFloat)  // less the rounding of the group's adds and E_L add
                    clear = __fadd_rd(__fadd_rd(m0, Dgrp[g & 1]), -d.geps) > __fsub_ru(uc, elg[g]);
                else
                    clear = __fadd_rd(m0, Dgrp[g & 1]) > uc - elg[g];
                const bool skip = __all_sync(kFull, clear);
                if (__builtin_expect(skip, 1)) {
                    static_for<15>([&](auto tc) {
                        constexpr int t = decltype(tc)::value + 1, p = 16 * decltype(gc)::value + t, kk = ctzc(t);
                        add_row<TC, S, ADDM, ((p >> (kk + 1)) & 1) != 0>(E, Mr[kk]);
                    });
                } else {
                    // the group's states as in the interleaved form: column minima + E_L, running
                    // minimum compared with the threshold at the group's end
                    TC ev[V], rm;
                    static_for<16>([&](auto tc) {
                        constexpr int t = decltype(tc)::value, p = 16 * decltype(gc)::value + t, kk = t > 0 ? ctzc(t) : 0;
                        TC mc;
                        if constexpr (t == 0)
                            mc = m0;
                        else
                            mc = add_min_interleaved<TC, S, ADDM, ((p >> (kk + 1)) & 1) != 0>(E, Mr[kk], (TC)a.zero);
                        if constexpr (t % V == 0)
                            vload<TC>(ELp + i0 + p, ev);
                        const TC mp = mc + ev[t % V];
                        rm = t == 0 ? mp : emin(rm, mp);
                    });
                    hit = hit || rm <= uc;
                }
            });
        } else {
        // Fast path: per step one add per column, a min over the columns, one add of the step's
        // E_L and half a 3-input min into the running minimum; one compare per half body.
        static_for<BODY>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            constexpr bool fused = ILV && MINM == 3 && p > 0 && ctzc(p) < RC;
            TC mfused{};
            if constexpr (fused) {
                constexpr int kk = ctzc(p);
                mfused = add_min_interleaved<TC, S, ADDM, ((p >> (kk + 1)) & 1) != 0>(E, Mr[kk], (TC)a.zero);
            } else if constexpr (p > 0) {
                constexpr int kk = ctzc(p);
                if constexpr (kk < RC) {
                    add_row<TC, S, ADDM, ((p >> (kk + 1)) & 1) != 0>(E, Mr[kk]);
                } else {
                    Pmid = P;
                    high_flip(RC, (blk & 1) ? -1 : 1);
                }
            }
            if constexpr (p % V == 0)
                vload<TC>(ELp + i0 + p, elv);
            TC mcols;
            if constexpr (fused)
                mcols = mfused;
            else
                mcols = tree_min<TC, MINM, S>(E);
            const TC mp = mcols + elv[p % V];
            constexpr int HALF = BODY / 2, ph = p % HALF;
            TC &acc = p < HALF ? acc_lo : acc_hi;
            if constexpr (ph % 2 == 0)
                mprev = mp;
            else if constexpr (ph == 1)
                acc = emin(mprev, mp);
            else
                acc = emin3(acc, mprev, mp);
            if constexpr (p == HALF - 1)
                hit = acc_lo <= uc;  // before the row-RC flip moves uc
        });
        hit = hit || acc_hi <= uc;
        }
        if (hit) {
            // Slow path (rare): rebuild every step of this body from the body-end registers and
            // record each column at or below the threshold.  Step p differs from the last step
            // by the register rows and row RC whose Gray bits differ.
            const int iend = i0 + BODY - 1;
            const int gend = iend ^ (iend >> 1);
            const TC *rowRC = Mt + (size_t)RC * NB;
#pragma unroll 1
            for (int p = 0; p < BODY; ++p) {
                const int i = i0 + p;
                const int gp = i ^ (i >> 1);
                TC sr[RC];
#pragma unroll
                for (int r = 0; r < RC; ++r)
                    sr[r] = (TC)(((gp >> r) & 1) - ((gend >> r) & 1));
                const int dRC = ((gp >> RC) & 1) - ((gend >> RC) & 1);
                const TC sRC = (TC)dRC;
                const TP Pp = dRC == 0 ? P : Pmid;
                const TC elp = ELp[i];
                TC tp = to_col<T>(Treg + mu - Pp, clampC) - elp;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    TC mv[V];
                    vload<TC>(rowRC + (g * 32 + lane) * V, mv);
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const int q = g * V + e;
                        TC ev = E[q];
#pragma unroll
                        for (int r = 0; r < RC; ++r)
                            ev = ev + sr[r] * Mr[r][q];
                        stage[q * 32 + lane] = ev + sRC * mv[e];
                    }
                }
                const uint64_t cb = cbase | ((uint64_t)gp << B);
                const TP Ep = Pp + (TP)elp;
#pragma unroll 1
                for (int q = 0; q < S; ++q) {
                    const TC ev = stage[q * 32 + lane];
                    if (ev <= tp) {
                        const TP Et = (TP)ev + Ep;
                        const uint32_t j = (uint32_t)(((q / V) * 32 + lane) * V + (q % V));
                        record<T>(a, inst, Et, cb | j);
                        if (K1 && Et < Treg) {
                            Treg = Et;
                            tp = to_col<T>(Treg + mu - Pp, clampC) - elp;
                            Tr<T>::thr_min(st, Et);
                        }
                    }
                }
            }
            u = Treg + mu - P;
            uc = to_col<T>(u, clampC);
        }
        if (blk + 1 < nblk) {
            const int ip = (blk + 1) * BODY;
            const int kk = __ffs(ip) - 1;
            high_flip(kk, ((ip >> (kk + 1)) & 1) ? -1 : 1);
        }
    }

    if constexpr (Tr<T>::kFloat) {
        // the walk ends at step 2^L - 1 (g = 2^(L-1)): the last segment's drift
        reanchor((1 << L) - 1);
        double dmax = (double)dl;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            dmax = fmax(dmax, __shfl_xor_sync(kFull, dmax, o));
        if (lane == 0)
            atomicMax(&st->drift, (unsigned long long)__double_as_longlong(dmax));
    }
}

// ---- one work unit, packed 16-bit columns (small integer instances) ----------------------------
// Word w = (g * 32 + lane) * V + e of a thread holds column w in its low lane and column
// w + NB/2 in its high lane, each biased by 2^15.  One 32-bit add moves both columns; the tree of
// packed unsigned mins leaves the two lane minima in one word, and the step's test compares the
// smaller lane with threshold - E_L (E_L is stored minus the bias, so that difference is already
// in lane units).  Everything else follows scan_unit.
template <int S, int RC, bool K1, int ADDM, int MINM, int ILV = 0>
__device__ __forceinline__ void scan_unit_packed(const ScanArgs &a, const Inst &d, int inst, uint64_t unit,
                                                 int32_t &Treg, int lane, uint32_t *stage, int32_t *wsm)
{
    using T = i16p;
    using F = int32_t;
    constexpr int V = 4;
    constexpr int G = S / V;
    constexpr int LOGV = ilog2c(V);
    constexpr int LOGG = ilog2c(G);
    constexpr int B = LOGV + 5 + LOGG + 1;
    constexpr int NW = 1 << (B - 1);  // words per table row
    constexpr int BODY = 1 << (RC + 1);
    const int n = d.n, L = d.L, k = d.k, BL = B + L;
    InstState *st = a.state + inst;
    const F *W = unit_matrix<T>(d);

    F f0, cx;
    unit_fields<T>(W, n, k, BL, unit, lane, f0, cx);
    __syncwarp();
    if (lane >= B && lane < BL)
        wsm[lane - B] = f0;
    __syncwarp();

    // Column fields of the low lane; the high lane adds the field of suffix bit B - 1.
    F lin_t, lin_e[V], lin_g[G];
    column_fields<F, V, G>(f0, lane, lin_t, lin_e, lin_g);
    const F vtop = __shfl_sync(kFull, f0, B - 1);

    const int32_t *Es = (const int32_t *)d.Es;
    uint32_t E[S];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        int32_t lo[V], hi[V];
        vload<int32_t>(Es + (g * 32 + lane) * V, lo);
        vload<int32_t>(Es + NW + (g * 32 + lane) * V, hi);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const F lin = lin_e[e] + lin_t + lin_g[g];
            E[g * V + e] = (uint32_t)(lo[e] + lin + kLaneBias) + ((uint32_t)(hi[e] + lin + vtop + kLaneBias) << 16);
        }
    }

    // Register rows: packed M_r plus w_r on both lanes.
    const uint32_t *Mt = (const uint32_t *)d.M;
    uint32_t Mr[RC][S];
#pragma unroll
    for (int r = 0; r < RC; ++r) {
        const uint32_t wr2 = (uint32_t)__shfl_sync(kFull, f0, B + r) * 65537u;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            uint32_t mv[V];
            vload<uint32_t>(Mt + (size_t)r * NW + (g * 32 + lane) * V, mv);
#pragma unroll
            for (int e = 0; e < V; ++e)
                Mr[r][g * V + e] = mv[e] + wr2;
        }
    }

    {
        const int32_t tg = Tr<T>::thr_load(st);
        Treg = K1 ? min(Treg, tg) : tg;
    }
    const int32_t mu = (int32_t)a.margin;
    int32_t P = cx;
    int32_t u = Treg + mu - P;

    auto high_flip = [&](int kk, int sgn) {
        if (!QUBO_DCHECK(kk >= RC && kk < L, st, 4))
            kk = RC;
        const uint32_t *row = Mt + (size_t)kk * NW;
        const uint32_t sg = (uint32_t)sgn;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            uint32_t mv[V];
            vload<uint32_t>(row + (g * 32 + lane) * V, mv);
#pragma unroll
            for (int e = 0; e < V; ++e)
                E[g * V + e] = E[g * V + e] + sg * mv[e];
        }
        P = P + sgn * wsm[kk];
        u = Treg + mu - P;
    };

    const int32_t *ELp = (const int32_t *)d.EL;
    const int nblk = 1 << (L - RC - 1);
    const uint64_t cbase = unit << BL;
    if (!QUBO_DCHECK(L >= RC + 1 && L <= kMaxWalkBits && nblk * BODY == (1 << L), st, 5))
        return;

    const uint32_t *EL2p = (const uint32_t *)d.EL;
    // the Gray walk, with E_L added per step (as int32) or fused into the packed minima
    auto walk = [&](auto elf) {
        for (int blk = 0; blk < nblk; ++blk) {
            const int i0 = blk * BODY;
            int32_t elv[V];
            uint32_t el2v[V];
            bool hit = false;
            int32_t Pmid = P;
            int32_t acc_lo, acc_hi, mprev;  // as in scan_unit, in lane units
            uint32_t acc2_lo, acc2_hi, mprev2;  // fused: packed running minima of (lanes + E_L - elmin)
            static_for<BODY>([&](auto pc) {
                constexpr int p = decltype(pc)::value;
                constexpr bool fused = ILV && MINM == 3 && p > 0 && ctzc(p) < RC;
                uint32_t mfused = 0;
                if constexpr (fused) {
                    constexpr int kk = ctzc(p);
                    mfused = add_min_interleaved<uint32_t, S, ADDM, ((p >> (kk + 1)) & 1) != 0>(E, Mr[kk],
                                                                                               (uint32_t)a.zero);
                } else if constexpr (p > 0) {
                    constexpr int kk = ctzc(p);
                    if constexpr (kk < RC) {
                        constexpr bool neg = (p >> (kk + 1)) & 1;
                        if constexpr (ADDM == 2 || ADDM == 3) {
                            const uint32_t z = (uint32_t)a.zero;
    #pragma unroll
                            for (int q = 0; q < S; ++q) {
                                if (q % (ADDM == 2 ? 4 : 8) == 0)
                                    E[q] = neg ? (E[q] - Mr[kk][q]) + z : (E[q] + Mr[kk][q]) + z;
                                else
                                    E[q] = neg ? E[q] - Mr[kk][q] : E[q] + Mr[kk][q];
                            }
                        } else {
    #pragma unroll
                            for (int q = 0; q < S; ++q)
                                E[q] = neg ? E[q] - Mr[kk][q] : E[q] + Mr[kk][q];
                        }
                    } else {
                        Pmid = P;
                        high_flip(RC, (blk & 1) ? -1 : 1);
                    }
                }
                uint32_t mw;
                if constexpr (fused)
                    mw = mfused;
                else
                    mw = tree_min<uint32_t, MINM, S>(E);
                constexpr int HALF = BODY / 2, ph = p % HALF;
                if constexpr (decltype(elf)::value) {
                    // E_L - elmin added to both halves at once (no carry: proven on the host), packed
                    // running minimum; the halves are combined once per half body
                    if constexpr (p % V == 0)
                        vload<uint32_t>(EL2p + i0 + p, el2v);
                    const uint32_t sp = mw + el2v[p % V];
                    uint32_t &acc2 = p < HALF ? acc2_lo : acc2_hi;
                    if constexpr (ph % 2 == 0)
                        mprev2 = sp;
                    else if constexpr (ph == 1)
                        acc2 = __vminu2(mprev2, sp);
                    else
                        acc2 = __vimin3_u16x2(acc2, mprev2, sp);
                    if constexpr (p == HALF - 1)
                        hit = min((int32_t)(acc2_lo & 0xffffu), (int32_t)(acc2_lo >> 16)) <= u - d.elmin + kLaneBias;
                } else {
                    if constexpr (p % V == 0)
                        vload<int32_t>(ELp + i0 + p, elv);
                    const int32_t mp = min((int32_t)(mw & 0xffffu), (int32_t)(mw >> 16)) + elv[p % V];
                    int32_t &acc = p < HALF ? acc_lo : acc_hi;
                    if constexpr (ph % 2 == 0)
                        mprev = mp;
                    else if constexpr (ph == 1)
                        acc = min(mprev, mp);
                    else
                        acc = __vimin3_s32(acc, mprev, mp);
                    if constexpr (p == HALF - 1)
                        hit = acc_lo <= u;
                }
            });
            if constexpr (decltype(elf)::value)
                hit = hit || min((int32_t)(acc2_hi & 0xffffu), (int32_t)(acc2_hi >> 16)) <= u - d.elmin + kLaneBias;
            else
                hit = hit || acc_hi <= u;
            if (hit) {
                const int iend = i0 + BODY - 1;
                const int gend = iend ^ (iend >> 1);
                const uint32_t *rowRC = Mt + (size_t)RC * NW;
    #pragma unroll 1
                for (int p = 0; p < BODY; ++p) {
                    const int i = i0 + p;
                    const int gp = i ^ (i >> 1);
                    uint32_t sr[RC];
    #pragma unroll
                    for (int r = 0; r < RC; ++r)
                        sr[r] = (uint32_t)(((gp >> r) & 1) - ((gend >> r) & 1));
                    const int dRC = ((gp >> RC) & 1) - ((gend >> RC) & 1);
                    const uint32_t sRC = (uint32_t)dRC;
                    const int32_t Pp = dRC == 0 ? P : Pmid;
                    const int32_t el = decltype(elf)::value ? (int32_t)(EL2p[i] & 0xffffu) + d.elmin : ELp[i] + kLaneBias;
                    int32_t tp = Treg + mu - Pp - el;
    #pragma unroll
                    for (int g = 0; g < G; ++g) {
                        uint32_t mv[V];
                        vload<uint32_t>(rowRC + (g * 32 + lane) * V, mv);
    #pragma unroll
                        for (int e = 0; e < V; ++e) {
                            const int q = g * V + e;
                            uint32_t ev = E[q];
    #pragma unroll
                            for (int r = 0; r < RC; ++r)
                                ev = ev + sr[r] * Mr[r][q];
                            stage[q * 32 + lane] = ev + sRC * mv[e];
                        }
                    }
                    const uint64_t cb = cbase | ((uint64_t)gp << B);
                    const int32_t Ep = Pp + el;
    #pragma unroll 1
                    for (int q = 0; q < 2 * S; ++q) {
                        const uint32_t word = stage[(q >> 1) * 32 + lane];
                        const int32_t col = (int32_t)((q & 1) ? (word >> 16) : (word & 0xffffu)) - kLaneBias;
                        if (col <= tp) {
                            const int32_t Et = col + Ep;
                            const int qw = q >> 1;
                            const uint32_t j = (uint32_t)(((qw / V) * 32 + lane) * V + (qw % V)) + ((q & 1) ? NW : 0);
                            record<T>(a, inst, Et, cb | j);
                            if (K1 && Et < Treg) {
                                Treg = Et;
                                tp = Treg + mu - Pp - el;
                                Tr<T>::thr_min(st, Et);
                            }
                        }
                    }
                }
                u = Treg + mu - P;
            }
            if (blk + 1 < nblk) {
                const int ip = (blk + 1) * BODY;
                const int kk = __ffs(ip) - 1;
                high_flip(kk, ((ip >> (kk + 1)) & 1) ? -1 : 1);
            }
        }



    };
    if constexpr (ILV == 2) {
        // fused-only kernel: the host runs it only on plans whose E_L is fused
        if (QUBO_DCHECK(d.el_fused, st, 8))
            walk(std::true_type{});
    } else {
        if (d.el_fused)
            walk(std::true_type{});
        else
            walk(std::false_type{});
    }
}

// Persistent work loop: a warp claims work units from the queue, kChunk at a time (the next claim
// is made before the current units are scanned, hiding the atomic), and counts the states it
// scanned locally, flushing the count when the instance changes and at exit.  Same-address
// atomics on the queue and on a state counter cap the unit rate near 1.5e8 units/s on GB300,
// which matters for kernels whose units take microseconds.
template <class T, unsigned long long kChunk, class UnitFn>
__device__ __forceinline__ void persistent_units(const ScanArgs &a, int lane, typename Tr<T>::TP &Treg,
                                                 UnitFn &&unit_fn)
{
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
        for (unsigned long long item = base; item < end; ++item) {
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
            if (!QUBO_DCHECK(inst >= 0 && inst < a.n_inst && item >= a.item_base[inst] && item < a.item_base[inst + 1],
                             a.state + (inst >= 0 && inst < a.n_inst ? inst : 0), 6))
                continue;
            const Inst d = a.inst[inst];
            if (!QUBO_DCHECK(d.small || item - a.item_base[inst] < d.units, a.state + inst, 7))
                continue;
            if (d.small) {
                small_unit<T>(a, d, inst, lane);  // counts its own states
            } else {
                unit_fn(d, inst, d.unit_begin + (item - a.item_base[inst]));
                done += 1ull << (d.B + d.L);
            }
        }
    }
    if (lane == 0 && done)
        atomicAdd(&a.state[cur].scanned, done);
}

template <class T, int S, int RC, bool K1, int MINB, int ADDM, int MINM, int ILV = 0>
__global__ void __launch_bounds__(kScanThreads, MINB) scan_kernel(const ScanArgs a)
{
    using TC = typename Tr<T>::TC;
    using TP = typename Tr<T>::TP;
    constexpr int kAncWarps = Tr<T>::kFloat ? kScanThreads / 32 : 1;  // float scans: re-anchoring base
    __shared__ TC stage_all[kScanThreads / 32][S * 32];
    __shared__ __align__(16) TC anc_all[kAncWarps][Tr<T>::kFloat ? S * 32 : 1];
    __shared__ TP wsm_all[kScanThreads / 32][kMaxWalkBits];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    TC *stage = stage_all[warp];
    TC *anc = anc_all[Tr<T>::kFloat ? warp : 0];
    TP *wsm = wsm_all[warp];
    TP Treg = (TP)0;
    // units take 0.1-30 ms here: one per claim keeps the end of a launch balanced
    persistent_units<T, 1>(a, lane, Treg, [&](const Inst &d, int inst, uint64_t unit) {
        if constexpr (Tr<T>::kPack == 2)
            scan_unit_packed<S, RC, K1, ADDM, MINM, ILV>(a, d, inst, unit, Treg, lane, stage, wsm);
        else
            scan_unit<T, S, RC, K1, ADDM, MINM, ILV>(a, d, inst, unit, Treg, lane, stage, wsm, anc);
    });
}

}  // namespace qubo
