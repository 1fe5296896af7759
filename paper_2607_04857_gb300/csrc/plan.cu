// Host-side planning (Sec. 3.3 split, accumulator choice, exactness checks, the factored scan's
// variable order, the initial threshold): pure host code, no device work.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <random>
#include <unordered_set>
#include <utility>
#include <vector>

#include "host.h"

namespace qubo {
namespace host {

// ------------------------------------------------------------------------------------------------
// Host-side preparation of one instance.
// ------------------------------------------------------------------------------------------------



PlanFields plan_fields(const HostInst &h)
{
    return {h.acc,   h.variant,  h.B,         h.L,     h.k,      h.small,  h.fix_bits, h.fix_value, h.unit_begin,
            h.units, h.sub_base, h.sub_count, h.items, h.states, h.clampC, h.col_lo,   h.col_hi,    h.el_fused,
            h.elmin};
}

void set_plan_fields(HostInst &h, const PlanFields &p)
{
    h.acc = p.acc;
    h.variant = p.variant;
    h.B = p.B;
    h.L = p.L;
    h.k = p.k;
    h.small = p.small;
    h.fix_bits = p.fix_bits;
    h.fix_value = p.fix_value;
    h.unit_begin = p.unit_begin;
    h.units = p.units;
    h.sub_base = p.sub_base;
    h.sub_count = p.sub_count;
    h.items = p.items;
    h.states = p.states;
    h.clampC = p.clampC;
    h.col_lo = p.col_lo;
    h.col_hi = p.col_hi;
    h.el_fused = p.el_fused;
    h.elmin = p.elmin;
}

bool dtype_ok(qubo_dtype dt) { return dt == QUBO_I16 || dt == QUBO_I32 || dt == QUBO_F32 || dt == QUBO_F64; }
bool dtype_float(qubo_dtype dt) { return dt == QUBO_F32 || dt == QUBO_F64; }

// Fold Q into U (U_ii = Q_ii, U_ij = Q_ij + Q_ji for i < j) and choose the accumulator.
int prepare(const void *Q, int n, qubo_dtype dt, uint32_t flags, HostInst &h)
{
    if (!Q || n < 1 || n > 64 || !dtype_ok(dt))
        return QUBO_ERR_ARG;
    h = HostInst();
    h.n = n;
    h.is_float = dtype_float(dt);
    auto qi = [&](int i, int j) -> int64_t {
        const size_t o = (size_t)i * n + j;
        return dt == QUBO_I16 ? (int64_t)((const int16_t *)Q)[o] : (int64_t)((const int32_t *)Q)[o];
    };
    auto qf = [&](int i, int j) -> double {
        const size_t o = (size_t)i * n + j;
        return dt == QUBO_F32 ? (double)((const float *)Q)[o] : ((const double *)Q)[o];
    };
    if (h.is_float) {
        h.Uf.assign((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = i; j < n; ++j) {
                const double v = i == j ? qf(i, i) : qf(i, j) + qf(j, i);
                if (!std::isfinite(v))
                    return QUBO_ERR_ARG;
                h.Uf[(size_t)i * n + j] = v;
                h.beta += std::fabs(v);
            }
        h.acc = (flags & QUBO_FLAG_PLAIN) ? ACC_F64 : ACC_F32;
    } else {
        h.Ui.assign((size_t)n * n, 0);
        int64_t beta = 0;
        for (int i = 0; i < n; ++i)
            for (int j = i; j < n; ++j) {
                const int64_t v = i == j ? qi(i, i) : qi(i, j) + qi(j, i);
                h.Ui[(size_t)i * n + j] = v;
                beta += v < 0 ? -v : v;
            }
        h.beta = (double)beta;
        // Every partial sum the scan forms (table entries, running energies, thresholds minus a
        // prefix energy) is bounded by 2*beta in magnitude: int32 is exact when beta < 2^30.
        if (beta >= (1ll << 62))
            return QUBO_ERR_OVERFLOW;
        h.acc = ((flags & QUBO_FLAG_PLAIN) || beta >= (1ll << 30)) ? ACC_I64 : ACC_I32;
    }
    return QUBO_OK;
}

int acc_bytes(Acc a) { return (a == ACC_I64 || a == ACC_F64) ? 8 : 4; }
bool acc_float(Acc a) { return a == ACC_F32 || a == ACC_F64 || a == ACC_F32Z; }
bool acc_factored(Acc a) { return a == ACC_I32Z || a == ACC_F32Z; }

// Suffix bits (log2 of the columns of one work unit) of an accumulator and kernel variant.
int acc_suffix_bits(Acc a, int variant)
{
    if (acc_factored(a))
        return zscan_suffix_bits(variant);
    return a == ACC_I16P ? packed_suffix_bits(variant) : suffix_bits(acc_bytes(a), variant);
}

// Columns held by one thread (two per word in the packed scan).
int acc_cols_per_thread(Acc a, int variant)
{
    if (acc_factored(a))
        return kZCols[(variant >= 0 && variant < kZVariants) ? variant : 0];
    return a == ACC_I16P ? 2 * packed_words(variant) : cols_per_thread(acc_bytes(a), variant);
}

// Walked rows a compiled variant keeps in registers (a walk needs at least one more bit).
int reg_rows_of(Acc a, int variant)
{
    const int v = variant >= 0 && variant < kScanVariants ? variant : 0;
    if (acc_factored(a))
        return 2;  // the factored scan needs at least 3 walked rows
    return a == ACC_I16P ? kPackedRegRows[v] : kVariantRegRows[acc_bytes(a) == 4 ? v : 0];
}

// Walked rows the run's kernel variant keeps in registers (a walk needs at least one more bit).
int variant_reg_rows(const HostInst &h)
{
    return reg_rows_of(h.acc, h.variant);
}

int plan(HostInst &h, int fix_bits, uint64_t fix_value, int split_k, int walk_bits)
{
    const int n = h.n;
    if (fix_bits < 0 || fix_bits > n || (fix_bits < 64 && fix_bits > 0 && (fix_value >> fix_bits) != 0))
        return QUBO_ERR_ARG;
    if (fix_bits == 0)
        fix_value = 0;
    h.fix_bits = fix_bits;
    h.fix_value = fix_value;
    const int free_bits = n - fix_bits;
    if (free_bits > 63)
        return QUBO_ERR_ARG;
    h.states = 1ull << free_bits;
    h.B = acc_suffix_bits(h.acc, h.variant);
    const int rc = variant_reg_rows(h);
    if (free_bits < h.B + rc + 1) {
        h.small = 1;
        h.L = h.k = 0;
        h.sub_base = fix_bits ? (fix_value << free_bits) : 0;
        h.sub_count = h.states;
        h.units = 0;
        h.items = 1;
        return QUBO_OK;
    }
    h.small = 0;
    int L;
    if (split_k > 0)
        L = n - h.B - split_k;
    else if (walk_bits > 0)
        L = walk_bits;
    else
        L = std::max(rc + 1, std::min(h.acc == ACC_F32          ? kFloatMaxWalkBits
                                      : h.acc == ACC_I32F       ? kI32FMaxWalkBits
                                      : acc_factored(h.acc) ? kZMaxWalkBits
                                                            : kDefaultMaxWalkBits,
                                      free_bits - h.B - kTargetUnitsLog2));
    const int k = n - h.B - L;
    if (L < rc + 1 || L > kMaxWalkBits || k < fix_bits || k > 63)
        return QUBO_ERR_ARG;
    h.L = L;
    h.k = k;
    h.units = 1ull << (k - fix_bits);
    h.unit_begin = fix_bits ? (fix_value << (k - fix_bits)) : 0;
    h.items = h.units;
    return QUBO_OK;
}

// Compiled scan variant: QUBO_SCAN_VARIANT overrides the measured default of the accumulator.
int scan_variant(Acc acc)
{
    const char *v = std::getenv("QUBO_SCAN_VARIANT");
    if (v) {
        const int x = std::atoi(v);
        if (x >= 0 && x < kScanVariants)
            return x;
    }
    switch (acc) {
    case ACC_F32: return kDefaultVariantF32;
    case ACC_I32F: return kDefaultVariantI32F;
    case ACC_I16P: return kDefaultVariantI16P;
    default: return kDefaultVariantI32;
    }
}

// The variant a run uses: the caller's (tuned) choice, else the accumulator's default.
int pick_variant(Acc acc, int requested) { return requested >= 0 ? requested : scan_variant(acc); }

// The default variant keeps five walked rows in registers and needs walks of at least six bits.
// When the walk is shorter (the caller's walk_bits, split_k leaving fewer walked bits, or a
// (sub)cube too small for 2^kTargetUnitsLog2 units walking four unrolled bodies each) and the
// caller named no variant, the run takes the measured best variant with fewer register rows and
// the same columns per thread, so the suffix split is unchanged; failing all, the one with the
// fewest rows.  A small instance's units are then short bodies: a unit that runs its unrolled
// body only once or twice pays for the straight-line code's instruction fetch, and a 64-step
// body made every launch of a small solve about 0.2 ms longer than an 8-step one.
int fit_variant(const HostInst &h, int fix_bits, int split_k, int walk_bits, int variant_req, int variant)
{
    if (variant_req >= 0 || std::getenv("QUBO_SCAN_VARIANT"))
        return variant;
    const int B = acc_suffix_bits(h.acc, variant);
    // the planner's own walk should give a unit at least four unrolled bodies (two more bits)
    const int slack = split_k > 0 || walk_bits > 0 ? 0 : 2;
    const int L = split_k > 0 ? h.n - B - split_k
                              : (walk_bits > 0 ? walk_bits : h.n - fix_bits - B - kTargetUnitsLog2 - slack);
    if (L >= reg_rows_of(h.acc, variant) + 1)
        return variant;
    static constexpr int kShorter4[] = {8, 3};       // 4 register rows (interleaved), 3
    static constexpr int kShorterP[] = {13, 8, 11};  // packed: 4, 3, 2 register rows (interleaved)
    const int *cand = h.acc == ACC_I16P ? kShorterP : kShorter4;
    const int nc = h.acc == ACC_I16P ? 3 : 2;
    int last = variant;
    for (int c = 0; c < nc; ++c) {
        if (acc_suffix_bits(h.acc, cand[c]) != B)
            continue;
        if (L >= reg_rows_of(h.acc, cand[c]) + 1)
            return cand[c];
        last = cand[c];
    }
    // no candidate fits the walk the planner aims at: the fewest rows, if the caller's walk allows
    const int Lmax = split_k > 0 ? h.n - B - split_k : (walk_bits > 0 ? walk_bits : h.n - fix_bits - B);
    return Lmax >= reg_rows_of(h.acc, last) + 1 ? last : variant;
}

// Integer energies can be scanned exactly in FP32 lanes when every value held in an FP32 lane stays
// below 2^24 in magnitude: the column values, the stored tables (E_s, the walked rows M_r with the
// register rows' fixed couplings folded in, E_L) and the clamped per-step threshold.  The unit
// fields, c(x_f) and the prefix part are int32.  The per-step threshold is clamped to +-C with
// C = max|column| + max|E_L| + 1, which leaves every decision unchanged, so |threshold - E_L| <=
// C + max|E_L| must stay below 2^24.  Quick accept: with nf = B + L non-fixed variables, every
// column value is a signed subset sum of the entries touching a non-fixed variable (S_nf bounds
// it) and every E_L value one of the entries among walked variables (S_ww).  Otherwise the
// column range is computed exactly per suffix pattern, E_L by enumeration, and every table row
// by the sum of |U| over its entries.
bool i32f_exact(const HostInst &h, int32_t *clampC)
{
    if (h.small || h.is_float)
        return false;
    const int n = h.n, nf = h.B + h.L, B = h.B, rc = variant_reg_rows(h);
    constexpr double kLimit = 16777216.0;
    double s_nf = 0.0, s_ww = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            const double a = std::fabs((double)h.Ui[(size_t)i * n + j]);
            if (i < nf)
                s_nf += a;
            if (i >= h.B && j < nf)
                s_ww += a;
        }
    if (s_nf + 2.0 * s_ww + 2.0 < kLimit) {
        *clampC = (int32_t)(s_nf + s_ww + 1.0);
        return true;
    }
    auto U = [&](int i, int j) { return i < j ? h.Ui[(size_t)i * n + j] : h.Ui[(size_t)j * n + i]; };
    for (int r = B; r < nf; ++r) {  // table row r: M_r[j] (+ w_r for a register row)
        double row = 0.0;
        for (int b = 0; b < B; ++b)
            row += std::fabs((double)U(r, b));
        if (r < B + rc)
            for (int f = nf; f < n; ++f)
                row += std::fabs((double)U(r, f));
        if (row >= kLimit)
            return false;
    }
    int64_t lo, hi;
    col_range_exact(h, lo, hi);
    const double el = (double)walked_energy_max(h);
    const double C = (double)std::max(-lo, hi) + el + 1.0;
    if (C + el + 1.0 >= kLimit)
        return false;
    *clampC = (int32_t)C;
    return true;
}

bool i32f_allowed()
{
    const char *v = std::getenv("QUBO_NO_I32F");
    return !(v && v[0] == '1');
}

// Range of every column value the plan's packed or FP32-lane kernel holds.  For suffix pattern j
// a column holds
//   E_s(j) + sum_{i outside the suffix} x_i c_i(j) + sum_{r < RC} x_r w_r,
// with c_i(j) = sum_{b in j} U_bi, w_r = sum_{f fixed} x_f U_rf (the couplings of the register
// rows folded into their table rows).  Its range over all outside bits is bounded by taking every
// c_i(j) and every U_rf at its sign's extreme, computed exactly for each j (O(2^B n)).
void col_range_exact(const HostInst &h, int64_t &lo, int64_t &hi)
{
    const int n = h.n, B = h.B, rc = variant_reg_rows(h), nf = h.B + h.L;
    auto U = [&](int i, int j) { return i < j ? h.Ui[(size_t)i * n + j] : h.Ui[(size_t)j * n + i]; };
    int64_t wpos = 0, wneg = 0;
    for (int r = B; r < B + rc; ++r)
        for (int f = nf; f < n; ++f) {
            const int64_t u = U(r, f);
            (u > 0 ? wpos : wneg) += u;
        }
    // c[j][i] for every variable i, built from j without its lowest bit
    const size_t NB = 1ull << B;
    std::vector<int64_t> c(NB * n, 0), es(NB, 0);
    lo = 0;
    hi = 0;
    for (size_t j = 1; j < NB; ++j) {
        const int b = __builtin_ctzll(j);
        const size_t jp = j & (j - 1);
        const int64_t *cp = &c[jp * n];
        int64_t *cj = &c[j * n];
        for (int i = 0; i < n; ++i)
            cj[i] = cp[i] + (i == b ? 0 : U(b, i));
        es[j] = es[jp] + U(b, b) + cp[b];
        int64_t up = es[j], dn = es[j];
        for (int i = B; i < n; ++i)
            (cj[i] > 0 ? up : dn) += cj[i];
        lo = std::min(lo, dn);
        hi = std::max(hi, up);
    }
    lo += wneg;
    hi += wpos;
}

// Largest |E_L(g)| over the 2^L walked patterns (the energy of the walked variables alone),
// enumerated in Gray order with a running field per variable.
int64_t walked_energy_max(const HostInst &h)
{
    const int n = h.n, B = h.B, L = h.L;
    auto U = [&](int i, int j) { return i < j ? h.Ui[(size_t)i * n + j] : h.Ui[(size_t)j * n + i]; };
    std::vector<int64_t> field(L, 0);  // sum of U over the set walked variables other than r
    std::vector<int> x(L, 0);
    int64_t e = 0, m = 0;
    for (uint64_t i = 1; i < (1ull << L); ++i) {
        const int r = __builtin_ctzll(i);
        const int s = x[r] ? -1 : 1;
        e += s * (U(B + r, B + r) + field[r]);
        x[r] ^= 1;
        for (int t = 0; t < L; ++t)
            if (t != r)
                field[t] += s * U(B + r, B + t);
        m = std::max(m, e < 0 ? -e : e);
    }
    return m;
}

// Integer energies can be scanned as packed 16-bit lanes when every column value the plan's
// kernel holds lies in [-32768, 32767].  The scan's threshold arithmetic (threshold - prefix -
// E_L + 2^15 in int32) asks beta < 2^29 as well.
bool i16p_exact(HostInst &h)
{
    if (h.small || h.is_float || h.beta >= 536870912.0)
        return false;
    const int n = h.n, B = h.B, rc = variant_reg_rows(h), nf = h.B + h.L;
    auto U = [&](int i, int j) { return i < j ? h.Ui[(size_t)i * n + j] : h.Ui[(size_t)j * n + i]; };
    // quick accept: the sum of |U| over every entry a column can contain
    int64_t crude = 0;
    for (int r = B; r < B + rc; ++r)
        for (int f = nf; f < n; ++f)
            crude += std::llabs(U(r, f));
    for (int b = 0; b < B; ++b)
        for (int i = b; i < n; ++i)
            crude += std::llabs(U(b, i));
    if (crude <= 32767) {
        h.col_lo = (int32_t)-crude;
        h.col_hi = (int32_t)crude;
        return true;
    }
    int64_t lo, hi;
    col_range_exact(h, lo, hi);
    if (lo < -32768 || hi > 32767)
        return false;
    h.col_lo = (int32_t)lo;
    h.col_hi = (int32_t)hi;
    return true;
}

// Packed scan of a proven plan: whether E_L can be added to the packed column minima of a step
// as one 32-bit add, E_L - elmin in both halves.  A half holds a column value plus 2^15, at most
// col_hi + 2^15; the sum stays at most 65535 (no carry into the other half) when
// col_hi + (max E_L - elmin) <= 32767.  Quick accept with elmin = the sum of the negative entries
// among the walked variables (a lower bound of every E_L, and E_L - elmin is at most S_ww, the sum
// of their |U|), else the exact E_L range by enumeration.  QUBO_NO_PACKED_FUSED=1 keeps the
// separate lane combine and add.
void i16p_fuse_el(HostInst &h)
{
    h.el_fused = 0;
    h.elmin = 0;
    const char *v = std::getenv("QUBO_NO_PACKED_FUSED");
    if (h.acc != ACC_I16P || h.small || (v && v[0] == '1'))
        return;
    const int n = h.n, B = h.B, L = h.L;
    auto U = [&](int i, int j) { return i < j ? h.Ui[(size_t)i * n + j] : h.Ui[(size_t)j * n + i]; };
    int64_t sww = 0, neg = 0;
    for (int r = 0; r < L; ++r)
        for (int t = r; t < L; ++t) {
            const int64_t w = U(B + r, B + t);
            sww += std::llabs(w);
            neg += w < 0 ? w : 0;
        }
    if ((int64_t)h.col_hi + sww <= 32767) {
        h.el_fused = 1;
        h.elmin = (int32_t)neg;
        return;
    }
    std::vector<int64_t> field(L, 0);
    std::vector<int> x(L, 0);
    int64_t e = 0, emin = 0, emax = 0;  // E_L of the empty pattern is 0
    for (uint64_t i = 1; i < (1ull << L); ++i) {
        const int r = __builtin_ctzll(i);
        const int sg = x[r] ? -1 : 1;
        e += sg * (U(B + r, B + r) + field[r]);
        x[r] ^= 1;
        for (int t = 0; t < L; ++t)
            if (t != r)
                field[t] += sg * U(B + r, B + t);
        emin = std::min(emin, e);
        emax = std::max(emax, e);
    }
    if ((int64_t)h.col_hi + (emax - emin) <= 32767) {
        h.el_fused = 1;
        h.elmin = (int32_t)emin;
    }
}

// Factored scan of sparse instances: choose up to kZMaxRows walked variables with no coupling
// to any of the B suffix variables (any order of the variables is allowed, Sec. 2.4), and a
// scan order: suffix, those zero rows, the other walked rows, the unit's fixed bits, then the
// sub-cube's fixed top bits in place.  Greedy: candidates by ascending degree join the zero rows
// while at least B variables remain that neither they nor the zero rows touch.  Returns Z and
// fills h.perm (h.B, h.L from the plan).
int zero_rows_search(HostInst &h)
{
    const int n = h.n, nf = n - h.fix_bits, B = h.B, L = h.L;
    if (h.small || nf < B + L)
        return 0;
    auto adj = [&](int a, int b) {
        const size_t o = (size_t)std::min(a, b) * n + std::max(a, b);
        return a != b && (h.is_float ? h.Uf[o] != 0.0 : h.Ui[o] != 0);
    };
    std::vector<int> deg(n, 0);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            deg[a] += adj(a, b);
    std::vector<int> order(nf);
    for (int v = 0; v < nf; ++v)
        order[v] = v;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return deg[a] < deg[b]; });
    std::vector<char> inZ(n, 0), touched(n, 0);
    std::vector<int> zrows;
    const int zmax = std::min(kZMaxRows, L);
    auto pool_size = [&](int extra) {
        int c = 0;
        for (int u = 0; u < nf; ++u)
            if (!inZ[u] && u != extra && !touched[u] && !adj(u, extra))
                ++c;
        return c;
    };
    for (int v : order) {
        if ((int)zrows.size() >= zmax)
            break;
        if (pool_size(v) < B)
            continue;
        inZ[v] = 1;
        zrows.push_back(v);
        for (int u = 0; u < n; ++u)
            if (adj(u, v))
                touched[u] = 1;
    }
    const int Z = (int)zrows.size();
    if (Z == 0)
        return 0;
    std::vector<int> suf, rest;
    for (int v : order) {
        if (inZ[v])
            continue;
        if ((int)suf.size() < B && !touched[v])
            suf.push_back(v);
        else
            rest.push_back(v);
    }
    if ((int)suf.size() < B)
        return 0;
    h.perm.assign(n, 0);
    int pos = 0;
    for (int v : suf)
        h.perm[pos++] = (uint8_t)v;
    for (int v : zrows)
        h.perm[pos++] = (uint8_t)v;
    for (int v : rest)
        h.perm[pos++] = (uint8_t)v;
    for (int v = nf; v < n; ++v)
        h.perm[pos++] = (uint8_t)v;
    return Z;
}

bool i32z_allowed()
{
    const char *v = std::getenv("QUBO_NO_I32Z");
    return !(v && v[0] == '1');
}

bool i16p_allowed()
{
    const char *v = std::getenv("QUBO_NO_I16P");
    return !(v && v[0] == '1');
}

// Accumulator, kernel variant and plan of one run.  Integer instances scan in packed 16-bit lanes
// or else in FP32 lanes when the plan keeps every value exact (and the plain form was not asked
// for), else in int32.
// Plan the factored scan (accumulator acc, ACC_I32Z or ACC_F32Z) when at least 3 walked rows can be
// factored out; true when planned.
bool plan_factored(HostInst &h, Acc acc, int fix_bits, uint64_t fix_value, int split_k, int walk_bits)
{
    // QUBO_ZSCAN_VARIANT pins the factored scan's column count (variant index)
    const char *zenv = std::getenv("QUBO_ZSCAN_VARIANT");
    const int z0 = zenv ? std::max(0, std::min(kZVariants - 1, std::atoi(zenv))) : 0;
    const int z1 = zenv ? z0 + 1 : kZVariants - 1;  // variant 3 is chosen below, not searched
    for (int zv = z0; zv < z1; ++zv) {
        h.acc = acc;
        h.variant = zv;
        if (plan(h, fix_bits, fix_value, split_k, walk_bits) != QUBO_OK || (h.Z = zero_rows_search(h)) < 3)
            continue;
        if (h.L - h.Z > kZMaxBlocksLog2) {
            // too many blocks for the per-warp table: a shorter walk, if the plan is ours
            if (split_k > 0 || walk_bits > 0 || plan(h, fix_bits, fix_value, 0, h.Z + kZMaxBlocksLog2) != QUBO_OK ||
                (h.Z = zero_rows_search(h)) < 3 || h.L - h.Z > kZMaxBlocksLog2)
                continue;
        }
        // every walked row factored: one block per unit, the kernel without column registers
        if (!zenv && h.variant == 0 && h.Z == h.L && h.Z >= 7)
            h.variant = 3;
        return true;
    }
    h.Z = 0;
    h.perm.clear();
    return false;
}

int plan_run(HostInst &h, int fix_bits, uint64_t fix_value, int split_k, int walk_bits, int variant_req,
             uint32_t flags, double margin)
{
    if ((h.acc == ACC_F32 || h.acc == ACC_F32Z) && !(flags & QUBO_FLAG_PLAIN)) {
        // the rounding bound is derived for the dense FP32 scan only
        if (!(flags & QUBO_FLAG_RIGOROUS) && i32z_allowed() && !h.no_factored &&
            plan_factored(h, ACC_F32Z, fix_bits, fix_value, split_k, walk_bits))
            return QUBO_OK;
        h.acc = ACC_F32;
        if (flags & QUBO_FLAG_RIGOROUS) {
            h.variant = pick_variant(h.acc, variant_req);
            h.variant = fit_variant(h, fix_bits, split_k, walk_bits, variant_req, h.variant);
            int st = plan(h, fix_bits, fix_value, split_k, walk_bits);
            if (st)
                return st;
            if (h.small)
                return QUBO_OK;
            const int a = fp32_rigorous_anchor_bits(h, margin);
            if (a >= 0) {
                h.anchor_bits = std::min(h.anchor_bits, a);
                return QUBO_OK;
            }
            h.acc = ACC_F64;  // no period is short enough: the FP64 scan
        }
    }
    if ((h.acc == ACC_I32 || h.acc == ACC_I32F || h.acc == ACC_I16P || h.acc == ACC_I32Z) &&
        !(flags & (QUBO_FLAG_PLAIN | QUBO_FLAG_INT32))) {
        Acc chosen = ACC_I32;
        // sparse instances: at least 3 walked rows factored out (8x fewer column updates)
        if (i32z_allowed() && plan_factored(h, ACC_I32Z, fix_bits, fix_value, split_k, walk_bits))
            return QUBO_OK;
        if (i16p_allowed()) {
            h.acc = ACC_I16P;
            h.variant = pick_variant(h.acc, variant_req);
            h.variant = fit_variant(h, fix_bits, split_k, walk_bits, variant_req, h.variant);
            if (plan(h, fix_bits, fix_value, split_k, walk_bits) == QUBO_OK && i16p_exact(h)) {
                chosen = ACC_I16P;
                i16p_fuse_el(h);
                h.variant = packed_variant_for(h.variant, h.el_fused);
            }
        }
        if (chosen == ACC_I32 && i32f_allowed()) {
            h.acc = ACC_I32F;
            h.variant = pick_variant(h.acc, variant_req);
            h.variant = fit_variant(h, fix_bits, split_k, walk_bits, variant_req, h.variant);
            if (plan(h, fix_bits, fix_value, split_k, walk_bits) == QUBO_OK && i32f_exact(h, &h.clampC))
                chosen = ACC_I32F;
            else if (split_k <= 0 && walk_bits <= 0 && h.L > kDefaultMaxWalkBits &&
                     plan(h, fix_bits, fix_value, 0, kDefaultMaxWalkBits) == QUBO_OK && i32f_exact(h, &h.clampC)) {
                chosen = ACC_I32F;  // a shorter walk keeps fewer values in the lanes
                walk_bits = kDefaultMaxWalkBits;
            }
        }
        h.acc = chosen;
    }
    h.variant = acc_bytes(h.acc) == 4 ? pick_variant(h.acc, variant_req) : 0;
    if (acc_bytes(h.acc) == 4)
        h.variant = fit_variant(h, fix_bits, split_k, walk_bits, variant_req, h.variant);
    if (h.acc == ACC_I16P)  // the fused-E_L-only build of the variant when E_L is fused
        h.variant = packed_variant_for(h.variant, h.el_fused);
    return plan(h, fix_bits, fix_value, split_k, walk_bits);
}

// Upper bound on the K-th lowest energy (with multiplicity) of the run's sub-cube: the K-th lowest
// energy among distinct states met by greedy one-flip descents from seeded random starts.  Any
// K distinct states of the range bound it from above; with fewer than K found, beta does.
double threshold_bound(const HostInst &h, int K, int restarts)
{
    const int n = h.n, fb = h.fix_bits, free_bits = n - fb;
    const uint64_t base = fb ? (h.fix_value << free_bits) : 0;
    const uint64_t fmask = free_bits >= 64 ? ~0ull : ((1ull << free_bits) - 1);
    auto U = [&](int i, int j) -> double {
        if (i > j)
            std::swap(i, j);
        return h.is_float ? h.Uf[(size_t)i * n + j] : (double)h.Ui[(size_t)i * n + j];
    };
    auto energy = [&](uint64_t x) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            if (!((x >> i) & 1))
                continue;
            acc += U(i, i);
            for (int j = i + 1; j < n; ++j)
                if ((x >> j) & 1)
                    acc += U(i, j);
        }
        return acc;
    };
    std::vector<std::pair<double, uint64_t>> seen;
    std::unordered_set<uint64_t> codes;
    double best1 = std::numeric_limits<double>::infinity();  // K = 1: the lowest state met
    uint64_t best1_x = 0;
    auto offer = [&](double E, uint64_t x) {
        if (K <= 1) {
            if (E < best1) {
                best1 = E;
                best1_x = x;
            }
            return;
        }
        if (codes.insert(x).second)
            seen.emplace_back(E, x);
    };
    std::mt19937_64 rng(0x9e3779b97f4a7c15ull ^ h.fix_value ^ ((uint64_t)n << 56));
    std::vector<double> hf(n);
    for (int r = 0; r < restarts; ++r) {
        uint64_t x = base | (r == 0 ? 0 : (rng() & fmask));
        double E = energy(x);
        for (int j = 0; j < n; ++j) {
            double a = 0.0;
            for (int i = 0; i < n; ++i)
                if (i != j && ((x >> i) & 1))
                    a += U(i, j);
            hf[j] = a;
        }
        for (int it = 0; it < 4 * n + 8; ++it) {
            int best = -1;
            double bd = 0.0;
            for (int v = 0; v < free_bits; ++v) {
                const double d = ((x >> v) & 1) ? -(U(v, v) + hf[v]) : (U(v, v) + hf[v]);
                if (d < bd) {
                    bd = d;
                    best = v;
                }
            }
            if (best < 0)
                break;
            const bool up = !((x >> best) & 1);
            x ^= 1ull << best;
            E += bd;
            for (int j = 0; j < n; ++j)
                if (j != best)
                    hf[j] += up ? U(best, j) : -U(best, j);
        }
        // the local minimum and all its one-flip neighbours
        offer(E, x);
        for (int v = 0; v < free_bits; ++v)
            offer(E + (((x >> v) & 1) ? -(U(v, v) + hf[v]) : (U(v, v) + hf[v])), x ^ (1ull << v));
    }
    if (K <= 1 && restarts > 0)
        seen.emplace_back(best1, best1_x);
    K = std::max(K, 1);
    if ((int)seen.size() < K)
        return h.beta;
    std::nth_element(seen.begin(), seen.begin() + (K - 1), seen.end());
    double t = seen[K - 1].first;
    if (h.is_float) {
        // the incremental energies above differ from the exact ones by rounding only
        t = energy(seen[K - 1].second);
        t += 1e-9 * (1.0 + h.beta);
    } else {
        t = std::nearbyint(t);
    }
    return std::min(t, h.beta);
}

}  // namespace host
}  // namespace qubo

namespace qubo {
namespace host {

// ---- rigorous rounding bound of the dense FP32 scan ----------------------------------------------
// The FP32 scan (Sec. 6.2, mixed precision with periodic correction) decides per state whether
// it reaches the threshold: column (E_s(j) + lin(j) + rows of the set walked bits, updated by one
// FP32 add or FMA per Gray step) + E_L(g) <= T + margin - P.  Every FP32 operation rounds to
// nearest, so its error is at most u = 2^-24 times the magnitude of its result; the tables are
// summed in FP64 and rounded once.  With magnitudes computed from the folded matrix for the
// run's split (suffix S = bits [0, B), walked bits [B, B + L), fixed bits F = the rest):
//   Cc    = max_j |E_s(j)| + sum_{i outside S} |c_i(j)| + sum_{r < RC} rF(r), with
//           c_i(j) = sum_{b in j} U_bi: bounds every column value (the register rows carry their
//           fixed couplings w_r) and every partial sum that forms one;
//   CL    = max_g |E_L(g)|;  bF = sum |U| within F;  rF(v) = sum_{f in F} |U_vf|;
//   rS(r) = sum_{b in S} |U_rb|;  CabsF = sum_{b in S} rF(b);  CP = bF + sum_{r >= RC} rF(r);
//   CT    = beta (1 + 2^-20) + margin (any threshold is a state's energy, rounded);
//   e64   = n^2 2^-52 beta (error of one FP64-summed table entry before its FP32 rounding),
//   u64   = 2^-52 (a generous FP64 rounding unit, for the per-unit fields summed in FP64),
// the error of the decision value of any state is at most
//   Ecol0 = 2u Cc + e64 + (B + 3) u CabsF + k u64 CabsF            base column: E_s + lin
//         + sum_{r < RC} [2u (rS(r) + rF(r)) + (u + k u64) rF(r)   register rows M_r + w_r
//                         + e64]
//         + sum_{r >= RC} [u rS(r) + e64]                         table rows
//         + (L - RC) u Cc                                         rows added at a re-anchoring
//   Ecol  = Ecol0 + ((1 + u)^t - 1) (Cc + Ecol0)                    t = 2^a steps since the anchor
//   EP0   = (u + (k + 8) u64) bF + sum_{r >= RC} (u + k u64) rF(r)  c(x_f) and the couplings w_r,
//         + (L - RC) u CP                                         each rounded once; re-anchoring
//   EP    = EP0 + ((1 + u)^(t / 2^(RC+1) + 1) - 1) (CP + EP0)        one add per row-RC-or-higher flip
//   Edec  = Ecol + (RC + 1) u (Cc + Ecol) + EP + (u CL + e64) + u (Cc + CL)
//         + u CT + u (CT + CP) + u (CT + CP + CL)                  slow-path rebuild, E_L, threshold
// (the fields and c(x_f) are FP64 sums of k terms, plus a five-level warp sum for c(x_f), each
// rounded to FP32 once; lin(j) adds at most B of the rounded fields in FP32, B + 2 additions).
// A state x of the answer has E(x) <= E(y) for the state y whose
// computed energy set the threshold, so it is recorded whenever 2 Edec <= margin; its FP64
// rescoring then decides.  The bound is a worst case over every state of the run.
// The plan-dependent magnitudes of the bound, computed once per (B, L, RC, margin) and kept in h.
const Fp32BoundTerms &fp32_bound_terms(const HostInst &h, double margin)
{
    Fp32BoundTerms &m = h.fp32_terms;
    const int rc = variant_reg_rows(h);
    if (m.valid && m.B == h.B && m.L == h.L && m.rc == rc && m.n == h.n && m.margin == margin)
        return m;
    const int n = h.n, B = h.B, L = h.L, k = h.k, nf = B + L;
    const double u = std::ldexp(1.0, -24);
    auto U = [&](int i, int j) { return i <= j ? h.Uf[(size_t)i * n + j] : h.Uf[(size_t)j * n + i]; };
    double beta = 0.0, bF = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            beta += std::fabs(U(i, j));
            if (i >= nf)
                bF += std::fabs(U(i, j));
        }
    std::vector<double> rF(nf, 0.0), rS(nf, 0.0);
    for (int v = 0; v < nf; ++v) {
        for (int f = nf; f < n; ++f)
            rF[v] += std::fabs(U(v, f));
        for (int b = 0; b < B; ++b)
            if (b != v)
                rS[v] += std::fabs(U(v, b));
    }
    double CabsF = 0.0;
    for (int b = 0; b < B; ++b)
        CabsF += rF[b];
    double CP = bF;
    for (int r = rc; r < L; ++r)
        CP += rF[B + r];
    // Cc: E_s(j) and c_i(j) by adding the lowest set bit of j to j without it
    const size_t NB = 1ull << B;
    std::vector<double> Es(NB, 0.0), absc(NB, 0.0), c(NB, 0.0);
    for (size_t j = 1; j < NB; ++j) {
        const int b0 = __builtin_ctzll(j);
        const size_t jp = j & (j - 1);
        double e = Es[jp] + U(b0, b0);
        for (int b = b0 + 1; b < B; ++b)
            if ((jp >> b) & 1)
                e += U(b0, b);
        Es[j] = e;
    }
    for (int i = B; i < n; ++i) {
        for (size_t j = 1; j < NB; ++j) {
            const int b0 = __builtin_ctzll(j);
            c[j] = c[j & (j - 1)] + U(b0, i);
            absc[j] += std::fabs(c[j]);
        }
    }
    double Cc = 0.0;
    for (size_t j = 0; j < NB; ++j)
        Cc = std::max(Cc, std::fabs(Es[j]) + absc[j]);
    for (int r = 0; r < rc; ++r)  // the register rows carry their fixed couplings w_r
        Cc += rF[B + r];
    // CL: E_L over every walked pattern in Gray order with a field vector
    double CL = 0.0;
    {
        std::vector<double> field(L, 0.0);
        std::vector<int> x(L, 0);
        double e = 0.0;
        for (uint64_t i = 1; i < (1ull << L); ++i) {
            const int r = __builtin_ctzll(i);
            const double s = x[r] ? -1.0 : 1.0;
            e += s * (U(B + r, B + r) + field[r]);
            x[r] ^= 1;
            for (int t = 0; t < L; ++t)
                if (t != r)
                    field[t] += s * U(B + r, B + t);
            CL = std::max(CL, std::fabs(e));
        }
        // the walk's own rounding is far below the slack of the bound; widen by it anyway
        CL *= 1.0 + std::ldexp(1.0, -30);
    }
    const double CT = beta * (1.0 + std::ldexp(1.0, -20)) + margin;
    const double e64 = (double)n * n * std::ldexp(1.0, -52) * beta;
    const double u64 = std::ldexp(1.0, -52);
    double Ecol0 = 2 * u * Cc + e64 + (B + 3) * u * CabsF + k * u64 * CabsF + (L - rc) * u * Cc;
    for (int r = 0; r < L; ++r)
        Ecol0 += r < rc ? 2 * u * (rS[B + r] + rF[B + r]) + (u + k * u64) * rF[B + r] + e64 : u * rS[B + r] + e64;
    double EP0 = u * bF + (k + 8) * u64 * bF + (L - rc) * u * CP;
    for (int r = rc; r < L; ++r)
        EP0 += u * rF[B + r] + k * u64 * rF[B + r];
    m.valid = true;
    m.n = n;
    m.B = B;
    m.L = L;
    m.rc = rc;
    m.margin = margin;
    m.Cc = Cc;
    m.CP = CP;
    m.Ecol0 = Ecol0;
    m.EP0 = EP0;
    m.rest = (u * CL + e64) + u * (Cc + CL) + u * CT + u * (CT + CP) + u * (CT + CP + CL);
    return m;
}

double fp32_error_bound(const HostInst &h, int anchor_bits, double margin)
{
    if (h.acc != ACC_F32 || h.small || h.Uf.empty())
        return 0.0;
    const Fp32BoundTerms &m = fp32_bound_terms(h, margin);
    const double u = std::ldexp(1.0, -24);
    const int a = std::min(std::max(anchor_bits, m.rc + 1), m.L);
    const double Ecol = m.Ecol0 + std::expm1(std::ldexp(1.0, a) * std::log1p(u)) * (m.Cc + m.Ecol0);
    const double tP = std::ldexp(1.0, std::max(0, a - m.rc - 1)) + 1.0;
    const double EP = m.EP0 + std::expm1(tP * std::log1p(u)) * (m.CP + m.EP0);
    return Ecol + (m.rc + 1) * u * (m.Cc + Ecol) + EP + m.rest;
}

// Longest re-anchoring period (log2 of walk steps, from one unrolled body up to the whole walk)
// whose rounding bound alone guarantees the FP32 scan's candidates: 2 fp32_error_bound <= margin.
// -1 when even one body is too long.
int fp32_rigorous_anchor_bits(const HostInst &h, double margin)
{
    if (h.acc != ACC_F32 || h.small || h.Uf.empty())
        return -1;
    const int rc = variant_reg_rows(h);
    for (int a = h.L; a >= rc + 1; --a)
        if (2.0 * fp32_error_bound(h, a, margin) <= margin)
            return a;
    return -1;
}

}  // namespace host
}  // namespace qubo
