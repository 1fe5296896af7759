// Host-side planning of a scan, shared by the planner (plan.cu) and the driver (api.cu): the
// prepared instance (folded matrix, bound, plan of the current run) and the functions that choose
// the accumulator, the split of the code into suffix, walked and fixed bits, the kernel variant,
// and the initial threshold.
#pragma once
#include <chrono>
#include <cstdint>
#include <vector>

#include "../../include/qubo.h"
#include "internal.h"

namespace qubo {
namespace host {

constexpr int kTargetUnitsLog2 = 15;   // aim for >= 2^15 work units per scan
constexpr double kDefaultMargin = 1e-3; // FP32 scans: candidate margin above the running minimum
constexpr int kDefaultMaxWalkBits = 12;
// Integers in FP32 lanes: 2^14-step walks (n=50: 0.7% faster than 2^12) when the plan stays exact
// in FP32 lanes, else the default length is tried.
constexpr int kI32FMaxWalkBits = 14;
// FP32 scans re-anchor every 2^kFloatAnchorBits walk steps (and at every unit start): 2^10 Gray
// steps keep the measured drift (2.4e-4 on the n=44 SK instance) well inside the budget of the
// default 1e-3 candidate margin; the drift guard shortens the period when it does not.  The walk
// itself can then be longer (fewer unit set-ups): 2^14 steps measured 5% faster than 2^10.
constexpr int kFloatAnchorBits = 10;
constexpr int kFloatMaxWalkBits = 14;
// The factored sparse scan reads the whole E_L table once per unit: 2^14 entries (64 KB) stay in
// L1 and amortise the unit set-up (measured against 2^11..2^16).
constexpr int kZMaxWalkBits = 14;

inline double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Plan-dependent magnitudes of the FP32 scan's rounding bound (fp32_error_bound), cached per plan.
struct Fp32BoundTerms {
    bool valid = false;
    int n = 0, B = 0, L = 0, rc = 0;
    double margin = 0.0;
    double Cc = 0.0, CP = 0.0, Ecol0 = 0.0, EP0 = 0.0, rest = 0.0;
};

// One instance prepared on the host and the plan of its current run.
struct HostInst {
    int n = 0;
    bool is_float = false;
    Acc acc = ACC_I32;
    std::vector<int64_t> Ui;  // folded upper-triangular (integer Q)
    std::vector<double> Uf;   // folded upper-triangular (float Q), FP64
    double beta = 0.0;        // sum |U_ij|
    // plan of the current run
    int variant = 0;  // compiled scan variant (fixes the columns per thread)
    int B = 0, L = 0, k = 0, small = 0;
    int fix_bits = 0;
    uint64_t fix_value = 0;
    uint64_t unit_begin = 0, units = 0, sub_base = 0, sub_count = 0;
    uint64_t items = 0, states = 0;
    double thr0 = 0.0;  // initial threshold (a bound on the K-th lowest energy of the range)
    int32_t clampC = 0; // ACC_I32F: threshold clamp
    int32_t col_lo = 0, col_hi = 0;  // ACC_I16P: proven range of every column value
    int32_t el_fused = 0, elmin = 0; // ACC_I16P: E_L added to the packed minima (i16p_fuse_el)
    int Z = 0;                  // ACC_I32Z / ACC_F32Z: walked rows without suffix couplings
    std::vector<uint8_t> perm;  // ACC_I32Z / ACC_F32Z: caller's variable at each scan position
    bool no_factored = false;   // the factored FP32 scan used up its margin: plan the dense one
    int anchor_bits = kFloatAnchorBits;  // ACC_F32: re-anchoring period (log2 of walk steps)
    mutable Fp32BoundTerms fp32_terms;   // ACC_F32: cached magnitudes of the rounding bound
};

// The plan part of a HostInst (what plan() and the exactness checks set), saved and restored
// without copying the matrices.
struct PlanFields {
    Acc acc;
    int variant, B, L, k, small, fix_bits;
    uint64_t fix_value, unit_begin, units, sub_base, sub_count, items, states;
    int32_t clampC, col_lo, col_hi, el_fused, elmin;
};

// Plans, saved and restored without the matrices.
PlanFields plan_fields(const HostInst &h);
void set_plan_fields(HostInst &h, const PlanFields &p);

// Input: dtype checks; fold Q into U, bound it (beta) and pick the accumulator (Sec. 1, 2.1).
bool dtype_ok(qubo_dtype dt);
bool dtype_float(qubo_dtype dt);
int prepare(const void *Q, int n, qubo_dtype dt, uint32_t flags, HostInst &h);

// Accumulators and compiled kernel variants.
int acc_bytes(Acc a);
bool acc_float(Acc a);
bool acc_factored(Acc a);
int acc_suffix_bits(Acc a, int variant);
int acc_cols_per_thread(Acc a, int variant);
int reg_rows_of(Acc a, int variant);
int variant_reg_rows(const HostInst &h);
int scan_variant(Acc acc = ACC_I32);
int pick_variant(Acc acc, int requested);

// The split n = k + L + B of a run (Sec. 3.3) and the accumulator it runs in: the exactness
// checks of the packed 16-bit and FP32-lane scans, the factored scan's variable order.
int plan(HostInst &h, int fix_bits, uint64_t fix_value, int split_k, int walk_bits);
bool i32f_exact(const HostInst &h, int32_t *clampC);
bool i32f_allowed();
void col_range_exact(const HostInst &h, int64_t &lo, int64_t &hi);
int64_t walked_energy_max(const HostInst &h);
bool i16p_exact(HostInst &h);
void i16p_fuse_el(HostInst &h);
bool i16p_allowed();
int zero_rows_search(HostInst &h);
bool i32z_allowed();
bool plan_factored(HostInst &h, Acc acc, int fix_bits, uint64_t fix_value, int split_k, int walk_bits);
int plan_run(HostInst &h, int fix_bits, uint64_t fix_value, int split_k, int walk_bits, int variant_req,
             uint32_t flags, double margin = kDefaultMargin);

// Initial threshold: a bound on the K-th lowest energy of the run's sub-cube from greedy descents.
double threshold_bound(const HostInst &h, int K, int restarts = 24);

// Dense FP32 scan: worst-case rounding error of a state's decision value at a re-anchoring period
// of 2^anchor_bits walk steps, and the longest period whose bound alone guarantees the candidates
// (2 bound <= margin; -1 if none).  0 / -1 for other accumulators.
const Fp32BoundTerms &fp32_bound_terms(const HostInst &h, double margin);
double fp32_error_bound(const HostInst &h, int anchor_bits, double margin);
int fp32_rigorous_anchor_bits(const HostInst &h, double margin);

}  // namespace host
}  // namespace qubo
