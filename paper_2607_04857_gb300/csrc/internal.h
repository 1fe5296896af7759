// Internal declarations shared by the host driver (api.cu) and the kernels of libqubo.so.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "zscan.h"

namespace qubo {

// ACC_I32F: integer energies scanned exactly in FP32 lanes (partial sums below 2^24).
// ACC_I16P: integer energies whose column values fit 16 bits, two columns per 32-bit word.
// ACC_I32Z / ACC_F32Z: int32 / FP32 energies of sparse instances: walked rows without couplings
// to the suffix variables are factored out of the column walk (scan_sparse.cu).
enum Acc : int32_t {
    ACC_I32 = 1,
    ACC_I64 = 2,
    ACC_F32 = 3,
    ACC_F64 = 4,
    ACC_I32F = 5,
    ACC_I16P = 6,
    ACC_I32Z = 7,
    ACC_F32Z = 8
};

// The shortest walk the allocation-free plan and the autotuner's walk sweep consider is
// kRegRows + 1 bits.  Each compiled variant keeps RC walked rows (2 to 5) in registers and
// unrolls its inner loop over 2^(RC+1) Gray steps, so that every register-row flip has a
// compile-time sign; a plan needs walk_bits >= RC + 1, checked per variant.
constexpr int kRegRows = 4;
// Compiled scan variants of the 4-byte accumulators: columns per thread S, register rows,
// minimum resident blocks per SM, how the adds are issued (0: compiler's choice, 4: FP32 adds as
// paired f32x2 operations, two columns per instruction, 5, 6, 7: a half, a quarter or three
// quarters of them paired; the paired modes do not apply to integer columns; 2, 3: in the
// interleaved form, one integer column in four / in eight updated by a 3-input add on the ALU
// pipe), 2- or 3-input mins, and the step form: 0, all adds first, then the min tree; 1, the adds
// interleaved with the first level of the min tree (each triple of columns reduced as soon as its
// adds are issued); 2 (integers in FP32 lanes and FP32; form 1 for int32), the grouped form: groups of 16 steps skip the min tree while a per-thread lower bound of the column
// minimum, moved by the steps' smallest column deltas, proves that no column can reach the
// threshold.  The 8-byte
// accumulators compile one variant: S = 16 with variant 0's register rows, blocks and min inputs.
constexpr int kScanVariants = 24;
constexpr int kVariantCols[kScanVariants] = {32, 16, 16, 16, 16, 16, 32, 16, 16, 16, 16, 16,
                                             16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16};
constexpr int kVariantRegRows[kScanVariants] = {3, 4, 4, 3, 4, 4, 3, 4, 4, 4, 4, 3, 3, 3, 3, 3, 5, 5, 5, 5, 5, 4, 5, 5};
constexpr int kVariantMinBlocks[kScanVariants] = {2, 3, 3, 3, 3, 3, 2, 3, 3, 3, 3, 4, 4, 4, 3, 3, 2, 2, 2, 2, 3, 3, 3, 3};
constexpr int kVariantAddMode[kScanVariants] = {0, 6, 7, 0, 0, 4, 4, 5, 6, 5, 4, 6, 4, 0, 4, 4, 6, 0, 3, 2, 4, 4, 0, 6};
constexpr int kVariantMinInputs[kScanVariants] = {3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3,
                                                  3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3};
constexpr int kVariantInterleave[kScanVariants] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2};
// The step form a kernel of an accumulator compiles for a variant: the grouped form only for FP32
// column adds (integers in FP32 lanes, FP32).
constexpr int step_form(int variant, bool fp32_columns)
{
    return kVariantInterleave[variant] == 2 && !fp32_columns ? 1 : kVariantInterleave[variant];
}
// Whether a plan's scan kernel runs the grouped form.
constexpr bool grouped_form(Acc acc, int variant)
{
    return (acc == ACC_I32F || acc == ACC_F32) && variant >= 0 && variant < kScanVariants &&
           kVariantInterleave[variant] == 2;
}
// Default variant per 4-byte accumulator (measured on GB300; see the profiles).
constexpr int kDefaultVariantI32 = 16;
constexpr int kDefaultVariantF32 = 22;
constexpr int kDefaultVariantI32F = 20;
constexpr int kDefaultVariantI16P = 14;
// Compiled variants of the packed 16-bit scan: S words per thread (2 S columns), register rows,
// minimum resident blocks per SM, and how the adds are issued (0: compiler's choice; 2 and 3: one
// add in four or in eight as a 3-input add with a runtime 0, which the ALU pipe executes, so
// that the ALU and FMA pipes share the adds).  All use 3-input mins.
// Variants 8-14 and 16-19 interleave the adds and the first min level as the 4-byte variants do
// (18 and 19 with one add in eight / in four on the ALU pipe, the others with plain adds), and
// carry both forms of the E_L step (added to the packed minimum, or after the lane combine),
// chosen per instance at run time.  Variants 20-23 are 14, 13, 8 and 11 compiled with the fused
// form alone (interleave 2), half the code, for plans whose E_L is fused.
constexpr int kPackedWords[kScanVariants] = {16, 16, 16, 16, 16, 32, 32, 16, 16, 16, 16, 16,
                                             32, 16, 16, 16, 32, 16, 16, 16, 16, 16, 16, 16};
constexpr int kPackedRegRows[kScanVariants] = {3, 3, 3, 3, 3, 2, 2, 2, 3, 3, 4, 2, 2, 4, 5, 4, 3, 5, 5, 5, 5, 4, 3, 2};
constexpr int kPackedMinBlocks[kScanVariants] = {3, 3, 3, 4, 4, 2, 2, 4, 3, 4, 3, 4, 2, 2, 2, 2, 2, 1, 2, 2, 2, 2, 3, 4};
constexpr int kPackedAddMode[kScanVariants] = {0, 3, 2, 0, 3, 0, 3, 3, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 3, 2, 0, 0, 0, 0};
constexpr int kPackedInterleave[kScanVariants] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 0, 1, 1, 1, 1, 2, 2, 2, 2};
// The packed variant a plan runs: the fused-only twin of a variant when its E_L is fused and the
// twin exists, else the variant that carries both forms.
constexpr int packed_variant_for(int variant, bool el_fused)
{
    constexpr int kBoth[4] = {14, 13, 8, 11};
    int both = variant;
    for (int t = 0; t < 4; ++t)
        if (variant == 20 + t)
            both = kBoth[t];
    if (el_fused)
        for (int t = 0; t < 4; ++t)
            if (both == kBoth[t])
                return 20 + t;
    return both;
}
constexpr bool packed_fused_only(int variant) { return variant >= 0 && variant < kScanVariants && kPackedInterleave[variant] == 2; }
// Threads per block of the scan kernel (4 warps; every warp owns one work unit at a time).
constexpr int kScanThreads = 128;
// Longest Gray walk inside one work unit (also the FP32 re-anchoring period).
constexpr int kMaxWalkBits = 16;
// Batched instances carry their index in the top bits of a candidate key.
constexpr int kInstShift = 40;
constexpr int kMaxBatchedN = 40;

// Candidate record.  `key` is the state code (single instance) or (instance << 40) | code
// (batched).  `e` is an int64 energy or the bit pattern of a double energy.
struct Rec {
    uint64_t key;
    int64_t e;
};

// Immutable per-instance description of one scan (device copy lives in the arena).
struct Inst {
    int32_t n;          // variables
    int32_t B;          // suffix bits (columns)
    int32_t L;          // walked prefix bits
    int32_t k;          // fixed bits per unit (n = B + L + k on the tabled path)
    int32_t small;      // 1: no split, every state evaluated directly
    int32_t clampC;     // ACC_I32F: clamp of the per-step threshold (max |column| + max |E_L| + 1)
    uint64_t unit_begin;  // first unit (value of the fixed bits) of this run
    uint64_t units;       // units in this run
    uint64_t sub_base;    // small path: first code
    uint64_t sub_count;   // small path: number of codes
    const void *W;        // symmetric coupling matrix in the accumulator type, n*n
    const double *W64;    // symmetric coupling matrix in FP64 (float instances), n*n
    const double *U64;    // folded upper-triangular matrix in FP64 (float rescore), n*n
    void *Es;             // 2^B suffix energies
    void *M;              // L x 2^B interaction rows (M_int restricted to the walked rows)
    void *EL;             // 2^L walked-prefix energies in Gray-walk order
    int64_t thr0;         // initial threshold (int64 value or double bits)
    int32_t Z;            // ACC_I32Z: walked rows 0..Z-1 have no coupling to a suffix variable
    int32_t anchor;       // float scans: re-anchor every 2^anchor walk steps (0 or >= L: at the end only)
    const uint8_t *perm;  // ACC_I32Z: variable of the caller's order at each scan position
    int32_t el_fused;     // ACC_I16P: E_L stored as (E_L - elmin) in both 16-bit halves and added to the
                          // packed column minima without a carry (the host proves the sums fit 16 bits)
    int32_t elmin;        // ACC_I16P with el_fused: a lower bound of every E_L value
    float geps;           // ACC_F32, grouped form: rounding allowance of a group's column updates
};

// Mutable per-instance state, updated with atomics.
struct InstState {
    unsigned long long thr;      // threshold in the accumulator's ordered encoding
    unsigned long long gmin;     // smallest recorded energy, same encoding
    unsigned long long scanned;  // states evaluated
    unsigned long long nrec;     // candidates offered
    unsigned long long dropped;  // candidates not stored (buffer full)
    unsigned long long drift;    // float: max re-anchoring drift (bits of a non-negative double)
    unsigned long long err;      // float: max |E_scan - E64| (bits of a non-negative double)
    unsigned long long dbg;      // QUBO_DEBUG builds: first failed device check (site number), else 0
};

// Device checks of a QUBO_DEBUG build (libqubo_debug.so): an index outside its table, a walked
// row outside the walk, a work item outside its instance.  The first failure of an instance
// records its site number in InstState::dbg and the access is skipped or clamped; the host then
// returns QUBO_ERR_INTERNAL.  Nothing traps.  Release builds compile the checks away.
#ifdef QUBO_DEBUG
#define QUBO_DCHECK(cond, st, site) ((cond) ? true : (atomicCAS(&(st)->dbg, 0ull, (unsigned long long)(site)), false))
#else
#define QUBO_DCHECK(cond, st, site) true
#endif

// Per-instance result written by the extraction kernel.
struct ResOut {
    int64_t min_i;
    double min_f;
    unsigned long long n_ties;
    unsigned long long n_written;
    unsigned long long n_near;
    int32_t nk;
    int32_t has;
};

struct ScanArgs {
    const Inst *inst;
    InstState *state;
    const uint64_t *item_base;   // n_inst + 1 prefix sums of the per-instance item counts
    int32_t n_inst;
    int32_t k1;                  // K <= 1: thresholds tighten as lower states are found
    uint64_t total_items;
    unsigned long long *queue;   // dynamic work counter (zeroed before launch)
    Rec *rec;
    unsigned long long rec_cap;
    unsigned long long *nrec;    // total candidates offered
    const volatile int *abort_flag;
    double margin;               // float scans: candidate margin above the threshold
    int32_t zero;                // the constant 0, passed at run time (packed 3-input-add variants)
    int32_t pad;
};

// Columns per thread (S) of the scan kernel for an accumulator of `bytes` bytes and a variant;
// a work unit covers 32*S columns, so the suffix has log2(32*S) bits.
constexpr int cols_per_thread(int bytes, int variant = 0)
{
    return bytes == 4 ? kVariantCols[(variant >= 0 && variant < kScanVariants) ? variant : 0] : 16;
}
constexpr int suffix_bits(int bytes, int variant = 0)
{
    return cols_per_thread(bytes, variant) == 32 ? 10 : 9;
}
// The packed 16-bit scan holds two columns in each of its S words: log2(64 S) suffix bits.
constexpr int packed_words(int variant)
{
    return kPackedWords[(variant >= 0 && variant < kScanVariants) ? variant : 0];
}
constexpr int packed_suffix_bits(int variant) { return packed_words(variant) == 32 ? 11 : 10; }

struct i32f;  // tag of the integer-in-FP32 accumulator (scan_impl.cuh)
struct i16p;  // tag of the packed 16-bit accumulator (scan_impl.cuh)

// ---- launchers (scan_*.cu, one translation unit per accumulator type) -------------------------
template <class T>
cudaError_t launch_tables_t(const Inst *d_inst, int n_inst, int max_entries, cudaStream_t s);
template <class T>
cudaError_t launch_scan_t(const ScanArgs &a, int blocks, int variant, cudaStream_t s);
template <class T>
int scan_blocks_per_sm_t(bool k1, int variant);

cudaError_t launch_zscan(const ScanArgs &a, int blocks, int variant, bool is_float, cudaStream_t s);
int zscan_blocks_per_sm(bool k1, int variant, bool is_float);

// ---- dispatch and finalize (finalize.cu) -----------------------------------------------------
cudaError_t launch_tables(Acc acc, const Inst *d_inst, int n_inst, int max_entries, cudaStream_t s);
cudaError_t launch_scan(Acc acc, const ScanArgs &a, int blocks, int variant, cudaStream_t s);
int scan_blocks_per_sm(Acc acc, bool k1, int variant);
cudaError_t launch_rescore(const Inst *d_inst, InstState *d_state, Rec *rec, const unsigned long long *d_nrec,
                           unsigned long long cap, bool batched, unsigned long long max_count, cudaStream_t s);
cudaError_t launch_sort(Rec *rec, const unsigned long long *d_nrec, unsigned long long cap, unsigned long long max_pow2,
                        bool batched, bool is_float, cudaStream_t s, int *launches);
cudaError_t launch_extract(const Inst *d_inst, const Rec *rec, const unsigned long long *d_nrec, unsigned long long cap,
                           int n_inst, bool batched, bool is_float, int topk, unsigned long long states_cap,
                           ResOut *res, uint64_t *ties, uint64_t *topk_codes, int64_t *topk_e,
                           unsigned long long *d_starts, cudaStream_t s);

// ---- host state shared by the entry points (api.cu) --------------------------------------------
// True while qubo_abort() is in force (until qubo_abort_clear()).
bool abort_requested();

}  // namespace qubo
