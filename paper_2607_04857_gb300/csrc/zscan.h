// Constants of the factored scan of sparse instances (scan_sparse.cu), shared with the host driver.
#pragma once

namespace qubo {

// Factored scan of sparse instances: columns per thread of each variant, the
// most zero rows (walked rows without suffix couplings) and the most column-walk blocks.
// Variant 3 is the one-block-per-unit kernel (every walked row factored, Z = L >= 7).
constexpr int kZVariants = 4;
constexpr int kZCols[kZVariants] = {64, 32, 16, 64};
constexpr int kZMaxRows = 14;
constexpr int kZMaxBlocksLog2 = 9;
constexpr int zscan_suffix_bits(int variant)
{
    return kZCols[(variant >= 0 && variant < kZVariants) ? variant : 0] == 64 ? 11
           : kZCols[(variant >= 0 && variant < kZVariants) ? variant : 0] == 32 ? 10 : 9;
}

}  // namespace qubo
