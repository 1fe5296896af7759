// Scan and table-build kernels instantiated for small integer instances: two biased 16-bit
// columns per 32-bit word.
#include "scan_impl.cuh"

namespace qubo {

namespace {
template <int VAR, bool K1>
constexpr auto kernel_of()
{
    constexpr int kS = packed_words(VAR);  // words per thread, two columns each
    static_assert(ilog2c(64 * kS) == packed_suffix_bits(VAR), "suffix bits must match the column layout");
    return scan_kernel<i16p, kS, kPackedRegRows[VAR], K1, kPackedMinBlocks[VAR], kPackedAddMode[VAR], 3>;
}

template <bool K1>
auto pick(int variant)
{
    switch (variant) {
    case 1: return kernel_of<1, K1>();
    case 2: return kernel_of<2, K1>();
    case 3: return kernel_of<3, K1>();
    case 4: return kernel_of<4, K1>();
    case 5: return kernel_of<5, K1>();
    case 6: return kernel_of<6, K1>();
    case 7: return kernel_of<7, K1>();
    default: return kernel_of<0, K1>();
    }
}
}  // namespace

template <>
cudaError_t launch_tables_t<i16p>(const Inst *d_inst, int n_inst, int max_entries, cudaStream_t s)
{
    if (n_inst <= 0)
        return cudaSuccess;
    const int threads = 256;
    int bx = (max_entries + threads - 1) / threads;
    if (bx < 1)
        bx = 1;
    if (bx > 4096)
        bx = 4096;
    tables_kernel<i16p><<<dim3(bx, n_inst), threads, 0, s>>>(d_inst);
    return cudaGetLastError();
}

template <>
cudaError_t launch_scan_t<i16p>(const ScanArgs &a, int blocks, int variant, cudaStream_t s)
{
    auto k = a.k1 ? pick<true>(variant) : pick<false>(variant);
    k<<<blocks, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <>
int scan_blocks_per_sm_t<i16p>(bool k1, int variant)
{
    int nb = 0;
    auto k = k1 ? pick<true>(variant) : pick<false>(variant);
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kScanThreads, 0);
    return e == cudaSuccess ? nb : -1;
}

}  // namespace qubo
