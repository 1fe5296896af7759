// Scan and table-build kernels instantiated for the int32_t accumulator.
#include "scan_impl.cuh"

namespace qubo {

namespace {
template <int VAR, bool K1>
constexpr auto kernel_of()
{
    constexpr int kS = cols_per_thread(sizeof(int32_t), VAR);
    static_assert(ilog2c(32 * kS) == suffix_bits(sizeof(int32_t), VAR), "suffix bits must match the column layout");
    return scan_kernel<int32_t, kS, kVariantRegRows[VAR], K1, kVariantMinBlocks[VAR], kVariantAddMode[VAR],
                       kVariantMinInputs[VAR], step_form(VAR, false)>;
}

template <bool K1, int... V>
auto pick_of(int variant, std::integer_sequence<int, V...>)
{
    using Fn = decltype(kernel_of<0, K1>());
    constexpr Fn table[] = {kernel_of<V, K1>()...};
    return table[(variant >= 0 && variant < (int)sizeof...(V)) ? variant : 0];
}

template <bool K1>
auto pick(int variant)
{
    return pick_of<K1>(variant, std::make_integer_sequence<int, kScanVariants>{});
}
}  // namespace

template <>
cudaError_t launch_tables_t<int32_t>(const Inst *d_inst, int n_inst, int max_entries, cudaStream_t s)
{
    if (n_inst <= 0)
        return cudaSuccess;
    const int threads = 256;
    int bx = (max_entries + threads - 1) / threads;
    if (bx < 1)
        bx = 1;
    if (bx > 4096)
        bx = 4096;
    tables_kernel<int32_t><<<dim3(bx, n_inst), threads, 0, s>>>(d_inst);
    return cudaGetLastError();
}

template <>
cudaError_t launch_scan_t<int32_t>(const ScanArgs &a, int blocks, int variant, cudaStream_t s)
{
    auto k = a.k1 ? pick<true>(variant) : pick<false>(variant);
    k<<<blocks, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <>
int scan_blocks_per_sm_t<int32_t>(bool k1, int variant)
{
    int nb = 0;
    auto k = k1 ? pick<true>(variant) : pick<false>(variant);
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kScanThreads, 0);
    return e == cudaSuccess ? nb : -1;
}

}  // namespace qubo
