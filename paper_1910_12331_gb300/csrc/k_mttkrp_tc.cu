// k_mttkrp_tc.cu -- all-mode MTTKRP on tcgen05 tensor cores (placeholder until
// the tensor-core kernel lands).
#include "tc.hpp"

namespace cpgn {

size_t split_cache_bytes(const cp_desc* d) {
    size_t t = 1;
    for (int n = 0; n < d->order; ++n) t *= (size_t)d->dims[n];
    return 2 * t * 2;
}

void split_cache_free(SplitCache& c) {
    if (c.planes) cudaFree(c.planes);
    if (c.fac) cudaFree(c.fac);
    c = SplitCache{};
}

cp_status tc_mttkrp_all(SplitCache&, const cp_desc*, const Shape&, const void*, Ptrs<const double>, Ptrs<double>,
                        cudaStream_t) {
    return CP_ERR_UNSUPPORTED;
}

cp_status tc_mttkrp_mode(SplitCache&, const cp_desc*, const Shape&, const void*, Ptrs<const double>, Ptrs<double>,
                         int, cudaStream_t) {
    return CP_ERR_UNSUPPORTED;
}

}  // namespace cpgn
