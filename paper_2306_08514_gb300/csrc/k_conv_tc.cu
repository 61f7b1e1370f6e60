// Tensor-core conv. FD-SRP GEMM (tcgen05).  Not built yet: the plan rejects tensor
// precisions until this path exists.
#include "srp_internal.h"

namespace srp {

bool conv_tc_supported(int, int, int) { return false; }

cudaError_t launch_conv_tc(const void*, const void*, const void*, const void*, OpType, float*,
                           unsigned long long*, int, int, int, int, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace srp
