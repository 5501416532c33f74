// gram_tc.cu -- S = <O^H O>^c on the 5th-generation tensor cores (placeholder until the
// tcgen05 kernel lands).
#include "vmc_internal.h"

namespace vmc {

cudaError_t launch_gram_tc(const __nv_bfloat16*, const __nv_bfloat16*, int64_t, int64_t, int64_t,
                           double, double2*, bool, unsigned*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace vmc
