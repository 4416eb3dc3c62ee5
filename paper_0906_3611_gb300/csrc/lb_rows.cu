// lb_rows.cu -- row-streaming fused step kernel (placeholder until written).
#include "lb_rows.h"

namespace lbk {

bool rows_supported(const Geom&, int) { return false; }

cudaError_t launch_step_rows(int, const void*, void*, const Geom&, const PhysD&, Status*,
                             cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace lbk
