// lb_rows.h -- launcher of the row-streaming fused step kernel (lb_rows.cu).
#pragma once

#include "lb_kernels.h"

namespace lbk {

// True if the row-streaming kernel handles this lattice and storage.
bool rows_supported(const Geom& g, int storage);

cudaError_t launch_step_rows(int storage, const void* src, void* dst, const Geom& g,
                             const PhysD& ph, Status* status, cudaStream_t st);

}  // namespace lbk
