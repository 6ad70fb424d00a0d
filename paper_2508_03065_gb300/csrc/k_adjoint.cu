// Adjoint (reverse-mode) kernels of the synthesis path.
#include "msrc_internal.h"

namespace msrc {

size_t backward_extra_bytes(const KernelArgs&) { return 0; }

cudaError_t launch_backward(const KernelArgs&, const float* const*, float* const*, double* const*,
                            double* const*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace msrc
