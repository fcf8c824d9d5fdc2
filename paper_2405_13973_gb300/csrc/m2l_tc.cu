// m2l_tc.cu -- M2L on the tensor cores (placeholder until the tcgen05 kernel
// lands: reports the mode as unsupported).
#include <cuda_runtime.h>

#include "internal.h"

namespace pt {

size_t m2l_tc_operand_bytes(int) { return 0; }
void m2l_tc_pack_operands(int, const double*, const double*, float*) {}
cudaError_t launch_m2l_tc(int, int, Workspace&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace pt
