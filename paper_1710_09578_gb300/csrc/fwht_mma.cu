// BF16 tensor-core Walsh-Hadamard transform (placeholder until the MMA kernel lands).
#include "fwht.h"

namespace fm {

fm_status fwht_mma_launch(FwhtArgs, int, cudaStream_t) {
  set_error("BF16 Hadamard modes are not built yet");
  return FM_ERR_UNSUPPORTED;
}

}  // namespace fm
