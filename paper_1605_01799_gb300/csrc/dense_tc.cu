// Dense A on the tensor cores (tcgen05): placeholder until the kernel lands.
#include "common.cuh"
#include "hopf_internal.h"

namespace hopf {

hopf_status dense_eval_tc(hopf_handle, DenseWs&, const float*, const float*, double*, float*, float*, int32_t*,
                          uint8_t*, cudaStream_t) {
  return fail(HOPF_EUNSUPPORTED, "tensor-core dense solver not built yet");
}

}  // namespace hopf
