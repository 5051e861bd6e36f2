// Forcing network (Sec. 2.2): placeholder until the tcgen05 network lands.
#include "nn_bridge.h"

namespace dgnn {
int nn_forcing_on_state(const nn_model*, const dg_ctx*, const double*, float*, int*, int*, cudaStream_t) {
  return fail(DG_ERR_UNSUPPORTED, "forcing network not built yet");
}
}  // namespace dgnn
