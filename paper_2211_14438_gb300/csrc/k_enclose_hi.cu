// Per-order enclosure kernels for Bernstein orders 9-16 (a separate
// translation unit so that the build compiles them in parallel).
#include "enclose_impl.cuh"

namespace bern {
#define BERN_ENC_INST(X)                                                                     \
  template cudaError_t launch_lb<X>(const Launch&, const Tables&, int, int64_t, int,         \
                                    const float*, const float*, int64_t, const int32_t*,     \
                                    float*, float*, EncloseOpts);
BERN_ENC_INST(9) BERN_ENC_INST(10) BERN_ENC_INST(11) BERN_ENC_INST(12)
BERN_ENC_INST(13) BERN_ENC_INST(14) BERN_ENC_INST(15) BERN_ENC_INST(16)
#undef BERN_ENC_INST
}  // namespace bern
