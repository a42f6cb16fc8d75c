// FP32 instances of the persistent FISTA loop (one kernel per transform length).
#include "k_fista.cuh"

namespace rix {
template int fista_loop<float>(const Ctx*, const FistaLoop<float>&, cudaStream_t);
}  // namespace rix
