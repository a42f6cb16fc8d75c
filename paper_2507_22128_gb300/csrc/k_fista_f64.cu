// FP64 instances of the persistent FISTA loop (one kernel per transform length).
#include "k_fista.cuh"

namespace rix {
template int fista_loop<double>(const Ctx*, const FistaLoop<double>&, cudaStream_t);
}  // namespace rix
