// FP64 instances of the persistent FISTA loop with the db1..db8 dictionary
// (one kernel per transform length).
#include "k_fista.cuh"

namespace rix {
template int fista_loop_dict<double, RIX_DICT_DB1_8>(const Ctx*, const FistaLoop<double>*, int, cudaStream_t);
}  // namespace rix
