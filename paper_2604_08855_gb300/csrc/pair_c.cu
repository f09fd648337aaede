// pair_c.cu -- explicit instantiations of the pair-multipole kernel (see pair.cuh).
#include "pair.cuh"

namespace ctb {
template cudaError_t launch_alm_L<9>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<9>(int);
template cudaError_t launch_alm_L<10>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<10>(int);
}  // namespace ctb
