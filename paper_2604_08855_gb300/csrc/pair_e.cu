// pair_e.cu -- explicit instantiations of the pair-multipole kernel (see pair.cuh).
#include "pair.cuh"

namespace ctb {
template cudaError_t launch_alm_L<16>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<16>(int);
template cudaError_t launch_alm_L<18>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<18>(int);
}  // namespace ctb
