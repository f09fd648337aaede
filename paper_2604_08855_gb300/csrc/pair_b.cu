// pair_b.cu -- explicit instantiations of the pair-multipole kernel (see pair.cuh).
#include "pair.cuh"

namespace ctb {
template cudaError_t launch_alm_L<6>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<6>(int);
template cudaError_t launch_alm_L<7>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<7>(int);
template cudaError_t launch_alm_L<8>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<8>(int);
}  // namespace ctb
