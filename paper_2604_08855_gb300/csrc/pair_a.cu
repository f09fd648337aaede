// pair_a.cu -- explicit instantiations of the pair-multipole kernel (see pair.cuh).
#include "pair.cuh"

namespace ctb {
template cudaError_t launch_alm_L<0>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<0>(int);
template cudaError_t launch_alm_L<1>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<1>(int);
template cudaError_t launch_alm_L<2>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<2>(int);
template cudaError_t launch_alm_L<3>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<3>(int);
template cudaError_t launch_alm_L<4>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<4>(int);
template cudaError_t launch_alm_L<5>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<5>(int);
}  // namespace ctb
