// pair_d.cu -- explicit instantiations of the pair-multipole kernel (see pair.cuh).
#include "pair.cuh"

namespace ctb {
template cudaError_t launch_alm_L<12>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<12>(int);
template cudaError_t launch_alm_L<14>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<14>(int);
}  // namespace ctb
