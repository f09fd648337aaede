// pair_f.cu -- explicit instantiations of the pair-multipole kernel (see pair.cuh).
#include "pair.cuh"

namespace ctb {
template cudaError_t launch_alm_L<20>(const AlmArgs&, int, int, cudaStream_t);
template int alm_occupancy_L<20>(int);
}  // namespace ctb
