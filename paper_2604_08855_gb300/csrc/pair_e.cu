// pair_e.cu -- explicit instantiations of the pair-multipole kernel (see pair.cuh).
#include "pair.cuh"

namespace ctb {
template cudaError_t launch_pair_L<16>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<16>(int);
template cudaError_t launch_pair_L<18>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<18>(int);
}  // namespace ctb
