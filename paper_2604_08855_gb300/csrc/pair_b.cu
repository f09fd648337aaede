// pair_b.cu -- explicit instantiations of the pair-multipole kernel (see pair.cuh).
#include "pair.cuh"

namespace ctb {
template cudaError_t launch_pair_L<6>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<6>(int);
template cudaError_t launch_pair_L<7>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<7>(int);
template cudaError_t launch_pair_L<8>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<8>(int);
}  // namespace ctb
