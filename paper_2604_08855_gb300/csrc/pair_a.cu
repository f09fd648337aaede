// pair_a.cu -- explicit instantiations of the pair-multipole kernel (see pair.cuh).
#include "pair.cuh"

namespace ctb {
template cudaError_t launch_pair_L<0>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<0>(int);
template cudaError_t launch_pair_L<1>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<1>(int);
template cudaError_t launch_pair_L<2>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<2>(int);
template cudaError_t launch_pair_L<3>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<3>(int);
template cudaError_t launch_pair_L<4>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<4>(int);
template cudaError_t launch_pair_L<5>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<5>(int);
}  // namespace ctb
