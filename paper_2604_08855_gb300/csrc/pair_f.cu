// pair_f.cu -- explicit instantiations of the pair-multipole kernel (see pair.cuh).
#include "pair.cuh"

namespace ctb {
template cudaError_t launch_pair_L<20>(const PairArgs&, int, int, cudaStream_t);
template int pair_occupancy_L<20>(int);
}  // namespace ctb
