// Single-precision instantiation of the exact exchange's fused grid passes.
#include "k_exx_grid.cuh"
namespace roks {
template void exx_batch_grid<float>(const ExxArgs<float>&, int, int, bool, cudaStream_t);
}
