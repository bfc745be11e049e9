// Single-precision instantiation of the band and grid transforms.
#include "k_fft_impl.cuh"
namespace roks {
ROKS_INSTANTIATE_FFT(float)
}
