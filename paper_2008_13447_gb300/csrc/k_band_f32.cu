// k_band_f32.cu -- FP32 instantiation of the band kernel (k_band.cuh).
#include "k_band.cuh"

namespace mad {

template void launch_band<float>(const BandArgs<float> &, bool, int, cudaStream_t);
template int band_occupancy<float>(bool, int, int);
template size_t band_smem<float>(bool, int, int);

}  // namespace mad
