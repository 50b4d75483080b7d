// voronoi_f32.cu -- a2 kernels instantiated for FP32 positions, single-mesh launches.
// Each instantiation is its own translation unit so they compile in parallel.
#include "voronoi.cuh"

namespace trime {
template void launch_voronoi_impl<float, false>(const IterArgs<float>&, int, cudaStream_t);
}  // namespace trime
