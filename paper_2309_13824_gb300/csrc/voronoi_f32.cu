// voronoi_f32.cu -- a2 kernels instantiated for FP32 positions, single-mesh launches.
// Each instantiation is its own translation unit so they compile in parallel.
#include "voronoi.cuh"

namespace trime {
template void launch_voronoi_impl<float, false>(const IterArgs<float>&, int, cudaStream_t);
template void launch_voronoi_big<float>(const IterArgs<float>&, int32_t, float4*, int32_t*, int32_t*, cudaStream_t);
}  // namespace trime
