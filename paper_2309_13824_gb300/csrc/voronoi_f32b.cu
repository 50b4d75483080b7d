// voronoi_f32b.cu -- a2 kernels instantiated for FP32 positions, batched launches (a table of meshes).
// Each instantiation is its own translation unit so they compile in parallel.
#include "voronoi.cuh"

namespace trime {
template void launch_voronoi_impl<float, true>(const IterArgs<float>&, int, cudaStream_t);
}  // namespace trime
