// voronoi_f64b.cu -- a2 kernels instantiated for FP64 positions, batched launches (a table of meshes).
// Each instantiation is its own translation unit so they compile in parallel.
#include "voronoi.cuh"

namespace trime {
template void launch_voronoi_impl<double, true>(const IterArgs<double>&, int, cudaStream_t);
}  // namespace trime
