// voronoi_f64.cu -- a2 kernels instantiated for FP64 positions, single-mesh launches.
// Each instantiation is its own translation unit so they compile in parallel.
#include "voronoi.cuh"

namespace trime {
template void launch_voronoi_impl<double, false>(const IterArgs<double>&, int, cudaStream_t);
template void launch_voronoi_big<double>(const IterArgs<double>&, int32_t, float4*, int32_t*, int32_t*, cudaStream_t);

// device exact predicates on explicit queries (verification hook)
__global__ void k_predicates(const double* pts, const int32_t* ids, int32_t nq, int32_t* o_out, int32_t* c_out) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double* p = pts + 8 * (size_t)q;
    const int32_t* id = ids + 4 * (size_t)q;
    o_out[q] = orient_exact(p, p + 2, p + 4);
    c_out[q] = incircle_sos(p, id[0], p + 2, id[1], p + 4, id[2], p + 6, id[3]);
}

void launch_predicates(const double* pts, const int32_t* ids, int32_t nq, int32_t* o_out, int32_t* c_out,
                       cudaStream_t st) {
    if (nq > 0) k_predicates<<<(nq + 127) / 128, 128, 0, st>>>(pts, ids, nq, o_out, c_out);
}
}  // namespace trime
