// ssco_values.cu -- value construction upstream of assembly: cotangent edge
// weights of a triangle mesh from per-value-set vertex positions (the
// cotangent Laplacian of the paper's mesh-processing experiments, Sec. 5.3),
// computed on the device so that a value set can be given as geometry.
#include <cuda_runtime.h>

#include <cstdint>

#include "ssco.h"

namespace ssco {
namespace {

// One thread per (triangle, value set): the three corner cotangents
// cot = (u . v) / |u x v| (u, v the edges leaving the corner) are added,
// halved, to the edge opposite each corner.  Plain round-to-nearest
// operations (no contraction), and at most two contributions per edge of a
// manifold mesh, so the sums do not depend on the order of the atomics.
__global__ void k_cotan(const int32_t* __restrict__ tri, const int32_t* __restrict__ tri_edge, int64_t n_tri,
                        int64_t n_vert, int64_t n_edge, int32_t batch, const double* __restrict__ xy,
                        double* __restrict__ w, int32_t* __restrict__ n_bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (t >= n_tri || b >= batch) return;
    const double* p = xy + (int64_t)b * n_vert * 2;
    double* wb = w + (int64_t)b * n_edge;
    int v[3];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c] = tri[3 * t + c];
        const int e = tri_edge[3 * t + c];
        ok = ok && v[c] >= 0 && v[c] < n_vert && e >= 0 && e < n_edge;
    }
    if (!ok) {  // out-of-range ids: skipped and counted, never dereferenced
        if (n_bad && b == 0) atomicAdd(n_bad, 1);
        return;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int k = v[c], i = v[(c + 1) % 3], j = v[(c + 2) % 3];
        const double ux = __dsub_rn(p[2 * i], p[2 * k]), uy = __dsub_rn(p[2 * i + 1], p[2 * k + 1]);
        const double vx = __dsub_rn(p[2 * j], p[2 * k]), vy = __dsub_rn(p[2 * j + 1], p[2 * k + 1]);
        const double dot = __dadd_rn(__dmul_rn(ux, vx), __dmul_rn(uy, vy));
        const double cross = fabs(__dsub_rn(__dmul_rn(ux, vy), __dmul_rn(uy, vx)));
        atomicAdd(&wb[tri_edge[3 * t + c]], __ddiv_rn(__dmul_rn(0.5, dot), cross));
    }
}

}  // namespace
}  // namespace ssco

extern "C" ssco_status ssco_cotan_weights(const int32_t* tri, const int32_t* tri_edge, int64_t n_tri, int64_t n_vert,
                                          int64_t n_edge, int32_t batch, const double* xy, double* w,
                                          int32_t* n_bad, void* stream) {
    if (n_tri < 0 || n_vert < 0 || n_edge < 0 || batch < 1 || batch > 65535) return SSCO_ERR_INVALID_ARG;
    if ((n_tri > 0 && (!tri || !tri_edge || !xy)) || (n_edge > 0 && !w)) return SSCO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_edge > 0 && cudaMemsetAsync(w, 0, (size_t)batch * n_edge * sizeof(double), s) != cudaSuccess)
        return SSCO_ERR_CUDA;
    if (n_tri > 0) {
        const dim3 grid((unsigned)((n_tri + 255) / 256), (unsigned)batch);
        ssco::k_cotan<<<grid, 256, 0, s>>>(tri, tri_edge, n_tri, n_vert, n_edge, batch, xy, w, n_bad);
        if (cudaGetLastError() != cudaSuccess) return SSCO_ERR_CUDA;
    }
    return SSCO_OK;
}
