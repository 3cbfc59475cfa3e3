// ssco_values.cu -- value construction upstream of assembly, computed on
// the device so that a value set can be given as geometry: cotangent edge
// weights of a triangle mesh (the cotangent Laplacian of the paper's
// mesh-processing experiments, Sec. 5.3) and stiffness blocks of linear
// tetrahedra (the element blocks of Sec. 4.2.4's tagged dense blocks, for
// the 3D elasticity configurations); plus the adjoint of per-call element
// blocks.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "ssco.h"
#include "ssco_internal.h"

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

// Stiffness blocks of linear tetrahedra, one CTA per kTetThreads tets of one
// value set.  Phase 1, thread per tet: the barycentric gradients g_0..g_3
// (rows of J^-1 by cross products, g_0 = -(g_1+g_2+g_3)) and the scaled Lame
// constants V*lambda, V*mu into shared memory.  Phase 2, the CTA writes the
// tets' 78 packed entries each as one contiguous, coalesced run:
//   K[3a+i][3b+j] = V (lambda g_a[i] g_b[j] + mu g_a[j] g_b[i] + mu [i==j] g_a.g_b).
constexpr int kTetThreads = 128;
constexpr int kTetPacked = 78;  // 12 * 13 / 2

__global__ void __launch_bounds__(kTetThreads)
    k_tet_stiffness(const int32_t* __restrict__ tets, int64_t n_tet, int64_t n_node, const double* __restrict__ xyz,
                    const double* __restrict__ E, double lam1, double mu1, double* __restrict__ K,
                    int32_t* __restrict__ n_bad) {
    __shared__ double sg[kTetThreads][12];
    __shared__ double sc[kTetThreads][2];
    __shared__ uint8_t srs[kTetPacked][2];
    const int b = blockIdx.y;
    const int64_t t0 = (int64_t)blockIdx.x * kTetThreads;
    const int64_t t = t0 + threadIdx.x;
    if (threadIdx.x < kTetPacked) {  // packed index q -> (r, s), r >= s
        int q = threadIdx.x, r = 0;
        while ((r + 1) * (r + 2) / 2 <= q) ++r;
        srs[q][0] = (uint8_t)r;
        srs[q][1] = (uint8_t)(q - r * (r + 1) / 2);
    }
    if (t < n_tet) {
        int v[4];
        bool ids_ok = true;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            v[a] = tets[4 * t + a];
            ids_ok = ids_ok && v[a] >= 0 && v[a] < n_node;
        }
        double g[4][3] = {};
        double vl = 0.0, vm = 0.0;
        bool ok = ids_ok;
        if (ids_ok) {
            const double* X = xyz + (int64_t)b * n_node * 3;
            double c[3][3];  // edge vectors x_k - x_0: the columns of J
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int i = 0; i < 3; ++i) c[k][i] = X[3 * (int64_t)v[k + 1] + i] - X[3 * (int64_t)v[0] + i];
#pragma unroll
            for (int k = 0; k < 3; ++k) {  // row k of adj(J): c_{k+1} x c_{k+2}
                const double* p = c[(k + 1) % 3];
                const double* q = c[(k + 2) % 3];
                g[k + 1][0] = p[1] * q[2] - p[2] * q[1];
                g[k + 1][1] = p[2] * q[0] - p[0] * q[2];
                g[k + 1][2] = p[0] * q[1] - p[1] * q[0];
            }
            const double det = c[0][0] * g[1][0] + c[0][1] * g[1][1] + c[0][2] * g[1][2];
            ok = det != 0.0 && isfinite(det);
            if (ok) {
                const double inv = 1.0 / det;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    g[1][i] *= inv;
                    g[2][i] *= inv;
                    g[3][i] *= inv;
                    g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
                }
                const double Ve = fabs(det) / 6.0 * (E ? E[(int64_t)b * n_tet + t] : 1.0);
                vl = Ve * lam1;
                vm = Ve * mu1;
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a) g[a][0] = g[a][1] = g[a][2] = 0.0;
            }
        }
        // out-of-range ids are the same for every value set: counted once;
        // degenerate geometry is per value set
        if (n_bad && ((!ids_ok && b == 0) || (ids_ok && !ok))) atomicAdd(n_bad, 1);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) sg[threadIdx.x][3 * a + i] = g[a][i];
        sc[threadIdx.x][0] = vl;
        sc[threadIdx.x][1] = vm;
    }
    __syncthreads();
    const int64_t nt = n_tet - t0 < kTetThreads ? n_tet - t0 : kTetThreads;
    double* out = K + ((int64_t)b * n_tet + t0) * kTetPacked;
    for (int idx = threadIdx.x; idx < nt * kTetPacked; idx += kTetThreads) {
        const int tl = idx / kTetPacked, q = idx - tl * kTetPacked;
        const int r = srs[q][0], s = srs[q][1];
        const int a = r / 3, i = r - 3 * a, bb = s / 3, j = s - 3 * bb;
        const double* ga = sg[tl] + 3 * a;
        const double* gb = sg[tl] + 3 * bb;
        double val = sc[tl][0] * ga[i] * gb[j] + sc[tl][1] * ga[j] * gb[i];
        if (i == j) val += sc[tl][1] * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
        out[idx] = val;
    }
}

// Adjoint of per-call element blocks: entry (r, s) of element e adds to
// K_uv and K_vu (u, v its global DOFs), so dloss/dentry = -(mu_u x_v +
// mu_v x_u) for r > s and -mu_u x_u for r = s; 0 on a fixed DOF.
__global__ void k_grad_blocks(const int32_t* __restrict__ dofs, const int64_t* __restrict__ off,
                              const int32_t* __restrict__ dim, const int32_t* __restrict__ vbase, int64_t nblk,
                              const double* __restrict__ mu, const double* __restrict__ x, int64_t n,
                              double* __restrict__ vbar, int64_t m) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nblk) return;
    const int b = blockIdx.y;
    const double* mb = mu + (int64_t)b * n;
    const double* xb = x + (int64_t)b * n;
    const int32_t* d = dofs + off[g];
    double* out = vbar + (int64_t)b * m + vbase[g];
    const int dm = dim[g];
    int p = 0;
    for (int i = 0; i < dm; ++i) {
        const int u = d[i];
        for (int j = 0; j <= i; ++j, ++p) {
            const int v = d[j];
            double val = 0.0;
            if (u >= 0 && v >= 0) val = i == j ? -(mb[u] * xb[u]) : -(mb[u] * xb[v] + mb[v] * xb[u]);
            out[p] = val;
        }
    }
}

}  // namespace

int launch_grad_blocks(Plan& P, const double* mu, const double* x, double* vals_bar, void* stream) {
    const int64_t nblk = (int64_t)P.blk_dim.size();
    if (nblk == 0) return 0;
    const uint8_t* tab = P.d_tab;
    const dim3 grid((unsigned)((nblk + 127) / 128), (unsigned)P.B);
    k_grad_blocks<<<grid, 128, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const int32_t*>(tab + P.toff.blk_dofs), reinterpret_cast<const int64_t*>(tab + P.toff.blk_off),
        reinterpret_cast<const int32_t*>(tab + P.toff.blk_dim), reinterpret_cast<const int32_t*>(tab + P.toff.blk_vbase),
        nblk, mu, x, P.n, vals_bar, P.m);
    ++P.launches;
    return (int)cudaGetLastError();
}

}  // namespace ssco

extern "C" ssco_status ssco_tet_stiffness(const int32_t* tets, int64_t n_tet, int64_t n_node, int32_t batch,
                                          const double* xyz, const double* E, double nu, double* K_e,
                                          int32_t* n_bad, void* stream) {
    if (n_tet < 0 || n_node < 0 || batch < 1 || batch > 65535) return SSCO_ERR_INVALID_ARG;
    if (!(nu > -1.0 && nu < 0.5)) return SSCO_ERR_INVALID_ARG;
    if (n_tet > 0 && (!tets || !xyz || !K_e)) return SSCO_ERR_INVALID_ARG;
    if (n_tet == 0) return SSCO_OK;
    const double lam1 = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu1 = 1.0 / (2.0 * (1.0 + nu));
    const dim3 grid((unsigned)((n_tet + ssco::kTetThreads - 1) / ssco::kTetThreads), (unsigned)batch);
    ssco::k_tet_stiffness<<<grid, ssco::kTetThreads, 0, (cudaStream_t)stream>>>(tets, n_tet, n_node, xyz, E, lam1,
                                                                              mu1, K_e, n_bad);
    return cudaGetLastError() == cudaSuccess ? SSCO_OK : SSCO_ERR_CUDA;
}

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
