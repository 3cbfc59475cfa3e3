// ssco_expr_run.cu -- device runner of compiled sparse matrix expressions.
//
// Slots live instance-innermost ([slot][batch]): the threads of a warp take
// consecutive value sets of one scalar expression, so every factor gather is
// one contiguous run and every lane runs the same number of terms.  With one
// value set a warp takes 32 consecutive expressions of one term-count group
// and reads each term's factor indices as one coalesced run (the groups'
// term-major tables).  One launch per level (a level never reads its own
// results), plus the transposing copies in and out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ssco_expr_internal.h"
#include "ssco_gmac.cuh"

namespace ssco {
namespace {

// leaf [B][L] -> slots [1 + l][b]; slot 0 (the constant one) = 1
template <class T>
__global__ void k_expr_in(const T* __restrict__ leaf, int64_t L, int32_t B, T* __restrict__ slots) {
    __shared__ T tile[32][33];
    const int64_t l0 = (int64_t)blockIdx.x * 32;
    const int b0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int bb = ty; bb < 32; bb += 8) {
        const int b = b0 + bb;
        const int64_t l = l0 + tx;
        if (b < B && l < L) tile[bb][tx] = leaf[(int64_t)b * L + l];
    }
    __syncthreads();
    for (int ll = ty; ll < 32; ll += 8) {
        const int64_t l = l0 + ll;
        const int b = b0 + tx;
        if (b < B && l < L) slots[(1 + l) * B + b] = tile[tx][ll];
    }
    if (blockIdx.x == 0 && blockIdx.y == 0)
        for (int b = ty * 32 + tx; b < B; b += 256) slots[b] = T(1);
}

// one value set: slot 0 = 1 (the leaves are copied by cudaMemcpyAsync)
template <class T>
__global__ void k_expr_one(T* __restrict__ slots) {
    slots[0] = T(1);
}

// One level: thread f takes expression op_lo + f / B of the level for value
// set f % B (with one value set, one expression per thread), grid-strided
// over a grid capped at 16 CTAs per SM (fewer, longer-lived CTAs measured
// faster than one CTA per chunk of a group).  Its term-count group is found
// by binary search over the level's groups (consecutive runs of
// expressions).  The sum itself is the assembly's gather-MAC core, with a
// second gathered factor per term in groups that have products of two slots
// and the plain linear form (the assembly's own) in the others.
template <class T, bool kOne>
__global__ void __launch_bounds__(256)
    k_expr_level(const ExprProgram::Group* __restrict__ groups, int32_t g0, int32_t g1, int64_t op_lo, int64_t nops,
                const int32_t* __restrict__ i1, const int32_t* __restrict__ i2,
                const T* __restrict__ coef, int32_t B, int64_t slot0, T* __restrict__ slots) {
    const int64_t total = nops * (kOne ? 1 : B);
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t op = op_lo + (kOne ? f : f / B);
        const int32_t b = kOne ? 0 : (int32_t)(f % B);
        int32_t lo = g0, hi = g1 - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (groups[mid].op0 <= op)
                lo = mid;
            else
                hi = mid - 1;
        }
        const ExprProgram::Group g = groups[lo];
        const int32_t i = (int32_t)(op - g.op0);
        const T* __restrict__ x = slots + b;
        auto load = [x, B](int32_t s) { return x[(int64_t)s * (kOne ? 1 : B)]; };
        const T* cf = g.uniform ? nullptr : coef + g.coef_off + i;
        const T cu = (T)g.c_uniform;
        const T acc = g.quad ? gmac<T, true>(T(0), g.nterms, g.nmem, i1 + g.i1_off + i, i2 + g.i2_off + i, cf, cu, load)
                             : gmac<T, false>(T(0), g.nterms, g.nmem, i1 + g.i1_off + i, nullptr, cf, cu, load);
        slots[(slot0 + op) * (kOne ? 1 : B) + b] = acc;
    }
}

// slots [slot][b] -> out [B][N]: out[b][j] = ocoef[j] * slots[oslot[j]][b]
// (ocoef NULL: every factor is 1)
template <class T>
__global__ void k_expr_out(const T* __restrict__ slots, const int32_t* __restrict__ oslot,
                           const T* __restrict__ ocoef, int64_t N, int32_t B, T* __restrict__ out) {
    __shared__ T tile[32][33];
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int b0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int jj = ty; jj < 32; jj += 8) {
        const int64_t j = j0 + jj;
        const int b = b0 + tx;
        if (j < N && b < B) tile[jj][tx] = (ocoef ? ocoef[j] : T(1)) * slots[(int64_t)oslot[j] * B + b];
    }
    __syncthreads();
    for (int bb = ty; bb < 32; bb += 8) {
        const int b = b0 + bb;
        const int64_t j = j0 + tx;
        if (j < N && b < B) out[(int64_t)b * N + j] = tile[tx][bb];
    }
}

// one value set: a plain gather
template <class T>
__global__ void k_expr_out1(const T* __restrict__ slots, const int32_t* __restrict__ oslot,
                            const T* __restrict__ ocoef, int64_t N, T* __restrict__ out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = ocoef ? ocoef[j] * slots[oslot[j]] : slots[oslot[j]];
}

unsigned grid_for(int64_t work, int threads) {
    const int64_t cap = 152 * 16;  // persistent-ish cap: 16 CTAs of 256 per SM
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, cap));
}

template <class T>
int run(ExprProgram& E, const T* leaf, T* out, cudaStream_t s) {
    const uint8_t* tab = E.d_tab;
    T* slots = reinterpret_cast<T*>(E.d_ws);
    const int32_t B = E.B;
    const int64_t L = E.n_leaf_vals, N = E.n_out_vals;
    if (B == 1) {
        k_expr_one<T><<<1, 1, 0, s>>>(slots);
        if (L > 0 && cudaMemcpyAsync(slots + 1, leaf, (size_t)L * sizeof(T), cudaMemcpyDeviceToDevice, s))
            return 1;
    } else {
        const dim3 g((unsigned)std::max<int64_t>(1, (L + 31) / 32), (unsigned)((B + 31) / 32));
        k_expr_in<T><<<g, dim3(32, 8), 0, s>>>(leaf, L, B, slots);
    }
    const auto* groups = reinterpret_cast<const ExprProgram::Group*>(tab + E.toff.groups);
    const int32_t* i1 = reinterpret_cast<const int32_t*>(tab + E.toff.i1);
    const int32_t* i2 = reinterpret_cast<const int32_t*>(tab + E.toff.i2);
    const T* coef = reinterpret_cast<const T*>(tab + E.toff.coef);
    int32_t gcur = 0;
    for (int32_t l = 1; l <= E.n_levels(); ++l) {
        const int64_t op_lo = E.lvl_begin[l - 1], nops = E.lvl_begin[l] - op_lo;
        int32_t g1 = gcur;
        while (g1 < (int32_t)E.groups.size() && E.groups[g1].op0 < E.lvl_begin[l]) ++g1;
        if (nops <= 0) {
            gcur = g1;
            continue;
        }
        const unsigned g = grid_for(nops * B, 256);
        if (B == 1)
            k_expr_level<T, true><<<g, 256, 0, s>>>(groups, gcur, g1, op_lo, nops, i1, i2, coef, B, E.op_base(), slots);
        else
            k_expr_level<T, false><<<g, 256, 0, s>>>(groups, gcur, g1, op_lo, nops, i1, i2, coef, B, E.op_base(), slots);
        gcur = g1;
    }
    if (N > 0) {
        const int32_t* oslot = reinterpret_cast<const int32_t*>(tab + E.toff.out_slot);
        const T* ocoef = E.out_unit ? nullptr : reinterpret_cast<const T*>(tab + E.toff.out_coef);
        if (B == 1) {
            k_expr_out1<T><<<grid_for(N, 256), 256, 0, s>>>(slots, oslot, ocoef, N, out);
        } else {
            const dim3 g((unsigned)((N + 31) / 32), (unsigned)((B + 31) / 32));
            k_expr_out<T><<<g, dim3(32, 8), 0, s>>>(slots, oslot, ocoef, N, B, out);
        }
    }
    return cudaGetLastError() != cudaSuccess;
}

}  // namespace

int expr_launch_run(ExprProgram& E, const void* leaf_vals, void* out_vals, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (E.precision == SSCO_VALS_F32)
        return run<float>(E, static_cast<const float*>(leaf_vals), static_cast<float*>(out_vals), s);
    return run<double>(E, static_cast<const double*>(leaf_vals), static_cast<double*>(out_vals), s);
}

}  // namespace ssco
