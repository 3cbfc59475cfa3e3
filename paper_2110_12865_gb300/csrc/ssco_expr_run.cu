// ssco_expr_run.cu -- device runner of compiled sparse matrix expressions.
//
// Slots live instance-innermost ([slot][batch]): the threads of a warp take
// consecutive value sets of one scalar expression, so every factor gather is
// one contiguous run and every lane runs the same number of terms.  With one
// value set a warp takes 32 consecutive expressions of a level, which were
// ordered by term count at compile time.  One launch per level (a level
// never reads its own results), plus the transposing copies in and out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ssco_expr_internal.h"

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

// one level: slot (slot0 + op) = sum over terms of coef * f1 * f2
template <class T, bool kUnit>
__global__ void __launch_bounds__(256)
    k_expr_level(const int64_t* __restrict__ toff, const int32_t* __restrict__ f1, const int32_t* __restrict__ f2,
                 const T* __restrict__ coef, int64_t op0, int64_t nops, int32_t B, int64_t slot0,
                 T* __restrict__ slots) {
    const int64_t total = nops * B;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t op = op0 + t / B;
        const int b = (int)(t % B);
        T acc = T(0);
        const int64_t q1 = toff[op + 1];
        for (int64_t q = toff[op]; q < q1; ++q) {
            const T p = slots[(int64_t)f1[q] * B + b] * slots[(int64_t)f2[q] * B + b];
            if (kUnit)
                acc += p;
            else
                acc += coef[q] * p;
        }
        slots[(slot0 + op) * B + b] = acc;
    }
}

// slots [slot][b] -> out [B][N]: out[b][j] = ocoef[j] * slots[oslot[j]][b]
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
        if (j < N && b < B) tile[jj][tx] = ocoef[j] * slots[(int64_t)oslot[j] * B + b];
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
        out[j] = ocoef[j] * slots[oslot[j]];
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
    const int64_t* toff = reinterpret_cast<const int64_t*>(tab + E.toff.term_off);
    const int32_t* f1 = reinterpret_cast<const int32_t*>(tab + E.toff.f1);
    const int32_t* f2 = reinterpret_cast<const int32_t*>(tab + E.toff.f2);
    const T* coef = reinterpret_cast<const T*>(tab + E.toff.coef);
    for (int32_t l = 1; l <= E.n_levels(); ++l) {
        const int64_t op0 = E.lvl_begin[l - 1], nops = E.lvl_begin[l] - op0;
        if (nops <= 0) continue;
        const unsigned g = grid_for(nops * B, 256);
        if (E.unit_coef)
            k_expr_level<T, true><<<g, 256, 0, s>>>(toff, f1, f2, coef, op0, nops, B, E.op_base(), slots);
        else
            k_expr_level<T, false><<<g, 256, 0, s>>>(toff, f1, f2, coef, op0, nops, B, E.op_base(), slots);
    }
    if (N > 0) {
        const int32_t* oslot = reinterpret_cast<const int32_t*>(tab + E.toff.out_slot);
        const T* ocoef = reinterpret_cast<const T*>(tab + E.toff.out_coef);
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
