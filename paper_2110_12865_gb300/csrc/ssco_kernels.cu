// ssco_kernels.cu -- sm_103a kernels of the numeric phase and their launchers.
//
// Data layout (all per instance b, instance-outermost):
//   K      double [B][nnz_K]        assembled values, in assembly-group order
//   panel  T      [B][panel_total]  factor columns of every front, r x w col-major
//   upd    T      [B][upd_total]    update matrices, (r-w)^2 col-major (lower used)
//   pvec   T      [B][pvec_total]   forward-solve passing vectors (r-w per front)
//   vecT   T      [B][n]            rhs / y / x of the T-precision solves
//   bp, xp, rr, mu double [B][n]    permuted rhs, solution, residual; adjoint
// T = double (SSCO_FP64) or float (SSCO_FP32_REFINE).
//
// Schedule (host-built): assembly is one launch over all groups (Sec. 4.3/4.4
// leaf tables, coalesced term-major layout of Sec. 4.8).  The factorization
// visits the levels of the supernodal forest in increasing height; within a
// level, fronts are independent (Sec. 4.3 "no group member depends on
// another") and each size class is one launch.  A front's dense partial
// factorization is the tagged dense block of Sec. 4.2.4: its update matrix
// is a global intermediate (Sec. 4.2.1) consumed by its parent through a
// relative map (address coherence, Sec. 4.8).
#include <cuda_runtime.h>
#include <cooperative_groups.h>

#include <climits>
#include <cmath>
#include <algorithm>
#include <cstdint>
#include <vector>

#include "ssco_gmac.cuh"
#include "ssco_internal.h"
#include "ssco_tc.cuh"

namespace ssco {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Deterministic block reduction (fixed tree) of a sum and a max; result valid
// in thread 0.  blockDim.x must be a multiple of 32 and <= 1024.
__device__ void block_sum_max(double& s, double& mx) {
    __shared__ double ss[32], sm[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    s = warp_sum(s);
    mx = warp_max(mx);
    __syncthreads();
    if (lane == 0) {
        ss[wid] = s;
        sm[wid] = mx;
    }
    __syncthreads();
    if (wid == 0) {
        s = lane < nw ? ss[lane] : 0.0;
        mx = lane < nw ? sm[lane] : 0.0;
        s = warp_sum(s);
        mx = warp_max(mx);
    }
}

// --------------------------------------------------------------------------
// a1: assembly.  K[slot_base+i] = cadd + sum_t c_t vals[idx_t] (+ shift)
// --------------------------------------------------------------------------
template <class VT>
__global__ void __launch_bounds__(256) k_assemble(const AsmGroup* __restrict__ groups,
                                                  const AsmChunk* __restrict__ chunks,
                                                  const int32_t* __restrict__ idx,
                                                  const double* __restrict__ coef,
                                                  const VT* __restrict__ vals, int64_t m,
                                                  const double* __restrict__ shift, int32_t n_pats,
                                                  double* __restrict__ K, int64_t nnzK) {
    const AsmChunk ch = chunks[blockIdx.x];
    const AsmGroup g = groups[ch.group];
    const int i = ch.start + (int)threadIdx.x;
    if (i >= g.nmem) return;
    const int b = blockIdx.y;
    const VT* v = vals + (int64_t)b * m;
    double acc = gmac<double, false>(g.cadd, g.nterms, g.nmem, idx + g.idx_off + i, nullptr,
                                     g.uniform ? nullptr : coef + g.coef_off + i, g.coef,
                                     [v](int32_t p) { return (double)v[p]; });
    if (g.diag) acc += shift[(int64_t)b * n_pats + g.sys];
    K[(int64_t)b * nnzK + g.slot_base + i] = acc;
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// --------------------------------------------------------------------------
// a3: small fronts, one CTA per (front, instance), front resident in shared
// memory: gather K, extend-add children, partial Cholesky, write panel+update.
// --------------------------------------------------------------------------
// Column k of a front stored as a packed lower triangle (rows k..r-1)
// starts at packed_col(k, r); element (i, k), i >= k, sits at
// packed_col(k, r) + i - k.
__device__ __forceinline__ int packed_col(int k, int r) { return k * r - ((k * (k - 1)) >> 1); }

// Zero padding after a small front's packed triangle: the trailing update
// reads up to 3 x 16 rows / 3 x 16 columns past the last entry.
constexpr int kSmallPad = 128;

template <class T, int V>
struct VecOf;
template <>
struct VecOf<float, 4> {
    typedef float4 type;
};
template <>
struct VecOf<double, 2> {
    typedef double2 type;
};
template <>
struct VecOf<float, 2> {
    typedef float2 type;
};
template <>
struct VecOf<float, 1> {
    typedef float type;
};
template <>
struct VecOf<double, 1> {
    typedef double type;
};

template <class T, int V>
__device__ __forceinline__ void vld(const T* p, T (&x)[V]) {
    typedef typename VecOf<T, V>::type VT;
    const VT u = *reinterpret_cast<const VT*>(p);
    const T* e = reinterpret_cast<const T*>(&u);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = e[v];
}

template <class T, int V>
__device__ __forceinline__ void vst(T* p, const T (&x)[V]) {
    typedef typename VecOf<T, V>::type VT;
    VT u;
    T* e = reinterpret_cast<T*>(&u);
#pragma unroll
    for (int v = 0; v < V; ++v) e[v] = x[v];
    *reinterpret_cast<VT*>(p) = u;
}

// What a front's extend-add reads of a child; the first kChildRefs
// children's are loaded into shared memory when the CTA starts (one thread
// each, overlapping the zeroing of the front), so each child costs no
// dependent descriptor loads later.
struct ChildRef {
    int64_t upd_off, map_off;
    int32_t rc, pad;
};
constexpr int kChildRefs = 32;

__device__ __forceinline__ void prefetch_children(const DevTables& t, const FrontDesc& d, ChildRef* s_ch, int tid) {
    if (tid < min(d.nchild, kChildRefs)) {
        const FrontDesc& cd = t.fronts[t.child_ids[d.child_off + tid]];
        s_ch[tid] = ChildRef{cd.upd_off, cd.relmap_off, cd.r - cd.w, 0};
    }
}

__device__ __forceinline__ ChildRef child_ref(const DevTables& t, const FrontDesc& d, const ChildRef* s_ch, int c) {
    if (c < kChildRefs) return s_ch[c];
    const FrontDesc& cd = t.fronts[t.child_ids[d.child_off + c]];
    return ChildRef{cd.upd_off, cd.relmap_off, cd.r - cd.w, 0};
}

// Adds one child's update matrix (rc x rc, lower triangle, column-major;
// value set v at S + v * vstride) into the front's packed triangle F (V
// value sets interleaved) through the child's relative map: the warp walks
// (column kk, 32-row chunk) pairs of its columns kk = warp, warp + nw, ...,
// kEB pairs at a time, issuing all their loads before the shared-memory
// adds (one memory round trip per kEB pairs instead of per pair).
template <class T, int V>
__device__ __forceinline__ void extend_add(T* __restrict__ F, int r, const T* __restrict__ S, int64_t vstride,
                                           int nv, const int32_t* __restrict__ map, int rc, int warp, int nw,
                                           int lane) {
    constexpr int EB = V >= 4 ? 4 : 8;
    int kk = warp, i0 = warp;
    while (kk < rc) {
        int mi[EB], mk[EB];
        T sv[EB][V];
#pragma unroll
        for (int e = 0; e < EB; ++e) {
            const int ii = i0 + lane;
            const bool ok = kk < rc && ii < rc;
            mi[e] = ok ? map[ii] : -1;
            mk[e] = ok ? map[kk] : 0;
            const T* Sk = S + (int64_t)kk * rc + ii;
#pragma unroll
            for (int v = 0; v < V; ++v) sv[e][v] = (ok && v < nv) ? Sk[(int64_t)v * vstride] : T(0);
            if (kk < rc) {
                i0 += 32;
                if (i0 >= rc) {
                    kk += nw;
                    i0 = kk;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < EB; ++e) {
            if (mi[e] < 0) continue;
            T* Fe = F + (int64_t)(packed_col(mk[e], r) - mk[e] + mi[e]) * V;
            T x[V];
            vld<T, V>(Fe, x);
#pragma unroll
            for (int v = 0; v < V; ++v) x[v] += sv[e][v];
            vst<T, V>(Fe, x);
        }
    }
}

// Correctly rounded reciprocal (one instruction sequence instead of a
// division) for the pivot chain of the column steps.
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

template <class T>
__global__ void __launch_bounds__(256) k_front_small(const DevTables t, const int32_t* __restrict__ list,
                                                     const double* __restrict__ K, int64_t nnzK,
                                                     T* __restrict__ panel, int64_t panel_total,
                                                     T* __restrict__ upd, int64_t upd_total,
                                                     int32_t* __restrict__ bad_col, int32_t n_pats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* F = reinterpret_cast<T*>(smem_raw);  // packed lower triangle, r(r+1)/2
    const FrontDesc d = t.fronts[list[blockIdx.x]];
    const int b = blockIdx.y;
    const int r = d.r, w = d.w;
    const int lane = threadIdx.x, warp = threadIdx.y, nw = blockDim.y;
    const int tid = lane + 32 * warp, nth = 32 * nw;
    const int npk = r * (r + 1) / 2 + kSmallPad;
    __shared__ ChildRef s_ch[kChildRefs];
    prefetch_children(t, d, s_ch, tid);
    for (int q = tid; q < npk; q += nth) F[q] = T(0);
    __syncthreads();
    const double* Kb = K + (int64_t)b * nnzK;
    const int32_t* kl = t.klist + 2 * d.klist_off;
    for (int q = tid; q < d.klist_n; q += nth) {
        const int pos = kl[2 * q + 1];
        const int col = pos / r, row = pos - col * r;
        F[packed_col(col, r) + row - col] = (T)Kb[kl[2 * q]];
    }
    for (int c = 0; c < d.nchild; ++c) {
        __syncthreads();
        const ChildRef cr = child_ref(t, d, s_ch, c);
        extend_add<T, 1>(F, r, upd + (int64_t)b * upd_total + cr.upd_off, upd_total, 1, t.relmap + cr.map_off, cr.rc,
                         warp, nw, lane);
    }
    __syncthreads();
    // Blocked right-looking partial factorization.  Panels of kPanel columns
    // are factored column by column (each column scaled one step late, so one
    // barrier per column); the trailing matrix then takes one rank-kPanel
    // update with 4x4 register tiles per thread.
    constexpr int kPanel = 16;
    bool failed = false;
    const int tx = tid & 15, ty = tid >> 4, ny = nth >> 4;
    for (int j0 = 0; j0 < w; j0 += kPanel) {
        const int j1 = min(j0 + kPanel, w);
        T prev_inv = T(1), prev_l = T(1);
        for (int j = j0; j < j1; ++j) {
            T* Fj = F + packed_col(j, r) - j;
            T djj = Fj[j];
            if (!(djj > T(0))) {
                if (tid == 0 && !failed)
                    atomicMin(&bad_col[(int64_t)b * n_pats + d.sys], d.f + j - (int)t.sys_n_off[d.sys]);
                failed = true;
                djj = T(1);
            }
            const T invd = rcp_rn(djj);
            if (j > j0) {
                T* Fp = F + packed_col(j - 1, r) - (j - 1);
                for (int i = j + tid; i < r; i += nth) Fp[i] *= prev_inv;
                if (tid == 0) Fp[j - 1] = prev_l;
            }
            for (int k = j + 1 + warp; k < j1; k += nw) {
                const T lk = Fj[k] * invd;
                T* Fk = F + packed_col(k, r) - k;
                for (int i = k + lane; i < r; i += 32) Fk[i] -= Fj[i] * lk;
            }
            prev_inv = rsqrt(djj);
            prev_l = djj * prev_inv;
            __syncthreads();
        }
        {
            const int j = j1 - 1;
            T* Fj = F + packed_col(j, r) - j;
            for (int i = j + 1 + tid; i < r; i += nth) Fj[i] *= prev_inv;
            if (tid == 0) Fj[j] = prev_l;
        }
        __syncthreads();
        const int m = r - j1;
        if (m > 0) {
            const int tk_cols = 4 * ny;
            for (int c0 = 0; c0 < m; c0 += tk_cols) {
                for (int r0 = (c0 / 64) * 64; r0 < m; r0 += 64) {
                    T acc[4][4];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[a][q] = T(0);
                    int ii[4], kk[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        ii[a] = j1 + r0 + tx + 16 * a;
                        kk[a] = j1 + c0 + ty + ny * a;
                    }
                    // Rows or columns past r read the next column's entries
                    // or the zero padding (all within the allocation); they
                    // only reach accumulators the epilogue skips.
                    const T* Fi = F + packed_col(j0, r) - j0 + ii[0];
                    const T* Fk = F + packed_col(j0, r) - j0 + kk[0];
                    for (int j = j0; j < j1; ++j) {
                        T ra[4], cb[4];
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            ra[a] = Fi[16 * a];
                            cb[a] = Fk[ny * a];
                        }
                        Fi += r - j - 1;
                        Fk += r - j - 1;
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc[a][q] += ra[a] * cb[q];
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (kk[q] >= r) continue;
                        T* Fk = F + packed_col(kk[q], r) - kk[q];
#pragma unroll
                        for (int a = 0; a < 4; ++a)
                            if (ii[a] < r && ii[a] >= kk[q]) Fk[ii[a]] -= acc[a][q];
                    }
                }
            }
        }
        __syncthreads();
    }
    T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    for (int jj = warp; jj < w; jj += nw) {
        const T* Fj = F + packed_col(jj, r) - jj;
        for (int i = lane; i < r; i += 32) Pb[(int64_t)jj * r + i] = i >= jj ? Fj[i] : T(0);
    }
    const int ru = r - w;
    if (ru > 0) {
        T* Ub = upd + (int64_t)b * upd_total + d.upd_off;
        for (int kk = warp; kk < ru; kk += nw) {
            const T* Fk = F + packed_col(w + kk, r) - (w + kk);
            for (int ii = kk + lane; ii < ru; ii += 32) Ub[(int64_t)kk * ru + ii] = Fk[w + ii];
        }
    }
}

// Warp-per-(front, instance) variant of k_front_small for fronts of at most
// 64 rows: each warp assembles and factors its own front in a packed lower
// triangle in shared memory (rmax(rmax+1)/2 entries per warp), lane l
// owning rows l and l + 32; column-by-column right-looking with warp
// synchronisation only.  Eight fronts per CTA and no block barriers, for
// levels of many small fronts with few value sets (where one CTA per front
// spends its time in barriers).  Items are front-major.
template <class T>
__global__ void __launch_bounds__(256) k_front_warp(const DevTables t, const int32_t* __restrict__ list,
                                                    int32_t count, int32_t B, int32_t rmax,
                                                    const double* __restrict__ K, int64_t nnzK,
                                                    T* __restrict__ panel, int64_t panel_total,
                                                    T* __restrict__ upd, int64_t upd_total,
                                                    int32_t* __restrict__ bad_col, int32_t n_pats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t item = (int64_t)blockIdx.x * 8 + wib;
    if (item >= (int64_t)count * B) return;
    const int fi = (int)(item / B), b = (int)(item % B);
    const FrontDesc d = t.fronts[list[fi]];
    const int r = d.r, w = d.w;
    T* F = reinterpret_cast<T*>(smem_raw) + (int64_t)wib * (rmax * (rmax + 1) / 2);
    const int npk = r * (r + 1) / 2;
    for (int q = lane; q < npk; q += 32) F[q] = T(0);
    __syncwarp();
    const double* Kb = K + (int64_t)b * nnzK;
    const int32_t* kl = t.klist + 2 * d.klist_off;
    for (int q = lane; q < d.klist_n; q += 32) {
        const int pos = kl[2 * q + 1];
        const int col = pos / r, row = pos - col * r;
        F[packed_col(col, r) + row - col] = (T)Kb[kl[2 * q]];
    }
    for (int c = 0; c < d.nchild; ++c) {
        __syncwarp();
        const FrontDesc cd = t.fronts[t.child_ids[d.child_off + c]];
        const int rc = cd.r - cd.w;
        const int32_t* map = t.relmap + cd.relmap_off;
        const T* S = upd + (int64_t)b * upd_total + cd.upd_off;
        const int m0 = lane < rc ? map[lane] : 0, m1 = lane + 32 < rc ? map[lane + 32] : 0;
        for (int kk = 0; kk < rc; ++kk) {
            const int mk = __shfl_sync(0xffffffffu, kk < 32 ? m0 : m1, kk & 31);
            T* Fk = F + packed_col(mk, r) - mk;
            const T* Sk = S + (int64_t)kk * rc;
            if (lane >= kk && lane < rc) Fk[m0] += Sk[lane];
            if (lane + 32 >= kk && lane + 32 < rc) Fk[m1] += Sk[lane + 32];
        }
    }
    __syncwarp();
    // Panels of 8 columns: the panel's entries of the lane's two rows stay in
    // registers (p0, p1), the other rows' by shuffle; each trailing entry is
    // read and written once per panel.
    constexpr int PB = 8;
    bool failed = false;
    const int i0 = lane, i1 = lane + 32;
    for (int j0 = 0; j0 < w; j0 += PB) {
        const int j1 = min(j0 + PB, w);
        T p0[PB], p1[PB];
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            const int j = j0 + q;
            T v0 = T(0), v1 = T(0);
            if (j < j1) {
                const T* Fj = F + packed_col(j, r) - j;
                v0 = (i0 >= j && i0 < r) ? Fj[i0] : T(0);
                v1 = (i1 >= j && i1 < r) ? Fj[i1] : T(0);
                // left-looking within the panel: subtract the earlier panel
                // columns (row j's entries come from the lane holding row j)
#pragma unroll
                for (int pq = 0; pq < q; ++pq) {
                    const T ljp = __shfl_sync(0xffffffffu, j < 32 ? p0[pq] : p1[pq], j & 31);
                    v0 -= p0[pq] * ljp;
                    v1 -= p1[pq] * ljp;
                }
                T djj = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
                if (!(djj > T(0))) {
                    if (lane == 0 && !failed)
                        atomicMin(&bad_col[(int64_t)b * n_pats + d.sys], d.f + j - (int)t.sys_n_off[d.sys]);
                    failed = true;
                    djj = T(1);
                }
                const T ljj = sqrt(djj);
                const T inv = T(1) / ljj;
                v0 = i0 == j ? ljj : (i0 > j ? v0 * inv : T(0));
                v1 = i1 == j ? ljj : (i1 > j ? v1 * inv : T(0));
                T* Fw = F + packed_col(j, r) - j;
                if (i0 >= j && i0 < r) Fw[i0] = v0;
                if (i1 >= j && i1 < r) Fw[i1] = v1;
            }
            p0[q] = v0;
            p1[q] = v1;
        }
        // trailing update: F(i, k) -= sum_q L(i, j0+q) L(k, j0+q), k >= j1
        for (int k = j1; k < r; ++k) {
            T lk[PB];
#pragma unroll
            for (int q = 0; q < PB; ++q) lk[q] = __shfl_sync(0xffffffffu, k < 32 ? p0[q] : p1[q], k & 31);
            T* Fk = F + packed_col(k, r) - k;
            if (i0 >= k && i0 < r) {
                T a = Fk[i0];
#pragma unroll
                for (int q = 0; q < PB; ++q) a -= p0[q] * lk[q];
                Fk[i0] = a;
            }
            if (i1 >= k && i1 < r) {
                T a = Fk[i1];
#pragma unroll
                for (int q = 0; q < PB; ++q) a -= p1[q] * lk[q];
                Fk[i1] = a;
            }
        }
        __syncwarp();
    }
    T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    for (int jj = 0; jj < w; ++jj) {
        const T* Fj = F + packed_col(jj, r) - jj;
        for (int i = lane; i < r; i += 32) Pb[(int64_t)jj * r + i] = i >= jj ? Fj[i] : T(0);
    }
    const int ru = r - w;
    if (ru > 0) {
        T* Ub = upd + (int64_t)b * upd_total + d.upd_off;
        for (int kk = 0; kk < ru; ++kk) {
            const T* Fk = F + packed_col(w + kk, r) - (w + kk);
            for (int ii = kk + lane; ii < ru; ii += 32) Ub[(int64_t)kk * ru + ii] = Fk[w + ii];
        }
    }
}

// Instance-vectorized variant of k_front_small for small fronts and batches:
// one CTA factors the same front for V consecutive value sets, stored
// interleaved ([packed index][V]) so that one 16-byte shared-memory access
// serves all V and the index arithmetic is paid once per V fronts (the
// members of a group share one template expression, Sec. 4.8).
// Register budgets: V = 4 at 64 (four CTAs of 256 threads per SM), V = 2 at
// 85 (three), which holds its state without local memory; the two-set
// classes (128 and 160 rows) fit two or three CTAs per SM in shared memory.
template <class T, int V>
__global__ void __launch_bounds__(256, V == 2 ? 3 : 4)
    k_front_vec(const DevTables t, const int32_t* __restrict__ list, int32_t B, const double* __restrict__ K,
                int64_t nnzK, T* __restrict__ panel, int64_t panel_total, T* __restrict__ upd, int64_t upd_total,
                int32_t* __restrict__ bad_col, int32_t n_pats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* F = reinterpret_cast<T*>(smem_raw);
    const FrontDesc d = t.fronts[list[blockIdx.x]];
    const int b0 = blockIdx.y * V;
    const int nv = min(V, B - b0);
    const int r = d.r, w = d.w;
    const int lane = threadIdx.x, warp = threadIdx.y, nw = blockDim.y;
    const int tid = lane + 32 * warp, nth = 32 * nw;
    const int npk = r * (r + 1) / 2 + kSmallPad;
    __shared__ ChildRef s_ch[kChildRefs];
    prefetch_children(t, d, s_ch, tid);
    for (int q = tid; q < npk * V; q += nth) F[q] = T(0);
    __syncthreads();
    const int32_t* kl = t.klist + 2 * d.klist_off;
    for (int e = tid; e < d.klist_n; e += nth) {
        const int pos = kl[2 * e + 1], slot = kl[2 * e];
        const int col = pos / r, row = pos - col * r;
        T* dst = F + (int64_t)(packed_col(col, r) + row - col) * V;
        for (int v = 0; v < nv; ++v) dst[v] = (T)K[(int64_t)(b0 + v) * nnzK + slot];
    }
    for (int c = 0; c < d.nchild; ++c) {
        __syncthreads();
        const ChildRef cr = child_ref(t, d, s_ch, c);
        extend_add<T, V>(F, r, upd + (int64_t)b0 * upd_total + cr.upd_off, upd_total, nv, t.relmap + cr.map_off, cr.rc,
                         warp, nw, lane);
    }
    __syncthreads();
    constexpr int kPanel = 16;
    bool failed[V];
#pragma unroll
    for (int v = 0; v < V; ++v) failed[v] = false;
    const int tx = tid & 15, ty = tid >> 4, ny = nth >> 4;
    const int n_off = (int)t.sys_n_off[d.sys];
    for (int j0 = 0; j0 < w; j0 += kPanel) {
        const int j1 = min(j0 + kPanel, w);
        T prev_inv[V], prev_l[V];
#pragma unroll
        for (int v = 0; v < V; ++v) prev_inv[v] = prev_l[v] = T(1);
        for (int j = j0; j < j1; ++j) {
            T* Fj = F + (int64_t)(packed_col(j, r) - j) * V;
            T djj[V], invd[V];
            vld<T, V>(Fj + (int64_t)j * V, djj);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (!(djj[v] > T(0))) {
                    if (v < nv && tid == 0 && !failed[v])
                        atomicMin(&bad_col[(int64_t)(b0 + v) * n_pats + d.sys], d.f + j - n_off);
                    failed[v] = true;
                    djj[v] = T(1);
                }
                invd[v] = rcp_rn(djj[v]);
            }
            if (j > j0) {
                T* Fp = F + (int64_t)(packed_col(j - 1, r) - (j - 1)) * V;
                for (int i = j + tid; i < r; i += nth) {
                    T x[V];
                    vld<T, V>(Fp + (int64_t)i * V, x);
#pragma unroll
                    for (int v = 0; v < V; ++v) x[v] *= prev_inv[v];
                    vst<T, V>(Fp + (int64_t)i * V, x);
                }
                if (tid == 0) vst<T, V>(Fp + (int64_t)(j - 1) * V, prev_l);
            }
            for (int k = j + 1 + warp; k < j1; k += nw) {
                T lk[V];
                vld<T, V>(Fj + (int64_t)k * V, lk);
#pragma unroll
                for (int v = 0; v < V; ++v) lk[v] *= invd[v];
                T* Fk = F + (int64_t)(packed_col(k, r) - k) * V;
                for (int i = k + lane; i < r; i += 32) {
                    T x[V], y[V];
                    vld<T, V>(Fk + (int64_t)i * V, x);
                    vld<T, V>(Fj + (int64_t)i * V, y);
#pragma unroll
                    for (int v = 0; v < V; ++v) x[v] -= y[v] * lk[v];
                    vst<T, V>(Fk + (int64_t)i * V, x);
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                prev_inv[v] = rsqrt(djj[v]);
                prev_l[v] = djj[v] * prev_inv[v];
            }
            __syncthreads();
        }
        {
            const int j = j1 - 1;
            T* Fj = F + (int64_t)(packed_col(j, r) - j) * V;
            for (int i = j + 1 + tid; i < r; i += nth) {
                T x[V];
                vld<T, V>(Fj + (int64_t)i * V, x);
#pragma unroll
                for (int v = 0; v < V; ++v) x[v] *= prev_inv[v];
                vst<T, V>(Fj + (int64_t)i * V, x);
            }
            if (tid == 0) vst<T, V>(Fj + (int64_t)j * V, prev_l);
        }
        __syncthreads();
        const int m = r - j1;
        if (m > 0) {
            const int tk_cols = 2 * ny;
            for (int c0 = 0; c0 < m; c0 += tk_cols) {
                for (int r0 = (c0 / 64) * 64; r0 < m; r0 += 64) {
                    T acc[4][2][V];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int q = 0; q < 2; ++q)
#pragma unroll
                            for (int v = 0; v < V; ++v) acc[a][q][v] = T(0);
                    int ii[4], kk[2];
#pragma unroll
                    for (int a = 0; a < 4; ++a) ii[a] = j1 + r0 + tx + 16 * a;
#pragma unroll
                    for (int q = 0; q < 2; ++q) kk[q] = j1 + c0 + ty + ny * q;
                    // rows / columns past r read the next column's entries or
                    // the zero padding (within the allocation); they only
                    // reach accumulators the epilogue skips
                    const T* Fi = F + (int64_t)(packed_col(j0, r) - j0 + ii[0]) * V;
                    const T* Fk = F + (int64_t)(packed_col(j0, r) - j0 + kk[0]) * V;
                    for (int j = j0; j < j1; ++j) {
                        T ra[4][V], cb[2][V];
#pragma unroll
                        for (int a = 0; a < 4; ++a) vld<T, V>(Fi + (int64_t)(16 * a) * V, ra[a]);
#pragma unroll
                        for (int q = 0; q < 2; ++q) vld<T, V>(Fk + (int64_t)(ny * q) * V, cb[q]);
                        Fi += (int64_t)(r - j - 1) * V;
                        Fk += (int64_t)(r - j - 1) * V;
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int q = 0; q < 2; ++q)
#pragma unroll
                                for (int v = 0; v < V; ++v) acc[a][q][v] += ra[a][v] * cb[q][v];
                    }
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (kk[q] >= r) continue;
                        T* Fk = F + (int64_t)(packed_col(kk[q], r) - kk[q]) * V;
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            if (ii[a] < r && ii[a] >= kk[q]) {
                                T x[V];
                                vld<T, V>(Fk + (int64_t)ii[a] * V, x);
#pragma unroll
                                for (int v = 0; v < V; ++v) x[v] -= acc[a][q][v];
                                vst<T, V>(Fk + (int64_t)ii[a] * V, x);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    T* P0 = panel + (int64_t)b0 * panel_total + d.panel_off;
    for (int jj = warp; jj < w; jj += nw) {
        const T* Fj = F + (int64_t)(packed_col(jj, r) - jj) * V;
        for (int i = lane; i < r; i += 32) {
            T x[V];
            if (i >= jj)
                vld<T, V>(Fj + (int64_t)i * V, x);
            else
#pragma unroll
                for (int v = 0; v < V; ++v) x[v] = T(0);
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (v < nv) P0[(int64_t)v * panel_total + (int64_t)jj * r + i] = x[v];
        }
    }
    const int ru = r - w;
    if (ru > 0) {
        T* U0 = upd + (int64_t)b0 * upd_total + d.upd_off;
        for (int kk = warp; kk < ru; kk += nw) {
            const T* Fk = F + (int64_t)(packed_col(w + kk, r) - (w + kk)) * V;
            for (int ii = kk + lane; ii < ru; ii += 32) {
                T x[V];
                vld<T, V>(Fk + (int64_t)(w + ii) * V, x);
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (v < nv) U0[(int64_t)v * upd_total + (int64_t)kk * ru + ii] = x[v];
            }
        }
    }
}

// --------------------------------------------------------------------------
// a3': tiny subtrees.  Every front of the subtree has r <= 32 rows; one warp
// factors the whole subtree, children first, with lane i holding row i of
// the front in registers (column broadcasts by warp shuffles).  This folds
// the lowest levels of the forest into one launch of independent warps.
// --------------------------------------------------------------------------
constexpr int kTinyWarps = 8;

// Shared memory of the tiny kernels: each warp's own area (the front and
// K values, or the solve vector) and the subtree program.  With a batch that
// is a multiple of kTinyWarps, the warps of a CTA take the same subtree for
// consecutive value sets and share one copy of its program (loaded once per
// CTA instead of once per warp); otherwise each warp has its own.
inline bool tiny_share(int32_t B) { return B % kTinyWarps == 0; }
__host__ __device__ inline int tiny_prog_bytes(int prog_max) { return (prog_max * 4 + 15) & ~15; }
template <class T>
__host__ __device__ inline int tiny_factor_own(int k_max) {
    return ((32 * 33 + k_max) * (int)sizeof(T) + 15) & ~15;
}
template <class T>
__host__ __device__ inline int tiny_solve_own() {
    return (32 * (int)sizeof(T) + 15) & ~15;
}
template <class T>
inline int tiny_factor_bytes(bool share, int prog_max, int k_max) {
    return share ? tiny_prog_bytes(prog_max) + kTinyWarps * tiny_factor_own<T>(k_max)
                 : kTinyWarps * (tiny_factor_own<T>(k_max) + tiny_prog_bytes(prog_max));
}
template <class T>
inline int tiny_solve_bytes(bool share, int prog_max) {
    return share ? tiny_prog_bytes(prog_max) + kTinyWarps * tiny_solve_own<T>()
                 : kTinyWarps * (tiny_solve_own<T>() + tiny_prog_bytes(prog_max));
}

// Loads subtree st's program into shared memory (coalesced).
__device__ __forceinline__ void load_prog(const DevTables& t, int st, int32_t* prog, int lane) {
    const int64_t base = t.tiny_prog_off[st];
    const int total = (int)(t.tiny_prog_off[st + 1] - base);
    for (int i = lane; i < total; i += 32) prog[i] = t.tiny_prog[base + i];
    __syncwarp();
}
// Program of this warp's subtree in shared memory, and the warp's own area
// of `own` bytes: a CTA-wide copy (share) or one per warp.
__device__ __forceinline__ int32_t* tiny_setup(const DevTables& t, unsigned char* smem_raw, bool share, int st,
                                               int prog_max, int own, int wib, int lane, unsigned char** mine) {
    if (share) {
        int32_t* prog = reinterpret_cast<int32_t*>(smem_raw);
        const int64_t base = t.tiny_prog_off[st];
        const int total = (int)(t.tiny_prog_off[st + 1] - base);
        for (int i = threadIdx.x; i < total; i += blockDim.x) prog[i] = t.tiny_prog[base + i];
        __syncthreads();
        *mine = smem_raw + tiny_prog_bytes(prog_max) + (size_t)wib * own;
        return prog;
    }
    *mine = smem_raw + (size_t)wib * (own + tiny_prog_bytes(prog_max));
    int32_t* prog = reinterpret_cast<int32_t*>(*mine + own);
    load_prog(t, st, prog, lane);
    return prog;
}

__device__ __forceinline__ int64_t prog_i64(const int32_t* rec, int at) {
    return (int64_t)(uint32_t)rec[at] | ((int64_t)rec[at + 1] << 32);
}

// Partial Cholesky of one front of at most R rows held as lane-per-row
// registers (a[k] = F[lane][k]); writes the r x w panel and the (r-w)^2
// update.  Compact form: the pivot column is always a[0] and the registers
// shift left by one per step, so the step loop is a runtime loop (code size
// O(R) instead of O(R^2)).  Returns the first non-positive pivot's column
// or -1.
template <class T, int R>
__device__ __forceinline__ int tiny_chol_rows(T (*F)[33], int lane, int r, int w, T* __restrict__ Pf,
                                              T* __restrict__ Uf) {
    T a[R];
#pragma unroll
    for (int k = 0; k < R; ++k) a[k] = F[lane][k];
    int bad = -1;
#pragma unroll 1
    for (int j = 0; j < w; ++j) {
        T djj = __shfl_sync(0xffffffffu, a[0], j);
        if (!(djj > T(0))) {
            if (bad < 0) bad = j;
            djj = T(1);
        }
        const T ljj = sqrt(djj);
        const T inv = T(1) / ljj;
        if (lane == j)
            a[0] = ljj;
        else if (lane > j)
            a[0] *= inv;
        if (lane < r) Pf[(int64_t)j * r + lane] = lane >= j ? a[0] : T(0);
#pragma unroll
        for (int k = 1; k < R; ++k) {
            const T lkj = __shfl_sync(0xffffffffu, a[0], (j + k) & 31);
            if (lane >= j + k && j + k < r) a[k] -= a[0] * lkj;
        }
#pragma unroll
        for (int k = 0; k < R - 1; ++k) a[k] = a[k + 1];
        a[R - 1] = T(0);
    }
    if (lane < r) {
        const int ru = r - w;
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (k < ru && lane >= w + k) Uf[(int64_t)k * ru + (lane - w)] = a[k];
    }
    return bad;
}

// The same partial Cholesky for fronts of at most R <= 16 rows, fully
// unrolled: column k stays in register a[k] (no shifting) and every step's
// update of the later columns is one shuffle and one multiply-add per
// column with no per-lane predicate -- rows above a column's diagonal take
// values that are never stored.
template <class T, int R>
__device__ __forceinline__ int tiny_chol_rows_unrolled(T (*F)[33], int lane, int r, int w, T* __restrict__ Pf,
                                                       T* __restrict__ Uf) {
    T a[R];
#pragma unroll
    for (int k = 0; k < R; ++k) a[k] = F[lane][k];
    int bad = -1;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if (j < w) {
            T djj = __shfl_sync(0xffffffffu, a[j], j);
            if (!(djj > T(0))) {
                if (bad < 0) bad = j;
                djj = T(1);
            }
            const T ljj = sqrt(djj);
            const T inv = T(1) / ljj;
            a[j] = lane == j ? ljj : a[j] * inv;
            if (lane < r) Pf[(int64_t)j * r + lane] = lane >= j ? a[j] : T(0);
#pragma unroll
            for (int k = j + 1; k < R; ++k) a[k] -= a[j] * __shfl_sync(0xffffffffu, a[j], k);
        }
    }
    if (lane < r) {
        const int ru = r - w;
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (k >= w && k < r && lane >= k) Uf[(int64_t)(k - w) * ru + (lane - w)] = a[k];
    }
    return bad;
}

// A child's update matrix (rc <= RC rows, lower triangle, column-major)
// added into the front tile through its relative map: lane i holds row i;
// its entries are loaded together (the bound is fixed, so the loop unrolls)
// before they are added.
template <class T, int RC>
__device__ __forceinline__ void tiny_child_add(T (*F)[33], const int32_t* map, const T* __restrict__ S, int rc,
                                               int lane) {
    if (lane >= rc) return;
    T sv[RC];
#pragma unroll
    for (int kk = 0; kk < RC; ++kk) sv[kk] = kk <= lane ? S[lane + kk * rc] : T(0);
    const int mi = map[lane];
#pragma unroll
    for (int kk = 0; kk < RC; ++kk)
        if (kk <= lane) F[mi][map[kk]] += sv[kk];
}

template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
    k_tiny_factor(const DevTables t, int32_t n_tiny, int32_t B, int32_t prog_max, int32_t k_max,
                  const double* __restrict__ K, int64_t nnzK, T* __restrict__ panel, int64_t panel_total,
                  T* __restrict__ upd, int64_t upd_total, int32_t* __restrict__ bad_col, int32_t n_pats,
                  int32_t share) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t item = (int64_t)blockIdx.x * kTinyWarps + wib;
    if (!share && item >= (int64_t)n_tiny * B) return;
    const int st = (int)(item / B), b = (int)(item % B);
    unsigned char* mine;
    int32_t* prog = tiny_setup(t, smem_raw, share != 0, st, prog_max, tiny_factor_own<T>(k_max), wib, lane, &mine);
    T(*F)[33] = reinterpret_cast<T(*)[33]>(mine);
    T* Fflat = reinterpret_cast<T*>(mine);
    T* kv = reinterpret_cast<T*>(mine) + 32 * 33;
    const int nf = prog[0], nk = prog[1], rec_off = prog[2], k_off = prog[4], sys = prog[7];
    const double* Kb = K + (int64_t)b * nnzK;
    for (int e = lane; e < nk; e += 32) kv[e] = (T)Kb[prog[k_off + 2 * e]];
    T* Pb = panel + (int64_t)b * panel_total;
    T* Ub = upd + (int64_t)b * upd_total;
    const int n_off = (int)t.sys_n_off[sys];
    __syncwarp();
    for (int q = 0; q < nf; ++q) {
        const int32_t* rec = prog + rec_off + kTinyRecWords * q;
        const int r = rec[0], w = rec[1], f = rec[2], nchild = rec[3];
        const int kbeg = rec[5], kn = rec[6];
        const int64_t panel_off = prog_i64(rec, 10), upd_off = prog_i64(rec, 12);
        for (int k = 0; k < r; ++k) F[lane][k] = T(0);
        __syncwarp();
        for (int e = lane; e < kn; e += 32) Fflat[prog[k_off + 2 * (kbeg + e) + 1]] = kv[kbeg + e];
        for (int c = 0; c < nchild; ++c) {
            __syncwarp();
            const int32_t* crec = prog + rec_off + kTinyRecWords * prog[rec[4] + c];
            const int rc = crec[0] - crec[1];
            const int32_t* map = prog + crec[7];
            const T* S = Ub + prog_i64(crec, 12);
            if (rc <= 8)
                tiny_child_add<T, 8>(F, map, S, rc, lane);
            else if (rc <= 16)
                tiny_child_add<T, 16>(F, map, S, rc, lane);
            else if (lane < rc) {
                const int mi = map[lane];
                for (int kk = 0; kk <= lane; ++kk) F[mi][map[kk]] += S[lane + kk * rc];
            }
        }
        __syncwarp();
        // fronts of a subtree are visited children-first, not in column
        // order: record the first failing pivot of every front (atomicMin)
        int badj;
        if (r <= 8)
            badj = tiny_chol_rows_unrolled<T, 8>(F, lane, r, w, Pb + panel_off, Ub + upd_off);
        else if (r <= 16)
            badj = tiny_chol_rows_unrolled<T, 16>(F, lane, r, w, Pb + panel_off, Ub + upd_off);
        else
            badj = tiny_chol_rows<T, 32>(F, lane, r, w, Pb + panel_off, Ub + upd_off);
        if (badj >= 0 && lane == 0) atomicMin(&bad_col[(int64_t)b * n_pats + sys], f + badj - n_off);
        __syncwarp();
    }
}

// Forward / backward substitution with the w <= W columns of one tiny
// front; lane i holds row i.
template <class T, int W>
__device__ __forceinline__ T tiny_fwd_chain(const T* __restrict__ Pf, int lane, int r, int w, T v) {
    T a[W];
#pragma unroll
    for (int j = 0; j < W; ++j) a[j] = (j < w && lane < r) ? Pf[(int64_t)j * r + lane] : T(0);
    T dl = T(1);
#pragma unroll
    for (int j = 0; j < W; ++j)
        if (lane == j && j < w) dl = a[j];
    const T dinv = T(1) / dl;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        if (j < w) {
            const T yj = __shfl_sync(0xffffffffu, v, j) * __shfl_sync(0xffffffffu, dinv, j);
            if (lane == j)
                v = yj;
            else if (lane > j)
                v -= a[j] * yj;
        }
    }
    return v;
}

template <class T, int W>
__device__ __forceinline__ T tiny_bwd_chain(const T* __restrict__ Pf, int lane, int r, int w, T v) {
    T a[W];
#pragma unroll
    for (int j = 0; j < W; ++j) a[j] = (j < w && lane < r) ? Pf[(int64_t)j * r + lane] : T(0);
    T dl = T(1);
#pragma unroll
    for (int j = 0; j < W; ++j)
        if (lane == j && j < w) dl = a[j];
    const T dinv = T(1) / dl;
#pragma unroll
    for (int j = W - 1; j >= 0; --j) {
        if (j < w) {
            T s = (lane > j && lane < r) ? a[j] * v : T(0);
            s = warp_sum(s);
            if (lane == j) v = (v - s) * dinv;
        }
    }
    return v;
}

// FP32 tiny solves: at most 40 registers, six CTAs (48 warps) per SM; the
// few values kept in local memory cost less than the warps gained.
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 1)
    k_tiny_fwd(const DevTables t, int32_t n_tiny, int32_t B, int32_t prog_max, const T* __restrict__ panel,
               int64_t panel_total, T* __restrict__ vec, int64_t n, T* __restrict__ pvec, int64_t pvec_total,
               const int32_t* __restrict__ active, int32_t n_pats, int32_t share) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t item = (int64_t)blockIdx.x * kTinyWarps + wib;
    if (!share && item >= (int64_t)n_tiny * B) return;
    const int st = (int)(item / B), b = (int)(item % B);
    unsigned char* mine;
    int32_t* prog = tiny_setup(t, smem_raw, share != 0, st, prog_max, tiny_solve_own<T>(), wib, lane, &mine);
    T* vs = reinterpret_cast<T*>(mine);
    const int nf = prog[0], rec_off = prog[2];
    if (active && !active[(int64_t)b * n_pats + prog[7]]) return;
    const T* Pb = panel + (int64_t)b * panel_total;
    T* vb = vec + (int64_t)b * n;
    T* pv = pvec + (int64_t)b * pvec_total;
    for (int q = 0; q < nf; ++q) {
        const int32_t* rec = prog + rec_off + kTinyRecWords * q;
        const int r = rec[0], w = rec[1], f = rec[2], nchild = rec[3];
        const int64_t panel_off = prog_i64(rec, 10), pvec_off = prog_i64(rec, 14);
        vs[lane] = lane < w ? vb[f + lane] : T(0);
        for (int c = 0; c < nchild; ++c) {
            __syncwarp();
            const int32_t* crec = prog + rec_off + kTinyRecWords * prog[rec[4] + c];
            const int rc = crec[0] - crec[1];
            if (lane < rc) vs[prog[crec[7] + lane]] += pv[prog_i64(crec, 14) + lane];
        }
        __syncwarp();
        T v = vs[lane];
        if (w <= 8)
            v = tiny_fwd_chain<T, 8>(Pb + panel_off, lane, r, w, v);
        else if (w <= 16)
            v = tiny_fwd_chain<T, 16>(Pb + panel_off, lane, r, w, v);
        else
            v = tiny_fwd_chain<T, 32>(Pb + panel_off, lane, r, w, v);
        if (lane < w)
            vb[f + lane] = v;
        else if (lane < r)
            pv[pvec_off + lane - w] = v;
        __syncwarp();
    }
}

template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 1)
    k_tiny_bwd(const DevTables t, int32_t n_tiny, int32_t B, int32_t prog_max, const T* __restrict__ panel,
               int64_t panel_total, T* __restrict__ vec, int64_t n, const int32_t* __restrict__ active,
               int32_t n_pats, int32_t share) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t item = (int64_t)blockIdx.x * kTinyWarps + wib;
    if (!share && item >= (int64_t)n_tiny * B) return;
    const int st = (int)(item / B), b = (int)(item % B);
    unsigned char* mine;
    int32_t* prog = tiny_setup(t, smem_raw, share != 0, st, prog_max, tiny_solve_own<T>(), wib, lane, &mine);
    const int nf = prog[0], rec_off = prog[2];
    if (active && !active[(int64_t)b * n_pats + prog[7]]) return;
    const T* Pb = panel + (int64_t)b * panel_total;
    T* vb = vec + (int64_t)b * n;
    for (int q = nf - 1; q >= 0; --q) {
        const int32_t* rec = prog + rec_off + kTinyRecWords * q;
        const int r = rec[0], w = rec[1], f = rec[2];
        const int64_t panel_off = prog_i64(rec, 10);
        T v = lane < w ? vb[f + lane] : (lane < r ? vb[prog[rec[8] + lane - w]] : T(0));
        if (w <= 8)
            v = tiny_bwd_chain<T, 8>(Pb + panel_off, lane, r, w, v);
        else if (w <= 16)
            v = tiny_bwd_chain<T, 16>(Pb + panel_off, lane, r, w, v);
        else
            v = tiny_bwd_chain<T, 32>(Pb + panel_off, lane, r, w, v);
        if (lane < w) vb[f + lane] = v;
        __syncwarp();
    }
}

// --------------------------------------------------------------------------
// a4: big fronts (r > small_front_max), dense panel in global memory.
// --------------------------------------------------------------------------
// Panel and update initialised from the children's update matrices through
// inverse maps (pull, fixed child order => deterministic, no atomics).  One
// CTA per 64x64 tile of the lower triangle: the tile's rows and columns of
// up to 8 children's inverse maps are staged in shared memory, so each
// element costs one load per child that holds it.  Thread (tx, ty) owns
// row i0 + tx and columns j0 + ty + 4q, q < 16.
template <class T>
__global__ void __launch_bounds__(256) k_big_init(const DevTables t, const int32_t* __restrict__ list,
                                                  T* __restrict__ panel, int64_t panel_total,
                                                  T* __restrict__ upd, int64_t upd_total) {
    const FrontDesc d = t.fronts[list[blockIdx.y]];
    const int b = blockIdx.z;
    const int r = d.r, w = d.w;
    const int64_t nt = (r + 63) / 64;
    const int64_t tile = blockIdx.x;
    if (tile >= nt * (nt + 1) / 2) return;
    int64_t ti = (int64_t)((sqrt(8.0 * (double)tile + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > tile) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
    const int64_t tj = tile - ti * (ti + 1) / 2;
    const int i0 = (int)ti * 64, j0 = (int)tj * 64;
    __shared__ int32_t si[8][64], sj[8][64];
    __shared__ int64_t soff[8];
    __shared__ int32_t sld[8];
    const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
    const int i = i0 + tx;
    T acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = T(0);
    for (int cb = 0; cb < d.nchild; cb += 8) {
        const int nc = min(8, d.nchild - cb);
        if (cb > 0) __syncthreads();
        for (int e = tid; e < nc * 64; e += 256) {
            const int c = e >> 6, k = e & 63;
            const int32_t* inv = t.invmap + d.inv_off + (int64_t)(cb + c) * r;
            si[c][k] = i0 + k < r ? inv[i0 + k] : -1;
            sj[c][k] = j0 + k < r ? inv[j0 + k] : -1;
        }
        if (tid < nc) {
            const FrontDesc cd = t.fronts[t.child_ids[d.child_off + cb + tid]];
            soff[tid] = (int64_t)b * upd_total + cd.upd_off;
            sld[tid] = cd.r - cd.w;
        }
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
            const int a = si[c][tx];
            if (a < 0) continue;
            const T* U = upd + soff[c] + a;
            const int64_t rc = sld[c];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int bb = sj[c][ty + 4 * q];
                if (bb >= 0 && bb <= a) acc[q] += U[(int64_t)bb * rc];
            }
        }
    }
    if (i >= r) return;
    T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    T* Ub = upd + (int64_t)b * upd_total + d.upd_off;
    const int ru = r - w;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int j = j0 + ty + 4 * q;
        if (j > i) continue;
        if (j < w)
            Pb[(int64_t)j * r + i] = acc[q];
        else
            Ub[(int64_t)(j - w) * ru + (i - w)] = acc[q];
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_big_kscatter(const DevTables t, const int32_t* __restrict__ list,
                                                      const double* __restrict__ K, int64_t nnzK,
                                                      T* __restrict__ panel, int64_t panel_total) {
    const FrontDesc d = t.fronts[list[blockIdx.y]];
    const int b = blockIdx.z;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= d.klist_n) return;
    const int32_t* kl = t.klist + 2 * (d.klist_off + q);
    panel[(int64_t)b * panel_total + d.panel_off + kl[1]] += (T)K[(int64_t)b * nnzK + kl[0]];
}

// Tile (i0, j0) of a big-front update F[i, j] -= sum_{k0 <= l < k1} L[i, l] L[j, l]
// over rows jlo <= i < r and columns jlo <= j < jhi, j <= i, with
// k1 = min(k0 + nk, w), jlo = k1 and jhi = r (jend < 0: the whole trailing
// triangle, tiles enumerated row by row over the lower triangle) or
// jhi = min(jend, w) (the rest of the current panel block: a narrow
// trapezoid, tiles enumerated on its row x column grid).  Returns false for
// CTAs without a tile of this front.
__device__ __forceinline__ bool big_update_tile(int r, int w, int k0, int nk, int jend, int ts, int64_t tile,
                                                int& k1, int& jhi, int& i0, int& j0) {
    if (k0 >= w) return false;
    k1 = min(k0 + nk, w);
    const int jlo = k1;
    jhi = jend < 0 ? r : min(jend, w);
    if (jhi <= jlo) return false;
    const int64_t nrt = (r - jlo + ts - 1) / ts;
    int64_t ti, tj;
    if (jend < 0) {
        if (tile >= nrt * (nrt + 1) / 2) return false;
        ti = (int64_t)((sqrt(8.0 * (double)tile + 1.0) - 1.0) * 0.5);
        while (ti * (ti + 1) / 2 > tile) --ti;
        while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
        tj = tile - ti * (ti + 1) / 2;
    } else {
        const int64_t nct = (jhi - jlo + ts - 1) / ts;
        if (tile >= nrt * nct) return false;
        ti = tile / nct;
        tj = tile % nct;
        if (tj > ti) return false;
    }
    i0 = jlo + (int)ti * ts;
    j0 = jlo + (int)tj * ts;
    return true;
}

// Operand blocks of the tensor-core updates (FP32 factor).  The rows of
// the current panel block [C0, C0 + big_panel) of a big front are kept, per
// absolute 128-row tile t (rows 128 t ..) and 16-column chunk c (columns
// C0 + 16 c ..), as a 16 KB block: the TF32 high parts (x rounded to TF32)
// then the low parts (x - hi), each a 128 x 16 K-major tile of 8-row x
// 16-byte core matrices: float4 group g = 128 (k / 4) + (m % 128) at byte
// 16 g holds columns 4 (k / 4) .. + 3 of row m.  Block (t, c) of front q
// starts at float tc_off(q) + t kTcTileFloats + 4096 c of the instance's
// pack.  k_big_trsm writes them as it finishes each 32-column step; rows it
// has not written hold stale values that only reach masked outputs.
__device__ __forceinline__ float* tc_block(float* pack, int64_t pack_total, const FrontDesc& d, int b, int row,
                                           int chunk) {
    return pack + (int64_t)b * pack_total + d.tc_off + (int64_t)(row >> 7) * kTcTileFloats + (int64_t)chunk * 4096;
}

// Tile (i0, j0) (multiples of 128) of a tensor-core update; same update as
// big_update_tile, on the absolute 128-row grid of the operand blocks.
__device__ __forceinline__ bool tc_update_tile(int r, int w, int k0, int nk, int jend, int64_t tile, int& k1,
                                               int& jlo, int& jhi, int& i0, int& j0) {
    if (k0 >= w) return false;
    k1 = min(k0 + nk, w);
    jlo = k1;
    jhi = jend < 0 ? r : min(jend, w);
    if (jhi <= jlo) return false;
    const int t0 = jlo >> 7;
    const int64_t nrt = (r + 127) / 128 - t0;
    int64_t ti, tj;
    if (jend < 0) {
        if (tile >= nrt * (nrt + 1) / 2) return false;
        ti = (int64_t)((sqrt(8.0 * (double)tile + 1.0) - 1.0) * 0.5);
        while (ti * (ti + 1) / 2 > tile) --ti;
        while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
        tj = tile - ti * (ti + 1) / 2;
    } else {
        const int64_t nct = (jhi + 127) / 128 - t0;
        if (tile >= nrt * nct) return false;
        ti = tile / nct;
        tj = tile % nct;
        if (tj > ti) return false;
    }
    i0 = (t0 + (int)ti) * 128;
    j0 = (t0 + (int)tj) * 128;
    return true;
}

// Tensor-core trailing update (FP32 factor), the dense contraction of a big
// front: one CTA per 128x128 tile of the trailing lower triangle (see
// big_update_tile, jend < 0), two CTAs per SM.  Warp 8 lane 0 streams the
// tile's operand blocks (k_tc_pack) into a 3-stage shared-memory ring with
// bulk asynchronous copies and issues tcgen05.mma kind::tf32 on each landed
// chunk: hi*hi' + hi*lo' + lo*hi' accumulated in 128 tensor-memory columns
// (FP32-level accuracy from three TF32 products); each MMA commit frees its
// stage.  Warps 0-7 hold the epilogue: warp w reads tensor-memory lanes
// 32 (w % 4).. and columns 64 (w / 4)..+63 in two halves and subtracts
// them from the front, the first half's old values loaded before the wait.
// Every wait is bounded; on expiry the kernel raises *dev_err, drains its
// copies and MMAs (bounded), skips the update and frees its tensor memory.
constexpr int kTcStages = 3;
constexpr int kTcStageBytes = 32768;  // A block 16 KB + B block 16 KB
constexpr int kTcSmem = kTcStages * kTcStageBytes + 128;
constexpr uint32_t kTcWaitPolls = 1u << 24;

__global__ void __launch_bounds__(288, 2) k_big_update_tc(const DevTables t, const int32_t* __restrict__ list,
                                                          int kpack0, int k0, int nk, int jend,
                                                          const float* __restrict__ pack,
                                                          int64_t pack_total, float* __restrict__ panel,
                                                          int64_t panel_total, float* __restrict__ upd,
                                                          int64_t upd_total, int32_t* __restrict__ dev_err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const FrontDesc d = t.fronts[list[blockIdx.y]];
    const int b = blockIdx.z;
    const int r = d.r, w = d.w;
    if (d.tc_off < 0) return;
    int k1, jlo, jhi, i0, j0;
    if (!tc_update_tile(r, w, k0, nk, jend, blockIdx.x, k1, jlo, jhi, i0, j0)) return;
    const bool diag = i0 == j0;
    const int cfirst = (k0 - kpack0) >> 4;
    const float* pk = pack + (int64_t)b * pack_total + d.tc_off + (int64_t)cfirst * 4096;
    const float* Ablk = pk + (int64_t)(i0 >> 7) * kTcTileFloats;
    const float* Bblk = pk + (int64_t)(j0 >> 7) * kTcTileFloats;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + kTcStages * kTcStageBytes);
    uint64_t* empty = full + kTcStages;
    uint64_t* accb = empty + kTcStages;
    uint32_t* slot = reinterpret_cast<uint32_t*>(accb + 1);
    volatile int32_t* abort_flag = reinterpret_cast<volatile int32_t*>(slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nq = (k1 - k0 + 15) / 16;
    if (warp == 8) {
        tc::tmem_alloc(slot, 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(accb, 1);
        *abort_flag = 0;
        tc::mbar_init_fence();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *slot;
    const int ru = r - w;
    float* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    float* Ub = upd + (int64_t)b * upd_total + d.upd_off;
    if (warp == 8) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(128, 128);
            const uint32_t lbo = 16 * 128, sbo = 128;
            const uint32_t bytes = diag ? 16384u : 32768u;
            bool ok = true;
            int issued = 0, consumed = 0;
            for (int c = 0; c < nq + kTcStages - 1; ++c) {
                const int cm = c - (kTcStages - 1);
                if (cm >= 0) {
                    const int s = cm % kTcStages;
                    if (!tc::mbar_wait(&full[s], (uint32_t)(cm / kTcStages) & 1u, kTcWaitPolls)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const unsigned char* ah = smem_raw + s * kTcStageBytes;
                    const unsigned char* al = ah + 8192;
                    const unsigned char* bh = diag ? ah : ah + 16384;
                    const unsigned char* bl = diag ? al : ah + 24576;
#pragma unroll
                    for (int s8 = 0; s8 < 2; ++s8) {
                        const uint32_t koff = (uint32_t)s8 * 2 * lbo;
                        const uint64_t dah = tc::smem_desc_kmajor(ah + koff, lbo, sbo);
                        const uint64_t dal = tc::smem_desc_kmajor(al + koff, lbo, sbo);
                        const uint64_t dbh = tc::smem_desc_kmajor(bh + koff, lbo, sbo);
                        const uint64_t dbl = tc::smem_desc_kmajor(bl + koff, lbo, sbo);
                        tc::mma_tf32(taddr, dah, dbh, idesc, (cm > 0 || s8 > 0) ? 1u : 0u);
                        tc::mma_tf32(taddr, dah, dbl, idesc, 1u);
                        tc::mma_tf32(taddr, dal, dbh, idesc, 1u);
                    }
                    tc::mma_commit(&empty[s]);
                    consumed = cm + 1;
                }
                if (c < nq) {
                    const int s = c % kTcStages;
                    if (c >= kTcStages &&
                        !tc::mbar_wait(&empty[s], (uint32_t)(c / kTcStages - 1) & 1u, kTcWaitPolls)) {
                        ok = false;
                        break;
                    }
                    unsigned char* st = smem_raw + s * kTcStageBytes;
                    tc::mbar_arrive_expect_tx(&full[s], bytes);
                    tc::bulk_g2s(st, Ablk + (int64_t)c * 4096, 16384u, &full[s]);
                    if (!diag) tc::bulk_g2s(st + 16384, Bblk + (int64_t)c * 4096, 16384u, &full[s]);
                    issued = c + 1;
                }
            }
            if (ok) {
                tc::mma_commit(accb);
            } else {
                atomicExch(dev_err, 1);
                *abort_flag = 1;
                for (int cm = consumed; cm < issued; ++cm)
                    tc::mbar_wait(&full[cm % kTcStages], (uint32_t)(cm / kTcStages) & 1u, kTcWaitPolls);
                if (consumed > 0)
                    tc::mbar_wait(&empty[(consumed - 1) % kTcStages],
                                  (uint32_t)((consumed - 1) / kTcStages) & 1u, kTcWaitPolls);
                tc::mbar_arrive(accb);
            }
        }
        __syncwarp();
    } else {
        const int lq = warp & 3, ch = warp >> 2;
        const int i = i0 + 32 * lq + lane;
        bool ok = true;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int jb = j0 + 64 * ch + 32 * h;
            float cv[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int j = jb + c;
                cv[c] = 0.f;
                if (i < r && j <= i && j >= jlo && j < jhi)
                    cv[c] = j < w ? Pb[(int64_t)j * r + i] : Ub[(int64_t)(j - w) * ru + (i - w)];
            }
            if (h == 0) {
                if (!tc::mbar_wait(accb, 0, kTcWaitPolls)) {
                    ok = false;
                    if (lane == 0) atomicExch(dev_err, 1);
                }
                ok = __all_sync(0xffffffffu, ok && *abort_flag == 0);
                tc::fence_after_sync();
            }
            if (!ok) break;
            float v[4][8];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                tc::tmem_ld8(taddr + ((uint32_t)(32 * lq) << 16) + (uint32_t)(64 * ch + 32 * h + 8 * c), v[c]);
            tc::tmem_ld_wait();
            if (i < r) {
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int j = jb + c;
                    if (j <= i && j >= jlo && j < jhi) {
                        if (j < w)
                            Pb[(int64_t)j * r + i] = cv[c] - v[c >> 3][c & 7];
                        else
                            Ub[(int64_t)(j - w) * ru + (i - w)] = cv[c] - v[c >> 3][c & 7];
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 8) tc::tmem_dealloc(taddr, 128);
}

// Persistent tensor-core trailing update (FP32 factor, jend < 0): one CTA
// per SM walks the launch's work items -- (tile pair, front, value set),
// pair p of a front = row tile ti and the two column tiles 2tp, 2tp+1 of
// the trailing lower triangle on the absolute 128-row grid -- so that
// (a) the pair shares its A operand (one A block feeds two 128x128 MMAs),
// (b) operand chunks stream through a 4-stage ring continuously across
// items, and (c) two TMEM accumulators of 256 columns let the epilogue of
// item v run while the tensor core works on item v+1.  Warp 8 lane 0 loads
// (bulk copies into the ring) and issues MMAs; warps 0-3 (columns of the
// first tile) and 4-7 (second tile) run the epilogue.  Barriers: full/empty
// per stage, accfull (MMA commit) and accempty (8 epilogue warps) per
// accumulator.  Every wait is bounded and also gives up when another role
// has raised the CTA's abort flag; on expiry the kernel raises *dev_err,
// drains what it issued and frees its tensor memory.
constexpr int kTcpStages = 4;
constexpr int kTcpStageBytes = 49152;  // A, B0, B1 blocks of 16 KB
constexpr int kTcpSmem = kTcpStages * kTcpStageBytes + 256;
constexpr uint32_t kTcpPolls = 1u << 22;

struct TcpItem {
    bool valid;
    int r, w, k1, jlo, ti, tj0, tj1;  // tile indices absolute (x 128 rows)
    bool two;                          // second column tile inside the triangle
    int64_t panel_off, upd_off, tc_off;
    int b;
};

// Pairs of one front's trailing triangle with nrt row tiles: row tile ti
// holds ti / 2 + 1 pairs; pairs of row tiles 2u and 2u + 1 start at u(u+1).
__host__ __device__ inline int64_t tcp_pairs(int64_t nrt) {
    const int64_t U = nrt / 2, e = nrt & 1;
    return U * (U + 1) + e * (U + 1);
}

__device__ __forceinline__ TcpItem tcp_item(const DevTables& t, const int32_t* list, int count, int64_t npairs,
                                            int k0, int nk, int64_t it) {
    TcpItem x;
    x.valid = false;
    const int64_t p = it % npairs;
    const int q = (int)((it / npairs) % count);
    x.b = (int)(it / (npairs * count));
    const FrontDesc d = t.fronts[list[q]];
    if (d.tc_off < 0 || k0 >= d.w) return x;
    x.r = d.r;
    x.w = d.w;
    x.k1 = min(k0 + nk, d.w);
    x.jlo = x.k1;
    if (x.jlo >= d.r) return x;
    const int t0 = x.jlo >> 7;
    const int64_t nrt = (d.r + 127) / 128 - t0;
    if (p >= tcp_pairs(nrt)) return x;
    int64_t u = (int64_t)((sqrt(4.0 * (double)p + 1.0) - 1.0) * 0.5);
    while (u * (u + 1) > p) --u;
    while ((u + 1) * (u + 2) <= p) ++u;
    const int64_t rem = p - u * (u + 1);
    const int64_t ti = 2 * u + rem / (u + 1), tp = rem % (u + 1);
    if (ti >= nrt) return x;
    x.ti = t0 + (int)ti;
    x.tj0 = t0 + 2 * (int)tp;
    x.tj1 = x.tj0 + 1;
    x.two = 2 * tp + 1 <= ti;
    x.panel_off = d.panel_off;
    x.upd_off = d.upd_off;
    x.tc_off = d.tc_off;
    x.valid = true;
    return x;
}

__global__ void __launch_bounds__(288, 1) k_big_update_tcp(const DevTables t, const int32_t* __restrict__ list,
                                                           int32_t count, int32_t B, int64_t npairs, int k0, int nk,
                                                           const float* __restrict__ pack, int64_t pack_total,
                                                           float* __restrict__ panel, int64_t panel_total,
                                                           float* __restrict__ upd, int64_t upd_total,
                                                           int32_t* __restrict__ dev_err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + kTcpStages * kTcpStageBytes);
    uint64_t* empty = full + kTcpStages;
    uint64_t* accfull = empty + kTcpStages;
    uint64_t* accempty = accfull + 2;
    uint32_t* slot = reinterpret_cast<uint32_t*>(accempty + 2);
    volatile int32_t* abort_flag = reinterpret_cast<volatile int32_t*>(slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t items = npairs * count * B;
    if (warp == 8) {
        tc::tmem_alloc(slot, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kTcpStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&accfull[a], 1);
            tc::mbar_init(&accempty[a], 8);
        }
        *abort_flag = 0;
        tc::mbar_init_fence();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *slot;
    if (warp == 8) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(128, 128);
            const uint32_t lbo = 16 * 128, sbo = 128;
            // load cursor and MMA cursor over the same (item, chunk) sequence
            int64_t itl = blockIdx.x, itm = blockIdx.x;
            TcpItem xl = itl < items ? tcp_item(t, list, count, npairs, k0, nk, itl) : TcpItem{};
            TcpItem xm = xl;
            int cl = 0, cm = 0, vm = 0;
            int64_t gl = 0, gm = 0;
            bool ok = true;
            auto next_valid = [&](int64_t& it, TcpItem& x) {
                while (it < items) {
                    x = tcp_item(t, list, count, npairs, k0, nk, it);
                    if (x.valid) return;
                    it += gridDim.x;
                }
                x.valid = false;
            };
            if (itl < items && !xl.valid) {
                next_valid(itl, xl);
                xm = xl;
                itm = itl;
            }
            while (ok && itm < items && xm.valid) {
                // loads run up to kTcpStages chunks ahead of the MMAs
                while (itl < items && xl.valid && gl < gm + kTcpStages) {
                    const int st = (int)(gl % kTcpStages);
                    if (gl >= kTcpStages &&
                        !tc::mbar_wait_abort(&empty[st], (uint32_t)((gl / kTcpStages) - 1) & 1u, kTcpPolls,
                                             abort_flag)) {
                        ok = false;
                        break;
                    }
                    unsigned char* sb = smem_raw + st * kTcpStageBytes;
                    const float* pk = pack + (int64_t)xl.b * pack_total + xl.tc_off + (int64_t)cl * 4096;
                    tc::mbar_arrive_expect_tx(&full[st], xl.two ? 49152u : 32768u);
                    tc::bulk_g2s(sb, pk + (int64_t)xl.ti * kTcTileFloats, 16384u, &full[st]);
                    tc::bulk_g2s(sb + 16384, pk + (int64_t)xl.tj0 * kTcTileFloats, 16384u, &full[st]);
                    if (xl.two) tc::bulk_g2s(sb + 32768, pk + (int64_t)xl.tj1 * kTcTileFloats, 16384u, &full[st]);
                    ++gl;
                    if (++cl == (xl.k1 - k0 + 15) / 16) {
                        cl = 0;
                        itl += gridDim.x;
                        next_valid(itl, xl);
                    }
                }
                if (!ok) break;
                const int st = (int)(gm % kTcpStages);
                const int buf = vm & 1;
                if (!tc::mbar_wait_abort(&full[st], (uint32_t)(gm / kTcpStages) & 1u, kTcpPolls, abort_flag)) {
                    ok = false;
                    break;
                }
                if (cm == 0 && vm >= 2 &&
                    !tc::mbar_wait_abort(&accempty[buf], (uint32_t)((vm >> 1) - 1) & 1u, kTcpPolls, abort_flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const unsigned char* ah = smem_raw + st * kTcpStageBytes;
                const uint32_t d0 = taddr + (uint32_t)(buf * 256), d1 = d0 + 128;
#pragma unroll
                for (int s8 = 0; s8 < 2; ++s8) {
                    const uint32_t koff = (uint32_t)s8 * 2 * lbo;
                    const uint64_t dah = tc::smem_desc_kmajor(ah + koff, lbo, sbo);
                    const uint64_t dal = tc::smem_desc_kmajor(ah + 8192 + koff, lbo, sbo);
                    const uint64_t b0h = tc::smem_desc_kmajor(ah + 16384 + koff, lbo, sbo);
                    const uint64_t b0l = tc::smem_desc_kmajor(ah + 24576 + koff, lbo, sbo);
                    const uint32_t acc = (cm > 0 || s8 > 0) ? 1u : 0u;
                    tc::mma_tf32(d0, dah, b0h, idesc, acc);
                    tc::mma_tf32(d0, dah, b0l, idesc, 1u);
                    tc::mma_tf32(d0, dal, b0h, idesc, 1u);
                    if (xm.two) {
                        const uint64_t b1h = tc::smem_desc_kmajor(ah + 32768 + koff, lbo, sbo);
                        const uint64_t b1l = tc::smem_desc_kmajor(ah + 40960 + koff, lbo, sbo);
                        tc::mma_tf32(d1, dah, b1h, idesc, acc);
                        tc::mma_tf32(d1, dah, b1l, idesc, 1u);
                        tc::mma_tf32(d1, dal, b1h, idesc, 1u);
                    }
                }
                tc::mma_commit(&empty[st]);
                ++gm;
                if (++cm == (xm.k1 - k0 + 15) / 16) {
                    tc::mma_commit(&accfull[buf]);
                    cm = 0;
                    ++vm;
                    itm += gridDim.x;
                    next_valid(itm, xm);
                }
            }
            if (!ok) {
                atomicExch(dev_err, 1);
                *abort_flag = 1;
                // copies issued but not consumed, then the last MMAs
                for (int64_t g = gm; g < gl; ++g)
                    tc::mbar_wait(&full[g % kTcpStages], (uint32_t)(g / kTcpStages) & 1u, kTcpPolls);
                if (gm > 0)
                    tc::mbar_wait(&empty[(gm - 1) % kTcpStages], (uint32_t)((gm - 1) / kTcpStages) & 1u,
                                  kTcpPolls);
            }
        }
        __syncwarp();
    } else {
        // epilogue: warps 0-3 the first column tile, 4-7 the second
        const int lq = warp & 3, half = warp >> 2;
        int64_t it = blockIdx.x;
        int v = 0;
        while (it < items) {
            const TcpItem x = tcp_item(t, list, count, npairs, k0, nk, it);
            it += gridDim.x;
            if (!x.valid) continue;
            const int buf = v & 1;
            const bool mine = half == 0 || x.two;
            const int i = x.ti * 128 + 32 * lq + lane;
            const int j0 = (half == 0 ? x.tj0 : x.tj1) * 128;
            float* Pb = panel + (int64_t)x.b * panel_total + x.panel_off;
            float* Ub = upd + (int64_t)x.b * upd_total + x.upd_off;
            const int r = x.r, w = x.w, ru = r - w, jlo = x.jlo;
            float cv[32];
            if (mine) {
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int j = j0 + c;
                    cv[c] = 0.f;
                    if (i < r && j <= i && j >= jlo)
                        cv[c] = j < w ? Pb[(int64_t)j * r + i] : Ub[(int64_t)(j - w) * ru + (i - w)];
                }
            }
            bool got = tc::mbar_wait_abort(&accfull[buf], (uint32_t)(v >> 1) & 1u, kTcpPolls, abort_flag);
            got = __all_sync(0xffffffffu, got);
            if (!got) {
                if (lane == 0) {
                    atomicExch(dev_err, 1);
                    *abort_flag = 1;
                }
                break;
            }
            tc::fence_after_sync();
            if (mine) {
#pragma unroll 1
                for (int h = 0; h < 4; ++h) {
                    const int jb = j0 + 32 * h;
                    if (h > 0) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const int j = jb + c;
                            cv[c] = 0.f;
                            if (i < r && j <= i && j >= jlo)
                                cv[c] = j < w ? Pb[(int64_t)j * r + i] : Ub[(int64_t)(j - w) * ru + (i - w)];
                        }
                    }
                    float vv[4][8];
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        tc::tmem_ld8(taddr + ((uint32_t)(32 * lq) << 16) +
                                         (uint32_t)(buf * 256 + half * 128 + 32 * h + 8 * c),
                                     vv[c]);
                    tc::tmem_ld_wait();
                    if (i < r) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const int j = jb + c;
                            if (j <= i && j >= jlo) {
                                if (j < w)
                                    Pb[(int64_t)j * r + i] = cv[c] - vv[c >> 3][c & 7];
                                else
                                    Ub[(int64_t)(j - w) * ru + (i - w)] = cv[c] - vv[c >> 3][c & 7];
                            }
                        }
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&accempty[buf]);
            ++v;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 8) tc::tmem_dealloc(taddr, 512);
}

// Factor the 32x32 diagonal block of column block kb, one warp per front,
// lane i holding row i in registers.  Compact form: at step j the pivot
// column is always a[0] (the row's registers shift left by one per step), so
// the step loop is a runtime loop and only its 31-wide body is unrolled --
// a few hundred instructions instead of a fully unrolled 32 x 32 nest, which
// a one-warp launch would otherwise spend fetching.  Its own launch: the
// triangular solve below must read the factored block, and no CTA of one
// launch may overwrite what another CTA still has to load.
// Fused 32-column steps of a big front (k_big_trsm given a scratch area): every CTA
// of the step factors the step's 32 x 32 diagonal block itself (one warp,
// in shared memory) from the values in the panel, so the step needs no
// separate potrf launch; the panel's copy of the block is not overwritten
// during the step (other CTAs are still reading it) -- CTA 0 of each
// (front, value set) leaves the factored block in a scratch slot, and the
// next step's kernel (fused or k_big_potrf) writes it into the panel.
template <class T>
__device__ __forceinline__ void diag_copy_back(const T* __restrict__ Db, T* __restrict__ Pb, int r, int w, int pc,
                                               int tid, int nth) {
    const int nb = min(32, w - pc);
    for (int e = tid; e < 1024; e += nth) {
        const int i = e & 31, j = e >> 5;
        if (i < nb && j <= i) Pb[(int64_t)(pc + j) * r + pc + i] = Db[j * 32 + i];
    }
}

template <class T>
__global__ void __launch_bounds__(32) k_big_potrf(const DevTables t, const int32_t* __restrict__ list, int kb,
                                                  T* __restrict__ panel, int64_t panel_total,
                                                  int32_t* __restrict__ bad_col, int32_t n_pats,
                                                  const T* __restrict__ diag) {
    const FrontDesc d = t.fronts[list[blockIdx.x]];
    const int b = blockIdx.y;
    const int r = d.r, w = d.w;
    const int c0 = kb * 32;
    if (diag && kb >= 1 && c0 - 32 < w)
        diag_copy_back(diag + ((int64_t)b * gridDim.x + blockIdx.x) * 1024,
                       panel + (int64_t)b * panel_total + d.panel_off, r, w, c0 - 32, threadIdx.x, 32);
    if (c0 >= w) return;
    const int nbk = min(32, w - c0);
    T* Pb = panel + (int64_t)b * panel_total + d.panel_off + (int64_t)c0 * r + c0;
    const int i = threadIdx.x;
    T a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) a[k] = (i < nbk && k < nbk && k <= i) ? Pb[(int64_t)k * r + i] : T(0);
    bool failed = false;
#pragma unroll 1
    for (int j = 0; j < nbk; ++j) {
        T djj = __shfl_sync(0xffffffffu, a[0], j);
        if (!(djj > T(0))) {
            if (i == 0 && !failed)
                atomicMin(&bad_col[(int64_t)b * n_pats + d.sys], d.f + c0 + j - (int)t.sys_n_off[d.sys]);
            failed = true;
            djj = T(1);
        }
        const T ljj = sqrt(djj);
        if (i == j)
            a[0] = ljj;
        else if (i > j)
            a[0] /= ljj;
        if (i >= j && i < nbk) Pb[(int64_t)j * r + i] = a[0];
#pragma unroll
        for (int k = 1; k < 32; ++k) {
            const T lkj = __shfl_sync(0xffffffffu, a[0], (j + k) & 31);
            if (i >= j + k) a[k] -= a[0] * lkj;
        }
#pragma unroll
        for (int k = 0; k < 31; ++k) a[k] = a[k + 1];
        a[31] = T(0);
    }
}

// Rows below the diagonal block of column block kb: X = P[rows, blk] L_kk^{-T},
// 256 rows per CTA, one row per thread.
template <class T>
__global__ void __launch_bounds__(256) k_big_trsm(const DevTables t, const int32_t* __restrict__ list, int kb,
                                                  T* __restrict__ panel, int64_t panel_total,
                                                  float* __restrict__ pack, int64_t pack_total, int kpack0,
                                                  T* __restrict__ diag, int32_t* __restrict__ bad_col,
                                                  int32_t n_pats) {
    const FrontDesc d = t.fronts[list[blockIdx.y]];
    const int b = blockIdx.z;
    const int r = d.r, w = d.w;
    const int c0 = kb * 32;
    const int tid = threadIdx.x;
    T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    T* Db = diag ? diag + ((int64_t)b * gridDim.y + blockIdx.y) * 1024 : nullptr;
    if (Db && blockIdx.x == 0 && kb >= 1 && c0 - 32 < w) {
        diag_copy_back(Db, Pb, r, w, c0 - 32, tid, 256);
        __syncthreads();  // the slot is rewritten below
    }
    if (c0 >= w) return;
    const int nbk = min(32, w - c0);
    const int rbeg = c0 + nbk + (int)blockIdx.x * 256;
    if (!Db && rbeg >= r) return;
    __shared__ T Ld[32][33];
    if (Db) {
        // factor the diagonal block (the arithmetic of k_big_potrf)
        if (tid < 32) {
            const int i = tid;
            const T* Pd = Pb + (int64_t)c0 * r + c0;
            T a[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) a[k] = (i < nbk && k < nbk && k <= i) ? Pd[(int64_t)k * r + i] : T(0);
            bool failed = false;
#pragma unroll 1
            for (int j = 0; j < nbk; ++j) {
                T djj = __shfl_sync(0xffffffffu, a[0], j);
                if (!(djj > T(0))) {
                    if (i == 0 && !failed && blockIdx.x == 0)
                        atomicMin(&bad_col[(int64_t)b * n_pats + d.sys], d.f + c0 + j - (int)t.sys_n_off[d.sys]);
                    failed = true;
                    djj = T(1);
                }
                const T ljj = sqrt(djj);
                if (i == j)
                    a[0] = ljj;
                else if (i > j)
                    a[0] /= ljj;
                if (i >= j && i < nbk) Ld[i][j] = a[0];
#pragma unroll
                for (int k = 1; k < 32; ++k) {
                    const T lkj = __shfl_sync(0xffffffffu, a[0], (j + k) & 31);
                    if (i >= j + k) a[k] -= a[0] * lkj;
                }
#pragma unroll
                for (int k = 0; k < 31; ++k) a[k] = a[k + 1];
                a[31] = T(0);
            }
            for (int j = 0; j < 32; ++j)
                if (!(i < nbk && j <= i)) Ld[i][j] = T(1);
        }
        __syncthreads();
        if (blockIdx.x == 0)
            for (int e = tid; e < 1024; e += 256) {
                const int i = e & 31, j = e >> 5;
                if (i < nbk && j <= i) Db[j * 32 + i] = Ld[i][j];
            }
        if (rbeg >= r) return;
    } else {
        for (int e = tid; e < 32 * 32; e += 256) {
            const int i = e & 31, j = e >> 5;
            Ld[i][j] = (i < nbk && j <= i) ? Pb[(int64_t)(c0 + j) * r + c0 + i] : T(1);
        }
        __syncthreads();
    }
    const int row = rbeg + tid;
    if (row >= r) return;
    T x[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = j < nbk ? Pb[(int64_t)(c0 + j) * r + row] : T(0);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (j < nbk) {
            T s = x[j];
#pragma unroll
            for (int l = 0; l < j; ++l) s -= x[l] * Ld[j][l];
            x[j] = s / Ld[j][j];
        }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j)
        if (j < nbk) Pb[(int64_t)(c0 + j) * r + row] = x[j];
    if (sizeof(T) == 4 && pack && d.tc_off >= 0) {
        // The step's two 16-column operand chunks for the tensor-core
        // updates (columns past nbk are zero).
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float* blk = tc_block(pack, pack_total, d, b, row, ((c0 - kpack0) >> 4) + h);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float4 hi, lo;
                float* ph = &hi.x;
                float* pl = &lo.x;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float xv = (float)x[16 * h + 4 * q + u];
                    ph[u] = tc::to_tf32(xv);
                    pl[u] = xv - ph[u];
                }
                const int g = 128 * q + (row & 127);
                reinterpret_cast<float4*>(blk)[g] = hi;
                reinterpret_cast<float4*>(blk + 2048)[g] = lo;
            }
        }
    }
}

// SIMT update of a big front (FP64, or FP32 without tensor cores): the
// update of big_update_tile, CTA tile 64x64, 256 threads with 4x4 each,
// the inner dimension k1 - k0 consumed in 32-column shared-memory chunks.
template <class T>
__global__ void __launch_bounds__(256) k_big_update(const DevTables t, const int32_t* __restrict__ list, int k0,
                                                    int nk, int jend, T* __restrict__ panel, int64_t panel_total,
                                                    T* __restrict__ upd, int64_t upd_total) {
    const FrontDesc d = t.fronts[list[blockIdx.y]];
    const int b = blockIdx.z;
    const int r = d.r, w = d.w;
    int k1, jhi, i0, j0;
    if (!big_update_tile(r, w, k0, nk, jend, 64, blockIdx.x, k1, jhi, i0, j0)) return;
    T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    T* Ub = upd + (int64_t)b * upd_total + d.upd_off;
    const int ru = r - w;
    __shared__ T As[32][64 + 1];
    __shared__ T Bs[32][64 + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
    for (int kc = k0; kc < k1; kc += 32) {
        const int nbk = min(32, k1 - kc);
        if (kc > k0) __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = tid + q * 256;
            const int mm = e & 63, kk = e >> 6;
            const int ra = i0 + mm, rb = j0 + mm;
            As[kk][mm] = (ra < r && kk < nbk) ? Pb[(int64_t)(kc + kk) * r + ra] : T(0);
            Bs[kk][mm] = (rb < r && kk < nbk) ? Pb[(int64_t)(kc + kk) * r + rb] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            T a[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][tx + 16 * q];
                bv[q] = Bs[kk][ty + 16 * q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[q][p] += a[q] * bv[p];
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int j = j0 + ty + 16 * p;
        if (j >= jhi) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + tx + 16 * q;
            if (i >= r || i < j) continue;
            if (j < w)
                Pb[(int64_t)j * r + i] -= acc[q][p];
            else
                Ub[(int64_t)(j - w) * ru + (i - w)] -= acc[q][p];
        }
    }
}

// FP32 SIMT trailing update: CTA tile 128x128, 256 threads with 8x8 each
// (rows 4 + 4 and columns 4 + 4, read from shared memory as float4 with one
// wavefront per warp read), inner dimension in 16-column chunks, the next
// chunk's global loads in flight while the current one is multiplied.
__global__ void __launch_bounds__(256, 2) k_big_update_f32(const DevTables t, const int32_t* __restrict__ list,
                                                           int k0, int nk, int jend, float* __restrict__ panel,
                                                           int64_t panel_total, float* __restrict__ upd,
                                                           int64_t upd_total) {
    const FrontDesc d = t.fronts[list[blockIdx.y]];
    const int b = blockIdx.z;
    const int r = d.r, w = d.w;
    int k1, jhi, i0, j0;
    if (!big_update_tile(r, w, k0, nk, jend, 128, blockIdx.x, k1, jhi, i0, j0)) return;
    float* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    float* Ub = upd + (int64_t)b * upd_total + d.upd_off;
    const int ru = r - w;
    __shared__ __align__(16) float As[2][16][128];
    __shared__ __align__(16) float Bs[2][16][128];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ra0 = (warp & 1) * 64 + (lane & 7) * 4;   // rows ra0 + {0..3}, ra0 + 32 + {0..3}
    const int cb0 = (warp >> 1) * 32 + (lane >> 3) * 4;  // columns cb0 + {0..3}, cb0 + 16 + {0..3}
    const int lm = tid & 127, lk = tid >> 7;              // loader: row lm, chunk columns lk + 2u
    float la[8], lb[8];
    const bool ain = i0 + lm < r, bin = j0 + lm < r;
    auto gload = [&](int kc) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int kk = kc + lk + 2 * u;
            const bool kin = kk < k1;
            la[u] = (kin && ain) ? Pb[(int64_t)kk * r + i0 + lm] : 0.f;
            lb[u] = (kin && bin) ? Pb[(int64_t)kk * r + j0 + lm] : 0.f;
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            As[buf][lk + 2 * u][lm] = la[u];
            Bs[buf][lk + 2 * u][lm] = lb[u];
        }
    };
    float acc[8][8];
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = 0.f;
    const int nq = (k1 - k0 + 15) / 16;
    gload(k0);
    sstore(0);
    __syncthreads();
    for (int q = 0; q < nq; ++q) {
        const int buf = q & 1;
        if (q + 1 < nq) gload(k0 + 16 * (q + 1));
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ra0]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ra0 + 32]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][cb0]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][cb0 + 16]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int p = 0; p < 8; ++p)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[p][c] += a[p] * bv[c];
        }
        if (q + 1 < nq) sstore(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int j = j0 + cb0 + (c & 3) + 16 * (c >> 2);
        if (j >= jhi) continue;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const int i = i0 + ra0 + (p & 3) + 32 * (p >> 2);
            if (i >= r || i < j) continue;
            if (j < w)
                Pb[(int64_t)j * r + i] -= acc[p][c];
            else
                Ub[(int64_t)(j - w) * ru + (i - w)] -= acc[p][c];
        }
    }
}

// --------------------------------------------------------------------------
// a5: level-scheduled solves, one CTA per (front, instance).
// A front's vector for the forward sweep, by one warp: v[k] = own
// right-hand side (k < w) or 0, plus every child's passing vector through
// its relative map, children in order with a warp barrier between them
// (two children may reach the same row); each child's rows are loaded four
// chunks of 32 at a time before they are added.  CG: passing vectors
// written by other CTAs of the same launch are read past L1.
template <class T, bool CG>
__device__ __forceinline__ void gather_fwd(const DevTables& t, const FrontDesc& d, const T* __restrict__ vb,
                                           const T* __restrict__ pv, T* __restrict__ v, int lane) {
    const int r = d.r, w = d.w, nc = d.nchild;
    // lane c holds child c's descriptor (fetched in parallel, handed out by
    // shuffles), so a child costs no dependent descriptor loads in the loop
    long long my_pv = 0, my_map = 0;
    int my_rc = 0;
    if (lane < nc) {
        const FrontDesc& cd = t.fronts[t.child_ids[d.child_off + lane]];
        my_pv = cd.pvec_off;
        my_map = cd.relmap_off;
        my_rc = cd.r - cd.w;
    }
    for (int k = lane; k < r; k += 32) v[k] = k < w ? (CG ? __ldcg(vb + d.f + k) : vb[d.f + k]) : T(0);
    for (int c = 0; c < nc; ++c) {
        int rc;
        int64_t map_off, pv_off;
        if (c < 32) {
            rc = __shfl_sync(0xffffffffu, my_rc, c);
            map_off = __shfl_sync(0xffffffffu, my_map, c);
            pv_off = __shfl_sync(0xffffffffu, my_pv, c);
        } else {
            const FrontDesc& cd = t.fronts[t.child_ids[d.child_off + c]];
            rc = cd.r - cd.w;
            map_off = cd.relmap_off;
            pv_off = cd.pvec_off;
        }
        const int32_t* map = t.relmap + map_off;
        const T* src = pv + pv_off;
        __syncwarp();
        for (int k0 = 0; k0 < rc; k0 += 128) {
            int m[4];
            T x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + lane + 32 * u;
                m[u] = k < rc ? map[k] : -1;
                x[u] = k < rc ? (CG ? __ldcg(src + k) : src[k]) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (m[u] >= 0) v[m[u]] += x[u];
        }
    }
}

// A front's vector for the backward sweep, by one warp: its own columns'
// values and the (final) values at its other rows, up to 256 rows per batch
// of loads.  CG: values written by other CTAs of the same launch.
template <class T, bool CG>
__device__ __forceinline__ void gather_bwd(const FrontDesc& d, const int32_t* __restrict__ rows,
                                           const T* __restrict__ vb, T* __restrict__ v, int lane) {
    const int r = d.r, w = d.w;
    for (int k0 = 0; k0 < r; k0 += 256) {
        int idx[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + lane + 32 * u;
            idx[u] = k < w ? d.f + k : (k < r ? rows[k] : -1);
        }
        T x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = idx[u] >= 0 ? (CG ? __ldcg(vb + idx[u]) : vb[idx[u]]) : T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (k0 + lane + 32 * u < r) v[k0 + lane + 32 * u] = x[u];
    }
}

// --------------------------------------------------------------------------
// Stage the lower triangle of the 32x32 diagonal block starting at (jb, jb).
// and the reciprocals of its diagonal.
template <class T>
__device__ __forceinline__ void stage_diag(T (*Ld)[33], T* dinv, const T* __restrict__ Pb, int r, int jb, int nbk,
                                           int tid, int nth) {
    for (int e = tid; e < 32 * 32; e += nth) {
        const int i = e & 31, c = e >> 5;
        const T v = (i < nbk && c <= i) ? Pb[(int64_t)(jb + c) * r + jb + i] : T(0);
        Ld[i][c] = v;
        if (i == c) dinv[i] = i < nbk ? T(1) / v : T(0);
    }
}

template <class T>
__global__ void __launch_bounds__(512) k_fwd(const DevTables t, const int32_t* __restrict__ list,
                                             const T* __restrict__ panel, int64_t panel_total,
                                             T* __restrict__ vec, int64_t n, T* __restrict__ pvec,
                                             int64_t pvec_total, const int32_t* __restrict__ active,
                                             int32_t n_pats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* v = reinterpret_cast<T*>(smem_raw);
    __shared__ T Ld[2][32][33];
    __shared__ T dinv[2][32];
    __shared__ T yblk[32];
    const FrontDesc d = t.fronts[list[blockIdx.x]];
    const int b = blockIdx.y;
    if (active && !active[(int64_t)b * n_pats + d.sys]) return;
    const int r = d.r, w = d.w;
    const int tid = threadIdx.x, nth = blockDim.x;
    T* vb = vec + (int64_t)b * n;
    const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    T* pv = pvec + (int64_t)b * pvec_total;
    // the children's descriptors, fetched in parallel while the vector and
    // the first diagonal block are staged (instead of one dependent chain
    // per child inside the loop below)
    __shared__ ChildRef s_ch[kChildRefs];  // upd_off holds the child's passing-vector offset here
    if (tid < min(d.nchild, kChildRefs)) {
        const FrontDesc& cd = t.fronts[t.child_ids[d.child_off + tid]];
        s_ch[tid] = ChildRef{cd.pvec_off, cd.relmap_off, cd.r - cd.w, 0};
    }
    for (int k = tid; k < r; k += nth) v[k] = k < w ? vb[d.f + k] : T(0);
    stage_diag(Ld[0], dinv[0], Pb, r, 0, min(32, w), tid, nth);
    __syncthreads();
    // children's passing vectors: each thread's entry of the first four
    // children loaded together (one round trip), then added child by child
    const int nc4 = min(d.nchild, 4);
    int cm[4];
    T cx[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        cm[c] = -1;
        cx[c] = T(0);
        if (c < nc4 && tid < s_ch[c].rc) {
            cm[c] = t.relmap[s_ch[c].map_off + tid];
            cx[c] = pv[s_ch[c].upd_off + tid];
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (c >= nc4) break;
        if (c > 0) __syncthreads();  // two children may reach the same row
        if (cm[c] >= 0) v[cm[c]] += cx[c];
        for (int k = tid + nth; k < s_ch[c].rc; k += nth) v[t.relmap[s_ch[c].map_off + k]] += pv[s_ch[c].upd_off + k];
    }
    for (int c = 4; c < d.nchild; ++c) {
        __syncthreads();
        ChildRef cr;
        if (c < kChildRefs) {
            cr = s_ch[c];
        } else {
            const FrontDesc& cd = t.fronts[t.child_ids[d.child_off + c]];
            cr = ChildRef{cd.pvec_off, cd.relmap_off, cd.r - cd.w, 0};
        }
        const int32_t* map = t.relmap + cr.map_off;
        for (int k = tid; k < cr.rc; k += nth) v[map[k]] += pv[cr.upd_off + k];
    }
    __syncthreads();
    int buf = 0;
    for (int jb = 0; jb < w; jb += 32) {
        const int nbk = min(32, w - jb);
        // this thread's first row below the block: its panel entries are
        // loaded before the block's chain, so that the loads overlap it
        const int i0 = jb + nbk + tid;
        T pc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) pc[j] = (i0 < r && j < nbk) ? Pb[(int64_t)(jb + j) * r + i0] : T(0);
        if (tid < 32) {
            const int l = tid;
            T val = l < nbk ? v[jb + l] : T(0);
            for (int j = 0; j < nbk; ++j) {
                const T yj = __shfl_sync(0xffffffffu, val, j) * dinv[buf][j];
                if (l == j) val = yj;
                if (l > j) val -= Ld[buf][l][j] * yj;
            }
            if (l < nbk) v[jb + l] = val;
            yblk[l] = l < nbk ? val : T(0);  // zeros past the block: pc[j] * yblk[j] below must be 0 there
        } else if (jb + 32 < w) {
            stage_diag(Ld[buf ^ 1], dinv[buf ^ 1], Pb, r, jb + 32, min(32, w - jb - 32), tid - 32, nth - 32);
        }
        __syncthreads();
        if (i0 < r) {
            T acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = T(0);
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] += pc[j + u] * yblk[j + u];
            }
            v[i0] -= ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        }
        for (int i = i0 + nth; i < r; i += nth) {
            const T* col = Pb + (int64_t)jb * r + i;
            T acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = T(0);
            int j = 0;
            for (; j + 7 < nbk; j += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] += col[(int64_t)(j + u) * r] * yblk[j + u];
            }
            for (; j < nbk; ++j) acc[0] += col[(int64_t)j * r] * yblk[j];
            v[i] -= ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        }
        buf ^= 1;
        __syncthreads();
    }
    for (int k = tid; k < w; k += nth) vb[d.f + k] = v[k];
    for (int k = tid; k < r - w; k += nth) pv[d.pvec_off + k] = v[w + k];
}

template <class T>
__global__ void __launch_bounds__(512) k_bwd(const DevTables t, const int32_t* __restrict__ list,
                                             const T* __restrict__ panel, int64_t panel_total,
                                             T* __restrict__ vec, int64_t n, const int32_t* __restrict__ active,
                                             int32_t n_pats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* v = reinterpret_cast<T*>(smem_raw);
    __shared__ T Ld[2][32][33];
    __shared__ T dinv[2][32];
    __shared__ T dots[32];
    const FrontDesc d = t.fronts[list[blockIdx.x]];
    const int b = blockIdx.y;
    if (active && !active[(int64_t)b * n_pats + d.sys]) return;
    const int r = d.r, w = d.w;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
    T* vb = vec + (int64_t)b * n;
    const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    const int32_t* rows = t.rows + d.rows_off;
    const int nblk = (w + 31) / 32;
    // the last diagonal block staged with the vector; each later block is
    // staged by warps 1.. while warp 0 runs the current block's chain
    int buf = 0;
    if (nblk > 0) stage_diag(Ld[0], dinv[0], Pb, r, (nblk - 1) * 32, min(32, w - (nblk - 1) * 32), tid, nth);
    for (int k = tid; k < r; k += nth) v[k] = k < w ? vb[d.f + k] : vb[rows[k]];
    __syncthreads();
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int jb = bi * 32;
        const int nbk = min(32, w - jb);
        // two columns per pass (c and c + nw): eight loads in flight per lane
        for (int c = warp; c < nbk; c += 2 * nw) {
            const int c2 = c + nw;
            const T* col = Pb + (int64_t)(jb + c) * r;
            const T* col2 = Pb + (int64_t)(jb + (c2 < nbk ? c2 : c)) * r;
            T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
            T t0 = T(0), t1 = T(0), t2 = T(0), t3 = T(0);
            int i = jb + nbk + lane;
            for (; i + 96 < r; i += 128) {
                const T v0 = v[i], v1 = v[i + 32], v2 = v[i + 64], v3 = v[i + 96];
                s0 += col[i] * v0;
                s1 += col[i + 32] * v1;
                s2 += col[i + 64] * v2;
                s3 += col[i + 96] * v3;
                t0 += col2[i] * v0;
                t1 += col2[i + 32] * v1;
                t2 += col2[i + 64] * v2;
                t3 += col2[i + 96] * v3;
            }
            for (; i < r; i += 32) {
                s0 += col[i] * v[i];
                t0 += col2[i] * v[i];
            }
            const T s = warp_sum((s0 + s1) + (s2 + s3));
            const T s2v = warp_sum((t0 + t1) + (t2 + t3));
            if (lane == 0) {
                dots[c] = s;
                if (c2 < nbk) dots[c2] = s2v;
            }
        }
        __syncthreads();
        if (tid < 32) {
            const int l = tid;
            T val = l < nbk ? v[jb + l] - dots[l] : T(0);
            for (int j = nbk - 1; j >= 0; --j) {
                const T xj = __shfl_sync(0xffffffffu, val, j) * dinv[buf][j];
                if (l == j) val = xj;
                if (l < j) val -= Ld[buf][j][l] * xj;
            }
            if (l < nbk) v[jb + l] = val;
        } else if (bi > 0) {
            stage_diag(Ld[buf ^ 1], dinv[buf ^ 1], Pb, r, jb - 32, 32, tid - 32, nth - 32);
        }
        buf ^= 1;
        __syncthreads();
    }
    for (int k = tid; k < w; k += nth) vb[d.f + k] = v[k];
}

// The triangular solve with one front's 32-column diagonal block of
// nbk <= NB columns (starting at column jb), by one warp: forward, lane l
// holds row jb + l of the block and v_l on entry, y_l on return; backward,
// lane l holds column jb + l (its entries on and below the diagonal) and
// v_l - dot_l on entry, x_l on return.  Instantiated for NB = 8, 16, 32 so
// that the narrow fronts of the lower levels do not step through 32
// predicated columns.
template <class T, int NB>
__device__ __forceinline__ T diag_fwd(const T* __restrict__ Pb, int r, int jb, int nbk, int lane, T val) {
    T a[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) a[j] = (j < nbk && lane < nbk) ? Pb[(int64_t)(jb + j) * r + jb + lane] : T(0);
    T dl = T(1);
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (lane == j && j < nbk) dl = a[j];
    const T dinv = T(1) / dl;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (j < nbk) {
            const T yj = __shfl_sync(0xffffffffu, val, j) * __shfl_sync(0xffffffffu, dinv, j);
            if (lane == j)
                val = yj;
            else if (lane > j)
                val -= a[j] * yj;
        }
    }
    return val;
}

template <class T, int NB>
__device__ __forceinline__ T diag_bwd(const T* __restrict__ Pb, int r, int jb, int nbk, int lane, T val) {
    T a[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        a[j] = (lane < nbk && j < nbk && j >= lane) ? Pb[(int64_t)(jb + lane) * r + jb + j] : T(0);
#pragma unroll
    for (int j = NB - 1; j >= 0; --j) {
        if (j < nbk) {
            const T dj = __shfl_sync(0xffffffffu, a[j], j);
            const T xj = __shfl_sync(0xffffffffu, val, j) / dj;
            if (lane == j)
                val = xj;
            else if (lane < j)
                val -= a[j] * xj;
        }
    }
    return val;
}

template <class T>
__device__ __forceinline__ T diag_fwd_any(const T* __restrict__ Pb, int r, int jb, int nbk, int lane, T val) {
    if (nbk <= 8) return diag_fwd<T, 8>(Pb, r, jb, nbk, lane, val);
    if (nbk <= 16) return diag_fwd<T, 16>(Pb, r, jb, nbk, lane, val);
    return diag_fwd<T, 32>(Pb, r, jb, nbk, lane, val);
}

template <class T>
__device__ __forceinline__ T diag_bwd_any(const T* __restrict__ Pb, int r, int jb, int nbk, int lane, T val) {
    if (nbk <= 8) return diag_bwd<T, 8>(Pb, r, jb, nbk, lane, val);
    if (nbk <= 16) return diag_bwd<T, 16>(Pb, r, jb, nbk, lane, val);
    return diag_bwd<T, 32>(Pb, r, jb, nbk, lane, val);
}

// The same, for blocks known to be at most NBMAX columns wide (16 or 32):
// a kernel instantiated for NBMAX = 16 holds no 32-entry diagonal row, and
// so fits a smaller register budget.
template <class T, int NBMAX>
__device__ __forceinline__ T diag_fwd_upto(const T* __restrict__ Pb, int r, int jb, int nbk, int lane, T val) {
    if (NBMAX <= 16)
        return nbk <= 8 ? diag_fwd<T, 8>(Pb, r, jb, nbk, lane, val) : diag_fwd<T, 16>(Pb, r, jb, nbk, lane, val);
    return diag_fwd_any<T>(Pb, r, jb, nbk, lane, val);
}
template <class T, int NBMAX>
__device__ __forceinline__ T diag_bwd_upto(const T* __restrict__ Pb, int r, int jb, int nbk, int lane, T val) {
    if (NBMAX <= 16)
        return nbk <= 8 ? diag_bwd<T, 8>(Pb, r, jb, nbk, lane, val) : diag_bwd<T, 16>(Pb, r, jb, nbk, lane, val);
    return diag_bwd_any<T>(Pb, r, jb, nbk, lane, val);
}

// Warp-per-(front, instance) variants of the two solves for levels that
// supply many items (a batch of value sets): eight independent warps per
// CTA, no block barriers; the 32x32 diagonal block is held in registers
// (forward: lane = row, backward: lane = column) and the front's vector in
// shared memory.  Items are front-major, so the 8 warps of a CTA read the
// same index tables.
template <class T, int NBMAX>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (NBMAX <= 16 ? 6 : 4) : 1)
    k_fwd_warp(const DevTables t, const int32_t* __restrict__ list, int32_t count, int32_t B, int32_t rmax,
               const T* __restrict__ panel, int64_t panel_total, T* __restrict__ vec, int64_t n,
               T* __restrict__ pvec, int64_t pvec_total, const int32_t* __restrict__ active, int32_t n_pats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t item = (int64_t)blockIdx.x * 8 + wib;
    if (item >= (int64_t)count * B) return;
    const int fi = (int)(item / B), b = (int)(item % B);
    const FrontDesc d = t.fronts[list[fi]];
    if (active && !active[(int64_t)b * n_pats + d.sys]) return;
    T* v = reinterpret_cast<T*>(smem_raw) + (int64_t)wib * rmax;
    const int r = d.r, w = d.w;
    T* vb = vec + (int64_t)b * n;
    const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    T* pv = pvec + (int64_t)b * pvec_total;
    gather_fwd<T, false>(t, d, vb, pv, v, lane);
    __syncwarp();
    for (int jb = 0; jb < w; jb += 32) {
        const int nbk = min(32, w - jb);
        T val = lane < nbk ? v[jb + lane] : T(0);
        val = diag_fwd_upto<T, NBMAX>(Pb, r, jb, nbk, lane, val);
        if (lane < nbk) v[jb + lane] = val;
        __syncwarp();
        for (int i0 = jb + nbk; i0 < r; i0 += 32) {
            const int i = i0 + lane;
            if (i < r) {
                const T* col = Pb + (int64_t)jb * r + i;
                T acc[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] = T(0);
                int j = 0;
                for (; j + 7 < nbk; j += 8) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) acc[u] += col[(int64_t)(j + u) * r] * v[jb + j + u];
                }
                for (; j < nbk; ++j) acc[0] += col[(int64_t)j * r] * v[jb + j];
                v[i] -= ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
            }
        }
        __syncwarp();
    }
    for (int k = lane; k < w; k += 32) vb[d.f + k] = v[k];
    for (int k = lane; k < r - w; k += 32) pv[d.pvec_off + k] = v[w + k];
}

// FP32: at most 64 registers, four CTAs (32 warps) per SM; the warps of a
// level hide each other's load latency, and the dot products need no more.
// Levels whose fronts are all at most 16 columns wide run the NBMAX = 16
// instantiations of both warp solves at 40 registers (six CTAs per SM).
template <class T, int NBMAX>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (NBMAX <= 16 ? 6 : 4) : 1)
    k_bwd_warp(const DevTables t, const int32_t* __restrict__ list, int32_t count, int32_t B, int32_t rmax,
               const T* __restrict__ panel, int64_t panel_total, T* __restrict__ vec, int64_t n,
               const int32_t* __restrict__ active, int32_t n_pats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t item = (int64_t)blockIdx.x * 8 + wib;
    if (item >= (int64_t)count * B) return;
    const int fi = (int)(item / B), b = (int)(item % B);
    const FrontDesc d = t.fronts[list[fi]];
    if (active && !active[(int64_t)b * n_pats + d.sys]) return;
    T* v = reinterpret_cast<T*>(smem_raw) + (int64_t)wib * rmax;
    const int r = d.r, w = d.w;
    T* vb = vec + (int64_t)b * n;
    const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    const int32_t* rows = t.rows + d.rows_off;
    gather_bwd<T, false>(d, rows, vb, v, lane);
    __syncwarp();
    const int nblk = (w + 31) / 32;
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int jb = bi * 32;
        const int nbk = min(32, w - jb);
        T dot = T(0);
        if (lane < nbk) {
            const T* col = Pb + (int64_t)(jb + lane) * r;
            T d1 = T(0), d2 = T(0), d3 = T(0);
            int i = jb + nbk;
            for (; i + 3 < r; i += 4) {
                dot += col[i] * v[i];
                d1 += col[i + 1] * v[i + 1];
                d2 += col[i + 2] * v[i + 2];
                d3 += col[i + 3] * v[i + 3];
            }
            for (; i < r; ++i) dot += col[i] * v[i];
            dot += d1 + d2 + d3;
        }
        T val = lane < nbk ? v[jb + lane] - dot : T(0);
        val = diag_bwd_upto<T, NBMAX>(Pb, r, jb, nbk, lane, val);
        if (lane < nbk) v[jb + lane] = val;
        __syncwarp();
    }
    for (int k = lane; k < w; k += 32) vb[d.f + k] = v[k];
}

// --------------------------------------------------------------------------
// Dataflow launches.  A persistent grid walks a level-ordered list of items
// (a front for one value set, or for a group of V value sets); a warp or CTA
// takes the next item from a ticket counter and waits only for the items it
// depends on (its children in the factorization and the forward sweep, its
// parent in the backward sweep), whose done flags it polls.  Tickets are
// taken in list order by running warps or CTAs only, and an item depends
// only on earlier items, so the earliest unfinished item never waits: the
// schedule cannot deadlock, whatever number of CTAs is resident.  Every wait
// is bounded: on expiry (or once another waiter has given up) the waiter
// raises the plan's device error word (status TIMEOUT) and leaves the launch.
// The region of a launch: [0..31] tickets (word 31 is never set: the test
// hook waits on it), then done flags [slot][B].
// --------------------------------------------------------------------------
constexpr int kFlowFlags = 32;

__device__ __forceinline__ int32_t flow_ld_acquire(const int32_t* p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void flow_st_release(int32_t* p, int32_t v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// true once *flag >= want; false after max_polls polls, or as soon as
// another waiter has raised *dev_err.
__device__ bool flow_wait(const int32_t* flag, int32_t want, const int32_t* dev_err, uint32_t max_polls) {
    for (uint32_t it = 0;; ++it) {
        if (flow_ld_acquire(flag) >= want) return true;
        if (it >= max_polls || *(volatile const int32_t*)dev_err) return false;
        __nanosleep(it < 8 ? 64 : 256);
    }
}

// Forward sweep over the dataflow fronts.  One CTA of G warps per item
// (front, G consecutive value sets): the ticket, the front's descriptor and
// the children's done flags (one per item) are shared by the G warps, and
// warp w does the k_fwd_warp arithmetic for value set g*G + w.  Values that
// other CTAs of this launch wrote (the children's passing vectors) are read
// past L1 (ld.global.cg).
template <class T>
__global__ void __launch_bounds__(256, 2) k_flow_fwd(const DevTables t, int32_t n_front, int32_t B, int32_t rmax,
                                                     const T* __restrict__ panel, int64_t panel_total,
                                                     T* __restrict__ vec, int64_t n, T* __restrict__ pvec,
                                                     int64_t pvec_total, const int32_t* __restrict__ active,
                                                     int32_t n_pats, int32_t* __restrict__ flow,
                                                     int32_t* __restrict__ dev_err, uint32_t max_polls,
                                                     int32_t stall) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_item;
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, G = blockDim.x >> 5;
    T* v = reinterpret_cast<T*>(smem_raw) + (int64_t)wib * rmax;
    int32_t* flags = flow + kFlowFlags;
    const int nG = (B + G - 1) / G;
    const int64_t n_items = (int64_t)n_front * nG;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_item = atomicAdd(flow, 1);
            s_ok = 1;
        }
        __syncthreads();
        const int64_t item = s_item;
        if (item >= n_items) return;
        const int pos = (int)(item / nG), g = (int)(item - (int64_t)pos * nG);
        const int b = g * G + wib;
        const FrontDesc d = t.fronts[t.flow_solve[pos]];
        if (wib == 0) {
            bool ok = true;
            if (item == stall) ok = flow_wait(flow + 31, 1, dev_err, max_polls);
            for (int c = lane; ok && c < d.nchild; c += 32) {
                const int sl = t.flow_sslot[t.child_ids[d.child_off + c]];
                if (sl >= 0) ok = flow_wait(flags + (int64_t)sl * B + g, 1, dev_err, max_polls);
            }
            if (!__all_sync(0xffffffffu, ok) && lane == 0) {
                atomicExch(dev_err, 1);
                s_ok = 0;
            }
        }
        __syncthreads();
        if (!s_ok) return;
        if (b < B && !(active && !active[(int64_t)b * n_pats + d.sys])) {
            const int r = d.r, w = d.w;
            T* vb = vec + (int64_t)b * n;
            const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
            T* pv = pvec + (int64_t)b * pvec_total;
            gather_fwd<T, true>(t, d, vb, pv, v, lane);
            __syncwarp();
            for (int jb = 0; jb < w; jb += 32) {
                const int nbk = min(32, w - jb);
                T val = lane < nbk ? v[jb + lane] : T(0);
                val = diag_fwd_any<T>(Pb, r, jb, nbk, lane, val);
                if (lane < nbk) v[jb + lane] = val;
                __syncwarp();
                // rows below the block, four per lane (rows i0 + lane + 32u):
                // 8 columns x 4 rows = 32 independent loads in flight per lane
                const T* colb = Pb + (int64_t)jb * r;
                for (int i0 = jb + nbk; i0 < r; i0 += 128) {
                    int ii[4];
                    T acc[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        ii[u] = min(i0 + lane + 32 * u, r - 1);
                        acc[u] = T(0);
                    }
                    for (int j0 = 0; j0 < nbk; j0 += 8) {
                        T x[8][4];
#pragma unroll
                        for (int c = 0; c < 8; ++c)
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                x[c][u] = j0 + c < nbk ? colb[(int64_t)(j0 + c) * r + ii[u]] : T(0);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const T y = j0 + c < nbk ? v[jb + j0 + c] : T(0);
#pragma unroll
                            for (int u = 0; u < 4; ++u) acc[u] += x[c][u] * y;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (i0 + lane + 32 * u < r) v[ii[u]] -= acc[u];
                }
                __syncwarp();
            }
            for (int k = lane; k < w; k += 32) vb[d.f + k] = v[k];
            for (int k = lane; k < r - w; k += 32) pv[d.pvec_off + k] = v[w + k];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            flow_st_release(flags + (int64_t)pos * B + g, 1);
        }
    }
}

// Backward sweep over the dataflow fronts (parents first), CTA items as in
// the forward sweep: the k_bwd_warp arithmetic per value set, after the
// parent's done flag (which implies every ancestor's: each waited for its
// own parent).
template <class T>
__global__ void __launch_bounds__(256, 2) k_flow_bwd(const DevTables t, int32_t n_front, int32_t B, int32_t rmax,
                                                     const T* __restrict__ panel, int64_t panel_total,
                                                     T* __restrict__ vec, int64_t n,
                                                     const int32_t* __restrict__ active, int32_t n_pats,
                                                     int32_t* __restrict__ flow, int32_t* __restrict__ dev_err,
                                                     uint32_t max_polls) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_item;
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, G = blockDim.x >> 5;
    T* v = reinterpret_cast<T*>(smem_raw) + (int64_t)wib * rmax;
    int32_t* flags = flow + kFlowFlags;
    const int nG = (B + G - 1) / G;
    const int64_t n_items = (int64_t)n_front * nG;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_item = atomicAdd(flow + 1, 1);
            s_ok = 1;
        }
        __syncthreads();
        if (s_item >= n_items) return;
        const int64_t q = n_items - 1 - s_item;
        const int pos = (int)(q / nG), g = (int)(q - (int64_t)pos * nG);
        const int b = g * G + wib;
        const FrontDesc d = t.fronts[t.flow_solve[pos]];
        if (wib == 0) {
            bool ok = true;
            if (d.parent >= 0) {
                const int sl = t.flow_sslot[d.parent];
                if (sl >= 0) ok = flow_wait(flags + (int64_t)sl * B + g, 2, dev_err, max_polls);
            }
            if (!__all_sync(0xffffffffu, ok) && lane == 0) {
                atomicExch(dev_err, 1);
                s_ok = 0;
            }
        }
        __syncthreads();
        if (!s_ok) return;
        if (b < B && !(active && !active[(int64_t)b * n_pats + d.sys])) {
            const int r = d.r, w = d.w;
            T* vb = vec + (int64_t)b * n;
            const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
            const int32_t* rows = t.rows + d.rows_off;
            gather_bwd<T, true>(d, rows, vb, v, lane);
            __syncwarp();
            const int nblk = (w + 31) / 32;
            for (int bi = nblk - 1; bi >= 0; --bi) {
                const int jb = bi * 32;
                const int nbk = min(32, w - jb);
                // lane j: dot_j = sum over rows i below the block of L[i, jb+j] v[i]
                T dot = T(0);
                if (lane < nbk) {
                    const T* col = Pb + (int64_t)(jb + lane) * r;
                    T d1 = T(0), d2 = T(0), d3 = T(0);
                    int i = jb + nbk;
                    for (; i + 3 < r; i += 4) {
                        dot += col[i] * v[i];
                        d1 += col[i + 1] * v[i + 1];
                        d2 += col[i + 2] * v[i + 2];
                        d3 += col[i + 3] * v[i + 3];
                    }
                    for (; i < r; ++i) dot += col[i] * v[i];
                    dot += d1 + d2 + d3;
                }
                T val = lane < nbk ? v[jb + lane] - dot : T(0);
                val = diag_bwd_any<T>(Pb, r, jb, nbk, lane, val);
                if (lane < nbk) v[jb + lane] = val;
                __syncwarp();
            }
            for (int k = lane; k < w; k += 32) vb[d.f + k] = v[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            flow_st_release(flags + (int64_t)pos * B + g, 2);
        }
    }
}

// Small-front factorization as a dataflow launch: one CTA per item (front,
// V consecutive value sets interleaved entry by entry in shared memory, so
// one vector access serves all V).  Per item: zero the packed triangle and
// gather the front's K entries (independent of the children), wait for the
// children of this group, add their update matrices through the relative
// maps, then a blocked right-looking partial Cholesky in panels of kFlowNB
// columns with three barriers per panel: (1) the panel's diagonal block is
// factored in registers with warp shuffles (lane = row x value set; V / 2
// warps) and its L kept in shared memory; (2) every thread solves rows below
// the block against it (a triangular solve per row, L read as broadcasts);
// (3) the trailing triangle takes one rank-kFlowNB update in register tiles.
// Finally the panel and the update matrix go to global memory and the
// item's done flag is released.
constexpr int kFlowNB = 16;

//
// With ticket < 0 the same kernel serves one level's launch list instead:
// one CTA per item (blockIdx.x), no ticket, no waits, no flags (the
// children were factored by earlier launches on the stream); fl is then
// the level's front list and off is unused.
template <class T, int V>
__global__ void __launch_bounds__(256) k_front_flow(const DevTables t, const int32_t* __restrict__ fl, int32_t off,
                                                    int32_t count, int32_t B,
                                                    const double* __restrict__ K, int64_t nnzK,
                                                    T* __restrict__ panel, int64_t panel_total,
                                                    T* __restrict__ upd, int64_t upd_total,
                                                    int32_t* __restrict__ bad_col, int32_t n_pats,
                                                    int32_t* __restrict__ flow, int32_t ticket,
                                                    int32_t* __restrict__ dev_err, uint32_t max_polls,
                                                    int32_t stall) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NB = kFlowNB;
    constexpr int CB = V == 1 ? 4 : 2;  // trailing-update columns per thread (rows: 4)
    __shared__ int64_t s_item;
    __shared__ int s_ok;
    T* Ld = reinterpret_cast<T*>(smem_raw);  // [NB][NB][V] L of the diagonal block
    T* Li = Ld + NB * NB * V;                // [NB][V] reciprocals of its diagonal
    T* F = Li + NB * V;                      // packed lower triangle x V, then kSmallPad x V zeros
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int tid = threadIdx.x, nth = blockDim.x;
    int32_t* flags = flow + kFlowFlags;
    const int nG = (B + V - 1) / V;
    const int64_t n_items = (int64_t)count * nG;
    for (int rep = 0;; ++rep) {
        __syncthreads();
        if (tid == 0) {
            s_item = ticket >= 0 ? (int64_t)atomicAdd(flow + ticket, 1) : (rep == 0 ? (int64_t)blockIdx.x : n_items);
            s_ok = 1;
        }
        __syncthreads();
        const int64_t item = s_item;
        if (item >= n_items) return;
        const int q = (int)(item / nG), g = (int)(item - (int64_t)q * nG);
        const int b0 = g * V, nv = min(V, B - b0);
        const FrontDesc d = t.fronts[fl[q]];
        const int r = d.r, w = d.w;
        const int npk = r * (r + 1) / 2 + kSmallPad;
        for (int e = tid; e < npk * V; e += nth) F[e] = T(0);
        __syncthreads();
        {
            const int32_t* kl = t.klist + 2 * d.klist_off;
            for (int e = tid; e < d.klist_n; e += nth) {
                const int pos = kl[2 * e + 1], slot = kl[2 * e];
                const int col = pos / r, row = pos - col * r;
                T* dst = F + (int64_t)(packed_col(col, r) + row - col) * V;
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (v < nv) dst[v] = (T)K[(int64_t)(b0 + v) * nnzK + slot];
            }
        }
        if (warp == 0 && ticket >= 0) {
            bool ok = true;
            if (item == stall) ok = flow_wait(flow + 31, 1, dev_err, max_polls);
            for (int c = lane; ok && c < d.nchild; c += 32) {
                const int sl = t.flow_fslot[t.child_ids[d.child_off + c]];
                if (sl >= off && sl < off + count) ok = flow_wait(flags + (int64_t)sl * B + g, 1, dev_err, max_polls);
            }
            if (!__all_sync(0xffffffffu, ok) && lane == 0) {
                atomicExch(dev_err, 1);
                s_ok = 0;
            }
        }
        __syncthreads();
        if (!s_ok) return;
        // children's update matrices (written by other CTAs: read past L1)
        for (int c = 0; c < d.nchild; ++c) {
            const FrontDesc cd = t.fronts[t.child_ids[d.child_off + c]];
            const int rc = cd.r - cd.w;
            const int32_t* map = t.relmap + cd.relmap_off;
            const T* S0 = upd + (int64_t)b0 * upd_total + cd.upd_off;
            // the warp walks (column kk, 32-row chunk) pairs of its columns
            // (kk = warp, warp + nw, ...), EB pairs at a time: all their
            // loads are issued before the shared-memory adds
            constexpr int EB = V >= 4 ? 4 : 8;
            int kk = warp, i0 = warp;
            while (kk < rc) {
                int mi[EB], mk[EB];
                T sv[EB][V];
#pragma unroll
                for (int e = 0; e < EB; ++e) {
                    const int ii = i0 + lane;
                    const bool ok = kk < rc && ii < rc;
                    mi[e] = ok ? map[ii] : -1;
                    mk[e] = ok ? map[kk] : 0;
                    const T* Sk = S0 + (int64_t)kk * rc + ii;
#pragma unroll
                    for (int v = 0; v < V; ++v) sv[e][v] = (ok && v < nv) ? __ldcg(Sk + (int64_t)v * upd_total) : T(0);
                    if (kk < rc) {
                        i0 += 32;
                        if (i0 >= rc) {
                            kk += nw;
                            i0 = kk;
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < EB; ++e) {
                    if (mi[e] < 0) continue;
                    T* Fe = F + (int64_t)(packed_col(mk[e], r) - mk[e] + mi[e]) * V;
                    T x[V];
                    vld<T, V>(Fe, x);
#pragma unroll
                    for (int v = 0; v < V; ++v) x[v] += sv[e][v];
                    vst<T, V>(Fe, x);
                }
            }
            __syncthreads();
        }
        const int n_off = (int)t.sys_n_off[d.sys];
        const int dwarps = V >= 2 ? V / 2 : 1;  // warps factoring the diagonal block
        for (int j0 = 0; j0 < w; j0 += NB) {
            const int nb = min(NB, w - j0), j1 = j0 + nb;
            // (1) diagonal block: lane = (row i, value set v)
            if (warp < dwarps) {
                const int i = lane & 15, hi = lane & 16;
                const int v = V >= 2 ? 2 * warp + (lane >> 4) : 0;
                T a[NB];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    a[k] = (k < nb && k <= i && i < nb) ? F[(int64_t)(packed_col(j0 + k, r) + i - k) * V + v] : T(0);
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    if (j < nb) {
                        T dj = __shfl_sync(0xffffffffu, a[j], j + hi);
                        if (!(dj > T(0))) {
                            if (i == j && v < nv && (V >= 2 || hi == 0))
                                atomicMin(&bad_col[(int64_t)(b0 + v) * n_pats + d.sys], d.f + j0 + j - n_off);
                            dj = T(1);
                        }
                        // one reciprocal square root instead of a square
                        // root and a division on the pivot chain
                        const T inv = rsqrt(dj), lj = dj * inv;
                        if (i == j)
                            a[j] = lj;
                        else if (i > j)
                            a[j] *= inv;
#pragma unroll
                        for (int k = j + 1; k < NB; ++k) {
                            const T lk = __shfl_sync(0xffffffffu, a[j], k + hi);
                            if (i >= k) a[k] -= a[j] * lk;
                        }
                    }
                }
                if (i < nb && (V >= 2 || hi == 0)) {
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        if (k <= i) {
                            Ld[(i * NB + k) * V + v] = a[k];
                            F[(int64_t)(packed_col(j0 + k, r) + i - k) * V + v] = a[k];
                        }
                    }
                    Li[i * V + v] = T(1) / a[i];
                }
            }
            __syncthreads();
            // (2) rows below the block: x := x L^{-T}
            for (int i = j1 + tid; i < r; i += nth) {
                T x[NB][V];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (k < nb) vld<T, V>(F + (int64_t)(packed_col(j0 + k, r) + i - j0 - k) * V, x[k]);
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    if (k < nb) {
#pragma unroll
                        for (int m = 0; m < k; ++m) {
                            T l[V];
                            vld<T, V>(Ld + (k * NB + m) * V, l);
#pragma unroll
                            for (int v = 0; v < V; ++v) x[k][v] -= x[m][v] * l[v];
                        }
                        T iv[V];
                        vld<T, V>(Li + k * V, iv);
#pragma unroll
                        for (int v = 0; v < V; ++v) x[k][v] *= iv[v];
                        vst<T, V>(F + (int64_t)(packed_col(j0 + k, r) + i - j0 - k) * V, x[k]);
                    }
                }
            }
            __syncthreads();
            // (3) trailing triangle: F[i, k] -= L[i, j0:j1] L[k, j0:j1]^T
            const int m = r - j1;
            if (m > 0) {
                const int tx = tid & 15, ty = tid >> 4, ny = nth >> 4;
                const int tk_cols = CB * ny;
                for (int c0 = 0; c0 < m; c0 += tk_cols) {
                    for (int r0 = (c0 / 64) * 64; r0 < m; r0 += 64) {
                        T acc[4][CB][V];
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int c = 0; c < CB; ++c)
#pragma unroll
                                for (int v = 0; v < V; ++v) acc[a][c][v] = T(0);
                        int ii[4], kk[CB];
#pragma unroll
                        for (int a = 0; a < 4; ++a) ii[a] = j1 + r0 + tx + 16 * a;
#pragma unroll
                        for (int c = 0; c < CB; ++c) kk[c] = j1 + c0 + ty + ny * c;
                        // rows / columns past r read the next column's entries
                        // or the zero padding (within the allocation); they
                        // only reach accumulators the epilogue skips
                        const T* Fi = F + (int64_t)(packed_col(j0, r) - j0 + ii[0]) * V;
                        const T* Fk = F + (int64_t)(packed_col(j0, r) - j0 + kk[0]) * V;
                        for (int j = j0; j < j1; ++j) {
                            T ra[4][V], cb[CB][V];
#pragma unroll
                            for (int a = 0; a < 4; ++a) vld<T, V>(Fi + (int64_t)(16 * a) * V, ra[a]);
#pragma unroll
                            for (int c = 0; c < CB; ++c) vld<T, V>(Fk + (int64_t)(ny * c) * V, cb[c]);
                            Fi += (int64_t)(r - j - 1) * V;
                            Fk += (int64_t)(r - j - 1) * V;
#pragma unroll
                            for (int a = 0; a < 4; ++a)
#pragma unroll
                                for (int c = 0; c < CB; ++c)
#pragma unroll
                                    for (int v = 0; v < V; ++v) acc[a][c][v] += ra[a][v] * cb[c][v];
                        }
#pragma unroll
                        for (int c = 0; c < CB; ++c) {
                            if (kk[c] >= r) continue;
                            T* Fk2 = F + (int64_t)(packed_col(kk[c], r) - kk[c]) * V;
#pragma unroll
                            for (int a = 0; a < 4; ++a) {
                                if (ii[a] < r && ii[a] >= kk[c]) {
                                    T x[V];
                                    vld<T, V>(Fk2 + (int64_t)ii[a] * V, x);
#pragma unroll
                                    for (int v = 0; v < V; ++v) x[v] -= acc[a][c][v];
                                    vst<T, V>(Fk2 + (int64_t)ii[a] * V, x);
                                }
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
        // factor columns (lower part) and update matrix
        T* P0 = panel + (int64_t)b0 * panel_total + d.panel_off;
        for (int jj = warp; jj < w; jj += nw) {
            const T* Fj = F + (int64_t)(packed_col(jj, r) - jj) * V;
            for (int i = jj + lane; i < r; i += 32) {
                T x[V];
                vld<T, V>(Fj + (int64_t)i * V, x);
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (v < nv) P0[(int64_t)v * panel_total + (int64_t)jj * r + i] = x[v];
            }
        }
        const int ru = r - w;
        if (ru > 0) {
            T* U0 = upd + (int64_t)b0 * upd_total + d.upd_off;
            for (int kk = warp; kk < ru; kk += nw) {
                const T* Fk = F + (int64_t)(packed_col(w + kk, r) - (w + kk)) * V;
                for (int ii = kk + lane; ii < ru; ii += 32) {
                    T x[V];
                    vld<T, V>(Fk + (int64_t)(w + ii) * V, x);
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (v < nv) U0[(int64_t)v * upd_total + (int64_t)kk * ru + ii] = x[v];
                }
            }
        }
        __syncthreads();
        if (tid == 0 && ticket >= 0) {
            __threadfence();
            flow_st_release(flags + (int64_t)(off + q) * B + g, 1);
        }
    }
}

// --------------------------------------------------------------------------
// a6: vectors, residual and refinement control (FP64)
// --------------------------------------------------------------------------
__global__ void k_permute_in(const double* __restrict__ bu, const int32_t* __restrict__ perm, int64_t n,
                             double* __restrict__ bp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = (int64_t)blockIdx.y * n;
    bp[o + i] = bu[o + perm[i]];
}

__global__ void k_permute_out(const double* __restrict__ xp, const int32_t* __restrict__ perm, int64_t n,
                              double* __restrict__ xu) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = (int64_t)blockIdx.y * n;
    xu[o + perm[i]] = xp[o + i];
}

template <class T>
__global__ void k_to_T(const double* __restrict__ src, T* __restrict__ dst, int64_t total) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) dst[i] = (T)src[i];
}

template <class T>
__global__ void k_from_T(const T* __restrict__ src, double* __restrict__ dst, int64_t total) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) dst[i] = (double)src[i];
}

// per-system init: ||b||_2, counters
// Per-system norms in two passes: k_sys_partial reduces chunks of
// kSysChunk rows of every system over many CTAs (one per chunk and system),
// then k_sys_init / k_check combine a system's chunk results in chunk order
// (a fixed order: the same sums on every run).  One CTA per whole system
// left the GPU idle while the largest system's CTA walked its rows.
constexpr int kSysChunk = 2048;

__global__ void k_sys_partial(const double* __restrict__ v, const int64_t* __restrict__ sys_n_off, int32_t n_pats,
                              int64_t n, int32_t maxc, const int32_t* __restrict__ active, double* __restrict__ psum,
                              double* __restrict__ pmax) {
    const int c = blockIdx.x, s = blockIdx.y;
    if (active && !active[s]) return;
    const int b = s / n_pats, k = s % n_pats;
    const int64_t lo = sys_n_off[k] + (int64_t)c * kSysChunk;
    const int64_t hi = min(sys_n_off[k + 1], lo + kSysChunk);
    if (lo >= hi) return;
    const double* vb = v + (int64_t)b * n;
    double sum = 0.0, mx = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double a = vb[i];
        sum += a * a;
        mx = fmax(mx, fabs(a));
        if (!(fabs(a) <= 1.7976931348623157e308)) mx = INFINITY;
    }
    block_sum_max(sum, mx);
    if (threadIdx.x == 0) {
        psum[(int64_t)s * maxc + c] = sum;
        pmax[(int64_t)s * maxc + c] = mx;
    }
}

// Sum of squares and max magnitude of system s (valid in thread 0): from
// its chunk results when psum is given, else directly from its rows of v
// (one pass: plans with at least as many systems as SMs, where the systems
// alone spread over the GPU and a second launch would cost more).
__device__ __forceinline__ void sys_combine(const double* __restrict__ v, int64_t n,
                                            const int64_t* __restrict__ sys_n_off, int32_t n_pats, int s,
                                            int32_t maxc, const double* __restrict__ psum,
                                            const double* __restrict__ pmax, double& sum, double& mx) {
    const int b = s / n_pats, k = s % n_pats;
    sum = 0.0;
    mx = 0.0;
    if (psum) {
        const int nch = (int)((sys_n_off[k + 1] - sys_n_off[k] + kSysChunk - 1) / kSysChunk);
        for (int c = threadIdx.x; c < nch; c += blockDim.x) {
            sum += psum[(int64_t)s * maxc + c];
            mx = fmax(mx, pmax[(int64_t)s * maxc + c]);
        }
    } else {
        const double* vb = v + (int64_t)b * n;
        for (int64_t i = sys_n_off[k] + threadIdx.x; i < sys_n_off[k + 1]; i += blockDim.x) {
            const double a = vb[i];
            sum += a * a;
            mx = fmax(mx, fabs(a));
            if (!(fabs(a) <= 1.7976931348623157e308)) mx = INFINITY;
        }
    }
    block_sum_max(sum, mx);
}

__global__ void k_sys_init(const double* __restrict__ v, int64_t n, const int64_t* __restrict__ sys_n_off,
                           int32_t n_pats, int32_t maxc, const double* __restrict__ psum,
                           const double* __restrict__ pmax,
                           double* __restrict__ bnorm, int32_t* __restrict__ active,
                           int32_t* __restrict__ sstatus, int32_t* __restrict__ iters, double* __restrict__ resid,
                           double* __restrict__ r1, double* __restrict__ r2) {
    const int s = blockIdx.x;
    double sum, mx;
    sys_combine(v, n, sys_n_off, n_pats, s, maxc, psum, pmax, sum, mx);
    if (threadIdx.x == 0) {
        bnorm[s] = sqrt(sum);
        active[s] = 1;
        sstatus[s] = SSCO_OK;
        iters[s] = 0;
        resid[s] = 0.0;
        r1[s] = INFINITY;
        r2[s] = INFINITY;
    }
}

// rr = bp - K~ xp, symmetric CSR over permuted rows
__global__ void __launch_bounds__(256) k_resid(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                               const int32_t* __restrict__ slot, const double* __restrict__ K,
                                               int64_t nnzK, const double* __restrict__ bp,
                                               const double* __restrict__ xp, double* __restrict__ rr, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = blockIdx.y;
    const double* Kb = K + (int64_t)b * nnzK;
    const double* xb = xp + (int64_t)b * n;
    double s = 0.0;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) s += Kb[slot[q]] * xb[col[q]];
    rr[(int64_t)b * n + i] = bp[(int64_t)b * n + i] - s;
}

// residual test and refinement decision for one system per CTA
__global__ void k_check(const double* __restrict__ v, int64_t n, const int64_t* __restrict__ sys_n_off,
                        int32_t n_pats, int32_t maxc, const double* __restrict__ psum,
                        const double* __restrict__ pmax,
                        const double* __restrict__ bnorm, int32_t* __restrict__ active,
                        int32_t* __restrict__ sstatus, int32_t* __restrict__ iters, double* __restrict__ resid,
                        double* __restrict__ r1, double* __restrict__ r2, double* __restrict__ sigma,
                        int32_t* __restrict__ any_active, int it, int maxit, double tol, int refine,
                        const int32_t* __restrict__ it_dev) {
    const int s = blockIdx.x;
    if (!active[s]) return;
    if (it_dev) it = *it_dev;
    double sum, mx;
    sys_combine(v, n, sys_n_off, n_pats, s, maxc, psum, pmax, sum, mx);
    if (threadIdx.x != 0) return;
    const double rn = sqrt(sum);
    const double bn = bnorm[s];
    double res = bn > 0.0 ? rn / bn : (rn > 0.0 ? INFINITY : 0.0);
    if (!(mx <= 1.7976931348623157e308)) res = NAN;
    resid[s] = res;
    iters[s] = it;
    int act = 0;
    if (!(res == res) || isinf(res)) {
        sstatus[s] = SSCO_ERR_NONFINITE;
    } else if (res <= tol) {
        sstatus[s] = SSCO_OK;
    } else if (!refine || it >= maxit || (it >= 2 && res > 0.5 * r2[s])) {
        sstatus[s] = SSCO_ERR_NO_CONVERGE;
    } else {
        act = 1;
        sigma[s] = mx;
    }
    active[s] = act;
    r2[s] = r1[s];
    r1[s] = res;
    if (act) atomicAdd(any_active, 1);
}

template <class T>
__global__ void k_cast_scaled(const double* __restrict__ rr, const int32_t* __restrict__ row_sys, int32_t n_pats,
                              int64_t n, const int32_t* __restrict__ active, const double* __restrict__ sigma,
                              T* __restrict__ vecT) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = blockIdx.y;
    const int s = b * n_pats + row_sys[i];
    const int64_t o = (int64_t)b * n + i;
    vecT[o] = active[s] ? (T)(rr[o] / sigma[s]) : T(0);
}

template <class T>
__global__ void k_update(const T* __restrict__ vecT, const int32_t* __restrict__ row_sys, int32_t n_pats, int64_t n,
                         const int32_t* __restrict__ active, const double* __restrict__ sigma,
                         double* __restrict__ xp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = blockIdx.y;
    const int s = b * n_pats + row_sys[i];
    const int64_t o = (int64_t)b * n + i;
    if (active[s]) xp[o] += sigma[s] * (double)vecT[o];
}

// --------------------------------------------------------------------------
// GMRES-IR (refine_mode 1, 2): a correction solves K d = r by restarted
// GMRES in FP64 with the FP32 factor as right preconditioner, d = Z y with
// z_j = M^-1 v_j, M = L L^T (two FP32 triangular solves).  All active
// systems advance in lockstep; per-system masks stop a system's inner
// iteration when its residual estimate has fallen by kGmresEta.
// Orthogonalisation: classical Gram-Schmidt applied twice (CGS2).
// --------------------------------------------------------------------------
constexpr double kGmresEta = 1e-4;

// Per system: V_0 = r / beta with beta = resid * ||b|| (the 2-norm k_check
// measured), g = (beta, 0, ...), the inner mask from the outer mask.
__global__ void k_gm_start(const double* __restrict__ rr, const int32_t* __restrict__ row_sys, int32_t n_pats,
                           int64_t n, const int32_t* __restrict__ active, const double* __restrict__ resid,
                           const double* __restrict__ bnorm, double* __restrict__ V0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = blockIdx.y;
    const int s = b * n_pats + row_sys[i];
    const int64_t o = (int64_t)b * n + i;
    const double beta = resid[s] * bnorm[s];
    V0[o] = active[s] && beta > 0.0 ? rr[o] / beta : 0.0;
}

__global__ void k_gm_init(int64_t S, int m, const int32_t* __restrict__ active, const double* __restrict__ resid,
                          const double* __restrict__ bnorm, double* __restrict__ beta, double* __restrict__ g,
                          int32_t* __restrict__ gact, int32_t* __restrict__ kdone) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double bt = resid[s] * bnorm[s];
    beta[s] = bt;
    for (int i = 0; i <= m; ++i) g[s * (m + 1) + i] = i == 0 ? bt : 0.0;
    gact[s] = active[s] && bt > 0.0 ? 1 : 0;
    kdone[s] = 0;
}

// vecT = (T) V_j on masked systems (unit-norm vectors need no scaling)
template <class T>
__global__ void k_gm_cast(const double* __restrict__ v, const int32_t* __restrict__ row_sys, int32_t n_pats,
                          int64_t n, const int32_t* __restrict__ mask, T* __restrict__ vecT) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = blockIdx.y;
    const int64_t o = (int64_t)b * n + i;
    vecT[o] = mask[b * n_pats + row_sys[i]] ? (T)v[o] : T(0);
}

// z = (double) vecT, w = K z (symmetric CSR over permuted rows), masked
template <class T>
__global__ void __launch_bounds__(256) k_gm_spmv(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                 const int32_t* __restrict__ slot, const double* __restrict__ K,
                                                 int64_t nnzK, const int32_t* __restrict__ row_sys, int32_t n_pats,
                                                 int64_t n, const int32_t* __restrict__ mask,
                                                 const T* __restrict__ vecT, double* __restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = blockIdx.y;
    const int64_t o = (int64_t)b * n + i;
    if (!mask[b * n_pats + row_sys[i]]) {
        w[o] = 0.0;
        return;
    }
    const double* Kb = K + (int64_t)b * nnzK;
    const T* zb = vecT + (int64_t)b * n;
    double acc = 0.0;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) acc += Kb[slot[q]] * (double)zb[col[q]];
    w[o] = acc;
}

template <class T>
__global__ void k_gm_storez(const T* __restrict__ vecT, int64_t total, double* __restrict__ z) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) z[i] = (double)vecT[i];
}

// hp[s][i] = <V_i, w> over the rows of system s, i = ibase + blockIdx.y;
// with ibase = j + 1 and w = V_j+1 it is the squared norm <w, w>
__global__ void k_gm_dots(const double* __restrict__ V, int64_t vstride, int ibase, const double* __restrict__ w,
                          const int64_t* __restrict__ sys_n_off, int32_t n_pats, int64_t n,
                          const int32_t* __restrict__ mask, int m, double* __restrict__ hp) {
    const int s = blockIdx.x, i = ibase + (int)blockIdx.y;
    if (!mask[s]) return;
    const int b = s / n_pats, k = s % n_pats;
    const double* vi = V + i * vstride + (int64_t)b * n;
    const double* wb = w + (int64_t)b * n;
    double sum = 0.0, mx = 0.0;
    for (int64_t r = sys_n_off[k] + threadIdx.x; r < sys_n_off[k + 1]; r += blockDim.x) sum += vi[r] * wb[r];
    block_sum_max(sum, mx);
    if (threadIdx.x == 0) hp[(int64_t)s * (m + 1) + i] = sum;
}

// w -= sum_{i <= j} hp[s][i] V_i, and H[s][i][j] += hp[s][i]
__global__ void k_gm_orth(const double* __restrict__ V, int64_t vstride, const int32_t* __restrict__ row_sys,
                          int32_t n_pats, int64_t n, const int32_t* __restrict__ mask, int m, int j,
                          const double* __restrict__ hp, double* __restrict__ w) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int b = blockIdx.y;
    const int s = b * n_pats + row_sys[r];
    if (!mask[s]) return;
    const int64_t o = (int64_t)b * n + r;
    const double* h = hp + (int64_t)s * (m + 1);
    double acc = w[o];
    for (int i = 0; i <= j; ++i) acc -= h[i] * V[i * vstride + o];
    w[o] = acc;
}

__global__ void k_gm_hacc(int64_t S, int m, int j, const int32_t* __restrict__ mask, const double* __restrict__ hp,
                          double* __restrict__ H) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || !mask[s]) return;
    for (int i = 0; i <= j; ++i) H[(s * (m + 1) + i) * m + j] += hp[s * (m + 1) + i];
}

// Column j of each system's Hessenberg matrix: its subdiagonal ||w||, the
// earlier rotations, a new Givens rotation, the residual estimate |g_j+1|;
// a system whose estimate fell below eta * beta (or whose w vanished)
// leaves the inner iteration with k = j + 1 vectors.
__global__ void k_gm_givens(int64_t S, int m, int j, int32_t* __restrict__ mask, const double* __restrict__ hp,
                            double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                            double* __restrict__ g, const double* __restrict__ beta, double* __restrict__ hn,
                            int32_t* __restrict__ kdone, int32_t* __restrict__ any) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || !mask[s]) return;
    double* Hs = H + s * (m + 1) * m;
    double* c = cs + s * m;
    double* sv = sn + s * m;
    double* gs = g + s * (m + 1);
    const double wn = sqrt(fmax(hp[s * (m + 1) + j + 1], 0.0));
    hn[s] = wn;
    Hs[(j + 1) * m + j] = wn;
    for (int i = 0; i < j; ++i) {
        const double a = Hs[i * m + j], bb = Hs[(i + 1) * m + j];
        Hs[i * m + j] = c[i] * a + sv[i] * bb;
        Hs[(i + 1) * m + j] = -sv[i] * a + c[i] * bb;
    }
    const double a = Hs[j * m + j], bb = Hs[(j + 1) * m + j];
    const double rho = hypot(a, bb);
    const double cj = rho > 0.0 ? a / rho : 1.0, sj = rho > 0.0 ? bb / rho : 0.0;
    c[j] = cj;
    sv[j] = sj;
    Hs[j * m + j] = rho;
    Hs[(j + 1) * m + j] = 0.0;
    gs[j + 1] = -sj * gs[j];
    gs[j] = cj * gs[j];
    kdone[s] = j + 1;
    if (!(fabs(gs[j + 1]) > kGmresEta * beta[s]) || !(wn > 0.0) || j + 1 == m)
        mask[s] = 0;
    else
        atomicAdd(any, 1);
}

// V_j+1 = w / ||w|| on systems still iterating
__global__ void k_gm_next(const int32_t* __restrict__ row_sys, int32_t n_pats, int64_t n,
                          const int32_t* __restrict__ mask, const double* __restrict__ hn, double* __restrict__ w) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int b = blockIdx.y;
    const int s = b * n_pats + row_sys[r];
    if (!mask[s]) return;
    const int64_t o = (int64_t)b * n + r;
    w[o] /= hn[s];
}

// y = R^-1 g over the k = kdone rotated columns (upper triangular R), per system
__global__ void k_gm_backsolve(int64_t S, int m, const int32_t* __restrict__ active, const double* __restrict__ H,
                               const double* __restrict__ g, const int32_t* __restrict__ kdone,
                               double* __restrict__ y) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || !active[s]) return;
    const double* Hs = H + s * (m + 1) * m;
    const double* gs = g + s * (m + 1);
    double* ys = y + s * m;
    const int k = kdone[s];
    for (int i = k - 1; i >= 0; --i) {
        double acc = gs[i];
        for (int l = i + 1; l < k; ++l) acc -= Hs[i * m + l] * ys[l];
        const double d = Hs[i * m + i];
        ys[i] = d != 0.0 ? acc / d : 0.0;
    }
}

// x += sum_{i < k} y_i z_i
__global__ void k_gm_update(const double* __restrict__ Z, int64_t vstride, const int32_t* __restrict__ row_sys,
                            int32_t n_pats, int64_t n, const int32_t* __restrict__ active,
                            const int32_t* __restrict__ kdone, int m, const double* __restrict__ y,
                            double* __restrict__ xp) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int b = blockIdx.y;
    const int s = b * n_pats + row_sys[r];
    if (!active[s]) return;
    const int64_t o = (int64_t)b * n + r;
    const double* ys = y + (int64_t)s * m;
    double acc = 0.0;
    for (int i = 0; i < kdone[s]; ++i) acc += ys[i] * Z[i * vstride + o];
    xp[o] += acc;
}

// Systems that stopped with NO_CONVERGE are handed to the GMRES phase:
// active again, status OK, stagnation history reset.
__global__ void k_gm_reopen(int64_t S, int32_t* __restrict__ active, int32_t* __restrict__ sstatus,
                            double* __restrict__ r1, double* __restrict__ r2, int32_t* __restrict__ any) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    if (sstatus[s] == SSCO_ERR_NO_CONVERGE) {
        active[s] = 1;
        sstatus[s] = SSCO_OK;
        r1[s] = INFINITY;
        r2[s] = INFINITY;
        atomicAdd(any, 1);
    }
}

// Sets the refinement loop's condition (any system still active) and counts
// the corrections done; one thread.  Used inside a captured CUDA graph.
__global__ void k_set_cond(cudaGraphConditionalHandle h, const int32_t* __restrict__ anyp, int32_t* __restrict__ it_ctr) {
    cudaGraphSetConditional(h, *anyp > 0 ? 1u : 0u);
    *it_ctr += 1;
}

// --------------------------------------------------------------------------
// a7: adjoint reductions (original ordering)
// --------------------------------------------------------------------------
__global__ void k_grad_atwa(const DevTables t, int64_t nrows, const double* __restrict__ mu,
                            const double* __restrict__ x, int64_t n, double* __restrict__ vbar, int64_t m) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nrows) return;
    const int b = blockIdx.y;
    const double* mb = mu + (int64_t)b * n;
    const double* xb = x + (int64_t)b * n;
    double am = 0.0, ax = 0.0;
    for (int64_t q = t.g_rowptr[g]; q < t.g_rowptr[g + 1]; ++q) {
        const double a = t.g_aval[q];
        am += a * mb[t.g_colind[q]];
        ax += a * xb[t.g_colind[q]];
    }
    vbar[(int64_t)b * m + t.g_rows_all[g]] = -am * ax;
}

__global__ void k_grad_elem(const DevTables t, int64_t nelem, const double* __restrict__ mu,
                            const double* __restrict__ x, int64_t n, double* __restrict__ vbar, int64_t m) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nelem) return;
    const int b = blockIdx.y;
    const double* mb = mu + (int64_t)b * n;
    const double* xb = x + (int64_t)b * n;
    const int dim = t.e_dim[g];
    const int32_t* dofs = t.e_dofs + t.e_off[g];
    const double* K0 = t.e_K0 + t.e_k0off[g];
    double acc = 0.0;
    int p = 0;
    for (int i = 0; i < dim; ++i) {
        const int u = dofs[i];
        for (int j = 0; j <= i; ++j, ++p) {
            const int v = dofs[j];
            if (u < 0 || v < 0) continue;
            double c = mb[u] * xb[v];
            if (i != j) c += mb[v] * xb[u];
            acc += K0[p] * c;
        }
    }
    vbar[(int64_t)b * m + t.e_elems_all[g]] = -acc;
}

__global__ void k_shift_bar(const DevTables t, int32_t n_pats, int64_t n, const double* __restrict__ mu,
                            const double* __restrict__ x, double* __restrict__ sbar) {
    const int s = blockIdx.x;
    const int b = s / n_pats, k = s % n_pats;
    const double* mb = mu + (int64_t)b * n;
    const double* xb = x + (int64_t)b * n;
    double sum = 0.0, mx = 0.0;
    for (int64_t i = t.sys_n_off[k] + threadIdx.x; i < t.sys_n_off[k + 1]; i += blockDim.x)
        if (t.shifted[i]) {
            const int o = t.perm[i];
            sum += mb[o] * xb[o];
        }
    block_sum_max(sum, mx);
    if (threadIdx.x == 0) sbar[s] = -sum;
}

// --------------------------------------------------------------------------
inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

template <class T>
T* wsp(Plan& P, size_t off) {
    return reinterpret_cast<T*>(P.d_ws + off);
}

// Brackets one launch with two pooled events when profiling is on.
struct Prof {
    Plan& P;
    cudaStream_t s;
    int kind;
    int ev = -1;
    Prof(Plan& p, cudaStream_t st, int k) : P(p), s(st), kind(k) {
        P.launches++;
        if (P.prof && P.ev_used + 2 <= P.ev_pool.size()) {
            ev = (int)P.ev_used;
            P.ev_used += 2;
            cudaEventRecord((cudaEvent_t)P.ev_pool[ev], s);
        }
    }
    bool ended = false;
    // Records the end event; call right after the launch, before any host
    // work, so that host time is not charged to the kernel.
    void end() {
        if (ev >= 0 && !ended) {
            cudaEventRecord((cudaEvent_t)P.ev_pool[ev + 1], s);
            ended = true;
        }
    }
    void done(double flops, double bytes) {
        if (ev < 0) return;
        end();
        P.prof_recs.push_back(ProfRec{kind, ev, flops, bytes});
    }
};

// algorithmic work of one launch over a front list (host, profiling only)
struct Work {
    double flops = 0, bytes = 0;
};

Work work_front_small(const Plan& P, const LaunchList& ll) {
    Work w;
    for (int32_t q = 0; q < ll.count; ++q) {
        const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + q]];
        for (int32_t j = 0; j < d.w; ++j) w.flops += (double)(d.r - j) * (d.r - j);
        double ru = d.r - d.w;
        w.bytes += d.klist_n * 16.0 + ((double)d.r * d.w + ru * (ru + 1) / 2) * P.tsize;
        for (int32_t c = 0; c < d.nchild; ++c) {
            const FrontDesc& cd = P.fronts[P.child_ids[d.child_off + c]];
            double rc = cd.r - cd.w;
            w.bytes += rc * (rc + 1) / 2 * P.tsize + rc * 4;
        }
    }
    w.flops *= P.B;
    w.bytes *= P.B;
    return w;
}

Work work_solve(const Plan& P, const LaunchList& ll) {
    Work w;
    for (int32_t q = 0; q < ll.count; ++q) {
        const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + q]];
        double ent = (double)d.r * d.w - (double)d.w * (d.w - 1) / 2;
        w.flops += 2 * ent;
        w.bytes += ent * P.tsize + 2.0 * d.r * P.tsize;
    }
    w.flops *= P.B;
    w.bytes *= P.B;
    return w;
}

Work work_tiny(const Plan& P, bool solve) {
    Work w;
    for (int32_t f : P.tiny_list) {
        const FrontDesc& d = P.fronts[f];
        double ent = (double)d.r * d.w - (double)d.w * (d.w - 1) / 2;
        if (solve) {
            w.flops += 2 * ent;
            w.bytes += ent * P.tsize + 2.0 * d.r * P.tsize;
        } else {
            for (int32_t j = 0; j < d.w; ++j) w.flops += (double)(d.r - j) * (d.r - j);
            double ru = d.r - d.w;
            w.bytes += d.klist_n * 16.0 + ((double)d.r * d.w + ru * (ru + 1) / 2) * P.tsize * 2;
        }
    }
    w.flops *= P.B;
    w.bytes *= P.B;
    return w;
}

// algorithmic work of one factorization dataflow launch (its fronts, as
// work_front_small counts them) and of one dataflow solve sweep
Work work_flow_group(const Plan& P, const FlowGroup& g) {
    Work w;
    for (int32_t q = 0; q < g.count; ++q) {
        const FrontDesc& d = P.fronts[P.flow_fact[g.off + q]];
        for (int32_t j = 0; j < d.w; ++j) w.flops += (double)(d.r - j) * (d.r - j);
        double ru = d.r - d.w;
        w.bytes += d.klist_n * 16.0 + ((double)d.r * d.w - (double)d.w * (d.w - 1) / 2 + ru * (ru + 1) / 2) * P.tsize;
        for (int32_t c = 0; c < d.nchild; ++c) {
            const FrontDesc& cd = P.fronts[P.child_ids[d.child_off + c]];
            double rc = cd.r - cd.w;
            w.bytes += rc * (rc + 1) / 2 * P.tsize + rc * 4;
        }
    }
    w.flops *= P.B;
    w.bytes *= P.B;
    return w;
}

Work work_flow_solve(const Plan& P) {
    Work w;
    for (int32_t F : P.flow_solve) {
        const FrontDesc& d = P.fronts[F];
        double ent = (double)d.r * d.w - (double)d.w * (d.w - 1) / 2;
        w.flops += 2 * ent;
        w.bytes += ent * P.tsize + 2.0 * d.r * P.tsize;
    }
    w.flops *= P.B;
    w.bytes *= P.B;
    return w;
}

// Grid of a persistent dataflow launch: as many CTAs as fit on the device
// at once (more would only find the ticket counter exhausted), at most one
// per item.
template <class Kern>
unsigned flow_grid(Kern kernel, int threads, size_t smem, int64_t items) {
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) per = 1;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)per * n_sm));
}

// Host mirror of big_update_tile (ts > 0) or tc_update_tile (ts = 0): tiles
// of one front's update, and the update's multiply-adds (entries x K) and
// algorithmic bytes.
struct UpdShape {
    int64_t tiles = 0;
    double entries = 0, k = 0, rows = 0;
};
static UpdShape update_shape(const FrontDesc& d, int k0, int nk, int jend, int ts) {
    UpdShape u;
    if (k0 >= d.w) return u;
    const int k1 = std::min(k0 + nk, d.w), jlo = k1;
    const int jhi = jend < 0 ? d.r : std::min(jend, d.w);
    if (jhi <= jlo) return u;
    int64_t nrt, nct;
    if (ts > 0) {
        nrt = (d.r - jlo + ts - 1) / ts;
        nct = (jhi - jlo + ts - 1) / ts;
    } else {
        nrt = (d.r + 127) / 128 - jlo / 128;
        nct = (jhi + 127) / 128 - jlo / 128;
    }
    u.tiles = jend < 0 ? nrt * (nrt + 1) / 2 : nrt * nct;
    const double nc = jhi - jlo, m = d.r - jlo;
    u.entries = nc * m - nc * (nc - 1) / 2;
    u.k = k1 - k0;
    u.rows = m;
    return u;
}

// Tensor-core operand blocks of a big-front level are written (by
// k_big_trsm) and used when the factor is FP32, tensor cores are enabled and
// the panel block fits the blocks' chunk slots.
inline bool tc_level(const Plan& P, int tsize, int SB) {
    return tsize == 4 && P.tune.use_tc && P.tc_pack_total > 0 && SB <= kTcMaxPanel;
}

// One update of every front of a big-front level (see big_update_tile):
// F[i, j] -= L[i, k0:k1) L[j, k0:k1)^T; tensor cores (operand blocks of the
// panel block starting at column kpack0) for FP32 when enabled, SIMT
// otherwise.
template <class T>
void launch_big_update(Plan& P, const LaunchList& ll, const int32_t* list, int kpack0, int k0, int nk, int jend,
                       T* panel, T* upd, bool tc, cudaStream_t s) {
    const int B = P.B;
    const bool tcore = tc && (ll.rmax - k0) >= P.tune.tc_min_rows;
    const bool wide = sizeof(T) == 4 && jend < 0;
    const int ts = tcore ? 0 : (wide ? 128 : 64);
    int64_t tiles = 0;
    double fl = 0, by = 0;
    for (int32_t q = 0; q < ll.count; ++q) {
        const UpdShape u = update_shape(P.fronts[P.flow_rest[ll.list_off + q]], k0, nk, jend, ts);
        tiles = std::max(tiles, u.tiles);
        fl += 2 * u.entries * u.k;
        by += (2 * u.entries + u.rows * u.k) * P.tsize;
    }
    if (tiles == 0) return;
    if (tcore && jend < 0 && P.tune.use_tc >= 2 && kpack0 == k0) {
        int64_t npairs = 0;
        for (int32_t q = 0; q < ll.count; ++q) {
            const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + q]];
            if (k0 >= d.w) continue;
            const int jlo = std::min(k0 + nk, d.w);
            if (jlo >= d.r) continue;
            npairs = std::max(npairs, tcp_pairs((d.r + 127) / 128 - jlo / 128));
        }
        const int64_t items = npairs * ll.count * B;
        if (items == 0) return;
        static int n_sm = 0;
        if (n_sm == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
            if (n_sm <= 0) n_sm = 1;
        }
        Prof pu(P, s, SSCO_K_BIG_UPDATE_TC);
        k_big_update_tcp<<<(unsigned)std::min<int64_t>(items, n_sm), 288, kTcpSmem, s>>>(
            P.dt, list, ll.count, B, npairs, k0, nk, wsp<float>(P, P.ws.tcpack), P.tc_pack_total,
            reinterpret_cast<float*>(panel), P.panel_total, reinterpret_cast<float*>(upd), P.upd_total,
            wsp<int32_t>(P, P.ws.dev_err));
        if (pu.ev >= 0) pu.done(fl * B, by * B);
    } else if (tcore) {
        Prof pu(P, s, SSCO_K_BIG_UPDATE_TC);
        k_big_update_tc<<<dim3((unsigned)tiles, ll.count, B), 288, kTcSmem, s>>>(
            P.dt, list, kpack0, k0, nk, jend, wsp<float>(P, P.ws.tcpack), P.tc_pack_total,
            reinterpret_cast<float*>(panel), P.panel_total, reinterpret_cast<float*>(upd), P.upd_total,
            wsp<int32_t>(P, P.ws.dev_err));
        if (pu.ev >= 0) pu.done(fl * B, by * B);
    } else if (wide) {
        Prof pu(P, s, SSCO_K_BIG_GEMM);
        k_big_update_f32<<<dim3((unsigned)tiles, ll.count, B), 256, 0, s>>>(
            P.dt, list, k0, nk, jend, reinterpret_cast<float*>(panel), P.panel_total, reinterpret_cast<float*>(upd),
            P.upd_total);
        if (pu.ev >= 0) pu.done(fl * B, by * B);
    } else {
        Prof pu(P, s, SSCO_K_BIG_GEMM);
        k_big_update<T><<<dim3((unsigned)tiles, ll.count, B), 256, 0, s>>>(P.dt, list, k0, nk, jend, panel,
                                                                          P.panel_total, upd, P.upd_total);
        if (pu.ev >= 0) pu.done(fl * B, by * B);
    }
}

// Creates the plan's auxiliary streams and events on first use; returns how
// many are available (0 if creation failed, or while per-launch profiling is
// on, so that each launch's events time that kernel alone: everything then
// runs on the caller's stream).
inline int ensure_aux_streams(Plan& P) {
    if (P.prof) return 0;
    if (!P.aux_fork) {
        cudaEvent_t f;
        if (cudaEventCreateWithFlags(&f, cudaEventDisableTiming) != cudaSuccess) return 0;
        for (int i = 0; i < 4; ++i) {
            cudaStream_t st;
            cudaEvent_t e;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return 0;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return 0;
            P.aux_stream[i] = st;
            P.aux_join[i] = e;
        }
        P.aux_fork = f;
    }
    return 4;
}

template <class T>
int run_numeric(Plan& P, const void* vals, int32_t vdt, const double* shift, cudaStream_t s) {
    const int B = P.B;
    const int64_t S = (int64_t)B * P.n_pats;
    double* K = wsp<double>(P, P.ws.K);
    T* panel = wsp<T>(P, P.ws.panel);
    T* upd = wsp<T>(P, P.ws.upd);
    int32_t* bad = wsp<int32_t>(P, P.ws.bad_col);
    {
        Prof pr(P, s, SSCO_K_VECTOR);
        k_fill_i32<<<cdiv(S, 256), 256, 0, s>>>(bad, S, INT_MAX);
        pr.done(0, S * 4.0);
    }
    cudaMemsetAsync(P.d_ws + P.ws.dev_err, 0, 4, s);
    if (!P.chunks.empty()) {
        Prof pr(P, s, SSCO_K_ASSEMBLE);
        dim3 g((unsigned)P.chunks.size(), B);
        if (vdt == SSCO_VALS_F64)
            k_assemble<double><<<g, 256, 0, s>>>(P.dt.groups, P.dt.chunks, P.dt.asm_idx, P.dt.asm_coef,
                                                 (const double*)vals, P.m, shift, P.n_pats, K, P.nnzK);
        else
            k_assemble<float><<<g, 256, 0, s>>>(P.dt.groups, P.dt.chunks, P.dt.asm_idx, P.dt.asm_coef,
                                                (const float*)vals, P.m, shift, P.n_pats, K, P.nnzK);
        pr.end();
        if (pr.ev >= 0) {
            double fl = 0, by = 0, sv = vdt == SSCO_VALS_F64 ? 8 : 4;
            for (const AsmGroup& g2 : P.groups) {
                double t = (double)g2.nmem * g2.nterms;
                fl += 2 * t;
                by += t * (4 + sv + (g2.uniform ? 0 : 8)) + g2.nmem * 8.0;
            }
            pr.done(fl * B, by * B);
        }
    }
    if (P.n_tiny > 0) {
        Prof pr(P, s, SSCO_K_FRONT_TINY);
        const int64_t items = (int64_t)P.n_tiny * B;
        const bool share = tiny_share(B);
        k_tiny_factor<T><<<cdiv(items, kTinyWarps), 32 * kTinyWarps,
                           tiny_factor_bytes<T>(share, P.tiny_prog_max, P.tiny_k_max), s>>>(
            P.dt, P.n_tiny, B, P.tiny_prog_max, P.tiny_k_max, K, P.nnzK, panel, P.panel_total, upd, P.upd_total, bad,
            P.n_pats, share ? 1 : 0);
        pr.end();
        if (pr.ev >= 0) {
            Work w = work_tiny(P, false);
            pr.done(w.flops, w.bytes);
        }
    }
    // Small fronts below every big front: one persistent dataflow launch per
    // size group (children wait through done flags, not level boundaries).
    const bool fflow = (P.tune.flow & 2) && !P.fact_groups.empty() && (int64_t)P.flow_fact.size() * B < (1LL << 30);
    if (fflow) {
        int32_t* fl = wsp<int32_t>(P, P.ws.flow_fact);
        cudaMemsetAsync(fl, 0, 128 + (size_t)B * P.flow_fact.size() * 4, s);
        for (size_t gi = 0; gi < P.fact_groups.size(); ++gi) {
            const FlowGroup& g = P.fact_groups[gi];
            const size_t smem =
                ((size_t)kFlowNB * kFlowNB + kFlowNB + (size_t)g.rmax * (g.rmax + 1) / 2 + kSmallPad) * g.V * sizeof(T);
            const int64_t items = (int64_t)g.count * ((B + g.V - 1) / g.V);
            const int stall = gi == 0 ? P.tune.flow_stall : -1;
            const int th = 32 * g.nw;
            int32_t* derr = wsp<int32_t>(P, P.ws.dev_err);
            Prof pr(P, s, g.V > 1 ? SSCO_K_FRONT_VEC : SSCO_K_FRONT_SMALL);
#define SSCO_FLOW_LAUNCH(VV)                                                                                     \
    k_front_flow<T, VV><<<flow_grid(k_front_flow<T, VV>, th, smem, items), th, smem, s>>>(                      \
        P.dt, P.dt.flow_fact + g.off, g.off, g.count, B, K, P.nnzK, panel, P.panel_total, upd, P.upd_total, bad, \
        P.n_pats, fl, (int)gi, derr, P.tune.flow_polls, stall)
            // (the shared memory above is sized for g.V: exactly the
            // instantiation launched; build_flow makes g.V one of 1, 2 or 4,
            // 4 only for FP32)
            if (g.V == 1)
                SSCO_FLOW_LAUNCH(1);
            else if (g.V == 2)
                SSCO_FLOW_LAUNCH(2);
            else if (g.V == 4 && sizeof(T) == 4)
                SSCO_FLOW_LAUNCH(sizeof(T) == 4 ? 4 : 2);
            else
                return (int)cudaErrorInvalidConfiguration;
#undef SSCO_FLOW_LAUNCH
            pr.end();
            if (pr.ev >= 0) {
                Work w = work_flow_group(P, g);
                pr.done(w.flops, w.bytes);
            }
        }
    }
    const std::vector<LaunchList>& FL = fflow ? P.fact_rest : P.fact_launches;
    // The launch lists of one level (the size classes of small fronts, the
    // big fronts) are independent: all but the last go to the plan's
    // auxiliary streams, forked from s at the level's start and joined back
    // at the next level's (in a captured graph: parallel branches).
    const int n_aux = ensure_aux_streams(P);
    size_t lvl_begin = 0, lvl_end = 0;
    int nl = 0;
    auto join_level = [&]() {
        if (nl <= 1) return;
        for (int k = 0; k < std::min(nl - 1, n_aux); ++k) {
            cudaEventRecord((cudaEvent_t)P.aux_join[k], (cudaStream_t)P.aux_stream[k]);
            cudaStreamWaitEvent(s, (cudaEvent_t)P.aux_join[k], 0);
        }
    };
    for (size_t li = 0; li < FL.size(); ++li) {
        const LaunchList& ll = FL[li];
        if (li == lvl_end) {
            join_level();
            lvl_begin = li;
            lvl_end = li;
            while (lvl_end < FL.size() && FL[lvl_end].level == ll.level) ++lvl_end;
            nl = n_aux > 0 ? (int)(lvl_end - lvl_begin) : 1;
            if (nl > 1) {
                cudaEventRecord((cudaEvent_t)P.aux_fork, s);
                for (int k = 0; k < std::min(nl - 1, n_aux); ++k)
                    cudaStreamWaitEvent((cudaStream_t)P.aux_stream[k], (cudaEvent_t)P.aux_fork, 0);
            }
        }
        const int kk = (int)(li - lvl_begin);
        cudaStream_t st = (nl > 1 && kk < nl - 1) ? (cudaStream_t)P.aux_stream[kk % n_aux] : s;
        const int32_t* list = P.dt.flow_rest + ll.list_off;
        if (ll.cls > 0) {
            constexpr int V = sizeof(T) == 4 ? 4 : 2;
            if (ll.cls <= P.tune.warp_front_max && ll.rmax <= 64 && (int64_t)ll.count * B >= P.tune.warp_items) {
                Prof pr(P, st, SSCO_K_FRONT_SMALL);
                const int64_t items = (int64_t)ll.count * B;
                k_front_warp<T><<<cdiv(items, 8), 256, 8 * (size_t)ll.rmax * (ll.rmax + 1) / 2 * sizeof(T), st>>>(
                    P.dt, list, ll.count, B, ll.rmax, K, P.nnzK, panel, P.panel_total, upd, P.upd_total, bad,
                    P.n_pats);
                pr.end();
                if (pr.ev >= 0) {
                    Work w = work_front_small(P, ll);
                    pr.done(w.flops, w.bytes);
                }
                continue;
            }
            if (P.tune.front_core == 1) {
                // the dataflow kernel's core (three barriers per 16-column
                // panel), one CTA per (front, value-set group) of this list
                const int fV = ll.rmax <= 64 ? (sizeof(T) == 4 ? 4 : 2) : (ll.rmax <= 128 && sizeof(T) == 4 ? 2 : 1);
                int gV = fV;
                while (gV > 1 && gV > B) gV /= 2;
                const int th = ll.rmax <= 64 ? 128 : 256;
                const size_t fsm = ((size_t)kFlowNB * kFlowNB + kFlowNB + (size_t)ll.rmax * (ll.rmax + 1) / 2 +
                                    kSmallPad) * gV * sizeof(T);
                const unsigned grid = (unsigned)((int64_t)ll.count * ((B + gV - 1) / gV));
                int32_t* derr = wsp<int32_t>(P, P.ws.dev_err);
                Prof pr(P, st, gV > 1 ? SSCO_K_FRONT_VEC : SSCO_K_FRONT_SMALL);
                if (gV == 1)
                    k_front_flow<T, 1><<<grid, th, fsm, st>>>(P.dt, list, 0, ll.count, B, K, P.nnzK, panel,
                                                             P.panel_total, upd, P.upd_total, bad, P.n_pats, nullptr,
                                                             -1, derr, 0, -1);
                else if (gV == 2 || sizeof(T) == 8)
                    k_front_flow<T, 2><<<grid, th, fsm, st>>>(P.dt, list, 0, ll.count, B, K, P.nnzK, panel,
                                                             P.panel_total, upd, P.upd_total, bad, P.n_pats, nullptr,
                                                             -1, derr, 0, -1);
                else
                    k_front_flow<T, sizeof(T) == 4 ? 4 : 2><<<grid, th, fsm, st>>>(
                        P.dt, list, 0, ll.count, B, K, P.nnzK, panel, P.panel_total, upd, P.upd_total, bad, P.n_pats,
                        nullptr, -1, derr, 0, -1);
                pr.end();
                if (pr.ev >= 0) {
                    Work w = work_front_small(P, ll);
                    pr.done(w.flops, w.bytes);
                }
                continue;
            }
            const bool vec = ll.cls <= P.tune.vec_max_cls && B >= V;
            // FP32 classes above vec_max_cls: two value sets per CTA up to
            // vec2_max_cls (the index loads and barriers shared by two)
            const bool vec2 = !vec && sizeof(T) == 4 && ll.cls <= P.tune.vec2_max_cls && B >= 2;
            Prof pr(P, st, vec || vec2 ? SSCO_K_FRONT_VEC : SSCO_K_FRONT_SMALL);
            const int nw = ll.cls <= 32 ? 2 : (ll.cls <= 64 ? 4 : 8);
            const size_t smem = ((size_t)ll.rmax * (ll.rmax + 1) / 2 + kSmallPad) * sizeof(T);
            if (vec)
                k_front_vec<T, V><<<dim3(ll.count, (B + V - 1) / V), dim3(32, nw), smem * V, st>>>(
                    P.dt, list, B, K, P.nnzK, panel, P.panel_total, upd, P.upd_total, bad, P.n_pats);
            else if (vec2)
                k_front_vec<T, 2><<<dim3(ll.count, (B + 1) / 2), dim3(32, nw), smem * 2, st>>>(
                    P.dt, list, B, K, P.nnzK, panel, P.panel_total, upd, P.upd_total, bad, P.n_pats);
            else
                k_front_small<T><<<dim3(ll.count, B), dim3(32, nw), smem, st>>>(
                    P.dt, list, K, P.nnzK, panel, P.panel_total, upd, P.upd_total, bad, P.n_pats);
            pr.end();
            if (pr.ev >= 0) {
                Work w = work_front_small(P, ll);
                pr.done(w.flops, w.bytes);
            }
            continue;
        }
        {
            Prof pr(P, st, SSCO_K_BIG_INIT);
            k_big_init<T><<<dim3((unsigned)ll.max_lower_tiles, ll.count, B), 256, 0, st>>>(
                P.dt, list, panel, P.panel_total, upd, P.upd_total);
            pr.end();
            if (pr.ev >= 0) {
                double by = 0;
                for (int32_t q = 0; q < ll.count; ++q) {
                    const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + q]];
                    by += (double)d.r * (d.r + 1) / 2 * P.tsize;
                    for (int32_t c = 0; c < d.nchild; ++c) {
                        const FrontDesc& cd = P.fronts[P.child_ids[d.child_off + c]];
                        double rc = cd.r - cd.w;
                        by += rc * (rc + 1) / 2 * P.tsize + d.r * 4.0;
                    }
                }
                pr.done(0, by * B);
            }
        }
        {
            Prof pr(P, st, SSCO_K_BIG_KSCATTER);
            k_big_kscatter<T><<<dim3(cdiv(ll.max_klist, 256), ll.count, B), 256, 0, st>>>(P.dt, list, K, P.nnzK,
                                                                                       panel, P.panel_total);
            pr.end();
            if (pr.ev >= 0) {
                double by = 0;
                for (int32_t q = 0; q < ll.count; ++q)
                    by += P.fronts[P.flow_rest[ll.list_off + q]].klist_n * (16.0 + 2 * P.tsize);
                pr.done(0, by * B);
            }
        }
        // Panel blocks of P.tune.big_panel columns: each 32-column step is
        // factored (potrf, trsm) and applied only to the rest of its block
        // (narrow update, K = 32); the finished block then updates the whole
        // trailing triangle in one pass with K = big_panel, so the trailing
        // entries are read and written once per block instead of once per
        // 32 columns.
        // With tune.big_fuse every step but the level's last factors its
        // diagonal block inside the trsm launch (the block reaching the panel
        // one step later through a scratch slot); the last step keeps the
        // separate potrf, which also writes back the previous step's block.
        const int SB = std::max(32, P.tune.big_panel / 32 * 32);
        const bool tc = tc_level(P, (int)sizeof(T), SB);
        const int kb_last = (ll.wmax - 1) / 32;
        T* diag = wsp<T>(P, P.ws.diag);
        for (int C0 = 0; C0 < ll.wmax; C0 += SB) {
            const int Cend = C0 + SB;
            for (int c0 = C0; c0 < std::min(Cend, (int)ll.wmax); c0 += 32) {
                const int kb = c0 / 32;
                const bool fused = P.tune.big_fuse && kb < kb_last && (size_t)ll.count * B <= P.ws.diag_slots;
                if (!fused) {
                    Prof pd(P, st, SSCO_K_BIG_POTRF);
                    k_big_potrf<T><<<dim3(ll.count, B), 32, 0, st>>>(P.dt, list, kb, panel, P.panel_total, bad,
                                                                     P.n_pats,
                                                                     P.tune.big_fuse && kb >= 1 &&
                                                                             (size_t)ll.count * B <= P.ws.diag_slots
                                                                         ? diag
                                                                         : nullptr);
                    pd.end();
                    if (pd.ev >= 0) {
                        double fl = 0, by = 0;
                        for (int32_t q = 0; q < ll.count; ++q) {
                            const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + q]];
                            if (c0 >= d.w) continue;
                            double nbk = std::min(32, d.w - c0);
                            fl += nbk * nbk * nbk / 3;
                            by += nbk * nbk * P.tsize;
                        }
                        pd.done(fl * B, by * B);
                    }
                }
                {
                    Prof pr(P, st, SSCO_K_BIG_TRSM);
                    k_big_trsm<T><<<dim3(cdiv(ll.rmax - c0, 256), ll.count, B), 256, 0, st>>>(
                        P.dt, list, kb, panel, P.panel_total, tc ? wsp<float>(P, P.ws.tcpack) : nullptr,
                        P.tc_pack_total, C0, fused ? diag : nullptr, bad, P.n_pats);
                    pr.end();
                    if (pr.ev >= 0) {
                        double fl = 0, by = 0;
                        for (int32_t q = 0; q < ll.count; ++q) {
                            const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + q]];
                            if (c0 >= d.w) continue;
                            double nbk = std::min(32, d.w - c0), mrows = d.r - c0 - nbk;
                            fl += mrows * nbk * nbk + (fused ? nbk * nbk * nbk / 3 : 0);
                            by += 2 * (mrows + nbk) * nbk * P.tsize;
                        }
                        pr.done(fl * B, by * B);
                    }
                }
                if (c0 + 32 < Cend) launch_big_update<T>(P, ll, list, C0, c0, 32, Cend, panel, upd, tc, st);
            }
            launch_big_update<T>(P, ll, list, C0, C0, SB, -1, panel, upd, tc, st);
        }
    }
    join_level();
    return (int)cudaGetLastError();
}

// --------------------------------------------------------------------------
// a5': split solves of the largest fronts.  A level supplies only
// (fronts x instances) CTAs to the kernels above, and near the root that is
// a few dozen for fronts of millions of entries.  A front with r >=
// split_rows is instead solved by a sequence of launches over 256-column
// blocks, each spreading the block's dense update over many CTAs of 256
// threads (one per 256 rows or columns); the CTA that owns the next block
// then solves that block's 256 x 256 triangle, so each block costs one
// launch.  Same arithmetic as the kernels above (blocked substitution with
// the same factor), grouped differently.
// --------------------------------------------------------------------------
constexpr int kSplitCB = 256;

// v[0 .. nrows) := L_bb^{-1} v for the diagonal block at (jb0, jb0); all
// threads of the CTA take part.
template <class T>
__device__ void split_fwd_diag(const T* __restrict__ Pb, int r, int jb0, int nrows, T* v, T (*Ld)[33], T* dinv,
                               T* yblk) {
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int s = 0; s < nrows; s += 32) {
        const int nbk = min(32, nrows - s);
        stage_diag(Ld, dinv, Pb, r, jb0 + s, nbk, tid, nth);
        __syncthreads();
        if (tid < 32) {
            const int l = tid;
            T val = l < nbk ? v[s + l] : T(0);
            for (int j = 0; j < nbk; ++j) {
                const T yj = __shfl_sync(0xffffffffu, val, j) * dinv[j];
                if (l == j) val = yj;
                if (l > j) val -= Ld[l][j] * yj;
            }
            if (l < nbk) {
                v[s + l] = val;
                yblk[l] = val;
            }
        }
        __syncthreads();
        for (int i = s + nbk + tid; i < nrows; i += nth) {
            const T* col = Pb + (int64_t)(jb0 + s) * r + jb0 + i;
            T a0 = T(0), a1 = T(0);
            int j = 0;
            for (; j + 1 < nbk; j += 2) {
                a0 += col[(int64_t)j * r] * yblk[j];
                a1 += col[(int64_t)(j + 1) * r] * yblk[j + 1];
            }
            if (j < nbk) a0 += col[(int64_t)j * r] * yblk[j];
            v[i] -= a0 + a1;
        }
        __syncthreads();
    }
}

// x[0 .. ncols) := L_bb^{-T} x for the diagonal block at (jb0, jb0), x
// holding the block's right-hand side with every row past the block
// already applied; all threads of the CTA take part.
template <class T>
__device__ void split_bwd_diag(const T* __restrict__ Pb, int r, int jb0, int ncols, T* x, T (*Ld)[33], T* dinv,
                               T* dots) {
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
    for (int sb = (ncols + 31) / 32 - 1; sb >= 0; --sb) {
        const int s = sb * 32, nbk = min(32, ncols - s);
        stage_diag(Ld, dinv, Pb, r, jb0 + s, nbk, tid, nth);
        for (int c = warp; c < nbk; c += nw) {
            const T* col = Pb + (int64_t)(jb0 + s + c) * r + jb0;
            T acc = T(0);
            for (int i = s + nbk + lane; i < ncols; i += 32) acc += col[i] * x[i];
            acc = warp_sum(acc);
            if (lane == 0) dots[c] = acc;
        }
        __syncthreads();
        if (tid < 32) {
            const int l = tid;
            T val = l < nbk ? x[s + l] - dots[l] : T(0);
            for (int j = nbk - 1; j >= 0; --j) {
                const T xj = __shfl_sync(0xffffffffu, val, j) * dinv[j];
                if (l == j) val = xj;
                if (l < j) val -= Ld[j][l] * xj;
            }
            if (l < nbk) x[s + l] = val;
        }
        __syncthreads();
    }
}

// Forward, first launch: CTA p gathers rows 256p.. of the front's vector
// (own right-hand side plus the children's passing vectors, pulled through
// the inverse maps in child order); CTA 0 then solves column block 0.
template <class T>
__global__ void __launch_bounds__(256) k_fsplit_init(const DevTables t, const int32_t* __restrict__ list,
                                                     const T* __restrict__ panel, int64_t panel_total,
                                                     T* __restrict__ vec, int64_t n, T* __restrict__ pvec,
                                                     int64_t pvec_total, const int32_t* __restrict__ active,
                                                     int32_t n_pats) {
    const FrontDesc d = t.fronts[list[blockIdx.y]];
    const int b = blockIdx.z;
    if (active && !active[(int64_t)b * n_pats + d.sys]) return;
    const int r = d.r, w = d.w;
    const int row0 = (int)blockIdx.x * kSplitCB;
    if (row0 >= r) return;
    __shared__ T v[kSplitCB];
    __shared__ T Ld[32][33];
    __shared__ T dinv[32], yblk[32];
    __shared__ int64_t coff[32];
    const int tid = threadIdx.x;
    T* vb = vec + (int64_t)b * n;
    T* pv = pvec + (int64_t)b * pvec_total;
    const int i = row0 + tid;
    T val = (i < r && i < w) ? vb[d.f + i] : T(0);
    for (int cb = 0; cb < d.nchild; cb += 32) {
        const int nc = min(32, d.nchild - cb);
        __syncthreads();
        if (tid < nc) coff[tid] = t.fronts[t.child_ids[d.child_off + cb + tid]].pvec_off;
        __syncthreads();
        if (i < r)
            for (int c = 0; c < nc; ++c) {
                const int a = t.invmap[d.inv_off + (int64_t)(cb + c) * r + i];
                if (a >= 0) val += pv[coff[c] + a];
            }
    }
    if (blockIdx.x == 0) {
        v[tid] = val;
        __syncthreads();
        split_fwd_diag(panel + (int64_t)b * panel_total + d.panel_off, r, 0, min(kSplitCB, w), v, Ld, dinv, yblk);
        val = v[tid];
    }
    if (i < r) {
        if (i < w)
            vb[d.f + i] = val;
        else
            pv[d.pvec_off + i - w] = val;
    }
}

// Forward, column block k (columns c0 = 256k .. e): rows e .. r take
// v_i -= L[i, c0:e) y, 256 rows per CTA; CTA 0 then solves block k + 1.
template <class T>
__global__ void __launch_bounds__(256) k_fsplit_step(const DevTables t, const int32_t* __restrict__ list, int k,
                                                     const T* __restrict__ panel, int64_t panel_total,
                                                     T* __restrict__ vec, int64_t n, T* __restrict__ pvec,
                                                     int64_t pvec_total, const int32_t* __restrict__ active,
                                                     int32_t n_pats) {
    const FrontDesc d = t.fronts[list[blockIdx.y]];
    const int b = blockIdx.z;
    if (active && !active[(int64_t)b * n_pats + d.sys]) return;
    const int r = d.r, w = d.w;
    const int c0 = k * kSplitCB;
    if (c0 >= w) return;
    const int nbk = min(kSplitCB, w - c0), e = c0 + nbk;
    const int row0 = e + (int)blockIdx.x * kSplitCB;
    if (row0 >= r) return;
    __shared__ T y[kSplitCB], v[kSplitCB];
    __shared__ T Ld[32][33];
    __shared__ T dinv[32], yblk[32];
    const int tid = threadIdx.x;
    T* vb = vec + (int64_t)b * n;
    T* pv = pvec + (int64_t)b * pvec_total;
    const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    if (tid < nbk) y[tid] = vb[d.f + c0 + tid];
    __syncthreads();
    const int i = row0 + tid;
    T val = T(0);
    if (i < r) {
        val = i < w ? vb[d.f + i] : pv[d.pvec_off + i - w];
        const T* col = Pb + (int64_t)c0 * r + i;
        T acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = T(0);
        int j = 0;
        for (; j + 7 < nbk; j += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += col[(int64_t)(j + u) * r] * y[j + u];
        }
        for (; j < nbk; ++j) acc[0] += col[(int64_t)j * r] * y[j];
        val -= ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    }
    if (blockIdx.x == 0 && e < w) {
        v[tid] = val;
        __syncthreads();
        split_fwd_diag(Pb, r, e, min(kSplitCB, w - e), v, Ld, dinv, yblk);
        val = v[tid];
    }
    if (i < r) {
        if (i < w)
            vb[d.f + i] = val;
        else
            pv[d.pvec_off + i - w] = val;
    }
}

// Backward, first launch: the solution at the update rows w .. r (the
// parent's, final) is staged in shared memory; CTA p takes columns 256p..
// x_j -= L[w:r, j]^T x[w:r] (warp per column); the CTA of the last column
// block then solves it.
template <class T>
__global__ void __launch_bounds__(256) k_bsplit_init(const DevTables t, const int32_t* __restrict__ list,
                                                     const T* __restrict__ panel, int64_t panel_total,
                                                     T* __restrict__ vec, int64_t n,
                                                     const int32_t* __restrict__ active, int32_t n_pats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xr = reinterpret_cast<T*>(smem_raw);
    const FrontDesc d = t.fronts[list[blockIdx.y]];
    const int b = blockIdx.z;
    if (active && !active[(int64_t)b * n_pats + d.sys]) return;
    const int r = d.r, w = d.w, ru = r - w;
    const int col0 = (int)blockIdx.x * kSplitCB;
    if (col0 >= w) return;
    const int ncols = min(kSplitCB, w - col0);
    __shared__ T xs[kSplitCB];
    __shared__ T Ld[32][33];
    __shared__ T dinv[32], dots[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T* vb = vec + (int64_t)b * n;
    const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    const int32_t* rows = t.rows + d.rows_off;
    for (int k = tid; k < ru; k += kSplitCB) xr[k] = vb[rows[w + k]];
    __syncthreads();
    for (int c = warp; c < ncols; c += kSplitCB / 32) {
        const T* col = Pb + (int64_t)(col0 + c) * r + w;
        T a0 = T(0), a1 = T(0);
        int q = lane;
        for (; q + 32 < ru; q += 64) {
            a0 += col[q] * xr[q];
            a1 += col[q + 32] * xr[q + 32];
        }
        if (q < ru) a0 += col[q] * xr[q];
        const T s = warp_sum(a0 + a1);
        if (lane == 0) xs[c] = vb[d.f + col0 + c] - s;
    }
    __syncthreads();
    if (col0 + kSplitCB >= w) split_bwd_diag(Pb, r, col0, ncols, xs, Ld, dinv, dots);
    if (tid < ncols) vb[d.f + col0 + tid] = xs[tid];
}

// Backward, column block k (rows c0 = 256k .. e hold final x): CTA p takes
// columns 256p .. (< c0), x_j -= L[c0:e, j]^T x[c0:e] (warp per column);
// the CTA of block k - 1 then solves it.
template <class T>
__global__ void __launch_bounds__(256) k_bsplit_step(const DevTables t, const int32_t* __restrict__ list, int k,
                                                     const T* __restrict__ panel, int64_t panel_total,
                                                     T* __restrict__ vec, int64_t n,
                                                     const int32_t* __restrict__ active, int32_t n_pats) {
    const FrontDesc d = t.fronts[list[blockIdx.y]];
    const int b = blockIdx.z;
    if (active && !active[(int64_t)b * n_pats + d.sys]) return;
    const int r = d.r, w = d.w;
    const int c0 = k * kSplitCB;
    if (c0 >= w) return;
    const int nbk = min(kSplitCB, w - c0);
    const int col0 = (int)blockIdx.x * kSplitCB;
    if (col0 >= c0) return;
    __shared__ T xk[kSplitCB], xs[kSplitCB];
    __shared__ T Ld[32][33];
    __shared__ T dinv[32], dots[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T* vb = vec + (int64_t)b * n;
    const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    if (tid < nbk) xk[tid] = vb[d.f + c0 + tid];
    __syncthreads();
    for (int c = warp; c < kSplitCB; c += kSplitCB / 32) {
        const T* col = Pb + (int64_t)(col0 + c) * r + c0;
        T a0 = T(0), a1 = T(0);
        int q = lane;
        for (; q + 32 < nbk; q += 64) {
            a0 += col[q] * xk[q];
            a1 += col[q + 32] * xk[q + 32];
        }
        if (q < nbk) a0 += col[q] * xk[q];
        const T s = warp_sum(a0 + a1);
        if (lane == 0) xs[c] = vb[d.f + col0 + c] - s;
    }
    __syncthreads();
    if (col0 + kSplitCB == c0) split_bwd_diag(Pb, r, col0, kSplitCB, xs, Ld, dinv, dots);
    vb[d.f + col0 + tid] = xs[tid];
}

// --------------------------------------------------------------------------
// a5'': cluster solves.  A front with r >= cluster_rows is solved by one
// thread-block cluster of kClusterCS CTAs (one per SM) per value set: the
// front's rows are dealt to the CTAs in 32-row chunks (chunk c to rank
// c mod CS, kept in that CTA's shared memory), so the front's panel is
// read by CS SMs at once.  Per 32-column block one CTA -- the owner of the
// block's rows -- solves the block's triangle; the forward solve writes the
// block's y into every CTA's shared memory (distributed shared memory) and
// all CTAs update their own rows after one cluster barrier; the backward
// solve reduces the CTAs' partial dot products into the owner the same
// way.  One hardware cluster barrier per block; no launch per block.
// --------------------------------------------------------------------------
constexpr int kClusterCS = 8;
namespace cg = cooperative_groups;

// Local slot of front row i in its owner's chunk store.
__device__ __forceinline__ int cl_slot(int i) { return (i >> 5) / kClusterCS * 32 + (i & 31); }

template <class T>
__global__ void __launch_bounds__(256) k_fwd_cluster(const DevTables t, const int32_t* __restrict__ list,
                                                     const T* __restrict__ panel, int64_t panel_total,
                                                     T* __restrict__ vec, int64_t n, T* __restrict__ pvec,
                                                     int64_t pvec_total, const int32_t* __restrict__ active,
                                                     int32_t n_pats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* vl = reinterpret_cast<T*>(smem_raw);  // this CTA's chunks of the front vector
    __shared__ T ybuf[2][32];
    __shared__ int64_t coff[32];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const FrontDesc d = t.fronts[list[blockIdx.x / kClusterCS]];
    const int b = blockIdx.y;
    if (active && !active[(int64_t)b * n_pats + d.sys]) return;  // uniform over the cluster
    const int r = d.r, w = d.w, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nch = (r + 31) / 32;
    T* vb = vec + (int64_t)b * n;
    T* pv = pvec + (int64_t)b * pvec_total;
    const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    // own rows: right-hand side plus the children's passing vectors
    for (int cb = 0; cb < d.nchild; cb += 32) {
        const int nc = min(32, d.nchild - cb);
        __syncthreads();
        if (tid < nc) coff[tid] = t.fronts[t.child_ids[d.child_off + cb + tid]].pvec_off;
        __syncthreads();
        for (int c = rank + kClusterCS * (tid >> 5); c < nch; c += kClusterCS * 8) {
            const int i = 32 * c + lane;
            if (i >= r) continue;
            T val = cb == 0 ? (i < w ? vb[d.f + i] : T(0)) : vl[cl_slot(i)];
            for (int q = 0; q < nc; ++q) {
                const int a = t.invmap[d.inv_off + (int64_t)(cb + q) * r + i];
                if (a >= 0) val += pv[coff[q] + a];
            }
            vl[cl_slot(i)] = val;
        }
    }
    if (d.nchild == 0)
        for (int c = rank + kClusterCS * (tid >> 5); c < nch; c += kClusterCS * 8) {
            const int i = 32 * c + lane;
            if (i < r) vl[cl_slot(i)] = i < w ? vb[d.f + i] : T(0);
        }
    __syncthreads();
    cl.sync();  // every CTA of the cluster is running before any remote write
    const int nb = (w + 31) / 32;
    for (int k = 0; k < nb; ++k) {
        const int c0 = 32 * k, nbk = min(32, w - c0), buf = k & 1;
        if (k % kClusterCS == rank) {
            __syncthreads();  // this CTA's updates of the block's rows are done
            if (warp == 0) {
                T a[32];
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    a[j] = (j < nbk && lane < nbk) ? Pb[(int64_t)(c0 + j) * r + c0 + lane] : T(0);
                T val = lane < nbk ? vl[cl_slot(c0 + lane)] : T(0);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if (j < nbk) {
                        const T dj = __shfl_sync(0xffffffffu, a[j], j);
                        const T yj = __shfl_sync(0xffffffffu, val, j) / dj;
                        if (lane == j)
                            val = yj;
                        else if (lane > j)
                            val -= a[j] * yj;
                    }
                }
                if (lane < nbk) {
                    vl[cl_slot(c0 + lane)] = val;
                    for (int rk = 0; rk < kClusterCS; ++rk) cl.map_shared_rank(&ybuf[buf][0], rk)[lane] = val;
                }
            }
        }
        cl.sync();  // y of block k in every CTA
        // own rows past the block (chunks >= k): v_i -= L[i, block] y
        const int cfirst = k + ((rank - k % kClusterCS + kClusterCS) % kClusterCS);
        for (int c = cfirst + kClusterCS * (tid >> 5); c < nch; c += kClusterCS * 8) {
            const int i = 32 * c + lane;
            if (i < c0 + nbk || i >= r) continue;
            const T* col = Pb + (int64_t)c0 * r + i;
            T acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = T(0);
            int j = 0;
            for (; j + 7 < nbk; j += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] += col[(int64_t)(j + u) * r] * ybuf[buf][j + u];
            }
            for (; j < nbk; ++j) acc[0] += col[(int64_t)j * r] * ybuf[buf][j];
            vl[cl_slot(i)] -= ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        }
    }
    __syncthreads();
    for (int c = rank + kClusterCS * (tid >> 5); c < nch; c += kClusterCS * 8) {
        const int i = 32 * c + lane;
        if (i >= r) continue;
        if (i < w)
            vb[d.f + i] = vl[cl_slot(i)];
        else
            pv[d.pvec_off + i - w] = vl[cl_slot(i)];
    }
    cl.sync();  // no CTA leaves while a remote write to it may be pending
}

template <class T>
__global__ void __launch_bounds__(256) k_bwd_cluster(const DevTables t, const int32_t* __restrict__ list,
                                                     const T* __restrict__ panel, int64_t panel_total,
                                                     T* __restrict__ vec, int64_t n,
                                                     const int32_t* __restrict__ active, int32_t n_pats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xl = reinterpret_cast<T*>(smem_raw);
    __shared__ T part[2][kClusterCS][32];
    __shared__ T wpart[8][32];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const FrontDesc d = t.fronts[list[blockIdx.x / kClusterCS]];
    const int b = blockIdx.y;
    if (active && !active[(int64_t)b * n_pats + d.sys]) return;
    const int r = d.r, w = d.w, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nch = (r + 31) / 32;
    T* vb = vec + (int64_t)b * n;
    const T* Pb = panel + (int64_t)b * panel_total + d.panel_off;
    const int32_t* rows = t.rows + d.rows_off;
    for (int c = rank + kClusterCS * (tid >> 5); c < nch; c += kClusterCS * 8) {
        const int i = 32 * c + lane;
        if (i < r) xl[cl_slot(i)] = i < w ? vb[d.f + i] : vb[rows[i]];
    }
    __syncthreads();
    cl.sync();
    const int nb = (w + 31) / 32;
    for (int k = nb - 1; k >= 0; --k) {
        const int c0 = 32 * k, nbk = min(32, w - c0), buf = k & 1, owner = k % kClusterCS;
        __syncthreads();  // x of this CTA's rows (the owner's last solve) visible
        // partial dots of the block's columns over own rows past the block:
        // warp q takes own chunks q, q + 8, ...; lane = row; then per column
        // a warp sum, the 8 warps combined in shared memory.
        T acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = T(0);
        const int cfirst = k + ((rank - k % kClusterCS + kClusterCS) % kClusterCS);
        for (int c = cfirst + kClusterCS * warp; c < nch; c += kClusterCS * 8) {
            const int i = 32 * c + lane;
            if (i < c0 + nbk || i >= r) continue;
            const T xi = xl[cl_slot(i)];
            const T* rowp = Pb + (int64_t)c0 * r + i;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < nbk) acc[j] += rowp[(int64_t)j * r] * xi;
        }
#pragma unroll
        for (int sh = 16; sh >= 1; sh >>= 1) {
            const bool up = (lane & sh) != 0;
#pragma unroll
            for (int j = 0; j < sh; ++j) {
                const T send = up ? acc[j] : acc[j + sh];
                const T keep = up ? acc[j + sh] : acc[j];
                acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, sh);
            }
        }
        wpart[warp][lane] = acc[0];  // column `lane`'s sum over this warp's rows
        __syncthreads();
        if (warp == 0) {
            T sum = T(0);
#pragma unroll
            for (int q = 0; q < 8; ++q) sum += wpart[q][lane];
            cl.map_shared_rank(&part[buf][0][0], owner)[rank * 32 + lane] = sum;
        }
        cl.sync();  // all partials of block k at its owner
        if (rank == owner && warp == 0) {
            T a[32];
#pragma unroll
            for (int j = 0; j < 32; ++j)
                a[j] = (lane < nbk && j < nbk && j >= lane) ? Pb[(int64_t)(c0 + lane) * r + c0 + j] : T(0);
            T dot = T(0);
#pragma unroll
            for (int q = 0; q < kClusterCS; ++q) dot += part[buf][q][lane];
            T val = lane < nbk ? xl[cl_slot(c0 + lane)] - dot : T(0);
#pragma unroll
            for (int j = 31; j >= 0; --j) {
                if (j < nbk) {
                    const T dj = __shfl_sync(0xffffffffu, a[j], j);
                    const T xj = __shfl_sync(0xffffffffu, val, j) / dj;
                    if (lane == j)
                        val = xj;
                    else if (lane < j)
                        val -= a[j] * xj;
                }
            }
            if (lane < nbk) xl[cl_slot(c0 + lane)] = val;
        }
    }
    __syncthreads();
    for (int c = rank + kClusterCS * (tid >> 5); c < nch; c += kClusterCS * 8) {
        const int i = 32 * c + lane;
        if (i < w) vb[d.f + i] = xl[cl_slot(i)];
    }
    cl.sync();
}

// A level is solved warp-per-item when it supplies at least 8 warps per SM
// and its fronts' vectors fit 8 to a CTA; otherwise one CTA per item.
inline bool use_warp_solve(const Plan& P, const LaunchList& ll, int B) {
    return (int64_t)ll.count * B >= P.tune.warp_items && ll.rmax <= 1024;
}
inline int solve_threads(const Plan& P, const LaunchList& ll) {
    return ll.rmax <= 128 ? 128 : (ll.rmax <= 512 ? 256 : P.tune.solve_threads_big);
}

// Leading fronts of a solve level (sorted by rows, largest first) that take
// the split solves: r >= split_rows, a big front (inverse maps present) whose
// update rows fit the backward kernel's shared memory.
inline int split_count(const Plan& P, const LaunchList& ll) {
    const int thr = std::max(P.tune.split_rows, P.small_max + 1);
    int q = 0;
    while (q < ll.count) {
        const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + q]];
        if (d.r < thr || (d.nchild > 0 && d.inv_off < 0) || (size_t)(d.r - d.w) * P.tsize > 160 * 1024) break;
        ++q;
    }
    return q;
}

// Fronts after the split ones (positions q0 ..) of a solve level that take
// the cluster solves: r >= cluster_rows, a big front with inverse maps.
inline int cluster_count(const Plan& P, const LaunchList& ll, int q0) {
    const int thr = std::max(P.tune.cluster_rows, P.small_max + 1);
    int q = q0;
    while (q < ll.count) {
        const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + q]];
        if (d.r < thr || (d.nchild > 0 && d.inv_off < 0)) break;
        ++q;
    }
    return q - q0;
}

template <class T, class Kern, class... Args>
void launch_cluster(Plan& P, Kern kernel, int nfront, int B, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(kClusterCS * nfront), (unsigned)B, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kClusterCS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int e = (int)cudaLaunchKernelEx(&cfg, kernel, args...);
    if (e && !P.launch_err) P.launch_err = e;
}

template <class T>
size_t cluster_smem(const Plan& P, const LaunchList& ll, int q0, int q) {
    int rmax = 0;
    for (int f = q0; f < q0 + q; ++f) rmax = std::max(rmax, P.fronts[P.flow_rest[ll.list_off + f]].r);
    const int nch = (rmax + 31) / 32;
    return (size_t)((nch + kClusterCS - 1) / kClusterCS) * 32 * sizeof(T);
}

template <class T>
void run_split_fwd(Plan& P, const LaunchList& ll, int q, const int32_t* active, cudaStream_t s) {
    const int B = P.B;
    const int32_t* list = P.dt.flow_rest + ll.list_off;
    T* panel = wsp<T>(P, P.ws.panel);
    T* vecT = wsp<T>(P, P.ws.vecT);
    T* pvec = wsp<T>(P, P.ws.pvec);
    int rmax = 0, wmax = 0;
    double by0 = 0, fl0 = 0;
    for (int f = 0; f < q; ++f) {
        const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + f]];
        rmax = std::max(rmax, d.r);
        wmax = std::max(wmax, d.w);
        const double nb0 = std::min(kSplitCB, d.w);
        fl0 += nb0 * nb0;
        by0 += (nb0 * (nb0 + 1) / 2 + d.r * (2.0 + d.nchild)) * P.tsize + d.r * 4.0 * d.nchild;
    }
    {
        Prof pr(P, s, SSCO_K_FWD);
        k_fsplit_init<T><<<dim3(cdiv(rmax, kSplitCB), q, B), kSplitCB, 0, s>>>(
            P.dt, list, panel, P.panel_total, vecT, P.n, pvec, P.pvec_total, active, P.n_pats);
        if (pr.ev >= 0) pr.done(fl0 * B, by0 * B);
    }
    const int nb = cdiv(wmax, kSplitCB);
    for (int k = 0; k < nb; ++k) {
        int64_t g = 0;
        double fl = 0, by = 0;
        for (int f = 0; f < q; ++f) {
            const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + f]];
            const int c0 = k * kSplitCB;
            if (c0 >= d.w) continue;
            const int e = std::min(c0 + kSplitCB, d.w);
            g = std::max<int64_t>(g, cdiv(d.r - e, kSplitCB));
            const double nbk = e - c0, m = d.r - e, nn = std::min(kSplitCB, d.w - e);
            fl += 2 * m * nbk + (e < d.w ? nn * nn : 0);
            by += (m * nbk + (e < d.w ? nn * (nn + 1) / 2 : 0) + 2 * m + nbk) * P.tsize;
        }
        if (g == 0) continue;
        Prof pr(P, s, SSCO_K_FWD);
        k_fsplit_step<T><<<dim3((unsigned)g, q, B), kSplitCB, 0, s>>>(P.dt, list, k, panel, P.panel_total, vecT,
                                                                       P.n, pvec, P.pvec_total, active, P.n_pats);
        if (pr.ev >= 0) pr.done(fl * B, by * B);
    }
}

template <class T>
void run_split_bwd(Plan& P, const LaunchList& ll, int q, const int32_t* active, cudaStream_t s) {
    const int B = P.B;
    const int32_t* list = P.dt.flow_rest + ll.list_off;
    T* panel = wsp<T>(P, P.ws.panel);
    T* vecT = wsp<T>(P, P.ws.vecT);
    int wmax = 0, rumax = 0;
    double by0 = 0, fl0 = 0;
    for (int f = 0; f < q; ++f) {
        const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + f]];
        wmax = std::max(wmax, d.w);
        rumax = std::max(rumax, d.r - d.w);
        const double ru = d.r - d.w, nl = d.w - (double)((d.w - 1) / kSplitCB) * kSplitCB;
        fl0 += 2 * ru * d.w + nl * nl;
        by0 += (ru * d.w + nl * (nl + 1) / 2 + 2.0 * d.w + ru * cdiv(d.w, kSplitCB)) * P.tsize + ru * 4.0;
    }
    const int nb = cdiv(wmax, kSplitCB);
    {
        Prof pr(P, s, SSCO_K_BWD);
        k_bsplit_init<T><<<dim3(nb, q, B), kSplitCB, (size_t)rumax * sizeof(T), s>>>(
            P.dt, list, panel, P.panel_total, vecT, P.n, active, P.n_pats);
        if (pr.ev >= 0) pr.done(fl0 * B, by0 * B);
    }
    for (int k = nb - 1; k >= 1; --k) {
        double fl = 0, by = 0;
        for (int f = 0; f < q; ++f) {
            const FrontDesc& d = P.fronts[P.flow_rest[ll.list_off + f]];
            const int c0 = k * kSplitCB;
            if (c0 >= d.w) continue;
            const double nbk = std::min(kSplitCB, d.w - c0);
            fl += 2 * nbk * c0 + (double)kSplitCB * kSplitCB;
            by += (nbk * c0 + (double)kSplitCB * (kSplitCB + 1) / 2 + 2.0 * c0 + nbk) * P.tsize;
        }
        Prof pr(P, s, SSCO_K_BWD);
        k_bsplit_step<T><<<dim3(k, q, B), kSplitCB, 0, s>>>(P.dt, list, k, panel, P.panel_total, vecT, P.n, active,
                                                             P.n_pats);
        if (pr.ev >= 0) pr.done(fl * B, by * B);
    }
}

template <class T>
void run_trisolve(Plan& P, const int32_t* active, cudaStream_t s) {
    const int B = P.B;
    T* panel = wsp<T>(P, P.ws.panel);
    T* vecT = wsp<T>(P, P.ws.vecT);
    T* pvec = wsp<T>(P, P.ws.pvec);
    const unsigned tiny_grid = cdiv((int64_t)P.n_tiny * B, kTinyWarps);
    // fronts of at most flow_solve_rmax rows below every larger front: one
    // persistent dataflow launch per sweep (warp per front and value set)
    const bool sflow = (P.tune.flow & 1) && !P.flow_solve.empty() && (int64_t)P.flow_solve.size() * B < (1LL << 30);
    int32_t* sfl = wsp<int32_t>(P, P.ws.flow_solve);
    int32_t* derr = wsp<int32_t>(P, P.ws.dev_err);
    // items of G value sets (one warp each) per CTA
    const int G = std::min(8, B);
    const size_t fsmem = (size_t)G * P.flow_solve_rmax * sizeof(T);
    const int64_t fitems = (int64_t)P.flow_solve.size() * ((B + G - 1) / G);
    if (sflow) cudaMemsetAsync(sfl, 0, 128 + (size_t)P.flow_solve.size() * B * 4, s);
    if (P.n_tiny > 0) {
        Prof pr(P, s, SSCO_K_FWD);
        k_tiny_fwd<T><<<tiny_grid, 32 * kTinyWarps, tiny_solve_bytes<T>(tiny_share(B), P.tiny_prog_max), s>>>(
            P.dt, P.n_tiny, B, P.tiny_prog_max, panel, P.panel_total, vecT, P.n, pvec, P.pvec_total, active,
            P.n_pats, tiny_share(B) ? 1 : 0);
        pr.end();
        if (pr.ev >= 0) {
            Work w = work_tiny(P, true);
            pr.done(w.flops, w.bytes);
        }
    }
    if (sflow) {
        Prof pr(P, s, SSCO_K_FWD);
        k_flow_fwd<T><<<flow_grid(k_flow_fwd<T>, 32 * G, fsmem, fitems), 32 * G, fsmem, s>>>(
            P.dt, (int32_t)P.flow_solve.size(), B, P.flow_solve_rmax, panel, P.panel_total, vecT, P.n, pvec,
            P.pvec_total, active, P.n_pats, sfl, derr, P.tune.flow_polls, P.tune.flow_stall);
        pr.end();
        if (pr.ev >= 0) {
            Work w = work_flow_solve(P);
            pr.done(w.flops, w.bytes);
        }
    }
    const std::vector<LaunchList>& SL = sflow ? P.solve_rest : P.solve_launches;
    for (const LaunchList& ll0 : SL) {
        LaunchList ll = ll0;
        const int q = split_count(P, ll);
        if (q > 0) run_split_fwd<T>(P, ll, q, active, s);
        const int qc = cluster_count(P, ll, q);
        if (qc > 0) {
            Prof pr(P, s, SSCO_K_FWD);
            const int32_t* lst = P.dt.flow_rest + ll.list_off + q;
            launch_cluster<T>(P, k_fwd_cluster<T>, qc, B, cluster_smem<T>(P, ll, q, qc), s, P.dt, lst,
                              (const T*)panel, P.panel_total, vecT, P.n, pvec, P.pvec_total, active, P.n_pats);
            pr.end();
            if (pr.ev >= 0) {
                LaunchList sub = ll;
                sub.list_off += q;
                sub.count = qc;
                Work w = work_solve(P, sub);
                pr.done(w.flops, w.bytes);
            }
        }
        if (q + qc > 0) {
            ll.list_off += q + qc;
            ll.count -= q + qc;
            if (ll.count == 0) continue;
            ll.rmax = P.fronts[P.flow_rest[ll.list_off]].r;
        }
        Prof pr(P, s, SSCO_K_FWD);
        const size_t smem = (size_t)ll.rmax * sizeof(T);
        if (use_warp_solve(P, ll, B)) {
            const int64_t items = (int64_t)ll.count * B;
            auto kf = ll.wmax <= 16 ? k_fwd_warp<T, 16> : k_fwd_warp<T, 32>;
            kf<<<cdiv(items, 8), 256, 8 * smem, s>>>(P.dt, P.dt.flow_rest + ll.list_off, ll.count, B, ll.rmax, panel,
                                                     P.panel_total, vecT, P.n, pvec, P.pvec_total, active, P.n_pats);
        } else
            k_fwd<T><<<dim3(ll.count, B), solve_threads(P, ll), smem, s>>>(
                P.dt, P.dt.flow_rest + ll.list_off, panel, P.panel_total, vecT, P.n, pvec, P.pvec_total, active,
                P.n_pats);
        pr.end();
        if (pr.ev >= 0) {
            Work w = work_solve(P, ll);
            pr.done(w.flops, w.bytes);
        }
    }
    for (auto it = SL.rbegin(); it != SL.rend(); ++it) {
        LaunchList ll = *it;
        const int q = split_count(P, ll);
        if (q > 0) run_split_bwd<T>(P, ll, q, active, s);
        const int qc = cluster_count(P, ll, q);
        if (qc > 0) {
            Prof pr(P, s, SSCO_K_BWD);
            const int32_t* lst = P.dt.flow_rest + ll.list_off + q;
            launch_cluster<T>(P, k_bwd_cluster<T>, qc, B, cluster_smem<T>(P, ll, q, qc), s, P.dt, lst,
                              (const T*)panel, P.panel_total, vecT, P.n, active, P.n_pats);
            pr.end();
            if (pr.ev >= 0) {
                LaunchList sub = ll;
                sub.list_off += q;
                sub.count = qc;
                Work w = work_solve(P, sub);
                pr.done(w.flops, w.bytes);
            }
        }
        if (q + qc > 0) {
            ll.list_off += q + qc;
            ll.count -= q + qc;
            if (ll.count == 0) continue;
            ll.rmax = P.fronts[P.flow_rest[ll.list_off]].r;
        }
        Prof pr(P, s, SSCO_K_BWD);
        const size_t smem = (size_t)ll.rmax * sizeof(T);
        if (use_warp_solve(P, ll, B)) {
            const int64_t items = (int64_t)ll.count * B;
            auto kb = ll.wmax <= 16 ? k_bwd_warp<T, 16> : k_bwd_warp<T, 32>;
            kb<<<cdiv(items, 8), 256, 8 * smem, s>>>(P.dt, P.dt.flow_rest + ll.list_off, ll.count, B, ll.rmax, panel,
                                                     P.panel_total, vecT, P.n, active, P.n_pats);
        } else
            k_bwd<T><<<dim3(ll.count, B), solve_threads(P, ll), smem, s>>>(
                P.dt, P.dt.flow_rest + ll.list_off, panel, P.panel_total, vecT, P.n, active, P.n_pats);
        pr.end();
        if (pr.ev >= 0) {
            Work w = work_solve(P, ll);
            pr.done(w.flops, w.bytes);
        }
    }
    if (sflow) {
        Prof pr(P, s, SSCO_K_BWD);
        k_flow_bwd<T><<<flow_grid(k_flow_bwd<T>, 32 * G, fsmem, fitems), 32 * G, fsmem, s>>>(
            P.dt, (int32_t)P.flow_solve.size(), B, P.flow_solve_rmax, panel, P.panel_total, vecT, P.n, active,
            P.n_pats, sfl, derr, P.tune.flow_polls);
        pr.end();
        if (pr.ev >= 0) {
            Work w = work_flow_solve(P);
            pr.done(w.flops, w.bytes);
        }
    }
    if (P.n_tiny > 0) {
        Prof pr(P, s, SSCO_K_BWD);
        k_tiny_bwd<T><<<tiny_grid, 32 * kTinyWarps, tiny_solve_bytes<T>(tiny_share(B), P.tiny_prog_max), s>>>(
            P.dt, P.n_tiny, B, P.tiny_prog_max, panel, P.panel_total, vecT, P.n, active, P.n_pats,
            tiny_share(B) ? 1 : 0);
        pr.end();
        if (pr.ev >= 0) {
            Work w = work_tiny(P, true);
            pr.done(w.flops, w.bytes);
        }
    }
}

// One GMRES-IR correction of every active system: d = Z y from GMRES(m)
// on K d = r (r in rr from the last residual, beta = its 2-norm), then
// x += d.  Synchronizes once per inner step to stop when every system's
// residual estimate has converged.
template <class T>
int gmres_correction(Plan& P, cudaStream_t s);

// While capturing a graph: the refinement loop becomes a conditional WHILE
// node whose body is captured on body_stream.
struct GraphLoop {
    cudaStream_t body_stream;
};

// x = K^-1 b for all systems (b, x device, original ordering)
template <class T>
int run_solve(Plan& P, const double* b, double* x, cudaStream_t s, GraphLoop* gl = nullptr) {
    const int B = P.B;
    const int64_t n = P.n, S = (int64_t)B * P.n_pats;
    double* bp = wsp<double>(P, P.ws.bp);
    double* xp = wsp<double>(P, P.ws.xp);
    double* rr = wsp<double>(P, P.ws.rr);
    T* vecT = wsp<T>(P, P.ws.vecT);
    int32_t* active = wsp<int32_t>(P, P.ws.active);
    int32_t* sst = wsp<int32_t>(P, P.ws.sstatus);
    int32_t* iters = wsp<int32_t>(P, P.ws.iters);
    int32_t* anyp = wsp<int32_t>(P, P.ws.any_active);
    double* resid = wsp<double>(P, P.ws.resid);
    double* bnorm = wsp<double>(P, P.ws.bnorm);
    double* r1 = wsp<double>(P, P.ws.r1);
    double* r2 = wsp<double>(P, P.ws.r2);
    double* sigma = wsp<double>(P, P.ws.sigma);
    double* psum = wsp<double>(P, P.ws.sys_psum);
    double* pmax = wsp<double>(P, P.ws.sys_pmax);
    // per-system norms in two passes when the plan has fewer systems than SMs
    const bool chunked = S < 152 && P.ws.sys_maxc > 1;
    const double* K = wsp<double>(P, P.ws.K);
    const dim3 gv(cdiv(n, 256), B);
    const int refine = P.prec == SSCO_FP32_REFINE;
    const double nB = (double)n * B;
    const double spnz = (double)P.sp_rowptr.back() * B;
    {
        Prof pr(P, s, SSCO_K_VECTOR);
        k_permute_in<<<gv, 256, 0, s>>>(b, P.dt.perm, n, bp);
        pr.done(0, nB * 20);
    }
    {
        Prof pr(P, s, SSCO_K_CHECK);
        if (chunked) {
            k_sys_partial<<<dim3((unsigned)P.ws.sys_maxc, (unsigned)S), 256, 0, s>>>(
                bp, P.dt.sys_n_off, P.n_pats, n, P.ws.sys_maxc, nullptr, psum, pmax);
            P.launches++;
        }
        k_sys_init<<<(unsigned)S, 256, 0, s>>>(bp, n, P.dt.sys_n_off, P.n_pats, P.ws.sys_maxc, chunked ? psum : nullptr,
                                               pmax, bnorm, active, sst, iters, resid, r1, r2);
        pr.done(2 * nB, nB * 8);
    }
    {
        Prof pr(P, s, SSCO_K_VECTOR);
        k_to_T<T><<<cdiv((int64_t)B * n, 256), 256, 0, s>>>(bp, vecT, (int64_t)B * n);
        pr.done(0, nB * (8 + sizeof(T)));
    }
    run_trisolve<T>(P, nullptr, s);
    {
        Prof pr(P, s, SSCO_K_VECTOR);
        k_from_T<T><<<cdiv((int64_t)B * n, 256), 256, 0, s>>>(vecT, xp, (int64_t)B * n);
        pr.done(0, nB * (8 + sizeof(T)));
    }
    int32_t* it_ctr = wsp<int32_t>(P, P.ws.it_ctr);
    if (gl) {
        // device-side loop: prologue check, then WHILE(any active) { correct; check }
        cudaMemsetAsync(it_ctr, 0, 4, s);
        const int32_t* it_dev = it_ctr;
        auto check_step = [&](cudaStream_t st) {
            {
                Prof pr(P, st, SSCO_K_RESID);
                k_resid<<<gv, 256, 0, st>>>(P.dt.sp_rowptr, P.dt.sp_col, P.dt.sp_slot, K, P.nnzK, bp, xp, rr, n);
                pr.done(0, 0);
            }
            cudaMemsetAsync(anyp, 0, 4, st);
            Prof pc(P, st, SSCO_K_CHECK);
            if (chunked) {
                k_sys_partial<<<dim3((unsigned)P.ws.sys_maxc, (unsigned)S), 256, 0, st>>>(
                    rr, P.dt.sys_n_off, P.n_pats, n, P.ws.sys_maxc, active, psum, pmax);
                P.launches++;
            }
            k_check<<<(unsigned)S, 256, 0, st>>>(rr, n, P.dt.sys_n_off, P.n_pats, P.ws.sys_maxc,
                                                 chunked ? psum : nullptr, pmax, bnorm, active, sst, iters, resid,
                                                 r1, r2, sigma, anyp, 0, P.maxit, P.tol, refine, it_dev);
            pc.done(0, 0);
        };
        check_step(s);
        if (refine) {
            cudaStreamCaptureStatus cst;
            cudaGraph_t cg = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            const cudaGraphEdgeData* edata = nullptr;
            size_t ndeps = 0;
            int e = (int)cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, &edata, &ndeps);
            if (e) return e;
            cudaGraphConditionalHandle h;
            e = (int)cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault);
            if (e) return e;
            k_set_cond<<<1, 1, 0, s>>>(h, anyp, it_ctr);
            P.launches++;
            e = (int)cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, &edata, &ndeps);
            if (e) return e;
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cnode;
            e = (int)cudaGraphAddNode(&cnode, cg, deps, edata, ndeps, &cp);
            if (e) return e;
            e = (int)cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
            if (e) return e;
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            cudaStream_t bs = gl->body_stream;
            e = (int)cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
            if (e) return e;
            {
                Prof pr(P, bs, SSCO_K_VECTOR);
                k_cast_scaled<T><<<gv, 256, 0, bs>>>(rr, P.dt.row_sys, P.n_pats, n, active, sigma, vecT);
                pr.done(0, 0);
            }
            run_trisolve<T>(P, active, bs);
            {
                Prof pr(P, bs, SSCO_K_VECTOR);
                k_update<T><<<gv, 256, 0, bs>>>(vecT, P.dt.row_sys, P.n_pats, n, active, sigma, xp);
                pr.done(0, 0);
            }
            check_step(bs);
            k_set_cond<<<1, 1, 0, bs>>>(h, anyp, it_ctr);
            P.launches++;
            cudaGraph_t body_out = nullptr;
            e = (int)cudaStreamEndCapture(bs, &body_out);
            if (e) return e;
        }
        Prof pr(P, s, SSCO_K_VECTOR);
        k_permute_out<<<gv, 256, 0, s>>>(xp, P.dt.perm, n, x);
        pr.done(0, nB * 20);
        return (int)cudaGetLastError();
    }
    const int32_t* it_dev = nullptr;
    // refine_mode 1: every correction by GMRES-IR; 2: plain corrections,
    // then GMRES-IR for the systems those left NO_CONVERGE (with a fresh
    // budget of maxit corrections)
    bool gm_phase = refine && P.refine_mode == 1;
    int maxit = P.maxit;
    for (int it = 0;; ++it) {
        {
            Prof pr(P, s, SSCO_K_RESID);
            k_resid<<<gv, 256, 0, s>>>(P.dt.sp_rowptr, P.dt.sp_col, P.dt.sp_slot, K, P.nnzK, bp, xp, rr, n);
            pr.done(2 * spnz, (double)P.nnzK * B * 8 + spnz * 8 + nB * 24 + (double)P.sp_rowptr.back() * 8);
        }
        cudaMemsetAsync(anyp, 0, 4, s);
        {
            Prof pr(P, s, SSCO_K_CHECK);
            if (chunked) {
                k_sys_partial<<<dim3((unsigned)P.ws.sys_maxc, (unsigned)S), 256, 0, s>>>(
                    rr, P.dt.sys_n_off, P.n_pats, n, P.ws.sys_maxc, active, psum, pmax);
                P.launches++;
            }
            k_check<<<(unsigned)S, 256, 0, s>>>(rr, n, P.dt.sys_n_off, P.n_pats, P.ws.sys_maxc,
                                                chunked ? psum : nullptr, pmax, bnorm, active, sst, iters, resid,
                                                r1, r2, sigma, anyp, it, maxit, P.tol, refine, it_dev);
            pr.done(2 * nB, nB * 8);
        }
        if (!refine) break;
        int e = (int)cudaMemcpyAsync(P.h_flag, anyp, 4, cudaMemcpyDeviceToHost, s);
        if (!e) e = (int)cudaStreamSynchronize(s);
        if (e) return e;
        if (*P.h_flag == 0) {
            if (P.refine_mode != 2 || gm_phase) break;
            cudaMemsetAsync(anyp, 0, 4, s);
            k_gm_reopen<<<cdiv(S, 256), 256, 0, s>>>(S, active, sst, r1, r2, anyp);
            P.launches++;
            e = (int)cudaMemcpyAsync(P.h_flag, anyp, 4, cudaMemcpyDeviceToHost, s);
            if (!e) e = (int)cudaStreamSynchronize(s);
            if (e) return e;
            if (*P.h_flag == 0) break;
            gm_phase = true;
            maxit = it + P.maxit;
        }
        if (gm_phase) {
            e = gmres_correction<T>(P, s);
            if (e) return e;
            continue;
        }
        {
            Prof pr(P, s, SSCO_K_VECTOR);
            k_cast_scaled<T><<<gv, 256, 0, s>>>(rr, P.dt.row_sys, P.n_pats, n, active, sigma, vecT);
            pr.done(nB, nB * (12 + sizeof(T)));
        }
        run_trisolve<T>(P, active, s);
        {
            Prof pr(P, s, SSCO_K_VECTOR);
            k_update<T><<<gv, 256, 0, s>>>(vecT, P.dt.row_sys, P.n_pats, n, active, sigma, xp);
            pr.done(2 * nB, nB * (20 + sizeof(T)));
        }
    }
    {
        Prof pr(P, s, SSCO_K_VECTOR);
        k_permute_out<<<gv, 256, 0, s>>>(xp, P.dt.perm, n, x);
        pr.done(0, nB * 20);
    }
    int e = (int)cudaGetLastError();
    if (!e) e = P.launch_err;
    P.launch_err = 0;
    return e;
}

template <class T>
int gmres_correction(Plan& P, cudaStream_t s) {
    const int B = P.B, m = P.gmres_m;
    const int64_t n = P.n, S = (int64_t)B * P.n_pats, vstride = (int64_t)B * n;
    const dim3 gv(cdiv(n, 256), B);
    const unsigned gs = cdiv(S, 256);
    double* V = wsp<double>(P, P.ws.gm_V);
    double* Z = wsp<double>(P, P.ws.gm_Z);
    double* H = wsp<double>(P, P.ws.gm_H);
    double* g = wsp<double>(P, P.ws.gm_g);
    double* cs = wsp<double>(P, P.ws.gm_cs);
    double* sn = wsp<double>(P, P.ws.gm_sn);
    double* hp = wsp<double>(P, P.ws.gm_hp);
    double* y = wsp<double>(P, P.ws.gm_y);
    double* beta = wsp<double>(P, P.ws.gm_beta);
    double* hn = wsp<double>(P, P.ws.gm_hn);
    int32_t* gact = wsp<int32_t>(P, P.ws.gm_act);
    int32_t* kdone = wsp<int32_t>(P, P.ws.gm_k);
    int32_t* active = wsp<int32_t>(P, P.ws.active);
    int32_t* anyp = wsp<int32_t>(P, P.ws.any_active);
    const double* rr = wsp<double>(P, P.ws.rr);
    const double* resid = wsp<double>(P, P.ws.resid);
    const double* bnorm = wsp<double>(P, P.ws.bnorm);
    double* xp = wsp<double>(P, P.ws.xp);
    T* vecT = wsp<T>(P, P.ws.vecT);
    const double* K = wsp<double>(P, P.ws.K);
    cudaMemsetAsync(H, 0, (size_t)S * (m + 1) * m * 8, s);
    k_gm_init<<<gs, 256, 0, s>>>(S, m, active, resid, bnorm, beta, g, gact, kdone);
    k_gm_start<<<gv, 256, 0, s>>>(rr, P.dt.row_sys, P.n_pats, n, active, resid, bnorm, V);
    P.launches += 2;
    for (int j = 0; j < m; ++j) {
        double* W = V + (int64_t)(j + 1) * vstride;
        {
            Prof pr(P, s, SSCO_K_VECTOR);
            k_gm_cast<T><<<gv, 256, 0, s>>>(V + (int64_t)j * vstride, P.dt.row_sys, P.n_pats, n, gact, vecT);
            pr.done(0, (double)vstride * (8 + sizeof(T)));
        }
        run_trisolve<T>(P, gact, s);
        {
            Prof pr(P, s, SSCO_K_RESID);
            k_gm_storez<T><<<cdiv(vstride, 256), 256, 0, s>>>(vecT, vstride, Z + (int64_t)j * vstride);
            k_gm_spmv<T><<<gv, 256, 0, s>>>(P.dt.sp_rowptr, P.dt.sp_col, P.dt.sp_slot, K, P.nnzK, P.dt.row_sys,
                                           P.n_pats, n, gact, vecT, W);
            P.launches++;
            pr.done(0, 0);
        }
        {
            Prof pr(P, s, SSCO_K_CHECK);
            for (int pass = 0; pass < 2; ++pass) {  // CGS2
                k_gm_dots<<<dim3((unsigned)S, j + 1), 256, 0, s>>>(V, vstride, 0, W, P.dt.sys_n_off, P.n_pats, n,
                                                                  gact, m, hp);
                k_gm_orth<<<gv, 256, 0, s>>>(V, vstride, P.dt.row_sys, P.n_pats, n, gact, m, j, hp, W);
                k_gm_hacc<<<gs, 256, 0, s>>>(S, m, j, gact, hp, H);
                P.launches += 3;
            }
            k_gm_dots<<<dim3((unsigned)S, 1), 256, 0, s>>>(V, vstride, j + 1, W, P.dt.sys_n_off, P.n_pats, n, gact,
                                                          m, hp);
            cudaMemsetAsync(anyp, 0, 4, s);
            k_gm_givens<<<gs, 256, 0, s>>>(S, m, j, gact, hp, H, cs, sn, g, beta, hn, kdone, anyp);
            k_gm_next<<<gv, 256, 0, s>>>(P.dt.row_sys, P.n_pats, n, gact, hn, W);
            P.launches += 2;
            pr.done(0, 0);
        }
        int e = (int)cudaMemcpyAsync(P.h_flag, anyp, 4, cudaMemcpyDeviceToHost, s);
        if (!e) e = (int)cudaStreamSynchronize(s);
        if (e) return e;
        if (*P.h_flag == 0) break;
    }
    k_gm_backsolve<<<gs, 256, 0, s>>>(S, m, active, H, g, kdone, y);
    k_gm_update<<<gv, 256, 0, s>>>(Z, vstride, P.dt.row_sys, P.n_pats, n, active, kdone, m, y, xp);
    P.launches += 2;
    return (int)cudaGetLastError();
}

// Opt each kernel with dynamic shared memory into the largest size the
// device allows beside the kernel's static shared memory.
template <class K>
int allow_dynamic_smem(K kernel) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    int e = (int)cudaFuncGetAttributes(&fa, kernel);
    if (e) return e;
    return (int)cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes);
}

template <class T>
int set_attr_T() {
    int e = allow_dynamic_smem(k_front_small<T>);
    if (!e && sizeof(T) == 4) {
        e = (int)cudaFuncSetAttribute(k_big_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
        if (!e)
            e = (int)cudaFuncSetAttribute(k_big_update_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcpSmem);
    }
    if (!e) e = allow_dynamic_smem(k_front_vec<T, sizeof(T) == 4 ? 4 : 2>);
    if (!e && sizeof(T) == 4) e = allow_dynamic_smem(k_front_vec<T, 2>);
    if (!e) e = allow_dynamic_smem(k_tiny_factor<T>);
    if (!e) e = allow_dynamic_smem(k_tiny_fwd<T>);
    if (!e) e = allow_dynamic_smem(k_tiny_bwd<T>);
    if (!e) e = allow_dynamic_smem(k_fwd_warp<T, 16>);
    if (!e) e = allow_dynamic_smem(k_fwd_warp<T, 32>);
    if (!e) e = allow_dynamic_smem(k_bwd_warp<T, 16>);
    if (!e) e = allow_dynamic_smem(k_bwd_warp<T, 32>);
    if (!e) e = allow_dynamic_smem(k_fwd<T>);
    if (!e) e = allow_dynamic_smem(k_bwd<T>);
    if (!e) e = allow_dynamic_smem(k_bsplit_init<T>);
    if (!e) e = allow_dynamic_smem(k_front_warp<T>);
    if (!e) e = allow_dynamic_smem(k_fwd_cluster<T>);
    if (!e) e = allow_dynamic_smem(k_bwd_cluster<T>);
    if (!e) e = allow_dynamic_smem(k_flow_fwd<T>);
    if (!e) e = allow_dynamic_smem(k_flow_bwd<T>);
    if (!e) e = allow_dynamic_smem(k_front_flow<T, 1>);
    if (!e) e = allow_dynamic_smem(k_front_flow<T, 2>);
    if (!e && sizeof(T) == 4) e = allow_dynamic_smem(k_front_flow<T, sizeof(T) == 4 ? 4 : 2>);
    return e;
}

}  // namespace

const char* kernel_kind_name(int kind) {
    static const char* names[SSCO_K_COUNT] = {"assemble", "front_small", "big_init", "big_kscatter", "big_update",
                                              "big_potrf", "big_syrk", "fwd_solve", "bwd_solve", "resid",
                                              "check", "vector", "grad", "front_tiny", "big_trsm", "front_vec", "big_update_tc"};
    return kind >= 0 && kind < SSCO_K_COUNT ? names[kind] : "unknown";
}

int kernels_set_attributes(Plan& P) {
    int e = P.tsize == 8 ? set_attr_T<double>() : set_attr_T<float>();
    if (e) return e;
    return (int)cudaGetLastError();
}

int launch_reset_status(Plan& P, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t S = (int64_t)P.B * P.n_pats;
    k_fill_i32<<<cdiv(S, 256), 256, 0, s>>>(wsp<int32_t>(P, P.ws.bad_col), S, INT_MAX);
    k_fill_i32<<<cdiv(S, 256), 256, 0, s>>>(wsp<int32_t>(P, P.ws.sstatus), S, SSCO_OK);
    k_fill_i32<<<cdiv(S, 256), 256, 0, s>>>(wsp<int32_t>(P, P.ws.iters), S, 0);
    cudaMemsetAsync(P.d_ws + P.ws.resid, 0, (size_t)S * 8, s);
    return (int)cudaGetLastError();
}

int launch_numeric(Plan& P, const void* vals, int32_t vdt, const double* shift, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    return P.tsize == 8 ? run_numeric<double>(P, vals, vdt, shift, s) : run_numeric<float>(P, vals, vdt, shift, s);
}

// The FP32 refinement loop of a solve as a captured graph (conditional
// WHILE node, no host round trip per iteration), cached per (b, x) pair.
int solve_graph_run(Plan& P, const double* b, double* x, cudaStream_t stream) {
    int slot = -1;
    for (int i = 0; i < 2; ++i)
        if (P.s_exec[i] && P.s_key[i][0] == b && P.s_key[i][1] == x) slot = i;
    if (slot < 0) {
        slot = P.s_next;
        P.s_next ^= 1;
        if (P.s_exec[slot]) cudaGraphExecDestroy((cudaGraphExec_t)P.s_exec[slot]);
        if (P.s_graph[slot]) cudaGraphDestroy((cudaGraph_t)P.s_graph[slot]);
        P.s_exec[slot] = P.s_graph[slot] = nullptr;
        if (!P.g_stream) {
            int e = (int)cudaStreamCreateWithFlags((cudaStream_t*)&P.g_stream, cudaStreamNonBlocking);
            if (!e) e = (int)cudaStreamCreateWithFlags((cudaStream_t*)&P.g_body_stream, cudaStreamNonBlocking);
            if (e) return e;
        }
        cudaStream_t cs = (cudaStream_t)P.g_stream;
        P.launches = 0;
        int e = (int)cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e) return e;
        GraphLoop gl{(cudaStream_t)P.g_body_stream};
        const int e2 = P.tsize == 8 ? run_solve<double>(P, b, x, cs, &gl) : run_solve<float>(P, b, x, cs, &gl);
        cudaGraph_t g = nullptr;
        const int e3 = (int)cudaStreamEndCapture(cs, &g);
        if (e2 || e3) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return e2 ? e2 : e3;
        }
        cudaGraphExec_t ge = nullptr;
        e = (int)cudaGraphInstantiate(&ge, g, 0);
        if (e) {
            cudaGraphDestroy(g);
            return e;
        }
        P.s_graph[slot] = (void*)g;
        P.s_exec[slot] = (void*)ge;
        P.s_key[slot][0] = b;
        P.s_key[slot][1] = x;
        P.s_launches[slot] = P.launches;
    }
    P.launches = P.s_launches[slot];
    return (int)cudaGraphLaunch((cudaGraphExec_t)P.s_exec[slot], stream);
}

// FP32 plans with plain refinement run the solve as a captured graph (so the
// call does not synchronize); per-launch profiling, the autotuner's timings
// and plans set to no_graphs use the eager launches.
inline bool solve_by_graph(const Plan& P) {
    return P.prec == SSCO_FP32_REFINE && P.refine_mode == 0 && !P.prof && !P.eager_only && !P.no_graphs;
}

int launch_solve(Plan& P, const double* b, double* x, void* stream, bool* ok) {
    cudaStream_t s = (cudaStream_t)stream;
    *ok = true;
    if (solve_by_graph(P)) return solve_graph_run(P, b, x, s);
    return P.tsize == 8 ? run_solve<double>(P, b, x, s) : run_solve<float>(P, b, x, s);
}

// Assemble + refactor + solve as one CUDA graph (refinement loop on the
// device), captured on first use for these pointers and replayed afterwards.
template <class T>
int build_graph(Plan& P, const void* vals, int32_t vdt, const double* shift, const double* b, double* x) {
    if (!P.g_stream) {
        int e = (int)cudaStreamCreateWithFlags((cudaStream_t*)&P.g_stream, cudaStreamNonBlocking);
        if (!e) e = (int)cudaStreamCreateWithFlags((cudaStream_t*)&P.g_body_stream, cudaStreamNonBlocking);
        if (e) return e;
    }
    cudaStream_t cs = (cudaStream_t)P.g_stream;
    const bool prof = P.prof;
    P.prof = false;
    P.launches = 0;
    int e = (int)cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e) {
        P.prof = prof;
        return e;
    }
    GraphLoop gl{(cudaStream_t)P.g_body_stream};
    int e1 = run_numeric<T>(P, vals, vdt, shift, cs);
    int e2 = e1 ? e1 : run_solve<T>(P, b, x, cs, &gl);
    cudaGraph_t g = nullptr;
    int e3 = (int)cudaStreamEndCapture(cs, &g);
    P.prof = prof;
    if (e2 || e3) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return e2 ? e2 : e3;
    }
    cudaGraphExec_t ge = nullptr;
    e = (int)cudaGraphInstantiate(&ge, g, 0);
    if (e) {
        cudaGraphDestroy(g);
        return e;
    }
    P.g_graph = (void*)g;
    P.g_exec = (void*)ge;
    P.g_launches = P.launches;
    return 0;
}

void graph_release(Plan& P) {
    if (P.g_exec) cudaGraphExecDestroy((cudaGraphExec_t)P.g_exec);
    if (P.g_graph) cudaGraphDestroy((cudaGraph_t)P.g_graph);
    P.g_exec = P.g_graph = nullptr;
    if (P.m_exec) cudaGraphExecDestroy((cudaGraphExec_t)P.m_exec);
    if (P.m_graph) cudaGraphDestroy((cudaGraph_t)P.m_graph);
    P.m_exec = P.m_graph = nullptr;
    P.m_key.clear();
    for (int i = 0; i < 2; ++i) {
        if (P.s_exec[i]) cudaGraphExecDestroy((cudaGraphExec_t)P.s_exec[i]);
        if (P.s_graph[i]) cudaGraphDestroy((cudaGraph_t)P.s_graph[i]);
        P.s_exec[i] = P.s_graph[i] = nullptr;
        P.s_key[i][0] = P.s_key[i][1] = nullptr;
    }
    P.g_gen++;
}

void graph_destroy_streams(Plan& P) {
    if (P.g_stream) cudaStreamDestroy((cudaStream_t)P.g_stream);
    if (P.g_body_stream) cudaStreamDestroy((cudaStream_t)P.g_body_stream);
    P.g_stream = P.g_body_stream = nullptr;
    for (int i = 0; i < 4; ++i) {
        if (P.aux_stream[i]) cudaStreamDestroy((cudaStream_t)P.aux_stream[i]);
        if (P.aux_join[i]) cudaEventDestroy((cudaEvent_t)P.aux_join[i]);
        P.aux_stream[i] = P.aux_join[i] = nullptr;
    }
    if (P.aux_fork) cudaEventDestroy((cudaEvent_t)P.aux_fork);
    P.aux_fork = nullptr;
}

int launch_graph_run(Plan& P, const void* vals, int32_t vdt, const double* shift, const double* b, double* x,
                     void* stream) {
    if (P.refine_mode != 0) {  // the GMRES-IR loops are host-driven: eager calls
        bool ok = true;
        int e = launch_numeric(P, vals, vdt, shift, stream);
        return e ? e : launch_solve(P, b, x, stream, &ok);
    }
    const void* key[5] = {vals, shift, b, x, P.d_ws};
    bool same = P.g_exec && P.g_vdt == vdt;
    for (int i = 0; i < 5 && same; ++i) same = P.g_key[i] == key[i];
    if (!same) {
        graph_release(P);
        int e = P.tsize == 8 ? build_graph<double>(P, vals, vdt, shift, b, x)
                             : build_graph<float>(P, vals, vdt, shift, b, x);
        if (e) return e;
        for (int i = 0; i < 5; ++i) P.g_key[i] = key[i];
        P.g_vdt = vdt;
    }
    P.launches = P.g_launches;
    return (int)cudaGraphLaunch((cudaGraphExec_t)P.g_exec, (cudaStream_t)stream);
}

// Several plans' assemble + refactor + solve steps as the independent
// branches of ONE captured graph (each with its own device-side refinement
// loop): the capture forks from plans[0]'s capture stream to each plan's
// own capture stream and joins back.  Held by plans[0], re-captured when a
// plan, a pointer, a dtype or a plan's generation (bumped by every release
// of its graphs, e.g. after ssco_autotune or ssco_set_flow) changes.
template <class T>
int capture_branch(Plan& P, const void* vals, int32_t vdt, const double* shift, const double* b, double* x,
                   cudaStream_t cs) {
    GraphLoop gl{(cudaStream_t)P.g_body_stream};
    int e = run_numeric<T>(P, vals, vdt, shift, cs);
    return e ? e : run_solve<T>(P, b, x, cs, &gl);
}

int launch_graph_run_many(Plan* const* plans, int32_t n, const void* const* vals, const int32_t* vdt,
                          const double* const* shift, const double* const* b, double* const* x, void* stream) {
    for (int32_t i = 0; i < n; ++i)
        if (plans[i]->refine_mode != 0) {  // host-driven GMRES-IR loops: every plan eagerly, in turn
            for (int32_t k = 0; k < n; ++k) {
                int e = launch_graph_run(*plans[k], vals[k], vdt[k], shift[k], b[k], x[k], stream);
                if (e) return e;
            }
            return 0;
        }
    Plan& P0 = *plans[0];
    std::vector<const void*> key;
    for (int32_t i = 0; i < n; ++i) {
        const Plan& Pi = *plans[i];
        key.insert(key.end(), {(const void*)plans[i], (const void*)(uintptr_t)Pi.g_gen, vals[i], shift[i], b[i],
                               x[i], Pi.d_ws, (const void*)(intptr_t)vdt[i]});
    }
    if (!P0.m_exec || key != P0.m_key) {
        if (P0.m_exec) cudaGraphExecDestroy((cudaGraphExec_t)P0.m_exec);
        if (P0.m_graph) cudaGraphDestroy((cudaGraph_t)P0.m_graph);
        P0.m_exec = P0.m_graph = nullptr;
        P0.m_key.clear();
        for (int32_t i = 0; i < n; ++i) {
            Plan& Pi = *plans[i];
            if (!Pi.g_stream) {
                int e = (int)cudaStreamCreateWithFlags((cudaStream_t*)&Pi.g_stream, cudaStreamNonBlocking);
                if (!e) e = (int)cudaStreamCreateWithFlags((cudaStream_t*)&Pi.g_body_stream, cudaStreamNonBlocking);
                if (e) return e;
            }
        }
        cudaStream_t cs = (cudaStream_t)P0.g_stream;
        std::vector<cudaEvent_t> ev(2 * n, nullptr);
        for (auto& e1 : ev)
            if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) return (int)cudaErrorUnknown;
        std::vector<bool> prof(n);
        int64_t launches = 0;
        int err = (int)cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (!err) err = (int)cudaEventRecord(ev[0], cs);
        for (int32_t i = 0; i < n && !err; ++i) {
            Plan& Pi = *plans[i];
            cudaStream_t si = i == 0 ? cs : (cudaStream_t)Pi.g_stream;
            if (i > 0) err = (int)cudaStreamWaitEvent(si, ev[0], 0);
            prof[i] = Pi.prof;
            Pi.prof = false;
            Pi.launches = 0;
            if (!err)
                err = Pi.tsize == 8 ? capture_branch<double>(Pi, vals[i], vdt[i], shift[i], b[i], x[i], si)
                                    : capture_branch<float>(Pi, vals[i], vdt[i], shift[i], b[i], x[i], si);
            Pi.prof = prof[i];
            launches += Pi.launches;
            if (!err && i > 0) {
                err = (int)cudaEventRecord(ev[n + i], si);
                if (!err) err = (int)cudaStreamWaitEvent(cs, ev[n + i], 0);
            }
        }
        cudaGraph_t g = nullptr;
        const int e3 = (int)cudaStreamEndCapture(cs, &g);
        for (auto e1 : ev) cudaEventDestroy(e1);
        if (err || e3) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return err ? err : e3;
        }
        cudaGraphExec_t ge = nullptr;
        err = (int)cudaGraphInstantiate(&ge, g, 0);
        if (err) {
            cudaGraphDestroy(g);
            return err;
        }
        P0.m_graph = (void*)g;
        P0.m_exec = (void*)ge;
        P0.m_key = key;
        P0.m_launches = launches;
    }
    for (int32_t i = 0; i < n; ++i) plans[i]->launches = i == 0 ? P0.m_launches : 0;
    return (int)cudaGraphLaunch((cudaGraphExec_t)P0.m_exec, (cudaStream_t)stream);
}

// Coordinate descent over the dataflow-related knobs of every plan of a
// multi-plan graph, timed on that graph (ssco_graph_run_many: the plans as
// concurrent branches), so that a plan's choice accounts for the work of the
// others it overlaps with.  Each candidate re-captures the graph (the
// change releases the plan's graphs); median of `reps` replays after one
// warm-up; a candidate is kept when it is 1 % faster.
int autotune_many(Plan* const* plans, int32_t n, const void* const* vals, const int32_t* vdt,
                  const double* const* shift, const double* const* b, double* const* x, int32_t reps, void* stream,
                  double* best_ms) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    int e = (int)cudaEventCreate(&e0);
    if (!e) e = (int)cudaEventCreate(&e1);
    if (e) return e;
    auto measure = [&](double* ms_out) -> int {
        std::vector<float> t;
        for (int i = 0; i <= reps; ++i) {
            int r = (int)cudaEventRecord(e0, s);
            if (!r) r = launch_graph_run_many(plans, n, vals, vdt, shift, b, x, s);
            if (!r) r = (int)cudaEventRecord(e1, s);
            if (!r) r = (int)cudaEventSynchronize(e1);
            if (r) return r;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (i > 0) t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        *ms_out = t.empty() ? 0.0 : t[t.size() / 2];
        return 0;
    };
    double best = 0;
    e = measure(&best);
    // two sweeps: a plan's knob can pay off only after another plan's
    // knob has changed (their work overlaps in the graph)
    for (int32_t i = 0; i < 2 * n && !e; ++i) {
        Plan& P = *plans[i % n];
        struct Knob {
            int32_t* field;
            std::vector<int32_t> cand;
        };
        std::vector<Knob> knobs = {{&P.tune.flow, {0, 1, 2, 3}},
                                   {&P.tune.front_core, {0, 1}},
                                   {&P.tune.big_fuse, {0, 1}},
                                   {&P.tune.vec2_max_cls, P.tsize == 4 ? std::vector<int32_t>{0, 128, 160}
                                                                       : std::vector<int32_t>{0}}};
        for (Knob& k : knobs) {
            if (e) break;
            const int32_t keep = *k.field;
            int32_t arg = keep;
            // the current setting re-timed beside its candidates, so that a
            // lucky earlier timing does not hide a real gain of ~1 %
            double base = 0;
            if (k.cand.size() > 1) e = measure(&base);
            double arg_ms = base;
            for (int32_t c : k.cand) {
                if (e || c == keep) continue;
                *k.field = c;
                graph_release(P);
                double ms = 0;
                e = measure(&ms);
                if (e) break;
                if (ms < base * 0.995 && ms < arg_ms) {
                    arg_ms = ms;
                    arg = c;
                }
            }
            *k.field = arg;
            graph_release(P);
            if (k.cand.size() > 1) best = arg_ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms) *best_ms = best;
    return e;
}

// Coordinate descent over the launch-shape knobs: each candidate is timed
// (CUDA events, median of `reps` eager numeric + solve steps after one
// warm-up) on the caller's data; the fastest setting of each knob is kept.
int autotune(Plan& P, const void* vals, int32_t vdt, const double* shift, const double* b, double* x, int32_t reps,
             void* stream, double* best_ms) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    int e = (int)cudaEventCreate(&e0);
    if (!e) e = (int)cudaEventCreate(&e1);
    if (e) return e;
    const bool prof = P.prof;
    P.prof = false;
    P.eager_only = true;  // candidates change the launch shapes between timings
    auto measure = [&](double* ms_out) -> int {
        std::vector<float> t;
        for (int i = 0; i <= reps; ++i) {
            int r = (int)cudaEventRecord(e0, s);
            if (!r) r = launch_numeric(P, vals, vdt, shift, s);
            bool ok = true;
            if (!r) r = launch_solve(P, b, x, s, &ok);
            if (!r) r = (int)cudaEventRecord(e1, s);
            if (!r) r = (int)cudaEventSynchronize(e1);
            if (r) return r;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (i > 0) t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        *ms_out = t.empty() ? 0.0 : t[t.size() / 2];
        return 0;
    };
    struct Knob {
        int32_t* field;
        std::vector<int32_t> cand;
    };
    std::vector<Knob> knobs = {
        {&P.tune.flow, {0, 1, 2, 3}},
        {&P.tune.front_core, {0, 1}},
        {&P.tune.big_fuse, {0, 1}},
        {&P.tune.vec2_max_cls, {0, 128, 160}},
        {&P.tune.warp_items, {152, 2 * 152, 4 * 152, 8 * 152, 16 * 152, 1 << 30}},
        {&P.tune.vec_max_cls, {0, 64, 96}},
        {&P.tune.solve_threads_big, {256, 512}},
        {&P.tune.use_tc, {0, 1, 2}},
        {&P.tune.big_panel, {32, 64, 128, 256}},
        {&P.tune.split_rows, {1024, 2048, 4096, 1 << 30}},
        {&P.tune.warp_front_max, {0, 32, 48, 64}},
        {&P.tune.cluster_rows, {256, 512, 1024, 1 << 30}},
    };
    double best = 0;
    e = measure(&best);
    for (Knob& k : knobs) {
        if (e) break;
        const int32_t keep = *k.field;
        int32_t arg = keep;
        for (int32_t c : k.cand) {
            if (c == keep) continue;
            *k.field = c;
            double ms = 0;
            e = measure(&ms);
            if (e) break;
            if (ms < best * 0.98) {
                best = ms;
                arg = c;
            }
        }
        *k.field = arg;
    }
    P.prof = prof;
    P.eager_only = false;
    P.tune.tuned = e ? 0 : 1;
    graph_release(P);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms) *best_ms = best;
    return e;
}

int launch_backward(Plan& P, const double* x, const double* xbar, double* vals_bar, double* shift_bar,
                    double* b_bar, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    double* mu = wsp<double>(P, P.ws.mu);
    int e;
    if (solve_by_graph(P))
        e = solve_graph_run(P, xbar, mu, s);
    else
        e = P.tsize == 8 ? run_solve<double>(P, xbar, mu, s) : run_solve<float>(P, xbar, mu, s);
    if (e) return e;
    const int B = P.B;
    const int64_t n = P.n, S = (int64_t)B * P.n_pats;
    const int64_t nrows = (int64_t)P.g_rows_all.size(), nel = (int64_t)P.e_elems_all.size();
    if (nrows > 0) {
        Prof pr(P, s, SSCO_K_GRAD);
        k_grad_atwa<<<dim3(cdiv(nrows, 256), B), 256, 0, s>>>(P.dt, nrows, mu, x, n, vals_bar, P.m);
        pr.done(4.0 * P.g_colind.size() * B, (P.g_colind.size() * 28.0 + nrows * 8.0) * B);
    }
    if (nel > 0) {
        Prof pr(P, s, SSCO_K_GRAD);
        k_grad_elem<<<dim3(cdiv(nel, 128), B), 128, 0, s>>>(P.dt, nel, mu, x, n, vals_bar, P.m);
        pr.done(4.0 * P.e_K0.size() * B, (P.e_K0.size() * 8.0 + P.e_dofs.size() * 20.0) * B);
    }
    if (shift_bar) {
        Prof pr(P, s, SSCO_K_GRAD);
        k_shift_bar<<<(unsigned)S, 256, 0, s>>>(P.dt, P.n_pats, n, mu, x, shift_bar);
        pr.done(2.0 * n * B, 21.0 * n * B);
    }
    e = (int)cudaMemcpyAsync(b_bar, mu, (size_t)B * n * 8, cudaMemcpyDeviceToDevice, s);
    if (e) return e;
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free FP64 solve.  Its scratch (permuted right-hand side, solve
// vector, passing vectors) lives in one file-scope device array instead of
// the caller's workspace; only the factor is read from the bound workspace.
// The array is shared by every call on a device and keeps the last call's
// contents; every scratch word is written before it is read, so nothing
// needs clearing.  Calls that overlap on the GPU race on it.
// ---------------------------------------------------------------------------
constexpr size_t kStaticSolveScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_static_solve_scratch[kStaticSolveScratchBytes];
static void* g_static_scratch_addr[256] = {};  // per device: device address of the array

size_t static_solve_scratch_bytes() { return kStaticSolveScratchBytes; }

size_t static_solve_scratch_need(const Plan& P) {
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t B = (size_t)P.B, n = (size_t)P.n;
    return up(B * n * 8) + up(B * n * 8) + up(std::max<size_t>(B * (size_t)P.pvec_total * 8, 16));
}

// First call on a device (with that device current) looks up the array's
// device address; later calls reuse it.
int static_solve_scratch_addr(void** out) {
    int dev = 0;
    int e = (int)cudaGetDevice(&dev);
    if (e) return e;
    if (dev < 0 || dev >= 256) return (int)cudaErrorInvalidDevice;
    if (!g_static_scratch_addr[dev]) {
        void* p = nullptr;
        e = (int)cudaGetSymbolAddress(&p, g_static_solve_scratch);
        if (e) return e;
        g_static_scratch_addr[dev] = p;
    }
    *out = g_static_scratch_addr[dev];
    return 0;
}

int launch_solve_static(Plan& P, const double* b, double* x, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    void* base = nullptr;
    int e = static_solve_scratch_addr(&base);
    if (e) return e;
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    const int B = P.B;
    const int64_t n = P.n;
    uint8_t* sc = (uint8_t*)base;
    double* bp = (double*)sc;
    double* vec = (double*)(sc + up((size_t)B * n * 8));
    double* pvec = (double*)(sc + 2 * up((size_t)B * n * 8));
    const double* panel = wsp<double>(P, P.ws.panel);
    const dim3 gv(cdiv(n, 256), B);
    k_permute_in<<<gv, 256, 0, s>>>(b, P.dt.perm, n, bp);
    k_to_T<double><<<cdiv((int64_t)B * n, 256), 256, 0, s>>>(bp, vec, (int64_t)B * n);
    P.launches += 2;
    const unsigned tiny_grid = cdiv((int64_t)P.n_tiny * B, kTinyWarps);
    if (P.n_tiny > 0) {
        k_tiny_fwd<double><<<tiny_grid, 32 * kTinyWarps, tiny_solve_bytes<double>(false, P.tiny_prog_max), s>>>(
            P.dt, P.n_tiny, B, P.tiny_prog_max, panel, P.panel_total, vec, n, pvec, P.pvec_total, nullptr, P.n_pats,
            0);
        P.launches++;
    }
    for (const LaunchList& ll : P.solve_launches) {
        k_fwd<double><<<dim3(ll.count, B), 256, (size_t)ll.rmax * 8, s>>>(
            P.dt, P.dt.flow_rest + ll.list_off, panel, P.panel_total, vec, n, pvec, P.pvec_total, nullptr,
            P.n_pats);
        P.launches++;
    }
    for (auto it = P.solve_launches.rbegin(); it != P.solve_launches.rend(); ++it) {
        k_bwd<double><<<dim3(it->count, B), 256, (size_t)it->rmax * 8, s>>>(
            P.dt, P.dt.flow_rest + it->list_off, panel, P.panel_total, vec, n, nullptr, P.n_pats);
        P.launches++;
    }
    if (P.n_tiny > 0) {
        k_tiny_bwd<double><<<tiny_grid, 32 * kTinyWarps, tiny_solve_bytes<double>(false, P.tiny_prog_max), s>>>(
            P.dt, P.n_tiny, B, P.tiny_prog_max, panel, P.panel_total, vec, n, nullptr, P.n_pats, 0);
        P.launches++;
    }
    k_permute_out<<<gv, 256, 0, s>>>(vec, P.dt.perm, n, x);
    P.launches++;
    return (int)cudaGetLastError();
}

int profile_enable(Plan& P, int32_t max_launches) {
    for (void* e : P.ev_pool) cudaEventDestroy((cudaEvent_t)e);
    P.ev_pool.clear();
    P.prof_recs.clear();
    P.ev_used = 0;
    P.prof = max_launches > 0;
    for (int32_t i = 0; i < 2 * max_launches; ++i) {
        cudaEvent_t e;
        int r = (int)cudaEventCreate(&e);
        if (r) return r;
        P.ev_pool.push_back((void*)e);
    }
    return 0;
}

int profile_trace(Plan& P, int32_t* kinds, float* ms, double* flops, double* bytes, int64_t cap, int64_t* n) {
    int e = (int)cudaDeviceSynchronize();
    if (e) return e;
    *n = (int64_t)P.prof_recs.size();
    for (int64_t i = 0; i < *n && i < cap; ++i) {
        const ProfRec& r = P.prof_recs[i];
        float t = 0;
        e = (int)cudaEventElapsedTime(&t, (cudaEvent_t)P.ev_pool[r.ev], (cudaEvent_t)P.ev_pool[r.ev + 1]);
        if (e) return e;
        if (kinds) kinds[i] = r.kind;
        if (ms) ms[i] = t;
        if (flops) flops[i] = r.flops;
        if (bytes) bytes[i] = r.bytes;
    }
    return 0;
}

int profile_read(Plan& P, ssco_kernel_stat* out) {
    int e = (int)cudaDeviceSynchronize();
    if (e) return e;
    for (int k = 0; k < SSCO_K_COUNT; ++k) {
        out[k].kind = k;
        out[k].reserved = 0;
        out[k].launches = 0;
        out[k].ms = out[k].flops = out[k].bytes = 0;
    }
    for (const ProfRec& r : P.prof_recs) {
        float ms = 0;
        e = (int)cudaEventElapsedTime(&ms, (cudaEvent_t)P.ev_pool[r.ev], (cudaEvent_t)P.ev_pool[r.ev + 1]);
        if (e) return e;
        ssco_kernel_stat& o = out[r.kind];
        o.launches++;
        o.ms += ms;
        o.flops += r.flops;
        o.bytes += r.bytes;
    }
    P.prof_recs.clear();
    P.ev_used = 0;
    return 0;
}

}  // namespace ssco
