// ssco_internal.h -- plan layout shared by the host symbolic phase
// (ssco_symbolic.cpp), the C ABI (ssco_api.cpp) and the kernels
// (ssco_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ssco.h"

namespace ssco {

// Tiny-subtree programs (see build_tiny_programs in ssco_symbolic.cpp).
constexpr int32_t kTinyHdrWords = 8;
constexpr int32_t kTinyRecWords = 16;
constexpr int32_t kTinyProgWords = 1024;  // per subtree, shared memory per warp
constexpr int32_t kTinyMaxK = 256;        // K entries gathered per subtree
// Tensor-core operand blocks of a big FP32 front: per 128-row tile, up to
// kTcMaxPanel / 16 blocks of 128 x 16 TF32 high + low parts (4096 floats).
constexpr int32_t kTcMaxPanel = 256;
constexpr int64_t kTcTileFloats = (int64_t)(kTcMaxPanel / 16) * 4096;

// One front of the numeric partition (a fundamental or amalgamated
// supernode).  Its factor columns [f, f+w) are stored as a dense r x w
// column-major panel whose rows are rows[rows_off .. rows_off+r) (the first
// w of them are the front's own columns).  Its update (Schur complement)
// matrix is (r-w) x (r-w) column-major, lower triangle meaningful.
struct FrontDesc {
    int32_t f, w, r, parent;      // first column, width, rows, parent front or -1
    int32_t nchild, child_off;    // children: child_ids[child_off .. +nchild)
    int32_t klist_n, sys;         // number of K entries owned; pattern index
    int64_t klist_off;            // K entries: klist[2*(klist_off+t)] = {kslot, pos}
    int64_t rows_off;             // into rows[]
    int64_t panel_off;            // per-instance offset of the r x w panel
    int64_t upd_off;              // per-instance offset of the (r-w)^2 update
    int64_t pvec_off;             // per-instance offset of the (r-w) passing vector
    int64_t relmap_off;           // r-w positions of this front's update rows in
                                  // the parent's rows (-1 for a root)
    int64_t inv_off;              // big fronts: [nchild][r] inverse maps (-1 if none)
    int64_t tc_off;               // big FP32 fronts: per-instance offset (floats) of the
                                  // tensor-core operand blocks within its level (-1 if none)
};

// Assembly leaf table of one group (Sec. 4.3/4.4): members share a term
// count, a diagonal flag and (if uniform) the constant of every term.
// K[slot_base + i] = cadd + sum_t c_t * vals[idx[t*nmem + i]] (+ shift if diag)
struct AsmGroup {
    int32_t nmem, nterms, uniform, diag;
    int32_t sys, pad;
    double coef;        // uniform constant (uniform == 1)
    double cadd;        // constant added (1 for identity rows, else 0)
    int64_t idx_off;    // into asm_idx (term-major, member-innermost)
    int64_t coef_off;   // into asm_coef (varying groups only)
    int64_t slot_base;  // first K storage slot of the group
};

struct AsmChunk {
    int32_t group, start;
};

// A batch of fronts handled by one launch.
struct LaunchList {
    int32_t level;
    int32_t cls;        // small-front size class (max rows), or -1 for big fronts
    int64_t list_off;   // into front_lists
    int32_t count;
    int32_t rmax, wmax;
    int64_t max_lower_tiles;  // big: max tiles of 64x64 over the front's lower triangle
    int64_t max_syrk_tiles;   // big: max 64x64 lower tiles of the update block
    int32_t max_klist;        // big: max K entries per front
};

// One persistent launch of the small-front factorization dataflow: the
// fronts flow_fact[off .. off+count), level ascending, each factored for V
// value sets per item by a CTA of nw warps.  A front's group holds no front
// larger than the group's rmax, and every child of a front sits in the same
// or an earlier group (an earlier group has finished before the launch).
struct FlowGroup {
    int32_t off, count;
    int32_t rmax, V, nw;
    int32_t pad;
};

// Typed device pointers into the bound table buffer.
struct DevTables {
    const FrontDesc* fronts;
    const int32_t* rows;
    const int32_t* child_ids;
    const int32_t* relmap;
    const int32_t* invmap;
    const int32_t* klist;
    const int32_t* front_lists;
    const AsmGroup* groups;
    const AsmChunk* chunks;
    const int32_t* asm_idx;
    const double* asm_coef;
    const int64_t* sp_rowptr;   // symmetric CSR of K~ over permuted rows
    const int32_t* sp_col;
    const int32_t* sp_slot;
    const int32_t* perm;        // concatenated perm (new -> old)
    const int32_t* row_sys;     // pattern index of each permuted row
    const int64_t* sys_n_off;   // [n_pats+1] row ranges of patterns
    const int64_t* g_rowptr;    // ATWA rows (concatenated), for the adjoint
    const int32_t* g_colind;    // global (concatenated, original order) columns
    const double* g_aval;
    const int32_t* g_row_sys;   // pattern of each ATWA row (values index space)
    const int32_t* e_dofs;      // ELEM dofs (global, original order, -1 fixed)
    const double* e_K0;
    const int32_t* e_sys;       // pattern of each element
    const int64_t* e_off;       // per element: offset into e_dofs (dim varies per pattern)
    const int64_t* e_k0off;     // per element: offset into e_K0
    const int32_t* e_dim;       // per element: local DOF count
    const uint8_t* shifted;     // per permuted row: receives the shift (1) or not
    const int32_t* g_rows_all;  // value indices that are ATWA rows
    const int32_t* e_elems_all; // value indices that are elements
    const int32_t* tiny_list;   // fronts of every tiny subtree, children first
    const int32_t* tiny_off;    // [n_tiny+1] offsets into tiny_list
    const int32_t* tiny_prog;   // per-subtree programs
    const int64_t* tiny_prog_off;
    const int32_t* flow_fact;   // factor dataflow fronts, group-major, level ascending
    const int32_t* flow_fslot;  // per front: position in flow_fact, or -1
    const int32_t* flow_solve;  // solve dataflow fronts, level ascending
    const int32_t* flow_sslot;  // per front: position in flow_solve, or -1
    const int32_t* flow_rest;   // front lists of the per-level launches around the dataflow
};

// Byte offsets of every region of the caller's workspace.
struct WsLayout {
    size_t K, panel, upd, pvec, vecT, bp, xp, rr, mu, xbar_p;
    size_t bad_col, sstatus, iters, active, any_active, it_ctr, dev_err;
    size_t resid, bnorm, r1, r2, sigma, sbar;
    size_t st_vals, st_shift, st_b, st_x;
    size_t tcpack;
    size_t sys_psum, sys_pmax;     // per-system norms: chunk partial sums and maxima [S][sys_maxc]
    int32_t sys_maxc;              // ... chunks of the longest system
    size_t diag;                   // big fronts: one factored 32x32 diagonal block per (front, value set) of a level
    size_t diag_slots;             // ... number of such slots
    size_t flow_fact, flow_solve;  // dataflow tickets (32 words) + done flags [slot][B]
    size_t gm_V, gm_Z, gm_H, gm_g, gm_cs, gm_sn, gm_hp, gm_y, gm_beta, gm_hn, gm_act, gm_k;  // GMRES-IR
    size_t total;
};

// One profiled launch: two CUDA events from the plan's pool and the
// algorithmic work of the launch.
struct ProfRec {
    int32_t kind;
    int32_t ev;
    double flops, bytes;
};

// Launch-shape knobs chosen by ssco_autotune (defaults are the untuned ones).
struct Tunables {
    int32_t warp_items = 8 * 152;  // a solve level goes warp-per-item at >= this many items
    int32_t vec_max_cls = 96;      // largest size class factored V value sets per CTA
    int32_t vec2_max_cls = 0;      // FP32: larger classes up to this size factored two value sets per CTA
    int32_t solve_threads_big = 512;  // CTA size of solve levels with fronts > 512 rows
    int32_t use_tc = 1;            // FP32 big-front updates on tcgen05: 0 off, 1 per-tile CTAs,
                                   // 2 persistent CTAs for the wide trailing updates
    int32_t tc_min_rows = 128;     // ... when the trailing extent reaches this many rows
    int32_t big_panel = 256;       // big fronts: columns per trailing-update block
    int32_t split_rows = 2048;     // fronts with at least this many rows take the split solves
    int32_t cluster_rows = 512;    // ... below that, from this many rows: one CTA cluster per front
    int32_t warp_front_max = 0;    // small-front classes up to this size: one warp per front (levels
                                   // of >= warp_items fronts x value sets; autotuner option)
    int32_t front_core = 0;        // per-level small fronts: 0 column-step kernels (k_front_small/vec),
                                   // 1 the dataflow kernel's panel core, one CTA per item
    int32_t flow = 3;              // persistent dataflow launches: bit 0 the solve sweeps, bit 1 the
                                   // small-front factorization (0 = one launch per level and class)
    uint32_t flow_polls = 1u << 22;  // bound of every dataflow wait (polls of ~256 ns)
    int32_t flow_stall = -1;       // test hook: this item of the first dataflow launch waits on a
                                   // flag that nothing sets (the bounded-wait path); -1 = off
    int32_t big_fuse = 0;          // big fronts: 1 factors each 32-column step's diagonal block inside
                                   // the trsm launch (no separate potrf launch but the last)
    int32_t tuned = 0;
};

struct PatMeta {
    int32_t kind, n, m, dim;
    int64_t n_off, m_off;
};

struct Plan {
    int32_t launch_err = 0;  // first failed extended launch (cudaLaunchKernelEx) since the last check
    // options
    int32_t prec = SSCO_FP64;
    int32_t B = 1;
    double tol = 1e-10;
    int32_t maxit = 30;
    int32_t refine_mode = 0;  // 0 plain, 1 GMRES-IR, 2 plain then GMRES-IR where it stagnated
    int32_t gmres_m = 16;     // Krylov vectors per GMRES-IR correction
    int32_t small_max = 0;
    int32_t amalg = 1;
    int32_t tiny_max = 32;
    size_t tsize = 8;  // bytes of the factor type
    Tunables tune;

    int32_t n_pats = 0;
    std::vector<PatMeta> pats;
    int64_t n = 0, m = 0;

    // K~ (concatenated, lower CSC)
    std::vector<int64_t> Kcolptr;
    std::vector<int32_t> Krowind;
    std::vector<int32_t> kslot_of_q;  // CSC position -> storage slot
    int64_t nnzK = 0;

    // exact symbolic structures
    std::vector<int32_t> perm, parent, colcount, col_level;
    std::vector<int32_t> snode_first, sn_parent, sn_level;
    std::vector<int64_t> sn_rows_off;  // fundamental supernode rows (for exports)
    std::vector<int32_t> sn_rows;
    int64_t nnzL = 0;
    int32_t max_col_level = 0;
    double flops_exact = 0, flops_numeric = 0;

    // numeric partition
    std::vector<FrontDesc> fronts;
    std::vector<int32_t> front_first, front_level;
    std::vector<int32_t> rows, child_ids, relmap, invmap, klist, front_lists;
    std::vector<LaunchList> fact_launches;   // per level: small classes + big
    std::vector<LaunchList> solve_launches;  // per level: all fronts
    std::vector<int32_t> tiny_list, tiny_off;  // warp-per-subtree fronts
    int32_t n_tiny = 0;
    std::vector<int32_t> tiny_prog;
    std::vector<int64_t> tiny_prog_off;
    int32_t tiny_prog_max = 0, tiny_k_max = 0;
    int32_t n_levels = 0;
    int64_t panel_total = 0, upd_total = 0, pvec_total = 0;
    int64_t tc_pack_total = 0;  // floats per instance of tensor-core operand blocks (0 = none)
    int32_t max_rows = 0;
    // dataflow schedules, derived from the partition by build_flow (not
    // stored in plan files)
    std::vector<int32_t> flow_fact, flow_fslot, flow_solve, flow_sslot, flow_rest;
    std::vector<FlowGroup> fact_groups;
    int32_t flow_solve_rmax = 0;
    std::vector<LaunchList> fact_rest, solve_rest;  // per level, around the dataflow (into flow_rest)

    // assembly
    std::vector<AsmGroup> groups;
    std::vector<AsmChunk> chunks;
    std::vector<int32_t> asm_idx;
    std::vector<double> asm_coef;

    // SpMV / vectors
    std::vector<int64_t> sp_rowptr;
    std::vector<int32_t> sp_col, sp_slot, row_sys;
    std::vector<int64_t> sys_n_off;
    std::vector<uint8_t> shifted;

    // adjoint tables
    std::vector<int64_t> g_rowptr;
    std::vector<int32_t> g_colind, g_row_sys, g_rows_all;
    std::vector<double> g_aval;
    std::vector<int32_t> e_dofs, e_sys, e_dim, e_elems_all;
    std::vector<int64_t> e_off, e_k0off;
    std::vector<double> e_K0;
    // ELEM_BLOCKS elements: DOFs (global, original order, -1 fixed), offsets
    // into them, local DOF counts, and the value index of entry 0
    std::vector<int32_t> blk_dofs, blk_dim, blk_vbase;
    std::vector<int64_t> blk_off;

    // device binding
    std::vector<uint8_t> blob;   // host image of the device tables
    struct {
        size_t fronts, rows, child_ids, relmap, invmap, klist, front_lists, groups, chunks,
            asm_idx, asm_coef, sp_rowptr, sp_col, sp_slot, perm, row_sys, sys_n_off, g_rowptr,
            g_colind, g_aval, g_row_sys, e_dofs, e_K0, e_sys, e_off, e_k0off, e_dim, shifted,
            g_rows_all, e_elems_all, tiny_list, tiny_off, tiny_prog, tiny_prog_off, blk_dofs, blk_off,
            blk_dim, blk_vbase, flow_fact, flow_fslot, flow_solve, flow_sslot, flow_rest;
    } toff{};
    WsLayout ws{};
    uint8_t* d_tab = nullptr;
    uint8_t* d_ws = nullptr;
    DevTables dt{};
    bool bound = false;
    bool factored = false;
    int32_t* h_flag = nullptr;  // pinned host word for the refinement loop

    // captured assemble + refactor + solve graph (ssco_graph_run)
    void* g_stream = nullptr;
    void* g_body_stream = nullptr;
    void* g_graph = nullptr;
    void* g_exec = nullptr;
    const void* g_key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int32_t g_vdt = -1;
    int64_t g_launches = 0;
    uint64_t g_gen = 0;  // incremented whenever this plan's captured graphs are released

    // solve-only graphs of the FP32 refinement (ssco_solve, ssco_backward):
    // two cached (b, x) pointer pairs, least recently used replaced
    void* s_graph[2] = {nullptr, nullptr};
    void* s_exec[2] = {nullptr, nullptr};
    const void* s_key[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int64_t s_launches[2] = {0, 0};
    int32_t s_next = 0;
    bool eager_only = false;  // set while ssco_autotune times its candidates
    bool no_graphs = false;   // ssco_set_flow bit 4: FP32 solves launch eagerly (for profilers)

    // one graph over several plans (ssco_graph_run_many; held by the first plan)
    void* m_graph = nullptr;
    void* m_exec = nullptr;
    std::vector<const void*> m_key;  // plans, their generations, pointers and dtypes
    int64_t m_launches = 0;

    // auxiliary streams for the independent launch lists of a level, with a
    // fork event and one join event per stream (created on first use)
    void* aux_stream[4] = {nullptr, nullptr, nullptr, nullptr};
    void* aux_join[4] = {nullptr, nullptr, nullptr, nullptr};
    void* aux_fork = nullptr;

    std::string last_error;
    int64_t launches = 0;

    // per-kernel CUDA-event profiling (ssco_profile_enable / _read)
    bool prof = false;
    std::vector<void*> ev_pool;  // cudaEvent_t
    size_t ev_used = 0;
    std::vector<ProfRec> prof_recs;
};

// symbolic phase (ssco_symbolic.cpp)
ssco_status analyze_impl(const ssco_pattern* const* pats, int32_t n_pats, const ssco_op* op,
                         Plan& P);
void build_flow(Plan& P);
void build_blob(Plan& P);
void compute_ws_layout(Plan& P);
void export_L_pattern(const Plan& P, std::vector<int64_t>* colptr, std::vector<int32_t>* rowind);

// kernels (ssco_kernels.cu); each returns cudaError_t as int
int launch_numeric(Plan& P, const void* vals, int32_t vals_dtype, const double* shift, void* stream);
int launch_solve(Plan& P, const double* b, double* x, void* stream, bool* synced_ok);
int launch_backward(Plan& P, const double* x, const double* xbar, double* vals_bar,
                    double* shift_bar, double* b_bar, void* stream);
// vals_bar entries of ELEM_BLOCKS elements from mu and x (no-op without them)
int launch_grad_blocks(Plan& P, const double* mu, const double* x, double* vals_bar, void* stream);
int launch_reset_status(Plan& P, void* stream);
int launch_graph_run(Plan& P, const void* vals, int32_t vals_dtype, const double* shift, const double* b, double* x,
                     void* stream);
int launch_graph_run_many(Plan* const* plans, int32_t n, const void* const* vals, const int32_t* vals_dtype,
                          const double* const* shift, const double* const* b, double* const* x, void* stream);
void graph_release(Plan& P);
int autotune_many(Plan* const* plans, int32_t n, const void* const* vals, const int32_t* vals_dtype,
                  const double* const* shift, const double* const* b, double* const* x, int32_t reps, void* stream,
                  double* best_ms);
int autotune(Plan& P, const void* vals, int32_t vals_dtype, const double* shift, const double* b, double* x,
             int32_t reps, void* stream, double* best_ms);
void graph_destroy_streams(Plan& P);
int kernels_set_attributes(Plan& P);
const char* kernel_kind_name(int kind);
int profile_enable(Plan& P, int32_t max_launches);
size_t static_solve_scratch_bytes();
size_t static_solve_scratch_need(const Plan& P);
int launch_solve_static(Plan& P, const double* b, double* x, void* stream);
int profile_read(Plan& P, ssco_kernel_stat* out);
int profile_trace(Plan& P, int32_t* kinds, float* ms, double* flops, double* bytes, int64_t cap, int64_t* n);

}  // namespace ssco
