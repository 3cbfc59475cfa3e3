// ssco_api.cpp -- the extern "C" boundary declared in include/ssco.h.
// Host-side plan lifecycle, binding of caller memory, exports, plan files.
// The numeric work itself is launched from ssco_kernels.cu.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>

#include "ssco_internal.h"

using namespace ssco;

struct ssco_plan_s {
    Plan P;
};

namespace {

thread_local std::string g_err;

ssco_status fail(ssco_plan h, ssco_status s, const std::string& msg) {
    if (h) h->P.last_error = msg;
    g_err = msg;
    return s;
}

ssco_status cuda_fail(ssco_plan h, int e, const char* where) {
    return fail(h, SSCO_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString((cudaError_t)e));
}

template <class T>
T* tab_ptr(Plan& P, size_t off) {
    return reinterpret_cast<T*>(P.d_tab + off);
}

void set_dev_tables(Plan& P) {
    DevTables& d = P.dt;
    d.fronts = tab_ptr<FrontDesc>(P, P.toff.fronts);
    d.rows = tab_ptr<int32_t>(P, P.toff.rows);
    d.child_ids = tab_ptr<int32_t>(P, P.toff.child_ids);
    d.relmap = tab_ptr<int32_t>(P, P.toff.relmap);
    d.invmap = tab_ptr<int32_t>(P, P.toff.invmap);
    d.klist = tab_ptr<int32_t>(P, P.toff.klist);
    d.front_lists = tab_ptr<int32_t>(P, P.toff.front_lists);
    d.groups = tab_ptr<AsmGroup>(P, P.toff.groups);
    d.chunks = tab_ptr<AsmChunk>(P, P.toff.chunks);
    d.asm_idx = tab_ptr<int32_t>(P, P.toff.asm_idx);
    d.asm_coef = tab_ptr<double>(P, P.toff.asm_coef);
    d.sp_rowptr = tab_ptr<int64_t>(P, P.toff.sp_rowptr);
    d.sp_col = tab_ptr<int32_t>(P, P.toff.sp_col);
    d.sp_slot = tab_ptr<int32_t>(P, P.toff.sp_slot);
    d.perm = tab_ptr<int32_t>(P, P.toff.perm);
    d.row_sys = tab_ptr<int32_t>(P, P.toff.row_sys);
    d.sys_n_off = tab_ptr<int64_t>(P, P.toff.sys_n_off);
    d.g_rowptr = tab_ptr<int64_t>(P, P.toff.g_rowptr);
    d.g_colind = tab_ptr<int32_t>(P, P.toff.g_colind);
    d.g_aval = tab_ptr<double>(P, P.toff.g_aval);
    d.g_row_sys = tab_ptr<int32_t>(P, P.toff.g_row_sys);
    d.e_dofs = tab_ptr<int32_t>(P, P.toff.e_dofs);
    d.e_K0 = tab_ptr<double>(P, P.toff.e_K0);
    d.e_sys = tab_ptr<int32_t>(P, P.toff.e_sys);
    d.e_off = tab_ptr<int64_t>(P, P.toff.e_off);
    d.e_k0off = tab_ptr<int64_t>(P, P.toff.e_k0off);
    d.e_dim = tab_ptr<int32_t>(P, P.toff.e_dim);
    d.shifted = tab_ptr<uint8_t>(P, P.toff.shifted);
    d.g_rows_all = tab_ptr<int32_t>(P, P.toff.g_rows_all);
    d.e_elems_all = tab_ptr<int32_t>(P, P.toff.e_elems_all);
    d.tiny_list = tab_ptr<int32_t>(P, P.toff.tiny_list);
    d.tiny_off = tab_ptr<int32_t>(P, P.toff.tiny_off);
    d.tiny_prog = tab_ptr<int32_t>(P, P.toff.tiny_prog);
    d.tiny_prog_off = tab_ptr<int64_t>(P, P.toff.tiny_prog_off);
    d.flow_fact = tab_ptr<int32_t>(P, P.toff.flow_fact);
    d.flow_fslot = tab_ptr<int32_t>(P, P.toff.flow_fslot);
    d.flow_solve = tab_ptr<int32_t>(P, P.toff.flow_solve);
    d.flow_sslot = tab_ptr<int32_t>(P, P.toff.flow_sslot);
    d.flow_rest = tab_ptr<int32_t>(P, P.toff.flow_rest);
}

// ----- plan file (de)serialization -----------------------------------------
constexpr uint64_t kMagic = 0x314F4353534F4353ull;  // "SCOSSCO1"
constexpr uint32_t kVersion = 13;

// 64-bit FNV-1a (Fowler, Noll, Vo) over the payload bytes: the file ends
// with the digest, so a plan whose tables were damaged after saving is
// refused at load instead of indexing device memory with bad maps.
struct Fnv1a {
    uint64_t h = 0xcbf29ce484222325ull;
    void add(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 0x100000001b3ull;
    }
};
struct Writer {
    std::ofstream f;
    Fnv1a sum;
    void raw(const void* p, size_t n) {
        f.write(static_cast<const char*>(p), (std::streamsize)n);
        sum.add(p, n);
    }
    template <class T>
    bool pod(const T& v) {
        raw(&v, sizeof(T));
        return (bool)f;
    }
    template <class T>
    bool vec(const std::vector<T>& v) {
        uint64_t n = v.size();
        pod(n);
        if (n) raw(v.data(), n * sizeof(T));
        return (bool)f;
    }
};
struct Reader {
    std::ifstream f;
    Fnv1a sum;
    bool raw(void* p, size_t n) {
        f.read(static_cast<char*>(p), (std::streamsize)n);
        if (!f) return false;
        sum.add(p, n);
        return true;
    }
    template <class T>
    bool pod(T& v) {
        return raw(&v, sizeof(T));
    }
    template <class T>
    bool vec(std::vector<T>& v) {
        uint64_t n = 0;
        if (!pod(n)) return false;
        // a length that the rest of the file cannot hold is damage, not a size
        const std::streamoff here = f.tellg();
        if (here < 0 || n > (uint64_t)(size - here) / sizeof(T)) return false;
        v.resize(n);
        return n == 0 || raw(v.data(), n * sizeof(T));
    }
    std::streamoff size = 0;
};

template <class IO>
bool serialize(IO& io, Plan& P) {
    bool ok = true;
    auto S = [&](auto& x) { ok = ok && io.pod(x); };
    auto V = [&](auto& x) { ok = ok && io.vec(x); };
    S(P.prec); S(P.B); S(P.tol); S(P.maxit); S(P.refine_mode); S(P.gmres_m); S(P.small_max); S(P.amalg);
    S(P.tiny_max); S(P.tsize);
    S(P.n_pats); V(P.pats); S(P.n); S(P.m);
    V(P.Kcolptr); V(P.Krowind); V(P.kslot_of_q); S(P.nnzK);
    V(P.perm); V(P.parent); V(P.colcount); V(P.col_level);
    V(P.snode_first); V(P.sn_parent); V(P.sn_level); V(P.sn_rows_off); V(P.sn_rows);
    S(P.nnzL); S(P.max_col_level); S(P.flops_exact); S(P.flops_numeric);
    V(P.fronts); V(P.front_first); V(P.front_level); V(P.rows); V(P.child_ids); V(P.relmap);
    V(P.invmap); V(P.klist); V(P.front_lists); V(P.fact_launches); V(P.solve_launches);
    S(P.n_levels); S(P.panel_total); S(P.upd_total); S(P.pvec_total); S(P.max_rows);
    V(P.tiny_list); V(P.tiny_off); S(P.n_tiny);
    V(P.tiny_prog); V(P.tiny_prog_off); S(P.tiny_prog_max); S(P.tiny_k_max);
    S(P.tune);
    S(P.tc_pack_total);
    V(P.groups); V(P.chunks); V(P.asm_idx); V(P.asm_coef);
    V(P.sp_rowptr); V(P.sp_col); V(P.sp_slot); V(P.row_sys); V(P.sys_n_off); V(P.shifted);
    V(P.g_rowptr); V(P.g_colind); V(P.g_row_sys); V(P.g_rows_all); V(P.g_aval);
    V(P.e_dofs); V(P.e_sys); V(P.e_dim); V(P.e_elems_all); V(P.e_off); V(P.e_k0off); V(P.e_K0);
    V(P.blk_dofs); V(P.blk_off); V(P.blk_dim); V(P.blk_vbase);
    return ok;
}

// The launch lists size shared memory, register-budget instantiations and
// big-front tiles from their rmax / wmax / tile fields: on load these must
// equal the maxima over the listed fronts, which must exist, lie inside the
// front list and fit their size class.  A solve list is ordered largest
// front first (the sweeps peel off its split and cluster fronts and size the
// rest from the next front).
bool launch_lists_consistent(const Plan& P) {
    const int64_t nf = (int64_t)P.fronts.size(), nl = (int64_t)P.front_lists.size();
    auto check = [&](const std::vector<LaunchList>& lists) {
        for (const LaunchList& ll : lists) {
            if (ll.list_off < 0 || ll.count < 0 || ll.list_off > nl || ll.count > nl - ll.list_off) return false;
            int32_t rmax = 0, wmax = 0, klist = 0;
            int64_t lower = 0, syrk = 0;
            for (int32_t i = 0; i < ll.count; ++i) {
                const int32_t F = P.front_lists[ll.list_off + i];
                if (F < 0 || F >= nf) return false;
                const FrontDesc& d = P.fronts[F];
                if (d.w < 1 || d.r < d.w || (ll.cls > 0 && d.r > ll.cls)) return false;
                if (ll.cls == 0 && i > 0 && d.r > P.fronts[P.front_lists[ll.list_off + i - 1]].r) return false;
                rmax = std::max(rmax, d.r);
                wmax = std::max(wmax, d.w);
                const int64_t t = (d.r + 63) / 64, u = (d.r - d.w + 63) / 64;
                lower = std::max(lower, t * (t + 1) / 2);
                syrk = std::max(syrk, u * (u + 1) / 2);
                klist = std::max(klist, d.klist_n);
            }
            if (rmax != ll.rmax || wmax != ll.wmax) return false;
            if (ll.cls == -1 && (lower != ll.max_lower_tiles || syrk != ll.max_syrk_tiles || klist != ll.max_klist))
                return false;
        }
        return true;
    };
    return check(P.fact_launches) && check(P.solve_launches);
}

}  // namespace

extern "C" {

const char* ssco_status_string(ssco_status s) {
    switch (s) {
        case SSCO_OK: return "ok";
        case SSCO_ERR_INVALID_ARG: return "invalid argument";
        case SSCO_ERR_PATTERN: return "invalid pattern";
        case SSCO_ERR_NOT_SPD: return "matrix not positive definite";
        case SSCO_ERR_NONFINITE: return "non-finite value";
        case SSCO_ERR_NO_CONVERGE: return "refinement did not converge";
        case SSCO_ERR_TIMEOUT: return "device wait timed out";
        case SSCO_ERR_CUDA: return "CUDA error";
        case SSCO_ERR_OOM: return "buffer too small";
        case SSCO_ERR_UNSUPPORTED: return "unsupported";
        case SSCO_ERR_STATE: return "invalid call order";
    }
    return "unknown status";
}

const char* ssco_last_error(ssco_plan plan) { return plan ? plan->P.last_error.c_str() : g_err.c_str(); }

ssco_status ssco_analyze(const ssco_pattern* const* pats, int32_t n_pats, const ssco_op* op, ssco_plan* out) {
    if (!out) return fail(nullptr, SSCO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    ssco_plan h = new (std::nothrow) ssco_plan_s();
    if (!h) return fail(nullptr, SSCO_ERR_OOM, "host allocation failed");
    ssco_status s;
    try {
        s = analyze_impl(pats, n_pats, op, h->P);
    } catch (const std::bad_alloc&) {
        s = SSCO_ERR_OOM;
        h->P.last_error = "host allocation failed during analysis";
    } catch (const std::exception& ex) {
        s = SSCO_ERR_UNSUPPORTED;
        h->P.last_error = std::string("analysis failed: ") + ex.what();
    }
    if (s != SSCO_OK) {
        g_err = h->P.last_error;
        delete h;
        return s;
    }
    *out = h;
    return SSCO_OK;
}

ssco_status ssco_plan_info(ssco_plan h, ssco_info* o) {
    if (!h || !o) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    const Plan& P = h->P;
    std::memset(o, 0, sizeof(*o));
    o->n = P.n;
    o->n_pats = P.n_pats;
    o->batch = P.B;
    o->n_systems = (int64_t)P.B * P.n_pats;
    o->m = P.m;
    o->nnz_K = P.nnzK;
    o->nnz_L = P.nnzL;
    o->n_snodes = (int64_t)P.snode_first.size() - 1;
    o->n_fronts = (int64_t)P.fronts.size();
    o->n_levels = P.n_levels;
    o->max_col_level = P.max_col_level;
    o->panel_entries = P.panel_total;
    o->update_entries = P.upd_total;
    o->max_front_rows = P.max_rows;
    o->n_assembly_groups = (int64_t)P.groups.size();
    o->assembly_terms = (int64_t)P.asm_idx.size();
    o->tables_bytes = (int64_t)P.blob.size();
    o->workspace_bytes = (int64_t)P.ws.total;
    o->factor_flops = P.flops_numeric;
    o->factor_flops_exact = P.flops_exact;
    o->tune_warp_items = P.tune.warp_items;
    o->tune_vec_max_cls = P.tune.vec_max_cls;
    o->tune_solve_threads_big = P.tune.solve_threads_big;
    o->tuned = P.tune.tuned;
    o->tune_use_tc = P.tune.use_tc;
    o->tune_big_panel = P.tune.big_panel;
    o->tune_split_rows = P.tune.split_rows;
    o->tune_warp_front_max = P.tune.warp_front_max;
    o->tune_cluster_rows = P.tune.cluster_rows;
    o->tune_flow = P.tune.flow | (P.tune.front_core << 2) | (P.tune.big_fuse << 3) | ((int)P.no_graphs << 4);
    o->flow_fact_fronts = (int64_t)P.flow_fact.size();
    o->flow_solve_fronts = (int64_t)P.flow_solve.size();
    o->tune_vec2_max_cls = P.tune.vec2_max_cls;
    return SSCO_OK;
}

ssco_status ssco_plan_export(ssco_plan h, int32_t what, void* buf, size_t bytes) {
    if (!h || !buf) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    Plan& P = h->P;
    auto copy = [&](const void* src, size_t nb) -> ssco_status {
        if (bytes < nb) return fail(h, SSCO_ERR_OOM, "export buffer too small");
        if (nb) std::memcpy(buf, src, nb);
        return SSCO_OK;
    };
    switch (what) {
        case SSCO_EXPORT_PERM: return copy(P.perm.data(), P.perm.size() * 4);
        case SSCO_EXPORT_ETREE: return copy(P.parent.data(), P.parent.size() * 4);
        case SSCO_EXPORT_COLCOUNT: return copy(P.colcount.data(), P.colcount.size() * 4);
        case SSCO_EXPORT_L_COLPTR: {
            std::vector<int64_t> cp;
            export_L_pattern(P, &cp, nullptr);
            return copy(cp.data(), cp.size() * 8);
        }
        case SSCO_EXPORT_L_ROWIND: {
            if (bytes < (size_t)P.nnzL * 4) return fail(h, SSCO_ERR_OOM, "export buffer too small");
            std::vector<int32_t> ri;
            export_L_pattern(P, nullptr, &ri);
            return copy(ri.data(), ri.size() * 4);
        }
        case SSCO_EXPORT_COL_LEVEL: return copy(P.col_level.data(), P.col_level.size() * 4);
        case SSCO_EXPORT_SNODE_FIRST: return copy(P.snode_first.data(), P.snode_first.size() * 4);
        case SSCO_EXPORT_SN_PARENT: return copy(P.sn_parent.data(), P.sn_parent.size() * 4);
        case SSCO_EXPORT_SN_LEVEL: return copy(P.sn_level.data(), P.sn_level.size() * 4);
        case SSCO_EXPORT_K_COLPTR: return copy(P.Kcolptr.data(), P.Kcolptr.size() * 8);
        case SSCO_EXPORT_K_ROWIND: return copy(P.Krowind.data(), P.Krowind.size() * 4);
        case SSCO_EXPORT_GROUPS: {
            std::vector<int64_t> g;
            for (const AsmGroup& a : P.groups) {
                g.push_back(a.nmem);
                g.push_back(a.nterms);
                g.push_back(a.uniform);
                g.push_back(a.diag);
            }
            return copy(g.data(), g.size() * 8);
        }
        case SSCO_EXPORT_GROUP_COEF: {
            std::vector<double> c;
            for (const AsmGroup& a : P.groups) c.push_back(a.uniform ? a.coef : 0.0);
            return copy(c.data(), c.size() * 8);
        }
        case SSCO_EXPORT_FRONT_FIRST: return copy(P.front_first.data(), P.front_first.size() * 4);
        case SSCO_EXPORT_FRONT_LEVEL: return copy(P.front_level.data(), P.front_level.size() * 4);
    }
    return fail(h, SSCO_ERR_INVALID_ARG, "unknown export selector");
}

ssco_status ssco_bind(ssco_plan h, void* dev_tables, size_t tables_bytes, void* dev_ws, size_t ws_bytes,
                      void* stream) {
    if (!h || !dev_tables || !dev_ws) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    Plan& P = h->P;
    if (tables_bytes < P.blob.size() || ws_bytes < P.ws.total)
        return fail(h, SSCO_ERR_OOM, "table or workspace buffer smaller than ssco_plan_info reports");
    if (((uintptr_t)dev_tables & 255) || ((uintptr_t)dev_ws & 255))
        return fail(h, SSCO_ERR_INVALID_ARG, "device buffers must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    int e = cudaMemcpyAsync(dev_tables, P.blob.data(), P.blob.size(), cudaMemcpyHostToDevice, s);
    if (e) return cuda_fail(h, e, "table upload");
    e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(h, e, "table upload sync");
    graph_release(P);
    P.d_tab = (uint8_t*)dev_tables;
    P.d_ws = (uint8_t*)dev_ws;
    set_dev_tables(P);
    if (!P.h_flag) {
        e = cudaHostAlloc((void**)&P.h_flag, 64, cudaHostAllocDefault);
        if (e) return cuda_fail(h, e, "pinned flag allocation");
    }
    e = kernels_set_attributes(P);
    if (e) return cuda_fail(h, e, "kernel attributes");
    e = launch_reset_status(P, stream);
    if (e) return cuda_fail(h, e, "status reset");
    P.bound = true;
    P.factored = false;
    return SSCO_OK;
}

ssco_status ssco_numeric(ssco_plan h, const void* vals, int32_t vals_dtype, const double* shift, void* stream) {
    if (!h || !vals || !shift) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    if (vals_dtype != SSCO_VALS_F64 && vals_dtype != SSCO_VALS_F32)
        return fail(h, SSCO_ERR_INVALID_ARG, "unknown vals dtype");
    Plan& P = h->P;
    if (!P.bound) return fail(h, SSCO_ERR_STATE, "ssco_bind has not been called");
    P.launches = 0;
    int e = launch_numeric(P, vals, vals_dtype, shift, stream);
    if (e) return cuda_fail(h, e, "numeric launch");
    P.factored = true;
    return SSCO_OK;
}

ssco_status ssco_solve(ssco_plan h, const double* b, double* x, void* stream) {
    if (!h || !b || !x) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    Plan& P = h->P;
    if (!P.bound || !P.factored) return fail(h, SSCO_ERR_STATE, "ssco_numeric has not run on the bound workspace");
    if (b == x) return fail(h, SSCO_ERR_INVALID_ARG, "b and x alias");
    P.launches = 0;
    bool ok = true;
    int e = launch_solve(P, b, x, stream, &ok);
    if (e) return cuda_fail(h, e, "solve launch");
    return SSCO_OK;
}

ssco_status ssco_backward(ssco_plan h, const double* x, const double* xbar, double* vals_bar, double* shift_bar,
                          double* b_bar, void* stream) {
    if (!h || !x || !xbar || !vals_bar || !b_bar) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    Plan& P = h->P;
    if (!P.bound || !P.factored) return fail(h, SSCO_ERR_STATE, "ssco_numeric has not run on the bound workspace");
    P.launches = 0;
    int e = launch_backward(P, x, xbar, vals_bar, shift_bar, b_bar, stream);
    if (e) return cuda_fail(h, e, "backward launch");
    // ELEM_BLOCKS entries: b_bar now holds mu (same stream)
    e = launch_grad_blocks(P, b_bar, x, vals_bar, stream);
    if (e) return cuda_fail(h, e, "block gradient launch");
    return SSCO_OK;
}

ssco_status ssco_status_get(ssco_plan h, void* stream, int32_t* status, int32_t* iters, double* resid,
                            int32_t* bad_col) {
    if (!h) return fail(h, SSCO_ERR_INVALID_ARG, "NULL plan");
    Plan& P = h->P;
    if (!P.bound) return fail(h, SSCO_ERR_STATE, "not bound");
    cudaStream_t s = (cudaStream_t)stream;
    int e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(h, e, "status sync");
    size_t S = (size_t)P.B * P.n_pats;
    std::vector<int32_t> st(S), it(S), bc(S);
    std::vector<double> rs(S);
    e = cudaMemcpy(st.data(), P.d_ws + P.ws.sstatus, S * 4, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(it.data(), P.d_ws + P.ws.iters, S * 4, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(bc.data(), P.d_ws + P.ws.bad_col, S * 4, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(rs.data(), P.d_ws + P.ws.resid, S * 8, cudaMemcpyDeviceToHost);
    int32_t dev_err = 0;
    if (!e) e = cudaMemcpy(&dev_err, P.d_ws + P.ws.dev_err, 4, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(h, e, "status copy");
    if (dev_err)
        for (size_t i = 0; i < S; ++i) st[i] = SSCO_ERR_TIMEOUT;
    ssco_status worst = SSCO_OK;
    // With GMRES-IR the FP32 factor is only a preconditioner: a non-positive
    // FP32 pivot (replaced by 1, reported in bad_col) does not end the system,
    // whose status is the refinement's (OK once the FP64 residual met the
    // tolerance).
    const bool pivot_is_final = !(P.prec == SSCO_FP32_REFINE && P.refine_mode != 0);
    for (size_t i = 0; i < S; ++i) {
        int32_t sc = bc[i] != INT_MAX && pivot_is_final ? (int32_t)SSCO_ERR_NOT_SPD : st[i];
        if (status) status[i] = sc;
        if (iters) iters[i] = it[i];
        if (resid) resid[i] = rs[i];
        if (bad_col) bad_col[i] = bc[i] != INT_MAX ? bc[i] : -1;
        if (sc != SSCO_OK && worst == SSCO_OK) worst = (ssco_status)sc;
    }
    return worst;
}

ssco_status ssco_export_L(ssco_plan h, double* out, void* stream) {
    if (!h || !out) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    Plan& P = h->P;
    if (!P.bound || !P.factored) return fail(h, SSCO_ERR_STATE, "no factor to export");
    cudaStream_t s = (cudaStream_t)stream;
    int e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(h, e, "export sync");
    size_t nb = (size_t)P.B * P.panel_total * P.tsize;
    std::vector<uint8_t> host(nb);
    e = cudaMemcpy(host.data(), P.d_ws + P.ws.panel, nb, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(h, e, "export copy");
    std::vector<int64_t> cp;
    export_L_pattern(P, &cp, nullptr);
    std::vector<int32_t> pos(P.n, -1);
    int32_t ns = (int32_t)P.snode_first.size() - 1;
    int32_t F = -1;
    for (int32_t sn = 0; sn < ns; ++sn) {
        int32_t f = P.snode_first[sn], w = P.snode_first[sn + 1] - f;
        for (int32_t k = 0; k < w; ++k) {
            int32_t j = f + k;
            // front holding column j
            while (F + 1 < (int32_t)P.fronts.size() && P.front_first[F + 1] <= j) {
                if (F >= 0)
                    for (int32_t q = 0; q < P.fronts[F].r; ++q) pos[P.rows[P.fronts[F].rows_off + q]] = -1;
                ++F;
                for (int32_t q = 0; q < P.fronts[F].r; ++q) pos[P.rows[P.fronts[F].rows_off + q]] = q;
            }
            const FrontDesc& d = P.fronts[F];
            int64_t dst = cp[j];
            for (int64_t q = P.sn_rows_off[sn] + k; q < P.sn_rows_off[sn + 1]; ++q, ++dst) {
                int64_t src = d.panel_off + (int64_t)(j - d.f) * d.r + pos[P.sn_rows[q]];
                for (int32_t b = 0; b < P.B; ++b) {
                    int64_t sidx = (int64_t)b * P.panel_total + src;
                    double v = P.tsize == 8 ? reinterpret_cast<const double*>(host.data())[sidx]
                                            : (double)reinterpret_cast<const float*>(host.data())[sidx];
                    out[(int64_t)b * P.nnzL + dst] = v;
                }
            }
        }
    }
    return SSCO_OK;
}

ssco_status ssco_export_K(ssco_plan h, double* out, void* stream) {
    if (!h || !out) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    Plan& P = h->P;
    if (!P.bound || !P.factored) return fail(h, SSCO_ERR_STATE, "no values to export");
    cudaStream_t s = (cudaStream_t)stream;
    int e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(h, e, "export sync");
    std::vector<double> host((size_t)P.B * P.nnzK);
    e = cudaMemcpy(host.data(), P.d_ws + P.ws.K, host.size() * 8, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(h, e, "export copy");
    for (int32_t b = 0; b < P.B; ++b)
        for (int64_t q = 0; q < P.nnzK; ++q)
            out[(int64_t)b * P.nnzK + q] = host[(int64_t)b * P.nnzK + P.kslot_of_q[q]];
    return SSCO_OK;
}

ssco_status ssco_autotune(ssco_plan h, const void* vals, int32_t vals_dtype, const double* shift, const double* b,
                          double* x, int32_t reps, void* stream, double* best_ms) {
    if (!h || !vals || !shift || !b || !x || reps < 1) return fail(h, SSCO_ERR_INVALID_ARG, "bad argument");
    Plan& P = h->P;
    if (!P.bound) return fail(h, SSCO_ERR_STATE, "ssco_bind has not been called");
    int e = autotune(P, vals, vals_dtype, shift, b, x, reps, stream, best_ms);
    if (e) return cuda_fail(h, e, "autotune");
    P.factored = true;
    return SSCO_OK;
}

ssco_status ssco_graph_run(ssco_plan h, const void* vals, int32_t vals_dtype, const double* shift, const double* b,
                           double* x, void* stream) {
    if (!h || !vals || !shift || !b || !x) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    if (vals_dtype != SSCO_VALS_F64 && vals_dtype != SSCO_VALS_F32)
        return fail(h, SSCO_ERR_INVALID_ARG, "unknown vals dtype");
    Plan& P = h->P;
    if (!P.bound) return fail(h, SSCO_ERR_STATE, "ssco_bind has not been called");
    if (b == x) return fail(h, SSCO_ERR_INVALID_ARG, "b and x alias");
    int e = launch_graph_run(P, vals, vals_dtype, shift, b, x, stream);
    if (e) return cuda_fail(h, e, "graph capture or launch");
    P.factored = true;
    return SSCO_OK;
}

// Per-plan arguments of the multi-plan calls: every plan's pointers, dtype
// and uniqueness first (SSCO_ERR_INVALID_ARG), then their state (bound, b
// and x distinct), so that an argument error is reported whatever the state.
static ssco_status check_many(const ssco_plan* plans, int32_t n, const void* const* vals, const int32_t* vals_dtype,
                              const double* const* shift, const double* const* b, double* const* x,
                              std::vector<Plan*>& ps) {
    for (int32_t i = 0; i < n; ++i) {
        if (!plans[i]) return fail(nullptr, SSCO_ERR_INVALID_ARG, "NULL plan");
        for (int32_t k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return fail(plans[i], SSCO_ERR_INVALID_ARG, "a plan appears twice");
        if (!vals[i] || !shift[i] || !b[i] || !x[i]) return fail(plans[i], SSCO_ERR_INVALID_ARG, "NULL argument");
        if (vals_dtype[i] != SSCO_VALS_F64 && vals_dtype[i] != SSCO_VALS_F32)
            return fail(plans[i], SSCO_ERR_INVALID_ARG, "unknown vals dtype");
    }
    for (int32_t i = 0; i < n; ++i) {
        Plan& P = plans[i]->P;
        if (!P.bound) return fail(plans[i], SSCO_ERR_STATE, "ssco_bind has not been called");
        if (b[i] == x[i]) return fail(plans[i], SSCO_ERR_INVALID_ARG, "b and x alias");
        ps[i] = &P;
    }
    return SSCO_OK;
}

ssco_status ssco_graph_run_many(const ssco_plan* plans, int32_t n_plans, const void* const* vals,
                                const int32_t* vals_dtype, const double* const* shift, const double* const* b,
                                double* const* x, void* stream) {
    if (!plans || n_plans < 1 || n_plans > 1024 || !vals || !vals_dtype || !shift || !b || !x)
        return fail(nullptr, SSCO_ERR_INVALID_ARG, "NULL argument or plan count outside 1..1024");
    std::vector<Plan*> ps(n_plans);
    const ssco_status st = check_many(plans, n_plans, vals, vals_dtype, shift, b, x, ps);
    if (st != SSCO_OK) return st;
    int e = launch_graph_run_many(ps.data(), n_plans, vals, vals_dtype, shift, b, x, stream);
    if (e) return cuda_fail(plans[0], e, "multi-plan graph capture or launch");
    for (Plan* P : ps) P->factored = true;
    return SSCO_OK;
}

ssco_status ssco_autotune_many(const ssco_plan* plans, int32_t n_plans, const void* const* vals,
                               const int32_t* vals_dtype, const double* const* shift, const double* const* b,
                               double* const* x, int32_t reps, void* stream, double* best_ms) {
    if (!plans || n_plans < 1 || n_plans > 1024 || !vals || !vals_dtype || !shift || !b || !x || reps < 1)
        return fail(nullptr, SSCO_ERR_INVALID_ARG, "NULL argument, plan count outside 1..1024 or reps < 1");
    std::vector<Plan*> ps(n_plans);
    const ssco_status st = check_many(plans, n_plans, vals, vals_dtype, shift, b, x, ps);
    if (st != SSCO_OK) return st;
    int e = autotune_many(ps.data(), n_plans, vals, vals_dtype, shift, b, x, reps, stream, best_ms);
    if (e) return cuda_fail(plans[0], e, "multi-plan autotune");
    for (Plan* P : ps) P->factored = true;
    return SSCO_OK;
}

ssco_status ssco_refactor_solve_host(ssco_plan h, const void* vals, int32_t vals_dtype, const double* shift,
                                     const double* b, double* x, void* stream) {
    if (!h || !vals || !shift || !b || !x) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    if (vals_dtype != SSCO_VALS_F64 && vals_dtype != SSCO_VALS_F32)
        return fail(h, SSCO_ERR_INVALID_ARG, "unknown vals dtype");
    Plan& P = h->P;
    if (!P.bound) return fail(h, SSCO_ERR_STATE, "ssco_bind has not been called");
    cudaStream_t s = (cudaStream_t)stream;
    size_t vb = (size_t)P.B * P.m * (vals_dtype == SSCO_VALS_F64 ? 8 : 4);
    size_t nb = (size_t)P.B * P.n * 8;
    size_t sb = (size_t)P.B * P.n_pats * 8;
    int e = cudaMemcpyAsync(P.d_ws + P.ws.st_vals, vals, vb, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(P.d_ws + P.ws.st_shift, shift, sb, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(P.d_ws + P.ws.st_b, b, nb, cudaMemcpyHostToDevice, s);
    if (e) return cuda_fail(h, e, "host-to-device copy");
    e = launch_graph_run(P, P.d_ws + P.ws.st_vals, vals_dtype, (const double*)(P.d_ws + P.ws.st_shift),
                         (const double*)(P.d_ws + P.ws.st_b), (double*)(P.d_ws + P.ws.st_x), stream);
    if (e) return cuda_fail(h, e, "graph capture or launch");
    P.factored = true;
    e = cudaMemcpyAsync(x, P.d_ws + P.ws.st_x, nb, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(h, e, "device-to-host copy");
    return SSCO_OK;
}

int64_t ssco_last_launch_count(ssco_plan h) { return h ? h->P.launches : 0; }

ssco_status ssco_set_flow(ssco_plan h, int32_t flow, int64_t max_polls, int32_t stall_item) {
    if (!h) return fail(h, SSCO_ERR_INVALID_ARG, "NULL plan");
    if (flow < 0 || flow > 31 || max_polls < 0 || max_polls > 0xFFFFFFFFll || stall_item < -1)
        return fail(h, SSCO_ERR_INVALID_ARG, "flow must be 0..31, max_polls 0..2^32-1, stall_item >= -1");
    Plan& P = h->P;
    P.tune.flow = flow & 3;
    P.tune.front_core = (flow >> 2) & 1;
    P.tune.big_fuse = (flow >> 3) & 1;
    P.no_graphs = ((flow >> 4) & 1) != 0;
    if (max_polls > 0) P.tune.flow_polls = (uint32_t)max_polls;
    P.tune.flow_stall = stall_item;
    graph_release(P);
    return SSCO_OK;
}

ssco_status ssco_solve_noalloc(ssco_plan h, const double* b, double* x, void* stream) {
    if (!h || !b || !x) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    Plan& P = h->P;
    if (P.prec != SSCO_FP64) return fail(h, SSCO_ERR_UNSUPPORTED, "ssco_solve_noalloc needs an SSCO_FP64 plan");
    size_t need = static_solve_scratch_need(P), have = static_solve_scratch_bytes();
    if (need > have)
        return fail(h, SSCO_ERR_UNSUPPORTED,
                    "ssco_solve_noalloc: plan needs " + std::to_string(need) + " bytes of scratch, the static array holds " +
                        std::to_string(have));
    if (!P.bound || !P.factored) return fail(h, SSCO_ERR_STATE, "ssco_numeric has not run on the bound workspace");
    if (b == x) return fail(h, SSCO_ERR_INVALID_ARG, "b and x alias");
    P.launches = 0;
    int e = launch_solve_static(P, b, x, stream);
    if (e) return cuda_fail(h, e, "noalloc solve launch");
    return SSCO_OK;
}

ssco_status ssco_profile_enable(ssco_plan h, int32_t max_launches) {
    if (!h || max_launches < 0) return fail(h, SSCO_ERR_INVALID_ARG, "bad argument");
    int e = profile_enable(h->P, max_launches);
    if (e) return cuda_fail(h, e, "event pool");
    return SSCO_OK;
}

ssco_status ssco_profile_read(ssco_plan h, ssco_kernel_stat* out) {
    if (!h || !out) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    int e = profile_read(h->P, out);
    if (e) return cuda_fail(h, e, "profile read");
    return SSCO_OK;
}

const char* ssco_kernel_name(int32_t kind) { return kernel_kind_name(kind); }

ssco_status ssco_profile_trace(ssco_plan h, int32_t* kinds, float* ms, double* flops, double* bytes, int64_t cap,
                               int64_t* n) {
    if (!h || !n || cap < 0) return fail(h, SSCO_ERR_INVALID_ARG, "bad argument");
    int e = profile_trace(h->P, kinds, ms, flops, bytes, cap, n);
    if (e) return cuda_fail(h, e, "profile trace");
    return SSCO_OK;
}

ssco_status ssco_plan_save(ssco_plan h, const char* path) {
    if (!h || !path) return fail(h, SSCO_ERR_INVALID_ARG, "NULL argument");
    Writer w;
    w.f.open(path, std::ios::binary | std::ios::trunc);
    if (!w.f) return fail(h, SSCO_ERR_INVALID_ARG, std::string("cannot open ") + path);
    w.pod(kMagic);
    w.pod(kVersion);
    serialize(w, h->P);
    const uint64_t digest = w.sum.h;
    w.f.write(reinterpret_cast<const char*>(&digest), sizeof(digest));
    w.f.flush();
    if (!w.f) return fail(h, SSCO_ERR_INVALID_ARG, "write failed");
    return SSCO_OK;
}

ssco_status ssco_plan_load(const char* path, ssco_plan* out) {
    if (!path || !out) return fail(nullptr, SSCO_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    Reader r;
    r.f.open(path, std::ios::binary | std::ios::ate);
    if (!r.f) return fail(nullptr, SSCO_ERR_INVALID_ARG, std::string("cannot open ") + path);
    r.size = r.f.tellg();
    r.f.seekg(0);
    uint64_t magic = 0;
    uint32_t ver = 0;
    if (!r.pod(magic) || !r.pod(ver) || magic != kMagic || ver != kVersion)
        return fail(nullptr, SSCO_ERR_INVALID_ARG, "not a plan file of this version");
    ssco_plan h = new (std::nothrow) ssco_plan_s();
    if (!h) return fail(nullptr, SSCO_ERR_OOM, "host allocation failed");
    bool ok = false;
    try {  // a damaged length field must not take the process down
        ok = serialize(r, h->P);
    } catch (const std::exception&) {
        ok = false;
    }
    const uint64_t got = r.sum.h;
    uint64_t digest = 0;
    char extra = 0;
    ok = ok && (bool)r.f.read(reinterpret_cast<char*>(&digest), sizeof(digest)) && digest == got &&
         !r.f.read(&extra, 1);
    // options that size the workspace must be in their documented ranges
    ok = ok && h->P.refine_mode >= 0 && h->P.refine_mode <= 2 && h->P.gmres_m >= 1 && h->P.gmres_m <= 64;
    if (!ok) {
        delete h;
        return fail(nullptr, SSCO_ERR_INVALID_ARG, "truncated or corrupt plan file (checksum)");
    }
    if (!launch_lists_consistent(h->P)) {
        delete h;
        return fail(nullptr, SSCO_ERR_INVALID_ARG, "inconsistent plan file (launch lists)");
    }
    build_blob(h->P);
    compute_ws_layout(h->P);
    *out = h;
    return SSCO_OK;
}

void ssco_destroy(ssco_plan h) {
    if (!h) return;
    if (!h->P.ev_pool.empty()) profile_enable(h->P, 0);
    graph_release(h->P);
    graph_destroy_streams(h->P);
    if (h->P.h_flag) cudaFreeHost(h->P.h_flag);
    delete h;
}

}  // extern "C"
