// ssco_symbolic.cpp -- host symbolic phase: everything that depends only on
// the sparsity structure, computed once per plan.
//
// Mapping to the paper's method (Sec. 4):
//  * Unrolling the program for a fixed structure (Sec. 3.1/4.7) is done at
//    the granularity of K entries (assembly) and of dense fronts (Cholesky):
//    per-entry expression trees of L would be far too many (the factor of a
//    3D problem has ~1e8-1e9 entries), so a front -- a fundamental or
//    relaxed-amalgamated supernode -- plays the role of an explicitly tagged
//    dense block (Sec. 4.2.4) whose intermediates (the update matrix) are
//    global intermediates stored once (Sec. 4.2.1).
//  * Grouping by structure and level (Sec. 4.3): assembly entries are grouped
//    by (pattern, term count, diagonal flag, constant-add); fronts by
//    (height in the supernodal forest, size class).  Height (longest path
//    from the leaves) guarantees no front depends on another of its level.
//  * Leaf harvesting (Sec. 4.4, App. B): each assembly group stores its leaf
//    table term-major / member-innermost (the coalesced layout of Sec. 4.8);
//    a constant shared by all terms of a group (+-1 for incidence matrices)
//    is folded into the group ("uniform") instead of being stored per term.
//  * Address coherence (Sec. 4.8): a front addresses its rows through one
//    relative map per (child, parent) pair instead of per-entry indices.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "ssco_internal.h"

namespace ssco {

namespace {

struct Term {
    int32_t row;
    int32_t vidx;
    double coef;
};

ssco_status bad(Plan& P, ssco_status s, const std::string& msg) {
    P.last_error = msg;
    return s;
}

ssco_status validate(Plan& P, const ssco_pattern* p, int k) {
    std::string pre = "pattern " + std::to_string(k) + ": ";
    if (!p) return bad(P, SSCO_ERR_INVALID_ARG, pre + "NULL pattern");
    if (p->kind != SSCO_KIND_ATWA && p->kind != SSCO_KIND_ELEM && p->kind != SSCO_KIND_ELEM_BLOCKS)
        return bad(P, SSCO_ERR_INVALID_ARG, pre + "unknown kind");
    if (p->n < 1 || p->m < 0) return bad(P, SSCO_ERR_INVALID_ARG, pre + "n must be >= 1, m >= 0");
    std::vector<int32_t> mark((size_t)p->n, -1);
    if (p->kind == SSCO_KIND_ATWA) {
        if (!p->rowptr) return bad(P, SSCO_ERR_INVALID_ARG, pre + "rowptr is NULL");
        if (p->rowptr[0] != 0) return bad(P, SSCO_ERR_PATTERN, pre + "rowptr[0] != 0");
        for (int32_t e = 0; e < p->m; ++e)
            if (p->rowptr[e + 1] < p->rowptr[e])
                return bad(P, SSCO_ERR_PATTERN, pre + "rowptr decreases at row " + std::to_string(e));
        int64_t nnz = p->rowptr[p->m];
        if (nnz > 0 && (!p->colind || !p->aval))
            return bad(P, SSCO_ERR_INVALID_ARG, pre + "colind/aval is NULL");
        for (int32_t e = 0; e < p->m; ++e) {
            for (int64_t a = p->rowptr[e]; a < p->rowptr[e + 1]; ++a) {
                int32_t c = p->colind[a];
                if (c < 0 || c >= p->n)
                    return bad(P, SSCO_ERR_PATTERN, pre + "column index out of range in row " + std::to_string(e));
                if (mark[c] == e)
                    return bad(P, SSCO_ERR_PATTERN, pre + "duplicate column in row " + std::to_string(e));
                mark[c] = e;
                if (!std::isfinite(p->aval[a]))
                    return bad(P, SSCO_ERR_NONFINITE, pre + "non-finite entry of A");
            }
        }
    } else {
        if (p->elem_dim < 1 || p->elem_dim > 64)
            return bad(P, SSCO_ERR_INVALID_ARG, pre + "elem_dim must be in [1, 64]");
        const bool blocks = p->kind == SSCO_KIND_ELEM_BLOCKS;  // element blocks come per call
        if (p->m > 0 && (!p->elem_dofs || (!blocks && !p->elem_K0)))
            return bad(P, SSCO_ERR_INVALID_ARG, pre + "elem_dofs/elem_K0 is NULL");
        int64_t npk = (int64_t)p->elem_dim * (p->elem_dim + 1) / 2;
        if (blocks && (int64_t)p->m * npk >= (int64_t)INT32_MAX)
            return bad(P, SSCO_ERR_UNSUPPORTED, pre + "element block values exceed int32");
        for (int32_t e = 0; e < p->m; ++e) {
            for (int32_t i = 0; i < p->elem_dim; ++i) {
                int32_t d = p->elem_dofs[(int64_t)e * p->elem_dim + i];
                if (d < -1 || d >= p->n)
                    return bad(P, SSCO_ERR_PATTERN, pre + "DOF index out of range in element " + std::to_string(e));
                if (d >= 0) {
                    if (mark[d] == e)
                        return bad(P, SSCO_ERR_PATTERN, pre + "duplicate DOF in element " + std::to_string(e));
                    mark[d] = e;
                }
            }
            for (int64_t q = 0; q < npk && !blocks; ++q)
                if (!std::isfinite(p->elem_K0[(int64_t)e * npk + q]))
                    return bad(P, SSCO_ERR_NONFINITE, pre + "non-finite element block entry");
        }
    }
    if (p->perm) {
        std::vector<char> seen((size_t)p->n, 0);
        for (int32_t i = 0; i < p->n; ++i) {
            int32_t v = p->perm[i];
            if (v < 0 || v >= p->n || seen[v]) return bad(P, SSCO_ERR_PATTERN, pre + "perm is not a permutation");
            seen[v] = 1;
        }
    }
    return SSCO_OK;
}

constexpr int32_t kClasses[] = {32, 64, 96, 128, 160, 192, 224, 256, 288, 320};

// Program of one tiny subtree (int32 words), loaded whole into shared memory
// by the warp that runs it:
//   header [kTinyHdrWords]: nfronts, nk, rec_off, child_off, k_off, map_off, total, sys
//   per front (children first) [kTinyRecWords]: r, w, f, nchild, child list
//     offset, first K entry, K count, relmap offset (into the parent, -1 for
//     the subtree root), below-rows offset, pad, panel_off (2 words), upd_off
//     (2), pvec_off (2)
//   child lists (local front indices), K entries (kslot, row*33 + col),
//   relative maps, below-row lists (global row indices).
void build_tiny_programs(Plan& P) {
    P.tiny_prog.clear();
    P.tiny_prog_off.assign(1, 0);
    P.tiny_prog_max = 0;
    P.tiny_k_max = 0;
    std::vector<int32_t> local(P.fronts.size(), -1);
    for (int32_t st = 0; st < P.n_tiny; ++st) {
        const int32_t q0 = P.tiny_off[st], q1 = P.tiny_off[st + 1], nfq = q1 - q0;
        for (int32_t q = q0; q < q1; ++q) local[P.tiny_list[q]] = q - q0;
        int64_t nch = 0, nk = 0, nmap = 0;
        for (int32_t q = q0; q < q1; ++q) {
            const FrontDesc& d = P.fronts[P.tiny_list[q]];
            nch += d.nchild;
            nk += d.klist_n;
            nmap += d.r - d.w;
        }
        const int64_t rec_off = kTinyHdrWords, child_off = rec_off + (int64_t)kTinyRecWords * nfq;
        const int64_t k_off = child_off + nch, map_off = k_off + 2 * nk, rows_off = map_off + nmap;
        const int64_t total = rows_off + nmap;
        std::vector<int32_t> g(total, 0);
        g[0] = nfq;
        g[1] = (int32_t)nk;
        g[2] = (int32_t)rec_off;
        g[3] = (int32_t)child_off;
        g[4] = (int32_t)k_off;
        g[5] = (int32_t)map_off;
        g[6] = (int32_t)total;
        g[7] = P.fronts[P.tiny_list[q0]].sys;
        int64_t cpos = child_off, kpos = 0, mpos = map_off, rpos = rows_off;
        for (int32_t q = q0; q < q1; ++q) {
            const FrontDesc& d = P.fronts[P.tiny_list[q]];
            int32_t* rec = &g[rec_off + (int64_t)kTinyRecWords * (q - q0)];
            rec[0] = d.r;
            rec[1] = d.w;
            rec[2] = d.f;
            rec[3] = d.nchild;
            rec[4] = (int32_t)cpos;
            rec[5] = (int32_t)kpos;
            rec[6] = d.klist_n;
            for (int32_t c = 0; c < d.nchild; ++c) g[cpos++] = local[P.child_ids[d.child_off + c]];
            for (int32_t e = 0; e < d.klist_n; ++e) {
                const int32_t slot = P.klist[2 * (d.klist_off + e)], pos = P.klist[2 * (d.klist_off + e) + 1];
                const int32_t col = pos / d.r, row = pos % d.r;
                g[k_off + 2 * (kpos + e)] = slot;
                g[k_off + 2 * (kpos + e) + 1] = row * 33 + col;
            }
            kpos += d.klist_n;
            const bool has_parent_inside = d.parent >= 0 && local[d.parent] >= 0;
            rec[7] = has_parent_inside ? (int32_t)mpos : -1;
            for (int32_t k = 0; k < d.r - d.w; ++k) g[mpos++] = has_parent_inside ? P.relmap[d.relmap_off + k] : 0;
            rec[8] = (int32_t)rpos;
            for (int32_t k = 0; k < d.r - d.w; ++k) g[rpos++] = P.rows[d.rows_off + d.w + k];
            rec[10] = (int32_t)(d.panel_off & 0xffffffff);
            rec[11] = (int32_t)(d.panel_off >> 32);
            rec[12] = (int32_t)(d.upd_off & 0xffffffff);
            rec[13] = (int32_t)(d.upd_off >> 32);
            rec[14] = (int32_t)(d.pvec_off & 0xffffffff);
            rec[15] = (int32_t)(d.pvec_off >> 32);
        }
        for (int32_t q = q0; q < q1; ++q) local[P.tiny_list[q]] = -1;
        P.tiny_prog.insert(P.tiny_prog.end(), g.begin(), g.end());
        P.tiny_prog_off.push_back((int64_t)P.tiny_prog.size());
        P.tiny_prog_max = std::max<int32_t>(P.tiny_prog_max, (int32_t)total);
        P.tiny_k_max = std::max<int32_t>(P.tiny_k_max, (int32_t)nk);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
ssco_status analyze_impl(const ssco_pattern* const* pats, int32_t n_pats, const ssco_op* op, Plan& P) {
    if (!pats || n_pats < 1 || !op) return bad(P, SSCO_ERR_INVALID_ARG, "pats/op NULL or n_pats < 1");
    if (op->precision != SSCO_FP64 && op->precision != SSCO_FP32_REFINE)
        return bad(P, SSCO_ERR_INVALID_ARG, "unknown precision");
    if (op->batch < 1) return bad(P, SSCO_ERR_INVALID_ARG, "batch must be >= 1");
    // value sets are a grid dimension of the level launches
    if (op->batch > 65535) return bad(P, SSCO_ERR_INVALID_ARG, "batch must be <= 65535");
    P.prec = op->precision;
    P.B = op->batch;
    P.tol = op->refine_tol > 0 ? op->refine_tol : 1e-10;
    P.maxit = op->refine_max_iter > 0 ? op->refine_max_iter : 30;
    if (op->refine_mode < 0 || op->refine_mode > 2) return bad(P, SSCO_ERR_INVALID_ARG, "refine_mode must be 0, 1 or 2");
    if (op->gmres_restart < 0 || op->gmres_restart > 64)
        return bad(P, SSCO_ERR_INVALID_ARG, "gmres_restart must be in 0..64");
    P.refine_mode = op->precision == SSCO_FP32_REFINE ? op->refine_mode : 0;
    P.gmres_m = op->gmres_restart > 0 ? op->gmres_restart : 16;
    if (op->vec2_max_cls != 0 && op->vec2_max_cls != 128 && op->vec2_max_cls != 160)
        return bad(P, SSCO_ERR_INVALID_ARG, "vec2_max_cls must be 0, 128 or 160");
    P.tune.vec2_max_cls = op->precision == SSCO_FP32_REFINE ? op->vec2_max_cls : 0;
    P.tsize = P.prec == SSCO_FP64 ? 8 : 4;
    // One CTA per (front, instance) holds the front as a packed lower
    // triangle in shared memory (r(r+1)/2 * sizeof(T) <= 227 KB).  Its
    // column steps are sequential, so wide fronts only pay off there when the
    // batch supplies many CTAs; otherwise they take the multi-CTA path.
    int32_t smax_default = P.B >= 32 ? (P.prec == SSCO_FP64 ? 224 : 320) : (P.prec == SSCO_FP64 ? 160 : 224);
    P.small_max = op->small_front_max > 0 ? std::min(op->small_front_max, smax_default) : smax_default;
    P.amalg = op->amalgamate;
    P.tiny_max = op->tiny_front_max == 0 ? 32 : (op->tiny_front_max < 0 ? 0 : std::min(op->tiny_front_max, 32));
    P.n_pats = n_pats;
    P.tune.use_tc = op->tensor_cores < 0 ? 0 : (op->tensor_cores == 2 ? 2 : 1);
    if (op->big_panel != 0 && (op->big_panel < 32 || op->big_panel > 1024 || op->big_panel % 32 != 0))
        return bad(P, SSCO_ERR_INVALID_ARG, "big_panel must be 0 or a multiple of 32 in [32, 1024]");
    if (op->big_panel > 0) P.tune.big_panel = op->big_panel;
    if (op->split_rows < -1) return bad(P, SSCO_ERR_INVALID_ARG, "split_rows must be >= -1");
    // Defaults by batch: few value sets leave the level kernels short of
    // CTAs, so large fronts get a CTA cluster each (measured on the 24^3
    // elasticity: 78 vs 52 systems/s); with many value sets the clusters
    // only add cost and the multi-launch split pays from 1024 rows (48^3,
    // 16 value sets).
    P.tune.split_rows = P.B >= 8 ? 1024 : 2048;
    P.tune.cluster_rows = P.B <= 4 ? 512 : (1 << 30);
    if (op->split_rows != 0) P.tune.split_rows = op->split_rows < 0 ? (1 << 30) : op->split_rows;
    if (op->warp_front_max < -1 || op->warp_front_max > 64)
        return bad(P, SSCO_ERR_INVALID_ARG, "warp_front_max must be in [-1, 64]");
    P.tune.warp_front_max = op->warp_front_max > 0 ? op->warp_front_max : 0;
    if (op->cluster_rows < -1) return bad(P, SSCO_ERR_INVALID_ARG, "cluster_rows must be >= -1");
    if (op->cluster_rows != 0) P.tune.cluster_rows = op->cluster_rows < 0 ? (1 << 30) : op->cluster_rows;

    for (int k = 0; k < n_pats; ++k) {
        ssco_status s = validate(P, pats[k], k);
        if (s != SSCO_OK) return s;
    }
    // --- concatenation -----------------------------------------------------
    P.pats.resize(n_pats);
    int64_t n = 0, m = 0;
    for (int k = 0; k < n_pats; ++k) {
        PatMeta& pm = P.pats[k];
        pm.kind = pats[k]->kind;
        pm.n = pats[k]->n;
        pm.dim = pats[k]->kind == SSCO_KIND_ATWA ? 0 : pats[k]->elem_dim;
        // values per set: one per row / element, or every packed block entry
        pm.m = pats[k]->kind == SSCO_KIND_ELEM_BLOCKS ? pats[k]->m * (pm.dim * (pm.dim + 1) / 2) : pats[k]->m;
        pm.n_off = n;
        pm.m_off = m;
        n += pm.n;
        m += pm.m;
    }
    if (n >= (int64_t)INT32_MAX || m >= (int64_t)INT32_MAX)
        return bad(P, SSCO_ERR_UNSUPPORTED, "total n or m exceeds int32");
    P.n = n;
    P.m = m;
    P.perm.resize(n);
    std::vector<int32_t> iperm(n);
    for (int k = 0; k < n_pats; ++k) {
        const PatMeta& pm = P.pats[k];
        for (int32_t i = 0; i < pm.n; ++i) {
            int32_t old = pats[k]->perm ? pats[k]->perm[i] : i;
            P.perm[pm.n_off + i] = (int32_t)(pm.n_off + old);
            iperm[pm.n_off + old] = (int32_t)(pm.n_off + i);
        }
    }

    // --- K~ pattern and per-entry terms ------------------------------------
    std::vector<int64_t> tcount(n + 1, 0);
    std::vector<char> referenced(n, 0);
    for (int k = 0; k < n_pats; ++k) {
        const ssco_pattern* p = pats[k];
        if (p->kind == SSCO_KIND_ATWA) {
            for (int32_t e = 0; e < p->m; ++e)
                for (int64_t a = p->rowptr[e]; a < p->rowptr[e + 1]; ++a)
                    for (int64_t b = a; b < p->rowptr[e + 1]; ++b) {
                        int32_t u = iperm[P.pats[k].n_off + p->colind[a]];
                        int32_t v = iperm[P.pats[k].n_off + p->colind[b]];
                        tcount[std::min(u, v) + 1]++;
                    }
        } else {
            int32_t d = p->elem_dim;
            for (int32_t e = 0; e < p->m; ++e)
                for (int32_t i = 0; i < d; ++i)
                    for (int32_t j = 0; j <= i; ++j) {
                        int32_t gu = p->elem_dofs[(int64_t)e * d + i], gv = p->elem_dofs[(int64_t)e * d + j];
                        if (gu < 0 || gv < 0) continue;
                        int32_t u = iperm[P.pats[k].n_off + gu], v = iperm[P.pats[k].n_off + gv];
                        tcount[std::min(u, v) + 1]++;
                        referenced[u] = referenced[v] = 1;
                    }
        }
    }
    for (int64_t j = 0; j < n; ++j) tcount[j + 1] += tcount[j];
    std::vector<Term> terms((size_t)tcount[n]);
    {
        std::vector<int64_t> fill(tcount.begin(), tcount.end() - 1);
        for (int k = 0; k < n_pats; ++k) {
            const ssco_pattern* p = pats[k];
            const PatMeta& pm = P.pats[k];
            if (p->kind == SSCO_KIND_ATWA) {
                for (int32_t e = 0; e < p->m; ++e)
                    for (int64_t a = p->rowptr[e]; a < p->rowptr[e + 1]; ++a)
                        for (int64_t b = a; b < p->rowptr[e + 1]; ++b) {
                            int32_t u = iperm[pm.n_off + p->colind[a]];
                            int32_t v = iperm[pm.n_off + p->colind[b]];
                            Term t{std::max(u, v), (int32_t)(pm.m_off + e), p->aval[a] * p->aval[b]};
                            terms[fill[std::min(u, v)]++] = t;
                        }
            } else {
                int32_t d = p->elem_dim;
                for (int32_t e = 0; e < p->m; ++e) {
                    int32_t q = 0;
                    for (int32_t i = 0; i < d; ++i)
                        for (int32_t j = 0; j <= i; ++j, ++q) {
                            int32_t gu = p->elem_dofs[(int64_t)e * d + i], gv = p->elem_dofs[(int64_t)e * d + j];
                            if (gu < 0 || gv < 0) continue;
                            int32_t u = iperm[pm.n_off + gu], v = iperm[pm.n_off + gv];
                            const int64_t npk = (int64_t)d * (d + 1) / 2;
                            // ELEM: E_e times the constant entry; ELEM_BLOCKS: the entry itself
                            Term t = p->kind == SSCO_KIND_ELEM_BLOCKS
                                         ? Term{std::max(u, v), (int32_t)(pm.m_off + e * npk + q), 1.0}
                                         : Term{std::max(u, v), (int32_t)(pm.m_off + e), p->elem_K0[e * npk + q]};
                            terms[fill[std::min(u, v)]++] = t;
                        }
                }
            }
        }
    }
    // per column: stable sort by row (generation order kept within a row)
    std::vector<int32_t> row_sys(n);
    for (int k = 0; k < n_pats; ++k)
        for (int64_t i = P.pats[k].n_off; i < P.pats[k].n_off + P.pats[k].n; ++i) row_sys[i] = k;
    P.Kcolptr.assign(n + 1, 0);
    P.Krowind.clear();
    // slots in CSC order with their term ranges
    std::vector<int64_t> slot_tbeg, slot_tend;
    std::vector<int32_t> slot_diag;   // 1: receives the shift
    std::vector<double> slot_cadd;
    slot_tbeg.reserve(tcount[n] / 2 + n);
    for (int64_t j = 0; j < n; ++j) {
        auto b0 = terms.begin() + tcount[j], b1 = terms.begin() + tcount[j + 1];
        std::stable_sort(b0, b1, [](const Term& x, const Term& y) { return x.row < y.row; });
        int k = row_sys[j];
        bool elem = P.pats[k].kind != SSCO_KIND_ATWA;
        // diagonal first, always present
        int64_t t = tcount[j];
        int64_t te = t;
        while (te < tcount[j + 1] && terms[te].row == j) ++te;
        P.Krowind.push_back((int32_t)j);
        slot_tbeg.push_back(t);
        slot_tend.push_back(te);
        if (elem && !referenced[j]) {
            slot_diag.push_back(0);
            slot_cadd.push_back(1.0);
        } else {
            slot_diag.push_back(1);
            slot_cadd.push_back(0.0);
        }
        t = te;
        while (t < tcount[j + 1]) {
            int32_t r = terms[t].row;
            te = t;
            while (te < tcount[j + 1] && terms[te].row == r) ++te;
            P.Krowind.push_back(r);
            slot_tbeg.push_back(t);
            slot_tend.push_back(te);
            slot_diag.push_back(0);
            slot_cadd.push_back(0.0);
            t = te;
        }
        P.Kcolptr[j + 1] = (int64_t)P.Krowind.size();
    }
    P.nnzK = (int64_t)P.Krowind.size();
    if (P.nnzK >= (int64_t)INT32_MAX) return bad(P, SSCO_ERR_UNSUPPORTED, "nnz(K) exceeds int32");

    // --- assembly groups (Sec. 4.3 / 4.4) ---------------------------------
    {
        struct Key {
            int32_t sys, nterms, diag;
            double cadd;
            bool operator<(const Key& o) const {
                if (sys != o.sys) return sys < o.sys;
                if (diag != o.diag) return diag < o.diag;
                if (cadd != o.cadd) return cadd < o.cadd;
                return nterms < o.nterms;
            }
        };
        std::vector<int64_t> order(P.nnzK);
        std::iota(order.begin(), order.end(), 0);
        std::vector<int32_t> slot_col(P.nnzK);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t q = P.Kcolptr[j]; q < P.Kcolptr[j + 1]; ++q) slot_col[q] = (int32_t)j;
        auto key_of = [&](int64_t q) {
            return Key{row_sys[slot_col[q]], (int32_t)(slot_tend[q] - slot_tbeg[q]), slot_diag[q], slot_cadd[q]};
        };
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key_of(a) < key_of(b); });
        P.kslot_of_q.assign(P.nnzK, 0);
        P.groups.clear();
        P.asm_idx.clear();
        P.asm_coef.clear();
        int64_t g0 = 0;
        while (g0 < P.nnzK) {
            Key kk = key_of(order[g0]);
            int64_t g1 = g0;
            while (g1 < P.nnzK) {
                Key k2 = key_of(order[g1]);
                if (k2.sys != kk.sys || k2.nterms != kk.nterms || k2.diag != kk.diag || k2.cadd != kk.cadd) break;
                ++g1;
            }
            AsmGroup g{};
            g.nmem = (int32_t)(g1 - g0);
            g.nterms = kk.nterms;
            g.diag = kk.diag;
            g.sys = kk.sys;
            g.cadd = kk.cadd;
            g.slot_base = g0;
            // uniform constant?
            bool uniform = true;
            double c0 = 0.0;
            bool have = false;
            for (int64_t i = g0; i < g1 && uniform; ++i)
                for (int64_t t = slot_tbeg[order[i]]; t < slot_tend[order[i]]; ++t) {
                    if (!have) {
                        c0 = terms[t].coef;
                        have = true;
                    } else if (terms[t].coef != c0) {
                        uniform = false;
                        break;
                    }
                }
            g.uniform = uniform ? 1 : 0;
            g.coef = uniform ? c0 : 0.0;
            g.idx_off = (int64_t)P.asm_idx.size();
            g.coef_off = uniform ? 0 : (int64_t)P.asm_coef.size();
            P.asm_idx.resize(P.asm_idx.size() + (size_t)g.nmem * g.nterms);
            if (!uniform) P.asm_coef.resize(P.asm_coef.size() + (size_t)g.nmem * g.nterms);
            for (int64_t i = g0; i < g1; ++i) {
                int64_t q = order[i];
                P.kslot_of_q[q] = (int32_t)i;
                for (int32_t t = 0; t < g.nterms; ++t) {
                    const Term& tm = terms[slot_tbeg[q] + t];
                    P.asm_idx[g.idx_off + (int64_t)t * g.nmem + (i - g0)] = tm.vidx;
                    if (!uniform) P.asm_coef[g.coef_off + (int64_t)t * g.nmem + (i - g0)] = tm.coef;
                }
            }
            P.groups.push_back(g);
            g0 = g1;
        }
        P.chunks.clear();
        for (size_t gi = 0; gi < P.groups.size(); ++gi)
            for (int32_t s = 0; s < P.groups[gi].nmem; s += 256) P.chunks.push_back(AsmChunk{(int32_t)gi, s});
    }
    std::vector<Term>().swap(terms);

    // --- elimination forest (Liu's algorithm with path compression) --------
    // strict-lower row lists of K~
    std::vector<int64_t> rptr(n + 1, 0);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = P.Kcolptr[j] + 1; q < P.Kcolptr[j + 1]; ++q) rptr[P.Krowind[q] + 1]++;
    for (int64_t i = 0; i < n; ++i) rptr[i + 1] += rptr[i];
    std::vector<int32_t> rcol(rptr[n]);
    {
        std::vector<int64_t> fill(rptr.begin(), rptr.end() - 1);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t q = P.Kcolptr[j] + 1; q < P.Kcolptr[j + 1]; ++q) rcol[fill[P.Krowind[q]]++] = (int32_t)j;
    }
    P.parent.assign(n, -1);
    {
        std::vector<int32_t> anc(n, -1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t q = rptr[i]; q < rptr[i + 1]; ++q) {
                int32_t r = rcol[q];
                while (anc[r] != -1 && anc[r] != i) {
                    int32_t t = anc[r];
                    anc[r] = (int32_t)i;
                    r = t;
                }
                if (anc[r] == -1) {
                    anc[r] = (int32_t)i;
                    P.parent[r] = (int32_t)i;
                }
            }
    }
    // --- column counts by row-subtree traversal ----------------------------
    P.colcount.assign(n, 1);
    {
        std::vector<int32_t> mark(n, -1);
        for (int64_t i = 0; i < n; ++i) {
            mark[i] = (int32_t)i;
            for (int64_t q = rptr[i]; q < rptr[i + 1]; ++q) {
                int32_t k = rcol[q];
                while (mark[k] != i) {
                    mark[k] = (int32_t)i;
                    P.colcount[k]++;
                    k = P.parent[k];
                }
            }
        }
    }
    std::vector<int64_t>().swap(rptr);
    std::vector<int32_t>().swap(rcol);
    P.nnzL = 0;
    P.flops_exact = 0;
    for (int64_t j = 0; j < n; ++j) {
        P.nnzL += P.colcount[j];
        P.flops_exact += (double)P.colcount[j] * P.colcount[j];
    }
    // column levels (height)
    P.col_level.assign(n, 0);
    std::vector<int32_t> nchild(n, 0);
    for (int64_t j = 0; j < n; ++j)
        if (P.parent[j] >= 0) {
            nchild[P.parent[j]]++;
            P.col_level[P.parent[j]] = std::max(P.col_level[P.parent[j]], P.col_level[j] + 1);
        }
    P.max_col_level = 0;
    for (int64_t j = 0; j < n; ++j) P.max_col_level = std::max(P.max_col_level, P.col_level[j]);

    // --- fundamental supernodes -------------------------------------------
    P.snode_first.clear();
    for (int64_t j = 0; j < n; ++j) {
        bool joins = j > 0 && P.parent[j - 1] == j && nchild[j] == 1 && P.colcount[j] == P.colcount[j - 1] - 1;
        if (!joins) P.snode_first.push_back((int32_t)j);
    }
    int32_t ns = (int32_t)P.snode_first.size();
    P.snode_first.push_back((int32_t)n);
    std::vector<int32_t> col2sn(n);
    for (int32_t s = 0; s < ns; ++s)
        for (int32_t j = P.snode_first[s]; j < P.snode_first[s + 1]; ++j) col2sn[j] = s;
    P.sn_parent.assign(ns, -1);
    P.sn_level.assign(ns, 0);
    for (int32_t s = 0; s < ns; ++s) {
        int32_t last = P.snode_first[s + 1] - 1;
        if (P.parent[last] >= 0) P.sn_parent[s] = col2sn[P.parent[last]];
    }
    for (int32_t s = 0; s < ns; ++s)
        if (P.sn_parent[s] >= 0) P.sn_level[P.sn_parent[s]] = std::max(P.sn_level[P.sn_parent[s]], P.sn_level[s] + 1);
    // supernode row structures
    {
        std::vector<int32_t> sn_head(ns, -1), sn_next(ns, -1);
        for (int32_t s = ns - 1; s >= 0; --s)
            if (P.sn_parent[s] >= 0) {
                sn_next[s] = sn_head[P.sn_parent[s]];
                sn_head[P.sn_parent[s]] = s;
            }
        std::vector<int32_t> mark(n, -1);
        P.sn_rows_off.assign(ns + 1, 0);
        P.sn_rows.clear();
        std::vector<int32_t> below;
        for (int32_t s = 0; s < ns; ++s) {
            int32_t f = P.snode_first[s], l = P.snode_first[s + 1] - 1;
            below.clear();
            for (int32_t j = f; j <= l; ++j)
                for (int64_t q = P.Kcolptr[j]; q < P.Kcolptr[j + 1]; ++q) {
                    int32_t i = P.Krowind[q];
                    if (i > l && mark[i] != s) {
                        mark[i] = s;
                        below.push_back(i);
                    }
                }
            for (int32_t c = sn_head[s]; c >= 0; c = sn_next[c])
                for (int64_t q = P.sn_rows_off[c]; q < P.sn_rows_off[c + 1]; ++q) {
                    int32_t i = P.sn_rows[q];
                    if (i > l && mark[i] != s) {
                        mark[i] = s;
                        below.push_back(i);
                    }
                }
            std::sort(below.begin(), below.end());
            for (int32_t j = f; j <= l; ++j) P.sn_rows.push_back(j);
            P.sn_rows.insert(P.sn_rows.end(), below.begin(), below.end());
            P.sn_rows_off[s + 1] = (int64_t)P.sn_rows.size();
            if ((int64_t)(l - f + 1) + (int64_t)below.size() != P.colcount[f])
                return bad(P, SSCO_ERR_PATTERN, "internal: supernode structure disagrees with column counts");
        }
    }

    // --- numeric partition: relaxed amalgamation of adjacent child fronts --
    struct FB {
        int32_t f, w, r;
        double zeros;
        int32_t last_sn;
    };
    std::vector<FB> fb;
    for (int32_t s = 0; s < ns; ++s) {
        FB cur{P.snode_first[s], P.snode_first[s + 1] - P.snode_first[s],
               (int32_t)(P.sn_rows_off[s + 1] - P.sn_rows_off[s]), 0.0, s};
        if (P.amalg > 0 && !fb.empty() && P.sn_parent[fb.back().last_sn] == s) {
            const FB& c = fb.back();
            int32_t wm = c.w + cur.w;
            int32_t rm = c.w + cur.r;
            double zeros = c.zeros + (double)c.w * (double)(rm - c.r);
            double entries = (double)wm * rm - (double)wm * (wm - 1) / 2.0;
            double zf = zeros / entries;
            bool ok = wm <= 4 || (wm <= 16 && zf <= 0.8) || (wm <= 48 && zf <= 0.1) || zf <= 0.05;
            if (ok && rm <= 16384) {
                fb.back() = FB{c.f, wm, rm, zeros, s};
                continue;
            }
        }
        fb.push_back(cur);
    }
    int32_t nf = (int32_t)fb.size();
    P.front_first.resize(nf + 1);
    std::vector<int32_t> col2f(n);
    for (int32_t F = 0; F < nf; ++F) {
        P.front_first[F] = fb[F].f;
        for (int32_t j = fb[F].f; j < fb[F].f + fb[F].w; ++j) col2f[j] = F;
    }
    P.front_first[nf] = (int32_t)n;
    P.fronts.assign(nf, FrontDesc{});
    P.rows.clear();
    P.panel_total = P.upd_total = P.pvec_total = 0;
    P.max_rows = 0;
    P.flops_numeric = 0;
    for (int32_t F = 0; F < nf; ++F) {
        FrontDesc& d = P.fronts[F];
        const FB& b = fb[F];
        int32_t s = b.last_sn;
        d.f = b.f;
        d.w = b.w;
        d.r = b.r;
        d.sys = row_sys[b.f];
        d.rows_off = (int64_t)P.rows.size();
        for (int32_t j = b.f; j < P.snode_first[s]; ++j) P.rows.push_back(j);
        P.rows.insert(P.rows.end(), P.sn_rows.begin() + P.sn_rows_off[s], P.sn_rows.begin() + P.sn_rows_off[s + 1]);
        if ((int64_t)P.rows.size() - d.rows_off != d.r)
            return bad(P, SSCO_ERR_PATTERN, "internal: front row count mismatch");
        d.parent = d.r > d.w ? col2f[P.rows[d.rows_off + d.w]] : -1;
        d.panel_off = P.panel_total;
        d.upd_off = P.upd_total;
        d.pvec_off = P.pvec_total;
        P.panel_total += (int64_t)d.r * d.w;
        P.upd_total += (int64_t)(d.r - d.w) * (d.r - d.w);
        P.pvec_total += d.r - d.w;
        P.max_rows = std::max(P.max_rows, d.r);
        for (int32_t k = 0; k < d.w; ++k) P.flops_numeric += (double)(d.r - k) * (d.r - k);
        d.relmap_off = -1;
        d.inv_off = -1;
        d.tc_off = -1;
        d.nchild = 0;
    }
    // children lists (ascending child id)
    {
        std::vector<int32_t> cnt(nf, 0);
        for (int32_t F = 0; F < nf; ++F)
            if (P.fronts[F].parent >= 0) cnt[P.fronts[F].parent]++;
        int32_t off = 0;
        for (int32_t F = 0; F < nf; ++F) {
            P.fronts[F].child_off = off;
            off += cnt[F];
        }
        P.child_ids.assign(off, 0);
        for (int32_t F = 0; F < nf; ++F) {
            int32_t p = P.fronts[F].parent;
            if (p >= 0) P.child_ids[P.fronts[p].child_off + P.fronts[p].nchild++] = F;
        }
    }
    // levels (height) of the numeric forest
    P.front_level.assign(nf, 0);
    for (int32_t F = 0; F < nf; ++F) {
        int32_t p = P.fronts[F].parent;
        if (p >= 0) P.front_level[p] = std::max(P.front_level[p], P.front_level[F] + 1);
    }
    P.n_levels = 0;
    for (int32_t F = 0; F < nf; ++F) P.n_levels = std::max(P.n_levels, P.front_level[F] + 1);
    // relative maps, inverse maps, K lists
    {
        std::vector<int32_t> pos(n, -1);
        P.relmap.clear();
        P.invmap.clear();
        P.klist.clear();
        for (int32_t F = 0; F < nf; ++F) {
            FrontDesc& d = P.fronts[F];
            for (int32_t k = 0; k < d.r; ++k) pos[P.rows[d.rows_off + k]] = k;
            bool big = d.r > P.small_max;
            if (big && d.nchild > 0) {
                d.inv_off = (int64_t)P.invmap.size();
                P.invmap.resize(P.invmap.size() + (size_t)d.nchild * d.r, -1);
            }
            for (int32_t c = 0; c < d.nchild; ++c) {
                FrontDesc& cd = P.fronts[P.child_ids[d.child_off + c]];
                cd.relmap_off = (int64_t)P.relmap.size();
                for (int32_t k = 0; k < cd.r - cd.w; ++k) {
                    int32_t row = P.rows[cd.rows_off + cd.w + k];
                    int32_t pp = pos[row];
                    if (pp < 0) return bad(P, SSCO_ERR_PATTERN, "internal: child row missing in parent front");
                    P.relmap.push_back(pp);
                    if (big) P.invmap[d.inv_off + (int64_t)c * d.r + pp] = k;
                }
            }
            d.klist_off = (int64_t)P.klist.size() / 2;
            for (int32_t j = d.f; j < d.f + d.w; ++j)
                for (int64_t q = P.Kcolptr[j]; q < P.Kcolptr[j + 1]; ++q) {
                    int32_t i = P.Krowind[q];
                    P.klist.push_back(P.kslot_of_q[q]);
                    P.klist.push_back((int32_t)((int64_t)(j - d.f) * d.r + pos[i]));
                }
            d.klist_n = (int32_t)((int64_t)P.klist.size() / 2 - d.klist_off);
            for (int32_t k = 0; k < d.r; ++k) pos[P.rows[d.rows_off + k]] = -1;
        }
    }
    // tiny subtrees: every front of the subtree has at most tiny_max rows;
    // one warp factors / solves a whole subtree, children first.
    std::vector<char> in_tiny(nf, 0);
    std::vector<int32_t> sched(nf, 0);
    int32_t n_sched = 0;
    {
        P.tiny_list.clear();
        P.tiny_off.assign(1, 0);
        if (P.tiny_max > 0) {
            // eligible: the whole subtree has r <= tiny_max and its program
            // (see build_tiny_programs) fits kTinyProgWords / kTinyMaxK
            std::vector<char> ok(nf, 1);
            std::vector<int64_t> words(nf, 0), kents(nf, 0);
            for (int32_t F = 0; F < nf; ++F) {
                const FrontDesc& d = P.fronts[F];
                words[F] += kTinyRecWords + d.nchild + 2 * d.klist_n + 2 * (d.r - d.w);
                kents[F] += d.klist_n;
                if (d.r > P.tiny_max || words[F] + kTinyHdrWords > kTinyProgWords || kents[F] > kTinyMaxK) ok[F] = 0;
                if (d.parent >= 0) {
                    words[d.parent] += words[F];
                    kents[d.parent] += kents[F];
                    if (!ok[F]) ok[d.parent] = 0;
                }
            }
            in_tiny = ok;
            std::vector<int32_t> stack;
            for (int32_t F = 0; F < nf; ++F) {
                int32_t p = P.fronts[F].parent;
                if (!in_tiny[F] || (p >= 0 && in_tiny[p])) continue;
                // postorder of the subtree rooted at F
                stack.assign(1, F);
                std::vector<int32_t> order;
                while (!stack.empty()) {
                    int32_t x = stack.back();
                    stack.pop_back();
                    order.push_back(x);
                    const FrontDesc& d = P.fronts[x];
                    for (int32_t c = 0; c < d.nchild; ++c) stack.push_back(P.child_ids[d.child_off + c]);
                }
                std::reverse(order.begin(), order.end());  // children before parents
                P.tiny_list.insert(P.tiny_list.end(), order.begin(), order.end());
                P.tiny_off.push_back((int32_t)P.tiny_list.size());
            }
        }
        P.n_tiny = (int32_t)P.tiny_off.size() - 1;
        build_tiny_programs(P);
        for (int32_t F = 0; F < nf; ++F) {
            if (in_tiny[F]) continue;
            int32_t p = P.fronts[F].parent;
            n_sched = std::max(n_sched, sched[F] + 1);
            if (p >= 0) sched[p] = std::max(sched[p], sched[F] + 1);
        }
    }
    // launch lists per scheduling level (fronts outside tiny subtrees)
    {
        std::vector<std::vector<int32_t>> by_level(n_sched);
        for (int32_t F = 0; F < nf; ++F)
            if (!in_tiny[F]) by_level[sched[F]].push_back(F);
        P.front_lists.clear();
        P.fact_launches.clear();
        P.solve_launches.clear();
        for (int32_t L = 0; L < n_sched; ++L) {
            const auto& fl = by_level[L];
            // solve: all fronts of the level, largest first
            {
                std::vector<int32_t> srt(fl);
                std::stable_sort(srt.begin(), srt.end(),
                                 [&](int32_t a, int32_t b) { return P.fronts[a].r > P.fronts[b].r; });
                LaunchList ll{};
                ll.level = L;
                ll.cls = 0;
                ll.list_off = (int64_t)P.front_lists.size();
                ll.count = (int32_t)srt.size();
                for (int32_t F : srt) {
                    ll.rmax = std::max(ll.rmax, P.fronts[F].r);
                    ll.wmax = std::max(ll.wmax, P.fronts[F].w);
                }
                P.front_lists.insert(P.front_lists.end(), srt.begin(), srt.end());
                P.solve_launches.push_back(ll);
            }
            // factor: small fronts by size class, then big fronts
            for (int32_t ci = 0; ci < (int32_t)(sizeof(kClasses) / sizeof(kClasses[0])); ++ci) {
                int32_t hi = kClasses[ci];
                int32_t lo = ci == 0 ? 0 : kClasses[ci - 1];
                if (lo >= P.small_max) break;
                hi = std::min(hi, P.small_max);
                LaunchList ll{};
                ll.level = L;
                ll.cls = hi;
                ll.list_off = (int64_t)P.front_lists.size();
                for (int32_t F : fl)
                    if (P.fronts[F].r > lo && P.fronts[F].r <= hi) {
                        P.front_lists.push_back(F);
                        ll.count++;
                        ll.rmax = std::max(ll.rmax, P.fronts[F].r);
                        ll.wmax = std::max(ll.wmax, P.fronts[F].w);
                    }
                if (ll.count > 0) P.fact_launches.push_back(ll);
            }
            LaunchList bl{};
            bl.level = L;
            bl.cls = -1;
            bl.list_off = (int64_t)P.front_lists.size();
            int64_t tc_level = 0;
            for (int32_t F : fl) {
                FrontDesc& d = P.fronts[F];
                if (d.r <= P.small_max) continue;
                if (P.tsize == 4 && P.tune.use_tc) {
                    d.tc_off = tc_level;
                    tc_level += (int64_t)((d.r + 127) / 128) * kTcTileFloats;
                    P.tc_pack_total = std::max(P.tc_pack_total, tc_level);
                }
                P.front_lists.push_back(F);
                bl.count++;
                bl.rmax = std::max(bl.rmax, d.r);
                bl.wmax = std::max(bl.wmax, d.w);
                int64_t t = (d.r + 63) / 64;
                bl.max_lower_tiles = std::max(bl.max_lower_tiles, t * (t + 1) / 2);
                int64_t u = (d.r - d.w + 63) / 64;
                bl.max_syrk_tiles = std::max(bl.max_syrk_tiles, u * (u + 1) / 2);
                bl.max_klist = std::max(bl.max_klist, d.klist_n);
            }
            if (bl.count > 65535)  // the big-front kernels put the level's fronts in grid y
                return bad(P, SSCO_ERR_UNSUPPORTED, "more than 65535 multi-CTA fronts in one level");
            if (bl.count > 0) P.fact_launches.push_back(bl);
        }
    }

    // --- symmetric CSR of K~ for the FP64 residual -------------------------
    {
        P.sp_rowptr.assign(n + 1, 0);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t q = P.Kcolptr[j]; q < P.Kcolptr[j + 1]; ++q) {
                int32_t i = P.Krowind[q];
                P.sp_rowptr[i + 1]++;
                if (i != j) P.sp_rowptr[j + 1]++;
            }
        for (int64_t i = 0; i < n; ++i) P.sp_rowptr[i + 1] += P.sp_rowptr[i];
        P.sp_col.assign(P.sp_rowptr[n], 0);
        P.sp_slot.assign(P.sp_rowptr[n], 0);
        std::vector<int64_t> fill(P.sp_rowptr.begin(), P.sp_rowptr.end() - 1);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t q = P.Kcolptr[j]; q < P.Kcolptr[j + 1]; ++q) {
                int32_t i = P.Krowind[q];
                P.sp_col[fill[i]] = (int32_t)j;
                P.sp_slot[fill[i]++] = P.kslot_of_q[q];
                if (i != j) {
                    P.sp_col[fill[j]] = i;
                    P.sp_slot[fill[j]++] = P.kslot_of_q[q];
                }
            }
        // columns come out ascending within each row: row i first receives
        // (j, .) from every column j < i in order, then its own column i.
        P.row_sys = row_sys;
        P.sys_n_off.resize(n_pats + 1);
        for (int k = 0; k < n_pats; ++k) P.sys_n_off[k] = P.pats[k].n_off;
        P.sys_n_off[n_pats] = n;
        P.shifted.assign(n, 1);
        for (int64_t j = 0; j < n; ++j)
            if (P.pats[row_sys[j]].kind != SSCO_KIND_ATWA && !referenced[j]) P.shifted[j] = 0;
    }

    // --- adjoint tables (original ordering, concatenated) -------------------
    {
        P.g_rowptr.assign(1, 0);
        P.g_colind.clear();
        P.g_aval.clear();
        P.g_row_sys.clear();
        P.g_rows_all.clear();
        P.e_dofs.clear();
        P.e_K0.clear();
        P.e_sys.clear();
        P.e_off.clear();
        P.e_k0off.clear();
        P.e_dim.clear();
        P.e_elems_all.clear();
        P.blk_dofs.clear();
        P.blk_off.clear();
        P.blk_dim.clear();
        P.blk_vbase.clear();
        for (int k = 0; k < n_pats; ++k) {
            const ssco_pattern* p = pats[k];
            const PatMeta& pm = P.pats[k];
            if (p->kind == SSCO_KIND_ATWA) {
                for (int32_t e = 0; e < p->m; ++e) {
                    for (int64_t a = p->rowptr[e]; a < p->rowptr[e + 1]; ++a) {
                        P.g_colind.push_back((int32_t)(pm.n_off + p->colind[a]));
                        P.g_aval.push_back(p->aval[a]);
                    }
                    P.g_rowptr.push_back((int64_t)P.g_colind.size());
                    P.g_row_sys.push_back(k);
                    P.g_rows_all.push_back((int32_t)(pm.m_off + e));
                }
            } else if (p->kind == SSCO_KIND_ELEM_BLOCKS) {
                int32_t d = p->elem_dim;
                int64_t npk = (int64_t)d * (d + 1) / 2;
                for (int32_t e = 0; e < p->m; ++e) {
                    P.blk_off.push_back((int64_t)P.blk_dofs.size());
                    P.blk_dim.push_back(d);
                    P.blk_vbase.push_back((int32_t)(pm.m_off + e * npk));
                    for (int32_t i = 0; i < d; ++i) {
                        int32_t g = p->elem_dofs[(int64_t)e * d + i];
                        P.blk_dofs.push_back(g < 0 ? -1 : (int32_t)(pm.n_off + g));
                    }
                }
            } else {
                int32_t d = p->elem_dim;
                int64_t npk = (int64_t)d * (d + 1) / 2;
                for (int32_t e = 0; e < p->m; ++e) {
                    P.e_off.push_back((int64_t)P.e_dofs.size());
                    P.e_k0off.push_back((int64_t)P.e_K0.size());
                    P.e_dim.push_back(d);
                    P.e_sys.push_back(k);
                    P.e_elems_all.push_back((int32_t)(pm.m_off + e));
                    for (int32_t i = 0; i < d; ++i) {
                        int32_t g = p->elem_dofs[(int64_t)e * d + i];
                        P.e_dofs.push_back(g < 0 ? -1 : (int32_t)(pm.n_off + g));
                    }
                    P.e_K0.insert(P.e_K0.end(), p->elem_K0 + (int64_t)e * npk, p->elem_K0 + (int64_t)(e + 1) * npk);
                }
            }
        }
    }
    build_blob(P);
    compute_ws_layout(P);
    return SSCO_OK;
}

// ---------------------------------------------------------------------------
namespace {
template <class T>
size_t put(std::vector<uint8_t>& blob, const std::vector<T>& v) {
    size_t off = (blob.size() + 255) & ~(size_t)255;
    blob.resize(off + std::max<size_t>(v.size() * sizeof(T), 16), 0);
    if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}
}  // namespace


// Dataflow schedules.  The fronts outside tiny subtrees are handed to
// persistent launches that walk many levels at once: every front is an item
// (per value set, or per group of V value sets) taken in level order by
// whichever warp or CTA is free, and it waits only for its own children (the
// factorization and the forward sweep) or its own parent (the backward
// sweep) through per-item done flags, instead of for a whole level (Sec. 4.3
// groups a level's independent expressions; the flags keep exactly the
// dependencies that grouping respects).
//   factor: fronts with no big (multi-CTA) front below them, in groups by
//     the largest front of their subtree (so a child never sits in a later
//     group than its parent); groups run in increasing size, one launch each.
//   solve:  fronts of at most kFlowSolveRmax rows with no larger front below
//     them, one warp per (front, value set).
// Fronts outside the dataflow keep their per-level launches (fact_rest,
// solve_rest; lists in flow_rest, which starts with a copy of front_lists).
constexpr int32_t kFlowSolveRmax = 256;

void build_flow(Plan& P) {
    const int32_t nf = (int32_t)P.fronts.size();
    std::vector<char> tiny(nf, 0);
    for (int32_t F : P.tiny_list) tiny[F] = 1;
    // height among the fronts outside tiny subtrees; the largest front of
    // each subtree (children precede parents in front order)
    std::vector<int32_t> lvl(nf, 0), sub_r(nf, 0);
    std::vector<char> solve_ok(nf, 1);
    const int32_t srmax = std::min(kFlowSolveRmax, std::max(P.small_max, 32));
    for (int32_t F = 0; F < nf; ++F) {
        const FrontDesc& d = P.fronts[F];
        sub_r[F] = std::max(sub_r[F], d.r);
        if (d.r > srmax) solve_ok[F] = 0;
        const int32_t p = d.parent;
        if (p < 0) continue;
        sub_r[p] = std::max(sub_r[p], sub_r[F]);
        if (!tiny[F]) {
            lvl[p] = std::max(lvl[p], lvl[F] + 1);
            if (!solve_ok[F]) solve_ok[p] = 0;
        }
    }
    std::vector<int32_t> order;
    for (int32_t F = 0; F < nf; ++F)
        if (!tiny[F]) order.push_back(F);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (lvl[a] != lvl[b]) return lvl[a] < lvl[b];
        return P.fronts[a].r > P.fronts[b].r;
    });
    // factor groups by the largest front of the subtree
    const int32_t T = (int32_t)P.tsize;
    struct Cls {
        int32_t hi, V, nw;
    };
    std::vector<Cls> cls;
    if (T == 4)
        cls = {{64, 4, 4}, {128, 2, 8}, {P.small_max, 1, 8}};
    else
        cls = {{64, 2, 4}, {128, 1, 8}, {P.small_max, 1, 8}};
    P.flow_fact.clear();
    P.flow_fslot.assign(nf, -1);
    P.fact_groups.clear();
    int32_t lo = 0;
    for (const Cls& c : cls) {
        const int32_t hi = std::min(c.hi, P.small_max);
        if (hi <= lo) continue;
        FlowGroup g{};
        g.off = (int32_t)P.flow_fact.size();
        g.V = c.V;  // a power of two the kernel is instantiated for, at most the batch
        while (g.V > 1 && g.V > P.B) g.V /= 2;
        g.nw = c.nw;
        for (int32_t F : order)
            if (sub_r[F] > lo && sub_r[F] <= hi) {
                P.flow_fslot[F] = (int32_t)P.flow_fact.size();
                P.flow_fact.push_back(F);
                g.rmax = std::max(g.rmax, P.fronts[F].r);
            }
        g.count = (int32_t)P.flow_fact.size() - g.off;
        if (g.count > 0) P.fact_groups.push_back(g);
        lo = hi;
    }
    P.flow_solve.clear();
    P.flow_sslot.assign(nf, -1);
    P.flow_solve_rmax = 0;
    for (int32_t F : order)
        if (solve_ok[F]) {
            P.flow_sslot[F] = (int32_t)P.flow_solve.size();
            P.flow_solve.push_back(F);
            P.flow_solve_rmax = std::max(P.flow_solve_rmax, P.fronts[F].r);
        }
    // per-level launches of the other fronts (same level lists, filtered)
    P.flow_rest = P.front_lists;
    auto filter = [&](const std::vector<LaunchList>& src, const std::vector<int32_t>& slot,
                      std::vector<LaunchList>& dst) {
        dst.clear();
        for (const LaunchList& ll : src) {
            LaunchList q = ll;
            q.list_off = (int64_t)P.flow_rest.size();
            q.count = 0;
            q.rmax = q.wmax = 0;
            for (int32_t i = 0; i < ll.count; ++i) {
                const int32_t F = P.front_lists[ll.list_off + i];
                if (slot[F] >= 0) continue;
                P.flow_rest.push_back(F);
                q.count++;
                q.rmax = std::max(q.rmax, P.fronts[F].r);
                q.wmax = std::max(q.wmax, P.fronts[F].w);
            }
            if (q.count > 0) dst.push_back(q);
        }
    };
    filter(P.fact_launches, P.flow_fslot, P.fact_rest);
    filter(P.solve_launches, P.flow_sslot, P.solve_rest);
}

void build_blob(Plan& P) {
    std::vector<uint8_t>& b = P.blob;
    b.clear();
    build_flow(P);
    P.toff.fronts = put(b, P.fronts);
    P.toff.rows = put(b, P.rows);
    P.toff.child_ids = put(b, P.child_ids);
    P.toff.relmap = put(b, P.relmap);
    P.toff.invmap = put(b, P.invmap);
    P.toff.klist = put(b, P.klist);
    P.toff.front_lists = put(b, P.front_lists);
    P.toff.groups = put(b, P.groups);
    P.toff.chunks = put(b, P.chunks);
    P.toff.asm_idx = put(b, P.asm_idx);
    P.toff.asm_coef = put(b, P.asm_coef);
    P.toff.sp_rowptr = put(b, P.sp_rowptr);
    P.toff.sp_col = put(b, P.sp_col);
    P.toff.sp_slot = put(b, P.sp_slot);
    P.toff.perm = put(b, P.perm);
    P.toff.row_sys = put(b, P.row_sys);
    P.toff.sys_n_off = put(b, P.sys_n_off);
    P.toff.g_rowptr = put(b, P.g_rowptr);
    P.toff.g_colind = put(b, P.g_colind);
    P.toff.g_aval = put(b, P.g_aval);
    P.toff.g_row_sys = put(b, P.g_row_sys);
    P.toff.e_dofs = put(b, P.e_dofs);
    P.toff.e_K0 = put(b, P.e_K0);
    P.toff.e_sys = put(b, P.e_sys);
    P.toff.e_off = put(b, P.e_off);
    P.toff.e_k0off = put(b, P.e_k0off);
    P.toff.e_dim = put(b, P.e_dim);
    P.toff.shifted = put(b, P.shifted);
    P.toff.g_rows_all = put(b, P.g_rows_all);
    P.toff.e_elems_all = put(b, P.e_elems_all);
    P.toff.tiny_list = put(b, P.tiny_list);
    P.toff.tiny_off = put(b, P.tiny_off);
    P.toff.tiny_prog = put(b, P.tiny_prog);
    P.toff.tiny_prog_off = put(b, P.tiny_prog_off);
    P.toff.blk_dofs = put(b, P.blk_dofs);
    P.toff.blk_off = put(b, P.blk_off);
    P.toff.blk_dim = put(b, P.blk_dim);
    P.toff.blk_vbase = put(b, P.blk_vbase);
    P.toff.flow_fact = put(b, P.flow_fact);
    P.toff.flow_fslot = put(b, P.flow_fslot);
    P.toff.flow_solve = put(b, P.flow_solve);
    P.toff.flow_sslot = put(b, P.flow_sslot);
    P.toff.flow_rest = put(b, P.flow_rest);
    b.resize((b.size() + 255) & ~(size_t)255);
}

void compute_ws_layout(Plan& P) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (std::max<size_t>(bytes, 16) + 255) & ~(size_t)255;
        return o;
    };
    const size_t B = (size_t)P.B, n = (size_t)P.n, S = (size_t)P.B * P.n_pats;
    WsLayout& w = P.ws;
    w.K = take(B * P.nnzK * 8);
    w.panel = take(B * P.panel_total * P.tsize);
    w.upd = take(B * P.upd_total * P.tsize);
    w.pvec = take(B * P.pvec_total * P.tsize);
    w.vecT = take(B * n * P.tsize);
    w.bp = take(B * n * 8);
    w.xp = take(B * n * 8);
    w.rr = take(B * n * 8);
    w.mu = take(B * n * 8);
    w.xbar_p = take(B * n * 8);
    w.bad_col = take(S * 4);
    w.sstatus = take(S * 4);
    w.iters = take(S * 4);
    w.active = take(S * 4);
    w.any_active = take(4);
    w.it_ctr = take(4);
    w.dev_err = take(4);
    w.resid = take(S * 8);
    {
        int64_t longest = 1;
        for (size_t k = 0; k + 1 < P.sys_n_off.size(); ++k)
            longest = std::max<int64_t>(longest, P.sys_n_off[k + 1] - P.sys_n_off[k]);
        w.sys_maxc = (int32_t)((longest + 2047) / 2048);  // chunks of 2048 rows (kSysChunk)
        w.sys_psum = take(S * (size_t)w.sys_maxc * 8);
        w.sys_pmax = take(S * (size_t)w.sys_maxc * 8);
    }
    w.bnorm = take(S * 8);
    w.r1 = take(S * 8);
    w.r2 = take(S * 8);
    w.sigma = take(S * 8);
    w.sbar = take(S * 8);
    w.st_vals = take(B * (size_t)P.m * 8);
    w.st_shift = take(S * 8);
    w.st_b = take(B * n * 8);
    w.st_x = take(B * n * 8);
    w.tcpack = take(B * (size_t)P.tc_pack_total * 4);
    {
        size_t big_count = 0;
        for (const LaunchList& ll : P.fact_launches)
            if (ll.cls < 0) big_count = std::max<size_t>(big_count, (size_t)ll.count);
        w.diag = take(B * big_count * 1024 * P.tsize);
        w.diag_slots = B * big_count;
    }
    w.flow_fact = take(128 + B * P.flow_fact.size() * 4);
    w.flow_solve = take(128 + B * P.flow_solve.size() * 4);
    {
        // GMRES-IR: Krylov basis V (m+1 vectors), preconditioned vectors Z
        // (m), per system the Hessenberg matrix, rotations, right-hand side
        const size_t m = P.refine_mode ? (size_t)P.gmres_m : 0;
        w.gm_V = take(m ? (m + 1) * B * n * 8 : 0);
        w.gm_Z = take(m * B * n * 8);
        w.gm_H = take(m ? S * (m + 1) * m * 8 : 0);
        w.gm_g = take(m ? S * (m + 1) * 8 : 0);
        w.gm_cs = take(S * m * 8);
        w.gm_sn = take(S * m * 8);
        w.gm_hp = take(m ? S * (m + 1) * 8 : 0);
        w.gm_y = take(S * m * 8);
        w.gm_beta = take(m ? S * 8 : 0);
        w.gm_hn = take(m ? S * 8 : 0);
        w.gm_act = take(m ? S * 4 : 0);
        w.gm_k = take(m ? S * 4 : 0);
    }
    w.total = off;
}

void export_L_pattern(const Plan& P, std::vector<int64_t>* colptr, std::vector<int32_t>* rowind) {
    int32_t ns = (int32_t)P.snode_first.size() - 1;
    if (colptr) {
        colptr->assign(P.n + 1, 0);
        for (int64_t j = 0; j < P.n; ++j) (*colptr)[j + 1] = (*colptr)[j] + P.colcount[j];
    }
    if (rowind) {
        rowind->clear();
        rowind->reserve(P.nnzL);
        for (int32_t s = 0; s < ns; ++s) {
            int32_t f = P.snode_first[s], w = P.snode_first[s + 1] - f;
            for (int32_t k = 0; k < w; ++k)
                rowind->insert(rowind->end(), P.sn_rows.begin() + P.sn_rows_off[s] + k,
                               P.sn_rows.begin() + P.sn_rows_off[s + 1]);
        }
    }
}

}  // namespace ssco
