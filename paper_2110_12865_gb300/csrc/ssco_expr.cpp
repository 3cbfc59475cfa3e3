// ssco_expr.cpp -- host compiler of fixed-pattern sparse matrix expressions.
//
// The method of the paper (Sec. 4) applied to sparse algebra: the expression
// DAG is executed once symbolically, entry by entry.  Every entry that needs
// arithmetic (an ADD entry present in both operands, every MUL entry) becomes
// one scalar expression, a sum of products of two slots; structurally equal
// scalar expressions are merged by hashing their canonical form (Sec. 4.2's
// structural hashing; slots are the leaves of Sec. 4.4 and the stored
// intermediates of Sec. 4.2.1); each expression's level is one more than the
// highest level among its factors (the longest path from the leaves, so a
// level never holds an expression together with one it depends on, Sec. 4.3),
// and the level groups are written out as index tables (leaf harvesting,
// Sec. 4.4), slots of one level contiguous (outputs written consecutively,
// Sec. 4.8).  Scaling and transposition only relabel entries.
//
// Optional steps (ssco_expr_opts): algebraic hashing (Sec. 4.1.2, App. A)
// merges expressions equal as polynomials and drops those equal to zero;
// factorization (App. D) takes a slot shared by several products of a sum
// out of them; the global decomposition (Sec. 4.2.1) keeps a linear
// intermediate stored only if it is referenced at least t_ref times and has
// at least t_compl terms, and expands the others into their users.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <fstream>
#include <new>

#include "ssco_expr_internal.h"

namespace ssco {
namespace {

thread_local std::string g_expr_err;

struct Handle {
    double c;   // the entry's value is c * slot s
    int32_t s;
};
struct Term {
    int32_t f1, f2;  // factor slots, f1 >= f2 (slot 0 = the constant one)
    double c;
};

// 64-bit mixing step (the finalizer of splitmix64) folded over the terms
uint64_t mix(uint64_t h, uint64_t x) {
    h ^= x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    h ^= h >> 30;
    h *= 0xbf58476d1ce4e5b9ull;
    h ^= h >> 27;
    h *= 0x94d049bb133111ebull;
    return h ^ (h >> 31);
}

// ---- algebraic keys (Sec. 4.1.2, App. A) ----------------------------------
// A slot's key is the value of its polynomial in the leaf variables at
// kAlgPoints seeded points of the prime field Z_p, p = 2^61 - 1: a leaf
// variable takes a pseudo-random nonzero element per point, the constant one
// takes 1, sums add and products multiply (the paper's rule for + and *).
// A coefficient is a finite double, exactly m 2^e with an integer m; it maps
// to m 2^e mod p, which is exact because 2 is invertible mod p (2^61 = 1), so
// the keys of the stored tables' own coefficients are exact as well.
// Polynomials that are equal get equal keys whatever their structure; two
// different ones of degree d agree at one random point with probability at
// most d / p (Schwartz-Zippel), at all points with its kAlgPoints-th power.
constexpr uint64_t kP = (1ull << 61) - 1;
constexpr int kAlgPoints = 3;

uint64_t fadd(uint64_t a, uint64_t b) {
    const uint64_t s = a + b;
    return s >= kP ? s - kP : s;
}
uint64_t fneg(uint64_t a) { return a ? kP - a : 0; }
uint64_t fmul(uint64_t a, uint64_t b) {  // a, b < p: a b < p^2, and 2^61 = 1 mod p
    const unsigned __int128 z = (unsigned __int128)a * b;
    const uint64_t s = ((uint64_t)z & kP) + (uint64_t)(z >> 61);
    return s >= kP ? s - kP : s;
}
uint64_t finv(uint64_t a) {  // a^(p-2) = 1/a (Fermat), a != 0
    uint64_t r = 1;
    for (uint64_t e = kP - 2; e; e >>= 1) {
        if (e & 1) r = fmul(r, a);
        a = fmul(a, a);
    }
    return r;
}
uint64_t fdyadic(double c) {  // the field image of a finite double
    if (c == 0.0) return 0;
    int e = 0;
    const double f = std::frexp(std::fabs(c), &e);       // |c| = f 2^e, f in [0.5, 1)
    const uint64_t m = (uint64_t)std::ldexp(f, 53);      // exact: < 2^53 < p
    const int k = (((e - 53) % 61) + 61) % 61;           // 2^(e - 53) = 2^k mod p
    const uint64_t r = fmul(m, 1ull << k);
    return c < 0 ? fneg(r) : r;
}
uint64_t splitmix(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}
uint64_t leaf_key(int64_t s, int j) { return 1 + splitmix(0x5a17c0de00000000ull ^ ((uint64_t)s << 2 | (uint64_t)j)) % (kP - 1); }
// a real point as well (values in [0.5, 1.5)), to name the factor between
// two expressions whose keys are proportional
double leaf_real(int64_t s) { return 0.5 + (double)(splitmix(0x7ea1000000000000ull ^ (uint64_t)s) >> 11) * 0x1p-53; }

// The double c with field image r near the real ratio q, if there is one:
// q itself, its neighbours, or q rounded to fewer significant bits (the
// multiples that occur -- 2, -1, 0.5, products of the SCALE factors -- are
// short binary fractions or the doubles the factors multiply to).
bool recover_factor(double q, uint64_t r, double* c) {
    if (!std::isfinite(q) || q == 0.0) return false;
    double x = q;
    for (int k = 0; k < 3; ++k, x = std::nextafter(x, HUGE_VAL))
        if (fdyadic(x) == r) return *c = x, true;
    x = std::nextafter(q, -HUGE_VAL);
    for (int k = 0; k < 2; ++k, x = std::nextafter(x, -HUGE_VAL))
        if (fdyadic(x) == r) return *c = x, true;
    int e = 0;
    const double f = std::frexp(q, &e);
    for (int b = 48; b >= 1; b -= (b > 16 ? 4 : 1)) {
        x = std::ldexp(std::nearbyint(std::ldexp(f, b)), e - b);
        if (x != 0.0 && fdyadic(x) == r) return *c = x, true;
    }
    return false;
}

// Scalar expressions under construction, merged by structural hashing.
struct Builder {
    int64_t base = 0;  // slot id of the first stored expression
    std::vector<int32_t> level, nt;
    std::vector<int64_t> tbeg;
    std::vector<uint64_t> hash;
    std::vector<Term> pool;
    // open addressing: (expression index + 1, high hash bits); index 0 = empty
    std::vector<uint64_t> table;
    static uint64_t slot_of(int64_t i, uint64_t h) { return (uint64_t)(i + 1) | (h & 0xffffffff00000000ull); }
    int64_t n_unrolled = 0;
    bool overflow = false;
    std::vector<Term> t;  // the expression being built

    // optional steps
    bool algebraic = false;   // algebraic hashing
    int32_t factor_min = 0;   // factorization: a slot shared by >= this many products (0 = off)
    int64_t n_alg_merged = 0, n_alg_zero = 0, n_factored = 0;
    // per stored expression: its keys, the inverse of its first key and its
    // value at the real point (algebraic hashing only)
    std::vector<uint64_t> akey, ainv;
    std::vector<double> areal;
    // slots by normalized key (keys 1.. divided by key 0): every slot whose
    // key 0 is nonzero, the constant and the leaves included
    struct AlgEntry {
        uint64_t n1, n2;
        int64_t slot1;  // slot + 1; 0 = empty
    };
    std::vector<AlgEntry> atab;
    int64_t a_count = 0;

    int32_t level_of(int32_t s) const { return s >= base ? level[s - base] : 0; }

    uint64_t key_of(int64_t s, int j) const {
        return s == 0 ? 1 : s < base ? leaf_key(s, j) : akey[(size_t)(s - base) * kAlgPoints + j];
    }
    uint64_t inv_of(int64_t s) const {
        return s == 0 ? 1 : s < base ? finv(leaf_key(s, 0)) : ainv[(size_t)(s - base)];
    }
    double real_of(int64_t s) const { return s == 0 ? 1.0 : s < base ? leaf_real(s) : areal[(size_t)(s - base)]; }

    size_t alg_probe(uint64_t n1, uint64_t n2) const {
        const size_t cap = atab.size();
        size_t p = (size_t)mix(n1, n2) & (cap - 1);
        while (atab[p].slot1 && !(atab[p].n1 == n1 && atab[p].n2 == n2)) p = (p + 1) & (cap - 1);
        return p;
    }
    void alg_insert(int64_t slot, uint64_t n1, uint64_t n2) {
        if (2 * (a_count + 1) > (int64_t)atab.size()) {
            std::vector<AlgEntry> old;
            old.swap(atab);
            atab.assign(std::max<size_t>(1 << 16, old.size() * 2), AlgEntry{0, 0, 0});
            for (const AlgEntry& e : old)
                if (e.slot1) atab[alg_probe(e.n1, e.n2)] = e;
        }
        const size_t p = alg_probe(n1, n2);
        if (atab[p].slot1) return;  // keep the first slot of this key
        atab[p] = AlgEntry{n1, n2, slot + 1};
        ++a_count;
    }
    // the constant one and every leaf, before the first expression
    void alg_start() {
        if (!algebraic) return;
        for (int64_t s = 0; s < base; ++s) {
            const uint64_t i0 = inv_of(s);
            alg_insert(s, fmul(key_of(s, 1), i0), fmul(key_of(s, 2), i0));
        }
    }

    void rehash(size_t cap) {
        table.assign(cap, 0);
        for (size_t i = 0; i < level.size(); ++i) {
            size_t p = hash[i] & (cap - 1);
            while (table[p]) p = (p + 1) & (cap - 1);
            table[p] = slot_of((int64_t)i, hash[i]);
        }
    }

    // Canonical form of the sum in `v` (in place): factor pairs ordered,
    // terms sorted, equal pairs merged, zero terms dropped.  Returns the
    // handle when no expression is needed (a constant multiple of one slot,
    // or zero); otherwise {0, -1} with the form's hash in *h.
    static Handle canon(std::vector<Term>& v, uint64_t* h) {
        for (Term& x : v)
            if (x.f1 < x.f2) std::swap(x.f1, x.f2);
        if (v.size() > 1) {
            std::sort(v.begin(), v.end(), [](const Term& a, const Term& b) {
                return a.f1 != b.f1 ? a.f1 < b.f1 : a.f2 < b.f2;
            });
            size_t w = 0;
            for (size_t r = 0; r < v.size(); ++r) {
                if (w > 0 && v[w - 1].f1 == v[r].f1 && v[w - 1].f2 == v[r].f2)
                    v[w - 1].c += v[r].c;  // equal factor pairs: one product
                else
                    v[w++] = v[r];
            }
            v.resize(w);
        }
        v.erase(std::remove_if(v.begin(), v.end(), [](const Term& x) { return x.c == 0.0; }), v.end());
        if (v.empty()) return {0.0, 0};
        if (v.size() == 1 && v[0].f2 == 0) return {v[0].c, v[0].f1};
        uint64_t hh = 0;
        for (const Term& x : v) {
            uint64_t cb;
            std::memcpy(&cb, &x.c, 8);
            hh = mix(mix(hh, ((uint64_t)(uint32_t)x.f1 << 32) | (uint32_t)x.f2), cb);
        }
        *h = hh;
        return {0.0, -1};
    }

    void prefetch(uint64_t h) const {
        if (!table.empty()) __builtin_prefetch(&table[h & (table.size() - 1)]);
    }

    // The stored expression with canonical terms tt[0..n) and hash h: an
    // equal earlier one, or a new one.
    Handle lookup_insert(const Term* tt, size_t n, uint64_t h) {
        if (table.empty()) rehash(1 << 16);
        size_t cap = table.size(), p = h & (cap - 1);
        while (table[p]) {
            const int32_t i = (int32_t)(table[p] & 0xffffffffull) - 1;
            if ((table[p] >> 32) == (h >> 32) && hash[i] == h && nt[i] == (int32_t)n) {
                const Term* q = pool.data() + tbeg[i];
                bool same = true;
                for (size_t k = 0; k < n && same; ++k)
                    same = q[k].f1 == tt[k].f1 && q[k].f2 == tt[k].f2 && q[k].c == tt[k].c;
                if (same) return {1.0, (int32_t)(base + i)};
            }
            p = (p + 1) & (cap - 1);
        }
        // algebraic hashing: an expression equal to zero needs no slot; one
        // equal to c times an existing slot reuses it
        uint64_t k[kAlgPoints] = {0, 0, 0}, n1 = 0, n2 = 0, i0 = 0;
        double real = 0.0;
        if (algebraic) {
            for (size_t q = 0; q < n; ++q) {
                const uint64_t c = fdyadic(tt[q].c);
                for (int j = 0; j < kAlgPoints; ++j)
                    k[j] = fadd(k[j], fmul(c, fmul(key_of(tt[q].f1, j), key_of(tt[q].f2, j))));
                real += tt[q].c * real_of(tt[q].f1) * real_of(tt[q].f2);
            }
            if (k[0] == 0 && k[1] == 0 && k[2] == 0) {
                ++n_alg_zero;
                return {0.0, 0};
            }
            if (k[0] != 0) {
                i0 = finv(k[0]);
                n1 = fmul(k[1], i0);
                n2 = fmul(k[2], i0);
                const AlgEntry& e = atab[alg_probe(n1, n2)];
                double c = 0.0;
                if (e.slot1) {
                    const int64_t s = e.slot1 - 1;
                    if (recover_factor(real / real_of(s), fmul(k[0], inv_of(s)), &c)) {
                        ++n_alg_merged;
                        return {c, (int32_t)s};
                    }
                }
            }
        }
        const int64_t idx = (int64_t)level.size();
        if (base + idx >= (int64_t)INT32_MAX - 1) {
            overflow = true;
            return {0.0, 0};
        }
        if (algebraic) {
            akey.insert(akey.end(), k, k + kAlgPoints);
            ainv.push_back(i0);
            areal.push_back(real);
            if (k[0] != 0) alg_insert(base + idx, n1, n2);
        }
        int32_t lv = 0;
        for (size_t k = 0; k < n; ++k) lv = std::max(lv, std::max(level_of(tt[k].f1), level_of(tt[k].f2)));
        level.push_back(lv + 1);
        nt.push_back((int32_t)n);
        tbeg.push_back((int64_t)pool.size());
        hash.push_back(h);
        pool.insert(pool.end(), tt, tt + n);
        table[p] = slot_of(idx, h);
        if (2 * level.size() > cap) rehash(cap * 2);
        return {1.0, (int32_t)(base + idx)};
    }

    // Factorization (App. D) of the canonical sum v, in place: while some
    // slot is a factor of at least factor_min of its products, the slot
    // shared by the most (the smallest on ties) is taken out -- its
    // partners' sum becomes a linear expression of its own (merged by
    // hashing like any other) and those products become one.  A linear sum
    // has distinct slots, so the partners' sum is never factored again.
    bool factor(std::vector<Term>& v) {
        bool any = false;
        std::vector<int32_t> fs;
        std::vector<Term> inner, rest;
        for (;;) {
            fs.clear();
            for (const Term& x : v) {
                if (x.f1 > 0) fs.push_back(x.f1);
                if (x.f2 > 0 && x.f2 != x.f1) fs.push_back(x.f2);
            }
            std::sort(fs.begin(), fs.end());
            int32_t best = -1;
            size_t most = 0;
            for (size_t i = 0; i < fs.size();) {
                size_t j = i;
                while (j < fs.size() && fs[j] == fs[i]) ++j;
                if (j - i > most) most = j - i, best = fs[i];
                i = j;
            }
            if (most < 2 || (int64_t)most < factor_min) return any;
            inner.clear();
            rest.clear();
            for (const Term& x : v) {
                if (x.f1 == best || x.f2 == best)
                    inner.push_back(Term{x.f1 == best ? x.f2 : x.f1, 0, x.c});
                else
                    rest.push_back(x);
            }
            const Handle h = materialize_vec(inner);
            if (h.c != 0.0) rest.push_back(Term{best, h.s, h.c});
            v.swap(rest);
            ++n_factored;
            any = true;
        }
    }

    // The sum of the terms in v (reordered in place), as a handle: a
    // constant multiple of one slot needs no expression; anything else is
    // stored once.
    Handle materialize_vec(std::vector<Term>& v) {
        ++n_unrolled;
        uint64_t h = 0;
        Handle d = canon(v, &h);
        if (d.s < 0 && factor_min > 0 && factor(v)) d = canon(v, &h);
        return d.s >= 0 ? d : lookup_insert(v.data(), v.size(), h);
    }
    Handle materialize() { return materialize_vec(t); }

    // materialize() for a batch of sums (the entries of one row of a
    // product): all canonical forms first, their table slots prefetched,
    // then the lookups, so that the table's cache misses overlap.
    std::vector<Term> bt;
    std::vector<size_t> boff;
    std::vector<uint64_t> bh;
    std::vector<Handle> direct;
    void materialize_batch(const std::vector<Term>& terms, const std::vector<int64_t>& off, size_t count,
                           std::vector<Handle>& out) {
        if (factor_min > 0) {  // factored one at a time
            for (size_t x = 0; x < count; ++x) {
                t.assign(terms.begin() + off[x], terms.begin() + off[x + 1]);
                out.push_back(materialize());
            }
            return;
        }
        bt.clear();
        boff.assign(1, 0);
        bh.resize(count);
        direct.resize(count);
        for (size_t x = 0; x < count; ++x) {
            t.assign(terms.begin() + off[x], terms.begin() + off[x + 1]);
            direct[x] = canon(t, &bh[x]);
            if (direct[x].s < 0) {
                bt.insert(bt.end(), t.begin(), t.end());
                prefetch(bh[x]);
            }
            boff.push_back(bt.size());
        }
        n_unrolled += (int64_t)count;
        for (size_t x = 0; x < count; ++x)
            out.push_back(direct[x].s >= 0 ? direct[x] : lookup_insert(bt.data() + boff[x], boff[x + 1] - boff[x], bh[x]));
    }
};

ssco_status bad(ssco_status s, const std::string& msg) {
    g_expr_err = msg;
    return s;
}

ssco_status validate(const ssco_expr_node* nodes, int32_t n_nodes, const int32_t* outputs, int32_t n_out,
                     int32_t batch, int32_t precision, std::vector<int32_t>& rows, std::vector<int32_t>& cols) {
    if (!nodes || n_nodes < 1 || !outputs || n_out < 1) return bad(SSCO_ERR_INVALID_ARG, "no nodes or no outputs");
    if (batch < 1 || batch > 65535) return bad(SSCO_ERR_INVALID_ARG, "batch must be in [1, 65535]");
    if (precision != SSCO_VALS_F64 && precision != SSCO_VALS_F32)
        return bad(SSCO_ERR_INVALID_ARG, "precision must be SSCO_VALS_F64 or SSCO_VALS_F32");
    rows.assign(n_nodes, 0);
    cols.assign(n_nodes, 0);
    int64_t leaf_vals = 0;
    for (int32_t i = 0; i < n_nodes; ++i) {
        const ssco_expr_node& nd = nodes[i];
        const std::string pre = "node " + std::to_string(i) + ": ";
        auto operand = [&](int32_t a) { return a >= 0 && a < i; };
        switch (nd.op) {
            case SSCO_EXPR_LEAF: {
                if (nd.rows < 0 || nd.cols < 0) return bad(SSCO_ERR_INVALID_ARG, pre + "negative shape");
                if (!nd.rowptr) return bad(SSCO_ERR_INVALID_ARG, pre + "rowptr is NULL");
                if (nd.rowptr[0] != 0) return bad(SSCO_ERR_PATTERN, pre + "rowptr[0] != 0");
                for (int32_t r = 0; r < nd.rows; ++r)
                    if (nd.rowptr[r + 1] < nd.rowptr[r]) return bad(SSCO_ERR_PATTERN, pre + "rowptr decreases");
                const int64_t nnz = nd.rowptr[nd.rows];
                if (nnz > 0 && !nd.colind) return bad(SSCO_ERR_INVALID_ARG, pre + "colind is NULL");
                if (nd.vmap) {
                    if (nd.n_vals < 0) return bad(SSCO_ERR_INVALID_ARG, pre + "negative n_vals");
                    for (int64_t q = 0; q < nnz; ++q)
                        if (nd.vmap[q] < 0 || nd.vmap[q] >= nd.n_vals)
                            return bad(SSCO_ERR_PATTERN, pre + "vmap entry out of range");
                }
                for (int32_t r = 0; r < nd.rows; ++r)
                    for (int64_t q = nd.rowptr[r]; q < nd.rowptr[r + 1]; ++q) {
                        if (nd.colind[q] < 0 || nd.colind[q] >= nd.cols)
                            return bad(SSCO_ERR_PATTERN, pre + "column index out of range");
                        if (q > nd.rowptr[r] && nd.colind[q] <= nd.colind[q - 1])
                            return bad(SSCO_ERR_PATTERN, pre + "columns not strictly increasing in a row");
                    }
                leaf_vals += nd.vmap ? nd.n_vals : nnz;
                rows[i] = nd.rows;
                cols[i] = nd.cols;
                break;
            }
            case SSCO_EXPR_ADD:
                if (!operand(nd.a) || !operand(nd.b)) return bad(SSCO_ERR_INVALID_ARG, pre + "bad operand");
                if (rows[nd.a] != rows[nd.b] || cols[nd.a] != cols[nd.b])
                    return bad(SSCO_ERR_INVALID_ARG, pre + "ADD of different shapes");
                rows[i] = rows[nd.a];
                cols[i] = cols[nd.a];
                break;
            case SSCO_EXPR_SCALE:
                if (!operand(nd.a)) return bad(SSCO_ERR_INVALID_ARG, pre + "bad operand");
                if (!std::isfinite(nd.alpha)) return bad(SSCO_ERR_NONFINITE, pre + "non-finite alpha");
                rows[i] = rows[nd.a];
                cols[i] = cols[nd.a];
                break;
            case SSCO_EXPR_MUL:
                if (!operand(nd.a) || !operand(nd.b)) return bad(SSCO_ERR_INVALID_ARG, pre + "bad operand");
                if (cols[nd.a] != rows[nd.b]) return bad(SSCO_ERR_INVALID_ARG, pre + "MUL of incompatible shapes");
                rows[i] = rows[nd.a];
                cols[i] = cols[nd.b];
                break;
            case SSCO_EXPR_TRANSPOSE:
                if (!operand(nd.a)) return bad(SSCO_ERR_INVALID_ARG, pre + "bad operand");
                rows[i] = cols[nd.a];
                cols[i] = rows[nd.a];
                break;
            default:
                return bad(SSCO_ERR_INVALID_ARG, pre + "unknown op");
        }
    }
    for (int32_t k = 0; k < n_out; ++k)
        if (outputs[k] < 0 || outputs[k] >= n_nodes) return bad(SSCO_ERR_INVALID_ARG, "output id out of range");
    if (leaf_vals + 1 >= (int64_t)INT32_MAX) return bad(SSCO_ERR_UNSUPPORTED, "leaf values exceed int32 slots");
    return SSCO_OK;
}

// Global decomposition (Sec. 4.2.1) of the expressions in bd into nb.
// Reference counts are taken over the stored expressions' products and the
// outputs.  A linear expression (every product has the constant one as a
// factor) that is no output and is referenced fewer than t_ref times or has
// fewer than t_compl terms (its complexity: one multiply-add per term) is
// not stored: its terms are substituted into every product that uses it.  A
// product is never substituted (its users' terms would get three factors).
// The expressions that stay are rebuilt in level order, so that hashing
// merges what the substitution made equal.
void decompose(Builder& bd, std::vector<std::vector<Handle>>& outh, int32_t t_ref, int32_t t_compl, Builder& nb,
               int64_t* n_inlined) {
    const int64_t n = (int64_t)bd.level.size(), base = bd.base;
    std::vector<int32_t> refs(n, 0);
    std::vector<uint8_t> keep(n, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t q = bd.tbeg[i]; q < bd.tbeg[i] + bd.nt[i]; ++q) {
            if (bd.pool[q].f1 >= base) ++refs[bd.pool[q].f1 - base];
            if (bd.pool[q].f2 >= base) ++refs[bd.pool[q].f2 - base];
        }
    for (const auto& o : outh)
        for (const Handle& h : o)
            if (h.s >= base) keep[h.s - base] = 1;
    for (int64_t i = 0; i < n; ++i) {
        bool linear = true;
        for (int64_t q = bd.tbeg[i]; q < bd.tbeg[i] + bd.nt[i] && linear; ++q) linear = bd.pool[q].f2 == 0;
        if (!linear || (refs[i] >= t_ref && bd.nt[i] >= t_compl)) keep[i] = 1;
    }
    std::vector<int32_t>().swap(refs);
    // level order (operands first)
    int32_t max_lv = 0;
    for (int64_t i = 0; i < n; ++i) max_lv = std::max(max_lv, bd.level[i]);
    std::vector<int64_t> cnt((size_t)max_lv + 2, 0);
    std::vector<int64_t> order(n);
    for (int64_t i = 0; i < n; ++i) cnt[bd.level[i] + 1]++;
    for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
    for (int64_t i = 0; i < n; ++i) order[cnt[bd.level[i]]++] = i;
    // each old expression as a list of new handles (one, or an inlined sum)
    std::vector<int64_t> mbeg(n, 0), mlen(n, 0);
    std::vector<Handle> mpool;
    std::vector<Handle> lin;
    auto sub = [&](int32_t s, const Handle** b, int64_t* len, Handle* own) {
        if (s < base) {
            *own = Handle{1.0, s};
            *b = own;
            *len = 1;
        } else {
            *b = mpool.data() + mbeg[s - base];
            *len = mlen[s - base];
        }
    };
    for (int64_t i : order) {
        nb.t.clear();
        for (int64_t q = bd.tbeg[i]; q < bd.tbeg[i] + bd.nt[i]; ++q) {
            const Term x = bd.pool[q];
            const Handle *A, *B;
            int64_t na, nbb;
            Handle oa, ob;
            sub(x.f1, &A, &na, &oa);
            sub(x.f2, &B, &nbb, &ob);
            for (int64_t u = 0; u < na; ++u)
                for (int64_t v = 0; v < nbb; ++v) nb.t.push_back(Term{A[u].s, B[v].s, x.c * A[u].c * B[v].c});
        }
        mbeg[i] = (int64_t)mpool.size();
        if (keep[i]) {
            mpool.push_back(nb.materialize());
        } else {  // linear: every product is (slot, the constant one)
            lin.clear();
            for (const Term& x : nb.t) lin.push_back(Handle{x.c, x.f1 ? x.f1 : x.f2});
            std::sort(lin.begin(), lin.end(), [](const Handle& a, const Handle& b) { return a.s < b.s; });
            size_t w = 0;
            for (size_t r = 0; r < lin.size(); ++r) {
                if (w > 0 && lin[w - 1].s == lin[r].s)
                    lin[w - 1].c += lin[r].c;
                else
                    lin[w++] = lin[r];
            }
            lin.resize(w);
            lin.erase(std::remove_if(lin.begin(), lin.end(), [](const Handle& h) { return h.c == 0.0; }), lin.end());
            mpool.insert(mpool.end(), lin.begin(), lin.end());
            ++*n_inlined;
        }
        mlen[i] = (int64_t)mpool.size() - mbeg[i];
    }
    for (auto& o : outh)
        for (Handle& h : o)
            if (h.s >= base) {  // kept: one handle (none if it vanished)
                const int64_t i = h.s - base;
                h = mlen[i] ? Handle{h.c * mpool[mbeg[i]].c, mpool[mbeg[i]].s} : Handle{0.0, 0};
            }
    nb.n_unrolled = bd.n_unrolled;
}

ssco_status compile(const ssco_expr_node* nodes, int32_t n_nodes, const int32_t* outputs, int32_t n_out,
                    const ssco_expr_opts& opt, ExprProgram& E) {
    const int32_t batch = opt.batch, precision = opt.precision, inline_terms = opt.inline_terms;
    std::vector<int32_t> rows, cols;
    ssco_status st = validate(nodes, n_nodes, outputs, n_out, batch, precision, rows, cols);
    if (st != SSCO_OK) return st;
    if (inline_terms < 0 || inline_terms > 16) return bad(SSCO_ERR_INVALID_ARG, "inline_terms must be in [0, 16]");
    if (opt.algebraic < 0 || opt.algebraic > 1) return bad(SSCO_ERR_INVALID_ARG, "algebraic must be 0 or 1");
    if (opt.factor_min < 0 || opt.factor_min == 1) return bad(SSCO_ERR_INVALID_ARG, "factor_min must be 0 or >= 2");
    if (opt.t_ref < 0 || opt.t_compl < 0) return bad(SSCO_ERR_INVALID_ARG, "t_ref and t_compl must be >= 0");
    if (opt.reserved != 0) return bad(SSCO_ERR_INVALID_ARG, "reserved option must be 0");
    E.B = batch;
    E.precision = precision;
    // last use of every node, so that its entries can be released
    std::vector<int32_t> last(n_nodes, -1);
    for (int32_t i = 0; i < n_nodes; ++i) {
        if (nodes[i].op != SSCO_EXPR_LEAF) last[nodes[i].a] = i;
        if (nodes[i].op == SSCO_EXPR_ADD || nodes[i].op == SSCO_EXPR_MUL) last[nodes[i].b] = i;
    }
    for (int32_t k = 0; k < n_out; ++k) last[outputs[k]] = n_nodes;
    auto leaf_count = [&](const ssco_expr_node& nd) { return nd.vmap ? nd.n_vals : nd.rowptr[nd.rows]; };
    int64_t leaf_vals = 0;
    for (int32_t i = 0; i < n_nodes; ++i)
        if (nodes[i].op == SSCO_EXPR_LEAF) leaf_vals += leaf_count(nodes[i]);
    E.n_leaf_vals = leaf_vals;
    Builder bd;
    bd.base = 1 + leaf_vals;
    bd.algebraic = opt.algebraic != 0;
    bd.factor_min = opt.factor_min;
    bd.alg_start();
    std::vector<ExprCsr> pat(n_nodes);
    // Every entry of a node is a short linear combination of slots: one
    // handle, or, with inlining, up to `inline_terms` handles kept local
    // (not stored) and expanded into the products that use them.
    struct Entries {
        std::vector<int64_t> off{0};
        std::vector<Handle> h;
        void push(const Handle* b, const Handle* e) {
            h.insert(h.end(), b, e);
            off.push_back((int64_t)h.size());
        }
        void push1(Handle x) {
            h.push_back(x);
            off.push_back((int64_t)h.size());
        }
        int64_t n(int64_t e) const { return off[e + 1] - off[e]; }
        const Handle* at(int64_t e) const { return h.data() + off[e]; }
    };
    std::vector<Entries> ev(n_nodes);
    std::vector<Handle> lin;
    // canonical local combination: equal slots merged, zero coefficients dropped
    auto canon_lin = [](std::vector<Handle>& v) {
        std::sort(v.begin(), v.end(), [](const Handle& a, const Handle& b) { return a.s < b.s; });
        size_t w = 0;
        for (size_t r = 0; r < v.size(); ++r) {
            if (w > 0 && v[w - 1].s == v[r].s)
                v[w - 1].c += v[r].c;
            else
                v[w++] = v[r];
        }
        v.resize(w);
        v.erase(std::remove_if(v.begin(), v.end(), [](const Handle& x) { return x.c == 0.0; }), v.end());
    };
    // a combination as one handle: stored unless it is a multiple of one slot
    auto store_lin = [&](const Handle* b, int64_t n) {
        bd.t.clear();
        for (int64_t k = 0; k < n; ++k) bd.t.push_back(Term{b[k].s, 0, b[k].c});
        return bd.materialize();
    };
    std::vector<int32_t> mark, cnt;
    int64_t leaf_off = 0;
    for (int32_t i = 0; i < n_nodes; ++i) {
        const ssco_expr_node& nd = nodes[i];
        ExprCsr& P = pat[i];
        Entries& H = ev[i];
        P.rows = rows[i];
        P.cols = cols[i];
        if (nd.op == SSCO_EXPR_LEAF) {
            const int64_t nnz = nd.rowptr[nd.rows];
            P.rp.assign(nd.rowptr, nd.rowptr + nd.rows + 1);
            P.ci.assign(nd.colind, nd.colind + nnz);
            for (int64_t q = 0; q < nnz; ++q) H.push1({1.0, (int32_t)(1 + leaf_off + (nd.vmap ? nd.vmap[q] : q))});
            leaf_off += leaf_count(nd);
        } else if (nd.op == SSCO_EXPR_SCALE) {
            P.rp = pat[nd.a].rp;
            P.ci = pat[nd.a].ci;
            H = ev[nd.a];
            for (Handle& h : H.h) h.c *= nd.alpha;
        } else if (nd.op == SSCO_EXPR_TRANSPOSE) {
            const ExprCsr& A = pat[nd.a];
            const Entries& HA = ev[nd.a];
            P.rp.assign(P.rows + 1, 0);
            for (int32_t c : A.ci) P.rp[c + 1]++;
            for (int32_t r = 0; r < P.rows; ++r) P.rp[r + 1] += P.rp[r];
            P.ci.resize(A.ci.size());
            std::vector<int64_t> src(A.ci.size()), fill(P.rp.begin(), P.rp.end() - 1);
            for (int32_t r = 0; r < A.rows; ++r)
                for (int64_t q = A.rp[r]; q < A.rp[r + 1]; ++q) {
                    const int64_t p = fill[A.ci[q]]++;
                    P.ci[p] = r;
                    src[p] = q;
                }
            for (int64_t p = 0; p < (int64_t)src.size(); ++p) H.push(HA.at(src[p]), HA.at(src[p]) + HA.n(src[p]));
        } else if (nd.op == SSCO_EXPR_ADD) {
            const ExprCsr &A = pat[nd.a], &Bm = pat[nd.b];
            const Entries &HA = ev[nd.a], &HB = ev[nd.b];
            P.rp.assign(1, 0);
            for (int32_t r = 0; r < P.rows; ++r) {
                int64_t p = A.rp[r], q = Bm.rp[r];
                while (p < A.rp[r + 1] || q < Bm.rp[r + 1]) {
                    const int32_t ca = p < A.rp[r + 1] ? A.ci[p] : INT32_MAX;
                    const int32_t cb = q < Bm.rp[r + 1] ? Bm.ci[q] : INT32_MAX;
                    if (ca == cb) {
                        lin.assign(HA.at(p), HA.at(p) + HA.n(p));
                        lin.insert(lin.end(), HB.at(q), HB.at(q) + HB.n(q));
                        if (inline_terms > 0) canon_lin(lin);
                        if (inline_terms > 0 && (int64_t)lin.size() <= inline_terms)
                            H.push(lin.data(), lin.data() + lin.size());   // kept local
                        else
                            H.push1(store_lin(lin.data(), (int64_t)lin.size()));
                        P.ci.push_back(ca);
                        ++p, ++q;
                    } else if (ca < cb) {
                        H.push(HA.at(p), HA.at(p) + HA.n(p));
                        P.ci.push_back(ca);
                        ++p;
                    } else {
                        H.push(HB.at(q), HB.at(q) + HB.n(q));
                        P.ci.push_back(cb);
                        ++q;
                    }
                }
                P.rp.push_back((int64_t)P.ci.size());
            }
        } else {  // MUL: entry (r, j) = sum over k of A(r, k) B(k, j), local sums expanded
            const ExprCsr &A = pat[nd.a], &Bm = pat[nd.b];
            const Entries &HA = ev[nd.a], &HB = ev[nd.b];
            mark.assign(P.cols, -1);
            cnt.assign(P.cols, 0);
            std::vector<int32_t> jl;
            std::vector<int64_t> off;
            std::vector<Term> terms;
            std::vector<Handle> row;
            P.rp.assign(1, 0);
            for (int32_t r = 0; r < P.rows; ++r) {
                jl.clear();
                for (int64_t p = A.rp[r]; p < A.rp[r + 1]; ++p) {
                    const int32_t k = A.ci[p];
                    for (int64_t q = Bm.rp[k]; q < Bm.rp[k + 1]; ++q) {
                        const int32_t j = Bm.ci[q];
                        if (mark[j] != r) {
                            mark[j] = r;
                            cnt[j] = 0;
                            jl.push_back(j);
                        }
                        cnt[j] += (int32_t)(HA.n(p) * HB.n(q));
                    }
                }
                std::sort(jl.begin(), jl.end());
                off.assign(jl.size() + 1, 0);
                for (size_t x = 0; x < jl.size(); ++x) {
                    off[x + 1] = off[x] + cnt[jl[x]];
                    cnt[jl[x]] = (int32_t)x;  // now: the column's position in jl
                }
                terms.resize(off.back());
                std::vector<int64_t> fill(off.begin(), off.end() - 1);
                for (int64_t p = A.rp[r]; p < A.rp[r + 1]; ++p) {
                    const int32_t k = A.ci[p];
                    for (int64_t q = Bm.rp[k]; q < Bm.rp[k + 1]; ++q) {
                        int64_t& f = fill[cnt[Bm.ci[q]]];
                        for (const Handle *a = HA.at(p), *ae = a + HA.n(p); a < ae; ++a)
                            for (const Handle *b = HB.at(q), *be = b + HB.n(q); b < be; ++b)
                                terms[f++] = Term{a->s, b->s, a->c * b->c};
                    }
                }
                row.clear();
                bd.materialize_batch(terms, off, jl.size(), row);
                for (const Handle& h : row) H.push1(h);
                P.ci.insert(P.ci.end(), jl.begin(), jl.end());
                P.rp.push_back((int64_t)P.ci.size());
            }
        }
        if (bd.overflow) return bad(SSCO_ERR_UNSUPPORTED, "stored intermediates exceed int32 slots");
        // release the entries of operands used for the last time
        const int32_t ops[2] = {nd.op == SSCO_EXPR_LEAF ? -1 : nd.a,
                                (nd.op == SSCO_EXPR_ADD || nd.op == SSCO_EXPR_MUL) ? nd.b : -1};
        for (int32_t o : ops)
            if (o >= 0 && last[o] == i) {
                Entries().h.swap(ev[o].h);
                std::vector<int64_t>{0}.swap(ev[o].off);
                std::vector<int64_t>().swap(pat[o].rp);
                std::vector<int32_t>().swap(pat[o].ci);
            }
    }
    // outputs: every entry as one handle (local combinations stored now)
    std::vector<std::vector<Handle>> outh(n_out);
    for (int32_t k = 0; k < n_out; ++k) {
        const Entries& H = ev[outputs[k]];
        for (int64_t e = 0; e + 1 < (int64_t)H.off.size(); ++e)
            outh[k].push_back(H.n(e) == 1 ? *H.at(e) : store_lin(H.at(e), H.n(e)));
    }
    if (bd.overflow) return bad(SSCO_ERR_UNSUPPORTED, "stored intermediates exceed int32 slots");
    int64_t n_inlined = 0;
    if (opt.t_ref > 0 || opt.t_compl > 0) {
        Builder nb;
        nb.base = bd.base;
        nb.algebraic = bd.algebraic;
        nb.factor_min = bd.factor_min;
        nb.alg_start();
        decompose(bd, outh, opt.t_ref, opt.t_compl, nb, &n_inlined);
        nb.n_alg_merged += bd.n_alg_merged;
        nb.n_alg_zero += bd.n_alg_zero;
        nb.n_factored += bd.n_factored;
        bd = std::move(nb);
        if (bd.overflow) return bad(SSCO_ERR_UNSUPPORTED, "stored intermediates exceed int32 slots");
    }
    E.n_alg_merged = bd.n_alg_merged;
    E.n_alg_zero = bd.n_alg_zero;
    E.n_factored = bd.n_factored;
    E.n_inlined = n_inlined;
    // level order: by level, then term count, then creation (two stable
    // counting passes: term count, then level)
    const int64_t n_ops = (int64_t)bd.level.size();
    std::vector<int32_t> order(n_ops), rank(n_ops), tmp(n_ops);
    {
        int32_t max_nt = 0, max_lv = 0;
        for (int64_t i = 0; i < n_ops; ++i) {
            max_nt = std::max(max_nt, bd.nt[i]);
            max_lv = std::max(max_lv, bd.level[i]);
        }
        std::vector<int64_t> cnt((size_t)std::max(max_nt, max_lv) + 2, 0);
        for (int64_t i = 0; i < n_ops; ++i) cnt[bd.nt[i] + 1]++;
        for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
        for (int64_t i = 0; i < n_ops; ++i) tmp[cnt[bd.nt[i]]++] = (int32_t)i;
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int64_t i = 0; i < n_ops; ++i) cnt[bd.level[i] + 1]++;
        for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
        for (int64_t r = 0; r < n_ops; ++r) order[cnt[bd.level[tmp[r]]]++] = tmp[r];
    }
    std::vector<int32_t>().swap(tmp);
    for (int64_t r = 0; r < n_ops; ++r) rank[order[r]] = (int32_t)r;
    const int64_t base = bd.base;
    auto remap = [&](int32_t s) { return s >= base ? (int32_t)(base + rank[s - base]) : s; };
    const int32_t max_level = n_ops ? bd.level[order[n_ops - 1]] : 0;
    E.lvl_begin.assign(max_level + 1, 0);
    for (int64_t r = 0; r < n_ops; ++r) E.lvl_begin[bd.level[order[r]]] = r + 1;
    for (int32_t l = 1; l <= max_level; ++l) E.lvl_begin[l] = std::max(E.lvl_begin[l], E.lvl_begin[l - 1]);
    E.term_off.assign(n_ops + 1, 0);
    E.f1.resize(bd.pool.size());
    E.f2.resize(bd.pool.size());
    E.coef.resize(bd.pool.size());
    std::vector<Term> tt;
    for (int64_t r = 0; r < n_ops; ++r) {
        const int32_t i = order[r];
        tt.assign(bd.pool.begin() + bd.tbeg[i], bd.pool.begin() + bd.tbeg[i] + bd.nt[i]);
        for (Term& x : tt) {
            x.f1 = remap(x.f1);
            x.f2 = remap(x.f2);
            if (x.f1 < x.f2) std::swap(x.f1, x.f2);
        }
        std::sort(tt.begin(), tt.end(), [](const Term& a, const Term& b) {
            return a.f1 != b.f1 ? a.f1 < b.f1 : a.f2 < b.f2;
        });
        const int64_t o = E.term_off[r];
        for (size_t k = 0; k < tt.size(); ++k) {
            E.f1[o + k] = tt[k].f1;
            E.f2[o + k] = tt[k].f2;
            E.coef[o + k] = tt[k].c;
        }
        E.term_off[r + 1] = o + (int64_t)tt.size();
    }
    E.n_ops = n_ops;
    E.n_terms = (int64_t)bd.pool.size();
    E.n_slots = base + n_ops;
    E.n_unrolled = bd.n_unrolled;
    E.unit_coef = 1;
    for (double c : E.coef)
        if (c != 1.0) E.unit_coef = 0;
    E.out_slot.clear();
    E.out_coef.clear();
    E.out_pat.clear();
    for (int32_t k = 0; k < n_out; ++k) {
        const int32_t o = outputs[k];
        E.out_pat.push_back(pat[o]);
        for (const Handle& h : outh[k]) {
            E.out_slot.push_back(remap(h.s));
            E.out_coef.push_back(h.c);
        }
    }
    E.n_out_vals = (int64_t)E.out_slot.size();
    expr_layout_tables(E);
    return SSCO_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Program files: magic, version, the program, then a 64-bit FNV-1a digest
// of everything before it (the plan files' scheme).
constexpr uint64_t kExprMagic = 0x315058454F435353ull;  // "SSCOEXP1"
constexpr uint32_t kExprVersion = 1;

struct Fnv {
    uint64_t h = 0xcbf29ce484222325ull;
    void add(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 0x100000001b3ull;
    }
};
struct Out {
    std::ofstream f;
    Fnv sum;
    template <class T>
    void pod(const T& v) {
        f.write(reinterpret_cast<const char*>(&v), sizeof(T));
        sum.add(&v, sizeof(T));
    }
    template <class T>
    void vec(const std::vector<T>& v) {
        pod((uint64_t)v.size());
        if (!v.empty()) {
            f.write(reinterpret_cast<const char*>(v.data()), (std::streamsize)(v.size() * sizeof(T)));
            sum.add(v.data(), v.size() * sizeof(T));
        }
    }
};
struct In {
    std::ifstream f;
    Fnv sum;
    std::streamoff size = 0;
    template <class T>
    bool pod(T& v) {
        f.read(reinterpret_cast<char*>(&v), sizeof(T));
        if (!f) return false;
        sum.add(&v, sizeof(T));
        return true;
    }
    template <class T>
    bool vec(std::vector<T>& v) {
        uint64_t n = 0;
        if (!pod(n)) return false;
        const std::streamoff here = f.tellg();
        if (here < 0 || n > (uint64_t)(size - here) / sizeof(T)) return false;  // damage, not a size
        v.resize(n);
        if (n) {
            f.read(reinterpret_cast<char*>(v.data()), (std::streamsize)(n * sizeof(T)));
            if (!f) return false;
            sum.add(v.data(), n * sizeof(T));
        }
        return true;
    }
};

}  // namespace

size_t expr_value_bytes(const ExprProgram& E) { return E.precision == SSCO_VALS_F32 ? 4 : 8; }

size_t expr_workspace_bytes(const ExprProgram& E) {
    return align256((size_t)E.n_slots * E.B * expr_value_bytes(E));
}

void expr_layout_tables(ExprProgram& E) {
    // groups: runs of equal term count inside a level (the compiler orders
    // a level's expressions by term count, so a level has one run per count)
    E.groups.clear();
    int64_t n1 = 0, n2 = 0, nc = 0;
    for (int32_t l = 0; l < E.n_levels(); ++l) {
        for (int64_t op = E.lvl_begin[l]; op < E.lvl_begin[l + 1];) {
            const int64_t nt = E.term_off[op + 1] - E.term_off[op];
            int64_t r = op + 1;
            while (r < E.lvl_begin[l + 1] && E.term_off[r + 1] - E.term_off[r] == nt) ++r;
            ExprProgram::Group g{};
            g.nterms = (int32_t)nt;
            g.nmem = (int32_t)(r - op);
            g.op0 = op;
            g.quad = 0;
            g.uniform = 1;
            g.c_uniform = nt > 0 ? E.coef[E.term_off[op]] : 1.0;
            for (int64_t q = E.term_off[op]; q < E.term_off[r]; ++q) {
                if (E.f2[q] != 0) g.quad = 1;
                if (E.coef[q] != g.c_uniform) g.uniform = 0;
            }
            const int64_t cells = nt * g.nmem;
            g.i1_off = n1;
            n1 += cells;
            g.i2_off = g.quad ? n2 : 0;
            if (g.quad) n2 += cells;
            g.coef_off = g.uniform ? 0 : nc;
            if (!g.uniform) nc += cells;
            E.groups.push_back(g);
            op = r;
        }
    }
    E.n_i1 = n1, E.n_i2 = n2, E.n_coef = nc;
    E.out_unit = 1;
    for (double c : E.out_coef)
        if (c != 1.0) E.out_unit = 0;
    const size_t vb = expr_value_bytes(E);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(std::max<size_t>(bytes, 16));
        return o;
    };
    E.toff.groups = take(E.groups.size() * sizeof(ExprProgram::Group));
    E.toff.i1 = take((size_t)n1 * 4);
    E.toff.i2 = take((size_t)n2 * 4);
    E.toff.coef = take((size_t)nc * vb);
    E.toff.out_slot = take(E.out_slot.size() * 4);
    E.toff.out_coef = take(E.out_unit ? 0 : E.out_coef.size() * vb);
    E.toff.total = off;
}

std::vector<uint8_t> expr_table_image(const ExprProgram& E) {
    std::vector<uint8_t> img(E.toff.total, 0);
    const bool f32 = E.precision == SSCO_VALS_F32;
    auto put_val = [&](size_t at, double v) {
        if (f32) {
            const float x = (float)v;
            std::memcpy(img.data() + at, &x, 4);
        } else {
            std::memcpy(img.data() + at, &v, 8);
        }
    };
    const size_t vb = expr_value_bytes(E);
    if (!E.groups.empty())
        std::memcpy(img.data() + E.toff.groups, E.groups.data(), E.groups.size() * sizeof(ExprProgram::Group));
    int32_t* i1 = reinterpret_cast<int32_t*>(img.data() + E.toff.i1);
    int32_t* i2 = reinterpret_cast<int32_t*>(img.data() + E.toff.i2);
    for (const ExprProgram::Group& g : E.groups)
        for (int32_t m = 0; m < g.nmem; ++m) {
            const int64_t q0 = E.term_off[g.op0 + m];
            for (int32_t t = 0; t < g.nterms; ++t) {
                const int64_t cell = (int64_t)t * g.nmem + m;
                i1[g.i1_off + cell] = E.f1[q0 + t];
                if (g.quad) i2[g.i2_off + cell] = E.f2[q0 + t];
                if (!g.uniform) put_val(E.toff.coef + (size_t)(g.coef_off + cell) * vb, E.coef[q0 + t]);
            }
        }
    if (!E.out_slot.empty()) std::memcpy(img.data() + E.toff.out_slot, E.out_slot.data(), E.out_slot.size() * 4);
    if (!E.out_unit)
        for (size_t j = 0; j < E.out_coef.size(); ++j) put_val(E.toff.out_coef + j * vb, E.out_coef[j]);
    return img;
}

}  // namespace ssco

using ssco::g_expr_err;

extern "C" {

ssco_status ssco_expr_compile(const ssco_expr_node* nodes, int32_t n_nodes, const int32_t* outputs, int32_t n_out,
                              int32_t batch, int32_t precision, int32_t inline_terms, ssco_expr* out) {
    ssco_expr_opts o;
    std::memset(&o, 0, sizeof(o));
    o.batch = batch;
    o.precision = precision;
    o.inline_terms = inline_terms;
    return ssco_expr_compile_opts(nodes, n_nodes, outputs, n_out, &o, out);
}

ssco_status ssco_expr_compile_opts(const ssco_expr_node* nodes, int32_t n_nodes, const int32_t* outputs,
                                   int32_t n_out, const ssco_expr_opts* opts, ssco_expr* out) {
    if (!out || !opts) return ssco::bad(SSCO_ERR_INVALID_ARG, "NULL output handle or options");
    *out = nullptr;
    ssco_expr e = new (std::nothrow) ssco_expr_s();
    if (!e) return ssco::bad(SSCO_ERR_OOM, "host allocation failed");
    ssco_status st;
    try {
        st = ssco::compile(nodes, n_nodes, outputs, n_out, *opts, e->E);
    } catch (const std::bad_alloc&) {
        st = ssco::bad(SSCO_ERR_OOM, "host allocation failed while compiling");
    } catch (const std::exception& ex) {
        st = ssco::bad(SSCO_ERR_UNSUPPORTED, std::string("compile failed: ") + ex.what());
    }
    if (st != SSCO_OK) {
        delete e;
        return st;
    }
    *out = e;
    return SSCO_OK;
}

ssco_status ssco_expr_get_info(ssco_expr e, ssco_expr_info* o) {
    if (!e || !o) return ssco::bad(SSCO_ERR_INVALID_ARG, "NULL argument");
    const ssco::ExprProgram& E = e->E;
    std::memset(o, 0, sizeof(*o));
    o->n_leaf_vals = E.n_leaf_vals;
    o->n_out_vals = E.n_out_vals;
    o->n_slots = E.n_slots;
    o->n_ops = E.n_ops;
    o->n_terms = E.n_terms;
    o->n_unrolled = E.n_unrolled;
    o->n_alg_merged = E.n_alg_merged;
    o->n_alg_zero = E.n_alg_zero;
    o->n_factored = E.n_factored;
    o->n_inlined = E.n_inlined;
    o->n_levels = E.n_levels();
    o->batch = E.B;
    o->precision = E.precision;
    o->unit_coef = E.unit_coef;
    o->table_bytes = E.toff.total;
    o->workspace_bytes = ssco::expr_workspace_bytes(E);
    return SSCO_OK;
}

ssco_status ssco_expr_export(ssco_expr e, int32_t what, void* buf, uint64_t bytes) {
    if (!e || !buf) return ssco::bad(SSCO_ERR_INVALID_ARG, "NULL argument");
    const ssco::ExprProgram& E = e->E;
    const void* src = nullptr;
    size_t n = 0;
    switch (what) {
        case SSCO_EXPR_EXPORT_LEVELS: src = E.lvl_begin.data(), n = E.lvl_begin.size() * 8; break;
        case SSCO_EXPR_EXPORT_TERM_OFF: src = E.term_off.data(), n = E.term_off.size() * 8; break;
        case SSCO_EXPR_EXPORT_F1: src = E.f1.data(), n = E.f1.size() * 4; break;
        case SSCO_EXPR_EXPORT_F2: src = E.f2.data(), n = E.f2.size() * 4; break;
        case SSCO_EXPR_EXPORT_COEF: src = E.coef.data(), n = E.coef.size() * 8; break;
        case SSCO_EXPR_EXPORT_OUT_SLOT: src = E.out_slot.data(), n = E.out_slot.size() * 4; break;
        case SSCO_EXPR_EXPORT_OUT_COEF: src = E.out_coef.data(), n = E.out_coef.size() * 8; break;
        default: return ssco::bad(SSCO_ERR_INVALID_ARG, "unknown export");
    }
    if (bytes < n) return ssco::bad(SSCO_ERR_INVALID_ARG, "export buffer too small");
    if (n) std::memcpy(buf, src, n);
    return SSCO_OK;
}

ssco_status ssco_expr_output_shape(ssco_expr e, int32_t k, int32_t* rows, int32_t* cols, int64_t* nnz) {
    if (!e || k < 0 || k >= (int32_t)e->E.out_pat.size()) return ssco::bad(SSCO_ERR_INVALID_ARG, "bad output");
    const ssco::ExprCsr& P = e->E.out_pat[k];
    if (rows) *rows = P.rows;
    if (cols) *cols = P.cols;
    if (nnz) *nnz = (int64_t)P.ci.size();
    return SSCO_OK;
}

ssco_status ssco_expr_output_pattern(ssco_expr e, int32_t k, int64_t* rowptr, int32_t* colind) {
    if (!e || k < 0 || k >= (int32_t)e->E.out_pat.size()) return ssco::bad(SSCO_ERR_INVALID_ARG, "bad output");
    const ssco::ExprCsr& P = e->E.out_pat[k];
    if (rowptr) std::memcpy(rowptr, P.rp.data(), P.rp.size() * 8);
    if (colind && !P.ci.empty()) std::memcpy(colind, P.ci.data(), P.ci.size() * 4);
    return SSCO_OK;
}

ssco_status ssco_expr_bind(ssco_expr e, void* dev_tables, void* dev_ws, void* stream) {
    if (!e || !dev_tables || !dev_ws) return ssco::bad(SSCO_ERR_INVALID_ARG, "NULL argument");
    if ((reinterpret_cast<uintptr_t>(dev_tables) | reinterpret_cast<uintptr_t>(dev_ws)) & 255)
        return ssco::bad(SSCO_ERR_INVALID_ARG, "device buffers must be 256-byte aligned");
    ssco::ExprProgram& E = e->E;
    const std::vector<uint8_t> img = ssco::expr_table_image(E);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(dev_tables, img.data(), img.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        E.last_error = "table upload failed";
        return SSCO_ERR_CUDA;
    }
    E.d_tab = static_cast<uint8_t*>(dev_tables);
    E.d_ws = static_cast<uint8_t*>(dev_ws);
    E.bound = true;
    return SSCO_OK;
}

ssco_status ssco_expr_run(ssco_expr e, const void* leaf_vals, void* out_vals, void* stream) {
    if (!e) return ssco::bad(SSCO_ERR_INVALID_ARG, "NULL program");
    ssco::ExprProgram& E = e->E;
    if (!E.bound) {
        E.last_error = "ssco_expr_bind has not run";
        return SSCO_ERR_STATE;
    }
    if ((E.n_leaf_vals > 0 && !leaf_vals) || (E.n_out_vals > 0 && !out_vals)) {
        E.last_error = "NULL values";
        return SSCO_ERR_INVALID_ARG;
    }
    if (ssco::expr_launch_run(E, leaf_vals, out_vals, stream)) {
        E.last_error = "launch failed";
        return SSCO_ERR_CUDA;
    }
    return SSCO_OK;
}

ssco_status ssco_expr_save(ssco_expr e, const char* path) {
    if (!e || !path) return ssco::bad(SSCO_ERR_INVALID_ARG, "NULL argument");
    const ssco::ExprProgram& E = e->E;
    ssco::Out o;
    o.f.open(path, std::ios::binary | std::ios::trunc);
    if (!o.f) return ssco::bad(SSCO_ERR_INVALID_ARG, std::string("cannot open ") + path);
    o.pod(ssco::kExprMagic);
    o.pod(ssco::kExprVersion);
    o.pod(E.B), o.pod(E.precision), o.pod(E.unit_coef);
    o.pod(E.n_leaf_vals), o.pod(E.n_out_vals), o.pod(E.n_slots), o.pod(E.n_ops), o.pod(E.n_terms), o.pod(E.n_unrolled);
    o.vec(E.lvl_begin), o.vec(E.term_off), o.vec(E.f1), o.vec(E.f2), o.vec(E.coef), o.vec(E.out_slot),
        o.vec(E.out_coef);
    o.pod((uint64_t)E.out_pat.size());
    for (const ssco::ExprCsr& P : E.out_pat) o.pod(P.rows), o.pod(P.cols), o.vec(P.rp), o.vec(P.ci);
    const uint64_t digest = o.sum.h;
    o.f.write(reinterpret_cast<const char*>(&digest), sizeof(digest));
    o.f.flush();
    return o.f ? SSCO_OK : ssco::bad(SSCO_ERR_INVALID_ARG, "write failed");
}

ssco_status ssco_expr_load(const char* path, ssco_expr* out) {
    if (!path || !out) return ssco::bad(SSCO_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    ssco::In in;
    in.f.open(path, std::ios::binary | std::ios::ate);
    if (!in.f) return ssco::bad(SSCO_ERR_INVALID_ARG, std::string("cannot open ") + path);
    in.size = in.f.tellg();
    in.f.seekg(0);
    uint64_t magic = 0;
    uint32_t ver = 0;
    if (!in.pod(magic) || !in.pod(ver) || magic != ssco::kExprMagic || ver != ssco::kExprVersion)
        return ssco::bad(SSCO_ERR_INVALID_ARG, "not an expression program file of this version");
    ssco_expr e = new (std::nothrow) ssco_expr_s();
    if (!e) return ssco::bad(SSCO_ERR_OOM, "host allocation failed");
    ssco::ExprProgram& E = e->E;
    bool ok = false;
    try {
        uint64_t n_pat = 0;
        ok = in.pod(E.B) && in.pod(E.precision) && in.pod(E.unit_coef) && in.pod(E.n_leaf_vals) &&
             in.pod(E.n_out_vals) && in.pod(E.n_slots) && in.pod(E.n_ops) && in.pod(E.n_terms) &&
             in.pod(E.n_unrolled) && in.vec(E.lvl_begin) && in.vec(E.term_off) && in.vec(E.f1) && in.vec(E.f2) &&
             in.vec(E.coef) && in.vec(E.out_slot) && in.vec(E.out_coef) && in.pod(n_pat) && n_pat < (1u << 20);
        for (uint64_t k = 0; ok && k < n_pat; ++k) {
            ssco::ExprCsr P;
            ok = in.pod(P.rows) && in.pod(P.cols) && in.vec(P.rp) && in.vec(P.ci);
            E.out_pat.push_back(std::move(P));
        }
    } catch (const std::exception&) {
        ok = false;
    }
    const uint64_t got = in.sum.h;
    uint64_t digest = 0;
    char extra = 0;
    ok = ok && (bool)in.f.read(reinterpret_cast<char*>(&digest), sizeof(digest)) && digest == got &&
         !in.f.read(&extra, 1);
    // the tables must describe a program the runner can execute safely
    // (counts first, so that no size below is negative and no .back() is
    // taken of an empty table)
    ok = ok && E.B >= 1 && E.B <= 65535 && (E.precision == SSCO_VALS_F64 || E.precision == SSCO_VALS_F32) &&
         E.n_leaf_vals >= 0 && E.n_out_vals >= 0 && E.n_ops >= 0 && E.n_terms >= 0 &&
         E.n_slots == 1 + E.n_leaf_vals + E.n_ops && E.n_slots < (int64_t)INT32_MAX && !E.lvl_begin.empty() && E.lvl_begin.front() == 0 &&
         E.lvl_begin.back() == E.n_ops && (int64_t)E.term_off.size() == E.n_ops + 1 && E.term_off.front() == 0 &&
         E.term_off.back() == E.n_terms && (int64_t)E.f1.size() == E.n_terms && (int64_t)E.f2.size() == E.n_terms &&
         (int64_t)E.coef.size() == E.n_terms && (int64_t)E.out_slot.size() == E.n_out_vals &&
         (int64_t)E.out_coef.size() == E.n_out_vals;
    for (size_t l = 1; ok && l < E.lvl_begin.size(); ++l) ok = E.lvl_begin[l] >= E.lvl_begin[l - 1];
    for (int64_t i = 0; ok && i < E.n_ops; ++i) ok = E.term_off[i + 1] >= E.term_off[i];
    // every term of a level reads only the constant, the leaves and the
    // outputs of earlier levels (a level never reads its own or later slots)
    for (size_t l = 0; ok && l + 1 < E.lvl_begin.size(); ++l) {
        const int64_t lim = 1 + E.n_leaf_vals + E.lvl_begin[l];
        for (int64_t q = E.term_off[E.lvl_begin[l]]; ok && q < E.term_off[E.lvl_begin[l + 1]]; ++q)
            ok = E.f1[q] >= 0 && E.f1[q] < lim && E.f2[q] >= 0 && E.f2[q] < lim;
    }
    for (int64_t j = 0; ok && j < E.n_out_vals; ++j) ok = E.out_slot[j] >= 0 && E.out_slot[j] < E.n_slots;
    if (!ok) {
        delete e;
        return ssco::bad(SSCO_ERR_INVALID_ARG, "truncated, inconsistent or corrupt program file");
    }
    ssco::expr_layout_tables(E);
    *out = e;
    return SSCO_OK;
}

const char* ssco_expr_last_error(ssco_expr e) { return e ? e->E.last_error.c_str() : g_expr_err.c_str(); }

void ssco_expr_destroy(ssco_expr e) { delete e; }

}  // extern "C"
