// ssco_expr_internal.h -- compiled program of a fixed-pattern sparse matrix
// expression: level-ordered scalar expressions (sums of products of two
// slots) with their harvested index tables, shared by the host compiler and
// the device runner.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ssco.h"

namespace ssco {

struct ExprCsr {
    int32_t rows = 0, cols = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
};

struct ExprProgram {
    int32_t B = 1;
    int32_t precision = SSCO_VALS_F64;
    int64_t n_leaf_vals = 0, n_out_vals = 0, n_slots = 0, n_ops = 0, n_terms = 0, n_unrolled = 0;
    // what the optional compile steps did (not saved in program files)
    int64_t n_alg_merged = 0, n_alg_zero = 0, n_factored = 0, n_inlined = 0;
    int32_t unit_coef = 1;
    std::vector<int64_t> lvl_begin;  // [n_levels + 1] op ranges (op i is slot op_base + i)
    std::vector<int64_t> term_off;   // [n_ops + 1]
    std::vector<int32_t> f1, f2;     // factor slots per term (f2 = 0: the constant one)
    std::vector<double> coef;        // per term
    std::vector<int32_t> out_slot;   // per output value
    std::vector<double> out_coef;
    std::vector<ExprCsr> out_pat;
    int64_t op_base() const { return 1 + n_leaf_vals; }
    int32_t n_levels() const { return (int32_t)lvl_begin.size() - 1; }

    // device form (built from the tables above by expr_layout_tables): the
    // expressions of a level in groups of equal term count -- the assembly
    // groups' form -- with term-major, member-innermost factor tables (the
    // second factor only for groups with a product of two slots, the
    // coefficients only for groups whose coefficients differ)
    struct Group {
        int32_t nterms, nmem;
        int32_t quad, uniform;  // quad: some term has two slot factors
        int64_t op0;            // first expression (slot op_base + op0)
        int64_t i1_off, i2_off, coef_off;
        double c_uniform;
    };
    std::vector<Group> groups;       // level by level, ascending op0
    int32_t out_unit = 1;            // every output factor is 1 (no factor table)
    int64_t n_i1 = 0, n_i2 = 0, n_coef = 0;
    struct {
        size_t groups, i1, i2, coef, out_slot, out_coef, total;
    } toff{};
    uint8_t* d_tab = nullptr;
    uint8_t* d_ws = nullptr;
    bool bound = false;
    std::string last_error;
};

size_t expr_value_bytes(const ExprProgram& E);
size_t expr_workspace_bytes(const ExprProgram& E);
void expr_layout_tables(ExprProgram& E);
std::vector<uint8_t> expr_table_image(const ExprProgram& E);
int expr_launch_run(ExprProgram& E, const void* leaf_vals, void* out_vals, void* stream);

}  // namespace ssco

struct ssco_expr_s {
    ssco::ExprProgram E;
};
