"""The oracle's pins catch planted mistakes.

Each case copies the oracle's C source with one plausible mistake (a dropped
term, a flipped sign, a wrong index, a transposed operand), builds it with the
oracle's own flags and runs the pin module against that build
(``SSCO_ORACLE_LIB``).  The pins must fail by assertion, not by a crash, so a
test that passed against the mutant, or a pin that never looked at the mutated
step, would show up here.  CPU only.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ssco_oracle.c")

# (name, exact text in the oracle, planted replacement)
MUTANTS = [
    ("assembly drops the shift",
     "val[colptr[u]] += shift; /* diagonal first in column */",
     "val[colptr[u]] += 0.0 * shift; /* diagonal first in column */"),
    ("element assembly drops the shift",
     "if (touched[u]) val[colptr[u]] += shift;",
     "if (touched[u]) val[colptr[u]] += 0.0 * shift;"),
    ("Cholesky update added instead of subtracted",
     "acc[Li[p]] -= ljk * Lval[p];",
     "acc[Li[p]] += ljk * Lval[p];"),
    ("factorization skips K's diagonal entry",
     "if (s->Krowind[p] >= j) acc[s->Krowind[p]] += Kval[p];",
     "if (s->Krowind[p] > j) acc[s->Krowind[p]] += Kval[p];"),
    ("failing pivot recorded one column late",
     "            bad = j;\n            break;",
     "            bad = j + 1;\n            break;"),
    ("pivot without the square root",
     "double ljj = sqrt(d);",
     "double ljj = d;"),
    ("forward solve reads the wrong entry",
     "y[Li[p]] -= Lval[p] * y[j];",
     "y[Li[p]] -= Lval[p] * y[Li[p]];"),
    ("backward solve with the transposed operand",
     "t -= Lval[p] * y[Li[p]];",
     "t -= Lval[p] * y[j];"),
    ("adjoint of the weights with the wrong sign",
     "wbar[e] = -am * ax;",
     "wbar[e] = am * ax;"),
    ("element adjoint takes the wrong mirrored term",
     "if (i != j) g += k * mu[v] * x[u];",
     "if (i != j) g += k * mu[u] * x[v];"),
    ("elimination tree takes the largest row",
     "s->parent[j] = len > 1 ? buf[1] : -1;",
     "s->parent[j] = len > 1 ? buf[len - 1] : -1;"),
    ("supernode joins a column with several children",
     "s->parent[j - 1] == j && nchild[j] == 1 &&",
     "s->parent[j - 1] == j && nchild[j] >= 1 &&"),
    ("supernode joins without the column-count condition",
     "s->colcount[j] == s->colcount[j - 1] - 1;",
     "s->colcount[j] <= s->colcount[j - 1];"),
    ("column level from the shortest path",
     "if (s->col_level[c] + 1 > lv) lv = s->col_level[c] + 1;",
     "if (lv == 0 || s->col_level[c] + 1 < lv) lv = s->col_level[c] + 1;"),
    ("supernode parent from the supernode's first column",
     "int32_t last = s->snode_first[k + 1] - 1;",
     "int32_t last = s->snode_first[k];"),
    ("permutation applies perm where its inverse belongs",
     "int32_t a = iperm[rowind[p]], b = iperm[j];",
     "int32_t a = perm[rowind[p]], b = perm[j];"),
    ("cotangent weight without the half",
     "w[tri_edge[3 * t + c]] += 0.5 * dot / cross;",
     "w[tri_edge[3 * t + c]] += dot / cross;"),
    ("block adjoint repeats one half of the mirrored pair",
     "-(mu[u] * x[v] + mu[v] * x[u])",
     "-(mu[u] * x[v] + mu[u] * x[v])"),
    ("tet stiffness with lambda replaced by mu",
     "double lam = Ee * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));",
     "double lam = Ee / (2.0 * (1.0 + nu));"),
    ("tet stiffness with tensor instead of engineering shear",
     "D[r + 3][r + 3] = mu;",
     "D[r + 3][r + 3] = 2.0 * mu;"),
]


def run_pins_against(tmp_path, source: str):
    """Builds `source` as the oracle library and runs the pin module on it."""
    mut = tmp_path / "ssco_oracle_variant.c"
    mut.write_text(source)
    lib = tmp_path / "libssco_oracle_variant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
                           "-o", str(lib), str(mut), "-lm"])
    env = dict(os.environ, SSCO_ORACLE_LIB=str(lib))
    return subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                           "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_pins_pass_on_the_unchanged_source_built_the_same_way(tmp_path):
    """Control: the harness itself (separate build, library override) leaves
    the pins green, so a failure below comes from the planted mistake."""
    r = run_pins_against(tmp_path, open(SRC).read())
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,orig,planted", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_fail_on_planted_mistake(tmp_path, name, orig, planted):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation site not unique or gone: {orig}"
    r = run_pins_against(tmp_path, src.replace(orig, planted))
    # exit code 1: a pin failed by assertion (a crash or an error would be
    # another code, and 0 would mean no pin noticed the mistake)
    assert r.returncode == 1, f"{name}: pins exit {r.returncode}\n{r.stdout[-2000:]}\n{r.stderr[-1000:]}"
    assert "FAILED" in r.stdout


# ---------------------------------------------------------------------------
# The sparse-expression evaluators are Python: each mutant is the wrapper's
# source with one planted mistake, executed as a module of its own and put in
# place of the oracle inside the pin module for the expression pins.
# ---------------------------------------------------------------------------
EXPR_MUTANTS = [
    ("sum keeps only the second operand",
     "d[key] = d.get(key, 0.0) + v",
     "d[key] = v"),
    ("product keeps only the last term",
     "d[(i, j)] = d.get((i, j), 0.0) + a * b",
     "d[(i, j)] = a * b"),
    ("transpose leaves the entries in place",
     "mats.append((ca, ra, {(j, i): v for (i, j), v in A.items()}))",
     "mats.append((ca, ra, {(i, j): v for (i, j), v in A.items()}))"),
    ("scaling ignores its factor",
     "mats.append((ra, ca, {key: al * v for key, v in A.items()}))",
     "mats.append((ra, ca, {key: v for key, v in A.items()}))"),
    ("shared leaf values all read through the map's first entry",
     "v = float(leaf_vals[off + (int(vm[q]) if vm is not None else q)])",
     "v = float(leaf_vals[off + (int(vm[0]) if vm is not None else q)])"),
    ("row of a sum keeps only the second operand",
     "r[j] = r.get(j, 0.0) + v",
     "r[j] = v"),
    ("row of a product keeps only the last term",
     "r[j] = r.get(j, 0.0) + a * b",
     "r[j] = a * b"),
    ("row of a scaling ignores its factor",
     "r = {j: nd[2] * v for j, v in row(nd[1], i).items()}",
     "r = {j: v for j, v in row(nd[1], i).items()}"),
]
EXPR_PINS = ["test_expr_oracle_matches_dense_evaluation", "test_expr_oracle_tridiagonal_cube_closed_form",
             "test_expr_oracle_weighted_laplacian_of_a_path", "test_expr_row_oracle_equals_full_oracle",
             "test_expr_oracle_shared_values_equal_expanded_values"]


def expression_pins_failing(monkeypatch, source: str):
    """Runs the expression pins against `source` as the oracle module; returns
    the pins that failed by assertion (any other exception propagates)."""
    import types

    import test_oracle_pins as T
    from oracle import oracle as real
    mod = types.ModuleType("oracle_variant")
    mod.__file__ = real.__file__
    exec(compile(source, real.__file__, "exec"), mod.__dict__)
    monkeypatch.setattr(T, "O", mod)
    failed = []
    for pin in EXPR_PINS:
        try:
            getattr(T, pin)()
        except AssertionError:
            failed.append(pin)
    return failed


def test_expression_pins_pass_on_the_unchanged_wrapper(monkeypatch):
    from oracle import oracle as real
    assert expression_pins_failing(monkeypatch, open(real.__file__).read()) == []


@pytest.mark.parametrize("name,orig,planted", EXPR_MUTANTS, ids=[m[0] for m in EXPR_MUTANTS])
def test_expression_pins_fail_on_planted_mistake(monkeypatch, name, orig, planted):
    from oracle import oracle as real
    src = open(real.__file__).read()
    assert src.count(orig) == 1, f"mutation site not unique or gone: {orig}"
    assert expression_pins_failing(monkeypatch, src.replace(orig, planted)), name
