"""The oracles' pins catch plausible mistakes.

Each case plants one mistake in one oracle function, of the kind a restatement of the paper (or of
the warm-start network's calculus) could contain (a dropped term, a wrong sign, a wrong index set,
a transposed operand, a reversed order): the function's source is edited in memory at one place,
compiled, and swapped in for the duration of the test.  Then the pins of that oracle run
(test_oracle_structure and test_oracle_method for the method, test_gnn_oracle for the network),
and at least one of them must fail.  Nothing is written to disk and nothing here touches the CUDA
path.
"""
import inspect
import itertools
import textwrap
import warnings

import pytest

from oracle import a2ls_oracle as O
from oracle import gnn_oracle as G
from tests import test_gnn_oracle as TG
from tests import test_oracle_fast as TF
from tests import test_oracle_method as TM
from tests import test_oracle_structure as TS


def _pins(modules):
    """Every pin of the given test modules with every parameter combination."""
    out = []
    for mod in modules:
        for name in sorted(dir(mod)):
            if not name.startswith("test_"):
                continue
            f = getattr(mod, name)
            axes = []
            for m in getattr(f, "pytestmark", []):
                if m.name != "parametrize":
                    continue
                names = m.args[0]
                names = [a.strip() for a in names.split(",")] if isinstance(names, str) else list(names)
                values = []
                for v in m.args[1]:
                    v = v.values if hasattr(v, "values") else v
                    values.append(tuple(v) if len(names) > 1 else (v,))
                axes.append([dict(zip(names, v)) for v in values])
            for combo in itertools.product(*axes):
                kw = {}
                for d in combo:
                    kw.update(d)
                out.append((f"{mod.__name__}.{name}{kw}", f, kw))
    return out


def _mutant(module, func_name: str, old: str, new: str):
    """The function func_name of `module` with the one occurrence of `old` in its source replaced."""
    src = textwrap.dedent(inspect.getsource(getattr(module, func_name)))
    assert src.count(old) == 1, (func_name, old)
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<{func_name} with a planted mistake>", "exec"), ns)
    return ns[func_name]


# name: (function, text in the oracle, planted replacement)
MUTANTS = {
    # Section 2: the graph of A + A^T, delta layers, the local order, R_i
    "graph_of_A_only": ("adjacency_lists", "(abs(A) + abs(A.T))", "abs(A)"),
    "overlap_one_layer_short": ("overlapping_subdomains", "for _ in range(delta)", "for _ in range(delta - 1)"),
    "overlap_layers_unsorted_union": ("overlapping_subdomains", "layers.extend(sorted(new))",
                                      "layers.extend(sorted(new, reverse=True))"),
    "pou_ones_on_overlap": ("partition_of_unity", "np.zeros(s.n_i - s.n_I)", "np.ones(s.n_i - s.n_I)"),
    "pou_multiplicity_not_inverted": ("partition_of_unity", "1.0 / count[s.idx]", "count[s.idx] / count.max()"),
    # Definition 3.1: s_i and A~_ii
    "lump_signed": ("lumped_row_sums", "Ar = abs(A.tocsr()[sub.gamma])", "Ar = A.tocsr()[sub.gamma]"),
    "lump_wrong_set": ("lumped_row_sums", "outside[sub.idx] = False", "outside[sub.gamma] = False"),
    "splitting_plus": ("block_splitting", "-= s[j]", "+= s[j]"),
    "splitting_on_wrong_rows": ("block_splitting", "At[nI + j, nI + j]", "At[j, j]"),
    # Eqs. 3.1-3.2: pencil, kernel part, order, real basis
    "gevp_without_D": ("local_gevp", "B = (d[:, None] * Aii) * d[None, :]", "B = Aii"),
    "gevp_swapped_pencil": ("local_gevp", "lam, a = sla.eig(Bc, Cc)", "lam, a = sla.eig(Cc, Bc)"),
    "gevp_smallest_first": ("_select_eigenpairs", "np.lexsort((-lam.imag, -np.abs(lam)))",
                            "np.lexsort((-lam.imag, np.abs(lam)))"),
    "gevp_pair_real_part_twice": ("_select_eigenpairs", "np.stack([u.real, u.imag], axis=1)",
                                  "np.stack([u.real, u.real], axis=1)"),
    "gevp_kernel_part_dropped": ("_kernel_part", "return VK @ Vt[:r].T", "return VK[:, :0]"),
    # Eq. 3.2: the threshold |lambda| > 1/tau
    "tau_threshold_not_inverted": ("_select_eigenpairs", "np.abs(lam) > 1.0 / tau", "np.abs(lam) > tau"),
    "tau_threshold_doubled": ("_select_eigenpairs", "np.abs(lam) > 1.0 / tau", "np.abs(lam) > 2.0 / tau"),
    # coarse space and Eq. 2.2 / 2.4
    "coarse_operator_transposed": ("coarse_space_from_W", "Phi.T @ (A @ Phi)", "Phi.T @ (A.T @ Phi)"),
    "coarse_columns_not_orthonormalised": ("orthonormal_columns", "return Q[:, keep]", "return W"),
    "coarse_correction_transposed_restriction": ("coarse_correction", "c = sla.lu_solve(cs.E_lu, g)",
                                                 "c = sla.lu_solve(cs.E_lu, g, trans=1)"),
    "deflated_without_residual_update": ("apply", "return q + one(P, r - P.A @ q)", "return q + one(P, r)"),
    "deflated_sign_of_update": ("apply", "return q + one(P, r - P.A @ q)", "return q + one(P, r + P.A @ q)"),
    "ras_without_D": ("apply_ras", "z[idx] += d * sla.lu_solve(lu, r[idx])", "z[idx] += sla.lu_solve(lu, r[idx])"),
    # Section 4: GMRES
    "gmres_mgs_wrong_vector": ("gmres", "w = w - H[i, j] * V[:, i]", "w = w - H[i, j] * V[:, j]"),
    "gmres_givens_rhs_sign": ("gmres", "g[j + 1] = -sn[j] * g[j]", "g[j + 1] = sn[j] * g[j]"),
    "gmres_flexible_uses_V": ("gmres", "x = x + Zs[:, :k] @ y", "x = x + V[:, :k] @ y"),
    "gmres_unpreconditioned_update": ("gmres", "x = x + Mop(V[:, :k] @ y)", "x = x + V[:, :k] @ y"),
    "gmres_restart_ignores_iterate": ("gmres", "r = b - Aop(x)", "r = b - Aop(0 * x)"),
    # Eqs. 2.1-2.2: local matrices, local factors, R_0^H
    "local_matrix_transposed": ("local_matrix", "return A.tocsr()[idx][:, idx].toarray()",
                                "return A.tocsr()[idx][:, idx].toarray().T"),
    "local_solves_with_splitting": ("setup", "local_lu.append(sla.lu_factor(Aii))",
                                    "local_lu.append(sla.lu_factor(block_splitting(A, s)))"),
    "prolongation_rows_reversed": ("assemble_phi", "restriction(s, n).T @ sp.csr_matrix(w)",
                                "restriction(s, n).T @ sp.csr_matrix(w[::-1])"),
    "coarse_correction_prolongs_g": ("coarse_correction", "return cs.Phi @ c", "return cs.Phi @ g"),
    # kernel detection: a threshold far too loose counts small singular values as null
    "null_space_threshold_loose": ("_null_space", "tol = M.shape[0] * EPS * (sv[0] if len(sv) else 0.0)",
                                   "tol = 1e-3 * (sv[0] if len(sv) else 0.0)"),
    # Section 3.2: the bound
    "bound_kc_plus_one_dropped": ("condition_bound", "(kc + 1)", "kc"),
    "multiplicity_counts_once": ("multiplicity_number", "count[s.idx] += 1", "count[s.interior] += 1"),
}

# the warm-start network (forward, propagation, loss, backward, Adam, bfloat16 rounding)
GNN_MUTANTS = {
    "edge_weight_scale": ("graph_and_features", "/ (2.0 * den[mutual])", "/ den[mutual]"),
    "overlap_flag_on_interior": ("graph_and_features", "X[n_I:, 3] = 1.0", "X[:n_I, 3] = 1.0"),
    "propagation_weights_swapped": ("propagate", "(1.0 - ALPHA) * (S @ p) + ALPHA * p0",
                                    "ALPHA * (S @ p) + (1.0 - ALPHA) * p0"),
    "adjoint_last_term_dropped": ("propagate_adjoint", "return g + acc", "return acc"),
    "forward_aggregates_with_S": ("forward", "m = W @ h", "m = S @ h"),
    "forward_rounds_biases": ("forward", "(round_bf16(v) if bf16 and k.startswith(\"W\") else v)",
                              "(round_bf16(v) if bf16 else v)"),
    "loss_gradient_sign": ("loss_and_dY", "dY = -2.0 * R @ C.T / m", "dY = 2.0 * R @ C.T / m"),
    "backward_aggregation_dropped": ("backward", "dh = dpre @ P[f\"W_s{t}\"].T + W.T @ (dpre @ P[f\"W_n{t}\"].T)",
                                     "dh = dpre @ P[f\"W_s{t}\"].T"),
    "backward_neighbour_grad_transposed": ("backward", "grads[f\"W_n{t}\"] = c[f\"m{t}\"].T @ dpre",
                                           "grads[f\"W_n{t}\"] = dpre.T @ c[f\"m{t}\"]"),
    "backward_bias_doubled": ("backward", "grads[f\"b_{t}\"] = dpre.sum(axis=0)",
                              "grads[f\"b_{t}\"] = 2.0 * dpre.sum(axis=0)"),
    "backward_relu_mask_of_wrong_layer": ("backward", "dpre = dh * (c[f\"pre{t}\"] > 0)",
                                          "dpre = dh * (c[f\"pre{t - 1}\"] > 0)"),
    "adam_without_bias_correction": ("adam_step", "mhat = m / (1.0 - beta1 ** t)", "mhat = m"),
    "bf16_truncates": ("round_bf16", "((f + 0x7FFF + lsb) >> 16) << 16", "(f >> 16) << 16"),
    "sample_mean_over_all": ("sample_loss_grad", "return (tot / cnt, g / cnt) if cnt else (0.0, g)",
                             "return (tot / len(subdomains), g / len(subdomains)) if cnt else (0.0, g)"),
}

# the oracle-fast local eigensolve (Arnoldi on the inverted pencil), pinned by the dense-QZ oracle
FAST_MUTANTS = {
    "fast_operator_without_D": ("local_gevp_fast", "B = (Dm @ sp.csr_matrix(Aii) @ Dm).tocsr()",
                                "B = sp.csr_matrix(Aii)"),
    "fast_operator_transposed": ("local_gevp_fast", "return lu.solve(rhs)[:n]", "return lu.solve(rhs, trans=\"T\")[:n]"),
    "fast_smallest_magnitude": ("local_gevp_fast", 'which="LM"', 'which="SM"'),
    "fast_splitting_sign": ("sparse_local_matrices", "-= s[j]", "+= s[j]"),
}

SUITES = {"method": (O, (TS, TM), MUTANTS), "network": (G, (TG,), GNN_MUTANTS), "fast": (O, (TF,), FAST_MUTANTS)}
PINS = {name: _pins(mods) for name, (_, mods, _) in SUITES.items()}
CASES = [(suite, m) for suite, (_, _, muts) in SUITES.items() for m in sorted(muts)]


@pytest.mark.parametrize("suite,mutant", CASES)
def test_pins_catch_planted_mistake(suite, mutant, monkeypatch):
    module, _, muts = SUITES[suite]
    func, old, new = muts[mutant]
    monkeypatch.setattr(module, func, _mutant(module, func, old, new))
    failed = None
    for label, f, kw in PINS[suite]:
        try:
            with warnings.catch_warnings():
                warnings.simplefilter("ignore")
                f(**kw)
        except Exception:  # an assertion, or an error raised by the planted mistake
            failed = label
            break
    assert failed is not None, f"no pin fails with the planted mistake {mutant}"


@pytest.mark.parametrize("suite", sorted(SUITES))
def test_unmutated_copies_pass(suite):
    """The compile-and-swap mechanism itself changes nothing: every pin passes on copies of the
    oracle functions compiled from their unedited source."""
    module, _, muts = SUITES[suite]
    funcs = sorted({f for f, _, _ in muts.values()})
    mp = pytest.MonkeyPatch()
    try:
        for func in funcs:
            src = textwrap.dedent(inspect.getsource(getattr(module, func)))
            ns = dict(vars(module))
            exec(compile(src, f"<{func} copy>", "exec"), ns)
            mp.setattr(module, func, ns[func])
        for label, f, kw in PINS[suite]:
            with warnings.catch_warnings():
                warnings.simplefilter("ignore")
                f(**kw)
    finally:
        mp.undo()
