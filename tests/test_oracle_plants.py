"""The pins catch plausible mistakes in the oracle.  With the environment
variable ORACLE_PLANT = k the oracle carries mistake k: the binding either
builds and loads gap_oracle.c compiled with -DORACLE_PLANT=k, or (for the
mistakes planted in the Python module: variance, CUR, compression) switches
on a line marked "planted k" there.  For each planted
mistake a subprocess runs the pin meant to catch it and must see it fail on
an assertion; where a weaker check would not see the mistake, that check
runs too and must still pass, which shows why the specific pin is needed.
The mistakes are dropped terms or factors, wrong signs, wrong indices or
exponents and transposed operands, in every part of the oracle."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

B, S_, P, K = ("tests/test_oracle_basis.py::", "tests/test_oracle_soap.py::", "tests/test_oracle_predict.py::",
               "tests/test_oracle_knm.py::")
V, CU, CO = "tests/test_oracle_variance.py::", "tests/test_oracle_cur.py::", "tests/test_oracle_compression.py::"

# k: (mistake, pins that must fail, checks that must still pass)
PLANTS = {
    1: ("power spectrum without the sqrt 2 of off-diagonal channel pairs (Eq. 22)",
        [S_ + "test_single_neighbour_closed_form"], []),
    2: ("wrong sign of the projection in d p_hat = (I - p_hat p_hat^T) dp / |p| (Eq. 24)",
        [P + "test_forces_by_finite_differences"], []),
    3: ("kernel exponent zeta + 1 in the local energy and the K_NM rows alike (Eq. 13)",
        [K + "test_kernel_exponent_by_homogeneity"],
        [P + "test_forces_by_finite_differences", K + "test_knm_times_alpha_reproduces_predict"]),
    4: ("virial sign (Appendix: stress has the opposite sign)", [P + "test_virial_by_finite_strain"], []),
    5: ("force sign F = +dE/dr (Eq. 3)", [P + "test_forces_by_finite_differences"],
        [P + "test_energy_is_sum_of_local_and_forces_sum_to_zero"]),
    6: ("Y_l,m and Y_l,-m exchanged", [B + "test_ylm_matches_scipy"],
        [S_ + "test_descriptor_invariances", B + "test_ylm_orthonormal_and_addition_theorem"]),
    7: ("4 pi dropped from the radial integral (Eq. 20)", [B + "test_radial_integral_against_direct_quadrature"],
        [S_ + "test_descriptor_invariances", P + "test_forces_by_finite_differences"]),
    8: ("periodic images of the central atom itself dropped", [S_ + "test_neighbour_count_diamond"], []),
    9: ("sign of the cutoff function's derivative (Eq. 18)", [B + "test_fcut_eq18_piecewise"], []),
    10: ("whole two-body pair term given to each atom (Eqs. 10-11)", [P + "test_two_body_dimer_closed_form"],
         [P + "test_two_body_plus_soap_forces_by_finite_differences"]),
    11: ("least-squares right-hand side not scaled by S^-1/2 (Eq. 6)",
         [K + "test_qr_solution_equals_normal_equations"], []),
    12: ("K_NM force rows with the sign of +grad (text after Eq. 4)", [K + "test_knm_times_alpha_reproduces_predict"],
         []),
    13: ("modified spherical Bessel series term off by one", [B + "test_bessel_closed_forms"], []),
    14: ("Jacobi parameters (2, 6) of the radial basis swapped", [B + "test_radial_basis_orthonormal"], []),
    15: ("embedding weights read as [species][K] instead of [K][species] (Eq. 25)",
         [S_ + "test_embedding_weights_are_channel_by_species"], [S_ + "test_species_coupling_reductions"]),
    26: ("fractional coordinates through the transposed inverse cell",
         [S_ + "test_cell_choice_does_not_matter"], [S_ + "test_descriptor_invariances"]),
    27: ("K_MM with the exponent zeta + 1 (Eq. 13)", [K + "test_kernel_exponent_by_homogeneity"],
         [K + "test_kmm_symmetric_psd", K + "test_qr_solution_equals_normal_equations"]),
    28: ("sampled forces without the neighbours' terms", [P + "test_sampled_equals_full"], []),
    29: ("normal equations weighted by 1/sigma instead of 1/sigma^2 (Eq. 4)",
         [K + "test_qr_solution_equals_normal_equations"], []),
    30: ("sign of the two-body kernel's Gaussian derivative (Eq. 11)",
         [P + "test_two_body_plus_soap_forces_by_finite_differences"], []),
    31: ("central Gaussian in every species channel, not only its own (Eq. 19)",
         [S_ + "test_isolated_atom_closed_form", S_ + "test_species_coupling_reductions"],
         [S_ + "test_single_neighbour_closed_form"]),
    33: ("Cholesky factor without the update of each row by the earlier ones",
         [K + "test_qr_solution_equals_normal_equations", K + "test_teacher_student_fit"], []),
    # planted in the module oracle/__init__.py (predictive variance, CUR, compression)
    16: ("sign of the (A^T A)^-1 term of the predictive variance",
         [V + "test_sparse_points_observed_directly_is_the_full_gp"], [V + "test_kernel_rows_reproduce_local_energies"]),
    17: ("variance's A without the S^-1/2 row scaling (Eq. 5)",
         [V + "test_sparse_points_observed_directly_is_the_full_gp"],
         [V + "test_no_data_gives_the_prior", V + "test_variance_decreases_as_data_are_added"]),
    18: ("leverage scores without the 1/k", [CU + "test_scores_sum_to_one_and_match_the_hat_matrix"],
         [CU + "test_scores_invariant_to_rotation_and_scale"]),
    19: ("duplicate rows not skipped (Sec. 3.2.2)", [CU + "test_diagonal_design_picks_the_dominant_directions"],
         [CU + "test_selection_order_and_default_rank"]),
    20: ("rows chosen by the smallest scores", [CU + "test_selection_order_and_default_rank"],
         [CU + "test_scores_sum_to_one_and_match_the_hat_matrix"]),
    21: ("tensor sketch with w on both sides (u ignored; Sec. 3.3.3)", [CO + "test_sketch_identity_in_expectation"],
         [CO + "test_compressed_descriptors_are_rotation_invariant"]),
    22: ("nu_S = 1 summing the first species index instead of the second", [CO + "test_nu_one_orders_keep_the_first_index"],
         [CO + "test_nu_full_orders_keep_the_kernel_and_zero_orders_sum_channels",
          CO + "test_compressed_descriptors_are_rotation_invariant"]),
    23: ("'trivial' recipe indexing species alpha instead of channel alpha n_max",
         [CO + "test_matrix_identity_and_trivial_entries"], [CO + "test_compressed_descriptors_are_rotation_invariant"]),
    24: ("compressed descriptor not renormalised (Sec. 3.3.4)", [CO + "test_decomposition_with_unit_weights_is_the_diagonal"],
         [CO + "test_compressed_descriptors_are_rotation_invariant"]),
    32: ("exponent zeta + 1 in the compressed local energies (Eqs. 2, 13)",
         [CO + "test_identity_map_energies_equal_the_uncompressed_oracle"], []),
    25: ("nu_R = 1 summing the first radial index instead of the second", [CO + "test_nu_one_orders_keep_the_first_index"],
         [CO + "test_nu_full_orders_keep_the_kernel_and_zero_orders_sum_channels",
          CO + "test_compressed_descriptors_are_rotation_invariant"]),
}


WORKERS = max(2, min(16, os.cpu_count() or 2))


def _run(k, nodes):
    # the oracle's OpenMP threads share the cores with the other workers
    env = dict(os.environ, ORACLE_PLANT=str(k), OMP_NUM_THREADS=str(max(1, (os.cpu_count() or 2) // WORKERS)))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", *nodes], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    lines = r.stdout.strip().splitlines()
    return r.returncode, (lines[-1] if lines else ""), r.stdout[-3000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def runs():
    """Every subprocess run of the table, in parallel: the planted variants
    of gap_oracle.c are compiled first, then each pin that must fail runs on
    its own and the checks that must pass run together."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(WORKERS) as ex:
        c_src = open(os.path.join(ROOT, "oracle", "gap_oracle.c")).read()
        list(ex.map(lambda k: subprocess.run([sys.executable, "-c", "import oracle; oracle.build()"], cwd=ROOT,
                                             env=dict(os.environ, ORACLE_PLANT=str(k)), check=True, timeout=600),
                    [k for k in sorted(PLANTS) if f"PLANT({k})" in c_src]))
        jobs = [(k, (node,)) for k, (_, catch, _) in PLANTS.items() for node in catch]
        jobs += [(k, tuple(miss)) for k, (_, _, miss) in PLANTS.items() if miss]
        return dict(zip(jobs, ex.map(lambda j: _run(*j), jobs)))


@pytest.mark.parametrize("k", sorted(PLANTS))
def test_pin_catches_planted_mistake(runs, k):
    what, catch, miss = PLANTS[k]
    for node in catch:
        rc, last, log = runs[(k, (node,))]
        assert rc == 1 and "failed" in last and "error" not in last, f"planted {k} ({what}) not caught by {node}:\n{log}"
        # an assertion of the pin, or the oracle's own check of a factorisation
        assert "AssertionError" in log or "assert " in log or "LinAlgError" in log, log
    if miss:
        rc, last, log = runs[(k, tuple(miss))]
        assert rc == 0 and "passed" in last, f"planted {k}: {miss} expected to pass:\n{log}"


def test_every_planted_mistake_is_listed():
    import re
    c_src = open(os.path.join(ROOT, "oracle", "gap_oracle.c")).read()
    py_src = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    planted = {int(k) for k in re.findall(r"PLANT\((\d+)\)", c_src)}
    py = {int(k) for k in re.findall(r"_PLANT [=!]= (\d+)", py_src)}
    assert planted.isdisjoint(py) and planted | py == set(PLANTS)
    import oracle
    assert set(oracle._PY_PLANTS) == py
