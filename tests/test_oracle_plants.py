"""The pins catch plausible mistakes in the oracle.  gap_oracle.c compiles
mistake k when built with -DORACLE_PLANT=k (the oracle binding builds and
loads that variant when the environment variable ORACLE_PLANT is k).  For
each planted mistake a subprocess runs the pin meant to catch it and must
see it fail on an assertion; where a weaker check would not see the mistake,
that check runs too and must still pass, which shows why the specific pin is
needed.  The mistakes are a dropped term or factor, a wrong sign, a wrong
index or exponent, and a transposed operand, one in each part of the
oracle."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

B, S_, P, K = ("tests/test_oracle_basis.py::", "tests/test_oracle_soap.py::", "tests/test_oracle_predict.py::",
               "tests/test_oracle_knm.py::")

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
}


def _run(k, nodes):
    env = dict(os.environ, ORACLE_PLANT=str(k))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", *nodes], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    lines = r.stdout.strip().splitlines()
    return r.returncode, (lines[-1] if lines else ""), r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.parametrize("k", sorted(PLANTS))
def test_pin_catches_planted_mistake(k):
    what, catch, miss = PLANTS[k]
    for node in catch:
        rc, last, log = _run(k, [node])
        assert rc == 1 and "failed" in last and "error" not in last, f"planted {k} ({what}) not caught by {node}:\n{log}"
        assert "AssertionError" in log or "assert " in log, log
    if miss:
        rc, last, log = _run(k, miss)
        assert rc == 0 and "passed" in last, f"planted {k}: {miss} expected to pass:\n{log}"


def test_every_planted_mistake_is_listed():
    src = open(os.path.join(ROOT, "oracle", "gap_oracle.c")).read()
    planted = {int(t.split(")")[0]) for t in src.split("PLANT(")[1:] if t.split(")")[0].isdigit()}
    assert planted == set(PLANTS)
