"""The pins catch plausible mistakes in the oracle.

Each case copies oracle/gqt_oracle.cpp, plants one mistake (a dropped term, a
wrong sign or index, a wrong constant), compiles the copy on the CPU and runs
the pins of test_oracle_pins.py against it: at least one pin must fail."""
import os
import subprocess
import tempfile

import pytest

import oracle as O
from tests import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(O.__file__), "gqt_oracle.cpp")

# (name, exact text in the oracle, replacement)
MUTATIONS = [
    ("drop on-site term", "cplx s = (h.eps[i] / h.dE) * x[i];", "cplx s = 0.0;"),
    ("recursion sign", "t2[i] = 2.0 * ht[i] - t0[i];\n    mu[m]", "t2[i] = 2.0 * ht[i] + t0[i];\n    mu[m]"),
    ("conjugate l dropped", "s += std::conj(a[i]) * b[i];", "s += a[i] * b[i];"),
    ("evolution phase sign", "(sign > 0) ? cplx(0.0, -1.0) : cplx(0.0, 1.0);\n  std::vector<cplx> t0(psi",
     "(sign > 0) ? cplx(0.0, 1.0) : cplx(0.0, -1.0);\n  std::vector<cplx> t0(psi"),
    ("evolution factor 2", "cplx c = 2.0 * phase * std::cyl_bessel_j(1.0, x);\n    for (int64_t i = 0; i < n; ++i) out[i] += c * t1[i];",
     "cplx c = phase * std::cyl_bessel_j(1.0, x);\n    for (int64_t i = 0; i < n; ++i) out[i] += c * t1[i];"),
    ("commutator dx sign", "s += (-h.dx[i * h.K + k]) * (h.hop[i * h.K + k] / h.dE) * x[j];",
     "s += (h.dx[i * h.K + k]) * (h.hop[i * h.K + k] / h.dE) * x[j];"),
    ("commutator term dropped", "w2[i] = 2.0 * a[i] + 2.0 * b[i] - w0[i];", "w2[i] = 2.0 * b[i] - w0[i];"),
    ("velocity without i", "s += I * h.dx[i * h.K + k] * h.hop[i * h.K + k] * x[j];",
     "s += h.dx[i * h.K + k] * h.hop[i * h.K + k] * x[j];"),
    ("VAC evolves with U(+dt)", "evolve(h, a.data(), dt[k], -1, Np[k], tmp.data());",
     "evolve(h, a.data(), dt[k], +1, Np[k], tmp.data());"),
    ("MSD missing U px term", "px[i] = xu[i] + upx[i];", "px[i] = xu[i];"),
    ("Jackson alpha 1/M", "const double a = 1.0 / (M + 1.0);", "const double a = 1.0 / M;"),
    ("KPM (2 - delta) dropped", "s += g[n] * (n == 0 ? 1.0 : 2.0) * std::cos(n * th)", "s += g[n] * std::cos(n * th)"),
    ("KPM prefactor N/Omega dropped", "out[(int64_t)r * NE + e] = 2.0 * n_over_omega /", "out[(int64_t)r * NE + e] = 2.0 /"),
    ("sigma_VAC rectangle rule", "0.5 * dt[k - 1] * (vac[(int64_t)(k - 1) * NE + e] + vac[(int64_t)k * NE + e]);",
     "dt[k - 1] * vac[(int64_t)k * NE + e];"),
    ("adjoint factor 2 dropped", "const double f = (m == 1 ? 1.0 : 2.0) / h.dE;", "const double f = 1.0 / h.dE;"),
    ("adjoint velocity sign", "const cplx mI(0.0, -1.0);", "const cplx mI(0.0, 1.0);"),
    ("Kubo-Bastin directions swapped", "apply_vd(h, d_a, rq, u.data());", "apply_vd(h, d_b, rq, u.data());"),
    ("Kubo-Bastin B_n without velocity", "for (int n = 0; n < M; ++n) apply_vd(h, d_b, Tn[n].data(), B[n].data());",
     "for (int n = 0; n < M; ++n) B[n] = Tn[n];"),
    ("Kubo-Bastin resolvent phase sign", "std::exp(-I * (double)n * th) * (x + I * (double)n * s)",
     "std::exp(I * (double)n * th) * (x + I * (double)n * s)"),
    ("Kubo-Bastin (2 - delta) dropped", "w[n] = (n == 0 ? 1.0 : 2.0) * (kernel == 0", "w[n] = (1.0) * (kernel == 0"),
    ("Kubo-Bastin prefactor 2/Omega", "sigma[j] = 2.0 / area * run;", "sigma[j] = 1.0 / area * run;"),
    ("Fermi function sign", "return 1.0 / (1.0 + std::exp((e - mu[q]) / kT));",
     "return 1.0 / (1.0 + std::exp((mu[q] - e) / kT));"),
    ("Fermi step half weight", "e > mu[q] ? 0.0 : 0.5", "e > mu[q] ? 0.0 : 1.0"),
]

PINS = [
    lambda: P.test_dos_moments_match_exact_diagonalisation("honeycomb", True),
    lambda: P.test_general_moments_l_neq_r(),
    lambda: P.test_constant_diagonal_closed_form(),
    lambda: P.test_evolution_matches_matrix_exponential("square", True, 1),
    lambda: P.test_commutator_matches_daleckii_krein("square", True),
    lambda: P.test_velocity_is_i_commutator(),
    lambda: P.test_vac_moments_match_definition("square", True),
    lambda: P.test_msd_moments_match_definition("square", True),
    lambda: P.test_jackson_kernel_properties(),
    lambda: P.test_jackson_kernel_autocorrelation_form(),
    lambda: P.test_kpm_normalisation_chebyshev_gauss(),
    lambda: P.test_kpm_chain_band_centre(),
    lambda: P.test_sigma_rules(),
    lambda: P.test_cheb_adjoint_matches_daleckii_krein(),
    lambda: P.test_vac_loss_gradient_matches_finite_differences(),
    lambda: P.test_kb_moments_match_exact_trace("xy"),
    lambda: P.test_kb_moments_vanish_by_mirror_symmetry(),
    lambda: P.test_kubo_bastin_reconstruction_closed_forms(),
    lambda: P.test_kubo_bastin_fermi_limits_and_quadrature(),
]


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory() as d:
        yield d
    O.use_library(None)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(workdir, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/found: {name}"
    path = os.path.join(workdir, f"mut_{abs(hash(name))}.cpp")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = path[:-4] + ".so"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-o", so, path])
    O.use_library(so)
    try:
        caught = []
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                caught.append(pin)
        assert caught, f"no pin caught the planted mistake: {name}"
    finally:
        O.use_library(None)


def test_jackson_mutation_caught_by_autocorrelation_pin_alone(workdir):
    """The Jackson kernel's alpha (Eq. 31) is pinned by its autocorrelation construction,
    not only by properties that a wrong alpha also satisfies."""
    src = open(SRC).read()
    old, new = "const double a = 1.0 / (M + 1.0);", "const double a = 1.0 / M;"
    path = os.path.join(workdir, "mut_jackson_alone.cpp")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = path[:-4] + ".so"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-o", so, path])
    O.use_library(so)
    try:
        P.test_jackson_kernel_properties()  # the properties alone do not see it
        with pytest.raises(AssertionError):
            P.test_jackson_kernel_autocorrelation_form()
    finally:
        O.use_library(None)
