"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each one."""
import numpy as np
import pytest

from oracle import etd, phi as phimod
import test_oracle_scheme as scheme_pins


def _dense_pin():
    scheme_pins.test_eigen_path_matches_dense_expm((4, 5), (0.25, 0.2), 2, 0.5)


def test_unmutated_pin_passes():
    _dense_pin()


def test_dropped_phi2_term_is_caught(monkeypatch):
    orig = etd.Stepper.__init__

    def init(self, *a, **k):
        orig(self, *a, **k)
        self.phi2 = np.zeros_like(self.phi2)
    monkeypatch.setattr(etd.Stepper, "__init__", init)
    with pytest.raises(AssertionError):
        _dense_pin()


def test_transposed_eigenvector_operand_is_caught(monkeypatch):
    def forward(U, Ps):
        for a, P in enumerate(Ps):
            U = etd.mode_product(P, U, a)        # P instead of P^T
        return U
    monkeypatch.setattr(etd, "forward", forward)
    with pytest.raises(AssertionError):
        _dense_pin()


def test_wrong_stage_time_fraction_is_caught(monkeypatch):
    orig = etd.Stepper.__init__

    def init(self, Ps, H, tau, scheme, c2=0.5):
        orig(self, Ps, H, tau, scheme, c2)
        self.Ec = phimod.phi(0, -tau * H)        # stage uses e^{-tau H} instead of e^{-c2 tau H}
    monkeypatch.setattr(etd.Stepper, "__init__", init)
    with pytest.raises(AssertionError):
        _dense_pin()


def test_wrong_phi_index_is_caught(monkeypatch):
    orig = phimod.phi

    def bad(k, z):
        return orig(k + 1 if k == 2 else k, z)   # phi_3 where phi_2 belongs
    monkeypatch.setattr(etd, "phi", bad)
    with pytest.raises(AssertionError):
        _dense_pin()


def test_reaction_sign_error_is_caught(monkeypatch):
    monkeypatch.setattr(etd, "allen_cahn", lambda flin=1.0, fcub=-1.0: (lambda t, u: -flin * u + fcub * u ** 3))
    with pytest.raises(AssertionError):
        _dense_pin()


# ---------------------------------------------------------------- periodic path and Flory-Huggins
import test_oracle_periodic as periodic_pins
from oracle import fem


def test_periodic_pins_pass_unmutated():
    periodic_pins.test_periodic_eigen_path_matches_dense_expm((4, 5), (0.25, 0.2), 2, "flory_huggins")
    periodic_pins.test_periodic_step_matches_the_dft_route((16, 12), 2)


def test_missing_wrap_element_is_caught(monkeypatch):
    """Periodic assembly that forgets the element joining node N-1 to node 0."""
    orig = fem.assemble_1d

    def bad(N, h, bc="dirichlet"):
        A, B = orig(N, h, bc)
        if bc == "periodic":
            A, B = A.copy(), B.copy()
            me, ke = fem.element_mass_1d(h), fem.element_stiffness_1d(h)
            for (i, j), (a, b) in zip([(N - 1, N - 1), (N - 1, 0), (0, N - 1), (0, 0)],
                                      [(0, 0), (0, 1), (1, 0), (1, 1)]):
                A[i, j] -= me[a, b]
                B[i, j] -= ke[a, b]
        return A, B
    monkeypatch.setattr(fem, "assemble_1d", bad)
    monkeypatch.setattr("oracle.spectral.assemble_1d", bad)
    with pytest.raises(AssertionError):
        periodic_pins.test_periodic_step_matches_the_dft_route((16, 12), 2)


def test_flory_huggins_log_sign_error_is_caught(monkeypatch):
    monkeypatch.setattr(etd, "flory_huggins", lambda th, thc: (
        lambda t, u: 0.5 * th * np.log((1.0 + u) / (1.0 - u)) + thc * u))
    with pytest.raises(AssertionError):
        periodic_pins.test_periodic_eigen_path_matches_dense_expm((4, 5), (0.25, 0.2), 1, "flory_huggins")


# ---------------------------------------------------------------- nonhomogeneous Dirichlet data
import test_oracle_boundary as boundary_pins
from oracle import boundary as obnd


def _planted_source(monkeypatch, drop_gdot=False, flip_k=False):
    orig = obnd.boundary_source

    def bad(N, h, D, f, data):
        def data2(t):
            g, gd = data(t)
            return g, (0 * gd if drop_gdot else gd)
        src = orig(N, h, -D if flip_k else D, f, data2)   # flipping D flips the K_IB g term only
        return src
    monkeypatch.setattr(obnd, "boundary_source", bad)


def test_boundary_pins_pass_unmutated():
    boundary_pins.test_example52_converges_to_the_semidiscrete_solution(2, 2.0)


def test_dropped_boundary_time_derivative_is_caught(monkeypatch):
    _planted_source(monkeypatch, drop_gdot=True)
    with pytest.raises(AssertionError):
        boundary_pins.test_example52_converges_to_the_semidiscrete_solution(2, 2.0)


def test_boundary_stiffness_sign_error_is_caught(monkeypatch):
    _planted_source(monkeypatch, flip_k=True)
    with pytest.raises(AssertionError):
        boundary_pins.test_linear_field_is_a_discrete_steady_state((6, 5), (1 / 6, 0.2), 2)
