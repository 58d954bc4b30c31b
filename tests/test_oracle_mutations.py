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
