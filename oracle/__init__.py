"""CPU oracle for the exponential-integrator Q1 finite-element method (EIFE1 / EIFE2).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call, link or execute this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference arm of
``bench.py`` use it. It shares no code with the CUDA library (no kernels, headers, tables or
constant generators); both sides receive the same seeded inputs from
``paper_2209_11922_gb300.inputs``, which holds none of the method's arithmetic.

Everything is FP64 NumPy/SciPy, written for readability, not speed:

* ``fem``      Q1 element integrals and assembly of the 1D matrices A, B and the global M, K
               (Section 2.1, eq. (2.5); Section 4, eq. (4.1)).
* ``spectral`` simultaneous diagonalisation of A and B by an orthogonal matrix (Section 4), done
               numerically with a library symmetric eigensolver, not with the closed form.
* ``phi``      the phi-functions of Section 2.2 by Gauss-Legendre quadrature of their defining
               integral (|z| <= 1) and by the recurrence phi_{k+1} = (phi_k - 1/k!)/z otherwise.
* ``etd``      the EIFE1 step, eq. (2.13), and the EIFE2 step, eq. (2.14), in the spectral form of
               eqs. (4.2)-(4.4), with dense per-axis products (tensor mode products of Section 4).
* ``monitors`` mass 1^T M U, the discrete energy, max|u|.
* ``transforms`` the orthonormal DST-I of one axis from its definition (kernel-level parity).
* ``boundary`` nonhomogeneous Dirichlet data as a time-dependent part of f (Section 4).
* ``sno``      the spectral neural operator used as the learned coarse propagator (forward pass,
               its chain-rule gradient, Adam) and the Parareal iteration.

Readings of the paper taken here:

* the sine eigenvector matrix is used in its orthonormal form S = sqrt(2/N) P (Section 4 calls P
  orthogonal, but P P^T = (N/2) I);
* the reaction tensor F has entries from nodal values of f, i.e. F = M f(U) (group finite
  element reading of Section 4), so the spectral ODE is dU~/dt = -H (.) U~ + S f(S U~);
* c2 = 1/2 in EIFE2 (Section 5);
* u(0) is the given nodal field (the P_h u0 of eq. (2.5) is replaced by nodal data);
* periodic boundary conditions (Section 4, closing remarks): the printed eigenvalue formulas are
  garbled; the eigenvalues are those of the circulant A = (h/6) circ(4, 1, .., 1) and
  B = (1/h) G^P, lambda^A_i = (h/3)(2 + cos theta_i), lambda^B_i = (2/h)(1 - cos theta_i),
  theta_i = 2 pi (i - 1)/N, pinned by the tests; the oracle itself diagonalises numerically;
* Example 5.3's energy: the potential integral by nodal (lumped) quadrature.

Parity status of each function is stated in its docstring; functions without an independent pin
say "parity unpinned".
"""
from . import fem, spectral, phi, etd, monitors, transforms, sno, boundary  # noqa: F401
