"""CPU oracle for the Heisenberg-picture PEPO method (test infrastructure only).

This package is the slow, literal, complex128 reference that the CUDA path is
checked against.  It is *test infrastructure*: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path (the ``libpepo`` CUDA
library and its Python binding) never imports, links or calls anything here,
and this package imports nothing from the product.

Representation (deliberately different from the GPU path):
  * every site tensor carries its physical leg as a literal 2x2 operator pair
    ``[..., s, s']`` in complex128 (the GPU stores real Pauli coefficients);
  * gates act by literal conjugation ``g^dagger O g`` with the 2x2 / 4x4
    unitaries (the GPU uses real Pauli transfer matrices);
  * the bond update is the gauge change, QR reduction, gate, truncated SVD
    and inverse gauge change of Sec. 2.5 "Gate Update" (Eqs. 11-12), each
    written with plain numpy calls and no fusion.

Modules
  lattice   geometry and the four-colour bond partition (Sec. 2.3)
  gates     unitaries and the Trotter schedule (Eq. 6 / Sec. 2.3)
  dense     brute-force 2^N x 2^N operator evolution (Eq. 3-5)
  pepo      the operator network and the bond update (Sec. 2.5, Alg. 1)
  bp        double- and single-layer belief propagation, Bethe value
            (Eq. 13, 14, 7, 8, 9, 15)
  contract  exact contraction of small networks (Sec. 2.6 step 1)
  run       the time loop (Fig. 1 pipeline)

Parity status of each function is stated in its module header.
"""
