"""CPU oracle for batched affine elliptic-curve arithmetic (gECC, arXiv 2501.03245).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle is the plain mathematical definition of every result the GPU path
produces, written with Python integers (``%``, ``pow``) and, for the timed CPU
baseline, a separate plain C++ big-integer implementation (``oracle/cpp``).  It
shares no code, constants or helpers with the CUDA path.

Modules
  curves   curve parameters (short Weierstrass, Eqn 1) and their derivations
  ec       affine group law (Eqn 2-3 and the PDBL slope, Section 2.1.1),
           double-and-add (Algorithm 1), naive multi-scalar multiplication
  field    modular multiplication / Montgomery's trick batch inversion
           (Section 2.2, Algorithm 2, Section 2.2.1)
  ecdsa    ECDSA signing and verification (standard SEC 1 / FIPS 186-4 equations;
           the paper only says verification is one FPMUL plus one UPMUL)
  tiny     brute-force enumeration of small prime-field curves
  cpp      plain C++ bigint oracle (Barrett reduction, Jacobian coordinates),
           loaded through ctypes; the timed CPU baseline

Parity status of every function is recorded in its module docstring.
"""
