"""FP64 CPU oracle for extended diffraction tomography (test infrastructure only).

This package is the plain, slow, obviously correct statement of what the GPU library
computes.  It exists to check the CUDA path and is imported only by the tests, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the library itself
never imports it and shares no code with it.

Contents (each function cites the part of the paper it follows):

* :mod:`oracle.green`  the 1D reference Green's function of a layered medium
  (the Green's-function equation of Section "Two dimensions" after a lateral Fourier
  transform; the paper does not say how to compute it in layers, the reading used is a
  stable reflectivity recursion).
* :mod:`oracle.edt2d`  the decoupled 2D method: data transform (Fourier transform over
  midpoint/offset, written on a periodic shot/receiver grid), the per-wavenumber kernel M
  (eq. M with the aperture sinc reduced to a delta), the Hermitian split (eq. Split), the
  damped least-squares solve by Householder QR, Hermitian completion (eq. VSym) and the
  inverse transform; plus the spectral Born forward model and its adjoint.
* :mod:`oracle.edt3d`  the finite-aperture / 3D geometry (Section "A practical 3D
  geometry" with the aperture sinc of eq. M kept as the window's Dirichlet kernel):
  midpoint and half-offset-window transforms, the kernel K(k_m, w, z) of every recorded
  half-offset, the split per pair {k_m, -k_m}, the same damped QR solve, forward model and
  adjoint.
* :mod:`oracle.brute`  independent brute-force references used only to pin the above:
  space-domain Born summation (eq. Born) and a finite-difference solve of the 1D
  Green's-function equation.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``.  The end-to-end
inversion cannot be pinned against printed numbers because the paper prints none (its
figures are absent); it is pinned by noise-free recovery, optimality and adjoint tests.
"""
