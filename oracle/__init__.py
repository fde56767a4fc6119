"""Plain, slow, FP64 CPU oracle for the discrete Fourier integral operator (FIO) problem.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import it. The product (the CUDA path, its C ABI
and the host factor builder) never imports it, and it imports nothing from the product.

Modules
-------
fio_oracle    The operator K by its definition (grids, phase, dense matrix, matrix-free rows),
              K f, K* u, the dense LU solve of u = K f, CG on the normal equations, and a
              Gauss-Jordan brute force for tiny cases.  Paper section 1 (eq. 1.3-1.6) and the
              workloads of section 6 (Examples 1 and 3).
factor_apply  Reads a packed factor buffer byte by byte and applies the butterfly product
              (section 2, eq. for K-dot and its adjoint) and the inverse-factor product
              G-dot = R_L ... R_1 A_0^{-1} R_1^* ... R_L^* (section 4, eqs. for G-dot in 1D
              and 2D) as plain sparse-matrix products, one factor at a time.

Parity status of each function is stated in its module header.
"""
