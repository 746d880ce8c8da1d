"""Plain FP64 CPU oracle for the Duo & Zhang finite-difference fractional Laplacian.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this package;
only the tests, `__graft_entry__.smoke()` and the CPU-baseline legs of `bench.py`
use it.  It shares no code with the CUDA path: its quadrature, coefficient
assembly, dense operator, FFT embedding (SciPy pocketfft) and solvers are written
here from the paper, independently of the GPU kernels.

Modules
-------
scheme   -- c_{d,alpha}, element weights, far field, the coefficients a_k
            (Sec. 2 eqs. amn/a00, Sec. 4 a_mns/a000), the dense matrix
            (eqs. A-2D/A-3D) and the literal element-by-element evaluation
            (eqs. I0L-2D / eq-3D1).
fast     -- the same operator applied through a circulant embedding with SciPy FFTs
            (the "FFT-based fast algorithm" the paper asserts after eq. A-2D),
            validated against the dense matrix.
solvers  -- plain conjugate gradients, the semi-implicit Allen-Cahn step, the
            multilevel Strang circulant preconditioner.
netprecond -- FP64 forward/backward of the per-frequency MLP preconditioner
            (parity unpinned by the paper; pinned by finite differences).

Every function cites the passage of the paper it follows.  Readings of the paper
where it is silent or garbled are stated where they are used.
"""
