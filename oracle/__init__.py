"""CPU oracle for the kernel-compensated Yee Maxwell operator and its
eigensolver (test infrastructure only).

Plain, slow, FP64 numpy code written from the paper, used to prove the CUDA
library right.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import it; the library never does, and the
oracle never imports the library.  The only code the two sides share is the
seeded input description in ``workloads``, which holds none of the method's
arithmetic.

Modules
-------
stencils      finite-difference coefficients and circulant first rows
              (Sec. 2.1 eq. yee:D0D1; Sec. 2.5 eqs. kc:highord:stencil,
              kc:high:coef, Table tab:kc:fd1d)
yee           real-space Yee operators A, A^H, B, B^H and the compensated
              operator A M A^H + gamma B^H B (Sec. 2.1-2.3)
permittivity  staggered sampling of a structure and the per-cell discrete
              inverse permittivity M_Trivial (Sec. 2.1, Sec. 3.1-3.2.1)
crossdof      M_CrossDoF, the symmetrised cross-DoF transfer form of the
              discrete inverse permittivity (Sec. 3.2.2)
fourier       DFT matrix, circulant symbols, Fourier-basis operator and the
              FFT-diagonal preconditioner (Lemma 2.1, Prop. 2.8, Sec. 2.4)
penalty       the penalty-coefficient rules (Prop. 2.5, Remark 2.6)
eig           dense spectra, homogeneous-medium spectra, textbook LOBPCG
              (Sec. 4)
learned       the gated 3D convolution correction of K_P^{-1} (no counterpart
              in the paper): forward pass, loss gradient by the chain rule,
              the corrected preconditioner T(r) and its training pairs

Every function that has no independent pin says "parity unpinned" in its
docstring.  At present every function, and every shape branch of the
staggered sampling (sphere, rod, box, gyroid), is pinned by a test in
``tests/test_oracle_*.py`` that a planted slip fails
(``tests/test_oracle_mutations.py``).
"""
