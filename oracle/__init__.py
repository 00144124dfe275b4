"""FP64 CPU oracle for the Black-Scholes Parareal path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library: every
formula here is written out from the paper (Ibrahim, Goetschel, Ruprecht,
"Space-time parallel scaling of Parareal with a physics-informed Fourier Neural
Operator coarse propagator applied to the Black-Scholes equation", PASC'25).

Modules
  closed_forms  Margrabe, one-asset Black-Scholes, cash-or-nothing (Sec. 3.2)
  fd            eq. (fd) assembled as a sparse matrix, implicit Euler by sparse LU
  parareal      textbook Parareal, eq. (parareal), with the defect norm
  fno           FP64 FNO / PINO forward (Sec. 3.4, 3.5)
  resample      bilinear resampling; the numerical coarse model on a coarser grid (Sec. 4.4)
  fd_nd         eq. (bse_general) for n assets discretised like eq. (fd) (19-point stencil
                at n = 3), implicit Euler by sparse LU
  physics       the PDE term of the PINO training loss (Sec. 3.5, eq. bs_totalloss) and its
                gradient

Pinning: every function is checked by ``tests/test_oracle_*.py`` against facts
the mathematics fixes (exactness of centred differences on x^a y^b, a, b <= 2,
closed forms, Parareal invariants, brute force on tiny grids, numpy.fft).
"""
