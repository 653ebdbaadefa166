"""Oracle: a plain, slow FP64 CPU implementation of the free-space Spectral Ewald
method for stokeslet, stresslet and rotlet sums.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only users.
The product path (the CUDA library and its Python binding) never imports,
links or runs anything here, and this package never imports the product.

  * ``direct``  O1: the FP64 direct O(N^2) sums and their gradients (ground truth).
  * ``se``      O2: the paper's algorithm step by step in FP64 (CPU).
  * ``periodic`` O3: the triply periodic sums by plain Ewald summation (FP64).
  * ``greens``  closed forms: (truncated) harmonic and biharmonic transforms,
                screening functions, self-interaction limit.
  * ``params``  the truncation-error estimates of Tables 2 and 3.
"""
