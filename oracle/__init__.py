"""Oracles for the windowed Fourier projection (WFP) method — TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference legs of
`bench.py` may import anything here.  The CUDA library never imports, links or runs
these files, and they share no code with it; both sides only read inputs drawn by
`paper_2507_07823_gb300.workloads`.

* `volterra` (Oracle A): direct all-to-all march of the Volterra system (eq. IEfree /
  eq. periodicIE) with exact integrals of p-point interpolants.  It is the "truth"
  the windowed scheme approximates and is pinned by closed forms in `tests/`.
* `wfp` (Oracle B): the paper's discrete WFP scheme (eq. periodicIE_disc and Sec. 4.4)
  written step by step with direct Fourier sums, a plain sparse matrix for the local
  part and a direct sparse solve.  The CUDA path is compared against it element by
  element.
* `adjoint`: the reverse-time transposed march of Oracle B's scheme, giving the gradient of
  a receiver misfit with respect to the stiffnesses (and to a host forcing); pinned by
  central differences of Oracle B and by the complex-step derivative of Oracle A (its
  complex build, `volterra.march_complex_step`).
"""
