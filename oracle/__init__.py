"""FP64 CPU oracle of the periodized DMK method (test infrastructure only).

This package is a plain, slow, deliberately unoptimised restatement of what the
method computes, written from the paper "Fast summation on rectangular cuboids
with arbitrary periodicity in the DMK framework" (Krantz, af Klinteberg,
Tornberg). Every function cites the section or equation it follows.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never imports, links or calls
anything here, and nothing here imports the CUDA library: the two share no code.

Modules
-------
pswf      zeroth-order prolate window phi, Phi, phi-hat (Sec. 2.2, Remark PSWF_eval)
params    per-tolerance parameters and plan rules (Sec. 6.1, Tables 1 and 5)
symbols   truncated Green's-function symbols and kernel symbols (Sec. 5.2, App. B-D)
kernels   residual kernels, difference-kernel symbols, self terms (Sec. 2, App. B)
tree      forest of octrees, 2:1 balance, interaction recursion (Sec. 3.1.1, 4.1)
dmk       the evaluation: upward, root far field, downward, leaf (Sec. 3.1, 4.2-4.3, 5.3)
ewald     independent Ewald-type references on tiny inputs (Sec. 1, Eq. ewald-split): Laplace,
          every D; the Stokeslet, D = 1-3, by Hasimoto's split of the Oseen tensor

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
values fixed by the paper or by mathematics; none is "parity unpinned" except
where its own docstring says so.
"""
