"""FP64 CPU oracle for the NPGA hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously correct NumPy restatement of what
the method computes.  It exists to check the CUDA path and is not part of
the product: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  It shares no code with the CUDA
path (no kernels, helpers, tables or constants); both sides take their
inputs from the ``synth`` module, which draws random numbers only.

Modules and the parts of the paper they restate:

* ``center``     -- sample mean and centered factor L (Sec. 2.1).
* ``projection`` -- simplex projection by sorting (Eqs. simplex-tau /
  simplex-proj), halfspace projection (Eq. proj-halfspace) and the exact
  projection onto F by the scalar dual search of Eq. projF-dualpath, finished
  exactly on the identified support.
* ``npga``       -- unified objective/gradient (Eq. npga-unified-grad), the
  power method for ||L_eff||_2 (Sec. 3.1 remark), Algorithm 1 (NPGA) with the
  fixed step, the KKT stopping residual (Sec. 3.1, stopping condition), the
  Frank--Wolfe gap certificate and the solver gap metric of Sec. 5.2.
* ``strmodel``   -- Sketch--Truncate--Ridge (Sec. 2.5, App. D.3).
* ``bruteforce`` -- exhaustive active-set enumeration for n <= 10 and the
  vertex list of F, used to pin the functions above.
* ``adjoint``    -- reverse-mode derivative of the unrolled NPGA solve.

Precision is FP64 throughout unless a function says otherwise.
"""
