"""CPU FP64 oracle for the low-scaling GW polarizability and self-energy.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
links anything in this package: only the tests, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA library (no kernels, headers, helpers or
constants); the two meet only at the seeded inputs of ``synth``.

Every routine is a plain, slow, numpy FP64 statement of one equation of the
paper (arXiv 2104.09857), cited in its docstring.  numpy's matmul/einsum serve
as library primitives; there is no blocking, fusion or reordering beyond what
the cited equation states.

Modules
  chi    Eq. 2 (Green's functions), Eq. 3 (polarizability) with the block
         filter of the Computational Methods section; MO-route identity;
         brute-force loops; per-block evaluation for large systems.
"""
