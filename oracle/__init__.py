"""FP64 CPU oracle for stratified Monte Carlo with heuristic tree search.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call or build anything in this
package.  The product path (``paper_1902_07916_gb300``) never touches it and
the two share no code.

Modules:
  sampler.c      -- Philox4x32-10 stream, integrands, per-(cell, trial) sums
  zmc_oracle.py  -- the tree search, step by step (Sec. 2.1, Fig. 1)
  closed_forms.py-- analytic integrals of the registry integrands
  build.py       -- compiles sampler.c with gcc
"""
