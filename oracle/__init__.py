"""CPU oracle for RAMBO (arXiv 1910.02611).

TEST INFRASTRUCTURE ONLY.  Imported by the tests, the smoke check and the
benchmark's CPU-baseline leg; never by the GPU library or its binding.

- ``rambo_oracle.c`` / ``oracle.py``: plain RAMBO on B*R separate Bloom filters,
  Algorithm 1 and Algorithm 2 step by step (Secs. 2, 3.1, 3.2, 3.2.1).
- ``brute.py``: exact multiple-set-membership answers and the "exact cell"
  RAMBO answer by brute force over Python sets, for tiny inputs.
"""
